// Rotations (Fig. 1 item 11, Rot) of ciphertexts of several rings, ring degrees and levels in one
// call: each stage of the hybrid key switch runs as one launch over every ciphertext, whatever its
// ring (the automorphism of c1, ModUp's inverse NTT, conversion and NTT, the key inner product,
// ModDown's inverse NTT, conversion and NTT, and the epilogue with sigma_g(c0)).  The arithmetic
// of every stage is that of the one-ring rotation (Eval::rotate), so each result equals the
// rotation alone.
#include <algorithm>
#include <cstring>

#include "launch_util.cuh"
#include "host_math.h"
#include "runtime.h"

namespace hx {

namespace {

// a job table of each kind packed into one host buffer (256-byte aligned parts), copied once
struct Tables {
    std::vector<unsigned char> host;
    template <class J> size_t add(const std::vector<J> &v)
    {
        const size_t off = (host.size() + 255) & ~size_t(255);
        host.resize(off + v.size() * sizeof(J));
        if (!v.empty()) std::memcpy(host.data() + off, v.data(), v.size() * sizeof(J));
        return off;
    }
};

NttJob ntt_job(const hx_context &ctx, uint64_t *data, int rows, const std::vector<int> &primes)
{
    NttJob j{};
    j.data = data;
    j.primes = ctx.t.primes;
    j.tw_fwd = ctx.t.tw_fwd;
    j.tw_inv = ctx.t.tw_inv;
    j.log_n = ctx.log_n;
    j.n_rows = rows;
    j.n_limbs = (int)primes.size();
    for (size_t i = 0; i < primes.size(); i++) j.prime[i] = (int16_t)primes[i];
    return j;
}

} // namespace

std::vector<Cts> rotate_jobs(const std::vector<RotateJob> &in, cudaStream_t s)
{
    struct Work {
        hx_context *ctx;
        const Cts *a;
        uint64_t g;
        const SwitchKey *key;
        int N, L, K, A, nd, ext, B;
        BufPtr t, coef, D, acc, conv;
        Cts out;
    };
    std::vector<Cts> out(in.size());
    std::vector<Work> w;
    std::vector<size_t> w_of;
    // every check and key lookup before any device work
    int dev = -1;
    for (size_t i = 0; i < in.size(); i++) {
        const RotateJob &J = in[i];
        HX_CHECK(J.ctx && J.ks && J.a.d && J.a.comps == 2 && J.a.B >= 1 && J.a.limbs >= 1, HX_EINVAL,
                 "a rotation job needs a ciphertext, its context and its keys");
        HX_CHECK(dev < 0 || J.ctx->device == dev, HX_EINVAL, "jobs on several devices");
        dev = J.ctx->device;
        hx_context &ctx = *J.ctx;
        const uint64_t g = galois_for_step(J.step, ctx.log_n);
        if (g == 1) continue;  // the identity: a copy, below
        HX_CHECK(ctx.log_n >= 11 && ctx.log_n <= 16, HX_EINVAL, "ring degree outside 2^11..2^16");
        Eval ev(ctx, s);
        Work x{};
        x.ctx = &ctx;
        x.a = &J.a;
        x.g = g;
        x.key = &ev.rot_key(*J.ks, g);
        x.N = ctx.N;
        x.L = J.a.limbs;
        x.K = ctx.K;
        x.A = ctx.alpha;
        x.nd = (x.L + x.A - 1) / x.A;
        x.ext = x.L + x.K;
        x.B = J.a.B;
        HX_CHECK(x.ext <= 64, HX_EINVAL, "too many limbs for a several-ring transform");
        w.push_back(std::move(x));
        w_of.push_back(i);
    }
    for (size_t i = 0; i < in.size(); i++)
        if (galois_for_step(in[i].step, in[i].ctx->log_n) == 1) out[i] = Eval(*in[i].ctx, s).copy(in[i].a);
    if (w.empty()) return out;

    // buffers and job tables
    std::vector<AutomorphismJob> aj;
    std::vector<NttJob> n1, n2, n3, n4;
    std::vector<ConvertJob> c1, c2;
    std::vector<KeyIpJob> kj;
    std::vector<ModDownJob> mj;
    int max_a = 1, max_k = 1;
    for (Work &x : w) {
        hx_context &ctx = *x.ctx;
        const size_t N = x.N;
        const int L = x.L, K = x.K, ext = x.ext, nd = x.nd, B = x.B;
        x.t = std::make_shared<DevBuf>((size_t)B * L * N, s);
        x.coef = std::make_shared<DevBuf>((size_t)B * L * N, s);
        x.D = std::make_shared<DevBuf>((size_t)B * nd * ext * N, s);
        x.acc = std::make_shared<DevBuf>((size_t)B * 2 * ext * N, s);
        x.conv = std::make_shared<DevBuf>((size_t)B * 2 * L * N, s);
        x.out = Eval(ctx, s).alloc(B, 2, L);
        x.out.scale = x.a->scale;
        max_a = std::max(max_a, x.A);
        max_k = std::max(max_k, K);
        const View tv{x.t->p, (size_t)L * N, (size_t)L * N};
        const View c1v{x.a->d + x.a->cstride(N), x.a->bstride(N), x.a->cstride(N)};
        const View accv{x.acc->p, (size_t)2 * ext * N, (size_t)ext * N};
        // sigma_g(c1)
        aj.push_back(AutomorphismJob{tv, c1v, x.g, 1, ctx.log_n, ctx.t.primes, ew_blocks((int)N, 1), L, B, 0});
        // ModUp: inverse NTT of a copy, conversion of every digit, forward NTT of the extended rows
        std::vector<int> q_rows(L), ext_primes(ext), p_rows(K);
        for (int r = 0; r < L; r++) q_rows[r] = r;
        for (int r = 0; r < ext; r++) ext_primes[r] = r < L ? r : ctx.n_q + (r - L);
        for (int r = 0; r < K; r++) p_rows[r] = ctx.n_q + r;
        n1.push_back(ntt_job(ctx, x.coef->p, B * L, q_rows));
        c1.push_back(ConvertJob{ctx.t.modup + (size_t)L * ctx.dnum, View{x.D->p, (size_t)nd * ext * N, 0},
                                View{x.coef->p, (size_t)L * N, 0}, ctx.t.primes, nd, (int)N, x.A, (size_t)ext * N, 0,
                                ew_blocks((int)N, 2), 1, B * nd, 0});
        // a digit's own rows of D are never read (the inner product takes them from sigma_g(c1))
        n2.push_back(ntt_job(ctx, x.D->p, B * nd * ext, ext_primes));
        kj.push_back(KeyIpJob{accv, x.D->p, x.t->p, x.key->buf->p, (size_t)L * N, ctx.t.primes, ctx.n_all, ctx.n_q,
                              K, x.A, L, nd, ctx.log_n, nd <= kRedcFewTerms ? 1 : 0, 1, ew_blocks((int)N, 2), ext, B,
                              0});
        // ModDown: inverse NTT of the special rows, conversion to Q, forward NTT, epilogue
        for (int b = 0; b < B; b++)
            for (int c = 0; c < 2; c++)
                n3.push_back(ntt_job(ctx, x.acc->p + ((size_t)(b * 2 + c) * ext + L) * N, K, p_rows));
        const ModDownTable *md = ctx.t.moddown + L;
        c2.push_back(ConvertJob{reinterpret_cast<const ConvTable *>(md), View{x.conv->p, (size_t)L * N, 0},
                                View{x.acc->p, (size_t)ext * N, 0}, ctx.t.primes, 1, (int)N, K, 0, 0,
                                ew_blocks((int)N, 2), 1, 2 * B, 0});
        n4.push_back(ntt_job(ctx, x.conv->p, 2 * B * L, q_rows));
        mj.push_back(ModDownJob{x.out.view((int)N), accv, View{x.conv->p, (size_t)2 * L * N, (size_t)L * N},
                                x.a->view((int)N), md, ctx.t.primes, 1, ctx.log_n, x.g, ew_blocks((int)N, 2), L,
                                2 * B, 0});
    }
    const long long ba = plan_job_blocks(aj), bc1 = plan_job_blocks(c1), bk = plan_job_blocks(kj),
                    bc2 = plan_job_blocks(c2), bm = plan_job_blocks(mj);
    int t1c, t1r, t2c, t2r, t3c, t3r, t4c, t4r;
    plan_ntt_jobs(n1, &t1c, &t1r);
    plan_ntt_jobs(n2, &t2c, &t2r);
    plan_ntt_jobs(n3, &t3c, &t3r);
    plan_ntt_jobs(n4, &t4c, &t4r);
    Tables tb;
    const size_t oa = tb.add(aj), o1 = tb.add(n1), oc1 = tb.add(c1), o2 = tb.add(n2), ok = tb.add(kj),
                 o3 = tb.add(n3), oc2 = tb.add(c2), o4 = tb.add(n4), om = tb.add(mj);
    DevBuf dev_tables((tb.host.size() + 7) / 8, s);
    unsigned char *d = reinterpret_cast<unsigned char *>(dev_tables.p);
    HX_CUDA(cudaMemcpyAsync(d, tb.host.data(), tb.host.size(), cudaMemcpyHostToDevice, s));
    hx_context &c0 = *w[0].ctx;
    std::atomic<uint64_t> *launches = &c0.counters[C_LAUNCH];
    const int n_sm = c0.t.n_sm;

    launch_automorphism_jobs(s, reinterpret_cast<const AutomorphismJob *>(d + oa), (int)aj.size(), ba, launches);
    for (Work &x : w)
        HX_CUDA(cudaMemcpyAsync(x.coef->p, x.t->p, sizeof(uint64_t) * x.B * x.L * x.N, cudaMemcpyDeviceToDevice, s));
    launch_ntt_jobs(s, reinterpret_cast<const NttJob *>(d + o1), (int)n1.size(), t1c, t1r, true, n_sm, launches);
    launch_convert_jobs(s, reinterpret_cast<const ConvertJob *>(d + oc1), (int)c1.size(), bc1, max_a, launches);
    launch_ntt_jobs(s, reinterpret_cast<const NttJob *>(d + o2), (int)n2.size(), t2c, t2r, false, n_sm, launches);
    launch_key_ip_jobs(s, reinterpret_cast<const KeyIpJob *>(d + ok), (int)kj.size(), bk, launches);
    launch_ntt_jobs(s, reinterpret_cast<const NttJob *>(d + o3), (int)n3.size(), t3c, t3r, true, n_sm, launches);
    launch_convert_jobs(s, reinterpret_cast<const ConvertJob *>(d + oc2), (int)c2.size(), bc2, max_k, launches);
    launch_ntt_jobs(s, reinterpret_cast<const NttJob *>(d + o4), (int)n4.size(), t4c, t4r, false, n_sm, launches);
    launch_moddown_jobs(s, reinterpret_cast<const ModDownJob *>(d + om), (int)mj.size(), bm, launches);

    for (size_t k = 0; k < w.size(); k++) {
        hx_context &ctx = *w[k].ctx;
        ctx.counters[C_ROT] += w[k].B;
        ctx.counters[C_KS] += w[k].B;
        ctx.counters[C_MODUP] += w[k].B;
        out[w_of[k]] = w[k].out;
    }
    return out;  // the work buffers and the tables go back to the pool in the stream's order
}

} // namespace hx
