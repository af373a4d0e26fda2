// Key generation, encryption and collective decryption (Fig. 1 items 1-6) at
// toy scale: the parties are simulated in this process; their randomness is
// drawn on the host from SplitMix64 streams and the ring arithmetic runs on
// the device with the evaluation kernels.
#include <cstring>

#include "runtime.h"

namespace hx {

namespace {

std::vector<int> iota_vec(int a, int n)
{
    std::vector<int> v(n);
    for (int i = 0; i < n; i++) v[i] = a + i;
    return v;
}

// signed coefficients (host) -> NTT-form residues over primes 0..rows-1 (device)
void signed_polys_to_ntt(hx_context &ctx, cudaStream_t s, const std::vector<int64_t> &host, int n_polys, int rows,
                         uint64_t *dst)
{
    Eval ev(ctx, s);
    DevBuf tmp((size_t)n_polys * ctx.N, s);
    HX_CUDA(cudaMemcpyAsync(tmp.p, host.data(), sizeof(int64_t) * host.size(), cudaMemcpyHostToDevice, s));
    launch_signed_to_rows(ev.lc(), dst, reinterpret_cast<const int64_t *>(tmp.p), rows, n_polys, ctx.N,
                          ctx.d_prime_ids);
    ev.ntt_inplace(dst, (size_t)rows * ctx.N, n_polys, iota_vec(0, rows), iota_vec(0, rows), false);
    HX_CUDA(cudaStreamSynchronize(s));
}

void gen_switch_key(hx_context &ctx, hx_keyset &ks, uint64_t key_id, const uint64_t *sp, SwitchKey &out,
                    cudaStream_t s)
{
    const int N = ctx.N, n_all = ctx.n_all, n_q = ctx.n_q, K = ctx.K;
    Eval ev(ctx, s);
    out.buf = std::make_shared<DevBuf>((size_t)ctx.dnum * 2 * n_all * N, s);
    std::vector<uint64_t> a((size_t)n_all * N);
    std::vector<int64_t> e(N);
    std::vector<uint64_t> gad(n_all);
    DevBuf e_ntt((size_t)n_all * N, s);
    DevBuf gad_d(n_all, s);
    uint64_t P_mod[64];
    for (int i = 0; i < n_q; i++) {
        uint64_t v = 1;
        for (int k = 0; k < K; k++) v = hmul(v, ctx.primes[n_q + k] % ctx.primes[i], ctx.primes[i]);
        P_mod[i] = v;
    }
    for (int j = 0; j < ctx.dnum; j++) {
        Stream sa(ks.seed, P_KEY_A, key_id, j);
        for (int r = 0; r < n_all; r++) sample_uniform(sa, ctx.primes[r], a.data() + (size_t)r * N, N);
        Stream se(ks.seed, P_KEY_E, key_id, j);
        for (int i = 0; i < N; i++) e[i] = ctx.cdt->draw(se);
        for (int r = 0; r < n_all; r++) gad[r] = (r >= j * K && r < std::min((j + 1) * K, n_q)) ? P_mod[r] : 0;
        uint64_t *bj = out.buf->p + (size_t)(2 * j) * n_all * N;
        uint64_t *aj = bj + (size_t)n_all * N;
        HX_CUDA(cudaMemcpyAsync(aj, a.data(), sizeof(uint64_t) * a.size(), cudaMemcpyHostToDevice, s));
        HX_CUDA(cudaMemcpyAsync(gad_d.p, gad.data(), sizeof(uint64_t) * n_all, cudaMemcpyHostToDevice, s));
        signed_polys_to_ntt(ctx, s, e, 1, n_all, e_ntt.p);
        launch_keygen_b(ev.lc(), bj, aj, e_ntt.p, ks.s_ntt->p, sp, gad_d.p, n_all, nullptr, true);
        HX_CUDA(cudaStreamSynchronize(s));  // host staging vectors are reused
    }
}

} // namespace

void keygen(hx_context &ctx, hx_keyset &ks, int n_parties, uint64_t seed, cudaStream_t s)
{
    HX_CHECK(n_parties >= 1 && n_parties <= 64, HX_EINVAL, "n_parties must be in [1, 64]");
    const int N = ctx.N, n_all = ctx.n_all, n_q = ctx.n_q;
    Eval ev(ctx, s);
    ks.ctx = &ctx;
    ks.n_parties = n_parties;
    ks.seed = seed;
    ks.s.assign(N, 0);
    for (int p = 0; p < n_parties; p++) {
        std::vector<int64_t> sp(N);
        Stream st(seed, P_SK, p, 0);
        sample_ternary(st, sp.data(), N);
        for (int i = 0; i < N; i++) ks.s[i] += sp[i];
        ks.s_parts.push_back(sp);
    }
    ks.s_ntt = std::make_shared<DevBuf>((size_t)n_all * N, s);
    signed_polys_to_ntt(ctx, s, ks.s, 1, n_all, ks.s_ntt->p);
    ks.s_parts0 = std::make_shared<DevBuf>((size_t)n_parties * N, s);
    std::vector<int64_t> flat;
    for (auto &v : ks.s_parts) flat.insert(flat.end(), v.begin(), v.end());
    signed_polys_to_ntt(ctx, s, flat, n_parties, 1, ks.s_parts0->p);
    // collective public key (b, a) = (-a s + e, a) over Q
    ks.pk = std::make_shared<DevBuf>((size_t)2 * n_q * N, s);
    std::vector<uint64_t> a((size_t)n_q * N);
    Stream sa(seed, P_PK_A, 0, 0);
    for (int r = 0; r < n_q; r++) sample_uniform(sa, ctx.primes[r], a.data() + (size_t)r * N, N);
    std::vector<int64_t> e(N);
    Stream se(seed, P_PK_E, 0, 0);
    for (int i = 0; i < N; i++) e[i] = ctx.cdt->draw(se);
    DevBuf e_ntt((size_t)n_q * N, s);
    signed_polys_to_ntt(ctx, s, e, 1, n_q, e_ntt.p);
    uint64_t *pa = ks.pk->p + (size_t)n_q * N;
    HX_CUDA(cudaMemcpyAsync(pa, a.data(), sizeof(uint64_t) * a.size(), cudaMemcpyHostToDevice, s));
    launch_keygen_b(ev.lc(), ks.pk->p, pa, e_ntt.p, ks.s_ntt->p, nullptr, nullptr, n_q, nullptr, false);
    // relinearisation key: s' = s^2
    DevBuf s2((size_t)n_all * N, s);
    launch_mul_rows(ev.lc(), s2.p, ks.s_ntt->p, ks.s_ntt->p, n_all);
    gen_switch_key(ctx, ks, 0, s2.p, ks.relin, s);
    HX_CUDA(cudaStreamSynchronize(s));
}

void add_rotation_keys(hx_context &ctx, hx_keyset &ks, const std::vector<int64_t> &steps, cudaStream_t s)
{
    Eval ev(ctx, s);
    const size_t N = ctx.N;
    DevBuf sg((size_t)ctx.n_all * N, s);
    for (int64_t k : steps) {
        const uint64_t g = galois_for_step(k, ctx.log_n);
        if (g == 1 || ks.rot.count(g)) continue;
        launch_automorphism(ev.lc(), View{sg.p, 0, 0}, View{ks.s_ntt->p, 0, 0}, g, 1, 1, ctx.n_all);
        SwitchKey key;
        gen_switch_key(ctx, ks, g, sg.p, key, s);
        ks.rot[g] = key;
    }
    HX_CUDA(cudaStreamSynchronize(s));
}

Cts encrypt_coeffs(hx_context &ctx, const hx_keyset &ks, const int64_t *m, double scale, int limbs, uint64_t seed,
                   uint32_t tag, uint32_t index, cudaStream_t s)
{
    HX_CHECK(limbs >= 1 && limbs <= ctx.n_q, HX_EINVAL, "bad level");
    const int N = ctx.N;
    Eval ev(ctx, s);
    std::vector<int64_t> host((size_t)4 * N);
    Stream sv(seed, P_ENC_V, tag, index), s0(seed, P_ENC_E0, tag, index), s1(seed, P_ENC_E1, tag, index);
    sample_ternary(sv, host.data(), N);
    for (int i = 0; i < N; i++) host[N + i] = ctx.cdt->draw(s0);
    for (int i = 0; i < N; i++) host[2 * N + i] = ctx.cdt->draw(s1);
    memcpy(host.data() + 3 * N, m, sizeof(int64_t) * N);
    DevBuf polys((size_t)4 * limbs * N, s);
    signed_polys_to_ntt(ctx, s, host, 4, limbs, polys.p);
    Cts c = ev.alloc(1, 2, limbs);
    c.scale = scale;
    const size_t st = (size_t)limbs * N;
    launch_encrypt_combine(ev.lc(), c.d, polys.p, polys.p + st, polys.p + 2 * st, polys.p + 3 * st, ks.pk->p,
                           ctx.n_q, limbs);
    return c;
}

std::vector<int64_t> decrypt_coeffs(hx_context &ctx, const hx_keyset &ks, const Cts &c, cudaStream_t s)
{
    HX_CHECK(c.comps == 2, HX_EINVAL, "decryption needs a 2-component ciphertext");
    const int N = ctx.N, np = ks.n_parties, B = c.B;
    Eval ev(ctx, s);
    DevBuf sh((size_t)B * (np + 1) * N, s);
    launch_ddec_shares(ev.lc(), sh.p, c.view(N), ks.s_parts0->p, np, B);
    ev.ntt_inplace(sh.p, (size_t)N, B * (np + 1), {0}, {0}, true);
    std::vector<uint64_t> host((size_t)B * (np + 1) * N);
    HX_CUDA(cudaMemcpyAsync(host.data(), sh.p, sizeof(uint64_t) * host.size(), cudaMemcpyDeviceToHost, s));
    HX_CUDA(cudaStreamSynchronize(s));
    const uint64_t q = ctx.primes[0];
    std::vector<int64_t> out((size_t)B * N);
    for (int b = 0; b < B; b++)
        for (int i = 0; i < N; i++) {
            uint64_t acc = 0;  // each party's share is added on the host (DDec)
            for (int p = 0; p <= np; p++) {
                acc += host[((size_t)b * (np + 1) + p) * N + i];
                if (acc >= q) acc -= q;
            }
            out[(size_t)b * N + i] = acc > q / 2 ? (int64_t)acc - (int64_t)q : (int64_t)acc;
        }
    return out;
}

} // namespace hx
