// Context construction: primes, roots, twiddles and the RNS conversion tables
// of hybrid key switching and rescaling, all resident in HBM.
#include <cstring>

#include "runtime.h"

namespace hx {

DevBuf::DevBuf(size_t w, cudaStream_t s) : words(w), stream(s)
{
    if (w == 0) return;
    cudaError_t e = cudaMallocAsync((void **)&p, w * sizeof(uint64_t), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error{HX_ENOMEM, std::string("device allocation of ") + std::to_string(w * 8) + " bytes failed: " +
                                   cudaGetErrorString(e)};
    }
}

DevBuf::DevBuf(size_t w, bool) : words(w), pooled(false)
{
    if (w == 0) return;
    cudaError_t e = cudaMalloc((void **)&p, w * sizeof(uint64_t));
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error{HX_ENOMEM, std::string("device allocation of ") + std::to_string(w * 8) + " bytes failed: " +
                                   cudaGetErrorString(e)};
    }
}

DevBuf::~DevBuf()
{
    if (!p || !owned) return;
    if (pooled)
        cudaFreeAsync(p, stream);
    else
        cudaFree(p);
}

namespace {

template <class T> T *upload(const std::vector<T> &v)
{
    T *d = nullptr;
    HX_CUDA(cudaMalloc((void **)&d, sizeof(T) * v.size()));
    HX_CUDA(cudaMemcpy(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return d;
}

uint64_t mont_neg_inv(uint64_t q)
{
    uint64_t inv = q;  // Newton iteration for q^-1 mod 2^64 (q odd)
    for (int i = 0; i < 6; i++) inv *= 2 - q * inv;
    return (uint64_t)0 - inv;
}

unsigned bitrev(unsigned x, int bits)
{
    unsigned r = 0;
    for (int i = 0; i < bits; i++) {
        r = (r << 1) | (x & 1);
        x >>= 1;
    }
    return r;
}

uint64_t to_mont_host(uint64_t x, uint64_t q) { return (uint64_t)(((u128)x << 64) % q); }

} // namespace

void build_context(hx_context &c, const hx_params &p)
{
    HX_CHECK(p.log_n >= 11 && p.log_n <= 16, HX_EINVAL, "log_n must be in [11, 16]");
    HX_CHECK(p.n_q >= 1 && p.n_q <= 32 && p.n_p >= 1 && p.n_p <= HX_MAX_P, HX_EINVAL, "need 1..32 Q primes, 1..6 P primes");
    std::vector<int> bits;
    for (int i = 0; i < p.n_q; i++) bits.push_back(p.q_bits[i]);
    for (int i = 0; i < p.n_p; i++) bits.push_back(p.p_bits[i]);
    for (int b : bits) HX_CHECK(b >= 20 && b <= 61, HX_EINVAL, "prime sizes must be in [20, 61] bits");
    HX_CHECK(p.sigma > 0 && p.sigma < 100 && p.log2_scale > 0 && p.log2_scale < 62, HX_EINVAL, "bad sigma or scale");
    HX_CUDA(cudaGetDevice(&c.device));
    HX_CUDA(cudaDeviceGetAttribute(&c.t.n_sm, cudaDevAttrMultiProcessorCount, c.device));
    c.log_n = p.log_n;
    c.N = 1 << p.log_n;
    c.n_q = p.n_q;
    c.K = p.n_p;
    c.n_all = p.n_q + p.n_p;
    HX_CHECK(p.alpha >= 0 && p.alpha <= HX_MAX_P + 1, HX_EINVAL, "alpha must be in [0, 7] (0: one per special prime)");
    c.alpha = p.alpha ? p.alpha : p.n_p;
    c.dnum = (p.n_q + c.alpha - 1) / c.alpha;
    c.scale = std::pow(2.0, p.log2_scale);
    c.sigma = p.sigma;
    c.primes = choose_primes(p.log_n, bits);
    const int N = c.N, n_all = c.n_all, n_q = c.n_q, K = c.K;

    // keep freed stream-ordered memory cached in the pool
    cudaMemPool_t pool;
    HX_CUDA(cudaDeviceGetDefaultMemPool(&pool, c.device));
    uint64_t thr = ~0ull;
    HX_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));

    c.h_primes.resize(n_all);
    std::vector<ulonglong2> twf((size_t)n_all * N), twi((size_t)n_all * N);
    std::vector<uint64_t> pw(N), pwi(N);
    for (int i = 0; i < n_all; i++) {
        const uint64_t q = c.primes[i];
        const uint64_t psi = find_psi(q, c.log_n);
        c.psi.push_back(psi);
        PrimeConst &P = c.h_primes[i];
        memset(&P, 0, sizeof(P));
        P.q = q;
        P.mneg = mont_neg_inv(q);
        P.bar = shoup_companion(1, q);
        P.r_mod = (uint64_t)(((u128)1 << 64) % q);
        P.r_mod_sh = shoup_companion(P.r_mod, q);
        P.n_inv = hinv((uint64_t)N % q, q);
        P.n_inv_sh = shoup_companion(P.n_inv, q);
        const uint64_t psi_inv = hinv(psi, q);
        pw[0] = pwi[0] = 1;
        for (int k = 1; k < N; k++) {
            pw[k] = hmul(pw[k - 1], psi, q);
            pwi[k] = hmul(pwi[k - 1], psi_inv, q);
        }
        for (int k = 0; k < N; k++) {
            const uint64_t w = pw[bitrev(k, c.log_n)], wi = pwi[bitrev(k, c.log_n)];
            twf[(size_t)i * N + k] = make_ulonglong2(w, shoup_companion(w, q));
            twi[(size_t)i * N + k] = make_ulonglong2(wi, shoup_companion(wi, q));
        }
        P.n_inv_w1 = hmul(P.n_inv, twi[(size_t)i * N + 1].x, q);
        P.n_inv_w1_sh = shoup_companion(P.n_inv_w1, q);
    }

    // ModUp tables, by (limbs, digit)
    c.h_modup.assign((size_t)(n_q + 1) * c.dnum, ConvTable{});
    const int A = c.alpha;
    for (int l = 1; l <= n_q; l++) {
        const int ext = l + K, nd = (l + A - 1) / A;
        for (int j = 0; j < nd; j++) {
            ConvTable &T = c.h_modup[(size_t)l * c.dnum + j];
            memset(&T, 0, sizeof(T));
            const int lo = j * A, hi = std::min((j + 1) * A, l);
            T.n_src = hi - lo;
            for (int i = lo; i < hi; i++) {
                T.src_row[i - lo] = i;
                T.src_prime[i - lo] = i;
            }
            int nd_ = 0;
            for (int r = 0; r < ext; r++) {
                if (r >= lo && r < hi) continue;
                T.dst_row[nd_] = r;
                T.dst_prime[nd_] = r < l ? r : n_q + (r - l);
                nd_++;
            }
            T.n_dst = nd_;
            for (int i = 0; i < T.n_src; i++) {
                const uint64_t qi = c.primes[lo + i];
                uint64_t qh = 1;
                for (int k = lo; k < hi; k++)
                    if (k != lo + i) qh = hmul(qh, c.primes[k] % qi, qi);
                T.inv[i] = hinv(qh, qi);
                T.inv_sh[i] = shoup_companion(T.inv[i], qi);
                for (int d = 0; d < T.n_dst; d++) {
                    const uint64_t t = c.primes[T.dst_prime[d]];
                    uint64_t qt = 1;
                    for (int k = lo; k < hi; k++)
                        if (k != lo + i) qt = hmul(qt, c.primes[k] % t, t);
                    T.w[i][d] = qt;
                    T.w_sh[i][d] = shoup_companion(qt, t);
                }
            }
        }
    }
    // ModDown tables, by limbs: P -> Q_l
    c.h_moddown.assign(n_q + 1, ModDownTable{});
    for (int l = 1; l <= n_q; l++) {
        ModDownTable &M = c.h_moddown[l];
        memset(&M, 0, sizeof(M));
        ConvTable &T = M.conv;
        T.n_src = K;
        T.n_dst = l;
        for (int k = 0; k < K; k++) {
            T.src_row[k] = l + k;
            T.src_prime[k] = n_q + k;
        }
        for (int i = 0; i < l; i++) {
            T.dst_row[i] = i;
            T.dst_prime[i] = i;
        }
        for (int k = 0; k < K; k++) {
            const uint64_t pk = c.primes[n_q + k];
            uint64_t ph = 1;
            for (int m = 0; m < K; m++)
                if (m != k) ph = hmul(ph, c.primes[n_q + m] % pk, pk);
            T.inv[k] = hinv(ph, pk);
            T.inv_sh[k] = shoup_companion(T.inv[k], pk);
            for (int i = 0; i < l; i++) {
                const uint64_t t = c.primes[i];
                uint64_t pt = 1;
                for (int m = 0; m < K; m++)
                    if (m != k) pt = hmul(pt, c.primes[n_q + m] % t, t);
                T.w[k][i] = pt;
                T.w_sh[k][i] = shoup_companion(pt, t);
            }
        }
        for (int i = 0; i < l; i++) {
            const uint64_t t = c.primes[i];
            uint64_t Pm = 1;
            for (int m = 0; m < K; m++) Pm = hmul(Pm, c.primes[n_q + m] % t, t);
            M.pinv[i] = hinv(Pm, t);
            M.pinv_sh[i] = shoup_companion(M.pinv[i], t);
        }
    }
    // Rescale tables, by limbs (top prime l-1)
    c.h_rescale.assign(n_q + 1, RescaleTable{});
    for (int l = 2; l <= n_q; l++) {
        RescaleTable &R = c.h_rescale[l];
        memset(&R, 0, sizeof(R));
        const uint64_t qt = c.primes[l - 1];
        R.half = (qt - 1) / 2;
        for (int i = 0; i < l - 1; i++) {
            const uint64_t q = c.primes[i];
            R.qinv[i] = hinv(qt % q, q);
            R.qinv_sh[i] = shoup_companion(R.qinv[i], q);
            R.half_mod[i] = R.half % q;
        }
    }
    // relinearisation + rescale tables, by limbs: divide by P q_top, q_top = q_{l-1}
    c.h_relin_rs.assign(n_q + 1, RelinRescaleTable{});
    for (int l = 2; l <= n_q; l++) {
        RelinRescaleTable &M = c.h_relin_rs[l];
        memset(&M, 0, sizeof(M));
        ConvTable &T = M.conv;
        T.n_src = K + 1;
        T.n_dst = l - 1;
        for (int k = 0; k <= K; k++) {  // sources: q_top, then the special primes (rows l-1 .. l+K-1)
            T.src_row[k] = l - 1 + k;
            T.src_prime[k] = k == 0 ? l - 1 : n_q + k - 1;
        }
        for (int i = 0; i < l - 1; i++) {
            T.dst_row[i] = i;
            T.dst_prime[i] = i;
        }
        auto prod_mod = [&](int skip, uint64_t t) {  // (P q_top / source skip) mod t, or P q_top mod t
            uint64_t v = 1;
            for (int k = 0; k <= K; k++)
                if (k != skip) v = hmul(v, c.primes[T.src_prime[k]] % t, t);
            return v;
        };
        for (int k = 0; k <= K; k++) {
            const uint64_t sk = c.primes[T.src_prime[k]];
            T.inv[k] = hinv(prod_mod(k, sk), sk);
            T.inv_sh[k] = shoup_companion(T.inv[k], sk);
            for (int i = 0; i < l - 1; i++) {
                T.w[k][i] = prod_mod(k, c.primes[i]);
                T.w_sh[k][i] = shoup_companion(T.w[k][i], c.primes[i]);
            }
        }
        // h = floor(P q_top / 2) = (P q_top - 1) / 2, the product being odd: h = (P q_top - 1) * 2^-1 mod t
        auto half_mod = [&](uint64_t t) {
            const uint64_t pq = prod_mod(-1, t);
            return hmul((pq + t - 1) % t, (t + 1) / 2, t);
        };
        T.shift = 1;
        for (int k = 0; k <= K; k++) {
            T.add_src[k] = half_mod(c.primes[T.src_prime[k]]);
            T.inv_d[k] = 1.0 / (double)c.primes[T.src_prime[k]];
        }
        for (int i = 0; i < l - 1; i++) {
            T.sub_dst[i] = half_mod(c.primes[i]);
            T.prod_mod[i] = prod_mod(-1, c.primes[i]);
        }
        for (int i = 0; i < l; i++) {
            const uint64_t t = c.primes[i];
            uint64_t Pm = 1;
            for (int m = 0; m < K; m++) Pm = hmul(Pm, c.primes[n_q + m] % t, t);
            M.pmod[i] = Pm;
            M.pmod_sh[i] = shoup_companion(Pm, t);
            if (i < l - 1) {
                M.pqinv[i] = hinv(prod_mod(-1, t), t);
                M.pqinv_sh[i] = shoup_companion(M.pqinv[i], t);
            }
        }
    }
    c.t.primes = upload(c.h_primes);
    c.t.tw_fwd = upload(twf);
    c.t.tw_inv = upload(twi);
    c.t.modup = upload(c.h_modup);
    c.t.moddown = upload(c.h_moddown);
    c.t.rescale = upload(c.h_rescale);
    c.t.relin_rs = upload(c.h_relin_rs);
    std::vector<int> ids(n_all);
    for (int i = 0; i < n_all; i++) ids[i] = i;
    c.d_prime_ids = upload(ids);
    c.enc.reset(new Encoder(c.log_n));
    c.cdt.reset(new GaussianCdt(c.sigma));
}

SideStream &side_stream(hx_context &ctx, cudaStream_t main)
{
    std::lock_guard<std::mutex> lk(ctx.side_mu);
    if (ctx.profiling) {
        // per-kernel timing runs the chains one after another on the caller's stream, so every
        // launch's event interval is that kernel alone
        SideStream &ser = ctx.side_serial[main];
        if (!ser.e[0])
            for (auto &e : ser.e) HX_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ser.s = ser.s2 = main;
        return ser;
    }
    SideStream &ss = ctx.side[main];
    if (!ss.s) {
        HX_CUDA(cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking));
        HX_CUDA(cudaStreamCreateWithFlags(&ss.s2, cudaStreamNonBlocking));
        for (auto &e : ss.e) HX_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    return ss;
}

cudaStream_t group_stream(hx_context &ctx, cudaStream_t main, size_t i)
{
    if (ctx.profiling) return main;
    std::lock_guard<std::mutex> lk(ctx.side_mu);
    while (ctx.group_streams.size() <= i) {
        cudaStream_t s = nullptr;
        HX_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        ctx.group_streams.push_back(s);
    }
    return ctx.group_streams[i];
}

void destroy_context(hx_context &c)
{
    cudaDeviceSynchronize();
    c.plans.clear();
    c.plans_pinned.clear();
    c.mask_real.clear();
    if (c.plan_stream) {
        cudaStreamSynchronize(c.plan_stream);
        cudaStreamDestroy(c.plan_stream);
    }
    for (auto &kv : c.side) {
        for (auto &e : kv.second.e)
            if (e) cudaEventDestroy(e);
        if (kv.second.s) cudaStreamDestroy(kv.second.s);
        if (kv.second.s2) cudaStreamDestroy(kv.second.s2);
    }
    c.side.clear();
    for (auto &kv : c.side_serial)
        for (auto &e : kv.second.e)
            if (e) cudaEventDestroy(e);
    c.side_serial.clear();
    for (cudaStream_t s : c.group_streams) cudaStreamDestroy(s);
    c.group_streams.clear();
    cudaFree(c.t.primes);
    cudaFree(c.t.tw_fwd);
    cudaFree(c.t.tw_inv);
    cudaFree(c.t.modup);
    cudaFree(c.t.moddown);
    cudaFree(c.t.relin_rs);
    cudaFree(c.t.rescale);
    cudaFree(c.d_prime_ids);
}

Cts gather(hx_context &ctx, const hx_ct *const *cts, size_t count, cudaStream_t s)
{
    HX_CHECK(count >= 1, HX_EINVAL, "empty batch");
    for (size_t i = 0; i < count; i++) {
        HX_CHECK(cts[i], HX_EINVAL, "null ciphertext in a batch");
        // a ciphertext of another context has another row length: never let it reach a copy or kernel
        HX_CHECK(cts[i]->ctx == &ctx, HX_EINVAL, "ciphertext of another context in a batch");
    }
    const Cts &f = cts[0]->c;
    for (size_t i = 0; i < count; i++) {
        HX_CHECK(cts[i]->c.limbs == f.limbs && cts[i]->c.comps == f.comps, HX_ESCALE,
                 "batch entries must share level and shape");
        HX_CHECK(cts[i]->c.scale == f.scale, HX_ESCALE, "batch entries must share the scale");
    }
    Eval ev(ctx, s);
    Cts out = ev.alloc((int)count, f.comps, f.limbs);
    out.scale = f.scale;
    const size_t N = ctx.N;
    for (size_t i = 0; i < count; i++)
        for (int c = 0; c < f.comps; c++)
            HX_CUDA(cudaMemcpyAsync(out.d + i * out.bstride(N) + c * out.cstride(N),
                                    cts[i]->c.d + c * cts[i]->c.cstride(N), sizeof(uint64_t) * f.limbs * N,
                                    cudaMemcpyDeviceToDevice, s));
    return out;
}

void scatter(hx_context &ctx, const Cts &b, hx_ct **out, cudaStream_t s)
{
    const size_t N = ctx.N;
    Eval ev(ctx, s);
    for (int i = 0; i < b.B; i++) {
        hx_ct *h = new hx_ct;
        h->ctx = &ctx;
        h->c = ev.alloc(1, b.comps, b.limbs);
        h->c.scale = b.scale;
        for (int c = 0; c < b.comps; c++)
            HX_CUDA(cudaMemcpyAsync(h->c.d + c * h->c.cstride(N), b.d + i * b.bstride(N) + c * b.cstride(N),
                                    sizeof(uint64_t) * b.limbs * N, cudaMemcpyDeviceToDevice, s));
        out[i] = h;
    }
}

} // namespace hx
