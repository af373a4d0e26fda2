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
        const int A = ctx.alpha;  // digit j: primes j*A .. min((j+1)*A, n_q) - 1
        for (int r = 0; r < n_all; r++) gad[r] = (r >= j * A && r < std::min((j + 1) * A, n_q)) ? P_mod[r] : 0;
        uint64_t *bj = out.buf->p + (size_t)(2 * j) * n_all * N;
        uint64_t *aj = bj + (size_t)n_all * N;
        HX_CUDA(cudaMemcpyAsync(aj, a.data(), sizeof(uint64_t) * a.size(), cudaMemcpyHostToDevice, s));
        HX_CUDA(cudaMemcpyAsync(gad_d.p, gad.data(), sizeof(uint64_t) * n_all, cudaMemcpyHostToDevice, s));
        signed_polys_to_ntt(ctx, s, e, 1, n_all, e_ntt.p);
        launch_keygen_b(ev.lc(), bj, aj, e_ntt.p, ks.s_ntt->p, sp, gad_d.p, n_all, nullptr, true);
        HX_CUDA(cudaStreamSynchronize(s));  // host staging vectors are reused
    }
}

// Fig. 1 item 13, every party's share for entry b at limb l, summed:
//   out0 = c0 + sum_i (s_i c1 + u_i b' + e0_i),  out1 = sum_i (u_i a' + e1_i)
// S: [n_parties][limbs][N]; R: [B][n_parties][3 (u, e0, e1)][limbs][N]; pk: [2][n_q][N]
__global__ void k_pcks(View out, View ct, const uint64_t *__restrict__ S, const uint64_t *__restrict__ R,
                       const uint64_t *__restrict__ pk, const PrimeConst *__restrict__ primes, int np, int limbs,
                       int n_q, int n)
{
    const int l = blockIdx.y, bi = blockIdx.z;
    const PrimeConst P = primes[l];
    const uint64_t *c0 = ct.p + bi * ct.bstride + (size_t)l * n, *c1 = c0 + ct.cstride;
    const uint64_t *pb = pk + (size_t)l * n, *pa = pk + ((size_t)n_q + l) * n;
    const size_t poly = (size_t)limbs * n;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        uint64_t h0 = c0[j], h1 = 0;
        const uint64_t x1 = c1[j], bb = pb[j], aa = pa[j];
        for (int i = 0; i < np; i++) {
            const uint64_t *r = R + ((size_t)bi * np + i) * 3 * poly + (size_t)l * n + j;
            const uint64_t u = r[0], e0 = r[poly], e1 = r[2 * poly];
            const uint64_t s0 = addmod(mulmod(S[i * poly + (size_t)l * n + j], x1, P), mulmod(u, bb, P), P.q);
            h0 = addmod(h0, addmod(s0, e0, P.q), P.q);
            h1 = addmod(h1, addmod(mulmod(u, aa, P), e1, P.q), P.q);
        }
        out.p[bi * out.bstride + (size_t)l * n + j] = h0;
        out.p[bi * out.bstride + out.cstride + (size_t)l * n + j] = h1;
    }
}

// Fig. 1 item 14, re-encryption side for entry b at limb l:
//   out0 = W[b][0] + sum_i (W[b][1+i] - s_i a_b),  out1 = a_b
// W: [B][1 + n_parties][n_q][N] (NTT of m' and of the parties' -M'_i + e1_i); A: [B][n_q][N];
// S: [n_parties][n_q][N]
__global__ void k_dboot_combine(View out, const uint64_t *__restrict__ W, const uint64_t *__restrict__ A,
                                const uint64_t *__restrict__ S, const PrimeConst *__restrict__ primes, int np, int n_q,
                                int n)
{
    const int l = blockIdx.y, bi = blockIdx.z;
    const PrimeConst P = primes[l];
    const size_t poly = (size_t)n_q * n;
    const uint64_t *w = W + (size_t)bi * (np + 1) * poly + (size_t)l * n;
    const uint64_t *a = A + (size_t)bi * poly + (size_t)l * n;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        uint64_t c = w[j];
        const uint64_t aj = a[j];
        for (int i = 0; i < np; i++)
            c = addmod(c, submod(w[(size_t)(i + 1) * poly + j], mulmod(S[i * poly + (size_t)l * n + j], aj, P), P.q),
                       P.q);
        out.p[bi * out.bstride + (size_t)l * n + j] = c;
        out.p[bi * out.bstride + out.cstride + (size_t)l * n + j] = aj;
    }
}

constexpr uint64_t kGammaK = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ uint64_t kmix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// value j of the wide uniform sampler: (d_2j * 2^64 + d_(2j+1)) mod m, d_i = mix64(st + (i+1) gamma)
__device__ __forceinline__ uint64_t uniform_wide_at(uint64_t st, int j, uint64_t m)
{
    const uint64_t hi = kmix64(st + (uint64_t)(2 * j + 1) * kGammaK);
    const uint64_t lo = kmix64(st + (uint64_t)(2 * j + 2) * kGammaK);
    return (uint64_t)((((unsigned __int128)hi << 64) | lo) % m);
}

// draw j of the discrete Gaussian (cumulative table th, 2*bound+1 entries)
__device__ __forceinline__ int64_t gauss_at(uint64_t st, int j, const uint64_t *__restrict__ th, int bound)
{
    const uint64_t x = kmix64(st + (uint64_t)(j + 1) * kGammaK) >> 1;
    int idx = 0;
    while (idx < 2 * bound && x >= th[idx]) idx++;
    return (int64_t)idx - bound;
}

__device__ __forceinline__ double round_half_away_dev(double x)
{
    const double r = floor(__dadd_rn(fabs(x), 0.5));
    return x < 0 ? -r : r;
}

// Fig. 1 item 14, the masked decryption side for entry b, coefficient j: every party's share
// c1*s_i (sh, coefficient form mod q_0, after c0) plus its mask M_i and e0_i, summed with c0;
// the centered sum rescaled to the output scale (W[b][0]) and every party's re-encryption
// coefficients -round(M_i * ratio) + e1_i (W[b][1+i]).  st: [B][n_parties][3] stream states
// (mask, e0, e1).
__global__ void k_dboot_shares(int64_t *W, const uint64_t *__restrict__ sh, const uint64_t *__restrict__ st,
                               const uint64_t *__restrict__ th, int gbound, uint64_t mbound, uint64_t q0, double ratio,
                               int np, int n)
{
    const int b = blockIdx.y;
    const uint64_t *shb = sh + (size_t)b * (np + 1) * n;
    int64_t *Wb = W + (size_t)b * (np + 1) * n;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        uint64_t v = shb[j];
        for (int i = 0; i < np; i++) {
            const uint64_t *s3 = st + ((size_t)b * np + i) * 3;
            const int64_t M = (int64_t)uniform_wide_at(s3[0], j, 2 * mbound + 1) - (int64_t)mbound;
            const int64_t add = M + gauss_at(s3[1], j, th, gbound);
            uint64_t t = shb[(size_t)(i + 1) * n + j];
            t = add >= 0 ? (t + (uint64_t)add) % q0 : (t + q0 - ((uint64_t)(-add)) % q0) % q0;
            v = (v + t) % q0;
            Wb[(size_t)(i + 1) * n + j] =
                -(int64_t)round_half_away_dev(__dmul_rn((double)M, ratio)) + gauss_at(s3[2], j, th, gbound);
        }
        const int64_t c = v > q0 / 2 ? (int64_t)v - (int64_t)q0 : (int64_t)v;
        Wb[j] = (int64_t)round_half_away_dev(__dmul_rn((double)c, ratio));
    }
}

// the common reference polynomial of entry b: row r uniform mod q_r (NTT form), stream st[b][r]
__global__ void k_dboot_crp(uint64_t *A, const uint64_t *__restrict__ st, const PrimeConst *__restrict__ primes,
                            int nq, int n)
{
    const int r = blockIdx.y, b = blockIdx.z;
    const uint64_t q = primes[r].q, s0 = st[(size_t)b * nq + r];
    uint64_t *o = A + ((size_t)b * nq + r) * n;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) o[j] = uniform_wide_at(s0, j, q);
}

int blocks_for(int n) { return (n + 255) / 256; }

// the parties' ternary shares as NTT-form residues over primes 0..rows-1
BufPtr party_shares_ntt(hx_context &ctx, const hx_keyset &ks, int rows, cudaStream_t s)
{
    std::vector<int64_t> flat;
    for (auto &v : ks.s_parts) flat.insert(flat.end(), v.begin(), v.end());
    BufPtr out = std::make_shared<DevBuf>((size_t)ks.n_parties * rows * ctx.N, s);
    signed_polys_to_ntt(ctx, s, flat, ks.n_parties, rows, out->p);
    return out;
}

// DDec shares at q_0 in coefficient form, host copy: [B][1 + n_parties][N] (c0, then c1*s_i)
std::vector<uint64_t> ddec_share_polys(hx_context &ctx, const hx_keyset &ks, const Cts &c, cudaStream_t s)
{
    const int N = ctx.N, np = ks.n_parties, B = c.B;
    Eval ev(ctx, s);
    DevBuf sh((size_t)B * (np + 1) * N, s);
    launch_ddec_shares(ev.lc(), sh.p, c.view(N), ks.s_parts0->p, np, B);
    ev.ntt_inplace(sh.p, (size_t)N, B * (np + 1), {0}, {0}, true);
    std::vector<uint64_t> host((size_t)B * (np + 1) * N);
    HX_CUDA(cudaMemcpyAsync(host.data(), sh.p, sizeof(uint64_t) * host.size(), cudaMemcpyDeviceToHost, s));
    HX_CUDA(cudaStreamSynchronize(s));
    return host;
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
    const std::vector<uint64_t> host = ddec_share_polys(ctx, ks, c, s);
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

// Fig. 1 item 13: collective public-key switch of every entry of ct to the
// public key of `to`.  Party i draws u_i (ternary), e0_i, e1_i (Gaussian) from
// streams (seed, purpose, i, b) and contributes (s_i c1 + u_i b' + e0_i,
// u_i a' + e1_i); the sums are added to (c0, 0).
Cts dkeyswitch(hx_context &ctx, const hx_keyset &from, const hx_keyset &to, const Cts &ct, uint64_t seed,
               cudaStream_t s)
{
    HX_CHECK(ct.comps == 2, HX_EINVAL, "key switching needs a 2-component ciphertext");
    const int N = ctx.N, np = from.n_parties, L = ct.limbs, B = ct.B;
    Eval ev(ctx, s);
    BufPtr S = party_shares_ntt(ctx, from, L, s);
    std::vector<int64_t> host((size_t)B * np * 3 * N);
    for (int b = 0; b < B; b++)
        for (int i = 0; i < np; i++) {
            int64_t *r = host.data() + ((size_t)b * np + i) * 3 * N;
            Stream su(seed, P_PCKS_U, i, b), s0(seed, P_PCKS_E0, i, b), s1(seed, P_PCKS_E1, i, b);
            sample_ternary(su, r, N);
            for (int k = 0; k < N; k++) r[N + k] = ctx.cdt->draw(s0);
            for (int k = 0; k < N; k++) r[2 * N + k] = ctx.cdt->draw(s1);
        }
    DevBuf R((size_t)B * np * 3 * L * N, s);
    signed_polys_to_ntt(ctx, s, host, B * np * 3, L, R.p);
    Cts out = ev.alloc(B, 2, L);
    out.scale = ct.scale;
    k_pcks<<<dim3(blocks_for(N), L, B), 256, 0, s>>>(out.view(N), ct.view(N), S->p, R.p, to.pk->p, ctx.t.primes, np, L,
                                                    ctx.n_q, N);
    HX_CUDA(cudaGetLastError());
    ctx.counters[C_LAUNCH] += 1;
    HX_CUDA(cudaStreamSynchronize(s));  // host staging buffers go out of scope
    return out;
}

// Fig. 1 item 14: collective refresh of every entry b (seed seeds[b], refresh
// index `counter`).  Party i adds a uniform mask M_i in [-bound, bound] (bound =
// (floor(q_0/4) - 1) / n_parties) and Gaussian e0_i to its decryption share at
// q_0, so the combined v = c0 + sum_i (c1 s_i + M_i + e0_i) mod q_0 is the
// masked plaintext Delta_ct m + e + sum M_i (|v| < q_0/2); m' = round(v *
// Delta/Delta_ct).  With a common reference polynomial a (uniform over Q, in
// NTT form), party i's re-encryption share is -s_i a - M'_i + e1_i, M'_i =
// round(M_i * Delta/Delta_ct); the output (m' + sum_i shares, a) is at the top
// level and scale Delta.
Cts dbootstrap(hx_context &ctx, const hx_keyset &ks, const Cts &ct, const std::vector<uint64_t> &seeds, int counter,
               cudaStream_t s)
{
    HX_CHECK(ct.comps == 2, HX_EINVAL, "refresh needs a 2-component ciphertext");
    HX_CHECK((int)seeds.size() == ct.B, HX_EINVAL, "one refresh seed per batch entry");
    const int N = ctx.N, np = ks.n_parties, B = ct.B, nq = ctx.n_q;
    const uint64_t q0 = ctx.primes[0];
    const uint64_t bound = (q0 / 4 - 1) / (uint64_t)np;
    const double ratio = ctx.scale / ct.scale;
    Eval ev(ctx, s);
    // every party's decryption share c1*s_i at q_0, coefficient form, on the device
    DevBuf sh((size_t)B * (np + 1) * N, s);
    launch_ddec_shares(ev.lc(), sh.p, ct.view(N), ks.s_parts0->p, np, B);
    ev.ntt_inplace(sh.p, (size_t)N, B * (np + 1), {0}, {0}, true);
    // stream states: masks and errors per (entry, party), the reference polynomial per (entry, row)
    std::vector<uint64_t> st((size_t)B * np * 3), st_crp((size_t)B * nq);
    for (int b = 0; b < B; b++) {
        for (int i = 0; i < np; i++) {
            st[((size_t)b * np + i) * 3 + 0] = Stream(seeds[b], P_DB_MASK, i, counter).state;
            st[((size_t)b * np + i) * 3 + 1] = Stream(seeds[b], P_DB_E0, i, counter).state;
            st[((size_t)b * np + i) * 3 + 2] = Stream(seeds[b], P_DB_E1, i, counter).state;
        }
        for (int r = 0; r < nq; r++) st_crp[(size_t)b * nq + r] = Stream(seeds[b], P_DB_CRP, r, counter).state;
    }
    DevBuf st_d(st.size(), s), stc_d(st_crp.size(), s), th_d(ctx.cdt->th.size(), s);
    HX_CUDA(cudaMemcpyAsync(st_d.p, st.data(), sizeof(uint64_t) * st.size(), cudaMemcpyHostToDevice, s));
    HX_CUDA(cudaMemcpyAsync(stc_d.p, st_crp.data(), sizeof(uint64_t) * st_crp.size(), cudaMemcpyHostToDevice, s));
    HX_CUDA(cudaMemcpyAsync(th_d.p, ctx.cdt->th.data(), sizeof(uint64_t) * ctx.cdt->th.size(), cudaMemcpyHostToDevice,
                            s));
    DevBuf W((size_t)B * (np + 1) * N, s), Wd((size_t)B * (np + 1) * nq * N, s), Ad((size_t)B * nq * N, s);
    k_dboot_shares<<<dim3(blocks_for(N), B), 256, 0, s>>>(reinterpret_cast<int64_t *>(W.p), sh.p, st_d.p, th_d.p,
                                                          ctx.cdt->bound, bound, q0, ratio, np, N);
    k_dboot_crp<<<dim3(blocks_for(N), nq, B), 256, 0, s>>>(Ad.p, stc_d.p, ctx.t.primes, nq, N);
    HX_CUDA(cudaGetLastError());
    // the rescaled plaintext and the parties' re-encryption coefficients over Q, NTT form
    launch_signed_to_rows(ev.lc(), Wd.p, reinterpret_cast<const int64_t *>(W.p), nq, B * (np + 1), (size_t)N,
                          ctx.d_prime_ids);
    ev.ntt_inplace(Wd.p, (size_t)nq * N, B * (np + 1), iota_vec(0, nq), iota_vec(0, nq), false);
    BufPtr S = party_shares_ntt(ctx, ks, nq, s);
    Cts out = ev.alloc(B, 2, nq);
    out.scale = ctx.scale;
    k_dboot_combine<<<dim3(blocks_for(N), nq, B), 256, 0, s>>>(out.view(N), Wd.p, Ad.p, S->p, ctx.t.primes, np, nq, N);
    HX_CUDA(cudaGetLastError());
    ctx.counters[C_LAUNCH] += 3;
    ctx.counters[C_REFRESH] += B;
    HX_CUDA(cudaStreamSynchronize(s));  // the host stream-state vectors go out of scope
    return out;
}

} // namespace hx
