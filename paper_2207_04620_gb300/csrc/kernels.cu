// Device kernels of the RNS-CKKS hot path other than the NTT (ntt.cu) and
// their launchers: elementwise products and sums, automorphisms, fast basis
// conversion, key inner products and ModDown epilogues, rescale, keys and
// encryption pieces, aggregation and the ALU calibration.
#include <algorithm>
#include <cstdio>

#include "launch_util.cuh"

namespace hx {

namespace {

__device__ __forceinline__ int brv_bits(unsigned x, int bits) { return (int)(__brev(x) >> (32 - bits)); }

// index of the NTT slot that the automorphism X -> X^g brings to slot j:
// 2brv(j')+1 = (2brv(j)+1)*g mod 2N
__device__ __forceinline__ int galois_src(int j, uint64_t g, int log_n)
{
    const uint64_t two_n_mask = (2ull << log_n) - 1;
    uint64_t e = ((2ull * (uint64_t)brv_bits(j, log_n) + 1) * g) & two_n_mask;
    return brv_bits((unsigned)((e - 1) >> 1), log_n);
}

// A block's coordinates and its grid's extent: the hardware's, or those of one job inside a launch
// that runs the same kernel body over the jobs of several rings (see the several-ring key switch)
struct Blk {
    int x, y, z, gx, gy, gz;
    __device__ __forceinline__ static Blk hw()
    {
        return Blk{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z, (int)gridDim.x, (int)gridDim.y, (int)gridDim.z};
    }
};

// ---- elementwise ----------------------------------------------------------------
// grid: x over pairs of coefficients, y = limb, z = b*comps + comp

__global__ void k_add(View out, View a, View b, const PrimeConst *__restrict__ primes, int comps, int n, bool sub)
{
    const int l = blockIdx.y, bc = blockIdx.z, bi = bc / comps, ci = bc % comps;
    const uint64_t q = primes[l].q;
    const size_t oo = bi * out.bstride + ci * out.cstride + (size_t)l * n;
    const size_t oa = bi * a.bstride + ci * a.cstride + (size_t)l * n;
    const size_t ob = bi * b.bstride + ci * b.cstride + (size_t)l * n;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) * 2; j < n; j += gridDim.x * blockDim.x * 2) {
        const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(a.p + oa + j);
        const ulonglong2 y = *reinterpret_cast<const ulonglong2 *>(b.p + ob + j);
        ulonglong2 r;
        r.x = sub ? submod(x.x, y.x, q) : addmod(x.x, y.x, q);
        r.y = sub ? submod(x.y, y.y, q) : addmod(x.y, y.y, q);
        *reinterpret_cast<ulonglong2 *>(out.p + oo + j) = r;
    }
}

__global__ void k_copy(View out, View a, int comps, int n)
{
    const int l = blockIdx.y, bc = blockIdx.z, bi = bc / comps, ci = bc % comps;
    const size_t oo = bi * out.bstride + ci * out.cstride + (size_t)l * n;
    const size_t oa = bi * a.bstride + ci * a.cstride + (size_t)l * n;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) * 2; j < n; j += gridDim.x * blockDim.x * 2)
        *reinterpret_cast<ulonglong2 *>(out.p + oo + j) = *reinterpret_cast<const ulonglong2 *>(a.p + oa + j);
}

// Alg. 6 Aggregation: the sum over parties of one gradient ciphertext, times a
// constant, streamed from the parties' buffers in place (16-byte loads, four
// parties in flight per thread, a Barrett reduction every 4 terms).
__global__ void k_aggregate(View out, const AggSrc *__restrict__ src, int n_parties, int count,
                            const __grid_constant__ Scalars C, const PrimeConst *__restrict__ primes, int comps, int n)
{
    const int l = blockIdx.y, bc = blockIdx.z, m = bc / comps, ci = bc % comps;
    const PrimeConst P = primes[l];
    const size_t off = (size_t)l * n;
    uint64_t *o = out.p + m * out.bstride + ci * out.cstride + off;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) * 2; j < n; j += gridDim.x * blockDim.x * 2) {
        uint64_t s0 = 0, s1 = 0;
        int i = 0;
        for (; i + 4 <= n_parties; i += 4) {
            ulonglong2 x[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const AggSrc a = src[(size_t)(i + u) * count + m];
                x[u] = __ldcs(reinterpret_cast<const ulonglong2 *>(a.p + ci * a.cstride + off + j));
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                s0 += x[u].x;
                s1 += x[u].y;
            }
            s0 = reduce64(s0, P.q, P.bar);  // below q + 4q < 2^64 before the reduction
            s1 = reduce64(s1, P.q, P.bar);
        }
        for (; i < n_parties; i++) {
            const AggSrc a = src[(size_t)i * count + m];
            const ulonglong2 x = __ldcs(reinterpret_cast<const ulonglong2 *>(a.p + ci * a.cstride + off + j));
            s0 = reduce64(s0 + x.x, P.q, P.bar);
            s1 = reduce64(s1 + x.y, P.q, P.bar);
        }
        ulonglong2 r;
        r.x = shoup(reduce64(s0, P.q, P.bar), C.v[l], C.sh[l], P.q);
        r.y = shoup(reduce64(s1, P.q, P.bar), C.v[l], C.sh[l], P.q);
        *reinterpret_cast<ulonglong2 *>(o + j) = r;
    }
}

// one thread: both components of batch entry bi at two adjacent coefficients, so every mask
// word loaded (16 bytes, two coefficients) serves four products; NB >= the number of babies
template <int NB>
__global__ void __launch_bounds__(128) k_lintrans_mac(const __grid_constant__ MacArgs A,
                                                      const PrimeConst *__restrict__ primes, int B, int limbs, int n)
{
    // batch entries vary fastest over the grid: the blocks reading one mask tile run together and
    // share it through L2 (a plan's masks are larger than L2)
    const int bi = blockIdx.x, l = blockIdx.z;
    const PrimeConst P = primes[l];
    const size_t ob0 = bi * A.baby_bstride + (size_t)l * n, ob1 = ob0 + A.baby_cstride;
    const size_t gstride = (size_t)B * 2 * limbs * n;
    const size_t oo0 = (size_t)bi * 2 * limbs * n + (size_t)l * n, oo1 = oo0 + (size_t)limbs * n;
    for (int j = (blockIdx.y * blockDim.x + threadIdx.x) * 2; j < n; j += gridDim.y * blockDim.x * 2) {
        ulonglong2 v0[NB], v1[NB];
#pragma unroll
        for (int m = 0; m < NB; m++) {
            if (m < A.n_baby) {
                v0[m] = *reinterpret_cast<const ulonglong2 *>(A.baby[m] + ob0 + j);
                v1[m] = *reinterpret_cast<const ulonglong2 *>(A.baby[m] + ob1 + j);
            }
        }
        for (int g = 0; g < A.n_group; g++) {
            Acc128 a0, a1, b0, b1;  // (component, coefficient)
#pragma unroll
            for (int m = 0; m < NB; m++) {
                const uint64_t *mk = A.mask[g][m];
                if (m < A.n_baby && mk) {
                    const ulonglong2 w = *reinterpret_cast<const ulonglong2 *>(mk + (size_t)l * n + j);
                    a0.mac(v0[m].x, w.x);
                    a1.mac(v0[m].y, w.y);
                    b0.mac(v1[m].x, w.x);
                    b1.mac(v1[m].y, w.y);
                }
            }
            *reinterpret_cast<ulonglong2 *>(A.out + g * gstride + oo0 + j) =
                make_ulonglong2(redc_few(a0.hi, a0.lo, P), redc_few(a1.hi, a1.lo, P));
            *reinterpret_cast<ulonglong2 *>(A.out + g * gstride + oo1 + j) =
                make_ulonglong2(redc_few(b0.hi, b0.lo, P), redc_few(b1.hi, b1.lo, P));
        }
    }
}

// out_c = a_c * pt  with pt in Montgomery form (pt * 2^64 mod q): one reduction
__global__ void k_mul_plain(View out, View a, const uint64_t *__restrict__ pt, const PrimeConst *__restrict__ primes,
                            int n)
{
    const int l = blockIdx.y, bc = blockIdx.z, bi = bc / 2, ci = bc % 2;
    const PrimeConst P = primes[l];
    const size_t oo = bi * out.bstride + ci * out.cstride + (size_t)l * n;
    const size_t oa = bi * a.bstride + ci * a.cstride + (size_t)l * n;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) * 2; j < n; j += gridDim.x * blockDim.x * 2) {
        const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(a.p + oa + j);
        const ulonglong2 w = *reinterpret_cast<const ulonglong2 *>(pt + (size_t)l * n + j);
        ulonglong2 r;
        r.x = redc_few(__umul64hi(x.x, w.x), x.x * w.x, P);
        r.y = redc_few(__umul64hi(x.y, w.y), x.y * w.y, P);
        *reinterpret_cast<ulonglong2 *>(out.p + oo + j) = r;
    }
}

// out = a * s_l (Shoup constant per limb)
__global__ void k_mul_scalar(View out, View a, const __grid_constant__ Scalars sc, const PrimeConst *__restrict__ primes,
                             int comps, int n)
{
    const int l = blockIdx.y, bc = blockIdx.z, bi = bc / comps, ci = bc % comps;
    const uint64_t q = primes[l].q, w = sc.v[l], wsh = sc.sh[l];
    const size_t oo = bi * out.bstride + ci * out.cstride + (size_t)l * n;
    const size_t oa = bi * a.bstride + ci * a.cstride + (size_t)l * n;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) * 2; j < n; j += gridDim.x * blockDim.x * 2) {
        const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(a.p + oa + j);
        ulonglong2 r;
        r.x = shoup(x.x, w, wsh, q);
        r.y = shoup(x.y, w, wsh, q);
        *reinterpret_cast<ulonglong2 *>(out.p + oo + j) = r;
    }
}

// out = a with s_l added to every slot of c0 (a constant polynomial in NTT form)
__global__ void k_add_scalar_c0(View out, View a, const __grid_constant__ Scalars sc,
                                const PrimeConst *__restrict__ primes, int n)
{
    const int l = blockIdx.y, bc = blockIdx.z, bi = bc / 2, ci = bc % 2;
    const uint64_t q = primes[l].q, s = ci == 0 ? sc.v[l] : 0;
    const size_t oo = bi * out.bstride + ci * out.cstride + (size_t)l * n;
    const size_t oa = bi * a.bstride + ci * a.cstride + (size_t)l * n;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) * 2; j < n; j += gridDim.x * blockDim.x * 2) {
        const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(a.p + oa + j);
        *reinterpret_cast<ulonglong2 *>(out.p + oo + j) = make_ulonglong2(addmod(x.x, s, q), addmod(x.y, s, q));
    }
}

// (a0,a1) x (b0,b1) -> (a0b0, a0b1+a1b0, a1b1), optionally added to out; mont: each product
// left as its Montgomery reduction (times 2^-64), for sums that are brought back once at the end
// two adjacent coefficients per thread, 16-byte loads and stores
__device__ __forceinline__ void tensor_one(uint64_t a0, uint64_t a1, uint64_t b0, uint64_t b1, const PrimeConst &P,
                                           bool mont, uint64_t &r0, uint64_t &r1, uint64_t &r2)
{
    Acc128 d1;
    d1.mac(a0, b1);
    d1.mac(a1, b0);
    r0 = redc_few(__umul64hi(a0, b0), a0 * b0, P);
    r1 = redc_few(d1.hi, d1.lo, P);
    r2 = redc_few(__umul64hi(a1, b1), a1 * b1, P);
    if (!mont) {
        r0 = shoup(r0, P.r_mod, P.r_mod_sh, P.q);
        r1 = shoup(r1, P.r_mod, P.r_mod_sh, P.q);
        r2 = shoup(r2, P.r_mod, P.r_mod_sh, P.q);
    }
}

__global__ void k_tensor(View out, View a, View b, const PrimeConst *__restrict__ primes, int n, bool acc, bool mont)
{
    const int l = blockIdx.y, bi = blockIdx.z;
    const PrimeConst P = primes[l];
    const size_t la = bi * a.bstride + (size_t)l * n, lb = bi * b.bstride + (size_t)l * n;
    const size_t lo = bi * out.bstride + (size_t)l * n;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) * 2; j < n; j += gridDim.x * blockDim.x * 2) {
        const ulonglong2 a0 = *reinterpret_cast<const ulonglong2 *>(a.p + la + j);
        const ulonglong2 a1 = *reinterpret_cast<const ulonglong2 *>(a.p + la + a.cstride + j);
        const ulonglong2 b0 = *reinterpret_cast<const ulonglong2 *>(b.p + lb + j);
        const ulonglong2 b1 = *reinterpret_cast<const ulonglong2 *>(b.p + lb + b.cstride + j);
        uint64_t x0, x1, x2, y0, y1, y2;
        tensor_one(a0.x, a1.x, b0.x, b1.x, P, mont, x0, x1, x2);
        tensor_one(a0.y, a1.y, b0.y, b1.y, P, mont, y0, y1, y2);
        ulonglong2 r0 = make_ulonglong2(x0, y0), r1 = make_ulonglong2(x1, y1), r2 = make_ulonglong2(x2, y2);
        ulonglong2 *o0 = reinterpret_cast<ulonglong2 *>(out.p + lo + j);
        ulonglong2 *o1 = reinterpret_cast<ulonglong2 *>(out.p + lo + out.cstride + j);
        ulonglong2 *o2 = reinterpret_cast<ulonglong2 *>(out.p + lo + 2 * out.cstride + j);
        if (acc) {
            const ulonglong2 x0 = *o0, x1 = *o1, x2 = *o2;
            r0.x = addmod(r0.x, x0.x, P.q), r0.y = addmod(r0.y, x0.y, P.q);
            r1.x = addmod(r1.x, x1.x, P.q), r1.y = addmod(r1.y, x1.y, P.q);
            r2.x = addmod(r2.x, x2.x, P.q), r2.y = addmod(r2.y, x2.y, P.q);
        }
        *o0 = r0;
        *o1 = r1;
        *o2 = r2;
    }
}

// out = sigma_g(in) (accumulate: out += sigma_g(in), rows modulo prime index = row)
__device__ __forceinline__ void automorphism_body(const Blk &b, View out, View in, uint64_t g, int comps, int log_n,
                                                  bool accumulate, const PrimeConst *__restrict__ primes)
{
    const int n = 1 << log_n;
    const int l = b.y, bc = b.z, bi = bc / comps, ci = bc % comps;
    const size_t oo = bi * out.bstride + ci * out.cstride + (size_t)l * n;
    const size_t oi = bi * in.bstride + ci * in.cstride + (size_t)l * n;
    const uint64_t q = accumulate ? primes[l].q : 0;
    for (int j = b.x * blockDim.x + threadIdx.x; j < n; j += b.gx * blockDim.x) {
        const uint64_t v = in.p[oi + galois_src(j, g, log_n)];
        out.p[oo + j] = accumulate ? addmod(out.p[oo + j], v, q) : v;
    }
}

__global__ void k_automorphism(View out, View in, uint64_t g, int comps, int log_n, bool accumulate,
                               const PrimeConst *__restrict__ primes)
{
    automorphism_body(Blk::hw(), out, in, g, comps, log_n, accumulate, primes);
}

// Fast basis conversion; grid: x over coefficients, z = b * groups + grp (at most MK sources: register
// arrays sized to it)
template <int MK>
__device__ __forceinline__ void basis_convert_body(const Blk &b, const ConvTable *__restrict__ tabs, View out, View in,
                                                   const PrimeConst *__restrict__ primes, int groups, size_t gstride_out,
                                                   size_t gstride_in, int n)
{
    // two adjacent coefficients per thread (16-byte loads and stores); the table's constants
    // staged in shared memory once per block
    const int bz = b.z, bi = bz / groups, gi = bz % groups;
    const ConvTable &T = tabs[gi];
    __shared__ uint64_t sw[MAXK * MAXP], swsh[MAXK * MAXP];
    __shared__ uint64_t sq[MAXP], sbar[MAXP];
    __shared__ uint64_t ssq[MAXK], sinv[MAXK], sinvsh[MAXK], sadd[MAXK], ssub[MAXP], spq[MAXP];
    __shared__ double sinvd[MAXK];
    __shared__ int sdrow[MAXP], ssrow[MAXK];
    const int ns = T.n_src, nd = T.n_dst;
    const bool shift = T.shift != 0;
    for (int i = threadIdx.x; i < ns * nd; i += blockDim.x) {
        sw[i] = T.w[i / nd][i % nd];
        swsh[i] = T.w_sh[i / nd][i % nd];
    }
    for (int d = threadIdx.x; d < nd; d += blockDim.x) {
        const PrimeConst P = primes[T.dst_prime[d]];
        sq[d] = P.q;
        sbar[d] = P.bar;
        sdrow[d] = T.dst_row[d];
        ssub[d] = T.sub_dst[d];
        spq[d] = T.prod_mod[d];
    }
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
        ssq[i] = primes[T.src_prime[i]].q;
        sinv[i] = T.inv[i];
        sinvsh[i] = T.inv_sh[i];
        ssrow[i] = T.src_row[i];
        sadd[i] = T.add_src[i];
        sinvd[i] = T.inv_d[i];
    }
    __syncthreads();
    const uint64_t *src = in.p + bi * in.bstride + gi * gstride_in;
    uint64_t *dst = out.p + bi * out.bstride + gi * gstride_out;
    for (int j = (b.x * blockDim.x + threadIdx.x) * 2; j < n; j += b.gx * blockDim.x * 2) {
        uint64_t y0[MK], y1[MK];
#pragma unroll
        for (int i = 0; i < MK; i++) {
            if (i < ns) {
                ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(src + (size_t)ssrow[i] * n + j);
                if (shift) {
                    x.x = addmod(x.x, sadd[i], ssq[i]);
                    x.y = addmod(x.y, sadd[i], ssq[i]);
                }
                y0[i] = shoup(x.x, sinv[i], sinvsh[i], ssq[i]);
                y1[i] = shoup(x.y, sinv[i], sinvsh[i], ssq[i]);
            }
        }
        uint64_t u0 = 0, u1 = 0;  // overshoot of the fast conversion (shifted tables only)
        if (shift) {
            double v0 = 0.0, v1 = 0.0;  // products and sums rounded to nearest, in source order
#pragma unroll
            for (int i = 0; i < MK; i++)
                if (i < ns) {
                    v0 = __dadd_rn(v0, __dmul_rn(__ull2double_rn(y0[i]), sinvd[i]));
                    v1 = __dadd_rn(v1, __dmul_rn(__ull2double_rn(y1[i]), sinvd[i]));
                }
            u0 = __double2ull_rd(v0);
            u1 = __double2ull_rd(v1);
        }
        for (int d = 0; d < nd; d++) {
            // each term a Shoup product below 2q, the running sum kept below 2q
            const uint64_t q = sq[d], bar = sbar[d], two_q = 2 * q;
            uint64_t s0 = 0, s1 = 0;
#pragma unroll
            for (int i = 0; i < MK; i++)
                if (i < ns) {
                    const uint64_t w = sw[i * nd + d], wsh = swsh[i * nd + d];
                    s0 += shoup_lazy(y0[i], w, wsh, q);
                    s1 += shoup_lazy(y1[i], w, wsh, q);
                    if (s0 >= two_q) s0 -= two_q;
                    if (s1 >= two_q) s1 -= two_q;
                }
            ulonglong2 r;
            r.x = csub(s0, q);
            r.y = csub(s1, q);
            if (shift) {  // u <= sources - 1 <= 6, so u * (product mod q) < 2^64
                r.x = submod(submod(r.x, reduce64(u0 * spq[d], q, bar), q), ssub[d], q);
                r.y = submod(submod(r.y, reduce64(u1 * spq[d], q, bar), q), ssub[d], q);
            }
            *reinterpret_cast<ulonglong2 *>(dst + (size_t)sdrow[d] * n + j) = r;
        }
    }
}

template <int MK>  // at most MK sources (register arrays sized to it; four blocks per SM up to 4)
__global__ void __launch_bounds__(256, MK <= 4 ? 4 : 2)
    k_basis_convert(const ConvTable *__restrict__ tabs, View out, View in, const PrimeConst *__restrict__ primes,
                    int groups, size_t gstride_out, size_t gstride_in, int n)
{
    basis_convert_body<MK>(Blk::hw(), tabs, out, in, primes, groups, gstride_out, gstride_in, n);
}

// Key inner product of hybrid key switching: for ext row t (Q_l then P),
// acc_h[t] = sum_j src_j[t][galois(n)] * key[j][h][row(t)][n], where src_j is
// the NTT-form input itself on digit j's own rows and the ModUp output D_j
// elsewhere.  Keys are in Montgomery form, so one reduction gives the sum.
__device__ __forceinline__ void key_ip_body(const Blk &b, View acc, const uint64_t *__restrict__ D,
                                            const uint64_t *__restrict__ dnt, size_t dnt_bstride,
                                            const uint64_t *__restrict__ key, const PrimeConst *__restrict__ primes,
                                            int n_all, int n_q, int K, int alpha, int limbs, int ndig, uint64_t g,
                                            int log_n, bool accumulate, bool few)
{
    const int n = 1 << log_n;
    const int t = b.y, bi = b.z;
    const int ext = limbs + K;
    const int pr = t < limbs ? t : n_q + (t - limbs);
    const PrimeConst P = primes[pr];
    const size_t dig_stride = (size_t)ext * n;
    const uint64_t *Db = D + (size_t)bi * ndig * dig_stride;
    const uint64_t *db = dnt + bi * dnt_bstride;
    const int own_digit = t < limbs ? t / alpha : -1;  // digit j holds Q rows j*alpha ..
    // two adjacent outputs per thread: 16-byte key loads and stores, the sources gathered
    for (int j = (b.x * blockDim.x + threadIdx.x) * 2; j < n; j += b.gx * blockDim.x * 2) {
        const int js0 = g == 1 ? j : galois_src(j, g, log_n), js1 = g == 1 ? j + 1 : galois_src(j + 1, g, log_n);
        Acc128 a0, a1, b0, b1;
        for (int d = 0; d < ndig; d++) {
            const uint64_t *row = (d == own_digit) ? db + (size_t)t * n : Db + d * dig_stride + (size_t)t * n;
            const uint64_t x0 = row[js0], x1 = row[js1];
            const uint64_t *kd = key + (size_t)d * 2 * n_all * n + (size_t)pr * n + j;
            const ulonglong2 k0 = *reinterpret_cast<const ulonglong2 *>(kd);
            const ulonglong2 k1 = *reinterpret_cast<const ulonglong2 *>(kd + (size_t)n_all * n);
            a0.mac(x0, k0.x);
            b0.mac(x1, k0.y);
            a1.mac(x0, k1.x);
            b1.mac(x1, k1.y);
        }
        ulonglong2 r0, r1;
        if (few) {
            r0 = make_ulonglong2(redc_few(a0.hi, a0.lo, P), redc_few(b0.hi, b0.lo, P));
            r1 = make_ulonglong2(redc_few(a1.hi, a1.lo, P), redc_few(b1.hi, b1.lo, P));
        } else {
            r0 = make_ulonglong2(mont128(a0.hi, a0.lo, P), mont128(b0.hi, b0.lo, P));
            r1 = make_ulonglong2(mont128(a1.hi, a1.lo, P), mont128(b1.hi, b1.lo, P));
        }
        ulonglong2 *o0 = reinterpret_cast<ulonglong2 *>(acc.p + bi * acc.bstride + (size_t)t * n + j);
        ulonglong2 *o1 = reinterpret_cast<ulonglong2 *>(acc.p + bi * acc.bstride + acc.cstride + (size_t)t * n + j);
        if (accumulate) {
            const ulonglong2 p0 = *o0, p1 = *o1;
            r0.x = addmod(r0.x, p0.x, P.q), r0.y = addmod(r0.y, p0.y, P.q);
            r1.x = addmod(r1.x, p1.x, P.q), r1.y = addmod(r1.y, p1.y, P.q);
        }
        *o0 = r0;
        *o1 = r1;
    }
}

__global__ void k_key_ip(View acc, const uint64_t *__restrict__ D, const uint64_t *__restrict__ dnt, size_t dnt_bstride,
                         const uint64_t *__restrict__ key, const PrimeConst *__restrict__ primes, int n_all, int n_q,
                         int K, int alpha, int limbs, int ndig, uint64_t g, int log_n, bool accumulate, bool few)
{
    key_ip_body(Blk::hw(), acc, D, dnt, dnt_bstride, key, primes, n_all, n_q, K, alpha, limbs, ndig, g, log_n, accumulate,
                few);
}

// Two hoisted rotations of one ciphertext (Galois elements g1, g2) selected
// by a mask before ModDown, in the extended basis:
//   z_h[t] = c*y_h[t] + v[t]*(x_h[t] - y_h[t]),  x = <sigma_g1(D), swk1>, y = <sigma_g2(D), swk2>
// v (rows Q_l then P) is in Montgomery form; cs holds c mod each row's prime.
__global__ void k_key_ip_mux(View out, const uint64_t *__restrict__ D, const uint64_t *__restrict__ dnt,
                             size_t dnt_bstride, const uint64_t *__restrict__ key1, const uint64_t *__restrict__ key2,
                             const uint64_t *__restrict__ v, const __grid_constant__ Scalars cs,
                             const PrimeConst *__restrict__ primes, int n_all, int n_q, int K, int alpha, int limbs,
                             int ndig, uint64_t g1, uint64_t g2, int log_n, bool few)
{
    const int n = 1 << log_n;
    const int t = blockIdx.y, bi = blockIdx.z;
    const int ext = limbs + K;
    const int pr = t < limbs ? t : n_q + (t - limbs);
    const PrimeConst P = primes[pr];
    const size_t dig_stride = (size_t)ext * n;
    const uint64_t *Db = D + (size_t)bi * ndig * dig_stride;
    const uint64_t *db = dnt + bi * dnt_bstride;
    const int own_digit = t < limbs ? t / alpha : -1;  // digit j holds Q rows j*alpha ..
    const uint64_t c = cs.v[t], csh = cs.sh[t];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int j1 = galois_src(j, g1, log_n), j2 = galois_src(j, g2, log_n);
        Acc128 x0, x1, y0, y1;
        for (int d = 0; d < ndig; d++) {
            const uint64_t *row = (d == own_digit) ? db + (size_t)t * n : Db + d * dig_stride + (size_t)t * n;
            const uint64_t a = row[j1], b = row[j2];
            const size_t ko = (size_t)d * 2 * n_all * n + (size_t)pr * n + j;
            x0.mac(a, key1[ko]);
            x1.mac(a, key1[ko + (size_t)n_all * n]);
            y0.mac(b, key2[ko]);
            y1.mac(b, key2[ko + (size_t)n_all * n]);
        }
        // v holds the special primes' rows first, then the chain's (a mask of any level is a prefix)
        const uint64_t vv = v[(size_t)(t < limbs ? K + t : t - limbs) * n + j];
        const uint64_t xr0 = few ? redc_few(x0.hi, x0.lo, P) : mont128(x0.hi, x0.lo, P);
        const uint64_t yr0 = few ? redc_few(y0.hi, y0.lo, P) : mont128(y0.hi, y0.lo, P);
        const uint64_t xr1 = few ? redc_few(x1.hi, x1.lo, P) : mont128(x1.hi, x1.lo, P);
        const uint64_t yr1 = few ? redc_few(y1.hi, y1.lo, P) : mont128(y1.hi, y1.lo, P);
        const uint64_t d0 = submod(xr0, yr0, P.q), d1 = submod(xr1, yr1, P.q);
        const uint64_t z0 = addmod(shoup(yr0, c, csh, P.q), redc_few(__umul64hi(vv, d0), vv * d0, P), P.q);
        const uint64_t z1 = addmod(shoup(yr1, c, csh, P.q), redc_few(__umul64hi(vv, d1), vv * d1, P), P.q);
        out.p[bi * out.bstride + (size_t)t * n + j] = z0;
        out.p[bi * out.bstride + out.cstride + (size_t)t * n + j] = z1;
    }
}

// premasked keys: rows t of the extended basis (Q_l then P), digits d < ndig
__global__ void k_premask_keys(uint64_t *out, const uint64_t *__restrict__ key1, const uint64_t *__restrict__ key2,
                               const uint64_t *__restrict__ v, const __grid_constant__ Scalars cR,
                               const PrimeConst *__restrict__ primes, int n_all, int n_q, int K, int limbs, int ndig,
                               int n)
{
    const int t = blockIdx.y, dh = blockIdx.z, d = dh / 2, h = dh % 2;
    const int ext = limbs + K;
    const int pr = t < limbs ? t : n_q + (t - limbs);
    const PrimeConst P = primes[pr];
    const size_t ko = ((size_t)d * 2 + h) * n_all * n + (size_t)pr * n;
    uint64_t *o1 = out + (((size_t)d * 2 + h) * ext + t) * n;
    uint64_t *o2 = o1 + (size_t)ndig * 2 * ext * n;
    const uint64_t cr = cR.v[t];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        // v: the special primes' rows first, then the chain's
        const uint64_t vv = v[(size_t)(t < limbs ? K + t : t - limbs) * n + j], k1 = key1[ko + j], k2 = key2[ko + j];
        const uint64_t w = submod(cr, vv, P.q);  // (c - v) in Montgomery form
        o1[j] = redc_few(__umul64hi(vv, k1), vv * k1, P);
        o2[j] = redc_few(__umul64hi(w, k2), w * k2, P);
    }
}

__global__ void k_key_ip_mux_pm(View out, const uint64_t *__restrict__ D, const uint64_t *__restrict__ dnt,
                                size_t dnt_bstride, const uint64_t *__restrict__ pk,
                                const PrimeConst *__restrict__ primes, int n_q, int K, int alpha, int limbs, int ndig,
                                uint64_t g1, uint64_t g2, int log_n, bool few)
{
    const int n = 1 << log_n;
    const int t = blockIdx.y, bi = blockIdx.z;
    const int ext = limbs + K;
    const int pr = t < limbs ? t : n_q + (t - limbs);
    const PrimeConst P = primes[pr];
    const size_t dig_stride = (size_t)ext * n;
    const uint64_t *Db = D + (size_t)bi * ndig * dig_stride;
    const uint64_t *db = dnt + bi * dnt_bstride;
    const int own_digit = t < limbs ? t / alpha : -1;  // digit j holds Q rows j*alpha ..
    const size_t half = (size_t)ndig * 2 * ext * n;
    // two adjacent outputs per thread: 16-byte key loads and stores, the sources gathered
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) * 2; j < n; j += gridDim.x * blockDim.x * 2) {
        const int j1a = galois_src(j, g1, log_n), j2a = galois_src(j, g2, log_n);
        const int j1b = galois_src(j + 1, g1, log_n), j2b = galois_src(j + 1, g2, log_n);
        Acc128 z0a, z1a, z0b, z1b;
        for (int d = 0; d < ndig; d++) {
            const uint64_t *row = (d == own_digit) ? db + (size_t)t * n : Db + d * dig_stride + (size_t)t * n;
            const uint64_t xa = row[j1a], ya = row[j2a], xb = row[j1b], yb = row[j2b];
            const size_t o = ((size_t)d * 2 * ext + t) * n + j;
            const ulonglong2 p0 = *reinterpret_cast<const ulonglong2 *>(pk + o);
            const ulonglong2 q0 = *reinterpret_cast<const ulonglong2 *>(pk + half + o);
            const ulonglong2 p1 = *reinterpret_cast<const ulonglong2 *>(pk + o + dig_stride);
            const ulonglong2 q1 = *reinterpret_cast<const ulonglong2 *>(pk + half + o + dig_stride);
            z0a.mac(xa, p0.x);
            z0a.mac(ya, q0.x);
            z1a.mac(xa, p1.x);
            z1a.mac(ya, q1.x);
            z0b.mac(xb, p0.y);
            z0b.mac(yb, q0.y);
            z1b.mac(xb, p1.y);
            z1b.mac(yb, q1.y);
        }
        ulonglong2 r0, r1;
        if (few) {
            r0 = make_ulonglong2(redc_few(z0a.hi, z0a.lo, P), redc_few(z0b.hi, z0b.lo, P));
            r1 = make_ulonglong2(redc_few(z1a.hi, z1a.lo, P), redc_few(z1b.hi, z1b.lo, P));
        } else {
            r0 = make_ulonglong2(mont128(z0a.hi, z0a.lo, P), mont128(z0b.hi, z0b.lo, P));
            r1 = make_ulonglong2(mont128(z1a.hi, z1a.lo, P), mont128(z1b.hi, z1b.lo, P));
        }
        *reinterpret_cast<ulonglong2 *>(out.p + bi * out.bstride + (size_t)t * n + j) = r0;
        *reinterpret_cast<ulonglong2 *>(out.p + bi * out.bstride + out.cstride + (size_t)t * n + j) = r1;
    }
}

// ALU calibration: chains of Shoup products (the NTT butterfly's multiplication)
// and of 64x64 -> 128-bit multiply-accumulates (the key inner product's), eight
// independent chains per thread, every SM busy; the results are written so the
// work is kept.
__global__ void k_calib_shoup(uint64_t *out, int iters, uint64_t q, uint64_t w, uint64_t wsh)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t y[8];
#pragma unroll
    for (int c = 0; c < 8; c++) y[c] = (uint64_t)t * 8 + c;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < 8; c++) y[c] = shoup_lazy(y[c], w, wsh, q) + (uint64_t)c;
    }
    uint64_t x = 0;
#pragma unroll
    for (int c = 0; c < 8; c++) x ^= y[c];
    out[t] = x;
}

__global__ void k_calib_mac(uint64_t *out, int iters, uint64_t k0, uint64_t k1)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t x[8];
    Acc128 acc[8];
#pragma unroll
    for (int c = 0; c < 8; c++) x[c] = (uint64_t)t * 8 + c + 1;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < 8; c++) {
            acc[c].mac(x[c], (i & 1) ? k1 : k0);
            x[c] ^= acc[c].lo >> 7;
        }
    }
    uint64_t r = 0;
#pragma unroll
    for (int c = 0; c < 8; c++) r ^= acc[c].lo ^ acc[c].hi;
    out[t] = r;
}

// ModDown epilogue of k_key_ip_mux: out_h = (z_h - conv_h) * P^-1, plus for h = 0
// c*sigma_g2(c0) + v*(sigma_g1(c0) - sigma_g2(c0))
__global__ void k_moddown_final_mux(View out, View acc, View conv, const ModDownTable *__restrict__ tab,
                                    const PrimeConst *__restrict__ primes, View src, const uint64_t *__restrict__ v,
                                    const __grid_constant__ Scalars cs, uint64_t g1, uint64_t g2, int log_n)
{
    const int n = 1 << log_n;
    const int t = blockIdx.y, bc = blockIdx.z, bi = bc / 2, ci = bc % 2;
    const PrimeConst P = primes[t];
    const uint64_t q = P.q, w = tab->pinv[t], wsh = tab->pinv_sh[t];
    const uint64_t *a = acc.p + bi * acc.bstride + ci * acc.cstride + (size_t)t * n;
    const uint64_t *cv = conv.p + bi * conv.bstride + ci * conv.cstride + (size_t)t * n;
    uint64_t *o = out.p + bi * out.bstride + ci * out.cstride + (size_t)t * n;
    const uint64_t *c0 = src.p + bi * src.bstride + (size_t)t * n;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) * 2; j < n; j += gridDim.x * blockDim.x * 2) {
        const ulonglong2 av = *reinterpret_cast<const ulonglong2 *>(a + j);
        const ulonglong2 cw = *reinterpret_cast<const ulonglong2 *>(cv + j);
        uint64_t r[2] = {shoup(submod(av.x, cw.x, q), w, wsh, q), shoup(submod(av.y, cw.y, q), w, wsh, q)};
        if (ci == 0) {
            const ulonglong2 vv2 = *reinterpret_cast<const ulonglong2 *>(v + (size_t)t * n + j);
            const uint64_t vs[2] = {vv2.x, vv2.y};
#pragma unroll
            for (int u = 0; u < 2; u++) {
                const uint64_t s1 = c0[galois_src(j + u, g1, log_n)], s2 = c0[galois_src(j + u, g2, log_n)];
                const uint64_t d = submod(s1, s2, q);
                const uint64_t sel =
                    addmod(shoup(s2, cs.v[t], cs.sh[t], q), redc_few(__umul64hi(vs[u], d), vs[u] * d, P), q);
                r[u] = addmod(r[u], sel, q);
            }
        }
        *reinterpret_cast<ulonglong2 *>(o + j) = make_ulonglong2(r[0], r[1]);
    }
}

// out_c[t] = (acc_c[t] - conv_c[t]) * P^-1 (+ add_c[t][galois(j)] for the components in add_mask)
__device__ __forceinline__ void moddown_final_body(const Blk &b, View out, View acc, View conv,
                                                   const ModDownTable *__restrict__ tab,
                                                   const PrimeConst *__restrict__ primes, View add, int add_mask,
                                                   uint64_t g, int log_n)
{
    const int n = 1 << log_n;
    const int t = b.y, bc = b.z, bi = bc / 2, ci = bc % 2;
    const uint64_t q = primes[t].q, w = tab->pinv[t], wsh = tab->pinv_sh[t];
    const uint64_t *a = acc.p + bi * acc.bstride + ci * acc.cstride + (size_t)t * n;
    const uint64_t *cv = conv.p + bi * conv.bstride + ci * conv.cstride + (size_t)t * n;
    uint64_t *o = out.p + bi * out.bstride + ci * out.cstride + (size_t)t * n;
    const bool has = (add_mask >> ci) & 1;
    const uint64_t *ap = has ? add.p + bi * add.bstride + ci * add.cstride + (size_t)t * n : nullptr;
    for (int j = (b.x * blockDim.x + threadIdx.x) * 2; j < n; j += b.gx * blockDim.x * 2) {
        const ulonglong2 av = *reinterpret_cast<const ulonglong2 *>(a + j);
        const ulonglong2 cw = *reinterpret_cast<const ulonglong2 *>(cv + j);
        ulonglong2 r;
        r.x = shoup(submod(av.x, cw.x, q), w, wsh, q);
        r.y = shoup(submod(av.y, cw.y, q), w, wsh, q);
        if (has) {
            if (g == 1) {
                const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(ap + j);
                r.x = addmod(r.x, x.x, q);
                r.y = addmod(r.y, x.y, q);
            } else {
                r.x = addmod(r.x, ap[galois_src(j, g, log_n)], q);
                r.y = addmod(r.y, ap[galois_src(j + 1, g, log_n)], q);
            }
        }
        *reinterpret_cast<ulonglong2 *>(o + j) = r;
    }
}

__global__ void k_moddown_final(View out, View acc, View conv, const ModDownTable *__restrict__ tab,
                                const PrimeConst *__restrict__ primes, View add, int add_mask, uint64_t g, int log_n)
{
    moddown_final_body(Blk::hw(), out, acc, conv, tab, primes, add, add_mask, g, log_n);
}

// r_i = ([x + floor(q_t/2)]_{q_t} mod q_i - floor(q_t/2) mod q_i) for the lower limbs
__global__ void k_rescale_prep(View r, View xtop, const RescaleTable *__restrict__ tab,
                               const PrimeConst *__restrict__ primes, int comps, int top, int n,
                               const __grid_constant__ Scalars sc, bool scaled)
{
    const int i = blockIdx.y, bc = blockIdx.z, bi = bc / comps, ci = bc % comps;
    const uint64_t qt = primes[top].q, half = tab->half;
    const PrimeConst Pi = primes[i];
    const uint64_t hm = tab->half_mod[i];
    const uint64_t *x = xtop.p + bi * xtop.bstride + ci * xtop.cstride;
    uint64_t *o = r.p + bi * r.bstride + ci * r.cstride + (size_t)i * n;
    // two adjacent coefficients per thread (16-byte loads and stores)
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) * 2; j < n; j += gridDim.x * blockDim.x * 2) {
        ulonglong2 xv = *reinterpret_cast<const ulonglong2 *>(x + j);
        if (scaled) {  // the input times an integer: the inverse NTT is linear, so scale its output
            xv.x = shoup(xv.x, sc.v[top], sc.sh[top], qt);
            xv.y = shoup(xv.y, sc.v[top], sc.sh[top], qt);
        }
        const uint64_t v0 = csub(xv.x + half, qt), v1 = csub(xv.y + half, qt);
        *reinterpret_cast<ulonglong2 *>(o + j) = make_ulonglong2(submod(reduce64(v0, Pi.q, Pi.bar), hm, Pi.q),
                                                                 submod(reduce64(v1, Pi.q, Pi.bar), hm, Pi.q));
    }
}

__global__ void k_rescale_final(View out, View in, View r, const RescaleTable *__restrict__ tab,
                                const PrimeConst *__restrict__ primes, int comps, int n,
                                const __grid_constant__ Scalars sc, bool scaled)
{
    const int i = blockIdx.y, bc = blockIdx.z, bi = bc / comps, ci = bc % comps;
    const uint64_t q = primes[i].q, w = tab->qinv[i], wsh = tab->qinv_sh[i];
    const uint64_t *a = in.p + bi * in.bstride + ci * in.cstride + (size_t)i * n;
    const uint64_t *rr = r.p + bi * r.bstride + ci * r.cstride + (size_t)i * n;
    uint64_t *o = out.p + bi * out.bstride + ci * out.cstride + (size_t)i * n;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) * 2; j < n; j += gridDim.x * blockDim.x * 2) {
        ulonglong2 av = *reinterpret_cast<const ulonglong2 *>(a + j);
        if (scaled) {
            av.x = shoup(av.x, sc.v[i], sc.sh[i], q);
            av.y = shoup(av.y, sc.v[i], sc.sh[i], q);
        }
        const ulonglong2 rv = *reinterpret_cast<const ulonglong2 *>(rr + j);
        *reinterpret_cast<ulonglong2 *>(o + j) =
            make_ulonglong2(shoup(submod(av.x, rv.x, q), w, wsh, q), shoup(submod(av.y, rv.y, q), w, wsh, q));
    }
}

// Relinearisation + rescale (division by P q_top).  Row l-1 (q_top) of each key-switched
// component becomes y = acc + (P mod q_top) d, the value the conversion reads there.
__global__ void k_relin_rs_top(View acc, View d, const RelinRescaleTable *__restrict__ tab,
                               const PrimeConst *__restrict__ primes, int top, int n)
{
    const int bc = blockIdx.z, bi = bc / 2, ci = bc % 2;
    const uint64_t q = primes[top].q, w = tab->pmod[top], wsh = tab->pmod_sh[top];
    uint64_t *a = acc.p + bi * acc.bstride + ci * acc.cstride + (size_t)top * n;
    const uint64_t *x = d.p + bi * d.bstride + ci * d.cstride + (size_t)top * n;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) * 2; j < n; j += gridDim.x * blockDim.x * 2) {
        const ulonglong2 av = *reinterpret_cast<const ulonglong2 *>(a + j);
        const ulonglong2 xv = *reinterpret_cast<const ulonglong2 *>(x + j);
        *reinterpret_cast<ulonglong2 *>(a + j) =
            make_ulonglong2(addmod(av.x, shoup(xv.x, w, wsh, q), q), addmod(av.y, shoup(xv.y, w, wsh, q), q));
    }
}

// out_i = (acc_i + P d_i - r_i) (P q_top)^-1 on the l-1 lower rows, r the converted remainder
__global__ void k_relin_rs_final(View out, View acc, View d, View conv, const RelinRescaleTable *__restrict__ tab,
                                 const PrimeConst *__restrict__ primes, int n)
{
    const int i = blockIdx.y, bc = blockIdx.z, bi = bc / 2, ci = bc % 2;
    const uint64_t q = primes[i].q, pm = tab->pmod[i], pmsh = tab->pmod_sh[i];
    const uint64_t w = tab->pqinv[i], wsh = tab->pqinv_sh[i];
    const size_t row = (size_t)i * n;
    const uint64_t *a = acc.p + bi * acc.bstride + ci * acc.cstride + row;
    const uint64_t *x = d.p + bi * d.bstride + ci * d.cstride + row;
    const uint64_t *r = conv.p + bi * conv.bstride + ci * conv.cstride + row;
    uint64_t *o = out.p + bi * out.bstride + ci * out.cstride + row;
    for (int j = (blockIdx.x * blockDim.x + threadIdx.x) * 2; j < n; j += gridDim.x * blockDim.x * 2) {
        const ulonglong2 av = *reinterpret_cast<const ulonglong2 *>(a + j);
        const ulonglong2 xv = *reinterpret_cast<const ulonglong2 *>(x + j);
        const ulonglong2 rv = *reinterpret_cast<const ulonglong2 *>(r + j);
        const uint64_t y0 = addmod(av.x, shoup(xv.x, pm, pmsh, q), q), y1 = addmod(av.y, shoup(xv.y, pm, pmsh, q), q);
        *reinterpret_cast<ulonglong2 *>(o + j) =
            make_ulonglong2(shoup(submod(y0, rv.x, q), w, wsh, q), shoup(submod(y1, rv.y, q), w, wsh, q));
    }
}

__global__ void k_expand_masks(double *slots, const uint8_t *__restrict__ bits, int hh, int beta, size_t S)
{
    const int r = blockIdx.y;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < S; i += (size_t)gridDim.x * blockDim.x)
        slots[(size_t)r * S + i] = (double)bits[(size_t)r * hh + i / beta];
}

// b = e - a*s + gad_r * s'  (all NTT form, row r modulo prime r); optionally
// b and a are left in Montgomery form for the key inner product.
__global__ void k_keygen_b(uint64_t *b, uint64_t *a, const uint64_t *e, const uint64_t *s, const uint64_t *sp,
                           const uint64_t *gad, const PrimeConst *__restrict__ primes, int n, bool to_mont)
{
    const int r = blockIdx.y;
    const PrimeConst P = primes[r];
    const uint64_t gr = gad ? gad[r] : 0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const size_t k = (size_t)r * n + j;
        uint64_t v = submod(e[k], mulmod(a[k], s[k], P), P.q);
        if (gr) v = addmod(v, mulmod(gr, sp[k], P), P.q);
        if (to_mont) {
            v = shoup(v, P.r_mod, P.r_mod_sh, P.q);
            a[k] = shoup(a[k], P.r_mod, P.r_mod_sh, P.q);
        }
        b[k] = v;
    }
}

// c0 = v*pk_b + e0 + m, c1 = v*pk_a + e1 on the first `limbs` primes
__global__ void k_encrypt_combine(uint64_t *ct, const uint64_t *v, const uint64_t *e0, const uint64_t *e1,
                                  const uint64_t *m, const uint64_t *pk, const PrimeConst *__restrict__ primes,
                                  int n_q, int limbs, int n)
{
    const int l = blockIdx.y;
    const PrimeConst P = primes[l];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const size_t k = (size_t)l * n + j;
        const uint64_t vb = mulmod(v[k], pk[k], P);
        const uint64_t va = mulmod(v[k], pk[(size_t)n_q * n + k], P);
        ct[k] = addmod(addmod(vb, e0[k], P.q), m[k], P.q);
        ct[(size_t)limbs * n + k] = addmod(va, e1[k], P.q);
    }
}

// signed coefficients -> residues: out[p][r][j] = in[p][j] mod q_{prime[r]}
__global__ void k_signed_to_rows(uint64_t *out, const int64_t *in, int rows, size_t in_stride, const int *prime,
                                 const PrimeConst *__restrict__ primes, int n)
{
    const int r = blockIdx.y, p = blockIdx.z;
    const uint64_t q = primes[prime[r]].q;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int64_t v = in[p * in_stride + j];
        const uint64_t m = v >= 0 ? (uint64_t)v % q : (q - ((uint64_t)(-v) % q)) % q;
        out[((size_t)p * rows + r) * n + j] = m;
    }
}

__global__ void k_to_mont(uint64_t *p, const int *prime, const PrimeConst *__restrict__ primes, int n)
{
    const int r = blockIdx.y;
    const PrimeConst P = primes[prime[r]];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const size_t k = (size_t)r * n + j;
        p[k] = shoup(p[k], P.r_mod, P.r_mod_sh, P.q);
    }
}

__global__ void k_mul_rows(uint64_t *out, const uint64_t *a, const uint64_t *b, const PrimeConst *__restrict__ primes,
                           int n)
{
    const int r = blockIdx.y;
    const PrimeConst P = primes[r];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const size_t k = (size_t)r * n + j;
        out[k] = mulmod(a[k], b[k], P);
    }
}

__global__ void k_ddec_shares(uint64_t *out, View ct, const uint64_t *shares, const PrimeConst *__restrict__ primes,
                              int np, int n)
{
    const int p = blockIdx.y, bi = blockIdx.z;
    const PrimeConst P = primes[0];
    const uint64_t *c0 = ct.p + bi * ct.bstride;
    const uint64_t *c1 = c0 + ct.cstride;
    uint64_t *o = out + ((size_t)bi * (np + 1) + p) * n;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        o[j] = p == 0 ? c0[j] : mulmod(c1[j], shares[(size_t)(p - 1) * n + j], P);
}

// ---- several rings in one launch per key-switching stage ----------------------------------------
// The job of flat block bid: the last whose block0 <= bid (block0 ascending, the first 0); b gets
// the coordinates that job's own grid gives the block.
template <class J>
__device__ __forceinline__ const J &job_of_block(const J *__restrict__ jobs, int n_jobs, long long bid, Blk &b)
{
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].block0 <= bid) lo = mid;
        else hi = mid - 1;
    }
    const J &j = jobs[lo];
    const long long local = bid - j.block0, plane = (long long)j.gx * j.gy;
    b = Blk{(int)(local % j.gx), (int)((local / j.gx) % j.gy), (int)(local / plane), j.gx, j.gy, j.gz};
    return j;
}

__global__ void k_automorphism_jobs(const AutomorphismJob *__restrict__ jobs, int n_jobs)
{
    Blk b;
    const AutomorphismJob &J = job_of_block(jobs, n_jobs, blockIdx.x, b);
    automorphism_body(b, J.out, J.in, J.g, J.comps, J.log_n, false, J.primes);
}

template <int MK>
__global__ void __launch_bounds__(256, MK <= 4 ? 4 : 2) k_convert_jobs(const ConvertJob *__restrict__ jobs, int n_jobs)
{
    Blk b;
    const ConvertJob &J = job_of_block(jobs, n_jobs, blockIdx.x, b);
    basis_convert_body<MK>(b, J.tabs, J.out, J.in, J.primes, J.groups, J.gstride_out, J.gstride_in, J.n);
}

__global__ void k_key_ip_jobs(const KeyIpJob *__restrict__ jobs, int n_jobs)
{
    Blk b;
    const KeyIpJob &J = job_of_block(jobs, n_jobs, blockIdx.x, b);
    key_ip_body(b, J.acc, J.D, J.dnt, J.dnt_bstride, J.key, J.primes, J.n_all, J.n_q, J.K, J.alpha, J.limbs, J.ndig,
                J.g, J.log_n, false, J.few != 0);
}

__global__ void k_moddown_jobs(const ModDownJob *__restrict__ jobs, int n_jobs)
{
    Blk b;
    const ModDownJob &J = job_of_block(jobs, n_jobs, blockIdx.x, b);
    moddown_final_body(b, J.out, J.acc, J.conv, J.tab, J.primes, J.add, J.add_mask, J.g, J.log_n);
}

} // namespace

const char *const kclass_names[K_NCLASS] = {"ntt", "key_inner_product", "basis_convert", "moddown_final",
                                            "rescale", "tensor", "mul_plain", "add_sub_copy", "automorphism",
                                            "aggregate", "other"};

cudaEvent_t Profiler::get()
{
    if (pool.empty()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
}

void Profiler::clear()
{
    for (auto &r : recs) {
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    recs.clear();
}

void launch_add(const LaunchCtx &c, View out, View a, View b, int B, int comps, int limbs, bool sub)
{
    Timed tm_(c, K_ELEM, 24.0 * B * comps * limbs * c.N);
    dim3 grid(ew_blocks(c.N, 2), limbs, B * comps);
    k_add<<<grid, 256, 0, c.stream>>>(out, a, b, c.t->primes, comps, c.N, sub);
    post(c);
}

void launch_copy(const LaunchCtx &c, View out, View a, int B, int comps, int limbs)
{
    Timed tm_(c, K_ELEM, 16.0 * B * comps * limbs * c.N);
    dim3 grid(ew_blocks(c.N, 2), limbs, B * comps);
    k_copy<<<grid, 256, 0, c.stream>>>(out, a, comps, c.N);
    post(c);
}

void launch_aggregate(const LaunchCtx &c, View out, const AggSrc *src_dev, int n_parties, int count, int comps,
                      int limbs, const Scalars &C)
{
    Timed tm_(c, K_AGG, 8.0 * (n_parties + 1.0) * count * comps * limbs * c.N);
    HX_CHECK(count * comps < 65536 && limbs < 65536, HX_EINVAL, "aggregation batch too large");
    dim3 grid(ew_blocks(c.N, 2), limbs, count * comps);
    k_aggregate<<<grid, 256, 0, c.stream>>>(out, src_dev, n_parties, count, C, c.t->primes, comps, c.N);
    post(c);
}

void launch_mul_plain(const LaunchCtx &c, View out, View a, const uint64_t *pt, int B, int limbs)
{
    Timed tm_(c, K_MULPT, 8.0 * (4 * B + 1) * limbs * c.N);
    dim3 grid(ew_blocks(c.N, 2), limbs, B * 2);
    k_mul_plain<<<grid, 256, 0, c.stream>>>(out, a, pt, c.t->primes, c.N);
    post(c);
}

void launch_mul_scalar(const LaunchCtx &c, View out, View a, const Scalars &sc, int B, int comps, int limbs)
{
    Timed tm_(c, K_ELEM, 16.0 * B * comps * limbs * c.N);
    dim3 grid(ew_blocks(c.N, 2), limbs, B * comps);
    k_mul_scalar<<<grid, 256, 0, c.stream>>>(out, a, sc, c.t->primes, comps, c.N);
    post(c);
}

void launch_add_scalar_c0(const LaunchCtx &c, View out, View a, const Scalars &sc, int B, int limbs)
{
    Timed tm_(c, K_ELEM, 32.0 * B * limbs * c.N);
    dim3 grid(ew_blocks(c.N, 2), limbs, B * 2);
    k_add_scalar_c0<<<grid, 256, 0, c.stream>>>(out, a, sc, c.t->primes, c.N);
    post(c);
}

void launch_tensor(const LaunchCtx &c, View out3, View a, View b, int B, int limbs, bool accumulate, bool mont)
{
    Timed tm_(c, K_TENSOR, 8.0 * B * limbs * c.N * (accumulate ? 10 : 7));
    dim3 grid(ew_blocks(c.N, 2), limbs, B);
    k_tensor<<<grid, 256, 0, c.stream>>>(out3, a, b, c.t->primes, c.N, accumulate, mont);
    post(c);
}

void launch_automorphism(const LaunchCtx &c, View out, View in, uint64_t g, int B, int comps, int limbs,
                         bool accumulate)
{
    Timed tm_(c, K_AUTO, (accumulate ? 24.0 : 16.0) * B * comps * limbs * c.N);
    dim3 grid(ew_blocks(c.N, 1), limbs, B * comps);
    k_automorphism<<<grid, 256, 0, c.stream>>>(out, in, g, comps, c.log_n, accumulate, c.t->primes);
    post(c);
}

void launch_basis_convert(const LaunchCtx &c, const ConvTable *tab_dev, int max_src, View out, View in, int B,
                          int groups, size_t gstride_out, size_t gstride_in, double alg_bytes)
{
    Timed tm_(c, K_CONV, alg_bytes);
    HX_CHECK(B * groups < 65536, HX_EINVAL, "conversion batch too large");
    HX_CHECK(max_src >= 1 && max_src <= MAXK, HX_EINVAL, "too many conversion sources");
    dim3 grid(ew_blocks(c.N, 2), 1, B * groups);
    if (max_src <= 4)
        k_basis_convert<4><<<grid, 256, 0, c.stream>>>(tab_dev, out, in, c.t->primes, groups, gstride_out, gstride_in,
                                                       c.N);
    else
        k_basis_convert<MAXK><<<grid, 256, 0, c.stream>>>(tab_dev, out, in, c.t->primes, groups, gstride_out,
                                                          gstride_in, c.N);
    post(c);
}

void launch_key_ip(const LaunchCtx &c, View acc, const uint64_t *D, const uint64_t *dnt, size_t dnt_bstride,
                   const uint64_t *key, int n_all, int n_q, int K, int alpha, int limbs, int ndig, uint64_t g, int B,
                   bool accumulate)
{
    Timed tm_(c, K_KEYIP, 8.0 * c.N * ((double)B * ndig * (limbs + K) + 2.0 * ndig * (limbs + K) + 2.0 * B * (limbs + K)));
    dim3 grid(ew_blocks(c.N, 2), limbs + K, B);
    k_key_ip<<<grid, 256, 0, c.stream>>>(acc, D, dnt, dnt_bstride, key, c.t->primes, n_all, n_q, K, alpha, limbs, ndig, g,
                                         c.log_n, accumulate, ndig <= kRedcFewTerms);
    post(c);
}

void launch_lintrans_mac(const LaunchCtx &c, const MacArgs &a, int B, int limbs, int n_terms)
{
    Timed tm_(c, K_MULPT, 8.0 * limbs * c.N * ((double)B * 2 * (a.n_baby + a.n_group) + n_terms));
    HX_CHECK(B >= 1 && limbs < 65536, HX_EINVAL, "bad BSGS batch");
    dim3 grid(B, (c.N / 2 + 127) / 128, limbs);
    if (a.n_baby <= 4) k_lintrans_mac<4><<<grid, 128, 0, c.stream>>>(a, c.t->primes, B, limbs, c.N);
    else if (a.n_baby <= 8) k_lintrans_mac<8><<<grid, 128, 0, c.stream>>>(a, c.t->primes, B, limbs, c.N);
    else k_lintrans_mac<16><<<grid, 128, 0, c.stream>>>(a, c.t->primes, B, limbs, c.N);
    post(c);
}

void launch_key_ip_mux(const LaunchCtx &c, View out, const uint64_t *D, const uint64_t *dnt, size_t dnt_bstride,
                       const uint64_t *key1, const uint64_t *key2, const uint64_t *v, const Scalars &cs, int n_all,
                       int n_q, int K, int alpha, int limbs, int ndig, uint64_t g1, uint64_t g2, int B)
{
    Timed tm_(c, K_KEYIP, 8.0 * c.N * ((double)B * ndig * (limbs + K) + 4.0 * ndig * (limbs + K) + (limbs + K) +
                                        2.0 * B * (limbs + K)));
    dim3 grid(ew_blocks(c.N, 1), limbs + K, B);
    k_key_ip_mux<<<grid, 256, 0, c.stream>>>(out, D, dnt, dnt_bstride, key1, key2, v, cs, c.t->primes, n_all, n_q, K,
                                             alpha, limbs, ndig, g1, g2, c.log_n, ndig <= kRedcFewTerms);
    post(c);
}

void launch_premask_keys(const LaunchCtx &c, uint64_t *out, const uint64_t *key1, const uint64_t *key2,
                         const uint64_t *v, const Scalars &cR, int n_all, int n_q, int K, int limbs, int ndig)
{
    dim3 grid(ew_blocks(c.N, 1), limbs + K, ndig * 2);
    k_premask_keys<<<grid, 256, 0, c.stream>>>(out, key1, key2, v, cR, c.t->primes, n_all, n_q, K, limbs, ndig, c.N);
    post(c);
}

void launch_key_ip_mux_pm(const LaunchCtx &c, View out, const uint64_t *D, const uint64_t *dnt, size_t dnt_bstride,
                          const uint64_t *pk, int n_q, int K, int alpha, int limbs, int ndig, uint64_t g1, uint64_t g2,
                          int B)
{
    Timed tm_(c, K_KEYIP, 8.0 * c.N * ((double)B * ndig * (limbs + K) + 4.0 * ndig * (limbs + K) +
                                        2.0 * B * (limbs + K)));
    dim3 grid(ew_blocks(c.N, 2), limbs + K, B);
    k_key_ip_mux_pm<<<grid, 256, 0, c.stream>>>(out, D, dnt, dnt_bstride, pk, c.t->primes, n_q, K, alpha, limbs, ndig, g1, g2,
                                                c.log_n, 2 * ndig <= kRedcFewTerms);
    post(c);
}

void alu_calibrate(const LaunchCtx &c, uint64_t q, double *shoup_per_s, double *mac_per_s)
{
    const int blocks = c.t->n_sm * 8, threads = 256, iters = 1024;
    uint64_t *buf = nullptr;
    HX_CUDA(cudaMallocAsync(&buf, sizeof(uint64_t) * blocks * threads, c.stream));
    cudaEvent_t e[3];
    for (auto &x : e) HX_CUDA(cudaEventCreate(&x));
    const uint64_t w = (q >> 1) | 1, wsh = (uint64_t)(((unsigned __int128)w << 64) / q);
    k_calib_shoup<<<blocks, threads, 0, c.stream>>>(buf, 16, q, w, wsh);  // warm-up
    k_calib_mac<<<blocks, threads, 0, c.stream>>>(buf, 16, w, wsh);
    HX_CUDA(cudaEventRecord(e[0], c.stream));
    k_calib_shoup<<<blocks, threads, 0, c.stream>>>(buf, iters, q, w, wsh);
    HX_CUDA(cudaEventRecord(e[1], c.stream));
    k_calib_mac<<<blocks, threads, 0, c.stream>>>(buf, iters, w, wsh);
    HX_CUDA(cudaEventRecord(e[2], c.stream));
    HX_CUDA(cudaEventSynchronize(e[2]));
    float ms1 = 0, ms2 = 0;
    HX_CUDA(cudaEventElapsedTime(&ms1, e[0], e[1]));
    HX_CUDA(cudaEventElapsedTime(&ms2, e[1], e[2]));
    for (auto &x : e) cudaEventDestroy(x);
    HX_CUDA(cudaFreeAsync(buf, c.stream));
    const double ops = 8.0 * blocks * threads * iters;
    *shoup_per_s = ops / (ms1 * 1e-3);
    *mac_per_s = ops / (ms2 * 1e-3);
}

void launch_moddown_final_mux(const LaunchCtx &c, View out, View acc, View conv, const ModDownTable *tab, int B,
                              int limbs, View src, const uint64_t *v, const Scalars &cs, uint64_t g1, uint64_t g2)
{
    Timed tm_(c, K_MODDOWN, 8.0 * B * limbs * c.N * 9.0);
    dim3 grid(ew_blocks(c.N, 2), limbs, B * 2);
    k_moddown_final_mux<<<grid, 256, 0, c.stream>>>(out, acc, conv, tab, c.t->primes, src, v, cs, g1, g2, c.log_n);
    post(c);
}

void launch_moddown_final(const LaunchCtx &c, View out, View acc, View conv, const ModDownTable *tab, int B,
                          int limbs, View add, int add_mask, uint64_t g)
{
    Timed tm_(c, K_MODDOWN, 8.0 * B * 2 * limbs * c.N * ((add_mask ? 4.0 : 3.0)));
    dim3 grid(ew_blocks(c.N, 2), limbs, B * 2);
    k_moddown_final<<<grid, 256, 0, c.stream>>>(out, acc, conv, tab, c.t->primes, add, add_mask, g, c.log_n);
    post(c);
}

void launch_expand_masks(const LaunchCtx &c, double *slots, const uint8_t *bits, int m, int hh, int beta, size_t S)
{
    HX_CHECK(m >= 1 && m < 65536 && (size_t)hh * beta == S, HX_EINVAL, "bad mask expansion");
    dim3 grid((unsigned)std::min<size_t>((S + 255) / 256, 4096), m, 1);
    k_expand_masks<<<grid, 256, 0, c.stream>>>(slots, bits, hh, beta, S);
    post(c);
}

void launch_relin_rs_top(const LaunchCtx &c, View acc, View d, const RelinRescaleTable *tab, int B, int limbs)
{
    Timed tm_(c, K_RESCALE, 24.0 * B * 2 * c.N);
    dim3 grid(ew_blocks(c.N, 2), 1, B * 2);
    k_relin_rs_top<<<grid, 256, 0, c.stream>>>(acc, d, tab, c.t->primes, limbs - 1, c.N);
    post(c);
}

void launch_relin_rs_final(const LaunchCtx &c, View out, View acc, View d, View conv, const RelinRescaleTable *tab,
                           int B, int limbs)
{
    Timed tm_(c, K_MODDOWN, 32.0 * B * 2 * (limbs - 1) * c.N);
    dim3 grid(ew_blocks(c.N, 2), limbs - 1, B * 2);
    k_relin_rs_final<<<grid, 256, 0, c.stream>>>(out, acc, d, conv, tab, c.t->primes, c.N);
    post(c);
}

void launch_rescale_prep(const LaunchCtx &c, View r, View xtop, const RescaleTable *tab, int B, int comps, int top,
                         const Scalars *sc)
{
    Timed tm_(c, K_RESCALE, 8.0 * B * comps * (top + 1) * c.N);
    dim3 grid(ew_blocks(c.N, 2), top, B * comps);
    k_rescale_prep<<<grid, 256, 0, c.stream>>>(r, xtop, tab, c.t->primes, comps, top, c.N, sc ? *sc : Scalars{},
                                               sc != nullptr);
    post(c);
}

void launch_rescale_final(const LaunchCtx &c, View out, View in, View r, const RescaleTable *tab, int B, int comps,
                          int top, const Scalars *sc)
{
    Timed tm_(c, K_RESCALE, 24.0 * B * comps * top * c.N);
    dim3 grid(ew_blocks(c.N, 2), top, B * comps);
    k_rescale_final<<<grid, 256, 0, c.stream>>>(out, in, r, tab, c.t->primes, comps, c.N, sc ? *sc : Scalars{},
                                                sc != nullptr);
    post(c);
}

void launch_keygen_b(const LaunchCtx &c, uint64_t *b, const uint64_t *a, const uint64_t *e, const uint64_t *s,
                     const uint64_t *sp, const uint64_t *gad, int rows, const int *, bool to_mont)
{
    dim3 grid(ew_blocks(c.N, 1), rows, 1);
    k_keygen_b<<<grid, 256, 0, c.stream>>>(b, const_cast<uint64_t *>(a), e, s, sp, gad, c.t->primes, c.N, to_mont);
    post(c);
}

void launch_encrypt_combine(const LaunchCtx &c, uint64_t *ct, const uint64_t *v, const uint64_t *e0,
                            const uint64_t *e1, const uint64_t *m, const uint64_t *pk, int n_q, int limbs)
{
    dim3 grid(ew_blocks(c.N, 1), limbs, 1);
    k_encrypt_combine<<<grid, 256, 0, c.stream>>>(ct, v, e0, e1, m, pk, c.t->primes, n_q, limbs, c.N);
    post(c);
}

void launch_signed_to_rows(const LaunchCtx &c, uint64_t *out, const int64_t *in, int rows, int n_in_polys,
                           size_t in_stride, const int *prime_dev)
{
    dim3 grid(ew_blocks(c.N, 1), rows, n_in_polys);
    k_signed_to_rows<<<grid, 256, 0, c.stream>>>(out, in, rows, in_stride, prime_dev, c.t->primes, c.N);
    post(c);
}

void launch_to_mont(const LaunchCtx &c, uint64_t *p, int rows, const int *prime_dev)
{
    dim3 grid(ew_blocks(c.N, 1), rows, 1);
    k_to_mont<<<grid, 256, 0, c.stream>>>(p, prime_dev, c.t->primes, c.N);
    post(c);
}

void launch_mul_rows(const LaunchCtx &c, uint64_t *out, const uint64_t *a, const uint64_t *b, int rows)
{
    dim3 grid(ew_blocks(c.N, 1), rows, 1);
    k_mul_rows<<<grid, 256, 0, c.stream>>>(out, a, b, c.t->primes, c.N);
    post(c);
}

void launch_ddec_shares(const LaunchCtx &c, uint64_t *out, View ct, const uint64_t *shares, int n_parties, int B)
{
    dim3 grid(ew_blocks(c.N, 1), n_parties + 1, B);
    k_ddec_shares<<<grid, 256, 0, c.stream>>>(out, ct, shares, c.t->primes, n_parties, c.N);
    post(c);
}

// ---- several rings in one launch per key-switching stage: launchers ----------------------------
static void check_job_grid(long long blocks, int n_jobs)
{
    HX_CHECK(n_jobs >= 1 && blocks >= 1 && blocks < (1ll << 31), HX_EINVAL, "bad several-ring job grid");
}

void launch_automorphism_jobs(cudaStream_t s, const AutomorphismJob *jobs, int n_jobs, long long blocks,
                              std::atomic<uint64_t> *launches)
{
    check_job_grid(blocks, n_jobs);
    k_automorphism_jobs<<<(unsigned)blocks, 256, 0, s>>>(jobs, n_jobs);
    HX_CUDA(cudaGetLastError());
    if (launches) *launches += 1;
}

void launch_convert_jobs(cudaStream_t s, const ConvertJob *jobs, int n_jobs, long long blocks, int max_src,
                         std::atomic<uint64_t> *launches)
{
    check_job_grid(blocks, n_jobs);
    HX_CHECK(max_src >= 1 && max_src <= MAXK, HX_EINVAL, "too many conversion sources");
    if (max_src <= 4) k_convert_jobs<4><<<(unsigned)blocks, 256, 0, s>>>(jobs, n_jobs);
    else k_convert_jobs<MAXK><<<(unsigned)blocks, 256, 0, s>>>(jobs, n_jobs);
    HX_CUDA(cudaGetLastError());
    if (launches) *launches += 1;
}

void launch_key_ip_jobs(cudaStream_t s, const KeyIpJob *jobs, int n_jobs, long long blocks,
                        std::atomic<uint64_t> *launches)
{
    check_job_grid(blocks, n_jobs);
    k_key_ip_jobs<<<(unsigned)blocks, 256, 0, s>>>(jobs, n_jobs);
    HX_CUDA(cudaGetLastError());
    if (launches) *launches += 1;
}

void launch_moddown_jobs(cudaStream_t s, const ModDownJob *jobs, int n_jobs, long long blocks,
                         std::atomic<uint64_t> *launches)
{
    check_job_grid(blocks, n_jobs);
    k_moddown_jobs<<<(unsigned)blocks, 256, 0, s>>>(jobs, n_jobs);
    HX_CUDA(cudaGetLastError());
    if (launches) *launches += 1;
}

} // namespace hx
