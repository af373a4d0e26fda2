// Client-side encoding and encryption of a batch on the device (Fig. 1 items 3
// and 5): the canonical-embedding encoder as a batched 2N-point FFT in
// double-double arithmetic and the encryption randomness drawn from the same
// counter-based SplitMix64 streams as the host path, so every ciphertext equals
// hx_encrypt's.
//
// Encoding is exact: coefficient i is scale * (2/N) * sum_j z_j cos(pi (i e_j
// mod 2N)/N) rounded half away from zero (a value within 2^-20 of a
// half-integer taken as that half-integer).  The sum is carried in
// double-double numbers (about 106 bits; exact products by fused multiply-add,
// Knuth's two-sum), so its error is far inside that band and the integer is the
// one the exact value gives -- the host encoder's, whatever the order of the
// operations.
#include "runtime.h"

namespace hx {

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr int kFftTile = 1024;  // points of the sub-transforms done in shared memory

__device__ __forceinline__ uint64_t dmix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ---- double-double arithmetic, every operation rounded once (explicit _rn intrinsics: no
// contraction by the compiler)
struct ddv {
    double hi, lo;
};

__device__ __forceinline__ ddv dd_two_sum(double a, double b)
{
    const double s = __dadd_rn(a, b), v = __dsub_rn(s, a);
    return ddv{s, __dadd_rn(__dsub_rn(a, __dsub_rn(s, v)), __dsub_rn(b, v))};
}

__device__ __forceinline__ ddv dd_fast(double a, double b)
{
    const double s = __dadd_rn(a, b);
    return ddv{s, __dsub_rn(b, __dsub_rn(s, a))};
}

__device__ __forceinline__ ddv dd_plus(ddv x, ddv y)
{
    const ddv s = dd_two_sum(x.hi, y.hi), t = dd_two_sum(x.lo, y.lo);
    const ddv u = dd_fast(s.hi, __dadd_rn(s.lo, t.hi));
    return dd_fast(u.hi, __dadd_rn(u.lo, t.lo));
}

__device__ __forceinline__ ddv dd_minus(ddv x, ddv y) { return dd_plus(x, ddv{-y.hi, -y.lo}); }

__device__ __forceinline__ ddv dd_times(ddv x, ddv y)
{
    const double p = __dmul_rn(x.hi, y.hi);
    const double e = __fma_rn(x.hi, y.hi, -p);  // exact error of the leading product
    const double c = __fma_rn(x.hi, y.lo, __dmul_rn(x.lo, y.hi));
    return dd_fast(p, __dadd_rn(e, c));
}

__device__ __forceinline__ ddv dd_times_d(ddv x, double d)
{
    const double p = __dmul_rn(x.hi, d);
    return dd_fast(p, __fma_rn(x.lo, d, __fma_rn(x.hi, d, -p)));
}

// a complex double-double point: (re.hi, re.lo, im.hi, im.lo)
__device__ __forceinline__ void butterfly(double4 &u, double4 &v, const double4 w)
{
    const ddv vr{v.x, v.y}, vi{v.z, v.w}, wr{w.x, w.y}, wi{w.z, w.w};
    const ddv tr = dd_minus(dd_times(vr, wr), dd_times(vi, wi));
    const ddv ti = dd_plus(dd_times(vr, wi), dd_times(vi, wr));
    const ddv ur{u.x, u.y}, ui{u.z, u.w};
    const ddv a = dd_plus(ur, tr), b = dd_plus(ui, ti), c = dd_minus(ur, tr), d = dd_minus(ui, ti);
    u = make_double4(a.hi, a.lo, b.hi, b.lo);
    v = make_double4(c.hi, c.lo, d.hi, d.lo);
}

// hi + lo rounded half away from zero, |value - (k + 1/2)| <= 2^-20 counting as the tie;
// *bad set past 2^62
__device__ __forceinline__ int64_t round_coeff(ddv x, int *bad)
{
    if (!(fabs(x.hi) < 4611686018427387904.0)) {
        *bad = 1;
        return 0;
    }
    const double i1 = rint(x.hi), i2 = rint(x.lo);
    const double f = __dadd_rn(__dsub_rn(x.hi, i1), __dsub_rn(x.lo, i2));
    int64_t k = (int64_t)i1 + (int64_t)i2;
    const double g = fabs(f);
    if (fabs(__dsub_rn(g, 0.5)) <= 0x1p-20) {
        // tie at k + 1/2 (f > 0) or k - 1/2 (f < 0): away from zero
        if (f > 0) k += (k >= 0) ? 1 : 0;
        else k -= (k <= 0) ? 1 : 0;
    } else if (f > 0.5) {
        k += 1;
    } else if (f < -0.5) {
        k -= 1;
    }
    if (k >= (int64_t(1) << 62) || k <= -(int64_t(1) << 62)) *bad = 1;
    return k;
}

// The 2N-point transform's input holds slot j at the bit-reversed positions of the odd exponents
// e_j and 2N - e_j, and zeros at every even exponent.  Bit reversal sends even exponents to the
// first half, so the first half stays zero through every stage but the last, whose butterflies
// then give A_i = w_i B_i (i < N, w_i = roots[i]) from the second half B alone.  The transform
// therefore runs on the second half only (N points, compact: position p at p - N), and the last
// stage is folded into the coefficients' read-out; every double-double value is the one the full
// transform computes (adding a zero returns the other operand exactly).
__global__ void k_enc_place(double4 *A, const double *slots, size_t n_slots, const int *e, int log_m, int half_n)
{
    const int b = blockIdx.y;
    const int m = 1 << log_m, n = m >> 1;
    double4 *a = A + (size_t)b * n;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < half_n; j += gridDim.x * blockDim.x) {
        const double z = (size_t)j < n_slots ? slots[(size_t)b * n_slots + j] : 0.0;
        const unsigned p1 = __brev((unsigned)e[j]) >> (32 - log_m);
        const unsigned p2 = __brev((unsigned)((m - e[j]) & (m - 1))) >> (32 - log_m);
        a[p1 - n] = make_double4(z, 0.0, 0.0, 0.0);
        a[p2 - n] = make_double4(z, 0.0, 0.0, 0.0);
    }
}

// stages len = 2 .. kFftTile (radix-2 decimation in time) on contiguous tiles of the compact
// second half in shared memory
__global__ void __launch_bounds__(kFftTile / 2) k_enc_fft_tile(double4 *A, const double4 *__restrict__ roots, int log_m)
{
    __shared__ double4 s[kFftTile];
    const int m = 1 << log_m;
    double4 *a = A + (size_t)blockIdx.y * (m >> 1) + (size_t)blockIdx.x * kFftTile;
    for (int i = threadIdx.x; i < kFftTile; i += blockDim.x) s[i] = a[i];
    __syncthreads();
    for (int len = 2; len <= kFftTile; len <<= 1) {
        const int half = len >> 1, step = m / len;
        for (int t = threadIdx.x; t < kFftTile / 2; t += blockDim.x) {
            const int g = t / half, k = t % half, i = g * len + k;
            double4 u = s[i], v = s[i + half];
            butterfly(u, v, roots[(size_t)k * step]);
            s[i] = u;
            s[i + half] = v;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < kFftTile; i += blockDim.x) a[i] = s[i];
}

// one later stage (kFftTile < len <= N) over the compact second half in global memory
__global__ void k_enc_fft_stage(double4 *A, const double4 *__restrict__ roots, int log_m, int len)
{
    const int m = 1 << log_m, half = len >> 1, step = m / len;
    double4 *a = A + (size_t)blockIdx.y * (m >> 1);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m / 4; t += gridDim.x * blockDim.x) {
        const int g = t / half, k = t % half, i = g * len + k;
        double4 u = a[i], v = a[i + half];
        butterfly(u, v, roots[(size_t)k * step]);
        a[i] = u;
        a[i + half] = v;
    }
}

// Re A_i = Re(w_i B_i), the last stage's butterfly on a zero first-half entry
__device__ __forceinline__ ddv enc_last_re(const double4 bi, const double4 w)
{
    return dd_minus(dd_times(ddv{bi.x, bi.y}, ddv{w.x, w.y}), dd_times(ddv{bi.z, bi.w}, ddv{w.z, w.w}));
}

// coefficient i = round(Re A_i / N * scale) under round_coeff; a coefficient past 2^62 sets *err
__global__ void k_enc_round(int64_t *out, size_t out_stride, const double4 *A, const double4 *__restrict__ roots,
                            int n, double scale, int *err)
{
    const int b = blockIdx.y;
    const double4 *a = A + (size_t)b * n;
    const double inv_n = 1.0 / n;  // a power of two: exact
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int bad = 0;
        const ddv re = enc_last_re(a[i], roots[i]);
        const ddv m{__dmul_rn(re.hi, inv_n), __dmul_rn(re.lo, inv_n)};
        const int64_t v = round_coeff(dd_times_d(m, scale), &bad);
        if (bad) atomicExch(err, 1);
        out[b * out_stride + i] = bad ? 0 : v;
    }
}

// the encoder's real coefficients m_i = Re(a_i) / n (double-double), before the scale
__global__ void k_enc_real(double2 *m, size_t m_stride, const double4 *A, const double4 *__restrict__ roots, int n)
{
    const int b = blockIdx.y;
    const double4 *a = A + (size_t)b * n;
    const double inv_n = 1.0 / n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const ddv re = enc_last_re(a[i], roots[i]);
        m[b * m_stride + i] = make_double2(__dmul_rn(re.hi, inv_n), __dmul_rn(re.lo, inv_n));
    }
}

// out row r = round(m[idx[r]] * scale): k_enc_round's last steps on cached coefficients
__global__ void k_enc_round_rows(int64_t *out, const double2 *m, const int *idx, int n, double scale, int *err)
{
    const int r = blockIdx.y;
    const double2 *mr = m + (size_t)idx[r] * n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int bad = 0;
        const double2 v = mr[i];
        const int64_t c = round_coeff(dd_times_d(ddv{v.x, v.y}, scale), &bad);
        if (bad) atomicExch(err, 1);
        out[(size_t)r * n + i] = bad ? 0 : c;
    }
}

// encryption randomness of entry b: poly 0 ternary (v), 1 and 2 Gaussian (e0, e1);
// state0[b*3 + p] is the stream's initial state, draw i = mix64(state0 + (i+1) gamma)
__global__ void k_enc_sample(int64_t *out, size_t entry_stride, const uint64_t *__restrict__ state0,
                             const uint64_t *__restrict__ th, int bound, int n)
{
    const int b = blockIdx.z, p = blockIdx.y;
    const uint64_t st = state0[b * 3 + p];
    int64_t *o = out + b * entry_stride + (size_t)p * n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint64_t r = dmix64(st + (uint64_t)(i + 1) * kGamma);
        if (p == 0) {
            const uint64_t t = r % 3;
            o[i] = t == 2 ? -1 : (int64_t)t;
        } else {
            const uint64_t x = r >> 1;
            int idx = 0;
            while (idx < 2 * bound && x >= th[idx]) idx++;
            o[i] = (int64_t)idx - bound;
        }
    }
}

int grid_for(size_t work) { return (int)std::min<size_t>((work + 255) / 256, 4096); }

// device copies of the host encoder's tables (2N-th roots, 5^j mod 2N) and of
// the Gaussian sampler's thresholds, built once per context
const EncTables &enc_tables(hx_context &ctx)
{
    std::call_once(ctx.enc_once, [&] {
        const int N = ctx.N;
        EncTables &t = ctx.enc_dev;
        // the host encoder's double-double roots e^(-2 pi i k / 2N), k < N, as (re.hi, re.lo, im.hi, im.lo)
        std::vector<double> r4((size_t)4 * N);
        for (int k = 0; k < N; k++) {
            r4[4 * k] = ctx.enc->roots_re[k].hi;
            r4[4 * k + 1] = ctx.enc->roots_re[k].lo;
            r4[4 * k + 2] = ctx.enc->roots_im[k].hi;
            r4[4 * k + 3] = ctx.enc->roots_im[k].lo;
        }
        t.roots = std::make_shared<DevBuf>((size_t)4 * N, true);
        HX_CUDA(cudaMemcpy(t.roots->p, r4.data(), sizeof(double) * r4.size(), cudaMemcpyHostToDevice));
        std::vector<int> e32(N / 2);
        for (int j = 0; j < N / 2; j++) e32[j] = (int)ctx.enc->e[j];
        t.e = std::make_shared<DevBuf>((size_t)(N / 2 + 1) / 2, true);
        HX_CUDA(cudaMemcpy(t.e->p, e32.data(), sizeof(int) * e32.size(), cudaMemcpyHostToDevice));
        t.th = std::make_shared<DevBuf>(ctx.cdt->th.size(), true);
        HX_CUDA(cudaMemcpy(t.th->p, ctx.cdt->th.data(), sizeof(uint64_t) * ctx.cdt->th.size(),
                           cudaMemcpyHostToDevice));
    });
    HX_CHECK(ctx.enc_dev.roots && ctx.enc_dev.e && ctx.enc_dev.th, HX_ECUDA, "encoder tables are missing");
    return ctx.enc_dev;
}

// the 2N-point transforms of `count` slot vectors up to their last stage, in place in A
// ([count][N] complex double-double: the second halves, see k_enc_place)
void enc_transform(hx_context &ctx, const EncTables &t, double4 *a, const double *slots_dev, size_t n_slots,
                          int count, cudaStream_t s)
{
    const int N = ctx.N, log_m = ctx.log_n + 1;
    const double4 *roots = reinterpret_cast<const double4 *>(t.roots->p);
    HX_CUDA(cudaMemsetAsync(a, 0, sizeof(double4) * (size_t)N * count, s));
    k_enc_place<<<dim3(grid_for(N / 2), count), 256, 0, s>>>(a, slots_dev, n_slots,
                                                             reinterpret_cast<const int *>(t.e->p), log_m, N / 2);
    k_enc_fft_tile<<<dim3(N / kFftTile, count), kFftTile / 2, 0, s>>>(a, roots, log_m);
    for (int len = 2 * kFftTile; len <= N; len <<= 1)
        k_enc_fft_stage<<<dim3(grid_for(N / 2), count), 256, 0, s>>>(a, roots, log_m, len);
    HX_CUDA(cudaGetLastError());
    ctx.counters[C_LAUNCH] += 2 + (log_m - 11);
}

// vectors transformed per pass: bounds the complex double-double work buffer (32 B per point)
constexpr int kEncChunk = 64;

} // namespace

// coefficients of the canonical-embedding encoding of `count` slot vectors
// (device, [count][N] int64), equal to Encoder::encode's
void encode_batch(hx_context &ctx, const double *slots_dev, size_t n_slots, int count, double scale, int64_t *out,
                  size_t out_stride, cudaStream_t s)
{
    const int N = ctx.N;
    HX_CHECK(N % kFftTile == 0, HX_EINVAL, "the device encoder needs N >= 1024");
    HX_CHECK(n_slots <= (size_t)N / 2 && count >= 1 && count < 65536, HX_EINVAL, "bad slot batch");
    const EncTables &t = enc_tables(ctx);
    const double4 *roots = reinterpret_cast<const double4 *>(t.roots->p);
    const int chunk = std::min(count, kEncChunk);
    DevBuf A((size_t)4 * N * chunk, s);
    DevBuf err(1, s);
    HX_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    double4 *a = reinterpret_cast<double4 *>(A.p);
    for (int b0 = 0; b0 < count; b0 += chunk) {
        const int c = std::min(chunk, count - b0);
        enc_transform(ctx, t, a, slots_dev + (size_t)b0 * n_slots, n_slots, c, s);
        k_enc_round<<<dim3(grid_for(N), c), 256, 0, s>>>(out + (size_t)b0 * out_stride, out_stride, a, roots, N, scale,
                                                         reinterpret_cast<int *>(err.p));
        HX_CUDA(cudaGetLastError());
        ctx.counters[C_LAUNCH] += 1;
    }
    int herr = 0;
    HX_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    HX_CUDA(cudaStreamSynchronize(s));
    HX_CHECK(herr == 0, HX_EINVAL, "encoded coefficient exceeds 2^62");
}

// the real coefficients of the encoding of every slot vector (scale not yet applied), as
// double-double pairs [count][N]: encode_batch's coefficients are their rounded products with
// the scale
void encode_real_batch(hx_context &ctx, const double *slots_dev, size_t n_slots, int count, double2 *m_out,
                       cudaStream_t s)
{
    const int N = ctx.N;
    HX_CHECK(N % kFftTile == 0, HX_EINVAL, "the device encoder needs N >= 1024");
    HX_CHECK(n_slots <= (size_t)N / 2 && count >= 1 && count < 65536, HX_EINVAL, "bad slot batch");
    const EncTables &t = enc_tables(ctx);
    const double4 *roots = reinterpret_cast<const double4 *>(t.roots->p);
    const int chunk = std::min(count, kEncChunk);
    DevBuf A((size_t)4 * N * chunk, s);
    double4 *a = reinterpret_cast<double4 *>(A.p);
    for (int b0 = 0; b0 < count; b0 += chunk) {
        const int c = std::min(chunk, count - b0);
        enc_transform(ctx, t, a, slots_dev + (size_t)b0 * n_slots, n_slots, c, s);
        k_enc_real<<<dim3(grid_for(N), c), 256, 0, s>>>(m_out + (size_t)b0 * N, (size_t)N, a, roots, N);
        HX_CUDA(cudaGetLastError());
        ctx.counters[C_LAUNCH] += 1;
    }
    HX_CUDA(cudaStreamSynchronize(s));  // the work buffer is released at return
}

// rows[r] of the output = the encoding at `scale` of the slot vector whose real coefficients
// are row idx_dev[r] of m (count rows, N coefficients each)
void encode_rows_from_real(hx_context &ctx, const double2 *m, const int *idx_dev, int count, double scale,
                           int64_t *out, cudaStream_t s)
{
    HX_CHECK(count >= 1 && count < 65536, HX_EINVAL, "bad row count");
    DevBuf err(1, s);
    HX_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    k_enc_round_rows<<<dim3(grid_for(ctx.N), count), 256, 0, s>>>(out, m, idx_dev, ctx.N, scale,
                                                                  reinterpret_cast<int *>(err.p));
    HX_CUDA(cudaGetLastError());
    int herr = 0;
    HX_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    HX_CUDA(cudaStreamSynchronize(s));
    HX_CHECK(herr == 0, HX_EINVAL, "encoded coefficient exceeds 2^62");
}

// Enc(pk, Ecd(slots_b)) for every b, seeds[b] as hx_encrypt's seed (tag 0, index 0)
Cts encrypt_batch(hx_context &ctx, const hx_keyset &ks, const double *slots_dev, size_t n_slots, int count, int limbs,
                  const uint64_t *seeds, cudaStream_t s)
{
    HX_CHECK(limbs >= 1 && limbs <= ctx.n_q, HX_EINVAL, "bad level");
    const int N = ctx.N;
    Eval ev(ctx, s);
    const EncTables &t = enc_tables(ctx);
    // per entry: [v, e0, e1, m] signed coefficients
    DevBuf raw((size_t)count * 4 * N, s);
    int64_t *r = reinterpret_cast<int64_t *>(raw.p);
    std::vector<uint64_t> st((size_t)count * 3);
    for (int b = 0; b < count; b++) {
        st[b * 3 + 0] = Stream(seeds[b], P_ENC_V, 0, 0).state;
        st[b * 3 + 1] = Stream(seeds[b], P_ENC_E0, 0, 0).state;
        st[b * 3 + 2] = Stream(seeds[b], P_ENC_E1, 0, 0).state;
    }
    DevBuf st_dev(st.size(), s);
    HX_CUDA(cudaMemcpyAsync(st_dev.p, st.data(), sizeof(uint64_t) * st.size(), cudaMemcpyHostToDevice, s));
    k_enc_sample<<<dim3(grid_for(N), 3, count), 256, 0, s>>>(r, (size_t)4 * N, st_dev.p, t.th->p, ctx.cdt->bound, N);
    HX_CUDA(cudaGetLastError());
    ctx.counters[C_LAUNCH] += 1;
    encode_batch(ctx, slots_dev, n_slots, count, ctx.scale, r + 3 * (size_t)N, (size_t)4 * N, s);
    // residues over the first `limbs` primes, NTT form: [count*4][limbs][N]
    DevBuf polys((size_t)count * 4 * limbs * N, s);
    launch_signed_to_rows(ev.lc(), polys.p, r, limbs, count * 4, (size_t)N, ctx.d_prime_ids);
    std::vector<int> rows(limbs);
    for (int l = 0; l < limbs; l++) rows[l] = l;
    ev.ntt_inplace(polys.p, (size_t)limbs * N, count * 4, rows, rows, false);
    Cts c = ev.alloc(count, 2, limbs);
    c.scale = ctx.scale;
    const size_t st4 = (size_t)limbs * N;
    for (int b = 0; b < count; b++) {
        const uint64_t *pb = polys.p + (size_t)b * 4 * st4;
        launch_encrypt_combine(ev.lc(), c.d + (size_t)b * c.bstride(N), pb, pb + st4, pb + 2 * st4, pb + 3 * st4,
                               ks.pk->p, ctx.n_q, limbs);
    }
    HX_CUDA(cudaStreamSynchronize(s));  // the staging buffers above are released at return
    return c;
}

} // namespace hx
