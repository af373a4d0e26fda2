// The negacyclic NTT of one limb = Cooley-Tukey (forward, natural ->
// bit-reversed order, psi powers merged into the twiddles) and
// Gentleman-Sande (inverse), split into a column phase (the first log2(N1)
// stages: N1 rows of stride N2) and a row phase (the remaining stages on N2
// contiguous words), each staged through shared memory.  Every global word is
// read and written once per phase with 128-byte coalesced row segments.
#include <algorithm>
#include <cstdio>
#include <memory>

#include "launch_util.cuh"

namespace hx {

namespace {

// ---- NTT ----------------------------------------------------------------------
//
// A phase holds, in shared memory, n_sub independent sub-transforms of M = 2^L
// points (element e of sub-transform k at sh[k*sk + e*se (+ e/16 padding)]).
// Its L local stages run as two register passes: each thread loads 2^R
// elements spaced t = M >> (S0+R) apart, applies R radix-2 stages in
// registers (2^R - 1 twiddle loads for R*2^(R-1) butterflies) and stores them
// back.  Global stage of local stage s is g0 + s; the twiddle of a butterfly
// at global stage G on global element j is tw[2^G + (j >> (log N - G))].

__device__ __forceinline__ void bf_ct(uint64_t &x, uint64_t &y, const ulonglong2 w, uint64_t q, uint64_t two_q)
{
    uint64_t a = x;
    if (a >= two_q) a -= two_q;
    const uint64_t t = shoup_lazy(y, w.x, w.y, q);
    x = a + t;
    y = a - t + two_q;
}

__device__ __forceinline__ void bf_gs(uint64_t &x, uint64_t &y, const ulonglong2 w, uint64_t q, uint64_t two_q)
{
    uint64_t u = x + y;
    if (u >= two_q) u -= two_q;
    const uint64_t d = x - y + two_q;
    x = u;
    y = shoup_lazy(d, w.x, w.y, q);
}

template <int L, int R, int S0, bool INV, bool KFAST, bool PAD>
__device__ __forceinline__ void ntt_pass(uint64_t *sh, int n_sub, int sk, int se, const ulonglong2 *__restrict__ tw,
                                         int g0, int blk0, int blk_step, uint64_t q, int nthr)
{
    constexpr int M = 1 << L, RR = 1 << R, TL = M >> (S0 + R), ITEMS = M >> R;
    const uint64_t two_q = 2 * q;
    for (int w = threadIdx.x; w < ITEMS * n_sub; w += nthr) {
        const int k = KFAST ? w % n_sub : w / ITEMS;
        const int u = KFAST ? w / n_sub : w % ITEMS;
        const int hi = u / TL, lo = u % TL;
        const int base = hi * TL * RR + lo;
        const int blk = blk0 + k * blk_step;
        uint64_t v[RR];
#pragma unroll
        for (int m = 0; m < RR; m++) {
            const int e = base + m * TL;
            v[m] = sh[k * sk + e * se + (PAD ? 2 * (e >> 4) : 0)];
        }
        if (!INV) {
#pragma unroll
            for (int vv = 0; vv < R; vv++) {
                const int s = S0 + vv, half = RR >> (vv + 1);
                const int tbase = (1 << (g0 + s)) + (blk << s) + (hi << vv);
#pragma unroll
                for (int gl = 0; gl < (1 << vv); gl++) {
                    const ulonglong2 wv = tw[tbase + gl];
#pragma unroll
                    for (int j = 0; j < half; j++) bf_ct(v[gl * 2 * half + j], v[gl * 2 * half + j + half], wv, q, two_q);
                }
            }
        } else {
#pragma unroll
            for (int vv = R - 1; vv >= 0; vv--) {
                const int s = S0 + vv, half = RR >> (vv + 1);
                const int tbase = (1 << (g0 + s)) + (blk << s) + (hi << vv);
#pragma unroll
                for (int gl = 0; gl < (1 << vv); gl++) {
                    const ulonglong2 wv = tw[tbase + gl];
#pragma unroll
                    for (int j = 0; j < half; j++) bf_gs(v[gl * 2 * half + j], v[gl * 2 * half + j + half], wv, q, two_q);
                }
            }
        }
#pragma unroll
        for (int m = 0; m < RR; m++) {
            const int e = base + m * TL;
            sh[k * sk + e * se + (PAD ? 2 * (e >> 4) : 0)] = v[m];
        }
    }
}

// The column phase's last register pass, its results stored straight to global memory (word e
// of column k at dst + e*N2 + k): consecutive threads hold consecutive columns, so each warp
// store covers whole COLS-word row segments and the phase needs no shared-memory round trip
// for its output.  Forward: outputs stay lazy (below 4q) for the row phase.  Inverse: the pass
// ends with stage 0, whose butterfly also applies N^-1 -- x' = (x+y) N^-1 and
// y' = (x-y) psi^-brv(1) N^-1, one product each instead of a butterfly product and two
// scalings -- and the outputs are fully reduced.
template <int LOGM, int R, int S0, int COLS, bool INV>
__device__ __forceinline__ void ntt_pass_out(const uint64_t *sh, const ulonglong2 *__restrict__ tw, const PrimeConst &P,
                                             uint64_t *dst, int N2, int nthr)
{
    constexpr int M = 1 << LOGM, RR = 1 << R, TL = M >> (S0 + R), ITEMS = M >> R;
    const uint64_t q = P.q, two_q = 2 * q;
    for (int w = threadIdx.x; w < ITEMS * COLS; w += nthr) {
        const int k = w % COLS, u = w / COLS;
        const int hi = u / TL, lo = u % TL;
        const int base = hi * TL * RR + lo;
        uint64_t v[RR];
#pragma unroll
        for (int m = 0; m < RR; m++) v[m] = sh[k + (base + m * TL) * COLS];
        if (!INV) {
#pragma unroll
            for (int vv = 0; vv < R; vv++) {
                const int s = S0 + vv, half = RR >> (vv + 1);
                const int tbase = (1 << s) + (hi << vv);
#pragma unroll
                for (int gl = 0; gl < (1 << vv); gl++) {
                    const ulonglong2 wv = tw[tbase + gl];
#pragma unroll
                    for (int j = 0; j < half; j++) bf_ct(v[gl * 2 * half + j], v[gl * 2 * half + j + half], wv, q, two_q);
                }
            }
        } else {
#pragma unroll
            for (int vv = R - 1; vv >= 1; vv--) {
                const int s = S0 + vv, half = RR >> (vv + 1);
                const int tbase = (1 << s) + (hi << vv);
#pragma unroll
                for (int gl = 0; gl < (1 << vv); gl++) {
                    const ulonglong2 wv = tw[tbase + gl];
#pragma unroll
                    for (int j = 0; j < half; j++) bf_gs(v[gl * 2 * half + j], v[gl * 2 * half + j + half], wv, q, two_q);
                }
            }
            static_assert(!INV || S0 == 0, "the inverse output pass must end with stage 0");
#pragma unroll
            for (int j = 0; j < RR / 2; j++) {
                uint64_t x = v[j] + v[j + RR / 2];
                if (x >= two_q) x -= two_q;
                const uint64_t d = v[j] - v[j + RR / 2] + two_q;
                v[j] = shoup(x, P.n_inv, P.n_inv_sh, q);
                v[j + RR / 2] = shoup(d, P.n_inv_w1, P.n_inv_w1_sh, q);
            }
        }
#pragma unroll
        for (int m = 0; m < RR; m++) dst[(size_t)(base + m * TL) * N2 + k] = v[m];
    }
}

template <int L, bool ALT = false> struct Split {
    // first pass (stages 0..R1-1) and second pass; ALT swaps the two radices of an odd L
    static constexpr int R1 = ALT ? L / 2 : (L + 1) / 2;
    static constexpr int R2 = L - R1;
};

// Asynchronous global->shared copies (cp.async): the next tile streams in while
// the current one is transformed.
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all_but_one() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// tile t of a phase -> (group, row, position along the row)
struct TileId {
    int g, row, bx;
};
__device__ __forceinline__ TileId tile_of(int t, int nb, int n_rows)
{
    TileId r;
    r.bx = t % nb;
    const int rest = t / nb;
    r.row = rest % n_rows;
    r.g = rest / n_rows;
    return r;
}

// column phase: the first LOGM stages on M rows of stride N2 (COLS adjacent columns
// per tile); each block loops over tiles with the next tile (and its twiddles,
// indices below M) prefetched into the other half of shared memory
template <int LOGM, int COLS, bool INV, bool ALT>
__global__ void __launch_bounds__((1 << (LOGM - Split<LOGM, ALT>::R1)) * COLS)
k_ntt_cols(const __grid_constant__ NttRows R, const PrimeConst *__restrict__ primes,
           const ulonglong2 *__restrict__ tw_all, int log_n, int n_tiles)
{
    constexpr int M = 1 << LOGM, E = M * COLS, R1 = Split<LOGM, ALT>::R1, R2 = Split<LOGM, ALT>::R2;
    constexpr int T = (M >> R1) * COLS;
    extern __shared__ uint64_t sh[];
    uint64_t *buf[2] = {sh, sh + E};
    ulonglong2 *stw[2] = {reinterpret_cast<ulonglong2 *>(sh + 2 * E), reinterpret_cast<ulonglong2 *>(sh + 2 * E) + M};
    const int N = 1 << log_n, N2 = N >> LOGM, nb = N2 / COLS;
    auto prefetch = [&](int t, int slot) {
        const TileId id = tile_of(t, nb, R.n_rows);
        const int pr = R.prime[id.row];
        const uint64_t *src = INV ? R.dst + (size_t)id.g * R.dst_gs + (size_t)R.dst_off[id.row] * N
                                  : R.src + (size_t)id.g * R.src_gs + (size_t)R.src_off[id.row] * N;
        const int c0 = id.bx * COLS;
        for (int i = threadIdx.x; i < E / 2; i += T) {  // 16-byte pieces of COLS-word row segments
            const int r = (2 * i) / COLS, c = (2 * i) % COLS;
            cp_async16(buf[slot] + 2 * i, src + (size_t)r * N2 + c0 + c);
        }
        const ulonglong2 *tw = tw_all + (size_t)pr * N;
        for (int i = threadIdx.x; i < M; i += T) cp_async16(stw[slot] + i, tw + i);
        cp_async_commit();
    };
    int t = blockIdx.x, slot = 0;
    if (t < n_tiles) prefetch(t, 0);
    for (; t < n_tiles; t += gridDim.x, slot ^= 1) {
        const int tn = t + gridDim.x;
        if (tn < n_tiles) {
            prefetch(tn, slot ^ 1);
            cp_async_wait_all_but_one();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
        const TileId id = tile_of(t, nb, R.n_rows);
        const PrimeConst P = primes[R.prime[id.row]];
        uint64_t *dst = R.dst + (size_t)id.g * R.dst_gs + (size_t)R.dst_off[id.row] * N;
        const int c0 = id.bx * COLS;
        uint64_t *b = buf[slot];
        if (!INV) {
            ntt_pass<LOGM, R1, 0, false, true, false>(b, COLS, 1, COLS, stw[slot], 0, 0, 0, P.q, T);
            __syncthreads();
            ntt_pass_out<LOGM, R2, R1, COLS, false>(b, stw[slot], P, dst + c0, N2, T);
        } else {
            ntt_pass<LOGM, R2, R1, true, true, false>(b, COLS, 1, COLS, stw[slot], 0, 0, 0, P.q, T);
            __syncthreads();
            ntt_pass_out<LOGM, R1, 0, COLS, true>(b, stw[slot], P, dst + c0, N2, T);
        }
        __syncthreads();  // this half is refilled by the prefetch two tiles later
    }
}

// row phase: the remaining LOGM stages on ROWS contiguous blocks of M words per tile
// (padded layout, one spare word per 16), next tile prefetched in 8-byte pieces
template <int LOGM, int ROWS, bool INV, bool ALT>
__global__ void __launch_bounds__((1 << (LOGM - Split<LOGM, ALT>::R1)) * ROWS)
k_ntt_rows(const __grid_constant__ NttRows R, const PrimeConst *__restrict__ primes,
           const ulonglong2 *__restrict__ tw_all, int log_n, int n_tiles)
{
    constexpr int M = 1 << LOGM, E = M * ROWS, R1 = Split<LOGM, ALT>::R1, R2 = Split<LOGM, ALT>::R2;
    constexpr int T = (M >> R1) * ROWS;
    constexpr int SK = M + M / 8;  // padded block stride (two spare words per 16)
    extern __shared__ uint64_t sh[];
    uint64_t *buf[2] = {sh, sh + ROWS * SK};
    const int N = 1 << log_n;
    const int g0 = log_n - LOGM;
    const int nb = (N >> LOGM) / ROWS;
    auto prefetch = [&](int t, int slot) {
        const TileId id = tile_of(t, nb, R.n_rows);
        const uint64_t *src = INV ? R.src + (size_t)id.g * R.src_gs + (size_t)R.src_off[id.row] * N
                                  : R.dst + (size_t)id.g * R.dst_gs + (size_t)R.dst_off[id.row] * N;
        const size_t base = (size_t)id.bx * ROWS * M;
        for (int i = threadIdx.x; i < E / 2; i += T) {  // 16-byte pieces: pairs stay in one padding group
            const int k = (2 * i) / M, e = (2 * i) % M;
            cp_async16(buf[slot] + k * SK + e + 2 * (e >> 4), src + base + 2 * i);
        }
        cp_async_commit();
    };
    int t = blockIdx.x, slot = 0;
    if (t < n_tiles) prefetch(t, 0);
    for (; t < n_tiles; t += gridDim.x, slot ^= 1) {
        const int tn = t + gridDim.x;
        if (tn < n_tiles) {
            prefetch(tn, slot ^ 1);
            cp_async_wait_all_but_one();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
        const TileId id = tile_of(t, nb, R.n_rows);
        const int pr = R.prime[id.row];
        const PrimeConst P = primes[pr];
        const uint64_t q = P.q, two_q = 2 * q;
        const ulonglong2 *tw = tw_all + (size_t)pr * N;
        uint64_t *dst = R.dst + (size_t)id.g * R.dst_gs + (size_t)R.dst_off[id.row] * N;
        const int r_base = id.bx * ROWS;
        const size_t base = (size_t)r_base * M;
        uint64_t *b = buf[slot];
        if (!INV) {
            ntt_pass<LOGM, R1, 0, false, false, true>(b, ROWS, SK, 1, tw, g0, r_base, 1, q, T);
            __syncthreads();
            ntt_pass<LOGM, R2, R1, false, false, true>(b, ROWS, SK, 1, tw, g0, r_base, 1, q, T);
            __syncthreads();
            for (int i = threadIdx.x; i < E / 2; i += T) {  // pairs (e even, e+1) share a padding group
                const int k = (2 * i) / M, e = (2 * i) % M;
                const int sidx = k * SK + e + 2 * (e >> 4);
                uint64_t v0 = b[sidx], v1 = b[sidx + 1];
                if (v0 >= two_q) v0 -= two_q;
                if (v0 >= q) v0 -= q;
                if (v1 >= two_q) v1 -= two_q;
                if (v1 >= q) v1 -= q;
                *reinterpret_cast<ulonglong2 *>(dst + base + 2 * i) = make_ulonglong2(v0, v1);
            }
        } else {
            ntt_pass<LOGM, R2, R1, true, false, true>(b, ROWS, SK, 1, tw, g0, r_base, 1, q, T);
            __syncthreads();
            ntt_pass<LOGM, R1, 0, true, false, true>(b, ROWS, SK, 1, tw, g0, r_base, 1, q, T);
            __syncthreads();
            for (int i = threadIdx.x; i < E / 2; i += T) {
                const int k = (2 * i) / M, e = (2 * i) % M;
                const int sidx = k * SK + e + 2 * (e >> 4);
                *reinterpret_cast<ulonglong2 *>(dst + base + 2 * i) = make_ulonglong2(b[sidx], b[sidx + 1]);
            }
        }
        __syncthreads();
    }
}

// tile widths the autotuner chooses from (sub-transforms per block); a variant is a width index
// plus NTT_WIDTHS if the phase's two register passes swap radices (odd phase sizes only)
constexpr const int *kNttTiles = kNttTileWidths;

template <int LOGM, int COLS, bool INV, bool ALT>
void ntt_cols_w(const LaunchCtx &c, const NttRows &rows)
{
    constexpr int M = 1 << LOGM;
    constexpr int E = M * COLS;
    constexpr int T = (M >> Split<LOGM, ALT>::R1) * COLS;
    const int N2 = c.N >> LOGM;
    HX_CHECK(N2 % COLS == 0, HX_EINVAL, "NTT tile wider than the ring");
    const long long n_tiles = (long long)(N2 / COLS) * rows.n_rows * rows.n_groups;
    HX_CHECK(n_tiles < (1ll << 31), HX_EINVAL, "NTT batch too large");
    const size_t smem = (size_t)E * 16 + (size_t)M * 32;  // two tiles + two twiddle sets
    static const bool attr =  // thread-safe one-time setup
        cudaFuncSetAttribute(k_ntt_cols<LOGM, COLS, INV, ALT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) == cudaSuccess;
    (void)attr;
    static const int per_sm = [&] {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_ntt_cols<LOGM, COLS, INV, ALT>, T, smem);
        return v;
    }();
    const int grid = (int)std::min<long long>(n_tiles, (long long)std::max(1, per_sm) * c.t->n_sm);
    k_ntt_cols<LOGM, COLS, INV, ALT><<<grid, T, smem, c.stream>>>(rows, c.t->primes, INV ? c.t->tw_inv : c.t->tw_fwd,
                                                                 c.log_n, (int)n_tiles);
}

template <int LOGM, int ROWS, bool INV, bool ALT>
void ntt_rows_w(const LaunchCtx &c, const NttRows &rows)
{
    constexpr int M = 1 << LOGM;
    constexpr int T = (M >> Split<LOGM, ALT>::R1) * ROWS;
    const int N1 = c.N >> LOGM;
    HX_CHECK(N1 % ROWS == 0, HX_EINVAL, "NTT tile wider than the ring");
    const long long n_tiles = (long long)(N1 / ROWS) * rows.n_rows * rows.n_groups;
    HX_CHECK(n_tiles < (1ll << 31), HX_EINVAL, "NTT batch too large");
    const size_t smem = (size_t)ROWS * (M + M / 8) * 16;  // two tiles
    static const bool attr =  // thread-safe one-time setup
        cudaFuncSetAttribute(k_ntt_rows<LOGM, ROWS, INV, ALT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) == cudaSuccess;
    (void)attr;
    static const int per_sm = [&] {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_ntt_rows<LOGM, ROWS, INV, ALT>, T, smem);
        return v;
    }();
    const int grid = (int)std::min<long long>(n_tiles, (long long)std::max(1, per_sm) * c.t->n_sm);
    k_ntt_rows<LOGM, ROWS, INV, ALT><<<grid, T, smem, c.stream>>>(rows, c.t->primes, INV ? c.t->tw_inv : c.t->tw_fwd,
                                                                 c.log_n, (int)n_tiles);
}

template <bool INV, int LOGM, bool ALT>
void ntt_phase_a(const LaunchCtx &c, const NttRows &r, bool cols, int wi)
{
    switch (wi) {
    case 0: cols ? ntt_cols_w<LOGM, 4, INV, ALT>(c, r) : ntt_rows_w<LOGM, 4, INV, ALT>(c, r); break;
    case 1: cols ? ntt_cols_w<LOGM, 8, INV, ALT>(c, r) : ntt_rows_w<LOGM, 8, INV, ALT>(c, r); break;
    case 2: cols ? ntt_cols_w<LOGM, 16, INV, ALT>(c, r) : ntt_rows_w<LOGM, 16, INV, ALT>(c, r); break;
    default: cols ? ntt_cols_w<LOGM, 32, INV, ALT>(c, r) : ntt_rows_w<LOGM, 32, INV, ALT>(c, r); break;
    }
}

template <bool INV, int LOGM>
void ntt_phase_l(const LaunchCtx &c, const NttRows &r, bool cols, int var)
{
    // the tile must not be wider than the other dimension of the ring
    const int other = c.N >> LOGM;
    int wi = var % NTT_WIDTHS;
    while (wi > 0 && kNttTiles[wi] > other) wi--;
    if ((LOGM & 1) && var >= NTT_WIDTHS) ntt_phase_a<INV, LOGM, (LOGM & 1) != 0>(c, r, cols, wi);
    else ntt_phase_a<INV, LOGM, false>(c, r, cols, wi);
}

template <bool INV>
void ntt_phase(const LaunchCtx &c, const NttRows &r, bool cols, int logm, int var)
{
    switch (logm) {
    case 5: ntt_phase_l<INV, 5>(c, r, cols, var); break;
    case 6: ntt_phase_l<INV, 6>(c, r, cols, var); break;
    case 7: ntt_phase_l<INV, 7>(c, r, cols, var); break;
    case 8: ntt_phase_l<INV, 8>(c, r, cols, var); break;
    default: throw Error{HX_EINVAL, "unsupported NTT size"};
    }
}

// ---- several rings in one launch ------------------------------------------------
// A job is n_rows rows of one ring (its own N, primes and twiddles), transformed
// in place.  One persistent kernel per phase walks the tiles of every job, the
// next tile (and for the column phase its twiddles) streaming into the other
// half of shared memory while the current one is transformed; a tile's phase
// size picks the template instance, with the tile width chosen so every
// instance runs 128 threads.

constexpr int kMultiT = 128;
template <int LOGM> struct MultiW {  // tile width per phase size: (M >> R1) * W = 128 threads
    static constexpr int W = kMultiT / ((1 << LOGM) >> Split<LOGM>::R1);
};
constexpr int kMultiColsBuf = 2048 + 2 * 256;  // words: the largest column tile and its twiddles
constexpr int kMultiRowsBuf = 8 * (256 + 32);  // words: the largest padded row tile

struct MultiTile {
    uint64_t *row;
    const ulonglong2 *tw;
    const PrimeConst *primes;
    int pr, logm, log_n, bx;
};

__device__ __forceinline__ MultiTile multi_tile(const NttJob *jobs, int n_jobs, int t, bool cols, bool inv)
{
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if ((cols ? jobs[mid].tile0_cols : jobs[mid].tile0_rows) <= t) lo = mid;
        else hi = mid - 1;
    }
    const NttJob &J = jobs[lo];
    MultiTile m;
    const int local = t - (cols ? J.tile0_cols : J.tile0_rows);
    m.log_n = J.log_n;
    m.logm = cols ? J.log_n / 2 : J.log_n - J.log_n / 2;
    const int n = 1 << J.log_n;
    const int W = kMultiT / ((1 << m.logm) >> ((m.logm + 1) / 2));
    const int nb = (n >> m.logm) / W;
    const int r = local / nb;
    m.bx = local % nb;
    m.pr = J.prime[r % J.n_limbs];
    m.primes = J.primes;
    m.row = J.data + (size_t)r * n;
    m.tw = (inv ? J.tw_inv : J.tw_fwd) + (size_t)m.pr * n;
    return m;
}

template <int LOGM>
__device__ void multi_cols_load(uint64_t *b, const MultiTile &m)
{
    constexpr int M = 1 << LOGM, COLS = MultiW<LOGM>::W, E = M * COLS;
    const int N2 = (1 << m.log_n) >> LOGM, c0 = m.bx * COLS;
    ulonglong2 *stw = reinterpret_cast<ulonglong2 *>(b + 2048);
    for (int i = threadIdx.x; i < E / 2; i += kMultiT) {
        const int r = (2 * i) / COLS, c = (2 * i) % COLS;
        cp_async16(b + 2 * i, m.row + (size_t)r * N2 + c0 + c);
    }
    for (int i = threadIdx.x; i < M; i += kMultiT) cp_async16(stw + i, m.tw + i);
}

template <int LOGM, bool INV>
__device__ void multi_cols_run(uint64_t *b, const MultiTile &m, const PrimeConst &P)
{
    constexpr int M = 1 << LOGM, COLS = MultiW<LOGM>::W, E = M * COLS;
    constexpr int R1 = Split<LOGM>::R1, R2 = Split<LOGM>::R2;
    const int N2 = (1 << m.log_n) >> LOGM, c0 = m.bx * COLS;
    const ulonglong2 *stw = reinterpret_cast<const ulonglong2 *>(b + 2048);
    if (!INV) {
        ntt_pass<LOGM, R1, 0, false, true, false>(b, COLS, 1, COLS, stw, 0, 0, 0, P.q, kMultiT);
        __syncthreads();
        ntt_pass<LOGM, R2, R1, false, true, false>(b, COLS, 1, COLS, stw, 0, 0, 0, P.q, kMultiT);
        __syncthreads();
        for (int i = threadIdx.x; i < E; i += kMultiT) m.row[(size_t)(i / COLS) * N2 + c0 + (i % COLS)] = b[i];
    } else {
        ntt_pass<LOGM, R2, R1, true, true, false>(b, COLS, 1, COLS, stw, 0, 0, 0, P.q, kMultiT);
        __syncthreads();
        ntt_pass<LOGM, R1, 0, true, true, false>(b, COLS, 1, COLS, stw, 0, 0, 0, P.q, kMultiT);
        __syncthreads();
        for (int i = threadIdx.x; i < E; i += kMultiT)
            m.row[(size_t)(i / COLS) * N2 + c0 + (i % COLS)] = shoup(b[i], P.n_inv, P.n_inv_sh, P.q);
    }
}

template <int LOGM>
__device__ void multi_rows_load(uint64_t *b, const MultiTile &m)
{
    constexpr int M = 1 << LOGM, ROWS = MultiW<LOGM>::W, E = M * ROWS, SK = M + M / 8;
    const size_t base = (size_t)m.bx * ROWS * M;
    for (int i = threadIdx.x; i < E; i += kMultiT) {
        const int k = i / M, e = i % M;
        cp_async8(b + k * SK + e + 2 * (e >> 4), m.row + base + i);
    }
}

template <int LOGM, bool INV>
__device__ void multi_rows_run(uint64_t *b, const MultiTile &m, const PrimeConst &P)
{
    constexpr int M = 1 << LOGM, ROWS = MultiW<LOGM>::W, E = M * ROWS, SK = M + M / 8;
    constexpr int R1 = Split<LOGM>::R1, R2 = Split<LOGM>::R2;
    const int g0 = m.log_n - LOGM, r_base = m.bx * ROWS;
    const size_t base = (size_t)r_base * M;
    const uint64_t q = P.q, two_q = 2 * q;
    if (!INV) {
        ntt_pass<LOGM, R1, 0, false, false, true>(b, ROWS, SK, 1, m.tw, g0, r_base, 1, q, kMultiT);
        __syncthreads();
        ntt_pass<LOGM, R2, R1, false, false, true>(b, ROWS, SK, 1, m.tw, g0, r_base, 1, q, kMultiT);
        __syncthreads();
        for (int i = threadIdx.x; i < E; i += kMultiT) {
            const int k = i / M, e = i % M;
            uint64_t v = b[k * SK + e + 2 * (e >> 4)];
            if (v >= two_q) v -= two_q;
            if (v >= q) v -= q;
            m.row[base + i] = v;
        }
    } else {
        ntt_pass<LOGM, R2, R1, true, false, true>(b, ROWS, SK, 1, m.tw, g0, r_base, 1, q, kMultiT);
        __syncthreads();
        ntt_pass<LOGM, R1, 0, true, false, true>(b, ROWS, SK, 1, m.tw, g0, r_base, 1, q, kMultiT);
        __syncthreads();
        for (int i = threadIdx.x; i < E; i += kMultiT) {
            const int k = i / M, e = i % M;
            m.row[base + i] = b[k * SK + e + 2 * (e >> 4)];
        }
    }
}

template <bool INV, bool COLS_PHASE>
__global__ void __launch_bounds__(kMultiT) k_ntt_multi(const NttJob *__restrict__ jobs, int n_jobs, int n_tiles)
{
    extern __shared__ uint64_t sh[];
    constexpr int BUF = COLS_PHASE ? kMultiColsBuf : kMultiRowsBuf;
    auto load = [&](const MultiTile &m, int slot) {
        uint64_t *b = sh + slot * BUF;
        switch (m.logm) {
        case 5: COLS_PHASE ? multi_cols_load<5>(b, m) : multi_rows_load<5>(b, m); break;
        case 6: COLS_PHASE ? multi_cols_load<6>(b, m) : multi_rows_load<6>(b, m); break;
        case 7: COLS_PHASE ? multi_cols_load<7>(b, m) : multi_rows_load<7>(b, m); break;
        default: COLS_PHASE ? multi_cols_load<8>(b, m) : multi_rows_load<8>(b, m); break;
        }
        cp_async_commit();
    };
    int t = blockIdx.x, slot = 0;
    MultiTile cur{};
    if (t < n_tiles) {
        cur = multi_tile(jobs, n_jobs, t, COLS_PHASE, INV);
        load(cur, 0);
    }
    for (; t < n_tiles; t += gridDim.x, slot ^= 1) {
        const int tn = t + gridDim.x;
        MultiTile nxt{};
        if (tn < n_tiles) {
            nxt = multi_tile(jobs, n_jobs, tn, COLS_PHASE, INV);
            load(nxt, slot ^ 1);
            cp_async_wait_all_but_one();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
        const PrimeConst P = cur.primes[cur.pr];
        uint64_t *b = sh + slot * BUF;
        switch (cur.logm) {
        case 5: COLS_PHASE ? multi_cols_run<5, INV>(b, cur, P) : multi_rows_run<5, INV>(b, cur, P); break;
        case 6: COLS_PHASE ? multi_cols_run<6, INV>(b, cur, P) : multi_rows_run<6, INV>(b, cur, P); break;
        case 7: COLS_PHASE ? multi_cols_run<7, INV>(b, cur, P) : multi_rows_run<7, INV>(b, cur, P); break;
        default: COLS_PHASE ? multi_cols_run<8, INV>(b, cur, P) : multi_rows_run<8, INV>(b, cur, P); break;
        }
        __syncthreads();  // this half is refilled by the prefetch two tiles later
        cur = nxt;
    }
}

// ---- end of the several-ring kernels

} // namespace

// ---- launcher (host code: it picks the tuned variants and the phase split of the kernels above)
void launch_ntt(const LaunchCtx &c, const NttRows &rows, bool inverse)
{
    Timed tm_(c, K_NTT, 16.0 * rows.n_rows * rows.n_groups * c.N);
    if (rows.n_rows <= 0 || rows.n_groups <= 0) return;
    HX_CHECK(rows.n_rows <= MAX_NTT_ROWS && rows.n_groups < 65536, HX_EINVAL, "NTT batch too large");
    const int *v = c.t->ntt_var[ntt_bucket((long long)rows.n_rows * rows.n_groups)];
    const int logm1 = c.log_n / 2 + ((c.log_n & 1) && v[4] ? 1 : 0), logm2 = c.log_n - logm1;
    if (!inverse) {
        ntt_phase<false>(c, rows, true, logm1, v[0]);
        ntt_phase<false>(c, rows, false, logm2, v[1]);
    } else {
        ntt_phase<true>(c, rows, false, logm2, v[3]);
        ntt_phase<true>(c, rows, true, logm1, v[2]);
    }
    post(c, 2);
}
// ---- end of the launcher

// ---- autotuner (host code: it times the phase kernels and changes none of them)
void autotune_ntt(const LaunchCtx &c, uint64_t *buf, int rows, int *best, float *ms_out)
{
    // times every tile width of each phase on `rows` limbs (one prime each) in place, for each
    // split of an odd log N between the phases
    NttRows *r = new NttRows();
    std::unique_ptr<NttRows> guard(r);
    r->src = r->dst = buf;
    r->src_gs = r->dst_gs = 0;
    r->n_groups = 1;
    r->n_rows = rows;
    for (int i = 0; i < rows; i++) {
        r->src_off[i] = r->dst_off[i] = (int16_t)i;
        r->prime[i] = 0;
    }
    cudaEvent_t e0, e1;
    HX_CUDA(cudaEventCreate(&e0));
    HX_CUDA(cudaEventCreate(&e1));
    // Each variant's time is the best of three rounds of five transforms, the rounds interleaved
    // over the variants so drift hits them alike.  A variant replaces the default (width 16: four
    // warps per block in the 128-point phases) only when it is clearly faster: the widths' isolated
    // times differ by about their noise (1-2 % at the batch sizes of a product's launches), and
    // blocks of the default size share the SMs best with the kernels of concurrent chains.  The
    // other split of an odd log N replaces the default one on the same rule, by the sum of its
    // four phases' times.
    constexpr int kDefault = 2, kRounds = 3, kRuns = 5;
    constexpr float kClearWin = 0.98f;
    float split_ms[2] = {0.f, 0.f};
    int split_best[2][4];
    float split_phase_ms[2][4];
    const int n_splits = (c.log_n & 1) ? 2 : 1;
    for (int sp = 0; sp < n_splits; sp++) {
        const int logm1 = c.log_n / 2 + sp, logm2 = c.log_n - logm1;
        for (int ph = 0; ph < 4; ph++) {
            const bool cols = ph == 0 || ph == 2, inv = ph >= 2;
            const int logm = cols ? logm1 : logm2;
            float t[NTT_VARIANTS];
            bool ok[NTT_VARIANTS];
            for (int v = 0; v < NTT_VARIANTS; v++) {
                t[v] = 1e30f;
                ok[v] = kNttTiles[v % NTT_WIDTHS] <= (c.N >> logm) && (v < NTT_WIDTHS || (logm & 1));
            }
            for (int round = 0; round < kRounds; round++)
                for (int v = 0; v < NTT_VARIANTS; v++) {
                    if (!ok[v]) continue;
                    auto run = [&]() {
                        if (inv) ntt_phase<true>(c, *r, cols, logm, v);
                        else ntt_phase<false>(c, *r, cols, logm, v);
                    };
                    run();  // warm-up
                    HX_CUDA(cudaEventRecord(e0, c.stream));
                    for (int it = 0; it < kRuns; it++) run();
                    HX_CUDA(cudaEventRecord(e1, c.stream));
                    HX_CUDA(cudaEventSynchronize(e1));
                    float ms = 0;
                    HX_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    t[v] = std::min(t[v], ms / kRuns);
                }
            int pick = ok[kDefault] ? kDefault : -1;
            for (int v = 0; v < NTT_VARIANTS; v++) {
                if (!ok[v] || v == pick) continue;
                if (pick < 0 || t[v] < (pick == kDefault ? kClearWin : 1.0f) * t[pick]) pick = v;
            }
            split_best[sp][ph] = pick < 0 ? kDefault : pick;
            split_phase_ms[sp][ph] = pick < 0 ? 0.f : t[pick];
            split_ms[sp] += split_phase_ms[sp][ph];
        }
    }
    const int sp = (n_splits == 2 && split_ms[1] < kClearWin * split_ms[0]) ? 1 : 0;
    for (int ph = 0; ph < 4; ph++) {
        best[ph] = split_best[sp][ph];
        if (ms_out) ms_out[ph] = split_phase_ms[sp][ph];
    }
    best[4] = sp;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    HX_CUDA(cudaGetLastError());
}
// ---- end of the autotuner

// ---- several rings: launcher
void plan_ntt_jobs(std::vector<NttJob> &jobs, int *tiles_cols, int *tiles_rows)
{
    int tc = 0, tr = 0;
    for (auto &J : jobs) {
        HX_CHECK(J.log_n >= 11 && J.log_n <= 16, HX_EINVAL, "ring degree outside 2^11..2^16");
        HX_CHECK(J.n_limbs >= 1 && J.n_limbs <= 64 && J.n_rows >= 0, HX_EINVAL, "bad job rows");
        const int n = 1 << J.log_n, l1 = J.log_n / 2, l2 = J.log_n - l1;
        const int w1 = 128 / ((1 << l1) >> ((l1 + 1) / 2)), w2 = 128 / ((1 << l2) >> ((l2 + 1) / 2));
        J.tile0_cols = tc;
        J.tile0_rows = tr;
        const long long c = (long long)J.n_rows * ((n >> l1) / w1), r = (long long)J.n_rows * ((n >> l2) / w2);
        HX_CHECK(tc + c < (1ll << 31) && tr + r < (1ll << 31), HX_EINVAL, "NTT batch too large");
        tc += (int)c;
        tr += (int)r;
    }
    *tiles_cols = tc;
    *tiles_rows = tr;
}

void launch_ntt_jobs(cudaStream_t s, const NttJob *jp, int n_jobs, int tc, int tr, bool inverse, int n_sm,
                     std::atomic<uint64_t> *launches)
{
    if (tc == 0) return;
    // two halves of shared memory per block (current tile, next tile)
    const size_t smem_c = 2 * sizeof(uint64_t) * kMultiColsBuf, smem_r = 2 * sizeof(uint64_t) * kMultiRowsBuf;
    const int grid_c = std::min(tc, n_sm * 8), grid_r = std::min(tr, n_sm * 8);
    if (!inverse) {
        k_ntt_multi<false, true><<<grid_c, kMultiT, smem_c, s>>>(jp, n_jobs, tc);
        k_ntt_multi<false, false><<<grid_r, kMultiT, smem_r, s>>>(jp, n_jobs, tr);
    } else {
        k_ntt_multi<true, false><<<grid_r, kMultiT, smem_r, s>>>(jp, n_jobs, tr);
        k_ntt_multi<true, true><<<grid_c, kMultiT, smem_c, s>>>(jp, n_jobs, tc);
    }
    HX_CUDA(cudaGetLastError());
    if (launches) *launches += 2;
}

void launch_ntt_multi(cudaStream_t s, const std::vector<NttJob> &jobs_in, bool inverse, int n_sm,
                      std::atomic<uint64_t> *launches)
{
    std::vector<NttJob> jobs = jobs_in;
    int tc = 0, tr = 0;
    plan_ntt_jobs(jobs, &tc, &tr);
    if (tc == 0) return;
    void *jd = nullptr;
    HX_CUDA(cudaMallocAsync(&jd, jobs.size() * sizeof(NttJob), s));
    HX_CUDA(cudaMemcpyAsync(jd, jobs.data(), jobs.size() * sizeof(NttJob), cudaMemcpyHostToDevice, s));
    try {
        launch_ntt_jobs(s, reinterpret_cast<const NttJob *>(jd), (int)jobs.size(), tc, tr, inverse, n_sm, launches);
    } catch (...) {
        cudaFreeAsync(jd, s);
        throw;
    }
    HX_CUDA(cudaFreeAsync(jd, s));
    HX_CUDA(cudaStreamSynchronize(s));  // the host job vector is released at return
}

// ---- end of the several-ring launcher

} // namespace hx
