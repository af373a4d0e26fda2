// Internal structures shared by the host runtime and the kernel launchers.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/hx.h"
#include "modarith.cuh"

namespace hx {

constexpr int MAXP = HX_MAX_Q + HX_MAX_P;
constexpr int MAXK = HX_MAX_P + 1;  // conversion sources: the special primes, plus q_top when RS joins ModDown
constexpr int MAX_NTT_ROWS = 1024;
constexpr int NTT_WIDTHS = 4;    // tile widths 4, 8, 16, 32 (sub-transforms per block)
constexpr int kNttTileWidths[NTT_WIDTHS] = {4, 8, 16, 32};
constexpr int NTT_VARIANTS = 2 * NTT_WIDTHS;  // a width, with the register passes' radices as is or swapped
// NTT batch sizes tuned separately: a launch of n limbs uses the first bucket with n <= its bound
constexpr int NTT_BUCKETS = 4;
constexpr int kNttBucketMax[NTT_BUCKETS] = {64, 256, 768, 1 << 30};
constexpr int kNttBucketTune[NTT_BUCKETS] = {48, 176, 512, 1024};  // limbs timed for each bucket
inline int ntt_bucket(long long limbs)
{
    int b = 0;
    while (b < NTT_BUCKETS - 1 && limbs > kNttBucketMax[b]) b++;
    return b;
}

// Fast basis conversion table (Han-Ki hybrid key switching, no correction):
// out_t = sum_i [x_i * qhat_i^-1]_{q_i} * (qhat_i mod t)  (mod t), every term a Shoup product
struct ConvTable {
    int n_src, n_dst;
    int src_row[MAXK];        // rows of the source buffer
    int src_prime[MAXK];      // prime indices (Q then P)
    int dst_row[MAXP];        // rows of the destination buffer
    int dst_prime[MAXP];
    uint64_t inv[MAXK], inv_sh[MAXK];   // [qhat_i^-1]_{q_i} with Shoup companion
    uint64_t w[MAXK][MAXP], w_sh[MAXK][MAXP];  // qhat_i mod t with its Shoup companion
    // shift != 0: the rounded division's remainder.  Convert x + h exactly (the overshoot
    // u = floor(sum_i y_i / q_i), summed in FP64, times the source product is removed),
    // then subtract h
    int shift;
    uint64_t add_src[MAXK];             // h mod q_i
    double inv_d[MAXK];                 // 1 / q_i in FP64
    uint64_t sub_dst[MAXP];             // h mod t
    uint64_t prod_mod[MAXP];            // (product of the sources) mod t
};

struct ModDownTable {
    ConvTable conv;                      // P -> Q_l
    uint64_t pinv[MAXP], pinv_sh[MAXP];  // P^-1 mod q_i, Shoup
};

// relinearisation and rescale in one division by P * q_top (limbs l -> l-1)
struct RelinRescaleTable {
    ConvTable conv;                      // {q_top, P} -> Q_{l-1}, shifted by h = floor(P q_top / 2)
    uint64_t pmod[MAXP], pmod_sh[MAXP];  // P mod q_i, i < l
    uint64_t pqinv[MAXP], pqinv_sh[MAXP];  // (P q_top)^-1 mod q_i, i < l-1
};

struct RescaleTable {
    uint64_t half;                                   // floor(q_top / 2)
    uint64_t qinv[MAXP], qinv_sh[MAXP];              // q_top^-1 mod q_i
    uint64_t half_mod[MAXP];                         // half mod q_i
};

// Rows of a batched NTT: for group g in [0,n_groups) and row r in
// [0,n_rows), the source row is src + g*src_gs + src_off[r]*N and the
// destination row dst + g*dst_gs + dst_off[r]*N (equal for in-place use),
// taken modulo prime index prime[r].
struct NttRows {
    const uint64_t *src;
    uint64_t *dst;
    size_t src_gs, dst_gs;
    int n_groups;
    int n_rows;
    int16_t src_off[MAX_NTT_ROWS];
    int16_t dst_off[MAX_NTT_ROWS];
    int16_t prime[MAX_NTT_ROWS];
};

struct Scalars {
    uint64_t v[MAXP], sh[MAXP];
};

// Inner sums of a baby-step/giant-step linear transform: for every group g,
// out_g = sum_m baby_m (.) mask[g][m] over the babies whose mask is present.
constexpr int MAC_MAX_BABY = 16, MAC_MAX_GROUP = 32;
struct MacArgs {
    int n_baby, n_group;
    const uint64_t *baby[MAC_MAX_BABY];
    size_t baby_bstride, baby_cstride;
    const uint64_t *mask[MAC_MAX_GROUP][MAC_MAX_BABY];  // Montgomery form, [limbs][N]; null if absent
    uint64_t *out;                                      // [group][B][2][limbs][N]
};

// A batch of polynomials with `comps` components of `limbs` rows each:
// word (b, c, l, j) at p + b*bstride + c*cstride + l*N + j.
struct View {
    uint64_t *p;
    size_t bstride, cstride;
};

struct DeviceTables {
    PrimeConst *primes = nullptr;   // [n_all]
    ulonglong2 *tw_fwd = nullptr;   // [n_all][N] (psi^brv(k), Shoup)
    ulonglong2 *tw_inv = nullptr;   // [n_all][N] (psi^-brv(k), Shoup)
    ConvTable *modup = nullptr;     // [(n_q+1) * dnum] by (limbs, digit)
    ModDownTable *moddown = nullptr;// [n_q+1] by limbs
    RescaleTable *rescale = nullptr;// [n_q+1] by limbs
    RelinRescaleTable *relin_rs = nullptr;  // [n_q+1] by limbs
    // NTT variant per batch-size bucket and phase (fwd cols, fwd rows, inv cols, inv rows)
    // per bucket: the four phases' variants (forward column, forward row, inverse column, inverse
    // row), then the split of an odd log N (0: the column phase takes floor(log N / 2) stages, 1: ceil)
    int ntt_var[NTT_BUCKETS][5] = {{2, 2, 2, 2, 0}, {2, 2, 2, 2, 0}, {2, 2, 2, 2, 0}, {2, 2, 2, 2, 0}};
    int n_sm = 1;                   // multiprocessors of the device
};

// Per-kernel-class timing with CUDA events recorded on the launching stream
// (enabled only while profiling; the events bracket every launch of a class).
struct Profiler {
    struct Rec {
        int cls;
        cudaEvent_t a, b;
        double bytes;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get();
    void clear();
};
enum KClass { K_NTT, K_KEYIP, K_CONV, K_MODDOWN, K_RESCALE, K_TENSOR, K_MULPT, K_ELEM, K_AUTO, K_AGG, K_MISC, K_NCLASS };
extern const char *const kclass_names[K_NCLASS];

// ---- kernel launchers (kernels.cu) ----------------------------------------------
struct LaunchCtx {
    int log_n, N;
    const DeviceTables *t;
    cudaStream_t stream;
    std::atomic<uint64_t> *launches;
    Profiler *prof = nullptr;
};

void launch_ntt(const LaunchCtx &c, const NttRows &rows, bool inverse);
// one job of a multi-ring NTT: n_rows rows of 2^log_n words at data (in place), row r modulo
// prime[r % n_limbs] of its own context's tables
struct NttJob {
    uint64_t *data;
    const PrimeConst *primes;
    const ulonglong2 *tw_fwd, *tw_inv;
    int log_n, n_rows, n_limbs;
    int tile0_cols, tile0_rows;  // filled by the launcher
    int16_t prime[64];
};
// every job's transform in one launch per phase (several ring degrees together)
void launch_ntt_multi(cudaStream_t s, const std::vector<NttJob> &jobs, bool inverse, int n_sm,
                      std::atomic<uint64_t> *launches);

// times every NTT variant (tile width, radix split) of each phase on `rows` limbs of buf and
// writes the fastest per phase
void autotune_ntt(const LaunchCtx &c, uint64_t *buf, int rows, int *best, float *ms_out);
void launch_add(const LaunchCtx &c, View out, View a, View b, int B, int comps, int limbs, bool sub);
void launch_copy(const LaunchCtx &c, View out, View a, int B, int comps, int limbs);
// one ciphertext read in place: component c, limb l at p + c*cstride + l*N
struct AggSrc {
    const uint64_t *p;
    uint64_t cstride;
};
// out[m] = C * sum_i src[i*count + m] (per limb, C given as Scalars), for m < count
void launch_aggregate(const LaunchCtx &c, View out, const AggSrc *src_dev, int n_parties, int count, int comps,
                      int limbs, const Scalars &C);
void launch_mul_plain(const LaunchCtx &c, View out, View a, const uint64_t *pt_mont, int B, int limbs);
void launch_mul_scalar(const LaunchCtx &c, View out, View a, const Scalars &sc, int B, int comps, int limbs);
void launch_add_scalar_c0(const LaunchCtx &c, View out, View a, const Scalars &sc, int B, int limbs);
// mont: the products left times 2^-64 (Montgomery reductions), to be scaled back once after summing
void launch_tensor(const LaunchCtx &c, View out3, View a, View b, int B, int limbs, bool accumulate,
                   bool mont = false);
void launch_automorphism(const LaunchCtx &c, View out, View in, uint64_t g, int B, int comps, int limbs,
                         bool accumulate = false);
// alg_bytes: one read of every source row and one write of every destination row (profiling)
void launch_basis_convert(const LaunchCtx &c, const ConvTable *tab_dev, int max_src, View out, View in, int B,
                          int groups, size_t gstride_out, size_t gstride_in, double alg_bytes = 0.0);
void launch_key_ip(const LaunchCtx &c, View acc, const uint64_t *D, const uint64_t *dnt, size_t dnt_bstride,
                   const uint64_t *key, int n_all, int n_q, int K, int alpha, int limbs, int ndig, uint64_t g, int B,
                   bool accumulate = false);
// out_c = (acc_c - conv_c) * P^-1, plus add_c[galois(j)] for the components set in add_mask
void launch_moddown_final(const LaunchCtx &c, View out, View acc, View conv, const ModDownTable *tab, int B,
                          int limbs, View add, int add_mask, uint64_t add_galois);

// ---- several rings in one launch per key-switching stage (one job = one ring's batch) ----------
// Each kernel runs the body of its one-ring counterpart over every job: a flat grid whose block
// b belongs to the job with the largest block0 <= b, at the coordinates that job's own grid
// (gx, gy, gz) would give it.
struct AutomorphismJob {
    View out, in;
    uint64_t g;
    int comps, log_n;
    const PrimeConst *primes;
    int gx, gy, gz;
    long long block0;
};
struct ConvertJob {
    const ConvTable *tabs;
    View out, in;
    const PrimeConst *primes;
    int groups, n, max_src;
    size_t gstride_out, gstride_in;
    int gx, gy, gz;
    long long block0;
};
struct KeyIpJob {
    View acc;
    const uint64_t *D, *dnt, *key;
    size_t dnt_bstride;
    const PrimeConst *primes;
    int n_all, n_q, K, alpha, limbs, ndig, log_n, few;
    uint64_t g;
    int gx, gy, gz;
    long long block0;
};
struct ModDownJob {
    View out, acc, conv, add;
    const ModDownTable *tab;
    const PrimeConst *primes;
    int add_mask, log_n;
    uint64_t g;
    int gx, gy, gz;
    long long block0;
};
// Fills every job's block0; returns the blocks of the grid over all of them.
template <class J> long long plan_job_blocks(std::vector<J> &jobs)
{
    long long total = 0;
    for (auto &j : jobs) {
        j.block0 = total;
        total += (long long)j.gx * j.gy * j.gz;
    }
    return total;
}
// one grid over the jobs of a table already on the device (blocks from plan_job_blocks)
void launch_automorphism_jobs(cudaStream_t s, const AutomorphismJob *jobs, int n_jobs, long long blocks,
                              std::atomic<uint64_t> *launches);
void launch_convert_jobs(cudaStream_t s, const ConvertJob *jobs, int n_jobs, long long blocks, int max_src,
                         std::atomic<uint64_t> *launches);
void launch_key_ip_jobs(cudaStream_t s, const KeyIpJob *jobs, int n_jobs, long long blocks,
                        std::atomic<uint64_t> *launches);
void launch_moddown_jobs(cudaStream_t s, const ModDownJob *jobs, int n_jobs, long long blocks,
                         std::atomic<uint64_t> *launches);
// the NTT over several rings in two steps: tile offsets of every job (host), then the two phase
// launches over a job table already on the device
void plan_ntt_jobs(std::vector<NttJob> &jobs, int *tiles_cols, int *tiles_rows);
void launch_ntt_jobs(cudaStream_t s, const NttJob *jobs, int n_jobs, int tiles_cols, int tiles_rows, bool inverse,
                     int n_sm, std::atomic<uint64_t> *launches);
void launch_lintrans_mac(const LaunchCtx &c, const MacArgs &a, int B, int limbs, int n_terms);
// two hoisted rotations selected by a mask in the extended basis (see kernels.cu)
void launch_key_ip_mux(const LaunchCtx &c, View out, const uint64_t *D, const uint64_t *dnt, size_t dnt_bstride,
                       const uint64_t *key1, const uint64_t *key2, const uint64_t *v, const Scalars &cs, int n_all,
                       int n_q, int K, int alpha, int limbs, int ndig, uint64_t g1, uint64_t g2, int B);
// premasked keys of one selection: out = [2][ndig][2][ext][N] with
// out[0] = v (.) key1, out[1] = (c - v) (.) key2 on the rows of the extended basis (Montgomery form);
// cR[t] = c * 2^64 mod (prime of row t)
void launch_premask_keys(const LaunchCtx &c, uint64_t *out, const uint64_t *key1, const uint64_t *key2,
                         const uint64_t *v, const Scalars &cR, int n_all, int n_q, int K, int limbs, int ndig);
// the inner products of a selection with premasked keys: z_h = sum_d sigma_g1(D_d) pk[0][d][h]
// + sigma_g2(D_d) pk[1][d][h], one Montgomery reduction
void launch_key_ip_mux_pm(const LaunchCtx &c, View out, const uint64_t *D, const uint64_t *dnt, size_t dnt_bstride,
                          const uint64_t *pk, int n_q, int K, int alpha, int limbs, int ndig, uint64_t g1, uint64_t g2,
                          int B);
// measured rates of Shoup products and 128-bit multiply-accumulates on every SM (per second)
void alu_calibrate(const LaunchCtx &c, uint64_t q, double *shoup_per_s, double *mac_per_s);
void launch_moddown_final_mux(const LaunchCtx &c, View out, View acc, View conv, const ModDownTable *tab, int B,
                              int limbs, View src, const uint64_t *v, const Scalars &cs, uint64_t g1, uint64_t g2);
// slots[r*S + t*beta + j] = bits[r*hh + t] for j < beta (masks expanded over the packed matrices)
void launch_expand_masks(const LaunchCtx &c, double *slots, const uint8_t *bits, int m, int hh, int beta, size_t S);
void launch_relin_rs_top(const LaunchCtx &c, View acc, View d, const RelinRescaleTable *tab, int B, int limbs);
void launch_relin_rs_final(const LaunchCtx &c, View out, View acc, View d, View conv, const RelinRescaleTable *tab,
                           int B, int limbs);
void launch_rescale_prep(const LaunchCtx &c, View r, View xtop, const RescaleTable *tab, int B, int comps, int top,
                         const Scalars *sc = nullptr);
void launch_rescale_final(const LaunchCtx &c, View out, View in, View r, const RescaleTable *tab, int B, int comps,
                          int top, const Scalars *sc = nullptr);
void launch_keygen_b(const LaunchCtx &c, uint64_t *b, const uint64_t *a, const uint64_t *e, const uint64_t *s,
                     const uint64_t *sp, const uint64_t *gadget_mask, int rows, const int *prime_of_row_dev,
                     bool to_mont);
void launch_encrypt_combine(const LaunchCtx &c, uint64_t *ct, const uint64_t *v, const uint64_t *e0,
                            const uint64_t *e1, const uint64_t *m, const uint64_t *pk, int n_q, int limbs);
void launch_signed_to_rows(const LaunchCtx &c, uint64_t *out, const int64_t *in, int rows, int n_in_polys,
                           size_t in_stride, const int *prime_dev);
void launch_to_mont(const LaunchCtx &c, uint64_t *p, int rows, const int *prime_dev);

// ---- error handling -------------------------------------------------------------
void set_error(const std::string &msg);
struct Error {
    hx_status code;
    std::string msg;
};
#define HX_CUDA(call)                                                                                      \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess)                                                                             \
            throw ::hx::Error{HX_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};              \
    } while (0)
#define HX_CHECK(cond, code, msg)                                                                          \
    do {                                                                                                   \
        if (!(cond)) throw ::hx::Error{code, msg};                                                         \
    } while (0)

} // namespace hx

namespace hx {
// rows r of out/a/b modulo prime r: out = a * b
void launch_mul_rows(const LaunchCtx &c, uint64_t *out, const uint64_t *a, const uint64_t *b, int rows);
// out[b][0] = c0 limb 0, out[b][1+p] = c1 limb 0 * share_p (NTT form, prime 0)
void launch_ddec_shares(const LaunchCtx &c, uint64_t *out, View ct, const uint64_t *shares, int n_parties, int B);
} // namespace hx
