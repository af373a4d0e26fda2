// Host runtime: context, keys, batched ciphertext buffers and the evaluator.
#pragma once
#include <map>
#include <tuple>
#include <cstdint>
#include <memory>
#include <mutex>
#include <vector>

#include "host_math.h"
#include "internal.h"

namespace hx {

enum Counter { C_ADD, C_MULPT, C_ROT, C_ROT_HOIST, C_MULCT, C_KS, C_MODUP, C_RESCALE, C_REFRESH, C_LAUNCH, C_NUM };

// stream-ordered device allocation (cudaMallocAsync on the device's pool)
struct DevBuf {
    uint64_t *p = nullptr;
    size_t words = 0;
    cudaStream_t stream = nullptr;
    bool pooled = true;  // false: plain cudaMalloc (outlives graph captures)
    bool owned = true;   // false: a view into a buffer someone else keeps alive
    DevBuf(size_t w, cudaStream_t s);
    DevBuf(size_t w, bool persistent);
    DevBuf(uint64_t *view, size_t w) : p(view), words(w), pooled(false), owned(false) {}
    ~DevBuf();
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
};
typedef std::shared_ptr<DevBuf> BufPtr;

// `B` ciphertexts (or 3-component tensors) of `comps` x `limbs` rows; storage
// [B][comps][cap][N] so that a level drop keeps the buffer.
struct Cts {
    BufPtr buf;
    uint64_t *d = nullptr;
    int B = 0, comps = 2, limbs = 0, cap = 0;
    double scale = 0;
    size_t cstride(int N) const { return (size_t)cap * N; }
    size_t bstride(int N) const { return (size_t)comps * cap * N; }
    View view(int N) const { return View{d, bstride(N), cstride(N)}; }
};

struct SwitchKey {
    BufPtr buf;  // [dnum][2][n_all][N] Montgomery form
};

} // namespace hx

namespace hx {
struct EncTables {  // device tables of the client-side encoder
    BufPtr roots, e, th;
};
// a second stream paired with a caller's stream, for independent chains of one
// schedule (fork/join by events; inside a capture it joins the same graph)
struct SideStream {
    cudaStream_t s = nullptr, s2 = nullptr;  // two side streams
    cudaEvent_t e[8] = {};
};
} // namespace hx

struct hx_context {
    int log_n = 0, N = 0, n_q = 0, K = 0, n_all = 0, dnum = 0;
    int alpha = 0;  // primes per key-switching digit (dnum = ceil(n_q / alpha))
    std::vector<uint64_t> primes;  // Q then P
    std::vector<uint64_t> psi;
    double scale = 0, sigma = 0;
    std::vector<hx::PrimeConst> h_primes;
    std::vector<hx::ConvTable> h_modup;        // [(n_q+1) * dnum]
    std::vector<hx::ModDownTable> h_moddown;   // [n_q+1]
    std::vector<hx::RescaleTable> h_rescale;   // [n_q+1]
    std::vector<hx::RelinRescaleTable> h_relin_rs;  // [n_q+1]
    hx::DeviceTables t;
    hx::DeviceTables *t_dev = nullptr;
    int *d_prime_ids = nullptr;                // 0..n_all-1
    std::unique_ptr<hx::Encoder> enc;
    std::unique_ptr<hx::GaussianCdt> cdt;
    std::atomic<uint64_t> counters[hx::C_NUM] = {};
    // cached plans by (kind, h, limbs), shared with the calls that use them; beyond
    // plan_limit bytes the least recently used plans that no call holds are freed
    struct PlanEntry {
        std::shared_ptr<hx_matmul_plan> p;
        uint64_t last = 0;
        size_t bytes = 0;
    };
    std::mutex plan_mu;  // guards the fields below
    std::map<std::tuple<int, int, int>, PlanEntry> plans;
    size_t plan_limit = SIZE_MAX, plan_bytes = 0;
    uint64_t plan_tick = 0, plan_evictions = 0;
    cudaStream_t plan_stream = nullptr;  // builds cached plans; their masks are freed in its order
    // the encoder's real coefficients (double-double) of every mask of a plan shape (kind, h,
    // Alg. 3 or not), in plan order: a plan at any level only scales and rounds them (guarded by
    // mask_real_mu)
    std::mutex mask_real_mu;
    std::map<std::tuple<int, int, bool>, hx::BufPtr> mask_real;
    std::vector<std::shared_ptr<const hx_matmul_plan>> plans_pinned;  // used inside a stream capture
    int device = 0;
    hx::Profiler prof;
    bool profiling = false;
    std::once_flag enc_once;
    hx::EncTables enc_dev;
    std::mutex side_mu;
    std::map<cudaStream_t, hx::SideStream> side;         // keyed by the caller's stream
    std::map<cudaStream_t, hx::SideStream> side_serial;  // profiling: the caller's stream itself
    std::vector<cudaStream_t> group_streams;  // groups of one batched call run side by side (guarded by side_mu)
};

struct hx_keyset {
    hx_context *ctx = nullptr;
    uint64_t uid = 0;  // unique per keyset of the process (plans bound to keys check it)
    int n_parties = 0;
    uint64_t seed = 0;
    std::vector<std::vector<int64_t>> s_parts;  // ternary shares
    std::vector<int64_t> s;                     // sum of the shares
    hx::BufPtr s_ntt;                           // [n_all][N]
    hx::BufPtr s_parts0;                        // [n_parties][N] share mod q_0, NTT form
    hx::BufPtr pk;                              // [2][n_q][N]
    hx::SwitchKey relin;
    std::map<uint64_t, hx::SwitchKey> rot;      // galois element -> key
};

struct hx_ct {
    hx_context *ctx = nullptr;
    hx::Cts c;  // B = 1
};

struct hx_matmul_exec {
    hx_context *ctx = nullptr;
    const hx_keyset *ks = nullptr;
    const hx_matmul_plan *plan = nullptr;
    size_t count = 0;
    hx::Cts A, B, out;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    int64_t launches = 0;
};

struct hx_matmul_plan {
    hx_context *ctx = nullptr;
    int kind = 0;  // 0: HE-MatMult (Alg. 3), 1: transpose (App. C)
    int h = 0, limbs = 0, beta = 0, b = 0;
    bool alg3 = true;
    struct Mask {
        int kind;  // 0 mu, 1 zeta, 2 v, 3 transpose diagonal
        int index;
        int limbs;
        bool extended;  // stored over the special primes, then q_0..q_{limbs-1}
        double scale;
        std::vector<int32_t> vec;  // logical 0/1 vector of length h^2
        hx::BufPtr pt;             // [limbs][N] Montgomery form, NTT
    };
    std::vector<Mask> masks;
    std::map<std::pair<int, int>, int> index;
    // Step 2 selection folded into the rotation keys of one keyset (optional):
    // premasked[k] = [2][ndig][2][ext][N], v_k * swk(k) and (c - v_k) * swk(k-h)
    uint64_t bound_uid = 0;
    std::vector<hx::BufPtr> premasked;
    std::vector<hx::BufPtr> storage;  // batched mask buffers the masks' views point into
    // a plan for a lower level is a view of the top-level plan of its shape: its masks are the
    // first rows of the base plan's (mask coefficients do not depend on the level)
    std::shared_ptr<const hx_matmul_plan> base;
};

namespace hx {

// ---- evaluator (eval.cu) ----------------------------------------------------
struct Eval {
    hx_context &ctx;
    cudaStream_t s;
    LaunchCtx lc()
    {
        return LaunchCtx{ctx.log_n, ctx.N, &ctx.t, s, &ctx.counters[C_LAUNCH], ctx.profiling ? &ctx.prof : nullptr};
    }
    Eval(hx_context &c, cudaStream_t st) : ctx(c), s(st) {}

    Cts alloc(int B, int comps, int limbs);
    Cts add(const Cts &a, const Cts &b, bool sub = false);
    void add_inplace(Cts &a, const Cts &b);
    Cts mul_plain(const Cts &a, const uint64_t *pt_mont, double pt_scale);
    Cts mul_int(const Cts &a, int64_t c, double new_scale = 0);
    Cts add_const(const Cts &a, double value);
    // mont: the products times 2^-64 (Montgomery form), for a sum scaled back once by from_mont
    Cts tensor(const Cts &a, const Cts &b, bool mont = false);
    void tensor_acc(Cts &acc, const Cts &a, const Cts &b, bool mont = false);
    void from_mont(Cts &a);  // a *= 2^64, in place
    Cts relinearize(const Cts &d, const SwitchKey &rk);
    Cts rescale(const Cts &a, int64_t c = 1);  // rescale(c * a), c an integer scalar
    Cts relin_rescale(const Cts &d, const SwitchKey &rk);  // rescale(relinearize(d)) as one division
    Cts drop(const Cts &a, int limbs);  // shares storage
    Cts copy(const Cts &a);
    Cts rotate(const Cts &a, int64_t k, const hx_keyset &ks);
    std::vector<Cts> rotate_hoisted(const Cts &a, const std::vector<int64_t> &ks, const hx_keyset &keys);
    // hoisting in two steps: the ModUp of c1 once, then any number of rotations
    BufPtr hoist(const Cts &a);
    Cts rotate_hoisted_one(const Cts &a, const BufPtr &D, int64_t k, const hx_keyset &keys);
    // v . Rot(a, k1) + (1 - v) . Rot(a, k2) from the ModUp D of a; the selection is applied in
    // the extended basis before one ModDown; v_ext: mask over P then Q_l (Montgomery), encoded
    // at scale v_scale whose integer value is c.  premasked (optional): the two rotation keys
    // already multiplied by v and c - v (premask_keys), so the inner product gives the selection
    Cts hoisted_mux(const Cts &a, const BufPtr &D, int64_t k1, int64_t k2, const uint64_t *v_ext, double v_scale,
                    uint64_t c, const hx_keyset &keys, const uint64_t *premasked = nullptr);
    void check_same(const Cts &a, const Cts &b);

    // hybrid key switching pieces
    BufPtr modup(const View &d, int B, int limbs);
    Cts ks_finish(const BufPtr &D, const View &dnt, int B, int limbs, const SwitchKey &key, uint64_t g,
                  const View &add, int add_mask, uint64_t add_g);
    // ModDown of an extended-basis pair accv ([B][2][limbs+K][N]) plus `add`
    Cts moddown_add(const View &accv, int B, int limbs, const View &add, int add_mask, uint64_t add_g);
    // sum_i Rot(ct_i, k_i) with a single ModDown (terms with k = 0 are added unrotated)
    Cts rotate_sum(const std::vector<std::pair<Cts, int64_t>> &items, const hx_keyset &keys);
    void ntt_inplace(uint64_t *p, size_t gstride, int groups, const std::vector<int> &rows_off,
                     const std::vector<int> &rows_prime, bool inverse);
    void ntt_oop(const uint64_t *src, size_t sgs, uint64_t *dst, size_t dgs, int groups,
                 const std::vector<int> &src_off, const std::vector<int> &dst_off, const std::vector<int> &prime,
                 bool inverse);
    const SwitchKey &rot_key(const hx_keyset &ks, uint64_t g);
};

// one rotation of a several-ring call: a ciphertext batch of its context, by `step` slots
struct RotateJob {
    hx_context *ctx;
    const hx_keyset *ks;
    Cts a;
    int64_t step;
};
// the rotations, every stage of their key switches one launch over all jobs (multi.cu)
std::vector<Cts> rotate_jobs(const std::vector<RotateJob> &jobs, cudaStream_t s);

Scalars scalars_for(const hx_context &ctx, int limbs, int64_t c);
void upload_plaintext(hx_context &ctx, cudaStream_t s, const int64_t *coeffs, int limbs, uint64_t *dst_mont);
// the same over p_0..p_{K-1} then q_0..q_{limbs-1} (an extended mask's row order)
void upload_plaintext_ext(hx_context &ctx, cudaStream_t s, const int64_t *coeffs, int limbs, uint64_t *dst_mont);
// the same from N signed coefficients already on the device (extended: over the special primes too)
void plaintext_from_device(hx_context &ctx, cudaStream_t s, const int64_t *dcoeffs, int limbs, bool extended,
                           uint64_t *dst);

// ---- keys / encryption (keys.cu) ---------------------------------------------
void keygen(hx_context &ctx, hx_keyset &ks, int n_parties, uint64_t seed, cudaStream_t s);
void add_rotation_keys(hx_context &ctx, hx_keyset &ks, const std::vector<int64_t> &steps, cudaStream_t s);
Cts encrypt_coeffs(hx_context &ctx, const hx_keyset &ks, const int64_t *m, double scale, int limbs, uint64_t seed,
                   uint32_t tag, uint32_t index, cudaStream_t s);
// centered coefficients of c0 + c1 s mod q_0 for every batch entry: [B][N]
std::vector<int64_t> decrypt_coeffs(hx_context &ctx, const hx_keyset &ks, const Cts &c, cudaStream_t s);
Cts dkeyswitch(hx_context &ctx, const hx_keyset &from, const hx_keyset &to, const Cts &ct, uint64_t seed,
               cudaStream_t s);
Cts dbootstrap(hx_context &ctx, const hx_keyset &ks, const Cts &ct, const std::vector<uint64_t> &seeds, int counter,
               cudaStream_t s);

// ---- schedules (schedules.cu) -------------------------------------------------
hx_matmul_plan *make_plan(hx_context &ctx, int h, int limbs, cudaStream_t s);
// the context's plan for (h, limbs) with library masks, built on first use (thread-safe)
std::shared_ptr<const hx_matmul_plan> cached_plan(hx_context &ctx, int h, int limbs);
void trim_plan_cache(hx_context &ctx);  // caller holds plan_mu
// keeps a cached plan referenced until stream s has run the work enqueued so far
// (does not throw; on failure it waits for s)
void hold_plan_until(hx_context &ctx, cudaStream_t s, std::shared_ptr<const hx_matmul_plan> p) noexcept;
// a cached plan for one call on stream s, held past the call's work however the call ends
struct PlanUse {
    hx_context &ctx;
    cudaStream_t s;
    std::shared_ptr<const hx_matmul_plan> p;
    PlanUse(hx_context &c, cudaStream_t st, std::shared_ptr<const hx_matmul_plan> q) : ctx(c), s(st), p(std::move(q)) {}
    ~PlanUse() { hold_plan_until(ctx, s, std::move(p)); }
    PlanUse(const PlanUse &) = delete;
    PlanUse &operator=(const PlanUse &) = delete;
};
hx_matmul_plan *make_transpose_plan(hx_context &ctx, int h, int limbs, cudaStream_t s);
std::shared_ptr<const hx_matmul_plan> cached_transpose_plan(hx_context &ctx, int h, int limbs);
std::vector<int64_t> transpose_rotation_steps(int h, int beta);
Cts transpose_batch(hx_context &ctx, const hx_keyset &ks, const hx_matmul_plan &plan, const Cts &x, cudaStream_t s);
std::vector<int64_t> plan_rotation_steps(int h, int beta, int limbs, int t = 0);  // t = 0: t = h
Cts matmul_batch(hx_context &ctx, const hx_keyset &ks, const hx_matmul_plan &plan, const Cts &A, const Cts &B,
                 cudaStream_t s, int t = 0);  // t < h: the cut k-sum of the rectangular product
// folds the Step 2 selection masks of plan into copies of the rotation keys of ks
void bind_plan_keys(hx_context &ctx, hx_matmul_plan &plan, const hx_keyset &ks, cudaStream_t s);
Cts rmatmul_batch(hx_context &ctx, const hx_keyset &ks, const hx_matmul_plan &plan, const Cts &At, const Cts &B, int t,
                  cudaStream_t s);
// refresh randomness of entry b: SplitMix64 streams keyed by refresh_seeds[b] (tag 1 + refresh index)
Cts sign_batch(hx_context &ctx, const hx_keyset &ks, const Cts &x, int d, int k, bool relu, bool allow_refresh,
               const std::vector<uint64_t> &refresh_seeds, cudaStream_t s);
struct DenseResult {
    Cts E, M, dW;
};
// the encodings' real coefficients before the scale, double-double (hi, lo) per coefficient
void encode_real_batch(hx_context &ctx, const double *slots_dev, size_t n_slots, int count, double2 *m_out,
                       cudaStream_t s);
void encode_rows_from_real(hx_context &ctx, const double2 *m, const int *idx_dev, int count, double scale,
                           int64_t *out, cudaStream_t s);
void encode_batch(hx_context &ctx, const double *slots_dev, size_t n_slots, int count, double scale, int64_t *out,
                  size_t out_stride, cudaStream_t s);
Cts encrypt_batch(hx_context &ctx, const hx_keyset &ks, const double *slots_dev, size_t n_slots, int count, int limbs,
                  const uint64_t *seeds, cudaStream_t s);
struct DensePlans {
    const hx_matmul_plan *fwd = nullptr, *transpose = nullptr, *bwd = nullptr;  // null: the cached plan
};
DenseResult dense_batch(hx_context &ctx, const hx_keyset &ks, const DensePlans &plans, const Cts &W, const Cts &X,
                        const Cts &G, int h, int d, int k, double input_div, uint64_t refresh_seed, cudaStream_t s);
std::vector<int64_t> dense_rotation_steps(int h, int beta);
Cts aggregate(hx_context &ctx, const std::vector<const Cts *> &grads, int n_parties, const Cts &models, double c_real,
              cudaStream_t s);

// ---- context (context.cu) -------------------------------------------------------
// the side stream paired with `main` (created on first use, destroyed with the context)
SideStream &side_stream(hx_context &ctx, cudaStream_t main);
// stream i of the context's pool for the independent groups of one batched call (created on first
// use, destroyed with the context); while profiling, `main` itself, so the groups run in turn
cudaStream_t group_stream(hx_context &ctx, cudaStream_t main, size_t i);
void build_context(hx_context &ctx, const hx_params &p);
void destroy_context(hx_context &ctx);
Cts gather(hx_context &ctx, const hx_ct *const *cts, size_t count, cudaStream_t s);
void scatter(hx_context &ctx, const Cts &b, hx_ct **out, cudaStream_t s);

} // namespace hx
