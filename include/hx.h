/*
 * hx -- GB300-native RNS-CKKS evaluation for the Hercules packed matrix
 * product and composite-polynomial sign/ReLU (arXiv 2207.04620).
 *
 * C ABI.  Plain pointers and sizes only.  All handles are opaque and owned
 * by the library; free them with the matching *_destroy.  Functions return
 * HX_OK (0) or a negative hx_status; on error no output handle is produced
 * (*out stays NULL) and hx_last_error() describes the failure (thread-local
 * string, valid until the next call on the same thread).
 *
 * Streams: a `void* stream` argument is a cudaStream_t (NULL = legacy default
 * stream).  Device work is enqueued on it; results held in handles are valid
 * once that stream has completed.  Host buffers passed in are borrowed for the
 * duration of the call only.
 *
 * Ciphertexts live in device memory, limb-major: component c, limb l,
 * coefficient slot j at word (c*limbs + l)*N + j, every limb in the NTT
 * (evaluation) representation: slot j of limb l holds a(psi_l^(2 brv(j)+1))
 * mod q_l.  Limb l of a ciphertext with `limbs` limbs is modulo q_l; the
 * special primes p_k follow the Q primes in every prime list.
 *
 * Paper references: Fig. 1 (the MCKKS API, Sec. 2.2) defines SecKeyGen,
 * DKeyGen, Ecd/Dcd, Enc, DDec, Add, Sub, Mul_pt, Mul_ct, Rot, RS; Alg. 2/3,
 * Eqs. (5)-(16), App. B and App. E define the packed h x h product; Sec. 4
 * and Alg. 5 define g_d, its k-fold composition and ReLU.
 */
#ifndef HX_H
#define HX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int hx_status;
#define HX_OK 0
#define HX_EINVAL (-1)   /* bad argument, shape or parameter */
#define HX_ENOMEM (-2)   /* device allocation failed or HBM budget exceeded */
#define HX_ELEVEL (-3)   /* not enough levels (limbs) left for the operation */
#define HX_ESCALE (-4)   /* operands' scales or levels do not match */
#define HX_EKEY (-5)     /* a needed rotation or relinearisation key is missing */
#define HX_ETIMEOUT (-6) /* a bounded device wait gave up */
#define HX_ECUDA (-7)    /* a CUDA runtime call failed */
#define HX_EPARTY (-8)   /* a party's share is missing in a collective step */

#define HX_MAX_Q 60
#define HX_MAX_P 6

typedef struct hx_context hx_context;
typedef struct hx_keyset hx_keyset;
typedef struct hx_ct hx_ct;
typedef struct hx_matmul_plan hx_matmul_plan;

/* Parameters (Sec. 2.2: R_Q = Z_Q[X]/(X^N+1), Q = q_0...q_{L-1}).
 * log_n in [11, 16]; n_q Q primes of q_bits[i] bits (q_0 first), n_p special
 * primes of p_bits[k] bits (hybrid key switching); key-switching digits of
 * alpha consecutive Q primes (0 = n_p; at most 7; a digit's product should
 * stay near or below the special primes' product, or the switch adds noise
 * in proportion); every size in [20, 61].  Primes: for each size in this order, the largest
 * prime below 2^bits that is 1 mod 2N and not yet chosen.  Default encoding
 * scale 2^log2_scale; error sampler width sigma (discrete Gaussian on
 * [-floor(6 sigma), floor(6 sigma)]). */
typedef struct hx_params {
    int log_n;
    int n_q;
    int q_bits[HX_MAX_Q];
    int n_p;
    int p_bits[HX_MAX_P];
    double log2_scale;
    double sigma;
    int alpha;  /* primes per key-switching digit; 0 = n_p */
} hx_params;

const char *hx_last_error(void);

/* ---- context -------------------------------------------------------------- */
/* Builds primes, roots, NTT twiddles and RNS conversion tables on the current
 * CUDA device.  Returns HX_EINVAL for unsupported parameters. */
hx_status hx_context_create(const hx_params *p, hx_context **out);
void hx_context_destroy(hx_context *ctx);
/* Writes the n_q + n_p primes (Q then P) to out[0..cap); returns the count or
 * a negative status. */
int hx_context_primes(const hx_context *ctx, uint64_t *out, int cap);
/* ring degree N */
int hx_context_n(const hx_context *ctx);

/* ---- keys (Fig. 1 items 1-2; host-side toy-scale multiparty) -------------- */
/* SecKeyGen for n_parties simulated parties (ternary shares), DKeyGen of the
 * collective public key for s = sum of shares, the relinearisation key and
 * one Galois key per entry of rot_steps (rotation by k slots to the left,
 * i.e. R(m, k) of Sec. 3.2; k is taken mod N/2).  Randomness: SplitMix64
 * streams derived from `seed`.  Evaluation keys are uploaded to HBM. */
hx_status hx_keygen(hx_context *ctx, int n_parties, uint64_t seed, const int32_t *rot_steps, size_t n_steps,
                    hx_keyset **out);
/* Adds Galois keys for more rotation steps (no-op for present ones). */
hx_status hx_keyset_add_rotations(hx_context *ctx, hx_keyset *ks, const int32_t *rot_steps, size_t n_steps);
/* Exports a switching key (galois = 0: relinearisation key) in the library's
 * canonical layout [dnum][2 (b, a)][n_q + n_p][N] (NTT form, standard
 * residues) into host memory; returns words written or a negative status. */
int64_t hx_keyset_export_switch_key(const hx_keyset *ks, uint64_t galois, uint64_t *host, size_t cap);
/* Exports the public key [2 (b, a)][n_q][N]. */
int64_t hx_keyset_export_public_key(const hx_keyset *ks, uint64_t *host, size_t cap);
void hx_keyset_destroy(hx_keyset *ks);
/* Keyset checkpoint: keys are a deterministic function of (seed, parties,
 * Galois elements), so the file holds that recipe: "HXKS0001", u32 log_n,
 * n_q, n_p, n_parties, u64 seed, u32 n_galois, alpha (primes per digit), the
 * u64 moduli of Q then P,
 * the u64 Galois elements of the rotation keys ascending, little-endian.
 * Loading checks the magic, ring, chain and moduli against the context and
 * regenerates the same keys (HX_EINVAL for a file of another context). */
hx_status hx_keyset_save(hx_context *ctx, const hx_keyset *ks, const char *path);
hx_status hx_keyset_load(hx_context *ctx, const char *path, hx_keyset **out);

/* ---- encoding / encryption / decryption (Fig. 1 items 3-6) ---------------- */
/* Ecd: n <= N/2 real slots -> N signed integer coefficients at `scale`
 * (canonical embedding, slot j at zeta^(5^j), rounding half away from zero). */
hx_status hx_encode(const hx_context *ctx, const double *slots, size_t n, double scale, int64_t *coeffs);
/* Enc(pk, Ecd(slots)) at `limbs` limbs (0 = all Q primes), default scale. */
hx_status hx_encrypt(hx_context *ctx, const hx_keyset *ks, const double *slots, size_t n, int limbs, uint64_t seed,
                     hx_ct **out);
/* Client side on the device: Ecd of `count` slot vectors (host, [count][n],
 * n <= N/2, N >= 512) by a batched 2N-point FP64 FFT that repeats the host
 * encoder's operations one by one, so coeffs ([count][N], host) equal
 * hx_encode's bit for bit; HX_EINVAL if a coefficient reaches 2^62. */
hx_status hx_encode_batch(hx_context *ctx, const double *slots, size_t n, size_t count, double scale, int64_t *coeffs,
                          void *stream);
/* Enc(pk, Ecd(slots_i)) for i < count with the device encoder and the
 * encryption randomness drawn on the device from the same SplitMix64 streams
 * (seed seeds[i], tag 0, index 0): out[i] equals hx_encrypt(..., seeds[i]). */
hx_status hx_encrypt_batch(hx_context *ctx, const hx_keyset *ks, const double *slots, size_t n, size_t count, int limbs,
                           const uint64_t *seeds, hx_ct **out, void *stream);
/* Enc(pk, m) for N signed integer coefficients m at `scale`; tag/index select
 * the SplitMix64 streams of the encryption randomness. */
hx_status hx_encrypt_coeffs(hx_context *ctx, const hx_keyset *ks, const int64_t *coeffs, double scale, int limbs,
                            uint64_t seed, uint32_t tag, uint32_t index, hx_ct **out);
/* DDec: every simulated party's share c1*s_i is computed on the device, the
 * shares are summed with c0 on the host modulo q_0 and decoded (Dcd).  Writes
 * min(n, N/2) real slots. */
hx_status hx_decrypt(hx_context *ctx, const hx_keyset *ks, const hx_ct *ct, double *slots, size_t n);
/* The same collective decryption stopped before decoding: N centered integer
 * coefficients of c0 + c1*s mod q_0. */
hx_status hx_decrypt_coeffs(hx_context *ctx, const hx_keyset *ks, const hx_ct *ct, int64_t *coeffs);

/* Collective decryption (DDec, Sec. 2.2) with the parties that actually sent
 * their shares: present[i] != 0 for party i, n_present = the key set's party
 * count (HX_EINVAL otherwise).  Every party's share is needed; a missing one
 * returns HX_EPARTY, naming the party, before any work.  Otherwise as
 * hx_decrypt. */
hx_status hx_decrypt_parties(hx_context *ctx, const hx_keyset *ks, const hx_ct *ct, const uint8_t *present,
                             size_t n_present, double *slots, size_t n);

/* ---- ciphertext handles ---------------------------------------------------- */
/* Import residues [comps][limbs][N] (NTT form) from host memory. */
hx_status hx_ct_import(hx_context *ctx, const uint64_t *host, int comps, int limbs, double scale, hx_ct **out);
/* Export residues [comps][limbs][N]; returns words written or a negative status. */
int64_t hx_ct_export(const hx_ct *ct, uint64_t *host, size_t cap);
hx_status hx_ct_info(const hx_ct *ct, int *comps, int *limbs, double *scale);
/* Checkpoint a ciphertext to a file / restore it: "HXCT0001", then u32 log_n,
 * comps, limbs, 0, f64 scale, the u64 moduli of its limbs, and the residues
 * [comps][limbs][N] (NTT form), little-endian.  Loading checks the magic, the
 * ring degree and the moduli against the context (HX_EINVAL otherwise).  Keys
 * are not stored: keygen is deterministic in (seed, parties, steps). */
hx_status hx_ct_save(hx_context *ctx, const hx_ct *ct, const char *path);
hx_status hx_ct_load(hx_context *ctx, const char *path, hx_ct **out);

void hx_ct_destroy(hx_ct *ct);

/* ---- single operations on handles (Fig. 1 items 7-12) ----------------------- */
/* Add/Sub need equal limbs and scales within a relative 2^-20 (else
 * HX_ESCALE); the output scale is a's. */
hx_status hx_add(hx_context *ctx, const hx_ct *a, const hx_ct *b, hx_ct **out, void *stream);
hx_status hx_sub(hx_context *ctx, const hx_ct *a, const hx_ct *b, hx_ct **out, void *stream);
/* Mul_pt with the plaintext of N signed coefficients pt encoded at pt_scale. */
hx_status hx_mul_plain(hx_context *ctx, const hx_ct *a, const int64_t *pt, double pt_scale, hx_ct **out,
                       void *stream);
/* multiplication by an integer constant; new_scale <= 0 keeps the scale */
hx_status hx_mul_int(hx_context *ctx, const hx_ct *a, int64_t c, double new_scale, hx_ct **out, void *stream);
/* adds the constant round(value * scale) to every slot */
hx_status hx_add_const(hx_context *ctx, const hx_ct *a, double value, hx_ct **out, void *stream);
/* Mul_ct without relinearisation: 3 components (d0, d1, d2). */
hx_status hx_tensor(hx_context *ctx, const hx_ct *a, const hx_ct *b, hx_ct **out, void *stream);
/* 3 components -> 2 by hybrid key switching of d2 with the relinearisation key. */
hx_status hx_relinearize(hx_context *ctx, const hx_keyset *ks, const hx_ct *d, hx_ct **out, void *stream);
/* RS: divide by the top prime with rounding to nearest and drop it. */
hx_status hx_rescale(hx_context *ctx, const hx_ct *a, hx_ct **out, void *stream);
/* Relinearisation and RS of a 3-component tensor in one division: with
 * acc the key inner product of d2 (before ModDown) and y = acc + P*(d0, d1),
 * each output coefficient is round(y / (P*q_top)), one level down, scale /
 * q_top.  The remainder modulo P*q_top is converted exactly (the fast
 * conversion's overshoot is counted in FP64 and removed), so a coefficient
 * is off by one only where that FP64 sum lies within rounding of an integer.
 * One ModDown NTT pass fewer than hx_relinearize + hx_rescale; the two agree
 * within 2 per coefficient.  HX_ELEVEL at one limb. */
hx_status hx_relin_rescale(hx_context *ctx, const hx_keyset *ks, const hx_ct *d, hx_ct **out, void *stream);
/* discard the top limbs down to `limbs` (exact) */
hx_status hx_drop(hx_context *ctx, const hx_ct *a, int limbs, hx_ct **out, void *stream);
/* Rot(a, k): slots move left by k (R(m, k)); HX_EKEY without the Galois key. */
hx_status hx_rotate(hx_context *ctx, const hx_keyset *ks, const hx_ct *a, int32_t k, hx_ct **out, void *stream);
/* One rotation of a several-ring call: ciphertext ct of context ctx rotated by
 * `step` slots with ctx's key set ks. */
typedef struct {
    hx_context *ctx;
    const hx_keyset *ks;
    const hx_ct *ct;
    int64_t step;
} hx_rotate_job;
/* Rot (Fig. 1 item 11) of ciphertexts of any contexts (ring degrees 2^11 ..
 * 2^16, prime chains, levels) in one call.  Each stage of their hybrid key
 * switches runs as one launch over every job: the automorphism, ModUp's
 * inverse NTT, basis conversion and NTT, the key inner product, ModDown's
 * inverse NTT, conversion and NTT, and the epilogue (13 launches in all).  The
 * stage kernels run the bodies of the one-ring ones, so out[i] (a handle of
 * jobs[i].ctx) equals hx_rotate of job i residue for residue.  A step of 0
 * mod N/2 copies.  The contexts must share one device.  Every check (null
 * fields, handles of another context, HX_EKEY for a missing Galois key) comes
 * before any device work; on an error no output is set.  count <= 65535. */
hx_status hx_rotate_jobs(const hx_rotate_job *jobs, size_t count, hx_ct **out, void *stream);
/* n rotations of one ciphertext sharing a single ModUp of c1 (hoisting). */
hx_status hx_rotate_hoisted(hx_context *ctx, const hx_keyset *ks, const hx_ct *a, const int32_t *steps, int n,
                            hx_ct **outs, void *stream);

/* Rotation that allocates no device memory.  The paper has no counterpart:
 * this serves callers that cannot request device memory when they rotate (a
 * process whose memory manager already holds the device, a latency-bound
 * loop that must avoid cudaMalloc's synchronisation, a host that forbids
 * plug-ins from allocating after start-up).  `in` and `out` are device
 * buffers of one ciphertext, [2][limbs][N] words, NTT form, at `limbs`
 * limbs (distinct, caller-owned).  Every intermediate lives in one static
 * device array of HX_NOALLOC_SCRATCH_BYTES that the library holds on every
 * device it is loaded on until the process exits; a rotation needing more
 * (8*N*(4*limbs + (ceil(limbs/alpha) + 2)*(limbs + n_p)) bytes, alpha the
 * primes per key-switching digit: about 12 MB for N=2^14 at 8 limbs, 48 MB
 * for N=2^16 at 8 limbs) returns HX_EINVAL, as do keys of another context and
 * overlapping `in` and `out`.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.  All
 * calls share the array: calls whose work overlaps on the GPU (other streams,
 * other threads) race and must be serialised by the caller.  The result is
 * identical to hx_rotate's. */
#define HX_NOALLOC_SCRATCH_BYTES (16ull << 20)
hx_status hx_rotate_noalloc(hx_context *ctx, const hx_keyset *ks, const uint64_t *in, int limbs, uint64_t *out,
                            int32_t k, void *stream);

/* ---- raw kernels on caller device buffers (for parity tests and benches) --- */
/* Several rings in one launch per phase: every job's polynomials (its own
 * context, so its own N, primes and twiddles) are transformed in place by one
 * column-phase and one row-phase launch over the tiles of all jobs, with the
 * same residues as hx_ntt on each job.  data: device [n_polys][n_limbs][N]
 * words; prime_idx: host, n_limbs prime indices (rows of a polynomial).
 * N from 2^11 to 2^16; all contexts on the current device; returns after the
 * launches (the job table is staged on the stream). */
typedef struct hx_ntt_job {
    const hx_context *ctx;
    uint64_t *data;
    int n_polys;
    int n_limbs;
    const int32_t *prime_idx;
} hx_ntt_job;
hx_status hx_ntt_multi(const hx_ntt_job *jobs, int n_jobs, int inverse, void *stream);

/* In-place forward (inverse != 0: inverse) negacyclic NTT of n_polys
 * polynomials laid out [n_polys][limbs][N] in device memory; limb l is taken
 * modulo prime index prime_idx[l] (host array; index into Q then P). */
hx_status hx_ntt(hx_context *ctx, uint64_t *dev, int n_polys, int limbs, const int32_t *prime_idx, int inverse,
                 void *stream);

/* The cached HE-MatMult and transpose plans (encoded masks, one per (h, level))
 * that hx_matmul, the batch calls without a plan, the dense layer and the
 * server build on first use.  bytes > 0 caps the device memory they hold: past
 * it the least recently used plans that no call is using are freed (a call
 * keeps its plan until its stream has run the work that reads it; plans used
 * inside a stream capture stay for the context's life); 0 = no cap (the
 * default).  Info: plans, bytes held, cap (0 = none), plans freed so far;
 * returns the count (4). */
hx_status hx_context_set_plan_cache(hx_context *ctx, uint64_t bytes);
int hx_context_plan_cache_info(hx_context *ctx, uint64_t *out, int cap);

/* ---- HE-MatMult (Alg. 3 with App. B and App. E) ----------------------------- */
/* A plan fixes h (a power of two, h*h <= N/2, beta = (N/2)/h^2 products per
 * ciphertext pair) and the input level.  limbs >= 4 runs Alg. 3; limbs == 3
 * runs the depth-2 rearrangement; fewer returns HX_ELEVEL.  Its diagonal
 * masks are encoded by the library at one fixed scale, 2^round(log2 scale) of
 * the context, at every level (a product's scale after a mask and a rescale by
 * q_(l-1) is scale * 2^e / q_(l-1), carried in the ciphertext);
 * hx_matmul_plan_set_mask replaces mask i (in the plan's documented order: mu
 * diagonals l = -h+1..h-1, zeta diagonals l = 0..h-1, then for Alg. 3 the v_k
 * masks k = 1..h-1) by N signed integer coefficients, to be encoded at that
 * scale. */
hx_status hx_matmul_plan_create(hx_context *ctx, int h, int limbs, hx_matmul_plan **out);
int hx_matmul_plan_num_masks(const hx_matmul_plan *plan);
hx_status hx_matmul_plan_set_mask(hx_context *ctx, hx_matmul_plan *plan, int i, const int64_t *coeffs);
/* Folds Step 2's selection masks into copies of the rotation keys of `ks`
 * (for every k: v_k * swk(k) and (q_t - v_k) * swk(k - h) on the extended
 * basis), so each selection is one inner product over both keys and one
 * reduction instead of two inner products, two reductions and the mask
 * product.  Products with these keys give the same residues.  Costs
 * hx_matmul_plan_bound_bytes(plan) of device memory (2(h-1) masked keys at the
 * product's Step-2 level); replacing a mask with hx_matmul_plan_set_mask
 * unbinds.  Alg. 3 plans (>= 4 limbs) only. */
hx_status hx_matmul_plan_bind_keys(hx_context *ctx, hx_matmul_plan *plan, const hx_keyset *ks, void *stream);
int64_t hx_matmul_plan_bound_bytes(const hx_matmul_plan *plan);
void hx_matmul_plan_destroy(hx_matmul_plan *plan);
/* Rotation steps (mod N/2, sorted, no 0) a product of this shape uses;
 * returns the count (writes at most cap) or a negative status. */
int hx_matmul_rotation_steps(const hx_context *ctx, int h, int limbs, int32_t *out, int cap);
/* One product (Alg. 3, HE-MatMult, Sec. 3.3: A.B = sum_k phi^k(mu(A)) (.)
 * pi^k(zeta(B)), Eq. (2), with the baby-step/giant-step linear transforms of
 * App. B and the ι_β packing of App. E): out = A x B for each of the beta
 * packed pairs.  A and B: ciphertexts of this context at one level (at least 4
 * limbs for Alg. 3, exactly 3 for the depth-2 form) and scale; the plan is the
 * context's cached one for (h, level).  HX_EKEY if a rotation key of
 * hx_matmul_rotation_steps is missing. */
hx_status hx_matmul(hx_context *ctx, const hx_keyset *ks, const hx_ct *A, const hx_ct *B, int h, hx_ct **out,
                    void *stream);
/* `count` independent products (Alg. 3 with App. B and App. E, as hx_matmul)
 * through one batched schedule: every kernel launch covers the whole batch
 * and key reads are shared.  A[i], B[i]: ciphertexts of this context, all at
 * one level and scale (HX_ESCALE otherwise).  plan may be NULL (the context's
 * cached plan with library masks for the inputs' level).  out: `count` new
 * handles, valid when `stream` completes; on error every out[i] is NULL. */
hx_status hx_matmul_batch(hx_context *ctx, const hx_keyset *ks, const hx_matmul_plan *plan, const hx_ct *const *A,
                          const hx_ct *const *B, int h, size_t count, hx_ct **out, void *stream);
/* A batch with a matrix size per entry (Alg. 3 per entry, App. E packing per
 * h): entries of one (h[i], level, scale) are grouped, each group runs as one
 * batched product (cached plans), and the groups run side by side on streams
 * of the context (forked from and joined back to `stream`); out[i] is entry
 * i's product, identical to hx_matmul on that pair alone.  A[i] and B[i] must
 * share level and scale (HX_ESCALE); on any error every out[i] is NULL. */
hx_status hx_matmul_batch_mixed(hx_context *ctx, const hx_keyset *ks, const hx_ct *const *A, const hx_ct *const *B,
                                const int *h, size_t count, hx_ct **out, void *stream);
/* Products over several rings in one call (Alg. 3 per entry, App. E packing):
 * job i multiplies A and B of its own context (any ring degree, prime chain
 * and level) with that context's key set and matrix size h.  Jobs of one
 * (context, key set, h, level, scale) form a batched group; the groups run
 * side by side on streams forked from and joined back to `stream`, so
 * products of different rings and levels overlap on the device.  out[i] is
 * job i's product (a handle of job i's context), identical to hx_matmul on
 * that pair alone.  Every handle must belong to its job's context (HX_EINVAL)
 * and all contexts to one device; on any error every out[i] is NULL. */
typedef struct hx_matmul_job {
    hx_context *ctx;
    const hx_keyset *ks;
    const hx_ct *A;
    const hx_ct *B;
    int h;
} hx_matmul_job;
hx_status hx_matmul_jobs(const hx_matmul_job *jobs, size_t count, hx_ct **out, void *stream);

/* ---- rectangular product (App. D) ------------------------------------------------ */
/* Rectangular product (App. D, Alg. "41"): At[i] packs A~ = (A; ...; A), the
 * h/t vertical copies of a t x h matrix A (t a power of two dividing h), in
 * each of its beta positions; B[i] packs h x h matrices.  The result packs
 * h/t vertical copies of A.B (t x h), so it can enter another rectangular
 * product as it is.  Same plan, level and scale rules as hx_matmul_batch
 * (3 levels with >= 4 limbs, 2 with 3 limbs); Step 2/3 run t - 1 terms
 * instead of h - 1, then log2(h/t) rotate-and-add folds by t*h*2^e rows. */
hx_status hx_rmatmul_batch(hx_context *ctx, const hx_keyset *ks, const hx_matmul_plan *plan, const hx_ct *const *At,
                           const hx_ct *const *B, int h, int t, size_t count, hx_ct **out, void *stream);
/* Rotation steps of hx_rmatmul_batch at `limbs`; returns the count, writes up to cap. */
int hx_rmatmul_rotation_steps(const hx_context *ctx, int h, int t, int limbs, int32_t *out, int cap);

/* ---- transpose (App. C) ---------------------------------------------------------- */
/* A^T for each of the beta packed h x h matrices of `count` ciphertexts at one
 * level (>= 2 limbs): sum over the 2h-1 diagonals (h-1)s of U^T with the
 * baby-step/giant-step split, one rescale.  plan may be NULL (library masks);
 * a transpose plan's masks are the diagonals s = -h+1..h-1 in that order and
 * can be replaced with hx_matmul_plan_set_mask. */
hx_status hx_transpose_plan_create(hx_context *ctx, int h, int limbs, hx_matmul_plan **out);
int hx_transpose_rotation_steps(const hx_context *ctx, int h, int32_t *out, int cap);
hx_status hx_transpose(hx_context *ctx, const hx_keyset *ks, const hx_matmul_plan *plan, const hx_ct *const *x,
                       int h, size_t count, hx_ct **out, void *stream);

/* A captured batched product: the whole schedule of hx_matmul_batch for
 * `count` ciphertext pairs at the plan's level, recorded once into a CUDA graph
 * (its temporary allocations become graph memory nodes) over persistent input
 * and output buffers.  hx_matmul_exec_run copies the inputs in, launches the
 * graph on `stream` and returns fresh output handles; the residues equal
 * hx_matmul_batch's.  Runs of one executor must not overlap. */
typedef struct hx_matmul_exec hx_matmul_exec;
hx_status hx_matmul_exec_create(hx_context *ctx, const hx_keyset *ks, const hx_matmul_plan *plan, size_t count,
                                double scale, hx_matmul_exec **out);
hx_status hx_matmul_exec_run(hx_matmul_exec *ex, const hx_ct *const *A, const hx_ct *const *B, hx_ct **out,
                             void *stream);
/* kernel launches one replay contains */
int64_t hx_matmul_exec_launches(const hx_matmul_exec *ex);
void hx_matmul_exec_destroy(hx_matmul_exec *ex);
/* The same replay with host buffers: copies host_A and host_B
 * ([count][2][limbs][N] words each, the executor's level and scale) to the
 * device, replays the graph and copies the products ([count][2][out_limbs][N],
 * hx_matmul_exec_out_info) to host_out, all enqueued on `stream`; returns
 * without waiting.  The buffers must stay valid until the stream has reached
 * this point; page-locked buffers let the copies run asynchronously.  Calls on
 * one executor must be ordered (one stream, or waited for): they share its
 * device buffers.  Two executors on two streams overlap one batch's copies
 * with the other's evaluation. */
hx_status hx_matmul_exec_run_host(hx_matmul_exec *ex, const uint64_t *host_A, const uint64_t *host_B,
                                  uint64_t *host_out, void *stream);
hx_status hx_matmul_exec_out_info(const hx_matmul_exec *ex, int *limbs, double *scale);


/* ---- sign / ReLU (Sec. 4, Alg. 5) ------------------------------------------ */
/* g_d^(k)(x) (relu = 0) or ReLU(x) = x (1 + g_d^(k)(x)) / 2 (relu = 1), d in
 * [1, 4].  When the next composition no longer fits in the remaining levels,
 * the ciphertext is refreshed by the collective DBootstrap protocol
 * (hx_dbootstrap, masked decryption shares and re-encryption shares,
 * randomness from refresh_seed) if allow_refresh != 0, else HX_ELEVEL.  In the batch call,
 * entry i uses refresh_seed + i, so every entry's result equals the single
 * call's with that seed. */
hx_status hx_sign_approx(hx_context *ctx, const hx_keyset *ks, const hx_ct *x, int d, int k, int relu,
                         int allow_refresh, uint64_t refresh_seed, hx_ct **out, void *stream);
hx_status hx_sign_approx_batch(hx_context *ctx, const hx_keyset *ks, const hx_ct *const *x, size_t count, int d,
                               int k, int relu, int allow_refresh, uint64_t refresh_seed, hx_ct **out, void *stream);

/* ---- one dense layer, feedforward and backpropagation (Fig. 5) ------------------ */
/* Blocks of h x h, beta = (N/2)/h^2 per ciphertext, packed as in App. E:
 *   W[i*groups + g]  packs W_{i,j}, j = beta*g .. beta*g + beta - 1, at positions 0..beta-1
 *   X[g]             packs X_j for the same j (the inputs of a batch of h as columns)
 *   G[i]             packs the upstream gradient G_i at position 0, zero elsewhere
 * all W and X at one level and scale, G at a level no lower than the activation's.
 * Outputs (new handles, owned by the caller):
 *   E[i]   position 0: E_i = sum_j W_{i,j} X_j (other positions hold partial sums)
 *   M[i]   position 0: ReLU(E_i) = E_i (1 + s_i) / 2, s_i = g_d^(k)(E_i / input_div)
 *   dW[i*groups + g]  position p: L_i X_{beta*g+p}^T, L_i = ((1 + s_i)/2) . G_i
 * Steps: one batched HE-MatMult over all (i, g); sums over g; a rotate-and-add
 * fold of the beta positions; the composite sign (entry i refreshed with
 * refresh_seed + i, as in hx_sign_approx_batch); L_i copied to every position
 * by rotations; the X_g transposed (App. C) and brought to L's level and scale;
 * a second batched HE-MatMult.  The three plans (NULL: the context's cached
 * plan for the level reached) are a matmul plan at W's level, a transpose plan
 * at X's level and a matmul plan at L's level.  Rotation keys:
 * hx_dense_rotation_steps.
 * Errors: HX_EINVAL (shapes, h), HX_ELEVEL (chain too short), HX_EKEY. */
hx_status hx_dense_layer(hx_context *ctx, const hx_keyset *ks, const hx_matmul_plan *fwd_plan,
                         const hx_matmul_plan *transpose_plan, const hx_matmul_plan *bwd_plan, const hx_ct *const *W,
                         const hx_ct *const *X, const hx_ct *const *G, int h, int n_out, int groups, int d, int k,
                         double input_div, uint64_t refresh_seed, hx_ct **E, hx_ct **M, hx_ct **dW, void *stream);
/* Rotation steps hx_dense_layer uses (both HE-MatMult variants, the transpose,
 * and +-2^t for t < log2(beta)); returns their count, writes up to cap. */
int hx_dense_rotation_steps(const hx_context *ctx, int h, int32_t *out, int cap);

/* ---- collective protocols (Fig. 1 items 13-14, toy scale, parties simulated) ---- */
/* DKeySwitch: re-encrypts ct (under the collective key of `from`) under the
 * public key of `to` without decryption.  Party i draws u_i (ternary) and
 * e0_i, e1_i (Gaussian, the context's sigma) from SplitMix64 streams (seed,
 * purpose, i, 0) and contributes (s_i*c1 + u_i*b' + e0_i, u_i*a' + e1_i); the
 * result (c0 + sum, sum) keeps ct's level and scale and decrypts under `to`. */
hx_status hx_dkeyswitch(hx_context *ctx, const hx_keyset *from, const hx_keyset *to, const hx_ct *ct, uint64_t seed,
                        hx_ct **out, void *stream);
/* DBootstrap: collective refresh to the top level and the default scale.
 * Each party masks its decryption share at q_0 with a uniform M_i in
 * [-bound, bound], bound = (floor(q_0/4) - 1)/n_parties, so the combined value
 * is Delta_ct*m + e + sum M_i (|m| small enough that it stays below q_0/4);
 * it is rescaled to Delta and re-encrypted against a common reference
 * polynomial with shares -s_i*a - round(M_i*Delta/Delta_ct) + e1_i.  The same
 * protocol refreshes inside hx_sign_approx (refresh index k uses stream
 * index k; batch entry i the seed refresh_seed + i). */
hx_status hx_dbootstrap(hx_context *ctx, const hx_keyset *ks, const hx_ct *ct, uint64_t seed, hx_ct **out, void *stream);

/* ---- server aggregation (Alg. 6, Aggregation) ------------------------------------ */
/* out[m] = models[m] - eta_over_bn * sum_i grads[i*count + m] for m < count:
 * the parties' encrypted gradients are summed in one streaming pass that
 * reads them in place (16-byte loads, HBM-bound), the factor eta/(B*N) is the
 * integer constant of a level adjustment (round(-eta_over_bn * scale_model *
 * q_t / scale_grad), t = limbs - 1) applied in the same pass, then one rescale
 * and the addition to the model dropped to t limbs.  All gradients share one
 * scale and the models' level (>= 2 limbs); the result is at limbs - 1 with
 * the model's scale.  Errors: HX_EINVAL, HX_ESCALE, HX_ELEVEL. */
hx_status hx_aggregate(hx_context *ctx, const hx_ct *const *grads, size_t n_parties, const hx_ct *const *models,
                       size_t count, double eta_over_bn, hx_ct **out, void *stream);

/* ---- serving (continuous batching) ----------------------------------------------- */
/* A request server on the current device.  Requests queue on the host; a
 * dispatcher forms a batch from the oldest pending request and the other
 * pending requests of the same signature (context, keys, kind, level and h, or
 * d/k/relu) whenever one of n_lanes CUDA streams is idle and the batch's
 * estimated device memory fits in what hbm_budget_bytes leaves after the
 * registered keys; the lanes run concurrently.  Rotations are the exception to
 * the signature: pending rotations of every context and level form one batch,
 * run as one launch per key-switching stage over all of them (as
 * hx_rotate_jobs).  Each result equals the same request computed alone
 * (hx_matmul, hx_sign_approx with its refresh_seed, or hx_rotate).  Submitted
 * ciphertexts stay referenced until their request completes, so the caller
 * may destroy its handles at once. */
typedef struct hx_server hx_server;
hx_status hx_server_create(size_t hbm_budget_bytes, int n_lanes, int max_batch, hx_server **out);
/* counts a keyset's device bytes against the budget (HX_ENOMEM if it does not fit) */
hx_status hx_server_register_keys(hx_server *sv, const hx_keyset *ks);
/* HX_ENOMEM if the request alone exceeds the budget */
hx_status hx_server_submit_matmul(hx_server *sv, hx_context *ctx, const hx_keyset *ks, const hx_ct *A,
                                  const hx_ct *B, int h, uint64_t *id);
hx_status hx_server_submit_sign(hx_server *sv, hx_context *ctx, const hx_keyset *ks, const hx_ct *x, int d, int k,
                                int relu, uint64_t refresh_seed, uint64_t *id);
/* a rotation of x by `step` slots (Rot, Fig. 1 item 11) with ctx's keys ks */
hx_status hx_server_submit_rotate(hx_server *sv, hx_context *ctx, const hx_keyset *ks, const hx_ct *x, int64_t step,
                                  uint64_t *id);
/* Moves up to cap completed requests out: ids, result handles (NULL on error),
 * statuses and latencies (submission to completion of its batch on the GPU,
 * ms).  wait != 0 blocks until at least one completes or nothing is pending.
 * Returns the number moved. */
int hx_server_poll(hx_server *sv, int wait, uint64_t *ids, hx_ct **results, int32_t *status, double *latency_ms,
                   int cap);
/* completed, batches, largest batch, most lanes busy at once, peak admitted
 * bytes, key bytes, remaining budget, pending requests, requests expired at
 * their deadline; returns the count (9) */
int hx_server_stats(hx_server *sv, uint64_t *out, int cap);
/* Deadline of a queued request, ms after its submission.  If it is still
 * queued when the deadline passes it completes with status HX_ETIMEOUT, a
 * NULL result and no GPU work; once dispatched it runs to the end.  HX_EINVAL
 * if the request is not queued any more. */
hx_status hx_server_set_deadline(hx_server *sv, uint64_t id, double ms);
/* paused != 0 holds every queued request (deadlines still expire; a blocking
 * poll returns when one does); 0 resumes.  hx_server_destroy resumes before it
 * drains. */
hx_status hx_server_pause(hx_server *sv, int paused);
/* waits for every submitted request, then stops the threads */
void hx_server_destroy(hx_server *sv);

/* ---- ALU calibration ------------------------------------------------------------ */
/* Measured throughput on this device of the two 64-bit multiplication forms
 * the path is built from: Shoup products y*w - umulhi(y, w')*q (one per NTT
 * butterfly) and 64x64 -> 128-bit multiply-accumulates (one per key inner
 * product term), eight independent chains per thread on every SM.  These are
 * the ceilings of the integer-issue-bound kernels, reported beside the HBM
 * roofline. */
hx_status hx_alu_calibrate(hx_context *ctx, double *shoup_per_s, double *mac_per_s, void *stream);

/* ---- counters -------------------------------------------------------------- */
/* Operation counters since the last reset, in this order: Add, Mul_pt,
 * Rot (full), Rot (hoisted), Mul_ct, KeySwitch, ModUp, Rescale, Refresh,
 * kernel launches.  Returns the number of counters. */
int hx_counters(const hx_context *ctx, uint64_t *out, int cap);
void hx_counters_reset(hx_context *ctx);

/* ---- autotuning ------------------------------------------------------------- */
/* NTT autotuner.  Each of the four phase kernels (forward column, forward
 * row, inverse column, inverse row) has variants: a tile width (4, 8, 16 or 32
 * sub-transforms per block, i.e. columns or limb rows per block) and, for an
 * odd number of stages in the phase, the order of its two register passes'
 * radices (e.g. 16 then 8, or 8 then 16).  The best variant depends on the
 * batch: launches are grouped into buckets by their number of limbs (up to 64,
 * 256, 768, more), and each bucket is timed on its own batch (48, 176, 512 and
 * 1024 limbs) on this device, each variant's time the best of three rounds.
 * Per (bucket, phase) the default (width 16, swapped radices off) is kept
 * unless another variant is more than 2 % faster, in which case the fastest is
 * kept: alone the widths differ by about their timing noise, and blocks of the
 * default size share the SMs best with concurrently running kernels.  For an
 * odd log N both splits of the stages between the two phases are tuned this
 * way, and the other split replaces the default (the column phase taking
 * floor(log N / 2) stages) when the sum of its phases' times is more than 2 %
 * lower.  The table belongs to the context.  Every variant computes identical residues.
 * The call runs on `stream` and synchronizes it.  choice[4] (may be
 * NULL) receives the variants of the 256-limb bucket as signed widths
 * (negative: swapped radices). */
hx_status hx_autotune(hx_context *ctx, int32_t *choice, void *stream);
/* Sets (set != NULL: signed widths per phase, in the order above, for every
 * bucket, with the default phase split) and/or reads (get != NULL: the
 * 256-limb bucket) the NTT variants. */
hx_status hx_ntt_tiles(hx_context *ctx, const int32_t *set, int32_t *get);
/* Sets the split of an odd log N between the two NTT phases for every bucket
 * (0: the column phase takes floor(log N / 2) stages, 1: the other half; no
 * effect for an even log N).  HX_EINVAL for another value. */
hx_status hx_ntt_split(hx_context *ctx, int split);
/* The tuning table: per bucket seven integers (largest limb count of the
 * bucket, limbs it was timed on, the four phases' signed widths, then the split
 * of an odd log N: 0 when the column phase takes floor(log N / 2) stages, 1 when
 * it takes the other half).  Writes at most cap integers; returns the table's
 * length. */
int hx_ntt_tuning(const hx_context *ctx, int32_t *out, int cap);

/* ---- profiling ------------------------------------------------------------- */
/* While enabled, every kernel launch of the context is bracketed by CUDA events
 * recorded on its launching stream, grouped by kernel class.  Enabling clears
 * earlier records.  hx_profile_read synchronizes the device and reports class
 * i (0-based): its name, the number of launches, their summed duration in ms
 * and their summed algorithmic bytes (the reads and writes the operation needs
 * at least, 8 bytes per residue); returns the number of classes, or HX_EINVAL
 * for i out of range.  While enabled, the product's independent chains run one
 * after another on the caller's stream (not on side streams), so each event
 * interval is one kernel running alone. */
hx_status hx_profile_enable(hx_context *ctx, int on);
int hx_profile_read(hx_context *ctx, int i, char *name, size_t cap, uint64_t *launches, double *ms, double *bytes);

#ifdef __cplusplus
}
#endif
#endif
