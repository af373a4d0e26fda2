// extern "C" entry points of include/hx.h: argument checks, handle management
// and error translation around the runtime.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <stdexcept>

#include "runtime.h"

using namespace hx;

namespace {

thread_local std::string g_err;

#define HX_TRY try {
#define HX_END                                                                                                     \
    }                                                                                                              \
    catch (const hx::Error &e)                                                                                     \
    {                                                                                                              \
        g_err = e.msg;                                                                                             \
        return e.code;                                                                                             \
    }                                                                                                              \
    catch (const std::bad_alloc &)                                                                                 \
    {                                                                                                              \
        g_err = "host allocation failed";                                                                          \
        return HX_ENOMEM;                                                                                          \
    }                                                                                                              \
    catch (const std::exception &e)                                                                                \
    {                                                                                                              \
        g_err = e.what();                                                                                          \
        return HX_EINVAL;                                                                                          \
    }

cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

hx_ct *wrap(hx_context *ctx, const Cts &c)
{
    hx_ct *h = new hx_ct;
    h->ctx = ctx;
    h->c = c;
    return h;
}

void need(bool c, const char *msg)
{
    if (!c) throw hx::Error{HX_EINVAL, msg};
}

// Every handle records the context it was made in.  A handle of another context (another
// ring degree or prime chain) would reach the kernels with that context's row length and
// table indices, so it is rejected before any device work.
void mine(const hx_context *ctx, const hx_keyset *ks) { need(ks->ctx == ctx, "keys of another context"); }
void mine(const hx_context *ctx, const hx_ct *c) { need(c->ctx == ctx, "ciphertext of another context"); }
void mine(const hx_context *ctx, const hx_matmul_plan *p) { need(p->ctx == ctx, "plan of another context"); }

} // namespace

namespace hx {
void set_error(const std::string &msg) { g_err = msg; }
} // namespace hx

namespace {

// One group of a batched product call: entries of one context, key set, h, level and scale,
// evaluated as one batched HE-MatMult.
struct MatmulGroup {
    hx_context *ctx;
    const hx_keyset *ks;
    int h;
    std::vector<size_t> idx;  // positions in the call's entry list
    std::vector<const hx_ct *> A, B;
};

// Runs the groups side by side: each on a stream of its context's pool, forked from s by an event,
// so the schedules of different rings, levels and sizes overlap on the device.  After the join,
// the products are copied into the outputs on s; each group's own buffers are released on its
// stream only after s has made those copies.
void run_matmul_groups(std::vector<MatmulGroup> &groups, cudaStream_t s, hx_ct **out, size_t count)
{
    struct Running {
        hx_context *ctx = nullptr;
        cudaStream_t gs = nullptr;
        Cts r;
    };
    std::vector<Running> run(groups.size());
    std::vector<hx_ct *> res(count, nullptr);
    cudaEvent_t fork = nullptr, copied = nullptr;
    std::vector<cudaEvent_t> done;
    auto release = [&] {
        if (fork) cudaEventDestroy(fork);
        if (copied) cudaEventDestroy(copied);
        for (cudaEvent_t e : done) cudaEventDestroy(e);
    };
    try {
        HX_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        HX_CUDA(cudaEventCreateWithFlags(&copied, cudaEventDisableTiming));
        HX_CUDA(cudaEventRecord(fork, s));
        std::map<hx_context *, size_t> next;  // next pool stream of each context
        for (size_t g = 0; g < groups.size(); g++) {
            MatmulGroup &G = groups[g];
            const cudaStream_t gs = group_stream(*G.ctx, s, next[G.ctx]++);
            if (gs != s) HX_CUDA(cudaStreamWaitEvent(gs, fork, 0));
            run[g].ctx = G.ctx;
            run[g].gs = gs;
            Cts a = gather(*G.ctx, G.A.data(), G.A.size(), gs);
            Cts b = gather(*G.ctx, G.B.data(), G.B.size(), gs);
            PlanUse plan(*G.ctx, gs, cached_plan(*G.ctx, G.h, a.limbs));
            run[g].r = matmul_batch(*G.ctx, *G.ks, *plan.p, a, b, gs);
            cudaEvent_t e = nullptr;
            HX_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            done.push_back(e);
            HX_CUDA(cudaEventRecord(e, gs));
        }
        for (cudaEvent_t e : done) HX_CUDA(cudaStreamWaitEvent(s, e, 0));
        for (size_t g = 0; g < groups.size(); g++) {
            std::vector<hx_ct *> part(groups[g].idx.size(), nullptr);
            scatter(*groups[g].ctx, run[g].r, part.data(), s);
            for (size_t k = 0; k < part.size(); k++) res[groups[g].idx[k]] = part[k];
        }
        HX_CUDA(cudaEventRecord(copied, s));
        for (auto &R : run)
            if (R.gs && R.gs != s) HX_CUDA(cudaStreamWaitEvent(R.gs, copied, 0));
    } catch (...) {
        // the caller's stream still waits for whatever the started groups launched, so inputs it
        // frees after the error are not read afterwards (best effort: the error is rethrown)
        cudaEvent_t j = nullptr;
        if (cudaEventCreateWithFlags(&j, cudaEventDisableTiming) == cudaSuccess) {
            for (auto &R : run)
                if (R.gs && R.gs != s && cudaEventRecord(j, R.gs) == cudaSuccess) cudaStreamWaitEvent(s, j, 0);
            cudaEventDestroy(j);
        }
        for (hx_ct *c : res) delete c;
        release();
        throw;
    }
    release();
    std::copy(res.begin(), res.end(), out);
}

} // namespace

extern "C" {

const char *hx_last_error(void) { return g_err.c_str(); }

hx_status hx_context_create(const hx_params *p, hx_context **out)
{
    HX_TRY
    need(p && out, "null argument");
    *out = nullptr;
    std::unique_ptr<hx_context> c(new hx_context);
    build_context(*c, *p);
    *out = c.release();
    return HX_OK;
    HX_END
}

void hx_context_destroy(hx_context *ctx)
{
    if (!ctx) return;
    destroy_context(*ctx);
    delete ctx;
}

int hx_context_primes(const hx_context *ctx, uint64_t *out, int cap)
{
    if (!ctx || (!out && cap > 0)) return HX_EINVAL;
    for (int i = 0; i < ctx->n_all && i < cap; i++) out[i] = ctx->primes[i];
    return ctx->n_all;
}

int hx_context_n(const hx_context *ctx) { return ctx ? ctx->N : HX_EINVAL; }

hx_status hx_keygen(hx_context *ctx, int n_parties, uint64_t seed, const int32_t *rot_steps, size_t n_steps,
                    hx_keyset **out)
{
    HX_TRY
    need(ctx && out && (rot_steps || n_steps == 0), "null argument");
    *out = nullptr;
    std::unique_ptr<hx_keyset> ks(new hx_keyset);
    static std::atomic<uint64_t> next_uid{1};
    ks->uid = next_uid++;
    keygen(*ctx, *ks, n_parties, seed, nullptr);
    std::vector<int64_t> st(rot_steps, rot_steps + n_steps);
    add_rotation_keys(*ctx, *ks, st, nullptr);
    *out = ks.release();
    return HX_OK;
    HX_END
}

// keyset file: "HXKS0001", u32 log_n, n_q, n_p, n_parties, u64 seed, u32 n_galois, alpha,
// u64 moduli[n_q + n_p], u64 galois[n_galois] ascending, little-endian.  Keys are a
// deterministic function of (seed, parties, Galois elements), so the file holds that recipe.
hx_status hx_keyset_save(hx_context *ctx, const hx_keyset *ks, const char *path)
{
    HX_TRY
    need(ctx && ks && path && ks->ctx == ctx, "null argument or keys of another context");
    std::vector<uint64_t> gal;
    for (const auto &kv : ks->rot) gal.push_back(kv.first);
    std::sort(gal.begin(), gal.end());
    FILE *f = fopen(path, "wb");
    HX_CHECK(f, HX_EINVAL, std::string("cannot write ") + path);
    const uint32_t hdr[4] = {(uint32_t)ctx->log_n, (uint32_t)ctx->n_q, (uint32_t)ctx->K, (uint32_t)ks->n_parties};
    const uint32_t cnt[2] = {(uint32_t)gal.size(), (uint32_t)ctx->alpha};
    bool ok = fwrite("HXKS0001", 1, 8, f) == 8 && fwrite(hdr, 4, 4, f) == 4 && fwrite(&ks->seed, 8, 1, f) == 1 &&
              fwrite(cnt, 4, 2, f) == 2 && fwrite(ctx->primes.data(), 8, ctx->n_all, f) == (size_t)ctx->n_all &&
              fwrite(gal.data(), 8, gal.size(), f) == gal.size();
    ok = (fclose(f) == 0) && ok;
    HX_CHECK(ok, HX_EINVAL, std::string("short write to ") + path);
    return HX_OK;
    HX_END
}

hx_status hx_keyset_load(hx_context *ctx, const char *path, hx_keyset **out)
{
    HX_TRY
    need(ctx && path && out, "null argument");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    HX_CHECK(f, HX_EINVAL, std::string("cannot read ") + path);
    char magic[8];
    uint32_t hdr[4], cnt[2];
    uint64_t seed = 0;
    std::vector<uint64_t> mod, gal;
    bool ok = fread(magic, 1, 8, f) == 8 && fread(hdr, 4, 4, f) == 4 && fread(&seed, 8, 1, f) == 1 &&
              fread(cnt, 4, 2, f) == 2;
    if (ok) ok = memcmp(magic, "HXKS0001", 8) == 0 && hdr[0] == (uint32_t)ctx->log_n &&
                 hdr[1] == (uint32_t)ctx->n_q && hdr[2] == (uint32_t)ctx->K && hdr[3] >= 1 && hdr[3] <= 64 &&
                 cnt[0] <= (uint32_t)ctx->N && cnt[1] == (uint32_t)ctx->alpha;
    if (ok) {
        mod.resize(ctx->n_all);
        gal.resize(cnt[0]);
        ok = fread(mod.data(), 8, mod.size(), f) == mod.size() && fread(gal.data(), 8, gal.size(), f) == gal.size() &&
             fgetc(f) == EOF;
        for (int i = 0; ok && i < ctx->n_all; i++) ok = mod[i] == ctx->primes[i];
    }
    fclose(f);
    HX_CHECK(ok, HX_EINVAL, std::string(path) + " is not a keyset file of this context");
    // each Galois element back to its rotation step: 5^k mod 2N for k in [0, N/2)
    std::vector<int64_t> steps;
    const uint64_t two_n = 2ull * ctx->N;
    for (uint64_t g : gal) {
        uint64_t x = 1;
        int64_t k = 0;
        for (; k < ctx->N / 2 && x != g; k++) x = x * 5 % two_n;
        HX_CHECK(x == g, HX_EINVAL, "Galois element " + std::to_string(g) + " is not a power of 5");
        steps.push_back(k);
    }
    std::vector<int32_t> st(steps.begin(), steps.end());
    return hx_keygen(ctx, (int)hdr[3], seed, st.data(), st.size(), out);
    HX_END
}

hx_status hx_keyset_add_rotations(hx_context *ctx, hx_keyset *ks, const int32_t *rot_steps, size_t n_steps)
{
    HX_TRY
    need(ctx && ks && (rot_steps || n_steps == 0), "null argument");
    mine(ctx, ks);
    std::vector<int64_t> st(rot_steps, rot_steps + n_steps);
    add_rotation_keys(*ctx, *ks, st, nullptr);
    return HX_OK;
    HX_END
}

int64_t hx_keyset_export_switch_key(const hx_keyset *ks, uint64_t galois, uint64_t *host, size_t cap)
{
    HX_TRY
    need(ks && host, "null argument");
    const hx_context &c = *ks->ctx;
    const SwitchKey *k = nullptr;
    if (galois == 0)
        k = &ks->relin;
    else {
        auto it = ks->rot.find(galois);
        if (it == ks->rot.end()) throw hx::Error{HX_EKEY, "no key for this Galois element"};
        k = &it->second;
    }
    const size_t words = (size_t)c.dnum * 2 * c.n_all * c.N;
    need(cap >= words, "buffer too small");
    HX_CUDA(cudaDeviceSynchronize());
    HX_CUDA(cudaMemcpy(host, k->buf->p, words * 8, cudaMemcpyDeviceToHost));
    // Montgomery form -> standard residues: x * 2^-64 mod q
    for (size_t r = 0; r < (size_t)c.dnum * 2 * c.n_all; r++) {
        const uint64_t q = c.primes[r % c.n_all];
        const uint64_t rinv = hinv((uint64_t)(((u128)1 << 64) % q), q);
        for (int j = 0; j < c.N; j++) host[r * c.N + j] = hmul(host[r * c.N + j], rinv, q);
    }
    return (int64_t)words;
    HX_END
}

int64_t hx_keyset_export_public_key(const hx_keyset *ks, uint64_t *host, size_t cap)
{
    HX_TRY
    need(ks && host, "null argument");
    const size_t words = (size_t)2 * ks->ctx->n_q * ks->ctx->N;
    need(cap >= words, "buffer too small");
    HX_CUDA(cudaDeviceSynchronize());
    HX_CUDA(cudaMemcpy(host, ks->pk->p, words * 8, cudaMemcpyDeviceToHost));
    return (int64_t)words;
    HX_END
}

void hx_keyset_destroy(hx_keyset *ks)
{
    if (!ks) return;
    cudaDeviceSynchronize();
    delete ks;
}

hx_status hx_encode(const hx_context *ctx, const double *slots, size_t n, double scale, int64_t *coeffs)
{
    HX_TRY
    need(ctx && (slots || n == 0) && coeffs, "null argument");
    need(n <= (size_t)ctx->N / 2 && scale > 0, "too many slots or bad scale");
    ctx->enc->encode(slots, n, scale, coeffs);
    return HX_OK;
    HX_END
}

hx_status hx_encrypt(hx_context *ctx, const hx_keyset *ks, const double *slots, size_t n, int limbs, uint64_t seed,
                     hx_ct **out)
{
    HX_TRY
    need(ctx && ks && (slots || n == 0) && out, "null argument");
    *out = nullptr;
    mine(ctx, ks);
    need(n <= (size_t)ctx->N / 2, "too many slots");
    std::vector<int64_t> m(ctx->N);
    ctx->enc->encode(slots, n, ctx->scale, m.data());
    Cts c = encrypt_coeffs(*ctx, *ks, m.data(), ctx->scale, limbs ? limbs : ctx->n_q, seed, 0, 0, nullptr);
    HX_CUDA(cudaStreamSynchronize(nullptr));
    *out = wrap(ctx, c);
    return HX_OK;
    HX_END
}

hx_status hx_encode_batch(hx_context *ctx, const double *slots, size_t n, size_t count, double scale, int64_t *coeffs,
                          void *stream)
{
    HX_TRY
    need(ctx && slots && coeffs && count >= 1 && count < 65536 && n <= (size_t)ctx->N / 2 && scale > 0,
         "bad argument");
    cudaStream_t s = S(stream);
    DevBuf in(std::max<size_t>(1, n * count), s), out((size_t)ctx->N * count, s);
    if (n) HX_CUDA(cudaMemcpyAsync(in.p, slots, sizeof(double) * n * count, cudaMemcpyHostToDevice, s));
    encode_batch(*ctx, reinterpret_cast<const double *>(in.p), n, (int)count, scale,
                 reinterpret_cast<int64_t *>(out.p), (size_t)ctx->N, s);
    HX_CUDA(cudaMemcpyAsync(coeffs, out.p, sizeof(int64_t) * ctx->N * count, cudaMemcpyDeviceToHost, s));
    HX_CUDA(cudaStreamSynchronize(s));
    return HX_OK;
    HX_END
}

hx_status hx_encrypt_batch(hx_context *ctx, const hx_keyset *ks, const double *slots, size_t n, size_t count, int limbs,
                           const uint64_t *seeds, hx_ct **out, void *stream)
{
    HX_TRY
    need(ctx && ks && slots && seeds && out && count >= 1 && count < 65536 && n <= (size_t)ctx->N / 2,
         "bad argument");
    for (size_t i = 0; i < count; i++) out[i] = nullptr;
    mine(ctx, ks);
    cudaStream_t s = S(stream);
    DevBuf in(std::max<size_t>(1, n * count), s);
    if (n) HX_CUDA(cudaMemcpyAsync(in.p, slots, sizeof(double) * n * count, cudaMemcpyHostToDevice, s));
    Cts c = encrypt_batch(*ctx, *ks, reinterpret_cast<const double *>(in.p), n, (int)count,
                          limbs ? limbs : ctx->n_q, seeds, s);
    scatter(*ctx, c, out, s);
    HX_CUDA(cudaStreamSynchronize(s));
    return HX_OK;
    HX_END
}

hx_status hx_encrypt_coeffs(hx_context *ctx, const hx_keyset *ks, const int64_t *coeffs, double scale, int limbs,
                            uint64_t seed, uint32_t tag, uint32_t index, hx_ct **out)
{
    HX_TRY
    need(ctx && ks && coeffs && out, "null argument");
    *out = nullptr;
    mine(ctx, ks);
    Cts c = encrypt_coeffs(*ctx, *ks, coeffs, scale, limbs ? limbs : ctx->n_q, seed, tag, index, nullptr);
    HX_CUDA(cudaStreamSynchronize(nullptr));
    *out = wrap(ctx, c);
    return HX_OK;
    HX_END
}

hx_status hx_decrypt_coeffs(hx_context *ctx, const hx_keyset *ks, const hx_ct *ct, int64_t *coeffs)
{
    HX_TRY
    need(ctx && ks && ct && coeffs, "null argument");
    mine(ctx, ks);
    mine(ctx, ct);
    HX_CUDA(cudaDeviceSynchronize());
    std::vector<int64_t> v = decrypt_coeffs(*ctx, *ks, ct->c, nullptr);
    memcpy(coeffs, v.data(), sizeof(int64_t) * ctx->N);
    return HX_OK;
    HX_END
}

hx_status hx_decrypt(hx_context *ctx, const hx_keyset *ks, const hx_ct *ct, double *slots, size_t n)
{
    HX_TRY
    need(ctx && ks && ct && (slots || n == 0), "null argument");
    mine(ctx, ks);
    mine(ctx, ct);
    HX_CUDA(cudaDeviceSynchronize());
    std::vector<int64_t> v = decrypt_coeffs(*ctx, *ks, ct->c, nullptr);
    ctx->enc->decode(v.data(), ct->c.scale, slots, std::min(n, (size_t)ctx->N / 2));
    return HX_OK;
    HX_END
}

hx_status hx_decrypt_parties(hx_context *ctx, const hx_keyset *ks, const hx_ct *ct, const uint8_t *present,
                             size_t n_present, double *slots, size_t n)
{
    HX_TRY
    need(ctx && ks && ct && present && (slots || n == 0), "null argument");
    mine(ctx, ks);
    mine(ctx, ct);
    need(n_present == (size_t)ks->n_parties, "one flag per party of the key set");
    for (int i = 0; i < ks->n_parties; i++)
        HX_CHECK(present[i], HX_EPARTY,
                 "party " + std::to_string(i) + " sent no decryption share; DDec needs all " +
                     std::to_string(ks->n_parties) + " parties");
    HX_CUDA(cudaDeviceSynchronize());
    std::vector<int64_t> v = decrypt_coeffs(*ctx, *ks, ct->c, nullptr);
    ctx->enc->decode(v.data(), ct->c.scale, slots, std::min(n, (size_t)ctx->N / 2));
    return HX_OK;
    HX_END
}

// ciphertext file: "HXCT0001", u32 log_n, comps, limbs, 0, f64 scale, u64 moduli[limbs],
// u64 residues[comps][limbs][N] (NTT form), all little-endian
hx_status hx_ct_save(hx_context *ctx, const hx_ct *ct, const char *path)
{
    HX_TRY
    need(ctx && ct && path, "null argument");
    mine(ctx, ct);
    const Cts &c = ct->c;
    const size_t N = ctx->N, words = (size_t)c.comps * c.limbs * N;
    std::vector<uint64_t> host(words);
    HX_CUDA(cudaDeviceSynchronize());
    for (int k = 0; k < c.comps; k++)
        HX_CUDA(cudaMemcpy(host.data() + (size_t)k * c.limbs * N, c.d + k * c.cstride(N), sizeof(uint64_t) * c.limbs * N,
                           cudaMemcpyDeviceToHost));
    FILE *f = fopen(path, "wb");
    HX_CHECK(f, HX_EINVAL, std::string("cannot write ") + path);
    const uint32_t hdr[4] = {(uint32_t)ctx->log_n, (uint32_t)c.comps, (uint32_t)c.limbs, 0};
    bool ok = fwrite("HXCT0001", 1, 8, f) == 8 && fwrite(hdr, 4, 4, f) == 4 && fwrite(&c.scale, 8, 1, f) == 1 &&
              fwrite(ctx->primes.data(), 8, c.limbs, f) == (size_t)c.limbs &&
              fwrite(host.data(), 8, words, f) == words;
    ok = (fclose(f) == 0) && ok;
    HX_CHECK(ok, HX_EINVAL, std::string("short write to ") + path);
    return HX_OK;
    HX_END
}

hx_status hx_ct_load(hx_context *ctx, const char *path, hx_ct **out)
{
    HX_TRY
    need(ctx && path && out, "null argument");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    HX_CHECK(f, HX_EINVAL, std::string("cannot read ") + path);
    char magic[8];
    uint32_t hdr[4];
    double scale = 0;
    bool ok = fread(magic, 1, 8, f) == 8 && fread(hdr, 4, 4, f) == 4 && fread(&scale, 8, 1, f) == 1;
    std::vector<uint64_t> mod, host;
    if (ok) ok = memcmp(magic, "HXCT0001", 8) == 0 && hdr[0] == (uint32_t)ctx->log_n && hdr[1] >= 2 && hdr[1] <= 3 &&
                 hdr[2] >= 1 && hdr[2] <= (uint32_t)ctx->n_q && scale > 0;
    if (ok) {
        mod.resize(hdr[2]);
        ok = fread(mod.data(), 8, hdr[2], f) == hdr[2];
        for (uint32_t l = 0; ok && l < hdr[2]; l++) ok = mod[l] == ctx->primes[l];
    }
    if (ok) {
        host.resize((size_t)hdr[1] * hdr[2] * ctx->N);
        ok = fread(host.data(), 8, host.size(), f) == host.size() && fgetc(f) == EOF;
    }
    fclose(f);
    HX_CHECK(ok, HX_EINVAL, std::string(path) + " is not a ciphertext file of this context");
    Eval ev(*ctx, nullptr);
    Cts c = ev.alloc(1, (int)hdr[1], (int)hdr[2]);
    c.scale = scale;
    HX_CUDA(cudaMemcpy(c.d, host.data(), sizeof(uint64_t) * host.size(), cudaMemcpyHostToDevice));
    *out = wrap(ctx, c);
    return HX_OK;
    HX_END
}

hx_status hx_ct_import(hx_context *ctx, const uint64_t *host, int comps, int limbs, double scale, hx_ct **out)
{
    HX_TRY
    need(ctx && host && out, "null argument");
    *out = nullptr;
    need(comps >= 2 && comps <= 3 && limbs >= 1 && limbs <= ctx->n_q && scale > 0, "bad ciphertext shape");
    Eval ev(*ctx, nullptr);
    Cts c = ev.alloc(1, comps, limbs);
    c.scale = scale;
    HX_CUDA(cudaMemcpy(c.d, host, sizeof(uint64_t) * comps * limbs * ctx->N, cudaMemcpyHostToDevice));
    *out = wrap(ctx, c);
    return HX_OK;
    HX_END
}

int64_t hx_ct_export(const hx_ct *ct, uint64_t *host, size_t cap)
{
    HX_TRY
    need(ct && host, "null argument");
    const Cts &c = ct->c;
    const size_t N = ct->ctx->N, words = (size_t)c.comps * c.limbs * N;
    need(cap >= words, "buffer too small");
    HX_CUDA(cudaDeviceSynchronize());
    for (int k = 0; k < c.comps; k++)
        HX_CUDA(cudaMemcpy(host + (size_t)k * c.limbs * N, c.d + k * c.cstride(N), sizeof(uint64_t) * c.limbs * N,
                           cudaMemcpyDeviceToHost));
    return (int64_t)words;
    HX_END
}

hx_status hx_ct_info(const hx_ct *ct, int *comps, int *limbs, double *scale)
{
    if (!ct) return HX_EINVAL;
    if (comps) *comps = ct->c.comps;
    if (limbs) *limbs = ct->c.limbs;
    if (scale) *scale = ct->c.scale;
    return HX_OK;
}

void hx_ct_destroy(hx_ct *ct) { delete ct; }

#define ONE_IN(a) need(ctx && (a) && out, "null argument"); *out = nullptr; Eval ev(*ctx, S(stream));

hx_status hx_add(hx_context *ctx, const hx_ct *a, const hx_ct *b, hx_ct **out, void *stream)
{
    HX_TRY
    ONE_IN(a && b)
    mine(ctx, a);
    mine(ctx, b);
    *out = wrap(ctx, ev.add(a->c, b->c, false));
    return HX_OK;
    HX_END
}

hx_status hx_sub(hx_context *ctx, const hx_ct *a, const hx_ct *b, hx_ct **out, void *stream)
{
    HX_TRY
    ONE_IN(a && b)
    mine(ctx, a);
    mine(ctx, b);
    *out = wrap(ctx, ev.add(a->c, b->c, true));
    return HX_OK;
    HX_END
}

hx_status hx_mul_plain(hx_context *ctx, const hx_ct *a, const int64_t *pt, double pt_scale, hx_ct **out,
                       void *stream)
{
    HX_TRY
    ONE_IN(a && pt)
    mine(ctx, a);
    DevBuf p((size_t)a->c.limbs * ctx->N, S(stream));
    upload_plaintext(*ctx, S(stream), pt, a->c.limbs, p.p);
    *out = wrap(ctx, ev.mul_plain(a->c, p.p, pt_scale));
    return HX_OK;
    HX_END
}

hx_status hx_mul_int(hx_context *ctx, const hx_ct *a, int64_t c, double new_scale, hx_ct **out, void *stream)
{
    HX_TRY
    ONE_IN(a)
    mine(ctx, a);
    *out = wrap(ctx, ev.mul_int(a->c, c, new_scale));
    return HX_OK;
    HX_END
}

hx_status hx_add_const(hx_context *ctx, const hx_ct *a, double value, hx_ct **out, void *stream)
{
    HX_TRY
    ONE_IN(a)
    mine(ctx, a);
    *out = wrap(ctx, ev.add_const(a->c, value));
    return HX_OK;
    HX_END
}

hx_status hx_tensor(hx_context *ctx, const hx_ct *a, const hx_ct *b, hx_ct **out, void *stream)
{
    HX_TRY
    ONE_IN(a && b)
    mine(ctx, a);
    mine(ctx, b);
    *out = wrap(ctx, ev.tensor(a->c, b->c));
    return HX_OK;
    HX_END
}

hx_status hx_relinearize(hx_context *ctx, const hx_keyset *ks, const hx_ct *d, hx_ct **out, void *stream)
{
    HX_TRY
    ONE_IN(ks && d)
    mine(ctx, ks);
    mine(ctx, d);
    *out = wrap(ctx, ev.relinearize(d->c, ks->relin));
    return HX_OK;
    HX_END
}

hx_status hx_relin_rescale(hx_context *ctx, const hx_keyset *ks, const hx_ct *d, hx_ct **out, void *stream)
{
    HX_TRY
    ONE_IN(ks && d)
    mine(ctx, ks);
    mine(ctx, d);
    *out = wrap(ctx, ev.relin_rescale(d->c, ks->relin));
    return HX_OK;
    HX_END
}

hx_status hx_rescale(hx_context *ctx, const hx_ct *a, hx_ct **out, void *stream)
{
    HX_TRY
    ONE_IN(a)
    mine(ctx, a);
    *out = wrap(ctx, ev.rescale(a->c));
    return HX_OK;
    HX_END
}

hx_status hx_drop(hx_context *ctx, const hx_ct *a, int limbs, hx_ct **out, void *stream)
{
    HX_TRY
    ONE_IN(a)
    mine(ctx, a);
    need(limbs >= 1 && limbs <= a->c.limbs, "bad level");
    Cts c = ev.copy(ev.drop(a->c, limbs));
    *out = wrap(ctx, c);
    return HX_OK;
    HX_END
}

hx_status hx_rotate(hx_context *ctx, const hx_keyset *ks, const hx_ct *a, int32_t k, hx_ct **out, void *stream)
{
    HX_TRY
    ONE_IN(ks && a)
    mine(ctx, ks);
    mine(ctx, a);
    *out = wrap(ctx, ev.rotate(a->c, k, *ks));
    return HX_OK;
    HX_END
}

hx_status hx_rotate_jobs(const hx_rotate_job *jobs, size_t count, hx_ct **out, void *stream)
{
    HX_TRY
    need(jobs && out && count >= 1 && count < 65536, "bad argument");
    for (size_t i = 0; i < count; i++) out[i] = nullptr;
    std::vector<RotateJob> v(count);
    for (size_t i = 0; i < count; i++) {
        const hx_rotate_job &J = jobs[i];
        need(J.ctx && J.ks && J.ct, "null job field");
        mine(J.ctx, J.ks);
        mine(J.ctx, J.ct);
        v[i] = RotateJob{J.ctx, J.ks, J.ct->c, J.step};
    }
    std::vector<Cts> r = rotate_jobs(v, S(stream));
    std::vector<std::unique_ptr<hx_ct>> h(count);
    for (size_t i = 0; i < count; i++) h[i].reset(wrap(jobs[i].ctx, r[i]));
    for (size_t i = 0; i < count; i++) out[i] = h[i].release();
    return HX_OK;
    HX_END
}

hx_status hx_rotate_hoisted(hx_context *ctx, const hx_keyset *ks, const hx_ct *a, const int32_t *steps, int n,
                            hx_ct **outs, void *stream)
{
    HX_TRY
    need(ctx && ks && a && steps && outs && n >= 0, "null argument");
    for (int i = 0; i < n; i++) outs[i] = nullptr;
    mine(ctx, ks);
    mine(ctx, a);
    Eval ev(*ctx, S(stream));
    std::vector<int64_t> st(steps, steps + n);
    std::vector<Cts> r = ev.rotate_hoisted(a->c, st, *ks);
    for (int i = 0; i < n; i++) outs[i] = wrap(ctx, r[i]);
    return HX_OK;
    HX_END
}

hx_status hx_ntt(hx_context *ctx, uint64_t *dev, int n_polys, int limbs, const int32_t *prime_idx, int inverse,
                 void *stream)
{
    HX_TRY
    need(ctx && dev && prime_idx && n_polys >= 0 && limbs >= 1, "null argument");
    need(limbs <= MAX_NTT_ROWS && n_polys < 65536, "too many rows");
    std::vector<int> off(limbs), pr(limbs);
    for (int l = 0; l < limbs; l++) {
        need(prime_idx[l] >= 0 && prime_idx[l] < ctx->n_all, "bad prime index");
        off[l] = l;
        pr[l] = prime_idx[l];
    }
    Eval ev(*ctx, S(stream));
    ev.ntt_inplace(dev, (size_t)limbs * ctx->N, n_polys, off, pr, inverse != 0);
    return HX_OK;
    HX_END
}

hx_status hx_ntt_multi(const hx_ntt_job *jobs, int n_jobs, int inverse, void *stream)
{
    HX_TRY
    need(jobs && n_jobs >= 1 && n_jobs <= 4096, "bad job list");
    std::vector<NttJob> v(n_jobs);
    int dev = -1;
    for (int i = 0; i < n_jobs; i++) {
        const hx_ntt_job &j = jobs[i];
        need(j.ctx && (j.data || j.n_polys == 0) && j.prime_idx && j.n_polys >= 0, "null job field");
        need(j.n_limbs >= 1 && j.n_limbs <= 64, "a job has 1..64 limbs");
        need(dev < 0 || j.ctx->device == dev, "jobs on several devices");
        dev = j.ctx->device;
        NttJob &J = v[i];
        J.data = j.data;
        J.primes = j.ctx->t.primes;
        J.tw_fwd = j.ctx->t.tw_fwd;
        J.tw_inv = j.ctx->t.tw_inv;
        J.log_n = j.ctx->log_n;
        J.n_rows = j.n_polys * j.n_limbs;
        J.n_limbs = j.n_limbs;
        J.tile0_cols = J.tile0_rows = 0;
        for (int l = 0; l < j.n_limbs; l++) {
            need(j.prime_idx[l] >= 0 && j.prime_idx[l] < j.ctx->n_all, "bad prime index");
            J.prime[l] = (int16_t)j.prime_idx[l];
        }
    }
    hx_context *c0 = const_cast<hx_context *>(jobs[0].ctx);
    launch_ntt_multi(S(stream), v, inverse != 0, c0->t.n_sm, &c0->counters[C_LAUNCH]);
    return HX_OK;
    HX_END
}

hx_status hx_matmul_plan_create(hx_context *ctx, int h, int limbs, hx_matmul_plan **out)
{
    HX_TRY
    need(ctx && out, "null argument");
    *out = nullptr;
    *out = make_plan(*ctx, h, limbs, nullptr);
    return HX_OK;
    HX_END
}

int hx_matmul_plan_num_masks(const hx_matmul_plan *plan) { return plan ? (int)plan->masks.size() : HX_EINVAL; }

hx_status hx_matmul_plan_set_mask(hx_context *ctx, hx_matmul_plan *plan, int i, const int64_t *coeffs)
{
    HX_TRY
    need(ctx && plan && coeffs && i >= 0 && i < (int)plan->masks.size(), "bad mask index");
    mine(ctx, plan);
    auto &m = plan->masks[i];
    plan->bound_uid = 0;  // keys premasked with the old mask no longer apply
    plan->premasked.clear();
    if (m.extended)
        upload_plaintext_ext(*ctx, nullptr, coeffs, m.limbs, m.pt->p);
    else
        upload_plaintext(*ctx, nullptr, coeffs, m.limbs, m.pt->p);
    return HX_OK;
    HX_END
}

hx_status hx_matmul_plan_bind_keys(hx_context *ctx, hx_matmul_plan *plan, const hx_keyset *ks, void *stream)
{
    HX_TRY
    need(ctx && plan && ks, "null argument");
    mine(ctx, plan);
    mine(ctx, ks);
    bind_plan_keys(*ctx, *plan, *ks, S(stream));
    return HX_OK;
    HX_END
}

int64_t hx_matmul_plan_bound_bytes(const hx_matmul_plan *plan)
{
    if (!plan) return HX_EINVAL;
    int64_t b = 0;
    for (auto &p : plan->premasked)
        if (p) b += (int64_t)p->words * 8;
    return b;
}

void hx_matmul_plan_destroy(hx_matmul_plan *plan)
{
    if (!plan) return;
    cudaDeviceSynchronize();
    delete plan;
}

int hx_matmul_rotation_steps(const hx_context *ctx, int h, int limbs, int32_t *out, int cap)
{
    if (!ctx || h < 2 || (h & (h - 1)) || h * h > ctx->N / 2 || limbs < 3) return HX_EINVAL;
    std::vector<int64_t> st = plan_rotation_steps(h, ctx->N / 2 / (h * h), limbs);
    for (int i = 0; i < (int)st.size() && i < cap; i++) out[i] = (int32_t)st[i];
    return (int)st.size();
}

hx_status hx_context_set_plan_cache(hx_context *ctx, uint64_t bytes)
{
    HX_TRY
    need(ctx, "null argument");
    std::lock_guard<std::mutex> lk(ctx->plan_mu);
    ctx->plan_limit = bytes ? (size_t)bytes : SIZE_MAX;
    trim_plan_cache(*ctx);
    return HX_OK;
    HX_END
}

int hx_context_plan_cache_info(hx_context *ctx, uint64_t *out, int cap)
{
    if (!ctx || (!out && cap > 0)) return HX_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->plan_mu);
    const uint64_t v[4] = {(uint64_t)ctx->plans.size(), (uint64_t)ctx->plan_bytes,
                           ctx->plan_limit == SIZE_MAX ? 0 : (uint64_t)ctx->plan_limit, ctx->plan_evictions};
    for (int i = 0; i < 4 && i < cap; i++) out[i] = v[i];
    return 4;
}

hx_status hx_matmul(hx_context *ctx, const hx_keyset *ks, const hx_ct *A, const hx_ct *B, int h, hx_ct **out,
                    void *stream)
{
    HX_TRY
    need(ctx && ks && A && B && out, "null argument");
    *out = nullptr;
    mine(ctx, ks);
    mine(ctx, A);
    mine(ctx, B);
    PlanUse p(*ctx, S(stream), cached_plan(*ctx, h, A->c.limbs));
    *out = wrap(ctx, matmul_batch(*ctx, *ks, *p.p, A->c, B->c, S(stream)));
    return HX_OK;
    HX_END
}

hx_status hx_matmul_batch(hx_context *ctx, const hx_keyset *ks, const hx_matmul_plan *plan, const hx_ct *const *A,
                          const hx_ct *const *B, int h, size_t count, hx_ct **out, void *stream)
{
    HX_TRY
    need(ctx && ks && A && B && out && count >= 1, "null argument");
    for (size_t i = 0; i < count; i++) out[i] = nullptr;
    need(count < 4096, "batch too large");
    mine(ctx, ks);
    if (plan) mine(ctx, plan);
    Cts a = gather(*ctx, A, count, S(stream));
    Cts b = gather(*ctx, B, count, S(stream));
    PlanUse held(*ctx, S(stream), plan ? nullptr : cached_plan(*ctx, h, a.limbs));
    const hx_matmul_plan *p = plan ? plan : held.p.get();
    need(p->h == h && p->kind == 0, "plan built for another h");
    Cts r = matmul_batch(*ctx, *ks, *p, a, b, S(stream));
    scatter(*ctx, r, out, S(stream));
    return HX_OK;
    HX_END
}

int hx_rmatmul_rotation_steps(const hx_context *ctx, int h, int t, int limbs, int32_t *out, int cap)
{
    if (!ctx || h < 2 || (h & (h - 1)) || h * h > ctx->N / 2 || limbs < 3) return HX_EINVAL;
    if (t < 1 || t > h || (t & (t - 1))) return HX_EINVAL;
    std::vector<int64_t> st = plan_rotation_steps(h, ctx->N / 2 / (h * h), limbs, t);
    for (int i = 0; i < (int)st.size() && i < cap; i++) out[i] = (int32_t)st[i];
    return (int)st.size();
}

hx_status hx_matmul_batch_mixed(hx_context *ctx, const hx_keyset *ks, const hx_ct *const *A, const hx_ct *const *B,
                                const int *h, size_t count, hx_ct **out, void *stream)
{
    HX_TRY
    need(ctx && ks && A && B && h && out && count >= 1 && count < 65536, "bad argument");
    for (size_t i = 0; i < count; i++) out[i] = nullptr;
    mine(ctx, ks);
    std::vector<hx_matmul_job> jobs(count);
    for (size_t i = 0; i < count; i++) jobs[i] = hx_matmul_job{ctx, ks, A[i], B[i], h[i]};
    return hx_matmul_jobs(jobs.data(), count, out, stream);
    HX_END
}

hx_status hx_matmul_jobs(const hx_matmul_job *jobs, size_t count, hx_ct **out, void *stream)
{
    HX_TRY
    need(jobs && out && count >= 1 && count < 65536, "bad argument");
    for (size_t i = 0; i < count; i++) out[i] = nullptr;
    // entries of one (context, keys, h, level, scale) form a group, in order of first appearance
    std::map<std::tuple<hx_context *, const hx_keyset *, int, int, double>, size_t> gid;
    std::vector<MatmulGroup> groups;
    int dev = -1;
    for (size_t i = 0; i < count; i++) {
        const hx_matmul_job &J = jobs[i];
        need(J.ctx && J.ks && J.A && J.B, "null job field");
        mine(J.ctx, J.ks);
        mine(J.ctx, J.A);
        mine(J.ctx, J.B);
        need(dev < 0 || J.ctx->device == dev, "jobs on several devices");
        dev = J.ctx->device;
        need(J.h >= 2 && (J.h & (J.h - 1)) == 0 && J.h * J.h <= J.ctx->N / 2,
             "h must be a power of two with h^2 <= N/2");
        HX_CHECK(J.A->c.comps == 2 && J.B->c.comps == 2 && J.A->c.limbs == J.B->c.limbs &&
                     J.A->c.scale == J.B->c.scale,
                 HX_ESCALE, "entry " + std::to_string(i) + ": A and B must be ciphertexts of one level and scale");
        const auto key = std::make_tuple(J.ctx, J.ks, J.h, J.A->c.limbs, J.A->c.scale);
        auto it = gid.find(key);
        if (it == gid.end()) {
            it = gid.emplace(key, groups.size()).first;
            groups.push_back(MatmulGroup{J.ctx, J.ks, J.h, {}, {}, {}});
        }
        MatmulGroup &G = groups[it->second];
        G.idx.push_back(i);
        G.A.push_back(J.A);
        G.B.push_back(J.B);
    }
    run_matmul_groups(groups, S(stream), out, count);
    return HX_OK;
    HX_END
}

hx_status hx_rmatmul_batch(hx_context *ctx, const hx_keyset *ks, const hx_matmul_plan *plan, const hx_ct *const *At,
                           const hx_ct *const *B, int h, int t, size_t count, hx_ct **out, void *stream)
{
    HX_TRY
    need(ctx && ks && At && B && out && count >= 1 && count < 4096, "bad argument");
    for (size_t i = 0; i < count; i++) out[i] = nullptr;
    mine(ctx, ks);
    if (plan) mine(ctx, plan);
    Cts a = gather(*ctx, At, count, S(stream));
    Cts b = gather(*ctx, B, count, S(stream));
    PlanUse held(*ctx, S(stream), plan ? nullptr : cached_plan(*ctx, h, a.limbs));
    const hx_matmul_plan *p = plan ? plan : held.p.get();
    need(p->h == h && p->kind == 0, "plan built for another h");
    scatter(*ctx, rmatmul_batch(*ctx, *ks, *p, a, b, t, S(stream)), out, S(stream));
    return HX_OK;
    HX_END
}

hx_status hx_transpose_plan_create(hx_context *ctx, int h, int limbs, hx_matmul_plan **out)
{
    HX_TRY
    need(ctx && out, "null argument");
    *out = nullptr;
    *out = make_transpose_plan(*ctx, h, limbs, nullptr);
    return HX_OK;
    HX_END
}

int hx_transpose_rotation_steps(const hx_context *ctx, int h, int32_t *out, int cap)
{
    if (!ctx || h < 2 || (h & (h - 1)) || h * h > ctx->N / 2) return HX_EINVAL;
    std::vector<int64_t> st = transpose_rotation_steps(h, ctx->N / 2 / (h * h));
    for (int i = 0; i < (int)st.size() && i < cap; i++) out[i] = (int32_t)st[i];
    return (int)st.size();
}

hx_status hx_transpose(hx_context *ctx, const hx_keyset *ks, const hx_matmul_plan *plan, const hx_ct *const *x,
                       int h, size_t count, hx_ct **out, void *stream)
{
    HX_TRY
    need(ctx && ks && x && out && count >= 1 && count < 4096, "bad argument");
    for (size_t i = 0; i < count; i++) out[i] = nullptr;
    mine(ctx, ks);
    if (plan) mine(ctx, plan);
    Cts a = gather(*ctx, x, count, S(stream));
    PlanUse held(*ctx, S(stream), plan ? nullptr : cached_transpose_plan(*ctx, h, a.limbs));
    const hx_matmul_plan *p = plan ? plan : held.p.get();
    need(p->h == h && p->kind == 1, "plan built for another shape");
    scatter(*ctx, transpose_batch(*ctx, *ks, *p, a, S(stream)), out, S(stream));
    return HX_OK;
    HX_END
}

hx_status hx_matmul_exec_create(hx_context *ctx, const hx_keyset *ks, const hx_matmul_plan *plan, size_t count,
                                double scale, hx_matmul_exec **out)
{
    HX_TRY
    need(ctx && ks && plan && out && count >= 1 && count < 4096 && scale > 0, "bad argument");
    *out = nullptr;
    mine(ctx, ks);
    mine(ctx, plan);
    std::unique_ptr<hx_matmul_exec> ex(new hx_matmul_exec);
    ex->ctx = ctx;
    ex->ks = ks;
    ex->plan = plan;
    ex->count = count;
    const size_t N = ctx->N;
    auto persistent = [&](int limbs) {
        Cts c;
        c.B = (int)count;
        c.comps = 2;
        c.limbs = c.cap = limbs;
        c.buf = std::make_shared<DevBuf>((size_t)count * 2 * limbs * N, true);
        c.d = c.buf->p;
        c.scale = scale;
        return c;
    };
    ex->A = persistent(plan->limbs);
    ex->B = persistent(plan->limbs);
    ex->out = persistent(plan->alg3 ? plan->limbs - 3 : plan->limbs - 2);  // allocated before the capture
    HX_CUDA(cudaMemset(ex->A.d, 0, sizeof(uint64_t) * ex->A.bstride(N) * count));
    HX_CUDA(cudaMemset(ex->B.d, 0, sizeof(uint64_t) * ex->B.bstride(N) * count));
    HX_CUDA(cudaDeviceSynchronize());
    HX_CUDA(cudaStreamCreateWithFlags(&ex->cap, cudaStreamNonBlocking));
    side_stream(*ctx, ex->cap);  // the schedule's side stream exists before the capture starts
    const uint64_t l0 = ctx->counters[C_LAUNCH];
    uint64_t saved[C_NUM];
    for (int i = 0; i < C_NUM; i++) saved[i] = ctx->counters[i];
    const bool prof = ctx->profiling;
    ctx->profiling = false;
    cudaGraph_t graph = nullptr;
    HX_CUDA(cudaStreamBeginCapture(ex->cap, cudaStreamCaptureModeThreadLocal));
    try {
        Cts r = matmul_batch(*ctx, *ks, *plan, ex->A, ex->B, ex->cap);
        HX_CHECK(r.limbs == ex->out.limbs, HX_EINVAL, "unexpected output level");
        ex->out.scale = r.scale;
        HX_CUDA(cudaMemcpyAsync(ex->out.d, r.d, sizeof(uint64_t) * r.bstride(N) * count, cudaMemcpyDeviceToDevice,
                                ex->cap));
    } catch (...) {
        cudaStreamEndCapture(ex->cap, &graph);
        if (graph) cudaGraphDestroy(graph);
        ctx->profiling = prof;
        throw;
    }
    HX_CUDA(cudaStreamEndCapture(ex->cap, &graph));
    ctx->profiling = prof;
    ex->launches = (int64_t)(ctx->counters[C_LAUNCH] - l0);
    for (int i = 0; i < C_NUM; i++) ctx->counters[i] = saved[i];  // a capture executes nothing
    cudaError_t e = cudaGraphInstantiate(&ex->exec, graph, 0);
    cudaGraphDestroy(graph);
    HX_CUDA(e);
    *out = ex.release();
    return HX_OK;
    HX_END
}

hx_status hx_matmul_exec_run(hx_matmul_exec *ex, const hx_ct *const *A, const hx_ct *const *B, hx_ct **out,
                             void *stream)
{
    HX_TRY
    need(ex && A && B && out, "null argument");
    hx_context &ctx = *ex->ctx;
    const size_t N = ctx.N;
    for (size_t i = 0; i < ex->count; i++) {
        out[i] = nullptr;
        need(A[i] && B[i], "null ciphertext");
        mine(ex->ctx, A[i]);
        mine(ex->ctx, B[i]);
        HX_CHECK(A[i]->c.limbs == ex->plan->limbs && B[i]->c.limbs == ex->plan->limbs, HX_ELEVEL,
                 "inputs are not at the executor's level");
        HX_CHECK(A[i]->c.scale == ex->A.scale && B[i]->c.scale == ex->A.scale, HX_ESCALE,
                 "inputs must have the executor's scale");
    }
    cudaStream_t s = S(stream);
    for (size_t i = 0; i < ex->count; i++)
        for (int c = 0; c < 2; c++) {
            HX_CUDA(cudaMemcpyAsync(ex->A.d + i * ex->A.bstride(N) + c * ex->A.cstride(N),
                                    A[i]->c.d + c * A[i]->c.cstride(N), sizeof(uint64_t) * ex->A.limbs * N,
                                    cudaMemcpyDeviceToDevice, s));
            HX_CUDA(cudaMemcpyAsync(ex->B.d + i * ex->B.bstride(N) + c * ex->B.cstride(N),
                                    B[i]->c.d + c * B[i]->c.cstride(N), sizeof(uint64_t) * ex->B.limbs * N,
                                    cudaMemcpyDeviceToDevice, s));
        }
    HX_CUDA(cudaGraphLaunch(ex->exec, s));
    ctx.counters[C_LAUNCH] += ex->launches;
    scatter(ctx, ex->out, out, s);
    return HX_OK;
    HX_END
}

hx_status hx_matmul_exec_run_host(hx_matmul_exec *ex, const uint64_t *host_A, const uint64_t *host_B,
                                  uint64_t *host_out, void *stream)
{
    HX_TRY
    need(ex && host_A && host_B && host_out, "null argument");
    const size_t N = ex->ctx->N;
    cudaStream_t s = S(stream);
    // the executor's buffers are [count][2][limbs][N] with no gaps, the host layout
    HX_CUDA(cudaMemcpyAsync(ex->A.d, host_A, sizeof(uint64_t) * ex->A.bstride(N) * ex->count, cudaMemcpyHostToDevice,
                            s));
    HX_CUDA(cudaMemcpyAsync(ex->B.d, host_B, sizeof(uint64_t) * ex->B.bstride(N) * ex->count, cudaMemcpyHostToDevice,
                            s));
    HX_CUDA(cudaGraphLaunch(ex->exec, s));
    ex->ctx->counters[C_LAUNCH] += ex->launches;
    HX_CUDA(cudaMemcpyAsync(host_out, ex->out.d, sizeof(uint64_t) * ex->out.bstride(N) * ex->count,
                            cudaMemcpyDeviceToHost, s));
    return HX_OK;
    HX_END
}

hx_status hx_matmul_exec_out_info(const hx_matmul_exec *ex, int *limbs, double *scale)
{
    if (!ex) return HX_EINVAL;
    if (limbs) *limbs = ex->out.limbs;
    if (scale) *scale = ex->out.scale;
    return HX_OK;
}

int64_t hx_matmul_exec_launches(const hx_matmul_exec *ex) { return ex ? ex->launches : HX_EINVAL; }

void hx_matmul_exec_destroy(hx_matmul_exec *ex)
{
    if (!ex) return;
    cudaDeviceSynchronize();
    if (ex->exec) cudaGraphExecDestroy(ex->exec);
    if (ex->cap) cudaStreamDestroy(ex->cap);
    delete ex;
}

hx_status hx_sign_approx(hx_context *ctx, const hx_keyset *ks, const hx_ct *x, int d, int k, int relu,
                         int allow_refresh, uint64_t refresh_seed, hx_ct **out, void *stream)
{
    HX_TRY
    need(ctx && ks && x && out, "null argument");
    *out = nullptr;
    mine(ctx, ks);
    mine(ctx, x);
    *out = wrap(ctx, sign_batch(*ctx, *ks, x->c, d, k, relu != 0, allow_refresh != 0, {refresh_seed}, S(stream)));
    return HX_OK;
    HX_END
}

hx_status hx_sign_approx_batch(hx_context *ctx, const hx_keyset *ks, const hx_ct *const *x, size_t count, int d,
                               int k, int relu, int allow_refresh, uint64_t refresh_seed, hx_ct **out, void *stream)
{
    HX_TRY
    need(ctx && ks && x && out && count >= 1 && count < 4096, "bad argument");
    for (size_t i = 0; i < count; i++) out[i] = nullptr;
    mine(ctx, ks);
    Cts a = gather(*ctx, x, count, S(stream));
    std::vector<uint64_t> seeds(count);
    for (size_t i = 0; i < count; i++) seeds[i] = refresh_seed + i;
    Cts r = sign_batch(*ctx, *ks, a, d, k, relu != 0, allow_refresh != 0, seeds, S(stream));
    scatter(*ctx, r, out, S(stream));
    return HX_OK;
    HX_END
}

hx_status hx_dense_layer(hx_context *ctx, const hx_keyset *ks, const hx_matmul_plan *fwd_plan,
                         const hx_matmul_plan *transpose_plan, const hx_matmul_plan *bwd_plan, const hx_ct *const *W,
                         const hx_ct *const *X, const hx_ct *const *G, int h, int n_out, int groups, int d, int k,
                         double input_div, uint64_t refresh_seed, hx_ct **E, hx_ct **M, hx_ct **dW, void *stream)
{
    HX_TRY
    need(ctx && ks && W && X && G && E && M && dW, "null argument");
    need(n_out >= 1 && groups >= 1 && (size_t)n_out * groups < 4096, "bad block counts");
    for (int i = 0; i < n_out; i++) E[i] = M[i] = nullptr;
    for (int i = 0; i < n_out * groups; i++) dW[i] = nullptr;
    need(h >= 2 && (h & (h - 1)) == 0 && h * h <= ctx->N / 2, "h must be a power of two with h^2 <= N/2");
    mine(ctx, ks);
    for (const hx_matmul_plan *p : {fwd_plan, transpose_plan, bwd_plan})
        if (p) mine(ctx, p);
    std::vector<const hx_ct *> wg((size_t)n_out * groups);
    for (int i = 0; i < n_out; i++)
        for (int g = 0; g < groups; g++) wg[(size_t)g * n_out + i] = W[(size_t)i * groups + g];
    Cts w = gather(*ctx, wg.data(), wg.size(), S(stream));
    Cts x = gather(*ctx, X, groups, S(stream));
    Cts gr = gather(*ctx, G, n_out, S(stream));
    need(!fwd_plan || fwd_plan->kind == 0, "fwd_plan is not a matmul plan");
    need(!bwd_plan || bwd_plan->kind == 0, "bwd_plan is not a matmul plan");
    need(!transpose_plan || transpose_plan->kind == 1, "transpose_plan is not a transpose plan");
    DensePlans plans;
    plans.fwd = fwd_plan;
    plans.transpose = transpose_plan;
    plans.bwd = bwd_plan;
    DenseResult r = dense_batch(*ctx, *ks, plans, w, x, gr, h, d, k, input_div, refresh_seed, S(stream));
    std::vector<hx_ct *> dg((size_t)n_out * groups);
    scatter(*ctx, r.E, E, S(stream));
    scatter(*ctx, r.M, M, S(stream));
    scatter(*ctx, r.dW, dg.data(), S(stream));
    for (int i = 0; i < n_out; i++)
        for (int g = 0; g < groups; g++) dW[(size_t)i * groups + g] = dg[(size_t)g * n_out + i];
    return HX_OK;
    HX_END
}

int hx_dense_rotation_steps(const hx_context *ctx, int h, int32_t *out, int cap)
{
    if (!ctx || h < 2 || (h & (h - 1)) || h * h > ctx->N / 2) return HX_EINVAL;
    std::vector<int64_t> st = dense_rotation_steps(h, ctx->N / 2 / (h * h));
    for (int i = 0; i < (int)st.size() && i < cap; i++) out[i] = (int32_t)st[i];
    return (int)st.size();
}

hx_status hx_aggregate(hx_context *ctx, const hx_ct *const *grads, size_t n_parties, const hx_ct *const *models,
                       size_t count, double eta_over_bn, hx_ct **out, void *stream)
{
    HX_TRY
    need(ctx && grads && models && out && n_parties >= 1 && count >= 1 && count < 4096 && n_parties < 65536,
         "bad argument");
    for (size_t i = 0; i < count; i++) out[i] = nullptr;
    std::vector<const Cts *> g(n_parties * count);
    for (size_t i = 0; i < g.size(); i++) {
        need(grads[i] && grads[i]->ctx == ctx, "gradient from another context");
        g[i] = &grads[i]->c;
    }
    Cts m = gather(*ctx, models, count, S(stream));
    scatter(*ctx, aggregate(*ctx, g, (int)n_parties, m, eta_over_bn, S(stream)), out, S(stream));
    return HX_OK;
    HX_END
}

hx_status hx_dkeyswitch(hx_context *ctx, const hx_keyset *from, const hx_keyset *to, const hx_ct *ct, uint64_t seed,
                        hx_ct **out, void *stream)
{
    HX_TRY
    need(ctx && from && to && ct && out, "null argument");
    *out = nullptr;
    need(from->ctx == ctx && to->ctx == ctx && ct->ctx == ctx, "keys or ciphertext from another context");
    *out = wrap(ctx, dkeyswitch(*ctx, *from, *to, ct->c, seed, S(stream)));
    return HX_OK;
    HX_END
}

hx_status hx_dbootstrap(hx_context *ctx, const hx_keyset *ks, const hx_ct *ct, uint64_t seed, hx_ct **out, void *stream)
{
    HX_TRY
    need(ctx && ks && ct && out, "null argument");
    *out = nullptr;
    need(ks->ctx == ctx && ct->ctx == ctx, "keys or ciphertext from another context");
    *out = wrap(ctx, dbootstrap(*ctx, *ks, ct->c, {seed}, 0, S(stream)));
    return HX_OK;
    HX_END
}

hx_status hx_alu_calibrate(hx_context *ctx, double *shoup_per_s, double *mac_per_s, void *stream)
{
    HX_TRY
    need(ctx && shoup_per_s && mac_per_s, "null argument");
    Eval ev(*ctx, S(stream));
    alu_calibrate(ev.lc(), ctx->primes[0], shoup_per_s, mac_per_s);
    return HX_OK;
    HX_END
}

int hx_counters(const hx_context *ctx, uint64_t *out, int cap)
{
    if (!ctx) return HX_EINVAL;
    for (int i = 0; i < C_NUM && i < cap; i++) out[i] = ctx->counters[i];
    return C_NUM;
}

void hx_counters_reset(hx_context *ctx)
{
    if (ctx)
        for (int i = 0; i < C_NUM; i++) ctx->counters[i] = 0;
}

// a tuned NTT variant as the signed width of the public calls: negative = swapped radices
static int variant_width(int v) { return v >= NTT_WIDTHS ? -kNttTileWidths[v % NTT_WIDTHS] : kNttTileWidths[v]; }

hx_status hx_autotune(hx_context *ctx, int32_t *choice, void *stream)
{
    HX_TRY
    need(ctx, "null argument");
    // one scratch buffer for the largest batch timed; every bucket of batch sizes is tuned on
    // its own number of limbs (the widths that fill the SMs best depend on the batch)
    const int rows_max = std::min(kNttBucketTune[NTT_BUCKETS - 1], MAX_NTT_ROWS);
    DevBuf buf((size_t)rows_max * ctx->N, S(stream));
    HX_CUDA(cudaMemsetAsync(buf.p, 0, sizeof(uint64_t) * rows_max * ctx->N, S(stream)));
    Eval ev(*ctx, S(stream));
    for (int b = 0; b < NTT_BUCKETS; b++) {
        int best[5] = {2, 2, 2, 2, 0};
        float ms[4];
        autotune_ntt(ev.lc(), buf.p, std::min(kNttBucketTune[b], rows_max), best, ms);
        for (int i = 0; i < 5; i++) ctx->t.ntt_var[b][i] = best[i];
    }
    if (choice)
        for (int i = 0; i < 4; i++) choice[i] = variant_width(ctx->t.ntt_var[1][i]);
    return HX_OK;
    HX_END
}

hx_status hx_ntt_tiles(hx_context *ctx, const int32_t *set, int32_t *get)
{
    HX_TRY
    need(ctx, "null argument");
    if (set) {
        int v[4];
        for (int i = 0; i < 4; i++) {
            v[i] = -1;
            for (int k = 0; k < NTT_WIDTHS; k++) {
                if (set[i] == kNttTileWidths[k]) v[i] = k;
                if (set[i] == -kNttTileWidths[k]) v[i] = k + NTT_WIDTHS;
            }
            need(v[i] >= 0, "tile width must be 4, 8, 16 or 32 (negative: swapped radices)");
        }
        for (int b = 0; b < NTT_BUCKETS; b++) {
            for (int i = 0; i < 4; i++) ctx->t.ntt_var[b][i] = v[i];
            ctx->t.ntt_var[b][4] = 0;  // the default split of an odd log N
        }
    }
    if (get)
        for (int i = 0; i < 4; i++) get[i] = variant_width(ctx->t.ntt_var[1][i]);
    return HX_OK;
    HX_END
}

hx_status hx_ntt_split(hx_context *ctx, int split)
{
    HX_TRY
    need(ctx && (split == 0 || split == 1), "split must be 0 or 1");
    for (int b = 0; b < NTT_BUCKETS; b++) ctx->t.ntt_var[b][4] = split;
    return HX_OK;
    HX_END
}

int hx_ntt_tuning(const hx_context *ctx, int32_t *out, int cap)
{
    if (!ctx || (!out && cap > 0)) return HX_EINVAL;
    int n = 0;
    for (int b = 0; b < NTT_BUCKETS; b++) {
        const int32_t row[7] = {kNttBucketMax[b], kNttBucketTune[b], variant_width(ctx->t.ntt_var[b][0]),
                                variant_width(ctx->t.ntt_var[b][1]), variant_width(ctx->t.ntt_var[b][2]),
                                variant_width(ctx->t.ntt_var[b][3]), ctx->t.ntt_var[b][4]};
        for (int k = 0; k < 7; k++, n++)
            if (n < cap) out[n] = row[k];
    }
    return n;
}

hx_status hx_profile_enable(hx_context *ctx, int on)
{
    HX_TRY
    need(ctx, "null argument");
    HX_CUDA(cudaDeviceSynchronize());
    ctx->prof.clear();
    ctx->profiling = on != 0;
    return HX_OK;
    HX_END
}

int hx_profile_read(hx_context *ctx, int i, char *name, size_t cap, uint64_t *launches, double *ms, double *bytes)
{
    HX_TRY
    need(ctx, "null argument");
    if (i < 0 || i >= K_NCLASS) return HX_EINVAL;
    HX_CUDA(cudaDeviceSynchronize());
    uint64_t n = 0;
    double t = 0, b = 0;
    for (auto &r : ctx->prof.recs)
        if (r.cls == i) {
            float e = 0;
            HX_CUDA(cudaEventElapsedTime(&e, r.a, r.b));
            n++;
            t += e;
            b += r.bytes;
        }
    if (name && cap) {
        strncpy(name, kclass_names[i], cap - 1);
        name[cap - 1] = 0;
    }
    if (launches) *launches = n;
    if (ms) *ms = t;
    if (bytes) *bytes = b;
    return K_NCLASS;
    HX_END
}

} // extern "C"
