// A slot rotation that allocates no device memory.
//
// Some callers cannot ask the CUDA runtime for memory at the moment they
// need a rotation: an application whose memory manager has already claimed
// the device (cudaMalloc then fails although that manager has room), a
// latency-critical loop that cannot afford cudaMalloc's implicit
// synchronisation, or a host that forbids plug-in code from allocating after
// start-up.  hx_rotate_noalloc serves them: the caller passes the input and
// output ciphertext buffers, and every intermediate of the key switch lives in
// one static device array of fixed size that the library reserves on each
// device it is loaded on, until the process exits.
#include <mutex>
#include <new>
#include <stdexcept>

#include "runtime.h"

namespace {

constexpr size_t kScratchWords = HX_NOALLOC_SCRATCH_BYTES / sizeof(uint64_t);
__device__ __align__(256) uint64_t g_rot_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint64_t *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the static scratch array for the current device, looked
// up once per device (host code cannot use the array's name as an address).
uint64_t *scratch_for_current_device()
{
    int dev = 0;
    HX_CUDA(cudaGetDevice(&dev));
    HX_CHECK(dev >= 0 && dev < kMaxDevices, HX_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        HX_CUDA(cudaGetSymbolAddress(&p, g_rot_scratch));
        g_scratch_ptr[dev] = static_cast<uint64_t *>(p);
    }
    return g_scratch_ptr[dev];
}

} // namespace

using namespace hx;

extern "C" hx_status hx_rotate_noalloc(hx_context *ctx, const hx_keyset *ks, const uint64_t *in, int limbs,
                                       uint64_t *out, int32_t k, void *stream)
{
    try {
        HX_CHECK(ctx && ks && in && out, HX_EINVAL, "null argument");
        HX_CHECK(limbs >= 1 && limbs <= ctx->n_q, HX_EINVAL, "bad level");
        const int N = ctx->N, K = ctx->K, A = ctx->alpha, ext = limbs + K, nd = (limbs + A - 1) / A;
        const size_t n = (size_t)N;
        // tmp and coef: limbs rows each; D: nd*ext rows; acc: 2*ext rows; conv: 2*limbs rows
        const size_t need = n * (4 * (size_t)limbs + (size_t)(nd + 2) * ext);
        HX_CHECK(need <= kScratchWords, HX_EINVAL,
                 "rotation needs " + std::to_string(need * 8) + " bytes of scratch, more than the " +
                     std::to_string((unsigned long long)HX_NOALLOC_SCRATCH_BYTES) + "-byte static scratch");
        // keys of another context would be read with this context's row length and strides
        HX_CHECK(ks->ctx == ctx, HX_EINVAL, "keys of another context");
        // the last kernel reads sigma_g(c0) from `in` at permuted indices while it writes `out`
        const size_t words = 2 * (size_t)limbs * N;
        HX_CHECK(out + words <= in || in + words <= out, HX_EINVAL, "in and out overlap");
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        const uint64_t g = galois_for_step(k, ctx->log_n);
        if (g == 1) {
            HX_CUDA(cudaMemcpyAsync(out, in, sizeof(uint64_t) * 2 * limbs * n, cudaMemcpyDeviceToDevice, s));
            return HX_OK;
        }
        auto it = ks->rot.find(g);
        HX_CHECK(it != ks->rot.end(), HX_EKEY, "missing Galois key for element " + std::to_string(g));
        uint64_t *base = scratch_for_current_device();
        uint64_t *tmp = base, *coef = tmp + limbs * n, *D = coef + limbs * n, *acc = D + (size_t)nd * ext * n;
        uint64_t *conv = acc + 2 * (size_t)ext * n;
        LaunchCtx lc{ctx->log_n, N, &ctx->t, s, &ctx->counters[C_LAUNCH], nullptr};
        const View vin{const_cast<uint64_t *>(in), 2 * limbs * n, limbs * n};
        // sigma_g(c1), then ModUp of it
        launch_automorphism(lc, View{tmp, limbs * n, n}, View{vin.p + vin.cstride, vin.bstride, vin.cstride}, g, 1, 1,
                            limbs);
        NttRows r;
        r.src = tmp;
        r.dst = coef;
        r.src_gs = r.dst_gs = limbs * n;
        r.n_groups = 1;
        r.n_rows = limbs;
        for (int l = 0; l < limbs; l++) r.src_off[l] = r.dst_off[l] = r.prime[l] = (int16_t)l;
        launch_ntt(lc, r, true);
        launch_basis_convert(lc, ctx->t.modup + (size_t)limbs * ctx->dnum, A, View{D, (size_t)nd * ext * n, 0},
                             View{coef, limbs * n, 0}, 1, nd, (size_t)ext * n, 0);
        r.src = r.dst = D;
        r.src_gs = r.dst_gs = (size_t)nd * ext * n;
        r.n_rows = 0;
        for (int j = 0; j < nd; j++) {
            const int lo = j * A, hi = std::min((j + 1) * A, limbs);
            for (int row = 0; row < ext; row++) {
                if (row >= lo && row < hi) continue;
                r.src_off[r.n_rows] = r.dst_off[r.n_rows] = (int16_t)(j * ext + row);
                r.prime[r.n_rows] = (int16_t)(row < limbs ? row : ctx->n_q + (row - limbs));
                r.n_rows++;
            }
        }
        launch_ntt(lc, r, false);
        // key inner product and ModDown, sigma_g(c0) added to the first component
        View accv{acc, 2 * (size_t)ext * n, (size_t)ext * n};
        launch_key_ip(lc, accv, D, tmp, limbs * n, it->second.buf->p, ctx->n_all, ctx->n_q, K, A, limbs, nd, 1, 1);
        r.src = r.dst = acc;
        r.src_gs = r.dst_gs = (size_t)ext * n;
        r.n_groups = 2;
        r.n_rows = K;
        for (int kk = 0; kk < K; kk++) {
            r.src_off[kk] = r.dst_off[kk] = (int16_t)(limbs + kk);
            r.prime[kk] = (int16_t)(ctx->n_q + kk);
        }
        launch_ntt(lc, r, true);
        launch_basis_convert(lc, reinterpret_cast<const ConvTable *>(ctx->t.moddown + limbs), ctx->K,
                             View{conv, limbs * n, 0}, View{acc, (size_t)ext * n, 0}, 2, 1, 0, 0);
        r.src = r.dst = conv;
        r.src_gs = r.dst_gs = limbs * n;
        r.n_rows = limbs;
        for (int l = 0; l < limbs; l++) r.src_off[l] = r.dst_off[l] = r.prime[l] = (int16_t)l;
        launch_ntt(lc, r, false);
        launch_moddown_final(lc, View{out, 2 * limbs * n, limbs * n}, accv, View{conv, 2 * limbs * n, limbs * n},
                             ctx->t.moddown + limbs, 1, limbs, vin, 1, g);
        ctx->counters[C_ROT] += 1;
        ctx->counters[C_KS] += 1;
        ctx->counters[C_MODUP] += 1;
        return HX_OK;
    } catch (const hx::Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return HX_ENOMEM;
    } catch (const std::exception &e) {  // e.g. std::system_error from the mutex
        set_error(e.what());
        return HX_EINVAL;
    }
}
