// Schedules of the paper's method on batched ciphertexts:
//  * HE-LinTrans (Alg. 2) with the baby-step/giant-step split of App. B,
//  * HE-MatMult (Alg. 3) with the multiplexer trick of App. B and the
//    iota_beta packing of App. E, plus a depth-2 rearrangement of Steps 2-3
//    for chains with exactly two levels above q_0,
//  * the composite sign g_d^(k) and ReLU (Sec. 4, Alg. 5) with a host
//    simulation of DBootstrap when the levels run out.
#include <algorithm>
#include <cmath>

#include <set>

#include <tuple>

#include "runtime.h"

namespace hx {

namespace {

int baby_steps(int h)
{
    int lg = 0;
    while ((1 << lg) < h) lg++;
    return 1 << ((lg + 1) / 2);  // 2^ceil(log2(h)/2)
}

int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
int posmod(int a, int b) { return ((a % b) + b) % b; }

// diagonal vectors of Sec. 3.6 (logical length h^2)
std::vector<int32_t> diag_mu(int h, int k)
{
    std::vector<int32_t> v(h * h, 0);
    for (int t = 0; t < h * h; t++) {
        if (k >= 0)
            v[t] = (t - h * k >= 0 && t - h * k < h - k);
        else
            v[t] = (t - (h + k) * h >= -k && t - (h + k) * h < h);
    }
    return v;
}
std::vector<int32_t> diag_zeta(int h, int k)
{
    std::vector<int32_t> v(h * h, 0);
    for (int t = 0; t < h * h; t++) v[t] = (t % h == k);
    return v;
}
std::vector<int32_t> diag_v(int h, int k)
{
    std::vector<int32_t> v(h * h, 0);
    for (int t = 0; t < h * h; t++) v[t] = ((t % h) < h - k);
    return v;
}
// diagonal (h-1)s of the transpose (App. C): 1 at t = (h+1)i + s, max(0,-s) <= i < h - max(0,s)
std::vector<int32_t> diag_transpose(int h, int sh)
{
    std::vector<int32_t> v(h * h, 0);
    for (int t = 0; t < h * h; t++) {
        const int d = t - sh;
        if (d % (h + 1) != 0) continue;
        const int i = d >= 0 ? d / (h + 1) : -((-d + h) / (h + 1));
        v[t] = (i >= std::max(0, -sh) && i < h - std::max(0, sh));
    }
    return v;
}

// R(v, r): (v_r, ..., v_{n-1}, v_0, ..., v_{r-1})
std::vector<int32_t> rot(const std::vector<int32_t> &v, int r)
{
    const int n = (int)v.size();
    std::vector<int32_t> o(n);
    for (int t = 0; t < n; t++) o[t] = v[posmod(t + r, n)];
    return o;
}

} // namespace

std::vector<int64_t> plan_rotation_steps(int h, int beta, int limbs, int t)
{
    t = t ? t : h;
    const int b = baby_steps(h);
    const bool alg3 = limbs >= 4;
    std::vector<int64_t> s;
    for (int l = -h + 1; l < h; l++) {
        s.push_back((int64_t)beta * posmod(l, b));
        s.push_back((int64_t)beta * b * floordiv(l, b));
    }
    if (alg3) {
        for (int l = 0; l < h; l++) {
            s.push_back((int64_t)beta * h * (l % b));
            s.push_back((int64_t)beta * h * b * (l / b));
        }
    } else {
        for (int l = 1; l < h; l++) s.push_back((int64_t)beta * h * l);
    }
    for (int k = 1; k < t; k++) {
        s.push_back((int64_t)beta * k);
        s.push_back((int64_t)beta * (k - h));
        s.push_back((int64_t)beta * h * k);
    }
    for (int e = t; e < h; e *= 2) s.push_back((int64_t)beta * h * e);
    const int64_t n = (int64_t)beta * h * h;
    std::vector<int64_t> out;
    for (int64_t x : s) {
        int64_t r = ((x % n) + n) % n;
        if (r) out.push_back(r);
    }
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
    return out;
}

void encode_plan_masks(hx_context &ctx, hx_matmul_plan &pl, cudaStream_t s);

// The masks' scale: the power of two nearest the context's scale, the same at every level (an
// integer, so the multiplexer's constant and the Step-3 multiplier are exact); a product's scale
// after the mask and the rescale by q_(l-1) is then tracked as scale * 2^e / q_(l-1)
static int mask_scale_log2(const hx_context &ctx) { return (int)std::lround(std::log2(ctx.scale)); }
static double mask_scale(const hx_context &ctx) { return std::ldexp(1.0, mask_scale_log2(ctx)); }
static uint64_t mask_scale_int(const hx_context &ctx) { return (uint64_t)1 << mask_scale_log2(ctx); }

// whether the masks' real coefficients of a plan shape are cached (then the 0/1 vectors are not needed)
static bool mask_real_cached(hx_context &ctx, int kind, int h, bool alg3)
{
    std::lock_guard<std::mutex> lk(ctx.mask_real_mu);
    return ctx.mask_real.count(std::make_tuple(kind, h, alg3)) != 0;
}

hx_matmul_plan *make_plan(hx_context &ctx, int h, int limbs, cudaStream_t s)
{
    HX_CHECK(h >= 2 && (h & (h - 1)) == 0 && h * h <= ctx.N / 2, HX_EINVAL, "h must be a power of two with h^2 <= N/2");
    HX_CHECK(limbs <= ctx.n_q, HX_EINVAL, "level above the chain");
    HX_CHECK(limbs >= 3, HX_ELEVEL, "HE-MatMult needs at least 3 limbs");
    std::unique_ptr<hx_matmul_plan> p(new hx_matmul_plan);
    p->ctx = &ctx;
    p->h = h;
    p->limbs = limbs;
    p->beta = ctx.N / 2 / (h * h);
    p->b = baby_steps(h);
    p->alg3 = limbs >= 4;
    const int b = p->b;
    auto add = [&](int kind, int idx, std::vector<int32_t> vec, int lm, bool extended) {
        hx_matmul_plan::Mask m;
        m.kind = kind;
        m.index = idx;
        m.limbs = lm;
        m.extended = extended;
        m.scale = mask_scale(ctx);
        m.vec = std::move(vec);
        p->index[{kind, idx}] = (int)p->masks.size();
        p->masks.push_back(std::move(m));
    };
    const bool vecs = !mask_real_cached(ctx, 0, h, p->alg3);  // else the encodings are already known
    using V = std::vector<int32_t>;
    for (int l = -h + 1; l < h; l++) add(0, l, vecs ? rot(diag_mu(h, l), -b * floordiv(l, b)) : V(), limbs, false);
    for (int l = 0; l < h; l++)
        add(1, l, !vecs ? V() : p->alg3 ? rot(diag_zeta(h, l), -h * b * (l / b)) : diag_zeta(h, l), limbs, false);
    if (p->alg3)  // Step 2 selects after rotating: v_k itself, in the extended basis
        for (int k = 1; k < h; k++) add(2, k, vecs ? diag_v(h, k) : V(), limbs - 1, true);
    encode_plan_masks(ctx, *p, s);
    return p.release();
}

static std::vector<int> iota_rows(int n)
{
    std::vector<int> v(n);
    for (int i = 0; i < n; i++) v[i] = i;
    return v;
}

void encode_plan_masks(hx_context &ctx, hx_matmul_plan &pl, cudaStream_t s)
{
    hx_matmul_plan *p = &pl;
    const int hh = p->h * p->h, M_all = (int)p->masks.size();
    const size_t S = (size_t)ctx.N / 2, N = ctx.N;
    Eval ev(ctx, s);
    // The encoder's real coefficients of every mask depend on the plan's shape only (kind, h,
    // Alg. 3 or the depth-2 form), not on its level: they are computed once per context -- the
    // 0/1 vectors (one byte per matrix entry) go up, are expanded over the beta packed matrices
    // and transformed by the device encoder -- and a plan at any level scales and rounds them
    // (the same coefficients as encoding at that scale, bit for bit).
    const auto shape = std::make_tuple(p->kind, p->h, p->alg3);
    BufPtr real;
    {
        std::lock_guard<std::mutex> lk(ctx.mask_real_mu);
        auto it = ctx.mask_real.find(shape);
        if (it != ctx.mask_real.end()) real = it->second;
    }
    if (!real) {
        std::vector<uint8_t> bits((size_t)M_all * hh);
        for (int r = 0; r < M_all; r++)
            for (int t = 0; t < hh; t++) bits[(size_t)r * hh + t] = p->masks[r].vec[t] != 0;
        DevBuf dbits((bits.size() + 7) / 8, s), dslots((size_t)M_all * S, s);
        HX_CUDA(cudaMemcpyAsync(dbits.p, bits.data(), bits.size(), cudaMemcpyHostToDevice, s));
        launch_expand_masks(ev.lc(), reinterpret_cast<double *>(dslots.p), reinterpret_cast<const uint8_t *>(dbits.p),
                            M_all, hh, p->beta, S);
        real = std::make_shared<DevBuf>((size_t)2 * M_all * N, true);  // double-double per coefficient
        encode_real_batch(ctx, reinterpret_cast<const double *>(dslots.p), S, M_all,
                          reinterpret_cast<double2 *>(real->p), s);
        HX_CUDA(cudaStreamSynchronize(s));
        std::lock_guard<std::mutex> lk(ctx.mask_real_mu);
        auto ins = ctx.mask_real.emplace(shape, real);  // another call may have made it meanwhile
        real = ins.first->second;
    }
    // masks of one scale and basis form a group, moved to NTT and Montgomery form in one batch;
    // every mask is a view into the group's buffer
    std::map<std::tuple<double, int, bool>, std::vector<int>> groups;
    for (int i = 0; i < M_all; i++) {
        const auto &m = p->masks[i];
        groups[std::make_tuple(m.scale, m.limbs, m.extended)].push_back(i);
    }
    for (auto &grp : groups) {
        const std::vector<int> &ids = grp.second;
        const int M = (int)ids.size(), limbs = std::get<1>(grp.first);
        const bool ext = std::get<2>(grp.first);
        const int rows = ext ? limbs + ctx.K : limbs;
        std::vector<int> pr(rows), idx(ids.begin(), ids.end()), prM((size_t)M * rows);
        // an extended mask's rows: the special primes first, then q_0 .. q_(limbs-1), so the mask of a
        // lower level is a prefix of the top level's
        for (int t = 0; t < rows; t++) pr[t] = !ext ? t : t < ctx.K ? ctx.n_q + t : t - ctx.K;
        for (int r = 0; r < M; r++) std::copy(pr.begin(), pr.end(), prM.begin() + (size_t)r * rows);
        DevBuf dpr((prM.size() + 1) / 2, s), didx((idx.size() + 1) / 2, s);
        HX_CUDA(cudaMemcpyAsync(dpr.p, prM.data(), sizeof(int) * prM.size(), cudaMemcpyHostToDevice, s));
        HX_CUDA(cudaMemcpyAsync(didx.p, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, s));
        DevBuf dco((size_t)M * N, s);
        int64_t *co = reinterpret_cast<int64_t *>(dco.p);
        encode_rows_from_real(ctx, reinterpret_cast<const double2 *>(real->p), reinterpret_cast<const int *>(didx.p), M,
                              std::get<0>(grp.first), co, s);
        BufPtr G = std::make_shared<DevBuf>((size_t)M * rows * N, s);
        const int *idp = reinterpret_cast<const int *>(dpr.p);
        launch_signed_to_rows(ev.lc(), G->p, co, rows, M, N, idp);
        ev.ntt_inplace(G->p, (size_t)rows * N, M, iota_rows(rows), pr, false);
        launch_to_mont(ev.lc(), G->p, M * rows, idp);
        for (int r = 0; r < M; r++)
            p->masks[ids[r]].pt = std::make_shared<DevBuf>(G->p + (size_t)r * rows * N, (size_t)rows * N);
        p->storage.push_back(G);
        HX_CUDA(cudaStreamSynchronize(s));  // the staging buffers are released at the end of the group
    }
}

hx_matmul_plan *make_transpose_plan(hx_context &ctx, int h, int limbs, cudaStream_t s)
{
    HX_CHECK(h >= 2 && (h & (h - 1)) == 0 && h * h <= ctx.N / 2, HX_EINVAL, "h must be a power of two with h^2 <= N/2");
    HX_CHECK(limbs >= 2 && limbs <= ctx.n_q, HX_ELEVEL, "the transpose needs a level to rescale");
    std::unique_ptr<hx_matmul_plan> p(new hx_matmul_plan);
    p->ctx = &ctx;
    p->kind = 1;
    p->h = h;
    p->limbs = limbs;
    p->beta = ctx.N / 2 / (h * h);
    p->b = baby_steps(h);
    p->alg3 = false;
    const bool vecs = !mask_real_cached(ctx, 1, h, false);
    for (int sh = -h + 1; sh < h; sh++) {
        hx_matmul_plan::Mask m;
        m.kind = 3;
        m.index = sh;
        m.limbs = limbs;
        m.extended = false;
        m.scale = mask_scale(ctx);
        if (vecs) m.vec = rot(diag_transpose(h, sh), -(h - 1) * p->b * floordiv(sh, p->b));
        p->index[{3, sh}] = (int)p->masks.size();
        p->masks.push_back(std::move(m));
    }
    encode_plan_masks(ctx, *p, s);
    return p.release();
}

namespace {

size_t plan_device_bytes(const hx_matmul_plan &p)
{
    size_t b = 0;
    for (const auto &g : p.storage) b += g->words * sizeof(uint64_t);
    for (const auto &m : p.masks)
        if (m.pt && m.pt->owned) b += m.pt->words * sizeof(uint64_t);
    return b;
}

std::shared_ptr<const hx_matmul_plan> cached_base(hx_context &ctx, int kind, int h, int limbs);

// A plan for `limbs` limbs as a view of `base` (same kind, h and variant, base->limbs >= limbs).
// The masks' coefficients do not depend on the level (one fixed scale), and a mask's NTT rows for
// q_0 .. q_(l-1) are the first rows of the top level's (an extended mask keeps the special primes'
// rows first), so the view's masks point into the base's buffers and the view keeps it alive.
std::shared_ptr<const hx_matmul_plan> level_view(const std::shared_ptr<const hx_matmul_plan> &base, int limbs)
{
    if (base->limbs == limbs) return base;
    const hx_context &ctx = *base->ctx;
    std::shared_ptr<hx_matmul_plan> v(new hx_matmul_plan);
    v->ctx = base->ctx;
    v->kind = base->kind;
    v->h = base->h;
    v->limbs = limbs;
    v->beta = base->beta;
    v->b = base->b;
    v->alg3 = base->alg3;
    v->index = base->index;
    for (const auto &bm : base->masks) {
        hx_matmul_plan::Mask m;
        m.kind = bm.kind;
        m.index = bm.index;
        m.extended = bm.extended;
        m.scale = bm.scale;
        m.limbs = bm.limbs - (base->limbs - limbs);  // limbs, or limbs - 1 for the Step-2 selections
        const size_t rows = (size_t)(m.extended ? m.limbs + ctx.K : m.limbs);
        m.pt = std::make_shared<DevBuf>(bm.pt->p, rows * ctx.N);
        v->masks.push_back(std::move(m));
    }
    v->base = base;
    return v;
}

// The plan of (kind, h, limbs): a view of the context's cached plan of its shape at the top of the
// chain (the depth-2 product, which only runs at 3 limbs, has its own), built on first use
// (outside the lock, on the context's plan stream); the cache may then drop least recently used
// plans no call holds
std::shared_ptr<const hx_matmul_plan> cached(hx_context &ctx, int kind, int h, int limbs)
{
    HX_CHECK(limbs >= 1 && limbs <= ctx.n_q, HX_EINVAL, "level above the chain");
    HX_CHECK(kind == 0 || limbs >= 2, HX_ELEVEL, "the transpose needs a level to rescale");
    const int base_limbs = (kind == 0 && limbs < 4) ? limbs : ctx.n_q;
    return level_view(cached_base(ctx, kind, h, base_limbs), limbs);
}

std::shared_ptr<const hx_matmul_plan> cached_base(hx_context &ctx, int kind, int h, int limbs)
{
    const auto key = std::make_tuple(kind, h, limbs);
    cudaStream_t ps;
    {
        std::lock_guard<std::mutex> lk(ctx.plan_mu);
        auto it = ctx.plans.find(key);
        if (it != ctx.plans.end()) {
            it->second.last = ++ctx.plan_tick;
            return it->second.p;
        }
        if (!ctx.plan_stream) HX_CUDA(cudaStreamCreateWithFlags(&ctx.plan_stream, cudaStreamNonBlocking));
        ps = ctx.plan_stream;
    }
    std::shared_ptr<hx_matmul_plan> built(kind == 0 ? make_plan(ctx, h, limbs, ps)
                                                    : make_transpose_plan(ctx, h, limbs, ps));
    std::lock_guard<std::mutex> lk(ctx.plan_mu);
    auto it = ctx.plans.find(key);
    if (it == ctx.plans.end()) {  // else another call built it meanwhile: keep that one
        hx_context::PlanEntry e;
        e.p = std::move(built);
        e.bytes = plan_device_bytes(*e.p);
        ctx.plan_bytes += e.bytes;
        it = ctx.plans.emplace(key, std::move(e)).first;
    }
    it->second.last = ++ctx.plan_tick;
    std::shared_ptr<const hx_matmul_plan> held = it->second.p;  // not evictable while returned
    trim_plan_cache(ctx);
    return held;
}

void release_plan(void *p) { delete static_cast<std::shared_ptr<const hx_matmul_plan> *>(p); }

} // namespace

void hold_plan_until(hx_context &ctx, cudaStream_t s, std::shared_ptr<const hx_matmul_plan> p) noexcept
{
    if (!p) return;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess || st != cudaStreamCaptureStatusNone) {
        cudaGetLastError();  // a captured graph may replay the work at any time: keep the plan
        std::lock_guard<std::mutex> lk(ctx.plan_mu);
        ctx.plans_pinned.push_back(std::move(p));
        return;
    }
    // the reference is dropped by a host function once s reaches this point; it is never
    // the last one (the cache frees only plans it alone holds), so no CUDA call runs there
    auto *ref = new std::shared_ptr<const hx_matmul_plan>(std::move(p));
    if (cudaLaunchHostFunc(s, release_plan, ref) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(s);
        delete ref;
    }
}

void trim_plan_cache(hx_context &ctx)
{
    while (ctx.plan_bytes > ctx.plan_limit) {
        auto victim = ctx.plans.end();
        for (auto it = ctx.plans.begin(); it != ctx.plans.end(); ++it)
            if (it->second.p.use_count() == 1 && (victim == ctx.plans.end() || it->second.last < victim->second.last))
                victim = it;
        if (victim == ctx.plans.end()) return;  // everything left is in use
        // no call holds it and every stream that used it has passed that work (calls hold
        // their plan until then), so its masks go back to the pool in the plan stream's order
        ctx.plan_bytes -= victim->second.bytes;
        ctx.plans.erase(victim);
        ctx.plan_evictions++;
    }
}

std::shared_ptr<const hx_matmul_plan> cached_transpose_plan(hx_context &ctx, int h, int limbs)
{
    return cached(ctx, 1, h, limbs);
}

std::vector<int64_t> transpose_rotation_steps(int h, int beta)
{
    const int b = baby_steps(h);
    const int64_t n = (int64_t)beta * h * h;
    std::vector<int64_t> out;
    for (int sh = -h + 1; sh < h; sh++)
        for (int64_t x : {(int64_t)beta * (h - 1) * posmod(sh, b), (int64_t)beta * (h - 1) * b * floordiv(sh, b)}) {
            const int64_t r = ((x % n) + n) % n;
            if (r) out.push_back(r);
        }
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
    return out;
}

std::shared_ptr<const hx_matmul_plan> cached_plan(hx_context &ctx, int h, int limbs)
{
    return cached(ctx, 0, h, limbs);
}

namespace {

const uint64_t *mask_pt(const hx_matmul_plan &p, int kind, int idx, double *scale)
{
    auto it = p.index.find({kind, idx});
    HX_CHECK(it != p.index.end(), HX_EINVAL, "missing mask");
    *scale = p.masks[it->second].scale;
    return p.masks[it->second].pt->p;
}

// Alg. 2 over diagonals stride*l, l in [lmin, lmax], split l = b*i + j:
// sum_i Rot( sum_j Mul_pt(Rot(ct, stride*j), mask_l), stride*b*i ); not rescaled.
Cts lintrans(Eval &ev, const hx_keyset &ks, const Cts &ct, int lmin, int lmax, int stride, const hx_matmul_plan &p,
             int kind)
{
    const int b = p.b, beta = p.beta;
    std::map<int, std::vector<std::pair<int, int>>> groups;
    std::vector<int> js;
    for (int l = lmin; l <= lmax; l++) {
        const int i = floordiv(l, b), j = posmod(l, b);
        groups[i].push_back({j, l});
        if (std::find(js.begin(), js.end(), j) == js.end()) js.push_back(j);
    }
    std::sort(js.begin(), js.end());
    std::vector<int64_t> steps;
    for (int j : js) steps.push_back((int64_t)beta * stride * j);
    std::vector<Cts> babies = ev.rotate_hoisted(ct, steps, ks);
    std::map<int, int> jpos;
    for (size_t k = 0; k < js.size(); k++) jpos[js[k]] = (int)k;
    // every inner sum sum_j Mul_pt(baby_j, mask_(i,j)) in one fused launch
    HX_CHECK((int)js.size() <= MAC_MAX_BABY && (int)groups.size() <= MAC_MAX_GROUP, HX_EINVAL,
             "linear transform too wide for the fused inner sums");
    const int N = ev.ctx.N, B = ct.B, limbs = ct.limbs;
    std::unique_ptr<MacArgs> ma(new MacArgs());
    ma->n_baby = (int)js.size();
    ma->n_group = (int)groups.size();
    for (size_t m = 0; m < js.size(); m++) ma->baby[m] = babies[m].d;
    ma->baby_bstride = babies[0].bstride(N);
    ma->baby_cstride = babies[0].cstride(N);
    double sc = 0;
    int g = 0, n_terms = 0;
    for (auto &kv : groups) {
        for (auto &jl : kv.second) {
            ma->mask[g][jpos[jl.first]] = mask_pt(p, kind, jl.second, &sc);
            n_terms++;
        }
        g++;
    }
    BufPtr inner_buf = std::make_shared<DevBuf>((size_t)ma->n_group * B * 2 * limbs * N, ev.s);
    ma->out = inner_buf->p;
    launch_lintrans_mac(ev.lc(), *ma, B, limbs, n_terms);
    ev.ctx.counters[C_MULPT] += (uint64_t)B * n_terms;
    ev.ctx.counters[C_ADD] += (uint64_t)B * (n_terms - ma->n_group);
    std::vector<std::pair<Cts, int64_t>> items;
    g = 0;
    for (auto &kv : groups) {
        Cts inner;
        inner.buf = inner_buf;
        inner.d = inner_buf->p + (size_t)g * B * 2 * limbs * N;
        inner.B = B;
        inner.comps = 2;
        inner.limbs = inner.cap = limbs;
        inner.scale = ct.scale * sc;
        items.push_back({inner, (int64_t)beta * stride * b * kv.first});
        g++;
    }
    // giant steps: one ModDown for the whole sum
    return ev.rotate_sum(items, ks);
}

// t < h: only the terms k < t of Steps 2-3 (the rectangular product, App. D)
Cts matmul_alg3(Eval &ev, const hx_keyset &ks, const hx_matmul_plan &p, const Cts &A, const Cts &B, int t)
{
    hx_context &ctx = ev.ctx;
    const int h = p.h, beta = p.beta;
    // three chains on three streams: the B side (B0 = U^zeta b, its hoisted ModUp and every
    // B^(k) = Rot(B0, h*k)) on side stream sb; the selections A^(k) and their products for even k
    // on the main stream and for odd k on side stream sa, each into its own accumulator.  Every
    // buffer a stream reads from another is released on its own stream only after that stream
    // has waited for the read; everything is joined before the accumulators are summed.
    SideStream &ss = side_stream(ctx, ev.s);
    Eval evb(ctx, ss.s), eva(ctx, ss.s2);
    cudaEvent_t *e = ss.e;  // 0 fork, 1 B0 ready, 2 A0 ready, 3/4 B^(k) ready, 5/6 B^(k) used, 7 joins
    HX_CUDA(cudaEventRecord(e[0], ev.s));
    HX_CUDA(cudaStreamWaitEvent(ss.s, e[0], 0));
    HX_CUDA(cudaStreamWaitEvent(ss.s2, e[0], 0));
    Cts B0 = evb.rescale(lintrans(evb, ks, B, 0, h - 1, h, p, 1));
    BufPtr DB = evb.hoist(B0);  // one ModUp serves every B^(k)
    HX_CUDA(cudaEventRecord(e[1], ss.s));
    Cts A0 = ev.rescale(lintrans(ev, ks, A, -h + 1, h - 1, 1, p, 0));
    BufPtr DA = ev.hoist(A0);
    // Step 2 (App. B multiplexer after hoisting): A^(k) = v_k . Rot(A0, k) + (1 - v_k) . Rot(A0, k-h),
    // all rotations of A0 from one ModUp, the selection before a single ModDown per k.  A^(k)
    // keeps the mask scale (no rescale per k); B^(k) = Rot(B0, h*k) stays at the same level.
    const uint64_t cm = mask_scale_int(ctx);  // the masks' scale as an integer: c of the multiplexer
    Cts acc_odd = ev.alloc(A0.B, 3, A0.limbs);  // the odd-k accumulator, zero, owned by the main stream
    HX_CUDA(cudaMemsetAsync(acc_odd.d, 0, sizeof(uint64_t) * acc_odd.bstride(ctx.N) * acc_odd.B, ev.s));
    HX_CUDA(cudaEventRecord(e[2], ev.s));
    HX_CUDA(cudaStreamWaitEvent(ss.s2, e[2], 0));
    HX_CUDA(cudaStreamWaitEvent(ev.s, e[1], 0));
    // Step 3's products are summed in Montgomery form (each times 2^-64) and scaled back once
    Cts acc = ev.tensor(ev.mul_int(A0, (int64_t)cm, A0.scale * (double)cm), B0, true);
    acc_odd.scale = acc.scale;
    HX_CUDA(cudaEventRecord(e[5], ev.s));
    HX_CUDA(cudaStreamWaitEvent(ss.s, e[5], 0));  // B0's read by the main stream comes before its release
    Cts held[2];  // B^(k) stays alive until its consumer's use is ordered before the release
    for (int k = 1; k < t; k++) {
        const int par = k & 1;
        if (held[par].buf) {  // B^(k-2): released on sb after its consumer (same parity) used it
            HX_CUDA(cudaStreamWaitEvent(ss.s, e[5 + par], 0));
            held[par] = Cts();
        }
        held[par] = evb.rotate_hoisted_one(B0, DB, (int64_t)beta * h * k, ks);
        HX_CUDA(cudaEventRecord(e[3 + par], ss.s));
        Eval &ec = par ? eva : ev;
        double sc;
        const uint64_t *v = mask_pt(p, 2, k, &sc);
        const uint64_t *pm = (p.bound_uid && p.bound_uid == ks.uid) ? p.premasked[k]->p : nullptr;
        Cts Ak = ec.hoisted_mux(A0, DA, (int64_t)beta * k, (int64_t)beta * (k - h), v, sc, cm, ks, pm);
        HX_CUDA(cudaStreamWaitEvent(ec.s, e[3 + par], 0));
        ec.tensor_acc(par ? acc_odd : acc, Ak, held[par], true);
        HX_CUDA(cudaEventRecord(e[5 + par], ec.s));
    }
    for (int par = 0; par < 2; par++)
        if (held[par].buf) {
            HX_CUDA(cudaStreamWaitEvent(ss.s, e[5 + par], 0));
            held[par] = Cts();
        }
    B0 = Cts();  // the B-side buffers go back to the pool on sb, before the join
    DB.reset();
    HX_CUDA(cudaEventRecord(e[7], ss.s));
    HX_CUDA(cudaStreamWaitEvent(ev.s, e[7], 0));
    HX_CUDA(cudaEventRecord(e[7], ss.s2));
    HX_CUDA(cudaStreamWaitEvent(ev.s, e[7], 0));
    ev.add_inplace(acc, acc_odd);
    ev.from_mont(acc);
    // Step 3: one relinearisation, then the two rescales
    return ev.rescale(ev.rescale(ev.relinearize(acc, ks.relin)));
}

Cts matmul_depth2(Eval &ev, const hx_keyset &ks, const hx_matmul_plan &p, const Cts &A, const Cts &B, int t)
{
    const int h = p.h, beta = p.beta;
    Cts A0 = ev.rescale(lintrans(ev, ks, A, -h + 1, h - 1, 1, p, 0));
    std::vector<int64_t> st;
    for (int l = 1; l < h; l++) st.push_back((int64_t)beta * h * l);
    std::vector<Cts> Rb = ev.rotate_hoisted(B, st, ks);
    std::vector<Cts> prefix(h + 1);  // prefix[m] = S_m = sum_{l<m} T_l
    for (int l = 0; l < h; l++) {
        double sc;
        const uint64_t *pt = mask_pt(p, 1, l, &sc);
        Cts T = ev.mul_plain(l == 0 ? B : Rb[l - 1], pt, sc);
        prefix[l + 1] = l == 0 ? T : ev.add(prefix[l], T);
    }
    Rb.clear();
    const Cts &Bfull = prefix[h];
    Cts B0 = ev.rescale(Bfull);
    std::vector<int64_t> ast;
    for (int k = 1; k < t; k++) ast.push_back((int64_t)beta * k);
    for (int k = 1; k < t; k++) ast.push_back((int64_t)beta * (k - h));
    std::vector<Cts> RA = ev.rotate_hoisted(A0, ast, ks);
    Cts acc = ev.tensor(A0, B0, true);  // summed in Montgomery form, scaled back once
    for (int k = 1; k < t; k++) {
        Cts X = ev.rescale(prefix[h - k]);
        Cts Y = ev.rescale(ev.add(Bfull, prefix[h - k], true));
        ev.tensor_acc(acc, RA[k - 1], ev.rotate(X, (int64_t)beta * h * k, ks), true);
        ev.tensor_acc(acc, RA[t - 1 + k - 1], ev.rotate(Y, (int64_t)beta * h * k, ks), true);
    }
    ev.from_mont(acc);
    return ev.rescale(ev.relinearize(acc, ks.relin));
}

} // namespace

Cts transpose_batch(hx_context &ctx, const hx_keyset &ks, const hx_matmul_plan &plan, const Cts &x, cudaStream_t s)
{
    HX_CHECK(plan.kind == 1, HX_EINVAL, "not a transpose plan");
    HX_CHECK(x.comps == 2 && x.limbs == plan.limbs, HX_ELEVEL, "input is not at the plan's level");
    Eval ev(ctx, s);
    return ev.rescale(lintrans(ev, ks, x, -plan.h + 1, plan.h - 1, plan.h - 1, plan, 3));
}

Cts matmul_batch(hx_context &ctx, const hx_keyset &ks, const hx_matmul_plan &plan, const Cts &A, const Cts &B,
                 cudaStream_t s, int t)
{
    t = t ? t : plan.h;
    HX_CHECK(t >= 1 && t <= plan.h, HX_EINVAL, "t must be in [1, h]");
    HX_CHECK(plan.kind == 0, HX_EINVAL, "not a matmul plan");
    HX_CHECK(A.comps == 2 && B.comps == 2 && A.B == B.B, HX_EINVAL, "matmul needs two batches of ciphertexts");
    HX_CHECK(A.limbs == plan.limbs && B.limbs == plan.limbs, HX_ELEVEL, "inputs are not at the plan's level");
    HX_CHECK(A.scale == B.scale, HX_ESCALE, "inputs must share the scale");
    Eval ev(ctx, s);
    return plan.alg3 ? matmul_alg3(ev, ks, plan, A, B, t) : matmul_depth2(ev, ks, plan, A, B, t);
}

void bind_plan_keys(hx_context &ctx, hx_matmul_plan &plan, const hx_keyset &ks, cudaStream_t s)
{
    HX_CHECK(plan.kind == 0 && plan.alg3, HX_EINVAL, "only Alg. 3 product plans select in Step 2");
    HX_CHECK(ks.ctx == &ctx && ks.uid, HX_EINVAL, "keys from another context");
    const int h = plan.h, beta = plan.beta, K = ctx.K, limbs = plan.limbs - 1;  // A0's level
    const int ext = limbs + K, nd = (limbs + ctx.alpha - 1) / ctx.alpha;
    const size_t N = ctx.N;
    Eval ev(ctx, s);
    std::vector<BufPtr> pm(h);
    for (int k = 1; k < h; k++) {
        const uint64_t g1 = galois_for_step((int64_t)beta * k, ctx.log_n);
        const uint64_t g2 = galois_for_step((int64_t)beta * (k - h), ctx.log_n);
        auto it1 = ks.rot.find(g1), it2 = ks.rot.find(g2);
        HX_CHECK(it1 != ks.rot.end() && it2 != ks.rot.end(), HX_EKEY, "missing Galois key for Step 2");
        double sc;
        const uint64_t *v = mask_pt(plan, 2, k, &sc);
        const uint64_t c = mask_scale_int(ctx);  // the integer value of the masks' scale
        Scalars cR;
        for (int t = 0; t < ext; t++) {
            const uint64_t q = ctx.primes[t < limbs ? t : ctx.n_q + (t - limbs)];
            cR.v[t] = (uint64_t)(((u128)(c % q) << 64) % q);
            cR.sh[t] = 0;
        }
        pm[k] = std::make_shared<DevBuf>((size_t)2 * nd * 2 * ext * N, true);
        launch_premask_keys(ev.lc(), pm[k]->p, it1->second.buf->p, it2->second.buf->p, v, cR, ctx.n_all, ctx.n_q, K,
                            limbs, nd);
    }
    HX_CUDA(cudaStreamSynchronize(s));
    plan.premasked = std::move(pm);
    plan.bound_uid = ks.uid;
}

// App. D, Alg. "41": A~ packs h/t vertical copies of a t x h matrix; the k-sum
// cut to t terms, then log2(h/t) rotate-and-add folds by t*h*2^e rows leave
// h/t copies of A.B
Cts rmatmul_batch(hx_context &ctx, const hx_keyset &ks, const hx_matmul_plan &plan, const Cts &At, const Cts &B, int t,
                  cudaStream_t s)
{
    HX_CHECK(t >= 1 && plan.h % t == 0 && (t & (t - 1)) == 0, HX_EINVAL, "t must be a power of two dividing h");
    Cts out = matmul_batch(ctx, ks, plan, At, B, s, t);
    Eval ev(ctx, s);
    for (int e = t; e < plan.h; e *= 2) out = ev.add(out, ev.rotate(out, (int64_t)plan.beta * plan.h * e, ks));
    return out;
}

// ---- Sec. 4: composite sign ------------------------------------------------------

namespace {

int64_t binom(int n, int k)
{
    int64_t r = 1;
    for (int i = 1; i <= k; i++) r = r * (n - k + i) / i;
    return r;
}

// n_j with g_d(m) = sum_j n_j m^(2j+1) / 2^(2d-1), from
// g_d(m) = sum_i 4^-i C(2i,i) m (1-m^2)^i
std::vector<int64_t> g_int_coeffs(int d)
{
    std::vector<int64_t> n(d + 1, 0);
    for (int j = 0; j <= d; j++) {
        int64_t twice = 0;  // 2 * 2^(2d-1) * coefficient
        for (int i = j; i <= d; i++)
            twice += (j % 2 ? -1 : 1) * binom(2 * i, i) * binom(i, j) * ((int64_t)1 << (2 * d - 2 * i));
        n[j] = twice / 2;
    }
    return n;
}

// a * b, relinearised and rescaled in one division by P q_top (reading R21)
Cts square_rs(Eval &ev, const hx_keyset &ks, const Cts &a, const Cts &b)
{
    return ev.relin_rescale(ev.tensor(a, b), ks.relin);
}

// bring ct to `target` limbs at scale target_scale, times c_real: drop to
// target+1 limbs, multiply by round(c_real*target_scale*q_target/scale),
// rescale; the result is declared to have target_scale
Cts level_adjust(Eval &ev, const Cts &ct, int target, double c_real, double target_scale)
{
    HX_CHECK(ct.limbs > target, HX_ELEVEL, "cannot raise the level");
    Cts x = ct.limbs > target + 1 ? ev.drop(ct, target + 1) : ct;
    const uint64_t qt = ev.ctx.primes[target];
    const double c = round_half_away(c_real * target_scale * (double)qt / ct.scale);
    HX_CHECK(std::fabs(c) < 4.6e18, HX_EINVAL, "level-adjust constant too large");
    Cts y = ev.rescale(x, (int64_t)c);
    y.scale = target_scale;
    return y;
}

// one application of g_d, 1 <= d <= 4 (Sec. 4, reading R8): with y = x^2,
// P(y) = n0 + n1 y + n2 y^2 + y^2 (n3 y + n4 y^2) (the terms this d has), then
// x * P with the 2^-(2d-1) folded into x's level adjustment; four ciphertext
// products for d = 3 and 4
Cts eval_g(Eval &ev, const hx_keyset &ks, const Cts &x, int d)
{
    const std::vector<int64_t> n = g_int_coeffs(d);
    Cts y1 = square_rs(ev, ks, x, x), y2, top;
    if (d >= 2) y2 = square_rs(ev, ks, y1, y1);
    if (d >= 3) {
        Cts B = ev.mul_int(level_adjust(ev, y1, y2.limbs, 1.0, y2.scale), n[3]);
        if (d == 4) ev.add_inplace(B, ev.mul_int(y2, n[4]));
        top = square_rs(ev, ks, y2, B);
    }
    const Cts &lead = d >= 3 ? top : (d == 2 ? y2 : y1);
    const int lp = lead.limbs;
    const double sp = lead.scale;
    Cts P = d >= 3 ? top : Cts();
    const Cts *ys[3] = {nullptr, &y1, &y2};
    for (int j = 1; j <= std::min(d, 2); j++) {
        const Cts &yj = *ys[j];
        Cts t = yj.limbs > lp ? level_adjust(ev, yj, lp, (double)n[j], sp) : ev.mul_int(yj, n[j]);
        if (!P.buf)
            P = t;
        else
            ev.add_inplace(P, t);
    }
    P = ev.add_const(P, (double)n[0]);
    Cts xa = level_adjust(ev, x, lp, 1.0 / std::ldexp(1.0, 2 * d - 1), sp);
    return square_rs(ev, ks, xa, P);
}

// levels one application of eval_g consumes: y, y^2 and y^2 B(y) as d needs them, then x * P
int g_depth(int d) { return std::min(d, 3) + 1; }

} // namespace

Cts sign_batch(hx_context &ctx, const hx_keyset &ks, const Cts &x, int d, int k, bool relu, bool allow_refresh,
               const std::vector<uint64_t> &refresh_seeds, cudaStream_t s)
{
    HX_CHECK((int)refresh_seeds.size() == x.B, HX_EINVAL, "one refresh seed per batch entry");
    HX_CHECK(d >= 1 && d <= 4 && k >= 1 && k <= 64, HX_EINVAL, "need 1 <= d <= 4 and 1 <= k <= 64");
    HX_CHECK(x.comps == 2, HX_EINVAL, "sign needs ciphertexts");
    Eval ev(ctx, s);
    const int dg = g_depth(d);
    Cts m = x;
    int refreshes = 0;
    for (int it = 0; it < k; it++) {
        const int need = dg + ((relu && it == k - 1) ? 1 : 0);
        if (m.limbs - 1 < need) {
            HX_CHECK(allow_refresh, HX_ELEVEL, "levels exhausted");
            HX_CHECK(ctx.n_q - 1 >= need, HX_ELEVEL, "chain too short for one composition");
            m = dbootstrap(ctx, ks, m, refresh_seeds, refreshes++, s);
        }
        m = eval_g(ev, ks, m, d);
    }
    if (!relu) return m;
    Cts s1 = ev.add_const(m, 1.0);
    Cts xa = level_adjust(ev, x, m.limbs, 0.5, m.scale);
    return square_rs(ev, ks, xa, s1);
}

// ---- Fig. 5: one dense layer, feedforward then backpropagation ------------------
//
// W holds the weight blocks g-major (entry g*n_out + i packs W_{i,j} for
// j = beta*g .. beta*g + beta - 1 at positions 0..beta-1), X the input
// blocks (entry g packs X_j the same way), G the upstream gradient (entry i
// packs G_i at position 0, zero elsewhere).

namespace {

Cts slice(const hx_context &ctx, const Cts &a, int first, int count)
{
    Cts o = a;
    o.B = count;
    o.d = a.d + (size_t)first * a.bstride(ctx.N);
    return o;
}

// entry g*times + i = a[g]
Cts repeat_each(Eval &ev, const Cts &a, int times)
{
    Cts o = ev.alloc(a.B * times, a.comps, a.limbs);
    o.scale = a.scale;
    const size_t N = ev.ctx.N;
    for (int g = 0; g < a.B; g++)
        launch_copy(ev.lc(), View{o.d + (size_t)g * times * o.bstride(N), o.bstride(N), o.cstride(N)},
                    View{a.d + (size_t)g * a.bstride(N), 0, a.cstride(N)}, times, a.comps, a.limbs);
    return o;
}

// entry g*a.B + i = a[i]
Cts repeat_block(Eval &ev, const Cts &a, int times)
{
    Cts o = ev.alloc(a.B * times, a.comps, a.limbs);
    o.scale = a.scale;
    const size_t N = ev.ctx.N;
    for (int g = 0; g < times; g++)
        launch_copy(ev.lc(), View{o.d + (size_t)g * a.B * o.bstride(N), o.bstride(N), o.cstride(N)}, a.view(ev.ctx.N),
                    a.B, a.comps, a.limbs);
    return o;
}

} // namespace

std::vector<int64_t> dense_rotation_steps(int h, int beta)
{
    std::set<int64_t> st;
    for (int limbs : {3, 4})
        for (int64_t k : plan_rotation_steps(h, beta, limbs)) st.insert(k);
    for (int64_t k : transpose_rotation_steps(h, beta)) st.insert(k);
    const int64_t S = (int64_t)beta * h * h;
    for (int64_t t = 1; t < beta; t *= 2) {
        st.insert(t);
        st.insert(S - t);
    }
    return std::vector<int64_t>(st.begin(), st.end());
}

DenseResult dense_batch(hx_context &ctx, const hx_keyset &ks, const DensePlans &plans, const Cts &W, const Cts &X,
                        const Cts &G, int h, int d, int k, double input_div, uint64_t refresh_seed, cudaStream_t s)
{
    const int n_out = G.B, groups = X.B;
    HX_CHECK(W.comps == 2 && X.comps == 2 && G.comps == 2, HX_EINVAL, "dense layer needs ciphertexts");
    HX_CHECK(n_out >= 1 && groups >= 1 && W.B == n_out * groups, HX_EINVAL, "need n_out*groups weight ciphertexts");
    HX_CHECK(input_div > 0, HX_EINVAL, "input_div must be positive");
    const int64_t S = ctx.N / 2;
    const int beta = (int)(S / ((int64_t)h * h));
    Eval ev(ctx, s);
    // feedforward: every block product in one batched HE-MatMult
    PlanUse pf_held(ctx, s, plans.fwd ? nullptr : cached_plan(ctx, h, W.limbs));
    const hx_matmul_plan *pf = plans.fwd ? plans.fwd : pf_held.p.get();
    HX_CHECK(pf->h == h, HX_EINVAL, "feedforward plan built for another h");
    Cts P = matmul_batch(ctx, ks, *pf, W, repeat_each(ev, X, n_out), s);
    Cts E = ev.copy(slice(ctx, P, 0, n_out));
    for (int g = 1; g < groups; g++) ev.add_inplace(E, slice(ctx, P, g * n_out, n_out));
    for (int t = 1; t < beta; t *= 2) E = ev.add(E, ev.rotate(E, t, ks));  // position 0 sums the beta positions
    // E / input_div at E's scale, one level down (a scale of input_div * Delta would square away from
    // Delta through the composition)
    HX_CHECK(E.limbs >= 2, HX_ELEVEL, "levels exhausted before the activation");
    Cts Ein = level_adjust(ev, E, E.limbs - 1, 1.0 / input_div, E.scale);
    std::vector<uint64_t> seeds(n_out);
    for (int i = 0; i < n_out; i++) seeds[i] = refresh_seed + (uint64_t)i;
    Cts s1 = ev.add_const(sign_batch(ctx, ks, Ein, d, k, false, true, seeds, s), 1.0);  // 2 phi'(E)
    HX_CHECK(G.limbs >= s1.limbs && s1.limbs >= 2, HX_ELEVEL, "levels exhausted before the activation");
    DenseResult r;
    r.E = E;
    r.M = square_rs(ev, ks, ev.drop(E, s1.limbs), s1);  // ReLU(E) = E (1 + s) / 2
    r.M.scale *= 2;
    // backpropagation: L = phi'(E) . G, copied to every packed position
    Cts L = square_rs(ev, ks, s1, ev.drop(G, s1.limbs));
    L.scale *= 2;
    for (int t = 1; t < beta; t *= 2) L = ev.add(L, ev.rotate(L, S - t, ks));
    PlanUse pt_held(ctx, s, plans.transpose ? nullptr : cached_transpose_plan(ctx, h, X.limbs));
    const hx_matmul_plan *pt = plans.transpose ? plans.transpose : pt_held.p.get();
    HX_CHECK(pt->h == h, HX_EINVAL, "transpose plan built for another h");
    Cts XT = transpose_batch(ctx, ks, *pt, X, s);
    HX_CHECK(XT.limbs > L.limbs, HX_ELEVEL, "transposed inputs below the gradient's level");
    Cts XTa = level_adjust(ev, XT, L.limbs, 1.0, L.scale);
    PlanUse pb_held(ctx, s, plans.bwd ? nullptr : cached_plan(ctx, h, L.limbs));
    const hx_matmul_plan *pb = plans.bwd ? plans.bwd : pb_held.p.get();
    HX_CHECK(pb->h == h, HX_EINVAL, "backpropagation plan built for another h");
    r.dW = matmul_batch(ctx, ks, *pb, repeat_block(ev, L, groups), repeat_each(ev, XTa, n_out), s);
    return r;
}

// ---- Alg. 6 Aggregation ----------------------------------------------------------
// out[m] = models[m] - c_real * sum_i grads[i*count + m]: the sum and the integer
// constant of the level adjustment (round(-c_real * scale_model * q_t / scale_grad),
// t = limbs - 1) in one streaming pass over the parties' ciphertexts in place,
// then the rescale by q_t and the addition to the model one level down.

Cts aggregate(hx_context &ctx, const std::vector<const Cts *> &grads, int n_parties, const Cts &models, double c_real,
              cudaStream_t s)
{
    const int count = models.B;
    HX_CHECK(n_parties >= 1 && (int)grads.size() == n_parties * count, HX_EINVAL, "need n_parties*count gradients");
    const Cts &g0 = *grads[0];
    HX_CHECK(models.comps == 2 && models.limbs >= 2, HX_ELEVEL, "the update needs a level to rescale");
    for (const Cts *g : grads) {
        HX_CHECK(g->B == 1 && g->comps == 2 && g->limbs == models.limbs, HX_ESCALE,
                 "gradients must be ciphertexts at the models' level");
        HX_CHECK(g->scale == g0.scale, HX_ESCALE, "gradients must share the scale");
    }
    Eval ev(ctx, s);
    const int L = models.limbs, target = L - 1;
    const double cr = round_half_away(-c_real * models.scale * (double)ctx.primes[target] / g0.scale);
    HX_CHECK(std::fabs(cr) < 4.6e18, HX_EINVAL, "update constant too large");
    std::vector<AggSrc> tab(grads.size());
    for (size_t i = 0; i < grads.size(); i++) tab[i] = AggSrc{grads[i]->d, (uint64_t)grads[i]->cstride(ctx.N)};
    DevBuf tab_dev((tab.size() * sizeof(AggSrc) + 7) / 8, s);
    HX_CUDA(cudaMemcpyAsync(tab_dev.p, tab.data(), tab.size() * sizeof(AggSrc), cudaMemcpyHostToDevice, s));
    Cts sum = ev.alloc(count, 2, L);
    sum.scale = g0.scale;
    launch_aggregate(ev.lc(), sum.view(ctx.N), reinterpret_cast<const AggSrc *>(tab_dev.p), n_parties, count, 2, L,
                     scalars_for(ctx, L, (int64_t)cr));
    Cts upd = ev.rescale(sum);
    upd.scale = models.scale;
    return ev.add(ev.drop(models, target), upd);
}

} // namespace hx
