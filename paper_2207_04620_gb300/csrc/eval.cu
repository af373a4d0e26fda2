// Batched homomorphic evaluation (Fig. 1 items 7-12).  Every operation acts on
// a batch of B ciphertexts with one launch per kernel; hybrid key switching is
// ModUp (iNTT, fast basis conversion per digit, NTT) -> key inner product ->
// ModDown (iNTT of the special limbs, conversion P -> Q_l, NTT, subtract and
// multiply by P^-1).
#include <cmath>

#include "runtime.h"

namespace hx {

Cts Eval::alloc(int B, int comps, int limbs)
{
    Cts c;
    c.B = B;
    c.comps = comps;
    c.limbs = limbs;
    c.cap = limbs;
    c.buf = std::make_shared<DevBuf>((size_t)B * comps * limbs * ctx.N, s);
    c.d = c.buf->p;
    return c;
}

void Eval::check_same(const Cts &a, const Cts &b)
{
    HX_CHECK(a.B == b.B, HX_EINVAL, "batch sizes differ");
    HX_CHECK(a.limbs == b.limbs, HX_ESCALE, "level mismatch");
    HX_CHECK(std::fabs(a.scale / b.scale - 1.0) <= std::ldexp(1.0, -20), HX_ESCALE, "scale mismatch");
}

Cts Eval::add(const Cts &a, const Cts &b, bool sub)
{
    check_same(a, b);
    HX_CHECK(a.comps == b.comps, HX_EINVAL, "component count mismatch");
    Cts o = alloc(a.B, a.comps, a.limbs);
    o.scale = a.scale;
    launch_add(lc(), o.view(ctx.N), a.view(ctx.N), b.view(ctx.N), a.B, a.comps, a.limbs, sub);
    ctx.counters[C_ADD] += a.B;
    return o;
}

void Eval::add_inplace(Cts &a, const Cts &b)
{
    check_same(a, b);
    launch_add(lc(), a.view(ctx.N), a.view(ctx.N), b.view(ctx.N), a.B, a.comps, a.limbs, false);
    ctx.counters[C_ADD] += a.B;
}

Cts Eval::mul_plain(const Cts &a, const uint64_t *pt, double pt_scale)
{
    HX_CHECK(a.comps == 2, HX_EINVAL, "Mul_pt needs a 2-component ciphertext");
    Cts o = alloc(a.B, 2, a.limbs);
    o.scale = a.scale * pt_scale;
    launch_mul_plain(lc(), o.view(ctx.N), a.view(ctx.N), pt, a.B, a.limbs);
    ctx.counters[C_MULPT] += a.B;
    return o;
}

Scalars scalars_for(const hx_context &ctx, int limbs, int64_t c)
{
    Scalars sc;
    for (int l = 0; l < limbs; l++) {
        const uint64_t q = ctx.primes[l];
        uint64_t v = c >= 0 ? (uint64_t)c % q : (q - ((uint64_t)(-(c + 1)) + 1) % q) % q;
        sc.v[l] = v;
        sc.sh[l] = shoup_companion(v, q);
    }
    return sc;
}

Cts Eval::mul_int(const Cts &a, int64_t c, double new_scale)
{
    Cts o = alloc(a.B, a.comps, a.limbs);
    o.scale = new_scale > 0 ? new_scale : a.scale;
    launch_mul_scalar(lc(), o.view(ctx.N), a.view(ctx.N), scalars_for(ctx, a.limbs, c), a.B, a.comps, a.limbs);
    return o;
}

Cts Eval::add_const(const Cts &a, double value)
{
    const double r = round_half_away(value * a.scale);
    HX_CHECK(std::fabs(r) < 9.2e18, HX_EINVAL, "constant too large");
    Cts o = alloc(a.B, 2, a.limbs);
    o.scale = a.scale;
    launch_add_scalar_c0(lc(), o.view(ctx.N), a.view(ctx.N), scalars_for(ctx, a.limbs, (int64_t)r), a.B, a.limbs);
    return o;
}

Cts Eval::tensor(const Cts &a, const Cts &b, bool mont)
{
    HX_CHECK(a.B == b.B && a.limbs == b.limbs && a.comps == 2 && b.comps == 2, HX_ESCALE, "tensor operands differ");
    Cts o = alloc(a.B, 3, a.limbs);
    o.scale = a.scale * b.scale;
    launch_tensor(lc(), o.view(ctx.N), a.view(ctx.N), b.view(ctx.N), a.B, a.limbs, false, mont);
    ctx.counters[C_MULCT] += a.B;
    return o;
}

void Eval::from_mont(Cts &a)
{
    Scalars sc;
    for (int l = 0; l < a.limbs; l++) {
        sc.v[l] = ctx.h_primes[l].r_mod;  // 2^64 mod q_l
        sc.sh[l] = ctx.h_primes[l].r_mod_sh;
    }
    launch_mul_scalar(lc(), a.view(ctx.N), a.view(ctx.N), sc, a.B, a.comps, a.limbs);
}

void Eval::tensor_acc(Cts &acc, const Cts &a, const Cts &b, bool mont)
{
    HX_CHECK(a.B == b.B && a.limbs == b.limbs && acc.limbs == a.limbs && acc.comps == 3, HX_ESCALE,
             "tensor operands differ");
    HX_CHECK(std::fabs(acc.scale / (a.scale * b.scale) - 1.0) <= std::ldexp(1.0, -20), HX_ESCALE, "scale mismatch");
    launch_tensor(lc(), acc.view(ctx.N), a.view(ctx.N), b.view(ctx.N), a.B, a.limbs, true, mont);
    ctx.counters[C_MULCT] += a.B;
    ctx.counters[C_ADD] += a.B;
}

Cts Eval::drop(const Cts &a, int limbs)
{
    HX_CHECK(limbs >= 1 && limbs <= a.limbs, HX_EINVAL, "bad level drop");
    Cts o = a;
    o.limbs = limbs;
    return o;
}

Cts Eval::copy(const Cts &a)
{
    Cts o = alloc(a.B, a.comps, a.limbs);
    o.scale = a.scale;
    launch_copy(lc(), o.view(ctx.N), a.view(ctx.N), a.B, a.comps, a.limbs);
    return o;
}

void Eval::ntt_inplace(uint64_t *p, size_t gstride, int groups, const std::vector<int> &off,
                       const std::vector<int> &prime, bool inverse)
{
    ntt_oop(p, gstride, p, gstride, groups, off, off, prime, inverse);
}

void Eval::ntt_oop(const uint64_t *src, size_t sgs, uint64_t *dst, size_t dgs, int groups,
                   const std::vector<int> &src_off, const std::vector<int> &dst_off, const std::vector<int> &prime,
                   bool inverse)
{
    if (prime.empty() || groups == 0) return;
    NttRows *r = new NttRows;
    std::unique_ptr<NttRows> guard(r);
    r->src = src;
    r->dst = dst;
    r->src_gs = sgs;
    r->dst_gs = dgs;
    r->n_groups = groups;
    HX_CHECK(prime.size() <= (size_t)MAX_NTT_ROWS, HX_EINVAL, "too many NTT rows");
    r->n_rows = (int)prime.size();
    for (size_t i = 0; i < prime.size(); i++) {
        r->src_off[i] = (int16_t)src_off[i];
        r->dst_off[i] = (int16_t)dst_off[i];
        r->prime[i] = (int16_t)prime[i];
    }
    launch_ntt(lc(), *r, inverse);
}

static std::vector<int> iota_vec(int a, int n)
{
    std::vector<int> v(n);
    for (int i = 0; i < n; i++) v[i] = a + i;
    return v;
}

BufPtr Eval::modup(const View &d, int B, int limbs)
{
    const int N = ctx.N, K = ctx.K, A = ctx.alpha, ext = limbs + K, nd = (limbs + A - 1) / A;
    DevBuf coef((size_t)B * limbs * N, s);
    ntt_oop(d.p, d.bstride, coef.p, (size_t)limbs * N, B, iota_vec(0, limbs), iota_vec(0, limbs), iota_vec(0, limbs),
            true);
    BufPtr D = std::make_shared<DevBuf>((size_t)B * nd * ext * N, s);
    launch_basis_convert(lc(), ctx.t.modup + (size_t)limbs * ctx.dnum, A, View{D->p, (size_t)nd * ext * N, 0},
                         View{coef.p, (size_t)limbs * N, 0}, B, nd, (size_t)ext * N, 0, 8.0 * N * B * nd * ext);
    std::vector<int> off, pr;
    for (int j = 0; j < nd; j++) {
        const int lo = j * A, hi = std::min((j + 1) * A, limbs);
        for (int r = 0; r < ext; r++) {
            if (r >= lo && r < hi) continue;
            off.push_back(j * ext + r);
            pr.push_back(r < limbs ? r : ctx.n_q + (r - limbs));
        }
    }
    ntt_inplace(D->p, (size_t)nd * ext * N, B, off, pr, false);
    ctx.counters[C_MODUP] += B;
    return D;
}

Cts Eval::ks_finish(const BufPtr &D, const View &dnt, int B, int limbs, const SwitchKey &key, uint64_t g,
                    const View &add, int add_mask, uint64_t add_g)
{
    const int N = ctx.N, K = ctx.K, ext = limbs + K, nd = (limbs + ctx.alpha - 1) / ctx.alpha;
    DevBuf acc((size_t)B * 2 * ext * N, s);
    View accv{acc.p, (size_t)2 * ext * N, (size_t)ext * N};
    launch_key_ip(lc(), accv, D->p, dnt.p, dnt.bstride, key.buf->p, ctx.n_all, ctx.n_q, K, ctx.alpha, limbs, nd, g, B);
    ctx.counters[C_KS] += B;
    return moddown_add(accv, B, limbs, add, add_mask, add_g);
}

Cts Eval::moddown_add(const View &accv, int B, int limbs, const View &add, int add_mask, uint64_t add_g)
{
    const int N = ctx.N, K = ctx.K, ext = limbs + K;
    ntt_inplace(accv.p, (size_t)ext * N, 2 * B, iota_vec(limbs, K), iota_vec(ctx.n_q, K), true);
    DevBuf conv((size_t)B * 2 * limbs * N, s);
    launch_basis_convert(lc(), reinterpret_cast<const ConvTable *>(ctx.t.moddown + limbs), ctx.K,
                         View{conv.p, (size_t)limbs * N, 0}, View{accv.p, (size_t)ext * N, 0}, 2 * B, 1, 0, 0,
                         8.0 * N * 2 * B * (K + limbs));
    ntt_inplace(conv.p, (size_t)limbs * N, 2 * B, iota_vec(0, limbs), iota_vec(0, limbs), false);
    Cts o = alloc(B, 2, limbs);
    launch_moddown_final(lc(), o.view(N), accv, View{conv.p, (size_t)2 * limbs * N, (size_t)limbs * N},
                         ctx.t.moddown + limbs, B, limbs, add, add_mask, add_g);
    return o;
}

Cts Eval::rotate_sum(const std::vector<std::pair<Cts, int64_t>> &items, const hx_keyset &keys)
{
    HX_CHECK(!items.empty(), HX_EINVAL, "empty rotation sum");
    const Cts &f = items[0].first;
    const int N = ctx.N, K = ctx.K, limbs = f.limbs, B = f.B, ext = limbs + K, nd = (limbs + ctx.alpha - 1) / ctx.alpha;
    Cts base = alloc(B, 2, limbs);
    base.scale = f.scale;
    HX_CUDA(cudaMemsetAsync(base.d, 0, sizeof(uint64_t) * base.bstride(N) * B, s));
    DevBuf acc((size_t)B * 2 * ext * N, s);
    View accv{acc.p, (size_t)2 * ext * N, (size_t)ext * N};
    bool any = false;
    for (auto &it : items) {
        const Cts &ct = it.first;
        check_same(ct, f);
        const uint64_t g = galois_for_step(it.second, ctx.log_n);
        if (g == 1) {
            add_inplace(base, ct);
            continue;
        }
        const SwitchKey &key = rot_key(keys, g);
        Cts t = alloc(B, 1, limbs);
        View c1{ct.d + ct.cstride(N), ct.bstride(N), ct.cstride(N)};
        launch_automorphism(lc(), t.view(N), c1, g, B, 1, limbs);
        BufPtr D = modup(t.view(N), B, limbs);
        launch_key_ip(lc(), accv, D->p, t.d, t.bstride(N), key.buf->p, ctx.n_all, ctx.n_q, K, ctx.alpha, limbs, nd, 1, B,
                      any);
        launch_automorphism(lc(), base.view(N), ct.view(N), g, B, 1, limbs, true);  // base.c0 += sigma_g(c0)
        any = true;
        ctx.counters[C_ROT] += B;
        ctx.counters[C_KS] += B;
        ctx.counters[C_ADD] += B;
    }
    if (!any) return base;
    Cts o = moddown_add(accv, B, limbs, base.view(N), 3, 1);
    o.scale = f.scale;
    return o;
}

Cts Eval::relinearize(const Cts &d, const SwitchKey &rk)
{
    HX_CHECK(d.comps == 3, HX_EINVAL, "relinearisation needs 3 components");
    HX_CHECK(rk.buf, HX_EKEY, "no relinearisation key");
    const size_t N = ctx.N;
    View d2{d.d + 2 * d.cstride(N), d.bstride(N), d.cstride(N)};
    BufPtr D = modup(d2, d.B, d.limbs);
    Cts o = ks_finish(D, d2, d.B, d.limbs, rk, 1, d.view(N), 3, 1);
    o.scale = d.scale;
    return o;
}

// Relinearisation and RS in one division by P q_top: the key inner product of d_2 over
// Q_l and P; y_c = acc_c + P d_c (only q_top's row is formed in memory, the lower rows in
// the epilogue); the remainder [y_c + h]_{P q_top} - h converted from q_top and the special
// primes to Q_{l-1}; out_c = (y_c - remainder) (P q_top)^-1.
Cts Eval::relin_rescale(const Cts &d, const SwitchKey &rk)
{
    HX_CHECK(d.comps == 3, HX_EINVAL, "relinearisation needs 3 components");
    HX_CHECK(rk.buf, HX_EKEY, "no relinearisation key");
    HX_CHECK(d.limbs >= 2, HX_ELEVEL, "no level left to rescale");
    const int N = ctx.N, K = ctx.K, L = d.limbs, B = d.B, ext = L + K, nd = (L + ctx.alpha - 1) / ctx.alpha;
    View d2{d.d + 2 * d.cstride(N), d.bstride(N), d.cstride(N)};
    BufPtr D = modup(d2, B, L);
    DevBuf acc((size_t)B * 2 * ext * N, s);
    View accv{acc.p, (size_t)2 * ext * N, (size_t)ext * N};
    launch_key_ip(lc(), accv, D->p, d2.p, d2.bstride, rk.buf->p, ctx.n_all, ctx.n_q, K, ctx.alpha, L, nd, 1, B);
    ctx.counters[C_KS] += B;
    D.reset();
    const RelinRescaleTable *tab = ctx.t.relin_rs + L;
    launch_relin_rs_top(lc(), accv, d.view(N), tab, B, L);
    std::vector<int> rows = iota_vec(L - 1, K + 1), primes(K + 1);
    primes[0] = L - 1;
    for (int k = 0; k < K; k++) primes[k + 1] = ctx.n_q + k;
    ntt_inplace(acc.p, (size_t)ext * N, 2 * B, rows, primes, true);
    DevBuf conv((size_t)B * 2 * (L - 1) * N, s);
    launch_basis_convert(lc(), reinterpret_cast<const ConvTable *>(tab), K + 1, View{conv.p, (size_t)(L - 1) * N, 0},
                         View{acc.p, (size_t)ext * N, 0}, 2 * B, 1, 0, 0, 8.0 * N * 2 * B * (K + L));
    ntt_inplace(conv.p, (size_t)(L - 1) * N, 2 * B, iota_vec(0, L - 1), iota_vec(0, L - 1), false);
    Cts o = alloc(B, 2, L - 1);
    launch_relin_rs_final(lc(), o.view(N), accv, d.view(N),
                          View{conv.p, (size_t)2 * (L - 1) * N, (size_t)(L - 1) * N}, tab, B, L);
    o.scale = d.scale / (double)ctx.primes[L - 1];
    ctx.counters[C_RESCALE] += B;
    return o;
}

const SwitchKey &Eval::rot_key(const hx_keyset &ks, uint64_t g)
{
    auto it = ks.rot.find(g);
    HX_CHECK(it != ks.rot.end(), HX_EKEY, "missing Galois key for element " + std::to_string(g));
    return it->second;
}

Cts Eval::rotate(const Cts &a, int64_t k, const hx_keyset &ks)
{
    const uint64_t g = galois_for_step(k, ctx.log_n);
    if (g == 1) return copy(a);
    const SwitchKey &key = rot_key(ks, g);
    const size_t N = ctx.N;
    Cts t = alloc(a.B, 1, a.limbs);
    View c1{a.d + a.cstride(N), a.bstride(N), a.cstride(N)};
    launch_automorphism(lc(), t.view(N), c1, g, a.B, 1, a.limbs);
    BufPtr D = modup(t.view(N), a.B, a.limbs);
    Cts o = ks_finish(D, t.view(N), a.B, a.limbs, key, 1, a.view(N), 1, g);
    o.scale = a.scale;
    ctx.counters[C_ROT] += a.B;
    return o;
}

BufPtr Eval::hoist(const Cts &a)
{
    const size_t N = ctx.N;
    View c1{a.d + a.cstride(N), a.bstride(N), a.cstride(N)};
    return modup(c1, a.B, a.limbs);
}

Cts Eval::rotate_hoisted_one(const Cts &a, const BufPtr &D, int64_t k, const hx_keyset &keys)
{
    const size_t N = ctx.N;
    const uint64_t g = galois_for_step(k, ctx.log_n);
    if (g == 1) return copy(a);
    const SwitchKey &key = rot_key(keys, g);
    View c1{a.d + a.cstride(N), a.bstride(N), a.cstride(N)};
    Cts o = ks_finish(D, c1, a.B, a.limbs, key, g, a.view(N), 1, g);
    o.scale = a.scale;
    ctx.counters[C_ROT] += a.B;
    ctx.counters[C_ROT_HOIST] += a.B;
    return o;
}

Cts Eval::hoisted_mux(const Cts &a, const BufPtr &D, int64_t k1, int64_t k2, const uint64_t *v_ext, double v_scale,
                      uint64_t c, const hx_keyset &keys, const uint64_t *premasked)
{
    const int N = ctx.N, K = ctx.K, limbs = a.limbs, ext = limbs + K, nd = (limbs + ctx.alpha - 1) / ctx.alpha, B = a.B;
    const uint64_t g1 = galois_for_step(k1, ctx.log_n), g2 = galois_for_step(k2, ctx.log_n);
    HX_CHECK(g1 != 1 && g2 != 1, HX_EINVAL, "selection needs two proper rotations");
    const SwitchKey &key1 = rot_key(keys, g1), &key2 = rot_key(keys, g2);
    Scalars cs;
    for (int t = 0; t < ext; t++) {
        const uint64_t q = ctx.primes[t < limbs ? t : ctx.n_q + (t - limbs)];
        cs.v[t] = c % q;
        cs.sh[t] = shoup_companion(cs.v[t], q);
    }
    const View c1{a.d + a.cstride(N), a.bstride(N), a.cstride(N)};
    DevBuf z((size_t)B * 2 * ext * N, s);
    View zv{z.p, (size_t)2 * ext * N, (size_t)ext * N};
    if (premasked)
        launch_key_ip_mux_pm(lc(), zv, D->p, c1.p, c1.bstride, premasked, ctx.n_q, K, ctx.alpha, limbs, nd, g1, g2, B);
    else
        launch_key_ip_mux(lc(), zv, D->p, c1.p, c1.bstride, key1.buf->p, key2.buf->p, v_ext, cs, ctx.n_all, ctx.n_q, K,
                          ctx.alpha, limbs, nd, g1, g2, B);
    ntt_inplace(z.p, (size_t)ext * N, 2 * B, iota_vec(limbs, K), iota_vec(ctx.n_q, K), true);
    DevBuf conv((size_t)B * 2 * limbs * N, s);
    launch_basis_convert(lc(), reinterpret_cast<const ConvTable *>(ctx.t.moddown + limbs), ctx.K,
                         View{conv.p, (size_t)limbs * N, 0}, View{z.p, (size_t)ext * N, 0}, 2 * B, 1, 0, 0,
                         8.0 * N * 2 * B * (ctx.K + limbs));
    ntt_inplace(conv.p, (size_t)limbs * N, 2 * B, iota_vec(0, limbs), iota_vec(0, limbs), false);
    Cts o = alloc(B, 2, limbs);
    launch_moddown_final_mux(lc(), o.view(N), zv, View{conv.p, (size_t)2 * limbs * N, (size_t)limbs * N},
                             ctx.t.moddown + limbs, B, limbs, a.view(N), v_ext + (size_t)K * N, cs, g1, g2);
    o.scale = a.scale * v_scale;
    ctx.counters[C_ROT] += 2 * B;
    ctx.counters[C_ROT_HOIST] += 2 * B;
    ctx.counters[C_MULPT] += B;
    ctx.counters[C_ADD] += B;
    ctx.counters[C_KS] += B;
    return o;
}

std::vector<Cts> Eval::rotate_hoisted(const Cts &a, const std::vector<int64_t> &ks, const hx_keyset &keys)
{
    BufPtr D;
    std::vector<Cts> out;
    for (int64_t k : ks) {
        if (!D && galois_for_step(k, ctx.log_n) != 1) D = hoist(a);
        out.push_back(rotate_hoisted_one(a, D, k, keys));
    }
    return out;
}

Cts Eval::rescale(const Cts &a, int64_t c)
{
    HX_CHECK(a.limbs >= 2, HX_ELEVEL, "no level left to rescale");
    const int N = ctx.N, top = a.limbs - 1, comps = a.comps, B = a.B;
    DevBuf xtop((size_t)B * comps * N, s);
    ntt_oop(a.d, a.cstride(N), xtop.p, (size_t)N, B * comps, {top}, {0}, {top}, true);
    DevBuf r((size_t)B * comps * top * N, s);
    View rv{r.p, (size_t)comps * top * N, (size_t)top * N};
    const RescaleTable *tab = ctx.t.rescale + a.limbs;
    // rescale(c * a) for an integer c: a's residues times c in the two elementwise passes
    // (the top limb after its inverse NTT), the same values as multiplying first
    const Scalars sc = c != 1 ? scalars_for(ctx, a.limbs, c) : Scalars{};
    const Scalars *scp = c != 1 ? &sc : nullptr;
    launch_rescale_prep(lc(), rv, View{xtop.p, (size_t)comps * N, (size_t)N}, tab, B, comps, top, scp);
    ntt_inplace(r.p, (size_t)top * N, B * comps, iota_vec(0, top), iota_vec(0, top), false);
    Cts o = alloc(B, comps, top);
    launch_rescale_final(lc(), o.view(N), a.view(N), rv, tab, B, comps, top, scp);
    o.scale = a.scale / (double)ctx.primes[top];
    ctx.counters[C_RESCALE] += B;
    return o;
}

void plaintext_from_device(hx_context &ctx, cudaStream_t s, const int64_t *dcoeffs, int limbs, bool extended,
                           uint64_t *dst)
{
    Eval ev(ctx, s);
    if (!extended) {
        launch_signed_to_rows(ev.lc(), dst, dcoeffs, limbs, 1, ctx.N, ctx.d_prime_ids);
        ev.ntt_inplace(dst, 0, 1, iota_vec(0, limbs), iota_vec(0, limbs), false);
        launch_to_mont(ev.lc(), dst, limbs, ctx.d_prime_ids);
        return;
    }
    const int ext = limbs + ctx.K;
    std::vector<int> pr(ext);
    for (int t = 0; t < ext; t++) pr[t] = t < limbs ? t : ctx.n_q + (t - limbs);
    DevBuf ids((ext + 1) / 2, s);
    HX_CUDA(cudaMemcpyAsync(ids.p, pr.data(), sizeof(int) * ext, cudaMemcpyHostToDevice, s));
    const int *idp = reinterpret_cast<const int *>(ids.p);
    launch_signed_to_rows(ev.lc(), dst, dcoeffs, ext, 1, ctx.N, idp);
    ev.ntt_inplace(dst, 0, 1, iota_vec(0, ext), pr, false);
    launch_to_mont(ev.lc(), dst, ext, idp);
    HX_CUDA(cudaStreamSynchronize(s));  // the prime-index staging buffer is released at return
}

void upload_plaintext(hx_context &ctx, cudaStream_t s, const int64_t *coeffs, int limbs, uint64_t *dst)
{
    Eval ev(ctx, s);
    DevBuf tmp((size_t)ctx.N, s);
    HX_CUDA(cudaMemcpyAsync(tmp.p, coeffs, sizeof(int64_t) * ctx.N, cudaMemcpyHostToDevice, s));
    launch_signed_to_rows(ev.lc(), dst, reinterpret_cast<const int64_t *>(tmp.p), limbs, 1, ctx.N, ctx.d_prime_ids);
    ev.ntt_inplace(dst, 0, 1, iota_vec(0, limbs), iota_vec(0, limbs), false);
    launch_to_mont(ev.lc(), dst, limbs, ctx.d_prime_ids);
    HX_CUDA(cudaStreamSynchronize(s));  // the pageable source must outlive the copy
}

void upload_plaintext_ext(hx_context &ctx, cudaStream_t s, const int64_t *coeffs, int limbs, uint64_t *dst)
{
    Eval ev(ctx, s);
    const int ext = limbs + ctx.K;
    std::vector<int> pr(ext);  // the special primes' rows first, then q_0 .. q_{limbs-1}
    for (int t = 0; t < ext; t++) pr[t] = t < ctx.K ? ctx.n_q + t : t - ctx.K;
    DevBuf tmp((size_t)ctx.N, s);
    DevBuf ids((ext + 1) / 2, s);
    HX_CUDA(cudaMemcpyAsync(tmp.p, coeffs, sizeof(int64_t) * ctx.N, cudaMemcpyHostToDevice, s));
    HX_CUDA(cudaMemcpyAsync(ids.p, pr.data(), sizeof(int) * ext, cudaMemcpyHostToDevice, s));
    const int *idp = reinterpret_cast<const int *>(ids.p);
    launch_signed_to_rows(ev.lc(), dst, reinterpret_cast<const int64_t *>(tmp.p), ext, 1, ctx.N, idp);
    ev.ntt_inplace(dst, 0, 1, iota_vec(0, ext), pr, false);
    launch_to_mont(ev.lc(), dst, ext, idp);
    HX_CUDA(cudaStreamSynchronize(s));
}

} // namespace hx
