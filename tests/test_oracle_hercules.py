"""Pins of the oracle's Sec. 3 / Sec. 4 layer against the values the paper
prints (tests/golden/), against brute-force permutation matrices, against
FP64 A@B and against exact rational arithmetic."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import ckks as C
from oracle import hercules as H

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def rows_to_matrix(rows):
    n = len(rows)
    U = np.zeros((n, n), dtype=np.int64)
    for r, c in enumerate(rows):
        U[r, c] = 1
    return U


def test_fig2_permutation_matrices_and_vectors():
    g = gold("fig2_h3.json")
    h = g["h"]
    assert np.array_equal(H.perm_matrix(h, "mu"), rows_to_matrix(g["U_mu_rows"]))
    assert np.array_equal(H.perm_matrix(h, "zeta"), rows_to_matrix(g["U_zeta_rows"]))
    assert np.array_equal(H.perm_matrix(h, "V", 1), rows_to_matrix(g["V1_rows"]))
    assert np.array_equal(H.perm_matrix(h, "V", 2), rows_to_matrix(g["V2_rows"]))
    assert np.array_equal(H.perm_matrix(h, "P", 1), rows_to_matrix(g["P1_rows"]))
    assert np.array_equal(H.perm_matrix(h, "P", 2), rows_to_matrix(g["P2_rows"]))
    a = np.arange(9)
    assert list(H.perm_matrix(h, "mu") @ a) == g["U_mu_a"]
    assert list(H.perm_matrix(h, "zeta") @ a) == g["U_zeta_b"]
    for k, v in g["u_mu"].items():
        assert list(H.diag_mu(h, int(k))) == v
    for k, v in g["u_zeta"].items():
        assert list(H.diag_zeta(h, int(k) // h)) == v
    assert list(H.diag_v(h, 1)) == g["v"]["1"] and list(H.diag_v_neg(h, 1)) == g["v"]["-2"]
    assert list(H.diag_v(h, 2)) == g["v"]["2"] and list(H.diag_v_neg(h, 2)) == g["v"]["-1"]
    for k in (1, 2):
        assert list(H.diagonal(H.perm_matrix(h, "P", k), h * k)) == g["p"][str(h * k)]
    A = np.arange(9).reshape(3, 3)
    assert H.phi(H.mu(A), 1).tolist() == g["phi1_mu_A"]
    assert H.phi(H.mu(A), 2).tolist() == g["phi2_mu_A"]
    assert H.pi_(H.zeta(A), 1).tolist() == g["pi1_zeta_B"]
    assert H.pi_(H.zeta(A), 2).tolist() == g["pi2_zeta_B"]


@pytest.mark.parametrize("h", [2, 3, 4, 5, 8, 16])
def test_diagonal_formulas_match_permutation_matrices(h):
    Umu, Uz, UT = H.perm_matrix(h, "mu"), H.perm_matrix(h, "zeta"), H.perm_matrix(h, "T")
    n = h * h
    nz = [k for k in range(n) if H.diagonal(Umu, k).any()]
    assert len(nz) == 2 * h - 1
    for k in range(-h + 1, h):
        assert np.array_equal(H.diagonal(Umu, k), H.diag_mu(h, k))
    assert sorted(k for k in range(n) if H.diagonal(Uz, k).any()) == [h * k for k in range(h)]
    for k in range(h):
        assert np.array_equal(H.diagonal(Uz, h * k), H.diag_zeta(h, k))
    for k in range(1, h):
        V = H.perm_matrix(h, "V", k)
        assert sorted(j for j in range(n) if H.diagonal(V, j).any()) == sorted({k, (k - h) % n})
        assert np.array_equal(H.diagonal(V, k), H.diag_v(h, k))
        assert np.array_equal(H.diagonal(V, k - h), H.diag_v_neg(h, k))
        P = H.perm_matrix(h, "P", k)
        assert [j for j in range(n) if H.diagonal(P, j).any()] == [h * k]
    for s in range(-h + 1, h):
        assert np.array_equal(H.diagonal(UT, (h - 1) * s), H.diag_transpose(h, s))
    # Eq. (1): U m = sum_k u_k . R(m, k)
    m = np.random.default_rng(h).normal(size=n)
    assert np.allclose(sum(H.diagonal(Umu, k) * H.R(m, k) for k in range(n)), Umu @ m)


@pytest.mark.parametrize("h", [2, 3, 4, 7, 16])
def test_eq2_product_identity(h):
    rng = np.random.default_rng(h)
    A, B = rng.normal(size=(h, h)), rng.normal(size=(h, h))
    S = sum(H.phi(H.mu(A), k) * H.pi_(H.zeta(B), k) for k in range(h))
    assert np.allclose(S, A @ B)


@pytest.mark.parametrize("h,beta", [(3, 1), (4, 1), (4, 4), (8, 2), (16, 2), (32, 1)])
@pytest.mark.parametrize("variant", ["alg3", "depth2"])
def test_slot_schedules_give_matrix_product(h, beta, variant):
    rng = np.random.default_rng(h * beta)
    As = [rng.uniform(-1, 1, (h, h)) for _ in range(beta)]
    Bs = [rng.uniform(-1, 1, (h, h)) for _ in range(beta)]
    out = H.unpack(H.slot_matmul(H.pack(As, h, beta), H.pack(Bs, h, beta), h, beta, variant), h, beta)
    for o, A, B in zip(out, As, Bs):
        assert np.abs(o - A @ B).max() < 1e-12


@pytest.mark.parametrize("h", [3, 4, 8])
def test_slot_transpose(h):
    a = np.random.default_rng(h).normal(size=h * h)
    assert np.allclose(H.slot_transpose(a, h), a.reshape(h, h).T.reshape(-1))


class _DryCt:
    def __init__(self, limbs, scale):
        self.limbs, self.scale = limbs, scale


class DryEvaluator(C.Evaluator):
    """Counts the schedule's operations without computing them."""

    def __init__(self, ctx):
        self.ctx, self.counts = ctx, {}


    def add(self, a, b):
        self._count("Add")
        return a

    sub = add

    def mul_plain(self, ct, pt, sc):
        self._count("Mul_pt")
        return _DryCt(ct.limbs, ct.scale * sc)

    def mul_int(self, ct, c, new_scale=None):
        return _DryCt(ct.limbs, ct.scale if new_scale is None else new_scale)

    def tensor(self, a, b):
        self._count("Mul_ct")
        return _DryCt(a.limbs, a.scale * b.scale)

    def relinearize(self, d):
        return d

    def rescale(self, ct):
        self._count("Rescale")
        return _DryCt(ct.limbs - 1, ct.scale / self.ctx.q[ct.limbs - 1])

    def drop(self, ct, limbs):
        return _DryCt(limbs, ct.scale)

    def rotate(self, ct, k):
        if C.galois_element(k, self.ctx.N) != 1:
            self._count("Rot")
        return ct

    def rotate_hoisted(self, ct, steps):
        for k in steps:
            self.rotate(ct, k)
        return [ct for _ in steps]

    def hoist(self, ct):
        return None

    def rotate_sum(self, items):
        for ct, k in items:
            self.rotate(ct, k)
        self._count("Add", len(items) - 1)
        return items[0][0]

    def hoisted_mux(self, ct, digits, k1, k2, v_ext, v_scale, c):
        self.rotate(ct, k1)
        self.rotate(ct, k2)
        self._count("Mul_pt")
        self._count("Add")
        return _DryCt(ct.limbs, ct.scale * v_scale)


class _DryMasks(H.MaskProvider):
    def plaintext(self, kind, k, extended=False):
        i = self.index[(kind, k)]
        return None, float(self.ctx.q[self.entries[i][3] - 1])


def test_table1_operation_counts_h64():
    t1 = gold("table1_opcounts.json")
    h = 64
    rh = int(math.isqrt(h))
    ctx = C.Context(14, [60] + [45] * 7, [60, 60], 45)
    masks = _DryMasks(ctx, h, 8)
    beta = masks.beta
    ev = DryEvaluator(ctx)
    x = _DryCt(8, ctx.scale)
    H.lintrans_bsgs(ev, x, range(-h + 1, h), 1, masks, "mu")
    s11 = dict(ev.counts)
    ev.counts = {}
    H.lintrans_bsgs(ev, x, range(h), h, masks, "zeta")
    s12 = dict(ev.counts)
    ev.counts = {}
    H.matmul(ev, x, x, h, masks)
    tot = dict(ev.counts)
    # Table I per step (Add/Mul_pt/Rot), with our exact counts
    assert s11["Mul_pt"] == 2 * h - 1 <= 2 * h and s11["Rot"] == 22 <= 3 * rh
    assert s12["Mul_pt"] == h and s12["Rot"] == 14 <= 2 * rh
    step2_rot = tot["Rot"] - s11["Rot"] - s12["Rot"]
    step2_mulpt = tot["Mul_pt"] - s11["Mul_pt"] - s12["Mul_pt"]
    assert step2_rot == 3 * (h - 1) <= 3 * h and step2_mulpt == h - 1 <= h
    assert tot["Mul_ct"] == h
    assert tot["Rot"] == 225 <= t1["rotations_h64"] == 3 * h + 5 * rh
    assert tot["Mul_pt"] <= 4 * h and tot["Add"] <= 6 * h
    assert tot["Rescale"] == 4   # two after Step 1, two after the single relinearisation
    steps = H.matmul_rotation_steps(h, beta, 8)
    assert all(k % beta == 0 for k in steps) and len({C.galois_element(k, ctx.N) for k in steps}) == len(steps)


def test_g_coefficients_match_paper_and_lemmas():
    g = gold("g_coeffs.json")
    for d in range(1, 5):
        printed = [Fraction(a, b) for a, b in g["g"][str(d)]]
        assert H.g_coeffs(d) == printed
        n = H.g_int_coeffs(d)
        assert [Fraction(v, 2 ** (2 * d - 1)) for v in n] == printed
        # Prop. I-III: odd, g(1) = 1, g'(m) = p_d (1 - m^2)^d
        assert sum(printed) == 1
        deriv = [c * (2 * j + 1) for j, c in enumerate(printed)]
        want = [H.p_d(d) * math.comb(d, j) * (-1) ** j for j in range(d + 1)]
        assert deriv == want
        # Lemma 3.1
        assert H.p_d(d) == sum(Fraction(math.comb(2 * i, i), 4 ** i) for i in range(d + 1)) == printed[0]
    assert H.p_d(4) == Fraction(315, 128)


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_lemmas_3_2_3_3_and_theorem_3_5(d):
    m = np.linspace(0, 1, 20001)
    gd = H.g_eval(d, m)
    pd = float(H.p_d(d))
    assert np.all(1 - gd >= -1e-15)
    assert np.all(1 - gd <= (1 - m) ** pd + 1e-12)                 # Lemma 3.2
    assert np.all(1 - gd <= 2 ** d * (1 - m) ** (d + 1) + 1e-12)   # Lemma 3.3
    for log_delta, sigma in ((8, 20), (20, 20)):
        delta = 2.0 ** -log_delta
        k, x = 0, delta
        while 1 - x > 2.0 ** -sigma:
            x = H.g_eval(d, x)
            k += 1
        bound = math.log2(1 / delta) / math.log2(pd) + math.log2(sigma - 1) / math.log2(d + 1)
        assert k <= math.ceil(bound) + 2   # Thm 3.5 without its O(1) term, plus slack


def test_sign_composition_error_for_config_inputs():
    x = np.concatenate([np.linspace(2 ** -8, 1, 50001), -np.linspace(2 ** -8, 1, 50001)])
    err = np.abs(H.g_iter(4, 8, x) - np.sign(x)).max()
    assert err <= 2 ** -20
    # fewer compositions are not enough at |x| = 2^-8
    assert abs(H.g_iter(4, 7, 2 ** -8) - 1) > 2 ** -20


@pytest.fixture(scope="module")
def enc_ctx():
    ctx = C.Context(10, [60, 40, 40, 40, 40], [60], 40)
    return ctx


@pytest.mark.parametrize("limbs", [3, 5])
def test_encrypted_matmul_oracle(enc_ctx, limbs):
    ctx = C.Context(10, [60] + [40] * (limbs - 1), [60], 40)
    h = 8
    beta = ctx.S // (h * h)
    ks = C.keygen(ctx, 2, 5, rot_steps=H.matmul_rotation_steps(h, beta, limbs))
    rng = np.random.default_rng(limbs)
    As = [rng.uniform(-1, 1, (h, h)) for _ in range(beta)]
    Bs = [rng.uniform(-1, 1, (h, h)) for _ in range(beta)]
    A = C.encrypt(ctx, ks, H.pack(As, h, beta), 11)
    B = C.encrypt(ctx, ks, H.pack(Bs, h, beta), 12)
    ev = C.Evaluator(ctx, ks)
    out = H.matmul(ev, A, B, h)
    assert out.limbs == limbs - (3 if limbs >= 4 else 2)
    got = H.unpack(C.decrypt(ctx, ks, out), h, beta)
    assert max(np.abs(g - a @ b).max() for g, a, b in zip(got, As, Bs)) < 2 ** -18


def test_encrypted_transpose_oracle():
    ctx = C.Context(10, [60, 40, 40], [60], 40)
    h = 8
    beta = ctx.S // (h * h)
    ks = C.keygen(ctx, 2, 3, rot_steps=H.transpose_rotation_steps(h, beta))
    ms = [np.random.default_rng(i).uniform(-1, 1, (h, h)) for i in range(beta)]
    out = H.transpose(C.Evaluator(ctx, ks), C.encrypt(ctx, ks, H.pack(ms, h, beta), 5), h)
    got = H.unpack(C.decrypt(ctx, ks, out), h, beta)
    assert out.limbs == 2 and max(np.abs(g - m.T).max() for g, m in zip(got, ms)) < 2 ** -20


def test_encrypted_sign_and_relu_oracle():
    ctx = C.Context(9, [60] + [40] * 15, [60] * 3, 40)
    ks = C.keygen(ctx, 2, 9)
    rng = np.random.default_rng(3)
    x = rng.uniform(2 ** -8, 1, ctx.S) * rng.choice([-1, 1], ctx.S)
    ct = C.encrypt(ctx, ks, x, 21)
    ev = C.Evaluator(ctx, ks)
    s = H.sign_approx(ev, ct, 4, 8, refresh_seed=77)
    assert ev.counts["Refresh"] == 2 and s.limbs == 8
    assert np.abs(C.decrypt(ctx, ks, s) - H.g_iter(4, 8, x)).max() < 2 ** -18
    r = H.sign_approx(C.Evaluator(ctx, ks), ct, 4, 8, relu=True, refresh_seed=77)
    assert np.abs(C.decrypt(ctx, ks, r) - np.maximum(x, 0)).max() < 2 ** -18
    with pytest.raises(ValueError):
        H.sign_approx(C.Evaluator(ctx, ks), ct, 4, 8)


def test_dense_layer_oracle():
    """Fig. 5, one layer: the oracle's encrypted feedforward and backpropagation
    decrypt to the FP64 computation of the same functions: E = W X,
    M = E (1 + g_d^(k)(E/4)) / 2 and dW_j = (((1 + g_d^(k)(E/4)) / 2) . G) X_j^T,
    on ragged shapes (rows and inputs not multiples of h, a partly filled
    second group), with one refresh per output block inside the sign."""
    from paper_2207_04620_gb300 import workloads as wl
    h, d, k, div = 8, 2, 5, 4.0
    ctx = C.Context(10, [60] + [40] * 15, [60] * 3, 40)
    beta = ctx.S // (h * h)
    ks = C.keygen(ctx, 2, 91, rot_steps=H.dense_rotation_steps(h, beta))
    ev = C.Evaluator(ctx, ks)
    W, X, G = wl.dense_inputs(5, 14, 90, h)
    Wp, Xp, Gp = wl.dense_pack(W, X, G, h, beta)
    n_out, groups = len(Wp), len(Xp)
    assert (n_out, groups) == (2, 2)
    Wc = [[C.encrypt(ctx, ks, Wp[i][g], 200 + 10 * i + g) for g in range(groups)] for i in range(n_out)]
    Xc = [C.encrypt(ctx, ks, Xp[g], 300 + g) for g in range(groups)]
    Gc = [C.encrypt(ctx, ks, Gp[i], 400 + i) for i in range(n_out)]
    E, M, dW = H.dense_layer(ev, Wc, Xc, Gc, h, d, k, div, refresh_seed=17)
    assert ev.counts.get("Refresh", 0) == n_out
    Eb = wl.blocks(W, h)
    Xb = [r[0] for r in wl.blocks(X, h)]
    Gb = [r[0] for r in wl.blocks(G, h)]
    for i in range(n_out):
        e_ref = sum(a @ b for a, b in zip(Eb[i], Xb))
        s_ref = H.g_iter(d, k, e_ref / div)
        l_ref = (1 + s_ref) / 2 * Gb[i]
        e = H.unpack(C.decrypt(ctx, ks, E[i]), h, beta)[0]
        m = H.unpack(C.decrypt(ctx, ks, M[i]), h, beta)[0]
        assert np.abs(e - e_ref).max() < 2 ** -16
        assert np.abs(m - e_ref * (1 + s_ref) / 2).max() < 2 ** -14
        for g in range(groups):
            got = H.unpack(C.decrypt(ctx, ks, dW[i][g]), h, beta)
            for p in range(beta):
                j = beta * g + p
                want = l_ref @ Xb[j].T if j < len(Xb) else np.zeros((h, h))
                assert np.abs(got[p] - want).max() < 2 ** -14


def test_aggregate_oracle():
    """Alg. 6 Aggregation: the updated model decrypts to w - eta/(B N) * sum_i g_i
    (FP64), for 5 parties and two model ciphertexts; the level drops by one and
    the model's scale is kept."""
    ctx = C.Context(10, [60, 40, 40, 40], [60], 40)
    ks = C.keygen(ctx, 2, 7)
    ev = C.Evaluator(ctx, ks)
    rng = np.random.default_rng(3)
    n_parties, count, c = 5, 2, 0.01 / (4 * 5)
    w = [rng.uniform(-1, 1, ctx.S) for _ in range(count)]
    g = [[rng.uniform(-1, 1, ctx.S) for _ in range(count)] for _ in range(n_parties)]
    wc = [C.encrypt(ctx, ks, w[m], 10 + m) for m in range(count)]
    gc = [[C.encrypt(ctx, ks, g[i][m], 100 + 10 * i + m) for m in range(count)] for i in range(n_parties)]
    out = H.aggregate(ev, gc, wc, c)
    for m in range(count):
        assert out[m].limbs == wc[m].limbs - 1 and out[m].scale == wc[m].scale
        want = w[m] - c * sum(g[i][m] for i in range(n_parties))
        assert np.abs(C.decrypt(ctx, ks, out[m]) - want).max() < 2 ** -22


@pytest.mark.parametrize("h,t", [(4, 1), (4, 2), (8, 2), (8, 4), (16, 4), (16, 8), (32, 8)])
@pytest.mark.parametrize("variant", ["alg3", "depth2"])
def test_slot_rectangular_matmul(h, t, variant):
    """App. D: with A~ = (A; ...; A) (h/t copies of a t x h matrix A), the cut
    k-sum plus the row-block folds leaves h/t copies of A.B (t x h) in every
    packed matrix; also a direct check of the key lemma's consequence: row
    block j of sum_{i<t} phi^i(mu(A~)) . pi^i(zeta(B)) is the k = j t + i part."""
    beta = 2
    rng = np.random.default_rng(100 * h + t)
    As = [rng.uniform(-1, 1, (t, h)) for _ in range(beta)]
    Bs = [rng.uniform(-1, 1, (h, h)) for _ in range(beta)]
    At = [np.vstack([A] * (h // t)) for A in As]
    out = H.unpack(H.slot_rmatmul(H.pack(At, h, beta), H.pack(Bs, h, beta), h, t, beta, variant), h, beta)
    for o, A, B in zip(out, As, Bs):
        assert np.abs(o - np.vstack([A @ B] * (h // t))).max() < 1e-12
    A, B = As[0], Bs[0]
    part = sum(H.phi(H.mu(At[0]), i) * H.pi_(H.zeta(B), i) for i in range(t))
    for j in range(h // t):
        want = sum((H.phi(H.mu(np.vstack([A] * (h // t))), j * t + i) * H.pi_(H.zeta(B), j * t + i))[:t]
                   for i in range(t))
        assert np.allclose(part[j * t:(j + 1) * t], want)


def test_rectangular_operation_counts_h64():
    """App. D Table (Alg. "41"): Step 2 takes 3(t-1) rotations and t-1 masks,
    Step 3 t ciphertext products, Step 4 log2(h/t) rotations; Step 1 is the
    square product's."""
    h, t = 64, 8
    ctx = C.Context(14, [60] + [45] * 7, [60, 60], 45)
    masks = _DryMasks(ctx, h, 8)
    ev = DryEvaluator(ctx)
    x = _DryCt(8, ctx.scale)
    H.matmul(ev, x, x, h, masks)
    sq = dict(ev.counts)
    ev.counts = {}
    H.rmatmul(ev, x, x, h, t, masks)
    rc = dict(ev.counts)
    step1_rot = sq["Rot"] - 3 * (h - 1)
    assert rc["Rot"] == step1_rot + 3 * (t - 1) + int(math.log2(h // t))
    assert rc["Mul_ct"] == t
    assert rc["Mul_pt"] == sq["Mul_pt"] - (h - t)
    beta = masks.beta
    steps = H.matmul_rotation_steps(h, beta, 8, t)
    assert set(steps) < set(H.matmul_rotation_steps(h, beta, 8)) | {beta * h * e for e in (8, 16, 32)}
    assert {beta * h * e for e in (8, 16, 32)} <= set(steps)


@pytest.mark.parametrize("limbs", [3, 5])
def test_encrypted_rectangular_matmul_oracle(limbs):
    """HE-RMatMult on ciphertexts decrypts to h/t copies of A.B for every packed pair."""
    ctx = C.Context(10, [60] + [40] * (limbs - 1), [60], 40)
    h, t = 8, 2
    beta = ctx.S // (h * h)
    ks = C.keygen(ctx, 2, 6, rot_steps=H.matmul_rotation_steps(h, beta, limbs, t))
    rng = np.random.default_rng(7 + limbs)
    As = [rng.uniform(-1, 1, (t, h)) for _ in range(beta)]
    Bs = [rng.uniform(-1, 1, (h, h)) for _ in range(beta)]
    At = C.encrypt(ctx, ks, H.pack([np.vstack([A] * (h // t)) for A in As], h, beta), 13)
    B = C.encrypt(ctx, ks, H.pack(Bs, h, beta), 14)
    out = H.rmatmul(C.Evaluator(ctx, ks), At, B, h, t)
    got = H.unpack(C.decrypt(ctx, ks, out), h, beta)
    assert max(np.abs(g - np.vstack([a @ b] * (h // t))).max() for g, a, b in zip(got, As, Bs)) < 2 ** -18


def test_eval_g_structure_and_values():
    """One application of g_d (reading R8) on a ciphertext: decrypts to g_d(x) for d = 1..4,
    uses g_depth(d) levels and min(d, 3) + 1 ciphertext products (x^2, y^2, y^2 B(y), x P
    as d needs them); the scale stays the context's."""
    ctx = C.Context(9, [60] + [40] * 6, [60] * 3, 40)
    ks = C.keygen(ctx, 2, 5)
    rng = np.random.default_rng(8)
    x = rng.uniform(-1, 1, ctx.S)
    ct = C.encrypt(ctx, ks, x, 13)
    for d in (1, 2, 3, 4):
        ev = C.Evaluator(ctx, ks)
        out = H.eval_g(ev, ct, d)
        assert out.limbs == ct.limbs - H.g_depth(d)
        assert H.g_depth(d) == {1: 2, 2: 3, 3: 4, 4: 4}[d]
        assert ev.counts["KeySwitch"] == min(d, 3) + 1
        assert np.abs(C.decrypt(ctx, ks, out) - H.g_eval(d, x)).max() < 2 ** -20
        assert abs(out.scale / ctx.scale - 1) < 2 ** -10


def test_level_adjust_scales_and_drops():
    """level_adjust brings a ciphertext to a lower level at a chosen scale, times a real
    constant: the decryption is c * m within the rounding of the integer constant."""
    ctx = C.Context(9, [60] + [40] * 4, [60, 60], 40)
    ks = C.keygen(ctx, 2, 6)
    x = np.linspace(-1, 1, ctx.S)
    ct = C.encrypt(ctx, ks, x, 3)
    ev = C.Evaluator(ctx, ks)
    for target, c, sc in ((3, 1.0, ctx.scale), (1, -2.5, 2.0 ** 38), (2, 1 / 128, 2.0 ** 41)):
        y = H.level_adjust(ev, ct, target, c, sc)
        assert y.limbs == target and y.scale == sc
        assert np.abs(C.decrypt(ctx, ks, y) - c * x).max() < 2 ** -20
    with pytest.raises(ValueError):
        H.level_adjust(ev, ct, ct.limbs, 1.0, ctx.scale)
