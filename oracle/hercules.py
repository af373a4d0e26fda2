"""Oracle for the paper's packed matrix product and composite sign -- TEST
INFRASTRUCTURE ONLY (see oracle/ckks.py for the rules on who may import it).

Sec. 3 (packed h x h matrix product with O(h) rotations), App. B (baby-step /
giant-step and the multiplexer trick), App. C (transpose), App. E (parallel
matrices, iota_beta) and Sec. 4 (composite polynomial g_d^(k), Alg. 5), each
written from the paper's formulas.  Vectors here are "logical" slot vectors of
length n = h^2; `expand` maps them to the S = beta*h^2 CKKS slots (App. E).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from . import ckks as C

# ----------------------------------------------------------------------------
# Vectors, rotations, encodings (Sec. 3.2, 3.4, App. E)
# ----------------------------------------------------------------------------


def R(m: np.ndarray, k: int) -> np.ndarray:
    """R(m, k) = (m_k, ..., m_{n-1}, m_0, ..., m_{k-1})  (Sec. 3.2)."""
    return np.roll(m, -k)


def iota_inv(A: np.ndarray) -> np.ndarray:
    """Row-major matrix -> vector, a_{h*i+j} = A_{i,j} (Sec. 3.4)."""
    return np.asarray(A).reshape(-1)


def pack(mats, h: int, beta: int) -> np.ndarray:
    """iota_beta^-1: slot beta*(h*i+j)+k holds (A_k)_{i,j}; missing matrices are zero (App. E)."""
    out = np.zeros(beta * h * h)
    for k, A in enumerate(mats):
        out[k::beta] = iota_inv(A)
    return out


def unpack(slots: np.ndarray, h: int, beta: int) -> list:
    return [np.asarray(slots[k: beta * h * h: beta]).reshape(h, h) for k in range(beta)]


def expand(u: np.ndarray, beta: int) -> np.ndarray:
    """A logical mask over n = h^2 positions acting on every packed matrix: u'[beta*t + j] = u[t]."""
    return np.repeat(u, beta)


def baby_steps(h: int) -> int:
    """b = 2^ceil(log2(h)/2) (reading R3: the power-of-two split also covers h = 32, 128)."""
    return 1 << math.ceil(math.log2(h) / 2) if h > 1 else 1


# ----------------------------------------------------------------------------
# Permutations and their diagonal vectors (Sec. 3.3, 3.5, Eqs. (1), (5)-(16))
# ----------------------------------------------------------------------------


def mu(A):
    h = A.shape[0]
    return np.array([[A[i, (i + j) % h] for j in range(h)] for i in range(h)])


def zeta(A):
    h = A.shape[0]
    return np.array([[A[(i + j) % h, j] for j in range(h)] for i in range(h)])


def phi(A, k=1):
    h = A.shape[0]
    return np.array([[A[i, (j + k) % h] for j in range(h)] for i in range(h)])


def pi_(A, k=1):
    h = A.shape[0]
    return np.array([[A[(i + k) % h, j] for j in range(h)] for i in range(h)])


def perm_matrix(h: int, kind: str, k: int = 0) -> np.ndarray:
    """Matrix representations U^mu, U^zeta (Eqs. 5-6), V^k, P^k (Eqs. 7-8) and
    the transpose U^T (App. C) as 0/1 matrices on R^(h^2)."""
    n = h * h
    U = np.zeros((n, n), dtype=np.int64)
    for i in range(h):
        for j in range(h):
            if kind == "mu":
                t = h * i + (i + j) % h
            elif kind == "zeta":
                t = h * ((i + j) % h) + j
            elif kind == "V":
                t = h * i + (j + k) % h
            elif kind == "P":
                t = h * ((i + k) % h) + j
            elif kind == "T":
                t = h * j + i
            else:
                raise ValueError(kind)
            U[h * i + j, t] = 1
    return U


def diagonal(U: np.ndarray, k: int) -> np.ndarray:
    """k-th diagonal vector u_k = (U_{0,k}, U_{1,k+1}, ..., U_{n-1,k-1}) (Sec. 3.2)."""
    n = U.shape[0]
    return np.array([U[t, (t + k) % n] for t in range(n)])


def diag_mu(h: int, k: int) -> np.ndarray:
    """u^mu_k, -h < k < h, from the two case formulas of Step 1-1 (Sec. 3.6)."""
    t = np.arange(h * h)
    if k >= 0:
        return ((t - h * k >= 0) & (t - h * k < h - k)).astype(np.int64)
    return ((t - (h + k) * h >= -k) & (t - (h + k) * h < h)).astype(np.int64)


def diag_zeta(h: int, k: int) -> np.ndarray:
    """u^zeta_{h*k}, 0 <= k < h: nonzero exactly at the (k + h*i)-th entries (Step 1-2)."""
    t = np.arange(h * h)
    return (t % h == k).astype(np.int64)


def diag_v(h: int, k: int) -> np.ndarray:
    """v_k, 1 <= k < h: 1 iff [t]_h < h - k (Step 2)."""
    t = np.arange(h * h)
    return ((t % h) < h - k).astype(np.int64)


def diag_v_neg(h: int, k: int) -> np.ndarray:
    """v_{k-h}: 1 iff h - k <= [t]_h < h (Step 2)."""
    t = np.arange(h * h)
    return ((t % h) >= h - k).astype(np.int64)


def diag_transpose(h: int, s: int) -> np.ndarray:
    """Diagonal (h-1)*s of U^T, -h < s < h (App. C, reading R4: the printed
    case i < 0 is wrong; the mask is 1 at t = (h+1)*i + s for
    max(0,-s) <= i < h - max(0,s))."""
    t = np.arange(h * h)
    i = (t - s) // (h + 1)
    ok = ((t - s) % (h + 1) == 0) & (i >= max(0, -s)) & (i < h - max(0, s))
    return ok.astype(np.int64)


# ----------------------------------------------------------------------------
# Matrix-product plan: which masks, at which level and scale (readings R2, R3, R7, R9)
# ----------------------------------------------------------------------------


def matmul_variant(limbs: int) -> str:
    """Alg. 3 needs 3 rescales (masks of Step 1, the Step 2 mask, the ct x ct
    product); with exactly 2 levels above q_0 the depth-2 rearrangement runs."""
    if limbs >= 4:
        return "alg3"
    if limbs == 3:
        return "depth2"
    raise ValueError("HE-MatMult needs at least 3 limbs, got %d" % limbs)


def plan_masks(h: int, limbs: int):
    """Ordered list of (kind, index, logical mask vector, limbs of the
    ciphertext it multiplies) for one product:
      mu   : l = -h+1..h-1, vector R(u^mu_l, -b*floor(l/b))            at `limbs`
      zeta : l = 0..h-1, R(u^zeta_{hl}, -h*b*floor(l/b)) for Alg. 3,
             u^zeta_{hl} unrotated for the depth-2 variant              at `limbs`
      v    : k = 1..h-1, v_k (Step 2 selects after rotating)              at `limbs`-1 (Alg. 3 only),
             used in the extended basis q_0..q_{l-1}, p_0..p_{K-1}
    Every mask is encoded at mask_scale(ctx), whatever the level (reading R7)."""
    variant = matmul_variant(limbs)
    b = baby_steps(h)
    out = []
    for l in range(-h + 1, h):
        out.append(("mu", l, R(diag_mu(h, l), -b * (l // b)), limbs))
    for l in range(h):
        if variant == "alg3":
            out.append(("zeta", l, R(diag_zeta(h, l), -h * b * (l // b)), limbs))
        else:
            out.append(("zeta", l, diag_zeta(h, l), limbs))
    if variant == "alg3":
        for k in range(1, h):
            out.append(("v", k, diag_v(h, k), limbs - 1))
    return out


def matmul_rotation_steps(h: int, beta: int, limbs: int, t: int | None = None) -> list:
    """Every rotation amount one product uses, reduced mod S = beta*h^2
    (rotations are cyclic on the slots), sorted, without 0; with t < h those of
    the rectangular product (k < t, plus the row-block folds)."""
    t = h if t is None else t
    variant = matmul_variant(limbs)
    b = baby_steps(h)
    s = set()
    for l in range(-h + 1, h):
        s.add(beta * (l % b))
        s.add(beta * b * (l // b))
    if variant == "alg3":
        for l in range(h):
            s.add(beta * h * (l % b))
            s.add(beta * h * b * (l // b))
        for k in range(1, t):
            s.update({beta * k, beta * (k - h), beta * h * k})
    else:
        for l in range(1, h):
            s.add(beta * h * l)
        for k in range(1, t):
            s.update({beta * k, beta * (k - h), beta * h * k})
    e = t
    while e < h:
        s.add(beta * h * e)
        e *= 2
    n_slots = beta * h * h
    return sorted({k % n_slots for k in s} - {0})


def mask_scale(ctx: C.Context) -> int:
    """Reading R7: every plan mask is encoded at one fixed integer scale, the power of two
    nearest the context's scale, at every level (so a mask's coefficients do not depend on the
    level); Mul_pt then RS by q_{l-1} leaves scale * 2^e / q_{l-1}, tracked exactly."""
    return 1 << round(math.log2(ctx.scale))


class MaskProvider:
    """Encodes plan masks with the oracle encoder (at mask_scale(ctx), every level);
    `coeffs` exposes the signed integer coefficients so a test can hand the
    very same plaintexts to another implementation."""

    def __init__(self, ctx: C.Context, h: int, limbs: int):
        self.ctx, self.h, self.limbs = ctx, h, limbs
        self.beta = ctx.S // (h * h)
        self.entries = plan_masks(h, limbs)
        self.index = {(kind, k): i for i, (kind, k, _, _) in enumerate(self.entries)}
        self._coeffs: dict = {}

    def coeffs(self, i: int) -> np.ndarray:
        if i not in self._coeffs:
            kind, k, vec, lm = self.entries[i]
            self._coeffs[i] = C.encode_real(self.ctx.N, expand(vec, self.beta), float(mask_scale(self.ctx)))
        return self._coeffs[i]

    def plaintext(self, kind: str, k: int, extended: bool = False):
        """NTT-form mask over q_0..q_{l-1} (and p_0..p_{K-1} if extended)."""
        i = self.index[(kind, k)]
        lm = self.entries[i][3]
        prim = self.ctx.q[:lm] + (self.ctx.p if extended else [])
        pt = self.ctx.ntt(self.ctx.signed_to_rows(self.coeffs(i), prim), prim)
        return pt, float(mask_scale(self.ctx))


# ----------------------------------------------------------------------------
# Alg. 2 with baby-step/giant-step (App. B), Alg. 3 and the depth-2 variant
# ----------------------------------------------------------------------------


def lintrans_bsgs(ev: C.Evaluator, ct: C.Ciphertext, ls, stride: int, masks: MaskProvider, kind: str):
    """HE-LinTrans over diagonals stride*l, l in `ls` (Alg. 2), split as
    l = b*i + j (App. B): sum_i Rot( sum_j Mul_pt(Rot(ct, stride*j), R(u_l, -stride*b*i)), stride*b*i ).
    Baby rotations share one ModUp; the result is NOT rescaled."""
    b = baby_steps(masks.h)
    beta = masks.beta
    groups: dict = {}
    for l in ls:
        groups.setdefault(l // b, []).append((l % b, l))
    js = sorted({j for g in groups.values() for j, _ in g})
    babies = dict(zip(js, ev.rotate_hoisted(ct, [beta * stride * j for j in js])))
    items = []
    for i in sorted(groups):
        inner = None
        for j, l in groups[i]:
            pt, sc = masks.plaintext(kind, l)
            term = ev.mul_plain(babies[j], pt, sc)
            inner = term if inner is None else ev.add(inner, term)
        items.append((inner, beta * stride * b * i))
    # giant steps: one ModDown for the whole sum (reading R10)
    return ev.rotate_sum(items)


def matmul(ev: C.Evaluator, A: C.Ciphertext, B: C.Ciphertext, h: int, masks: MaskProvider | None = None,
           t: int | None = None):
    """HE-MatMult of beta = S/h^2 packed pairs (Alg. 3 / App. E).  With t < h
    only the terms k < t of Step 2/3 are formed (Alg. "41", lines 3-10)."""
    if A.limbs != B.limbs:
        raise ValueError("A and B must be at the same level")
    t = h if t is None else t
    masks = masks or MaskProvider(ev.ctx, h, A.limbs)
    if matmul_variant(A.limbs) == "alg3":
        return _matmul_alg3(ev, A, B, h, masks, t)
    return _matmul_depth2(ev, A, B, h, masks, t)


def rmatmul(ev: C.Evaluator, At: C.Ciphertext, B: C.Ciphertext, h: int, t: int, masks: MaskProvider | None = None):
    """HE-RMatMult (App. D, Alg. "41"): At packs A~ = (A; ...; A), h/t vertical
    copies of a t x h matrix A (t a power of two dividing h).  The square
    schedule with its k-sum cut to k < t leaves, in row block j, the terms
    k = j t + i of A.B; log2(h/t) rotate-and-add steps by t*h*2^e rows fold
    the blocks, so every block holds A.B (h/t copies, as the input)."""
    if t < 1 or h % t or t & (t - 1):
        raise ValueError("t must be a power of two dividing h")
    out = matmul(ev, At, B, h, masks, t)
    beta = ev.ctx.S // (h * h)
    e = t
    while e < h:
        out = ev.add(out, ev.rotate(out, beta * h * e))
        e *= 2
    return out


def _matmul_alg3(ev, A, B, h, masks, t=None):
    t = h if t is None else t
    beta = masks.beta
    # Step 1-1 / 1-2: A0 = U^mu a, B0 = U^zeta b
    A0 = ev.rescale(lintrans_bsgs(ev, A, range(-h + 1, h), 1, masks, "mu"))
    B0 = ev.rescale(lintrans_bsgs(ev, B, range(h), h, masks, "zeta"))
    # Step 2 (App. B multiplexer, applied after hoisting): A^(k) = v_k . R(A0, k)
    # + (1 - v_k) . R(A0, k-h); every rotation of A0 shares one ModUp and the
    # selection happens in the extended basis before a single ModDown per k.
    # A^(k) stays at scale Delta*c (c = the masks' scale as an integer; no rescale
    # per k); B^(k) = R(B0, h*k) stays at the same level; A^(0) = c * A0.
    qt = mask_scale(ev.ctx)
    DA = ev.hoist(A0)
    Bk = [B0] + ev.rotate_hoisted(B0, [beta * h * k for k in range(1, t)])
    # Step 3: sum_k A^(k) (x) B^(k), one relinearisation, then the two rescales
    acc = ev.tensor(ev.mul_int(A0, qt, new_scale=A0.scale * float(qt)), Bk[0])
    for k in range(1, t):
        v_ext, sc = masks.plaintext("v", k, extended=True)
        Ak = ev.hoisted_mux(A0, DA, beta * k, beta * (k - h), v_ext, sc, qt)
        acc = ev.add(acc, ev.tensor(Ak, Bk[k]))
    return ev.rescale(ev.rescale(ev.relinearize(acc)))


def _matmul_depth2(ev, A, B, h, masks, t=None):
    """Reading R9: with T_l = u^zeta_{hl} . R(b, hl) and S_m = sum_{l<m} T_l,
    v_k . R(B0, hk) = R(S_{h-k}, hk) and v_{k-h} . R(B0, hk) = R(B0 - S_{h-k}, hk),
    so A.B = A0.B0 + sum_{k>=1} R(A0,k).R(S_{h-k},hk) + R(A0,k-h).R(B0-S_{h-k},hk)
    needs one level for the masks and one for the ct x ct products."""
    t = h if t is None else t
    beta = masks.beta
    A0 = ev.rescale(lintrans_bsgs(ev, A, range(-h + 1, h), 1, masks, "mu"))
    Rb = [B] + ev.rotate_hoisted(B, [beta * h * l for l in range(1, h)])
    T = []
    for l in range(h):
        pt, sc = masks.plaintext("zeta", l)
        T.append(ev.mul_plain(Rb[l], pt, sc))
    prefix = [None, T[0]]          # prefix[m] = S_m
    for l in range(1, h):
        prefix.append(ev.add(prefix[-1], T[l]))
    Bfull = prefix[h]
    B0 = ev.rescale(Bfull)
    RA = ev.rotate_hoisted(A0, [beta * k for k in range(1, t)] + [beta * (k - h) for k in range(1, t)])
    acc = ev.tensor(A0, B0)
    for k in range(1, t):
        X = ev.rescale(prefix[h - k])
        Y = ev.rescale(ev.sub(Bfull, prefix[h - k]))
        acc = ev.add(acc, ev.tensor(RA[k - 1], ev.rotate(X, beta * h * k)))
        acc = ev.add(acc, ev.tensor(RA[t - 1 + k - 1], ev.rotate(Y, beta * h * k)))
    return ev.rescale(ev.relinearize(acc))


# ----------------------------------------------------------------------------
# FP64 slot-space model of the same schedules (no encryption; pins Eq. (2))
# ----------------------------------------------------------------------------


def slot_matmul(a: np.ndarray, b: np.ndarray, h: int, beta: int = 1, variant: str = "alg3",
                t: int | None = None) -> np.ndarray:
    """Runs the masks and rotations of `matmul` on plain slot vectors (terms k < t)."""
    t = h if t is None else t
    n = beta * h * h
    Rb_ = lambda v, k: np.roll(v, -(beta * k) % n)
    bb = baby_steps(h)
    A0 = np.zeros(n)
    for l in range(-h + 1, h):
        i, j = l // bb, l % bb
        A0 += Rb_(expand(R(diag_mu(h, l), -bb * i), beta) * Rb_(a, j), bb * i)
    if variant == "alg3":
        B0 = np.zeros(n)
        for l in range(h):
            i, j = l // bb, l % bb
            B0 += Rb_(expand(R(diag_zeta(h, l), -h * bb * i), beta) * Rb_(b, h * j), h * bb * i)
        out = A0 * B0
        for k in range(1, t):
            v = expand(diag_v(h, k), beta)
            Ak = v * Rb_(A0, k) + (1 - v) * Rb_(A0, k - h)
            out += Ak * Rb_(B0, h * k)
        return out
    T = [expand(diag_zeta(h, l), beta) * Rb_(b, h * l) for l in range(h)]
    Sm = np.cumsum(np.vstack([np.zeros(n)] + T), axis=0)
    out = A0 * Sm[h]
    for k in range(1, t):
        out += Rb_(A0, k) * Rb_(Sm[h - k], h * k) + Rb_(A0, k - h) * Rb_(Sm[h] - Sm[h - k], h * k)
    return out


def slot_rmatmul(a: np.ndarray, b: np.ndarray, h: int, t: int, beta: int = 1, variant: str = "alg3") -> np.ndarray:
    """`rmatmul` on plain slot vectors: the cut k-sum, then the row-block folds."""
    n = beta * h * h
    out = slot_matmul(a, b, h, beta, variant, t)
    e = t
    while e < h:
        out = out + np.roll(out, -(beta * h * e) % n)
        e *= 2
    return out


def slot_transpose(a: np.ndarray, h: int, beta: int = 1) -> np.ndarray:
    n = beta * h * h
    out = np.zeros(n)
    for s in range(-h + 1, h):
        out += expand(diag_transpose(h, s), beta) * np.roll(a, -(beta * (h - 1) * s) % n)
    return out


def transpose_masks(h: int):
    """Masks of the transpose, in plan order s = -h+1..h-1: R(t_(h-1)s, -(h-1)*b*floor(s/b))."""
    b = baby_steps(h)
    return [("T", sh, R(diag_transpose(h, sh), -(h - 1) * b * (sh // b))) for sh in range(-h + 1, h)]


def transpose_rotation_steps(h: int, beta: int) -> list:
    b = baby_steps(h)
    st = set()
    for sh in range(-h + 1, h):
        st.add(beta * (h - 1) * (sh % b))
        st.add(beta * (h - 1) * b * (sh // b))
    n = beta * h * h
    return sorted({k % n for k in st} - {0})


class TransposeMasks(MaskProvider):
    """Mask plaintexts of App. C's transpose (diagonals (h-1)s), encoded at mask_scale(ctx)."""

    def __init__(self, ctx: C.Context, h: int, limbs: int):
        self.ctx, self.h, self.limbs = ctx, h, limbs
        self.beta = ctx.S // (h * h)
        self.entries = [(kind, sh, vec, limbs) for kind, sh, vec in transpose_masks(h)]
        self.index = {(kind, k): i for i, (kind, k, _, _) in enumerate(self.entries)}
        self._coeffs = {}


def transpose(ev: C.Evaluator, ct: C.Ciphertext, h: int, masks: "TransposeMasks | None" = None):
    """App. C: U^T a = sum_s t_{(h-1)s} . R(a, (h-1)s) over the 2h-1 diagonals,
    baby-step/giant-step split on s, then one rescale."""
    masks = masks or TransposeMasks(ev.ctx, h, ct.limbs)
    return ev.rescale(lintrans_bsgs(ev, ct, range(-h + 1, h), h - 1, masks, "T"))


# ----------------------------------------------------------------------------
# Sec. 4: g_d, p_d, composite sign, AppMax / ReLU (Alg. 5; readings R8, R17)
# ----------------------------------------------------------------------------


def g_coeffs(d: int) -> list:
    """Coefficients (Fractions) of m^1, m^3, ..., m^(2d+1) in
    g_d(m) = sum_{i=0}^{d} 4^-i C(2i,i) m (1-m^2)^i."""
    c = [Fraction(0)] * (d + 1)
    for i in range(d + 1):
        w = Fraction(math.comb(2 * i, i), 4 ** i)
        for j in range(i + 1):  # (1-m^2)^i = sum_j C(i,j) (-m^2)^j
            c[j] += w * math.comb(i, j) * (-1) ** j
    return c


def g_int_coeffs(d: int) -> list:
    """The same coefficients as integers n_j with g_d = sum_j n_j m^(2j+1) / 2^(2d-1)."""
    den = 2 ** (2 * d - 1)
    out = []
    for f in g_coeffs(d):
        v = f * den
        assert v.denominator == 1
        out.append(int(v))
    return out


def p_d(d: int) -> Fraction:
    """p_d = (2d+1)/4^d * C(2d, d) (Lemma 3.1)."""
    return Fraction(2 * d + 1, 4 ** d) * math.comb(2 * d, d)


def g_eval(d: int, m):
    """FP64 g_d(m) with the integer coefficients (Horner in m^2)."""
    n = g_int_coeffs(d)
    y = np.asarray(m, dtype=np.float64) ** 2
    acc = np.zeros_like(y) + n[-1]
    for c in reversed(n[:-1]):
        acc = acc * y + c
    return np.asarray(m) * acc / 2.0 ** (2 * d - 1)


def g_iter(d: int, k: int, m):
    for _ in range(k):
        m = g_eval(d, m)
    return m


def _rha(x: float) -> int:
    return int(C.round_half_away(np.array([x]))[0])


def level_adjust(ev: C.Evaluator, ct: C.Ciphertext, target: int, c_real: float, target_scale: float):
    """Brings ct to `target` limbs at scale `target_scale`, multiplying its
    message by c_real: drop to target+1 limbs, multiply by the integer
    C = round(c_real * target_scale * q_target / scale), rescale by q_target.
    The result's scale is declared to be target_scale (the integer rounding
    of C changes the message by a relative 2^-(bits of C))."""
    if ct.limbs <= target:
        raise ValueError("cannot raise the level")
    x = ev.drop(ct, target + 1) if ct.limbs > target + 1 else ct
    qt = ev.ctx.q[target]
    c = _rha(c_real * target_scale * float(qt) / ct.scale)
    ev._count("Mul_const")
    y = ev.rescale(ev.mul_int(x, c))
    y.scale = target_scale
    return y


def _square_rs(ev, a, b):
    """a * b, relinearised and rescaled in one division by P q_top (reading R21)."""
    return ev.relin_rescale(ev.tensor(a, b))


def eval_g(ev: C.Evaluator, x: C.Ciphertext, d: int) -> C.Ciphertext:
    """One application of g_d (1 <= d <= 4) on a ciphertext (reading R8).
    With y = x^2 and g_d(x) = x P(y) / 2^(2d-1), P(y) = sum_j n_j y^j with the
    integer n_j of Sec. 4, P is split as n0 + n1 y + n2 y^2 + y^2 B(y) with
    B(y) = n3 y + n4 y^2 (the terms present for this d): y and y^2 by squaring,
    B at y^2's level, one product y^2 * B, the remaining terms brought to that
    level, then x * P with the 2^-(2d-1) folded into the level adjustment of x.
    Four ciphertext products for d = 3 and 4, two and three for d = 1 and 2.
    Operands of one product always share level and scale."""
    if not 1 <= d <= 4:
        raise ValueError("eval_g covers 1 <= d <= 4")
    n = g_int_coeffs(d)
    y = {1: _square_rs(ev, x, x)}
    if d >= 2:
        y[2] = _square_rs(ev, y[1], y[1])
    top = None  # y^2 B(y)
    if d >= 3:
        y1 = level_adjust(ev, y[1], y[2].limbs, 1.0, y[2].scale)
        B = ev.mul_int(y1, n[3])
        if d == 4:
            B = ev.add(B, ev.mul_int(y[2], n[4]))
        top = _square_rs(ev, y[2], B)
    lead = top if top is not None else y[min(d, 2)]
    lp, sp = lead.limbs, lead.scale
    terms = [top] if top is not None else []
    for j in range(1, min(d, 2) + 1):
        if y[j].limbs > lp:
            terms.append(level_adjust(ev, y[j], lp, float(n[j]), sp))
        else:
            terms.append(ev.mul_int(y[j], n[j]))
    P = terms[0]
    for t in terms[1:]:
        P = ev.add(P, t)
    P = ev.add_const(P, float(n[0]))
    xa = level_adjust(ev, x, lp, 1.0 / 2 ** (2 * d - 1), sp)
    return _square_rs(ev, xa, P)


def g_depth(d: int) -> int:
    """Levels one application of eval_g consumes: y, y^2 and y^2 B(y) take one
    level each (as many as d needs), x * P one more."""
    return min(d, 3) + 1


def refresh(ev: C.Evaluator, ct: C.Ciphertext, seed: int, counter: int) -> C.Ciphertext:
    """DBootstrap (Fig. 1 item 14) between compositions (reading R17): the
    collective refresh protocol to the top level and the default scale."""
    ev._count("Refresh")
    return C.dbootstrap(ev.ctx, ev.ks, ct, seed, counter)


def sign_approx(ev: C.Evaluator, x: C.Ciphertext, d: int, k: int, relu: bool = False,
                refresh_seed: int | None = None) -> C.Ciphertext:
    """g_d^(k)(x) (Sec. 4.2) or ReLU(x) = x (1 + g_d^(k)(x)) / 2 (Sec. 4.4).
    Before a composition whose depth (plus the final ReLU product) no longer
    fits, the ciphertext is refreshed if a refresh seed is given."""
    dg = g_depth(d)
    m = x
    refreshes = 0
    for it in range(k):
        need = dg + (1 if (relu and it == k - 1) else 0)
        if m.limbs - 1 < need:
            if refresh_seed is None:
                raise ValueError("levels exhausted")
            m = refresh(ev, m, refresh_seed, refreshes)
            refreshes += 1
        m = eval_g(ev, m, d)
    if not relu:
        return m
    s1 = ev.add_const(m, 1.0)
    xa = level_adjust(ev, x, m.limbs, 0.5, m.scale)
    return _square_rs(ev, xa, s1)


# ----------------------------------------------------------------------------
# Fig. 5: one dense layer, feedforward then backpropagation (reading R19)
# ----------------------------------------------------------------------------


def dense_layer(ev: C.Evaluator, W, X, G, h: int, d: int, k: int, input_div: float, refresh_seed: int,
                masks: dict | None = None):
    """One dense layer over h x h blocks packed beta = S/h^2 per ciphertext.

    W[i][g] packs W_{i,j}, j = beta*g + p at position p; X[g] packs X_j (a
    batch of h inputs as columns); G[i] packs the upstream gradient G_i at
    position 0.  Feedforward: E_i = sum_j W_{i,j} X_j, i.e. the block products,
    their sum over g and a rotate-and-add over the beta positions (position 0
    then holds E_i); s_i = g_d^(k)(E_i / input_div); ReLU(E_i) = E_i (1+s_i)/2.
    Backpropagation: L_i = phi'(E_i) . G_i with phi' = (1+s_i)/2, copied to
    every position by rotations, and dW_{i,j} = L_i X_j^T with the X_j
    transposed (App. C) and brought to L's level and scale.
    masks: optional {"fwd", "transpose", "bwd"} mask providers."""
    masks = masks or {}
    S = ev.ctx.S
    beta = S // (h * h)
    n_out, groups = len(W), len(X)
    fwd = masks.get("fwd") or MaskProvider(ev.ctx, h, X[0].limbs)
    E = []
    for i in range(n_out):
        acc = None
        for g in range(groups):
            p = matmul(ev, W[i][g], X[g], h, fwd)
            acc = p if acc is None else ev.add(acc, p)
        t = 1
        while t < beta:
            acc = ev.add(acc, ev.rotate(acc, t))
            t *= 2
        E.append(acc)
    M, L = [], []
    for i in range(n_out):
        # E / input_div at E's scale, one level down (a scale of input_div * Delta would square
        # away from Delta through the composition)
        e_in = level_adjust(ev, E[i], E[i].limbs - 1, 1.0 / input_div, E[i].scale)
        s1 = ev.add_const(sign_approx(ev, e_in, d, k, refresh_seed=refresh_seed + i), 1.0)
        m = _square_rs(ev, ev.drop(E[i], s1.limbs), s1)
        m.scale *= 2
        li = _square_rs(ev, s1, ev.drop(G[i], s1.limbs))
        li.scale *= 2
        t = 1
        while t < beta:
            li = ev.add(li, ev.rotate(li, S - t))
            t *= 2
        M.append(m)
        L.append(li)
    tr = masks.get("transpose") or TransposeMasks(ev.ctx, h, X[0].limbs)
    XT = [level_adjust(ev, transpose(ev, x, h, tr), L[0].limbs, 1.0, L[0].scale) for x in X]
    bwd = masks.get("bwd") or MaskProvider(ev.ctx, h, L[0].limbs)
    dW = [[matmul(ev, L[i], XT[g], h, bwd) for g in range(groups)] for i in range(n_out)]
    return E, M, dW


def dense_rotation_steps(h: int, beta: int) -> list:
    """Rotations dense_layer uses: both HE-MatMult variants, the transpose, +-2^t for 2^t < beta."""
    st = set(matmul_rotation_steps(h, beta, 4)) | set(matmul_rotation_steps(h, beta, 3))
    st |= set(transpose_rotation_steps(h, beta))
    n = beta * h * h
    t = 1
    while t < beta:
        st |= {t, n - t}
        t *= 2
    return sorted(st)


# ----------------------------------------------------------------------------
# Alg. 6, Aggregation: the server's model update
# ----------------------------------------------------------------------------


def aggregate(ev: C.Evaluator, grads, models, eta_over_bn: float):
    """grads[i][m]: party i's encrypted gradient for model ciphertext m.
    The server sums the parties' gradients (Add), multiplies the sum by
    eta/(B*N) and subtracts it from the model (Mul_pt, Sub).  The constant is
    applied as a level adjustment of the sum to one level below the model at
    the model's scale (its integer round(-eta/(B*N) * scale_w * q_t / scale_g),
    then RS), so the update is added to the model dropped to that level."""
    out = []
    for m, w in enumerate(models):
        acc = grads[0][m]
        for i in range(1, len(grads)):
            acc = ev.add(acc, grads[i][m])
        upd = level_adjust(ev, acc, w.limbs - 1, -eta_over_bn, w.scale)
        out.append(ev.add(ev.drop(w, w.limbs - 1), upd))
    return out
