"""CPU CKKS oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow RNS-CKKS written from the MCKKS description (Sec. 2.2, Fig. 1 of
the paper) and the readings listed under "Readings" in the design notes.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this module.  It shares no code with the CUDA library: both sides follow
the same written specification independently.

Representation
--------------
* Ring R_Q = Z_Q[X]/(X^N+1), Q = q_0 ... q_{L-1} (Sec. 2.2); special primes
  p_0 .. p_{K-1} for hybrid key switching.
* A polynomial is a uint64 array ``[limbs, N]`` of residues, limb i modulo the
  i-th prime of its basis.  Ciphertext components are kept in the NTT
  (evaluation) representation: slot j of a limb holds a(psi^(2 brv(j)+1)).
* A ciphertext is (c0, c1) with c0 + c1*s = Delta*m + e (Fig. 1 items 5-6).

Every modular product goes through ``ckks_ref.c`` (``(u128)a*b % q``).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libckks_ref.so")
_lib = None

U64P = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle's C primitives with gcc (plain -O2, OpenMP over rows)."""
    src = os.path.join(_HERE, "ckks_ref.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        c_int, u64 = ctypes.c_int, ctypes.c_uint64
        L.ref_powmod.restype = u64
        L.ref_powmod.argtypes = [u64, u64, u64]
        L.ref_ntt_direct.argtypes = [U64P, U64P, c_int, u64, u64]
        L.ref_ntt_forward_rows.argtypes = [U64P, c_int, c_int, U64P, U64P]
        L.ref_ntt_inverse_rows.argtypes = [U64P, c_int, c_int, U64P, U64P]
        L.ref_negacyclic_schoolbook.argtypes = [U64P, U64P, U64P, c_int, u64]
        for name in ("ref_rows_add", "ref_rows_sub", "ref_rows_mul"):
            getattr(L, name).argtypes = [U64P, U64P, U64P, c_int, c_int, U64P]
        L.ref_rows_neg.argtypes = [U64P, U64P, c_int, c_int, U64P]
        L.ref_rows_mul_scalar.argtypes = [U64P, U64P, U64P, c_int, c_int, U64P]
        L.ref_rows_add_scalar.argtypes = [U64P, U64P, U64P, c_int, c_int, U64P]
        L.ref_rows_reduce.argtypes = [U64P, U64P, c_int, c_int, U64P]
        L.ref_automorphism_ntt.argtypes = [U64P, U64P, c_int, c_int, u64]
        L.ref_automorphism_coef.argtypes = [U64P, U64P, c_int, c_int, u64, U64P]
        L.ref_basis_convert.argtypes = [U64P, U64P, c_int, c_int, U64P, U64P, c_int, U64P, U64P]
        _lib = L
    return _lib


def _u64(xs) -> np.ndarray:
    return np.ascontiguousarray(np.array([int(x) for x in xs], dtype=np.uint64))


# ----------------------------------------------------------------------------
# Number theory (primes and roots; readings R13)
# ----------------------------------------------------------------------------

def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 2^64 (the first 12 prime bases)."""
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for p in small:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def find_primes(log_n: int, bits: list[int]) -> list[int]:
    """For each requested size b, in order: the largest prime q < 2^b with
    q = 1 (mod 2N) not already chosen."""
    two_n = 2 << log_n
    chosen: list[int] = []
    for b in bits:
        c = (1 << b) - two_n + 1
        while not is_prime(c) or c in chosen:
            c -= two_n
            if c <= two_n:
                raise ValueError("no prime of %d bits for N=2^%d" % (b, log_n))
        chosen.append(c)
    return chosen


def find_psi(q: int, n: int) -> int:
    """psi = x^((q-1)/2N) for the smallest x >= 2 such that psi^N = -1 (mod q),
    i.e. psi is a primitive 2N-th root of unity."""
    e = (q - 1) // (2 * n)
    x = 2
    while True:
        psi = pow(x, e, q)
        if pow(psi, n, q) == q - 1:
            return psi
        x += 1


def brv(x: int, bits: int) -> int:
    return int(format(x, "0%db" % bits)[::-1], 2) if bits else 0


def galois_element(k: int, n: int) -> int:
    """Rotation R(m, k) (left by k slots, Sec. 3.2) is X -> X^(5^k mod 2N)."""
    return pow(5, k % (n // 2), 2 * n)


# ----------------------------------------------------------------------------
# Randomness: SplitMix64 (Steele, Lea, Flood 2014), one stream per purpose
# ----------------------------------------------------------------------------

GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1

PURPOSE_SK, PURPOSE_PK_A, PURPOSE_PK_E = 1, 2, 3
PURPOSE_KEY_A, PURPOSE_KEY_E = 4, 5
PURPOSE_ENC_V, PURPOSE_ENC_E0, PURPOSE_ENC_E1 = 6, 7, 8
PURPOSE_SMUDGE = 9
PURPOSE_PCKS_U, PURPOSE_PCKS_E0, PURPOSE_PCKS_E1 = 10, 11, 12
PURPOSE_DB_MASK, PURPOSE_DB_E0, PURPOSE_DB_E1, PURPOSE_DB_CRP = 13, 14, 15, 16


def mix64(z: int) -> int:
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def _mix64_np(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based SplitMix64 stream for (seed, purpose, a, b):
    state_0 = seed XOR mix64(key + GAMMA), key = purpose<<56 | a<<32 | b;
    draw i returns mix64(state_0 + (i+1)*GAMMA)."""

    def __init__(self, seed: int, purpose: int, a: int = 0, b: int = 0):
        key = ((purpose & 0xFF) << 56) | ((a & 0xFFFFFF) << 32) | (b & 0xFFFFFFFF)
        self.state = (seed ^ mix64((key + GAMMA) & M64)) & M64
        self.count = 0

    def draws(self, n: int) -> np.ndarray:
        idx = np.arange(self.count + 1, self.count + 1 + n, dtype=np.uint64)
        with np.errstate(over="ignore"):
            st = np.uint64(self.state) + idx * np.uint64(GAMMA)
        self.count += n
        return _mix64_np(st)


def sample_uniform(stream: Stream, q: int, n: int) -> np.ndarray:
    """Uniform residues mod q by rejection on bitlen(q)-bit draws (low bits)."""
    mask = np.uint64((1 << q.bit_length()) - 1)
    out = np.empty(0, dtype=np.uint64)
    while out.size < n:
        r = stream.draws(n - out.size) & mask
        ok = r < np.uint64(q)
        # draws past the n-th acceptance must not be consumed
        acc = np.flatnonzero(ok)
        need = n - out.size
        if acc.size >= need:
            last = acc[need - 1]
            stream.count -= (r.size - 1 - last)
            out = np.concatenate([out, r[acc[:need]]])
        else:
            out = np.concatenate([out, r[ok]])
    return out


def sample_uniform_wide(stream: Stream, m: int, n: int) -> np.ndarray:
    """Uniform residues mod m without rejection: value j is (d_2j * 2^64 + d_(2j+1)) mod m for the
    stream's draws d (reading R17: every value depends on its own two draws only, bias below
    m / 2^128)."""
    d = stream.draws(2 * n)
    hi = d[0::2].astype(object)
    lo = d[1::2].astype(object)
    return np.array([int((int(a) << 64) | int(b)) % m for a, b in zip(hi, lo)], dtype=np.uint64)


def sample_ternary(stream: Stream, n: int) -> np.ndarray:
    """Coefficients in {-1, 0, 1}: draw % 3 mapped 0->0, 1->1, 2->-1."""
    r = (stream.draws(n) % np.uint64(3)).astype(np.int64)
    r[r == 2] = -1
    return r


def gaussian_thresholds(sigma: float) -> tuple[int, list[int]]:
    """CDT table of the discrete Gaussian of parameter sigma on [-B, B],
    B = floor(6 sigma): T_k = floor(2^63 * cum_k / total), weights
    exp(-k^2 / (2 sigma^2)) summed in increasing k."""
    bound = int(math.floor(6.0 * sigma))
    two_s2 = 2.0 * sigma * sigma
    w = [math.exp(-float(k * k) / two_s2) for k in range(-bound, bound + 1)]
    total = 0.0
    for x in w:
        total += x
    cum = 0.0
    th = []
    for x in w:
        cum += x
        th.append(int(math.floor((cum / total) * 9223372036854775808.0)))
    return bound, th


def sample_gaussian(stream: Stream, n: int, sigma: float) -> np.ndarray:
    """value = (smallest k with (draw >> 1) < T_k) - B, clamped to B."""
    bound, th = gaussian_thresholds(sigma)
    r = stream.draws(n) >> np.uint64(1)
    idx = np.searchsorted(np.array(th, dtype=np.uint64), r, side="right")
    idx = np.minimum(idx, 2 * bound)
    return idx.astype(np.int64) - bound


# ----------------------------------------------------------------------------
# Context
# ----------------------------------------------------------------------------

class Context:
    """Parameters: ring degree 2^log_n, Q primes of the given sizes (q_0
    first), special primes, default scale 2^log2_scale, error width sigma, and
    alpha, the primes per key-switching digit (reading R11; None = one per
    special prime)."""

    def __init__(self, log_n: int, q_bits, p_bits, log2_scale: float, sigma: float = 3.2, alpha: int | None = None):
        self.log_n = log_n
        self.N = 1 << log_n
        self.S = self.N // 2
        primes = find_primes(log_n, list(q_bits) + list(p_bits))
        self.q = primes[: len(q_bits)]
        self.p = primes[len(q_bits):]
        self.n_q, self.K = len(self.q), len(self.p)
        self.alpha = alpha or self.K
        self.dnum = -(-self.n_q // self.alpha)
        self.scale = 2.0 ** log2_scale
        self.sigma = sigma
        self.psi = {x: find_psi(x, self.N) for x in primes}
        self.P = math.prod(self.p)

    # -- row helpers ---------------------------------------------------------
    def ntt(self, a: np.ndarray, primes) -> np.ndarray:
        out = np.ascontiguousarray(a, dtype=np.uint64).copy()
        rows = out.reshape(-1, self.N)
        lib().ref_ntt_forward_rows(rows, rows.shape[0], self.log_n, _u64(primes), _u64(self.psi[x] for x in primes))
        return out

    def intt(self, a: np.ndarray, primes) -> np.ndarray:
        out = np.ascontiguousarray(a, dtype=np.uint64).copy()
        rows = out.reshape(-1, self.N)
        lib().ref_ntt_inverse_rows(rows, rows.shape[0], self.log_n, _u64(primes), _u64(self.psi[x] for x in primes))
        return out

    def _binop(self, fn, a, b, primes):
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        out = np.empty_like(a)
        getattr(lib(), fn)(out, a, b, len(primes), self.N, _u64(primes))
        return out

    def add(self, a, b, primes):
        return self._binop("ref_rows_add", a, b, primes)

    def sub(self, a, b, primes):
        return self._binop("ref_rows_sub", a, b, primes)

    def mul(self, a, b, primes):
        return self._binop("ref_rows_mul", a, b, primes)

    def neg(self, a, primes):
        a = np.ascontiguousarray(a, dtype=np.uint64)
        out = np.empty_like(a)
        lib().ref_rows_neg(out, a, len(primes), self.N, _u64(primes))
        return out

    def mul_scalar(self, a, scalars, primes):
        a = np.ascontiguousarray(a, dtype=np.uint64)
        out = np.empty_like(a)
        lib().ref_rows_mul_scalar(out, a, _u64(scalars), len(primes), self.N, _u64(primes))
        return out

    def add_scalar(self, a, scalars, primes):
        a = np.ascontiguousarray(a, dtype=np.uint64)
        out = np.empty_like(a)
        lib().ref_rows_add_scalar(out, a, _u64(scalars), len(primes), self.N, _u64(primes))
        return out

    def automorphism(self, a, g: int) -> np.ndarray:
        a = np.ascontiguousarray(a, dtype=np.uint64)
        out = np.empty_like(a)
        lib().ref_automorphism_ntt(out, a, a.size // self.N, self.log_n, g)
        return out

    def signed_to_rows(self, v: np.ndarray, primes) -> np.ndarray:
        """Integer coefficients (int64 or Python ints) -> residues per prime."""
        out = np.empty((len(primes), self.N), dtype=np.uint64)
        v = np.asarray(v)
        for i, t in enumerate(primes):
            if v.dtype == object:
                out[i] = np.array([int(x) % t for x in v], dtype=np.uint64)
            else:  # every prime here is below 2^62, so int64 arithmetic is exact
                out[i] = np.mod(v.astype(np.int64), np.int64(t)).astype(np.uint64)
        return out

    def basis_convert(self, x: np.ndarray, src, dst) -> np.ndarray:
        """Fast basis conversion (no correction): residues of one integer
        modulo `src` -> residues modulo `dst` (coefficient representation)."""
        Qs = math.prod(src)
        qhat = [Qs // t for t in src]
        qhat_inv = [pow(qh % t, -1, t) for qh, t in zip(qhat, src)]
        qhat_mod = [qh % d for qh in qhat for d in dst]
        out = np.empty((len(dst), self.N), dtype=np.uint64)
        lib().ref_basis_convert(out, np.ascontiguousarray(x, dtype=np.uint64), self.N, len(src), _u64(src),
                                _u64(qhat_inv), len(dst), _u64(dst), _u64(qhat_mod))
        return out


# ----------------------------------------------------------------------------
# Encoding (Fig. 1 item 3, Ecd; reading R14)
# ----------------------------------------------------------------------------
#
# Coefficient i of the encoding of real slots z at scale D is the exact real
#     x_i = D * (2/N) * sum_j z_j cos(pi * (i * e_j mod 2N) / N),   e_j = 5^j mod 2N,
# rounded half away from zero; a value within TIE_BAND of a half-integer is taken
# as that half-integer.  The sum is evaluated in double-double arithmetic (about
# 106 bits), whose error is many orders of magnitude below the band, so the
# integer is the one the exact value gives.

TIE_BAND = 2.0 ** -20


def round_half_away(x: np.ndarray) -> np.ndarray:
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def slot_exponents(n: int) -> np.ndarray:
    """e_j = 5^j mod 2N: slot j is the value at zeta^(e_j), zeta = exp(i pi/N)."""
    s = n // 2
    e = np.empty(s, dtype=np.int64)
    v = 1
    for j in range(s):
        e[j] = v
        v = v * 5 % (2 * n)
    return e


# ---- double-double arithmetic: a value is the unevaluated sum hi + lo of two doubles
# (Dekker 1971; Knuth, TAOCP vol. 2, 4.2.2).  Each step is one IEEE double operation
# rounded once (numpy never fuses a product into a sum).

def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _fast_two_sum(a, b):  # |a| >= |b|
    s = a + b
    return s, b - (s - a)


def _split(a):
    c = 134217729.0 * a  # 2^27 + 1
    hi = c - (c - a)
    return hi, a - hi


def _two_prod(a, b):
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def dd_add(x, y):
    s, e = _two_sum(x[0], y[0])
    t, f = _two_sum(x[1], y[1])
    s, e = _fast_two_sum(s, e + t)
    return _fast_two_sum(s, e + f)


def dd_neg(x):
    return -x[0], -x[1]


def dd_mul(x, y):
    p, e = _two_prod(x[0], y[0])
    return _fast_two_sum(p, e + (x[0] * y[1] + x[1] * y[0]))


def dd_mul_double(x, d):
    p, e = _two_prod(x[0], d)
    return _fast_two_sum(p, e + x[1] * d)


# ---- roots of unity from a 45-digit decimal evaluation

def _decimal_pi(ctx):
    """pi by Machin's formula 16 atan(1/5) - 4 atan(1/239), in the given decimal context."""
    from decimal import Decimal

    def atan_inv(k):
        x = Decimal(1) / k
        x2 = x * x
        term, total, n = x, x, 1
        eps = Decimal(10) ** -(ctx.prec + 2)
        while abs(term) > eps:
            term = -term * x2
            n += 2
            total += term / n
        return total

    return 16 * atan_inv(5) - 4 * atan_inv(239)


def _decimal_cos_sin(phi, ctx):
    """Taylor series of cos and sin at |phi| <= pi/4."""
    from decimal import Decimal

    eps = Decimal(10) ** -(ctx.prec + 2)
    c, s = Decimal(1), phi
    term_c, term_s, k = Decimal(1), phi, 0
    p2 = phi * phi
    while abs(term_c) > eps or abs(term_s) > eps:
        term_c = -term_c * p2 / ((2 * k + 1) * (2 * k + 2))
        term_s = -term_s * p2 / ((2 * k + 2) * (2 * k + 3))
        c += term_c
        s += term_s
        k += 1
    return c, s


def _to_dd(d):
    from decimal import Decimal

    hi = float(d)
    return hi, float(d - Decimal(hi))


_ROOTS: dict = {}


def roots_dd(m: int):
    """w^k = exp(-2 pi i k / m) for k < m/2 as double-double (re, im) arrays: cos and sin of
    2 pi k/m evaluated in 45-digit decimal arithmetic by Taylor series after reduction to an
    angle of at most pi/4 (k = m/8 is pi/4), then rounded to double-double."""
    if m in _ROOTS:
        return _ROOTS[m]
    from decimal import Context

    dctx = Context(prec=45)
    pi = _decimal_pi(dctx)
    m8 = m // 8
    table = [_decimal_cos_sin(dctx.multiply(pi, dctx.divide(2 * j, m)), dctx) for j in range(m8 + 1)]
    re_h, re_l, im_h, im_l = (np.empty(m // 2) for _ in range(4))
    for k in range(m // 2):
        if k <= m8:
            c, s = table[k]
        elif k <= 2 * m8:
            s, c = table[2 * m8 - k]
        elif k <= 3 * m8:
            s, c = table[k - 2 * m8]
            c = -c
        else:
            c, s = table[4 * m8 - k]
            c = -c
        re_h[k], re_l[k] = _to_dd(c)
        im_h[k], im_l[k] = _to_dd(-s)  # exp(-i theta) = cos theta - i sin theta
    _ROOTS[m] = ((re_h, re_l), (im_h, im_l))
    return _ROOTS[m]


def fft_dd(re, im):
    """Unnormalised DFT X_i = sum_k a_k exp(-2 pi i ik/m) along the last axis, double-double
    complex values given as (hi, lo) pairs of arrays; radix-2 decimation in frequency
    (Gentleman-Sande) with natural-order input, result returned in natural order."""
    m = re[0].shape[-1]
    (wr_h, wr_l), (wi_h, wi_l) = roots_dd(m)
    lead = re[0].shape[:-1]
    x = [a.copy() for a in (re[0], re[1], im[0], im[1])]
    h = m // 2
    while h >= 1:
        blocks = m // (2 * h)
        v = [a.reshape(lead + (blocks, 2, h)) for a in x]
        a_re = (v[0][..., 0, :], v[1][..., 0, :])
        a_im = (v[2][..., 0, :], v[3][..., 0, :])
        b_re = (v[0][..., 1, :], v[1][..., 1, :])
        b_im = (v[2][..., 1, :], v[3][..., 1, :])
        step = m // (2 * h)
        w_re = (wr_h[: h * step : step], wr_l[: h * step : step])
        w_im = (wi_h[: h * step : step], wi_l[: h * step : step])
        s_re, s_im = dd_add(a_re, b_re), dd_add(a_im, b_im)
        d_re, d_im = dd_add(a_re, dd_neg(b_re)), dd_add(a_im, dd_neg(b_im))
        t_re = dd_add(dd_mul(d_re, w_re), dd_neg(dd_mul(d_im, w_im)))
        t_im = dd_add(dd_mul(d_re, w_im), dd_mul(d_im, w_re))
        out = [np.empty_like(a) for a in v]
        for o, top, bot in zip(out, (s_re[0], s_re[1], s_im[0], s_im[1]), (t_re[0], t_re[1], t_im[0], t_im[1])):
            o[..., 0, :] = top
            o[..., 1, :] = bot
        x = [o.reshape(lead + (m,)) for o in out]
        h //= 2
    bits = m.bit_length() - 1
    rev = np.array([int(format(i, "0%db" % bits)[::-1], 2) for i in range(m)])
    return (x[0][..., rev], x[1][..., rev]), (x[2][..., rev], x[3][..., rev])


def encode_real_coeffs(n: int, z) -> tuple:
    """m_i = (2/N) sum_j z_j cos(pi (i e_j mod 2N)/N) for i < N, as double-double arrays
    (hi, lo) of shape z.shape[:-1] + (N,): the encoding before the scale.  z: real slots
    (last axis, at most N/2, zero-padded)."""
    z = np.asarray(z, dtype=np.float64)
    lead = z.shape[:-1]
    s = n // 2
    zz = np.zeros(lead + (s,))
    zz[..., : z.shape[-1]] = z
    e = slot_exponents(n)
    big = np.zeros(lead + (2 * n,))
    big[..., e] = zz
    big[..., (2 * n - e) % (2 * n)] = zz  # the conjugate of a real slot
    zero = np.zeros_like(big)
    (xr_h, xr_l), _ = fft_dd((big, zero), (zero, zero))
    return xr_h[..., :n] / n, xr_l[..., :n] / n  # division by a power of two is exact


def round_dd(x) -> np.ndarray:
    """Round hi + lo half away from zero (int64), a value within TIE_BAND of a half-integer
    taken as the half-integer.  Integer and fractional parts are split from each word exactly."""
    hi, lo = np.asarray(x[0], dtype=np.float64), np.asarray(x[1], dtype=np.float64)
    if np.any(~np.isfinite(hi)) or np.max(np.abs(hi), initial=0.0) >= 2.0 ** 62:
        raise OverflowError("encoded coefficient exceeds 2^62")
    r1, r2 = np.rint(hi), np.rint(lo)
    d = (hi - r1) + (lo - r2)  # both differences exact; |d| <= 1
    base = r1.astype(np.int64) + r2.astype(np.int64)
    tie = np.abs(np.abs(d) - 0.5) <= TIE_BAND
    up = np.where(tie, d > 0, d > 0.5)
    down = np.where(tie, d < 0, d < -0.5)
    c = base + up.astype(np.int64) - down.astype(np.int64)
    # a tie x = base + sign(d)/2 rounds away from zero: toward +inf above zero, -inf below
    neg_tie_up = tie & (d > 0) & (base < 0)    # x = base + 1/2 < 0: goes to base
    pos_tie_dn = tie & (d < 0) & (base > 0)    # x = base - 1/2 > 0: goes to base
    c = c - neg_tie_up.astype(np.int64) + pos_tie_dn.astype(np.int64)
    if np.max(np.abs(c), initial=0) >= 2 ** 62:
        raise OverflowError("encoded coefficient exceeds 2^62")
    return c


def scale_round(m, scale: float) -> np.ndarray:
    """c_i = round(scale * m_i) under the rule of round_dd, m a double-double array."""
    return round_dd(dd_mul_double(m, float(scale)))


def encode_real(n: int, z, scale: float) -> np.ndarray:
    """Slots -> signed integer coefficients (Ecd): c_i = round(scale * m_i) with m_i the
    exact canonical-embedding coefficient (see the section comment).  z may carry leading
    batch axes."""
    return scale_round(encode_real_coeffs(n, z), scale)


def decode(n: int, coeffs: np.ndarray, scale: float) -> np.ndarray:
    """Centered integer coefficients -> complex slots: z_j = sum_i c_i zeta^(i e_j) / scale."""
    e = slot_exponents(n)
    big = np.zeros(2 * n, dtype=np.complex128)
    big[:n] = np.asarray(coeffs, dtype=np.float64)
    y = np.fft.ifft(big) * (2 * n)
    return y[e] / scale


# ----------------------------------------------------------------------------
# Keys, encryption, decryption (Fig. 1 items 1-6; readings R15, R16)
# ----------------------------------------------------------------------------

@dataclass
class SwitchKey:
    b: np.ndarray  # [dnum, n_q + K, N] NTT form over q_0..q_{L-1}, p_0..p_{K-1}
    a: np.ndarray


@dataclass
class KeySet:
    seed: int
    s_parts: list           # per-party ternary secrets (signed int64 coefficients)
    s: np.ndarray           # sum of the shares (signed)
    s_ntt: np.ndarray       # [n_q + K, N]
    s_parts_ntt: list       # per party, [n_q + K, N]
    pk_b: np.ndarray        # [n_q, N]
    pk_a: np.ndarray
    relin: SwitchKey | None = None
    rot: dict = field(default_factory=dict)  # galois element -> SwitchKey


@dataclass
class Ciphertext:
    c: np.ndarray   # [2, limbs, N] NTT form over q_0..q_{limbs-1}
    scale: float

    @property
    def limbs(self) -> int:
        return self.c.shape[1]

    def copy(self) -> "Ciphertext":
        return Ciphertext(self.c.copy(), self.scale)


def all_primes(ctx: Context):
    return ctx.q + ctx.p


def gen_switch_key(ctx: Context, ks: KeySet, key_id: int, sp_ntt: np.ndarray) -> SwitchKey:
    """swk_j = (-a_j s + e_j + P * [1 on digit j's primes] * s', a_j) over PQ
    (reading R11: the gadget factor P*Qhat_j*[Qhat_j^-1]_{Q_j} is P modulo the
    primes of digit j and 0 modulo every other prime)."""
    prim = all_primes(ctx)
    rows = len(prim)
    B = np.empty((ctx.dnum, rows, ctx.N), dtype=np.uint64)
    A = np.empty((ctx.dnum, rows, ctx.N), dtype=np.uint64)
    for j in range(ctx.dnum):
        st = Stream(ks.seed, PURPOSE_KEY_A, key_id, j)
        a = np.stack([sample_uniform(st, t, ctx.N) for t in prim])
        e = sample_gaussian(Stream(ks.seed, PURPOSE_KEY_E, key_id, j), ctx.N, ctx.sigma)
        e_ntt = ctx.ntt(ctx.signed_to_rows(e, prim), prim)
        b = ctx.sub(e_ntt, ctx.mul(a, ks.s_ntt, prim), prim)
        lo, hi = j * ctx.alpha, min((j + 1) * ctx.alpha, ctx.n_q)
        sub_p = prim[lo:hi]
        gad = ctx.mul_scalar(sp_ntt[lo:hi], [ctx.P % t for t in sub_p], sub_p)
        b[lo:hi] = ctx.add(b[lo:hi], gad, sub_p)
        B[j], A[j] = b, a
    return SwitchKey(B, A)


def keygen(ctx: Context, n_parties: int, seed: int, rot_steps=(), relin: bool = True) -> KeySet:
    """SecKeyGen for every party, s = sum of shares (reading R16), then the
    collective public key, the relinearisation key (s' = s^2) and one Galois
    key per rotation step (s' = sigma_g(s))."""
    prim = all_primes(ctx)
    parts = [sample_ternary(Stream(seed, PURPOSE_SK, party, 0), ctx.N) for party in range(n_parties)]
    s = np.sum(parts, axis=0).astype(np.int64)
    s_ntt = ctx.ntt(ctx.signed_to_rows(s, prim), prim)
    parts_ntt = [ctx.ntt(ctx.signed_to_rows(x, prim), prim) for x in parts]
    st = Stream(seed, PURPOSE_PK_A, 0, 0)
    a = np.stack([sample_uniform(st, t, ctx.N) for t in ctx.q])
    e = sample_gaussian(Stream(seed, PURPOSE_PK_E, 0, 0), ctx.N, ctx.sigma)
    e_ntt = ctx.ntt(ctx.signed_to_rows(e, ctx.q), ctx.q)
    b = ctx.sub(e_ntt, ctx.mul(a, s_ntt[: ctx.n_q], ctx.q), ctx.q)
    ks = KeySet(seed, parts, s, s_ntt, parts_ntt, b, a)
    if relin:
        ks.relin = gen_switch_key(ctx, ks, 0, ctx.mul(s_ntt, s_ntt, prim))
    for k in rot_steps:
        add_rotation_key(ctx, ks, k)
    return ks


def add_rotation_key(ctx: Context, ks: KeySet, k: int) -> None:
    g = galois_element(k, ctx.N)
    if g != 1 and g not in ks.rot:
        ks.rot[g] = gen_switch_key(ctx, ks, g, ctx.automorphism(ks.s_ntt, g))


def encrypt_coeffs(ctx: Context, ks: KeySet, m: np.ndarray, scale: float, limbs: int, seed: int,
                   tag: int = 0, index: int = 0) -> Ciphertext:
    """Enc(pk, m) = (v*pk_b + e0 + m, v*pk_a + e1) over the first `limbs`
    primes; m are signed integer coefficients (an encoded plaintext)."""
    prim = ctx.q[:limbs]
    v = sample_ternary(Stream(seed, PURPOSE_ENC_V, tag, index), ctx.N)
    e0 = sample_gaussian(Stream(seed, PURPOSE_ENC_E0, tag, index), ctx.N, ctx.sigma)
    e1 = sample_gaussian(Stream(seed, PURPOSE_ENC_E1, tag, index), ctx.N, ctx.sigma)
    vn = ctx.ntt(ctx.signed_to_rows(v, prim), prim)
    e0n = ctx.ntt(ctx.signed_to_rows(e0, prim), prim)
    e1n = ctx.ntt(ctx.signed_to_rows(e1, prim), prim)
    mn = ctx.ntt(ctx.signed_to_rows(m, prim), prim)
    c0 = ctx.add(ctx.add(ctx.mul(vn, ks.pk_b[:limbs], prim), e0n, prim), mn, prim)
    c1 = ctx.add(ctx.mul(vn, ks.pk_a[:limbs], prim), e1n, prim)
    return Ciphertext(np.stack([c0, c1]), float(scale))


def encrypt(ctx: Context, ks: KeySet, slots, seed: int, limbs: int | None = None, scale: float | None = None,
            tag: int = 0, index: int = 0) -> Ciphertext:
    scale = ctx.scale if scale is None else scale
    limbs = ctx.n_q if limbs is None else limbs
    return encrypt_coeffs(ctx, ks, encode_real(ctx.N, slots, scale), scale, limbs, seed, tag, index)


def centered(x: np.ndarray, q: int) -> np.ndarray:
    x = x.astype(object)
    return np.array([int(v) - q if int(v) > q // 2 else int(v) for v in x], dtype=object)


def decrypt_poly(ctx: Context, ks: KeySet, ct: Ciphertext, smudge_sigma: float = 0.0, smudge_seed: int = 0):
    """Collective DDec restricted to q_0 (the plaintext is far below q_0/2):
    c0 + sum_i c1*s_i, each party adding its share; returns the centered
    integer coefficients (int64)."""
    q0 = [ctx.q[0]]
    acc = ct.c[0, :1].copy()
    for i, sp in enumerate(ks.s_parts_ntt):
        share = ctx.mul(ct.c[1, :1], sp[:1], q0)
        if smudge_sigma > 0:
            e = sample_gaussian(Stream(smudge_seed, PURPOSE_SMUDGE, i, 0), ctx.N, smudge_sigma)
            share = ctx.add(share, ctx.ntt(ctx.signed_to_rows(e, q0), q0), q0)
        acc = ctx.add(acc, share, q0)
    coef = ctx.intt(acc, q0)[0].astype(np.int64)
    q = ctx.q[0]
    coef = np.where(coef > q // 2, coef - q, coef)  # q < 2^63 so int64 is safe
    return coef


def dkeyswitch(ctx: Context, ks_from: KeySet, ks_to: KeySet, ct: Ciphertext, seed: int, index: int = 0) -> Ciphertext:
    """DKeySwitch (Fig. 1 item 13), the collective public-key switch (reading
    R20): party i draws u_i (ternary), e0_i, e1_i (Gaussian) and publishes
    h0_i = s_i c1 + u_i b' + e0_i and h1_i = u_i a' + e1_i, with (b', a') the
    target public key; the new ciphertext is (c0 + sum h0_i, sum h1_i).  It
    decrypts under the target secret s' because b' + a' s' is small."""
    prim = ctx.q[: ct.limbs]
    h0 = ct.c[0].copy()
    h1 = np.zeros_like(h0)
    for i, sp in enumerate(ks_from.s_parts_ntt):
        u = sample_ternary(Stream(seed, PURPOSE_PCKS_U, i, index), ctx.N)
        e0 = sample_gaussian(Stream(seed, PURPOSE_PCKS_E0, i, index), ctx.N, ctx.sigma)
        e1 = sample_gaussian(Stream(seed, PURPOSE_PCKS_E1, i, index), ctx.N, ctx.sigma)
        un = ctx.ntt(ctx.signed_to_rows(u, prim), prim)
        e0n = ctx.ntt(ctx.signed_to_rows(e0, prim), prim)
        e1n = ctx.ntt(ctx.signed_to_rows(e1, prim), prim)
        share0 = ctx.add(ctx.add(ctx.mul(sp[: ct.limbs], ct.c[1], prim), ctx.mul(un, ks_to.pk_b[: ct.limbs], prim), prim),
                         e0n, prim)
        share1 = ctx.add(ctx.mul(un, ks_to.pk_a[: ct.limbs], prim), e1n, prim)
        h0 = ctx.add(h0, share0, prim)
        h1 = ctx.add(h1, share1, prim)
    return Ciphertext(np.stack([h0, h1]), ct.scale)


def dbootstrap(ctx: Context, ks: KeySet, ct: Ciphertext, seed: int, counter: int = 0) -> Ciphertext:
    """DBootstrap (Fig. 1 item 14), the collective refresh (reading R17):
    1. party i masks its decryption share at q_0: c1 s_i + M_i + e0_i with M_i
       uniform in [-bound, bound], bound = (floor(q_0/4) - 1) // n_parties
       (sample_uniform_wide, stream (seed, purpose, party, refresh index));
    2. v = centered(c0 + sum of the shares mod q_0) = Delta_ct m + e + sum M_i,
       which stays below q_0/2, is rescaled: m' = round(v Delta / Delta_ct);
    3. against a common reference polynomial a (uniform over Q, NTT form, row r
       from stream (seed, purpose, r, refresh index)),
       party i publishes -s_i a - round(M_i Delta / Delta_ct) + e1_i, and the
       refreshed ciphertext is (m' + sum of those shares, a) at the top level
       and scale Delta."""
    N, q0, prim = ctx.N, ctx.q[0], ctx.q
    n_p = len(ks.s_parts)
    bound = (q0 // 4 - 1) // n_p
    ratio = ctx.scale / ct.scale
    q0l = [q0]
    acc = ctx.intt(ct.c[0, :1], q0l)[0].astype(object)
    w_parts = []
    for i, sp in enumerate(ks.s_parts_ntt):
        M = sample_uniform_wide(Stream(seed, PURPOSE_DB_MASK, i, counter), 2 * bound + 1, N).astype(np.int64) - bound
        e0 = sample_gaussian(Stream(seed, PURPOSE_DB_E0, i, counter), N, ctx.sigma)
        share = ctx.intt(ctx.mul(ct.c[1, :1], sp[:1], q0l), q0l)[0].astype(object)
        acc = (acc + share + (M + e0).astype(object)) % q0
        e1 = sample_gaussian(Stream(seed, PURPOSE_DB_E1, i, counter), N, ctx.sigma)
        w_parts.append(-round_half_away(M.astype(np.float64) * ratio).astype(np.int64) + e1)
    v = np.array([int(x) - q0 if int(x) > q0 // 2 else int(x) for x in acc], dtype=np.int64)
    m_new = round_half_away(v.astype(np.float64) * ratio).astype(np.int64)
    a = np.stack([sample_uniform_wide(Stream(seed, PURPOSE_DB_CRP, r, counter), t, N) for r, t in enumerate(prim)])
    c0 = ctx.ntt(ctx.signed_to_rows(m_new, prim), prim)
    for i, sp in enumerate(ks.s_parts_ntt):
        w = ctx.ntt(ctx.signed_to_rows(w_parts[i], prim), prim)
        c0 = ctx.add(c0, ctx.sub(w, ctx.mul(sp[: ctx.n_q], a, prim), prim), prim)
    return Ciphertext(np.stack([c0, a]), float(ctx.scale))


def decrypt(ctx: Context, ks: KeySet, ct: Ciphertext, n: int | None = None) -> np.ndarray:
    z = decode(ctx.N, decrypt_poly(ctx, ks, ct), ct.scale).real
    return z if n is None else z[:n]


# -- checkpoint files ----------------------------------------------------------
# Layout (little-endian): b"HXCT0001"; u32 log_n, comps, limbs, 0; f64 scale;
# u64 modulus of each limb; u64 residues [comps][limbs][N] in NTT form.

CT_MAGIC = b"HXCT0001"


def save_ciphertext(path: str, ctx: Context, ct: Ciphertext) -> None:
    comps, limbs = ct.c.shape[0], ct.c.shape[1]
    with open(path, "wb") as f:
        f.write(CT_MAGIC)
        f.write(np.array([ctx.log_n, comps, limbs, 0], dtype="<u4").tobytes())
        f.write(np.array([ct.scale], dtype="<f8").tobytes())
        f.write(np.array(ctx.q[:limbs], dtype="<u8").tobytes())
        f.write(np.ascontiguousarray(ct.c, dtype="<u8").tobytes())


def load_ciphertext(path: str, ctx: Context) -> Ciphertext:
    raw = open(path, "rb").read()
    if raw[:8] != CT_MAGIC:
        raise ValueError("not a ciphertext file")
    log_n, comps, limbs, _ = np.frombuffer(raw, dtype="<u4", count=4, offset=8)
    if log_n != ctx.log_n:
        raise ValueError("ring degree differs from the context")
    scale = float(np.frombuffer(raw, dtype="<f8", count=1, offset=24)[0])
    moduli = np.frombuffer(raw, dtype="<u8", count=limbs, offset=32)
    if [int(x) for x in moduli] != list(ctx.q[:limbs]):
        raise ValueError("moduli differ from the context")
    words = int(comps) * int(limbs) * ctx.N
    body = 32 + 8 * int(limbs)
    if len(raw) != body + 8 * words:
        raise ValueError("truncated ciphertext file")
    c = np.frombuffer(raw, dtype="<u8", count=words, offset=body).astype(np.uint64)
    return Ciphertext(c.reshape(int(comps), int(limbs), ctx.N), scale)


# Keyset recipe (little-endian): b"HXKS0001"; u32 log_n, n_q, n_p, n_parties; u64 seed;
# u32 number of Galois keys, primes per digit; u64 moduli of Q then P; u64 Galois elements
# ascending.
# Keys are a deterministic function of (seed, parties, Galois elements).

KS_MAGIC = b"HXKS0001"


def save_keyset(path: str, ctx: Context, ks: KeySet) -> None:
    gal = sorted(ks.rot)
    with open(path, "wb") as f:
        f.write(KS_MAGIC)
        f.write(np.array([ctx.log_n, ctx.n_q, ctx.K, len(ks.s_parts)], dtype="<u4").tobytes())
        f.write(np.array([ks.seed], dtype="<u8").tobytes())
        f.write(np.array([len(gal), ctx.alpha], dtype="<u4").tobytes())
        f.write(np.array(ctx.q + ctx.p, dtype="<u8").tobytes())
        f.write(np.array(gal, dtype="<u8").tobytes())


def load_keyset(path: str, ctx: Context) -> KeySet:
    raw = open(path, "rb").read()
    if raw[:8] != KS_MAGIC:
        raise ValueError("not a keyset file")
    log_n, n_q, n_p, parties = (int(v) for v in np.frombuffer(raw, dtype="<u4", count=4, offset=8))
    seed = int(np.frombuffer(raw, dtype="<u8", count=1, offset=24)[0])
    n_gal, alpha = (int(v) for v in np.frombuffer(raw, dtype="<u4", count=2, offset=32))
    if (log_n, n_q, n_p, alpha) != (ctx.log_n, ctx.n_q, ctx.K, ctx.alpha):
        raise ValueError("keyset of another ring, chain or digit size")
    moduli = [int(v) for v in np.frombuffer(raw, dtype="<u8", count=n_q + n_p, offset=40)]
    if moduli != ctx.q + ctx.p:
        raise ValueError("moduli differ from the context")
    off = 40 + 8 * (n_q + n_p)
    if len(raw) != off + 8 * n_gal:
        raise ValueError("truncated keyset file")
    ks = keygen(ctx, parties, seed)
    for g in (int(v) for v in np.frombuffer(raw, dtype="<u8", count=n_gal, offset=off)):
        ks.rot[g] = gen_switch_key(ctx, ks, g, ctx.automorphism(ks.s_ntt, g))
    return ks


def decrypt_crt(ctx: Context, ks: KeySet, ct: Ciphertext) -> list:
    """Full-modulus decryption with CRT reconstruction in Python integers
    (pins only): centered c0 + c1*s mod q_0...q_{limbs-1}."""
    prim = ctx.q[: ct.limbs]
    x = ctx.add(ct.c[0], ctx.mul(ct.c[1], ks.s_ntt[: ct.limbs], prim), prim)
    coef = ctx.intt(x, prim)
    Q = math.prod(prim)
    out = []
    for i in range(ctx.N):
        v = 0
        for t, qi in enumerate(prim):
            qh = Q // qi
            v += int(coef[t, i]) * qh * pow(qh, -1, qi)
        v %= Q
        out.append(v - Q if v > Q // 2 else v)
    return out


# ----------------------------------------------------------------------------
# Homomorphic evaluation (Fig. 1 items 7-12; readings R6, R10, R11, R12)
# ----------------------------------------------------------------------------

class ScaleError(ValueError):
    pass


class Evaluator:
    """Server-side evaluation on NTT-form ciphertexts.  `counts` records the
    operations in the units of Table I (Add, Mul_pt, Rot, Mul_ct) plus the
    key switches, rescales and hoisted rotations actually performed."""

    SCALE_TOL = 2.0 ** -20

    def __init__(self, ctx: Context, ks: KeySet):
        self.ctx, self.ks = ctx, ks
        self.counts: dict[str, int] = {}

    def _count(self, name: str, n: int = 1) -> None:
        self.counts[name] = self.counts.get(name, 0) + n

    def _prim(self, limbs: int):
        return self.ctx.q[:limbs]

    def _check(self, a: Ciphertext, b: Ciphertext) -> None:
        if a.limbs != b.limbs:
            raise ValueError("level mismatch: %d vs %d limbs" % (a.limbs, b.limbs))
        if abs(a.scale / b.scale - 1.0) > self.SCALE_TOL:
            raise ScaleError("scale mismatch: %r vs %r" % (a.scale, b.scale))

    # -- additive ---------------------------------------------------------------
    def add(self, a: Ciphertext, b: Ciphertext) -> Ciphertext:
        self._check(a, b)
        self._count("Add")
        pr = self._prim(a.limbs)
        return Ciphertext(np.stack([self.ctx.add(a.c[i], b.c[i], pr) for i in range(a.c.shape[0])]), a.scale)

    def sub(self, a: Ciphertext, b: Ciphertext) -> Ciphertext:
        self._check(a, b)
        self._count("Add")
        pr = self._prim(a.limbs)
        return Ciphertext(np.stack([self.ctx.sub(a.c[i], b.c[i], pr) for i in range(a.c.shape[0])]), a.scale)

    def add_const(self, ct: Ciphertext, value: float) -> Ciphertext:
        """Adds the constant polynomial round(value * scale) (every NTT slot of c0)."""
        c = int(round_half_away(np.array([value * ct.scale]))[0])
        pr = self._prim(ct.limbs)
        out = ct.c.copy()
        out[0] = self.ctx.add_scalar(ct.c[0], [c % t for t in pr], pr)
        return Ciphertext(out, ct.scale)

    # -- multiplicative -----------------------------------------------------------
    def mul_plain(self, ct: Ciphertext, pt_ntt: np.ndarray, pt_scale: float) -> Ciphertext:
        """Mul_pt with an NTT-form plaintext of at least ct.limbs limbs."""
        self._count("Mul_pt")
        pr = self._prim(ct.limbs)
        pt = pt_ntt[: ct.limbs]
        return Ciphertext(np.stack([self.ctx.mul(ct.c[i], pt, pr) for i in range(2)]), ct.scale * pt_scale)

    def mul_int(self, ct: Ciphertext, c: int, new_scale: float | None = None) -> Ciphertext:
        """Multiplication by an integer constant (no level consumed)."""
        pr = self._prim(ct.limbs)
        sc = [c % t for t in pr]
        out = np.stack([self.ctx.mul_scalar(ct.c[i], sc, pr) for i in range(ct.c.shape[0])])
        return Ciphertext(out, ct.scale if new_scale is None else new_scale)

    def tensor(self, a: Ciphertext, b: Ciphertext) -> Ciphertext:
        """(a0,a1) x (b0,b1) -> (a0b0, a0b1 + a1b0, a1b1), decrypting under (1, s, s^2)."""
        if a.limbs != b.limbs:
            raise ValueError("level mismatch")
        self._count("Mul_ct")
        pr = self._prim(a.limbs)
        m = self.ctx.mul
        d0 = m(a.c[0], b.c[0], pr)
        d1 = self.ctx.add(m(a.c[0], b.c[1], pr), m(a.c[1], b.c[0], pr), pr)
        d2 = m(a.c[1], b.c[1], pr)
        return Ciphertext(np.stack([d0, d1, d2]), a.scale * b.scale)

    def relinearize(self, d: Ciphertext) -> Ciphertext:
        ks0, ks1 = self.keyswitch(d.c[2], self.ks.relin, d.limbs)
        pr = self._prim(d.limbs)
        return Ciphertext(np.stack([self.ctx.add(d.c[0], ks0, pr), self.ctx.add(d.c[1], ks1, pr)]), d.scale)

    def mul_relin(self, a: Ciphertext, b: Ciphertext) -> Ciphertext:
        return self.relinearize(self.tensor(a, b))

    def relin_rescale(self, d: Ciphertext) -> Ciphertext:
        """Relinearisation followed by RS as one division (reading R21).  With
        acc_c the key inner product of d_2 over Q_l and P (hybrid key switching,
        before ModDown), y_c = acc_c + P d_c is the relinearised component
        times P, an element of Z_{Q_l P}.  Dividing by P q_top with rounding:
        h = floor(P q_top / 2), the remainder r = [y_c + h]_{P q_top} - h is
        taken from the residues of y_c + h at q_top and the special primes by
        basis conversion made exact with the floating-point correction of
        Halevi, Polyakov and Shoup (2019): with z_i = [x_i shat_i^-1]_{s_i}
        the fast conversion sum_i z_i shat_i overshoots by u P q_top,
        u = floor(sum_i z_i / s_i), evaluated in FP64 (products and sums
        rounded to nearest, left to right) and subtracted.  Then
        out_c = (y_c - r) (P q_top)^-1 over q_0 .. q_{l-2}: round(y_c / (P q_top)),
        off by one only where that FP64 sum falls within rounding of an
        integer."""
        if d.limbs < 2:
            raise ValueError("no level left to rescale")
        self._count("KeySwitch")
        self._count("Rescale")
        ctx = self.ctx
        L = d.limbs
        top = L - 1
        qs, lower, qt = ctx.q[:L], ctx.q[:top], ctx.q[top]
        src = [qt] + ctx.p
        Pq = ctx.P * qt
        h = Pq // 2
        a0, a1 = self.inner_product(self.modup(d.c[2], L), self.ks.relin, L)
        out = []
        for acc, dc in ((a0, d.c[0]), (a1, d.c[1])):
            y = ctx.add(acc[:L], ctx.mul_scalar(dc, [ctx.P % t for t in qs], qs), qs)
            z = ctx.intt(np.concatenate([y[top:L], acc[L:]]), src)
            z = ctx.add_scalar(z, [h % t for t in src], src)
            zs = ctx.mul_scalar(z, [pow(Pq // t % t, -1, t) for t in src], src)
            v = np.zeros(ctx.N)
            for i, t in enumerate(src):
                v = v + zs[i].astype(np.float64) * (1.0 / float(t))
            u = np.floor(v).astype(np.uint64)
            r = ctx.basis_convert(z, src, lower)
            for i, t in enumerate(lower):
                tt = np.uint64(t)
                over = (u * np.uint64(Pq % t)) % tt  # u <= K <= 6: no 64-bit overflow for t < 2^61
                r[i] = (r[i] + (tt - over)) % tt
                r[i] = (r[i] + (tt - np.uint64(h % t))) % tt
            r = ctx.ntt(r, lower)
            out.append(ctx.mul_scalar(ctx.sub(y[:top], r, lower), [pow(Pq % t, -1, t) for t in lower], lower))
        return Ciphertext(np.stack(out), d.scale / float(qt))

    # -- levels -----------------------------------------------------------------
    def drop(self, ct: Ciphertext, limbs: int) -> Ciphertext:
        """Discard the top primes (exact; the scale is unchanged)."""
        if limbs > ct.limbs or limbs < 1:
            raise ValueError("bad drop")
        return Ciphertext(ct.c[:, :limbs].copy(), ct.scale)

    def rescale(self, ct: Ciphertext) -> Ciphertext:
        """RS: c' = round(c / q_top) limb-wise (reading R12): with
        x = [c]_{q_top} + floor(q_top/2) taken in [0, q_top), the remainder
        r = x - floor(q_top/2) is removed from every lower limb before the
        multiplication by q_top^-1."""
        if ct.limbs < 2:
            raise ValueError("no level left to rescale")
        self._count("Rescale")
        ctx = self.ctx
        top = ct.limbs - 1
        qt = ctx.q[top]
        half = (qt - 1) // 2
        lower = ctx.q[:top]
        out = np.empty((ct.c.shape[0], top, ctx.N), dtype=np.uint64)
        for comp in range(ct.c.shape[0]):
            x = ctx.intt(ct.c[comp, top:top + 1], [qt])[0]
            x = (x + np.uint64(half)) % np.uint64(qt)
            r = np.empty((top, ctx.N), dtype=np.uint64)
            for i, qi in enumerate(lower):
                r[i] = (x % np.uint64(qi) + np.uint64(qi) - np.uint64(half % qi)) % np.uint64(qi)
            r = ctx.ntt(r, lower)
            diff = ctx.sub(ct.c[comp, :top], r, lower)
            out[comp] = ctx.mul_scalar(diff, [pow(qt, -1, qi) for qi in lower], lower)
        return Ciphertext(out, ct.scale / float(qt))

    # -- hybrid key switching ---------------------------------------------------------
    def modup(self, d: np.ndarray, limbs: int) -> list:
        """ModUp: for every digit j (alpha consecutive primes of Q_l), the digit's
        residues are extended by fast basis conversion to all other primes of
        Q_l and to the special primes.  Returns NTT-form arrays over
        q_0..q_{limbs-1}, p_0..p_{K-1}; on the digit's own primes the input is
        copied unchanged."""
        ctx = self.ctx
        self._count("ModUp")
        coef = ctx.intt(d, ctx.q[:limbs])
        ext = ctx.q[:limbs] + ctx.p
        digits = []
        for j in range(-(-limbs // ctx.alpha)):
            lo, hi = j * ctx.alpha, min((j + 1) * ctx.alpha, limbs)
            src = ctx.q[lo:hi]
            tgt_idx = [i for i in range(len(ext)) if not lo <= i < hi]
            tgt = [ext[i] for i in tgt_idx]
            conv = ctx.ntt(ctx.basis_convert(coef[lo:hi], src, tgt), tgt)
            D = np.empty((len(ext), ctx.N), dtype=np.uint64)
            D[lo:hi] = d[lo:hi]
            D[tgt_idx] = conv
            digits.append(D)
        return digits

    def key_rows(self, limbs: int):
        return list(range(limbs)) + list(range(self.ctx.n_q, self.ctx.n_q + self.ctx.K))

    def inner_product(self, digits: list, key: SwitchKey, limbs: int, galois: int | None = None):
        """sum_j sigma_g(D_j) * swk_j over Q_l and P (both key halves)."""
        ctx = self.ctx
        ext = ctx.q[:limbs] + ctx.p
        rows = self.key_rows(limbs)
        acc0 = np.zeros((len(ext), ctx.N), dtype=np.uint64)
        acc1 = np.zeros_like(acc0)
        for j, D in enumerate(digits):
            Dg = ctx.automorphism(D, galois) if galois is not None else D
            acc0 = ctx.add(acc0, ctx.mul(Dg, key.b[j][rows], ext), ext)
            acc1 = ctx.add(acc1, ctx.mul(Dg, key.a[j][rows], ext), ext)
        return acc0, acc1

    def moddown(self, x: np.ndarray, limbs: int) -> np.ndarray:
        """ModDown: (x - Conv_{P->Q_l}([x]_P)) * P^-1 (reading R11)."""
        ctx = self.ctx
        qs = ctx.q[:limbs]
        xp = ctx.intt(x[limbs:], ctx.p)
        conv = ctx.ntt(ctx.basis_convert(xp, ctx.p, qs), qs)
        return ctx.mul_scalar(ctx.sub(x[:limbs], conv, qs), [pow(ctx.P % t, -1, t) for t in qs], qs)

    def keyswitch(self, d: np.ndarray, key: SwitchKey, limbs: int):
        self._count("KeySwitch")
        digits = self.modup(d, limbs)
        a0, a1 = self.inner_product(digits, key, limbs)
        return self.moddown(a0, limbs), self.moddown(a1, limbs)

    def _rot_key(self, k: int):
        g = galois_element(k, self.ctx.N)
        if g == 1:
            return g, None
        if g not in self.ks.rot:
            add_rotation_key(self.ctx, self.ks, k)
        return g, self.ks.rot[g]

    def rotate(self, ct: Ciphertext, k: int) -> Ciphertext:
        """Rot(ct, k) realising R(m, k) (left rotation by k slots; reading R1):
        the automorphism is applied to (c0, c1), then sigma_g(c1) is switched
        from sigma_g(s) back to s."""
        g, key = self._rot_key(k)
        if key is None:
            return ct.copy()
        self._count("Rot")
        pr = self._prim(ct.limbs)
        c0 = self.ctx.automorphism(ct.c[0], g)
        c1 = self.ctx.automorphism(ct.c[1], g)
        ks0, ks1 = self.keyswitch(c1, key, ct.limbs)
        return Ciphertext(np.stack([self.ctx.add(c0, ks0, pr), ks1]), ct.scale)

    def rotate_sum(self, items) -> Ciphertext:
        """sum_i Rot(ct_i, k_i) with one ModDown for the whole sum: each term's
        key-switch output stays in the extended basis P*Q until the end.  All
        ct_i share level and scale; a term with k = 0 is added unrotated."""
        ctx = self.ctx
        limbs = items[0][0].limbs
        ext = ctx.q[:limbs] + ctx.p
        pr = self._prim(limbs)
        base = [np.zeros((limbs, ctx.N), dtype=np.uint64) for _ in range(2)]
        acc = None
        for ct, k in items:
            g, key = self._rot_key(k)
            if key is None:
                base = [ctx.add(base[i], ct.c[i], pr) for i in range(2)]
                continue
            self._count("Rot")
            self._count("KeySwitch")
            c0 = ctx.automorphism(ct.c[0], g)
            c1 = ctx.automorphism(ct.c[1], g)
            x0, x1 = self.inner_product(self.modup(c1, limbs), key, limbs)
            acc = [x0, x1] if acc is None else [ctx.add(acc[0], x0, ext), ctx.add(acc[1], x1, ext)]
            base[0] = ctx.add(base[0], c0, pr)
        self._count("Add", len(items) - 1)
        if acc is not None:
            base = [ctx.add(base[0], self.moddown(acc[0], limbs), pr), ctx.add(base[1], self.moddown(acc[1], limbs), pr)]
        return Ciphertext(np.stack(base), items[0][0].scale)

    def hoist(self, ct: Ciphertext) -> list:
        """The ModUp of c1 shared by several rotations of ct."""
        return self.modup(ct.c[1], ct.limbs)

    def hoisted_mux(self, ct: Ciphertext, digits: list, k1: int, k2: int, v_ext: np.ndarray, v_scale: float,
                    c: int) -> Ciphertext:
        """v . Rot(ct, k1) + (1 - v) . Rot(ct, k2) from one ModUp (`digits`),
        with the selection applied before ModDown in the extended basis P*Q:
          Z = c*IP_{k2} + v*(IP_{k1} - IP_{k2}),  out = (C0 + MD(Z_0), MD(Z_1)),
          C0 = c*sigma_{k2}(c0) + v*(sigma_{k1}(c0) - sigma_{k2}(c0)),
        where v is the mask encoded at scale `c` = v_scale (rows: Q_l then P) and
        c*x stands for the encoding of 1 at that scale.  The result has scale
        ct.scale * v_scale."""
        ctx = self.ctx
        limbs = ct.limbs
        ext = ctx.q[:limbs] + ctx.p
        pr = self._prim(limbs)
        g1, key1 = self._rot_key(k1)
        g2, key2 = self._rot_key(k2)
        x0, x1 = self.inner_product(digits, key1, limbs, galois=g1)
        y0, y1 = self.inner_product(digits, key2, limbs, galois=g2)
        cs = [c % t for t in ext]
        z = [ctx.add(ctx.mul_scalar(y, cs, ext), ctx.mul(v_ext, ctx.sub(x, y, ext), ext), ext)
             for x, y in ((x0, y0), (x1, y1))]
        m0, m1 = self.moddown(z[0], limbs), self.moddown(z[1], limbs)
        s1 = ctx.automorphism(ct.c[0], g1)
        s2 = ctx.automorphism(ct.c[0], g2)
        c0 = ctx.add(ctx.mul_scalar(s2, cs[:limbs], pr), ctx.mul(v_ext[:limbs], ctx.sub(s1, s2, pr), pr), pr)
        self._count("Rot", 2)
        self._count("RotHoisted", 2)
        self._count("Mul_pt")
        self._count("Add")
        return Ciphertext(np.stack([ctx.add(c0, m0, pr), m1]), ct.scale * v_scale)

    def rotate_hoisted(self, ct: Ciphertext, steps) -> list:
        """Several rotations of one ciphertext sharing a single ModUp of c1
        (reading R10): Rot_k = (sigma_g(c0) + MD(<sigma_g(D), swk_g>_0),
        MD(<sigma_g(D), swk_g>_1))."""
        steps = list(steps)
        pr = self._prim(ct.limbs)
        need = [k for k in steps if galois_element(k, self.ctx.N) != 1]
        digits = self.modup(ct.c[1], ct.limbs) if need else None
        out = []
        for k in steps:
            g, key = self._rot_key(k)
            if key is None:
                out.append(ct.copy())
                continue
            self._count("Rot")
            self._count("RotHoisted")
            a0, a1 = self.inner_product(digits, key, ct.limbs, galois=g)
            ks0, ks1 = self.moddown(a0, ct.limbs), self.moddown(a1, ct.limbs)
            c0 = self.ctx.automorphism(ct.c[0], g)
            out.append(Ciphertext(np.stack([self.ctx.add(c0, ks0, pr), ks1]), ct.scale))
        return out
