"""Pins of the oracle's ring arithmetic against definitions computed
independently (pure Python integers, sympy), not against the oracle itself."""
import math
import random

import numpy as np
import pytest
import sympy

from oracle import ckks as C


def py_negacyclic(a, b, q):
    n = len(a)
    out = [0] * n
    for i in range(n):
        for j in range(n):
            k = i + j
            if k < n:
                out[k] = (out[k] + a[i] * b[j]) % q
            else:
                out[k - n] = (out[k - n] - a[i] * b[j]) % q
    return out


@pytest.mark.parametrize("log_n,bits", [(4, [50, 40]), (10, [60, 40, 40]), (12, [60, 40, 40, 60]),
                                        (14, [60] + [45] * 7 + [60, 60])])
def test_primes_are_the_largest_ntt_friendly_primes(log_n, bits):
    qs = C.find_primes(log_n, bits)
    two_n = 2 << log_n
    assert len(set(qs)) == len(qs)
    for q, b in zip(qs, bits):
        assert sympy.isprime(q) and q % two_n == 1 and q < (1 << b) and q.bit_length() == b
    # nothing larger and still unused was skipped
    for idx, (q, b) in enumerate(zip(qs, bits)):
        c = (1 << b) - two_n + 1
        while c > q:
            assert not sympy.isprime(c) or c in qs[:idx]
            c -= two_n


def test_psi_is_primitive_2n_th_root():
    for log_n in (3, 10, 14, 16):
        n = 1 << log_n
        for q in C.find_primes(log_n, [60, 45, 40]):
            psi = C.find_psi(q, n)
            assert pow(psi, n, q) == q - 1 and pow(psi, 2 * n, q) == 1


@pytest.mark.parametrize("log_n", [1, 2, 3, 5, 8])
def test_fast_ntt_equals_definition(log_n):
    n = 1 << log_n
    rng = random.Random(log_n)
    for q in C.find_primes(log_n, [60, 40]):
        psi = C.find_psi(q, n)
        a = [rng.randrange(q) for _ in range(n)]
        # definition evaluated with Python integers
        want = []
        for j in range(n):
            x = pow(psi, 2 * C.brv(j, log_n) + 1, q)
            want.append(sum(a[i] * pow(x, i, q) for i in range(n)) % q)
        ctx_rows = np.array([a], dtype=np.uint64)
        C.lib().ref_ntt_forward_rows(ctx_rows, 1, log_n, C._u64([q]), C._u64([psi]))
        assert [int(v) for v in ctx_rows[0]] == want
        direct = np.zeros(n, dtype=np.uint64)
        C.lib().ref_ntt_direct(direct, np.array(a, dtype=np.uint64), log_n, q, psi)
        assert [int(v) for v in direct] == want


@pytest.mark.parametrize("log_n", [4, 7])
def test_ntt_product_equals_schoolbook(log_n):
    ctx = C.Context(log_n, [60, 40], [50], 30)
    rng = random.Random(7)
    for q in ctx.q + ctx.p:
        a = [rng.randrange(q) for _ in range(ctx.N)]
        b = [rng.randrange(q) for _ in range(ctx.N)]
        fa = ctx.ntt(np.array([a], dtype=np.uint64), [q])
        fb = ctx.ntt(np.array([b], dtype=np.uint64), [q])
        prod = ctx.intt(ctx.mul(fa, fb, [q]), [q])[0]
        assert [int(v) for v in prod] == py_negacyclic(a, b, q)


def test_inverse_ntt_roundtrip_large():
    ctx = C.Context(14, [60, 45], [60], 45)
    rng = np.random.default_rng(0)
    x = np.stack([rng.integers(0, q, ctx.N, dtype=np.uint64) for q in ctx.q + ctx.p])
    y = ctx.intt(ctx.ntt(x, ctx.q + ctx.p), ctx.q + ctx.p)
    assert np.array_equal(x, y)


def test_automorphism_ntt_matches_coefficient_definition_and_composes():
    log_n = 6
    ctx = C.Context(log_n, [50], [50], 30)
    q = ctx.q[0]
    rng = random.Random(3)
    a = [rng.randrange(q) for _ in range(ctx.N)]
    for g in (5, 25, 3, 2 * ctx.N - 1):
        # definition: a(X^g) reduced mod X^N + 1, with Python integers
        want = [0] * ctx.N
        for i, c in enumerate(a):
            e = i * g % (2 * ctx.N)
            if e < ctx.N:
                want[e] = (want[e] + c) % q
            else:
                want[e - ctx.N] = (want[e - ctx.N] - c) % q
        fa = ctx.ntt(np.array([a], dtype=np.uint64), [q])
        got = ctx.intt(ctx.automorphism(fa, g), [q])[0]
        assert [int(v) for v in got] == want
    fa = ctx.ntt(np.array([a], dtype=np.uint64), [q])
    g1, g2 = 5, 125
    assert np.array_equal(ctx.automorphism(ctx.automorphism(fa, g1), g2),
                          ctx.automorphism(fa, g1 * g2 % (2 * ctx.N)))
    # rotation by S slots is the identity element
    assert C.galois_element(ctx.S, ctx.N) == 1


def test_basis_conversion_is_exact_up_to_multiple_of_source_modulus():
    ctx = C.Context(5, [60, 45, 45, 45], [60, 60], 40)
    src, dst = ctx.q[1:4], [ctx.q[0]] + ctx.p
    Q = math.prod(src)
    rng = random.Random(11)
    xs = [rng.randrange(Q) for _ in range(ctx.N)]
    x = np.array([[v % t for v in xs] for t in src], dtype=np.uint64)
    out = ctx.basis_convert(x, src, dst)
    for c, v in enumerate(xs):
        us = set()
        for r, t in enumerate(dst):
            # out = v + u*Q (mod t) with 0 <= u < len(src)
            cand = [u for u in range(len(src)) if (v + u * Q) % t == int(out[r, c])]
            assert cand, "not of the form v + uQ"
            us.add(cand[0])
        assert len(us) == 1


def test_moddown_exact_on_multiples_of_P():
    ctx = C.Context(5, [60, 45, 45], [60, 60], 40)
    ks = C.keygen(ctx, 1, 1, relin=False)
    ev = C.Evaluator(ctx, ks)
    rng = random.Random(5)
    limbs = 3
    ys = [rng.randrange(math.prod(ctx.q)) for _ in range(ctx.N)]
    ext = ctx.q + ctx.p
    x = np.array([[(y * ctx.P) % t for y in ys] for t in ext], dtype=np.uint64)
    xn = ctx.ntt(x, ext)
    got = ctx.intt(ev.moddown(xn, limbs), ctx.q)
    assert all(int(got[r, c]) == ys[c] % ctx.q[r] for r in range(limbs) for c in range(ctx.N))
