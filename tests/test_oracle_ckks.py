"""Pins of the oracle's CKKS layer: encoding against the canonical-embedding
definition, encryption round trips within the noise bound, homomorphic ops
against plaintext arithmetic, rescale against exact integer rounding."""
import math
import struct

import numpy as np
import pytest

from oracle import ckks as C


def test_splitmix64_published_first_outputs():
    # SplitMix64 started from state 0 (Steele, Lea & Flood; Vigna's reference code)
    st, outs = 0, []
    for _ in range(3):
        st = (st + C.GAMMA) & C.M64
        outs.append(C.mix64(st))
    assert outs == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    s = C.Stream(5, 1, 2, 3)
    a = s.draws(4)
    s2 = C.Stream(5, 1, 2, 3)
    b = np.concatenate([s2.draws(1), s2.draws(3)])
    assert np.array_equal(a, b)


def test_samplers():
    n = 1 << 16
    t = C.sample_ternary(C.Stream(1, C.PURPOSE_SK), n)
    assert set(np.unique(t)) == {-1, 0, 1}
    assert all(abs(np.mean(t == v) - 1 / 3) < 0.01 for v in (-1, 0, 1))
    g = C.sample_gaussian(C.Stream(1, C.PURPOSE_PK_E), n, 3.2)
    assert abs(np.std(g) - 3.2) < 0.05 and abs(np.mean(g)) < 0.05 and np.abs(g).max() <= 19
    q = (1 << 45) - 12345
    u = C.sample_uniform(C.Stream(2, C.PURPOSE_KEY_A), q, n)
    assert u.max() < q and abs(np.mean(u.astype(np.float64)) / q - 0.5) < 0.01
    # rejection consumes exactly the draws up to the last accepted one
    s = C.Stream(3, C.PURPOSE_KEY_A)
    C.sample_uniform(s, 11, 100)
    raw = C.Stream(3, C.PURPOSE_KEY_A).draws(s.count) & np.uint64(15)
    assert int((raw < 11).sum()) == 100 and int(raw[-1]) < 11
    # the wide sampler: value j from draws 2j and 2j+1 only; uniform over [0, m)
    m = (1 << 57) + 12345
    w = C.sample_uniform_wide(C.Stream(4, C.PURPOSE_DB_MASK), m, n)
    d = C.Stream(4, C.PURPOSE_DB_MASK).draws(2 * n)
    assert all(int(w[j]) == ((int(d[2 * j]) << 64) + int(d[2 * j + 1])) % m for j in (0, 1, 7, n - 1))
    assert w.max() < m and abs(np.mean(w.astype(np.float64)) / m - 0.5) < 0.01
    small = C.sample_uniform_wide(C.Stream(5, C.PURPOSE_DB_CRP), 7, n)
    assert all(abs(np.mean(small == v) - 1 / 7) < 0.01 for v in range(7))


def exact_encoding(n, z, scale, band=2.0 ** -20):
    """The encoding straight from its definition in 60-digit arithmetic (mpmath): x_i =
    scale * (2/N) * sum_j z_j cos(pi (i e_j mod 2N) / N), rounded half away from zero, a
    value within `band` of a half-integer counted as the half-integer."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    e = [pow(5, j, 2 * n) for j in range(n // 2)]
    cos_t = [mp.cos(mp.pi * t / n) for t in range(2 * n)]
    zs = [(j, mp.mpf(float(v))) for j, v in enumerate(z) if v != 0]
    half, out = mp.mpf(1) / 2, []
    for i in range(n):
        acc = mp.mpf(0)
        for j, v in zs:
            acc += v * cos_t[(i * e[j]) % (2 * n)]
        x = mp.mpf(float(scale)) * 2 * acc / n
        f = mp.floor(x)
        frac = x - f
        if abs(frac - half) <= band:
            r = f + 1 if x > 0 else f
        else:
            r = f + 1 if frac > half else f
        out.append(int(r))
    return np.array(out, dtype=np.int64)


def _encoding_cases(n):
    rng = np.random.default_rng(n)
    s = n // 2
    masks = np.zeros(s)
    masks[rng.choice(s, s // 3, replace=False)] = 1.0
    yield rng.uniform(-1, 1, s), 2.0 ** 30
    yield rng.uniform(-1, 1, s), 2.0 ** 45
    yield rng.uniform(-1, 1, s), float(C.find_primes(int(math.log2(n)), [60])[0])
    yield masks, float(C.find_primes(int(math.log2(n)), [45])[0])
    yield np.repeat(masks[: s // 4], 4), float(C.find_primes(int(math.log2(n)), [40])[0])
    # exact ties: a quarter of the slots set makes x_0 = scale/2, a half-integer for odd scales
    tie = np.zeros(s)
    tie[: n // 4] = 1.0
    yield tie, float(2 ** 45 - 1)
    yield -tie, float(2 ** 45 - 1)


@pytest.mark.parametrize("log_n", [4, 6, 8])
def test_encoding_is_the_exactly_rounded_definition(log_n):
    n = 1 << log_n
    for z, scale in _encoding_cases(n):
        want = exact_encoding(n, z, scale)
        got = C.encode_real(n, z, scale)
        assert np.array_equal(got, want), (log_n, scale, np.flatnonzero(got != want)[:8])


def test_encoding_ties_round_away_from_zero():
    n = 1 << 6
    tie = np.zeros(n // 2)
    tie[: n // 4] = 1.0
    scale = float(2 ** 45 - 1)  # x_0 = scale / 2 exactly
    assert C.encode_real(n, tie, scale)[0] == 2 ** 44
    assert C.encode_real(n, -tie, scale)[0] == -(2 ** 44)
    # one slot at scale 12 on N = 16: x_0 = 12 * (2/16) = 1.5 -> 2, and -1.5 -> -2
    z = np.zeros(8)
    z[0] = 1.0
    assert C.encode_real(16, z, 12.0)[0] == 2 and C.encode_real(16, -z, 12.0)[0] == -2
    # the band: the double-double rounding rule on values near, in and past it
    hi = np.array([2.5, 2.5, 2.5, -2.5, 7.0, 2.0 ** 53])
    lo = np.array([0.0, 2.0 ** -22, 2.0 ** -19, -(2.0 ** -22), 0.4999, 0.75])
    assert list(C.round_dd((hi, lo))) == [3, 3, 3, -3, 7, 2 ** 53 + 1]
    assert list(C.round_dd((np.array([2.5]), np.array([-(2.0 ** -19)])))) == [2]


def test_encoding_fft_matches_direct_double_double_sum():
    """At N = 2^11 the FFT-based encoder equals the O(N^2) sum of the definition, also taken
    in double-double (same roots table, no FFT), coefficient for coefficient."""
    n = 1 << 11
    z = np.random.default_rng(11).uniform(-1, 1, n // 2)
    e = C.slot_exponents(n)
    (cr_h, cr_l), _ = C.roots_dd(4 * n)  # cos(2 pi k / 4N) = cos(pi k / 2N), k < 2N
    cos_h = np.concatenate([cr_h[0::2], -cr_h[0::2]])  # cos(pi t / N), t < 2N
    cos_l = np.concatenate([cr_l[0::2], -cr_l[0::2]])
    i = np.arange(n)
    acc = (np.zeros(n), np.zeros(n))
    for j in range(n // 2):
        t = (i * int(e[j])) % (2 * n)
        acc = C.dd_add(acc, C.dd_mul_double((cos_h[t], cos_l[t]), z[j]))
    m = (acc[0] * (2.0 / n), acc[1] * (2.0 / n))
    for scale in (2.0 ** 45, float(C.find_primes(11, [60])[0])):
        assert np.array_equal(C.scale_round(m, scale), C.encode_real(n, z, scale))


def test_encoding_matches_polynomial_evaluation():
    # evaluating the integer polynomial at zeta^(5^j) (numpy polyval) gives back the slots
    n = 1 << 8
    z = np.random.default_rng(8).uniform(-1, 1, n // 2)
    a = C.encode_real(n, z, 2.0 ** 30)
    zeta = np.exp(1j * np.pi / n)
    for j in range(n // 2):
        x = zeta ** pow(5, j, 2 * n)
        v = np.polyval(a[::-1].astype(np.float64), x) / 2.0 ** 30
        assert abs(v - z[j]) < 2 ** -20
    dec = C.decode(n, a, 2.0 ** 30).real
    assert np.abs(dec - z).max() < 2 ** -20


def test_encode_decode_precision_at_2_40():
    n = 1 << 12
    z = np.random.default_rng(0).uniform(-1, 1, n // 2)
    assert np.abs(C.decode(n, C.encode_real(n, z, 2.0 ** 40), 2.0 ** 40).real - z).max() < 2 ** -30


@pytest.fixture(scope="module")
def small():
    ctx = C.Context(10, [60, 40, 40, 40], [60, 60], 40)
    ks = C.keygen(ctx, 3, 7, rot_steps=[1, 5, -3])
    return ctx, ks


def test_encrypt_decrypt_roundtrip_within_noise_bound(small):
    ctx, ks = small
    z = np.random.default_rng(1).uniform(-1, 1, ctx.S)
    ct = C.encrypt(ctx, ks, z, seed=3)
    # fresh noise v*e + e0 + e1*s: |coeff| <~ 6 sigma (1 + 2 n_parties sqrt(N)); slots add sqrt(N)
    bound = 6 * ctx.sigma * (1 + 2 * 3 * math.sqrt(ctx.N)) * math.sqrt(ctx.N) / ctx.scale
    assert np.abs(C.decrypt(ctx, ks, ct) - z).max() < bound
    # the q_0-only decryption equals the full CRT decryption (the plaintext is far below q_0/2)
    full = C.decrypt_crt(ctx, ks, ct)
    assert [int(v) for v in C.decrypt_poly(ctx, ks, ct)] == full


def test_homomorphic_ops(small):
    ctx, ks = small
    rng = np.random.default_rng(2)
    z, w = rng.uniform(-1, 1, ctx.S), rng.uniform(-1, 1, ctx.S)
    a, b = C.encrypt(ctx, ks, z, 4), C.encrypt(ctx, ks, w, 5)
    ev = C.Evaluator(ctx, ks)
    tol = 2 ** -20
    assert np.abs(C.decrypt(ctx, ks, ev.add(a, b)) - (z + w)).max() < tol
    assert np.abs(C.decrypt(ctx, ks, ev.sub(a, b)) - (z - w)).max() < tol
    m = ev.rescale(ev.mul_relin(a, b))
    assert m.limbs == 3 and np.abs(C.decrypt(ctx, ks, m) - z * w).max() < tol
    for k in (1, 5, -3):
        r = ev.rotate(a, k)
        assert np.abs(C.decrypt(ctx, ks, r) - np.roll(z, -k)).max() < tol
    hs = ev.rotate_hoisted(a, [1, 5, -3, 0])
    for k, r in zip([1, 5, -3, 0], hs):
        assert np.abs(C.decrypt(ctx, ks, r) - np.roll(z, -k)).max() < tol
    pt = C.encode_real(ctx.N, w, float(ctx.q[3]))
    ptn = ctx.ntt(ctx.signed_to_rows(pt, ctx.q), ctx.q)
    mp = ev.rescale(ev.mul_plain(a, ptn, float(ctx.q[3])))
    assert mp.scale == ctx.scale and np.abs(C.decrypt(ctx, ks, mp) - z * w).max() < tol
    assert np.abs(C.decrypt(ctx, ks, ev.add_const(a, 0.25)) - (z + 0.25)).max() < tol
    assert np.abs(C.decrypt(ctx, ks, ev.mul_int(a, -3)) - (-3 * z)).max() < tol


def test_rescale_is_exact_rounded_division(small):
    ctx, ks = small
    ev = C.Evaluator(ctx, ks)
    ct = C.encrypt(ctx, ks, np.ones(4), 9)
    out = ev.rescale(ct)
    Q, Qp = math.prod(ctx.q), math.prod(ctx.q[:3])
    qt = ctx.q[3]
    for comp in range(2):
        X = ctx.intt(ct.c[comp], ctx.q)
        Y = ctx.intt(out.c[comp], ctx.q[:3])
        for c in range(0, ctx.N, 37):
            x = sum(int(X[r, c]) * (Q // t) * pow(Q // t, -1, t) for r, t in enumerate(ctx.q)) % Q
            y = sum(int(Y[r, c]) * (Qp // t) * pow(Qp // t, -1, t) for r, t in enumerate(ctx.q[:3])) % Qp
            assert y == ((x + qt // 2) // qt) % Qp
    assert out.scale == ct.scale / qt


def test_keyswitch_decrypts_to_product_with_target_key(small):
    ctx, ks = small
    ev = C.Evaluator(ctx, ks)
    rng = np.random.default_rng(4)
    limbs = 4
    d = np.stack([rng.integers(0, q, ctx.N, dtype=np.uint64) for q in ctx.q])
    k0, k1 = ev.keyswitch(d, ks.relin, limbs)
    s2 = ctx.mul(ks.s_ntt[:limbs], ks.s_ntt[:limbs], ctx.q)
    lhs = ctx.add(k0, ctx.mul(k1, ks.s_ntt[:limbs], ctx.q), ctx.q)
    rhs = ctx.mul(d, s2, ctx.q)
    diff = ctx.intt(ctx.sub(lhs, rhs, ctx.q), ctx.q)
    # the key-switching error is small: dnum * N * sigma * q_max / P plus the ModDown rounding
    bound = ctx.dnum * ctx.N * 20 * max(ctx.q) // ctx.P + ctx.N * 4
    for r, q in enumerate(ctx.q):
        err = [int(v) if int(v) <= q // 2 else int(v) - q for v in diff[r]]
        assert max(abs(e) for e in err) < bound
        if r:  # one small integer polynomial, seen identically modulo every prime
            assert err == err0
        err0 = err


def test_dkeyswitch_moves_ciphertext_to_target_key(small):
    """DKeySwitch (Fig. 1 item 13): after the collective switch the ciphertext
    decrypts under the target (server) key to the same slots, within the
    added noise u*e' + e0 + e1*s' (summed over 3 parties), and no longer under
    the collective key; level and scale are kept."""
    ctx, ks = small
    server = C.keygen(ctx, 1, 99, relin=False)
    z = np.random.default_rng(5).uniform(-1, 1, ctx.S)
    ct = C.encrypt(ctx, ks, z, seed=8, limbs=3)
    out = C.dkeyswitch(ctx, ks, server, ct, seed=21)
    assert out.limbs == 3 and out.scale == ct.scale
    bound = 3 * 6 * ctx.sigma * (2 + 2 * math.sqrt(ctx.N)) * math.sqrt(ctx.N) / ctx.scale
    assert np.abs(C.decrypt(ctx, server, out) - z).max() < bound + 2 ** -25
    assert np.abs(C.decrypt(ctx, ks, out) - z).max() > 1.0


def test_dbootstrap_refreshes_to_top_level(small):
    """DBootstrap (Fig. 1 item 14): a ciphertext at one limb with scale 2^38
    comes back at the top level with the default scale and the same slots
    (the parties' masks, up to 2^57, cancel: an uncancelled mask would show
    as an error near 2^17); refreshes with another seed or counter differ."""
    ctx, ks = small
    z = np.random.default_rng(6).uniform(-1, 1, ctx.S)
    ct = C.encrypt(ctx, ks, z, seed=9, limbs=1, scale=2.0 ** 38)
    out = C.dbootstrap(ctx, ks, ct, seed=31, counter=0)
    assert out.limbs == ctx.n_q and out.scale == ctx.scale
    assert np.abs(C.decrypt(ctx, ks, out) - z).max() < 2 ** -20
    other = C.dbootstrap(ctx, ks, ct, seed=31, counter=1)
    assert not np.array_equal(other.c, out.c)
    assert np.abs(C.decrypt(ctx, ks, other) - z).max() < 2 ** -20


def test_ciphertext_file_layout_and_round_trip(small, tmp_path):
    ctx, ks = small
    ct = C.encrypt(ctx, ks, [0.25, -1.5, 3.0], seed=9, limbs=3)
    path = str(tmp_path / "ct.bin")
    C.save_ciphertext(path, ctx, ct)
    raw = open(path, "rb").read()
    # the layout written out field by field
    want = b"HXCT0001" + struct.pack("<4I", ctx.log_n, 2, 3, 0) + struct.pack("<d", ct.scale)
    want += struct.pack("<3Q", *ctx.q[:3])
    want += b"".join(struct.pack("<Q", int(x)) for x in ct.c.reshape(-1))
    assert raw == want
    back = C.load_ciphertext(path, ctx)
    assert back.scale == ct.scale and np.array_equal(back.c, ct.c)
    assert np.allclose(C.decrypt(ctx, ks, back, 3), [0.25, -1.5, 3.0], atol=1e-6)
    for bad in (b"HXCT0002" + raw[8:], raw[:-8], raw[:32] + struct.pack("<Q", ctx.q[0] + 2) + raw[40:]):
        open(path, "wb").write(bad)
        with pytest.raises(ValueError):
            C.load_ciphertext(path, ctx)


def _crt(rows, primes):
    Q = math.prod(primes)
    return [sum(int(rows[r, c]) * (Q // t) * pow(Q // t, -1, t) for r, t in enumerate(primes)) % Q
            for c in range(rows.shape[1])]


def test_relin_rescale_is_the_rounded_division_by_p_qtop(small):
    """The fused relinearisation + rescale against exact integers: the
    relinearised component times P is y = acc + P d (acc the key inner product
    before ModDown, whose own pins are above); CRT-reconstructed, each output
    coefficient must be round(y / (P q_top)) (the corrected conversion is exact
    but for an FP64 sum within rounding of an integer: off by one at most), and
    the two-step rescale(relinearize(d)) must agree within 2."""
    ctx, ks = small
    ev = C.Evaluator(ctx, ks)
    rng = np.random.default_rng(12)
    a = C.encrypt(ctx, ks, rng.uniform(-1, 1, ctx.S), 31)
    b = C.encrypt(ctx, ks, rng.uniform(-1, 1, ctx.S), 32)
    d = ev.tensor(a, b)
    L = d.limbs
    out = ev.relin_rescale(d)
    two = ev.rescale(ev.relinearize(d))
    assert out.limbs == L - 1 and out.scale == two.scale
    qs, lower, qt = ctx.q[:L], ctx.q[:L - 1], ctx.q[L - 1]
    Pq = ctx.P * qt
    Ql = math.prod(lower)
    acc = ev.inner_product(ev.modup(d.c[2], L), ks.relin, L)
    for comp in range(2):
        # y over Q_l and P, coefficient form: acc, plus P d_c on the Q rows
        yq = ctx.intt(ctx.add(acc[comp][:L], ctx.mul_scalar(d.c[comp], [ctx.P % t for t in qs], qs), qs), qs)
        yp = ctx.intt(acc[comp][L:], ctx.p)
        Y = _crt(np.concatenate([yq, yp])[:, ::29], qs + ctx.p)
        O = _crt(ctx.intt(out.c[comp], lower)[:, ::29], lower)
        T = _crt(ctx.intt(two.c[comp], lower)[:, ::29], lower)
        exact = 0
        for y, o, t in zip(Y, O, T):
            e = ((y + Pq // 2) // Pq - o) % Ql
            assert min(e, Ql - e) <= 1
            exact += e == 0
            diff = (o - t) % Ql
            assert min(diff, Ql - diff) <= 2
        assert exact == len(Y)
    # 2 per coefficient in c0 and c1 is at most 2 (1 + ||s||_1) per coefficient of the phase,
    # and a slot sums N coefficients
    z = C.decrypt(ctx, ks, out)
    assert np.abs(z - C.decrypt(ctx, ks, two)).max() < ctx.N * 2 * (1 + ctx.N) / out.scale
    assert np.abs(z - C.decrypt(ctx, ks, a) * C.decrypt(ctx, ks, b)).max() < 2 ** -20


def test_keyset_file_layout_and_regeneration(small, tmp_path):
    ctx, ks = small   # 3 parties, seed 7, rotations 1, 5, -3
    path = str(tmp_path / "keys.bin")
    C.save_keyset(path, ctx, ks)
    raw = open(path, "rb").read()
    gal = sorted(ks.rot)
    want = b"HXKS0001" + struct.pack("<4I", ctx.log_n, ctx.n_q, ctx.K, 3) + struct.pack("<Q", 7)
    want += struct.pack("<2I", len(gal), ctx.alpha) + struct.pack("<%dQ" % (ctx.n_q + ctx.K), *(ctx.q + ctx.p))
    want += struct.pack("<%dQ" % len(gal), *gal)
    assert raw == want and len(gal) == 3
    back = C.load_keyset(path, ctx)
    assert np.array_equal(back.s_ntt, ks.s_ntt) and np.array_equal(back.pk_b, ks.pk_b)
    assert np.array_equal(back.relin.b, ks.relin.b) and sorted(back.rot) == gal
    for g in gal:
        assert np.array_equal(back.rot[g].b, ks.rot[g].b) and np.array_equal(back.rot[g].a, ks.rot[g].a)
    for bad in (b"HXKS0002" + raw[8:], raw[:-8], raw[:40] + struct.pack("<Q", ctx.q[0] + 2) + raw[48:]):
        open(path, "wb").write(bad)
        with pytest.raises(ValueError):
            C.load_keyset(path, ctx)


def test_prime_chain_and_rounding_helpers():
    sympy = pytest.importorskip("sympy")
    ctx = C.Context(12, [60, 40, 40, 40], [60, 60], 40)
    primes = ctx.q + ctx.p
    assert len(set(primes)) == len(primes)
    for q, bits in zip(primes, [60, 40, 40, 40, 60, 60]):
        assert sympy.isprime(q) and q % (2 * ctx.N) == 1 and q < 2 ** bits and q > 2 ** (bits - 1)
        for m in range(q - 40, q + 40, 2):  # the oracle's primality test agrees with sympy nearby
            assert C.is_prime(m) == sympy.isprime(m)
    # each is the largest such prime of its size below the previous one of that size (reading R13)
    for q, bits in ((ctx.q[1], 40), (ctx.q[2], 40)):
        m = q + 2 * ctx.N
        while m < 2 ** bits:
            assert not sympy.isprime(m) or m in primes
            m += 2 * ctx.N
    assert list(C.round_half_away(np.array([0.5, -0.5, 1.5, -1.5, 2.49, -2.51]))) == [1, -1, 2, -2, 2, -3]
    for q in ctx.q:
        psi = ctx.psi[q]
        assert pow(psi, 2 * ctx.N, q) == 1 and pow(psi, ctx.N, q) == q - 1


@pytest.mark.parametrize("alpha", [1, 2, 4])
def test_keyswitch_with_digits_of_alpha_primes(alpha):
    """Hybrid key switching with digits of alpha primes (reading R11; alpha above K when the
    digit products stay near P): the switched ciphertext decrypts under the target key within
    the noise bound, and products, rotations and the fused relinearise-rescale stay accurate."""
    ctx = C.Context(10, [60] + [40] * 7, [60] * 3, 40, alpha=alpha)
    assert ctx.dnum == -(-8 // alpha)
    ks = C.keygen(ctx, 2, 11, rot_steps=[1, -4])
    assert ks.relin.b.shape[0] == ctx.dnum
    ev = C.Evaluator(ctx, ks)
    rng = np.random.default_rng(alpha)
    limbs = 7
    d = np.stack([rng.integers(0, q, ctx.N, dtype=np.uint64) for q in ctx.q[:limbs]])
    k0, k1 = ev.keyswitch(d, ks.relin, limbs)
    pr = ctx.q[:limbs]
    s2 = ctx.mul(ks.s_ntt[:limbs], ks.s_ntt[:limbs], pr)
    diff = ctx.intt(ctx.sub(ctx.add(k0, ctx.mul(k1, ks.s_ntt[:limbs], pr), pr), ctx.mul(d, s2, pr), pr), pr)
    # the digit products (up to 2^180 for alpha = 4) against P (about 2^180): noise of a few
    # thousand units against a scale of 2^40
    digit_bits = max(sum(math.log2(q) for q in ctx.q[j * alpha:(j + 1) * alpha]) for j in range(ctx.dnum))
    bound = ctx.dnum * ctx.N * 20 * 2 ** (digit_bits - math.log2(ctx.P)) + ctx.N * 4
    err = [int(v) if int(v) <= ctx.q[0] // 2 else int(v) - ctx.q[0] for v in diff[0]]
    assert max(abs(e) for e in err) < bound
    z, w = rng.uniform(-1, 1, ctx.S), rng.uniform(-1, 1, ctx.S)
    a, b = C.encrypt(ctx, ks, z, 5, limbs=limbs), C.encrypt(ctx, ks, w, 6, limbs=limbs)
    assert np.abs(C.decrypt(ctx, ks, ev.relin_rescale(ev.tensor(a, b))) - z * w).max() < 2 ** -20
    assert np.abs(C.decrypt(ctx, ks, ev.rotate(a, -4)) - np.roll(z, 4)).max() < 2 ** -20
