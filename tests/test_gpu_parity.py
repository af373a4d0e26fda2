"""GPU parity: the CUDA library, called through its C ABI, against the oracle
element by element (bit-exact residues), and decrypted results against FP64."""
import numpy as np
import pytest

from oracle import ckks as C
from oracle import hercules as Hc
from paper_2207_04620_gb300 import hx, workloads

from hxpair import PARAMS, Pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2207_04620_gb300 import build

    build.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def cfg0():
    pr = Pair("cfg0", rot_steps=[1, 3, -5, 64, 200])
    yield pr
    pr.close()


@pytest.fixture(scope="module")
def alg3():
    pr = Pair("alg3", n_parties=3, rot_steps=[1, 7, -2])
    yield pr
    pr.close()


# ---- a1: NTT -----------------------------------------------------------------------

@pytest.mark.parametrize("log_n", [11, 12, 13, 14, 15, 16])
def test_ntt_bit_exact(log_n):
    import torch

    octx = C.Context(log_n, [60, 45, 40], [61], 40)
    ctx = hx.hx_context_create(log_n, [60, 45, 40], [61], 40)
    try:
        primes = octx.q + octx.p
        n_polys = 3
        x = workloads.residues(log_n, primes, n_polys, octx.N)
        want_f = octx.ntt(x, primes * n_polys)
        dev = torch.from_numpy(x.view(np.int64).copy()).cuda()
        hx.hx_ntt(ctx, dev.data_ptr(), n_polys, [0, 1, 2, 3], inverse=False)
        torch.cuda.synchronize()
        got = dev.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want_f)
        hx.hx_ntt(ctx, dev.data_ptr(), n_polys, [0, 1, 2, 3], inverse=True)
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy().view(np.uint64), x)
        # inverse on independent data
        want_i = octx.intt(x, primes * n_polys)
        dev = torch.from_numpy(x.view(np.int64).copy()).cuda()
        hx.hx_ntt(ctx, dev.data_ptr(), n_polys, [0, 1, 2, 3], inverse=True)
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy().view(np.uint64), want_i)
    finally:
        hx.hx_context_destroy(ctx)


def test_ntt_multi_ring_one_launch_bit_exact():
    """Rings of six degrees (2^11 .. 2^16) with uneven limb and polynomial counts
    in one launch per phase: forward and inverse equal the oracle's transform
    of every job."""
    import torch

    specs = [(11, 3, 2), (12, 1, 3), (13, 4, 1), (14, 2, 2), (15, 5, 1), (16, 2, 1)]  # (log_n, limbs, polys)
    ctxs, octxs, xs, devs, jobs = [], [], [], [], []
    try:
        for ln, limbs, polys in specs:
            qb = [60] + [45] * (limbs - 1)
            octx = C.Context(ln, qb, [61], 45)
            ctx = hx.hx_context_create(ln, qb, [61], 45)
            primes = octx.q[:limbs]
            x = workloads.residues(ln + limbs, primes, polys, octx.N)
            dev = torch.from_numpy(x.view(np.int64).copy()).cuda()
            ctxs.append(ctx)
            octxs.append((octx, primes * polys))
            xs.append(x)
            devs.append(dev)
            jobs.append((ctx, dev.data_ptr(), polys, list(range(limbs))))
        hx.hx_ntt_multi(jobs, inverse=False)
        torch.cuda.synchronize()
        for (octx, pr), x, dev in zip(octxs, xs, devs):
            assert np.array_equal(dev.cpu().numpy().view(np.uint64), octx.ntt(x, pr))
        hx.hx_ntt_multi(jobs, inverse=True)
        torch.cuda.synchronize()
        for x, dev in zip(xs, devs):
            assert np.array_equal(dev.cpu().numpy().view(np.uint64), x)
        for (octx, pr), x, dev in zip(octxs, xs, devs):
            dev.copy_(torch.from_numpy(x.view(np.int64).copy()).cuda())
        hx.hx_ntt_multi(jobs, inverse=True)
        torch.cuda.synchronize()
        for (octx, pr), x, dev in zip(octxs, xs, devs):
            assert np.array_equal(dev.cpu().numpy().view(np.uint64), octx.intt(x, pr))
    finally:
        for c in ctxs:
            hx.hx_context_destroy(c)


@pytest.mark.parametrize("log_n", [11, 14, 15, 16])
def test_ntt_every_tile_width_and_autotune(log_n):
    import torch

    octx = C.Context(log_n, [60, 45], [61], 40)
    ctx = hx.hx_context_create(log_n, [60, 45], [61], 40)
    try:
        primes = octx.q + octx.p
        x = workloads.residues(3, primes, 2, octx.N)
        want = octx.ntt(x, primes * 2)
        widths = ([4] * 4, [8] * 4, [16] * 4, [32] * 4, [8, 32, 16, 8], [-4, -8, -16, -32], [-16, 4, 32, -8])
        # an odd log N also runs with the column phase taking the larger half of the stages
        for w, split in [(w, sp) for w in widths for sp in ((0, 1) if log_n & 1 else (0,))]:
            hx.hx_ntt_tiles(ctx, w)
            hx.hx_ntt_split(ctx, split)
            dev = torch.from_numpy(x.view(np.int64).copy()).cuda()
            hx.hx_ntt(ctx, dev.data_ptr(), 2, [0, 1, 2])
            torch.cuda.synchronize()
            assert np.array_equal(dev.cpu().numpy().view(np.uint64), want), (w, split)
            hx.hx_ntt(ctx, dev.data_ptr(), 2, [0, 1, 2], inverse=True)
            torch.cuda.synchronize()
            assert np.array_equal(dev.cpu().numpy().view(np.uint64), x), (w, split)
        chosen = hx.hx_autotune(ctx)
        assert all(abs(c) in (4, 8, 16, 32) for c in chosen) and hx.hx_ntt_tiles(ctx) == chosen
        table = hx.hx_ntt_tuning(ctx)
        assert len(table) == 4 and table[1]["widths"] == chosen
        assert all(t["split"] in ((0, 1) if log_n & 1 else (0,)) for t in table)
        assert [t["max_limbs"] for t in table][:3] == [64, 256, 768]
        # the tuned variants of every bucket give the same residues (a small and a large batch)
        for polys in (2, 200):
            y = workloads.residues(4, primes, polys, octx.N)
            dev = torch.from_numpy(y.view(np.int64).copy()).cuda()
            hx.hx_ntt(ctx, dev.data_ptr(), polys, [0, 1, 2])
            torch.cuda.synchronize()
            got = dev.cpu().numpy().view(np.uint64)
            assert np.array_equal(got[:3], octx.ntt(y[:3], primes)) and np.array_equal(got[-3:], octx.ntt(y[-3:], primes))
    finally:
        hx.hx_context_destroy(ctx)


def test_ntt_edge_cases(cfg0):
    import torch

    # zero polynomials, the maximum residue q-1 everywhere, and an empty batch
    q = cfg0.octx.q
    x = np.stack([np.zeros(cfg0.N, dtype=np.uint64), np.full(cfg0.N, q[1] - 1, dtype=np.uint64)])
    dev = torch.from_numpy(x.view(np.int64).copy()).cuda()
    hx.hx_ntt(cfg0.ctx, dev.data_ptr(), 1, [0, 1])
    hx.hx_ntt(cfg0.ctx, dev.data_ptr(), 0, [0, 1])
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy().view(np.uint64), cfg0.octx.ntt(x, [q[0], q[1]]))
    with pytest.raises(hx.HxError):
        hx.hx_ntt(cfg0.ctx, dev.data_ptr(), 1, [0, 99])


# ---- keys, encryption, decryption --------------------------------------------------

def test_keygen_bit_exact(cfg0):
    o, ctx = cfg0.oks, cfg0.ctx
    pk = hx.hx_keyset_export_public_key(ctx, cfg0.ks, cfg0.octx.n_q)
    assert np.array_equal(pk[0], o.pk_b) and np.array_equal(pk[1], o.pk_a)
    n_all = cfg0.octx.n_q + cfg0.octx.K
    rk = hx.hx_keyset_export_switch_key(ctx, cfg0.ks, 0, cfg0.octx.dnum, n_all)
    assert np.array_equal(rk[:, 0], o.relin.b) and np.array_equal(rk[:, 1], o.relin.a)
    for g, key in o.rot.items():
        k = hx.hx_keyset_export_switch_key(ctx, cfg0.ks, g, cfg0.octx.dnum, n_all)
        assert np.array_equal(k[:, 0], key.b) and np.array_equal(k[:, 1], key.a)


def test_encrypt_and_decrypt_bit_exact(alg3):
    z = workloads.sign_inputs(5, alg3.octx.S)
    m = C.encode_real(alg3.N, z, alg3.octx.scale)
    for limbs, tag, index in ((5, 0, 0), (3, 2, 7)):
        want = C.encrypt_coeffs(alg3.octx, alg3.oks, m, alg3.octx.scale, limbs, 99, tag, index)
        h = hx.hx_encrypt_coeffs(alg3.ctx, alg3.ks, m, alg3.octx.scale, limbs, 99, tag, index)
        assert alg3.same(h, want)
        assert np.array_equal(hx.hx_decrypt_coeffs(alg3.ctx, alg3.ks, h), C.decrypt_poly(alg3.octx, alg3.oks, want))
        hx.hx_ct_destroy(h)


def _encoder_inputs(pr):
    S = pr.octx.S
    rng = np.random.default_rng(S)
    mask = (rng.uniform(0, 1, S) < 0.3).astype(np.float64)
    quarter = np.zeros(S)
    quarter[: pr.N // 4] = 1.0  # coefficient 0 at an odd scale is an exact half-integer
    return [(workloads.sign_inputs(6, S), 2.0 ** 40), (rng.uniform(-1, 1, S), 2.0 ** 45),
            (rng.uniform(-1, 1, S), float(pr.octx.q[0])), (mask, float(pr.octx.q[-1])),
            (quarter, float(2 ** 45 - 1)), (-quarter, float(2 ** 45 - 1)), (rng.uniform(-1, 1, S // 3), 2.0 ** 45)]


@pytest.mark.parametrize("which", ["cfg0", "alg3"])
def test_library_encoders_equal_oracle_encoder(which, cfg0, alg3):
    """Ecd (Fig. 1 item 3): the library's host encoder (hx_encode) and its device
    encoder (hx_encode_batch) give the oracle's coefficients exactly -- both are
    the exactly rounded canonical-embedding sum -- for random slots, masks,
    partial vectors, 40- to 60-bit scales and exact ties."""
    pr = cfg0 if which == "cfg0" else alg3
    cases = _encoder_inputs(pr)
    for z, scale in cases:
        want = C.encode_real(pr.N, z, scale)
        assert np.array_equal(hx.hx_encode(pr.ctx, z, scale), want), scale
        got = hx.hx_encode_batch(pr.ctx, np.stack([z, z]), scale)
        assert np.array_equal(got[0], want) and np.array_equal(got[1], want), scale


def test_library_encryption_equals_oracle_encryption(alg3):
    """Enc(pk, Ecd(z)) (Fig. 1 items 3 and 5) end to end: hx_encrypt (host
    encoder) and hx_encrypt_batch (device encoder and samplers) equal the
    oracle's encryption of the same slots under the same seed, residue for
    residue, at the top level and two levels down."""
    pr = alg3
    z = np.random.default_rng(77).uniform(-1, 1, (4, pr.octx.S))
    for limbs in (pr.octx.n_q, 3):
        outs = hx.hx_encrypt_batch(pr.ctx, pr.ks, z, [500 + i for i in range(4)], limbs=limbs)
        for i in range(4):
            want = C.encrypt(pr.octx, pr.oks, z[i], 500 + i, limbs=limbs)
            assert pr.same(outs[i], want), (limbs, i)
            h = hx.hx_encrypt(pr.ctx, pr.ks, z[i], limbs, 500 + i)
            assert pr.same(h, want), (limbs, i)
            hx.hx_ct_destroy(h)
            hx.hx_ct_destroy(outs[i])


def test_encrypt_decrypt_roundtrip_library(cfg0):
    z = workloads.sign_inputs(7, cfg0.octx.S)
    h = hx.hx_encrypt(cfg0.ctx, cfg0.ks, z, 0, 42)
    # fresh noise v*e + e0 + e1*s: |coeff| < 6 sigma (1 + 2 n_parties sqrt(N)), slots add sqrt(N)
    n = cfg0.N
    bound = 6 * 3.2 * (1 + 2 * cfg0.n_parties * np.sqrt(n)) * np.sqrt(n) / 2.0 ** 40
    assert np.abs(hx.hx_decrypt(cfg0.ctx, cfg0.ks, h) - z).max() < bound
    hx.hx_ct_destroy(h)


# ---- a2-a5: evaluation primitives --------------------------------------------------

def test_evaluation_primitives_bit_exact(alg3):
    pr, octx, ctx = alg3, alg3.octx, alg3.ctx
    ev = C.Evaluator(octx, pr.oks)
    z, w = workloads.sign_inputs(1, octx.S), workloads.sign_inputs(2, octx.S)
    A, B = pr.encrypt(z, 11), pr.encrypt(w, 12)
    a, b = pr.to_lib(A), pr.to_lib(B)
    handles = []

    def chk(h, want):
        handles.append(h)
        assert pr.same(h, want)
        return h

    chk(hx.hx_add(ctx, a, b), ev.add(A, B))
    chk(hx.hx_sub(ctx, a, b), ev.sub(A, B))
    pt = C.encode_real(octx.N, w, float(octx.q[4]))
    ptn = octx.ntt(octx.signed_to_rows(pt, octx.q), octx.q)
    chk(hx.hx_mul_plain(ctx, a, pt, float(octx.q[4])), ev.mul_plain(A, ptn, float(octx.q[4])))
    for c in (3, -7, int(octx.q[2]), -(1 << 40) - 5):
        chk(hx.hx_mul_int(ctx, a, c), ev.mul_int(A, c))
    chk(hx.hx_add_const(ctx, a, -0.375), ev.add_const(A, -0.375))
    T = ev.tensor(A, B)
    t = chk(hx.hx_tensor(ctx, a, b), T)
    R = ev.relinearize(T)
    r = chk(hx.hx_relinearize(ctx, pr.ks, t), R)
    chk(hx.hx_rescale(ctx, r), ev.rescale(R))
    chk(hx.hx_rescale(ctx, t), ev.rescale(T))          # 3-component rescale
    chk(hx.hx_drop(ctx, a, 2), ev.drop(A, 2))
    for k in (1, 7, -2, 0):
        chk(hx.hx_rotate(ctx, pr.ks, a, k), ev.rotate(A, k))
    hs = hx.hx_rotate_hoisted(ctx, pr.ks, a, [1, 7, -2])
    for h_, W in zip(hs, ev.rotate_hoisted(A, [1, 7, -2])):
        chk(h_, W)
    # the same operations one level lower (partial last digit of the gadget)
    A3, a3 = ev.drop(A, 3), hx.hx_drop(ctx, a, 3)
    handles.append(a3)
    chk(hx.hx_rotate(ctx, pr.ks, a3, 7), ev.rotate(A3, 7))
    chk(hx.hx_relinearize(ctx, pr.ks, hx.hx_tensor(ctx, a3, a3)), ev.relinearize(ev.tensor(A3, A3)))
    for h_ in handles + [a, b]:
        hx.hx_ct_destroy(h_)


@pytest.mark.parametrize("name", ["cfg0", "alg3", "sign"])   # K = 1, 2, 3 special primes
def test_relin_rescale_bit_exact(name):
    """Relinearisation + RS in one division (hx_relin_rescale) against the
    oracle at every level of the chain, and against the two-step path in slots."""
    pr = Pair(name)
    try:
        ev = C.Evaluator(pr.octx, pr.oks)
        top = len(pr.p["q_bits"])
        rng = np.random.default_rng(5)
        for limbs in range(top, 1, -1):
            a = pr.encrypt(rng.uniform(-1, 1, 64), 50 + limbs, limbs=limbs)
            b = pr.encrypt(rng.uniform(-1, 1, 64), 60 + limbs, limbs=limbs)
            d = ev.tensor(a, b)
            hd = hx.hx_tensor(pr.ctx, pr.to_lib(a), pr.to_lib(b))
            out = hx.hx_relin_rescale(pr.ctx, pr.ks, hd)
            assert pr.same(out, ev.relin_rescale(d)), limbs
            two = hx.hx_rescale(pr.ctx, hx.hx_relinearize(pr.ctx, pr.ks, hd))
            z, w = hx.hx_decrypt(pr.ctx, pr.ks, out, 64), hx.hx_decrypt(pr.ctx, pr.ks, two, 64)
            assert np.abs(z - w).max() < 2 ** -20
        one = hx.hx_tensor(pr.ctx, *(pr.to_lib(pr.encrypt(np.ones(4), 70 + i, limbs=1)) for i in range(2)))
        with pytest.raises(hx.HxError) as e:
            hx.hx_relin_rescale(pr.ctx, pr.ks, one)
        assert e.value.code == -3
    finally:
        pr.close()


def test_digits_of_four_primes_bit_exact():
    """Key-switching digits of alpha = 4 primes (three special primes, 40-bit chain): keys,
    rotations, relinearisation, the fused relinearise-rescale and one g_4 composition equal
    the oracle's with the same digits, residue for residue."""
    pr = Pair("sign_a4", rot_steps=[1, -3])
    try:
        octx, ev = pr.octx, C.Evaluator(pr.octx, pr.oks)
        assert octx.alpha == 4 and octx.dnum == 4
        n_all = octx.n_q + octx.K
        rk = hx.hx_keyset_export_switch_key(pr.ctx, pr.ks, 0, octx.dnum, n_all)
        assert np.array_equal(rk[:, 0], pr.oks.relin.b) and np.array_equal(rk[:, 1], pr.oks.relin.a)
        for g, key in pr.oks.rot.items():
            k = hx.hx_keyset_export_switch_key(pr.ctx, pr.ks, g, octx.dnum, n_all)
            assert np.array_equal(k[:, 0], key.b) and np.array_equal(k[:, 1], key.a)
        rng = np.random.default_rng(3)
        for limbs in (16, 11, 5):   # 4, 3 and 2 digits, the last ones partial
            A = pr.encrypt(rng.uniform(-1, 1, 64), 10 + limbs, limbs=limbs)
            B = pr.encrypt(rng.uniform(-1, 1, 64), 30 + limbs, limbs=limbs)
            a, b = pr.to_lib(A), pr.to_lib(B)
            assert pr.same(hx.hx_rotate(pr.ctx, pr.ks, a, -3), ev.rotate(A, -3))
            d = hx.hx_tensor(pr.ctx, a, b)
            assert pr.same(hx.hx_relinearize(pr.ctx, pr.ks, d), ev.relinearize(ev.tensor(A, B)))
            assert pr.same(hx.hx_relin_rescale(pr.ctx, pr.ks, d), ev.relin_rescale(ev.tensor(A, B)))
        x = pr.encrypt(workloads.sign_inputs(4, octx.S), 9)
        want = Hc.sign_approx(C.Evaluator(octx, pr.oks), x, 4, 1)
        assert pr.same(hx.hx_sign_approx(pr.ctx, pr.ks, pr.to_lib(x), 4, 1, allow_refresh=False), want)
    finally:
        pr.close()


def test_error_statuses(cfg0):
    ctx = cfg0.ctx
    a = cfg0.to_lib(cfg0.encrypt(np.ones(4), 1))
    with pytest.raises(hx.HxError) as e:
        hx.hx_rotate(ctx, cfg0.ks, a, 2)  # no key for 2
    assert e.value.code == -5
    b = hx.hx_mul_int(ctx, a, 2, new_scale=3.0)
    with pytest.raises(hx.HxError) as e:
        hx.hx_add(ctx, a, b)
    assert e.value.code == -4
    one = hx.hx_drop(ctx, a, 1)
    with pytest.raises(hx.HxError) as e:
        hx.hx_rescale(ctx, one)
    assert e.value.code == -3
    with pytest.raises(hx.HxError) as e:
        hx.hx_matmul(ctx, cfg0.ks, one, one, 16)
    assert e.value.code == -3
    with pytest.raises(hx.HxError):
        hx.hx_matmul_plan_create(ctx, 12, 3)    # h not a power of two
    with pytest.raises(hx.HxError):
        hx.hx_matmul_plan_create(ctx, 1, 3)     # 1x1 blocks are a plain slot product, not HE-MatMult
    # empty and malformed batches are refused before any launch
    for call in (lambda: hx.hx_matmul_batch(ctx, cfg0.ks, 0, [], [], 16),
                 lambda: hx.hx_sign_approx_batch(ctx, cfg0.ks, [], 2, 1),
                 lambda: hx.hx_aggregate(ctx, [], 0, [a], 0.1),
                 lambda: hx.hx_rmatmul_batch(ctx, cfg0.ks, 0, [a], [a], 16, 3),   # t not a power of two
                 lambda: hx.hx_dense_layer(ctx, cfg0.ks, [a], [a], [a], 16, 0, 1, 2, 1, 4.0),  # no output block
                 lambda: hx.hx_encode_batch(ctx, np.ones((1, 1 << 20)), 2.0 ** 40)):  # more slots than N/2
        with pytest.raises(hx.HxError) as e:
            call()
        assert e.value.code == -1
    for h_ in (a, b, one):
        hx.hx_ct_destroy(h_)


def test_checkpoint_files_cross_read(alg3, tmp_path):
    # the oracle writes, the library reads, and the other way round, bit for bit
    pr = alg3
    ct = pr.encrypt(np.linspace(-1, 1, 8), 77, limbs=4)
    p_or, p_lib = str(tmp_path / "oracle.ct"), str(tmp_path / "lib.ct")
    C.save_ciphertext(p_or, pr.octx, ct)
    h = hx.hx_ct_load(pr.ctx, p_or)
    assert pr.same(h, ct)
    r = hx.hx_rotate(pr.ctx, pr.ks, h, 7)
    hx.hx_ct_save(pr.ctx, r, p_lib)
    back = C.load_ciphertext(p_lib, pr.octx)
    assert np.array_equal(back.c, C.Evaluator(pr.octx, pr.oks).rotate(ct, 7).c) and back.scale == ct.scale
    C.save_ciphertext(p_or, pr.octx, back)
    assert open(p_lib, "rb").read() == open(p_or, "rb").read()
    # files of another ring, with a wrong modulus or cut short are refused
    raw = open(p_lib, "rb").read()
    other = C.Context(11, [60, 45], [60], 45)
    C.save_ciphertext(p_or, other, C.Ciphertext(np.zeros((2, 2, 1 << 11), np.uint64), 2.0 ** 45))
    for bad in (None, raw[:-8], raw[:32] + (int(raw[32]) ^ 2).to_bytes(1, "little") + raw[33:], raw + b"\0"):
        if bad is not None:
            open(p_or, "wb").write(bad)
        with pytest.raises(hx.HxError) as e:
            hx.hx_ct_load(pr.ctx, p_or)
        assert e.value.code == -1
    for x in (h, r):
        hx.hx_ct_destroy(x)


def test_keyset_files_cross_read(alg3, tmp_path):
    """Keyset recipe files: the library writes, the oracle regenerates the same keys, and the
    other way round; every rotation key and the public key agree residue for residue."""
    pr = alg3
    octx = pr.octx
    dnum, n_all = octx.dnum, octx.n_q + octx.K
    p_lib, p_or = str(tmp_path / "lib.ks"), str(tmp_path / "oracle.ks")
    hx.hx_keyset_save(pr.ctx, pr.ks, p_lib)
    oks = C.load_keyset(p_lib, octx)
    assert sorted(oks.rot) == sorted(pr.oks.rot)
    for g in oks.rot:
        got = hx.hx_keyset_export_switch_key(pr.ctx, pr.ks, g, dnum, n_all)
        assert np.array_equal(got[:, 0], oks.rot[g].b) and np.array_equal(got[:, 1], oks.rot[g].a)
    C.save_keyset(p_or, octx, pr.oks)
    assert open(p_or, "rb").read() == open(p_lib, "rb").read()
    ks2 = hx.hx_keyset_load(pr.ctx, p_or)
    try:
        pk = hx.hx_keyset_export_public_key(pr.ctx, ks2, octx.n_q)
        assert np.array_equal(pk[0], pr.oks.pk_b) and np.array_equal(pk[1], pr.oks.pk_a)
        for g in pr.oks.rot:
            got = hx.hx_keyset_export_switch_key(pr.ctx, ks2, g, dnum, n_all)
            assert np.array_equal(got[:, 0], pr.oks.rot[g].b)
    finally:
        hx.hx_keyset_destroy(ks2)
    raw = open(p_or, "rb").read()
    for bad in (raw[:-8], raw[:40] + (int(raw[40]) ^ 2).to_bytes(1, "little") + raw[41:], raw + b"\0"):
        open(p_or, "wb").write(bad)
        with pytest.raises(hx.HxError) as e:
            hx.hx_keyset_load(pr.ctx, p_or)
        assert e.value.code == -1


def test_decrypt_needs_every_party(alg3):
    pr = alg3
    z = np.linspace(-2, 2, 16)
    a = pr.to_lib(pr.encrypt(z, 5))
    full = hx.hx_decrypt(pr.ctx, pr.ks, a, 16)
    assert np.array_equal(hx.hx_decrypt_parties(pr.ctx, pr.ks, a, [1] * pr.n_parties, 16), full)
    assert np.allclose(full, z, atol=1e-6)
    for missing in range(pr.n_parties):
        flags = [int(i != missing) for i in range(pr.n_parties)]
        with pytest.raises(hx.HxError) as e:
            hx.hx_decrypt_parties(pr.ctx, pr.ks, a, flags, 16)
        assert e.value.code == -8 and ("party %d" % missing) in str(e.value)
    with pytest.raises(hx.HxError) as e:
        hx.hx_decrypt_parties(pr.ctx, pr.ks, a, [1] * (pr.n_parties - 1), 16)
    assert e.value.code == -1
    hx.hx_ct_destroy(a)


# ---- a6-a7: HE-MatMult ----------------------------------------------------------------

def _matmul_case(name, h, seeds, count):
    p = PARAMS[name]
    limbs = len(p["q_bits"])
    beta = (1 << p["log_n"]) // 2 // (h * h)
    steps = Hc.matmul_rotation_steps(h, beta, limbs)
    pr = Pair(name, rot_steps=steps)
    assert hx.hx_matmul_rotation_steps(pr.ctx, h, limbs) == steps
    return pr, beta, limbs


@pytest.mark.parametrize("name,h", [("cfg0", 16), ("alg3", 8), ("alg3", 32),
                                    ("cfg0", 2), ("alg3", 2), ("alg3", 4)])   # smallest blocks: one baby step
def test_matmul_bit_exact_and_accurate(name, h):
    pr, beta, limbs = _matmul_case(name, h, 0, 2)
    try:
        octx = pr.octx
        masks = Hc.MaskProvider(octx, h, limbs)
        # the library's own masks (its device encoder), never the oracle's: the residues below
        # then also pin the plan's encodings against the oracle's
        plan = hx.hx_matmul_plan_create(pr.ctx, h, limbs)
        assert hx.hx_matmul_plan_num_masks(plan) == len(masks.entries)
        count = 2
        mats_a = [workloads.matrices(10 + i, beta, h) for i in range(count)]
        mats_b = [workloads.matrices(20 + i, beta, h) for i in range(count)]
        A = [pr.encrypt(workloads.pack(m, h, beta), 30 + i) for i, m in enumerate(mats_a)]
        B = [pr.encrypt(workloads.pack(m, h, beta), 40 + i) for i, m in enumerate(mats_b)]
        outs = hx.hx_matmul_batch(pr.ctx, pr.ks, plan, [pr.to_lib(x) for x in A], [pr.to_lib(x) for x in B], h)
        ev = C.Evaluator(octx, pr.oks)
        for i in range(count):
            want = Hc.matmul(ev, A[i], B[i], h, masks)
            assert pr.same(outs[i], want)
            got = workloads.unpack(hx.hx_decrypt(pr.ctx, pr.ks, outs[i]), h, beta)
            err = max(np.abs(g - a @ b).max() for g, a, b in zip(got, mats_a[i], mats_b[i]))
            assert err <= 2 ** -20, err
        hx.hx_matmul_plan_destroy(plan)
    finally:
        pr.close()


@pytest.mark.parametrize("name,h,t", [("cfg0", 16, 4), ("alg3", 8, 2), ("alg3", 16, 1), ("alg3", 16, 8)])
def test_rectangular_matmul_bit_exact(name, h, t):
    """App. D (Alg. "41") through hx_rmatmul_batch: residues equal the oracle's
    HE-RMatMult for both variants (cfg0 runs the depth-2 one) and the result
    decrypts to h/t copies of A.B for every packed pair."""
    p = PARAMS[name]
    limbs = len(p["q_bits"])
    beta = (1 << p["log_n"]) // 2 // (h * h)
    steps = Hc.matmul_rotation_steps(h, beta, limbs, t)
    pr = Pair(name, rot_steps=steps)
    try:
        assert hx.hx_rmatmul_rotation_steps(pr.ctx, h, t, limbs) == steps
        masks = Hc.MaskProvider(pr.octx, h, limbs)
        plan = hx.hx_matmul_plan_create(pr.ctx, h, limbs)
        for i in range(len(masks.entries)):
            hx.hx_matmul_plan_set_mask(pr.ctx, plan, i, masks.coeffs(i))
        rng = np.random.default_rng(h + t)
        As = [[rng.uniform(-1, 1, (t, h)) for _ in range(beta)] for _ in range(2)]
        Bs = [workloads.matrices(60 + i, beta, h) for i in range(2)]
        At = [pr.encrypt(workloads.pack([np.vstack([a] * (h // t)) for a in As[i]], h, beta), 70 + i)
              for i in range(2)]
        Bc = [pr.encrypt(workloads.pack(Bs[i], h, beta), 80 + i) for i in range(2)]
        outs = hx.hx_rmatmul_batch(pr.ctx, pr.ks, plan, [pr.to_lib(c) for c in At], [pr.to_lib(c) for c in Bc], h, t)
        for i in range(2):
            want = Hc.rmatmul(C.Evaluator(pr.octx, pr.oks), At[i], Bc[i], h, t, masks)
            assert pr.same(outs[i], want)
            got = workloads.unpack(hx.hx_decrypt(pr.ctx, pr.ks, outs[i]), h, beta)
            err = max(np.abs(g - np.vstack([a @ b] * (h // t))).max() for g, a, b in zip(got, As[i], Bs[i]))
            assert err < 2 ** -16
            hx.hx_ct_destroy(outs[i])
        hx.hx_matmul_plan_destroy(plan)
    finally:
        pr.close()


def test_rotations_over_three_rings_one_launch_per_stage_bit_exact():
    """hx_rotate_jobs: rotations of ciphertexts of three rings (N = 2^12, 2^13, 2^14), at several
    levels and steps (negative ones and the identity among them), every key-switching stage one
    launch over all of them; each result equals hx_rotate of its job, and one per ring equals
    the oracle's rotation.  A job whose keys lack the Galois key fails the whole call before any
    device work."""
    specs = {"alg3": [(1, 5), (-3, 4), (7, 2), (0, 5)], "alg3_13": [(5, 6), (-1, 3)], "cfg1": [(2, 8), (-6, 5)]}
    pairs = {name: Pair(name, rot_steps=sorted({k for k, _ in js if k})) for name, js in specs.items()}
    try:
        jobs, plain, oracle_rot = [], [], []
        for name, js in specs.items():
            pr = pairs[name]
            for i, (k, limbs) in enumerate(js):
                x = np.random.default_rng(300 + i).uniform(-1, 1, pr.octx.S)
                A = pr.encrypt(x, 310 + i, limbs=limbs)
                h = pr.to_lib(A)
                jobs.append((pr.ctx, pr.ks, h, k))
                plain.append(hx.hx_rotate(pr.ctx, pr.ks, h, k))
                oracle_rot.append(C.Evaluator(pr.octx, pr.oks).rotate(A, k) if i == 0 else None)
        outs = hx.hx_rotate_jobs(jobs)
        for (ctx, ks, h, k), o, p, want in zip(jobs, outs, plain, oracle_rot):
            assert np.array_equal(hx.hx_ct_export(ctx, o), hx.hx_ct_export(ctx, p)), k
            assert hx.hx_ct_info(o) == hx.hx_ct_info(p)
            if want is not None:
                assert np.array_equal(hx.hx_ct_export(ctx, o), want.c)
        for o in outs + plain:
            hx.hx_ct_destroy(o)
        # the third ring's keys hold no key for step 3: the call fails and hands back nothing
        with pytest.raises(hx.HxError):
            hx.hx_rotate_jobs([jobs[0], (pairs["cfg1"].ctx, pairs["cfg1"].ks, jobs[-1][2], 3)])
        for j in jobs:
            hx.hx_ct_destroy(j[2])
    finally:
        for pr in pairs.values():
            pr.close()


def test_products_over_two_rings_in_one_call_bit_exact():
    """hx_matmul_jobs: products of two rings (N = 2^12 and 2^13, chains of 5 and 6 limbs), two
    levels and two matrix sizes in one call, the groups running side by side on the device;
    every entry equals the oracle's HE-MatMult of its pair bit for bit and decrypts to A@B."""
    specs = [("alg3", 8, 5), ("alg3", 16, 4), ("alg3_13", 8, 6), ("alg3_13", 8, 4), ("alg3", 8, 5)]
    pairs = {}
    for name in ("alg3", "alg3_13"):
        S = (1 << PARAMS[name]["log_n"]) // 2
        steps = set()
        for n2, h, limbs in specs:
            if n2 == name:
                steps |= set(Hc.matmul_rotation_steps(h, S // (h * h), limbs))
        pairs[name] = Pair(name, rot_steps=sorted(steps))
    try:
        jobs, want, mats = [], [], []
        for i, (name, h, limbs) in enumerate(specs):
            pr = pairs[name]
            beta = pr.octx.S // (h * h)
            ma, mb = workloads.matrices(90 + i, beta, h), workloads.matrices(95 + i, beta, h)
            A = pr.encrypt(workloads.pack(ma, h, beta), 400 + i, limbs=limbs)
            B = pr.encrypt(workloads.pack(mb, h, beta), 500 + i, limbs=limbs)
            jobs.append((pr.ctx, pr.ks, pr.to_lib(A), pr.to_lib(B), h))
            want.append(Hc.matmul(C.Evaluator(pr.octx, pr.oks), A, B, h, Hc.MaskProvider(pr.octx, h, limbs)))
            mats.append((ma, mb, beta))
        outs = hx.hx_matmul_jobs(jobs)
        for (name, h, limbs), o, w, (ma, mb, beta) in zip(specs, outs, want, mats):
            pr = pairs[name]
            assert pr.same(o, w), (name, h, limbs)
            got = workloads.unpack(hx.hx_decrypt(pr.ctx, pr.ks, o), h, beta)
            assert max(np.abs(g - a @ b).max() for g, a, b in zip(got, ma, mb)) <= 2 ** -18
            hx.hx_ct_destroy(o)
        for j in jobs:
            hx.hx_ct_destroy(j[2])
            hx.hx_ct_destroy(j[3])
    finally:
        for pr in pairs.values():
            pr.close()


def test_products_over_two_rings_error_in_one_group_leaves_the_library_usable():
    """hx_matmul_jobs whose second group (N = 2^13, a key set without rotation keys) fails
    after the first group (N = 2^12) has launched its schedule: the call returns the error,
    hands back no outputs, and the first group's products, run again alone, still equal the
    oracle bit for bit."""
    h, limbs = 8, 5
    good = Pair("alg3", rot_steps=Hc.matmul_rotation_steps(h, (1 << PARAMS["alg3"]["log_n"]) // 2 // (h * h), limbs))
    bad = Pair("alg3_13", rot_steps=[])
    try:
        beta = good.octx.S // (h * h)
        ma, mb = workloads.matrices(70, beta, h), workloads.matrices(71, beta, h)
        A = good.encrypt(workloads.pack(ma, h, beta), 600, limbs=limbs)
        B = good.encrypt(workloads.pack(mb, h, beta), 601, limbs=limbs)
        beta13 = bad.octx.S // (h * h)
        A13 = bad.encrypt(workloads.pack(workloads.matrices(72, beta13, h), h, beta13), 602)
        B13 = bad.encrypt(workloads.pack(workloads.matrices(73, beta13, h), h, beta13), 603)
        ga, gb, ba, bb = good.to_lib(A), good.to_lib(B), bad.to_lib(A13), bad.to_lib(B13)
        with pytest.raises(hx.HxError):
            hx.hx_matmul_jobs([(good.ctx, good.ks, ga, gb, h), (bad.ctx, bad.ks, ba, bb, h)])
        out = hx.hx_matmul_jobs([(good.ctx, good.ks, ga, gb, h)])[0]
        assert good.same(out, Hc.matmul(C.Evaluator(good.octx, good.oks), A, B, h, Hc.MaskProvider(good.octx, h, limbs)))
        for c in (out, ga, gb, ba, bb):
            hx.hx_ct_destroy(c)
    finally:
        good.close()
        bad.close()


def test_matmul_library_masks_end_to_end():
    """The product path: library encryption, library masks, library decryption;
    config 0 (N=2^12, h=16, one product with the other packed slots zero)."""
    pr, beta, limbs = _matmul_case("cfg0", 16, 0, 1)
    try:
        A = workloads.matrices(0, 1, 16)
        B = workloads.matrices(1, 1, 16)
        a = hx.hx_encrypt(pr.ctx, pr.ks, workloads.pack(A, 16, beta), 0, 5)
        b = hx.hx_encrypt(pr.ctx, pr.ks, workloads.pack(B, 16, beta), 0, 6)
        out = hx.hx_matmul(pr.ctx, pr.ks, a, b, 16)
        got = workloads.unpack(hx.hx_decrypt(pr.ctx, pr.ks, out), 16, beta)
        assert np.abs(got[0] - A[0] @ B[0]).max() <= 2 ** -20
        assert all(np.abs(g).max() <= 2 ** -20 for g in got[1:])
    finally:
        pr.close()


def test_matmul_batched_equals_one_at_a_time():
    pr, beta, limbs = _matmul_case("alg3", 8, 0, 3)
    try:
        h = 8
        cts_a = [hx.hx_encrypt(pr.ctx, pr.ks, workloads.pack(workloads.matrices(i, beta, h), h, beta), 0, i)
                 for i in range(3)]
        cts_b = [hx.hx_encrypt(pr.ctx, pr.ks, workloads.pack(workloads.matrices(9 + i, beta, h), h, beta), 0, 9 + i)
                 for i in range(3)]
        batched = hx.hx_matmul_batch(pr.ctx, pr.ks, 0, cts_a, cts_b, h)
        for i in range(3):
            single = hx.hx_matmul(pr.ctx, pr.ks, cts_a[i], cts_b[i], h)
            assert np.array_equal(hx.hx_ct_export(pr.ctx, single), hx.hx_ct_export(pr.ctx, batched[i]))
    finally:
        pr.close()


@pytest.mark.parametrize("h", [8, 16])
def test_transpose_bit_exact(h):
    p = PARAMS["alg3"]
    beta = (1 << p["log_n"]) // 2 // (h * h)
    pr = Pair("alg3", rot_steps=Hc.transpose_rotation_steps(h, beta))
    try:
        assert hx.hx_transpose_rotation_steps(pr.ctx, h) == Hc.transpose_rotation_steps(h, beta)
        masks = Hc.TransposeMasks(pr.octx, h, pr.octx.n_q)
        plan = hx.hx_transpose_plan_create(pr.ctx, h, pr.octx.n_q)
        assert hx.hx_matmul_plan_num_masks(plan) == 2 * h - 1  # library masks, as encoded by the library
        mats = [workloads.matrices(70 + i, beta, h) for i in range(2)]
        cts = [pr.encrypt(workloads.pack(m, h, beta), 80 + i) for i, m in enumerate(mats)]
        outs = hx.hx_transpose(pr.ctx, pr.ks, plan, [pr.to_lib(c) for c in cts], h)
        for i in range(2):
            assert pr.same(outs[i], Hc.transpose(C.Evaluator(pr.octx, pr.oks), cts[i], h, masks))
            got = workloads.unpack(hx.hx_decrypt(pr.ctx, pr.ks, outs[i]), h, beta)
            assert max(np.abs(g - m.T).max() for g, m in zip(got, mats[i])) < 2 ** -20
        hx.hx_matmul_plan_destroy(plan)
    finally:
        pr.close()


def test_dense_layer_bit_exact():
    """Fig. 5, one layer through hx_dense_layer: E, ReLU(E) and dW equal the
    oracle's composition bit for bit (ragged shapes: 30 x 180 weights, 12 input
    blocks in two groups of beta = 8, one refresh per output block), and decrypt
    to the FP64 computation of the same functions."""
    h, d, k, div, seed = 16, 2, 5, 4.0, 31
    p = PARAMS["sign"]
    S = (1 << p["log_n"]) // 2
    beta = S // (h * h)
    pr = Pair("sign", rot_steps=Hc.dense_rotation_steps(h, beta))
    try:
        assert hx.hx_dense_rotation_steps(pr.ctx, h) == Hc.dense_rotation_steps(h, beta)
        W, X, G = workloads.dense_inputs(7, 30, 180, h)
        Wp, Xp, Gp = workloads.dense_pack(W, X, G, h, beta)
        n_out, groups = len(Wp), len(Xp)
        Wc = [[pr.encrypt(Wp[i][g], 500 + 10 * i + g) for g in range(groups)] for i in range(n_out)]
        Xc = [pr.encrypt(Xp[g], 600 + g) for g in range(groups)]
        Gc = [pr.encrypt(Gp[i], 700 + i) for i in range(n_out)]
        top = pr.octx.n_q
        # level of L: E at top-3, E/div one lower, then the compositions with refreshes
        m, dg = top - 4, Hc.g_depth(d)
        for _ in range(k):
            if m - 1 < dg:
                m = top
            m -= dg
        lb = m - 1
        masks = {"fwd": Hc.MaskProvider(pr.octx, h, top), "transpose": Hc.TransposeMasks(pr.octx, h, top),
                 "bwd": Hc.MaskProvider(pr.octx, h, lb)}
        # the context's cached plans with the library's own masks
        E, M, dW = hx.hx_dense_layer(pr.ctx, pr.ks, [pr.to_lib(c) for row in Wc for c in row],
                                     [pr.to_lib(c) for c in Xc], [pr.to_lib(c) for c in Gc], h, n_out, groups, d, k,
                                     div, refresh_seed=seed)
        ev = C.Evaluator(pr.octx, pr.oks)
        oE, oM, odW = Hc.dense_layer(ev, Wc, Xc, Gc, h, d, k, div, seed, masks=masks)
        assert oM[0].limbs == lb
        for i in range(n_out):
            assert pr.same(E[i], oE[i]) and pr.same(M[i], oM[i])
            for g in range(groups):
                assert pr.same(dW[i * groups + g], odW[i][g])
        Wb = workloads.blocks(W, h)
        Xb = [r[0] for r in workloads.blocks(X, h)]
        Gb = [r[0] for r in workloads.blocks(G, h)]
        for i in range(n_out):
            e_ref = sum(a @ b for a, b in zip(Wb[i], Xb))
            s_ref = Hc.g_iter(d, k, e_ref / div)
            l_ref = (1 + s_ref) / 2 * Gb[i]
            e = workloads.unpack(hx.hx_decrypt(pr.ctx, pr.ks, E[i]), h, beta)[0]
            mm = workloads.unpack(hx.hx_decrypt(pr.ctx, pr.ks, M[i]), h, beta)[0]
            assert np.abs(e - e_ref).max() < 2 ** -16
            assert np.abs(mm - e_ref * (1 + s_ref) / 2).max() < 2 ** -14
            for g in range(groups):
                got = workloads.unpack(hx.hx_decrypt(pr.ctx, pr.ks, dW[i * groups + g]), h, beta)
                for q in range(beta):
                    j = beta * g + q
                    want = l_ref @ Xb[j].T if j < len(Xb) else np.zeros((h, h))
                    assert np.abs(got[q] - want).max() < 2 ** -14
    finally:
        pr.close()


@pytest.mark.parametrize("n_parties", [1, 5, 9])
def test_aggregate_bit_exact(alg3, n_parties):
    """Alg. 6 Aggregation through hx_aggregate (the parties' gradients read in
    place; 1, 5 and 9 parties cover the four-party chunks and the tail) equals
    the oracle's Add/level-adjust/Add chain and decrypts to w - c * sum_i g_i."""
    pr = alg3
    count, c = 3, 0.05 / (8 * max(n_parties, 1))
    rng = np.random.default_rng(40 + n_parties)
    w = [rng.uniform(-1, 1, pr.N // 2) for _ in range(count)]
    g = [[rng.uniform(-1, 1, pr.N // 2) for _ in range(count)] for _ in range(n_parties)]
    wc = [pr.encrypt(w[m], 900 + m) for m in range(count)]
    gc = [[pr.encrypt(g[i][m], 1000 + 10 * i + m) for m in range(count)] for i in range(n_parties)]
    outs = hx.hx_aggregate(pr.ctx, [pr.to_lib(x) for row in gc for x in row], n_parties,
                           [pr.to_lib(x) for x in wc], c)
    want = Hc.aggregate(C.Evaluator(pr.octx, pr.oks), gc, wc, c)
    for m in range(count):
        assert pr.same(outs[m], want[m])
        ref = w[m] - c * sum(g[i][m] for i in range(n_parties))
        assert np.abs(hx.hx_decrypt(pr.ctx, pr.ks, outs[m]) - ref).max() < 2 ** -22
        hx.hx_ct_destroy(outs[m])


def test_dkeyswitch_bit_exact(alg3):
    """DKeySwitch (Fig. 1 item 13) from the 3-party key to a 1-party server key:
    residues equal the oracle's protocol, and the result decrypts under the
    server key."""
    pr = alg3
    server = hx.hx_keygen(pr.ctx, 1, 99, [])
    oserver = C.keygen(pr.octx, 1, 99, relin=False)
    try:
        z = np.random.default_rng(12).uniform(-1, 1, pr.N // 2)
        ct = pr.encrypt(z, 77, limbs=3)
        out = hx.hx_dkeyswitch(pr.ctx, pr.ks, server, pr.to_lib(ct), 21)
        assert pr.same(out, C.dkeyswitch(pr.octx, pr.oks, oserver, ct, 21))
        assert np.abs(hx.hx_decrypt(pr.ctx, server, out) - z).max() < 2 ** -25
        hx.hx_ct_destroy(out)
    finally:
        hx.hx_keyset_destroy(server)


def test_dbootstrap_bit_exact(alg3):
    """DBootstrap (Fig. 1 item 14) of a one-limb ciphertext at scale 2^40:
    residues equal the oracle's protocol (masked shares, common reference
    polynomial), the output is at the top level and decrypts to the input."""
    pr = alg3
    z = np.random.default_rng(13).uniform(-1, 1, pr.N // 2)
    ct = C.encrypt(pr.octx, pr.oks, z, 78, limbs=1, scale=2.0 ** 40)
    out = hx.hx_dbootstrap(pr.ctx, pr.ks, pr.to_lib(ct), 31)
    want = C.dbootstrap(pr.octx, pr.oks, ct, 31, 0)
    assert want.limbs == pr.octx.n_q and pr.same(out, want)
    assert np.abs(hx.hx_decrypt(pr.ctx, pr.ks, out) - z).max() < 2 ** -20
    hx.hx_ct_destroy(out)


@pytest.mark.parametrize("n", [None, 1000])
def test_device_encode_and_encrypt_equal_host(alg3, n):
    """The client-side batch on the device (FP64 FFT encoder, SplitMix64
    samplers) gives the host encoder's coefficients and hx_encrypt's
    ciphertexts bit for bit, at the top level and one level down, for full and
    partial slot vectors; oversize coefficients are rejected."""
    pr = alg3
    n = pr.N // 2 if n is None else n
    z = np.random.default_rng(n).uniform(-1, 1, (5, n))
    scale = 2.0 ** 45
    coeffs = hx.hx_encode_batch(pr.ctx, z, scale)
    for i in range(5):
        assert np.array_equal(coeffs[i], hx.hx_encode(pr.ctx, z[i], scale))
    for limbs in (0, 3):
        outs = hx.hx_encrypt_batch(pr.ctx, pr.ks, z, [300 + i for i in range(5)], limbs=limbs)
        for i in range(5):
            ref = hx.hx_encrypt(pr.ctx, pr.ks, z[i], limbs, 300 + i)
            assert np.array_equal(hx.hx_ct_export(pr.ctx, outs[i]), hx.hx_ct_export(pr.ctx, ref))
            hx.hx_ct_destroy(ref)
            hx.hx_ct_destroy(outs[i])
    with pytest.raises(hx.HxError):
        hx.hx_encode_batch(pr.ctx, z * 1e9, 2.0 ** 45)


@pytest.mark.slow
def test_matmul_config1_bit_exact():
    """Config 1 shape: N=2^14, 8 limbs, h=64 (beta=2), one ciphertext pair."""
    pr, beta, limbs = _matmul_case("cfg1", 64, 0, 1)
    try:
        h = 64
        masks = Hc.MaskProvider(pr.octx, h, limbs)
        plan = hx.hx_matmul_plan_create(pr.ctx, h, limbs)  # the library's own masks
        ma, mb = workloads.matrices(1, beta, h), workloads.matrices(2, beta, h)
        A, B = pr.encrypt(workloads.pack(ma, h, beta), 3), pr.encrypt(workloads.pack(mb, h, beta), 4)
        out = hx.hx_matmul_batch(pr.ctx, pr.ks, plan, [pr.to_lib(A)], [pr.to_lib(B)], h)[0]
        want = Hc.matmul(C.Evaluator(pr.octx, pr.oks), A, B, h, masks)
        assert pr.same(out, want)
        got = workloads.unpack(hx.hx_decrypt(pr.ctx, pr.ks, out), h, beta)
        assert max(np.abs(g - a @ b).max() for g, a, b in zip(got, ma, mb)) <= 2 ** -18
    finally:
        pr.close()


@pytest.mark.slow
def test_matmul_config1_full_batch_graph_sampled_bit_exact():
    """Config 1 at full size in the launch configuration the bench times: 16
    ciphertext pairs (32 products of 64x64) through the captured graph with the
    Step-2 keys premasked, the plan built exactly as the bench builds it (the
    library's own masks, no mask set from outside); pairs 0 and 15 equal the
    oracle's HE-MatMult bit for bit and every product decrypts to A@B within
    2^-18."""
    pr, beta, limbs = _matmul_case("cfg1", 64, 0, 1)
    try:
        h, pairs = 64, 16
        masks = Hc.MaskProvider(pr.octx, h, limbs)
        plan = hx.hx_matmul_plan_create(pr.ctx, h, limbs)
        hx.hx_matmul_plan_bind_keys(pr.ctx, plan, pr.ks)
        ma = [workloads.matrices(2 * i, beta, h) for i in range(pairs)]
        mb = [workloads.matrices(2 * i + 1, beta, h) for i in range(pairs)]
        A = [pr.encrypt(workloads.pack(ma[i], h, beta), 10 + i) for i in range(pairs)]
        B = [pr.encrypt(workloads.pack(mb[i], h, beta), 50 + i) for i in range(pairs)]
        ex = hx.hx_matmul_exec_create(pr.ctx, pr.ks, plan, pairs, A[0].scale)
        outs = hx.hx_matmul_exec_run(ex, [pr.to_lib(c) for c in A], [pr.to_lib(c) for c in B])
        for i in (0, pairs - 1):
            assert pr.same(outs[i], Hc.matmul(C.Evaluator(pr.octx, pr.oks), A[i], B[i], h, masks))
        for i in range(pairs):
            got = workloads.unpack(hx.hx_decrypt(pr.ctx, pr.ks, outs[i]), h, beta)
            assert max(np.abs(g - a @ b).max() for g, a, b in zip(got, ma[i], mb[i])) <= 2 ** -18
            hx.hx_ct_destroy(outs[i])
        hx.hx_matmul_exec_destroy(ex)
        hx.hx_matmul_plan_destroy(plan)
    finally:
        pr.close()


@pytest.mark.slow
def test_sign_config2_full_batch_sampled_bit_exact():
    """Config 2 at full size as the bench runs it: 64 ciphertexts of 16384 slots,
    N=2^15, 16 limbs, g_4^(8) with two collective refreshes per entry in one
    batch call; entries 0 and 63 equal the oracle bit for bit and every entry
    decrypts to the FP64 composite within 2^-16."""
    pr = Pair("cfg2")
    try:
        octx, count = pr.octx, 64
        xs = [workloads.sign_inputs(500 + i, octx.S) for i in range(count)]
        cts = [pr.encrypt(x, 900 + i) for i, x in enumerate(xs)]
        outs = hx.hx_sign_approx_batch(pr.ctx, pr.ks, [pr.to_lib(c) for c in cts], 4, 8, allow_refresh=True,
                                       refresh_seed=101)
        for i in (0, count - 1):
            ev = C.Evaluator(octx, pr.oks)
            assert pr.same(outs[i], Hc.sign_approx(ev, cts[i], 4, 8, refresh_seed=101 + i))
            assert ev.counts["Refresh"] == 2
        for i in range(count):
            got = hx.hx_decrypt(pr.ctx, pr.ks, outs[i])
            assert np.abs(got - Hc.g_iter(4, 8, xs[i])).max() < 2 ** -16
            hx.hx_ct_destroy(outs[i])
    finally:
        pr.close()


@pytest.mark.slow
def test_dense_config3_forward_products_full_size_sampled_bit_exact():
    """The forward block products of config 3's dense layer at full size: N=2^15,
    16 limbs (60 + 15 x 40 bit), three 60-bit special primes, h = 64 packed beta = 4
    per ciphertext.  The four products W_{0,g} X_g of the layer's first output block
    (784 inputs = 13 blocks in four groups, the last one ragged) run as one batch
    through the library's own plan at the top level, as the layer's feedforward
    runs them; group 0 equals the oracle's HE-MatMult bit for bit and every product
    decrypts to its block products within 2^-16 (scale 2^40; the oracle's own
    product is about 2^-18.7 off)."""
    cfg = workloads.CONFIGS["cfg3_dense784x128_n15"]
    pr, beta, limbs = _matmul_case("cfg2", cfg["h"], 0, 1)  # the same ring and prime chain
    try:
        h = cfg["h"]
        assert (pr.N, limbs, beta) == (1 << cfg["log_n"], len(cfg["q_bits"]), 4)
        W, X, G = workloads.dense_inputs(3, cfg["rows"], cfg["n_in"], cfg["batch"])
        Wp, Xp, _ = workloads.dense_pack(W, X, G, h, beta)
        groups = len(Xp)
        Wc = [pr.encrypt(Wp[0][g], 1000 + g) for g in range(groups)]
        Xc = [pr.encrypt(Xp[g], 2000 + g) for g in range(groups)]
        plan = hx.hx_matmul_plan_create(pr.ctx, h, limbs)
        outs = hx.hx_matmul_batch(pr.ctx, pr.ks, plan, [pr.to_lib(c) for c in Wc], [pr.to_lib(c) for c in Xc], h)
        want = Hc.matmul(C.Evaluator(pr.octx, pr.oks), Wc[0], Xc[0], h, Hc.MaskProvider(pr.octx, h, limbs))
        assert pr.same(outs[0], want)
        Wb, Xb = workloads.blocks(W, h), [r[0] for r in workloads.blocks(X, h)]
        for g in range(groups):
            got = workloads.unpack(hx.hx_decrypt(pr.ctx, pr.ks, outs[g]), h, beta)
            for p in range(beta):
                j = beta * g + p
                ref = Wb[0][j] @ Xb[j] if j < len(Xb) else np.zeros((h, h))
                assert np.abs(got[p] - ref).max() <= 2 ** -16
            hx.hx_ct_destroy(outs[g])
        hx.hx_matmul_plan_destroy(plan)
    finally:
        pr.close()


@pytest.mark.slow
def test_dense_config3_full_size_against_fp64():
    """Config 3 at full size (784 -> 128, batch 64, h = 64, N = 2^15, 16 limbs) through
    hx_dense_layer with the library's plans: E, ReLU(E) and dW decrypt to the FP64
    computation of the same functions (g_4^(8)(E/4) for the sign)."""
    cfg = workloads.CONFIGS["cfg3_dense784x128_n15"]
    h, d, k, div = cfg["h"], cfg["d"], cfg["k"], cfg["input_div"]
    ctx = hx.hx_context_create(cfg["log_n"], cfg["q_bits"], cfg["p_bits"], cfg["log2_scale"])
    try:
        ks = hx.hx_keygen(ctx, 2, 81, hx.hx_dense_rotation_steps(ctx, h))
        beta = (1 << cfg["log_n"]) // 2 // (h * h)
        W, X, G = workloads.dense_inputs(3, cfg["rows"], cfg["n_in"], cfg["batch"])
        Wp, Xp, Gp = workloads.dense_pack(W, X, G, h, beta)
        n_out, groups = len(Wp), len(Xp)
        assert (n_out, groups) == (2, 4)
        Wc = [hx.hx_encrypt(ctx, ks, Wp[i][g], 0, 1000 + 10 * i + g) for i in range(n_out) for g in range(groups)]
        Xc = [hx.hx_encrypt(ctx, ks, Xp[g], 0, 2000 + g) for g in range(groups)]
        Gc = [hx.hx_encrypt(ctx, ks, Gp[i], 0, 3000 + i) for i in range(n_out)]
        E, M, dW = hx.hx_dense_layer(ctx, ks, Wc, Xc, Gc, h, n_out, groups, d, k, div, refresh_seed=5)
        Wb = workloads.blocks(W, h)
        Xb = [r[0] for r in workloads.blocks(X, h)]
        Gb = [r[0] for r in workloads.blocks(G, h)]
        for i in range(n_out):
            e_ref = sum(a @ b for a, b in zip(Wb[i], Xb))
            s_ref = Hc.g_iter(d, k, e_ref / div)
            l_ref = (1 + s_ref) / 2 * Gb[i]
            e = workloads.unpack(hx.hx_decrypt(ctx, ks, E[i]), h, beta)[0]
            m = workloads.unpack(hx.hx_decrypt(ctx, ks, M[i]), h, beta)[0]
            assert np.abs(e - e_ref).max() < 2 ** -12
            assert np.abs(m - e_ref * (1 + s_ref) / 2).max() < 2 ** -12
            for g in range(groups):
                got = workloads.unpack(hx.hx_decrypt(ctx, ks, dW[i * groups + g]), h, beta)
                for q in range(beta):
                    j = beta * g + q
                    want = l_ref @ Xb[j].T if j < len(Xb) else np.zeros((h, h))
                    assert np.abs(got[q] - want).max() < 2 ** -9
        for c in E + M + dW + Wc + Xc + Gc:
            hx.hx_ct_destroy(c)
        hx.hx_keyset_destroy(ks)
    finally:
        hx.hx_context_destroy(ctx)


@pytest.mark.slow
def test_matmul_largest_h_at_n15_against_fp64():
    """The largest product a 2^15 ring packs: h = 128 (beta = 1, every slot used), Alg. 3
    at 5 limbs with the library's masks; the decryption equals A@B (128-term dot products)."""
    h, ln = 128, 15
    qb = [60, 45, 45, 45, 45]
    ctx = hx.hx_context_create(ln, qb, [60, 60], 45)
    try:
        ks = hx.hx_keygen(ctx, 2, 9, hx.hx_matmul_rotation_steps(ctx, h, len(qb)))
        a, b = workloads.matrices(71, 1, h)[0], workloads.matrices(72, 1, h)[0]
        A = hx.hx_encrypt(ctx, ks, workloads.pack([a], h, 1), 0, 1)
        B = hx.hx_encrypt(ctx, ks, workloads.pack([b], h, 1), 0, 2)
        out = hx.hx_matmul(ctx, ks, A, B, h)
        assert hx.hx_ct_info(out)[1] == len(qb) - 3
        got = workloads.unpack(hx.hx_decrypt(ctx, ks, out), h, 1)[0]
        assert np.abs(got - a @ b).max() < 2 ** -14
        for c in (A, B, out):
            hx.hx_ct_destroy(c)
        hx.hx_keyset_destroy(ks)
    finally:
        hx.hx_context_destroy(ctx)


# ---- a8: composite sign and ReLU ------------------------------------------------------

@pytest.mark.parametrize("relu", [False, True])
def test_sign_bit_exact_with_refresh(relu):
    pr = Pair("sign")
    try:
        octx = pr.octx
        xs = [workloads.sign_inputs(50 + i, octx.S) for i in range(2)]
        cts = [pr.encrypt(x, 60 + i) for i, x in enumerate(xs)]
        outs = hx.hx_sign_approx_batch(pr.ctx, pr.ks, [pr.to_lib(c) for c in cts], 4, 8, relu=relu,
                                       allow_refresh=True, refresh_seed=777)
        for i in range(2):
            ev = C.Evaluator(octx, pr.oks)
            want = Hc.sign_approx(ev, cts[i], 4, 8, relu=relu, refresh_seed=777 + i)
            assert ev.counts["Refresh"] == 2
            assert pr.same(outs[i], want)
            got = hx.hx_decrypt(pr.ctx, pr.ks, outs[i])
            ref = Hc.g_iter(4, 8, xs[i])
            ref = xs[i] * (1 + ref) / 2 if relu else ref
            assert np.abs(got - ref).max() < 2 ** -18
        with pytest.raises(hx.HxError) as e:
            hx.hx_sign_approx(pr.ctx, pr.ks, pr.to_lib(cts[0]), 4, 8, allow_refresh=False)
        assert e.value.code == -3
    finally:
        pr.close()


def test_sign_degrees_1_to_4_single_composition():
    pr = Pair("sign")
    try:
        x = workloads.sign_inputs(3, pr.octx.S)
        ct = pr.encrypt(x, 4)
        for d in (1, 2, 3, 4):
            ev = C.Evaluator(pr.octx, pr.oks)
            want = Hc.sign_approx(ev, ct, d, 1)
            h = hx.hx_sign_approx(pr.ctx, pr.ks, pr.to_lib(ct), d, 1, allow_refresh=False)
            assert pr.same(h, want)
    finally:
        pr.close()


def test_matmul_graph_executor_equals_batched_call():
    pr, beta, limbs = _matmul_case("alg3", 8, 0, 2)
    try:
        h = 8
        A = [hx.hx_encrypt(pr.ctx, pr.ks, workloads.pack(workloads.matrices(i, beta, h), h, beta), 0, i)
             for i in range(2)]
        B = [hx.hx_encrypt(pr.ctx, pr.ks, workloads.pack(workloads.matrices(5 + i, beta, h), h, beta), 0, 5 + i)
             for i in range(2)]
        plan = hx.hx_matmul_plan_create(pr.ctx, h, limbs)
        want = [hx.hx_ct_export(pr.ctx, o) for o in hx.hx_matmul_batch(pr.ctx, pr.ks, plan, A, B, h)]
        scale = hx.hx_ct_info(A[0])[2]
        ex = hx.hx_matmul_exec_create(pr.ctx, pr.ks, plan, 2, scale)
        assert hx.hx_matmul_exec_launches(ex) > 100
        for _ in range(2):  # replays reuse the graph's memory
            got = hx.hx_matmul_exec_run(ex, A, B)
            for g, w in zip(got, want):
                assert np.array_equal(hx.hx_ct_export(pr.ctx, g), w)
                hx.hx_ct_destroy(g)
        # the host-buffer replay: page-locked inputs in, products out, same residues
        import torch

        host_a = torch.from_numpy(np.stack([hx.hx_ct_export(pr.ctx, x) for x in A]).view(np.int64)).pin_memory()
        host_b = torch.from_numpy(np.stack([hx.hx_ct_export(pr.ctx, x) for x in B]).view(np.int64)).pin_memory()
        out_limbs, out_scale = hx.hx_matmul_exec_out_info(ex)
        assert out_limbs == want[0].shape[1]
        host_out = torch.zeros((2, 2, out_limbs, pr.N), dtype=torch.int64).pin_memory()
        stream = torch.cuda.Stream()
        hx.hx_matmul_exec_run_host(ex, host_a.data_ptr(), host_b.data_ptr(), host_out.data_ptr(), stream=stream)
        stream.synchronize()
        for i in range(2):
            assert np.array_equal(host_out[i].numpy().view(np.uint64), want[i])
        hx.hx_matmul_exec_destroy(ex)
        # keys premasked with the plan's Step 2 selection: the same residues
        hx.hx_matmul_plan_bind_keys(pr.ctx, plan, pr.ks)
        assert hx.hx_matmul_plan_bound_bytes(plan) > 0
        for g, w in zip(hx.hx_matmul_batch(pr.ctx, pr.ks, plan, A, B, h), want):
            assert np.array_equal(hx.hx_ct_export(pr.ctx, g), w)
            hx.hx_ct_destroy(g)
        hx.hx_matmul_plan_destroy(plan)
    finally:
        pr.close()
