"""Continuous-batching server: every result equals the same request computed
alone, requests are batched and overlap across lanes, admission respects the
HBM budget, and queued requests past their deadline complete with HX_ETIMEOUT."""
import numpy as np
import pytest

from oracle import hercules as Hc
from paper_2207_04620_gb300 import hx, workloads

from hxpair import PARAMS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2207_04620_gb300 import build

    build.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = PARAMS["alg3"]
    ctx = hx.hx_context_create(p["log_n"], p["q_bits"], p["p_bits"], p["log2_scale"])
    s = (1 << p["log_n"]) // 2
    steps = sorted(set(Hc.matmul_rotation_steps(8, s // 64, 5)) | set(Hc.matmul_rotation_steps(16, s // 256, 5)))
    ks = hx.hx_keygen(ctx, 2, 31, steps)
    yield ctx, ks, s
    hx.hx_keyset_destroy(ks)
    hx.hx_context_destroy(ctx)


def _requests(ctx, ks, s):
    """(kind, args) of a mixed stream: matmuls of h = 8 and 16 at 5 and 4 limbs, signs of d = 2 and 4."""
    reqs = []
    for i in range(10):
        if i % 3 == 2:
            d = 4 if i % 2 else 2
            x = hx.hx_encrypt(ctx, ks, workloads.sign_inputs(i, s), 5, 100 + i)
            reqs.append(("sign", (x, d, 1, 1000 + i)))
        else:
            h = 8 if i % 2 else 16
            beta = s // (h * h)
            limbs = 5 if i % 4 < 2 else 4
            a = hx.hx_encrypt(ctx, ks, workloads.pack(workloads.matrices(i, beta, h), h, beta), limbs, 200 + i)
            b = hx.hx_encrypt(ctx, ks, workloads.pack(workloads.matrices(50 + i, beta, h), h, beta), limbs, 300 + i)
            reqs.append(("matmul", (a, b, h)))
    return reqs


def _submit(sv, ctx, ks, kind, args):
    if kind == "matmul":
        return hx.hx_server_submit_matmul(sv, ctx, ks, *args)
    if kind == "rotate":
        return hx.hx_server_submit_rotate(sv, ctx, ks, *args)
    x, d, k, seed = args
    return hx.hx_server_submit_sign(sv, ctx, ks, x, d, k, relu=False, refresh_seed=seed)


def _alone(ctx, ks, kind, args):
    if kind == "matmul":
        return hx.hx_matmul(ctx, ks, *args)
    if kind == "rotate":
        return hx.hx_rotate(ctx, ks, *args)
    x, d, k, seed = args
    return hx.hx_sign_approx(ctx, ks, x, d, k, relu=False, allow_refresh=True, refresh_seed=seed)


def _collect(sv, n):
    got = {}
    while len(got) < n:
        for rid, res, st, lat in hx.hx_server_poll(sv, wait=True):
            got[rid] = (res, st, lat)
    return got


def test_results_in_the_mix_equal_results_alone(setup):
    ctx, ks, s = setup
    reqs = _requests(ctx, ks, s)
    sv = hx.hx_server_create(64 << 30, 3, 4)
    hx.hx_server_register_keys(sv, ks)
    ids = [_submit(sv, ctx, ks, kind, args) for kind, args in reqs]
    got = _collect(sv, len(ids))
    stats = hx.hx_server_stats(sv)
    hx.hx_server_destroy(sv)
    assert stats["completed"] == len(reqs) and stats["batches"] < len(reqs)  # some requests shared a batch
    for rid, (kind, args) in zip(ids, reqs):
        res, st, lat = got[rid]
        assert st == 0 and lat > 0
        alone = _alone(ctx, ks, kind, args)
        assert np.array_equal(hx.hx_ct_export(ctx, res), hx.hx_ct_export(ctx, alone)), kind
        hx.hx_ct_destroy(res)
        hx.hx_ct_destroy(alone)


def test_admission_by_budget_and_rejection(setup):
    ctx, ks, s = setup
    h, beta = 8, s // 64
    a = hx.hx_encrypt(ctx, ks, workloads.pack(workloads.matrices(1, beta, h), h, beta), 5, 1)
    b = hx.hx_encrypt(ctx, ks, workloads.pack(workloads.matrices(2, beta, h), h, beta), 5, 2)
    one = 48 * 2 * 5 * (2 * s) * 8          # the server's estimate for one such product
    sv = hx.hx_server_create(one + one // 2, 3, 8)   # room for exactly one at a time
    ids = [hx.hx_server_submit_matmul(sv, ctx, ks, a, b, h) for _ in range(4)]
    hx.hx_ct_destroy(a)                      # the server keeps its own reference
    hx.hx_ct_destroy(b)
    got = _collect(sv, 4)
    stats = hx.hx_server_stats(sv)
    assert all(got[i][1] == 0 for i in ids)
    assert stats["max_busy_lanes"] == 1 and stats["peak_admitted_bytes"] <= one + one // 2
    outs = [hx.hx_ct_export(ctx, got[i][0]) for i in ids]
    assert all(np.array_equal(o, outs[0]) for o in outs)
    hx.hx_server_destroy(sv)
    tiny = hx.hx_server_create(one // 2, 1, 1)
    c = hx.hx_encrypt(ctx, ks, np.ones(4), 5, 3)
    with pytest.raises(hx.HxError) as e:
        hx.hx_server_submit_matmul(tiny, ctx, ks, c, c, h)
    assert e.value.code == -2
    hx.hx_server_destroy(tiny)


def test_deadline_expires_queued_requests_only(setup):
    ctx, ks, s = setup
    h, beta = 8, s // 64
    a = hx.hx_encrypt(ctx, ks, workloads.pack(workloads.matrices(3, beta, h), h, beta), 5, 4)
    b = hx.hx_encrypt(ctx, ks, workloads.pack(workloads.matrices(4, beta, h), h, beta), 5, 5)
    sv = hx.hx_server_create(64 << 30, 2, 4)
    hx.hx_server_pause(sv, True)            # hold the queue so the deadlines below act on queued requests
    late = hx.hx_server_submit_matmul(sv, ctx, ks, a, b, h)
    kept = hx.hx_server_submit_matmul(sv, ctx, ks, a, b, h)
    hx.hx_server_set_deadline(sv, late, 0.0)
    hx.hx_server_set_deadline(sv, kept, 60e3)
    first = hx.hx_server_poll(sv, wait=True)  # the expiry wakes the poll while the queue is still held
    assert [(rid, res, st) for rid, res, st, _ in first] == [(late, None, -6)]
    assert hx.hx_server_stats(sv)["pending"] == 1
    hx.hx_server_pause(sv, False)
    got = _collect(sv, 1)
    assert got[kept][1] == 0
    alone = hx.hx_matmul(ctx, ks, a, b, h)
    assert np.array_equal(hx.hx_ct_export(ctx, got[kept][0]), hx.hx_ct_export(ctx, alone))
    with pytest.raises(hx.HxError) as e:     # no longer queued
        hx.hx_server_set_deadline(sv, kept, 1.0)
    assert e.value.code == -1
    stats = hx.hx_server_stats(sv)
    assert stats["expired"] == 1 and stats["completed"] == 2
    hx.hx_server_destroy(sv)
    for x in (a, b, alone, got[kept][0]):
        hx.hx_ct_destroy(x)


def test_plan_cache_cap_frees_unused_plans(setup):
    """The cache holds one plan per matrix size (a lower level's plan is a view of the
    top level's: the masks do not depend on the level).  With a 1-byte cap every cached
    plan but the one in use is freed after each call; products stay identical to the
    uncapped ones, also through the server."""
    ctx, ks, s = setup
    reqs = [r for r in _requests(ctx, ks, s) if r[0] == "matmul"]
    want = [hx.hx_ct_export(ctx, hx.hx_matmul(ctx, ks, *args)) for _, args in reqs]
    levels = {(args[2], hx.hx_ct_info(args[0])[1]) for _, args in reqs}
    assert len(levels) > len({h for h, _ in levels})  # several levels of one size were used
    assert hx.hx_context_plan_cache_info(ctx)["plans"] == len({h for h, _ in levels})
    hx.hx_context_set_plan_cache(ctx, 1)
    info = hx.hx_context_plan_cache_info(ctx)
    assert info["plans"] == 0 and info["bytes"] == 0 and info["cap"] == 1
    for (kind, args), w in zip(reqs, want):
        assert np.array_equal(hx.hx_ct_export(ctx, hx.hx_matmul(ctx, ks, *args)), w)
        assert hx.hx_context_plan_cache_info(ctx)["plans"] <= 1
    sv = hx.hx_server_create(64 << 30, 3, 4)
    ids = [_submit(sv, ctx, ks, kind, args) for kind, args in reqs]
    got = _collect(sv, len(ids))
    hx.hx_server_destroy(sv)
    for rid, w in zip(ids, want):
        assert got[rid][1] == 0 and np.array_equal(hx.hx_ct_export(ctx, got[rid][0]), w)
    assert hx.hx_context_plan_cache_info(ctx)["evicted"] >= len(reqs) // 2
    hx.hx_context_set_plan_cache(ctx, 0)


def test_resident_keys_count_once_against_the_budget(setup):
    ctx, ks, s = setup
    ks2 = hx.hx_keygen(ctx, 2, 33, [1, 2])

    def key_bytes(k):
        probe = hx.hx_server_create(1 << 40, 1, 1)
        hx.hx_server_register_keys(probe, k)
        b = hx.hx_server_stats(probe)["key_bytes"]
        hx.hx_server_destroy(probe)
        return b

    kb1, kb2 = key_bytes(ks), key_bytes(ks2)
    sv = hx.hx_server_create(kb1 + kb2, 1, 1)       # exactly the two keysets
    hx.hx_server_register_keys(sv, ks)
    hx.hx_server_register_keys(sv, ks2)
    hx.hx_server_register_keys(sv, ks)              # registering again counts nothing
    st = hx.hx_server_stats(sv)
    assert st["key_bytes"] == kb1 + kb2 and st["budget_left"] == 0
    hx.hx_server_destroy(sv)
    sv = hx.hx_server_create(kb1 + kb2 - 1, 1, 1)
    hx.hx_server_register_keys(sv, ks)
    with pytest.raises(hx.HxError) as e:
        hx.hx_server_register_keys(sv, ks2)
    assert e.value.code == -2
    hx.hx_server_destroy(sv)
    hx.hx_keyset_destroy(ks2)


def test_mixed_size_batch_equals_products_alone(setup):
    """hx_matmul_batch_mixed: entries of different h and level in one call, grouped inside;
    each product equals hx_matmul on that pair alone, and a malformed entry fails the whole
    call with no outputs."""
    ctx, ks, s = setup
    reqs = [args for kind, args in _requests(ctx, ks, s) if kind == "matmul"]
    A, B, H = [r[0] for r in reqs], [r[1] for r in reqs], [r[2] for r in reqs]
    assert len(set(H)) == 2 and len({hx.hx_ct_info(a)[1] for a in A}) == 2
    outs = hx.hx_matmul_batch_mixed(ctx, ks, A, B, H)
    for a, b, h, o in zip(A, B, H, outs):
        alone = hx.hx_matmul(ctx, ks, a, b, h)
        assert np.array_equal(hx.hx_ct_export(ctx, o), hx.hx_ct_export(ctx, alone))
        hx.hx_ct_destroy(alone)
        hx.hx_ct_destroy(o)
    low = hx.hx_drop(ctx, B[1], hx.hx_ct_info(B[1])[1] - 1)
    with pytest.raises(hx.HxError) as e:
        hx.hx_matmul_batch_mixed(ctx, ks, A[:2], [B[0], low], H[:2])
    assert e.value.code == -4
    with pytest.raises(hx.HxError) as e:
        hx.hx_matmul_batch_mixed(ctx, ks, A[:2], B[:2], [H[0], 12])   # not a power of two
    assert e.value.code == -1
    hx.hx_ct_destroy(low)


def test_two_rings_in_one_server_equal_requests_alone(setup):
    """One server over two contexts of different ring degree and chain length (N = 2^12 with
    5 limbs, N = 2^13 with 6 limbs): a stream of matmuls, signs and rotations of both rings at
    several levels, submitted together, batched (matmuls and signs per signature, rotations of
    both rings together) and run across lanes; every result equals the same request computed
    alone, bit for bit."""
    ctx, ks, s = setup
    p = PARAMS["alg3_13"]
    ctx2 = hx.hx_context_create(p["log_n"], p["q_bits"], p["p_bits"], p["log2_scale"])
    s2 = (1 << p["log_n"]) // 2
    steps2 = sorted(set(Hc.matmul_rotation_steps(8, s2 // 64, 6)) | set(Hc.matmul_rotation_steps(8, s2 // 64, 4))
                    | set(Hc.matmul_rotation_steps(16, s2 // 256, 5)))
    ks2 = hx.hx_keygen(ctx2, 2, 41, steps2)
    try:
        reqs = [(ctx, ks, kind, args) for kind, args in _requests(ctx, ks, s)[:6]]
        for i, (h, limbs) in enumerate(((8, 6), (16, 5), (8, 4), (8, 6))):
            beta = s2 // (h * h)
            a = hx.hx_encrypt(ctx2, ks2, workloads.pack(workloads.matrices(700 + i, beta, h), h, beta), limbs, 70 + i)
            b = hx.hx_encrypt(ctx2, ks2, workloads.pack(workloads.matrices(800 + i, beta, h), h, beta), limbs, 80 + i)
            reqs.append((ctx2, ks2, "matmul", (a, b, h)))
        for i, d in enumerate((2, 4)):
            x = hx.hx_encrypt(ctx2, ks2, workloads.sign_inputs(60 + i, s2), 6, 90 + i)
            reqs.append((ctx2, ks2, "sign", (x, d, 1, 2000 + i)))
        st1 = Hc.matmul_rotation_steps(8, s // 64, 5)  # steps the first ring's keys hold
        for i, (k, limbs) in enumerate(((st1[0], 5), (st1[-1], 3), (0, 4))):
            x = hx.hx_encrypt(ctx, ks, np.random.default_rng(900 + i).uniform(-1, 1, s), limbs, 95 + i)
            reqs.append((ctx, ks, "rotate", (x, k)))
        for i, (k, limbs) in enumerate(((steps2[0], 6), (steps2[-1], 2))):
            x = hx.hx_encrypt(ctx2, ks2, np.random.default_rng(950 + i).uniform(-1, 1, s2), limbs, 97 + i)
            reqs.append((ctx2, ks2, "rotate", (x, k)))
        order = np.random.default_rng(5).permutation(len(reqs))  # the rings interleaved
        reqs = [reqs[i] for i in order]
        sv = hx.hx_server_create(64 << 30, 3, 4)
        hx.hx_server_register_keys(sv, ks)
        hx.hx_server_register_keys(sv, ks2)
        ids = [_submit(sv, c, k, kind, args) for c, k, kind, args in reqs]
        got = _collect(sv, len(ids))
        stats = hx.hx_server_stats(sv)
        hx.hx_server_destroy(sv)
        assert stats["completed"] == len(reqs)
        for rid, (c, k, kind, args) in zip(ids, reqs):
            res, st, lat = got[rid]
            assert st == 0 and lat > 0
            alone = _alone(c, k, kind, args)
            assert np.array_equal(hx.hx_ct_export(c, res), hx.hx_ct_export(c, alone)), (kind, c == ctx2)
            hx.hx_ct_destroy(res)
            hx.hx_ct_destroy(alone)
    finally:
        hx.hx_keyset_destroy(ks2)
        hx.hx_context_destroy(ctx2)


def test_rotations_of_two_rings_form_one_batch(setup):
    """Rotation requests of two rings (N = 2^12 and 2^13) queued while the server is paused go
    out as one batch (one launch per key-switching stage over both rings) and each equals
    hx_rotate alone."""
    ctx, ks, s = setup
    p = PARAMS["alg3_13"]
    ctx2 = hx.hx_context_create(p["log_n"], p["q_bits"], p["p_bits"], p["log2_scale"])
    s2 = (1 << p["log_n"]) // 2
    ks2 = hx.hx_keygen(ctx2, 2, 47, [1, -5])
    st1 = Hc.matmul_rotation_steps(8, s // 64, 5)
    try:
        reqs = []
        for i, (c, k_, n, st, limbs) in enumerate([(ctx, ks, s, st1[0], 5), (ctx2, ks2, s2, 1, 6), (ctx, ks, s, st1[1], 2),
                                                  (ctx2, ks2, s2, -5, 3), (ctx2, ks2, s2, 1, 4)]):
            x = hx.hx_encrypt(c, k_, np.random.default_rng(400 + i).uniform(-1, 1, n), limbs, 40 + i)
            reqs.append((c, k_, "rotate", (x, st)))
        sv = hx.hx_server_create(64 << 30, 2, 16)
        hx.hx_server_register_keys(sv, ks)
        hx.hx_server_register_keys(sv, ks2)
        hx.hx_server_pause(sv, True)
        ids = [_submit(sv, c, k_, kind, args) for c, k_, kind, args in reqs]
        hx.hx_server_pause(sv, False)
        got = _collect(sv, len(ids))
        stats = hx.hx_server_stats(sv)
        hx.hx_server_destroy(sv)
        assert stats["completed"] == len(reqs) and stats["batches"] == 1 and stats["largest_batch"] == len(reqs)
        for rid, (c, k_, kind, args) in zip(ids, reqs):
            res, st, lat = got[rid]
            assert st == 0
            alone = _alone(c, k_, kind, args)
            assert np.array_equal(hx.hx_ct_export(c, res), hx.hx_ct_export(c, alone))
            hx.hx_ct_destroy(res)
            hx.hx_ct_destroy(alone)
            hx.hx_ct_destroy(args[0])
    finally:
        hx.hx_keyset_destroy(ks2)
        hx.hx_context_destroy(ctx2)


def test_several_ring_call_equals_products_alone(setup):
    """hx_matmul_jobs with both rings: the same results as hx_matmul on each pair alone."""
    ctx, ks, s = setup
    p = PARAMS["alg3_13"]
    ctx2 = hx.hx_context_create(p["log_n"], p["q_bits"], p["p_bits"], p["log2_scale"])
    s2 = (1 << p["log_n"]) // 2
    ks2 = hx.hx_keygen(ctx2, 2, 43, sorted(set(Hc.matmul_rotation_steps(16, s2 // 256, 6))))
    try:
        jobs = [(ctx, ks, a, b, h) for _, (a, b, h) in [r for r in _requests(ctx, ks, s) if r[0] == "matmul"][:3]]
        beta = s2 // 256
        for i in range(2):
            a = hx.hx_encrypt(ctx2, ks2, workloads.pack(workloads.matrices(30 + i, beta, 16), 16, beta), 6, 30 + i)
            b = hx.hx_encrypt(ctx2, ks2, workloads.pack(workloads.matrices(40 + i, beta, 16), 16, beta), 6, 40 + i)
            jobs.insert(1 + 2 * i, (ctx2, ks2, a, b, 16))
        outs = hx.hx_matmul_jobs(jobs)
        for (c, k, a, b, h), o in zip(jobs, outs):
            alone = hx.hx_matmul(c, k, a, b, h)
            assert np.array_equal(hx.hx_ct_export(c, o), hx.hx_ct_export(c, alone))
            hx.hx_ct_destroy(alone)
            hx.hx_ct_destroy(o)
        with pytest.raises(hx.HxError) as e:  # a job whose keys belong to the other ring
            hx.hx_matmul_jobs([jobs[0], (ctx, ks2, jobs[0][2], jobs[0][3], jobs[0][4])])
        assert e.value.code == -1
    finally:
        hx.hx_keyset_destroy(ks2)
        hx.hx_context_destroy(ctx2)
