"""Handles carry the context they were made in, and every entry point rejects a
key set, ciphertext or plan of another context with HX_EINVAL before any device
work (a foreign handle has another row length, so it must never reach a copy
or a kernel).

The foreign handles come from a context of the LARGER ring (N = 2^13, the same
chain), passed to entry points of the N = 2^12 context.  Every foreign buffer
is therefore larger than what the home context would read from it: even an
entry point that failed to check would stay inside its buffers.  No test here
passes a smaller ring's handle to a larger context."""
import numpy as np
import pytest

from paper_2207_04620_gb300 import hx, workloads

pytestmark = pytest.mark.gpu

CHAIN = dict(q_bits=[60, 45, 45, 45, 45], p_bits=[60, 60], log2_scale=45)
H = 8
SEED = 99


@pytest.fixture(scope="module")
def two():
    from paper_2207_04620_gb300 import build

    build.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    home = hx.hx_context_create(12, **CHAIN)
    far = hx.hx_context_create(13, **CHAIN)
    steps = sorted(set(hx.hx_matmul_rotation_steps(home, H, 5)) | {1})
    ks_h = hx.hx_keygen(home, 2, SEED, steps)
    ks_f = hx.hx_keygen(far, 2, SEED, [1])
    s_h = workloads.sign_inputs(1, 2048)
    s_f = workloads.sign_inputs(1, 4096)
    ct_h = hx.hx_encrypt(home, ks_h, s_h, seed=3)
    ct_f = hx.hx_encrypt(far, ks_f, s_f, seed=3)
    plan_f = hx.hx_matmul_plan_create(far, H, 5)
    objs = dict(home=home, far=far, ks_h=ks_h, ks_f=ks_f, ct_h=ct_h, ct_f=ct_f, plan_f=plan_f, s_h=s_h)
    yield objs
    hx.hx_matmul_plan_destroy(plan_f)
    for c in (ct_h, ct_f):
        hx.hx_ct_destroy(c)
    hx.hx_keyset_destroy(ks_h)
    hx.hx_keyset_destroy(ks_f)
    hx.hx_context_destroy(home)
    hx.hx_context_destroy(far)


def _rejects(fn, *args, **kw):
    with pytest.raises(hx.HxError) as e:
        fn(*args, **kw)
    assert e.value.code == -1, (fn.__name__, e.value.code, str(e.value))
    assert "another context" in str(e.value), (fn.__name__, str(e.value))


def test_single_operations_reject_foreign_handles(two):
    c, a, f, kh, kf = two["home"], two["ct_h"], two["ct_f"], two["ks_h"], two["ks_f"]
    pt = np.zeros(4096, dtype=np.int64)
    _rejects(hx.hx_add, c, a, f)
    _rejects(hx.hx_add, c, f, a)
    _rejects(hx.hx_sub, c, a, f)
    _rejects(hx.hx_mul_plain, c, f, pt, 2.0 ** 45)
    _rejects(hx.hx_mul_int, c, f, 3)
    _rejects(hx.hx_add_const, c, f, 0.5)
    _rejects(hx.hx_tensor, c, f, a)
    _rejects(hx.hx_rescale, c, f)
    _rejects(hx.hx_drop, c, f, 3)
    _rejects(hx.hx_rotate, c, kf, a, 1)
    _rejects(hx.hx_rotate, c, kh, f, 1)
    _rejects(hx.hx_rotate_hoisted, c, kf, a, [1])
    _rejects(hx.hx_rotate_hoisted, c, kh, f, [1])
    d = hx.hx_tensor(c, a, a)
    try:
        _rejects(hx.hx_relinearize, c, kf, d)
        _rejects(hx.hx_relin_rescale, c, kf, d)
    finally:
        hx.hx_ct_destroy(d)


def test_client_calls_reject_foreign_keys(two):
    c, kf, kh, f = two["home"], two["ks_f"], two["ks_h"], two["ct_f"]
    s = two["s_h"]
    _rejects(hx.hx_encrypt, c, kf, s, seed=1)
    _rejects(hx.hx_encrypt_batch, c, kf, np.stack([s, s]), [1, 2])
    _rejects(hx.hx_encrypt_coeffs, c, kf, np.zeros(4096, dtype=np.int64), 2.0 ** 45, 5, 1)
    _rejects(hx.hx_decrypt, c, kf, two["ct_h"])
    _rejects(hx.hx_decrypt, c, kh, f)
    _rejects(hx.hx_decrypt_coeffs, c, kh, f)
    _rejects(hx.hx_decrypt_parties, c, kh, f, [1, 1])
    _rejects(hx.hx_keyset_add_rotations, c, kf, [2])
    _rejects(hx.hx_dkeyswitch, c, kh, kf, two["ct_h"], 1)
    _rejects(hx.hx_dbootstrap, c, kh, f, 1)


def test_ct_save_rejects_foreign_ciphertext(two, tmp_path):
    _rejects(hx.hx_ct_save, two["home"], two["ct_f"], str(tmp_path / "x.hxct"))


def test_method_calls_reject_foreign_handles(two):
    c, a, f, kh, kf = two["home"], two["ct_h"], two["ct_f"], two["ks_h"], two["ks_f"]
    _rejects(hx.hx_matmul, c, kf, a, a, H)
    _rejects(hx.hx_matmul, c, kh, a, f, H)
    _rejects(hx.hx_matmul_batch, c, kf, 0, [a], [a], H)
    _rejects(hx.hx_matmul_batch, c, kh, 0, [a, f], [a, a], H)
    _rejects(hx.hx_matmul_batch, c, kh, two["plan_f"], [a], [a], H)
    _rejects(hx.hx_matmul_batch_mixed, c, kh, [a, f], [a, a], [H, H])
    _rejects(hx.hx_matmul_batch_mixed, c, kf, [a], [a], [H])
    _rejects(hx.hx_rmatmul_batch, c, kh, 0, [f], [a], H, 2)
    _rejects(hx.hx_transpose, c, kh, 0, [f], H)
    _rejects(hx.hx_transpose, c, kf, 0, [a], H)
    _rejects(hx.hx_sign_approx, c, kh, f, 4, 1)
    _rejects(hx.hx_sign_approx, c, kf, a, 4, 1)
    _rejects(hx.hx_sign_approx_batch, c, kh, [a, f], 4, 1)
    _rejects(hx.hx_dense_layer, c, kh, [f], [a], [a], H, 1, 1, 4, 1, 4.0)
    _rejects(hx.hx_dense_layer, c, kf, [a], [a], [a], H, 1, 1, 4, 1, 4.0)
    _rejects(hx.hx_aggregate, c, [a, f], 2, [a], 0.01)
    _rejects(hx.hx_aggregate, c, [a], 1, [f], 0.01)
    _rejects(hx.hx_matmul_plan_bind_keys, c, two["plan_f"], kh)
    _rejects(hx.hx_matmul_plan_set_mask, c, two["plan_f"], 0, np.zeros(4096, dtype=np.int64))
    _rejects(hx.hx_matmul_exec_create, c, kf, two["plan_f"], 1, 2.0 ** 45)


def test_executor_rejects_foreign_inputs(two):
    c, a, f, kh = two["home"], two["ct_h"], two["ct_f"], two["ks_h"]
    plan = hx.hx_matmul_plan_create(c, H, 5)
    try:
        _, _, scale = hx.hx_ct_info(a)
        ex = hx.hx_matmul_exec_create(c, kh, plan, 1, scale)
        try:
            _rejects(hx.hx_matmul_exec_run, ex, [f], [a])
            _rejects(hx.hx_matmul_exec_run, ex, [a], [f])
        finally:
            hx.hx_matmul_exec_destroy(ex)
    finally:
        hx.hx_matmul_plan_destroy(plan)


def test_server_rejects_foreign_handles(two):
    c, a, f, kh, kf = two["home"], two["ct_h"], two["ct_f"], two["ks_h"], two["ks_f"]
    sv = hx.hx_server_create(8 << 30, 1, 4)
    try:
        _rejects(hx.hx_server_submit_matmul, sv, c, kh, a, f, H)
        _rejects(hx.hx_server_submit_matmul, sv, c, kf, a, a, H)
        _rejects(hx.hx_server_submit_sign, sv, c, kh, f, 4, 1)
        _rejects(hx.hx_server_submit_sign, sv, c, kf, a, 4, 1)
    finally:
        hx.hx_server_destroy(sv)


def test_noalloc_rotation_rejects_foreign_keys(two):
    import torch

    c, kf = two["home"], two["ks_f"]
    # real device buffers of the home ring's size: nothing is read if the check holds
    x = torch.zeros(2 * 5 * 4096, dtype=torch.int64, device="cuda")
    y = torch.zeros_like(x)
    _rejects(hx.hx_rotate_noalloc, c, kf, x.data_ptr(), 5, y.data_ptr(), 1)
