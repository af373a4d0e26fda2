"""hx_rotate_noalloc: the rotation for callers that cannot allocate device
memory (their memory manager owns the device, or allocation latency is not
allowed) must give exactly what hx_rotate gives, call after call, although all
its intermediates live in one shared static device array."""
import numpy as np
import pytest

from paper_2207_04620_gb300 import hx, workloads

from hxpair import Pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pair():
    from paper_2207_04620_gb300 import build

    build.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pr = Pair("alg3", rot_steps=[1, 7, -2])
    yield pr
    pr.close()


def test_noalloc_rotation_matches_hx_rotate_twice(pair):
    import torch

    limbs = pair.octx.n_q
    for call, (seed, k) in enumerate(((1, 7), (2, -2))):
        ct = pair.encrypt(workloads.sign_inputs(seed, pair.octx.S), 10 + seed)
        h = pair.to_lib(ct)
        rot = hx.hx_rotate(pair.ctx, pair.ks, h, k)
        want = hx.hx_ct_export(pair.ctx, rot)
        hx.hx_ct_destroy(rot)
        dev_in = torch.from_numpy(ct.c.view(np.int64).copy()).cuda()
        dev_out = torch.empty_like(dev_in)
        hx.hx_rotate_noalloc(pair.ctx, pair.ks, dev_in.data_ptr(), limbs, dev_out.data_ptr(), k,
                             stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        got = dev_out.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want), "call %d differs from hx_rotate" % call
        hx.hx_ct_destroy(h)


def test_noalloc_rejects_oversized_rotation(pair):
    import torch

    # N = 2^16 with 8 limbs needs about 48 MB of scratch, above the static 16 MiB.  The
    # buffers are real device buffers of that ciphertext's size, so a rejection that came
    # later than the host-side checks would still stay inside them.
    ctx = hx.hx_context_create(16, [60] + [45] * 7, [60, 60], 45)
    try:
        x = torch.zeros(2 * 8 * (1 << 16), dtype=torch.int64, device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(hx.HxError) as e:
            hx.hx_rotate_noalloc(ctx, pair.ks, x.data_ptr(), 8, y.data_ptr(), 1)
        assert e.value.code == -1 and "static scratch" in str(e.value)
    finally:
        hx.hx_context_destroy(ctx)


def test_noalloc_rejects_overlapping_buffers(pair):
    import torch

    limbs = pair.octx.n_q
    x = torch.zeros(3 * 2 * limbs * pair.N, dtype=torch.int64, device="cuda")
    with pytest.raises(hx.HxError) as e:
        hx.hx_rotate_noalloc(pair.ctx, pair.ks, x.data_ptr(), limbs, x.data_ptr() + 8 * limbs * pair.N, 1)
    assert e.value.code == -1 and "overlap" in str(e.value)
