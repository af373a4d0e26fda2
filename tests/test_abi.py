"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/hx.h declares; the Python binding covers exactly those."""
import os
import re

from paper_2207_04620_gb300 import build, hx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    text = open(os.path.join(ROOT, "include", "hx.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hx_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    build.build()
    lib = hx.lib()
    names = header_symbols()
    assert len(names) >= 40
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(hx.declared_symbols()) == names


def test_no_gpu_fails_loudly_or_runs():
    # without a device the first call must raise, never fall back to host code
    try:
        ctx = hx.hx_context_create(12, [60, 40, 40], [60], 40)
    except hx.HxError as e:
        assert e.code == -7
    else:
        hx.hx_context_destroy(ctx)


def test_bad_parameters_rejected_before_any_device_work():
    import pytest

    for args in ((9, [60], [60], 40), (12, [], [60], 40), (12, [60, 70], [60], 40), (12, [60], [], 40)):
        with pytest.raises(hx.HxError) as e:
            hx.hx_context_create(*args)
        assert e.value.code in (-1, -7)
