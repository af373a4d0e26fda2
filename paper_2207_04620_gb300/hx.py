"""Python binding of libhx (include/hx.h): ctypes argument marshalling only.

Every function keeps the C name and forwards to the CUDA library; all
computation happens in the library's kernels.  Handles are opaque integers.
If libhx.so has not been built the first call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhx.so")
_lib = None

c_int, c_double, c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_size_t
c_u64, c_i64, c_u32, c_vp = ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p
P_u64 = ctypes.POINTER(ctypes.c_uint64)
P_i64 = ctypes.POINTER(ctypes.c_int64)
P_i32 = ctypes.POINTER(ctypes.c_int32)
P_dbl = ctypes.POINTER(ctypes.c_double)
PP = ctypes.POINTER(c_vp)

HX_MAX_Q, HX_MAX_P = 60, 6
STATUS = {0: "HX_OK", -1: "HX_EINVAL", -2: "HX_ENOMEM", -3: "HX_ELEVEL", -4: "HX_ESCALE", -5: "HX_EKEY",
          -6: "HX_ETIMEOUT", -7: "HX_ECUDA", -8: "HX_EPARTY"}
COUNTERS = ["Add", "Mul_pt", "Rot", "RotHoisted", "Mul_ct", "KeySwitch", "ModUp", "Rescale", "Refresh", "launches"]


class HxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


class hx_params(ctypes.Structure):
    _fields_ = [("log_n", c_int), ("n_q", c_int), ("q_bits", c_int * HX_MAX_Q), ("n_p", c_int),
                ("p_bits", c_int * HX_MAX_P), ("log2_scale", c_double), ("sigma", c_double), ("alpha", c_int)]


_SIGS = {
    "hx_last_error": (ctypes.c_char_p, []),
    "hx_context_create": (c_int, [ctypes.POINTER(hx_params), PP]),
    "hx_context_destroy": (None, [c_vp]),
    "hx_context_primes": (c_int, [c_vp, P_u64, c_int]),
    "hx_context_n": (c_int, [c_vp]),
    "hx_keygen": (c_int, [c_vp, c_int, c_u64, P_i32, c_size_t, PP]),
    "hx_keyset_add_rotations": (c_int, [c_vp, c_vp, P_i32, c_size_t]),
    "hx_keyset_export_switch_key": (c_i64, [c_vp, c_u64, P_u64, c_size_t]),
    "hx_keyset_export_public_key": (c_i64, [c_vp, P_u64, c_size_t]),
    "hx_keyset_destroy": (None, [c_vp]),
    "hx_encode": (c_int, [c_vp, P_dbl, c_size_t, c_double, P_i64]),
    "hx_decrypt_parties": (c_int, [c_vp, c_vp, c_vp, ctypes.POINTER(ctypes.c_uint8), c_size_t, P_dbl, c_size_t]),
    "hx_ct_save": (c_int, [c_vp, c_vp, ctypes.c_char_p]),
    "hx_matmul_batch_mixed": (c_int, [c_vp, c_vp, PP, PP, P_i32, c_size_t, PP, c_vp]),
    "hx_matmul_jobs": (c_int, [c_vp, c_size_t, PP, c_vp]),
    "hx_keyset_save": (c_int, [c_vp, c_vp, ctypes.c_char_p]),
    "hx_keyset_load": (c_int, [c_vp, ctypes.c_char_p, PP]),
    "hx_ct_load": (c_int, [c_vp, ctypes.c_char_p, PP]),
    "hx_encode_batch": (c_int, [c_vp, P_dbl, c_size_t, c_size_t, c_double, P_i64, c_vp]),
    "hx_encrypt_batch": (c_int, [c_vp, c_vp, P_dbl, c_size_t, c_size_t, c_int, P_u64, PP, c_vp]),
    "hx_encrypt": (c_int, [c_vp, c_vp, P_dbl, c_size_t, c_int, c_u64, PP]),
    "hx_encrypt_coeffs": (c_int, [c_vp, c_vp, P_i64, c_double, c_int, c_u64, c_u32, c_u32, PP]),
    "hx_decrypt": (c_int, [c_vp, c_vp, c_vp, P_dbl, c_size_t]),
    "hx_decrypt_coeffs": (c_int, [c_vp, c_vp, c_vp, P_i64]),
    "hx_ct_import": (c_int, [c_vp, P_u64, c_int, c_int, c_double, PP]),
    "hx_ct_export": (c_i64, [c_vp, P_u64, c_size_t]),
    "hx_ct_info": (c_int, [c_vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int), P_dbl]),
    "hx_ct_destroy": (None, [c_vp]),
    "hx_add": (c_int, [c_vp, c_vp, c_vp, PP, c_vp]),
    "hx_sub": (c_int, [c_vp, c_vp, c_vp, PP, c_vp]),
    "hx_mul_plain": (c_int, [c_vp, c_vp, P_i64, c_double, PP, c_vp]),
    "hx_mul_int": (c_int, [c_vp, c_vp, c_i64, c_double, PP, c_vp]),
    "hx_add_const": (c_int, [c_vp, c_vp, c_double, PP, c_vp]),
    "hx_tensor": (c_int, [c_vp, c_vp, c_vp, PP, c_vp]),
    "hx_relinearize": (c_int, [c_vp, c_vp, c_vp, PP, c_vp]),
    "hx_rescale": (c_int, [c_vp, c_vp, PP, c_vp]),
    "hx_relin_rescale": (c_int, [c_vp, c_vp, c_vp, PP, c_vp]),
    "hx_drop": (c_int, [c_vp, c_vp, c_int, PP, c_vp]),
    "hx_rotate": (c_int, [c_vp, c_vp, c_vp, ctypes.c_int32, PP, c_vp]),
    "hx_rotate_hoisted": (c_int, [c_vp, c_vp, c_vp, P_i32, c_int, PP, c_vp]),
    "hx_ntt": (c_int, [c_vp, c_vp, c_int, c_int, P_i32, c_int, c_vp]),
    "hx_rotate_noalloc": (c_int, [c_vp, c_vp, c_vp, c_int, c_vp, ctypes.c_int32, c_vp]),
    "hx_ntt_multi": (c_int, [c_vp, c_int, c_int, c_vp]),
    "hx_matmul_plan_create": (c_int, [c_vp, c_int, c_int, PP]),
    "hx_matmul_plan_num_masks": (c_int, [c_vp]),
    "hx_matmul_plan_set_mask": (c_int, [c_vp, c_vp, c_int, P_i64]),
    "hx_matmul_plan_destroy": (None, [c_vp]),
    "hx_matmul_rotation_steps": (c_int, [c_vp, c_int, c_int, P_i32, c_int]),
    "hx_matmul": (c_int, [c_vp, c_vp, c_vp, c_vp, c_int, PP, c_vp]),
    "hx_matmul_batch": (c_int, [c_vp, c_vp, c_vp, PP, PP, c_int, c_size_t, PP, c_vp]),
    "hx_matmul_plan_bind_keys": (c_int, [c_vp, c_vp, c_vp, c_vp]),
    "hx_matmul_plan_bound_bytes": (c_i64, [c_vp]),
    "hx_rmatmul_batch": (c_int, [c_vp, c_vp, c_vp, PP, PP, c_int, c_int, c_size_t, PP, c_vp]),
    "hx_rmatmul_rotation_steps": (c_int, [c_vp, c_int, c_int, c_int, P_i32, c_int]),
    "hx_transpose_plan_create": (c_int, [c_vp, c_int, c_int, PP]),
    "hx_transpose_rotation_steps": (c_int, [c_vp, c_int, P_i32, c_int]),
    "hx_transpose": (c_int, [c_vp, c_vp, c_vp, PP, c_int, c_size_t, PP, c_vp]),
    "hx_matmul_exec_create": (c_int, [c_vp, c_vp, c_vp, c_size_t, c_double, PP]),
    "hx_matmul_exec_run": (c_int, [c_vp, PP, PP, PP, c_vp]),
    "hx_matmul_exec_launches": (c_i64, [c_vp]),
    "hx_matmul_exec_run_host": (c_int, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "hx_matmul_exec_out_info": (c_int, [c_vp, ctypes.POINTER(c_int), ctypes.POINTER(c_double)]),
    "hx_matmul_exec_destroy": (None, [c_vp]),
    "hx_sign_approx": (c_int, [c_vp, c_vp, c_vp, c_int, c_int, c_int, c_int, c_u64, PP, c_vp]),
    "hx_sign_approx_batch": (c_int, [c_vp, c_vp, PP, c_size_t, c_int, c_int, c_int, c_int, c_u64, PP, c_vp]),
    "hx_dense_layer": (c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, PP, PP, PP, c_int, c_int, c_int, c_int, c_int, c_double,
                                c_u64, PP, PP, PP, c_vp]),
    "hx_dense_rotation_steps": (c_int, [c_vp, c_int, P_i32, c_int]),
    "hx_alu_calibrate": (c_int, [c_vp, P_dbl, P_dbl, c_vp]),
    "hx_aggregate": (c_int, [c_vp, PP, c_size_t, PP, c_size_t, c_double, PP, c_vp]),
    "hx_dkeyswitch": (c_int, [c_vp, c_vp, c_vp, c_vp, c_u64, PP, c_vp]),
    "hx_dbootstrap": (c_int, [c_vp, c_vp, c_vp, c_u64, PP, c_vp]),
    "hx_context_set_plan_cache": (c_int, [c_vp, c_u64]),
    "hx_context_plan_cache_info": (c_int, [c_vp, P_u64, c_int]),
    "hx_server_create": (c_int, [c_size_t, c_int, c_int, PP]),
    "hx_server_register_keys": (c_int, [c_vp, c_vp]),
    "hx_server_submit_matmul": (c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, c_int, P_u64]),
    "hx_server_submit_sign": (c_int, [c_vp, c_vp, c_vp, c_vp, c_int, c_int, c_int, c_u64, P_u64]),
    "hx_server_submit_rotate": (c_int, [c_vp, c_vp, c_vp, c_vp, c_i64, P_u64]),
    "hx_server_poll": (c_int, [c_vp, c_int, P_u64, PP, P_i32, P_dbl, c_int]),
    "hx_server_stats": (c_int, [c_vp, P_u64, c_int]),
    "hx_server_destroy": (None, [c_vp]),
    "hx_server_set_deadline": (c_int, [c_vp, c_u64, ctypes.c_double]),
    "hx_server_pause": (c_int, [c_vp, c_int]),
    "hx_counters": (c_int, [c_vp, P_u64, c_int]),
    "hx_counters_reset": (None, [c_vp]),
    "hx_autotune": (c_int, [c_vp, P_i32, c_vp]),
    "hx_ntt_tiles": (c_int, [c_vp, P_i32, P_i32]),
    "hx_ntt_tuning": (c_int, [c_vp, P_i32, c_int]),
    "hx_ntt_split": (c_int, [c_vp, c_int]),
    "hx_rotate_jobs": (c_int, [c_vp, c_size_t, PP, c_vp]),
    "hx_profile_enable": (c_int, [c_vp, c_int]),
    "hx_profile_read": (c_int, [c_vp, c_int, ctypes.c_char_p, c_size_t, P_u64, P_dbl, P_dbl]),
}


def lib():
    """Loads libhx.so (built by paper_2207_04620_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhx.so is not built (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def declared_symbols() -> list:
    return list(_SIGS)


def _chk(st: int) -> int:
    if st < 0:
        raise HxError(st, lib().hx_last_error().decode())
    return st


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)  # torch.cuda.Stream


def _u64p(a):
    return a.ctypes.data_as(P_u64)


def _i64p(a):
    return a.ctypes.data_as(P_i64)


def _i32arr(xs):
    a = np.ascontiguousarray(np.array(list(xs), dtype=np.int32))
    return a, a.ctypes.data_as(P_i32)


def _out():
    return c_vp()


# ---- context -----------------------------------------------------------------

def hx_context_create(log_n: int, q_bits, p_bits, log2_scale: float, sigma: float = 3.2, alpha: int = 0) -> int:
    p = hx_params()
    p.alpha = int(alpha)
    p.log_n, p.n_q, p.n_p = log_n, len(q_bits), len(p_bits)
    for i, b in enumerate(q_bits):
        p.q_bits[i] = b
    for i, b in enumerate(p_bits):
        p.p_bits[i] = b
    p.log2_scale, p.sigma = float(log2_scale), float(sigma)
    out = _out()
    _chk(lib().hx_context_create(ctypes.byref(p), ctypes.byref(out)))
    return out.value


def hx_context_destroy(ctx: int) -> None:
    lib().hx_context_destroy(ctx)


def hx_context_primes(ctx: int) -> list:
    buf = np.zeros(HX_MAX_Q + HX_MAX_P, dtype=np.uint64)
    n = _chk(lib().hx_context_primes(ctx, _u64p(buf), buf.size))
    return [int(x) for x in buf[:n]]


def hx_context_n(ctx: int) -> int:
    return _chk(lib().hx_context_n(ctx))


# ---- keys ----------------------------------------------------------------------

def hx_keygen(ctx: int, n_parties: int, seed: int, rot_steps=()) -> int:
    arr, ptr = _i32arr(rot_steps)
    out = _out()
    _chk(lib().hx_keygen(ctx, n_parties, seed, ptr, arr.size, ctypes.byref(out)))
    return out.value


def hx_keyset_add_rotations(ctx: int, ks: int, steps) -> None:
    arr, ptr = _i32arr(steps)
    _chk(lib().hx_keyset_add_rotations(ctx, ks, ptr, arr.size))


def hx_keyset_export_switch_key(ctx: int, ks: int, galois: int, dnum: int, n_all: int) -> np.ndarray:
    n = hx_context_n(ctx)
    buf = np.zeros(dnum * 2 * n_all * n, dtype=np.uint64)
    _chk(lib().hx_keyset_export_switch_key(ks, galois, _u64p(buf), buf.size))
    return buf.reshape(dnum, 2, n_all, n)


def hx_keyset_export_public_key(ctx: int, ks: int, n_q: int) -> np.ndarray:
    n = hx_context_n(ctx)
    buf = np.zeros(2 * n_q * n, dtype=np.uint64)
    _chk(lib().hx_keyset_export_public_key(ks, _u64p(buf), buf.size))
    return buf.reshape(2, n_q, n)


def hx_keyset_destroy(ks: int) -> None:
    lib().hx_keyset_destroy(ks)


# ---- encoding, encryption ---------------------------------------------------------

def hx_encode(ctx: int, slots, scale: float) -> np.ndarray:
    z = np.ascontiguousarray(np.asarray(slots, dtype=np.float64))
    out = np.zeros(hx_context_n(ctx), dtype=np.int64)
    _chk(lib().hx_encode(ctx, z.ctypes.data_as(P_dbl), z.size, scale, _i64p(out)))
    return out


def hx_encode_batch(ctx: int, slots, scale: float, stream=None) -> np.ndarray:
    """slots: [count][n] array; returns [count][N] int64 coefficients (device encoder)."""
    z = np.ascontiguousarray(np.asarray(slots, dtype=np.float64))
    count, n = z.shape
    out = np.zeros((count, hx_context_n(ctx)), dtype=np.int64)
    _chk(lib().hx_encode_batch(ctx, z.ctypes.data_as(P_dbl), n, count, float(scale), _i64p(out), _stream(stream)))
    return out


def hx_encrypt_batch(ctx: int, ks: int, slots, seeds, limbs: int = 0, stream=None) -> list:
    z = np.ascontiguousarray(np.asarray(slots, dtype=np.float64))
    count, n = z.shape
    sd = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    assert sd.size == count
    outs = (c_vp * count)()
    _chk(lib().hx_encrypt_batch(ctx, ks, z.ctypes.data_as(P_dbl), n, count, limbs, _u64p(sd), outs, _stream(stream)))
    return [outs[i] for i in range(count)]


def hx_encrypt(ctx: int, ks: int, slots, limbs: int = 0, seed: int = 0) -> int:
    z = np.ascontiguousarray(np.asarray(slots, dtype=np.float64))
    out = _out()
    _chk(lib().hx_encrypt(ctx, ks, z.ctypes.data_as(P_dbl), z.size, limbs, seed, ctypes.byref(out)))
    return out.value


def hx_encrypt_coeffs(ctx: int, ks: int, coeffs, scale: float, limbs: int, seed: int, tag: int = 0,
                      index: int = 0) -> int:
    m = np.ascontiguousarray(np.asarray(coeffs, dtype=np.int64))
    out = _out()
    _chk(lib().hx_encrypt_coeffs(ctx, ks, _i64p(m), scale, limbs, seed, tag, index, ctypes.byref(out)))
    return out.value


def hx_decrypt(ctx: int, ks: int, ct: int, n: int | None = None) -> np.ndarray:
    n = hx_context_n(ctx) // 2 if n is None else n
    out = np.zeros(n, dtype=np.float64)
    _chk(lib().hx_decrypt(ctx, ks, ct, out.ctypes.data_as(P_dbl), n))
    return out


def hx_decrypt_coeffs(ctx: int, ks: int, ct: int) -> np.ndarray:
    out = np.zeros(hx_context_n(ctx), dtype=np.int64)
    _chk(lib().hx_decrypt_coeffs(ctx, ks, ct, _i64p(out)))
    return out


# ---- ciphertext handles -----------------------------------------------------------

def hx_ct_import(ctx: int, residues: np.ndarray, scale: float) -> int:
    a = np.ascontiguousarray(residues, dtype=np.uint64)
    comps, limbs, _ = a.shape
    out = _out()
    _chk(lib().hx_ct_import(ctx, _u64p(a), comps, limbs, scale, ctypes.byref(out)))
    return out.value


def hx_decrypt_parties(ctx: int, ks: int, ct: int, present, n: int | None = None) -> np.ndarray:
    """DDec with a party mask (truthy = that party's share arrived)."""
    flags = np.ascontiguousarray(np.asarray(present, dtype=np.uint8))
    n = hx_context_n(ctx) // 2 if n is None else n
    out = np.zeros(n)
    _chk(lib().hx_decrypt_parties(ctx, ks, ct, flags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), flags.size,
                                  out.ctypes.data_as(P_dbl), n))
    return out


def hx_keyset_save(ctx: int, ks: int, path: str) -> None:
    _chk(lib().hx_keyset_save(ctx, ks, path.encode()))


def hx_keyset_load(ctx: int, path: str) -> int:
    out = _out()
    _chk(lib().hx_keyset_load(ctx, path.encode(), ctypes.byref(out)))
    return out.value


def hx_ct_save(ctx: int, ct: int, path: str) -> None:
    _chk(lib().hx_ct_save(ctx, ct, path.encode()))


def hx_ct_load(ctx: int, path: str) -> int:
    out = _out()
    _chk(lib().hx_ct_load(ctx, path.encode(), ctypes.byref(out)))
    return out.value


def hx_ct_info(ct: int):
    c, l, s = c_int(), c_int(), c_double()
    _chk(lib().hx_ct_info(ct, ctypes.byref(c), ctypes.byref(l), ctypes.byref(s)))
    return c.value, l.value, s.value


def hx_ct_export(ctx: int, ct: int) -> np.ndarray:
    comps, limbs, _ = hx_ct_info(ct)
    n = hx_context_n(ctx)
    buf = np.zeros(comps * limbs * n, dtype=np.uint64)
    _chk(lib().hx_ct_export(ct, _u64p(buf), buf.size))
    return buf.reshape(comps, limbs, n)


def hx_ct_destroy(ct: int) -> None:
    lib().hx_ct_destroy(ct)


# ---- single operations --------------------------------------------------------------

def _op(name, *args, stream=None):
    out = _out()
    _chk(getattr(lib(), name)(*args, ctypes.byref(out), _stream(stream)))
    return out.value


def hx_add(ctx, a, b, stream=None):
    return _op("hx_add", ctx, a, b, stream=stream)


def hx_sub(ctx, a, b, stream=None):
    return _op("hx_sub", ctx, a, b, stream=stream)


def hx_mul_plain(ctx, a, pt_coeffs, pt_scale, stream=None):
    m = np.ascontiguousarray(np.asarray(pt_coeffs, dtype=np.int64))
    return _op("hx_mul_plain", ctx, a, _i64p(m), pt_scale, stream=stream)


def hx_mul_int(ctx, a, c, new_scale=0.0, stream=None):
    return _op("hx_mul_int", ctx, a, int(c), float(new_scale), stream=stream)


def hx_add_const(ctx, a, value, stream=None):
    return _op("hx_add_const", ctx, a, float(value), stream=stream)


def hx_tensor(ctx, a, b, stream=None):
    return _op("hx_tensor", ctx, a, b, stream=stream)


def hx_relinearize(ctx, ks, d, stream=None):
    return _op("hx_relinearize", ctx, ks, d, stream=stream)


def hx_relin_rescale(ctx, ks, d, stream=None):
    return _op("hx_relin_rescale", ctx, ks, d, stream=stream)


def hx_rescale(ctx, a, stream=None):
    return _op("hx_rescale", ctx, a, stream=stream)


def hx_drop(ctx, a, limbs, stream=None):
    return _op("hx_drop", ctx, a, limbs, stream=stream)


def hx_rotate(ctx, ks, a, k, stream=None):
    return _op("hx_rotate", ctx, ks, a, int(k), stream=stream)


def hx_rotate_hoisted(ctx, ks, a, steps, stream=None) -> list:
    arr, ptr = _i32arr(steps)
    outs = (c_vp * max(1, arr.size))()
    _chk(lib().hx_rotate_hoisted(ctx, ks, a, ptr, arr.size, outs, _stream(stream)))
    return [outs[i] for i in range(arr.size)]


def hx_rotate_noalloc(ctx: int, ks: int, in_ptr: int, limbs: int, out_ptr: int, k: int, stream=None) -> None:
    """Rotation of the ciphertext at device address in_ptr ([2][limbs][N] words) into out_ptr,
    using the library's static scratch instead of device allocations."""
    _chk(lib().hx_rotate_noalloc(ctx, ks, in_ptr, limbs, out_ptr, int(k), _stream(stream)))


def hx_ntt(ctx: int, dev_ptr: int, n_polys: int, prime_idx, inverse: bool = False, stream=None) -> None:
    arr, ptr = _i32arr(prime_idx)
    _chk(lib().hx_ntt(ctx, dev_ptr, n_polys, arr.size, ptr, int(bool(inverse)), _stream(stream)))


class _NttJob(ctypes.Structure):
    _fields_ = [("ctx", c_vp), ("data", c_vp), ("n_polys", c_int), ("n_limbs", c_int), ("prime_idx", P_i32)]


def hx_ntt_multi(jobs, inverse: bool = False, stream=None) -> None:
    """jobs: (ctx, device pointer, n_polys, prime indices) per ring; one launch per phase for all."""
    arr = (_NttJob * len(jobs))()
    keep = []
    for i, (ctx, ptr, n_polys, primes) in enumerate(jobs):
        pa, pp = _i32arr(primes)
        keep.append(pa)
        arr[i] = _NttJob(ctx, ptr, n_polys, pa.size, pp)
    _chk(lib().hx_ntt_multi(arr, len(jobs), int(bool(inverse)), _stream(stream)))


# ---- HE-MatMult ----------------------------------------------------------------------

def hx_matmul_plan_create(ctx: int, h: int, limbs: int) -> int:
    out = _out()
    _chk(lib().hx_matmul_plan_create(ctx, h, limbs, ctypes.byref(out)))
    return out.value


def hx_matmul_plan_num_masks(plan: int) -> int:
    return _chk(lib().hx_matmul_plan_num_masks(plan))


def hx_matmul_plan_set_mask(ctx: int, plan: int, i: int, coeffs) -> None:
    m = np.ascontiguousarray(np.asarray(coeffs, dtype=np.int64))
    _chk(lib().hx_matmul_plan_set_mask(ctx, plan, i, _i64p(m)))


def hx_matmul_plan_bind_keys(ctx: int, plan: int, ks: int, stream=None) -> None:
    _chk(lib().hx_matmul_plan_bind_keys(ctx, plan, ks, _stream(stream)))


def hx_matmul_plan_bound_bytes(plan: int) -> int:
    return int(lib().hx_matmul_plan_bound_bytes(plan))


def hx_matmul_plan_destroy(plan: int) -> None:
    lib().hx_matmul_plan_destroy(plan)


def hx_matmul_rotation_steps(ctx: int, h: int, limbs: int) -> list:
    buf = np.zeros(4096, dtype=np.int32)
    n = _chk(lib().hx_matmul_rotation_steps(ctx, h, limbs, buf.ctypes.data_as(P_i32), buf.size))
    return [int(x) for x in buf[:n]]


def hx_context_set_plan_cache(ctx: int, bytes_cap: int) -> None:
    _chk(lib().hx_context_set_plan_cache(ctx, int(bytes_cap)))


def hx_context_plan_cache_info(ctx: int) -> dict:
    buf = np.zeros(4, dtype=np.uint64)
    _chk(lib().hx_context_plan_cache_info(ctx, _u64p(buf), 4))
    return {"plans": int(buf[0]), "bytes": int(buf[1]), "cap": int(buf[2]), "evicted": int(buf[3])}


def hx_matmul(ctx, ks, A, B, h, stream=None) -> int:
    return _op("hx_matmul", ctx, ks, A, B, h, stream=stream)


def hx_matmul_batch(ctx, ks, plan, As, Bs, h, stream=None) -> list:
    n = len(As)
    if len(Bs) != n:
        raise ValueError("A and B batches differ in length")
    a = (c_vp * n)(*As)
    b = (c_vp * n)(*Bs)
    outs = (c_vp * n)()
    _chk(lib().hx_matmul_batch(ctx, ks, plan, a, b, h, n, outs, _stream(stream)))
    return [outs[i] for i in range(n)]


def hx_matmul_batch_mixed(ctx: int, ks: int, A, B, h, stream=None) -> list:
    """Products A[i] . B[i] with their own matrix size h[i] (grouped by size and level inside)."""
    n = len(A)
    if len(B) != n or len(h) != n or n == 0:
        raise ValueError("A, B and h need one entry each per product")
    a, b, out = (c_vp * n)(*A), (c_vp * n)(*B), (c_vp * n)()
    hs = np.ascontiguousarray(np.asarray(h, dtype=np.int32))
    _chk(lib().hx_matmul_batch_mixed(ctx, ks, a, b, hs.ctypes.data_as(P_i32), n, out, _stream(stream)))
    return [out[i] for i in range(n)]


class _MatmulJob(ctypes.Structure):
    _fields_ = [("ctx", c_vp), ("ks", c_vp), ("A", c_vp), ("B", c_vp), ("h", c_int)]


class _RotateJob(ctypes.Structure):
    _fields_ = [("ctx", c_vp), ("ks", c_vp), ("ct", c_vp), ("step", c_i64)]


def hx_rotate_jobs(jobs, stream=None) -> list:
    """Rotations over several rings in one call, each key-switching stage one launch over all of
    them: jobs = [(ctx, ks, ct, step), ...]; returns one handle per job (of that job's context)."""
    n = len(jobs)
    if n == 0:
        raise ValueError("no jobs")
    arr = (_RotateJob * n)(*[_RotateJob(*j) for j in jobs])
    out = (c_vp * n)()
    _chk(lib().hx_rotate_jobs(arr, n, out, _stream(stream)))
    return [out[i] for i in range(n)]


def hx_matmul_jobs(jobs, stream=None) -> list:
    """Products over several rings in one call: jobs = [(ctx, ks, A, B, h), ...]; returns one
    product handle per job (of that job's context)."""
    n = len(jobs)
    if n == 0:
        raise ValueError("no jobs")
    arr = (_MatmulJob * n)(*[_MatmulJob(*j) for j in jobs])
    out = (c_vp * n)()
    _chk(lib().hx_matmul_jobs(arr, n, out, _stream(stream)))
    return [out[i] for i in range(n)]


def hx_rmatmul_batch(ctx, ks, plan, Ats, Bs, h, t, stream=None) -> list:
    n = len(Ats)
    if len(Bs) != n:
        raise ValueError("A and B batches differ in length")
    a = (c_vp * n)(*Ats)
    b = (c_vp * n)(*Bs)
    outs = (c_vp * n)()
    _chk(lib().hx_rmatmul_batch(ctx, ks, plan, a, b, h, t, n, outs, _stream(stream)))
    return [outs[i] for i in range(n)]


def hx_rmatmul_rotation_steps(ctx: int, h: int, t: int, limbs: int) -> list:
    buf = np.zeros(4096, dtype=np.int32)
    n = _chk(lib().hx_rmatmul_rotation_steps(ctx, h, t, limbs, buf.ctypes.data_as(P_i32), buf.size))
    return [int(x) for x in buf[:n]]


def hx_transpose_plan_create(ctx: int, h: int, limbs: int) -> int:
    out = _out()
    _chk(lib().hx_transpose_plan_create(ctx, h, limbs, ctypes.byref(out)))
    return out.value


def hx_transpose_rotation_steps(ctx: int, h: int) -> list:
    buf = np.zeros(4096, dtype=np.int32)
    n = _chk(lib().hx_transpose_rotation_steps(ctx, h, buf.ctypes.data_as(P_i32), buf.size))
    return [int(x) for x in buf[:n]]


def hx_transpose(ctx, ks, plan, xs, h, stream=None) -> list:
    n = len(xs)
    a = (c_vp * n)(*xs)
    outs = (c_vp * n)()
    _chk(lib().hx_transpose(ctx, ks, plan, a, h, n, outs, _stream(stream)))
    return [outs[i] for i in range(n)]


def hx_matmul_exec_create(ctx, ks, plan, count, scale) -> int:
    out = _out()
    _chk(lib().hx_matmul_exec_create(ctx, ks, plan, count, float(scale), ctypes.byref(out)))
    return out.value


def hx_matmul_exec_run(ex, As, Bs, stream=None) -> list:
    n = len(As)
    if len(Bs) != n:
        raise ValueError("A and B batches differ in length")
    a = (c_vp * n)(*As)
    b = (c_vp * n)(*Bs)
    outs = (c_vp * n)()
    _chk(lib().hx_matmul_exec_run(ex, a, b, outs, _stream(stream)))
    return [outs[i] for i in range(n)]


def hx_matmul_exec_run_host(ex, host_a: int, host_b: int, host_out: int, stream=None) -> None:
    """host_a, host_b, host_out: host addresses of [count][2][limbs][N] words (page-locked for
    asynchronous copies); returns once the copies and the replay are enqueued."""
    _chk(lib().hx_matmul_exec_run_host(ex, host_a, host_b, host_out, _stream(stream)))


def hx_matmul_exec_out_info(ex):
    limbs, scale = c_int(), c_double()
    _chk(lib().hx_matmul_exec_out_info(ex, ctypes.byref(limbs), ctypes.byref(scale)))
    return limbs.value, scale.value


def hx_matmul_exec_launches(ex) -> int:
    return _chk(lib().hx_matmul_exec_launches(ex))


def hx_matmul_exec_destroy(ex) -> None:
    lib().hx_matmul_exec_destroy(ex)


# ---- sign / ReLU -------------------------------------------------------------------

def hx_sign_approx(ctx, ks, x, d, k, relu=False, allow_refresh=True, refresh_seed=0, stream=None) -> int:
    return _op("hx_sign_approx", ctx, ks, x, d, k, int(relu), int(allow_refresh), refresh_seed, stream=stream)


def hx_sign_approx_batch(ctx, ks, xs, d, k, relu=False, allow_refresh=True, refresh_seed=0, stream=None) -> list:
    n = len(xs)
    a = (c_vp * n)(*xs)
    outs = (c_vp * n)()
    _chk(lib().hx_sign_approx_batch(ctx, ks, a, n, d, k, int(relu), int(allow_refresh), refresh_seed, outs,
                                    _stream(stream)))
    return [outs[i] for i in range(n)]


# ---- dense layer (Fig. 5) ----------------------------------------------------------------

def hx_dense_layer(ctx, ks, W, X, G, h, n_out, groups, d, k, input_div, refresh_seed=0, plans=(0, 0, 0),
                   stream=None):
    """W: n_out*groups handles (i-major), X: groups handles, G: n_out handles; plans: (feedforward,
    transpose, backpropagation) plan handles, 0 for the cached ones; returns (E, M, dW)."""
    if n_out >= 1 and groups >= 1 and (len(W) != n_out * groups or len(X) != groups or len(G) != n_out):
        raise ValueError("need n_out*groups weights, groups inputs and n_out gradients")
    w = (c_vp * len(W))(*W)
    x = (c_vp * len(X))(*X)
    g = (c_vp * len(G))(*G)
    e = (c_vp * n_out)()
    m = (c_vp * n_out)()
    dw = (c_vp * (n_out * groups))()
    _chk(lib().hx_dense_layer(ctx, ks, plans[0], plans[1], plans[2], w, x, g, h, n_out, groups, d, k,
                              float(input_div), refresh_seed, e, m, dw, _stream(stream)))
    return [e[i] for i in range(n_out)], [m[i] for i in range(n_out)], [dw[i] for i in range(n_out * groups)]


def hx_dense_rotation_steps(ctx: int, h: int) -> list:
    buf = np.zeros(4096, dtype=np.int32)
    n = _chk(lib().hx_dense_rotation_steps(ctx, h, buf.ctypes.data_as(P_i32), buf.size))
    return [int(x) for x in buf[:n]]


# ---- collective protocols (Fig. 1 items 13-14) ---------------------------------------------

def hx_dkeyswitch(ctx, ks_from, ks_to, ct, seed, stream=None) -> int:
    return _op("hx_dkeyswitch", ctx, ks_from, ks_to, ct, seed, stream=stream)


def hx_dbootstrap(ctx, ks, ct, seed, stream=None) -> int:
    return _op("hx_dbootstrap", ctx, ks, ct, seed, stream=stream)


# ---- aggregation (Alg. 6) -----------------------------------------------------------------

def hx_aggregate(ctx, grads, n_parties, models, eta_over_bn, stream=None) -> list:
    """grads: n_parties*len(models) handles, party-major; returns the updated models."""
    count = len(models)
    if len(grads) != n_parties * count:
        raise ValueError("need n_parties * len(models) gradients")
    g = (c_vp * len(grads))(*grads)
    m = (c_vp * count)(*models)
    outs = (c_vp * count)()
    _chk(lib().hx_aggregate(ctx, g, n_parties, m, count, float(eta_over_bn), outs, _stream(stream)))
    return [outs[i] for i in range(count)]


# ---- serving ------------------------------------------------------------------------------

SERVER_STATS = ["completed", "batches", "largest_batch", "max_busy_lanes", "peak_admitted_bytes", "key_bytes",
                "budget_left", "pending", "expired"]


def hx_server_create(hbm_budget_bytes: int, n_lanes: int, max_batch: int) -> int:
    out = _out()
    _chk(lib().hx_server_create(int(hbm_budget_bytes), n_lanes, max_batch, ctypes.byref(out)))
    return out.value


def hx_server_register_keys(sv: int, ks: int) -> None:
    _chk(lib().hx_server_register_keys(sv, ks))


def hx_server_submit_matmul(sv, ctx, ks, A, B, h) -> int:
    rid = c_u64()
    _chk(lib().hx_server_submit_matmul(sv, ctx, ks, A, B, h, ctypes.byref(rid)))
    return rid.value


def hx_server_submit_sign(sv, ctx, ks, x, d, k, relu=False, refresh_seed=0) -> int:
    rid = c_u64()
    _chk(lib().hx_server_submit_sign(sv, ctx, ks, x, d, k, int(relu), refresh_seed, ctypes.byref(rid)))
    return rid.value


def hx_server_submit_rotate(sv, ctx, ks, x, step) -> int:
    rid = c_u64()
    _chk(lib().hx_server_submit_rotate(sv, ctx, ks, x, int(step), ctypes.byref(rid)))
    return rid.value


def hx_server_poll(sv: int, wait: bool = True, cap: int = 256) -> list:
    """[(id, result handle or None, status, latency ms)]"""
    ids = np.zeros(cap, dtype=np.uint64)
    res = (c_vp * cap)()
    st = np.zeros(cap, dtype=np.int32)
    lat = np.zeros(cap, dtype=np.float64)
    n = _chk(lib().hx_server_poll(sv, int(bool(wait)), _u64p(ids), res, st.ctypes.data_as(P_i32),
                                  lat.ctypes.data_as(P_dbl), cap))
    return [(int(ids[i]), res[i], int(st[i]), float(lat[i])) for i in range(n)]


def hx_server_stats(sv: int) -> dict:
    buf = np.zeros(len(SERVER_STATS), dtype=np.uint64)
    n = _chk(lib().hx_server_stats(sv, _u64p(buf), len(SERVER_STATS)))
    return {SERVER_STATS[i]: int(buf[i]) for i in range(min(n, len(SERVER_STATS)))}


def hx_server_set_deadline(sv: int, rid: int, ms: float) -> None:
    _chk(lib().hx_server_set_deadline(sv, rid, float(ms)))


def hx_server_pause(sv: int, paused: bool) -> None:
    _chk(lib().hx_server_pause(sv, int(bool(paused))))


def hx_server_destroy(sv: int) -> None:
    lib().hx_server_destroy(sv)


# ---- counters ------------------------------------------------------------------------

def hx_alu_calibrate(ctx: int, stream=None):
    """(Shoup products per second, 128-bit multiply-accumulates per second) measured on the device."""
    a, b = c_double(), c_double()
    _chk(lib().hx_alu_calibrate(ctx, ctypes.byref(a), ctypes.byref(b), _stream(stream)))
    return a.value, b.value


def hx_counters(ctx: int) -> dict:
    buf = np.zeros(16, dtype=np.uint64)
    n = _chk(lib().hx_counters(ctx, _u64p(buf), buf.size))
    return {COUNTERS[i]: int(buf[i]) for i in range(n)}


def hx_counters_reset(ctx: int) -> None:
    lib().hx_counters_reset(ctx)


# ---- autotuning --------------------------------------------------------------------------

def hx_autotune(ctx: int, stream=None) -> list:
    """Picks the fastest NTT variants on this device for each bucket of batch sizes; returns
    those of the 256-limb bucket per phase (forward column, forward row, inverse column,
    inverse row) as signed tile widths (negative: swapped radices)."""
    arr = np.zeros(4, dtype=np.int32)
    _chk(lib().hx_autotune(ctx, arr.ctypes.data_as(P_i32), _stream(stream)))
    return [int(x) for x in arr]


def hx_ntt_tuning(ctx: int) -> list:
    """The autotuner's table: per bucket {max_limbs, tuned_limbs, widths[4] (signed widths),
    split (of an odd log N: 1 when the column phase takes the larger half of the stages)}."""
    out = np.zeros(64, dtype=np.int32)
    n = _chk(lib().hx_ntt_tuning(ctx, out.ctypes.data_as(P_i32), out.size))
    return [{"max_limbs": int(out[i]), "tuned_limbs": int(out[i + 1]), "widths": [int(x) for x in out[i + 2:i + 6]],
             "split": int(out[i + 6])} for i in range(0, n, 7)]


def hx_ntt_split(ctx: int, split: int) -> None:
    """Sets the split of an odd log N between the NTT phases for every bucket (0: the column phase
    takes floor(log N / 2) stages, 1: the other half)."""
    _chk(lib().hx_ntt_split(ctx, int(split)))


def hx_ntt_tiles(ctx: int, widths=None) -> list:
    """Sets the NTT variants per phase for every batch bucket (if given; signed tile widths 4,
    8, 16, 32, negative for swapped radices) and returns those of the 256-limb bucket."""
    get = np.zeros(4, dtype=np.int32)
    setp = None
    if widths is not None:
        arr = np.ascontiguousarray(np.array(widths, dtype=np.int32))
        setp = arr.ctypes.data_as(P_i32)
    _chk(lib().hx_ntt_tiles(ctx, setp, get.ctypes.data_as(P_i32)))
    return [int(x) for x in get]


# ---- profiling --------------------------------------------------------------------------

def hx_profile_enable(ctx: int, on: bool) -> None:
    _chk(lib().hx_profile_enable(ctx, int(bool(on))))


def hx_profile_read(ctx: int) -> dict:
    """{class name: (launches, total ms, algorithmic bytes)} for the classes with launches."""
    out = {}
    i = 0
    while True:
        name = ctypes.create_string_buffer(64)
        n, ms, b = c_u64(), c_double(), c_double()
        total = _chk(lib().hx_profile_read(ctx, i, name, 64, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(b)))
        if n.value:
            out[name.value.decode()] = (int(n.value), ms.value, b.value)
        i += 1
        if i >= total:
            return out
