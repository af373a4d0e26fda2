"""Seeded synthetic inputs with the shapes of the paper's workloads.

No CKKS arithmetic lives here: only random matrices and slot vectors, so the
same inputs can be handed to the CUDA library and to the oracle.
"""
from __future__ import annotations

import numpy as np

# Parameter sets of the benchmark configurations (prime sizes in bits).
CONFIGS = {
    "cfg0_matmul16_n12": dict(log_n=12, q_bits=[60, 40, 40], p_bits=[60], log2_scale=40, h=16),
    "cfg1_matmul64_n14": dict(log_n=14, q_bits=[60] + [45] * 7, p_bits=[60, 60], log2_scale=45, h=64, batch=32),
    "cfg2_sign_n15": dict(log_n=15, q_bits=[60] + [40] * 15, p_bits=[60] * 3, log2_scale=40, count=64, d=4, k=8),
}


def matrices(seed: int, count: int, h: int, low: float = -1.0, high: float = 1.0) -> list:
    """`count` h x h FP64 matrices with entries uniform in [low, high)."""
    rng = np.random.default_rng(seed)
    return [rng.uniform(low, high, (h, h)) for _ in range(count)]


def pack(mats, h: int, beta: int) -> np.ndarray:
    """Slot vector holding `beta` matrices interleaved: slot beta*(h*i+j)+k is (A_k)_{i,j}."""
    out = np.zeros(beta * h * h)
    for k, A in enumerate(mats):
        out[k::beta] = np.asarray(A).reshape(-1)
    return out


def unpack(slots, h: int, beta: int) -> list:
    return [np.asarray(slots[k: beta * h * h: beta]).reshape(h, h) for k in range(beta)]


def sign_inputs(seed: int, n: int, min_abs: float = 2.0 ** -8) -> np.ndarray:
    """n values uniform in [-1, -min_abs] U [min_abs, 1]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(min_abs, 1.0, n) * rng.choice([-1.0, 1.0], n)


def residues(seed: int, primes, rows_per_prime: int, n: int) -> np.ndarray:
    """Uniform residues: array [rows_per_prime * len(primes), n], row r modulo primes[r % len(primes)]."""
    rng = np.random.default_rng(seed)
    out = np.empty((rows_per_prime, len(primes), n), dtype=np.uint64)
    for r in range(rows_per_prime):
        for i, q in enumerate(primes):
            out[r, i] = rng.integers(0, q, n, dtype=np.uint64)
    return out.reshape(-1, n)
