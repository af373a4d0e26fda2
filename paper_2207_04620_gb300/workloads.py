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
    "cfg3_dense784x128_n15": dict(log_n=15, q_bits=[60] + [40] * 15, p_bits=[60] * 3, log2_scale=40, h=64, rows=128,
                                  n_in=784, batch=64, d=4, k=8, input_div=4.0),
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


def dense_inputs(seed: int, rows: int, n_in: int, batch: int, w_sigma: float = 0.05, g_sigma: float = 0.1):
    """Weights N(0, w_sigma) of shape rows x n_in, inputs U[0,1] of shape n_in x batch (one input per
    column) and an upstream gradient N(0, g_sigma) of shape rows x batch."""
    rng = np.random.default_rng(seed)
    return (rng.normal(0.0, w_sigma, (rows, n_in)), rng.uniform(0.0, 1.0, (n_in, batch)),
            rng.normal(0.0, g_sigma, (rows, batch)))


def blocks(M, h: int) -> list:
    """h x h blocks of M zero-padded to multiples of h, as a list of block rows."""
    M = np.asarray(M)
    r, c = -(-M.shape[0] // h), -(-M.shape[1] // h)
    P = np.zeros((r * h, c * h))
    P[: M.shape[0], : M.shape[1]] = M
    return [[P[i * h:(i + 1) * h, j * h:(j + 1) * h] for j in range(c)] for i in range(r)]


def dense_pack(W, X, G, h: int, beta: int):
    """Slot vectors of one dense layer: Wp[i][g] packs W_{i,j} for j = beta*g + p at position p,
    Xp[g] the X_j likewise, Gp[i] the gradient block G_i at position 0."""
    Wb, Xb, Gb = blocks(W, h), [r[0] for r in blocks(X, h)], [r[0] for r in blocks(G, h)]
    groups = -(-len(Xb) // beta)
    Wp = [[pack(Wb[i][g * beta:(g + 1) * beta], h, beta) for g in range(groups)] for i in range(len(Wb))]
    Xp = [pack(Xb[g * beta:(g + 1) * beta], h, beta) for g in range(groups)]
    Gp = [pack([Gb[i]], h, beta) for i in range(len(Gb))]
    return Wp, Xp, Gp


def residues(seed: int, primes, rows_per_prime: int, n: int) -> np.ndarray:
    """Uniform residues: array [rows_per_prime * len(primes), n], row r modulo primes[r % len(primes)]."""
    rng = np.random.default_rng(seed)
    out = np.empty((rows_per_prime, len(primes), n), dtype=np.uint64)
    for r in range(rows_per_prime):
        for i, q in enumerate(primes):
            out[r, i] = rng.integers(0, q, n, dtype=np.uint64)
    return out.reshape(-1, n)
