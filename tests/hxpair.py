"""Test helpers: one parameter set built twice, in the CUDA library (through
its C ABI) and in the oracle, with the same seeds.  Inputs for both sides come
from the oracle or from paper_2207_04620_gb300.workloads only."""
from __future__ import annotations

import numpy as np

from oracle import ckks as C
from paper_2207_04620_gb300 import hx

PARAMS = {
    # config 0 of the benchmark: N=2^12, 60 + 40 + 40, special 60, scale 2^40
    "cfg0": dict(log_n=12, q_bits=[60, 40, 40], p_bits=[60], log2_scale=40),
    # small chain with 4 levels (Alg. 3) and two special primes
    "alg3": dict(log_n=12, q_bits=[60, 45, 45, 45, 45], p_bits=[60, 60], log2_scale=45),
    # the next ring with one more level (several-ring batches and serving)
    "alg3_13": dict(log_n=13, q_bits=[60, 45, 45, 45, 45, 45], p_bits=[60, 60], log2_scale=45),
    # config 1 of the benchmark: N=2^14, 60 + 7*45, two 60-bit special primes, scale 2^45
    "cfg1": dict(log_n=14, q_bits=[60] + [45] * 7, p_bits=[60, 60], log2_scale=45),
    # the sign chain of config 2 on a smaller ring: 60 + 15*40, three special primes
    "sign": dict(log_n=12, q_bits=[60] + [40] * 15, p_bits=[60] * 3, log2_scale=40),
    # config 2 itself: N=2^15
    "cfg2": dict(log_n=15, q_bits=[60] + [40] * 15, p_bits=[60] * 3, log2_scale=40),
    # the sign chain with key-switching digits of four primes (about P each)
    "sign_a4": dict(log_n=12, q_bits=[60] + [40] * 15, p_bits=[60] * 3, log2_scale=40, alpha=4),
}


class Pair:
    def __init__(self, name: str, n_parties: int = 2, seed: int = 1234, rot_steps=()):
        p = PARAMS[name]
        self.p = p
        self.octx = C.Context(p["log_n"], p["q_bits"], p["p_bits"], p["log2_scale"], alpha=p.get("alpha"))
        self.ctx = hx.hx_context_create(p["log_n"], p["q_bits"], p["p_bits"], p["log2_scale"], alpha=p.get("alpha", 0))
        assert hx.hx_context_primes(self.ctx) == self.octx.q + self.octx.p
        self.seed, self.n_parties = seed, n_parties
        self.rot_steps = list(rot_steps)
        self.oks = C.keygen(self.octx, n_parties, seed, rot_steps=self.rot_steps)
        self.ks = hx.hx_keygen(self.ctx, n_parties, seed, self.rot_steps)
        self.N = self.octx.N

    def close(self):
        hx.hx_keyset_destroy(self.ks)
        hx.hx_context_destroy(self.ctx)

    def to_lib(self, ct: C.Ciphertext) -> int:
        return hx.hx_ct_import(self.ctx, ct.c, ct.scale)

    def from_lib(self, h: int) -> C.Ciphertext:
        comps, limbs, scale = hx.hx_ct_info(h)
        return C.Ciphertext(hx.hx_ct_export(self.ctx, h), scale)

    def same(self, h: int, ct: C.Ciphertext) -> bool:
        got = self.from_lib(h)
        return got.c.shape == ct.c.shape and np.array_equal(got.c, ct.c) and got.scale == ct.scale

    def encrypt(self, slots, seed: int, limbs=None) -> C.Ciphertext:
        return C.encrypt(self.octx, self.oks, slots, seed, limbs=limbs)
