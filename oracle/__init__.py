"""CPU oracle for the RNS-CKKS hot path of the Hercules method -- TEST
INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import, call, link or execute anything under oracle/.  It shares no code with
the CUDA library (paper_2207_04620_gb300/): both follow the same written
specification, each in its own code.

Parity status: every function here is pinned by tests/test_oracle_*.py
against definitions (direct NTT evaluation, schoolbook convolution, CRT with
Python integers, sympy primality), against values printed in the paper
(tests/golden/) or against FP64 plaintext results.  Nothing is "parity
unpinned".
"""
