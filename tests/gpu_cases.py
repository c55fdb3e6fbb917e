"""Shared seeded cases for the GPU parity tests (inputs only; no method arithmetic)."""
import numpy as np

import workloads as W

# (name, dim, N, p, perturb, seed, leaf, pprime, levels, cheb_degree)
CASES = [
    ("2d_q2_32_config1", 2, 32, 2, 0.0, 0, 64, 1, 3, 2),
    ("3d_q3_4_pp2", 3, 4, 3, 0.2, 11, 64, 2, 3, 3),
    ("2d_q1_24_pp0", 2, 24, 1, 0.1, 5, 30, 0, 2, 3),
    ("3d_q2_6_pp1_L4", 3, 6, 2, 0.2, 7, 20, 1, 4, 3),
    ("2d_q4_9_pp2_ragged", 2, 9, 4, 0.15, 9, 37, 2, 3, 3),
]


def make(case):
    name, d, N, p, pert, seed, leaf, pp, L, k = case
    P = W.poisson(d, N, p, perturb=pert, seed=seed)
    params = dict(leaf_size=leaf, pprime=pp, levels=L, cheb_degree=k)
    return P, params
