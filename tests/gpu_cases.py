"""Shared seeded cases for the GPU parity tests (inputs only; no method arithmetic)."""
import numpy as np

import workloads as W

# (name, dim, N, p, perturb, seed, leaf, pprime, levels, cheb_degree[, element])
# element "Q" (default): tensor-product Q_p cells; "P": P_p simplices of the Kuhn triangulation
CASES = [
    ("2d_q2_32_config1", 2, 32, 2, 0.0, 0, 64, 1, 3, 2),
    ("3d_q3_4_pp2", 3, 4, 3, 0.2, 11, 64, 2, 3, 3),
    ("2d_q1_24_pp0", 2, 24, 1, 0.1, 5, 30, 0, 2, 3),
    ("3d_q2_6_pp1_L4", 3, 6, 2, 0.2, 7, 20, 1, 4, 3),
    ("2d_q4_9_pp2_ragged", 2, 9, 4, 0.15, 9, 37, 2, 3, 3),
    ("2d_p2_simplex_24_pp1", 2, 24, 2, 0.1, 3, 64, 1, 3, 3, "P"),
    ("3d_p2_simplex_5_pp1", 3, 5, 2, 0.2, 13, 40, 1, 3, 3, "P"),
]


def make(case):
    name, d, N, p, pert, seed, leaf, pp, L, k = case[:10]
    element = case[10] if len(case) > 10 else "Q"
    if element == "P":
        P = W.poisson_simplex(d, N, p, perturb=pert, seed=seed)
    else:
        P = W.poisson(d, N, p, perturb=pert, seed=seed)
    params = dict(leaf_size=leaf, pprime=pp, levels=L, cheb_degree=k)
    return P, params
