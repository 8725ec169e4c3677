"""Seeded synthetic workloads shaped like the paper's experiments (arXiv
1905.03525, Sec. 4: n = 2^k nodes, edge factor 16, Graph 500 parameters
a = 0.57, b = c = 0.19, d = 0.05, and the skewed a = 0.9, b = c = 0.025,
d = 0.05).  This module only draws inputs -- parameters, sizes, seeds and
arrival times -- with numpy's PCG64; it holds none of the generator's
arithmetic, so the library path and the CPU oracle can both consume it.
"""
from __future__ import annotations

import numpy as np

G500 = (0.57, 0.19, 0.19, 0.05)
SKEWED = (0.9, 0.025, 0.025, 0.05)


def noisy_levels(k: int, base=G500, amp: float = 0.05, seed: int = 34) -> np.ndarray:
    """Per-level parameters (k x 4): every one of a, b, c, d of every level
    moved by an independent U(-amp, amp), clipped at 0, then the row divided
    by its sum (smoothing by perturbed parameters, Sec. 3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P = np.asarray(base, np.float64)[None, :] + rng.uniform(-amp, amp, size=(k, 4))
    P = np.maximum(P, 0.0)
    return P / P.sum(axis=1, keepdims=True)


def batched_graphs(n: int = 4096, seed: int = 4096, k_range=(10, 24), log2m_range=(12.0, 26.0),
                   alpha=(57.0, 19.0, 19.0, 5.0)):
    """n graphs: k ~ U{k_range}, m = round(2^U(log2m_range)), (a, b, c, d) ~
    Dirichlet(alpha), per-graph seed = seed + index."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ks = rng.integers(k_range[0], k_range[1] + 1, size=n)
    ms = np.rint(np.exp2(rng.uniform(log2m_range[0], log2m_range[1], size=n))).astype(np.int64)
    P = rng.dirichlet(alpha, size=n)
    return [{"k": int(ks[i]), "m": int(ms[i]), "abcd": tuple(float(x) for x in P[i]),
             "seed": int(seed + i)} for i in range(n)]


def served_trace(n: int, rate: float = 2000.0, seed: int = 2000, k_range=(12, 30),
                 edge_factors=(4, 8, 16, 32), alpha=(57.0, 19.0, 19.0, 5.0)):
    """n requests with Poisson arrivals (mean `rate` per second): k ~ U{k_range},
    edge factor uniform in `edge_factors`, m = ef * 2^k, parameters ~
    Dirichlet(alpha), per-request seed = seed + index."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n)
    t = np.cumsum(gaps) - gaps[0]
    ks = rng.integers(k_range[0], k_range[1] + 1, size=n)
    efs = rng.choice(np.asarray(edge_factors), size=n)
    P = rng.dirichlet(alpha, size=n)
    return [{"arrival": float(t[i]), "k": int(ks[i]), "ef": int(efs[i]), "m": int(efs[i]) << int(ks[i]),
             "abcd": tuple(float(x) for x in P[i]), "seed": int(seed + i)} for i in range(n)]


# A 3 x 3 initiator for stochastic Kronecker graphs (Sec. 3): skewed toward
# the first cell like the Graph 500 2 x 2 parameters, rows and columns not
# symmetric.
KRON3 = ((0.40, 0.15, 0.05), (0.12, 0.10, 0.04), (0.06, 0.03, 0.05))
