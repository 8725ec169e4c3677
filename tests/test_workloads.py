"""The seeded input generators produce the workloads as stated: per-level
noise (C3), the batched graph mix (C4) and the served request trace (C5).
Properties only -- ranges, sums, means within sampling error, determinism."""
import numpy as np

from paper_1905_03525_gb300.workloads import G500, KRON3, SKEWED, batched_graphs, noisy_levels, served_trace


def test_parameter_sets():
    assert abs(sum(G500) - 1.0) < 1e-12 and abs(sum(SKEWED) - 1.0) < 1e-12
    assert abs(np.sum(KRON3) - 1.0) < 1e-12


def test_noisy_levels():
    P = noisy_levels(34)
    assert P.shape == (34, 4)
    assert np.all(P >= 0) and np.allclose(P.sum(axis=1), 1.0, atol=1e-12)
    # each entry moved by at most 0.05 before the row is renormalised (row sum within 1 +- 0.2)
    assert np.all(np.abs(P - np.asarray(G500)) < 0.05 / 0.8 + 0.05)
    assert np.array_equal(P, noisy_levels(34)) and not np.array_equal(P, noisy_levels(34, seed=35))


def test_batched_graphs_mix():
    gs = batched_graphs(4096)
    ks = np.array([g["k"] for g in gs])
    ms = np.array([g["m"] for g in gs])
    P = np.array([g["abcd"] for g in gs])
    assert ks.min() == 10 and ks.max() == 24 and len(set(ks.tolist())) == 15
    assert ms.min() >= 2 ** 12 and ms.max() <= 2 ** 26
    # log2 m uniform on [12, 26]: mean 19, standard deviation 14 / sqrt(12)
    assert abs(np.log2(ms).mean() - 19.0) < 5 * (14 / np.sqrt(12)) / np.sqrt(len(gs))
    assert np.allclose(P.sum(axis=1), 1.0, atol=1e-12) and np.all(P > 0)
    # Dirichlet(57, 19, 19, 5): mean (0.57, 0.19, 0.19, 0.05), var of a = 0.57 * 0.43 / 101
    assert np.all(np.abs(P.mean(axis=0) - np.array([0.57, 0.19, 0.19, 0.05])) < 5 * np.sqrt(0.57 * 0.43 / 101 / len(gs)))
    assert [g["seed"] for g in gs] == list(range(4096, 4096 + 4096))
    assert gs == batched_graphs(4096)


def test_served_trace():
    n, rate = 4096, 2000.0
    tr = served_trace(n, rate)
    t = np.array([r["arrival"] for r in tr])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    # exponential gaps with mean 1/rate: the mean of n - 1 gaps within 5 standard errors
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / rate) < 5 * (1 / rate) / np.sqrt(len(gaps))
    ks = np.array([r["k"] for r in tr])
    assert ks.min() == 12 and ks.max() == 30
    assert {r["ef"] for r in tr} == {4, 8, 16, 32}
    assert all(r["m"] == r["ef"] << r["k"] for r in tr)
    assert all(abs(sum(r["abcd"]) - 1.0) < 1e-12 for r in tr)
    assert tr == served_trace(n, rate)
