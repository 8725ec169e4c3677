"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test checks the oracle against something the paper or mathematics fixes:
table sizes printed in Fig. 1, the Kronecker closed form of the R-MAT
process (Sec. 1), the Kraft equality of a complete prefix code, the greedy
max-min property of the table-construction fragment (Sec. 2), exact integer
alias-table reconstruction, an independent Philox implementation (PyTorch's
open-source engine header), and chi-square tests against closed-form
marginals.  A plausible slip in the oracle (b and c swapped, row and column
bits swapped, a wrong Philox word order, an off-by-one in the stop rule or in
the Vose loop) fails at least one of them.
"""
import itertools
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
G500 = (0.57, 0.19, 0.19, 0.05)
ASYM = (0.5, 0.2, 0.25, 0.05)  # b != c, so a b/c or row/col slip shows
SKEWED = (0.9, 0.03, 0.05, 0.02)


def kronecker(P_levels, k):
    """Closed form of the R-MAT process (Sec. 1): P(row, col) is the product
    over levels t of the quadrant probability selected by bit t of row and
    column (a: 0/0, b: 0/1, c: 1/0, d: 1/1)."""
    P = np.asarray(P_levels, np.float64).reshape(-1, 4)
    if P.shape[0] == 1:
        P = np.repeat(P, k, axis=0)
    n = 1 << k
    out = np.ones((n, n))
    r = np.arange(n)[:, None]
    c = np.arange(n)[None, :]
    for t in range(k):
        rb = (r >> (k - 1 - t)) & 1
        cb = (c >> (k - 1 - t)) & 1
        q = 2 * rb + cb
        out = out * P[t][q]
    return out


def read_sizes():
    rows = []
    with open(os.path.join(GOLDEN, "fig1_table_sizes.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kind, x, n = line.split()
            rows.append((kind, int(x), int(n)))
    return rows


# ---------------------------------------------------------------- Philox --

def _torch_philox_words(pairs, nwords):
    """Words from PyTorch's open-source at::philox_engine (header-only)."""
    import torch.utils.cpp_extension as cx
    src = ["#include <ATen/core/PhiloxRNGEngine.h>", "#include <cstdio>", "int main(){"]
    for seed, sub in pairs:
        src.append(f"{{ at::philox_engine e({seed}ULL, {sub}ULL, 0);"
                   f" for (int i = 0; i < {nwords}; ++i) printf(\"%u\\n\", e()); }}")
    src.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        cpp = os.path.join(d, "p.cpp")
        exe = os.path.join(d, "p")
        with open(cpp, "w") as f:
            f.write("\n".join(src))
        inc = [f"-I{p}" for p in cx.include_paths()]
        subprocess.run(["g++", "-std=c++17", *inc, cpp, "-o", exe], check=True,
                       stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return np.array([int(x) for x in out], np.uint64).reshape(len(pairs), nwords)


def test_philox_matches_independent_engine():
    pairs = [(0, 0), (1, 0), (1, 5), (2**64 - 1, 2**64 - 1), (0x123456789ABCDEF0, 2**32 + 7),
             (42, 2**35 - 1)]
    ref = _torch_philox_words(pairs, 12)
    for i, (seed, e) in enumerate(pairs):
        got = [oracle.word(seed, e, n) for n in range(12)]
        assert got == [int(x) for x in ref[i]], (seed, e)


def test_philox_block_layout():
    # word n of edge e is word n % 4 of block (q = n // 4, e).
    seed, e = 0xDEADBEEF12345678, 987654321012
    for n in range(10):
        q = n // 4
        ctr = [q & 0xFFFFFFFF, q >> 32, e & 0xFFFFFFFF, e >> 32]
        blk = oracle.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32])
        assert oracle.word(seed, e, n) == int(blk[n % 4])


# ---------------------------------------------------------- table sizes --

@pytest.mark.parametrize("kind,x,n", [r for r in read_sizes() if (r[0] == "variable" and r[1] <= 20)
                                      or (r[0] == "fixed" and r[1] <= 9)])
def test_table_sizes_fig1(kind, x, n):
    if kind == "variable":
        t = oracle.Table.variable(*G500, 30, 1 << x)
        assert t.entries == n
        t2 = oracle.Table.variable(0.9, 0.025, 0.025, 0.05, 64, 1 << x)  # Fig. 1 skewed series
        assert t2.entries == n
    else:
        t = oracle.Table.fixed([G500], x)
        assert t.entries == n
    assert t.bits == math.ceil(math.log2(n))


# ------------------------------------------------------ prefix-code shape --

def _paths(t):
    out = []
    for i in range(t.entries):
        L = int(t.len[i])
        s = int(t.sym[i])
        out.append(tuple((s >> (62 - 2 * j)) & 3 for j in range(L)))
    return out


@pytest.mark.parametrize("params,k,bound", [(G500, 26, 4096), (ASYM, 20, 1000),
                                             ((0.9, 0.025, 0.025, 0.05), 64, 8192),
                                             (G500, 6, 4096)])
def test_variable_table_is_complete_prefix_code(params, k, bound):
    t = oracle.Table.variable(*params, k, bound)
    paths = _paths(t)
    Lmax = max(len(p) for p in paths)
    # Kraft equality of a complete 4-ary prefix code, in exact integers.
    assert sum(4 ** (Lmax - len(p)) for p in paths) == 4 ** Lmax
    # Canonical (lexicographic) order and no entry is a prefix of the next.
    for x, y in zip(paths, paths[1:]):
        assert x < y and y[:len(x)] != x
    assert Lmax <= min(k, 32)


@pytest.mark.parametrize("params,k,bound", [(G500, 26, 4096), (ASYM, 26, 2000),
                                             ((0.9, 0.025, 0.025, 0.05), 64, 8192)])
def test_variable_table_greedy_maxmin(params, k, bound):
    """The table-construction fragment always expands the most probable entry,
    so every expanded (internal) node is at least as probable as every leaf
    that could still have been expanded."""
    t = oracle.Table.variable(*params, k, bound)
    paths = _paths(t)
    P = dict(zip(range(4), params))
    s = sum(params)
    def prob(path):
        p = 1.0
        for sym in path:
            p = p * (P[sym] / s)
        return p
    internal = {p[:j] for p in paths for j in range(len(p))}
    cap = min(k, 32)
    min_internal = min(prob(x) for x in internal)
    max_open_leaf = max(prob(p) for p in paths if len(p) < cap)
    assert max_open_leaf <= min_internal
    # Leaf probabilities recomputed from the symbols agree with the table.
    for i, path in enumerate(paths):
        assert t.p[i] == prob(path)


def test_depth_cap_gives_full_fixed_table():
    # With k = 3 every path stops at depth 3: the table is all 64 paths.
    v = oracle.Table.variable(*ASYM, 3, 4096)
    f = oracle.Table.fixed([ASYM], 3)
    assert v.entries == 64
    assert np.array_equal(v.sym[:64], f.sym[:64])
    assert np.array_equal(v.p[:64], f.p[:64])
    assert np.array_equal(v.w[:64], f.w[:64])


# ----------------------------------------------------- quantise + alias --

@pytest.mark.parametrize("maker", [
    lambda: oracle.Table.variable(*G500, 26, 4096),
    lambda: oracle.Table.variable(*ASYM, 16, 300),
    lambda: oracle.Table.variable(0.9, 0.025, 0.025, 0.05, 64, 8192),
    lambda: oracle.Table.fixed([G500], 4),
    lambda: oracle.Table.fixed([ASYM], 6),
    lambda: oracle.Table.fixed([(1.0, 0.0, 0.0, 0.0)], 2),
])
def test_weights_and_alias_roundtrip(maker):
    t = maker()
    N = 1 << t.bits
    C = 1 << (32 - t.bits)
    w = t.w.astype(object)
    assert sum(w) == 2 ** 32
    # |w_i - p_i 2^32| < 1 and the +1s went to the largest fractional parts.
    x = [math.ldexp(float(pi), 32) for pi in t.p]
    frac = [xi - math.floor(xi) for xi in x]
    bumped = [int(w[i]) - math.floor(x[i]) for i in range(N)]
    assert all(b in (0, 1) for b in bumped)
    if any(bumped) and not all(bumped):
        assert min(frac[i] for i in range(N) if bumped[i]) >= max(frac[i] for i in range(N) if not bumped[i])
    # Rebuild the weights from the alias table: column j gives thr_j to j and
    # C - thr_j to alias_j (C to j when it aliases itself).
    rebuilt = [0] * N
    for j in range(N):
        a = int(t.alias[j])
        th = int(t.thr[j])
        assert 0 <= th < C and 0 <= a < N
        if a == j:
            rebuilt[j] += C
        else:
            rebuilt[j] += th
            rebuilt[a] += C - th
    assert rebuilt == [int(v) for v in w]


def test_draw_frequencies_match_weights():
    t = oracle.Table.fixed([ASYM], 3)  # 64 entries, b = 6
    rng = np.random.default_rng(7)
    us = rng.integers(0, 2 ** 32, size=200_000, dtype=np.uint64)
    counts = np.zeros(1 << t.bits)
    for u in us:
        counts[t.draw(int(u))] += 1
    expected = t.w.astype(np.float64) / 2 ** 32 * len(us)
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert stats.chi2.sf(chi2, len(counts) - 1) > 1e-3


# -------------------------------------------- exact edge distributions --

def _distribution_cases():
    yield "fixed l=4, k=4 (G500)", [oracle.Table.fixed([G500], 4)], G500, 4
    yield "fixed l=4, k=4 (asym)", [oracle.Table.fixed([ASYM], 4)], ASYM, 4
    yield "fixed l=1, k=4", [oracle.Table.fixed([ASYM], 1)], ASYM, 4
    yield "fixed l=3, k=4 (cut)", [oracle.Table.fixed([ASYM], 3)], ASYM, 4
    yield "variable 2^12, k=4", [oracle.Table.variable(*ASYM, 4, 4096)], ASYM, 4
    yield "variable 2^12, k=5 (cap)", [oracle.Table.variable(*ASYM, 5, 4096)], ASYM, 5
    yield "variable 2^6, k=5", [oracle.Table.variable(*ASYM, 5, 64)], ASYM, 5
    yield "variable 2^9, k=6", [oracle.Table.variable(*G500, 6, 512)], G500, 6
    rng = np.random.default_rng(3)
    Pl = rng.dirichlet([5, 3, 2, 1], size=5)
    yield "levels l=2, k=5", oracle.level_groups(Pl, 5, 2), Pl, 5
    yield "levels l=3, k=5", oracle.level_groups(Pl, 5, 3), Pl, 5


@pytest.mark.parametrize("name,tables,P,k", list(_distribution_cases()), ids=lambda v: v if isinstance(v, str) else "")
def test_exact_distribution_equals_kronecker(name, tables, P, k):
    dist = oracle.edge_distribution(tables, k, quantised=False)
    ref = kronecker(P, k)
    assert np.abs(dist - ref).max() <= 1e-12
    # After quantisation every entry's probability moves by < 2^-32, so a
    # cell reached through at most D draws moves by < D * (entries per draw)
    # * 2^-32.
    q = oracle.edge_distribution(tables, k, quantised=True)
    assert abs(q.sum() - 1.0) <= 1e-12
    draws = len(tables) if len(tables) > 1 else math.ceil(k / min(int(l) for l in tables[0].len[:tables[0].entries]))
    n_max = max(1 << t.bits for t in tables)
    assert np.abs(q - ref).max() <= draws * n_max * 2.0 ** -32


# ------------------------------------------------------- sampled output --

def _quadrant_counts(row, col, k):
    counts = np.zeros((k, 4))
    for t in range(k):
        rb = (row >> np.uint64(k - 1 - t)) & np.uint64(1)
        cb = (col >> np.uint64(k - 1 - t)) & np.uint64(1)
        q = (2 * rb + cb).astype(np.int64)
        counts[t] = np.bincount(q, minlength=4)
    return counts


def _chi2_pvalue(counts, probs):
    expected = probs * counts.sum()
    keep = expected > 0
    chi2 = (((counts - expected) ** 2)[keep] / expected[keep]).sum()
    return stats.chi2.sf(chi2, keep.sum() - 1)


@pytest.mark.parametrize("sampler", ["alias_variable", "alias_fixed", "naive"])
def test_per_level_quadrant_frequencies(sampler):
    k, m = 12, 1 << 19
    if sampler == "alias_variable":
        row, col = oracle.generate([oracle.Table.variable(*ASYM, k, 4096)], k, 11, 0, m)
    elif sampler == "alias_fixed":
        row, col = oracle.generate([oracle.Table.fixed([ASYM], 5)], k, 12, 0, m)
    else:
        row, col = oracle.generate_naive([ASYM], k, 13, 0, m)
    counts = _quadrant_counts(row, col, k)
    for t in range(k):
        assert _chi2_pvalue(counts[t], np.array(ASYM)) > 1e-3, t
    # Row bit 1 w.p. c + d, column bit 1 w.p. b + d, at every level.
    for t in range(k):
        assert abs(counts[t][2:].sum() / m - (ASYM[2] + ASYM[3])) < 5 * math.sqrt(0.25 / m)
        assert abs(counts[t][[1, 3]].sum() / m - (ASYM[1] + ASYM[3])) < 5 * math.sqrt(0.25 / m)


@pytest.mark.parametrize("ell", [2, 3])
def test_per_level_generation_follows_each_levels_parameters(ell):
    """Per-level tables (one fixed-l table per group of l levels): generated
    edges take level t's quadrant with level t's own parameters, and the
    joint law of all k = 6 levels is their Kronecker product."""
    k, m = 6, 1 << 19
    P = np.random.default_rng(40 + ell).dirichlet([6, 3, 2, 1], size=k)
    row, col = oracle.generate(oracle.level_groups(P, k, ell), k, 21, 0, m)
    counts = _quadrant_counts(row, col, k)
    for t in range(k):
        assert _chi2_pvalue(counts[t], P[t]) > 1e-3, t
    joint = np.bincount(row.astype(np.int64) * (1 << k) + col.astype(np.int64), minlength=1 << (2 * k)).astype(float)
    probs = kronecker(P, k).ravel()
    small = probs * m < 5  # cells expecting fewer than 5 edges are pooled into one
    cc = np.concatenate([[joint[small].sum()], joint[~small]])
    pp = np.concatenate([[probs[small].sum()], probs[~small]])
    assert _chi2_pvalue(cc, pp) > 1e-3


def test_full_joint_distribution_k6():
    k, m = 6, 1 << 20
    t = oracle.Table.variable(*ASYM, k, 700)
    row, col = oracle.generate([t], k, 5, 0, m)
    counts = np.bincount((row.astype(np.int64) << k) | col.astype(np.int64), minlength=1 << (2 * k))
    probs = oracle.edge_distribution([t], k, quantised=True).ravel()
    # pool cells with small expectation
    order = np.argsort(probs)
    exp_sorted = probs[order] * m
    small = np.cumsum(exp_sorted) < 50
    c_small, p_small = counts[order][small].sum(), probs[order][small].sum()
    c = np.concatenate([[c_small], counts[order][~small]])
    p = np.concatenate([[p_small], probs[order][~small]])
    assert _chi2_pvalue(c, p) > 1e-3
    assert np.abs(probs - kronecker(ASYM, k).ravel()).max() < 1e-8


def test_two_sample_alias_vs_naive():
    k, m = 8, 1 << 19
    ra, ca = oracle.generate([oracle.Table.variable(*ASYM, k, 2048)], k, 21, 0, m)
    rn, cn = oracle.generate_naive([ASYM], k, 22, 0, m)
    # degree-like statistics: row histogram and column histogram
    for xa, xn in ((ra, rn), (ca, cn)):
        ha = np.bincount(xa.astype(np.int64), minlength=1 << k)
        hn = np.bincount(xn.astype(np.int64), minlength=1 << k)
        keep = (ha + hn) > 20
        table = np.vstack([ha[keep], hn[keep]])
        p = stats.chi2_contingency(table)[1]
        assert p > 1e-3


def test_undirected_mirrors_lower_triangle():
    k, m = 5, 1 << 18
    t = oracle.Table.fixed([ASYM], 5)
    r, c = oracle.generate([t], k, 9, 0, m, undirected=True)
    assert np.all(r <= c)
    rd, cd = oracle.generate([t], k, 9, 0, m, undirected=False)
    assert np.array_equal(r, np.minimum(rd, cd)) and np.array_equal(c, np.maximum(rd, cd))
    K = kronecker(ASYM, k)
    fold = np.triu(K + K.T) - np.diag(np.diag(K))
    counts = np.bincount((r.astype(np.int64) << k) | c.astype(np.int64), minlength=1 << (2 * k))
    keep = fold.ravel() > 0
    assert counts[~keep].sum() == 0
    assert _chi2_pvalue(counts[keep].astype(float), fold.ravel()[keep]) > 1e-3


def test_edges_depend_only_on_global_index():
    t = oracle.Table.variable(*G500, 26, 4096)
    r0, c0 = oracle.generate([t], 26, 77, 1000, 64)
    r1, c1 = oracle.generate([t], 26, 77, 990, 100)
    assert np.array_equal(r0, r1[10:74]) and np.array_equal(c0, c1[10:74])
    r2, _ = oracle.generate([t], 26, 78, 1000, 64)
    assert not np.array_equal(r0, r2)


def test_edge_uses_words_in_order():
    # Fixed l=4, k=16: edge e uses exactly words 0..3 of its stream, one per
    # draw, top levels first.
    t = oracle.Table.fixed([G500], 4)
    seed, e = 5, 123456
    row, col = oracle.generate([t], 16, seed, e, 1)
    r = c = 0
    for n in range(4):
        sel = t.draw(oracle.word(seed, e, n))
        for j in range(4):
            s = (int(t.sym[sel]) >> (62 - 2 * j)) & 3
            r = (r << 1) | (s >> 1)
            c = (c << 1) | (s & 1)
    assert (int(row[0]), int(col[0])) == (r, c)
    # fixed tables: entry index = path digits
    assert all(int(t.sym[i]) >> 56 == i for i in range(256))


# ------------------------------------------------------ Sec. 2 numbers --

def test_entropy_and_gain_sec2():
    vals = {}
    with open(os.path.join(GOLDEN, "sec2_entropy.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k_, v = line.split()
                vals[k_] = float(v)
    P = [vals[x] for x in "abcd"]
    H = -sum(p * math.log2(p) for p in P)
    assert round(H, 2) == vals["H"]
    assert round(2 / H, 2) == vals["gain"]
    # The variable table of 4093 entries yields about 2/H times more levels
    # per draw than the fixed table of 4096 entries (6 levels).
    t = oracle.Table.variable(*P, 30, 4096)
    mean_len = float((t.p * t.len).sum())
    assert abs(mean_len / 6 - 2 / H) < 0.1


def test_invalid_arguments_rejected():
    with pytest.raises(ValueError):
        oracle.Table.variable(0.5, 0.5, 0.5, 0.5, 10, 4096)  # sum != 1
    with pytest.raises(ValueError):
        oracle.Table.variable(*G500, 10, 4)  # bound < 5
    with pytest.raises(ValueError):
        oracle.Table.variable(-0.1, 0.5, 0.5, 0.1, 10, 4096)
    with pytest.raises(ValueError):
        oracle.Table.fixed([G500], 13)


def test_draw_keeps_column_with_probability_thr_over_C_exactly():
    """Walker's alias method: a draw landing in column j keeps j for exactly
    thr[j] of the C residuals and yields alias[j] for the others.  With a
    4^12-entry table C = 256, so every residual of a column can be tried; with
    the exact weight reconstruction above this pins P(entry) = w / 2^32."""
    t = oracle.Table.fixed([ASYM], 12)
    b = t.bits
    C = 1 << (32 - b)
    for j in list(range(0, 1 << b, 262139))[:64]:
        sel = [t.draw((j << (32 - b)) | r) for r in range(C)]
        keep = sum(1 for s in sel if s == j)
        if int(t.alias[j]) == j:
            assert keep == C
        else:
            assert keep == int(t.thr[j])
            assert all(s == t.alias[j] for s in sel[int(t.thr[j]):])


# ------------------------------------------------------------ scrambling --

@pytest.mark.parametrize("k,seed", [(1, 3), (2, 9), (5, 1), (12, 7), (16, 123456789)])
def test_scramble_is_a_bijection(k, seed):
    c = oracle.scramble_constants(seed, k)
    assert all(int(x) & 1 for x in c[0::2])            # multipliers odd
    assert all(int(x) < (1 << k) for x in c)
    imgs = [oracle.scramble(x, k, c) for x in range(1 << k)]
    assert sorted(imgs) == list(range(1 << k))
    if k >= 5:
        assert sum(1 for x, y in zip(range(1 << k), imgs) if x != y) > (1 << k) // 2


def test_scramble_relabels_vertices_only():
    """Scrambling is a relabelling: the scrambled graph has exactly the edges
    (pi(r), pi(c)) of the plain one, so its degree multiset is unchanged and
    its edge distribution is the Kronecker distribution moved by pi."""
    k, m = 6, 1 << 18
    t = oracle.Table.variable(*ASYM, k, 500)
    r0, c0 = oracle.generate([t], k, 31, 0, m)
    rs, cs = oracle.generate_scrambled([t], k, 99, 31, 0, m)
    consts = oracle.scramble_constants(99, k)
    pi = np.array([oracle.scramble(x, k, consts) for x in range(1 << k)], np.uint64)
    assert np.array_equal(rs, pi[r0.astype(np.int64)]) and np.array_equal(cs, pi[c0.astype(np.int64)])
    deg0 = np.sort(np.bincount(r0.astype(np.int64), minlength=1 << k))
    degs = np.sort(np.bincount(rs.astype(np.int64), minlength=1 << k))
    assert np.array_equal(deg0, degs)
    K = kronecker(ASYM, k)
    moved = np.zeros_like(K)
    moved[np.ix_(pi.astype(np.int64), pi.astype(np.int64))] = K
    counts = np.bincount((rs.astype(np.int64) << k) | cs.astype(np.int64), minlength=1 << (2 * k)).astype(float)
    probs = moved.ravel()
    order = np.argsort(probs)
    small = np.cumsum(probs[order] * m) < 50
    cc = np.concatenate([[counts[order][small].sum()], counts[order][~small]])
    pp = np.concatenate([[probs[order][small].sum()], probs[order][~small]])
    assert _chi2_pvalue(cc, pp) > 1e-3


# ------------------------------------------------------ partitioned graphs --

def _binned_gof(samples, n, p, min_expected=20.0):
    """Chi-square p-value of integer samples against the exact Bin(n, p) pmf
    (scipy), tails pooled until every bin expects >= min_expected."""
    samples = np.asarray(samples, np.int64)
    N = len(samples)
    lo = int(stats.binom.ppf(1e-7, n, p))
    hi = int(stats.binom.ppf(1 - 1e-7, n, p))
    xs = np.arange(lo, hi + 1)
    pmf = stats.binom.pmf(xs, n, p)
    pmf[0] += stats.binom.cdf(lo - 1, n, p)
    pmf[-1] += stats.binom.sf(hi, n, p)
    cnt = np.bincount(np.clip(samples, lo, hi) - lo, minlength=len(xs)).astype(float)
    # pool adjacent bins left to right until each expects enough
    ec, pc, acc_c, acc_p = [], [], 0.0, 0.0
    for c, q in zip(cnt, pmf):
        acc_c += c
        acc_p += q
        if acc_p * N >= min_expected:
            ec.append(acc_c)
            pc.append(acc_p)
            acc_c = acc_p = 0.0
    if acc_p > 0:
        ec[-1] += acc_c
        pc[-1] += acc_p
    return _chi2_pvalue(np.array(ec), np.array(pc))


@pytest.mark.parametrize("n,p", [(7, 0.3), (40, 0.2), (2000, 0.004),      # inversion
                                 (60, 0.4), (100, 0.5), (10 ** 6, 0.19),  # BTRS
                                 (25, 0.85), (3000, 0.57)])               # n - Bin(n, 1 - p)
def test_binomial_matches_exact_pmf(n, p):
    xs = [oracle.binomial(n, p, 11, 7, node, 1) for node in range(20000)]
    assert min(xs) >= 0 and max(xs) <= n
    assert _binned_gof(xs, n, p) > 1e-3


def test_binomial_degenerate_cases_and_large_n():
    assert oracle.binomial(0, 0.3, 1, 0, 0, 0) == 0
    assert oracle.binomial(12345, 0.0, 1, 0, 0, 0) == 0
    assert oracle.binomial(12345, 1.0, 1, 0, 0, 0) == 12345
    n, p = 1 << 30, 0.57
    xs = np.array([oracle.binomial(n, p, 3, 1, node, 0) for node in range(3000)], np.float64)
    sd = math.sqrt(n * p * (1 - p))
    assert abs(xs.mean() - n * p) < 5 * sd / math.sqrt(len(xs))
    assert 0.9 < xs.var() / sd ** 2 < 1.1


def test_quadrant_split_is_multinomial():
    """The three conditional binomials of one split give the multinomial law
    of (n_a, n_b, n_c, n_d) with the quadrants in a, b, c, d order (b != c so
    a swapped pair shows); m = 3: all 20 outcomes."""
    m, S = 3, 30000
    outcomes = [o for o in itertools.product(range(m + 1), repeat=4) if sum(o) == m]
    index = {o: i for i, o in enumerate(outcomes)}
    counts = np.zeros(len(outcomes))
    for seed in range(S):
        tl = oracle.partition(ASYM, 1, m, seed)
        q = [0, 0, 0, 0]
        for R, C, n in zip(tl["row"], tl["col"], tl["count"]):
            q[2 * int(R) + int(C)] = int(n)
        counts[index[tuple(q)]] += 1
    probs = np.array([stats.multinomial.pmf(o, m, ASYM) for o in outcomes])
    assert _chi2_pvalue(counts, probs) > 1e-3


def test_tile_counts_expectation_and_numbering():
    t, m, S = 2, 5000, 400
    K = kronecker(ASYM, t)
    tot = np.zeros((1 << t, 1 << t))
    for seed in range(S):
        tl = oracle.partition(ASYM, t, m, seed)
        assert int(tl["count"].sum()) == m and (tl["count"] > 0).all()
        assert np.array_equal(tl["first"], np.concatenate([[0], np.cumsum(tl["count"])[:-1]]).astype(np.uint64))
        # quadtree order: interleaved bits (row, col) of the tiles increase
        z = [sum(((int(r) >> b & 1) << (2 * b + 1)) | ((int(c) >> b & 1) << (2 * b)) for b in range(t))
             for r, c in zip(tl["row"], tl["col"])]
        assert z == sorted(z)
        tot[tl["row"].astype(int), tl["col"].astype(int)] += tl["count"]
    assert _chi2_pvalue(tot.ravel(), K.ravel()) > 1e-3


def test_partition_rows_are_communication_free():
    """A PE that owns some tile rows gets exactly the global tiles of those
    rows, with the same counts and edge numbers."""
    t, m = 5, 1 << 28
    full = oracle.partition(G500, t, m, 9)
    key = lambda d: {(int(r), int(c)): (int(n), int(f)) for r, c, n, f in zip(d["row"], d["col"], d["count"], d["first"])}
    g = key(full)
    seen = {}
    for r0, r1 in [(0, 3), (3, 4), (4, 17), (17, 32)]:
        part = key(oracle.partition(G500, t, m, 9, r0, r1))
        assert all(r0 <= r < r1 for r, _ in part)
        assert all(g[rc] == v for rc, v in part.items())
        seen.update(part)
    assert seen == g
    assert sum(n for n, _ in g.values()) == m


def test_partitioned_graph_has_the_kronecker_distribution():
    k, t, m = 6, 2, 1 << 18
    table = oracle.Table.variable(*ASYM, k, 40)
    tiles, (r, c) = oracle.generate_partitioned(table, ASYM, k, t, m, 5)
    assert len(r) == m
    pos = 0
    for R, C, n in zip(tiles["row"], tiles["col"], tiles["count"]):
        sl = slice(pos, pos + int(n))
        assert ((r[sl] >> np.uint64(k - t)) == R).all() and ((c[sl] >> np.uint64(k - t)) == C).all()
        pos += int(n)
    counts = np.bincount((r.astype(np.int64) << k) | c.astype(np.int64), minlength=1 << (2 * k)).astype(float)
    probs = kronecker(ASYM, k).ravel()
    order = np.argsort(probs)
    small = np.cumsum(probs[order] * m) < 50
    cc = np.concatenate([[counts[order][small].sum()], counts[order][~small]])
    pp = np.concatenate([[probs[order][small].sum()], probs[order][~small]])
    assert _chi2_pvalue(cc, pp) > 1e-3


def test_partition_depth_zero_is_the_plain_graph():
    table = oracle.Table.variable(*G500, 20, 500)
    tiles, (r, c) = oracle.generate_partitioned(table, G500, 20, 0, 5000, 77)
    assert list(tiles["count"]) == [5000] and list(tiles["first"]) == [0]
    r0, c0 = oracle.generate([table], 20, 77, 0, 5000)
    assert np.array_equal(r, r0) and np.array_equal(c, c0)


# ---------------------------------------------- larger Kronecker initiators --

THETA3 = np.array([[0.40, 0.15, 0.05], [0.12, 0.10, 0.04], [0.06, 0.03, 0.05]])  # asymmetric
THETA4 = np.arange(1, 17, dtype=np.float64).reshape(4, 4)[::-1] ** 1.5
THETA3 = THETA3 / THETA3.sum()
THETA4 = THETA4 / THETA4.sum()


def kron_power(theta, k):
    """Closed form of the stochastic Kronecker graph: theta^(x k), the first
    factor giving the most significant digit."""
    K = np.ones((1, 1))
    for _ in range(k):
        K = np.kron(K, theta)
    return K


@pytest.mark.parametrize("kind,args", [("variable", (G500, 26, 4096)), ("variable", (ASYM, 10, 100)),
                                       ("variable", (SKEWED, 40, 2000)), ("fixed", (ASYM, 4))])
def test_kron_with_two_by_two_initiator_is_rmat(kind, args):
    """n0 = 2 is R-MAT: same tables, same edges."""
    if kind == "variable":
        P, k, bound = args
        kt = oracle.KronTable.variable(np.array(P).reshape(2, 2), 2, k, bound)
        rt = oracle.Table.variable(*P, k, bound)
    else:
        P, ell = args
        k = 12
        kt = oracle.KronTable.fixed(np.array(P).reshape(2, 2), 2, ell)
        rt = oracle.Table.fixed([P], ell)
    for f in ("len", "p", "w", "thr", "alias"):
        assert np.array_equal(getattr(kt, f), getattr(rt, f)), f
    for i in range(rt.entries):
        L = int(rt.len[i])
        assert [int(x) for x in kt.sym[i, :L]] == [int(rt.sym[i]) >> (62 - 2 * t) & 3 for t in range(L)]
    a, b = oracle.kron_generate(kt, k, 3, 77, 5000), oracle.generate([rt], k, 3, 77, 5000)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("theta,n0,k,kind,x", [(THETA3, 3, 3, "variable", 60), (THETA3, 3, 3, "fixed", 2),
                                               (THETA4, 4, 2, "variable", 50), (THETA3, 3, 4, "variable", 200)])
def test_kron_exact_distribution_equals_kronecker_power(theta, n0, k, kind, x):
    t = oracle.KronTable.variable(theta, n0, k, x) if kind == "variable" else oracle.KronTable.fixed(theta, n0, x)
    D = oracle.kron_edge_distribution(t, k)
    assert np.abs(D - kron_power(theta, k)).max() <= 1e-12
    Dq = oracle.kron_edge_distribution(t, k, quantised=True)
    assert np.abs(Dq - kron_power(theta, k)).max() <= 8 * (1 << t.bits) * 2.0 ** -32


@pytest.mark.parametrize("n0,bound", [(3, 104), (3, 4096), (4, 1000), (5, 4096), (16, 5000)])
def test_kron_table_sizes_and_prefix_code(n0, bound):
    S = n0 * n0
    theta = np.random.default_rng(n0).dirichlet(np.ones(S)).reshape(n0, n0)
    t = oracle.KronTable.variable(theta, n0, 12, bound)
    assert t.entries == max(1 + (S - 1) * ((bound - 2) // (S - 1)), 1)   # largest 1 + (S-1)j < bound
    L = t.len[:t.entries].astype(np.float64)
    assert abs((float(S) ** -L).sum() - 1.0) < 1e-12                      # complete prefix code (Kraft)
    assert abs(t.p[:t.entries].sum() - 1.0) < 1e-12
    # greedy max-min: every open leaf is no likelier than every expanded node
    leaves = {tuple(int(v) for v in t.sym[i, :int(t.len[i])]) for i in range(t.entries)}
    internal = {lf[:j] for lf in leaves for j in range(len(lf))}
    pr = lambda path: float(np.prod([theta.ravel()[s] for s in path]))
    assert min(pr(n) for n in internal) >= max(pr(lf) for lf in leaves) * (1 - 1e-12)


def test_kron_fixed_entries_are_digits_and_depth_is_capped():
    t = oracle.KronTable.fixed(THETA3, 3, 3)
    for j in (0, 1, 80, 729 - 1, 500):
        assert [int(v) for v in t.sym[j, :3]] == [j // 81 % 9, j // 9 % 9, j % 9]
    skew = np.array([[0.9, 0.02, 0.02], [0.02, 0.01, 0.01], [0.01, 0.005, 0.005]])
    t = oracle.KronTable.variable(skew / skew.sum(), 3, 40, 1 << 16)
    assert t.max_len == 20          # 3^20 <= 2^32 < 3^21


def test_kron_generated_edges_follow_kronecker_power():
    k, m = 4, 1 << 18
    t = oracle.KronTable.variable(THETA3, 3, k, 300)
    r, c = oracle.kron_generate(t, k, 9, 0, m)
    nv = 3 ** k
    counts = np.bincount(r.astype(np.int64) * nv + c.astype(np.int64), minlength=nv * nv).astype(float)
    probs = kron_power(THETA3, k).ravel()
    order = np.argsort(probs)
    small = np.cumsum(probs[order] * m) < 50
    cc = np.concatenate([[counts[order][small].sum()], counts[order][~small]])
    pp = np.concatenate([[probs[order][small].sum()], probs[order][~small]])
    assert _chi2_pvalue(cc, pp) > 1e-3


@pytest.mark.parametrize("n,span", [(1, 3), (50, 4), (2000, 30), (5000, 1 << 20)])
def test_dedup_first_is_the_first_seen_filter(n, span):
    """Against the plain definition: walk the edges in order, keep an edge iff
    its (row, col) was not seen before."""
    rng = np.random.default_rng(n)
    r = rng.integers(0, span, n).astype(np.uint64)
    c = rng.integers(0, span, n).astype(np.uint64)
    seen, keep = set(), []
    for i in range(n):
        if (int(r[i]), int(c[i])) not in seen:
            seen.add((int(r[i]), int(c[i])))
            keep.append(i)
    dr, dc = oracle.dedup_first(r, c)
    assert np.array_equal(dr, r[keep]) and np.array_equal(dc, c[keep])
