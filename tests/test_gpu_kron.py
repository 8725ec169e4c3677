"""GPU parity for stochastic Kronecker graphs with an n0 x n0 initiator
(Sec. 3): the k_kron kernel through the C ABI against the CPU oracle, bit for
bit."""
import numpy as np
import pytest

import oracle
import paper_1905_03525_gb300 as rm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THETA3 = np.array([[0.40, 0.15, 0.05], [0.12, 0.10, 0.04], [0.06, 0.03, 0.05]])
THETA3 = THETA3 / THETA3.sum()


def _theta(n0, seed):
    th = np.random.default_rng(seed).dirichlet(np.linspace(4.0, 0.5, n0 * n0)).reshape(n0, n0)
    return th / th.sum()


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1905_03525_gb300 import build
    build.build()
    yield
    torch.cuda.synchronize()
    rm.rmat_check_device_errors()


def pairs(t, wide):
    h = t.cpu().numpy()
    h = h.view(np.uint64) if wide else h.view(np.uint32)
    return h[:, 0].astype(np.uint64), h[:, 1].astype(np.uint64)


def assert_same(gpu, ref):
    bad = np.nonzero((gpu[0] != ref[0]) | (gpu[1] != ref[1]))[0]
    assert bad.size == 0, f"{bad.size} edges differ; first at {bad[:5]}: {gpu[0][bad[:2]]} vs {ref[0][bad[:2]]}"


CASES = [
    (3, 12, "variable", 500, 100_003, 0),          # u32
    (3, 20, "variable", 4096, 60_000, 7 << 33),    # u32, 3^20 close to 2^32, large offset
    (3, 30, "variable", 4096, 40_000, 5),          # u64
    (3, 40, "variable", 8192, 20_000, 0),          # deepest k, long paths
    (3, 20, "variable", 8192, 50_000, 3),          # u32 IDs, 9-level paths, 197 KB table
    (4, 16, "variable", 2000, 30_000, 1),          # n0^k = 2^32 exactly: u32
    (5, 13, "fixed", 2, 30_000, 3),
    (16, 8, "variable", 5000, 30_000, 0),          # 16^8 = 2^32
    (16, 16, "variable", 300, 20_000, 11),         # 16^16 = 2^64: u64
    (3, 9, "variable", 60, 1, 99),                 # one edge
]


@pytest.mark.parametrize("n0,k,kind,x,m,e0", CASES)
def test_kron_matches_oracle(n0, k, kind, x, m, e0):
    th = THETA3 if n0 == 3 else _theta(n0, n0)
    if kind == "variable":
        t, ot = rm.rmat_build_table_kron(th, n0, k, x), oracle.KronTable.variable(th, n0, k, x)
    else:
        t, ot = rm.rmat_build_table_kron_fixed(th, n0, k, x), oracle.KronTable.fixed(th, n0, x)
    wide = rm.rmat_table_info(t)["index_bytes"] == 8
    out = rm.empty_edges_for(t, m)
    rm.rmat_generate(t, 17, e0, m, out)
    torch.cuda.synchronize()
    assert_same(pairs(out, wide), oracle.kron_generate(ot, k, 17, e0, m))


def test_kron_bench_shape_through_both_kernels():
    """The 3 x 3 bench table (k = 17, bound 4096): whole 512-edge tiles go to
    the contract-case kernel and the ragged tail to the general one; an output
    that is only 8-byte aligned takes the general kernel throughout.  Both
    equal the oracle."""
    from paper_1905_03525_gb300.workloads import KRON3
    th = np.array(KRON3)
    t, ot = rm.rmat_build_table_kron(th, 3, 17, 4096), oracle.KronTable.variable(th, 3, 17, 4096)
    m, e0 = (1 << 20) + 77, 12345
    ref = oracle.kron_generate(ot, 17, 1, e0, m)
    out = rm.empty_edges_for(t, m + 1)
    rm.rmat_generate(t, 1, e0, m, out[:m])
    torch.cuda.synchronize()
    assert_same(pairs(out[:m], False), ref)
    rm.rmat_generate(t, 1, e0, m, out[1:])
    torch.cuda.synchronize()
    assert_same(pairs(out[1:], False), ref)


def test_kron_host_output_and_chunks():
    t = rm.rmat_build_table_kron(THETA3, 3, 18, 1024)
    m = 200_001
    host = rm.empty_edges_for(t, m, device="cpu", pin_memory=True)
    rm.rmat_generate_host(t, 5, 123, m, host)
    dev = rm.empty_edges_for(t, m)
    rm.rmat_generate(t, 5, 123, 100_000, dev[:100_000])
    rm.rmat_generate(t, 5, 123 + 100_000, m - 100_000, dev[100_000:])
    torch.cuda.synchronize()
    assert torch.equal(host, dev.cpu())


def test_kron_full_size_sampled():
    """n0 = 3, k = 17 (1.3e8 vertices), m = 2^30, bound 4096: sampled runs of
    edges against the oracle, and the top-level cell frequencies."""
    k, m = 17, 1 << 30
    t = rm.rmat_build_table_kron(THETA3, 3, k, 4096)
    ot = oracle.KronTable.variable(THETA3, 3, k, 4096)
    out = rm.empty_edges_for(t, m)
    rm.rmat_generate(t, 1, 0, m, out)
    torch.cuda.synchronize()
    rng = np.random.default_rng(17)
    for s in sorted({0, m - 2048, *map(int, rng.integers(0, m - 2048, 14))}):
        assert_same(pairs(out[s:s + 2048], False), oracle.kron_generate(ot, k, 1, s, 2048))
    rows = out[:, 0].view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    cols = out[:, 1].view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    top = (rows // 3 ** (k - 1)) * 3 + cols // 3 ** (k - 1)
    counts = torch.bincount(top, minlength=9).cpu().numpy().astype(float)
    p = THETA3.ravel()
    z = (counts - p * m) / np.sqrt(m * p * (1 - p))
    assert np.all(np.abs(z) < 6), z
    del out
    torch.cuda.empty_cache()
