"""The table built on the GPU (rmat_build_table_gpu) equals the oracle's and
the host build's, field for field, and generates the same edges."""
import numpy as np
import pytest

import oracle
import paper_1905_03525_gb300 as rm
from paper_1905_03525_gb300.workloads import G500, SKEWED

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ASYM = (0.5, 0.2, 0.25, 0.05)
UNIFORM = (0.25, 0.25, 0.25, 0.25)   # every node of a level ties: the cut falls inside a tie class


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1905_03525_gb300 import build
    build.build()
    yield
    torch.cuda.synchronize()
    rm.rmat_check_device_errors()


CASES = [(G500, 26, 4096), (G500, 26, 5), (G500, 26, 6), (G500, 26, 1 << 16), (ASYM, 20, 1000),
         (SKEWED, 30, 8192), (G500, 3, 4096), (G500, 7, 50_000), (UNIFORM, 26, 4096), (UNIFORM, 26, 4097),
         (G500, 40, 1 << 20), ((0.45, 0.25, 0.2, 0.1), 64, 77_777)]


@pytest.mark.parametrize("params,k,bound", CASES)
def test_gpu_built_table_equals_oracle(params, k, bound):
    t = rm.rmat_build_table_gpu(*params, k, bound)
    ex = rm.rmat_table_export(t)
    ot = oracle.Table.variable(*params, k, bound)
    assert (ex["entries"], ex["bits"], ex["max_len"]) == (ot.entries, ot.bits, ot.max_len)
    for f in ("sym", "len", "p", "w", "thr", "alias"):
        assert np.array_equal(ex[f], getattr(ot, f)), f
    h = rm.rmat_build_table(*params, k, bound)
    assert rm.rmat_table_info(t) == rm.rmat_table_info(h)


@pytest.mark.parametrize("params,k,bound", [(G500, 26, 4096), (SKEWED, 30, 8192), (G500, 40, 1 << 20)])
def test_gpu_built_table_generates_the_same_edges(params, k, bound):
    t = rm.rmat_build_table_gpu(*params, k, bound)
    h = rm.rmat_build_table(*params, k, bound)
    m = 300_001
    a, b = rm.empty_edges(m, k), rm.empty_edges(m, k)
    rm.rmat_generate(t, 9, 1 << 20, m, a)
    rm.rmat_generate(h, 9, 1 << 20, m, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    # and the table serves a batch like a host-built one
    bt = rm.rmat_batch_create()
    c = rm.empty_edges(m, k)
    rm.rmat_batch_add(bt, t, 9, 1 << 20, m, c)
    rm.rmat_batch_launch(bt)
    torch.cuda.synchronize()
    assert torch.equal(a, c)


def test_gpu_build_rejects_zero_parameters():
    with pytest.raises(rm.RmatError):
        rm.rmat_build_table_gpu(1.0, 0.0, 0.0, 0.0, 26, 4096)
