"""Failure detection without faulting the GPU: a device wait that can never be
satisfied runs out after its bound, the kernel records the error and exits,
the host reads RMAT_ERR_TIMEOUT, and the context keeps working."""
import numpy as np
import pytest

import oracle
import paper_1905_03525_gb300 as rm
from paper_1905_03525_gb300.workloads import G500

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1905_03525_gb300 import build
    build.build()


def test_bounded_wait_runs_out_and_is_reported():
    rm.rmat_check_device_errors()            # nothing pending
    with pytest.raises(rm.RmatError) as ei:
        rm.rmat_selftest_bounded_wait(2000)
    assert "RMAT_ERR_TIMEOUT" in str(ei.value)
    rm.rmat_check_device_errors()            # the word was read and cleared
    # the context is intact: a generation right after matches the oracle
    k, m = 20, 50_000
    t = rm.rmat_build_table(*G500, k, 1024)
    out = rm.empty_edges(m, k)
    rm.rmat_generate(t, 5, 0, m, out)
    torch.cuda.synchronize()
    h = out.cpu().numpy().view(np.uint32)
    r, c = oracle.generate([oracle.Table.variable(*G500, k, 1024)], k, 5, 0, m)
    assert np.array_equal(h[:, 0], r) and np.array_equal(h[:, 1], c)
