"""The autotuner returns shapes and tables that exist, and generation under
the tuned choices gives the same bytes as under the defaults."""
import pytest

import paper_1905_03525_gb300 as rm
from paper_1905_03525_gb300.workloads import G500, batched_graphs, noisy_levels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def tmp_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("RMAT_TUNE_CACHE", str(tmp_path))
    from paper_1905_03525_gb300 import build
    build.build()


def test_tune_launch_and_table():
    from paper_1905_03525_gb300 import autotune
    t = rm.rmat_build_table(*G500, 26, 4096)
    m = 1 << 20
    ref = rm.empty_edges(m, 26)
    rm.rmat_generate(t, 3, 0, m, ref)
    shape, rate = autotune.tune_launch(t, sample_edges=1 << 22)
    assert shape in autotune.LAUNCH_SHAPES and rate > 0
    out = rm.empty_edges(m, 26)
    rm.rmat_generate(t, 3, 0, m, out)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    # cached on the second call
    assert autotune.tune_launch(t, sample_edges=1 << 22)[0] == shape
    best = autotune.tune_table(20, G500, sample_edges=1 << 20, bounds=[256, 4096], ells=[4, 5])
    assert best["kind"] in ("variable", "fixed") and best["edges_per_s"] > 0
    lv = autotune.tune_levels(34, noisy_levels(34), rm.RMAT_UNDIRECTED, sample_edges=1 << 20, ells=(5, 6))
    assert lv["ell"] in (5, 6)


def test_plan_batch_tables_fit_the_batch_kernel():
    from paper_1905_03525_gb300 import autotune
    gs = batched_graphs(24, seed=9, k_range=(10, 14), log2m_range=(10.0, 16.0))
    tables, choices = autotune.plan_batch(gs, sample_edges=1 << 18)
    budget = autotune.batch_blob_budget()
    assert len(tables) == len(gs)
    for t, g in zip(tables, gs):
        info = rm.rmat_table_info(t)
        assert info["k"] == g["k"] and info["device_image_bytes"] <= max(budget, 8 * g["m"] + 4096)
