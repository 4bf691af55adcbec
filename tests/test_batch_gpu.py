"""Batched launch: realisations of uneven grid sizes captured into one CUDA
graph give exactly the results of eager one-at-a-time calls."""
import numpy as np
import pytest

import fields
import oracle
from paper_1705_06284_gb300.batch import GraphBatch

pytestmark = pytest.mark.gpu


def test_graph_batch_equals_eager(tmp_path, monkeypatch):
    import paper_1705_06284_gb300.batch as bt
    monkeypatch.setattr(bt, "_TUNE_CACHE", str(tmp_path / "tune.json"))
    rng = np.random.default_rng(5)
    fl = []
    for i in range(10):
        N = int(rng.choice([16, 24, 32]))
        f = fields.lognormal(N, 0.5, -1.5, seed=100 + i) if i % 2 else \
            fields.bubbles(N, 2.0, 0.4, seed=200 + i)
        fl.append(f.astype(np.float32))
    L_for = lambda N: float(N)
    edges_for = lambda N: fields.linear_edges(N, float(N), 5)
    gb = GraphBatch(fl, L_for, edges_for, precision="bf16x3", tune=True)
    try:
        gb.run_eager()
        eager = gb.results()
        gb.capture()
        for _ in range(2):
            gb.replay()
        graph = gb.results()
    finally:
        gb.close()
    for (t1, B1, P1), (t2, B2, P2) in zip(eager, graph):
        assert np.array_equal(B1, B2) and np.array_equal(P1, P2, equal_nan=True)
    # one realisation against the oracle (exact counts, B within BF16x3 tolerance)
    f0 = fl[0].astype(np.float64)
    N0 = fl[0].shape[0]
    ref = oracle.direct_bispectrum(f0, float(N0), edges_for(N0))
    assert np.array_equal(eager[0][0], ref["triplets"])
