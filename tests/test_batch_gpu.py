"""Batched launches: realisations of uneven grid sizes, grouped by grid and
evaluated with one fbs_bispectrum_batch per group (one launch per stage for
all of a group's fields), captured into one CUDA graph.  The graph gives
exactly the eager batched results; the batched results equal one call per
field up to the rounding of the contraction's point ranges (1e-5 of the
field's largest |B|), and the oracle's within the precision's tolerance on
the gated triplets; multi-level plans batch too."""
import numpy as np
import pytest

import fields
import oracle
import paper_1705_06284_gb300 as fbs
from gpu_util import TOL, gate_mask, rel_err
from paper_1705_06284_gb300.batch import GraphBatch

pytestmark = pytest.mark.gpu


def _fields(n, seed=5):
    rng = np.random.default_rng(seed)
    fl = []
    for i in range(n):
        N = int(rng.choice([16, 24, 32]))
        f = fields.lognormal(N, 0.5, -1.5, seed=100 + i) if i % 2 else fields.bubbles(N, 2.0, 0.4, seed=200 + i)
        fl.append(f.astype(np.float32))
    return fl


@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
def test_graph_of_batches_equals_eager_and_single_calls(tmp_path, monkeypatch, precision):
    import paper_1705_06284_gb300.batch as bt
    monkeypatch.setattr(bt, "_TUNE_CACHE", str(tmp_path / "tune.json"))
    fl = _fields(12)
    L_for = lambda N: float(N)
    edges_for = lambda N: fields.linear_edges(N, float(N), 5)
    gb = GraphBatch(fl, L_for, edges_for, precision=precision, tune=(precision != "fp32"))
    try:
        assert len(gb.groups) >= 2
        gb.run_eager()
        eager = gb.results()
        gb.capture()
        for _ in range(2):
            gb.replay()
        graph = gb.results()
        gb.run_one_at_a_time()
        single = gb.results()
    finally:
        gb.close()
    for (t1, B1, P1), (t2, B2, P2), (t3, B3, P3) in zip(eager, graph, single):
        assert np.array_equal(B1, B2) and np.array_equal(P1, P2, equal_nan=True)
        assert np.array_equal(P1, P3, equal_nan=True)  # same z-stage partials, same order
        # the contraction's point ranges differ (CTAs per field): rounding of the
        # order of the precision, far below the largest |B| of the field
        assert np.all(np.abs(B1 - B3) <= 1e-5 * np.max(np.abs(B3)))
    # every realisation of one grid against the oracle
    for k, f in enumerate(fl[:4]):
        f64 = f.astype(np.float64)
        N = f.shape[0]
        ref = oracle.direct_bispectrum(f64, float(N), edges_for(N))
        assert np.array_equal(eager[k][0], ref["triplets"])
        M = oracle.fft_estimator(f64, float(N), edges_for(N), triplets=ref["triplets"])["M"]
        g = gate_mask(ref["B"], M, ref["N_tri"])
        if g.any():
            assert rel_err(eager[k][1], ref["B"])[g].max() < TOL[precision]


def test_batch_on_multi_level_plans(monkeypatch):
    import torch
    monkeypatch.setenv("FBS_LEVEL_COST", "-1e15")
    monkeypatch.setenv("FBS_MIN_LEVEL_GRID", "0")
    N, L = 48, 60.0
    edges = fields.log_edges(N, L, 8)
    fl = [torch.from_numpy(fields.quadratic_local(N, 0.5, -1.5, 0.3, seed=300 + i).astype(np.float32)).cuda()
          for i in range(5)]
    with fbs.Plan(N, L, edges, precision="bf16x3") as plan:
        assert len(plan.levels) >= 2
        B, P = plan.bispectrum_batch(fl)
        plan.check()
        for i, f in enumerate(fl):
            Bs, Ps = plan.bispectrum(f)
            torch.cuda.synchronize()
            Bs, Ps = Bs.cpu().numpy(), Ps.cpu().numpy()
            assert np.array_equal(P[i].cpu().numpy(), Ps, equal_nan=True)
            assert np.all(np.abs(B[i].cpu().numpy() - Bs) <= 1e-5 * np.max(np.abs(Bs)))
