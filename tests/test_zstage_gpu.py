"""The register x, y and z stages (the z stage a C2R of two real rows per
complex line, Eq. delta_nr) at every evaluation grid with a compile-time
kernel, against the FP64 oracle.

Full-grid plans put the inverse transforms on the input grid N itself, so
each N below runs the register x, y and z stages of that length.  P depends on the z
stage's own sums of squares and B on the shell fields it writes: both are
compared with the oracle's FFT estimator (FP32 path, so the contraction adds
no BF16 rounding), B on the triplets gated on the cancellation-free scale.
"""
import numpy as np
import pytest

import fields
import oracle
import paper_1705_06284_gb300 as fbs
from gpu_util import TOL, gate_mask, rel_err, run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N", [64, 72, 96, 108, 128, 144, 192, 216])
def test_register_z_stage_every_grid(N):
    L = float(N)
    edges = fields.linear_edges(N, L, 4)
    f32 = fields.lognormal(N, 0.5, -1.5, seed=400 + N).astype(np.float32)
    with fbs.Plan(N, L, edges, precision="fp32", full_grid=True) as plan:
        assert plan.eval_grid == N
        B, P = run(plan, f32)
        e = oracle.fft_estimator(f32.astype(np.float64), L, edges, triplets=plan.triplets)
        assert np.array_equal(plan.N_tri, e["N_tri"])
        ok = np.isfinite(e["P"])
        assert np.array_equal(np.isnan(P), ~ok)
        assert np.all(rel_err(P[ok], e["P"][ok]) < 1e-5)
        g = gate_mask(e["B"], e["M"], e["N_tri"])
        assert g.sum() >= 3
        r = rel_err(B, e["B"])
        print("z stage N=%d: %d gated, max rel %.2e" % (N, int(g.sum()), float(r[g].max())))
        assert r[g].max() < TOL["fp32"]
