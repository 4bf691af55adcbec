"""Theory averaged over each bin triplet's exact triangles, on the GPU.

``theory.local``, ``theory.bubbles`` and ``theory.tree_level`` build separable
terms and average them with fbs_plan_triangle_average (FP64 weighted count
fields); the oracle evaluates each model on every closed triangle of the
triplet and averages (the definition of the paper's bin-averaged theory
points, Sec. 3.3).  FP64 on both sides: 1e-9 relative."""
import math

import numpy as np
import pytest

import fields
import oracle
import paper_1705_06284_gb300 as fbs
from paper_1705_06284_gb300 import theory

pytestmark = pytest.mark.gpu


def _norm(k):
    return np.linalg.norm(k, axis=1)


@pytest.mark.parametrize("N,L,nb,kind", [(16, 60.0, 4, "lin"), (24, 50.0, 6, "log")])
def test_models_match_per_triangle_average(N, L, nb, kind):
    edges = fields.linear_edges(N, L, nb) if kind == "lin" else fields.log_edges(N, L, nb)
    Pk = lambda k: 1.0 / (1.0 + (k * 3.0) ** 2)
    kappa, f, R, x = 3.0 / 7.0, 0.4, 4.0, 0.7
    with fbs.Plan(N, L, edges, precision="bf16x3") as plan:
        trip = plan.triplets
        got_local = theory.local(plan, Pk, f)
        got_bub = theory.bubbles(plan, R, x)
        got_tree = theory.tree_level(plan, Pk, kappa)
        got_pb = theory.bubbles_power(plan, R, x)
        shells = plan.shell.copy()
    ref_local, cnt = oracle.triangle_average_direct(
        N, L, edges, trip, lambda a, b, c: 2 * f * (Pk(_norm(a)) * Pk(_norm(b)) + Pk(_norm(b)) * Pk(_norm(c))
                                                   + Pk(_norm(c)) * Pk(_norm(a))))
    n = (1 - x) / (4 * math.pi * R ** 3 / 3)
    W = lambda k: theory.tophat_window(_norm(k) * R)
    ref_bub, _ = oracle.triangle_average_direct(N, L, edges, trip,
                                                lambda a, b, c: -(1 - x) ** 3 * W(a) * W(b) * W(c) / n ** 2)

    def F(a, b):
        ka, kb = _norm(a), _norm(b)
        mu = np.sum(a * b, axis=1) / (ka * kb)
        return (1 + kappa) / 2 + mu / 2 * (ka / kb + kb / ka) + (1 - kappa) / 2 * mu * mu
    ref_tree, _ = oracle.triangle_average_direct(
        N, L, edges, trip, lambda a, b, c: 2 * F(a, b) * Pk(_norm(a)) * Pk(_norm(b))
        + 2 * F(b, c) * Pk(_norm(b)) * Pk(_norm(c)) + 2 * F(c, a) * Pk(_norm(c)) * Pk(_norm(a)))
    for got, ref in ((got_local, ref_local), (got_bub, ref_bub), (got_tree, ref_tree)):
        assert np.allclose(got, ref, rtol=1e-9, atol=1e-12 * np.max(np.abs(ref)))
    # the shell-averaged bubble power spectrum (Eq. BharPk) over each bin's modes
    thr = oracle.thresholds(edges, L)
    bins = oracle.bin_index(N, thr)
    kk = 2 * math.pi / L * np.sqrt(oracle.mode_squares(N).astype(float))
    pk = (1 - x) ** 2 * theory.tophat_window(kk * R) ** 2 / n
    for b in range(len(thr) - 1):
        if shells[b]:
            assert abs(got_pb[b] - pk[bins == b].mean()) <= 1e-12 * abs(pk[bins == b].mean())
        else:
            assert np.isnan(got_pb[b])


def test_theory_on_a_multi_level_plan(monkeypatch):
    # items on several evaluation grids: each level sums its own triplets
    monkeypatch.setenv("FBS_LEVEL_COST", "-1e15")
    monkeypatch.setenv("FBS_MIN_LEVEL_GRID", "0")
    N, L = 32, 80.0
    edges = fields.log_edges(N, L, 8)
    with fbs.Plan(N, L, edges, precision="fp32") as plan:
        assert len(plan.levels) >= 2
        got = theory.bubbles(plan, 3.0, 0.6)
        trip = plan.triplets
    n = (1 - 0.6) / (4 * math.pi * 27.0 / 3)
    W = lambda k: theory.tophat_window(_norm(k) * 3.0)
    ref, _ = oracle.triangle_average_direct(N, L, edges, trip, lambda a, b, c: -(0.4) ** 3 * W(a) * W(b) * W(c) / n ** 2)
    assert np.allclose(got, ref, rtol=1e-9, atol=1e-12 * np.max(np.abs(ref)))
