"""Diagonal-resolved trispectrum on the GPU (pair spectra and shell-restricted
Gram products) against the oracle's FFT route, which is pinned to brute
force: exact counts per diagonal shell, and T_D within 1e-4 on the
(quadruplet, shell) items with N_D >= 100 and |num_D| >= 1e-3 of the
cancellation-free scale sum |F_ab| |F_cd| over the shell."""
import math

import numpy as np
import pytest

import fields
import oracle
import paper_1705_06284_gb300 as fbs
from gpu_util import rel_err

pytestmark = pytest.mark.gpu


def _diag_edges(N, L, nd):
    """q = 0 alone, then nd - 1 shells up to the largest diagonal that can close."""
    kf = 2 * math.pi / L
    top = 0.5 * N * kf
    return np.concatenate([[0.0], np.linspace(0.5 * kf, top, nd)])


def _run(plan, f32, L, edges, dedges):
    import torch
    plan.set_diagonal(dedges)
    TD = plan.trispectrum_diagonal(torch.from_numpy(f32).cuda()).cpu().numpy()
    ref = oracle.diagonal_trispectrum(f32.astype(np.float64), L, edges, dedges, plan.quads)
    assert plan.N_D_exact == ref["cnt"]
    assert np.array_equal(plan.N_D, np.array([[float(v) for v in r] for r in ref["cnt"]]))
    cnt = plan.N_D
    g = (cnt >= 100) & (np.abs(ref["num"]) >= 1e-3 * ref["mag"])
    assert np.array_equal(np.isnan(TD), cnt == 0)
    r = rel_err(TD, ref["T"])
    rest = (cnt > 0) & ~g
    err_rest = np.abs(TD - ref["T"]) * cnt / np.where(ref["mag"] > 0, ref["mag"], 1.0)
    return g, r, rest, err_rest


@pytest.mark.parametrize("N,L,kind,nb,nd,precision", [(16, 50.0, "lin", 4, 6, "fp32"),
                                                      (24, 60.0, "log", 6, 8, "bf16x3"),
                                                      (32, 100.0, "lin", 5, 10, "fp32")])
def test_diagonal_trispectrum_matches_oracle(N, L, kind, nb, nd, precision):
    edges = fields.linear_edges(N, L, nb) if kind == "lin" else fields.log_edges(N, L, nb)
    f32 = fields.quadratic_local(N, 1.0, -1.5, 0.3, seed=81).astype(np.float32)
    with fbs.Plan(N, L, edges, precision=precision, trispectrum=True) as plan:
        dedges = _diag_edges(N, L, nd)
        g, r, rest, err_rest = _run(plan, f32, L, edges, dedges)
        # covering diagonal shells: the split counts add up to the quadruple counts
        assert [sum(row) for row in plan.N_D_exact] == plan.N_quad_exact
    print("diagonal T N=%d: %d gated, max rel %.2e" % (N, int(g.sum()), float(r[g].max())))
    assert g.sum() >= 10
    assert r[g].max() < 1e-4
    V, npix = L ** 3, float(N) ** 3
    # elsewhere |num_D - ref| <= 1e-6 of the cancellation-free scale (FP32 pair spectra)
    assert np.all(err_rest[rest] <= 1e-6 * V ** 3 / npix ** 4)


def test_diagonal_trispectrum_on_levels(monkeypatch):
    monkeypatch.setenv("FBS_LEVEL_COST", "-1e15")
    monkeypatch.setenv("FBS_MIN_LEVEL_GRID", "0")
    N, L = 48, 60.0
    edges = fields.log_edges(N, L, 8)
    f32 = fields.quadratic_local(N, 1.0, -1.5, 0.3, seed=82).astype(np.float32)
    with fbs.Plan(N, L, edges, precision="fp32", trispectrum=True) as plan:
        assert len(set(plan.quad_level.tolist())) >= 2
        g, r, _, _ = _run(plan, f32, L, edges, _diag_edges(N, L, 6))
    assert g.sum() >= 10 and r[g].max() < 1e-4
