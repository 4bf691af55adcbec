"""Non-cubic grids and complex fields (fbs_gplan_*) against the oracle's FFT
estimator on the same grid (pinned to an all-pairs brute force): the closed
triplets and their exact counts, B and P (complex) within 1e-4 on triplets
with N_tri >= 100 and |B| >= 1e-3 of the cancellation-free scale."""
import math

import numpy as np
import pytest

import oracle
import paper_1705_06284_gb300 as fbs

pytestmark = pytest.mark.gpu

CASES = [((24, 32, 48), (60.0, 80.0, 120.0), "complex", 41), ((32, 32, 16), (50.0, 50.0, 25.0), "real", 42),
         ((36, 24, 27), (40.0, 30.0, 45.0), "complex", 43), ((64, 48, 32), (100.0, 90.0, 50.0), "complex", 44)]


def _field(shape, kind, seed):
    rng = np.random.default_rng(seed)
    # a little structure: a squared Gaussian term makes the bispectrum nonzero
    g = rng.standard_normal(shape) + (1j * rng.standard_normal(shape) if kind == "complex" else 0)
    return (g + 0.3 * g * g).astype(np.complex64 if kind == "complex" else np.float32)


def _edges(shape, Ls, nb):
    kmin = 2 * math.pi / max(Ls)
    kmax = 2 * math.pi * min(n / 4.0 / L for n, L in zip(shape, Ls))
    return np.geomspace(1.2 * kmin, 0.999 * kmax, nb + 1)


def _scale(f, Ls, edges, trip):
    """sum_n |I_a I_b I_c| normalised like B (cancellation-free scale)."""
    shape = f.shape
    npix = float(np.prod(shape))
    V = float(np.prod(Ls))
    bins = oracle.general_bin_index(shape, Ls, edges)
    D = np.fft.fftn(f.astype(np.complex128))
    I = {b: np.fft.ifftn(np.where(bins == b, D, 0)) * npix for b in set(trip.ravel().tolist())}
    return np.array([(V * V / npix ** 3) * np.sum(np.abs(I[a] * I[b] * I[c])) / npix for a, b, c in trip])


@pytest.mark.parametrize("shape,Ls,kind,seed", CASES)
def test_general_plan_matches_oracle(shape, Ls, kind, seed):
    import torch
    f = _field(shape, kind, seed)
    edges = _edges(shape, Ls, 6)
    with fbs.GeneralPlan(shape, Ls, edges) as plan:
        ref = oracle.general_bispectrum(f.astype(np.complex128), Ls, edges)
        assert np.array_equal(plan.triplets, ref["triplets"])
        assert np.array_equal(plan.N_tri, ref["N_tri"])
        assert np.array_equal(plan.shell, ref["shell"])
        B, P = plan.bispectrum(torch.from_numpy(f).cuda())
        Bh, Ph = plan.bispectrum(f)  # host field: the same numbers
        assert np.array_equal(B, Bh) and np.array_equal(P, Ph, equal_nan=True)
    Mg = _scale(f, Ls, edges, ref["triplets"]) / np.maximum(ref["N_tri"], 1)
    g = (ref["N_tri"] >= 100) & (np.abs(ref["B"]) >= 1e-3 * Mg)
    r = np.abs(B - ref["B"]) / np.abs(ref["B"])
    print("general %s %s: %d/%d gated, max rel %.2e" % (shape, kind, int(g.sum()), len(g), float(r[g].max())))
    assert g.sum() >= 5 and r[g].max() < 1e-4
    ok = ref["shell"] > 0
    assert np.all(np.abs(P[ok] - ref["P"][ok]) <= 1e-4 * np.abs(ref["P"][ok]))
    if kind == "real":
        assert np.all(np.abs(B.imag) <= 1e-4 * Mg)


def test_general_plan_rejects_wrapped_bins_unless_allowed():
    shape, Ls = (16, 16, 32), (10.0, 10.0, 10.0)
    edges = [0.5, 1.0, 2.0, 3.0]  # past N_x k_f,x / 4 = 2.51 along x
    with pytest.raises(fbs.FbsError):
        fbs.GeneralPlan(shape, Ls, edges)
    with fbs.GeneralPlan(shape, Ls, edges, allow_aliased=True) as plan:
        assert plan.ntrip > 0
