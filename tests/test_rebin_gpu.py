"""Fine bins, then (k1, k2, cos theta) cells, on the GPU against the oracle.

A plan on one-pixel bins (Sec. 3.1's advice) is evaluated on the device and
its triplets regrouped by fbs_rebin into cells of (k1, k2, cos theta); the
oracle aggregates its own all-pairs ordered direct sums over ordered bin
triples (Eq. bi_direct).  Counts must agree exactly; B within the tolerance
of the precision on cells with >= 100 ordered triples and |B| >= 1e-3 of the
cells' cancellation-free scale.
"""
import itertools
import math

import numpy as np
import pytest

import fields
import oracle
import paper_1705_06284_gb300 as fbs
from gpu_util import TOL, rel_err

pytestmark = pytest.mark.gpu


def _cell_scale(trip, ntri, M, k_rep, ke, me):
    """Count-weighted cancellation-free scale of every cell."""
    nk, nmu = len(ke) - 1, len(me) - 1
    num = np.zeros((nk, nk, nmu))
    den = np.zeros((nk, nk, nmu))
    for t, n, m in zip(trip, ntri, M):
        for x, y, z in set(itertools.permutations(t)):
            k1, k2, k3 = k_rep[x], k_rep[y], k_rep[z]
            mu = min(1.0, max(-1.0, (k1 * k1 + k2 * k2 - k3 * k3) / (2 * k1 * k2)))
            K1 = np.searchsorted(ke, k1, side="right") - 1
            K2 = np.searchsorted(ke, k2, side="right") - 1
            MU = np.searchsorted(me, mu, side="right") - 1
            if 0 <= K1 < nk and 0 <= K2 < nk and 0 <= MU < nmu:
                num[K1, K2, MU] += m * n
                den[K1, K2, MU] += n
    with np.errstate(invalid="ignore", divide="ignore"):
        return num / den


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_one_pixel_bins_rebinned_match_oracle(precision):
    import torch
    N, L = 32, 100.0
    kf = 2 * math.pi / L
    edges = kf * np.arange(1, 9)            # one-pixel bins from k_f to N k_f/4
    ke = kf * np.array([1.0, 3.0, 5.0, 8.0])
    me = np.linspace(-1.0, 1.0001, 5)
    f32 = fields.quadratic_local(N, 1.0, -1.5, 0.3, seed=81).astype(np.float32)
    f64 = f32.astype(np.float64)
    Bref, cref, _ = oracle.rebinned_bispectrum(f64, L, edges, ke, me)
    with fbs.Plan(N, L, edges, precision=precision) as plan, fbs.Rebin(plan, ke, me) as rb:
        plan.bispectrum(torch.from_numpy(f32).cuda())
        B = rb.bispectrum()
        assert np.array_equal(rb.counts, cref)
        assert np.array_equal(np.isnan(B), cref == 0)
        thr = np.asarray(plan.thresholds, dtype=np.float64)
        k_rep = 0.5 * kf * (np.sqrt(thr[:-1]) + np.sqrt(thr[1:]))
        M = oracle.fft_estimator(f64, L, edges, triplets=plan.triplets)["M"]
        scale = _cell_scale(plan.triplets, plan.N_tri, M, k_rep, ke, me)
        g = (cref >= 100) & (np.abs(Bref) >= 1e-3 * scale)
        r = rel_err(B, Bref)
        assert g.sum() >= 5
        print("rebinned %s: %d of %d cells gated, max rel %.2e" % (precision, int(g.sum()), int((cref > 0).sum()),
                                                                  float(r[g].max())))
        assert r[g].max() < TOL[precision]
        # device outputs give the same cells
        dB = torch.empty(rb.nk * rb.nk * rb.nmu, dtype=torch.float64, device="cuda")
        rb.bispectrum(dB)
        torch.cuda.synchronize()
        assert np.array_equal(dB.cpu().numpy().reshape(B.shape), B, equal_nan=True)
