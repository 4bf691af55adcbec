"""Connected trispectrum on the GPU against the oracle.

fbs_trispectrum_connected leaves out the paired quadruples of the four-shell
estimator (the P x P terms).  On tiny grids it is compared with the oracle's
direct sum that skips them mode by mode (exact unpaired counts); on larger
grids with the oracle's FP64 FFT estimator minus the pairing terms.  The
connected part is what is left of the raw sum after the paired sum is taken
away, so its error is that of the raw sum, a fraction of the raw sum's
cancellation-free scale Tc_M: quadruplets with N_conn >= 100 and
|Tc| >= 0.05 Tc_M are held to 1e-4 (FP32) or 2e-4 (BF16x3) of Tc, the others
to that fraction of 0.05 Tc_M.
"""
import numpy as np
import pytest

import fields
import oracle
import paper_1705_06284_gb300 as fbs
from gpu_util import TOL, rel_err

pytestmark = pytest.mark.gpu


def _run(plan, f32):
    import torch
    Tc, T, B, P = plan.trispectrum_connected(torch.from_numpy(f32).cuda())
    plan.check()
    return tuple(x.cpu().numpy() for x in (Tc, T, B, P))


@pytest.mark.parametrize("N,L,nb,precision", [(8, 40.0, 3, "fp32"), (12, 30.0, 3, "bf16x3")])
def test_connected_matches_direct_sum(N, L, nb, precision):
    edges = fields.linear_edges(N, L, nb)
    f32 = fields.quadratic_local(N, 2.0, -1.5, 0.3, seed=71).astype(np.float32)
    f64 = f32.astype(np.float64)
    d = oracle.direct_trispectrum(f64, L, edges, connected=True)
    with fbs.Plan(N, L, edges, precision=precision, trispectrum=True) as plan:
        Tc, T, B, P = _run(plan, f32)
        # quadruplets with unpaired quadruples are exactly the oracle's connected set
        has = plan.N_conn > 0.5
        assert np.array_equal(plan.quads[has], d["quads"])
        assert np.array_equal(plan.N_conn[has].astype(np.int64), d["N_quad"])
        assert np.all(np.isnan(Tc[~has]))
        e = oracle.fft_estimator(f64, L, edges, triplets=[], quads=plan.quads)
        scale = e["Tc_M"][has]
        g = (d["N_quad"] >= 100) & (np.abs(d["T"]) >= 0.05 * scale)
        r = rel_err(Tc[has], d["T"])
        assert g.sum() >= 2
        assert r[g].max() < TOL[precision], float(r[g].max())
        rest = (d["N_quad"] >= 100) & ~g
        assert np.all(np.abs(Tc[has] - d["T"])[rest] <= TOL[precision] * 0.05 * scale[rest])
        # the raw T of the same call is the plain four-shell estimator
        assert np.all(rel_err(T, e["T"])[plan.N_quad >= 100] < 1e-3)


@pytest.mark.parametrize("N,L,nb,kind,precision", [(32, 100.0, 5, "lin", "fp32"), (32, 100.0, 5, "lin", "bf16x3"),
                                                    (48, 60.0, 8, "log", "bf16x3")])
def test_connected_matches_fft_estimator(N, L, nb, kind, precision):
    edges = fields.linear_edges(N, L, nb) if kind == "lin" else fields.log_edges(N, L, nb)
    f32 = fields.quadratic_local(N, 1.0, -1.5, 0.3, seed=72).astype(np.float32)
    with fbs.Plan(N, L, edges, precision=precision, trispectrum=True) as plan:
        Tc, T, B, P = _run(plan, f32)
        e = oracle.fft_estimator(f32.astype(np.float64), L, edges, triplets=[], quads=plan.quads)
        assert np.allclose(plan.N_conn, e["N_conn"], rtol=1e-12)
        g = (plan.N_conn >= 100) & (np.abs(e["Tc"]) >= 0.05 * e["Tc_M"])
        paired = (plan.quads[:, 0] == plan.quads[:, 1]) & (plan.quads[:, 2] == plan.quads[:, 3])
        r = rel_err(Tc, e["Tc"])
        assert g.sum() >= 10 and (g & paired).sum() >= 1
        print("connected T N=%d %s %s: %d gated (%d with pairings), max rel %.2e"
              % (N, kind, precision, int(g.sum()), int((g & paired).sum()), float(r[g].max())))
        assert r[g].max() < TOL[precision]
        rest = (plan.N_conn >= 100) & ~g
        assert np.all(np.abs(Tc - e["Tc"])[rest] <= TOL[precision] * 0.05 * e["Tc_M"][rest])
        # quadruplets without pairings: Tc is the raw T (up to the order of two divisions)
        assert np.allclose(Tc[~paired], T[~paired], rtol=1e-13, atol=0)
