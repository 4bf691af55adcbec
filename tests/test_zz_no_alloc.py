"""The allocation-free triple-sum entry point against the plan path.

Some callers cannot call cudaMalloc (their device memory belongs to another
allocator, or the process reserves it all up front); fbs_triple_sums_noalloc
serves them with a static scratch array.  This test feeds it FP32 shell
fields built by the FP64 oracle (Eq. delta_nr) and checks its sums against
the raw sums of fbs_bispectrum on the same field, within the FP32 tolerance
of the other tests (1e-4 relative on gated triplets), on two calls in a row.
Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

import fields
import oracle
import paper_1705_06284_gb300 as fbs
from gpu_util import gate_mask, rel_err

pytestmark = pytest.mark.gpu


def test_noalloc_matches_plan_sums_twice():
    import torch
    N, L = 32, 100.0
    edges = fields.linear_edges(N, L, 6)
    f32 = fields.lognormal(N, 0.5, -2.0, seed=0).astype(np.float32)
    f64 = f32.astype(np.float64)
    with fbs.Plan(N, L, edges, precision="fp32") as plan:
        B, P = plan.bispectrum(torch.from_numpy(f32).cuda())
        torch.cuda.synchronize()
        num_plan, _, _ = plan.sums()
        trip = plan.triplets.copy()
        ntri = plan.N_tri.copy()
    # shell fields of every bin from the oracle, stacked [bin][x][y][z]
    D = oracle.spectrum(f64)
    bins = oracle.bin_index(N, oracle.thresholds(edges, L))
    nb = len(edges) - 1
    I = np.stack([oracle.shell_field(D, bins, b) for b in range(nb)]).astype(np.float32)
    dI = torch.from_numpy(I).cuda()
    dabc = torch.from_numpy(trip.astype(np.int32).ravel()).cuda()
    npts = N ** 3
    M = oracle.fft_estimator(f64, L, edges, triplets=trip)
    g = gate_mask(M["B"], M["M"], ntri)
    assert g.sum() >= 20
    stream = torch.cuda.current_stream().cuda_stream
    prev = None
    for call in range(2):
        num = torch.full((len(trip),), float("nan"), dtype=torch.float64, device="cuda")
        fbs.fbs_triple_sums_noalloc(dI.data_ptr(), nb, npts, npts, dabc.data_ptr(), len(trip),
                                    num.data_ptr(), stream)
        torch.cuda.synchronize()
        got = num.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_err(got, num_plan)[g].max() < 1e-4
        if prev is not None:
            assert np.array_equal(got, prev)  # same inputs, fixed reduction order
        prev = got


def test_noalloc_rejects_oversize():
    import torch
    dI = torch.zeros(8, device="cuda")
    dabc = torch.zeros(3 * 4097, dtype=torch.int32, device="cuda")
    num = torch.zeros(4097, dtype=torch.float64, device="cuda")
    with pytest.raises(fbs.FbsError) as e:
        fbs.fbs_triple_sums_noalloc(dI.data_ptr(), 1, 8, 8, dabc.data_ptr(), 4097, num.data_ptr())
    assert e.value.status == -1
    assert "exceeds the maximum" in str(e.value)
