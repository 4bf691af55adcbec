"""The allocation-free triple-sum entry point, checked against the oracle.

Some callers cannot call cudaMalloc: their device memory belongs to another
allocator that must account for every byte, or the process reserves it all up
front.  fbs_triple_sums_noalloc serves them with a static scratch array.  This
test feeds it FP32 shell fields built by the FP64 oracle (Eq. delta_nr) and
checks its sums against the oracle's FP64 sums sum_x I_a I_b I_c (and against
the plan path's raw sums) within the FP32 tolerance of the other tests (1e-4
relative on gated triplets), on two calls in a row that must agree bit for
bit.  It also covers fields laid out with a stride larger than their length,
a field index outside the caller's array (NaN for that triplet only, no
access) and the largest accepted triplet count.  Kept in a file of its own
that pytest collects last.
"""
import numpy as np
import pytest

import fields
import oracle
import paper_1705_06284_gb300 as fbs
from gpu_util import gate_mask, rel_err

pytestmark = pytest.mark.gpu

MAX_TRIP = 4096


def _setup():
    import torch
    N, L = 32, 100.0
    edges = fields.linear_edges(N, L, 6)
    f32 = fields.lognormal(N, 0.5, -2.0, seed=0).astype(np.float32)
    f64 = f32.astype(np.float64)
    with fbs.Plan(N, L, edges, precision="fp32") as plan:
        plan.bispectrum(torch.from_numpy(f32).cuda())
        torch.cuda.synchronize()
        num_plan, _, _ = plan.sums()
        trip = plan.triplets.copy()
        ntri = plan.N_tri.copy()
    # shell fields of every bin from the oracle, stacked [bin][x][y][z]
    D = oracle.spectrum(f64)
    bins = oracle.bin_index(N, oracle.thresholds(edges, L))
    nb = len(edges) - 1
    I = np.stack([oracle.shell_field(D, bins, b) for b in range(nb)]).astype(np.float32)
    M = oracle.fft_estimator(f64, L, edges, triplets=trip)
    g = gate_mask(M["B"], M["M"], ntri)
    assert g.sum() >= 20
    return N, nb, I, trip, M["num"], num_plan, g


def _call(dI, nfields, stride, npts, abc):
    import torch
    dabc = torch.from_numpy(np.ascontiguousarray(abc, dtype=np.int32).ravel()).cuda()
    n = len(abc)
    num = torch.full((n,), 12345.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    fbs.fbs_triple_sums_noalloc(dI.data_ptr(), nfields, stride, npts, dabc.data_ptr(), n,
                                num.data_ptr(), stream)
    torch.cuda.synchronize()
    return num.cpu().numpy()


def test_noalloc_matches_oracle_twice():
    import torch
    N, nb, I, trip, num_ref, num_plan, g = _setup()
    dI = torch.from_numpy(I).cuda()
    npts = N ** 3
    prev = None
    for call in range(2):
        got = _call(dI, nb, npts, npts, trip)
        assert np.all(np.isfinite(got))
        assert rel_err(got, num_ref)[g].max() < 1e-4     # FP64 oracle sums
        assert rel_err(got, num_plan)[g].max() < 1e-4    # the plan path on the same field
        if prev is not None:
            assert np.array_equal(got, prev)  # same inputs, fixed reduction order
        prev = got


def test_noalloc_strided_fields_bad_index_and_max_count():
    import torch
    N, nb, I, trip, num_ref, num_plan, g = _setup()
    npts = N ** 3
    stride = npts + 37  # fields padded apart; the pad holds values that must not be read
    Ipad = np.full((nb, stride), 1e30, dtype=np.float32)
    Ipad[:, :npts] = I.reshape(nb, npts)
    dI = torch.from_numpy(Ipad).cuda()
    base = _call(dI, nb, stride, npts, trip)
    assert rel_err(base, num_ref)[g].max() < 1e-4
    # one triplet names a field past the caller's array: NaN there only
    bad = trip.copy()
    bad[3] = (0, 1, nb)
    got = _call(dI, nb, stride, npts, bad)
    assert np.isnan(got[3])
    keep = np.arange(len(trip)) != 3
    assert np.array_equal(got[keep], base[keep])
    # the largest accepted count: the triplets repeated to 4096 entries
    reps = np.resize(trip, (MAX_TRIP, 3))
    big = _call(dI, nb, stride, npts, reps)
    assert np.array_equal(big, np.resize(base, MAX_TRIP))


def test_noalloc_rejects_oversize():
    import torch
    dI = torch.zeros(8, device="cuda")
    dabc = torch.zeros(3 * (MAX_TRIP + 1), dtype=torch.int32, device="cuda")
    num = torch.zeros(MAX_TRIP + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(fbs.FbsError) as e:
        fbs.fbs_triple_sums_noalloc(dI.data_ptr(), 1, 8, 8, dabc.data_ptr(), MAX_TRIP + 1, num.data_ptr())
    assert e.value.status == -1
    assert "exceeds the maximum" in str(e.value)
