"""A plan following another plan's spectrum (fbs_plan_follow): a trispectrum
plan evaluates the field a bispectrum plan has just transformed, with no
upload or forward transform of its own, and gives exactly the results of
the same plan evaluating the field itself; its misuses are refused."""
import numpy as np
import pytest

import fields
import paper_1705_06284_gb300 as fbs

pytestmark = pytest.mark.gpu


def test_follower_equals_standalone_bit_for_bit():
    import torch
    N, L = 48, 60.0
    eB, eT = fields.log_edges(N, L, 10), fields.log_edges(N, L, 6)
    f = [torch.from_numpy(fields.quadratic_local(N, 1.0, -1.5, 0.3, seed=90 + i).astype(np.float32)).cuda()
         for i in range(2)]
    with fbs.Plan(N, L, eB, precision="bf16x3") as pb, \
            fbs.Plan(N, L, eT, precision="bf16x3", trispectrum=True) as alone, \
            fbs.Plan(N, L, eT, precision="bf16x3", trispectrum=True) as pt:
        pt.follow(pb)
        for fld in f:  # two fields in a row: the follower reads the latest spectrum
            Bb, Pb = pb.bispectrum(fld)
            T1, B1, P1 = pt.trispectrum(None)
            T0, B0, P0 = alone.trispectrum(fld)
            torch.cuda.synchronize()
            assert torch.equal(T1, T0) and torch.equal(B1, B0)
            assert torch.equal(torch.nan_to_num(P1), torch.nan_to_num(P0))
        pt.check()
        with pytest.raises(fbs.FbsError):  # a follower takes no field of its own
            pt.trispectrum(f[0])
        pt.follow(None)  # detached: its own field again
        T2, _, _ = pt.trispectrum(f[1])
        torch.cuda.synchronize()
        assert torch.equal(T2, T0)


def test_follow_needs_a_large_enough_spectrum_and_the_same_grid():
    N, L = 32, 50.0
    kf = 2 * np.pi / L
    low = np.linspace(kf, 0.15 * N * kf, 5)  # top edge below the follower's
    with fbs.Plan(N, L, low, precision="fp32") as small, \
            fbs.Plan(N, L, fields.linear_edges(N, L, 5), precision="fp32", trispectrum=True) as t, \
            fbs.Plan(2 * N, L, fields.linear_edges(2 * N, L, 5), precision="fp32") as other:
        with pytest.raises(fbs.FbsError):
            t.follow(small)
        with pytest.raises(fbs.FbsError):
            t.follow(other)
