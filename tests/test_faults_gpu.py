"""Failure paths on the GPU, made without a GPU fault.

* Timeout: the plan option FBS_OPT_TC_WAIT_LIMIT shortens the hand-off waits
  of the tensor-core contraction to one clock cycle, so the first wait that is
  not immediately satisfied gives up.  The kernel then stops issuing work,
  drains what is in flight (those waits keep their long limit), frees its
  tensor memory and returns; the host must see FBS_ERR_TIMEOUT and NaN B and T,
  and the next evaluation with the default limit must give the same numbers as
  before (and the oracle's).
* Out of memory: a process-wide device budget below a plan's needs refuses the
  plan on the host exactly as a failed cudaMalloc would: FBS_ERR_OOM, no plan
  and no bytes left behind.
"""
import numpy as np
import pytest

import fields
import oracle
import paper_1705_06284_gb300 as fbs
from gpu_util import TOL, gate_mask, rel_err

pytestmark = pytest.mark.gpu

FBS_ERR_OOM, FBS_ERR_TIMEOUT = -3, -5


def _case():
    N, L = 32, 100.0
    edges = fields.linear_edges(N, L, 6)
    f32 = fields.lognormal(N, 0.5, -2.0, seed=0).astype(np.float32)
    return N, L, edges, f32


def test_timeout_is_reported_and_the_plan_recovers():
    import torch
    N, L, edges, f32 = _case()
    dev = torch.from_numpy(f32).cuda()
    with fbs.Plan(N, L, edges, precision="bf16x3", trispectrum=True) as plan:
        T0, B0, P0 = plan.trispectrum(dev)
        plan.check()  # a normal evaluation reports nothing
        T0, B0, P0 = T0.cpu().numpy(), B0.cpu().numpy(), P0.cpu().numpy()

        plan.set_option(fbs.FBS_OPT_TC_WAIT_LIMIT, 1)
        # device outputs: the call only enqueues; the timeout is reported by check()
        T, B, P = plan.trispectrum(dev)
        with pytest.raises(fbs.FbsError) as e:
            plan.check()
        assert e.value.status == FBS_ERR_TIMEOUT
        assert np.all(np.isnan(B.cpu().numpy())) and np.all(np.isnan(T.cpu().numpy()))
        assert np.array_equal(P.cpu().numpy(), P0)  # the FFT stages are unaffected
        plan.check()  # reported once, then cleared

        # pageable host outputs: the call waits and reports directly
        Bh, Ph = np.empty(plan.ntrip), np.empty(plan.nbins)
        with pytest.raises(fbs.FbsError) as e:
            plan.bispectrum(dev, Bh, Ph)
        assert e.value.status == FBS_ERR_TIMEOUT
        assert np.all(np.isnan(Bh))

        # an asynchronous caller learns of it at its next call, which runs nothing
        plan.trispectrum(dev)
        torch.cuda.synchronize()
        with pytest.raises(fbs.FbsError) as e:
            plan.trispectrum(dev)
        assert e.value.status == FBS_ERR_TIMEOUT

        # back to the default limit: the same numbers as before the timeouts
        plan.set_option(fbs.FBS_OPT_TC_WAIT_LIMIT, 0)
        T1, B1, P1 = plan.trispectrum(dev)
        plan.check()
        assert np.array_equal(B1.cpu().numpy(), B0)
        assert np.array_equal(T1.cpu().numpy(), T0)
        ref = oracle.direct_bispectrum(f32.astype(np.float64), L, edges)
        M = oracle.fft_estimator(f32.astype(np.float64), L, edges, triplets=ref["triplets"])["M"]
        g = gate_mask(ref["B"], M, ref["N_tri"])
        assert g.sum() > 10
        assert rel_err(B0, ref["B"])[g].max() < TOL["bf16x3"]


def test_device_budget_refuses_a_plan_with_no_leak():
    import torch
    N, L, edges, f32 = _case()
    before = fbs.fbs_device_bytes_in_use()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        fbs.fbs_set_device_budget(before + 4096)  # 4 KiB more than the plans hold now
        with pytest.raises(fbs.FbsError) as e:
            fbs.Plan(N, L, edges, precision="bf16x3")
        assert e.value.status == FBS_ERR_OOM
        assert fbs.fbs_device_bytes_in_use() == before
    finally:
        fbs.fbs_set_device_budget(0)
    torch.cuda.synchronize()
    # nothing of the refused plan stays allocated (allow for allocator slack)
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)
    with fbs.Plan(N, L, edges, precision="bf16x3") as plan:
        assert fbs.fbs_device_bytes_in_use() == before + plan.device_bytes
    assert fbs.fbs_device_bytes_in_use() == before
