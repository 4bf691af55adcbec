"""GPU parity of the tensor-core (tcgen05) contraction: BF16x3 within 2e-4
relative of the FP64 oracle on gated triplets, exact counts; plain BF16
error is reported, not gated."""
import numpy as np
import pytest

import fields
import oracle
import paper_1705_06284_gb300 as fbs
from gpu_util import check_bispectrum, check_trispectrum, gate_mask, rel_err, run

pytestmark = pytest.mark.gpu


def _field(kind, N, seed):
    if kind == "lognormal":
        return fields.lognormal(N, 0.6, -1.5, seed=seed)
    if kind == "bubbles":
        return fields.bubbles(N, max(1.5, N / 10), 0.4, seed=seed)
    return fields.quadratic_local(N, 0.5, -1.5, 0.3, seed=seed)


def test_tc_tiny_first():
    """Smallest case first: one pair tile, Npad = 16."""
    N, L = 16, 50.0
    edges = fields.linear_edges(N, L, 3)
    f32 = _field("lognormal", N, 1).astype(np.float32)
    with fbs.Plan(N, L, edges, precision="bf16x3") as plan:
        B, P = run(plan, f32)
        gmax, amax, ng = check_bispectrum(plan, B, P, f32, L, edges, "bf16x3")
    print("tiny: gated %d max %.2e all %.2e" % (ng, gmax, amax))


TC_CASES = [
    (24, 80.0, "lin", 5, "quadratic", 4),
    (32, 100.0, "lin", 6, "lognormal", 0),
    (32, 100.0, "log", 8, "bubbles", 5),
    (48, 60.0, "lin", 12, "lognormal", 6),     # several pair tiles
    (64, 200.0, "lin", 16, "quadratic", 7),
    (72, 72.0, "lin", 4, "lognormal", 8),
]


@pytest.mark.parametrize("N,L,kind,nb,fk,seed", TC_CASES)
def test_bf16x3_matches_direct_oracle(N, L, kind, nb, fk, seed):
    edges = fields.linear_edges(N, L, nb) if kind == "lin" else fields.log_edges(N, L, nb)
    f32 = _field(fk, N, seed).astype(np.float32)
    with fbs.Plan(N, L, edges, precision="bf16x3") as plan:
        B, P = run(plan, f32)
        gmax, amax, ng = check_bispectrum(plan, B, P, f32, L, edges, "bf16x3")
        plan.set_precision("bf16")
        B1, _ = run(plan, f32)
        plan.set_precision("fp32")
        B32, _ = run(plan, f32)
    ref = oracle.direct_bispectrum(f32.astype(np.float64), L, edges)
    M = oracle.fft_estimator(f32.astype(np.float64), L, edges, triplets=ref["triplets"])["M"]
    g = gate_mask(ref["B"], M, ref["N_tri"])
    e1 = rel_err(B1, ref["B"])[g].max() if g.any() else 0.0
    e32 = rel_err(B32, ref["B"])[g].max() if g.any() else 0.0
    print("N=%d pairs-tiles ok: bf16x3 %.2e  bf16 %.2e (reported)  fp32 %.2e" % (N, gmax, e1, e32))


def test_bf16x3_many_pairs_several_groups():
    """64 narrow linear bins on a 96^3 grid: more pair tiles than one CTA's
    tensor memory holds, so the tiles split into several CTA groups."""
    N, L = 96, 96.0
    edges = fields.linear_edges(N, L, 64)
    f32 = _field("lognormal", N, 21).astype(np.float32)
    with fbs.Plan(N, L, edges, precision="bf16x3") as plan:
        npairs = len({(int(t[1]), int(t[2])) for t in plan.triplets})
        assert npairs > 1024
        B, P = run(plan, f32)
        gmax, amax, ng = check_bispectrum(plan, B, P, f32, L, edges, "bf16x3")
    print("96^3 x 64: %d pairs, gated %d max %.2e" % (npairs, ng, gmax))


def test_bf16x3_deterministic_and_host_buffers():
    N, L = 32, 100.0
    edges = fields.linear_edges(N, L, 6)
    f32 = _field("bubbles", N, 3).astype(np.float32)
    with fbs.Plan(N, L, edges, precision="bf16x3") as plan:
        Bd, Pd = run(plan, f32, device=True)
        Bh, Ph = run(plan, f32, device=False)
        Bd2, _ = run(plan, f32, device=True)
        assert np.array_equal(Bd, Bh) and np.array_equal(Bd, Bd2)


@pytest.mark.parametrize("N,nb,kind", [(16, 4, "lin"), (32, 6, "log"), (48, 8, "lin")])
def test_trispectrum_bf16x3_matches_oracle(N, nb, kind):
    """Quadruplets as a Gram of pair products on the tensor cores."""
    import torch
    L = 60.0
    edges = fields.linear_edges(N, L, nb) if kind == "lin" else fields.log_edges(N, L, nb)
    f32 = _field("bubbles", N, 13).astype(np.float32)
    with fbs.Plan(N, L, edges, precision="bf16x3", trispectrum=True) as plan:
        T, B, P = plan.trispectrum(torch.from_numpy(f32).cuda())
        torch.cuda.synchronize()
        T, B, P = T.cpu().numpy(), B.cpu().numpy(), P.cpu().numpy()
        check_bispectrum(plan, B, P, f32, L, edges, "bf16x3")
        assert plan.quad_counts_exact
        m, n = check_trispectrum(plan, T, f32, L, edges, 2e-4)
    print("T N=%d quads %d gated %d max %.2e" % (N, len(T), n, m))


@pytest.mark.parametrize("N,nb,quads", [(32, 6, False), (48, 12, False), (32, 6, True)])
def test_wide_orientation_matches(monkeypatch, N, nb, quads):
    """The wide tensor-core kernel (left rows [hi; lo] as operand A, right
    pair products as operand B with N <= 256; BF16x4) matches the oracle."""
    import torch
    L = 70.0
    edges = fields.linear_edges(N, L, nb)
    f32 = _field("lognormal", N, 31).astype(np.float32)
    with fbs.Plan(N, L, edges, precision="bf16x3", trispectrum=quads) as plan:
        plan.set_tc_wide(True)
        if quads:
            T, B, P = plan.trispectrum(torch.from_numpy(f32).cuda())
            torch.cuda.synchronize()
            B, P, T = B.cpu().numpy(), P.cpu().numpy(), T.cpu().numpy()
            check_trispectrum(plan, T, f32, L, edges, 2e-4)
        else:
            B, P = run(plan, f32)
        check_bispectrum(plan, B, P, f32, L, edges, "bf16x3")


@pytest.mark.parametrize("quads", [False, True])
def test_warp_roles_give_identical_results(quads):
    """FBS_OPT_TC_ROLES 1 (16 warps form the pair products and build operand B
    in turn) and 2 (8 + 8 warps concurrently), at the same 64-point pipeline
    steps, issue the same MMAs in the same order: bit-identical sums, and
    both match the oracle."""
    import torch
    N, L, nb = 48, 60.0, 10
    edges = fields.linear_edges(N, L, nb)
    f32 = _field("quadratic", N, 31).astype(np.float32)
    f = torch.from_numpy(f32).cuda()
    out = {}
    with fbs.Plan(N, L, edges, precision="bf16x3", trispectrum=quads) as plan:
        plan.set_option(fbs.FBS_OPT_TC_CHUNK, 1)  # the same 64-point steps for both
        plan.set_option(fbs.FBS_OPT_TC_STACK, 1)  # the same MMAs (stacking needs 16 product warps)
        for roles in (1, 2):
            plan.set_option(fbs.FBS_OPT_TC_ROLES, roles)
            if quads:
                T, B, P = plan.trispectrum(f)
            else:
                B, P = plan.bispectrum(f)
                T = None
            torch.cuda.synchronize()
            out[roles] = (B.cpu().numpy(), P.cpu().numpy(), None if T is None else T.cpu().numpy())
        assert np.array_equal(out[1][0], out[2][0])
        assert np.array_equal(out[1][1], out[2][1])
        if quads:
            assert np.array_equal(out[1][2], out[2][2])
            check_trispectrum(plan, out[2][2], f32, L, edges, 2e-4)
        check_bispectrum(plan, out[2][0], out[2][1], f32, L, edges, "bf16x3")


@pytest.mark.parametrize("quads", [False, True])
def test_chunk_sizes_agree(quads):
    """FBS_OPT_TC_CHUNK 1 (64-point pipeline steps) and 2 (128-point steps,
    two K-atoms per step) both match the oracle and agree with each other to
    rounding (the CTAs' point ranges differ, so the sums are grouped
    differently)."""
    import torch
    N, L, nb = 48, 60.0, 10
    edges = fields.linear_edges(N, L, nb)
    f32 = _field("lognormal", N, 33).astype(np.float32)
    f = torch.from_numpy(f32).cuda()
    out = {}
    with fbs.Plan(N, L, edges, precision="bf16x3", trispectrum=quads) as plan:
        for chunk in (1, 2):
            plan.set_option(fbs.FBS_OPT_TC_CHUNK, chunk)
            if quads:
                T, B, P = plan.trispectrum(f)
            else:
                B, P = plan.bispectrum(f)
                T = None
            torch.cuda.synchronize()
            out[chunk] = (B.cpu().numpy(), P.cpu().numpy(), None if T is None else T.cpu().numpy())
            check_bispectrum(plan, out[chunk][0], out[chunk][1], f32, L, edges, "bf16x3")
            if quads:
                check_trispectrum(plan, out[chunk][2], f32, L, edges, 2e-4)
        ref = oracle.direct_bispectrum(f32.astype(np.float64), L, edges)
        M = oracle.fft_estimator(f32.astype(np.float64), L, edges, triplets=ref["triplets"])["M"]
        g = gate_mask(ref["B"], M, ref["N_tri"])
        # each is within the BF16x3 gate of the oracle; so is their difference
        assert np.all(np.abs(out[1][0] - out[2][0])[g] <= 2e-4 * np.abs(ref["B"][g]))


@pytest.mark.parametrize("N,L,nb,kind", [(48, 60.0, 12, "lin"), (64, 200.0, 16, "log")])
def test_pair_cover_matches_oracle(N, L, nb, kind):
    """FBS_OPT_TC_PAIRS 0 (each triplet carried by one of its three pairs,
    greedy set cover) and 1 (by its two largest bins): both match the oracle
    and agree with each other within the BF16x3 gate."""
    import torch
    edges = fields.linear_edges(N, L, nb) if kind == "lin" else fields.log_edges(N, L, nb)
    f32 = _field("bubbles", N, 61).astype(np.float32)
    f = torch.from_numpy(f32).cuda()
    out = {}
    ref = oracle.direct_bispectrum(f32.astype(np.float64), L, edges)
    with fbs.Plan(N, L, edges, precision="bf16x3") as plan:
        for pairs in (0, 1):
            plan.set_option(fbs.FBS_OPT_TC_PAIRS, pairs)
            B, P = plan.bispectrum(f)
            torch.cuda.synchronize()
            out[pairs] = B.cpu().numpy()
            check_bispectrum(plan, out[pairs], P.cpu().numpy(), f32, L, edges, "bf16x3", ref=ref)
    M = oracle.fft_estimator(f32.astype(np.float64), L, edges, triplets=ref["triplets"])["M"]
    g = gate_mask(ref["B"], M, ref["N_tri"])
    assert np.all(np.abs(out[0] - out[1])[g] <= 2e-4 * np.abs(ref["B"][g]))


def test_pair_cover_trispectrum_matches_oracle():
    """Trispectrum pass with FBS_OPT_TC_PAIRS 0 (each quadruplet's pairing and
    inner/outer roles chosen by a cover that keeps one 128-row outer tile and
    few inner rows) and 1 (inner (a, b), outer (c, d)): both match the FP64
    estimator for T and the oracle for B."""
    import torch
    N, L, nb = 48, 60.0, 10
    edges = fields.log_edges(N, L, nb)
    f32 = _field("quadratic", N, 71).astype(np.float32)
    f = torch.from_numpy(f32).cuda()
    ref = oracle.direct_bispectrum(f32.astype(np.float64), L, edges)
    out = {}
    with fbs.Plan(N, L, edges, precision="bf16x3", trispectrum=True) as plan:
        for pairs in (0, 1):
            plan.set_option(fbs.FBS_OPT_TC_PAIRS, pairs)
            T, B, P = plan.trispectrum(f)
            torch.cuda.synchronize()
            out[pairs] = T.cpu().numpy()
            check_trispectrum(plan, out[pairs], f32, L, edges, 2e-4)
            check_bispectrum(plan, B.cpu().numpy(), P.cpu().numpy(), f32, L, edges, "bf16x3", ref=ref)


@pytest.mark.parametrize("quads,N,nb", [(False, 64, 16), (True, 48, 10), (True, 96, 8)])
def test_merged_hi_lo_products_match_oracle(quads, N, nb):
    """FBS_OPT_TC_MERGE 0 (hi and lo rows of the inner operand in one MMA of
    N = 2 Npad, lo*hi in a second) and 1 (three MMAs per K step) both meet the
    BF16x3 gate against the oracle; the 96^3 case runs several accumulator
    flushes per CTA."""
    import torch
    L = float(N)
    edges = fields.linear_edges(N, L, nb)
    f32 = _field("quadratic", N, 34).astype(np.float32)
    f = torch.from_numpy(f32).cuda()
    out = {}
    with fbs.Plan(N, L, edges, precision="bf16x3", trispectrum=quads) as plan:
        for merge in (0, 1):
            plan.set_option(fbs.FBS_OPT_TC_MERGE, merge)
            if quads:
                T, B, P = plan.trispectrum(f)
            else:
                B, P = plan.bispectrum(f)
                T = None
            torch.cuda.synchronize()
            plan.check()
            out[merge] = (B.cpu().numpy(), P.cpu().numpy(), None if T is None else T.cpu().numpy())
            if N <= 64:
                check_bispectrum(plan, out[merge][0], out[merge][1], f32, L, edges, "bf16x3")
            if quads:
                check_trispectrum(plan, out[merge][2], f32, L, edges, 2e-4)
        # the two assignments of the products round differently, nothing more
        big = np.abs(out[1][0]) > 1e-3 * np.abs(out[1][0]).max()
        assert np.all(np.abs(out[0][0] - out[1][0])[big] <= 2e-4 * np.abs(out[1][0][big]) + 1e-6 * np.abs(out[1][0]).max())


@pytest.mark.parametrize("quads,N,nb,roles", [(False, 64, 16, 1), (False, 64, 28, 1), (False, 96, 64, 1),
                                              (True, 96, 8, 1), (True, 48, 10, 2)])
def test_operand_b_stage_depths_give_identical_sums(quads, N, nb, roles):
    """FBS_OPT_TC_BSTAGES 2, 3 and 4 (the depth of the operand-B ring in
    shared memory; each accumulator flush deferred until the next step's
    operands are handed off) issue the same MMAs into the same accumulators in
    the same order: bit-identical sums, tensor-core job diagnostics that name
    the depth used, and the oracle's values.  96^3 runs several flushes per
    CTA, 64^3 one deferred flush and the last; 28 and 64 bins give CTAs with
    several pair tiles (up to the A ring's depth the flush is deferred, past
    it not); roles 2 has the operand-B warps apart from the pair-product
    warps."""
    import torch
    L = float(N)
    edges = fields.linear_edges(N, L, nb)
    f32 = _field("quadratic", N, 35).astype(np.float32)
    f = torch.from_numpy(f32).cuda()
    out = {}
    with fbs.Plan(N, L, edges, precision="bf16x3", trispectrum=quads) as plan:
        plan.set_option(fbs.FBS_OPT_TC_ROLES, roles)
        for depth in (2, 3, 4):
            plan.set_option(fbs.FBS_OPT_TC_BSTAGES, depth)
            if quads:
                T, B, P = plan.trispectrum(f)
            else:
                B, P = plan.bispectrum(f)
                T = None
            torch.cuda.synchronize()
            plan.check()
            used = [j["stages"][1] for lvl in plan.tc_info() for j in lvl.values()]
            assert used and all(2 <= u <= depth for u in used)
            if depth == 2:
                assert all(u == 2 for u in used)
            out[depth] = (B.cpu().numpy(), P.cpu().numpy(), None if T is None else T.cpu().numpy())
        for depth in (3, 4):
            assert np.array_equal(out[2][0], out[depth][0])
            if quads:
                assert np.array_equal(out[2][2], out[depth][2])
        if quads:
            check_trispectrum(plan, out[4][2], f32, L, edges, 2e-4)
        if N <= 64 and nb <= 16:
            check_bispectrum(plan, out[4][0], out[4][1], f32, L, edges, "bf16x3")


@pytest.mark.parametrize("N,nb,kind", [(48, 10, "lin"), (96, 8, "lin"), (64, 16, "log")])
def test_inner_pairs_from_operand_a_are_identical(N, nb, kind):
    """FBS_OPT_TC_BFROMA 0 (in a one-tile trispectrum pass the operand-A
    warps also store each inner pair row's product into operand B) and 1
    (every inner row built from the field stage) form the same FP32 products
    and splits: bit-identical sums that match the oracle, and diagnostics
    that say which launch took the inner pairs from operand A."""
    import torch
    L = float(N)
    edges = fields.linear_edges(N, L, nb) if kind == "lin" else fields.log_edges(N, L, nb)
    f32 = _field("quadratic", N, 36).astype(np.float32)
    f = torch.from_numpy(f32).cuda()
    out, used = {}, {}
    with fbs.Plan(N, L, edges, precision="bf16x3", trispectrum=True) as plan:
        plan.set_option(fbs.FBS_OPT_TC_STACK, 1)  # the same MMAs (without the feed a small job stacks)
        for opt in (0, 1):
            plan.set_option(fbs.FBS_OPT_TC_BFROMA, opt)
            T, B, P = plan.trispectrum(f)
            torch.cuda.synchronize()
            plan.check()
            out[opt] = (B.cpu().numpy(), T.cpu().numpy())
            used[opt] = [lvl["fused"]["b_from_a"] for lvl in plan.tc_info() if "fused" in lvl]
        assert used[1] and not any(used[1])
        assert any(used[0]), used
        assert np.array_equal(out[0][0], out[1][0])
        assert np.array_equal(out[0][1], out[1][1])
        check_trispectrum(plan, out[0][1], f32, L, edges, 2e-4)


@pytest.mark.parametrize("quads,N,nb,kind", [(False, 48, 10, "lin"), (False, 64, 12, "log"), (True, 48, 8, "lin")])
def test_stacked_operand_a_matches_oracle(quads, N, nb, kind):
    """FBS_OPT_TC_STACK 0 (a tile of at most 64 outer pairs: operand A's hi
    rows in 0..63 and lo rows in 64..127, one MMA per K step that also forms
    the lo*lo products) and 1 (two MMAs per K step) both meet the BF16x3 gate
    against the oracle and agree to rounding; the diagnostics report the
    stacked launches (merged = 2).  The trispectrum case turns the operand-A
    feed off (the two exclude each other)."""
    import torch
    L = float(N)
    edges = fields.linear_edges(N, L, nb) if kind == "lin" else fields.log_edges(N, L, nb)
    f32 = _field("quadratic", N, 37).astype(np.float32)
    f = torch.from_numpy(f32).cuda()
    out, shape = {}, {}
    with fbs.Plan(N, L, edges, precision="bf16x3", trispectrum=quads) as plan:
        plan.set_option(fbs.FBS_OPT_TC_BFROMA, 1)
        for stack in (0, 1):
            plan.set_option(fbs.FBS_OPT_TC_STACK, stack)
            if quads:
                T, B, P = plan.trispectrum(f)
            else:
                B, P = plan.bispectrum(f)
                T = None
            torch.cuda.synchronize()
            plan.check()
            out[stack] = (B.cpu().numpy(), P.cpu().numpy(), None if T is None else T.cpu().numpy())
            shape[stack] = [j["merged"] for lvl in plan.tc_info() for j in lvl.values()]
        assert 2 in shape[0], shape
        assert 2 not in shape[1], shape
        for stack in (0, 1):
            check_bispectrum(plan, out[stack][0], out[stack][1], f32, L, edges, "bf16x3")
            if quads:
                check_trispectrum(plan, out[stack][2], f32, L, edges, 2e-4)
        big = np.abs(out[1][0]) > 1e-3 * np.abs(out[1][0]).max()
        assert np.all(np.abs(out[0][0] - out[1][0])[big] <= 2e-4 * np.abs(out[1][0][big]) + 1e-6 * np.abs(out[1][0]).max())
