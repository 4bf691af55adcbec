"""GPU parity: the CUDA path through the C ABI versus the FP64 oracle.

Counts are compared bit-exactly; B, P and T within the tolerances of the
precision mode (FP32: 1e-4 relative on triplets with N_tri >= 100 and a
non-negligible |B|; see tests/gpu_util.py)."""
import math
import os

import numpy as np
import pytest

import fields
import oracle
import paper_1705_06284_gb300 as fbs
from gpu_util import TOL, check_bispectrum, check_trispectrum, gate_mask, rel_err, run

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    meta, rows = {}, []
    for line in open(os.path.join(HERE, "golden", "lognormal32_lin6.txt")):
        if line.startswith("# ") and line.split()[1] in ("edges", "P", "shell"):
            meta[line.split()[1]] = [float(v) for v in line.split()[2:]]
        elif not line.startswith("#"):
            rows.append(line.split())
    trip = np.array([[int(r[0]), int(r[1]), int(r[2])] for r in rows], dtype=np.int32)
    ntri = np.array([int(r[3]) for r in rows], dtype=np.int64)
    B = np.array([float(r[4]) for r in rows])
    M = np.array([float(r[5]) for r in rows])
    return meta, trip, ntri, B, M


def test_lognormal32_golden_fp32():
    """The 32^3 lognormal configuration against the stored oracle values."""
    meta, trip, ntri, Bref, M = _golden()
    N, L = 32, 100.0
    f32 = fields.lognormal(N, 0.5, -2.0, seed=0).astype(np.float32)
    with fbs.Plan(N, L, meta["edges"], precision="fp32") as plan:
        assert plan.ntrip == 49
        assert np.array_equal(plan.triplets, trip)
        assert np.array_equal(plan.N_tri, ntri)
        assert list(plan.shell) == [int(v) for v in meta["shell"]]
        B, P = run(plan, f32)
    g = gate_mask(Bref, M, ntri)
    assert g.sum() >= 30
    assert rel_err(B, Bref)[g].max() < 1e-4
    assert np.all(rel_err(P, np.array(meta["P"])) < 1e-5)


CASES = [
    # (N, L, kind, nbins, field, seed)
    (8, 10.0, "lin", 2, "lognormal", 1),
    (12, 30.0, "lin", 3, "bubbles", 2),
    (16, 50.0, "log", 5, "lognormal", 3),
    (24, 80.0, "lin", 5, "quadratic", 4),      # radix 3
    (32, 100.0, "log", 8, "bubbles", 5),
    (48, 60.0, "lin", 6, "lognormal", 6),      # radix 3, several tiles
    (64, 200.0, "lin", 8, "quadratic", 7),
    (72, 72.0, "lin", 4, "lognormal", 8),      # 2^3 3^2
]


def _field(kind, N, seed):
    if kind == "lognormal":
        return fields.lognormal(N, 0.6, -1.5, seed=seed)
    if kind == "bubbles":
        return fields.bubbles(N, max(1.5, N / 10), 0.4, seed=seed)
    return fields.quadratic_local(N, 0.5, -1.5, 0.3, seed=seed)


@pytest.mark.parametrize("N,L,kind,nb,fk,seed", CASES)
def test_fp32_matches_direct_oracle(N, L, kind, nb, fk, seed):
    edges = fields.linear_edges(N, L, nb) if kind == "lin" else fields.log_edges(N, L, nb)
    f32 = _field(fk, N, seed).astype(np.float32)
    with fbs.Plan(N, L, edges, precision="fp32") as plan:
        B, P = run(plan, f32)
        gmax, amax, ng = check_bispectrum(plan, B, P, f32, L, edges, "fp32")
    print("N=%d gated=%d max gated rel %.2e, max rel %.2e" % (N, ng, gmax, amax))


def test_small_slabs_and_ragged_chunks(monkeypatch):
    """Force many thin slabs (slab point counts not multiples of the chunk)."""
    monkeypatch.setenv("FBS_SLAB_MB", "1")
    N, L = 24, 50.0
    edges = fields.linear_edges(N, L, 4)
    f32 = _field("lognormal", N, 11).astype(np.float32)
    with fbs.Plan(N, L, edges, precision="fp32") as plan:
        B, P = run(plan, f32)
        check_bispectrum(plan, B, P, f32, L, edges, "fp32")


def test_host_buffers_match_device_buffers():
    N, L = 32, 100.0
    edges = fields.linear_edges(N, L, 6)
    f32 = _field("bubbles", N, 3).astype(np.float32)
    with fbs.Plan(N, L, edges) as plan:
        Bd, Pd = run(plan, f32, device=True)
        Bh, Ph = run(plan, f32, device=False)
        assert isinstance(Bh, np.ndarray)
        assert np.array_equal(Bd, Bh) and np.array_equal(Pd, Ph)
        # repeated calls are deterministic
        Bd2, _ = run(plan, f32, device=True)
        assert np.array_equal(Bd, Bd2)


def test_empty_bins_and_nan_power():
    # log bins on a small grid: the narrow low shells hold no lattice point
    N, L = 32, 2 * math.pi
    edges = np.geomspace(1.0, 8.0, 17)
    f32 = _field("lognormal", N, 1).astype(np.float32)
    with fbs.Plan(N, L, edges) as plan:
        assert (plan.shell == 0).sum() >= 3
        B, P = run(plan, f32)
        check_bispectrum(plan, B, P, f32, L, edges, "fp32")
        assert np.all(np.isnan(P[plan.shell == 0]))
        assert not np.any(np.isin(plan.triplets, np.nonzero(plan.shell == 0)[0]))


def test_aliased_full_cover_sum_rules():
    """Shells covering every mode (closure modulo N): sum N_tri = N_pix^2 and
    the skewness sum rule (Eq. skew) hold on the GPU path too."""
    N, L = 12, 30.0
    kf = 2 * math.pi / L
    top = 3 * (N // 2) ** 2 + 1
    edges = [kf * math.sqrt(s) for s in (0.0, 3.5, 10.5, 30.5, top + 0.5)]
    f32 = _field("lognormal", N, 2).astype(np.float32)
    with fbs.Plan(N, L, edges, allow_aliased=True) as plan:
        B, P = run(plan, f32)
        ref = oracle.direct_bispectrum(f32.astype(np.float64), L, edges)
        check_bispectrum(plan, B, P, f32, L, edges, "fp32", ref=ref)
        # ordered-sum rule: every ordered (m1, m2) closes with one m3
        nb = len(edges) - 1
        tot = 0
        for (a, b, c), n in zip(plan.triplets, plan.N_tri):
            perms = len({(a, b, c), (a, c, b), (b, a, c), (b, c, a), (c, a, b), (c, b, a)})
            tot += perms * int(n)
        assert tot == (N ** 3) ** 2
        V, npix = L ** 3, float(N ** 3)
        skew = 0.0
        for (a, b, c), n, Bv in zip(plan.triplets, plan.N_tri, B):
            perms = len({(a, b, c), (a, c, b), (b, a, c), (b, c, a), (c, a, b), (c, b, a)})
            skew += perms * n * Bv
        skew /= V * V
        f = f32.astype(np.float64)
        assert abs(skew - np.mean(f ** 3)) <= 1e-4 * np.mean(np.abs(f) ** 3)


def test_trispectrum_matches_oracle():
    N, L = 16, 40.0
    edges = fields.linear_edges(N, L, 4)
    f32 = _field("bubbles", N, 9).astype(np.float32)
    with fbs.Plan(N, L, edges, trispectrum=True) as plan:
        import torch
        T, B, P = plan.trispectrum(torch.from_numpy(f32).cuda())
        torch.cuda.synchronize()
        T, B, P = T.cpu().numpy(), B.cpu().numpy(), P.cpu().numpy()
        check_bispectrum(plan, B, P, f32, L, edges, "fp32")
        g = oracle.fft_estimator(f32.astype(np.float64), L, edges, triplets=[], quads=plan.quads)
        assert plan.quad_counts_exact
        assert np.array_equal(plan.N_quad, g["N_quad"])
        # every candidate with a non-zero count is in the plan
        nb = len(edges) - 1
        allq = [(a, b, c, d) for a in range(nb) for b in range(a, nb) for c in range(b, nb)
                for d in range(c, nb)]
        ga = oracle.fft_estimator(f32.astype(np.float64), L, edges, triplets=[], quads=allq)
        closed = [q for q, n in zip(allq, ga["N_quad"]) if n > 0]
        assert [tuple(q) for q in plan.quads] == closed
        r = rel_err(T, g["T"])
        assert np.all(r[plan.N_quad >= 100] < 1e-4), float(r.max())


def test_trispectrum_direct_tiny():
    N, L = 8, 20.0
    edges = fields.linear_edges(N, L, 2)
    f32 = _field("lognormal", N, 4).astype(np.float32)
    t = oracle.direct_trispectrum(f32.astype(np.float64), L, edges)
    with fbs.Plan(N, L, edges, trispectrum=True) as plan:
        T, B, P = plan.trispectrum(f32)
        assert np.array_equal(plan.quads, t["quads"])
        assert np.array_equal(plan.N_quad, t["N_quad"])
        assert np.all(rel_err(T, t["T"]) < 1e-4)


def test_plane_waves_closed_form_on_gpu():
    # B of three plane waves on a closed triangle (closed form in the oracle pins)
    N, L = 16, 2 * math.pi
    A, phi = (0.7, -0.4, 1.3), (0.3, -1.1, 2.0)
    f = fields.plane_waves(N, [((1, 0, 0), A[0], phi[0]), ((0, 2, 0), A[1], phi[1]),
                               ((-1, -2, 0), A[2], phi[2])])
    edges = [0.9, 1.1, 1.9, 2.1, 2.2, 2.3]
    f32 = f.astype(np.float32)
    with fbs.Plan(N, L, edges, allow_aliased=True) as plan:
        B, P = run(plan, f32)
        num, _, _ = plan.sums()
        i = [k for k, t in enumerate(plan.triplets) if tuple(t) == (0, 2, 4)][0]
        npix = N ** 3
        expect = 2 * (npix / 2) ** 3 * np.prod(A) * math.cos(sum(phi)) * npix
        assert abs(num[i] - expect) <= 1e-4 * abs(expect)


@pytest.mark.parametrize("N,L,nb,precision,quads,M", [
    (64, 200.0, 8, "fp32", False, 48),
    (72, 72.0, 4, "bf16x3", False, 54),      # M = 2 * 3^3: radix-3 only inverse stages
    (32, 100.0, 6, "fp32", True, 32),        # 4R + 1 > 24: no smaller grid
    (48, 60.0, 6, "bf16x3", False, 36),
])
def test_reduced_grid_matches_full_grid(N, L, nb, precision, quads, M):
    """A SINGLE_GRID plan evaluates the shell fields on M^3 (M > 3R, or 4R with
    quadruplets) and rescales the sums by (N/M)^3; a FULL_GRID plan evaluates
    on N^3.  Both must agree with each other and with the oracle."""
    edges = fields.linear_edges(N, L, nb)
    f32 = _field("quadratic", N, 11).astype(np.float32)
    with fbs.Plan(N, L, edges, precision=precision, trispectrum=quads, single_grid=True) as red, \
            fbs.Plan(N, L, edges, precision=precision, trispectrum=quads, full_grid=True) as full:
        assert red.eval_grid == M
        assert full.eval_grid == N
        assert np.array_equal(red.N_tri, full.N_tri)
        if quads:
            import torch
            f = torch.from_numpy(f32).cuda()
            Tr, Br, Pr = red.trispectrum(f)
            Tf, Bf, Pf = full.trispectrum(f)
            torch.cuda.synchronize()
            Br, Bf, Pr, Pf, Tr, Tf = (x.cpu().numpy() for x in (Br, Bf, Pr, Pf, Tr, Tf))
            assert np.array_equal(Tr, Tf)  # same grid, same kernels: bit-identical
        else:
            Br, Pr = run(red, f32)
            Bf, Pf = run(full, f32)
        check_bispectrum(red, Br, Pr, f32, L, edges, precision)
        check_bispectrum(full, Bf, Pf, f32, L, edges, precision)
    assert np.all(rel_err(Pr, Pf)[np.isfinite(Pf)] < 2e-5)


def test_aliased_plans_use_the_input_grid():
    N, L = 32, 100.0
    edges = fields.linear_edges(N, L, 4)
    with fbs.Plan(N, L, edges, allow_aliased=True) as plan:
        assert plan.eval_grid == N


def test_host_fields_back_to_back_without_waiting():
    """Pinned host fields with device outputs: each call only enqueues work and
    returns.  The host copy runs on the plan's copy stream, which overlaps the
    other plan's kernels but must not overwrite the staging buffer before the
    previous forward transform has read it: every result equals the
    device-field result bit for bit."""
    import torch
    N, L = 48, 60.0
    eB, eT = fields.linear_edges(N, L, 6), fields.linear_edges(N, L, 4)
    fs = {"1": _field("quadratic", N, 41).astype(np.float32), "2": _field("lognormal", N, 42).astype(np.float32)}
    dev = torch.device("cuda")
    with fbs.Plan(N, L, eB, precision="bf16x3") as pb, \
            fbs.Plan(N, L, eT, precision="bf16x3", trispectrum=True) as pt:
        ref = {}
        for k, f in fs.items():
            d = torch.from_numpy(f).to(dev)
            B, P = pb.bispectrum(d)
            T, B4, P4 = pt.trispectrum(d)
            torch.cuda.synchronize()
            ref[k] = (B.cpu().numpy(), T.cpu().numpy())
        hosts = {k: torch.from_numpy(f).pin_memory() for k, f in fs.items()}
        outs = []
        for _ in range(3):
            for k in ("1", "2"):
                B = torch.empty(pb.ntrip, dtype=torch.float64, device=dev)
                P = torch.empty(pb.nbins, dtype=torch.float64, device=dev)
                pb.bispectrum(hosts[k], B, P)
                T = torch.empty(pt.nquad, dtype=torch.float64, device=dev)
                B4 = torch.empty(pt.ntrip, dtype=torch.float64, device=dev)
                P4 = torch.empty(pt.nbins, dtype=torch.float64, device=dev)
                pt.trispectrum(hosts[k], T, B4, P4)
                outs.append((k, B, T))
        torch.cuda.synchronize()
        for k, B, T in outs:
            assert np.array_equal(B.cpu().numpy(), ref[k][0])
            assert np.array_equal(T.cpu().numpy(), ref[k][1])


def test_pinned_host_outputs_filled_once_the_stream_passes():
    """Page-locked host outputs: the call enqueues the copies and returns; after
    the plan's stream is synchronised they hold the device-output results."""
    import torch
    N, L = 32, 100.0
    edges = fields.linear_edges(N, L, 6)
    f32 = _field("lognormal", N, 51).astype(np.float32)
    with fbs.Plan(N, L, edges, precision="bf16x3") as plan:
        Bd, Pd = plan.bispectrum(torch.from_numpy(f32).cuda())
        torch.cuda.synchronize()
        Bh = torch.full((plan.ntrip,), float("nan"), dtype=torch.float64).pin_memory()
        Ph = torch.full((plan.nbins,), float("nan"), dtype=torch.float64).pin_memory()
        plan.bispectrum(torch.from_numpy(f32).pin_memory(), Bh, Ph)
        torch.cuda.current_stream().synchronize()
        assert np.array_equal(Bh.numpy(), Bd.cpu().numpy())
        assert np.array_equal(Ph.numpy(), Pd.cpu().numpy(), equal_nan=True)


@pytest.mark.parametrize("N,L,kind,nb,precision,quads", [
    (64, 200.0, "log", 12, "fp32", False),
    (64, 200.0, "log", 12, "bf16x3", False),
    (96, 96.0, "lin", 10, "bf16x3", False),
    (48, 60.0, "log", 8, "bf16x3", True),
    (48, 60.0, "log", 8, "fp32", True),
])
def test_levels_match_single_grid_and_oracle(monkeypatch, N, L, kind, nb, precision, quads):
    """Items summed on per-level grids (each M above the item's degree
    R_a + R_b + R_c (+ R_d)) give the same B, P, T as one grid for all, and the
    oracle's.  A negative FBS_LEVEL_COST makes these small plans split into
    levels; FBS_MIN_LEVEL_GRID=32 keeps every level at M >= 32 (below that a
    BF16x3 sum's rounding, which grows like (N/M)^(3/2), reaches the 2e-4
    gate on cancelling triplets; plans use M >= 64)."""
    import torch
    monkeypatch.setenv("FBS_LEVEL_COST", "-1e15")
    monkeypatch.setenv("FBS_MIN_LEVEL_GRID", "32")
    edges = fields.linear_edges(N, L, nb) if kind == "lin" else fields.log_edges(N, L, nb)
    f32 = _field("quadratic", N, 61).astype(np.float32)
    f = torch.from_numpy(f32).cuda()
    with fbs.Plan(N, L, edges, precision=precision, trispectrum=quads) as lv, \
            fbs.Plan(N, L, edges, precision=precision, trispectrum=quads, single_grid=True) as one:
        assert len(lv.levels) >= 2 and len(one.levels) == 1
        assert np.array_equal(lv.triplets, one.triplets) and np.array_equal(lv.N_tri, one.N_tri)
        assert sum(l["ntrip"] for l in lv.levels) == lv.ntrip
        if quads:
            assert np.array_equal(lv.quads, one.quads) and np.array_equal(lv.N_quad, one.N_quad)
            assert sum(l["nquad"] for l in lv.levels) == lv.nquad
            Tl, Bl, Pl = lv.trispectrum(f)
            To, Bo, Po = one.trispectrum(f)
        else:
            Bl, Pl = lv.bispectrum(f)
            Bo, Po = one.bispectrum(f)
        lv.check()
        one.check()
        Bl, Pl, Bo, Po = (x.cpu().numpy() for x in (Bl, Pl, Bo, Po))
        ok = np.isfinite(Po)
        assert np.array_equal(np.isnan(Pl), np.isnan(Po))
        assert np.all(rel_err(Pl[ok], Po[ok]) < 2e-5)
        gmax, amax, ng = check_bispectrum(lv, Bl, Pl, f32, L, edges, precision)
        if quads:
            tol = TOL[precision] if precision in TOL else 1e-3
            m, n = check_trispectrum(lv, Tl.cpu().numpy(), f32, L, edges, tol)
            print("levels %s T: %d gated, max rel %.2e" % ([l["M"] for l in lv.levels], n, m))
    print("levels %s (N=%d %s %s): %d gated, max rel %.2e" % ([l["M"] for l in lv.levels], N, kind,
                                                              precision, ng, gmax))


def test_plan_from_exported_counts_equals_fresh_plan():
    """fbs_plan_create_from_counts skips the plan-time count pass with the
    closed items and exact counts of an equal plan: the same tables, levels
    and results bit for bit; a blob for other edges is refused."""
    import torch
    N, L = 48, 60.0
    edges = fields.log_edges(N, L, 8)
    f = torch.from_numpy(_field("quadratic", N, 91).astype(np.float32)).cuda()
    with fbs.Plan(N, L, edges, precision="bf16x3", trispectrum=True) as a:
        blob = a.export_counts()
        Ta, Ba, Pa = (x.cpu().numpy() for x in a.trispectrum(f))
        with fbs.Plan(N, L, edges, precision="bf16x3", trispectrum=True, counts=blob) as b:
            assert np.array_equal(a.triplets, b.triplets) and np.array_equal(a.N_tri, b.N_tri)
            assert np.array_equal(a.quads, b.quads) and np.array_equal(a.N_quad, b.N_quad)
            assert a.levels == b.levels and np.array_equal(a.N_conn, b.N_conn)
            Tb, Bb, Pb = (x.cpu().numpy() for x in b.trispectrum(f))
            assert np.array_equal(Ta, Tb) and np.array_equal(Ba, Bb)
            assert np.array_equal(Pa, Pb, equal_nan=True)
    with pytest.raises(fbs.FbsError) as e:
        fbs.Plan(N, L, fields.log_edges(N, L, 9), precision="bf16x3", trispectrum=True, counts=blob)
    assert e.value.status == -1
    with pytest.raises(fbs.FbsError):
        fbs.Plan(N, L, edges, precision="bf16x3", counts=blob)  # flags differ (no trispectrum)
