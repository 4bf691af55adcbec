"""Full-size parity in the benchmark's launch configuration.

At 256^3 and 512^3 the all-pairs oracle is out of reach, so:
* the closed-triplet set is compared with the oracle's witness search;
* exact counts and B are compared on sampled triplets whose shells are small
  enough for the direct sum (Eq. bi_direct) triplet by triplet, gated on the
  cancellation-free scale M of the FP64 fields of their (few) bins;
* the wide high-k shells (up to 1.8M modes, where the FP32 inverse transforms
  carry their largest error) are compared with the oracle's FP64 FFT
  estimator restricted to a few top bins, gated on the cancellation-free
  scale M of the FP64 fields (the same gate as on small grids);
* the 16-bin trispectrum plan of the benchmark (its fused triplet and
  quadruplet pass) is compared the same way on every quadruplet and triplet
  of its top five bins;
* P is compared with the direct mode average on every bin.
"""
import math

import numpy as np
import pytest

import fields
import oracle
import paper_1705_06284_gb300 as fbs
from gpu_util import TOL, gate_mask, rel_err

pytestmark = pytest.mark.gpu


def _sample(plan, shell, budget=4e7, n=40, maxbins=10, seed=0):
    """Triplets with |S_a||S_b| <= budget (direct sums triplet by triplet),
    drawn at random but only over a few distinct bins (the FP64 FFT estimator
    then needs only their fields for the cancellation-free scale)."""
    cand = [i for i, (a, b, c) in enumerate(plan.triplets) if shell[a] * shell[b] <= budget]
    rng = np.random.default_rng(seed)
    rng.shuffle(cand)
    out, bins = [], set()
    for i in cand:
        t = set(int(v) for v in plan.triplets[i])
        if len(bins | t) <= maxbins:
            out.append(i)
            bins |= t
        if len(out) == n:
            break
    return sorted(out)


def _run_fullsize(N, L, edges, field64, precision, nsample=40, maxbins=10):
    import torch
    f32 = field64.astype(np.float32)
    f64 = f32.astype(np.float64)
    with fbs.Plan(N, L, edges, precision=precision) as plan:
        B, P = plan.bispectrum(torch.from_numpy(f32).cuda())
        plan.check()
        B, P = B.cpu().numpy(), P.cpu().numpy()
        trip, ntri, shell = plan.triplets.copy(), plan.N_tri.copy(), plan.shell.copy()
        lev = np.array([plan.levels[i]["M"] for i in plan.trip_level])
        # the full closed-triplet set equals the oracle's
        closed = oracle.closed_triplets(N, L, edges)
        assert np.array_equal(trip, closed)
        Pref, S = oracle.power_spectrum(f64, L, edges)
        assert np.array_equal(shell, S)
        ok = S > 0
        assert np.all(rel_err(P[ok], Pref[ok]) < 1e-4)
        idx = _sample(plan, shell, n=nsample, maxbins=maxbins)
        assert len(idx) >= 10
        Bref, num, numi, cnt = oracle.direct_triplets(f64, L, edges, trip[idx])
        assert np.array_equal(cnt, ntri[idx])
        # the cancellation-free scale of each sampled triplet from the FP64 fields
        M = oracle.fft_estimator(f64, L, edges, triplets=trip[idx])["M"]
        g = gate_mask(Bref, M, ntri[idx])
        r = rel_err(B[idx], Bref)
        for m in sorted(set(lev[idx].tolist())):
            sel = g & (lev[idx] == m)
            if sel.any():
                print("   level M=%d: %d gated, max rel %.2e" % (m, int(sel.sum()), float(r[sel].max())))
        assert g.sum() >= 5
        assert np.all(r[g] < TOL[precision]), (float(r[g].max()))
        return float(r[g].max()), int(g.sum())


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_bubbles256_lin32(precision):
    N, L = 256, 256.0
    edges = fields.linear_edges(N, L, 32)
    f = fields.bubbles(N, 6.0, 0.5, seed=1)
    m, n = _run_fullsize(N, L, edges, f, precision)
    print("256^3 bubbles %s: %d sampled gated, max rel %.2e" % (precision, n, m))


def test_quadratic512_log64_bf16x3():
    N, L = 512, 1000.0
    kf = 2 * math.pi / L
    edges = np.geomspace(kf, 0.25 * N * kf, 65)
    f = fields.quadratic_local(N, 0.3, -1.5, 0.1, seed=2)
    m, n = _run_fullsize(N, L, edges, f, "bf16x3", nsample=30)
    print("512^3 quadratic-local bf16x3: %d sampled gated, max rel %.2e" % (n, m))


def _bench_512():
    N, L = 512, 1000.0
    kf = 2 * math.pi / L
    f32 = fields.quadratic_local(N, 0.3, -1.5, 0.1, seed=2).astype(np.float32)
    return N, L, kf, f32


def test_quadratic512_log64_top_bins_bf16x3():
    """Every closed triplet of five of the top 16 log bins (shells of 0.3M to
    1.8M modes) against the FP64 FFT estimator (Eqs. delta_nr, Jeong_BI)."""
    import torch
    N, L, kf, f32 = _bench_512()
    edges = np.geomspace(kf, 0.25 * N * kf, 65)
    top = {50, 54, 58, 61, 63}
    with fbs.Plan(N, L, edges, precision="bf16x3") as plan:
        B, P = plan.bispectrum(torch.from_numpy(f32).cuda())
        plan.check()
        B = B.cpu().numpy()
        sel = [i for i, t in enumerate(plan.triplets) if set(int(v) for v in t) <= top]
        trip, ntri = plan.triplets[sel], plan.N_tri[sel]
    assert len(sel) >= 30
    ref = oracle.fft_estimator(f32.astype(np.float64), L, edges, triplets=trip)
    assert np.array_equal(ref["N_tri"], ntri)
    g = gate_mask(ref["B"], ref["M"], ntri)
    assert g.sum() >= 5
    r = rel_err(B[sel], ref["B"])
    print("512^3 x 64 log, top bins %s: %d of %d triplets gated, max rel %.2e (all: %.2e)"
          % (sorted(top), int(g.sum()), len(sel), float(r[g].max()), float(r.max())))
    assert r[g].max() < TOL["bf16x3"]


def test_quadratic512_log16_trispectrum_top_bins_bf16x3():
    """The benchmark's 16-bin trispectrum plan (fused tensor-core pass at
    M = 512): closed quadruplets and triplets of its top five bins against
    the FP64 FFT estimator (Eq. Jeong_gen with p = 4 and p = 3).  Quadruple
    counts of these shells pass 2^63: the largest sampled ones are compared
    exactly with the oracle's integer pair-count route, the rest as FP64
    sums."""
    import torch
    N, L, kf, f32 = _bench_512()
    edges = np.geomspace(kf, 0.25 * N * kf, 17)
    top = {11, 12, 13, 14, 15}
    with fbs.Plan(N, L, edges, precision="bf16x3", trispectrum=True) as plan:
        T, B, P = plan.trispectrum(torch.from_numpy(f32).cuda())
        plan.check()
        T, B = T.cpu().numpy(), B.cpu().numpy()
        qs = [i for i, q in enumerate(plan.quads) if set(int(v) for v in q) <= top]
        ts = [i for i, t in enumerate(plan.triplets) if set(int(v) for v in t) <= top]
        # bounded host work: at most 32 quadruplets and 16 triplets, spread evenly
        qs = qs[:: max(1, -(-len(qs) // 32))]
        ts = ts[:: max(1, -(-len(ts) // 16))]
        quads, nq = plan.quads[qs], plan.N_quad[qs]
        nq_exact = [plan.N_quad_exact[i] for i in qs]
        trip, ntri = plan.triplets[ts], plan.N_tri[ts]
        assert plan.quad_counts_exact
    assert len(qs) >= 20 and len(ts) >= 10
    assert all(float(v) == c for v, c in zip(nq_exact, nq))
    big = np.argsort(nq)[-3:]
    ex = oracle.quad_counts_exact(N, L, edges, quads[big])
    print("512^3 x 16 log exact quadruple counts:", ex)
    assert max(ex) >= 2 ** 63
    assert [nq_exact[i] for i in big] == ex
    ref = oracle.fft_estimator(f32.astype(np.float64), L, edges, triplets=trip, quads=quads)
    assert np.array_equal(ref["N_tri"], ntri)
    assert np.allclose(nq, ref["qden"] / float(N) ** 3, rtol=1e-12)
    gq = (nq >= 100) & (np.abs(ref["T"]) >= 1e-3 * ref["qM"])
    rq = rel_err(T[qs], ref["T"])
    gt = gate_mask(ref["B"], ref["M"], ntri)
    rt = rel_err(B[ts], ref["B"])
    print("512^3 x 16 log T plan, top bins: %d/%d quads gated, max rel %.2e; %d/%d triplets gated, max rel %.2e"
          % (int(gq.sum()), len(qs), float(rq[gq].max()), int(gt.sum()), len(ts), float(rt[gt].max())))
    assert gq.sum() >= 10 and gt.sum() >= 5
    assert rq[gq].max() < TOL["bf16x3"]
    assert rt[gt].max() < TOL["bf16x3"]
