"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests touch the CUDA library.  Each pin is chosen so that a
plausible slip in the oracle (a dropped term, a wrong sign or index, a
transposed operand, a wrong normalisation power) fails at least one:

* DFT convention  -- naive O(N^6) sum (Eq. DeltaFFTtoDelta).
* Closure/binning -- pure-Python brute force over mode triples; hand-derived
                     lattice counts on an 8^3 grid.
* Estimator       -- direct sum == FFT estimator (the Kronecker-delta identity
                     of Sec. 2 turning Eq. gen_Nspec3 into Eq. gen_Nspec4).
* Normalisation   -- skewness sum rule (Eq. skew) pins V^2/N_pix^3; the
                     variance sum rule pins V/N_pix^2 for P; the kurtosis sum
                     rule pins V^3/N_pix^4 for T.
* Count sum rule  -- full-cover shells give sum N_tri = N_pix^2.
* Symmetry        -- ordered sums are invariant under bin permutations.
* Closed forms    -- three/four plane waves with a closed triangle.
* Statistics      -- Gaussian null; quadratic-local tree level 2f[P1P2+cyc].
"""
import itertools
import math

import numpy as np
import pytest

import fields
import oracle


def _full_cover_edges(N, L):
    """Edges from 0 to beyond the corner of the grid: every mode in a bin."""
    kf = 2 * math.pi / L
    top = 3 * (N // 2) ** 2 + 1
    sq = [0.0, 2.5, 6.5, 12.5, 24.5, float(top) + 0.5]
    return [kf * math.sqrt(s) for s in sq]


# ---------------------------------------------------------------- DFT pin
@pytest.mark.parametrize("N", [4, 6, 8])
def test_spectrum_matches_naive_dft(N):
    rng = np.random.default_rng(N)
    f = rng.standard_normal((N, N, N))
    D = oracle.spectrum(f)
    n = np.arange(N)
    ph = np.exp(-2j * np.pi * np.outer(n, n) / N)  # [m, n]
    naive = np.zeros((N, N, N), dtype=complex)
    for mx in range(N):
        for my in range(N):
            for mz in range(N):
                naive[mx, my, mz] = np.sum(f * ph[mx][:, None, None] * ph[my][None, :, None]
                                           * ph[mz][None, None, :])
    assert np.max(np.abs(D - naive)) <= 1e-12 * np.max(np.abs(naive))


# ---------------------------------------------------------------- thresholds
def test_thresholds_rule():
    L = 2 * math.pi  # k_f = 1
    # whole multiples of k_f land exactly; in-between values round up
    thr = oracle.thresholds([1.0, 2.0, 2.5, 3.0 + 1e-13, 8.0], L)
    assert list(thr) == [1, 4, 7, 9, 64]
    L2 = 100.0
    kf = 2 * math.pi / L2
    e = np.linspace(kf, 8 * kf, 7)
    thr2 = oracle.thresholds(e, L2)
    # 1, (13/6)^2=4.69, (10/3)^2=11.1, 4.5^2=20.25, (17/3)^2=32.1, (41/6)^2=46.7, 64
    assert list(thr2) == [1, 5, 12, 21, 33, 47, 64]


# ---------------------------------------------------------------- brute force
def _brute_counts(N, thr, D):
    """Pure-Python enumeration of ordered closed triples over binned modes."""
    nb = len(thr) - 1
    f = np.fft.fftfreq(N, d=1.0 / N).astype(int)
    modes = []
    for ix in range(N):
        for iy in range(N):
            for iz in range(N):
                m2 = f[ix] ** 2 + f[iy] ** 2 + f[iz] ** 2
                for b in range(nb):
                    if thr[b] <= m2 < thr[b + 1]:
                        modes.append((ix, iy, iz, b))
    cnt = np.zeros((nb,) * 3, dtype=np.int64)
    num = np.zeros((nb,) * 3)
    arr = np.array(modes)
    key = {(m[0], m[1], m[2]): m[3] for m in modes}
    for (ax, ay, az, ab) in modes:
        for (bx, by, bz, bb) in modes:
            c = ((-ax - bx) % N, (-ay - by) % N, (-az - bz) % N)
            if c in key:
                cnt[ab, bb, key[c]] += 1
                num[ab, bb, key[c]] += (D[ax, ay, az] * D[bx, by, bz] * D[c]).real
    return cnt, num, len(arr)


def test_direct_sum_matches_brute_force():
    N, L = 8, 2 * math.pi
    f = fields.lognormal(N, 0.6, -1.0, seed=3)
    edges = [1.0, 1.5, 2.2, 2.9]
    thr = oracle.thresholds(edges, L)
    num, numi, cnt, done = oracle.direct_sums(f, thr)
    bc, bn, nm = _brute_counts(N, thr, oracle.spectrum(f))
    assert done == nm
    assert np.array_equal(cnt, bc)
    assert np.allclose(num, bn, rtol=1e-12, atol=1e-9 * np.max(np.abs(bn)))


# Hand-derived ordered triangle counts on an 8^3 grid with k_f = 1 and the
# single-|m|^2 shells A = {|m|^2=1} (6 modes), B = {2} (12), C = {3} (8),
# D = {4} (6).  With m3 = -(m1+m2): |m3|^2 = |m1|^2 + |m2|^2 + 2 m1.m2, so
# each count is (#m1) x (#m2 with the required dot product).
#   AAA: 1+1+2d=1 -> d=-1/2 impossible                       -> 0
#   AAB: d=0, m2 one of 4 axes orthogonal to m1              -> 6*4  = 24
#   AAD: d=1, m2 = m1                                         -> 6*1  = 6
#   ABC: d=0, m2 of type (0,+-1,+-1) orthogonal to m1        -> 6*4  = 24
#   BBB: 2+2+2d=2 -> d=-1, e.g. (1,1,0): (-1,0,+-1),(0,-1,+-1)-> 12*4 = 48
#   BBD: d=0, (1,1,0) -> (1,-1,0),(-1,1,0)                    -> 12*2 = 24
#   CCD: 3+3+2d=4 -> d=-1, two minus signs of three          -> 8*3  = 24
#   ACD: d=0 impossible (m2 has no zero component)            -> 0
#   BCC: 2+3+2d=3 -> d=-1 impossible for s1+s2 in {-2,0,2}   -> 0
#   DDD: 4+4+2d=4 -> d=-2 impossible (d in {0,+-4})           -> 0
HAND_COUNTS = {(0, 0, 0): 0, (0, 0, 1): 24, (0, 0, 3): 6, (0, 1, 2): 24, (1, 1, 1): 48,
               (1, 1, 3): 24, (2, 2, 3): 24, (0, 2, 3): 0, (1, 2, 2): 0, (3, 3, 3): 0}


def test_hand_derived_lattice_counts():
    N, L = 8, 2 * math.pi
    edges = [1.0, 1.2, 1.5, 1.8, 2.1]  # -> |m|^2 in {1},{2},{3},{4}
    thr = oracle.thresholds(edges, L)
    assert list(thr) == [1, 2, 3, 4, 5]
    assert list(oracle.shell_sizes(N, thr)) == [6, 12, 8, 6]
    f = fields.lognormal(N, 0.5, -2.0, seed=0)
    _, _, cnt, _ = oracle.direct_sums(f, thr)
    for (a, b, c), v in HAND_COUNTS.items():
        for p in set(itertools.permutations((a, b, c))):
            assert cnt[p] == v, (p, cnt[p], v)
    fe = oracle.fft_estimator(f, L, edges, triplets=list(HAND_COUNTS))
    assert [int(x) for x in fe["N_tri"]] == list(HAND_COUNTS.values())


# ---------------------------------------------------------------- identity
@pytest.mark.parametrize("N,nb,seed,kind", [(8, 3, 1, "lin"), (12, 4, 2, "lin"), (16, 5, 3, "log"),
                                            (12, 3, 4, "full")])
def test_direct_equals_fft_estimator(N, nb, seed, kind):
    L = 50.0
    f = fields.lognormal(N, 0.8, -1.5, seed=seed)
    if kind == "lin":
        edges = fields.linear_edges(N, L, nb)
    elif kind == "log":
        edges = fields.log_edges(N, L, nb)
    else:
        edges = _full_cover_edges(N, L)
    d = oracle.direct_bispectrum(f, L, edges)
    assert len(d["triplets"]) > 0
    g = oracle.fft_estimator(f, L, edges, triplets=d["triplets"])
    assert np.array_equal(d["N_tri"], g["N_tri"])
    scale = np.max(np.abs(d["num"]))
    assert np.max(np.abs(d["num"] - g["num"] / N ** 3)) <= 1e-12 * scale
    ok = np.isfinite(d["P"])
    assert np.allclose(d["P"][ok], g["P"][ok], rtol=1e-12)


def test_imaginary_part_cancels():
    N, L = 16, 80.0
    f = fields.bubbles(N, 2.5, 0.4, seed=5)
    d = oracle.direct_bispectrum(f, L, fields.linear_edges(N, L, 4))
    assert np.max(np.abs(d["num_im"])) <= 1e-12 * np.max(np.abs(d["num"]))


def test_permutation_symmetry():
    N, L = 12, 30.0
    f = fields.lognormal(N, 0.7, -2.0, seed=9)
    thr = oracle.thresholds(fields.linear_edges(N, L, 4), L)
    num, _, cnt, _ = oracle.direct_sums(f, thr)
    for p in itertools.permutations(range(3)):
        assert np.array_equal(cnt, np.transpose(cnt, p))
        assert np.allclose(num, np.transpose(num, p), rtol=1e-12, atol=1e-12 * np.max(np.abs(num)))


# ---------------------------------------------------------------- sum rules
def test_count_sum_rule_full_cover():
    N, L = 8, 10.0
    thr = oracle.thresholds(_full_cover_edges(N, L), L)
    f = fields.lognormal(N, 0.5, -2.0, seed=0)
    _, _, cnt, _ = oracle.direct_sums(f, thr)
    assert int(cnt.sum()) == (N ** 3) ** 2


def test_skewness_sum_rule_pins_bispectrum_normalisation():
    # Eq. skew: gamma = <delta^3> = int d3k1/(2pi)^3 int d3k2/(2pi)^3 B.  On the
    # lattice int d3k/(2pi)^3 -> (1/V) sum_m, so mean(delta^3) =
    # (1/V^2) sum over ordered (a,b,c) of N_tri(abc) * B(abc).
    N, L = 8, 37.0
    f = fields.lognormal(N, 0.9, -1.0, seed=4)
    d = oracle.direct_bispectrum(f, L, _full_cover_edges(N, L))
    num, cnt = d["ordered_num"], d["ordered_cnt"]
    V, npix = L ** 3, float(N ** 3)
    Bord = np.where(cnt > 0, (V * V / npix ** 3) * num / np.maximum(cnt, 1), 0.0)
    lhs = float(np.sum(cnt * Bord)) / V ** 2
    assert abs(lhs - float(np.mean(f ** 3))) <= 1e-11 * float(np.mean(np.abs(f) ** 3))


def test_variance_sum_rule_pins_power_normalisation():
    # sigma^2 = int d3k/(2pi)^3 P(k)  ->  mean(delta^2) = (1/V) sum_b |S_b| P_b
    # for shells covering every mode (the mean of delta enters through m = 0).
    N, L = 10, 21.0
    f = fields.lognormal(N, 0.7, -1.5, seed=8)
    edges = _full_cover_edges(N, L)
    P, S = oracle.power_spectrum(f, L, edges)
    ok = S > 0
    lhs = float(np.sum(S[ok] * P[ok])) / L ** 3
    assert abs(lhs - float(np.mean(f ** 2))) <= 1e-12 * float(np.mean(f ** 2))
    g = oracle.fft_estimator(f, L, edges, triplets=[], bins_needed=np.nonzero(ok)[0])
    assert np.allclose(g["P"][ok], P[ok], rtol=1e-12)


def test_kurtosis_sum_rule_pins_trispectrum_normalisation():
    # <delta^4> = (1/V^3) sum over ordered (a,b,c,d) N_quad T   (raw p = 4 estimator)
    N, L = 6, 13.0
    f = fields.lognormal(N, 0.8, -1.0, seed=6)
    kf = 2 * math.pi / L
    edges = [0.0, kf * 1.2, kf * 1.8, kf * 5.5]  # covers |m|^2 <= 27
    t = oracle.direct_trispectrum(f, L, edges)
    num, cnt = t["ordered_num"], t["ordered_cnt"]
    assert int(cnt.sum()) == (N ** 3) ** 3
    V, npix = L ** 3, float(N ** 3)
    T = np.where(cnt > 0, (V ** 3 / npix ** 4) * num / np.maximum(cnt, 1), 0.0)
    lhs = float(np.sum(cnt * T)) / V ** 3
    assert abs(lhs - float(np.mean(f ** 4))) <= 1e-11 * float(np.mean(f ** 4))


# ---------------------------------------------------------------- closed forms
def test_three_plane_waves_closed_form():
    # delta = sum_j A_j cos(2 pi m_j.n/N + phi_j), m1+m2+m3 = 0, |m_j| in
    # distinct single-|m|^2 shells.  D(+-m_j) = (N^3 A_j/2) e^{+-i phi_j}, so
    # the only closed ordered triples in the sorted bin triple (a,b,c) are
    # (m1,m2,m3) and (-m1,-m2,-m3):  num = 2 (N^3/2)^3 A1A2A3 cos(phi1+phi2+phi3).
    N, L = 16, 2 * math.pi
    m1, m2 = (1, 0, 0), (0, 2, 0)
    m3 = (-1, -2, 0)
    A = (0.7, -0.4, 1.3)
    phi = (0.3, -1.1, 2.0)
    f = fields.plane_waves(N, [(m1, A[0], phi[0]), (m2, A[1], phi[1]), (m3, A[2], phi[2])])
    edges = [0.9, 1.1, 1.9, 2.1, 2.2, 2.3]  # |m|^2: {1}, {2,3}, {4}, {}, {5}
    thr = oracle.thresholds(edges, L)
    assert list(thr) == [1, 2, 4, 5, 5, 6]
    d = oracle.direct_bispectrum(f, L, edges)
    # the triangle sits in bins (0, 2, 4); its count is the full lattice count
    idx = [i for i, t in enumerate(d["triplets"]) if tuple(t) == (0, 2, 4)]
    assert len(idx) == 1
    i = idx[0]
    npix = N ** 3
    expect = 2 * (npix / 2) ** 3 * A[0] * A[1] * A[2] * math.cos(sum(phi))
    assert abs(d["num"][i] - expect) <= 1e-10 * abs(expect)
    V = L ** 3
    assert abs(d["B"][i] - V * V / npix ** 3 * expect / d["N_tri"][i]) <= 1e-12 * abs(d["B"][i])
    # every other triplet sees no closed wave triangle
    others = np.delete(d["num"], i)
    assert np.all(np.abs(others) <= 1e-9 * abs(expect))


def test_four_plane_waves_closed_form_trispectrum():
    N, L = 8, 2 * math.pi
    ms = [(1, 0, 0), (0, 1, 0), (0, 0, 2), (-1, -1, -2)]
    A = (0.5, 0.8, -0.6, 0.9)
    phi = (0.2, 0.9, -0.4, 1.7)
    f = fields.plane_waves(N, list(zip(ms, A, phi)))
    edges = [0.9, 1.1, 1.9, 2.1, 2.4, 2.5]  # {1}, {2,3}, {4}, {5}, {6}
    thr = oracle.thresholds(edges, L)
    assert list(thr) == [1, 2, 4, 5, 6, 7]
    t = oracle.direct_trispectrum(f, L, edges)
    # (m1,m2,m3,m4) lies in bins (0,0,2,4): |m4|^2 = 6.  Ordered quadruples of
    # the wave set closing in that sorted bin order: m1<->m2 swap and the global
    # sign flip -> 4 terms, each (N^3/2)^4 A1A2A3A4 cos(sum phi).  Quadruples
    # like (m1, -m1, m2, -m2) are in other bin patterns.
    i = [k for k, q in enumerate(t["quads"]) if tuple(q) == (0, 0, 2, 4)][0]
    npix = N ** 3
    expect = 4 * (npix / 2) ** 4 * np.prod(A) * math.cos(sum(phi))
    assert abs(t["num"][i] - expect) <= 1e-10 * abs(expect)
    # the FFT estimator (Eq. Jeong_gen with p = 4) reaches the same number
    g = oracle.fft_estimator(f, L, edges, triplets=[], quads=[(0, 0, 2, 4)])
    assert abs(g["qnum"][0] / npix - expect) <= 1e-10 * abs(expect)
    assert g["N_quad"][0] == t["N_quad"][i]


def test_trispectrum_direct_equals_fft_estimator():
    N, L = 8, 40.0
    f = fields.lognormal(N, 0.8, -1.5, seed=12)
    edges = fields.linear_edges(N, L, 3)
    t = oracle.direct_trispectrum(f, L, edges)
    g = oracle.fft_estimator(f, L, edges, triplets=[], quads=t["quads"])
    assert np.array_equal(g["N_quad"], t["N_quad"])
    assert np.allclose(g["qnum"] / N ** 3, t["num"], rtol=1e-10,
                       atol=1e-12 * np.max(np.abs(t["num"])))


# ---------------------------------------------------------------- statistics
def test_gaussian_null():
    # For a Gaussian field the bispectrum has zero mean and, to leading order,
    # Var(B) = s V P_a P_b P_c / N_tri (s = 1, 2, 6 for scalene, isosceles,
    # equilateral).  Pool z-scores over triplets and realisations.
    N, L, slope = 24, 100.0, -1.0
    edges = fields.linear_edges(N, L, 5)
    zs = []
    for seed in range(3):
        g = fields.gaussian(N, slope, 1.0, seed=100 + seed)
        d = oracle.direct_bispectrum(g, L, edges)
        P = d["P"]
        for (a, b, c), B, n in zip(d["triplets"], d["B"], d["N_tri"]):
            if n < 200:
                continue
            s = 6 if a == b == c else (2 if (a == b or b == c) else 1)
            var = s * L ** 3 * P[a] * P[b] * P[c] / n
            zs.append(B / math.sqrt(var))
    zs = np.array(zs)
    assert len(zs) > 20
    assert abs(zs.mean()) < 4.0 / math.sqrt(len(zs))
    assert 0.5 < zs.std() < 2.0


def test_quadratic_local_tree_level():
    # delta = g + f (g^2 - <g^2>) has, at tree level, B = 2f[P1P2 + P2P3 + P3P1]
    # with P the spectrum of g.  Average the theory over the exact closed
    # triangles of each bin triple (as the paper does for its theory points),
    # fit B_measured = r B_tree with Gaussian weights, and require r ~ 1.
    N, L, slope, sg, fnl = 32, 200.0, -1.5, 0.1, 1.0
    edges = fields.linear_edges(N, L, 5)
    thr = oracle.thresholds(edges, L)
    nb = len(thr) - 1
    V, npix = L ** 3, float(N ** 3)
    bins = oracle.bin_index(N, thr)
    m = np.sqrt(oracle.mode_squares(N).astype(float))
    num_r, den_r = 0.0, 0.0
    for seed in range(3):
        A = fields.gaussian_spectrum_amplitude(N, slope, sg, seed=200 + seed)
        Pm = np.where(m > 0, (V / npix ** 2) * A * np.where(m > 0, m, 1.0) ** slope, 0.0)
        # W_b(x) = unnormalised inverse DFT of P(m) on shell b; Sigma over
        # closed triples of P(m1)P(m2) = (1/N_pix) sum_x W_a W_b N_c.
        W = [np.fft.ifftn(np.where(bins == b, Pm, 0.0)).real * npix for b in range(nb)]
        Cf = [np.fft.ifftn((bins == b).astype(float)).real * npix for b in range(nb)]
        delta = fields.quadratic_local(N, fnl, slope, sg, seed=200 + seed)
        d = oracle.direct_bispectrum(delta, L, edges)
        for (a, b, c), B, n in zip(d["triplets"], d["B"], d["N_tri"]):
            if n < 500:
                continue
            pp = (np.sum(W[a] * W[b] * Cf[c]) + np.sum(Cf[a] * W[b] * W[c])
                  + np.sum(W[a] * Cf[b] * W[c])) / npix
            Bt = 2 * fnl * pp / n
            s = 6 if a == b == c else (2 if (a == b or b == c) else 1)
            P = d["P"]
            var = s * V * P[a] * P[b] * P[c] / n
            num_r += B * Bt / var
            den_r += Bt * Bt / var
    r = num_r / den_r
    sig = 1.0 / math.sqrt(den_r)
    assert sig < 0.2
    assert abs(r - 1.0) < 4 * sig + 0.05, (r, sig)


# ---------------------------------------------------------------- stored values
def _read_golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    meta, rows = {}, []
    for line in open(path):
        if line.startswith("# ") and line.split()[1] in ("edges", "P", "shell"):
            k = line.split()[1]
            meta[k] = [float(v) for v in line.split()[2:]]
        elif not line.startswith("#"):
            rows.append(line.split())
    return meta, rows


def test_golden_lognormal32_reproduces():
    meta, rows = _read_golden("lognormal32_lin6.txt")
    N, L = 32, 100.0
    f = fields.lognormal(N, 0.5, -2.0, seed=0).astype(np.float32).astype(np.float64)
    d = oracle.direct_bispectrum(f, L, meta["edges"])
    assert len(rows) == len(d["triplets"]) == 49
    for r, t, n, B in zip(rows, d["triplets"], d["N_tri"], d["B"]):
        assert [int(v) for v in r[:4]] == [int(t[0]), int(t[1]), int(t[2]), int(n)]
        assert abs(float(r[4]) - B) <= 1e-12 * abs(B)
    assert [int(v) for v in meta["shell"]] == list(d["shell"])


# ---------------------------------------------------------------- evaluation grid
def _embed_shell_field(D, bins, b, M):
    """Shell field of bin b evaluated on an M^3 grid: the same modes (all with
    |m_j| < M/2) placed at m mod M, unnormalised inverse DFT of length M."""
    N = D.shape[0]
    f = np.fft.fftfreq(N, 1.0 / N).astype(int)
    idx = np.nonzero(bins == b)
    E = np.zeros((M, M, M), dtype=np.complex128)
    E[f[idx[0]] % M, f[idx[1]] % M, f[idx[2]] % M] = D[idx]
    return (np.fft.ifftn(E) * M ** 3).real


@pytest.mark.parametrize("order,M", [(3, 20), (3, 24), (4, 28)])
def test_products_sum_on_reduced_grid(order, M):
    """A product of `order` shell fields holding only modes with |m_j| <= R is a
    trigonometric polynomial of degree <= order*R per axis, so its sum over the
    N^3 grid is (N/M)^3 times its sum over any M^3 grid with M > order*R (the
    device path evaluates on such an M).  Checked in FP64 on every triplet /
    quadruplet of a small plan; M = order*R exactly (aliased) must differ."""
    N, L = 32, 100.0
    kf = 2 * math.pi / L
    edges = kf * np.array([0.5, 2.5, 4.5, 6.5])  # R = 6
    R = 6
    f = fields.quadratic_local(N, 0.5, -1.5, 0.3, seed=5)
    D = oracle.spectrum(f)
    bins = oracle.bin_index(N, oracle.thresholds(edges, L))
    nb = 3
    full = [oracle.shell_field(D, bins, b) for b in range(nb)]
    red = [_embed_shell_field(D, bins, b, M) for b in range(nb)]
    alias = [_embed_shell_field(D, bins, b, order * R) for b in range(nb)]
    scale = (N / M) ** 3
    worst_alias = 0.0
    for combo in itertools.combinations_with_replacement(range(nb), order):
        pf = np.prod([full[b] for b in combo], axis=0)
        pr = np.prod([red[b] for b in combo], axis=0)
        pa = np.prod([alias[b] for b in combo], axis=0)
        ref = pf.sum()
        mag = np.abs(pf).sum()
        assert abs(scale * pr.sum() - ref) <= 1e-12 * mag, combo
        worst_alias = max(worst_alias, abs((N / (order * R)) ** 3 * pa.sum() - ref) / mag)
    assert worst_alias > 1e-6  # one grid point too few aliases some product


# ---------------------------------------------------------------- triplet subsets
# The full-size GPU tests take their closed-triplet set from
# oracle.closed_triplets (a pruned witness search) and their reference sums
# from oracle.direct_triplets (per-triplet loops over S_a x S_b).  Both are
# pinned here to the all-pairs definition (direct_sums) on grids small enough
# for it: linear bins, log bins with empty shells, and plans whose top edge
# passes N k_f/4 so that closure modulo N differs from exact closure.
def _subset_case(kind, N, L, nb):
    kf = 2 * math.pi / L
    if kind == "lin":
        return fields.linear_edges(N, L, nb)
    if kind == "log":
        return fields.log_edges(N, L, nb)
    if kind == "aliased":  # up to 0.45 N k_f: wrapped sums close modulo N
        return np.linspace(kf, 0.45 * N * kf, nb + 1)
    return _full_cover_edges(N, L)


SUBSET_CASES = [("lin", 12, 50.0, 5, 1), ("log", 16, 60.0, 12, 2), ("log", 20, 30.0, 9, 3),
                ("aliased", 10, 20.0, 4, 4), ("aliased", 12, 7.0, 6, 5), ("full", 8, 10.0, None, 6)]


@pytest.mark.parametrize("kind,N,L,nb,seed", SUBSET_CASES)
def test_closed_triplets_equals_all_pairs_counts(kind, N, L, nb, seed):
    edges = _subset_case(kind, N, L, nb)
    thr = oracle.thresholds(edges, L)
    S = oracle.shell_sizes(N, thr)
    if kind == "log":
        assert np.any(S == 0)  # the pin must cover empty shells
    f = fields.lognormal(N, 0.6, -1.5, seed=seed)
    _, _, cnt, _ = oracle.direct_sums(f, thr)
    k = len(thr) - 1
    expect = [(a, b, c) for a in range(k) for b in range(a, k) for c in range(b, k) if cnt[a, b, c] > 0]
    got = [tuple(int(v) for v in t) for t in oracle.closed_triplets(N, L, edges)]
    assert len(expect) > 0
    assert got == expect


@pytest.mark.parametrize("kind,N,L,nb,seed", SUBSET_CASES)
def test_direct_triplets_equals_all_pairs_sums(kind, N, L, nb, seed):
    edges = _subset_case(kind, N, L, nb)
    thr = oracle.thresholds(edges, L)
    f = fields.bubbles(N, 2.0, 0.4, seed=seed) if seed % 2 else fields.lognormal(N, 0.8, -1.0, seed=seed)
    num, numi, cnt, _ = oracle.direct_sums(f, thr)
    k = len(thr) - 1
    S = oracle.shell_sizes(N, thr)
    # every sorted triple of non-empty bins (closed or not), plus every
    # ordering of a few of them (the ordered sum is over m1 in S_a, m2 in S_b)
    trip = [(a, b, c) for a in range(k) for b in range(a, k) for c in range(b, k) if S[a] and S[b] and S[c]]
    extra = [p for t in trip[:: max(1, len(trip) // 6)] for p in set(itertools.permutations(t))]
    allt = np.array(trip + extra, dtype=np.int32)
    B, n, ni, c = oracle.direct_triplets(f, L, edges, allt)
    ref_n = np.array([num[a, b, cc] for a, b, cc in allt])
    ref_i = np.array([numi[a, b, cc] for a, b, cc in allt])
    ref_c = np.array([cnt[a, b, cc] for a, b, cc in allt])
    assert np.array_equal(c, ref_c)
    assert ref_c.sum() > 0
    scale = np.max(np.abs(ref_n))
    assert np.max(np.abs(n - ref_n)) <= 1e-12 * scale
    assert np.max(np.abs(ni - ref_i)) <= 1e-12 * scale
    V, npix = L ** 3, float(N ** 3)
    closed = ref_c > 0
    assert np.allclose(B[closed], (V * V / npix ** 3) * ref_n[closed] / ref_c[closed], rtol=1e-12,
                       atol=1e-12 * np.max(np.abs(B)))


def test_count_modes_equals_shell_sizes():
    for N, L, nb in [(12, 50.0, 5), (16, 30.0, 9)]:
        thr = oracle.thresholds(fields.log_edges(N, L, nb), L)
        assert oracle.count_modes(N, thr) == int(oracle.shell_sizes(N, thr).sum())


# ---------------------------------------------------------------- connected trispectrum
def _brute_quads(N, thr, D, connected):
    """Pure-Python ordered quadruple sums over binned modes, pairings left out
    when `connected` (m_i + m_j = 0 mod N for any two of the four modes)."""
    nb = len(thr) - 1
    f = np.fft.fftfreq(N, d=1.0 / N).astype(int)
    modes = []
    for ix in range(N):
        for iy in range(N):
            for iz in range(N):
                m2 = f[ix] ** 2 + f[iy] ** 2 + f[iz] ** 2
                for b in range(nb):
                    if thr[b] <= m2 < thr[b + 1]:
                        modes.append(((ix, iy, iz), b))
    key = dict(modes)
    num = np.zeros((nb,) * 4)
    cnt = np.zeros((nb,) * 4, dtype=np.int64)
    neg = lambda m: ((-m[0]) % N, (-m[1]) % N, (-m[2]) % N)
    for m1, b1 in modes:
        for m2, b2 in modes:
            for m3, b3 in modes:
                m4 = ((-m1[0] - m2[0] - m3[0]) % N, (-m1[1] - m2[1] - m3[1]) % N, (-m1[2] - m2[2] - m3[2]) % N)
                if m4 not in key:
                    continue
                ms = (m1, m2, m3, m4)
                if connected and any(ms[j] == neg(ms[i]) for i in range(4) for j in range(i + 1, 4)):
                    continue
                k = (b1, b2, b3, key[m4])
                cnt[k] += 1
                num[k] += (D[m1] * D[m2] * D[m3] * D[m4]).real
    return num, cnt


def test_connected_trispectrum_matches_brute_force():
    N, L = 6, 2 * math.pi
    f = fields.lognormal(N, 0.7, -1.0, seed=21)
    edges = [0.9, 1.2, 1.5, 1.8]  # |m|^2 in {1}, {2}, {3}: includes a = b = c = d and a = b < c = d
    thr = oracle.thresholds(edges, L)
    D = oracle.spectrum(f)
    bn, bc = _brute_quads(N, thr, D, connected=True)
    t = oracle.direct_trispectrum(f, L, edges, connected=True)
    assert np.array_equal(t["ordered_cnt"], bc)
    assert np.allclose(t["ordered_num"], bn, rtol=1e-12, atol=1e-12 * np.max(np.abs(bn)))
    raw = oracle.direct_trispectrum(f, L, edges)
    assert np.any(raw["ordered_cnt"] > t["ordered_cnt"])  # pairings were present and removed


@pytest.mark.parametrize("N,L,kind,seed", [(8, 40.0, "lin", 22), (6, 13.0, "full", 23), (8, 2 * math.pi, "fine", 24)])
def test_connected_direct_equals_fft_minus_pairings(N, L, kind, seed):
    """The two routes to the connected trispectrum: the direct sum with the
    paired quadruples left out, and the FFT estimator (Eq. Jeong_gen, p = 4)
    minus the pairing terms from S2, S4 and the self-conjugate modes."""
    f = fields.lognormal(N, 0.8, -1.5, seed=seed)
    if kind == "lin":
        edges = fields.linear_edges(N, L, 3)
    elif kind == "full":
        kf = 2 * math.pi / L
        edges = [0.0, kf * 1.2, kf * 1.8, kf * 5.5]  # every mode, DC and Nyquist corners included
    else:
        edges = [0.9, 1.1, 1.5, 1.8, 2.1]  # single |m|^2 shells {1}, {2}, {3}, {4}
    t = oracle.direct_trispectrum(f, L, edges, connected=True)
    allq = oracle.direct_trispectrum(f, L, edges)["quads"]
    g = oracle.fft_estimator(f, L, edges, triplets=[], quads=allq)
    conn = np.array([tuple(q) in {tuple(x) for x in t["quads"]} for q in allq])
    assert np.allclose(g["N_conn"][~conn], 0.0)
    assert np.array_equal(np.rint(g["N_conn"][conn]).astype(np.int64), t["N_quad"])
    scale = np.max(np.abs(g["qnum"])) / N ** 3
    assert np.max(np.abs(g["qnum"][conn] / N ** 3 - g["pair_sum"][conn] - t["num"])) <= 1e-10 * scale
    assert np.allclose(g["Tc"][conn], t["T"], rtol=1e-8, atol=1e-10 * np.max(np.abs(g["T"])))


def test_connected_kurtosis_sum_rule():
    # With shells covering every mode, the unpaired ordered quadruples add up
    # to N_pix^3 sum delta^4 - 3 N_pix^2 (sum delta^2)^2 + 3 sum |D|^4 - sum_Z D^4
    # (Parseval for the paired sums), i.e. the fourth cumulant on the grid.
    N, L = 6, 13.0
    f = fields.lognormal(N, 0.9, -1.0, seed=25)
    kf = 2 * math.pi / L
    edges = [0.0, kf * 1.2, kf * 1.8, kf * 5.5]
    t = oracle.direct_trispectrum(f, L, edges, connected=True)
    D = oracle.spectrum(f)
    npix = float(N ** 3)
    a2 = np.abs(D) ** 2
    i = np.arange(N)
    sc1 = (i == 0) | (2 * i == N)
    sc = sc1[:, None, None] & sc1[None, :, None] & sc1[None, None, :]
    rhs = npix ** 3 * np.sum(f ** 4) - 3 * npix ** 2 * np.sum(f ** 2) ** 2 + 3 * np.sum(a2 ** 2) \
        - np.sum(D.real[sc] ** 4)
    lhs = np.sum(t["ordered_num"])
    assert abs(lhs - rhs) <= 1e-10 * npix ** 3 * np.sum(f ** 4)


def test_connected_trispectrum_gaussian_null():
    # For a Gaussian field every closed quadruple's expectation is a sum of
    # pairings, so the connected part has zero mean while the raw T of
    # (a, a, c, c) carries the P_a P_c part.
    N, L = 16, 50.0
    edges = fields.linear_edges(N, L, 3)
    raw, conn = [], []
    for seed in range(6):
        g = fields.gaussian(N, -1.0, 1.0, seed=300 + seed)
        qd = [(0, 0, 1, 1), (0, 0, 2, 2), (1, 1, 2, 2), (1, 1, 1, 1), (2, 2, 2, 2)]
        e = oracle.fft_estimator(g, L, edges, triplets=[], quads=qd)
        raw.append(e["T"])
        conn.append(e["Tc"])
    raw, conn = np.array(raw), np.array(conn)
    assert np.all(raw.mean(0) > 0)
    assert np.all(np.abs(conn.mean(0)) < 0.1 * raw.mean(0))


# ---------------------------------------------------------------- (k1, k2, theta) cells
def test_rebinned_bispectrum_matches_brute_force():
    # every closed ordered triple of modes, put in its cell by its bins'
    # representative k, in plain Python
    N, L = 8, 2 * math.pi
    f = fields.lognormal(N, 0.6, -1.0, seed=31)
    edges = [1.0, 1.5, 2.2, 2.9, 3.4]
    thr = oracle.thresholds(edges, L)
    k_rep = np.array([1.2, 1.8, 2.5, 3.1])
    ke = [1.0, 2.0, 3.5]
    me = [-1.0, -0.5, 0.0, 0.5, 1.0001]
    B, cc, cn = oracle.rebinned_bispectrum(f, L, edges, ke, me, k_rep=k_rep)
    D = oracle.spectrum(f)
    fr = np.fft.fftfreq(N, d=1.0 / N).astype(int)
    modes = {}
    for ix in range(N):
        for iy in range(N):
            for iz in range(N):
                m2 = fr[ix] ** 2 + fr[iy] ** 2 + fr[iz] ** 2
                for b in range(len(thr) - 1):
                    if thr[b] <= m2 < thr[b + 1]:
                        modes[(ix, iy, iz)] = b
    bn = np.zeros_like(cn)
    bc = np.zeros_like(cc)
    for m1, a in modes.items():
        for m2, b in modes.items():
            m3 = ((-m1[0] - m2[0]) % N, (-m1[1] - m2[1]) % N, (-m1[2] - m2[2]) % N)
            if m3 not in modes:
                continue
            k1, k2, k3 = k_rep[a], k_rep[b], k_rep[modes[m3]]
            mu = min(1.0, max(-1.0, (k1 * k1 + k2 * k2 - k3 * k3) / (2 * k1 * k2)))
            K1 = np.searchsorted(ke, k1, side="right") - 1
            K2 = np.searchsorted(ke, k2, side="right") - 1
            MU = np.searchsorted(me, mu, side="right") - 1
            if 0 <= K1 < 2 and 0 <= K2 < 2 and 0 <= MU < 4:
                bc[K1, K2, MU] += 1
                bn[K1, K2, MU] += (D[m1] * D[m2] * D[m3]).real
    assert np.array_equal(cc, bc)
    assert np.allclose(cn, bn, rtol=1e-12, atol=1e-12 * np.max(np.abs(bn)))
    assert cc.sum() > 0 and np.isnan(B[cc == 0]).all()


def test_rebinned_single_cell_is_the_count_weighted_mean():
    # one cell holding every configuration: the direct estimator over all
    # ordered closed triples, i.e. the N_tri-weighted mean of the fine B
    N, L = 12, 40.0
    f = fields.bubbles(N, 2.0, 0.4, seed=32)
    edges = fields.linear_edges(N, L, 4)
    B, cc, cn = oracle.rebinned_bispectrum(f, L, edges, [0.0, 10.0], [-1.0, 1.0001])
    d = oracle.direct_bispectrum(f, L, edges)
    cnt, num = d["ordered_cnt"], d["ordered_num"]
    V, npix = L ** 3, float(N ** 3)
    assert cc[0, 0, 0] == cnt.sum()
    assert abs(B[0, 0, 0] - (V * V / npix ** 3) * num.sum() / cnt.sum()) <= 1e-12 * abs(B[0, 0, 0])
    # and the weighted mean over sorted triplets with their permutation multiplicity
    w = sum(len(set(itertools.permutations(t))) * n * b for t, n, b in zip(d["triplets"], d["N_tri"], d["B"]))
    c = sum(len(set(itertools.permutations(t))) * n for t, n in zip(d["triplets"], d["N_tri"]))
    assert abs(B[0, 0, 0] - w / c) <= 1e-12 * abs(B[0, 0, 0])


# ---------------------------------------------------------------- theory over exact triangles
def _tables(N, L, funcs):
    kf = 2 * math.pi / L
    s = np.arange(3 * (N // 2) ** 2 + 1, dtype=np.float64)
    k = kf * np.sqrt(s)
    return np.stack([f(k) for f in funcs])


def test_triangle_average_of_one_is_one_and_counts_match():
    N, L = 12, 40.0
    edges = fields.linear_edges(N, L, 4)
    d = oracle.direct_bispectrum(fields.lognormal(N, 0.5, -1.0, seed=41), L, edges)
    avg, cnt = oracle.triangle_average(N, L, edges, d["triplets"], _tables(N, L, [np.ones_like]), [(0, 0, 0)], [1.0])
    assert np.array_equal(cnt, d["N_tri"])
    assert np.allclose(avg, 1.0, rtol=1e-15, atol=0)


def test_triangle_average_local_model_equals_fft_route():
    # 2f sum_closed [P1 P2 + P2 P3 + P3 P1] / N_tri by enumeration, against
    # (1/N_pix) sum_x (W_a W_b C_c + ...) with W the inverse DFT of P on the
    # shell and C the count field (the Kronecker-delta identity of Sec. 2)
    N, L, f = 16, 60.0, 0.7
    edges = fields.linear_edges(N, L, 4)
    thr = oracle.thresholds(edges, L)
    trip = oracle.closed_triplets(N, L, edges)
    Pk = lambda k: np.where(k > 0, 1.0 / np.maximum(k, 1e-30) ** 1.5, 0.0)
    avg, cnt = oracle.triangle_average(N, L, edges, trip, _tables(N, L, [Pk, np.ones_like]),
                                       [(0, 0, 1), (1, 0, 0), (0, 1, 0)], [2 * f] * 3)
    bins = oracle.bin_index(N, thr)
    kf = 2 * math.pi / L
    kk = kf * np.sqrt(oracle.mode_squares(N).astype(float))
    npix = float(N ** 3)
    W = {b: (np.fft.ifftn(np.where(bins == b, Pk(kk), 0.0)) * npix).real for b in range(len(thr) - 1)}
    C = {b: (np.fft.ifftn((bins == b).astype(float)) * npix).real for b in range(len(thr) - 1)}
    for (a, b, c), v, n in zip(trip, avg, cnt):
        ref = 2 * f * (np.sum(W[a] * W[b] * C[c]) + np.sum(C[a] * W[b] * W[c]) + np.sum(W[a] * C[b] * W[c])) / npix / n
        assert abs(v - ref) <= 1e-10 * abs(ref)


def test_tree_level_separable_form_equals_per_triangle_kernel():
    # Eq. PT_Bi evaluated with the wave vectors of every triangle, against
    # its separable form in u = k^2 (k1.k2 = (k3^2 - k1^2 - k2^2)/2 on a
    # closed triangle), both averaged over the same triangles
    N, L, kappa = 12, 30.0, 3.0 / 7.0
    edges = fields.linear_edges(N, L, 3)
    trip = oracle.closed_triplets(N, L, edges)
    Pk = lambda k: np.where(k > 0, 1.0 / (1.0 + np.maximum(k, 1e-30) ** 2), 0.0)

    def F(x, y):
        kx, ky = np.linalg.norm(x, axis=1), np.linalg.norm(y, axis=1)
        mu = np.sum(x * y, axis=1) / (kx * ky)
        return (1 + kappa) / 2 + mu / 2 * (kx / ky + ky / kx) + (1 - kappa) / 2 * mu * mu

    def model(k1, k2, k3):
        P1, P2, P3 = (Pk(np.linalg.norm(k, axis=1)) for k in (k1, k2, k3))
        return 2 * F(k1, k2) * P1 * P2 + 2 * F(k2, k3) * P2 * P3 + 2 * F(k3, k1) * P3 * P1

    ref, cnt = oracle.triangle_average_direct(N, L, edges, trip, model)
    u = lambda k: k * k
    funcs = [Pk, lambda k: np.where(k > 0, Pk(k) / np.maximum(u(k), 1e-30), 0.0), u, lambda k: Pk(k) * u(k),
             lambda k: u(k) ** 2, np.ones_like]
    one = [(0, 0, 5, (1 + kappa) / 2), (0, 1, 2, kappa / 2), (1, 0, 2, kappa / 2), (3, 1, 5, -(1 + kappa) / 4),
           (1, 3, 5, -(1 + kappa) / 4), (1, 1, 4, (1 - kappa) / 4)]
    terms, coef = [], []
    for cyc in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        for fx, fy, fz, c in one:
            t = [0, 0, 0]
            t[cyc[0]], t[cyc[1]], t[cyc[2]] = fx, fy, fz
            terms.append(t)
            coef.append(c)
    avg, cnt2 = oracle.triangle_average(N, L, edges, trip, _tables(N, L, funcs), terms, coef)
    assert np.array_equal(cnt, cnt2)
    assert np.allclose(avg, ref, rtol=1e-9, atol=1e-12 * np.max(np.abs(ref)))


# ---------------------------------------------------------------- exact quadruple counts
QUAD_COUNT_CASES = [("lin", 8, 40.0, 3), ("log", 10, 25.0, 4), ("lin", 12, 30.0, 4), ("aliased", 10, 20.0, 3),
                    ("full", 8, 10.0, None)]


@pytest.mark.parametrize("kind,N,L,nb", QUAD_COUNT_CASES)
def test_quad_counts_exact_equal_brute_force(kind, N, L, nb):
    """The pair-count route gives the brute-force ordered quadruple counts of
    every candidate (a <= b <= c <= d), including the zero ones."""
    edges = _subset_case(kind, N, L, nb)
    f = fields.lognormal(N, 0.5, -1.5, seed=11)
    d = oracle.direct_trispectrum(f, L, edges)
    cnt = d["ordered_cnt"]
    k = cnt.shape[0]
    cand = [q for q in itertools.combinations_with_replacement(range(k), 4)]
    ex = oracle.quad_counts_exact(N, L, edges, cand)
    assert ex == [int(cnt[q]) for q in cand]
    assert any(v == 0 for v in ex) or kind in ("full", "aliased")  # wrapped sums close every candidate


def test_quad_counts_exact_sum_rule_full_cover():
    """Every mode in a bin: the ordered counts over all bin 4-tuples add up to
    the number of closed mode quadruples, N_pix^3."""
    N, L = 8, 10.0
    edges = _full_cover_edges(N, L)
    nb = len(edges) - 1
    cand = list(itertools.combinations_with_replacement(range(nb), 4))
    ex = oracle.quad_counts_exact(N, L, edges, cand)
    total = 0
    for q, v in zip(cand, ex):
        perms = math.factorial(4)
        for b in set(q):
            perms //= math.factorial(q.count(b))
        total += perms * v
    assert total == (N ** 3) ** 3


def test_quad_counts_exact_match_rounded_fft_sums():
    """Below 2^53 the rounded FP64 count-field sums of the FFT estimator are
    the same integers."""
    N, L = 24, 60.0
    edges = fields.log_edges(N, L, 6)
    f = fields.lognormal(N, 0.5, -1.5, seed=12)
    quads = list(itertools.combinations_with_replacement(range(6), 4))
    e = oracle.fft_estimator(f, L, edges, triplets=[], quads=quads)
    ex = oracle.quad_counts_exact(N, L, edges, quads)
    assert max(ex) < 2 ** 53
    assert ex == [int(v) for v in e["N_quad"]]


# ---------------------------------------------------------------- diagonal-resolved trispectrum
def _diag_edges(N, L, top=None):
    """Diagonal shells from 0 (the paired q = 0 alone first) to beyond the
    corner of the grid."""
    kf = 2 * math.pi / L
    top = top if top is not None else 3 * (N // 2) ** 2 + 1
    sq = [0.0, 0.5, 2.5, 6.5, 12.5, float(top) + 0.5]
    return [kf * math.sqrt(s) for s in sq]


@pytest.mark.parametrize("N,L,kind,nb,seed", [(8, 40.0, "lin", 3, 21), (10, 25.0, "log", 4, 22)])
def test_diagonal_trispectrum_fft_route_equals_brute_force(N, L, kind, nb, seed):
    edges = fields.linear_edges(N, L, nb) if kind == "lin" else fields.log_edges(N, L, nb)
    dedges = _diag_edges(N, L)
    f = fields.quadratic_local(N, 1.0, -1.5, 0.3, seed=seed)
    d = oracle.direct_trispectrum_diagonal(f, L, edges, dedges)
    k = d["cnt"].shape[0]
    quads = list(itertools.combinations_with_replacement(range(k), 4))
    e = oracle.diagonal_trispectrum(f, L, edges, dedges, quads)
    scale = max(1e-300, float(np.abs(d["num"]).max()))
    for i, q in enumerate(quads):
        assert e["cnt"][i] == [int(v) for v in d["cnt"][q]]
        assert np.allclose(e["num"][i], d["num"][q], rtol=1e-10, atol=1e-12 * scale)
        assert np.allclose(e["num_im"][i], 0.0, atol=1e-10 * scale)  # real field: the sums are real


def test_diagonal_bins_add_up_to_the_raw_trispectrum():
    """Diagonal shells covering every |k1 + k2|: the diagonal sums and counts
    add up to the plain four-shell sum and count of each quadruplet."""
    N, L = 8, 40.0
    edges = fields.linear_edges(N, L, 3)
    f = fields.lognormal(N, 0.5, -1.5, seed=23)
    raw = oracle.direct_trispectrum(f, L, edges)
    e = oracle.diagonal_trispectrum(f, L, edges, _diag_edges(N, L), raw["quads"])
    assert [sum(row) for row in e["cnt"]] == [int(v) for v in raw["N_quad"]]
    assert np.allclose(e["num"].sum(axis=1), raw["num"], rtol=1e-10, atol=1e-12 * np.abs(raw["num"]).max())


def test_diagonal_zero_shell_is_the_paired_term():
    """The shell holding only q = k1 + k2 = 0: for (a, a, c, c) its
    quadruples are m2 = -m1, m4 = -m3, so the sum is S2_a S2_c (S2 the
    shell's sum of |D|^2) and the count |S_a| |S_c|; other quadruplets have
    none."""
    N, L = 10, 30.0
    edges = fields.linear_edges(N, L, 3)
    f = fields.lognormal(N, 0.5, -1.5, seed=24)
    thr = oracle.thresholds(edges, L)
    bins = oracle.bin_index(N, thr)
    D = oracle.spectrum(f)
    a2 = np.abs(D) ** 2
    S2 = [float(a2[bins == b].sum()) for b in range(3)]
    S = [int((bins == b).sum()) for b in range(3)]
    quads = list(itertools.combinations_with_replacement(range(3), 4))
    e = oracle.diagonal_trispectrum(f, L, edges, _diag_edges(N, L), quads)
    for i, (a, b, c, d) in enumerate(quads):
        if a == b and c == d:
            assert e["cnt"][i][0] == S[a] * S[c]
            assert math.isclose(e["num"][i, 0], S2[a] * S2[c], rel_tol=1e-12)
        else:
            assert e["cnt"][i][0] == 0 and abs(e["num"][i, 0]) <= 1e-12 * max(S2) ** 2  # FFT rounding only


# ---------------------------------------------------------------- non-cubic boxes, complex fields
def _complex_field(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


GENERAL_CASES = [((6, 8, 10), (30.0, 40.0, 55.0), "complex", 31), ((8, 8, 12), (20.0, 20.0, 33.0), "real", 32),
                 ((5, 9, 6), (10.0, 21.0, 13.0), "complex", 33)]


def _general_edges(shape, Ls, nb):
    kmin = 2 * math.pi / max(Ls)
    kmax = 2 * math.pi * min(n / 4.0 / L for n, L in zip(shape, Ls))
    return np.geomspace(0.9 * kmin, kmax, nb + 1)


@pytest.mark.parametrize("shape,Ls,kind,seed", GENERAL_CASES)
def test_general_fft_route_equals_brute_force(shape, Ls, kind, seed):
    f = _complex_field(shape, seed)
    if kind == "real":
        f = f.real
    edges = _general_edges(shape, Ls, 4)
    e = oracle.general_bispectrum(f, Ls, edges)
    num, cnt = oracle.general_direct_sums(f, Ls, edges)
    closed = [tuple(t) for t in np.argwhere(cnt > 0) if t[0] <= t[1] <= t[2]]
    assert [tuple(t) for t in e["triplets"]] == sorted(closed)
    for t, (a, b, c) in enumerate(e["triplets"]):
        assert e["N_tri"][t] == cnt[a, b, c]
        assert abs(e["num"][t] - num[a, b, c]) <= 1e-10 * np.abs(num).max()
    if kind == "real":
        assert np.abs(e["num"].imag).max() <= 1e-10 * np.abs(e["num"]).max()


def test_general_cubic_real_case_is_the_cubic_estimator():
    N, L = 16, 40.0
    f = fields.lognormal(N, 0.5, -1.5, seed=34)
    edges = fields.log_edges(N, L, 5) * 1.0001  # away from |m|^2 ties
    g = oracle.general_bispectrum(f, (L, L, L), edges)
    c = oracle.fft_estimator(f, L, edges, triplets=g["triplets"])
    assert np.array_equal(g["N_tri"], c["N_tri"])
    assert np.allclose(g["B"].real, c["B"], rtol=1e-10, atol=1e-12 * np.abs(c["B"]).max())
    ok = np.isfinite(c["P"])
    assert np.allclose(g["P"].real[ok], c["P"][ok], rtol=1e-10)


def test_general_axis_permutation_and_conjugation():
    shape, Ls = (6, 8, 10), (30.0, 40.0, 55.0)
    f = _complex_field(shape, 35)
    edges = _general_edges(shape, Ls, 4)
    e = oracle.general_bispectrum(f, Ls, edges)
    # the same data with the axes relabelled
    t = oracle.general_bispectrum(np.transpose(f, (1, 2, 0)), (Ls[1], Ls[2], Ls[0]), edges)
    assert np.array_equal(t["triplets"], e["triplets"]) and np.array_equal(t["N_tri"], e["N_tri"])
    assert np.allclose(t["B"], e["B"], rtol=1e-10, atol=1e-12 * np.abs(e["B"]).max())
    # conj(delta) has D'(m) = conj D(-m): B and P become their conjugates
    c = oracle.general_bispectrum(np.conj(f), Ls, edges)
    assert np.allclose(c["B"], np.conj(e["B"]), rtol=1e-10, atol=1e-12 * np.abs(e["B"]).max())
    ok = np.isfinite(e["P"].real)
    assert np.allclose(c["P"][ok], np.conj(e["P"][ok]), rtol=1e-10)
