"""FP64 CPU oracle for the FFT polyspectrum estimator (arXiv 1705.06284).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this
package.  It shares no code with the CUDA library and never imports it; the
only module both sides use is the input generator package ``fields``.

Two independent routes to the same numbers:

* :func:`direct_bispectrum` -- the definition, Eq. bi_direct over full
  shells: an all-pairs sum over modes of Re[D(m1) D(m2) D(m3)] with
  m3 = -(m1+m2) (mod N), plus brute-force triangle counts (plain C in
  ``direct.c``).
* :func:`fft_estimator` -- the paper's own estimator, Eqs. delta_nr,
  Jeong_gen, Jeong_PS and Jeong_BI, written literally in NumPy FP64: mask the
  spectrum to each shell, inverse-FFT (unnormalised) to the shell fields
  I_b(x) and count fields N_b(x), and take real-space products.

Substituting the DFT form of the Kronecker delta (Sec. 2, the identity that
turns Eq. gen_Nspec3 into Eq. gen_Nspec4) shows the two are equal up to
rounding; the pins in ``tests/test_oracle.py`` check that and more.

Readings of the paper this oracle takes where the text is silent or garbled:

* Normalisation: B = V^2/N_pix^3 * num/(N_pix N_tri) as in Eq. Jeong_BI
  (Eq. bi_direct's 1/(2 pi)^3 is the continuum form; the discrete derivation
  of Eqs. gen_Nspec1-2 gives H^p/V with H = V/N_pix).  P uses V/N_pix^2
  (Eq. Jeong_PS) and the trispectrum V^3/N_pix^4 (Eq. Jeong_gen, p = 4).
* Shells: the scalar |m| (spherically averaged spectra), membership
  lo <= |m| k_f < hi, evaluated as thr[b] <= |m|^2 < thr[b+1] on integers.
* Closure: modulo the grid (the FFT's Kronecker delta), components reduced
  into [-N/2, N/2).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

try:  # the same library transforms, multithreaded, where scipy is present
    import scipy.fft as _sfft

    def _fftn(a):
        return _sfft.fftn(a, workers=-1)

    def _ifftn(a):
        return _sfft.ifftn(a, workers=-1)

    def _rfftn(a):
        return _sfft.rfftn(a, workers=-1)

    def _irfftn(a, s):
        return _sfft.irfftn(a, s=s, workers=-1)
except Exception:  # pragma: no cover
    _fftn, _ifftn = np.fft.fftn, np.fft.ifftn
    _rfftn = np.fft.rfftn

    def _irfftn(a, s):
        return np.fft.irfftn(a, s=s)

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``direct.c`` into ``liboracle.so`` (gcc, OpenMP)."""
    src = os.path.join(_HERE, "direct.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99",
                               src, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64p = ctypes.POINTER(ctypes.c_int64)
            dp = ctypes.POINTER(ctypes.c_double)
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.oracle_num_threads.restype = ctypes.c_int
            lib.oracle_count_modes.restype = ctypes.c_int64
            lib.oracle_count_modes.argtypes = [ctypes.c_int, ctypes.c_int, i64p]
            lib.oracle_direct_bispectrum.restype = ctypes.c_int64
            lib.oracle_direct_bispectrum.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, i64p,
                                                     dp, dp, i64p, ctypes.c_int64, ctypes.c_int64]
            lib.oracle_direct_triplets.restype = None
            lib.oracle_direct_triplets.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, i64p,
                                                   ctypes.c_int, i32p, dp, dp, i64p]
            lib.oracle_closed_triplets.restype = None
            lib.oracle_closed_triplets.argtypes = [ctypes.c_int, ctypes.c_int, i64p, ctypes.c_int,
                                                   i32p, i32p]
            lib.oracle_triangle_sums.restype = None
            lib.oracle_triangle_sums.argtypes = [ctypes.c_int, ctypes.c_int, i64p, ctypes.c_int, i32p, ctypes.c_int,
                                                 ctypes.c_int64, dp, ctypes.c_int, i32p, dp, dp, i64p]
            lib.oracle_direct_trispectrum_diag.restype = None
            lib.oracle_direct_trispectrum_diag.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, i64p, ctypes.c_int,
                                                           i64p, dp, dp, i64p]
            lib.oracle_direct_trispectrum.restype = None
            lib.oracle_direct_trispectrum.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, i64p,
                                                      dp, dp, i64p, ctypes.c_int]
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def num_threads() -> int:
    """OpenMP threads the C oracle runs with."""
    return int(_load().oracle_num_threads())


# --------------------------------------------------------------------------
# Units, bins and the spectrum (Eqs. FFTconventions, DeltaFFTtoDelta).
# --------------------------------------------------------------------------

def k_fundamental(L: float) -> float:
    """k_f = 2 pi / L (Sec. 2)."""
    return 2.0 * math.pi / L


def thresholds(edges, L: float) -> np.ndarray:
    """Integer thresholds on |m|^2 for physical bin edges.

    Bin b holds the modes with edges[b] <= |m| k_f < edges[b+1].  With
    s = (edge/k_f)^2 (FP64), the smallest integer |m|^2 meeting |m| k_f >=
    edge is ceil(s).  Edges that are whole multiples of k_f give an s a few
    ulps away from an integer; s is snapped to that integer first when
    |s - round(s)| <= 1e-9 max(1, s), so that such edges fall exactly where
    they were meant to.
    """
    kf = k_fundamental(L)
    e = np.asarray(edges, dtype=np.float64)
    out = np.empty(e.shape, dtype=np.int64)
    for i, v in enumerate(e):
        if v <= 0.0:
            out[i] = 0
            continue
        s = (v / kf) * (v / kf)
        r = round(s)
        if abs(s - r) <= 1e-9 * max(1.0, s):
            s = float(r)
        out[i] = int(math.ceil(s))
    if np.any(np.diff(out) < 0):
        raise ValueError("edges must be ascending")
    return out


def spectrum(field: np.ndarray) -> np.ndarray:
    """Unnormalised forward DFT, D(m) = sum_n delta(n) e^{-2 pi i m.n/N}
    (Eq. DeltaFFTtoDelta), full complex box in FFT index order."""
    return _fftn(np.asarray(field, dtype=np.float64))


def mode_squares(N: int) -> np.ndarray:
    """|m|^2 on the full grid, components wrapped into [-N/2, N/2)."""
    f = np.fft.fftfreq(N, d=1.0 / N).astype(np.int64)
    return f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2


def bin_index(N: int, thr) -> np.ndarray:
    """Bin of every grid mode (-1 when in no bin)."""
    thr = np.asarray(thr, dtype=np.int64)
    m2 = mode_squares(N)
    b = np.searchsorted(thr, m2, side="right") - 1
    b[(m2 < thr[0]) | (m2 >= thr[-1])] = -1
    return b


def shell_sizes(N: int, thr) -> np.ndarray:
    """|S_b|: number of modes in each bin."""
    b = bin_index(N, thr)
    nb = len(thr) - 1
    return np.bincount(b[b >= 0].ravel(), minlength=nb).astype(np.int64)


# --------------------------------------------------------------------------
# Route 1: the direct-measurement definition (Eq. bi_direct, full shells).
# --------------------------------------------------------------------------

def direct_sums(field, thr, m1_start: int = 0, m1_stride: int = 1):
    """Ordered all-pairs sums (num, num_im, cnt) of shape (nb, nb, nb).

    Returns also the number of m1 modes processed (all of them unless a
    sample is asked for with ``m1_stride > 1``).
    """
    return direct_sums_from_spectrum(spectrum(field), thr, m1_start, m1_stride)


def direct_sums_from_spectrum(D, thr, m1_start: int = 0, m1_stride: int = 1):
    """:func:`direct_sums` on a precomputed full spectrum D (FFT order)."""
    lib = _load()
    N = D.shape[0]
    re = np.ascontiguousarray(D.real)
    im = np.ascontiguousarray(D.imag)
    thr = np.ascontiguousarray(thr, dtype=np.int64)
    nb = len(thr) - 1
    num = np.zeros(nb ** 3)
    numi = np.zeros(nb ** 3)
    cnt = np.zeros(nb ** 3, dtype=np.int64)
    done = lib.oracle_direct_bispectrum(N, _p(re, ctypes.c_double), _p(im, ctypes.c_double), nb,
                                        _p(thr, ctypes.c_int64), _p(num, ctypes.c_double),
                                        _p(numi, ctypes.c_double), _p(cnt, ctypes.c_int64),
                                        int(m1_start), int(m1_stride))
    sh = (nb, nb, nb)
    return num.reshape(sh), numi.reshape(sh), cnt.reshape(sh), int(done)


def count_modes(N: int, thr) -> int:
    thr = np.ascontiguousarray(thr, dtype=np.int64)
    return int(_load().oracle_count_modes(N, len(thr) - 1, _p(thr, ctypes.c_int64)))


def direct_bispectrum(field, L: float, edges):
    """Bispectrum by direct measurement over full shells (Eq. bi_direct).

    Returns a dict with
      ``triplets`` (ntrip, 3) int32, lexicographic a <= b <= c with N_tri > 0;
      ``N_tri``   (ntrip,) int64 ordered-triple counts;
      ``B``       (ntrip,) FP64, V^2/N_pix^3 * num/N_tri;
      ``num``     (ntrip,) FP64 ordered sums of Re[D1 D2 D3];
      ``num_im``  (ntrip,) FP64 ordered sums of Im[D1 D2 D3] (zero in exact
                  arithmetic);
      ``P``       (nbins,) FP64 power spectrum (shell mode average);
      ``shell``   (nbins,) int64 |S_b|.
    """
    field = np.asarray(field, dtype=np.float64)
    N = field.shape[0]
    thr = thresholds(edges, L)
    num, numi, cnt, _ = direct_sums(field, thr)
    nb = len(thr) - 1
    trip, n, ni, c = [], [], [], []
    for a in range(nb):
        for b in range(a, nb):
            for cc in range(b, nb):
                if cnt[a, b, cc] > 0:
                    trip.append((a, b, cc))
                    n.append(num[a, b, cc])
                    ni.append(numi[a, b, cc])
                    c.append(cnt[a, b, cc])
    V = float(L) ** 3
    npix = float(N) ** 3
    trip = np.array(trip, dtype=np.int32).reshape(-1, 3)
    n = np.array(n)
    c = np.array(c, dtype=np.int64)
    B = (V * V / npix ** 3) * n / np.maximum(c, 1)
    P, S = power_spectrum(field, L, edges)
    return {"triplets": trip, "N_tri": c, "B": B, "num": n, "num_im": np.array(ni),
            "P": P, "shell": S, "ordered_num": num, "ordered_cnt": cnt}


def direct_triplets(field, L: float, edges, triplets):
    """Direct sums for selected (a, b, c) only: cost sum |S_a||S_b|.

    Returns (B, num, num_im, N_tri) for the requested triplets (ordered
    triples with m1 in S_a, m2 in S_b, m3 in S_c).
    """
    lib = _load()
    field = np.asarray(field, dtype=np.float64)
    N = field.shape[0]
    D = spectrum(field)
    re = np.ascontiguousarray(D.real)
    im = np.ascontiguousarray(D.imag)
    thr = np.ascontiguousarray(thresholds(edges, L))
    abc = np.ascontiguousarray(np.asarray(triplets, dtype=np.int32).reshape(-1, 3))
    nt = abc.shape[0]
    num = np.zeros(nt)
    numi = np.zeros(nt)
    cnt = np.zeros(nt, dtype=np.int64)
    lib.oracle_direct_triplets(N, _p(re, ctypes.c_double), _p(im, ctypes.c_double), len(thr) - 1,
                               _p(thr, ctypes.c_int64), nt, _p(abc, ctypes.c_int32),
                               _p(num, ctypes.c_double), _p(numi, ctypes.c_double),
                               _p(cnt, ctypes.c_int64))
    V = float(L) ** 3
    npix = float(N) ** 3
    B = (V * V / npix ** 3) * num / np.maximum(cnt, 1)
    return B, num, numi, cnt


def closed_triplets(N: int, L: float, edges) -> np.ndarray:
    """Every bin triple a <= b <= c with N_tri > 0, lexicographic.

    Triples whose largest shell cannot be reached by the sum of the other two
    (min |m_c| > max |m_a| + max |m_b|, the triangle inequality for exact
    closure) are dropped without search; this holds when every component is
    below N/4 (then closure modulo N is exact closure).  The rest are decided
    by a witness search over the shells' modes.
    """
    thr = np.ascontiguousarray(thresholds(edges, L))
    nb = len(thr) - 1
    m2 = mode_squares(N)
    b = bin_index(N, thr)
    S = np.bincount(b[b >= 0].ravel(), minlength=nb)
    lo = np.full(nb, np.inf)
    hi = np.full(nb, -np.inf)
    for k in range(nb):
        if S[k]:
            v = m2[b == k]
            lo[k], hi[k] = math.sqrt(v.min()), math.sqrt(v.max())
    exact = thr[-1] <= (N * N + 15) // 16
    cand = []
    for a in range(nb):
        for bb in range(a, nb):
            for c in range(bb, nb):
                if not (S[a] and S[bb] and S[c]):
                    continue
                if exact and lo[c] > hi[a] + hi[bb] + 1e-9:
                    continue
                cand.append((a, bb, c))
    abc = np.ascontiguousarray(np.array(cand, dtype=np.int32).reshape(-1, 3))
    flag = np.zeros(len(abc), dtype=np.int32)
    if len(abc):
        _load().oracle_closed_triplets(N, nb, _p(thr, ctypes.c_int64), len(abc),
                                       _p(abc, ctypes.c_int32), _p(flag, ctypes.c_int32))
    return abc[flag > 0]


def direct_trispectrum(field, L: float, edges, connected: bool = False):
    """Trispectrum by direct measurement (p = 4 case of Eq. gen_Nspec3) over
    ordered quadruples; O(|M|^3), tiny grids only.

    ``connected``: leave out every quadruple in which a pair of its modes sums
    to zero modulo N (the pairing terms, which carry the disconnected P x P
    parts of a Gaussian field); the paper is silent on this part of the
    four-shell estimator, and this exclusion is the reading taken for the
    connected trispectrum.

    Returns dict with ``quads`` (nq, 4) a<=b<=c<=d with N_quad > 0,
    ``N_quad``, ``T`` = V^3/N_pix^4 * num/N_quad, ``num``, ``num_im``.
    """
    lib = _load()
    field = np.asarray(field, dtype=np.float64)
    N = field.shape[0]
    D = spectrum(field)
    re = np.ascontiguousarray(D.real)
    im = np.ascontiguousarray(D.imag)
    thr = np.ascontiguousarray(thresholds(edges, L))
    nb = len(thr) - 1
    num = np.zeros(nb ** 4)
    numi = np.zeros(nb ** 4)
    cnt = np.zeros(nb ** 4, dtype=np.int64)
    lib.oracle_direct_trispectrum(N, _p(re, ctypes.c_double), _p(im, ctypes.c_double), nb,
                                  _p(thr, ctypes.c_int64), _p(num, ctypes.c_double),
                                  _p(numi, ctypes.c_double), _p(cnt, ctypes.c_int64), 1 if connected else 0)
    sh = (nb,) * 4
    num, numi, cnt = num.reshape(sh), numi.reshape(sh), cnt.reshape(sh)
    quads, n, ni, c = [], [], [], []
    for a in range(nb):
        for b in range(a, nb):
            for cc in range(b, nb):
                for d in range(cc, nb):
                    if cnt[a, b, cc, d] > 0:
                        quads.append((a, b, cc, d))
                        n.append(num[a, b, cc, d])
                        ni.append(numi[a, b, cc, d])
                        c.append(cnt[a, b, cc, d])
    V = float(L) ** 3
    npix = float(N) ** 3
    n = np.array(n)
    c = np.array(c, dtype=np.int64)
    T = (V ** 3 / npix ** 4) * n / np.maximum(c, 1)
    return {"quads": np.array(quads, dtype=np.int32).reshape(-1, 4), "N_quad": c, "T": T,
            "num": n, "num_im": np.array(ni), "ordered_num": num, "ordered_cnt": cnt}


def pairing_terms(D: np.ndarray, bins: np.ndarray, quads):
    """Sum and count of the paired ordered quadruples of each (a<=b<=c<=d).

    A closed quadruple (m1, m2, m3, m4) in S_a x S_b x S_c x S_d is paired when
    m1 + m2, m1 + m3 or m2 + m3 is 0 modulo N (with the closure, the three
    pairings).  Since |-m| = |m|, m1 + m2 = 0 needs a = b and then c = d; the
    other two pairings need a = b = c = d.  By inclusion-exclusion over the
    three events, with S2_b = sum_{S_b} |D|^2, S4_b = sum_{S_b} |D|^4 and Z_b
    the self-conjugate modes of S_b (m = -m mod N, where D is real):
      a = b < c = d :  sum = S2_a S2_c,                count = |S_a| |S_c|
      a = b = c = d :  sum = 3 S2^2 - 3 S4 + sum_Z D^4, count = 3|S|^2 - 3|S| + |Z|
      otherwise     :  0.
    Returns (sums, counts) as FP64 arrays."""
    N = D.shape[0]
    q = np.asarray(quads, dtype=np.int64).reshape(-1, 4)
    nb = max(int(bins.max()) + 1, int(q.max()) + 1 if len(q) else 0)
    a2 = D.real ** 2 + D.imag ** 2
    sel = bins >= 0
    S = np.bincount(bins[sel].ravel(), minlength=nb).astype(np.float64)
    S2 = np.bincount(bins[sel].ravel(), weights=a2[sel].ravel(), minlength=nb)
    S4 = np.bincount(bins[sel].ravel(), weights=(a2 * a2)[sel].ravel(), minlength=nb)
    # self-conjugate modes: every component 0 or N/2
    idx = np.arange(N)
    sc1 = (idx == 0) | (2 * idx == N)
    sc = sc1[:, None, None] & sc1[None, :, None] & sc1[None, None, :] & sel
    Zc = np.bincount(bins[sc].ravel(), minlength=nb).astype(np.float64)
    Z4 = np.bincount(bins[sc].ravel(), weights=(D.real ** 4)[sc].ravel(), minlength=nb)
    sums = np.zeros(len(q))
    cnts = np.zeros(len(q))
    for i, (a, b, c, d) in enumerate(q):
        if a != b or c != d:
            continue
        if a != c:
            sums[i] = S2[a] * S2[c]
            cnts[i] = S[a] * S[c]
        else:
            sums[i] = 3 * S2[a] ** 2 - 3 * S4[a] + Z4[a]
            cnts[i] = 3 * S[a] ** 2 - 3 * S[a] + Zc[a]
    return sums, cnts


def pair_counts(bins: np.ndarray, a: int, b: int) -> np.ndarray:
    """C_ab(q) = #{m1 in S_a, m2 in S_b : m1 + m2 = q (mod N)} on the N^3 grid
    of q (FFT index order), as int64: the cyclic convolution of the two
    shells' indicator arrays, taken with a library FFT and rounded.  The
    FFT's error is of order 1e-16 |S_a| |S_b| log N, far below 1/2 for any
    grid this oracle runs on; a value further than 0.25 from an integer
    raises."""
    N = bins.shape[0]
    fa = _rfftn((bins == a).astype(np.float64))
    fb = fa if b == a else _rfftn((bins == b).astype(np.float64))
    c = _irfftn(fa * fb, (N, N, N))
    r = np.rint(c)
    if r.size and float(np.max(np.abs(c - r))) > 0.25:
        raise ArithmeticError("pair-count convolution is not integral")
    return r.astype(np.int64)


def quad_counts_exact(N: int, L: float, edges, quads) -> list:
    """Exact ordered quadruple counts (the denominator of Eq. gen_Nspec3 with
    p = 4) as Python integers, which hold the counts past 2^63 of wide shells:
      N_quad(a, b, c, d) = #{(m1, m2, m3, m4) in S_a x S_b x S_c x S_d :
                             m1 + m2 + m3 + m4 = 0 (mod N)}
                         = sum_q C_ab(q) C_cd(-q)      (see :func:`pair_counts`),
    the sum taken in exact integer arithmetic (int64 per grid plane where its
    products cannot overflow, Python integers across planes)."""
    thr = thresholds(edges, L)
    bins = bin_index(N, thr)
    cache = {}

    def C(a, b):
        k = (min(a, b), max(a, b))
        if k not in cache:
            cache[k] = pair_counts(bins, k[0], k[1])
        return cache[k]

    out = []
    for a, b, c, d in np.asarray(quads, dtype=np.int64).reshape(-1, 4):
        Cab = C(int(a), int(b))
        Ccd = C(int(c), int(d))
        # C_cd(-q): index (-i) mod N along every axis
        neg = np.roll(Ccd[::-1, ::-1, ::-1], 1, axis=(0, 1, 2))
        big = int(Cab.max(initial=0)) * int(neg.max(initial=0))
        total = 0
        if big * N * N < 2 ** 62:
            for x in range(N):
                total += int(np.sum(Cab[x] * neg[x], dtype=np.int64))
        else:
            for x in range(N):
                for y in range(N):
                    total += sum(int(u) * int(v) for u, v in zip(Cab[x, y], neg[x, y]))
        out.append(total)
    return out


def direct_trispectrum_diagonal(field, L: float, edges, diag_edges):
    """Diagonal-resolved trispectrum by direct measurement (tiny grids): the
    ordered closed quadruples of Eq. gen_Nspec3 (p = 4) split by the bin D of
    their diagonal q = k1 + k2 (shells on |q| like the bins, thresholds from
    ``diag_edges``).  Returns the ordered arrays num, num_im, cnt of shape
    (nb, nb, nb, nb, nD)."""
    lib = _load()
    field = np.asarray(field, dtype=np.float64)
    N = field.shape[0]
    D = spectrum(field)
    re = np.ascontiguousarray(D.real)
    im = np.ascontiguousarray(D.imag)
    thr = np.ascontiguousarray(thresholds(edges, L))
    dthr = np.ascontiguousarray(thresholds(diag_edges, L))
    nb, nd = len(thr) - 1, len(dthr) - 1
    num = np.zeros(nb ** 4 * nd)
    numi = np.zeros(nb ** 4 * nd)
    cnt = np.zeros(nb ** 4 * nd, dtype=np.int64)
    lib.oracle_direct_trispectrum_diag(N, _p(re, ctypes.c_double), _p(im, ctypes.c_double), nb,
                                       _p(thr, ctypes.c_int64), nd, _p(dthr, ctypes.c_int64),
                                       _p(num, ctypes.c_double), _p(numi, ctypes.c_double),
                                       _p(cnt, ctypes.c_int64))
    sh = (nb,) * 4 + (nd,)
    return {"num": num.reshape(sh), "num_im": numi.reshape(sh), "cnt": cnt.reshape(sh)}


def diagonal_trispectrum(field, L: float, edges, diag_edges, quads):
    """Diagonal-resolved trispectrum, the FFT route (FP64 NumPy).  For a
    quadruplet (a, b, c, d) and a diagonal bin D, the closed quadruples with
    k1 + k2 = q in shell D:
      num_D = sum_{q in S_D} F_ab(q) F_cd(-q),  F_ab(q) = sum_{m1 + m2 = q} D(m1) D(m2),
    and F_ab is the forward DFT of the product of two shell fields divided by
    N_pix (F_ab = DFT[I_a I_b] / N_pix, the Kronecker-delta identity of Sec. 2
    applied to the pair); the count is sum_{q in S_D} C_ab(q) C_cd(-q) of the
    integer pair counts (:func:`pair_counts`).  T_D = V^3/N_pix^4 num_D / N_D
    (the normalisation of Eq. Jeong_gen with p = 4), NaN where N_D = 0.
    Returns dict with ``num`` (nq, nD) FP64 real parts, ``num_im``, ``cnt``
    (nq, nD) Python integers, ``T`` (nq, nD) and ``mag`` (nq, nD), the
    cancellation-free scale sum_{q in S_D} |F_ab(q)| |F_cd(-q)|."""
    field = np.asarray(field, dtype=np.float64)
    N = field.shape[0]
    npix = float(N) ** 3
    V = float(L) ** 3
    thr = thresholds(edges, L)
    dthr = thresholds(diag_edges, L)
    nd = len(dthr) - 1
    bins = bin_index(N, thr)
    dbin = bin_index(N, dthr)
    Dk = spectrum(field)
    neg = lambda A: np.roll(A[::-1, ::-1, ::-1], 1, axis=(0, 1, 2))  # A(-q mod N)
    I, F, C = {}, {}, {}

    def shell(b):
        if b not in I:
            I[b] = shell_field(Dk, bins, b)
        return I[b]

    def pair_spec(a, b):
        if (a, b) not in F:
            F[(a, b)] = _fftn(shell(a) * shell(b)) / npix
        return F[(a, b)]

    def pair_cnt(a, b):
        if (a, b) not in C:
            C[(a, b)] = pair_counts(bins, a, b)
        return C[(a, b)]

    q = np.asarray(quads, dtype=np.int64).reshape(-1, 4)
    num = np.zeros((len(q), nd))
    numi = np.zeros((len(q), nd))
    mag = np.zeros((len(q), nd))
    cnt = [[0] * nd for _ in range(len(q))]
    for i, (a, b, c, d) in enumerate(q):
        prod = pair_spec(int(a), int(b)) * neg(pair_spec(int(c), int(d)))
        aprod = np.abs(prod)
        cc = pair_cnt(int(a), int(b)) * neg(pair_cnt(int(c), int(d)))
        for D in range(nd):
            sel = dbin == D
            num[i, D] = float(np.sum(prod.real[sel]))
            mag[i, D] = float(np.sum(aprod[sel]))
            numi[i, D] = float(np.sum(prod.imag[sel]))
            cnt[i][D] = int(np.sum(cc[sel], dtype=np.int64)) if int(cc.max(initial=0)) * cc.size < 2 ** 62 \
                else sum(int(v) for v in cc[sel])
    nc = np.array([[float(v) for v in row] for row in cnt]).reshape(len(q), nd)
    with np.errstate(invalid="ignore", divide="ignore"):
        T = np.where(nc > 0, (V ** 3 / npix ** 4) * num / np.where(nc > 0, nc, 1.0), np.nan)
    return {"num": num, "num_im": numi, "cnt": cnt, "T": T, "mag": mag}


# --------------------------------------------------------------------------
# Non-cubic boxes and complex fields (Sec. 2: the footnote on non-cubic data
# and the remark that Eq. Jeong_gen applies to complex data through complex
# DFTs).  Grid N_x x N_y x N_z, box L_x x L_y x L_z, mode m with components
# in FFT order; k = 2 pi (m_x/L_x, m_y/L_y, m_z/L_z); V = L_x L_y L_z and
# N_pix = N_x N_y N_z take the places of L^3 and N^3.
# --------------------------------------------------------------------------

def general_mode_s(shape, Ls) -> np.ndarray:
    """s(m) = (m_x/L_x)^2 + (m_y/L_y)^2 + (m_z/L_z)^2 = |k|^2 / (2 pi)^2 on the
    grid (FFT order), evaluated in that order in FP64."""
    f = [np.concatenate([np.arange(0, (n + 1) // 2), np.arange(-(n // 2), 0)]).astype(np.float64) for n in shape]
    ux = f[0] / float(Ls[0])
    uy = f[1] / float(Ls[1])
    uz = f[2] / float(Ls[2])
    return (ux[:, None, None] * ux[:, None, None] + uy[None, :, None] * uy[None, :, None]) + \
        uz[None, None, :] * uz[None, None, :]


def general_thresholds(edges) -> np.ndarray:
    """t_b = (edge_b / (2 pi))^2: bin b holds t_b <= s(m) < t_{b+1}."""
    out = []
    for e in np.asarray(edges, dtype=np.float64):
        u = float(e) / (2.0 * math.pi)
        out.append(u * u)
    return np.array(out)


def general_bin_index(shape, Ls, edges) -> np.ndarray:
    t = general_thresholds(edges)
    s = general_mode_s(shape, Ls)
    b = np.searchsorted(t, s, side="right") - 1
    b[(s < t[0]) | (s >= t[-1])] = -1
    return b


def general_bispectrum(field, Ls, edges):
    """The FFT estimator on a non-cubic grid for a real or complex field
    (Eqs. delta_nr, Jeong_PS, Jeong_BI with complex DFTs), FP64:
      D = DFT[delta] (complex, no Hermitian half), I_b = unnormalised inverse
      DFT of D on S_b (complex), N_b the same of the indicator (real: every
      shell is symmetric under m -> -m modulo the grid),
      B = V^2/N_pix^3 sum_n I_a I_b I_c / (N_pix N_tri)   (complex),
      P = V/N_pix^2   sum_n I_b I_b / (N_pix |S_b|)        (complex: for a
          complex field Eq. Jeong_PS pairs D(m) with D(-m)),
    over every a <= b <= c of non-empty bins with N_tri > 0 (closure modulo
    the grid along each axis).  Returns dict with triplets, N_tri, num
    (complex ordered sums sum_n I_a I_b I_c / N_pix), B, P, shell."""
    field = np.asarray(field)
    shape = field.shape
    npix = float(np.prod(shape))
    V = float(Ls[0]) * float(Ls[1]) * float(Ls[2])
    bins = general_bin_index(shape, Ls, edges)
    nb = len(edges) - 1
    D = _fftn(field.astype(np.complex128))
    S = np.bincount(bins[bins >= 0].ravel(), minlength=nb).astype(np.int64)
    I = {b: _ifftn(np.where(bins == b, D, 0.0)) * npix for b in range(nb) if S[b]}
    C = {b: (_ifftn((bins == b).astype(np.complex128)) * npix).real for b in range(nb) if S[b]}
    P = np.full(nb, np.nan + 0j)
    for b in I:
        P[b] = (V / npix ** 2) * complex(np.sum(I[b] * I[b])) / (npix * S[b])
    trip, cnt, num = [], [], []
    for a in I:
        for b in I:
            if b < a:
                continue
            for c in I:
                if c < b:
                    continue
                n = float(np.sum(C[a] * C[b] * C[c])) / npix
                r = round(n)
                if abs(n - r) > 0.25:
                    raise ArithmeticError("count sum is not an integer")
                if r > 0:
                    trip.append((a, b, c))
                    cnt.append(r)
                    num.append(complex(np.sum(I[a] * I[b] * I[c])) / npix)
    cnt = np.array(cnt, dtype=np.int64)
    num = np.array(num, dtype=np.complex128)
    B = (V * V / npix ** 3) * num / np.maximum(cnt, 1)
    return {"triplets": np.array(trip, dtype=np.int32).reshape(-1, 3), "N_tri": cnt, "num": num, "B": B, "P": P,
            "shell": S}


def general_direct_sums(field, Ls, edges):
    """Ordered all-pairs sums by the definition (tiny grids): for every m1, m2
    with m3 = -(m1 + m2) modulo the grid along each axis, D(m1) D(m2) D(m3)
    and 1 added to (bin m1, bin m2, bin m3).  Returns (num complex, cnt) of
    shape (nb, nb, nb)."""
    field = np.asarray(field)
    shape = field.shape
    nb = len(edges) - 1
    bins = general_bin_index(shape, Ls, edges)
    D = _fftn(field.astype(np.complex128))
    idx = np.argwhere(bins >= 0)
    num = np.zeros((nb, nb, nb), dtype=np.complex128)
    cnt = np.zeros((nb, nb, nb), dtype=np.int64)
    n = np.array(shape)
    for m1 in idx:
        m3 = (-(m1[None, :] + idx)) % n
        b3 = bins[m3[:, 0], m3[:, 1], m3[:, 2]]
        ok = b3 >= 0
        a = bins[tuple(m1)]
        b2 = bins[idx[ok, 0], idx[ok, 1], idx[ok, 2]]
        v = D[tuple(m1)] * D[idx[ok, 0], idx[ok, 1], idx[ok, 2]] * D[m3[ok, 0], m3[ok, 1], m3[ok, 2]]
        np.add.at(num, (a, b2, b3[ok]), v)
        np.add.at(cnt, (a, b2, b3[ok]), 1)
    return num, cnt


def rebinned_bispectrum(field, L: float, edges, k_edges, mu_edges, k_rep=None):
    """Fine bins, then (k1, k2, cos theta) cells (Sec. 3.1: bin finely, then
    rebin; theta is the triangle's internal angle between k1 and k2, the
    reading of Fig. theta_illus taken here: cos theta = (k1^2 + k2^2 -
    k3^2)/(2 k1 k2)).  Every ordered bin triple (a, b, c) with closed triples
    is the configuration k1 = k_rep[a], k2 = k_rep[b], k3 = k_rep[c]; a cell
    sums the ordered direct sums and counts (Eq. bi_direct) of the
    configurations inside it.  The representative sides of a closed triplet
    can break the triangle inequality by up to a bin width; cos theta is then
    clamped to [-1, 1] (the degenerate, squeezed or folded, end).  ``k_rep`` defaults to the midpoint of each fine
    bin's edges on the integer shells (sqrt(thr[b]) and sqrt(thr[b+1]) in k_f
    units).  Returns (B, counts, num) of shape (nk, nk, nmu); empty cells NaN."""
    field = np.asarray(field, dtype=np.float64)
    N = field.shape[0]
    thr = thresholds(edges, L)
    nb = len(thr) - 1
    kf = k_fundamental(L)
    if k_rep is None:
        k_rep = 0.5 * kf * (np.sqrt(thr[:-1].astype(np.float64)) + np.sqrt(thr[1:].astype(np.float64)))
    ke = np.asarray(k_edges, dtype=np.float64)
    me = np.asarray(mu_edges, dtype=np.float64)
    nk, nmu = len(ke) - 1, len(me) - 1
    num, _, cnt, _ = direct_sums(field, thr)
    cn = np.zeros((nk, nk, nmu))
    cc = np.zeros((nk, nk, nmu), dtype=np.int64)

    def cell(v, e):
        if not (e[0] <= v < e[-1]):
            return -1
        return int(np.searchsorted(e, v, side="right")) - 1
    for a in range(nb):
        for b in range(nb):
            for c in range(nb):
                if cnt[a, b, c] == 0:
                    continue
                k1, k2, k3 = k_rep[a], k_rep[b], k_rep[c]
                K1, K2 = cell(k1, ke), cell(k2, ke)
                mu = min(1.0, max(-1.0, (k1 * k1 + k2 * k2 - k3 * k3) / (2 * k1 * k2)))
                MU = cell(mu, me)
                if K1 < 0 or K2 < 0 or MU < 0:
                    continue
                cn[K1, K2, MU] += num[a, b, c]
                cc[K1, K2, MU] += cnt[a, b, c]
    V = float(L) ** 3
    npix = float(N) ** 3
    with np.errstate(invalid="ignore", divide="ignore"):
        B = np.where(cc > 0, (V * V / npix ** 3) * cn / np.maximum(cc, 1), np.nan)
    return B, cc, cn


def triangle_average(N: int, L: float, edges, triplets, tables, terms, coef):
    """Separable models averaged over each triplet's closed triangles (the
    paper's theory points are the theory evaluated on every triangle of a bin
    and averaged, Sec. 3.3): out[t] = (1/N_tri) sum over ordered closed
    (m1, m2, m3) in S_a x S_b x S_c of sum_k coef[k] f_i(|m1|) f_j(|m2|)
    f_l(|m3|), with f tabulated at integer |m|^2 (``tables`` [nfunc][nw]).
    Plain enumeration of the triangles.  Returns (average, N_tri)."""
    thr = np.ascontiguousarray(thresholds(edges, L))
    abc = np.ascontiguousarray(np.asarray(triplets, dtype=np.int32).reshape(-1, 3))
    w = np.ascontiguousarray(tables, dtype=np.float64)
    t = np.ascontiguousarray(terms, dtype=np.int32).reshape(-1, 3)
    c = np.ascontiguousarray(coef, dtype=np.float64).ravel()
    if w.shape[1] <= 3 * (N // 2) ** 2:
        raise ValueError("tables must cover every |m|^2 of the grid")
    out = np.zeros(len(abc))
    cnt = np.zeros(len(abc), dtype=np.int64)
    _load().oracle_triangle_sums(N, len(thr) - 1, _p(thr, ctypes.c_int64), len(abc), _p(abc, ctypes.c_int32),
                                 w.shape[0], w.shape[1], _p(w, ctypes.c_double), len(c), _p(t, ctypes.c_int32),
                                 _p(c, ctypes.c_double), _p(out, ctypes.c_double), _p(cnt, ctypes.c_int64))
    with np.errstate(invalid="ignore", divide="ignore"):
        return out / cnt, cnt


def triangle_average_direct(N: int, L: float, edges, triplets, model):
    """Any model B(k1_vec, k2_vec, k3_vec) (physical wave vectors, arrays of
    shape (n, 3)) averaged over each triplet's closed ordered triangles by
    evaluating it on every triangle: the definition, for checking separable
    forms.  Small grids only.  Returns (average, N_tri)."""
    thr = thresholds(edges, L)
    kf = k_fundamental(L)
    f = np.fft.fftfreq(N, d=1.0 / N).astype(np.int64)
    g = np.stack(np.meshgrid(f, f, f, indexing="ij"), -1).reshape(-1, 3)
    b = bin_index(N, thr).ravel()
    out, cnt = [], []
    for a_, b_, c_ in np.asarray(triplets).reshape(-1, 3):
        m1 = g[b == a_]
        m2 = g[b == b_]
        p1 = np.repeat(m1, len(m2), axis=0)
        p2 = np.tile(m2, (len(m1), 1))
        m3 = -(p1 + p2)
        m3 = (m3 + N // 2) % N - N // 2  # wrapped into [-N/2, N/2)
        s3 = np.sum(m3 * m3, axis=1)
        in_c = (s3 >= thr[c_]) & (s3 < thr[c_ + 1])
        v = model(kf * p1[in_c], kf * p2[in_c], kf * m3[in_c])
        out.append(float(np.sum(v)) / max(1, int(in_c.sum())))
        cnt.append(int(in_c.sum()))
    return np.array(out), np.array(cnt, dtype=np.int64)


def power_spectrum(field, L: float, edges):
    """Power spectrum by direct measurement: P_b = V/N_pix^2 * <|D(m)|^2>
    over the modes of shell b (the textbook estimator the paper compares
    against in Sec. 3.3).  Empty shells give NaN.  Returns (P, |S_b|)."""
    field = np.asarray(field, dtype=np.float64)
    N = field.shape[0]
    thr = thresholds(edges, L)
    D = spectrum(field)
    b = bin_index(N, thr)
    nb = len(thr) - 1
    p2 = (D.real ** 2 + D.imag ** 2)
    sel = b >= 0
    s = np.bincount(b[sel].ravel(), weights=p2[sel].ravel(), minlength=nb)
    S = np.bincount(b[sel].ravel(), minlength=nb).astype(np.int64)
    V = float(L) ** 3
    npix = float(N) ** 3
    with np.errstate(invalid="ignore", divide="ignore"):
        P = (V / npix ** 2) * s / S
    P[S == 0] = np.nan
    return P, S


# --------------------------------------------------------------------------
# Route 2: the paper's FFT estimator in FP64 (Eqs. delta_nr .. Jeong_BI).
# --------------------------------------------------------------------------

def shell_field(D: np.ndarray, bins: np.ndarray, b: int) -> np.ndarray:
    """I_b(n) = sum_{m in S_b} D(m) e^{+2 pi i m.n/N} (Eq. delta_nr, first
    line): mask the spectrum to the shell and apply the unnormalised inverse
    DFT (NumPy's ifftn divides by N_pix, so multiply back)."""
    npix = D.size
    return (_ifftn(np.where(bins == b, D, 0.0)) * npix).real


def count_field(bins: np.ndarray, b: int) -> np.ndarray:
    """N_b(n) = sum_{m in S_b} e^{+2 pi i m.n/N} (Eq. delta_nr, second
    line): the unnormalised inverse DFT of the shell indicator."""
    npix = bins.size
    return (_ifftn((bins == b).astype(np.complex128)) * npix).real


def fft_estimator(field, L: float, edges, triplets=None, quads=None, bins_needed=None):
    """The paper's FFT polyspectrum estimator, FP64 NumPy, literal.

    Builds I_b and N_b for the bins in use, then
      P_b  = V/N_pix^2   sum_x I_b^2      / sum_x N_b^2          (Eq. Jeong_PS)
      B    = V^2/N_pix^3 sum_x I_a I_b I_c / sum_x N_a N_b N_c   (Eq. Jeong_BI)
      T    = V^3/N_pix^4 sum_x I_a I_b I_c I_d / sum_x N_a..N_d  (Eq. Jeong_gen)
    ``triplets`` / ``quads`` default to every a<=b<=c (a<=b<=c<=d) of
    non-empty bins.  Returns a dict with the sums, the counts rounded from
    sum N..N / N_pix, the estimates, ``M`` (the cancellation-free scale of
    each triplet, V^2/N_pix^3 sum_x |I_a I_b I_c| / sum_x N_a N_b N_c) and,
    for quadruplets, ``qM`` (the same with four fields and V^3/N_pix^4), and
    the connected trispectrum ``Tc`` = V^3/N_pix^4 (sum_x prod I / N_pix -
    paired sum) / N_conn, ``N_conn`` the unpaired quadruple count (see
    :func:`pairing_terms`), with its cancellation-free scale ``Tc_M``.
    """
    field = np.asarray(field, dtype=np.float64)
    N = field.shape[0]
    npix = float(N) ** 3
    V = float(L) ** 3
    thr = thresholds(edges, L)
    nb = len(thr) - 1
    D = spectrum(field)
    bins = bin_index(N, thr)
    S = np.bincount(bins[bins >= 0].ravel(), minlength=nb)
    use = set()
    if triplets is None:
        triplets = [(a, b, c) for a in range(nb) for b in range(a, nb) for c in range(b, nb)
                    if S[a] and S[b] and S[c]]
    for t in triplets:
        use.update(int(v) for v in t)
    if quads is not None:
        for q in quads:
            use.update(int(v) for v in q)
    if bins_needed is not None:
        use.update(int(v) for v in bins_needed)
    I, C = {}, {}
    for b in sorted(use):
        I[b] = shell_field(D, bins, b)
        C[b] = count_field(bins, b)
    out = {"bins": sorted(use)}
    P = np.full(nb, np.nan)
    for b in sorted(use):
        if S[b]:
            P[b] = (V / npix ** 2) * float(np.sum(I[b] * I[b])) / float(np.sum(C[b] * C[b]))
    out["P"] = P
    trip = np.asarray(triplets, dtype=np.int32).reshape(-1, 3)
    num = np.zeros(len(trip))
    den = np.zeros(len(trip))
    mag = np.zeros(len(trip))
    for i, (a, b, c) in enumerate(trip):
        prod = I[a] * I[b] * I[c]
        num[i] = float(np.sum(prod))
        mag[i] = float(np.sum(np.abs(prod)))
        den[i] = float(np.sum(C[a] * C[b] * C[c]))
    out["triplets"] = trip
    out["num"] = num
    out["den"] = den
    out["N_tri"] = np.rint(den / npix).astype(np.int64)
    with np.errstate(invalid="ignore", divide="ignore"):
        out["B"] = (V * V / npix ** 3) * num / den
        out["M"] = (V * V / npix ** 3) * mag / den
    if quads is not None:
        qd = np.asarray(quads, dtype=np.int32).reshape(-1, 4)
        qn = np.zeros(len(qd))
        qmag = np.zeros(len(qd))
        qden = np.zeros(len(qd))
        for i, (a, b, c, d) in enumerate(qd):
            prod = I[a] * I[b] * I[c] * I[d]
            qn[i] = float(np.sum(prod))
            qmag[i] = float(np.sum(np.abs(prod)))
            qden[i] = float(np.sum(C[a] * C[b] * C[c] * C[d]))
        out["quads"] = qd
        out["qnum"] = qn
        out["qden"] = qden
        # counts past 2^63 do not fit int64: there N_quad is the FP64 sum
        q = qden / npix
        out["N_quad"] = np.where(q < 9.2e18, np.rint(np.minimum(q, 9.2e18)), q).astype(np.float64)
        with np.errstate(invalid="ignore", divide="ignore"):
            out["T"] = (V ** 3 / npix ** 4) * qn / qden
            out["qM"] = (V ** 3 / npix ** 4) * qmag / qden
        # connected part: the sum of Eq. gen_Nspec4 over closed quadruples is
        # sum_x prod I / N_pix; remove the paired quadruples (pairing_terms)
        psum, pcnt = pairing_terms(D, bins, qd)
        out["pair_sum"], out["pair_cnt"] = psum, pcnt
        out["N_conn"] = qden / npix - pcnt
        with np.errstate(invalid="ignore", divide="ignore"):
            out["Tc"] = (V ** 3 / npix ** 4) * (qn / npix - psum) / out["N_conn"]
            out["Tc_M"] = (V ** 3 / npix ** 4) * qmag / npix / out["N_conn"]
    return out
