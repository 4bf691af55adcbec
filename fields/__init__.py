"""Seeded synthetic input fields for the FFT polyspectrum estimator.

This module only *synthesises* inputs: it holds none of the estimator's
arithmetic (no shell binning, no products, no normalisation).  Both the
CUDA library's tests/benchmarks and the FP64 oracle draw their inputs from
here, so that both sides see bit-identical fields.

All fields are generated on the host in FP64, C order ``[x][y][z]`` (x
slowest), on a periodic N^3 grid.  Random numbers come from
``numpy.random.default_rng(seed)`` (PCG64).

Workloads (they stand in for the paper's data, which is not available):

* ``lognormal``      -- delta = exp(g - sigma^2/2) - 1, g Gaussian with
                        P(k) ~ k^slope (a weakly/moderately non-Gaussian
                        density-like field; stands in for the N-body density
                        field of Sec. 3.2 of the paper).
* ``bubbles``        -- equal-radius ionised spheres at uniform random
                        centres with periodic wrap and overlap allowed, added
                        until the ionised fraction first reaches the target;
                        delta = x_HI/<x_HI> - 1 (the toy reionisation model of
                        Sec. 3.3 of the paper, the Bharadwaj & Ali picture).
* ``quadratic_local``-- delta = g + f (g^2 - <g^2>), g Gaussian with
                        P(k) ~ k^slope (closed-form tree-level bispectrum
                        2f[P1P2+P2P3+P3P1]).
* ``gaussian``       -- g alone (bispectrum null).
* ``plane_waves``    -- a finite sum of cosines on lattice wavevectors
                        (closed-form spectra for exact checks).
"""
from __future__ import annotations

import math

import numpy as np

try:  # multithreaded FFTs when scipy is present (it is on both machines)
    import scipy.fft as _fft

    def _rfftn(a):
        return _fft.rfftn(a, workers=-1)

    def _irfftn(a, shape):
        return _fft.irfftn(a, s=shape, workers=-1)
except Exception:  # pragma: no cover
    def _rfftn(a):
        return np.fft.rfftn(a)

    def _irfftn(a, shape):
        return np.fft.irfftn(a, s=shape)


def _kmag_half(N: int) -> np.ndarray:
    """|m| on the rfftn half grid, components in lattice units."""
    f = np.fft.fftfreq(N, d=1.0 / N)
    fz = np.arange(N // 2 + 1, dtype=np.float64)
    m2 = f[:, None, None] ** 2 + f[None, :, None] ** 2 + fz[None, None, :] ** 2
    return np.sqrt(m2)


def gaussian(N: int, slope: float, sigma: float, seed: int) -> np.ndarray:
    """Gaussian random field with P(k) proportional to k^slope, P(0) = 0.

    White standard normals in real space are coloured by sqrt(P(|m|)) in
    Fourier space, transformed back, and rescaled so that the grid rms is
    exactly ``sigma`` (the grid mean is zero because P(0) = 0).
    """
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((N, N, N))
    wk = _rfftn(w)
    k = _kmag_half(N)
    amp = np.zeros_like(k)
    nz = k > 0
    amp[nz] = k[nz] ** (0.5 * slope)
    g = _irfftn(wk * amp, (N, N, N))
    g -= g.mean()
    rms = math.sqrt(float(np.mean(g * g)))
    return g * (sigma / rms)


def lognormal(N: int, sigma: float = 0.5, slope: float = -2.0, seed: int = 0) -> np.ndarray:
    """delta = exp(g - sigma^2/2) - 1 with g = gaussian(N, slope, sigma, seed)."""
    g = gaussian(N, slope, sigma, seed)
    return np.exp(g - 0.5 * sigma * sigma) - 1.0


def quadratic_local(N: int, f: float = 0.3, slope: float = -1.5, sigma_g: float = 0.1,
                    seed: int = 2) -> np.ndarray:
    """delta = g + f (g^2 - <g^2>), g Gaussian with rms sigma_g, P ~ k^slope."""
    g = gaussian(N, slope, sigma_g, seed)
    g2 = g * g
    return g + f * (g2 - g2.mean())


def gaussian_spectrum_amplitude(N: int, slope: float, sigma: float, seed: int) -> float:
    """Amplitude A such that E|G(m)|^2 = A |m|^slope for ``gaussian(...)``.

    G is the unnormalised forward DFT of the generated field.  The white
    noise has E|W(m)|^2 = N^3; colouring multiplies by |m|^(slope/2) and the
    final rescale by sigma/rms_realised.  Returned for theory overlays of the
    quadratic-local test (the realised rescale is reproduced exactly).
    """
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((N, N, N))
    wk = _rfftn(w)
    k = _kmag_half(N)
    amp = np.zeros_like(k)
    nz = k > 0
    amp[nz] = k[nz] ** (0.5 * slope)
    g = _irfftn(wk * amp, (N, N, N))
    g -= g.mean()
    rms = math.sqrt(float(np.mean(g * g)))
    s = sigma / rms
    return float(N ** 3) * s * s


def bubbles(N: int, R: float = 6.0, x_ion: float = 0.5, seed: int = 1,
            return_count: bool = False):
    """Equal-radius ionised spheres, periodic wrap, overlap allowed.

    Bubble centres are uniform in [0, N)^3 (continuous).  A cell n (integer
    coordinates) is ionised when its minimum-image distance to a centre is
    <= R.  Bubbles are added one at a time until the ionised fraction first
    reaches ``x_ion``.  Returns delta = x_HI/<x_HI> - 1 (x_HI in {0, 1}).
    """
    if not (0.0 < x_ion < 1.0):
        raise ValueError("x_ion must lie in (0, 1)")
    rng = np.random.default_rng(seed)
    ion = np.zeros((N, N, N), dtype=bool)
    target = int(math.ceil(x_ion * N ** 3))
    n_ion = 0
    r = int(math.ceil(R)) + 1
    off = np.arange(-r, r + 1)
    nb = 0
    while n_ion < target:
        c = rng.uniform(0.0, N, size=3)
        base = np.floor(c).astype(np.int64)
        ix = base[0] + off
        iy = base[1] + off
        iz = base[2] + off
        dx = ix - c[0]
        dy = iy - c[1]
        dz = iz - c[2]
        d2 = dx[:, None, None] ** 2 + dy[None, :, None] ** 2 + dz[None, None, :] ** 2
        sel = d2 <= R * R
        gx, gy, gz = np.nonzero(sel)
        xs = np.mod(ix[gx], N)
        ys = np.mod(iy[gy], N)
        zs = np.mod(iz[gz], N)
        newly = ~ion[xs, ys, zs]
        n_ion += int(np.count_nonzero(newly))
        ion[xs, ys, zs] = True
        nb += 1
    xhi = (~ion).astype(np.float64)
    delta = xhi / xhi.mean() - 1.0
    if return_count:
        return delta, nb
    return delta


def plane_waves(N: int, waves) -> np.ndarray:
    """delta(n) = sum_j A_j cos(2 pi m_j . n / N + phi_j).

    ``waves`` is a sequence of ``((mx, my, mz), A, phi)`` with integer m.
    For m_j != 0 and 2 m_j != 0 (mod N) the unnormalised DFT of one wave is
    (N^3 A/2) e^{+i phi} at +m_j and (N^3 A/2) e^{-i phi} at -m_j.
    """
    n = np.arange(N, dtype=np.float64)
    out = np.zeros((N, N, N))
    for (m, A, phi) in waves:
        ph = (2.0 * math.pi / N) * (m[0] * n[:, None, None] + m[1] * n[None, :, None]
                                    + m[2] * n[None, None, :])
        out += A * np.cos(ph + phi)
    return out


def linear_edges(N: int, L: float, nbins: int) -> np.ndarray:
    """``nbins`` linear bins from k_f to k_Ny/2 = N k_f/4 (physical k units)."""
    kf = 2.0 * math.pi / L
    return np.linspace(kf, 0.25 * N * kf, nbins + 1)


def log_edges(N: int, L: float, nbins: int) -> np.ndarray:
    """``nbins`` log-spaced bins from k_f to k_Ny/2 = N k_f/4."""
    kf = 2.0 * math.pi / L
    return np.geomspace(kf, 0.25 * N * kf, nbins + 1)
