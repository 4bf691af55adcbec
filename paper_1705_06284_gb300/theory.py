"""Theory averaged over the exact triangles of each bin triplet.

The paper compares its FFT measurements with theory evaluated on every
triangle that contributes to a bin and averaged over them (Sec. 3.3): for the
oscillatory window of the bubble model the average differs strongly from the
theory at the bin centre.  Every model here is a sum of separable terms
coef * f1(|k1|) f2(|k2|) f3(|k3|), and ``Plan.triangle_average`` (the C ABI's
fbs_plan_triangle_average) averages such sums over the ordered closed
triangles of each of the plan's triplets on the GPU, in FP64, with the
Kronecker-delta identity of Sec. 2 (weighted count fields, no enumeration).
This module only builds the tables and terms.

Models:
* ``local``: delta = g + f (g^2 - <g^2>), tree level 2 f [P1 P2 + P2 P3 + P3 P1].
* ``bubbles``: equal-radius ionised spheres (Eq. BharBk),
  B = -(1 - x_HI)^3 W(k1 R) W(k2 R) W(k3 R) / n^2 with (1 - x_HI) = (4 pi R^3/3) n
  and W the Fourier transform of the spherical top hat.
* ``tree_level``: Eq. PT_Bi, B = 2 F(k1, k2) P1 P2 + cyc with
  F = (1 + kappa)/2 + (k1.k2 / (2 k1 k2)) (k1/k2 + k2/k1)
      + ((1 - kappa)/2) (k1.k2 / (k1 k2))^2.
  On a closed triangle k1.k2 = (k3^2 - k1^2 - k2^2)/2, so with u = k^2 and
  Q = P/u each cyclic term 2 F(x, y) P_x P_y (z the third side) is
      (1 + kappa)/2  P_x P_y            + kappa/2 (P_x Q_y + Q_x P_y) u_z
    - (1 + kappa)/4 (P_x u_x Q_y + Q_x P_y u_y) + (1 - kappa)/4 Q_x Q_y u_z^2.
"""
from __future__ import annotations

import math

import numpy as np


def _k_of_s(plan):
    """Physical k at every integer |m|^2 below the plan's top threshold."""
    nw = int(plan.thresholds[-1])
    kf = 2 * math.pi / plan.L
    return kf * np.sqrt(np.arange(max(nw, 1), dtype=np.float64))


def tophat_window(y):
    """Fourier transform of the unit spherical top hat, W(0) = 1."""
    y = np.asarray(y, dtype=np.float64)
    out = np.ones_like(y)
    nz = np.abs(y) > 1e-6
    yy = y[nz]
    out[nz] = 3.0 * (np.sin(yy) - yy * np.cos(yy)) / yy ** 3
    small = ~nz
    out[small] = 1.0 - y[small] ** 2 / 10.0
    return out


def local(plan, Pk, f):
    """Bin-averaged tree-level bispectrum of a local quadratic field,
    2 f [P1 P2 + P2 P3 + P3 P1]; Pk: callable of physical k (0 at k = 0)."""
    k = _k_of_s(plan)
    P = np.where(k > 0, Pk(np.where(k > 0, k, 1.0)), 0.0)
    tables = np.stack([P, np.ones_like(P)])
    terms = [(0, 0, 1), (1, 0, 0), (0, 1, 0)]
    return plan.triangle_average(tables, terms, [2.0 * f] * 3)


def bubbles(plan, R, x_HI):
    """Bin-averaged bispectrum of equal-radius ionised spheres (Eq. BharBk) of
    radius R (physical length units) at neutral fraction x_HI."""
    k = _k_of_s(plan)
    n = (1.0 - x_HI) / (4.0 * math.pi * R ** 3 / 3.0)
    W = tophat_window(k * R)
    return plan.triangle_average(W[None, :], [(0, 0, 0)], [-(1.0 - x_HI) ** 3 / n ** 2])


def bubbles_power(plan, R, x_HI):
    """Shell-averaged power spectrum of the same model (Eq. BharPk),
    (1 - x_HI)^2 W^2(kR) / n, averaged over every mode of each bin
    (NaN for empty bins)."""
    k = _k_of_s(plan)
    n = (1.0 - x_HI) / (4.0 * math.pi * R ** 3 / 3.0)
    return plan.shell_average((1.0 - x_HI) ** 2 * tophat_window(k * R) ** 2 / n)


def tree_level(plan, Pk, kappa=3.0 / 7.0):
    """Bin-averaged tree-level perturbation-theory bispectrum (Eq. PT_Bi);
    Pk: the linear power spectrum, callable of physical k; kappa = 3/7
    Omega_m^(-1/143) for LCDM."""
    k = _k_of_s(plan)
    u = k * k
    pos = k > 0
    P = np.where(pos, Pk(np.where(pos, k, 1.0)), 0.0)
    Q = np.where(pos, P / np.where(pos, u, 1.0), 0.0)
    ONE, U, U2, PU = np.ones_like(u), u, u * u, P * u
    tables = np.stack([P, Q, U, PU, U2, ONE])
    iP, iQ, iU, iPU, iU2, i1 = range(6)
    # 2 F(x, y) P_x P_y as (f_x, f_y, f_z, coefficient)
    one = [(iP, iP, i1, (1 + kappa) / 2), (iP, iQ, iU, kappa / 2), (iQ, iP, iU, kappa / 2),
           (iPU, iQ, i1, -(1 + kappa) / 4), (iQ, iPU, i1, -(1 + kappa) / 4), (iQ, iQ, iU2, (1 - kappa) / 4)]
    terms, coef = [], []
    # the three cyclic terms: (x, y, z) = (k1, k2, k3), (k2, k3, k1), (k3, k1, k2)
    for cyc in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        for fx, fy, fz, c in one:
            t = [0, 0, 0]
            t[cyc[0]], t[cyc[1]], t[cyc[2]] = fx, fy, fz
            terms.append(tuple(t))
            coef.append(c)
    return plan.triangle_average(tables, terms, coef)
