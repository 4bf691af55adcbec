"""Shared helpers of the GPU parity tests (no estimator arithmetic here)."""
import numpy as np

import oracle

# Tolerances (on triplets with N_tri >= 100 and |B| >= 1e-3 of the
# cancellation-free scale M): FP32 1e-4 relative, BF16x3 2e-4 relative.
TOL = {"fp32": 1e-4, "bf16x3": 2e-4}


def run(plan, field32, device=True):
    import torch
    if device:
        f = torch.from_numpy(field32).cuda()
        B, P = plan.bispectrum(f)
        torch.cuda.synchronize()
        return B.cpu().numpy(), P.cpu().numpy()
    return plan.bispectrum(field32)


def gate_mask(ref_B, ref_M, ntri):
    return (ntri >= 100) & (np.abs(ref_B) >= 1e-3 * ref_M)


def rel_err(got, ref):
    return np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)


def check_bispectrum(plan, B, P, field32, L, edges, precision, ref=None, M=None):
    """Compare a plan's output with the direct oracle (exact counts, gated B).

    Returns (max gated rel err, max rel err over all triplets, n gated)."""
    f64 = field32.astype(np.float64)
    if ref is None:
        ref = oracle.direct_bispectrum(f64, L, edges)
    assert np.array_equal(plan.triplets, ref["triplets"]), "closed-triplet set differs"
    assert np.array_equal(plan.N_tri, ref["N_tri"]), "triangle counts differ"
    assert np.array_equal(plan.shell, ref["shell"]), "shell sizes differ"
    if M is None:
        M = oracle.fft_estimator(f64, L, edges, triplets=ref["triplets"])["M"]
    g = gate_mask(ref["B"], M, ref["N_tri"])
    r = rel_err(B, ref["B"])
    ok = np.isfinite(ref["P"])
    assert np.array_equal(np.isnan(P), ~ok), "empty-shell NaN pattern differs"
    assert np.all(rel_err(P[ok], ref["P"][ok]) < TOL.get(precision, 1e-4)), "P mismatch"
    gmax = float(r[g].max()) if g.any() else 0.0
    if precision in TOL:
        assert gmax < TOL[precision], ("B mismatch", gmax, int(np.argmax(np.where(g, r, 0))))
    return gmax, float(r.max()) if len(r) else 0.0, int(g.sum())


def check_trispectrum(plan, T, field32, L, edges, tol):
    """T against the FP64 FFT estimator on quadruplets with N_quad >= 100 and
    |T| >= 1e-3 of the cancellation-free scale sum_x |I_a I_b I_c I_d|.
    Returns (max gated rel err, n gated)."""
    f64 = field32.astype(np.float64)
    g = oracle.fft_estimator(f64, L, edges, triplets=[], quads=plan.quads)
    assert np.array_equal(plan.N_quad, g["N_quad"])
    N = field32.shape[0]
    D = oracle.spectrum(f64)
    bins = oracle.bin_index(N, oracle.thresholds(edges, L))
    I = {b: oracle.shell_field(D, bins, b) for b in set(plan.quads.ravel().tolist())}
    mag = np.array([np.sum(np.abs(I[a] * I[b] * I[c] * I[d])) for a, b, c, d in plan.quads])
    keep = (plan.N_quad >= 100) & (np.abs(g["qnum"]) >= 1e-3 * mag)
    r = rel_err(T, g["T"])
    assert keep.sum() > 0
    assert np.all(r[keep] < tol), float(r[keep].max())
    return float(r[keep].max()), int(keep.sum())
