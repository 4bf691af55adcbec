"""Write the stored oracle results used by the tests.

Calls only ``oracle`` and ``fields``.  The paper prints no numeric worked
example (its accuracy results are figures only), so every stored value here
is the FP64 oracle's, on the seeded synthetic workload named in the file.

Run from the repository root:  python tests/golden/make_golden.py
"""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import fields  # noqa: E402
import oracle  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def lognormal32():
    """32^3 lognormal (sigma 0.5, P ~ k^-2, seed 0), L = 100, 6 linear bins
    from k_f to k_Ny/2.  The field is rounded to FP32 first: that is what
    the GPU library receives."""
    N, L = 32, 100.0
    f = fields.lognormal(N, 0.5, -2.0, seed=0).astype(np.float32).astype(np.float64)
    edges = fields.linear_edges(N, L, 6)
    d = oracle.direct_bispectrum(f, L, edges)
    g = oracle.fft_estimator(f, L, edges, triplets=d["triplets"])
    path = os.path.join(HERE, "lognormal32_lin6.txt")
    with open(path, "w") as fh:
        fh.write("# FP64 direct-measurement oracle (Eq. bi_direct, full shells) on the 32^3\n")
        fh.write("# lognormal field: sigma=0.5, P~k^-2, seed 0, FP32-rounded; L=100; 6 linear\n")
        fh.write("# bins from k_f to N k_f/4.  Written by tests/golden/make_golden.py.\n")
        fh.write("# edges " + " ".join(repr(float(e)) for e in edges) + "\n")
        fh.write("# P " + " ".join(repr(float(p)) for p in d["P"]) + "\n")
        fh.write("# shell " + " ".join(str(int(s)) for s in d["shell"]) + "\n")
        fh.write("# a b c N_tri B M\n")
        for t, n, B, M in zip(d["triplets"], d["N_tri"], d["B"], g["M"]):
            fh.write("%d %d %d %d %r %r\n" % (t[0], t[1], t[2], n, float(B), float(M)))
    return path


if __name__ == "__main__":
    print(lognormal32())
