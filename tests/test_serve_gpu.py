"""Serving loop: requests of mixed grid sizes and bin sets overlap on the
device, and every result is the same alone and in the mix (the kernels use
fixed reduction orders, so "the same" is bit-identical here)."""
import math

import numpy as np
import pytest

import fields
import oracle
import paper_1705_06284_gb300 as fbs
from paper_1705_06284_gb300.serve import EstimatorServer, Request, latency_percentiles

pytestmark = pytest.mark.gpu


def _requests(n, seed=0):
    rng = np.random.default_rng(seed)
    pool = {N: [fields.lognormal(N, 0.6, -1.5, seed=10 + N).astype(np.float32),
                fields.bubbles(N, max(1.5, N / 10), 0.4, seed=20 + N).astype(np.float32)]
            for N in (16, 24, 32)}
    reqs = []
    for i in range(n):
        N = int(rng.choice([16, 24, 32]))
        nb = int(rng.integers(3, 9))
        L = 50.0
        edges = tuple(fields.linear_edges(N, L, nb))
        reqs.append(Request(i, pool[N][i % 2], L, edges, arrival=0.002 * i,
                            precision=str(rng.choice(["fp32", "bf16x3"]))))
    return reqs


def test_mix_equals_alone():
    reqs = _requests(14)
    srv = EstimatorServer(hbm_budget=8 << 30, slots=3)
    try:
        mixed = srv.run(reqs, realtime=True)
    finally:
        srv.close()
    assert [r.rid for r in mixed] == list(range(len(reqs)))
    for req, res in zip(reqs, mixed):
        one = EstimatorServer(hbm_budget=8 << 30, slots=1)
        try:
            alone = one.run([Request(req.rid, req.field, req.L, req.edges, 0.0, req.precision)],
                            realtime=False)[0]
        finally:
            one.close()
        assert np.array_equal(res.triplets, alone.triplets)
        assert np.array_equal(res.B, alone.B), req.rid
        assert np.array_equal(res.P, alone.P, equal_nan=True)
    lat = latency_percentiles(mixed)
    assert lat["p99_ms"] >= lat["p50_ms"] > 0
    # and one of them against the oracle
    r0, q0 = mixed[0], reqs[0]
    ref = oracle.direct_bispectrum(q0.field.astype(np.float64), q0.L, q0.edges)
    assert np.array_equal(r0.N_tri, ref["N_tri"])


def test_tight_budget_waits_and_evicts():
    reqs = _requests(8, seed=3)
    srv = EstimatorServer(hbm_budget=1 << 30, slots=2)
    try:
        res = srv.run(reqs, realtime=False)
    finally:
        srv.close()
    assert len(res) == len(reqs)
    assert srv.held == 0
