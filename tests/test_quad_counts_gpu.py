"""Exact ordered quadruple counts of the library (128-bit integers from
pair-count convolutions on the level grids) against the oracle's integer
pair-count route, itself pinned to brute force: every closed quadruplet and
no other, on single- and multi-level plans and on wrapped plans."""
import itertools

import numpy as np
import pytest

import fields
import oracle
import paper_1705_06284_gb300 as fbs

pytestmark = pytest.mark.gpu

CASES = [(16, 50.0, "lin", 4, False), (24, 60.0, "log", 6, False), (32, 100.0, "lin", 5, False),
         (12, 7.0, "wrapped", 4, True)]


def _edges(N, L, kind, nb):
    if kind == "lin":
        return fields.linear_edges(N, L, nb)
    if kind == "log":
        return fields.log_edges(N, L, nb)
    kf = 2 * np.pi / L
    return np.linspace(kf, 0.45 * N * kf, nb + 1)


def _check(plan, N, L, edges):
    nb = len(edges) - 1
    shell = plan.shell
    cand = [q for q in itertools.combinations_with_replacement(range(nb), 4) if all(shell[b] > 0 for b in q)]
    ex = oracle.quad_counts_exact(N, L, edges, cand)
    closed = [(q, v) for q, v in zip(cand, ex) if v > 0]
    assert [tuple(int(b) for b in q) for q in plan.quads] == [q for q, _ in closed]
    assert plan.N_quad_exact == [v for _, v in closed]
    assert plan.quad_counts_exact
    assert np.array_equal(plan.N_quad, np.array([float(v) for _, v in closed]))


@pytest.mark.parametrize("N,L,kind,nb,wrapped", CASES)
def test_exact_quad_counts_match_oracle(N, L, kind, nb, wrapped):
    edges = _edges(N, L, kind, nb)
    with fbs.Plan(N, L, edges, precision="fp32", trispectrum=True, allow_aliased=wrapped) as plan:
        _check(plan, N, L, edges)


def test_exact_quad_counts_on_levels(monkeypatch):
    monkeypatch.setenv("FBS_LEVEL_COST", "-1e15")
    monkeypatch.setenv("FBS_MIN_LEVEL_GRID", "0")
    N, L = 48, 60.0
    edges = fields.log_edges(N, L, 8)
    with fbs.Plan(N, L, edges, precision="bf16x3", trispectrum=True) as plan:
        assert len(set(plan.quad_level.tolist())) >= 2
        _check(plan, N, L, edges)


def test_exact_quad_counts_survive_export(monkeypatch):
    N, L = 24, 60.0
    edges = fields.log_edges(N, L, 6)
    with fbs.Plan(N, L, edges, precision="fp32", trispectrum=True) as a:
        blob = a.export_counts()
        with fbs.Plan(N, L, edges, precision="fp32", trispectrum=True, counts=blob) as b:
            assert b.N_quad_exact == a.N_quad_exact
            assert np.array_equal(b.N_conn, a.N_conn)
