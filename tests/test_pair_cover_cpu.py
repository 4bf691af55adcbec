"""Host logic of the tensor-core contraction, on CPU: the greedy pair covers
that choose which pair product carries each triplet, and which pairing (and
which pair as the inner row) carries each quadruplet.  The C++ unit is
compiled with the host compiler into a small driver; the checks are the
properties the device code relies on (every item carried by one of its own
pairs, distinct (outer, inner) slots, the outer set within one tile) and
the reduction in outer / inner rows at the 512^3 workloads' bin layouts."""
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

import fields
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1705_06284_gb300", "csrc")

DRIVER = r'''
#include <cstdio>
#include "pair_cover.h"
int main() {
    char mode; int nb, n;
    if (scanf(" %c %d %d", &mode, &nb, &n) != 3) return 2;
    if (mode == 'T') {
        std::vector<std::array<int, 3>> t(n);
        for (auto &x : t) if (scanf("%d %d %d", &x[0], &x[1], &x[2]) != 3) return 2;
        for (int k : fbs::cover_triplet_pairs(nb, t)) printf("%d\n", k);
        return 0;
    }
    int nf; if (scanf("%d", &nf) != 1) return 2;
    std::vector<std::array<int, 4>> q(n);
    for (auto &x : q) if (scanf("%d %d %d %d", &x[0], &x[1], &x[2], &x[3]) != 4) return 2;
    std::vector<int> fixed(nf);
    for (auto &f : fixed) if (scanf("%d", &f) != 1) return 2;
    std::vector<std::pair<int, int>> a;
    const bool ok = fbs::cover_quad_pairings(nb, q, fixed, a);
    printf("%d\n", ok ? 1 : 0);
    if (ok) for (auto &p : a) printf("%d %d\n", p.first, p.second);
    return 0;
}
'''


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("cover")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), os.path.join(CSRC, "pair_cover.cpp"),
                    "-o", str(exe)], check=True, capture_output=True, text=True)
    return str(exe)


def _run(exe, text):
    r = subprocess.run([exe], input=text, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    return r.stdout.split()


def _shell_sizes(thr):
    """|S_b| for thresholds below (N/2)^2: for every (x, y) count the integers
    z with thr[b] <= x^2 + y^2 + z^2 < thr[b+1] (O(R^2), no N^3 arrays)."""
    top = int(thr[-1])
    R = int(np.ceil(np.sqrt(top)))
    r2 = (np.arange(-R, R + 1)[:, None] ** 2 + np.arange(-R, R + 1)[None, :] ** 2).ravel()

    def below(t):  # number of (x, y, z) with x^2 + y^2 + z^2 < t
        rem = t - r2
        ok = rem > 0
        zmax = np.floor(np.sqrt(np.maximum(rem - 1, 0))).astype(np.int64)  # z^2 <= rem - 1
        return int(np.sum(np.where(ok, 2 * zmax + 1, 0)))
    c = [below(int(t)) for t in thr]
    return np.diff(c)


def _interval_sets(N, L, nb):
    e = fields.log_edges(N, L, nb)
    thr = oracle.thresholds(e, L)
    lo = np.sqrt(thr[:-1].astype(float))
    hi = np.sqrt(np.maximum(thr[1:].astype(float) - 1, 0))
    sizes = _shell_sizes(thr)
    ok = [b for b in range(nb) if sizes[b] > 0]
    trips = [t for t in itertools.combinations_with_replacement(ok, 3) if hi[t[0]] + hi[t[1]] >= lo[t[2]]]
    quads = [q for q in itertools.combinations_with_replacement(ok, 4)
             if hi[q[0]] + hi[q[1]] + hi[q[2]] >= lo[q[3]]]
    return trips, quads


def _cover_trips(exe, nb, trips):
    text = "T %d %d\n" % (nb, len(trips)) + "".join("%d %d %d\n" % t for t in trips)
    return [int(k) for k in _run(exe, text)]


def test_triplet_cover_valid_and_smaller(driver):
    nb = 64
    trips, _ = _interval_sets(512, 1000.0, nb)
    keys = _cover_trips(driver, nb, trips)
    assert len(keys) == len(trips)
    slots = set()
    for (a, b, c), k in zip(trips, keys):
        x, y = divmod(k, nb)
        assert (x, y) in {(a, b), (a, c), (b, c)}
        rest = [a, b, c]
        rest.remove(x)
        rest.remove(y)
        assert (k, rest[0]) not in slots  # one item per (outer pair, inner bin)
        slots.add((k, rest[0]))
    bc = {(b, c) for a, b, c in trips}
    assert len(set(keys)) <= 0.75 * len(bc)  # 378 instead of 546 pairs at this layout
    assert keys == _cover_trips(driver, nb, trips)  # deterministic


def test_triplet_cover_tiny_random(driver):
    rng = np.random.default_rng(3)
    nb = 7
    all_t = list(itertools.combinations_with_replacement(range(nb), 3))
    trips = [all_t[i] for i in sorted(rng.choice(len(all_t), 40, replace=False))]
    keys = _cover_trips(driver, nb, trips)
    for (a, b, c), k in zip(trips, keys):
        assert divmod(k, nb) in {(a, b), (a, c), (b, c)}


def test_quadruplet_cover_valid_within_one_tile(driver):
    nb = 16
    trips, quads = _interval_sets(512, 1000.0, nb)
    fixed = sorted({b * nb + c for a, b, c in trips})
    text = "Q %d %d %d\n" % (nb, len(quads), len(fixed)) + "".join("%d %d %d %d\n" % q for q in quads) + \
        " ".join(map(str, fixed)) + "\n"
    out = _run(driver, text)
    assert out[0] == "1"
    pairs = [(int(out[1 + 2 * i]), int(out[2 + 2 * i])) for i in range(len(quads))]
    slots = set()
    for (a, b, c, d), (inner, outer) in zip(quads, pairs):
        ip, op = divmod(inner, nb), divmod(outer, nb)
        assert ip[0] <= ip[1] and op[0] <= op[1]
        assert sorted(ip + op) == [a, b, c, d]
        assert (outer, inner) not in slots
        slots.add((outer, inner))
    outer_rows = {o for _, o in pairs} | set(fixed)
    assert len(outer_rows) <= 128
    inner_rows = {i for i, _ in pairs}
    assert len(inner_rows) <= 64  # 50 instead of 136 inner pairs at this layout
