"""Host logic of the evaluation levels, on CPU.

A plan sums each item's product of shell fields on a grid M above the
product's degree R_a + R_b + R_c (+ R_d) and above 2 R of each of its bins;
it groups the items into a few such grids by a work model.  The C++ unit
(levels.cpp) is compiled with the host compiler into a small driver; the
checks are the properties the device path relies on: every item on a grid it
fits (the smallest chosen one), every bin of an item evaluated on that item's
level, every level's grid above twice its bins' largest component, every
non-empty bin's power spectrum taken from exactly one level that evaluates it,
and the grids few and ascending.  At the 512^3 bin layouts the chosen levels
must also cut the model's point work well below one grid for all.
"""
import itertools
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from test_pair_cover_cpu import _shell_sizes

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1705_06284_gb300", "csrc")

DRIVER = r'''
#include <cstdio>
#include "levels.h"
int main() {
    int N, nb, maxl, single, nfast, n;
    if (scanf("%d %d %d %d", &N, &nb, &maxl, &single) != 4) return 2;
    std::vector<int> R(nb);
    for (auto &r : R) if (scanf("%d", &r) != 1) return 2;
    if (scanf("%d", &nfast) != 1) return 2;
    std::vector<int> fast(nfast);
    for (auto &f : fast) if (scanf("%d", &f) != 1) return 2;
    if (scanf("%d", &n) != 1) return 2;
    std::vector<fbs::LevelItem> items(n);
    for (auto &it : items)
        if (scanf("%d %d %d %d %d %d", &it.arity, &it.b[0], &it.b[1], &it.b[2], &it.b[3], &it.need) != 6) return 2;
    fbs::LevelChoice c = fbs::choose_levels(N, nb, R, items, single, fast, maxl);
    printf("%zu\n", c.grids.size());
    for (int g : c.grids) printf("%d ", g);
    printf("\n");
    for (int l : c.item_level) printf("%d ", l);
    printf("\n");
    for (int l : c.bin_level) printf("%d ", l);
    printf("\n");
    for (auto &bs : c.bins) {
        printf("%zu", bs.size());
        for (int b : bs) printf(" %d", b);
        printf("\n");
    }
    return 0;
}
'''

FAST = [64, 72, 96, 108, 128, 144, 192, 216, 256, 288, 384, 512]


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("levels")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), os.path.join(CSRC, "levels.cpp"),
                    "-o", str(exe)], check=True, capture_output=True, text=True)
    return str(exe)


def _admissible(N):
    out = []
    for M in range(8, N + 1, 2):
        m = M
        while m % 2 == 0:
            m //= 2
        while m % 3 == 0:
            m //= 3
        if m == 1:
            out.append(M)
    return out


def _layout(N, L, nb, quads, log=True):
    kf = 2 * math.pi / L
    e = np.geomspace(kf, 0.25 * N * kf, nb + 1) if log else np.linspace(kf, 0.25 * N * kf, nb + 1)
    thr = oracle.thresholds(e, L)
    sizes = _shell_sizes(thr)
    R = [min(math.isqrt(int(thr[b + 1]) - 1), N // 2) if sizes[b] else -1 for b in range(nb)]
    lo = np.sqrt(thr[:-1].astype(float))
    hi = np.sqrt(np.maximum(thr[1:].astype(float) - 1, 0))
    ok = [b for b in range(nb) if sizes[b]]
    items = [t for t in itertools.combinations_with_replacement(ok, 3) if hi[t[0]] + hi[t[1]] >= lo[t[2]] - 1e-9]
    if quads:
        items += [q for q in itertools.combinations_with_replacement(ok, 4)
                  if hi[q[0]] + hi[q[1]] + hi[q[2]] >= lo[q[3]] - 1e-9]
    adm = _admissible(N)

    def need(t):
        s = max(sum(R[b] for b in t), 2 * max(R[b] for b in t))
        return next((M for M in adm if M > s), N)
    return R, items, [need(t) for t in items]


def _choose(exe, N, R, items, needs, maxl=4, single=0, fast=FAST):
    text = "%d %d %d %d\n%s\n%d %s\n%d\n" % (N, len(R), maxl, single, " ".join(map(str, R)), len(fast),
                                             " ".join(map(str, fast)), len(items))
    text += "".join("%d %s %d\n" % (len(t), " ".join(map(str, list(t) + [0] * (4 - len(t)))), n)
                    for t, n in zip(items, needs))
    r = subprocess.run([exe], input=text, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.strip().split("\n")
    ng = int(lines[0])
    grids = [int(v) for v in lines[1].split()]
    item_level = [int(v) for v in lines[2].split()] if items else []
    k = 3 if items else 2
    bin_level = [int(v) for v in lines[k].split()]
    bins = [[int(v) for v in ln.split()[1:]] for ln in lines[k + 1:k + 1 + ng]]
    return grids, item_level, bin_level, bins


def _check(N, R, items, needs, grids, item_level, bin_level, bins, maxl):
    assert grids == sorted(set(grids)) and all(8 <= g <= N for g in grids)
    assert len(grids) <= maxl + sum(1 for r in R if r >= 0)  # P-only levels are extra
    for t, n, l in zip(items, needs, item_level):
        assert grids[l] >= n                       # the item fits its level's grid
        assert l == 0 or grids[l - 1] < n          # ... the smallest chosen one
        assert set(t) <= set(bins[l])              # its bins are evaluated there
    for l, bs in enumerate(bins):
        assert bs == sorted(set(bs))
        for b in bs:
            assert R[b] >= 0 and grids[l] > 2 * R[b]
    for b, r in enumerate(R):
        if r < 0:
            assert bin_level[b] == -1
        else:
            assert b in bins[bin_level[b]]


def _model(grids, item_level, items, bins, R):
    """Points x (bins + pairs) of the chosen levels, the quantity the model weighs."""
    tot = 0.0
    for l, M in enumerate(grids):
        its = [t for t, lv in zip(items, item_level) if lv == l]
        pairs = {t[-2:] for t in its}
        tot += M ** 3 * (4 * len(bins[l]) + 0.7 * len(pairs) + len(bins[l]))
    return tot


@pytest.mark.parametrize("nb,quads,minlev", [(64, False, 2), (16, True, 1)])
def test_levels_at_512_layouts(driver, nb, quads, minlev):
    N = 512
    R, items, needs = _layout(N, 1000.0, nb, quads)
    grids, il, bl, bins = _choose(driver, N, R, items, needs)
    _check(N, R, items, needs, grids, il, bl, bins, 4)
    assert minlev <= len(grids) <= 4
    one = _choose(driver, N, R, items, needs, maxl=1)
    _check(N, R, items, needs, *one, 1)
    assert len(one[0]) == 1
    if minlev > 1:
        # the 64-bin triplets: far less point work than one grid for every item
        # (the 16-bin trispectrum layout keeps one grid: a full tile per point
        # at every level would cost more than it saves)
        assert _model(grids, il, items, bins, R) < 0.6 * _model(*one[:2], items, one[3], R)
    assert (grids, il) == _choose(driver, N, R, items, needs)[:2]  # deterministic


def test_single_grid_and_linear_bins(driver):
    N = 256
    R, items, needs = _layout(N, 256.0, 32, False, log=False)
    grids, il, bl, bins = _choose(driver, N, R, items, needs, single=192)
    assert grids == [192] and set(il) == {0}
    _check(N, R, items, [192] * len(items), grids, il, bl, bins, 1)
    grids, il, bl, bins = _choose(driver, N, R, items, needs)
    _check(N, R, items, needs, grids, il, bl, bins, 4)


def test_bins_without_items_get_a_level(driver):
    # bin 3 is in no item; bin 4 (R = 60) needs a grid above 120, above every item's
    N = 256
    R = [2, 3, 5, 8, 60]
    items = [(0, 0, 1), (0, 1, 2), (1, 1, 2)]
    adm = _admissible(N)
    needs = [next(M for M in adm if M > max(sum(R[b] for b in t), 2 * max(R[b] for b in t))) for t in items]
    grids, il, bl, bins = _choose(driver, N, R, items, needs)
    _check(N, R, items, needs, grids, il, bl, bins, 4)
    assert grids[bl[4]] > 120 and grids[bl[3]] > 16
    R2 = [2, -1, 5]  # an empty bin gets no level
    grids, il, bl, bins = _choose(driver, N, R2, [(0, 0, 2)], [16])
    assert bl[1] == -1


def test_random_layouts(driver):
    rng = np.random.default_rng(5)
    for trial in range(20):
        N = int(rng.choice([64, 96, 128, 192, 256]))
        nb = int(rng.integers(3, 12))
        R = sorted(int(v) for v in rng.integers(1, N // 4, size=nb))
        R = [r if rng.random() > 0.1 else -1 for r in R]
        ok = [b for b in range(nb) if R[b] >= 0]
        items = [t for t in itertools.combinations_with_replacement(ok, 3) if rng.random() < 0.5]
        adm = _admissible(N)
        needs = [next((M for M in adm if M > max(sum(R[b] for b in t), 2 * max(R[b] for b in t))), N)
                 for t in items]
        maxl = int(rng.integers(1, 5))
        grids, il, bl, bins = _choose(driver, N, R, items, needs, maxl=maxl)
        _check(N, R, items, needs, grids, il, bl, bins, maxl)
