"""Batched estimation of many realisations with uneven grid sizes.

Realisations are grouped by grid size, each group evaluated by one batched
library call (fbs_bispectrum_batch: one launch per stage for all of the
group's fields), and those calls are captured into one CUDA graph and
replayed: the host issues a single launch for the whole batch.  Every kernel
is the library's; this module only groups, captures and replays.  An autotuner picks, per plan, the contraction's
orientation, pipeline step, pair assignment, warp roles and slab size that
run fastest on the plan's own problem, and caches the choice.
"""
from __future__ import annotations

import json
import os
import time
from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import Plan

_TUNE_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


_BUILD_ID = None


def _build_id():
    """Library build (hash of libfbs.so) and device name: a choice timed on
    another build or another GPU model is not reused."""
    global _BUILD_ID
    if _BUILD_ID is None:
        import hashlib
        import torch
        from ._build import LIB
        h = hashlib.sha1(open(LIB, "rb").read()).hexdigest()[:16]
        _BUILD_ID = "%s|%s" % (h, torch.cuda.get_device_name())
    return _BUILD_ID


def _key(N, L, edges, precision):
    return "%d|%r|%s|%s|%s" % (N, float(L), ",".join("%.12g" % e for e in edges), precision, _build_id())


# Tunable options of a plan (fbs_plan_set_option) and the values tried; the
# first value of each is the library's default.
TUNABLE = (
    ("chunk", 3, (0, 1)),       # FBS_OPT_TC_CHUNK: 128-point steps where they fit / 64-point steps
    ("pairs", 4, (0, 1)),       # FBS_OPT_TC_PAIRS: greedy pair cover / plain (b, c) pairs
    ("wide", 1, (0, 1)),        # FBS_OPT_TC_WIDE: pair products on M / stacked left rows on M
    ("roles", 2, (0, 2)),       # FBS_OPT_TC_ROLES: 16 product warps / 8 + 8 concurrent roles
    ("slab", 6, (0, 32, 8)),    # FBS_OPT_SLAB_PLANES: planned slabs / at most 32 or 8 planes
    ("merge", 7, (0, 1)),       # FBS_OPT_TC_MERGE: hi and lo rows of B in one MMA where they fit / never
    ("bstages", 8, (0, 2)),     # FBS_OPT_TC_BSTAGES: deepest operand-B ring that fits / two stages
    ("bfroma", 9, (0, 1)),      # FBS_OPT_TC_BFROMA: inner pair rows from operand A where it applies / never
    ("stack", 10, (0, 1)),      # FBS_OPT_TC_STACK: A's hi and lo stacked on M where it applies / never
)


def _apply(plan, choice):
    for name, opt, _ in TUNABLE:
        plan.set_option(opt, int(choice.get(name, 0)))


def autotune(plan: Plan, field, repeats: int = 3, cache: str = _TUNE_CACHE, batch=None) -> Dict[str, float]:
    """Pick the plan's options by timing them on ``field`` (a device tensor),
    or on batched calls over the list ``batch`` of device tensors: coordinate
    descent over TUNABLE from the defaults, keeping a change only when it is
    faster by more than 2% (batched calls: the options they use, pipeline
    step, pair assignment, warp roles and the merged hi/lo products).  The choice is cached per (N, L,
    edges, precision, batch size, library build, device)."""
    import torch
    key = _key(plan.N, plan.L, plan.edges, plan.precision) + ("|batch%d" % len(batch) if batch else "")
    table = {}
    if os.path.exists(cache):
        try:
            table = json.load(open(cache))
        except Exception:
            table = {}
    if key in table:
        _apply(plan, table[key]["choice"])
        return table[key]
    nf = len(batch) if batch else 1
    B = torch.empty((nf, plan.ntrip), dtype=torch.float64, device=field.device)
    P = torch.empty((nf, plan.nbins), dtype=torch.float64, device=field.device)
    run = (lambda: plan.bispectrum_batch(batch, B, P)) if batch else (lambda: plan.bispectrum(field, B[0], P[0]))
    tunable = [t for t in TUNABLE if not batch or t[0] in ("chunk", "pairs", "roles", "merge")]

    def timed(choice):
        _apply(plan, choice)
        run()  # warm-up (builds the option's tables)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(repeats):
            run()
        e1.record()
        torch.cuda.synchronize()
        plan.check()
        return e0.elapsed_time(e1) / repeats

    best = {name: vals[0] for name, _, vals in TUNABLE}
    tried = {}
    best_ms = timed(best)
    tried[json.dumps(best, sort_keys=True)] = best_ms
    if plan.precision != "fp32":
        for name, _, vals in tunable:
            for v in vals[1:]:
                cand = dict(best, **{name: v})
                k = json.dumps(cand, sort_keys=True)
                if k not in tried:
                    tried[k] = timed(cand)
                if tried[k] < 0.98 * best_ms:
                    best, best_ms = cand, tried[k]
    elif not batch:  # the FP32 contraction has no tensor-core options: slabs only
        for v in next(vals for name, _, vals in TUNABLE if name == "slab")[1:]:
            cand = dict(best, slab=v)
            ms = timed(cand)
            if ms < 0.98 * best_ms:
                best, best_ms = cand, ms
    _apply(plan, best)
    table[key] = {"choice": best, "ms": best_ms, "tried": len(tried)}
    try:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        with open(cache + ".tmp", "w") as fh:
            json.dump(table, fh)
        os.replace(cache + ".tmp", cache)
    except Exception:
        pass
    return table[key]


class GraphBatch:
    """Many realisations of uneven grid sizes in one CUDA graph of batched
    launches.

    Realisations are grouped by grid size; each group is one plan and one
    fbs_bispectrum_batch call, so every stage runs once per group for all of
    its realisations (the field taken from a grid dimension), and the graph
    holds a few dozen launches however many realisations there are.
    fields: sequence of float32 [N][N][N] arrays/tensors (any mix of N).
    edges_for: callable N -> bin edges (physical k units) for that grid.
    """

    def __init__(self, fields, L_for, edges_for, precision="bf16x3", tune=True, device=0):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.stream = torch.cuda.Stream(device=self.dev)
        self.fields = [f if isinstance(f, torch.Tensor) and f.is_cuda
                       else torch.as_tensor(np.ascontiguousarray(f, dtype=np.float32)).to(self.dev)
                       for f in fields]
        self.groups: Dict[int, dict] = {}
        self.where: List[Tuple[int, int]] = []  # realisation -> (grid, index in its group)
        self.tuning = {}
        for f in self.fields:
            N = f.shape[0]
            if N not in self.groups:
                self.groups[N] = {"plan": Plan(N, L_for(N), edges_for(N), precision=precision, stream=self.stream),
                                  "fields": []}
            g = self.groups[N]
            self.where.append((N, len(g["fields"])))
            g["fields"].append(f)
        for N, g in self.groups.items():
            pl, nf = g["plan"], len(g["fields"])
            g["B"] = torch.empty((nf, pl.ntrip), dtype=torch.float64, device=self.dev)
            g["P"] = torch.empty((nf, pl.nbins), dtype=torch.float64, device=self.dev)
            if tune:
                with torch.cuda.stream(self.stream):
                    self.tuning[N] = autotune(pl, g["fields"][0], batch=g["fields"])
        self.graph = None

    @property
    def plans(self):
        return {N: g["plan"] for N, g in self.groups.items()}

    def run_eager(self):
        """One batched call per grid size (the same launches the graph holds)."""
        with self.torch.cuda.stream(self.stream):
            for g in self.groups.values():
                g["plan"].bispectrum_batch(g["fields"], g["B"], g["P"])

    def run_one_at_a_time(self, precision=None):
        """The same realisations with one fbs_bispectrum call each (comparison)."""
        with self.torch.cuda.stream(self.stream):
            for g in self.groups.values():
                pl = g["plan"]
                for i, f in enumerate(g["fields"]):
                    pl.bispectrum(f, g["B"][i], g["P"][i])

    def capture(self):
        torch = self.torch
        self.run_eager()  # warm-up: buffers and field lists exist before the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream, capture_error_mode="relaxed"):
            for grp in self.groups.values():
                grp["plan"].bispectrum_batch(grp["fields"], grp["B"], grp["P"])
        self.graph = g
        return g

    def replay(self):
        """Launch the captured graph on the batch's stream (where the eager
        calls and the timing events run)."""
        with self.torch.cuda.stream(self.stream):
            self.graph.replay()

    def results(self):
        """(triplets, B, P) of every realisation, in input order."""
        self.torch.cuda.synchronize()
        host = {N: (g["B"].cpu().numpy(), g["P"].cpu().numpy()) for N, g in self.groups.items()}
        return [(self.groups[N]["plan"].triplets, host[N][0][i], host[N][1][i]) for N, i in self.where]

    def close(self):
        self.torch.cuda.synchronize()
        self.graph = None
        for g in self.groups.values():
            g["plan"].close()
        self.groups.clear()
