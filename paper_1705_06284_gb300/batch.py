"""Batched estimation of many realisations with uneven grid sizes.

All realisations of a batch are enqueued once, captured into one CUDA graph
(one plan per distinct (N, L, edges), every launch of every realisation in
order on one stream), and the graph is replayed: the host issues a single
launch for the whole batch.  Every kernel is the library's; this module only
captures and replays.  A small autotuner picks, per plan, the tensor-core
orientation that runs fastest on the plan's own problem and caches it.
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


def autotune(plan: Plan, field, repeats: int = 3, cache: str = _TUNE_CACHE) -> Dict[str, float]:
    """Time the plan's tensor-core orientations on ``field`` (a device tensor)
    and keep the fastest; the choice is cached per (N, L, edges, precision)."""
    import torch
    key = _key(plan.N, plan.L, plan.edges, plan.precision)
    table = {}
    if os.path.exists(cache):
        try:
            table = json.load(open(cache))
        except Exception:
            table = {}
    if key in table:
        plan.set_tc_wide(bool(table[key]["wide"]))
        return table[key]
    if plan.precision == "fp32":
        return {"wide": False, "ms": {}}
    B = torch.empty(plan.ntrip, dtype=torch.float64, device=field.device)
    P = torch.empty(plan.nbins, dtype=torch.float64, device=field.device)
    ms = {}
    for wide in (False, True):
        plan.set_tc_wide(wide)
        plan.bispectrum(field, B, P)  # warm-up (builds the orientation's tables)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(repeats):
            plan.bispectrum(field, B, P)
        torch.cuda.synchronize()
        ms["wide" if wide else "narrow"] = 1e3 * (time.perf_counter() - t0) / repeats
    best = ms["wide"] < ms["narrow"]
    plan.set_tc_wide(best)
    table[key] = {"wide": best, "ms": ms}
    try:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        with open(cache + ".tmp", "w") as fh:
            json.dump(table, fh)
        os.replace(cache + ".tmp", cache)
    except Exception:
        pass
    return table[key]


class GraphBatch:
    """Capture the bispectra of many realisations into one CUDA graph.

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
        self.plans: Dict[Tuple, Plan] = {}
        self.items: List[Tuple[Plan, object, object, object]] = []
        self.tuning = {}
        for f in self.fields:
            N = f.shape[0]
            key = (N,)
            if key not in self.plans:
                pl = Plan(N, L_for(N), edges_for(N), precision=precision, stream=self.stream)
                if tune:
                    with torch.cuda.stream(self.stream):
                        self.tuning[N] = autotune(pl, f)
                self.plans[key] = pl
            pl = self.plans[key]
            B = torch.empty(pl.ntrip, dtype=torch.float64, device=self.dev)
            P = torch.empty(pl.nbins, dtype=torch.float64, device=self.dev)
            self.items.append((pl, f, B, P))
        self.graph = None

    def run_eager(self):
        with self.torch.cuda.stream(self.stream):
            for pl, f, B, P in self.items:
                pl.bispectrum(f, B, P)

    def capture(self):
        torch = self.torch
        self.run_eager()  # warm-up: every plan's first call happens outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream, capture_error_mode="relaxed"):
            for pl, f, B, P in self.items:
                pl.bispectrum(f, B, P)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def results(self):
        self.torch.cuda.synchronize()
        return [(pl.triplets, B.cpu().numpy(), P.cpu().numpy()) for pl, f, B, P in self.items]

    def close(self):
        self.torch.cuda.synchronize()
        self.graph = None
        for pl in self.plans.values():
            pl.close()
        self.plans.clear()
