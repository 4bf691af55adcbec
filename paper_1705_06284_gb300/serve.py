"""Continuous-batching serving loop for estimator requests.

Requests arrive over time (a likelihood sampler asking for the bispectrum of
one field after another, with mixed grid sizes and bin sets).  The server
keeps plans resident on the device, admits a request as soon as a slot (a
CUDA stream) is free and its plan fits the HBM budget, overlaps the work of
all admitted requests on the device, and reports per-request latency from
arrival to a host-visible result.

Plans are built off the admission loop: a builder thread runs the library's
plan creation (its host work and its device work on a stream of its own) while
the loop keeps polling completions and admitting requests whose plans are
ready.  The plan-time results of every plan built (the closed items and their
exact counts, fbs_plan_export_counts) are kept by key (N, L, edges,
precision), so a plan evicted under the budget and needed again is rebuilt
without the FP64 count pass; ``count_cache_dir`` also keeps them on disk
across processes.

Every estimator step runs in ``libfbs.so`` through the C ABI; this module
only schedules: host->device copy of the field on the slot's stream, one
``fbs_bispectrum`` call, device->host copy of the outputs, and a CUDA event
that is polled without blocking.  Results are bit-identical to running each
request alone (the kernels use fixed reduction orders).
"""
from __future__ import annotations

import collections
import concurrent.futures
import dataclasses
import hashlib
import os
import time
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import FbsError, Plan, fbs_set_slab_budget

FBS_ERR_ARG = -1


@dataclasses.dataclass
class Request:
    rid: int
    field: np.ndarray          # float32 [N][N][N] on the host
    L: float
    edges: Tuple[float, ...]
    arrival: float = 0.0       # seconds after the start of the run
    precision: str = "bf16x3"


@dataclasses.dataclass
class Result:
    rid: int
    triplets: np.ndarray
    N_tri: np.ndarray
    B: np.ndarray
    P: np.ndarray
    arrival: float
    admitted: float
    done: float
    error: Optional[str] = None   # set when the request was refused or cancelled (no B, P)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def plan_bytes_estimate(N: int, nbins: int, slab_budget: int = 8 << 30) -> int:
    """Device bytes a plan needs at its peak (plan-time FP64 count fields
    included), used for admission before the plan exists."""
    planes = max(1, min(N, slab_budget // max(1, nbins * N * N * 4)))
    shell = nbins * planes * N * N * 4
    scratch = 3 * N * N * (N // 4 + 1) * 8 + N ** 3 * 4
    counts = nbins * (N // 2 + 1) ** 3 * 8
    return shell + scratch + counts + (64 << 20)


class _Slot:
    def __init__(self, torch, dev):
        self.stream = torch.cuda.Stream(device=dev)
        self.busy = None  # (request, plan entry, event, outputs, t_admit)


class EstimatorServer:
    """Serve bispectrum requests with overlap on one GPU.

    hbm_budget: bytes of device memory the server's plans and buffers may hold.
    slots: concurrent requests in flight (one CUDA stream each).
    build_async: build plans on a builder thread (default) instead of inline.
    count_cache_dir: directory for the plan-time counts (optional).
    slab_bytes: shell-field slab buffer of the server's plans (smaller slabs
    keep more plans resident); set process-wide while the server is open.
    """

    NEVER = "never"  # _plan_for: the request cannot fit even with every idle plan evicted

    FRESH_S = 5.0  # a new plan is not evicted before its first use (or this long)

    def __init__(self, hbm_budget: int = 120 << 30, slots: int = 4, device: int = 0,
                 build_async: bool = True, count_cache_dir: Optional[str] = None, slab_bytes: int = 1 << 30):
        import torch
        self.torch = torch
        self.slab_bytes = int(slab_bytes)
        fbs_set_slab_budget(self.slab_bytes)
        self.dev = torch.device("cuda", device)
        self.budget = int(hbm_budget)
        self.slots = [_Slot(torch, self.dev) for _ in range(slots)]
        # key -> list of entries {"plan", "bytes", "busy", "last", "dfield"}
        self.plans: Dict[tuple, List[dict]] = collections.defaultdict(list)
        self.held = 0
        self.plan_creations = 0
        self.plans_from_cache = 0
        self.counts_cache: Dict[tuple, bytes] = {}
        self.count_cache_dir = count_cache_dir
        self._cancelled = set()
        self._failed: Dict[tuple, str] = {}  # key -> why its plan could not be built
        # key -> (future, bytes reserved for it, bytes of its field copies)
        self._building: Dict[tuple, Tuple[concurrent.futures.Future, int, int]] = {}
        self._pool = concurrent.futures.ThreadPoolExecutor(max_workers=1) if build_async else None
        self._build_stream = torch.cuda.Stream(device=self.dev) if build_async else None

    # -- plan cache under the budget
    def _key(self, req: Request):
        return (req.field.shape[0], float(req.L), tuple(float(e) for e in req.edges), req.precision)

    def _evict_for(self, need: int) -> bool:
        now = time.perf_counter()
        idle = [(e["last"], k, e) for k, lst in self.plans.items() for e in lst
                if not e["busy"] and e.get("fresh_until", 0.0) <= now]
        idle.sort(key=lambda t: t[0])
        while self.held + need > self.budget and idle:
            _, k, e = idle.pop(0)
            e["plan"].close()
            self.plans[k].remove(e)
            self.held -= e["bytes"]
        return self.held + need <= self.budget

    def _count_file(self, key):
        h = hashlib.sha1(repr(key[:3]).encode()).hexdigest()[:24]
        return os.path.join(self.count_cache_dir, "plan_counts_%s.bin" % h)

    def _cached_counts(self, key):
        c = self.counts_cache.get(key[:3])
        if c is None and self.count_cache_dir:
            p = self._count_file(key)
            if os.path.exists(p):
                c = open(p, "rb").read()
                self.counts_cache[key[:3]] = c
        return c

    def _build(self, req: Request, key, stream):
        """Create the plan (runs on the builder thread, or inline)."""
        counts = self._cached_counts(key)
        try:
            plan = Plan(req.field.shape[0], req.L, np.asarray(req.edges), precision=req.precision, stream=stream,
                        counts=counts)
        except FbsError as e:
            if counts is None or e.status != FBS_ERR_ARG:
                raise
            # a stored blob of another library version or plan: count afresh
            self.counts_cache.pop(key[:3], None)
            counts = None
            plan = Plan(req.field.shape[0], req.L, np.asarray(req.edges), precision=req.precision, stream=stream)
        if counts is None:
            blob = plan.export_counts()
            self.counts_cache[key[:3]] = blob
            if self.count_cache_dir:
                os.makedirs(self.count_cache_dir, exist_ok=True)
                tmp = self._count_file(key) + ".tmp%d" % os.getpid()
                with open(tmp, "wb") as fh:
                    fh.write(blob)
                os.replace(tmp, self._count_file(key))
        return plan, counts is not None

    def _register(self, key, plan, from_cache, reserved, field_bytes):
        self.plan_creations += 1
        self.plans_from_cache += int(from_cache)
        e = {"plan": plan, "bytes": plan.device_bytes + field_bytes, "busy": False,
             "last": time.perf_counter(), "dfield": None,
             "fresh_until": time.perf_counter() + self.FRESH_S}  # kept for the request it was built for
        self.held += e["bytes"] - reserved
        self.plans[key].append(e)
        return e

    def _poll_builds(self):
        for key, (fut, reserved, fbytes) in list(self._building.items()):
            if fut.done():
                del self._building[key]
                try:
                    plan, from_cache = fut.result()
                except Exception as ex:  # its requests are refused, the loop goes on
                    self.held -= reserved
                    self._failed[key] = "plan creation failed: %s" % str(ex)[:200]
                    continue
                self._register(key, plan, from_cache, reserved, fbytes)

    def _plan_for(self, req: Request, stream):
        """An idle plan for the request, None when it must wait (for busy work
        to finish, or for its plan to be built), or NEVER when it can never
        fit."""
        key = self._key(req)
        for e in self.plans[key]:
            if not e["busy"]:
                e["plan"].set_stream(stream)
                return e
        if key in self._building:
            return None
        if key in self._failed:
            return self.NEVER
        N = req.field.shape[0]
        if self._pool is not None and self._building:
            return None  # one build at a time: the next starts when this one is done
        need = plan_bytes_estimate(N, len(req.edges) - 1, self.slab_bytes) + 2 * req.field.nbytes
        if need > self.budget:
            return self.NEVER
        if not self._evict_for(need):
            # busy plans, plans kept for their first request and builds in
            # flight free up later: wait; otherwise it can never fit
            now = time.perf_counter()
            busy = any(e["busy"] or e.get("fresh_until", 0.0) > now for lst in self.plans.values() for e in lst) \
                or bool(self._building)
            return None if busy else self.NEVER
        if self._pool is not None:
            self.held += need  # reserved until the plan exists
            self._building[key] = (self._pool.submit(self._build, req, key, self._build_stream), need,
                                   2 * req.field.nbytes)
            return None
        plan, from_cache = self._build(req, key, stream)
        e = self._register(key, plan, from_cache, 0, 2 * req.field.nbytes)
        # the estimate admitted it; if the real plan is larger, make room or undo
        if self.held > self.budget and not self._evict_for(0):
            e["busy"] = True  # keep it out of its own eviction while we decide
            busy = any(x["busy"] for lst in self.plans.values() for x in lst if x is not e)
            plan.close()
            self.plans[key].remove(e)
            self.held -= e["bytes"]
            return None if busy else self.NEVER
        return e

    # -- one request on one slot
    def _submit(self, slot: _Slot, req: Request, entry: dict, t0: float):
        torch = self.torch
        plan = entry["plan"]
        N = req.field.shape[0]
        entry["busy"] = True
        entry["fresh_until"] = 0.0
        with torch.cuda.stream(slot.stream):
            if entry["dfield"] is None or entry["dfield"].shape[0] != N:
                entry["dfield"] = torch.empty((N, N, N), dtype=torch.float32, device=self.dev)
            host = torch.from_numpy(req.field)
            if not host.is_pinned():
                host = host.pin_memory()
            entry["dfield"].copy_(host, non_blocking=True)
            B = torch.empty(plan.ntrip, dtype=torch.float64, device=self.dev)
            P = torch.empty(plan.nbins, dtype=torch.float64, device=self.dev)
            plan.bispectrum(entry["dfield"], B, P)
            Bh = torch.empty(plan.ntrip, dtype=torch.float64, pin_memory=True)
            Ph = torch.empty(plan.nbins, dtype=torch.float64, pin_memory=True)
            Bh.copy_(B, non_blocking=True)
            Ph.copy_(P, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(slot.stream)
        slot.busy = (req, entry, ev, (B, P, Bh, Ph, host), time.perf_counter() - t0)

    def cancel(self, rid: int):
        """Cancel a request that has not been admitted yet (it returns a
        Result with error "cancelled"); admitted requests run to the end."""
        self._cancelled.add(rid)

    def _refuse(self, req: Request, why: str, realtime: bool, t0: float) -> Result:
        empty = np.zeros(0)
        t = time.perf_counter() - t0
        return Result(req.rid, np.zeros((0, 3), dtype=np.int32), np.zeros(0, dtype=np.int64), empty, empty,
                      req.arrival if realtime else 0.0, t, t, error=why)

    def run(self, requests: Sequence[Request], realtime: bool = True,
            deadline_s: Optional[float] = None) -> List[Result]:
        """Serve ``requests`` (sorted by arrival).  With ``realtime`` a request
        is not admitted before its arrival time; otherwise arrivals are
        ignored (all requests are available at once).  A request whose plan
        and buffers cannot fit the budget even with every idle plan evicted
        is refused (Result.error) instead of holding up the queue.  Requests
        wait in arrival order for a free slot; one whose plan is being built
        lets later requests with ready plans go first.  With ``deadline_s``,
        requests not admitted within that many seconds of the start are
        refused ("deadline"); admitted ones run to the end."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting: List[Request] = []
        results: List[Result] = []
        t0 = time.perf_counter()
        while pending or waiting or any(s.busy for s in self.slots) or self._building:
            now = time.perf_counter() - t0
            if deadline_s is not None and now > deadline_s and (pending or waiting):
                for r in list(waiting) + list(pending):
                    results.append(self._refuse(r, "deadline", realtime, t0))
                waiting, pending = [], collections.deque()
            while pending and (not realtime or pending[0].arrival <= now):
                waiting.append(pending.popleft())
            if self._cancelled and waiting:
                keep = []
                for r in waiting:
                    if r.rid in self._cancelled:
                        results.append(self._refuse(r, "cancelled", realtime, t0))
                    else:
                        keep.append(r)
                waiting = keep
            if self._building:
                self._poll_builds()
            # completions (non-blocking)
            for s in self.slots:
                if s.busy and s.busy[2].query():
                    req, entry, ev, bufs, t_adm = s.busy
                    _, _, Bh, Ph, _ = bufs
                    plan = entry["plan"]
                    results.append(Result(req.rid, plan.triplets.copy(), plan.N_tri.copy(),
                                          Bh.numpy().copy(), Ph.numpy().copy(),
                                          req.arrival if realtime else 0.0, t_adm,
                                          time.perf_counter() - t0))
                    entry["busy"] = False
                    entry["last"] = time.perf_counter()
                    s.busy = None
            # admissions: in arrival order over the free slots; a request whose
            # plan is not ready (being built, or waiting for memory) does not
            # block the ones behind it
            progressed = False
            free = [s for s in self.slots if not s.busy]
            i = 0
            while free and i < len(waiting):
                req = waiting[i]
                entry = self._plan_for(req, free[0].stream)
                if entry is self.NEVER:
                    waiting.pop(i)
                    why = self._failed.get(self._key(req), "does not fit the HBM budget")
                    results.append(self._refuse(req, why, realtime, t0))
                    progressed = True
                    continue
                if entry is None:
                    i += 1
                    continue
                waiting.pop(i)
                self._submit(free.pop(0), req, entry, t0)
                progressed = True
            if not progressed:
                time.sleep(0.0002)
        return sorted(results, key=lambda r: r.rid)

    def close(self):
        self.torch.cuda.synchronize()
        if self._pool is not None:
            for key, (fut, reserved, fbytes) in list(self._building.items()):
                try:
                    plan, _ = fut.result()
                    plan.close()
                except Exception:  # a failed build left nothing to close
                    pass
            self._building.clear()
            self._pool.shutdown(wait=True)
        for lst in self.plans.values():
            for e in lst:
                e["plan"].close()
        self.plans.clear()
        self.held = 0
        fbs_set_slab_budget(0)  # plans created after the server get the default slab again


def latency_percentiles(results: Sequence[Result]) -> Dict[str, float]:
    lat = np.array([r.latency for r in results if r.error is None])
    if lat.size == 0:
        return {"p50_ms": None, "p99_ms": None, "mean_ms": None}
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3)}
