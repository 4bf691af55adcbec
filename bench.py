"""Benchmark of the FFT polyspectrum estimator on one GB300 (or N replicas).

Workload (one "step"): one 512^3 quadratic-local field (delta = g + f(g^2 -
<g^2>), g Gaussian with P ~ k^-1.5, sigma_g = 0.1, f = 0.3), bispectrum over
all closed triplets of 64 log bins from k_f to N k_f/4 with P(k), plus the
four-shell trispectrum on 16 log bins (which also yields B and P on those
bins).  Counts are plan-time (outside the step).  Inputs are resident in HBM
when the timed region starts; the field (512 MiB) and the shell-field slabs
(GiBs) are larger than L2, so no extra flush is needed.

Metric: closed triplets of the 64-bin plan x fields / wall time
(triangle-bins/s).  ``e2e`` repeats the measurement through the C ABI with
a pinned host field and host outputs (host<->device copies inside the timed
region).  ``--impl reference`` times the FP64 CPU oracle (direct
measurement, Eq. bi_direct) on a bounded sample of the same workload.

With --gpus N > 1 (torchrun, one process per GPU) every rank runs its own
replica on its own field (the estimator has no exchange step); value is the
total over ranks divided by the slowest rank's time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

_T0 = time.perf_counter()
_PHASES = {}


def _phase(name):
    """Progress on stderr (the JSON line stays alone on stdout) and the time
    each phase began, for the line's ``phase_s``."""
    t = time.perf_counter() - _T0
    _PHASES[name] = round(t, 1)
    print("[bench +%.1fs] %s" % (t, name), file=sys.stderr, flush=True)

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID, L_BOX, NB_B, NB_T = 512, 1000.0, 64, 16
FIELD_KW = dict(f=0.3, slope=-1.5, sigma_g=0.1)


def workload(args):
    return {"workload": "quadratic_local_%d^3_B%dlog_T%dlog" % (args.N, args.nb, args.nbt),
            "N": args.N, "L": L_BOX, "bins_B": args.nb, "bins_T": args.nbt,
            "field": "quadratic-local f=0.3 slope=-1.5 sigma_g=0.1 seed=2+rank",
            "l2": "inputs larger than L2 (field %d MiB, shell-field slabs > 1 GiB)"
                  % (4 * args.N ** 3 >> 20)}


def edges(N, nb):
    kf = 2 * math.pi / L_BOX
    return np.geomspace(kf, 0.25 * N * kf, nb + 1)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _find(d, *keys):
    for k in keys:
        if k in d:
            return float(d[k])
    for v in d.values():
        if isinstance(v, dict):
            r = _find(v, *keys)
            if r is not None:
                return r
    return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # samples go to a per-process file under the system temporary directory
        # (FBS_CLOCKS_DIR overrides it, e.g. to keep the samples of a run)
        import tempfile
        d = os.environ.get("FBS_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, "fbs_clocks_gpu%d_pid%d.csv" % (index, os.getpid()))

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


CPU_SAMPLE_M1 = 1536  # m1 modes of the oracle's timed sample (about 15 s on 16 Grace cores at 512^3)


def cpu_baseline(args, n_sample=CPU_SAMPLE_M1):
    """FP64 direct-measurement oracle on a fixed, deterministic sample of m1
    modes (every k-th mode of the binned modes, k = modes // n_sample), taken
    as two interleaved halves.

    The full-workload time is the FP64 FFT of the field (timed once) plus the
    all-pairs sum time per m1 mode (timed on the sample) times the number of
    binned modes; ``spread`` is the relative difference of the two halves'
    per-mode rates (the sampling uncertainty of the extrapolation)."""
    import fields
    import oracle
    N = args.N
    thr = oracle.thresholds(edges(N, args.nb), L_BOX)
    nm = oracle.count_modes(N, thr)
    f = fields.quadratic_local(N, seed=2, **FIELD_KW).astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    D = oracle.spectrum(f)
    t_fft = time.perf_counter() - t0
    stride = max(1, nm // max(1, n_sample))
    # the call's fixed cost (listing the binned modes), timed with one m1 mode
    t0 = time.perf_counter()
    oracle.direct_sums_from_spectrum(D, thr, 0, max(1, nm))
    t_fixed = time.perf_counter() - t0
    rates, t_s, done = [], 0.0, 0
    for start in (0, stride):
        t0 = time.perf_counter()
        _, _, _, d = oracle.direct_sums_from_spectrum(D, thr, start, 2 * stride)
        dt = time.perf_counter() - t0
        t_s += dt
        done += d
        rates.append(max(0.0, dt - t_fixed) / max(1, d))
    rate = 0.5 * (rates[0] + rates[1])
    t_full = t_fft + t_fixed + rate * nm
    spread = abs(rates[0] - rates[1]) / max(1e-300, rate)
    return t_full, {"m1_sampled": int(done), "m1_total": int(nm), "sample_s": t_s, "fixed_s": t_fixed,
                    "fft_s": t_fft, "cores": oracle.num_threads(), "spread": spread}


def run_reference(args, ntrip_hint=None):
    """--impl reference: the FP64 CPU oracle, each step a bounded sample."""
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import fields  # noqa: F401
    times = []
    info = None
    # a fixed strided sample each step, sized so the whole run takes about a
    # minute of sampling (a quarter of the cpu_baseline leg's sample at the
    # default 13 steps)
    n_sample = max(16, min(CPU_SAMPLE_M1, int(CPU_SAMPLE_M1 * 13 / 4 / max(1, args.steps + args.warmup))))
    for i in range(args.warmup + args.steps):
        t_full, info = cpu_baseline(args, n_sample=n_sample)
        if i >= args.warmup:
            times.append(t_full)
    ntrip = ntrip_hint
    t = float(np.mean(times))
    val = ntrip / t
    line = {"impl": "reference", "metric": "bispectrum triangle-bins/s", "value": val,
            "unit": "triangle-bins/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload(args),
            "cpu_baseline": {"value": val, "unit": "triangle-bins/s", "cores": info["cores"],
                             "kind": "oracle",
                             "sample": "direct all-pairs sum over a fixed sample of %d of %d m1 modes "
                                       "per step (every k-th binned mode), scaled to all modes; halves "
                                       "differ by %.0f%%" % (info["m1_sampled"], info["m1_total"],
                                                             100 * info["spread"])},
            "e2e": {"value": val, "unit": "triangle-bins/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=os.environ.get("FBS_BENCH_PRECISION", "bf16x3"))
    ap.add_argument("--N", type=int, default=N_GRID)
    ap.add_argument("--nb", type=int, default=NB_B)
    ap.add_argument("--nbt", type=int, default=NB_T)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-workloads", action="store_true")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if world > 1 and rank != 0:
            return
        # the closed-triplet count is the plan's; the oracle's all-pairs sum
        # produces every triplet of the workload at once
        import oracle
        e = edges(args.N, args.nb)
        thr = oracle.thresholds(e, L_BOX)
        ntrip = _closed_triplets_oracle(args.N, thr)
        run_reference(args, ntrip_hint=ntrip)
        return

    import torch
    import fields
    import paper_1705_06284_gb300 as fbs

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()

    N = args.N
    f64 = fields.quadratic_local(N, seed=2 + rank, **FIELD_KW)
    f32 = f64.astype(np.float32)
    del f64
    field = torch.from_numpy(f32).to(dev)
    eB, eT = edges(N, args.nb), edges(N, args.nbt)
    t0 = time.perf_counter()
    _phase("plans")
    planB = fbs.Plan(N, L_BOX, eB, precision=args.precision, timing=True, stream=stream)
    planT = fbs.Plan(N, L_BOX, eT, precision=args.precision, trispectrum=True, timing=True, stream=stream)
    # one upload and one forward transform of the field serve both plans
    # (fbs_plan_follow: the trispectrum plan reads the bispectrum plan's
    # spectrum on the shared stream)
    planT.follow(planB)
    plan_s = time.perf_counter() - t0
    B = torch.empty(planB.ntrip, dtype=torch.float64, device=dev)
    P = torch.empty(planB.nbins, dtype=torch.float64, device=dev)
    T = torch.empty(planT.nquad, dtype=torch.float64, device=dev)
    B16 = torch.empty(planT.ntrip, dtype=torch.float64, device=dev)
    P16 = torch.empty(planT.nbins, dtype=torch.float64, device=dev)

    def step(fld, outs):
        planB.bispectrum(fld, outs[0], outs[1])
        planT.trispectrum(None, outs[2], outs[3], outs[4])

    outs_dev = (B, P, T, B16, P16)
    _phase("warmup and timed steps")
    for _ in range(args.warmup):
        step(field, outs_dev)
    torch.cuda.synchronize()
    planB.kernel_times(reset=True)
    planT.kernel_times(reset=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(field, outs_dev)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    kB = planB.kernel_times(reset=True)
    kT = planT.kernel_times(reset=True)
    launches = sum(v[1] for v in kB.values()) + sum(v[1] for v in kT.values())

    # e2e: pinned host field in, pinned host outputs back, through the C ABI,
    # as a streaming caller would run it: both plans' calls of step k are
    # enqueued (the bispectrum plan copies the field on its copy stream, the
    # trispectrum plan follows its spectrum), then the host waits for the
    # results of step k-1 (two output sets), so the field copy of step k runs
    # under the kernels of step k-1.  Every step copies
    # its field in and its results out; the loop ends with every result on
    # the host.
    e2e = None
    if not args.no_e2e:
        _phase("e2e")
        hfield = torch.from_numpy(f32).pin_memory()
        sizes = (planB.ntrip, planB.nbins, planT.nquad, planT.ntrip, planT.nbins)
        outs_sets = [tuple(torch.empty(n, dtype=torch.float64).pin_memory() for n in sizes) for _ in range(2)]
        done = [torch.cuda.Event(), torch.cuda.Event()]
        checksum = [0.0]

        def e2e_run(nsteps):
            for k in range(nsteps):
                step(hfield, outs_sets[k % 2])
                done[k % 2].record(stream)
                if k >= 1:
                    done[(k - 1) % 2].synchronize()
                    checksum[0] += float(outs_sets[(k - 1) % 2][0][0])  # the host reads step k-1
            done[(nsteps - 1) % 2].synchronize()
            checksum[0] += float(outs_sets[(nsteps - 1) % 2][0][0])

        e2e_run(2)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_run(args.steps)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.steps
        planB.kernel_times(reset=True)
        planT.kernel_times(reset=True)
        h2d = f32.nbytes  # one upload per step for both plans
        d2h = 8 * (planB.ntrip + planB.nbins + planT.nquad + planT.ntrip + planT.nbins)
        e2e = {"value": None, "unit": "triangle-bins/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "_s": e2e_s,
               "mode": "streaming: host field copied in and results read back every step; "
                       "the host reads step k-1's results while step k runs"}
        outs_host = tuple(t.numpy() for t in outs_sets[(args.steps - 1) % 2])
        # sanity: host outputs equal device outputs
        if not np.allclose(outs_host[0], B.cpu().numpy(), rtol=0, atol=0):
            e2e["mismatch"] = True

    ms_max, e2e_max = max_over_ranks(dist, [ms, e2e["_s"] if e2e else 0.0], device=dev)
    value = whole_job_rate(world, planB.ntrip, ms_max / 1e3)

    # roofline of the dominant kernel class (largest share of the timed region)
    pk, pk_src = peaks()
    allk = {("B:" + k): v for k, v in kB.items()}
    allk.update({("T:" + k): v for k, v in kT.items()})
    top = max(allk.items(), key=lambda kv: kv[1][0])
    roof = roofline(top, planB, planT, N, pk, pk_src, clocks, args.steps)
    roof_fft = roofline_fft(kB, kT, planB, planT, N, pk, pk_src, args.steps)

    line = {"metric": "bispectrum triangle-bins/s", "value": value, "unit": "triangle-bins/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16x3": "bf16x3", "bf16": "bf16"}[args.precision],
            "data": "synthetic", "config": dict(workload(args), ntrip_B=planB.ntrip,
                                                nquad_T=planT.nquad, precision_B=args.precision,
                                                precision_T=args.precision, parallelism="replicas%d" % world),
            "roofline": roof, "roofline_fft": roof_fft, "clocks": clocks, "gpu_launches": int(launches),
            "levels": {"B": [l["M"] for l in planB.levels], "T": [l["M"] for l in planT.levels]},
            "levels_detail": {"B": planB.levels, "T": planT.levels},
            "tc_jobs": {"B": planB.tc_info(), "T": planT.tc_info()},
            "plan_s": plan_s, "count_margin": [planB.count_margin, planT.count_margin],
            "quad_counts_exact": planT.quad_counts_exact,
            "kernel_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in allk.items() if v[1]}}
    if e2e:
        e2e["value"] = whole_job_rate(world, planB.ntrip, e2e_max)
        e2e.pop("_s", None)
        line["e2e"] = e2e
    if rank == 0 and not args.no_plain and world == 1:
        _phase("plain_fp32_gpu")
        # plain FP32 GPU path on the same field (comparison only)
        try:
            thrB = np.asarray(planB.thresholds)
            plain_fp32_gpu(field, N, L_BOX, thrB, planB.triplets, dev)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            numP = plain_fp32_gpu(field, N, L_BOX, thrB, planB.triplets, dev)
            torch.cuda.synchronize()
            tp = time.perf_counter() - t0
            planB.bispectrum(field, B, P)
            ours, _, _ = planB.sums()
            numP = numP.cpu().numpy()
            big = np.abs(ours) > 1e-3 * np.abs(ours).max()
            line["plain_fp32_gpu"] = {
                "value": planB.ntrip / tp, "unit": "triangle-bins/s", "ms_per_field": 1e3 * tp,
                "what": "cuFFT R2C + per-bin mask + cuFFT C2R, FP32 pair products x FP32 GEMV per "
                        "outer pair, FP64 across x chunks (torch.fft / torch matmul)",
                "speedup_of_ours": (planB.ntrip / (ms_max / 1e3)) / (planB.ntrip / tp),
                "max_rel_diff_vs_ours": float(np.max(np.abs(numP[big] - ours[big]) / np.abs(ours[big])))}
        except Exception as ex:
            line["plain_fp32_gpu"] = {"value": None, "error": str(ex)[:200]}
    if rank == 0 and not args.no_plain and world == 1:
        _phase("cufft_fft_stage")
        try:
            ms_cu, nb_cu = cufft_fft_stage(field, N, np.asarray(planB.thresholds), dev)
            ours_fft = sum(kB.get(c, (0, 0))[0] for c in FFT_CLASSES) / args.steps
            line["cufft_fft_stage"] = {
                "ms_per_field": ms_cu, "bins": nb_cu, "ours_ms_per_field": ours_fft,
                "speedup_of_ours": ms_cu / ours_fft if ours_fft else None,
                "what": "cuFFT R2C of the field + one masked C2R per non-empty bin of the 64-bin plan on "
                        "the full N^3 grid (torch.fft); ours: the FFT kernels of the same plan"}
        except Exception as ex:
            line["cufft_fft_stage"] = {"value": None, "error": str(ex)[:200]}
    if rank == 0 and not args.no_workloads and world == 1:
        _phase("workloads")
        try:
            import fields
            wl = {}
            f1 = fields.lognormal(32, 0.5, -2.0, seed=0).astype(np.float32)
            wl["lognormal_32^3_lin6"] = workload_line(32, 100.0, fields.linear_edges(32, 100.0, 6), f1,
                                                      args.precision, steps=50)
            f2 = fields.bubbles(256, 6.0, 0.5, seed=1).astype(np.float32)
            wl["bubbles_256^3_lin32"] = workload_line(256, 256.0, fields.linear_edges(256, 256.0, 32), f2,
                                                      args.precision, steps=10)
            line["workloads"] = wl
        except Exception as ex:
            line["workloads"] = {"error": str(ex)[:200]}
    if rank == 0 and not args.no_batch and world == 1:
        _phase("batched")
        try:
            line["batched"] = batched_run(precision=args.precision)
        except Exception as ex:
            line["batched"] = {"value": None, "error": str(ex)[:200]}
    if rank == 0 and not args.no_serve and world == 1:
        _phase("serving")
        try:
            line["serving"] = serving_run(precision=args.precision)
        except Exception as ex:
            line["serving"] = {"value": None, "error": str(ex)[:200]}
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        _phase("cpu_baseline")
        try:
            t_full, info = cpu_baseline(args)
            line["cpu_baseline"] = {"value": planB.ntrip / t_full, "unit": "triangle-bins/s",
                                    "cores": info["cores"], "kind": "oracle",
                                    "sampling_spread": info["spread"],
                                    "sample": "FP64 direct all-pairs sum (Eq. bi_direct) over a fixed sample "
                                              "of %d of %d m1 modes (every k-th binned mode, %.1f s) scaled "
                                              "to all modes, plus the call's fixed cost (%.1f s) and the FP64 "
                                              "FFT (%.1f s); the sample's two interleaved halves differ by "
                                              "%.0f%% per mode"
                                              % (info["m1_sampled"], info["m1_total"], info["sample_s"],
                                                 info["fixed_s"], info["fft_s"], 100 * info["spread"])}
        except Exception as ex:  # the baseline must not sink the bench line
            line["cpu_baseline"] = {"value": None, "error": str(ex)[:200]}
    if rank == 0:
        _phase("done")
        line["phase_s"] = dict(_PHASES)
        print(json.dumps(line), flush=True)
    planB.close()
    planT.close()
    if dist:
        dist.destroy_process_group()


def _serving_requests(n_req, rate, seed, precision, every_key=False):
    """Config-5 request stream: Poisson arrivals at `rate`, grids uniform over
    {64, 128, 192, 256, 384}, lognormal or bubble fields (50/50), 8..48
    linear bins.  A small seeded pool of fields per grid (pinned host memory)
    is cycled; requests differ in field, bins and arrival.  `every_key`: one
    request for each (grid, bin count) in a seeded random order instead (a
    warm-up that leaves every plan's counts cached)."""
    import torch
    import fields
    from paper_1705_06284_gb300.serve import Request
    rng = np.random.default_rng(seed)
    grids = [64, 128, 192, 256, 384]
    pool = {}
    for N in grids:
        pool[N] = [torch.from_numpy(fields.lognormal(N, 0.6, -2.0, seed=seed + N).astype(np.float32)).pin_memory(),
                   torch.from_numpy(fields.bubbles(N, max(3.0, N / 40), 0.5, seed=seed + 2 * N)
                                    .astype(np.float32)).pin_memory()]
    t, reqs = 0.0, []
    keys = [(N, nb) for N in grids for nb in range(8, 49)]
    if every_key:
        keys = [keys[i] for i in rng.permutation(len(keys))]
        n_req = len(keys)
    for i in range(n_req):
        t += rng.exponential(1.0 / rate)
        if every_key:
            N, nb = keys[i]
        else:
            N = int(rng.choice(grids))
            nb = int(rng.integers(8, 49))
        L = float(N)
        reqs.append(Request(i, pool[N][int(rng.integers(0, 2))].numpy(), L,
                            tuple(np.linspace(2 * math.pi / L, 0.25 * N * 2 * math.pi / L, nb + 1)),
                            arrival=t, precision=precision))
    return reqs


def serving_run(n_req=1000, rate=200.0, seed=7, budget=120 << 30, slots=4, precision="bf16x3",
                plain_max_s=60.0, deadline_s=90.0, warm_deadline_s=150.0):
    """Continuous-batching serving of a Poisson request stream (config 5), in
    `precision` and in the library's FP32, against the plain FP32 GPU path on
    the same stream.  A warm-up stream with one request per (grid, bin count)
    (205 plan keys, other seed) runs first; it leaves plans resident and every
    plan's counts cached, as a server in steady state has them.  The plain path serves the stream's
    requests one after another in arrival order (it has no overlap), given each
    request's closed triplets (plan-time information), until `plain_max_s` of
    wall time.  Each stream is refused past `deadline_s` (requests not yet
    admitted then count as refused), which bounds the phase; the two servers
    share the plan-time counts cache."""
    import torch
    from paper_1705_06284_gb300.serve import EstimatorServer, latency_percentiles
    out = {"requests": n_req, "warmup": "one request per (grid, bin count)", "arrival_rate_per_s": rate,
           "slots": slots, "hbm_budget_gib": budget >> 30, "deadline_s": deadline_s,
           "plan_slab_gib": 1}
    ref = {}
    counts = {}
    for prec in ([precision, "fp32"] if precision != "fp32" else ["fp32"]):
        srv = EstimatorServer(hbm_budget=budget, slots=slots)
        srv.counts_cache = counts
        _phase("serving warm-up (%s)" % prec)
        warm = srv.run(_serving_requests(0, rate, seed + 1000, prec, every_key=True), realtime=True,
                       deadline_s=warm_deadline_s)
        out["warmup_served_" + prec] = sum(1 for r in warm if r.error is None)
        created0, cached0 = srv.plan_creations, srv.plans_from_cache
        reqs = _serving_requests(n_req, rate, seed, prec)
        _phase("serving timed stream (%s)" % prec)
        t0 = time.perf_counter()
        res = srv.run(reqs, realtime=True, deadline_s=deadline_s)
        wall = time.perf_counter() - t0
        ok = [r for r in res if r.error is None]
        tri = sum(len(r.B) for r in ok)
        d = {"value": tri / wall, "unit": "triangle-bins/s", "wall_s": wall, "served": len(ok),
             "refused": len(res) - len(ok), "refused_deadline": sum(1 for r in res if r.error == "deadline"),
             "plans_created": srv.plan_creations - created0,
             "plans_from_cached_counts": srv.plans_from_cache - cached0,
             "plans_created_in_warmup": created0}
        d.update(latency_percentiles(res))
        srv.close()
        out["ours_" + prec] = d
        ref[prec] = {r.rid: r for r in ok}
    # the plain FP32 GPU path on the same stream, one request after another
    _phase("serving plain FP32 path")
    reqs = _serving_requests(n_req, rate, seed, "fp32")
    dev = torch.device("cuda")
    base = ref.get("fp32") or ref[precision]
    t0 = time.perf_counter()
    done_prev, lat, tri, served, worst = 0.0, [], 0, 0, 0.0
    for r in reqs:
        if time.perf_counter() - t0 > plain_max_s or r.rid not in base:
            break
        now = time.perf_counter() - t0
        if now < r.arrival:
            time.sleep(r.arrival - now)
        N = r.field.shape[0]
        import oracle  # noqa: F401  (thresholds only: same integer rule as the library's)
        thr = np.asarray(oracle.thresholds(r.edges, r.L))
        fld = torch.from_numpy(r.field).to(dev, non_blocking=True)
        num = plain_fp32_gpu(fld, N, r.L, thr, base[r.rid].triplets, dev).cpu().numpy()
        done = time.perf_counter() - t0
        lat.append(done - r.arrival)
        tri += len(num)
        served += 1
        ntri = base[r.rid].N_tri
        V, npix = r.L ** 3, float(N) ** 3
        Bp = (V * V / npix ** 3) * num / (npix * ntri)
        big = ntri >= 100
        if big.any():
            rel = np.abs(Bp[big] - base[r.rid].B[big]) / np.maximum(np.abs(base[r.rid].B[big]), 1e-300)
            worst = max(worst, float(np.median(rel)))
    wall = time.perf_counter() - t0
    lat = np.array(lat)
    out["plain_fp32"] = {"value": tri / wall if wall > 0 else None, "unit": "triangle-bins/s", "wall_s": wall,
                         "served": served, "p50_ms": float(np.percentile(lat, 50) * 1e3) if served else None,
                         "p99_ms": float(np.percentile(lat, 99) * 1e3) if served else None,
                         "median_rel_diff_vs_ours": worst,
                         "what": "cuFFT R2C + per-bin masked C2R + FP32 GEMV per outer pair, one request at a time "
                                 "in arrival order on the same stream (a prefix of it when the plain path cannot "
                                 "keep up); closed triplets given"}
    out["value"] = out["ours_" + precision]["value"]
    out["unit"] = "triangle-bins/s"
    for k in ("p50_ms", "p99_ms"):
        out[k] = out["ours_" + precision][k]
    return out


def batched_run(n_real=256, seed=1000, reps=3, precision="bf16x3"):
    """Config 4: 256 realisations with grids uniform over {64, 96, 128}^3 (half
    lognormal with sigma in [0.3, 1.0], half bubbles with R in [3, 8] cells and
    ionised fraction in [0.2, 0.8]), 24 linear bins each.  Batched launches
    (one fbs_bispectrum_batch per grid size) captured into one CUDA graph,
    against the same realisations one call at a time, at equal precision (the
    bench precision, then FP32).  The fields come from a seeded pool of 8 per
    grid size, cycled over the realisations (the work per realisation does not
    depend on the values)."""
    import torch
    import fields
    from paper_1705_06284_gb300.batch import GraphBatch
    rng = np.random.default_rng(seed)
    grids = [64, 96, 128]
    pool = {}
    for N in grids:
        lst = []
        for i in range(8):
            if i % 2 == 0:
                f = fields.lognormal(N, float(rng.uniform(0.3, 1.0)), -2.0, seed=seed + 10 * N + i)
            else:
                f = fields.bubbles(N, float(rng.uniform(3.0, 8.0)), float(rng.uniform(0.2, 0.8)),
                                   seed=seed + 10 * N + i)
            lst.append(torch.from_numpy(f.astype(np.float32)).cuda())
        pool[N] = lst
    order = [int(rng.choice(grids)) for _ in range(n_real)]
    # distinct tensors (cycled values): every realisation is its own field in memory
    fl = [pool[N][i % 8].clone() for i, N in enumerate(order)]
    L_for = lambda N: float(N)
    edges_for = lambda N: np.linspace(2 * math.pi / N, 0.25 * N * 2 * math.pi / N, 25)
    out = {"realisations": n_real, "grids": grids, "bins": 24}

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(gb.stream)
        for _ in range(reps):
            fn()
        e1.record(gb.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    for prec in ([precision, "fp32"] if precision != "fp32" else ["fp32"]):
        gb = GraphBatch(fl, L_for, edges_for, precision=prec, tune=(prec != "fp32"))
        ntri = sum(gb.groups[N]["plan"].ntrip for N, _ in gb.where)
        ms_one = timed(gb.run_one_at_a_time)
        ms_eager = timed(gb.run_eager)
        gb.capture()
        ms_graph = timed(gb.replay)
        d = {"graph_batched": {"value": ntri / (ms_graph / 1e3), "unit": "triangle-bins/s", "ms_per_batch": ms_graph},
             "eager_batched": {"value": ntri / (ms_eager / 1e3), "unit": "triangle-bins/s", "ms_per_batch": ms_eager},
             "one_at_a_time": {"value": ntri / (ms_one / 1e3), "unit": "triangle-bins/s", "ms_per_batch": ms_one},
             "graph_vs_one_at_a_time": ms_one / ms_graph,
             "launch_groups": len(gb.groups)}
        if prec != "fp32":
            d["tuning"] = {str(k): v for k, v in gb.tuning.items()}
        out[prec] = d
        gb.close()
    out["value"] = out[precision]["graph_batched"]["value"]
    out["unit"] = "triangle-bins/s"
    return out


def plain_fp32_gpu(field, N, L, thr, triplets, dev):
    """The plain FP32 GPU comparator (not the product): cuFFT R2C of the field,
    per bin a mask and a cuFFT C2R (unnormalised) to I_b, then for every
    outer pair (b, c) the FP32 product I_b I_c and FP32 dot products with the
    I_a of its triplets over x chunks, summed across chunks in FP64."""
    import torch
    f = torch.fft.rfftn(field)                     # cuFFT, unnormalised forward
    fx = torch.fft.fftfreq(N, d=1.0 / N, device=dev)
    fz = torch.arange(N // 2 + 1, device=dev, dtype=fx.dtype)
    m2 = (fx[:, None, None] ** 2 + fx[None, :, None] ** 2 + fz[None, None, :] ** 2).round().to(torch.int64)
    nb = len(thr) - 1
    I = torch.empty((nb, N * N * N), dtype=torch.float32, device=dev)
    npix = float(N) ** 3
    for b in range(nb):
        mask = (m2 >= int(thr[b])) & (m2 < int(thr[b + 1]))
        I[b] = (torch.fft.irfftn(torch.where(mask, f, torch.zeros_like(f)), s=(N, N, N)) * npix).reshape(-1)
    num = torch.zeros(len(triplets), dtype=torch.float64, device=dev)
    groups = {}
    for t, (a, b, c) in enumerate(triplets):
        groups.setdefault((int(b), int(c)), []).append((int(a), t))
    CH = 1 << 24
    for (b, c), lst in groups.items():
        aidx = torch.tensor([a for a, _ in lst], device=dev)
        tidx = torch.tensor([t for _, t in lst], device=dev)
        acc = torch.zeros(len(lst), dtype=torch.float64, device=dev)
        for x0 in range(0, N ** 3, CH):
            P = I[b, x0:x0 + CH] * I[c, x0:x0 + CH]
            acc += (I[aidx, x0:x0 + CH] @ P).double()
        num[tidx] = acc
    return num


def _closed_triplets_oracle(N, thr):
    """Closed-triplet count of the workload from the oracle alone (witness
    search over the shells), so that the reference arm never loads the CUDA
    library."""
    import oracle
    return len(oracle.closed_triplets(N, L_BOX, edges(N, len(thr) - 1)))


# DRAM bytes of one launch (dram__bytes_read.sum + dram__bytes_write.sum from
# one ncu capture of the current kernel build) per algorithmic byte of the
# launch (every bin's shell-field value of the slab read once); scaled to the
# bench's launch by its points.  A kernel class without a capture of its
# current build has no entry (the roofline's traffic is then null).
NCU_TRAFFIC_RATIO = {
    "contract_tc": ((768.424448e6 + 3.262976e6) / (54 * 3538944 * 4.0),
                    "ncu DRAM bytes of the bispectrum pass at 256^3, level M = 192, 54 bins, 3,538,944 points "
                    "(the bispectrum-pass capture of the current build), scaled by points"),
    "contract_quad_tc": ((540.220672e6 + 3.666944e6) / (16 * 8388608 * 4.0),
                         "ncu DRAM bytes of the fused triplet+quadruplet pass at 256^3, 16 log bins, "
                         "8,388,608 points (the trispectrum-pass capture of the current build), scaled by points"),
}


def max_over_ranks(dist, values, device=None):
    """Each value's maximum over the ranks (the slowest replica's time); the
    values unchanged without a process group.  NCCL groups need a CUDA
    device, gloo groups a CPU tensor (device=None)."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_rate(world, units_per_rank, seconds_max):
    """Units all replicas processed (each rank the same workload on its own
    field) over the slowest rank's time: weak scaling."""
    return world * units_per_rank / seconds_max


def _level_sets(plan):
    """Per evaluation level: (M, bins, triplets, quadruplets) of the plan."""
    out = []
    for li, lv in enumerate(plan.levels):
        tr = plan.triplets[plan.trip_level == li]
        qd = plan.quads[plan.quad_level == li] if plan.nquad else np.zeros((0, 4), dtype=np.int32)
        out.append((lv["M"], lv["nbins"], tr, qd))
    return out


def contraction_flops_per_step(plan, quads):
    """Algorithmic flops of one evaluation's contractions: per point of each
    level's grid, 2 (multiply-add) per item, plus one multiply per distinct
    outer pair product (b, c) of the triplets (and (c, d) of the quadruplets)
    and per distinct inner pair (a, b) of the quadruplets."""
    tot = 0.0
    for M, nb, tr, qd in _level_sets(plan):
        pairs = {(int(t[1]), int(t[2])) for t in tr}
        items = len(tr)
        inner = 0
        if quads:
            pairs |= {(int(q[2]), int(q[3])) for q in qd}
            inner = len({(int(q[0]), int(q[1])) for q in qd})
            items += len(qd)
        tot += float(M) ** 3 * (2 * items + len(pairs) + inner)
    return tot


def shell_field_bytes_per_step(plan):
    """Bytes of the shell fields of one evaluation (FP32, every level's bins on
    its grid): what the z stage writes and the contraction reads."""
    return sum(4.0 * nb * float(M) ** 3 for M, nb, _, _ in _level_sets(plan))


def fft_stage_bytes_per_step(plan, N, forward=True):
    """Algorithmic HBM bytes of one evaluation's FFT stage (forward R2C of the
    field and the pruned spectrum box written, unless the plan follows
    another plan's spectrum; every shell's modes read once per level that
    evaluates it; every shell field written)."""
    thr = np.asarray(plan.thresholds)
    R = int(np.floor(np.sqrt(max(int(thr[-1]) - 1, 0))))
    box = (2 * R + 1) ** 2 * (R + 1) * 8.0
    shell_read = 0.0
    for M, nb, tr, qd in _level_sets(plan):  # the modes of every bin a level's items use
        bins = set(np.unique(tr).tolist()) | set(np.unique(qd).tolist())
        shell_read += 8.0 * sum(int(plan.shell[b]) for b in bins)
    return (4.0 * N ** 3 + box if forward else 0.0) + shell_read + shell_field_bytes_per_step(plan)


def roofline(top, planB, planT, N, pk, pk_src, clocks, steps):
    """Algorithmic work of the dominant kernel class in one step / its CUDA-event
    time in one step (the sum of its launches on the plan's stream): the same
    ratio as work per launch over mean launch duration, with launches of
    several evaluation levels of different sizes."""
    name, (ms_tot, n) = top
    which, cls = name.split(":", 1)
    plan = planB if which == "B" else planT
    ms_step = ms_tot / steps
    out = {"kernel": name, "launches": n, "avg_ms": ms_tot / max(1, n), "ms_per_step": ms_step,
           "launches_per_step": n / steps}
    hbm = _find(pk, "hbm_gbs", "hbm_GBs", "copy_gbs") or 6800.0
    bf16 = _find(pk, "bf16_tflops_sustained") or 1700.0
    if cls in ("contract_fp32", "contract_quad"):
        flops = contraction_flops_per_step(plan, cls == "contract_quad")
        sm_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12  # FP32 FMA lanes x 2 flop x clock
        ach = flops / (ms_step * 1e-3) / 1e12
        out.update({"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": None,
                    "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x %.0f MHz (derived)" % sm_mhz})
    elif cls in ("contract_tc", "contract_quad_tc"):
        # the trispectrum plan's pass ("contract_quad_tc") also contracts the plan's triplets
        flops = contraction_flops_per_step(plan, cls == "contract_quad_tc")
        ach = flops / (ms_step * 1e-3) / 1e12
        ratio = NCU_TRAFFIC_RATIO.get(cls)
        # per launch, like `achieved`: the TMA ring reads every evaluated shell field once
        traffic = ratio[0] * shell_field_bytes_per_step(plan) * steps / max(1, n) if ratio else None
        out.update({"bound": "tensor", "achieved": ach, "peak": bf16, "unit": "TFLOP/s",
                    "frac": ach / bf16, "traffic": traffic,
                    "traffic_source": ratio[1] if ratio else None,
                    "peak_source": "bf16_tflops_sustained (%s)" % pk_src})
    else:
        byts = shell_field_bytes_per_step(plan) if cls == "inv_z" else \
            fft_stage_bytes_per_step(plan, N, forward=getattr(plan, "leader", None) is None)
        ach = byts / (ms_step * 1e-3) / 1e9
        out.update({"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                    "frac": ach / hbm, "traffic": None, "peak_source": "hbm_gbs (%s)" % pk_src})
    return out


FFT_CLASSES = ("fwd_z", "fwd_y", "fwd_x", "inv_x", "inv_y", "inv_z")


def roofline_fft(kB, kT, planB, planT, N, pk, pk_src, steps):
    """The FFT stage of a step (forward and pruned inverse transforms of both
    plans) against HBM: algorithmic bytes / summed FFT kernel time."""
    hbm = _find(pk, "hbm_gbs", "hbm_GBs", "copy_gbs") or 6800.0
    ms = sum(kB.get(c, (0, 0))[0] + kT.get(c, (0, 0))[0] for c in FFT_CLASSES) / steps
    byts = fft_stage_bytes_per_step(planB, N, forward=getattr(planB, "leader", None) is None) + \
        fft_stage_bytes_per_step(planT, N, forward=getattr(planT, "leader", None) is None)
    ach = byts / (ms * 1e-3) / 1e9
    zb = shell_field_bytes_per_step(planB) + shell_field_bytes_per_step(planT)
    zms = (kB.get("inv_z", (0, 0))[0] + kT.get("inv_z", (0, 0))[0]) / steps
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "bytes_per_step": byts, "ms_per_step": ms,
            "inv_z": {"achieved": zb / (zms * 1e-3) / 1e9, "frac": zb / (zms * 1e-3) / 1e9 / hbm,
                      "bytes_per_step": zb, "ms_per_step": zms},
            "peak_source": "hbm_gbs (%s)" % pk_src,
            "what": "fwd_z/y/x (once: the trispectrum plan follows the bispectrum plan's spectrum) + inv_x/y/z of both plans; bytes: field read, spectrum box written, "
                    "shell modes read per level, shell fields written"}


def cufft_fft_stage(field, N, thr, dev, reps=3):
    """cuFFT alone doing the FFT work of the plain method for the bispectrum
    plan's bins (comparison only): R2C of the field, then per bin a masked
    C2R on the full N^3 grid.  Returns ms per field."""
    import torch
    fx = torch.fft.fftfreq(N, d=1.0 / N, device=dev)
    fz = torch.arange(N // 2 + 1, device=dev, dtype=fx.dtype)
    m2 = (fx[:, None, None] ** 2 + fx[None, :, None] ** 2 + fz[None, None, :] ** 2).round().to(torch.int64)
    masks = [((m2 >= int(thr[b])) & (m2 < int(thr[b + 1]))) for b in range(len(thr) - 1)]
    masks = [m for m in masks if bool(m.any())]
    out = torch.empty((N, N, N), dtype=torch.float32, device=dev)

    def once():
        f = torch.fft.rfftn(field)
        for m in masks:
            out.copy_(torch.fft.irfftn(f * m, s=(N, N, N)))
    once()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        once()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, len(masks)


def workload_line(N, L, edges, field32, precision, steps=10, warmup=3):
    """Throughput of one workload through the library (device field and
    outputs): closed triplets x fields / time, CUDA events on the plan's stream."""
    import torch
    import paper_1705_06284_gb300 as fbs
    f = torch.from_numpy(field32).cuda()
    with fbs.Plan(N, L, edges, precision=precision) as plan:
        B = torch.empty(plan.ntrip, dtype=torch.float64, device=f.device)
        P = torch.empty(plan.nbins, dtype=torch.float64, device=f.device)
        for _ in range(warmup):
            plan.bispectrum(f, B, P)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            plan.bispectrum(f, B, P)
        e1.record()
        torch.cuda.synchronize()
        plan.check()
        ms = e0.elapsed_time(e1) / steps
        return {"value": plan.ntrip / (ms * 1e-3), "unit": "triangle-bins/s", "ms_per_field": ms,
                "ntrip": plan.ntrip, "precision": precision, "levels": [l["M"] for l in plan.levels]}


if __name__ == "__main__":
    main()
