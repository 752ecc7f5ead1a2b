#!/usr/bin/env python
"""Benchmark of the AINV-preconditioned CG solve of the ocean free-surface
system (PCG solves/s at rtol 1e-10; HBM GB/s per iteration; roofline of the
dominant kernel) on one B300, or on N GPUs as independent replicas.

Step = one complete solve (pack b, r0 = b - A x0, s0 = M^-1 r0, the PCG loop
to ||r|| / ||b|| <= 1e-10, final x update, true-residual check, unpack x) of a
synthetic seeded grid through the library's C ABI. The factor is built once
before timing (as in the paper, where it is a setup step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import gridgen  # noqa: E402

METRIC = "PCG solves/s & HBM GB/s per iter at rtol 1e-10, mixed vs FP64; p99 latency"
UNIT = "solves/s"

# pattern codes of the C ABI
TRIL_A, TRIL_A2, BAND_T, DIAG = 0, 1, 3, 4

WORKLOADS = {
    # the largest grid of the configurations (eddy-resolving, 13.2M points): the
    # working set (~1.5 GB) is far above the 126 MB L2, so every iteration streams HBM
    "orca12-fp64": dict(grid=gridgen.ORCA12, ci=4, pattern=TRIL_A2, tau=0.05, q=0, prec=0, rtol=1e-10),
    "orca12-fp64-trilA": dict(grid=gridgen.ORCA12, ci=4, pattern=TRIL_A, tau=0.0, q=0, prec=0, rtol=1e-10),
    "orca025-fp64": dict(grid=gridgen.ORCA025, ci=2, pattern=TRIL_A2, tau=0.05, q=0, prec=0, rtol=1e-10),
    "coarse-fp64": dict(grid=gridgen.COARSE, ci=1, pattern=TRIL_A2, tau=0.05, q=0, prec=0, rtol=1e-10),
    # binary32 inner PCG inside binary64 iterative refinement, same acceptance (true residual <= 1e-10)
    "orca12-mixed": dict(grid=gridgen.ORCA12, ci=4, pattern=TRIL_A2, tau=0.05, q=0, prec=1, rtol=1e-10),
    "orca12-mixed-trilA": dict(grid=gridgen.ORCA12, ci=4, pattern=TRIL_A, tau=0.0, q=0, prec=1, rtol=1e-10),
    "orca025-mixed": dict(grid=gridgen.ORCA025, ci=2, pattern=TRIL_A2, tau=0.05, q=0, prec=1, rtol=1e-10),
    # 64 ensemble members of uneven sizes (182x149 .. 1442x1021), one batched call per step
    "batch64-mixed": dict(kind="batch", ci=3, pattern=TRIL_A2, tau=0.05, q=0, prec=1, rtol=1e-10, members=64),
    "batch64-fp64": dict(kind="batch", ci=3, pattern=TRIL_A2, tau=0.05, q=0, prec=0, rtol=1e-10, members=64),
    # open-loop Poisson stream (200 req/s) over resident grids, continuous batching
    "serve-mixed": dict(kind="serve", ci=4, pattern=TRIL_A2, tau=0.05, q=0, prec=1, rtol=1e-10, rate=200.0,
                        seconds=60.0, warm_s=5.0),
}
BATCH_SIZES = [gridgen.COARSE, gridgen.ORCA1, gridgen.ORCA05, gridgen.ORCA025]
DEFAULT_WORKLOAD = "orca12-fp64"

# FP64 arithmetic of this B300 from its unit counts and clock, for comparison
# with the measured rate (pcg_fp64_fma_rate): 2 FMA per clock per SM, 148 SMs,
# 2.032 GHz maximum SM clock, 2 flops per FMA.
FP64_DERIVED_TFLOPS = 2 * 148 * 2.032e9 * 2 / 1e12


def measure_fp64_peak(pcg, gpu):
    """The binary64 FMA rate of this GPU, measured by the library's own kernel
    (independent FMA chains, one full wave of resident blocks, CUDA events),
    best of three runs of 10 launches, with the SM clock sampled meanwhile."""
    sampler = _sample_clocks(gpu)
    runs = [pcg.pcg_fp64_fma_rate(10) for _ in range(3)]
    clocks = sampler.stop()
    best = max(r[0] for r in runs)
    return {"tflops": best, "runs_tflops": [r[0] for r in runs], "ms_per_launch": min(r[1] for r in runs),
            "derived_tflops": FP64_DERIVED_TFLOPS, "frac_of_derived": best / FP64_DERIVED_TFLOPS, "clocks": clocks}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mp = json.load(f)
        return float(mp["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _z_offdiag_per_wet(pcg, h):
    D, rows, vals = pcg.pcg_ainv_export(h)
    return float((rows >= 0).sum()) / max(len(D), 1)


def _record_iterations():
    path = os.path.join(ROOT, "oracle", "iterations.json")
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def oracle_prepare(wl, grid):
    """Oracle setup for a workload: assembly and factor (untimed, like the GPU's)."""
    import oracle
    P = oracle.OracleProblem.from_grid(grid)
    assert P.ainv(wl["pattern"], wl["tau"], wl["q"]) == oracle.OK
    return P, P.to_wet(grid.b)


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _mem_available():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 8 << 30


def _save_grid(grid, path):
    np.savez(path, nx=grid.nx, ny=grid.ny, wet=grid.wet, c_e=grid.c_e, c_n=grid.c_n, shift=grid.shift, b=grid.b)


def _load_oracle(path, pattern, tau, q):
    sys.path.insert(0, ROOT)
    import oracle
    d = np.load(path)
    P = oracle.OracleProblem(int(d["nx"]), int(d["ny"]), d["wet"], d["c_e"], d["c_n"], d["shift"])
    assert P.ainv(pattern, tau, q) == oracle.OK
    return P, P.to_wet(d["b"])


def _oracle_tight_worker(grid_path, out_path, pattern, tau, q):
    """Spawned process: the oracle's own PCG to rtol 1e-13 (a tight reference
    solution of A x = b), written as the wet-compressed vector."""
    P, b = _load_oracle(grid_path, pattern, tau, q)
    res = P.pcg(b, rtol=1e-13, max_iter=20 * P.n)
    np.save(out_path, res.x)


def _oracle_solve_worker(grid_path, pattern, tau, q, rtol, barrier, queue):
    """Spawned process: one whole oracle solve of its own replica of the
    workload, timed after every worker has built its factor."""
    P, b = _load_oracle(grid_path, pattern, tau, q)
    barrier.wait()
    t = time.perf_counter()
    res = P.pcg(b, rtol=rtol)
    queue.put((time.perf_counter() - t, res.iters, res.status))


def start_tight_reference(grid_path, out_path, wl):
    """The oracle's tight reference of the workload, computed in a spawned
    process while the GPU is measured."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    proc = ctx.Process(target=_oracle_tight_worker, args=(grid_path, out_path, wl["pattern"], wl["tau"], wl["q"]))
    proc.start()
    return proc


def oracle_baseline(grid_path, wl, grid):
    """The FP64 CPU oracle, as it stands, on the workload itself: one whole
    solve on one host core, then one whole solve per worker process on as many
    host cores as memory allows (about 3.5 GB per full-size oracle), all
    started together; aggregate solves/s = workers / slowest worker's time."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    args = (grid_path, wl["pattern"], wl["tau"], wl["q"], wl["rtol"])

    def run(n):
        barrier, queue = ctx.Barrier(n), ctx.Queue()
        procs = [ctx.Process(target=_oracle_solve_worker, args=args + (barrier, queue)) for _ in range(n)]
        for p_ in procs:
            p_.start()
        out = [queue.get() for _ in range(n)]
        for p_ in procs:
            p_.join()
        return out

    one = run(1)[0]
    per_worker = 3.5e9 * (grid.nx * grid.ny) / 13.2e6
    n_all = max(1, min(os.cpu_count() or 1, int(_mem_available() * 0.8 / max(per_worker, 1e8))))
    allr = run(n_all)
    slowest = max(r[0] for r in allr)
    model = _cpu_model()
    return {"value": 1.0 / one[0], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one whole serial FP64 oracle solve of the {grid.nx}x{grid.ny} workload at rtol "
                      f"{wl['rtol']:g} ({one[1]} iterations, {one[0]:.3g} s, status {one[2]}), factor built before",
            "cpu_model": model, "nproc": os.cpu_count(),
            "all_cores": {"value": n_all / slowest, "unit": UNIT, "cores": n_all, "kind": "oracle",
                          "sample": f"{n_all} concurrent processes, one whole oracle solve each of its own replica "
                                    f"of the workload (slowest {slowest:.3g} s, fastest "
                                    f"{min(r[0] for r in allr):.3g} s); workers limited by host memory"
                                    f" ({_mem_available() / 2**30:.0f} GiB available) and cores",
                          "cpu_model": model}}


def oracle_sample(wl_name, wl, grid, prepared, seconds_target=15.0):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload:
    a run of whole oracle PCG iterations on the full grid. Returns the sample's
    wall time and the fraction of a solve it covers (its iterations over the
    oracle's own iteration count for this grid and preconditioner, recorded by
    oracle/record_iterations.py)."""
    P, b = prepared
    t = time.perf_counter()
    P.pcg(b, rtol=0.0, max_iter=2, max_replace=0)
    t2 = time.perf_counter() - t
    iters = max(2, min(200, int(seconds_target / max(t2 / 2, 1e-6))))
    t = time.perf_counter()
    P.pcg(b, rtol=0.0, max_iter=iters, max_replace=0)
    dt = time.perf_counter() - t
    recs = _record_iterations()
    rec = recs.get(wl_name) or recs.get(wl_name.replace("-mixed", "-fp64"))
    if rec is None:
        rec = P.pcg(b, rtol=wl["rtol"]).iters
    return dt, iters / rec, iters, rec


def run_reference(args, wl_name, wl):
    """The reference arm: the FP64 CPU oracle as it stands (the paper ships no
    code), on one host core. A step is a bounded sample of whole oracle PCG
    iterations of the workload; value = solves covered by the timed steps over
    their time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    grid = gridgen.make_grid(seed=gridgen.seed_for(wl["ci"]), **wl["grid"])
    prepared = oracle_prepare(wl, grid)
    times, fracs, last = [], [], None
    for step in range(args.warmup + args.steps):
        dt, frac, iters, rec = oracle_sample(wl_name, wl, grid, prepared, seconds_target=args.ref_seconds)
        if step >= args.warmup:
            times.append(dt)
            fracs.append(frac)
            last = (iters, rec, dt)
    val = sum(fracs) / sum(times)
    sample = (f"{last[0]} serial FP64 oracle PCG iterations per step on the full {grid.nx}x{grid.ny} grid "
              f"(incl. the initial and final residuals; {last[2]:.1f} s), {last[0]}/{last[1]} of the oracle's "
              f"iterations per solve at rtol {wl['rtol']:g}")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl_name, "grid": f"{grid.nx}x{grid.ny}", "n_wet": int(grid.wet.sum()),
                   "pattern": wl["pattern"], "drop_tol": wl["tau"], "rtol": wl["rtol"],
                   "solves_per_step": sum(fracs) / len(fracs)},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "cpu_model": _cpu_model()},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _traffic_record(kernel_key, tiles):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the
    current kernel source and strip shape (profiles/traffic.txt: key bytes
    source_sha tiles)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    src = os.path.join(ROOT, "paper_1210_1878_b300", "csrc", "kernels.cuh")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        for line in open(path):
            p = line.split()
            if len(p) >= 4 and p[0] == kernel_key and p[2] == sha and p[3] == tiles:
                return float(p[1])
    except Exception:
        pass
    return None


def _sample_clocks(gpu):
    c = ClockSampler(gpu)
    c.start()
    time.sleep(0.3)
    return c


def _setup_grids(pcg, specs, setup_kw):
    """Generate and factor grids on host threads (the library's set-up call
    releases the interpreter lock); returns (grids, handles, seconds)."""
    from concurrent.futures import ThreadPoolExecutor
    t = time.perf_counter()

    def one(spec):
        cfg, seed = spec
        g = gridgen.make_grid(seed=seed, **cfg)
        return g, pcg.ainv_setup_grid(g, **setup_kw)

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        out = list(ex.map(one, specs))
    return [o[0] for o in out], [o[1] for o in out], time.perf_counter() - t


def _time_batched(pcg, torch, hs, bs, xs, opts, steps, warmup):
    for _ in range(warmup):
        pcg.pcg_solve_batched(hs, bs, xs, opts)
    torch.cuda.synchronize()
    l0 = pcg.pcg_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    worst = 0.0
    for _ in range(steps):
        rc, stats = pcg.pcg_solve_batched(hs, bs, xs, opts)
        worst = max(worst, max(st.true_relres for st in stats))
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"value": len(hs) / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "worst_true_relres": worst, "gpu_launches": int(pcg.pcg_kernel_launches() - l0)}


def measure_batch(args, wl, steps, warmup):
    """64 uneven ensemble grids (configuration: sizes drawn from 182x149 ..
    1442x1021, one seed each). Timed: the 64 as sequential binary64 single
    solves on the strips a single solve gets by default; then, with strip
    shapes autotuned for a batch member (objective 1), one pcg_solve_batched
    call per step in binary64 and in the mixed mode (every launch covers the
    work units of all unconverged members; the loop runs in one graph)."""
    import torch
    import paper_1210_1878_b300 as pcg
    rng = np.random.default_rng(gridgen.seed_for(wl["ci"]))
    picks = rng.integers(0, len(BATCH_SIZES), size=wl["members"])
    specs = [(BATCH_SIZES[k], gridgen.seed_for(wl["ci"], m)) for m, k in enumerate(picks)]
    grids, hs, setup_s = _setup_grids(pcg, specs, dict(pattern=wl["pattern"], drop_tol=wl["tau"],
                                                       tile_x=args.tile_x, tile_y=args.tile_y))
    bs = [torch.from_numpy(g.b).cuda() for g in grids]
    xs = [torch.zeros_like(b) for b in bs]
    o64 = pcg.make_opts(rtol=wl["rtol"], max_iter=5000, prec=0)
    om = pcg.make_opts(rtol=wl["rtol"], max_iter=5000, prec=1, inner_rtol=args.inner_rtol)
    # sequential binary64 single solves (default strips), one warm pass
    for h, b, x in zip(hs, bs, xs):
        pcg.pcg_solve(h, b, x, o64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    worst_seq = 0.0
    for h, b, x in zip(hs, bs, xs):
        worst_seq = max(worst_seq, pcg.pcg_solve(h, b, x, o64).true_relres)
    e1.record()
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    sampler = _sample_clocks(int(os.environ.get("LOCAL_RANK", "0")))
    t = time.perf_counter()
    tiles = {0: {}, 1: {}}
    for prec in (0, 1):
        if not args.tile_x and not args.tile_y:
            for h, g in zip(hs, grids):
                tiles[prec][f"{g.nx}x{g.ny}"] = list(pcg.pcg_autotune(h, prec, objective=1))
    tune_s = time.perf_counter() - t
    fp64 = _time_batched(pcg, torch, hs, bs, xs, o64, steps, warmup)
    mixed = _time_batched(pcg, torch, hs, bs, xs, om, steps, warmup)
    clocks = sampler.stop()
    # end to end (mixed) with pinned host buffers
    bh = [torch.from_numpy(g.b.copy()).pin_memory() for g in grids]
    xh = [torch.zeros_like(b).pin_memory() for b in bh]
    pcg.pcg_solve_batched(hs, bh, xh, om)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(max(1, args.e2e_steps)):
        pcg.pcg_solve_batched(hs, bh, xh, om)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / max(1, args.e2e_steps)
    vec_bytes = sum(g.nx * g.ny * 8 for g in grids)
    sizes = {}
    for g in grids:
        sizes[f"{g.nx}x{g.ny}"] = sizes.get(f"{g.nx}x{g.ny}", 0) + 1
    out = {"workload": "batch64", "members": len(hs), "sizes": sizes, "pattern": "tril(A^2)",
           "drop_tol": wl["tau"], "rtol": wl["rtol"],
           "mixed_batched": mixed, "fp64_batched": fp64,
           "fp64_sequential": {"value": len(hs) / (seq_ms / 1e3), "unit": UNIT, "ms_per_batch": seq_ms,
                               "worst_true_relres": worst_seq},
           "e2e_mixed": {"value": len(hs) / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": vec_bytes,
                         "d2h_bytes_per_step": vec_bytes},
           "setup_s": setup_s, "autotune_s": tune_s,
           "tiles_autotuned": {"fp64": tiles[0], "mixed": tiles[1]},
           "resident_gb": sum(h.resident_bytes for h in hs) / 1e9, "clocks": clocks}
    for h in hs:
        h.close()
    return out


def run_batch(args, wl_name, wl):
    blk = measure_batch(args, wl, args.steps, args.warmup)
    main = blk["mixed_batched"] if wl["prec"] == 1 else blk["fp64_batched"]
    line = {
        "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if wl["prec"] == 1 else "f64", "data": "synthetic",
        "config": {"workload": wl_name, **{k: v for k, v in blk.items() if k not in ("clocks", "e2e_mixed")}},
        "e2e": blk["e2e_mixed"] if wl["prec"] == 1 else None,
        "gpu_launches": main["gpu_launches"], "clocks": blk["clocks"],
    }
    print(json.dumps(line))
    return 0


def measure_serve(args, wl, seconds, warm_s):
    """Open-loop Poisson arrivals (mean rate wl['rate']) of solve requests over a
    resident pool of grids (8 x 362x292, 4 x 1442x1021, 2 x 4322x3059; requests
    pick a size 60/30/10 and a grid of that size uniformly); each request is
    the next timestep of its grid (b <- b + 0.01 N(0,1), warm start from the
    last solution). Latency = scheduled arrival -> completion; requests that
    arrive in the first warm_s seconds are not counted."""
    import torch
    import paper_1210_1878_b300 as pcg
    rng = np.random.default_rng(gridgen.seed_for(wl["ci"]))
    pool = [(gridgen.ORCA1, 8), (gridgen.ORCA025, 4), (gridgen.ORCA12, 2)]
    if args.serve_small:
        pool = [(gridgen.ORCA1, 8), (gridgen.ORCA025, 4)]
    specs, size_of = [], []
    for si, (cfg, cnt) in enumerate(pool):
        for m in range(cnt):
            specs.append((cfg, gridgen.seed_for(wl["ci"], 10 * si + m)))
            size_of.append(si)
    grids, hs, setup_s = _setup_grids(pcg, specs, dict(pattern=wl["pattern"], drop_tol=wl["tau"]))
    # strip shapes for the grids as members of the server's mix (throughput objective)
    tiles = {f"{g.nx}x{g.ny}": list(pcg.pcg_autotune(h, wl["prec"], objective=1)) for h, g in zip(hs, grids)}
    opts = pcg.make_opts(rtol=wl["rtol"], max_iter=5000, prec=wl["prec"], inner_rtol=args.inner_rtol)
    srv = pcg.Server(hbm_budget_bytes=150 << 30, max_slots=16, chunk_iters=args.chunk, opts=opts)
    gids = [srv.register(h) for h in hs]
    # timestep increments (two per grid, reused cyclically, land already zero),
    # right-hand sides and outputs all on the device
    cur, noise, outs = [], [], []
    for k, g in enumerate(grids):
        wet = torch.from_numpy(g.wet.astype(np.float64)).cuda()
        cur.append(torch.from_numpy(g.b).cuda())
        noise.append([wet * torch.from_numpy(0.01 * np.random.default_rng(1000 * k + j).standard_normal((g.ny, g.nx))).cuda()
                      for j in range(2)])
        outs.append(torch.zeros((g.ny, g.nx), dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    total = seconds + warm_s
    gaps = rng.exponential(1.0 / wl["rate"], size=int(wl["rate"] * total * 1.5) + 10)
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < total]
    size_pick = rng.choice(3 if not args.serve_small else 2, size=len(arrivals),
                           p=[0.6, 0.3, 0.1] if not args.serve_small else [2 / 3, 1 / 3])
    by_size = {si: [k for k, s_ in enumerate(size_of) if s_ == si] for si in set(size_of)}
    grid_pick = [by_size[sp][rng.integers(0, len(by_size[sp]))] for sp in size_pick]
    steps_done = [0] * len(grids)
    ids, late, call_ms = [], [], []
    sampler = _sample_clocks(int(os.environ.get("LOCAL_RANK", "0")))
    t0 = time.perf_counter()
    for t_arr, k in zip(arrivals, grid_pick):
        now = time.perf_counter() - t0
        if t_arr > now:
            time.sleep(t_arr - now)
        else:
            late.append(now - t_arr)
        ta = time.perf_counter()
        cur[k].add_(noise[k][steps_done[k] % 2])
        steps_done[k] += 1
        tb = time.perf_counter()
        rid = srv.submit(gids[k], cur[k], outs[k], warm_start=True)
        tc = time.perf_counter()
        call_ms.append(((tb - ta) * 1e3, (tc - tb) * 1e3))
        ids.append((t_arr, k, rid, tc - t0))
    results = []
    for t_arr, k, rid, t_sub in ids:
        rc, st = srv.wait(rid, timeout_ms=600000)
        # latency from the scheduled arrival (so a late submission counts against it)
        results.append((t_arr, k, rc, st.seconds + (t_sub - t_arr), st.true_relres, st.iters))
    elapsed = time.perf_counter() - t0
    clocks = sampler.stop()
    srv_stats = srv.stats()
    srv.close()
    for h in hs:
        h.close()
    meas = [r for r in results if r[0] >= warm_s]
    lat = np.array([r[3] * 1e3 for r in meas])
    ok = [r for r in meas if r[2] == pcg.PCG_OK]

    def pct(a, q):
        if len(a) == 0:
            return None
        srt = np.sort(a)
        return float(srt[min(len(srt) - 1, max(0, int(math.ceil(q * len(srt))) - 1))])

    per_size = {}
    for si in sorted(set(size_of)):
        ls_ = np.array([r[3] * 1e3 for r in meas if size_of[r[1]] == si])
        cfg = pool[si][0]
        per_size[f"{cfg['nx']}x{cfg['ny']}"] = {"n": int(len(ls_)), "p50_ms": pct(ls_, 0.5), "p99_ms": pct(ls_, 0.99)}
    return {"workload": "serve", "value": len(results) / elapsed, "unit": UNIT,
            "precision": "binary32 inner / binary64 refinement" if wl["prec"] == 1 else "binary64",
            "arrival_rate_per_s": wl["rate"], "seconds": seconds, "warm_s": warm_s,
            "requests": len(results), "measured": len(meas),
            "failed": len(results) - sum(1 for r in results if r[2] == pcg.PCG_OK),
            "latency_ms": {"p50": pct(lat, 0.5), "p99": pct(lat, 0.99),
                           "mean": float(lat.mean()) if len(lat) else None, "per_size": per_size},
            "worst_true_relres": max((r[4] for r in ok), default=None),
            "submit_late_p99_ms": (float(np.percentile(late, 99)) * 1e3) if late else 0.0,
            "client_submit_ms_p99": float(np.percentile([c[1] for c in call_ms], 99)) if call_ms else 0.0,
            "grids": {f"{c['nx']}x{c['ny']}": n for c, n in pool}, "hbm_budget_gb": 150, "max_slots": 16,
            "chunk_iters": args.chunk, "tiles_autotuned": tiles, "setup_s": setup_s,
            "server_stats": srv_stats, "clocks": clocks}


def run_serve(args, wl_name, wl):
    seconds = args.serve_seconds if args.serve_seconds > 0 else wl["seconds"]
    blk = measure_serve(args, wl, seconds, min(wl["warm_s"], seconds / 4))
    line = {
        "metric": METRIC, "value": blk["value"], "unit": UNIT, "n_gpus": 1, "steps": blk["requests"], "warmup": 0,
        "ms_per_step": 1e3 / blk["value"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if wl["prec"] == 1 else "f64", "data": "synthetic",
        "config": {"workload": wl_name, **{k: v for k, v in blk.items()
                                            if k not in ("latency_ms", "server_stats", "clocks", "value")}},
        "latency_ms": blk["latency_ms"], "server_stats": blk["server_stats"], "clocks": blk["clocks"],
    }
    print(json.dumps(line))
    return 0


def _kernel_roofline(pcg, h, b, wl, prec, n_wet, zbar, workload, fp64_peak):
    """Per-kernel roofline, live: mean CUDA-event duration of each of the two
    kernels of an iteration over 20 launches, against the algorithmic bytes
    (or binary64 flops) of one launch. fp64_peak: (TFLOP/s, how it was
    obtained) of the FP64 pipe."""
    mixed = prec == 1
    ms_k1, ms_k2 = pcg.pcg_profile_kernels(h, b, iters=20, prec=prec)
    w = 4 if mixed else 8
    bytes_k1 = n_wet * w * 9                   # read s, d, x, a, c_e, c_n; write d, x, q
    bytes_k2 = n_wet * w * (5 + zbar)          # read r, q, Z, D^-1; write r, s
    flops_k1 = n_wet * 15.0                    # d (1 FMA), x (1 FMA), A d (1 mul + 4 FMA), d.q (1 FMA)
    flops_k2 = n_wet * (4 * zbar + 7)          # r (1 FMA), Z^T (zbar FMA + 1 mul), Z (zbar FMA), 2 dots
    fp64_k1 = flops_k1 if not mixed else n_wet * 2.0          # binary32 kernels: only the dots in binary64
    fp64_k2 = flops_k2 if not mixed else n_wet * 4.0
    hbm_peak, peak_kind = _peaks()
    dom = "k_precond" if ms_k2 >= ms_k1 else "k_stencil"
    ms_dom, by, fl = (ms_k2, bytes_k2, fp64_k2) if dom == "k_precond" else (ms_k1, bytes_k1, fp64_k1)
    gbs = by / (ms_dom * 1e-3) / 1e9
    tflops = fl / (ms_dom * 1e-3) / 1e12
    t_hbm = by / (hbm_peak * 1e9)
    fp64_tflops, fp64_kind = fp64_peak
    t_alu = fl / (fp64_tflops * 1e12)
    kname = dom + ("<float>" if mixed else "<double>")
    tiles = "%dx%d" % pcg.pcg_tiles(h, prec)
    traffic = _traffic_record(f"{kname}:{workload}", tiles)
    if t_alu > t_hbm:
        roof = {"bound": "alu", "achieved": tflops, "peak": fp64_tflops, "unit": "TFLOP/s",
                "frac": tflops / fp64_tflops, "traffic": traffic, "peak_kind": fp64_kind,
                "hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                        "peak_kind": peak_kind + " (of measured copy bandwidth)" if peak_kind == "measured" else peak_kind}}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "traffic": traffic, "peak_kind": peak_kind}
    it_bytes = bytes_k1 + bytes_k2
    if traffic is not None:
        # the ncu DRAM bytes of one launch over the live launch time
        roof["dram_gbs"] = traffic / (ms_dom * 1e-3) / 1e9
        roof["dram_frac"] = roof["dram_gbs"] / hbm_peak
    roof.update({"kernel": kname, "tiles": tiles, "ms_per_launch": ms_dom, "alg_bytes_per_launch": by,
                 "per_iteration": {"ms_stencil": ms_k1, "ms_precond": ms_k2, "alg_bytes": it_bytes,
                                   "alg_gbs": it_bytes / ((ms_k1 + ms_k2) * 1e-3) / 1e9,
                                   "hbm_frac": it_bytes / ((ms_k1 + ms_k2) * 1e-3) / 1e9 / hbm_peak}})
    return roof


def _l2_label(torch, ws_bytes):
    """Whether one iteration's working set (the algorithmic bytes of the two
    kernels) streams from HBM or can stay in the L2 between iterations; for an
    L2-resident grid a fraction of the HBM roofline is not meaningful. The L2
    is split between the GPU's two dies: an 82 MB working set (1442 x 1021,
    binary32) still hit the L2 only 51-54 % of the time (ncu, warm caches), so
    half the L2 is the bound used here."""
    try:
        l2 = int(torch.cuda.get_device_properties(0).L2_cache_size)
    except Exception:
        l2 = 126 * 2 ** 20
    if ws_bytes > l2 // 2:
        return ("streams from HBM (working set ~%.3f GB per iteration vs %d MB L2, %d MB per die)"
                % (ws_bytes / 1e9, l2 >> 20, l2 >> 21))
    return ("L2-resident (working set ~%.1f MB per iteration within one die's %d MB of L2): the HBM "
            "fraction is not meaningful here" % (ws_bytes / 1e6, l2 >> 21))


def max_over_ranks(value, device="cuda"):
    """The maximum of a per-rank float over the process group (the slowest
    rank's time decides a replicated run); the value itself when not
    distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicated_rate(units_per_rank, ms_max, world):
    """Whole-job throughput of N independent replicas: every rank did the
    same units, the job took the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1e3)


def _time_solves(pcg, torch, h, b, x, opts, steps, warmup, stream, barrier, world):
    for _ in range(warmup):
        st = pcg.pcg_solve(h, b, x, opts)
    barrier()
    torch.cuda.synchronize()
    l0 = pcg.pcg_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for _ in range(steps):
        stats.append(pcg.pcg_solve(h, b, x, opts))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = pcg.pcg_kernel_launches() - l0
    ms = max_over_ranks(e0.elapsed_time(e1))
    assert all(s.status == pcg.PCG_OK for s in stats), [s.as_dict() for s in stats if s.status]
    return ms, stats, launches


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--ref-seconds", type=float, default=4.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="binary64 workloads: skip the mixed-precision companion")
    ap.add_argument("--no-batch", action="store_true", help="default workload: skip the batch block")
    ap.add_argument("--no-serve", action="store_true", help="default workload: skip the serving block")
    ap.add_argument("--no-err", action="store_true", help="skip the error against the oracle's tight reference")
    ap.add_argument("--no-shard", action="store_true", help="default workload: skip the row-band block")
    ap.add_argument("--no-fp64-peak", action="store_true",
                    help="use the derived FP64 peak instead of measuring it (for launch-list profiling)")
    ap.add_argument("--serve-block-seconds", type=float, default=20.0)
    ap.add_argument("--kernels-only", action="store_true",
                    help="set up the workload and launch each kernel of an iteration 3 times (for ncu)")
    ap.add_argument("--inner-rtol", type=float, default=0.0)
    ap.add_argument("--tile-x", type=int, default=0)
    ap.add_argument("--tile-y", type=int, default=0)
    ap.add_argument("--chunk", type=int, default=8)
    ap.add_argument("--serve-seconds", type=float, default=0.0)
    ap.add_argument("--serve-small", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, args.workload, wl)
    if wl.get("kind") == "batch":
        return run_batch(args, args.workload, wl)
    if wl.get("kind") == "serve":
        return run_serve(args, args.workload, wl)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # each rank solves its own replica of the workload (independent problems)
    grid = gridgen.make_grid(seed=gridgen.seed_for(wl["ci"]), **wl["grid"])
    solo = rank == 0 and world == 1 and not args.kernels_only
    tmpdir = tight = None
    if solo and not (args.no_err and args.no_cpu_baseline):
        # the oracle's inputs on disk for its processes; the tight reference is
        # computed in a spawned process while the GPU is measured
        import tempfile
        tmpdir = tempfile.mkdtemp(prefix="pcg_bench_")
        grid_path = os.path.join(tmpdir, "grid.npz")
        _save_grid(grid, grid_path)
        if not args.no_err:
            tight = start_tight_reference(grid_path, os.path.join(tmpdir, "x_ref.npy"), wl)

    import torch
    import paper_1210_1878_b300 as pcg

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    t = time.perf_counter()
    h = pcg.ainv_setup_grid(grid, pattern=wl["pattern"], drop_tol=wl["tau"], band_q=wl["q"], tile_x=args.tile_x,
                            tile_y=args.tile_y)
    setup_s = time.perf_counter() - t
    n_wet = h.n_wet
    stream = torch.cuda.current_stream()
    b = torch.from_numpy(grid.b).cuda()
    x = torch.zeros_like(b)
    if args.kernels_only:
        ms = pcg.pcg_profile_kernels(h, b, iters=3, prec=wl["prec"])
        print(json.dumps({"ms_stencil": ms[0], "ms_precond": ms[1], "tiles": "%dx%d" % pcg.pcg_tiles(h, wl["prec"])}))
        h.close()
        return 0
    zbar = _z_offdiag_per_wet(pcg, h)
    opts = pcg.make_opts(rtol=wl["rtol"], max_iter=5000, prec=wl["prec"], inner_rtol=args.inner_rtol)
    if args.no_fp64_peak:
        fp64 = {"tflops": FP64_DERIVED_TFLOPS, "derived_tflops": FP64_DERIVED_TFLOPS, "measured": False}
        fp64_peak = (FP64_DERIVED_TFLOPS, "derived: 2 FMA per clock per SM x 148 SMs x 2.032 GHz (not measured in this run)")
    else:
        fp64 = measure_fp64_peak(pcg, local)
        fp64_peak = (fp64["tflops"], "measured: binary64 FMA rate of this GPU (pcg_fp64_fma_rate, best of 3 x 10 "
                                     "launches at SM clock %s MHz)" % fp64["clocks"].get("sm_mhz"))

    for _ in range(args.warmup):
        pcg.pcg_solve(h, b, x, opts)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ms, stats, launches = _time_solves(pcg, torch, h, b, x, opts, args.steps, 0, stream, barrier, world)
    clocks = sampler.stop()
    x_main = x.cpu().numpy()
    st = stats[-1]
    iters = st.iters
    ms_per_step = ms / args.steps
    value = replicated_rate(args.steps, ms, world)
    worst_true = max(s.true_relres for s in stats)

    # end to end through the C ABI with pinned host buffers (copies inside the timed region):
    # one handle, each solve waited for before the next
    bh = torch.from_numpy(grid.b.copy()).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    pcg.pcg_solve(h, bh, xh, opts)
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e2.record(stream)
    for _ in range(args.e2e_steps):
        pcg.pcg_solve(h, bh, xh, opts)
    e3.record(stream)
    torch.cuda.synchronize()
    ms_e2e_serial = max_over_ranks(e2.elapsed_time(e3))
    # and pipelined: two handles of the grid (pcg_clone), solves alternating
    # between them, each synchronised only before its handle is used again, so
    # that one solve's host copies (on its handle's copy stream) overlap the
    # other's iterations
    h2 = pcg.pcg_clone(h)
    bh2 = torch.from_numpy(grid.b.copy()).pin_memory()
    xh2 = torch.zeros_like(bh2).pin_memory()
    pcg.pcg_solve(h2, bh2, xh2, opts)
    pipe = [(h, bh, xh), (h2, bh2, xh2)]
    pipe_stats = []
    torch.cuda.synchronize()
    e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e4.record(stream)
    for k in range(args.e2e_steps):
        hh, bb, xx = pipe[k % 2]
        pipe_stats.append(pcg.pcg_solve(hh, bb, xx, opts, sync=False))
    pipe_rc = [pcg.pcg_sync(hh) for hh, _, _ in pipe]
    e5.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e4.elapsed_time(e5))
    if any(rc != pcg.PCG_OK for rc in pipe_rc) or any(s.status != pcg.PCG_OK for s in pipe_stats):
        raise RuntimeError("pipelined end-to-end solves did not converge")
    if not (np.array_equal(xh.numpy(), xh2.numpy()) and np.array_equal(xh.numpy(), x_main)):
        raise RuntimeError("pipelined end-to-end solutions differ from the device-timed solve")
    h2.close()
    e2e_value = replicated_rate(args.e2e_steps, ms_e2e, world)
    vec_bytes = grid.nx * grid.ny * 8

    roof = _kernel_roofline(pcg, h, b, wl, wl["prec"], n_wet, zbar, args.workload, fp64_peak)
    roof["l2_resident"] = _l2_label(torch, n_wet * (4 if wl["prec"] == 1 else 8) * (14 + zbar)).startswith("L2")

    # binary64 workloads: the same grid and right-hand side solved in the mixed
    # precision mode (binary32 inner PCG, binary64 refinement; same acceptance
    # test: true binary64 relative residual <= rtol)
    mixed = x_mixed = None
    if wl["prec"] == 0 and not args.no_mixed:
        om = pcg.make_opts(rtol=wl["rtol"], max_iter=5000, prec=1, inner_rtol=args.inner_rtol)
        steps_m = max(3, args.steps // 2)
        ms_m, stats_m, launches_m = _time_solves(pcg, torch, h, b, x, om, steps_m, args.warmup, stream, barrier,
                                                 world)
        x_mixed = x.cpu().numpy()
        mixed = {"value": replicated_rate(steps_m, ms_m, world), "unit": UNIT, "ms_per_step": ms_m / steps_m,
                 "steps": steps_m, "dtype": "f32+f64", "iters_per_solve": stats_m[-1].iters,
                 "outer_per_solve": stats_m[-1].outer_iters,
                 "worst_true_relres": max(s.true_relres for s in stats_m), "gpu_launches": int(launches_m),
                 "roofline": _kernel_roofline(pcg, h, b, wl, 1, n_wet, zbar, args.workload, fp64_peak)}

    # the same binary64 solve as row bands of one grid (the multi-GPU layout of
    # a single large grid, run on this GPU): the cost of the band-edge exchange
    shard = None
    if solo and wl["prec"] == 0 and args.workload == DEFAULT_WORKLOAD and not args.no_shard:
        sh = pcg.Shard(h, 2)
        row0, halo = sh.bands()
        for _ in range(args.warmup):
            sh.solve(b, x, opts)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps_s = max(3, args.steps // 2)
        e0.record(stream)
        worst_s = 0.0
        for _ in range(steps_s):
            sts = sh.solve(b, x, opts)
            worst_s = max(worst_s, sts.true_relres)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_s = e0.elapsed_time(e1) / steps_s
        shard = {"bands": 2, "row0": [int(v) for v in row0], "halo_rows": halo, "value": 1e3 / ms_s, "unit": UNIT,
                 "ms_per_step": ms_s, "steps": steps_s, "iters_per_solve": sts.iters,
                 "worst_true_relres": worst_s, "vs_whole_grid": (1e3 / ms_s) / value,
                 "layout": "bands on one GPU: one launch over both bands' units, shared reduction, halo rows "
                           "copied between band planes after each kernel"}
        sh.close()
    h.close()

    # batching and serving on the same GPU (the metric's "mixed vs FP64" over
    # batched and served solves, with p99 latency)
    batch = serve = None
    if solo and args.workload == DEFAULT_WORKLOAD:
        if not args.no_batch:
            batch = measure_batch(args, WORKLOADS["batch64-mixed"], args.steps, args.warmup)
        if not args.no_serve:
            serve = measure_serve(args, WORKLOADS["serve-mixed"], args.serve_block_seconds,
                                  min(5.0, args.serve_block_seconds / 4))

    # accuracy against the oracle's tight reference (outside every timed region)
    err = None
    if tight is not None:
        import oracle
        tight.join()
        x_ref = np.load(os.path.join(tmpdir, "x_ref.npy"))
        P = oracle.OracleProblem.from_grid(grid)
        bw = P.to_wet(grid.b)
        err = {"x_ref": "oracle PCG to rtol 1e-13, same preconditioner", "solutions": {}}
        for name, xs_ in (("fp64", x_main), ("mixed", x_mixed)):
            if xs_ is None:
                continue
            xw = P.to_wet(xs_)
            err["solutions"][name] = {
                "err_vs_oracle": float(np.linalg.norm(xw - x_ref) / np.linalg.norm(x_ref)),
                "true_relres_by_oracle": float(np.linalg.norm(bw - P.spmv(xw)) / np.linalg.norm(bw))}
        del P
        if mixed is not None:
            mixed["err_vs_oracle"] = err["solutions"]["mixed"]["err_vs_oracle"]

    cpu = None
    if solo and not args.no_cpu_baseline:
        cpu = oracle_baseline(os.path.join(tmpdir, "grid.npz"), wl, grid)
    if tmpdir:
        import shutil
        shutil.rmtree(tmpdir, ignore_errors=True)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if wl["prec"] == 1 else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "grid": f"{grid.nx}x{grid.ny}", "n_wet": n_wet,
                       "pattern": {0: "tril(A)", 1: "tril(A^2)", 3: "band(T)", 4: "diag"}[wl["pattern"]],
                       "drop_tol": wl["tau"], "z_offdiag_per_wet": zbar, "rtol": wl["rtol"],
                       "iters_per_solve": iters, "outer_per_solve": st.outer_iters,
                       "precision": "binary32 inner / binary64 refinement" if wl["prec"] == 1 else "binary64",
                       "worst_true_relres": worst_true, "setup_s": setup_s,
                       "l2": _l2_label(torch, n_wet * (4 if wl["prec"] == 1 else 8) * (14 + zbar)),
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": vec_bytes,
                    "d2h_bytes_per_step": vec_bytes, "steps": args.e2e_steps,
                    "pipeline": "two handles of the grid (pcg_clone), pinned host b and x, solves alternating and "
                                "each synchronised before its handle is reused: one solve's host copies overlap "
                                "the other's iterations",
                    "serial": {"value": replicated_rate(args.e2e_steps, ms_e2e_serial, world), "unit": UNIT,
                               "note": "one handle, each solve synchronised before the next"}},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "roofline": roof,
            "fp64_peak": fp64,
            "cpu_baseline": cpu,
        }
        if mixed is not None:
            line["mixed"] = mixed
        if err is not None:
            line["accuracy"] = err
        if batch is not None:
            line["batch"] = batch
        if serve is not None:
            line["serve"] = serve
        if shard is not None:
            line["shard"] = shard
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
