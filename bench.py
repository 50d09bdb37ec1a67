#!/usr/bin/env python
"""Benchmark of the GB300 adAFAC solver.

One step = one complete solve of the workload to a normalised residual of
1e-8 (Eq. 10) from u = 0, with the inputs resident in HBM: reset, then the
number of adAFAC-Jac cycles the solve needs (found in the warm-up).  The
metric is vertex updates per second (the paper's cost unit: updates of every
level's unknowns, sum over l of (3^l - 1)^d per cycle) over the whole job;
ms_per_step is the time to 1e-8.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank solves its own replica (the method needs no
exchange between independent solves): weak scaling, max time over ranks.
``--impl reference`` times the CPU FP64 oracle (rank 0 only) on the same
workload: one oracle cycle per step, the steps spread over the host cores.
"""
import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")
# The request server runs its requests on 32 streams.  With the driver's
# default of 8 hardware work queues, streams share queues and a small
# request's kernels wait behind a large request's; 32 queues keep them
# apart.  Read once, when the process creates its CUDA context.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import argparse  # noqa: E402
import json  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import tempfile  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "vertex-updates/s (adAFAC cycles to 1e-8 normalised residual)"
UNIT = "vertex-updates/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return p, "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        # the first query initialises NVML, which can stall the GPU: wait for
        # the first sample before the timed region starts
        t0 = time.time()
        while self.proc is not None and time.time() - t0 < 10.0:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.05)
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, flag in zip(names, parts[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s, p in zip(sm, power) if p > 200.0] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def _algorithmic_bytes(kind, w, precision, eps_scalar):
    """Bytes the method must move per launch of a fine-level kernel: the state
    read or written once (interior dofs of the finest level)."""
    N = (3 ** w.depth - 1) ** w.dim
    wb = 4 if precision == "mixed" else 8
    eps_b = 0 if eps_scalar else wb
    # BoxMG: the weights that are not zero by structure, (1 + 2 + 2)^d per
    # 3^d fine vertices (a vertex on a coarse plane along an axis takes one
    # corner there, any other two); d-linear weights are constants
    p_b = (5.0 / 3.0) ** w.dim * wb if w.transfer == "boxmg" else 0
    invd_b = 0 if eps_scalar else wb                     # inverse diagonal per vertex
    if precision == "mixed":
        per = {"fine_residual": 4 + 4 + 4 + eps_b,      # e, rhs in; residual out
               "fine_update": 4 + 4 + 4 + p_b + invd_b,  # residual, e in; e out
               "fine_restrict": 4 + p_b,                # residual in
               "refine": 8 + 8 + 4 + 8 * (not eps_scalar),  # u, b in; rhs32 out
               "fine_down": 4 + 4 + 4,                  # e, rhs in; e out
               "fine_up": 4 + 4,                        # e, rhs in
               "fine_down_u": 4 + 4 + 8 + 8 + 4}        # e, rhs, u in; u, other e out
    else:
        per = {"fine_residual": 8 + 8 + 8 + eps_b,
               "fine_update": 8 + 8 + 8 + p_b + invd_b,
               "fine_restrict": 8 + p_b,
               "refine": 0,
               "fine_down": 0, "fine_up": 0, "fine_down_u": 0}
    return int(round(per[kind] * N))


def _host_cpu():
    """Cores this process may run on (nproc) and the CPU model (lscpu)."""
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            key, _, val = line.partition(":")
            if key.strip() == "Model name":
                model = val.strip()
                break
    except Exception:
        pass
    return cores, model


def _oracle_hierarchy(w):
    """The oracle's level hierarchy of the workload (FP64 setup, untimed)."""
    from oracle import cycle as oc
    eps, sc = w.eps()
    t0 = time.perf_counter()
    H = oc.build_hierarchy(w.dim, w.depth, eps, sc, w.f(), w.transfer)
    return H, time.perf_counter() - t0


def run_oracle_sample(w, seconds: float):
    """Times the FP64 oracle's adAFAC-Jac cycles on the bench workload itself
    on one host core: the hierarchy is built untimed, then cycles run from
    u = 0 until ``seconds`` have passed (at least one)."""
    from oracle import cycle as oc
    H, tb = _oracle_hierarchy(w)
    u = np.zeros_like(H.b)
    upd = sum(w.level_dofs())
    t0 = time.perf_counter()
    n = 0
    while True:
        u = oc.cycle(H, u)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": n * upd / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} FP64 adAFAC-Jac cycle(s) of {w.name} (the bench workload, dim "
                      f"{w.dim}, depth {w.depth}) from u = 0, numpy on 1 host core, {dt:.1f} s; "
                      f"hierarchy setup {tb:.1f} s untimed"}


# hierarchy shared by the forked workers of the reference arm
_POOL_H = None


def _oracle_step(_):
    from oracle import cycle as oc
    oc.cycle(_POOL_H, np.zeros_like(_POOL_H.b))
    return 0


def bench_reference(args, w):
    """The reference arm: the FP64 oracle on the bench workload, on all host
    cores.  The hierarchy is built once (untimed) and shared with forked
    worker processes (copy on write; this process never touches a GPU).  A
    step is one oracle adAFAC-Jac cycle from u = 0; the K timed steps run on
    P workers at once, so ms_per_step is the wall time of the K steps / K."""
    global _POOL_H
    ws_, rank, _ = _dist()
    if rank != 0:
        return
    import multiprocessing as mp
    H, tb = _oracle_hierarchy(w)
    cores, model = _host_cpu()
    # a cycle holds about 16 vertex arrays besides the hierarchy
    per_task = 16 * 8 * (3 ** w.depth + 1) ** w.dim
    try:
        avail = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_AVPHYS_PAGES")
    except (ValueError, OSError):
        avail = per_task * cores
    workers = max(1, min(cores, max(args.steps, 1), int(0.5 * avail // per_task)))
    _POOL_H = H
    with mp.get_context("fork").Pool(workers) as pool:
        if args.warmup:
            pool.map(_oracle_step, range(args.warmup), chunksize=1)
        t0 = time.perf_counter()
        pool.map(_oracle_step, range(args.steps), chunksize=1)
        dt = time.perf_counter() - t0
    upd = sum(w.level_dofs())
    value = args.steps * upd / dt
    sample = (f"{args.steps} FP64 oracle adAFAC-Jac cycles of {w.name} (the bench workload, "
              f"dim {w.dim}, depth {w.depth}) from u = 0, one per step, numpy in {workers} "
              f"forked processes (1 thread each) on {cores} host cores ({model}); hierarchy "
              f"setup {tb:.1f} s untimed")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": _config(w, args),
           "run": {"precision": "fp64", "cycles_per_step": 1, "host_cores": cores,
                   "host_cpu": model, "workers": workers},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


L2_BYTES = 126 * 2 ** 20


def _needs_flush(w, precision):
    """Flush L2 between steps unless the fine-level arrays a step touches
    (u, b in FP64; mixed: two FP32 corrections and the FP32 right-hand side)
    exceed twice the L2 size."""
    per = 8 + 8 + (4 + 4 + 4 if precision == "mixed" else 8 + 8)
    return (3 ** w.depth + 1) ** w.dim * per < 2 * L2_BYTES


def _tuning_summary(t):
    """The launch shapes the autotuner chose (None when it was not run)."""
    if not t:
        return None
    if t["path"] == 1:
        shapes = {"sweep_nz": t["sweep_nz"], "sweep_nz_down": t["sweep_nz_down"]}
    elif t["path"] == 2:
        shapes = {k: t[k] for k in ("res_bx", "res_by", "res_zr", "upd_bx", "upd_by")}
    else:
        shapes = {}
    return dict(shapes, candidates=t["candidates"], us_default=round(t["us_default"], 2),
                us_tuned=round(t["us_tuned"], 2))


def _config(w, args):
    """The workload (the same in both arms): problem, method, tolerance."""
    return {"workload": w.name, "dim": w.dim, "depth": w.depth,
            "fine_dofs": (3 ** w.depth - 1) ** w.dim, "dofs_all_levels": sum(w.level_dofs()),
            "variant": "adAFAC-Jac", "transfer": w.transfer, "rtilde": "truncated",
            "tol": args.tol,
            "l2": "L2 flushed between steps" if _needs_flush(w, args.precision)
                  else "working set of a step larger than L2",
            "parallelism": f"replicas x{args.gpus}"}


def max_over_ranks(value, dist, device):
    """The largest of the ranks' values: the job takes as long as its slowest
    replica.  dist None (one process) returns value."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, cycles, updates_per_cycle, ms):
    """Vertex updates per second of the whole job: every rank solves its own
    replica (steps solves of `cycles` cycles each) within ms milliseconds."""
    return world * steps * cycles * updates_per_cycle / (ms / 1e3)


def bench_ours(args, w):
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_1903_10367_gb300 import adafac
    adafac.load()
    eps, sc = w.eps()
    f = w.f()
    eps_arg = float(eps[0]) if sc else eps
    opts = adafac.default_options(transfer=w.transfer, precision=args.precision)
    S = adafac.Solver(w.dim, w.depth, eps_arg, f, opts)
    # launch shapes of the fine-level kernels chosen by the library's autotuner
    # (timed here once; later handles of this shape take the stored choice)
    tuning = None if args.no_autotune else S.autotune(5)
    upd_cycle = sum(w.level_dofs())
    # warm-up: full solves; the cycle count of one solve defines a step
    cycles = None
    for i in range(max(args.warmup, 1)):
        S.reset()
        c, rel = S.solve(args.tol, args.max_cycles)
        if cycles is None:
            cycles = c
        assert c == cycles, "cycle count of the solve must be reproducible"
    flush = None
    if _needs_flush(w, args.precision):
        l2_bytes = max(L2_BYTES, torch.cuda.get_device_properties(dev).L2_cache_size)
        flush = torch.empty(4 * l2_bytes // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        if flush is not None:
            flush.fill_(1.0)
        S.reset()
        S.cycle(cycles)

    # timed region
    clocks = Clocks(dev) if rank == 0 else None
    if clocks:
        clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = S.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = S.launch_count() - l0
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop() if clocks else None
    rel_final = S.residual_norm()[0]
    if not rel_final <= args.tol * 1.0000001:
        raise RuntimeError(f"solve did not reach the tolerance: {rel_final}")
    ms = max_over_ranks(ms, dist, "cuda")
    value = job_throughput(world, args.steps, cycles, upd_cycle, ms)
    # roofline: per-kernel CUDA-event timing over a second timed region
    S.timing(True)
    for _ in range(args.steps):
        step()
    kinds = ["fine_down", "fine_up", "fine_down_u", "fine_residual", "fine_update",
             "fine_restrict", "refine"]
    kt = {k: S.timing_read(k) for k in kinds}
    S.timing(False)
    dom = max(kinds, key=lambda k: kt[k][0])
    dom_ms, dom_n = kt[dom]
    peaks, src = _peaks()
    alg = _algorithmic_bytes(dom, w, args.precision, sc)
    achieved = alg / (dom_ms / dom_n / 1e3) / 1e9 if dom_n else None
    traffic, capture_shape = _traffic_from_profile(dom, w, tuning)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"] if achieved else None,
                "traffic": traffic, "peak_source": f"hbm_gbs of {src}",
                "traffic_launch_shape": capture_shape if traffic and _shape_differs(
                    capture_shape, tuning) else None,
                "algorithmic_bytes_per_launch": alg,
                "avg_launch_us": 1e3 * dom_ms / dom_n if dom_n else None,
                "share_of_step": dom_ms / max(1e-9, sum(v[0] for v in kt.values())),
                "per_kernel_ms": {k: round(v[0] / args.steps, 4) for k, v in kt.items()}}
    # FP64 single-instance comparator on the same workload (time to 1e-8)
    fp64 = None
    if not args.no_fp64_comparator and rank == 0:
        S64 = adafac.Solver(w.dim, w.depth, eps_arg, f,
                            adafac.default_options(transfer=w.transfer, precision="fp64"))
        c64, _ = S64.solve(args.tol, args.max_cycles)
        S64.reset()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        S64.cycle(c64)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64 = {"ms_to_tol": e0.elapsed_time(e1), "cycles": c64,
                "value": c64 * upd_cycle / (e0.elapsed_time(e1) / 1e3), "unit": UNIT}
        S64.close()
    # end to end through the public API from pinned host buffers
    e2e = _e2e(args, w, eps, sc, f, opts, upd_cycle, cycles, adafac, torch, tuning is not None)
    S.close()
    if rank != 0:
        return
    cpu = None if args.no_cpu_baseline else run_oracle_sample(w, args.cpu_seconds)
    serving = run_serving(args.serve_requests) if args.serve_requests > 0 else None
    adaptive = (run_adaptive(args.adaptive_depth, precision=args.adaptive_precision)
                if args.adaptive_depth > 0 else None)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 cycles + f64 refinement" if args.precision == "mixed" else "f64",
           "data": "synthetic", "config": _config(w, args),
           "run": {"precision": args.precision, "cycles_per_step": cycles,
                   "tuning": _tuning_summary(tuning)},
           "time_to_tol_ms": ms / args.steps, "e2e": e2e, "gpu_launches": launches,
           "roofline": roofline, "clocks": clk, "cpu_baseline": cpu,
           "fp64_comparator": fp64, "serving": serving, "adaptive": adaptive}
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def _e2e(args, w, eps, sc, f, opts, upd_cycle, cycles, adafac, torch, tune):
    """Setup from host buffers, solve to the tolerance, read the solution back
    (with the autotuner's stored launch shapes when the bench tuned them)."""
    if args.e2e_steps <= 0:
        return None
    f_pin = torch.from_numpy(f).pin_memory()
    eps_pin = None if sc else torch.from_numpy(eps).pin_memory()
    out = torch.empty(f.shape, dtype=torch.float64).pin_memory()
    nbytes = adafac.workspace_size(w.dim, w.depth, opts)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    times = []
    for i in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S = adafac.Solver(w.dim, w.depth, float(eps[0]) if sc else eps_pin.numpy(),
                          f_pin.numpy(), opts, workspace=ws)
        if tune:
            S.autotune(5)
        c, rel = S.solve(args.tol, args.max_cycles)
        S.solution(out.numpy())
        t1 = time.perf_counter()
        S.close()
        if i > 0:
            times.append(t1 - t0)
    t = statistics.mean(times)
    h2d = f.nbytes + (8 if sc else eps.nbytes)
    return {"value": cycles * upd_cycle / t, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(f.nbytes), "ms_per_step": 1e3 * t,
            "includes": "setup (H2D copies, BoxMG/Galerkin), stored launch shapes, solve to tol, "
                        "D2H of u"}


# Sources of the kernels whose DRAM counters profiles/traffic.json records,
# per workload: counters taken on another build of them do not describe this one.
TRAFFIC_SOURCES = {
    "poisson3d_d5": ("sweep3.cu", "sweep3.cuh", "common.cuh", "mbarrier.cuh"),
    "jump3d_d5": ("level.cu", "common.cuh"),
}


def kernel_source_hash(files=("sweep3.cu", "sweep3.cuh", "common.cuh", "mbarrier.cuh")):
    """Fingerprint of the sources of profiled fine-level kernels (by default
    the 3-D sweeps and the refinement residual)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1903_10367_gb300", "csrc")
    h = hashlib.sha256()
    for name in files:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def run_serving(count: int, seed: int = 1903):
    """The serving configuration: a seeded stream of ``count`` solves (80 % 2-D
    depth 3..6, 20 % 3-D depth 3..5, random-block eps 1 / 1e-2, BoxMG, mixed
    precision, to 1e-8) through the request server.  First the whole stream at
    once (saturated throughput), then the same stream with Poisson arrivals at
    0.8 x that throughput (p50 / p99 latency from submission to the solution in
    host memory).  The comparator solves every request alone with plain FP64
    cycles on a single handle, one after another (setup + solve + copy of u)."""
    import torch
    from paper_1903_10367_gb300 import adafac
    reqs = wl.serving_requests(count, seed)
    om = adafac.default_options(transfer="boxmg", precision="mixed")
    o64 = adafac.default_options(transfer="boxmg", precision="fp64")
    free, _ = torch.cuda.mem_get_info()
    pool = int(min(0.6 * free, 96 << 30))
    srv = adafac.Server(pool, n_streams=32, max_running=32)

    def submit(r):
        return srv.submit(r.dim, r.depth, r.eps, r.f, om, 1e-8, 3000)

    def drain(tickets):
        while any(srv.poll(t)["state"] in ("pending", "running") for t in tickets):
            time.sleep(0.0005)
        infos = [srv.poll(t) for t in tickets]
        for t in tickets:
            srv.fetch(t)
        return infos

    drain([submit(r) for r in reqs[:8]])          # warm-up
    t0 = time.perf_counter()
    infos = drain([submit(r) for r in reqs])
    t_sat = time.perf_counter() - t0
    ok = all(i["state"] == "done" and i["rel"] <= 1e-8 for i in infos)
    lam_sat = count / t_sat
    upd = sum(i["cycles"] * sum(wl.Workload("r", r.dim, r.depth, "blocks").level_dofs())
              for i, r in zip(infos, reqs))
    lam = 0.8 * lam_sat
    start = time.perf_counter()
    tickets = []
    for r in reqs:
        target = start + r.arrival / lam
        while True:
            dt = target - time.perf_counter()
            if dt <= 0:
                break
            time.sleep(min(dt, 0.0005))
        tickets.append(submit(r))
    infos_open = drain(tickets)
    t_open = time.perf_counter() - start
    srv.close()
    lat = np.array([i["latency_ms"] for i in infos_open])
    ok = ok and all(i["state"] == "done" and i["rel"] <= 1e-8 for i in infos_open)
    # every request alone on one handle, one after another (setup + solve to
    # 1e-8 + copy of u): FP64 cycles (the comparator) and mixed precision
    def alone(opts):
        out = []
        for r in reqs:
            t1 = time.perf_counter()
            S = adafac.Solver(r.dim, r.depth, r.eps, r.f, opts)
            S.solve(1e-8, 3000)
            S.solution()
            S.close()
            out.append(1e3 * (time.perf_counter() - t1))
        return np.array(out)

    single = alone(o64)
    single_mixed = alone(om)
    classes = {}
    for key in sorted({(r.dim, r.depth) for r in reqs}):
        idx = [i for i, r in enumerate(reqs) if (r.dim, r.depth) == key]
        m64, mmx = float(np.median(single[idx])), float(np.median(single_mixed[idx]))
        classes[f"{key[0]}d_depth{key[1]}"] = {
            "requests": len(idx), "fp64_alone_ms": round(m64, 3), "mixed_alone_ms": round(mmx, 3),
            "fp64_over_mixed": round(m64 / mmx, 2)}
    # matched load: Poisson arrivals at 0.8 x the FP64 single-instance
    # throughput, which a one-at-a-time FP64 server sustains.  The mixed
    # server runs live on the first requests of the stream; the FP64 server's
    # FIFO latencies follow from its measured service times at the same
    # arrival instants.
    lam64 = count / (single.sum() / 1e3)
    lam_m = 0.8 * lam64
    n_m = min(count, 60)
    srv = adafac.Server(pool, n_streams=32, max_running=32)
    start = time.perf_counter()
    tickets = []
    for r in reqs[:n_m]:
        target = start + r.arrival / lam_m
        while True:
            dt = target - time.perf_counter()
            if dt <= 0:
                break
            time.sleep(min(dt, 0.0005))
        tickets.append(submit(r))
    infos_m = drain(tickets)
    srv.close()
    lat_m = np.array([i["latency_ms"] for i in infos_m])
    ok = ok and all(i["state"] == "done" and i["rel"] <= 1e-8 for i in infos_m)
    fifo, free_at = [], 0.0
    for r, svc in zip(reqs[:n_m], single[:n_m]):
        arr = 1e3 * r.arrival / lam_m
        free_at = max(arr, free_at) + svc
        fifo.append(free_at - arr)
    fifo = np.array(fifo)
    # batched refinement steps (path BATCHED): the stream without its 3-D
    # depth-5 requests (whose level kernels fill the GPU), saturated, with
    # three path choices: level kernels for every request, AUTO (batched on
    # the smallest grids), batched for every request up to 2-D depth 5 and
    # 3-D depth 3
    small = [r for r in reqs if not (r.dim == 3 and r.depth >= 5)]
    policies = {
        "level_kernels": lambda r: "levelwise",
        "auto": lambda r: "auto",
        "batched_up_to_64k_vertices": lambda r: (
            "batched" if (r.dim == 2 and r.depth <= 5) or (r.dim == 3 and r.depth <= 3)
            else "auto"),
    }
    batched = {"requests": len(small), "stream": "the mix without its 3-D depth-5 requests"}
    for name, pol in policies.items():
        srv = adafac.Server(pool, n_streams=32, max_running=64)
        opts = {p: adafac.default_options(transfer="boxmg", precision="mixed", path=p)
                for p in ("levelwise", "auto", "batched")}
        sub = lambda r: srv.submit(r.dim, r.depth, r.eps, r.f, opts[pol(r)], 1e-8, 3000)
        drain([sub(r) for r in small[:8]])
        t0 = time.perf_counter()
        inf = drain([sub(r) for r in small])
        dt = time.perf_counter() - t0
        srv.close()
        ok = ok and all(i["state"] == "done" and i["rel"] <= 1e-8 for i in inf)
        batched[name] = {"requests_per_s": len(small) / dt,
                         "p50_ms": float(np.percentile([i["latency_ms"] for i in inf], 50))}
    return {
        "requests": count, "seed": seed,
        "mix": "80% 2-D depth U{3..6}, 20% 3-D depth U{3..5}; eps blocks of level-min(3, depth-1) "
               "cells, 1 or 1e-2; f = 1; BoxMG + Galerkin; to 1e-8",
        "all_converged": bool(ok),
        "saturated_requests_per_s": lam_sat,
        "saturated_vertex_updates_per_s": upd / t_sat,
        "offered_requests_per_s": lam, "offered_load": "0.8 x saturated throughput",
        "open_loop_s": t_open,
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()),
        "server": {"pool_bytes": pool, "streams": 32, "max_running": 32,
                   "cuda_device_max_connections": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS"),
                   "precision": "mixed (FP32 cycles, FP64 refinement)"},
        "fp64_single_instance": {
            "requests_per_s": count / (single.sum() / 1e3),
            "p50_ms": float(np.percentile(single, 50)), "p99_ms": float(np.percentile(single, 99)),
            "mean_ms": float(single.mean()),
            "how": "each request alone: setup + FP64 solve to 1e-8 + copy of u, back to back"},
        "throughput_vs_fp64_single": lam_sat / (count / (single.sum() / 1e3)),
        "mixed_single_instance": {
            "requests_per_s": count / (single_mixed.sum() / 1e3),
            "p50_ms": float(np.percentile(single_mixed, 50)),
            "p99_ms": float(np.percentile(single_mixed, 99)),
            "how": "each request alone: setup + mixed solve to 1e-8 + copy of u, back to back"},
        "per_class_alone": classes,
        "batched_kernels_saturated": batched,
        "matched_load": {
            "offered_requests_per_s": lam_m, "offered_load": "0.8 x FP64 single-instance throughput",
            "requests": n_m,
            "mixed_server": {"p50_ms": float(np.percentile(lat_m, 50)),
                             "p99_ms": float(np.percentile(lat_m, 99))},
            "fp64_single_instance_fifo": {
                "p50_ms": float(np.percentile(fifo, 50)), "p99_ms": float(np.percentile(fifo, 99)),
                "how": "FIFO queue of the measured FP64 service times at the same arrival instants"}},
    }


def band_flags(d, L, L_base, centre, radius, width):
    """Refinement flags of the adaptive workload's tree: depth L_base
    everywhere and L within `width` of the circle (sphere) of `radius` about
    `centre` (x first); a cell is cut when it reaches within width of the
    circle, with its half-diagonal as the margin.  One flag array per level
    l < L, shape (3^l,)*d, last axis x."""
    ctr = np.asarray(centre, dtype=float)
    out = []
    for l in range(1, L):
        n = 3 ** l
        h = 1.0 / n
        if l < L_base:
            out.append(np.ones((n,) * d, dtype=bool))
            continue
        idx = np.indices((n,) * d)
        c = np.stack([(idx[d - 1 - k] + 0.5) * h for k in range(d)], axis=-1)
        r = np.sqrt(((c - ctr) ** 2).sum(-1))
        out.append(np.abs(r - radius) <= width + 0.5 * np.sqrt(d) * h)
    return out


def run_adaptive(depth: int, base: int = 3, moves: int = 4, every: int = 5, shift: float = 0.01,
                 tol: float = 1e-8, precision: str = "mixed"):
    """The adaptive workload on the GPU (FP64 cycles on the generating system):
    2-D, depth `base` everywhere and `depth` within 0.05 of the circle r = 0.3
    about the centre, f = 1, eps = 1; the band moves +x by `shift` after every
    `every` cycles, `moves` times (the iterate carried over by the transfer),
    then cycles to `tol`.  Reports the host build of a tree's system, the
    transfer, the time per cycle and the cycles."""
    import torch
    from paper_1903_10367_gb300 import adafac
    d = 2
    f = np.ones((3 ** depth + 1,) * d)
    o = adafac.default_options(precision=precision)
    ctr = np.array([0.5, 0.5])
    builds, transfers, cyc_ms = [], [], []
    t0 = time.perf_counter()
    G = adafac.AdaptiveSolver(d, depth, band_flags(d, depth, base, ctr, 0.3, 0.05), 1.0, f, o)
    builds.append(time.perf_counter() - t0)
    nodes = [G.count]
    st = torch.cuda.current_stream()
    total = 0
    rel = 1.0
    for m in range(moves + 1):
        steps = every if m < moves else 100000
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        k = 0
        if m < moves:
            G.cycle(steps)
            k = steps
        else:
            k, rel = G.solve(tol, 5000)
        e1.record(st)
        torch.cuda.synchronize()
        cyc_ms.append(e0.elapsed_time(e1) / k)
        total += k
        if m < moves:
            ctr = ctr + np.array([shift, 0.0])
            t0 = time.perf_counter()
            N = adafac.AdaptiveSolver(d, depth, band_flags(d, depth, base, ctr, 0.3, 0.05), 1.0, f, o)
            builds.append(time.perf_counter() - t0)
            t0 = time.perf_counter()
            N.transfer_from(G)
            transfers.append(time.perf_counter() - t0)
            G.close()
            G = N
            nodes.append(G.count)
    cycles, rel = total, G.residual_norm()[0]
    G.close()
    return {"dim": d, "depth": depth, "base_depth": base, "leaf_nodes": nodes,
            "moves": moves, "every": every, "shift": shift, "cycles": cycles, "rel": rel,
            "ms_per_cycle_median": float(np.median(cyc_ms)),
            "build_s_median": float(np.median(builds)),
            "transfer_ms_median": 1e3 * float(np.median(transfers)) if transfers else None,
            "precision": precision,
            "how": "system build per tree (host tree and leaf nodes, device grids); cycles timed "
                   "with CUDA events (the last phase includes the norm tests of the solve)"}


def _traffic_from_profile(kind, w, tuning=None, table=None):
    """DRAM bytes (read + write) per launch of this kernel from the committed
    ncu summary (profiles/traffic.json) and the launch shape of that capture,
    or (None, None) when the summary was taken on other kernel sources or
    holds no figure for the kernel."""
    try:
        if table is None:
            with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
                table = json.load(fh)
        entry = table.get(w.name)
        files = TRAFFIC_SOURCES.get(w.name)
        if not entry or not files or entry.get("source_hash") != kernel_source_hash(files):
            return None, None
        return entry.get("bytes", {}).get(kind), entry.get("launch_shape")
    except Exception:
        return None, None


def _shape_differs(capture_shape, tuning):
    """True when the traffic capture ran other launch shapes than the timed run."""
    if not capture_shape:
        return False
    run = {k: (tuning or {}).get(k) for k in capture_shape}
    return run != capture_shape


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="poisson3d_d5", choices=sorted(wl.WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--max-cycles", type=int, default=5000)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-comparator", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes instead of the autotuned ones")
    ap.add_argument("--adaptive-depth", type=int, default=0,
                    help="depth of the moving-band adaptive run on the GPU (0: skip)")
    ap.add_argument("--adaptive-precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--serve-requests", type=int, default=200,
                    help="requests of the serving stream run after the solve (0: skip)")
    args = ap.parse_args()
    w = wl.get(args.workload)
    if args.impl == "reference":
        bench_reference(args, w)
    else:
        bench_ours(args, w)


if __name__ == "__main__":
    main()
