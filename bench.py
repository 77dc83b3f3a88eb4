#!/usr/bin/env python
"""Benchmark of the implicit moving-mesh UGKS on one GB300 (per rank).

Workload (default): the thermal rarefied MEMS overset case -- Cartesian
background 256x128 + body-fitted O-grid 128x32 around a heated plate
(Tw = 1.5) translating sinusoidally, 32x32 velocities on [-6, 6], Kn = 0.1,
10 inner iterations per physical step.  A timed "step" is one physical step
of the outer loop: prescribed motion, overset assembly, implicit UGKS step
(all inner iterations).  Metric: cell-velocity updates per second per
implicit (inner) iteration = N_field_cells * N_v * n_inner / t_step.
Inputs resident in HBM; f alone (FP32, 302 MB) exceeds the 129 MB L2, so no
L2 flush is needed between steps.

--impl reference times the FP64 numpy oracle (the paper publishes no code)
on the host cores on a bounded sample of the same workload.
Multi-GPU (torchrun): every rank runs an independent replica (weak scaling,
no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# the oracle baseline is reported as single-threaded: keep numpy's BLAS on one core
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

from paper_2604_09984_gb300 import workloads as wl  # noqa: E402

METRIC = "cell·velocity updates/s per implicit step, FP32-mixed vs FP64 plain; %HBM peak"
UNIT = "cell·vel·iter/s"
FALLBACK_HBM = 6800.0


def make_case(name, kn, mesh=None):
    if name == "mems":
        if mesh:       # "NBIxNBJ+NOIxNOJ": a reduced MEMS mesh (profiler captures)
            bg, og = mesh.split("+")
            nbi, nbj = (int(v) for v in bg.split("x"))
            noi, noj = (int(v) for v in og.split("x"))
            return wl.mems(nbi=nbi, nbj=nbj, noi=noi, noj=noj, Kn=kn)
        return wl.mems(Kn=kn)
    if name == "channel":
        return wl.channel()
    if name == "tsto":
        return wl.tsto()
    raise SystemExit("unknown workload " + name)


def workload_label(case):
    b = case.blocks
    return "%s: %s cells, %dx%d velocities, Kn=%g, %d inner/step" % (
        case.name, "+".join("%dx%d" % (x.ni, x.nj) for x in b), case.nvx, case.nvy,
        case.meta.get("Kn", 0.0), case.n_inner)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", FALLBACK_HBM)), "measured"
    return FALLBACK_HBM, "fallback"


class Clocks:
    """nvidia-smi sampler (SM clock, max, throttle reasons) for the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def field_cells(solver):
    _, _, st, _ = solver.moments()
    return int((st == 0).sum())


def algorithmic_bytes(group, pair_bytes, nfield, nv, nc):
    """Minimum DRAM bytes of one launch of a kernel group:
    flux reads f and writes the flux divergence; residual reads f, the
    divergence and the level-n term (written on the first inner iteration)
    and writes the residual; micro_fwd reads the residual and writes the
    forward increment in place; micro_bwd reads the increment and f and
    writes f; face_reduce and moments read f once."""
    per = {"flux": 2 * nfield, "residual": 4 * nfield, "micro_fwd": 2 * nfield,
           "micro_bwd": 3 * nfield, "face_reduce": nc, "moments": nfield, "interp": 0}
    return per.get(group, 0) * nv * pair_bytes


def csrc_sha256():
    import glob
    import hashlib
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_2604_09984_gb300", "csrc", "*"))):
        with open(p, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def ncu_traffic(group):
    """DRAM bytes (read + write) per launch of a kernel group of the default
    workload from the committed ncu summary, or None when the CUDA sources
    changed since that capture."""
    p = os.path.join(ROOT, "profiles", "kernels_mems_fp32.md")
    if not os.path.exists(p):
        return None
    sha, traffic = None, {}
    for line in open(p):
        w = line.split()
        if line.startswith("CUDA sources: sha256") and len(w) >= 4:
            sha = w[3]
        elif len(w) == 3 and w[0] == "traffic":
            traffic[w[1]] = int(w[2])
    if sha != csrc_sha256():
        return None
    return traffic.get(group)


def max_over_ranks(ms, dist, device):
    """Slowest rank's time (the whole job's time); ms itself with one rank."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_sync(dist):
    """Device idle on this rank, then all ranks at the same point."""
    import torch
    if torch.cuda.is_available():
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()


def time_arm(case, precision, steps, warmup, device, profile, tune=True, dist=None):
    import torch
    from paper_2604_09984_gb300 import ugks as U
    s = U.Solver(case, precision, device=device)
    s.tiles = None
    for n in range(warmup):
        s.advance()
        if n == 0 and tune:
            s.autotune()          # sweep tiles for this workload, before the timed steps
    rank_sync(dist)
    nfield = field_cells(s)
    if profile:
        s.profile_read(reset=True)
        s.profile(True)
    l0 = s.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(s.stream)
    # motion, assembly and implicit step issued without waiting on the device
    # (ugks_advance_batch with one instance; an assembly error would surface
    # at the next synchronising call, the rank barrier below)
    for _ in range(steps):
        U.advance_batch([s])
    ev1.record(s.stream)
    rank_sync(dist)
    s.moments()                              # synchronising call: reports any deferred error
    ms = ev0.elapsed_time(ev1)
    launches = s.launch_count() - l0
    prof = None
    if profile:
        s.profile(False)
        prof = s.profile_read(reset=True)
    return s, ms, nfield, launches, prof


def e2e_arm(s, steps):
    """Same metric through the public API with host buffers: per step the
    motion parameters go host->device, and W, q, status and wall loads come
    back into pinned host memory."""
    import torch
    nb = len(s.case.blocks)
    W = torch.empty((s.nc, 4), dtype=torch.float64).pin_memory()
    q = torch.empty((s.nc, 2), dtype=torch.float64).pin_memory()
    st = torch.empty(s.nc, dtype=torch.int32).pin_memory()
    wall = torch.empty((nb, 4), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    from paper_2604_09984_gb300 import ugks as U
    t0 = time.perf_counter()
    ev0.record(s.stream)
    for _ in range(steps):
        U.advance_batch([s])                 # no wait until the results are read
        s.moments(W, q, st, wall)            # synchronises: W, q, status, wall loads on the host
    ev1.record(s.stream)
    torch.cuda.synchronize()
    wall_s = time.perf_counter() - t0
    ms = max(ev0.elapsed_time(ev1), wall_s * 1e3)
    h2d = 6 * 8 * nb
    d2h = W.numel() * 8 + q.numel() * 8 + st.numel() * 4 + wall.numel() * 8
    return ms, h2d, d2h


def batch_arm(cases, steps, warmup, device, dist=None):
    """Batched serving: one solver (FP32) per instance, each on its own
    stream, advanced together through ugks_advance_batch.  Device time from
    an event every instance stream waits on to an event that waits on every
    instance stream."""
    import torch
    from paper_2604_09984_gb300 import ugks as U
    streams = [torch.cuda.Stream(device=device) for _ in cases]
    solvers = [U.Solver(c, U.FP32, device=device, stream=st) for c, st in zip(cases, streams)]
    for n in range(warmup):
        U.advance_batch(solvers)
        if n == 0:
            for s in solvers:     # per-instance sweep tiles
                s.autotune()
    rank_sync(dist)
    tiles = sorted({s.tiles for s in solvers})
    nfield = [field_cells(s) for s in solvers]
    l0 = sum(s.launch_count() for s in solvers)
    main_st = torch.cuda.current_stream(device)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(main_st)
    for st in streams:
        st.wait_event(ev0)
    t0 = time.perf_counter()
    for _ in range(steps):
        U.advance_batch(solvers)
    host_s = time.perf_counter() - t0
    for st in streams:
        e = torch.cuda.Event()
        e.record(st)
        main_st.wait_event(e)
    ev1.record(main_st)
    rank_sync(dist)
    ms = ev0.elapsed_time(ev1)
    launches = sum(s.launch_count() for s in solvers) - l0
    units = sum(n * c.nv * c.n_inner for n, c in zip(nfield, cases)) * steps
    # end to end: motion parameters in, W/q/status/wall loads of every
    # instance back to pinned host memory each step
    outs = []
    for s in solvers:
        outs.append((torch.empty((s.nc, 4), dtype=torch.float64).pin_memory(),
                     torch.empty((s.nc, 2), dtype=torch.float64).pin_memory(),
                     torch.empty(s.nc, dtype=torch.int32).pin_memory(),
                     torch.empty((len(s.case.blocks), 4), dtype=torch.float64).pin_memory()))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        U.advance_batch(solvers)
        for s, o in zip(solvers, outs):
            s.moments(*o)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    h2d = sum(6 * 8 * len(c.blocks) for c in cases)
    d2h = sum(sum(t.numel() * t.element_size() for t in o) for o in outs)
    for s in solvers:
        s.close()
    return ms, units, launches, host_s, e2e_s, h2d, d2h, sum(nfield), tiles


def run_batch(args, world, rank, device, dist=None):
    cases = wl.mems_batch(n=args.instances)
    steps = max(1, args.steps)
    warmup = max(3, args.warmup)
    clk = Clocks(int(device.split(":")[1]))
    clk.start()
    ms, units, launches, host_s, e2e_s, h2d, d2h, nfield, tiles = batch_arm(cases, steps, warmup, device, dist)
    clocks = clk.stop()
    ms = max_over_ranks(ms, dist, device)
    value = units * world / (ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "mems_batch: %d independent oscillating-plate instances, %d field cells, "
                               "%.3g cell-velocities, 20^2-40^2 velocities, Kn 0.01-2, 10 inner/step"
                               % (len(cases), nfield, sum(c.ncells * c.nv for c in cases)),
                   "precision": "FP32 f and per-velocity arithmetic, FP64 moments/geometry",
                   "l2": "inputs larger than L2", "streams": len(cases),
                   "tiles": "autotuned per instance (sweep items, velocities per lane, rings fwd/bwd, face chunk, "
                            "threads per face): %s" % tiles,
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "host_issue_ms_per_step": host_s * 1e3 / steps,
        "clocks": clocks,
        "e2e": {"value": units * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": None,
        "cpu_baseline": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def cpu_sample_case(kn):
    # same geometry family, physics and velocity grid as the timed workload,
    # at a background/O-grid resolution the numpy oracle finishes in ~10-30 s
    return wl.mems(nbi=64, nbj=32, noi=48, noj=12, Kn=kn, stretch=1.15, n_inner=3)


def cpu_baseline(kn, steps=1):
    from oracle.run import Run
    case = cpu_sample_case(kn)
    r = Run(case)
    t0 = time.perf_counter()
    units = 0
    for _ in range(steps):
        r.step()
        units += int((r.status == 0).sum()) * case.nv * case.n_inner
    dt = time.perf_counter() - t0
    return {"value": units / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "FP64 numpy oracle, %d step(s) of %s" % (steps, workload_label(case)),
            "seconds": dt}


def _oracle_job(kn):
    """One physical step of the oracle sample in a worker process: (units, s)."""
    from oracle.run import Run
    case = cpu_sample_case(kn)
    r = Run(case)
    t0 = time.perf_counter()
    r.step()
    return int((r.status == 0).sum()) * case.nv * case.n_inner, time.perf_counter() - t0


def cpu_baseline_multicore(kn):
    """The oracle on all host cores: one independent sample step per core in
    worker processes started with spawn (no fork after CUDA has started);
    throughput = all units / wall time of the slowest worker's step."""
    import multiprocessing as mp
    ncore = os.cpu_count() or 1
    nproc = max(1, min(ncore, 16))
    ctx = mp.get_context("spawn")
    with ctx.Pool(nproc) as pool:
        t0 = time.perf_counter()
        res = pool.map(_oracle_job, [kn] * nproc)
        wall = time.perf_counter() - t0
    units = sum(u for u, _ in res)
    step_s = max(t for _, t in res)
    return {"value": units / step_s, "unit": UNIT, "cores": nproc, "kind": "oracle",
            "host_cores": ncore, "wall_s_with_startup": wall,
            "sample": "FP64 numpy oracle, %d independent processes x 1 step of %s"
                      % (nproc, workload_label(cpu_sample_case(kn)))}


def run_reference(args, rank, world):
    if rank != 0:
        return
    kn = args.kn
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(kn, 1)
    t0 = time.perf_counter()
    res = [cpu_baseline(kn, 1) for _ in range(args.steps)]
    el = time.perf_counter() - t0
    v = statistics.median([r["value"] for r in res])
    case = make_case(args.workload, kn)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_label(case),
                                             "reference": "FP64 numpy oracle on host cores (no published code)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": res[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def dominant_roofline(prof, nfield, nv, nc, pair, peak, peak_kind, traffic=None):
    """Roofline of the streaming kernel group (one that moves f) with the most
    device time on the step's stream: its algorithmic bytes per launch over
    its event-timed duration per launch.  (The macro LU-SGS runs on a second
    stream beside the flux kernel and moves no f.)"""
    groups = {g: v for g, v in prof.items() if v[1] > 0}
    streaming = {g: v for g, v in groups.items() if algorithmic_bytes(g, pair, nfield, nv, nc) > 0}
    dom = max(streaming or groups, key=lambda g: groups[g][0])
    dms, dn = groups[dom]
    abytes = algorithmic_bytes(dom, pair, nfield, nv, nc)
    if abytes > 0:
        ach = abytes / (dms / dn * 1e-3) / 1e9
        return {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": traffic, "peak_kind": peak_kind,
                "bytes_per_launch": abytes, "ms_per_launch": dms / dn}
    return {"kernel": dom, "bound": "alu", "achieved": None, "peak": None, "unit": None,
            "frac": None, "traffic": None, "ms_per_launch": dms / dn}


def kernel_table(prof, nfield, nv, nc, pair):
    groups = {g: v for g, v in prof.items() if v[1] > 0}
    tot = sum(v[0] for v in groups.values())
    out = {}
    for g, (gms, gn) in groups.items():
        b = algorithmic_bytes(g, pair, nfield, nv, nc)
        out[g] = {"ms_total": round(gms, 3), "launches": gn, "share": round(gms / tot, 4)}
        if b:
            out[g]["GBps"] = round(b / (gms / gn * 1e-3) / 1e9, 1)
    return out


def profiled_steps(s, steps):
    """Per-group device times (CUDA events around every launch) over `steps`
    further physical steps of solver s; separate from the timed steps, whose
    clock sees no event bracketing."""
    s.profile_read(reset=True)
    s.profile(True)
    for _ in range(steps):
        s.advance()
    s.profile(False)
    return s.profile_read(reset=True)


def fp64_probe(device):
    """Measured FP64 rates of this GPU (ugks_probe_fp64): fused multiply-adds
    and exponentials per second, CUDA events on the launch stream."""
    import ctypes
    import torch
    from paper_2604_09984_gb300 import ugks as U
    lib = U.load()
    nb, nt = 152 * 16, 256
    out = torch.empty(nb * nt, dtype=torch.float64, device=device)
    st = torch.cuda.current_stream(device)
    res = {}
    for kind, iters, per in ((0, 2048, 16), (1, 256, 4)):
        ms = None
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            r = lib.ugks_probe_fp64(ctypes.c_void_p(out.data_ptr()), kind, nb, nt, iters,
                                    ctypes.c_void_p(st.cuda_stream))
            e1.record(st)
            torch.cuda.synchronize()
            if r != U.OK:
                return None
            t = e0.elapsed_time(e1)
            ms = t if ms is None else min(ms, t)
        res[kind] = nb * nt * iters * per / (ms * 1e-3)
    return {"fma_tflops": res[0] / 1e12, "exp_per_s": res[1], "threads": nb * nt,
            "how": "independent FP64 FMA / exp chains, best of 3 launches, CUDA events"}


def extra_workload(name, device, steps, warmup, peak, peak_kind, tune):
    """Whole-step rate of another paper-shaped workload (reported beside the
    headline): the two-body separation (C3-like) or the batched MEMS sweep."""
    import torch
    from paper_2604_09984_gb300 import ugks as U
    if name == "mems_batch":
        cases = wl.mems_batch()
        ms, units, launches, host_s, e2e_s, h2d, d2h, nfield, tiles = batch_arm(cases, steps, warmup, device)
        torch.cuda.empty_cache()
        return {"workload": "mems_batch: %d instances, %d field cells, 20^2-40^2 velocities, Kn 0.01-2"
                            % (len(cases), nfield),
                "value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
                "e2e": {"value": units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "roofline": None,
                "note": "per-instance kernels on 64 streams; roofline of the single-instance headline applies"}
    case = make_case(name, 0.01)
    s, ms, nfield, launches, _ = time_arm(case, U.FP32, steps, warmup, device, profile=False, tune=tune)
    prof = profiled_steps(s, 1)
    value = nfield * case.nv * case.n_inner * steps / (ms * 1e-3)
    roof = dominant_roofline(prof, nfield, case.nv, s.nc, 8, peak, peak_kind)
    tab = kernel_table(prof, nfield, case.nv, s.nc, 8)
    s.close()
    del s
    torch.cuda.empty_cache()
    return {"workload": workload_label(case), "value": value, "unit": UNIT, "ms_per_step": ms / steps,
            "steps": steps, "gpu_launches": launches, "roofline": roof, "kernels": tab}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mems", choices=["mems", "channel", "tsto", "mems_batch"])
    ap.add_argument("--instances", type=int, default=64, help="mems_batch: number of instances")
    ap.add_argument("--kn", type=float, default=0.1)
    ap.add_argument("--mesh", default=None,
                    help="mems: background and O-grid cells as NBIxNBJ+NOIxNOJ (default 256x128+128x32)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-plain comparison arm")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-bf16", action="store_true", help="skip the bf16-storage experiment arm")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the two-body and batched workloads reported beside the headline")
    ap.add_argument("--extra-steps", type=int, default=2)
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default sweep tile (for profiler runs, where the tuner's timings are distorted)")
    args = ap.parse_args()
    if args.workload == "mems_batch" or not args.no_extra:
        # one hardware work queue per instance stream (read when CUDA starts)
        os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
        if dist is not None:
            dist.destroy_process_group()
        return

    import torch
    from paper_2604_09984_gb300 import ugks as U
    device = "cuda:%d" % local
    torch.cuda.set_device(local)
    if args.workload == "mems_batch":
        run_batch(args, world, rank, device, dist)
        if dist is not None:
            dist.destroy_process_group()
        return
    case = make_case(args.workload, args.kn, args.mesh)
    steps = max(1, args.steps)
    warmup = max(3, args.warmup)
    peak, peak_kind = peaks()

    # the headline: timed steps with no per-launch event bracketing
    clk = Clocks(local)
    clk.start()
    s, ms, nfield, launches, _ = time_arm(case, U.FP32, steps, warmup, device, profile=False,
                                          tune=not args.no_tune, dist=dist)
    clocks = clk.stop()
    ms = max_over_ranks(ms, dist, device)
    units = nfield * case.nv * case.n_inner * steps * world
    value = units / (ms * 1e-3)
    # per-group table and the dominant kernel's roofline from separate
    # profiled steps (CUDA events on the stream each group is launched on)
    prof = profiled_steps(s, min(steps, 5))
    pair = 8
    default = args.workload == "mems" and args.kn == 0.1 and not args.mesh
    dom_tab = kernel_table(prof, nfield, case.nv, s.nc, pair)
    roof = dominant_roofline(prof, nfield, case.nv, s.nc, pair, peak, peak_kind)
    if default and roof.get("kernel"):
        roof["traffic"] = ncu_traffic(roof["kernel"])
    e2e_ms, h2d, d2h = e2e_arm(s, steps)
    e2e_val = nfield * case.nv * case.n_inner * steps * world / (e2e_ms * 1e-3)
    tiles = s.tiles
    s.close()
    del s
    torch.cuda.empty_cache()
    fp64 = None
    if not args.no_fp64:
        n64 = max(3, args.fp64_steps)
        s64, ms64, nf64, _, _ = time_arm(case, U.FP64, n64, 3, device, profile=False, tune=not args.no_tune)
        prof64 = profiled_steps(s64, 1)
        v64 = nf64 * case.nv * case.n_inner * n64 / (ms64 * 1e-3)
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": ms64 / n64, "steps": n64,
                "speedup_fp32_over_fp64": value / world / v64,
                "kernels": kernel_table(prof64, nf64, case.nv, s64.nc, 16)}
        r64 = dominant_roofline(prof64, nf64, case.nv, s64.nc, 16, peak, peak_kind)
        r64["note"] = "the FP64 path is bound by the FP64 pipe (probe below), not by HBM"
        fp64["roofline"] = r64
        s64.close()
        del s64
        torch.cuda.empty_cache()
        fp64["fp64_probe"] = fp64_probe(device)
    bf16 = None
    if not args.no_bf16:
        # experiment: f stored as bf16 pairs (same FP32 arithmetic)
        sb, msb, nfb, _, _ = time_arm(case, U.BF16F, steps, warmup, device, profile=False,
                                      tune=not args.no_tune)
        vb = nfb * case.nv * case.n_inner * steps / (msb * 1e-3)
        bf16 = {"value": vb, "unit": UNIT, "ms_per_step": msb / steps, "speedup_over_fp32": vb / (value / world),
                "note": "experiment: f stored as bf16 pairs, FP32 arithmetic; errors ~1e-3 relative"}
        sb.close()
        del sb
        torch.cuda.empty_cache()
    extra = None
    if not args.no_extra and args.workload == "mems" and world == 1:
        extra = {}
        for name in ("tsto", "mems_batch"):
            extra[name] = extra_workload(name, device, max(1, args.extra_steps), 3, peak, peak_kind,
                                         not args.no_tune)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_label(case),
                   "precision": "FP32 f and per-velocity arithmetic; FP64 moments, macroscopic update, "
                                "per-face interface state and geometry",
                   "l2": "inputs larger than L2 (f alone %.0f MB)" % (s_bytes(case) / 1e6),
                   "field_cells": nfield, "nv": case.nv, "n_inner": case.n_inner,
                   "tiles": ("autotuned (sweeps: items per warp step, velocities per lane, rings fwd/bwd; "
                             "face kernels: velocities per chunk, threads per face): %s" % (tiles,))
                   if tiles else "default (sweeps: 2 velocities per lane, rings of 4 steps; face kernels: 16, 2)",
                   "timing": "headline steps without per-launch events; kernel table and roofline from "
                             "separate profiled steps",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "per_physical_step": value / case.n_inner,
        "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roof,
        "kernels": dom_tab,
        "fp64_plain": fp64,
        "bf16_f_storage": bf16,
        "other_workloads": extra,
    }
    if rank == 0 and not args.no_cpu and world == 1:
        single = cpu_baseline(args.kn, steps=2)
        multi = cpu_baseline_multicore(args.kn)
        multi["single_core"] = single
        line["cpu_baseline"] = multi
    elif rank == 0:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def s_bytes(case):
    return case.ncells * case.nv * 8


if __name__ == "__main__":
    main()
