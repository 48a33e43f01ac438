"""Throughput of the PPML step on GB300: Mcell-updates/s, FP32 (headline) and FP64.

Workload: 3D point blast, 256^3 cells on [-0.5, 0.5]^3, gamma = 5/3, rho = 1, p = 1e-5,
E = 1 in the 8 central cells, outflow, CFL 0.2 (synthetic, seeded; no dataset).  One
step = Eulerian stage + Lagrangian stage + energy correction + CFL step + FP64 sums, all
in libppml.so through its C ABI.  The state (6 x 67 MB in FP32) is far larger than L2,
so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ppml|reference]
                       [--all-configs] [--cpu-table]
Under torchrun with N > 1 each rank advances its own replica (the grid is not split
across GPUs); value = all ranks' cell-updates / max-over-ranks time.

The line's "configs" object times the other workloads on the GPU beside the headline: the
1D Sod run to t = 0.2 (launch-bound), the planar Sod 128^3 in FP32 and FP64, and the 512^3
galactic disk (hydro steps with gravity; the Poisson solve between them untimed; a few
steps by default, --steps of them with --all-configs).  "fp32_double_float" times the same
256^3 step on a double-float state (rho, m, rho E as float pairs).  --cpu-table instead
times the FP64 oracle, as it stands, on a bounded sample of every workload with one thread
and with all host cores (no GPU use) and prints that table as its one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PPML Mcell-updates/s per step, FP32 vs FP64, and % of GB300 HBM roofline"
N_CELLS_SIDE = 256
# algorithmic bytes per cell per step (FP32 state): Eulerian reads 6 fields, writes 5;
# Lagrangian reads 6, writes 6.  FP64 doubles them.
BYTES_EUL = {4: 44, 8: 88}
BYTES_LAG = {4: 48, 8: 96}
# algorithmic FP32 operations per cell (add, mul, fma, min, compare, select, sqrt and
# divide each counted once) of the Lagrangian stage: 18 (field, axis) line updates of
# 62 (slope 12, face 4, parabola 26, upwind average 17, update 3), the velocity template
# and face velocities 57, energy correction 30, CFL terms 12, compensated sums 42.
OPS_LAG = 18 * 62 + 57 + 30 + 12 + 42
# Eulerian stage: per axis v and p parabolas 84, face constants 15, four averages 32,
# face solution 9, updates 8, v = m / rho 1; plus 6 for rho E and rho eps.
OPS_EUL = 3 * (84 + 15 + 32 + 9 + 8 + 1) + 6
# DRAM bytes of one Lagrangian launch measured by ncu (dram__bytes_read + write, one launch
# of the 256^3 point blast, the timed workload itself; see profiles/).
NCU_LAG_DRAM_BYTES_256 = 486.10e6 + 381.00e6
SMS, FP32_LANES = 152, 128


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def max_over_ranks(x, dist=None, device=None):
    """Largest value of x over all ranks (the job's time is the slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(cells_per_rank, steps, world, ms):
    """Cell-updates per second of the whole job (all ranks' work over the slowest time), in
    Mcell-updates/s."""
    return world * cells_per_rank * steps / (ms * 1e-3) / 1e6


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [x.strip() for x in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "1"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(workload_steps=1, max_seconds=30.0):
    """The FP64 oracle (as it stands) on the host cores: steps of the same 256^3 point
    blast, bounded in time.  Returns (Mcell-updates/s, cores, sample description)."""
    import oracle
    from paper_1607_01105_gb300 import inputs
    pb = inputs.point_blast_3d(N_CELLS_SIDE)
    g = oracle.Grid(pb.n, pb.h, pb.gamma, pb.bc, pb.cfl, rho_mean=oracle.mean_density(pb.u))
    u = pb.u
    dt = oracle.cfl_dt(g, u)
    t0 = time.perf_counter()
    steps = 0
    while steps < workload_steps:
        u, dg = oracle.step(g, u, dt)
        dt = dg["dt_cfl"]
        steps += 1
        if time.perf_counter() - t0 > max_seconds:
            break
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return pb.cells * steps / el / 1e6, cores, f"{steps} oracle step(s) of the 256^3 point blast from t=0", el


def _oracle_grid(pb):
    import oracle
    return oracle.Grid(pb.n, pb.h, pb.gamma, pb.bc, pb.cfl, rho_mean=oracle.mean_density(pb.u))


def _oracle_steps(pb, max_steps, max_seconds, phi=None):
    """Oracle steps of pb from t = 0 until max_steps or max_seconds (at least one); the
    CFL step of each comes from the previous step's diagnostics.  Returns (steps, s)."""
    import oracle
    g = _oracle_grid(pb)
    u = pb.u
    dt = oracle.cfl_dt(g, u)
    steps, el = 0, 0.0
    while steps < max_steps and (steps == 0 or el < max_seconds):
        t0 = time.perf_counter()
        u, dg = oracle.step(g, u, dt, phi=phi)
        el += time.perf_counter() - t0
        dt = dg["dt_cfl"]
        steps += 1
    return steps, el


def oracle_config_table(disk_n, max_seconds=15.0):
    """The FP64 oracle (as it stands) on a bounded sample of each workload, with the
    OpenMP thread count of this process.  Returns {workload: {mcups, seconds, sample}}."""
    import oracle
    from oracle import exact
    from paper_1607_01105_gb300 import inputs
    out = {}

    def put(name, updates, el, sample):
        out[name] = {"mcups": updates / el / 1e6, "seconds": el, "sample": sample}

    pb = inputs.sod_1d(256)
    t0 = time.perf_counter()
    _, _, steps, _ = oracle.run(_oracle_grid(pb), pb.u, pb.t_end)
    put("sod_1d_256", pb.cells * steps, time.perf_counter() - t0,
        f"full run to t = {pb.t_end}: {steps} steps")
    for name, pb in (("planar_sod_128", inputs.planar_sod_3d(128)),
                     ("point_blast_256", inputs.point_blast_3d(256))):
        steps, el = _oracle_steps(pb, 10, max_seconds)
        put(name, pb.cells * steps, el, f"{steps} step(s) from t = 0")
    bb = inputs.batched_riemann(max_speed=exact.riemann_max_speed)
    updates, el, done = 0.0, 0.0, 0
    for i in range(bb.ncells.size):
        n = int(bb.ncells[i])
        sl = slice(bb.offsets[i], bb.offsets[i + 1])
        z = np.zeros(n)
        u = [bb.u[0][sl], bb.u[1][sl], z, z, bb.u[2][sl], bb.u[3][sl]]
        g = oracle.Grid((n, 1, 1), (float(bb.h[i]), 1.0, 1.0), bb.gamma, (0,) * 6, bb.cfl,
                        rho_mean=float(np.mean(bb.u[0][sl])))
        t0 = time.perf_counter()
        _, _, steps, _ = oracle.run(g, [x[None, None, :] for x in u], float(bb.t_end[i]))
        el += time.perf_counter() - t0
        updates += n * steps
        done += 1
        if el > max_seconds:
            break
    put("batched_riemann_512", updates, el,
        f"instances 0..{done - 1} of the 512 (in generator order), each run to its end time")
    pb = inputs.galactic_disk(n=disk_n)
    steps, el = _oracle_steps(pb, 2, max_seconds, phi=pb.extra["phi_halo"])
    put("galactic_disk", pb.cells * steps, el,
        f"{disk_n}^3 disk, {steps} hydro step(s) with the fixed halo potential")
    return out


def cpu_table(args):
    """Oracle timings of every workload with 1 thread and with all host cores, each in a
    fresh process (OMP_NUM_THREADS fixed at its start); one JSON line."""
    cores = os.cpu_count() or 1
    table = {}
    for threads, disk_n in ((1, 128), (cores, 512)):
        env = dict(os.environ, OMP_NUM_THREADS=str(threads))
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-table-worker",
                            "--disk-n", str(disk_n)], env=env, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"oracle table worker ({threads} threads) failed:\n{r.stderr[-2000:]}")
        table[str(threads)] = json.loads(r.stdout.strip().splitlines()[-1])
    print(json.dumps({"cpu_table": table, "kind": "oracle", "unit": "Mcell-updates/s",
                      "cores": cores, "data": "synthetic"}), flush=True)
    return 0


def gpu_configs(args, dev, stream, barrier, disk_steps):
    """GPU timings of the other workloads through the same C ABI (CUDA events on the
    launching stream): the 1D Sod 256 run to t = 0.2 (the steps of the full run, counted
    in an untimed run first, then launched back to back from t = 0 on a fresh grid), the
    planar Sod 128^3 (warm-up, then timed steps) and optionally the 512^3 galactic disk
    (hydro steps with the periodic self-gravity solve plus the halo potential; each
    Poisson solve outside the timed events)."""
    import torch
    from paper_1607_01105_gb300 import inputs, ppml
    out = {}
    kinds = ((ppml.PPML_F32, "f32"), (ppml.PPML_F64, "f64"))

    def events():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    pb = inputs.sod_1d(256)
    res = {}
    for dtype, name in kinds:
        u = ppml.to_device(pb.u, dtype)
        v = [torch.empty_like(x) for x in u]
        g = ppml.Grid(pb.n, pb.h, pb.gamma, pb.cfl, pb.bc, dtype, u0=u, t_end=pb.t_end)
        uu, vv, steps = [x.clone() for x in u], v, 0
        while g.diag(raise_nonphysical=False)["dt_next"] > 0.0 and steps < 100000:
            g.step(uu, vv, 0.0)
            uu, vv = vv, uu
            steps += 1
        g.close()
        g = ppml.Grid(pb.n, pb.h, pb.gamma, pb.cfl, pb.bc, dtype, u0=u, t_end=pb.t_end)
        uu, vv = [x.clone() for x in u], v
        e0, e1 = events()
        barrier()
        e0.record(stream)
        for _ in range(steps):
            g.step(uu, vv, 0.0)
            uu, vv = vv, uu
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        t = g.diag(raise_nonphysical=False)["t"]
        g.close()
        res[name] = {"value": pb.cells * steps / (ms * 1e-3) / 1e6, "ms": ms, "steps": steps,
                     "t": t}
    out["sod_1d_256"] = dict(res, unit="Mcell-updates/s",
                             workload="Sod (Table 2 row 1), 256 cells, CFL 0.4, outflow, run to "
                                      "t = 0.2, through the grid path (three launches per step)")
    # the same run as a batch of one instance: the whole run in one persistent launch
    res = {}
    for dtype, name in kinds:
        st = [torch.as_tensor(np.asarray(pb.u[f]).ravel()).to(dev, ppml.torch_dtype(dtype))
              for f in (0, 1, 4, 5)]
        b = ppml.Batch([pb.cells], [pb.h[0]], [pb.t_end], pb.gamma, pb.cfl, dtype)
        e0, e1 = events()
        barrier()
        e0.record(stream)
        b.step(st, 1 << 30)
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        t, steps = b.status()
        b.close()
        res[name] = {"value": pb.cells * steps[0] / (ms * 1e-3) / 1e6, "ms": ms,
                     "steps": int(steps[0]), "t": float(t[0])}
    out["sod_1d_256_batch"] = dict(res, unit="Mcell-updates/s",
                                   workload="the same Sod run as a batch of one instance "
                                            "(ppml_batch_step: one launch for the whole run)")
    pb = inputs.planar_sod_3d(128)
    res = {}
    for dtype, name in kinds:
        steps = args.steps if dtype == ppml.PPML_F32 else max(3, args.steps // 10)
        u = ppml.to_device(pb.u, dtype)
        v = [torch.empty_like(x) for x in u]
        g = ppml.Grid(pb.n, pb.h, pb.gamma, pb.cfl, pb.bc, dtype, u0=u)
        for _ in range(args.warmup):
            g.step(u, v, 0.0)
            u, v = v, u
        e0, e1 = events()
        barrier()
        e0.record(stream)
        for _ in range(steps):
            g.step(u, v, 0.0)
            u, v = v, u
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        g.close()
        res[name] = {"value": pb.cells * steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps,
                     "steps": steps}
    out["planar_sod_128"] = dict(res, unit="Mcell-updates/s",
                                 workload="planar Sod 128^3, split on x = 0.5, outflow in x, "
                                          "periodic in y and z, CFL 0.2")
    if disk_steps > 0:
        pb = inputs.galactic_disk(n=512)
        dtype = ppml.PPML_F32
        u = ppml.to_device(pb.u, dtype)
        v = [torch.empty_like(x) for x in u]
        g = ppml.Grid(pb.n, pb.h, pb.gamma, pb.cfl, pb.bc, dtype, u0=u)
        halo = torch.as_tensor(pb.extra["phi_halo"].ravel()).to(dev, torch.float32)
        phi = torch.empty_like(u[0])
        ms, steps = 0.0, disk_steps
        for k in range(min(args.warmup, 3) + steps):
            g.poisson_periodic(u[0], phi, 1.0)
            phi.add_(halo)
            e0, e1 = events()
            barrier()
            e0.record(stream)
            g.step_phi(u, v, phi, 0.0)
            e1.record(stream)
            barrier()
            if k >= min(args.warmup, 3):
                ms += e0.elapsed_time(e1)
            u, v = v, u
        g.close()
        out["galactic_disk_512"] = {
            "f32": {"value": pb.cells * steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps,
                    "steps": steps},
            "unit": "Mcell-updates/s",
            "workload": "galactic disk 512^3 (exponential disk in a fixed halo, G = 1), FP32; "
                        "hydro steps with gravity, each step timed alone, the Poisson solve "
                        "before it untimed"}
        del u, v, phi, halo
        torch.cuda.empty_cache()
    return out


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(1)
    t0 = time.perf_counter()
    tot_cells = 0
    for _ in range(args.steps):
        v, cores, sample, el = cpu_baseline(1)
        vals.append(el)
        tot_cells += N_CELLS_SIDE ** 3
    el = time.perf_counter() - t0
    value = tot_cells / el / 1e6
    line = {"metric": METRIC, "value": value, "unit": "Mcell-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "point_blast_3d 256^3, gamma=5/3, CFL 0.2, outflow",
                       "global_batch": 1, "seq_len": 0, "parallelism": "host cores (OpenMP)"},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value,
                             "unit": "Mcell-updates/s",
                             "sample": f"{args.steps} timed oracle steps of the 256^3 point blast"},
            "e2e": {"value": value, "unit": "Mcell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def profile_run(args):
    """K plain FP32 steps of the n^3 point blast, untimed (for ncu captures: launch k of a
    stage kernel is step k's)."""
    import torch
    from paper_1607_01105_gb300 import inputs, ppml
    torch.cuda.set_device(0)
    pb = inputs.point_blast_3d(args.n)
    u = ppml.to_device(pb.u, ppml.PPML_F32)
    v = [torch.empty_like(x) for x in u]
    grid = ppml.Grid(pb.n, pb.h, pb.gamma, pb.cfl, pb.bc, ppml.PPML_F32, u0=u)
    for _ in range(args.steps):
        grid.step(u, v, 0.0)
        u, v = v, u
    torch.cuda.synchronize()
    print(json.dumps({"profile_run": args.n, "steps": args.steps, "t": grid.diag()["t"]}))
    return 0


def slab_bench(args):
    """The FP32 step of the n^3 point blast split into z slabs (one per rank; on one GPU,
    --emulate-ranks slabs driven by this process): exchange of U^n and U* halo planes,
    both stages, all-reduce of the CFL maxima and sums, per step.  Strong scaling: value =
    the whole grid's cell-updates / max-over-ranks time."""
    import torch
    import torch.distributed as dist
    from paper_1607_01105_gb300 import inputs, ppml, slab
    import oracle  # mean density of the input only (the vacuum threshold's reference)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local if world > 1 else 0)
    if world > 1:
        dist.init_process_group("nccl")
    pb = inputs.point_blast_3d(args.n)
    rho_ref = oracle.mean_density(pb.u)
    if world > 1:
        layouts = [slab.SlabLayout(pb.n, pb.bc, world, rank)]
        comm = slab.DistComm(dist, layouts[0])
    else:
        k = max(1, args.emulate_ranks)
        layouts = [slab.SlabLayout(pb.n, pb.bc, k, r) for r in range(k)]
        comm = slab.LocalComm(layouts)
    stages = [slab.Stages(ppml, L, pb.h, pb.gamma, pb.cfl, ppml.PPML_F32,
                          [slab.pad_field(L, u, torch.float32, "cuda") for u in pb.u], rho_ref)
              for L in layouts]
    slab.start(stages, comm)
    for _ in range(args.warmup):
        slab.step(stages, comm)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as cs:
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            slab.step(stages, comm)
        e1.record(stream)
        barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, torch.device("cuda", torch.cuda.current_device()))
    if rank == 0:
        value = pb.cells * args.steps / (ms * 1e-3) / 1e6
        nslab = world if world > 1 else len(layouts)
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "Mcell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"point_blast_3d {args.n}^3 split into {nslab} z slabs "
                                   f"({[L.nz for L in layouts] if world == 1 else 'one per rank'} "
                                   f"planes), FP32; halo exchange of U^n and U*, all-reduce of the "
                                   f"CFL maxima and sums every step",
                       "global_batch": 1, "seq_len": 0,
                       "parallelism": f"z-slabs x{world}" if world > 1 else
                                      f"{nslab} slabs in one process (plane copies)"},
            "gpu_launches": 4 * len(layouts) * args.steps,  # two stages, reduce, apply
            "clocks": cs.summary()}), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ppml", choices=["ppml", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=N_CELLS_SIDE)
    ap.add_argument("--all-configs", action="store_true")
    ap.add_argument("--cpu-table", action="store_true")
    ap.add_argument("--cpu-table-worker", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--disk-n", type=int, default=512, help=argparse.SUPPRESS)
    ap.add_argument("--decomp", default="replicas", choices=["replicas", "slab"],
                    help="ranks run replicas of the grid (default) or z slabs of one grid")
    ap.add_argument("--emulate-ranks", type=int, default=2,
                    help="--decomp slab on one GPU: slabs driven by this one process")
    ap.add_argument("--profile-run", action="store_true",
                    help="only run --steps plain FP32 steps of the --n^3 point blast (x-major "
                         "tiles, device CFL step) and exit: the program a profiler captures")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.cpu_table_worker:
        print(json.dumps(oracle_config_table(args.disk_n)), flush=True)
        return 0
    if args.cpu_table:
        return cpu_table(args)
    if args.profile_run:
        return profile_run(args)
    if args.decomp == "slab":
        return slab_bench(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_1607_01105_gb300 import inputs, ppml

    pb = inputs.point_blast_3d(args.n)
    cells = pb.cells
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks_(x):
        return max_over_ranks(x, dist, dev)

    results = {}
    # batched uneven 1D Riemann problems (512 instances, 128..4096 cells): one persistent
    # launch advances every instance to its own end time
    from oracle import exact
    bb = inputs.batched_riemann(max_speed=exact.riemann_max_speed)
    bst = [torch.as_tensor(x).to(dev, torch.float32) for x in bb.u]
    batch = ppml.Batch(bb.ncells, bb.h, bb.t_end, bb.gamma, bb.cfl, ppml.PPML_F32)
    # CTA size per instance picked by the library's autotuner (untimed; scratch copies)
    b_threads, b_tune = batch.tune(bst, trial_steps=20, stream=stream)
    barrier()
    b0 = torch.cuda.Event(enable_timing=True)
    b1 = torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    batch.step(bst, 1 << 30)
    b1.record(stream)
    barrier()
    bms = b0.elapsed_time(b1)
    bt_t, bt_steps = batch.status()
    batch_updates = float(np.dot(bb.ncells.astype(np.float64), np.asarray(bt_steps, dtype=np.float64)))
    results["batch"] = {"ms": max_over_ranks_(bms), "updates": batch_updates,
                        "instances": int(bb.ncells.size), "cells": int(bb.cells),
                        "done": int(sum(1 for t, te in zip(bt_t, bb.t_end) if t >= te)),
                        "threads": b_threads, "tune_ms": {str(k): v for k, v in b_tune.items()}}
    # the same FP32 batch on a double-float state (rho, m, rho E as float pairs)
    bst = [torch.as_tensor(x).to(dev, torch.float32) for x in bb.u]
    blo = [(torch.as_tensor(x).to(dev) - y.double()).float() for x, y in zip(bb.u[:3], bst[:3])]
    batch_df = ppml.Batch(bb.ncells, bb.h, bb.t_end, bb.gamma, bb.cfl, ppml.PPML_F32)
    batch_df.set_threads(b_threads)
    barrier()
    b0.record(stream)
    batch_df.step(bst, 1 << 30, lo=blo)
    b1.record(stream)
    barrier()
    _, bdf_steps = batch_df.status()
    results["batch_df"] = {"ms": max_over_ranks_(b0.elapsed_time(b1)),
                           "updates": float(np.dot(bb.ncells.astype(np.float64),
                                                   np.asarray(bdf_steps, dtype=np.float64)))}
    batch.close()
    batch_df.close()
    del bst, blo
    # the same batch in FP64 (its own autotuned CTA size)
    bst64 = [torch.as_tensor(x).to(dev, torch.float64) for x in bb.u]
    batch64 = ppml.Batch(bb.ncells, bb.h, bb.t_end, bb.gamma, bb.cfl, ppml.PPML_F64)
    b64_threads, _ = batch64.tune(bst64, trial_steps=5, stream=stream)
    barrier()
    b0.record(stream)
    batch64.step(bst64, 1 << 30)
    b1.record(stream)
    barrier()
    b64ms = b0.elapsed_time(b1)
    _, b64_steps = batch64.status()
    results["batch64"] = {"ms": max_over_ranks_(b64ms), "threads": b64_threads,
                          "updates": float(np.dot(bb.ncells.astype(np.float64),
                                                  np.asarray(b64_steps, dtype=np.float64)))}
    batch64.close()
    del bst64
    for dtype, name, df in ((ppml.PPML_F32, "f32", False), (ppml.PPML_F32, "f32df", True),
                            (ppml.PPML_F64, "f64", False)):
        elt = 4 if dtype == ppml.PPML_F32 else 8
        u = ppml.to_device(pb.u, dtype, lo=df)
        v = [torch.empty_like(x) for x in u]
        grid = ppml.Grid(pb.n, pb.h, pb.gamma, pb.cfl, pb.bc, dtype, u0=u)
        tile_tune = None
        if name == "f32":  # tile launch order picked by the library's autotuner (untimed)
            tile_tune = grid.tune(u, trial_steps=5)
            tile_order = tile_tune[0]
        elif dtype == ppml.PPML_F32:
            grid.set_order(tile_order)
        steps = args.steps if dtype == ppml.PPML_F32 else max(3, args.steps // 10)
        if df:
            steps = max(3, args.steps // 2)
        for _ in range(args.warmup):
            grid.step(u, v, 0.0)
            u, v = v, u
        barrier()
        grid.profile(True)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as cs:
            barrier()
            ev0.record(stream)
            for _ in range(steps):
                grid.step(u, v, 0.0)
                u, v = v, u
            ev1.record(stream)
            barrier()
        ms = ev0.elapsed_time(ev1)
        kms, ksteps = grid.kernel_times()
        grid.profile(False)
        d = grid.diag(raise_nonphysical=False)
        ms = max_over_ranks_(ms)
        results[name] = {"ms": ms, "steps": steps, "kernel_ms": [x / ksteps for x in kms],
                         "clocks": cs.summary(), "elt": elt, "diag": d, "tile_tune": tile_tune}
        # end to end through host buffers (FP32 headline only): every step copies its input
        # state from pinned host memory, steps, and copies the new state back to pinned host
        # memory, all inside the timed region.  Uploads and downloads run on their own
        # streams with two device buffers each, so the upload of step k overlaps the step
        # and the download of step k-1 (events order every reuse of a buffer).
        if name == "f32":
            hin = [x.cpu().pin_memory() for x in u]
            hout = [[torch.empty(x.shape, dtype=x.dtype).pin_memory() for x in hin]
                    for _ in range(2)]
            dev_in = [u, [torch.empty_like(x) for x in u]]
            dev_out = [v, [torch.empty_like(x) for x in u]]
            s_up, s_down = torch.cuda.Stream(), torch.cuda.Stream()
            ev_up = [torch.cuda.Event() for _ in range(2)]
            ev_step = [torch.cuda.Event() for _ in range(2)]
            ev_down = [torch.cuda.Event() for _ in range(2)]
            e_steps = max(6, steps // 2)
            e2e_ms = []
            for _rep in range(3):  # three end-to-end runs: the median is reported
                torch.cuda.synchronize()
                barrier()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s_up.wait_stream(stream)
                s_down.wait_stream(stream)
                for k in range(e_steps):
                    i = k % 2
                    if k >= 2:
                        s_up.wait_event(ev_step[i])  # step k-2 has read dev_in[i]
                    with torch.cuda.stream(s_up):
                        for dst, src in zip(dev_in[i], hin):
                            dst.copy_(src, non_blocking=True)
                    ev_up[i].record(s_up)
                    stream.wait_event(ev_up[i])
                    if k >= 2:
                        stream.wait_event(ev_down[i])  # step k-2's result has left dev_out[i]
                    grid.step(dev_in[i], dev_out[i], 0.0, stream=stream)
                    ev_step[i].record(stream)
                    s_down.wait_event(ev_step[i])
                    with torch.cuda.stream(s_down):
                        for dst, src in zip(hout[i], dev_out[i]):
                            dst.copy_(src, non_blocking=True)
                    ev_down[i].record(s_down)
                stream.wait_stream(s_up)
                stream.wait_stream(s_down)
                e1.record(stream)
                barrier()
                e2e_ms.append(max_over_ranks_(e0.elapsed_time(e1)))
            results["e2e"] = {"ms": statistics.median(e2e_ms), "ms_runs": e2e_ms, "steps": e_steps,
                              "h2d": 6 * cells * elt, "d2h": 6 * cells * elt}
            # the same step mid-run: advance (untimed) toward half the time at which the blast
            # radius reaches 0.4, at most 4000 steps, then time as many steps again
            t_mid, adv = 0.5 * pb.t_end, 0
            while grid.diag(raise_nonphysical=False)["t"] < t_mid and adv < 4000:
                for _ in range(100):
                    grid.step(u, v, 0.0)
                    u, v = v, u
                adv += 100
            barrier()
            m0 = torch.cuda.Event(enable_timing=True)
            m1 = torch.cuda.Event(enable_timing=True)
            m0.record(stream)
            for _ in range(steps):
                grid.step(u, v, 0.0)
                u, v = v, u
            m1.record(stream)
            barrier()
            dm = grid.diag(raise_nonphysical=False)
            results["mid"] = {"ms": max_over_ranks_(m0.elapsed_time(m1)), "steps": steps,
                              "t": dm["t"], "steps_before": args.warmup + steps + e_steps + adv,
                              "t_end": pb.t_end}
        grid.close()
        del u, v
        torch.cuda.empty_cache()

    configs = gpu_configs(args, dev, stream, barrier, args.steps if args.all_configs else 6)
    # measured FMA throughput of the device (the arithmetic roofline denominators)
    fma_peak = {"f32": ppml.fma_peak(ppml.PPML_F32, 200000, stream=stream),
                "f64": ppml.fma_peak(ppml.PPML_F64, 4000, stream=stream)}

    if rank == 0:
        peak, peak_kind = load_peaks()
        r32, r64, rdf = results["f32"], results["f64"], results["f32df"]
        value = whole_job_rate(cells, r32["steps"], world, r32["ms"])
        v64 = whole_job_rate(cells, r64["steps"], world, r64["ms"])
        keul, klag, kfin = r32["kernel_ms"]
        clk = r32["clocks"].get("sm_max_mhz") or 2070.0
        alu_peak = SMS * FP32_LANES * clk * 1e6 / 1e12  # FP32 lane operations, Top/s
        lag_ops = OPS_LAG * cells / (klag * 1e-3) / 1e12
        eul_ops = OPS_EUL * cells / (keul * 1e-3) / 1e12
        lag_gbs = BYTES_LAG[4] * cells / (klag * 1e-3) / 1e9
        eul_gbs = BYTES_EUL[4] * cells / (keul * 1e-3) / 1e9
        step_bytes = (BYTES_EUL[4] + BYTES_LAG[4]) * cells
        e2e = results["e2e"]
        e2e_val = whole_job_rate(cells, e2e["steps"], world, e2e["ms"])
        e2e_runs = [whole_job_rate(cells, e2e["steps"], world, x) for x in e2e["ms_runs"]]
        line = {
            "metric": METRIC, "value": value, "unit": "Mcell-updates/s", "n_gpus": world,
            "steps": r32["steps"], "warmup": args.warmup, "ms_per_step": r32["ms"] / r32["steps"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"point_blast_3d {args.n}^3, gamma=5/3, rho=1, p=1e-5, E=1 in "
                                   f"the 8 central cells, CFL 0.2, outflow; FP32 state; dt, sums and "
                                   f"the energy difference at FP64-class accuracy",
                       "global_batch": 1, "seq_len": 0,
                       "tile_order": r32["tile_tune"][0],
                       "tile_order_trial_ms": {str(k): v for k, v in r32["tile_tune"][1].items()},
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "no flush: state 403 MB x 2 + U* 336 MB > 129 MB L2"},
            "roofline": {"bound": "alu", "kernel": "lagrangian_tile<float>",
                         "achieved": lag_ops, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": lag_ops / alu_peak,
                         "hbm_frac": lag_gbs / peak,
                         "hbm_achieved_gbs": lag_gbs,
                         "peak_basis": f"{SMS} SMs x {FP32_LANES} FP32 lanes x {clk:.0f} MHz, "
                                       "one operation per lane per clock (FMA counted once)",
                         "algorithmic_ops_per_cell": OPS_LAG,
                         "traffic": NCU_LAG_DRAM_BYTES_256 if args.n == 256 else None,
                         "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                         "launch of the 256^3 point blast (51.7 B/cell; 48 "
                                         "algorithmic)",
                         "kernel_ms": {"eulerian": keul, "lagrangian": klag, "finalize": kfin},
                         "eulerian": {"achieved": eul_ops, "frac": eul_ops / alu_peak,
                                      "algorithmic_ops_per_cell": OPS_EUL},
                         "hbm": {"peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                                 "lagrangian_achieved": lag_gbs, "lagrangian_frac": lag_gbs / peak,
                                 "eulerian_achieved": eul_gbs, "eulerian_frac": eul_gbs / peak,
                                 "algorithmic_bytes_per_cell": BYTES_EUL[4] + BYTES_LAG[4],
                                 "step_frac": step_bytes / (r32["ms"] / r32["steps"] * 1e-3) / 1e9 / peak}},
            "fp64": {"value": v64, "unit": "Mcell-updates/s", "ms_per_step": r64["ms"] / r64["steps"],
                     "steps": r64["steps"], "kernel_ms": r64["kernel_ms"],
                     "roofline": {"bound": "alu", "kernel": "lagrangian_tile<double>",
                                  "achieved": OPS_LAG * cells / (r64["kernel_ms"][1] * 1e-3) / 1e12,
                                  "peak": fma_peak["f64"] / 1e12, "unit": "TFLOP/s",
                                  "frac": OPS_LAG * cells / (r64["kernel_ms"][1] * 1e-3) / fma_peak["f64"],
                                  "peak_kind": "measured FP64 FMA throughput (ppml_fma_peak), "
                                               "an FMA counted once",
                                  "algorithmic_ops_per_cell": OPS_LAG,
                                  "note": "IEEE division and square root are sequences of "
                                          "several FP64 instructions but count once"}},
            "fma_peak_measured": {"f32_tfma_s": fma_peak["f32"] / 1e12,
                                  "f64_tfma_s": fma_peak["f64"] / 1e12,
                                  "lagrangian_f32_frac_of_measured": lag_ops * 1e12 / fma_peak["f32"]},
            "batch_riemann": {"value": results["batch"]["updates"] / (results["batch"]["ms"] * 1e-3) / 1e6,
                              "unit": "Mcell-updates/s", "ms": results["batch"]["ms"],
                              "instances": results["batch"]["instances"],
                              "cells": results["batch"]["cells"],
                              "finished": results["batch"]["done"], "dtype": "f32",
                              "cta_threads": results["batch"]["threads"],
                              "fp64": {"value": results["batch64"]["updates"]
                                       / (results["batch64"]["ms"] * 1e-3) / 1e6,
                                       "ms": results["batch64"]["ms"],
                                       "cta_threads": results["batch64"]["threads"]},
                              "double_float": {"value": results["batch_df"]["updates"]
                                               / (results["batch_df"]["ms"] * 1e-3) / 1e6,
                                               "ms": results["batch_df"]["ms"]},
                              "tune_ms_20_steps": results["batch"]["tune_ms"],
                              "workload": "512 uneven 1D Riemann problems (128..4096 cells), "
                                          "each run to its own end time in one persistent launch"},
            "mid_run": {"value": whole_job_rate(cells, results["mid"]["steps"], world, results["mid"]["ms"]),
                        "unit": "Mcell-updates/s", "ms_per_step": results["mid"]["ms"] / results["mid"]["steps"],
                        "t": results["mid"]["t"], "t_end": results["mid"]["t_end"],
                        "steps_before": results["mid"]["steps_before"],
                        "note": "same FP32 step timed after advancing toward half the end time "
                                "(at most 4000 steps; t reached is given)"},
            "e2e": {"value": e2e_val, "unit": "Mcell-updates/s",
                    "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
                    "runs": e2e_runs, "min": min(e2e_runs), "stat": "median of 3 runs"},
            "fp32_double_float": {
                "value": whole_job_rate(cells, rdf["steps"], world, rdf["ms"]),
                "unit": "Mcell-updates/s", "ms_per_step": rdf["ms"] / rdf["steps"],
                "steps": rdf["steps"], "kernel_ms": rdf["kernel_ms"],
                "note": "the same FP32 step on a double-float state: rho, m, rho E stored as "
                        "float pairs (+36 B/cell/step), updates and the energy difference in "
                        "double-float"},
            "configs": configs,
            "gpu_launches": 3 * r32["steps"],
            "clocks": r32["clocks"],
            "clocks_fp64": r64["clocks"],
        }
        if not args.no_cpu_baseline:
            cv, cores, sample, el = cpu_baseline(1)
            line["cpu_baseline"] = {"value": cv, "unit": "Mcell-updates/s", "cores": cores,
                                    "kind": "oracle", "sample": sample, "seconds": el}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
