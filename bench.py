"""Benchmark: fine-level velocity DoF/s per AGCA V-cycle and Stokes solve time
to a 1e-8 relative residual, on synthetic 8-sphere sinker problems.

Workload (default): 64^3 pressure cubes (128^3 velocity cubes, 6,440,067
velocity DoF, 6 levels), 8 tanh-smoothed spherical sinkers with seeded
centres in [0.2, 0.8]^3, radius 0.08, width 0.01, jump 1e6, threshold nu = 10.
A step is one V(2,2) cycle of the mixed-precision preconditioner (FP32 cycle)
on a residual resident in HBM; the whole-solve times (setup and MINRES to
1e-8, FP64 and mixed) are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs an independent replica of the workload
(weak scaling, no collective on the data path); rank 0 prints one JSON line.
--impl reference times the CPU oracle on the host cores instead.
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

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "fine-level velocity DoF/s per V-cycle; Stokes solve time to 1e-8 rel. residual"
UNIT = "DoF/s"


def workload_params(N):
    return dict(N=N, n_sinkers=8, radius=0.08, width=0.01, dr=1e6, nu=10.0)


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _init_pg(world, backend):
    if world > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)
        return dist
    return None


def _barrier(dist):
    if dist is not None:
        dist.barrier()


def _max_over_ranks(dist, value, device):
    if dist is None:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.first = ""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            # nvidia-smi's start-up (NVML initialisation) must not overlap the timed region
            self.first = self.proc.stdout.readline()
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.first + out).strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per finest-level
# stencil launch of the 64^3 workload, mean over the four launches of one
# V-cycle (pre-smoothing 109.8 MB, residual 106.0 MB, first post-smoothing step
# 135.0 MB, last step with the FP64-widened result 183.2 MB), from one ncu
# capture of the current kernel; the algorithmic bytes of the same launches
# average 154.6 MB (part of the inputs is still in L2 from the previous launch)
FINE_STENCIL_DRAM_BYTES = 133.5e6


def bench_levels(N):
    """Levels of the benchmark hierarchy: coarsen the 2N velocity grid while
    it stays even with >= 4 cubes (the library's default)."""
    n, L = 2 * N, 1
    while n % 2 == 0 and n // 2 >= 4:
        n //= 2
        L += 1
    return L


def arm_config(N, L, flagged, world):
    return {"workload": "8-sphere sinker, jump 1e6, nu 10, V(2,2) mixed AGCA cycle",
            "N_pressure": N, "velocity_cubes": 2 * N, "levels": L, "velocity_dofs": 3 * (2 * N + 1) ** 3,
            "flagged_per_level": flagged, "global_batch": world, "seq_len": None,
            "parallelism": f"replicas{world}",
            "l2": "inputs larger than L2 (cycle working set ~0.3 GB > 129 MB), no flush"}


def oracle_vcycle_rate(seconds=15.0, N=16):
    """CPU oracle: DoF/s of its V-cycle on the same field family at a size it
    handles in seconds (the 64^3 hierarchy does not fit its sparse matrices)."""
    from oracle import agca as oagca
    from synth import random_vector, sphere_sinkers

    prm = workload_params(N)
    p = sphere_sinkers(N, prm["n_sinkers"], prm["radius"], prm["width"], prm["dr"])
    L = {8: 3, 16: 4, 32: 5}.get(N, 4)
    H = oagca.Hierarchy(N, L, p.eta, prm["nu"])
    n = 3 * H.mesh[L].nv
    r = random_vector(n, 3) * H.mask[L]
    H.vcycle(r)
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < seconds:
        H.vcycle(r)
        k += 1
    dt = (time.perf_counter() - t0) / k
    dofs = 3 * (2 * N + 1) ** 3
    # the V-cycle's work is scipy CSR products, which run on one thread
    return dofs / dt, k, dt, 1


def run_reference(args):
    """The oracle as it stands, timed on the host cores: each step is one
    oracle V-cycle of the benchmark's field family at 16^3 pressure cubes (a
    bounded sample of the 64^3 workload, whose hierarchy the oracle's sparse
    matrices do not fit in seconds), reported as DoF/s on the same config."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import agca as oagca
    from synth import random_vector, sphere_sinkers

    Nw = args.N or 64
    Lw = bench_levels(Nw)
    pw = workload_params(Nw)
    pfull = sphere_sinkers(Nw, pw["n_sinkers"], pw["radius"], pw["width"], pw["dr"])
    _, _, _, flags = oagca.flag_hierarchy(Nw, Lw, pfull.eta, pw["nu"])
    flagged = [int(flags[l].sum()) for l in range(1, Lw)]
    del pfull

    N = 16
    prm = workload_params(N)
    p = sphere_sinkers(N, prm["n_sinkers"], prm["radius"], prm["width"], prm["dr"])
    H = oagca.Hierarchy(N, 4, p.eta, prm["nu"])
    n = 3 * H.mesh[4].nv
    r = random_vector(n, 3) * H.mask[4]
    for _ in range(args.warmup):
        H.vcycle(r)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        H.vcycle(r)
    dt = (time.perf_counter() - t0) / args.steps
    dofs = 3 * (2 * N + 1) ** 3
    value = dofs / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": arm_config(Nw, Lw, flagged, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} oracle V-cycles at 16^3 pressure cubes of the same "
                                       f"8-sphere field family ({dt * 1e3:.0f} ms each; scipy CSR products "
                                       f"on one thread)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args, dev, stream):
    """The 24-problem batch (uneven 32^3/48^3/64^3 sinkers): batched V-cycle
    throughput against the same problems cycled one by one, and batched solve
    time to 1e-8 against sequential solves."""
    import paper_2511_13109_gb300 as pkg
    from synth import batch_problems

    probs = batch_problems(device=dev)
    if args.batch_n:
        probs = probs[:args.batch_n]
    etas = [torch.from_numpy(p.eta).to(dev) for p in probs]
    fbars = [torch.from_numpy(p.fbar.ravel()).to(dev) for p in probs]
    out = {"problems": len(probs), "sizes": [p.N for p in probs]}
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        b = pkg.Batch([p.N for p in probs], pkg.MIXED, device=dev, stream=stream)
        b.prepare(etas, 10.0)
        stream.synchronize()
        out["setup_s"] = time.perf_counter() - t0
        rs = [torch.rand(3 * c.V[c.L], dtype=torch.float64, device=dev) * 2 - 1 for c in b.contexts]
        zs = [torch.empty_like(r) for r in rs]
        dofs = sum(3 * c.V[c.L] for c in b.contexts)
        for _ in range(3):
            b.vcycle(rs, zs)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = 20
        e0.record(stream)
        for _ in range(k):
            b.vcycle(rs, zs)
        e1.record(stream)
        e1.synchronize()
        out["batched_vcycle_dofs_per_s"] = dofs / (e0.elapsed_time(e1) / k * 1e-3)
        singles = []
        for p, eta in zip(probs, etas):
            c = pkg.Context(p.N, pkg.default_levels(p.N), pkg.MIXED, device=dev, stream=stream)
            c.prepare(eta, 10.0)
            singles.append(c)
        for c, r, z in zip(singles, rs, zs):
            c.vcycle(r, z)
        e0.record(stream)
        for _ in range(k):
            for c, r, z in zip(singles, rs, zs):
                c.vcycle(r, z)
        e1.record(stream)
        e1.synchronize()
        out["sequential_vcycle_dofs_per_s"] = dofs / (e0.elapsed_time(e1) / k * 1e-3)
        if not args.no_solve:
            bs = [b.load_vector(i, f) for i, f in enumerate(fbars)]
            stream.synchronize()
            t0 = time.perf_counter()
            xs, its, rel = b.solve(bs, 1e-8, 40000)
            stream.synchronize()
            out["batched_solve_s"] = time.perf_counter() - t0
            out["batched_iters"] = its
            out["batched_max_relres"] = max(rel)
            t0 = time.perf_counter()
            for c, bb in zip(singles, bs):
                c.solve(bb, 1e-8, 40000)
            stream.synchronize()
            out["sequential_solve_s"] = time.perf_counter() - t0
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=64)
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--batch", action="store_true", help="also run the 24-problem batch")
    ap.add_argument("--batch-n", type=int, default=0)
    ap.add_argument("--solve-iters", type=int, default=0,
                    help="profiling aid: run only K MINRES iterations of the workload's mixed solve "
                         "inside the NVTX range 'solve', print one short JSON line and exit")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = _init_pg(world, "nccl")

    import __graft_entry__

    __graft_entry__.build()
    import paper_2511_13109_gb300 as pkg
    from synth import sphere_sinkers_on_device

    prm = workload_params(args.N)
    N = prm["N"]
    L = pkg.default_levels(N)
    # element fields generated on the device (no host copies: 26 GB at N = 256)
    eta, fbar, _ = sphere_sinkers_on_device(N, prm["n_sinkers"], prm["radius"], prm["width"], prm["dr"], device=dev)
    fbar = fbar.reshape(-1)

    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        ctx = pkg.Context(N, L, pkg.MIXED, device=dev, stream=stream)
        ctx.prepare(eta, prm["nu"])
        if args.no_solve and args.solve_iters <= 0:
            fbar = None  # only the solves load it
        t_tune = time.perf_counter()
        tune_cache = os.path.join(tempfile.mkdtemp(prefix="agca_bench_"), "tiles.txt")
        tuned = ctx.autotune(reps=10, cache=tune_cache) if not args.no_tune else {}
        t_tune = time.perf_counter() - t_tune
        if args.solve_iters > 0:
            b = ctx.load_vector(fbar)
            stream.synchronize()
            torch.cuda.nvtx.range_push("solve")
            try:
                _, its, rel = ctx.solve(b, 1e-8, args.solve_iters)
            except pkg.AgcaError as e:  # stopped at the iteration limit above the tolerance
                its, rel = args.solve_iters, str(e)
            stream.synchronize()
            torch.cuda.nvtx.range_pop()
            if rank == 0:
                print(json.dumps({"solve_iters": its, "relres": rel}), flush=True)
            return 0
        n3 = 3 * ctx.V[L]
        g = torch.Generator(device=dev)
        g.manual_seed(1234 + rank)
        r = torch.rand(n3, dtype=torch.float64, device=dev, generator=g) * 2 - 1
        z = torch.empty_like(r)
        for _ in range(args.warmup):
            ctx.vcycle(r, z)
        stream.synchronize()
        _barrier(dist)
        clocks = ClockSampler(local)
        launches0 = ctx.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        for _ in range(args.steps):
            ctx.vcycle(r, z)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        e1.synchronize()
        torch.cuda.synchronize(dev)
        ms_total = e0.elapsed_time(e1)
        clk = clocks.stop()
        launches = ctx.launch_count() - launches0
        _barrier(dist)
        ms_total = _max_over_ranks(dist, ms_total, dev)
        ms_step = ms_total / args.steps
        dofs = 3 * ctx.V[L]
        value = dofs * world / (ms_step * 1e-3)

        # per-launch timing of the dominant (finest-level stencil) kernels
        ctx.profile_fine(True)
        for _ in range(min(args.steps, 500)):
            ctx.vcycle(r, z)
        k_ms, k_bytes, k_launches = ctx.profile_fine(False)
        achieved = k_bytes / (k_ms * 1e-3) / 1e9
        peaks = _peaks()
        peak = peaks.get("hbm_gbs", 6800.0)

        # end to end through the API with host buffers: every step copies its
        # residual in from pinned host memory and its result back out.  Steps
        # are pipelined: two device buffer pairs, one copy stream per
        # direction, so step i's copies overlap the cycles of steps i -+ 1
        r_h = r.cpu().pin_memory()
        z_h = torch.empty_like(r_h).pin_memory()
        r_d = [torch.empty_like(r) for _ in range(2)]
        z_d = [torch.empty_like(r) for _ in range(2)]
        h2d, d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        ev = lambda: [torch.cuda.Event() for _ in range(2)]
        in_ready, cycle_done, out_done = ev(), ev(), ev()

        def e2e_steps(k):
            start = torch.cuda.Event(enable_timing=True)
            start.record(stream)
            h2d.wait_event(start)
            for i in range(k):
                j = i % 2
                if i >= 2:
                    h2d.wait_event(cycle_done[j])  # r_d[j] consumed by step i-2
                with torch.cuda.stream(h2d):
                    r_d[j].copy_(r_h, non_blocking=True)
                in_ready[j].record(h2d)
                stream.wait_event(in_ready[j])
                if i >= 2:
                    stream.wait_event(out_done[j])  # z_d[j] read back by step i-2
                ctx.vcycle(r_d[j], z_d[j])
                cycle_done[j].record(stream)
                d2h.wait_event(cycle_done[j])
                with torch.cuda.stream(d2h):
                    z_h.copy_(z_d[j], non_blocking=True)
                out_done[j].record(d2h)
            stream.wait_event(out_done[(k - 1) % 2])
            end = torch.cuda.Event(enable_timing=True)
            end.record(stream)
            end.synchronize()
            return start.elapsed_time(end)

        e_steps = max(10, min(args.steps, 200))
        e2e_steps(4)
        e2e_ms = _max_over_ranks(dist, e2e_steps(e_steps) / e_steps, dev)
        e2e_value = dofs * world / (e2e_ms * 1e-3)

        # FP64 cycle beside it
        ctx64 = pkg.Context(N, L, pkg.FP64, device=dev, stream=stream)
        ctx64.prepare(eta, prm["nu"])
        for _ in range(3):
            ctx64.vcycle(r, z)
        k64 = max(5, min(args.steps // 20, 100))
        e0.record(stream)
        for _ in range(k64):
            ctx64.vcycle(r, z)
        e1.record(stream)
        e1.synchronize()
        fp64_ms = e0.elapsed_time(e1) / k64

        solve = None
        if not args.no_solve:
            solve = {}
            for name, prec in (("mixed", pkg.MIXED), ("fp64", pkg.FP64)):
                times = []
                for rep in range(3):
                    torch.cuda.synchronize(dev)
                    t0 = time.perf_counter()
                    c = pkg.Context(N, L, prec, device=dev, stream=stream)
                    c.prepare(eta, prm["nu"])
                    if prec == pkg.MIXED and not args.no_tune:
                        c.autotune(10, tune_cache)  # tile shapes read back from the cycle's tuning run
                    b = c.load_vector(fbar)
                    torch.cuda.synchronize(dev)
                    t1 = time.perf_counter()
                    x, its, rel = c.solve(b, 1e-8, 20000)
                    torch.cuda.synchronize(dev)
                    t2 = time.perf_counter()
                    times.append((t2 - t0, t1 - t0, t2 - t1, its, rel))
                    del c
                times.sort()
                tot, st, sv, its, rel = times[len(times) // 2]
                solve[name] = {"time_to_1e-8_s": tot, "setup_s": st, "solve_s": sv, "minres_iters": its,
                               "relres": rel}

    batch = run_batch(args, dev, stream) if args.batch else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, k, dt, cores = oracle_vcycle_rate(12.0)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{k} oracle V-cycles at 16^3 pressure cubes of the same 8-sphere field family "
                         f"({dt * 1e3:.0f} ms each; scipy CSR products on one thread)"}

    if rank == 0:
        flagged = [ctx.level_info(l).n_flag for l in range(1, L)]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": arm_config(N, L, flagged, world),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": FINE_STENCIL_DRAM_BYTES if N == 64 else None,
                         "traffic_unit": "DRAM bytes per finest-level stencil launch (ncu)",
                         "kernel": "finest-level stencil (Chebyshev/residual epilogues), FP32",
                         "launches_timed": k_launches, "peak_source": "measured hbm_gbs"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(r.numel() * 8),
                    "d2h_bytes_per_step": int(z.numel() * 8),
                    "pipeline": "2 buffer pairs; H2D and D2H streams overlap the neighbouring steps' cycles"},
            "gpu_launches": int(launches),
            "clocks": clk,
            "fp64_vcycle": {"value": dofs / (fp64_ms * 1e-3), "unit": UNIT, "ms_per_step": fp64_ms},
            "autotune": {"seconds": t_tune, "tiles": {f"L{l}m{m}": list(v) for (l, m), v in tuned.items()}},
            "solve": solve,
            "batch": batch,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
