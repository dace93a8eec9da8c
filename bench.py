"""Benchmark: fine-level velocity DoF/s per AGCA V-cycle and Stokes solve time
to a 1e-8 relative residual, on synthetic sinker problems.

Workload (default): the mixed-precision-at-scale configuration: 128^3
pressure cubes (256^3 velocity cubes, 50,923,779 velocity DoF, 2,146,689
pressure DoF, 7 levels), log10 viscosity = sum of 20 seeded Gaussian bumps
(amplitudes in [-3, 3], widths in [0.03, 0.15]) clipped to [-3, 3], forcing
f_z = -(log10 mu + 3)/6, AGCA threshold nu = 10.

A step is one V(2,2) cycle of the FP64 AGCA preconditioner on a residual
resident in HBM (`value`, dtype f64: the paper's precision).  Beside it, on
the same field: the mixed-precision cycle (FP32 smoothing, transfers and
coarse applies), setup + MINRES time to 1e-8 for the FP64 and mixed solvers,
AGCA (nu = 10) against pure DCA (no flagged element) on the 8-sphere 64^3
field with jump 1e6, the 24-problem batch (uneven 32^3/48^3/64^3 single
sinkers, batched against one by one), and the CPU oracle on the host cores.

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
NU = 10.0
NU_DCA = 1e300  # no element's max/min viscosity ratio reaches it: pure DCA on every coarse level

# FP64 arithmetic peak from the unit counts and clock: 152 SMs x 2 FP64
# fused multiply-adds per SM and clock x 2 flops x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per finest-level
# stencil launch, mean over the four launches of one V-cycle, from one ncu
# capture of the current kernels at 64^3 pressure cubes scaled by the vertex
# count (x 7.907) to 128^3 (None where no capture of the current kernel exists)
FINE_STENCIL_DRAM_BYTES = {("logbump", 128, "f64"): 5.298e9, ("logbump", 128, "f32"): 1.059e9}


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
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
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


def bench_levels(N):
    """Levels of the benchmark hierarchy: coarsen the 2N velocity grid while
    it stays even with >= 4 cubes (the library's default)."""
    n, L = 2 * N, 1
    while n % 2 == 0 and n // 2 >= 4:
        n //= 2
        L += 1
    return L


def workload_name(field, N, L):
    if field == "logbump":
        return (f"20 Gaussian log10-viscosity bumps clipped to [1e-3, 1e3], {N}^3 pressure cubes "
                f"({3 * (2 * N + 1) ** 3:,} velocity DoF, {L} levels), AGCA nu 10, V(2,2) cycle")
    return (f"8 tanh spheres r 0.08 w 0.01 jump 1e6, {N}^3 pressure cubes "
            f"({3 * (2 * N + 1) ** 3:,} velocity DoF, {L} levels), AGCA nu 10, V(2,2) cycle")


def arm_config(field, N, L, flagged, world):
    return {"workload": workload_name(field, N, L), "field": field,
            "N_pressure": N, "velocity_cubes": 2 * N, "levels": L, "velocity_dofs": 3 * (2 * N + 1) ** 3,
            "pressure_dofs": (N + 1) ** 3, "flagged_per_level": flagged, "global_batch": world, "seq_len": None,
            "parallelism": f"replicas{world}",
            "l2": "inputs larger than L2 (one FP64 velocity vector is "
                  f"{3 * (2 * N + 1) ** 3 * 8 / 1e6:.0f} MB > 129 MB), no flush"}


def make_field(field, N, dev):
    """(eta (E,), fbar (3E,)) on the device."""
    if field == "logbump":
        from synth import gaussian_logbumps_on_device

        eta, fbar = gaussian_logbumps_on_device(N, device=dev)
    else:
        from synth import sphere_sinkers_on_device

        eta, fbar, _ = sphere_sinkers_on_device(N, 8, 0.08, 0.01, 1e6, device=dev)
    return eta, fbar.reshape(-1)


def host_field(field, N):
    from synth import gaussian_logbumps, sphere_sinkers

    return gaussian_logbumps(N) if field == "logbump" else sphere_sinkers(N, 8, 0.08, 0.01, 1e6)


# ------------------------------------------------------------------ CPU oracle
def oracle_timings(field, seconds=10.0, N=16, solve=True):
    """The oracle as it stands, on the host cores: DoF/s of its V-cycle on the
    workload's field family at a size it handles in seconds, and its MINRES
    solve to 1e-8 at the same size.  scipy's CSR products run on one thread."""
    from oracle import agca as oagca
    from oracle import stokes as ostokes
    from synth import random_vector

    p = host_field(field, N)
    L = bench_levels(N)
    t0 = time.perf_counter()
    H = oagca.Hierarchy(N, L, p.eta, NU)
    setup_s = time.perf_counter() - t0
    n = 3 * H.mesh[L].nv
    r = random_vector(n, 3) * H.mask[L]
    H.vcycle(r)
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < seconds:
        H.vcycle(r)
        k += 1
    dt = (time.perf_counter() - t0) / k
    out = {"N": N, "levels": L, "vcycles": k, "vcycle_ms": dt * 1e3, "vcycle_dofs_per_s": n / dt,
           "setup_s": setup_s}
    if solve:
        S = ostokes.Stokes(H)
        b = S.rhs(p.fbar)
        t0 = time.perf_counter()
        x, its = S.minres(b, 1e-8, 20000)
        out["solve_s"] = time.perf_counter() - t0
        out["minres_iters"] = its
        out["relres"] = float(np.linalg.norm(b - S.K(x)) / np.linalg.norm(b))
    return out


def _cores():
    try:
        import threadpoolctl

        info = threadpoolctl.threadpool_info()
        blas = max((i.get("num_threads", 1) for i in info), default=1)
    except Exception:  # noqa: BLE001
        blas = None
    return os.cpu_count(), blas


def run_reference(args):
    """--impl reference: the oracle as it stands, timed on the host cores.
    Each step is one oracle V-cycle of the workload's field family at 16^3
    pressure cubes (a bounded sample: the oracle's sparse matrices of the
    128^3 hierarchy take tens of GB and minutes per cycle); the config names
    the size actually timed."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import agca as oagca
    from synth import random_vector

    N = 16
    L = bench_levels(N)
    p = host_field(args.field, N)
    H = oagca.Hierarchy(N, L, p.eta, NU)
    n = 3 * H.mesh[L].nv
    r = random_vector(n, 3) * H.mask[L]
    for _ in range(args.warmup):
        H.vcycle(r)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        H.vcycle(r)
    dt = (time.perf_counter() - t0) / args.steps
    value = n / dt
    ncpu, blas = _cores()
    cfg = arm_config(args.field, N, L, [int(H.flags[l].sum()) for l in range(1, L)], 1)
    cfg["sample_of"] = workload_name(args.field, args.N, bench_levels(args.N))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "host_cpu_count": ncpu,
                             "blas_threads": blas, "kind": "oracle",
                             "sample": f"{args.steps} oracle V-cycles at {N}^3 pressure cubes of the same field "
                                       f"family ({dt * 1e3:.0f} ms each; scipy CSR products on one thread)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU parts
def time_cycles(ctx, r, z, steps, stream, nvtx=None):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if nvtx:
        torch.cuda.nvtx.range_push(nvtx)
    e0.record(stream)
    for _ in range(steps):
        ctx.vcycle(r, z)
    e1.record(stream)
    if nvtx:
        torch.cuda.nvtx.range_pop()
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def fine_profile(ctx, r, z, reps):
    """Per-launch CUDA-event times of the finest-level stencil launches over
    reps cycles: (mean ms per launch, algorithmic bytes and flops per launch)."""
    ctx.profile_fine(True)
    for _ in range(reps):
        ctx.vcycle(r, z)
    ms, by, fl, n = ctx.profile_fine(False)
    return ms / n, by / n, fl / n, n


def e2e_rate(ctx, r, dofs, steps, stream, dev):
    """The same cycle through the API with host buffers: every step copies its
    residual in from pinned host memory and its result back out.  Steps are
    pipelined: two device buffer pairs, one copy stream per direction, so
    step i's copies overlap the cycles of steps i -+ 1."""
    r_h = r.cpu().pin_memory()
    z_h = torch.empty_like(r_h).pin_memory()
    r_d = [torch.empty_like(r) for _ in range(2)]
    z_d = [torch.empty_like(r) for _ in range(2)]
    h2d, d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev = lambda: [torch.cuda.Event() for _ in range(2)]  # noqa: E731
    in_ready, cycle_done, out_done = ev(), ev(), ev()

    def run(k):
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

    run(3)
    ms = run(steps) / steps
    return dofs / (ms * 1e-3), ms, int(r.numel() * 8)


def timed_solve(pkg, N, L, prec, eta, fbar, nu, dev, stream, maxit, tune_cache=None):
    """Setup (flags, Galerkin, diagonals, lambda, coarsest factor) + MINRES to
    1e-8 from x = 0, wall clock with the device synchronised on both sides."""
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    c = pkg.Context(N, L, prec, device=dev, stream=stream)
    c.prepare(eta, nu)
    if tune_cache is not None:
        c.autotune(10, tune_cache)  # tile shapes read back from the cycle's tuning run
    b = c.load_vector(fbar)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    try:
        x, its, rel = c.solve(b, 1e-8, maxit)
        conv = True
    except pkg.AgcaError as e:  # stopped at the iteration limit above the tolerance
        if e.status != 4:
            raise
        x, its, rel, conv = None, maxit, float("nan"), False
    torch.cuda.synchronize(dev)
    t2 = time.perf_counter()
    nflag = [c.level_info(l).n_flag for l in range(1, L)]
    del c
    return {"time_to_1e-8_s": t2 - t0, "setup_s": t1 - t0, "solve_s": t2 - t1, "minres_iters": its,
            "relres": rel, "converged": conv, "flagged_per_level": nflag}, x


def solves(pkg, N, L, eta, fbar, dev, stream, tune64, tune32, reps_mixed=3):
    out = {}
    res, x64 = timed_solve(pkg, N, L, pkg.FP64, eta, fbar, NU, dev, stream, 20000, tune64)
    out["fp64"] = res
    runs = []
    xm = None
    for _ in range(reps_mixed):
        res, xm = timed_solve(pkg, N, L, pkg.MIXED, eta, fbar, NU, dev, stream, 20000, tune32)
        runs.append(res)
    runs.sort(key=lambda d: d["time_to_1e-8_s"])
    out["mixed"] = dict(runs[len(runs) // 2], repetitions=reps_mixed)
    out["fp64"]["repetitions"] = 1
    if x64 is not None and xm is not None:
        # both solutions reach the 1e-8 residual: their difference bounds the
        # mixed solution's error against the FP64 one at that tolerance
        out["mixed_vs_fp64_rel_diff"] = float(torch.linalg.vector_norm(xm - x64) / torch.linalg.vector_norm(x64))
    return out


def agca_vs_dca(pkg, dev, stream):
    """AGCA (nu = 10) against pure DCA on the 8-sphere 64^3 field with jump
    1e6 (Sec. 4.2: DCA loses robustness at unaligned jumps): mixed solves to
    1e-8, iterations and time, same field and forcing."""
    N = 64
    L = bench_levels(N)
    eta, fbar = make_field("spheres", N, dev)
    out = {"workload": workload_name("spheres", N, L) + ", mixed solve to 1e-8"}
    for name, nu, maxit in (("agca_nu10", NU, 20000), ("dca", NU_DCA, 20000)):
        res, _ = timed_solve(pkg, N, L, pkg.MIXED, eta, fbar, nu, dev, stream, maxit)
        out[name] = res
    # the paper's outer solver on the same field: FGMRES + block-triangular + BFBT
    c = pkg.Context(N, L, pkg.MIXED, device=dev, stream=stream)
    c.prepare(eta, NU)
    b = c.load_vector(fbar)
    # restart length and CG steps per Z solve: restarted at 50 the Krylov
    # space is lost before this field converges; GB300's memory holds 300
    # Krylov pairs (32 GB at 64^3)
    for restart, zi in ((50, 30), (300, 100)):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        try:
            _, its, rel = c.solve_fgmres(b, 1e-8, 600, restart, "bfbt", zi)
        except pkg.AgcaError as e:
            if e.status != 4:
                raise
            its, rel = 600, float("nan")
        torch.cuda.synchronize(dev)
        out[f"agca_nu10_fgmres{restart}_bfbt_zcg{zi}"] = {"iters": its, "relres": rel,
                                                          "solve_s": time.perf_counter() - t0}
    del c
    return out


def coefficient_study(pkg, dev, stream, N=32):
    """The axes of the paper's convergence study (Sec. 4, Figs. 7-9) at
    32^3 pressure cubes, mixed solves to 1e-8:
    * coefficient approximations (Sec. 3.2) on the unaligned cube eta_2 with
      DR 1e6: the finest coefficient by the 4-point rule (analytic) or as
      the mean of the P1 interpolant, the coarse DCA coefficient analytic on
      the coarse elements, P1 on the coarse grid, or the arithmetic /
      harmonic / geometric projection of the children; each with pure DCA
      and with AGCA at nu = 10;
    * the threshold nu on the tanh cube eta_3 (omega 10, DR 1e6, Fig. 9):
      flagged elements, stored Galerkin bytes and iterations."""
    from synth import cube_field, field_problem, level_coefficients, p1_element_means

    L = bench_levels(N)

    def run(eta, fbar, nu, proj=0, lc=None):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        c = pkg.Context(N, L, pkg.MIXED, device=dev, stream=stream)
        c.set_viscosity(eta)
        c.set_coarse_projection(proj)
        gbytes = c.flag(nu)
        for l, v in (lc or {}).items():
            c.set_level_coefficient(l, torch.from_numpy(v).to(dev))
        c.setup()
        b = c.load_vector(fbar)
        try:
            _, its, rel = c.solve(b, 1e-8, 20000)
        except pkg.AgcaError as e:
            if e.status != 4:
                raise
            its, rel = 20000, float("nan")
        torch.cuda.synchronize(dev)
        out = {"minres_iters": its, "relres": rel, "time_to_1e-8_s": time.perf_counter() - t0,
               "flagged": int(sum(c.level_info(l).n_flag for l in range(1, L))), "galerkin_store_bytes": gbytes}
        del c
        return out

    out = {"N_pressure": N, "levels": L}
    fn2 = cube_field("unaligned", 1e6)
    p2 = field_problem(N, fn2)
    fbar2 = torch.from_numpy(p2.fbar.ravel()).to(dev)
    eta_q = torch.from_numpy(p2.eta).to(dev)
    eta_p1 = torch.from_numpy(p1_element_means(2 * N, fn2)).to(dev)
    variants = {"analytic": (eta_q, 0, level_coefficients(fn2, N, L, "analytic")),
                "p1": (eta_p1, 0, level_coefficients(fn2, N, L, "p1")),
                "arithmetic": (eta_q, 0, None), "harmonic": (eta_q, 1, None), "geometric": (eta_q, 2, None)}
    approx = {}
    for name, (eta, proj, lc) in variants.items():
        approx[name] = {"dca": run(eta, fbar2, NU_DCA, proj, lc), "agca_nu10": run(eta, fbar2, NU, proj, lc)}
    out["approximations_unaligned_cube_dr1e6"] = approx
    fn3 = cube_field("tanh", 1e6, omega=10.0)
    p3 = field_problem(N, fn3)
    eta3 = torch.from_numpy(p3.eta).to(dev)
    fbar3 = torch.from_numpy(p3.fbar.ravel()).to(dev)
    out["nu_sweep_tanh_cube_omega10_dr1e6"] = {f"{nu:g}": run(eta3, fbar3, nu) for nu in (1.5, 3.0, 10.0, 100.0,
                                                                                         1e4, NU_DCA)}
    # the paper's outer solver (Sec. 4) against MINRES on the unaligned cube,
    # AGCA with the analytic coarse coefficient (where DCA fails)
    lc = level_coefficients(fn2, N, L, "analytic")
    c = pkg.Context(N, L, pkg.MIXED, device=dev, stream=stream)
    c.set_viscosity(eta_q)
    c.flag(NU)
    for l, v in lc.items():
        c.set_level_coefficient(l, torch.from_numpy(v).to(dev))
    c.setup()
    b = c.load_vector(fbar2)
    solvers = {}
    for name, call in (("minres_blockdiag_mass", lambda: c.solve(b, 1e-8, 20000)),
                       ("fgmres_blocktri_mass_restart50", lambda: c.solve_fgmres(b, 1e-8, 20000, 50, "mass")),
                       ("fgmres_blocktri_bfbt_restart50_zcg10", lambda: c.solve_fgmres(b, 1e-8, 20000, 50, "bfbt", 10)),
                       ("fgmres_blocktri_bfbt_restart50_zcg40", lambda: c.solve_fgmres(b, 1e-8, 20000, 50, "bfbt", 40))):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        try:
            _, its, rel = call()
        except pkg.AgcaError as e:
            if e.status != 4:
                raise
            its, rel = 20000, float("nan")
        torch.cuda.synchronize(dev)
        solvers[name] = {"iters": its, "relres": rel, "solve_s": time.perf_counter() - t0}
    out["outer_solvers_unaligned_cube_dr1e6_analytic_agca"] = solvers
    del c
    return out


def run_batch(args, dev, stream):
    """The 24-problem batch (uneven 32^3/48^3/64^3 single sinkers): batched
    V-cycle throughput against the same problems cycled one by one, and
    batched solve time to 1e-8 against sequential solves."""
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
        b.prepare(etas, NU)
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
            c.prepare(eta, NU)
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
            try:
                xs, its, rel = b.solve(bs, 1e-8, 40000)
                out["batched_iters"] = its
                out["batched_max_relres"] = max(rel)
            except pkg.AgcaError as e:  # some problem stopped above the tolerance
                if e.status != 4:
                    raise
                out["batched_not_converged"] = True
            stream.synchronize()
            out["batched_solve_s"] = time.perf_counter() - t0

            def one_by_one(contexts):
                """Sequential solves; the problems that stop above the tolerance are listed."""
                failed, iters = [], []
                t0 = time.perf_counter()
                for i, (c, bb) in enumerate(zip(contexts, bs)):
                    c = c() if callable(c) else c
                    try:
                        iters.append(c.solve(bb, 1e-8, 40000)[1])
                    except pkg.AgcaError as e:
                        if e.status != 4:
                            raise
                        failed.append(i)
                        iters.append(None)
                    del c
                stream.synchronize()
                return time.perf_counter() - t0, iters, failed

            t, iters, failed = one_by_one(singles)
            out["sequential_mixed_solve_s"], out["sequential_mixed_iters"] = t, iters
            if failed:
                out["sequential_mixed_not_converged"] = failed

            # the plain FP64 form of the same problems, one by one
            def fp64_context(p, eta):
                def make():
                    c = pkg.Context(p.N, pkg.default_levels(p.N), pkg.FP64, device=dev, stream=stream)
                    c.prepare(eta, NU)
                    return c
                return make

            t, iters, failed = one_by_one([fp64_context(p, eta) for p, eta in zip(probs, etas)])
            out["sequential_fp64_solve_s"], out["sequential_fp64_iters"] = t, iters
            if failed:
                out["sequential_fp64_not_converged"] = failed
        del singles, b
    return out


def batch_cycles():
    """The batch workload's mixed V-cycle batched and one problem at a time,
    each once inside its own NVTX range (for a launch-list capture) and then
    timed over 10 cycles with CUDA events; prints one JSON line."""
    import __graft_entry__

    __graft_entry__.build()
    import paper_2511_13109_gb300 as pkg
    from synth import batch_problems

    dev = torch.device("cuda", 0)
    probs = batch_problems(device=dev)
    etas = [torch.from_numpy(p.eta).to(dev) for p in probs]
    s = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(s):
        b = pkg.Batch([p.N for p in probs], pkg.MIXED, device=dev, stream=s)
        b.prepare(etas, NU)
        rs = [torch.rand(3 * c.V[c.L], dtype=torch.float64, device=dev) * 2 - 1 for c in b.contexts]
        singles = []
        for p, eta in zip(probs, etas):
            c = pkg.Context(p.N, pkg.default_levels(p.N), pkg.MIXED, device=dev, stream=s)
            c.prepare(eta, NU)
            singles.append(c)
        for _ in range(3):
            b.vcycle(rs)
            for c, r in zip(singles, rs):
                c.vcycle(r)
        s.synchronize()
        for name, run in (("batched", lambda: b.vcycle(rs)),
                          ("single", lambda: [c.vcycle(r) for c, r in zip(singles, rs)])):
            torch.cuda.nvtx.range_push(name)
            run()
            s.synchronize()
            torch.cuda.nvtx.range_pop()
        out = {}
        for name, run in (("batched_ms", lambda: b.vcycle(rs)),
                          ("one_by_one_ms", lambda: [c.vcycle(r) for c, r in zip(singles, rs)])):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(10):
                run()
            e1.record(s)
            e1.synchronize()
            out[name] = e0.elapsed_time(e1) / 10
    print(json.dumps({"batch_cycles": out, "problems": len(probs)}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--field", default="logbump", choices=["logbump", "spheres"])
    ap.add_argument("--mixed-steps", type=int, default=200, help="timed mixed-precision cycles")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-dca", action="store_true")
    ap.add_argument("--no-study", action="store_true", help="skip the coefficient / nu study at 32^3")
    ap.add_argument("--batch-n", type=int, default=0)
    ap.add_argument("--cycles-only", action="store_true",
                    help="profiling aid: warm-up and timed cycles of both precisions only, one short JSON line")
    ap.add_argument("--batch-cycles", action="store_true",
                    help="profiling aid: one batched mixed V-cycle of the 24-problem batch (NVTX range "
                         "'batched') and the same cycles one by one (range 'single'), then both timed")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.batch_cycles:
        return batch_cycles()

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = _init_pg(world, "nccl")

    import __graft_entry__

    __graft_entry__.build()
    import paper_2511_13109_gb300 as pkg

    N = args.N
    L = pkg.default_levels(N)
    eta, fbar = make_field(args.field, N, dev)
    stream = torch.cuda.Stream(device=dev)
    tune_dir = tempfile.mkdtemp(prefix="agca_bench_")
    with torch.cuda.stream(stream):
        ctx = pkg.Context(N, L, pkg.FP64, device=dev, stream=stream)
        ctx.prepare(eta, NU)
        t_tune = time.perf_counter()
        tune64 = os.path.join(tune_dir, "tiles64.txt")
        tuned = ctx.autotune(reps=5, cache=tune64) if not args.no_tune else {}
        t_tune = time.perf_counter() - t_tune
        dofs = 3 * ctx.V[L]
        g = torch.Generator(device=dev)
        g.manual_seed(1234 + rank)
        r = torch.rand(dofs, dtype=torch.float64, device=dev, generator=g) * 2 - 1
        z = torch.empty_like(r)

        # ---- the timed region: K FP64 V(2,2) cycles
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
        value = dofs * world / (ms_step * 1e-3)

        # ---- the mixed-precision cycle on the same field
        ctxm = pkg.Context(N, L, pkg.MIXED, device=dev, stream=stream)
        ctxm.prepare(eta, NU)
        tune32 = os.path.join(tune_dir, "tiles32.txt")
        tunedm = ctxm.autotune(reps=10, cache=tune32) if not args.no_tune else {}
        for _ in range(max(3, args.warmup)):
            ctxm.vcycle(r, z)
        mixed_ms = time_cycles(ctxm, r, z, args.mixed_steps, stream, nvtx="mixed")
        if args.cycles_only:
            if rank == 0:
                print(json.dumps({"fp64_ms": ms_step, "mixed_ms": mixed_ms}), flush=True)
            return 0

        # ---- dominant kernels: per-launch CUDA-event times of the finest stencils
        k64_ms, k64_bytes, k64_flops, k64_n = fine_profile(ctx, r, z, min(max(args.steps, 5), 50))
        k32_ms, k32_bytes, _, k32_n = fine_profile(ctxm, r, z, 200)
        peaks = _peaks()
        hbm_peak = peaks.get("hbm_gbs")
        hbm_src = "measured hbm_gbs (MEASURED_PEAKS.json)" if hbm_peak else "fallback 6800 GB/s"
        hbm_peak = hbm_peak or 6800.0

        # ---- end to end through the API with host buffers
        e_steps = max(5, min(args.steps, 50))
        e2e_value, e2e_ms, nbytes = e2e_rate(ctx, r, dofs, e_steps, stream, dev)
        e2e_value = dofs * world / (_max_over_ranks(dist, e2e_ms, dev) * 1e-3)

        solve = None
        if not args.no_solve:
            solve = solves(pkg, N, L, eta, fbar, dev, stream, None if args.no_tune else tune64,
                           None if args.no_tune else tune32)
        flagged = [ctx.level_info(l).n_flag for l in range(1, L)]
        del ctxm

    dca = None
    if not args.no_solve and not args.no_dca:
        dca = agca_vs_dca(pkg, dev, stream)
    batch = run_batch(args, dev, stream) if not args.no_batch else None
    study = coefficient_study(pkg, dev, stream) if not (args.no_solve or args.no_study) else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        o = oracle_timings(args.field, 10.0, 16, solve=not args.no_solve)
        ncpu, blas = _cores()
        cpu = {"value": o["vcycle_dofs_per_s"], "unit": UNIT, "cores": 1, "host_cpu_count": ncpu,
               "blas_threads": blas, "kind": "oracle",
               "sample": f"{o['vcycles']} oracle V-cycles at 16^3 pressure cubes of the same field family "
                         f"({o['vcycle_ms']:.0f} ms each; scipy CSR products on one thread)",
               "oracle_16cubed": o}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": arm_config(args.field, N, L, flagged, world),
            "roofline": {"bound": "alu", "achieved": k64_flops / (k64_ms * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": k64_flops / (k64_ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                         "traffic": FINE_STENCIL_DRAM_BYTES.get((args.field, N, "f64")),
                         "kernel": "finest-level FP64 stencil (Chebyshev/residual epilogues)",
                         "launch_ms": k64_ms, "algorithmic_flops_per_launch": k64_flops,
                         "algorithmic_bytes_per_launch": k64_bytes,
                         "hbm_frac_of_measured": k64_bytes / (k64_ms * 1e-3) / 1e9 / hbm_peak,
                         "launches_timed": k64_n,
                         "peak_source": "FP64 FMA rate from unit counts and clock (152 SMs x 2/clk x 2 flops x "
                                        "2.07 GHz); flops count a fused multiply-add as 2"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                    "pipeline": "2 buffer pairs; H2D and D2H streams overlap the neighbouring steps' cycles"},
            "gpu_launches": int(launches),
            "clocks": clk,
            "mixed_vcycle": {
                "value": dofs / (mixed_ms * 1e-3), "unit": UNIT, "ms_per_step": mixed_ms, "steps": args.mixed_steps,
                "dtype": "f32 cycle (FP64 input and output)",
                "roofline": {"bound": "hbm", "achieved": k32_bytes / (k32_ms * 1e-3) / 1e9, "peak": hbm_peak,
                             "unit": "GB/s", "frac": k32_bytes / (k32_ms * 1e-3) / 1e9 / hbm_peak,
                             "traffic": FINE_STENCIL_DRAM_BYTES.get((args.field, N, "f32")),
                             "kernel": "finest-level FP32 stencil (Chebyshev/residual epilogues)",
                             "launch_ms": k32_ms, "algorithmic_bytes_per_launch": k32_bytes,
                             "launches_timed": k32_n, "peak_source": hbm_src}},
            "autotune": {"seconds": t_tune, "fp64": {f"L{l}m{m}": list(v) for (l, m), v in tuned.items()},
                         "mixed": {f"L{l}m{m}": list(v) for (l, m), v in tunedm.items()}},
            "solve": solve,
            "agca_vs_dca": dca,
            "coefficient_study": study,
            "batch": batch,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
