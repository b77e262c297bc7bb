#!/usr/bin/env python
"""Benchmark of the GB300 SEM pressure-Poisson solve.

One step = one full pressure-type Poisson solve from a zero guess: the whole
hot path (operator, gather-scatter, masking, Chebyshev-Jacobi smoothing in
FP32, tensor-product transfers, FP64 coarse solve, FP64 flexible CG with its
inner products) on the mixed-precision workload

    box of 48^3 = 110,592 trilinear hexahedra, N = 7, vertices jittered
    +-10% of h (seed 3), Neumann, smooth random mean-free right-hand side,
    p-multigrid 7-3-1, Chebyshev(3)-Jacobi smoother in FP32, FP64 coarse
    solve (CG preconditioned by a lattice multigrid V-cycle), FlexCG in FP64
    to a relative residual of 1e-8.

value = unique dofs solved per second (GDOF/s, whole job over all ranks).
The working set (about 6 GB) is far larger than the 129 MB L2, so no L2 flush
is needed between steps.  Besides the headline line the JSON carries the
dominant kernel's roofline (measured live with CUDA events on the launching
stream inside the timed region), an end-to-end number through the host-buffer
entry point, the CPU oracle's throughput on a bounded sample, the FP64/FP32
operator throughput at 64^3 elements (HBM roofline), SM clocks sampled during
the timed region and the number of library kernels launched.

--impl reference times the CPU oracle (the only reference there is) on a
bounded sample of the same workload.  With torchrun, every rank runs an
independent replica (the solve is not sharded: replicas only).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Poisson solve time to 1e-8 (GDOF/s) & Ax GB/s vs HBM roofline; p50/p99 latency"
E_SIDE, ORDER, MESH_SEED, RHS_SEED = 48, 7, 3, 3
TOL = 1e-8
CHEB_DEGREE, COARSE_TOL, COARSE_MAXIT, COARSE_MODE = 3, 2e-1, 30, 1
# pMG schedule of the headline: 7-4-2-1 (7 outer iterations) measured faster
# than the halving schedule 7-3-1 (9 iterations); the named configuration
# (7-3-1, Chebyshev degree 2) is measured in the same run ("named_config")
ORDERS = "7,4,2,1"
SMOOTHER = "f32"
SMOOTHER_DTYPES = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}  # sem_dtype values
WORKLOAD = ("mixed-precision Neumann pressure solve: E=48^3=110592 jittered hexes (+-10% h, "
            "seed 3), N=7, pMG 7-4-2-1, Chebyshev(3)-Jacobi smoother in FP32, FP64 coarse solve "
            "(CG + FP32 lattice multigrid V(2,2), tol 2e-1, <=30 it), FP64 FlexCG to 1e-8 "
            "from x=0")
# Fallback peaks of the recipe, used only when MEASURED_PEAKS.json is absent.
FALLBACK_HBM_GBS = 6800.0
# FP64 pipe: 152 SMs x 2 FP64 FMA per clock x 2 flop x 2.07 GHz (the part's
# nominal 1.25 TFLOP/s; an FMA-chain probe on a GB300 measured 1.195).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# The FP64 operator runs in FP32-pair arithmetic: one FP64-equivalent FMA
# costs 12 FP32-pipe instructions, so its ALU roof is the FP32 issue rate
# (152 SMs x 128 lanes x 2.07 GHz) / 12 x 2 flop.
PAIR_INSTR_PER_FMA = 12
PAIR_PEAK_TFLOPS = 152 * 128 * 2.07e9 / PAIR_INSTR_PER_FMA * 2 / 1e12
# DRAM traffic of one fine-level FP64 operator launch per local point (the
# form with the inner product folded in, as in the solve), from an ncu capture
# of that kernel on a 24^3 case, valid while the kernel source is unchanged.
AX_TRAFFIC = {"source_sha256": "2c501da0dc26ea66228f2a74a4e74d7a574e1eeb4a3a83b57351d3f2e2c2f52b",
              "bytes_per_point": 63.72}
# The same for the smoother's assembled FP32 operator, per factor storage
# (ncu capture on a 32^3 case), valid while ax32.cu is unchanged.
AX32_TRAFFIC = {"f32": {"source_sha256": "a797ec83846c77963b93140f5d48cb141371698a98aac0655e34ba1e0aeb1190",
                        "bytes_per_point": 31.26},
                "f16": {"source_sha256": "a797ec83846c77963b93140f5d48cb141371698a98aac0655e34ba1e0aeb1190",
                        "bytes_per_point": 18.63}}


def parse_args():
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=15)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--side", type=int, default=E_SIDE, help="elements per direction")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the operator sweep, e2e and CPU-baseline legs")
    p.add_argument("--no-serve", action="store_true",
                   help="skip the batched (config 4) and serving (config 5) legs")
    p.add_argument("--host-loop", action="store_true",
                   help="time FlexCG's host-driven loop instead of the CUDA-graph loop")
    p.add_argument("--breakdown", action="store_true",
                   help="after the timed region, time every kernel class of one more solve")
    p.add_argument("--coarse-maxit", type=int, default=COARSE_MAXIT)
    p.add_argument("--coarse-tol", type=float, default=COARSE_TOL)
    p.add_argument("--cheb-degree", type=int, default=CHEB_DEGREE)
    p.add_argument("--ax-only", type=int, default=0, metavar="SIDE",
                   help="profiling aid: build a SIDE^3 mesh of the workload's recipe, apply "
                        "the assembled FP32 operator twice with FP32 and with FP16 factors, exit")
    p.add_argument("--ax-order", type=int, default=ORDER,
                   help="order N of the --ax-only mesh")
    p.add_argument("--solver", default="flexcg", choices=["flexcg", "fgmres"],
                   help="outer FP64 solver (FGMRES: flexible GMRES, classical Gram-Schmidt)")
    p.add_argument("--restart", type=int, default=20, help="FGMRES vectors per cycle")
    p.add_argument("--schwarz", action="store_true",
                   help="Chebyshev-accelerated overlapping Schwarz smoother (FDM local solves) "
                        "instead of Chebyshev-Jacobi")
    p.add_argument("--orders", default=ORDERS,
                   help="pMG schedule, fine to coarse (the fine order first)")
    p.add_argument("--schwarz-tf32", action="store_true",
                   help="Chebyshev-Schwarz smoothing with TF32 local solves on the tensor cores")
    p.add_argument("--schwarz-tc", action="store_true",
                   help="Chebyshev-Schwarz smoothing with the local solves on the tensor cores")
    p.add_argument("--smoother", default=SMOOTHER, choices=["f64", "f32", "f16", "bf16"],
                   help="arithmetic/storage of the smoothed pMG levels")
    p.add_argument("--coarse-mode", type=int, default=COARSE_MODE,
                   help="0: Jacobi-PCG, 1: multigrid-preconditioned CG on the N=1 lattice")
    return p.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def job_time_ms(pg, local_ms, device):
    """Wall time of the whole job: the slowest rank's time (all-reduce MAX
    over the process group; the local time when there is none)."""
    if pg is None:
        return float(local_ms)
    import torch

    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_value(world, units_per_rank, ms_per_step):
    """Whole-job throughput in G units per second: every rank solves its own
    replica (weak scaling), so the job processes world x units per step."""
    return world * units_per_rank / (ms_per_step / 1e3) / 1e9


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rhs_on_device(sem, torch, mesh, dev, step=None):
    """Neumann right-hand side b = gs(B f) minus its unique-dof mean, with f the
    seeded smooth random field of the input module, evaluated on the mesh's own
    GLL coordinates.  With step = n: the n-th member of the smooth sequence of
    inputs.fourier_sequence (successive solves)."""
    from paper_2110_01716_gb300 import inputs

    n = mesh.n_local
    X = [torch.empty(n, device=dev, dtype=torch.float64) for _ in range(3)]
    for d in range(3):
        sem.sem_mesh_field(mesh, d, X[d])
    Bm = torch.empty(n, device=dev, dtype=torch.float64)
    sem.sem_mesh_field(mesh, sem.SEM_FIELD_MASS, Bm)
    if step is None:
        a, k, phi = inputs.fourier_modes(RHS_SEED)
        om = [0.0] * len(a)
        step = 0
    else:
        a, k, phi, om = inputs.fourier_sequence(RHS_SEED)
    f = torch.zeros(n, device=dev, dtype=torch.float64)
    for m in range(len(a)):
        f += float(a[m]) * torch.cos(2 * torch.pi * (float(k[m, 0]) * X[0] + float(k[m, 1]) * X[1]
                                                     + float(k[m, 2]) * X[2]) + float(phi[m])
                                     + float(om[m]) * step)
    b = Bm * f
    sem.sem_gs(mesh, sem.SEM_F64, b)
    ones = torch.ones_like(b)
    mean = sem.sem_dot(mesh, b, ones) / mesh.n_global
    b -= mean
    del X, Bm, f, ones
    return b


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def source_sha(*names):
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2110_01716_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def traced_ms(sem, fn, reps=10, warm=3):
    """Device time of one call of fn: the sum of the library's own per-launch
    CUDA-event timings (each kernel launch bracketed on its stream), median
    over reps calls.  Host-side work inside a call (the staged operator's
    read of its wait flag) is not counted."""
    for _ in range(warm):
        fn()
    sem.sem_trace_enable(True, "*")
    sem.sem_trace_read(reset=True)
    per = []
    for _ in range(reps):
        fn()
        tr = sem.sem_trace_read(reset=True)
        per.append(sum(v["total_ms"] for v in tr.values()))
    sem.sem_trace_enable(False, "")
    return statistics.median(per)


def operator_sweep(sem, torch, dev, hbm):
    """FP64 / FP32 operator throughput at 64^3 elements, N=7 (stored and
    recomputed geometry), median of 20 launches after 3 warm-ups, timed by
    the library's per-launch events."""
    from paper_2110_01716_gb300 import inputs

    out = {}
    k = 64
    N = ORDER
    for geom, gname, arith in ((sem.SEM_GEOM_STORED, "stored", sem.SEM_ARITH_PAIR),
                               (sem.SEM_GEOM_STORED, "stored_native", sem.SEM_ARITH_NATIVE),
                               (sem.SEM_GEOM_TRILINEAR, "trilinear", sem.SEM_ARITH_NATIVE)):
        mesh = sem.Mesh(k, k, k, N, sem.SEM_DIRICHLET, geom,
                        verts=inputs.box_vertices(k, k, k, 0.1, 2 + k), f64_arith=arith)
        n = mesh.n_local
        kinds = ((sem.SEM_F64, torch.float64, "f64"), (sem.SEM_F32, torch.float32, "f32"))
        if gname == "stored_native":
            kinds = kinds[:1]
        if gname == "stored":
            kinds = kinds + ((sem.SEM_F16, torch.float32, "f16g"), (sem.SEM_BF16, torch.float32, "bf16g"))
        for dt, tdt, name in kinds:
            u = torch.rand(n, device=dev, dtype=tdt, generator=torch.Generator(dev).manual_seed(5))
            w = torch.empty_like(u)
            ms = traced_ms(sem, lambda: sem.sem_ax(mesh, dt, u, w, sem.SEM_AX_LOCAL), reps=20)
            esz = 8 if name == "f64" else 4
            stored = gname.startswith("stored")
            gsz = 2 if name in ("f16g", "bf16g") else esz
            bpp = 2 * esz + (6 * gsz if stored else 0)
            bytes_alg = n * bpp + (mesh.ex * mesh.ey * mesh.ez * 24 * 8 if not stored else 0)
            flops = n * (12 * (N + 1) + 15)
            out[f"{name}_{gname}"] = {
                "E": k ** 3, "ms": round(ms, 4), "gdofs_local": round(n / ms / 1e6, 3),
                "GB_s": round(bytes_alg / ms / 1e6, 1), "hbm_frac": round(bytes_alg / ms / 1e6 / hbm, 4),
                "TFLOP_s": round(flops / ms / 1e9, 3)}
            del u, w
        mesh.close()
        torch.cuda.empty_cache()
    return out


def size_sweep(sem, torch, dev, hbm, sides=(16, 32, 48, 64)):
    """Config 2 across sizes: E = k^3, N = 7, stored factors, seed 2 + k.  Per
    size and precision: the local operator, gather-scatter alone (sem_gs) and
    the assembled operator (sem_ax with SEM_AX_ASSEMBLED: the fused path),
    median of 10 calls after 3 warm-ups (the device time of every kernel a
    call launches, summed)."""
    from paper_2110_01716_gb300 import inputs

    def median_ms(fn):
        return traced_ms(sem, fn, reps=10)

    out = {}
    for k in sides:
        mesh = sem.Mesh(k, k, k, ORDER, sem.SEM_DIRICHLET,
                        verts=inputs.box_vertices(k, k, k, 0.1, 2 + k))
        n = mesh.n_local
        row = {"E": k ** 3, "n_local": n}
        for dt, tdt, name, esz in ((sem.SEM_F64, torch.float64, "f64", 8),
                                   (sem.SEM_F32, torch.float32, "f32", 4)):
            u = torch.rand(n, device=dev, dtype=tdt, generator=torch.Generator(dev).manual_seed(5))
            w = torch.empty_like(u)
            ax = median_ms(lambda: sem.sem_ax(mesh, dt, u, w, sem.SEM_AX_LOCAL))
            gs = median_ms(lambda: sem.sem_gs(mesh, dt, w))
            asm = median_ms(lambda: sem.sem_ax(mesh, dt, u, w, sem.SEM_AX_ASSEMBLED))
            bpp = 2 * esz + 6 * esz
            row[name] = {"ax_local_ms": round(ax, 4), "gs_ms": round(gs, 4),
                         "ax_assembled_ms": round(asm, 4),
                         "ax_local_hbm_frac": round(n * bpp / ax / 1e6 / hbm, 4),
                         "assembled_gdofs_local": round(n / asm / 1e6, 2)}
            del u, w
        out[str(k)] = row
        mesh.close()
        torch.cuda.empty_cache()
    return out


def named_config_leg(sem, torch, mesh, b, x, args, ng, steps=5, warmup=2):
    """The solve in the configuration the workload is named with (pMG 7-3-1,
    Chebyshev(2)-Jacobi in FP32; same mesh, right-hand side, coarse solve and
    tolerance), timed like the headline."""
    stream = torch.cuda.current_stream()
    P = sem.Pmg(mesh, orders=(7, 3, 1), cheb_degree=2, lanczos_steps=20, seed=0,
                smoother_dtype=SMOOTHER_DTYPES[args.smoother], coarse_tol=args.coarse_tol,
                coarse_maxit=args.coarse_maxit, coarse_mode=args.coarse_mode)
    ms, info = [], None
    for i in range(warmup + steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = sem.sem_solve(mesh, P, b, x, sem.SEM_SOLVER_FLEXCG, tol=TOL, max_iter=200,
                             zero_guess=True)
        e1.record(stream)
        e1.synchronize()
        if i >= warmup:
            ms.append(e0.elapsed_time(e1))
    P.close()
    t = statistics.mean(ms)
    return {"orders": "7,3,1", "cheb_degree": 2, "ms_per_solve": round(t, 2),
            "iters": info["iters"], "value": ng / (t / 1e3) / 1e9, "unit": "GDOF/s"}


def _rel_diff_mean_free(sem, torch, mesh, x, ref):
    """max |(x - mean x) - (ref - mean ref)| / max |ref - mean ref|, means over
    the unique dofs (a Neumann solution is defined up to a constant)."""
    ones = torch.ones_like(ref)
    ng = mesh.n_global
    xr = ref - sem.sem_dot(mesh, ref, ones) / ng
    xd = x - sem.sem_dot(mesh, x, ones) / ng
    num = (xd - xr).abs().max().item()
    den = xr.abs().max().item()
    del ones, xr, xd
    return num / den if den > 0 else float("nan")


def precision_leg(sem, torch, mesh, b, args, ng, steps=3, warmup=1):
    """Mixed precision against all-FP64 on the bench workload (E = 48^3,
    N = 7, Neumann, same right-hand side, coarse solve and tolerance): the
    pMG smoother in FP64, FP32, and FP32 arithmetic with FP16 / BF16 factors,
    on the headline schedule and on the named one (7-3-1, Chebyshev(2)).
    Reports ms per solve, iterations, the speed-up over the FP64 smoother of
    the same schedule, and each solution's difference from the FP64-smoother
    solution (max norm, mean-free, relative)."""
    stream = torch.cuda.current_stream()
    headline = tuple(int(o) for o in args.orders.split(","))
    legs = [("f64", headline, args.cheb_degree), ("f32", headline, args.cheb_degree),
            ("f16", headline, args.cheb_degree), ("bf16", headline, args.cheb_degree),
            ("f64", (7, 3, 1), 2), ("f32", (7, 3, 1), 2)]
    out, ref = {}, {}
    for sm, orders, deg in legs:
        P = sem.Pmg(mesh, orders=orders, cheb_degree=deg, lanczos_steps=20, seed=0,
                    smoother_dtype=SMOOTHER_DTYPES[sm], coarse_tol=args.coarse_tol,
                    coarse_maxit=args.coarse_maxit, coarse_mode=args.coarse_mode)
        x = torch.zeros_like(b)
        ms, info = [], None
        for i in range(warmup + steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = sem.sem_solve(mesh, P, b, x, sem.SEM_SOLVER_FLEXCG, tol=TOL, max_iter=200,
                                 zero_guess=True)
            e1.record(stream)
            e1.synchronize()
            if info["status"] != sem.SEM_OK:
                raise SystemExit(f"precision leg: {sm} smoother {orders} did not converge")
            if i >= warmup:
                ms.append(e0.elapsed_time(e1))
        P.close()
        sched = "-".join(str(o) for o in orders) + f"/cheb{deg}"
        t = statistics.mean(ms)
        rec = {"ms": round(t, 2), "iters": info["iters"],
               "final_rel_res": info["res"] / info["bnorm"]}
        if sm == "f64":
            ref[sched] = (x, t)
        else:
            x64, t64 = ref[sched]
            rec["speedup_vs_f64"] = round(t64 / t, 2)
            rec["rel_diff_vs_f64_solution"] = _rel_diff_mean_free(sem, torch, mesh, x, x64)
            del x
        out.setdefault(sched, {})[sm] = rec
    del ref
    torch.cuda.empty_cache()
    return out


def precision_errors_leg(sem, torch, dev, args, side=12):
    """Final-solution error of every precision variant against the FP64
    oracle: the bench recipe on a side^3 box (N = 7, Neumann, the oracle's own
    right-hand side copied to the device), GPU FlexCG + pMG (headline
    schedule) to 1e-8 with the smoother in FP64, FP32, FP16 and BF16 factor
    storage; the oracle's FlexCG + pMG (7-3-1) solution to the same 1e-8, and
    to 1e-12 (the discrete solution to round-off) as references.  Errors are
    max-norm, relative, after removing each solution's unique-dof mean."""
    import numpy as np

    import oracle
    from paper_2110_01716_gb300 import inputs

    oracle.build()
    v = inputs.box_vertices(side, side, side, 0.1, MESH_SEED)
    P = oracle.PMG(side, side, side, [7, 3, 1], 1, v, cheb_degree=2, lanczos_steps=20, seed=0,
                   coarse_tol=1e-2, coarse_maxit=50)
    L = P.levels[0]
    a, k, phi = inputs.fourier_modes(RHS_SEED)
    X = L.X
    f = sum(a[m] * np.cos(2 * np.pi * (k[m, 0] * X[:, 0] + k[m, 1] * X[:, 1] + k[m, 2] * X[:, 2])
                          + phi[m]) for m in range(len(a))).ravel()
    bo = L.gs(L.B * f)
    bo -= L.dot(bo, np.ones(L.nl)) / L.ng
    x8, i8 = P.flexpcg(bo, tol=1e-8, maxit=200)
    x12, i12 = P.flexpcg(bo, tol=1e-12, maxit=400)

    def mean_free(x):
        return x - L.dot(x, np.ones(L.nl)) / L.ng

    r8, r12 = mean_free(x8), mean_free(x12)
    mesh = sem.Mesh(side, side, side, ORDER, sem.SEM_NEUMANN, sem.SEM_GEOM_STORED, verts=v)
    bd = torch.tensor(bo, device=dev)
    orders = tuple(int(o) for o in args.orders.split(","))
    out = {"side": side, "n_global": L.ng, "oracle_iters": {"1e-8": i8["iters"], "1e-12": i12["iters"]},
           "oracle_1e-8_vs_1e-12": float(np.max(np.abs(r8 - r12)) / np.max(np.abs(r12)))}
    for sm in ("f64", "f32", "f16", "bf16"):
        Pg = sem.Pmg(mesh, orders=orders, cheb_degree=args.cheb_degree, lanczos_steps=20, seed=0,
                     smoother_dtype=SMOOTHER_DTYPES[sm], coarse_tol=args.coarse_tol,
                     coarse_maxit=args.coarse_maxit, coarse_mode=args.coarse_mode)
        xd = torch.zeros_like(bd)
        info = sem.sem_solve(mesh, Pg, bd, xd, sem.SEM_SOLVER_FLEXCG, tol=TOL, max_iter=200,
                             zero_guess=True)
        Pg.close()
        xg = mean_free(xd.cpu().numpy())
        res = np.linalg.norm(L.ax(xd.cpu().numpy()) - bo) / np.linalg.norm(bo)
        out[sm] = {"iters": info["iters"],
                   "rel_err_vs_oracle_1e-8": float(np.max(np.abs(xg - r8)) / np.max(np.abs(r8))),
                   "rel_err_vs_oracle_1e-12": float(np.max(np.abs(xg - r12)) / np.max(np.abs(r12))),
                   "residual_by_oracle": float(res)}
    mesh.close()
    return out


def config1_leg(sem, torch, dev, steps=5, warmup=2):
    """Config 1 on the GPU: E = 8^3, N = 7, jitter 0.1 (seed 1), Dirichlet,
    manufactured u* = sin(pi x) sin(pi y) sin(pi z), Jacobi-PCG to 1e-10 from
    zero; time per solve, iterations, GDOF/s and max error against u*."""
    from paper_2110_01716_gb300 import inputs

    v = inputs.box_vertices(8, 8, 8, 0.1, 1)
    mesh = sem.Mesh(8, 8, 8, ORDER, sem.SEM_DIRICHLET, sem.SEM_GEOM_STORED, verts=v)
    n = mesh.n_local
    X = [torch.empty(n, device=dev, dtype=torch.float64) for _ in range(3)]
    for d in range(3):
        sem.sem_mesh_field(mesh, d, X[d])
    Bm = torch.empty(n, device=dev, dtype=torch.float64)
    mask = torch.empty(n, device=dev, dtype=torch.float64)
    sem.sem_mesh_field(mesh, sem.SEM_FIELD_MASS, Bm)
    sem.sem_mesh_field(mesh, sem.SEM_FIELD_MASK, mask)
    us = torch.sin(torch.pi * X[0]) * torch.sin(torch.pi * X[1]) * torch.sin(torch.pi * X[2])
    b = Bm * 3 * torch.pi ** 2 * us
    sem.sem_gs(mesh, sem.SEM_F64, b)
    b *= mask
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()
    ms, info = [], None
    for i in range(warmup + steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = sem.sem_solve(mesh, None, b, x, sem.SEM_SOLVER_PCG, tol=1e-10, max_iter=2000,
                             check_every=10, zero_guess=True)
        e1.record(stream)
        e1.synchronize()
        if i >= warmup:
            ms.append(e0.elapsed_time(e1))
    err = (x - us * mask).abs().max().item()
    t = statistics.mean(ms)
    out = {"workload": "config 1: E=8^3, N=7, Dirichlet, manufactured, Jacobi-PCG to 1e-10",
           "ms_per_solve": round(t, 3), "iters": info["iters"], "status": info["status"],
           "gdofs": mesh.n_global / (t / 1e3) / 1e9, "max_err_vs_exact": err}
    mesh.close()
    return out


def projection_sequence(sem, torch, mesh, pmg, dev, solver, restart, steps=16, Lmax=30):
    """Successive solves on the smooth right-hand-side sequence (same mesh and
    preconditioner): plain solves from x = 0 against projected solves with an
    Lmax-vector space (Sec. 3).  Reports per-solve time and iterations."""
    stream = torch.cuda.current_stream()
    out = {"steps": steps, "Lmax": Lmax}
    proj = sem.Projection(mesh, Lmax)
    for mode in ("plain", "projected"):
        ms, its = [], []
        for n in range(steps):
            b = rhs_on_device(sem, torch, mesh, dev, step=n)
            x = torch.zeros_like(b)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if mode == "plain":
                info = sem.sem_solve(mesh, pmg, b, x, solver, tol=TOL, max_iter=200,
                                     restart=restart, zero_guess=True)
            else:
                info = sem.sem_solve_projected(mesh, pmg, proj, b, x, solver, tol=TOL,
                                               max_iter=200, restart=restart)
            e1.record(stream)
            e1.synchronize()
            if info["status"] != sem.SEM_OK:
                raise SystemExit(f"projection sequence: solve {n} ({mode}) did not converge")
            ms.append(e0.elapsed_time(e1))
            its.append(info["iters"])
            del b, x
        half = steps // 2
        out[mode] = {"iters": its, "ms": [round(v, 2) for v in ms],
                     "mean_ms_second_half": round(sum(ms[half:]) / (steps - half), 2)}
    proj.close()
    out["speedup_second_half"] = round(out["plain"]["mean_ms_second_half"]
                                       / out["projected"]["mean_ms_second_half"], 2)
    torch.cuda.empty_cache()
    return out


def batch_orders(N):
    o = [N]
    if 1 < N // 2 < N:
        o.append(N // 2)
    if N > 1:
        o.append(1)
    return tuple(o)


def batch_leg(sem, torch, inputs, dev, count=64, reps=5):
    """Config 4: 64 independent problems (E log-uniform in [64, 8192] on
    near-cubic boxes, N in {5, 7, 9}, manufactured right-hand side, Dirichlet,
    FlexCG + pMG (N, N/2, 1) to 1e-8), solved (a) one after another with
    sem_solve, FP64 smoother and FP32 smoother, and (b) all at once by one
    launch of the batch's CUDA graph (sem_batch, FP32 smoother), its work split
    picked by the batch autotuner.  Setup is excluded from all three (it is
    reported apart); times are CUDA events around the solves, and every leg
    leaves its solutions on the device."""
    inst = inputs.batch_instances(4, count)
    stream = torch.cuda.current_stream()
    meshes, bs = [], []
    for d in inst:
        m = sem.Mesh(d["ex"], d["ey"], d["ez"], d["N"], sem.SEM_DIRICHLET, jitter=0.1,
                     seed=d["seed"])
        n = m.n_local
        X = [torch.empty(n, device=dev, dtype=torch.float64) for _ in range(4)]
        for k in range(3):
            sem.sem_mesh_field(m, k, X[k])
        sem.sem_mesh_field(m, sem.SEM_FIELD_MASS, X[3])
        b = X[3] * 3 * torch.pi ** 2 * torch.sin(torch.pi * X[0]) * torch.sin(torch.pi * X[1]) \
            * torch.sin(torch.pi * X[2])
        sem.sem_gs(m, sem.SEM_F64, b)
        mask = torch.empty_like(b)
        sem.sem_mesh_field(m, sem.SEM_FIELD_MASK, mask)
        b *= mask
        meshes.append(m)
        bs.append(b)
        del X, mask

    def sequential(smoother):
        pmgs = [sem.Pmg(m, orders=batch_orders(d["N"]), cheb_degree=3, smoother_dtype=smoother,
                        coarse_tol=0.2, coarse_maxit=30, coarse_mode=sem.SEM_COARSE_MG)
                for m, d in zip(meshes, inst)]
        xs = [torch.zeros_like(b) for b in bs]

        def run():
            its = []
            for m, P, b, x in zip(meshes, pmgs, bs, xs):
                f = sem.sem_solve(m, P, b, x, sem.SEM_SOLVER_FLEXCG, tol=1e-8, max_iter=200,
                                  zero_guess=True)
                if f["status"] != sem.SEM_OK:
                    raise SystemExit("batch leg: a sequential solve failed")
                its.append(f["iters"])
            return its

        run()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its = run()
        e1.record(stream)
        e1.synchronize()
        for P in pmgs:
            P.close()
        return e0.elapsed_time(e1) / 1e3, its

    t64, _ = sequential(sem.SEM_F64)
    t32, its32 = sequential(sem.SEM_F32)
    hb = [b.cpu().numpy() for b in bs]
    # solutions stay on the device, as in the sequential legs (a host x would
    # add a 571 MB device-to-host copy to every timed launch)
    reqs = [sem.make_request(d["ex"], d["ey"], d["ez"], d["N"], sem.SEM_DIRICHLET, 0.1, d["seed"],
                             b=b, tol=1e-8) for d, b in zip(inst, hb)]
    for m in meshes:
        m.close()
    del meshes, bs
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    B = sem.Batch(reqs, smoother_dtype=sem.SEM_F32, cheb_degree=3, coarse_tol=0.2,
                  coarse_maxit=30, coarse_ctas=1, keep=hb)
    setup_s = time.perf_counter() - t0
    infos = B.solve()
    default_ms = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = B.solve()
        e1.record(stream)
        e1.synchronize()
        default_ms.append(e0.elapsed_time(e1))
    chosen, tuned_ms = B.autotune(candidates=(1.0, 0.5, 0.25), reps=3)
    ms = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = B.solve()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    info = B.info()
    B.close()
    if any(f["status"] != sem.SEM_OK for f in infos):
        raise SystemExit("batch leg: a batched solve failed")
    tb = statistics.median(ms) / 1e3
    return {"instances": count,
            "workload": "config 4: E log-uniform [64, 8192], N in {5,7,9}, manufactured RHS, "
                        "Dirichlet, FlexCG+pMG (N, N/2, 1) to 1e-8, setup excluded, solutions "
                        "left on the device in every leg",
            "fp64_sequential_s": round(t64, 4), "fp32_sequential_s": round(t32, 4),
            "batched_s": round(tb, 4), "batched_default_split_s": round(
                statistics.median(default_ms) / 1e3, 4),
            "solves_per_s": round(count / tb, 1),
            "speedup_vs_fp64_sequential": round(t64 / tb, 2),
            "speedup_vs_fp32_sequential": round(t32 / tb, 2),
            "autotuned_ax_fill_by_order": {str(k): v for k, v in sorted(chosen.items())},
            "autotune_note": "orders absent keep the default split (2 units per CTA slot)",
            "graph_nodes": info["graph_nodes"], "setup_s": round(setup_s, 2),
            "arena_GB": round(info["dev_bytes"] / 1e9, 2),
            "iters_mean": round(sum(f["iters"] for f in infos) / count, 2),
            "same_iters_as_sequential_fp32": [f["iters"] for f in infos] == its32}


def _serve_stream(sem, S, stream, shapes=None):
    """Submit the arrival stream (each request at its time) and wait for all;
    returns (latencies sorted, span seconds).  shapes: replace each request's
    mesh by shapes[i] (a finite population of meshes)."""
    tickets = []
    t0 = time.perf_counter()
    for i, r in enumerate(stream):
        now = time.perf_counter() - t0
        if r["t"] > now:
            time.sleep(r["t"] - now)
        m = shapes[i] if shapes is not None else r
        tickets.append(S.submit(m["ex"], m["ey"], m["ez"], m["N"], sem.SEM_DIRICHLET, 0.1,
                                m["seed"], tol=r["tol"]))
    infos = [S.wait(t) for t in tickets]
    span = time.perf_counter() - t0
    if any(f["status"] != sem.SEM_OK for f in infos):
        raise SystemExit("serve leg: a request failed")
    return sorted(f["time_ms"] for f in infos), span


def _capacity(sem, S, reqs):
    t0 = time.perf_counter()
    tk = [S.submit(r["ex"], r["ey"], r["ez"], r["N"], sem.SEM_DIRICHLET, 0.1, r["seed"],
                   tol=r["tol"]) for r in reqs]
    for t in tk:
        S.wait(t)
    return len(reqs) / (time.perf_counter() - t0)


def _pct(lat):
    return {"p50": round(lat[len(lat) // 2], 2),
            "p99": round(lat[min(len(lat) - 1, int(0.99 * len(lat)))], 2)}


def serve_leg(sem, inputs, workers=None, count=1000, load=0.8, population=12):
    """Config 5: Poisson arrivals at `load` times the measured capacity, E
    log-uniform in [512, 65536], N = 7, tolerance in {1e-6, 1e-8, 1e-10};
    latency = submit -> completion.  (a) Every request brings its own mesh:
    setup included, no cache.  (b) The same arrivals and tolerances on a
    population of `population` meshes drawn from the same distribution, whose
    setups the server has cached before the stream starts (pre-warmed: every
    request reuses a resident mesh, hierarchy and workspace).  The capacity
    of each case is measured first on 32 requests with the same workers."""
    probe = inputs.arrival_stream(5, 32, 1.0)
    if workers is None:
        sample = [sem.make_request(r["ex"], r["ey"], r["ez"], r["N"], sem.SEM_DIRICHLET, 0.1,
                                   r["seed"], tol=r["tol"]) for r in probe[:16]]
        workers, _ = sem.server_autotune(sample, max_workers=8, cache_per_shape=0)
    out = {"requests": count, "workers": workers,
           "workload": "config 5: Poisson arrivals, E log-uniform [512, 65536], N=7, "
                       "tol in {1e-6,1e-8,1e-10}"}
    # (a) setup included
    S = sem.Server(workers=workers, cache_per_shape=0)
    cap = _capacity(sem, S, probe)
    lat, span = _serve_stream(sem, S, inputs.arrival_stream(5, count, load * cap))
    st = S.stats()
    S.close()
    out["setup_included"] = {"capacity_solves_per_s": round(cap, 2),
                             "offered_rate": round(load * cap, 2),
                             "achieved_solves_per_s": round(count / span, 2),
                             "latency_ms": _pct(lat), "setups_built": st["setups_built"]}
    # (b) pre-warmed cache over a finite mesh population: up to `copies`
    # idle setups per mesh, built by `copies` concurrent requests per mesh
    shapes = inputs.arrival_stream(55, population, 1.0)
    rng = __import__("random").Random(56)
    copies = 3
    S = sem.Server(workers=workers, cache_per_shape=copies)
    warm = [S.submit(m["ex"], m["ey"], m["ez"], m["N"], sem.SEM_DIRICHLET, 0.1, m["seed"],
                     tol=1e-6) for m in shapes for _ in range(copies)]
    for t in warm:
        S.wait(t)
    pick = [shapes[rng.randrange(population)] for _ in range(count)]
    cap = _capacity(sem, S, [dict(pick[i], tol=probe[i]["tol"]) for i in range(len(probe))])
    st0 = S.stats()
    lat, span = _serve_stream(sem, S, inputs.arrival_stream(5, count, load * cap), shapes=pick)
    st = S.stats()
    S.close()
    out["prewarmed"] = {"population": population, "cached_per_mesh": copies,
                        "capacity_solves_per_s": round(cap, 2),
                        "offered_rate": round(load * cap, 2),
                        "achieved_solves_per_s": round(count / span, 2),
                        "latency_ms": _pct(lat),
                        "setups_built_in_stream": st["setups_built"] - st0["setups_built"],
                        "setups_reused_in_stream": st["setups_reused"] - st0["setups_reused"],
                        "hbm_in_use_GB": round(st["hbm_in_use"] / 1e9, 2)}
    out["latency_ms"] = out["setup_included"]["latency_ms"]
    return out


def oracle_sample_solve(side=12):
    """One oracle FlexCG + pMG solve on a side^3 box of the same recipe.
    Returns (seconds, unique dofs, iterations, threads)."""
    import numpy as np

    import oracle
    from paper_2110_01716_gb300 import inputs

    oracle.build()
    v = inputs.box_vertices(side, side, side, 0.1, MESH_SEED)
    P = oracle.PMG(side, side, side, [7, 3, 1], 1, v, cheb_degree=2, lanczos_steps=20, seed=0,
                   coarse_tol=1e-2, coarse_maxit=50)
    L = P.levels[0]
    a, k, phi = inputs.fourier_modes(RHS_SEED)
    X = L.X
    f = sum(a[m] * np.cos(2 * np.pi * (k[m, 0] * X[:, 0] + k[m, 1] * X[:, 1] + k[m, 2] * X[:, 2])
                          + phi[m]) for m in range(len(a))).ravel()
    b = L.gs(L.B * f)
    b -= L.dot(b, np.ones(L.nl)) / L.ng
    t0 = time.perf_counter()
    x, info = P.flexpcg(b, tol=TOL, maxit=200)
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return dt, L.ng, info["iters"], threads


def oracle_extrapolated(sample_s, sample_iters, sample_side, side, gpu_iters, n_global):
    """The oracle's full-size solve time, extrapolated: the sample's seconds
    per iteration scaled by the element count (side / sample_side)^3, times
    the GPU's iteration count.  Optimistic for the oracle, whose Jacobi-PCG
    coarse solve needs more iterations on a larger coarse grid."""
    per_it = sample_s / max(sample_iters, 1) * (side / sample_side) ** 3
    solve_s = per_it * gpu_iters
    return {"kind": "extrapolated", "per_iteration_s": per_it, "iterations": gpu_iters,
            "solve_s": solve_s, "gdofs": n_global / solve_s / 1e9,
            "basis": f"{sample_side}^3 sample: seconds per iteration x (E / {sample_side}^3) "
                     "x the GPU's iterations"}


def oracle_timings():
    """The oracle on this host, on one core and on all of them: config 1 (the
    8^3-element, N = 7 Dirichlet manufactured solve, Jacobi-PCG to 1e-10)
    and config 2 at 16^3, 24^3 and 32^3 elements (local operator,
    gather-scatter and the assembled operator, u ~ U(-1, 1))."""
    import numpy as np

    import oracle
    from paper_2110_01716_gb300 import inputs

    oracle.build()
    allc = os.cpu_count() or 1
    out = {}
    for label, nth in (("all_cores", allc), ("one_core", 1)):
        used = oracle.set_threads(nth)
        row = {"threads": used}
        v = inputs.box_vertices(8, 8, 8, 0.1, 1)
        L = oracle.Level(8, 8, 8, ORDER, 0, v)
        X = L.X
        us = (np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])).ravel()
        b = L.assembled_rhs(3 * np.pi ** 2 * us)
        t0 = time.perf_counter()
        _, info = L.pcg(b, tol=1e-10, maxit=2000)
        dt = time.perf_counter() - t0
        row["config1_pcg"] = {"s": round(dt, 3), "iters": info["iters"],
                              "gdofs": round(L.ng / dt / 1e9, 6)}
        del L
        for k in (16, 24, 32):
            L2 = oracle.Level(k, k, k, ORDER, 0, inputs.box_vertices(k, k, k, 0.1, 2 + k))
            u = np.random.default_rng(2 + k).uniform(-1, 1, L2.nl)
            t0 = time.perf_counter()
            w = L2.ax_local(u)
            t1 = time.perf_counter()
            L2.gs(w)
            t2 = time.perf_counter()
            L2.ax(u)
            t3 = time.perf_counter()
            row[f"config2_{k}cube"] = {"ax_local_s": round(t1 - t0, 4), "gs_s": round(t2 - t1, 4),
                                       "ax_assembled_s": round(t3 - t2, 4),
                                       "ax_local_gdofs": round(L2.nl / (t1 - t0) / 1e9, 4)}
            del L2, u, w
        out[label] = row
    oracle.set_threads(allc)
    return out


def summary_of(line):
    """The figures a reader needs first, in one small object."""
    r = line.get("roofline", {})
    other = r.get("other", {})
    out = {"ms_per_solve": round(line["ms_per_step"], 2), "iters": line["iters"][0],
           "GDOF_s": round(line["value"], 4),
           "e2e_GDOF_s": round(line.get("e2e", {}).get("value", float("nan")), 4),
           "roofline": {r.get("kernel"): round(r.get("frac") or 0, 3),
                        other.get("kernel"): round(other.get("frac") or 0, 3)}}
    prec = line.get("precision", {})
    for sched, legs in prec.items():
        out["fp64_smoother_" + sched] = {sm: [v["ms"], v["iters"], v.get("speedup_vs_f64")]
                                         for sm, v in legs.items()}
    pe = line.get("precision_errors", {})
    if pe:
        out["err_vs_oracle"] = {sm: pe[sm]["rel_err_vs_oracle_1e-12"]
                                for sm in ("f64", "f32", "f16", "bf16") if sm in pe}
    if "serve" in line:
        sv = line["serve"]
        out["serve_p50_p99_ms"] = {k: [sv[k]["latency_ms"]["p50"], sv[k]["latency_ms"]["p99"]]
                                   for k in ("setup_included", "prewarmed") if k in sv}
    if "batch" in line:
        out["batch_solves_per_s"] = line["batch"].get("solves_per_s")
    if "config1" in line:
        out["config1_ms"] = line["config1"]["ms_per_solve"]
    return out


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    side = 12
    for _ in range(args.warmup):
        oracle_sample_solve(side)
    times, ng, iters, threads = [], 0, 0, 1
    for _ in range(args.steps):
        dt, ng, iters, threads = oracle_sample_solve(side)
        times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = ng / (ms / 1e3) / 1e9
    sample = (f"oracle FlexCG+pMG 7-3-1 solve to 1e-8 on a {side}^3-element box of the same "
              f"recipe (N=7, Neumann, {ng} unique dofs, {iters} iterations), setup excluded")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GDOF/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "reference_sample": sample},
            "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch

    from paper_2110_01716_gb300 import build, inputs, sem

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.ax_only:
        build.build()
        k = args.ax_only
        mesh = sem.Mesh(k, k, k, args.ax_order, sem.SEM_NEUMANN, sem.SEM_GEOM_STORED,
                        verts=inputs.box_vertices(k, k, k, 0.1, MESH_SEED))
        u = torch.rand(mesh.n_local, device=dev, dtype=torch.float32,
                       generator=torch.Generator(dev).manual_seed(5)) * 2 - 1
        w = torch.empty_like(u)
        for kind in (sem.SEM_F32, sem.SEM_F16):
            for _ in range(2):
                sem.sem_ax(mesh, kind, u, w, sem.SEM_AX_ASSEMBLED)
        torch.cuda.synchronize()
        print(json.dumps({"ax_only": k, "N": args.ax_order, "n_local": mesh.n_local}))
        return 0
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    build.build()
    hbm, hbm_src = measured_peaks()

    side = args.side
    verts = inputs.box_vertices(side, side, side, 0.1, MESH_SEED)
    mesh = sem.Mesh(side, side, side, ORDER, sem.SEM_NEUMANN, sem.SEM_GEOM_STORED, verts=verts)
    orders = tuple(int(o) for o in args.orders.split(","))
    if orders[0] != ORDER:
        raise SystemExit(f"--orders must start with the fine order {ORDER}")
    pmg = sem.Pmg(mesh, orders=orders, cheb_degree=args.cheb_degree, lanczos_steps=20, seed=0,
                  smoother_dtype=SMOOTHER_DTYPES[args.smoother], coarse_tol=args.coarse_tol,
                  coarse_maxit=args.coarse_maxit, coarse_mode=args.coarse_mode,
                  smoother=(sem.SEM_SMOOTH_ASM_TF32 if args.schwarz_tf32 else
                            sem.SEM_SMOOTH_ASM_TC if args.schwarz_tc else
                            sem.SEM_SMOOTH_ASM if args.schwarz else sem.SEM_SMOOTH_JACOBI))
    b = rhs_on_device(sem, torch, mesh, dev)
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()

    solver = sem.SEM_SOLVER_FGMRES if args.solver == "fgmres" else sem.SEM_SOLVER_FLEXCG

    # FlexCG runs its iterations 2.. as one CUDA-graph launch with the stopping
    # test on the device (use_graph; the same kernels and bits as the host
    # loop): the initial V-cycle and iteration 1 stay host-launched, so the
    # kernels of the roofline entry are event-timed there, and the graph's
    # launches are counted per class from the tally taken at its capture
    use_graph = solver == sem.SEM_SOLVER_FLEXCG and not args.host_loop

    def step(graph=use_graph):  # from x = 0 (the solver zeroes x and skips the product with it)
        return sem.sem_solve(mesh, pmg, b, x, solver, tol=TOL, max_iter=200, check_every=1,
                             restart=args.restart, zero_guess=True, use_graph=graph)

    for _ in range(max(args.warmup, 0)):
        info = step()
    # timed region
    smoother_key = {"f32": "ax32_f32", "f16": "ax32_f16g", "bf16": "ax32_bf16g"}.get(args.smoother)
    keys = [f"ax_f64pair_N{ORDER}"] + ([f"{smoother_key}_N{ORDER}"] if smoother_key else [])
    sem.sem_trace_enable(True, "|".join(keys))
    sem.sem_trace_read(reset=True)
    clocks = ClockSampler(local)
    clocks.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    infos = []
    for s in range(args.steps):
        infos.append(step())
        ev[s + 1].record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clk = clocks.stop()
    trace = sem.sem_trace_read(reset=True)
    sem.sem_trace_enable(False, "")
    step_ms = [ev[s].elapsed_time(ev[s + 1]) for s in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    total_ms = job_time_ms(pg, total_ms, dev)
    ms_per_step = total_ms / args.steps
    ng = mesh.n_global
    value = job_value(world, ng, ms_per_step)
    for inf in infos:
        if inf["status"] != sem.SEM_OK:
            raise SystemExit(f"solve did not converge: {inf}")

    nl = mesh.n_local
    launches = sum(v["launches"] for v in trace.values())

    def timed(key):
        # average event-timed launch; share of the step from every launch of
        # the class (graph replays included)
        ent = trace.get(key, {"launches": 0, "timed": 0, "total_ms": 0.0})
        per = ent["total_ms"] / max(ent["timed"], 1)
        share = per * ent["launches"] / total_ms if total_ms > 0 else None
        return per, share, ent["timed"]

    # FP64 operator in FP32-pair arithmetic (FP32-pipe bound)
    key64 = f"ax_f64pair_N{ORDER}"
    ax_ms, ax_share, ax_n = timed(key64)
    flops_pt = 12 * (ORDER + 1) + 15
    ax_tflops = nl * flops_pt / (ax_ms / 1e3) / 1e12 if ax_ms > 0 else None
    traffic64 = None
    if AX_TRAFFIC["source_sha256"] == source_sha("pair.cuh") and AX_TRAFFIC["bytes_per_point"]:
        traffic64 = AX_TRAFFIC["bytes_per_point"] * nl
    roof64 = {"bound": "alu", "achieved": ax_tflops, "peak": PAIR_PEAK_TFLOPS,
              "unit": "TFLOP/s", "frac": (ax_tflops / PAIR_PEAK_TFLOPS) if ax_tflops else None,
              "traffic": traffic64, "kernel": key64,
              "per_launch_ms": ax_ms, "launches_timed": ax_n, "share_of_step": ax_share,
              "algorithmic": f"{flops_pt} flop/pt x {nl} local pts per launch",
              "peak_source": "derived: FP32 issue 152 SM x 128 lanes x 2.07 GHz / "
                             f"{PAIR_INSTR_PER_FMA} instr per FP64-equivalent FMA x 2 flop "
                             f"(native FP64 pipe: {FP64_PEAK_TFLOPS:.3f})"}
    roofline = roof64
    if smoother_key:
        # the smoother's fused FP32 operator on stored factors (HBM bound):
        # u and w in FP32 plus six factors per point (FP32 or 16-bit)
        key32 = f"{smoother_key}_N{ORDER}"
        s_ms, s_share, s_n = timed(key32)
        gsz = 4 if args.smoother == "f32" else 2
        bpp = 8 + 6 * gsz + (4.0 / (ORDER + 1) ** 3 if gsz == 2 else 0.0)
        s_gbs = bpp * nl / (s_ms / 1e3) / 1e9 if s_ms > 0 else None
        rec = AX32_TRAFFIC.get(args.smoother)
        traffic32 = None
        if rec and rec["source_sha256"] == source_sha("ax32.cu"):
            traffic32 = rec["bytes_per_point"] * nl
        roof32 = {"bound": "hbm", "achieved": s_gbs, "peak": hbm, "unit": "GB/s",
                  "frac": (s_gbs / hbm) if s_gbs else None, "traffic": traffic32,
                  "kernel": key32, "per_launch_ms": s_ms, "launches_timed": s_n,
                  "share_of_step": s_share,
                  "algorithmic": f"{bpp:.3f} B/pt x {nl} local pts = {bpp * nl / 1e9:.3f} GB per launch",
                  "peak_source": f"HBM {hbm} GB/s {hbm_src}"}
        # the dominant kernel (largest share of the step) is the headline roofline
        if (s_share or 0) >= (ax_share or 0):
            roofline = dict(roof32, other=roof64)
        else:
            roofline = dict(roof64, other=roof32)

    line = {"metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+" + args.smoother, "data": "synthetic",
            "config": {"workload": WORKLOAD, "E": side ** 3, "N": ORDER, "n_local": nl,
                       "solver": args.solver, "smoother": args.smoother,
                       "smoothing": ("chebyshev-schwarz-tf32" if args.schwarz_tf32 else
                                     "chebyshev-schwarz-tc" if args.schwarz_tc else
                                     "chebyshev-schwarz" if args.schwarz else "chebyshev-jacobi"),
                       "orders": args.orders, "cheb_degree": args.cheb_degree,
                       "coarse_tol": args.coarse_tol,
                       "coarse_maxit": args.coarse_maxit, "coarse_mode": args.coarse_mode,
                       "n_global": ng, "parallelism": "replicas" if world > 1 else "single",
                       "loop": ("cuda graph: iterations 2.. in one launch, stopping test on "
                                "the device" if use_graph else "host-driven"),
                       "l2": "inputs larger than L2 (working set ~6 GB), no flush"},
            "iters": [inf["iters"] for inf in infos],
            "final_rel_res": max(inf["res"] / inf["bnorm"] for inf in infos),
            "latency_ms": {"p50": statistics.median(step_ms),
                           "p99": sorted(step_ms)[min(len(step_ms) - 1,
                                                      int(0.99 * len(step_ms)))]},
            "roofline": roofline, "gpu_launches": launches,
            "trace_classes": {k: v["launches"] for k, v in sorted(trace.items())},
            "clocks": clk}

    if args.breakdown:
        # one untimed solve with every launch bracketed by events (Table-1 style)
        sem.sem_trace_enable(True, "*")
        sem.sem_trace_read(reset=True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(graph=False)  # host-launched, so that every kernel is timed
        e1.record(stream)
        torch.cuda.synchronize()
        bd = sem.sem_trace_read(reset=True)
        sem.sem_trace_enable(False, "")
        tot = e0.elapsed_time(e1)
        line["breakdown"] = {"solve_ms": tot, "kernel_ms": sum(v["total_ms"] for v in bd.values()),
                             "coarse_iters_last_vcycle": pmg.coarse_iters(),
                             "classes": {k: [v["launches"], round(v["total_ms"], 3)]
                                         for k, v in sorted(bd.items(),
                                                            key=lambda kv: -kv[1]["total_ms"])}}

    if not args.no_extras and rank == 0:
        ex = {}
        if solver == sem.SEM_SOLVER_FLEXCG:
            # the same solves with the other loop (host-driven when the
            # timed region ran the graph, and the other way round), right
            # after the timed region so that both see the same GPU state: the
            # host-driven loop reads <r, r> after every iteration
            gt = []
            for i in range(args.warmup + args.steps):
                ge0 = torch.cuda.Event(enable_timing=True)
                ge1 = torch.cuda.Event(enable_timing=True)
                ge0.record(stream)
                ginf = step(graph=not use_graph)
                ge1.record(stream)
                torch.cuda.synchronize()
                if i >= args.warmup:
                    gt.append(ge0.elapsed_time(ge1))
            other = statistics.mean(gt)
            ex["graph"] = {"ms_per_solve": ms_per_step if use_graph else other,
                           "host_loop_ms_per_solve": other if use_graph else ms_per_step,
                           "timed_region_loop": "graph" if use_graph else "host",
                           "iters": ginf["iters"],
                           "value": ng / ((ms_per_step if use_graph else other) / 1e3) / 1e9,
                           "unit": "GDOF/s"}
        # end to end through the host-buffer entry point: host b in, host x
        # out (pinned host memory), from x = 0 (x's input is neither read nor
        # copied)
        bh = b.cpu().pin_memory()
        xh = torch.zeros(nl, dtype=torch.float64).pin_memory()
        # as many warm-up calls as the timed region has (the first one
        # captures the graph again for this x buffer)
        for _ in range(max(3, args.warmup)):
            sem.sem_solve_host(mesh, pmg, bh, xh, solver, tol=TOL, max_iter=200,
                               restart=args.restart, zero_guess=True, use_graph=use_graph)
        torch.cuda.synchronize()
        per_step = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ts = time.perf_counter()
            sem.sem_solve_host(mesh, pmg, bh, xh, solver, tol=TOL, max_iter=200,
                               restart=args.restart, zero_guess=True, use_graph=use_graph)
            per_step.append(time.perf_counter() - ts)  # the call returns after its copy out
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.steps
        # the host link's rate on these very buffers, after the timed region:
        # the part of the end-to-end time the copies take
        db = torch.empty(nl, dtype=torch.float64, device=dev)
        rates = {}
        for name, dst, src in (("h2d_GBps", db, bh), ("d2h_GBps", xh, db)):
            best = None
            for _ in range(3):
                c0 = torch.cuda.Event(enable_timing=True)
                c1 = torch.cuda.Event(enable_timing=True)
                c0.record(stream)
                dst.copy_(src, non_blocking=True)
                c1.record(stream)
                c1.synchronize()
                t = c0.elapsed_time(c1)
                best = t if best is None else min(best, t)
            rates[name] = round(nl * 8 / (best / 1e3) / 1e9, 1)
        del db
        line["e2e"] = {"value": ng / e2e_s / 1e9, "unit": "GDOF/s",
                       "h2d_bytes_per_step": nl * 8, "d2h_bytes_per_step": nl * 8,
                       "ms_per_step": round(e2e_s * 1e3, 2),
                       "ms_per_step_median": round(statistics.median(per_step) * 1e3, 2),
                       "ms_per_step_max": round(max(per_step) * 1e3, 2), **rates}
        del bh, xh
        if solver == sem.SEM_SOLVER_FLEXCG:
            ex["named_config"] = named_config_leg(sem, torch, mesh, b, x, args, ng)
            ex["precision"] = precision_leg(sem, torch, mesh, b, args, ng)
        ex["projection"] = projection_sequence(sem, torch, mesh, pmg, dev, solver, args.restart)
        pmg.close()
        mesh.close()
        del b, x
        torch.cuda.empty_cache()
        ex["config1"] = config1_leg(sem, torch, dev)
        if not args.no_serve:
            ex["batch"] = batch_leg(sem, torch, inputs, dev)
            ex["serve"] = serve_leg(sem, inputs)
        ex["ax_sweep_64cube"] = operator_sweep(sem, torch, dev, hbm)
        ex["ax_gs_sizes"] = size_sweep(sem, torch, dev, hbm)
        if world == 1:
            ex["precision_errors"] = precision_errors_leg(sem, torch, dev, args)
            dt, ng_s, it_s, threads = oracle_sample_solve(12)
            ex["oracle_timings"] = oracle_timings()
            ex["oracle_timings"]["config3_extrapolated"] = oracle_extrapolated(
                dt, it_s, 12, side, line["iters"][0], ng)
            line["cpu_baseline"] = {
                "value": ng_s / dt / 1e9, "unit": "GDOF/s", "cores": threads, "kind": "oracle",
                "sample": f"oracle FlexCG+pMG 7-3-1 solve to 1e-8 on a {12}^3-element box of the "
                          f"same recipe ({ng_s} unique dofs, {it_s} iterations, {dt:.1f} s)"}
        # long sweeps first and the legs that matter last, so that a reader of
        # the end of the line sees them; a compact summary closes the line
        for key in ("ax_sweep_64cube", "ax_gs_sizes", "oracle_timings", "projection", "config1",
                    "batch", "serve", "graph", "named_config", "precision_errors", "precision"):
            if key in ex:
                line[key] = ex.pop(key)
        line["summary"] = summary_of(line)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
