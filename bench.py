#!/usr/bin/env python
"""Benchmark: MGR-preconditioned FGMRES(30) time to a 1e-8 relative residual on the 128^3 x 3
two-phase two-component NCP workload (FP32 hierarchy / FP64 Krylov, FP64 beside it), with the HBM
roofline fraction of the dominant kernel.

A step is one pass of the hot path over one synthetic Jacobian resident in HBM: mgr_setup (global
relaxation blocks, the three reductions with their R(AP) products, AMG setup on the pressure system,
FP32 cast) followed by fgmres_solve from x0 = 0 to ||b - A x|| <= 1e-8 ||b||.  value = milliseconds
per step (lower is better).  One JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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
sys.path.insert(0, ROOT)

METRIC = "MGR-FGMRES time-to-1e-8 residual & HBM GB/s fraction, 128^3x3; FP32-mix vs FP64"
WORKLOAD = "ncp3d_128_layered"
RTOL, RESTART, MAXIT = 1e-8, 30, 1000
# Solver settings used for the 3-D workloads: strength threshold 0.58 (the middle of the range 0.55-0.6
# where the iteration count is lowest: 41-42 at 128^3, against 50 at 0.5 and 48 at 0.62) and
# interpolation truncation to 4 entries keep the AMG operator complexity low on the 25-63 point
# pressure stencils; omega-Jacobi (0.8) smoothing converges in fewer iterations than l1-Jacobi on
# these operators; one l1-Jacobi sweep on the saturation and gas-absent constraint blocks (levels 2
# and 3) converges in fewer outer iterations than two; the AMG coarsens down to at most 64 rows,
# whose dense inverse is cheap to build.
SOLVER = dict(amg_theta=0.58, amg_pmax=4, amg_smoother=0, amg_omega=0.8, amg_max_coarse=64, frelax_sweeps=[1, 1, 1])
# The two-level unsaturated workloads (section 6.1): injective R at both reductions, three
# l1-Jacobi sweeps on the saturation block, V(2,2) on the pressure system, default AMG settings.
UNSAT_SOLVER = dict(restrict_type=[0, 0], frelax_type=[1, 1], frelax_sweeps=[1, 3], amg_pre=2, amg_post=2)
L2_BYTES = 129 * 1024 * 1024


SOLVE_KERNELS = ("mgr_apply", "amg_tail", "bsr3_spmv_f64", "mdot", "mupdate", "global_relax", "bsr_resid_split",
                 "frelax0", "frelax1", "frelax2", "frelax3", "restrict0", "restrict1", "restrict2", "restrict3",
                 "interp0", "interp1", "interp2", "interp3", "amg0_rows", "amg1_rows", "amg2_rows", "amgc_rows",
                 "amg0_restrict", "amg1_restrict", "amgc_restrict", "amg0_prolong", "amg1_prolong", "amgc_prolong",
                 "famg_rows", "famg_transfer")
SETUP_KERNELS = ("setup_total", "setup_mgr_level", "setup_mgr_rap", "setup_amg", "setup_amg_strength",
                 "setup_amg_pmis", "setup_amg_extpi", "extpi_pattern", "extpi_weights", "setup_amg_transpose",
                 "setup_amg_rap", "setup_dense_inverse", "setup_cast_alloc", "spgemm", "fused_small", "fused_copy",
                 "spgemm_numeric", "sym_ub", "sym_count", "sym_fill", "sym_block", "sym_bitmap",
                 "rap_mgr0_AP", "rap_mgr0_RAP", "rap_mgr1_AP", "rap_mgr1_RAP", "rap_mgr2_AP", "rap_mgr2_RAP",
                 "rap_amg0_AP", "rap_amg0_PtAP", "rap_amg1_AP", "rap_amg1_PtAP", "rap_amgc_AP", "rap_amgc_PtAP",
                 "spgemm_extpi", "setup_famg")
KERNEL_NAMES = SOLVE_KERNELS + SETUP_KERNELS
# DRAM bytes over algorithmic bytes of one launch, from one ncu capture of the kernel on an 80^3
# instance of the workload (dram__bytes_read.sum + dram__bytes_write.sum); the traffic of a full-size
# launch is this ratio times its algorithmic bytes, which scale with the entries it streams.
# k_bsr_sell<double> (FP64 SpMV): 295.11 MB for 298.14 MB.  (The multi-dot has changed since its
# counters were taken: no entry, so its traffic is reported as null.)
TRAFFIC = {"bsr3_spmv_f64": 295.114240e6 / 298137608.0}
# Krylov kernels bound by GB300's FP64 FMA rate: their FMAs per launch.  The multi-dot does one FMA
# per 8-byte element it reads (V_k . w and w . w), i.e. its algorithmic bytes / 8; the 3x3-block SpMV
# 9 per stored block.
FP64_BOUND = ("bsr3_spmv_f64", "mdot")
# FGMRES(30) iterations of the oracle (FP64) on the full-size instances, measured once (the GPU's
# FP64-hierarchy count agrees within one, checked by the full-size parity test): the CPU baseline's
# sample solve is scaled per iteration to this count.
FULL_SIZE_ITERATIONS = {"ncp3d_128_layered": 41}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--grid", type=int, default=0, help="scaled instance: n^3 cells of the workload recipe")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-full", action="store_true", help="time the oracle on the full-size instance (minutes)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--solver", default="", help="JSON dict of solver options overriding the defaults")
    ap.add_argument("--newton", type=int, default=0,
                    help="instead of the linear benchmark: this many backward Euler steps of the semi-smooth "
                         "Newton loop on the workload, the linear solves on the GPU")
    ap.add_argument("--linear-rtol", type=float, default=RTOL, help="linear tolerance of the Newton mode")
    args = ap.parse_args()
    if args.workload.startswith("unsat2d"):
        SOLVER.clear()
        SOLVER.update(UNSAT_SOLVER)
    if args.solver:
        SOLVER.update(json.loads(args.solver))
    return args


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """Largest value over the ranks (the job's time is its slowest replica)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_config(cfg, rank: int):
    """Replicas only: every rank solves the same workload recipe independently (no data exchange)."""
    return cfg


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _cpu_sample_cfg(cfg, n):
    """A smaller instance of the workload recipe with about n^3 cells and the same aspect ratio."""
    import dataclasses
    cells = cfg.nx * cfg.ny * cfg.nz
    dim = 3 if cfg.nz > 1 else 2
    f = min(1.0, (n ** 3 / cells) ** (1.0 / dim))
    return dataclasses.replace(cfg, nx=max(1, round(cfg.nx * f)), ny=max(1, round(cfg.ny * f)),
                               nz=max(1, round(cfg.nz * f)) if cfg.nz > 1 else 1)


def run_oracle_sample(cfg, n_sample):
    """Oracle (FP64, one thread) setup + solve on an n_sample^3 instance of the workload recipe."""
    import ncpgen
    import oracle
    sc = _cpu_sample_cfg(cfg, n_sample)
    p = ncpgen.make_problem(sc)
    b = ncpgen.normals(p.n, 2)
    t0 = time.perf_counter()
    o = oracle.OracleMGR(p.rowptr, p.colind, p.values, p.cf_marker, **SOLVER)
    t1 = time.perf_counter()
    x, info = o.fgmres(b, rtol=RTOL, restart=RESTART, maxit=MAXIT)
    t2 = time.perf_counter()
    return dict(cells=p.nb, setup_s=t1 - t0, solve_s=t2 - t1, iterations=info["iterations"],
                converged=info["converged"])


def oracle_estimate(cfg, workload, n_sample, full_iterations=None):
    """The oracle's time for the full-size workload from a bounded n_sample^3 instance of its recipe:
    setup scaled by cell count, solve scaled by cell count and per iteration to the full-size
    iteration count (a sample converges in fewer iterations than the full grid).  Returns
    (milliseconds, description)."""
    r = run_oracle_sample(cfg, n_sample)
    cells = cfg.nx * cfg.ny * cfg.nz
    f = cells / r["cells"]
    it = full_iterations or FULL_SIZE_ITERATIONS.get(workload) or r["iterations"]
    ms = (r["setup_s"] * f + r["solve_s"] / r["iterations"] * it * f) * 1e3
    desc = (f"{n_sample}^3 instance of the {workload} recipe, FP64 oracle on 1 core: setup {r['setup_s']:.2f} s "
            f"x{f:.1f} (cells) + solve {r['solve_s']:.2f} s for {r['iterations']} iterations, scaled per "
            f"iteration to the full grid's {it} and x{f:.1f} (cells)")
    return ms, desc, r


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _shape(m, kind, lev):
    import ctypes
    import paper_1801_08464_gb300 as mg
    nr, nc, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    mg.lib().mgr_matrix_shape(m._h, kind, lev, ctypes.byref(nr), ctypes.byref(nc), ctypes.byref(nnz))
    return nr.value, nnz.value


def run_newton(a, cfg, config, rank):
    """Semi-smooth Newton (section 3.1) over a.newton time steps from the workload's state, every
    linear solve by MGR-FGMRES on the GPU (FP32 hierarchy, FP64 Krylov), the Jacobians assembled on
    the host by the input generator; reports nonlinear (NS) and linear (LS) iteration counts, LS/NS
    and the GPU time of the linear solves (setup + solve), the host assembly and copies apart."""
    import numpy as np
    import torch

    import ncpgen
    from paper_1801_08464_gb300.newton import MgrLinearSolver, semismooth_newton
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    tol = 1e-5
    solve = MgrLinearSolver(precision="mixed", rtol=a.linear_rtol, restart=RESTART, maxit=MAXIT, **SOLVER)
    p = ncpgen.make_problem(cfg)
    u = p.state.reshape(-1).copy()
    # warm-up: one Newton step of the first time step (not counted)
    semismooth_newton(lambda v: ncpgen.newton_system(cfg, v, u), u, solve, tol=tol, max_steps=1)
    steps, t0 = [], time.perf_counter()
    for _ in range(a.newton):
        u_old = u.copy()
        u, hist, ok = semismooth_newton(lambda v: ncpgen.newton_system(cfg, v, u_old), u, solve, tol=tol)
        steps.append((hist, ok))
    wall = (time.perf_counter() - t0) * 1e3
    ns = sum(len(h) - 1 for h, _ in steps)
    ls = sum(x.lin_iterations for h, _ in steps for x in h)
    gpu_ms = sum(x.setup_ms + x.solve_ms for h, _ in steps for x in h)
    out = {"metric": "semi-smooth Newton with MGR-FGMRES linear solves: LS/NS and linear-solve time",
           "value": gpu_ms / max(ns, 1), "unit": "ms per Newton step (GPU setup + solve)", "n_gpus": 1,
           "steps": a.newton, "higher_is_better": False, "dtype": "f32+f64", "data": "synthetic",
           "config": dict(config, newton_tol=tol, linear_rtol=a.linear_rtol),
           "converged": all(ok for _, ok in steps), "NS": ns, "LS": ls, "LS_per_NS": ls / max(ns, 1),
           "active_set_changes": sum(x.active_changes for h, _ in steps for x in h),
           "pattern_uploads": solve.pattern_uploads,
           "per_time_step": [{"newton_steps": len(h) - 1, "residuals": [x.resnorm for x in h],
                              "linear_iterations": [x.lin_iterations for x in h[:-1]]} for h, _ in steps],
           "gpu_linear_ms": gpu_ms, "wall_ms_including_host_assembly": wall,
           "final_resnorm": steps[-1][0][-1].resnorm if steps else None,
           "S_l_range": [float(np.min(u[1::3])), float(np.max(u[1::3]))]}
    solve.close()
    if rank == 0:
        print(json.dumps(out))


def main():
    a = _args()
    if a.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    import ncpgen
    cfg = ncpgen.WORKLOADS[a.workload]
    if a.grid:
        cfg = _cpu_sample_cfg(cfg, a.grid)
    grid = [cfg.nx, cfg.ny, cfg.nz]
    cells = cfg.nx * cfg.ny * cfg.nz
    # FP64 BSR values of the 7- (5-) point pattern: below twice L2 the bench flushes L2 before each step
    in_bytes = 72 * (cells + 2 * 3 * cells) + 8 * 3 * cells
    flush_l2 = in_bytes < 2 * L2_BYTES
    config = {"workload": a.workload, "grid": grid, "unknowns": 3 * cells,
              "precision": "fp32 hierarchy, fp64 krylov", "rtol": RTOL, "restart": RESTART,
              "solver": SOLVER,
              "l2": ("L2 flushed (a 512 MB write, outside the timed events) before every timed step" if flush_l2
                     else "inputs larger than L2 (FP64 BSR values > 1 GB)"),
              "parallelism": f"replicas x{a.gpus}"}

    if a.newton and a.impl == "ours":
        run_newton(a, cfg, config, rank)
        return

    if a.impl == "reference":
        if rank != 0:
            return
        n_s = 48
        for _ in range(a.warmup):
            run_oracle_sample(cfg, n_s)
        vals = []
        for _ in range(a.steps):
            v, sample, r = oracle_estimate(cfg, a.workload, n_s)
            vals.append(v)
        v = statistics.mean(vals)
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": a.gpus,
                          "steps": a.steps, "warmup": a.warmup, "ms_per_step": v,
                          "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": config,
                          "cpu_baseline": {"value": v, "unit": "ms", "cores": 1, "kind": "oracle", "sample": sample},
                          "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                          "iterations": r["iterations"]}))
        return

    import numpy as np
    import torch

    import paper_1801_08464_gb300 as mg
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    p = ncpgen.make_problem(replica_config(cfg, rank))
    b_h = ncpgen.normals(p.n, 2)
    A = mg.BSR3.from_numpy(p.rowptr, p.colind, p.values)
    mk = torch.as_tensor(p.cf_marker, device="cuda")
    b = torch.as_tensor(b_h, device="cuda")
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def _max(v):
        return max_over_ranks(v, dist, "cuda")

    def step(m):
        m.setup(A, mk)
        x.zero_()
        _, info = m.fgmres(A, b, x, rtol=RTOL, restart=RESTART, maxit=MAXIT)
        return info

    def timed(prec, steps, profile=False):
        m = mg.MGR(precision=prec, **SOLVER)
        infos = []
        waits = {}
        for wi in range(a.warmup):
            if wi == a.warmup - 1:
                # host waits on the GPU (read-backs, synchronisations) of one setup and one solve
                w0 = mg.host_wait_count()
                m.setup(A, mk)
                w1 = mg.host_wait_count()
                x.zero_()
                m.fgmres(A, b, x, rtol=RTOL, restart=RESTART, maxit=MAXIT)
                waits = {"setup": w1 - w0, "solve": mg.host_wait_count() - w1}
            else:
                step(m)
        kt_full, dom = {}, None
        if profile:
            # one more untimed step with every kernel timed: the per-kernel table, and the choice of
            # the dominant solve kernel, whose launches alone are then timed inside the timed region
            # (recording every kernel there would add event overhead to the measured steps)
            m.profile(True)
            step(m)
            kt_full = {k: m.kernel_time(k) + (m.kernel_bytes(k), m.kernel_bytes_stored(k)) for k in KERNEL_NAMES}
            m.profile(False)
            solve = [k for k in SOLVE_KERNELS if kt_full[k][0] and kt_full[k][2]]
            dom = max(solve, key=lambda k: kt_full[k][1]) if solve else None
            # small systems replay the apply as a CUDA graph, which profiling turns off: their
            # dominant kernel is timed in the profiled step instead
            # (with the whole applications and the coarse end of the V-cycle as two scopes of their own)
            if dom and not flush_l2:
                m.profile(True, only=[dom, "mgr_apply", "amg_tail"])
        barrier()
        sampler = ClockSampler(local) if (profile and rank == 0) else None
        l0 = mg.launch_count()
        setup_ms = []
        if flush_l2:
            # small inputs: each step timed alone, after a write larger than L2
            junk = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for k in range(steps):
                junk.fill_(k & 0xFF)
                ev[k][0].record(stream)
                info = step(m)
                ev[k][1].record(stream)
                setup_ms.append(m.stats()["setup_ms"])
                infos.append(info)
            torch.cuda.synchronize()
            total = sum(e0.elapsed_time(e1) for e0, e1 in ev)
            del junk
        else:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                info = step(m)
                setup_ms.append(m.stats()["setup_ms"])
                infos.append(info)
            e1.record(stream)
            torch.cuda.synchronize()
            total = e0.elapsed_time(e1)
        launches = mg.launch_count() - l0
        clocks = sampler.stop() if sampler else None
        ms = _max(total) / steps
        if dom and flush_l2:
            kt_dom = (dom, kt_full[dom])
        else:
            kt_dom = (dom, m.kernel_time(dom) + (m.kernel_bytes(dom), m.kernel_bytes_stored(dom))) if dom else None
        live = {k: m.kernel_time(k) for k in ("mgr_apply", "amg_tail")} if (dom and not flush_l2) else {}
        mem = m.memory_bytes()
        L, na = m.levels()
        hier = {"mgr": [list(_shape(m, mg.MAT_LEVEL, l)) for l in range(L + 1)],
                "amg": [list(_shape(m, mg.MAT_AMG_A, k)) for k in range(na)]}
        m.close()
        return ms, infos, setup_ms, launches, clocks, (kt_full, kt_dom, live), mem, hier, waits

    # GB300's FP64 FMA rate, measured (the roofline of the FP64-bound Krylov kernels), with the SM
    # clock sampled while the probe runs
    fp64_probe = None
    if rank == 0:
        sampler = ClockSampler(local)
        mg.probe_fp64_fma(4096, 2)
        g, ms_l = mg.probe_fp64_fma(4096, 40)
        ck = sampler.stop()
        fp64_probe = {"gfma_per_s": g, "ms_per_launch": ms_l, "launches": 40,
                      "kernel": "8 independent FMA chains of 4096 per thread, full-occupancy grid",
                      "clocks": ck}
        if ck and ck.get("sm_mhz"):
            fp64_probe["fma_per_clock_per_sm"] = g * 1e9 / (ck["sm_mhz"] * 1e6) / torch.cuda.get_device_properties(
                local).multi_processor_count
    ms, infos, setup_ms, launches, clocks, (kt, kt_dom, live), mem, hier, waits = timed("mixed", a.steps, profile=True)
    xr = x.cpu().numpy()
    relres = float(np.linalg.norm(b_h - p.to_scipy() @ xr) / np.linalg.norm(b_h))
    out = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
           "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64", "data": "synthetic", "config": config,
           "iterations": infos[-1]["iterations"], "setup_ms": statistics.mean(setup_ms),
           "solve_ms": statistics.mean(i["solve_ms"] for i in infos), "relres_true": relres,
           "solves_per_s_all_gpus": a.gpus * 1000.0 / ms, "gpu_launches": int(launches),
           "host_waits_per_step": waits,
           "device_memory_gb": mem / 1e9, "hierarchy_rows_nnz": hier}
    # per-kernel achieved algorithmic bandwidth of the solve kernels, from the untimed profiled step
    # (bytes declared by the library for each launch, divided by the CUDA-event time of the launches);
    # frac counts a 4-byte column index per sparse entry, frac_stored the column form the sliced
    # layouts hold (one-byte codes or 16-bit offsets where they apply)
    peak, peak_kind = _peaks()
    rk = {}
    for k in SOLVE_KERNELS:
        n_k, t_k, by_k, bs_k = kt.get(k, (0, 0.0, 0.0, 0.0))
        if n_k and by_k and t_k > 0:
            gbs = by_k / (t_k * 1e-3) / 1e9
            rk[k] = {"launches": n_k, "ms": t_k, "achieved_gbs": gbs, "frac": gbs / peak,
                     "frac_stored": bs_k / (t_k * 1e-3) / 1e9 / peak, "bytes_per_launch": by_k / n_k}
    out["kernel_bandwidth"] = rk
    # the whole preconditioner application: the algorithmic bytes of every apply kernel of the
    # profiled step, per application, over the time of whole applications inside the timed region
    # (one event pair per application: no per-kernel events between the launches)
    app = [k for k in rk if k not in ("bsr3_spmv_f64", "mdot", "mupdate")]
    n_app = kt.get("mgr_apply", (0,))[0]
    if app and n_app:
        t_prof = sum(kt[k][1] for k in app)
        by_a, bs_a = sum(kt[k][2] for k in app) / n_app, sum(kt[k][3] for k in app) / n_app
        n_live, t_live = live.get("mgr_apply", (0, 0.0))
        ra = {"kernels": "mgr_apply (global relaxation, level residuals, F-relaxation, restriction, interpolation, "
                         "AMG V-cycle)", "bound": "hbm", "bytes_per_apply": by_a, "bytes_stored_per_apply": bs_a,
              "ms_per_apply_kernels_profiled": t_prof / n_app, "peak": peak, "unit": "GB/s", "peak_source": peak_kind}
        if n_live:
            us = t_live / n_live * 1e3
            ra.update({"us_per_apply": us, "applies_timed": n_live, "achieved": by_a / (us * 1e-6) / 1e9,
                       "frac": by_a / (us * 1e-6) / 1e9 / peak, "frac_stored": bs_a / (us * 1e-6) / 1e9 / peak})
            n_t, t_t = live.get("amg_tail", (0, 0.0))
            if n_t:
                ra["us_per_apply_amg_tail"] = t_t / n_t * 1e3
        out["roofline_apply"] = ra
    sb = {}
    for k in SETUP_KERNELS:
        n_k, t_k, by_k, _ = kt.get(k, (0, 0.0, 0.0, 0.0))
        if n_k and by_k and t_k > 0:
            sb[k] = {"calls": n_k, "ms": t_k, "achieved_gbs": by_k / (t_k * 1e-3) / 1e9}
    out["setup_bandwidth"] = sb
    # the setup's products (the top kernels of the launch list) are bound by instruction issue in
    # shared-memory hashing, not by HBM: their algorithmic rate is reported against HBM for scale only
    rap = [k for k in sb if k.startswith("rap_") or k == "spgemm_extpi"]
    if rap:
        t_s = sum(sb[k]["ms"] for k in rap)
        by_s = sum(kt[k][2] for k in rap)
        out["roofline_setup"] = {"kernel": "spgemm (k_spgemm_tiny, k_spgemm_fused_chunk, k_spgemm_chunk_list)",
                                 "bound": "issue", "ms": t_s, "achieved_gbs": by_s / (t_s * 1e-3) / 1e9,
                                 "frac_of_hbm": by_s / (t_s * 1e-3) / 1e9 / peak, "calls": sum(sb[k]["calls"] for k in rap)}
    if kt_dom:
        k, (n_k, t_k, by_k, _) = kt_dom
        per_launch = by_k / n_k
        us = t_k / n_k * 1e3
        achieved = per_launch / (us * 1e-6) / 1e9
        tr = TRAFFIC.get(k)
        if k in FP64_BOUND and fp64_probe:
            # bound by GB300's FP64 FMA rate (ncu: FP64 pipe ~87-91 % active), reported against the
            # rate measured by the FMA-chain probe in this run, with the HBM fraction beside it
            fma_launch = 9.0 * p.colind.shape[0] if k == "bsr3_spmv_f64" else per_launch / 8.0
            fma = fma_launch / (us * 1e-6) / 1e9
            out["roofline"] = {"kernel": k, "bound": "alu", "achieved": fma, "peak": fp64_probe["gfma_per_s"],
                               "unit": "GFMA/s", "frac": fma / fp64_probe["gfma_per_s"],
                               "peak_source": "measured in this run: FP64 FMA-chain probe (mgr_probe_fp64_fma)",
                               "fma_per_launch": fma_launch, "traffic": tr * per_launch if tr else None,
                               "bytes_per_launch": per_launch, "hbm_achieved_gbs": achieved,
                               "hbm_frac": achieved / peak, "hbm_peak_source": peak_kind,
                               "avg_launch_us": us, "launches": n_k}
        else:
            out["roofline"] = {"kernel": k, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                               "frac": achieved / peak, "peak_source": peak_kind,
                               "traffic": tr * per_launch if tr else None, "bytes_per_launch": per_launch,
                               "avg_launch_us": us, "launches": n_k}
    if fp64_probe:
        out["fp64_probe"] = fp64_probe
    out["kernel_ms_one_step"] = {k: v[1] for k, v in kt.items() if v[0]}
    if clocks:
        out["clocks"] = clocks
    if not a.no_fp64:
        ms64, infos64, setup64, _, _, _, _, _, _ = timed("fp64", max(1, a.steps))
        out["fp64"] = {"ms_per_step": ms64, "iterations": infos64[-1]["iterations"],
                       "setup_ms": statistics.mean(setup64), "solve_ms": statistics.mean(i["solve_ms"] for i in infos64),
                       "speedup_mixed_vs_fp64": ms64 / ms}
    if not a.no_e2e:
        # end to end through the public API with host buffers: pinned host -> device copies of the
        # matrix, marker and rhs, setup, solve, and the solution back to the host, every step
        hp = {k: torch.as_tensor(v).pin_memory() for k, v in
              dict(rp=p.rowptr, ci=p.colind, v=p.values, mk=p.cf_marker, b=b_h).items()}
        xh = torch.empty(p.n, dtype=torch.float64).pin_memory()
        m = mg.MGR(precision="mixed", **SOLVER)
        h2d = sum(t.numel() * t.element_size() for t in hp.values())
        d2h = xh.numel() * xh.element_size()

        def e2e_step():
            Ad = mg.BSR3(hp["rp"].cuda(non_blocking=True), hp["ci"].cuda(non_blocking=True),
                         hp["v"].cuda(non_blocking=True))
            mkd = hp["mk"].cuda(non_blocking=True)
            bd = hp["b"].cuda(non_blocking=True)
            m.setup(Ad, mkd)
            xd, _ = m.fgmres(Ad, bd, rtol=RTOL, restart=RESTART, maxit=MAXIT)
            xh.copy_(xd, non_blocking=True)

        for _ in range(a.warmup):
            e2e_step()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        m.close()
        out["e2e"] = {"value": _max(e0.elapsed_time(e1)) / a.steps, "unit": "ms",
                      "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        it_full = (out.get("fp64") or {}).get("iterations") or out["iterations"]
        if a.cpu_full:
            r = run_oracle_sample(cfg, max(cfg.nx, cfg.ny, cfg.nz))
            v = (r["setup_s"] + r["solve_s"]) * 1e3
            sample = (f"the full {a.workload} instance, FP64 oracle on 1 core: setup {r['setup_s']:.1f} s + solve "
                      f"{r['solve_s']:.1f} s ({r['iterations']} iterations)")
        else:
            v, sample, r = oracle_estimate(cfg, a.workload, 64, it_full)
        out["cpu_baseline"] = {"value": v, "unit": "ms", "cores": 1, "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
