#!/usr/bin/env python3
"""Benchmark: FGMRES + p-multilevel V-cycle solve of the statically condensed
HHO Stokes system on one GB300 (arXiv 2009.13840, Secs. 3-4).

Workload (one "step" = one full solve to a 1e-8 relative residual with the
assembled operator and RHS resident in HBM): 128 x 128 squares split into
32768 triangles, interior vertices jittered by +-0.2h (SplitMix64 seed 0),
Dirichlet on x=0, y=0, y=1 and Neumann on x=1, manufactured field
u = (sin(pi x) cos(pi y), -cos(pi x) sin(pi y)), p = sin(2 pi x) sin(2 pi y),
k = 3, v-cond static condensation, p-levels 3-2-1-0.  The headline solve uses
the mixed-precision V-cycle (FP32 level operators, smoother vectors, dot
products and coarse solve; FP64 only for stored scalars) inside FP64 FGMRES;
the plain FP64 V-cycle is timed on the same problem for the speedup.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload family instead.  ``--probe-spmv`` only
runs three FP32 and one FP64 level-0 operator launches on the workload (the
small command for ncu captures of the roofline kernel) and prints nothing.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FGMRES+p-MG time & DOFs/s to 1e-8 rel. residual; V-cycle GB/s vs HBM peak"
UNIT = "DOF/s"
# DRAM bytes (read + write) of one FP32 level-0 operator launch on the default
# workload, from the ncu capture summarised in
# profiles/k_spmv_b_level0_tri128_k3_vcond.md (kernel unchanged since)
SPMV_F32_TRAFFIC = {("tri", 128, 3, "v"): 144323072 + 3200512}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--k", type=int, default=3)
    ap.add_argument("--cond", default="v", choices=["v", "vp"])
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--sample-n", type=int, default=24, help="mesh size of the CPU-oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"], help="V-cycle precision of the headline")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--probe-spmv", action="store_true", help="three FP32 and one FP64 level-0 operator launches")
    ap.add_argument("--coarse-fp32", type=int, default=1, choices=[0, 1],
                    help="FP32 coarse solve inside the FP32 V-cycle (velocity-only condensation default)")
    return ap.parse_args()


def workload(n, k, cond):
    from synthetic import tri_mesh, fields
    mesh = tri_mesh(n, jitter=0.2, seed=0, neumann_sides=(1,))
    return mesh, fields.TrigStokes2D(), f"tri{n}x{n}-jit0.2-seed0-mixedBC k={k} {cond}-cond levels {k}..0"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """Samples nvidia-smi every 200 ms while active."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def oracle_sample(n_s, k, cond, rtol):
    """The oracle as it stands on a bounded sample: returns (DOF/s, ndof, its, seconds)."""
    from oracle.hho import HHO
    from oracle.pmg import PMG, fgmres
    mesh, fld, _ = workload(n_s, k, cond)
    h = HHO(mesh, k, cond)
    rhs = h.assemble_rhs(*h.data_values(fld))
    pmg = PMG(h, list(range(k, -1, -1)))
    t0 = time.perf_counter()
    x, its, rr = fgmres(h.S, pmg.apply, rhs, rtol=rtol, null=h.null_vector())
    dt = time.perf_counter() - t0
    return h.ndof / dt, h.ndof, its, dt


def cpu_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    vals = []
    info = None
    for i in range(args.warmup + args.steps):
        v, ndof, its, dt = oracle_sample(args.sample_n, args.k, args.cond, args.rtol)
        if i >= args.warmup:
            vals.append(v)
            info = (ndof, its, dt)
    value = float(np.mean(vals))
    ndof, its, dt = info
    sample = (f"oracle FGMRES+p-MG solve on tri{args.sample_n}x{args.sample_n} (same family as the "
              f"workload, {ndof} DOFs, {its} iterations, {dt:.2f} s per solve); setup excluded")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload(args.n, args.k, args.cond)[2], "sample": f"tri{args.sample_n}"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def spmv_bytes(ctx, level=0, value_bytes=8):
    """Algorithmic bytes of one level SpMV: stored values, column indices, x read, y written."""
    r, c, v = ctx.level_coo(level)
    n = ctx.ndof(level)
    m = ctx.mesh
    nf, ne = m.n_face, m.n_elem
    N = np.diff(m.elem_face_ptr)
    fe = m.face_elem
    # face slots per face row: 1 + sum over its elements of (|F_T| - 1)
    nsl = 1 + np.where(fe[:, 0] >= 0, N[fe[:, 0]] - 1, 0) + np.where(fe[:, 1] >= 0, N[np.maximum(fe[:, 1], 0)] - 1, 0)
    idx_bytes = 4 * (int(nsl.sum()) + nf + 2 * nf + int(N.sum()) + ne)
    return v.size * value_bytes + idx_bytes + 2 * n * value_bytes


def run_ours(args):
    import torch
    import torch.distributed as dist
    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2009_13840_gb300 import build, hho
    build.build()
    mesh, fld, wname = workload(args.n, args.k, args.cond)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = hho.Context(mesh, args.k, args.cond, stream=stream)
        f, gD, gN = hho.data_arrays(ctx, fld)
        ctx.assemble(f, gD, gN)
        degrees = list(range(args.k, -1, -1))
        ndof = ctx.ndof(0)
        if args.probe_spmv:
            ctx.pmg_setup(degrees, smooth_its=2, prec="fp32")
            xp = torch.randn(ndof, dtype=torch.float64, device="cuda")
            yp = torch.empty_like(xp)
            xf, yf = xp.float(), torch.empty(ndof, dtype=torch.float32, device="cuda")
            for _ in range(3):
                ctx.spmv_f32(0, xf, yf)
            ctx.spmv(0, xp, yp)
            torch.cuda.synchronize()
            ctx.close()
            return
        x = torch.empty(ndof, dtype=torch.float64, device="cuda")
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

        def timed_solves(steps, tag, clocks=None):
            times, infos = [], []
            for _ in range(steps):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.nvtx.range_push(tag)
                e0.record(stream)
                info = ctx.solve(x, rtol=args.rtol)
                e1.record(stream)
                e1.synchronize()
                torch.cuda.nvtx.range_pop()
                times.append(e0.elapsed_time(e1))
                infos.append(info)
            return float(np.mean(times)), infos

        # plain FP64 V-cycle on the same problem (for the speedup of the mixed one)
        fp64 = None
        if args.prec == "fp32" and not args.no_fp64_compare:
            ctx.pmg_setup(degrees, smooth_its=2, prec="fp64")
            for _ in range(args.warmup):
                ctx.solve(x, rtol=args.rtol)
            ms64, inf64 = timed_solves(args.steps, "fp64_step")
            fp64 = {"ms_per_solve": ms64, "fgmres_iterations": inf64[-1]["iterations"],
                    "rel_residual": inf64[-1]["rel_residual"], "dof_per_s": ndof / (ms64 / 1e3)}
        ctx.set_option("coarse_fp32", args.coarse_fp32 if args.prec == "fp32" else 0)
        ctx.pmg_setup(degrees, smooth_its=2, prec=args.prec)
        for _ in range(args.warmup):
            info = ctx.solve(x, rtol=args.rtol)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        l0 = ctx.launch_count()
        with Clocks(local) as clk:
            ms, infos = timed_solves(args.steps, "timed_step")
            torch.cuda.synchronize()
        launches = ctx.launch_count() - l0
        if ws > 1:
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        value = ws * ndof / (ms / 1e3)

        # dominant kernel: the level-0 operator of the V-cycle, timed live with CUDA events on its stream
        def time_kernel(fn, reps=20):
            kt = []
            for i in range(reps + 3):
                flush.fill_(2.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                if i >= 3:
                    kt.append(e0.elapsed_time(e1))
            return float(np.mean(kt))

        xs = torch.randn(ndof, dtype=torch.float64, device="cuda")
        ys = torch.empty_like(xs)
        ms64_k = time_kernel(lambda: ctx.spmv(0, xs, ys))
        nb64 = spmv_bytes(ctx, 0, 8)
        peak, peak_kind = peaks()
        if args.prec == "fp32":
            xs32, ys32 = xs.float(), torch.empty(ndof, dtype=torch.float32, device="cuda")
            ms_k = time_kernel(lambda: ctx.spmv_f32(0, xs32, ys32))
            nbytes = spmv_bytes(ctx, 0, 4)
            kname = "k_spmv_b<float> (level 0, V-cycle operator, FP32)"
        else:
            ms_k, nbytes, kname = ms64_k, nb64, "k_spmv_b<double> (level 0)"
        achieved = nbytes / (ms_k / 1e3) / 1e9
        # end-to-end through the public API with host buffers
        hf, hgD, hgN = f.cpu().pin_memory(), gD.cpu().pin_memory(), gN.cpu().pin_memory()
        hx = torch.empty(ndof, dtype=torch.float64).pin_memory()
        df, dgD, dgN = torch.empty_like(f), torch.empty_like(gD), torch.empty_like(gN)
        et = []
        for i in range(args.warmup + args.steps):
            flush.fill_(3.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            df.copy_(hf, non_blocking=True)
            dgD.copy_(hgD, non_blocking=True)
            dgN.copy_(hgN, non_blocking=True)
            ctx.assemble(df, dgD, dgN)
            ctx.solve(x, rtol=args.rtol)
            hx.copy_(x, non_blocking=True)
            stream.synchronize()
            if i >= args.warmup:
                et.append(time.perf_counter() - t0)
        e2e_s = float(np.mean(et))
        if ws > 1:
            t = torch.tensor([e2e_s], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, nd, its, dt = oracle_sample(args.sample_n, args.k, args.cond, args.rtol)
        cpu = {"value": v, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
               "sample": f"oracle FGMRES+p-MG solve on tri{args.sample_n}x{args.sample_n} of the same family "
                         f"({nd} DOFs, {its} its, {dt:.2f} s); setup excluded"}
    if rank == 0:
        last = infos[-1]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 FGMRES + f32 V-cycle" if args.prec == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": wname, "vcycle_precision": args.prec,
                       "coarse_precision": "fp32" if (args.prec == "fp32" and args.coarse_fp32) else "fp64",
                       "dofs": ndof,
                       "fgmres_iterations": last["iterations"], "coarse_iterations": last["coarse_iterations"],
                       "rel_residual_fp64": last["rel_residual"], "fp64_vcycle": fp64,
                       "speedup_vs_fp64_vcycle": (fp64["ms_per_solve"] / ms) if fp64 else None,
                       "l2": "flushed between steps (512 MiB write)", "parallelism": "replicas" if ws > 1 else "single"},
            "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": (SPMV_F32_TRAFFIC.get(("tri", args.n, args.k, args.cond))
                                     if args.prec == "fp32" else None),
                         "bytes_per_launch": nbytes, "ms_per_launch": ms_k,
                         "fp64_outer_spmv": {"achieved": nb64 / (ms64_k / 1e3) / 1e9, "bytes_per_launch": nb64,
                                             "ms_per_launch": ms64_k}},
            "cpu_baseline": cpu,
            "e2e": {"value": ws * ndof / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int((f.numel() + gD.numel() + gN.numel()) * 8),
                    "d2h_bytes_per_step": int(ndof * 8)},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
