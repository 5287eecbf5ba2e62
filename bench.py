#!/usr/bin/env python3
"""Benchmark: FGMRES + p-multilevel V-cycle solve of the statically condensed
HHO Stokes system on one GB300 (arXiv 2009.13840, Secs. 3-4).

Default workload (one "step" = one full solve to a 1e-8 relative residual with
the assembled operator and right-hand side resident in HBM): the unit cube
split into 32^3 hexahedra with planar faces, grid planes jittered by +-0.15h
(SplitMix64 seed 0), all-Dirichlet, manufactured field
u = curl(sin(pi x) sin(pi y) sin(pi z) (1,1,1)), p = cos(pi x) cos(pi y)
cos(pi z), k = 3, velocity-pressure (v&p) static condensation, p-levels
3-2-1-0 (3.07 M condensed unknowns).  The headline solve uses the
mixed-precision V-cycle (FP32 level operators, smoother vectors and
arithmetic) inside FP64 FGMRES; the plain FP64 V-cycle is timed on the same
problem for the speedup.  Other workloads: --workload c2 (128 x 128 jittered
triangles, mixed boundary conditions, k = 3, velocity-only condensation),
c1 (16 x 16 quadrilaterals, all-Dirichlet, k = 3, v&p, FP64), sweep (the
128 x 128 triangle mesh over k = 1..5, both condensations, FP64 and FP32
V-cycles; one JSON line per case), batch, learned.

Prints one JSON line (sweep: one per case).  ``--impl reference`` times the
FP64 CPU oracle on a bounded sample of the same workload family instead.
``--probe-spmv`` only runs three FP32 and one FP64 level-0 operator launches on
the workload (the small command for ncu captures of the roofline kernel) and
prints nothing.
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
L2_BYTES = 129 * 1024 * 1024  # GB300 L2
UNIT = "DOF/s"
# DRAM bytes (read + write) of one FP32 level-0 operator launch, from the ncu
# captures summarised under profiles/ (kernels unchanged since); keyed by
# (mesh, n, k, condensation).  The 32^3 entries are the 16^3 captures (v&p:
# 516.5 MB per launch, 1.035x its algorithmic bytes; HHO-hp: 894.1 MB, 1.022x)
# scaled by the ratio of the algorithmic bytes (7.976): the full-size workload is
# too large for a multi-pass capture.
SPMV_F32_TRAFFIC = {("tri", 128, 3, "v"): 144286208 + 3245056, ("hex", 32, 3, "vp"): 4119717980,
                    ("hex", 32, 3, "hp"): round((892412928 + 1694208) * 6979174400 / 874983424)}

# the named workloads (the paper's configurations and the comparison schemes); command-line values override
SPECS = {
    "c3": dict(mesh="hex", n=32, k=3, cond="vp", prec="fp32", coarse_fp32=1, sample_n=4),
    "c2": dict(mesh="tri", n=128, k=3, cond="v", prec="fp32", coarse_fp32=1, sample_n=24),
    "c1": dict(mesh="quad", n=16, k=3, cond="vp", prec="fp64", coarse_fp32=0, sample_n=16),
    "learned": dict(mesh="hex", n=48, k=3, cond="vp", prec="fp32", coarse_fp32=1, sample_n=4),
    # HHO-hp (Scheme 2) on the C2 and C3 meshes
    "hp2": dict(mesh="tri", n=128, k=3, cond="hp", prec="fp32", coarse_fp32=1, sample_n=24),
    "hp3": dict(mesh="hex", n=32, k=3, cond="hp", prec="fp32", coarse_fp32=1, sample_n=4),
    # uncondensed HHO-dp on the C2 mesh (the reference point of the condensation gains), block ILU(0) smoother
    "unc2": dict(mesh="tri", n=128, k=3, cond="unc", prec="fp32", coarse_fp32=1, sample_n=16, smoother="ilu"),
    # the DG scheme (Scheme 3) on 40 x 40 jittered triangles, k=3: its coarse level (k=0, 9600 unknowns) is the
    # largest the dense coarse solve takes
    "dg2": dict(mesh="tri", n=40, k=3, cond="dg", prec="fp32", coarse_fp32=1, sample_n=10),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3",
                    choices=["c3", "c2", "c1", "sweep", "batch", "learned", "hp2", "hp3", "unc2", "dg2"],
                    help="c3: 32^3 jittered hexahedra, k=3, v&p (default); c2: 128x128 jittered triangles, k=3, "
                         "v-cond; c1: 16x16 quadrilaterals, k=3, v&p, FP64; sweep: the c2 mesh over k=1..5, both "
                         "condensations, FP64 and FP32 V-cycles; batch: many independent small problems; learned: "
                         "the learned smoother against the plain one; hp2 / hp3: HHO-hp (Scheme 2) on the c2 "
                         "triangle mesh (k=3) and the c3 hexahedral mesh (k=3); unc2: uncondensed HHO-dp on the c2 "
                         "mesh (k=3, block ILU(0) smoother); dg2: the DG scheme (BR2, Scheme 3) on 40x40 jittered "
                         "triangles (k=3)")
    ap.add_argument("--mesh", default=None, choices=["tri", "hex", "quad"],
                    help="override the workload's mesh family (tri: n x n squares split into triangles; hex: n^3 "
                         "jittered hexahedra; quad: n x n quadrilaterals)")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--k", type=int, default=None)
    ap.add_argument("--cond", default=None, choices=["v", "vp", "hp", "unc", "dg"],
                    help="Scheme 1 with velocity-only (v) or velocity-pressure (vp) condensation, Scheme 2 "
                         "(HHO-hp, hybrid pressure, every element unknown condensed), Scheme 1 uncondensed (unc), "
                         "or the DG scheme (dg, Scheme 3)")
    ap.add_argument("--prec", default=None, choices=["fp32", "fp64"], help="V-cycle precision of the headline")
    ap.add_argument("--coarse-fp32", type=int, default=None, choices=[0, 1],
                    help="FP32 coarse solve inside the FP32 V-cycle")
    ap.add_argument("--smoother", default=None, choices=["jacobi", "ilu"],
                    help="preconditioner of the smoother's GMRES: block Jacobi or block ILU(0)")
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--sample-n", type=int, default=None, help="mesh size of the CPU-oracle sample")
    ap.add_argument("--oracle-faces", type=int, default=12,
                    help="faces (DG: elements) of the full-size solution whose residual rows the oracle recomputes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--probe-spmv", action="store_true", help="three FP32 and one FP64 level-0 operator launches")
    ap.add_argument("--profile-region", action="store_true",
                    help="bracket the timed solves with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--learned-train-n", type=int, default=None,
                    help="mesh size the learned smoother is trained on (default 24 for hexahedra, 32 for triangles)")
    ap.add_argument("--learned-samples", type=int, default=100000, help="training pairs (one per face and vector)")
    ap.add_argument("--batch-n", type=int, default=256, help="problems in the batched workload")
    ap.add_argument("--batch-seed", type=int, default=12345)
    ap.add_argument("--batch-cond", default="v", choices=["v", "vp"])
    ap.add_argument("--solve-graph", type=int, default=0, choices=[0, 1],
                    help="1: the single solve runs as one captured CUDA graph with device-side convergence tests")
    ap.add_argument("--batch-graph", type=int, default=1, choices=[0, 1],
                    help="1: each group's batched solve is one captured CUDA graph with device-side control; "
                         "0: host-driven FGMRES loop")
    ap.add_argument("--batch-compare", type=int, default=16,
                    help="problems of the batch also solved one by one for the batching speedup (0: skip)")
    args = ap.parse_args()
    spec = SPECS.get(args.workload, SPECS["c2"] if args.workload == "sweep" else SPECS["c3"])
    if args.workload == "learned" and args.mesh == "tri":  # the 2D variant of the learned workload
        spec = dict(SPECS["c2"], n=128)
    for key in ("mesh", "n", "k", "cond", "prec", "sample_n"):
        if getattr(args, key) is None:
            setattr(args, key, spec[key])
    if args.coarse_fp32 is None:
        args.coarse_fp32 = spec["coarse_fp32"]
    if args.smoother is None:
        args.smoother = spec.get("smoother", "jacobi")
    return args


def workload(n, k, cond, mesh_kind):
    """(mesh, field, name) of a workload family member (seeded, synthetic)."""
    from synthetic import tri_mesh, hex_mesh, quad_mesh, fields
    if mesh_kind == "hex":
        mesh = hex_mesh(n, jitter=0.15, seed=0)
        return mesh, fields.CurlStokes3D(), f"hex{n}^3-jit0.15-seed0-allDirichlet k={k} {cond}-cond levels {k}..0"
    if mesh_kind == "quad":
        mesh = quad_mesh(n, jitter=0.0)
        return mesh, fields.TrigStokes2D(), f"quad{n}x{n}-uniform-allDirichlet k={k} {cond}-cond levels {k}..0"
    mesh = tri_mesh(n, jitter=0.2, seed=0, neumann_sides=(1,))
    scheme = "DG-BR2 (Scheme 3)" if cond == "dg" else f"{cond}-cond"
    return mesh, fields.TrigStokes2D(), f"tri{n}x{n}-jit0.2-seed0-mixedBC k={k} {scheme} levels {k}..0"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(v, ws, device):
    """Max of a per-rank scalar over the process group (the slowest rank's
    time); v itself when ws == 1."""
    if ws <= 1:
        return float(v)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ws, seconds):
    """Whole-job throughput of ws replicas: the units all ranks processed over
    the slowest rank's time."""
    return ws * units_per_rank / seconds


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


def one_thread():
    """Context limiting the BLAS pools to one thread: the oracle's loops are
    serial Python and its sparse products single-threaded, so the CPU baseline
    is stated as what it is, a one-core run."""
    try:
        import threadpoolctl
        return threadpoolctl.threadpool_limits(1)
    except Exception:
        import contextlib
        return contextlib.nullcontext()


def oracle_disc(mesh, k, cond):
    """The oracle's discretisation: Scheme 1 (v, vp) or Scheme 2 (hp)."""
    if cond == "hp":
        from oracle.hho_hp import HHOhp
        return HHOhp(mesh, k)
    if cond == "dg":
        from oracle.dg import DG
        return DG(mesh, k)
    from oracle.hho import HHO
    return HHO(mesh, k, cond)


def oracle_sample(args, steps=1):
    """The oracle as it stands on a bounded sample of the workload family: the
    hierarchy is built once (timed as setup), then `steps` FGMRES solves are
    timed.  Returns (DOF/s of the last solve, ndof, its, solve seconds, setup
    seconds)."""
    from oracle.pmg import PMG, fgmres
    n_s = args.sample_n
    mesh, fld, _ = workload(n_s, args.k, args.cond, args.mesh)
    with one_thread():
        t0 = time.perf_counter()
        h = oracle_disc(mesh, args.k, args.cond)
        rhs = h.assemble_rhs(*h.data_values(fld))
        pmg = PMG(h, list(range(args.k, -1, -1)), smoother=args.smoother)
        t_setup = time.perf_counter() - t0
        rates = []
        for _ in range(max(1, steps)):
            t0 = time.perf_counter()
            x, its, rr = fgmres(h.S, pmg.apply, rhs, rtol=args.rtol, null=h.null_vector())
            dt = time.perf_counter() - t0
            rates.append((h.ndof / dt, dt))
    return rates, h.ndof, its, t_setup


def sample_name(args):
    return {"hex": f"hex{args.sample_n}^3", "quad": f"quad{args.sample_n}x{args.sample_n}",
            "tri": f"tri{args.sample_n}x{args.sample_n}"}[args.mesh]


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    rates, ndof, its, t_setup = oracle_sample(args, steps=args.warmup + args.steps)
    timed = rates[args.warmup:] or rates[-1:]
    value = float(np.mean([r[0] for r in timed]))
    dt = float(np.mean([r[1] for r in timed]))
    full = workload(args.n, args.k, args.cond, args.mesh)
    sample = (f"oracle FGMRES+p-MG solve on {sample_name(args)} (same family as the workload; {ndof} DOFs, "
              f"{its} iterations, {dt:.2f} s per solve, {t_setup:.1f} s setup excluded), one thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": full[2], "sample": sample_name(args)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _dimP(nv, deg):
    if deg < 0:
        return 0
    return {0: 1, 1: deg + 1, 2: (deg + 1) * (deg + 2) // 2, 3: (deg + 1) * (deg + 2) * (deg + 3) // 6}[nv]


def level_counts(mesh, k_l, cond):
    """(n, stored values z, index bytes, Jacobi values J, b, nP) of the level of
    degree k_l: the face-block operator of the condensed system (stored blocks
    of every face row and element row) and the block-Jacobi data."""
    d = mesh.dim
    if cond == "dg":  # element blocks of (d+1) n_E; slot 0 the element, then its neighbours across interior faces
        b, ne = (d + 1) * _dimP(d, k_l), mesh.n_elem
        fe = mesh.face_elem
        inner = fe[(fe[:, 0] >= 0) & (fe[:, 1] >= 0)]
        nsl = 1 + np.bincount(inner.ravel(), minlength=ne)
        return ne * b, b * b * int(nsl.sum()), 4 * (int(nsl.sum()) + ne), ne * b * b, b, 0
    b = (d + 1 if cond == "hp" else d) * _dimP(d - 1, k_l)  # HHO-hp: face pressure as one more component
    nP = 0 if cond == "hp" else 1 if cond == "vp" else (d + 1) * _dimP(d, k_l) if cond == "unc" else _dimP(d, k_l)
    nf, ne = mesh.n_face, mesh.n_elem
    N = np.diff(mesh.elem_face_ptr)
    fe = mesh.face_elem
    nsl = 1 + np.where(fe[:, 0] >= 0, N[fe[:, 0]] - 1, 0) + np.where(fe[:, 1] >= 0, N[np.maximum(fe[:, 1], 0)] - 1, 0)
    z = b * b * int(nsl.sum()) + 2 * b * nP * int(N.sum()) + ne * nP * nP
    idx = 4 * (int(nsl.sum()) + nf + 2 * nf + int(N.sum()) + ne)
    J = nf * b * b + ne * nP * nP
    return nf * b + ne * nP, z, idx, J, b, nP


def spmv_bytes(mesh, k_l, cond, value_bytes):
    """Algorithmic bytes of one level operator product: stored values, column
    indices, x read, y written."""
    n, z, idx, _, _, _ = level_counts(mesh, k_l, cond)
    return z * value_bytes + idx + 2 * n * value_bytes


def vcycle_bytes(mesh, degrees, cond, s, coarse_values, coarse_s, m=2, smoother="jacobi"):
    """Algorithmic bytes of one V-cycle (Algorithm MG_V with m GMRES smoothing
    steps): per level above the coarse one (2m+3) operator products (pre/post
    Arnoldi steps, the post-smoother's initial residual, the fused defect),
    2m block-Jacobi applies (block ILU(0): 2m sweeps over factors the size of
    the level operator), 6m n_l vector passes of orthogonalisation and
    updates, 3 n_l of transfers; the coarse solve reads its stored operators
    once and two vectors."""
    tot = 0
    for kl in degrees[:-1]:
        n, z, idx, J, b, nP = level_counts(mesh, kl, cond)
        tot += (2 * m + 3) * (z * s + idx + 2 * n * s)
        if smoother == "ilu":  # block ILU(0) factors on the operator's block pattern, one sweep each way
            tot += 2 * m * (z * s + idx + 2 * n * s)
        else:
            tot += 2 * m * (J * s + 2 * n * s)
        tot += 6 * m * n * s + 3 * n * s
    nL = level_counts(mesh, degrees[-1], cond)[0]
    tot += coarse_values * coarse_s + 2 * nL * coarse_s
    return int(tot)


def oracle_check(mesh, k, cond, fld, x, b_gpu, Sx_gpu, faces, seed=0):
    """Rows of the full-size system recomputed by the oracle from its own local
    systems (oracle/sampled.py) at sampled faces and their elements' kept
    pressures: the oracle's residual b - S x of the GPU solution x on those
    rows against the GPU's own residual there, relative to each row's scale
    |b_i| + sum_T max|S_T| ||x_T||_1 (the bound that element Schur complements
    agreeing to a relative eps put on the rows: eps times it), and the
    oracle's residual on the rows scaled
    to the global right-hand side (||r_S|| / ||b|| * sqrt(n / |S|), an estimate
    of the global relative residual)."""
    from oracle.sampled import residual_rows, sample_interior_faces
    with one_thread():
        t0 = time.perf_counter()
        sf = sample_interior_faces(mesh, faces, seed)
        rows, r, b, sc = residual_rows(mesh, k, cond, fld, x, sf, with_scale=True)
        dt = time.perf_counter() - t0
    return dict({"faces": int(len(sf))}, **_row_check(rows, r, b, sc, b_gpu, Sx_gpu, dt))


def oracle_check_dg(mesh, k, fld, x, b_gpu, Sx_gpu, count, seed=0):
    """The DG scheme's counterpart of oracle_check: the oracle recomputes the
    element rows of `count` sampled elements (oracle/sampled.py, from the
    submesh of those elements and their neighbours)."""
    from oracle.sampled import residual_rows_dg, sample_elements
    with one_thread():
        t0 = time.perf_counter()
        se = sample_elements(mesh, count, seed)
        rows, r, b, sc = residual_rows_dg(mesh, k, fld, x, se, with_scale=True)
        dt = time.perf_counter() - t0
    return dict({"elements": int(len(se))}, **_row_check(rows, r, b, sc, b_gpu, Sx_gpu, dt))


def _row_check(rows, r, b, sc, b_gpu, Sx_gpu, dt):
    r_gpu = b_gpu[rows] - Sx_gpu[rows]
    return {"rows": int(len(rows)),
            "system_rows_max_diff_rel": float(np.max(np.abs(r - r_gpu) / sc)),
            "rhs_rows_max_diff_rel": float(np.abs(b - b_gpu[rows]).max() / np.abs(b_gpu[rows]).max()),
            "residual_rows_scaled": float(np.linalg.norm(r) / np.linalg.norm(b_gpu) * np.sqrt(len(b_gpu) / len(rows))),
            "seconds": dt}


def run_ours(args):
    import torch
    import torch.distributed as dist
    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2009_13840_gb300 import build, hho
    build.build()
    mesh, fld, wname = workload(args.n, args.k, args.cond, args.mesh)
    degrees = list(range(args.k, -1, -1))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = hho.Context(mesh, args.k, args.cond, stream=stream)
        torch.cuda.synchronize()
        t_setup = time.perf_counter() - t0
        ctx.set_option("solve_graph_single", args.solve_graph)
        f, gD, gN = hho.data_arrays(ctx, fld)  # input preparation (host evaluation of the data)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.assemble(f, gD, gN)
        torch.cuda.synchronize()
        t_asm = time.perf_counter() - t0
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

        def timed_solves(steps, tag):
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

        def time_on_stream(fn, reps):
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

        peak, peak_kind = peaks()
        # plain FP64 V-cycle on the same problem (for the speedup of the mixed one)
        fp64 = None
        if args.prec == "fp32" and not args.no_fp64_compare:
            ctx.set_option("smoother", 1 if args.smoother == "ilu" else 0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.pmg_setup(degrees, smooth_its=2, prec="fp64")
            torch.cuda.synchronize()
            t_pmg64 = time.perf_counter() - t0
            for _ in range(args.warmup):
                ctx.solve(x, rtol=args.rtol)
            ms64, inf64 = timed_solves(args.steps, "fp64_step")
            fp64 = {"ms_per_solve": ms64, "fgmres_iterations": inf64[-1]["iterations"],
                    "rel_residual": inf64[-1]["rel_residual"], "dof_per_s": ndof / (ms64 / 1e3),
                    "pmg_setup_s": t_pmg64}
        ctx.set_option("coarse_fp32", args.coarse_fp32 if args.prec == "fp32" else 0)
        ctx.set_option("smoother", 1 if args.smoother == "ilu" else 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.pmg_setup(degrees, smooth_its=2, prec=args.prec)
        torch.cuda.synchronize()
        t_pmg = time.perf_counter() - t0
        coarse = ctx.coarse_info()
        for _ in range(args.warmup):
            info = ctx.solve(x, rtol=args.rtol)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        l0 = ctx.launch_count()
        with Clocks(local) as clk:
            if args.profile_region:
                torch.cuda.profiler.start()
            ms, infos = timed_solves(args.steps, "timed_step")
            torch.cuda.synchronize()
            if args.profile_region:
                torch.cuda.profiler.stop()
        launches = ctx.launch_count() - l0
        ms = max_over_ranks(ms, ws, "cuda")
        value = whole_job_rate(ndof, ws, ms / 1e3)
        x_host = x.cpu().numpy()
        # the GPU's right-hand side and S x of the benched solution (for the oracle's row check)
        b_dev = torch.empty(ndof, dtype=torch.float64, device="cuda")
        ctx.assemble(f, gD, gN, b_dev)
        sx_dev = torch.empty(ndof, dtype=torch.float64, device="cuda")
        ctx.spmv(0, x, sx_dev)
        b_host, sx_host = b_dev.cpu().numpy(), sx_dev.cpu().numpy()
        del b_dev, sx_dev

        # V-cycle: algorithmic bytes over its time (graph replay, inputs larger than L2 or L2 flushed)
        s_val = 4 if args.prec == "fp32" else 8
        cs = 4 if (args.prec == "fp32" and args.coarse_fp32) else 8
        vbytes = vcycle_bytes(mesh, degrees, args.cond, s_val, coarse["values_per_solve"], cs, smoother=args.smoother)
        rv = torch.randn(ndof, dtype=torch.float64, device="cuda")
        zv = torch.empty_like(rv)
        ms_v = time_on_stream(lambda: ctx.vcycle(rv, zv), 10)
        vgbs = vbytes / (ms_v / 1e3) / 1e9

        # dominant kernel: the level-0 operator of the V-cycle, timed live with CUDA events on its stream
        xs = torch.randn(ndof, dtype=torch.float64, device="cuda")
        ys = torch.empty_like(xs)
        ms64_k = time_on_stream(lambda: ctx.spmv(0, xs, ys), 20)
        nb64 = spmv_bytes(mesh, args.k, args.cond, 8)
        if args.prec == "fp32":
            xs32, ys32 = xs.float(), torch.empty(ndof, dtype=torch.float32, device="cuda")
            ms_k = time_on_stream(lambda: ctx.spmv_f32(0, xs32, ys32), 20)
            nbytes = spmv_bytes(mesh, args.k, args.cond, 4)
            kname = ("k_spmv_b<30, float> (level 0, V-cycle operator, FP32, DG element blocks)" if args.cond == "dg"
                     else "k_spmv_v<float> (level 0, V-cycle operator, FP32, row-interleaved)")
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
        e2e_s = max_over_ranks(float(np.mean(et)), ws, "cuda")
        # error norms of the discrete solution against the manufactured field (Sec. 5.2.2 columns)
        loc = ctx.recover(x)
        xe = ctx.quad_nodes("elem").cpu().numpy()
        uex = torch.from_numpy(hho._chunked(fld.u, xe)).cuda()
        gex = torch.from_numpy(hho._chunked(fld.grad_u, xe)).cuda()
        pex = torch.from_numpy(hho._chunked(fld.p, xe)).cuda()
        err = ctx.errors(loc, uex, gex, pex)
        del loc, uex, gex, pex
    cpu = check = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rates, nd, its, ts = oracle_sample(args)
        v, dt = rates[-1]
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"oracle FGMRES+p-MG solve on {sample_name(args)} of the same family ({nd} DOFs against "
                         f"{ndof} in the workload, {its} its, {dt:.2f} s per solve, {ts:.1f} s setup excluded), "
                         f"one thread"}
        # the oracle recomputes residual rows of the full-size GPU solution at sampled faces (DG: elements)
        if args.cond == "dg":
            check = oracle_check_dg(mesh, args.k, fld, x_host, b_host, sx_host, args.oracle_faces)
        else:
            check = oracle_check(mesh, args.k, args.cond, fld, x_host, b_host, sx_host, args.oracle_faces)
    if rank == 0:
        last = infos[-1]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 FGMRES + f32 V-cycle" if args.prec == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": wname, "vcycle_precision": args.prec, "smoother": args.smoother,
                       "solve_control": "graph" if args.solve_graph else "host",
                       "coarse_precision": "fp32" if (args.prec == "fp32" and args.coarse_fp32) else "fp64",
                       "coarse_solver": coarse, "dofs": ndof, "coarse_dofs": ctx.ndof(len(degrees) - 1),
                       "fgmres_iterations": last["iterations"], "coarse_iterations": last["coarse_iterations"],
                       "rel_residual_fp64": last["rel_residual"], "fp64_vcycle": fp64,
                       "speedup_vs_fp64_vcycle": (fp64["ms_per_solve"] / ms) if fp64 else None,
                       "setup_s": {"hho_setup": t_setup, "assemble": t_asm, "pmg_setup": t_pmg,
                                   "total": t_setup + t_asm + t_pmg},
                       "solve_s": ms / 1e3,
                       "vcycle": {"ms": ms_v, "algorithmic_bytes": vbytes, "achieved_gbs": vgbs,
                                  "frac_of_measured_hbm": vgbs / peak},
                       "errors_vs_exact": err, "oracle_check": check,
                       "l2": "flushed between steps (512 MiB write); " + (
                           "operators larger than L2" if nbytes > L2_BYTES else
                           f"level-0 operator ({nbytes / 1e6:.0f} MB) smaller than L2: cold only after each flush"),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": (SPMV_F32_TRAFFIC.get((args.mesh, args.n, args.k, args.cond))
                                     if args.prec == "fp32" else None),
                         "bytes_per_launch": nbytes, "ms_per_launch": ms_k,
                         "fp64_outer_spmv": {"achieved": nb64 / (ms64_k / 1e3) / 1e9, "bytes_per_launch": nb64,
                                             "ms_per_launch": ms64_k}},
            "cpu_baseline": cpu,
            "e2e": {"value": whole_job_rate(ndof, ws, e2e_s), "unit": UNIT,
                    "h2d_bytes_per_step": int((f.numel() + gD.numel() + gN.numel()) * 8),
                    "d2h_bytes_per_step": int(ndof * 8)},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


def run_sweep(args):
    """The 128 x 128 triangle workload over k = 1..5, both condensations, FP64
    and FP32 V-cycles: one JSON line per case (solve time, DOF/s, iterations,
    true residual, setup times, V-cycle GB/s)."""
    import torch
    from paper_2009_13840_gb300 import build, hho
    build.build()
    peak, _ = peaks()
    stream = torch.cuda.Stream()
    for k in range(1, 6):
        for cond in ("v", "vp"):
            mesh, fld, wname = workload(args.n, k, cond, "tri")
            degrees = list(range(k, -1, -1))
            with torch.cuda.stream(stream):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ctx = hho.Context(mesh, k, cond, stream=stream)
                ctx.assemble(*hho.data_arrays(ctx, fld))
                torch.cuda.synchronize()
                t_setup = time.perf_counter() - t0
                ndof = ctx.ndof(0)
                x = torch.empty(ndof, dtype=torch.float64, device="cuda")
                for prec in ("fp64", "fp32"):
                    ctx.set_option("coarse_fp32", 1 if (prec == "fp32" and cond == "v") else 0)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    ctx.pmg_setup(degrees, smooth_its=2, prec=prec)
                    torch.cuda.synchronize()
                    t_pmg = time.perf_counter() - t0
                    for _ in range(args.warmup):
                        ctx.solve(x, rtol=args.rtol, maxit=2000)
                    ts, info = [], None
                    for _ in range(args.steps):
                        info = ctx.solve(x, rtol=args.rtol, maxit=2000)
                        ts.append(info["solve_ms"])
                    ms = float(np.mean(ts))
                    coarse = ctx.coarse_info()
                    rv = torch.randn(ndof, dtype=torch.float64, device="cuda")
                    zv = torch.empty_like(rv)
                    ctx.vcycle(rv, zv)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for _ in range(10):
                        ctx.vcycle(rv, zv)
                    e1.record(stream)
                    e1.synchronize()
                    ms_v = e0.elapsed_time(e1) / 10
                    s_val = 4 if prec == "fp32" else 8
                    cs = 4 if (prec == "fp32" and cond == "v") else 8
                    vb = vcycle_bytes(mesh, degrees, cond, s_val, coarse["values_per_solve"], cs)
                    print(json.dumps({"workload": wname, "k": k, "cond": cond, "vcycle_precision": prec, "dofs": ndof,
                                      "solve_ms": ms, "dof_per_s": ndof / (ms / 1e3),
                                      "fgmres_iterations": info["iterations"], "rel_residual": info["rel_residual"],
                                      "setup_s": t_setup, "pmg_setup_s": t_pmg, "vcycle_ms": ms_v,
                                      "vcycle_gbs": vb / (ms_v / 1e3) / 1e9,
                                      "vcycle_frac": vb / (ms_v / 1e3) / 1e9 / peak}), flush=True)
                ctx.close()


def oracle_batch_sample(probs, cond, rtol, budget_s=15.0):
    """The oracle as it stands on the first problems of the batch, solved one by
    one until about budget_s seconds of solves: returns (DOF/s, problems, DOFs, seconds)."""
    from oracle.hho import HHO
    from oracle.pmg import PMG, fgmres
    dofs, secs, done = 0, 0.0, 0
    ctl = one_thread()
    ctl.__enter__()
    for pr in probs:
        h = HHO(pr.mesh, pr.k, cond)
        rhs = h.assemble_rhs(*h.data_values(pr.field))
        pmg = PMG(h, list(range(pr.k, -1, -1)))
        t0 = time.perf_counter()
        fgmres(h.S, pmg.apply, rhs, rtol=rtol, null=h.null_vector())
        secs += time.perf_counter() - t0
        dofs += h.ndof
        done += 1
        if secs >= budget_s:
            break
    ctl.__exit__(None, None, None)
    return dofs / secs, done, dofs, secs


def run_batch(args):
    """Batched workload: independent 2D problems (quad or triangle meshes of 8^2 to
    64^2 cells, jitter 0.2h, k in 1..4, homogeneous Dirichlet data, forcing of 8
    random trigonometric modes), one union context per degree k; one step solves
    every problem to its own 1e-8 relative residual."""
    import torch
    from paper_2009_13840_gb300 import build, hho
    from synthetic.batch import BatchField, batch_problems, group_by_degree, union_mesh
    build.build()
    probs = batch_problems(args.batch_n, seed=args.batch_seed)
    groups = group_by_degree(probs)
    stream = torch.cuda.Stream()
    cf = 1 if (args.prec == "fp32" and args.batch_cond == "v") else 0

    def make(idx, k):
        m, fo, eo, sh = union_mesh([probs[i].mesh for i in idx])
        ctx = hho.Context(m, k, args.batch_cond, stream=stream)
        ctx.set_batch(fo, eo)
        data = hho.data_arrays(ctx, BatchField([probs[i].field for i in idx], sh))
        ctx.assemble(*data)
        ctx.set_option("coarse_fp32", cf)
        ctx.set_option("solve_graph", args.batch_graph)
        ctx.pmg_setup(list(range(k, -1, -1)), smooth_its=2, prec=args.prec)
        return ctx, data

    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        G = []
        for k, idx in groups.items():
            ctx, data = make(idx, k)
            tune = ctx.autotune(reps=3)
            x = torch.empty(ctx.ndof(0), dtype=torch.float64, device="cuda")
            G.append(dict(k=k, idx=idx, ctx=ctx, x=x, tune=tune, data=data))
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        ndof = sum(g["ctx"].ndof(0) for g in G)
        flush = torch.empty(512 * 2**20 // 4, dtype=torch.float32, device="cuda")

        def step():
            res = []
            for g in G:
                info, its, rr = g["ctx"].solve_batch(g["x"], rtol=args.rtol)
                res.append((info, its, rr))
            return res

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        launches0 = sum(g["ctx"].launch_count() for g in G)
        times, last = [], None
        with Clocks(torch.cuda.current_device()) as clk:
            for _ in range(args.steps):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                last = step()
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
        launches = sum(g["ctx"].launch_count() for g in G) - launches0
        ms = float(np.mean(times))
        its = np.concatenate([r[1] for r in last])
        rr = np.concatenate([r[2] for r in last])
        # end to end: data from pinned host memory, assembly, solve, solution back
        hdata = [[t.cpu().pin_memory() for t in g["data"]] for g in G]
        hx = [torch.empty(g["x"].numel(), dtype=torch.float64).pin_memory() for g in G]
        et = []
        for i in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            for g, hd, hxx in zip(G, hdata, hx):
                dd = [torch.empty_like(t, device="cuda").copy_(t, non_blocking=True) for t in hd]
                g["ctx"].assemble(*dd)
                g["ctx"].solve_batch(g["x"], rtol=args.rtol)
                hxx.copy_(g["x"], non_blocking=True)
            stream.synchronize()
            if i >= args.warmup:
                et.append(time.perf_counter() - t1)
        e2e_s = float(np.mean(et))
        h2d = int(sum(t.numel() * 8 for hd in hdata for t in hd))
        d2h = int(ndof * 8)
        # batching speedup: the first problems solved one by one against the same problems as a batch
        cmp = None
        if args.batch_compare > 0:
            sub = list(range(min(args.batch_compare, len(probs))))
            seq_ms = 0.0
            seq_its = []
            for i in sub:
                pr = probs[i]
                c1 = hho.Context(pr.mesh, pr.k, args.batch_cond, stream=stream)
                c1.assemble(*hho.data_arrays(c1, pr.field))
                c1.set_option("coarse_fp32", cf)
                c1.pmg_setup(list(range(pr.k, -1, -1)), smooth_its=2, prec=args.prec)
                x1 = torch.empty(c1.ndof(0), dtype=torch.float64, device="cuda")
                c1.solve(x1, rtol=args.rtol)
                info = c1.solve(x1, rtol=args.rtol)
                seq_ms += info["solve_ms"]
                seq_its.append(info["iterations"])
                c1.close()
            sg = group_by_degree([probs[i] for i in sub])
            bat_ms = 0.0
            bat_its = []
            for k, idx in sg.items():
                c2, _ = make([sub[i] for i in idx], k)
                x2 = torch.empty(c2.ndof(0), dtype=torch.float64, device="cuda")
                c2.solve_batch(x2, rtol=args.rtol)
                info, its2, _ = c2.solve_batch(x2, rtol=args.rtol)
                bat_ms += info["solve_ms"]
                bat_its += list(its2)
                c2.close()
            cmp = {"problems": len(sub), "sequential_ms": seq_ms, "batched_ms": bat_ms,
                   "speedup": seq_ms / bat_ms, "sequential_iterations_mean": float(np.mean(seq_its)),
                   "batched_iterations_mean": float(np.mean(bat_its))}
    cpu = None
    if not args.no_cpu_baseline:
        v, npb, nd, dt = oracle_batch_sample(probs, args.batch_cond, args.rtol)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"oracle FGMRES+p-MG solves of the first {npb} problems of the batch one by one "
                         f"({nd} DOFs, {dt:.1f} s); setup excluded; one thread"}
    wname = (f"batch{args.batch_n}-seed{args.batch_seed} quad/tri 8^2..64^2 jit0.2 k=1..4 "
             f"{args.batch_cond}-cond all-Dirichlet trig-forcing, one union context per k")
    line = {
        "metric": METRIC, "value": ndof / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 FGMRES + f32 V-cycle" if args.prec == "fp32" else "f64",
        "data": "synthetic",
        "config": {"workload": wname, "problems": len(probs), "dofs": ndof, "vcycle_precision": args.prec,
                   "groups": [{"k": g["k"], "problems": len(g["idx"]), "dofs": g["ctx"].ndof(0),
                               "autotuned": g["tune"]} for g in G],
                   "iterations_max": int(its.max()), "iterations_mean": float(its.mean()),
                   "rel_residual_max": float(rr.max()), "setup_s": setup_s,
                   "l2": "flushed between steps (512 MiB write)", "parallelism": "single",
                   "vs_sequential": cmp},
        "cpu_baseline": cpu,
        "e2e": {"value": ndof / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    for g in G:
        g["ctx"].close()


def run_learned(args):
    """Learned smoother: a two-layer MLP (hidden 128, BF16, first layer on the
    tensor cores) trained on the GPU on the finest-level post-smoother pairs of
    the FP64 V-cycle, taken on a smaller mesh of the workload family (default:
    24^3 jittered hexahedra, seed 1, k = 3, v&p condensation, about 10^5
    pairs), then used in the FP32 V-cycle of the evaluation mesh (default
    48^3 hexahedra, seed 0); one step = one solve to 1e-8 with the learned
    smoother, timed against the plain block-Jacobi smoother on the same
    problem.  --mesh tri gives the 2D variant (32x32 -> 128x128 triangles)."""
    import torch
    from paper_2009_13840_gb300 import build, hho
    build.build()
    cond, k = "vp", args.k
    train_n = args.learned_train_n or (24 if args.mesh == "hex" else 32)
    stream = torch.cuda.Stream()
    degrees = list(range(k, -1, -1))
    with torch.cuda.stream(stream):
        from synthetic import hex_mesh, tri_mesh
        if args.mesh == "hex":
            from synthetic import fields as F_
            tmesh, fld = hex_mesh(train_n, jitter=0.15, seed=1), F_.CurlStokes3D()
        else:
            tmesh, fld, _ = workload(train_n, k, cond, args.mesh)
        tr = hho.Context(tmesh, k, cond, stream=stream)
        tr.assemble(*hho.data_arrays(tr, fld))
        tr.pmg_setup(degrees, smooth_its=2, prec="fp64")
        tr.mlp_init(hidden=128, seed=11)
        n_vec = max(1, -(-args.learned_samples // tmesh.n_face))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nsamp = tr.mlp_generate(n_vec=n_vec, seed=3, kind=2)
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        loss = tr.mlp_train(steps=1500, batch=4096, lr=1e-3, seed=5)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        W = tr.mlp_weights()
        dims = tr.mlp_dims()
        tr.close()
        del tr
        torch.cuda.empty_cache()
        mesh, fld, wname = workload(args.n, k, cond, args.mesh)
        ctx = hho.Context(mesh, k, cond, stream=stream)
        f, gD, gN = hho.data_arrays(ctx, fld)
        ctx.assemble(f, gD, gN)
        ctx.set_option("coarse_fp32", args.coarse_fp32 if args.prec == "fp32" else 0)
        ctx.pmg_setup(degrees, smooth_its=2, prec=args.prec)
        ctx.mlp_init(hidden=128, seed=0)
        ctx.mlp_weights(W)
        ndof = ctx.ndof(0)
        x = torch.empty(ndof, dtype=torch.float64, device="cuda")
        flush = torch.empty(512 * 2**20 // 4, dtype=torch.float32, device="cuda")

        def timed(learned, steps):
            ctx.set_option("learned_smoother", learned)
            for _ in range(args.warmup):
                ctx.solve(x, rtol=args.rtol, maxit=2000)
            times, info = [], None
            for _ in range(steps):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                info = ctx.solve(x, rtol=args.rtol, maxit=2000)
                times.append(info["solve_ms"])
            return float(np.mean(times)), info

        ms_plain, inf_plain = timed(0, max(1, args.steps // 2))
        # the learned correction alone (tensor-core inference kernel) on a finest-level vector
        rv = torch.randn(ndof, dtype=torch.float64, device="cuda")
        zv = torch.zeros_like(rv)
        ctx.mlp_apply(rv, zv)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(10):
            ctx.mlp_apply(rv, zv)
        e1.record(stream)
        e1.synchronize()
        ms_apply = e0.elapsed_time(e1) / 10
        flops_apply = 2.0 * mesh.n_face * dims["din"] * dims["hid"] + 2.0 * mesh.n_face * dims["hid"] * dims["dout"]
        launches0 = ctx.launch_count()
        with Clocks(torch.cuda.current_device()) as clk:
            ms, inf = timed(1, args.steps)
        launches = ctx.launch_count() - launches0
        hf, hgD, hgN = f.cpu().pin_memory(), gD.cpu().pin_memory(), gN.cpu().pin_memory()
        hx = torch.empty(ndof, dtype=torch.float64).pin_memory()
        et = []
        for i in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            dd = [torch.empty_like(t, device="cuda").copy_(t, non_blocking=True) for t in (hf, hgD, hgN)]
            ctx.assemble(*dd)
            ctx.solve(x, rtol=args.rtol, maxit=2000)
            hx.copy_(x, non_blocking=True)
            stream.synchronize()
            if i >= args.warmup:
                et.append(time.perf_counter() - t1)
        ctx.close()
    line = {
        "metric": METRIC, "value": ndof / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 FGMRES + f32 V-cycle + bf16 MLP" if args.prec == "fp32" else "f64 + bf16 MLP",
        "data": "synthetic",
        "config": {"workload": wname + " learned smoother", "dofs": ndof, "vcycle_precision": args.prec,
                   "fgmres_iterations": inf["iterations"], "rel_residual_fp64": inf["rel_residual"],
                   "plain_smoother": {"ms_per_solve": ms_plain, "fgmres_iterations": inf_plain["iterations"],
                                      "dof_per_s": ndof / (ms_plain / 1e3)},
                   "speedup_vs_plain": ms_plain / ms,
                   "mlp_apply": {"ms": ms_apply, "tflops": flops_apply / (ms_apply / 1e3) / 1e12,
                                 "din": dims["din"], "hidden": dims["hid"], "dout": dims["dout"]},
                   "training": {"mesh": f"{args.mesh}{train_n}", "samples": int(nsamp), "vectors": n_vec,
                                "steps": 1500, "batch": 4096, "hidden": 128, "generate_s": gen_s,
                                "seconds": train_s, "loss_first": float(loss[:10].mean()),
                                "loss_last": float(loss[-50:].mean())},
                   "l2": "flushed between steps (512 MiB write)", "parallelism": "single"},
        "cpu_baseline": None,
        "e2e": {"value": ndof / float(np.mean(et)), "unit": UNIT,
                "h2d_bytes_per_step": int((f.numel() + gD.numel() + gN.numel()) * 8),
                "d2h_bytes_per_step": int(ndof * 8)},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "sweep":
        run_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
