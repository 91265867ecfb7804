#!/usr/bin/env python
"""Benchmark: factor + solve of the direct-indirect Burton-Miller system vs the ordinary one on
GB300, through the C ABI (libbm.so).

Workload: star curve r = 1 + 0.3 cos 5t, N = 4096 nodes (mixed 12288 x 12288, ordinary
8192 x 8192), k_out = 20, k_in = 30, 1 plane wave + 64 seeded complex Gaussian right-hand sides.
A step = factor + solve (all 65 right-hand sides, refined to backward error <= 1e-9) + far field
of the mixed system, then factor + solve of the ordinary system (the comparison).  The system is
assembled once before the timed region (its time is reported under "phases").
value = solves/s of the mixed system = nrhs / (factor + solve seconds), whole job over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec 3xtf32|tf32|fp64] [--impl reference]

Multi-GPU: independent replicas (one process per GPU under torchrun; no collective in the data
path), barrier + max over ranks around the timed region.
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

import workloads as W  # noqa: E402


METRIC = "factor+solve ms, solves/s: direct-indirect vs ordinary BM on 1 GB300 @relerr 1e-9"
UNIT = "solves/s"
PREC = {"fp64": 0, "tf32": 1, "3xtf32": 2}
DTYPE = {"fp64": "c128 (f64)", "tf32": "c64 factor (tf32 tensor cores) + f64 refinement",
         "3xtf32": "c64 factor (3xtf32 tensor cores) + f64 refinement"}


def workload_cfg(w: W.Workload, prec: str):
    return {
        "workload": f"star r=1+0.3cos5t, N={w.N} (mixed {3 * w.N}x{3 * w.N} as 4 NxN blocks, ordinary "
                    f"{2 * w.N}x{2 * w.N}), k_out={w.k_out}, k_in={w.k_in}, {w.n_plane} plane wave + "
                    f"{w.n_gauss} Gaussian RHS (seed {w.seed})",
        "formulation": "direct-indirect (Theorem thm:LU Schur path) vs ordinary Burton-Miller LU",
        "precision": prec,
        "refine_tol": 1e-9,
        "l2": "operands larger than L2 (mixed FP64 blocks 1.07 GB, FP32 packs 1.6 GB; L2 129 MB)",
    }


# --------------------------------------------------------------------------------------------
# distributed helpers (replicas only)
# --------------------------------------------------------------------------------------------
def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("BM_BENCH_GLOO") is None else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, v: float) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) > 8 for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# --------------------------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# --------------------------------------------------------------------------------------------
def oracle_problem(w: W.Workload):
    """The oracle's assembled blocks of the workload's mixed system and its right-hand sides (the
    plane wave and the seeded Gaussian columns), built on the host; not timed."""
    import oracle as O
    g = O.nodes(w.curve, w.N)
    P = O.default_params(w.k_out, w.k_in)
    blocks = O.mixed_blocks(g, P)
    Bp = O.rhs_plane_wave(g, P, [0.0], W.MIXED)
    Bg = W.place_rhs(W.gaussian_g(w.N, w.n_gauss, w.seed), w.N, W.MIXED)
    return blocks, np.concatenate([Bp, Bg], 1)


def _column_work(n: int) -> np.ndarray:
    """Relative cost of eliminating column k of an n x n matrix by the oracle's unblocked LU: the
    rank-1 update touches (n - k - 1)^2 entries (plus a per-column constant for the pivot search,
    row swap and scaling, taken as 4 n entries' worth)."""
    k = np.arange(n, dtype=np.float64)
    return (n - k - 1.0) ** 2 + 4.0 * n


def oracle_factor_solve_steps(blocks, B, nsteps: int):
    """The oracle's whole factor + solve of the mixed system (Theorem thm:LU: Schur complement by
    numpy matmul; unblocked LU with partial pivoting; Corollary lem:for_ssm_RHS solve), run as
    `nsteps` consecutive pieces of about equal LU work.  A generator: yields after each piece, so a
    caller can time the pieces one by one; their times add up to the time of the whole run."""
    from oracle.dense import lu_factor_columns, lu_solve, schur_complement
    M13, M23, M31, M32 = blocks
    N = M13.shape[0]
    cw = np.cumsum(_column_work(N))
    bounds = [int(np.searchsorted(cw, cw[-1] * (i + 1) / nsteps)) + 1 for i in range(nsteps)]
    bounds[-1] = N
    gen = lu_factor_columns(schur_complement(blocks))
    done = 0
    result = None
    for i in range(nsteps):
        while done < bounds[i]:
            try:
                next(gen)
                done += 1
            except StopIteration as fin:
                result = fin.value
                done = N
        if i == nsteps - 1:
            if result is None:
                try:
                    next(gen)
                except StopIteration as fin:
                    result = fin.value
            LU, piv = result
            b1, b2, b3 = B[:N], B[N:2 * N], B[2 * N:]
            z3 = lu_solve(LU, piv, b3 - M31 @ b1 - M32 @ b2)
            np.concatenate([b1 - M13 @ z3, b2 - M23 @ z3, z3], 0)
        yield i


def oracle_sample(w: W.Workload, ncols: int):
    """Bounded sample of the oracle's factor + solve of the workload itself (same N): the whole
    Schur complement, the first `ncols` columns of the unblocked LU, and a full Corollary solve
    (its cost does not depend on the values), each timed; the remaining LU columns are charged at
    the measured rate per unit of column work (n - k - 1)^2 + 4n."""
    from oracle.dense import lu_factor_columns, lu_solve, schur_complement
    blocks, B = oracle_problem(w)
    M13, M23, M31, M32 = blocks
    N = w.N
    t0 = time.perf_counter()
    U = schur_complement(blocks)
    t_schur = time.perf_counter() - t0
    gen = lu_factor_columns(U)
    t0 = time.perf_counter()
    for _ in range(ncols):
        next(gen)
    t_cols = time.perf_counter() - t0
    cw = _column_work(N)
    t_lu = t_cols * cw.sum() / cw[:ncols].sum()
    piv = np.arange(N)
    t0 = time.perf_counter()
    b1, b2, b3 = B[:N], B[N:2 * N], B[2 * N:]
    z3 = lu_solve(U, piv, b3 - M31 @ b1 - M32 @ b2)
    np.concatenate([b1 - M13 @ z3, b2 - M23 @ z3, z3], 0)
    t_solve = time.perf_counter() - t0
    total = t_schur + t_lu + t_solve
    return {"value": w.nrhs / total, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"oracle at the workload's own N={N}: Schur complement (numpy matmul, all cores) "
                      f"{t_schur:.2f} s, the first {ncols} of {N} unblocked-LU columns {t_cols:.2f} s "
                      f"(one thread; the other columns charged at that rate per unit of column work "
                      f"(n-k-1)^2+4n: {t_lu:.1f} s), Corollary solve of {w.nrhs} RHS {t_solve:.2f} s",
            "seconds_measured": t_schur + t_cols + t_solve, "seconds_total": total}


def oracle_other_configs():
    """The oracle on two more workloads, measured directly (no scaling within a run): the circle
    R = 1, N = 256, k_out = 2, k_in = 3, one plane wave (the section 5.1 shape; mixed Schur path and
    ordinary 2N dense LU, factor + solve), and one contour point of the contour batch (ellipse
    1.0/0.6, N = 1024, k_out = z_0 on the circle of centre 5 and radius 0.5, k_in = 1.5 k_out, 16
    Gaussian probe columns; assembly, Schur-path factor and Corollary solve).  Every one of the 32
    points has the same size and cost, so the batch total is given as 32 x that point, marked as
    such."""
    import oracle as O
    from oracle.dense import lu_factor, lu_solve, schur_complement
    from oracle.ssm import contour

    def corollary_solve(blocks, LU, piv, B):
        M13, M23, M31, M32 = blocks
        n = M13.shape[1]
        b1, b2, b3 = B[:n], B[n:2 * n], B[2 * n:]
        z3 = lu_solve(LU, piv, b3 - M31 @ b1 - M32 @ b2)
        return np.concatenate([b1 - M13 @ z3, b2 - M23 @ z3, z3], 0)

    out = {}
    g = O.nodes(W.circle(1.0), 256)
    P = O.default_params(2.0, 3.0)
    blocks = O.mixed_blocks(g, P)
    Bm = O.rhs_plane_wave(g, P, [0.0], W.MIXED)
    Ao = O.ordinary_matrix(g, P)
    Bo = O.rhs_plane_wave(g, P, [0.0], W.ORDINARY)
    t0 = time.perf_counter()
    LU, piv = lu_factor(schur_complement(blocks))
    corollary_solve(blocks, LU, piv, Bm)
    t1 = time.perf_counter()
    LUo, pivo = lu_factor(Ao)
    lu_solve(LUo, pivo, Bo)
    t2 = time.perf_counter()
    out["circle_n256"] = {"mixed_ms": (t1 - t0) * 1e3, "ordinary_ms": (t2 - t1) * 1e3,
                          "what": "factor + solve of one plane wave, FP64, measured directly"}
    z, _, _ = contour(5.0, 0.5, 32)
    V = W.gaussian_full(3 * 1024, 16, 0)
    t0 = time.perf_counter()
    g = O.nodes(W.ellipse(1.0, 0.6), 1024)
    P = O.default_params(z[0], 1.5 * z[0])
    blocks = O.mixed_blocks(g, P)
    t1 = time.perf_counter()
    LU, piv = lu_factor(schur_complement(blocks))
    t2 = time.perf_counter()
    corollary_solve(blocks, LU, piv, V)
    t3 = time.perf_counter()
    pt = t3 - t0
    out["ssm_point_n1024"] = {"assemble_ms": (t1 - t0) * 1e3, "factor_ms": (t2 - t1) * 1e3,
                              "solve_ms": (t3 - t2) * 1e3, "point_ms": pt * 1e3,
                              "batch_of_32_ms_extrapolated": 32 * pt * 1e3,
                              "what": "one contour point measured directly; the 32-point figure is 32 x it"}
    out["cores"] = os.cpu_count()
    out["kind"] = "oracle"
    return out


def run_reference(args, ws, rank):
    """The reference arm: the CPU oracle's whole factor + solve of the benchmark workload, measured
    directly (no extrapolation), split into --steps pieces of about equal LU work; --warmup untimed
    full factor + solves of the same scatterer at N = 256 come first."""
    if rank != 0:
        return
    w = W.scaled(W.STAR_N4096, 1024) if args.quick else W.STAR_N4096
    t_wall = time.perf_counter()
    small = W.scaled(w, 256)
    sb, sB = oracle_problem(small)
    for _ in range(args.warmup):
        for _i in oracle_factor_solve_steps(sb, sB, 1):
            pass
    blocks, B = oracle_problem(w)
    per = []
    gen = oracle_factor_solve_steps(blocks, B, args.steps)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        next(gen)
        per.append(time.perf_counter() - t0)
    total = float(np.sum(per))
    val = w.nrhs / total
    sample = (f"the oracle's whole factor+solve of the workload (N={w.N}, nrhs={w.nrhs}) measured directly: "
              f"numpy matmul Schur complement (all cores), unblocked LU (one thread), Corollary solve; "
              f"{args.steps} steps of equal LU work, {total:.1f} s in all")
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128 (f64, numpy)", "data": "synthetic",
            "config": workload_cfg(w, "fp64 oracle"), "impl": "reference",
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "seconds_factor_solve": total, "step_seconds": per, "wall_s": time.perf_counter() - t_wall}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------------
def colmajor_dev(rows, cols, torch, pinned=False, device="cuda"):
    if pinned:
        return torch.zeros((cols, rows), dtype=torch.complex128, pin_memory=True).t()
    return torch.zeros((cols, rows), dtype=torch.complex128, device=device).t()


def build_rhs(bm, h, w, form, torch):
    nsys = 3 * w.N if form == bm.BM_MIXED else 2 * w.N
    Bp = colmajor_dev(nsys, 1, torch)
    bm.bm_rhs_plane_wave(h, [0.0], Bp)
    G = W.place_rhs(W.gaussian_g(w.N, w.n_gauss, w.seed), w.N, form)
    B = torch.cat([Bp, torch.from_numpy(G).to("cuda")], 1)
    return colmajor_copy(B, torch)


def colmajor_copy(B, torch):
    out = torch.zeros((B.shape[1], B.shape[0]), dtype=torch.complex128, device=B.device).t()
    out.copy_(B)
    return out


def lu_work(n: int, NB: int = 256, nbp: int = 32) -> dict:
    """Algorithmic work of the blocked LU of an n x n complex matrix as the library blocks it (outer
    panels of NB columns, sub-panels of nbp): real flops (8 per complex multiply-add) of the
    sub-panel factorisations, of the rank-nbp updates inside each outer panel and of the trailing
    updates; and the bytes of the outer panels' row interchanges and U12 blocks (8-byte complex,
    read and written once)."""
    panel = inner = trail = 0.0
    swap_bytes = 0.0
    for J in range(0, n, NB):
        jb = min(NB, n - J)
        for j in range(J, J + jb, nbp):
            ib = min(nbp, J + jb - j)
            m = n - j
            panel += 8.0 * sum((m - c - 1) * (ib - c) for c in range(ib))
            rest = J + jb - j - ib
            if rest > 0:
                inner += 8.0 * (m - ib) * ib * rest
        mm = n - J - jb
        trail += 8.0 * mm * mm * jb
        swap_bytes += 16.0 * (2.0 * jb * (n - jb) + jb * mm)
    return {"panel": panel, "inner": inner, "trailing": trail, "swap_bytes": swap_bytes}


def roofline_from_profile(prof, N: int, nrhs: int, prec: int, iters: int, peaks: dict, src: str):
    """Roofline of the kernel with the largest summed device time in one mixed factor + solve
    (prof: (name, launches, ms) from bm_profile, largest first).  achieved = the kernel's algorithmic
    work in the step / its summed time (= work per launch / average launch time); the work of each
    kernel is its share of the method's arithmetic (real flops, 8 per complex multiply-add) or of
    its compulsory memory traffic, never the implementation's instruction count."""
    sm = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    fp32 = 152 * 128 * 2 * sm / 1e12                       # FP32 FMA TFLOP/s, unit counts x clock
    tf32 = peaks["bf16_tflops"] * (1.1 / 2.25)             # measured bf16 x nominal tf32/bf16 ratio
    hbm = peaks["hbm_gbs"]
    # where each peak comes from ("of measured" or "of fallback" for the peaks file's own figures)
    peak_src = {fp32: "derived: 152 SMs x 128 FP32 lanes x 2 flops x max SM clock",
                tf32: f"{src} bf16 x nominal TF32/bf16 ratio 1.1/2.25", hbm: src}
    lw = lu_work(N)
    work = {
        "resid_df_kernel (+ split-K reduction)": ("alu", 8.0 * 4 * N * N * nrhs, fp32, "TFLOP/s",
                                                  "4N^2 nrhs complex MACs x 8 real flops vs the FP32 FMA rate "
                                                  "(152 SMs x 128 lanes x 2 x clock)"),
        "resid_tc_kernel (+ split-K reduction)": ("hbm", 16.0 * 4 * N * N, hbm, "GB/s",
                                                  "the FP64 operator (4N^2 complex entries x 16 bytes) read once per "
                                                  "residual vs the measured copy bandwidth"),
        "cgemm_tc_kernel (Schur complement)": ("tensor", 16.0 * N ** 3, tf32, "TFLOP/s",
                                               "16 N^3 real flops (4M) vs the TF32 figure (measured bf16 x 1.1/2.25)"),
        "cgemm_tc_kernel (trailing update)": ("tensor", lw["trailing"], tf32, "TFLOP/s",
                                              "sum over outer panels of 8 m^2 NB real flops vs the TF32 figure"),
        "panel_lc_kernel": ("alu", lw["panel"], fp32, "TFLOP/s",
                            "unblocked LU flops of the 32-column sub-panels vs the FP32 FMA rate"),
        "panel_kernel": ("alu", lw["panel"], fp32, "TFLOP/s",
                         "unblocked LU flops of the sub-panels vs the FP32 FMA rate"),
        "cgemm_simt_kernel (panel update)": ("alu", lw["inner"], fp32, "TFLOP/s",
                                             "rank-32 updates inside the outer panels vs the FP32 FMA rate"),
        "swap_trsm_kernel (block row)": ("hbm", lw["swap_bytes"], hbm, "GB/s",
                                         "row interchanges of the outer panels' 2 NB rows and the U12 blocks, "
                                         "8-byte complex read + written"),
        "trsv_g_step_kernel": ("hbm", float(iters) * N * N * 8, hbm, "GB/s",
                               "the FP32 factors (N^2 x 8 bytes) read once per triangular-solve pair"),
        "trsv_flow_kernel": ("hbm", float(iters) * N * N * 8, hbm, "GB/s",
                             "the FP32 factors (N^2 x 8 bytes) read once per triangular-solve pair"),
        "cgemm_tc_kernel (skinny, + split-K reduction)": ("hbm", float(iters) * 4 * N * N * 8, hbm, "GB/s",
                                                          "[M31 M32] and [M13; M23] in complex FP32 read once per "
                                                          "correction"),
    }
    rows = []
    for name, launches, ms in prof:
        if name not in work:
            continue
        bound, amount, peak, unit, how = work[name]
        scale = 1e12 if unit == "TFLOP/s" else 1e9
        achieved = amount / (ms * 1e-3) / scale
        rows.append({"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                     "frac": achieved / peak, "traffic": None, "launches": launches, "ms_total": ms,
                     "ms_per_launch": ms / launches, "work_per_step": amount, "work": how,
                     "frac_note": peak_src.get(peak, src)})
    top_name = prof[0][0] if prof else None
    roof = next((r for r in rows if r["kernel"] == top_name), rows[0] if rows else None)
    return roof, {"kernels": [r for r in rows if r is not roof]}


def run_ours(args, ws, rank, local):
    import torch
    from paper_2512_14193_gb300 import build as BLD
    BLD.build()
    from paper_2512_14193_gb300 import bm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    w = W.STAR_N4096
    if args.quick or args.n:
        w = W.scaled(W.STAR_N4096, args.n or 1024)
    prec = PREC[args.prec]
    phases = {}

    hm = bm.bm_create(local, stream.cuda_stream)
    ho = bm.bm_create(local, stream.cuda_stream)
    opts = bm.make_opts(prec, eager=args.eager)
    p = w.curve.params4()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    # assembly (timed once each, outside the step)
    for name, h, form in (("mixed", hm, bm.BM_MIXED), ("ordinary", ho, bm.BM_ORDINARY)):
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        bm.bm_assemble(h, w.curve.kind, p, w.N, w.k_out, w.k_in, form, opts)
        e1.record(stream)
        torch.cuda.synchronize()
        phases[f"assemble_{name}_ms"] = e0.elapsed_time(e1)

    Bm = build_rhs(bm, hm, w, bm.BM_MIXED, torch)
    Bo = build_rhs(bm, ho, w, bm.BM_ORDINARY, torch)
    Xm = colmajor_dev(3 * w.N, w.nrhs, torch)
    Xo = colmajor_dev(2 * w.N, w.nrhs, torch)
    M_ff = 256
    th = 2 * np.pi * np.arange(M_ff) / M_ff
    U = colmajor_dev(M_ff, w.nrhs, torch)

    def step(rec=None):
        ts = [ev() for _ in range(6)] if rec is not None else None
        if ts:
            ts[0].record(stream)
        assert bm.bm_factor(hm) == 0
        if ts:
            ts[1].record(stream)
        im = bm.bm_solve(hm, Bm, Xm)
        if ts:
            ts[2].record(stream)
        bm.bm_far_field(hm, Xm, th, U)
        if ts:
            ts[3].record(stream)
        assert bm.bm_factor(ho) == 0
        if ts:
            ts[4].record(stream)
        io = bm.bm_solve(ho, Bo, Xo)
        if ts:
            ts[5].record(stream)
            rec.append((ts, im.backward_error, io.backward_error, im.iterations, io.iterations,
                        im.t_residual_ms, io.t_residual_ms))
        return im, io

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(ws)
    rec = []
    l0 = bm.bm_kernel_launches(hm) + bm.bm_kernel_launches(ho)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier(ws)
        t0 = ev()
        t0.record(stream)
        for _ in range(args.steps):
            step(rec)
        t1 = ev()
        t1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
    launches = bm.bm_kernel_launches(hm) + bm.bm_kernel_launches(ho) - l0
    total_ms = t0.elapsed_time(t1)
    f_m = np.median([r[0][0].elapsed_time(r[0][1]) for r in rec])
    s_m = np.median([r[0][1].elapsed_time(r[0][2]) for r in rec])
    ff = np.median([r[0][2].elapsed_time(r[0][3]) for r in rec])
    f_o = np.median([r[0][3].elapsed_time(r[0][4]) for r in rec])
    s_o = np.median([r[0][4].elapsed_time(r[0][5]) for r in rec])
    res_m = np.median([r[5] for r in rec])
    mixed_ms = allmax(ws, f_m + s_m)
    ord_ms = allmax(ws, f_o + s_o)
    value = ws * w.nrhs / (mixed_ms * 1e-3)
    phases.update({"factor_mixed_ms": f_m, "solve_mixed_ms": s_m, "far_field_ms": ff, "factor_ordinary_ms": f_o,
                   "solve_ordinary_ms": s_o, "residual_fp64_mixed_ms_per_solve": res_m,
                   "step_ms": total_ms / args.steps,
                   "refine_iterations_mixed": int(rec[-1][3]), "refine_iterations_ordinary": int(rec[-1][4]),
                   "backward_error_mixed": float(max(r[1] for r in rec)),
                   "backward_error_ordinary": float(max(r[2] for r in rec))})

    # ---- per-kernel breakdown of one factor + solve, and the roofline of the dominant kernel ----
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        src = "of measured"
    except (OSError, ValueError):
        peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
        src = "of fallback"
    N = w.N
    prof_m = bm.bm_profile(hm, Bm, Xm)
    prof_o = bm.bm_profile(ho, Bo, Xo)
    iters_m = int(rec[-1][3])
    roof, extra = roofline_from_profile(prof_m, N, w.nrhs, prec, iters_m, peaks, src)
    extra["profile_mixed"] = [{"kernel": k, "launches": l, "ms": m} for k, l, m in prof_m]
    extra["profile_ordinary"] = [{"kernel": k, "launches": l, "ms": m} for k, l, m in prof_o]
    # the residual and the Schur product also timed alone, in their normal launch configuration
    reps = 5
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record(stream)
    bm.bm_enqueue_probe(hm, bm.BM_PROBE_RESIDUAL, reps)
    b.record(stream)
    torch.cuda.synchronize()
    extra["residual_alone_ms_per_launch"] = a.elapsed_time(b) / reps
    if prec != 0:
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        bm.bm_enqueue_probe(hm, bm.BM_PROBE_SCHUR, reps)
        b.record(stream)
        torch.cuda.synchronize()
        t_schur = a.elapsed_time(b) / reps
        tf32 = peaks["bf16_tflops"] * (1.1 / 2.25)
        extra["schur_alone"] = {"ms_per_launch": t_schur, "tflops_algorithmic_4m": 16.0 * N ** 3 / (t_schur * 1e-3) / 1e12,
                                "frac_tf32": 16.0 * N ** 3 / (t_schur * 1e-3) / 1e12 / tf32,
                                "tflops_issued": 16.0 * N ** 3 * (3 if prec == 2 else 1) / (t_schur * 1e-3) / 1e12}
        bm.bm_factor(hm)

    # ---- end to end through the C ABI with pinned host buffers ----
    Bh = colmajor_dev(3 * N, w.nrhs, torch, pinned=True)
    Bh.copy_(Bm.cpu())
    Xh = colmajor_dev(3 * N, w.nrhs, torch, pinned=True)
    e2e = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t_a = time.perf_counter()
        bm.bm_factor(hm)
        bm.bm_solve(hm, Bh, Xh)
        t_b = time.perf_counter()
        if i >= args.warmup:
            e2e.append(t_b - t_a)
    e2e_s = allmax(ws, float(np.median(e2e)))
    hbytes = 3 * N * w.nrhs * 16

    # ---- accuracy against the FP64 path, and the other precisions / residual modes of config 2 ----
    extras = {}
    if ws == 1 and not args.no_extras:
        got = _guarded(lambda: fp64_compare(bm, local, stream, w, Bm, Xm, torch, ev))
        if isinstance(got, tuple):
            extras["fp64_path"], X64 = got
            extras["refined_to_1e-12"] = _guarded(
                lambda: tight_refinement(bm, local, stream, w, Bm, X64, torch, ev, prec))
            del X64
        else:
            extras["fp64_path"] = got
        extras["resid_fp64_all"] = _guarded(
            lambda: mode_timing(bm, local, stream, w, Bm, torch, ev, prec, bm.BM_RESID_FP64_ALL))
    asm_evals = float(w.N) * (w.N - 1)          # (H0, H1) pairs: N(N-1)/2 unordered pairs x 2 wavenumbers
    phases["assembly_mixed_hankel_evals_per_s"] = asm_evals / (phases["assemble_mixed_ms"] * 1e-3)
    phases["assembly_mixed_write_gbs"] = 4.0 * w.N * w.N * 16 / (phases["assemble_mixed_ms"] * 1e-3) / 1e9

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(w, 64 if args.quick else 128)
        cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample", "seconds_measured")}
        extras["cpu_oracle_other_configs"] = _guarded(oracle_other_configs)

    bm.bm_destroy(hm)
    bm.bm_destroy(ho)
    if ws == 1 and not args.no_extras:
        extras["circle_n256"] = _guarded(lambda: circle_latency(bm, local, stream, torch, ev))
        if not args.quick:
            extras["kite_n16384"] = _guarded(lambda: kite_large(bm, local, stream, torch, ev, args.config5_fp64))
    ssm = None if args.no_ssm else _guarded(lambda: ssm_measure(bm, local))
    serve = None if args.no_serve else _guarded(lambda: serve_measure(bm, local, n_req=args.serve_requests))
    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mixed_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.prec], "data": "synthetic",
            "config": workload_cfg(w, args.prec),
            "ordinary": {"ms": ord_ms, "solves_per_s": ws * w.nrhs / (ord_ms * 1e-3),
                         "speedup_mixed_over_ordinary": ord_ms / mixed_ms},
            "phases": phases, "roofline": roof, "roofline_extra": extra,
            "cpu_baseline": cpu,
            "e2e": {"value": ws * w.nrhs / e2e_s, "unit": UNIT, "h2d_bytes_per_step": hbytes,
                    "d2h_bytes_per_step": hbytes, "ms": e2e_s * 1e3,
                    "path": "bm_factor + bm_solve with pinned host B/X (copies inside bm_solve)"},
            "clocks": clk.summary(), "gpu_launches": int(launches)}
    line.update(extras)
    if ssm is not None:
        line["ssm"] = ssm
    if serve is not None:
        line["serving"] = serve
    print(json.dumps(line), flush=True)


def _guarded(fn):
    """Run one of the secondary measurements (other configurations, precisions, the serving stream,
    the CPU baselines).  A failure there is reported in the line as {"error": ...} instead of
    losing the headline measurement, which is already taken when these run."""
    try:
        return fn()
    except Exception as e:
        return {"error": f"{type(e).__name__}: {e}"}


def _time_factor_solve(bm, h, B, X, stream, torch, ev, steps: int, warmup: int = 1):
    """Median factor + solve device time (ms) of a handle, with the last solve's report."""
    info = None
    for _ in range(warmup):
        bm.bm_factor(h)
        info = bm.bm_solve(h, B, X)
    t = []
    for _ in range(steps):
        a, b, c = ev(), ev(), ev()
        a.record(stream)
        assert bm.bm_factor(h) == 0
        b.record(stream)
        info = bm.bm_solve(h, B, X)
        c.record(stream)
        torch.cuda.synchronize()
        t.append((a.elapsed_time(b), b.elapsed_time(c)))
    f = float(np.median([x[0] for x in t]))
    s = float(np.median([x[1] for x in t]))
    return f, s, info


def fp64_compare(bm, device, stream, w, Bm, Xm, torch, ev):
    """The FP64 path on the same system and right-hand sides: its factor + solve time, and the
    forward relative error of the benchmark's refined CF32 solution against it (per column, the
    largest), which is the metric's "relerr"."""
    h = bm.bm_create(device, stream.cuda_stream)
    try:
        bm.bm_assemble(h, w.curve.kind, w.curve.params4(), w.N, w.k_out, w.k_in, bm.BM_MIXED, bm.make_opts(0))
        X64 = colmajor_dev(3 * w.N, w.nrhs, torch)
        f, s, info = _time_factor_solve(bm, h, Bm, X64, stream, torch, ev, steps=3)
        d = _relerr_cols(Xm, X64)
        return {"factor_ms": f, "solve_ms": s, "ms": f + s, "solves_per_s": w.nrhs / ((f + s) * 1e-3),
                "backward_error": info.backward_error,
                "relerr_cf32_vs_fp64_max_col": float(d.max().item()),
                "relerr_cf32_vs_fp64_plane_wave": float(d[0].item()),
                "note": "relerr = ||x_cf32 - x_fp64||_2 / ||x_fp64||_2 per right-hand side over all 3N unknowns"}, X64
    finally:
        bm.bm_destroy(h)


def _relerr_cols(X, Xref):
    return (X - Xref).abs().pow(2).sum(0).sqrt() / Xref.abs().pow(2).sum(0).sqrt()


def tight_refinement(bm, device, stream, w, Bm, X64, torch, ev, prec, tol: float = 1e-12):
    """The benchmark's factor + solve refined further, to backward error `tol` instead of 1e-9: what
    a forward relative error below 1e-9 against the FP64 path costs (the FP64 path's own forward
    error is about cond x 1e-16)."""
    h = bm.bm_create(device, stream.cuda_stream)
    try:
        bm.bm_assemble(h, w.curve.kind, w.curve.params4(), w.N, w.k_out, w.k_in, bm.BM_MIXED,
                       bm.make_opts(prec, refine_tol=tol))
        X = colmajor_dev(3 * w.N, w.nrhs, torch)
        f, s, info = _time_factor_solve(bm, h, Bm, X, stream, torch, ev, steps=3)
        d = _relerr_cols(X, X64)
        return {"refine_tol": tol, "factor_ms": f, "solve_ms": s, "ms": f + s,
                "solves_per_s": w.nrhs / ((f + s) * 1e-3), "iterations": info.iterations,
                "backward_error": info.backward_error,
                "relerr_cf32_vs_fp64_max_col": float(d.max().item())}
    finally:
        bm.bm_destroy(h)


def mode_timing(bm, device, stream, w, Bm, torch, ev, prec, resid_mode):
    """Factor + solve of config 2 with another refinement-residual mode (every residual in FP64)."""
    h = bm.bm_create(device, stream.cuda_stream)
    try:
        bm.bm_assemble(h, w.curve.kind, w.curve.params4(), w.N, w.k_out, w.k_in, bm.BM_MIXED,
                       bm.make_opts(prec, residual=resid_mode))
        X = colmajor_dev(3 * w.N, w.nrhs, torch)
        f, s, info = _time_factor_solve(bm, h, Bm, X, stream, torch, ev, steps=3)
        return {"refine_residual": int(resid_mode), "factor_ms": f, "solve_ms": s, "ms": f + s,
                "solves_per_s": w.nrhs / ((f + s) * 1e-3), "iterations": info.iterations,
                "backward_error": info.backward_error, "t_residual_ms": info.t_residual_ms}
    finally:
        bm.bm_destroy(h)


def circle_latency(bm, device, stream, torch, ev):
    """Config 1 (section 5.1 shape): circle R = 1, N = 256, k0 = 2, k1 = 3, one plane wave, FP64;
    factor + solve latency of the direct-indirect (768 unknowns, Schur path) and ordinary (512)
    systems, median of 20 after 3 warm-ups."""
    out = {"workload": "circle R=1, N=256, k_out=2, k_in=3, 1 plane wave, FP64"}
    for name, form in (("mixed", bm.BM_MIXED), ("ordinary", bm.BM_ORDINARY)):
        h = bm.bm_create(device, stream.cuda_stream)
        try:
            bm.bm_assemble(h, W.CIRCLE, (1.0, 0.0, 0.0, 0.0), 256, 2.0, 3.0, form, bm.make_opts(0))
            nsys = 768 if form == bm.BM_MIXED else 512
            B = colmajor_dev(nsys, 1, torch)
            bm.bm_rhs_plane_wave(h, [0.0], B)
            X = colmajor_dev(nsys, 1, torch)
            f, s, info = _time_factor_solve(bm, h, B, X, stream, torch, ev, steps=20, warmup=3)
            out[name] = {"factor_us": f * 1e3, "solve_us": s * 1e3, "us": (f + s) * 1e3,
                         "backward_error": info.backward_error}
        finally:
            bm.bm_destroy(h)
    out["speedup_mixed_over_ordinary"] = out["ordinary"]["us"] / out["mixed"]["us"]
    return out


def kite_large(bm, device, stream, torch, ev, with_fp64: bool):
    """Config 5: kite, N = 16384 (mixed 49152 unknowns as four 16384^2 blocks; ordinary 32768^2),
    k0 = 100, k1 = 150, 1 plane wave + 7 Gaussian RHS (seed 0); complex 3xTF32 factors + refinement
    to 1e-9 for both formulations (and the FP64 mixed path when asked: about a minute)."""
    w = W.KITE_N16384
    out = {"workload": "kite N=16384, k_out=100, k_in=150, 1 plane wave + 7 Gaussian RHS (seed 0)"}
    runs = [("mixed_3xtf32", bm.BM_MIXED, 2), ("ordinary_3xtf32", bm.BM_ORDINARY, 2)]
    if with_fp64:
        runs.append(("mixed_fp64", bm.BM_MIXED, 0))
    for name, form, prec in runs:
        h = bm.bm_create(device, stream.cuda_stream)
        try:
            torch.cuda.synchronize()
            a, b = ev(), ev()
            a.record(stream)
            bm.bm_assemble(h, w.curve.kind, w.curve.params4(), w.N, w.k_out, w.k_in, form, bm.make_opts(prec))
            b.record(stream)
            torch.cuda.synchronize()
            B = build_rhs(bm, h, w, form, torch)
            X = colmajor_dev(B.shape[0], w.nrhs, torch)
            steps = 1 if prec == 0 else 3
            f, s, info = _time_factor_solve(bm, h, B, X, stream, torch, ev, steps=steps, warmup=1)
            out[name] = {"assemble_ms": a.elapsed_time(b), "factor_ms": f, "solve_ms": s, "ms": f + s,
                         "solves_per_s": w.nrhs / ((f + s) * 1e-3), "iterations": info.iterations,
                         "backward_error": info.backward_error, "steps": steps}
        finally:
            bm.bm_destroy(h)
            torch.cuda.synchronize()
    out["speedup_mixed_over_ordinary_3xtf32"] = out["ordinary_3xtf32"]["ms"] / out["mixed_3xtf32"]["ms"]
    return out


def ssm_measure(bm, device: int):
    """Contour batch (block Sakurai-Sugiura, section 5.3): ellipse 1.0/0.6, N = 1024, mixed system,
    k_in = 1.5 k_out, circle centre 5 radius 0.5, 32 points, 16 Gaussian probes, 4 moments, all 32
    points in one batch (batched assembly and Schur launches, concurrent LU graphs, the panel
    cluster autotuned on the warm-up call and reused).  The FP32 tensor-core path (every residual
    from nine-digit tensor-core products, refined to the FP64 path's accuracy) against the FP64
    path; a warm-up call each (which also keeps the batch's handles for the timed call), then one
    timed call (wall clock of bm_ssm)."""
    N, L, P = 1024, 16, 32
    V = np.asfortranarray(W.gaussian_full(3 * N, L, 0))
    cv = W.ellipse(1.0, 0.6)
    out = {"workload": "ellipse 1.0/0.6, N=1024 (mixed), k_in=1.5 k_out, circle centre 5 radius 0.5, "
                       "32 points, 16 probes (seed 0), 4 moments, rank cut 1e-6"}
    for name, opts in (("3xtf32", bm.make_opts(2, refine_tol=1e-15, residual=bm.BM_RESID_TC_ALL)),
                       ("fp64", bm.make_opts(0))):
        cl = 0
        for rep in range(2):
            t0 = time.perf_counter()
            om, sig, info = bm.bm_ssm(device, cv.kind, cv.params4(), N, W.MIXED, opts, 5.0, 0.5, P, 4, 1.5, V,
                                      rank_tol=1e-6, panel_cluster=cl)
            t = time.perf_counter() - t0
            if rep == 0:
                tuned = list(info.tune_ms)
            cl = info.panel_cluster
        out[name] = {"ms": t * 1e3, "contour_points_per_s": P / t, "solves_per_s": P * L / t, "rank": info.rank,
                     "n_inside": info.n_inside, "max_backward_error": info.max_backward_error,
                     "max_refine_iterations": info.max_iterations, "assemble_ms": info.t_assemble_ms,
                     "factor_ms": info.t_factor_ms, "solve_ms": info.t_solve_ms, "batch": info.batch,
                     "panel_cluster_autotuned": info.panel_cluster,
                     "autotune_factor_ms_cluster_16_8_4": tuned if any(tuned) else list(info.tune_ms)}
    out["speedup_3xtf32_over_fp64"] = out["fp64"]["ms"] / out["3xtf32"]["ms"]
    bm.bm_ssm_release(device)
    return out


def serve_measure(bm, device: int, n_req: int = 300, slots: int = 8, loads=(0.5, 0.8, 1.0)):
    """Serving stream (first n_req requests of workloads.serving_stream, seed 0: star curves, N in
    {256 .. 8192}, complex k_out, k_in = 1.5 k_out, 1..64 Gaussian right-hand sides each, mixed
    system, 3xTF32 + refinement to 1e-9).  Capacity: all requests submitted at once, wall time to
    drain.  Latency: the same requests arriving as a Poisson process at each load x that capacity;
    p50 / p99 of submit-to-done per load."""
    reqs = W.serving_stream(n_req, seed=0)
    Bs = [np.asfortranarray(W.place_rhs(W.gaussian_g(r["N"], r["nrhs"], 1000 + i), r["N"], W.MIXED))
          for i, r in enumerate(reqs)]
    opts = bm.make_opts(2)

    def run(arrivals):
        s = bm.bm_server_create(device, slots=slots, opts=opts)
        Xs = [np.zeros_like(B, order="F") for B in Bs]
        t0 = time.perf_counter()
        tickets = []
        for r, B, X, ta in zip(reqs, Bs, Xs, arrivals):
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets.append(bm.bm_server_submit(s, r["curve"].kind, r["curve"].params4(), r["N"], r["k_out"],
                                               r["k_in"], W.MIXED, B, X))
        res = [bm.bm_server_wait(s, t) for t in tickets]
        wall = time.perf_counter() - t0
        st = bm.bm_server_stats_get(s)
        bm.bm_server_destroy(s)
        return res, wall, st

    run([0.0] * 8)  # warm-up (the first 8 requests): memory pool, libraries
    res, wall, st = run([0.0] * n_req)
    cap = n_req / wall
    nrhs_tot = sum(r["nrhs"] for r in reqs)
    sweep = []
    worst = max(r.backward_error for r in res)
    mif, mifb = st.max_in_flight, st.max_in_flight_bytes
    for load in loads:
        lam = load * cap
        res2, wall2, st2 = run([r["t"] / lam for r in reqs])
        lat = np.array([r.t_queue_ms + r.t_service_ms for r in res2])
        sweep.append({"load": load, "rate_requests_per_s": lam, "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99)), "solves_per_s": nrhs_tot / wall2})
        worst = max(worst, max(r.backward_error for r in res2))
        mif, mifb = max(mif, st2.max_in_flight), max(mifb, st2.max_in_flight_bytes)
    at08 = min(sweep, key=lambda x: abs(x["load"] - 0.8))
    return {"workload": f"first {n_req} of the 2000 requests of the serving stream (seed 0): star curves, N in "
                        "{256..8192}, Re k_out in [2, 40], Im in [-0.5, 0], k_in = 1.5 k_out, nrhs 1..64; "
                        "mixed system, 3xTF32 + refinement to 1e-9",
            "slots": slots, "capacity_requests_per_s": cap, "capacity_solves_per_s": nrhs_tot / wall,
            "poisson_rate_requests_per_s": at08["rate_requests_per_s"], "p50_ms": at08["p50_ms"],
            "p99_ms": at08["p99_ms"], "solves_per_s_at_rate": at08["solves_per_s"], "load_sweep": sweep,
            "max_backward_error": worst, "max_in_flight": mif, "max_in_flight_gb": mifb / 1e9,
            "budget_gb": st.budget_bytes / 1e9}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--prec", choices=list(PREC), default="3xtf32")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ssm", action="store_true", help="skip the contour-batch (Sakurai-Sugiura) timing")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-stream timing")
    ap.add_argument("--serve-requests", type=int, default=300, help="requests of the serving stream to run")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64 comparison, the residual-mode timing and configs 1 and 5")
    ap.add_argument("--config5-fp64", action="store_true", help="also time the FP64 mixed path at N=16384")
    ap.add_argument("--quick", action="store_true", help="N=1024 instead of 4096 (smoke-sized)")
    ap.add_argument("--n", type=int, default=0, help="another N for the same star workload (profiling sizes)")
    ap.add_argument("--eager", action="store_true",
                    help="launch the factor and solve kernels one by one instead of as CUDA graphs (for ncu)")
    args = ap.parse_args()
    ws, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
