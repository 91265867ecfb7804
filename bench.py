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


def profiled_traffic(summary: str, n: int):
    """DRAM bytes per launch from a committed ncu summary under profiles/, scaled from the captured
    N to n by the summary's rule ((n/N)^2 for operator-bound kernels), or None when the kernel's
    source has changed since the counters were taken (hash recorded in the summary)."""
    import hashlib
    import re
    try:
        txt = open(os.path.join(ROOT, "profiles", summary)).read()
        m = re.search(r"traffic_bytes_per_launch_n(\d+): (\d+)", txt)
        src = re.search(r"^source: (\S+)", txt, re.M).group(1)
        h = re.search(r"source_sha256_12: ([0-9a-f]+)", txt).group(1)
        cur = hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest()[:12]
        if m is None or cur != h:
            return None
        n0, b0 = int(m.group(1)), int(m.group(2))
        return b0 * (n / n0) ** 2
    except (OSError, AttributeError):
        return None

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
_ORACLE_CACHE = {}


def oracle_sample(w: W.Workload, n_sample: int, reps: int):
    """Time the oracle's factor+solve (Theorem thm:LU path: numpy matmul Schur complement,
    unblocked LU, Corollary lem:for_ssm_RHS solve) of the same scatterer at N = n_sample with the
    workload's nrhs, and scale the time by (N / n_sample)^3 to the workload's N.  The oracle's
    assembly of the sample system is done once and not timed (the metric is factor + solve)."""
    import oracle as O
    from oracle.dense import lu_factor, lu_solve, schur_complement
    ws = W.scaled(w, n_sample)
    if n_sample not in _ORACLE_CACHE:
        g = O.nodes(ws.curve, ws.N)
        P = O.default_params(ws.k_out, ws.k_in)
        blocks = O.mixed_blocks(g, P)
        Bp = O.rhs_plane_wave(g, P, [0.0], W.MIXED)
        Bg = W.place_rhs(W.gaussian_g(ws.N, ws.n_gauss, ws.seed), ws.N, W.MIXED)
        _ORACLE_CACHE[n_sample] = (blocks, np.concatenate([Bp, Bg], 1))
    blocks, B = _ORACLE_CACHE[n_sample]
    M13, M23, M31, M32 = blocks
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        LU, piv = lu_factor(schur_complement(blocks))
        b1, b2, b3 = B[:ws.N], B[ws.N:2 * ws.N], B[2 * ws.N:]
        z3 = lu_solve(LU, piv, b3 - M31 @ b1 - M32 @ b2)
        _x = np.concatenate([b1 - M13 @ z3, b2 - M23 @ z3, z3], 0)
        times.append(time.perf_counter() - t0)
    scale = (w.N / n_sample) ** 3
    t_full = float(np.median(times)) * scale
    return {"value": w.nrhs / t_full, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"oracle factor+solve at N={n_sample} (same star, k, nrhs={w.nrhs}), median of {reps}, "
                      f"scaled by (N/{n_sample})^3 = {scale:.0f} to N={w.N}; numpy BLAS matmul on all cores, "
                      f"unblocked LU loop in one thread",
            "seconds_sample": float(np.median(times)), "seconds_scaled": t_full}


def run_reference(args, ws, rank):
    w = W.STAR_N4096
    if rank != 0:
        return
    n_sample = 768 if args.quick else 1024
    t0 = time.perf_counter()
    per = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample(w, n_sample, 1)
        if i >= args.warmup:
            per.append(r["seconds_scaled"])
    t_step = float(np.median(per))
    val = w.nrhs / t_step
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128 (f64, numpy)", "data": "synthetic",
            "config": workload_cfg(w, "fp64 oracle"), "impl": "reference",
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
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
    opts = bm.make_opts(prec)
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

    # ---- roofline of the hot kernels (own events on the library's stream) ----
    roof = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        src = "of measured"
    except (OSError, ValueError):
        peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
        src = "of fallback"
    N = w.N
    reps = 5
    # FP64 residual (2 complex GEMMs per residual: [M13;M23] x3 and [M31 M32] [x1;x2])
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record(stream)
    bm.bm_enqueue_probe(hm, bm.BM_PROBE_RESIDUAL, reps)
    b.record(stream)
    torch.cuda.synchronize()
    t_res = a.elapsed_time(b) / reps
    cmacs = 4.0 * N * N * w.nrhs                  # complex multiply-adds of one residual b - A x
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    if prec != 0:
        # double-float on the FP32 pipe: 36 FP32 instructions per complex multiply-add
        # (3 real products (re a re x, im a im x, (re a + im a)(re x + im x)) x [TwoProd 2 +
        # TwoSum 6 + 2 accumulate] + 6 cross-term FMAs); peak = 152 SMs x 128 FP32 lanes x SM
        # clock (FMA, add and multiply each issue once per lane per cycle)
        ops = 36.0 * cmacs
        peak = 152 * 128 * sm_mhz * 1e6 / 1e12
        roof_res = {"kernel": "resid_df_kernel (double-float residual b - A x on the FP32 pipe, all products in "
                              "one launch; timed with its iterate split and split-K reduction)", "bound": "alu",
                    "achieved": ops / (t_res * 1e-3) / 1e12, "peak": peak, "unit": "T FP32-instr/s",
                    "frac": ops / (t_res * 1e-3) / 1e12 / peak,
                    "traffic": profiled_traffic("resid_df_star_n2048.md", N), "ms_per_launch": t_res,
                    "traffic_note": "dram bytes read+written per launch, ncu at N=2048 scaled by (N/2048)^2 "
                                    "(operator planes); null once the kernel source changed",
                    "peak_source": f"152 SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz (unit counts x clock)"}
    else:
        flops_res = 8.0 * cmacs
        peak = 152 * 4 * sm_mhz * 1e6 / 1e12      # 2 DFMA per SM per cycle (1.19 TFLOP/s measured)
        roof_res = {"kernel": "cgemm_simt_kernel<Z64> x2 (FP64 residual b - A x)", "bound": "alu",
                    "achieved": flops_res / (t_res * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                    "frac": flops_res / (t_res * 1e-3) / 1e12 / peak, "traffic": None, "ms_per_launch": t_res / 2,
                    "peak_source": f"152 SMs x 2 DFMA/cycle x {sm_mhz:.0f} MHz (unit counts x clock)"}
    # Schur complement on the tensor cores (overwrites U33: re-factor afterwards)
    if prec != 0:
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        bm.bm_enqueue_probe(hm, bm.BM_PROBE_SCHUR, reps)
        b.record(stream)
        torch.cuda.synchronize()
        t_schur = a.elapsed_time(b) / reps
        nprod = 3 if prec == 2 else 1
        flops = 16.0 * N ** 3 * nprod            # 2N^3 complex MACs x 8 real flops x TF32 products
        tf32_peak = peaks["bf16_tflops"] * (1.1 / 2.25)
        roof_tc = {"kernel": "cgemm_tc_kernel (tcgen05 kind::tf32, Schur complement U33)", "bound": "tensor",
                   "achieved": flops / (t_schur * 1e-3) / 1e12, "peak": tf32_peak, "unit": "TFLOP/s",
                   "frac": flops / (t_schur * 1e-3) / 1e12 / tf32_peak, "traffic": None, "ms_per_launch": t_schur,
                   "peak_source": f"bf16 burst {src} x 1.1/2.25 (nominal tf32/bf16 dense ratio)",
                   "flop_count": f"16 N^3 x {nprod} TF32 product(s) per complex 4M product"}
        bm.bm_factor(hm)
    # dominant kernel of the mixed factor+solve: the one with the larger share of the step
    share_res = 2 * t_res / (f_m + s_m)
    if prec != 0 and (t_schur / (f_m + s_m)) > share_res:
        roof = roof_tc
        extra = {"fp64_residual": roof_res}
    else:
        roof = roof_res
        extra = {"tensor_schur": roof_tc} if prec != 0 else {}
    roof = dict(roof)
    roof["frac_note"] = src

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

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(W.STAR_N4096, 768 if args.quick else 1024, 2)
        cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}

    bm.bm_destroy(hm)
    bm.bm_destroy(ho)
    ssm = None if args.no_ssm else ssm_measure(bm, local)
    serve = None if args.no_serve else serve_measure(bm, local)
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
    if ssm is not None:
        line["ssm"] = ssm
    if serve is not None:
        line["serving"] = serve
    print(json.dumps(line), flush=True)


def ssm_measure(bm, device: int):
    """Contour batch (block Sakurai-Sugiura, section 5.3): ellipse 1.0/0.6, N = 1024, mixed system,
    k_in = 1.5 k_out, circle centre 5 radius 0.5, 32 points, 16 Gaussian probes, 4 moments.  The
    FP32 tensor-core path (FP64 residuals, refined to the FP64 path's accuracy) against the FP64
    path; a warm-up call each, then one timed call (wall clock of bm_ssm)."""
    N, L, P = 1024, 16, 32
    V = np.asfortranarray(W.gaussian_full(3 * N, L, 0))
    cv = W.ellipse(1.0, 0.6)
    out = {"workload": "ellipse 1.0/0.6, N=1024 (mixed), k_in=1.5 k_out, circle centre 5 radius 0.5, "
                       "32 points, 16 probes (seed 0), 4 moments, rank cut 1e-6"}
    for name, opts in (("3xtf32", bm.make_opts(2, refine_tol=1e-15, residual=bm.BM_RESID_FP64_ALL)),
                       ("fp64", bm.make_opts(0))):
        for rep in range(2):
            t0 = time.perf_counter()
            om, sig, info = bm.bm_ssm(device, cv.kind, cv.params4(), N, W.MIXED, opts, 5.0, 0.5, P, 4, 1.5, V,
                                      rank_tol=1e-6)
            t = time.perf_counter() - t0
        out[name] = {"ms": t * 1e3, "contour_points_per_s": P / t, "solves_per_s": P * L / t, "rank": info.rank,
                     "n_inside": info.n_inside, "max_backward_error": info.max_backward_error,
                     "max_refine_iterations": info.max_iterations}
    out["speedup_3xtf32_over_fp64"] = out["fp64"]["ms"] / out["3xtf32"]["ms"]
    return out


def serve_measure(bm, device: int, n_req: int = 120, slots: int = 8):
    """Serving stream (first n_req requests of workloads.serving_stream, seed 0: star curves, N in
    {256 .. 8192}, complex k_out, k_in = 1.5 k_out, 1..64 Gaussian right-hand sides each, mixed
    system, 3xTF32 + refinement to 1e-9).  Capacity: all requests submitted at once, wall time to
    drain.  Latency: the same requests arriving as a Poisson process at 0.8 x that capacity;
    p50 / p99 of submit-to-done."""
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
    lam = 0.8 * cap
    arrivals = [r["t"] / lam for r in reqs]
    res2, wall2, st2 = run(arrivals)
    lat = np.array([r.t_queue_ms + r.t_service_ms for r in res2])
    return {"workload": f"first {n_req} requests of the serving stream (seed 0): star curves, N in "
                        "{256..8192}, Re k_out in [2, 40], Im in [-0.5, 0], k_in = 1.5 k_out, nrhs 1..64; "
                        "mixed system, 3xTF32 + refinement to 1e-9",
            "slots": slots, "capacity_requests_per_s": cap, "capacity_solves_per_s": nrhs_tot / wall,
            "poisson_rate_requests_per_s": lam, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "solves_per_s_at_rate": nrhs_tot / wall2,
            "max_backward_error": max(r.backward_error for r in res + res2),
            "max_in_flight": max(st.max_in_flight, st2.max_in_flight),
            "max_in_flight_gb": max(st.max_in_flight_bytes, st2.max_in_flight_bytes) / 1e9,
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
    ap.add_argument("--quick", action="store_true", help="N=1024 instead of 4096 (smoke-sized)")
    ap.add_argument("--n", type=int, default=0, help="another N for the same star workload (profiling sizes)")
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
