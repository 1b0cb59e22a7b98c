"""GMLS stencil-generation benchmark (one JSON line on rank 0).

Workload (the 2D Stokes operators of the compatible GMLS scheme, arXiv
2104.14447 Sec. 3): 262,144 targets on a 512 x 512 jittered grid in the unit
square (h = 1/512, jitter +-h/4, seed 0), sources = targets.  One step is the
whole hot path:

  cell-list build -> 36- and 48-nearest-neighbour lists (eps = 1.5 d_k) ->
  scalar Taylor degree-4 stencils (15 terms; pressure gradient and the
  component-wise divergence) -> divergence-free degree-4 stencils (20 terms,
  96 x 20 systems; vector Laplacian) -> three CSR operators.

value: targets/s of the whole job (every target gets all three operators).
The default precision is FP32 Householder QR with refinement against
float-float (FP64-class) residuals; ``--precision fp64`` times the plain FP64
path.  The 36-nearest lists are the first 36 entries of the 48-nearest lists
(one search; both are prefixes of the same (d^2, id) order).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 it runs under torch.distributed.run, one rank per GPU; every rank
processes its own copy of the workload (independent problems: weak scaling,
no data-path collective; only the timing is reduced).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_AXIS = 512
K_SCALAR, K_DIVFREE, EPS_FACTOR, DEGREE = 36, 48, 1.5, 4
E2E_CHUNKS = 4  # default target ranges of the end-to-end pipeline (copies overlap compute)
METRIC = "GMLS targets/sec"
WORKLOAD = "stokes2d-512x512: scalar m=4 (36 nbrs; grad, div) + div-free m=4 (48 nbrs; vector Laplacian) + CSR"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


# ALU peaks of one GB300 from unit counts and the maximum SM clock (2070 MHz):
#   FP32: 152 SMs x 128 FMA lanes x 2 flop x 2.07 GHz = 80.5 TFLOP/s
#   FP64: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz     = 1.26 TFLOP/s
P32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
P64_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


# FP32 operations of one compensated float-float product-accumulate (Dot2 step):
# TwoProd (1 mul + 1 fma), two cross-term fmas, TwoSum (6 adds), 2 adds;
# an fma counts as 2.
DOT2_FLOPS = 15


# DRAM bytes (read + write) per target of the divergence-free register-kernel
# launch, from ncu on the 384 x 384 grid (147,456 targets: 33.95 MB read,
# 168.58 MB written); the algorithmic floor is the 1,536 B of FP64 weights
# per target (2 rows x 48 neighbours x 2 components), some of which is still
# in L2 when the kernel ends
DIVFREE_DRAM_BYTES_PER_TARGET = (33.947648e6 + 168.576256e6) / 147456


def flops_per_target(M, n, rows, iters):
    """Algorithmic FP32 flops of one target of the float-float kernel:
    QR 2Mn^2 - 2n^3/3; per functional row the initial solve (2n^2 triangular +
    4Mn for Q); per refinement iteration and row the residuals f = By - s and
    g = lambda - B^T s (2Mn compensated products) and the correction
    (2n^2 + 8Mn).  The float-float tile build is not counted."""
    f32 = (2 * M * n * n - 2 * n ** 3 / 3 + rows * (2 * n * n + 4 * M * n)
           + iters * rows * (2 * M * n * DOT2_FLOPS + 8 * M * n + 2 * n * n))
    return f32, 0.0


def flops_per_target_fp64(M, n, rows):
    """FP64 path: QR and the initial solve, all on the FP64 pipe."""
    return 2 * M * n * n - 2 * n ** 3 / 3 + rows * (2 * n * n + 4 * M * n)


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"gmls_clocks_{os.getpid()}.csv")

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return None
        try:
            rows = [r.split(", ") for r in open(self.path).read().strip().splitlines()]
            os.unlink(self.path)
        except OSError:
            return None
        rows = [r for r in rows if len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def workload_points():
    from paper_2104_14447_gb300 import inputs

    return inputs.jittered_grid(2, N_AXIS, seed=0)


def set_n_axis(v):
    """Grid size per axis (512 is the benchmark; smaller values only for profiling)."""
    global N_AXIS
    N_AXIS = int(v)


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2104_14447_gb300 import build, gmls, shard

    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prec = gmls.FP64 if args.precision == "fp64" else gmls.FP32_REFINE
    x_host = workload_points()
    n = x_host.shape[1]
    x_dev = torch.from_numpy(x_host).to(dev)
    ctx = gmls.Context(local_rank, arena_bytes=args.arena_gb << 30)
    stream = ctx.stream
    # output buffers of the three operators (sizes are fixed by k)
    nnz_grad, nnz_div, nnz_vl = n * K_SCALAR * 2, n * K_SCALAR * 2, n * K_DIVFREE * 2 * 2
    bufs = {}
    for name, rows, nnz in (("grad", 2 * n, nnz_grad), ("div", n, nnz_div), ("vl", 2 * n, nnz_vl)):
        bufs[name] = (torch.empty(rows + 1, dtype=torch.int64, device=dev),
                      torch.empty(nnz, dtype=torch.int32, device=dev),
                      torch.empty(nnz, dtype=torch.float64, device=dev))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    ev_k = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def step(x_src, k_events=None):
        cid = ctx.cloud(x_src)
        n48 = ctx.neighbors(cid, K_DIVFREE, EPS_FACTOR)
        n36 = ctx.neighbors_prefix(n48, K_SCALAR, EPS_FACTOR)  # the 36 nearest = first 36 of the 48
        s_sc = ctx.stencils(n36, gmls.SCALAR, DEGREE, [gmls.GRAD, gmls.DIV], precision=prec)
        if k_events:
            k_events[0].record(stream)
        s_df = ctx.stencils(n48, gmls.DIVFREE, DEGREE, [gmls.VEC_LAPLACIAN], precision=prec)
        if k_events:
            k_events[1].record(stream)
        ctx.assemble_csr(s_sc, gmls.GRAD, out=bufs["grad"])
        ctx.assemble_csr(s_sc, gmls.DIV, out=bufs["div"])
        ctx.assemble_csr(s_df, gmls.VEC_LAPLACIAN, out=bufs["vl"])
        return cid, n48, n36, s_sc, s_df

    def release(ids):
        for h in reversed(ids):
            ctx.release(h)

    for _ in range(args.warmup):
        release(step(x_dev))
    torch.cuda.synchronize()
    # refinement statistics of this workload (one untimed step)
    ids = step(x_dev)
    it_sc = ctx.export(ids[3], gmls.X_ITERS, torch.uint8).float()
    it_df = ctx.export(ids[4], gmls.X_ITERS, torch.uint8).float()
    st_df = ctx.export(ids[4], gmls.X_STATUS, torch.uint8)
    st_sc = ctx.export(ids[3], gmls.X_STATUS, torch.uint8)
    fb = int(((st_df & gmls.T_FP64_FALLBACK) != 0).sum()) + int(((st_sc & gmls.T_FP64_FALLBACK) != 0).sum())
    mean_it_sc, mean_it_df = float(it_sc.mean()), float(it_df.mean())
    release(ids)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    launches0 = ctx.launch_count()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local_rank) as clk:
        for s in range(args.steps):
            flush.fill_(s & 0xFF)  # evict L2 between timed steps (outside the events)
            ev[s][0].record(stream)
            ids = step(x_dev, kev[s])
            ev[s][1].record(stream)
            release(ids)
        torch.cuda.synchronize()
    launches = ctx.launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    kern_ms = [a.elapsed_time(b) for a, b in kev]
    total_ms = shard.max_over_ranks(float(np.sum(step_ms)), dev)

    # e2e: the same step through the C ABI from pinned host input to host operators
    x_pin = torch.from_numpy(x_host).pin_memory()
    host_out = {k: tuple(torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for v in bufs[k]) for k in bufs}
    d2h = sum(t.numel() * t.element_size() for v in bufs.values() for t in v)
    d2h += 8 * 3 * ((len(args.e2e_fractions.split(",")) if args.e2e_fractions else args.e2e_ranges) - 1)  # shared row pointers
    h2d = x_pin.numel() * x_pin.element_size()
    # The targets are processed in --e2e-ranges contiguous ranges so that the
    # operators of the first ranges travel to the host (on two copy streams)
    # while the GPU computes the rest: per range the 48-nearest lists, the
    # divergence-free stencils and their CSR rows; then per range the
    # 36-nearest prefix lists, the scalar stencils and the gradient and
    # divergence CSR rows.  Each range writes its rows in place in the
    # operator (gmls_assemble_csr_at), so the host receives the operators
    # themselves.
    copy_streams = [torch.cuda.Stream(dev) for _ in range(args.e2e_copy_streams)]
    if args.e2e_fractions:
        fr = np.array([float(v) for v in args.e2e_fractions.split(",")])
        bounds = [0] + [int(round(n * v)) for v in np.cumsum(fr / fr.sum())[:-1]] + [n]
    else:
        bounds = [n * c // args.e2e_ranges for c in range(args.e2e_ranges + 1)]
    n_ranges = len(bounds) - 1
    chunk_tg = [torch.arange(a, b, dtype=torch.int32, device=dev) for a, b in zip(bounds[:-1], bounds[1:])]
    per_target = {"vl": (2, K_DIVFREE * 2), "grad": (2, K_SCALAR), "div": (1, K_SCALAR * 2)}  # rows, nnz per row

    def chunk_views(kname, c):
        """(device views, host views, nonzero offset) of range c's rows."""
        rows, per_row = per_target[kname]
        a, b = bounds[c], bounds[c + 1]
        lo, hi = a * rows * per_row, b * rows * per_row
        rp, col, val = bufs[kname]
        hrp, hcol, hval = host_out[kname]
        sl_r, sl_n = slice(a * rows, b * rows + 1), slice(lo, hi)
        return (rp[sl_r], col[sl_n], val[sl_n]), (hrp[sl_r], hcol[sl_n], hval[sl_n]), lo

    def assemble_and_ship(sid, fn, kname, c, which):
        dev_out, host_dst, lo = chunk_views(kname, c)
        ctx.assemble_csr(sid, fn, out=dev_out, nnz_offset=lo)
        done = torch.cuda.Event()
        done.record(stream)
        cs = copy_streams[which]
        cs.wait_event(done)
        with torch.cuda.stream(cs):
            for dst, src in zip(host_dst, dev_out):
                dst.copy_(src, non_blocking=True)

    def step_e2e(x_src):
        cid = ctx.cloud(x_src)
        ids = [cid]
        n48s = []
        for c in range(n_ranges):
            n48 = ctx.neighbors(cid, K_DIVFREE, EPS_FACTOR, targets=chunk_tg[c])
            s_df = ctx.stencils(n48, gmls.DIVFREE, DEGREE, [gmls.VEC_LAPLACIAN], precision=prec)
            assemble_and_ship(s_df, gmls.VEC_LAPLACIAN, "vl", c, c % len(copy_streams))
            n48s.append(n48)
            ids += [n48, s_df]
        for c in range(n_ranges):
            n36 = ctx.neighbors_prefix(n48s[c], K_SCALAR, EPS_FACTOR)
            s_sc = ctx.stencils(n36, gmls.SCALAR, DEGREE, [gmls.GRAD, gmls.DIV], precision=prec)
            assemble_and_ship(s_sc, gmls.GRAD, "grad", c, (2 * c) % len(copy_streams))
            assemble_and_ship(s_sc, gmls.DIV, "div", c, (2 * c + 1) % len(copy_streams))
            ids += [n36, s_sc]
        return ids

    def release_e2e(ids):
        for h in reversed(ids):
            ctx.release(h)

    e2e_ms = []
    for s in range(max(3, min(args.steps, 7)) + 1):
        flush.fill_(s & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ids = step_e2e(x_pin)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        release_e2e(ids)
    e2e_ms = e2e_ms[1:]
    # the host operators equal the device step's (checked once, untimed)
    ids = step(x_dev)
    torch.cuda.synchronize()
    e2e_equal = all(torch.equal(h, d.cpu()) for k in bufs for h, d in zip(host_out[k], bufs[k]))
    release(ids)

    # roofline of the dominant kernel (the divergence-free stencil launch)
    M_df, n_df, rows_df = K_DIVFREE * 2, 20, 2
    k_avg = float(np.mean(kern_ms)) * 1e-3
    if prec == gmls.FP32_REFINE:
        f32, _ = flops_per_target(M_df, n_df, rows_df, mean_it_df)
        flops, peak, pipe = n * f32, P32_TFLOPS, "fp32"
    else:
        f64 = flops_per_target_fp64(M_df, n_df, rows_df)
        flops, peak, pipe = n * f64, P64_TFLOPS, "fp64"
    achieved = flops / k_avg / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": n * DIVFREE_DRAM_BYTES_PER_TARGET if prec == gmls.FP32_REFINE else None,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch on the "
                                  "384 x 384 grid, per target, times the targets of this launch",
                "kernel": "stencil_fast_kernel<divfree, 2D, m=4> (96x20 systems)"
                if prec == gmls.FP32_REFINE else "stencil_kernel<double> (96x20 systems)",
                "pipe": pipe, "flops_per_target": flops / n, "mean_refine_iters": mean_it_df,
                "peak_source": "unit counts x 2070 MHz (152 SMs x 128 FP32 lanes; FP64 1/64 of that)",
                "kernel_ms": k_avg * 1e3}
    # the same step captured once as a CUDA graph and replayed
    graph_ms = None
    if args.graph:
        gstream = torch.cuda.Stream(dev)
        gctx = gmls.Context(local_rank, arena_bytes=args.arena_gb << 30, stream=gstream)
        with torch.cuda.stream(gstream):
            ids_g = None
            ctx_save = ctx
            # one eager run on this context fills its autotuner cache, then capture
            for capture in (False, True):
                if capture:
                    gctx.capture_begin()
                cid = gctx.cloud(x_dev)
                n48 = gctx.neighbors(cid, K_DIVFREE, EPS_FACTOR)
                n36 = gctx.neighbors_prefix(n48, K_SCALAR, EPS_FACTOR)
                s_sc = gctx.stencils(n36, gmls.SCALAR, DEGREE, [gmls.GRAD, gmls.DIV], precision=prec)
                s_df = gctx.stencils(n48, gmls.DIVFREE, DEGREE, [gmls.VEC_LAPLACIAN], precision=prec)
                gctx.assemble_csr(s_sc, gmls.GRAD, out=bufs["grad"])
                gctx.assemble_csr(s_sc, gmls.DIV, out=bufs["div"])
                gctx.assemble_csr(s_df, gmls.VEC_LAPLACIAN, out=bufs["vl"])
                if capture:
                    gid = gctx.capture_end()
                    ids_g = (cid, n48, n36, s_sc, s_df)
                else:
                    gctx.sync()
                    for h in (s_df, s_sc, n36, n48, cid):
                        gctx.release(h)
            for _ in range(3):
                gctx.graph_launch(gid)
            gstream.synchronize()
            gms = []
            for s_ in range(args.steps):
                flush.fill_(s_ & 0xFF)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(gstream)
                gctx.graph_launch(gid)
                b.record(gstream)
                gms.append((a, b))
            gstream.synchronize()
            graph_ms = float(np.mean([a.elapsed_time(b) for a, b in gms]))
            gctx.release(gid)
            for h in reversed(ids_g):
                gctx.release(h)
        gctx.close()
        del ctx_save

    tune = {}
    for r in ctx.tune_log():
        key = f"{'scalar' if r['basis'] == 0 else 'divfree'} m={r['degree']} rows<={r['rows']}"
        v = r["variant"]
        place = {0: "", 1: ", split tiles", 2: ", global tiles"}[v >> 3] if v > 0 else ""
        name = {-1: "register", -2: "register 16 lanes", -3: "factored div-free"}.get(v, f"{v & 7} warp(s)/target{place}")
        tune.setdefault(key, {})[name] = round(r["ms"], 3)

    value = shard.job_throughput(n, args.steps, world, total_ms)
    out = {
        "metric": METRIC, "value": value, "unit": "targets/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if prec == gmls.FP32_REFINE else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "targets_per_gpu": n, "precision": args.precision,
                   "degree": DEGREE, "neighbours": [K_SCALAR, K_DIVFREE], "eps_factor": EPS_FACTOR,
                   "weight": "(1-r/eps)_+^4", "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"independent replicas x{world}" if world > 1 else "1 GPU"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "e2e": {"value": n * world / (float(np.median(e2e_ms)) * 1e-3), "unit": "targets/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": float(np.median(e2e_ms)), "ms_steps": [round(v, 3) for v in e2e_ms], "target_ranges": n_ranges, "range_bounds": bounds,
                "host_operators_equal_device_step": e2e_equal},
        "gpu_launches": int(launches),
        "refinement": {"mean_iters_scalar": mean_it_sc, "mean_iters_divfree": mean_it_df, "fp64_fallback_targets": fb},
        "roofline": roofline,
        "clocks": clk.summary(),
        "autotune_ms": tune,
    }
    if graph_ms is not None:
        out["graph"] = {"ms_per_step": graph_ms, "targets_per_s": n * world / (graph_ms * 1e-3)}
    return out, ctx


SERVE_K = {(2, 0, 2): 12, (2, 0, 3): 20, (2, 0, 4): 36, (2, 1, 2): 22, (2, 1, 3): 34, (2, 1, 4): 48,
           (3, 0, 2): 20, (3, 0, 3): 40, (3, 0, 4): 84, (3, 1, 2): 42, (3, 1, 3): 80, (3, 1, 4): 136}


def stokes_system(ctx, steps=5):
    """The Stokes collocation system (Sec. 3.2) on the benchmark grid with the
    outermost lattice layer as the Dirichlet / Neumann boundary: stencils
    (curl curl on the divergence-free basis; gradient and Neumann-constrained
    Laplacian on the scalar basis), then per timed step assembly of the block
    CSR, its right-hand side and one A x.  Reports times, bytes moved against
    the measured HBM peak, and the manufactured-field residual."""
    import torch

    from paper_2104_14447_gb300 import gmls, inputs

    x = workload_points()
    n = x.shape[1]
    bflag, nrm = inputs.box_boundary(2, N_AXIS)
    d = inputs.stokes_manufactured_2d(x, 1.0)
    stream = ctx.stream
    cid = ctx.cloud(x, normals=nrm, bflags=bflag)
    nv = ctx.neighbors(cid, K_DIVFREE, EPS_FACTOR)
    npr = ctx.neighbors_prefix(nv, K_SCALAR, EPS_FACTOR)
    sv = ctx.stencils(nv, gmls.DIVFREE, DEGREE, [gmls.CURLCURL], precision=gmls.FP32_REFINE)
    sp = ctx.stencils(npr, gmls.SCALAR, DEGREE, [gmls.GRAD, gmls.LAPLACIAN], precision=gmls.FP32_REFINE,
                      neumann=True)
    n_rows, nnz = ctx.stokes_size(sv, sp, 1.0)
    rp = torch.empty(n_rows + 1, dtype=torch.int64, device=ctx.device)
    col = torch.empty(nnz, dtype=torch.int32, device=ctx.device)
    val = torch.empty(nnz, dtype=torch.float64, device=ctx.device)
    f, w, div_f = (torch.from_numpy(np.ascontiguousarray(a)).to(ctx.device) for a in (d["f"], d["w"], d["div_f"]))
    xe = torch.from_numpy(np.concatenate([d["u"].T.reshape(-1), d["p"], [0.0]])).to(ctx.device)
    b = torch.empty(n_rows, dtype=torch.float64, device=ctx.device)
    y = torch.empty(n_rows, dtype=torch.float64, device=ctx.device)
    P = gmls.StokesParams(sv, sp, 1.0)
    lib, h = ctx.lib, ctx.h
    import ctypes

    ptr = lambda t: ctypes.c_void_p(t.data_ptr())

    def assemble():
        ctx._check(lib.gmls_stokes_assemble(h, ctypes.byref(P), ptr(rp), ptr(col), ptr(val)))
        ctx._check(lib.gmls_stokes_rhs(h, ctypes.byref(P), ptr(f), ptr(w), ptr(div_f), ptr(b)))

    def spmv():
        ctx._check(lib.gmls_csr_spmv(h, n_rows, ptr(rp), ptr(col), ptr(val), ptr(xe), ptr(y)))

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=ctx.device)
    for _ in range(2):
        assemble()
        spmv()
    ta, tm = [], []
    for s in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(s & 0xFF)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            assemble()
            e[1].record(stream)
            spmv()
            e[2].record(stream)
        torch.cuda.synchronize()
        ta.append(e[0].elapsed_time(e[1]))
        tm.append(e[1].elapsed_time(e[2]))
    r = (y - b).cpu().numpy()
    bf = bflag.astype(bool)
    mom = np.abs(r[:2 * n]).reshape(n, 2)
    pr = np.abs(r[2 * n:3 * n])
    nb = int(np.sum(bf))
    # bytes: assembly reads the weights it scatters (nnz doubles, mostly) and
    # both neighbour lists, writes col + val + row_ptr; A x reads val, col,
    # row_ptr, writes y (x, 6.3 MB, stays in L2)
    asm_bytes = nnz * (8 + 4 + 8) + (n_rows + 1) * 8 + n * (K_DIVFREE + K_SCALAR) * 4 + n_rows * 8
    spmv_bytes = nnz * (8 + 4) + (n_rows + 1) * 8 + n_rows * 8 + n_rows * 8
    peaks, src = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    ta_m, tm_m = float(np.median(ta)), float(np.median(tm))
    for hd in (sp, sv, npr, nv, cid):
        ctx.release(hd)
    return {"workload": f"stokes2d-{N_AXIS}x{N_AXIS} collocation system, {nb} boundary points, nu = 1",
            "n_rows": n_rows, "nnz": nnz, "assemble_ms": ta_m, "spmv_ms": tm_m,
            "assemble_gbs": asm_bytes / ta_m / 1e6, "spmv_gbs": spmv_bytes / tm_m / 1e6,
            "spmv_frac_hbm": spmv_bytes / tm_m / 1e6 / hbm, "peak_source": src,
            "residual_max": {"momentum_interior": float(mom[~bf].max()), "pressure_interior": float(pr[~bf].max()),
                             "pressure_boundary": float(pr[bf].max()), "dirichlet": float(mom[bf].max())},
            "l2": "flushed before each timed step (256 MB write)"}


def shapes(ctx):
    """Stencil stage of every (dimension, basis, degree) shape the serving
    stream draws, and of the staggered basis, on one cloud per dimension (2D: 400 x 400 jittered grid,
    160,000 targets; 3D: 50^3, 125,000), FP32 + refinement against plain
    FP64 (the same launch path with GMLS_FP64), CUDA events around one
    gmls_stencils call after a warm-up call; the kernel variant the
    autotuner chose for the FP32 path."""
    import torch

    from paper_2104_14447_gb300 import gmls, inputs

    out = {}
    for dim, n_axis in ((2, 400), (3, 50)):
        x = inputs.jittered_grid(dim, n_axis, seed=1)
        n = x.shape[1]
        cid = ctx.cloud(x)
        # the serving shapes, then the staggered basis (Sec. 2.4; gradient and
        # Laplacian of the line-integral potential)
        cases = [((d, b, m), k) for (d, b, m), k in SERVE_K.items()]
        cases += [((2, gmls.STAGGERED, 2), 24), ((2, gmls.STAGGERED, 3), 36), ((2, gmls.STAGGERED, 4), 48),
                  ((3, gmls.STAGGERED, 2), 40)]
        for (d, b, m), k in cases:
            if d != dim:
                continue
            fns = [gmls.VEC_LAPLACIAN] if b == gmls.DIVFREE else [gmls.GRAD, gmls.LAPLACIAN]
            nid = ctx.neighbors(cid, k, EPS_FACTOR)
            ms = {}
            for name, prec in (("fp32_refine", gmls.FP32_REFINE), ("fp64", gmls.FP64)):
                ctx.release(ctx.stencils(nid, b, m, fns, precision=prec))  # warm-up / autotune
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(ctx.stream)
                sid = ctx.stencils(nid, b, m, fns, precision=prec)
                e1.record(ctx.stream)
                torch.cuda.synchronize()
                ms[name] = e0.elapsed_time(e1)
                ctx.release(sid)
            ctx.release(nid)
            rows = k * (d if b == gmls.DIVFREE else 1)
            tl = [r for r in ctx.tune_log() if r["dim"] == d and r["basis"] == b and r["degree"] == m
                  and r["precision"] == gmls.FP32_REFINE and r["rows"] == rows and not r["bucketed"]]
            v = min(tl, key=lambda r: r["ms"])["variant"] if tl else None
            name = None if v is None else ({-1: "register", -2: "register 16 lanes"}.get(v) or
                                           f"{v & 7} warp(s)/target" + {0: "", 1: ", split tiles",
                                                                        2: ", global tiles"}[v >> 3])
            key = f"{d}d {['scalar', 'divfree', 'staggered'][b]} m={m} k={k}"
            out[key] = {"targets": n, "system": f"{rows} x {gmls_basis_size(d, b, m)}",
                        "fp32_refine_Mtargets_s": n / ms["fp32_refine"] / 1e3, "fp64_Mtargets_s": n / ms["fp64"] / 1e3,
                        "speedup": ms["fp64"] / ms["fp32_refine"], "fp32_variant": name}
        ctx.release(cid)
    return out


def gmls_basis_size(d, b, m):
    """Number of basis functions: scalar Taylor C(m + d, d); divergence-free
    vector polynomials of degree <= m in d dimensions; staggered: monomials of
    degree 1..m+1 (the span of the line integrals of the vector monomials)."""
    from math import comb

    if b == 0:
        return comb(m + d, d)
    if b == 2:
        return comb(m + 1 + d, d) - 1
    full = d * comb(m + d, d)
    return full - (comb(m - 1 + d, d))  # minus the divergence map's rank (onto degree m - 1)


def porous_stokes(ctx, pc, n80, n40, ssc, flush, steps=3, nu=1.0):
    """The 3D Stokes collocation system (Sec. 3.2) on the porous cube, from
    the porous step's neighbour lists and Neumann-constrained scalar stencils
    plus degree-3 divergence-free curl curl stencils: assembly + right-hand
    side and one A x, CUDA events on the context stream, L2 flushed, bytes
    against the measured HBM rate; then, at full size, the residual of the
    cubic Stokes data (inputs.stokes_cubic_3d, inside the degree-3 bases, so
    every row but the zero-mean one holds up to the stencils' rounding),
    relative to sum |a| |x| + |b| per row."""
    import ctypes

    import torch

    from paper_2104_14447_gb300 import gmls, inputs

    x = pc["x"]
    n = x.shape[1]
    stream = ctx.stream
    scc = ctx.stencils(n80, gmls.DIVFREE, 3, [gmls.CURLCURL], precision=gmls.FP32_REFINE)
    n_rows, nnz = ctx.stokes_size(scc, ssc, nu)
    rp = torch.empty(n_rows + 1, dtype=torch.int64, device=ctx.device)
    col = torch.empty(nnz, dtype=torch.int32, device=ctx.device)
    val = torch.empty(nnz, dtype=torch.float64, device=ctx.device)
    d = inputs.stokes_cubic_3d(x, nu)
    f, w, div_f = (torch.from_numpy(np.ascontiguousarray(a)).to(ctx.device) for a in (d["f"], d["w"], d["div_f"]))
    xe = torch.from_numpy(np.concatenate([d["u"].T.reshape(-1), d["p"], [0.0]])).to(ctx.device)
    b = torch.empty(n_rows, dtype=torch.float64, device=ctx.device)
    y = torch.empty(n_rows, dtype=torch.float64, device=ctx.device)
    P = gmls.StokesParams(scc, ssc, nu)
    lib, h = ctx.lib, ctx.h
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())

    def assemble():
        ctx._check(lib.gmls_stokes_assemble(h, ctypes.byref(P), ptr(rp), ptr(col), ptr(val)))
        ctx._check(lib.gmls_stokes_rhs(h, ctypes.byref(P), ptr(f), ptr(w), ptr(div_f), ptr(b)))

    def spmv(v, xv, out):
        ctx._check(lib.gmls_csr_spmv(h, n_rows, ptr(rp), ptr(col), ptr(v), ptr(xv), ptr(out)))

    assemble()
    spmv(val, xe, y)
    ta, tm = [], []
    for s in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(s & 0xFF)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            assemble()
            e[1].record(stream)
            spmv(val, xe, y)
            e[2].record(stream)
        torch.cuda.synchronize()
        ta.append(e[0].elapsed_time(e[1]))
        tm.append(e[1].elapsed_time(e[2]))
    with torch.cuda.stream(stream):
        scale = torch.empty_like(y)
        aval = val.abs()
        spmv(aval, xe.abs(), scale)
        del aval
        rel = (y - b).abs() / (scale + b.abs())
        bf = torch.from_numpy(pc["bflag"].astype(bool)).to(ctx.device)
        mom = rel[:3 * n].reshape(n, 3).amax(dim=1)
        pr = rel[3 * n:4 * n]
        res = {"momentum_interior": float(mom[~bf].max()), "dirichlet": float(mom[bf].max()),
               "pressure_interior": float(pr[~bf].max()), "pressure_boundary": float(pr[bf].max())}
    torch.cuda.synchronize()
    ctx.release(scc)
    peaks, src = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    asm_bytes = nnz * (8 + 4 + 8) + (n_rows + 1) * 8 + n * (80 + 40) * 4 + n_rows * 8
    spmv_bytes = nnz * (8 + 4) + (n_rows + 1) * 8 + 2 * n_rows * 8
    ta_m, tm_m = float(np.median(ta)), float(np.median(tm))
    return {"system": f"{n_rows} rows ({n} points x 3 velocity + pressure + multiplier), nu = {nu}",
            "n_rows": n_rows, "nnz": nnz, "assemble_ms": ta_m, "spmv_ms": tm_m,
            "assemble_gbs": asm_bytes / ta_m / 1e6, "spmv_gbs": spmv_bytes / tm_m / 1e6,
            "spmv_frac_hbm": spmv_bytes / tm_m / 1e6 / hbm, "peak_source": src,
            "cubic_data_max_rel_residual": res,
            "l2": "flushed before each timed step (256 MB write)"}


def porous_3d(ctx, n_axis=128, steps=3, n_sample=48, stokes=True):
    """The 3D porous-medium workload: a jittered n_axis^3 lattice in the unit
    cube minus 64 random non-overlapping spheres, boundary targets on the
    sphere surfaces and cube faces with their geometric normals.  Per step:
    kNN-80 lists and their 40-nearest prefix, degree-3 scalar stencils
    (gradient, Laplacian; Neumann constraint at boundary targets), degree-3
    divergence-free stencils (vector Laplacian, 240 x 50 systems), FP32 with
    float-float refinement, and the three CSR operators.  Device-timed per
    stage with CUDA events on the context stream, inputs resident, L2 flushed
    before each step; stencil errors on a sample of boundary and interior
    targets against the oracle."""
    import torch

    from paper_2104_14447_gb300 import gmls, inputs

    pc = inputs.porous_cube(n_axis=n_axis)
    x = pc["x"]
    n = x.shape[1]
    stream = ctx.stream
    cid = ctx.cloud(x, normals=pc["normals"], bflags=pc["bflag"])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=ctx.device)
    prec = gmls.FP32_REFINE

    def step(ev=None):
        rec = (lambda i: ev[i].record(stream)) if ev else (lambda i: None)
        rec(0)
        n80 = ctx.neighbors(cid, 80, EPS_FACTOR)
        n40 = ctx.neighbors_prefix(n80, 40, EPS_FACTOR)
        rec(1)
        ssc = ctx.stencils(n40, gmls.SCALAR, 3, [gmls.GRAD, gmls.LAPLACIAN], precision=prec, neumann=True)
        rec(2)
        sdf = ctx.stencils(n80, gmls.DIVFREE, 3, [gmls.VEC_LAPLACIAN], precision=prec)
        rec(3)
        csr = [ctx.assemble_csr(ssc, gmls.GRAD), ctx.assemble_csr(ssc, gmls.LAPLACIAN),
               ctx.assemble_csr(sdf, gmls.VEC_LAPLACIAN)]
        rec(4)
        return n80, n40, ssc, sdf, csr

    def release(h):
        for hd in (h[3], h[2], h[1], h[0]):
            ctx.release(hd)

    release(step())  # warm-up (autotunes the two shapes)
    torch.cuda.synchronize()
    times = []
    for s in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(s & 0xFF)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        torch.cuda.nvtx.range_push("porous_step")  # lets a profiler select the timed launches
        h = step(ev)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        times.append([ev[i].elapsed_time(ev[i + 1]) for i in range(4)])
        if s < steps - 1:
            release(h)
    med = np.median(np.array(times), axis=0)
    step_ms = float(np.sum(med))
    st_sc = ctx.export(h[2], gmls.X_STATUS, torch.uint8).cpu().numpy()
    st_df = ctx.export(h[3], gmls.X_STATUS, torch.uint8).cpu().numpy()
    # GPU outputs of a sample of boundary and interior targets, for the
    # oracle comparison of the CPU-baseline leg (porous_oracle_errors)
    bidx = np.flatnonzero(pc["bflag"])
    iidx = np.flatnonzero(pc["bflag"] == 0)
    half = n_sample // 2
    sample = np.unique(np.concatenate([bidx[(inputs.uniform(2, 96, half) * len(bidx)).astype(np.int64)],
                                       iidx[(inputs.uniform(2, 97, half) * len(iidx)).astype(np.int64)]]))
    sample = sample.astype(np.int32)
    gpu_sample = {"x": x, "bflag": pc["bflag"], "normals": pc["normals"], "sample": sample, "ops": []}
    for key, nh, sh, k, kind, code in (("grad", h[1], h[2], 40, "scalar", gmls.GRAD),
                                       ("laplacian", h[1], h[2], 40, "scalar", gmls.LAPLACIAN),
                                       ("vec_laplacian", h[0], h[3], 80, "divfree", gmls.VEC_LAPLACIAN)):
        idx = ctx.export(nh, gmls.X_NBR_INDEX, torch.int32).cpu().numpy().reshape(n, k)[sample]
        _, rows, nc, _ = ctx.stencil_info(sh, code)
        wg = ctx.weights(sh, code).cpu().numpy().reshape(n, rows, k, nc)[sample]
        gpu_sample["ops"].append((key, k, kind, idx, wg))
    stokes_out = None
    if stokes:
        ctx.release(h[3])  # the vector Laplacian stencils and the step's CSR operators: room for the system
        h[4].clear()
        stokes_out = porous_stokes(ctx, pc, h[0], h[1], h[2], flush)
        for hd in (h[2], h[1], h[0]):
            ctx.release(hd)
    else:
        release(h)
    ctx.release(cid)
    tune = {}
    for r in ctx.tune_log():
        if r["dim"] == 3 and r["degree"] == 3 and not r["bucketed"]:
            v = r["variant"]
            place = {0: "", 1: ", split tiles", 2: ", global tiles"}[v >> 3] if v > 0 else ""
            name = {-1: "register", -2: "register 16 lanes", -3: "factored div-free"}.get(v, f"{v & 7} warp(s)/target{place}")
            key = f"{'scalar' if r['basis'] == 0 else 'divfree'} m=3 rows<={r['rows']}"
            tune.setdefault(key, {})[name] = round(r["ms"], 3)
    qr_flops = 2 * 240 * 50 ** 2 - 2 * 50 ** 3 / 3  # Householder QR of one 240 x 50 system
    return {"workload": f"porous cube {n_axis}^3 lattice minus 64 spheres: {n} points, "
                        f"{int(pc['bflag'].sum())} on a boundary, degree 3, k = 40 / 80, FP32 + refinement",
            "targets": n, "porosity": float(pc["porosity"]), "step_ms": step_ms, "targets_per_s": n / step_ms * 1e3,
            "stage_ms": {"neighbours": float(med[0]), "scalar_stencils": float(med[1]),
                         "divfree_stencils": float(med[2]), "csr": float(med[3])},
            "divfree_targets_per_s": n / float(med[2]) * 1e3,
            "divfree_qr_tflops": qr_flops * n / float(med[2]) / 1e9,
            "fp64_redo": {"scalar": int(np.sum((st_sc & gmls.T_FP64_FALLBACK) != 0)),
                          "divfree": int(np.sum((st_df & gmls.T_FP64_FALLBACK) != 0))},
            "tune_ms": tune, "l2": "flushed before each timed step (256 MB write)",
            "stokes_system": stokes_out}, gpu_sample


def porous_oracle_errors(gs):
    """CPU-baseline leg of the porous section: the oracle's kNN lists and
    stencils on the sampled targets against the GPU's."""
    import oracle

    x, sample = gs["x"], gs["sample"]
    errs, lists_equal = {}, True
    for key, k, kind, idx, wg in gs["ops"]:
        oi, oe = oracle.knn(x, sample, k, EPS_FACTOR, method="grid")
        lists_equal &= bool(np.array_equal(idx, oi))
        off = np.arange(0, len(sample) * k + 1, k)
        extra = dict(bflag=gs["bflag"][sample], normals=gs["normals"].T[sample]) if kind == "scalar" else {}
        wo, _, _ = oracle.stencils(x, sample, off, oi.reshape(-1), oe, kind, 3, key, **extra)
        w = wg.reshape(wo.shape)
        a = np.abs(w - wo).reshape(len(sample), wo.shape[1], -1).max(axis=2)
        b = np.abs(wo).reshape(len(sample), wo.shape[1], -1).max(axis=2)
        errs[key] = float(np.max(a / np.where(b > 0, b, 1.0)))
    return {"sample": f"{len(sample)} targets, half drawn from the boundary, half from the interior",
            "neighbour_lists_equal_oracle": lists_equal, "max_rel_err_vs_oracle": errs}


BASIS_SIZE = {(2, 2): 6, (2, 3): 10, (2, 4): 15, (3, 2): 10, (3, 3): 20, (3, 4): 35}


def batched_uneven(ctx, n_per_dim=500_000, steps=3, n_sample=32):
    """The uneven batch: a 2D and a 3D jittered cloud of n_per_dim targets
    each, degree U{2,3,4} per target, radius lists at 1.8 x the distance of
    the Q(d, m)-th nearest neighbour (Q the basis size, at most 160 entries),
    20 % one-sided targets (half-space filter).  Per cloud one bucketed
    persistent stencil launch (scalar basis; gradient and Laplacian) and the
    gradient CSR; FP32 + refinement timed per stage over `steps` steps (L2
    flushed before each), one FP64 step beside it."""
    import torch

    from paper_2104_14447_gb300 import gmls, inputs

    clouds = inputs.mixed_batch(n_per_dim)
    stream = ctx.stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=ctx.device)
    prepared = []
    for c in clouds:
        d = c["dim"]
        kpt = np.array([BASIS_SIZE[(d, int(m))] for m in c["degree"]], dtype=np.int32)
        cid = ctx.cloud(c["x"])
        prepared.append((c, cid, torch.from_numpy(c["halfspace"]).to(ctx.device),
                         torch.from_numpy(kpt).to(ctx.device), torch.from_numpy(c["degree"]).to(ctx.device)))

    def step(prec, ev=None):
        rec = (lambda i: ev[i].record(stream)) if ev else (lambda i: None)
        hs_out = []
        rec(0)
        for c, cid, hs, kpt, deg in prepared:
            nid = ctx.neighbors(cid, 35 if c["dim"] == 3 else 15, 1.8, mode=gmls.RADIUS, cap=160, halfspace=hs,
                                k_per_target=kpt)
            hs_out.append([nid])
        rec(1)
        for (c, cid, hs, kpt, deg), h in zip(prepared, hs_out):
            h.append(ctx.stencils(h[0], gmls.SCALAR, 0, [gmls.GRAD, gmls.LAPLACIAN], precision=prec,
                                  degree_per_target=deg))
        rec(2)
        for h in hs_out:
            h.append(ctx.assemble_csr(h[1], gmls.GRAD))
        rec(3)
        return hs_out

    def release(hs_out):
        for h in hs_out:
            ctx.release(h[1])
            ctx.release(h[0])

    release(step(gmls.FP32_REFINE))  # warm-up: autotunes every (degree, row class) bucket
    torch.cuda.synchronize()
    res = {}
    for name, prec, nsteps in (("fp32_refine", gmls.FP32_REFINE, steps), ("fp64", gmls.FP64, 1)):
        if prec == gmls.FP64:
            release(step(prec))  # its own warm-up (bucket choices of the FP64 kernel)
        times = []
        for s in range(nsteps):
            with torch.cuda.stream(stream):
                flush.fill_(s & 0xFF)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            torch.cuda.nvtx.range_push("batched_step")
            h = step(prec, ev)
            torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
            times.append([ev[i].elapsed_time(ev[i + 1]) for i in range(3)])
            if not (prec == gmls.FP32_REFINE and s == nsteps - 1):
                release(h)
        med = np.median(np.array(times), axis=0)
        res[name] = {"step_ms": float(np.sum(med)), "targets_per_s": 2 * n_per_dim / float(np.sum(med)) * 1e3,
                     "stage_ms": {"neighbours": float(med[0]), "stencils": float(med[1]), "csr": float(med[2])}}
        if prec == gmls.FP32_REFINE:
            keep = h
    stats, gpu_sample = {}, []
    for (c, cid, hs, kpt, deg), h in zip(prepared, keep):
        d = c["dim"]
        off = ctx.export(h[0], gmls.X_NBR_OFFSETS, torch.int64).cpu().numpy()
        nst = ctx.export(h[0], gmls.X_NBR_STATUS, torch.uint8).cpu().numpy()
        st = ctx.export(h[1], gmls.X_STATUS, torch.uint8).cpu().numpy()
        cnt = np.diff(off)
        stats[f"{d}d"] = {"neighbours_min": int(cnt.min()), "neighbours_mean": float(cnt.mean()),
                          "neighbours_max": int(cnt.max()),
                          "too_few_neighbours": int(np.sum((nst & gmls.T_TOO_FEW_NEIGHBOURS) != 0)),
                          "rank_deficient": int(np.sum((st & gmls.T_RANK_DEFICIENT) != 0)),
                          "fp64_redo": int(np.sum((st & gmls.T_FP64_FALLBACK) != 0)),
                          "one_sided": int(c["one_sided"].sum())}
        # GPU outputs of a sample (half one-sided) for the CPU-baseline leg's oracle check
        ok = np.flatnonzero((nst == 0) & ((st & (gmls.T_RANK_DEFICIENT | gmls.T_UNSUPPORTED)) == 0))
        os_ = ok[c["one_sided"][ok]]
        ins = ok[~c["one_sided"][ok]]
        half = n_sample // 2
        sample = np.unique(np.concatenate([os_[(inputs.uniform(3, 90 + d, half) * len(os_)).astype(np.int64)],
                                           ins[(inputs.uniform(3, 92 + d, half) * len(ins)).astype(np.int64)]]))
        idx = ctx.export(h[0], gmls.X_NBR_INDEX, torch.int32).cpu().numpy()
        wgrad = ctx.weights(h[1], gmls.GRAD).cpu().numpy()
        lists = [idx[off[t]:off[t + 1]] for t in sample]
        ws = [wgrad[off[t] * d:off[t + 1] * d] for t in sample]
        gpu_sample.append({"dim": d, "x": c["x"], "degree": c["degree"], "halfspace": c["halfspace"],
                           "sample": sample.astype(np.int32), "lists": lists, "w": ws})
    release(keep)
    for _, cid, _, _, _ in prepared:
        ctx.release(cid)
    tune = {}
    for r in ctx.tune_log():
        if r["bucketed"]:
            v = r["variant"]
            place = {0: "", 1: ", split", 2: ", global"}[v >> 3]
            key = f"{r['dim']}d m={r['degree']} rows<={r['rows']}{' fp64' if r['precision'] == gmls.FP64 else ''}"
            tune.setdefault(key, {})[f"{v & 7}w{place}"] = round(r["ms"], 3)
    return {"workload": f"uneven batch: 2D and 3D jittered clouds of {n_per_dim} targets each, degree U{{2,3,4}}, "
                        "radius lists at 1.8 x the Q(d,m)-th neighbour distance (<= 160), 20 % one-sided, "
                        "scalar basis (gradient, Laplacian), one bucketed launch per cloud",
            "targets": 2 * n_per_dim, **res, "speedup_vs_fp64": res["fp64"]["step_ms"] / res["fp32_refine"]["step_ms"],
            "stats": stats, "tune_ms": tune, "l2": "flushed before each timed step (256 MB write)"}, gpu_sample


def batched_oracle_errors(gsamples):
    """CPU-baseline leg of the uneven batch: the oracle's radius lists and
    gradient stencils of the sampled targets against the GPU's."""
    import oracle

    out = {}
    for g in gsamples:
        d, x, sample = g["dim"], g["x"], g["sample"]
        lists_equal, worst = True, 0.0
        for m in (2, 3, 4):
            qs = np.flatnonzero(g["degree"][sample] == m)
            if len(qs) == 0:
                continue
            tg = sample[qs]
            hs = g["halfspace"][tg]
            _, oe = oracle.knn(x, tg, BASIS_SIZE[(d, m)], 1.8, halfspace=hs, method="grid")
            ooff, oidx = oracle.radius(x, tg, oe, 160, halfspace=hs, method="grid")
            wo, _, _ = oracle.stencils(x, tg, ooff, oidx, oe, "scalar", m, "grad")
            for r, q in enumerate(qs):
                lists_equal &= bool(np.array_equal(oidx[ooff[r]:ooff[r + 1]], g["lists"][q]))
                w = g["w"][q].reshape(wo[r].shape)
                worst = max(worst, float(np.max(np.abs(w - wo[r])) / np.max(np.abs(wo[r]))))
        out[f"{d}d"] = {"sample": f"{len(sample)} targets, half one-sided", "lists_equal_oracle": lists_equal,
                        "max_rel_err_vs_oracle": worst}
    return out


def stokes_solve(ctx, n_axis=128, full=True):
    """Global solve of the Stokes system (Sec. 3.3) on an n_axis^2 grid by
    GMRES(100) with right Jacobi preconditioning (gmls_gmres), to a relative
    residual of 1e-10; RMS errors of the solved velocity and (mean-free)
    pressure against the manufactured field.  full: solved three times --
    interior pressure rows from the scalar Laplacian, then from the
    staggered one (Sec. 3.2; its stencil time is that of a first call), then
    the first system on its equilibrated rows (row_scaling); else only the
    last of these."""
    import torch

    from paper_2104_14447_gb300 import gmls, inputs

    x = inputs.jittered_grid(2, n_axis, seed=0)
    n = x.shape[1]
    bflag, nrm = inputs.box_boundary(2, n_axis)
    d = inputs.stokes_manufactured_2d(x, 1.0)
    cid = ctx.cloud(x, normals=nrm, bflags=bflag)
    nv = ctx.neighbors(cid, K_DIVFREE, EPS_FACTOR)
    npr = ctx.neighbors_prefix(nv, K_SCALAR, EPS_FACTOR)
    sv = ctx.stencils(nv, gmls.DIVFREE, DEGREE, [gmls.CURLCURL], precision=gmls.FP32_REFINE)
    sp = ctx.stencils(npr, gmls.SCALAR, DEGREE, [gmls.GRAD, gmls.LAPLACIAN], precision=gmls.FP32_REFINE,
                      neumann=True)
    b = ctx.stokes_rhs(sv, sp, 1.0, d["f"], d["w"], d["div_f"])

    def solve(ss, row_scaling=False):
        rp, col, val = ctx.stokes_assemble(sv, sp, 1.0, ss)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sol, its, rel = ctx.gmres(rp, col, val, b, restart=100, max_iter=20000, rtol=1e-10, row_scaling=row_scaling)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        s = sol.cpu().numpy()
        us, ps = s[:2 * n].reshape(n, 2).T, s[2 * n:3 * n]
        eu = float(np.sqrt(np.mean((us - d["u"]) ** 2)))
        ep = float(np.sqrt(np.mean(((ps - ps.mean()) - (d["p"] - d["p"].mean())) ** 2)))
        return {"unknowns": int(rp.shape[0] - 1), "nnz": int(col.shape[0]), "iterations": its, "rel_residual": rel,
                "seconds": el, "rms_error_velocity": eu, "rms_error_pressure": ep}

    if not full:
        out = {"grid": f"{n_axis}x{n_axis}", "solver": "GMRES(100), row equilibration + right Jacobi",
               "interior_pressure_laplacian": "scalar GMLS, degree 4"}
        out.update(solve(0, True))
        for hd in (sp, sv, npr, nv, cid):
            ctx.release(hd)
        return out
    out = {"grid": f"{n_axis}x{n_axis}", "solver": "GMRES(100), right Jacobi",
           "interior_pressure_laplacian": "scalar GMLS, degree 4"}
    out.update(solve(0))
    out["row_scaled"] = solve(0, True)
    # the paper's choice for points inside the domain: the staggered
    # Laplacian (Sec. 2.4) of degree 3, on the scalar neighbour lists
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record(ctx.stream)
    ss = ctx.stencils(npr, gmls.STAGGERED, DEGREE - 1, [gmls.LAPLACIAN], precision=gmls.FP32_REFINE)
    e[1].record(ctx.stream)
    torch.cuda.synchronize()
    st = {"interior_pressure_laplacian": f"staggered GMLS, degree {DEGREE - 1}",
          "staggered_stencils_ms": e[0].elapsed_time(e[1])}
    st.update(solve(ss))
    out["staggered_interior"] = st
    for hd in (ss, sp, sv, npr, nv, cid):
        ctx.release(hd)
    return out


def serving(n_requests, seed=0):
    """Poisson arrivals (200 req/s) of stencil requests -- 2D/3D clouds of
    log-uniform 1e3..5e5 points, degree 2..4, scalar (gradient + Laplacian) or
    divergence-free (vector Laplacian) basis -- through the continuous-batching
    server (FP32 + refinement), and the same stream through the plain
    per-request FP64 path (one request at a time, in arrival order)."""
    import threading

    import torch

    from paper_2104_14447_gb300 import gmls, inputs

    reqs = inputs.request_stream(n_requests, 200.0, seed)
    clouds = []
    for r in reqs:
        n_axis = max(3, int(round(r["n"] ** (1.0 / r["dim"]))))
        clouds.append(inputs.jittered_grid(r["dim"], n_axis, seed=r["seed"]))
    spec = []
    for r in reqs:
        b = gmls.SCALAR if r["basis"] == "scalar" else gmls.DIVFREE
        fns = [gmls.GRAD, gmls.LAPLACIAN] if b == gmls.SCALAR else [gmls.VEC_LAPLACIAN]
        spec.append((b, r["degree"], SERVE_K[(r["dim"], b, r["degree"])], fns))
    total_targets = sum(c.shape[1] for c in clouds)
    offered = total_targets / max(reqs[-1]["t"], 1e-9)

    def run_server():
        srv = gmls.Server(torch.cuda.current_device(), arena_bytes=48 << 30, streams=4, max_inflight=8)
        tickets = [None] * len(reqs)
        t0 = time.perf_counter()

        def client():
            for i, r in enumerate(reqs):
                dt = r["t"] - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                b, m, k, fns = spec[i]
                tickets[i] = srv.submit(clouds[i], b, m, k, fns, precision=gmls.FP32_REFINE)

        th = threading.Thread(target=client)
        th.start()
        pending = set(range(len(reqs)))
        while pending:
            for i in list(pending):
                if tickets[i] is not None and srv.wait(tickets[i], 0):
                    srv.release(tickets[i])
                    pending.discard(i)
            time.sleep(0.0005)
        th.join()
        st = srv.stats()
        srv.close()
        return st

    def run_plain_fp64():
        ctx = gmls.Context(torch.cuda.current_device(), arena_bytes=48 << 30)
        ctx.set_option(gmls.OPT_AUTOTUNE, 0)
        lat, t0 = [], time.perf_counter()
        for i, r in enumerate(reqs):
            dt = r["t"] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            b, m, k, fns = spec[i]
            cid = ctx.cloud(clouds[i])
            nid = ctx.neighbors(cid, k, 1.5)
            sid = ctx.stencils(nid, b, m, fns, precision=gmls.FP64)
            ctx.sync()
            lat.append((time.perf_counter() - t0 - r["t"]) * 1e3)
            for h in (sid, nid, cid):
                ctx.release(h)
        el = time.perf_counter() - t0
        ctx.close()
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "targets_per_s": total_targets / el, "elapsed_s": el}

    srv = run_server()
    plain = run_plain_fp64()
    return {"requests": n_requests, "rate_per_s": 200.0, "targets": int(total_targets),
            "offered_targets_per_s": offered,
            "continuous_batching_fp32_refine": {"p50_ms": srv["p50_ms"], "p99_ms": srv["p99_ms"],
                                                "targets_per_s": srv["targets_per_s"], "elapsed_s": srv["elapsed_s"]},
            "plain_per_request_fp64": plain,
            "note": "bounded sample of the serving stream (first requests of the seeded Poisson sequence)"}


def oracle_pipeline(x, targets, threads=None):
    """The oracle as it stands on the same workload (a sample of targets)."""
    import oracle

    n = x.shape[1]
    i36, e36 = oracle.knn(x, targets, K_SCALAR, EPS_FACTOR, method="grid")
    i48, e48 = oracle.knn(x, targets, K_DIVFREE, EPS_FACTOR, method="grid")
    nt = len(targets)
    off36 = np.arange(0, nt * K_SCALAR + 1, K_SCALAR)
    off48 = np.arange(0, nt * K_DIVFREE + 1, K_DIVFREE)
    wg, _, _ = oracle.stencils(x, targets, off36, i36.reshape(-1), e36, "scalar", DEGREE, "grad")
    wd, _, _ = oracle.stencils(x, targets, off36, i36.reshape(-1), e36, "scalar", DEGREE, "div")
    wv, _, _ = oracle.stencils(x, targets, off48, i48.reshape(-1), e48, "divfree", DEGREE, "vec_laplacian")
    oracle.csr(off36, i36.reshape(-1), wg, n)
    oracle.csr(off36, i36.reshape(-1), wd, n)
    oracle.csr(off48, i48.reshape(-1), wv, n)
    return {"grad": wg, "div": wd, "vl": wv, "idx36": i36, "idx48": i48}


def cpu_baseline(ctx=None, sample_stride=1):
    """Time the oracle on the host cores; with a GPU context also report the
    GPU path's error against it on a sample of targets."""
    import oracle

    oracle.build()
    x = workload_points()
    n = x.shape[1]
    targets = np.arange(0, n, sample_stride, dtype=np.int32)
    t0 = time.perf_counter()
    res = oracle_pipeline(x, targets)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"value": len(targets) / dt, "unit": "targets/s", "cores": cores, "kind": "oracle",
           "sample": f"{len(targets)} of {n} targets (every {sample_stride}th), full pipeline incl. kNN and CSR",
           "seconds": dt}
    if ctx is not None:
        out["max_rel_err_vs_oracle"] = gpu_error(ctx, x, res, targets)
    return out


def gpu_error(ctx, x, res, targets):
    """max over sampled (target, row) of |w_gpu - w_oracle|_inf / |w_oracle|_inf."""
    import torch

    from paper_2104_14447_gb300 import gmls

    n = x.shape[1]
    samp = np.arange(len(targets))  # every target the oracle computed
    errs = {}
    cid = ctx.cloud(torch.from_numpy(x).to(ctx.device))
    for key, k, basis, fn in (("grad", K_SCALAR, gmls.SCALAR, gmls.GRAD), ("div", K_SCALAR, gmls.SCALAR, gmls.DIV),
                              ("vl", K_DIVFREE, gmls.DIVFREE, gmls.VEC_LAPLACIAN)):
        nid = ctx.neighbors(cid, k, EPS_FACTOR)
        sid = ctx.stencils(nid, basis, DEGREE, [fn], precision=gmls.FP32_REFINE)
        _, rows, nc, _ = ctx.stencil_info(sid, fn)
        wg = ctx.weights(sid, fn).cpu().numpy().reshape(n, rows, k, nc)[targets[samp]]
        wo = res[key][samp]
        a = np.abs(wg - wo).reshape(len(samp), rows, -1).max(axis=2)
        b = np.abs(wo).reshape(len(samp), rows, -1).max(axis=2)
        errs[key] = float(np.max(a / np.where(b > 0, b, 1.0)))
        ctx.release(sid)
        ctx.release(nid)
    ctx.release(cid)
    return errs


# --------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle, as it stands, on the host cores (this workload's CPU program)."""
    import oracle

    oracle.build()
    x = workload_points()
    n = x.shape[1]
    stride = args.ref_stride
    targets = np.arange(0, n, stride, dtype=np.int32)
    for _ in range(args.warmup):
        oracle_pipeline(x, targets)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_pipeline(x, targets)
        times.append(time.perf_counter() - t0)
    total = float(np.sum(times))
    value = len(targets) * args.steps / total
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = f"{len(targets)} of {n} targets per step (every {stride}th), full pipeline incl. kNN and CSR"
    return {"metric": METRIC, "value": value, "unit": "targets/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "targets_per_gpu": n, "precision": "fp64 (oracle)",
                       "degree": DEGREE, "neighbours": [K_SCALAR, K_DIVFREE], "eps_factor": EPS_FACTOR},
            "cpu_baseline": {"value": value, "unit": "targets/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "targets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32_refine", "fp64"], default="fp32_refine")
    ap.add_argument("--arena-gb", type=int, default=24)
    ap.add_argument("--ref-stride", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-stokes", action="store_true", help="skip the Stokes-system section")
    ap.add_argument("--no-porous", action="store_true", help="skip the 3D porous-medium section")
    ap.add_argument("--porous-n-axis", type=int, default=128, help="lattice of the porous section (profiling)")
    ap.add_argument("--no-batched", action="store_true", help="skip the uneven-batch section")
    ap.add_argument("--no-shapes", action="store_true", help="skip the per-shape FP32 / FP64 section")
    ap.add_argument("--e2e-ranges", type=int, default=E2E_CHUNKS, help="target ranges of the end-to-end pipeline")
    ap.add_argument("--e2e-fractions", default=None, help="relative sizes of the end-to-end ranges, e.g. 4,3,2,1")
    ap.add_argument("--e2e-copy-streams", type=int, default=2, help="copy streams of the end-to-end pipeline")
    ap.add_argument("--batched-n", type=int, default=500_000, help="targets per cloud of the uneven batch")
    ap.add_argument("--only", choices=["porous", "batched"], default=None,
                    help="profiling: run only this section (--steps timed steps) and print it")
    ap.add_argument("--n-axis", type=int, default=512, help="profiling only; the benchmark is 512")
    ap.add_argument("--serve-requests", type=int, default=60, help="serving sample size (0: skip)")
    ap.add_argument("--no-graph", dest="graph", action="store_false")
    args = ap.parse_args()
    set_n_axis(args.n_axis)
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if args.only:
        from paper_2104_14447_gb300 import build, gmls

        build.build()
        ctx = gmls.Context(local_rank, arena_bytes=args.arena_gb << 30)
        if args.only == "porous":
            res = porous_3d(ctx, n_axis=args.porous_n_axis, steps=args.steps, stokes=False)[0]
        else:
            res = batched_uneven(ctx, n_per_dim=args.batched_n, steps=args.steps)[0]
        print(json.dumps(res), flush=True)
        ctx.close()
        return
    if world > 1:
        import torch

        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    out, ctx = run_ours(args, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(ctx)
    if rank == 0 and world == 1 and not args.no_stokes:
        out["stokes_system"] = stokes_system(ctx)
        out["stokes_system"]["solve"] = stokes_solve(ctx)
        out["stokes_system"]["solve_256"] = stokes_solve(ctx, 256, full=False)
    if rank == 0 and world == 1 and not args.no_porous:
        out["porous_3d"], gs = porous_3d(ctx, n_axis=args.porous_n_axis)
        if not args.no_cpu_baseline:  # the oracle's side of the sampled comparison
            out["porous_3d"]["oracle_check"] = porous_oracle_errors(gs)
    if rank == 0 and world == 1 and not args.no_shapes:
        out["shapes"] = shapes(ctx)
    if rank == 0 and world == 1 and not args.no_batched:
        out["batched_uneven"], gsb = batched_uneven(ctx, n_per_dim=args.batched_n)
        if not args.no_cpu_baseline:  # the oracle's side of the sampled comparison
            out["batched_uneven"]["oracle_check"] = batched_oracle_errors(gsb)
    if rank == 0 and world == 1 and args.serve_requests > 0:
        out["serving"] = serving(args.serve_requests)
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
