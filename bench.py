"""GMLS stencil-generation benchmark (one JSON line on rank 0).

Headline workload (the 3D porous medium, the largest configuration that fits
one GPU): a jittered 128^3 lattice in the unit cube minus 64 random
non-overlapping spheres of radius 0.05-0.12 (1,763,183 points; 142,894 of
them on a sphere surface or cube face, with the geometric normal), sources =
targets.  One step is the whole hot path:

  cell-list build -> 80-nearest lists (eps = 1.5 d_k) and their 40-nearest
  prefix -> scalar Taylor degree-3 stencils (20 terms; gradient and
  Laplacian, with the Neumann constraint of Sec. 2.3 at boundary targets) ->
  divergence-free degree-3 stencils (50 terms, 240 x 50 systems; vector
  Laplacian) -> three CSR operators.

value: targets/s of the whole job (every target gets all three operators),
inputs resident on the device, L2 flushed between timed steps.  FP32
Householder QR with refinement against float-float (FP64-class) residuals.

Secondary sections: the 2D Stokes operators on a 512 x 512 grid (262,144
targets, scalar m = 4 and div-free m = 4, FP32 + refinement and FP64), the
1,024-target 2D FP64 case, the uneven batch (1,000,000 mixed targets, one
bucketed launch per cloud), the serving stream, every serving shape, the
Stokes block systems and solves, and the 3D polynomial and trigonometric
Stokes tests of Sec. 4.1 through the GPU operators (N = 6..96 per axis).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 it runs under torch.distributed.run, one rank per GPU; every rank
processes its own copy of the workload (independent problems: weak scaling,
no data-path collective; only the timing is reduced).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import mmap
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GMLS targets/sec"
# headline: 3D porous medium
P_N_AXIS = 128
P_K_SCALAR, P_K_DIVFREE, P_DEGREE = 40, 80, 3
WORKLOAD = ("porous3d-128: 128^3 jittered lattice minus 64 spheres; scalar m=3 (40 nbrs; grad, Laplacian, "
            "Neumann at boundary targets) + div-free m=3 (80 nbrs, 240x50; vector Laplacian) + CSR")
# secondary: 2D Stokes operators on the 512 x 512 grid
N_AXIS = 512
K_SCALAR, K_DIVFREE, EPS_FACTOR, DEGREE = 36, 48, 1.5, 4
E2E_CHUNKS = 4  # default target ranges of the end-to-end pipelines (copies overlap compute)
WORKLOAD_2D = "stokes2d-512x512: scalar m=4 (36 nbrs; grad, div) + div-free m=4 (48 nbrs; vector Laplacian) + CSR"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


def alu_peaks(dev):
    """FP32 / FP64 pipe peaks of the device (TFLOP/s) from its SM count and the
    maximum SM clock: 128 FP32 FMA lanes and 2 FP64 FMA units per SM, 2 flop
    per FMA.  MEASURED_PEAKS.json holds HBM and bf16 figures only, so these
    are unit counts (the clock from that file, else 2070 MHz)."""
    import torch

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks, src = _peaks()
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    p32 = sms * 128 * 2 * mhz * 1e6 / 1e12
    p64 = sms * 2 * 2 * mhz * 1e6 / 1e12
    return p32, p64, f"unit counts: {sms} SMs x 128 FP32 lanes (FP64: x 2 units) x 2 flop x {mhz:.0f} MHz ({src} clock)"


def alg_flops(M, n, L, iters):
    """Algorithmic flops of one target (the scope table's count): Householder
    QR of the M x n tile 2Mn^2 - 2n^3/3; per functional row the apply
    n^2 + 4Mn; per refinement iteration and row the residual 4Mn.  The
    float-float emulation, the basis evaluation and the padding are not
    counted."""
    return 2 * M * n * n - 2 * n ** 3 / 3 + L * (n * n + 4 * M * n) + iters * L * 4 * M * n


def src_sha(*names):
    """Short hash of kernel sources, to tie a stored ncu figure to the code it measured."""
    h = hashlib.sha256()
    for nm in names:
        with open(os.path.join(ROOT, "paper_2104_14447_gb300", "csrc", nm), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# DRAM bytes (read + write) per launch measured by ncu on the timed launch
# (dram__bytes_read.sum + dram__bytes_write.sum, one pass), with the hash of
# the kernel sources it was taken on; a different hash reports null
DFX_TRAFFIC = {"bytes": 700560384 + 10561089536, "sha": "f5e8cff84e6f2b6f",
               "sources": ("stencil_dfx.cuh", "stencil_fast.cuh", "ff.cuh"),
               "command": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none --nvtx "
                          "--nvtx-include porous_step/ -k regex:stencil_dfx -c 1 python bench.py --no-secondary "
                          "--no-e2e --no-cpu-baseline --steps 1 --warmup 3"}


class HostBuffers:
    """Page-locked host buffers for the end-to-end results.  With
    ``huge=True``: anonymous memory advised as transparent huge pages,
    touched, then registered with CUDA (cudaHostRegister); else the usual
    page-locked allocation (pin_memory).  On a host whose memory has been in
    use a while the usual allocation ends up in scattered base pages, and
    device-to-host copies into it then run at a fraction of the link's rate."""

    def __init__(self, huge):
        self.huge = huge
        self.regs = []

    def empty(self, shape, dtype):
        import torch

        if self.huge:
            nbytes = int(np.prod(shape)) * torch.empty((), dtype=dtype).element_size()
            try:
                mm = mmap.mmap(-1, max(nbytes, 1))
                mm.madvise(mmap.MADV_HUGEPAGE)
                t = torch.frombuffer(mm, dtype=torch.uint8, count=max(nbytes, 1))[:nbytes]
                t.fill_(0)  # touch: the pages exist before they are locked
                rc = torch.cuda.cudart().cudaHostRegister(t.data_ptr(), max(nbytes, 1), 0)
                if int(rc) == 0:
                    self.regs.append(t.data_ptr())
                    return t.view(dtype).view(shape)
            except (OSError, ValueError, RuntimeError, AttributeError):
                pass
        return torch.empty(shape, dtype=dtype, pin_memory=True)

    def close(self):
        """Unlock the registered buffers (call with no copy in flight, before
        the tensors go)."""
        import torch

        for p in self.regs:
            torch.cuda.cudart().cudaHostUnregister(p)
        self.regs = []


class Clocks:
    """nvidia-smi samples during the timed region."""

    _count = 0

    def __init__(self, index):
        self.index = index
        self.proc = None
        Clocks._count += 1  # one file per sampler: several may be read in one process
        self.path = os.path.join(tempfile.gettempdir(), f"gmls_clocks_{os.getpid()}_{Clocks._count}.csv")

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


# ------------------------------------------------------ headline: porous 3D
def porous_step_fn(ctx, prec, bufs):
    """One step of the porous-medium hot path on the context (cloud given as
    (x, normals, bflags) tensors, device or pinned host); returns the handles."""
    from paper_2104_14447_gb300 import gmls

    stream = ctx.stream

    def step(src, ev=None):
        rec = (lambda i: ev[i].record(stream)) if ev else (lambda i: None)
        rec(0)
        cid = ctx.cloud(src[0], normals=src[1], bflags=src[2])
        rec(1)
        n80 = ctx.neighbors(cid, P_K_DIVFREE, EPS_FACTOR)
        n40 = ctx.neighbors_prefix(n80, P_K_SCALAR, EPS_FACTOR)  # the 40 nearest = first 40 of the 80
        rec(2)
        ssc = ctx.stencils(n40, gmls.SCALAR, P_DEGREE, [gmls.GRAD, gmls.LAPLACIAN], precision=prec, neumann=True)
        rec(3)
        sdf = ctx.stencils(n80, gmls.DIVFREE, P_DEGREE, [gmls.VEC_LAPLACIAN], precision=prec)
        rec(4)
        ctx.assemble_csr(ssc, gmls.GRAD, out=bufs["grad"])
        ctx.assemble_csr(ssc, gmls.LAPLACIAN, out=bufs["lap"])
        ctx.assemble_csr(sdf, gmls.VEC_LAPLACIAN, out=bufs["vl"])
        rec(5)
        return cid, n80, n40, ssc, sdf

    return step


def run_headline(args, rank, world, local_rank):
    """The 3D porous-medium step: device-timed throughput (inputs resident),
    stage times, the roofline of the dominant kernel (the divergence-free
    stencil launch), the same step end to end through the C ABI from pinned
    host input to host CSR operators, and the GPU outputs of a seeded 5 %
    target sample for the oracle comparison."""
    import torch

    from paper_2104_14447_gb300 import build, gmls, inputs, shard

    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prec = gmls.FP32_REFINE
    pc = inputs.porous_cube(n_axis=args.porous_n_axis)
    n = pc["x"].shape[1]
    host = (torch.from_numpy(pc["x"]), torch.from_numpy(np.ascontiguousarray(pc["normals"])),
            torch.from_numpy(pc["bflag"]))
    dsrc = tuple(t.to(dev) for t in host)
    ctx = gmls.Context(local_rank, arena_bytes=args.arena_gb << 30)
    stream = ctx.stream
    # operators: gradient (3 rows x 40), Laplacian (1 x 40), vector Laplacian (3 x 80 x 3 components)
    per_target = {"grad": (3, P_K_SCALAR), "lap": (1, P_K_SCALAR), "vl": (3, 3 * P_K_DIVFREE)}
    bufs = {}
    for name, (rows, per_row) in per_target.items():
        nnz = n * rows * per_row
        bufs[name] = (torch.empty(n * rows + 1, dtype=torch.int64, device=dev),
                      torch.empty(nnz, dtype=torch.int32, device=dev),
                      torch.empty(nnz, dtype=torch.float64, device=dev))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    step = porous_step_fn(ctx, prec, bufs)

    def release(ids):
        for h in reversed(ids):
            ctx.release(h)

    for _ in range(args.warmup):
        release(step(dsrc))
    torch.cuda.synchronize()
    # refinement statistics of this workload (one untimed step)
    ids = step(dsrc)
    it_sc = ctx.export(ids[3], gmls.X_ITERS, torch.uint8).float()
    it_df = ctx.export(ids[4], gmls.X_ITERS, torch.uint8).float()
    st_sc = ctx.export(ids[3], gmls.X_STATUS, torch.uint8)
    st_df = ctx.export(ids[4], gmls.X_STATUS, torch.uint8)
    redo = {"scalar": int(((st_sc & gmls.T_FP64_FALLBACK) != 0).sum()),
            "divfree": int(((st_df & gmls.T_FP64_FALLBACK) != 0).sum())}
    mean_it_sc, mean_it_df = float(it_sc.mean()), float(it_df.mean())
    iters_hist = {str(i): int((it_df == i).sum()) for i in range(5) if int((it_df == i).sum())}
    release(ids)
    torch.cuda.synchronize()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    launches0 = ctx.launch_count()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local_rank) as clk:
        for s in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(s & 0xFF)  # evict L2 between timed steps (outside the events)
            torch.cuda.nvtx.range_push("porous_step")  # lets a profiler select the timed launches
            ids = step(dsrc, evs[s])
            torch.cuda.nvtx.range_pop()
            release(ids)
        torch.cuda.synchronize()
    launches = ctx.launch_count() - launches0
    stage = np.array([[e[i].elapsed_time(e[i + 1]) for i in range(5)] for e in evs])
    step_ms = [float(e[0].elapsed_time(e[5])) for e in evs]
    total_ms = shard.max_over_ranks(float(np.sum(step_ms)), dev)

    # roofline of the dominant kernel: the divergence-free stencil launch
    # (240 x 50 systems, 3 functional rows), CUDA events on the context stream
    k_avg = float(np.mean(stage[:, 3])) * 1e-3
    p32, p64, peak_src = alu_peaks(dev)
    f_t = alg_flops(3 * P_K_DIVFREE, 50, 3, mean_it_df)
    achieved = n * f_t / k_avg / 1e12
    sha = src_sha(*DFX_TRAFFIC["sources"])
    traffic = DFX_TRAFFIC["bytes"] if DFX_TRAFFIC["sha"] == sha else None
    out_bytes = n * 3 * P_K_DIVFREE * 3 * 8  # FP64 weights written
    roofline = {"bound": "alu", "achieved": achieved, "peak": p32, "unit": "TFLOP/s", "frac": achieved / p32,
                "traffic": traffic,
                "traffic_note": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the timed launch "
                                 f"({DFX_TRAFFIC['command']})") if traffic else
                                "null: no ncu figure for the current kernel sources",
                "algorithmic_output_bytes": out_bytes,
                "kernel": "stencil_dfx_kernel<3, 3> (factored div-free QR, FP32 + float-float refinement; "
                          "240 x 50 systems)",
                "pipe": "fp32", "flops_per_target": f_t, "mean_refine_iters": mean_it_df,
                "flop_count": "2Mn^2 - 2n^3/3 + L (n^2 + 4Mn) + iters L 4Mn, M = 240, n = 50, L = 3",
                "peak_source": peak_src, "kernel_ms": k_avg * 1e3}

    # end to end through the C ABI: pinned host coordinates, normals and
    # flags in; the three CSR operators back in pinned host memory.  The
    # targets go through in ranges so that the operators of the first ranges
    # travel to the host (on copy streams) while the GPU computes the rest:
    # per range the 80-nearest lists, the divergence-free stencils and their
    # operator rows, written in place by gmls_assemble_csr_at; then per range
    # the 40-nearest prefix lists, the scalar stencils and their two operators.
    e2e = None
    if not args.no_e2e:
        pin = tuple(t.pin_memory() for t in host)
        hb = HostBuffers(args.e2e_host == "huge")
        host_out = {k: tuple(hb.empty(v.shape, v.dtype) for v in bufs[k]) for k in bufs}
        n_ranges = args.e2e_ranges
        bounds = [n * c // n_ranges for c in range(n_ranges + 1)]
        d2h = sum(t.numel() * t.element_size() for v in bufs.values() for t in v) + 8 * 3 * (n_ranges - 1)
        h2d = sum(t.numel() * t.element_size() for t in pin)
        copy_streams = [torch.cuda.Stream(dev) for _ in range(args.e2e_copy_streams)]
        chunk_tg = [torch.arange(a, b, dtype=torch.int32, device=dev) for a, b in zip(bounds[:-1], bounds[1:])]

        def ship(sid, fn, kname, c, which):
            rows, per_row = per_target[kname]
            a, b = bounds[c], bounds[c + 1]
            lo, hi = a * rows * per_row, b * rows * per_row
            sl = (slice(a * rows, b * rows + 1), slice(lo, hi), slice(lo, hi))
            dev_out = tuple(t[q] for t, q in zip(bufs[kname], sl))
            ctx.assemble_csr(sid, fn, out=dev_out, nnz_offset=lo)
            done = torch.cuda.Event()
            done.record(stream)
            cs = copy_streams[which % len(copy_streams)]
            cs.wait_event(done)
            with torch.cuda.stream(cs):
                for dst, src, q in zip(host_out[kname], dev_out, sl):
                    dst[q].copy_(src, non_blocking=True)

        def step_e2e():
            cid = ctx.cloud(pin[0], normals=pin[1], bflags=pin[2])
            ids, n80s = [cid], []
            for c in range(n_ranges):
                n80 = ctx.neighbors(cid, P_K_DIVFREE, EPS_FACTOR, targets=chunk_tg[c])
                sdf = ctx.stencils(n80, gmls.DIVFREE, P_DEGREE, [gmls.VEC_LAPLACIAN], precision=prec)
                ship(sdf, gmls.VEC_LAPLACIAN, "vl", c, c)
                n80s.append(n80)
                ids += [n80, sdf]
            for c in range(n_ranges):
                n40 = ctx.neighbors_prefix(n80s[c], P_K_SCALAR, EPS_FACTOR)
                ssc = ctx.stencils(n40, gmls.SCALAR, P_DEGREE, [gmls.GRAD, gmls.LAPLACIAN], precision=prec,
                                   neumann=True)
                ship(ssc, gmls.GRAD, "grad", c, 2 * c)
                ship(ssc, gmls.LAPLACIAN, "lap", c, 2 * c + 1)
                ids += [n40, ssc]
            return ids

        e2e_ms = []
        with Clocks(local_rank) as e2e_clk:
            for s in range(max(3, min(args.steps, 9)) + 1):
                with torch.cuda.stream(stream):
                    flush.fill_(s & 0xFF)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ids = step_e2e()
                torch.cuda.synchronize()  # every range's copies done: the operators are on the host
                e2e_ms.append((time.perf_counter() - t0) * 1e3)
                release(ids)
        e2e_ms = e2e_ms[1:]
        # the host operators equal the device step's, bit for bit (checked once, untimed, on the device)
        ids = step(dsrc)
        torch.cuda.synchronize()
        equal = all(torch.equal(h.to(dev, non_blocking=True), d) for k in bufs for h, d in zip(host_out[k], bufs[k]))
        release(ids)
        e2e = {"value": n * world / (float(np.median(e2e_ms)) * 1e-3), "unit": "targets/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": float(np.median(e2e_ms)), "ms_steps": [round(v, 3) for v in e2e_ms],
               "target_ranges": n_ranges, "copy_streams": len(copy_streams),
               "host_operators_equal_device_step": equal, "host_buffers": args.e2e_host,
               "clocks": e2e_clk.summary()}
        torch.cuda.synchronize()
        hb.close()
        del host_out, pin

    # GPU outputs of a seeded 5 % target sample for the oracle comparison
    ids = step(dsrc)
    m = max(1, int(round(0.05 * n)))
    sample = np.unique((inputs.uniform(7, 131, m) * n).astype(np.int64)).astype(np.int32)
    sdev = torch.from_numpy(sample.astype(np.int64)).to(dev)
    gs = {"pc": pc, "sample": sample, "ops": []}
    for key, nh, sh, k, kind, code in (("grad", ids[2], ids[3], P_K_SCALAR, "scalar", gmls.GRAD),
                                       ("laplacian", ids[2], ids[3], P_K_SCALAR, "scalar", gmls.LAPLACIAN),
                                       ("vec_laplacian", ids[1], ids[4], P_K_DIVFREE, "divfree", gmls.VEC_LAPLACIAN)):
        idx = ctx.export(nh, gmls.X_NBR_INDEX, torch.int32).view(n, k)[sdev].cpu().numpy()
        _, rows, nc, _ = ctx.stencil_info(sh, code)
        wg = ctx.weights(sh, code).view(n, rows, k, nc)[sdev].cpu().numpy()
        gs["ops"].append((key, k, kind, idx, wg))
    release(ids)

    tune = tune_names(ctx, lambda r: r["dim"] == 3 and not r["bucketed"])
    value = shard.job_throughput(n, args.steps, world, total_ms)
    med = np.median(stage, axis=0)
    out = {
        "metric": METRIC, "value": value, "unit": "targets/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+ff", "data": "synthetic",
        "config": {"workload": WORKLOAD, "targets_per_gpu": n, "points": n,
                   "boundary_targets": int(pc["bflag"].sum()), "porosity": float(pc["porosity"]),
                   "precision": "fp32 QR + float-float refinement (FP64 redo of flagged targets)",
                   "degree": P_DEGREE, "neighbours": [P_K_SCALAR, P_K_DIVFREE], "eps_factor": EPS_FACTOR,
                   "weight": "(1-r/eps)_+^4", "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"independent replicas x{world}" if world > 1 else "1 GPU"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "stage_ms": {"cell_list": float(med[0]), "neighbours": float(med[1]), "scalar_stencils": float(med[2]),
                     "divfree_stencils": float(med[3]), "csr": float(med[4])},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "refinement": {"mean_iters_scalar": mean_it_sc, "mean_iters_divfree": mean_it_df,
                       "divfree_iters_histogram": iters_hist, "fp64_redo_targets": redo},
        "roofline": roofline,
        "clocks": clk.summary(),
        "autotune_ms": tune,
    }
    return out, ctx, gs


def tune_names(ctx, keep):
    """The autotuner's timings (ms) by shape and kernel variant."""
    tune = {}
    for r in ctx.tune_log():
        if not keep(r):
            continue
        key = (f"{r['dim']}d {['scalar', 'divfree', 'staggered'][r['basis']]} m={r['degree']} rows<={r['rows']}"
               f"{' fp64' if r['precision'] == 0 else ''}{' bucketed' if r['bucketed'] else ''}")
        tune.setdefault(key, {})[variant_name(r["variant"])] = round(r["ms"], 3)
    return tune


def variant_name(v):
    if v is None:
        return None
    if v < 0:
        return {-1: "register", -2: "register 16 lanes", -3: "factored div-free", -4: "register 8 lanes"}.get(v, str(v))
    place = {0: "", 1: ", split tiles", 2: ", global tiles"}.get(v >> 3, "")
    return f"{v & 7} warp(s)/target{place}"


def porous_cpu_baseline(gs, threads_all=None):
    """The oracle as it stands on the host cores over the seeded 5 % target
    sample of the porous workload (kNN lists, both prefix-free scalar and
    div-free stencils, CSR), all cores; a 0.5 % sample on one core; and the
    GPU outputs of the same 5 % sample against the oracle's (every target,
    every functional row: max relative error and the error over the bar
    max(1e-9, 1e-15 kappa))."""
    import oracle

    oracle.build()
    pc, sample = gs["pc"], gs["sample"]
    x = pc["x"]
    n = x.shape[1]
    cores = os.cpu_count() or 1

    def run(tg):
        ns = len(tg)
        i80, e80 = oracle.knn(x, tg, P_K_DIVFREE, EPS_FACTOR, method="grid")
        i40, e40 = oracle.knn(x, tg, P_K_SCALAR, EPS_FACTOR, method="grid")
        off40, off80 = np.arange(0, ns * P_K_SCALAR + 1, P_K_SCALAR), np.arange(0, ns * P_K_DIVFREE + 1, P_K_DIVFREE)
        extra = dict(bflag=pc["bflag"][tg], normals=pc["normals"].T[tg])
        res = {}
        for key, kind, i, o, e, ex in (("grad", "scalar", i40, off40, e40, extra),
                                        ("laplacian", "scalar", i40, off40, e40, extra),
                                        ("vec_laplacian", "divfree", i80, off80, e80, {})):
            w, _, diag = oracle.stencils(x, tg, o, i.reshape(-1), e, kind, P_DEGREE, key, **ex)
            oracle.csr(o, i.reshape(-1), w, n)
            res[key] = (i, w, diag)
        return res

    oracle.set_threads(cores)
    t0 = time.perf_counter()
    res = run(sample)
    dt = time.perf_counter() - t0
    one = sample[::10]
    oracle.set_threads(1)
    t1 = time.perf_counter()
    run(one)
    dt1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    errs, scaled, lists_equal = {}, {}, True
    for key, k, kind, idx, wg in gs["ops"]:
        oi, wo, diag = res[key]
        lists_equal &= bool(np.array_equal(idx, oi))
        w = wg.reshape(wo.shape)
        a = np.abs(w - wo).reshape(len(sample), wo.shape[1], -1).max(axis=2)
        b = np.abs(wo).reshape(len(sample), wo.shape[1], -1).max(axis=2)
        rel = a / np.where(b > 0, b, 1.0)
        kap = diag[:, 0] / np.maximum(diag[:, 1], 1e-300)
        errs[key] = float(rel.max())
        scaled[key] = float((rel / np.maximum(1e-9, 1e-15 * kap)[:, None]).max())
    return {"value": len(sample) / dt, "unit": "targets/s", "cores": cores, "kind": "oracle",
            "sample": (f"seeded 5 % of the targets ({len(sample)} of {n}), full pipeline incl. kNN and CSR; "
                       "the rate extrapolates linearly to the whole workload"),
            "seconds": dt, "cpu_model": cpu_model(),
            "single_core": {"value": len(one) / dt1, "unit": "targets/s", "sample": f"{len(one)} targets (every "
                            "10th of the 5 % sample)", "seconds": dt1},
            "gpu_vs_oracle": {"targets_compared": int(len(sample)), "neighbour_lists_equal": lists_equal,
                              "max_rel_err": errs, "max_err_over_bar": scaled,
                              "bar": "max(1e-9, 1e-15 kappa) per (target, row), kappa from the oracle's FP64 factor"}}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return None


# --------------------------------------------- secondary: 2D Stokes operators
def stokes2d_section(ctx, args, prec_name="fp32_refine"):
    """The 2D Stokes operators on the 512 x 512 grid (262,144 targets): cell
    list, 48-nearest lists and their 36-nearest prefix, scalar degree-4
    stencils (gradient, divergence), divergence-free degree-4 stencils (96 x
    20 systems, vector Laplacian), three CSR operators.  Device-timed
    throughput, the roofline of the divergence-free stencil launch, the same
    step end to end (pinned host input to host operators) and captured as a
    CUDA graph (FP32 path), and the GPU error against the oracle on a sample."""
    import torch

    from paper_2104_14447_gb300 import gmls

    dev = ctx.device
    prec = gmls.FP64 if prec_name == "fp64" else gmls.FP32_REFINE
    x_host = workload_points()
    n = x_host.shape[1]
    x_dev = torch.from_numpy(x_host).to(dev)
    stream = ctx.stream
    nnz_grad, nnz_div, nnz_vl = n * K_SCALAR * 2, n * K_SCALAR * 2, n * K_DIVFREE * 2 * 2
    bufs = {}
    for name, rows, nnz in (("grad", 2 * n, nnz_grad), ("div", n, nnz_div), ("vl", 2 * n, nnz_vl)):
        bufs[name] = (torch.empty(rows + 1, dtype=torch.int64, device=dev),
                      torch.empty(nnz, dtype=torch.int32, device=dev),
                      torch.empty(nnz, dtype=torch.float64, device=dev))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

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
    for s in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(s & 0xFF)
        ev[s][0].record(stream)
        torch.cuda.nvtx.range_push("stokes2d_step")  # lets a profiler select the timed launches
        ids = step(x_dev, kev[s])
        torch.cuda.nvtx.range_pop()
        ev[s][1].record(stream)
        release(ids)
    torch.cuda.synchronize()
    launches = ctx.launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    kern_ms = [a.elapsed_time(b) for a, b in kev]
    total_ms = float(np.sum(step_ms))
    k_avg = float(np.mean(kern_ms)) * 1e-3
    p32, p64, peak_src = alu_peaks(dev)
    if prec == gmls.FP32_REFINE:
        f_t, peak, pipe = alg_flops(2 * K_DIVFREE, 20, 2, mean_it_df), p32, "fp32"
    else:
        f_t, peak, pipe = alg_flops(2 * K_DIVFREE, 20, 2, 0), p64, "fp64"
    achieved = n * f_t / k_avg / 1e12
    tl = [r for r in ctx.tune_log() if r["dim"] == 2 and r["basis"] == gmls.DIVFREE and r["degree"] == DEGREE
          and r["precision"] == prec and not r["bucketed"]]
    chosen = variant_name(min(tl, key=lambda r: r["ms"])["variant"]) if tl else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": f"divergence-free stencil launch, 96 x 20 systems ({chosen or 'heuristic'})",
                "pipe": pipe, "flops_per_target": f_t, "mean_refine_iters": mean_it_df if prec != gmls.FP64 else 0,
                "flop_count": "2Mn^2 - 2n^3/3 + L (n^2 + 4Mn) + iters L 4Mn, M = 96, n = 20, L = 2",
                "peak_source": peak_src, "kernel_ms": k_avg * 1e3}
    out = {"workload": WORKLOAD_2D, "targets": n, "precision": prec_name, "value": n * args.steps / total_ms * 1e3,
           "unit": "targets/s", "ms_per_step": total_ms / args.steps, "gpu_launches": int(launches),
           "refinement": {"mean_iters_scalar": mean_it_sc, "mean_iters_divfree": mean_it_df,
                          "fp64_fallback_targets": fb} if prec != gmls.FP64 else None,
           "roofline": roofline}
    if prec == gmls.FP64:
        return out

    # e2e: the same step through the C ABI from pinned host input to host operators
    x_pin = torch.from_numpy(x_host).pin_memory()
    hb = HostBuffers(args.e2e_host == "huge")
    host_out = {k: tuple(hb.empty(v.shape, v.dtype) for v in bufs[k]) for k in bufs}
    n_ranges = args.e2e_ranges
    d2h = sum(t.numel() * t.element_size() for v in bufs.values() for t in v) + 8 * 3 * (n_ranges - 1)
    h2d = x_pin.numel() * x_pin.element_size()
    copy_streams = [torch.cuda.Stream(dev) for _ in range(args.e2e_copy_streams)]
    bounds = [n * c // n_ranges for c in range(n_ranges + 1)]
    chunk_tg = [torch.arange(a, b, dtype=torch.int32, device=dev) for a, b in zip(bounds[:-1], bounds[1:])]
    per_target = {"vl": (2, K_DIVFREE * 2), "grad": (2, K_SCALAR), "div": (1, K_SCALAR * 2)}  # rows, nnz per row

    def assemble_and_ship(sid, fn, kname, c, which):
        rows, per_row = per_target[kname]
        a, b = bounds[c], bounds[c + 1]
        lo, hi = a * rows * per_row, b * rows * per_row
        sl = (slice(a * rows, b * rows + 1), slice(lo, hi), slice(lo, hi))
        dev_out = tuple(t[q] for t, q in zip(bufs[kname], sl))
        ctx.assemble_csr(sid, fn, out=dev_out, nnz_offset=lo)
        done = torch.cuda.Event()
        done.record(stream)
        cs = copy_streams[which % len(copy_streams)]
        cs.wait_event(done)
        with torch.cuda.stream(cs):
            for dst, src, q in zip(host_out[kname], dev_out, sl):
                dst[q].copy_(src, non_blocking=True)

    def step_e2e(x_src):
        cid = ctx.cloud(x_src)
        ids = [cid]
        n48s = []
        for c in range(n_ranges):
            n48 = ctx.neighbors(cid, K_DIVFREE, EPS_FACTOR, targets=chunk_tg[c])
            s_df = ctx.stencils(n48, gmls.DIVFREE, DEGREE, [gmls.VEC_LAPLACIAN], precision=prec)
            assemble_and_ship(s_df, gmls.VEC_LAPLACIAN, "vl", c, c)
            n48s.append(n48)
            ids += [n48, s_df]
        for c in range(n_ranges):
            n36 = ctx.neighbors_prefix(n48s[c], K_SCALAR, EPS_FACTOR)
            s_sc = ctx.stencils(n36, gmls.SCALAR, DEGREE, [gmls.GRAD, gmls.DIV], precision=prec)
            assemble_and_ship(s_sc, gmls.GRAD, "grad", c, 2 * c)
            assemble_and_ship(s_sc, gmls.DIV, "div", c, 2 * c + 1)
            ids += [n36, s_sc]
        return ids

    e2e_ms = []
    for s in range(max(3, min(args.steps, 7)) + 1):
        with torch.cuda.stream(stream):
            flush.fill_(s & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ids = step_e2e(x_pin)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        release(ids)
    e2e_ms = e2e_ms[1:]
    ids = step(x_dev)
    torch.cuda.synchronize()
    e2e_equal = all(torch.equal(h, d.cpu()) for k in bufs for h, d in zip(host_out[k], bufs[k]))
    release(ids)
    torch.cuda.synchronize()
    hb.close()
    del host_out
    out["e2e"] = {"value": n / (float(np.median(e2e_ms)) * 1e-3), "unit": "targets/s",
                  "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                  "ms_per_step": float(np.median(e2e_ms)), "ms_steps": [round(v, 3) for v in e2e_ms],
                  "target_ranges": n_ranges, "host_operators_equal_device_step": e2e_equal}

    # the same step captured once as a CUDA graph and replayed
    if args.graph:
        gstream = torch.cuda.Stream(dev)
        gctx = type(ctx)(ctx.device.index or 0, arena_bytes=args.arena_gb << 30, stream=gstream)
        with torch.cuda.stream(gstream):
            ids_g = None
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
        out["graph"] = {"ms_per_step": graph_ms, "targets_per_s": n / (graph_ms * 1e-3)}
    out["autotune_ms"] = tune_names(ctx, lambda r: r["dim"] == 2 and not r["bucketed"])
    return out


SERVE_K = {(2, 0, 2): 12, (2, 0, 3): 20, (2, 0, 4): 36, (2, 1, 2): 22, (2, 1, 3): 34, (2, 1, 4): 48,
           (3, 0, 2): 20, (3, 0, 3): 40, (3, 0, 4): 84, (3, 1, 2): 42, (3, 1, 3): 80, (3, 1, 4): 136}


def polynomial_tables_3d(ctx, sizes=(6, 12, 24, 48, 96), degrees=(2, 4), rtol=1e-12):
    """The 3D tests of Sec. 4.1 through the GPU operators: the Stokes problem
    on [-1, 1]^3 (jittered lattice of N points per axis, the box's outer
    layer Dirichlet, Neumann pressure rows there) with degree-m stencils (FP32
    + refinement) on the fixed-k lists and GMRES(100) with row equilibration
    to rtol.  Data: a quadratic (m = 2) or quartic (m = 4) divergence-free
    velocity and pressure, which the bases reproduce exactly (the paper's
    tables report L2 errors of 6.8e-12 to 2.1e-9 and 1.6e-12 to 9.2e-9 for
    N = 6 to 96); and the trigonometric field of the paper's convergence
    study, with the observed order between successive N.  Per case:
    unknowns, iterations, seconds, L2 (RMS) and max errors of the solved
    velocity and mean-free pressure."""
    import torch

    from paper_2104_14447_gb300 import gmls, inputs

    k_tab = {2: (42, 20), 4: (136, 84)}  # (div-free, scalar) neighbours

    def solve_case(m, na, data):
        kv, kp = k_tab[m]
        x = inputs.jittered_grid(3, na, seed=na) * 2.0 - 1.0
        n = x.shape[1]
        bflag, nrm = inputs.box_boundary(3, na)
        d = data(x)
        cid = ctx.cloud(x, normals=nrm, bflags=bflag)
        nv = ctx.neighbors(cid, kv, EPS_FACTOR)
        npr = ctx.neighbors_prefix(nv, kp, EPS_FACTOR)
        sv = ctx.stencils(nv, gmls.DIVFREE, m, [gmls.CURLCURL], precision=gmls.FP32_REFINE)
        sp = ctx.stencils(npr, gmls.SCALAR, m, [gmls.GRAD, gmls.LAPLACIAN], precision=gmls.FP32_REFINE, neumann=True)
        rp, col, val = ctx.stokes_assemble(sv, sp, 1.0, 0)
        b = ctx.stokes_rhs(sv, sp, 1.0, d["f"], d["w"], d["div_f"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sol, its, rel = ctx.gmres(rp, col, val, b, restart=100, max_iter=20000, rtol=rtol, row_scaling=True)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        s = sol.cpu().numpy()
        eu = s[:3 * n].reshape(n, 3).T - d["u"]
        ep = (s[3 * n:4 * n] - s[3 * n:4 * n].mean()) - (d["p"] - d["p"].mean())
        row = {"N": na, "points": n, "unknowns": int(rp.shape[0] - 1), "nnz": int(col.shape[0]), "iterations": its,
               "rel_residual": rel, "converged": bool(np.isfinite(rel) and rel <= rtol), "seconds": el,
               "l2_error_velocity": float(np.sqrt(np.mean(eu ** 2))),
               "l2_error_pressure": float(np.sqrt(np.mean(ep ** 2))),
               "max_error_velocity": float(np.abs(eu).max()), "max_error_pressure": float(np.abs(ep).max())}
        del rp, col, val, b, sol
        for hd in (sp, sv, npr, nv, cid):
            ctx.release(hd)
        return row

    out = {"domain": "[-1, 1]^3, jittered lattice, outer layer Dirichlet",
           "solver": f"GMRES(100), row equilibration + right Jacobi, rtol {rtol:g}", "nu": 1.0,
           "precision": "fp32 + float-float refinement", "tables": {}}
    for m in degrees:
        out["tables"]["quadratic" if m == 2 else "quartic"] = [
            solve_case(m, na, lambda x, m=m: inputs.stokes_polynomial_3d(x, m, 1.0)) for na in sizes]
    for m in degrees:
        rows = [solve_case(m, na, lambda x: inputs.stokes_trig_3d(x, 1.0)) for na in sizes if na >= 12]
        for prev, row in zip(rows[:-1], rows[1:]):  # h = 2 / (N - 1)
            hr = np.log((row["N"] - 1) / (prev["N"] - 1))
            row["order_velocity"] = float(np.log(prev["l2_error_velocity"] / row["l2_error_velocity"]) / hr)
            row["order_pressure"] = float(np.log(prev["l2_error_pressure"] / row["l2_error_pressure"]) / hr)
        out["tables"][f"trigonometric_degree{m}"] = rows
    return out


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
            name = variant_name(v)
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


def porous_stokes_section(ctx, pc):
    """Lists and Neumann-constrained scalar stencils of the headline step,
    then the 3D Stokes block system on them (porous_stokes)."""
    import torch

    from paper_2104_14447_gb300 import gmls

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=ctx.device)
    cid = ctx.cloud(pc["x"], normals=pc["normals"], bflags=pc["bflag"])
    n80 = ctx.neighbors(cid, P_K_DIVFREE, EPS_FACTOR)
    n40 = ctx.neighbors_prefix(n80, P_K_SCALAR, EPS_FACTOR)
    ssc = ctx.stencils(n40, gmls.SCALAR, P_DEGREE, [gmls.GRAD, gmls.LAPLACIAN], precision=gmls.FP32_REFINE,
                       neumann=True)
    res = porous_stokes(ctx, pc, n80, n40, ssc, flush)
    for h in (ssc, n40, n80, cid):
        ctx.release(h)
    return res


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
        for i, ((c, cid, hs, kpt, deg), h) in enumerate(zip(prepared, hs_out)):
            h.append(ctx.stencils(h[0], gmls.SCALAR, 0, [gmls.GRAD, gmls.LAPLACIAN], precision=prec,
                                  degree_per_target=deg))
            rec(2 + i)  # one bucketed launch per cloud
        for h in hs_out:
            h.append(ctx.assemble_csr(h[1], gmls.GRAD))
        rec(4)
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
        with Clocks(torch.cuda.current_device()) as clk:
            for s in range(nsteps):
                with torch.cuda.stream(stream):
                    flush.fill_(s & 0xFF)
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
                torch.cuda.nvtx.range_push("batched_step")
                h = step(prec, ev)
                torch.cuda.nvtx.range_pop()
                torch.cuda.synchronize()
                times.append([ev[i].elapsed_time(ev[i + 1]) for i in range(4)])
                if not (prec == gmls.FP32_REFINE and s == nsteps - 1):
                    release(h)
        med = np.median(np.array(times), axis=0)
        res[name] = {"step_ms": float(np.sum(med)), "targets_per_s": 2 * n_per_dim / float(np.sum(med)) * 1e3,
                     "stage_ms": {"neighbours": float(med[0]), "stencils": float(med[1] + med[2]),
                                  "stencils_2d": float(med[1]), "stencils_3d": float(med[2]), "csr": float(med[3])},
                     "stencils_3d_steps_ms": [round(t[2], 3) for t in times], "clocks": clk.summary()}
        if prec == gmls.FP32_REFINE:
            keep = h
            stencil_ms = (float(med[1]), float(med[2]))
    stats, gpu_sample = {}, []
    classes = np.array([32, 64, 96, 128, 160, 192, 256, 384, 512, 768, 1024])  # the bucketing's row classes
    flops_alg, flops_pad = [], []
    for (c, cid, hs, kpt, deg), h in zip(prepared, keep):
        d = c["dim"]
        off = ctx.export(h[0], gmls.X_NBR_OFFSETS, torch.int64).cpu().numpy()
        nst = ctx.export(h[0], gmls.X_NBR_STATUS, torch.uint8).cpu().numpy()
        st = ctx.export(h[1], gmls.X_STATUS, torch.uint8).cpu().numpy()
        its = ctx.export(h[1], gmls.X_ITERS, torch.uint8).cpu().numpy().astype(np.float64)
        cnt = np.diff(off)
        # scope-table flops per target on the unpadded rows (M = k, n = Q(d, m),
        # L = d + 1 solve rows: gradient and Laplacian) and on the row class
        # the target was bucketed into (the tile it ran in)
        ok = (nst & gmls.T_TOO_FEW_NEIGHBOURS) == 0
        qn = np.array([BASIS_SIZE[(d, int(m))] for m in c["degree"]], dtype=np.float64)
        M = cnt.astype(np.float64)
        Mp = classes[np.minimum(np.searchsorted(classes, cnt), len(classes) - 1)].astype(np.float64)
        flops_alg.append(float(np.sum(alg_flops(M, qn, d + 1, its)[ok])))
        flops_pad.append(float(np.sum(alg_flops(Mp, qn, d + 1, its)[ok])))
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
    import torch as _t

    p32, _, peak_src = alu_peaks(_t.device("cuda", _t.cuda.current_device()))
    roof = {}
    for i, d in enumerate((2, 3)):
        a = flops_alg[i] / (stencil_ms[i] * 1e-3) / 1e12
        roof[f"{d}d"] = {"achieved": a, "frac": a / p32, "kernel_ms": stencil_ms[i],
                         "padding_waste": flops_pad[i] / flops_alg[i] - 1.0}
    a_all = sum(flops_alg) / (sum(stencil_ms) * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": a_all, "peak": p32, "unit": "TFLOP/s", "frac": a_all / p32,
                "traffic": None, "kernel": "bucketed persistent stencil launches (one per cloud), FP32 + refinement",
                "flop_count": "sum over targets of 2Mn^2 - 2n^3/3 + L (n^2 + 4Mn) + iters L 4Mn with the unpadded "
                              "M = k, n = Q(d, m), L = d + 1",
                "padding_waste": sum(flops_pad) / sum(flops_alg) - 1.0,
                "padding_note": "flops on the row class each target was bucketed into over the unpadded flops, minus 1",
                "per_cloud": roof, "peak_source": peak_src}
    return {"workload": f"uneven batch: 2D and 3D jittered clouds of {n_per_dim} targets each, degree U{{2,3,4}}, "
                        "radius lists at 1.8 x the Q(d,m)-th neighbour distance (<= 160), 20 % one-sided, "
                        "scalar basis (gradient, Laplacian), one bucketed launch per cloud",
            "targets": 2 * n_per_dim, **res, "speedup_vs_fp64": res["fp64"]["step_ms"] / res["fp32_refine"]["step_ms"],
            "roofline": roofline,
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


def stokes_solve(ctx, n_axis=128, full=True, rtol=1e-10):
    """Global solve of the Stokes system (Sec. 3.3) on an n_axis^2 grid by
    GMRES(100) with right Jacobi preconditioning (gmls_gmres), to a relative
    residual of rtol (for the row-equilibrated legs: of R (b - A x); the
    unscaled residual is reported beside it, and "converged" says whether the
    target was met); RMS errors of the solved velocity and (mean-free)
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
        sol, its, rel = ctx.gmres(rp, col, val, b, restart=100, max_iter=20000, rtol=rtol, row_scaling=row_scaling)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        # the unscaled relative residual ||b - A x|| / ||b|| (with row scaling,
        # rel_residual is that of the equilibrated rows R (b - A x))
        ax = ctx.spmv(rp, col, val, sol)
        ctx.sync()
        true_rel = float(torch.linalg.norm(b - ax) / torch.linalg.norm(b))
        s = sol.cpu().numpy()
        us, ps = s[:2 * n].reshape(n, 2).T, s[2 * n:3 * n]
        eu = float(np.sqrt(np.mean((us - d["u"]) ** 2)))
        ep = float(np.sqrt(np.mean(((ps - ps.mean()) - (d["p"] - d["p"].mean())) ** 2)))
        return {"unknowns": int(rp.shape[0] - 1), "nnz": int(col.shape[0]), "iterations": its, "rel_residual": rel,
                "unscaled_rel_residual": true_rel, "converged": bool(np.isfinite(rel) and rel <= rtol),
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


def serving(n_requests, nmax=5e4, rates=(100.0, 200.0), seed=0):
    """The serving stream: Poisson arrivals of stencil requests -- 2D/3D
    clouds of log-uniform nmin..nmax points, degree 2..4, scalar (gradient +
    Laplacian) or divergence-free (vector Laplacian) basis -- through the
    continuous-batching server (FP32 + refinement) and through the plain
    per-request FP64 path (one request at a time, in arrival order), at each
    offered rate.  The same requests at every rate (arrival times scale as
    1 / rate).  Latency = arrival to completion; targets/s = completed
    targets over the time from the first arrival to the last completion."""
    import threading

    import torch

    from paper_2104_14447_gb300 import gmls, inputs

    base = inputs.request_stream(n_requests, 1.0, seed, nmax=nmax)  # arrival times at 1 request/s
    clouds = []
    for r in base:
        n_axis = max(3, int(round(r["n"] ** (1.0 / r["dim"]))))
        clouds.append(inputs.jittered_grid(r["dim"], n_axis, seed=r["seed"]))
    spec = []
    for r in base:
        b = gmls.SCALAR if r["basis"] == "scalar" else gmls.DIVFREE
        fns = [gmls.GRAD, gmls.LAPLACIAN] if b == gmls.SCALAR else [gmls.VEC_LAPLACIAN]
        spec.append((b, r["degree"], SERVE_K[(r["dim"], b, r["degree"])], fns))
    total_targets = int(sum(c.shape[1] for c in clouds))

    def run_server(rate):
        srv = gmls.Server(torch.cuda.current_device(), arena_bytes=48 << 30, streams=4, max_inflight=8)
        tickets = [None] * len(base)
        t0 = time.perf_counter()

        def client():
            for i, r in enumerate(base):
                dt = r["t"] / rate - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                b, m, k, fns = spec[i]
                tickets[i] = srv.submit(clouds[i], b, m, k, fns, precision=gmls.FP32_REFINE)

        th = threading.Thread(target=client)
        th.start()
        pending = set(range(len(base)))
        while pending:
            for i in list(pending):
                if tickets[i] is not None and srv.wait(tickets[i], 0):
                    srv.release(tickets[i])
                    pending.discard(i)
            time.sleep(0.0005)
        th.join()
        st = srv.stats()
        srv.close()
        return {"p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
                "targets_per_s": st["targets_per_s"], "elapsed_s": st["elapsed_s"]}

    def run_plain_fp64(rate):
        ctx = gmls.Context(torch.cuda.current_device(), arena_bytes=48 << 30)
        ctx.set_option(gmls.OPT_AUTOTUNE, 0)
        lat, t0 = [], time.perf_counter()
        for i, r in enumerate(base):
            dt = r["t"] / rate - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            b, m, k, fns = spec[i]
            cid = ctx.cloud(clouds[i])
            nid = ctx.neighbors(cid, k, 1.5)
            sid = ctx.stencils(nid, b, m, fns, precision=gmls.FP64)
            ctx.sync()
            lat.append((time.perf_counter() - t0 - r["t"] / rate) * 1e3)
            for h in (sid, nid, cid):
                ctx.release(h)
        el = time.perf_counter() - t0 - base[0]["t"] / rate
        ctx.close()
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(np.mean(lat)), "targets_per_s": total_targets / el, "elapsed_s": el}

    out = {"requests": n_requests, "targets": total_targets,
           "request_mix": f"2D/3D (p = 1/2), n log-uniform in [1e3, {nmax:.0e}], degree U{{2,3,4}}, scalar or "
                          "div-free basis (p = 1/2), k from the fixed-k table",
           "size_cap": (f"n <= {nmax:.0e} instead of 5e5, so that {n_requests} requests run in about a minute "
                        "per arm" if nmax < 5e5 else None),
           "rates": {}}
    for rate in rates:
        offered = total_targets / (base[-1]["t"] / rate)
        srv = run_server(rate)
        plain = run_plain_fp64(rate)
        out["rates"][f"{rate:g}_per_s"] = {
            "offered_targets_per_s": offered,
            "continuous_batching_fp32_refine": srv, "plain_per_request_fp64": plain,
            "regime": "below capacity (latency)" if srv["targets_per_s"] >= 0.95 * offered else "backlog",
            "p99_speedup_vs_fp64": plain["p99_ms"] / srv["p99_ms"] if srv["p99_ms"] > 0 else None,
            "throughput_speedup_vs_fp64": srv["targets_per_s"] / plain["targets_per_s"]}
    return out


def stokes2d_oracle_check(ctx, n_sample=2000):
    """The 2D section's GPU weights (FP32 + refinement) on a seeded sample of
    targets against the oracle's, with the oracle's neighbour lists."""
    import torch

    import oracle
    from paper_2104_14447_gb300 import gmls, inputs

    oracle.build()
    x = workload_points()
    n = x.shape[1]
    sample = np.unique((inputs.uniform(9, 5, n_sample) * n).astype(np.int64)).astype(np.int32)
    sdev = torch.from_numpy(sample.astype(np.int64)).to(ctx.device)
    cid = ctx.cloud(x)
    errs, lists_equal = {}, True
    for key, k, basis, fn, kind in (("grad", K_SCALAR, gmls.SCALAR, gmls.GRAD, "scalar"),
                                    ("div", K_SCALAR, gmls.SCALAR, gmls.DIV, "scalar"),
                                    ("vec_laplacian", K_DIVFREE, gmls.DIVFREE, gmls.VEC_LAPLACIAN, "divfree")):
        nid = ctx.neighbors(cid, k, EPS_FACTOR)
        sid = ctx.stencils(nid, basis, DEGREE, [fn], precision=gmls.FP32_REFINE)
        _, rows, nc, _ = ctx.stencil_info(sid, fn)
        wg = ctx.weights(sid, fn).view(n, rows, k, nc)[sdev].cpu().numpy()
        idx = ctx.export(nid, gmls.X_NBR_INDEX, torch.int32).view(n, k)[sdev].cpu().numpy()
        oi, oe = oracle.knn(x, sample, k, EPS_FACTOR, method="grid")
        lists_equal &= bool(np.array_equal(idx, oi))
        off = np.arange(0, len(sample) * k + 1, k)
        wo, _, _ = oracle.stencils(x, sample, off, oi.reshape(-1), oe, kind, DEGREE, key)
        a = np.abs(wg.reshape(wo.shape) - wo).reshape(len(sample), wo.shape[1], -1).max(axis=2)
        b = np.abs(wo).reshape(len(sample), wo.shape[1], -1).max(axis=2)
        errs[key] = float(np.max(a / np.where(b > 0, b, 1.0)))
        ctx.release(sid)
        ctx.release(nid)
    ctx.release(cid)
    return {"sample": f"{len(sample)} seeded targets", "neighbour_lists_equal": lists_equal,
            "max_rel_err_vs_oracle": errs}


def small_2d(ctx, steps=20):
    """The 1,024-target case: 32 x 32 jittered grid in the unit square (seed
    0), 12 nearest neighbours, eps = 1.5 d_12, degree-2 scalar basis,
    Laplacian and gradient, plain FP64 on one stream; launch- and
    latency-bound (1,024 targets cannot fill the GPU)."""
    import torch

    from paper_2104_14447_gb300 import gmls, inputs

    x = torch.from_numpy(inputs.jittered_grid(2, 32, seed=0)).to(ctx.device)
    n = x.shape[1]

    def step():
        cid = ctx.cloud(x)
        nid = ctx.neighbors(cid, 12, EPS_FACTOR)
        sid = ctx.stencils(nid, gmls.SCALAR, 2, [gmls.LAPLACIAN, gmls.GRAD], precision=gmls.FP64)
        csr = [ctx.assemble_csr(sid, gmls.LAPLACIAN), ctx.assemble_csr(sid, gmls.GRAD)]
        return (cid, nid, sid), csr

    for _ in range(3):
        h, _ = step()
        for hd in reversed(h):
            ctx.release(hd)
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        h, _ = step()
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        for hd in reversed(h):
            ctx.release(hd)
    med = float(np.median(ms))
    return {"workload": "2D 32x32 jittered grid, 12 nbrs, scalar m=2, Laplacian + gradient, FP64, one stream",
            "targets": n, "ms_per_step": med, "targets_per_s": n / med * 1e3,
            "roofline": "not meaningful: launch- and latency-bound"}


# --------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle, as it stands, on the host cores: the headline workload (the
    porous cube), each step a seeded 1 % sample of its targets through the
    whole pipeline (kNN lists, scalar and div-free stencils, CSR)."""
    import oracle
    from paper_2104_14447_gb300 import inputs

    oracle.build()
    pc = inputs.porous_cube(n_axis=args.porous_n_axis)
    x = pc["x"]
    n = x.shape[1]
    m = max(1, int(round(0.01 * n)))
    targets = np.unique((inputs.uniform(7, 133, m) * n).astype(np.int64)).astype(np.int32)
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)

    def run():
        ns = len(targets)
        i80, e80 = oracle.knn(x, targets, P_K_DIVFREE, EPS_FACTOR, method="grid")
        i40, e40 = oracle.knn(x, targets, P_K_SCALAR, EPS_FACTOR, method="grid")
        off40, off80 = np.arange(0, ns * P_K_SCALAR + 1, P_K_SCALAR), np.arange(0, ns * P_K_DIVFREE + 1, P_K_DIVFREE)
        extra = dict(bflag=pc["bflag"][targets], normals=pc["normals"].T[targets])
        for kind, key, i, o, e, ex in (("scalar", "grad", i40, off40, e40, extra),
                                        ("scalar", "laplacian", i40, off40, e40, extra),
                                        ("divfree", "vec_laplacian", i80, off80, e80, {})):
            w, _, _ = oracle.stencils(x, targets, o, i.reshape(-1), e, kind, P_DEGREE, key, **ex)
            oracle.csr(o, i.reshape(-1), w, n)

    for _ in range(args.warmup):
        run()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        run()
        times.append(time.perf_counter() - t0)
    total = float(np.sum(times))
    value = len(targets) * args.steps / total
    sample = (f"seeded 1 % of the targets per step ({len(targets)} of {n}), full pipeline incl. kNN and CSR; "
              "the rate extrapolates linearly to the whole workload")
    return {"metric": METRIC, "value": value, "unit": "targets/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "targets_per_gpu": n, "precision": "fp64 (oracle)",
                       "degree": P_DEGREE, "neighbours": [P_K_SCALAR, P_K_DIVFREE], "eps_factor": EPS_FACTOR},
            "cpu_baseline": {"value": value, "unit": "targets/s", "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "targets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--arena-gb", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement of the headline")
    ap.add_argument("--no-secondary", action="store_true", help="headline only")
    ap.add_argument("--no-stokes", action="store_true", help="skip the Stokes-system sections")
    ap.add_argument("--porous-n-axis", type=int, default=P_N_AXIS, help="lattice of the headline (profiling only)")
    ap.add_argument("--no-batched", action="store_true", help="skip the uneven-batch section")
    ap.add_argument("--no-shapes", action="store_true", help="skip the per-shape FP32 / FP64 section")
    ap.add_argument("--e2e-ranges", type=int, default=E2E_CHUNKS, help="target ranges of the end-to-end pipelines")
    ap.add_argument("--e2e-copy-streams", type=int, default=2, help="copy streams of the end-to-end pipelines")
    ap.add_argument("--e2e-host", choices=["huge", "pinned"], default="huge",
                    help="host result buffers: huge-page memory registered with CUDA, or pin_memory")
    ap.add_argument("--batched-n", type=int, default=500_000, help="targets per cloud of the uneven batch")
    ap.add_argument("--poly-sizes", type=int, nargs="+", default=[6, 12, 24, 48, 96],
                    help="points per axis of the 3D polynomial tables (Sec. 4.1)")
    ap.add_argument("--only", choices=["batched", "stokes2d", "poly3d", "shapes"], default=None,
                    help="profiling: run only this secondary section (--steps timed steps) and print it")
    ap.add_argument("--n-axis", type=int, default=512, help="2D section grid (profiling only; the benchmark is 512)")
    ap.add_argument("--serve-requests", type=int, default=2000, help="serving stream length (0: skip)")
    ap.add_argument("--serve-nmax", type=float, default=5e4, help="largest request (points) of the serving stream")
    ap.add_argument("--no-graph", dest="graph", action="store_false")
    ap.add_argument("--solve-512", action="store_true", help="also solve the 512 x 512 Stokes system (rtol 1e-10, 1e-12)")
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
        if args.only == "stokes2d":
            res = stokes2d_section(ctx, args)
        elif args.only == "poly3d":
            res = polynomial_tables_3d(ctx, sizes=tuple(args.poly_sizes))
        elif args.only == "shapes":
            res = shapes(ctx)
        else:
            res = batched_uneven(ctx, n_per_dim=args.batched_n, steps=args.steps)[0]
        print(json.dumps(res), flush=True)
        ctx.close()
        return
    if world > 1:
        import torch

        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    out, ctx, gs = run_headline(args, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = porous_cpu_baseline(gs)
    pc = gs["pc"]
    del gs
    if rank == 0 and world == 1 and not args.no_secondary:
        if not args.no_stokes:
            out["porous_stokes_system"] = porous_stokes_section(ctx, pc)
        sec = {"fp32_refine": stokes2d_section(ctx, args), "fp64": stokes2d_section(ctx, args, "fp64")}
        if not args.no_cpu_baseline:
            sec["oracle_check"] = stokes2d_oracle_check(ctx)
        if not args.no_stokes:
            sec["stokes_system"] = stokes_system(ctx)
            sec["stokes_system"]["solve"] = stokes_solve(ctx)
            sec["stokes_system"]["solve_256"] = stokes_solve(ctx, 256, full=False)
            if args.solve_512:  # opt-in: about 5 s of GMRES
                sec["stokes_system"]["solve_512"] = stokes_solve(ctx, 512, full=False)
                sec["stokes_system"]["solve_512_rtol_1e-12"] = stokes_solve(ctx, 512, full=False, rtol=1e-12)
        out["stokes2d_512"] = sec
        if not args.no_stokes:
            out["polynomial_3d"] = polynomial_tables_3d(ctx, sizes=tuple(args.poly_sizes))
        out["small_2d_1024"] = small_2d(ctx)
        if not args.no_shapes:
            out["shapes"] = shapes(ctx)
        if not args.no_batched:
            out["batched_uneven"], gsb = batched_uneven(ctx, n_per_dim=args.batched_n)
            if not args.no_cpu_baseline:  # the oracle's side of the sampled comparison
                out["batched_uneven"]["oracle_check"] = batched_oracle_errors(gsb)
        if args.serve_requests > 0:
            out["serving"] = serving(args.serve_requests, nmax=args.serve_nmax)
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        import torch

        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
