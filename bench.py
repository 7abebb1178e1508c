#!/usr/bin/env python
"""Benchmark of the MBIR full-range ISAM solve (Alg. 1) on GB300.

Workload (N = 1): the 1024 A-scan x 2048 spectral-sample B-scan, layered
tissue-like specimen, 12-bit counts with background subtraction, FP32; one
step = one MBIR solve of `--iters` (200) FISTA iterations including lambda =
0.01 ||A^H s_d||_inf and the relative-residual evaluation every 20 iterations.
The Lipschitz constant is a per-geometry constant cached in the plan (first
warm-up step).  value = FISTA iterations per second over all ranks; ranks
solve independent B-scans (replicas, weak scaling, no data-path collective).

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FISTA iters/s (A+Aᴴ) at 1024×2048 B-scan & 256²×2048 vol; % HBM roofline"
UNIT = "iter/s"
CHECK_EVERY = 20
L2_FLUSH_BYTES = 256 << 20     # > 129 MB L2


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the A+A^H, FP64, cuFFT, calibration, batch and volume lines")
    ap.add_argument("--no-volume", action="store_true", help="skip the 256^2 x 2048 volume line")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="seconds of oracle work per host core in the CPU baseline")
    ap.add_argument("--cpu-workers", type=int, default=0,
                    help="host processes for the CPU baseline (0: all cores)")
    ap.add_argument("--no-batch", action="store_true", help="skip the 96-B-scan batch line")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the built-in launch shapes (for runs under a profiler)")
    ap.add_argument("--batch-iters", type=int, default=200)
    ap.add_argument("--calib-steps", type=int, default=50,
                    help="Adam steps timed in the calibration line")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--L", type=float, default=0.0,
                    help="Lipschitz constant to use (0: power-iteration estimate, cached)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU oracle timing (the reported baseline and the reference arm)
# ----------------------------------------------------------------------------
ORACLE_SLICE = 64          # A-scans per oracle process


def _oracle_slice_rate(job):
    """One host process: FP64 oracle FISTA iterations on a 64-A-scan slice of
    the B-scan workload (same band, spectral and depth sampling, dispersion),
    timed for `seconds` after one warm iteration.  Returns (iterations,
    seconds) for that slice."""
    seconds, index = job
    from oracle import isam_oracle as O
    from paper_1905_06058_gb300 import inputs as I
    wl = I.config2(dtype=np.complex64)
    g = wl.geom
    nxs = ORACLE_SLICE
    lo = (index * nxs) % g.nx
    g.nx = nxs
    eta = wl.eta[:, lo:lo + nxs].astype(np.complex128)
    op = O.IsamOracle(g, "nufft")
    s = op.forward(eta)
    lam = 0.01 * np.abs(op.adjoint(s)).max()
    L = 1.4
    O.fista(op.forward, op.adjoint, s, lam, L, max_iter=1, shape=op.image_shape)   # warm
    n, t0 = 0, time.perf_counter()
    while True:
        O.fista(op.forward, op.adjoint, s, lam, L, max_iter=1, shape=op.image_shape)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds and n >= 2:
            break
    return n, el


def oracle_iteration_rate(seconds: float, workers: int = 0):
    """The FP64 oracle on all host cores: `workers` processes (spawned, one
    thread each) time FISTA iterations concurrently, each on its own 64-A-scan
    slice of the 1024 x 2048 B-scan.  The cost of an iteration is linear in the
    A-scans (per-column NUFFTs; the lateral FFT is a small part), so the
    full-B-scan rate is the sum of the slices' rates x 64 / 1024."""
    import multiprocessing as mp
    workers = workers or os.cpu_count() or 1
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                           "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(workers) as pool:
            res = pool.map(_oracle_slice_rate, [(seconds, i) for i in range(workers)])
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    slice_rate = sum(n / el for n, el in res)
    rate = slice_rate * ORACLE_SLICE / 1024
    n_tot = sum(n for n, _ in res)
    el_max = max(el for _, el in res)
    sample = (f"FP64 NumPy oracle (nufft mode, J=6): {workers} host processes, one thread each, "
              f"each timing FISTA iterations on its own {ORACLE_SLICE}-A-scan slice of the "
              f"1024x2048 B-scan ({n_tot} slice iterations in {el_max:.1f} s); the summed slice "
              f"rate scaled by {ORACLE_SLICE}/1024 (extrapolated)")
    return {"value": rate, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample,
            "extrapolated_from_ascans": ORACLE_SLICE}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    per_step = max(args.cpu_seconds / max(args.steps, 1), 0.5)
    t0 = time.perf_counter()
    cpu = oracle_iteration_rate(per_step * args.steps, args.cpu_workers)
    rate = cpu["value"]
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / rate * args.iters, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "bscan_1024x2048_fp32", "nx": 1024, "nk": 2048, "nz": 2048,
                       "iters_per_step": args.iters},
            "cpu_baseline": cpu,
            "extrapolated_from_ascans": ORACLE_SLICE,
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def algorithmic_bytes(cls: str, n_img: int, n_spec: int, real_bytes=4) -> int:
    """Compulsory HBM bytes per launch of each kernel class (B-scan layout)."""
    c = 2 * real_bytes
    return {"ax_fwd": c * (n_img + n_spec),          # read eta_hat, write S
            "ax_adj": c * (n_spec + n_img),          # read R_hat, write G_hat
            "ax_fused": c * 2 * n_img + c * n_spec // 2,   # eta_hat in, u_hat (or G) out,
                                                            # half of F s_d
            # u_hat, z^{k-1} in; z^k, eta_hat^{k+1} out (the residual-check
            # iterations, 1 in 20, also read z^{k-2}: counted as the 4-array pass)
            "lat_update": c * n_img * 4}.get(cls)


# Per-launch figures of the dominant kernels from one ncu capture each
# (profiles/, caches flushed before each replayed launch).  A capture holds
# for the kernel sources it was taken from: `sha` is the hash of those files
# (kernel_sources_sha); when the sources have changed since, the figures are
# reported as null.  dram: dram__bytes_read.sum + dram__bytes_write.sum;
# table: the part of the reads that is the plan's Stolt table (16 B per
# (|q| class, k) sample, read once per launch from DRAM when the caches are
# cold); smem_wavefronts: l1tex__data_pipe_lsu_wavefronts_mem_shared.sum.
# Volume figures are per launch of the 256 x 256 x 2048 case, scaled from a
# 128 x 128 x 2048 capture by the column pairs (32,770 / 8,194).
KERNEL_SOURCES = {
    "ax_fused": ["k_axial.cuh", "k_axial.cu", "fft_smem.cuh", "fft_col16.cuh", "internal.cuh",
                 "common.cuh"],
    "lat_update": ["k_lateral.cu", "fft_smem.cuh", "internal.cuh", "common.cuh"],
}
NCU_CAPTURES = {
    "bscan_1024x2048": {
        "ax_fused": {"sha": "42f5dcc0e5acc4f1", "dram": 42414080, "table": 16809984,
                     "smem_wavefronts": 6623241},
        "lat_update": {"sha": "aa2e880b8cc2d1e4", "dram": 34312448, "table": 0,
                       "smem_wavefronts": 2414784},
    },
    "volume_256x256x2048": {
        # 128 x 128 x 2048 capture with the plan's Stolt table: 781,895,936 B and
        # 116,578,155 wavefronts over 8,194 pairs
        "ax_fused": {"sha": "42f5dcc0e5acc4f1", "dram": 3127011206, "table": 545292288,
                     "smem_wavefronts": 466227256},
    },
}


def kernel_sources_sha(kind: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_1905_06058_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def capture_of(workload: str, kind: str):
    c = NCU_CAPTURES.get(workload, {}).get(kind)
    if c and c["sha"] == kernel_sources_sha(kind):
        return c
    return None


def roofline_of(kern: dict, kind: str, abytes: int, workload: str, peak: float, peak_src: str,
                sm_mhz, sms: int, note: str) -> dict:
    """HBM roofline of one kernel class from the live per-launch CUDA-event
    average, plus the fraction of the shared-memory pipe (one wavefront per SM
    per cycle) its captured wavefront count takes at the measured clock."""
    avg_ms = kern[kind]["ms"] / max(kern[kind]["launches"], 1)
    achieved = abytes / (avg_ms / 1000.0) / 1e9
    cap = capture_of(workload, kind)
    r = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
         "frac": achieved / peak, "traffic": cap["dram"] if cap else None, "kernel": kind,
         "bytes_per_launch": abytes, "avg_launch_us": avg_ms * 1000.0,
         "peak_source": peak_src, "note": note}
    if cap:
        r["traffic_split"] = {"algorithmic": abytes, "stolt_table": cap.get("table", 0),
                              "capture_sha": cap["sha"]}
        if cap.get("smem_wavefronts") and sm_mhz:
            cyc = sms * sm_mhz * 1e6 * avg_ms / 1000.0
            r["smem_pipe"] = {"counter": "l1tex__data_pipe_lsu_wavefronts_mem_shared.sum",
                              "wavefronts_per_launch": cap["smem_wavefronts"],
                              "sms": sms, "sm_mhz": sm_mhz,
                              "frac": cap["smem_wavefronts"] / cyc}
    else:
        r["traffic_note"] = "no ncu capture of the current kernel sources"
    return r


def reduce_over_ranks(torch, elapsed, units, world, device):
    """Whole-job timing: the slowest rank's elapsed time and the units (FISTA
    iterations) of all ranks.  Ranks solve independent problems, so this scalar
    reduction is the only collective."""
    if world <= 1:
        return float(elapsed), float(units)
    import torch.distributed as dist
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.barrier()
    return float(t[0]), float(u[0])


def make_problem(torch, plan, wl, seed):
    from paper_1905_06058_gb300 import inputs as I
    eta = torch.from_numpy(wl.eta.astype(np.complex64)).cuda()
    s_clean = plan.forward(eta).cpu().numpy()
    k = wl.geom.k_min + (wl.geom.k_max - wl.geom.k_min) / (wl.geom.nk - 1) * np.arange(wl.geom.nk)
    s = I.detector_counts(s_clean, k, np.random.default_rng(seed))
    return torch.from_numpy(s).cuda(), eta


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    import __graft_entry__ as G
    if rank == 0:
        G.build()
    if world > 1:
        torch.distributed.barrier()
    G.build()
    from paper_1905_06058_gb300 import inputs as I
    from paper_1905_06058_gb300.isam import Plan

    wl = I.config2(dtype=np.complex64)
    if rank:
        wl.eta = I.layered_specimen(np.random.default_rng(wl.seed + 7919 * rank), wl.eta.shape,
                                    6, 0.02, 200, np.complex64)
    g = wl.geom
    plan = Plan(g, precision="fp32")
    s_d, _ = make_problem(torch, plan, wl, wl.seed + rank)
    # launch shapes timed on this plan (profilers distort that timing: they use
    # --no-autotune, the built-in shapes)
    tuned = plan.autotune() if not args.no_autotune else "built-in shapes"
    out = torch.empty(plan.image_shape, dtype=torch.complex64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    opts = dict(lambda_rel=wl.lambda_rel, max_iter=args.iters, tol=1e-12, check_every=CHECK_EVERY,
                L=args.L)

    for _ in range(args.warmup):
        plan.solve(s_d, out=out, **opts)
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    launches = 0
    iters_done = 0
    infos = []
    for i in range(args.steps):
        flush.zero_()                           # evict L2 between timed steps
        ev[i][0].record(stream)
        _, info = plan.solve(s_d, out=out, **opts)
        ev[i][1].record(stream)
        launches += plan.last_launch_count()
        iters_done += info["iterations"]
        infos.append(info)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    # the same steps again with every kernel launch bracketed by CUDA events on
    # the plan's stream: per-kernel average durations for the roofline
    plan.profile(True)
    for i in range(args.steps):
        flush.zero_()
        plan.solve(s_d, out=out, **opts)
    prof = plan.profile_read()
    plan.profile(False)
    total_ms, all_iters = reduce_over_ranks(torch, total_ms, iters_done, world, "cuda")
    value = all_iters / (total_ms / 1000.0)

    # dominant kernel and its live roofline
    n_img, n_spec = plan.image_shape[1] * plan.image_shape[2], plan.spec_shape[1] * plan.spec_shape[2]
    kern = {k: {"ms": v[0], "launches": v[1], "share": None} for k, v in prof.items()}
    tot = sum(v["ms"] for v in kern.values()) or 1.0
    for v in kern.values():
        v["share"] = v["ms"] / tot
    dom = max((k for k in kern if algorithmic_bytes(k, n_img, n_spec)), key=lambda k: kern[k]["ms"])
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    roofline = roofline_of(kern, dom, algorithmic_bytes(dom, n_img, n_spec), "bscan_1024x2048",
                           peak, peak_src, clk.get("sm_mhz"), sms,
                           "the B-scan's per-iteration working set (~72 MiB) fits the 129 MB "
                           "L2: L2 is flushed only between 200-iteration steps, so this is "
                           "algorithmic bytes over time, not DRAM-bound throughput")
    per_iter_bytes = sum(algorithmic_bytes(k, n_img, n_spec) for k in ("ax_fused", "lat_update"))
    iter_gbs = per_iter_bytes * value / max(world, 1) / 1e9

    # end to end through the host-buffer C-ABI entry point
    s_h = s_d.cpu().pin_memory()
    o_h = torch.empty(plan.image_shape, dtype=torch.complex64).pin_memory()
    plan.solve_host(s_h, o_h, **opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_iters = 0
    for _ in range(args.steps):
        info = plan.solve_host(s_h, o_h, **opts)
        e2e_iters += info["iterations"]
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s, e2e_iters = reduce_over_ranks(torch, e2e_s, e2e_iters, world, "cuda")
    e2e = {"value": e2e_iters / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(s_h.numel() * 4), "d2h_bytes_per_step": int(o_h.numel() * 8)}

    extras = {}
    if not args.no_extras and rank == 0:
        extras = run_extras(torch, plan, s_d, wl, args, infos[-1]["L"],
                            dict(peak=peak, peak_src=peak_src, sm_mhz=clk.get("sm_mhz"),
                                 sms=sms))

    if rank == 0:
        cpu = oracle_iteration_rate(args.cpu_seconds, args.cpu_workers) \
            if world == 1 and not args.no_cpu else None
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "bscan_1024x2048_fp32", "nx": 1024, "nk": 2048,
                           "nz": 2048, "iters_per_step": args.iters, "nufft_J": 6,
                           "lambda_rel": wl.lambda_rel, "check_every": CHECK_EVERY,
                           "l2": "flushed between timed steps (256 MiB write)",
                           "parallelism": f"replicas x{world}",
                           "autotuned": tuned},
                "gpu_launches": launches, "clocks": clk, "e2e": e2e, "roofline": roofline,
                "cpu_baseline": cpu,
                "iteration_gbs_algorithmic": iter_gbs,
                "kernels": kern, "rr_last": infos[-1]["rr"] if infos else None,
                "extras": extras}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_extras(torch, plan, s_d, wl, args, L, roof):
    """A+A^H applications/s, the plain FP64 GPU path, cuFFT, calibration, the
    batch and the volume."""
    from paper_1905_06058_gb300 import inputs as I
    from paper_1905_06058_gb300.isam import Plan
    ex = {}
    x = torch.empty(plan.image_shape, dtype=torch.complex64, device="cuda")
    y = torch.empty(plan.spec_shape, dtype=torch.float32, device="cuda")
    plan.adjoint(s_d, out=x)
    for _ in range(3):
        plan.forward(x, out=y)
        plan.adjoint(y, out=x)
    torch.cuda.synchronize()
    reps = 50
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        plan.forward(x, out=y)
        plan.adjoint(y, out=x)
    b.record()
    torch.cuda.synchronize()
    ex["aah_per_s"] = reps / (a.elapsed_time(b) / 1000.0)
    # plain FP64 GPU path (same kernels instantiated for double), same workload
    p64 = Plan(wl.geom, precision="fp64")
    s64 = s_d.double()
    o64 = torch.empty(plan.image_shape, dtype=torch.complex128, device="cuda")
    it64 = 20
    p64.solve(s64, out=o64, lambda_rel=wl.lambda_rel, max_iter=2, L=L)
    torch.cuda.synchronize()
    a.record()
    _, info = p64.solve(s64, out=o64, lambda_rel=wl.lambda_rel, max_iter=it64, L=L)
    b.record()
    torch.cuda.synchronize()
    ex["fp64_iters_per_s"] = it64 / (a.elapsed_time(b) / 1000.0)
    p64.close()
    ex["cufft_comparison_us"] = cufft_comparison(torch, plan)
    ex["calibration"] = run_calibration(torch, args.calib_steps)
    if not args.no_batch:
        ex["batch"] = run_batch(torch, args.batch_iters)
    if not args.no_volume:
        ex["volume"] = run_volume(torch, roof)
    return ex


def cufft_comparison(torch, plan):
    """cuFFT (through torch.fft) on the transforms one FISTA iteration needs, for
    comparison with the hand-written kernels: two lateral FFTs (forward and
    inverse, length nx over nz columns) and two zero-padded axial FFTs (length
    K = 2 nz over nx columns).  Device time per call, microseconds."""
    ny, nx, nz = plan.image_shape
    x = torch.randn(nx, nz, dtype=torch.complex64, device="cuda")
    y = torch.randn(nx, nz, dtype=torch.complex64, device="cuda")
    out = {}
    for name, fn in (("lateral_fft_nx", lambda: torch.fft.fft(x, dim=0)),
                     ("axial_fft_2nz_zero_padded", lambda: torch.fft.fft(y, n=2 * nz, dim=1))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 50
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        out[name] = a.elapsed_time(b) / reps * 1000.0
    out["per_iteration_4_ffts"] = 2 * out["lateral_fft_nx"] + 2 * out["axial_fft_2nz_zero_padded"]
    return out


def run_calibration(torch, steps: int):
    """Calibration of (a2, a3, z0): Adam steps on the data fidelity of 16 B-scans
    (512 x 2048) through K = 20 unrolled FISTA iterations with checkpoints every
    5; one step is the unrolled solves, the model, and the gradient of all
    B-scans.  The spectra are made by the plan's own model at the hidden theta
    plus Gaussian noise; lambda and L are fixed at the start theta."""
    from paper_1905_06058_gb300 import calib
    from paper_1905_06058_gb300 import inputs as I
    from paper_1905_06058_gb300.isam import Plan
    wl = I.config5()
    plan = Plan(wl.geom)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(wl.K)
    spectra = []
    for eta in wl.etas:
        s = plan.forward(torch.from_numpy(eta).cuda())
        sigma = float(torch.linalg.vector_norm(s)) / (s.numel() ** 0.5 * 10 ** (wl.snr_db / 20))
        spectra.append(s + sigma * torch.randn(s.shape, generator=gen, device="cuda"))
    plan.set_model(wl.start[:4].tolist(), float(wl.start[4]))
    L = plan.lipschitz(iters=100, rtol=1e-6)
    lams = [wl.lambda_rel * plan.max_abs(plan.adjoint(s)) for s in spectra]
    calib.calibrate(plan, spectra, wl.start, lams, L, wl.K, wl.every, steps=1)   # warm-up
    res = calib.calibrate(plan, spectra, wl.start, lams, L, wl.K, wl.every, steps=steps)
    scale = calib.theta_scales(wl.geom)
    truth = np.array(list(wl.geom.disp) + [wl.geom.z0])
    err = lambda th: [float(abs(th[i] - truth[i]) / scale[i]) for i in (1, 2, 4)]
    norm = sum(float(torch.sum(s.double() ** 2)) for s in spectra)
    th = torch.from_numpy(truth)
    truth_loss = sum(float(calib.data_fidelity(s, th, plan, lm, L, wl.K, wl.every))
                     for s, lm in zip(spectra, lams)) / norm
    plan.close()
    return {"workload": wl.name, "K": wl.K, "checkpoint_every": wl.every, "steps": steps,
            "adam_steps_per_s": steps / res.seconds,
            "ms_per_bscan_step": res.seconds / steps / len(spectra) * 1e3,
            "loss_first": res.losses[0], "loss_last": res.losses[-1], "loss_best": res.best_loss,
            "loss_at_hidden_theta": truth_loss,
            "theta_error_start_a2_a3_z0": err(wl.start), "theta_error_end_a2_a3_z0": err(res.theta),
            "theta_error_best_a2_a3_z0": err(res.best_theta),
            "units": "a_i: rad at the band edge; z0: fraction of the depth range"}


def run_batch(torch, iters: int):
    """96 B-scans of uneven size (Nx 256..1024, Nk 1024/2048, own NA, dispersion,
    focus and lambda), each plan autotuned (isam_autotune), `iters` FISTA
    iterations each, recorded as one CUDA graph
    and replayed with one launch; against the same solves issued one after
    another through isam_solve.  Spectra come from each plan's own model plus
    30 dB noise; L from 50 power iterations (x 1.01)."""
    import time
    from paper_1905_06058_gb300 import inputs as I
    from paper_1905_06058_gb300.isam import Batch, Plan
    t_setup = time.perf_counter()
    ents = []
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4)
    for e in I.config4():
        plan = Plan(e.geom)
        s = plan.forward(torch.from_numpy(I.batch_specimen(e)).cuda())
        sigma = float(torch.linalg.vector_norm(s)) / (s.numel() ** 0.5 * 10 ** 1.5)
        s = s + sigma * torch.randn(s.shape, generator=gen, device="cuda")
        L = 1.01 * plan.lipschitz(iters=50, rtol=1e-6)
        plan.autotune()
        out = torch.empty(plan.image_shape, dtype=torch.complex64, device="cuda")
        ents.append((plan, s, out, dict(lambda_rel=e.lambda_rel, max_iter=iters, L=L)))
    b = Batch(ents)
    setup_s = time.perf_counter() - t_setup
    b.run()                                               # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    infos = b.run()
    t_graph = time.perf_counter() - t0
    entry_ms = sorted(b.entry_ms())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for plan, s, out, kw in ents:
        plan.solve(s, out=out, **kw)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    total = iters * len(ents)
    work = sum(p.geom.nx * p.geom.nk for p, *_ in ents) / (1024 * 2048)
    res = {"workload": f"{len(ents)} B-scans, Nx 256..1024, Nk 1024/2048",
           "iters_each": iters, "graph_kernels": b.kernel_count(),
           "graph_s": t_graph, "graph_iters_per_s": total / t_graph,
           "sequential_solve_s": t_seq, "sequential_iters_per_s": total / t_seq,
           "entry_latency_ms": {"p50": float(np.percentile(entry_ms, 50)),
                                "p95": float(np.percentile(entry_ms, 95)),
                                "min": entry_ms[0], "max": entry_ms[-1],
                                "definition": "device time from the graph's start to the end "
                                              "of each entry's solve (timing events recorded "
                                              "in the graph)"},
           "bscan_1024x2048_equivalents": work,
           "statuses_ok": sum(1 for i in infos if i["status"] == 0), "setup_s": setup_s}
    b.close()
    for plan, *_ in ents:
        plan.close()
    return res


def run_volume(torch, roof=None):
    """The 256 x 256 x 2048 volume (FP32): FISTA iterations/s over a timed
    40-iteration solve, A + A^H applications/s, and the roofline of its dominant
    kernel from a second, event-instrumented solve.  Every array is 1 GiB (8x the
    L2), so the kernels stream from DRAM.  L from 30 power iterations."""
    from paper_1905_06058_gb300 import inputs as I
    from paper_1905_06058_gb300.isam import Plan
    wl = I.config3(dtype=np.complex64)
    plan = Plan(wl.geom, precision="fp32")
    eta = torch.from_numpy(wl.eta).cuda()
    s = plan.forward(eta)
    del eta
    L = plan.lipschitz(iters=30, rtol=1e-6)
    out = torch.empty(plan.image_shape, dtype=torch.complex64, device="cuda")
    plan.solve(s, out=out, lambda_rel=wl.lambda_rel, max_iter=2, L=L)
    torch.cuda.synchronize()
    it = 40
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    plan.solve(s, out=out, lambda_rel=wl.lambda_rel, max_iter=it, L=L)
    b.record()
    torch.cuda.synchronize()
    rate = it / (a.elapsed_time(b) / 1000.0)
    # per-kernel device time of the same solve, every launch bracketed by events
    plan.profile(True)
    plan.solve(s, out=out, lambda_rel=wl.lambda_rel, max_iter=10, L=L)
    prof = plan.profile_read()
    plan.profile(False)
    kern = {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items() if v[1]}
    # standalone A + A^H applications (C-ABI operators)
    y = torch.empty(plan.spec_shape, dtype=torch.float32, device="cuda")
    plan.forward(out, out=y)
    plan.adjoint(y, out=out)
    torch.cuda.synchronize()
    reps = 5
    a.record()
    for _ in range(reps):
        plan.forward(out, out=y)
        plan.adjoint(y, out=out)
    b.record()
    torch.cuda.synchronize()
    aah = reps / (a.elapsed_time(b) / 1000.0)
    n = wl.geom.nx * wl.geom.ny * wl.geom.nz
    plan.close()
    res = {"workload": wl.name, "iters_per_s": rate, "aah_per_s": aah, "L_estimate_iters": 30,
           "timed_iterations": it, "kernels": kern,
           "iteration_gbs_algorithmic": 60 * n * rate / 1e9}
    if roof:
        res["roofline"] = roofline_of(kern, "ax_fused", 20 * n, "volume_256x256x2048",
                                      roof["peak"], roof["peak_src"], roof["sm_mhz"], roof["sms"],
                                      "every array is 1 GiB (8x the L2): DRAM-bound inputs")
    return res


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
