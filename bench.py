"""Benchmark of the ADMM reconstruction hot path on GB300.

One step = one complete reconstruction of the N=128 workload (12 coils, 64
golden-angle spokes x 256 readout samples, 30 ADMM x 8 CG iterations,
lambda=1e-3, beta=1): DFT-factor generation for the step's trajectory
(Alg. 1) followed by Alg. 4 with Alg. 2 inside, in the BF16x3 tensor-core
form.  The TF32 tensor-core form and the plain FP32 form are timed beside it
on the same GPU.  Other workloads: --workload n256 (N=256, 32 coils, 128 x
512 samples, 50 x 10 iterations), batch64 (64 heterogeneous reconstructions
in one launch), serve (the serving loop under Poisson arrivals).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload W]

Prints one JSON line.  Each rank reconstructs its own problems (independent
reconstructions: weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

# single-reconstruction workloads: N=128 (the headline), N=256, and the
# paper's two shapes with its Table I parameters and tolerance exits
WORKLOADS = {"n128": synth.config_medium, "n256": synth.config_large,
             "paper128x64": synth.config_paper_128x64, "paper1024x512": synth.config_paper_1024x512}
# the paper's own times for its shapes (TPU v3, float32-equivalent; context, another machine)
PAPER_TIMES_S = {"paper_128x64_c12_s13x128": {"2 TPU v3 cores": 0.1363, "16 TPU v3 cores": 0.0356},
                 "paper_1024x512_c12_s101x1024": {"128 TPU v3 cores": 3.387, "2048 TPU v3 cores": 0.286}}
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# product kernels on this workload, from one ncu capture each (the summaries
# under profiles/ give the command), keyed by a hash of the product kernels'
# sources as captured: a changed kernel reports traffic null until it is
# captured again.
NCU_TRAFFIC = {
    ("adj_tc_kernel", "n128_c12_s64x256"): (40.44e6, "4e07d50614bdf6d9", "profiles/adj_tc_kernel_n128.md"),
    ("fwd_tc_kernel", "n128_c12_s64x256"): (51.99e6, "4e07d50614bdf6d9", "profiles/fwd_tc_kernel_n128.md"),
    ("adj_tc_kernel", "n256_c32_s128x512"): (1303.54e6, "4e07d50614bdf6d9", "profiles/adj_tc_kernel_n256.md"),
}
TC_SOURCES = ("nudft_tc.cu", "tc_ptx.cuh")


def tc_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in TC_SOURCES:
        with open(os.path.join(ROOT, "paper_2006_14080_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(kernel: str, workload: str):
    entry = NCU_TRAFFIC.get((kernel, workload))
    if entry is None or entry[1] != tc_source_hash():
        return None, None
    return entry[0], entry[2]


def max_over_ranks_fn(dist, device):
    """The maximum over ranks of a host number (the slowest rank's clock); the
    identity without a process group."""
    def reduce_max(v: float) -> float:
        if dist is None:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return reduce_max


def whole_job_rate(units_per_rank: float, slowest_ms: float, world: int) -> float:
    """Units all ranks processed per second of the slowest rank."""
    return world * units_per_rank / (slowest_ms / 1e3)


def gemm_peak_tflops(tf32: bool, seconds: float = 3.0, n: int = 8192):
    """cuBLAS FP32 GEMM throughput on this GPU (TF32 tensor cores when tf32,
    else the FFMA path): (best of 10 single calls, mean over a back-to-back
    loop of `seconds`), in TFLOP/s; the denominators of the TF32 and FP32
    forms, which MEASURED_PEAKS.json does not carry."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = tf32
    try:
        a = torch.randn(n, n, device="cuda")
        b = torch.randn(n, n, device="cuda")
        c = torch.empty(n, n, device="cuda")
        flops = 2.0 * n ** 3
        for _ in range(3):
            torch.matmul(a, b, out=c)
        best = float("inf")
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        reps = max(1, int(seconds * 1e3 / best))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            torch.matmul(a, b, out=c)
        e1.record()
        e1.synchronize()
        sustained = reps * flops / (e0.elapsed_time(e1) * 1e-3) / 1e12
        del a, b, c
        return flops / (best * 1e-3) / 1e12, sustained
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            m = json.load(fh)
        return m, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def problem(workload: str = "n128"):
    return WORKLOADS[workload]()


def workload_name(p) -> str:
    return f"{p.name}_admm{p.admm_iters}x{p.cg_iters}"


def metric_name(p) -> str:
    size = f"N={p.nx}" if p.nx == p.ny else f"{p.nx}x{p.ny}"
    angles = "golden-angle" if p.angles == "golden" else "uniform-angle"
    tol = "" if not (p.rtol or p.atol) else f" (rtol {p.rtol:g}, atol {p.atol:g} exits)"
    return (f"ADMM recon/s, {size} image, {p.nc} coils, {p.spokes} {angles} spokes x {p.readout} samples, "
            f"{p.admm_iters} ADMM x {p.cg_iters} CG{tol}, BF16x3 tensor-core NUDFT (TF32 and FP32 forms beside)")


def normal_ops_per_recon(p):
    # A x0 plus one A d per CG step in every outer step, plus F^H d once (half an op)
    return p.admm_iters * (p.cg_iters + 1) + 0.5


def useful_flops_per_product(p):
    # complex MACs of one separable DFT product, 8 real flops each
    return 8.0 * p.nk * p.nx * p.ny * p.nc


def cg_step_bytes(p, ksplit):
    """Algorithmic bytes of one CG-step launch (BF16x3 form): reads of the
    partial images (ksplit per coil, rows padded to 64 pixels), the coil maps
    and d, r, x; writes of A d, x, r', d' and the next forward operand (BF16
    hi + lo per coil and pixel)."""
    nx_pad = -(-p.nx // 64) * 64
    npix = p.nx * p.ny
    reads = 8.0 * (ksplit * p.nc * nx_pad * p.ny + p.nc * nx_pad * p.ny + 3 * npix)
    writes = 8.0 * (4 * npix + p.nc * npix)
    return reads + writes


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [q.strip() for q in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        loaded = [v for v in sm if v > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def with_cpu_leg(args, rank, world) -> bool:
    """The CPU-baseline leg (the FP64 oracle on the host) runs on rank 0 of a
    one-GPU run only."""
    return not args.no_cpu_baseline and world == 1 and rank == 0


def oracle_measurement(p):
    """CPU-baseline leg: the problem's measurement formed with the FP64 oracle's
    forward operator plus the seeded noise (how the stored oracle
    reconstructions under tests/golden were made)."""
    import oracle
    return oracle.measurements(p)


def kspace_is_oracle(kspace_np, gpath) -> bool:
    """Whether kspace_np is the input of the stored oracle reconstruction
    (its L2 norm and sampled entries match the stored fingerprint)."""
    g = np.load(gpath)
    flat = np.asarray(kspace_np).reshape(-1)
    norm = float(np.linalg.norm(flat.astype(np.complex128)))
    return abs(norm - float(g["d_norm"])) <= 1e-9 * float(g["d_norm"]) and \
        np.array_equal(flat[g["d_idx"]], g["d_samples"])


def clock_scaled_peak(pk, clocks):
    """Dense BF16 peak for the product kernels: the measured burst figure when
    they ran at the maximum SM clock (median within 3% of it), else the
    measured sustained figure (a kernel held below the maximum clock by the
    power cap through a long step, as the sustained cuBLAS loop was)."""
    burst = float(pk["bf16_tflops"])
    sustained = float(pk.get("bf16_tflops_sustained", burst))
    sm, smax = clocks.get("sm_mhz"), clocks.get("sm_max_mhz")
    if not sm or not smax:
        return burst, "burst bf16 (no clock samples)"
    if float(sm) >= 0.97 * float(smax):
        return burst, f"burst bf16 (median SM clock {sm:.0f} of {smax:.0f} MHz)"
    return sustained, f"sustained bf16 (median SM clock {sm:.0f} of {smax:.0f} MHz, below the maximum)"


def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_2006_14080_gb300 as mr

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    p = problem(args.workload)
    # a created (non-legacy) stream: the library captures each reconstruction
    # into a CUDA graph on first use and replays it on such streams
    torch.cuda.set_stream(torch.cuda.Stream(device=dev))
    stream = torch.cuda.current_stream()
    traj = torch.from_numpy(p.traj).to(dev)
    maps = torch.from_numpy(p.maps).to(dev)
    ximg = torch.from_numpy(p.image_true).to(dev)

    # measurement: the phantom's k-space plus the seeded noise.  On rank 0 of a
    # one-GPU run the CPU-baseline leg forms it with the FP64 oracle's forward
    # operator, exactly as the stored oracle reconstructions were made, so that
    # the reported NRMSE compares images of the same input; otherwise with the
    # library's FP32 forward operator.
    kspace_np, measurement = None, "library FP32 forward operator + seeded noise"
    if with_cpu_leg(args, rank, world) and os.path.exists(os.path.join(ROOT, "tests", "golden",
                                                                        f"admm_{p.name}.npz")):
        kspace_np = oracle_measurement(p)
        measurement = "FP64 oracle forward operator + seeded noise (the stored oracle reconstruction's input)"
    if kspace_np is None:
        with mr.Plan(p.nx, p.ny, p.nc, traj, "fp32") as plan32:
            d_clean = mr.nudft_forward(plan32, ximg, maps).cpu().numpy()
        kspace_np = synth.add_noise(d_clean, p.noise, p.noise_level)
    kspace = torch.from_numpy(kspace_np).to(dev)

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    max_over_ranks = max_over_ranks_fn(dist, dev)

    def timed_steps(plan, out, steps, warmup, host=None, plan_timed=False):
        """Returns (per-step device ms list, launches per step)."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]

        def one(i_ev=None):
            if host is not None:
                # end-to-end: pinned host inputs in, image out, all inside the timed region
                h_traj, h_k, h_maps, h_out, d_traj, d_k, d_maps = host
                d_traj.copy_(h_traj, non_blocking=True)
                d_k.copy_(h_k, non_blocking=True)
                d_maps.copy_(h_maps, non_blocking=True)
                plan.set_trajectory(d_traj)
                mr.admm_reconstruct(plan, d_k, d_maps, p.lam, p.beta, p.admm_iters, p.cg_iters, out=out,
                                    rtol=p.rtol, atol=p.atol)
                h_out.copy_(out, non_blocking=True)
            else:
                plan.set_trajectory(traj)
                mr.admm_reconstruct(plan, kspace, maps, p.lam, p.beta, p.admm_iters, p.cg_iters, out=out,
                                    rtol=p.rtol, atol=p.atol)

        for _ in range(warmup):
            one()
        barrier()
        if plan_timed:
            plan.read_timing()  # forget the warm-up launches
        l0 = plan.launch_count()
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            one()
            ev[i][1].record(stream)
        barrier()
        launches = plan.launch_count() - l0
        return [a.elapsed_time(b) for a, b in ev], launches

    forms = set(args.forms.split(","))
    results = {}
    out = torch.empty((p.nx, p.ny), dtype=torch.complex64, device=dev)
    with mr.Plan(p.nx, p.ny, p.nc, traj, "bf16x3") as plan:
        if args.tiles:  # fixed schedule (e.g. to profile the configuration a tuned run chose)
            plan.set_tiles(*(int(v) for v in args.tiles.split(",")))
            tuned = plan.config()
        else:
            tuned = plan.autotune(repeats=5)  # set-up, outside the timed region
        gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local_rank)).split(",")[local_rank]) \
            if os.environ.get("CUDA_VISIBLE_DEVICES") else local_rank
        with ClockSampler(gpu_index) as clk:
            # headline: each reconstruction replays the captured CUDA graph
            times, launches = timed_steps(plan, out, args.steps, args.warmup)
            # kernel durations: the same steps launched directly, every product
            # and reduction launch bracketed by CUDA events on this stream
            plan.set_timing(True)
            ktimes, _ = timed_steps(plan, out, max(2, args.steps // 4), 1, plan_timed=True)
            timing = plan.read_timing()
            plan.set_timing(False)
        results["bf16x3"] = (times, launches, timing, clk.summary())
        kernel_pass_ms = sum(ktimes)
        x_bf16 = out.cpu().numpy()

        e2e_times, h2d, d2h = [float("nan")], 0, 0
        if "e2e" in forms:
            # end to end through the same API with pinned host buffers
            host = (torch.from_numpy(p.traj).pin_memory(), torch.from_numpy(kspace_np).pin_memory(),
                    torch.from_numpy(p.maps).pin_memory(),
                    torch.empty((p.nx, p.ny), dtype=torch.complex64).pin_memory(),
                    torch.empty_like(traj), torch.empty_like(kspace), torch.empty_like(maps))
            e2e_times, _ = timed_steps(plan, out, args.steps, max(1, args.warmup // 2), host=host)
            h2d = sum(t.numel() * t.element_size() for t in host[:3])
            d2h = host[3].numel() * host[3].element_size()

    fp32_steps = max(2, min(args.steps, 3))
    t32, l32, timing32, x_fp32 = [float("nan")], 0, {"fwd_ms": 0, "fwd_launches": 0, "adj_ms": 0,
                                                      "adj_launches": 0}, None
    if "fp32" in forms:
        with mr.Plan(p.nx, p.ny, p.nc, traj, "fp32") as plan32:
            plan32.set_timing(True)
            t32, l32 = timed_steps(plan32, out, fp32_steps, 1, plan_timed=True)
            timing32 = plan32.read_timing()
            x_fp32 = out.cpu().numpy()

    tf32 = None
    if "tf32" in forms:
        with mr.Plan(p.nx, p.ny, p.nc, traj, "tf32") as plan_t:
            tuned_t = plan_t.autotune(repeats=5)
            tt, lt_ = timed_steps(plan_t, out, args.steps, args.warmup)
            x_tf32 = out.cpu().numpy()
            plan_t.set_timing(True)
            timed_steps(plan_t, out, max(2, args.steps // 4), 1, plan_timed=True)
            timing_t = plan_t.read_timing()
        tf32 = (tt, lt_, timing_t, tuned_t, x_tf32)

    # denominators of the TF32 and FP32 forms (cuBLAS GEMMs, outside every timed region)
    gemm_peaks = {}
    for name, on in (("tf32", True), ("fp32", False)):
        if name in forms:
            burst, sustained = gemm_peak_tflops(on)
            gemm_peaks[name] = {"burst": burst, "sustained": sustained}

    # ---------------------------------------------------------------- report
    times, launches, timing, clocks = results["bf16x3"]
    total_ms = max_over_ranks(sum(times))
    e2e_ms = max_over_ranks(sum(e2e_times))
    t32_ms = max_over_ranks(sum(t32))
    if rank != 0:
        return None
    recon_s = whole_job_rate(args.steps, total_ms, world)
    flops_prod = useful_flops_per_product(p)
    pk, pk_kind = peaks()
    # dominant kernel: the product kernel with the larger share of the timed region
    fwd_avg = timing["fwd_ms"] / max(1, timing["fwd_launches"])
    adj_avg = timing["adj_ms"] / max(1, timing["adj_launches"])
    dom = "adj" if timing["adj_ms"] >= timing["fwd_ms"] else "fwd"
    dom_avg_ms = adj_avg if dom == "adj" else fwd_avg
    executed = 3.0 * flops_prod  # hi*hi + hi*lo + lo*hi bf16 tensor products
    achieved = executed / (dom_avg_ms * 1e-3) / 1e12
    peak_tf, peak_note = clock_scaled_peak(pk, clocks)
    # with tolerance exits the operator count is data-dependent: count the
    # ADMM steps one reconstruction takes and leave the TFLOP/s out
    tol_steps = None
    if p.rtol > 0 or p.atol > 0:
        import torch
        with mr.Plan(p.nx, p.ny, p.nc, traj, "bf16x3") as plan_c:
            ah = torch.full((p.admm_iters,), -1.0, dtype=torch.float64, device=dev)
            mr.admm_reconstruct(plan_c, kspace, maps, p.lam, p.beta, p.admm_iters, p.cg_iters, out=out,
                                rtol=p.rtol, atol=p.atol, alpha_hist=ah)
            tol_steps = int((ah >= 0).sum().item())
    useful_tflops_step = None if tol_steps is not None else \
        normal_ops_per_recon(p) * 2 * flops_prod / (total_ms / args.steps * 1e-3) / 1e12
    dom_kernel = "adj_tc_kernel" if dom == "adj" else "fwd_tc_kernel"
    traffic, traffic_src = captured_traffic(dom_kernel, p.name)
    red_avg = timing["red_ms"] / max(1, timing["red_launches"])
    red_bytes = cg_step_bytes(p, (tuned or {}).get("adj_ksplit", 0) or 0)
    nrmse_vs_golden = None
    gpath = os.path.join(ROOT, "tests", "golden", f"admm_{p.name}.npz")
    if os.path.exists(gpath) and kspace_is_oracle(kspace_np, gpath):
        xg = np.load(gpath)["x"]
        nrmse_vs_golden = {"bf16x3": float(np.linalg.norm(x_bf16 - xg) / np.linalg.norm(xg))}
        if x_fp32 is not None:
            nrmse_vs_golden["fp32"] = float(np.linalg.norm(x_fp32 - xg) / np.linalg.norm(xg))
    line = {
        "metric": metric_name(p),
        "value": recon_s,
        "unit": "recon/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16x3/f32",
        "data": f"synthetic (seeded ellipse phantom, Gaussian coil maps, {p.angles}-angle radial, "
                f"{100 * p.noise_level:g}% noise)",
        "config": {"workload": workload_name(p), "nx": p.nx, "ny": p.ny, "coils": p.nc, "spokes": p.spokes,
                   "readout": p.readout, "admm_iters": p.admm_iters, "cg_iters": p.cg_iters, "lambda": p.lam,
                   "beta": p.beta, "l2": "flushed (512 MB write) between timed steps",
                   "step": "factor generation for the step's trajectory + full ADMM reconstruction"},
        "e2e": {"value": whole_job_rate(args.steps, e2e_ms, world), "unit": "recon/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "tuning": tuned,
        "roofline": {"bound": "tensor", "kernel": dom_kernel,
                     "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s", "frac": achieved / peak_tf,
                     "traffic": traffic, "traffic_unit": "bytes per launch", "traffic_source": traffic_src,
                     "note": f"executed bf16 tensor flops (3 products x 8*nk*nx*ny*nc) per launch / mean launch "
                             f"time ({dom_avg_ms:.4f} ms over {timing[dom + '_launches']} launches, CUDA events on "
                             f"the launching stream in a directly-launched pass of the same steps); peak = "
                             f"{pk_kind} {peak_note}"},
        "nudft": {"fwd_ms_per_launch": fwd_avg, "adj_ms_per_launch": adj_avg,
                  "fwd_useful_tflops": flops_prod / (fwd_avg * 1e-3) / 1e12,
                  "adj_useful_tflops": flops_prod / (adj_avg * 1e-3) / 1e12,
                  "product_share_of_step": (timing["fwd_ms"] + timing["adj_ms"]) / kernel_pass_ms,
                  "reduce_ms_per_launch": red_avg,
                  "reduce_share_of_step": timing["red_ms"] / kernel_pass_ms,
                  "reduce_bytes_per_launch": red_bytes,
                  "reduce_gbs": red_bytes / (red_avg * 1e-3) / 1e9 if red_avg > 0 else None,
                  "reduce_note": "the CG-step kernel: algorithmic bytes (partial images, maps, state, next forward "
                                 "operand) per launch / mean event-timed launch; served mostly from L2 (the "
                                 "partial images stay there between the adjoint and this kernel), so the HBM copy "
                                 "peak bounds it only loosely",
                  "direct_launch_ms_per_step": kernel_pass_ms / len(ktimes),
                  "recon_useful_tflops": useful_tflops_step},
        "fp32_form": {"value": whole_job_rate(fp32_steps, t32_ms, world), "unit": "recon/s",
                      "ms_per_step": t32_ms / fp32_steps, "gpu_launches": l32,
                      "fwd_ms_per_launch": timing32["fwd_ms"] / max(1, timing32["fwd_launches"]),
                      "adj_ms_per_launch": timing32["adj_ms"] / max(1, timing32["adj_launches"])},
        "gemm_peaks_tflops": gemm_peaks,
        "tf32_form": None,
        "nrmse_vs_fp64_oracle": nrmse_vs_golden,
        "measurement": measurement,
        "tolerances": None if tol_steps is None else {"rtol": p.rtol, "atol": p.atol, "admm_steps_taken": tol_steps,
                                                      "admm_iters_max": p.admm_iters, "cg_iters_max": p.cg_iters},
        "paper_context_s": PAPER_TIMES_S.get(p.name),
        "clocks": clocks,
    }
    if tf32 is not None:
        tt, lt_, timing_t, tuned_t, x_tf32 = tf32
        tt_ms = max_over_ranks(sum(tt))
        f_avg = timing_t["fwd_ms"] / max(1, timing_t["fwd_launches"])
        a_avg = timing_t["adj_ms"] / max(1, timing_t["adj_launches"])
        # one TF32 product executes the useful flops once; TF32 dense peak =
        # the cuBLAS TF32 GEMM measured in this run (sustained), else the
        # measured BF16 peak x the nominal TF32/BF16 ratio (1.1 / 2.25 PFLOP/s)
        if "tf32" in gemm_peaks:
            tf32_peak, tf32_note = gemm_peaks["tf32"]["sustained"], "cuBLAS TF32 GEMM 8192^3, measured in this run"
        else:
            tf32_peak, tf32_note = peak_tf * 1.1 / 2.25, f"{pk_kind} sustained bf16 x 1.1/2.25 (nominal TF32/BF16)"
        line["tf32_form"] = {
            "value": whole_job_rate(args.steps, tt_ms, world), "unit": "recon/s", "ms_per_step": tt_ms / args.steps,
            "gpu_launches": lt_, "tuning": tuned_t, "fwd_ms_per_launch": f_avg, "adj_ms_per_launch": a_avg,
            "fwd_tflops": flops_prod / (f_avg * 1e-3) / 1e12, "adj_tflops": flops_prod / (a_avg * 1e-3) / 1e12,
            "peak_tflops": tf32_peak, "peak_note": tf32_note,
            "adj_frac": flops_prod / (a_avg * 1e-3) / 1e12 / tf32_peak,
            "fwd_frac": flops_prod / (f_avg * 1e-3) / 1e12 / tf32_peak,
        }
    if line["fp32_form"] is not None and "fp32" in gemm_peaks:
        f32 = line["fp32_form"]
        pk32 = gemm_peaks["fp32"]["sustained"]
        f32.update({"fwd_tflops": flops_prod / (f32["fwd_ms_per_launch"] * 1e-3) / 1e12,
                    "adj_tflops": flops_prod / (f32["adj_ms_per_launch"] * 1e-3) / 1e12,
                    "peak_tflops": pk32, "peak_note": "cuBLAS FP32 GEMM (FFMA, TF32 off) 8192^3, measured in this run"})
        f32["adj_frac"] = f32["adj_tflops"] / pk32
        f32["fwd_frac"] = f32["fwd_tflops"] / pk32
    if tf32 is not None:
        if nrmse_vs_golden is not None:
            xg = np.load(gpath)["x"]
            nrmse_vs_golden["tf32"] = float(np.linalg.norm(x_tf32 - xg) / np.linalg.norm(xg))
    if "fp32" not in forms:
        line["fp32_form"] = None
    if "e2e" not in forms:
        line["e2e"] = None
    if args.extras and world == 1 and args.workload == "n128":
        # the other single-GPU workloads, each as a sub-object of this line
        line["small"] = small_block(args, mr, dev, with_cpu_leg(args, rank, world))
        line["large"] = large_block(args, mr, dev, pk, pk_kind)
        line["serve"] = serve_block(args, mr, dev)
    if with_cpu_leg(args, rank, world):
        line["cpu_baseline"] = cpu_baseline(p, args.cpu_seconds)
    return line


def _graph_rate(mr, plan, p, kspace, maps, out, steps, warmup, flush, stream, traj=None):
    """recon/s of one plan with graph replay: warm-up, then `steps` timed
    reconstructions (CUDA events on the launching stream, L2 flushed before
    each).  Returns (recon/s, ms per step, launches per step)."""
    import torch
    def one():
        if traj is not None:
            plan.set_trajectory(traj)
        mr.admm_reconstruct(plan, kspace, maps, p.lam, p.beta, p.admm_iters, p.cg_iters, out=out)
    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    l0 = plan.launch_count()
    for e0, e1 in ev:
        flush.zero_()
        e0.record(stream)
        one()
        e1.record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    return 1e3 / ms, ms, (plan.launch_count() - l0) // steps


def small_block(args, mr, dev, oracle_input):
    """The N=32 workload (4 coils, 16 uniform spokes x 64, 10 ADMM x 5 CG) in
    the FP32 and BF16x3 forms: recon/s and NRMSE against the stored FP64
    oracle reconstruction of the same input."""
    import torch
    p = synth.config_small()
    stream = torch.cuda.current_stream()
    traj, maps = torch.from_numpy(p.traj).to(dev), torch.from_numpy(p.maps).to(dev)
    if oracle_input:
        kspace_np = oracle_measurement(p)
    else:
        with mr.Plan(p.nx, p.ny, p.nc, traj, "fp32") as p32:
            kspace_np = synth.add_noise(mr.nudft_forward(p32, torch.from_numpy(p.image_true).to(dev),
                                                         maps).cpu().numpy(), p.noise, p.noise_level)
    kspace = torch.from_numpy(kspace_np).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    out = torch.empty((p.nx, p.ny), dtype=torch.complex64, device=dev)
    gpath = os.path.join(ROOT, "tests", "golden", f"admm_{p.name}.npz")
    same = os.path.exists(gpath) and kspace_is_oracle(kspace_np, gpath)
    res = {"workload": workload_name(p), "steps": args.steps, "warmup": args.warmup}
    for prec in ("fp32", "bf16x3"):
        with mr.Plan(p.nx, p.ny, p.nc, traj, prec) as plan:
            rate, ms, launches = _graph_rate(mr, plan, p, kspace, maps, out, args.steps, args.warmup, flush, stream)
            x = out.cpu().numpy()
        entry = {"value": rate, "unit": "recon/s", "ms_per_step": ms, "gpu_launches_per_step": launches}
        if same:
            xg = np.load(gpath)["x"]
            entry["nrmse_vs_fp64_oracle"] = float(np.linalg.norm(x - xg) / np.linalg.norm(xg))
        res[prec] = entry
    return res


def large_block(args, mr, dev, pk, pk_kind):
    """The N=256 workload (32 coils, 128 golden-angle spokes x 512, 50 ADMM x
    10 CG) in the BF16x3 form: recon/s with graph replay (1 warm-up, 2 timed
    steps, L2 flushed), and the roofline of its dominant product kernel from
    one directly-launched, event-timed reconstruction.  Input: the library's
    FP32 forward operator plus the seeded noise (image parity at this size is
    a GPU test against the oracle's 3 x 3 reconstruction)."""
    import torch
    p = synth.config_large()
    stream = torch.cuda.current_stream()
    traj, maps = torch.from_numpy(p.traj).to(dev), torch.from_numpy(p.maps).to(dev)
    with mr.Plan(p.nx, p.ny, p.nc, traj, "fp32") as p32:
        d = mr.nudft_forward(p32, torch.from_numpy(p.image_true).to(dev), maps).cpu().numpy()
    kspace = torch.from_numpy(synth.add_noise(d, p.noise, p.noise_level)).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    out = torch.empty((p.nx, p.ny), dtype=torch.complex64, device=dev)
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or 0)
    with mr.Plan(p.nx, p.ny, p.nc, traj, "bf16x3") as plan:
        tuned = plan.autotune(repeats=3)
        with ClockSampler(gpu_index) as clk:
            rate, ms, launches = _graph_rate(mr, plan, p, kspace, maps, out, 2, 1, flush, stream)
            plan.set_timing(True)
            plan.read_timing()
            mr.admm_reconstruct(plan, kspace, maps, p.lam, p.beta, p.admm_iters, p.cg_iters, out=out)
            timing = plan.read_timing()
            plan.set_timing(False)
    clocks = clk.summary()
    flops_prod = useful_flops_per_product(p)
    fwd_avg = timing["fwd_ms"] / max(1, timing["fwd_launches"])
    adj_avg = timing["adj_ms"] / max(1, timing["adj_launches"])
    dom = "adj" if timing["adj_ms"] >= timing["fwd_ms"] else "fwd"
    dom_avg = adj_avg if dom == "adj" else fwd_avg
    achieved = 3.0 * flops_prod / (dom_avg * 1e-3) / 1e12
    peak_tf, peak_note = clock_scaled_peak(pk, clocks)
    kern = "adj_tc_kernel" if dom == "adj" else "fwd_tc_kernel"
    traffic, traffic_src = captured_traffic(kern, p.name)
    return {"workload": workload_name(p), "value": rate, "unit": "recon/s", "ms_per_step": ms, "steps": 2,
            "warmup": 1, "gpu_launches_per_step": launches, "tuning": tuned,
            "useful_tflops": normal_ops_per_recon(p) * 2 * flops_prod / (ms * 1e-3) / 1e12,
            "nudft": {"fwd_ms_per_launch": fwd_avg, "adj_ms_per_launch": adj_avg,
                      "reduce_ms_per_launch": timing["red_ms"] / max(1, timing["red_launches"])},
            "roofline": {"bound": "tensor", "kernel": kern, "achieved": achieved, "peak": peak_tf,
                         "unit": "TFLOP/s", "frac": achieved / peak_tf, "traffic": traffic,
                         "traffic_source": traffic_src,
                         "note": f"executed bf16 tensor flops per launch / mean launch time ({dom_avg:.4f} ms); "
                                 f"peak = {pk_kind} {peak_note}"},
            "clocks": clocks}


def serve_block(args, mr, dev):
    """A short serving run (requests sized as the batch items, Poisson
    arrivals at 0.8 x the measured burst capacity) for the p50/p99 latency of
    the served BF16x3 form."""
    res = serve_measure(args, mr, dev, n_requests=args.line_serve_requests, rates=[0.8], precisions=["bf16x3"],
                        waves=1, warmup=1)
    head = res["bf16x3"]["sweep"][0]
    return {"workload": f"serve{args.line_serve_requests}_poisson", "value": head["value"], "unit": "recon/s",
            "latency_ms": {"p50": head["p50_ms"], "p99": head["p99_ms"], "max": head["max_ms"]},
            "burst_capacity_recon_s": res["bf16x3"]["burst_capacity_recon_s"],
            "arrival_rate_recon_s": head["arrival_rate_recon_s"], "requests": head["requests"],
            "timing": "host wall clock, submit to image in host memory"}


def run_batch(args, rank, world, local_rank):
    """64 heterogeneous reconstructions (N in {64..256}, 8-32 coils, 32-200
    golden-angle spokes of 2N samples, 30 ADMM x 8 CG) in one batched launch
    per step; each rank runs its own batch."""
    import torch
    import paper_2006_14080_gb300 as mr

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    torch.cuda.set_stream(torch.cuda.Stream(device=dev))
    stream = torch.cuda.current_stream()
    probs = [synth.batch_item(j) for j in range(args.batch_items)]
    items, plans = [], []
    useful = 0.0
    for p in probs:
        traj = torch.from_numpy(p.traj).to(dev)
        maps = torch.from_numpy(p.maps).to(dev)
        with mr.Plan(p.nx, p.ny, p.nc, traj, "fp32") as p32:
            d_clean = mr.nudft_forward(p32, torch.from_numpy(p.image_true).to(dev), maps).cpu().numpy()
        kspace = torch.from_numpy(synth.add_noise(d_clean, p.noise, p.noise_level)).to(dev)
        plan = mr.Plan(p.nx, p.ny, p.nc, traj, "bf16x3")
        plans.append(plan)
        items.append({"plan": plan, "kspace": kspace, "coil_maps": maps,
                      "out": torch.empty((p.nx, p.ny), dtype=torch.complex64, device=dev),
                      "lam": p.lam, "beta": p.beta, "admm_iters": p.admm_iters, "cg_iters": p.cg_iters})
        useful += normal_ops_per_recon(p) * 2 * useful_flops_per_product(p)
    resident = sum(pl.device_bytes() for pl in plans)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    batch = mr.Batch()
    for _ in range(max(1, args.warmup)):
        batch.reconstruct(items)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local_rank)).split(",")[local_rank]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES") else local_rank
    with ClockSampler(gpu_index) as clk:
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            batch.reconstruct(items)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        # end to end: every step copies each item's k-space and coil maps in from
        # pinned host memory and its image out, around the same batched launch
        host = [(it["kspace"].cpu().pin_memory(), it["coil_maps"].cpu().pin_memory(),
                 torch.empty_like(it["out"], device="cpu").pin_memory()) for it in items]
        ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            ev2[i][0].record(stream)
            for it, (hk, hm, _) in zip(items, host):
                it["kspace"].copy_(hk, non_blocking=True)
                it["coil_maps"].copy_(hm, non_blocking=True)
            batch.reconstruct(items)
            for it, (_, _, ho) in zip(items, host):
                ho.copy_(it["out"], non_blocking=True)
            ev2[i][1].record(stream)
        torch.cuda.synchronize()
    # the same items one after another, each through its own plan's cached
    # reconstruction graph (the comparison for the batched launch)
    for it in items:
        mr.admm_reconstruct(it["plan"], it["kspace"], it["coil_maps"], it["lam"], it["beta"], it["admm_iters"],
                            it["cg_iters"], out=it["out"])
    torch.cuda.synchronize()
    seq_ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    flush.zero_()
    seq_ev[0].record(stream)
    for it in items:
        mr.admm_reconstruct(it["plan"], it["kspace"], it["coil_maps"], it["lam"], it["beta"], it["admm_iters"],
                            it["cg_iters"], out=it["out"])
    seq_ev[1].record(stream)
    torch.cuda.synchronize()
    seq_ms = max_over_ranks_fn(dist, dev)(seq_ev[0].elapsed_time(seq_ev[1]))
    total_ms = max_over_ranks_fn(dist, dev)(sum(a.elapsed_time(b) for a, b in ev))
    e2e_ms = max_over_ranks_fn(dist, dev)(sum(a.elapsed_time(b) for a, b in ev2))
    h2d = sum(hk.numel() * hk.element_size() + hm.numel() * hm.element_size() for hk, hm, _ in host)
    d2h = sum(ho.numel() * ho.element_size() for _, _, ho in host)
    launches = batch.launch_count()
    batch.close()
    for pl in plans:
        pl.close()
    if rank != 0:
        return None
    n = len(items)
    return {
        "metric": f"ADMM recon/s, batch of {n} heterogeneous reconstructions (N 64-256, 8-32 coils, 32-200 "
                  f"golden-angle spokes x 2N, 30 ADMM x 8 CG), BF16x3, one batched graph launch per step",
        "value": whole_job_rate(n * args.steps, total_ms, world), "unit": "recon/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3/f32",
        "data": "synthetic (seeded per item)",
        "config": {"workload": f"batch{n}_hetero_admm30x8", "items": n, "l2": "flushed between timed steps",
                   "resident_plan_bytes": resident},
        "useful_tflops": useful * args.steps / (total_ms / 1e3) / 1e12,
        "sequential": {"value": n / (seq_ms / 1e3), "unit": "recon/s", "ms": seq_ms,
                       "note": "the same items reconstructed one after another on the same stream, each replaying "
                               "its plan's captured graph (one timed pass)"},
        "e2e": {"value": whole_job_rate(n * args.steps, e2e_ms, world), "unit": "recon/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches * args.steps,  # kernels in one replay x timed steps
        "clocks": clk.summary(),
    }


def serve_measure(args, mr, dev, n_requests, rates, precisions, waves, warmup):
    """Serving measurement: `n_requests` heterogeneous requests (sizes as the
    batch items, each with its own phantom, maps, noise and trajectory)
    arriving from host memory as a Poisson process, admitted under a
    device-memory budget and run concurrently.  Per precision: a burst of the
    first requests measures the server's capacity; then each arrival rate (a
    multiple of that capacity) gets `waves` waves (the first rate) or one
    (the others) of the requests.  Latency = submission to image in host
    memory (host wall clock)."""
    import threading
    import torch

    probs = [synth.serve_request(r) for r in range(n_requests)]
    reqs = []
    for p in probs:
        traj = torch.from_numpy(p.traj).to(dev)
        maps = torch.from_numpy(p.maps).to(dev)
        with mr.Plan(p.nx, p.ny, p.nc, traj, "fp32") as p32:
            d_clean = mr.nudft_forward(p32, torch.from_numpy(p.image_true).to(dev), maps).cpu().numpy()
        reqs.append((p.traj.astype(np.float32), synth.add_noise(d_clean, p.noise, p.noise_level).astype(np.complex64),
                     p.maps.astype(np.complex64), p.lam, p.beta, p.admm_iters, p.cg_iters))
    torch.cuda.synchronize()
    budget = int(args.serve_budget_gb * (1 << 30))

    def wave(srv, items, gaps):
        lat, tickets = [], []
        t0 = time.perf_counter()

        def feed():
            t_next = t0
            for r, g in zip(items, gaps):
                t_next += g
                dt = t_next - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                tickets.append(srv.submit(*r))
        th = threading.Thread(target=feed)
        th.start()
        q = 0
        while q < len(items):
            while len(tickets) <= q:
                time.sleep(1e-4)
            lat.append(srv.wait(tickets[q])[1])
            q += 1
        th.join()
        return time.perf_counter() - t0, lat

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, max(0, math.ceil(q * len(v)) - 1))]

    results = {}
    rng = np.random.default_rng(2020)
    for prec in precisions:
        items = reqs if prec != "fp32" else reqs[: max(1, min(len(reqs), args.serve_fp32_requests))]
        cap_items = items[: max(1, min(len(items), args.serve_capacity_requests))]
        with mr.Server(budget, max_inflight=args.serve_inflight, precision=prec) as srv:
            burst_s = 0.0
            for _ in range(max(1, warmup if prec != "fp32" else 1)):
                burst_s, _ = wave(srv, cap_items, [0.0] * len(cap_items))
            capacity = len(cap_items) / burst_s
            sweep = []
            for k, mult in enumerate(rates):
                nw = waves if (k == 0 and prec != "fp32") else 1
                # the first rate takes every request; the rest of the sweep a prefix
                wave_items = items if k == 0 or args.serve_sweep_requests <= 0 else \
                    items[: min(len(items), args.serve_sweep_requests)]
                total_s, lats = 0.0, []
                for _ in range(nw):
                    gaps = [0.0] + list(rng.exponential(1.0 / (mult * capacity), len(wave_items) - 1))
                    t, lat = wave(srv, wave_items, gaps)
                    total_s += t
                    lats += lat
                sweep.append({"rate_x_capacity": mult, "arrival_rate_recon_s": mult * capacity,
                              "requests": len(wave_items) * nw, "value": len(wave_items) * nw / total_s,
                              "p50_ms": pct(lats, 0.50), "p99_ms": pct(lats, 0.99), "max_ms": max(lats),
                              "wall_s": total_s})
            st = srv.stats()
        results[prec] = {"burst_capacity_recon_s": capacity, "capacity_requests": len(cap_items),
                         "sweep": sweep, "peak_resident_bytes": st["peak_resident_bytes"],
                         "cache": {k: st[k] for k in ("plan_hits", "plan_retargets", "maps_reused",
                                                      "graph_replays")}}
    return results


def run_serve(args, rank, world, local_rank):
    """The serving loop alone (--workload serve): value = requests / (last
    completion - first submission) at the first arrival rate, in the first
    precision listed."""
    import torch
    import paper_2006_14080_gb300 as mr

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    rates = [float(v) for v in args.serve_rates.split(",")]
    precisions = args.serve_precisions.split(",")
    with ClockSampler(local_rank) as clk:
        results = serve_measure(args, mr, dev, args.serve_requests, rates, precisions, args.steps, args.warmup)
    head = results[precisions[0]]["sweep"][0]
    n = args.serve_requests
    return {
        "metric": f"served ADMM recon/s, {n} heterogeneous requests (N 64-256, 8-32 coils, 32-200 "
                  "golden-angle spokes x 2N, 30 ADMM x 8 CG; own phantom, maps and trajectory each) from host "
                  f"memory, Poisson arrivals at {rates[0]} x burst capacity, {precisions[0].upper()}",
        "value": head["value"], "unit": "recon/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * head["wall_s"] / max(1, args.steps), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3/f32" if precisions[0] == "bf16x3" else precisions[0],
        "data": "synthetic (seeded per request)",
        "latency_ms": {"p50": head["p50_ms"], "p99": head["p99_ms"], "max": head["max_ms"]},
        "forms": results,
        "config": {"workload": f"serve{n}_poisson", "budget_bytes": int(args.serve_budget_gb * (1 << 30)),
                   "max_inflight": args.serve_inflight, "rates_x_capacity": rates,
                   "fp32_requests": min(n, args.serve_fp32_requests),
                   "timing": "host wall clock, submit to image in host memory"},
        "clocks": clk.summary(),
    }


# complex MACs above which one oracle normal operator takes too long to time
# whole (N=256: 1.4e11, about 45 s on 16 cores): the sample is then the
# forward operator on a slice of the k-space samples, scaled to a normal operator
ORACLE_WHOLE_OP_MACS = 2e10


def oracle_sample(p, budget_s):
    """Time the FP64 oracle's normal operator (Eq. 11) at the workload's size;
    one reconstruction needs normal_ops_per_recon() of them.  Returns
    (seconds per normal operator, timed calls, threads, description)."""
    import oracle
    rng = np.random.default_rng(7)
    x = synth.random_complex(rng, (p.nx, p.ny)).astype(np.complex128)
    macs = float(p.nk) * p.nx * p.ny * p.nc
    if macs <= ORACLE_WHOLE_OP_MACS:
        call, scale = (lambda: oracle.normal(p.traj, p.maps, p.beta, x)), 1.0
        what = "FP64 normal operators (Eq. 11) at full size"
    else:
        m = max(1, int(p.nk * ORACLE_WHOLE_OP_MACS / 4 / macs))
        sub = np.ascontiguousarray(p.traj[:m])
        call, scale = (lambda: oracle.forward(sub, x, p.maps)), 2.0 * p.nk / m
        what = (f"FP64 forward operators on the first {m} of {p.nk} k-space samples at full image and coil "
                f"size, scaled by {scale:.1f} to one normal operator (forward + adjoint over all samples)")
    call()  # warm (threads, pages)
    times = []
    t_start = time.time()
    while not times or (time.time() - t_start < budget_s and len(times) < 8):
        t0 = time.perf_counter()
        call()
        times.append(time.perf_counter() - t0)
    per_op = statistics.median(times) * scale
    return per_op, len(times), oracle.get_threads(), what


def host_cpu():
    """The host's logical CPU count and model name (from /proc/cpuinfo where
    it names one, else the platform's processor string)."""
    import platform
    model = ""
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                key = ln.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in ln:
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
            for ln in out.splitlines():
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return os.cpu_count(), model or platform.processor() or platform.machine()


def one_thread_normal_op_s(p):
    """Seconds of one FP64 oracle normal operator on one host thread, from
    the forward operator on a slice of the k-space samples (about 1e9 complex
    MACs) scaled to forward + adjoint over all samples."""
    import oracle
    threads = oracle.get_threads()
    oracle.set_threads(1)
    try:
        rng = np.random.default_rng(7)
        x = synth.random_complex(rng, (p.nx, p.ny)).astype(np.complex128)
        m = max(1, min(p.nk, int(1e9 / (p.nx * p.ny * p.nc))))
        sub = np.ascontiguousarray(p.traj[:m])
        t0 = time.perf_counter()
        oracle.forward(sub, x, p.maps)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(threads)
    return dt * 2.0 * p.nk / m, m


def cpu_baseline(p, budget_s):
    per_op, n, threads, what = oracle_sample(p, budget_s)
    nproc, model = host_cpu()
    one_op, m = one_thread_normal_op_s(p)
    return {"value": 1.0 / (per_op * normal_ops_per_recon(p)), "unit": "recon/s", "cores": threads,
            "kind": "oracle", "nproc": nproc, "cpu_model": model,
            "one_thread_value": 1.0 / (one_op * normal_ops_per_recon(p)),
            "sample": f"{n} timed calls: {what} ({workload_name(p)}), {per_op:.2f} s per normal operator on "
                      f"{threads} threads, scaled by {normal_ops_per_recon(p)} operators per reconstruction "
                      f"(extrapolated); one thread: the forward operator on {m} of {p.nk} samples, "
                      f"{one_op:.1f} s per normal operator when scaled"}


def run_reference(args, rank):
    """The oracle arm: each step times one FP64 normal operator (Eq. 11) of
    the workload, the unit of work a reconstruction repeats
    normal_ops_per_recon() times; value = recon/s extrapolated from the timed
    operators (labelled as such), ms_per_step = the measured time per step."""
    if rank != 0:
        return None
    p = problem(args.workload if args.workload in WORKLOADS else "n128")
    per_op_s = []
    for _ in range(args.warmup):
        oracle_sample(p, 0.0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        per_op, _, threads, what = oracle_sample(p, 0.0)
        per_op_s.append(per_op)
    wall = time.perf_counter() - t0
    ops = normal_ops_per_recon(p)
    value = args.steps / (sum(per_op_s) * ops)
    nproc, model = host_cpu()
    return {
        "impl": "reference", "metric": metric_name(p), "value": value, "unit": "recon/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_name(p)},
        "extrapolated": True,
        "timed": f"{args.steps} steps, each one FP64 normal operator ({what}); a reconstruction is {ops} of them, "
                 f"so value = steps / (sum of operator times x {ops})",
        "cpu_baseline": {"value": value, "unit": "recon/s", "cores": threads, "kind": "oracle", "nproc": nproc,
                         "cpu_model": model,
                         "sample": f"each step: {what}, scaled by {ops} operators per reconstruction"},
        "e2e": {"value": value, "unit": "recon/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--workload", default="n128",
                    choices=["n128", "n256", "paper128x64", "paper1024x512", "batch64", "serve"],
                    help="n128: the single N=128 reconstruction (default); n256: the N=256, 32-coil "
                         "reconstruction; paper128x64 / paper1024x512: the paper's two shapes with its Table I "
                         "parameters and tolerance exits; batch64: 64 heterogeneous reconstructions in one "
                         "batched launch; serve: the serving loop under Poisson arrivals")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="single-reconstruction workloads: leave out the N=32, N=256 and serving sub-objects")
    ap.add_argument("--line-serve-requests", type=int, default=24,
                    help="requests of the serving sub-object of the default line")
    ap.add_argument("--batch-items", type=int, default=64)
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-inflight", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=float, default=32.0)
    ap.add_argument("--serve-rates", default="0.8",
                    help="comma list of arrival rates as multiples of the measured burst capacity")
    ap.add_argument("--serve-precisions", default="bf16x3",
                    help="comma list of forms to serve (bf16x3, tf32, fp32); the first is the headline")
    ap.add_argument("--serve-capacity-requests", type=int, default=64,
                    help="requests in the burst that measures capacity")
    ap.add_argument("--serve-sweep-requests", type=int, default=0,
                    help="requests per wave at the rates after the first (0: all)")
    ap.add_argument("--serve-fp32-requests", type=int, default=24,
                    help="requests per wave for the FP32 form (about 2 s per request)")
    ap.add_argument("--tiles", default="",
                    help="'C,F,A': coils per forward tile, forward stages and adjoint stages instead of "
                         "autotuning them")
    ap.add_argument("--forms", default="",
                    help="comma list of what to run: bf16x3 (always), e2e (host-buffer run), fp32 (plain FP32 "
                         "form), tf32 (TF32 tensor-core form); default all four for n128, all but fp32 for "
                         "n256 (whose FP32 form takes about half a minute per reconstruction)")
    args = ap.parse_args()
    if not args.forms:
        args.forms = "bf16x3,e2e,tf32" if args.workload in ("n256", "paper1024x512") else "bf16x3,e2e,fp32,tf32"
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank)
    elif args.workload == "batch64":
        line = run_batch(args, rank, world, local_rank)
    elif args.workload == "serve":
        line = run_serve(args, rank, world, local_rank)
    else:
        line = run_gpu(args, rank, world, local_rank)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
