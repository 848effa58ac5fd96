#!/usr/bin/env python
"""Benchmark: 128x128 Wiener-posterior samples/s on one GB300 (messenger-field Gibbs sampler, Alg. 1).

Workload (one "step"): the paper-shaped 128x128 problem (P ~ k^-2 with k0 = 1/32, noise variance
U[0.01, 1], 10% of the pixels missing in two rectangles plus scattered pixels), 1024 independent chains
x 100 posterior samples (thin 1, s0 = 0) in one call of the C ABI ``wf_sample_ex``. Inputs are seeded
synthetic data of that shape (``paper_1810_02821_gb300.synth.config_paper128``).

Printed JSON line (rank 0):
  value      samples/s with inputs resident in HBM (events around each step; L2 flushed between steps)
  e2e        same metric through the same C call with host buffers: pinned H2D of the inputs, and every
             sample stored by the kernel into page-locked host memory, inside the timed region
  roofline   the fused sampler kernel k_sample<128,1>: FFT flops (5 n log2 n per sweep) per launch over
             its event-timed duration, against the FP32 FMA throughput measured on the device
             (wf_measure_fp32_peak: every SM filled with independent FMA chains, CUDA events, best launch)
  cpu_baseline  the FP64 oracle on the host cores, on a bounded sample of the same workload
  batched_vs_plain  the 1024-chain launch against one chain per launch
  batch_mixed_sizes 4096 images of mixed sizes (40% 64^2, 40% 128^2, 15% 256^2, 5% 512^2), each a Wiener
             solve to 1e-5 plus 64 samples, as one CUDA-graph replay with autotuned launch shapes, against
             one image per call
  plain_32x32, precision_1024x1024, differentiation_256x256
             the other workloads: the 32x32 plain case, the 1024x1024 solve to FP64 residual 1e-7, and
             likelihood gradients / Wiener-map VJPs of 64 images of 256x256
  bf16_sample_storage, hierarchical_band_sampler, spin2_shear_sampler, large_image_sampler
             the headline workload with BF16 sample storage (kernel and end-to-end rates), the sampler with
             band-power draws, the shear pair, and the 256x256 / 512x512 samplers on thread-block clusters
             against the global-memory kernels

``--impl reference`` times the oracle itself (the reference arm for this build) and prints the same line.
Multi-GPU (torchrun): every rank runs the same workload on different chains (replicas, weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H = W = 128
N_CHAINS = 1024
N_SAMPLES = 100
METRIC = "128x128 Wiener-posterior samples/s (1 GB300)"
UNIT = "samples/s"
FLOPS_PER_SWEEP = 5.0 * H * W * math.log2(H * W)   # two real 2D FFTs at 2.5 n log2 n each
FP32_LANES = 128   # FP32 FMA lanes per SM (for the derived figure shown beside the measured peak)
# FP32 roofline denominator: measured on the device by wf_measure_fp32_peak before the extra workloads
# (set in main); the derived SMs x lanes x 2 x max clock figure is reported only as a note
FP32_PEAK_TFLOPS = None
WORKLOAD = "paper-shaped 128x128 image, 1024 independent chains x 100 posterior samples per step"
PROFILE = os.path.join(ROOT, "profiles", "k_sample_128_paper128.txt")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wf", choices=["wf", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the plain, single-chain and batch measurements")
    ap.add_argument("--no-batch", action="store_true", help="skip the mixed-size batch measurement")
    ap.add_argument("--large-path", choices=("auto", "cluster", "global"), default="auto",
                    help="256x256 / 512x512 kernels outside the large-image comparison: automatic (default), "
                         "thread-block clusters or the global-memory kernels")
    ap.add_argument("--large-chains", type=int, default=456,
                    help="chains of the 256x256 large-image sampler measurement (512x512: a third)")
    ap.add_argument("--large-samples", type=int, default=20,
                    help="samples per chain of the 256x256 measurement (512x512: half)")
    ap.add_argument("--extras", default="batch,plain,precision,grad,bf16,band,spin2,large",
                    help="extra workloads (comma list of batch, plain, precision, grad, bf16, band, spin2, large)")
    ap.add_argument("--batch-images", type=int, default=4096, help="images of the mixed-size batch")
    ap.add_argument("--precision-max-iter", type=int, default=400000,
                    help="profiling only: sweep cap of each solve of the 1024x1024 precision case")
    ap.add_argument("--batch-samples", type=int, default=64,
                    help="profiling only: samples per image of the mixed-size batch (0: Wiener solves only)")
    ap.add_argument("--batch-large-streams", type=int, default=8,
                    help="large-image chunks per size class of the untuned batch replay")
    ap.add_argument("--chains", type=int, default=N_CHAINS, help="profiling only: chains per step")
    ap.add_argument("--samples", type=int, default=N_SAMPLES, help="profiling only: samples per chain")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def replica_chain_offset(rank: int, chains: int) -> int:
    """Replicas only: rank r runs chains [r*chains, (r+1)*chains) (Philox chain words), no collective."""
    return rank * chains


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest of the ranks' values (timed-region length): every rank gets it (all-reduce MAX)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(units_per_rank: int, world: int, max_ms: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / (max_ms / 1e3)


# the sources k_sample<128,1> is compiled from (kernel, register FFT and RNG, launcher, translation unit)
SAMPLE_KERNEL_SOURCES = ("wf_math.cuh", "wf_gibbs.cuh", "wf_launch.h", "wf_k128.cu")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in SAMPLE_KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1810_02821_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of k_sample<128,1> from the committed ncu summary, if the kernel sources
    are unchanged since it was taken (its 'csrc_hash' line); else None."""
    if not os.path.exists(PROFILE):
        return None
    vals = {}
    for line in open(PROFILE):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("csrc_hash") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_workload"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts after the first sample: nvidia-smi's start-up (driver queries) can
            # otherwise delay the first timed launches by milliseconds
            t0 = time.time()
            while not self.lines and self.proc.poll() is None and time.time() - t0 < 5.0:
                time.sleep(0.01)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measure_fp32_peak(dev, local: int, target_ms: float = 7.0, reps: int = 5):
    """FP32 FMA throughput of this GPU: launches of the library's FMA-rate kernel (scalar FFMA and the
    paired FFMA2 form) sized to about the headline kernel's launch length, best of ``reps`` each, with the
    SM clock sampled meanwhile. Changes no device setting."""
    import torch
    from paper_1810_02821_gb300 import wf
    props = torch.cuda.get_device_properties(dev)
    out = {}
    with ClockSampler(local) as clk:
        for paired in (False, True):
            _, ms = wf.wf_measure_fp32_peak(paired, 4096)                 # warm-up and calibration
            iters = max(1024, int(4096 * target_ms / max(ms, 1e-3)))
            best = 0.0
            for _ in range(reps):
                tf, ms = wf.wf_measure_fp32_peak(paired, iters)
                best = max(best, tf)
            out["paired_tflops" if paired else "scalar_tflops"] = best
            out["paired_ms" if paired else "scalar_ms"] = ms
    c = clk.summary()
    sms = props.multi_processor_count
    mx = c.get("sm_max_mhz") or 2070.0
    out.update({"tflops": max(out["scalar_tflops"], out["paired_tflops"]), "sms": sms,
                "sm_mhz_median": c.get("sm_mhz"), "sm_max_mhz": c.get("sm_max_mhz"), "reasons": c.get("reasons"),
                "derived_tflops": sms * FP32_LANES * 2 * mx * 1e6 / 1e12,
                "how": f"wf_measure_fp32_peak: {sms} SMs x full occupancy x 256 threads x 16 independent FMA "
                       f"chains, scalar and paired forms, best of {reps} launches of ~{target_ms:.0f} ms each "
                       "(CUDA events)"})
    return out


def cpu_baseline(target_s: float = 12.0):
    """The FP64 oracle (as it stands) on the host cores, on a bounded sample of the same workload."""
    import numpy as np
    from oracle import messenger as M
    from paper_1810_02821_gb300 import synth
    p = synth.config_paper128(0)
    M.sample(p.d, p.Ndiag, p.mask, p.Pk, 1, seed=1)            # warm caches
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < target_s:
        M.sample(p.d, p.Ndiag, p.mask, p.Pk, 10, seed=1, chain=n)
        n += 10
    dt = time.perf_counter() - t0
    threads = os.cpu_count()
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            threads = max(i.get("num_threads", 1) for i in info)
    except Exception:
        pass
    return {"value": n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} sweeps (= samples) of one 128x128 chain of the same problem, {dt:.1f} s; "
                      f"host has {os.cpu_count()} cores"}


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import messenger as M
    from paper_1810_02821_gb300 import synth
    p = synth.config_paper128(0)
    per_step = 8   # samples per step: a bounded slice of the 1024 x 100 workload
    for i in range(a.warmup):
        M.sample(p.d, p.Ndiag, p.mask, p.Pk, per_step, seed=1, chain=i)
    t0 = time.perf_counter()
    for i in range(a.steps):
        M.sample(p.d, p.Ndiag, p.mask, p.Pk, per_step, seed=1, chain=1000 + i)
    dt = time.perf_counter() - t0
    v = per_step * a.steps / dt
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + f" (reference arm: {per_step} samples of one chain per step)",
                       "image": "128x128"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} sweeps of one 128x128 chain per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_mixed(dev, n_images: int = 4096, n_samples: int = 64, n_plain: int = 64, large_streams: int = 8):
    """Mixed-size batch: Wiener solve to 1e-5 plus n_samples samples per image, all images in one graph
    replay (launch shapes autotuned on the batch), against the same work one image per call."""
    import torch
    from paper_1810_02821_gb300 import synth, wf
    probs = synth.config_batch(n_images, seed=0)
    imgs = [wf.BatchImage(*[torch.from_numpy(x).to(dev) for x in (q.d, q.Ndiag, q.mask, q.Pk)], seed=i, chain=i)
            for i, q in enumerate(probs)]
    sizes = [q.d.shape[0] for q in probs]
    del probs
    stream = torch.cuda.current_stream()

    def replay_ms(g, reps=2):
        g.launch()
        g.results(allow_not_converged=True)                 # warm-up replay
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            g.launch(stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    with wf.BatchGraph(imgs, n_samples=n_samples, tol=1e-5, large_streams=large_streams) as g:
        default_ms = replay_ms(g)
    t_tune = time.perf_counter()
    tuned, _ = wf.wf_batch_autotune(imgs, n_samples=n_samples, reps=1, tol=1e-5)   # on the timed batch itself
    t_tune = time.perf_counter() - t_tune
    with wf.BatchGraph(imgs, n_samples=n_samples, tol=1e-5, **tuned) as g:
        ms = replay_ms(g)
        g.results(allow_not_converged=True)
    ok = sum(im.status == 0 for im in imgs)
    flops = sum((im.iters + n_samples) * 5.0 * h * h * math.log2(h * h) for im, h in zip(imgs, sizes))
    pix = sum(h * h for h in sizes)
    # the same work one image per call: Wiener solve, then the samples from it
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(n_plain):
        im = imgs[i]
        # the batch's own solve: the plain FP32 iteration to 1e-5 (no FP64 refinement)
        r = wf.wf_solve_ex(im.d, im.Ndiag, im.mask, im.Pk, tol=1e-5, refine=0, allow_not_converged=True)
        if n_samples > 0:
            wf.wf_sample_ex(im.d, im.Ndiag, im.mask, im.Pk, seed=i, n_samples=n_samples, chain_offset=i,
                            init_s=r.s, out=im.out_samples.unsqueeze(0))
    torch.cuda.synchronize()
    plain_ms_per_image = (time.perf_counter() - t0) * 1e3 / n_plain
    plain_pix = sum(sizes[:n_plain])
    counts = {f"{h}x{h}": sizes.count(h) for h in sorted(set(sizes))}
    achieved = flops / (ms / 1e3) / 1e12
    return {
        "workload": f"{n_images} images {counts}, Wiener solve to 1e-5 + {n_samples} samples each, one graph replay",
        "ms": ms, "images_per_s": n_images / (ms / 1e3), "samples_per_s": n_images * n_samples / (ms / 1e3),
        "pixel_samples_per_s": pix * n_samples / (ms / 1e3), "solves_ok": ok,
        "mean_solve_sweeps": statistics.mean(im.iters for im in imgs),
        "untuned_ms": default_ms, "tuned_launch_shape": tuned, "autotune_s": t_tune,
        "plain_one_image_per_call_ms_per_image": plain_ms_per_image,
        "speedup_vs_plain": plain_ms_per_image * n_images / ms,
        "plain_sample_note": f"first {n_plain} images (mixed sizes) timed one call each, scaled to the batch",
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS,
                     "flops": flops, "flops_note": "5 n log2 n per solve or sample sweep (level norms excluded)"},
        "output_bytes": pix * n_samples * 4, "plain_pixels_timed": plain_pix,
    }


def plain_32(dev):
    """32x32 plain-method case: Wiener solve to 1e-6, then 1000 samples of one chain from s0 = 0."""
    import torch
    from paper_1810_02821_gb300 import synth, wf
    p = synth.config_plain32(0)
    d, Nd, mk, Pk = [torch.from_numpy(x).to(dev) for x in (p.d, p.Ndiag, p.mask, p.Pk)]
    wf.wf_solve_ex(d, Nd, mk, Pk, tol=1e-6)
    wf.wf_sample_ex(d, Nd, mk, Pk, seed=0, n_samples=1000)
    stream = torch.cuda.current_stream()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    r = wf.wf_solve_ex(d, Nd, mk, Pk, tol=1e-6)
    e1.record(stream)
    wf.wf_sample_ex(d, Nd, mk, Pk, seed=0, n_samples=1000)
    e2.record(stream)
    e2.synchronize()
    return {"workload": "32x32, Wiener solve to 1e-6 then 1000 samples of one chain",
            "solve_ms": e0.elapsed_time(e1), "solve_sweeps": r.iters,
            "gibbs_steps_per_s_one_chain": 1000 / (e1.elapsed_time(e2) / 1e3)}


def precision_1024(dev, max_iter: int = 400000):
    """1024x1024 precision case: Wiener solve to FP64 relative residual 1e-7 (iterative refinement).
    max_iter below the default (profiling only) caps the sweeps of each solve, so the result is then not
    converged."""
    import torch
    from paper_1810_02821_gb300 import synth, wf
    p = synth.config_precision(1024, seed=0)
    d, Nd, mk, Pk = [torch.from_numpy(x).to(dev) for x in (p.d, p.Ndiag, p.mask, p.Pk)]
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = wf.wf_solve_ex(d, Nd, mk, Pk, tol=1e-7, refine=8, refine_tol=1e-3, max_iter=max_iter,
                       allow_not_converged=max_iter < 400000)
    e1.record(stream)
    e1.synchronize()
    return {"workload": "1024x1024, P ~ k^-1.5, noise variance U[0.001, 0.1], 25% in 200 circular holes; "
                        "Wiener solve to FP64 relative residual 1e-7",
            "time_to_solution_s": e0.elapsed_time(e1) / 1e3, "sweeps": r.iters, "fp64_resid": r.resid,
            "status": r.status}


def differentiation_256(dev, n_images: int = 64, n_probes: int = 8):
    """64 images of 256x256 with P = A (k/k0)^n, N = alpha sigma2: log-likelihood gradient (quadratic term,
    one solve; trace term, n_probes solves) and the Wiener-map VJP (one adjoint solve) per image."""
    import numpy as np
    import torch
    from paper_1810_02821_gb300 import synth, wf
    rng = np.random.default_rng(0)
    H = 256
    imgs = []
    for i in range(n_images):
        amp, slope = float(rng.uniform(0.5, 2.0)), float(rng.uniform(-2.5, -1.5))
        q = synth.make_problem(H, seed=1000 + i, amp=amp, slope=slope, k0=1.0 / H, sigma2=(0.01, 0.2),
                               mask_frac=0.1)
        imgs.append((amp, slope, [torch.from_numpy(x).to(dev) for x in (q.d, q.Ndiag, q.mask)]))
    g = torch.randn((H, H), device=dev)
    wf.wf_loglike_grad(*imgs[0][2], imgs[0][0], imgs[0][1], 1.0 / H, 1.0, n_probes=1, tol=1e-6)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for amp, slope, (d, s2, mk) in imgs:
        wf.wf_loglike_grad(d, s2, mk, amp, slope, 1.0 / H, 1.0, n_probes=n_probes, tol=1e-6)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for amp, slope, (d, s2, mk) in imgs:
        s, _ = wf.wf_wiener_vjp(d, s2, mk, amp, slope, 1.0 / H, 1.0, tol=1e-6)
        wf.wf_wiener_vjp(d, s2, mk, amp, slope, 1.0 / H, 1.0, g, s_w=s, tol=1e-6)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    batch = [(d, s2, mk, amp, slope, 1.0 / H, 1.0, i) for i, (amp, slope, (d, s2, mk)) in enumerate(imgs)]
    wf.wf_loglike_grad_batch(batch[:2], n_probes=n_probes, tol=1e-6)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    wf.wf_loglike_grad_batch(batch, n_probes=n_probes, tol=1e-6)
    torch.cuda.synchronize()
    t4 = time.perf_counter()
    return {"workload": f"{n_images} images 256x256, gradient of lnL in (A, n, alpha) with {n_probes} probes, "
                        "and the Wiener-map VJP, one image per call; the gradient also batched",
            "loglike_grad_batched_images_per_s": n_images / (t4 - t3),
            "loglike_grad_batched_solves_per_s": n_images * (1 + n_probes) / (t4 - t3),
            "loglike_grad_images_per_s": n_images / (t1 - t0),
            "loglike_grad_solves_per_s": n_images * (1 + n_probes) / (t1 - t0),
            "vjp_images_per_s": n_images / (t2 - t1), "vjp_solves_per_s": 2 * n_images / (t2 - t1)}


def reduced_output(dev, steps: int = 3):
    """The headline workload with samples stored as BF16 (chain in FP32, each sample rounded once): kernel
    throughput and end-to-end throughput with half the device-to-host bytes."""
    import torch
    from paper_1810_02821_gb300 import synth, wf
    p = synth.config_paper128(0)
    host = [torch.from_numpy(x).pin_memory() for x in (p.d, p.Ndiag, p.mask, p.Pk)]
    d, Nd, mk, Pk = [x.to(dev) for x in host]
    dout = torch.empty((N_CHAINS, N_SAMPLES, H, W), dtype=torch.bfloat16, device=dev)
    hout = torch.empty(dout.shape, dtype=torch.bfloat16, pin_memory=True)
    hout.zero_()  # untimed first touch of the pinned pages
    stream = torch.cuda.current_stream()
    wf.wf_sample_ex(d, Nd, mk, Pk, seed=1, n_samples=N_SAMPLES, n_chains=N_CHAINS, out=dout, out_dtype="bf16")
    ks = []
    for i in range(steps):
        wf.wf_sample_ex(d, Nd, mk, Pk, seed=2 + i, n_samples=N_SAMPLES, n_chains=N_CHAINS, out=dout,
                        out_dtype="bf16")
        ks.append(wf.wf_last_kernel_ms())
    del dout
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):  # inputs from pinned host memory, samples written into pinned host memory
        dd, nn, mm, pp = [x.to(dev, non_blocking=True) for x in host]
        wf.wf_sample_ex(dd, nn, mm, pp, seed=50 + i, n_samples=N_SAMPLES, n_chains=N_CHAINS, out=hout,
                        out_dtype="bf16")
    e1.record(stream)
    e1.synchronize()
    kms = statistics.mean(ks)
    return {"workload": "paper-shaped 128x128, 1024 chains x 100 samples, samples stored as BF16",
            "kernel_samples_per_s": N_CHAINS * N_SAMPLES / (kms / 1e3), "kernel_ms": kms,
            "e2e_samples_per_s": N_CHAINS * N_SAMPLES * steps / (e0.elapsed_time(e1) / 1e3),
            "d2h_bytes_per_step": hout.numel() * 2}


def band_sampler(dev):
    """Hierarchical Gibbs sampler on the headline workload: 1024 chains x 100 sweeps of the paper-shaped
    128x128 problem with the power spectrum drawn in integer-radius bands every sweep."""
    import numpy as np
    import torch
    from paper_1810_02821_gb300 import synth, wf
    p = synth.config_paper128(0)
    d, Nd, mk, Pk = [torch.from_numpy(x).to(dev) for x in (p.d, p.Ndiag, p.mask, p.Pk)]
    ky = np.fft.fftfreq(H) * H
    r = np.sqrt(ky[:, None] ** 2 + np.arange(W // 2 + 1)[None, :] ** 2)
    bins = np.floor(r).astype(np.int32) - 1
    bins[0, 0] = -1
    nb = int(bins.max()) + 1
    bt = torch.from_numpy(bins).to(dev)
    P0 = torch.ones(nb, device=dev)
    wf.wf_sample_band(d, Nd, mk, Pk, bt, P0, seed=1, n_samples=N_SAMPLES, n_chains=N_CHAINS)
    ks = []
    for i in range(3):
        wf.wf_sample_band(d, Nd, mk, Pk, bt, P0, seed=2 + i, n_samples=N_SAMPLES, n_chains=N_CHAINS)
        ks.append(wf.wf_last_kernel_ms())
    kms = statistics.mean(ks)
    res = {"workload": f"paper-shaped 128x128, 1024 chains x 100 sweeps, {nb} radial band powers drawn each sweep",
           "samples_per_s": N_CHAINS * N_SAMPLES / (kms / 1e3), "kernel_ms": kms,
           "n_bins": nb}
    # 256^2 and 512^2: one thread-block cluster per chain
    for Hl, chains, ns in ((256, 456, 20), (512, 76, 10)):
        q = synth.make_problem(Hl, seed=Hl, mask_frac=0.1, slope=-2.0, k0=1.0 / 32, sigma2=(0.05, 0.5))
        args = [torch.from_numpy(x).to(dev) for x in (q.d, q.Ndiag, q.mask, q.Pk)]
        kyl = np.fft.fftfreq(Hl) * Hl
        rl = np.sqrt(kyl[:, None] ** 2 + np.arange(Hl // 2 + 1)[None, :] ** 2)
        bl = np.floor(rl).astype(np.int32) - 1
        bl[0, 0] = -1
        nbl = int(bl.max()) + 1
        btl, P0l = torch.from_numpy(bl).to(dev), torch.ones(nbl, device=dev)
        wf.wf_sample_band(*args, btl, P0l, seed=1, n_samples=ns, n_chains=chains)
        ks = []
        for i in range(3):
            wf.wf_sample_band(*args, btl, P0l, seed=2 + i, n_samples=ns, n_chains=chains)
            ks.append(wf.wf_last_kernel_ms())
        kl = statistics.mean(ks)
        res[f"{Hl}x{Hl}"] = {"workload": f"{Hl}x{Hl}, {chains} chains x {ns} sweeps (all kept), {nbl} radial band "
                                         "powers drawn each sweep, one thread-block cluster per chain",
                             "samples_per_s": chains * ns / (kl / 1e3), "kernel_ms": kl, "n_bins": nbl,
                             "roofline": _fft_roofline(Hl, chains * ns, kl)}
    return res


def _fft_roofline(H: int, sweeps: int, kernel_ms: float, fields: int = 1) -> dict:
    """ALU roofline of `sweeps` field sweeps of H x H (5 n log2 n flops each: the sweep's two real 2D
    transforms) against the measured FP32 FMA peak."""
    n = H * H
    achieved = 5.0 * n * math.log2(n) * fields * sweeps / (kernel_ms / 1e3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_TFLOPS}


def spin2_sampler(dev, n_chains: int = 512):
    """Spin-2 (shear) sampler: the paper-shaped 128x128 problem as one shear component and a second
    component of the same noise model, E spectrum as the headline's, B = 0.2 E; 512 chains x 100 sweeps."""
    import numpy as np
    import torch
    from paper_1810_02821_gb300 import synth, wf
    p = synth.config_paper128(0)
    rng = np.random.default_rng(1)
    d2 = np.where(p.mask == 1, 0.0, rng.standard_normal(p.d.shape)).astype(np.float32)
    N2 = rng.uniform(0.01, 1.0, p.d.shape).astype(np.float32)
    args = [torch.from_numpy(np.ascontiguousarray(x)).to(dev)
            for x in (p.d, d2, p.Ndiag, N2, p.mask, p.Pk, (0.2 * p.Pk).astype(np.float32))]
    wf.wf_sample_spin2(*args, seed=1, n_samples=N_SAMPLES, n_chains=n_chains)
    ks = []
    for i in range(3):
        wf.wf_sample_spin2(*args, seed=2 + i, n_samples=N_SAMPLES, n_chains=n_chains)
        ks.append(wf.wf_last_kernel_ms())
    kms = statistics.mean(ks)
    res = {"workload": f"128x128 shear pair, {n_chains} chains x 100 sweeps (4 real 2D FFTs per sweep)",
           "samples_per_s": n_chains * N_SAMPLES / (kms / 1e3), "kernel_ms": kms,
           "roofline": {"bound": "alu", "achieved": 2 * FLOPS_PER_SWEEP * n_chains * N_SAMPLES / (kms / 1e3) / 1e12,
                        "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": 2 * FLOPS_PER_SWEEP * n_chains * N_SAMPLES / (kms / 1e3) / 1e12 / FP32_PEAK_TFLOPS}}
    # 256^2 and 512^2: both components of a chain in one thread-block cluster
    for Hl, chains, ns in ((256, 228, 20), (512, 36, 10)):
        q = synth.make_problem(Hl, seed=Hl, mask_frac=0.1, slope=-2.0, k0=1.0 / 32, sigma2=(0.05, 0.5))
        d2l = np.where(q.mask == 1, 0.0, rng.standard_normal(q.d.shape)).astype(np.float32)
        N2l = rng.uniform(0.05, 0.5, q.d.shape).astype(np.float32)
        argl = [torch.from_numpy(np.ascontiguousarray(x)).to(dev)
                for x in (q.d, d2l, q.Ndiag, N2l, q.mask, q.Pk, (0.2 * q.Pk).astype(np.float32))]
        wf.wf_sample_spin2(*argl, seed=1, n_samples=ns, n_chains=chains)
        ks = []
        for i in range(3):
            wf.wf_sample_spin2(*argl, seed=2 + i, n_samples=ns, n_chains=chains)
            ks.append(wf.wf_last_kernel_ms())
        kl = statistics.mean(ks)
        res[f"{Hl}x{Hl}"] = {"workload": f"{Hl}x{Hl} shear pair, {chains} chains x {ns} sweeps (all kept), "
                                         "both components of a chain in one thread-block cluster",
                             "samples_per_s": chains * ns / (kl / 1e3), "kernel_ms": kl,
                             "roofline": _fft_roofline(Hl, chains * ns, kl, fields=2)}
    return res


def large_sampler(dev, chains256: int = 456, samples256: int = 20):
    """Samplers for 256x256 and 512x512 (one thread-block cluster per chain, field in distributed shared
    memory) against the global-memory sampler on the same problem: paper-like field model (slope -2,
    k0 = 1/32, noise variance U[0.05, 0.5], 10% masked); by default 456 chains x 20 samples (256^2) and
    152 chains x 10 samples (512^2), every sweep kept."""
    import torch
    from paper_1810_02821_gb300 import synth, wf
    res = {}
    for H, chains, ns in ((256, chains256, samples256), (512, max(1, chains256 // 3), max(1, samples256 // 2))):
        p = synth.make_problem(H, seed=H, mask_frac=0.1, slope=-2.0, k0=1.0 / 32, sigma2=(0.05, 0.5))
        args = [torch.from_numpy(x).to(dev) for x in (p.d, p.Ndiag, p.mask, p.Pk)]
        out = torch.empty((chains, ns, H, H), device=dev)
        row = {"workload": f"{H}x{H}, {chains} chains x {ns} samples"}
        for mode in ("cluster", "global"):
            prev = wf.wf_set_large_image_sampler(mode)
            try:
                wf.wf_sample_ex(*args, seed=1, n_samples=ns, n_chains=chains, out=out)
                ks = []
                for i in range(3):
                    wf.wf_sample_ex(*args, seed=2 + i, n_samples=ns, n_chains=chains, out=out)
                    ks.append(wf.wf_last_kernel_ms())
            finally:
                wf.wf_set_large_image_sampler(prev)
            kms = statistics.mean(ks)
            n = H * H
            flops = 5.0 * n * math.log2(n) * chains * ns
            row[mode] = {"kernel_ms": kms, "samples_per_s": chains * ns / (kms / 1e3),
                         "pixel_sweeps_per_s": chains * ns * n / (kms / 1e3),
                         "roofline": {"bound": "alu", "achieved": flops / (kms / 1e3) / 1e12,
                                      "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                                      "frac": flops / (kms / 1e3) / 1e12 / FP32_PEAK_TFLOPS}}
        row["cluster_vs_global"] = row["global"]["kernel_ms"] / row["cluster"]["kernel_ms"]
        res[f"{H}x{H}"] = row
        del out
    return res


def main():
    global N_CHAINS, N_SAMPLES, FP32_PEAK_TFLOPS
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    N_CHAINS, N_SAMPLES = a.chains, a.samples
    import torch
    from paper_1810_02821_gb300 import build, synth, wf
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    wf.load_library()
    wf.wf_set_kernel_timing(True)
    wf.wf_set_large_image_sampler(a.large_path)
    dev = torch.device("cuda", local)
    p = synth.config_paper128(0)
    host = [torch.from_numpy(x) for x in (p.d, p.Ndiag, p.mask, p.Pk)]
    d, Nd, mk, Pk = [x.to(dev) for x in host]
    out = torch.empty((N_CHAINS, N_SAMPLES, H, W), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    chain0 = replica_chain_offset(rank, N_CHAINS)

    def step(seed, o=out):
        return wf.wf_sample_ex(d, Nd, mk, Pk, seed=seed, n_samples=N_SAMPLES, n_chains=N_CHAINS,
                               chain_offset=chain0, out=o)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for i in range(a.warmup):
        step(1 + i)
    barrier()
    stream = torch.cuda.current_stream()
    step_ms, kern_ms = [], []
    with ClockSampler(local) as clk:
        barrier()
        for i in range(a.steps):
            flush.fill_(float(i))                         # evict L2 between timed steps (not timed)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(100 + i)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            kern_ms.append(wf.wf_last_kernel_ms())
        barrier()
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    value = aggregate_throughput(N_CHAINS * N_SAMPLES * a.steps, world, total_ms)
    fp32_peak = measure_fp32_peak(dev, local)
    FP32_PEAK_TFLOPS = fp32_peak["tflops"]

    # end to end through the same call with host buffers: each step copies its inputs from pinned host
    # memory to the device and the kernel stores its samples straight into a page-locked host buffer over
    # the CPU-GPU link (the call's mapped-host output form), so the step ends with all of its samples in
    # host memory; no device staging buffer, no separate copy.
    e2e = None
    if not a.no_e2e:
        hin = [x.pin_memory() for x in host]
        hout = torch.empty(out.shape, dtype=torch.float32, pin_memory=True)
        hout.zero_()  # untimed first touch of the pinned pages
        h2d = sum(x.numel() * x.element_size() for x in hin)
        d2h = hout.numel() * hout.element_size()
        e2e_steps = max(1, min(a.steps, 5))
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(e2e_steps):
            dd, nn, mm, pp = [x.to(dev, non_blocking=True) for x in hin]
            wf.wf_sample_ex(dd, nn, mm, pp, seed=500 + i, n_samples=N_SAMPLES, n_chains=N_CHAINS,
                            chain_offset=chain0, out=hout)
        e1.record(stream)
        e1.synchronize()
        ems = max_over_ranks(e0.elapsed_time(e1), world, dev)
        e2e = {"value": aggregate_throughput(N_CHAINS * N_SAMPLES * e2e_steps, world, ems), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_steps,
               "note": "inputs copied from pinned host memory each step; the kernel writes the samples into "
                       "page-locked host memory over the CPU-GPU link (mapped output), so the link's "
                       "device-to-host rate bounds this number"}
        del hout

    plain = single = None
    if a.no_extras:
        n_plain = 0
    # batched (one launch for all chains) against plain (one chain per launch)
    n_plain = 0 if a.no_extras else 16
    if n_plain:
        o1 = torch.empty((1, N_SAMPLES, H, W), dtype=torch.float32, device=dev)
        wf.wf_sample_ex(d, Nd, mk, Pk, seed=9, n_samples=N_SAMPLES, n_chains=1, out=o1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for c in range(n_plain):
            wf.wf_sample_ex(d, Nd, mk, Pk, seed=9, n_samples=N_SAMPLES, n_chains=1, chain_offset=chain0 + c,
                            out=o1)
        e1.record(stream)
        e1.synchronize()
        plain = n_plain * N_SAMPLES / (e0.elapsed_time(e1) / 1e3)

        # one long chain (every 10th of 10^4 sweeps kept): sweeps/s of a single chain
        ol = torch.empty((1, 1000, H, W), dtype=torch.float32, device=dev)
        e0.record(stream)
        wf.wf_sample_ex(d, Nd, mk, Pk, seed=3, n_samples=1000, n_chains=1, thin=10, out=ol)
        e1.record(stream)
        e1.synchronize()
        single = 1e4 / (e0.elapsed_time(e1) / 1e3)

    if rank != 0:
        return
    batch = None
    other = {}
    if not a.no_extras:
        del out
        torch.cuda.empty_cache()
        want = set(a.extras.split(","))
        jobs = [(k, name, fn) for k, name, fn in (
            ("batch", "batch_mixed_sizes",
             lambda dv: batch_mixed(dv, n_images=a.batch_images, n_samples=a.batch_samples,
                                    large_streams=a.batch_large_streams)),
            ("plain", "plain_32x32", plain_32),
            ("precision", "precision_1024x1024", lambda dv: precision_1024(dv, a.precision_max_iter)),
            ("grad", "differentiation_256x256", differentiation_256),
            ("bf16", "bf16_sample_storage", reduced_output),
            ("band", "hierarchical_band_sampler", band_sampler),
            ("spin2", "spin2_shear_sampler", spin2_sampler),
            ("large", "large_image_sampler",
             lambda dv: large_sampler(dv, a.large_chains, a.large_samples))) if k in want and not (k == "batch" and a.no_batch)]
        for _, name, fn in jobs:
            try:
                other[name] = fn(dev)
            except Exception as ex:  # reported, never fatal for the headline line
                other[name] = {"error": f"{type(ex).__name__}: {ex}"}
        batch = other.pop("batch_mixed_sizes", None)
    kms = statistics.mean(kern_ms)
    flops = FLOPS_PER_SWEEP * N_CHAINS * N_SAMPLES
    achieved = flops / (kms / 1e3) / 1e12
    traffic = profiled_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": total_ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "image": "128x128", "chains": N_CHAINS, "samples_per_chain": N_SAMPLES,
                   "thin": 1, "l2": "flushed between timed steps (256 MiB write outside the step events)",
                   "parallelism": f"replicas x{world}"},
        "gibbs_steps_per_s": value,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": traffic,
                     "kernel": "wf::k_sample<128,1>", "kernel_ms": kms,
                     "flops_per_launch": flops,
                     "peak_note": "of measured: FP32 FMA throughput of this GPU (fp32_peak); derived "
                                  f"{fp32_peak['sms']} SMs x {FP32_LANES} lanes x 2 x max clock = "
                                  f"{fp32_peak['derived_tflops']:.1f} TFLOP/s shown only as a note"},
        "fp32_peak": fp32_peak,
        "batched_vs_plain": ({"batched": value, "plain_one_chain_per_launch": plain, "speedup": value / plain,
                              "plain_chains_timed": n_plain} if plain else None),
        "single_chain_sweeps_per_s": single,
        "batch_mixed_sizes": batch,
        **other,
        "clocks": clk.summary(),
        "gpu_launches": 3 * a.steps,
    }
    if e2e:
        line["e2e"] = e2e
    if not a.no_cpu_baseline and world >= 1:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
