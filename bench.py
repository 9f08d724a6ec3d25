"""Benchmark of the modelling hot path: Gpt-updates/s and HBM roofline fraction.

Workload: forward modelling with density on a 512x512x256 model
(576x576x320 padded, 32-cell sponge, h = 12.5 m, dt = 1 ms, 4000 steps),
seeded layered velocity with Gaussian anomalies, Gardner density, one
Ricker 10 Hz shot and 256x256 receivers (every 2 cells at z = 4).  One
benchmark step is one mamute_model call: coefficient preparation, the 4000
fused time steps (stencil, sponge, source injection, receiver sampling) and
the seismogram transpose.  Inputs are resident in HBM before the timed
region and every array is larger than L2.

Prints one JSON line.  It also carries a "gradient" object: FWI gradient
shots/s of the 256^3 single-shot workload (2000 steps, automatic storage)
through mamute_gradient, with its own CUDA-event time, bandwidth over the
step loop and clocks (the headline value is the modelling number alone).
--impl reference times the FP64 oracle on the host cores instead (a bounded
sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpt-updates/s"
UNIT = "Gpt/s"



KERNEL_SOURCES = ["paper_2502_12350_gb300/csrc/stencil_impl.cuh",
                  "paper_2502_12350_gb300/csrc/stencil_fwd.cu",
                  "paper_2502_12350_gb300/csrc/stencil_pair.cu",
                  "paper_2502_12350_gb300/csrc/common.cuh"]
PML_SOURCES = KERNEL_SOURCES + ["paper_2502_12350_gb300/csrc/cpml.cu",
                                "paper_2502_12350_gb300/csrc/cpml.h"]


def kernel_source_hash(sources=KERNEL_SOURCES) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def kernel_traffic(w, kernel="step_kernel_forward", sources=KERNEL_SOURCES):
    """DRAM bytes per launch of the forward kernel from the committed ncu
    summary of this workload, or None if the kernel source changed since."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{w.name}.md")
    try:
        fields = {}
        with open(path) as f:
            for line in f:
                if ":" in line and line.startswith("- "):
                    k, v = line[2:].split(":", 1)
                    fields[k.strip()] = v.strip().strip("`")
        if fields.get("source_sha256") != kernel_source_hash(sources):
            return None
        return int(fields["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        loaded = [s for s in sm if mx and s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(nt=None, kind="model"):
    from paper_2502_12350_gb300 import synth
    if kind == "model_small":
        return synth.forward_small() if nt is None else synth.forward_small(nt=nt)
    if kind == "model_mid":  # 256x256x128 with density: arrays still larger than L2
        return synth.forward_density(nt=nt or 4000, nx=256, ny=256, nz=128)
    return synth.forward_density() if nt is None else synth.forward_density(nt=nt)


def cpu_model() -> str:
    """Host CPU model name (lscpu, else /proc/cpuinfo), for the baseline line."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_oracle_rate(w, steps_lo=2, steps_hi=6, repeats=1):
    """Oracle Gpt/s on the host cores: full grid, the difference of runs of
    steps_hi and steps_lo time steps (so that set-up cancels), median over
    `repeats` runs of steps_hi against one run of steps_lo."""
    from oracle import oracle
    og = oracle.make_grid(w.nx, w.ny, w.nz, w.border, w.h, w.dt, steps_hi)
    wav = w.wavelet[:steps_hi].astype(np.float64)

    def run(ns):
        og.nt = ns
        t0 = time.perf_counter()
        oracle.model(og, w.vel, w.src_xyz, wav[:ns], w.rec_offset, w.rec_xyz, rho=w.rho)
        return time.perf_counter() - t0

    t_lo = run(steps_lo)
    rates, total = [], t_lo
    for _ in range(repeats):
        t_hi = run(steps_hi)
        total += t_hi
        rates.append(w.n_padded * (steps_hi - steps_lo) / max(t_hi - t_lo, 1e-9) / 1e9)
    rate = statistics.median(rates)
    cores = os.cpu_count()
    sample = (f"{steps_hi - steps_lo} time steps of the full {w.padded[2]}x{w.padded[1]}x"
              f"{w.padded[0]} padded grid (a {steps_hi}-step FP64 oracle run minus a "
              f"{steps_lo}-step one, median of {repeats}), OpenMP over z planes on "
              f"{cores} cores of {cpu_model()}")
    return rate, cores, sample, total


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = workload(nt=8)
    rates = []
    for _ in range(args.warmup):
        cpu_oracle_rate(w, 1, 2)
    for _ in range(args.steps):
        r, cores, sample, _ = cpu_oracle_rate(w, 1, 3)
        rates.append(r)
    v = statistics.median(rates)
    # one step of the metric is the whole 4000-step modelling call; its time
    # is extrapolated from the sample's rate
    ms_full = w.n_padded * 4000 / (v * 1e9) * 1e3 if v > 0 else None
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_full, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "forward_512x512x256_density_4000steps",
                       "padded": [576, 576, 320], "nt": 4000,
                       "ms_per_step": "extrapolated from the sample's rate"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


GRAD_FWD_BYTES = (16, 4)  # per padded point (u^n, u^{n-1}, A, new level), per interior point (term store)
GRAD_ADJ_BYTES = (24, 4)  # per padded point (psi levels, A, accumulator read + write), per interior point (term read)
# CPML gradient, per (point, axis) pair of a layer: forward Psi_a, Zeta_a read and
# written; reverse their multipliers read and written and the scratch y_a, z_a
# written and read
PML_GRAD_PAIR_BYTES = (16, 32)


def gradient_metrics(workload, steps, warmup, autotune=False, snapshots=0, nt=None, pml=False):
    """FWI gradient throughput through mamute_gradient on one GPU: shots/s,
    Gpt-updates/s of forward + adjoint work, CUDA-event time on the library's
    stream, and the step loop's bandwidth against the algorithmic bytes of
    the all-terms mode (each forward step reads u^n, u^{n-1}, A and writes
    the new level, 16 B per padded point, and stores the imaging term, 4 B
    per interior point; each adjoint step reads two psi levels and A, writes
    the new level, reads and writes the accumulator, 24 B per padded point,
    and reads the stored term, 4 B per interior point).  With pml, the
    convolutional PML instead of the sponge (every imaging term kept), plus
    PML_GRAD_PAIR_BYTES per (point, axis) pair of the layers."""
    import ctypes

    import torch

    from paper_2502_12350_gb300 import build, mamute, synth
    build.build()
    dev = torch.device("cuda", 0)
    if workload == "gradient_single":
        w = synth.gradient_single() if nt is None else synth.gradient_single(nt=nt)
    else:
        w = synth.batched_shots() if nt is None else synth.batched_shots(nt=nt)
    g = mamute.grid_of(w, cerjan=0.0, pml=1) if pml else mamute.grid_of(w)
    stream = torch.cuda.current_stream(dev)
    ctx = mamute.Context(0, stream.cuda_stream)
    lib = mamute.load()
    lib.mamute_ctx_set_timing.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.mamute_ctx_last_timing.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_longlong),
                                           ctypes.POINTER(ctypes.c_longlong)]
    lib.mamute_ctx_set_timing(ctx._h, 1)
    vtrue = torch.from_numpy(w.vel).to(dev)
    vinit = torch.from_numpy(w.vel_init).to(dev)
    n_rec = int(w.rec_offset[-1])
    dobs = torch.empty((n_rec, w.nt), device=dev)
    ctx.model(g, vtrue, None, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, dobs,
              aperture=w.aperture)
    grad = torch.empty_like(vinit)

    tiles = None
    if autotune:  # measured adjoint decomposition (outside the timed region)
        from paper_2502_12350_gb300 import autotune as at
        # tune with the storage mode the full run takes: every term kept for
        # the single shot (134 GB fits), checkpointing for the 64-shot batch
        ns = snapshots if snapshots != 0 else (-1 if workload == "gradient_single" else 16)
        tiles = at.tune_gradient(ctx, g, vinit, None, w.src_xyz, w.wavelet, w.rec_offset,
                                 w.rec_xyz, dobs, aperture=w.aperture, n_snapshots=ns)

    def step():
        return ctx.gradient(g, vinit, None, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, dobs,
                            grad, aperture=w.aperture, n_snapshots=snapshots, tiles=tiles)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches, steps_per_call, loop_ms = 0, 0, []
    with ClockSampler(0) as clk:
        ev0.record(stream)
        for _ in range(steps):
            J = step()
            lm, sl, tl = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_longlong()
            lib.mamute_ctx_last_timing(ctx._h, ctypes.byref(lm), ctypes.byref(sl), ctypes.byref(tl))
            launches += tl.value
            steps_per_call = sl.value
            loop_ms.append(lm.value)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    if w.aperture is not None:
        pts_shot = [int(a[1] - a[0] + 2 * w.border) * int(a[3] - a[2] + 2 * w.border) *
                    int(w.nz + 2 * w.border) for a in w.aperture]
        int_shot = [int(a[1] - a[0]) * int(a[3] - a[2]) * int(w.nz) for a in w.aperture]
    else:
        pts_shot = [int(w.n_padded)] * w.n_src
        int_shot = [int(w.nx * w.ny * w.nz)] * w.n_src
    all_terms = steps_per_call == 2 * w.nt  # one forward and one adjoint launch per step
    out = {"value": w.n_src / (ms / 1e3), "unit": "shots/s", "ms_per_gradient": ms,
           "workload": w.name, "shots": w.n_src, "nt": w.nt,
           "points_per_step": int(sum(pts_shot)), "snapshots": snapshots,
           "storage": "all imaging terms" if all_terms else "revolve checkpoints",
           "tiles": tiles if tiles is not None else "cost model",
           "step_launches_per_gradient": steps_per_call,
           "gpt_updates_per_s": sum(pts_shot) * steps_per_call / (ms / 1e3) / 1e9,
           "misfit": J, "gpu_launches": int(launches), "clocks": clk.summary()}
    if all_terms:
        peak, peak_kind = _peaks()
        byts = w.nt * sum(GRAD_FWD_BYTES[0] * p + GRAD_FWD_BYTES[1] * q +
                          GRAD_ADJ_BYTES[0] * p + GRAD_ADJ_BYTES[1] * q
                          for p, q in zip(pts_shot, int_shot))
        if pml:
            Nx, Ny, Nz = w.nx + 2 * w.border, w.ny + 2 * w.border, w.nz + 2 * w.border
            pairs = 2 * w.border * (Ny * Nz + Nx * Nz + Nx * Ny) * w.n_src
            byts += w.nt * sum(PML_GRAD_PAIR_BYTES) * pairs
        lms = statistics.median(loop_ms)
        ach = byts / (lms / 1e3) / 1e9
        out["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                           "frac": ach / peak, "traffic": None, "peak_kind": peak_kind,
                           "kernel": "step_kernel<forward+store> and step_kernel<adjoint, stored term>" +
                                     (" with the per-axis CPML kernels" if pml else ""),
                           "algorithmic_bytes_per_gradient": byts, "loop_ms": lms,
                           "bytes_per_point": {"forward": list(GRAD_FWD_BYTES),
                                               "adjoint": list(GRAD_ADJ_BYTES)}}
    ctx.close()
    return out


def run_gradient_bench(args):
    """FWI gradient throughput (shots/s and Gpt-updates/s of forward + adjoint
    work) through mamute_gradient, on one GPU."""
    gm = gradient_metrics(args.workload, args.steps, args.warmup, args.autotune, args.snapshots,
                          args.nt, pml=args.boundary == "pml")
    line = {"metric": "FWI gradient shots/s", "value": gm["value"], "unit": "shots/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": gm["ms_per_gradient"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict({k: gm[k] for k in ("workload", "shots", "nt", "points_per_step",
                                               "snapshots", "storage", "tiles",
                                               "step_launches_per_gradient")},
                           boundary="convolutional PML" if args.boundary == "pml" else "sponge"),
            "gpt_updates_per_s": gm["gpt_updates_per_s"], "misfit": gm["misfit"],
            "gpu_launches": gm["gpu_launches"], "clocks": gm["clocks"]}
    if "roofline" in gm:
        line["roofline"] = gm["roofline"]
    print(json.dumps(line), flush=True)
    return 0


def run_cnn_bench(args):
    """Training step of the preconditioner network (4 convolutions forward,
    3 input gradients, 4 weight gradients, loss, Adam) on the 160x160x80
    volume; FLOPs count the channel-padded (16 x 16) products."""
    import torch

    from paper_2502_12350_gb300 import build, cnn, mamute
    build.build()
    dev = torch.device("cuda", 0)
    ctx = mamute.Context(0)
    D, H, W = 80, 160, 160
    net = cnn.Net(ctx, seed=0)
    rng = np.random.default_rng(0)
    x = np.zeros((D, H, W, 16), np.float32)
    x[..., :2] = rng.standard_normal((D, H, W, 2))
    bits = (x.view(np.uint32) >> 16).astype(np.uint16).view(np.int16)
    xt = torch.from_numpy(bits).to(dev)
    tt = torch.from_numpy(rng.standard_normal((D, H, W)).astype(np.float32)).to(dev)
    for _ in range(args.warmup):
        net.train_step(xt, tt)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    ev0.record(stream)
    for _ in range(args.steps):
        net.train_step(xt, tt)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    flops = 11 * 2.0 * 27 * 16 * 16 * D * H * W  # 4 fwd + 3 dgrad + 4 wgrad convolutions
    # The dominant kernel alone: one 16 -> 16 forward convolution (layer 2),
    # CUDA events on the stream the library launches on, averaged over 20 calls.
    h = net.acts[1]
    conv_args = (ctx._h, D, H, W, cnn._p(h), cnn._p(net.wf[1]), cnn._p(net.b[1]), 1, None, None,
                 cnn._p(net.acts[2]))
    for _ in range(3):
        net.lib.mamute_conv3d(*conv_args)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(20):
        net.lib.mamute_conv3d(*conv_args)
    ev1.record(stream)
    torch.cuda.synchronize()
    conv_ms = ev0.elapsed_time(ev1) / 20
    peak = 1913.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["bf16_tflops"])
    except Exception:
        pass
    tf = flops / (ms / 1e3) / 1e12
    conv_tf = 2.0 * 27 * 16 * 16 * D * H * W / (conv_ms / 1e3) / 1e12
    line = {"metric": "network training step TFLOP/s", "value": tf, "unit": "TFLOP/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic", "config": {"workload": "cnn_4x3^3_16ch_80x160x160"},
            "roofline": {"bound": "tensor", "achieved": conv_tf, "peak": peak, "unit": "TFLOP/s",
                         "frac": conv_tf / peak, "traffic": None, "peak_kind": "measured",
                         "kernel": "conv_tc_kernel (16 -> 16, 3x3x3, tcgen05)",
                         "flops_per_voxel": 2 * 27 * 16 * 16, "kernel_ms": conv_ms,
                         "training_step_tflops": tf}}
    ctx.close()
    print(json.dumps(line), flush=True)
    return 0


def run_postproc_bench(args):
    """Gradient smoothing and data time resampling (mamute_smooth,
    mamute_resample) on one GPU: CUDA-event time per API call, inputs resident
    on the device.  Smoothing: Bessel and Laplace filters of the 600x600x200
    gradient of the 64-shot workload, a forward and an inverse dense DCT-II
    pass per axis of 2 n_a flops per point (FP32 ALU bound: 152 SMs x 128
    lanes x 2 flops x 2.07 GHz).  Resampling: sinc, 65,536 traces of 4000
    samples to 1000 (the headline's receivers), every input sample read and
    every output sample written once; the host builds the CSR matrix inside
    each call."""
    import torch

    from paper_2502_12350_gb300 import build, mamute
    build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = mamute.Context(0, stream.cuda_stream)
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)

    def per_call_ms(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    nx, ny, nz, h = 600, 600, 200, 10.0
    grad = torch.randn((nz, ny, nx), device=dev, generator=gen)  # 288 MB: larger than L2
    out = torch.empty_like(grad)
    alu_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    flops = 2 * 2 * (nx + ny + nz) * nx * ny * nz
    smooth = {}
    for mode, name in ((mamute.SMOOTH_BESSEL, "bessel"), (mamute.SMOOTH_LAPLACE, "laplace")):
        ms = per_call_ms(lambda: ctx.smooth(h, mode, grad, out, lengths=[4 * h] * 3))
        tf = flops / (ms / 1e3) / 1e12
        smooth[name] = {"ms": ms, "tflops": tf, "frac_fp32_alu": tf / alu_peak}
    ntr, nt_in, nt_out, dt_in = 65536, 4000, 1000, 5e-4
    x = torch.randn((ntr, nt_in), device=dev, generator=gen)
    y = torch.empty((ntr, nt_out), device=dev)
    ms_r = per_call_ms(lambda: ctx.resample(x, dt_in, nt_out, 4 * dt_in, mamute.INTERP_SINC, y))
    ms_t = per_call_ms(lambda: ctx.resample(y, dt_in, nt_out, 4 * dt_in, mamute.INTERP_SINC, x,
                                            adjoint=True))
    peak, peak_kind = _peaks()
    byts = 4 * ntr * (nt_in + nt_out)
    line = {"metric": "gradient smoothing ms (Bessel, 600x600x200)", "value": smooth["bessel"]["ms"],
            "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
            "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "postproc", "gradient": [nx, ny, nz], "h": h,
                       "lengths": [4 * h] * 3, "traces": ntr, "nt_in": nt_in, "nt_out": nt_out,
                       "l2": "inputs larger than L2 (288 MB gradient, 1.3 GB of traces)"},
            "smoothing": dict(smooth, bound="fp32 alu", peak_tflops=alu_peak,
                              flops_per_call=flops),
            "resampling": {"ms": ms_r, "ms_transpose": ms_t, "bytes_per_call": byts,
                           "achieved_gbs": byts / (ms_r / 1e3) / 1e9,
                           "frac": byts / (ms_r / 1e3) / 1e9 / peak, "peak": peak,
                           "peak_kind": peak_kind}}
    ctx.close()
    print(json.dumps(line), flush=True)
    return 0


def run_gn_bench(args):
    """Exact Gauss-Newton-diagonal labels of the 160x160x80 learned-
    preconditioner workload (12 shots, 64 receivers, 1500 steps)."""
    import time as _t

    import torch

    from paper_2502_12350_gb300 import build, mamute, synth
    build.build()
    dev = torch.device("cuda", 0)
    ctx = mamute.Context(0)
    import ctypes
    w = synth.fwi_small(model_id=5000) if args.nt is None else synth.fwi_small(model_id=5000, nt=args.nt)
    g = mamute.grid_of(w)
    v = torch.from_numpy(w.vel).to(dev)
    hd = torch.empty_like(v)
    lib = mamute.load()
    lib.mamute_ctx_set_timing.argtypes = [ctypes.c_void_p, ctypes.c_int]
    D, LL = ctypes.c_double, ctypes.c_longlong
    lib.mamute_ctx_dft_timing.argtypes = [ctypes.c_void_p, ctypes.POINTER(D), ctypes.POINTER(LL),
                                          ctypes.POINTER(D)]
    lib.mamute_ctx_set_timing(ctx._h, 1)
    for _ in range(args.warmup):
        ctx.gn_diagonal(g, v, None, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, hd)
    torch.cuda.synchronize()
    dft_ms, dft_n, macs = 0.0, 0, 0.0
    with ClockSampler(0) as clk:
        t0 = _t.perf_counter()
        for _ in range(args.steps):
            ctx.gn_diagonal(g, v, None, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, hd)
            ms, n, m = D(), LL(), D()
            lib.mamute_ctx_dft_timing(ctx._h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(m))
            dft_ms, dft_n, macs = dft_ms + ms.value, dft_n + n.value, macs + m.value
        torch.cuda.synchronize()
        sec = (_t.perf_counter() - t0) / args.steps
    props = w.n_src + int(w.rec_offset[1])
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        peaks = json.load(f)
    # The DFT runs on the tensor cores (kind::tf32, hi / lo split: three
    # products per pair) when the point count is a multiple of 4, else on the
    # FP32 ALUs.  Useful work: 4 flops per (point, sample, bin); executed
    # contraction: 3 products x 2 flops x 2 rows (cos, sin) per bin.
    tensor = (w.nx * w.ny * w.nz) % 4 == 0
    useful = 4.0 * macs / (dft_ms * 1e-3) / 1e12 if dft_ms > 0 else None
    if tensor:
        # dense tf32 peak: the measured bf16 figure (sustained: the DFT runs
        # inside a seconds-long label computation) x the nominal 1.1 / 2.25
        peak = peaks.get("bf16_tflops_sustained", 1712.9) * 1.1 / 2.25
        achieved = 12.0 * macs / (dft_ms * 1e-3) / 1e12 if dft_ms > 0 else None
        rl = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
              "frac": achieved / peak if achieved else None, "traffic": None,
              "peak_kind": "measured bf16 sustained x nominal tf32/bf16 ratio 1.1/2.25",
              "kernel": "dft_tc_kernel (tcgen05 kind::tf32, 3 products)",
              "flops_per_unit": 12, "useful_tflops": useful,
              "unit_of_work": "point x sample x bin"}
    else:
        # FP32 ALU peak: 152 SMs x 128 FP32 lanes x 2 flops per FMA x max SM clock
        alu_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        rl = {"bound": "alu", "achieved": useful, "peak": alu_peak, "unit": "TFLOP/s",
              "frac": useful / alu_peak if useful else None, "traffic": None,
              "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x sm_max_mhz",
              "kernel": "dft_kernel (with twiddles)", "flops_per_unit": 4,
              "unit_of_work": "point x sample x bin"}
    line = {"metric": "GN-diagonal labels/s", "value": 1.0 / sec, "unit": "models/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "nt": w.nt, "propagations": props,
                       "gpt_updates_per_s": props * w.n_padded * w.nt / sec / 1e9},
            "roofline": dict(rl, dft_share_of_step=dft_ms / args.steps / (sec * 1e3),
                             dft_launches_per_step=dft_n // max(args.steps, 1)),
            "clocks": clk.summary()}
    ctx.close()
    print(json.dumps(line), flush=True)
    return 0


def pml_bytes_per_step(w):
    """Algorithmic DRAM bytes of one CPML time step: u^n, u^{n-1}, A (and
    A m2) read and u^{n+1} written at every padded point, plus the two memory
    variables of each axis read and written at the points in that axis's
    layer."""
    Nx, Ny, Nz = w.nx + 2 * w.border, w.ny + 2 * w.border, w.nz + 2 * w.border
    base = (20 if w.rho is not None else 16) * Nx * Ny * Nz
    layer = 2 * w.border * (Ny * Nz + Nx * Nz + Nx * Ny)  # (point, axis) pairs in a layer
    return base + 16 * layer


def pml_line(args, w, world, total_ms, value, e2e, vel_h, rho_h, seis_h, launches, step_ms, peak,
             peak_kind, clocks):
    alg = pml_bytes_per_step(w)
    achieved = alg / (step_ms / 1e3) / 1e9
    n_rec = int(w.rec_offset[-1])
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name + f"_{w.nt}steps_cpml", "boundary": "convolutional PML",
                   "padded": list(w.padded)[::-1], "nt": w.nt, "shots": 1, "receivers": n_rec,
                   "l2": "every array (%d MB) is larger than L2" % (w.n_padded * 4 // 2**20),
                   "parallelism": "replicas" if world > 1 else "single"},
        "e2e": {"value": e2e, "unit": UNIT,
                "h2d_bytes_per_step": int(vel_h.numel() * 4 + (0 if rho_h is None else rho_h.numel() * 4)),
                "d2h_bytes_per_step": int(seis_h.numel() * 4)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": kernel_traffic(w, "cpml_step", PML_SOURCES),
                     "peak_kind": peak_kind,
                     "kernel": "CPML time step (per-axis Psi launches + step_kernel + per-axis correction launches + record_kernel)",
                     "bytes_per_step": alg, "step_ms": step_ms},
        "clocks": clocks,
    }


def pml_cpu_baseline(w):
    """The CPML oracle on a bounded sample: the model cropped to 64^3 (same
    border), 6 time steps, operator assembly excluded."""
    from oracle import cpml as ocpml
    from oracle import oracle as orc
    n, nt = 64, 6
    vel = np.ascontiguousarray(w.vel[:n, :n, :n], np.float64)
    rho = None if w.rho is None else np.ascontiguousarray(w.rho[:n, :n, :n], np.float64)
    g = orc.make_grid(n, n, n, w.border, w.h, w.dt, nt)
    src = np.array([[n // 2 * w.h] * 3])
    rec = np.array([[n // 2 * w.h, n // 2 * w.h, 4 * w.h]])
    op = ocpml.Operators(orc, g, vel, rho, w.fpeak)
    sn, scale, S = ocpml._shot(op, src, 0, [0, 1], rec)
    t0 = time.perf_counter()
    ocpml.forward(op, w.wavelet[:nt].astype(np.float64), sn, scale, S)
    dt = time.perf_counter() - t0
    pts = (n + 2 * w.border) ** 3 * nt
    return {"value": pts / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"CPML oracle (scipy sparse products, FP64, one thread) on the model "
                      f"cropped to {n}^3 with border {w.border}, {nt} time steps after operator "
                      f"assembly"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--nt", type=int, default=None, help="time steps (default: the workload's 4000)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--time-blocking", type=int, default=0, choices=[0, 2],
                    help="model workloads: 2 = two time steps per launch (two-level kernel)")
    ap.add_argument("--boundary", default="sponge", choices=["sponge", "pml"],
                    help="model and gradient_single workloads: absorbing boundary (pml: "
                         "convolutional PML)")
    ap.add_argument("--no-gradient", action="store_true",
                    help="skip the 256^3 FWI gradient object of the headline line")
    ap.add_argument("--workload", default="model",
                    choices=["model", "model_small", "model_mid", "gradient_single",
                             "gradient_batched", "cnn", "gn_labels", "postproc"],
                    help="model: the headline modelling benchmark; gradient_*: FWI gradient "
                         "shots/s on the 256^3 single-shot or the 64-shot aperture workload")
    ap.add_argument("--autotune", action="store_true",
                    help="gradient workloads: measured adjoint decomposition (autotune.py)")
    ap.add_argument("--snapshots", type=int, default=0,
                    help="gradient workloads: revolve slots (0 = from free memory, -1 = all)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload.startswith("gradient"):
        return run_gradient_bench(args)
    if args.workload == "cnn":
        return run_cnn_bench(args)
    if args.workload == "gn_labels":
        return run_gn_bench(args)
    if args.workload == "postproc":
        return run_postproc_bench(args)

    import torch
    import torch.distributed as dist

    from paper_2502_12350_gb300 import build, mamute

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()

    w = workload(args.nt, args.workload)
    nt = w.nt
    pml = args.boundary == "pml"
    g = mamute.grid_of(w, cerjan=0.0, pml=1) if pml else mamute.grid_of(w)
    stream = torch.cuda.current_stream(dev)
    ctx = mamute.Context(local, stream.cuda_stream)
    lib = mamute.load()
    import ctypes
    lib.mamute_ctx_set_timing.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.mamute_ctx_last_timing.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_longlong),
                                           ctypes.POINTER(ctypes.c_longlong)]
    lib.mamute_ctx_set_timing(ctx._h, 1)
    vel = torch.from_numpy(w.vel).to(dev)
    rho = None if w.rho is None else torch.from_numpy(w.rho).to(dev)
    n_rec = int(w.rec_offset[-1])
    seis = torch.empty((n_rec, nt), device=dev)

    def step():
        ctx.model(g, vel, rho, w.src_xyz, w.wavelet, w.rec_offset, w.rec_xyz, seis,
                  time_blocking=args.time_blocking)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    loop_ms, launches, step_launches = [], 0, 0
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
            ms = ctypes.c_double()
            sl, tl = ctypes.c_longlong(), ctypes.c_longlong()
            lib.mamute_ctx_last_timing(ctx._h, ctypes.byref(ms), ctypes.byref(sl), ctypes.byref(tl))
            loop_ms.append(ms.value)
            launches += tl.value
            step_launches = sl.value
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_ms = ev0.elapsed_time(ev1)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    pts = w.n_padded * nt
    value = world * pts * args.steps / (total_ms / 1e3) / 1e9

    # End to end through the host-buffer entry point (pinned host memory).
    vel_h = torch.from_numpy(w.vel).pin_memory()
    rho_h = None if w.rho is None else torch.from_numpy(w.rho).pin_memory()
    seis_h = torch.empty((n_rec, nt), pin_memory=True)
    e2e_steps = max(1, min(args.steps, 3))

    def host_step():
        ctx.model_host(g, vel_h.numpy(), None if rho_h is None else rho_h.numpy(), w.src_xyz,
                       w.wavelet, w.rec_offset, w.rec_xyz, seis_h.numpy(),
                       time_blocking=args.time_blocking)

    host_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        host_step()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = world * pts / e2e_s / 1e9

    peak, peak_kind = _peaks()
    kernel_ms = statistics.median(loop_ms) / max(step_launches, 1)
    if pml:
        line = pml_line(args, w, world, total_ms, value, e2e, vel_h, rho_h, seis_h, launches,
                        kernel_ms, peak, peak_kind, clk.summary())
        ctx.close()
        if rank == 0 and not args.no_cpu_baseline:
            line["cpu_baseline"] = pml_cpu_baseline(w)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return 0
    # Algorithmic bytes per point and launch: u^n, u^{n-1}, A (and A m2) read
    # once, one new level written per time step the launch advances (two on
    # the two-level kernel).
    steps_per_launch = nt / max(step_launches, 1)
    two_level = steps_per_launch > 1.5
    reads = 16 if w.rho is not None else 12
    bpp = reads + 4 * (2 if two_level else 1)
    achieved = bpp * w.n_padded / (kernel_ms / 1e3) / 1e9
    kname = "pair_kernel_forward" if two_level else "step_kernel_forward"
    traffic = kernel_traffic(w, kname)

    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name + f"_{nt}steps",
                   "padded": list(w.padded)[::-1], "nt": nt, "shots": 1, "receivers": n_rec,
                   "l2": ("every array (%d MB) is larger than L2" % (w.n_padded * 4 // 2**20)
                          if w.n_padded * 4 > 129 * 2**20 else
                          "arrays fit in L2: the HBM roofline is reported but not binding"),
                   "parallelism": "replicas" if world > 1 else "single"},
        "e2e": {"value": e2e, "unit": UNIT,
                "h2d_bytes_per_step": int(vel_h.numel() * 4 + (0 if rho_h is None else rho_h.numel() * 4)),
                "d2h_bytes_per_step": int(seis_h.numel() * 4)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": ("pair_kernel (two time steps per launch)" if two_level
                                else "step_kernel<forward>"),
                     "bytes_per_point": bpp, "steps_per_launch": steps_per_launch,
                     "kernel_ms": kernel_ms},
        "clocks": clocks,
    }
    ctx.close()
    del vel, rho, seis
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_gradient and args.nt is None and args.workload == "model":
        # FWI gradient throughput of the 256^3 single-shot workload (2000 steps,
        # automatic storage), timed on its own; the headline value is unchanged.
        line["gradient"] = gradient_metrics("gradient_single", steps=3, warmup=2)
    if rank == 0 and not args.no_cpu_baseline:
        r, cores, sample, _ = cpu_oracle_rate(w, 2, 22, repeats=3)
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
