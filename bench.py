#!/usr/bin/env python3
"""Benchmark: batched neural-BRDF evaluation on one GB300 (or N replicas).

One step = one pass of the whole evaluation path (latent fetch, frame MLP,
frame build, direction transform, decoder MLP, RGB store) over one 1920x1080
frame of queries (2,073,600) with the FP16 tensor-core path: 2048^2 x 8 FP16
latent pyramid with 12 levels, frame MLP 8-16-6, decoder 14-64-64-3, uv from
a random smooth warp, lod from the warp's footprint, cosine-hemisphere
directions (synthetic, seeded).  The L2 is flushed (256 MiB write) before
every timed step, outside the timed kernel.

Printed (rank 0), one JSON line: evals/s of that step (value), the same
through the C ABI with host buffers (e2e), the roofline of the kernel, the
FP32 and FP8 forms of the same workload with their speed-ups, the serving
stream's p50/p99 frame latency, the FP64 oracle on the host cores
(cpu_baseline) and the clocks seen while timing.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--no-serve] [--serve-frames F] [--serve-repeats R] [--no-sweep] [--legs L]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "neural-BRDF evals/s FP16/FP8 vs plain FP32 at stated error; p50/p99 frame ms"
WORKLOAD = "fp16-2048sq-1920x1080"
# FP32 FMA (non-tensor) peak: 152 SMs x 128 lanes x 2 FLOP x 2070 MHz
ALU_PEAK_TFLOPS = round(152 * 128 * 2 * 2.07e9 / 1e12, 1)
# matrix FLOPs per query of the reverse mode (frame MLP 8-16-6, decoder
# 14-64-64-3): forward recompute, deltas and weight gradients, 3 x 10,816
BWD_FLOPS_PER_QUERY = 3 * 2 * (8 * 16 + 16 * 6 + 14 * 64 + 64 * 64 + 64 * 3)
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-frames", type=int, default=720)
    ap.add_argument("--serve-repeats", type=int, default=4)
    ap.add_argument("--serve-trace", default=None, help="write every served frame's timeline (.npz) here")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--legs", default="precision,paper,binned,scene,sampling",
                    help="which of the sweep legs run (comma list; --no-sweep runs none)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-sweep4k", action="store_true")
    ap.add_argument("--train-steps", type=int, default=2000)
    return ap.parse_args()


# ----------------------------------------------------------------------------
# distributed plumbing (replicas: no data-path collective)
# ----------------------------------------------------------------------------
def dist_setup(args, backend=None):
    """Rank, world size and local GPU from the torchrun environment; one
    process group per job (NCCL for the GPU arm; gloo where no GPU is used)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = backend or ("nccl" if args.impl == "ours" else "gloo")
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    """SM clock, power and clock-event reasons sampled every ~2 ms from NVML
    (libnvidia-ml through ctypes; read-only queries) while the timed region
    runs, so that even a short region gets samples.  Falls back to
    `nvidia-smi -lms 100` where NVML cannot be loaded."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index, period_s=0.002):
        self.dev = device_index
        self.period = period_s
        self.samples = []
        self.proc = None
        self.lines = []
        self.nvml = None
        self._stop = threading.Event()
        try:
            self._nvml_open()
        except Exception:
            self.nvml = None

    def _nvml_open(self):
        import ctypes as C
        lib = C.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit")
        h = C.c_void_p()
        ok = False
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.dev).uuid)
            ok = lib.nvmlDeviceGetHandleByUUID(("GPU-" + uuid).encode(), C.byref(h)) == 0
        except Exception:
            ok = False
        if not ok and lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(self.dev), C.byref(h)) != 0:
            raise OSError("nvml handle")
        mx = C.c_uint()
        lib.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(mx))
        self.nvml, self.h, self.max_mhz, self.C = lib, h, float(mx.value), C
        self.reason_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def _nvml_loop(self):
        C, lib, h = self.C, self.nvml, self.h
        clk, mw, rs = C.c_uint(), C.c_uint(), C.c_ulonglong()
        while not self._stop.is_set():
            if lib.nvmlDeviceGetClockInfo(h, 1, C.byref(clk)) == 0:
                p = float(mw.value) / 1000.0 if lib.nvmlDeviceGetPowerUsage(h, C.byref(mw)) == 0 else None
                r = int(rs.value) if self.reason_fn(h, C.byref(rs)) == 0 else 0
                self.samples.append((float(clk.value), p, r))
            time.sleep(self.period)

    def start(self):
        if self.nvml is not None:
            self.thread = threading.Thread(target=self._nvml_loop, daemon=True)
            self.thread.start()
            return
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.nvml is not None:
            self._stop.set()
            self.thread.join(timeout=5)
            sm = [s[0] for s in self.samples]
            power = [s[1] for s in self.samples if s[1] is not None]
            reasons = set()
            for _, _, r in self.samples:
                for bit, name in self.REASONS.items():
                    if r & bit:
                        reasons.add(name)
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz,
                    "reasons": sorted(reasons), "samples": len(sm), "source": "nvml, 2 ms period",
                    "power_w_max": max(power) if power else None}
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi, 100 ms period",
                "power_w_max": max(power) if power else None}


# ----------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------
def workload():
    import workloads as W
    return W.workload(2)


def unique_texel_bytes(w):
    """Compulsory texel bytes of one launch: distinct texels the 1080p frame
    touches (both levels of every trilinear fetch) x 16 bytes."""
    q = w["queries"]
    W0, H0, L = w["W0"], w["H0"], w["L"]
    sizes = [(max(1, W0 >> l), max(1, H0 >> l)) for l in range(L)]
    offs = np.cumsum([0] + [a * b for a, b in sizes])
    lod = np.nan_to_num(q["lod"].astype(np.float32), nan=0.0)
    l = np.clip(lod, 0, L - 1)
    l0 = np.floor(l).astype(np.int64)
    t = l - l0
    l1 = np.minimum(l0 + 1, L - 1)
    idx = []
    for lev_arr, keep in ((l0, np.ones_like(t, bool)), (l1, t != 0)):
        u = q["u"][keep].astype(np.float32)
        v = q["v"][keep].astype(np.float32)
        lv = lev_arr[keep]
        Wl = np.array([s[0] for s in sizes])[lv]
        Hl = np.array([s[1] for s in sizes])[lv]
        x = u * Wl.astype(np.float32) - np.float32(0.5)
        y = v * Hl.astype(np.float32) - np.float32(0.5)
        x0 = np.floor(x).astype(np.int64)
        y0 = np.floor(y).astype(np.int64)
        for dx in (0, 1):
            for dy in (0, 1):
                xi = np.mod(x0 + dx, Wl)
                yi = np.mod(y0 + dy, Hl)
                idx.append(offs[lv] + yi * Wl + xi)
    return int(np.unique(np.concatenate(idx)).size) * 16


def kernel_sha():
    h = hashlib.sha256()
    for f in ("eval_tc.cuh", "eval_f16.cu", "common.cuh", "tc_ptx.cuh"):
        with open(os.path.join(ROOT, "paper_2305_02678_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the FP16 kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "eval_f16_1920x1080.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    s = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", txt)
    if not m or not s or s.group(1) != kernel_sha():
        return None
    return float(m.group(1))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    return 6800.0, 1900.0, "fallback"


# FP32 FMA rate of this GPU: every thread runs 16 independent chains of
# dependent FMAs (enough to fill the pipes), grid = a multiple of the SMs.
_FFMA_SRC = r"""
#include <cuda_runtime.h>
__global__ void __launch_bounds__(256) ffma_loop(float* out, int iters, float a, float b) {
  float x[16];
  #pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = threadIdx.x * 1e-3f + k;
  for (int i = 0; i < iters; ++i) {
    #pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.0f;
  #pragma unroll
  for (int k = 0; k < 16; ++k) s += x[k];
  if (s == 1234.5f) out[0] = s;  // keeps the chains live
}
extern "C" float ffma_tflops(int sms) {
  float* out = nullptr;
  if (cudaMalloc(&out, 4) != cudaSuccess) return -1.0f;
  const int blocks = sms * 8, threads = 256, iters = 8192;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  ffma_loop<<<blocks, threads>>>(out, 64, 0.999f, 1e-3f);  // warm-up
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    ffma_loop<<<blocks, threads>>>(out, iters, 0.999f, 1e-3f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const cudaError_t e = cudaGetLastError();
  cudaFree(out);
  if (e != cudaSuccess) return -1.0f;
  return (float)(2.0 * 16.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12);
}
"""


def measured_fp32_fma_tflops(num_sms):
    """FP32 FMA throughput measured with a small kernel compiled here (nvcc);
    None where it cannot be built."""
    import ctypes
    import subprocess
    import tempfile
    try:
        d = tempfile.mkdtemp(prefix="ffma_")
        src, lib = os.path.join(d, "ffma.cu"), os.path.join(d, "libffma.so")
        with open(src, "w") as f:
            f.write(_FFMA_SRC)
        subprocess.check_call(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                               "-Xcompiler", "-fPIC", "-shared", "-o", lib, src])
        L = ctypes.CDLL(lib)
        L.ffma_tflops.restype = ctypes.c_float
        v = float(L.ffma_tflops(int(num_sms)))
        return round(v, 1) if v > 0 else None
    except Exception:
        return None


def measured_fp8_tflops(dev):
    """Dense E4M3 tensor throughput: torch._scaled_mm (cuBLASLt) on 8192^3,
    best of 10 (a library GEMM, as the bf16 peak in MEASURED_PEAKS.json)."""
    import torch
    try:
        n = 8192
        a = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn).t()
        one = torch.ones((), device=dev)
        for _ in range(3):
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        best = 1e30
        for _ in range(10):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
            e.record()
            torch.cuda.synchronize()
            best = min(best, s.elapsed_time(e))
        del a, b
        return round(2.0 * n ** 3 / (best * 1e-3) / 1e12, 1)
    except Exception:
        return None


# ----------------------------------------------------------------------------
# timing helpers
# ----------------------------------------------------------------------------
def time_launches(fn, steps, warmup, flush, stream):
    """Per-step CUDA-event times (ms) of fn(), L2 flushed before each step."""
    import torch
    for _ in range(warmup):
        flush()
        fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        times.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in times]


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def run_ours(args):
    import torch

    import workloads as W
    from paper_2305_02678_gb300 import Context
    from paper_2305_02678_gb300 import binding as B

    world, rank, local = dist_setup(args)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = workload()
    q = w["queries"]
    n = int(q["u"].shape[0])
    m = w["model"]
    stream = torch.cuda.current_stream(dev)
    ctx = Context(local)
    mat16 = ctx.material(w["W0"], w["H0"], w["L"], w["pyramid"], m["frame"], m["decoder"], precision=B.NAM_PREC_F16)
    dq = {k: torch.from_numpy(v).to(dev) for k, v in q.items() if k != "xi"}
    out16 = torch.empty((n, 3), device=dev)
    flush_buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def flush():
        flush_buf.fill_(1.0)

    def step16():
        B.nam_eval(ctx.h, mat16.h, dq, n, out16, stream, 0)

    # ---- headline: FP16 path, device-resident inputs --------------------
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t_wall0 = time.perf_counter()
    times = time_launches(step16, args.steps, args.warmup, flush, stream)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    barrier(world)
    ms = statistics.fmean(times)
    ms_max = max_over_ranks(world, ms, dev)
    ctx.check()
    value = world * n / (ms_max * 1e-3)

    # ---- e2e: host buffers through the C ABI, copies inside the timed region
    pinned = {k: torch.from_numpy(v).pin_memory() for k, v in q.items() if k != "xi"}
    host_out = torch.empty((n, 3), dtype=torch.float32).pin_memory()

    def step_host():
        B.nam_eval_host(ctx.h, mat16.h, pinned, n, host_out, stream, 0)

    e2e_times = time_launches(step_host, max(3, args.steps // 2), 2, flush, stream)
    e2e_ms = max_over_ranks(world, statistics.fmean(e2e_times), dev)
    # the same through the staged-copy path (device staging area, chunked
    # copies overlapping the kernels), for comparison
    staged_times = time_launches(lambda: B.nam_eval_host(ctx.h, mat16.h, pinned, n, host_out, stream,
                                                         B.NAM_HOST_STAGED), max(3, args.steps // 2), 2, flush,
                                 stream)
    staged_ms = statistics.fmean(staged_times)
    h2d = sum(int(t.numel()) * 4 for t in pinned.values())
    d2h = n * 12
    # the host link's own rate: the step's input bytes pinned -> device as one
    # copy (the e2e step moves them plus the RGB the other way, concurrently)
    link_src = torch.empty(h2d // 4, dtype=torch.float32).pin_memory()
    link_dst = torch.empty(h2d // 4, device=dev)
    link_times = time_launches(lambda: link_dst.copy_(link_src, non_blocking=True), max(3, args.steps // 2), 2,
                               flush, stream)
    link_gbs = h2d / (statistics.fmean(link_times) * 1e-3) / 1e9
    del link_src, link_dst

    # ---- roofline of the FP16 kernel ------------------------------------
    hbm, tflops, peak_kind = measured_peaks()
    texel_bytes = unique_texel_bytes(w)
    io_bytes = n * (9 * 4 + 12)
    weight_bytes = int(mat16.info.resident_bytes - w["pyramid"].nbytes - mat16.info.n_params * 4)
    alg_bytes = io_bytes + texel_bytes + weight_bytes
    alg_flops = 2 * n * (8 * 16 + 16 * 6 + 14 * 64 + 64 * 64 + 64 * 3)
    t_s = ms * 1e-3
    achieved = alg_bytes / t_s / 1e9
    t_roof = max(alg_bytes / (hbm * 1e9), alg_flops / (tflops * 1e12))
    props = torch.cuda.get_device_properties(dev)
    peaks_here = {"fp32_fma_tflops": measured_fp32_fma_tflops(props.multi_processor_count),
                  "fp8_e4m3_tensor_tflops": measured_fp8_tflops(dev),
                  "how": "FP32: a kernel of 16 independent FMA chains per thread over 8 x SMs blocks of 256 "
                         "threads (best of 5); FP8: torch._scaled_mm e4m3 8192^3 (best of 10)"}
    roofline = {"bound": "hbm" if alg_bytes / (hbm * 1e9) >= alg_flops / (tflops * 1e12) else "tensor",
                "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "traffic": profiled_traffic(), "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                "alg_bytes_per_launch": alg_bytes, "alg_flops_per_launch": alg_flops,
                "tensor_time_at_peak_us": round(alg_flops / (tflops * 1e12) * 1e6, 2),
                "roofline_time_us": round(t_roof * 1e6, 2), "kernel": "eval_f16_kernel<64,frame MLP,2 hidden,f16 latents>",
                "measured_peaks_here": peaks_here}

    # ---- precision sweep on the same workload ----------------------------
    sweep = {}
    out8 = None
    legs = set() if args.no_sweep else set(args.legs.split(","))
    if "precision" in legs:
        mat32 = ctx.material(w["W0"], w["H0"], w["L"], w["pyramid"], m["frame"], m["decoder"],
                             precision=B.NAM_PREC_F32)
        out32 = torch.empty((n, 3), device=dev)
        t32 = time_launches(lambda: B.nam_eval(ctx.h, mat32.h, dq, n, out32, stream, 0),
                            max(3, args.steps // 4), 2, flush, stream)
        ms32 = statistics.fmean(t32)
        sweep["fp32_evals_per_s"] = round(n / (ms32 * 1e-3), 1)
        sweep["fp32_ms"] = round(ms32, 4)
        sweep["fp16_speedup_vs_fp32"] = round(ms32 / ms, 2)
        mat32.destroy()
        # FP8: static activation scales from a 65,536-query calibration batch
        cq = W.calibration_queries(2)
        dcq = {k: torch.from_numpy(v).to(dev) for k, v in cq.items() if k != "xi"}
        scales = B.nam_fp8_calibrate(ctx.h, mat16.h, dcq, len(cq["u"]), stream)[:3]
        mat8 = ctx.material(w["W0"], w["H0"], w["L"], w["pyramid"], m["frame"], m["decoder"],
                            precision=B.NAM_PREC_FP8, act_scale=scales)
        out8 = torch.empty((n, 3), device=dev)
        t8 = time_launches(lambda: B.nam_eval(ctx.h, mat8.h, dq, n, out8, stream, 0), max(3, args.steps // 2), 2,
                           flush, stream)
        ms8 = statistics.fmean(t8)
        sweep["fp8_evals_per_s"] = round(n / (ms8 * 1e-3), 1)
        sweep["fp8_ms"] = round(ms8, 4)
        sweep["fp8_speedup_vs_fp32"] = round(ms32 / ms8, 2)
        sweep["fp8_act_scales"] = [float(x) for x in scales]
        mat8.destroy()
    # ---- serving stream (its own context; before the legs that leave large
    # host and device allocations behind in this process) --------------------
    serving = None
    if not args.no_serve and rank == 0:
        serving = run_serving(local, args.serve_frames, repeats=args.serve_repeats, trace=args.serve_trace)
    # ---- precision sweep at 3840x2160 ---------------------------------------
    sweep4k, outs4k = None, None
    if not args.no_sweep4k:
        sweep4k, outs4k = run_sweep_4k(ctx, dev, stream, flush, args)
    # ---- the paper's decoder sizes with its frame form ----------------------
    paper = None
    if "paper" in legs:
        paper = run_paper_decoders(ctx, dev, stream, flush, w, dq, n, args)
    # ---- per-pixel materials through the binning pre-pass ------------------
    binned = None
    if "binned" in legs:
        binned = run_binned(ctx, dev, stream, flush, w, dq, n, args)
    # ---- the synthetic-scene harness at 1080p --------------------------------
    scene = None
    if "scene" in legs:
        scene = run_scene(ctx, dev, stream, args)
    # ---- importance sampling on the 1080p frame ------------------------------
    sampling = None
    if "sampling" in legs:
        sampling = run_sampling(ctx, dev, stream, flush, w, dq, n, args, texel_bytes=texel_bytes)
    # ---- training: 2,000 Adam steps on the procedural GGX target ------------
    training = None
    if args.train_steps > 0 and rank == 0:
        training = run_training(ctx, dev, stream, args.train_steps, fma_peak=peaks_here["fp32_fma_tflops"])
        if args.train_steps >= 10:
            training["albedo_head"] = run_albedo_head(ctx, dev, stream, min(1000, args.train_steps))
            training["encoder_bootstrap"] = run_encoder_bootstrap(ctx, dev, stream, args.train_steps // 2,
                                                                  args.train_steps - args.train_steps // 2)

    # ---- CPU baseline: the FP64 oracle on the host cores -------------------
    cpu = None
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        cpu = cpu_baseline(w, out16.cpu().numpy(), args.cpu_seconds,
                           None if out8 is None else out8.cpu().numpy(), outs4k)

    mat16.destroy()
    ctx.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_max, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "queries_per_step": n, "pyramid": "2048x2048x8 fp16, 12 levels",
                       "frame_mlp": "8-16-6", "decoder": "14-64-64-3", "filter": "trilinear",
                       "l2": "flushed (256 MiB write) before every timed step, outside the timed kernel",
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": round(world * n / (e2e_ms * 1e-3), 1), "unit": "evals/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 4),
                    "api": "nam_eval_host with pinned host queries and output: the kernel reads the inputs and "
                           "writes the RGB in host memory directly where the device reads host page tables, "
                           "else staged copies",
                    "staged_copies_ms_per_step": round(staged_ms, 4),
                    "link": {"h2d_gbs_measured": round(link_gbs, 1),
                             "bound_ms": round(h2d / (link_gbs * 1e9) * 1e3, 4),
                             "frac": round(h2d / (link_gbs * 1e9) * 1e3 / e2e_ms, 3),
                             "note": "the input bytes of a step over the host link's measured rate (one pinned "
                                     "copy of the same size); the RGB flows the other way at the same time"}},
            "gpu_launches": args.steps,
            "roofline": roofline,
            "precision_sweep": sweep,
            "precision_sweep_3840x2160": sweep4k,
            "paper_decoders": paper,
            "binned_materials": binned,
            "scene_harness": scene,
            "importance_sampling": sampling,
            "training": training,
            "serving": serving,
            "cpu_baseline": cpu,
            "clocks": clk,
            "timed_region_wall_s": round(t_wall, 3),
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_sweep_4k(ctx, dev, stream, flush, args):
    """The 3840x2160 sweep: same pyramid and MLPs, FP32 / FP16 / FP8 kernels,
    device-resident queries, L2 flushed before each timed launch.  Returns
    timings and the three outputs for the error report of cpu_baseline."""
    import torch

    import workloads as W
    from paper_2305_02678_gb300 import binding as B
    w = W.workload(3)
    q = w["queries"]
    n = int(q["u"].shape[0])
    m = w["model"]
    dq = {k: torch.from_numpy(v).to(dev) for k, v in q.items() if k != "xi"}
    mat16 = ctx.material(w["W0"], w["H0"], w["L"], w["pyramid"], m["frame"], m["decoder"], precision=B.NAM_PREC_F16)
    cq = W.calibration_queries(3)
    dcq = {k: torch.from_numpy(v).to(dev) for k, v in cq.items() if k != "xi"}
    scales = B.nam_fp8_calibrate(ctx.h, mat16.h, dcq, len(cq["u"]), stream)[:3]
    mats = {"fp32": ctx.material(w["W0"], w["H0"], w["L"], w["pyramid"], m["frame"], m["decoder"],
                                 precision=B.NAM_PREC_F32),
            "fp16": mat16,
            "fp8": ctx.material(w["W0"], w["H0"], w["L"], w["pyramid"], m["frame"], m["decoder"],
                                precision=B.NAM_PREC_FP8, act_scale=scales)}
    res, outs = {"workload": "fp16-2048sq-3840x2160", "queries": n, "fp8_act_scales": [float(x) for x in scales]}, {}
    steps = max(3, args.steps // 2)
    for name, mat in mats.items():
        out = torch.empty((n, 3), device=dev)
        t = time_launches(lambda: B.nam_eval(ctx.h, mat.h, dq, n, out, stream, 0), steps, 2, flush, stream)
        ms = statistics.fmean(t)
        res[f"{name}_ms"] = round(ms, 4)
        res[f"{name}_evals_per_s"] = round(n / (ms * 1e-3), 1)
        outs[name] = out
    for name in ("fp16", "fp8"):
        res[f"{name}_speedup_vs_fp32"] = round(res["fp32_ms"] / res[f"{name}_ms"], 2)
    # the FP16 launch against the same roofline as the 1080p headline
    hbm, _, peak_kind = measured_peaks()
    weight_bytes = int(mat16.info.resident_bytes - w["pyramid"].nbytes - mat16.info.n_params * 4)
    alg = n * (9 * 4 + 12) + unique_texel_bytes(w) + weight_bytes
    gbs = alg / (res["fp16_ms"] * 1e-3) / 1e9
    res["fp16_roofline"] = {"bound": "hbm", "alg_bytes_per_launch": alg, "achieved": round(gbs, 1), "unit": "GB/s",
                            "peak": hbm, "frac": round(gbs / hbm, 4), "peak_source": peak_kind}
    k = 1 << 20   # error sample: the first 1,048,576 queries
    host = {name: o[:k].cpu().numpy() for name, o in outs.items()}
    for mat in mats.values():
        mat.destroy()
    return res, {"w": w, "sample": k, "out": host}


def run_paper_decoders(ctx, dev, stream, flush, w, dq, n, args):
    """The paper's three decoder sizes (2 x 16, 2 x 32, 3 x 64 hidden units)
    with its frame form (linear 8 -> 12, two frames, 20 decoder inputs), FP16
    on the 1080p frame (same pyramid and queries), seeded random weights."""
    import workloads as W
    from paper_2305_02678_gb300 import binding as B
    out = {"workload": "fp16-2048sq-1920x1080, frame 8->12 (2 frames), decoder 20-H..-3"}
    rng = W.rng_streams(W.SEEDS[2] + 21, 3)
    for k, (H, NH) in enumerate(((16, 2), (32, 2), (64, 3))):
        model = W.make_model(rng[k], (20,) + (H,) * NH + (3,), (8, 12))
        mat = ctx.material(w["W0"], w["H0"], w["L"], w["pyramid"], model["frame"], model["decoder"],
                           precision=B.NAM_PREC_F16)
        import torch
        o = torch.empty((n, 3), device=dev)
        t = statistics.fmean(time_launches(lambda: B.nam_eval(ctx.h, mat.h, dq, n, o, stream, 0),
                                           max(3, args.steps // 2), 2, flush, stream))
        out[f"{NH}x{H}_ms"] = round(t, 4)
        out[f"{NH}x{H}_evals_per_s"] = round(n / (t * 1e-3), 1)
        mat.destroy()
    return out


def run_binned(ctx, dev, stream, flush, w, dq, n, args, n_mat=16):
    """Per-query material ids with no tile coherence: 16 FP16 materials (the
    1080p pyramid, seeded decoders and frame MLPs of their own), a uniformly
    random material per pixel, evaluated through nam_eval_binned (device
    histogram, scan, a permutation of the query indices by material, one
    chunked launch that reads through it and writes in place); against the
    single-material launch of the headline; then per-tile selection on the
    same ids and both on 16 screen regions."""
    import torch

    import workloads as W
    from paper_2305_02678_gb300 import binding as B
    rng = W.rng_streams(W.SEEDS[2] + 31, n_mat + 1)
    mats = []
    for k in range(n_mat):
        model = W.make_model(rng[k], (14, 64, 64, 3), (8, 16, 6))
        mats.append(ctx.material(w["W0"], w["H0"], w["L"], w["pyramid"], model["frame"], model["decoder"],
                                 precision=B.NAM_PREC_F16))
    ids = torch.from_numpy(rng[n_mat].integers(0, n_mat, n).astype(np.int32)).to(dev)
    o = torch.empty((n, 3), device=dev)
    handles = [m.h for m in mats]
    t = statistics.fmean(time_launches(lambda: B.nam_eval_binned(ctx.h, handles, dq, ids, n, o, stream, 0),
                                       max(3, args.steps // 2), 2, flush, stream))
    t1 = statistics.fmean(time_launches(lambda: B.nam_eval(ctx.h, mats[0].h, dq, n, o, stream, 0),
                                        max(3, args.steps // 2), 2, flush, stream))
    reps = max(3, args.steps // 2)
    # per-tile selection on the same per-pixel ids: every tile holds several
    # of the 16 materials, so every query goes through binning
    t_sel_pp = statistics.fmean(time_launches(lambda: B.nam_eval_select(ctx.h, handles, dq, ids, n, o, stream, 0),
                                              reps, 2, flush, stream))
    # screen regions: the pixels of the 1920x1080 frame (queries in row-major
    # pixel order) take the material of the nearest of 16 random sites, so a
    # 128-pixel run is mixed only where a region boundary crosses it
    width = 1920
    sites = W.rng_streams(W.SEEDS[2] + 32, 1)[0].random((n_mat, 2)) * np.array([width, n // width])
    px = (np.arange(n) % width).astype(np.float32)
    py = (np.arange(n) // width).astype(np.float32)
    best = np.full(n, np.inf, np.float32)
    reg = np.zeros(n, np.int32)
    for k, (sx, sy) in enumerate(sites):
        d = (px - sx) ** 2 + (py - sy) ** 2
        upd = d < best
        best[upd], reg[upd] = d[upd], k
    tiles = np.pad(reg, (0, (-n) % 128), mode="edge").reshape(-1, 128)
    coherent = float(np.mean(np.all(tiles == tiles[:, :1], axis=1)))
    kt = np.array([np.unique(t).size for t in tiles])
    passes = float(np.mean(kt))
    binned_tiles = float(np.mean(kt > B.NAM_SELECT_MAX_PASSES))
    rids = torch.from_numpy(reg).to(dev)
    t_sel = statistics.fmean(time_launches(lambda: B.nam_eval_select(ctx.h, handles, dq, rids, n, o, stream, 0),
                                           reps, 2, flush, stream))
    t_bin_reg = statistics.fmean(time_launches(lambda: B.nam_eval_binned(ctx.h, handles, dq, rids, n, o, stream, 0),
                                               reps, 2, flush, stream))
    for m in mats:
        m.destroy()
    ctx.check()
    return {"workload": f"fp16-2048sq-1920x1080, {n_mat} materials, material drawn per pixel",
            "binned_ms": round(t, 4), "binned_evals_per_s": round(n / (t * 1e-3), 1),
            "single_material_ms": round(t1, 4), "overhead_vs_single": round(t / t1, 3),
            "note": "binning passes (count, plan, a permutation of the query indices by material) plus the "
                    "chunked tensor-core launch, which reads each query through the permutation, writes its RGB "
                    "in place, and restages a warpgroup's weights when its chunk's material changes",
            "select": {
                "per_pixel_ms": round(t_sel_pp, 4), "per_pixel_vs_binned": round(t_sel_pp / t, 3),
                "regions_workload": f"{n_mat} screen regions (nearest of {n_mat} random sites), "
                                    f"{coherent:.3f} of the 128-query tiles coherent, "
                                    f"{passes:.3f} materials per tile",
                "regions_tiles_binned_by_select": round(binned_tiles, 3),
                "regions_select_ms": round(t_sel, 4), "regions_binned_ms": round(t_bin_reg, 4),
                "note": f"nam_eval_select, in place: a 128-query tile with k <= {B.NAM_SELECT_MAX_PASSES} "
                        "materials runs as k tensor-core passes (one per material); the queries of tiles with "
                        "more are binned by material (the binning passes limited to those tiles) and run in "
                        "coherent chunks; three small passes build the pass table"}}


def run_scene(ctx, dev, stream, args, width=1920, height=1080):
    """The synthetic-scene harness at 1920x1080: a ground plane and three
    spheres with four FP16 materials (1024^2 x 8 pyramids, 11 levels, frame
    MLP 8-16-6, decoder 14-64-64-3, sampler 11-32-32-32-9); per frame the
    G-buffer, material binning, one BSDF sample and one light sample per
    pixel with MIS and shadow rays (nam_scene_render_direct)."""
    import torch

    import workloads as W
    from paper_2305_02678_gb300 import binding as B
    rng = W.rng_streams(W.SEEDS[2] + 41, 13)
    W0, L = 1024, 11
    mats = []
    for k in range(4):
        pyr = W.make_pyramid(rng[k], W0, W0, L, dtype=np.float16)
        model = W.make_model(rng[4 + k], (14, 64, 64, 3), (8, 16, 6))
        smp = W.make_mlp(rng[8 + k], (11, 32, 32, 32, 9))
        mats.append(ctx.material(W0, W0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F16,
                                 sampler=smp))
    sc = B.make_scene(width, height, (0.0, 1.6, -6.0), (0.0, 0.7, 0.0), (0.0, 1.0, 0.0), 0.9,
                      [(-1.6, 1.0, 0.0, 1.0, 1), (0.4, 0.6, -0.6, 0.6, 2), (1.9, 1.2, 1.0, 1.2, 3)],
                      0.0, 0, 2.0, 1.5)
    n = width * height
    bounces = 3
    var = torch.from_numpy(rng[12].random((bounces, n, 5)).astype(np.float32)).to(dev)
    img = torch.empty((n, 3), device=dev)
    handles = [m.h for m in mats]
    reps = max(3, args.steps // 2)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    ms = timed(lambda: B.nam_scene_render_direct(ctx.h, sc, handles, var[0], img, stream))
    ms_paths = timed(lambda: B.nam_scene_render_paths(ctx.h, sc, handles, bounces, var, img, stream))
    for m in mats:
        m.destroy()
    ctx.check()
    return {"workload": f"scene {width}x{height}: ground plane + 3 spheres, 4 FP16 materials with samplers",
            "ms_per_frame": round(ms, 4), "frames_per_s": round(1e3 / ms, 1),
            "paths_bounces": bounces, "paths_ms_per_frame": round(ms_paths, 4),
            "note": "direct: G-buffer, material binning (one device-to-host read of the four counts), "
                    "nam_sample + nam_sample_pdf + 2 x nam_eval per material range, shading with shadow rays; "
                    "paths: the same at each of up to 3 vertices, continuing along the BSDF sample"}


def run_sampling(ctx, dev, stream, flush, w, dq, n, args, texel_bytes=None):
    """nam_sample (direction + density) and nam_sample_pdf over the 1080p
    frame with a seeded 11-32-32-32-9 sampler network, L2 flushed before each
    timed launch.  The network runs on the tensor cores (binary16 hi/lo
    splits, FP32 accuracy); roofline: HBM, per query 12 B of u, v, lod, 12 B
    of wi, 12 B of variates, 12 B of direction and 4 B of density out, plus
    the frame's compulsory texel bytes once."""
    import torch

    import workloads as W
    from paper_2305_02678_gb300 import binding as B
    m = w["model"]
    rng = W.rng_streams(W.SEEDS[2] + 11, 2)
    sampler = W.make_mlp(rng[0], (11, 32, 32, 32, 9))
    mat = ctx.material(w["W0"], w["H0"], w["L"], w["pyramid"], m["frame"], m["decoder"], precision=B.NAM_PREC_F16,
                       sampler=sampler)
    u = torch.from_numpy(rng[1].random((n, 3)).astype(np.float32)).to(dev)
    wo = torch.empty((n, 3), device=dev)
    pdf = torch.empty(n, device=dev)
    steps = max(3, args.steps // 2)
    t_s = statistics.fmean(time_launches(lambda: B.nam_sample(ctx.h, mat.h, dq, n, u, wo, pdf, stream), steps, 2,
                                         flush, stream))
    t_p = statistics.fmean(time_launches(lambda: B.nam_sample_pdf(ctx.h, mat.h, dq, n, pdf, stream), steps, 2, flush,
                                         stream))
    mat.destroy()
    ctx.check()
    if texel_bytes is None:
        texel_bytes = unique_texel_bytes(w)
    alg = 52 * n + texel_bytes
    peak, _, src = measured_peaks()
    gbs = alg / (t_s * 1e-3) / 1e9
    return {"workload": "fp16-2048sq-1920x1080 + sampler 11-32-32-32-9 (FP32 weights, tensor cores)", "queries": n,
            "sample_ms": round(t_s, 4), "samples_per_s": round(n / (t_s * 1e-3), 1),
            "pdf_ms": round(t_p, 4), "pdf_evals_per_s": round(n / (t_p * 1e-3), 1),
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "unit": "GB/s", "peak": peak,
                         "frac": round(gbs / peak, 4), "peak_source": f"{src} (hbm_gbs)",
                         "alg_bytes_per_launch": alg, "alg_flops_per_launch": 2 * 2688 * n}}


def run_training(ctx, dev, stream, steps, batch=262144, pool=8, fma_peak=None):
    """Fit a 1024^2 x 8 FP32 latent pyramid (11 levels) with the frame MLP and
    a 14-64-64-3 decoder to the procedural GGX-over-Lambert target: `steps`
    fused steps (forward, log-L1 loss, reverse mode with atomic pyramid
    scatter, Adam) on batches of 262,144 uniform queries, cycling through a
    pool of `pool` pre-drawn batches resident on the device."""
    import torch

    import workloads as W
    from paper_2305_02678_gb300 import binding as B
    w = W.workload(4)
    m = w["model"]
    mat = ctx.material(w["W0"], w["H0"], w["L"], w["pyramid"], m["frame"], m["decoder"], precision=B.NAM_PREC_F32,
                       trainable=True)
    rng = W.rng_streams(W.SEEDS[4] + 7, 1)[0]
    batches = []
    for _ in range(pool):
        q = W.uniform_queries(rng, batch, 10.0)
        y = torch.from_numpy(W.target_rgb(w["target"], q)).to(dev)
        batches.append(({k: torch.from_numpy(v).to(dev) for k, v in q.items() if k != "xi"}, y))
    losses = []
    for s in range(1, 4):   # warm-up steps are real steps of the same run
        dq, y = batches[s % pool]
        losses.append(B.nam_train_step(ctx.h, mat.h, dq, y, batch, step=s, stream=stream))
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for s in range(4, steps + 1):
        dq, y = batches[s % pool]
        want = s % 100 == 0 or s == steps
        l = B.nam_train_step(ctx.h, mat.h, dq, y, batch, step=s, stream=stream, want_loss=want)
        if want:
            losses.append(l)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / (steps - 3)
    # the reverse-mode kernel alone (nam_backward: the step's kernel without
    # the fused loss) on one batch, for its ALU roofline
    g = torch.Generator(device=dev)
    g.manual_seed(W.SEEDS[4] + 8)
    gr = torch.randn((batch, 3), device=dev, generator=g) * (1.0 / (3 * batch))
    gp = torch.zeros(mat.info.n_params, device=dev)
    gz = torch.zeros((mat.info.texels, 8), device=dev)
    dq0 = batches[0][0]
    for _ in range(3):
        B.nam_backward(ctx.h, mat.h, dq0, batch, gr, gp, gz, stream)
    torch.cuda.synchronize()
    reps = 20
    a.record(stream)
    for _ in range(reps):
        B.nam_backward(ctx.h, mat.h, dq0, batch, gr, gp, gz, stream)
    b.record(stream)
    torch.cuda.synchronize()
    bwd_ms = a.elapsed_time(b) / reps
    tflops = BWD_FLOPS_PER_QUERY * batch / (bwd_ms * 1e-3) / 1e12
    # the FP32 FMA peak measured on this GPU when there is one, else the unit
    # count x clock figure
    peak = fma_peak if fma_peak and fma_peak > 0 else ALU_PEAK_TFLOPS
    peak_note = ("measured here (16 independent FMA chains per thread)" if peak != ALU_PEAK_TFLOPS
                 else "152 SMs x 128 lanes at 2.07 GHz")
    mat.destroy()
    ctx.check()
    return {"workload": "train-1024sq-262144", "steps": steps, "batch": batch, "ms_per_step": round(ms, 4),
            "backward_ms": round(bwd_ms, 4),
            "backward_roofline": {"kernel": "backward_kernel, H = 64, frame MLP", "bound": "alu",
                                  "achieved": round(tflops, 2), "peak": peak, "unit": "TFLOP/s",
                                  "frac": round(tflops / peak, 4),
                                  "flops_per_query": BWD_FLOPS_PER_QUERY,
                                  "note": "matrix FLOPs (2 per multiply-add) of the forward recompute, the "
                                          "deltas and the weight gradients; FP32 FMA peak " + peak_note},
            "steps_per_s": round(1e3 / ms, 1), "samples_per_s": round(batch * 1e3 / ms, 1),
            "loss_first": round(losses[0], 5), "loss_last": round(losses[-1], 5),
            "loss_every_100": [round(x, 5) for x in losses[3:]],
            "note": "each step: one kernel for the FP32 forward, the log-L1 loss and the hand-written reverse "
                    "mode (atomic pyramid scatter), then Adam over 11.18 M pyramid + MLP parameters; loss read "
                    "back every 100 steps"}


def run_encoder_bootstrap(ctx, dev, stream, enc_steps, fine_steps, batch=131072, pool=4):
    """The two training phases of Sec. 5.1 on the training workload's material
    and decoder shape, with footprint-filtered data (a query at lod l stands
    for a Gaussian footprint of 2^l texels; its target BRDF and material
    parameters are means over up to 8 points of it): an encoder 4-32-32-8
    from the parameters (albedo RGB, roughness) to the latent, trained
    end-to-end with the decoder for `enc_steps` steps; the 1024^2 x 8 pyramid
    (11 levels) baked from it (coarse levels from 2x2-mean parameters); then
    `fine_steps` texel finetuning steps.  Against direct optimisation of the
    random texture for enc_steps + fine_steps steps on the same batches."""
    import torch

    import workloads as W
    from paper_2305_02678_gb300 import binding as B
    w = W.workload(4)
    m = w["model"]
    target = w["target"]
    enc = W.make_mlp(W.rng_streams(W.SEEDS[4] + 21, 1)[0], (4, 32, 32, 8))
    rng = W.rng_streams(W.SEEDS[4] + 22, 2)
    batches = []
    for _ in range(pool):
        q = W.uniform_queries(rng[0], batch, 10.0)
        y, a = W.filtered_targets(rng[1], target, q, w["W0"])
        batches.append(({k: torch.from_numpy(v).to(dev) for k, v in q.items() if k != "xi"},
                        torch.from_numpy(y).to(dev), torch.from_numpy(a).to(dev)))
    ta = torch.from_numpy(W.texel_attributes(target, w["W0"], w["H0"], w["L"])).to(dev)

    def every_100(s, last):
        return s % 100 == 0 or s == last or s == 1

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    mat = ctx.material(w["W0"], w["H0"], w["L"], w["pyramid"], m["frame"], m["decoder"], precision=B.NAM_PREC_F32,
                       trainable=True, encoder=enc)
    enc_losses = []
    for s in range(1, enc_steps + 1):
        dq, y, a = batches[s % pool]
        if s == 4:
            ev[0].record(stream)
        l = B.nam_train_step_encoded(ctx.h, mat.h, dq, a, y, batch, lr_params=1e-3, step=s, stream=stream,
                                     want_loss=every_100(s, enc_steps))
        if l is not None:
            enc_losses.append(l)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ev[2].record(stream)
    B.nam_encoder_bake(ctx.h, mat.h, ta, stream)
    ev[3].record(stream)
    fine_losses = []
    for s in range(1, fine_steps + 1):
        dq, y, _ = batches[s % pool]
        if s == 4:
            ev[4].record(stream)
        l = B.nam_train_step(ctx.h, mat.h, dq, y, batch, step=s, stream=stream, want_loss=every_100(s, fine_steps))
        if l is not None:
            fine_losses.append(l)
    ev[5].record(stream)
    torch.cuda.synchronize()
    enc_ms = ev[0].elapsed_time(ev[1]) / (enc_steps - 3)
    bake_ms = ev[2].elapsed_time(ev[3])
    fine_ms = ev[4].elapsed_time(ev[5]) / (fine_steps - 3)
    texels = mat.info.texels
    mat.destroy()
    # direct optimisation of the random texture on the same batches
    mat = ctx.material(w["W0"], w["H0"], w["L"], w["pyramid"], m["frame"], m["decoder"], precision=B.NAM_PREC_F32,
                       trainable=True)
    total = enc_steps + fine_steps
    direct = []
    for s in range(1, total + 1):
        dq, y, _ = batches[s % pool]
        l = B.nam_train_step(ctx.h, mat.h, dq, y, batch, step=s, stream=stream, want_loss=every_100(s, total))
        if l is not None:
            direct.append(l)
    mat.destroy()
    ctx.check()
    return {"workload": "encoder-bootstrap-1024sq-131072-filtered", "encoder": "4-32-32-8", "batch": batch,
            "encoder_steps": enc_steps, "encoder_ms_per_step": round(enc_ms, 4),
            "encoder_samples_per_s": round(batch * 1e3 / enc_ms, 1),
            "encoder_loss_every_100": [round(x, 5) for x in enc_losses],
            "bake_ms": round(bake_ms, 4), "bake_texels": texels,
            "finetune_steps": fine_steps, "finetune_ms_per_step": round(fine_ms, 4),
            "finetune_loss_every_100": [round(x, 5) for x in fine_losses],
            "direct_steps": total, "direct_loss_every_100": [round(x, 5) for x in direct],
            "note": "footprint-filtered targets and parameters; encoder phase: encoder kernel, fused forward + "
                    "loss + reverse mode with latents from the encoder, encoder reverse mode, Adam on frame, "
                    "decoder and encoder; bake: the encoder over every texel; finetuning and direct: the "
                    "training step of the training leg"}


def run_albedo_head(ctx, dev, stream, steps, batch=131072, pool=4, n_test=64, W0=256, L=9):
    """The optional albedo head (the paper's albedo inference) on the training
    workload's procedural material: a W0^2 x 8 pyramid (L levels, N(0, 0.1)),
    frame MLP 8-16-6 and a 14-64-64-6 decoder (RGB, then the albedo), trained
    with nam_train_step_albedo (log-L1 on the RGB plus the L2 albedo term
    against one-sample estimates pi f(x, wi, wo), wi cosine-weighted) on
    uniform lod-0 queries, so that every finest texel sees some 2,000 noisy
    albedo samples over 1,000 steps; reports the step time and the head's
    mean |albedo - Eq. 2| at n_test lod-0 points, the integral by a 96 x 96
    midpoint rule."""
    import torch

    import workloads as W
    from paper_2305_02678_gb300 import binding as B
    target = W.workload(4, scale=1 / 262144)["target"]
    rng = W.rng_streams(W.SEEDS[4] + 31, 4)
    pyr = W.make_pyramid(rng[0], W0, W0, L, dtype=np.float32, std=0.1)
    model = W.make_model(rng[0], (14, 64, 64, 6), (8, 16, 6))
    batches = []
    for _ in range(pool):
        q = W.uniform_queries(rng[1], batch, 0.0)
        batches.append(({k: torch.from_numpy(v).to(dev) for k, v in q.items()},
                        torch.from_numpy(W.target_rgb(target, q)).to(dev),
                        torch.from_numpy(W.albedo_targets(rng[2], target, q)).to(dev)))
    tq = W.uniform_queries(rng[3], n_test, 0.0)
    k = 96
    s_, p_ = np.meshgrid((np.arange(k) + 0.5) / k, (np.arange(k) + 0.5) / k * 2 * np.pi, indexing="ij")
    ct, st = np.sqrt(s_.ravel()), np.sqrt(1 - s_.ravel())
    wi = np.stack([st * np.cos(p_.ravel()), st * np.sin(p_.ravel()), ct])
    ref = np.zeros((n_test, 3))
    for j in range(n_test):
        wo = np.repeat(np.array([[tq["wox"][j]], [tq["woy"][j]], [tq["woz"][j]]], np.float64), k * k, axis=1)
        f = target(np.full(k * k, float(tq["u"][j])), np.full(k * k, float(tq["v"][j])), wi, wo)
        ref[j] = np.pi * f.mean(axis=0)
    dtq = {kk: torch.from_numpy(v).to(dev) for kk, v in tq.items()}
    mat = ctx.material(W0, W0, L, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F32, trainable=True)

    def albedo_error():
        _, a = mat.eval_albedo(dtq, stream=stream)
        return float(np.mean(np.abs(a.cpu().numpy() - ref)))

    e0 = albedo_error()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    losses = []
    for s in range(1, steps + 1):
        dq, y, ya = batches[s % pool]
        if s == 4:
            ev[0].record(stream)
        l = B.nam_train_step_albedo(ctx.h, mat.h, dq, y, ya, batch, lr_params=3e-3, lr_pyramid=1e-2, step=s,
                                    stream=stream, want_loss=(s % 100 == 0 or s == 1 or s == steps))
        if l is not None:
            losses.append(l)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / (steps - 3)
    e1 = albedo_error()
    mat.destroy()
    ctx.check()
    return {"workload": f"albedo-head-{W0}sq-{batch}-lod0", "decoder": "14-64-64-6", "batch": batch, "steps": steps,
            "ms_per_step": round(ms, 4), "samples_per_s": round(batch * 1e3 / ms, 1),
            "loss_every_100": [round(x, 5) for x in losses],
            "albedo_mean_abs_error": {"before": round(e0, 4), "after": round(e1, 4),
                                      "reference_mean": round(float(ref.mean()), 4), "points": n_test},
            "note": "one fused kernel for forward, both losses and reverse mode (six outputs), then Adam; "
                    "error against a 96 x 96 midpoint quadrature of Eq. 2 at lod 0"}


def _host_cpu_counters():
    """Process context switches and, where the container exposes them, the
    cgroup's CPU-quota throttling counters (cgroup v2 cpu.stat)."""
    import resource
    ru = resource.getrusage(resource.RUSAGE_SELF)
    out = {"voluntary_csw": ru.ru_nvcsw, "involuntary_csw": ru.ru_nivcsw}
    try:
        with open("/sys/fs/cgroup/cpu.stat") as f:
            for line in f:
                k, v = line.split()
                if k in ("nr_periods", "nr_throttled", "throttled_usec"):
                    out[k] = int(v)
        with open("/sys/fs/cgroup/cpu.max") as f:
            out["cpu_max"] = f.read().strip()
    except OSError:
        pass
    return out


def run_serving(device, n_frames, rate=240.0, n_mat=16, budget=40 << 30, warmup_frames=None, repeats=4,
                lead_s=0.1, trace=None):
    """Serving stream: Poisson frame arrivals at `rate`/s, resolutions drawn
    from 720p/1080p/1440p/2160p, 16 FP16 materials (own 2048^2 x 8 pyramid
    and 14-64-64-3 decoder each), one material per 64x64 tile drawn
    uniformly, frames admitted under a 40 GB budget, `repeats` streams back to
    back in one context.  Frames go through nam_submit with pinned host inputs
    up to `lead_s` ahead of their arrival times; the library holds each until
    it arrives, so the driver's own timing does not enter the latency
    (finish - arrival).  The first `warmup_frames` (default 10%) of each
    stream are excluded from its percentiles.  Every frame's timeline is
    split into: release (arrival -> admission), gpu_wait (start of enqueue ->
    first copy on the device), h2d, kernel, d2h and observe (RGB in host
    memory -> completion seen by the serving thread)."""
    import ctypes as C

    import torch

    import workloads as W
    from paper_2305_02678_gb300 import Context
    from paper_2305_02678_gb300 import binding as B

    if warmup_frames is None:
        warmup_frames = max(1, n_frames // 10)
    total = n_frames + warmup_frames
    rngs = W.rng_streams(W.SEEDS[5], 2 * n_mat + 3 + repeats)
    ctx = Context(device, hbm_budget_bytes=budget, serve_streams=4, serve_queue_depth=4096)
    mats = []
    for k in range(n_mat):
        pyr = W.make_pyramid(rngs[k], 2048, 2048, 12, dtype=np.float16)
        model = W.make_model(rngs[n_mat + k], (14, 64, 64, 3), (8, 16, 6))
        mats.append(ctx.material(2048, 2048, 12, pyr, model["frame"], model["decoder"], precision=B.NAM_PREC_F16))
    mat_arr = (C.c_void_p * n_mat)(*[m.h for m in mats])
    res = [(1280, 720), (1920, 1080), (2560, 1440), (3840, 2160)]
    frames = []
    for (wd, ht) in res:
        q = W.warp_queries(rngs[2 * n_mat], wd, ht, 2048, 2048, order="tile")
        pinned = {k: torch.from_numpy(v).pin_memory() for k, v in q.items() if k != "xi"}
        out = torch.empty((wd * ht, 3), dtype=torch.float32).pin_memory()
        tiles = W.tile_ranges(wd, ht)
        frames.append((wd * ht, pinned, out, tiles))
    runs = [_serving_stream(B, C, ctx, mats, mat_arr, frames, rngs[2 * n_mat + 1 + r], total, warmup_frames, rate,
                            n_mat, lead_s) for r in range(repeats)]
    # the same streams with the frames' queries and RGB in device memory (a
    # renderer's G-buffer): no host link in the loop
    dframes = [(n, {k: v.to(f"cuda:{device}") for k, v in pinned.items()},
                torch.empty((n, 3), device=f"cuda:{device}"), tiles) for n, pinned, _, tiles in frames]
    druns = [_serving_stream(B, C, ctx, mats, mat_arr, dframes, rngs[2 * n_mat + 1 + r], total, warmup_frames, rate,
                             n_mat, lead_s, flags=B.NAM_FRAME_DEVICE) for r in range(repeats)]
    for m in mats:
        m.destroy()
    ctx.close()
    if trace:
        # columns: resolution index, arrival, submit, admit, start, enqueued, gpu begin, kernel begin, kernel end,
        # gpu end, finish (s), queries, slot, in flight at admission; one array per stream
        np.savez(trace, **{f"run{r}": x.pop("_rows") for r, x in enumerate(runs)},
                 **{f"device_run{r}": x.pop("_rows") for r, x in enumerate(druns)})
    for x in runs + druns:
        x.pop("_rows", None)
    out = dict(runs[0])
    out.update({"frames": n_frames, "warmup_frames": warmup_frames, "rate_fps": rate, "materials": n_mat,
                "budget_bytes": budget, "repeats": repeats, "submit_lead_ms": lead_s * 1e3,
                "resident_bytes_materials": int(sum(m.info.resident_bytes for m in mats)),
                "p50_frame_ms_runs": [r["p50_frame_ms"] for r in runs],
                "p99_frame_ms_runs": [r["p99_frame_ms"] for r in runs],
                "p99_spread": round(max(r["p99_frame_ms"] for r in runs) / min(r["p99_frame_ms"] for r in runs), 3),
                "runs": runs[1:],
                "device_frames": {
                    "p50_frame_ms_runs": [r["p50_frame_ms"] for r in druns],
                    "p99_frame_ms_runs": [r["p99_frame_ms"] for r in druns],
                    "p99_spread": round(max(r["p99_frame_ms"] for r in druns) / min(r["p99_frame_ms"] for r in druns), 3),
                    "evals_per_s_runs": [r["evals_per_s"] for r in druns],
                    "breakdown": druns[0]["breakdown"], "slowest_frames": druns[0]["slowest_frames"],
                    "note": "NAM_FRAME_DEVICE: queries and RGB in device memory, only the work table is uploaded"},
                "latency": "finish - scheduled Poisson arrival on the nam_now() clock; host->device copy of the "
                           "frame's inputs, kernel and device->host copy of its RGB included"})
    return out

def _serving_stream(B, C, ctx, mats, mat_arr, frames, rng, total, warmup_frames, rate, n_mat, lead_s, flags=0):
    """One Poisson stream of `total` frames through nam_submit; see run_serving."""
    arrivals = np.cumsum(rng.exponential(1.0 / rate, total))
    which = rng.integers(0, len(frames), total)
    # every frame's tile -> material table, built before the stream starts
    tables = []
    for i in range(total):
        st = np.array(frames[which[i]][3], dtype=np.int64)
        arr = np.zeros(len(st), dtype=[("start", "<i8"), ("count", "<i4"), ("material", "<i4")])
        arr["start"], arr["count"], arr["material"] = st[:, 0], st[:, 1], rng.integers(0, n_mat, len(st))
        tables.append(arr)
    cpu0 = _host_cpu_counters()
    tickets = []
    t0 = B.nam_now() + lead_s + 0.02
    for i in range(total):
        n, pinned, out, _ = frames[which[i]]
        items = tables[i]
        f = B.nam_frame()
        f.n_queries = n
        f.q = B.make_queries(pinned)
        f.items = items.ctypes.data
        f.n_items = len(items)
        f.n_materials = n_mat
        f.materials = C.addressof(mat_arr)
        f.rgb_out = out.data_ptr()
        f.flags = flags
        f.arrival_s = t0 + arrivals[i]
        ahead = f.arrival_s - lead_s - B.nam_now()
        if ahead > 0:
            time.sleep(ahead)
        tickets.append(B.nam_submit(ctx.h, f))
    failed = 0
    rows = []
    for i, t in enumerate(tickets):
        st, fs = B.nam_wait(ctx.h, t, 60_000_000_000)
        failed += st != 0
        if i >= warmup_frames and st == 0:
            rows.append((which[i], fs.arrival_s, fs.submit_s, fs.admit_s, fs.start_s, fs.enqueued_s, fs.gpu_begin_s,
                         fs.gpu_kernel_begin_s, fs.gpu_kernel_end_s, fs.gpu_end_s, fs.finish_s, fs.n_queries,
                         fs.slot, fs.in_flight_at_admit))
    cpu1 = _host_cpu_counters()
    a = np.array(rows, dtype=np.float64)
    arr_s, sub_s, adm_s, sta_s, enq_s, gb_s, kb_s, ke_s, ge_s, fin_s = (a[:, k] for k in range(1, 11))
    lat = (fin_s - arr_s) * 1e3
    span = fin_s.max() - arr_s.min()
    timed = gb_s > 0
    parts = {"release": adm_s - arr_s, "enqueue": enq_s - sta_s, "gpu_wait": gb_s - sta_s, "h2d": kb_s - gb_s,
             "kernel": ke_s - kb_s, "d2h": ge_s - ke_s, "observe": fin_s - ge_s}

    def pct(x, p):
        return round(float(np.percentile(x, p)), 3) if len(x) else None

    breakdown = {k: {"p50_ms": pct(v[timed] * 1e3, 50), "p99_ms": pct(v[timed] * 1e3, 99),
                     "max_ms": round(float(v[timed].max() * 1e3), 3) if timed.any() else None}
                 for k, v in parts.items()}
    slow = np.argsort(lat)[-5:]
    by_res = {}
    for k, (n, *_rest) in enumerate(frames):
        sel = a[:, 0] == k
        by_res[str(n)] = {"frames": int(sel.sum()), "p50_ms": pct(lat[sel], 50), "p99_ms": pct(lat[sel], 99)}
    return {"failed": int(failed), "p50_frame_ms": pct(lat, 50), "p99_frame_ms": pct(lat, 99),
            "max_frame_ms": round(float(lat.max()), 3),
            "breakdown": breakdown,
            "slowest_frames": [{"queries": int(a[j, 11]), "slot": int(a[j, 12]), "in_flight_at_admit": int(a[j, 13]),
                                "submit_ahead_ms": round(float((arr_s[j] - sub_s[j]) * 1e3), 3),
                                **{k: round(float(v[j] * 1e3), 3) for k, v in parts.items()},
                                "total_ms": round(float(lat[j]), 3)} for j in slow],
            "submit_ahead_ms_min": round(float((arr_s - sub_s).min() * 1e3), 3),
            "evals_per_s": round(float(a[:, 11].sum() / span), 1),
            "offered_evals_per_s": round(rate * float(np.mean([f[0] for f in frames])), 1),
            "by_queries": by_res, "_rows": a,
            "host_cpu": {k: (cpu1[k] - cpu0[k]) if isinstance(cpu0.get(k), int) else cpu1[k] for k in cpu1}}


def _oracle_rate(O, om, q, nthreads, seconds, k0=16384):
    """evals/s of the FP64 oracle over consecutive chunks of k0 queries of q
    (from the start, wrapping around), about `seconds` of work; returns
    (rate, queries, seconds)."""
    import workloads as W
    n_total = int(q["u"].shape[0])
    k = min(k0, n_total)
    done, dt, start = 0, 0.0, 0
    while dt < seconds or done == 0:
        c = min(k, n_total - start)
        sub = W.slice_queries(q, start, c)
        t0 = time.perf_counter()
        O.eval(om, sub, nthreads=nthreads)
        dt += time.perf_counter() - t0
        done += c
        start = (start + c) % n_total
    return done / dt, done, dt


def _graded(O, g, o, kappa, tol, gain=None):
    """The graded parity of a GPU result g against oracle values o: max
    relative error (tau = RMS of o) with the bound on kappa <= 50, and what
    the conditioning-aware bound (frame error times the decoder's direction
    gain) covers beyond."""
    ok, st = O.parity(g, o, kappa, tol, gain=gain)
    n_ill = st["ill_conditioned"]
    return {"bound": tol, "pass": ok, "max_kappa_le_50": st["max_rel_well_conditioned"], "max": st["max_rel"],
            "mean": st["mean_rel"], "worst_over_bound": round(st["worst_over_bound"], 4),
            "kappa_gt_50": {"queries": n_ill, "share": round(n_ill / max(st["n"], 1), 5),
                            "max": st["max_rel_ill_conditioned"]}}


def cpu_baseline(w, gpu_out16, seconds, gpu_out8=None, outs4k=None):
    """FP64 oracle (as it stands) on the host cores over bounded samples of
    the workloads: the 1080p frame (the headline, all cores), and at all
    cores and one thread the 1080p frame, the 65,536-query FP32 workload and
    the 4K frame (when the 4K sweep ran); also the GPU results' graded errors
    against the oracle on the first queries of the frames."""
    import oracle.oracle as O
    import workloads as W
    O.build()
    cores = os.cpu_count() or 1
    om = O.Model.from_workload(w, params="fp16")
    q = w["queries"]
    rate, done, dt = _oracle_rate(O, om, q, cores, 0.5 * seconds, k0=65536)
    timings = {"1920x1080 fp16 params": {"threads_all": round(rate, 1)}}
    r1, _, _ = _oracle_rate(O, om, q, 1, 0.15 * seconds, k0=4096)
    timings["1920x1080 fp16 params"]["threads_1"] = round(r1, 1)
    w1 = W.workload(1)
    om1 = O.Model.from_workload(w1)
    timings["65536q fp32 (256^2 x 9, 14-32-32-3)"] = {
        "threads_all": round(_oracle_rate(O, om1, w1["queries"], cores, 0.1 * seconds, k0=65536)[0], 1),
        "threads_1": round(_oracle_rate(O, om1, w1["queries"], 1, 0.05 * seconds, k0=4096)[0], 1)}
    if outs4k is not None:
        w4 = outs4k["w"]
        om4 = O.Model.from_workload(w4, params="fp16")
        timings["3840x2160 fp16 params"] = {
            "threads_all": round(_oracle_rate(O, om4, w4["queries"], cores, 0.1 * seconds, k0=65536)[0], 1),
            "threads_1": round(_oracle_rate(O, om4, w4["queries"], 1, 0.1 * seconds, k0=4096)[0], 1)}
    # graded errors on the first 200,000 queries of the 1080p frame
    c = min(200000, int(q["u"].shape[0]))
    sub = W.slice_queries(q, 0, c)
    ref = O.eval(om, sub, nthreads=cores)
    kappa = O.frame_condition(om, sub)
    master = O.eval(O.Model.from_workload(w), sub, nthreads=cores)
    e_master = O.relative_error(gpu_out16[:c], master)
    err16 = {"queries": c, "vs_oracle_fp16_params_fp64_activations": _graded(O, gpu_out16[:c], ref, kappa, 2e-3,
                                                                              O.band_gain(om, sub, kappa)),
             "vs_fp32_master_oracle_max": e_master[0], "vs_fp32_master_oracle_mean": e_master[1]}
    fp8 = None
    if gpu_out8 is not None:
        om8 = O.Model.from_workload(w, params="fp8")
        ref8 = O.eval(om8, sub, nthreads=cores)
        e8m = O.relative_error(gpu_out8[:c], master)
        fp8 = {"queries": c, "vs_oracle_fp8_params_fp64_activations": _graded(O, gpu_out8[:c], ref8, kappa, 3e-2,
                                                                             O.band_gain(om8, sub, kappa)),
               "vs_fp32_master_oracle_max": e8m[0], "vs_fp32_master_oracle_mean": e8m[1]}
    err4k = None
    if outs4k is not None:
        w4, k4 = outs4k["w"], outs4k["sample"]
        sub4 = W.slice_queries(w4["queries"], 0, k4)
        om4m = O.Model.from_workload(w4)
        master4 = O.eval(om4m, sub4, nthreads=cores)
        kappa4 = O.frame_condition(om4m, sub4)
        err4k = {"queries": k4}
        for name, g in outs4k["out"].items():
            if name == "fp32":
                err4k["fp32_vs_oracle_fp32_params"] = _graded(O, g, master4, kappa4, 1e-5,
                                                              O.band_gain(om4m, sub4, kappa4))
            else:
                om4 = O.Model.from_workload(w4, params=name)
                o4 = O.eval(om4, sub4, nthreads=cores)
                err4k[f"{name}_vs_oracle_{name}_params_fp64_activations"] = _graded(
                    O, g, o4, kappa4, 2e-3 if name == "fp16" else 3e-2, O.band_gain(om4, sub4, kappa4))
                e = O.relative_error(g, master4)
                err4k[f"{name}_vs_fp32_master_oracle"] = {"max": e[0], "mean": e[1]}
    return {"value": round(rate, 1), "unit": "evals/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} queries: the 1920x1080 workload's queries in order, wrapping around "
                      f"(FP64, FP16-quantised parameters, {cores} threads)",
            "seconds": round(dt, 2), "timings_evals_per_s": timings,
            "gpu_fp16_error": err16, "gpu_fp8_error": fp8, "gpu_error_3840x2160_sample": err4k}


# ----------------------------------------------------------------------------
# reference arm: the FP64 oracle timed on the host cores
# ----------------------------------------------------------------------------
def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle.oracle as O
    import workloads as W
    O.build()
    w = workload()
    om = O.Model.from_workload(w, params="fp16")
    cores = os.cpu_count() or 1
    q = w["queries"]
    n_total = int(q["u"].shape[0])
    # each step: a bounded contiguous sample of the workload, cycling through it
    k = 1 << 17
    for i in range(args.warmup):
        O.eval(om, W.slice_queries(q, (i * k) % (n_total - k), k), nthreads=cores)
    times = []
    for i in range(args.steps):
        s = (i * k) % (n_total - k)
        sub = W.slice_queries(q, s, k)
        t0 = time.perf_counter()
        O.eval(om, sub, nthreads=cores)
        times.append(time.perf_counter() - t0)
    ms = statistics.fmean(times) * 1e3
    v = k / (ms * 1e-3)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "queries_per_step": k, "sample": "131072 consecutive queries per step"},
        "cpu_baseline": {"value": round(v, 1), "unit": "evals/s", "cores": cores, "kind": "oracle",
                         "sample": "131072-query slices of the 1920x1080 workload, FP64 oracle, all host cores"},
        "e2e": {"value": round(v, 1), "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
