"""Benchmark of the space-variant elliptical box-spline filter on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = the whole hot path over one synthetic 2048x2048 uint8 image with
a per-pixel (sigma, rho, theta) field (sigma 1-32 px, rho 1-8, theta from a
smooth vector field), N = 4 directions: the per-pixel scale map (Sec. 3.2.2),
the pre-integration (Algorithm 1 step 2) and the 16-tap finite difference
with Zwart-Powell interpolation (Algorithm 1 step 3), through the C ABI call
bsf_filter.  Inputs are resident in HBM before the timed region; between
timed steps a 512 MiB buffer is written to flush the 129 MB L2.

For N > 1 (torchrun), each rank runs an independent replica on its own GPU
(the path has no exchange step); value = pixels of all ranks / max time.

--impl reference times the FP64 CPU oracle (Algorithm 1 restated, single
thread) on a bounded crop of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "u2048_u8_n4"
METRIC = "Gpixels/s filtered (N=4,6) at ≤1e-5 rel err vs FP64 oracle; % HBM roofline; p50/p99"
SIGMA_MAX = 32.0
# algorithmic 32-bit integer operations per output pixel of the exact stencil,
# counted from its formulation per tap: 56 for the 28 64-bit additions of the
# nine-point ZP combinations, 22 for the eleven 64x32-bit products, 14 for the
# 64-bit sums of the products and the three tap accumulators, 11 for tap
# offset, cell index and the two truncations, 15 for bounds and clamping,
# 6 for addresses: 124 per tap, 16 taps
STENCIL_INT_OPS_PER_PX = 16 * 124
# the same count for the 128-bit fixed-point stencil (float32 images): four
# 32-bit words per addition (112), eight 32x32 partial products per 128x32
# product (88), two words per product sum and accumulator (28), 32 for
# position, truncation, bounds and addresses: 260 per tap
STENCIL_INT_OPS_PER_PX_U128 = 16 * 260
# six directions: 64 taps x 24 lattice points x 15 coefficients x 5 twenty-bit limbs,
# one int32 multiply-add each
HEX6_IMAD_PER_PX = 64 * 24 * 15 * 5
# Benchmarked workloads: (params kind, largest sigma or scale, forward+backward).
BENCH_WORKLOADS = {
    "u2048_u8_n4": ("srt", 32.0, False),
    "u2048_f32_n4": ("srt", 32.0, False),
    "b4c3_4096_f32_n4": ("srt", 48.0, False),
    "b4c3_4096_f32_n6": ("srt", 48.0, False),
    "b8_1024_f32_scales": ("scales", 24.0, True),
}
WORKLOAD_TEXT = {
    "u2048_u8_n4": "2048x2048 u8 image (uniform 0-255), N=4, per-pixel (sigma 1-32 px, rho 1-8 clamped to "
                   "Prop. 3.1, theta from a smooth vector field), exact int64 path",
    "u2048_f32_n4": "2048x2048 f32 copy of the u8 image, N=4, sigma 1-32 px, rho 1-8, theta from a smooth "
                    "vector field, exact 128-bit fixed-point path",
    "b4c3_4096_f32_n4": "batch 4 x 3 channels x 4096x4096 f32 (uniform + 3 gratings), sigma 2-48 px, rho 1-6, "
                        "theta uniform, filtered with N=4, exact 128-bit fixed-point path",
    "b4c3_4096_f32_n6": "batch 4 x 3 channels x 4096x4096 f32 (uniform + 3 gratings), sigma 2-48 px, rho 1-6, "
                        "theta uniform, N=6 (64-tap stencil) on the hexagonal lattice of spacing 0.5 px, FP64",
    "b8_1024_f32_scales": "batch 8 x 1024x1024 f32, learnable scale field a_k in [1,24]; one step = forward "
                          "filter + backward (gradients for image and scales)",
}
STENCIL_SOURCES = ["paper_1003_2022_gb300/csrc/stencil4.cu", "paper_1003_2022_gb300/csrc/map4.cuh",
                   "paper_1003_2022_gb300/csrc/bsf_common.cuh"]


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.lines: list[tuple[float, str]] = []
        self.gpu = gpu_index
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = [ln for (t, ln) in self.lines if self.t0 is not None and self.t0 - 0.15 <= t <= self.t1 + 0.15]
        if not rows:
            rows = [ln for (_, ln) in self.lines[-3:]]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in rows:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(ms: float, device=None) -> float:
    """The largest of the ranks' timed-region durations (the job's time when
    independent replicas run one per GPU); the local value without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_value(units_per_rank: float, ms_max: float, world_size: int) -> float:
    """Whole-job throughput of replicas: the units all ranks processed / the max time."""
    return world_size * units_per_rank / (ms_max / 1e3)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def stencil_traffic():
    """DRAM bytes per launch of the stencil from the committed ncu record, or None
    if the kernel's sources changed since that capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            rec = json.load(fh)["k_stencil4_exact<u64,SRT>"]
        h = hashlib.sha256()
        for f in STENCIL_SOURCES:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest()[:16] != rec["sources_sha256_16"]:
            return None
        return rec["bytes_per_launch"]
    except Exception:
        return None


def alu_peak_tops():
    """Issue-rate bound of 32-bit integer ALU work: 152 SMs x 128 lanes x max SM clock."""
    return 152 * 128 * 2.070e9 / 1e12


def _inputs(size=None, workload=WORKLOAD):
    """(B, C, H, W) image and (B, K, H, W) parameter planes of a workload."""
    from paper_1003_2022_gb300 import synth
    if synth.WORKLOADS[workload]["B"] == 1 and "scales" not in synth.WORKLOADS[workload]:
        f, p = synth.workload_inputs(workload, seed=0, H=size, W=size)
        return f[None, None], p[None]
    return synth.batch_inputs(workload, seed=0, H=size, W=size)


def cpu_baseline_run(f, p, crop=192, seed=0):
    """The oracle (Algorithm 1 restated in FP64/int64, scale map in FP64) on a
    crop of the workload; returns (pixels/s, seconds, description)."""
    import oracle
    H, W = f.shape
    rng = np.random.default_rng(seed)
    y0 = int(rng.integers(0, H - crop))
    x0 = int(rng.integers(0, W - crop))
    fc = np.ascontiguousarray(f[y0:y0 + crop, x0:x0 + crop])
    pc = np.ascontiguousarray(p[:, y0:y0 + crop, x0:x0 + crop]).astype(np.float64)
    P = int(np.ceil(0.5 * 8.364 * SIGMA_MAX)) + 4
    t = time.perf_counter()
    a, _ = oracle.map4(pc, oracle.KIND_SRT)
    out, bad = oracle.alg1_filter4(fc.astype(np.int64), a, P, integer=True)
    dt = time.perf_counter() - t
    desc = (f"oracle map4 + preint4_i64 + stencil4 (FP64 ZP weights from the exact box spline), "
            f"single thread, one {crop}x{crop} crop of the 2048x2048 workload")
    return crop * crop / dt, dt, desc


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    f, p = _inputs()
    f, p = f[0, 0], p[0]
    import oracle
    oracle.build()
    for i in range(args.warmup):
        cpu_baseline_run(f, p, crop=48, seed=1000 + i)
    tot_px, tot_s = 0, 0.0
    for i in range(args.steps):
        v, dt, desc = cpu_baseline_run(f, p, crop=64, seed=i)
        tot_px += 64 * 64
        tot_s += dt
    value = tot_px / tot_s / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gpixels/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": "2048x2048 u8 image, N=4, sigma 1-32 px, rho 1-8, "
                                                    "theta from a smooth vector field; one 64x64 crop per step",
                                        "parallelism": "replicas"},
        "cpu_baseline": {"value": value, "unit": "Gpixels/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} crops of 64x64 px (one per step)"},
        "e2e": {"value": value, "unit": "Gpixels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local if ws > 1 else 0}")
    torch.cuda.set_device(dev)
    from paper_1003_2022_gb300 import _lib as L
    from paper_1003_2022_gb300 import api

    from paper_1003_2022_gb300 import synth as _synth
    kind_name, smax, train = BENCH_WORKLOADS[args.workload]
    N = _synth.WORKLOADS[args.workload]["N"]
    f_np, p_np = _inputs(args.size, args.workload)
    B, C, H, W = f_np.shape
    u8 = f_np.dtype == np.uint8
    dtype = L.BSF_U8 if u8 else L.BSF_F32
    kind = L.BSF_PARAM_SRT if kind_name == "srt" else L.BSF_PARAM_SCALES
    f = torch.from_numpy(f_np).to(dev)
    p = torch.from_numpy(p_np).to(dev)
    out = torch.empty((B, C, H, W), dtype=torch.float32, device=dev)
    if train:
        gout = torch.from_numpy(np.random.default_rng(3).standard_normal((B, C, H, W)).astype(np.float32)).to(dev)
        gimg = torch.empty((B, C, H, W), dtype=torch.float32, device=dev)
        gsc = torch.empty_like(p)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    ctx = api.context(dev)
    opts = api.make_opts("exact" if args.precision == "exact" else "fp64", max_scale=smax)
    stream = torch.cuda.current_stream(dev)
    sptr = int(stream.cuda_stream)

    def step(img=f, prm=p, o=out):
        rc = L.bsf_filter(ctx, img.data_ptr(), dtype, B, C, H, W, N, prm.data_ptr(), kind, opts, o.data_ptr(), sptr)
        if rc != 0:
            raise L.BsfError(rc, "bsf_filter")
        if train:
            rc = L.bsf_filter_backward(ctx, img.data_ptr(), dtype, B, C, H, W, 4, prm.data_ptr(), gout.data_ptr(),
                                       gimg.data_ptr(), gsc.data_ptr(), opts, sptr)
            if rc != 0:
                raise L.BsfError(rc, "bsf_filter_backward")

    for _ in range(args.warmup):
        flush.fill_(1)
        step()
    torch.cuda.synchronize(dev)
    if api.device_status(dev) & ~(1 << L.BSF_EINFEASIBLE):
        raise RuntimeError("device status error during warm-up")

    sampler = ClockSampler(dev.index if ws == 1 else local)
    sampler.start()
    time.sleep(0.3)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.t0 = time.time()
    L.bsf_profile_begin(ctx)
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize(dev)
    sampler.t1 = time.time()
    ms_pre, ms_st, nl = L.bsf_profile_end(ctx)
    if ws > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    t_max = max_over_ranks(total_ms, dev)
    time.sleep(0.25)
    sampler.stop()
    clocks = sampler.summary()

    # end to end: pinned host buffers; every step copies its inputs in and its result(s) out
    f_h = torch.from_numpy(f_np).pin_memory()
    p_h = torch.from_numpy(p_np).pin_memory()
    o_h = torch.empty((B, C, H, W), dtype=torch.float32).pin_memory()
    e2e_steps = max(3, min(args.steps, 50))
    d2h = out.numel() * 4
    if train:
        # forward + backward: H2D of image and field, the two calls, D2H of output and gradients
        f_d = torch.empty_like(f)
        p_d = torch.empty_like(p)
        gi_h = torch.empty_like(o_h)
        gs_h = torch.empty(tuple(p.shape), dtype=torch.float32).pin_memory()
        d2h += gimg.numel() * 4 + gsc.numel() * 4

        def e2e_step():
            f_d.copy_(f_h, non_blocking=True)
            p_d.copy_(p_h, non_blocking=True)
            step(f_d, p_d, out)
            o_h.copy_(out, non_blocking=True)
            gi_h.copy_(gimg, non_blocking=True)
            gs_h.copy_(gsc, non_blocking=True)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        torch.cuda.synchronize(dev)
        e2e_ms = 1e3 * (time.perf_counter() - t0)
        e2e_how = "torch copies + bsf_filter + bsf_filter_backward on one stream"
    else:
        # bsf_filter_host: the library's host-buffer entry point, copies of one step
        # overlapping the kernels of the previous one
        def e2e_step():
            rc = L.bsf_filter_host(ctx, f_h.data_ptr(), dtype, B, C, H, W, N, p_h.data_ptr(), kind, opts,
                                   o_h.data_ptr())
            if rc != 0:
                raise L.BsfError(rc, "bsf_filter_host")

        for _ in range(2):
            e2e_step()
        L.check(L.bsf_host_sync(ctx), "bsf_host_sync")
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        L.check(L.bsf_host_sync(ctx), "bsf_host_sync")
        e2e_ms = 1e3 * (time.perf_counter() - t0)
        e2e_how = "bsf_filter_host (host buffers, pipelined across steps), host wall clock"
    status = api.device_status(dev)
    if status & ~(1 << L.BSF_EINFEASIBLE):
        raise RuntimeError(f"device status error {status}")

    npx = B * C * H * W
    value = replicas_value(npx * args.steps, t_max, ws) / 1e9
    e2e_value = ws * npx * e2e_steps / (e2e_ms / 1e3) / 1e9
    # stencil launches in the timed region (one per strip and batch chunk of each forward call)
    n_st = max(nl, 1)
    st_ms = ms_st / n_st
    ops_px = STENCIL_INT_OPS_PER_PX if u8 else STENCIL_INT_OPS_PER_PX_U128
    px_per_launch = npx * args.steps / n_st
    achieved = ops_px * px_per_launch / (st_ms / 1e3) / 1e12
    peak = alu_peak_tops()
    traffic = stencil_traffic() if (args.workload == WORKLOAD and args.size in (None, 2048)
                                    and args.precision == "exact") else None
    kname = f"k_stencil4_exact<{'u64' if u8 else 'u128'},{kind_name.upper()}>"
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": kname,
                "kernel_ms": st_ms, "preintegrate_ms": ms_pre / n_st,
                "peak_note": "152 SMs x 128 lanes x 2070 MHz, 32-bit integer ops (derived; an add-chain probe "
                             "reached 37.1 Tops/s, a multiply-add chain 19.1 Tops/s)",
                "int_ops_per_px": ops_px,
                "algorithmic_bytes_per_launch": int((12 + 4 + 8 * (1 if u8 else 2)) * px_per_launch)}
    # the HBM side of both kernels, against the measured copy bandwidth
    peaks, peak_src = _peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    P = api.halo_for(smax, kind_name)
    elem = 8 if (u8 or args.precision != "exact") else 16
    nstrip_one = (W + 2 * P) <= (4096 if elem == 8 else 3072)
    pre_bytes = (H + 2 * P) * (W + 2 * P) * ((1 if u8 else 4) + elem) * B * C if nstrip_one else None
    pre_ms = ms_pre / n_st
    roofline["hbm"] = {
        "peak_gbs": hbm_peak, "peak_source": peak_src,
        "stencil_dram_gbs": traffic / (st_ms * 1e6) if traffic else None,
        "stencil_frac": traffic / (st_ms * 1e6) / hbm_peak if traffic else None,
        "preintegrate_algorithmic_bytes": pre_bytes,
        "preintegrate_gbs": pre_bytes / (pre_ms * 1e6) if pre_bytes else None,
        "preintegrate_frac": pre_bytes / (pre_ms * 1e6) / hbm_peak if pre_bytes else None,
    }
    if args.precision != "exact":
        roofline["kernel"] = f"k_stencil4_f64<{kind_name.upper()}>"
        roofline["note"] = "all-FP64 form: the integer op count does not apply; compare kernel_ms"
    # kernels per forward call: 7 for the pre-integration and 1 stencil per strip/chunk; the
    # backward adds the gradient stencil and its scans
    launches = 8 * nl
    if train:
        # per batch chunk: 7 pre-integration kernels, the scale-gradient and scatter kernels,
        # 4 transposed scans
        P = api.halo_for(smax, kind_name)
        per = (H + 2 * P) * (W + 2 * P) * ((8 if u8 else 16) + 8) * C
        chunks = -(-B // max(1, min(B, (16 << 30) // per)))
        launches += 13 * chunks * args.steps
    if N == 6:
        # six directions: the stencil's exact integer part is 64 taps x 24 lattice points x 15
        # coefficients, each the product of a small integer coefficient and a 96-bit window
        # value in five 20-bit limbs (5 int32 multiply-adds into 32-bit sums), against the
        # int32 multiply-add rate (152 SMs x 64 per clock x 2070 MHz)
        ops_px6 = HEX6_IMAD_PER_PX
        achieved6 = ops_px6 * px_per_launch / (st_ms / 1e3) / 1e12
        peak6 = 152 * 64 * 2.070e9 / 1e12
        roofline = {"bound": "alu", "achieved": achieved6, "peak": peak6, "unit": "Tops/s",
                    "frac": achieved6 / peak6, "traffic": None, "kernel": "k_hex6_stencil",
                    "kernel_ms": st_ms, "preintegrate_ms": ms_pre / n_st,
                    "peak_note": "int32 multiply-add rate, 152 SMs x 64 per clock x 2070 MHz (derived; a "
                                 "multiply-add chain probe reached 19.1 Tops/s); int32 multiply-adds of the exact "
                                 "coefficient sums, 64 taps x 24 points x 15 coefficients x 5 twenty-bit limbs",
                    "int_madds_per_px": ops_px6,
                    "launches_per_step": n_st / args.steps,
                    "preintegrate_note": "scale map + window transfer and six exact running sums, per chunk"}
        launches = args.steps + 2 * nl
    line = {
        "metric": METRIC, "value": value, "unit": "Gpixels/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if N == 6 else (("int64" if u8 else "int128") if args.precision == "exact" else "f64"),
        "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload] if args.size is None else
                   f"{WORKLOAD_TEXT[args.workload]} (resized to {H}x{W})",
                   "workload_id": args.workload,
                   "precision": args.precision, "l2": "flushed between timed steps (512 MiB write)",
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99))},
        "roofline": roofline,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "Gpixels/s", "h2d_bytes_per_step": f_np.nbytes + p_np.nbytes,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps, "how": e2e_how},
        "gpu_launches": launches,
    }
    if rank == 0 and not args.no_cpu_baseline and args.workload == WORKLOAD:
        v, dt, desc = cpu_baseline_run(f_np[0, 0], p_np[0], crop=args.cpu_crop)
        line["cpu_baseline"] = {"value": v / 1e9, "unit": "Gpixels/s", "cores": 1, "kind": "oracle",
                                "sample": f"{desc}; {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_serve(args):
    """Serving stream shaped like the request workload: square images with side
    log-uniform in [256, 4096], 1 or 3 channels, N in {4, 6}, sigma 1-40, rho 1-8,
    Poisson arrivals at 0.7x the measured saturation rate.  Bounded sample:
    args.requests requests whose images and fields are crops (at seeded offsets)
    of device-resident 4096x4096 pools, so the loop measures the device side."""
    import torch
    from paper_1003_2022_gb300 import synth
    from paper_1003_2022_gb300.serve import Request, Server
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(2024)
    S = args.pool_side
    pools = []
    for k in range(2):
        img = torch.from_numpy(np.stack([synth.image(S, S, seed=500 + k, dtype="f32", sub=c) for c in range(3)]))
        prm = torch.from_numpy(synth.srt_field(S, S, seed=500 + k, sigma=(1.0, 40.0), rho=(1.0, 8.0)))
        pools.append((img.to(dev), prm.to(dev)))

    def make(n, rate):
        reqs, t = [], 0.0
        for i in range(n):
            side = int(round(np.exp(rng.uniform(np.log(256), np.log(S)))))
            C = 1 if rng.random() < 0.5 else 3
            N = 4 if rng.random() < 0.5 else 6
            img, prm = pools[i % 2]
            y0, x0 = (int(rng.integers(0, S - side + 1)) for _ in range(2))
            reqs.append(Request(i, img[:C, y0:y0 + side, x0:x0 + side], prm[:, y0:y0 + side, x0:x0 + side],
                                N=N, arrival=t, max_scale=40.0))
            if rate:
                t += float(rng.exponential(1.0 / rate))
        return reqs

    srv = Server(slots=args.slots, budget_bytes=int(args.hbm_gb * (1 << 30)), device=0, copy_back=False)
    try:
        srv.run(make(8, 0))  # warm-up: contexts grow their buffers
        _, sat = srv.run(make(args.requests, 0))
        rate = 0.7 * sat["completed"] / sat["makespan_s"] * (args.requests / max(sat["completed"], 1))
        _, st = srv.run(make(args.requests, rate))
    finally:
        srv.close()
    line = {"metric": METRIC, "value": st["gpixels_per_s"], "unit": "Gpixels/s", "n_gpus": 1,
            "steps": args.requests, "warmup": 8, "ms_per_step": 1e3 * st["makespan_s"] / args.requests,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int128", "data": "synthetic",
            "config": {"workload": f"serving stream: {args.requests} requests, side log-uniform 256-{S}, 1 or 3 "
                                   "channels f32, N in {4,6} (N=6 on the hexagonal lattice, FP64), sigma 1-40, rho 1-8, "
                                   "Poisson arrivals at 0.7x saturation", "slots": args.slots,
                       "hbm_budget_gb": args.hbm_gb, "arrival_rate_per_s": rate,
                       "saturation_gpixels_per_s": sat["gpixels_per_s"]},
            "serving": st}
    print(json.dumps(line), flush=True)
    return 0


def run_smooth(args):
    """Feature-preserving smoothing (Sec. 4.2) on a 2048x2048 f32 image of noisy
    concentric rings: one step = the adaptive covariance field (structure
    tensor, its window filtered by the box spline, the covariance map) plus the
    space-variant filter with that field.  Also reports the PSNR against the
    clean rings of the noisy input, of the best of three isotropic filters of
    the same area and of the adaptive filter."""
    import torch
    from paper_1003_2022_gb300 import _lib as L
    from paper_1003_2022_gb300 import api, synth
    dev = torch.device("cuda:0")
    H = W = args.size or 2048
    clean = synth.rings_image(H, W, period=8.0)
    noisy = torch.from_numpy(synth.add_noise(clean, 0.15, seed=5)).to(dev)
    cl = torch.from_numpy(clean).to(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    sw, s0, tau = 2.0, 1.0, 0.005

    def psnr(x):
        return float(10 * torch.log10(1.0 / torch.mean((x - cl) ** 2)))

    def step():
        return api.adaptive_smooth(noisy, sigma_w=sw, sigma0=s0, tau=tau)

    for _ in range(args.warmup):
        flush.fill_(1)
        out = step()
    torch.cuda.synchronize(dev)
    ctx = api.context(dev)
    stream = torch.cuda.current_stream(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    sampler.t0 = time.time()
    L.bsf_profile_begin(ctx)
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        evs[i][0].record(stream)
        out = step()
        evs[i][1].record(stream)
    torch.cuda.synchronize(dev)
    sampler.t1 = time.time()
    ms_pre, ms_st, nl = L.bsf_profile_end(ctx)
    sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total = sum(step_ms)
    p_ad = psnr(out)
    p_iso = -1e9
    for s in (0.8, 1.0, 1.2):
        iso = torch.zeros((3, H, W), device=dev)
        iso[0] = iso[2] = s * s
        p_iso = max(p_iso, psnr(api.filter(noisy, iso, kind="cov", max_scale=s)))
    if api.device_status(dev) & ~(1 << L.BSF_EINFEASIBLE):
        raise RuntimeError("device status error")
    line = {"metric": METRIC, "value": H * W * args.steps / (total / 1e3) / 1e9, "unit": "Gpixels/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int128", "data": "synthetic",
            "config": {"workload": f"feature-preserving smoothing of {H}x{W} f32 concentric rings (period 8 px) "
                                   "with Gaussian noise 0.15: structure tensor (window std 2 px), adaptive "
                                   "covariance (sigma0 1 px, tau 0.005), space-variant filter",
                       "l2": "flushed between timed steps (512 MiB write)",
                       "filter_ms_per_step": ms_st / args.steps, "preintegrate_ms_per_step": ms_pre / args.steps,
                       "filter_launches_per_step": nl / args.steps},
            "psnr_db": {"noisy": psnr(noisy), "isotropic_best": p_iso, "adaptive": p_ad},
            "clocks": sampler.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_sizes(args):
    """Run time against kernel size (the paper's computation-time table): one
    2048x2048 u8 image filtered with a constant (sigma, rho, theta) field for
    sigma = 1 .. 32 px; the halo of the pre-integrated buffer grows with sigma,
    the per-pixel work of the finite difference does not."""
    import torch
    from paper_1003_2022_gb300 import _lib as L
    from paper_1003_2022_gb300 import api, synth
    dev = torch.device("cuda:0")
    H = W = args.size or 2048
    f = torch.from_numpy(synth.image(H, W, seed=0, dtype="u8")).to(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    ctx = api.context(dev)
    stream = torch.cuda.current_stream(dev)
    rows = []
    for rho, theta in ((1.0, 0.0), (4.0, 0.4)):
        for sigma in (1.0, 2.0, 4.0, 8.0, 16.0, 32.0):
            prm = torch.from_numpy(synth.constant_srt(H, W, sigma, rho, theta)).to(dev)
            out = torch.empty((H, W), dtype=torch.float32, device=dev)
            for _ in range(args.warmup):
                api.filter(f, prm, kind="srt", max_scale=sigma, out=out)
            torch.cuda.synchronize(dev)
            L.bsf_profile_begin(ctx)
            evs = []
            for i in range(args.steps):
                flush.fill_(i & 0xFF)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                api.filter(f, prm, kind="srt", max_scale=sigma, out=out)
                e1.record(stream)
                evs.append((e0, e1))
            torch.cuda.synchronize(dev)
            ms_pre, ms_st, nl = L.bsf_profile_end(ctx)
            rows.append({"sigma": sigma, "rho": rho, "theta": theta, "halo": api.halo_for(sigma),
                         "ms_per_step": sum(a.elapsed_time(b) for a, b in evs) / args.steps,
                         "stencil_ms": ms_st / nl, "preintegrate_ms": ms_pre / nl})
    if api.device_status(dev) & ~(1 << L.BSF_EINFEASIBLE):
        raise RuntimeError("device status error")
    print(json.dumps({"mode": "sizes", "workload": f"{H}x{W} u8, constant (sigma, rho, theta) fields",
                      "rows": rows}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="exact", choices=["exact", "fp64"])
    ap.add_argument("--cpu-crop", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--size", type=int, default=None, help="square image side (default: the 2048 workload)")
    ap.add_argument("--mode", default="filter", choices=["filter", "serve", "smooth", "sizes"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(BENCH_WORKLOADS))
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--hbm-gb", type=float, default=48.0)
    ap.add_argument("--pool-side", type=int, default=4096)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    from paper_1003_2022_gb300 import build
    build.build()
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "smooth":
        return run_smooth(args)
    if args.mode == "sizes":
        return run_sizes(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
