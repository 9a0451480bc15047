"""Benchmark of the space-variant elliptical box-spline filter on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload ID]

One step = the whole hot path, through the C ABI call bsf_filter, over the
default workload: a batch of 4 RGB 4096x4096 float32 images (uniform [0,1)
plus three seeded gratings) with a per-pixel (sigma, rho, theta) field per
image (sigma 2-48 px, rho 1-6, theta uniform), N = 6 directions: the scale
map (Sec. 3.2.2 with the six-directional kurtosis norm), the transfer to the
hexagonal lattice and the six running sums (Algorithm 1 step 2), and the
64-tap finite difference (Algorithm 1 step 3).  --workload u2048_u8_n4 runs
the 2048x2048 uint8 image with N = 4 (sigma 1-32, rho 1-8), and so on.
Inputs are resident in HBM before the timed region; between timed steps a
512 MiB buffer is written to flush the 129 MB L2.

For N > 1 (torchrun), each rank runs an independent replica on its own GPU
(the path has no exchange step); value = pixels of all ranks / max time.

--impl reference times the FP64 CPU oracle (Algorithm 1 restated, with the
oracle's own scale map) on the host cores, one bounded crop of the same
workload per step.
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

WORKLOAD = "b4c3_4096_f32_n6"
METRIC = "Gpixels/s filtered (N=4,6) at ≤1e-5 rel err vs FP64 oracle; % HBM roofline; p50/p99"
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
# six directions: the exact coefficient sums on the tensor cores.  Per round a warp's
# 24 mma.sync.m16n8k16 (3 words x 4 bytes x 2 k-steps; 16 x 8 x 16 multiply-adds each)
# cover 8 taps: 3 x 4096 FLOP per tap, 64 taps per pixel
HEX6_TC_FLOP_PER_PX = 64 * 3 * 2 * 16 * 8 * 16
# the method's work per output pixel as the hot-path table counts it: N = 4, 16 taps x
# (partition select + 7 ZP weights + 7 multiply-adds) ~ 1.0k operations; N = 6, 64 taps,
# 2.5k-4k operations (the midpoint is used)
METHOD_OPS_PER_PX = {4: 1000, 6: 3250}
METHOD_OPS_NOTE = {4: "16 taps x (partition select + 7 ZP weights + 7 multiply-adds) ~ 1.0k ops/px",
                   6: "64 taps, 2.5k-4k ops/px (midpoint 3250)"}
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
                        "theta uniform, N=6 (64-tap stencil) on the hexagonal lattice of spacing 0.5 px, exact 128-bit "
                        "window sums and coefficient sums, double-float remainder",
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


def preint_algorithmic_bytes(nimg: int, H: int, W: int, P: int, in_bytes: int, elem: int) -> int:
    """Algorithmic HBM bytes of one pre-integration call over nimg images: every
    buffer element written once, every image sample its strip needs read once.
    Wide rows are cut into vertical strips exactly as the library does (a band
    CTA holds at most 4096 int64/double or 3072 128-bit elements of a row, 2048
    when a batch of 128-bit buffers fills several waves), so a strip reads the
    image columns of its outputs +- P."""
    many_waves = (H + 2 * P) * nimg > 64 * 152
    maxw = (2048 if many_waves else 3072) if elem == 16 else 4096
    Wfull = W + 2 * P
    nstrip = 1 if Wfull <= maxw else -(-W // (maxw - 2 * P))
    Ws = -(-W // nstrip)
    tot = 0
    for sidx in range(nstrip):
        col0 = sidx * Ws
        ws = W if nstrip == 1 else min(Ws, W - col0)
        wp = ws + 2 * P
        cols_read = min(W, col0 + ws + P) - max(0, col0 - P)
        tot += nimg * ((H + 2 * P) * wp * elem + H * cols_read * in_bytes)
    return tot


def alu_peak_tops():
    """Issue-rate bound of 32-bit integer ALU work: 152 SMs x 128 lanes x max SM clock."""
    return 152 * 128 * 2.070e9 / 1e12


def _inputs(size=None, workload=WORKLOAD, first_only=False, sigma_max=None):
    """(B, C, H, W) image and (B, K, H, W) parameter planes of a workload
    (first_only: the first batch entry alone, generated from the same seed)."""
    from paper_1003_2022_gb300 import synth
    if synth.WORKLOADS[workload]["B"] == 1 and "scales" not in synth.WORKLOADS[workload]:
        f, p = synth.workload_inputs(workload, seed=0, H=size, W=size)
        return f[None, None], p[None]
    sig = None if sigma_max is None else (synth.WORKLOADS[workload]["sigma"][0], sigma_max)
    return synth.batch_inputs(workload, seed=0, H=size, W=size, B=1 if first_only else None, sigma=sig)


def _map6_chunk(args):
    """One worker's share of the oracle's six-directional map (spawned process)."""
    from oracle import n6
    params, kind = args
    return n6.map6(params, kind)[0]


class OracleRunner:
    """The FP64 oracle on the host cores, for the CPU baseline and the reference
    arm: Algorithm 1 restated (O-alg) with the oracle's own scale map, on a crop
    of the workload's first image.  N = 4: ``map4`` + ``preint4`` + ``stencil4``
    (C, OpenMP over rows and pixels).  N = 6: ``n6.map6`` (numpy, KKT map, in a
    pool of spawned processes) + ``n6.alg1_hex_c`` (C, OpenMP over pixels).
    ``cores``: the host threads / processes used."""

    def __init__(self, N: int, u8: bool, sigma_max: float):
        import oracle
        oracle.build()
        self.N, self.u8, self.smax = N, u8, sigma_max
        self.threads = oracle.num_threads()
        self.pool = None
        if N == 6:
            import multiprocessing as mp
            self.pool = mp.get_context("spawn").Pool(os.cpu_count() or 1)
            self.pool.map(_map6_chunk, [(np.ones((3, 1)), 2)] * (os.cpu_count() or 1))  # import in every worker
        self.cores = max(self.threads, os.cpu_count() or 1) if N == 6 else self.threads

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()

    def run(self, f, p, crop: int, seed: int):
        """Filter one crop x crop crop (zero outside it) at a seeded offset;
        returns seconds."""
        import oracle
        from oracle import n6
        H, W = f.shape
        rng = np.random.default_rng(seed)
        y0 = int(rng.integers(0, H - crop + 1))
        x0 = int(rng.integers(0, W - crop + 1))
        fc = np.ascontiguousarray(f[y0:y0 + crop, x0:x0 + crop])
        pc = np.ascontiguousarray(p[:, y0:y0 + crop, x0:x0 + crop]).astype(np.float64)
        t = time.perf_counter()
        if self.N == 4:
            a, _ = oracle.map4(pc, oracle.KIND_SRT)
            P = int(np.ceil(0.5 * 8.364 * self.smax)) + 4
            if self.u8:
                oracle.alg1_filter4(fc.astype(np.int64), a, P, integer=True)
            else:
                oracle.alg1_filter4(fc.astype(np.float64), a, P, integer=False)
        else:
            flat = pc.reshape(3, -1)
            parts = np.array_split(np.arange(flat.shape[1]), 4 * len(self.pool._pool))
            a = np.concatenate(self.pool.map(_map6_chunk, [(flat[:, ix], 2) for ix in parts if ix.size]), axis=1)
            n6.alg1_hex_c(fc.astype(np.float64), a.reshape(6, crop, crop), None, 0.5)
        return time.perf_counter() - t

    def describe(self, crop: int, n: int) -> str:
        if self.N == 4:
            steps = ("oracle map4 + preint4 (int64 for u8, FP64 for f32) + stencil4 (FP64 ZP weights from the exact "
                     "box spline), C with OpenMP")
        else:
            steps = ("oracle n6.map6 (KKT map, numpy, spawned processes) + n6.alg1_hex_c (transfer to the hexagonal "
                     "lattice, six FP64 running sums, 64-tap stencil with the exact element, C with OpenMP)")
        return f"{steps}; {n} crop(s) of {crop}x{crop} px of the workload's first image"


def oracle_direct_rate(f, p, N: int, budget_s: float = 8.0, seed: int = 5):
    """O-direct (the plain definition summed over each footprint) on sampled
    pixels of the full first image: pixels/s with the oracle's scales.  N = 4:
    C (``direct4``, OpenMP); N = 6: numpy (``n6.direct6_hex``, one pixel at a
    time).  Pixels are added until the time budget is spent (at most 4096)."""
    import oracle
    from oracle import n6
    H, W = f.shape
    rng = np.random.default_rng(seed)
    done, t_tot, batch = 0, 0.0, 16 if N == 6 else 512
    f64 = f.astype(np.float64)
    while done < 4096 and t_tot < budget_s:
        n = 1 if N == 6 else batch
        idx = rng.choice(H * W, size=n, replace=False)
        t = time.perf_counter()
        if N == 4:
            a, _ = oracle.map4(p.reshape(3, -1)[:, idx].astype(np.float64)[:, :, None], oracle.KIND_SRT)
            A = np.zeros((4, H * W))
            A[:, idx] = a[:, :, 0]
            oracle.direct4(f64, A.reshape(4, H, W), idx)
        else:
            a, _ = n6.map6(p.reshape(3, -1)[:, idx].astype(np.float64), 2)
            y, x = divmod(int(idx[0]), W)
            r = int(np.ceil(0.5 * np.sum(a[:, 0]))) + 2
            ya, xa = max(0, y - r), max(0, x - r)
            fc = f64[ya:min(H, y + r + 1), xa:min(W, x + r + 1)]
            A = np.zeros((6,) + fc.shape)
            A[:, y - ya, x - xa] = a[:, 0]
            n6.direct6_hex(fc, A, np.array([(y - ya) * fc.shape[1] + (x - xa)]), 0.5, origin=(xa, ya))
        t_tot += time.perf_counter() - t
        done += n
    return done / t_tot, done, t_tot


def run_reference(args):
    """The oracle, as it stands, on the host cores, on the workload of our arm:
    every step filters one bounded crop of it (O-alg with the oracle's map)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_1003_2022_gb300 import synth as _synth
    N = _synth.WORKLOADS[args.workload]["N"]
    _, smax, _ = BENCH_WORKLOADS[args.workload]
    f, p = _inputs(args.size, args.workload, first_only=True)
    u8 = f.dtype == np.uint8
    f, p = f[0, 0], p[0]
    crop = 32 if N == 6 else 96
    runner = OracleRunner(N, u8, smax)
    try:
        for i in range(args.warmup):
            runner.run(f, p, crop=crop // 2, seed=1000 + i)
        tot_s = 0.0
        for i in range(args.steps):
            tot_s += runner.run(f, p, crop=crop, seed=i)
    finally:
        runner.close()
    value = args.steps * crop * crop / tot_s / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gpixels/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD_TEXT[args.workload] + f"; one {crop}x{crop} crop "
                                        "per step", "workload_id": args.workload, "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": "Gpixels/s", "cores": runner.cores, "kind": "oracle",
                         "sample": runner.describe(crop, args.steps)},
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
    f_np, p_np = _inputs(args.size, args.workload, sigma_max=args.sigma_max)
    if args.sigma_max is not None:
        smax = args.sigma_max
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
    opts = api.make_opts("exact" if args.precision == "exact" else "fp64", max_scale=smax,
                         hex_spacing=args.hex_spacing, map_lut=args.map_lut, staging=args.staging)
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
    e2e_steps = max(3, min(args.steps, 5 if N == 6 else 50))
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
    # stencil launches in the timed region (one per strip and batch chunk of each forward call;
    # for N = 6 one per window chunk)
    n_st = max(nl, 1)
    st_ms = ms_st / n_st
    px_per_launch = npx * args.steps / n_st
    peaks, peak_src = _peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak = alu_peak_tops()
    # the method's own work per output pixel (the finite difference with its
    # interpolation, as the hot-path table counts it), not this implementation's
    method_ops = METHOD_OPS_PER_PX[N]
    achieved = method_ops * px_per_launch / (st_ms / 1e3) / 1e12
    if N == 4:
        impl_ops = STENCIL_INT_OPS_PER_PX if u8 else STENCIL_INT_OPS_PER_PX_U128
        kname = f"k_stencil4_exact<{'u64' if u8 else 'u128'},{kind_name.upper()}>"
        impl = {"what": "int32 operations of the exact integer form (64-bit or 128-bit emulation)",
                "ops_per_px": impl_ops, "achieved_tops": impl_ops * px_per_launch / (st_ms / 1e3) / 1e12}
        impl["frac"] = impl["achieved_tops"] / peak
        traffic = stencil_traffic() if (args.workload == "u2048_u8_n4" and args.size in (None, 2048)
                                        and args.precision == "exact") else None
        alg_bytes = int((12 + 4 + 8 * (1 if u8 else 2)) * px_per_launch)
    else:
        kname = "k_hex6_stencil"
        tc_peak = float(peaks.get("bf16_tflops", 1887.8))
        impl = {"what": "tensor-core FLOP of the exact coefficient sums (FP16 bytes x FP16 coefficients, "
                        "FP32 sums, mma.sync.m16n8k16): 64 taps x 3 mma of 4096 FLOP",
                "flop_per_px": HEX6_TC_FLOP_PER_PX,
                "achieved_tflops": HEX6_TC_FLOP_PER_PX * px_per_launch / (st_ms / 1e3) / 1e12,
                "peak": tc_peak,
                "peak_note": "measured dense bf16 (burst) of the GB300; FP16 runs at the bf16 rate"}
        impl["frac"] = impl["achieved_tflops"] / impl["peak"]
        traffic = None
        alg_bytes = int((12 + 4 + 16) * px_per_launch)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": kname, "kernel_ms": st_ms, "launches_per_step": n_st / args.steps,
                "preintegrate_ms": ms_pre / n_st,
                "method_ops_per_px": method_ops,
                "method_ops_note": METHOD_OPS_NOTE[N],
                "peak_note": "derived: 152 SMs x 128 lanes x 2070 MHz, 32-bit integer or FP32 operations (an "
                             "add-chain probe reached 37.1 Tops/s); MEASURED_PEAKS.json holds no integer peak",
                "implementation": impl,
                "algorithmic_bytes_per_launch": alg_bytes}
    # the HBM side of both steps, against the measured copy bandwidth
    if N == 4:
        P = api.halo_for(smax, kind_name)
        elem = 8 if (u8 or args.precision != "exact") else 16
        pre_bytes = preint_algorithmic_bytes(B * C, H, W, P, 1 if u8 else 4, elem)
        pre_ms = ms_pre / n_st
        roofline["hbm"] = {
            "peak_gbs": hbm_peak, "peak_source": peak_src,
            "stencil_dram_gbs": traffic / (st_ms * 1e6) if traffic else None,
            "stencil_frac": traffic / (st_ms * 1e6) / hbm_peak if traffic else None,
            "stencil_algorithmic_frac": alg_bytes / (st_ms * 1e6) / hbm_peak,
            "preintegrate_algorithmic_bytes": pre_bytes * args.steps / n_st,
            "preintegrate_gbs": pre_bytes * args.steps / n_st / (pre_ms * 1e6),
            "preintegrate_frac": pre_bytes * args.steps / n_st / (pre_ms * 1e6) / hbm_peak,
        }
    else:
        roofline["hbm"] = {"peak_gbs": hbm_peak, "peak_source": peak_src,
                           "stencil_algorithmic_frac": alg_bytes / (st_ms * 1e6) / hbm_peak,
                           "preintegrate_note": "map, window transfer and six exact running sums per chunk: "
                                                "compute-bound, not an HBM stream"}
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
        launches = args.steps + 2 * nl  # the map once per call, then windows + stencil per chunk
    if N == 6:
        dtype_s = "int128+double-float"
    elif args.precision == "exact":
        dtype_s = "int64" if u8 else "int128"
    else:
        dtype_s = "f64"
    line = {
        "metric": METRIC, "value": value, "unit": "Gpixels/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": dtype_s,
        "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload] if args.size is None else
                   f"{WORKLOAD_TEXT[args.workload]} (resized to {H}x{W})",
                   "workload_id": args.workload, **({"hex_spacing": args.hex_spacing} if N == 6 else {}),
                   **({"sigma_max": args.sigma_max} if args.sigma_max is not None else {}),
                   **({"map": "table"} if args.map_lut else {}),
                   **({"stencil_staging": "tma"} if args.staging == "tma" else {}),
                   "precision": args.precision, "l2": "flushed between timed steps (512 MiB write)",
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99))},
        "roofline": roofline,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "Gpixels/s", "h2d_bytes_per_step": f_np.nbytes + p_np.nbytes,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps, "how": e2e_how},
        "gpu_launches": launches,
    }
    if rank == 0 and not args.no_cpu_baseline and not train and args.precision == "exact":
        runner = OracleRunner(N, u8, smax)
        try:
            crop = args.cpu_crop or (256 if N == 6 else 1024)
            dt = runner.run(f_np[0, 0], p_np[0], crop=crop, seed=0)
        finally:
            runner.close()
        line["cpu_baseline"] = {"value": crop * crop / dt / 1e9, "unit": "Gpixels/s", "cores": runner.cores,
                                "kind": "oracle", "sample": f"{runner.describe(crop, 1)}; {dt:.1f} s",
                                "nproc": os.cpu_count()}
        rate, n_od, t_od = oracle_direct_rate(f_np[0, 0], p_np[0], N)
        line["oracle_direct"] = {"value": rate, "unit": "pixels/s", "pixels": n_od, "seconds": t_od,
                                 "cores": runner.threads if N == 4 else 1,
                                 "what": "the plain definition summed over each sampled pixel's footprint "
                                         "(with the oracle's scale map), full image"}
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
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int128+double-float",
            "data": "synthetic",
            "config": {"workload": f"serving stream: {args.requests} requests, side log-uniform 256-{S}, 1 or 3 "
                                   "channels f32, N in {4,6} (N=6 on the hexagonal lattice, exact integer + double-float), "
                                   "sigma 1-40, rho 1-8, "
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
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default: about 30-60 s of work)")
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="exact", choices=["exact", "fp64"])
    ap.add_argument("--cpu-crop", type=int, default=None, help="side of the oracle's crop (default 256 for N=6, "
                                                                "1024 for N=4)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--size", type=int, default=None, help="square image side (default: the 2048 workload)")
    ap.add_argument("--mode", default="filter", choices=["filter", "serve", "smooth", "sizes"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(BENCH_WORKLOADS))
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--hbm-gb", type=float, default=48.0)
    ap.add_argument("--pool-side", type=int, default=4096)
    ap.add_argument("--hex-spacing", type=float, default=0.5, help="N=6: lattice spacing h (1, 0.5, 0.25, 0.125)")
    ap.add_argument("--sigma-max", type=float, default=None, help="batched workloads: cap the size field at this sigma")
    ap.add_argument("--staging", choices=["l1", "tma"], default="l1",
                    help="N=4 u8: the stencil reads its buffer through L1 or from TMA-staged shared-memory boxes")
    ap.add_argument("--map-lut", action="store_true",
                    help="N=6: read the scale map from its table (an approximation) instead of solving it per pixel")
    args = ap.parse_args()
    from paper_1003_2022_gb300 import synth as _synth
    heavy = _synth.WORKLOADS[args.workload]["N"] == 6
    if args.steps is None:
        args.steps = 10 if heavy else (20 if args.workload.startswith("b4c3") else 200)
    if args.warmup is None:
        args.warmup = 3 if heavy else 10
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
