"""Continuous-batching request loop for the space-variant box-spline filter.

Requests (an image of any size and channel count, its (sigma, rho, theta)
field, N) arrive over time.  The server keeps S slots; each slot is a CUDA
stream with its own library context, so its pre-integrated buffers and scan
carries stay on the device and are reused by later requests.  A request is
admitted as soon as a slot is free and its device footprint fits the HBM
budget left by the requests in flight; requests that arrive while others run
join immediately, and their copies and kernels overlap on the device.

The scheduling policy (`Scheduler`) is plain host logic: FIFO with skip-ahead
(a request that does not fit lets later, smaller ones pass; it keeps its
place at the head), requests that can never fit or use an unsupported N are
rejected with a reason.  `Server` binds it to the GPU through the C ABI.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

SUPPORTED_N = (4, 6)


@dataclass
class Request:
    rid: int
    image: object                # (C, H, W) uint8/float32: numpy array (host) or CUDA tensor (device)
    params: object               # (3, H, W) float32 (sigma, rho, theta): numpy array or CUDA tensor
    N: int = 4
    arrival: float = 0.0         # seconds after the stream start
    max_scale: float = 0.0       # largest sigma of the field (0: take it from params)
    cancel_at: float = math.inf  # withdrawn at this time (seconds) if not admitted by then


@dataclass
class Result:
    rid: int
    status: str                  # "ok" or the rejection reason
    out: object = None           # (C, H, W) float32 host array when copied back
    t_arrival: float = 0.0
    t_admit: float = math.nan
    t_done: float = math.nan
    nbytes: int = 0
    samples: int = 0

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


def halo_for_sigma(max_sigma: float) -> int:
    # the library's rule for COV/SRT fields: ext <= 8.364 sigma_max, P = ceil(ext/2) + 4
    return int(math.ceil(0.5 * 8.3640 * max_sigma)) + 4


def _max_sigma(params) -> float:
    """Largest finite sigma of a (sigma, rho, theta) field (NaN pixels ignored)."""
    s0 = params[0]
    if hasattr(s0, "nan_to_num"):
        return float(s0.nan_to_num(nan=0.0, posinf=0.0).max())
    s0 = np.asarray(s0)
    fin = s0[np.isfinite(s0)]
    return float(fin.max()) if fin.size else 0.0


def footprint_bytes(C: int, H: int, W: int, image_itemsize: int, max_sigma: float, N: int = 4) -> int:
    """Device bytes one request holds while in flight: image, field, output and
    the library's scratch.  N = 4: pre-integrated buffers (8 B/elem for uint8,
    16 B for float32) and scan carries.  N = 6: FP64 scales (48 B/px) and the
    lattice windows of the 64-pixel tiles (spacing 0.5 px, 16 B per lattice
    point), at most 8 GiB of them per chunk, in two buffers (the windows of the
    next chunk are pre-integrated while the current chunk's stencil runs)."""
    io = C * H * W * image_itemsize + 3 * H * W * 4 + C * H * W * 4
    if N == 6:
        # half-extent of a footprint: sum_k a_k |cos theta_k| / 2 <= sqrt(3 sum_k a_k^2) / 2
        # = sqrt(36 tr C) / 2 <= 4.25 sigma; a window spans R = 64 + 2 ext + 10 px and holds
        # about 5.46 R x 2.31 R lattice points of 16 B (an upper bound: tiles with
        # large footprints share windows)
        R = 64 + 2 * 4.25 * max_sigma + 10
        tiles = math.ceil(H / 64) * math.ceil(W / 64)
        win = min(8 << 30, int(tiles * C * 16 * 5.46 * R * 2.31 * R))
        return io + 48 * H * W + 2 * win
    P = halo_for_sigma(max_sigma)
    Hp, Wp = H + 2 * P, W + 2 * P
    elem = 8 if image_itemsize == 1 else 16
    bh = min(max(8, (Hp * C + 151) // 152), 64)
    nb = (Hp + bh - 1) // bh
    buf = C * Hp * Wp * elem
    carries = 10 * C * nb * Wp * elem
    return buf + carries + io


class Scheduler:
    """Slots and HBM budget bookkeeping (no GPU)."""

    def __init__(self, slots: int, budget_bytes: int):
        self.slots = slots
        self.budget = budget_bytes
        self.inflight: dict[int, int] = {}  # rid -> bytes
        self.free_slots = list(range(slots))[::-1]
        self.slot_of: dict[int, int] = {}
        self.pending: deque = deque()
        self.peak_bytes = 0
        self._used = 0

    def used(self) -> int:
        return self._used

    def offer(self, rid: int, nbytes: int, N: int) -> str | None:
        """Queue a request; returns a rejection reason, or None when queued."""
        if N not in SUPPORTED_N:
            return f"unsupported N={N}"
        if nbytes > self.budget:
            return f"footprint {nbytes} B exceeds the HBM budget {self.budget} B"
        self.pending.append((rid, nbytes))
        return None

    def admit(self) -> list[tuple[int, int]]:
        """Admit queued requests into free slots while memory allows: (rid, slot) pairs."""
        out = []
        skipped = []
        while self.pending and self.free_slots:
            rid, nb = self.pending.popleft()
            if self._used + nb <= self.budget:
                slot = self.free_slots.pop()
                self.inflight[rid] = nb
                self.slot_of[rid] = slot
                self._used += nb
                out.append((rid, slot))
                self.peak_bytes = max(self.peak_bytes, self._used)
            else:
                skipped.append((rid, nb))
        # requests passed over keep their places at the head of the queue
        self.pending.extendleft(reversed(skipped))
        return out

    def cancel(self, rid: int) -> bool:
        """Withdraw a queued request; False if it is not queued (admitted or unknown)."""
        for i, (r, _) in enumerate(self.pending):
            if r == rid:
                del self.pending[i]
                return True
        return False

    def complete(self, rid: int) -> int:
        """Release a finished request's memory and slot; returns the slot."""
        self._used -= self.inflight.pop(rid)
        slot = self.slot_of.pop(rid)
        self.free_slots.append(slot)
        return slot


def percentiles(lat: list[float]) -> dict:
    if not lat:
        return {"p50_ms": None, "p99_ms": None}
    a = np.asarray(lat) * 1e3
    return {"p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
            "mean_ms": float(a.mean()), "max_ms": float(a.max())}


class Server:
    """GPU executor of the scheduler: one stream and one library context per slot."""

    def __init__(self, slots: int = 4, budget_bytes: int = 32 << 30, device: int = 0, copy_back: bool = True):
        import torch

        from . import _lib as L
        self.torch = torch
        self.L = L
        self.dev = torch.device(f"cuda:{device}")
        self.sched = Scheduler(slots, budget_bytes)
        self.copy_back = copy_back
        with torch.cuda.device(self.dev):
            self.streams = [torch.cuda.Stream(self.dev) for _ in range(slots)]
            self.ctxs = [L.bsf_create(device) for _ in range(slots)]

    def close(self):
        for c in self.ctxs:
            self.L.bsf_destroy(c)
        self.ctxs = []

    def _launch(self, req: Request, slot: int):
        torch, L = self.torch, self.L
        st = self.streams[slot]
        C, H, W = req.image.shape
        with torch.cuda.stream(st):
            if torch.is_tensor(req.image):  # device-resident request: contiguous copies on the slot stream
                img_h = prm_h = None
                img = req.image.contiguous()
                prm = req.params.contiguous()
            else:
                img_h = torch.from_numpy(np.ascontiguousarray(req.image)).pin_memory()
                prm_h = torch.from_numpy(np.ascontiguousarray(req.params, dtype=np.float32)).pin_memory()
                img = img_h.to(self.dev, non_blocking=True)
                prm = prm_h.to(self.dev, non_blocking=True)
            out = torch.empty((C, H, W), dtype=torch.float32, device=self.dev)
            opts = L.default_opts()
            opts.max_scale = float(req.max_scale or _max_sigma(req.params))
            dtype = L.BSF_U8 if img.dtype == torch.uint8 else L.BSF_F32
            rc = L.bsf_filter(self.ctxs[slot], img.data_ptr(), dtype, 1, C, H, W, req.N, prm.data_ptr(),
                              L.BSF_PARAM_SRT, opts, out.data_ptr(), int(st.cuda_stream))
            host = None
            if rc == L.BSF_OK and self.copy_back:
                host = torch.empty((C, H, W), dtype=torch.float32).pin_memory()
                host.copy_(out, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        # keep the tensors alive until the event has passed
        return rc, ev, (img_h, prm_h, img, prm, out, host)

    def run(self, requests: list[Request], poll_s: float = 0.0) -> tuple[list[Result], dict]:
        """Serve requests arriving at their `arrival` times (seconds after start)."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        by_id = {r.rid: r for r in reqs}
        results = {r.rid: Result(r.rid, "pending", t_arrival=r.arrival, samples=int(np.prod(tuple(r.image.shape))))
                   for r in reqs}
        running: dict[int, tuple] = {}
        # withdrawals in time order; one that falls before its own arrival is applied at arrival
        cancels = sorted((max(r.cancel_at, r.arrival), r.rid) for r in reqs if r.cancel_at < math.inf)
        ci = 0
        nxt = 0
        t0 = time.perf_counter()
        max_depth = 0
        while nxt < len(reqs) or self.sched.pending or running:
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                r = reqs[nxt]
                nxt += 1
                C, H, W = r.image.shape
                isz = r.image.element_size() if self.torch.is_tensor(r.image) else r.image.dtype.itemsize
                nb = footprint_bytes(C, H, W, isz, r.max_scale or _max_sigma(r.params), r.N)
                results[r.rid].nbytes = nb
                why = self.sched.offer(r.rid, nb, r.N)
                if why is not None:
                    results[r.rid].status = why
                    results[r.rid].t_done = now
            while ci < len(cancels) and cancels[ci][0] <= now:
                rid = cancels[ci][1]
                ci += 1
                if results[rid].status == "pending" and self.sched.cancel(rid):
                    results[rid].status = "cancelled"
                    results[rid].t_done = now
            for rid in list(running):
                rc, ev, keep = running[rid]
                if ev.query():
                    t = time.perf_counter() - t0
                    res = results[rid]
                    res.t_done = t
                    slot = self.sched.slot_of[rid]
                    # per-pixel conditions of this request (the slot's context serves one request at a time)
                    dev_st = self.L.bsf_get_device_status(self.ctxs[slot], int(self.streams[slot].cuda_stream))
                    bad = dev_st & ~(1 << self.L.BSF_EINFEASIBLE)
                    if rc != self.L.BSF_OK:
                        res.status = f"bsf status {rc}"
                    elif bad:
                        codes = [c for c in range(1, 32) if bad & (1 << c)]
                        res.status = "invalid pixels: " + "; ".join(self.L.status_string(c) for c in codes)
                    else:
                        res.status = "ok"
                    if keep[5] is not None:
                        res.out = keep[5].numpy()
                    self.sched.complete(rid)
                    del running[rid]
            for rid, slot in self.sched.admit():
                results[rid].t_admit = time.perf_counter() - t0
                running[rid] = self._launch(by_id[rid], slot)
            max_depth = max(max_depth, len(self.sched.pending))
            if poll_s:
                time.sleep(poll_s)
        makespan = time.perf_counter() - t0
        done = [r for r in results.values() if r.status == "ok"]
        samples = sum(r.samples for r in done)
        n_cancel = sum(r.status == "cancelled" for r in results.values())
        n_invalid = sum(r.status.startswith("invalid") for r in results.values())
        stats = {"requests": len(reqs), "completed": len(done),
                 "rejected": len(reqs) - len(done) - n_cancel - n_invalid, "cancelled": n_cancel,
                 "invalid": n_invalid, "makespan_s": makespan,
                 "gpixels_per_s": samples / makespan / 1e9, "peak_bytes": self.sched.peak_bytes,
                 "max_queue_depth": max_depth}
        stats.update(percentiles([r.latency for r in done]))
        return [results[r.rid] for r in reqs], stats
