"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds only random-number generation and reshaping: none of the
filter's arithmetic.  Both the CUDA path (bench, tests) and the oracle side of
the tests draw their inputs from here, so both see identical bytes.

Recipe (numpy PCG64, one sub-seed per field):
  * images: uniform f32 in [0, 1), or uniform u8 in {0..255}; the batched N=6
    workload adds three seeded sinusoidal gratings of amplitude 0.25 and
    spatial frequency |k| in [1/64, 1/8] cycles/px;
  * smooth fields: white noise Gaussian-blurred with std = side/16 px
    (computed on a grid 16x coarser than the image, blur std = side/256
    coarse px, periodic, then upsampled with a cubic spline), rank-normalised
    to U[0, 1] and mapped affinely to the requested range;
  * orientation from a vector field: theta = atan2(v, u) mod pi of two
    independent smooth fields centred at zero.
"""
from __future__ import annotations

import numpy as np

try:  # scipy is on both machines; keep the import local to the generators
    from scipy import ndimage as _ndi
except Exception:  # pragma: no cover
    _ndi = None


def _rng(seed: int, sub: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(sub)]))


def image(H: int, W: int, seed: int, dtype: str = "f32", sub: int = 0) -> np.ndarray:
    """Uniform image: 'f32' in [0,1) or 'u8' in {0..255}."""
    g = _rng(seed, 100 + sub)
    if dtype == "u8":
        return g.integers(0, 256, size=(H, W), dtype=np.uint8)
    return g.random((H, W), dtype=np.float32)


def gratings_image(H: int, W: int, seed: int, sub: int = 0) -> np.ndarray:
    """U[0,1) plus three sinusoidal gratings (amplitude 0.25 each), f32."""
    g = _rng(seed, 200 + sub)
    f = g.random((H, W)).astype(np.float64)
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    for _ in range(3):
        fr = g.uniform(1 / 64, 1 / 8)
        ang = g.uniform(0, np.pi)
        ph = g.uniform(0, 2 * np.pi)
        f += 0.25 * np.sin(2 * np.pi * fr * (np.cos(ang) * x + np.sin(ang) * y) + ph)
    return f.astype(np.float32)


def _smooth_noise(H: int, W: int, g: np.random.Generator) -> np.ndarray:
    cs = 16
    hc, wc = H // cs + 6, W // cs + 6
    z = g.standard_normal((hc, wc))
    blur = max(1.0, max(H, W) / 16.0 / cs)  # std side/16 px, in coarse px
    if _ndi is not None:
        z = _ndi.gaussian_filter(z, blur, mode="wrap")
        up = _ndi.zoom(z, cs, order=3)
    else:  # plain nearest fallback (never used where scipy exists)
        up = np.kron(z, np.ones((cs, cs)))
    return up[3 * cs // 2:3 * cs // 2 + H, 3 * cs // 2:3 * cs // 2 + W]


def smooth_field(H: int, W: int, seed: int, sub: int, lo: float, hi: float) -> np.ndarray:
    """Smooth random field, rank-normalised to U[0,1], mapped to [lo, hi] (f64)."""
    z = _smooth_noise(H, W, _rng(seed, sub))
    r = np.empty(z.size)
    r[np.argsort(z, axis=None, kind="stable")] = (np.arange(z.size) + 0.5) / z.size
    return lo + (hi - lo) * r.reshape(H, W)


def orientation_field(H: int, W: int, seed: int, sub: int) -> np.ndarray:
    """theta = atan2(v, u) mod pi of a smooth zero-mean vector field."""
    g = _rng(seed, sub)
    u = _smooth_noise(H, W, g)
    v = _smooth_noise(H, W, g)
    return np.mod(np.arctan2(v, u), np.pi)


def srt_field(H: int, W: int, seed: int, sigma=(2.0, 8.0), rho=(1.0, 4.0), theta: str = "uniform",
              sigma_log: bool = False) -> np.ndarray:
    """(sigma, rho, theta) planes, shape (3, H, W), float32.

    sigma: major-axis std in px; rho: elongation lambda_max / lambda_min;
    theta: 'uniform' (smooth field mapped to [0, pi)) or 'vector' (from a
    smooth vector field).
    """
    if sigma_log:
        s = np.exp(smooth_field(H, W, seed, 1, np.log(sigma[0]), np.log(sigma[1])))
    else:
        s = smooth_field(H, W, seed, 1, sigma[0], sigma[1])
    r = smooth_field(H, W, seed, 2, rho[0], rho[1])
    if theta == "vector":
        t = orientation_field(H, W, seed, 3)
    else:
        t = smooth_field(H, W, seed, 3, 0.0, np.pi)
    t = np.minimum(t, np.nextafter(np.pi, 0))
    return np.stack([s, r, t]).astype(np.float32)


def scale_field(H: int, W: int, seed: int, lo: float = 1.0, hi: float = 24.0) -> np.ndarray:
    """Four independent smooth fields in [lo, hi]: a learnable scale vector
    a = (a1..a4) per pixel, shape (4, H, W), float32."""
    return np.stack([smooth_field(H, W, seed, 40 + k, lo, hi) for k in range(4)]).astype(np.float32)


def rings_image(H: int, W: int, period: float = 8.0, cy: float | None = None, cx: float | None = None,
                contrast: float = 0.4) -> np.ndarray:
    """Concentric rings 0.5 + contrast * sin(2 pi r / period) around (cy, cx): an
    oriented pattern whose orientation changes everywhere (f32)."""
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    cy = 0.5 * (H - 1) if cy is None else cy
    cx = 0.5 * (W - 1) if cx is None else cx
    r = np.hypot(y - cy, x - cx)
    return (0.5 + contrast * np.sin(2.0 * np.pi * r / period)).astype(np.float32)


def add_noise(f: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """f plus white Gaussian noise of std sigma (f32)."""
    g = _rng(seed, 300)
    return (f.astype(np.float64) + sigma * g.standard_normal(f.shape)).astype(np.float32)


def constant_srt(H: int, W: int, sigma: float, rho: float, theta: float) -> np.ndarray:
    """A constant (sigma, rho, theta) field, shape (3, H, W), float32."""
    out = np.empty((3, H, W), dtype=np.float32)
    out[0], out[1], out[2] = sigma, rho, theta
    return out


# Workloads: shapes and parameter ranges of the paper-shaped configurations.
WORKLOADS = {
    # 256x256 f32 U[0,1), N=4, smooth (sigma 2-8, rho 1-4, theta uniform)
    "u256_f32_n4": dict(B=1, C=1, H=256, W=256, dtype="f32", N=4, sigma=(2.0, 8.0), rho=(1.0, 4.0),
                        theta="uniform"),
    # 2048x2048 u8 U{0..255}, N=4, sigma 1-32, rho 1-8, theta from a smooth vector field
    "u2048_u8_n4": dict(B=1, C=1, H=2048, W=2048, dtype="u8", N=4, sigma=(1.0, 32.0), rho=(1.0, 8.0),
                        theta="vector"),
    # same image as f32
    "u2048_f32_n4": dict(B=1, C=1, H=2048, W=2048, dtype="f32", N=4, sigma=(1.0, 32.0), rho=(1.0, 8.0),
                         theta="vector"),
    # batch of 4 RGB 4096x4096 f32 U[0,1) + gratings, sigma 2-48, rho 1-6, theta uniform,
    # filtered with six directions (the paper-shaped batch) or with four
    "b4c3_4096_f32_n6": dict(B=4, C=3, H=4096, W=4096, dtype="f32g", N=6, sigma=(2.0, 48.0), rho=(1.0, 6.0),
                             theta="uniform"),
    "b4c3_4096_f32_n4": dict(B=4, C=3, H=4096, W=4096, dtype="f32g", N=4, sigma=(2.0, 48.0), rho=(1.0, 6.0),
                             theta="uniform"),
    # batch of 8 1024x1024 f32 U[0,1) with a learnable scale field a_k in [1, 24]
    "b8_1024_f32_scales": dict(B=8, C=1, H=1024, W=1024, dtype="f32", N=4, scales=(1.0, 24.0)),
}


def workload_inputs(name: str, seed: int = 0, H: int | None = None, W: int | None = None):
    """Image (H, W) and (sigma, rho, theta) planes (3, H, W) for a named
    single-image workload.

    H, W override the size (same distributions) for reduced parity cases.
    """
    cfg = WORKLOADS[name]
    H = H or cfg["H"]
    W = W or cfg["W"]
    if cfg["dtype"] == "u8":
        f = image(H, W, seed, "u8")
    else:
        f = image(H, W, seed, "f32")
    p = srt_field(H, W, seed, cfg["sigma"], cfg["rho"], cfg["theta"])
    return f, p


def batch_inputs(name: str, seed: int = 0, H: int | None = None, W: int | None = None, B: int | None = None,
                 sigma: tuple | None = None):
    """Images (B, C, H, W) and parameter planes (B, K, H, W) of a batched
    workload: K = 3 (sigma, rho, theta) planes, or K = 4 scale planes for the
    learnable-scale workload.  Batch entry b uses the sub-seed seed + b.
    sigma: another (lo, hi) range of the size field than the workload's."""
    cfg = dict(WORKLOADS[name])
    if sigma is not None:
        cfg["sigma"] = tuple(sigma)
    H = H or cfg["H"]
    W = W or cfg["W"]
    B = B or cfg["B"]
    C = cfg["C"]
    imgs = np.empty((B, C, H, W), dtype=np.uint8 if cfg["dtype"] == "u8" else np.float32)
    K = 4 if "scales" in cfg else 3
    prm = np.empty((B, K, H, W), dtype=np.float32)
    for b in range(B):
        for c in range(C):
            if cfg["dtype"] == "f32g":
                imgs[b, c] = gratings_image(H, W, seed + b, sub=c)
            else:
                imgs[b, c] = image(H, W, seed + b, cfg["dtype"], sub=c)
        if K == 4:
            prm[b] = scale_field(H, W, seed + b, *cfg["scales"])
        else:
            prm[b] = srt_field(H, W, seed + b, cfg["sigma"], cfg["rho"], cfg["theta"])
    return imgs, prm
