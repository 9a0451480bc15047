"""Torch-facing calls of the filter: device memory and streams come from
PyTorch, every step runs in libbsf (CUDA).

    out = filter(image, params, kind="srt")          # (B,C,H,W) -> (B,C,H,W) float32

image: uint8 or float32 CUDA tensor of shape (H,W), (C,H,W) with B=1, or
(B,C,H,W).  params: float32 CUDA tensor of the parameter planes of each
batch entry, shape (K,H,W) or (B,K,H,W): K=4 scale vectors a (kind
"scales"), or K=3 covariances (C11,C12,C22) (kind "cov"), or (sigma, rho,
theta) (kind "srt").
"""
from __future__ import annotations

import threading

import torch

from . import _lib as L

_KINDS = {"scales": L.BSF_PARAM_SCALES, "cov": L.BSF_PARAM_COV, "srt": L.BSF_PARAM_SRT}
_PREC = {"exact": L.BSF_PREC_EXACT, "fp64": L.BSF_PREC_FP64}
_ctx: dict[int, int] = {}
_ctx_lock = threading.Lock()


def context(device: int | torch.device | None = None) -> int:
    """The library context bound to a CUDA device (created on first use)."""
    if device is None:
        device = torch.cuda.current_device()
    idx = device.index if isinstance(device, torch.device) else int(device)
    with _ctx_lock:
        if idx not in _ctx:
            with torch.cuda.device(idx):
                _ctx[idx] = L.bsf_create(idx)
        return _ctx[idx]


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def make_opts(precision="exact", halo=0, max_scale=0.0, eps=1e-3, eta=1e-3, strict=False,
              iterations=1, hex_spacing=0.5, rel_bound=1e-3, boundary="zero", map_lut=False,
              staging="l1") -> L.bsf_opts:
    o = L.default_opts()
    o.map_lut = 1 if map_lut else 0
    o.staging = {"l1": L.BSF_STAGING_L1, "tma": L.BSF_STAGING_TMA}[staging]
    o.boundary = {"zero": L.BSF_BOUNDARY_ZERO, "reflect": L.BSF_BOUNDARY_REFLECT}[boundary]
    o.iterations = int(iterations)
    o.hex_spacing = float(hex_spacing)
    o.rel_bound = float(rel_bound)
    o.precision = _PREC[precision]
    o.halo = int(halo)
    o.max_scale = float(max_scale)
    o.eps = float(eps)
    o.eta = float(eta)
    o.strict = 1 if strict else 0
    return o


def _as4d(image: torch.Tensor) -> torch.Tensor:
    if image.dim() == 2:
        return image[None, None]
    if image.dim() == 3:
        return image[None]
    if image.dim() == 4:
        return image
    raise ValueError("image must be (H,W), (C,H,W) or (B,C,H,W)")


def filter(image: torch.Tensor, params: torch.Tensor, kind: str = "srt", N: int = 4, precision: str = "exact",
           halo: int = 0, max_scale: float = 0.0, eps: float = 1e-3, eta: float = 1e-3, strict: bool = False,
           out: torch.Tensor | None = None, stream=None, iterations: int = 1,
           hex_spacing: float = 0.5, rel_bound: float = 1e-3, boundary: str = "zero",
           map_lut: bool = False, staging: str = "l1") -> torch.Tensor:
    """Space-variant elliptical box-spline filter fbar[n] = sum_k f[k] beta_{a(n)}(n-k).

    N = 4 or 6 directions; N = 6 runs on the hexagonal lattice of spacing
    hex_spacing (the C header describes the transfer of the image to it).
    iterations = m > 1 applies the iterated box spline of Sec. 3.3 (m passes
    with the widths a / sqrt(m)).  rel_bound: the six-directional map's lower
    bound p_k >= max(eps, rel_bound * sum p) (see bsf_opts).  boundary: "zero"
    (f = 0 outside the image) or "reflect" (half-sample symmetric extension).
    map_lut: N = 6 only, read the map from its table instead of solving it per
    pixel (an approximation; see bsf_opts.map_lut).  staging: "l1" or "tma",
    how the four-directional exact stencil reads its buffer (same results)."""
    img = _as4d(image)
    if not img.is_cuda:
        raise ValueError("image must be a CUDA tensor")
    if img.dtype not in (torch.uint8, torch.float32):
        raise ValueError("image dtype must be uint8 or float32")
    img = img.contiguous()
    B, C, H, W = img.shape
    prm = params if params.dim() == 4 else params[None]
    if prm.dtype != torch.float32 or not prm.is_cuda:
        raise ValueError("params must be a float32 CUDA tensor")
    prm = prm.contiguous()
    K = N if kind == "scales" else 3
    if tuple(prm.shape) != (B, K, H, W):
        raise ValueError(f"params shape {tuple(prm.shape)} != {(B, K, H, W)}")
    if out is None:
        out = torch.empty((B, C, H, W), dtype=torch.float32, device=img.device)
    dtype = L.BSF_U8 if img.dtype == torch.uint8 else L.BSF_F32
    opts = make_opts(precision, halo, max_scale, eps, eta, strict, iterations, hex_spacing, rel_bound, boundary,
                     map_lut, staging)
    rc = L.bsf_filter(context(img.device), img.data_ptr(), dtype, B, C, H, W, N, prm.data_ptr(), _KINDS[kind],
                      opts, out.data_ptr(), _stream_ptr(stream))
    L.check(rc, "bsf_filter")
    return out.reshape(image.shape) if image.dim() < 4 else out


def scales_from_cov(params: torch.Tensor, kind: str = "srt", N: int = 4, eps: float = 1e-3, eta: float = 1e-3,
                    stream=None, rel_bound: float = 1e-3, map_lut: bool = False):
    """Per-pixel optimal scale vectors (Sec. 3.2.2): (3, ...) planes -> ((N, ...), flags uint8)."""
    prm = params.contiguous()
    if prm.dtype != torch.float32 or not prm.is_cuda or prm.shape[0] != 3:
        raise ValueError("params must be a float32 CUDA tensor of shape (3, ...)")
    npix = prm[0].numel()
    scales = torch.empty((N,) + tuple(prm.shape[1:]), dtype=torch.float32, device=prm.device)
    flags = torch.empty(tuple(prm.shape[1:]), dtype=torch.uint8, device=prm.device)
    opts = make_opts(eps=eps, eta=eta, rel_bound=rel_bound, map_lut=map_lut)
    rc = L.bsf_scales_from_cov(context(prm.device), prm.data_ptr(), _KINDS[kind], npix, N, opts,
                               scales.data_ptr(), flags.data_ptr(), _stream_ptr(stream))
    L.check(rc, "bsf_scales_from_cov")
    return scales, flags


def preintegrate(image: torch.Tensor, halo: int, precision: str = "exact", N: int = 4, stream=None) -> torch.Tensor:
    """Algorithm 1 step 2 for one (H,W) image: the pre-integrated buffer as a
    tensor of shape (H+2P, W+2P) (int64 / 16-byte pairs as int64 (...,2) / float64)."""
    if image.dim() != 2 or not image.is_cuda:
        raise ValueError("image must be a 2-D CUDA tensor")
    img = image.contiguous()
    H, W = img.shape
    dtype = L.BSF_U8 if img.dtype == torch.uint8 else L.BSF_F32
    prec = _PREC[precision]
    nbytes = L.bsf_buffer_bytes(dtype, H, W, N, halo, prec)
    Hp, Wp = H + 2 * halo, W + 2 * halo
    if prec == L.BSF_PREC_FP64:
        buf = torch.empty((Hp, Wp), dtype=torch.float64, device=img.device)
    elif dtype == L.BSF_U8:
        buf = torch.empty((Hp, Wp), dtype=torch.int64, device=img.device)
    else:
        buf = torch.empty((Hp, Wp, 2), dtype=torch.int64, device=img.device)
    assert buf.numel() * buf.element_size() == nbytes
    rc = L.bsf_preintegrate(context(img.device), img.data_ptr(), dtype, H, W, N, halo, prec, buf.data_ptr(),
                            _stream_ptr(stream))
    L.check(rc, "bsf_preintegrate")
    return buf


def apply(buffer: torch.Tensor, image_dtype: torch.dtype, H: int, W: int, halo: int, params: torch.Tensor,
          kind: str = "scales", precision: str = "exact", N: int = 4, eps: float = 1e-3, eta: float = 1e-3,
          stream=None) -> torch.Tensor:
    """Algorithm 1 step 3 on a buffer from preintegrate(): (H, W) float32."""
    dtype = L.BSF_U8 if image_dtype == torch.uint8 else L.BSF_F32
    prm = params.contiguous()
    out = torch.empty((H, W), dtype=torch.float32, device=buffer.device)
    opts = make_opts(precision, halo=halo, eps=eps, eta=eta)
    rc = L.bsf_apply(context(buffer.device), buffer.data_ptr(), dtype, H, W, N, halo, prm.data_ptr(), _KINDS[kind],
                     opts, out.data_ptr(), _stream_ptr(stream))
    L.check(rc, "bsf_apply")
    return out


def structure_cov(image: torch.Tensor, sigma_w: float, sigma0: float, tau: float, stream=None) -> torch.Tensor:
    """Sec. 4.2: the adaptive covariance field of feature-preserving smoothing,
    (B, 3, H, W) float32 (C11, C12, C22) for an image of shape (H,W), (C,H,W) or
    (B,C,H,W): a window of the area of an isotropic Gaussian of std sigma0,
    stretched along the local orientation given by the structure tensor
    (window std sigma_w); tau is the gradient energy below which the window
    stays isotropic."""
    img = _as4d(image)
    if not img.is_cuda or img.dtype not in (torch.uint8, torch.float32):
        raise ValueError("image must be a uint8 or float32 CUDA tensor")
    img = img.contiguous()
    B, C, H, W = img.shape
    cov = torch.empty((B, 3, H, W), dtype=torch.float32, device=img.device)
    dtype = L.BSF_U8 if img.dtype == torch.uint8 else L.BSF_F32
    rc = L.bsf_structure_cov(context(img.device), img.data_ptr(), dtype, B, C, H, W, sigma_w, sigma0, tau,
                             cov.data_ptr(), _stream_ptr(stream))
    L.check(rc, "bsf_structure_cov")
    return cov


def adaptive_smooth(image: torch.Tensor, sigma_w: float = 2.0, sigma0: float = 1.0, tau: float = 0.005,
                    iterations: int = 1, stream=None) -> torch.Tensor:
    """Feature-preserving smoothing (Sec. 4.2): the filter with the covariance
    field of structure_cov, on the same image (output shaped like the input)."""
    cov = structure_cov(image, sigma_w, sigma0, tau, stream=stream)
    img = _as4d(image)
    out = filter(img, cov, kind="cov", stream=stream, iterations=iterations)
    return out.reshape(image.shape) if image.dim() < 4 else out


def device_status(device=None, stream=None) -> int:
    """Synchronise the stream and return (and clear) the device status bits."""
    return L.bsf_get_device_status(context(device), _stream_ptr(stream))


def halo_for(max_scale: float, kind: str = "srt") -> int:
    """Padding that covers every tap for fields whose largest footprint is bounded by max_scale
    (the same rule the library applies for opts.max_scale)."""
    import math
    ext = (2.41422 if kind == "scales" else 8.3640) * max_scale
    return int(math.ceil(0.5 * ext)) + 4


def filter_backward(image: torch.Tensor, scales: torch.Tensor, grad_out: torch.Tensor, need_image: bool = True,
                    need_scales: bool = True, N: int = 4, halo: int = 0, max_scale: float = 0.0, stream=None,
                    iterations: int = 1):
    """Gradients of sum(grad_out * filter(image, scales, iterations=m)) w.r.t. image and scales (kind "scales")."""
    img = _as4d(image).contiguous()
    B, C, H, W = img.shape
    sc = (scales if scales.dim() == 4 else scales[None]).contiguous()
    if tuple(sc.shape) != (B, 4, H, W) or sc.dtype != torch.float32:
        raise ValueError("scales must be float32 of shape (B,4,H,W)")
    g = grad_out.reshape(B, C, H, W).contiguous().to(torch.float32)
    gi = torch.empty((B, C, H, W), dtype=torch.float32, device=img.device) if need_image else None
    gs = torch.empty((B, 4, H, W), dtype=torch.float32, device=img.device) if need_scales else None
    dtype = L.BSF_U8 if img.dtype == torch.uint8 else L.BSF_F32
    opts = make_opts("exact", halo, max_scale, iterations=iterations)
    rc = L.bsf_filter_backward(context(img.device), img.data_ptr(), dtype, B, C, H, W, N, sc.data_ptr(),
                               g.data_ptr(), gi.data_ptr() if gi is not None else None,
                               gs.data_ptr() if gs is not None else None, opts, _stream_ptr(stream))
    L.check(rc, "bsf_filter_backward")
    if gi is not None and image.dim() < 4:
        gi = gi.reshape(image.shape)
    if gs is not None and scales.dim() < 4:
        gs = gs.reshape(scales.shape)
    return gi, gs


class BoxSplineFilter(torch.autograd.Function):
    """Differentiable space-variant box-spline filter: out = filter(image, scales).

    Gradients flow to the float32 image and to the per-pixel scale vectors
    (kind "scales"); both come from the CUDA adjoint (bsf_filter_backward).
    """

    @staticmethod
    def forward(ctx, image, scales, halo: int = 0, max_scale: float = 0.0, iterations: int = 1):
        out = filter(image, scales, kind="scales", halo=halo, max_scale=max_scale, iterations=iterations)
        ctx.save_for_backward(image, scales)
        ctx.halo = halo
        ctx.max_scale = max_scale
        ctx.iterations = iterations
        return out

    @staticmethod
    def backward(ctx, grad_out):
        image, scales = ctx.saved_tensors
        gi, gs = filter_backward(image, scales, grad_out, need_image=ctx.needs_input_grad[0],
                                 need_scales=ctx.needs_input_grad[1], halo=ctx.halo, max_scale=ctx.max_scale,
                                 iterations=ctx.iterations)
        return gi, gs, None, None, None


def box_spline_filter(image: torch.Tensor, scales: torch.Tensor, halo: int = 0, max_scale: float = 0.0,
                      iterations: int = 1):
    """Autograd entry point of the filter with a learnable scale field (iterations = m:
    the m-fold iterated spline of Sec. 3.3)."""
    return BoxSplineFilter.apply(image, scales, halo, max_scale, iterations)
