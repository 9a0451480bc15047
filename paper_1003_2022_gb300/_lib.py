"""ctypes binding of libbsf.so: the C ABI of include/bsf.h, same names.

Argument marshalling only.  Every step of the filter runs in the CUDA
library; if the library is missing this module raises instead of falling
back to anything else.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libbsf.so")

BSF_OK = 0
BSF_EINVAL = 1
BSF_EUNSUPPORTED = 2
BSF_ENOMEM = 3
BSF_ECUDA = 4
BSF_EHALO = 5
BSF_EINFEASIBLE = 6
BSF_EBADSCALE = 7
BSF_ERANGE = 8
BSF_ENOSCRATCH = 9
BSF_ETIMEOUT = 10
NOALLOC_SCRATCH_BYTES = 32 << 20

BSF_U8 = 0
BSF_F32 = 1

BSF_PARAM_SCALES = 0
BSF_PARAM_COV = 1
BSF_PARAM_SRT = 2

BSF_BOUNDARY_ZERO = 0
BSF_BOUNDARY_REFLECT = 1
BSF_STAGING_L1 = 0
BSF_STAGING_TMA = 1

BSF_PREC_EXACT = 0
BSF_PREC_FP64 = 1

# names exported by the library (must match include/bsf.h)
EXPORTS = [
    "bsf_default_opts", "bsf_create", "bsf_destroy", "bsf_filter", "bsf_scales_from_cov",
    "bsf_buffer_bytes", "bsf_preintegrate", "bsf_apply", "bsf_get_device_status", "bsf_status_string",
    "bsf_profile_begin", "bsf_profile_end", "bsf_filter_noalloc", "bsf_filter_backward", "bsf_filter_host",
    "bsf_host_sync", "bsf_structure_cov", "bsf_query_workspace", "bsf_set_wait_limit",
]


class bsf_opts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("eps", ctypes.c_float),
        ("eta", ctypes.c_float),
        ("strict", ctypes.c_int),
        ("halo", ctypes.c_int),
        ("max_scale", ctypes.c_float),
        ("iterations", ctypes.c_int),
        ("hex_spacing", ctypes.c_float),
        ("rel_bound", ctypes.c_float),
        ("boundary", ctypes.c_int),
        ("map_lut", ctypes.c_int),
        ("staging", ctypes.c_int),
    ]


class BsfError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: bsf status {code} ({status_string(code)})")


_lib = None


def load(path: str | None = None):
    """Load libbsf.so (built by paper_1003_2022_gb300.build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run `python -m paper_1003_2022_gb300.build`)")
    lib = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    op = ctypes.POINTER(bsf_opts)
    lib.bsf_default_opts.restype = None
    lib.bsf_default_opts.argtypes = [op]
    lib.bsf_create.restype = i32
    lib.bsf_create.argtypes = [ctypes.POINTER(vp), i32]
    lib.bsf_destroy.restype = i32
    lib.bsf_destroy.argtypes = [vp]
    lib.bsf_filter.restype = i32
    lib.bsf_filter.argtypes = [vp, vp, i32, i64, i64, i64, i64, i32, vp, i32, op, vp, vp]
    lib.bsf_scales_from_cov.restype = i32
    lib.bsf_scales_from_cov.argtypes = [vp, vp, i32, i64, i32, op, vp, vp, vp]
    lib.bsf_buffer_bytes.restype = i32
    lib.bsf_buffer_bytes.argtypes = [i32, i64, i64, i32, i32, i32, ctypes.POINTER(ctypes.c_size_t)]
    lib.bsf_preintegrate.restype = i32
    lib.bsf_preintegrate.argtypes = [vp, vp, i32, i64, i64, i32, i32, i32, vp, vp]
    lib.bsf_apply.restype = i32
    lib.bsf_apply.argtypes = [vp, vp, i32, i64, i64, i32, i32, vp, i32, op, vp, vp]
    lib.bsf_get_device_status.restype = i32
    lib.bsf_get_device_status.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int)]
    lib.bsf_profile_begin.restype = i32
    lib.bsf_profile_begin.argtypes = [vp]
    lib.bsf_profile_end.restype = i32
    lib.bsf_profile_end.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_int)]
    lib.bsf_filter_backward.restype = i32
    lib.bsf_filter_backward.argtypes = [vp, vp, i32, i64, i64, i64, i64, i32, vp, vp, vp, vp, op, vp]
    lib.bsf_filter_noalloc.restype = i32
    lib.bsf_filter_noalloc.argtypes = [vp, i32, i64, i64, i32, vp, i32, op, vp, vp]
    lib.bsf_filter_host.restype = i32
    lib.bsf_filter_host.argtypes = [vp, vp, i32, i64, i64, i64, i64, i32, vp, i32, op, vp]
    lib.bsf_host_sync.restype = i32
    lib.bsf_host_sync.argtypes = [vp]
    lib.bsf_structure_cov.restype = i32
    lib.bsf_structure_cov.argtypes = [vp, vp, i32, i64, i64, i64, i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                      vp, vp]
    lib.bsf_query_workspace.restype = i32
    lib.bsf_query_workspace.argtypes = [vp, i32, i64, i64, i64, i64, i32, i32, op, ctypes.POINTER(ctypes.c_size_t)]
    lib.bsf_set_wait_limit.restype = None
    lib.bsf_set_wait_limit.argtypes = [ctypes.c_uint]
    lib.bsf_status_string.restype = ctypes.c_char_p
    lib.bsf_status_string.argtypes = [i32]
    _lib = lib
    return lib


def status_string(code: int) -> str:
    try:
        return load().bsf_status_string(int(code)).decode()
    except Exception:
        return "?"


def check(code: int, where: str) -> None:
    if code != BSF_OK:
        raise BsfError(code, where)


def default_opts() -> bsf_opts:
    o = bsf_opts()
    load().bsf_default_opts(ctypes.byref(o))
    return o


# thin same-name wrappers (pointers are plain ints)
def bsf_create(device: int) -> int:
    h = ctypes.c_void_p()
    check(load().bsf_create(ctypes.byref(h), int(device)), "bsf_create")
    return h.value


def bsf_destroy(ctx: int) -> None:
    check(load().bsf_destroy(ctx), "bsf_destroy")


def bsf_filter(ctx, image, dtype, B, C, H, W, N, params, kind, opts, out, stream) -> int:
    return load().bsf_filter(ctx, image, dtype, B, C, H, W, N, params, kind,
                             ctypes.byref(opts) if opts is not None else None, out, stream)


def bsf_scales_from_cov(ctx, params, kind, npix, N, opts, scales, flags, stream) -> int:
    return load().bsf_scales_from_cov(ctx, params, kind, npix, N,
                                      ctypes.byref(opts) if opts is not None else None, scales, flags, stream)


def bsf_buffer_bytes(dtype, H, W, N, halo, precision) -> int:
    n = ctypes.c_size_t()
    check(load().bsf_buffer_bytes(dtype, H, W, N, halo, precision, ctypes.byref(n)), "bsf_buffer_bytes")
    return n.value


def bsf_query_workspace(ctx, dtype, B, C, H, W, N, kind, opts) -> int:
    """Scratch bytes the context needs for bsf_filter at this shape (host-only)."""
    n = ctypes.c_size_t()
    check(load().bsf_query_workspace(ctx, dtype, B, C, H, W, N, kind,
                                     ctypes.byref(opts) if opts is not None else None, ctypes.byref(n)),
          "bsf_query_workspace")
    return n.value


def bsf_preintegrate(ctx, image, dtype, H, W, N, halo, precision, buffer, stream) -> int:
    return load().bsf_preintegrate(ctx, image, dtype, H, W, N, halo, precision, buffer, stream)


def bsf_apply(ctx, buffer, dtype, H, W, N, halo, params, kind, opts, out, stream) -> int:
    return load().bsf_apply(ctx, buffer, dtype, H, W, N, halo, params, kind,
                            ctypes.byref(opts) if opts is not None else None, out, stream)


def bsf_filter_backward(ctx, image, dtype, B, C, H, W, N, scales, grad_out, grad_image, grad_scales, opts,
                        stream) -> int:
    return load().bsf_filter_backward(ctx, image, dtype, B, C, H, W, N, scales, grad_out, grad_image, grad_scales,
                                      ctypes.byref(opts) if opts is not None else None, stream)


def bsf_filter_host(ctx, image_host, dtype, B, C, H, W, N, params_host, kind, opts, out_host) -> int:
    """Pipelined filter of host buffers (returns before the work completes; see bsf_host_sync)."""
    return load().bsf_filter_host(ctx, image_host, dtype, B, C, H, W, N, params_host, kind,
                                  ctypes.byref(opts) if opts is not None else None, out_host)


def bsf_structure_cov(ctx, image, dtype, B, C, H, W, sigma_w, sigma0, tau, cov, stream) -> int:
    return load().bsf_structure_cov(ctx, image, dtype, B, C, H, W, float(sigma_w), float(sigma0), float(tau), cov,
                                    stream)


def bsf_host_sync(ctx) -> int:
    return load().bsf_host_sync(ctx)


def bsf_filter_noalloc(image, dtype, H, W, N, params, kind, opts, out, stream) -> int:
    """Allocation-free filter of one image (scratch is a fixed array inside the library)."""
    return load().bsf_filter_noalloc(image, dtype, H, W, N, params, kind,
                                     ctypes.byref(opts) if opts is not None else None, out, stream)


def bsf_set_wait_limit(polls: int) -> None:
    """Bound of the device waits between row bands (0: the default)."""
    load().bsf_set_wait_limit(int(polls))


def bsf_profile_begin(ctx) -> None:
    check(load().bsf_profile_begin(ctx), "bsf_profile_begin")


def bsf_profile_end(ctx):
    """(ms of pre-integration, ms of the finite difference, launches) since bsf_profile_begin."""
    a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    check(load().bsf_profile_end(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)), "bsf_profile_end")
    return a.value, b.value, n.value


def bsf_get_device_status(ctx, stream) -> int:
    s = ctypes.c_int()
    check(load().bsf_get_device_status(ctx, stream, ctypes.byref(s)), "bsf_get_device_status")
    return s.value
