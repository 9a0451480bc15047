"""The six-directional filter's window planner (csrc/hex6_plan.cpp), built on the
CPU with the host compiler through a small C harness (tests/hex6_plan_harness.cpp).

From the largest footprint half-extents of every 16 x 16 block the planner makes
the output tiles (16 x 16 where the footprints are small, 64 x 64, and groups of
64-tiles where they are large), one lattice window per tile, and the chunks the
kernels are launched on.  Checked here: every output pixel lies in exactly one
tile; the tile classes follow their rules; every tap of every pixel reads inside
its tile's window with the stencil's margins (so the kernel's halo check never
fires); the chunks respect their limits and lay the windows out without overlap;
bad extents are rejected."""
import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1003_2022_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SQ3 = math.sqrt(3.0)
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    out = str(tmp_path_factory.mktemp("plan") / "libhex6plan.so")
    cmd = [cxx, "-O1", "-std=c++17", "-shared", "-fPIC", "-I", CUDA_INC, "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "paper_1003_2022_gb300", "csrc", "hex6_plan.cpp"),
           os.path.join(HERE, "hex6_plan_harness.cpp"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    L = ctypes.CDLL(out)
    L.plan_run.restype = ctypes.c_int
    L.plan_run.argtypes = [ctypes.c_longlong] * 4 + [ctypes.c_double, ctypes.c_void_p, ctypes.c_ulonglong,
                                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.plan_tiles.argtypes = [ctypes.c_void_p]
    L.plan_chunks.argtypes = [ctypes.c_void_p]
    return L


def _plan(L, B, C, H, W, h, ext, budget):
    e = np.ascontiguousarray(ext, np.float32).view(np.uint32)
    nt, nc = ctypes.c_int(), ctypes.c_int()
    st = L.plan_run(B, C, H, W, h, e.ctypes.data, budget, ctypes.byref(nt), ctypes.byref(nc))
    if st != 0:
        return st, None, None
    tiles = np.zeros((nt.value, 10), np.int64)
    chunks = np.zeros((nc.value, 4), np.int64)
    L.plan_tiles(tiles.ctypes.data)
    L.plan_chunks(chunks.ctypes.data)
    return st, tiles, chunks


def _block_extents(B, H, W, seed, smax=48.0):
    """Largest half-extents (ex, ey) per 16 x 16 block from footprints of
    sigma 1-smax px (smooth fields) with an orientation-dependent aspect."""
    fy, fx = -(-H // 16), -(-W // 16)
    ext = np.zeros((B, fy, fx, 2), np.float32)
    for b in range(B):
        p = synth.srt_field(H, W, seed=seed + b, sigma=(1.0, smax), rho=(1.0, 6.0))
        s, th = p[0].astype(np.float64), p[2].astype(np.float64)
        ex = 4.25 * s * (0.6 + 0.4 * np.abs(np.cos(th)))
        ey = 4.25 * s * (0.6 + 0.4 * np.abs(np.sin(th)))
        pad = lambda a: np.pad(a, ((0, fy * 16 - H), (0, fx * 16 - W)))
        ext[b, ..., 0] = pad(ex).reshape(fy, 16, fx, 16).max(axis=(1, 3))
        ext[b, ..., 1] = pad(ey).reshape(fy, 16, fx, 16).max(axis=(1, 3))
    return ext


def _inside(t, x, y, h):
    """The stencil's halo test for taps at (x, y): cell (i0, j0) of the lattice
    point, storage row and column, and the margins its 24 points need."""
    tt = 2.0 * y / (h * SQ3)
    ss = x / h - 0.5 * tt
    i0, j0 = np.floor(ss).astype(np.int64), np.floor(tt).astype(np.int64)
    rr = j0 - t[2]
    cc = i0 - t[1] + 2 * rr
    return (rr >= 2) & (rr + 3 < t[4]) & (cc >= 6) & (cc + 9 < t[3])


# sigma up to 48 px at spacing 0.5 and 1; at 0.25 the lattice has twice the
# columns per pixel, and footprints beyond about 500 px along x do not fit a window
@pytest.mark.parametrize("H,W,h,smax", [(333, 517, 0.5, 48.0), (260, 300, 0.25, 20.0), (70, 1100, 1.0, 48.0)])
def test_plan_covers_the_image_and_windows_hold_the_taps(lib, H, W, h, smax):
    B, C = 2, 3
    ext = _block_extents(B, H, W, seed=40 + H, smax=smax)
    budget = 1 << 30
    st, tiles, chunks = _plan(lib, B, C, H, W, h, ext, budget)
    assert st == 0
    maxc = lib.plan_max_cols()
    cover = np.zeros((B, H, W), np.int32)
    shapes = {(16, 16), (64, 64), (128, 64), (256, 64), (256, 128)}
    for t in tiles:
        off, il, j0w, ncol, nrow, b, x0, y0, w, hh = (int(v) for v in t)
        assert (w, hh) in shapes and ncol <= maxc
        assert x0 % 16 == 0 and y0 % 16 == 0 and (w == 16 or (x0 % w == 0 and y0 % hh == 0))
        x1, y1 = min(W, x0 + w), min(H, y0 + hh)
        cover[b, y0:y1, x0:x1] += 1
        blocks = ext[b, y0 // 16:-(-y1 // 16), x0 // 16:-(-x1 // 16)]
        m64 = blocks.max(axis=-1)
        if w == 16:        # a 64-tile cut up: its largest half-extent is below 16 px
            t64 = ext[b, (y0 // 64) * 4:(y0 // 64) * 4 + 4, (x0 // 64) * 4:(x0 // 64) * 4 + 4].max()
            assert t64 < 16.0
        elif w * hh > 64 * 64:  # a group: every 64-tile at least 32 px and half the largest
            sub = [ext[b, yy:yy + 4, xx:xx + 4].max() for yy in range(y0 // 16, -(-y1 // 16), 4)
                   for xx in range(x0 // 16, -(-x1 // 16), 4)]
            assert min(sub) >= 32.0 and min(sub) >= 0.5 * max(sub)
        else:
            assert m64.max() >= 16.0
        # every tap of every pixel of every block: the footprint box of the block,
        # shifted as the stencil's first tap is, sampled along its boundary
        for by in range(blocks.shape[0]):
            for bx in range(blocks.shape[1]):
                ex, ey = (float(v) for v in blocks[by, bx])
                px0, py0 = x0 + 16 * bx, y0 + 16 * by
                px1, py1 = min(x1, px0 + 16) - 1, min(y1, py0 + 16) - 1
                xl, xh = px0 - ex - 0.5 * h, px1 + ex - 0.5 * h
                yl, yh = py0 - ey - 1.5 * SQ3 * h, py1 + ey - 1.5 * SQ3 * h
                ys = np.linspace(yl, yh, 64)
                xs = np.linspace(xl, xh, 64)
                pts_x = np.concatenate([np.full(64, xl), np.full(64, xh), xs, xs])
                pts_y = np.concatenate([ys, ys, np.full(64, yl), np.full(64, yh)])
                assert _inside(t, pts_x, pts_y, h).all(), (t, bx, by)
    assert (cover == 1).all()
    # chunks: consecutive runs of one tile shape, windows packed without overlap
    assert chunks[0, 0] == 0 and chunks[-1, 1] == len(tiles)
    assert (chunks[1:, 0] == chunks[:-1, 1]).all()
    for first, last, cols, nbytes in chunks:
        ts = tiles[first:last]
        assert 0 < last - first <= 65535 and nbytes <= budget
        assert len({(int(a), int(b)) for a, b in ts[:, 8:10]}) == 1
        sizes = C * ts[:, 3] * ts[:, 4]
        assert (ts[:, 0] == np.concatenate([[0], np.cumsum(sizes)[:-1]])).all()
        assert nbytes == 16 * sizes.sum() and cols == ts[:, 3].max()


def test_plan_groups_large_footprints(lib):
    """Uniform half-extents on 512 x 512: 40 px, 4 x 2 groups throughout;
    20 px (at least 16, below 32): 64-tiles; 3 px: 16-tiles."""
    H = W = 512
    fy = fx = 32
    for e, shape in [(40.0, (256, 128)), (20.0, (64, 64)), (3.0, (16, 16))]:
        ext = np.full((1, fy, fx, 2), e, np.float32)
        st, tiles, _ = _plan(lib, 1, 1, H, W, 0.5, ext, 1 << 30)
        assert st == 0
        assert {(int(a), int(b)) for a, b in tiles[:, 8:10]} == {shape}


def test_plan_rejects_bad_extents(lib):
    H, W = 100, 100
    ext = np.full((1, 7, 7, 2), 5.0, np.float32)
    for bad in (np.nan, np.inf, -1.0, 2e5):
        e = ext.copy()
        e[0, 3, 3, 0] = bad
        st, _, _ = _plan(lib, 1, 1, H, W, 0.5, e, 1 << 30)
        assert st == 1  # BSF_EINVAL
    # a window wider than the pre-integration holds
    e = np.full((1, 7, 7, 2), 900.0, np.float32)
    assert _plan(lib, 1, 1, H, W, 0.5, e, 1 << 30)[0] == 1


def _six_sums(mu):
    """The pre-integration's six running sums in a window's storage coordinates
    (row r, column c; the directions' backward steps in (rows, columns) are
    0: (0, 1), 30: (1, 3), 60: (1, 2), 90: (2, 3), 120: (1, 1), 150: (1, 0)),
    nested in that order as the kernel nests them, in exact integers."""
    S = np.array(mu, dtype=object)
    for dr, dc in ((0, 1), (1, 3), (1, 2), (2, 3), (1, 1), (1, 0)):
        T = S.copy()
        nrow, ncol = S.shape
        for r in range(nrow):
            for c in range(ncol):
                if r >= dr and c >= dc and (dr or dc):
                    T[r, c] = S[r, c] + T[r - dr, c - dc]
        S = T
    return S


def test_range_bound_of_the_window_sums():
    """The bound the pre-integration tests against 2^126 (no running sum can have
    wrapped 128 bits): |partial sums| <= max |mass| * ncol * n30 * n60 * n90 *
    n120 * nrow, with n_k the longest line of direction k in the window.  Exact
    sums of constant and sign-alternating masses stay within it, and the
    constant case comes within a modest factor of it."""
    for nrow, ncol in ((7, 11), (12, 30), (20, 9)):
        n30 = min(nrow - 1, (ncol - 1) // 3) + 1
        n60 = min(nrow - 1, (ncol - 1) // 2) + 1
        n90 = min((nrow - 1) // 2, (ncol - 1) // 3) + 1
        n120 = min(nrow - 1, ncol - 1) + 1
        bound = ncol * n30 * n60 * n90 * n120 * nrow
        ones = _six_sums(np.ones((nrow, ncol), dtype=object))
        alt = _six_sums(np.fromfunction(lambda r, c: (-1) ** (r + c), (nrow, ncol), dtype=int).astype(object))
        top = max(abs(v) for v in ones.ravel())
        assert top <= bound and max(abs(v) for v in alt.ravel()) <= bound
        assert top * 1000 >= bound
