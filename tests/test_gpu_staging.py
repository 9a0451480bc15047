"""The four-directional exact stencil with its buffer staged in shared memory
by the tensor-copy engine (opts.staging = BSF_STAGING_TMA) against the L1
form and the FP64 oracle.

Both forms evaluate the same exact integer sum (Algorithm 1 step 3 at the
per-pixel dyadic scales) and round once, so their outputs must agree bit for
bit; the oracle comparison (plain definition, 1e-5 normwise) pins the staged
form independently.  Cases: ragged tiles, tiles whose taps fall back to L1
loads (independent random scales per pixel), vertical strips, batches sharing
a parameter field, and a wait limit short enough to run out.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1003_2022_gb300 import _lib as L  # noqa: E402
from paper_1003_2022_gb300 import api, synth  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-5
DEV = "cuda:0"


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device(DEV)


def _nerr(got, ref):
    return float(np.abs(np.asarray(got, np.float64) - ref).max() / np.abs(ref).max())


def _both(f, p, kind, **kw):
    dev = _cuda()
    img, prm = torch.from_numpy(f).to(dev), torch.from_numpy(p).to(dev)
    api.device_status(dev)
    a = api.filter(img, prm, kind=kind, staging="l1", **kw).cpu().numpy()
    sa = api.device_status(dev)
    b = api.filter(img, prm, kind=kind, staging="tma", **kw).cpu().numpy()
    sb = api.device_status(dev)
    return a, sa, b, sb


def _same_bits(a, b):
    return np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("H,W", [(1, 1), (7, 45), (97, 141), (300, 517)])
def test_staged_equals_l1_and_oracle(H, W):
    """u8 image, sigma 1-8, rho 1-8 (smooth fields): ragged 32 x 8 tiles."""
    f = synth.image(H, W, seed=H + W, dtype="u8")
    p = synth.srt_field(H, W, seed=H * W, sigma=(1.0, 8.0), rho=(1.0, 8.0))
    a, sa, b, sb = _both(f, p, "srt", max_scale=8.0)
    assert sa == sb and sa & ~(1 << L.BSF_EINFEASIBLE) == 0
    assert _same_bits(a, b)
    am, _ = O.map4(p.astype(np.float64), O.KIND_SRT)
    idx = np.random.default_rng(H).choice(H * W, size=min(H * W, 300), replace=False)
    ref = O.direct4(f.astype(np.float64), am, idx)
    assert _nerr(b.ravel()[idx], ref) < TOL


def test_staged_with_taps_that_do_not_fit_their_box():
    """Independent random scales in [0.3, 9] per pixel: the cells one tap reads
    spread over more than a 40 x 16 box in most tiles, so those taps read
    through L1 while others are staged."""
    H, W = 96, 130
    f = synth.image(H, W, seed=5, dtype="u8")
    a4 = np.random.default_rng(6).uniform(0.3, 9.0, size=(4, H, W)).astype(np.float32)
    a, sa, b, sb = _both(f, a4, "scales", max_scale=9.0)
    assert sa == sb == 0
    assert _same_bits(a, b)
    ref = O.direct4(f.astype(np.float64), a4.astype(np.float64))
    assert _nerr(b, ref) < TOL


def test_staged_large_kernels_and_batch():
    """sigma 1-32 on a 2 x 2 batch of 256 x 288 images (shared field per batch
    entry): large footprints, so boxes start far from the tile."""
    dev = _cuda()
    B, C, H, W = 2, 2, 256, 288
    f = np.stack([np.stack([synth.image(H, W, seed=10 * b + c, dtype="u8") for c in range(C)]) for b in range(B)])
    p = np.stack([synth.srt_field(H, W, seed=40 + b, sigma=(1.0, 32.0), rho=(1.0, 8.0)) for b in range(B)])
    a, sa, b, sb = _both(f, p, "srt", max_scale=32.0)
    assert sa == sb and sa & ~(1 << L.BSF_EINFEASIBLE) == 0
    assert _same_bits(a, b)
    am, _ = O.map4(p[1].astype(np.float64), O.KIND_SRT)
    idx = np.random.default_rng(2).choice(H * W, size=120, replace=False)
    ref = O.direct4(f[1, 0].astype(np.float64), am, idx)
    assert _nerr(b[1, 0].ravel()[idx], ref) < TOL
    del dev


def test_staged_in_vertical_strips():
    """A u8 row wider than one band CTA holds: the buffer is cut into strips,
    each with its own tensor map origin."""
    H, W = 24, 4300
    f = synth.image(H, W, seed=31, dtype="u8")
    p = synth.srt_field(H, W, seed=31, sigma=(1.0, 4.0), rho=(1.0, 6.0))
    a, sa, b, sb = _both(f, p, "srt", max_scale=4.0)
    assert sa == sb and sa & ~(1 << L.BSF_EINFEASIBLE) == 0
    assert _same_bits(a, b)


def test_staging_is_ignored_by_the_float_form():
    H, W = 40, 70
    f = synth.image(H, W, seed=8, dtype="f32")
    p = synth.srt_field(H, W, seed=8, sigma=(1.0, 4.0), rho=(1.0, 4.0))
    a, sa, b, sb = _both(f, p, "srt", max_scale=4.0)
    assert sa == sb
    assert _same_bits(a, b)


def test_staged_wait_that_runs_out_is_reported():
    """With a one-poll bound the CTAs give up on their copies: BSF_ETIMEOUT is
    raised, their pixels are NaN (each waits, bounded, for its copies before it
    exits), and every pixel that was computed matches the L1 form."""
    dev = _cuda()
    H, W = 128, 160
    f = synth.image(H, W, seed=12, dtype="u8")
    p = synth.srt_field(H, W, seed=12, sigma=(1.0, 6.0), rho=(1.0, 4.0))
    img, prm = torch.from_numpy(f).to(dev), torch.from_numpy(p).to(dev)
    ref = api.filter(img, prm, kind="srt", max_scale=6.0).cpu().numpy()
    api.device_status(dev)
    L.bsf_set_wait_limit(1)
    try:
        out = api.filter(img, prm, kind="srt", max_scale=6.0, staging="tma").cpu().numpy()
        st = api.device_status(dev)
    finally:
        L.bsf_set_wait_limit(0)
    assert st & (1 << L.BSF_ETIMEOUT)
    done = ~np.isnan(out)
    assert done.sum() < out.size
    assert np.array_equal(out[done], ref[done])
    again = api.filter(img, prm, kind="srt", max_scale=6.0, staging="tma").cpu().numpy()
    assert api.device_status(dev) & (1 << L.BSF_ETIMEOUT) == 0
    assert _same_bits(again, ref)
