"""Backward pass (adjoint) of the CUDA path against the FP64 oracle.

* dL/dimage against the plain transpose sum_n g[n] beta_{a(n)}(n-k);
* dL/dscales against central finite differences (h = 1e-3, FP64) of the
  plain definition, on sampled pixels;
* the batch-8 1024x1024 learnable-scale workload through the autograd
  Function, checked on 64x64 crops.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1003_2022_gb300 import api, synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device(DEV)


def _nerr(got, ref):
    return float(np.abs(np.asarray(got, np.float64) - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("dtype", ["f32", "u8"])
def test_grad_image_matches_transpose(dtype):
    dev = _cuda()
    H, W = 48, 56
    rng = np.random.default_rng(7)
    f = synth.image(H, W, seed=7, dtype=dtype)
    a = rng.uniform(0.7, 7.0, size=(4, H, W)).astype(np.float32)
    g = rng.standard_normal((H, W)).astype(np.float32)
    gi, _ = api.filter_backward(torch.from_numpy(f).to(dev), torch.from_numpy(a).to(dev),
                                torch.from_numpy(g).to(dev), need_scales=False, max_scale=7.0)
    assert api.device_status(dev) == 0
    ref = O.adjoint4(g.astype(np.float64), a.astype(np.float64), np.arange(H * W)).reshape(H, W)
    assert _nerr(gi.cpu().numpy(), ref) < 1e-5


def test_grad_scales_matches_finite_differences():
    dev = _cuda()
    H, W = 40, 44
    rng = np.random.default_rng(8)
    f = synth.image(H, W, seed=8, dtype="f32")
    a = rng.uniform(1.0, 6.0, size=(4, H, W)).astype(np.float32)
    g = rng.standard_normal((H, W)).astype(np.float32)
    _, gs = api.filter_backward(torch.from_numpy(f).to(dev), torch.from_numpy(a).to(dev),
                                torch.from_numpy(g).to(dev), need_image=False, max_scale=6.0)
    assert api.device_status(dev) == 0
    gs = gs.cpu().numpy().astype(np.float64)
    idx = rng.choice(H * W, size=120, replace=False)
    fd = O.direct4_grad_fd(f.astype(np.float64), a.astype(np.float64), idx, h=1e-3)
    ref = fd * g.ravel()[idx].astype(np.float64)
    got = gs.reshape(4, -1)[:, idx]
    assert _nerr(got, ref) < 1e-4


def test_autograd_learnable_scales_workload():
    """Batch 8 of 1024x1024 f32 images with a learnable scale field a_k in
    [1, 24] (four smooth seeded fields from the shared generator, so both
    sides start from the same bytes); loss = sum(w * out) with a seeded
    weight w; gradients checked on 64x64 crops."""
    dev = _cuda()
    imgs, a0_np = synth.batch_inputs("b8_1024_f32_scales", seed=40)
    B, _, H, W = imgs.shape
    a0 = torch.from_numpy(a0_np).to(dev)
    image = torch.from_numpy(imgs).to(dev).requires_grad_(True)
    scales = a0.clone().requires_grad_(True)
    wgt = torch.from_numpy(np.random.default_rng(3).standard_normal((B, 1, H, W)).astype(np.float32)).to(dev)
    out = api.box_spline_filter(image, scales, max_scale=24.0)
    loss = (out * wgt).sum()
    loss.backward()
    assert api.device_status(dev) == 0
    gimg = image.grad.detach().cpu().numpy()
    gsc = scales.grad.detach().cpu().numpy()
    a_np = a0_np.astype(np.float64)
    w_np = wgt.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(11)
    for b in (0, 5):
        y0, x0 = int(rng.integers(100, H - 200)), int(rng.integers(100, W - 200))
        # the crop plus a margin covering every footprint that reaches it
        M = 40
        sl = (slice(y0 - M, y0 + 64 + M), slice(x0 - M, x0 + 64 + M))
        fw, aw, ww = imgs[b, 0][sl].astype(np.float64), a_np[b][:, sl[0], sl[1]], w_np[b, 0][sl]
        hh, wwid = fw.shape
        loc = np.array([(M + r) * wwid + (M + c) for r in range(0, 64, 7) for c in range(0, 64, 9)])
        ref_i = O.adjoint4(ww, aw, loc)
        got_i = np.array([gimg[b, 0][y0 + (p // wwid - M), x0 + (p % wwid - M)] for p in loc])
        assert _nerr(got_i, ref_i) < 1e-5
        fd = O.direct4_grad_fd(fw, aw, loc[:40], h=1e-3) * ww.ravel()[loc[:40]]
        got_s = np.stack([[gsc[b, k][y0 + (p // wwid - M), x0 + (p % wwid - M)] for p in loc[:40]]
                          for k in range(4)])
        assert _nerr(got_s, fd) < 1e-4


@pytest.mark.parametrize("m", [2, 3])
def test_iterated_filter_gradients(m):
    """The m-fold iterated filter (Sec. 3.3) through autograd: the image gradient
    equals the transpose applied m times (each pass with a / sqrt(m)), the
    scale gradient the central differences of the iterated plain definition."""
    dev = _cuda()
    H, W = 26, 30
    rng = np.random.default_rng(50 + m)
    f = synth.image(H, W, seed=50 + m, dtype="f32")
    a = rng.uniform(1.0, 5.0, size=(4, H, W)).astype(np.float32)
    g = rng.standard_normal((H, W)).astype(np.float32)
    fi = torch.from_numpy(f).to(dev).requires_grad_(True)
    sc = torch.from_numpy(a).to(dev).requires_grad_(True)
    (api.box_spline_filter(fi, sc, max_scale=5.0, iterations=m) * torch.from_numpy(g).to(dev)).sum().backward()
    assert api.device_status(dev) == 0
    a64 = a.astype(np.float64) / np.sqrt(m)
    gref = g.astype(np.float64)
    allpx = np.arange(H * W)
    for _ in range(m):
        gref = O.adjoint4(gref, a64, allpx).reshape(H, W)
    assert _nerr(fi.grad.cpu().numpy(), gref) < 1e-5
    # scale gradient on sampled pixels: central differences of sum(g * K^m f)
    idx = rng.choice(H * W, size=12, replace=False)
    h = 1e-3
    f64, g64, a0 = f.astype(np.float64), g.astype(np.float64), a.astype(np.float64)
    fd = np.empty((4, idx.size))
    for k in range(4):
        for j, pix in enumerate(idx):
            ap, am = a0.copy(), a0.copy()
            ap[k].flat[pix] += h
            am[k].flat[pix] -= h
            fd[k, j] = (np.sum(g64 * O.direct4_iterated(f64, ap, m)) - np.sum(g64 * O.direct4_iterated(f64, am, m))) / (2 * h)
    got = sc.grad.cpu().numpy().reshape(4, -1)[:, idx]
    assert _nerr(got, fd) < 1e-4
