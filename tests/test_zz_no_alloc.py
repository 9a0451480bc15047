"""bsf_filter_noalloc: the allocation-free entry point for callers that may
not allocate device memory (plugins whose host owns the memory budget,
loops where cudaMalloc/cudaFree would synchronise the device).

Its output must equal the regular bsf_filter output on the same inputs,
within the parity tolerance of the other tests, on two calls in a row (the
second reusing the shared fixed scratch that the first left behind), and the
oracle's plain definition on sampled pixels.  Oversize
images must be refused with BSF_ENOSCRATCH.  This file is collected last on
purpose, and also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1003_2022_gb300 import _lib as L  # noqa: E402
from paper_1003_2022_gb300 import api, synth  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_noalloc_matches_filter_on_two_calls(dtype):
    dev = _dev()
    torch.cuda.set_device(dev)
    H, W = 160, 136
    opts = api.make_opts(max_scale=6.0)
    stream = torch.cuda.current_stream(dev)
    for seed in (3, 4):  # two calls in a row through the shared scratch
        f = torch.from_numpy(synth.image(H, W, seed=seed, dtype=dtype)).to(dev)
        p = torch.from_numpy(synth.srt_field(H, W, seed=seed, sigma=(1.0, 6.0), rho=(1.0, 5.0))).to(dev)
        ref = api.filter(f, p, kind="srt", max_scale=6.0)
        out = torch.full((H, W), float("nan"), dtype=torch.float32, device=dev)
        rc = L.bsf_filter_noalloc(f.data_ptr(), L.BSF_U8 if dtype == "u8" else L.BSF_F32, H, W, 4, p.data_ptr(),
                                  L.BSF_PARAM_SRT, opts, out.data_ptr(), int(stream.cuda_stream))
        assert rc == L.BSF_OK, L.status_string(rc)
        torch.cuda.synchronize(dev)
        got, want = out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
        assert np.isfinite(got).all()
        assert np.abs(got - want).max() / np.abs(want).max() <= TOL
        # and against the oracle's plain definition itself on sampled pixels
        import oracle as O
        fn, pn = f.cpu().numpy().astype(np.float64), p.cpu().numpy().astype(np.float64)
        a, _ = O.map4(pn, O.KIND_SRT)
        idx = np.random.default_rng(seed).choice(H * W, size=64, replace=False)
        ref_o = O.direct4(fn, a, idx)
        assert np.abs(got.ravel()[idx] - ref_o).max() / np.abs(ref_o).max() <= TOL


def test_noalloc_reflect_boundary_matches_filter():
    """The reflected boundary through the allocation-free entry point equals
    bsf_filter with the same option."""
    dev = _dev()
    torch.cuda.set_device(dev)
    H, W = 96, 88
    opts = api.make_opts(max_scale=5.0, boundary="reflect")
    f = torch.from_numpy(synth.image(H, W, seed=8, dtype="u8")).to(dev)
    p = torch.from_numpy(synth.srt_field(H, W, seed=8, sigma=(1.0, 5.0), rho=(1.0, 4.0))).to(dev)
    ref = api.filter(f, p, kind="srt", max_scale=5.0, boundary="reflect")
    out = torch.full((H, W), float("nan"), dtype=torch.float32, device=dev)
    rc = L.bsf_filter_noalloc(f.data_ptr(), L.BSF_U8, H, W, 4, p.data_ptr(), L.BSF_PARAM_SRT, opts, out.data_ptr(),
                              int(torch.cuda.current_stream(dev).cuda_stream))
    assert rc == L.BSF_OK, L.status_string(rc)
    torch.cuda.synchronize(dev)
    assert torch.equal(out, ref)


def test_noalloc_refuses_oversize_image():
    dev = _dev()
    H, W = 3000, 3000
    opts = api.make_opts(max_scale=8.0)
    f = torch.zeros((1, 1), dtype=torch.uint8, device=dev)  # never read: the size check comes first
    rc = L.bsf_filter_noalloc(f.data_ptr(), L.BSF_U8, H, W, 4, f.data_ptr(), L.BSF_PARAM_SRT, opts, f.data_ptr(), 0)
    assert rc == L.BSF_ENOSCRATCH
    assert "fixed scratch" in L.status_string(rc)
