"""Feature-preserving smoothing (Sec. 4.2) on the GPU against the oracle:
the adaptive covariance field, the whole pipeline, and the PSNR gain over
isotropic smoothing on noisy rings at full size."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1003_2022_gb300 import _lib as L  # noqa: E402
from paper_1003_2022_gb300 import api, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _nerr(got, ref):
    return float(np.abs(np.asarray(got, np.float64) - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("C,dtype", [(1, "f32"), (3, "f32"), (1, "u8")])
def test_structure_cov_matches_oracle(C, dtype):
    dev = _cuda()
    H, W = 53, 70
    f = np.stack([synth.image(H, W, seed=60 + c, dtype=dtype, sub=c) for c in range(C)])
    tau = 0.01 if dtype == "f32" else 600.0
    cov = api.structure_cov(torch.from_numpy(f).to(dev), 1.5, 1.2, tau)[0].cpu().numpy()
    assert api.device_status(dev) == 0
    ref = O.structure_cov(f.astype(np.float64), 1.5, 1.2, tau)
    for k in range(3):
        assert _nerr(cov[k], ref[k]) < 1e-5, k


def test_adaptive_pipeline_matches_oracle():
    dev = _cuda()
    H = W = 72
    clean = synth.rings_image(H, W, period=7.0)
    noisy = synth.add_noise(clean, 0.1, seed=2)
    out = api.adaptive_smooth(torch.from_numpy(noisy).to(dev), sigma_w=2.0, sigma0=1.2, tau=0.005).cpu().numpy()
    assert api.device_status(dev) & ~(1 << L.BSF_EINFEASIBLE) == 0
    a, _ = O.map4(O.structure_cov(noisy.astype(np.float64), 2.0, 1.2, 0.005), O.KIND_COV)
    ref = O.direct4(noisy.astype(np.float64), a)
    assert _nerr(out, ref) < 1e-5


def test_adaptive_beats_isotropic_at_full_size():
    """2048 x 2048 noisy rings: the adaptive filter's PSNR exceeds the best of
    the isotropic filters of the same area tried."""
    dev = _cuda()
    H = W = 2048
    clean = synth.rings_image(H, W, period=8.0)
    noisy = torch.from_numpy(synth.add_noise(clean, 0.15, seed=5)).to(dev)
    cl = torch.from_numpy(clean).to(dev)

    def psnr(x):
        return float(10 * torch.log10(1.0 / torch.mean((x - cl) ** 2)))

    best_iso = -1e9
    for s0 in (0.8, 1.0, 1.2):
        iso = torch.zeros((3, H, W), device=dev)
        iso[0] = iso[2] = s0 * s0
        best_iso = max(best_iso, psnr(api.filter(noisy, iso, kind="cov", max_scale=s0)))
    ad = psnr(api.adaptive_smooth(noisy, sigma_w=2.0, sigma0=1.0, tau=0.005))
    assert api.device_status(dev) & ~(1 << L.BSF_EINFEASIBLE) == 0
    assert ad > best_iso + 1.0, (best_iso, ad)
