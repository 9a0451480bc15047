"""Pins of the oracle's feature-preserving smoothing (Sec. 4.2): the structure
tensor and the adaptive covariance field, checked against closed forms, and
the application's claim that adapting the window to the local orientation
beats isotropic smoothing on an oriented pattern."""
import numpy as np
import pytest

import oracle as O
from paper_1003_2022_gb300 import synth


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def test_constant_image_gives_isotropic_window():
    C = O.structure_cov(np.full((20, 24), 0.7), sigma_w=1.5, sigma0=1.3, tau=0.01)
    assert np.allclose(C[0], 1.3 ** 2, rtol=0, atol=1e-15)
    assert np.allclose(C[2], 1.3 ** 2, rtol=0, atol=1e-15)
    assert np.all(C[1] == 0.0)


def test_ramp_elongates_along_the_isolines():
    """f = alpha x + beta y: the interior gradient is (alpha, beta), J = m g g^T
    with m the window's lattice mass, so C stretches along g-perp with
    elongation (m |g|^2 + tau) / tau and keeps det C = sigma0^4."""
    H, W, al, be, sw, s0, tau = 40, 44, 0.3, -0.2, 1.2, 1.5, 0.01
    y, x = np.mgrid[0:H, 0:W].astype(float)
    C = O.structure_cov(al * x + be * y, sw, s0, tau)
    r, c = 20, 22  # interior: the window and the differences stay inside
    a = np.full(4, sw * np.sqrt(6.0))
    m = sum(O.beta4(a, r - k2, c - k1) for k2 in range(H) for k1 in range(W))  # lattice mass at (r, c)
    g = np.array([al, be])
    M = m * np.outer(g, g) + tau * np.eye(2)
    want = s0 * s0 * np.linalg.inv(M) * np.sqrt(np.linalg.det(M))
    got = np.array([[C[0, r, c], C[1, r, c]], [C[1, r, c], C[2, r, c]]])
    assert np.allclose(got, want, rtol=1e-10)
    w, v = np.linalg.eigh(got)
    assert abs(np.dot(v[:, 1], g)) < 1e-9 * np.linalg.norm(g)  # long axis perpendicular to the gradient
    assert np.isclose(w[1] / w[0], (m * g @ g + tau) / tau, rtol=1e-10)
    assert np.isclose(np.linalg.det(got), s0 ** 4, rtol=1e-12)


def test_transposed_image_swaps_the_axes():
    f = synth.image(18, 18, seed=3, dtype="f32").astype(float)
    C = O.structure_cov(f, 1.0, 1.2, 0.02)
    Ct = O.structure_cov(f.T, 1.0, 1.2, 0.02)
    assert np.allclose(Ct[0], C[2].T, rtol=1e-12)
    assert np.allclose(Ct[2], C[0].T, rtol=1e-12)
    assert np.allclose(Ct[1], C[1].T, rtol=1e-12)


def test_channels_add_their_tensors():
    f = np.stack([synth.image(16, 20, seed=4, dtype="f32", sub=c) for c in range(3)]).astype(float)
    J = O.structure_tensor(f, 1.0)
    assert np.allclose(J, sum(O.structure_tensor(f[c], 1.0) for c in range(3)), rtol=1e-12)


def test_adaptive_smoothing_beats_isotropic_on_rings():
    """The application's claim (Sec. 4.2: higher PSNR than isotropic smoothing
    of the same size on oriented patterns), on noisy concentric rings."""
    H = W = 96
    clean = synth.rings_image(H, W, period=8.0).astype(float)
    noisy = synth.add_noise(clean, 0.15, seed=1).astype(float)
    s0 = 1.0

    def psnr(x):
        return 10 * np.log10(1.0 / np.mean((x - clean) ** 2))

    iso = np.stack([np.full((H, W), s0 * s0), np.zeros((H, W)), np.full((H, W), s0 * s0)])
    a_iso, _ = O.map4(iso, O.KIND_COV)
    a_ad, _ = O.map4(O.structure_cov(noisy, 2.0, s0, 0.005), O.KIND_COV)
    p_noisy, p_iso, p_ad = psnr(noisy), psnr(O.direct4(noisy, a_iso)), psnr(O.direct4(noisy, a_ad))
    assert p_iso > p_noisy
    assert p_ad > p_iso + 1.0, (p_noisy, p_iso, p_ad)
