"""Pins of the six-directional oracle (oracle/n6.py) against what the paper and
the mathematics fix: the box spline of Eq. const evaluated by two independent
methods and against the exact four-directional area form, its mass, symmetry,
support, covariance (Eq. covariance) and Fourier transform; the hexagonal
transfer's conservation laws; Algorithm 1 on the hexagonal lattice against the
plain definition on the transferred measure; and the N-directional map of
Sec. 3.2.2 against the paper's closed-form four-directional steps, a generic
minimiser and the elongation bound of Prop. 3.1."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import n6

D4, D6 = n6.directions(4), n6.directions(6)


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def _cov(sigma, rho, theta):
    R = np.array([[math.cos(theta), -math.sin(theta)], [math.sin(theta), math.cos(theta)]])
    return R @ np.diag([sigma * sigma, sigma * sigma / rho]) @ R.T


# ---------------------------------------------------------------- box spline

def test_truncated_power_form_equals_the_area_form_for_four_directions():
    rng = np.random.default_rng(0)
    for _ in range(4):
        a = rng.uniform(0.5, 3.0, 4)
        P = rng.uniform(-4, 4, (150, 2))
        got = n6.betaN(D4, a, P[:, 0], P[:, 1])
        ref = np.array([O.beta4(a, x, y) for x, y in P])
        assert np.abs(got - ref).max() < 1e-13 * max(ref.max(), 1.0)


@pytest.mark.parametrize("N", [3, 5, 6])
def test_truncated_power_form_equals_successive_convolutions(N):
    rng = np.random.default_rng(N)
    th = n6.directions(N)
    a = rng.uniform(0.7, 2.5, N)
    ex, ey = n6.support_extent(th, a)
    for _ in range(3 if N == 6 else 6):
        x = rng.uniform(-0.8 * ex, 0.8 * ex)
        y = rng.uniform(-0.8 * ey, 0.8 * ey)
        ref = n6.betaN_recursive(th, a, x, y)
        got = float(n6.betaN(th, a, np.array(x), np.array(y)))
        assert abs(got - ref) < 1e-12, (x, y, got, ref)


def test_two_directions_give_the_parallelogram():
    th = np.array([0.0, math.pi / 3])
    a = np.array([1.5, 2.0])
    rng = np.random.default_rng(1)
    P = rng.uniform(-2.5, 2.5, (400, 2))
    got = n6.betaN(th, a, P[:, 0], P[:, 1])
    # coordinates in the basis (a1 u1, a2 u2)
    u1, u2 = np.array([1.0, 0.0]), np.array([0.5, math.sqrt(3) / 2])
    B = np.stack([a[0] * u1, a[1] * u2], 1)
    t = np.linalg.solve(B, P.T)
    inside = np.all(np.abs(t) < 0.5, axis=0)
    edge = np.any(np.abs(np.abs(t) - 0.5) < 1e-9, axis=0)
    area = a[0] * a[1] * math.sqrt(3) / 2
    assert np.allclose(got[~edge], np.where(inside, 1.0 / area, 0.0)[~edge], atol=1e-14)


def _grid(a, th, hstep):
    ex, ey = n6.support_extent(th, a)
    xs = np.arange(-ex - hstep, ex + hstep, hstep) + hstep / 2
    ys = np.arange(-ey - hstep, ey + hstep, hstep) + hstep / 2
    X, Y = np.meshgrid(xs, ys)
    return X, Y, n6.betaN(th, a, X, Y)


def test_six_directional_mass_symmetry_support_and_covariance():
    a = np.array([2.3, 1.1, 1.9, 2.6, 0.8, 1.5])
    hs = 0.03
    X, Y, B = _grid(a, D6, hs)
    w = hs * hs
    assert abs(B.sum() * w - 1.0) < 1e-6
    assert np.allclose(n6.betaN(D6, a, -X, -Y), B, atol=1e-11 * B.max())
    C = np.array([[np.sum(X * X * B), np.sum(X * Y * B)], [np.sum(X * Y * B), np.sum(Y * Y * B)]]) * w
    assert np.allclose(C, O.covarianceN(D6, a), atol=2e-4)
    assert B.min() > -1e-11 * B.max()
    # outside the support polygon {sum t_k a_k u_k, |t_k| <= 1/2}: zero
    out = []
    for j in range(6):
        nrm = np.array([-math.sin(D6[j]), math.cos(D6[j])])
        lim = 0.5 * np.sum(a * np.abs(nrm[0] * np.cos(D6) + nrm[1] * np.sin(D6)))
        out.append(np.abs(nrm[0] * X + nrm[1] * Y) > lim + 1e-9)
    assert np.abs(B[np.any(out, axis=0)]).max() < 1e-11 * B.max()


def test_six_directional_fourier_transform():
    """The transform of Eq. const is prod_k sinc(a_k u_k . w / 2)."""
    a = np.array([1.6, 2.1, 1.2, 1.9, 2.4, 1.0])
    hs = 0.02
    X, Y, B = _grid(a, D6, hs)
    for w1, w2 in [(0.0, 0.0), (0.7, 0.0), (0.4, -1.1), (1.5, 0.9), (-2.0, 0.3)]:
        got = float(np.sum(B * np.cos(w1 * X + w2 * Y)) * hs * hs)
        ref = float(O.box_spline_hat(D6, a, np.array(w1), np.array(w2)))
        assert abs(got - ref) < 2e-5, (w1, w2, got, ref)


def test_hexagonal_interpolation_element_is_a_partition_of_unity():
    """beta^6_b with b = h (1, sqrt3, 1, sqrt3, 1, sqrt3) has its direction
    vectors on the hexagonal lattice, so its lattice translates sum to the
    lattice density 2 / (sqrt(3) h^2) everywhere."""
    h = 0.5
    b = h * np.array(n6.HEX_LENGTHS)
    jj, ii = np.mgrid[-12:13, -16:17]
    LX, LY = n6.hex_position(ii, jj, h)
    rng = np.random.default_rng(2)
    for _ in range(5):
        y = rng.uniform(-0.5, 0.5, 2)
        s = float(np.sum(n6.betaN(D6, b, y[0] - LX, y[1] - LY)))
        assert abs(s * math.sqrt(3) / 2 * h * h - 1.0) < 1e-10


# ---------------------------------------------------------------- hexagonal transfer

@pytest.mark.parametrize("h", [1.0, 0.5, 0.3])
def test_transfer_keeps_mass_and_centre_of_every_pixel(h):
    rng = np.random.default_rng(3)
    for _ in range(6):
        H, W = 7, 9
        f = np.zeros((H, W))
        y, x = rng.integers(0, H), rng.integers(0, W)
        f[y, x] = 1.0
        I, J, m = n6.hex_splat(f, h)
        PX, PY = n6.hex_position(I, J, h)
        assert m.min() >= 0.0 and abs(m.sum() - 1.0) < 1e-14
        assert abs(np.sum(m * PX) - x) < 1e-12 and abs(np.sum(m * PY) - y) < 1e-12
        assert np.all(np.hypot(PX - x, PY - y)[m > 0] <= h + 1e-12)
    f = rng.uniform(0, 1, (6, 5))
    assert abs(n6.hex_splat(f, h)[2].sum() - f.sum()) < 1e-12


def test_algorithm1_on_the_hexagonal_lattice_equals_the_definition():
    """Eq. keyeqn with the hexagonal pre-integration reproduces the plain
    definition on the transferred measure (exact up to rounding)."""
    rng = np.random.default_rng(4)
    H, W = 9, 8
    f = rng.uniform(0, 1, (H, W))
    A = rng.uniform(0.6, 2.4, (6, H, W))
    idx = np.array([0, 11, 37, 52, 71])
    for h in (0.5, 1.0):
        ref = n6.direct6_hex(f, A, idx, h)
        got = n6.alg1_hex(f, A, idx, h)
        assert np.abs(got - ref).max() < 1e-9 * np.abs(ref).max()


def test_definition_on_a_crop_equals_the_whole_image():
    """The filter at a pixel depends only on the image inside its footprint:
    evaluated on a crop placed at its origin in the plane, it is unchanged."""
    rng = np.random.default_rng(8)
    H, W = 26, 31
    f = rng.uniform(0, 1, (H, W))
    A = rng.uniform(0.8, 2.0, (6, H, W))
    x, y = 17, 13
    ref = n6.direct6_hex(f, A, np.array([y * W + x]), 0.5)
    y0, x0 = 6, 9
    crop = f[y0:, x0:]
    got = n6.direct6_hex(crop, A[:, y0:, x0:], np.array([(y - y0) * (W - x0) + (x - x0)]), 0.5, origin=(x0, y0))
    assert abs(got[0] - ref[0]) < 1e-13


def test_transfer_error_falls_with_the_lattice_spacing():
    """Method error of the transfer against the definition on the pixel comb:
    second order in h on a smooth image."""
    H = W = 30
    yy, xx = np.mgrid[0:H, 0:W]
    f = 0.5 + 0.3 * np.sin(0.3 * xx + 0.2 * yy) + 0.2 * np.cos(0.17 * xx - 0.4 * yy)
    p, ok = n6.mapN_kkt(D6, np.eye(2) * 4.0, 1e-3)
    A = np.broadcast_to(np.sqrt(p)[:, None, None], (6, H, W)).copy()
    idx = np.array([15 * W + 15, 14 * W + 16])
    ref = n6.direct6(f, A, idx)
    errs = [np.abs(n6.direct6_hex(f, A, idx, h) - ref).max() for h in (1.0, 0.5, 0.25)]
    assert errs[0] > 3 * errs[1] > 9 * errs[2]
    assert errs[1] < 1e-3


# ---------------------------------------------------------------- covariance -> scales

def test_n_gon_elongation_bound_reproduces_prop_3_1():
    for phi in np.linspace(0.01, math.pi - 0.01, 23):
        if abs(math.fmod(2 * phi, math.pi / 2)) < 1e-9:
            continue
        assert math.isclose(n6.U_boundN(phi, 4), O.U_bound(phi), rel_tol=1e-12)
    assert math.isclose(n6.U_boundN(math.pi / 12, 6), (1 + math.cos(math.pi / 6)) / (1 - math.cos(math.pi / 6)))
    assert n6.U_boundN(0.0, 6) == math.inf and n6.U_boundN(math.pi / 6, 6) == math.inf


@pytest.mark.parametrize("rho,theta", [(1.0, 0.0), (2.0, 0.3), (3.0, math.pi / 8), (5.0, math.pi / 12), (4.0, 2.0),
                                       (5.7, math.pi / 8)])
def test_kkt_map_reproduces_the_papers_four_directional_steps(rho, theta):
    C = _cov(2.0, rho, theta)
    a4, flag = O.map4(np.array([C[0, 0], C[0, 1], C[1, 1]]).reshape(3, 1), O.KIND_COV)
    p, ok = n6.mapN_kkt(D4, C, 1e-3)
    assert ok and flag[0] == 0
    assert np.allclose(np.sqrt(p), a4[:, 0], rtol=1e-8, atol=1e-8)


@pytest.mark.parametrize("rho,theta", [(1.0, 0.0), (3.0, 0.4), (6.0, 0.26), (12.0, math.pi / 12), (2.5, 2.2)])
def test_six_directional_kkt_map(rho, theta):
    C = _cov(2.0, rho, theta)
    p, ok = n6.mapN_kkt(D6, C, 1e-3)
    assert ok
    assert np.allclose(O.covarianceN(D6, np.sqrt(p)), C, rtol=1e-12, atol=1e-12)
    assert p.min() >= 1e-3 - 1e-13 * 12 * np.trace(C)
    assert np.allclose(np.sqrt(p), O.mapN(D6, C, eps=1e-3), rtol=1e-7, atol=1e-7)


def test_six_directional_feasibility_matches_the_bound():
    phi = 0.2
    U = n6.U_boundN(phi, 6)
    _, ok = n6.mapN_kkt(D6, _cov(3.0, 0.999 * U, phi), 0.0)
    assert ok
    _, ok = n6.mapN_kkt(D6, _cov(3.0, 1.001 * U, phi), 0.0)
    assert not ok


def test_map6_flags():
    P = np.array([[2.0, 2.0, 2.0, 0.03, 2.0],
                  [1.0, 20.0, 3.0, 5.0, -1.0],
                  [0.0, 0.2, 0.5, 0.2, 0.0]])
    a, fl = n6.map6(P, 2)
    assert fl[0] == 0 and np.allclose(a[:, 0], 4.0)
    assert fl[1] & n6.FLAG_CLAMPED
    assert fl[2] == 0
    assert fl[3] & n6.FLAG_INFEASIBLE and np.all(a[:, 3] >= math.sqrt(1e-3) * (1 - 1e-12))
    # the bound is relative to the size: no width below sqrt(1e-3 T)
    assert a[:, 2].min() >= math.sqrt(1e-3 * 12.0 * (4.0 + 4.0 / 3.0)) * (1 - 1e-9)
    assert fl[4] == n6.FLAG_INVALID and np.all(np.isnan(a[:, 4]))
    # clamped pixel: the target after clamping is reproduced, at the bound's elongation
    lmax, lmin = 4.0, 4.0 / 20.0
    U = n6.U_boundN(0.2, 6, 1 - 6 * n6.REL_BOUND6)
    s = lmax + lmin
    lmin2 = s / (1 + (1 - 1e-3) * U)
    C2 = _cov(math.sqrt(s - lmin2), (s - lmin2) / lmin2, 0.2)
    assert np.allclose(O.covarianceN(D6, a[:, 1]), C2, rtol=1e-10, atol=1e-12)


def test_c_restatement_of_algorithm1_equals_the_numpy_one():
    """The C form of Algorithm 1 on the hexagonal lattice (used to time the CPU
    baseline) against the numpy form and the definition on the transferred
    image, on tiny images with h = 1/2 and 1/4: the same three steps, so the
    results agree to the FP64 cancellation level of both (about 1e-9 of the
    output here); a dropped term, a wrong sign or a transposed direction gives
    errors of order one.  Its pointwise box spline equals betaN."""
    from paper_1003_2022_gb300 import synth
    th = n6.directions(6)
    a = np.array([1.3, 0.7, 2.1, 1.1, 0.9, 1.6])
    for x in [(0.1, 0.2), (-0.5, 0.3), (1.0, -0.4), (0.0, 0.0), (3.0, 3.0)]:
        assert n6.beta6_c(a, *x) == pytest.approx(float(n6.betaN(th, a, np.array(x[0]), np.array(x[1]))),
                                                  rel=1e-12, abs=1e-14)
    for h, (H, W) in ((0.5, (9, 11)), (0.25, (6, 7))):
        f = synth.image(H, W, seed=2, dtype="f32").astype(np.float64)
        A = synth.scale_field(H, W, seed=3, lo=0.8, hi=3.0)
        A6 = np.concatenate([A, A[:2] * 0.9]).astype(np.float64)
        idx = np.array([0, 5, W + 3, H * W // 2, H * W - 1])
        c = n6.alg1_hex_c(f, A6, idx, h)
        py = n6.alg1_hex(f, A6, idx, h)
        ref = n6.direct6_hex(f, A6, idx, h)
        assert np.abs(c - py).max() < 2e-8 * np.abs(py).max()
        assert np.abs(c - ref).max() < 2e-8 * np.abs(ref).max()
    # every pixel of a tiny image (idx = None)
    f = synth.image(5, 6, seed=4, dtype="u8").astype(np.float64)
    A6 = np.full((6, 5, 6), 1.4)
    full = n6.alg1_hex_c(f, A6, None, 0.5)
    assert np.abs(full - n6.direct6_hex(f, A6, None, 0.5)).max() < 2e-8 * np.abs(full).max()
