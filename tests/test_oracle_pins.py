"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a second
independent evaluation, a closed form printed in the paper, an invariant, a
textbook special case, or brute force on a tiny input.  CPU only.
"""
import math
import os

import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(1234)
SCALES = [
    np.array([1.7, 2.3, 2.9, 1.1]),
    np.array([3.0, 0.4, 1.2, 5.5]),
    np.array([0.8, 0.9, 0.7, 1.3]),
    np.array([6.0, 6.0, 6.0, 6.0]),
]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_constants():
    out = {}
    with open(os.path.join(GOLDEN, "printed_constants.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, val = line.split()[:2]
            out[name] = float(val)
    return out


def _support_extent(a):
    return 0.5 * (a[0] + (a[1] + a[3]) / math.sqrt(2)), 0.5 * (a[2] + (a[1] + a[3]) / math.sqrt(2))


def _grid_moments(a, h=0.02):
    hx, hy = _support_extent(a)
    xs = np.arange(-hx - 0.5, hx + 0.5, h) + h / 2
    ys = np.arange(-hy - 0.5, hy + 0.5, h) + h / 2
    X1, X2 = np.meshgrid(xs, ys)
    B = O.beta4_grid(a, X1, X2)
    return X1, X2, B * h * h


# --------------------------------------------------------------- O-beta
@pytest.mark.parametrize("a", SCALES)
def test_beta_area_vs_line_integral(a):
    """Two independent exact evaluations of Eq. (const) agree."""
    hx, hy = _support_extent(a)
    pts = RNG.uniform([-hx - 0.3, -hy - 0.3], [hx + 0.3, hy + 0.3], size=(400, 2))
    for x1, x2 in pts:
        v1, v2 = O.beta4(a, x1, x2), O.beta4_lines(a, x1, x2)
        assert abs(v1 - v2) <= 1e-12 * max(1.0, abs(v1)) / np.prod(a) + 1e-13


@pytest.mark.parametrize("a", SCALES[:3])
def test_beta_mass_and_covariance(a):
    """Unit mass and the closed-form covariance Eq. covariance_ZP (Sec. 3.2.2)."""
    X1, X2, w = _grid_moments(a)
    assert abs(w.sum() - 1) < 1e-9
    C = np.array([[np.sum(w * X1 * X1), np.sum(w * X1 * X2)], [np.sum(w * X1 * X2), np.sum(w * X2 * X2)]])
    C_paper = O.covariance4(a)
    # the general form Eq. (covariance): (1/12) sum a_k^2 u_k u_k^T
    th = np.arange(4) * np.pi / 4
    C_gen = sum(a[k] ** 2 * np.outer([np.cos(th[k]), np.sin(th[k])], [np.cos(th[k]), np.sin(th[k])])
                for k in range(4)) / 12
    assert np.allclose(C_paper, C_gen, rtol=1e-14, atol=1e-14)
    assert np.allclose(C, C_paper, rtol=2e-5, atol=1e-6)


@pytest.mark.parametrize("a", SCALES[:2])
def test_beta_kurtosis_matrix_closed_form(a):
    """Fourth moments -> K = L - tr(C) C - 2 C^2 equals Eq. finalForm (App. E)."""
    X1, X2, w = _grid_moments(a, h=0.015)
    C = np.array([[np.sum(w * X1 * X1), np.sum(w * X1 * X2)], [np.sum(w * X1 * X2), np.sum(w * X2 * X2)]])
    r2 = X1 * X1 + X2 * X2
    # (x x^T)^2 = |x|^2 x x^T
    L = np.array([[np.sum(w * r2 * X1 * X1), np.sum(w * r2 * X1 * X2)],
                  [np.sum(w * r2 * X1 * X2), np.sum(w * r2 * X2 * X2)]])
    K = L - np.trace(C) * C - 2 * C @ C
    g = _golden_constants()
    mu2, mu4 = g["mu2_box"], g["mu4_box"]
    a4 = a ** 4
    K_paper = (mu4 - 3 * mu2 ** 2) * np.array([[a4[0] + 0.5 * (a4[1] + a4[3]), 0.5 * (a4[1] - a4[3])],
                                               [0.5 * (a4[1] - a4[3]), a4[2] + 0.5 * (a4[1] + a4[3])]])
    scale = np.abs(K_paper).max()
    assert np.allclose(K, K_paper, atol=2e-4 * scale)
    # ||K||^2 / (mu4 - 3 mu2^2)^2 = sum p^4 + (p1^2+p3^2)(p2^2+p4^2), p = a^2
    n2 = np.sum(K_paper ** 2) / (mu4 - 3 * mu2 ** 2) ** 2
    assert abs(n2 - O.kurtosis4_norm2(a ** 2)) < 1e-10 * n2


@pytest.mark.parametrize("a", SCALES)
def test_beta_symmetry_and_support(a):
    """beta(x) = beta(-x); zero outside the support polygon of Sec. 2.2.1."""
    hx, hy = _support_extent(a)
    for x1, x2 in RNG.uniform([-hx, -hy], [hx, hy], size=(200, 2)):
        assert abs(O.beta4(a, x1, x2) - O.beta4(a, -x1, -x2)) < 1e-13 / np.prod(a)
    # points outside the polygon {sum t_k a_k u_k, |t_k| <= 1/2}: beyond the extents
    for x1, x2 in [(hx + 1e-6, 0.0), (0.0, hy + 1e-6), (-hx - 1e-3, 0.2), (0.1, -hy - 1e-3)]:
        assert O.beta4(a, x1, x2) == 0.0
    # vertex of the octagon in direction (1,1): support function along (1,1)/sqrt2
    d = np.array([1.0, 1.0]) / math.sqrt(2)
    th = np.arange(4) * np.pi / 4
    hsupp = 0.5 * sum(a[k] * abs(np.cos(th[k]) * d[0] + np.sin(th[k]) * d[1]) for k in range(4))
    assert O.beta4(a, *(d * (hsupp + 1e-6))) == 0.0
    assert O.beta4(a, *(d * (hsupp - 1e-3))) > 0.0


def test_zp_partition_of_unity():
    """At b = (1, sqrt2, 1, sqrt2) the integer translates sum to one (App. F)."""
    for y in RNG.uniform(-0.5, 0.5, size=(50, 2)):
        s = sum(O.beta4(O.ZP_SCALES, y[0] - i, y[1] - j) for i in range(-3, 4) for j in range(-3, 4))
        assert abs(s - 1) < 1e-13
    # at most seven lattice points carry weight (App. F)
    for y in RNG.uniform(-0.5, 0.5, size=(50, 2)):
        nz = sum(O.beta4(O.ZP_SCALES, y[0] - i, y[1] - j) > 0 for i in range(-3, 4) for j in range(-3, 4))
        assert nz <= 7


def test_lattice_mass_exact_for_integer_scales():
    """sum_k beta_a(n-k) = 1 when a1, a3 are integers (Poisson summation with the
    Fourier form of App. A); not 1 in general."""
    def mass(a, n=(0.0, 0.0)):
        hx, hy = _support_extent(a)
        R = int(max(hx, hy)) + 2
        return sum(O.beta4(a, n[0] - i, n[1] - j) for i in range(-R, R + 1) for j in range(-R, R + 1))
    assert abs(mass(np.array([2.0, 1.3, 3.0, 2.2])) - 1) < 1e-12
    assert abs(mass(np.array([1.7, math.sqrt(2) * 2, 2.9, math.sqrt(2) * 1])) - 1) < 1e-12
    assert abs(mass(np.array([1.7, 2.3, 2.9, 1.1])) - 1) > 1e-4


# --------------------------------------------------------------- O-direct
def test_direct_constant_field_is_convolution():
    """A constant scale field reduces Eq. SVF_2D to ordinary 2-D discrete
    convolution with h[k] = beta_a(k), zero padded (independent loop)."""
    from scipy.signal import convolve2d
    a = np.array([2.3, 1.9, 3.1, 1.4])
    H, W = 13, 17
    f = RNG.random((H, W))
    af = np.broadcast_to(a[:, None, None], (4, H, W)).copy()
    out = O.direct4(f, af)
    R = 6
    k = np.arange(-R, R + 1)
    h = np.array([[O.beta4(a, k1, k2) for k1 in k] for k2 in k])  # h[k2, k1]
    ref = convolve2d(f, h, mode="same")
    assert np.allclose(out, ref, rtol=1e-13, atol=1e-14)


def test_direct_constant_image_mass():
    """f = c everywhere (interior pixels): fbar = c * sum_k beta_a(n-k)."""
    H, W = 21, 21
    f = np.full((H, W), 3.25)
    a = np.array([1.7, 2.3, 2.9, 1.1])
    af = np.broadcast_to(a[:, None, None], (4, H, W)).copy()
    out = O.direct4(f, af)
    m = sum(O.beta4(a, -i, -j) for i in range(-5, 6) for j in range(-5, 6))
    assert abs(out[10, 10] - 3.25 * m) < 1e-12
    a2 = np.array([2.0, 1.3, 3.0, 2.2])
    out2 = O.direct4(f, np.broadcast_to(a2[:, None, None], (4, H, W)).copy())
    assert abs(out2[10, 10] - 3.25) < 1e-12


def test_direct_separable_box_limit():
    """a2, a4 -> 0 leaves the separable box a1 x a3: the 1-D space-variant
    average of Eq. SVF (Dirac-comb image) applied along each axis."""
    H, W = 9, 11
    f = RNG.random((H, W))
    d = 1e-7
    a = np.array([2.5, d, 3.5, d])
    af = np.broadcast_to(a[:, None, None], (4, H, W)).copy()
    out = O.direct4(f, af)
    fp = np.pad(f, 1)
    ref = sum(fp[1 + j:1 + j + H, 1 + i:1 + i + W] for i in (-1, 0, 1) for j in (-1, 0, 1)) / (2.5 * 3.5)
    assert np.allclose(out, ref, rtol=1e-5, atol=1e-7)


def test_direct_space_variant_uses_local_scale():
    """Each pixel uses its own scale vector: compare against per-pixel constant-field runs."""
    H, W = 8, 9
    f = RNG.random((H, W))
    a = RNG.uniform(0.6, 3.0, size=(4, H, W))
    out = O.direct4(f, a)
    for (r, c) in [(0, 0), (3, 4), (7, 8), (5, 1)]:
        ac = np.broadcast_to(a[:, r, c][:, None, None], (4, H, W)).copy()
        assert abs(O.direct4(f, ac)[r, c] - out[r, c]) < 1e-14


# --------------------------------------------------------------- O-alg
def _brute_preint(f, P):
    """Definitions RS1-RS4 of Sec. 3.1 as explicit sums on the padded buffer
    (integer form: the two sqrt2 factors taken out)."""
    H, W = f.shape
    Hp, Wp = H + 2 * P, W + 2 * P
    x = np.zeros((Hp, Wp), dtype=object)
    x[P:P + H, P:P + W] = f.astype(object)
    g0 = np.zeros_like(x)
    g45 = np.zeros_like(x)
    g90 = np.zeros_like(x)
    G = np.zeros_like(x)
    for r in range(Hp):
        for c in range(Wp):
            g0[r, c] = sum(x[r, c - k] for k in range(0, c + 1))
    for r in range(Hp):
        for c in range(Wp):
            g45[r, c] = sum(g0[r - k, c - k] for k in range(0, min(r, c) + 1))
    for r in range(Hp):
        for c in range(Wp):
            g90[r, c] = sum(g45[r - k, c] for k in range(0, r + 1))
    for r in range(Hp):
        for c in range(Wp):
            G[r, c] = sum(g90[r - k, c + k] for k in range(0, min(r, Wp - 1 - c) + 1))
    return G


def test_preint_recursion_matches_running_sum_definitions():
    f = RNG.integers(0, 256, size=(5, 7))
    P = 3
    G = O.preint4_i64(f, P)
    Gb = _brute_preint(f, P)
    assert np.array_equal(G, Gb.astype(np.int64))


def test_preint_integer_form_equals_float_form():
    """g_b (with the sqrt2 factors) = 2 G (integer form) for integer images."""
    f = RNG.integers(0, 256, size=(11, 9))
    P = 5
    G = O.preint4_i64(f, P)
    gb = O.preint4_f64(f.astype(float), P)
    assert np.allclose(gb, 2.0 * G.astype(float), rtol=1e-13, atol=1e-9)


def test_preint_wraps_modulo_2_64():
    """Integer sums are kept modulo 2^64 (checked against Python integers)."""
    f = np.full((4, 4), 2 ** 61, dtype=np.int64)
    P = 2
    G = O.preint4_i64(f, P)
    Gb = _brute_preint(f.astype(object), P)
    wrapped = np.array([[((int(v) + 2 ** 63) % 2 ** 64) - 2 ** 63 for v in row] for row in Gb], dtype=np.int64)
    assert np.array_equal(G, wrapped)


def _table1_taps(a):
    s2 = math.sqrt(2)
    a1, a2p, a3, a4p = a[0], a[1] / s2, a[2], a[3] / s2
    env = {"a1": a1, "a2'": a2p, "a3": a3, "a4'": a4p}
    taps = []
    with open(os.path.join(GOLDEN, "table1_fd_mesh.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            i, e0, e1, sg = line.split()

            def ev(expr):
                expr = expr.replace("a2'", "A2").replace("a4'", "A4")
                return eval(expr, {}, {"a1": a1, "A2": a2p, "a3": a3, "A4": a4p})
            taps.append((int(i), ev(e0), ev(e1), 1 if sg == "+" else -1))
    return taps


def test_table1_matches_general_fd_mesh():
    """Table 1 equals Eq. FD_mesh: x_i = sum q_k a_k u_k, w_i = (-1)^sum q."""
    a = np.array([1.3, 2.1, 0.7, 3.3])
    th = np.arange(4) * np.pi / 4
    for i, x0, x1, sg in _table1_taps(a):
        q = [(i >> k) & 1 for k in range(4)]
        xi = sum(q[k] * a[k] * np.array([np.cos(th[k]), np.sin(th[k])]) for k in range(4))
        assert np.allclose(xi, [x0, x1], atol=1e-14)
        assert sg == (-1) ** sum(q)


@pytest.mark.parametrize("integer", [True, False])
def test_alg1_equals_direct_on_tiny_images(integer):
    """Algorithm 1 (pre-integration + ZP interpolation + 16 taps) computes the
    exact filter fbar[n] = sum_k f[k] beta_a(n-k) (Prop. 2.1, Eq. keyeqn)."""
    H, W = 9, 11
    if integer:
        f = RNG.integers(0, 256, size=(H, W)).astype(np.int64)
    else:
        f = RNG.random((H, W))
    a = RNG.uniform(0.5, 4.0, size=(4, H, W))
    P = 7
    out, bad = O.alg1_filter4(f, a, P, integer=integer)
    assert bad == 0
    ref = O.direct4(f.astype(float), a)
    err = np.abs(out - ref).max() / np.abs(ref).max()
    assert err < 1e-11, err


# --------------------------------------------------------------- O-map
def _cov_from_srt(sig, rho, th):
    lmax, lmin = sig ** 2, sig ** 2 / rho
    c, s = math.cos(th), math.sin(th)
    return np.array([[lmax * c * c + lmin * s * s, 0.5 * (lmax - lmin) * math.sin(2 * th)],
                     [0.5 * (lmax - lmin) * math.sin(2 * th), lmin * c * c + lmax * s * s]])


def test_map_isotropic_case():
    """C = sigma^2 I -> a_k = sigma sqrt(24/N) = sigma sqrt(6) (Theorem 2.2)."""
    g = _golden_constants()
    for sig in [0.7, 1.0, 2.5, 17.0]:
        a, fl = O.map4(np.array([[sig ** 2], [0.0], [sig ** 2]]), O.KIND_COV)
        assert fl[0] == 0
        assert np.allclose(a[:, 0], sig * g["iso_scale_factor_N4"], rtol=1e-12)


def _random_feasible_srt(n):
    out = []
    while len(out) < n:
        sig = RNG.uniform(0.8, 20)
        th = RNG.uniform(0, np.pi)
        rho = RNG.uniform(1, 0.9 * min(O.U_bound(th), 50))
        out.append((sig, rho, th))
    return out


def test_map_reproduces_covariance():
    """M p = c: the returned scales have exactly the target covariance (Eq. covariance_ZP)."""
    for sig, rho, th in _random_feasible_srt(200):
        C = _cov_from_srt(sig, rho, th)
        a, fl = O.map4(np.array([[C[0, 0]], [C[0, 1]], [C[1, 1]]]), O.KIND_COV)
        if fl[0] & 2:
            continue
        assert fl[0] == 0
        assert np.allclose(O.covariance4(a[:, 0]), C, rtol=1e-9, atol=1e-9 * sig ** 2)
        assert np.all(a[:, 0] ** 2 >= 1e-3 * (1 - 1e-9))


def _zeta(pb, t):
    p = np.array([pb[0] + t, pb[1] - t, pb[2] + t, pb[3] - t])
    return np.sum(p ** 4, axis=0) + (p[0] ** 2 + p[2] ** 2) * (p[1] ** 2 + p[3] ** 2)


def test_map_is_brute_force_minimiser():
    """t0 minimises zeta on [t_l, t_r]: compare with a 10^6-point grid search."""
    eps = 1e-3
    for sig, rho, th in _random_feasible_srt(40):
        C = _cov_from_srt(sig, rho, th)
        a, fl = O.map4(np.array([[C[0, 0]], [C[0, 1]], [C[1, 1]]]), O.KIND_COV, eps=eps)
        if fl[0]:
            continue
        c1, c2, c3 = 24 * C[0, 0], 24 * C[0, 1], 24 * C[1, 1]
        pb = np.array([(c1 - c2 - 2) / 2, c2 + 1, (c3 - c2 - 2) / 2, 1.0])
        tl, tr = max(eps - pb[0], eps - pb[2]), min(pb[1] - eps, pb[3] - eps)
        ts = np.linspace(tl, tr, 1_000_001)
        zs = _zeta(pb, ts)
        t_grid = ts[np.argmin(zs)]
        p = a[:, 0] ** 2
        t0 = p[0] - pb[0]
        assert _zeta(pb, t0) <= zs.min() * (1 + 1e-12) + 1e-9
        assert abs(t0 - t_grid) <= 2 * (tr - tl) / 1e6 + 1e-9 * abs(t0)


def test_zeta_prime_coefficients():
    """The cubic of Sec. 3.2.2 step (iii) is the derivative of the quartic zeta(t)."""
    for _ in range(50):
        pb = RNG.uniform(-5, 5, size=4)
        z1 = 32
        z2 = 24 * (pb[0] - pb[1] + pb[2] - pb[3])
        z3 = 16 * np.sum(pb ** 2) - 8 * (pb[0] + pb[2]) * (pb[1] + pb[3])
        z4 = (4 * (pb[0] ** 3 - pb[1] ** 3 + pb[2] ** 3 - pb[3] ** 3)
              + 2 * (pb[0] + pb[2]) * (pb[1] ** 2 + pb[3] ** 2) - 2 * (pb[1] + pb[3]) * (pb[0] ** 2 + pb[2] ** 2))
        t = RNG.uniform(-3, 3)
        h = 1e-5
        num = (_zeta(pb, t + h) - _zeta(pb, t - h)) / (2 * h)
        cub = ((z1 * t + z2) * t + z3) * t + z4
        assert abs(num - cub) < 1e-5 * max(1, abs(cub))


def test_map_fourfold_symmetry_corrected_permutation():
    """Rotating the target by +45 degrees cycles the optimal scales to
    (a4, a1, a2, a3) -- the symmetry behind the LUT of Sec. 3.2.2, with the
    permutation read in the direction that rotates the spline by +45 deg."""
    for sig, rho, th in _random_feasible_srt(30):
        if th >= 3 * np.pi / 4 or O.U_bound(th + np.pi / 4) < rho * 1.01:
            continue
        C0 = _cov_from_srt(sig, rho, th)
        C1 = _cov_from_srt(sig, rho, th + np.pi / 4)
        a0, f0 = O.map4(np.array([[C0[0, 0]], [C0[0, 1]], [C0[1, 1]]]), O.KIND_COV)
        a1, f1 = O.map4(np.array([[C1[0, 0]], [C1[0, 1]], [C1[1, 1]]]), O.KIND_COV)
        if f0[0] or f1[0]:
            continue
        assert np.allclose(a1[:, 0], a0[[3, 0, 1, 2], 0], rtol=1e-7, atol=1e-7)


def test_elongation_bound_printed_value_and_simplified_form():
    """Prop. 3.1: U(pi/8) = 3 + 2 sqrt2; U = (1+|s|+|c|)^2 / (2|s||c|), s,c = sin, cos of 2 phi."""
    g = _golden_constants()
    for k in range(1, 5):
        assert abs(O.U_bound((2 * k - 1) * np.pi / 8) - g["elongation_bound_pi_8"]) < 1e-12
    for phi in RNG.uniform(0.01, np.pi - 0.01, size=100):
        s, c = abs(math.sin(2 * phi)), abs(math.cos(2 * phi))
        if min(s, c) < 1e-6:
            continue
        assert abs(O.U_bound(phi) - (1 + s + c) ** 2 / (2 * s * c)) < 1e-9 * O.U_bound(phi)


def test_elongation_bound_is_supremum():
    """Random positive scale vectors never exceed U(theta_a) (Prop. 3.1)."""
    for _ in range(2000):
        a = np.exp(RNG.uniform(-3, 3, size=4))
        C = O.covariance4(a)
        ev, V = np.linalg.eigh(C)
        rho = ev[1] / ev[0]
        th = math.atan2(V[1, 1], V[0, 1]) % np.pi
        assert rho < O.U_bound(th) * (1 + 1e-9)


def test_map_clamps_beyond_bound():
    """rho above (1-eta) U(theta): lowered to (1-eta) U, size and orientation kept, flag 1."""
    eta = 1e-3
    for th in [np.pi / 8, 0.3, 1.1, 2.0, 2.9]:
        U = O.U_bound(th)
        sig, rho = 3.0, U * 1.5
        a, fl = O.map4(np.array([[sig], [rho], [th]]), O.KIND_SRT, eta=eta)
        assert fl[0] & 1
        C = O.covariance4(a[:, 0])
        ev, V = np.linalg.eigh(C)
        s_target = sig ** 2 * (1 + 1 / rho)
        assert abs(ev.sum() - s_target) < 1e-8 * s_target
        assert abs(ev[1] / ev[0] - (1 - eta) * U) < 1e-6 * U
        th_a = math.atan2(V[1, 1], V[0, 1]) % np.pi
        assert min(abs(th_a - th), np.pi - abs(th_a - th)) < 1e-7


def test_map_invalid_covariance():
    a, fl = O.map4(np.array([[1.0, np.nan], [2.0, 0.0], [1.0, 1.0]]), O.KIND_COV)
    assert fl[0] == 4 and fl[1] == 4
    assert np.all(np.isnan(a))


# --------------------------------------------------------------- O-adjoint / FD gradient
def test_adjoint_is_transpose_of_direct():
    """<g, K f> = <K^T g, f> for the space-variant operator (independent loops)."""
    H, W = 13, 15
    a = RNG.uniform(0.6, 4.0, size=(4, H, W))
    f = RNG.standard_normal((H, W))
    g = RNG.standard_normal((H, W))
    lhs = float(np.sum(g * O.direct4(f, a)))
    rhs = float(np.sum(O.adjoint4(g, a, np.arange(H * W)).reshape(H, W) * f))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_fd_scale_gradient_closed_form_separable_limit():
    """a = (a1, d, a3, d), d -> 0, no lattice point on the box edge: fbar =
    sum_{3x3} f / (a1 a3), so dfbar/da1 = -fbar/a1 and dfbar/da3 = -fbar/a3."""
    H, W = 9, 11
    f = RNG.random((H, W))
    d = 1e-6
    a = np.broadcast_to(np.array([2.5, d, 3.5, d])[:, None, None], (4, H, W)).copy()
    idx = np.array([3 * W + 4, 5 * W + 6, 4 * W + 5])
    fb = O.direct4(f, a, idx)
    fd = O.direct4_grad_fd(f, a, idx, h=1e-3)
    assert np.allclose(fd[0], -fb / 2.5, rtol=1e-5)
    assert np.allclose(fd[2], -fb / 3.5, rtol=1e-5)


def _corr_with_gaussian(a, m, h=0.025):
    """Normalised correlation of beta^{4,m}_{a/sqrt(m)} (m-fold continuous
    self-convolution, on a fine grid) with the Gaussian of the same covariance."""
    from scipy.signal import fftconvolve
    a = np.asarray(a, float) / np.sqrt(m)
    hx, hy = _support_extent(a)
    R = max(hx, hy) * m + 1.0
    xs = np.arange(-R, R + h / 2, h)
    X1, X2 = np.meshgrid(xs, xs)
    b = O.beta4_grid(a, X1, X2) * h * h
    bm = b
    for _ in range(m - 1):
        bm = fftconvolve(bm, b, mode="same")
    C = O.covariance4(a) * m
    Ci = np.linalg.inv(C)
    g = np.exp(-0.5 * (Ci[0, 0] * X1 * X1 + 2 * Ci[0, 1] * X1 * X2 + Ci[1, 1] * X2 * X2))
    return float(np.sum(bm * g) / np.sqrt(np.sum(bm * bm) * np.sum(g * g)))


def test_iterated_splines_approach_the_gaussian():
    """Sec. 3.3 / Fig. errorplots: at the critical orientation 22.5 deg the
    correlation of the optimal box spline with the target Gaussian is about
    95 % at its worst and rises to about 99 % for the twice-iterated spline."""
    th = np.pi / 8
    worst = {1: 1.0, 2: 1.0}
    for rho in (1.0, 2.0, 3.0, 4.0, 5.0):
        a, fl = O.map4(np.array([[3.0], [rho], [th]]), O.KIND_SRT)
        for m in (1, 2):
            worst[m] = min(worst[m], _corr_with_gaussian(a[:, 0], m))
    assert 0.93 < worst[1] < 0.975, worst
    assert worst[2] > 0.985, worst
    assert worst[2] > worst[1]


def test_beta4_is_c1_but_not_c2():
    """Smoothness C^{N-3} = C^1 (Sec. 2.2.1): along a line through the support the
    first differences change by O(h) between neighbouring steps everywhere,
    while the second differences jump by O(1) where the line crosses a knot."""
    a = np.array([2.3, 1.7, 3.1, 2.6])
    h = 1e-3
    t = np.arange(-4.0, 4.0, h)
    # a line in a generic direction, so that it crosses knot lines transversally
    x1, x2 = 0.83 * t + 0.11, 0.56 * t - 0.07
    b = O.beta4_grid(a, x1, x2)
    d1 = np.diff(b) / h
    d2 = np.diff(d1) / h
    assert np.abs(np.diff(d1)).max() < 50 * h          # first derivative continuous
    assert np.abs(np.diff(d2)).max() > 1e-2            # second derivative jumps somewhere
    assert np.abs(b).max() > 0.05


def test_reflected_boundary_definition():
    """The reflected boundary (reading R21): the padding is f[-1-i] = f[i],
    f[n+i] = f[n-1-i], periodic beyond one reflection; a constant image stays
    exactly constant at EVERY pixel for scales with unit lattice mass (a1, a3
    integers), where the zero boundary loses mass at the borders; away from the
    borders the two boundaries agree."""
    x = np.arange(5.0)
    pad = O.pad_reflect(x[None, :], 6)[6]
    want = [x[(i % 10) if (i % 10) < 5 else 9 - (i % 10)] for i in range(-6, 11)]
    assert np.array_equal(pad, want)
    H, W = 9, 11
    f = np.full((H, W), 3.0)
    a = np.zeros((4, H, W))
    a[0], a[1], a[2], a[3] = 3.0, 2.3, 2.0, 1.7
    assert np.abs(O.direct4_reflect(f, a) - 3.0).max() < 1e-12
    assert np.abs(O.direct4(f, a) - 3.0).max() > 0.5
    rng = np.random.default_rng(2)
    H, W = 24, 26
    f = rng.uniform(0, 1, (H, W))
    a = rng.uniform(0.5, 2.0, (4, H, W))
    inner = np.array([y * W + x for y in range(6, H - 6) for x in range(6, W - 6)])
    assert np.abs(O.direct4_reflect(f, a, inner) - O.direct4(f, a, inner)).max() < 1e-13
