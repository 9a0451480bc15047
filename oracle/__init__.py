"""FP64 CPU oracle for space-variant elliptical box-spline filtering.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it and shares no code with it.

Every function follows a passage of Chaudhury, Munoz-Barrutia and Unser,
"Fast space-variant elliptical filtering using box splines":

* ``beta4`` / ``beta4_lines``: the four-directional radially-uniform box spline
  of Eq. (const) (Sec. 2.2.1), evaluated exactly in two independent ways.
* ``direct4``: the plain definition fbar[n] = sum_k f[k] beta_{a(n)}(n-k)
  (Eq. SVF_2D with the Dirac-comb image used to derive Eq. keyeqn);
  ``pad_reflect`` / ``direct4_reflect``: the same with the image continued by
  half-sample symmetric reflection instead of zeros (the paper leaves the
  boundary condition open).
* ``preint4_i64`` / ``preint4_f64``: Algorithm 1 step 2 (Sec. 3.1, RS1-RS4).
* ``stencil4``: Algorithm 1 step 3 (Table 1, Eq. final_eqn, App. F).
* ``direct4_iterated``: the iterated box-spline filter of Sec. 3.3.
* ``adjoint4``: the transpose of the plain definition (gradient with respect
  to the image); ``direct4_grad_fd``: central differences of ``direct4`` with
  respect to the scales.
* ``map4``: the optimal scale vector of Sec. 3.2.2, steps (i)-(iii).
* ``U_bound``: the elongation bound of Prop. 3.1.
* ``box_spline_hat`` / ``covarianceN`` / ``kurtosis_normN2`` / ``mapN`` /
  ``gaussian_correlation``: the N-direction box spline in the Fourier domain
  (Eq. const as a convolution of N boxes), its covariance (Eq. covariance),
  the paper's kurtosis norm (Eq. finalForm, written for any N), the optimal
  scale vector for any N (minimal kurtosis norm at the target covariance), and
  the normalised correlation of an m-fold iterated spline with the Gaussian of
  the same covariance (Sec. 3.3, Fig. errorplots).
* ``structure_cov``: the adaptive covariance field of the feature-preserving
  smoothing application (Sec. 4.2): structure tensor J = w * (g g^T) with the
  plain-definition window, C = sigma0^2 adj(J + tau I) / sqrt(det(J + tau I)).

* ``n6`` (module): the six-directional spline (pointwise by two independent
  methods), its filter on the hexagonal lattice that the six directions need
  (the transfer of the image, the plain definition on it, Algorithm 1 on the
  lattice) and the N-directional map solved through its optimality conditions.

The C source is ``bsf_oracle.c``; it is compiled with gcc on first use (or by
``__graft_entry__.build()``) into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bsf_oracle.c")
_SRC6 = os.path.join(_HERE, "bsf_oracle6.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libbsf_oracle.so")

_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle C sources into a shared library (gcc, -O2, no fast-math;
    OpenMP for the loops over independent pixels and rows)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC6))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-fopenmp", "-o", tmp, _SRC, _SRC6,
                               "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.bo_beta4.restype = ctypes.c_double
        lib.bo_beta4.argtypes = [_dp, ctypes.c_double, ctypes.c_double]
        lib.bo_beta4_lines.restype = ctypes.c_double
        lib.bo_beta4_lines.argtypes = [_dp, ctypes.c_double, ctypes.c_double]
        lib.bo_direct4.restype = None
        lib.bo_direct4.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, _i64p, ctypes.c_int64, _dp]
        lib.bo_adjoint4.restype = None
        lib.bo_adjoint4.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double, _i64p, ctypes.c_int64,
                                    _dp]
        lib.bo_preint4_i64.restype = None
        lib.bo_preint4_i64.argtypes = [_i64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64p]
        lib.bo_preint4_f64.restype = None
        lib.bo_preint4_f64.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
        lib.bo_stencil4.restype = ctypes.c_int64
        lib.bo_stencil4.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _i64p,
                                    ctypes.c_int64, _dp]
        lib.bo_map4.restype = ctypes.c_int
        lib.bo_map4.argtypes = [_dp, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                _dp, _u8p]
        lib.bo_U_bound.restype = ctypes.c_double
        lib.bo_U_bound.argtypes = [ctypes.c_double]
        lib.bo_num_threads.restype = ctypes.c_int
        lib.bo_num_threads.argtypes = []
        lib.bo_beta6.restype = ctypes.c_double
        lib.bo_beta6.argtypes = [_dp, ctypes.c_double, ctypes.c_double]
        lib.bo_alg1_hex6.restype = ctypes.c_int
        lib.bo_alg1_hex6.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, _i64p, ctypes.c_int64, ctypes.c_double,
                                     _dp]
        _lib = lib
    return _lib


def num_threads() -> int:
    """Host threads the oracle's parallel loops use (OpenMP; OMP_NUM_THREADS caps it)."""
    return int(_load().bo_num_threads())


def _d(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _ptr(x, t):
    return x.ctypes.data_as(t)


SQRT2 = np.sqrt(2.0)
ZP_SCALES = np.array([1.0, SQRT2, 1.0, SQRT2])  # b of Sec. 3.1 (Zwart-Powell element)

KIND_SCALES, KIND_COV, KIND_SRT = 0, 1, 2
FLAG_CLAMPED, FLAG_INFEASIBLE, FLAG_INVALID = 1, 2, 4


def beta4(a, x1, x2) -> float:
    """beta^4_a(x1, x2), area form (exact up to rounding)."""
    a = _d(a)
    return _load().bo_beta4(_ptr(a, _dp), float(x1), float(x2))


def beta4_lines(a, x1, x2) -> float:
    """beta^4_a(x1, x2), line-integral recursion form (independent evaluation)."""
    a = _d(a)
    return _load().bo_beta4_lines(_ptr(a, _dp), float(x1), float(x2))


def beta4_grid(a, X1, X2) -> np.ndarray:
    """beta4 at every point of broadcastable arrays X1, X2."""
    X1, X2 = np.broadcast_arrays(np.asarray(X1, float), np.asarray(X2, float))
    lib = _load()
    a = _d(a)
    pa = _ptr(a, _dp)
    out = np.empty(X1.shape)
    for i, (u, v) in enumerate(zip(X1.ravel(), X2.ravel())):
        out.flat[i] = lib.bo_beta4(pa, float(u), float(v))
    return out


def _idx(idx, HW):
    if idx is None:
        return None, -1
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    if idx.size and (idx.min() < 0 or idx.max() >= HW):
        raise ValueError("pixel index out of range")
    return idx, idx.size


def direct4(f, a, idx=None) -> np.ndarray:
    """O-direct: fbar[n] = sum_k f[k] beta_{a(n)}(n - k), zero outside the image.

    f: (H, W) array; a: (4, H, W) scale planes; idx: optional flat pixel indices.
    Returns (H, W) (idx None) or the values at idx.
    """
    f = _d(f)
    H, W = f.shape
    a = _d(a)
    assert a.shape == (4, H, W)
    ii, n = _idx(idx, H * W)
    out = np.empty(H * W if n < 0 else n)
    _load().bo_direct4(_ptr(f, _dp), H, W, _ptr(a, _dp),
                       _ptr(ii, _i64p) if ii is not None else None, n, _ptr(out, _dp))
    return out.reshape(H, W) if n < 0 else out


def pad_reflect(f, P: int) -> np.ndarray:
    """The image continued by half-sample symmetric reflection, P samples on
    every side: f[-1-i] = f[i] and f[n+i] = f[n-1-i], repeated with period 2n
    when P exceeds the image (reading R21 of the paper's open "appropriate
    boundary conditions", Sec. 2.1; the zero extension is the default)."""
    return np.pad(np.asarray(f), int(P), mode="symmetric")


def direct4_reflect(f, a, idx=None) -> np.ndarray:
    """O-direct with the reflected boundary: the plain definition on the image
    padded by reflection (``pad_reflect``) far enough to hold every footprint,
    evaluated at the original pixels (their scales; the pad's scales are never
    used)."""
    f = _d(f)
    H, W = f.shape
    a = _d(a)
    P = int(np.ceil(0.5 * np.max(a[0] + (a[1] + a[3]) / SQRT2 + a[2]))) + 3
    fp = pad_reflect(f, P)
    ap = np.pad(a, ((0, 0), (P, P), (P, P)), mode="edge")
    Wp = W + 2 * P
    ii = np.arange(H * W) if idx is None else np.asarray(idx, np.int64).ravel()
    jj = (ii // W + P) * Wp + (ii % W + P)
    out = direct4(fp, ap, jj)
    return out.reshape(H, W) if idx is None else out


def adjoint4(g, a, idx) -> np.ndarray:
    """O-adjoint: sum_n g[n] beta_{a(n)}(n - k) at the flat points idx (gradient of
    sum g * fbar with respect to the image)."""
    g = _d(g)
    H, W = g.shape
    a = _d(a)
    assert a.shape == (4, H, W)
    ii, n = _idx(idx, H * W)
    out = np.empty(n)
    _load().bo_adjoint4(_ptr(g, _dp), H, W, _ptr(a, _dp), float(np.max(a)), _ptr(ii, _i64p), n, _ptr(out, _dp))
    return out


def direct4_iterated(f, a, m: int) -> np.ndarray:
    """Sec. 3.3: the m-fold iterated filter, i.e. the plain definition applied m
    times, each pass with the scale vectors a(n) / sqrt(m)."""
    a = _d(a) / np.sqrt(m)
    out = _d(f)
    for _ in range(m):
        out = direct4(out, a)
    return out


def direct4_grad_fd(f, a, idx, h: float = 1e-3) -> np.ndarray:
    """Central finite differences (step h, FP64) of O-direct with respect to each
    scale a_k at the pixels idx: returns (4, len(idx)).  a(n) enters only fbar[n]."""
    f = _d(f)
    a = _d(a)
    out = np.empty((4, len(idx)))
    for k in range(4):
        ap = a.copy()
        am = a.copy()
        ap[k].flat[idx] += h
        am[k].flat[idx] -= h
        out[k] = (direct4(f, ap, idx) - direct4(f, am, idx)) / (2 * h)
    return out


def preint4_i64(f_int, P: int) -> np.ndarray:
    """Algorithm 1 step 2 in integers (sqrt2 factors taken out, g_b = 2 G), mod 2^64.

    f_int: (H, W) integer image.  Returns G of shape (H+2P, W+2P), int64.
    """
    f = np.ascontiguousarray(f_int, dtype=np.int64)
    H, W = f.shape
    G = np.empty((H + 2 * P, W + 2 * P), dtype=np.int64)
    _load().bo_preint4_i64(_ptr(f, _i64p), H, W, int(P), _ptr(G, _i64p))
    return G


def preint4_f64(f, P: int) -> np.ndarray:
    """Algorithm 1 step 2 in FP64, literally (with the sqrt2 factors): returns g_b."""
    f = _d(f)
    H, W = f.shape
    gb = np.empty((H + 2 * P, W + 2 * P))
    _load().bo_preint4_f64(_ptr(f, _dp), H, W, int(P), _ptr(gb, _dp))
    return gb


def stencil4(gb, H: int, W: int, P: int, a, idx=None):
    """Algorithm 1 step 3: 16-tap FD mesh of Table 1 on the ZP-interpolated g_b.

    Returns (out, n_outside); pixels whose taps leave the buffer get NaN.
    """
    gb = _d(gb)
    assert gb.shape == (H + 2 * P, W + 2 * P)
    a = _d(a)
    assert a.shape == (4, H, W)
    ii, n = _idx(idx, H * W)
    out = np.empty(H * W if n < 0 else n)
    bad = _load().bo_stencil4(_ptr(gb, _dp), H, W, int(P), _ptr(a, _dp),
                              _ptr(ii, _i64p) if ii is not None else None, n, _ptr(out, _dp))
    return (out.reshape(H, W) if n < 0 else out), int(bad)


def alg1_filter4(f, a, P: int, integer: bool, idx=None):
    """Algorithm 1 end to end (O-alg): pre-integration then the local FD step."""
    f = np.asarray(f)
    H, W = f.shape
    if integer:
        G = preint4_i64(f, P)
        gb = 2.0 * G.astype(np.float64)
    else:
        gb = preint4_f64(f, P)
    return stencil4(gb, H, W, P, a, idx)


def map4(params, kind: int, eps: float = 1e-3, eta: float = 1e-3):
    """O-map: covariance (kind 1) or (sigma, rho, theta) (kind 2) -> scales.

    params: (3, ...) planes.  Returns (a of shape (4, ...), flags uint8 of shape (...)).
    """
    params = _d(params)
    shp = params.shape[1:]
    npix = int(np.prod(shp)) if shp else 1
    a = np.empty((4,) + shp)
    flags = np.empty(shp, dtype=np.uint8)
    _load().bo_map4(_ptr(params, _dp), int(kind), npix, float(eps), float(eta), _ptr(a, _dp),
                    _ptr(flags, _u8p))
    return a, flags


def U_bound(phi: float) -> float:
    """Prop. 3.1: supremum of the elongation at orientation phi in [0, pi)."""
    return _load().bo_U_bound(float(phi))


def covariance4(a) -> np.ndarray:
    """Eq. covariance_ZP: C_a = (1/24) [[2a1^2+a2^2+a4^2, a2^2-a4^2], [., 2a3^2+a2^2+a4^2]]."""
    a = np.asarray(a, float)
    p = a * a
    return np.array([[2 * p[0] + p[1] + p[3], p[1] - p[3]],
                     [p[1] - p[3], 2 * p[2] + p[1] + p[3]]]) / 24.0


def kurtosis4_norm2(p) -> float:
    """||K||^2 up to the factor (mu4 - 3 mu2^2)^2 (App. E): sum p^4 + (p1^2+p3^2)(p2^2+p4^2), p = a^2."""
    p = np.asarray(p, float)
    return float(np.sum(p ** 4) + (p[0] ** 2 + p[2] ** 2) * (p[1] ** 2 + p[3] ** 2))


def _central_gradient(f):
    """Central differences of one (H, W) plane, with the border replicated."""
    fp = np.pad(f, 1, mode="edge")
    return 0.5 * (fp[1:-1, 2:] - fp[1:-1, :-2]), 0.5 * (fp[2:, 1:-1] - fp[:-2, 1:-1])


def structure_tensor(f, sigma_w: float) -> np.ndarray:
    """Sec. 4.2: J = w * (g g^T) per pixel, (3, H, W) planes (J11, J12, J22).

    f: (H, W) or (C, H, W) (the products of the channels are summed);
    g: central differences with the border replicated; w: the isotropic
    four-directional box spline a_k = sigma_w sqrt(6) (the covariance of a
    Gaussian of std sigma_w), applied by the plain definition (``direct4``)."""
    f = _d(f)
    if f.ndim == 2:
        f = f[None]
    H, W = f.shape[1:]
    P = np.zeros((3, H, W))
    for c in range(f.shape[0]):
        gx, gy = _central_gradient(f[c])
        P[0] += gx * gx
        P[1] += gx * gy
        P[2] += gy * gy
    a = np.full((4, H, W), sigma_w * np.sqrt(6.0))
    return np.stack([direct4(P[k], a) for k in range(3)])


def structure_cov(f, sigma_w: float, sigma0: float, tau: float) -> np.ndarray:
    """Sec. 4.2: the adaptive covariance field, (3, H, W) planes (C11, C12, C22):
    C = sigma0^2 adj(M) / sqrt(det M), M = J + tau I (long axis along the
    eigenvector of the smallest eigenvalue of J, det C = sigma0^4)."""
    J = structure_tensor(f, sigma_w)
    m11, m12, m22 = J[0] + tau, J[1], J[2] + tau
    s = sigma0 * sigma0 / np.sqrt(m11 * m22 - m12 * m12)
    return np.stack([s * m22, -s * m12, s * m11])


def directions(N: int) -> np.ndarray:
    """theta_k = (k - 1) pi / N, k = 1..N (the radially-uniform directions)."""
    return np.arange(N) * np.pi / N


def box_spline_hat(theta, a, W1, W2) -> np.ndarray:
    """Fourier transform of beta^N_a at the angular frequencies (W1, W2): the box
    spline is the convolution of N centred boxes of length a_k along u_k (Eq.
    const), so its transform is prod_k sinc(a_k u_k . w / 2), sinc(x) = sin(x)/x."""
    r = np.ones_like(np.asarray(W1, float))
    for t, ak in zip(theta, a):
        r = r * np.sinc(0.5 * ak * (np.cos(t) * W1 + np.sin(t) * W2) / np.pi)
    return r


def covarianceN(theta, a) -> np.ndarray:
    """Eq. covariance: (1/12) sum_k a_k^2 u_k u_k^T."""
    C = np.zeros((2, 2))
    for t, ak in zip(theta, a):
        u = np.array([np.cos(t), np.sin(t)])
        C += ak * ak / 12.0 * np.outer(u, u)
    return C


def kurtosis_normN2(theta, p) -> float:
    """||K||^2 of K = sum_k p_k^2 u_k u_k^T (Eq. finalForm up to the factor
    (mu4 - 3 mu2^2)), p = a^2: sum_{k,m} p_k^2 p_m^2 cos^2(theta_k - theta_m).
    For N = 4 it equals kurtosis4_norm2."""
    p = np.asarray(p, float)
    d = np.subtract.outer(np.asarray(theta, float), np.asarray(theta, float))
    return float((p ** 2) @ (np.cos(d) ** 2) @ (p ** 2))


def mapN(theta, C, eps: float = 1e-9, starts: int = 24, seed: int = 0) -> np.ndarray:
    """The optimal scale vector for any N: minimise kurtosis_normN2 over p = a^2
    subject to (1/12) sum p_k u_k u_k^T = C and p >= eps (the criterion of Sec.
    3.2.2, for N directions; the feasible set is an (N-3)-dimensional polytope
    and the objective is convex on it), by SLSQP from several starting points.
    Returns a (length N)."""
    from scipy.optimize import minimize
    theta = np.asarray(theta, float)
    U = np.stack([np.cos(theta) ** 2, np.cos(theta) * np.sin(theta), np.sin(theta) ** 2], axis=1) / 12.0
    c = np.array([C[0][0], C[0][1], C[1][1]], float)
    D = np.cos(np.subtract.outer(theta, theta)) ** 2
    scale = float(np.trace(np.asarray(C, float)))

    def f(p):
        q = p * p
        return q @ D @ q / scale ** 4

    def g(p):
        q = p * p
        return 4.0 * p * (D @ q) / scale ** 4

    cons = {"type": "eq", "fun": lambda p: (U.T @ p - c) / scale, "jac": lambda p: U.T / scale}
    rng = np.random.default_rng(seed)
    best = None
    for _ in range(starts):
        p0 = rng.uniform(0.2, 2.0, theta.size) * 12.0 * scale / theta.size
        r = minimize(f, p0, jac=g, constraints=[cons], bounds=[(eps, None)] * theta.size, method="SLSQP",
                     options={"ftol": 1e-15, "maxiter": 1000})
        if r.success and np.abs(U.T @ r.x - c).max() < 1e-9 * scale and (best is None or r.fun < best.fun):
            best = r
    if best is None:
        raise RuntimeError("mapN: no feasible optimum found")
    return np.sqrt(best.x)


def gaussian_correlation(theta, a, C, m: int = 1, half_width: float | None = None, n: int = 801) -> float:
    """Normalised correlation <beta, g> / (||beta|| ||g||) of the m-fold iterated
    spline beta^{N,m} (m-fold convolution of beta_{a / sqrt m}) with the Gaussian
    g of covariance C, by Parseval on a frequency grid: both transforms are real
    and even."""
    C = np.asarray(C, float)
    if half_width is None:
        half_width = 12.0 / np.sqrt(np.linalg.eigvalsh(C)[0])
    w = np.linspace(-half_width, half_width, n)
    W1, W2 = np.meshgrid(w, w)
    b = box_spline_hat(theta, np.asarray(a, float) / np.sqrt(m), W1, W2) ** m
    gh = np.exp(-0.5 * (C[0, 0] * W1 * W1 + 2 * C[0, 1] * W1 * W2 + C[1, 1] * W2 * W2))
    return float(np.sum(b * gh) / np.sqrt(np.sum(b * b) * np.sum(gh * gh)))


from . import n6  # noqa: E402,F401  (six-directional oracle)
