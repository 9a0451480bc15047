"""Six-directional (N = 6) box spline and its space-variant filter on a
hexagonal lattice.  TEST INFRASTRUCTURE ONLY: the same rule as the rest of
``oracle/`` applies (only the tests, ``smoke()`` and the benchmark's CPU legs
may use it; the CUDA library shares no code with it).

The paper defines the radially-uniform box spline for any N (Eq. const, Sec.
2.2.1) and its O(1) filter through Eq. keyeqn (Sec. 2.2.2), but realises the
pre-integration only for N = 2 and 4: for N = 6 the principal directions are off
the pixel lattice, and the paper notes that the running sums would then need an
interpolated image (Sec. 3.3).  The reading taken here: the image f = sum_k f[k] delta(x - k) is transferred ONCE,
mass-preservingly, onto the hexagonal lattice

    Lambda_h = { h (i + j/2, j sqrt(3)/2) : i, j integers },

on which the six directions 0, 30, ..., 150 degrees are all lattice directions
(lattice vectors (1,0), (1,1), (0,1), (-1,2), (-1,1), (-2,1) in (i, j), of
lengths b = h (1, sqrt3, 1, sqrt3, 1, sqrt3)).  Each pixel's mass goes to the
three vertices of the lattice triangle that contains it, with its barycentric
weights (the transpose of linear interpolation on the triangulation): total
mass and centre of mass of every pixel are kept.  The six-directional filter
is then the plain definition applied to that measure,

    fbar[n] = sum_{m in Lambda_h} mu[m] beta^6_{a(n)}(n - m),          (direct6_hex)

and Algorithm 1 is exact on the hexagonal lattice (``alg1_hex``): its running
sums along the six lattice vectors need no interpolation, and F of Eq. keyeqn
is the lattice sum against beta^6_b with the b above.  ``direct6`` is the
definition on the pixel comb itself; the difference between the two is the
method error of the transfer, reported separately from implementation parity.

The box spline itself is evaluated pointwise in two independent ways:
``betaN`` through the truncated power (cone spline) of the N directions and
the 2^N-term difference of Eq. FD_mesh, and ``betaN_recursive`` by the
definition Eq. const read as successive one-dimensional convolutions with
scaled boxes, integrated exactly between the break points.

``mapN_kkt`` / ``map6``: the optimal scale vector of Sec. 3.2.2 for N
directions -- the kurtosis criterion (Eq. opt1) with the norm written for N
directions -- solved by enumerating the active sets of the bounds p >= eps and
keeping the point that satisfies the Karush-Kuhn-Tucker conditions.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

SQRT3 = math.sqrt(3.0)
# lattice vectors (i, j) of the six directions 0, 30, 60, 90, 120, 150 degrees
HEX_VECTORS = ((1, 0), (1, 1), (0, 1), (-1, 2), (-1, 1), (-2, 1))
HEX_LENGTHS = (1.0, SQRT3, 1.0, SQRT3, 1.0, SQRT3)

FLAG_CLAMPED, FLAG_INFEASIBLE, FLAG_INVALID = 1, 2, 4


def directions(N: int) -> np.ndarray:
    """theta_k = (k - 1) pi / N (Sec. 2.2.1)."""
    return np.arange(N) * np.pi / N


# ----------------------------------------------------------------------------
# pointwise box spline
# ----------------------------------------------------------------------------

def cone_spline(theta, X1, X2) -> np.ndarray:
    """Truncated power T(x) = vol{ t >= 0 : sum t_k u_k = x } of the unit
    directions u_k = (cos theta_k, sin theta_k) (pairwise independent, all in
    an open half-plane).  Its Laplace transform is prod_k 1/(p . u_k); by
    partial fractions in two variables,

        T(x) = sum_k (det(u_k, x))_+^(N-2) / ((N-2)! prod_{j != k} det(u_k, u_j))

    on the half-plane that holds the directions, and 0 outside it."""
    th = np.asarray(theta, float)
    n = th.size
    X1 = np.asarray(X1, float)
    X2 = np.asarray(X2, float)
    U = np.stack([np.cos(th), np.sin(th)], 1)
    out = np.zeros(np.broadcast(X1, X2).shape)
    for k in range(n):
        den = float(math.factorial(n - 2))
        for j in range(n):
            if j != k:
                den *= U[k, 0] * U[j, 1] - U[k, 1] * U[j, 0]
        d = U[k, 0] * X2 - U[k, 1] * X1
        out += np.where(d > 0.0, d ** (n - 2), 0.0) / den
    # the half-plane: bounded by the line through 0 along the middle of the
    # empty sector (max theta, min theta + pi)
    mid = 0.5 * (th.max() + th.min() + np.pi)
    v = (math.cos(mid), math.sin(mid))
    side = np.sign(v[0] * U[:, 1] - v[1] * U[:, 0])
    assert np.all(side == side[0]), "directions must lie in an open half-plane"
    inside = side[0] * (v[0] * X2 - v[1] * X1) > 0.0
    return np.where(inside, out, 0.0)


def betaN(theta, a, X1, X2) -> np.ndarray:
    """beta^N_a(x) of Eq. const, centred: the density of sum_k T_k a_k u_k with
    T_k uniform on [-1/2, 1/2].  Writing each box as the difference of two
    shifted half-lines gives the 2^N-term difference of Eq. FD_mesh applied to
    the cone spline:

        beta(x) = (1/prod a) sum_q (-1)^|q| T(x + sum_k a_k u_k / 2 - sum_k q_k a_k u_k)."""
    th = np.asarray(theta, float)
    a = np.asarray(a, float)
    n = th.size
    U = np.stack([np.cos(th), np.sin(th)], 1)
    c = 0.5 * (a[:, None] * U).sum(0)
    X1 = np.asarray(X1, float)
    X2 = np.asarray(X2, float)
    r = np.zeros(np.broadcast(X1, X2).shape)
    for q in itertools.product((0, 1), repeat=n):
        qv = np.array(q, float)
        s = c - (qv * a) @ U
        r += (-1.0) ** int(qv.sum()) * cone_spline(th, X1 + s[0], X2 + s[1])
    return r / float(np.prod(a))


def _gauss_legendre(npts: int):
    x, w = np.polynomial.legendre.leggauss(npts)
    return x, w


def betaN_recursive(theta, a, x1: float, x2: float) -> float:
    """beta^N_a(x) by the definition Eq. const as successive convolutions:
    beta^2 is the indicator of the parallelogram {t1 a1 u1 + t2 a2 u2} divided
    by its area, and beta^K(x) = (1/a_K) int_{-a_K/2}^{a_K/2} beta^(K-1)(x - s u_K) ds.
    The integrand is a polynomial of degree <= K-3 between the points where
    x - s u_K crosses a break line of beta^(K-1) (lines along u_j, j < K,
    through the points sum_{k<K, k != j} +-a_k u_k / 2), so Gauss-Legendre with
    two nodes per piece integrates it exactly.  Slow; for pins only."""
    th = np.asarray(theta, float)
    a = np.asarray(a, float)
    U = np.stack([np.cos(th), np.sin(th)], 1)

    def det(u, v):
        return u[0] * v[1] - u[1] * v[0]

    def inside_zonotope(K, x):
        # x in {sum_{k<K} t_k a_k u_k, |t_k| <= 1/2}: support-function test on the edge normals
        for j in range(K):
            nrm = (-U[j, 1], U[j, 0])
            lim = 0.5 * sum(a[k] * abs(nrm[0] * U[k, 0] + nrm[1] * U[k, 1]) for k in range(K))
            if abs(nrm[0] * x[0] + nrm[1] * x[1]) > lim * (1 + 1e-12):
                return False
        return True

    def beta(K, x):
        if K == 2:
            d = det(U[0], U[1])
            t1 = det(x, U[1]) / d / a[0]
            t2 = det(U[0], x) / d / a[1]
            if abs(t1) <= 0.5 and abs(t2) <= 0.5:
                return 1.0 / (a[0] * a[1] * abs(d))
            return 0.0
        uK = U[K - 1]
        half = 0.5 * a[K - 1]
        cuts = {-half, half}
        for j in range(K - 1):
            den = det(U[j], uK)
            others = [k for k in range(K - 1) if k != j]
            for eps in itertools.product((-0.5, 0.5), repeat=len(others)):
                p = sum(e * a[k] * U[k] for e, k in zip(eps, others)) if others else np.zeros(2)
                s = det(U[j], (x[0] - p[0], x[1] - p[1])) / den
                if -half < s < half:
                    cuts.add(s)
        cuts = sorted(cuts)
        gx, gw = _gauss_legendre(2)
        total = 0.0
        for s0, s1 in zip(cuts[:-1], cuts[1:]):
            if s1 - s0 <= 0.0:
                continue
            sm = 0.5 * (s0 + s1)
            if not inside_zonotope(K - 1, (x[0] - sm * uK[0], x[1] - sm * uK[1])):
                continue
            for xi, wi in zip(gx, gw):
                s = sm + 0.5 * (s1 - s0) * xi
                total += 0.5 * (s1 - s0) * wi * beta(K - 1, (x[0] - s * uK[0], x[1] - s * uK[1]))
        return total / a[K - 1]

    return beta(th.size, (float(x1), float(x2)))


def support_extent(theta, a) -> tuple[float, float]:
    """Half-widths (x, y) of the bounding box of the support polygon of beta_a
    (Sec. 2.2.1): sum_k a_k |cos theta_k| / 2 and sum_k a_k |sin theta_k| / 2."""
    th = np.asarray(theta, float)
    a = np.asarray(a, float)
    return 0.5 * float(np.sum(a * np.abs(np.cos(th)))), 0.5 * float(np.sum(a * np.abs(np.sin(th))))


# ----------------------------------------------------------------------------
# the hexagonal lattice and the transfer of the image
# ----------------------------------------------------------------------------

def hex_position(i, j, h: float):
    """Cartesian position (x, y) of the lattice point (i, j) of Lambda_h."""
    i = np.asarray(i, float)
    j = np.asarray(j, float)
    return h * (i + 0.5 * j), h * j * (SQRT3 / 2.0)


def hex_splat(f, h: float, origin=(0, 0)):
    """Transfer of the image f[y, x] (zero outside) to Lambda_h: the mass f[k]
    of pixel k = (x, y) is shared between the vertices of the lattice triangle
    that contains k, in proportion to its barycentric coordinates.  With
    ``origin`` = (ox, oy), pixel (x, y) of f sits at (x + ox, y + oy) of the
    plane that holds the lattice (f is a crop of a larger image).  Returns
    (I, J, mass) for the lattice points that receive mass."""
    f = np.asarray(f, float)
    H, W = f.shape
    yy, xx = np.mgrid[0:H, 0:W]
    t = 2.0 * (yy + origin[1]) / (h * SQRT3)
    s = (xx + origin[0]) / h - 0.5 * t
    i = np.floor(s).astype(np.int64)
    j = np.floor(t).astype(np.int64)
    sg = s - i
    tg = t - j
    low = (sg + tg) < 1.0
    vi = np.where(low[None], np.stack([i, i + 1, i]), np.stack([i + 1, i, i + 1]))
    vj = np.where(low[None], np.stack([j, j, j + 1]), np.stack([j + 1, j + 1, j]))
    w = np.where(low[None], np.stack([1.0 - sg - tg, sg, tg]), np.stack([sg + tg - 1.0, 1.0 - sg, 1.0 - tg]))
    vi, vj, m = vi.ravel(), vj.ravel(), (w * f[None]).ravel()
    key = vj * (1 << 32) + (vi + (1 << 31))
    uk, inv = np.unique(key, return_inverse=True)
    mass = np.zeros(uk.size)
    np.add.at(mass, inv, m)
    J = uk >> 32
    I = (uk & ((1 << 32) - 1)) - (1 << 31)
    return I, J, mass


# ----------------------------------------------------------------------------
# the filter
# ----------------------------------------------------------------------------

def _pixels(idx, H, W):
    idx = np.arange(H * W) if idx is None else np.asarray(idx, np.int64).ravel()
    return idx, idx % W, idx // W


def direct6(f, a, idx=None) -> np.ndarray:
    """The plain definition on the pixel comb, N = 6: fbar[n] = sum_k f[k]
    beta^6_{a(n)}(n - k), zero outside the image; a has shape (6, H, W)."""
    f = np.asarray(f, float)
    H, W = f.shape
    th = directions(6)
    idx, nx, ny = _pixels(idx, H, W)
    out = np.empty(idx.size)
    for o, (x, y, p) in enumerate(zip(nx, ny, idx)):
        ap = np.asarray(a, float).reshape(6, -1)[:, p]
        ex, ey = support_extent(th, ap)
        x0, x1 = max(0, int(math.floor(x - ex))), min(W - 1, int(math.ceil(x + ex)))
        y0, y1 = max(0, int(math.floor(y - ey))), min(H - 1, int(math.ceil(y + ey)))
        ky, kx = np.mgrid[y0:y1 + 1, x0:x1 + 1]
        out[o] = float(np.sum(f[y0:y1 + 1, x0:x1 + 1] * betaN(th, ap, x - kx, y - ky)))
    return out


def direct6_hex(f, a, idx=None, h: float = 0.5, origin=(0, 0)) -> np.ndarray:
    """The six-directional filter as defined on the hexagonal lattice: the
    plain definition applied to the transferred measure (module docstring).
    ``origin``: as in ``hex_splat`` (f and a are crops whose pixel (0, 0) sits
    at origin; the result is exact for pixels whose footprint the crop holds)."""
    f = np.asarray(f, float)
    H, W = f.shape
    th = directions(6)
    I, J, mass = hex_splat(f, h, origin)
    PX, PY = hex_position(I, J, h)
    PX = PX - origin[0]
    PY = PY - origin[1]
    idx, nx, ny = _pixels(idx, H, W)
    out = np.empty(idx.size)
    for o, (x, y, p) in enumerate(zip(nx, ny, idx)):
        ap = np.asarray(a, float).reshape(6, -1)[:, p]
        ex, ey = support_extent(th, ap)
        sel = (np.abs(PX - x) <= ex) & (np.abs(PY - y) <= ey)
        out[o] = float(np.sum(mass[sel] * betaN(th, ap, x - PX[sel], y - PY[sel])))
    return out


def alg1_hex(f, a, idx=None, h: float = 0.5) -> np.ndarray:
    """Algorithm 1 (Sec. 3.1) restated for N = 6 on Lambda_h, in FP64:

    1. transfer the image to the lattice (``hex_splat``);
    2. pre-integrate: g_b = Delta_b^{-6} mu, six running sums along the lattice
       vectors v_k, each times its length b_k (Eq. 2DRS with b_k u_k = h v_k);
    3. for every pixel, Eq. keyeqn: fbar[n] = sum_i w_i F(n + tau - x_i) with the
       64 taps of Eq. FD_mesh, tau = (1/2) sum_k (a_k - b_k) u_k and
       F(y) = sum_m g_b[m] beta^6_b(y - m).

    The lattice box holds every point that step 3 reads, and extends to the
    right far enough that the running sums along 120 and 150 degrees (which
    come from the lower right) start in the empty part below the image; the
    sums therefore equal those over the whole plane.  Small images only."""
    f = np.asarray(f, float)
    H, W = f.shape
    th = directions(6)
    U = np.stack([np.cos(th), np.sin(th)], 1)
    b = h * np.array(HEX_LENGTHS)
    A = np.asarray(a, float).reshape(6, -1)
    idx, nx, ny = _pixels(idx, H, W)
    # extent of everything step 3 reads: footprint + interpolation support
    ex = max(support_extent(th, A[:, p])[0] for p in idx) + float(np.sum(b)) + 2 * h
    ey = max(support_extent(th, A[:, p])[1] for p in idx) + float(np.sum(b)) + 2 * h
    j_lo = int(math.floor(-ey / (h * SQRT3 / 2))) - 2
    j_hi = int(math.ceil((H - 1 + ey) / (h * SQRT3 / 2))) + 2
    nrow = j_hi - j_lo + 1
    i_lo = int(math.floor(-ex / h - 0.5 * j_hi)) - 2
    i_hi = int(math.ceil((W - 1 + ex) / h - 0.5 * j_lo)) + 2 + 2 * nrow
    ncol = i_hi - i_lo + 1
    g = np.zeros((nrow, ncol))
    I, J, mass = hex_splat(f, h)
    np.add.at(g, (J - j_lo, I - i_lo), mass)
    for (di, dj), bk in zip(HEX_VECTORS, b):
        out = np.zeros_like(g)
        if dj == 0:
            out = np.cumsum(g, axis=1)
        else:
            for r in range(nrow):
                out[r] = g[r]
                if r - dj >= 0:
                    src = out[r - dj]
                    # out[r, c] += out[r - dj, c - di]
                    if di >= 0:
                        out[r, di:] += src[:ncol - di]
                    else:
                        out[r, :ncol + di] += src[-di:]
        g = bk * out
    jj, ii = np.mgrid[j_lo:j_hi + 1, i_lo:i_hi + 1]
    LX, LY = hex_position(ii, jj, h)
    bx, by = support_extent(th, b)
    res = np.empty(idx.size)
    for o, (x, y, p) in enumerate(zip(nx, ny, idx)):
        ap = A[:, p]
        tau = 0.5 * ((ap - b)[:, None] * U).sum(0)
        acc = 0.0
        for q in itertools.product((0, 1), repeat=6):
            qv = np.array(q, float)
            yq = np.array([x, y]) + tau - (qv * ap) @ U
            sel = (np.abs(LX - yq[0]) <= bx + 1e-9) & (np.abs(LY - yq[1]) <= by + 1e-9)
            F = float(np.sum(g[sel] * betaN(th, b, yq[0] - LX[sel], yq[1] - LY[sel])))
            acc += (-1.0) ** int(qv.sum()) * F
        res[o] = acc / float(np.prod(ap))
    return res


def alg1_hex_c(f, a, idx=None, h: float = 0.5) -> np.ndarray:
    """``alg1_hex`` restated in C (``bsf_oracle6.c``): the same three steps in
    the same order and in FP64, with step 3 visiting only the lattice points
    inside the support of beta_b around each tap instead of testing the whole
    box, and the pixels shared among the host threads.  This is the form fast
    enough to time on a crop of a real workload (the benchmark's CPU baseline);
    pinned against ``alg1_hex``."""
    from . import _load, _d, _ptr, _dp, _i64p
    f = _d(f)
    H, W = f.shape
    A = _d(np.asarray(a, float).reshape(6, H, W))
    idx_a = np.arange(H * W, dtype=np.int64) if idx is None else np.ascontiguousarray(np.asarray(idx).ravel(),
                                                                                       dtype=np.int64)
    out = np.empty(idx_a.size)
    rc = _load().bo_alg1_hex6(_ptr(f, _dp), H, W, _ptr(A, _dp), _ptr(idx_a, _i64p), idx_a.size, float(h),
                              _ptr(out, _dp))
    if rc != 0:
        raise MemoryError("bo_alg1_hex6: lattice box too large")
    return out


def beta6_c(a, x1: float, x2: float) -> float:
    """beta^6_a(x) as the C restatement evaluates it (truncated power, 64 corners)."""
    from . import _load, _d, _ptr, _dp
    a = _d(a)
    return float(_load().bo_beta6(_ptr(a, _dp), float(x1), float(x2)))


# ----------------------------------------------------------------------------
# covariance -> scales for N directions
# ----------------------------------------------------------------------------

def U_boundN(phi: float, N: int, shrink: float = 1.0) -> float:
    """Largest elongation of an N-directional box spline oriented at phi.  The
    covariance (1/12) sum p_k u_k u_k^T with p >= 0, divided by its trace, has
    the traceless part (1/2) z R, R the reflection at angle 2 phi, where z runs
    over the convex hull of the points exp(2 i theta_k): a regular N-gon
    inscribed in the unit circle.  At the angle 2 phi its boundary is at radius
    r = cos(pi/N) / cos(psi - pi/N), psi = 2 phi mod 2 pi/N, and the elongation
    is (1 + r)/(1 - r).  For N = 4 this is Prop. 3.1's U(theta).  With
    ``shrink`` < 1 the polygon is scaled by it: the bound when every p_k must
    keep a share (1 - shrink)/N of the trace."""
    psi = math.fmod(2.0 * phi, 2.0 * math.pi / N)
    if psi < 0:
        psi += 2.0 * math.pi / N
    r = shrink * math.cos(math.pi / N) / math.cos(psi - math.pi / N)
    if r >= 1.0:
        return math.inf
    return (1.0 + r) / (1.0 - r)


def _hess_grad(D, p):
    q = p * p
    Dq = D @ q
    g = 4.0 * p * Dq
    Hm = 8.0 * np.outer(p, p) * D + 4.0 * np.diag(Dq)
    return float(q @ Dq), g, Hm


def _solve_face(M, c, D, active, bound, scale):
    """min sum_{k,m} p_k^2 p_m^2 D_km  s.t. M p = c, p_k = bound (k in active):
    Newton's method with backtracking on the affine face (the objective is
    convex on all of R^N).  Returns p or None when the face is empty."""
    n = D.shape[0]
    E = np.zeros((len(active), n))
    for r, k in enumerate(active):
        E[r, k] = 1.0
    Aeq = np.vstack([M, E])
    beq = np.concatenate([c, np.full(len(active), bound)])
    if np.linalg.matrix_rank(Aeq) < Aeq.shape[0]:
        return None
    p0 = np.linalg.lstsq(Aeq, beq, rcond=None)[0]
    if np.abs(Aeq @ p0 - beq).max() > 1e-12 * scale:
        return None
    _, sv, vt = np.linalg.svd(Aeq)
    Z = vt[Aeq.shape[0]:].T
    if Z.shape[1] == 0:
        return p0
    u = np.zeros(Z.shape[1])
    for _ in range(200):
        p = p0 + Z @ u
        f0, g, Hm = _hess_grad(D, p)
        gz = Z.T @ g
        Hz = Z.T @ Hm @ Z
        step = -np.linalg.solve(Hz, gz)
        dec = -float(gz @ step)
        if dec <= 1e-30 * scale ** 4:
            break
        t = 1.0
        # backtracking (Armijo) only while the decrease is well above the rounding
        # of the objective: near the optimum the test sees rounding noise alone and
        # would shrink the step to nothing, while the full Newton step of a convex
        # quartic converges there quadratically
        if dec > 1e-11 * abs(f0):
            while t > 1e-12:
                pn = p0 + Z @ (u + t * step)
                qn = pn * pn
                if float(qn @ D @ qn) <= f0 - 0.25 * t * dec:
                    break
                t *= 0.5
        u = u + t * step
        if t * np.abs(step).max() <= 1e-16 * scale:
            break
    return p0 + Z @ u


def mapN_kkt(theta, C, eps: float = 1e-3, bound_only: bool = False):
    """Optimal p = a^2 for the target covariance C (Sec. 3.2.2, Eq. opt1 with the
    N-directional kurtosis norm sum_{k,m} p_k^2 p_m^2 cos^2(theta_k - theta_m)):
    minimise it subject to (1/12) sum_k p_k u_k u_k^T = C and p >= eps.  The
    objective is strictly convex, so the minimiser is the unique point that
    satisfies the Karush-Kuhn-Tucker conditions; every set of at most N - 3
    active bounds is tried in turn (Newton on its face), and the feasible point
    whose bound multipliers are non-negative is returned.  Returns (p, ok);
    ok is False when no p >= eps reproduces C."""
    th = np.asarray(theta, float)
    n = th.size
    M = np.stack([np.cos(th) ** 2, np.cos(th) * np.sin(th), np.sin(th) ** 2]) / 12.0
    C = np.asarray(C, float)
    c = np.array([C[0, 0], C[0, 1], C[1, 1]])
    D = np.cos(np.subtract.outer(th, th)) ** 2
    scale = max(12.0 * float(C[0, 0] + C[1, 1]), 1e-300)
    best = None
    for size in range(0, n - 2):
        for active in itertools.combinations(range(n), size):
            p = _solve_face(M, c, D, list(active), eps, scale)
            if p is None or np.any(p < eps - 1e-11 * scale):
                continue
            _, g, _ = _hess_grad(D, p)
            E = np.zeros((len(active), n))
            for r, k in enumerate(active):
                E[r, k] = 1.0
            A = np.vstack([M, E]).T
            mult, *_ = np.linalg.lstsq(A, g, rcond=None)
            gs = max(np.abs(g).max(), 1e-300)
            if np.abs(A @ mult - g).max() > 1e-8 * gs:
                continue
            if np.any(mult[3:] < -1e-8 * gs):
                continue
            val = float((p * p) @ D @ (p * p))
            if best is None or val < best[0]:
                best = (val, p)
        if best is not None and size == 0:
            break
    if best is None:
        return None, False
    return best[1], True


def _cov_from_params(v0, v1, v2, kind):
    """(C11, C12, C22) and the descriptors (lmax, lmin, theta) of one pixel; kind 1
    = covariance, kind 2 = (sigma, rho, theta) with lmax = sigma^2, lmin = lmax/rho."""
    if kind == 2:
        lmax = float(v0) * float(v0)
        lmin = lmax / float(v1) if v1 != 0 else math.inf
        th = float(v2)
    else:
        tr = v0 + v2
        d = math.sqrt((v0 - v2) ** 2 + 4 * v1 * v1)
        lmax = 0.5 * (tr + d)
        lmin = (v0 * v2 - v1 * v1) / lmax if lmax > 0 else float("nan")
        th = 0.5 * math.atan2(2 * v1, v0 - v2)
    return lmax, lmin, th


REL_BOUND6 = 1e-3


def map6(params, kind: int, eps: float = 1e-3, eta: float = 1e-3, rel_bound: float = REL_BOUND6):
    """Per-pixel scales for N = 6 from covariance planes (kind 1) or (sigma,
    rho, theta) planes (kind 2), shape (3, ...).  The same conventions as the
    four-directional map, except the lower bound: p_k >= max(eps, 1e-3 T),
    T = sum_k p_k = 12 tr C (reading: the bound of Eq. opt1 is any small
    positive number; taken relative to the size, it keeps the smallest width
    at least 0.077 times the typical one, which the six-directional GPU path
    needs for its accuracy).  Elongations beyond the bound U of that
    constraint (U_boundN with the hexagon scaled by 1 - 6e-3) are lowered to
    (1 - eta) U keeping lmax + lmin and the orientation (flag 1); when no
    p >= bound reproduces the covariance, the minimiser over p >= 0 is raised
    to the bound (flag 2); invalid input gives NaN scales (flag 4).
    ``rel_bound`` replaces the share 1e-3 of the trace (0: the bound is eps
    alone, the paper's form of the constraint; the hexagon is then unscaled).
    Returns (a of shape (6, ...), flags uint8)."""
    P = np.asarray(params, float)
    shp = P.shape[1:]
    flat = P.reshape(3, -1)
    th6 = directions(6)
    a = np.empty((6, flat.shape[1]))
    flags = np.zeros(flat.shape[1], np.uint8)
    for p in range(flat.shape[1]):
        v0, v1, v2 = flat[:, p]
        lmax, lmin, th = _cov_from_params(v0, v1, v2, kind)
        if not (np.isfinite(lmax) and np.isfinite(lmin) and np.isfinite(th) and lmin > 0 and lmax >= lmin):
            a[:, p] = np.nan
            flags[p] = FLAG_INVALID
            continue
        fl = 0
        U = U_boundN(th, 6, 1.0 - 6.0 * rel_bound)
        if lmax / lmin > (1.0 - eta) * U:
            s = lmax + lmin
            lmin = s / (1.0 + (1.0 - eta) * U)
            lmax = s - lmin
            fl |= FLAG_CLAMPED
        if kind == 1 and not fl:
            C = np.array([[v0, v1], [v1, v2]])
        else:
            m, d = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
            C = np.array([[m + d * math.cos(2 * th), d * math.sin(2 * th)],
                          [d * math.sin(2 * th), m - d * math.cos(2 * th)]])
        bound = max(eps, rel_bound * 12.0 * (C[0, 0] + C[1, 1]))
        pk, ok = mapN_kkt(th6, C, bound)
        if not ok:
            pk, ok = mapN_kkt(th6, C, 0.0)
            pk = np.maximum(pk, bound)
            fl |= FLAG_INFEASIBLE
        a[:, p] = np.sqrt(pk)
        flags[p] = fl
    return a.reshape((6,) + shp), flags.reshape(shp)
