"""Generate hex6_tables.h: the polynomial pieces of the interpolation element of
the six-directional filter on the hexagonal lattice, in exact rational
arithmetic.

On the lattice Lambda_h = { h (i + j/2, j sqrt3/2) } the six directions of the
radially-uniform spline (Sec. 2.2.1, theta_k = k pi/6) are the lattice vectors
xi = (1,0), (1,1), (0,1), (-1,2), (-1,1), (-2,1) in lattice coordinates (s, t).
With the scales b_k = h |xi_k| the element beta^6_b of Eq. keyeqn becomes, in
those coordinates, the box spline M with integer directions xi_k (the density
of sum_k T_k xi_k, T_k uniform on [-1/2, 1/2]); F(y) = sum_m g[m] M((s,t) - m)
up to a constant.

M is a piecewise quartic whose break lines are the lines through lattice
points along the six directions.  In the unit cell (sigma, tau) in [0,1)^2 of
the point (s, t) they are sigma + tau = 1, sigma = tau, 2 sigma + tau = 1, 2
and sigma + 2 tau = 1, 2: each of the two lattice triangles of the cell is cut
by its three medians into six pieces, twelve in all.  For every piece r and
every lattice offset (di, dj) the value M(sigma + di, tau + dj) is one
polynomial in (sigma, tau); the point it weighs is m = (floor(s) - di,
floor(t) - dj).

The pieces are computed from the truncated power of the directions (its
Laplace transform is prod_k 1/(p . xi_k); by partial fractions,
T(x) = sum_k det(xi_k, x)_+^4 / (4! prod_{j != k} det(xi_k, xi_j)) on the
half-plane that holds the directions) and the box spline as the 64-term
difference M(x) = sum_q (-1)^|q| T(x + c - sum_k q_k xi_k), c = sum_k xi_k / 2.
Every term's truncation is fixed on a piece, so each piece is an exact
polynomial.  The script checks the result: the weights of a piece sum to the
polynomial 1 (partition of unity), pieces agree with their neighbours to third
order across every break line (M is C^3), and M is non-negative and symmetric.

Run: python hex6_gen.py [out.h]  (writes next to this file by default).
"""
from __future__ import annotations

import itertools
import os
import sys
from fractions import Fraction as Fr
from math import gcd

XI = ((1, 0), (1, 1), (0, 1), (-1, 2), (-1, 1), (-2, 1))
DEG = 4
# monomials sigma^a tau^b, a + b <= 4, in a fixed order
MONOS = [(a, d - a) for d in range(DEG + 1) for a in range(d, -1, -1)]


def det(u, v):
    return u[0] * v[1] - u[1] * v[0]


# ---- bivariate polynomials over Q: dict (a, b) -> Fraction ----

def padd(p, q, s=1):
    r = dict(p)
    for k, v in q.items():
        r[k] = r.get(k, Fr(0)) + s * v
    return {k: v for k, v in r.items() if v != 0}


def pmul(p, q):
    r = {}
    for (a1, b1), v1 in p.items():
        for (a2, b2), v2 in q.items():
            k = (a1 + a2, b1 + b2)
            r[k] = r.get(k, Fr(0)) + v1 * v2
    return {k: v for k, v in r.items() if v != 0}


def ppow(p, n):
    r = {(0, 0): Fr(1)}
    for _ in range(n):
        r = pmul(r, p)
    return r


def peval(p, x, y):
    return sum(v * x ** a * y ** b for (a, b), v in p.items())


def pderiv(p, ds, dt):
    r = {}
    for (a, b), v in p.items():
        if a >= ds and b >= dt:
            c = v
            for i in range(ds):
                c *= a - i
            for i in range(dt):
                c *= b - i
            r[(a - ds, b - dt)] = r.get((a - ds, b - dt), Fr(0)) + c
    return {k: v for k, v in r.items() if v != 0}


# ---- the element ----

DEN = []
for k, xk in enumerate(XI):
    d = Fr(24)
    for j, xj in enumerate(XI):
        if j != k:
            d *= det(xk, xj)
    DEN.append(d)
CENTER = (Fr(sum(x[0] for x in XI), 2), Fr(sum(x[1] for x in XI), 2))
# half-plane holding the directions (angles 0 .. 153.4 deg): det(v, x) > 0 with v at ~169 deg
HALF = (-10, 2)
assert all(det(HALF, x) < 0 for x in XI) or all(det(HALF, x) > 0 for x in XI)
HSIGN = 1 if det(HALF, XI[0]) > 0 else -1


def piece(sample, di, dj):
    """M(sigma + di, tau + dj) as a polynomial in (sigma, tau) on the piece that
    contains `sample` (an interior point of the unit cell)."""
    poly = {}
    for q in itertools.product((0, 1), repeat=6):
        sh = (CENTER[0] - sum(qk * x[0] for qk, x in zip(q, XI)) + di,
              CENTER[1] - sum(qk * x[1] for qk, x in zip(q, XI)) + dj)
        # point x = (sigma, tau) + sh
        px = (sample[0] + sh[0], sample[1] + sh[1])
        if HSIGN * det(HALF, px) <= 0:
            continue
        sign = -1 if sum(q) % 2 else 1
        for k, xk in enumerate(XI):
            if det(xk, px) <= 0:
                continue
            # det(xk, (sigma, tau) + sh) = xk0 * (tau + sh1) - xk1 * (sigma + sh0)
            lin = padd({(0, 1): Fr(xk[0]), (1, 0): Fr(-xk[1])}, {(0, 0): xk[0] * sh[1] - xk[1] * sh[0]})
            poly = padd(poly, {kk: sign * v / DEN[k] for kk, v in ppow(lin, DEG).items()})
    return poly


def region_samples():
    """Twelve pieces of the unit cell: centroids of the six sub-triangles of the
    lower triangle (vertices (0,0), (1,0), (0,1)) and of the upper one."""
    g = (Fr(1, 3), Fr(1, 3))
    low = [(0, 0), (1, 0), (0, 1)]
    up = [(1, 1), (0, 1), (1, 0)]
    out = []
    for tri, cen in ((low, g), (up, (Fr(2, 3), Fr(2, 3)))):
        mids = [((tri[(i + 1) % 3][0] + tri[(i + 2) % 3][0]) / Fr(2), (tri[(i + 1) % 3][1] + tri[(i + 2) % 3][1]) / Fr(2))
                for i in range(3)]
        for v in range(3):
            for m in range(3):
                if m == v:
                    continue
                # sub-triangle (vertex v, midpoint of an edge through v, centroid)
                pts = [tri[v], mids[m], cen]
                out.append((sum(p[0] for p in pts) / 3, sum(p[1] for p in pts) / 3))
    return out


def region_code(s, t):
    """3-bit code of a point of the unit cell plus its triangle (bit 3)."""
    if s + t < 1:
        return (s > t) | ((2 * s + t > 1) << 1) | ((s + 2 * t > 1) << 2)
    return 8 | (s > t) | ((2 * s + t > 2) << 1) | ((s + 2 * t > 2) << 2)


def build():
    samples = region_samples()
    assert len(samples) == 12
    codes = [region_code(*s) for s in samples]
    assert len(set(codes)) == 12
    lut = [-1] * 16
    for r, c in enumerate(codes):
        lut[c] = r
    tables = []
    for r, smp in enumerate(samples):
        slots = []
        for dj in range(-3, 3):
            for di in range(-3, 3):
                p = piece(smp, di, dj)
                if p:
                    slots.append((di, dj, p))
        tables.append(slots)
    # codes that no open piece produces (a point on a break line, after rounding)
    # go to a piece that touches the same point
    for c in range(16):
        if lut[c] < 0:
            up = c >> 3
            cand = [r for r, cc in enumerate(codes) if (cc >> 3) == up and bin((cc ^ c) & 7).count("1") == 1]
            lut[c] = cand[0]
    check(samples, tables)
    return samples, tables, lut


def check(samples, tables):
    for r, slots in enumerate(tables):
        tot = {}
        for _, _, p in slots:
            tot = padd(tot, p)
        assert tot == {(0, 0): Fr(1)}, f"partition of unity fails on piece {r}"
        for di, dj, p in slots:
            v = peval(p, *samples[r])
            assert v >= 0
            # symmetry M(x) = M(-x): the weight of offset (di, dj) at (sigma, tau)
            # equals M(-(sigma + di), -(tau + dj)) = M((1 - sigma) + (-1 - di), (1 - tau) + (-1 - dj))
            s2 = (1 - samples[r][0], 1 - samples[r][1])
            r2 = next(k for k, sm in enumerate(samples) if region_code(*sm) == region_code(*s2))
            q = next((pp for a, b, pp in tables[r2] if a == -1 - di and b == -1 - dj), {})
            assert peval(q, *s2) == v
    # C^3 across the break lines: pieces that share an edge agree in all derivatives of order <= 3 there
    pts = [(Fr(1, 2), Fr(1, 2)), (Fr(1, 4), Fr(1, 4)), (Fr(1, 3), Fr(1, 3)), (Fr(1, 2), Fr(0)),
           (Fr(2, 5), Fr(1, 5)), (Fr(1, 5), Fr(3, 5)), (Fr(3, 5), Fr(4, 5))]
    for s, t in pts:
        near = []
        for r, slots in enumerate(tables):
            near.append({(a, b): p for a, b, p in slots})
        for a in range(-3, 3):
            for b in range(-3, 3):
                vals = []
                for r in range(12):
                    p = near[r].get((a, b), {})
                    vals.append([peval(pderiv(p, i, j - i), s, t) for j in range(4) for i in range(j + 1)])
                # among the pieces whose closure holds (s, t), all agree
                owners = [r for r in range(12) if on_closure(samples[r], s, t)]
                for r in owners[1:]:
                    assert vals[r] == vals[owners[0]], (s, t, a, b, r)


# ---- the symmetries of the element: one canonical piece ----

R60 = ((0, -1), (1, 1))   # rotation by 60 degrees, in lattice coordinates (columns: images of e1, e2)
SREF = ((1, 1), (0, -1))  # reflection across the s axis


def mmul(A, B):
    return tuple(tuple(sum(A[i][k] * B[k][j] for k in range(2)) for j in range(2)) for i in range(2))


def mapply(A, p):
    return (A[0][0] * p[0] + A[0][1] * p[1], A[1][0] * p[0] + A[1][1] * p[1])


def lattice_symmetries():
    """The twelve linear symmetries of the hexagonal lattice (rotations by
    multiples of 60 degrees, with and without a reflection) as integer matrices
    in lattice coordinates.  Each maps the six directions to themselves up to
    sign, so M (the box spline of those directions) is invariant under it."""
    out, A = [], ((1, 0), (0, 1))
    for _ in range(6):
        out += [A, mmul(A, SREF)]
        A = mmul(R60, A)
    dirs = set(XI) | {(-a, -b) for a, b in XI}
    for L in out:
        assert all(mapply(L, x) in dirs for x in XI)
        assert abs(L[0][0] * L[1][1] - L[0][1] * L[1][0]) == 1
    assert len(set(out)) == 12
    return out


def compose(p, L, v):
    """p(L x + v) as a polynomial in x = (sigma, tau)."""
    ps = {(1, 0): Fr(L[0][0]), (0, 1): Fr(L[0][1]), (0, 0): Fr(v[0])}
    pt = {(1, 0): Fr(L[1][0]), (0, 1): Fr(L[1][1]), (0, 0): Fr(v[1])}
    out = {}
    for (a, b), c in p.items():
        out = padd(out, {k: c * w for k, w in pmul(ppow(ps, a), ppow(pt, b)).items()})
    return out


def canonical_maps(samples, tables, canon):
    """For every piece r an affine lattice map phi_r(x) = L x + v that takes the
    canonical piece onto piece r (both in the unit cell).  The weight of the
    lattice point phi_r(m) at phi_r(x) is the weight of m at x, so a point of
    piece r is evaluated with the canonical piece's polynomials at
    x = phi_r^-1(sigma, tau), the slots read at phi_r of the canonical slots.
    Checked exactly: every polynomial of piece r composed with phi_r is the
    canonical one of its slot."""
    maps = []
    for r in range(12):
        found = None
        for L in lattice_symmetries():
            for v in itertools.product(range(-2, 3), repeat=2):
                x = mapply(L, samples[canon])
                x = (x[0] + v[0], x[1] + v[1])
                if 0 < x[0] < 1 and 0 < x[1] < 1 and region_code(*x) == region_code(*samples[r]):
                    found = (L, v)
                    break
            if found:
                break
        assert found, r
        L, v = found
        byoff = {(di, dj): p for di, dj, p in tables[r]}
        order = []
        for di, dj, p0 in tables[canon]:
            m = mapply(L, (-di, -dj))
            key = (-(m[0] + v[0]), -(m[1] + v[1]))
            assert compose(byoff[key], L, v) == p0, (r, di, dj)
            order.append(key)
        assert sorted(order) == sorted(byoff)
        maps.append((L, v, order))
    return maps


def on_closure(sample, s, t):
    """True if (s, t) is in the closed piece that contains `sample`."""
    lines = [lambda x, y: x + y - 1, lambda x, y: x - y, lambda x, y: 2 * x + y - 1, lambda x, y: 2 * x + y - 2,
             lambda x, y: x + 2 * y - 1, lambda x, y: x + 2 * y - 2, lambda x, y: x, lambda x, y: y,
             lambda x, y: x - 1, lambda x, y: y - 1]
    for f in lines:
        a, b = f(*sample), f(s, t)
        if a * b < 0:
            return False
    return True


def emit(path):
    samples, tables, lut = build()
    nslot = max(len(s) for s in tables)
    assert all(len(s) == nslot for s in tables)
    # the canonical piece: the one with the fewest non-zero coefficients
    nnz = [sum(len(p) for _, _, p in slots) for slots in tables]
    canon = min(range(12), key=lambda r: (nnz[r], r))
    maps = canonical_maps(samples, tables, canon)
    # integer coefficients of the canonical piece: every coefficient times the common denominator
    den = 1
    for slots in tables:
        for _, _, p in slots:
            for v in p.values():
                den = den * v.denominator // gcd(den, v.denominator)
    rows = []
    for _, _, p in tables[canon]:
        vals = []
        for m in MONOS:
            v = p.get(m, Fr(0)) * den
            assert v.denominator == 1
            vals.append(v.numerator)
        rows.append(vals)
    lines = ["// Generated by hex6_gen.py -- do not edit.",
             "// Pieces of the six-directional interpolation element on the hexagonal",
             "// lattice.  The twelve pieces of a lattice cell are images of one canonical",
             "// piece under lattice symmetries phi_r(x) = L_r x + v_r, which leave the element",
             "// invariant.  A point of the cell at fractional position (sigma, tau) in piece r",
             "// has, at x = L_r^-1 ((sigma, tau) - v_r), the canonical weights: lattice point",
             "// (floor(s) - HEX6_DI[r][k], floor(t) - HEX6_DJ[r][k]) weighs",
             "// sum_m C[k][m] x_1^a_m x_2^b_m / HEX6_DEN, C = HEX6_CCOEF_INIT (monomial order below).",
             "#pragma once", "",
             f"#define HEX6_NREGION 12", f"#define HEX6_NSLOT {nslot}", f"#define HEX6_NMONO {len(MONOS)}",
             f"#define HEX6_DEN {den}", f"#define HEX6_CANON {canon}", "",
             "// monomial exponents (a, b) of x_1^a x_2^b",
             "static __device__ const int HEX6_MONO_A[HEX6_NMONO] = {" + ", ".join(str(a) for a, _ in MONOS) + "};",
             "static __device__ const int HEX6_MONO_B[HEX6_NMONO] = {" + ", ".join(str(b) for _, b in MONOS) + "};",
             "",
             "// piece of a code: bit 3 = upper triangle (sigma + tau >= 1), bit 0 = sigma > tau,",
             "// bit 1 = 2 sigma + tau > 1 (lower) or > 2 (upper), bit 2 = sigma + 2 tau > 1 or > 2",
             "static __device__ const int HEX6_REGION_LUT[16] = {" + ", ".join(str(v) for v in lut) + "};", "",
             "// per piece: L_r^-1 (row-major, 4 entries), then v_r",
             "static __device__ const int HEX6_SYM[HEX6_NREGION][6] = {"]
    for L, v, _ in maps:
        dt = L[0][0] * L[1][1] - L[0][1] * L[1][0]
        inv = (L[1][1] * dt, -L[0][1] * dt, -L[1][0] * dt, L[0][0] * dt)
        lines.append("    {" + ", ".join(str(x) for x in inv + tuple(v)) + "},")
    lines.append("};")
    lines.append("// offsets (di, dj) per piece and canonical slot")
    for nm, c in (("HEX6_DI", 0), ("HEX6_DJ", 1)):
        lines.append(f"static __device__ const signed char {nm}[HEX6_NREGION][HEX6_NSLOT] = {{")
        for _, _, order in maps:
            lines.append("    {" + ", ".join(str(o[c]) for o in order) + "},")
        lines.append("};")
    lines.append("// the canonical piece's coefficients (times HEX6_DEN), per slot and monomial, as")
    lines.append("// an initializer")
    lines.append("#define HEX6_CCOEF_INIT \\")
    for k in range(nslot):
        lines.append("    " + ("{" if k == 0 else " ") + "{" + ", ".join(str(v) for v in rows[k]) + "}" +
                     ("}" if k == nslot - 1 else ", \\"))
    text = "\n".join(lines) + "\n"
    if path is None:
        return text
    with open(path, "w") as fh:
        fh.write(text)
    return text


if __name__ == "__main__":
    out = sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                                "hex6_tables.h")
    emit(out)
    print("wrote", out)
