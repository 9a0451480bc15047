// Covariance -> optimal scale vector for the four-directional box spline
// (Sec. 3.2.2), per pixel, in FP32.
//
// The problem: find p = (a1^2, a2^2, a3^2, a4^2) >= eps with M p = c,
// c = 24 (C11, C12, C22) (Eq. covariance_ZP), minimising the kurtosis norm
// ||K||^2 ~ sum p_k^4 + (p1^2 + p3^2)(p2^2 + p4^2) (Eq. opt1, App. E).
// The solutions of M p = c form a line; here it is parameterised
// symmetrically by w = (p2 + p4)/2:
//   p1 = a - w, p3 = c - w, p2 = w + d, p4 = w - d,   a = c1/2, c = c3/2, d = c2/2.
// Along the line the objective's derivative is, up to a factor 8, the cubic
//   g(w) = 8 w^3 - 6 s1 w^2 + (4 s2 + 8 d^2) w - (s3 + s1 d^2),
//   s1 = a + c, s2 = a^2 + c^2, s3 = a^3 + c^3.
// With w = z + s1/4 it becomes z^3 + P z + Q = 0,
//   P = ((5/2)(a^2 + c^2) - 3 a c + 8 d^2) / 8 > 0,
//   Q = s1 (d^2 - (a - c)^2 / 4) / 8,
// whose single real root (P > 0) is z = -Q / (A^2 + P/3 + B^2),
// A = cbrt(|Q|/2 + sqrt(Q^2/4 + P^3/27)), B = P / (3A): Cardano's formula
// written without cancellation.  The objective is convex, so the constrained
// minimiser is that root clamped to the feasible interval
// |d| + eps <= w <= min(a, c) - eps.  (The paper pivots p4 = 1 and enumerates
// the real roots of its cubic zeta'(t); both give the same minimiser.)
//
// In FP32 a component much smaller than the largest is a difference of terms
// of the size of the covariance and loses its relative accuracy; where the
// kernel is also small (largest p below 500 px^2), so that the filter is
// sensitive to that loss, the pixel is re-solved in FP64 (map4_refine64),
// starting from the FP32 root.
//
// Elongations beyond Prop. 3.1's bound U(theta) = (1 + |sin 2t| + |cos 2t|)^2
// / (2 |sin 2t| |cos 2t|) are lowered to (1 - eta) U keeping the size
// s = lambda_max + lambda_min and the orientation (flag bit 0).  If p >= eps
// is still infeasible, w is the interval midpoint and p is raised to eps
// (flag bit 1).  Non-finite or non-positive-definite input: NaN scales,
// flag bit 2.
#pragma once

#include <math.h>

struct map4_result {
    float a[4];
    int flag;
};

// sin and cos of x in [0, 2 pi) in FP64: reduction by pi/2 with a two-part
// constant, then the Taylor series of sin and cos on [-pi/4, pi/4] to degree
// 15 / 16 (truncation below 1e-16).
__device__ __forceinline__ void map4_sincos64(double x, double& sn, double& cs) {
    const double PIO2_HI = 1.5707963267948966, PIO2_LO = 6.123233995736766e-17;
    const double k = rint(x * 0.63661977236758134);
    const double r = fma(-k, PIO2_LO, fma(-k, PIO2_HI, x));
    const double r2 = r * r;
    const double s = r * (1.0 + r2 * (-1.0 / 6 + r2 * (1.0 / 120 + r2 * (-1.0 / 5040 + r2 * (1.0 / 362880 + r2 *
                     (-1.0 / 39916800 + r2 * (1.0 / 6227020800.0 + r2 * (-1.0 / 1307674368000.0))))))));
    const double c = 1.0 + r2 * (-0.5 + r2 * (1.0 / 24 + r2 * (-1.0 / 720 + r2 * (1.0 / 40320 + r2 * (-1.0 / 3628800 +
                     r2 * (1.0 / 479001600.0 + r2 * (-1.0 / 87178291200.0 + r2 * (1.0 / 20922789888000.0))))))));
    const int q = ((int)k) & 3;
    sn = q == 0 ? s : (q == 1 ? c : (q == 2 ? -s : -c));
    cs = q == 0 ? c : (q == 1 ? -s : (q == 2 ? -c : s));
}

// FP64 re-solve of one pixel, started from the FP32 root w32.  Used where a
// component of p is small compared with the largest: there FP32 loses it to
// cancellation (it is a difference of terms of the size of the covariance),
// and the filter is sensitive to it because two widths are tiny.
static __device__ __noinline__ void map4_refine64(int kind, float v0, float v1, float v2, float eps, float eta, bool clamp,
                                           float w32, float* pk) {
    double c1, c2, c3;
    if (kind == BSF_PARAM_COV && !clamp) {
        c1 = 24.0 * v0;
        c2 = 24.0 * v1;
        c3 = 24.0 * v2;
    } else {
        double lmax, lmin, s2, cc2;
        if (kind == BSF_PARAM_SRT) {
            lmax = (double)v0 * (double)v0;
            lmin = lmax / (double)v1;
            map4_sincos64(fmod(2.0 * (double)v2, 6.283185307179586476925), s2, cc2);
            if (s2 == 0.0 && cc2 == 0.0) cc2 = 1.0;
        } else {
            const double a = v0, b = v1, c = v2;
            const double D = sqrt((a - c) * (a - c) + 4.0 * b * b);
            lmax = 0.5 * (a + c + D);
            lmin = (a * c - b * b) / lmax;
            cc2 = D > 0.0 ? (a - c) / D : 1.0;
            s2 = D > 0.0 ? 2.0 * b / D : 0.0;
        }
        if (clamp) {
            const double as = fabs(s2), ac = fabs(cc2);
            const double U = (1.0 + as + ac) * (1.0 + as + ac) / (2.0 * as * ac);
            const double rc = (1.0 - (double)eta) * U, s = lmax + lmin;
            lmin = s / (1.0 + rc);
            lmax = s - lmin;
        }
        const double m = 0.5 * (lmax + lmin), d = 0.5 * (lmax - lmin);
        c1 = 24.0 * (m + d * cc2);
        c2 = 24.0 * (d * s2);
        c3 = 24.0 * (m - d * cc2);
    }
    const double a = 0.5 * c1, c = 0.5 * c3, hd = 0.5 * c2, e = eps;
    const double lo = fabs(hd) + e, hi = fmin(a, c) - e;
    const double s1 = a + c, s2 = a * a + c * c, s3 = a * a * a + c * c * c, d2 = hd * hd;
    const double k1 = 4.0 * s2 + 8.0 * d2, k0 = s3 + s1 * d2;
    double w = w32;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const double g = ((8.0 * w - 6.0 * s1) * w + k1) * w - k0;
        const double gp = (24.0 * w - 12.0 * s1) * w + k1;
        w -= g / gp;
    }
    w = fmin(fmax(w, lo), hi);
    pk[0] = (float)(a - w);
    pk[1] = (float)(w + hd);
    pk[2] = (float)(c - w);
    pk[3] = (float)(w - hd);
}

// kind: BSF_PARAM_COV (v0,v1,v2) = (C11, C12, C22) or BSF_PARAM_SRT (sigma, rho, theta)
__device__ __forceinline__ map4_result map4_solve(int kind, float v0, float v1, float v2, float eps, float eta) {
    map4_result R;
    R.flag = 0;
    float lmax, lmin, th;
    if (kind == BSF_PARAM_SRT) {
        lmax = v0 * v0;
        lmin = __fdividef(lmax, v1);
        th = v2;
    } else {
        const float tr = v0 + v2;
        const float dd = sqrtf((v0 - v2) * (v0 - v2) + 4.f * v1 * v1);
        lmax = 0.5f * (tr + dd);
        const float det = fmaf(v0, v2, -v1 * v1);
        lmin = det / lmax;
        th = 0.5f * atan2f(2.f * v1, v0 - v2);
    }
    if (!(isfinite(lmax) && isfinite(lmin) && isfinite(th)) || !(lmin > 0.f) || !(lmax >= lmin)) {
        R.a[0] = R.a[1] = R.a[2] = R.a[3] = __int_as_float(0x7fc00000);
        R.flag = 4;
        return R;
    }
    // sin, cos of 2 theta via the hardware approximation on [-pi, pi)
    // (absolute error ~2^-21): theta is taken modulo pi first
    float s2, c2;
    {
        float t2 = 2.f * th;
        t2 -= 6.28318530717958648f * floorf(t2 * 0.159154943091895336f);  // [0, 2 pi)
        __sincosf(t2 - 3.14159265358979324f, &s2, &c2);                    // shifted by pi
        s2 = -s2;
        c2 = -c2;
    }
    const float as = fabsf(s2), ac = fabsf(c2);
    const float rho = lmax / lmin;
    bool clamp = false;
    if (as * ac > 1e-12f) {
        const float U = __fdividef((1.f + as + ac) * (1.f + as + ac), 2.f * as * ac);
        const float rc = (1.f - eta) * U;
        if (rho > rc) {
            const float s = lmax + lmin;
            lmin = __fdividef(s, 1.f + rc);
            lmax = s - lmin;
            clamp = true;
            R.flag |= 1;
        }
    }
    float c1, c2v, c3;
    if (kind == BSF_PARAM_COV && !clamp) {
        c1 = 24.f * v0;
        c2v = 24.f * v1;
        c3 = 24.f * v2;
    } else {
        // descriptor D2 -> covariance, written with the double angle
        const float m = 0.5f * (lmax + lmin), d = 0.5f * (lmax - lmin);
        c1 = 24.f * (m + d * c2);
        c2v = 24.f * (d * s2);
        c3 = 24.f * (m - d * c2);
    }
    const float ha = 0.5f * c1, hc = 0.5f * c3, hd = 0.5f * c2v, ahd = fabsf(hd);
    const float lo = ahd + eps;
    const float cmin = fminf(ha, hc);
    const float hi = cmin - eps;
    float p1, p2, p3, p4;
    float w_root = 0.f;
    if (!(lo <= hi)) {
        const float w = 0.5f * (lo + hi);
        p1 = fmaxf(ha - w, eps);
        p3 = fmaxf(hc - w, eps);
        p2 = fmaxf(w + hd, eps);
        p4 = fmaxf(w - hd, eps);
        R.flag |= 2;
    } else {
        // normalised cubic (scale-free, avoids FP32 overflow of P^3)
        const float sc = ha + hc + ahd;
        const float isc = __frcp_rn(sc);
        const float an = ha * isc, cn = hc * isc, dn = hd * isc;
        const float P = (2.5f * (an * an + cn * cn) - 3.f * an * cn + 8.f * dn * dn) * 0.125f;
        const float amc = an - cn;
        const float Q = (an + cn) * (dn * dn - 0.25f * amc * amc) * 0.125f;
        const float rr = sqrtf(0.25f * Q * Q + P * P * P * (1.f / 27.f));
        const float A = cbrtf(0.5f * fabsf(Q) + rr);
        const float B = __fdividef(P, 3.f * A);
        float z = -__fdividef(Q, A * A + P * (1.f / 3.f) + B * B);
        z -= __fdividef(z * z * z + P * z + Q, 3.f * z * z + P);  // one Newton step against rounding
        float w = sc * (z + 0.25f * (an + cn));
        w = fminf(fmaxf(w, lo), hi);
        w_root = w;
        // each component from the nearer end of the interval, so that small
        // components keep their relative accuracy
        if (w - lo <= hi - w) {
            const float v = w - lo;
            p2 = (ahd + hd) + eps + v;
            p4 = (ahd - hd) + eps + v;
            p1 = ha - w;
            p3 = hc - w;
        } else {
            const float v = hi - w;
            p1 = (ha - cmin) + eps + v;
            p3 = (hc - cmin) + eps + v;
            p2 = w + hd;
            p4 = w - hd;
        }
    }
    if (!(R.flag & 2)) {
        // a component well below the largest and not pinned at eps: redo in FP64
        const float pmax = fmaxf(fmaxf(p1, p2), fmaxf(p3, p4));
        const float thr = 0.05f * pmax, pin = 1.0001f * eps;
        const bool small = (p1 < thr && p1 > pin) || (p2 < thr && p2 > pin) || (p3 < thr && p3 > pin) ||
                           (p4 < thr && p4 > pin);
        // only small kernels (widths below ~22 px) are sensitive enough to need it:
        // with fewer lattice points the output depends more sharply on the widths
        if (small && pmax < 500.f) {
            float pk[4];
            map4_refine64(kind, v0, v1, v2, eps, eta, clamp, w_root, pk);
            p1 = pk[0];
            p2 = pk[1];
            p3 = pk[2];
            p4 = pk[3];
        }
    }
    R.a[0] = sqrtf(fmaxf(p1, 0.f));
    R.a[1] = sqrtf(fmaxf(p2, 0.f));
    R.a[2] = sqrtf(fmaxf(p3, 0.f));
    R.a[3] = sqrtf(fmaxf(p4, 0.f));
    return R;
}
