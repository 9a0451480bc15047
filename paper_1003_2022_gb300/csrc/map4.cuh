// Covariance -> optimal scale vector for the four-directional box spline
// (Sec. 3.2.2), per pixel, in FP32.
//
// The problem: find p = (a1^2, a2^2, a3^2, a4^2) >= eps with M p = c,
// c = 24 (C11, C12, C22) (Eq. covariance_ZP), minimising the kurtosis norm
// ||K||^2 ~ sum p_k^4 + (p1^2 + p3^2)(p2^2 + p4^2) (Eq. opt1, App. E).
// The solutions of M p = c form a line; here it is parameterised
// symmetrically by u = p2 + p4:
//   p1 = (c1 - u)/2, p3 = (c3 - u)/2, p2 = (u + c2)/2, p4 = (u - c2)/2,
// feasible for |c2| + 2 eps <= u <= min(c1, c3) - 2 eps.  The objective is a
// quartic in u whose second derivative 4 sum p^2 - 2 (p1+p3)(p2+p4) is
// positive, so its minimiser on the interval is unique: an end point if the
// derivative does not change sign there, else the root found by a bracketed
// Newton iteration.  (The paper pivots p4 = 1 and enumerates the real roots
// of the cubic derivative; both give the same minimiser.)
//
// Elongations beyond Prop. 3.1's bound U(theta) = (1 + |sin 2t| + |cos 2t|)^2
// / (2 |sin 2t| |cos 2t|) are lowered to (1 - eta) U keeping the size
// s = lambda_max + lambda_min and the orientation (flag bit 0).  If p >= eps
// is still infeasible, u is the interval midpoint and p is raised to eps
// (flag bit 1).  Non-finite or non-positive-definite input: NaN scales,
// flag bit 2.
#pragma once

#include <math.h>

struct map4_result {
    float a[4];
    int flag;
};

__device__ __forceinline__ float map4_dzeta(float p1, float p2, float p3, float p4) {
    const float s13 = p1 + p3, s24 = p2 + p4;
    const float q13 = p1 * p1 + p3 * p3, q24 = p2 * p2 + p4 * p4;
    return 2.f * (p2 * p2 * p2 + p4 * p4 * p4 - p1 * p1 * p1 - p3 * p3 * p3) + q13 * s24 - s13 * q24;
}

// kind: BSF_PARAM_COV (v0,v1,v2) = (C11, C12, C22) or BSF_PARAM_SRT (sigma, rho, theta)
__device__ __forceinline__ map4_result map4_solve(int kind, float v0, float v1, float v2, float eps, float eta) {
    map4_result R;
    R.flag = 0;
    float lmax, lmin, th;
    if (kind == BSF_PARAM_SRT) {
        lmax = v0 * v0;
        lmin = lmax / v1;
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
    float s2, c2;
    sincosf(2.f * th, &s2, &c2);
    const float as = fabsf(s2), ac = fabsf(c2);
    const float rho = lmax / lmin;
    bool clamp = false;
    if (as * ac > 1e-12f) {
        const float U = (1.f + as + ac) * (1.f + as + ac) / (2.f * as * ac);
        const float rc = (1.f - eta) * U;
        if (rho > rc) {
            const float s = lmax + lmin;
            lmax = s * rc / (1.f + rc);
            lmin = s / (1.f + rc);
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
    const float ac2 = fabsf(c2v);
    const float lo = ac2 + 2.f * eps;
    const float cmin = fminf(c1, c3);
    const float hi = cmin - 2.f * eps;
    float p1, p2, p3, p4;
    if (!(lo <= hi)) {
        const float u = 0.5f * (lo + hi);
        p1 = fmaxf(0.5f * (c1 - u), eps);
        p3 = fmaxf(0.5f * (c3 - u), eps);
        p2 = fmaxf(0.5f * (u + c2v), eps);
        p4 = fmaxf(0.5f * (u - c2v), eps);
        R.flag |= 2;
    } else {
        // the four components as functions of u, written from the nearer end of
        // the interval to keep small components accurate
        auto comps = [&](float u, float& q1, float& q2, float& q3, float& q4) {
            if (u - lo <= hi - u) {
                const float v = u - lo;  // >= 0
                q2 = 0.5f * (ac2 + c2v) + eps + 0.5f * v;
                q4 = 0.5f * (ac2 - c2v) + eps + 0.5f * v;
                q1 = 0.5f * (c1 - u);
                q3 = 0.5f * (c3 - u);
            } else {
                const float w = hi - u;  // >= 0
                q1 = 0.5f * (c1 - cmin) + eps + 0.5f * w;
                q3 = 0.5f * (c3 - cmin) + eps + 0.5f * w;
                q2 = 0.5f * (u + c2v);
                q4 = 0.5f * (u - c2v);
            }
        };
        float u;
        comps(lo, p1, p2, p3, p4);
        const float dlo = map4_dzeta(p1, p2, p3, p4);
        float q1, q2, q3, q4;
        comps(hi, q1, q2, q3, q4);
        const float dhi = map4_dzeta(q1, q2, q3, q4);
        if (dlo >= 0.f) {
            u = lo;
        } else if (dhi <= 0.f) {
            u = hi;
            p1 = q1; p2 = q2; p3 = q3; p4 = q4;
        } else {
            float a = lo, b = hi;
            u = 0.5f * (lo + hi);
#pragma unroll 1
            for (int it = 0; it < 40; ++it) {
                comps(u, p1, p2, p3, p4);
                const float g = map4_dzeta(p1, p2, p3, p4);
                if (g > 0.f) b = u; else a = u;
                const float s13 = p1 + p3, s24 = p2 + p4;
                const float h2 = 4.f * (p1 * p1 + p2 * p2 + p3 * p3 + p4 * p4) - 2.f * s13 * s24;
                float un = u - g / h2;
                if (!(un > a && un < b)) un = 0.5f * (a + b);
                if (un == u || b - a <= 0.f) break;
                u = un;
            }
            comps(u, p1, p2, p3, p4);
        }
    }
    R.a[0] = sqrtf(fmaxf(p1, 0.f));
    R.a[1] = sqrtf(fmaxf(p2, 0.f));
    R.a[2] = sqrtf(fmaxf(p3, 0.f));
    R.a[3] = sqrtf(fmaxf(p4, 0.f));
    return R;
}
