// Six-directional filter (N = 6: theta_k = k pi / 6, Sec. 2.2.1) on the
// hexagonal lattice Lambda_h = { h (i + j/2, j sqrt3/2) }.
//
// Algorithm 1 (Sec. 3.1) needs every direction b_k u_k to be a lattice vector;
// on the pixel lattice that holds for N = 2 and 4 only, and for more
// directions the paper notes that the running sums would need an interpolated
// image (Sec. 3.3).  Here the image is transferred once, mass-preservingly, to
// Lambda_h, where all six directions are lattice vectors (1,0), (1,1), (0,1),
// (-1,2), (-1,1), (-2,1) in lattice coordinates (i, j), with b_k = h |v_k| =
// h (1, sqrt3, 1, sqrt3, 1, sqrt3).  Each pixel's mass goes to the vertices of
// the lattice triangle that holds it, in proportion to its barycentric
// coordinates; gathered per lattice point m, the weight of pixel k is the
// piecewise-linear hat of m at k.  On Lambda_h the algorithm is exact:
//   step 2: six running sums along the lattice vectors (Eq. 2DRS);
//   step 3: Eq. keyeqn, 64 taps of Eq. FD_mesh, F(y) = sum_m g[m] beta^6_b(y - m)
//           with the element's exact polynomial pieces (hex6_tables.h, 24
//           lattice points per tap).
// Sixth-order running sums of a whole image outgrow any fixed word (they grow
// like L^6 and the 64-tap difference cancels them), so each tile of output
// pixels (64 x 64, 16 x 16 for small footprints, groups of up to 4 x 2 64-tiles
// for large ones) gets its own window of the lattice, sized from the tile's
// largest footprint, holding the running sums exactly as 128-bit integers.  The window is a parallelogram with sides along 0 and 150
// degrees, stored row by row (row r = j - j0, column c = i - i_left + 2r): in
// those coordinates every lattice direction has non-negative components, so
// each running sum enters the window through its bottom or left side, where
// the sums over the whole plane are zero, and the window's sums equal the
// whole-plane ones.  The scale map for six directions (Sec. 3.2.2 with the
// kurtosis norm written for N directions) is solved per pixel by a primal
// active-set Newton method, in FP32 first and to its end in FP64.
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>

#include "bsf_common.cuh"
#include "bsf_internal.h"
#include "hex6_tables.h"
#include "map4.cuh"  // map4_sincos64: FP64 sin and cos from the Taylor series

namespace {

#define BSF_QNAN64 __longlong_as_double(0x7ff8000000000000LL)

// cos / sin of 2 theta_k, theta_k = k pi / 6, and the null-space basis of the
// covariance constraint, rows z_k = (cos 4 theta_k, sin 4 theta_k, (-1)^k)
// (orthogonal columns of norms^2 3, 3, 6).  In constant memory: the solver
// indexes them with the (per-lane) active constraints.
__constant__ double MAP6_C2[6] = {1.0, 0.5, -0.5, -1.0, -0.5, 0.5};
__constant__ double MAP6_S2[6] = {0.0, 0.86602540378443864676, 0.86602540378443864676, 0.0,
                                  -0.86602540378443864676, -0.86602540378443864676};
__constant__ double MAP6_Z[6][3] = {{1.0, 0.0, 1.0},
                                    {-0.5, 0.86602540378443864676, -1.0},
                                    {-0.5, -0.86602540378443864676, 1.0},
                                    {1.0, 0.0, -1.0},
                                    {-0.5, 0.86602540378443864676, 1.0},
                                    {-0.5, -0.86602540378443864676, -1.0}};

__constant__ float MAP6_C2F[6] = {1.0f, 0.5f, -0.5f, -1.0f, -0.5f, 0.5f};
__constant__ float MAP6_S2F[6] = {0.0f, 0.86602540378443864676f, 0.86602540378443864676f, 0.0f,
                                  -0.86602540378443864676f, -0.86602540378443864676f};
__constant__ float MAP6_ZF[6][3] = {{1.0f, 0.0f, 1.0f},
                                    {-0.5f, 0.86602540378443864676f, -1.0f},
                                    {-0.5f, -0.86602540378443864676f, 1.0f},
                                    {1.0f, 0.0f, -1.0f},
                                    {-0.5f, 0.86602540378443864676f, 1.0f},
                                    {-0.5f, -0.86602540378443864676f, -1.0f}};
// the constants above in the precision R of the solver
template <class R>
struct m6c;
template <>
struct m6c<double> {
    static __device__ __forceinline__ double c2(int k) { return MAP6_C2[k]; }
    static __device__ __forceinline__ double s2(int k) { return MAP6_S2[k]; }
    static __device__ __forceinline__ double z(int k, int l) { return MAP6_Z[k][l]; }
};
template <>
struct m6c<float> {
    static __device__ __forceinline__ float c2(int k) { return MAP6_C2F[k]; }
    static __device__ __forceinline__ float s2(int k) { return MAP6_S2F[k]; }
    static __device__ __forceinline__ float z(int k, int l) { return MAP6_ZF[k][l]; }
};

// ---- double-float (a pair of FP32 numbers, about 48 bits) ----
struct dflt {
    float hi, lo;
};
__device__ __forceinline__ dflt df_norm(float s, float e) {
    const float hi = s + e;
    return {hi, e - (hi - s)};
}
__device__ __forceinline__ dflt df_mul(dflt a, dflt b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_norm(p, e);
}
__device__ __forceinline__ dflt df_add(dflt a, dflt b) {
    // two-sum of the high parts, then the low parts
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    return df_norm(s, e);
}
// a * b + c in double-float
__device__ __forceinline__ dflt df_fma(dflt a, dflt b, dflt c) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float s = p + c.hi;
    const float bb = s - p;
    e += (p - (s - bb)) + (c.hi - bb);
    e += c.lo;
    return df_norm(s, e);
}
// Integer -> float conversions without 64-bit conversion instructions: those run on
// the FP64 pipe (1/64 of the FP32 rate on GB300) and, at 16 coefficients per tap,
// kept it 80 % busy in the stencil.  A 23-bit integer becomes a float exactly through
// its bit pattern: the float 2^23 (or 1.5 * 2^23 for a signed one) with the integer
// added to its mantissa, minus the same constant.
__device__ __forceinline__ float exact_f32_u23(unsigned c) {  // c < 2^23
    return __int_as_float(0x4B000000 | (int)c) - 8388608.0f;
}
__device__ __forceinline__ float exact_f32_s22(int c) {  // -2^22 <= c < 2^22
    return __int_as_float(0x4B400000 + c) - 12582912.0f;
}
// a 128-bit integer as a double-float (to about 48 bits): |a| normalised to 62 bits
// (v = a 2^(62 - n), n its bit length), v cut into 23 + 23 + 17 bits converted exactly,
// the two high parts added exactly (two-sum), the low one rounded into the low part, and
// the scale 2^(n - 62) applied (exact)
__device__ __forceinline__ dflt df_of_i128(i128 a) {
    const long long hw = (long long)(a >> 64);
    const unsigned long long lw = (unsigned long long)a;
    // bit length of |a| (one less for negative a: enough to place the top bit)
    const unsigned long long mh = (unsigned long long)(hw ^ (hw >> 63));
    const unsigned long long ml = lw ^ (unsigned long long)(hw >> 63);
    const int n = mh ? 128 - __clzll((long long)mh) : 64 - __clzll((long long)ml);
    // for n <= 62 the value is its low 64 bits (two's complement)
    const long long v = n > 62 ? (long long)(a >> (n - 62)) : (long long)(lw << (62 - n));
    const float f2 = exact_f32_s22((int)(v >> 40)) * 1099511627776.0f;               // * 2^40
    const float f1 = exact_f32_u23((unsigned)(v >> 17) & 0x7FFFFFu) * 131072.0f;      // * 2^17
    const float f0 = exact_f32_u23((unsigned)v & 0x1FFFFu);
    const float s = f2 + f1;
    const float bb = s - f2;
    const float e = ((f2 - (s - bb)) + (f1 - bb)) + f0;
    const float sc = __int_as_float((127 + n - 62) << 23);  // 2^(n - 62), exact
    return df_norm(s * sc, e * sc);
}
// the fraction (48 bits, x / 2^48) of a lattice coordinate as a double-float (exact):
// two 24-bit halves, each converted as a 32-bit integer (exact below 2^24)
__device__ __forceinline__ dflt df_of_frac48(long long x) {
    return {(float)(int)(x >> 24) * 5.9604644775390625e-8f, (float)(int)(x & 0xFFFFFF) * 3.552713678800501e-15f};
}

// ||K||^2 for six directions: sum_{k,m} p_k^2 p_m^2 cos^2(theta_k - theta_m)
// = (S0^2 + |S1|^2) / 2, S0 = sum q_k, S1 = sum q_k exp(2 i theta_k), q = p^2
template <class R>
__device__ __forceinline__ R kurt6(const R p[6]) {
    R s0 = 0, sr = 0, si = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const R q = p[k] * p[k];
        s0 += q;
        sr += q * m6c<R>::c2(k);
        si += q * m6c<R>::s2(k);
    }
    return R(0.5) * (s0 * s0 + sr * sr + si * si);
}

template <class R>
__device__ __forceinline__ void p_of_t(const R pbar[6], const R t[3], R p[6]) {
#pragma unroll
    for (int k = 0; k < 6; ++k)
        p[k] = pbar[k] + m6c<R>::z(k, 0) * t[0] + m6c<R>::z(k, 1) * t[1] + m6c<R>::z(k, 2) * t[2];
}

// A x = b for a symmetric positive definite d x d matrix, d = 1, 2, 3 (unrolled Cholesky)
template <class R>
__device__ __forceinline__ bool spd_solve(int d, const R A[3][3], const R b[3], R x[3]) {
    if (d == 1) {
        if (!(A[0][0] > R(0))) return false;
        x[0] = b[0] / A[0][0];
        return true;
    }
    if (d == 2) {
        const R det = A[0][0] * A[1][1] - A[0][1] * A[0][1];
        if (!(A[0][0] > R(0)) || !(det > R(0))) return false;
        const R id = R(1) / det;
        x[0] = (A[1][1] * b[0] - A[0][1] * b[1]) * id;
        x[1] = (A[0][0] * b[1] - A[0][1] * b[0]) * id;
        return true;
    }
    if (!(A[0][0] > R(0))) return false;
    const R l00 = sqrt(A[0][0]);
    const R l10 = A[1][0] / l00, l20 = A[2][0] / l00;
    const R d11 = A[1][1] - l10 * l10;
    if (!(d11 > R(0))) return false;
    const R l11 = sqrt(d11);
    const R l21 = (A[2][1] - l20 * l10) / l11;
    const R d22 = A[2][2] - l20 * l20 - l21 * l21;
    if (!(d22 > R(0))) return false;
    const R l22 = sqrt(d22);
    const R y0 = b[0] / l00, y1 = (b[1] - l10 * y0) / l11, y2 = (b[2] - l20 * y0 - l21 * y1) / l22;
    x[2] = y2 / l22;
    x[1] = (y1 - l21 * x[2]) / l11;
    x[0] = (y0 - l10 * x[1] - l20 * x[2]) / l00;
    return true;
}

// The active-set Newton iteration on the null-space coordinates t (p = pbar + Z t)
// from a feasible t with the working set wmask (nw bounds): a Newton step on the
// face of the working set, the ratio test against the other bounds, Armijo
// backtracking far from the optimum; on convergence (a step below step_tol * T)
// the bound multipliers, and the most negative one (below -mult_tol * |g|)
// leaves the working set.  R = float for the first pass, double for the last.
template <class R>
__device__ __forceinline__ void map6_newton(const R pbar[6], R lb, R T, R t[3], int& wmask, int& nw, int max_it, R step_tol,
                            R mult_tol, R armijo_rel) {
    for (int it = 0; it < max_it; ++it) {
        R p[6];
        p_of_t(pbar, t, p);
        R s0 = 0, sr = 0, si = 0;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const R q = p[k] * p[k];
            s0 += q;
            sr += q * m6c<R>::c2(k);
            si += q * m6c<R>::s2(k);
        }
        const R h0 = R(0.5) * (s0 * s0 + sr * sr + si * si);
        // gradient and Hessian in t: H = 4 (sg sg^T + mr mr^T + mi mi^T) + 4 Z^T diag(Dq) Z
        R g[3] = {0, 0, 0}, Hm[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        R sg[3] = {0, 0, 0}, mr[3] = {0, 0, 0}, mi[3] = {0, 0, 0};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const R dq = R(0.5) * (s0 + m6c<R>::c2(k) * sr + m6c<R>::s2(k) * si);
            const R gp = R(4) * p[k] * dq;
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                const R z = m6c<R>::z(k, l);
                g[l] += z * gp;
                sg[l] += p[k] * z;
                mr[l] += m6c<R>::c2(k) * p[k] * z;
                mi[l] += m6c<R>::s2(k) * p[k] * z;
#pragma unroll
                for (int m = 0; m <= l; ++m) Hm[l][m] += R(4) * dq * z * m6c<R>::z(k, m);
            }
        }
#pragma unroll
        for (int l = 0; l < 3; ++l)
#pragma unroll
            for (int m = 0; m <= l; ++m) {
                Hm[l][m] += R(4) * (sg[l] * sg[m] + mr[l] * mr[m] + mi[l] * mi[m]);
                Hm[m][l] = Hm[l][m];
            }
        // the first two bounds of the working set, and an orthonormal basis N of
        // the directions that keep them
        R za[3] = {0, 0, 0}, zb[3] = {0, 0, 0};
        int seen = 0;
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if ((wmask >> k) & 1) {
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    if (seen == 0) za[l] = m6c<R>::z(k, l);
                    if (seen == 1) zb[l] = m6c<R>::z(k, l);
                }
                ++seen;
            }
        const int d = 3 - nw;
        R N[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        if (nw == 1) {
            const R zn = sqrt(za[0] * za[0] + za[1] * za[1] + za[2] * za[2]);
            const R n1[3] = {za[0] / zn, za[1] / zn, za[2] / zn};
            // u: the unit vector of the smallest component of n1, made orthogonal to n1
            R u[3] = {0, 0, 0};
            const int e = (fabs(n1[1]) < fabs(n1[0])) ? ((fabs(n1[2]) < fabs(n1[1])) ? 2 : 1)
                                                         : ((fabs(n1[2]) < fabs(n1[0])) ? 2 : 0);
            const R dd = e == 0 ? n1[0] : (e == 1 ? n1[1] : n1[2]);
#pragma unroll
            for (int l = 0; l < 3; ++l) u[l] = (l == e ? R(1) : R(0)) - dd * n1[l];
            const R un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
            for (int l = 0; l < 3; ++l) u[l] /= un;
            const R v[3] = {n1[1] * u[2] - n1[2] * u[1], n1[2] * u[0] - n1[0] * u[2], n1[0] * u[1] - n1[1] * u[0]};
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                N[l][0] = u[l];
                N[l][1] = v[l];
            }
        } else if (nw == 2) {
            const R n[3] = {za[1] * zb[2] - za[2] * zb[1], za[2] * zb[0] - za[0] * zb[2],
                                 za[0] * zb[1] - za[1] * zb[0]};
            const R nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
#pragma unroll
            for (int l = 0; l < 3; ++l) N[l][0] = n[l] / nn;
        }
        R step[3] = {0, 0, 0}, dec = 0;
        if (d > 0) {
            R Hr[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, gr[3] = {0, 0, 0}, u[3] = {0, 0, 0};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a >= d) continue;
#pragma unroll
                for (int l = 0; l < 3; ++l) gr[a] -= N[l][a] * g[l];
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    if (b >= d) continue;
                    R sab = 0;
#pragma unroll
                    for (int l = 0; l < 3; ++l)
#pragma unroll
                        for (int m = 0; m < 3; ++m) sab += N[l][a] * Hm[l][m] * N[m][b];
                    Hr[a][b] = sab;
                }
            }
            if (!spd_solve(d, Hr, gr, u)) break;
#pragma unroll
            for (int l = 0; l < 3; ++l) step[l] = N[l][0] * u[0] + (d > 1 ? N[l][1] * u[1] : R(0)) +
                                                  (d > 2 ? N[l][2] * u[2] : R(0));
            dec = -(g[0] * step[0] + g[1] * step[1] + g[2] * step[2]);
        }
        // converged on the face when the Newton step is at the rounding level of t
        // (the decrement alone cannot tell: near the optimum it is rounding noise)
        const R smax = fmax(fabs(step[0]), fmax(fabs(step[1]), fabs(step[2])));
        if (d == 0 || dec <= R(0) || smax <= step_tol * T) {
            // converged on the face: bound multipliers from g = sum_{k in W} lambda_k z_k
            if (nw == 0) return;
            // (fixed trip counts with guards: every array index is known at compile time, so the
            // arrays stay in registers)
            R G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, rhs[3] = {0, 0, 0}, lam[3] = {0, 0, 0};
            int idx[3] = {0, 0, 0}, a = 0;
#pragma unroll
            for (int k = 0; k < 6; ++k)
                if ((wmask >> k) & 1) {
                    idx[0] = a == 0 ? k : idx[0];
                    idx[1] = a == 1 ? k : idx[1];
                    idx[2] = a == 2 ? k : idx[2];
                    ++a;
                }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (i >= nw) break;
                const int ki = idx[i];
                rhs[i] = m6c<R>::z(ki, 0) * g[0] + m6c<R>::z(ki, 1) * g[1] + m6c<R>::z(ki, 2) * g[2];
#pragma unroll
                for (int j2 = 0; j2 < 3; ++j2) {
                    if (j2 >= nw) break;
                    const int kj = idx[j2];
                    G[i][j2] = m6c<R>::z(ki, 0) * m6c<R>::z(kj, 0) + m6c<R>::z(ki, 1) * m6c<R>::z(kj, 1) +
                               m6c<R>::z(ki, 2) * m6c<R>::z(kj, 2);
                }
            }
            if (!spd_solve(nw, G, rhs, lam)) return;
            int worst = -1;
            const R gs = fmax(fabs(g[0]), fmax(fabs(g[1]), fabs(g[2])));
            R lw = -mult_tol * (gs + R(1e-30));
#pragma unroll
            for (int i = 0; i < 3; ++i)
                if (i < nw && lam[i] < lw) {
                    lw = lam[i];
                    worst = idx[i];
                }
            if (worst < 0) return;
            wmask &= ~(1 << worst);
            --nw;
            continue;
        }
        // longest step along the Newton direction that keeps p >= lb
        R amax = 1;
        int blk = -1;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if ((wmask >> k) & 1) continue;
            const R dp = m6c<R>::z(k, 0) * step[0] + m6c<R>::z(k, 1) * step[1] + m6c<R>::z(k, 2) * step[2];
            if (dp < R(0)) {
                const R ak = fmax(p[k] - lb, R(0)) / (-dp);
                if (ak < amax) {
                    amax = ak;
                    blk = k;
                }
            }
        }
        // backtracking (Armijo) while far from the optimum; near it the full Newton
        // step converges quadratically and the test would only see rounding noise
        R alpha = amax;
        if (dec > armijo_rel * h0) {
            for (int bt = 0; bt < 40; ++bt) {
                const R tn[3] = {t[0] + alpha * step[0], t[1] + alpha * step[1], t[2] + alpha * step[2]};
                R pn[6];
                p_of_t(pbar, tn, pn);
                if (kurt6(pn) <= h0 - R(0.25) * alpha * dec) break;
                alpha *= R(0.5);
            }
        }
#pragma unroll
        for (int l = 0; l < 3; ++l) t[l] += alpha * step[l];
        if (blk >= 0 && alpha == amax && nw < 3) {
            wmask |= 1 << blk;
            ++nw;
        }
    }
}

// ---- the last Newton steps of the map in double-float ----
__device__ __forceinline__ dflt df_of_double(double v) {
    const float hi = (float)v;
    return {hi, (float)(v - (double)hi)};
}
__device__ __forceinline__ double double_of_df(dflt a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dflt df_scale(dflt a, float c) {  // c a power of two or a small integer
    return df_norm(a.hi * c, fmaf(a.hi, c, -(a.hi * c)) + a.lo * c);
}
// the constants cos 2 theta_k, sin 2 theta_k and z_kl as double-float: 0, +-1/2, +-1 are exact,
// sqrt(3)/2 is split into its nearest float and the rest (folded at compile time once the
// loops over k are unrolled)
constexpr float M6_R3H = 0.8660253882408142f, M6_R3L = 1.5543625053737742e-08f;
__device__ __forceinline__ constexpr int m6_c2n(int k) { return k == 0 ? 2 : k == 1 ? 1 : k == 2 ? -1 : k == 3 ? -2 : k == 4 ? -1 : 1; }
__device__ __forceinline__ constexpr int m6_s2n(int k) { return (k == 1 || k == 2) ? 1 : (k == 4 || k == 5) ? -1 : 0; }
__device__ __forceinline__ dflt m6_dc2(int k) { return {0.5f * (float)m6_c2n(k), 0.f}; }
__device__ __forceinline__ dflt m6_ds2(int k) { return {(float)m6_s2n(k) * M6_R3H, (float)m6_s2n(k) * M6_R3L}; }
// z_k = (cos 4 theta_k, sin 4 theta_k, (-1)^k)
__device__ __forceinline__ dflt m6_dz(int k, int l) {
    if (l == 0) return {(k == 0 || k == 3) ? 1.f : -0.5f, 0.f};
    if (l == 1) {
        const float sg = (k == 1 || k == 4) ? 1.f : (k == 2 || k == 5) ? -1.f : 0.f;
        return {sg * M6_R3H, sg * M6_R3L};
    }
    return {(k & 1) ? -1.f : 1.f, 0.f};
}

// Newton steps on the face of the working set found by the FP32 iteration, with the
// gradient, the iterate t and p = pbar + Z t in double-float (about 48 bits) and the
// reduced Hessian in FP32: each step then removes the error of t down to the
// gradient's accuracy (an FP32 Hessian only slows the convergence to a factor of
// about 1e-7 per step).  Three steps from the FP32 solution reach the rounding level
// of the double-float gradient.  Returns p in double.
__device__ __forceinline__ void map6_polish(const double pbar_d[6], double lb, const double t_d[3], int wmask, int nw,
                            double p_out[6]) {
    dflt pbar[6], t[3];
#pragma unroll
    for (int k = 0; k < 6; ++k) pbar[k] = df_of_double(pbar_d[k]);
#pragma unroll
    for (int l = 0; l < 3; ++l) t[l] = df_of_double(t_d[l]);
    // the free directions of the face (FP32, orthonormal): the same construction as the
    // FP32 iteration
    float za[3] = {0, 0, 0}, zb[3] = {0, 0, 0};
    int seen = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k)
        if ((wmask >> k) & 1) {
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                if (seen == 0) za[l] = MAP6_ZF[k][l];
                if (seen == 1) zb[l] = MAP6_ZF[k][l];
            }
            ++seen;
        }
    const int d = 3 - nw;
    float N[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    if (nw == 1) {
        const float zn = sqrtf(za[0] * za[0] + za[1] * za[1] + za[2] * za[2]);
        const float n1[3] = {za[0] / zn, za[1] / zn, za[2] / zn};
        const int e = (fabsf(n1[1]) < fabsf(n1[0])) ? ((fabsf(n1[2]) < fabsf(n1[1])) ? 2 : 1)
                                                     : ((fabsf(n1[2]) < fabsf(n1[0])) ? 2 : 0);
        const float dd = e == 0 ? n1[0] : (e == 1 ? n1[1] : n1[2]);
        float u[3];
#pragma unroll
        for (int l = 0; l < 3; ++l) u[l] = (l == e ? 1.f : 0.f) - dd * n1[l];
        const float un = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
        for (int l = 0; l < 3; ++l) u[l] /= un;
        const float v[3] = {n1[1] * u[2] - n1[2] * u[1], n1[2] * u[0] - n1[0] * u[2], n1[0] * u[1] - n1[1] * u[0]};
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            N[l][0] = u[l];
            N[l][1] = v[l];
        }
    } else if (nw == 2) {
        const float n[3] = {za[1] * zb[2] - za[2] * zb[1], za[2] * zb[0] - za[0] * zb[2], za[0] * zb[1] - za[1] * zb[0]};
        const float nn = sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
#pragma unroll
        for (int l = 0; l < 3; ++l) N[l][0] = n[l] / nn;
    }
    dflt p[6];
    for (int it = 0; it < 3 && d > 0; ++it) {
#pragma unroll
        for (int k = 0; k < 6; ++k)
            p[k] = df_fma(m6_dz(k, 2), t[2], df_fma(m6_dz(k, 1), t[1], df_fma(m6_dz(k, 0), t[0], pbar[k])));
        // gradient of ||K||^2 = (S0^2 + Sr^2 + Si^2)/2 in t, S = sum q_k (1, c2_k, s2_k), q = p^2
        dflt q[6], s0 = {0.f, 0.f}, sr = {0.f, 0.f}, si = {0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            q[k] = df_mul(p[k], p[k]);
            s0 = df_add(s0, q[k]);
            sr = df_fma(m6_dc2(k), q[k], sr);
            si = df_fma(m6_ds2(k), q[k], si);
        }
        dflt g[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            // dK/dp_k = 4 p_k (s0 + c2_k sr + s2_k si) / 2
            const dflt dq = df_fma(m6_ds2(k), si, df_fma(m6_dc2(k), sr, s0));
            const dflt gp = df_scale(df_mul(p[k], dq), 2.f);
#pragma unroll
            for (int l = 0; l < 3; ++l) g[l] = df_fma(m6_dz(k, l), gp, g[l]);
        }
        // reduced gradient (double-float) and Hessian (FP32) on the face
        dflt gr[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        float Hr[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, grf[3] = {0, 0, 0}, du[3] = {0, 0, 0};
        float pf[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) pf[k] = p[k].hi;
        float Hm[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        {
            float f0 = 0, fr = 0, fi = 0;
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const float qq = pf[k] * pf[k];
                f0 += qq;
                fr += qq * MAP6_C2F[k];
                fi += qq * MAP6_S2F[k];
            }
            float sg[3] = {0, 0, 0}, mr[3] = {0, 0, 0}, mi[3] = {0, 0, 0};
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const float dq = 0.5f * (f0 + MAP6_C2F[k] * fr + MAP6_S2F[k] * fi);
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    const float z = MAP6_ZF[k][l];
                    sg[l] += pf[k] * z;
                    mr[l] += MAP6_C2F[k] * pf[k] * z;
                    mi[l] += MAP6_S2F[k] * pf[k] * z;
#pragma unroll
                    for (int m = 0; m <= l; ++m) Hm[l][m] += 4.f * dq * z * MAP6_ZF[k][m];
                }
            }
#pragma unroll
            for (int l = 0; l < 3; ++l)
#pragma unroll
                for (int m = 0; m <= l; ++m) {
                    Hm[l][m] += 4.f * (sg[l] * sg[m] + mr[l] * mr[m] + mi[l] * mi[m]);
                    Hm[m][l] = Hm[l][m];
                }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (a >= d) continue;
#pragma unroll
            for (int l = 0; l < 3; ++l) gr[a] = df_fma(dflt{-N[l][a], 0.f}, g[l], gr[a]);
            grf[a] = gr[a].hi + gr[a].lo;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (b >= d) continue;
                float sab = 0;
#pragma unroll
                for (int l = 0; l < 3; ++l)
#pragma unroll
                    for (int m = 0; m < 3; ++m) sab += N[l][a] * Hm[l][m] * N[m][b];
                Hr[a][b] = sab;
            }
        }
        if (!spd_solve(d, Hr, grf, du)) break;
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const float st = N[l][0] * du[0] + (d > 1 ? N[l][1] * du[1] : 0.f) + (d > 2 ? N[l][2] * du[2] : 0.f);
            t[l] = df_add(t[l], dflt{st, 0.f});
        }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        p[k] = df_fma(m6_dz(k, 2), t[2], df_fma(m6_dz(k, 1), t[1], df_fma(m6_dz(k, 0), t[0], pbar[k])));
        p_out[k] = double_of_df(p[k]);
    }
}

struct map6_p {
    double p[6];
    bool ok;
};

// minimise ||K||^2 over p = pbar + Z t with p >= lb: primal active set.  The
// start is a strictly feasible point built from the hexagon geometry of the
// covariance (the traceless part, normalised, is a convex combination of the
// centre and two neighbouring vertices exp(2 i theta_k)); the working set is a
// bit mask of the bounds held at lb.  Returns ok = false when no p >= lb
// reproduces the covariance.  (The result is returned by value: the scales
// must not travel through a pointer to the caller's local array, which the
// device build did not write back reliably.)
__device__ __forceinline__ map6_p map6_active_set(double T, double Zc, double Zs, double lb) {
    const double PI3 = 1.04719755119659774615;
    map6_p res;
    res.ok = true;
    double* p = res.p;
    double pbar[6];
    // (divisions by constants as multiplications: an FP64 division costs a dozen FP64 operations on
    // GB300's FP64 pipe, which the map is bound by; the results move by an ulp at most)
    constexpr double I3 = 1.0 / 3.0, I6 = 1.0 / 6.0;
#pragma unroll
    for (int k = 0; k < 6; ++k) pbar[k] = (T + 2.0 * (Zc * MAP6_C2[k] + Zs * MAP6_S2[k])) * I6;
    const double den = T - 6.0 * lb;
    if (!(den > 0.0)) {
        res.ok = false;
        return res;
    }
    const double iden = 1.0 / den;
    const double zr = Zc * iden, zi = Zs * iden;
    // the sector [k pi/3, (k+1) pi/3) holding the angle of (zr, zi): the one whose bisector
    // k pi/3 + pi/6 (30, 90, 150, 210, 270, 330 degrees) has the largest projection
    int ka = 0;
    {
        const double R3 = 0.86602540378443864676;
        const double d0 = R3 * zr + 0.5 * zi, d1 = zi, d2 = -R3 * zr + 0.5 * zi;
        const double pr[6] = {d0, d1, d2, -d0, -d1, -d2};
        double best = pr[0];
#pragma unroll
        for (int k = 1; k < 6; ++k)
            if (pr[k] > best) {
                best = pr[k];
                ka = k;
            }
    }
    (void)PI3;
    const int kb = (ka + 1) % 6;
    const double dt = MAP6_C2[ka] * MAP6_S2[kb] - MAP6_S2[ka] * MAP6_C2[kb];
    const double idt = 1.0 / dt;
    const double la = (zr * MAP6_S2[kb] - zi * MAP6_C2[kb]) * idt;
    const double lbb = (MAP6_C2[ka] * zi - MAP6_S2[ka] * zr) * idt;
    double l0 = 1.0 - la - lbb;
    if (l0 < -1e-12) {
        res.ok = false;
        return res;
    }
    l0 = fmax(l0, 0.0);
    double t[3] = {0.0, 0.0, 0.0};
    const double tiny = 1e-13 * T;
    int wmask = 0, nw = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double ps = lb + den * (l0 * I6 + (k == ka ? la : 0.0) + (k == kb ? lbb : 0.0));
        const double dps = ps - pbar[k];
        t[0] += MAP6_Z[k][0] * dps * I3;
        t[1] += MAP6_Z[k][1] * dps * I3;
        t[2] += MAP6_Z[k][2] * dps * I6;
        if (ps <= lb + tiny) {
            wmask |= 1 << k;
            ++nw;
        }
    }
    if (nw > 3) {  // the covariance is at a vertex of the feasible set: the only point
        p_of_t(pbar, t, p);
#pragma unroll
        for (int k = 0; k < 6; ++k) p[k] = fmax(p[k], lb);
        return res;
    }
    // single precision first, to about the rounding level of FP32; then the
    // same iteration in FP64 from there (typically one or two steps and the
    // multiplier check), so the result is the FP64 optimum
    float pbf[6], tf[3];
#pragma unroll
    for (int k = 0; k < 6; ++k) pbf[k] = (float)pbar[k];
#pragma unroll
    for (int l = 0; l < 3; ++l) tf[l] = (float)t[l];
    map6_newton<float>(pbf, (float)lb, (float)T, tf, wmask, nw, 30, 1e-5f, 1e-4f, 1e-5f);
#pragma unroll
    for (int l = 0; l < 3; ++l) t[l] = (double)tf[l];
    if (nw > 0) {  // onto the face of the working set exactly: p_k = lb for its bounds (least-norm change of t)
        double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, rhs[3] = {0, 0, 0}, mu[3] = {0, 0, 0};
        int idx[3] = {0, 0, 0}, a = 0;
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if ((wmask >> k) & 1) {
                idx[0] = a == 0 ? k : idx[0];
                idx[1] = a == 1 ? k : idx[1];
                idx[2] = a == 2 ? k : idx[2];
                ++a;
            }
        double pc[6];
        p_of_t(pbar, t, pc);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (i >= nw) break;
            double pci = pc[0];
#pragma unroll
            for (int k = 1; k < 6; ++k) pci = idx[i] == k ? pc[k] : pci;
            rhs[i] = lb - pci;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if (j >= nw) break;
                G[i][j] = MAP6_Z[idx[i]][0] * MAP6_Z[idx[j]][0] + MAP6_Z[idx[i]][1] * MAP6_Z[idx[j]][1] +
                          MAP6_Z[idx[i]][2] * MAP6_Z[idx[j]][2];
            }
        }
        if (spd_solve(nw, G, rhs, mu))
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (i >= nw) break;
#pragma unroll
                for (int l = 0; l < 3; ++l) t[l] += mu[i] * MAP6_Z[idx[i]][l];
            }
    }
    map6_polish(pbar, lb, t, wmask, nw, p);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        if ((wmask >> k) & 1) p[k] = lb;
        p[k] = fmax(p[k], lb);
    }
    return res;
}

struct map6_result {
    double a[6];
    int flag;
};

// rel (default 1e-3): the bound p_k >= rel T keeps the smallest width at least
// 0.077 times the typical one; the stencil's rounded (double-float) part loses
// accuracy like the square of that ratio for each width at the bound
// covariance (kind COV) or (sigma, rho, theta) (kind SRT) -> six scales; the
// flags and the elongation clamp follow the four-directional map
__device__ map6_result map6_solve(int kind, float v0f, float v1f, float v2f, double eps, double eta, double rel) {
    map6_result R;
    R.flag = 0;
    const double v0 = v0f, v1 = v1f, v2 = v2f;
    double lmax, lmin, c2, s2;
    if (kind == BSF_PARAM_SRT) {
        lmax = v0 * v0;
        lmin = lmax / v1;
        // 2 theta reduced by pi/2 inside the series routine (exact enough for |2 theta| < 64; larger
        // angles are taken modulo 2 pi first)
        const double x2 = 2.0 * v2;
        map4_sincos64(fabs(x2) < 64.0 ? x2 : fmod(x2, 6.283185307179586476925), s2, c2);
        if (!(v2 == v2) || fabs(v2) > 1e30) c2 = s2 = BSF_QNAN64;
    } else {
        const double D = sqrt((v0 - v2) * (v0 - v2) + 4.0 * v1 * v1);
        lmax = 0.5 * (v0 + v2 + D);
        lmin = (v0 * v2 - v1 * v1) / lmax;
        const double iD = D > 0.0 ? 1.0 / D : 0.0;
        c2 = D > 0.0 ? (v0 - v2) * iD : 1.0;
        s2 = D > 0.0 ? 2.0 * v1 * iD : 0.0;
    }
    if (!(isfinite(lmax) && isfinite(lmin) && isfinite(c2) && isfinite(s2)) || !(lmin > 0.0) || !(lmax >= lmin)) {
        for (int k = 0; k < 6; ++k) R.a[k] = BSF_QNAN64;
        R.flag = 4;
        return R;
    }
    // elongation bound for six directions: the normalised traceless part lies in
    // the regular hexagon with vertices exp(2 i theta_k), scaled by 1 - 6 delta so
    // that every p_k can keep the share delta = 1e-3 of the trace
    // cos(psi - pi/6), psi = 2 theta mod pi/3: the largest |projection| of (cos 2 theta,
    // sin 2 theta) on the directions 30, 90, 150 degrees (the bisectors of the sectors)
    const double R3 = 0.86602540378443864676;
    const double cpsi = fmax(fabs(R3 * c2 + 0.5 * s2), fmax(fabs(s2), fabs(0.5 * s2 - R3 * c2)));
    const double r = (1.0 - 6.0 * rel) * R3 / cpsi;
    bool clamp = false;
    {
        const double U = (1.0 + r) / (1.0 - r);
        const double rc = (1.0 - eta) * U;
        if (lmax / lmin > rc) {
            const double s = lmax + lmin;
            lmin = s / (1.0 + rc);
            lmax = s - lmin;
            clamp = true;
            R.flag |= 1;
        }
    }
    double T, Zc, Zs;
    if (kind == BSF_PARAM_COV && !clamp) {
        T = 12.0 * (v0 + v2);
        Zc = 12.0 * (v0 - v2);
        Zs = 24.0 * v1;
    } else {
        const double m = 0.5 * (lmax + lmin), d = 0.5 * (lmax - lmin);
        T = 24.0 * m;
        Zc = 24.0 * d * c2;
        Zs = 24.0 * d * s2;
    }
    // lower bound of p: eps, or the share rel of the trace T = sum p
    const double bound = fmax(eps, rel * T);
    map6_p P = map6_active_set(T, Zc, Zs, bound);
    if (!P.ok) {
        R.flag |= 2;
        P = map6_active_set(T, Zc, Zs, 0.0);
        if (!P.ok) {
            for (int k = 0; k < 6; ++k) R.a[k] = BSF_QNAN64;
            R.flag = 4;
            return R;
        }
        for (int k = 0; k < 6; ++k) P.p[k] = fmax(P.p[k], bound);
    }
    // a_k = sqrt(p_k): the FP32 root and one Newton step in FP64 (about 48 correct bits)
    for (int k = 0; k < 6; ++k) {
        const double pk = fmax(P.p[k], 0.0);
        const float r0 = sqrtf((float)pk);
        R.a[k] = r0 > 0.f ? (double)r0 + fma(-(double)r0, (double)r0, pk) * (double)(0.5f / r0) : 0.0;
    }
    return R;
}

__device__ __forceinline__ double cos_k(int k) {
    const double t[6] = {1.0, 0.86602540378443864676, 0.5, 0.0, -0.5, -0.86602540378443864676};
    return t[k];
}
__device__ __forceinline__ double sin_k(int k) {
    const double t[6] = {0.0, 0.5, 0.86602540378443864676, 1.0, 0.86602540378443864676, 0.5};
    return t[k];
}

// ---- the map as a table (optional fast mode, opts.map_lut) ----
// With the relative bound (R19) the problem is homogeneous: p(s C) = s p(C)
// (the paper's observation (O1), Sec. 3.2.2), so p / T depends only on the
// normalised traceless part z = (Zc, Zs) / T = e (cos 2 theta, sin 2 theta),
// e = (rho - 1) / (rho + 1).  The six directions are invariant under a rotation
// by pi/6 that shifts their indices (the six-directional form of (O2)), so
// p_k(2 theta) = p_{k-r}(2 theta - r pi/3).  The table holds p / T on a polar
// grid of that sector: 2 theta' in [0, pi/3] and u = e / e_c(theta') in [0, 1],
// e_c the elongation clamp, so that clamped pixels lie on the grid's last line.
// A lookup interpolates bilinearly, rotates, scales by T and then projects onto
// the covariance constraint (the least-norm change of p that restores
// sum p = T, sum p cos 2 theta_k = Zc, sum p sin 2 theta_k = Zs), so every
// table kernel keeps its target covariance; the interpolation touches only the
// kurtosis optimum.  Pixels the table cannot serve (eps binds, invalid input)
// take the exact solver.
constexpr int LUT6_NU = 512;  // cells along u = e / e_c
constexpr int LUT6_NP = 512;  // cells along 2 theta' in [0, pi/3]

// e_c: the largest e the clamp of map6_solve keeps at the orientation (c2, s2) = (cos, sin) 2 theta
template <typename T>
__device__ __forceinline__ T map6_ecap(T c2, T s2, T eta, T rel) {
    const T R3 = (T)0.86602540378443864676;
    const T cpsi = fmax(fabs(R3 * c2 + (T)0.5 * s2), fmax(fabs(s2), fabs((T)0.5 * s2 - R3 * c2)));
    const T r = ((T)1 - (T)6 * rel) * R3 / cpsi;
    const T rc = ((T)1 - eta) * ((T)1 + r) / ((T)1 - r);
    return (rc - (T)1) / (rc + (T)1);
}

__global__ void k_lut6_build(double eta, double rel, float* __restrict__ table) {
    const int n = (LUT6_NU + 1) * (LUT6_NP + 1);
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const int i = id / (LUT6_NP + 1), j = id % (LUT6_NP + 1);
    double s2, c2;
    sincos((double)j / LUT6_NP * 1.04719755119659774615, &s2, &c2);
    const double e = (double)i / LUT6_NU * map6_ecap(c2, s2, eta, rel);
    map6_p P = map6_active_set(1.0, e * c2, e * s2, rel);
    if (!P.ok) {
        P = map6_active_set(1.0, e * c2, e * s2, 0.0);
        for (int k = 0; k < 6; ++k) P.p[k] = fmax(P.p[k], rel);
    }
    float* t = table + (size_t)id * 8;
#pragma unroll
    for (int k = 0; k < 6; ++k) t[k] = (float)P.p[k];
    t[6] = t[7] = 0.f;
}

// the table's scales for one pixel; false when the exact solver must run
__device__ bool lut6_lookup(const float* __restrict__ table, int kind, float v0, float v1, float v2, double eps,
                            double eta, double rel, double a[6], int& flag) {
    // validity as the exact solver decides it (eigenvalues in FP64: the determinant of an
    // elongated covariance cancels); the rest in FP32
    double dmax, dmin;
    float T, Zc, Zs;
    if (kind == BSF_PARAM_SRT) {
        dmax = (double)v0 * (double)v0;
        dmin = dmax / (double)v1;
        if (!(fabsf(v2) < 64.f)) return false;
        float sn, cs;
        sincosf(2.f * v2, &sn, &cs);
        const float d = (float)(12.0 * (dmax - dmin));
        T = (float)(12.0 * (dmax + dmin));
        Zc = d * cs;
        Zs = d * sn;
    } else {
        const double a0 = v0, a1 = v1, a2 = v2;
        dmax = 0.5 * (a0 + a2 + sqrt((a0 - a2) * (a0 - a2) + 4.0 * a1 * a1));
        dmin = (a0 * a2 - a1 * a1) / dmax;
        T = 12.f * (v0 + v2);
        Zc = 12.f * (v0 - v2);
        Zs = 24.f * v1;
    }
    if (!(isfinite(dmax) && isfinite(dmin)) || !(dmin > 0.0) || !(dmax >= dmin) || rel <= 0.0) return false;
    if (rel * 12.0 * (dmax + dmin) < eps) return false;  // eps binds: not homogeneous
    const float zn = sqrtf(Zc * Zc + Zs * Zs);
    const float c2 = zn > 0.f ? Zc / zn : 1.f, s2 = zn > 0.f ? Zs / zn : 0.f;
    const float ec = map6_ecap(c2, s2, (float)eta, (float)rel);
    float e = zn / T;
    flag = 0;
    if (e > ec) {
        Zc *= ec / e;
        Zs *= ec / e;
        e = ec;
        flag = 1;
    }
    const float SEC = 1.04719755119659774615f;
    float phi = atan2f(s2, c2);
    if (phi < 0.f) phi += 6.28318530717958648f;
    int r = (int)(phi / SEC);
    r = r < 0 ? 0 : (r > 5 ? 5 : r);
    const float php = fminf(fmaxf(phi - (float)r * SEC, 0.f), SEC);
    const float u = fminf(e / ec, 1.f) * LUT6_NU, w = php / SEC * LUT6_NP;
    const int iu = min((int)u, LUT6_NU - 1), iw = min((int)w, LUT6_NP - 1);
    const float fu = u - (float)iu, fw = w - (float)iw;
    const float4* t00 = reinterpret_cast<const float4*>(table + ((size_t)iu * (LUT6_NP + 1) + iw) * 8);
    const float4* t01 = t00 + 2;
    const float4* t10 = t00 + 2 * (LUT6_NP + 1);
    const float4* t11 = t10 + 2;
    float v[6];
    {
        const float4 a0 = t00[0], a1 = t00[1], b0 = t01[0], b1 = t01[1];
        const float4 c0 = t10[0], c1 = t10[1], d0 = t11[0], d1 = t11[1];
        const float w00 = (1.f - fu) * (1.f - fw), w01 = (1.f - fu) * fw, w10 = fu * (1.f - fw), w11 = fu * fw;
        v[0] = w00 * a0.x + w01 * b0.x + w10 * c0.x + w11 * d0.x;
        v[1] = w00 * a0.y + w01 * b0.y + w10 * c0.y + w11 * d0.y;
        v[2] = w00 * a0.z + w01 * b0.z + w10 * c0.z + w11 * d0.z;
        v[3] = w00 * a0.w + w01 * b0.w + w10 * c0.w + w11 * d0.w;
        v[4] = w00 * a1.x + w01 * b1.x + w10 * c1.x + w11 * d1.x;
        v[5] = w00 * a1.y + w01 * b1.y + w10 * c1.y + w11 * d1.y;
    }
    float p[6], sT = 0.f, sC = 0.f, sS = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int src = (k - r + 6) % 6;
        float vk = v[0];
#pragma unroll
        for (int m = 1; m < 6; ++m) vk = (src == m) ? v[m] : vk;
        p[k] = T * vk;
        sT += p[k];
        sC += p[k] * MAP6_C2F[k];
        sS += p[k] * MAP6_S2F[k];
    }
    const float dT = T - sT, dC = Zc - sC, dS = Zs - sS, lb = (float)rel * T;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float pk = fmaxf(p[k] + (dT + 2.f * (dC * MAP6_C2F[k] + dS * MAP6_S2F[k])) * (1.f / 6.f), lb);
        a[k] = (double)sqrtf(pk);
    }
    return true;
}

// per pixel: scales (FP64, six planes per batch entry) and the largest
// footprint half-extents of each tile
__global__ void k_map6(const float* __restrict__ params, int kind, long long HW, int B, int W, int tile, int tiles_x,
                       int ntile, double eps, double eta, double rel, double ascale, double* __restrict__ scales,
                       unsigned* __restrict__ tile_ext, unsigned* __restrict__ status,
                       const float* __restrict__ lut) {
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid >= HW * B) return;
    const long long b = gid / HW, p = gid - b * HW;
    const int x = (int)(p % W), y = (int)(p / W);
    double a[6];
    int flag = 0;
    if (kind == BSF_PARAM_SCALES) {
        for (int k = 0; k < 6; ++k) {
            const double v = (double)params[(b * 6 + k) * HW + p] * ascale;
            a[k] = v;
            if (!(v > 0.0) || !isfinite(v)) flag = 4;
        }
        if (flag) raise_status(status, BSF_EBADSCALE);
    } else {
        const float* q = params + b * 3 * HW + p;
        if (lut != nullptr && lut6_lookup(lut, kind, q[0], q[HW], q[2 * HW], eps, eta, rel, a, flag)) {
            for (int k = 0; k < 6; ++k) a[k] *= ascale;
        } else {
            const map6_result R = map6_solve(kind, q[0], q[HW], q[2 * HW], eps, eta, rel);
            for (int k = 0; k < 6; ++k) a[k] = R.a[k] * ascale;
            flag = R.flag;
        }
        if (flag & 1) raise_status(status, BSF_EINFEASIBLE);
        if (flag & 4) raise_status(status, BSF_EBADSCALE);
    }
    for (int k = 0; k < 6; ++k) scales[(b * 6 + k) * HW + p] = flag & 4 ? BSF_QNAN64 : a[k];
    if (flag & 4) return;
    double ex = 0.0, ey = 0.0;
    for (int k = 0; k < 6; ++k) {
        ex += a[k] * fabs(cos_k(k));
        ey += a[k] * sin_k(k);
    }
    const float fx = (float)(0.5 * ex) * 1.0001f + 1e-3f, fy = (float)(0.5 * ey) * 1.0001f + 1e-3f;
    unsigned* te = tile_ext + ((size_t)b * ntile + (size_t)(y / tile) * tiles_x + (x / tile)) * 2;
    atomicMax(te, __float_as_uint(fx));
    atomicMax(te + 1, __float_as_uint(fy));
}

// the scales of bsf_scales_from_cov for N = 6 (float32, six planes, flags)
__global__ void k_map6_out(const float* __restrict__ params, int kind, long long npix, double eps, double eta,
                           double rel, float* __restrict__ scales, uint8_t* __restrict__ flags,
                           const float* __restrict__ lut) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= npix) return;
    double a[6];
    int flag = 0;
    if (lut == nullptr ||
        !lut6_lookup(lut, kind, params[p], params[npix + p], params[2 * npix + p], eps, eta, rel, a, flag)) {
        const map6_result R = map6_solve(kind, params[p], params[npix + p], params[2 * npix + p], eps, eta, rel);
        for (int k = 0; k < 6; ++k) a[k] = R.a[k];
        flag = R.flag;
    }
    for (int k = 0; k < 6; ++k) scales[k * npix + p] = (float)a[k];
    if (flags) flags[p] = (uint8_t)flag;
}

constexpr int PRE_THREADS = HEX6_PRE_THREADS;
constexpr int PRE_CPT = HEX6_PRE_CPT;  // window columns per thread
constexpr int MU_FRAC_BITS = 24;  // fixed point of the transferred masses

// step 2 on one window: transfer of the image and the six running sums, row by
// row.  The sums are exact: the masses are rounded once to fixed point with
// 24 fractional bits (a change of the measure of at most 2^-25 per lattice
// point) and summed in 128-bit integers (the largest windows need about 2^83),
// and the windows hold them exactly, times 2^24, as 128-bit integers.  The
// state of each sum (its last
// row, two for the 90-degree sum) is kept per column: in shared memory for
// the four sums whose rows shift by one to three columns (the neighbouring
// threads read them), in registers for the two that do not shift.
// Shared-memory index of window column c: one padding element after every
// eight columns, so that the lanes of a warp, which own columns PRE_CPT = 4
// apart, spread a 16-byte state access over all banks (each quarter-warp
// touches eight distinct 16-byte bank groups; without the padding, eight lanes
// share two of them).  Four columns per thread rather than eight halve the
// registers of the per-column states and double the warps per window: on the
// batch's largest windows one CTA per SM then holds 26 warps instead of 13.
__device__ __forceinline__ int pidx(int c) { return c + c / HEX6_PRE_PAD; }

// The stencil reads the window values as three 32-bit limbs of g + 2^95, so
// every value must lie in [-2^95, 2^95).  The kernel checks that and that no
// running sum can have wrapped around 128 bits (each partial sum is at most
// the largest |mass| times the product of the six line lengths in the
// window), and sets the window's flag otherwise (image values too large for
// the exact form; the stencil then writes NaN and raises BSF_ERANGE).
template <class InT>
__global__ void __launch_bounds__(PRE_THREADS) k_hex6_preint(const InT* __restrict__ img, int C, int H, int W,
                                                             double h, const hex6_tile* __restrict__ tiles,
                                                             u128* __restrict__ scratch, unsigned* __restrict__ wflag,
                                                             int reflect) {
    extern __shared__ u128 smq[];
    const hex6_tile tl = tiles[blockIdx.x];
    const int c = blockIdx.y;
    const int ncol = tl.ncol, nrow = tl.nrow;
    const int np = pidx(ncol) + 1;
    u128* s30 = smq;
    u128* s60 = s30 + np;
    u128* s90b = s60 + np;
    u128* s120 = s90b + np;
    u128* wt = s120 + np;  // warp totals
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x, nwarp = nthr >> 5;  // a multiple of 32, at most PRE_THREADS
    for (int k = tid; k < 4 * np; k += nthr) smq[k] = 0;
    const InT* f = img + ((size_t)tl.b * C + c) * (size_t)H * W;
    u128* G = scratch + tl.off + (long long)c * ncol * nrow;
    // The transfer weights need only single precision: an error in a mass is a
    // small change of the input measure, which the exact sums carry through
    // without amplification.  With h a power of two the lattice x-coordinates
    // h (i + j/2) are exact in FP32; the y-offset of a row is rounded once.
    const float hf = (float)h, ih = 1.0f / hf;
    const float rs3 = 0.57735026918962576451f;  // 1/sqrt3
    const double hy = h * 0.86602540378443864676;
    const float qscale = (float)(1 << MU_FRAC_BITS);
    const int c0 = tid * PRE_CPT;
    u128 s90a[PRE_CPT], s150[PRE_CPT], y[PRE_CPT];
#pragma unroll
    for (int e = 0; e < PRE_CPT; ++e) s90a[e] = s150[e] = 0;
    unsigned qbits = 0, big = 0;  // largest |mass| (FP32 bits; NaN above all); OR of |stored value| >> 95
    // the pixel row below each lattice row and the offset to it, in FP64 (the lattice row height
    // h sqrt3/2 is irrational): computed once per block by one thread, for row r + 1 while row r
    // runs (GB300's FP64 pipe takes about 64 cycles per warp instruction)
    __shared__ int row_ky0;
    __shared__ float row_dy0;
    auto row_pos = [&](int r) {
        const double pyd = hy * (double)(tl.j0w + r);
        const double kyd = floor(pyd);
        row_ky0 = (int)kyd;
        row_dy0 = (float)(kyd - pyd);  // (pixel row ky0) - (lattice row), in (-1, 0]
    };
    if (tid == 0) row_pos(0);
    __syncthreads();
    for (int r = 0; r < nrow; ++r) {
        const int j = tl.j0w + r;
        const int ky0 = row_ky0;
        const float dy0 = row_dy0;
        // the image row the lattice rows two to three ahead first need (their columns lie about
        // 1.5 h px per row further left), fetched into L1 now: one line per thread, no registers
        if (c0 < ncol) {
            const int kyp = ky0 + 2;
            const int kxp = (int)floorf(hf * ((float)(c0 + tl.i_left - 2 * r) + 0.5f * (float)j)) - 2;
            if (kyp >= 0 && kyp < H && kxp < W)
                asm volatile("prefetch.global.L1 [%0];" ::"l"(f + (size_t)kyp * W + (kxp > 0 ? kxp : 0)));
        }
        u128 run = 0;
#pragma unroll
        for (int e = 0; e < PRE_CPT; ++e) {
            const int cc = c0 + e;
            float mu = 0.f;
            if (cc < ncol) {
                const int i = cc + tl.i_left - 2 * r;
                const float px = hf * ((float)i + 0.5f * (float)j);
                const float kxf = floorf(px);
                const int kx0 = (int)kxf;
                const float dx0 = kxf - px;
#pragma unroll
                for (int dy = 0; dy < 2; ++dy) {
                    int ky = ky0 + dy;
                    if (reflect)
                        ky = reflect_index(ky, H);  // the image's half-sample symmetric extension
                    else if (ky < 0 || ky >= H)
                        continue;
                    const float ddy = (dy0 + (float)dy) * ih;
                    const float dt = 2.f * rs3 * ddy;
#pragma unroll
                    for (int dx = 0; dx < 2; ++dx) {
                        int kx = kx0 + dx;
                        if (reflect)
                            kx = reflect_index(kx, W);
                        else if (kx < 0 || kx >= W)
                            continue;
                        // lattice coordinates of pixel - lattice point; weight = the hat of the point
                        const float ds = (dx0 + (float)dx) * ih - rs3 * ddy;
                        const float w = 1.f - fmaxf(fabsf(ds), fmaxf(fabsf(dt), fabsf(ds + dt)));
                        if (w > 0.f) mu = fmaf(w, (float)f[(size_t)ky * W + kx], mu);
                    }
                }
            }
            run += (u128)(i128)f32_to_i64_rn(mu * qscale);  // saturates: at most 2^63 in magnitude
            qbits = max(qbits, __float_as_uint(fabsf(mu)));
            y[e] = run;
        }
        // block-wide scan of the thread totals (the 0-degree sum along the row)
        u128 v = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u128 u = shfl_up_T(v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) wt[warp] = v;
        __syncthreads();
        // every thread has read this row's position: the next row's can be written (read after
        // the row's last barrier)
        if (tid == 0 && r + 1 < nrow) row_pos(r + 1);
        // every warp scans the warp totals itself (no second barrier)
        u128 wsum = lane < nwarp ? wt[lane] : (u128)0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u128 u = shfl_up_T(wsum, o);
            if (lane >= o) wsum += u;
        }
        const u128 wprev = shfl_idx_T(wsum, warp > 0 ? warp - 1 : 0);
        const u128 off = (v - run) + (warp > 0 ? wprev : (u128)0);
        // the other five sums, one after the other: a sum whose row shifts reads
        // its neighbours' previous row, then (after a barrier) stores its own row
#pragma unroll
        for (int e = 0; e < PRE_CPT; ++e) {
            const int cc = c0 + e;
            y[e] += off;
            if (cc < ncol && cc >= 3) y[e] += s30[pidx(cc - 3)];
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < PRE_CPT; ++e) {
            const int cc = c0 + e;
            if (cc >= ncol) continue;
            s30[pidx(cc)] = y[e];
            if (cc >= 2) y[e] += s60[pidx(cc - 2)];
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < PRE_CPT; ++e) {
            const int cc = c0 + e;
            if (cc >= ncol) continue;
            s60[pidx(cc)] = y[e];
            if (cc >= 3) y[e] += s90b[pidx(cc - 3)];
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < PRE_CPT; ++e) {
            const int cc = c0 + e;
            if (cc >= ncol) continue;
            s90b[pidx(cc)] = s90a[e];  // the row before, for the row after next
            s90a[e] = y[e];
            if (cc >= 1) y[e] += s120[pidx(cc - 1)];
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < PRE_CPT; ++e) {
            const int cc = c0 + e;
            if (cc >= ncol) continue;
            s120[pidx(cc)] = y[e];
            y[e] += s150[e];
            s150[e] = y[e];
            G[(long long)r * ncol + cc] = y[e];  // exact, times 2^24
            const unsigned long long hi = (unsigned long long)(y[e] >> 64);
            big |= (unsigned)((hi ^ (unsigned long long)((long long)hi >> 63)) >> 31);
        }
    }
    // the window's flag: a value outside [-2^95, 2^95), or sums that may have wrapped
    __syncthreads();
    const unsigned wbad = __reduce_or_sync(0xffffffffu, big);
    const unsigned wq = __reduce_max_sync(0xffffffffu, qbits);
    unsigned* red = reinterpret_cast<unsigned*>(wt);
    if (lane == 0) {
        red[warp] = wbad;
        red[32 + warp] = wq;
    }
    __syncthreads();
    if (tid == 0) {
        unsigned bad = 0, qb = 0;
        for (int k = 0; k < nwarp; ++k) {
            bad |= red[k];
            qb = max(qb, red[32 + k]);
        }
        const double n30 = min(nrow - 1, (ncol - 1) / 3) + 1, n60 = min(nrow - 1, (ncol - 1) / 2) + 1;
        const double n90 = min((nrow - 1) / 2, (ncol - 1) / 3) + 1, n120 = min(nrow - 1, ncol - 1) + 1;
        const double bound = ((double)__uint_as_float(qb) * (double)qscale + 1.0) * (double)ncol * n30 * n60 * n90 *
                             n120 * (double)nrow;
        wflag[blockIdx.x * C + c] = (bad || !(bound < 0x1p126)) ? 1u : 0u;
    }
}

constexpr int ST_THREADS = 128;  // 32 x 4 pixels for 64-pixel tiles, 16 x 8 for 16-pixel tiles

// the canonical piece's coefficients C[slot][monomial] (integers, |C| <= 102)
__constant__ int HEX6_CC_CONST[HEX6_NSLOT][HEX6_NMONO] = HEX6_CCOEF_INIT;

// mma.sync m16n8k16 with FP16 operands and FP32 accumulation.  Every operand
// here is a small integer (window bytes as 1024 + byte, coefficients |c| <=
// 102), every product is exact and every partial sum an integer below 2^21,
// so the FP32 result is exact.
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1,
                                         float c0, float c1, float c2, float c3) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%11,%12,%13};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c0), "f"(c1), "f"(c2), "f"(c3));
}
// byte `sel` of two 32-bit words as the FP16 pair (1024 + byte of wa, 1024 + byte of wb)
__device__ __forceinline__ unsigned bytes_as_f16x2(unsigned wa, unsigned wb, unsigned sel) {
    return (__byte_perm(wa, wb, sel) & 0x00FF00FFu) | 0x64006400u;
}

constexpr float TC_MAGIC = 12582912.0f;   // 1.5 * 2^23: FP32 integers in (-2^22, 2^22) sit in its mantissa
constexpr int TC_MAGIC_BITS = 0x4B400000;  // its bit pattern
constexpr int TC_PSTRIDE = 17;             // 128-bit slots per pixel in the coefficient buffer

// step 3: the 64 taps of Eq. FD_mesh, each read from its window by the exact
// piecewise-quartic element (24 lattice points).  Exact where it matters:
//   - tap positions in 48-bit fixed point relative to the pixel's lattice cell
//     (each direction's step a_k u_k rounded once, so the 64 taps form an
//     exact affine mesh for scales perturbed by 2^-48 lattice units); the taps
//     are visited in Gray-code order, one step added or removed per tap;
//   - the twelve pieces of a cell are images of one canonical piece under
//     lattice symmetries that leave the element invariant: a tap of piece r is
//     evaluated at its image x in the canonical piece (exact, 48-bit), reading
//     the window at the piece's slot offsets;
//   - the canonical quartic, F = sum_m A_m x^m / 432, has integer coefficients
//     A_m = sum_k C[k][m] g[m_k] over the piece's 24 window values g, computed
//     exactly on the tensor cores: the values g + 2^95 (96 bits) are cut into
//     twelve bytes, each an exact FP16 number 1024 + byte; one mma.sync per
//     byte and half of the 24 slots multiplies the 16 x 32 coefficient matrix
//     (FP16, exact) by the bytes of eight taps, with FP32 sums that stay exact
//     integers; the twelve byte sums are recombined exactly in 64- and 128-bit
//     integers;
//   - the constant terms A_00, which carry the size of the sums, are added over
//     the 64 taps exactly, in 128-bit integers;
// and only the remaining terms (derivatives of the sums, smaller by the window
// size) are evaluated in double-float arithmetic.  No FP64 in the loop.
//
// Work layout: a warp owns 32 pixels (one per lane) and walks the 64 taps in
// rounds.  In round r (tap q = r / 4) the eight quads of the warp each take one
// tap -- quad n that of pixel 4 n + r % 4 -- and its four lanes load six of the
// tap's 24 window values each: exactly the B fragment of the mma (slots 2j,
// 2j+1, 2j+8, 2j+9, 2j+16, 2j+17 for lane j of the quad; slots 24-31 are zero).
// The coefficient matrix is the A fragment (rows: the 15 monomials and one
// zero row), held in registers.  The D fragment gives each lane two
// coefficients of two taps; after four rounds every pixel's tap q has its 15
// coefficients in shared memory, and the pixel's own lane evaluates the tap.
__global__ void __launch_bounds__(ST_THREADS, 5) k_hex6_stencil(const double* __restrict__ scales, int C, int H, int W,
                                                              double h, const hex6_tile* __restrict__ tiles,
                                                              const u128* __restrict__ scratch,
                                                              const unsigned* __restrict__ wflag,
                                                              float* __restrict__ out, unsigned* __restrict__ status) {
    __shared__ int soff[HEX6_NREGION][HEX6_NSLOT];
    __shared__ __align__(16) int sym[HEX6_NREGION][8];  // L_r^-1 and v_r of each piece
    __shared__ int lut[16];
    __shared__ long long stp[2][6][ST_THREADS];  // per thread: the six steps of the tap mesh
    // per warp and pixel: the tap's 16 coefficient rows, exact.  Row m of pixel P sits in slot
    // m ^ (2 (P >> 3)) of a 17-slot record: the four lanes that write the same row of
    // different pixels, and the eight consecutive pixels that read, hit distinct banks.
    __shared__ __align__(16) dflt sdf[ST_THREADS / 32][32][TC_PSTRIDE];
    __shared__ __align__(16) i128 sc0[ST_THREADS / 32][32];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    if (tid < 16) lut[tid] = HEX6_REGION_LUT[tid];
    if (tid < HEX6_NREGION * 8) sym[tid / 8][tid % 8] = (tid % 8) < 6 ? HEX6_SYM[tid / 8][tid % 8] : 0;
    const hex6_tile tl = tiles[blockIdx.y];
    const int ncol = tl.ncol;
    for (int k = tid; k < HEX6_NREGION * HEX6_NSLOT; k += ST_THREADS) {
        const int r = k / HEX6_NSLOT, sl = k % HEX6_NSLOT;
        // linear offset of the slot's lattice point from the tap's cell corner
        soff[r][sl] = -(int)HEX6_DJ[r][sl] * (ncol + 2) - (int)HEX6_DI[r][sl];
    }
    __syncthreads();
    const int c = blockIdx.z;
    if (wflag[blockIdx.y * C + c]) {  // window values beyond the exact range (uniform over the block)
        const int per_row = tl.w / (int)blockDim.x;
        const int x = tl.x0 + (blockIdx.x % per_row) * (int)blockDim.x + threadIdx.x;
        const int y = tl.y0 + (blockIdx.x / per_row) * (int)blockDim.y + threadIdx.y;
        if (x < W && y < H && x < tl.x0 + tl.w && y < tl.y0 + tl.hh) {
            raise_status(status, BSF_ERANGE);
            out[((size_t)tl.b * C + c) * ((long long)H * W) + (long long)y * W + x] = __int_as_float(0x7fc00000);
        }
        return;
    }
    // the coefficient matrix as the mma's A fragments: rows = monomials (row 15 zero),
    // columns = the 24 slots of the canonical piece (columns 24-31 zero)
    unsigned afr[2][4];
    {
        const int g = lane >> 2, t2 = 2 * (lane & 3);
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = g + ((q & 1) ? 8 : 0), col = 16 * ks + t2 + ((q & 2) ? 8 : 0);
                const int c0 = (row < HEX6_NMONO && col < HEX6_NSLOT) ? HEX6_CC_CONST[col][row] : 0;
                const int c1 = (row < HEX6_NMONO && col + 1 < HEX6_NSLOT) ? HEX6_CC_CONST[col + 1][row] : 0;
                const __half2 hv = __halves2half2(__int2half_rn(c0), __int2half_rn(c1));
                afr[ks][q] = *reinterpret_cast<const unsigned*>(&hv);
            }
    }
    const int per_row = tl.w / (int)blockDim.x;
    const int bx = blockIdx.x % per_row, by = blockIdx.x / per_row;
    const int x = tl.x0 + bx * (int)blockDim.x + threadIdx.x;
    const int y = tl.y0 + by * (int)blockDim.y + threadIdx.y;
    // lanes outside the image or the tile take part in the warp's work with unit
    // scales and write nothing
    const bool active = x < W && y < H && x < tl.x0 + tl.w && y < tl.y0 + tl.hh;
    const long long HW = (long long)H * W, p = (long long)y * W + x;
    double a[6], prod = 1.0;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        a[k] = active ? scales[((size_t)tl.b * 6 + k) * HW + p] : 1.0;
        bad |= !(a[k] > 0.0);
    }
    if (bad) {
#pragma unroll
        for (int k = 0; k < 6; ++k) a[k] = 1.0;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) prod *= a[k];
    const u128* G = scratch + tl.off + (long long)c * ncol * tl.nrow;
    const double SQ3 = 1.73205080756887729353;
    const double it2 = 2.0 / (h * SQ3), ih = 1.0 / h;
    const double SC = 281474976710656.0;  // 2^48
    // the first tap, n + tau, tau = (1/2) sum (a_k - b_k) u_k, b = h (1, sqrt3, 1, sqrt3, 1, sqrt3),
    // in lattice coordinates s = x/h - t/2, t = 2y/(h sqrt3): cell (ib, jb) and a 48-bit fraction
    double yx = (double)x, yy = (double)y;
    long long ds[6], dtt[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double bk = (k & 1) ? h * SQ3 : h;
        yx += 0.5 * (a[k] - bk) * cos_k(k);
        yy += 0.5 * (a[k] - bk) * sin_k(k);
        // the step -a_k u_k in lattice coordinates, rounded once to 48 fractional bits
        ds[k] = __double2ll_rn(-a[k] * (cos_k(k) * ih - 0.5 * it2 * sin_k(k)) * SC);
        dtt[k] = __double2ll_rn(-a[k] * sin_k(k) * it2 * SC);
    }
    const double t0 = yy * it2, s0 = yx * ih - 0.5 * t0;
    const double fib = floor(s0), fjb = floor(t0);
    const int ib = (int)fib, jb = (int)fjb;
    const long long bs = __double2ll_rn((s0 - fib) * SC), bt = __double2ll_rn((t0 - fjb) * SC);
    const long long M48 = (1LL << 48) - 1, ONE = 1LL << 48;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        stp[0][k][tid] = ds[k];
        stp[1][k][tid] = dtt[k];
    }
    __syncwarp();
    const int safe_base = 2 * ncol + 6;  // a cell whose 24 points lie inside every window
    const int j4 = lane & 3, quad0 = lane & ~3;
    const int s_lo = 2 * j4;             // this lane's slots: s_lo, +1, +8, +9, +16, +17
    const int g = lane >> 2;             // D rows g and g + 8; columns 2 j4, 2 j4 + 1
    bool halo_bad = false;
    i128 e00 = 0;            // exact sum over the taps of +-A_00
    dflt rest = {0.f, 0.f};  // the other terms
    long long sp = bs, tp = bt;  // the tap's position (Gray-code order: one step changes per tap)
    // this lane's own tap of the current group of four rounds
    int my_base = safe_base, my_reg = 0;
    long long my_x1 = 0, my_x2 = 0;
#pragma unroll 1
    for (int q = 0; q < 64; ++q) {
        // ---- the position of tap q of this lane's pixel
        const int gq = q ^ (q >> 1);
        if (q) {
            const int k = __ffs(q) - 1;
            const long long dsk = stp[0][k][tid], dtk = stp[1][k][tid];
            if ((gq >> k) & 1) {
                sp += dsk;
                tp += dtk;
            } else {
                sp -= dsk;
                tp -= dtk;
            }
        }
        {
            const int i0 = ib + (int)(sp >> 48), j0 = jb + (int)(tp >> 48);
            const long long sf = sp & M48, tf = tp & M48;
            int code;
            if (sf + tf < ONE)
                code = (sf > tf) | ((2 * sf + tf > ONE) << 1) | ((sf + 2 * tf > ONE) << 2);
            else
                code = 8 | (sf > tf) | ((2 * sf + tf > 2 * ONE) << 1) | ((sf + 2 * tf > 2 * ONE) << 2);
            const int reg = lut[code];
            const int rr = j0 - tl.j0w;
            const int cc = i0 - tl.i_left + 2 * rr;
            const bool inside = rr >= 2 && rr + 3 < tl.nrow && cc >= 6 && cc + 9 < ncol;
            halo_bad |= !inside && active && !bad;
            // the tap in the canonical piece: x = L_r^-1 ((sigma, tau) - v_r), exact (48-bit fractions)
            const int4 sl = *reinterpret_cast<const int4*>(&sym[reg][0]);
            const int2 sv = *reinterpret_cast<const int2*>(&sym[reg][4]);
            const long long xs = sf - (long long)sv.x * ONE, xt = tf - (long long)sv.y * ONE;
            my_x1 = sl.x * xs + sl.y * xt;
            my_x2 = sl.z * xs + sl.w * xt;
            my_base = inside ? rr * ncol + cc : safe_base;
            my_reg = reg;
        }
        // ---- four rounds: quad n takes tap q of pixel 4 n + i
#pragma unroll 1
        for (int i = 0; i < 4; ++i) {
            const int src = quad0 | i;
            const int tb = __shfl_sync(0xffffffffu, my_base, src);
            const int treg = __shfl_sync(0xffffffffu, my_reg, src);
            const u128* base = G + tb;
            uint4 u[6];
            u[0] = __ldg(reinterpret_cast<const uint4*>(base + soff[treg][s_lo]));
            u[1] = __ldg(reinterpret_cast<const uint4*>(base + soff[treg][s_lo + 1]));
            u[2] = __ldg(reinterpret_cast<const uint4*>(base + soff[treg][s_lo + 8]));
            u[3] = __ldg(reinterpret_cast<const uint4*>(base + soff[treg][s_lo + 9]));
            u[4] = __ldg(reinterpret_cast<const uint4*>(base + soff[treg][s_lo + 16]));
            u[5] = __ldg(reinterpret_cast<const uint4*>(base + soff[treg][s_lo + 17]));
#pragma unroll
            for (int s = 0; s < 6; ++s) u[s].z ^= 0x80000000u;  // bits 64-95 of g + 2^95
            // the four values of this lane (rows g, g + 8 x two taps): per group of four
            // bytes, gsum[w][v] = sum_b 2^(8 b) (byte sum b), exact in 64 bits
            long long gsum[3][4];
#pragma unroll
            for (int w = 0; w < 3; ++w) {
                unsigned b00[4], b01[4], b10[4];
#pragma unroll
                for (int bt = 0; bt < 4; ++bt) {
                    const unsigned sel = (unsigned)bt | ((4u + bt) << 8);
                    unsigned wv[6];
#pragma unroll
                    for (int s6 = 0; s6 < 6; ++s6) wv[s6] = w == 0 ? u[s6].x : (w == 1 ? u[s6].y : u[s6].z);
                    b00[bt] = bytes_as_f16x2(wv[0], wv[1], sel);
                    b01[bt] = bytes_as_f16x2(wv[2], wv[3], sel);
                    b10[bt] = bytes_as_f16x2(wv[4], wv[5], sel);
                }
                float d[4][4];
#pragma unroll
                for (int bt = 0; bt < 4; ++bt)
                    mma16816(d[bt], afr[0], b00[bt], b01[bt], TC_MAGIC, TC_MAGIC, TC_MAGIC, TC_MAGIC);
#pragma unroll
                for (int bt = 0; bt < 4; ++bt)
                    mma16816(d[bt], afr[1], b10[bt], 0u, d[bt][0], d[bt][1], d[bt][2], d[bt][3]);
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    // (bits - MAGIC) of two bytes, combined modulo 2^32: the true value is
                    // below 2^28 in magnitude, so the wrapped result is exact
                    const unsigned b0 = __float_as_uint(d[0][v]), b1 = __float_as_uint(d[1][v]);
                    const unsigned b2 = __float_as_uint(d[2][v]), b3 = __float_as_uint(d[3][v]);
                    const int x01 = (int)(b0 + 256u * b1 - 257u * (unsigned)TC_MAGIC_BITS);
                    const int x23 = (int)(b2 + 256u * b3 - 257u * (unsigned)TC_MAGIC_BITS);
                    gsum[w][v] = (long long)x01 + (long long)x23 * 65536;
                }
            }
            // hand the four coefficients to their pixels: columns 2 j4, 2 j4 + 1 are the taps
            // of quads 2 j4 and 2 j4 + 1, i.e. pixels 8 j4 + i and 8 j4 + 4 + i.  The value is
            // gsum0 + 2^32 gsum1 + 2^64 gsum2, assembled from 64-bit halves with one carry.
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const unsigned long long g0 = (unsigned long long)gsum[0][v];
                const unsigned long long lo = g0 + ((unsigned long long)gsum[1][v] << 32);
                const unsigned long long carry = lo < g0 ? 1ull : 0ull;
                const unsigned long long hi = (unsigned long long)(gsum[0][v] >> 63) +
                                              (unsigned long long)(gsum[1][v] >> 32) +
                                              (unsigned long long)gsum[2][v] + carry;
                const int row = g + ((v & 2) ? 8 : 0);
                const int pix = 8 * j4 + ((v & 1) ? 4 : 0) + i;
                const i128 av = (i128)(((u128)hi << 64) | lo);
                sdf[warp][pix][row ^ (2 * j4)] = df_of_i128(av);
                if (row == 0) sc0[warp][pix] = av;
            }
        }
        __syncwarp();
        // ---- this lane's tap q: F = (A_00 + sum_m A_m x^m) / 432, with the sign of the tap;
        // the quartic by Horner's rule in x1 over polynomials in x2 (monomial order of the
        // tables: 1, x1, x2, x1^2, x1 x2, x2^2, x1^3, x1^2 x2, x1 x2^2, x2^3, x1^4, ...)
        {
            const bool neg = __popc(gq) & 1;
            const dflt* rec = sdf[warp][lane];
            const int sw = 2 * (lane >> 3);
            const i128 A0 = sc0[warp][lane];
            e00 += neg ? -A0 : A0;
            dflt ad[HEX6_NMONO];
#pragma unroll
            for (int m = 1; m < HEX6_NMONO; ++m) ad[m] = rec[m ^ sw];
            const dflt sg = df_of_frac48(my_x1), tg = df_of_frac48(my_x2);
            const dflt p0 = df_mul(tg, df_fma(tg, df_fma(tg, df_fma(tg, ad[14], ad[9]), ad[5]), ad[2]));
            const dflt p1 = df_fma(tg, df_fma(tg, df_fma(tg, ad[13], ad[8]), ad[4]), ad[1]);
            const dflt p2 = df_fma(tg, df_fma(tg, ad[12], ad[7]), ad[3]);
            const dflt p3 = df_fma(tg, ad[11], ad[6]);
            const dflt fq = df_fma(sg, df_fma(sg, df_fma(sg, df_fma(sg, ad[10], p3), p2), p1), p0);
            rest = df_add(rest, neg ? dflt{-fq.hi, -fq.lo} : fq);
        }
        __syncwarp();
    }
    if (!active) return;
    float* o = out + ((size_t)tl.b * C + c) * HW + p;
    if (bad) {
        *o = __int_as_float(0x7fc00000);
        return;
    }
    if (halo_bad) {
        raise_status(status, BSF_EHALO);
        *o = __int_as_float(0x7fc00000);
        return;
    }
    // fbar = (1 / prod a) sum_q (-1)^|q| F(y_q); F = 6 h^4 sum_m g[m] M(.) / 432 with
    // the window holding the running sums times 2^24.  The constant parts of the
    // byte decomposition (the offsets 2^95 and 1024 per byte) are the same for
    // every tap and cancel in the alternating sum.
    const long long ehi = (long long)(e00 >> 64);
    const double ev = fma((double)ehi, 18446744073709551616.0, (double)(unsigned long long)e00);
    const double h2 = h * h;
    *o = (float)((ev + (double)rest.hi + (double)rest.lo) * (6.0 * h2 * h2 / (16777216.0 * HEX6_DEN)) / prod);
}
}  // namespace


size_t lut6_bytes() { return (size_t)(LUT6_NU + 1) * (LUT6_NP + 1) * 8 * sizeof(float); }

cudaError_t launch_lut6_build(double eta, double rel, float* table, cudaStream_t st) {
    const int n = (LUT6_NU + 1) * (LUT6_NP + 1);
    k_lut6_build<<<(n + 127) / 128, 128, 0, st>>>(eta, rel, table);
    return cudaGetLastError();
}

cudaError_t launch_map6(const float* params, int kind, int B, int H, int W, int tile, double eps, double eta,
                        double rel, double ascale, double* scales, unsigned* tile_ext, unsigned* status,
                        cudaStream_t st, const float* lut) {
    const long long HW = (long long)H * W, n = HW * B;
    const int tiles_x = (W + tile - 1) / tile, tiles_y = (H + tile - 1) / tile;
    k_map6<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(params, kind, HW, B, W, tile, tiles_x, tiles_x * tiles_y, eps,
                                                        eta, rel, ascale, scales, tile_ext, status, lut);
    return cudaGetLastError();
}

cudaError_t launch_map6_out(const float* params, int kind, long long npix, double eps, double eta, double rel,
                            float* scales, uint8_t* flags, cudaStream_t st, const float* lut) {
    if (npix == 0) return cudaSuccess;
    k_map6_out<<<(unsigned)((npix + 127) / 128), 128, 0, st>>>(params, kind, npix, eps, eta, rel, scales, flags,
                                                               lut);
    return cudaGetLastError();
}

cudaError_t launch_hex6_preint(int dtype_u8, const void* img, int C, int H, int W, double h, const hex6_tile* tiles,
                               int ntiles, int ncol_max, void* scratch, unsigned* wflag, cudaStream_t st,
                               int reflect) {
    const size_t smem = (4 * (size_t)(ncol_max + ncol_max / HEX6_PRE_PAD + 1) + 32) * sizeof(u128);
    // as many threads as the widest window of the chunk needs (PRE_CPT columns each, whole
    // warps): narrow windows take small blocks, several of them per SM
    if (ncol_max < 1 || ncol_max > PRE_THREADS * PRE_CPT) return cudaErrorInvalidValue;
    const int nthr = ((ncol_max + PRE_CPT - 1) / PRE_CPT + 31) / 32 * 32;
    dim3 grid(ntiles, C);
    // the attribute is the kernel's largest shared-memory size (set on every launch, the
    // same value each time: launches from several host threads never lower it for another);
    // each launch still asks only for its chunk's size
    const int smem_cap =
        (int)((4 * (size_t)(hex6_max_cols() + hex6_max_cols() / HEX6_PRE_PAD + 1) + 32) * sizeof(u128));
    if ((int)smem > smem_cap) return cudaErrorInvalidValue;
    if (dtype_u8) {
        cudaFuncSetAttribute(k_hex6_preint<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_cap);
        k_hex6_preint<uint8_t><<<grid, nthr, smem, st>>>((const uint8_t*)img, C, H, W, h, tiles, (u128*)scratch,
                                                                 wflag, reflect);
    } else {
        cudaFuncSetAttribute(k_hex6_preint<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_cap);
        k_hex6_preint<float><<<grid, nthr, smem, st>>>((const float*)img, C, H, W, h, tiles, (u128*)scratch,
                                                               wflag, reflect);
    }
    return cudaGetLastError();
}

cudaError_t launch_hex6_stencil(const double* scales, int C, int H, int W, int tile_w, int tile_h, double h,
                                const hex6_tile* tiles, int ntiles, const void* scratch, const unsigned* wflag,
                                float* out, unsigned* status, cudaStream_t st) {
    // 16 x 16 tiles, or 64-pixel tiles and their groups (64 x 64 up to 256 x 128)
    const bool fine = tile_w == 16 && tile_h == 16;
    const bool coarse = (tile_w == 64 || tile_w == 128 || tile_w == 256) && (tile_h == 64 || tile_h == 128);
    if (!fine && !coarse) return cudaErrorInvalidValue;
    const dim3 blk = tile_w == 16 ? dim3(16, 8) : dim3(32, 4);
    dim3 grid((tile_w / blk.x) * (tile_h / blk.y), ntiles, C);
    k_hex6_stencil<<<grid, blk, 0, st>>>(scales, C, H, W, h, tiles, (const u128*)scratch, wflag, out, status);
    return cudaGetLastError();
}
