/*
 * bsf_oracle.c -- plain, slow, FP64 CPU oracle for space-variant elliptical
 * filtering with radially-uniform box splines (Chaudhury, Munoz-Barrutia,
 * Unser, "Fast space-variant elliptical filtering using box splines").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * it is used by tests/, by __graft_entry__.smoke() and by the CPU-baseline
 * leg of bench.py.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * Conventions (paper Sec. 2.2.1):
 *   points x = (x1, x2), x1 = column index, x2 = row index;
 *   u_theta = (cos theta, sin theta), theta_k = (k-1) pi / N;
 *   beta^N_a = phi_{a1,theta1} * ... * phi_{aN,thetaN}  (Eq. const), where
 *   phi_{a,theta} is the density of s u_theta with s uniform on [-a/2, a/2].
 *
 * Parts:
 *   O-beta   bo_beta4 (area form), bo_beta4_lines (line-integral form)
 *   O-direct bo_direct4: fbar[n] = sum_k f[k] beta_{a(n)}(n - k)  (Eq. SVF_2D
 *            with the Dirac-comb image of Eq. keyeqn's derivation)
 *   O-alg    bo_preint4_i64 / bo_preint4_f64 (Algorithm 1 step 2) and
 *            bo_stencil4 (Algorithm 1 step 3, Table 1, Eq. final_eqn)
 *   O-map    bo_map4 (Sec. 3.2.2 steps (i)-(iii))
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SQRT2 1.41421356237309504880
#define INV_SQRT2 0.70710678118654752440

/* ------------------------------------------------------------------ */
/* O-beta, area form.                                                  */
/* beta^4_a(x) is the density of x = s1 u1 + s2 u2 + s3 u3 + s4 u4 with */
/* s_k uniform on [-a_k/2, a_k/2] (Eq. const, four directions 0, pi/4,  */
/* pi/2, 3pi/4).  Conditioning on (s2, s4) leaves (s1, s3) =             */
/* x - s2 u2 - s4 u4, so beta = area(R and Q) / (a1 a2 a3 a4) with       */
/* R = [-a2/2,a2/2] x [-a4/2,a4/2] and Q the four half-planes below.     */
/* ------------------------------------------------------------------ */
typedef struct { double u, v; } pt2;

/* keep the part of polygon p (n vertices) with al*u + be*v <= ga */
static int clip_halfplane(const pt2* p, int n, double al, double be, double ga, pt2* out) {
    int m = 0;
    for (int i = 0; i < n; ++i) {
        pt2 A = p[i], B = p[(i + 1) % n];
        double dA = al * A.u + be * A.v - ga;
        double dB = al * B.u + be * B.v - ga;
        if (dA <= 0) out[m++] = A;
        if ((dA < 0 && dB > 0) || (dA > 0 && dB < 0)) {
            double t = dA / (dA - dB);
            out[m].u = A.u + t * (B.u - A.u);
            out[m].v = A.v + t * (B.v - A.v);
            ++m;
        }
    }
    return m;
}

static double polygon_area(const pt2* p, int n) {
    double s = 0;
    for (int i = 0; i < n; ++i) {
        const pt2 A = p[i], B = p[(i + 1) % n];
        s += A.u * B.v - B.u * A.v;
    }
    return 0.5 * fabs(s);
}

double bo_beta4(const double a[4], double x1, double x2) {
    pt2 P[16], Q[16];
    int n = 4;
    P[0].u = -a[1] / 2; P[0].v = -a[3] / 2;
    P[1].u =  a[1] / 2; P[1].v = -a[3] / 2;
    P[2].u =  a[1] / 2; P[2].v =  a[3] / 2;
    P[3].u = -a[1] / 2; P[3].v =  a[3] / 2;
    /* s1 = x1 - (s2 - s4)/sqrt2 in [-a1/2, a1/2]; s3 = x2 - (s2 + s4)/sqrt2 in [-a3/2, a3/2] */
    n = clip_halfplane(P, n,  INV_SQRT2, -INV_SQRT2,  x1 + a[0] / 2, Q); if (n < 3) return 0;
    n = clip_halfplane(Q, n, -INV_SQRT2,  INV_SQRT2, -x1 + a[0] / 2, P); if (n < 3) return 0;
    n = clip_halfplane(P, n,  INV_SQRT2,  INV_SQRT2,  x2 + a[2] / 2, Q); if (n < 3) return 0;
    n = clip_halfplane(Q, n, -INV_SQRT2, -INV_SQRT2, -x2 + a[2] / 2, P); if (n < 3) return 0;
    return polygon_area(P, n) / (a[0] * a[1] * a[2] * a[3]);
}

/* ------------------------------------------------------------------ */
/* O-beta, line-integral form (a second, independent evaluation):      */
/*   beta^3(y) = (1/(a1 a2 a3)) |{s in [-a2/2,a2/2] :                   */
/*                |y1 - s/sqrt2| <= a1/2, |y2 - s/sqrt2| <= a3/2}|       */
/*   beta^4(x) = (1/a4) int_{-a4/2}^{a4/2} beta^3(x - s u4) ds           */
/* beta^3 is piecewise linear in s along the line; it is integrated     */
/* exactly with the trapezoid rule between all candidate breakpoints.   */
/* ------------------------------------------------------------------ */
static double beta3_line(const double a[4], double y1, double y2) {
    double lo = -a[1] / 2, hi = a[1] / 2, t;
    t = SQRT2 * (y1 - a[0] / 2); if (t > lo) lo = t;
    t = SQRT2 * (y1 + a[0] / 2); if (t < hi) hi = t;
    t = SQRT2 * (y2 - a[2] / 2); if (t > lo) lo = t;
    t = SQRT2 * (y2 + a[2] / 2); if (t < hi) hi = t;
    return hi > lo ? (hi - lo) / (a[0] * a[1] * a[2]) : 0.0;
}

static int cmp_double(const void* A, const void* B) {
    double a = *(const double*)A, b = *(const double*)B;
    return (a > b) - (a < b);
}

double bo_beta4_lines(const double a[4], double x1, double x2) {
    /* along y(s) = x - s u4 = (x1 + s/sqrt2, x2 - s/sqrt2) the six bounds are   */
    /* L = {-a2/2, sqrt2 x1 + s - a1/sqrt2... } : each is c + k s with k in {0,1,-1} */
    double c[6], k[6];
    c[0] = -a[1] / 2;                      k[0] = 0;   /* lower */
    c[1] = SQRT2 * x1 - SQRT2 * a[0] / 2;  k[1] = 1;   /* lower */
    c[2] = SQRT2 * x2 - SQRT2 * a[2] / 2;  k[2] = -1;  /* lower */
    c[3] = a[1] / 2;                       k[3] = 0;   /* upper */
    c[4] = SQRT2 * x1 + SQRT2 * a[0] / 2;  k[4] = 1;   /* upper */
    c[5] = SQRT2 * x2 + SQRT2 * a[2] / 2;  k[5] = -1;  /* upper */
    double bp[40];
    int nb = 0;
    bp[nb++] = -a[3] / 2;
    bp[nb++] = a[3] / 2;
    for (int i = 0; i < 6; ++i)
        for (int j = i + 1; j < 6; ++j)
            if (k[i] != k[j]) {
                double s = (c[j] - c[i]) / (k[i] - k[j]);
                if (s > -a[3] / 2 && s < a[3] / 2) bp[nb++] = s;
            }
    qsort(bp, nb, sizeof(double), cmp_double);
    double tot = 0;
    for (int i = 0; i + 1 < nb; ++i) {
        double s0 = bp[i], s1 = bp[i + 1];
        if (s1 <= s0) continue;
        double f0 = beta3_line(a, x1 + s0 * INV_SQRT2, x2 - s0 * INV_SQRT2);
        double f1 = beta3_line(a, x1 + s1 * INV_SQRT2, x2 - s1 * INV_SQRT2);
        tot += 0.5 * (s1 - s0) * (f0 + f1);
    }
    return tot / a[3];
}

/* ------------------------------------------------------------------ */
/* O-direct: the plain definition                                     */
/*   fbar[n] = sum_k f[k] beta^4_{a(n)}(n - k),  f zero outside image  */
/* a is given as 4 planes of H*W doubles (plane k holds a_{k+1}).       */
/* Only the listed pixels idx[0..npix) are evaluated (npix < 0: all).   */
/* ------------------------------------------------------------------ */
static int support_halfwidth(const double a[4], double* hx, double* hy) {
    /* support polygon {sum t_k a_k u_k, |t_k|<=1/2} (Sec. 2.2.1) */
    *hx = 0.5 * (a[0] + (a[1] + a[3]) * INV_SQRT2);
    *hy = 0.5 * (a[2] + (a[1] + a[3]) * INV_SQRT2);
    return 0;
}

void bo_direct4(const double* f, int H, int W, const double* a, const int64_t* idx, int64_t npix,
                double* out) {
    const int64_t HW = (int64_t)H * W;
    const int64_t count = npix < 0 ? HW : npix;
    /* pixels are independent: shared among the host threads */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < count; ++t) {
        const int64_t p = npix < 0 ? t : idx[t];
        const int n2 = (int)(p / W), n1 = (int)(p % W);
        double ak[4] = {a[p], a[HW + p], a[2 * HW + p], a[3 * HW + p]};
        double hx, hy;
        support_halfwidth(ak, &hx, &hy);
        int k1lo = (int)floor(n1 - hx) - 1, k1hi = (int)ceil(n1 + hx) + 1;
        int k2lo = (int)floor(n2 - hy) - 1, k2hi = (int)ceil(n2 + hy) + 1;
        if (k1lo < 0) k1lo = 0;
        if (k2lo < 0) k2lo = 0;
        if (k1hi > W - 1) k1hi = W - 1;
        if (k2hi > H - 1) k2hi = H - 1;
        double s = 0;
        for (int k2 = k2lo; k2 <= k2hi; ++k2)
            for (int k1 = k1lo; k1 <= k1hi; ++k1) {
                double fv = f[(int64_t)k2 * W + k1];
                if (fv == 0) continue;
                s += fv * bo_beta4(ak, (double)(n1 - k1), (double)(n2 - k2));
            }
        out[t] = s;
    }
}

/* ------------------------------------------------------------------ */
/* O-adjoint: the transpose of the plain definition,                   */
/*   (K^T g)[k] = sum_n g[n] beta^4_{a(n)}(n - k),                      */
/* the gradient of sum_n g[n] fbar[n] with respect to f[k].  Evaluated   */
/* for the listed points k by gathering over every pixel n whose support */
/* can reach k (support half-widths bounded by amax).                    */
/* ------------------------------------------------------------------ */
void bo_adjoint4(const double* g, int H, int W, const double* a, double amax, const int64_t* idx, int64_t npts,
                 double* out) {
    const int64_t HW = (int64_t)H * W;
    const int R = (int)ceil(0.5 * (amax + SQRT2 * amax)) + 2;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < npts; ++t) {
        const int k2 = (int)(idx[t] / W), k1 = (int)(idx[t] % W);
        double s = 0;
        for (int n2 = k2 - R; n2 <= k2 + R; ++n2) {
            if (n2 < 0 || n2 >= H) continue;
            for (int n1 = k1 - R; n1 <= k1 + R; ++n1) {
                if (n1 < 0 || n1 >= W) continue;
                const int64_t p = (int64_t)n2 * W + n1;
                if (g[p] == 0) continue;
                const double ak[4] = {a[p], a[HW + p], a[2 * HW + p], a[3 * HW + p]};
                s += g[p] * bo_beta4(ak, (double)(n1 - k1), (double)(n2 - k2));
            }
        }
        out[t] = s;
    }
}

/* ------------------------------------------------------------------ */
/* O-alg step 2: the four recursions of Algorithm 1 on a zero-padded   */
/* buffer of (H+2P) rows x (W+2P) columns holding f at offset (P,P),    */
/* every recursion started from zero initial values at the buffer edge. */
/*   g0[n1,n2]   = f[n1,n2] + g0[n1-1,n2]                    (RS1)       */
/*   g45[n1,n2]  = sqrt2 g0[n1,n2] + g45[n1-1,n2-1]          (RS2)       */
/*   g90[n1,n2]  = g45[n1,n2] + g90[n1,n2-1]                 (RS3)       */
/*   gb[n1,n2]   = sqrt2 g90[n1,n2] + gb[n1+1,n2-1]          (RS4)       */
/* Integer form: the two sqrt2 factors are taken out, G is the integer  */
/* result of the same recursions without them, and gb = 2 G exactly.   */
/* Integer arithmetic wraps modulo 2^64 (unsigned), as exact sums mod   */
/* 2^64 are all that any later exact integer combination needs.         */
/* ------------------------------------------------------------------ */
void bo_preint4_i64(const int64_t* f, int H, int W, int P, int64_t* Gout) {
    const int Hp = H + 2 * P, Wp = W + 2 * P;
    const int64_t n = (int64_t)Hp * Wp;
    uint64_t* g0 = (uint64_t*)calloc(n, 8);
    uint64_t* g45 = (uint64_t*)calloc(n, 8);
    uint64_t* g90 = (uint64_t*)calloc(n, 8);
    uint64_t* G = (uint64_t*)calloc(n, 8);
#define AT(A, c, r) A[(int64_t)(r) * Wp + (c)]
    /* RS1 runs along rows (rows independent); RS2-RS4 step from row r-1 to row r
       (the columns of one row independent) */
#pragma omp parallel for schedule(static)
    for (int r = 0; r < Hp; ++r)
        for (int c = 0; c < Wp; ++c) {
            uint64_t fv = 0;
            if (r >= P && r < P + H && c >= P && c < P + W) fv = (uint64_t)f[(int64_t)(r - P) * W + (c - P)];
            AT(g0, c, r) = fv + (c > 0 ? AT(g0, c - 1, r) : 0);
        }
    for (int r = 0; r < Hp; ++r) {
#pragma omp parallel for schedule(static)
        for (int c = 0; c < Wp; ++c)
            AT(g45, c, r) = AT(g0, c, r) + (c > 0 && r > 0 ? AT(g45, c - 1, r - 1) : 0);
    }
    for (int r = 0; r < Hp; ++r) {
#pragma omp parallel for schedule(static)
        for (int c = 0; c < Wp; ++c)
            AT(g90, c, r) = AT(g45, c, r) + (r > 0 ? AT(g90, c, r - 1) : 0);
    }
    for (int r = 0; r < Hp; ++r) {
#pragma omp parallel for schedule(static)
        for (int c = Wp - 1; c >= 0; --c)
            AT(G, c, r) = AT(g90, c, r) + (c + 1 < Wp && r > 0 ? AT(G, c + 1, r - 1) : 0);
    }
    memcpy(Gout, G, n * 8);
    free(g0); free(g45); free(g90); free(G);
}

void bo_preint4_f64(const double* f, int H, int W, int P, double* gbout) {
    const int Hp = H + 2 * P, Wp = W + 2 * P;
    const int64_t n = (int64_t)Hp * Wp;
    double* g0 = (double*)calloc(n, 8);
    double* g45 = (double*)calloc(n, 8);
    double* g90 = (double*)calloc(n, 8);
    double* gb = gbout;
#pragma omp parallel for schedule(static)
    for (int r = 0; r < Hp; ++r)
        for (int c = 0; c < Wp; ++c) {
            double fv = 0;
            if (r >= P && r < P + H && c >= P && c < P + W) fv = f[(int64_t)(r - P) * W + (c - P)];
            AT(g0, c, r) = fv + (c > 0 ? AT(g0, c - 1, r) : 0);
        }
    for (int r = 0; r < Hp; ++r) {
#pragma omp parallel for schedule(static)
        for (int c = 0; c < Wp; ++c)
            AT(g45, c, r) = SQRT2 * AT(g0, c, r) + (c > 0 && r > 0 ? AT(g45, c - 1, r - 1) : 0);
    }
    for (int r = 0; r < Hp; ++r) {
#pragma omp parallel for schedule(static)
        for (int c = 0; c < Wp; ++c)
            AT(g90, c, r) = AT(g45, c, r) + (r > 0 ? AT(g90, c, r - 1) : 0);
    }
    for (int r = 0; r < Hp; ++r) {
#pragma omp parallel for schedule(static)
        for (int c = Wp - 1; c >= 0; --c)
            AT(gb, c, r) = SQRT2 * AT(g90, c, r) + (c + 1 < Wp && r > 0 ? AT(gb, c + 1, r - 1) : 0);
    }
    free(g0); free(g45); free(g90);
#undef AT
}

/* ------------------------------------------------------------------ */
/* O-alg step 3 (Algorithm 1, Table 1, Eq. final_eqn):                 */
/*   fbar[n] = sum_{i=0}^{15} w_i F(n + tau - x_i)                      */
/*   F(y) = sum_m gb[m] beta^4_b(y - m),  b = (1, sqrt2, 1, sqrt2)       */
/* The ZP weights beta^4_b(y - m) come from bo_beta4 at a = b.          */
/* x_i = q1 a1 (1,0) + q2 a2' (1,1) + q3 a3 (0,1) + q4 a4' (-1,1) with   */
/* i = q1 + 2 q2 + 4 q3 + 8 q4 and a'_k = a_k / sqrt2 (Table 1);         */
/* w_i = (-1)^(q1+q2+q3+q4) / (a1 a2 a3 a4) (Eq. FD_mesh);               */
/* tau1 = (sqrt2 a1 + a2 - a4 - sqrt2) / (2 sqrt2),                     */
/* tau2 = (a2 + sqrt2 a3 + a4 - 3 sqrt2) / (2 sqrt2)  (Sec. 3.1 step 2).  */
/* gb is the buffer of bo_preint4_* (row-major, Wp columns, offset P).   */
/* Returns the number of pixels whose taps left the buffer (their       */
/* output is NaN).                                                       */
/* ------------------------------------------------------------------ */
int64_t bo_stencil4(const double* gb, int H, int W, int P, const double* a, const int64_t* idx,
                    int64_t npix, double* out) {
    const int Hp = H + 2 * P, Wp = W + 2 * P;
    const int64_t HW = (int64_t)H * W;
    const double bvec[4] = {1.0, SQRT2, 1.0, SQRT2};
    const int64_t count = npix < 0 ? HW : npix;
    int64_t bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : bad)
    for (int64_t t = 0; t < count; ++t) {
        const int64_t p = npix < 0 ? t : idx[t];
        const int n2 = (int)(p / W), n1 = (int)(p % W);
        const double a1 = a[p], a2 = a[HW + p], a3 = a[2 * HW + p], a4 = a[3 * HW + p];
        const double a2p = a2 * INV_SQRT2, a4p = a4 * INV_SQRT2;
        const double w = 1.0 / (a1 * a2 * a3 * a4);
        const double tau1 = (SQRT2 * a1 + a2 - a4 - SQRT2) / (2 * SQRT2);
        const double tau2 = (a2 + SQRT2 * a3 + a4 - 3 * SQRT2) / (2 * SQRT2);
        double s = 0;
        int outside = 0;
        for (int i = 0; i < 16; ++i) {
            const int q1 = i & 1, q2 = (i >> 1) & 1, q3 = (i >> 2) & 1, q4 = (i >> 3) & 1;
            const double xi1 = q1 * a1 + q2 * a2p - q4 * a4p;
            const double xi2 = q2 * a2p + q3 * a3 + q4 * a4p;
            const double wi = ((q1 + q2 + q3 + q4) & 1) ? -w : w;
            /* y in buffer coordinates */
            const double y1 = n1 + P + tau1 - xi1, y2 = n2 + P + tau2 - xi2;
            /* ZP interpolation: all lattice m with beta_b(y - m) possibly > 0 */
            double F = 0;
            const int m1c = (int)floor(y1 + 0.5), m2c = (int)floor(y2 + 0.5);
            for (int d2 = -2; d2 <= 2; ++d2)
                for (int d1 = -2; d1 <= 2; ++d1) {
                    const int m1 = m1c + d1, m2 = m2c + d2;
                    const double bw = bo_beta4(bvec, y1 - m1, y2 - m2);
                    if (bw == 0) continue;
                    if (m1 < 0 || m1 >= Wp || m2 < 0 || m2 >= Hp) { outside = 1; continue; }
                    F += gb[(int64_t)m2 * Wp + m1] * bw;
                }
            s += wi * F;
        }
        if (outside) { out[t] = NAN; ++bad; }
        else out[t] = s;
    }
    return bad;
}

/* ------------------------------------------------------------------ */
/* O-map (Sec. 3.2.2): covariance -> optimal scale vector, N = 4.        */
/* Input kinds: 1 = COV (C11, C12, C22) in px^2; 2 = SRT (sigma, rho,    */
/* theta) with sigma the std along the major axis: lambda_max = sigma^2, */
/* lambda_min = sigma^2 / rho, theta the major-axis orientation.         */
/* Params are 3 planes of npix doubles; a_out is 4 planes.                */
/*                                                                       */
/* Reading for elongations beyond Prop. 3.1's bound: when rho exceeds    */
/* (1 - eta) U(theta) it is lowered to that value keeping the size       */
/* s = lambda_max + lambda_min and theta (descriptor D1), and the pixel  */
/* is flagged 1.  If p >= eps is still infeasible, t is the midpoint of  */
/* [t_r, t_l], p is raised to eps, and the pixel is flagged 2.  A        */
/* covariance that is not positive definite or not finite gives NaN     */
/* scales and flag 4.                                                    */
/* ------------------------------------------------------------------ */
static double U_bound(double phi) {
    /* Prop. 3.1: U = (1+|nu|+sqrt(1+nu^2)) / (1+|nu|-sqrt(1+nu^2)),
       nu = (tan phi - cot phi)/2 * sign(pi/2 - phi).  Infinite at the four
       principal directions (nu infinite or nu = 0). */
    const double PI = 3.14159265358979323846;
    const double tn = tan(phi);
    if (!isfinite(tn) || fabs(tn) < 1e-300) return INFINITY;
    double sg = (phi < PI / 2) ? 1.0 : (phi > PI / 2 ? -1.0 : 0.0);
    if (sg == 0.0) return INFINITY;
    double nu = 0.5 * (tn - 1.0 / tn) * sg;
    double an = fabs(nu), r = sqrt(1.0 + nu * nu);
    double den = 1.0 + an - r;
    if (!(den > 0)) return INFINITY;
    return (1.0 + an + r) / den;
}

double bo_U_bound(double phi) { return U_bound(phi); }

static double zeta_val(const double pb[4], double t) {
    /* zeta(t) = sum_k (pb_k + e_k t)^4 + ((pb1+t)^2 + (pb3+t)^2)((pb2-t)^2 + (pb4-t)^2) */
    const double p1 = pb[0] + t, p2 = pb[1] - t, p3 = pb[2] + t, p4 = pb[3] - t;
    return p1 * p1 * p1 * p1 + p2 * p2 * p2 * p2 + p3 * p3 * p3 * p3 + p4 * p4 * p4 * p4 +
           (p1 * p1 + p3 * p3) * (p2 * p2 + p4 * p4);
}

/* all real roots of c0 t^3 + c1 t^2 + c2 t + c3 (c0 != 0); textbook
   trigonometric / Cardano solution, each root polished by two Newton steps */
static int cubic_real_roots(double c0, double c1, double c2, double c3, double r[3]) {
    const double PI = 3.14159265358979323846;
    const double A = c1 / c0, B = c2 / c0, C = c3 / c0;
    const double Q = (A * A - 3 * B) / 9.0;
    const double R = (2 * A * A * A - 9 * A * B + 27 * C) / 54.0;
    int n;
    if (R * R < Q * Q * Q) {
        const double th = acos(R / sqrt(Q * Q * Q));
        const double sq = -2 * sqrt(Q);
        r[0] = sq * cos(th / 3) - A / 3;
        r[1] = sq * cos((th + 2 * PI) / 3) - A / 3;
        r[2] = sq * cos((th - 2 * PI) / 3) - A / 3;
        n = 3;
    } else {
        double Aa = -copysign(cbrt(fabs(R) + sqrt(R * R - Q * Q * Q)), R);
        double Bb = (Aa != 0) ? Q / Aa : 0;
        r[0] = (Aa + Bb) - A / 3;
        n = 1;
    }
    for (int i = 0; i < n; ++i)
        for (int it = 0; it < 2; ++it) {
            const double t = r[i];
            const double f = ((c0 * t + c1) * t + c2) * t + c3;
            const double df = (3 * c0 * t + 2 * c1) * t + c2;
            if (df != 0) r[i] = t - f / df;
        }
    return n;
}

int bo_map4(const double* params, int kind, int64_t npix, double eps, double eta, double* a_out,
            uint8_t* flags) {
    const double PI = 3.14159265358979323846;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t p = 0; p < npix; ++p) {
        double C11, C12, C22;
        uint8_t flag = 0;
        if (kind == 2) {
            const double sg = params[p], rho = params[npix + p], th = params[2 * npix + p];
            const double lmax = sg * sg, lmin = sg * sg / rho;
            const double c = cos(th), s = sin(th);
            /* descriptor D2 -> covariance (Sec. 3.2.1) */
            C11 = lmax * c * c + lmin * s * s;
            C12 = 0.5 * (lmax - lmin) * sin(2 * th);
            C22 = lmin * c * c + lmax * s * s;
        } else {
            C11 = params[p]; C12 = params[npix + p]; C22 = params[2 * npix + p];
        }
        /* eigen-description (Eq. def_eigen) */
        const double tr = C11 + C22;
        const double dd = sqrt((C11 - C22) * (C11 - C22) + 4 * C12 * C12);
        double lmax = 0.5 * (tr + dd), lmin = 0.5 * (tr - dd);
        if (!(isfinite(C11) && isfinite(C12) && isfinite(C22)) || !(lmin > 0)) {
            for (int k = 0; k < 4; ++k) a_out[k * npix + p] = NAN;
            if (flags) flags[p] = 4;
            continue;
        }
        /* major-axis orientation in [0, pi) */
        double th = 0.5 * atan2(2 * C12, C11 - C22);
        if (th < 0) th += PI;
        const double rho = lmax / lmin;
        const double U = U_bound(th);
        if (rho > (1 - eta) * U) {
            const double s = lmax + lmin;
            const double rc = (1 - eta) * U;
            lmax = s * rc / (1 + rc);   /* descriptor D1 */
            lmin = s / (1 + rc);
            const double c = cos(th), sn = sin(th);
            C11 = lmax * c * c + lmin * sn * sn;
            C12 = 0.5 * (lmax - lmin) * sin(2 * th);
            C22 = lmin * c * c + lmax * sn * sn;
            flag |= 1;
        }
        /* (i) c = 24 (C11, C12, C22); particular solution with p4 = 1 */
        const double c1 = 24 * C11, c2 = 24 * C12, c3 = 24 * C22;
        double pb[4];
        pb[3] = 1.0;
        pb[1] = c2 + pb[3];
        pb[0] = (c1 - pb[1] - pb[3]) / 2;
        pb[2] = (c3 - pb[1] - pb[3]) / 2;
        /* (ii) feasible interval and the cubic zeta'(t) = z1 t^3 + z2 t^2 + z3 t + z4 */
        const double tl = fmax(eps - pb[0], eps - pb[2]);
        const double trr = fmin(pb[1] - eps, pb[3] - eps);
        double t0;
        if (tl > trr) {
            t0 = 0.5 * (tl + trr);
            flag |= 2;
        } else {
            const double z1 = 32;
            const double z2 = 24 * (pb[0] - pb[1] + pb[2] - pb[3]);
            const double z3 = 16 * (pb[0] * pb[0] + pb[1] * pb[1] + pb[2] * pb[2] + pb[3] * pb[3]) -
                              8 * (pb[0] + pb[2]) * (pb[1] + pb[3]);
            const double z4 = 4 * (pb[0] * pb[0] * pb[0] - pb[1] * pb[1] * pb[1] + pb[2] * pb[2] * pb[2] -
                                   pb[3] * pb[3] * pb[3]) +
                              2 * (pb[0] + pb[2]) * (pb[1] * pb[1] + pb[3] * pb[3]) -
                              2 * (pb[1] + pb[3]) * (pb[0] * pb[0] + pb[2] * pb[2]);
            /* (iii) candidates: real roots inside (tl, tr) and the two ends */
            double roots[3];
            const int nr = cubic_real_roots(z1, z2, z3, z4, roots);
            t0 = tl;
            double best = zeta_val(pb, tl);
            const double zr = zeta_val(pb, trr);
            if (zr < best) { best = zr; t0 = trr; }
            for (int i = 0; i < nr; ++i)
                if (roots[i] > tl && roots[i] < trr) {
                    const double z = zeta_val(pb, roots[i]);
                    if (z < best) { best = z; t0 = roots[i]; }
                }
        }
        double pk[4] = {pb[0] + t0, pb[1] - t0, pb[2] + t0, pb[3] - t0};
        for (int k = 0; k < 4; ++k) {
            if (flag & 2) pk[k] = fmax(pk[k], eps);
            a_out[k * npix + p] = sqrt(fmax(pk[k], 0.0));
        }
        if (flags) flags[p] = flag;
    }
    return 0;
}

/* Number of host threads the parallel loops above use (1 without OpenMP). */
int bo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
