/*
 * bsf_oracle6.c -- plain FP64 CPU restatement of Algorithm 1 for the
 * six-directional box spline on the hexagonal lattice (the same reading as
 * oracle/n6.py: the image transferred once to Lambda_h = { h (i + j/2,
 * j sqrt3/2) }, on which the directions theta_k = k pi/6 are the lattice
 * vectors (1,0), (1,1), (0,1), (-1,2), (-1,1), (-2,1) with lengths
 * b = h (1, sqrt3, 1, sqrt3, 1, sqrt3)).
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of oracle/: used by tests/ and by
 * the CPU-baseline leg of bench.py; it shares nothing with the CUDA library.
 * It exists because the numpy restatement (n6.alg1_hex) scans the whole
 * lattice box for every tap and cannot finish a crop of a real workload; the
 * steps, their order and the arithmetic (FP64 throughout) are the same, and
 * tests/test_oracle_hex6.py pins the two against each other.
 *
 *   step 1  transfer: each pixel's mass goes to the three vertices of the
 *           lattice triangle holding it, in proportion to its barycentric
 *           coordinates;
 *   step 2  pre-integration: six running sums along the lattice vectors, each
 *           times its length b_k (Eq. 2DRS with b_k u_k = h v_k);
 *   step 3  Eq. keyeqn: fbar[n] = (1/prod a) sum_q (-1)^|q| F(n + tau - x_q)
 *           over the 64 taps of Eq. FD_mesh, tau = (1/2) sum_k (a_k - b_k) u_k,
 *           F(y) = sum_m g[m] beta^6_b(y - m), beta^6_b by the truncated power
 *           of the six directions differenced over its 64 corners (Eq. const
 *           read through Eq. FD_mesh).
 * Pixels are independent in step 3: they run on all host threads (OpenMP).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SQRT3_6 1.73205080756887729353

static const int HV[6][2] = {{1, 0}, {1, 1}, {0, 1}, {-1, 2}, {-1, 1}, {-2, 1}};
static const double HLEN[6] = {1.0, SQRT3_6, 1.0, SQRT3_6, 1.0, SQRT3_6};

static void dirs6(double u[6][2]) {
    for (int k = 0; k < 6; ++k) {
        const double th = k * M_PI / 6.0;
        u[k][0] = cos(th);
        u[k][1] = sin(th);
    }
}

/* truncated power (cone spline) of the six unit directions:
   T(x) = sum_k det(u_k, x)_+^4 / (4! prod_{j != k} det(u_k, u_j)) on the open
   half-plane that holds the directions, 0 outside it */
static double cone6(const double u[6][2], const double den[6], const double v[2], double x1, double x2) {
    if (!(v[0] * x2 - v[1] * x1 > 0.0)) return 0.0;
    double s = 0.0;
    for (int k = 0; k < 6; ++k) {
        const double d = u[k][0] * x2 - u[k][1] * x1;
        if (d > 0.0) s += d * d * d * d / den[k];
    }
    return s;
}

/* beta^6_a(x), centred: (1/prod a) sum_q (-1)^|q| T(x + c - sum_k q_k a_k u_k),
   c = sum_k a_k u_k / 2 */
static double beta6(const double u[6][2], const double den[6], const double v[2], const double a[6], double x1,
                    double x2) {
    double c1 = 0.0, c2 = 0.0, pa = 1.0;
    for (int k = 0; k < 6; ++k) {
        c1 += 0.5 * a[k] * u[k][0];
        c2 += 0.5 * a[k] * u[k][1];
        pa *= a[k];
    }
    double r = 0.0;
    for (int q = 0; q < 64; ++q) {
        double s1 = c1, s2 = c2;
        int par = 0;
        for (int k = 0; k < 6; ++k)
            if ((q >> k) & 1) {
                s1 -= a[k] * u[k][0];
                s2 -= a[k] * u[k][1];
                par ^= 1;
            }
        const double t = cone6(u, den, v, x1 + s1, x2 + s2);
        r += par ? -t : t;
    }
    return r / pa;
}

static void cone_consts(const double u[6][2], double den[6], double v[2]) {
    for (int k = 0; k < 6; ++k) {
        double d = 24.0; /* 4! */
        for (int j = 0; j < 6; ++j)
            if (j != k) d *= u[k][0] * u[j][1] - u[k][1] * u[j][0];
        den[k] = d;
    }
    /* the half-plane's normal side: the middle of the empty sector (150, 180 degrees) */
    const double mid = 0.5 * (5.0 * M_PI / 6.0 + M_PI);
    v[0] = cos(mid);
    v[1] = sin(mid);
    /* directions on the positive side: det(v, u_k) > 0 for every k (checked by the pins) */
    if (v[0] * u[0][1] - v[1] * u[0][0] < 0.0) {
        v[0] = -v[0];
        v[1] = -v[1];
    }
}

/* beta^6_a at a point, for the pins (same evaluation as step 3 uses) */
double bo_beta6(const double a[6], double x1, double x2) {
    double u[6][2], den[6], v[2];
    dirs6(u);
    cone_consts(u, den, v);
    return beta6(u, den, v, a, x1, x2);
}

static void support_extent6(const double u[6][2], const double a[6], double* ex, double* ey) {
    double sx = 0.0, sy = 0.0;
    for (int k = 0; k < 6; ++k) {
        sx += a[k] * fabs(u[k][0]);
        sy += a[k] * fabs(u[k][1]);
    }
    *ex = 0.5 * sx;
    *ey = 0.5 * sy;
}

/* f: H x W image (row-major, FP64); a: six planes of H*W widths; idx: the
   npix pixels to evaluate (npix < 0: all); out: npix results.  Returns 0, or
   -1 when the lattice box cannot be allocated. */
int bo_alg1_hex6(const double* f, int H, int W, const double* a, const int64_t* idx, int64_t npix, double h,
                 double* out) {
    const int64_t HW = (int64_t)H * W, count = npix < 0 ? HW : npix;
    double u[6][2], den[6], v[2], b[6];
    dirs6(u);
    cone_consts(u, den, v);
    for (int k = 0; k < 6; ++k) b[k] = h * HLEN[k];
    /* the lattice box: every point step 3 reads (footprint + the support of
       beta_b), extended to the right so that the 120 and 150 degree sums
       start in the empty part below the image */
    double exm = 0.0, eym = 0.0;
    for (int64_t t = 0; t < count; ++t) {
        const int64_t p = npix < 0 ? t : idx[t];
        double ak[6], ex, ey;
        for (int k = 0; k < 6; ++k) ak[k] = a[k * HW + p];
        support_extent6(u, ak, &ex, &ey);
        if (ex > exm) exm = ex;
        if (ey > eym) eym = ey;
    }
    double bsum = 0.0;
    for (int k = 0; k < 6; ++k) bsum += b[k];
    const double ex = exm + bsum + 2 * h, ey = eym + bsum + 2 * h;
    const double hy = h * SQRT3_6 / 2.0;
    const int j_lo = (int)floor(-ey / hy) - 2, j_hi = (int)ceil((H - 1 + ey) / hy) + 2;
    const int nrow = j_hi - j_lo + 1;
    const int i_lo = (int)floor(-ex / h - 0.5 * j_hi) - 2;
    const int i_hi = (int)ceil((W - 1 + ex) / h - 0.5 * j_lo) + 2 + 2 * nrow;
    const int ncol = i_hi - i_lo + 1;
    double* g = (double*)calloc((size_t)nrow * ncol, sizeof(double));
    double* o2 = (double*)calloc((size_t)nrow * ncol, sizeof(double));
    if (!g || !o2) {
        free(g);
        free(o2);
        return -1;
    }
#define G(A, r, c) A[(size_t)(r) * ncol + (c)]
    /* step 1: the transfer (barycentric shares of each pixel's mass) */
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const double fv = f[(int64_t)y * W + x];
            const double tt = 2.0 * y / (h * SQRT3_6), ss = x / h - 0.5 * tt;
            const int i = (int)floor(ss), j = (int)floor(tt);
            const double sg = ss - i, tg = tt - j;
            int vi[3], vj[3];
            double w[3];
            if (sg + tg < 1.0) {
                vi[0] = i; vj[0] = j; w[0] = 1.0 - sg - tg;
                vi[1] = i + 1; vj[1] = j; w[1] = sg;
                vi[2] = i; vj[2] = j + 1; w[2] = tg;
            } else {
                vi[0] = i + 1; vj[0] = j + 1; w[0] = sg + tg - 1.0;
                vi[1] = i; vj[1] = j + 1; w[1] = 1.0 - sg;
                vi[2] = i + 1; vj[2] = j; w[2] = 1.0 - tg;
            }
            for (int k = 0; k < 3; ++k) G(g, vj[k] - j_lo, vi[k] - i_lo) += w[k] * fv;
        }
    /* step 2: six running sums, each times its length */
    for (int k = 0; k < 6; ++k) {
        const int di = HV[k][0], dj = HV[k][1];
        for (int r = 0; r < nrow; ++r)
            for (int c = 0; c < ncol; ++c) {
                double s = G(g, r, c);
                if (dj == 0) {
                    if (c > 0) s += G(o2, r, c - 1);
                } else if (r - dj >= 0 && c - di >= 0 && c - di < ncol) {
                    s += G(o2, r - dj, c - di);
                }
                G(o2, r, c) = s;
            }
        for (size_t e = 0; e < (size_t)nrow * ncol; ++e) g[e] = b[k] * o2[e];
    }
    double bx, by;
    support_extent6(u, b, &bx, &by);
    /* step 3: the 64 taps of every pixel */
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < count; ++t) {
        const int64_t p = npix < 0 ? t : idx[t];
        const int ny = (int)(p / W), nx = (int)(p % W);
        double ak[6], pa = 1.0, tau1 = 0.0, tau2 = 0.0;
        for (int k = 0; k < 6; ++k) {
            ak[k] = a[k * HW + p];
            pa *= ak[k];
            tau1 += 0.5 * (ak[k] - b[k]) * u[k][0];
            tau2 += 0.5 * (ak[k] - b[k]) * u[k][1];
        }
        double acc = 0.0;
        for (int q = 0; q < 64; ++q) {
            double y1 = nx + tau1, y2 = ny + tau2;
            int par = 0;
            for (int k = 0; k < 6; ++k)
                if ((q >> k) & 1) {
                    y1 -= ak[k] * u[k][0];
                    y2 -= ak[k] * u[k][1];
                    par ^= 1;
                }
            /* lattice points m with |m - y| inside the support box of beta_b */
            double F = 0.0;
            const int jlo = (int)ceil((y2 - by - 1e-9) / hy), jhi = (int)floor((y2 + by + 1e-9) / hy);
            for (int j = jlo; j <= jhi; ++j) {
                const int ilo = (int)ceil((y1 - bx - 1e-9) / h - 0.5 * j);
                const int ihi = (int)floor((y1 + bx + 1e-9) / h - 0.5 * j);
                for (int i = ilo; i <= ihi; ++i) {
                    const double lx = h * (i + 0.5 * j), ly = hy * j;
                    const double bw = beta6(u, den, v, b, y1 - lx, y2 - ly);
                    if (bw != 0.0) F += G(g, j - j_lo, i - i_lo) * bw;
                }
            }
            acc += par ? -F : F;
        }
        out[t] = acc / pa;
    }
#undef G
    free(g);
    free(o2);
    return 0;
}
