// Local finite difference with Zwart-Powell interpolation (Algorithm 1
// step 3; Table 1; Eq. final_eqn; App. F), four-directional box spline.
//
// For every pixel n with scale vector a = a(n):
//   fbar[n] = (1/(a1 a2 a3 a4)) sum_{i=0}^{15} (-1)^{|q|} F(n + tau - x_i),
//   F(y)    = sum_m g_b[m] beta_b(y - m),   g_b = 2 G,
// with x_i = q1 a1 (1,0) + q2 a2' (1,1) + q3 a3 (0,1) + q4 a4' (-1,1),
// a'_k = a_k / sqrt2, tau = ((a1 + a2' - a4' - 1)/2, (a2' + a3 + a4' - 3)/2).
// So fbar = (1/(a1 a2' a3 a4')) sum_i s_i sum_m G[m] beta_b(y_i - m).
//
// ZP interpolation.  Let m0 = round(y) and phi = y - m0 in [-1/2, 1/2)^2.
// On the cell around m0, F is a C1 piecewise quadratic whose only breaks are
// the cell's two diagonals (the ZP element is Eq. const at a = b =
// (1, sqrt2, 1, sqrt2); its knot lines are x, y in 1/2 + Z and x +- y in Z).
// Such a function is one quadratic plus a multiple of each truncated power
// across the diagonals.  With the 3x3 neighbourhood of m0 named
//     a b c        (row above)
//     d e f        (row of m0)
//     g h i        (row below)
// and x' = phi_x + 1/2, y' = phi_y + 1/2 in [0, 1) (origin at the cell's
// upper-left corner), the derivation from the element's polynomial pieces
// gives
//   16 F = 4 s + 8 (cx x' + cy y') + 16 (cxx x'^2 + 2 m x'y' + cyy y'^2)
//          + 16 A ((x' - y')_+)^2 + 16 B ((x' + y' - 1)_+)^2,
//   s = a + b + d + e,  u1 = d - f,  u2 = h - b,  m = (a - g) + u2,
//   cxx = (a + g) - (b + h) + 2 (f - e),   cyy = (a + g) + (b + h) - 2 (d + e),
//   cx = -2 u1 - cxx - m,   cy = 2 u2 - cyy - m,
//   A = u1 + u2 + (c - g),  B = u1 - u2 + (i - a).
// The nine loads have fixed offsets from m0, so the 32 lanes of a warp
// (consecutive pixels, neighbouring taps) read consecutive addresses.
//
// Exact integer form (MODE_U64 / MODE_U128).  a'_k is rounded to A_k 2^-q
// with a per-pixel q; then every tap position lies on the 2^-(q+1) grid, the
// mesh of Table 1 is exact for the rounded scales, and
//   S = 2^(2q+4) sum_i s_i F(y_i)
// is an integer combination of G.  It is evaluated modulo 2^64 / 2^128: the
// true S is bounded by 2^(2q+4) * max|f| * prod(a') * (lattice mass), and q
// is chosen per pixel so that this bound stays below 2^(ACC-2); then the
// wrapped result IS S, whatever the size of G.  The only rounding is the
// final conversion fbar = S 2^(2q-4-frac) / prod(A) in FP32.
//
// All-FP64 form (MODE_F64): the same formulas in double, positions and
// weights unrounded (Algorithm 1 computed literally).
#include "bsf_common.cuh"
#include "bsf_internal.h"
#include "map4.cuh"
#include "tma.cuh"

#include <climits>

namespace {

__device__ __forceinline__ int ilog2_ceil(float v) {
    // smallest integer e with 2^e >= v, for v > 0
    int e;
    const float m = frexpf(v, &e);  // v = m 2^e, m in [0.5, 1)
    return (m == 0.5f) ? e - 1 : e;
}

template <class T> __device__ __forceinline__ T mul_u32(T v, unsigned s) { return v * (T)s; }

template <int MODE> struct pixel_acc;

template <int MODE>
__device__ __forceinline__ void load_scales(int kind, const float* __restrict__ pr, size_t HW, size_t p, float eps,
                                            float eta, float& a1, float& a2, float& a3, float& a4, int& mflag) {
    mflag = 0;
    if (kind == BSF_PARAM_SCALES) {
        a1 = pr[p];
        a2 = pr[HW + p];
        a3 = pr[2 * HW + p];
        a4 = pr[3 * HW + p];
    } else {
        const map4_result R = map4_solve(kind, pr[p], pr[HW + p], pr[2 * HW + p], eps, eta);
        a1 = R.a[0];
        a2 = R.a[1];
        a3 = R.a[2];
        a4 = R.a[3];
        mflag = R.flag;
    }
}

// Tap i of a pixel at buffer position (bx, by) with integer scales A1..A4 on
// the 2^-(q+1) grid: the cell (cx, cy) of tau - x_i + 1/2, the offsets X, Y from
// the cell corner, the truncated-power arguments T1, T2 and the sign of the tap.
struct tap_geom {
    int cx, cy;
    unsigned X, Y, T1, T2;
    bool pos;
};
__device__ __forceinline__ tap_geom tap_at(int i, int A1, int A2, int A3, int A4, int sh1, int bx, int by) {
    const int two = 2 << (sh1 - 1), mask = two - 1;
    const int sg1 = (i & 1) ? -1 : 1, sg2 = (i & 2) ? -1 : 1, sg3 = (i & 4) ? -1 : 1, sg4 = (i & 8) ? -1 : 1;
    // tau - x_i + 1/2 in units of 2^-(q+1): cell index and offset from the cell corner
    const int tx = sg1 * A1 + sg2 * A2 - sg4 * A4;
    const int ty = sg2 * A2 + sg3 * A3 + sg4 * A4 - two;
    tap_geom g;
    g.cx = bx + (tx >> sh1);
    g.cy = by + (ty >> sh1);
    g.X = (unsigned)(tx & mask);
    g.Y = (unsigned)(ty & mask);
    g.T1 = (unsigned)max((int)g.X - (int)g.Y, 0);
    g.T2 = (unsigned)max((int)(g.X + g.Y) - two, 0);
    g.pos = (sg1 * sg2 * sg3 * sg4) > 0;
    return g;
}

// One tap's contribution to S = 2^(2q+2) SK + 2^(q+1) SL + SQ from the 3x3
// neighbourhood a..i of its cell (the ZP element of the header comment).
template <class T>
__device__ __forceinline__ void zp_tap(T a, T b, T c, T d, T e, T f, T g, T h, T ii, const tap_geom& t, T& SK,
                                       T& SL, T& SQ) {
    const T u1 = d - f, u2 = h - b;
    const T Ac = u1 + u2 + (c - g);
    const T Bc = u1 - u2 + (ii - a);
    const T m = (a - g) + u2;
    const T ag = a + g, bh = b + h;
    const T cxx = ag - bh + ((f - e) << 1);
    const T cyy = ag + bh - ((d + e) << 1);
    const T cxl = T(0) - (u1 << 1) - cxx - m;
    const T cyl = (u2 << 1) - cyy - m;
    const T sk = a + b + d + e;
    const T sl = mul_u32(cxl, t.X) + mul_u32(cyl, t.Y);
    const T sq = mul_u32(mul_u32(cxx, t.X) + mul_u32(m << 1, t.Y), t.X) + mul_u32(mul_u32(cyy, t.Y), t.Y) +
                 mul_u32(mul_u32(Ac, t.T1), t.T1) + mul_u32(mul_u32(Bc, t.T2), t.T2);
    if (t.pos) { SK += sk; SL += sl; SQ += sq; } else { SK -= sk; SL -= sl; SQ -= sq; }
}

// CTA shape of the exact stencil: 32 consecutive pixels of a row per warp,
// ROWS rows per CTA; the register bound keeps MINB CTAs resident per SM.
// Measured on GB300 (2048^2 workload): the 64-bit form runs best at 72
// registers, 28 warps per SM (4% faster than 80 registers, 24 warps); the
// 128-bit form is bound by its 16-byte loads and ran within 4% of the best at
// every bound tried from 80 to 168 registers, best at 80.
template <int MODE> struct stencil_shape { static constexpr int ROWS = 4, MINB = 7; };
template <> struct stencil_shape<MODE_U128> { static constexpr int ROWS = 8, MINB = 3; };

// Per-pixel set-up shared by the exact stencils: the scales (read, or from the
// fused map), the per-pixel exponent q, the integer scales A_k = round(a'_k 2^q)
// and the buffer position.  Pixels that cannot be filtered get NaN and a status
// bit here and come back with ok = false.
struct pix_setup {
    int A1, A2, A3, A4, q, sh1, bx, by;
    bool ok;
};

template <int MODE, int KIND>
__device__ __forceinline__ pix_setup setup_pixel(int n1, int n2, int im, int Hp, int Wp, int P, int H, int W, int C,
                                                 int col0, const float* __restrict__ params, float eps, float eta,
                                                 float ascale, float* __restrict__ out, unsigned* status) {
    constexpr int ACC = mode_traits<MODE>::ACC_BITS;
    constexpr int VAL = mode_traits<MODE>::VAL_BITS;
    pix_setup S;
    S.ok = false;
    const size_t HW = (size_t)H * W, p = (size_t)n2 * W + n1;
    const int K = (KIND == BSF_PARAM_SCALES) ? 4 : 3;
    const float* pr = params + (size_t)(im / C) * K * HW;
    float a1, a2, a3, a4;
    int mflag;
    load_scales<MODE>(KIND, pr, HW, p, eps, eta, a1, a2, a3, a4, mflag);
    a1 *= ascale;  // 1, or 1/sqrt(m) for a pass of the m-fold iterated filter
    a2 *= ascale;
    a3 *= ascale;
    a4 *= ascale;
    float* o = out + (size_t)im * HW + p;
    if (mflag & 1) raise_status(status, BSF_EINFEASIBLE);
    if (!(a1 > 0.f && a2 > 0.f && a3 > 0.f && a4 > 0.f) || !(a1 < 1e30f && a2 < 1e30f && a3 < 1e30f && a4 < 1e30f)) {
        raise_status(status, BSF_EBADSCALE);
        *o = __int_as_float(0x7fc00000);
        return S;
    }
    const float a2p = a2 * 0.70710678118654752f, a4p = a4 * 0.70710678118654752f;
    // bound on prod(a') * lattice mass
    const float Bm = fminf((a1 + 1.f) * (a3 + 1.f) * a2p * a4p, 0.5f * a1 * a3 * (2.f * a2p + 1.f) * (a4p + 1.f));
    int q = (ACC - 6 - VAL - ilog2_ceil(Bm)) >> 1;
    q = min(q, 24);
    q = min(q, 30 - ilog2_ceil(a1 + a2p + a3 + a4p + 3.f));
    if (q < 0) {
        raise_status(status, BSF_ERANGE);
        *o = __int_as_float(0x7fc00000);
        return S;
    }
    const float sc = ldexpf(1.f, q);
    const int A1 = __float2int_rn(a1 * sc), A2 = __float2int_rn(a2p * sc);
    const int A3 = __float2int_rn(a3 * sc), A4 = __float2int_rn(a4p * sc);
    if (A1 < 1 || A2 < 1 || A3 < 1 || A4 < 1) {
        raise_status(status, BSF_ERANGE);
        *o = __int_as_float(0x7fc00000);
        return S;
    }
    const int sh1 = q + 1;
    const int bx = n1 - col0 + P, by = n2 + P;
    const int two = 2 << q;
    // The tap offsets below range over tx in [-(A1+A2+A4), A1+A2+A4] and
    // ty in [-(A2+A3+A4), A2+A3+A4] - 2^(q+1), and every extreme is reached by
    // some tap; the 3x3 neighbourhood of each tap's cell lies in the buffer iff
    // the extreme cells are at least one element inside it.  Pixels whose
    // footprint leaves the buffer are flagged once, before any tap is read.
    {
        const int ex = A1 + A2 + A4, ey = A2 + A3 + A4;
        const bool inside = (bx + ((-ex) >> sh1) >= 1) & (bx + (ex >> sh1) <= Wp - 2) &
                            (by + ((-ey - two) >> sh1) >= 1) & (by + ((ey - two) >> sh1) <= Hp - 2);
        if (!inside) {
            raise_status(status, BSF_EHALO);
            *o = __int_as_float(0x7fc00000);
            return S;
        }
    }
    S = pix_setup{A1, A2, A3, A4, q, sh1, bx, by, true};
    return S;
}

template <int MODE, int KIND>
__global__ void __launch_bounds__(32 * stencil_shape<MODE>::ROWS, stencil_shape<MODE>::MINB) k_stencil4_exact(const void* __restrict__ buf, long long buf_stride, int Hp,
                                                         int Wp, int pitch, int P, int H, int W, int C, int col0,
                                                         int col1, const float* __restrict__ params, float eps,
                                                         float eta, float ascale, float* __restrict__ out,
                                                         unsigned* status) {
    typedef typename mode_traits<MODE>::T T;
    constexpr int FRAC = mode_traits<MODE>::FRAC_BITS;
    const int n1 = col0 + blockIdx.x * 32 + threadIdx.x;
    const int n2 = blockIdx.y * stencil_shape<MODE>::ROWS + threadIdx.y;
    const int im = blockIdx.z;
    if (n1 >= col1 || n2 >= H) return;
    const pix_setup ps = setup_pixel<MODE, KIND>(n1, n2, im, Hp, Wp, P, H, W, C, col0, params, eps, eta, ascale, out,
                                                 status);
    if (!ps.ok) return;
    const int A1 = ps.A1, A2 = ps.A2, A3 = ps.A3, A4 = ps.A4, q = ps.q, sh1 = ps.sh1, bx = ps.bx, by = ps.by;
    const T* G = (const T*)buf + (size_t)im * buf_stride;
    float* o = out + (size_t)im * ((size_t)H * W) + (size_t)n2 * W + n1;
    // S = 2^(2q+4) sum_i s_i F(y_i) = 2^(2q+2) SK + 2^(q+1) SL + SQ: the terms of
    // each power of two are summed over the taps first and shifted once
    T SK = T(0), SL = T(0), SQ = T(0);
    // unrolled by 8, not 16: half the code keeps the instruction cache warm
    // (measured 1.4% faster for the 64-bit form, 15% for the 128-bit one)
#pragma unroll 8
    for (int i = 0; i < 16; ++i) {
        const tap_geom t = tap_at(i, A1, A2, A3, A4, sh1, bx, by);
        const T* r0 = G + ((size_t)(t.cy - 1) * pitch + t.cx);
        const T* r1 = r0 + pitch;
        const T* r2 = r1 + pitch;
        zp_tap<T>(r0[-1], r0[0], r0[1], r1[-1], r1[0], r1[1], r2[-1], r2[0], r2[1], t, SK, SL, SQ);
    }
    const T S = (SK << (2 * q + 2)) + (SL << (q + 1)) + SQ;
    const float prodA = ((float)A1 * (float)A2) * ((float)A3 * (float)A4);
    float sf;
    if constexpr (MODE == MODE_U64) sf = __ll2float_rn((long long)S);
    else sf = i128_to_float(S);
    *o = ldexpf(__fdividef(sf, prodA), 2 * q - 4 - FRAC);
}

// The same exact 64-bit stencil with the pre-integrated buffer staged in shared
// memory by the tensor-copy engine (TMA) instead of read through L1.  A CTA
// covers 32 x 8 pixels; the 16 taps are taken in two phases of eight.  In each
// phase the CTA finds, per tap, the box of cells its pixels' 3x3 neighbourhoods
// span (the halo of the tile for that tap, sized by the tile's own scales), and
// one thread copies each box that fits TMA_BW x TMA_BH elements into shared
// memory; a tap whose box does not fit (a tile with strongly varying scales)
// is read from global memory as in k_stencil4_exact.  The arithmetic is the
// same, so the two kernels give the same bits.  Measured on the 2048^2 u8
// workload this form is 1.36x slower than the L1 gather (0.54 against 0.40
// ms): the stencil is bound by integer issue, not by its loads (which hit L1
// for 92 % of their sectors), and the box search, barriers and bank conflicts
// of the staged loads add instructions.  The box size changed the share of
// taps read through L1 (53 % at 40 x 12, 20 % at 64 x 16) but not the time.
constexpr int TMA_BW = 64;        // box width in elements (x 8 bytes: a multiple of 16)
constexpr int TMA_BH = 16;        // box height
constexpr int TMA_ROWS = 8;       // pixel rows per CTA
constexpr int TMA_PHASE_TAPS = 8;
constexpr int TMA_PHASES = 16 / TMA_PHASE_TAPS;
constexpr size_t TMA_SMEM = (size_t)TMA_PHASE_TAPS * TMA_BW * TMA_BH * sizeof(unsigned long long);

template <int KIND>
__global__ void __launch_bounds__(32 * TMA_ROWS, 3)
    k_stencil4_tma(const __grid_constant__ CUtensorMap gmap, const unsigned long long* __restrict__ buf,
                   long long buf_stride, int Hp, int Wp, int pitch, int P, int H, int W, int C, int col0, int col1,
                   const float* __restrict__ params, float eps, float eta, float ascale, float* __restrict__ out,
                   unsigned* status, unsigned polls) {
    typedef unsigned long long T;
    extern __shared__ __align__(128) unsigned char tma_smem[];
    __shared__ uint64_t bar;
    __shared__ int red[TMA_ROWS][4 * TMA_PHASE_TAPS];  // per warp and tap: min cx, max cx, min cy, max cy
    __shared__ int box[TMA_PHASE_TAPS][3];             // per tap: box origin x, y; staged or not
    const T* sbuf = reinterpret_cast<const T*>(tma_smem);
    const int lane = threadIdx.x, warp = threadIdx.y, tid = warp * 32 + lane;
    const int n1 = col0 + blockIdx.x * 32 + lane;
    const int n2 = blockIdx.y * TMA_ROWS + warp;
    const int im = blockIdx.z;
    pix_setup ps{1, 1, 1, 1, 0, 1, 0, 0, false};
    if (n1 < col1 && n2 < H)
        ps = setup_pixel<MODE_U64, KIND>(n1, n2, im, Hp, Wp, P, H, W, C, col0, params, eps, eta, ascale, out,
                                         status);
    const bool act = ps.ok;
    if (!act) ps = pix_setup{1, 1, 1, 1, 0, 1, 0, 0, false};  // neutral geometry for the reductions
    const T* G = buf + (size_t)im * buf_stride;
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    T SK = T(0), SL = T(0), SQ = T(0);
    unsigned parity = 0;
    for (int ph = 0; ph < TMA_PHASES; ++ph) {
        // the cells each tap of this phase reads, reduced over the CTA
#pragma unroll
        for (int j = 0; j < TMA_PHASE_TAPS; ++j) {
            const tap_geom t = tap_at(ph * TMA_PHASE_TAPS + j, ps.A1, ps.A2, ps.A3, ps.A4, ps.sh1, ps.bx, ps.by);
            const int mnx = __reduce_min_sync(0xffffffffu, act ? t.cx : INT_MAX);
            const int mxx = __reduce_max_sync(0xffffffffu, act ? t.cx : INT_MIN);
            const int mny = __reduce_min_sync(0xffffffffu, act ? t.cy : INT_MAX);
            const int mxy = __reduce_max_sync(0xffffffffu, act ? t.cy : INT_MIN);
            if (lane == 0) {
                red[warp][4 * j] = mnx;
                red[warp][4 * j + 1] = mxx;
                red[warp][4 * j + 2] = mny;
                red[warp][4 * j + 3] = mxy;
            }
        }
        __syncthreads();
        if (tid < TMA_PHASE_TAPS) {
            int mnx = INT_MAX, mxx = INT_MIN, mny = INT_MAX, mxy = INT_MIN;
#pragma unroll
            for (int w = 0; w < TMA_ROWS; ++w) {
                mnx = min(mnx, red[w][4 * tid]);
                mxx = max(mxx, red[w][4 * tid + 1]);
                mny = min(mny, red[w][4 * tid + 2]);
                mxy = max(mxy, red[w][4 * tid + 3]);
            }
            // x rounded down to an even element: 16-byte aligned start (8-byte elements)
            const int ox = (mnx - 1) & ~1, oy = mny - 1;
            box[tid][0] = ox;
            box[tid][1] = oy;
            box[tid][2] = (mnx <= mxx) && (mxx + 1 - ox < TMA_BW) && (mxy + 1 - oy < TMA_BH);
        }
        __syncthreads();
        if (tid == 0) {
            unsigned bytes = 0;
#pragma unroll
            for (int j = 0; j < TMA_PHASE_TAPS; ++j)
                if (box[j][2]) bytes += TMA_BW * TMA_BH * (unsigned)sizeof(T);
            // every read of the previous phase's boxes happened before the block barrier above
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar, bytes);
#pragma unroll
            for (int j = 0; j < TMA_PHASE_TAPS; ++j)
                if (box[j][2])
                    tma_load_3d(tma_smem + (size_t)j * TMA_BW * TMA_BH * sizeof(T), &gmap, box[j][0], box[j][1], im,
                                &bar);
        }
        const bool ok = mbar_wait(&bar, parity, polls);
        if (__syncthreads_or(!ok)) {
            // the copies did not arrive in time: wait once more (bounded) so that none is
            // still writing this block's shared memory when it exits, then report
            mbar_wait(&bar, parity, polls > (1u << 22) ? polls : (1u << 22));
            if (tid == 0) raise_status(status, BSF_ETIMEOUT);
            if (act) out[(size_t)im * ((size_t)H * W) + (size_t)n2 * W + n1] = __int_as_float(0x7fc00000);
            return;
        }
        parity ^= 1u;
        if (act) {
#pragma unroll 8
            for (int j = 0; j < TMA_PHASE_TAPS; ++j) {
                const tap_geom t = tap_at(ph * TMA_PHASE_TAPS + j, ps.A1, ps.A2, ps.A3, ps.A4, ps.sh1, ps.bx, ps.by);
                if (box[j][2]) {
                    const T* r0 = sbuf + j * (TMA_BW * TMA_BH) + (t.cy - 1 - box[j][1]) * TMA_BW + (t.cx - box[j][0]);
                    const T* r1 = r0 + TMA_BW;
                    const T* r2 = r1 + TMA_BW;
                    zp_tap<T>(r0[-1], r0[0], r0[1], r1[-1], r1[0], r1[1], r2[-1], r2[0], r2[1], t, SK, SL, SQ);
                } else {
                    const T* r0 = G + ((size_t)(t.cy - 1) * pitch + t.cx);
                    const T* r1 = r0 + pitch;
                    const T* r2 = r1 + pitch;
                    zp_tap<T>(r0[-1], r0[0], r0[1], r1[-1], r1[0], r1[1], r2[-1], r2[0], r2[1], t, SK, SL, SQ);
                }
            }
        }
    }
    if (!act) return;
    const int q = ps.q;
    const T S = (SK << (2 * q + 2)) + (SL << (q + 1)) + SQ;
    const float prodA = ((float)ps.A1 * (float)ps.A2) * ((float)ps.A3 * (float)ps.A4);
    out[(size_t)im * ((size_t)H * W) + (size_t)n2 * W + n1] =
        ldexpf(__fdividef(__ll2float_rn((long long)S), prodA), 2 * q - 4);
}

template <int KIND>
__global__ void __launch_bounds__(256) k_stencil4_f64(const double* __restrict__ buf, long long buf_stride, int Hp,
                                                       int Wp, int pitch, int P, int H, int W, int C, int col0,
                                                       int col1, const float* __restrict__ params, float eps,
                                                       float eta, float ascale, float* __restrict__ out,
                                                       unsigned* status) {
    const int n1 = col0 + blockIdx.x * 32 + threadIdx.x;
    const int n2 = blockIdx.y * 8 + threadIdx.y;
    const int im = blockIdx.z;
    if (n1 >= col1 || n2 >= H) return;
    const size_t HW = (size_t)H * W, p = (size_t)n2 * W + n1;
    const int K = (KIND == BSF_PARAM_SCALES) ? 4 : 3;
    const float* pr = params + (size_t)(im / C) * K * HW;
    float fa1, fa2, fa3, fa4;
    int mflag;
    load_scales<MODE_F64>(KIND, pr, HW, p, eps, eta, fa1, fa2, fa3, fa4, mflag);
    fa1 *= ascale;
    fa2 *= ascale;
    fa3 *= ascale;
    fa4 *= ascale;
    float* o = out + (size_t)im * HW + p;
    if (mflag & 1) raise_status(status, BSF_EINFEASIBLE);
    if (!(fa1 > 0.f && fa2 > 0.f && fa3 > 0.f && fa4 > 0.f) ||
        !(fa1 < 1e30f && fa2 < 1e30f && fa3 < 1e30f && fa4 < 1e30f)) {
        raise_status(status, BSF_EBADSCALE);
        *o = __int_as_float(0x7fc00000);
        return;
    }
    const double a1 = fa1, a3 = fa3;
    const double a2p = (double)fa2 * 0.70710678118654752440, a4p = (double)fa4 * 0.70710678118654752440;
    const double* G = buf + (size_t)im * buf_stride;
    const int bx = n1 - col0 + P, by = n2 + P;
    double S = 0.0;
    bool bad = false;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const double sg1 = (i & 1) ? -1.0 : 1.0, sg2 = (i & 2) ? -1.0 : 1.0;
        const double sg3 = (i & 4) ? -1.0 : 1.0, sg4 = (i & 8) ? -1.0 : 1.0;
        const double Ox = 0.5 * (sg1 * a1 + sg2 * a2p - sg4 * a4p - 1.0);
        const double Oy = 0.5 * (sg2 * a2p + sg3 * a3 + sg4 * a4p - 3.0);
        const double mxd = floor(Ox + 0.5), myd = floor(Oy + 0.5);
        const double fx = Ox - mxd, fy = Oy - myd;
        const int cx = bx + (int)mxd, cy = by + (int)myd;
        if (cx < 1 || cx > Wp - 2 || cy < 1 || cy > Hp - 2) {
            bad = true;
            continue;
        }
        double X, Y;
        int se, sf;
        {
            const double d1 = fx - fy, d2 = fx + fy;
            if (d2 >= 0) {
                if (d1 >= 0) { X = fx;  Y = fy;  se = 1;      sf = pitch; }
                else         { X = fy;  Y = -fx; se = pitch;  sf = -1;    }
            } else {
                if (d1 >= 0) { X = -fy; Y = fx;  se = -pitch; sf = 1;     }
                else         { X = -fx; Y = -fy; se = -1;     sf = -pitch; }
            }
        }
        const double* c = G + (size_t)cy * pitch + cx;
        const double g00 = c[0], gW = c[-se], gE = c[se], gS = c[-sf], gN = c[sf], gSE = c[se - sf],
                     gNE = c[se + sf];
        const double u = gS + gN, t = gSE + gNE;
        const double K1 = 4.0 * g00 + gW + gE + u;
        const double kx = gE - gW, ky = gN - gS;
        const double kxx = 2.0 * (gW - g00) - u + t;
        const double kxy = gS - gN - gSE + gNE;
        const double kyy = t + u - 2.0 * (g00 + gE);
        const double F = 0.125 * K1 + 0.5 * (kx * X + ky * Y) + 0.25 * ((kxx * X + 2.0 * kxy * Y) * X + kyy * Y * Y);
        S += (sg1 * sg2 * sg3 * sg4) * F;
    }
    if (bad) {
        raise_status(status, BSF_EHALO);
        *o = __int_as_float(0x7fc00000);
        return;
    }
    *o = (float)(S / (a1 * a2p * a3 * a4p));
}

__global__ void k_map4(const float* __restrict__ params, int kind, long long npix, float eps, float eta,
                       float* __restrict__ scales, uint8_t* __restrict__ flags) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const map4_result R = map4_solve(kind, params[p], params[npix + p], params[2 * npix + p], eps, eta);
#pragma unroll
    for (int k = 0; k < 4; ++k) scales[k * npix + p] = R.a[k];
    if (flags) flags[p] = (uint8_t)R.flag;
}

// largest footprint extent max(a1 + a2' + a4', a2' + a3 + a4') over a field
__global__ void k_extent4(const float* __restrict__ params, int kind, long long npix, float eps, float eta,
                          unsigned* __restrict__ ext_bits) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float e = 0.f;
    if (p < npix) {
        float a[4];
        if (kind == BSF_PARAM_SCALES) {
            for (int k = 0; k < 4; ++k) a[k] = params[k * npix + p];
        } else {
            const map4_result R = map4_solve(kind, params[p], params[npix + p], params[2 * npix + p], eps, eta);
            for (int k = 0; k < 4; ++k) a[k] = R.a[k];
        }
        const float a2p = a[1] * 0.70710678f, a4p = a[3] * 0.70710678f;
        e = fmaxf(a[0] + a2p + a4p, a2p + a[2] + a4p);
        if (!(e < 1e30f)) e = 0.f;  // invalid pixels are reported by the filter itself
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) e = fmaxf(e, __shfl_xor_sync(0xffffffffu, e, d));
    if ((threadIdx.x & 31) == 0 && e > 0.f) atomicMax(ext_bits, __float_as_uint(e));
}

}  // namespace

template <int MODE, int KIND>
static void launch_exact(const stencil_args& a, cudaStream_t st) {
    const int ws = a.Ws > 0 ? a.Ws : a.W;
    constexpr int R = stencil_shape<MODE>::ROWS;
    dim3 blk(32, R), grd((ws + 31) / 32, (a.H + R - 1) / R, a.nimg);
    k_stencil4_exact<MODE, KIND><<<grd, blk, 0, st>>>(a.buf, a.buf_stride, a.Hp, a.Wp, a.pitch, a.P, a.H, a.W, a.C,
                                                      a.col0, min(a.col0 + ws, a.W), a.params, a.eps, a.eta, a.ascale,
                                                      a.out, a.status);
}

typedef CUresult (*encode_tiled_fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, looked up once through the runtime (no link against the driver library)
static encode_tiled_fn tensor_map_encoder() {
    static encode_tiled_fn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return (encode_tiled_fn)f;
    }();
    return fn;
}

// the staged form needs 16-byte aligned rows and images for its tensor map
static bool tma_usable(const stencil_args& a) {
    return tensor_map_encoder() != nullptr && ((uintptr_t)a.buf % 16) == 0 && (a.pitch % 2) == 0 &&
           (a.buf_stride % 2) == 0;
}

template <int KIND>
static cudaError_t launch_tma(const stencil_args& a, cudaStream_t st) {
    const int ws = a.Ws > 0 ? a.Ws : a.W;
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)a.Wp, (cuuint64_t)a.Hp, (cuuint64_t)a.nimg};
    const cuuint64_t strides[2] = {(cuuint64_t)a.pitch * 8, (cuuint64_t)a.buf_stride * 8};
    const cuuint32_t boxd[3] = {TMA_BW, TMA_BH, 1}, estr[3] = {1, 1, 1};
    if (tensor_map_encoder()(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void*>(a.buf), dims, strides, boxd,
                             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    // the attribute is per device: set on every launch (a cheap host call, always the same value)
    const cudaError_t e =
        cudaFuncSetAttribute(k_stencil4_tma<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TMA_SMEM);
    if (e != cudaSuccess) return e;
    dim3 blk(32, TMA_ROWS), grd((ws + 31) / 32, (a.H + TMA_ROWS - 1) / TMA_ROWS, a.nimg);
    k_stencil4_tma<KIND><<<grd, blk, TMA_SMEM, st>>>(map, (const unsigned long long*)a.buf, a.buf_stride, a.Hp, a.Wp,
                                                     a.pitch, a.P, a.H, a.W, a.C, a.col0, min(a.col0 + ws, a.W),
                                                     a.params, a.eps, a.eta, a.ascale, a.out, a.status,
                                                     a.polls ? a.polls : (1u << 22));
    return cudaGetLastError();
}

template <int KIND>
static void launch_f64(const stencil_args& a, cudaStream_t st) {
    const int ws = a.Ws > 0 ? a.Ws : a.W;
    dim3 blk(32, 8), grd((ws + 31) / 32, (a.H + 7) / 8, a.nimg);
    k_stencil4_f64<KIND><<<grd, blk, 0, st>>>((const double*)a.buf, a.buf_stride, a.Hp, a.Wp, a.pitch, a.P, a.H,
                                              a.W, a.C, a.col0, min(a.col0 + ws, a.W), a.params, a.eps, a.eta,
                                              a.ascale, a.out, a.status);
}

template <int MODE>
static void launch_mode(const stencil_args& a, cudaStream_t st) {
    if constexpr (MODE == MODE_F64) {
        if (a.kind == BSF_PARAM_SCALES) launch_f64<BSF_PARAM_SCALES>(a, st);
        else if (a.kind == BSF_PARAM_COV) launch_f64<BSF_PARAM_COV>(a, st);
        else launch_f64<BSF_PARAM_SRT>(a, st);
    } else {
        if (a.kind == BSF_PARAM_SCALES) launch_exact<MODE, BSF_PARAM_SCALES>(a, st);
        else if (a.kind == BSF_PARAM_COV) launch_exact<MODE, BSF_PARAM_COV>(a, st);
        else launch_exact<MODE, BSF_PARAM_SRT>(a, st);
    }
}

cudaError_t launch_stencil4(int mode, const stencil_args& a, cudaStream_t st) {
    if (mode == MODE_U64 && a.staging == BSF_STAGING_TMA && tma_usable(a)) {
        if (a.kind == BSF_PARAM_SCALES) return launch_tma<BSF_PARAM_SCALES>(a, st);
        if (a.kind == BSF_PARAM_COV) return launch_tma<BSF_PARAM_COV>(a, st);
        return launch_tma<BSF_PARAM_SRT>(a, st);
    }
    if (mode == MODE_U64) launch_mode<MODE_U64>(a, st);
    else if (mode == MODE_U128) launch_mode<MODE_U128>(a, st);
    else launch_mode<MODE_F64>(a, st);
    return cudaGetLastError();
}

cudaError_t launch_map4(const float* params, int kind, long long npix, float eps, float eta, float* scales,
                        uint8_t* flags, cudaStream_t st) {
    if (npix <= 0) return cudaSuccess;
    k_map4<<<(unsigned)((npix + 255) / 256), 256, 0, st>>>(params, kind, npix, eps, eta, scales, flags);
    return cudaGetLastError();
}

cudaError_t launch_extent4(const float* params, int kind, long long npix, float eps, float eta, unsigned* ext_bits,
                           cudaStream_t st) {
    if (npix <= 0) return cudaSuccess;
    k_extent4<<<(unsigned)((npix + 255) / 256), 256, 0, st>>>(params, kind, npix, eps, eta, ext_bits);
    return cudaGetLastError();
}
