// Adjoint of the four-directional filter: gradients of L with respect to the
// scale field a and to the image f, given g = dL/dfbar.  The paper has no
// backward pass; it is derived here from the forward path of Algorithm 1.
//
// With the exact integer form of the forward pass (stencil4.cu),
//   fbar[n] = (1/P) sum_i s_i F(y_i),  P = a1 a2' a3 a4',
//   y_i = n + ((s1 a1 + s2 a2' - s4 a4' - 1)/2, (s2 a2' + s3 a3 + s4 a4' - 3)/2),
// with s_k = 1 - 2 q_k (Table 1).  Hence
//   dfbar/da_k = (1/P) sum_i s_i grad F(y_i) . dy_i/da_k - fbar / a_k,
// dy_i/da1 = (s1/2, 0), dy_i/da2 = (s2, s2)/(2 sqrt2), dy_i/da3 = (0, s3/2),
// dy_i/da4 = (-s4, s4)/(2 sqrt2).  grad F is the derivative of the cell's
// quadratic-plus-truncated-powers form, an integer combination of G like F
// itself, so the four sums are evaluated exactly modulo 2^64 / 2^128 with the
// same per-pixel dyadic scales as the forward pass: the gradient is that of
// the function the forward pass computes.
//
// dL/df = M^T S^T g: S^T scatters g[n] s_i / P times the nine ZP weights of
// every tap into an FP64 buffer (the weights are exact integers below 2^53;
// each product is assembled from integers, so the scatter does no FP64
// arithmetic on the SM), and M^T is the transpose of the four running sums,
// applied in the reverse order RS4^T, RS3^T, RS2^T, RS1^T: suffix sums along
// (-1,1), (0,1), (1,1) and (1,0), each stopping at the buffer edge (the exact
// transpose of the finite-buffer recursions).  The scattered weights of one
// pixel form a fourth-order difference, so after every suffix sum its share
// stays compact; the rounding of the scattered values is what the sums carry
// along (measured: 5e-8 normwise on a 2048 x 2048 image).
//
// The scale gradient (k_grad_scales) and the scatter (k_grad_scatter) are
// separate kernels: the first reads the pre-integrated buffer and is integer
// bound, the second reads none of it and is bound by the L2 atomics.
#include "bsf_common.cuh"
#include "bsf_internal.h"

namespace {

__device__ __forceinline__ int ilog2_ceil_g(float v) {
    int e;
    const float m = frexpf(v, &e);
    return (m == 0.5f) ? e - 1 : e;
}

template <class T> __device__ __forceinline__ T mulu(T v, unsigned s) { return v * (T)s; }

template <int MODE> __device__ __forceinline__ float to_float_s(typename mode_traits<MODE>::T v);
template <> __device__ __forceinline__ float to_float_s<MODE_U64>(unsigned long long v) {
    return __ll2float_rn((long long)v);
}
template <> __device__ __forceinline__ float to_float_s<MODE_U128>(u128 v) { return i128_to_float(v); }

// The per-pixel dyadic scales of the forward pass (the same arithmetic as the
// exact stencil): q and A_k = round(a'_k 2^q).  Returns false for a pixel the
// forward pass rejects (invalid scale or q < 0).
template <int MODE>
__device__ __forceinline__ bool grad_scales_of(float a1, float a2, float a3, float a4, int& q, int& A1, int& A2,
                                               int& A3, int& A4, unsigned* status) {
    constexpr int ACC = mode_traits<MODE>::ACC_BITS;
    constexpr int VAL = mode_traits<MODE>::VAL_BITS;
    if (!(a1 > 0.f && a2 > 0.f && a3 > 0.f && a4 > 0.f) || !(a1 < 1e30f && a2 < 1e30f && a3 < 1e30f && a4 < 1e30f)) {
        raise_status(status, BSF_EBADSCALE);
        return false;
    }
    const float a2p = a2 * 0.70710678118654752f, a4p = a4 * 0.70710678118654752f;
    const float Bm = fminf((a1 + 1.f) * (a3 + 1.f) * a2p * a4p, 0.5f * a1 * a3 * (2.f * a2p + 1.f) * (a4p + 1.f));
    q = (ACC - 6 - VAL - ilog2_ceil_g(Bm)) >> 1;
    q = min(q, 24);
    q = min(q, 30 - ilog2_ceil_g(a1 + a2p + a3 + a4p + 3.f));
    const float sc = ldexpf(1.f, q);
    A1 = __float2int_rn(a1 * sc);
    A2 = __float2int_rn(a2p * sc);
    A3 = __float2int_rn(a3 * sc);
    A4 = __float2int_rn(a4p * sc);
    if (q < 0 || A1 < 1 || A2 < 1 || A3 < 1 || A4 < 1) {
        raise_status(status, BSF_ERANGE);
        return false;
    }
    return true;
}

// Whether the 3x3 neighbourhoods of all 16 tap cells lie in the buffer: the tap
// offsets range over tx in [-(A1+A2+A4), A1+A2+A4] and ty in
// [-(A2+A3+A4), A2+A3+A4] - 2^(q+1), and each extreme is reached by a tap.
__device__ __forceinline__ bool taps_inside(int bx, int by, int q, int A1, int A2, int A3, int A4, int Wp, int Hp) {
    const int sh1 = q + 1, two = 2 << q;
    const int ex = A1 + A2 + A4, ey = A2 + A3 + A4;
    return (bx + ((-ex) >> sh1) >= 1) & (bx + (ex >> sh1) <= Wp - 2) & (by + ((-ey - two) >> sh1) >= 1) &
           (by + ((ey - two) >> sh1) <= Hp - 2);
}

// Scale gradient.  Per pixel and channel image, the exact integer sums
// S = 2^(2q+4) sum_i s_i F(y_i) and E_k = sum_i s_i 2^(2q+4) grad F(y_i) . dy_i/da_k
// (up to the factor relating X to the tap position), then
//   dfbar/da_k = E_k 2^(3q-4-frac)/prod(A) (times 1/sqrt2 for k = 2, 4) - fbar/a_k,
// multiplied by g and summed over the channels that share the field.
template <int MODE>
__global__ void __launch_bounds__(256, 2) k_grad_scales(const void* __restrict__ buf, long long buf_stride, int Hp,
                                                        int Wp, int pitch, int P, int H, int W, int C,
                                                        const float* __restrict__ scales,
                                                        const float* __restrict__ gout, float* __restrict__ gscales,
                                                        float ascale, unsigned* status) {
    typedef typename mode_traits<MODE>::T T;
    constexpr int FRAC = mode_traits<MODE>::FRAC_BITS;
    const int n1 = blockIdx.x * 32 + threadIdx.x;
    const int n2 = blockIdx.y * 8 + threadIdx.y;
    const int im = blockIdx.z;
    if (n1 >= W || n2 >= H) return;
    const size_t HW = (size_t)H * W, p = (size_t)n2 * W + n1;
    const float* pr = scales + (size_t)(im / C) * 4 * HW;
    const float a1 = pr[p] * ascale, a2 = pr[HW + p] * ascale, a3 = pr[2 * HW + p] * ascale,
                a4 = pr[3 * HW + p] * ascale;
    const float gv = gout[(size_t)im * HW + p] * ascale;  // d/da = ascale d/d(a ascale)
    float* gs = gscales + (size_t)(im / C) * 4 * HW + p;
    const float qnan = __int_as_float(0x7fc00000);
    int q, A1, A2, A3, A4;
    if (!grad_scales_of<MODE>(a1, a2, a3, a4, q, A1, A2, A3, A4, status)) {
        for (int k = 0; k < 4; ++k) atomicAdd(gs + k * HW, qnan);
        return;
    }
    const int bx = n1 + P, by = n2 + P;
    if (!taps_inside(bx, by, q, A1, A2, A3, A4, Wp, Hp)) {
        raise_status(status, BSF_EHALO);
        for (int k = 0; k < 4; ++k) atomicAdd(gs + k * HW, qnan);
        return;
    }
    const int sh1 = q + 1, two = 2 << q, mask = two - 1;
    const T* G = (const T*)buf + (size_t)im * buf_stride;
    T SK = T(0), SL = T(0), SQ = T(0), E1 = T(0), E2 = T(0), E3 = T(0), E4 = T(0);
#pragma unroll 4
    for (int i = 0; i < 16; ++i) {
        const int sg1 = (i & 1) ? -1 : 1, sg2 = (i & 2) ? -1 : 1, sg3 = (i & 4) ? -1 : 1, sg4 = (i & 8) ? -1 : 1;
        const int sgn = sg1 * sg2 * sg3 * sg4;
        const int tx = sg1 * A1 + sg2 * A2 - sg4 * A4;
        const int ty = sg2 * A2 + sg3 * A3 + sg4 * A4 - two;
        const int mx = tx >> sh1, my = ty >> sh1;
        const unsigned X = (unsigned)(tx & mask), Y = (unsigned)(ty & mask);
        const unsigned T1 = (unsigned)max((int)X - (int)Y, 0), T2 = (unsigned)max((int)(X + Y) - two, 0);
        const T* r0 = G + ((size_t)(by + my - 1) * pitch + (bx + mx));
        const T* r1 = r0 + pitch;
        const T* r2 = r1 + pitch;
        const T a = r0[-1], b = r0[0], c = r0[1];
        const T d = r1[-1], e = r1[0], f = r1[1];
        const T g = r2[-1], h = r2[0], ii = r2[1];
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
        const T px = mulu(cxx, X) + mulu(m, Y), py = mulu(m, X) + mulu(cyy, Y);
        const T pa = mulu(Ac, T1), pb = mulu(Bc, T2);
        const T sl = mulu(cxl, X) + mulu(cyl, Y);
        const T sq = mulu(px, X) + mulu(py, Y) + mulu(pa, T1) + mulu(pb, T2);
        // 2^(2q+4) dF/dX and dF/dY, up to the factor 2^(q+3) relating X to phi
        const T gX = (cxl << sh1) + ((px + pa + pb) << 1);
        const T gY = (cyl << sh1) + ((py - pa + pb) << 1);
        if (sgn > 0) { SK += sk; SL += sl; SQ += sq; } else { SK -= sk; SL -= sl; SQ -= sq; }
        const T dE1 = gX, dE3 = gY, dE2 = gX + gY, dE4 = gY - gX;
        if (sgn * sg1 > 0) E1 += dE1; else E1 -= dE1;
        if (sgn * sg2 > 0) E2 += dE2; else E2 -= dE2;
        if (sgn * sg3 > 0) E3 += dE3; else E3 -= dE3;
        if (sgn * sg4 > 0) E4 += dE4; else E4 -= dE4;
    }
    const T S = (SK << (2 * q + 2)) + (SL << (q + 1)) + SQ;
    const float sc = ldexpf(1.f, q);
    const float prodA = ((float)A1 * (float)A2) * ((float)A3 * (float)A4);
    const float fbar = ldexpf(__fdividef(to_float_s<MODE>(S), prodA), 2 * q - 4 - FRAC);
    const float ek = ldexpf(1.f, 3 * q - 4 - FRAC) / prodA;
    const float isq2 = 0.70710678118654752f;
    const float d1 = to_float_s<MODE>(E1) * ek - fbar * sc / (float)A1;
    const float d2 = to_float_s<MODE>(E2) * ek * isq2 - fbar * sc * isq2 / (float)A2;
    const float d3 = to_float_s<MODE>(E3) * ek - fbar * sc / (float)A3;
    const float d4 = to_float_s<MODE>(E4) * ek * isq2 - fbar * sc * isq2 / (float)A4;
    atomicAdd(gs, gv * d1);
    atomicAdd(gs + HW, gv * d2);
    atomicAdd(gs + 2 * HW, gv * d3);
    atomicAdd(gs + 3 * HW, gv * d4);
}

// The double nearest below |c w| for c = mc 2^ec (mc the 24-bit significand of
// a float) and an integer 0 < w < 2^53, with the given sign bit, built from the
// exact integer product (the 52 bits after the leading one are kept, the rest
// truncated): the FP64 scatter needs no FP64 arithmetic on the SM.
__device__ __forceinline__ double scaled_weight(unsigned mc, int ec, unsigned long long sgnbit, unsigned long long w) {
    const unsigned __int128 Pr = (unsigned __int128)w * mc;  // < 2^77
    const unsigned long long hi = (unsigned long long)(Pr >> 64), lo = (unsigned long long)Pr;
    const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
    const unsigned long long top = (unsigned long long)((Pr << lz) >> 64);  // leading one at bit 63
    const int E = 127 - lz + ec + 1023;
    if (E <= 0) return 0.0;  // below the normal range: negligible
    return __longlong_as_double((long long)(sgnbit | ((unsigned long long)E << 52) | ((top >> 11) & 0xFFFFFFFFFFFFFull)));
}

// Image gradient, first half: S^T g.  Every tap of every pixel scatters
// g[n] s_i / P~ times its nine ZP weights (exact integers below 2^(2q+4)) into
// an FP64 buffer of the padded size.  The per-pixel factor c = g 2^(2q-4)/prod(A)
// is rounded to float once (a relative scaling of the pixel's whole pattern,
// which keeps it an exact finite difference), and each product c w is formed
// from integers (scaled_weight).
template <int MODE>
__global__ void __launch_bounds__(256) k_grad_scatter(int Hp, int Wp, int pitch, int P, int H, int W, int C,
                                                      const float* __restrict__ scales, const float* __restrict__ gout,
                                                      double* __restrict__ hbuf, float ascale, unsigned* status) {
    const int n1 = blockIdx.x * 32 + threadIdx.x;
    const int n2 = blockIdx.y * 8 + threadIdx.y;
    const int im = blockIdx.z;
    if (n1 >= W || n2 >= H) return;
    const size_t HW = (size_t)H * W, p = (size_t)n2 * W + n1;
    const float* pr = scales + (size_t)(im / C) * 4 * HW;
    const float gv = gout[(size_t)im * HW + p];
    int q, A1, A2, A3, A4;
    if (!grad_scales_of<MODE>(pr[p] * ascale, pr[HW + p] * ascale, pr[2 * HW + p] * ascale, pr[3 * HW + p] * ascale, q,
                              A1, A2, A3, A4, status))
        return;
    const int bx = n1 + P, by = n2 + P;
    if (!taps_inside(bx, by, q, A1, A2, A3, A4, Wp, Hp)) {
        raise_status(status, BSF_EHALO);
        return;
    }
    const float prodA = ((float)A1 * (float)A2) * ((float)A3 * (float)A4);
    const float cg = ldexpf(gv / prodA, 2 * q - 4);
    const unsigned cb = __float_as_uint(cg);
    const int ebits = (int)((cb >> 23) & 0xFF);
    if (ebits == 0 || ebits == 0xFF) return;  // g = 0 (or below the normal range), or not finite
    const unsigned mc = (cb & 0x7FFFFFu) | 0x800000u;
    const int ec = ebits - 127 - 23;
    const unsigned long long sgn0 = (unsigned long long)(cb >> 31) << 63;
    const int sh1 = q + 1, two = 2 << q, mask = two - 1;
    double* hb = hbuf + (size_t)im * ((size_t)Hp * pitch);
    const long long t = two;
#pragma unroll 2
    for (int i = 0; i < 16; ++i) {
        const int sg1 = (i & 1) ? -1 : 1, sg2 = (i & 2) ? -1 : 1, sg3 = (i & 4) ? -1 : 1, sg4 = (i & 8) ? -1 : 1;
        const unsigned long long sgnbit = (sg1 * sg2 * sg3 * sg4 > 0) ? sgn0 : (sgn0 ^ (1ull << 63));
        const int tx = sg1 * A1 + sg2 * A2 - sg4 * A4;
        const int ty = sg2 * A2 + sg3 * A3 + sg4 * A4 - two;
        const int mx = tx >> sh1, my = ty >> sh1;
        const long long X = tx & mask, Y = ty & mask;
        const long long T1 = max(X - Y, 0ll), T2 = max(X + Y - t, 0ll);
        const long long xa = max(t - X - Y, 0ll);
        const long long X2 = X * X, Y2 = Y * Y, XY = X * Y, T12 = T1 * T1, T22 = T2 * T2, tt = t * t;
        const long long tX2 = 2 * t * X, tY2 = 2 * t * Y;
        // the nine ZP weights of this tap on the cell's 3x3 neighbourhood
        const long long w[9] = {
            xa * xa,                                              // (-1,-1)
            tt + tX2 - tY2 - X2 - 2 * XY + Y2 + T22 - T12,         // ( 0,-1)
            T12,                                                  // ( 1,-1)
            tt - tX2 + tY2 - 2 * Y2 + T12 + T22,                  // (-1, 0)
            tt + tX2 + tY2 - 2 * X2 - 2 * Y2,                     // ( 0, 0)
            2 * X2 - T12 - T22,                                   // ( 1, 0)
            X2 - 2 * XY + Y2 - T12,                               // (-1, 1)
            -X2 + 2 * XY + Y2 + T12 - T22,                        // ( 0, 1)
            T22};                                                 // ( 1, 1)
        double* h0 = hb + ((size_t)(by + my - 1) * pitch + (bx + mx));
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            if (w[k] == 0) continue;
            atomicAdd(h0 + (k / 3) * pitch + (k % 3) - 1, scaled_weight(mc, ec, sgnbit, (unsigned long long)w[k]));
        }
    }
}

// Transposed running sums.  Each is a suffix sum along a lattice direction d,
// out[p] = sum_{j >= 0} in[p + j d], stopping at the buffer edge (the exact
// transpose of the finite-buffer recursions), in place on nimg FP64 buffers.
//
// Directions (dx, 1): one thread per line, neighbouring threads on
// neighbouring lines, so every row is read and written coalesced; each
// thread walks its line from the bottom row up, with the loads of the next
// kChunk rows issued before the running sum consumes them.  One FP64 add per
// element.
constexpr int kChunk = 32;

__global__ void __launch_bounds__(128) k_suffix_lines(double* __restrict__ X, long long stride, int Hp, int Wp,
                                                      int pitch, int dx) {
    const int im = blockIdx.y;
    const int k = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    // line k holds the cells (x, y) with x = k + dx * y - off, off = (dx < 0 ? 0 : dx * (Hp - 1))
    const int off = dx > 0 ? Hp - 1 : 0;
    const int nlines = dx == 0 ? Wp : Wp + Hp - 1;
    if (k >= nlines) return;
    double* base = X + (size_t)im * stride;
    // x at row y: dx = 0: k;  dx = 1: k - off + y;  dx = -1: k - y
    auto xat = [&](int y) { return dx == 0 ? k : (dx > 0 ? k - off + y : k - y); };
    double run = 0.0;
    for (int y1 = Hp - 1; y1 >= 0; y1 -= kChunk) {
        double v[kChunk];
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
            const int y = y1 - j, x = xat(y);
            v[j] = (y >= 0 && x >= 0 && x < Wp) ? base[(size_t)y * pitch + x] : 0.0;
        }
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
            const int y = y1 - j, x = xat(y);
            run += v[j];
            if (y >= 0 && x >= 0 && x < Wp) base[(size_t)y * pitch + x] = run;
        }
    }
}

// Direction (1, 0), the last transpose: one warp per row, each lane owning a
// contiguous segment of it: local suffix sums, a warp scan of the segment
// totals, then the carry; the image window [P, P+H) x [P, P+W) of the result
// is written to out as float.
__global__ void __launch_bounds__(256) k_suffix_rows(const double* __restrict__ X, long long stride, int Hp, int Wp,
                                                     int pitch, float* __restrict__ out, int P, int H, int W) {
    const int im = blockIdx.y;
    const int y = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (y < P || y >= P + H) return;  // only image rows reach the output
    const double* row = X + (size_t)im * stride + (size_t)y * pitch;
    const int seg = (Wp + 31) / 32, x0 = lane * seg, x1 = min(Wp, x0 + seg);
    double tot = 0.0;
    for (int x = x0; x < x1; ++x) tot += row[x];
    // suffix over the lanes after this one
    double after = tot;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const double o = __shfl_down_sync(0xffffffffu, after, d);
        if (lane + d < 32) after += o;
    }
    double run = after - tot;  // sum of the segments to the right
    float* o = out + (size_t)im * H * W + (size_t)(y - P) * W;
    for (int x = x1 - 1; x >= x0; --x) {
        run += row[x];
        const int xx = x - P;
        if (xx >= 0 && xx < W) o[xx] = (float)run;
    }
}

}  // namespace

cudaError_t launch_grad4(int mode, const void* buf, long long buf_stride, int Hp, int Wp, int pitch, int P, int H,
                         int W, int C, int nimg, const float* scales, const float* gout, float* gscales, double* hbuf,
                         float ascale, unsigned* status, cudaStream_t st) {
    if (mode != MODE_U64 && mode != MODE_U128) return cudaErrorInvalidValue;
    dim3 blk(32, 8), grd((W + 31) / 32, (H + 7) / 8, nimg);
    if (gscales != nullptr) {
        if (mode == MODE_U64)
            k_grad_scales<MODE_U64><<<grd, blk, 0, st>>>(buf, buf_stride, Hp, Wp, pitch, P, H, W, C, scales, gout,
                                                          gscales, ascale, status);
        else
            k_grad_scales<MODE_U128><<<grd, blk, 0, st>>>(buf, buf_stride, Hp, Wp, pitch, P, H, W, C, scales, gout,
                                                           gscales, ascale, status);
    }
    if (hbuf != nullptr) {
        if (mode == MODE_U64)
            k_grad_scatter<MODE_U64><<<grd, blk, 0, st>>>(Hp, Wp, pitch, P, H, W, C, scales, gout, hbuf, ascale,
                                                           status);
        else
            k_grad_scatter<MODE_U128><<<grd, blk, 0, st>>>(Hp, Wp, pitch, P, H, W, C, scales, gout, hbuf, ascale,
                                                            status);
    }
    return cudaGetLastError();
}

cudaError_t launch_transpose_scans(double* hbuf, int nimg, int Hp, int Wp, int pitch, int P, int H, int W,
                                   float* gimage, cudaStream_t st) {
    const long long stride = (long long)Hp * pitch;
    const int dxs[3] = {-1, 0, 1};  // RS4^T, RS3^T, RS2^T; then RS1^T along the rows
    for (int k = 0; k < 3; ++k) {
        const int nlines = dxs[k] == 0 ? Wp : Wp + Hp - 1;
        k_suffix_lines<<<dim3((unsigned)((nlines + 127) / 128), nimg), 128, 0, st>>>(hbuf, stride, Hp, Wp, pitch,
                                                                                    dxs[k]);
    }
    k_suffix_rows<<<dim3((unsigned)((Hp + 7) / 8), nimg), 256, 0, st>>>(hbuf, stride, Hp, Wp, pitch, gimage, P, H, W);
    return cudaGetLastError();
}
