// Pre-integration for the four-directional box spline (Algorithm 1 step 2,
// recursions RS1-RS4 of Sec. 3.1), on a zero-padded buffer of Hp x Wp
// elements, every running sum started from zero at the buffer edge:
//
//   g0[x,y] = f[x,y] + g0[x-1,y]        (RS1, along (1,0))
//   g1[x,y] = g0[x,y] + g1[x-1,y-1]     (RS2, along (1,1); sqrt2 taken out)
//   g2[x,y] = g1[x,y] + g2[x,y-1]       (RS3, along (0,1))
//   G [x,y] = g2[x,y] + G [x+1,y-1]     (RS4, along (-1,1); sqrt2 taken out)
//
// so that g_b = 2 G.  In the integer forms every sum wraps modulo 2^64 or
// 2^128, which leaves any later integer combination exact modulo the same.
//
// GPU design (one sweep, HBM traffic = read f twice + write G once):
//   Phase 1  k_band (local mode): the padded rows are cut into bands of
//            band_h rows.  Each CTA owns one band over the full width and
//            runs the recursions row by row from a zero state (block-wide
//            prefix scan for RS1, register/shuffle neighbour exchange for
//            RS2-RS4).  It stores only the band's final state (g1,g2,G) of
//            its last row: L_b.
//   Phase 2  the true state S_b at the last row of every band follows from
//            S_b = L_b + T_{h_b}(S_{b-1}), T_h being the zero-input
//            response of the recursions over h rows.  T_h has a closed form
//            in prefix sums along the row (P1, PP1, Q1 of g1 and P2 of g2),
//            so S_b is resolved line by line: a diagonal recursion for g1, a
//            vertical one for g2 and an anti-diagonal one for G, each
//            sequential over bands and parallel over lines.
//   Phase 3  k_band (write mode): each CTA restarts its band from the true
//            carry-in S_{b-1} and writes G.
#include "bsf_common.cuh"
#include "bsf_internal.h"

namespace {

template <class T> __device__ __forceinline__ T warp_incl_scan(T v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = shfl_up_T(v, d);
        if (lane >= d) v += o;
    }
    return v;
}

template <int MODE> struct band_bounds { static constexpr int MAXT = (MODE == MODE_U128) ? 512 : 1024; };

template <int MODE, class InT, int CPT>
__global__ void __launch_bounds__(band_bounds<MODE>::MAXT) k_band(const InT* __restrict__ img, long long img_stride, int H, int W,
                                               int P, int Hp, int Wp, int pitch, int band_h, int nb,
                                               const typename mode_traits<MODE>::T* __restrict__ carry,
                                               typename mode_traits<MODE>::T* __restrict__ local,
                                               typename mode_traits<MODE>::T* __restrict__ G, long long G_stride) {
    typedef typename mode_traits<MODE>::T T;
    const int b = blockIdx.x, im = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int c0 = tid * CPT;
    const int y0 = b * band_h, y1 = min(Hp, y0 + band_h);
    __shared__ T s_tot[32];
    __shared__ T s_off[32];
    __shared__ T s_eg1[2][32];
    __shared__ T s_eG[2][32];
    // the vertical sum g2 is column-local: it lives in shared memory, one
    // slot per column, touched only by the thread that owns the column
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* g2 = reinterpret_cast<T*>(smem_raw) + c0;

    T g1[CPT], gG[CPT];
    if (carry != nullptr && b > 0) {
        const T* S = carry + ((size_t)im * nb + (b - 1)) * 3 * (size_t)Wp;
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            const int c = c0 + j;
            g1[j] = c < Wp ? S[c] : T(0);
            g2[j] = c < Wp ? S[Wp + c] : T(0);
            gG[j] = c < Wp ? S[2 * Wp + c] : T(0);
        }
    } else {
#pragma unroll
        for (int j = 0; j < CPT; ++j) g1[j] = g2[j] = gG[j] = T(0);
    }

    const InT* f = img + (size_t)im * img_stride;
    // prefetch of the next row's samples
    InT nxt[CPT];
    auto fetch = [&](int y, InT* dst) {
        const int iy = y - P;
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            const int ic = c0 + j - P;
            dst[j] = (y < y1 && iy >= 0 && iy < H && ic >= 0 && ic < W) ? f[(size_t)iy * W + ic] : InT(0);
        }
    };
    fetch(y0, nxt);
    for (int y = y0; y < y1; ++y) {
        T v[CPT];
#pragma unroll
        for (int j = 0; j < CPT; ++j) v[j] = load_sample<MODE, InT>(nxt[j]);
        fetch(y + 1, nxt);
#pragma unroll
        for (int j = 1; j < CPT; ++j) v[j] += v[j - 1];
        const T tot = v[CPT - 1];
        const T inc = warp_incl_scan(tot, lane);
        const int par = y & 1;
        if (lane == 31) {
            s_tot[warp] = inc;
            s_eg1[par][warp] = g1[CPT - 1];
        }
        if (lane == 0) s_eG[par][warp] = gG[0];
        const T g1_from_left = shfl_up_T(g1[CPT - 1], 1);
        const T gG_from_right = shfl_down_T(gG[0], 1);
        __syncthreads();
        if (warp == 0) {
            const T t = lane < nw ? s_tot[lane] : T(0);
            const T ti = warp_incl_scan(t, lane);
            s_off[lane] = ti - t;
        }
        __syncthreads();
        const T off = s_off[warp] + (inc - tot);
        const T left = lane > 0 ? g1_from_left : (warp > 0 ? s_eg1[par][warp - 1] : T(0));
        const T right = lane < 31 ? gG_from_right : (warp + 1 < nw ? s_eG[par][warp + 1] : T(0));
        T ng1[CPT];
#pragma unroll
        for (int j = 0; j < CPT; ++j) ng1[j] = (v[j] + off) + (j == 0 ? left : g1[j - 1]);
#pragma unroll
        for (int j = 0; j < CPT; ++j) g2[j] += ng1[j];
        T ngG[CPT];
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            T nb_ = (j + 1 < CPT) ? gG[j + 1] : right;
            if (c0 + j + 1 >= Wp) nb_ = T(0);
            ngG[j] = g2[j] + nb_;
        }
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            g1[j] = ng1[j];
            gG[j] = ngG[j];
        }
        if (G != nullptr) {
            T* row = G + (size_t)im * G_stride + (size_t)y * pitch;
#pragma unroll
            for (int j = 0; j < CPT; ++j)
                if (c0 + j < Wp) row[c0 + j] = gG[j];
        }
    }
    if (local != nullptr) {
        T* L = local + ((size_t)im * nb + b) * 3 * (size_t)Wp;
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            const int c = c0 + j;
            if (c < Wp) {
                L[c] = g1[j];
                L[Wp + c] = g2[j];
                L[2 * Wp + c] = gG[j];
            }
        }
    }
}

__device__ __forceinline__ int band_last_row(int b, int band_h, int Hp) { return min((b + 1) * band_h, Hp) - 1; }

// Phase 2a: S1_b[x] = L1_b[x] + S1_{b-1}[x - h_b]  (diagonal lines)
template <class T>
__global__ void k_carry_s1(const T* __restrict__ L, T* __restrict__ S, int Hp, int Wp, int band_h, int nb) {
    const int im = blockIdx.y;
    const int Ylast = Hp - 1, Y0 = band_last_row(0, band_h, Hp);
    const int X = blockIdx.x * blockDim.x + threadIdx.x;
    if (X >= Wp + (Ylast - Y0)) return;
    T run = T(0);
    for (int b = 0; b < nb; ++b) {
        const int x = X - (Ylast - band_last_row(b, band_h, Hp));
        if (x >= Wp) break;
        if (x < 0) continue;
        const size_t base = ((size_t)im * nb + b) * 3 * (size_t)Wp;
        const T val = L[base + x] + run;
        S[base + x] = val;
        run = val;
    }
}

template <class T> __device__ __forceinline__ T at0(const T* a, int i) { return i >= 0 ? a[i] : T(0); }

// Phase 2c: S2_b[x] = L2_b[x] + S2_{b-1}[x] + sum_{j=1..h_b} S1_{b-1}[x-j]  (columns)
template <class T>
__global__ void k_carry_s2(const T* __restrict__ L, T* __restrict__ S, const T* __restrict__ P1, int Hp, int Wp,
                           int band_h, int nb) {
    const int im = blockIdx.y;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= Wp) return;
    T run = T(0);
    for (int b = 0; b < nb; ++b) {
        const size_t base = ((size_t)im * nb + b) * 3 * (size_t)Wp;
        T val = L[base + Wp + x] + run;
        if (b > 0) {
            const int h = band_last_row(b, band_h, Hp) - band_last_row(b - 1, band_h, Hp);
            const T* p1 = P1 + ((size_t)im * nb + (b - 1)) * (size_t)Wp;
            val += at0(p1, x - 1) - at0(p1, x - h - 1);
        }
        S[base + Wp + x] = val;
        run = val;
    }
}

// Phase 2e: SG_b[x] = LG_b[x] + [x+h <= Wp-1] SG_{b-1}[x+h]
//          + sum_{j=j0..h} ( S2_{b-1}[x+h-j] + sum_{k=1..j} S1_{b-1}[x+h-j-k] ),
//   j0 = max(1, x+h-Wp+1)  (RS4 truncated at the right buffer edge)   (anti-diagonal lines)
template <class T>
__global__ void k_carry_sg(const T* __restrict__ L, T* __restrict__ S, const T* __restrict__ P1,
                           const T* __restrict__ PP1, const T* __restrict__ Q1, const T* __restrict__ P2, int Hp,
                           int Wp, int band_h, int nb) {
    const int im = blockIdx.y;
    const int Ylast = Hp - 1, Y0 = band_last_row(0, band_h, Hp);
    const int X = (int)(blockIdx.x * blockDim.x + threadIdx.x) - (Ylast - Y0);
    if (X >= Wp) return;
    T run = T(0);
    for (int b = 0; b < nb; ++b) {
        const int x = X + (Ylast - band_last_row(b, band_h, Hp));
        if (x < 0) break;
        if (x >= Wp) {
            run = T(0);
            continue;
        }
        const size_t base = ((size_t)im * nb + b) * 3 * (size_t)Wp;
        T val = L[base + 2 * Wp + x];
        if (b > 0) {
            const int h = band_last_row(b, band_h, Hp) - band_last_row(b - 1, band_h, Hp);
            const size_t pb = ((size_t)im * nb + (b - 1)) * (size_t)Wp;
            const int j0 = max(1, x + h - Wp + 1);
            if (x + h <= Wp - 1) val += run;
            val += at0(P2 + pb, x + h - j0) - at0(P2 + pb, x - 1);
            val += at0(PP1 + pb, x + h - 1 - j0) - at0(PP1 + pb, x - 2);
            val -= at0(Q1 + pb, x + h - 1 - 2 * j0) - at0(Q1 + pb, x - h - 3);
        }
        S[base + 2 * Wp + x] = val;
        run = val;
    }
}

// Inclusive prefix of get(i), i < n, along one row, by one CTA.
template <class T, class Get, class Put>
__device__ void block_row_scan(int n, Get get, Put put, T* smem /* 33 */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T carry = T(0);
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const T v = i < n ? get(i) : T(0);
        const T inc = warp_incl_scan(v, lane);
        if (lane == 31) smem[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const T t = lane < nw ? smem[lane] : T(0);
            const T ti = warp_incl_scan(t, lane);
            if (lane == nw - 1) smem[32] = ti;
            smem[lane] = ti - t;
        }
        __syncthreads();
        const T res = carry + smem[warp] + inc;
        if (i < n) put(i, res);
        carry += smem[32];
        __syncthreads();
    }
}

// Phase 2b: P1 = prefix(S1), PP1 = prefix(P1), Q1[x] = P1[x] + Q1[x-2]
template <class T>
__global__ void k_prefix1(const T* __restrict__ S, T* __restrict__ P1, T* __restrict__ PP1, T* __restrict__ Q1,
                          int Wp, int nb) {
    __shared__ T sm[33];
    const int b = blockIdx.x, im = blockIdx.y;
    const T* s1 = S + ((size_t)im * nb + b) * 3 * (size_t)Wp;
    const size_t pb = ((size_t)im * nb + b) * (size_t)Wp;
    T* p1 = P1 + pb;
    T* pp1 = PP1 + pb;
    T* q1 = Q1 + pb;
    block_row_scan<T>(Wp, [&](int i) { return s1[i]; }, [&](int i, T v) { p1[i] = v; }, sm);
    __syncthreads();
    block_row_scan<T>(Wp, [&](int i) { return p1[i]; }, [&](int i, T v) { pp1[i] = v; }, sm);
    block_row_scan<T>((Wp + 1) / 2, [&](int i) { return p1[2 * i]; }, [&](int i, T v) { q1[2 * i] = v; }, sm);
    block_row_scan<T>(Wp / 2, [&](int i) { return p1[2 * i + 1]; }, [&](int i, T v) { q1[2 * i + 1] = v; }, sm);
}

// Phase 2d: P2 = prefix(S2)
template <class T> __global__ void k_prefix2(const T* __restrict__ S, T* __restrict__ P2, int Wp, int nb) {
    __shared__ T sm[33];
    const int b = blockIdx.x, im = blockIdx.y;
    const T* s2 = S + ((size_t)im * nb + b) * 3 * (size_t)Wp + Wp;
    T* p2 = P2 + ((size_t)im * nb + b) * (size_t)Wp;
    block_row_scan<T>(Wp, [&](int i) { return s2[i]; }, [&](int i, T v) { p2[i] = v; }, sm);
}

}  // namespace

// ---------------------------------------------------------------- host side
scan_plan make_scan_plan(int Hp, int Wp, int nimg, size_t elem_bytes) {
    scan_plan p;
    // bands: about two CTAs per SM of a 152-SM part over the whole batch
    int bh = (int)((long long)Hp * nimg / 304);
    if (bh < 8) bh = 8;
    if (bh > 64) bh = 64;
    if (bh > Hp) bh = Hp;
    p.band_h = bh;
    p.nb = (Hp + bh - 1) / bh;
    const int maxt = elem_bytes > 8 ? 512 : 1024;
    p.cpt = 1;
    while (p.cpt < 8 && (Wp + p.cpt - 1) / p.cpt > maxt) p.cpt *= 2;
    p.threads = ((Wp + p.cpt - 1) / p.cpt + 31) / 32 * 32;
    p.smem = (size_t)p.threads * p.cpt * elem_bytes;
    p.ok = p.threads <= maxt;
    const size_t row = (size_t)nimg * p.nb * Wp * elem_bytes;
    p.work_bytes = row * 10;  // L (3), S (3), P1, PP1, Q1, P2
    return p;
}

template <int MODE, class InT, int CPT>
static void launch_band(const scan_plan& p, const InT* img, long long img_stride, int nimg, int H, int W, int P,
                        int Hp, int Wp, int pitch, const void* carry, void* local, void* G, long long G_stride,
                        cudaStream_t st) {
    typedef typename mode_traits<MODE>::T T;
    static bool attr_set = false;  // per instantiation: allow up to 96 KiB of g2 state
    if (!attr_set) {
        cudaFuncSetAttribute(k_band<MODE, InT, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        attr_set = true;
    }
    dim3 grid(p.nb, nimg);
    k_band<MODE, InT, CPT><<<grid, p.threads, p.smem, st>>>(img, img_stride, H, W, P, Hp, Wp, pitch, p.band_h, p.nb,
                                                        (const T*)carry, (T*)local, (T*)G, G_stride);
}

template <int MODE, class InT>
static void launch_band_cpt(const scan_plan& p, const InT* img, long long img_stride, int nimg, int H, int W, int P,
                            int Hp, int Wp, int pitch, const void* carry, void* local, void* G, long long G_stride,
                            cudaStream_t st) {
    switch (p.cpt) {
        case 1: launch_band<MODE, InT, 1>(p, img, img_stride, nimg, H, W, P, Hp, Wp, pitch, carry, local, G, G_stride, st); break;
        case 2: launch_band<MODE, InT, 2>(p, img, img_stride, nimg, H, W, P, Hp, Wp, pitch, carry, local, G, G_stride, st); break;
        case 4: launch_band<MODE, InT, 4>(p, img, img_stride, nimg, H, W, P, Hp, Wp, pitch, carry, local, G, G_stride, st); break;
        default: launch_band<MODE, InT, 8>(p, img, img_stride, nimg, H, W, P, Hp, Wp, pitch, carry, local, G, G_stride, st); break;
    }
}

template <int MODE, class InT>
cudaError_t launch_scan4(const InT* img, long long img_stride, int nimg, int H, int W, int P, void* G,
                         long long G_stride, int pitch, void* work, cudaStream_t st) {
    typedef typename mode_traits<MODE>::T T;
    const int Hp = H + 2 * P, Wp = W + 2 * P;
    const scan_plan p = make_scan_plan(Hp, Wp, nimg, sizeof(T));
    if (!p.ok) return cudaErrorInvalidValue;
    const size_t row = (size_t)nimg * p.nb * Wp;
    T* L = (T*)work;
    T* S = L + 3 * row;
    T* P1 = S + 3 * row;
    T* PP1 = P1 + row;
    T* Q1 = PP1 + row;
    T* P2 = Q1 + row;
    launch_band_cpt<MODE, InT>(p, img, img_stride, nimg, H, W, P, Hp, Wp, pitch, nullptr, L, nullptr, 0, st);
    {
        const int n = Wp + (Hp - 1 - min(p.band_h, Hp) + 1);
        dim3 g((n + 255) / 256, nimg);
        k_carry_s1<T><<<g, 256, 0, st>>>(L, S, Hp, Wp, p.band_h, p.nb);
    }
    k_prefix1<T><<<dim3(p.nb, nimg), 256, 0, st>>>(S, P1, PP1, Q1, Wp, p.nb);
    k_carry_s2<T><<<dim3((Wp + 255) / 256, nimg), 256, 0, st>>>(L, S, P1, Hp, Wp, p.band_h, p.nb);
    k_prefix2<T><<<dim3(p.nb, nimg), 256, 0, st>>>(S, P2, Wp, p.nb);
    {
        const int n = Wp + (Hp - 1 - min(p.band_h, Hp) + 1);
        dim3 g((n + 255) / 256, nimg);
        k_carry_sg<T><<<g, 256, 0, st>>>(L, S, P1, PP1, Q1, P2, Hp, Wp, p.band_h, p.nb);
    }
    launch_band_cpt<MODE, InT>(p, img, img_stride, nimg, H, W, P, Hp, Wp, pitch, S, nullptr, G, G_stride, st);
    return cudaGetLastError();
}

template cudaError_t launch_scan4<MODE_U64, uint8_t>(const uint8_t*, long long, int, int, int, int, void*, long long,
                                                     int, void*, cudaStream_t);
template cudaError_t launch_scan4<MODE_U128, float>(const float*, long long, int, int, int, int, void*, long long, int,
                                                    void*, cudaStream_t);
template cudaError_t launch_scan4<MODE_F64, uint8_t>(const uint8_t*, long long, int, int, int, int, void*, long long,
                                                     int, void*, cudaStream_t);
template cudaError_t launch_scan4<MODE_F64, float>(const float*, long long, int, int, int, int, void*, long long, int,
                                                   void*, cudaStream_t);
