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

// Threads per band CTA for each (form, columns per thread): the register
// state grows with both, so wider rows trade threads for registers.
__host__ __device__ constexpr int band_maxt(bool wide, int cpt) {
    return wide ? (cpt <= 1 ? 1024 : cpt == 2 ? 768 : cpt == 4 ? 512 : 384)
                : (cpt <= 2 ? 1024 : cpt == 4 ? 768 : 512);
}
template <int MODE, int CPT> struct band_bounds { static constexpr int MAXT = band_maxt(MODE == MODE_U128, CPT); };

template <int MODE, class InT, int CPT>
__global__ void __launch_bounds__(band_bounds<MODE, CPT>::MAXT) k_band(const InT* __restrict__ img, long long img_stride, int H, int W,
                                               int col0, int P, int Hp, int Wp, int pitch, int band_h, int nb,
                                               const typename mode_traits<MODE>::T* __restrict__ carry,
                                               typename mode_traits<MODE>::T* __restrict__ local,
                                               typename mode_traits<MODE>::T* __restrict__ G, long long G_stride,
                                               int reflect) {
    typedef typename mode_traits<MODE>::T T;
    const int b = blockIdx.x, im = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int c0 = tid * CPT;
    const int y0 = b * band_h, y1 = min(Hp, y0 + band_h);
    __shared__ T s_tot[2][32];
    __shared__ T s_eg1[2][32];
    __shared__ T s_eG[2][32];
    // the vertical sum g2 is column-local: each thread keeps its columns' states in
    // registers, except for the widest 128-bit form, whose registers would spill: there
    // they sit in shared memory (one slot per column, touched only by its thread)
    constexpr bool kG2Smem = MODE == MODE_U128 && CPT >= 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T g1[CPT], g2r[kG2Smem ? 1 : CPT], gG[CPT];
    auto g2 = [&](int j) -> T& {
        if constexpr (kG2Smem) return reinterpret_cast<T*>(smem_raw)[c0 + j];
        else return g2r[j];
    };
    if (carry != nullptr && b > 0) {
        const T* S = carry + ((size_t)im * nb + (b - 1)) * 3 * (size_t)Wp;
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            const int c = c0 + j;
            g1[j] = c < Wp ? S[c] : T(0);
            g2(j) = c < Wp ? S[Wp + c] : T(0);
            gG[j] = c < Wp ? S[2 * Wp + c] : T(0);
        }
    } else {
#pragma unroll
        for (int j = 0; j < CPT; ++j) g1[j] = g2(j) = gG[j] = T(0);
    }

    const InT* f = img + (size_t)im * img_stride;
    // samples of the next D rows are kept in flight in a register ring
    constexpr int D = 2;
    // the image columns of this thread that lie inside the image (fixed for the band)
    const int ic0 = c0 - P + col0;
    unsigned colmask = 0;
#pragma unroll
    for (int j = 0; j < CPT; ++j) colmask |= (ic0 + j >= 0 && ic0 + j < W) ? (1u << j) : 0u;
    auto fetch = [&](int y, InT* dst) {
        const int iy = y - P;
        if (reflect) {  // the symmetric extension fills the whole buffer (columns c0 + j < Wp)
#pragma unroll
            for (int j = 0; j < CPT; ++j)
                dst[j] = (y < y1 && c0 + j < Wp) ? f[(size_t)reflect_index(iy, H) * W + reflect_index(ic0 + j, W)]
                                                 : InT(0);
        } else {
            const bool rowok = y < y1 && iy >= 0 && iy < H;
            const InT* rowp = f + (size_t)(rowok ? iy : 0) * W + ic0;
#pragma unroll
            for (int j = 0; j < CPT; ++j) dst[j] = (rowok && ((colmask >> j) & 1u)) ? rowp[j] : InT(0);
        }
    };
    InT pre[D][CPT];
#pragma unroll
    for (int k = 0; k < D; ++k) fetch(y0 + k, pre[k]);
    for (int yb = y0; yb < y1; yb += D) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const int y = yb + k;
            if (y >= y1) break;  // uniform over the CTA
            T v[CPT];
#pragma unroll
            for (int j = 0; j < CPT; ++j) v[j] = load_sample<MODE, InT>(pre[k][j]);
            fetch(y + D, pre[k]);
#pragma unroll
            for (int j = 1; j < CPT; ++j) v[j] += v[j - 1];
            const T tot = v[CPT - 1];
            const T inc = warp_incl_scan(tot, lane);
            const int par = y & 1;
            if (lane == 31) {
                s_tot[par][warp] = inc;
                s_eg1[par][warp] = g1[CPT - 1];
            }
            if (lane == 0) s_eG[par][warp] = gG[0];
            const T g1_from_left = shfl_up_T(g1[CPT - 1], 1);
            const T gG_from_right = shfl_down_T(gG[0], 1);
            // one barrier per row: every warp sums the totals of the warps before it
            // (buffers alternate by row parity, so the next row cannot overwrite them early)
            __syncthreads();
            T before = lane < warp ? s_tot[par][lane] : T(0);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) before += shfl_down_T(before, d);
            const T off = shfl_idx_T(before, 0) + (inc - tot);
            const T left = lane > 0 ? g1_from_left : (warp > 0 ? s_eg1[par][warp - 1] : T(0));
            const T right = lane < 31 ? gG_from_right : (warp + 1 < nw ? s_eG[par][warp + 1] : T(0));
            T ng1[CPT];
#pragma unroll
            for (int j = 0; j < CPT; ++j) ng1[j] = (v[j] + off) + (j == 0 ? left : g1[j - 1]);
#pragma unroll
            for (int j = 0; j < CPT; ++j) g2(j) += ng1[j];
            T ngG[CPT];
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                T nb_ = (j + 1 < CPT) ? gG[j + 1] : right;
                if (c0 + j + 1 >= Wp) nb_ = T(0);
                ngG[j] = g2(j) + nb_;
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
    }
    if (local != nullptr) {
        T* L = local + ((size_t)im * nb + b) * 3 * (size_t)Wp;
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            const int c = c0 + j;
            if (c < Wp) {
                L[c] = g1[j];
                L[Wp + c] = g2(j);
                L[2 * Wp + c] = gG[j];
            }
        }
    }
}

__device__ __forceinline__ int band_last_row(int b, int band_h, int Hp) { return min((b + 1) * band_h, Hp) - 1; }

template <class T> __device__ __forceinline__ T at0(const T* a, int i) { return i >= 0 ? a[i] : T(0); }

// Phase 2 line scans.  Along every line of a family, the true band-end
// states obey S_b = v_b + S_{b-1} over the contiguous range of bands where
// the line lies inside the buffer, with v_b the band's local state plus the
// closed-form response to the previous band's lower-order states.  One warp
// owns one line; its lanes take 32 consecutive bands at a time and a warp
// prefix scan carries the running sum across the chunk.
template <class T, class GetV, class Put>
__device__ __forceinline__ void warp_band_scan(int b_lo, int b_hi, GetV getv, Put put) {
    const int lane = threadIdx.x & 31;
    // the values of four chunks of 32 bands are loaded before they are scanned: the loads
    // do not depend on the running sum, so their latencies overlap
    constexpr int PF = 4;
    T carry = T(0);
    for (int base = b_lo; base <= b_hi; base += 32 * PF) {
        T v[PF];
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            const int b = base + 32 * k + lane;
            v[k] = b <= b_hi ? getv(b) : T(0);
        }
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            if (base + 32 * k > b_hi) break;  // uniform over the warp
            const int b = base + 32 * k + lane;
            const T inc = warp_incl_scan(v[k], lane);
            if (b <= b_hi) put(b, carry + inc);
            carry += shfl_idx_T(inc, 31);
        }
    }
}

// Phase 2a: diagonal lines, x_b = X - (Ylast - Y_b):  S1_b[x_b] = L1_b[x_b] + S1_{b-1}[x_{b-1}]
template <class T>
__device__ void scan_s1_line(int X, int im, const T* __restrict__ L, T* __restrict__ S, int Hp, int Wp, int band_h,
                             int nb) {
    const int Ylast = Hp - 1, Y0 = band_last_row(0, band_h, Hp);
    if (X >= Wp + (Ylast - Y0)) return;
    // valid bands: 0 <= X - (Ylast - Y_b) < Wp, x increasing in b
    int b_lo = max(0, (Ylast - X + 1) / band_h - 1), b_hi = min(nb - 1, (Ylast - X + Wp) / band_h + 1);
    while (b_lo < nb && X - (Ylast - band_last_row(b_lo, band_h, Hp)) < 0) ++b_lo;
    while (b_hi >= b_lo && X - (Ylast - band_last_row(b_hi, band_h, Hp)) >= Wp) --b_hi;
    warp_band_scan<T>(b_lo, b_hi,
        [&](int b) {
            const int x = X - (Ylast - band_last_row(b, band_h, Hp));
            return L[((size_t)im * nb + b) * 3 * (size_t)Wp + x];
        },
        [&](int b, T v) {
            const int x = X - (Ylast - band_last_row(b, band_h, Hp));
            S[((size_t)im * nb + b) * 3 * (size_t)Wp + x] = v;
        });
}

// Phase 2c: columns:  S2_b[x] = L2_b[x] + sum_{j=1..h_b} S1_{b-1}[x-j] + S2_{b-1}[x]
template <class T>
__device__ void scan_s2_col(int x, int im, const T* __restrict__ L, T* __restrict__ S, const T* __restrict__ P1, int Hp,
                            int Wp, int band_h, int nb) {
    if (x >= Wp) return;
    warp_band_scan<T>(0, nb - 1,
        [&](int b) {
            T v = L[((size_t)im * nb + b) * 3 * (size_t)Wp + Wp + x];
            if (b > 0) {
                const int h = band_last_row(b, band_h, Hp) - band_last_row(b - 1, band_h, Hp);
                const T* p1 = P1 + ((size_t)im * nb + (b - 1)) * (size_t)Wp;
                v += at0(p1, x - 1) - at0(p1, x - h - 1);
            }
            return v;
        },
        [&](int b, T v) { S[((size_t)im * nb + b) * 3 * (size_t)Wp + Wp + x] = v; });
}

// Phase 2e: anti-diagonal lines, x_b = X + (Ylast - Y_b):
//   SG_b[x] = LG_b[x] + [x+h <= Wp-1] SG_{b-1}[x+h]
//           + sum_{j=j0..h} ( S2_{b-1}[x+h-j] + sum_{k=1..j} S1_{b-1}[x+h-j-k] ),
//   j0 = max(1, x+h-Wp+1)  (RS4 stops at the right buffer edge)
template <class T>
__device__ void scan_sg_line(int t, int im, const T* __restrict__ L, T* __restrict__ S, const T* __restrict__ P1,
                             const T* __restrict__ PP1, const T* __restrict__ Q1, const T* __restrict__ P2, int Hp,
                             int Wp, int band_h, int nb) {
    const int Ylast = Hp - 1, Y0 = band_last_row(0, band_h, Hp);
    const int X = t - (Ylast - Y0);
    if (X >= Wp) return;
    // valid bands: 0 <= X + (Ylast - Y_b) < Wp, x decreasing in b
    int b_lo = max(0, (X + Ylast - Wp + 1) / band_h - 1), b_hi = min(nb - 1, (X + Ylast) / band_h + 1);
    while (b_lo < nb && X + (Ylast - band_last_row(b_lo, band_h, Hp)) >= Wp) ++b_lo;
    while (b_hi >= b_lo && X + (Ylast - band_last_row(b_hi, band_h, Hp)) < 0) --b_hi;
    warp_band_scan<T>(b_lo, b_hi,
        [&](int b) {
            const int x = X + (Ylast - band_last_row(b, band_h, Hp));
            T v = L[((size_t)im * nb + b) * 3 * (size_t)Wp + 2 * Wp + x];
            if (b > 0) {
                const int h = band_last_row(b, band_h, Hp) - band_last_row(b - 1, band_h, Hp);
                const size_t pb = ((size_t)im * nb + (b - 1)) * (size_t)Wp;
                const int j0 = max(1, x + h - Wp + 1);
                v += at0(P2 + pb, x + h - j0) - at0(P2 + pb, x - 1);
                v += at0(PP1 + pb, x + h - 1 - j0) - at0(PP1 + pb, x - 2);
                v -= at0(Q1 + pb, x + h - 1 - 2 * j0) - at0(Q1 + pb, x - h - 3);
            }
            return v;
        },
        [&](int b, T v) {
            const int x = X + (Ylast - band_last_row(b, band_h, Hp));
            S[((size_t)im * nb + b) * 3 * (size_t)Wp + 2 * Wp + x] = v;
        });
}

template <class T> struct V3 {
    T a, b, c;
    __device__ __forceinline__ V3 operator+(const V3& o) const { return V3{a + o.a, b + o.b, c + o.c}; }
    __device__ __forceinline__ V3 operator-(const V3& o) const { return V3{a - o.a, b - o.b, c - o.c}; }
    __device__ __forceinline__ V3& operator+=(const V3& o) { a += o.a; b += o.b; c += o.c; return *this; }
    __device__ explicit V3(T z = T(0)) : a(z), b(z), c(z) {}
    __device__ V3(T x, T y, T w) : a(x), b(y), c(w) {}
};

// Inclusive prefix along one row of n <= blockDim * ITEMS elements by one
// CTA: each thread scans ITEMS consecutive elements, then a block scan of
// the thread totals.
template <class T, int ITEMS, class Get, class Put>
__device__ void block_row_scan(int n, Get get, Put put, T* smem /* 32 */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int i0 = threadIdx.x * ITEMS;
    T v[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) v[j] = (i0 + j < n) ? get(i0 + j) : T(0);
#pragma unroll
    for (int j = 1; j < ITEMS; ++j) v[j] += v[j - 1];
    const T tot = v[ITEMS - 1];
    const T inc = warp_incl_scan(tot, lane);
    if (lane == 31) smem[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const T t = lane < nw ? smem[lane] : T(0);
        const T ti = warp_incl_scan(t, lane);
        smem[lane] = ti - t;
    }
    __syncthreads();
    const T off = smem[warp] + (inc - tot);
#pragma unroll
    for (int j = 0; j < ITEMS; ++j)
        if (i0 + j < n) put(i0 + j, v[j] + off);
    __syncthreads();
}

// Phase 2b: P1 = prefix(S1), PP1 = prefix(P1), Q1[x] = P1[x] + Q1[x-2]
template <class T, int ITEMS>
__device__ void prefix1_band(int b, int im, const T* __restrict__ S, T* __restrict__ P1, T* __restrict__ PP1,
                             T* __restrict__ Q1, int Wp, int nb, T* sm, unsigned char* sm3_raw) {
    const T* s1 = S + ((size_t)im * nb + b) * 3 * (size_t)Wp;
    const size_t pb = ((size_t)im * nb + b) * (size_t)Wp;
    T* p1 = P1 + pb;
    T* pp1 = PP1 + pb;
    T* q1 = Q1 + pb;
    block_row_scan<T, ITEMS>(Wp, [&](int i) { return s1[i]; }, [&](int i, T v) { p1[i] = v; }, sm);
    // over pairs i: (P1[2i], P1[2i+1], P1[2i] + P1[2i+1]) -> Q1[2i], Q1[2i+1], PP1[2i+1];
    // PP1[2i] = PP1[2i+1] - P1[2i+1]
    // raw storage: V3 has a constructor, which shared memory does not run
    V3<T>* sm3 = reinterpret_cast<V3<T>*>(sm3_raw);
    block_row_scan<V3<T>, ITEMS / 2>((Wp + 1) / 2,
        [&](int i) {
            const T e = p1[2 * i], o = (2 * i + 1 < Wp) ? p1[2 * i + 1] : T(0);
            return V3<T>{e, o, e + o};
        },
        [&](int i, V3<T> v) {
            q1[2 * i] = v.a;
            const T o = (2 * i + 1 < Wp) ? p1[2 * i + 1] : T(0);
            pp1[2 * i] = v.c - o;
            if (2 * i + 1 < Wp) {
                q1[2 * i + 1] = v.b;
                pp1[2 * i + 1] = v.c;
            }
        },
        sm3);
}

// Phase 2d: P2 = prefix(S2)
template <class T, int ITEMS>
__device__ void prefix2_band(int b, int im, const T* __restrict__ S, T* __restrict__ P2, int Wp, int nb, T* sm) {
    const T* s2 = S + ((size_t)im * nb + b) * 3 * (size_t)Wp + Wp;
    T* p2 = P2 + ((size_t)im * nb + b) * (size_t)Wp;
    block_row_scan<T, ITEMS>(Wp, [&](int i) { return s2[i]; }, [&](int i, T v) { p2[i] = v; }, sm);
}

// Grid barrier of the carry kernel: every block is resident (cooperative
// launch), thread 0 of each block counts in and waits for the count of this
// barrier.  The wait is bounded: after CARRY_SPIN_LIMIT polls it raises
// BSF_ETIMEOUT and the block leaves the kernel (the buffer is then wrong and the
// status says so; nothing hangs).
constexpr unsigned CARRY_SPIN_LIMIT = 1u << 22;
__device__ __forceinline__ bool grid_barrier(unsigned* ctr, unsigned target, unsigned* status, unsigned spin_limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
        int ok = 1;
        for (unsigned it = 0;; ++it) {
            const unsigned v = *(volatile unsigned*)ctr;
            if (v >= target) break;
            if (it >= spin_limit) {
                if (status) atomicOr(status, 1u << BSF_ETIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Phase 2 in one launch: the five steps (diagonal lines, row prefixes of g1,
// columns, row prefixes of g2, anti-diagonal lines) as grid-stride loops over
// their lines or bands, separated by grid barriers.
constexpr int CARRY_THREADS = 512;
template <class T>
__global__ void __launch_bounds__(CARRY_THREADS) k_carries(const T* __restrict__ L, T* __restrict__ S,
                                                          T* __restrict__ P1, T* __restrict__ PP1,
                                                          T* __restrict__ Q1, T* __restrict__ P2, int Hp, int Wp,
                                                          int band_h, int nb, int nimg, unsigned* bar,
                                                          unsigned* status, unsigned spin_limit) {
    __shared__ T sm[32];
    __shared__ __align__(16) unsigned char sm3_raw[32 * sizeof(V3<T>)];
    const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * wpb + warp, nwarps = gridDim.x * wpb;
    const int nlines = Wp + (Hp - min(band_h, Hp));  // diagonal / anti-diagonal lines crossing the band ends
    unsigned target = 0;
    for (int t = gw; t < nlines * nimg; t += nwarps) scan_s1_line<T>(t % nlines, t / nlines, L, S, Hp, Wp, band_h, nb);
    if (!grid_barrier(bar, target += gridDim.x, status, spin_limit)) return;
    for (int t = blockIdx.x; t < nb * nimg; t += gridDim.x)
        prefix1_band<T, 8>(t % nb, t / nb, S, P1, PP1, Q1, Wp, nb, sm, sm3_raw);
    if (!grid_barrier(bar, target += gridDim.x, status, spin_limit)) return;
    for (int t = gw; t < Wp * nimg; t += nwarps) scan_s2_col<T>(t % Wp, t / Wp, L, S, P1, Hp, Wp, band_h, nb);
    if (!grid_barrier(bar, target += gridDim.x, status, spin_limit)) return;
    for (int t = blockIdx.x; t < nb * nimg; t += gridDim.x) prefix2_band<T, 8>(t % nb, t / nb, S, P2, Wp, nb, sm);
    if (!grid_barrier(bar, target += gridDim.x, status, spin_limit)) return;
    for (int t = gw; t < nlines * nimg; t += nwarps)
        scan_sg_line<T>(t % nlines, t / nlines, L, S, P1, PP1, Q1, P2, Hp, Wp, band_h, nb);
}

}  // namespace

// ---------------------------------------------------------------- host side
scan_plan make_scan_plan(int Hp, int Wp, int nimg, size_t elem_bytes) {
    scan_plan p;
    // bands: one wave of band CTAs (one per SM of a 152-SM part) over the whole batch
    int bh = (int)(((long long)Hp * nimg + 151) / 152);
    if (bh < 8) bh = 8;
    if (bh > 64) bh = 64;
    if (bh > Hp) bh = Hp;
    p.band_h = bh;
    p.nb = (Hp + bh - 1) / bh;
    const bool wide = elem_bytes > 8;
    p.cpt = 1;
    while (p.cpt < 8 && ((Wp + p.cpt - 1) / p.cpt + 31) / 32 * 32 > band_maxt(wide, p.cpt)) p.cpt *= 2;
    p.threads = ((Wp + p.cpt - 1) / p.cpt + 31) / 32 * 32;
    // the band kernel keeps its state in registers, but for the widest 128-bit form
    p.smem = (wide && p.cpt >= 8) ? (size_t)p.threads * p.cpt * elem_bytes : 0;
    p.ok = p.threads <= band_maxt(wide, p.cpt);
    const size_t row = (size_t)nimg * p.nb * Wp * elem_bytes;
    p.work_bytes = row * 10 + 256;  // L (3), S (3), P1, PP1, Q1, P2, and the carry kernel's barrier word
    return p;
}

int scan_max_width(size_t elem_bytes, bool narrow) {
    const bool wide = elem_bytes > 8;
    return (wide && narrow) ? 4 * band_maxt(true, 4) : 8 * band_maxt(wide, 8);
}

template <int MODE, class InT, int CPT>
static void launch_band(const scan_plan& p, const InT* img, long long img_stride, int nimg, int H, int W, int col0,
                        int P, int Hp, int Wp, int pitch, const void* carry, void* local, void* G, long long G_stride,
                        cudaStream_t st, int reflect) {
    typedef typename mode_traits<MODE>::T T;
    dim3 grid(p.nb, nimg);
    // Any dynamic shared memory opts in to one fixed cap (a row of at most 4096 16-byte elements):
    // the kernel's static shared memory (up to 3 KB) counts against the 48 KB default too, and a
    // fixed value keeps launches from several host threads from lowering it for one another; each
    // launch still asks for its own size
    constexpr int kBandSmemCap = 4096 * 16;
    if (p.smem > 0)
        cudaFuncSetAttribute(k_band<MODE, InT, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBandSmemCap);
    k_band<MODE, InT, CPT><<<grid, p.threads, p.smem, st>>>(img, img_stride, H, W, col0, P, Hp, Wp, pitch, p.band_h, p.nb,
                                                        (const T*)carry, (T*)local, (T*)G, G_stride, reflect);
}

template <int MODE, class InT>
static void launch_band_cpt(const scan_plan& p, const InT* img, long long img_stride, int nimg, int H, int W, int col0,
                            int P, int Hp, int Wp, int pitch, const void* carry, void* local, void* G,
                            long long G_stride, cudaStream_t st, int reflect) {
    switch (p.cpt) {
        case 1: launch_band<MODE, InT, 1>(p, img, img_stride, nimg, H, W, col0, P, Hp, Wp, pitch, carry, local, G, G_stride, st, reflect); break;
        case 2: launch_band<MODE, InT, 2>(p, img, img_stride, nimg, H, W, col0, P, Hp, Wp, pitch, carry, local, G, G_stride, st, reflect); break;
        case 4: launch_band<MODE, InT, 4>(p, img, img_stride, nimg, H, W, col0, P, Hp, Wp, pitch, carry, local, G, G_stride, st, reflect); break;
        default: launch_band<MODE, InT, 8>(p, img, img_stride, nimg, H, W, col0, P, Hp, Wp, pitch, carry, local, G, G_stride, st, reflect); break;
    }
}

template <int MODE, class InT>
cudaError_t launch_scan4(const InT* img, long long img_stride, int nimg, int H, int W, int P, void* G,
                         long long G_stride, int pitch, void* work, cudaStream_t st, int col0, int Ws, int reflect,
                         unsigned* status, unsigned spin_limit) {
    typedef typename mode_traits<MODE>::T T;
    if (Ws <= 0) Ws = W;
    const int Hp = H + 2 * P, Wp = Ws + 2 * P;
    const scan_plan p = make_scan_plan(Hp, Wp, nimg, sizeof(T));
    if (!p.ok) return cudaErrorInvalidValue;
    const size_t row = (size_t)nimg * p.nb * Wp;
    T* L = (T*)work;
    T* S = L + 3 * row;
    T* P1 = S + 3 * row;
    T* PP1 = P1 + row;
    T* Q1 = PP1 + row;
    T* P2 = Q1 + row;
    launch_band_cpt<MODE, InT>(p, img, img_stride, nimg, H, W, col0, P, Hp, Wp, pitch, nullptr, L, nullptr, 0, st,
                               reflect);
    // phase 2: one cooperative launch (every block resident, grid barriers between the steps)
    unsigned* bar = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(work) + (p.work_bytes - 256));
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, occ = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_carries<T>, CARRY_THREADS, 0)) != cudaSuccess)
        return e;
    const int nlines = Wp + (Hp - min(p.band_h, Hp));
    const long long want_w = (long long)max(nlines, Wp) * nimg;  // warps of the line steps
    const long long want = max((want_w + CARRY_THREADS / 32 - 1) / (CARRY_THREADS / 32), (long long)p.nb * nimg);
    const int grid = (int)max(1LL, min((long long)occ * nsm, want));
    int Hp_ = Hp, Wp_ = Wp, bh = p.band_h, nb = p.nb, ni = nimg;
    unsigned spin = spin_limit ? spin_limit : CARRY_SPIN_LIMIT;
    void* args[] = {&L, &S, &P1, &PP1, &Q1, &P2, &Hp_, &Wp_, &bh, &nb, &ni, &bar, &status, &spin};
    e = cudaLaunchCooperativeKernel((const void*)k_carries<T>, dim3(grid), dim3(CARRY_THREADS), args, 0, st);
    if (e != cudaSuccess) return e;
    launch_band_cpt<MODE, InT>(p, img, img_stride, nimg, H, W, col0, P, Hp, Wp, pitch, S, nullptr, G, G_stride, st,
                               reflect);
    return cudaGetLastError();
}

template cudaError_t launch_scan4<MODE_U64, uint8_t>(const uint8_t*, long long, int, int, int, int, void*, long long,
                                                     int, void*, cudaStream_t, int, int, int, unsigned*, unsigned);
template cudaError_t launch_scan4<MODE_U128, float>(const float*, long long, int, int, int, int, void*, long long, int,
                                                    void*, cudaStream_t, int, int, int, unsigned*, unsigned);
template cudaError_t launch_scan4<MODE_F64, uint8_t>(const uint8_t*, long long, int, int, int, int, void*, long long,
                                                     int, void*, cudaStream_t, int, int, int, unsigned*, unsigned);
template cudaError_t launch_scan4<MODE_F64, float>(const float*, long long, int, int, int, int, void*, long long, int,
                                                   void*, cudaStream_t, int, int, int, unsigned*, unsigned);
