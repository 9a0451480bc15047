// Feature-preserving smoothing (Sec. 4.2): the covariance field that adapts
// the filter to the local image structure.
//
// The structure tensor of Eq. eigen is J = w * (g g^T), g the image gradient
// and w an isotropic averaging window; its eigenvector of the smallest
// eigenvalue points along the feature (the orientation theta* of minimal
// intensity variation) and lambda_max / lambda_min is the elongation rho*.
// Here:
//   g      central differences, replicated at the image border,
//          summed over the channels (g g^T of every channel added);
//   w      the isotropic four-directional box spline itself (a_k = sigma_w
//          sqrt 6, the covariance of a Gaussian of std sigma_w), applied by
//          the exact filter of this library;
//   C(n)   = sigma0^2 adj(M) / sqrt(det M),  M = J(n) + tau I.
// C has det C = sigma0^4 (the area of the isotropic window of std sigma0),
// its long axis along the minimal-eigenvalue eigenvector of J and the
// elongation (lambda_max + tau) / (lambda_min + tau): where the image is flat
// (J << tau) the window is isotropic, along an edge or a stripe it is
// stretched along the feature.  tau regularises the ratio of the paper's
// rho* = lambda_max / lambda_min (defined there case by case for zero
// eigenvalues) and sets the gradient energy below which a region counts as
// uniform; C is a smooth function of J, so no eigen-decomposition is needed.
#include <algorithm>

#include "bsf_common.cuh"
#include "bsf_internal.h"

namespace {

template <class InT>
__device__ __forceinline__ float sample_f(const InT* p) { return (float)*p; }

// gradient products, summed over channels: prod = (gx^2, gx gy, gy^2) per batch entry
template <class InT>
__global__ void k_st_products(const InT* __restrict__ img, int B, int C, int H, int W, float* __restrict__ prod) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, b = blockIdx.z;
    if (x >= W || y >= H) return;
    const size_t HW = (size_t)H * W;
    const int xl = max(x - 1, 0), xr = min(x + 1, W - 1), yu = max(y - 1, 0), yd = min(y + 1, H - 1);
    float sxx = 0.f, sxy = 0.f, syy = 0.f;
    for (int c = 0; c < C; ++c) {
        const InT* f = img + ((size_t)b * C + c) * HW;
        const float gx = 0.5f * (sample_f(f + (size_t)y * W + xr) - sample_f(f + (size_t)y * W + xl));
        const float gy = 0.5f * (sample_f(f + (size_t)yd * W + x) - sample_f(f + (size_t)yu * W + x));
        sxx = fmaf(gx, gx, sxx);
        sxy = fmaf(gx, gy, sxy);
        syy = fmaf(gy, gy, syy);
    }
    float* o = prod + (size_t)b * 3 * HW + (size_t)y * W + x;
    o[0] = sxx;
    o[HW] = sxy;
    o[2 * HW] = syy;
}

__global__ void k_fill(float* __restrict__ p, size_t n, float v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

// C = sigma0^2 adj(J + tau I) / sqrt(det(J + tau I)), per pixel
__global__ void k_adaptive_cov(const float* __restrict__ J, long long HW, int B, float s0sq, float tau,
                               float* __restrict__ cov) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= HW * B) return;
    const long long b = i / HW, p = i - b * HW;
    const float* j = J + b * 3 * HW + p;
    const float m11 = j[0] + tau, m12 = j[HW], m22 = j[2 * HW] + tau;
    const float det = fmaf(m11, m22, -m12 * m12);
    float* c = cov + b * 3 * HW + p;
    if (!(det > 0.f)) {  // not finite, or J not positive semidefinite: isotropic
        c[0] = s0sq;
        c[HW] = 0.f;
        c[2 * HW] = s0sq;
        return;
    }
    const float s = s0sq / sqrtf(det);
    c[0] = s * m22;
    c[HW] = -s * m12;
    c[2 * HW] = s * m11;
}

}  // namespace

cudaError_t launch_st_products(const void* img, int dtype_u8, int B, int C, int H, int W, float* prod,
                               cudaStream_t st) {
    dim3 blk(32, 8), grd((W + 31) / 32, (H + 7) / 8, B);
    if (dtype_u8)
        k_st_products<uint8_t><<<grd, blk, 0, st>>>((const uint8_t*)img, B, C, H, W, prod);
    else
        k_st_products<float><<<grd, blk, 0, st>>>((const float*)img, B, C, H, W, prod);
    return cudaGetLastError();
}

cudaError_t launch_fill(float* p, size_t n, float v, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
    k_fill<<<blocks, 256, 0, st>>>(p, n, v);
    return cudaGetLastError();
}

cudaError_t launch_adaptive_cov(const float* J, long long HW, int B, float s0sq, float tau, float* cov,
                                cudaStream_t st) {
    const long long n = HW * B;
    if (n == 0) return cudaSuccess;
    k_adaptive_cov<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(J, HW, B, s0sq, tau, cov);
    return cudaGetLastError();
}
