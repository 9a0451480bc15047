// bsf_filter_noalloc: the whole filter for one image without any device
// allocation.  Its scratch (the pre-integrated buffer and the scan carries)
// lives in a fixed array compiled into the library, so the call never runs
// cudaMalloc, cudaFree or any allocating routine.  This serves callers that
// must not allocate device memory themselves: plugins inside a host
// application that owns the device memory budget, and latency-critical loops
// in which cudaMalloc/cudaFree would synchronise the device.
//
// Costs and limits of that choice:
//  * the array (BSF_NOALLOC_SCRATCH_BYTES) is reserved on every GPU that
//    loads the library, for the life of the process;
//  * every call shares it and it keeps the previous call's contents: calls
//    whose work overlaps on the GPU (different streams, or different host
//    threads on one device) race and must be serialised by the caller;
//  * the first call on a device looks up the array's device address (with
//    that device current); make that first call before any stream capture;
//  * there is no device status word: pixels with invalid scales or taps
//    outside the buffer come out as NaN.
#include <mutex>

#include "bsf_common.cuh"
#include "bsf_internal.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[BSF_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_mu;
constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

size_t round_up256(size_t n) { return (n + 255) & ~(size_t)255; }
}  // namespace

extern "C" bsf_status bsf_filter_noalloc(const void* image, int dtype, int64_t H, int64_t W, int N,
                                         const float* params, int kind, const bsf_opts* opts, float* out,
                                         void* stream) {
    if (!image || !params || !out || !opts) return BSF_EINVAL;
    if (H <= 0 || W <= 0 || H > (1 << 20) || W > (1 << 20)) return BSF_EINVAL;
    if (dtype != BSF_U8 && dtype != BSF_F32) return BSF_EINVAL;
    if (kind != BSF_PARAM_SCALES && kind != BSF_PARAM_COV && kind != BSF_PARAM_SRT) return BSF_EINVAL;
    if (opts->precision != BSF_PREC_EXACT && opts->precision != BSF_PREC_FP64) return BSF_EINVAL;
    if (opts->iterations > 1) return BSF_EINVAL;
    if (opts->boundary != BSF_BOUNDARY_ZERO && opts->boundary != BSF_BOUNDARY_REFLECT) return BSF_EINVAL;
    const int refl = opts->boundary == BSF_BOUNDARY_REFLECT;
    if (N != 4) return BSF_EUNSUPPORTED;
    // the halo must come from the options (no device reduction, which would need a result word)
    int P = opts->halo;
    if (P > kMaxHalo) return BSF_EINVAL;
    if (P <= 0) {
        if (!(opts->max_scale > 0.f) || opts->max_scale > 1e5f) return BSF_EINVAL;
        const float ext = (kind == BSF_PARAM_SCALES) ? 2.41422f * opts->max_scale : 8.3640f * opts->max_scale;
        P = (int)ceilf(0.5f * ext) + 4;
    }
    const int mode = opts->precision == BSF_PREC_FP64 ? MODE_F64 : (dtype == BSF_U8 ? MODE_U64 : MODE_U128);
    const size_t esz = mode == MODE_U128 ? 16 : 8;
    const int64_t Hp = H + 2 * (int64_t)P, Wp = W + 2 * (int64_t)P;  // at most 3 * 2^20 each
    // the buffer alone already beyond the scratch: reject before planning the scan
    if ((uint64_t)Hp * (uint64_t)Wp * esz > (uint64_t)BSF_NOALLOC_SCRATCH_BYTES) return BSF_ENOSCRATCH;
    const scan_plan plan = make_scan_plan((int)Hp, (int)Wp, 1, esz);
    const size_t buf_bytes = round_up256((size_t)(Hp * Wp) * esz);
    if (buf_bytes + plan.work_bytes > (size_t)BSF_NOALLOC_SCRATCH_BYTES) return BSF_ENOSCRATCH;
    if (!plan.ok) return BSF_EINVAL;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return BSF_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return BSF_EINVAL;
    unsigned char* base;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (g_scratch_ptr[dev] == nullptr) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || p == nullptr) return BSF_ECUDA;
            g_scratch_ptr[dev] = p;
        }
        base = (unsigned char*)g_scratch_ptr[dev];
    }
    void* G = base;
    void* work = base + buf_bytes;
    cudaStream_t st = (cudaStream_t)stream;
    // every element of the buffer and of the carry rows is written before it is
    // read, so nothing left from a previous call needs clearing
    if (mode == MODE_U64)
        e = launch_scan4<MODE_U64, uint8_t>((const uint8_t*)image, H * W, 1, (int)H, (int)W, P, G, Hp * Wp, (int)Wp,
                                            work, st, 0, 0, refl, nullptr, bsf_wait_limit());
    else if (mode == MODE_U128)
        e = launch_scan4<MODE_U128, float>((const float*)image, H * W, 1, (int)H, (int)W, P, G, Hp * Wp, (int)Wp,
                                           work, st, 0, 0, refl, nullptr, bsf_wait_limit());
    else if (dtype == BSF_U8)
        e = launch_scan4<MODE_F64, uint8_t>((const uint8_t*)image, H * W, 1, (int)H, (int)W, P, G, Hp * Wp, (int)Wp,
                                            work, st, 0, 0, refl, nullptr, bsf_wait_limit());
    else
        e = launch_scan4<MODE_F64, float>((const float*)image, H * W, 1, (int)H, (int)W, P, G, Hp * Wp, (int)Wp,
                                          work, st, 0, 0, refl, nullptr, bsf_wait_limit());
    if (e != cudaSuccess) return BSF_ECUDA;
    stencil_args a;
    a.buf = G;
    a.buf_stride = 0;
    a.Hp = (int)Hp;
    a.Wp = (int)Wp;
    a.pitch = (int)Wp;
    a.P = P;
    a.H = (int)H;
    a.W = (int)W;
    a.C = 1;
    a.nimg = 1;
    a.params = params;
    a.kind = kind;
    a.eps = opts->eps;
    a.eta = opts->eta;
    a.out = out;
    a.status = nullptr;
    e = launch_stencil4(mode, a, st);
    return e == cudaSuccess ? BSF_OK : BSF_ECUDA;
}
