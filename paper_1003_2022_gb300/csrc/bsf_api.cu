// C ABI of the GB300 box-spline filter (see include/bsf.h).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <mutex>
#include <vector>

#include <atomic>

#include "bsf_common.cuh"
#include "bsf_internal.h"

struct bsf_ctx {
    int device;
    unsigned* d_status;      // device status word
    unsigned* d_ext;         // scratch word for the extent reduction
    void* buf;               // pre-integrated buffers (library-owned)
    size_t buf_bytes;
    void* work;              // scan carry workspace
    size_t work_bytes;
    void* hbuf;              // FP64 scatter buffers of the adjoint
    size_t hbuf_bytes;
    void* iter;              // scaled fields and intermediate images of the iterated filter
    size_t iter_bytes;
    void* stbuf;             // structure-tensor planes of bsf_structure_cov
    size_t stbuf_bytes;
    std::mutex mu;
    // host-buffer pipeline (bsf_filter_host): three streams and two slots of
    // device buffers that alternate between calls
    struct host_slot {
        void* img = nullptr;
        size_t img_bytes = 0;
        void* prm = nullptr;
        size_t prm_bytes = 0;
        void* out = nullptr;
        size_t out_bytes = 0;
        cudaEvent_t in_ready = nullptr, comp_done = nullptr, out_done = nullptr;
    } hs[2];
    cudaStream_t s_h2d, s_comp, s_d2h;
    unsigned long long host_calls;
    // six-directional path (hex6.cu): FP64 scales, per-tile footprint extents,
    // window records and the lattice windows themselves
    void* h6_scales = nullptr;
    size_t h6_scales_bytes = 0;
    void* h6_ext = nullptr;
    size_t h6_ext_bytes = 0;
    void* h6_tiles = nullptr;
    size_t h6_tiles_bytes = 0;
    void* h6_win = nullptr;
    size_t h6_win_bytes = 0;
    void* h6_flag = nullptr;  // per (tile, channel) of a chunk: window values beyond the exact range
    size_t h6_flag_bytes = 0;
    // the windows of chunk i + 1 are pre-integrated on a side stream into the second of two
    // buffers while the stencil of chunk i runs on the caller's stream
    cudaStream_t h6_side = nullptr;
    // the map's table (opts.map_lut), built for one (eta, rel) pair at a time
    void* h6_lut = nullptr;
    double h6_lut_eta = -1.0, h6_lut_rel = -1.0;
    cudaEvent_t h6_ev_tiles = nullptr, h6_ev_pre[2] = {nullptr, nullptr}, h6_ev_st[2] = {nullptr, nullptr};
    bool profiling;
    size_t prof_used;                                // event sets recorded since begin
    // per launch: [0] pre-integration start, [1] its end (= stencil start unless [3] is used),
    // [2] stencil end, [3] stencil start when the two run on different streams
    std::vector<std::array<cudaEvent_t, 4>> prof;
    std::vector<char> prof_split;
};

static cudaError_t prof_mark(bsf_ctx* c, int which, cudaStream_t st) {
    if (!c->profiling) return cudaSuccess;
    if (which == 0) {
        if (c->prof_used == c->prof.size()) {
            std::array<cudaEvent_t, 4> t;
            for (int i = 0; i < 4; ++i) {
                cudaError_t e = cudaEventCreate(&t[i]);
                if (e != cudaSuccess) return e;
            }
            c->prof.push_back(t);
            c->prof_split.push_back(0);
        }
        c->prof_split[c->prof_used] = 0;
        ++c->prof_used;
    }
    if (which == 3) c->prof_split[c->prof_used - 1] = 1;
    return cudaEventRecord(c->prof[c->prof_used - 1][which], st);
}

static bsf_status map_cuda(cudaError_t e) {
    if (e == cudaSuccess) return BSF_OK;
    if (e == cudaErrorMemoryAllocation) return BSF_ENOMEM;
    return BSF_ECUDA;
}

#define BSF_TRY(expr)                          \
    do {                                       \
        cudaError_t e_ = (expr);               \
        if (e_ != cudaSuccess) return map_cuda(e_); \
    } while (0)

static cudaError_t grow(void** p, size_t* cur, size_t need) {
    if (*cur >= need && *p != nullptr) return cudaSuccess;
    if (*p) {
        cudaError_t e = cudaFree(*p);
        *p = nullptr;
        *cur = 0;
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMalloc(p, need);
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    *cur = need;
    return cudaSuccess;
}

static int mode_of(int dtype, int precision) {
    if (precision == BSF_PREC_FP64) return MODE_F64;
    return dtype == BSF_U8 ? MODE_U64 : MODE_U128;
}

static size_t elem_bytes(int mode) { return mode == MODE_U128 ? 16 : 8; }

// bound of the device waits between row bands (polls; 0 = the kernel's default)
static std::atomic<unsigned> g_wait_limit{0};
unsigned bsf_wait_limit() { return g_wait_limit.load(std::memory_order_relaxed); }

extern "C" {

void bsf_set_wait_limit(unsigned polls) { g_wait_limit.store(polls, std::memory_order_relaxed); }

void bsf_default_opts(bsf_opts* o) {
    if (!o) return;
    o->precision = BSF_PREC_EXACT;
    o->eps = 1e-3f;
    o->eta = 1e-3f;
    o->strict = 0;
    o->halo = 0;
    o->max_scale = 0.f;
    o->iterations = 1;
    o->hex_spacing = 0.5f;
    o->rel_bound = 1e-3f;
    o->boundary = BSF_BOUNDARY_ZERO;
    o->map_lut = 0;
    o->staging = BSF_STAGING_L1;
}

const char* bsf_status_string(bsf_status s) {
    switch (s) {
        case BSF_OK: return "ok";
        case BSF_EINVAL: return "invalid argument";
        case BSF_EUNSUPPORTED: return "unsupported N (N = 4 everywhere; N = 6 in bsf_filter, bsf_filter_host and bsf_scales_from_cov)";
        case BSF_ENOMEM: return "device allocation failed";
        case BSF_ECUDA: return "CUDA runtime error";
        case BSF_EHALO: return "a finite-difference tap left the pre-integrated buffer (halo too small)";
        case BSF_EINFEASIBLE: return "a covariance needed the elongation clamp (strict mode)";
        case BSF_EBADSCALE: return "a scale or covariance was not finite and positive";
        case BSF_ERANGE: return "a kernel too large for the exact integer form";
        case BSF_ENOSCRATCH: return "the image does not fit the fixed scratch of bsf_filter_noalloc";
        case BSF_ETIMEOUT: return "a bounded device wait between row bands of the pre-integration gave up";
        default: return "unknown status";
    }
}

bsf_status bsf_create(bsf_ctx** ctx, int device) {
    if (!ctx) return BSF_EINVAL;
    *ctx = nullptr;
    int n = 0;
    BSF_TRY(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return BSF_EINVAL;
    BSF_TRY(cudaSetDevice(device));
    bsf_ctx* c = new bsf_ctx();
    c->device = device;
    c->d_status = nullptr;
    c->d_ext = nullptr;
    c->buf = nullptr;
    c->buf_bytes = 0;
    c->work = nullptr;
    c->work_bytes = 0;
    c->hbuf = nullptr;
    c->hbuf_bytes = 0;
    c->iter = nullptr;
    c->iter_bytes = 0;
    c->stbuf = nullptr;
    c->stbuf_bytes = 0;
    c->profiling = false;
    c->prof_used = 0;
    c->s_h2d = c->s_comp = c->s_d2h = nullptr;
    c->host_calls = 0;
    cudaError_t e = cudaMalloc((void**)&c->d_status, 2 * sizeof(unsigned));
    if (e != cudaSuccess) {
        delete c;
        return map_cuda(e);
    }
    c->d_ext = c->d_status + 1;
    e = cudaMemset(c->d_status, 0, 2 * sizeof(unsigned));
    if (e != cudaSuccess) {
        cudaFree(c->d_status);
        delete c;
        return map_cuda(e);
    }
    *ctx = c;
    return BSF_OK;
}

bsf_status bsf_destroy(bsf_ctx* c) {
    if (!c) return BSF_EINVAL;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    if (c->buf) cudaFree(c->buf);
    if (c->work) cudaFree(c->work);
    if (c->hbuf) cudaFree(c->hbuf);
    if (c->iter) cudaFree(c->iter);
    if (c->stbuf) cudaFree(c->stbuf);
    for (void* p6 : {c->h6_scales, c->h6_ext, c->h6_tiles, c->h6_win, c->h6_flag, c->h6_lut})
        if (p6) cudaFree(p6);
    if (c->d_status) cudaFree(c->d_status);
    for (auto& h : c->hs) {
        if (h.img) cudaFree(h.img);
        if (h.prm) cudaFree(h.prm);
        if (h.out) cudaFree(h.out);
        if (h.in_ready) cudaEventDestroy(h.in_ready);
        if (h.comp_done) cudaEventDestroy(h.comp_done);
        if (h.out_done) cudaEventDestroy(h.out_done);
    }
    for (cudaStream_t s_ : {c->s_h2d, c->s_comp, c->s_d2h})
        if (s_) cudaStreamDestroy(s_);
    for (auto& t : c->prof)
        for (int i = 0; i < 4; ++i) cudaEventDestroy(t[i]);
    if (c->h6_side) cudaStreamDestroy(c->h6_side);
    for (cudaEvent_t e : {c->h6_ev_tiles, c->h6_ev_pre[0], c->h6_ev_pre[1], c->h6_ev_st[0], c->h6_ev_st[1]})
        if (e) cudaEventDestroy(e);
    delete c;
    return BSF_OK;
}

bsf_status bsf_profile_begin(bsf_ctx* c) {
    if (!c) return BSF_EINVAL;
    std::lock_guard<std::mutex> lock(c->mu);
    c->profiling = true;
    c->prof_used = 0;
    return BSF_OK;
}

bsf_status bsf_profile_end(bsf_ctx* c, double* ms_pre, double* ms_st, int* nlaunch) {
    if (!c) return BSF_EINVAL;
    std::lock_guard<std::mutex> lock(c->mu);
    BSF_TRY(cudaSetDevice(c->device));
    double a = 0, b = 0;
    for (size_t i = 0; i < c->prof_used; ++i) {
        BSF_TRY(cudaEventSynchronize(c->prof[i][2]));
        float t0 = 0, t1 = 0;
        BSF_TRY(cudaEventElapsedTime(&t0, c->prof[i][0], c->prof[i][1]));
        BSF_TRY(cudaEventElapsedTime(&t1, c->prof[i][c->prof_split[i] ? 3 : 1], c->prof[i][2]));
        a += t0;
        b += t1;
    }
    if (ms_pre) *ms_pre = a;
    if (ms_st) *ms_st = b;
    if (nlaunch) *nlaunch = (int)c->prof_used;
    c->profiling = false;
    c->prof_used = 0;
    return BSF_OK;
}

bsf_status bsf_buffer_bytes(int dtype, int64_t H, int64_t W, int N, int halo, int precision, size_t* bytes) {
    if (!bytes || H <= 0 || W <= 0 || halo < 2 || halo > kMaxHalo) return BSF_EINVAL;
    if (dtype != BSF_U8 && dtype != BSF_F32) return BSF_EINVAL;
    if (precision != BSF_PREC_EXACT && precision != BSF_PREC_FP64) return BSF_EINVAL;
    if (N != 4) return BSF_EUNSUPPORTED;
    const int64_t Hp = H + 2 * (int64_t)halo, Wp = W + 2 * (int64_t)halo;
    *bytes = (size_t)(Hp * Wp) * elem_bytes(mode_of(dtype, precision));
    return BSF_OK;
}

bsf_status bsf_get_device_status(bsf_ctx* c, void* stream, int* status) {
    if (!c || !status) return BSF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned h = 0;
    BSF_TRY(cudaStreamSynchronize(st));
    BSF_TRY(cudaMemcpyAsync(&h, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    BSF_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), st));
    BSF_TRY(cudaStreamSynchronize(st));
    *status = (int)h;
    return BSF_OK;
}

// the map's table for opts (null unless opts.map_lut); built on st and waited for once per
// (eta, rel), so that later calls on any stream see it complete.  The caller holds c->mu.
static cudaError_t map6_table(bsf_ctx* c, const bsf_opts& o, cudaStream_t st, const float** lut) {
    *lut = nullptr;
    if (!o.map_lut) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (!c->h6_lut && (e = cudaMalloc(&c->h6_lut, lut6_bytes())) != cudaSuccess) return e;
    if (c->h6_lut_eta != (double)o.eta || c->h6_lut_rel != (double)o.rel_bound) {
        c->h6_lut_eta = c->h6_lut_rel = -1.0;
        if ((e = launch_lut6_build(o.eta, o.rel_bound, (float*)c->h6_lut, st)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        c->h6_lut_eta = o.eta;
        c->h6_lut_rel = o.rel_bound;
    }
    *lut = (const float*)c->h6_lut;
    return cudaSuccess;
}

bsf_status bsf_scales_from_cov(bsf_ctx* c, const float* params, int kind, int64_t npix, int N, const bsf_opts* opts,
                               float* scales, uint8_t* flags, void* stream) {
    if (!c || !params || !scales || npix < 0) return BSF_EINVAL;
    if (kind != BSF_PARAM_COV && kind != BSF_PARAM_SRT) return BSF_EINVAL;
    if (N != 4 && N != 6) return BSF_EUNSUPPORTED;
    bsf_opts o;
    bsf_default_opts(&o);
    if (opts) o = *opts;
    if (N == 6 && !(o.rel_bound >= 0.f && o.rel_bound < 1.f / 6.f)) return BSF_EINVAL;
    BSF_TRY(cudaSetDevice(c->device));
    if (N == 6) {
        std::lock_guard<std::mutex> lock(c->mu);
        const float* lut = nullptr;
        BSF_TRY(map6_table(c, o, (cudaStream_t)stream, &lut));
        BSF_TRY(launch_map6_out(params, kind, (long long)npix, o.eps, o.eta, o.rel_bound, scales, flags,
                                 (cudaStream_t)stream, lut));
    }
    else
        BSF_TRY(launch_map4(params, kind, (long long)npix, o.eps, o.eta, scales, flags, (cudaStream_t)stream));
    return BSF_OK;
}

// halo from opts or from a device reduction over the parameter fields
static bsf_status resolve_halo(bsf_ctx* c, const float* params, int kind, int64_t nfield, int64_t HW, const bsf_opts& o,
                               cudaStream_t st, int* P) {
    if (o.halo > 0) {
        if (o.halo > kMaxHalo) return BSF_EINVAL;
        *P = o.halo;
        return BSF_OK;
    }
    float ext;
    if (o.max_scale > 0.f) {
        // SCALES: a1 + (a2 + a4)/sqrt2 <= (1 + sqrt2) max a.  COV/SRT: a1 <= sqrt(12 C11),
        // a2' + a4' <= sqrt(p2 + p4) <= sqrt(24 C11), C11 <= lambda_max (same along y).
        ext = (kind == BSF_PARAM_SCALES) ? 2.41422f * o.max_scale : 8.3640f * o.max_scale;
    } else {
        const int K = (kind == BSF_PARAM_SCALES) ? 4 : 3;
        unsigned h = 0;
        BSF_TRY(cudaMemsetAsync(c->d_ext, 0, sizeof(unsigned), st));
        for (int64_t b = 0; b < nfield; ++b)
            BSF_TRY(launch_extent4(params + (size_t)b * K * HW, kind, (long long)HW, o.eps, o.eta, c->d_ext, st));
        BSF_TRY(cudaMemcpyAsync(&h, c->d_ext, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        BSF_TRY(cudaStreamSynchronize(st));
        memcpy(&ext, &h, sizeof(float));
    }
    if (!(ext >= 0.f) || ext > 1e6f) return BSF_EINVAL;
    *P = (int)ceilf(0.5f * ext) + 4;
    return BSF_OK;
}

static cudaError_t run_scan(int mode, int dtype, const void* img, long long img_stride, int nimg, int H, int W, int P,
                            void* G, long long G_stride, int pitch, void* work, cudaStream_t st, int col0 = 0,
                            int Ws = 0, int reflect = 0, unsigned* status = nullptr) {
    if (mode == MODE_U64)
        return launch_scan4<MODE_U64, uint8_t>((const uint8_t*)img, img_stride, nimg, H, W, P, G, G_stride, pitch,
                                               work, st, col0, Ws, reflect, status, bsf_wait_limit());
    if (mode == MODE_U128)
        return launch_scan4<MODE_U128, float>((const float*)img, img_stride, nimg, H, W, P, G, G_stride, pitch,
                                              work, st, col0, Ws, reflect, status, bsf_wait_limit());
    if (dtype == BSF_U8)
        return launch_scan4<MODE_F64, uint8_t>((const uint8_t*)img, img_stride, nimg, H, W, P, G, G_stride, pitch,
                                               work, st, col0, Ws, reflect, status, bsf_wait_limit());
    return launch_scan4<MODE_F64, float>((const float*)img, img_stride, nimg, H, W, P, G, G_stride, pitch, work, st,
                                         col0, Ws, reflect, status, bsf_wait_limit());
}

static bool dims_ok(int64_t H, int64_t W) {
    return H > 0 && W > 0 && H <= (1 << 20) && W <= (1 << 20);
}

// Buffer layout of the four-directional path for a batch: the padded buffer
// per image, vertical strips where a row is wider than one band CTA holds, and
// the images per launch (shared by filter_pass and bsf_query_workspace).
struct n4_layout {
    int mode, nstrip, Ws, Hp, Wp, pitch;
    size_t per_img;  // bytes of one image's buffer
    int64_t bchunk;  // batch entries per launch
};
static bsf_status n4_layout_of(int dtype, int64_t B, int64_t C, int64_t H, int64_t W, int P, int precision,
                               n4_layout* L) {
    const int mode = mode_of(dtype, precision);
    // Rows wider than one band CTA can hold are cut into vertical strips.  The
    // filter at a pixel depends only on f inside its footprint, so each strip is
    // pre-integrated from the image columns it needs (its outputs +- P) and the
    // exact integer result is the same as with one buffer.
    // When the batch fills several waves of band CTAs (one per SM), the 128-bit
    // form runs faster with narrower strips (four columns per thread instead of
    // eight: fewer registers per column); one image at a time it does not.
    const bool many_waves = (long long)((int)H + 2 * P) * B * C > 64LL * 152;
    const int maxw = scan_max_width(elem_bytes(mode), many_waves);
    const int Wfull = (int)W + 2 * P;
    const int nstrip = Wfull <= maxw ? 1 : (int)((W + (maxw - 2 * P) - 1) / (maxw - 2 * P));
    if (nstrip > 1 && maxw - 2 * P < 64) return BSF_EINVAL;
    const int Ws = (int)((W + nstrip - 1) / nstrip);
    // rows padded to an even number of elements: 16-byte aligned rows for the staged stencil's tensor map
    const int Hp = (int)H + 2 * P, Wp = (nstrip == 1 ? (int)W : Ws) + 2 * P, pitch = (Wp + 1) & ~1;
    const size_t per_img = (size_t)Hp * pitch * elem_bytes(mode);
    // images per launch: whole batch entries, bounded by a 16 GiB buffer budget
    const size_t budget = (size_t)16 << 30;
    int64_t bchunk = std::max<int64_t>(1, (int64_t)(budget / (per_img * (size_t)C)));
    bchunk = std::min<int64_t>(bchunk, B);
    *L = n4_layout{mode, nstrip, Ws, Hp, Wp, pitch, per_img, bchunk};
    return BSF_OK;
}

// one pass of the filter (the caller holds the context lock)
static bsf_status filter_pass(bsf_ctx* c, const void* image, int dtype, int64_t B, int64_t C, int64_t H, int64_t W,
                              const float* params, int kind, const bsf_opts& o, float* out, cudaStream_t st,
                              float ascale = 1.f) {
    const int64_t HW = H * W;
    int P = 0;
    bsf_status s = resolve_halo(c, params, kind, B, HW, o, st, &P);
    if (s != BSF_OK) return s;
    n4_layout lay;
    const bsf_status ls = n4_layout_of(dtype, B, C, H, W, P, o.precision, &lay);
    if (ls != BSF_OK) return ls;
    const int mode = lay.mode, nstrip = lay.nstrip, Ws = lay.Ws, Hp = lay.Hp, Wp = lay.Wp, pitch = lay.pitch;
    const size_t per_img = lay.per_img;
    const int64_t bchunk = lay.bchunk;
    const int K = (kind == BSF_PARAM_SCALES) ? 4 : 3;
    const size_t esz = (dtype == BSF_U8) ? 1 : 4;
    for (int64_t b0 = 0; b0 < B; b0 += bchunk) {
        const int64_t nbat = std::min<int64_t>(bchunk, B - b0);
        const int nimg = (int)(nbat * C);
        const scan_plan plan = make_scan_plan(Hp, Wp, nimg, elem_bytes(mode));
        if (!plan.ok) return BSF_EINVAL;
        BSF_TRY(grow(&c->buf, &c->buf_bytes, per_img * nimg));
        BSF_TRY(grow(&c->work, &c->work_bytes, plan.work_bytes));
        const char* img0 = (const char*)image + (size_t)(b0 * C) * HW * esz;
        for (int sidx = 0; sidx < nstrip; ++sidx) {
            const int col0 = sidx * Ws;
            const int ws = nstrip == 1 ? (int)W : std::min(Ws, (int)W - col0);
            BSF_TRY(prof_mark(c, 0, st));
            BSF_TRY(run_scan(mode, dtype, img0, (long long)HW, nimg, (int)H, (int)W, P, c->buf,
                             (long long)Hp * pitch, pitch, c->work, st, col0, nstrip == 1 ? 0 : ws,
                             o.boundary == BSF_BOUNDARY_REFLECT, c->d_status));
            stencil_args a;
            a.col0 = col0;
            a.Ws = nstrip == 1 ? 0 : ws;
            a.buf = c->buf;
            a.buf_stride = (long long)Hp * pitch;
            a.Hp = Hp;
            a.Wp = (nstrip == 1 ? (int)W : ws) + 2 * P;
            a.pitch = pitch;
            a.P = P;
            a.H = (int)H;
            a.W = (int)W;
            a.C = (int)C;
            a.nimg = nimg;
            a.params = params + (size_t)b0 * K * HW;
            a.kind = kind;
            a.eps = o.eps;
            a.eta = o.eta;
            a.ascale = ascale;
            a.out = out + (size_t)(b0 * C) * HW;
            a.status = c->d_status;
            a.staging = o.staging;
            a.polls = bsf_wait_limit();
            BSF_TRY(prof_mark(c, 1, st));
            BSF_TRY(launch_stencil4(mode, a, st));
            BSF_TRY(prof_mark(c, 2, st));
        }
    }
    return BSF_OK;
}

// the six-directional filter on the hexagonal lattice (hex6.cu); the caller
// holds the context lock.  One synchronisation: the windows are planned on the
// host from the largest footprint of every 16 x 16 block, which the scale map
// reduces.  Output tiles are 64 x 64 pixels, groups of them where the
// footprints are large, or 16 x 16 where the footprints are small: the window
// of a tile spans the tile plus the footprint, and the running sums over it
// grow with its size to the sixth power, so small kernels get small windows.
static bsf_status filter6(bsf_ctx* c, const void* image, int dtype, int64_t B, int64_t C, int64_t H, int64_t W,
                          const float* params, int kind, const bsf_opts& o, float* out, cudaStream_t st,
                          float ascale = 1.f) {
    const int fine = 16;
    const double h = (double)o.hex_spacing;
    const int64_t HW = H * W;
    const int fx = (int)((W + fine - 1) / fine), fy = (int)((H + fine - 1) / fine);
    const int64_t nfine = (int64_t)fx * fy;
    const size_t ext_bytes = (size_t)B * nfine * 2 * sizeof(unsigned);
    BSF_TRY(grow(&c->h6_scales, &c->h6_scales_bytes, (size_t)B * 6 * HW * sizeof(double)));
    BSF_TRY(grow(&c->h6_ext, &c->h6_ext_bytes, ext_bytes));
    BSF_TRY(cudaMemsetAsync(c->h6_ext, 0, ext_bytes, st));
    BSF_TRY(prof_mark(c, 0, st));
    const float* lut = nullptr;
    if (kind != BSF_PARAM_SCALES) BSF_TRY(map6_table(c, o, st, &lut));
    BSF_TRY(launch_map6(params, kind, (int)B, (int)H, (int)W, fine, o.eps, o.eta, o.rel_bound, ascale, (double*)c->h6_scales,
                        (unsigned*)c->h6_ext, c->d_status, st, lut));
    std::vector<unsigned> ext((size_t)B * nfine * 2);
    BSF_TRY(cudaMemcpyAsync(ext.data(), c->h6_ext, ext_bytes, cudaMemcpyDeviceToHost, st));
    BSF_TRY(cudaStreamSynchronize(st));
    std::vector<hex6_tile> tl;
    std::vector<hex6_chunk> chunks;
    // chunks of at most 8 GiB of windows: enough windows of the largest
    // footprints for several blocks of the pre-integration on every SM
    const bsf_status ps = hex6_plan(B, C, H, W, h, ext.data(), (size_t)8 << 30, tl, chunks);
    if (ps != BSF_OK) return ps;
    size_t win = 0;
    for (auto& ch : chunks) win = std::max(win, ch.bytes);
    if (tl.empty()) return BSF_OK;
    BSF_TRY(grow(&c->h6_tiles, &c->h6_tiles_bytes, tl.size() * sizeof(hex6_tile)));
    // two window buffers: chunk i + 1 is pre-integrated on the side stream while the stencil
    // of chunk i runs on st; a buffer is reused only after the stencil that read it
    const size_t win_al = (win + 255) & ~(size_t)255;
    BSF_TRY(grow(&c->h6_win, &c->h6_win_bytes, 2 * win_al));
    size_t most = 0;
    for (auto& ch : chunks) most = std::max(most, ch.last - ch.first);
    const size_t flag_al = (most * (size_t)C * sizeof(unsigned) + 255) & ~(size_t)255;
    BSF_TRY(grow(&c->h6_flag, &c->h6_flag_bytes, 2 * flag_al));
    if (!c->h6_side) {
        BSF_TRY(cudaStreamCreateWithFlags(&c->h6_side, cudaStreamNonBlocking));
        for (cudaEvent_t* e : {&c->h6_ev_tiles, &c->h6_ev_pre[0], &c->h6_ev_pre[1], &c->h6_ev_st[0], &c->h6_ev_st[1]})
            BSF_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    cudaStream_t side = c->h6_side;
    BSF_TRY(cudaMemcpyAsync(c->h6_tiles, tl.data(), tl.size() * sizeof(hex6_tile), cudaMemcpyHostToDevice, st));
    // the side stream starts after everything enqueued on st so far (the image, the scales, the tiles)
    BSF_TRY(cudaEventRecord(c->h6_ev_tiles, st));
    BSF_TRY(cudaStreamWaitEvent(side, c->h6_ev_tiles, 0));
    const hex6_tile* dt = (const hex6_tile*)c->h6_tiles;
    for (size_t i = 0; i < chunks.size(); ++i) {
        const hex6_chunk& ch = chunks[i];
        const int n = (int)(ch.last - ch.first);
        const int k = (int)(i & 1);
        void* win_k = (char*)c->h6_win + k * win_al;
        unsigned* flag_k = (unsigned*)((char*)c->h6_flag + k * flag_al);
        if (i >= 2) BSF_TRY(cudaStreamWaitEvent(side, c->h6_ev_st[k], 0));
        if (i > 0) BSF_TRY(prof_mark(c, 0, side));
        BSF_TRY(launch_hex6_preint(dtype == BSF_U8, image, (int)C, (int)H, (int)W, h, dt + ch.first, n, ch.cols,
                                   win_k, flag_k, side, o.boundary == BSF_BOUNDARY_REFLECT));
        BSF_TRY(prof_mark(c, 1, side));
        BSF_TRY(cudaEventRecord(c->h6_ev_pre[k], side));
        BSF_TRY(cudaStreamWaitEvent(st, c->h6_ev_pre[k], 0));
        BSF_TRY(prof_mark(c, 3, st));
        BSF_TRY(launch_hex6_stencil((const double*)c->h6_scales, (int)C, (int)H, (int)W, tl[ch.first].w,
                                    tl[ch.first].hh, h, dt + ch.first, n, win_k, (const unsigned*)flag_k, out,
                                    c->d_status, st));
        BSF_TRY(cudaEventRecord(c->h6_ev_st[k], st));
        BSF_TRY(prof_mark(c, 2, st));
    }
    return BSF_OK;
}

// argument checks shared by bsf_filter and bsf_filter_host
static bsf_status filter_args(bsf_ctx* c, const void* image, int dtype, int64_t B, int64_t C, int64_t H, int64_t W,
                              int N, const float* params, int kind, const bsf_opts* opts, const float* out,
                              bsf_opts* o) {
    if (!c || !image || !params || !out) return BSF_EINVAL;
    if (B <= 0 || C <= 0 || !dims_ok(H, W)) return BSF_EINVAL;
    if (dtype != BSF_U8 && dtype != BSF_F32) return BSF_EINVAL;
    if (kind != BSF_PARAM_SCALES && kind != BSF_PARAM_COV && kind != BSF_PARAM_SRT) return BSF_EINVAL;
    if (N != 4 && N != 6) return BSF_EUNSUPPORTED;
    bsf_default_opts(o);
    if (opts) *o = *opts;
    if (o->precision != BSF_PREC_EXACT && o->precision != BSF_PREC_FP64) return BSF_EINVAL;
    if (o->iterations < 1 || o->iterations > 64) return BSF_EINVAL;
    if (o->boundary != BSF_BOUNDARY_ZERO && o->boundary != BSF_BOUNDARY_REFLECT) return BSF_EINVAL;
    if (N == 6 && !(o->rel_bound >= 0.f && o->rel_bound < 1.f / 6.f)) return BSF_EINVAL;
    if (N == 6 && !(o->hex_spacing == 1.f || o->hex_spacing == 0.5f || o->hex_spacing == 0.25f ||
                    o->hex_spacing == 0.125f))
        return BSF_EINVAL;
    return BSF_OK;
}

// the filter on device buffers, enqueued on st (the caller holds the context lock)
static bsf_status any_pass(bsf_ctx* c, int N, const void* image, int dtype, int64_t B, int64_t C, int64_t H,
                           int64_t W, const float* params, int kind, const bsf_opts& o, float* out, cudaStream_t st,
                           float ascale = 1.f) {
    if (N == 6) return filter6(c, image, dtype, B, C, H, W, params, kind, o, out, st, ascale);
    return filter_pass(c, image, dtype, B, C, H, W, params, kind, o, out, st, ascale);
}

static bsf_status filter_locked(bsf_ctx* c, const void* image, int dtype, int64_t B, int64_t C, int64_t H, int64_t W,
                                const float* params, int kind, const bsf_opts& o, float* out, cudaStream_t st,
                                int N = 4) {
    const int64_t HW = H * W;
    bsf_status s;
    if (o.iterations == 1) {
        s = any_pass(c, N, image, dtype, B, C, H, W, params, kind, o, out, st);
    } else {
        // iterated box spline (Sec. 3.3): m passes, each with the widths a / sqrt(m)
        // of the optimal scale vector a (the mapped widths are scaled, so the
        // covariance of each pass is C / m)
        const int m = o.iterations;
        const float asc = 1.f / sqrtf((float)m);
        const size_t ibytes = (size_t)B * C * HW * sizeof(float);
        BSF_TRY(grow(&c->iter, &c->iter_bytes, ibytes));
        float* tmp = (float*)c->iter;
        bsf_opts oi = o;
        if (o.max_scale > 0.f) oi.max_scale = o.max_scale * asc;
        // the halo of the unscaled field covers the scaled one; passes alternate
        // between tmp and out so that the last one lands in out
        float* dst = (m % 2 == 0) ? tmp : out;
        s = any_pass(c, N, image, dtype, B, C, H, W, params, kind, oi, dst, st, asc);
        for (int it = 1; it < m && s == BSF_OK; ++it) {
            float* src = dst;
            dst = (src == tmp) ? out : tmp;
            s = any_pass(c, N, src, BSF_F32, B, C, H, W, params, kind, oi, dst, st, asc);
        }
    }
    if (s != BSF_OK) return s;
    if (o.strict) {
        unsigned h = 0;
        BSF_TRY(cudaMemcpyAsync(&h, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        BSF_TRY(cudaStreamSynchronize(st));
        if (h & (1u << BSF_EINFEASIBLE)) return BSF_EINFEASIBLE;
    }
    return BSF_OK;
}

bsf_status bsf_query_workspace(bsf_ctx* c, int dtype, int64_t B, int64_t C, int64_t H, int64_t W, int N, int kind,
                               const bsf_opts* opts, size_t* bytes) {
    (void)c;
    if (!bytes || B <= 0 || C <= 0 || !dims_ok(H, W)) return BSF_EINVAL;
    if (dtype != BSF_U8 && dtype != BSF_F32) return BSF_EINVAL;
    if (kind != BSF_PARAM_SCALES && kind != BSF_PARAM_COV && kind != BSF_PARAM_SRT) return BSF_EINVAL;
    if (N != 4 && N != 6) return BSF_EUNSUPPORTED;
    bsf_opts o;
    bsf_default_opts(&o);
    if (opts) o = *opts;
    if (o.iterations < 1 || o.iterations > 64) return BSF_EINVAL;
    const int64_t HW = H * W;
    size_t total = o.iterations > 1 ? (size_t)B * C * HW * sizeof(float) : 0;  // intermediate image
    if (N == 4) {
        int P = o.halo;
        if (P <= 0) {
            // the halo rule of the filter; without halo or max_scale it depends on the field
            if (!(o.max_scale > 0.f) || o.max_scale > 1e5f) return BSF_EINVAL;
            const float ext = (kind == BSF_PARAM_SCALES) ? 2.41422f * o.max_scale : 8.3640f * o.max_scale;
            P = (int)ceilf(0.5f * ext) + 4;
        }
        if (P > kMaxHalo) return BSF_EINVAL;
        n4_layout lay;
        const bsf_status ls = n4_layout_of(dtype, B, C, H, W, P, o.precision, &lay);
        if (ls != BSF_OK) return ls;
        const int nimg = (int)(lay.bchunk * C);
        const scan_plan plan = make_scan_plan(lay.Hp, lay.Wp, nimg, elem_bytes(lay.mode));
        if (!plan.ok) return BSF_EINVAL;
        total += lay.per_img * (size_t)nimg + plan.work_bytes;
    } else {
        // an upper bound: the per-pixel scales and block extents, and windows of
        // 16 x 16 tiles at the largest footprint the bound allows (the planner's
        // 64-pixel tiles and tile groups need less per pixel), capped by its 8 GiB
        // chunk; tile records and window flags for every 16 x 16 tile
        if (!(o.max_scale > 0.f) || o.max_scale > 1e5f) return BSF_EINVAL;
        const double amax = kind == BSF_PARAM_SCALES ? (double)o.max_scale : sqrt(24.0) * o.max_scale;
        const double e = 0.5 * amax * 3.7320508075688772;  // sum_k |cos theta_k| = sum_k sin theta_k = 2 + sqrt3
        const int64_t tiles = B * ((H + 15) / 16) * ((W + 15) / 16);
        hex6_tile t;
        hex6_window(0, 0, 16, 16, (int)H, (int)W, e, e, (double)o.hex_spacing, &t);
        const double win = (double)tiles * C * t.ncol * t.nrow * 16.0;
        total += (size_t)B * 6 * HW * sizeof(double) + (size_t)tiles * 2 * sizeof(unsigned) +
                 (size_t)tiles * (sizeof(hex6_tile) + C * sizeof(unsigned)) +
                 2 * (size_t)std::min(win, (double)((size_t)8 << 30)) +  // two window buffers
                 (o.map_lut ? lut6_bytes() : 0);                           // the map's table
    }
    *bytes = total;
    return BSF_OK;
}

bsf_status bsf_filter(bsf_ctx* c, const void* image, int dtype, int64_t B, int64_t C, int64_t H, int64_t W, int N,
                      const float* params, int kind, const bsf_opts* opts, float* out, void* stream) {
    bsf_opts o;
    const bsf_status a = filter_args(c, image, dtype, B, C, H, W, N, params, kind, opts, out, &o);
    if (a != BSF_OK) return a;
    std::lock_guard<std::mutex> lock(c->mu);
    BSF_TRY(cudaSetDevice(c->device));
    return filter_locked(c, image, dtype, B, C, H, W, params, kind, o, out, (cudaStream_t)stream, N);
}

// Slot buffers grow only while no enqueued work of the pipeline is in flight.
static cudaError_t host_grow(bsf_ctx* c, void** p, size_t* cur, size_t need) {
    if (need <= *cur) return cudaSuccess;
    for (cudaStream_t s_ : {c->s_h2d, c->s_comp, c->s_d2h}) {
        cudaError_t e = cudaStreamSynchronize(s_);
        if (e != cudaSuccess) return e;
    }
    return grow(p, cur, need);
}

bsf_status bsf_filter_host(bsf_ctx* c, const void* image_host, int dtype, int64_t B, int64_t C, int64_t H, int64_t W,
                           int N, const float* params_host, int kind, const bsf_opts* opts, float* out_host) {
    bsf_opts o;
    const bsf_status a = filter_args(c, image_host, dtype, B, C, H, W, N, params_host, kind, opts, out_host, &o);
    if (a != BSF_OK) return a;
    std::lock_guard<std::mutex> lock(c->mu);
    BSF_TRY(cudaSetDevice(c->device));
    if (!c->s_h2d) {
        BSF_TRY(cudaStreamCreateWithFlags(&c->s_h2d, cudaStreamNonBlocking));
        BSF_TRY(cudaStreamCreateWithFlags(&c->s_comp, cudaStreamNonBlocking));
        BSF_TRY(cudaStreamCreateWithFlags(&c->s_d2h, cudaStreamNonBlocking));
        for (auto& h : c->hs) {
            BSF_TRY(cudaEventCreateWithFlags(&h.in_ready, cudaEventDisableTiming));
            BSF_TRY(cudaEventCreateWithFlags(&h.comp_done, cudaEventDisableTiming));
            BSF_TRY(cudaEventCreateWithFlags(&h.out_done, cudaEventDisableTiming));
        }
    }
    auto& h = c->hs[c->host_calls & 1];
    const int K = (kind == BSF_PARAM_SCALES) ? N : 3;
    const size_t ib = (size_t)(B * C * H * W) * (dtype == BSF_U8 ? 1 : 4);
    const size_t pb = (size_t)(B * K * H * W) * sizeof(float);
    const size_t ob = (size_t)(B * C * H * W) * sizeof(float);
    BSF_TRY(host_grow(c, &h.img, &h.img_bytes, ib));
    BSF_TRY(host_grow(c, &h.prm, &h.prm_bytes, pb));
    BSF_TRY(host_grow(c, &h.out, &h.out_bytes, ob));
    // inputs of this slot are overwritten once the kernels of its previous call have read them
    BSF_TRY(cudaStreamWaitEvent(c->s_h2d, h.comp_done, 0));
    BSF_TRY(cudaMemcpyAsync(h.img, image_host, ib, cudaMemcpyHostToDevice, c->s_h2d));
    BSF_TRY(cudaMemcpyAsync(h.prm, params_host, pb, cudaMemcpyHostToDevice, c->s_h2d));
    BSF_TRY(cudaEventRecord(h.in_ready, c->s_h2d));
    // the output of this slot is overwritten once its previous copy-out has finished
    BSF_TRY(cudaStreamWaitEvent(c->s_comp, h.in_ready, 0));
    BSF_TRY(cudaStreamWaitEvent(c->s_comp, h.out_done, 0));
    const bsf_status s = filter_locked(c, h.img, dtype, B, C, H, W, (const float*)h.prm, kind, o, (float*)h.out,
                                       c->s_comp, N);
    if (s != BSF_OK) return s;
    BSF_TRY(cudaEventRecord(h.comp_done, c->s_comp));
    BSF_TRY(cudaStreamWaitEvent(c->s_d2h, h.comp_done, 0));
    BSF_TRY(cudaMemcpyAsync(out_host, h.out, ob, cudaMemcpyDeviceToHost, c->s_d2h));
    BSF_TRY(cudaEventRecord(h.out_done, c->s_d2h));
    ++c->host_calls;
    return BSF_OK;
}

bsf_status bsf_host_sync(bsf_ctx* c) {
    if (!c) return BSF_EINVAL;
    std::lock_guard<std::mutex> lock(c->mu);
    if (!c->s_h2d) return BSF_OK;
    BSF_TRY(cudaSetDevice(c->device));
    for (cudaStream_t s_ : {c->s_h2d, c->s_comp, c->s_d2h}) BSF_TRY(cudaStreamSynchronize(s_));
    return BSF_OK;
}

bsf_status bsf_structure_cov(bsf_ctx* c, const void* image, int dtype, int64_t B, int64_t C, int64_t H, int64_t W,
                             float sigma_w, float sigma0, float tau, float* cov, void* stream) {
    if (!c || !image || !cov) return BSF_EINVAL;
    if (B <= 0 || C <= 0 || !dims_ok(H, W)) return BSF_EINVAL;
    if (dtype != BSF_U8 && dtype != BSF_F32) return BSF_EINVAL;
    if (!(sigma_w > 0.f && sigma_w < 1e4f) || !(sigma0 > 0.f && sigma0 < 1e4f) || !(tau > 0.f && tau < 1e30f))
        return BSF_EINVAL;
    std::lock_guard<std::mutex> lock(c->mu);
    BSF_TRY(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t HW = H * W;
    const size_t n3 = (size_t)(3 * B * HW);
    BSF_TRY(grow(&c->stbuf, &c->stbuf_bytes, (2 * n3 + (size_t)(4 * B * HW)) * sizeof(float)));
    float* prod = (float*)c->stbuf;
    float* J = prod + n3;
    float* prm = J + n3;
    BSF_TRY(launch_st_products(image, dtype == BSF_U8, (int)B, (int)C, (int)H, (int)W, prod, st));
    // the window: the isotropic box spline with the covariance of a Gaussian of std sigma_w
    const float a = sigma_w * 2.44948974278317810f;
    BSF_TRY(launch_fill(prm, (size_t)(4 * B * HW), a, st));
    bsf_opts o;
    bsf_default_opts(&o);
    o.max_scale = a;
    const bsf_status s = filter_locked(c, prod, BSF_F32, B, 3, H, W, prm, BSF_PARAM_SCALES, o, J, st);
    if (s != BSF_OK) return s;
    BSF_TRY(launch_adaptive_cov(J, (long long)HW, (int)B, sigma0 * sigma0, tau, cov, st));
    return BSF_OK;
}

// One backward pass of the filter with widths a * ascale on the input x
// (dtype): the image gradient into gimage (nullable) and the scale gradient,
// multiplied by ascale, added into gscales (nullable; zeroed by the caller).
static bsf_status backward_pass(bsf_ctx* c, const void* x, int dtype, int64_t B, int64_t C, int64_t H, int64_t W,
                                const float* scales, const float* gout, float* gimage, float* gscales, int P,
                                float ascale, cudaStream_t st) {
    const int64_t HW = H * W;
    const int mode = mode_of(dtype, BSF_PREC_EXACT);
    const int Hp = (int)H + 2 * P, Wp = (int)W + 2 * P, pitch = Wp;
    const size_t per_img = (size_t)Hp * pitch * elem_bytes(mode);
    const size_t per_h = (size_t)Hp * pitch * sizeof(double);
    const size_t budget = (size_t)16 << 30;
    int64_t bchunk = std::max<int64_t>(1, (int64_t)(budget / ((per_img + per_h) * (size_t)C)));
    bchunk = std::min<int64_t>(bchunk, B);
    const size_t esz = (dtype == BSF_U8) ? 1 : 4;
    for (int64_t b0 = 0; b0 < B; b0 += bchunk) {
        const int64_t nbat = std::min<int64_t>(bchunk, B - b0);
        const int nimg = (int)(nbat * C);
        const scan_plan plan = make_scan_plan(Hp, Wp, nimg, elem_bytes(mode));
        BSF_TRY(grow(&c->buf, &c->buf_bytes, per_img * nimg));
        BSF_TRY(grow(&c->work, &c->work_bytes, plan.work_bytes));
        double* hb = nullptr;
        if (gimage) {
            BSF_TRY(grow(&c->hbuf, &c->hbuf_bytes, per_h * nimg));
            hb = (double*)c->hbuf;
            BSF_TRY(cudaMemsetAsync(hb, 0, per_h * nimg, st));
        }
        const char* img0 = (const char*)x + (size_t)(b0 * C) * HW * esz;
        BSF_TRY(run_scan(mode, dtype, img0, (long long)HW, nimg, (int)H, (int)W, P, c->buf, (long long)Hp * pitch,
                         pitch, c->work, st, 0, 0, 0, c->d_status));
        BSF_TRY(launch_grad4(mode, c->buf, (long long)Hp * pitch, Hp, Wp, pitch, P, (int)H, (int)W, (int)C, nimg,
                             scales + (size_t)b0 * 4 * HW, gout + (size_t)(b0 * C) * HW,
                             gscales ? gscales + (size_t)b0 * 4 * HW : nullptr, hb, ascale, c->d_status, st));
        if (gimage)
            BSF_TRY(launch_transpose_scans(hb, nimg, Hp, Wp, pitch, P, (int)H, (int)W, gimage + (size_t)(b0 * C) * HW,
                                           st));
    }
    return BSF_OK;
}

bsf_status bsf_filter_backward(bsf_ctx* c, const void* image, int dtype, int64_t B, int64_t C, int64_t H, int64_t W,
                               int N, const float* scales, const float* grad_out, float* grad_image,
                               float* grad_scales, const bsf_opts* opts, void* stream) {
    if (!c || !image || !scales || !grad_out) return BSF_EINVAL;
    if (!grad_image && !grad_scales) return BSF_EINVAL;
    if (B <= 0 || C <= 0 || !dims_ok(H, W)) return BSF_EINVAL;
    if (dtype != BSF_U8 && dtype != BSF_F32) return BSF_EINVAL;
    if (N != 4) return BSF_EUNSUPPORTED;
    bsf_opts o;
    bsf_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision != BSF_PREC_EXACT) return BSF_EUNSUPPORTED;
    if (o.boundary != BSF_BOUNDARY_ZERO) return BSF_EUNSUPPORTED;  // the adjoint is written for f = 0 outside
    if (o.iterations < 1 || o.iterations > 64) return BSF_EINVAL;
    std::lock_guard<std::mutex> lock(c->mu);
    BSF_TRY(cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t HW = H * W;
    int P = 0;
    bsf_status s = resolve_halo(c, scales, BSF_PARAM_SCALES, B, HW, o, st, &P);
    if (s != BSF_OK) return s;
    // rows wider than one band CTA holds are rejected before anything runs (the adjoint has no strips)
    {
        const int mode = mode_of(dtype, o.precision);
        const int Hp = (int)H + 2 * P, Wp = (int)W + 2 * P;
        const size_t per = (size_t)Hp * Wp * (elem_bytes(mode) + sizeof(double)) * (size_t)C;
        const int64_t bchunk = std::min<int64_t>(B, std::max<int64_t>(1, (int64_t)(((size_t)16 << 30) / per)));
        if (!make_scan_plan(Hp, Wp, (int)(bchunk * C), elem_bytes(mode)).ok) return BSF_EINVAL;
        if (dtype == BSF_U8 && o.iterations > 1 &&
            !make_scan_plan(Hp, Wp, (int)(bchunk * C), elem_bytes(MODE_U128)).ok)
            return BSF_EINVAL;  // later passes run on float32 intermediates
    }
    if (grad_scales) BSF_TRY(cudaMemsetAsync(grad_scales, 0, (size_t)B * 4 * HW * sizeof(float), st));
    if (o.iterations == 1)
        return backward_pass(c, image, dtype, B, C, H, W, scales, grad_out, grad_image, grad_scales, P, 1.f, st);
    // iterated filter (Sec. 3.3): m passes with the widths a / sqrt(m).  The
    // forward intermediates f_1 .. f_{m-1} are recomputed and kept; the passes
    // are then differentiated in reverse, each image gradient feeding the next
    // and every pass adding its scale gradient (times 1/sqrt(m)).
    const int m = o.iterations;
    const float asc = 1.f / sqrtf((float)m);
    const size_t n = (size_t)(B * C * HW);
    BSF_TRY(grow(&c->iter, &c->iter_bytes, (size_t)(m + 1) * n * sizeof(float)));
    float* fk = (float*)c->iter;          // f_1 .. f_{m-1}
    float* g0 = fk + (size_t)(m - 1) * n;  // gradient ping-pong
    float* g1 = g0 + n;
    bsf_opts of = o;
    of.iterations = 1;
    if (o.max_scale > 0.f) of.max_scale = o.max_scale * asc;
    of.halo = P;
    for (int k = 1; k < m; ++k) {
        s = filter_pass(c, k == 1 ? image : (const void*)(fk + (size_t)(k - 2) * n), k == 1 ? dtype : BSF_F32, B, C,
                        H, W, scales, BSF_PARAM_SCALES, of, fk + (size_t)(k - 1) * n, st, asc);
        if (s != BSF_OK) return s;
    }
    const float* g = grad_out;
    for (int k = m; k >= 1; --k) {
        const void* x = k == 1 ? image : (const void*)(fk + (size_t)(k - 2) * n);
        float* gi = k == 1 ? grad_image : (g == g0 ? g1 : g0);
        s = backward_pass(c, x, k == 1 ? dtype : BSF_F32, B, C, H, W, scales, g, gi, grad_scales, P, asc, st);
        if (s != BSF_OK) return s;
        g = gi;
    }
    return BSF_OK;
}

bsf_status bsf_preintegrate(bsf_ctx* c, const void* image, int dtype, int64_t H, int64_t W, int N, int halo,
                            int precision, void* buffer, void* stream) {
    if (!c || !image || !buffer || !dims_ok(H, W) || halo < 2 || halo > kMaxHalo) return BSF_EINVAL;
    if (dtype != BSF_U8 && dtype != BSF_F32) return BSF_EINVAL;
    if (precision != BSF_PREC_EXACT && precision != BSF_PREC_FP64) return BSF_EINVAL;
    if (N != 4) return BSF_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(c->mu);
    BSF_TRY(cudaSetDevice(c->device));
    const int mode = mode_of(dtype, precision);
    const int Hp = (int)H + 2 * halo, Wp = (int)W + 2 * halo;
    const scan_plan plan = make_scan_plan(Hp, Wp, 1, elem_bytes(mode));
    if (!plan.ok) return BSF_EINVAL;  // a row wider than one band CTA holds (bsf_filter uses strips)
    BSF_TRY(grow(&c->work, &c->work_bytes, plan.work_bytes));
    BSF_TRY(run_scan(mode, dtype, image, (long long)H * W, 1, (int)H, (int)W, halo, buffer, (long long)Hp * Wp, Wp,
                     c->work, (cudaStream_t)stream, 0, 0, 0, c->d_status));
    return BSF_OK;
}

bsf_status bsf_apply(bsf_ctx* c, const void* buffer, int dtype, int64_t H, int64_t W, int N, int halo,
                     const float* params, int kind, const bsf_opts* opts, float* out, void* stream) {
    if (!c || !buffer || !params || !out || !dims_ok(H, W) || halo < 2 || halo > kMaxHalo) return BSF_EINVAL;
    if (dtype != BSF_U8 && dtype != BSF_F32) return BSF_EINVAL;
    if (kind != BSF_PARAM_SCALES && kind != BSF_PARAM_COV && kind != BSF_PARAM_SRT) return BSF_EINVAL;
    if (N != 4) return BSF_EUNSUPPORTED;
    bsf_opts o;
    bsf_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision != BSF_PREC_EXACT && o.precision != BSF_PREC_FP64) return BSF_EINVAL;
    BSF_TRY(cudaSetDevice(c->device));
    const int mode = mode_of(dtype, o.precision);
    stencil_args a;
    a.buf = buffer;
    a.buf_stride = 0;
    a.Hp = (int)H + 2 * halo;
    a.Wp = (int)W + 2 * halo;
    a.pitch = a.Wp;
    a.P = halo;
    a.H = (int)H;
    a.W = (int)W;
    a.C = 1;
    a.nimg = 1;
    a.params = params;
    a.kind = kind;
    a.eps = o.eps;
    a.eta = o.eta;
    a.out = out;
    a.status = c->d_status;
    BSF_TRY(launch_stencil4(mode, a, (cudaStream_t)stream));
    return BSF_OK;
}

}  // extern "C"
