// Host-side declarations shared by the translation units of libbsf.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

struct scan_plan {
    int band_h;         // rows per band
    int nb;             // bands per image
    int cpt;            // columns per thread in the band kernel
    int threads;        // threads per band CTA
    size_t work_bytes;  // carry workspace for all images of one launch
    size_t smem;        // dynamic shared memory of the band kernel (g2 state)
    bool ok;            // false: the row is too wide for one CTA
};

// largest halo (padding of the pre-integrated buffer, px) any entry point accepts: with
// H, W <= 2^20 the padded sizes and byte counts then stay far inside int and size_t
constexpr int kMaxHalo = 1 << 20;

scan_plan make_scan_plan(int Hp, int Wp, int nimg, size_t elem_bytes);
// widest buffer row one band CTA holds; narrow: the width at which the 128-bit
// form keeps four columns per thread (chosen for batches of several waves)
int scan_max_width(size_t elem_bytes, bool narrow = false);

// Pre-integration (RS1-RS4) of nimg images of H x W (stride img_stride
// elements) into buffers of Hp x pitch elements (stride G_stride elements).
// The buffer covers the image columns [col0 - P, col0 + Ws + P) (Ws <= 0:
// the whole width, col0 = 0), f taken as zero outside the image, or (reflect)
// as its half-sample symmetric extension over the whole buffer.  The carries
// between row bands run as one cooperative kernel whose grid barriers give up
// after spin_limit polls (0: the default bound) and raise BSF_ETIMEOUT in
// *status (if given) instead of waiting forever.
template <int MODE, class InT>
cudaError_t launch_scan4(const InT* img, long long img_stride, int nimg, int H, int W, int P, void* G,
                         long long G_stride, int pitch, void* work, cudaStream_t st, int col0 = 0, int Ws = 0,
                         int reflect = 0, unsigned* status = nullptr, unsigned spin_limit = 0);

// the process-wide bound of the device waits between row bands (bsf_set_wait_limit; 0 = default)
unsigned bsf_wait_limit();

// index i of the half-sample symmetric extension of 0..n-1 (period 2n: -1 -> 0, n -> n-1)
__host__ __device__ __forceinline__ int reflect_index(int i, int n) {
    const int p = 2 * n;
    int k = i % p;
    if (k < 0) k += p;
    return k < n ? k : p - 1 - k;
}

struct stencil_args {
    int col0 = 0;          // first output column of the strip the buffer covers
    int Ws = 0;            // its width (0: the whole image)
    const void* buf;
    long long buf_stride;  // elements between consecutive images' buffers
    int Hp, Wp, pitch, P, H, W;
    int C;                 // channels sharing one parameter field
    int nimg;              // images in this launch (a multiple of C)
    const float* params;   // parameter planes of the first image's field
    int kind;
    float eps, eta;
    float ascale = 1.f;    // widths multiplier (1/sqrt(m) in a pass of the m-fold iterated filter)
    float* out;
    unsigned* status;
    int staging = 0;       // opts.staging: BSF_STAGING_TMA selects the TMA-staged form (64-bit exact mode)
    unsigned polls = 0;    // bound of its waits (0: the default)
};

cudaError_t launch_stencil4(int mode, const stencil_args& a, cudaStream_t st);
cudaError_t launch_map4(const float* params, int kind, long long npix, float eps, float eta, float* scales,
                        uint8_t* flags, cudaStream_t st);
cudaError_t launch_extent4(const float* params, int kind, long long npix, float eps, float eta, unsigned* ext_bits,
                           cudaStream_t st);

// Adjoint (adjoint4.cu).
// ascale multiplies the widths (1/sqrt(m) in a pass of the m-fold iterated
// filter) and, by the chain rule, the scale gradient
cudaError_t launch_grad4(int mode, const void* buf, long long buf_stride, int Hp, int Wp, int pitch, int P, int H,
                         int W, int C, int nimg, const float* scales, const float* gout, float* gscales, double* hbuf,
                         float ascale, unsigned* status, cudaStream_t st);
cudaError_t launch_transpose_scans(double* hbuf, int nimg, int Hp, int Wp, int pitch, int P, int H, int W,
                                   float* gimage, cudaStream_t st);

// Feature-preserving smoothing (adaptive.cu).
cudaError_t launch_st_products(const void* img, int dtype_u8, int B, int C, int H, int W, float* prod,
                               cudaStream_t st);
cudaError_t launch_fill(float* p, size_t n, float v, cudaStream_t st);
cudaError_t launch_adaptive_cov(const float* J, long long HW, int B, float s0sq, float tau, float* cov,
                                cudaStream_t st);

// Six-directional filter on the hexagonal lattice (hex6.cu; planning in hex6_plan.cpp).
// One lattice window per (batch entry, output tile of 64 x 64 pixels; 16 x 16
// where the footprints are small; groups of 2 x 1, 4 x 1 or 4 x 2 64-tiles where
// they are large); channel c of the tile's image has its window at
// off + c * ncol * nrow elements (exact 128-bit running sums).
constexpr int HEX6_PRE_THREADS = 832;  // largest block of the pre-integration
constexpr int HEX6_PRE_CPT = 4;        // window columns per pre-integration thread
constexpr int HEX6_PRE_PAD = 8;        // one padding element per this many columns of a state row
struct hex6_tile {
    long long off;   // 16-byte elements from the chunk's window base
    int i_left;      // lattice column i of storage column 0 in row 0
    int j0w;         // lattice row j of storage row 0
    int ncol, nrow;  // storage size; column c of row r is lattice point (c + i_left - 2 r, j0w + r)
    int b;           // batch entry
    int x0, y0;      // first output pixel of the tile
    int w, hh;       // tile shape in pixels: 16 x 16, or 64, 128, 256 x 64, 128
};
// a run of tiles of one shape whose windows share one buffer
struct hex6_chunk {
    size_t first, last;  // tiles [first, last) of the plan
    int cols;            // widest window
    size_t bytes;        // windows of all channels
};
void hex6_window(int x0, int y0, int w, int hh, int H, int W, double ex, double ey, double h, hex6_tile* t);
int hex6_max_cols();
// tile records and chunks (at most `budget` bytes of windows and 65535 tiles,
// one tile shape each) from the largest footprint half-extents of every 16 x 16
// block: ext holds B * ceil(H/16) * ceil(W/16) pairs (ex, ey) as FP32 bits.
// BSF_EINVAL: an extent not finite or above 1e5 px, or a window too wide.
int hex6_plan(int64_t B, int64_t C, int64_t H, int64_t W, double h, const unsigned* ext, size_t budget,
              std::vector<hex6_tile>& tiles, std::vector<hex6_chunk>& chunks);
// rel: the lower bound p_k >= max(eps, rel * sum p) of the six-directional map (opts.rel_bound).
// lut: null, or the table of launch_lut6_build for the same (eta, rel) (opts.map_lut)
cudaError_t launch_map6(const float* params, int kind, int B, int H, int W, int tile, double eps, double eta,
                        double rel, double ascale, double* scales, unsigned* tile_ext, unsigned* status,
                        cudaStream_t st, const float* lut);
cudaError_t launch_map6_out(const float* params, int kind, long long npix, double eps, double eta, double rel,
                            float* scales, uint8_t* flags, cudaStream_t st, const float* lut);
// the six-directional map at sigma = 1 on a (ln rho, theta) grid: lut6_bytes() bytes of device memory
size_t lut6_bytes();
cudaError_t launch_lut6_build(double eta, double rel, float* table, cudaStream_t st);
cudaError_t launch_hex6_preint(int dtype_u8, const void* img, int C, int H, int W, double h, const hex6_tile* tiles,
                               int ntiles, int ncol_max, void* scratch, unsigned* wflag, cudaStream_t st,
                               int reflect = 0);
cudaError_t launch_hex6_stencil(const double* scales, int C, int H, int W, int tile_w, int tile_h, double h,
                                const hex6_tile* tiles, int ntiles, const void* scratch, const unsigned* wflag,
                                float* out, unsigned* status, cudaStream_t st);
