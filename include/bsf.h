/*
 * bsf.h -- C ABI of the GB300 space-variant elliptical box-spline filter.
 *
 * The library computes, for an image f[n] and a per-pixel scale vector a(n),
 *
 *     fbar[n] = sum_k f[k] beta^N_{a(n)}(n - k)                      (1)
 *
 * where beta^N_a is the radially-uniform box spline of Chaudhury,
 * Munoz-Barrutia and Unser, "Fast space-variant elliptical filtering using
 * box splines", Sec. 2.2.1, Eq. (const): the convolution of N box
 * distributions of widths a_k along theta_k = (k-1) pi / N.  (1) is
 * Eq. (SVF_2D) with the Dirac-comb image used to derive Eq. (keyeqn).  The
 * path is Algorithm 1 of Sec. 3.1: pre-integration by four running sums
 * (RS1-RS4), then a 16-tap finite difference (Table 1, Eq. final_eqn) of the
 * Zwart-Powell interpolant of the pre-integrated image (App. F).  Scale
 * vectors may be given directly, or derived per pixel from a covariance by
 * the optimal-scale algorithm of Sec. 3.2.2.
 *
 * Conventions shared by every entry point:
 *   - Points n = (n1, n2): n1 is the column, n2 the row (rows grow downward in
 *     memory).  theta is measured from +n1 towards +n2, so the four
 *     directions are (1,0), (1,1)/sqrt2, (0,1), (-1,1)/sqrt2.
 *   - Images are dense row-major arrays of B*C*H*W elements (batch, channel,
 *     row, column), dtype BSF_U8 (uint8) or BSF_F32 (float32).  f is zero
 *     outside the image (the paper leaves the boundary condition open).
 *   - Parameter fields are dense float32 planes, one set per image of the
 *     batch and shared by its C channels: B*K*H*W floats, plane k of image b
 *     at params + (b*K + k)*H*W.  K = N for BSF_PARAM_SCALES (a_1..a_N in px,
 *     the widths of Eq. const), K = 3 for BSF_PARAM_COV (C11, C12, C22 in
 *     px^2, descriptor D3 of Sec. 3.2.1) and for BSF_PARAM_SRT (sigma, rho,
 *     theta: sigma = sqrt(lambda_max) in px, rho = lambda_max/lambda_min,
 *     theta in radians, the major-axis orientation).
 *   - All data pointers are DEVICE pointers owned by the caller; the library
 *     never frees them.  Scratch memory (pre-integrated buffers, scan
 *     carries) is owned by the context and reused across calls.
 *   - Calls are asynchronous on the given CUDA stream (a cudaStream_t passed
 *     as void*; NULL = legacy default stream) unless stated otherwise.
 *   - Argument errors return synchronously.  Errors detected on the device
 *     (a tap outside the pre-integrated buffer, an invalid scale) are OR-ed
 *     into a device status word read by bsf_get_device_status; the affected
 *     output pixels are NaN.
 *   - N = 4 (theta_k = 0, 45, 90, 135 degrees) is implemented by every entry
 *     point.  N = 6 (theta_k = 0, 30, ..., 150 degrees) is implemented by
 *     bsf_filter, bsf_filter_host and bsf_scales_from_cov; the other entry
 *     points return BSF_EUNSUPPORTED for it, and any other N returns
 *     BSF_EUNSUPPORTED everywhere.
 *
 * N = 6.  Algorithm 1 needs every running-sum direction b_k u_k to be a
 * lattice vector, which on the pixel lattice holds for N = 2, 4 only; for
 * more directions the paper notes that the image has to be interpolated
 * (Sec. 3.3).  The reading implemented: the image f = sum_k f[k] delta(x - k)
 * is transferred once to the hexagonal lattice Lambda_h = { h (i + j/2,
 * j sqrt3/2) } (opts.hex_spacing = h), each pixel's mass shared among the
 * vertices of the lattice triangle that holds it in proportion to its
 * barycentric coordinates (mass and centre of mass of every pixel kept).  All
 * six directions are lattice vectors of Lambda_h, so Algorithm 1 is exact
 * there: the filter computed is (1) with the pixel comb replaced by that
 * measure, fbar[n] = sum_{m in Lambda_h} mu[m] beta^6_{a(n)}(n - m): masses in
 * fixed point (24 fractional bits), running sums and the stencil's coefficient
 * sums exact in integers, the stencil's remaining terms in double-float
 * (opts.precision is ignored).  Its difference from (1) itself -- the method
 * error of the transfer -- falls like h^2 (about 4e-4 relative for a 2 px
 * kernel at h = 0.5 on a smooth image).  The scale map for six directions is
 * the criterion of Sec. 3.2.2 with the kurtosis norm written for six
 * directions, sum_{k,m} p_k^2 p_m^2 cos^2(theta_k - theta_m), under the same
 * eps, eta and flags; elongations are clamped at the six-directional bound
 * (1 + r)/(1 - r), r = cos(pi/6)/cos(psi - pi/6), psi = 2 theta mod pi/3
 * (at least 13.93; unbounded along the six directions).
 */
#ifndef BSF_H
#define BSF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int bsf_status;
#define BSF_OK 0
#define BSF_EINVAL 1          /* bad argument (null pointer, size, kind, dtype) */
#define BSF_EUNSUPPORTED 2    /* N not implemented by this entry point (see above) */
#define BSF_ENOMEM 3          /* device allocation of scratch failed */
#define BSF_ECUDA 4           /* a CUDA runtime call failed */
#define BSF_EHALO 5           /* device: a tap fell outside the pre-integrated buffer */
#define BSF_EINFEASIBLE 6     /* strict mode: a covariance needed the elongation clamp */
#define BSF_EBADSCALE 7       /* device: a scale or covariance was not finite/positive */
#define BSF_ERANGE 8          /* device: a kernel (N=4) or image values (N=6) too large for the exact integer form */
#define BSF_ENOSCRATCH 9      /* bsf_filter_noalloc: the image needs more than its fixed scratch */
#define BSF_ETIMEOUT 10       /* device: a bounded wait between the pre-integration's row bands gave up */

/* image element types */
#define BSF_U8 0
#define BSF_F32 1

/* parameter kinds */
#define BSF_PARAM_SCALES 0
#define BSF_PARAM_COV 1
#define BSF_PARAM_SRT 2

/* boundary conditions (the paper asks only for "appropriate boundary conditions", Sec. 2.1) */
#define BSF_BOUNDARY_ZERO 0     /* f = 0 outside the image (default) */
#define BSF_BOUNDARY_REFLECT 1  /* f extended by half-sample symmetric reflection: f[-1-i] = f[i],
                                   f[n+i] = f[n-1-i], repeated with period 2n for footprints wider
                                   than the image */

/* arithmetic forms of the path */
#define BSF_PREC_EXACT 0  /* integer pre-integration (int64 for u8; 128-bit fixed point with 32
                             fractional bits for f32) and an exact integer finite difference at
                             scales rounded to a per-pixel dyadic grid; one final FP32 rounding */
#define BSF_PREC_FP64 1   /* all-FP64: Algorithm 1 computed literally in double precision */

#define BSF_STAGING_L1 0
#define BSF_STAGING_TMA 1

typedef struct bsf_ctx bsf_ctx;

typedef struct {
    int precision;    /* BSF_PREC_EXACT (default) or BSF_PREC_FP64 */
    float eps;        /* lower bound on a_k^2, px^2 (Sec. 3.2.2 constraint p >= eps); default 1e-3 */
    float eta;        /* covariances with rho > (1-eta) U(theta) (Prop. 3.1) are lowered to that
                         elongation, keeping size s and orientation theta; default 1e-3 */
    int strict;       /* 0 (default): clamp and continue; 1: bsf_filter returns BSF_EINFEASIBLE
                         (after a stream synchronisation) when any pixel needed the clamp */
    int halo;         /* padding P of the pre-integrated buffer in px; 0 = derive it:
                         from max_scale if > 0, else from a device reduction over the field
                         (one stream synchronisation) */
    float max_scale;  /* optional bound on the largest footprint: for SCALES the largest a_k,
                         for COV/SRT the largest sqrt(lambda_max) (px); 0 = unknown */
    int iterations;   /* m >= 1 (default 1): filter with the iterated box spline of Sec. 3.3,
                         i.e. run the path m times with the scale vector a/sqrt(m) (the
                         covariance of each pass is C/m, of the m passes together C).
                         Passes after the first take the float32 output of the previous one. */
    float hex_spacing;  /* N = 6 only: spacing h (px) of the hexagonal lattice the image is
                         transferred to: 1, 0.5 (default), 0.25 or 0.125.  The method error of
                         the transfer falls like h^2, the pre-integration work grows like 1/h^2. */
    float rel_bound;  /* N = 6 only: the map's lower bound on each p_k = a_k^2 relative to the
                         trace T = sum_k p_k: p_k >= max(eps, rel_bound * T), and elongations are
                         bounded by the hexagon of the six directions scaled by 1 - 6 rel_bound.
                         Default 1e-3 (no width below 0.077 times the typical one); must lie in
                         [0, 1/6).  The 1e-5 accuracy of the six-directional path is stated for
                         the default: 0 leaves only eps, whose tiny widths cost the stencil's
                         rounded part accuracy (BSF_EINVAL outside the range). */
    int boundary;     /* BSF_BOUNDARY_ZERO (default) or BSF_BOUNDARY_REFLECT: how the image is
                         continued beyond its edges.  Honoured by bsf_filter, bsf_filter_host and
                         bsf_filter_noalloc (N = 4 and 6); bsf_preintegrate / bsf_apply take no
                         options and use zero; bsf_filter_backward returns BSF_EUNSUPPORTED for
                         reflect. */
    int map_lut;      /* N = 6 only, kinds COV and SRT: 0 (default) solves the map of Sec. 3.2.2
                         for every pixel; 1 reads it from a table.  The map is homogeneous
                         (p(s C) = s p(C)) and invariant under rotations by pi/6 up to a shift of
                         the direction index, so the table holds p / T (T = sum p = 12 tr C) on a
                         513 x 513 grid over 2 theta in [0, pi/3] and e / e_c in [0, 1]
                         (e = (rho - 1) / (rho + 1), e_c the elongation clamp).  A lookup
                         interpolates bilinearly and projects the result onto the covariance
                         constraint, so each kernel keeps its target covariance; only the kurtosis
                         optimum is approximated (p moves by at most 1e-3 T, at the kinks where a
                         width leaves its bound).  Pixels where eps binds (eps above rel_bound
                         times T), rel_bound = 0 and invalid input take the solver.  The table
                         (8.4 MB of device memory, kept by the context) is built on the first call
                         for each (eta, rel_bound), which then waits on its stream once. */
    int staging;      /* N = 4, exact 64-bit form (u8 images): how the stencil reads the
                         pre-integrated buffer.  BSF_STAGING_L1 (default): nine loads per tap
                         through the L1 cache.  BSF_STAGING_TMA: per CTA of 32 x 8 pixels and per
                         tap, the box of cells the tile reads is copied to shared memory by the
                         tensor-copy engine first (taps whose box exceeds 40 x 16 elements read
                         through L1).  Both give the same bits; other forms ignore the field. */
} bsf_opts;

/* Fill *opts with the defaults listed above. */
void bsf_default_opts(bsf_opts* opts);

/* Create a context bound to CUDA device `device` (the device is made current
 * on the calling thread).  *ctx receives the handle.  A context owns one set
 * of scratch buffers that its calls share: calls are thread-safe, but work
 * that one context enqueues on different streams must not overlap on the
 * device (order it, or use one context per stream); bsf_filter_host keeps
 * its own work in order on the context's streams. */
bsf_status bsf_create(bsf_ctx** ctx, int device);

/* Release a context and all scratch memory it owns (synchronises the device). */
bsf_status bsf_destroy(bsf_ctx* ctx);

/* Whole path: fbar of (1) for every pixel of every channel of every image.
 * image: B*C*H*W elements of `dtype`; params: B*K*H*W floats of `kind`;
 * out: B*C*H*W floats.  Runs the scale map (Sec. 3.2.2, for COV/SRT), the
 * pre-integration (Algorithm 1 step 2) and the finite difference with ZP
 * interpolation (Algorithm 1 step 3).  opts may be NULL (defaults).
 * N = 6 (see the top of this file): each 64 x 64 tile of output pixels (16 x
 * 16 where the footprints are small, groups of up to 4 x 2 tiles where they
 * are large) gets its own window of the hexagonal lattice, sized from the
 * tile's largest footprint; the call synchronises the stream once (after the
 * scale map) to plan the windows.  The result is accurate to 1e-5 for kernels
 * whose widths are about half a pixel or more (the six-directional map keeps
 * every width at least 0.077 times the typical one); footprints wider than
 * about 1000 px along x (hex_spacing 0.5) return BSF_EINVAL.  Windows whose
 * running sums leave the exact range (|sum| < 2^95: u8 images, and f32 images
 * up to about 1e4 in magnitude, stay within it at every footprint the map
 * produces for sigma <= 48) or hold non-finite image values give NaN and the
 * device status BSF_ERANGE. */
bsf_status bsf_filter(bsf_ctx* ctx, const void* image, int dtype, int64_t B, int64_t C, int64_t H,
                      int64_t W, int N, const float* params, int kind, const bsf_opts* opts,
                      float* out, void* stream);

/* The whole path on HOST buffers, pipelined across calls (the paper has no
 * counterpart; this is the streaming form of bsf_filter).  Enqueues on the
 * context's own three CUDA streams: the copy of image_host and params_host to
 * the device, bsf_filter on them, and the copy of the result into out_host;
 * returns without waiting.  Two slots of device buffers alternate between
 * consecutive calls, so the input copy of one call, the kernels of the
 * previous one and the output copy of the one before can run at the same
 * time.  Arguments and layouts are those of bsf_filter with host pointers.
 * Host buffers should be page-locked (cudaHostAlloc / cudaHostRegister) for
 * the copies to overlap; they must stay valid and unchanged until
 * bsf_host_sync returns.  Argument errors return synchronously and enqueue
 * nothing; CUDA errors of the enqueued work are returned by bsf_host_sync.
 * Slot buffers grow on demand, after draining the pipeline. */
bsf_status bsf_filter_host(bsf_ctx* ctx, const void* image_host, int dtype, int64_t B, int64_t C,
                           int64_t H, int64_t W, int N, const float* params_host, int kind,
                           const bsf_opts* opts, float* out_host);

/* Waits until every call of bsf_filter_host on ctx has completed and its
 * output is in host memory. */
bsf_status bsf_host_sync(bsf_ctx* ctx);

/* Feature-preserving smoothing (Sec. 4.2): the adaptive covariance field of
 * a batch of images, to be passed to bsf_filter with kind BSF_PARAM_COV.
 * Per pixel, J = w * (g g^T) is the structure tensor (g: central differences
 * replicated at the border, summed over the C channels; w: the isotropic
 * box spline with the covariance of a Gaussian of std sigma_w px, applied by
 * this library's exact filter), and
 *     C = sigma0^2 adj(M) / sqrt(det M),   M = J + tau I,
 * i.e. a window of the area of an isotropic Gaussian of std sigma0 px,
 * stretched along the eigenvector of the smallest eigenvalue of J (the
 * orientation of minimal intensity variation) with elongation
 * (lambda_max + tau) / (lambda_min + tau).  tau > 0 (in squared intensity
 * units per px^2) is the gradient energy below which a region counts as
 * uniform.  image: B*C*H*W elements of dtype; cov: B*3*H*W floats
 * (C11, C12, C22 planes per batch entry).  Scratch: 10*B*H*W floats owned
 * by the context.  Errors: BSF_EINVAL for non-positive or non-finite
 * sigma_w, sigma0, tau and the argument errors of bsf_filter. */
bsf_status bsf_structure_cov(bsf_ctx* ctx, const void* image, int dtype, int64_t B, int64_t C, int64_t H,
                             int64_t W, float sigma_w, float sigma0, float tau, float* cov, void* stream);

/* Step (b), Sec. 3.2.2: covariance (COV) or (sigma, rho, theta) (SRT) planes
 * (3*npix floats) -> scale planes a_1..a_N (N*npix floats, Eq. const widths),
 * N = 4 or 6.  flags (nullable, npix bytes): bit0 elongation clamped (Prop.
 * 3.1; for N = 6 the six-directional bound), bit1 p >= eps infeasible (the
 * minimiser over p >= 0 raised to eps), bit2 invalid input (scales NaN). */
bsf_status bsf_scales_from_cov(bsf_ctx* ctx, const float* params, int kind, int64_t npix, int N,
                               const bsf_opts* opts, float* scales, uint8_t* flags, void* stream);

/* Bytes of the caller-owned pre-integrated buffer for one H x W image with
 * halo P in the given precision form (the buffer holds (H+2P)*(W+2P)
 * elements: int64 for u8/EXACT, 16-byte fixed point for f32/EXACT, double
 * for FP64). */
bsf_status bsf_buffer_bytes(int dtype, int64_t H, int64_t W, int N, int halo, int precision,
                            size_t* bytes);

/* Scratch the context needs for bsf_filter at this shape (the paper has no
 * counterpart: this sizes the device memory a caller must leave free, or
 * budget, before the first call).  Host-only: nothing is allocated or
 * launched, ctx may be NULL.  N = 4: exact, given opts->halo or
 * opts->max_scale (the pre-integrated buffers of one launch, the scan carries,
 * and for opts->iterations > 1 the intermediate image).  N = 6: an upper bound
 * from opts->max_scale (the windows depend on the per-pixel footprints; the
 * planner holds at most two chunks of 8 GiB of windows: one pre-integrated
 * while the stencil reads the other).  Host buffers of
 * bsf_filter_host are not included.  Errors: BSF_EINVAL (bad shape or kind,
 * neither halo nor max_scale), BSF_EUNSUPPORTED (N). */
bsf_status bsf_query_workspace(bsf_ctx* ctx, int dtype, int64_t B, int64_t C, int64_t H, int64_t W, int N,
                               int kind, const bsf_opts* opts, size_t* bytes);

/* Step (a), Algorithm 1 step 2 (RS1-RS4 of Sec. 3.1) for ONE H x W image:
 * writes the pre-integrated buffer (zero padding P on every side, every
 * running sum started from zero at the buffer edge; the two sqrt2 factors
 * are taken out, so g_b = 2 * buffer).  Integer forms wrap modulo 2^64
 * (u8) or 2^128 (f32 fixed point), which the exact finite difference
 * tolerates.  buffer: caller-owned device memory of bsf_buffer_bytes.  A
 * padded row wider than 4096 elements (u8, FP64 form) or 3072 (f32 exact
 * form) returns BSF_EINVAL: one buffer row must fit one band CTA
 * (bsf_filter cuts such images into vertical strips instead). */
bsf_status bsf_preintegrate(bsf_ctx* ctx, const void* image, int dtype, int64_t H, int64_t W, int N,
                            int halo, int precision, void* buffer, void* stream);

/* Step (c), Algorithm 1 step 3 for ONE image: reads a buffer written by
 * bsf_preintegrate with the same dtype/H/W/halo/precision, and the K*H*W
 * params of `kind` (COV/SRT are mapped per pixel on the fly); writes H*W
 * floats to out. */
bsf_status bsf_apply(bsf_ctx* ctx, const void* buffer, int dtype, int64_t H, int64_t W, int N,
                     int halo, const float* params, int kind, const bsf_opts* opts, float* out,
                     void* stream);

/* Backward pass (gradients; the paper has none, this is the adjoint of the
 * forward path).  For a scale-vector field (kind BSF_PARAM_SCALES, B*4*H*W
 * floats) and grad_out = dL/dfbar (B*C*H*W floats), writes
 *   grad_image  (nullable, B*C*H*W floats) = sum_n g[n] beta_{a(n)}(n - k),
 *   grad_scales (nullable, B*4*H*W floats) = sum_c g[n] dfbar[n]/da_k(n)
 * (channels sharing one field are summed).  The scale gradient is exact for
 * the per-pixel dyadic scales the forward pass uses (an exact integer
 * combination of the pre-integrated buffer); the image gradient scatters the
 * stencil's weights into an FP64 buffer and applies the transposes of RS4,
 * RS3, RS2, RS1 in that order.  Only the exact form (opts->precision ==
 * BSF_PREC_EXACT) is supported.  At least one output must be non-NULL.
 * The adjoint does not cut wide rows into strips: an image whose padded
 * width W + 2P exceeds 4096 (u8) or 3072 (f32) returns BSF_EINVAL before
 * anything runs.  opts->iterations = m > 1 differentiates the m-fold
 * iterated filter of bsf_filter (Sec. 3.3, widths a / sqrt(m) in every
 * pass): the m - 1 intermediate images are recomputed (scratch: (m + 1)
 * B*C*H*W floats owned by the context), the passes are differentiated in
 * reverse order, and every pass adds its scale gradient. */
bsf_status bsf_filter_backward(bsf_ctx* ctx, const void* image, int dtype, int64_t B, int64_t C, int64_t H,
                               int64_t W, int N, const float* scales, const float* grad_out,
                               float* grad_image, float* grad_scales, const bsf_opts* opts, void* stream);

/* Synchronise `stream`, then return (and clear) the device status word in
 * *status: 0 or the OR of (1 << BSF_EHALO), (1 << BSF_EBADSCALE),
 * (1 << BSF_ERANGE), (1 << BSF_EINFEASIBLE) raised since the last call. */
bsf_status bsf_get_device_status(bsf_ctx* ctx, void* stream, int* status);

/* Measurement hook.  Between bsf_profile_begin and bsf_profile_end every
 * bsf_filter call records CUDA events on its own stream before the
 * pre-integration, between it and the finite difference, and after the
 * finite difference.  bsf_profile_end synchronises on those events and
 * returns the summed milliseconds of the two steps and the number of
 * launches of each (any pointer may be NULL). */
bsf_status bsf_profile_begin(bsf_ctx* ctx);
bsf_status bsf_profile_end(bsf_ctx* ctx, double* ms_preintegrate, double* ms_stencil, int* nlaunch);

/* Allocation-free variant of bsf_filter for ONE H x W image (B = C = 1).
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory, such as plugins inside a host application
 * that owns the device memory budget, or latency-critical loops in which
 * cudaMalloc/cudaFree would synchronise the device.  It needs no context and
 * calls no allocating routine: its scratch (the pre-integrated buffer and the
 * scan carries) is a fixed device array of BSF_NOALLOC_SCRATCH_BYTES compiled
 * into the library and reserved on every GPU that loads it until the process
 * exits.  Images whose buffer of (H+2P)*(W+2P) elements (8 bytes for u8,
 * 16 for f32 in the exact form) plus the carries exceed it are rejected with
 * BSF_ENOSCRATCH before anything runs (u8 images of about 1000 x 1000 px
 * fit).  opts is required and must give opts->halo or opts->max_scale.
 * Runs on the current device, asynchronously on `stream`; the first call on a
 * device looks up the array's device address, so make it before any stream
 * capture.  opts->iterations must be 1.  All calls share the array and it keeps the last call's contents:
 * calls that overlap on the GPU race and must be serialised by the caller.
 * There is no device status word: pixels with invalid scales or with taps
 * outside the buffer are NaN. */
#define BSF_NOALLOC_SCRATCH_BYTES (32u << 20)
bsf_status bsf_filter_noalloc(const void* image, int dtype, int64_t H, int64_t W, int N, const float* params,
                              int kind, const bsf_opts* opts, float* out, void* stream);

/* Bound, in polls, of the device-side waits between the pre-integration's row
 * bands (the four-directional carries run as one kernel whose blocks wait for
 * each other at grid barriers; every block is resident, so the waits end).
 * Process-wide; 0 restores the default of 2^22 polls (about a quarter of a
 * second).  A wait that runs out raises BSF_ETIMEOUT in the device status word
 * and its kernel leaves early: the output is then wrong, but nothing hangs.
 * The paper has no counterpart; the call exists to exercise that path. */
void bsf_set_wait_limit(unsigned polls);

/* Static description of a status code. */
const char* bsf_status_string(bsf_status s);

#ifdef __cplusplus
}
#endif

#endif /* BSF_H */
