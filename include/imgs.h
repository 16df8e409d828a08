/*
 * imgs.h -- C ABI of the B300-native Image-GS rasteriser (libimgs.so).
 *
 * Tile-binned differentiable rasterisation of colored, anisotropic 2D
 * Gaussians (Image-GS, arXiv 2407.01866): per-Gaussian preprocessing and
 * tile binning, the top-K normalised forward render, its adjoint, the fused
 * L1 + Adam fit step, random-access decode and the batched fit form.
 *
 * Conventions shared by every call
 * --------------------------------
 * - All pointers named d_* or documented as "device" are CUDA device
 *   pointers owned by the caller and only borrowed for the duration of the
 *   stream-ordered call. The library allocates nothing in these calls, so a
 *   sequence of them can be captured into a CUDA graph.
 * - Every call is asynchronous on `stream` unless it says otherwise, and
 *   returns an igs_status. On failure, igs_last_error() gives a message for
 *   the calling thread.
 * - Images are planar float32 [n][H][W], contiguous. Pixel (h, w) is
 *   evaluated at its centre (w + 1/2, h + 1/2) in pixels; x runs along the
 *   width, y down the rows.
 * - A Gaussian is p = (mu, theta, t, c) (Eq. 3 with the inverse scale
 *   t = 1/s of Sec. 3.3 / Sec. 4.1): mu in [0,1]^2 (Sec. 4.1 maps the image
 *   to the unit square), theta the rotation angle, t = (t1, t2) inverse
 *   standard deviations in 1/px along R's columns, c in R^n.
 *   Covariance Sigma = R S S^T R^T (Eq. 2), S = diag(1/t1, 1/t2).
 * - A packed parameter / gradient row is (mu_x, mu_y, theta, t1, t2, c0..c_{n-1}).
 *
 * Binary32 decisions (fixed here so that any implementation, and the
 * oracle, selects identical sets). Every operation is rounded once to
 * nearest-even; fma is a single-rounding fused multiply-add:
 *   mx = mu_x * W, my = mu_y * H
 *   c  = round32(cos(theta) in float64), s = round32(sin(theta) in float64)
 *   T1 = t1*t1, T2 = t2*t2
 *   A00 = T1*(c*c) + T2*(s*s);  A11 = T1*(s*s) + T2*(c*c)
 *   A01 = (T1 - T2)*(c*s);      B = A01 + A01
 *   r = 3 / min(t1, t2)         (3-sigma enclosing circle, Sec. 3.2)
 *   Tile j = closed rect [X0,X1]x[Y0,Y1], X0 = tile*tx, X1 = min(X0+tile, W):
 *     ex = max(max(X0 - mx, mx - X1), 0), ey likewise;
 *     j in S(i)  <=>  ex*ex + ey*ey <= r*r
 *   Ranking key at (px, py):
 *     dx = px - mx, dy = py - my, h = fma(B, dy, A00*dx),
 *     q = fma(h, dx, (A11*dy)*dy)
 *   The K smallest (q, gaussian index) pairs of S_j are kept (Sec. 3.2,
 *   Sec. 4.1: K = 10); ties go to the smaller index.
 * Values (weights, colours, gradients) are float32; the blend is Eq. 5
 * evaluated as w_k = exp(-(q_k - q_min)/2), c = sum w_k c_k / sum w_k,
 * which equals Eq. 5 in exact arithmetic. An empty S_j renders 0.
 */
#ifndef IMGS_H
#define IMGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* igs_stream;

typedef enum {
  IGS_OK = 0,
  IGS_ERR_INVALID_ARG = 1, /* null pointer, bad size, unsupported K/tile/n */
  IGS_ERR_ALIGN = 2,       /* a pointer misses its documented alignment */
  IGS_ERR_CAPACITY = 3,    /* intersections M exceed the workspace capacity */
  IGS_ERR_CUDA = 4,        /* a CUDA runtime call failed (message has it) */
  IGS_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
  IGS_ERR_NONFINITE = 6    /* a parameter is NaN/Inf or an inverse scale <= 0 */
} igs_status;

typedef enum { IGS_F32 = 0, IGS_F16 = 1, IGS_BF16 = 2 } igs_dtype;

/* Device status flags written by kernels into igs_stats.flags. */
enum { IGS_FLAG_CAPACITY = 1u, IGS_FLAG_NONFINITE = 2u, IGS_FLAG_TIMEOUT = 4u,
       IGS_FLAG_INTERNAL = 8u /* a list entry out of range (library fault) */ };

/* A borrowed view of N Gaussians (Eq. 3). Each array holds one row per
 * Gaussian; *_stride is the distance in ELEMENTS between consecutive rows
 * (xy: >= 2, theta: >= 1, inv_scale: >= 2, color: >= n). All four arrays
 * have element type `dtype`; alignment: the element size. Device memory. */
typedef struct {
  const void* xy;
  const void* theta;
  const void* inv_scale;
  const void* color;
  int64_t xy_stride, theta_stride, inv_scale_stride, color_stride;
  int64_t N;
  int32_t n;      /* channels, 1..32 */
  int32_t dtype;  /* igs_dtype; F16/BF16 only for preprocess/forward/decode */
} igs_gaussians;

typedef struct {
  int32_t K;          /* top-K, one of 1,2,3,4,8,10,16 (Sec. 4.1: 10); 0 keeps
                         all of S_j (the "no top-K" ablation of Table 1) */
  int32_t tile;       /* logical tile edge in px, 8 or 16 (Sec. 4.1: 16);
                         it changes S_j and therefore the image */
  int32_t normalize;  /* 1: Eq. 5 (default). 0: the unnormalised sum
                         c = sum G_i c_i over the kept Gaussians (Eq. 4
                         restricted to S_j; Table 1 ablation) */
  /* fit step (Sec. 4.1): Adam learning rates per group */
  float lr_mu, lr_theta, lr_inv_scale, lr_color;
  double beta1, beta2;  /* double: 0.999 in float32 would move 1-beta2 by 1.3e-5 */
  float eps;
  /* clamps after each update (Sec. 3.1): theta, inverse scale, mean */
  float theta_min, theta_max, t_min, t_max, mu_min, mu_max;
  /* weight w of the SSIM term of the fit loss L1 + w L_SSIM (Sec. 4.1:
   * 0.1). 0 (default) fits against L1 alone with the fused adjoint; w > 0
   * runs forward render, igs_image_loss and the adjoint with that upstream
   * gradient (single image and batched form), and needs the larger
   * workspace igs_workspace_size / igs_batch_workspace_size report */
  float ssim_weight;
} igs_config;

/* Host-readable copy of the device status block of one workspace. */
typedef struct {
  uint32_t flags;        /* IGS_FLAG_* raised since the last preprocess */
  uint32_t reserved;
  int64_t m_needed;      /* intersections M of the last preprocess */
  int64_t evals;         /* Gaussian-pixel evaluations of one forward:
                            sum over tiles of |S_j| * pixels(j) */
  double loss_sum;       /* sum |c_r - c_t| of the last fused backward */
} igs_stats;

/* Binning result: device pointers into the caller's workspace. Filled by
 * igs_preprocess_bin; valid until the workspace is reused. */
typedef struct {
  int32_t H, W, tile, tiles_x, tiles_y, n;
  int64_t N, m_capacity;
  const int32_t* tile_range;  /* [T][2] = [start, end) into list */
  const int32_t* list;        /* [m_capacity] Gaussian indices grouped by
                                 tile; ascending within a tile of more than
                                 tile*tile entries, in no set order within
                                 a shorter one (the renderer ranks those) */
  const float* rec;           /* [N][8] preprocessed geometry (internal) */
  const float* trig;          /* [N][2] (cos, sin) (internal) */
  const float* color;         /* [N][n] float32 colours (internal) */
  void* status;               /* device status block (internal) */
  int32_t dtype;              /* storage of the binned parameters (IGS_F32...) */
  const void* rec16;          /* F16/BF16 storage: [N] 16-byte records of the
                                 stored mu bits and the binary32 conic, read
                                 by the render and decode loops (internal) */
  const void* color16;        /* F16/BF16 storage: [N][n] stored colour bits
                                 (internal); both NULL for F32 */
} igs_bins;

/* Library version: major*10000 + minor*100 + patch. */
int igs_version(void);

/* Copies the calling thread's last error message (NUL-terminated,
 * truncated to n bytes). Returns the message length. */
int igs_last_error(char* buf, size_t n);

/* Defaults of Sec. 4.1: K = 10, 16x16 tiles, learning rates
 * (mu, colour, inverse scale, theta) = (5e-4, 5e-3, 2e-3, 2e-3), Adam
 * betas (0.9, 0.999), eps 1e-8; clamps theta in [0, pi], t in [1e-3, 10],
 * mu in [0, 1]. */
void igs_default_config(igs_config* cfg);

/* Bytes of device workspace that igs_preprocess_bin needs for N Gaussians
 * with n channels on an H x W image and room for m_capacity tile-Gaussian
 * intersections. Host only; no CUDA call. H and W are 1..2^20, with at most
 * 65535 rows of tiles (the render grid's y extent); IGS_ERR_INVALID_ARG
 * otherwise, here and in igs_preprocess_bin. */
int igs_workspace_size(int64_t N, int32_t n, int32_t H, int32_t W,
                       const igs_config* cfg, int64_t m_capacity, size_t* bytes);

/* "Project/bin Gaussians to tiles" (Sec. 3.2): per-Gaussian preprocessing
 * (Eq. 2 inverse covariance, 3-sigma circle), exact tile-circle tests,
 * per-tile lists by prefix sums and slot cursors, lists longer than one
 * tile's pixel count sorted by index. `ws` is a device buffer
 * of at least igs_workspace_size() bytes, 256-byte aligned. Resets the status
 * block. If M > m_capacity the lists are truncated and IGS_FLAG_CAPACITY is
 * raised on the device (no host sync here: read it with igs_read_stats;
 * m_needed tells the capacity to use). Invalid parameters raise
 * IGS_FLAG_NONFINITE and that Gaussian is binned nowhere. */
int igs_preprocess_bin(const igs_gaussians* g, int32_t H, int32_t W,
                       const igs_config* cfg, void* ws, size_t ws_bytes,
                       int64_t m_capacity, igs_bins* out, igs_stream stream);

/* Forward render (Eq. 5 with top-K, Sec. 3.2) into d_img [n][H][W] float32
 * (16-byte aligned). Uses the bins of the same Gaussians. */
int igs_render_forward(const igs_bins* bins, const igs_config* cfg,
                       float* d_img, igs_stream stream);

/* Adjoint (Sec. 3.3: gradients through the K retained Gaussians, selection
 * held fixed). Overwrites d_grad [N][5+n] float32 (packed row order) with
 * dL/dp. The upstream gradient is d_grad_img [n][H][W] if non-NULL;
 * otherwise L = mean |c_r - c_t| over H*W*n against d_target [n][H][W]
 * (d|z|/dz = sign(z), sign(0) = 0) and sum |c_r - c_t| is added to the
 * status block's loss_sum. The gradient is with respect to the stored
 * parameter values (float16/bfloat16 storage: the values upcast exactly).
 * Tiles add their contributions with float atomics (16-byte vector atomics
 * where d_grad is 16-byte aligned and a row is a multiple of 4 floats), so
 * the rounding order of d_grad varies between calls; the loss is summed in
 * float32 per tile and in float64 across tiles. */
int igs_render_backward(const igs_gaussians* g, const igs_bins* bins,
                        const igs_config* cfg, const float* d_grad_img,
                        const float* d_target, float* d_grad, igs_stream stream);

/* Fit state for igs_fit_step: packed float32 parameters and Adam moments,
 * all [N][5+n] row-major, 16-byte aligned; d_step is a device int32 step
 * counter (0 before the first step), incremented by each step. */
typedef struct {
  float* params;
  float* grad;
  float* adam_m;
  float* adam_v;
  int32_t* step;
  int64_t N;
  int32_t n;
} igs_fit_state;

/* Adam update of a fit state from its current gradient (Sec. 4.1: Adam
 * with per-group learning rates; Sec. 3.1: clip theta, scales and means to
 * their ranges afterwards). Reads st->grad, updates params and moments in
 * place; uses step = *st->step + 1 for the bias correction and leaves
 * *st->step unchanged (igs_fit_step advances it). */
int igs_adam_update(const igs_fit_state* st, const igs_config* cfg, igs_stream stream);

/* One optimisation step (Sec. 3.3, Sec. 4.1): preprocess/bin, fused
 * forward + L1 + adjoint, Adam with per-group learning rates, clamps. No
 * host synchronisation; the sequence can be captured in a CUDA graph.
 * d_loss_out (nullable, device float) receives the step's mean L1 loss. */
int igs_fit_step(const igs_fit_state* st, const float* d_target, int32_t H,
                 int32_t W, const igs_config* cfg, void* ws, size_t ws_bytes,
                 int64_t m_capacity, float* d_loss_out, igs_stream stream);

/* One optimisation step with half-precision parameter storage (Sec. 4.1:
 * the Gaussians are kept in half precision, 16 bits per value): st->params
 * is the float32 master copy; d_params_half [N][5+n] (IGS_F16 or IGS_BF16,
 * 16-byte aligned) is the stored representation. The step rounds the master
 * to half (nearest even), bins, renders and differentiates the half values,
 * applies Adam to the master with that gradient, and leaves the half copy
 * as the rounding of the updated master. Otherwise as igs_fit_step. The
 * representation costs N (5+n) 16 / (H W) bits per pixel. This library
 * addition has no separate counterpart in the paper beyond Sec. 4.1's
 * storage format. */
int igs_fit_step_half(const igs_fit_state* st, void* d_params_half, int32_t half_dtype,
                      const float* d_target, int32_t H, int32_t W, const igs_config* cfg,
                      void* ws, size_t ws_bytes, int64_t m_capacity, float* d_loss_out,
                      igs_stream stream);

/* Random-access decode (Sec. 2.2 / abstract: per-pixel decode): colour at
 * Q arbitrary points d_xy [Q][2] = (x, y) in pixels, written to d_out
 * [Q][n]. A point belongs to tile (floor(x/tile), floor(y/tile)) clamped to
 * the grid and is evaluated at (x, y) itself; the rule is the same as the
 * forward render's. */
int igs_decode_points(const igs_bins* bins, const igs_config* cfg,
                      const float* d_xy, int64_t Q, float* d_out, igs_stream stream);

/* ---- Batched form: many images of uneven size fitted in one launch ----
 * B images with their own H_b x W_b and N_b Gaussians share one fit state:
 * parameters (and gradients, Adam moments) are the images' packed rows
 * concatenated in image order, [sum N_b][5+n]; targets are the images'
 * planar [n][H_b][W_b] float32 arrays concatenated in image order. Tiles
 * are 16x16 and every image keeps its own tile grid (S_j per image). */
typedef struct {
  int32_t B;          /* number of images, >= 1 */
  int32_t n;          /* channels, shared by all images */
  const int32_t* H;   /* [B] host array: image heights */
  const int32_t* W;   /* [B] host array: image widths */
  const int64_t* N;   /* [B] host array: Gaussians per image */
} igs_batch_shape;

/* Physical mapping of the persistent adjoint (chosen by igs_autotune_batch). */
typedef struct {
  int32_t ctas_per_sm;  /* persistent CTAs per SM, 1..8 (default 4) */
  int32_t stage;        /* Gaussians staged per round: 64, 128 or 256 (default 256) */
  int32_t order;        /* 0: tiles pulled from a device counter, 1: static round-robin */
} igs_batch_tuning;

/* Workspace bytes for a batch (host only). m_capacity bounds the total
 * tile-Gaussian intersections of all images. */
int igs_batch_workspace_size(const igs_batch_shape* shape, const igs_config* cfg,
                             int64_t m_capacity, size_t* bytes);

/* Writes the batch's per-image tables (sizes, tile and pixel offsets, the
 * image of every Gaussian) into the workspace. Call once per workspace and
 * shape, before capturing igs_fit_batch_step: it copies from host memory. */
int igs_batch_setup(const igs_batch_shape* shape, const igs_config* cfg, void* ws,
                    size_t ws_bytes, int64_t m_capacity, igs_stream stream);

/* One optimisation step of every image of the batch (Sec. 3.3, Sec. 4.1,
 * as igs_fit_step): batched preprocess/bin over the concatenated tile
 * space, one persistent fused forward + L1 + adjoint launch over all tiles,
 * Adam, clamps. With cfg->ssim_weight > 0 (Sec. 4.1: L1 + 0.1 L_SSIM) the
 * step renders every image (igs_render_forward_batch), evaluates each
 * image's loss and image-space gradient (as igs_image_loss) and runs the
 * persistent adjoint on that gradient; the workspace is larger (see
 * igs_batch_workspace_size). Stream-ordered, no host synchronisation,
 * graph-capturable after igs_batch_setup. tuning may be NULL (defaults).
 * d_loss_out (nullable, device float [B]) receives each image's mean loss
 * (L1, plus w (1 - SSIM) with the SSIM term). */
int igs_fit_batch_step(const igs_fit_state* st, const float* d_targets,
                       const igs_batch_shape* shape, const igs_config* cfg,
                       const igs_batch_tuning* tuning, void* ws, size_t ws_bytes,
                       int64_t m_capacity, float* d_loss_out, igs_stream stream);

/* Forward render (Eq. 5, Sec. 3.2) of every image of the batch into
 * d_imgs, the images' planar [n][H_b][W_b] float32 arrays concatenated in
 * image order. d_params [N][5+n] (N = sum N_b, 16-byte aligned) are the
 * concatenated packed rows. Bins the batch into the workspace (after
 * igs_batch_setup), then renders every tile of every image in one launch.
 * Stream-ordered, no host synchronisation. */
int igs_render_forward_batch(const float* d_params, int64_t N, const igs_batch_shape* shape,
                             const igs_config* cfg, void* ws, size_t ws_bytes,
                             int64_t m_capacity, float* d_imgs, igs_stream stream);

/* Adjoint (Sec. 3.3: gradients through the K retained Gaussians) of every
 * image of the batch for an external upstream gradient d_grad_imgs (the
 * images' dL/dc_r, laid out like d_imgs of igs_render_forward_batch), with
 * the persistent mapping `tuning` (NULL: defaults). d_grad [N][5+n]
 * (16-byte aligned) is overwritten with dL/dp in the packed order. Bins the
 * batch into the workspace first. Stream-ordered, no host synchronisation. */
int igs_render_backward_batch(const float* d_params, int64_t N, const float* d_grad_imgs,
                              const igs_batch_shape* shape, const igs_config* cfg,
                              const igs_batch_tuning* tuning, void* ws, size_t ws_bytes,
                              int64_t m_capacity, float* d_grad, igs_stream stream);

/* Chooses the persistent adjoint's mapping for this batch by timing every
 * candidate (CTAs per SM x stage x order) on the current parameters: bins
 * once, runs each candidate `reps` times, keeps the fastest. Parameters and
 * Adam state are not modified (st->grad is used as scratch). Synchronises
 * `stream`. best_ms (nullable, host) receives the winner's mean time. */
int igs_autotune_batch(const igs_fit_state* st, const float* d_targets,
                       const igs_batch_shape* shape, const igs_config* cfg, void* ws,
                       size_t ws_bytes, int64_t m_capacity, int32_t reps,
                       igs_batch_tuning* best, float* best_ms, igs_stream stream);

/* Forward render that allocates nothing and takes no workspace. The paper
 * has no counterpart: this is a convenience for callers that cannot call
 * cudaMalloc or hand the library a device buffer -- a plug-in inside a host
 * application that owns every allocation, a real-time thread where an
 * allocation may block or fail, or code held to a fixed device-memory
 * budget. It runs igs_preprocess_bin and igs_render_forward with their
 * scratch in one static device array of IGS_STATIC_SCRATCH_BYTES (32 MiB)
 * that every GPU which loads the library keeps until the process exits.
 * - Inputs g (device parameters) and output d_img [n][H][W] are the
 *   caller's, as for igs_render_forward.
 * - Sizes whose workspace cannot fit (large N, image or tile count) are
 *   rejected with IGS_ERR_CAPACITY before any GPU work; if the
 *   intersections found on the GPU do not fit, the call returns
 *   IGS_ERR_CAPACITY after rendering and the image is incomplete.
 * - The scratch is sized for binning only (igs_preprocess_bin's sections);
 *   an SSIM weight in cfg costs it nothing.
 * - The call synchronises `stream` at its end to read the status block.
 * - Every call looks up the array's device address on the current device
 *   (cudaGetSymbolAddress), so the address stays right after a device
 *   reset; the first call on a device also loads the library's module
 *   there, so make that first call before any stream capture.
 * - All calls share the one array, which keeps the last call's contents;
 *   every word a call reads is cleared or written by that call first.
 *   Calls that overlap on the GPU (other streams, other host threads) race
 *   on it: serialise them. */
#define IGS_STATIC_SCRATCH_BYTES (32u << 20)
int igs_render_forward_static(const igs_gaussians* g, int32_t H, int32_t W,
                              const igs_config* cfg, float* d_img, igs_stream stream);

/* Size in bytes of the static scratch used by igs_render_forward_static. */
int igs_static_scratch_bytes(size_t* bytes);

/* Image-space fitting loss (Sec. 3.3, Sec. 4.1: L1 + 0.1 L_SSIM) of a
 * rendering d_render against d_target ([n][H][W] float32 each):
 * L = mean |x - y| + w (1 - mean SSIM), means over channels and pixels,
 * d|z|/dz = sign(z) with sign(0) = 0. SSIM per channel with an 11 x 11
 * Gaussian window (sigma 1.5, normalised, zero-padded "same" correlation),
 * C1 = 0.01^2, C2 = 0.03^2 (data range 1). d_grad_img [n][H][W] receives
 * dL/dx; d_loss_out (nullable, device float) the loss. float32 arithmetic.
 * Scratch: igs_image_loss_workspace_size() bytes, 256-byte aligned. */
int igs_image_loss_workspace_size(int32_t n, int32_t H, int32_t W, size_t* bytes);
int igs_image_loss(const float* d_render, const float* d_target, int32_t n, int32_t H,
                   int32_t W, float ssim_weight, float* d_grad_img, float* d_loss_out,
                   void* ws, size_t ws_bytes, igs_stream stream);

/* Content-adaptive placement (Sec. 3.3). Both draws are independent and
 * decided exactly, so that they can be reproduced bit for bit:
 *   weights   binary32: Eq. 6 uses |grad I|_2 with, per channel, central
 *             differences (I[k+1] - I[k-1]) * 0.5 inside and one-sided
 *             differences at the borders (0 along an axis of length 1),
 *             accumulated s += gx*gx, s += gy*gy over channels, then sqrt;
 *             Eq. 7 uses the sum over channels of |c_r - c_t|
 *   integers  floor(min(w, 4096) * 2^24), non-finite -> 0; exclusive prefix
 *             sums give a 64-bit cumulative weight
 *   draw      from 53-bit integers r1, r2 (u = r / 2^53; the top 11 bits of the
 *             inputs are ignored): if r1 < floor(lambda * 2^53) or every weight
 *             is 0, pixel floor(r2 * H * W / 2^53); otherwise the last pixel
 *             whose exclusive prefix is <= floor(r2 * total / 2^53)
 *   Gaussian  mu = ((x + 0.5) / W, (y + 0.5) / H) in binary32, theta = 0,
 *             t = (0.2, 0.2) (5 px, Sec. 4.1), colour = the target at the pixel
 * Scratch: a device workspace of igs_placement_workspace_size() bytes,
 * 256-byte aligned. */
int igs_placement_workspace_size(int32_t H, int32_t W, size_t* bytes);

/* Eq. 6: N initial Gaussians drawn from the target d_target [n][H][W] with
 * uniform share lambda in [0, 1] (Sec. 4.1: 0.3). d_rand [N][2] holds (r1,
 * r2) per Gaussian; d_params [N][5+n] receives the packed rows. */
int igs_init_gaussians(const float* d_target, int32_t H, int32_t W, int32_t n, int64_t N,
                       double lambda, const uint64_t* d_rand, float* d_params, void* ws,
                       size_t ws_bytes, igs_stream stream);

/* Eq. 7: `count` Gaussians added where the rendering d_render [n][H][W]
 * (igs_render_forward of the current parameters) differs from d_target.
 * d_rand [count][2] (r1 is ignored). Writes rows [st->N, st->N + count) of
 * st->params and zeroes those rows of st->grad, st->adam_m and st->adam_v; the
 * arrays must have room for them, and the caller then raises N by count
 * (Sec. 4.1 starts from N/2 and adds N/8 every 500 steps). */
int igs_add_gaussians(const float* d_target, const float* d_render, int32_t H, int32_t W,
                      const uint64_t* d_rand, int64_t count, const igs_fit_state* st,
                      void* ws, size_t ws_bytes, igs_stream stream);

/* Synchronously copies the workspace's status block to *out (this call
 * synchronises `stream`). */
int igs_read_stats(const igs_bins* bins, igs_stats* out, igs_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* IMGS_H */
