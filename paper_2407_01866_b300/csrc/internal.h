// Host-side launchers shared between the C-ABI layer (api.cu) and the kernel
// translation units. Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"

namespace igs {

// Scan geometry: one block scans SCAN_THREADS * SCAN_PER_THREAD entries.
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_PER_THREAD = 2;
constexpr int SCAN_ITEMS = SCAN_THREADS * SCAN_PER_THREAD;

// Byte offsets of the workspace sections (all 256-byte aligned).
struct WsLayout {
  size_t status, rec, trig, color, rec16, col16, tcnt, toff, part, vals, tmp, wide, wide_geo, range;
  size_t total;
  int64_t part_len;     // scan partials entries
  int tiles_x, tiles_y;
};
WsLayout ws_layout(int64_t N, int n, int H, int W, int tile, int64_t m_cap);
// Same layout for T tiles in total (batched form: tiles of all images).
WsLayout ws_layout_tiles(int64_t N, int n, int64_t T, int64_t m_cap);
// Sets the calling thread's message returned by igs_last_error.
void set_last_error(const char* msg);

struct PrepParams {
  const void* xy;
  const void* theta;
  const void* inv_scale;
  const void* color;
  int64_t xy_stride, theta_stride, inv_scale_stride, color_stride;
  int64_t N;
  int n, H, W, tile, tiles_x, tiles_y;
  GRec* rec;
  float2* trig;
  float* color_out;
  // half-precision storage only: the hot record of the render and decode
  // loops (stored mu bits, binary32 conic) and the stored colour bits
  HRec* rec16;
  unsigned short* col16;
  unsigned int* tcnt;           // [T] hits per tile (zeroed before preprocess)
  unsigned long long* toff;     // [T] start of each tile's segment
  unsigned int* vals;           // [m_cap] Gaussian index per intersection
  unsigned int* tmp;            // [m_cap] merge buffer of long segments
  int* wide;                    // [N] Gaussians whose tile box is binned by a CTA
  float4* wide_geo;             // [N] their (mx, my, r, index bits), same order
  int64_t m_cap;
  DevStatus* status;
  // batched form: image of each Gaussian, per-image (H, W, tiles_x, tiles_y)
  // and first global tile; all null for a single image
  const int* img_of;
  const int4* img_dims;
  const int* tile_off;
};

struct RenderParams {
  const int2* range;   // [T] = [start, end)
  const int* list;     // gaussian index per intersection
  const GRec* rec;
  const float2* trig;
  const float* color;  // [N][n]
  // half-precision storage (hdt = 1: float16, 2: bfloat16; 0: none): the
  // render and decode loops read these 16-byte records and 2-byte colours
  // instead of rec / color (same binary32 values)
  const HRec* rec16;
  const unsigned short* col16;
  int hdt;
  int H, W, tiles_x, tiles_y, n;
  int N;                   // number of Gaussians (bounds guard on list entries)
  int normalize;           // 1: Eq. 5; 0: unnormalised sum over the kept Gaussians
  float* img;              // forward output [n][H][W]
  const float* grad_img;   // backward upstream gradient or null
  const float* target;     // L1 target when grad_img is null
  float* grad;             // [N][5+n]
  float inv_count;         // 1 / (H W n)
  DevStatus* status;
  // decode
  const float* qxy;
  float* qout;
  int64_t Q;
  int tile;
};

// Per-image tables of the batched form (device, inside the workspace).
struct BatchTables {
  int B;
  const int4* dims;            // (H, W, tiles_x, tiles_y) per image
  const int* tile_off;         // [B+1] first global tile of each image
  const long long* pix_off;    // [B+1] offset (floats) of each image's planes
  double* loss;                // [B] sum |c_r - c_t| per image
  unsigned int* work;          // next work item (tile) counter, zeroed per launch
  int T;                       // total tiles
  int order;                   // 0: dynamic counter, 1: static round-robin
};

cudaError_t launch_preprocess(const PrepParams& p, int dtype, cudaStream_t s);
cudaError_t launch_emit(const PrepParams& p, cudaStream_t s);
// Batched form: image index of every Gaussian from the per-image offsets.
cudaError_t launch_fill_image_of(int* img_of, const long long* gauss_off, int B, int64_t N,
                                 cudaStream_t s);
cudaError_t launch_tile_evals_batch(const int2* range, int T, const int4* dims,
                                    const int* tile_off, int B, int tile, DevStatus* status,
                                    cudaStream_t s);
// Exclusive scan of n u32 counts into u64 offsets; total goes to *total.
cudaError_t launch_scan_u32_to_u64(const unsigned int* in, unsigned long long* out, int64_t n,
                                   unsigned long long* part, unsigned long long* total,
                                   cudaStream_t s);
// Sorts every tile segment longer than sort_min by Gaussian index.
cudaError_t launch_segsort(unsigned int* vals, unsigned int* tmp,
                           const unsigned long long* toff, int T, DevStatus* status,
                           int64_t m_cap, int sort_min, cudaStream_t s);
cudaError_t launch_ranges(const unsigned long long* toff, int2* range, int T, int64_t m_cap,
                          int H, int W, int tile, int tiles_x, DevStatus* status,
                          cudaStream_t s);
// Whole binning sequence after the status reset: per-tile counts, scan,
// emit, segment sort, ranges (and, for one image, the evaluation count).
// Segments of at most sort_min entries (the renderer's one-stage capacity)
// are left in emission order; longer ones are sorted by Gaussian index.
cudaError_t run_binning(const PrepParams& p, int dtype, int T, unsigned long long* part,
                        int2* range, int sort_min, cudaStream_t s);

// Render family: return cudaErrorInvalidValue for an unsupported (tile, K, n).
cudaError_t launch_render_fwd(const RenderParams& p, int tile, int K, cudaStream_t s);
cudaError_t launch_render_bwd(const RenderParams& p, int tile, int K, cudaStream_t s);
// Persistent adjoint over a batch of images (16x16 tiles); stage in {64,128,256}.
cudaError_t launch_render_bwd_batch(const RenderParams& p, const BatchTables& bt, int K,
                                    int stage, int grid, cudaStream_t s);
// Forward render of every tile of a batch of images (16x16 tiles).
cudaError_t launch_render_fwd_batch(const RenderParams& p, const BatchTables& bt, int K,
                                    cudaStream_t s);
cudaError_t launch_decode(const RenderParams& p, int K, cudaStream_t s);
bool render_supported(int tile, int K, int n);

struct AdamParams {
  float* P;
  const float* G;
  float* m;
  float* v;
  int32_t* step;
  int64_t N;
  int n;
  float lr_mu, lr_theta, lr_t, lr_c, b1, b2, omb1, omb2, eps;
  float theta_min, theta_max, t_min, t_max, mu_min, mu_max;
  // a fit step's finalisation, done by the launch's last CTA (fin == nullptr:
  // none): *step += 1 and *fin_loss = fin->loss_sum * fin_inv_count
  DevStatus* fin;
  float fin_inv_count;
  float* fin_loss;
};
cudaError_t launch_adam(const AdamParams& a, cudaStream_t s);

// Content-adaptive placement (Sec. 3.3, Eq. 6 / Eq. 7): workspace sections
// (bytes, 256-aligned) for an image of HW pixels.
struct PlaceLayout {
  size_t weights, excl, part, total, bytes;
};
PlaceLayout place_layout(int64_t HW);
// Draws `count` pixels (render == nullptr: Eq. 6 from the target's gradient
// magnitudes with uniform share lambda; otherwise Eq. 7 from |render - target|)
// and writes new Gaussians to rows [row0, row0 + count) of params; zeroes those
// rows of grad, m, v when grad is non-null. rnd holds 2 * count 53-bit integers.
cudaError_t launch_place(const float* target, const float* render, int H, int W, int n,
                         const unsigned long long* rnd, int64_t count, double lambda,
                         float* params, int64_t row0, float* grad, float* m, float* v,
                         char* ws, cudaStream_t s);
// Image-space loss L1 + w (1 - SSIM) (Sec. 4.1) of rendering x against
// target y ([n][H][W] each): d_grad receives dL/dx, *acc (zeroed here) the
// sum over channels and pixels of |x - y| + w (1 - S), loss_out (nullable)
// the mean. scratch: image_loss_scratch_bytes(n, H, W) bytes, 256-aligned.
size_t image_loss_scratch_bytes(int n, int H, int W);
// Number of 32 x 32 loss tiles of an H x W image.
int ssim_tiles_of(int H, int W);
// L1 + w (1 - SSIM) of every image of a batch in one launch (w > 0): dims
// [B] = (H, W, 32-tiles across, 0), tile_off [B+1] the first 32-tile of each
// image, pix_off [B+1] the images' plane offsets (floats) in x, y and grad;
// acc [B] (zeroed here) receives each image's loss sum.
cudaError_t launch_image_loss_batch(const float* x, const float* y, int B, const int4* dims,
                                    const int* tile_off, const long long* pix_off, int tiles,
                                    int n, float w_ssim, float* grad, double* acc,
                                    cudaStream_t s);
cudaError_t launch_image_loss(const float* x, const float* y, int n, int H, int W,
                              float w_ssim, float* grad, double* acc, float* loss_out,
                              char* scratch, cudaStream_t s);
// Exclusive prefix sum of 64-bit integers; *total receives the sum.
cudaError_t launch_scan_u64(const unsigned long long* in, unsigned long long* out, int64_t n,
                            unsigned long long* part, unsigned long long* total,
                            cudaStream_t s);
// dst[i] = float16 (or bfloat16 if bf16) rounding of src[i], nearest even.
cudaError_t launch_round_params(const float* src, void* dst, bool bf16, int64_t count,
                                cudaStream_t s);
// Batched form: step counter and per-image mean L1 loss.
cudaError_t launch_finalize_batch(int32_t* step, const double* loss, const int4* dims, int B,
                                  int n, float* loss_out, cudaStream_t s);

}  // namespace igs
