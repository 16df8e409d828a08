// Batched form: many images of uneven size and Gaussian count fitted together.
//
// The images' Gaussians are concatenated (in image order) and binned in one
// pass over a concatenated tile space: image b owns global tiles
// [tile_off[b], tile_off[b+1]), and the per-tile counters, their scan and the
// atomic slots of the binning give every image its own S_j. One persistent
// launch of the fused
// forward + L1 + adjoint kernel then pulls tiles of all images from a device
// counter, which balances small and large images on the 148 SMs; Adam runs
// once over all parameters. The per-image tables live in the workspace after
// the single-image sections and are written once by igs_batch_setup.
//
// With the SSIM term (Sec. 4.1: L1 + 0.1 L_SSIM) a step renders every image
// (one launch over all tiles), evaluates each image's loss and its image-space
// gradient, and runs the persistent adjoint on that gradient. The batched
// forward and the adjoint of an external upstream gradient are also entry
// points of their own.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "imgs.h"
#include "internal.h"

namespace igs {

namespace {

constexpr int BATCH_TILE = 16;
constexpr int BATCH_MIN_STAGE = 64;  // smallest one-stage list of the batched adjoint

struct BatchGeom {
  WsLayout L;
  size_t dims, tile_off, pix_off, gauss_off, img_of, loss, work, total;
  // SSIM fits only (0 otherwise): renderings, their loss gradients, and the
  // image loss's 32 x 32 tile tables (per image (H, W, tiles across, 0) and
  // first tile)
  size_t img, gimg, ssim_dims, ssim_toff;
  int64_t Ntot, T, pixels, ssim_tiles;
  int B, n, Hmax, Wmax;
};

int bfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

int batch_geom(const igs_batch_shape* sh, const igs_config* cfg, int64_t m_cap, BatchGeom* G) {
  if (!sh || !cfg) return bfail(IGS_ERR_INVALID_ARG, "batch: NULL shape or config");
  if (!(cfg->ssim_weight >= 0.0f && cfg->ssim_weight <= 1e6f))
    return bfail(IGS_ERR_INVALID_ARG, "batch: ssim_weight must be finite and >= 0");
  if (sh->B < 1 || !sh->H || !sh->W || !sh->N)
    return bfail(IGS_ERR_INVALID_ARG, "batch: B < 1 or a NULL size array");
  if (sh->n < 1 || sh->n > 32) return bfail(IGS_ERR_INVALID_ARG, "batch: n = %d", sh->n);
  if (cfg->tile != BATCH_TILE)
    return bfail(IGS_ERR_INVALID_ARG, "batch: the batched form uses 16x16 tiles");
  if (!render_supported(cfg->tile, cfg->K, sh->n))
    return bfail(IGS_ERR_INVALID_ARG, "batch: unsupported K=%d", cfg->K);
  if (m_cap < 1 || m_cap > (int64_t)INT32_MAX)
    return bfail(IGS_ERR_INVALID_ARG, "batch: m_capacity out of range");
  int64_t N = 0, T = 0, pixels = 0;
  int Hmax = 0, Wmax = 0;
  for (int b = 0; b < sh->B; ++b) {
    const int H = sh->H[b], W = sh->W[b];
    if (H <= 0 || W <= 0 || H > (1 << 20) || W > (1 << 20) || sh->N[b] < 0)
      return bfail(IGS_ERR_INVALID_ARG, "batch: image %d has size %d x %d, N = %lld", b, H, W,
                   (long long)sh->N[b]);
    N += sh->N[b];
    T += (int64_t)((W + BATCH_TILE - 1) / BATCH_TILE) * ((H + BATCH_TILE - 1) / BATCH_TILE);
    pixels += (int64_t)H * W;
    Hmax = std::max(Hmax, H);
    Wmax = std::max(Wmax, W);
  }
  if (N > (int64_t)INT32_MAX || T > (int64_t)INT32_MAX)
    return bfail(IGS_ERR_INVALID_ARG, "batch: too many Gaussians or tiles");
  G->L = ws_layout_tiles(N, sh->n, T, m_cap);
  size_t o = G->L.total;
  const int B = sh->B;
  G->dims = o;      o = up256(o + sizeof(int4) * B);
  G->tile_off = o;  o = up256(o + sizeof(int) * (B + 1));
  G->pix_off = o;   o = up256(o + sizeof(long long) * (B + 1));
  G->gauss_off = o; o = up256(o + sizeof(long long) * (B + 1));
  G->img_of = o;    o = up256(o + sizeof(int) * (size_t)N);
  G->loss = o;      o = up256(o + sizeof(double) * B);
  G->work = o;      o = up256(o + sizeof(unsigned int));
  G->img = G->gimg = G->ssim_dims = G->ssim_toff = 0;
  G->ssim_tiles = 0;
  if (cfg->ssim_weight > 0.0f) {
    const size_t img_bytes = sizeof(float) * (size_t)sh->n * (size_t)pixels;
    G->img = o;       o = up256(o + img_bytes);
    G->gimg = o;      o = up256(o + img_bytes);
    G->ssim_dims = o; o = up256(o + sizeof(int4) * B);
    G->ssim_toff = o; o = up256(o + sizeof(int) * (B + 1));
    for (int b = 0; b < B; ++b) G->ssim_tiles += ssim_tiles_of(sh->H[b], sh->W[b]);
  }
  G->total = o;
  G->Ntot = N;
  G->T = T;
  G->pixels = pixels;
  G->B = B;
  G->n = sh->n;
  G->Hmax = Hmax;
  G->Wmax = Wmax;
  return IGS_OK;
}

#define BCUDA(call, where)                                                            \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return bfail(IGS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e_));            \
  } while (0)

int check_ws(const BatchGeom& G, void* ws, size_t ws_bytes) {
  if (!ws) return bfail(IGS_ERR_INVALID_ARG, "batch: workspace is NULL");
  if ((uintptr_t)ws % 256) return bfail(IGS_ERR_ALIGN, "batch: workspace must be 256-aligned");
  if (ws_bytes < G.total)
    return bfail(IGS_ERR_INVALID_ARG, "batch: workspace too small: %zu < %zu", ws_bytes, G.total);
  return IGS_OK;
}

BatchTables tables(const BatchGeom& G, char* base, int order) {
  BatchTables bt;
  bt.B = G.B;
  bt.dims = reinterpret_cast<const int4*>(base + G.dims);
  bt.tile_off = reinterpret_cast<const int*>(base + G.tile_off);
  bt.pix_off = reinterpret_cast<const long long*>(base + G.pix_off);
  bt.loss = reinterpret_cast<double*>(base + G.loss);
  bt.work = reinterpret_cast<unsigned int*>(base + G.work);
  bt.T = (int)G.T;
  bt.order = order;
  return bt;
}

// Bins the concatenated Gaussians of the fit state; returns render params.
// Lists longer than sort_min (the smallest stage the adjoint will run with)
// are sorted by Gaussian index; shorter ones are ranked by the renderer.
int batch_bin(const float* params, const BatchGeom& G, const igs_config* cfg, char* base,
              int64_t m_cap, int sort_min, RenderParams* rp, cudaStream_t s) {
  const WsLayout& L = G.L;
  DevStatus* status = reinterpret_cast<DevStatus*>(base + L.status);
  BCUDA(cudaMemsetAsync(status, 0, sizeof(DevStatus), s), "batch: reset status");
  const int np = 5 + G.n;
  PrepParams p;
  memset(&p, 0, sizeof(p));
  p.xy = params;
  p.theta = params + 2;
  p.inv_scale = params + 3;
  p.color = params + 5;
  p.xy_stride = p.theta_stride = p.inv_scale_stride = p.color_stride = np;
  p.N = G.Ntot;
  p.n = G.n;
  p.tile = BATCH_TILE;
  p.rec = reinterpret_cast<GRec*>(base + L.rec);
  p.trig = reinterpret_cast<float2*>(base + L.trig);
  p.color_out = reinterpret_cast<float*>(base + L.color);
  p.tcnt = reinterpret_cast<unsigned int*>(base + L.tcnt);
  p.toff = reinterpret_cast<unsigned long long*>(base + L.toff);
  p.vals = reinterpret_cast<unsigned int*>(base + L.vals);
  p.tmp = reinterpret_cast<unsigned int*>(base + L.tmp);
  p.wide = reinterpret_cast<int*>(base + L.wide);
  p.wide_geo = reinterpret_cast<float4*>(base + L.wide_geo);
  p.m_cap = m_cap;
  p.status = status;
  p.img_of = reinterpret_cast<const int*>(base + G.img_of);
  p.img_dims = reinterpret_cast<const int4*>(base + G.dims);
  p.tile_off = reinterpret_cast<const int*>(base + G.tile_off);
  unsigned long long* part = reinterpret_cast<unsigned long long*>(base + L.part);
  int2* range = reinterpret_cast<int2*>(base + L.range);
  BCUDA(run_binning(p, IGS_F32, (int)G.T, part, range, sort_min, s), "batch: binning");
  BCUDA(launch_tile_evals_batch(range, (int)G.T, p.img_dims, p.tile_off, G.B, BATCH_TILE,
                                status, s),
        "batch: evals");
  const unsigned int* vals = p.vals;
  memset(rp, 0, sizeof(*rp));
  rp->range = range;
  rp->list = reinterpret_cast<const int*>(vals);
  rp->rec = p.rec;
  rp->trig = p.trig;
  rp->color = p.color_out;
  rp->n = G.n;
  rp->N = (int)G.Ntot;
  rp->tile = BATCH_TILE;
  rp->status = status;
  return IGS_OK;
}

int sm_count() {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 148;
}

int check_tuning(const igs_batch_tuning& t) {
  if (t.ctas_per_sm < 1 || t.ctas_per_sm > 8 || (t.stage != 64 && t.stage != 128 && t.stage != 256) ||
      (t.order != 0 && t.order != 1))
    return bfail(IGS_ERR_INVALID_ARG, "batch: tuning (%d CTAs/SM, stage %d, order %d) invalid",
                 t.ctas_per_sm, t.stage, t.order);
  return IGS_OK;
}

// Adjoint of every image: zero grad and per-image sums, one persistent launch.
// With d_targets the upstream gradient is the fused L1 one; otherwise
// d_grad_imgs (concatenated planar images) is the upstream gradient.
int batch_adjoint(float* grad, const float* d_targets, const float* d_grad_imgs,
                  const BatchGeom& G, const igs_config* cfg, const igs_batch_tuning& tn,
                  char* base, RenderParams rp, cudaStream_t s) {
  BCUDA(cudaMemsetAsync(grad, 0, sizeof(float) * (size_t)G.Ntot * (5 + G.n), s),
        "batch: zero grad");
  if (d_targets)
    BCUDA(cudaMemsetAsync(base + G.loss, 0, sizeof(double) * G.B, s), "batch: zero losses");
  BCUDA(cudaMemsetAsync(base + G.work, 0, sizeof(unsigned int), s), "batch: zero counter");
  rp.target = d_targets;
  rp.grad_img = d_grad_imgs;
  rp.grad = grad;
  rp.normalize = cfg->normalize;
  const BatchTables bt = tables(G, base, tn.order);
  BCUDA(launch_render_bwd_batch(rp, bt, cfg->K, tn.stage, tn.ctas_per_sm * sm_count(), s),
        "batch: adjoint");
  return IGS_OK;
}

int check_state(const igs_fit_state* st, const BatchGeom& G, const float* d_targets) {
  if (!st || !st->params || !st->grad || !st->adam_m || !st->adam_v || !st->step)
    return bfail(IGS_ERR_INVALID_ARG, "batch: fit state has a NULL pointer");
  if (st->N != G.Ntot || st->n != G.n)
    return bfail(IGS_ERR_INVALID_ARG, "batch: fit state (N=%lld, n=%d) differs from the shape "
                 "(sum N=%lld, n=%d)", (long long)st->N, st->n, (long long)G.Ntot, G.n);
  if (!d_targets) return bfail(IGS_ERR_INVALID_ARG, "batch: targets are NULL");
  if ((uintptr_t)st->params % 16 || (uintptr_t)st->grad % 16 || (uintptr_t)d_targets % 4)
    return bfail(IGS_ERR_ALIGN, "batch: parameter arrays must be 16-byte aligned");
  return IGS_OK;
}

// Forward render of every image into the concatenated planar images d_imgs.
int batch_forward(const BatchGeom& G, const igs_config* cfg, char* base, RenderParams rp,
                  float* d_imgs, cudaStream_t s) {
  rp.img = d_imgs;
  rp.normalize = cfg->normalize;
  const BatchTables bt = tables(G, base, 0);
  BCUDA(launch_render_fwd_batch(rp, bt, cfg->K, s), "batch: forward");
  return IGS_OK;
}

// L1 + w (1 - SSIM) of every rendering against its target, one launch over
// the 32 x 32 loss tiles of all images: the image-space gradients into gimg,
// the per-image loss sums into the batch's loss table.
int batch_image_loss(const BatchGeom& G, const igs_config* cfg, const float* d_targets,
                     char* base, cudaStream_t s) {
  BCUDA(launch_image_loss_batch(reinterpret_cast<const float*>(base + G.img), d_targets, G.B,
                                reinterpret_cast<const int4*>(base + G.ssim_dims),
                                reinterpret_cast<const int*>(base + G.ssim_toff),
                                reinterpret_cast<const long long*>(base + G.pix_off),
                                (int)G.ssim_tiles, G.n, cfg->ssim_weight,
                                reinterpret_cast<float*>(base + G.gimg),
                                reinterpret_cast<double*>(base + G.loss), s),
        "batch: image loss");
  return IGS_OK;
}

// The packed parameters [N][5+n] (and the gradient, if given) must match the
// shape's Gaussian count and be 16-byte aligned.
int check_params(const float* params, const float* grad, const BatchGeom& G, int64_t N) {
  if (N != G.Ntot)
    return bfail(IGS_ERR_INVALID_ARG, "batch: N = %lld differs from the shape's sum %lld",
                 (long long)N, (long long)G.Ntot);
  if ((uintptr_t)params % 16 || (uintptr_t)grad % 16)
    return bfail(IGS_ERR_ALIGN, "batch: parameter arrays must be 16-byte aligned");
  return IGS_OK;
}

}  // namespace

}  // namespace igs

using namespace igs;

extern "C" int igs_render_forward_batch(const float* d_params, int64_t N,
                                        const igs_batch_shape* shape, const igs_config* cfg,
                                        void* ws, size_t ws_bytes, int64_t m_capacity,
                                        float* d_imgs, igs_stream stream) {
  BatchGeom G;
  if (int r = batch_geom(shape, cfg, m_capacity, &G)) return r;
  if (int r = check_ws(G, ws, ws_bytes)) return r;
  if (!d_params || !d_imgs) return bfail(IGS_ERR_INVALID_ARG, "batch forward: NULL pointer");
  if (int r = check_params(d_params, nullptr, G, N)) return r;
  if ((uintptr_t)d_imgs % 4) return bfail(IGS_ERR_ALIGN, "batch forward: images misaligned");
  char* base = static_cast<char*>(ws);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RenderParams rp;
  // lists longer than one forward stage (256) are sorted by index
  if (int r = batch_bin(d_params, G, cfg, base, m_capacity, BATCH_TILE * BATCH_TILE, &rp, s))
    return r;
  return batch_forward(G, cfg, base, rp, d_imgs, s);
}

extern "C" int igs_render_backward_batch(const float* d_params, int64_t N,
                                         const float* d_grad_imgs, const igs_batch_shape* shape,
                                         const igs_config* cfg, const igs_batch_tuning* tuning,
                                         void* ws, size_t ws_bytes, int64_t m_capacity,
                                         float* d_grad, igs_stream stream) {
  BatchGeom G;
  if (int r = batch_geom(shape, cfg, m_capacity, &G)) return r;
  if (int r = check_ws(G, ws, ws_bytes)) return r;
  if (!d_params || !d_grad_imgs || !d_grad)
    return bfail(IGS_ERR_INVALID_ARG, "batch backward: NULL pointer");
  if (int r = check_params(d_params, d_grad, G, N)) return r;
  if ((uintptr_t)d_grad_imgs % 4) return bfail(IGS_ERR_ALIGN, "batch backward: gradient misaligned");
  igs_batch_tuning tn = tuning ? *tuning : igs_batch_tuning{4, 256, 0};
  if (int r = check_tuning(tn)) return r;
  char* base = static_cast<char*>(ws);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RenderParams rp;
  if (int r = batch_bin(d_params, G, cfg, base, m_capacity, tn.stage, &rp, s)) return r;
  return batch_adjoint(d_grad, nullptr, d_grad_imgs, G, cfg, tn, base, rp, s);
}

extern "C" int igs_batch_workspace_size(const igs_batch_shape* shape, const igs_config* cfg,
                                        int64_t m_capacity, size_t* bytes) {
  if (!bytes) return bfail(IGS_ERR_INVALID_ARG, "batch: bytes is NULL");
  BatchGeom G;
  if (int r = batch_geom(shape, cfg, m_capacity, &G)) return r;
  *bytes = G.total;
  return IGS_OK;
}

extern "C" int igs_batch_setup(const igs_batch_shape* shape, const igs_config* cfg, void* ws,
                               size_t ws_bytes, int64_t m_capacity, igs_stream stream) {
  BatchGeom G;
  if (int r = batch_geom(shape, cfg, m_capacity, &G)) return r;
  if (int r = check_ws(G, ws, ws_bytes)) return r;
  const int B = G.B, n = G.n;
  std::vector<int4> dims(B);
  std::vector<int> tile_off(B + 1);
  std::vector<long long> pix_off(B + 1), gauss_off(B + 1);
  tile_off[0] = 0;
  pix_off[0] = gauss_off[0] = 0;
  for (int b = 0; b < B; ++b) {
    const int H = shape->H[b], W = shape->W[b];
    const int tx = (W + BATCH_TILE - 1) / BATCH_TILE, ty = (H + BATCH_TILE - 1) / BATCH_TILE;
    dims[b] = make_int4(H, W, tx, ty);
    tile_off[b + 1] = tile_off[b] + tx * ty;
    pix_off[b + 1] = pix_off[b] + (long long)n * H * W;
    gauss_off[b + 1] = gauss_off[b] + shape->N[b];
  }
  char* base = static_cast<char*>(ws);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  BCUDA(cudaMemcpyAsync(base + G.dims, dims.data(), sizeof(int4) * B, cudaMemcpyHostToDevice, s),
        "batch setup: dims");
  BCUDA(cudaMemcpyAsync(base + G.tile_off, tile_off.data(), sizeof(int) * (B + 1),
                        cudaMemcpyHostToDevice, s),
        "batch setup: tile offsets");
  BCUDA(cudaMemcpyAsync(base + G.pix_off, pix_off.data(), sizeof(long long) * (B + 1),
                        cudaMemcpyHostToDevice, s),
        "batch setup: pixel offsets");
  BCUDA(cudaMemcpyAsync(base + G.gauss_off, gauss_off.data(), sizeof(long long) * (B + 1),
                        cudaMemcpyHostToDevice, s),
        "batch setup: Gaussian offsets");
  if (G.ssim_dims) {
    std::vector<int4> sdims(B);
    std::vector<int> stoff(B + 1);
    stoff[0] = 0;
    for (int b = 0; b < B; ++b) {
      const int H = shape->H[b], W = shape->W[b];
      sdims[b] = make_int4(H, W, 0, 0);
      stoff[b + 1] = stoff[b] + ssim_tiles_of(H, W);
    }
    BCUDA(cudaMemcpyAsync(base + G.ssim_dims, sdims.data(), sizeof(int4) * B,
                          cudaMemcpyHostToDevice, s),
          "batch setup: loss tile sizes");
    BCUDA(cudaMemcpyAsync(base + G.ssim_toff, stoff.data(), sizeof(int) * (B + 1),
                          cudaMemcpyHostToDevice, s),
          "batch setup: loss tile offsets");
  }
  BCUDA(launch_fill_image_of(reinterpret_cast<int*>(base + G.img_of),
                             reinterpret_cast<const long long*>(base + G.gauss_off), B, G.Ntot, s),
        "batch setup: image of each Gaussian");
  BCUDA(cudaStreamSynchronize(s), "batch setup: sync");
  return IGS_OK;
}

extern "C" int igs_fit_batch_step(const igs_fit_state* st, const float* d_targets,
                                  const igs_batch_shape* shape, const igs_config* cfg,
                                  const igs_batch_tuning* tuning, void* ws, size_t ws_bytes,
                                  int64_t m_capacity, float* d_loss_out, igs_stream stream) {
  BatchGeom G;
  if (int r = batch_geom(shape, cfg, m_capacity, &G)) return r;
  if (int r = check_ws(G, ws, ws_bytes)) return r;
  if (int r = check_state(st, G, d_targets)) return r;
  igs_batch_tuning tn = tuning ? *tuning : igs_batch_tuning{4, 256, 0};
  if (int r = check_tuning(tn)) return r;
  char* base = static_cast<char*>(ws);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RenderParams rp;
  if (int r = batch_bin(st->params, G, cfg, base, m_capacity, tn.stage, &rp, s)) return r;
  if (cfg->ssim_weight > 0.0f) {
    if (int r = batch_forward(G, cfg, base, rp, reinterpret_cast<float*>(base + G.img), s))
      return r;
    if (int r = batch_image_loss(G, cfg, d_targets, base, s)) return r;
    if (int r = batch_adjoint(st->grad, nullptr, reinterpret_cast<const float*>(base + G.gimg),
                              G, cfg, tn, base, rp, s))
      return r;
  } else {
    if (int r = batch_adjoint(st->grad, d_targets, nullptr, G, cfg, tn, base, rp, s)) return r;
  }
  if (int r = igs_adam_update(st, cfg, stream)) return r;
  BCUDA(launch_finalize_batch(st->step, reinterpret_cast<const double*>(base + G.loss),
                              reinterpret_cast<const int4*>(base + G.dims), G.B, G.n, d_loss_out,
                              s),
        "batch: finalize");
  return IGS_OK;
}

extern "C" int igs_autotune_batch(const igs_fit_state* st, const float* d_targets,
                                  const igs_batch_shape* shape, const igs_config* cfg, void* ws,
                                  size_t ws_bytes, int64_t m_capacity, int32_t reps,
                                  igs_batch_tuning* best, float* best_ms, igs_stream stream) {
  BatchGeom G;
  if (int r = batch_geom(shape, cfg, m_capacity, &G)) return r;
  if (int r = check_ws(G, ws, ws_bytes)) return r;
  if (int r = check_state(st, G, d_targets)) return r;
  if (!best) return bfail(IGS_ERR_INVALID_ARG, "autotune: best is NULL");
  if (reps < 1) reps = 1;
  char* base = static_cast<char*>(ws);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RenderParams rp;
  // one binning serves every stage tried below
  if (int r = batch_bin(st->params, G, cfg, base, m_capacity, BATCH_MIN_STAGE, &rp, s)) return r;
  cudaEvent_t e0, e1;
  BCUDA(cudaEventCreate(&e0), "autotune: event");
  BCUDA(cudaEventCreate(&e1), "autotune: event");
  const int ctas[] = {2, 3, 4, 6, 8};
  const int stages[] = {64, 128, 256};
  float best_t = 1e30f;
  igs_batch_tuning win{4, 256, 0};
  int rc = IGS_OK;
  for (int order = 0; order < 2 && rc == IGS_OK; ++order)
    for (int c : ctas)
      for (int stg : stages) {
        if (rc != IGS_OK) break;
        const igs_batch_tuning tn{c, stg, order};
        rc = batch_adjoint(st->grad, d_targets, nullptr, G, cfg, tn, base, rp, s);  // warm-up
        if (rc) break;
        cudaEventRecord(e0, s);
        for (int i = 0; i < reps && rc == IGS_OK; ++i)
          rc = batch_adjoint(st->grad, d_targets, nullptr, G, cfg, tn, base, rp, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          rc = bfail(IGS_ERR_CUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
          break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (ms < best_t) {
          best_t = ms;
          win = tn;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != IGS_OK) return rc;
  *best = win;
  if (best_ms) *best_ms = best_t;
  return IGS_OK;
}
