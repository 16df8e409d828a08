// C ABI of libimgs.so: argument validation, workspace layout and the
// stream-ordered sequences behind each entry point. See include/imgs.h.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "imgs.h"
#include "internal.h"

namespace igs {

static thread_local std::string g_last_error;

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

static int cuda_fail(cudaError_t e, const char* where) {
  return fail(IGS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define IGS_CUDA(call, where)                         \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

WsLayout ws_layout(int64_t N, int n, int H, int W, int tile, int64_t m_cap) {
  WsLayout L = ws_layout_tiles(N, n, (int64_t)((W + tile - 1) / tile) * ((H + tile - 1) / tile),
                               m_cap);
  L.tiles_x = (W + tile - 1) / tile;
  L.tiles_y = (H + tile - 1) / tile;
  return L;
}

WsLayout ws_layout_tiles(int64_t N, int n, int64_t T, int64_t m_cap) {
  WsLayout L;
  L.tiles_x = L.tiles_y = 0;
  L.part_len = std::max<int64_t>(1, (T + SCAN_ITEMS - 1) / SCAN_ITEMS);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  L.status = take(sizeof(DevStatus));
  L.rec = take(sizeof(GRec) * (size_t)N);
  L.trig = take(sizeof(float2) * (size_t)N);
  L.color = take(sizeof(float) * (size_t)N * n);
  L.rec16 = take(sizeof(HRec) * (size_t)N);
  L.col16 = take(sizeof(unsigned short) * (size_t)N * n);
  L.tcnt = take(sizeof(unsigned int) * (size_t)T);
  L.toff = take(sizeof(unsigned long long) * (size_t)T);
  L.part = take(sizeof(unsigned long long) * (size_t)L.part_len);
  L.vals = take(sizeof(unsigned int) * (size_t)m_cap);
  L.tmp = take(sizeof(unsigned int) * (size_t)m_cap);
  L.wide = take(sizeof(int) * (size_t)N);
  L.wide_geo = take(sizeof(float4) * (size_t)N);
  L.range = take(sizeof(int2) * (size_t)T);
  L.total = o;
  return L;
}

static int check_config(const igs_config* cfg, int n) {
  if (!cfg) return fail(IGS_ERR_INVALID_ARG, "config is NULL");
  if (!(cfg->ssim_weight >= 0.0f && cfg->ssim_weight <= 1e6f))
    return fail(IGS_ERR_INVALID_ARG, "ssim_weight must be finite and >= 0");
  if (cfg->normalize != 0 && cfg->normalize != 1)
    return fail(IGS_ERR_INVALID_ARG, "normalize must be 0 or 1");
  if (!render_supported(cfg->tile, cfg->K, n))
    return fail(IGS_ERR_INVALID_ARG,
                "unsupported (tile=%d, K=%d, n=%d): tile 8 or 16, K in {0,1,2,3,4,8,10,16}, "
                "n in 1..32",
                cfg->tile, cfg->K, n);
  return IGS_OK;
}

static int check_image(int H, int W, int tile) {
  if (H <= 0 || W <= 0 || H > (1 << 20) || W > (1 << 20))
    return fail(IGS_ERR_INVALID_ARG, "bad image size %d x %d", H, W);
  // the render grid has one CTA per tile, (tiles_x, tiles_y), and a grid's
  // y extent is at most 65535
  if ((H + tile - 1) / tile > 65535)
    return fail(IGS_ERR_INVALID_ARG, "image height %d needs more than 65535 rows of %d-px tiles",
                H, tile);
  return IGS_OK;
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

static int check_gaussians(const igs_gaussians* g) {
  if (!g) return fail(IGS_ERR_INVALID_ARG, "gaussians is NULL");
  if (g->N < 0 || g->N > (int64_t)INT32_MAX)
    return fail(IGS_ERR_INVALID_ARG, "N = %lld out of range", (long long)g->N);
  if (g->n < 1 || g->n > 32) return fail(IGS_ERR_INVALID_ARG, "n = %d not in 1..32", g->n);
  if (g->dtype != IGS_F32 && g->dtype != IGS_F16 && g->dtype != IGS_BF16)
    return fail(IGS_ERR_INVALID_ARG, "dtype %d unknown", g->dtype);
  if (g->N > 0 && (!g->xy || !g->theta || !g->inv_scale || !g->color))
    return fail(IGS_ERR_INVALID_ARG, "a parameter array is NULL");
  if (g->N > 0 && (g->xy_stride < 2 || g->theta_stride < 1 || g->inv_scale_stride < 2 ||
                   g->color_stride < g->n))
    return fail(IGS_ERR_INVALID_ARG, "parameter row strides too small");
  const size_t es = g->dtype == IGS_F32 ? 4 : 2;
  if (!aligned(g->xy, es) || !aligned(g->theta, es) || !aligned(g->inv_scale, es) ||
      !aligned(g->color, es))
    return fail(IGS_ERR_ALIGN, "parameter arrays must be aligned to their element size");
  return IGS_OK;
}

static RenderParams render_params(const igs_bins* b) {
  RenderParams p;
  memset(&p, 0, sizeof(p));
  p.range = reinterpret_cast<const int2*>(b->tile_range);
  p.list = b->list;
  p.rec = reinterpret_cast<const GRec*>(b->rec);
  p.trig = reinterpret_cast<const float2*>(b->trig);
  p.color = b->color;
  p.H = b->H;
  p.W = b->W;
  p.tiles_x = b->tiles_x;
  p.tiles_y = b->tiles_y;
  p.n = b->n;
  p.N = (int)b->N;
  p.tile = b->tile;
  p.status = static_cast<DevStatus*>(b->status);
  p.inv_count = (float)(1.0 / ((double)b->H * b->W * b->n));
  if ((b->dtype == IGS_F16 || b->dtype == IGS_BF16) && b->rec16 && b->color16) {
    p.rec16 = static_cast<const HRec*>(b->rec16);
    p.col16 = static_cast<const unsigned short*>(b->color16);
    p.hdt = b->dtype == IGS_F16 ? 1 : 2;
  }
  return p;
}

static int check_bins(const igs_bins* b, const igs_config* cfg) {
  if (!b || !b->tile_range || !b->list || !b->rec || !b->status)
    return fail(IGS_ERR_INVALID_ARG, "bins not filled by igs_preprocess_bin");
  if (cfg && cfg->tile != b->tile)
    return fail(IGS_ERR_INVALID_ARG, "config tile %d differs from the binning tile %d",
                cfg->tile, b->tile);
  return IGS_OK;
}

}  // namespace igs

using namespace igs;

extern "C" {

int igs_version(void) { return 1 * 10000 + 0 * 100 + 0; }

int igs_last_error(char* buf, size_t n) {
  const std::string& s = g_last_error;
  if (buf && n) {
    const size_t k = std::min(n - 1, s.size());
    memcpy(buf, s.data(), k);
    buf[k] = 0;
  }
  return (int)s.size();
}

// Extra workspace of a fit step with the SSIM term, after the binning
// sections: the rendering, its image-space gradient and the loss scratch.
static size_t fit_extra_bytes(const igs_config* cfg, int n, int H, int W) {
  if (!(cfg->ssim_weight > 0.0f)) return 0;
  const size_t img = align_up(sizeof(float) * (size_t)n * H * W, 256);
  return 2 * img + image_loss_scratch_bytes(n, H, W);
}

// The fit step's loss and adjoint: the fused L1 adjoint, or (SSIM term) forward
// render, image loss and the adjoint of its image-space gradient.
static int fit_loss_adjoint(const igs_gaussians* g, const igs_bins* bins, const igs_config* cfg,
                            const float* d_target, float* d_grad, char* base, size_t binning_bytes,
                            igs_stream stream) {
  if (!(cfg->ssim_weight > 0.0f))
    return igs_render_backward(g, bins, cfg, nullptr, d_target, d_grad, stream);
  const int n = bins->n, H = bins->H, W = bins->W;
  const size_t img_bytes = align_up(sizeof(float) * (size_t)n * H * W, 256);
  float* img = reinterpret_cast<float*>(base + binning_bytes);
  float* gimg = reinterpret_cast<float*>(base + binning_bytes + img_bytes);
  char* scratch = base + binning_bytes + 2 * img_bytes;
  if (int r = igs_render_forward(bins, cfg, img, stream)) return r;
  IGS_CUDA(launch_image_loss(img, d_target, n, H, W, cfg->ssim_weight, gimg,
                             &static_cast<DevStatus*>(bins->status)->loss_sum, nullptr, scratch,
                             reinterpret_cast<cudaStream_t>(stream)),
           "image loss");
  return igs_render_backward(g, bins, cfg, gimg, nullptr, d_grad, stream);
}

void igs_default_config(igs_config* c) {
  if (!c) return;
  c->K = 10;
  c->tile = 16;
  c->normalize = 1;
  c->lr_mu = 5e-4f;
  c->lr_color = 5e-3f;
  c->lr_inv_scale = 2e-3f;
  c->lr_theta = 2e-3f;
  c->beta1 = 0.9;
  c->beta2 = 0.999;
  c->eps = 1e-8f;
  c->theta_min = 0.0f;
  c->theta_max = 3.14159265358979323846f;
  c->t_min = 1e-3f;
  c->t_max = 10.0f;
  c->mu_min = 0.0f;
  c->mu_max = 1.0f;
  c->ssim_weight = 0.0f;
}

int igs_workspace_size(int64_t N, int32_t n, int32_t H, int32_t W, const igs_config* cfg,
                       int64_t m_capacity, size_t* bytes) {
  if (!bytes) return fail(IGS_ERR_INVALID_ARG, "bytes is NULL");
  if (int r = check_config(cfg, n)) return r;
  if (int r = check_image(H, W, cfg->tile)) return r;
  if (N < 0 || m_capacity < 1 || m_capacity > (int64_t)INT32_MAX)
    return fail(IGS_ERR_INVALID_ARG, "N or m_capacity out of range");
  *bytes = ws_layout(N, n, H, W, cfg->tile, m_capacity).total + fit_extra_bytes(cfg, n, H, W);
  return IGS_OK;
}

int igs_preprocess_bin(const igs_gaussians* g, int32_t H, int32_t W, const igs_config* cfg,
                       void* ws, size_t ws_bytes, int64_t m_capacity, igs_bins* out,
                       igs_stream stream) {
  if (int r = check_gaussians(g)) return r;
  if (int r = check_config(cfg, g->n)) return r;
  if (int r = check_image(H, W, cfg->tile)) return r;
  if (!out) return fail(IGS_ERR_INVALID_ARG, "out is NULL");
  if (!ws) return fail(IGS_ERR_INVALID_ARG, "workspace is NULL");
  if (!aligned(ws, 256)) return fail(IGS_ERR_ALIGN, "workspace must be 256-byte aligned");
  if (m_capacity < 1 || m_capacity > (int64_t)INT32_MAX)
    return fail(IGS_ERR_INVALID_ARG, "m_capacity out of range");
  const WsLayout L = ws_layout(g->N, g->n, H, W, cfg->tile, m_capacity);
  if (ws_bytes < L.total)
    return fail(IGS_ERR_INVALID_ARG, "workspace too small: %zu < %zu bytes", ws_bytes, L.total);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  DevStatus* status = reinterpret_cast<DevStatus*>(base + L.status);
  IGS_CUDA(cudaMemsetAsync(status, 0, sizeof(DevStatus), s), "reset status");

  PrepParams p;
  memset(&p, 0, sizeof(p));
  p.xy = g->xy;
  p.theta = g->theta;
  p.inv_scale = g->inv_scale;
  p.color = g->color;
  p.xy_stride = g->xy_stride;
  p.theta_stride = g->theta_stride;
  p.inv_scale_stride = g->inv_scale_stride;
  p.color_stride = g->color_stride;
  p.N = g->N;
  p.n = g->n;
  p.H = H;
  p.W = W;
  p.tile = cfg->tile;
  p.tiles_x = L.tiles_x;
  p.tiles_y = L.tiles_y;
  p.rec = reinterpret_cast<GRec*>(base + L.rec);
  p.trig = reinterpret_cast<float2*>(base + L.trig);
  p.color_out = reinterpret_cast<float*>(base + L.color);
  if (g->dtype != IGS_F32) {
    p.rec16 = reinterpret_cast<HRec*>(base + L.rec16);
    p.col16 = reinterpret_cast<unsigned short*>(base + L.col16);
  }
  p.tcnt = reinterpret_cast<unsigned int*>(base + L.tcnt);
  p.toff = reinterpret_cast<unsigned long long*>(base + L.toff);
  p.vals = reinterpret_cast<unsigned int*>(base + L.vals);
  p.tmp = reinterpret_cast<unsigned int*>(base + L.tmp);
  p.wide = reinterpret_cast<int*>(base + L.wide);
  p.wide_geo = reinterpret_cast<float4*>(base + L.wide_geo);
  p.m_cap = m_capacity;
  p.status = status;
  unsigned long long* part = reinterpret_cast<unsigned long long*>(base + L.part);
  int2* range = reinterpret_cast<int2*>(base + L.range);
  // lists up to one render stage (tile^2 entries) are ranked by the renderer
  IGS_CUDA(run_binning(p, g->dtype, L.tiles_x * L.tiles_y, part, range, cfg->tile * cfg->tile, s),
           "binning");
  const unsigned int* vals = p.vals;

  out->H = H;
  out->W = W;
  out->tile = cfg->tile;
  out->tiles_x = L.tiles_x;
  out->tiles_y = L.tiles_y;
  out->n = g->n;
  out->N = g->N;
  out->m_capacity = m_capacity;
  out->tile_range = reinterpret_cast<const int32_t*>(range);
  out->list = reinterpret_cast<const int32_t*>(vals);
  out->rec = reinterpret_cast<const float*>(p.rec);
  out->trig = reinterpret_cast<const float*>(p.trig);
  out->color = p.color_out;
  out->status = status;
  out->dtype = g->dtype;
  out->rec16 = p.rec16;
  out->color16 = p.col16;
  return IGS_OK;
}

int igs_render_forward(const igs_bins* bins, const igs_config* cfg, float* d_img,
                       igs_stream stream) {
  if (int r = check_bins(bins, cfg)) return r;
  if (int r = check_config(cfg, bins->n)) return r;
  if (!d_img) return fail(IGS_ERR_INVALID_ARG, "image is NULL");
  if (!aligned(d_img, 4)) return fail(IGS_ERR_ALIGN, "image must be 4-byte aligned");
  RenderParams p = render_params(bins);
  p.normalize = cfg->normalize;
  p.img = d_img;
  IGS_CUDA(launch_render_fwd(p, cfg->tile, cfg->K, reinterpret_cast<cudaStream_t>(stream)),
           "render_forward");
  return IGS_OK;
}

int igs_render_backward(const igs_gaussians* g, const igs_bins* bins, const igs_config* cfg,
                        const float* d_grad_img, const float* d_target, float* d_grad,
                        igs_stream stream) {
  if (int r = check_gaussians(g)) return r;
  if (int r = check_bins(bins, cfg)) return r;
  if (int r = check_config(cfg, bins->n)) return r;
  if (g->N != bins->N || g->n != bins->n)
    return fail(IGS_ERR_INVALID_ARG, "gaussians (N=%lld, n=%d) differ from the bins (N=%lld, n=%d)",
                (long long)g->N, g->n, (long long)bins->N, bins->n);
  if (!d_grad) return fail(IGS_ERR_INVALID_ARG, "grad is NULL");
  if (!d_grad_img && !d_target)
    return fail(IGS_ERR_INVALID_ARG, "need an upstream gradient or an L1 target");
  if (!aligned(d_grad, 4) || (d_grad_img && !aligned(d_grad_img, 4)) ||
      (d_target && !aligned(d_target, 4)))
    return fail(IGS_ERR_ALIGN, "float arrays must be 4-byte aligned");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  IGS_CUDA(cudaMemsetAsync(d_grad, 0, sizeof(float) * (size_t)g->N * (5 + g->n), s),
           "zero grad");
  RenderParams p = render_params(bins);
  p.normalize = cfg->normalize;
  p.grad_img = d_grad_img;
  p.target = d_target;
  p.grad = d_grad;
  IGS_CUDA(launch_render_bwd(p, cfg->tile, cfg->K, s), "render_backward");
  return IGS_OK;
}

static int adam_params(const igs_fit_state* st, const igs_config* cfg, AdamParams* a) {
  if (!st || !st->params || !st->grad || !st->adam_m || !st->adam_v || !st->step)
    return fail(IGS_ERR_INVALID_ARG, "fit state has a NULL pointer");
  if (!cfg) return fail(IGS_ERR_INVALID_ARG, "config is NULL");
  if (st->N < 0 || st->n < 1 || st->n > 32)
    return fail(IGS_ERR_INVALID_ARG, "fit state sizes out of range");
  a->P = st->params;
  a->G = st->grad;
  a->m = st->adam_m;
  a->v = st->adam_v;
  a->step = st->step;
  a->N = st->N;
  a->n = st->n;
  a->lr_mu = cfg->lr_mu;
  a->lr_theta = cfg->lr_theta;
  a->lr_t = cfg->lr_inv_scale;
  a->lr_c = cfg->lr_color;
  a->b1 = (float)cfg->beta1;
  a->b2 = (float)cfg->beta2;
  a->omb1 = (float)(1.0 - cfg->beta1);
  a->omb2 = (float)(1.0 - cfg->beta2);
  a->eps = cfg->eps;
  a->theta_min = cfg->theta_min;
  a->theta_max = cfg->theta_max;
  a->t_min = cfg->t_min;
  a->t_max = cfg->t_max;
  a->mu_min = cfg->mu_min;
  a->mu_max = cfg->mu_max;
  a->fin = nullptr;
  a->fin_inv_count = 0.0f;
  a->fin_loss = nullptr;
  return IGS_OK;
}

int igs_adam_update(const igs_fit_state* st, const igs_config* cfg, igs_stream stream) {
  AdamParams a;
  if (int r = adam_params(st, cfg, &a)) return r;
  IGS_CUDA(launch_adam(a, reinterpret_cast<cudaStream_t>(stream)), "adam");
  return IGS_OK;
}

// A fit step's Adam update, whose last CTA also advances the step counter and
// writes the mean loss (the finalisation).
static int adam_and_finalize(const igs_fit_state* st, const igs_config* cfg, void* status,
                             int32_t H, int32_t W, float* d_loss_out, igs_stream stream) {
  AdamParams a;
  if (int r = adam_params(st, cfg, &a)) return r;
  a.fin = static_cast<DevStatus*>(status);
  a.fin_inv_count = (float)(1.0 / ((double)H * W * st->n));
  a.fin_loss = d_loss_out;
  IGS_CUDA(launch_adam(a, reinterpret_cast<cudaStream_t>(stream)), "adam");
  return IGS_OK;
}

int igs_fit_step(const igs_fit_state* st, const float* d_target, int32_t H, int32_t W,
                 const igs_config* cfg, void* ws, size_t ws_bytes, int64_t m_capacity,
                 float* d_loss_out, igs_stream stream) {
  if (!st || !st->params || !st->grad || !st->adam_m || !st->adam_v || !st->step)
    return fail(IGS_ERR_INVALID_ARG, "fit state has a NULL pointer");
  if (!d_target) return fail(IGS_ERR_INVALID_ARG, "target is NULL");
  if (!aligned(st->params, 16) || !aligned(st->grad, 16) || !aligned(st->adam_m, 16) ||
      !aligned(st->adam_v, 16) || !aligned(d_target, 4))
    return fail(IGS_ERR_ALIGN, "fit state arrays must be 16-byte aligned");
  igs_gaussians g;
  const int np = 5 + st->n;
  g.xy = st->params;
  g.theta = st->params + 2;
  g.inv_scale = st->params + 3;
  g.color = st->params + 5;
  g.xy_stride = g.theta_stride = g.inv_scale_stride = g.color_stride = np;
  g.N = st->N;
  g.n = st->n;
  g.dtype = IGS_F32;
  igs_bins bins;
  if (int r = igs_preprocess_bin(&g, H, W, cfg, ws, ws_bytes, m_capacity, &bins, stream))
    return r;
  const size_t binning_bytes = ws_layout(st->N, st->n, H, W, cfg->tile, m_capacity).total;
  if (ws_bytes < binning_bytes + fit_extra_bytes(cfg, st->n, H, W))
    return fail(IGS_ERR_INVALID_ARG, "workspace too small for the SSIM term");
  if (int r = fit_loss_adjoint(&g, &bins, cfg, d_target, st->grad, static_cast<char*>(ws),
                               binning_bytes, stream))
    return r;
  return adam_and_finalize(st, cfg, bins.status, H, W, d_loss_out, stream);
}

int igs_fit_step_half(const igs_fit_state* st, void* d_params_half, int32_t half_dtype,
                      const float* d_target, int32_t H, int32_t W, const igs_config* cfg,
                      void* ws, size_t ws_bytes, int64_t m_capacity, float* d_loss_out,
                      igs_stream stream) {
  if (!st || !st->params || !st->grad || !st->adam_m || !st->adam_v || !st->step)
    return fail(IGS_ERR_INVALID_ARG, "fit state has a NULL pointer");
  if (!d_params_half || !d_target) return fail(IGS_ERR_INVALID_ARG, "half copy or target is NULL");
  if (half_dtype != IGS_F16 && half_dtype != IGS_BF16)
    return fail(IGS_ERR_INVALID_ARG, "half storage must be IGS_F16 or IGS_BF16");
  if (!aligned(st->params, 16) || !aligned(st->grad, 16) || !aligned(st->adam_m, 16) ||
      !aligned(st->adam_v, 16) || !aligned(d_params_half, 16) || !aligned(d_target, 4))
    return fail(IGS_ERR_ALIGN, "fit state arrays must be 16-byte aligned");
  if (st->N < 0 || st->n < 1 || st->n > 32)
    return fail(IGS_ERR_INVALID_ARG, "fit state sizes out of range");
  const int np = 5 + st->n;
  const int64_t count = st->N * np;
  const bool bf16 = half_dtype == IGS_BF16;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  IGS_CUDA(launch_round_params(st->params, d_params_half, bf16, count, s), "round to half");
  uint16_t* h = static_cast<uint16_t*>(d_params_half);
  igs_gaussians g;
  g.xy = h;
  g.theta = h + 2;
  g.inv_scale = h + 3;
  g.color = h + 5;
  g.xy_stride = g.theta_stride = g.inv_scale_stride = g.color_stride = np;
  g.N = st->N;
  g.n = st->n;
  g.dtype = half_dtype;
  igs_bins bins;
  if (int r = igs_preprocess_bin(&g, H, W, cfg, ws, ws_bytes, m_capacity, &bins, stream))
    return r;
  const size_t binning_bytes = ws_layout(st->N, st->n, H, W, cfg->tile, m_capacity).total;
  if (ws_bytes < binning_bytes + fit_extra_bytes(cfg, st->n, H, W))
    return fail(IGS_ERR_INVALID_ARG, "workspace too small for the SSIM term");
  if (int r = fit_loss_adjoint(&g, &bins, cfg, d_target, st->grad, static_cast<char*>(ws),
                               binning_bytes, stream))
    return r;
  if (int r = adam_and_finalize(st, cfg, bins.status, H, W, d_loss_out, stream)) return r;
  IGS_CUDA(launch_round_params(st->params, d_params_half, bf16, count, s), "round to half");
  return IGS_OK;
}

int igs_decode_points(const igs_bins* bins, const igs_config* cfg, const float* d_xy, int64_t Q,
                      float* d_out, igs_stream stream) {
  if (int r = check_bins(bins, cfg)) return r;
  if (int r = check_config(cfg, bins->n)) return r;
  if (Q < 0) return fail(IGS_ERR_INVALID_ARG, "Q < 0");
  if (Q > 0 && (!d_xy || !d_out)) return fail(IGS_ERR_INVALID_ARG, "points or output NULL");
  if (!aligned(d_xy, 4) || !aligned(d_out, 4))
    return fail(IGS_ERR_ALIGN, "float arrays must be 4-byte aligned");
  RenderParams p = render_params(bins);
  p.normalize = cfg->normalize;
  p.qxy = d_xy;
  p.qout = d_out;
  p.Q = Q;
  IGS_CUDA(launch_decode(p, cfg->K, reinterpret_cast<cudaStream_t>(stream)), "decode");
  return IGS_OK;
}

int igs_image_loss_workspace_size(int32_t n, int32_t H, int32_t W, size_t* bytes) {
  if (!bytes) return fail(IGS_ERR_INVALID_ARG, "bytes is NULL");
  if (n < 1 || H < 1 || W < 1) return fail(IGS_ERR_INVALID_ARG, "sizes must be positive");
  *bytes = 256 + image_loss_scratch_bytes(n, H, W);
  return IGS_OK;
}

int igs_image_loss(const float* d_render, const float* d_target, int32_t n, int32_t H,
                   int32_t W, float ssim_weight, float* d_grad_img, float* d_loss_out,
                   void* ws, size_t ws_bytes, igs_stream stream) {
  if (n < 1 || H < 1 || W < 1) return fail(IGS_ERR_INVALID_ARG, "sizes must be positive");
  if (!d_render || !d_target || !d_grad_img || !ws)
    return fail(IGS_ERR_INVALID_ARG, "render, target, gradient or workspace NULL");
  if (!(ssim_weight >= 0.0f && ssim_weight <= 1e6f))
    return fail(IGS_ERR_INVALID_ARG, "ssim_weight must be finite and >= 0");
  if (!aligned(d_render, 4) || !aligned(d_target, 4) || !aligned(d_grad_img, 4) ||
      !aligned(d_loss_out, 4) || !aligned(ws, 256))
    return fail(IGS_ERR_ALIGN, "arrays 4-byte, workspace 256-byte aligned");
  if (ws_bytes < 256 + image_loss_scratch_bytes(n, H, W))
    return fail(IGS_ERR_INVALID_ARG, "image-loss workspace too small");
  char* base = static_cast<char*>(ws);
  IGS_CUDA(launch_image_loss(d_render, d_target, n, H, W, ssim_weight, d_grad_img,
                             reinterpret_cast<double*>(base), d_loss_out, base + 256,
                             reinterpret_cast<cudaStream_t>(stream)),
           "image loss");
  return IGS_OK;
}

int igs_placement_workspace_size(int32_t H, int32_t W, size_t* bytes) {
  if (!bytes) return fail(IGS_ERR_INVALID_ARG, "bytes is NULL");
  if (H < 1 || W < 1) return fail(IGS_ERR_INVALID_ARG, "image size must be positive");
  *bytes = place_layout((int64_t)H * W).bytes;
  return IGS_OK;
}

static int check_place(const float* d_target, int32_t H, int32_t W, int32_t n,
                       const uint64_t* d_rand, int64_t count, void* ws, size_t ws_bytes) {
  if (H < 1 || W < 1 || n < 1 || n > 32 || count < 0)
    return fail(IGS_ERR_INVALID_ARG, "sizes out of range");
  if (!d_target || !ws || (count > 0 && !d_rand))
    return fail(IGS_ERR_INVALID_ARG, "target, workspace or random numbers NULL");
  if (!aligned(d_target, 4) || !aligned(d_rand, 8) || !aligned(ws, 256))
    return fail(IGS_ERR_ALIGN, "target 4-, random numbers 8-, workspace 256-byte aligned");
  if (ws_bytes < place_layout((int64_t)H * W).bytes)
    return fail(IGS_ERR_INVALID_ARG, "placement workspace too small");
  return IGS_OK;
}

int igs_init_gaussians(const float* d_target, int32_t H, int32_t W, int32_t n, int64_t N,
                       double lambda, const uint64_t* d_rand, float* d_params, void* ws,
                       size_t ws_bytes, igs_stream stream) {
  if (int r = check_place(d_target, H, W, n, d_rand, N, ws, ws_bytes)) return r;
  if (!(lambda >= 0.0 && lambda <= 1.0)) return fail(IGS_ERR_INVALID_ARG, "lambda not in [0, 1]");
  if (N > 0 && !d_params) return fail(IGS_ERR_INVALID_ARG, "params NULL");
  if (!aligned(d_params, 4)) return fail(IGS_ERR_ALIGN, "params must be 4-byte aligned");
  IGS_CUDA(launch_place(d_target, nullptr, H, W, n,
                        reinterpret_cast<const unsigned long long*>(d_rand), N, lambda, d_params,
                        0, nullptr, nullptr, nullptr, static_cast<char*>(ws),
                        reinterpret_cast<cudaStream_t>(stream)),
           "init gaussians");
  return IGS_OK;
}

int igs_add_gaussians(const float* d_target, const float* d_render, int32_t H, int32_t W,
                      const uint64_t* d_rand, int64_t count, const igs_fit_state* st, void* ws,
                      size_t ws_bytes, igs_stream stream) {
  if (!st || !st->params || !st->grad || !st->adam_m || !st->adam_v)
    return fail(IGS_ERR_INVALID_ARG, "fit state has a NULL pointer");
  if (int r = check_place(d_target, H, W, st->n, d_rand, count, ws, ws_bytes)) return r;
  if (!d_render) return fail(IGS_ERR_INVALID_ARG, "render is NULL");
  if (!aligned(d_render, 4)) return fail(IGS_ERR_ALIGN, "render must be 4-byte aligned");
  IGS_CUDA(launch_place(d_target, d_render, H, W, st->n,
                        reinterpret_cast<const unsigned long long*>(d_rand), count, 0.0,
                        st->params, st->N, st->grad, st->adam_m, st->adam_v,
                        static_cast<char*>(ws), reinterpret_cast<cudaStream_t>(stream)),
           "add gaussians");
  return IGS_OK;
}

int igs_read_stats(const igs_bins* bins, igs_stats* out, igs_stream stream) {
  if (!bins || !bins->status || !out) return fail(IGS_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  static_assert(sizeof(igs_stats) == 32, "igs_stats layout");
  IGS_CUDA(cudaMemcpyAsync(out, bins->status, sizeof(igs_stats), cudaMemcpyDeviceToHost, s),
           "read stats");
  IGS_CUDA(cudaStreamSynchronize(s), "read stats sync");
  return IGS_OK;
}

}  // extern "C"
