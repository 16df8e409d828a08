// Per-tile forward render (Eq. 5 with top-K, Sec. 3.2), its adjoint
// (Sec. 3.3: gradients through the K retained Gaussians) fused with the L1
// loss, and random-access decode. Included by the translation units that
// instantiate and dispatch them.
//
// One CTA renders one logical tile (TILE x TILE pixels, one pixel per
// thread). The tile's list S_j is staged through shared memory in chunks of
// TILE*TILE Gaussians; every pixel ranks each candidate by its binary32 key q
// and keeps the K smallest in registers. The insertion network runs only
// when some lane of the warp improves on its current K-th key (warp vote),
// so the common reject costs one compare. Colours of the K winners are read
// once at the end (the blend needs only the K winners).
//
// The adjoint recomputes the selection and the weights (nothing is stored
// between forward and backward), forms dL/dq for each winner and reduces the
// per-pixel contributions of the tile in shared memory, one slot per list
// position, before one global atomic per (tile, Gaussian, parameter).
#pragma once
#include "internal.h"

namespace igs {

template <int NC> struct Chan { static constexpr int R = NC; };
template <> struct Chan<0> { static constexpr int R = 32; };  // runtime n <= 32

template <int NC>
__device__ __forceinline__ int nchan(const RenderParams& p) {
  return NC > 0 ? NC : p.n;
}

// Shared-memory gradient slots for the adjoint (one row of 5+n floats per
// list position); positions beyond the capacity use global atomics.
template <int NC> struct AccCap {
  static constexpr int NP = 5 + Chan<NC>::R;
  static constexpr int L = ((8192 / NP) / 32) * 32;
};

// Top-K selection over the tile's list for pixel (px, py).
template <int TILE, int K>
__device__ __forceinline__ void select_topk(const RenderParams& p, int2 range, float px,
                                            float py, float (&tq)[K], int (&tp)[K],
                                            float4* s_a, float* s_a11) {
  constexpr int NT = TILE * TILE;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    tq[k] = __int_as_float(0x7f800000);  // +inf
    tp[k] = -1;
  }
  for (int base = range.x; base < range.y; base += NT) {
    const int cnt = min(NT, range.y - base);
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      const int gid = p.list[base + threadIdx.x];
      if ((unsigned)gid < (unsigned)p.N) {
        const GRec g = p.rec[gid];
        s_a[threadIdx.x] = g.a;
        s_a11[threadIdx.x] = g.b.x;
      } else {  // corrupt list entry: a NaN key is never selected
        s_a[threadIdx.x] = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
        s_a11[threadIdx.x] = 0.0f;
        atomicOr(&p.status->flags, FLAG_INTERNAL);
      }
    }
    __syncthreads();
    const int rel = base - range.x;
#pragma unroll 4
    for (int j = 0; j < cnt; ++j) {
      const float4 a = s_a[j];
      const float q = rank_key(px, py, a.x, a.y, a.z, a.w, s_a11[j]);
      if (__any_sync(FULL_MASK, q < tq[K - 1])) topk_insert<K>(tq, tp, q, rel + j);
    }
  }
}

// Weights of the winners and the blended colour (Eq. 5, max-shifted).
template <int K, int NC>
__device__ __forceinline__ float blend(const RenderParams& p, int2 range, const float (&tq)[K],
                                       const int (&tp)[K], float (&w)[K], int (&gid)[K],
                                       float (&cr)[Chan<NC>::R]) {
  const int n = nchan<NC>(p);
#pragma unroll
  for (int c = 0; c < Chan<NC>::R; ++c) cr[c] = 0.0f;
  float Z = 0.0f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    w[k] = 0.0f;
    gid[k] = -1;
    if (tp[k] >= 0) {
      w[k] = exp2f((tq[0] - tq[k]) * HALF_LOG2E);
      Z += w[k];
      gid[k] = p.list[range.x + tp[k]];
      const float* col = p.color + (int64_t)gid[k] * n;
#pragma unroll
      for (int c = 0; c < Chan<NC>::R; ++c)
        if (NC > 0 || c < n) cr[c] = fmaf(w[k], col[c], cr[c]);
    }
  }
  const float iz = Z > 0.0f ? 1.0f / Z : 0.0f;
#pragma unroll
  for (int c = 0; c < Chan<NC>::R; ++c) cr[c] *= iz;
  return iz;
}

template <int TILE, int K, int NC>
__global__ void __launch_bounds__(TILE * TILE) k_render_fwd(RenderParams p) {
  constexpr int NT = TILE * TILE;
  __shared__ float4 s_a[NT];
  __shared__ float s_a11[NT];
  const int tile_id = blockIdx.x;
  const int tx = tile_id % p.tiles_x, ty = tile_id / p.tiles_x;
  const int x = tx * TILE + (int)(threadIdx.x % TILE);
  const int y = ty * TILE + (int)(threadIdx.x / TILE);
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const int2 range = p.range[tile_id];
  float tq[K];
  int tp[K];
  select_topk<TILE, K>(p, range, px, py, tq, tp, s_a, s_a11);
  if (x >= p.W || y >= p.H) return;
  float w[K];
  int gid[K];
  float cr[Chan<NC>::R];
  blend<K, NC>(p, range, tq, tp, w, gid, cr);
  const int n = nchan<NC>(p);
  const int64_t plane = (int64_t)p.H * p.W;
  const int64_t o = (int64_t)y * p.W + x;
#pragma unroll
  for (int c = 0; c < Chan<NC>::R; ++c)
    if (NC > 0 || c < n) p.img[c * plane + o] = cr[c];
}

template <int TILE, int K, int NC>
__global__ void __launch_bounds__(TILE * TILE) k_render_bwd(RenderParams p) {
  constexpr int NT = TILE * TILE;
  constexpr int NCR = Chan<NC>::R;
  constexpr int LCAP = AccCap<NC>::L;
  __shared__ float4 s_a[NT];
  __shared__ float s_a11[NT];
  __shared__ float s_acc[LCAP * AccCap<NC>::NP];
  __shared__ double s_loss[NT / 32];
  const int n = nchan<NC>(p);
  const int np = 5 + n;
  const int tile_id = blockIdx.x;
  const int tx = tile_id % p.tiles_x, ty = tile_id / p.tiles_x;
  const int x = tx * TILE + (int)(threadIdx.x % TILE);
  const int y = ty * TILE + (int)(threadIdx.x / TILE);
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const int2 range = p.range[tile_id];
  const int len = range.y - range.x;
  const int slots = min(len, LCAP);
  for (int i = threadIdx.x; i < slots * np; i += NT) s_acc[i] = 0.0f;

  float tq[K];
  int tp[K];
  select_topk<TILE, K>(p, range, px, py, tq, tp, s_a, s_a11);
  __syncthreads();  // s_acc zeroed before any contribution

  float loss = 0.0f;
  const bool inside = x < p.W && y < p.H;
  if (inside && len > 0) {
    float w[K];
    int gid[K];
    float cr[NCR];
    const float iz = blend<K, NC>(p, range, tq, tp, w, gid, cr);
    const int64_t plane = (int64_t)p.H * p.W;
    const int64_t o = (int64_t)y * p.W + x;
    float g[NCR];
    float gdot_r = 0.0f;
#pragma unroll
    for (int c = 0; c < NCR; ++c) {
      g[c] = 0.0f;
      if (NC > 0 || c < n) {
        if (p.grad_img) {
          g[c] = p.grad_img[c * plane + o];
        } else {
          const float d = cr[c] - p.target[c * plane + o];
          loss += fabsf(d);
          g[c] = sign_f(d) * p.inv_count;
        }
        gdot_r = fmaf(g[c], cr[c], gdot_r);
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (gid[k] < 0) continue;
      const int id = gid[k];
      const float wz = w[k] * iz;
      const float* col = p.color + (int64_t)id * n;
      float gdot = 0.0f;
#pragma unroll
      for (int c = 0; c < NCR; ++c)
        if (NC > 0 || c < n) gdot = fmaf(g[c], col[c], gdot);
      const float Gq = -0.5f * wz * (gdot - gdot_r);
      const GRec rc = p.rec[id];
      const float2 cs = p.trig[id];
      const float dx = px - rc.a.x, dy = py - rc.a.y;
      const float a = cs.x * dx + cs.y * dy;
      const float b = -cs.y * dx + cs.x * dy;
      const float t1 = rc.b.z, t2 = rc.b.w;
      const float T1 = t1 * t1, T2 = t2 * t2;
      const float Ta = T1 * a, Tb = T2 * b;
      float v[5];
      v[0] = Gq * -2.0f * (Ta * cs.x - Tb * cs.y) * (float)p.W;
      v[1] = Gq * -2.0f * (Ta * cs.y + Tb * cs.x) * (float)p.H;
      v[2] = Gq * 2.0f * a * b * (T1 - T2);
      v[3] = Gq * 2.0f * t1 * a * a;
      v[4] = Gq * 2.0f * t2 * b * b;
      const int pos = tp[k];
      if (pos < LCAP) {
        float* dst = s_acc + pos * np;
#pragma unroll
        for (int j = 0; j < 5; ++j) atomicAdd(dst + j, v[j]);
#pragma unroll
        for (int c = 0; c < NCR; ++c)
          if (NC > 0 || c < n) atomicAdd(dst + 5 + c, wz * g[c]);
      } else {
        float* dst = p.grad + (int64_t)id * np;
#pragma unroll
        for (int j = 0; j < 5; ++j) atomicAdd(dst + j, v[j]);
#pragma unroll
        for (int c = 0; c < NCR; ++c)
          if (NC > 0 || c < n) atomicAdd(dst + 5 + c, wz * g[c]);
      }
    }
  }
  if (!p.grad_img) {
    double l = warp_sum<double>((double)loss);
    if ((threadIdx.x & 31) == 0) s_loss[threadIdx.x >> 5] = l;
  }
  __syncthreads();
  if (!p.grad_img && threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < NT / 32; ++i) t += s_loss[i];
    if (t != 0.0) atomicAdd(&p.status->loss_sum, t);
  }
  for (int i = threadIdx.x; i < slots * np; i += NT) {
    const float v = s_acc[i];
    if (v != 0.0f) {
      const int pos = i / np, j = i - pos * np;
      const int id = p.list[range.x + pos];
      atomicAdd(p.grad + (int64_t)id * np + j, v);
    }
  }
}

// One thread per query point: its tile's list is walked from global memory.
template <int K, int NC>
__global__ void __launch_bounds__(256) k_decode(RenderParams p) {
  const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= p.Q) return;
  const float px = p.qxy[2 * qi], py = p.qxy[2 * qi + 1];
  const float inv = 1.0f / (float)p.tile;
  const float fx = fminf(fmaxf(floorf(px * inv), 0.0f), (float)(p.tiles_x - 1));
  const float fy = fminf(fmaxf(floorf(py * inv), 0.0f), (float)(p.tiles_y - 1));
  const int2 range = p.range[(int)fy * p.tiles_x + (int)fx];
  float tq[K];
  int tp[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    tq[k] = __int_as_float(0x7f800000);
    tp[k] = -1;
  }
  for (int j = range.x; j < range.y; ++j) {
    const int id = p.list[j];
    if ((unsigned)id >= (unsigned)p.N) continue;
    const GRec g = p.rec[id];
    const float q = rank_key(px, py, g.a.x, g.a.y, g.a.z, g.a.w, g.b.x);
    if (q < tq[K - 1]) topk_insert<K>(tq, tp, q, j - range.x);
  }
  float w[K];
  int gid[K];
  float cr[Chan<NC>::R];
  blend<K, NC>(p, range, tq, tp, w, gid, cr);
  const int n = nchan<NC>(p);
#pragma unroll
  for (int c = 0; c < Chan<NC>::R; ++c)
    if (NC > 0 || c < n) p.qout[qi * n + c] = cr[c];
}

// Dispatch over the supported K and channel counts.
#define IGS_FOR_K(M, ...)                          \
  switch (K) {                                     \
    case 1: M(1, __VA_ARGS__); break;              \
    case 2: M(2, __VA_ARGS__); break;              \
    case 3: M(3, __VA_ARGS__); break;              \
    case 4: M(4, __VA_ARGS__); break;              \
    case 8: M(8, __VA_ARGS__); break;              \
    case 10: M(10, __VA_ARGS__); break;            \
    case 16: M(16, __VA_ARGS__); break;            \
    default: return cudaErrorInvalidValue;         \
  }

#define IGS_NC_OF(n) ((n) == 1 ? 1 : (n) == 3 ? 3 : (n) == 4 ? 4 : (n) == 9 ? 9 : 0)

inline bool k_supported(int K) {
  return K == 1 || K == 2 || K == 3 || K == 4 || K == 8 || K == 10 || K == 16;
}

}  // namespace igs
