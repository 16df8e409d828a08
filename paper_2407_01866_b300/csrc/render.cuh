// Per-tile forward render (Eq. 5 with top-K, Sec. 3.2), its adjoint
// (Sec. 3.3: gradients through the K retained Gaussians) fused with the L1
// loss, and random-access decode. Included by the translation units that
// instantiate and dispatch them.
//
// One CTA renders one logical tile of TILE x TILE pixels, one pixel per
// thread; each warp owns a compact 8 x 4 block so that its pixels share
// most of their winners. The tile's list S_j (ascending Gaussian index) is
// staged through shared memory in chunks of TILE*TILE records.
//
//   pass A  keys only: every pixel keeps its K smallest ranking keys q with a
//           min/max insertion network, run only when some lane of the warp
//           improves on its K-th key (warp vote). Gives q_min and the
//           threshold tau = K-th smallest key.
//   pass B  list order: a candidate is a winner iff q < tau, or q == tau
//           while equal-key slots remain (K minus the keys below tau), which
//           is exactly the top-K of the (q, index) order. Winners are blended
//           with w = exp(-(q - q_min)/2) (Eq. 5).
//   pass C  (adjoint only) candidate-major: threads own (candidate, group of
//           pixels), re-test membership exactly from each pixel's (tau,
//           position of its last tau-valued winner), and accumulate dL/dq
//           moments in registers; one reduction and 5+n global atomics per
//           (tile, Gaussian). Nothing is stored between forward and adjoint.
#pragma once
#include "internal.h"

namespace igs {

template <int NC> struct Chan { static constexpr int R = NC; };
template <> struct Chan<0> { static constexpr int R = 32; };  // runtime n <= 32

template <int NC>
__device__ __forceinline__ int nchan(const RenderParams& p) {
  return NC > 0 ? NC : p.n;
}

// Local (x, y) of the pixel owned by thread t: warp w covers an 8 x 4 block.
template <int TILE>
__device__ __forceinline__ int2 pixel_of(int t) {
  constexpr int BPR = TILE / 8;  // 8-wide blocks per tile row
  const int w = t >> 5, lane = t & 31;
  return make_int2((w % BPR) * 8 + (lane & 7), (w / BPR) * 4 + (lane >> 3));
}

constexpr float F_INF = __builtin_huge_valf();

// Stage list entries [base, base+cnt) of the tile: geometry and index.
template <int NT>
__device__ __forceinline__ void stage_chunk(const RenderParams& p, int base, int cnt,
                                            float4* s_a, float* s_a11, int* s_gid) {
  if ((int)threadIdx.x < cnt) {
    const int gid = p.list[base + threadIdx.x];
    if ((unsigned)gid < (unsigned)p.N) {
      const GRec g = p.rec[gid];
      s_a[threadIdx.x] = g.a;
      s_a11[threadIdx.x] = g.b.x;
      s_gid[threadIdx.x] = gid;
    } else {  // corrupt list entry: a NaN key is never selected
      s_a[threadIdx.x] = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
      s_a11[threadIdx.x] = 0.0f;
      s_gid[threadIdx.x] = -1;
      atomicOr(&p.status->flags, FLAG_INTERNAL);
    }
  }
}

// Pass A: the K smallest keys at (px, py), ascending. CH list entries are
// staged per round ("Gaussians per stage", CH <= TILE*TILE).
template <int TILE, int K, int CH>
__device__ __forceinline__ void select_keys(const RenderParams& p, int2 range, float px,
                                            float py, float (&tq)[K], float4* s_a, float* s_a11,
                                            int* s_gid) {
#pragma unroll
  for (int k = 0; k < K; ++k) tq[k] = F_INF;
  for (int base = range.x; base < range.y; base += CH) {
    const int cnt = min(CH, range.y - base);
    __syncthreads();
    stage_chunk<CH>(p, base, cnt, s_a, s_a11, s_gid);
    __syncthreads();
#pragma unroll 4
    for (int j = 0; j < cnt; ++j) {
      const float4 a = s_a[j];
      const float q = rank_key(px, py, a.x, a.y, a.z, a.w, s_a11[j]);
      const bool better = q < tq[K - 1];
      if (__any_sync(FULL_MASK, better)) {
        float x = better ? q : F_INF;  // +inf (and NaN) insert nothing
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float lo = fminf(tq[k], x);
          x = fmaxf(tq[k], x);
          tq[k] = lo;
        }
      }
    }
  }
}

// Per-pixel result of pass B.
template <int NCR>
struct PixelBlend {
  float Z;          // sum of winner weights (0 if the pixel has none)
  float cr[NCR];    // blended colour
  float tau;        // K-th key (+inf if |S_j| < K)
  float q0;         // smallest key
  int posK;         // list position of the last tau-valued winner
};

// Pass B: exact top-K membership in list order and the blend of Eq. 5.
template <int TILE, int K, int NC, int CH>
__device__ __forceinline__ void blend_pass(const RenderParams& p, int2 range, float px,
                                           float py, const float (&tq)[K],
                                           PixelBlend<Chan<NC>::R>& r, float4* s_a,
                                           float* s_a11, int* s_gid) {
  constexpr int NCR = Chan<NC>::R;
  const int n = nchan<NC>(p);
  r.q0 = tq[0];
  r.tau = tq[K - 1];
  int lt = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) lt += tq[k] < r.tau ? 1 : 0;
  int eq_left = K - lt;  // tau-valued slots still open
  r.posK = -1;
  r.Z = 0.0f;
#pragma unroll
  for (int c = 0; c < NCR; ++c) r.cr[c] = 0.0f;
  for (int base = range.x; base < range.y; base += CH) {
    const int cnt = min(CH, range.y - base);
    __syncthreads();
    stage_chunk<CH>(p, base, cnt, s_a, s_a11, s_gid);
    __syncthreads();
    const int rel = base - range.x;
#pragma unroll 2
    for (int j = 0; j < cnt; ++j) {
      const float4 a = s_a[j];
      const float q = rank_key(px, py, a.x, a.y, a.z, a.w, s_a11[j]);
      bool win = q < r.tau;
      if (q == r.tau && eq_left > 0) {
        win = true;
        --eq_left;
        r.posK = rel + j;
      }
      if (__any_sync(FULL_MASK, win)) {
        if (win) {
          const float w = exp2f((r.q0 - q) * HALF_LOG2E);  // exactly 1 at q = q_min
          r.Z += w;
          const float* col = p.color + (int64_t)s_gid[j] * n;
#pragma unroll
          for (int c = 0; c < NCR; ++c)
            if (NC > 0 || c < n) r.cr[c] = fmaf(w, col[c], r.cr[c]);
        }
      }
    }
  }
  const float iz = r.Z > 0.0f ? 1.0f / r.Z : 0.0f;
#pragma unroll
  for (int c = 0; c < NCR; ++c) r.cr[c] *= iz;
}

// ---------------------------------------------------------------------------
// Fast path for tiles whose whole list fits one stage (the common case).
//
// Each warp orders the staged candidates by their key at the centre of its
// 8 x 4 block, so that pass A meets the winners first and its insertion
// network rarely runs late in the list. Pass A also records whether a
// candidate whose key equals the final threshold tau was dropped (a boundary
// tie). Without one, the winners are exactly the candidates with q <= tau,
// and pass B walks the same order and stops once every lane of the warp has
// found its K winners. A warp with a tie falls back to list order and the
// exact (q, index) rule. Pass B's ballots give, per (warp block, candidate),
// the mask of pixels where the candidate wins; the adjoint visits only those.
// ---------------------------------------------------------------------------

// Bitonic sort of this warp's candidates by key at (cx, cy); so[] gets the order.
template <int CH>
__device__ __forceinline__ void warp_order(int cnt, float cx, float cy, const float4* s_a,
                                           const float* s_a11, float* sk, short* so) {
  const int lane = threadIdx.x & 31;
  int P = 32;
  while (P < cnt) P <<= 1;
  for (int i = lane; i < P; i += 32) {
    float k = F_INF;
    if (i < cnt) {
      const float4 a = s_a[i];
      k = rank_key(cx, cy, a.x, a.y, a.z, a.w, s_a11[i]);
      if (!(k == k)) k = F_INF;
    }
    sk[i] = k;
    so[i] = (short)i;
  }
  __syncwarp();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < P; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const float a = sk[i], b = sk[l];
          if ((a > b) == ((i & k) == 0)) {
            sk[i] = b;
            sk[l] = a;
            const short t = so[i];
            so[i] = so[l];
            so[l] = t;
          }
        }
      }
      __syncwarp();
    }
  }
}

// Pass A over the warp's order; `tie` = a tau-valued candidate was dropped.
template <int K>
__device__ __forceinline__ void fast_keys(int cnt, float px, float py, const float4* s_a,
                                          const float* s_a11, const short* so, float (&tq)[K],
                                          bool& tie) {
#pragma unroll
  for (int k = 0; k < K; ++k) tq[k] = F_INF;
  float v_drop = F_INF;
#pragma unroll 2
  for (int o = 0; o < cnt; ++o) {
    const int j = so[o];
    const float4 a = s_a[j];
    const float q = rank_key(px, py, a.x, a.y, a.z, a.w, s_a11[j]);
    const float thr = tq[K - 1];
    const bool better = q < thr;
    if (q == thr) v_drop = fminf(v_drop, q);  // rejected at the threshold
    if (__any_sync(FULL_MASK, better)) {
      float x = better ? q : F_INF;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float lo = fminf(tq[k], x);
        x = fmaxf(tq[k], x);
        tq[k] = lo;
      }
      if (better && tq[K - 1] == thr) v_drop = fminf(v_drop, thr);  // evicted at it
    }
  }
  tie = tq[K - 1] < F_INF && v_drop == tq[K - 1];
}

// Pass B over the staged list: blend the winners and, if MASK, store the
// ballot of winning live pixels per candidate in mask_w[] (this warp's row).
template <int K, int NC, bool MASK>
__device__ __forceinline__ void fast_blend(const RenderParams& p, int cnt, float px, float py,
                                           bool live, const float (&tq)[K], bool warp_tie,
                                           const float4* s_a, const float* s_a11,
                                           const int* s_gid, const short* so,
                                           unsigned* mask_w, PixelBlend<Chan<NC>::R>& r) {
  constexpr int NCR = Chan<NC>::R;
  const int n = nchan<NC>(p);
  const int lane = threadIdx.x & 31;
  r.q0 = tq[0];
  r.tau = tq[K - 1];
  r.posK = 0x7fffffff;
  r.Z = 0.0f;
#pragma unroll
  for (int c = 0; c < NCR; ++c) r.cr[c] = 0.0f;
  if (!warp_tie) {
    const int need = min(K, cnt);
    int found = 0;
    for (int o = 0; o < cnt; ++o) {
      if (!__any_sync(FULL_MASK, found < need)) break;
      const int j = so[o];
      const float4 a = s_a[j];
      const float q = rank_key(px, py, a.x, a.y, a.z, a.w, s_a11[j]);
      const bool win = found < need && q <= r.tau;
      const unsigned bal = __ballot_sync(FULL_MASK, win);
      if (MASK) {
        const unsigned lb = __ballot_sync(FULL_MASK, win && live);
        if (lane == 0) mask_w[j] = lb;
      }
      if (bal && win) {
        ++found;
        const float w = exp2f((r.q0 - q) * HALF_LOG2E);
        r.Z += w;
        const float* col = p.color + (int64_t)s_gid[j] * n;
#pragma unroll
        for (int c = 0; c < NCR; ++c)
          if (NC > 0 || c < n) r.cr[c] = fmaf(w, col[c], r.cr[c]);
      }
    }
  } else {
    int lt = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) lt += tq[k] < r.tau ? 1 : 0;
    int eq_left = K - lt;
    for (int j = 0; j < cnt; ++j) {
      const float4 a = s_a[j];
      const float q = rank_key(px, py, a.x, a.y, a.z, a.w, s_a11[j]);
      bool win = q < r.tau;
      if (q == r.tau && eq_left > 0) {
        win = true;
        --eq_left;
        r.posK = j;
      }
      const unsigned bal = __ballot_sync(FULL_MASK, win && live);
      if (MASK && lane == 0) mask_w[j] = bal;
      if (win) {
        const float w = exp2f((r.q0 - q) * HALF_LOG2E);
        r.Z += w;
        const float* col = p.color + (int64_t)s_gid[j] * n;
#pragma unroll
        for (int c = 0; c < NCR; ++c)
          if (NC > 0 || c < n) r.cr[c] = fmaf(w, col[c], r.cr[c]);
      }
    }
  }
  const float iz = r.Z > 0.0f ? 1.0f / r.Z : 0.0f;
#pragma unroll
  for (int c = 0; c < NCR; ++c) r.cr[c] *= iz;
}

template <int TILE>
__device__ __forceinline__ float2 block_centre(int x0, int y0) {
  constexpr int BPR = TILE / 8;
  const int w = threadIdx.x >> 5;
  return make_float2((float)(x0 + (w % BPR) * 8 + 4), (float)(y0 + (w / BPR) * 4 + 2));
}

template <int TILE, int K, int NC>
__global__ void __launch_bounds__(TILE * TILE) k_render_fwd(RenderParams p) {
  constexpr int NT = TILE * TILE;
  constexpr int NWB = NT / 32;
  __shared__ float4 s_a[NT];
  __shared__ float s_a11[NT];
  __shared__ int s_gid[NT];
  __shared__ float s_key[NWB][NT];
  __shared__ short s_ord[NWB][NT];
  const int tile_id = blockIdx.x;
  const int tx = tile_id % p.tiles_x, ty = tile_id / p.tiles_x;
  const int2 lp = pixel_of<TILE>(threadIdx.x);
  const int x = tx * TILE + lp.x, y = ty * TILE + lp.y;
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const int2 range = p.range[tile_id];
  const int len = range.y - range.x;
  float tq[K];
  PixelBlend<Chan<NC>::R> r;
  if (len <= NT) {
    stage_chunk<NT>(p, range.x, len, s_a, s_a11, s_gid);
    __syncthreads();
    const int w = threadIdx.x >> 5;
    const float2 c = block_centre<TILE>(tx * TILE, ty * TILE);
    warp_order<NT>(len, c.x, c.y, s_a, s_a11, s_key[w], s_ord[w]);
    bool tie;
    fast_keys<K>(len, px, py, s_a, s_a11, s_ord[w], tq, tie);
    const bool warp_tie = __any_sync(FULL_MASK, tie);
    fast_blend<K, NC, false>(p, len, px, py, true, tq, warp_tie, s_a, s_a11, s_gid, s_ord[w],
                             nullptr, r);
  } else {
    select_keys<TILE, K, NT>(p, range, px, py, tq, s_a, s_a11, s_gid);
    blend_pass<TILE, K, NC, NT>(p, range, px, py, tq, r, s_a, s_a11, s_gid);
  }
  if (x >= p.W || y >= p.H) return;
  const int n = nchan<NC>(p);
  const int64_t plane = (int64_t)p.H * p.W;
  const int64_t o = (int64_t)y * p.W + x;
#pragma unroll
  for (int c = 0; c < Chan<NC>::R; ++c)
    if (NC > 0 || c < n) p.img[c * plane + o] = r.cr[c];
}

// Where one tile of one image lives (the batched form renders many images).
struct TileCtx {
  int2 range;        // [start, end) of the tile's list
  int x0, y0;        // tile origin in pixels
  int H, W;          // its image
  int64_t off;       // offset (floats) of the image in img / target / grad_img
  float inv_count;   // 1 / (H W n)
  double* loss_acc;  // where the tile adds sum |c_r - c_t|
};

// Dynamic shared-memory layout of the adjoint kernel (in 4-byte words), for
// NT pixels, n channels and CH Gaussians per stage.
struct BwdSmem {
  int a, a11, gid, ps0, ps1, gh, part, loss, key, ord, mask, items, inv, hist, total;
};
__host__ __device__ inline BwdSmem bwd_smem(int NT, int n, int CH) {
  const int NWB = NT / 32;
  BwdSmem L;
  int o = 0;
  L.a = o;     o += 4 * NT;          // float4 staged geometry
  L.a11 = o;   o += NT;
  L.gid = o;   o += NT;
  L.ps0 = o;   o += 4 * NT;          // float4 (px, py, tau, q0)
  L.ps1 = o;   o += 2 * NT;          // float2 (posK bits, beta)
  L.gh = o;    o += n * NT;          // per-pixel -g/(2Z), channel-major
  L.part = o;  o += (5 + n) * NT;    // pass C partial sums
  L.loss = o;  o += 2 * (NT / 32);   // doubles
  L.key = o;   o += NWB * CH;        // per-warp candidate order: keys
  L.ord = o;   o += (NWB * CH + 1) / 2;  // shorts
  L.mask = o;  o += NWB * CH;        // winner masks [warp block][candidate]
  L.items = o; o += NWB * CH;        // (candidate, block) work items
  L.inv = o;   o += (NWB * CH + 1) / 2;  // shorts: item position of (candidate, block)
  L.hist = o;  o += 36;
  L.total = o;
  return L;
}

// Adjoint pass C of the fast path: visit only the (candidate, warp block)
// items whose mask is non-empty, longest first so that the lanes of a warp
// get similar loops; each item's sums go to its own slot and every candidate
// adds its items' slots in block order (no shared atomics on floats).
template <int TILE, int NC, int CH>
__device__ __forceinline__ void fast_pass_c(const RenderParams& p, const TileCtx& t, int cnt,
                                            const float4* s_a, const float* s_a11,
                                            const int* s_gid, const unsigned* s_mask,
                                            const float4* s_ps0, const float2* s_ps1,
                                            const float* s_gh, float* s_part,
                                            unsigned* s_items, short* s_inv, int* s_hist) {
  constexpr int NT = TILE * TILE;
  constexpr int NWB = NT / 32;
  constexpr int NCR = Chan<NC>::R;
  const int n = nchan<NC>(p);
  const int np = 5 + n;
  const int nit = cnt * NWB;
  if (threadIdx.x < 36) s_hist[threadIdx.x] = 0;
  __syncthreads();
  for (int it = threadIdx.x; it < nit; it += NT) {
    const int j = it / NWB, wb = it - j * NWB;
    const int c = __popc(s_mask[wb * CH + j]);
    if (c) atomicAdd(&s_hist[32 - c], 1);  // bucket 0 holds the fullest items
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int b = 0; b < 33; ++b) {
      const int v = s_hist[b];
      s_hist[b] = run;
      run += v;
    }
    s_hist[33] = run;
  }
  __syncthreads();
  const int total = s_hist[33];
  for (int it = threadIdx.x; it < nit; it += NT) {
    const int j = it / NWB, wb = it - j * NWB;
    const int c = __popc(s_mask[wb * CH + j]);
    short pos = -1;
    if (c) {
      const int q = atomicAdd(&s_hist[32 - c], 1);
      s_items[q] = ((unsigned)j << 8) | (unsigned)wb;
      pos = (short)q;
    }
    s_inv[j * NWB + wb] = pos;
  }
  __syncthreads();

  float T[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  float Tc[NCR];
#pragma unroll
  for (int c = 0; c < NCR; ++c) Tc[c] = 0.0f;
  for (int rb = 0; rb < total; rb += NT) {
    const int it = rb + (int)threadIdx.x;
    if (it < total) {
      const unsigned code = s_items[it];
      const int j = (int)(code >> 8), wb = (int)(code & 255u);
      unsigned m = s_mask[wb * CH + j];
      const float4 a = s_a[j];
      const float a11 = s_a11[j];
      const float* col = p.color + (int64_t)s_gid[j] * n;
      float cc[NCR];
#pragma unroll
      for (int c = 0; c < NCR; ++c) cc[c] = (NC > 0 || c < n) ? col[c] : 0.0f;
      float S1 = 0.f, S2 = 0.f, S11 = 0.f, S12 = 0.f, S22 = 0.f;
      float Sc[NCR];
#pragma unroll
      for (int c = 0; c < NCR; ++c) Sc[c] = 0.0f;
      while (m) {
        const int i = wb * 32 + (__ffs(m) - 1);
        m &= m - 1;
        const float4 s0 = s_ps0[i];
        const float beta = s_ps1[i].y;
        const float dx = __fsub_rn(s0.x, a.x);
        const float dy = __fsub_rn(s0.y, a.y);
        const float h = __fmaf_rn(a.w, dy, __fmul_rn(a.z, dx));
        const float q = __fmaf_rn(h, dx, __fmul_rn(__fmul_rn(a11, dy), dy));
        const float w = exp2f((s0.w - q) * HALF_LOG2E);
        float gd = -beta;
#pragma unroll
        for (int c = 0; c < NCR; ++c)
          if (NC > 0 || c < n) gd = fmaf(s_gh[c * NT + i], cc[c], gd);
        const float Gq = w * gd;
        const float e1 = Gq * dx, e2 = Gq * dy;
        S1 += e1;
        S2 += e2;
        S11 = fmaf(e1, dx, S11);
        S12 = fmaf(e1, dy, S12);
        S22 = fmaf(e2, dy, S22);
#pragma unroll
        for (int c = 0; c < NCR; ++c)
          if (NC > 0 || c < n) Sc[c] = fmaf(w, s_gh[c * NT + i], Sc[c]);
      }
      float* dst = s_part + threadIdx.x * np;
      dst[0] = S1;
      dst[1] = S2;
      dst[2] = S11;
      dst[3] = S12;
      dst[4] = S22;
#pragma unroll
      for (int c = 0; c < NCR; ++c)
        if (NC > 0 || c < n) dst[5 + c] = Sc[c];
    }
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      const int j = threadIdx.x;
      for (int wb = 0; wb < NWB; ++wb) {
        const int pos = s_inv[j * NWB + wb];
        if (pos >= rb && pos < rb + NT) {
          const float* src = s_part + (pos - rb) * np;
#pragma unroll
          for (int k = 0; k < 5; ++k) T[k] += src[k];
#pragma unroll
          for (int c = 0; c < NCR; ++c)
            if (NC > 0 || c < n) Tc[c] += src[5 + c];
        }
      }
    }
    __syncthreads();
  }
  if ((int)threadIdx.x < cnt) {
    const int gid = s_gid[threadIdx.x];
    bool any = false;
    for (int wb = 0; wb < NWB; ++wb) any |= s_inv[threadIdx.x * NWB + wb] >= 0;
    if (any && (unsigned)gid < (unsigned)p.N) {
      const GRec rc = p.rec[gid];
      const float2 cs = p.trig[gid];
      const float A00 = rc.a.z, B = rc.a.w, A11 = rc.b.x, t1 = rc.b.z, t2 = rc.b.w;
      const float T1 = t1 * t1, T2 = t2 * t2;
      const float c2 = cs.x * cs.x, s2 = cs.y * cs.y, sc = cs.x * cs.y;
      const float d_mx = -(2.0f * A00 * T[0] + B * T[1]);
      const float d_my = -(B * T[0] + 2.0f * A11 * T[1]);
      const float dT1 = T[2] * c2 + T[4] * s2 + 2.0f * T[3] * sc;
      const float dT2 = T[2] * s2 + T[4] * c2 - 2.0f * T[3] * sc;
      const float d_th = (T1 - T2) * (2.0f * sc * (T[4] - T[2]) + 2.0f * (c2 - s2) * T[3]);
      float* gdst = p.grad + (int64_t)gid * np;
      atomicAdd(gdst + 0, d_mx * (float)t.W);
      atomicAdd(gdst + 1, d_my * (float)t.H);
      atomicAdd(gdst + 2, d_th);
      atomicAdd(gdst + 3, 2.0f * t1 * dT1);
      atomicAdd(gdst + 4, 2.0f * t2 * dT2);
#pragma unroll
      for (int c = 0; c < NCR; ++c)
        if (NC > 0 || c < n) atomicAdd(gdst + 5 + c, -2.0f * Tc[c]);
    }
  }
}

// Adjoint of one tile: passes A and B per pixel, then pass C per candidate.
template <int TILE, int K, int NC, int CH>
__device__ __forceinline__ void bwd_tile(const RenderParams& p, const TileCtx& t, float* smem) {
  constexpr int NT = TILE * TILE;
  constexpr int NCR = Chan<NC>::R;
  const int n = nchan<NC>(p);
  constexpr int NWB = NT / 32;
  const BwdSmem SL = bwd_smem(NT, n, CH);
  float4* s_a = reinterpret_cast<float4*>(smem + SL.a);
  float* s_a11 = smem + SL.a11;
  int* s_gid = reinterpret_cast<int*>(smem + SL.gid);
  float4* s_ps0 = reinterpret_cast<float4*>(smem + SL.ps0);
  float2* s_ps1 = reinterpret_cast<float2*>(smem + SL.ps1);
  float* s_gh = smem + SL.gh;
  float* s_part = smem + SL.part;
  double* s_loss = reinterpret_cast<double*>(smem + SL.loss);
  float* s_key = smem + SL.key;
  short* s_ord = reinterpret_cast<short*>(smem + SL.ord);
  unsigned* s_mask = reinterpret_cast<unsigned*>(smem + SL.mask);
  unsigned* s_items = reinterpret_cast<unsigned*>(smem + SL.items);
  short* s_inv = reinterpret_cast<short*>(smem + SL.inv);
  int* s_hist = reinterpret_cast<int*>(smem + SL.hist);

  const int2 lp = pixel_of<TILE>(threadIdx.x);
  const int x = t.x0 + lp.x, y = t.y0 + lp.y;
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const int2 range = t.range;

  // ---- passes A and B: per-pixel forward values and upstream gradient
  const int len = range.y - range.x;
  const bool fast = len <= CH;
  float tq[K];
  PixelBlend<NCR> r;
  if (fast) {
    __syncthreads();  // the previous tile of a persistent CTA is done with smem
    stage_chunk<CH>(p, range.x, len, s_a, s_a11, s_gid);
    for (int i = threadIdx.x; i < NWB * CH; i += NT) s_mask[i] = 0u;
    __syncthreads();
    const int w = threadIdx.x >> 5;
    const float2 c = block_centre<TILE>(t.x0, t.y0);
    warp_order<CH>(len, c.x, c.y, s_a, s_a11, s_key + w * CH, s_ord + w * CH);
    bool tie;
    fast_keys<K>(len, px, py, s_a, s_a11, s_ord + w * CH, tq, tie);
    const bool warp_tie = __any_sync(FULL_MASK, tie);
    fast_blend<K, NC, true>(p, len, px, py, x < t.W && y < t.H, tq, warp_tie, s_a, s_a11, s_gid,
                            s_ord + w * CH, s_mask + w * CH, r);
  } else {
    select_keys<TILE, K, CH>(p, range, px, py, tq, s_a, s_a11, s_gid);
    blend_pass<TILE, K, NC, CH>(p, range, px, py, tq, r, s_a, s_a11, s_gid);
  }

  float loss = 0.0f;
  const bool live = x < t.W && y < t.H && r.Z > 0.0f;
  float beta = 0.0f;
  const float iz = live ? 1.0f / r.Z : 0.0f;
  const int64_t plane = (int64_t)t.H * t.W;
  const int64_t o = t.off + (int64_t)y * t.W + x;
#pragma unroll
  for (int c = 0; c < NCR; ++c) {
    if (NC > 0 || c < n) {
      float g = 0.0f;
      if (live) {
        if (p.grad_img) {
          g = p.grad_img[c * plane + o];
        } else {
          const float d = r.cr[c] - p.target[c * plane + o];
          loss += fabsf(d);
          g = sign_f(d) * t.inv_count;
        }
      }
      const float gh = -0.5f * g * iz;  // dL/dq_k = w_k * (sum_c gh_c c_k,c - beta)
      beta = fmaf(gh, r.cr[c], beta);
      s_gh[c * NT + threadIdx.x] = gh;
    }
  }
  s_ps0[threadIdx.x] = make_float4(px, py, live ? r.tau : -F_INF, r.q0);
  s_ps1[threadIdx.x] = make_float2(__int_as_float(r.posK), beta);
  if (!p.grad_img) {
    const double l = warp_sum<double>((double)loss);
    if ((threadIdx.x & 31) == 0) s_loss[threadIdx.x >> 5] = l;
  }
  __syncthreads();
  if (!p.grad_img && threadIdx.x == 0) {
    double tot = 0.0;
    for (int i = 0; i < NT / 32; ++i) tot += s_loss[i];
    if (tot != 0.0) atomicAdd(t.loss_acc, tot);
  }

  // ---- pass C: candidate-major accumulation of the adjoint
  if (fast) {
    fast_pass_c<TILE, NC, CH>(p, t, len, s_a, s_a11, s_gid, s_mask, s_ps0, s_ps1, s_gh, s_part,
                              s_items, s_inv, s_hist);
    return;
  }
  const int np = 5 + n;
  for (int cbase = range.x; cbase < range.y; cbase += CH) {
    const int C = min(CH, range.y - cbase);
    const int G = max(1, NT / C);            // pixel groups per candidate
    const int PPG = (NT + G - 1) / G;        // pixels per group
    const int j = (int)threadIdx.x % C;
    const int grp = (int)threadIdx.x / C;
    float S1 = 0.f, S2 = 0.f, S11 = 0.f, S12 = 0.f, S22 = 0.f;
    float Sc[NCR];
#pragma unroll
    for (int c = 0; c < NCR; ++c) Sc[c] = 0.0f;
    const int gid = p.list[cbase + j];
    const bool act = grp < G && (unsigned)gid < (unsigned)p.N;
    if (act) {
      const int pos = cbase - range.x + j;
      const GRec rc = p.rec[gid];
      const float* col = p.color + (int64_t)gid * n;
      float cc[NCR];
#pragma unroll
      for (int c = 0; c < NCR; ++c) cc[c] = (NC > 0 || c < n) ? col[c] : 0.0f;
      const int i0 = grp * PPG, i1 = min(NT, i0 + PPG);
      for (int i = i0; i < i1; ++i) {
        const float4 s0 = s_ps0[i];
        const float2 s1 = s_ps1[i];
        // the ranking key of pass A, recomputed bit for bit (same sequence)
        const float dx = __fsub_rn(s0.x, rc.a.x);
        const float dy = __fsub_rn(s0.y, rc.a.y);
        const float h = __fmaf_rn(rc.a.w, dy, __fmul_rn(rc.a.z, dx));
        const float q = __fmaf_rn(h, dx, __fmul_rn(__fmul_rn(rc.b.x, dy), dy));
        const bool win = q < s0.z || (q == s0.z && pos <= __float_as_int(s1.x));
        if (win) {
          const float w = exp2f((s0.w - q) * HALF_LOG2E);
          float gd = -s1.y;
#pragma unroll
          for (int c = 0; c < NCR; ++c)
            if (NC > 0 || c < n) gd = fmaf(s_gh[c * NT + i], cc[c], gd);
          const float Gq = w * gd;
          const float e1 = Gq * dx, e2 = Gq * dy;
          S1 += e1;
          S2 += e2;
          S11 = fmaf(e1, dx, S11);
          S12 = fmaf(e1, dy, S12);
          S22 = fmaf(e2, dy, S22);
#pragma unroll
          for (int c = 0; c < NCR; ++c)
            if (NC > 0 || c < n) Sc[c] = fmaf(w, s_gh[c * NT + i], Sc[c]);
        }
      }
    }
    if (grp < G) {
      float* dst = s_part + (grp * C + j) * np;
      dst[0] = S1;
      dst[1] = S2;
      dst[2] = S11;
      dst[3] = S12;
      dst[4] = S22;
#pragma unroll
      for (int c = 0; c < NCR; ++c)
        if (NC > 0 || c < n) dst[5 + c] = Sc[c];
    }
    __syncthreads();
    if ((int)threadIdx.x < C && (unsigned)gid < (unsigned)p.N) {
      float T[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      for (int g2 = 0; g2 < G; ++g2) {
        const float* src = s_part + (g2 * C + j) * np;
#pragma unroll
        for (int k = 0; k < 5; ++k) T[k] += src[k];
      }
      const GRec rc = p.rec[gid];
      const float2 cs = p.trig[gid];
      const float A00 = rc.a.z, B = rc.a.w, A11 = rc.b.x, t1 = rc.b.z, t2 = rc.b.w;
      const float T1 = t1 * t1, T2 = t2 * t2;
      const float c2 = cs.x * cs.x, s2 = cs.y * cs.y, sc = cs.x * cs.y;
      // q = A00 dx^2 + B dx dy + A11 dy^2, d = x - mu_px
      const float d_mx = -(2.0f * A00 * T[0] + B * T[1]);
      const float d_my = -(B * T[0] + 2.0f * A11 * T[1]);
      const float dT1 = T[2] * c2 + T[4] * s2 + 2.0f * T[3] * sc;
      const float dT2 = T[2] * s2 + T[4] * c2 - 2.0f * T[3] * sc;
      const float d_th = (T1 - T2) * (2.0f * sc * (T[4] - T[2]) + 2.0f * (c2 - s2) * T[3]);
      float* gdst = p.grad + (int64_t)gid * np;
      atomicAdd(gdst + 0, d_mx * (float)t.W);
      atomicAdd(gdst + 1, d_my * (float)t.H);
      atomicAdd(gdst + 2, d_th);
      atomicAdd(gdst + 3, 2.0f * t1 * dT1);
      atomicAdd(gdst + 4, 2.0f * t2 * dT2);
      for (int c = 0; c < n; ++c) {
        float sc_ = 0.0f;
        for (int g2 = 0; g2 < G; ++g2) sc_ += s_part[(g2 * C + j) * np + 5 + c];
        atomicAdd(gdst + 5 + c, -2.0f * sc_);  // w g / Z = w * (-2 gh)
      }
    }
    __syncthreads();
  }
}

template <int TILE, int K, int NC>
__global__ void __launch_bounds__(TILE * TILE) k_render_bwd(RenderParams p) {
  extern __shared__ __align__(16) float smem[];
  const int tile_id = blockIdx.x;
  TileCtx t;
  t.range = p.range[tile_id];
  t.x0 = (tile_id % p.tiles_x) * TILE;
  t.y0 = (tile_id / p.tiles_x) * TILE;
  t.H = p.H;
  t.W = p.W;
  t.off = 0;
  t.inv_count = p.inv_count;
  t.loss_acc = &p.status->loss_sum;
  bwd_tile<TILE, K, NC, TILE * TILE>(p, t, smem);
}

__device__ __forceinline__ int image_of_tile(const BatchTables& bt, int tile) {
  int lo = 0, hi = bt.B - 1;  // largest b with tile_off[b] <= tile
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bt.tile_off[mid] <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Persistent adjoint over the concatenated tiles of many images: each CTA
// pulls tiles until none is left (no inter-CTA waits).
template <int TILE, int K, int NC, int CH>
__global__ void __launch_bounds__(TILE * TILE) k_render_bwd_batch(RenderParams p,
                                                                  BatchTables bt) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int s_item;
  int it = blockIdx.x;
  for (;;) {
    if (bt.order == 0) {
      if (threadIdx.x == 0) s_item = (int)atomicAdd(bt.work, 1u);
      __syncthreads();
      it = s_item;
      __syncthreads();
    }
    if (it >= bt.T) break;
    const int b = image_of_tile(bt, it);
    const int4 dm = bt.dims[b];
    const int local = it - bt.tile_off[b];
    TileCtx t;
    t.range = p.range[it];
    t.x0 = (local % dm.z) * TILE;
    t.y0 = (local / dm.z) * TILE;
    t.H = dm.x;
    t.W = dm.y;
    t.off = bt.pix_off[b];
    t.inv_count = 1.0f / ((float)dm.x * (float)dm.y * (float)nchan<NC>(p));
    t.loss_acc = bt.loss + b;
    bwd_tile<TILE, K, NC, CH>(p, t, smem);
    if (bt.order != 0) it += gridDim.x;
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
    tq[k] = F_INF;
    tp[k] = -1;
  }
  for (int j = range.x; j < range.y; ++j) {
    const int id = p.list[j];
    if ((unsigned)id >= (unsigned)p.N) continue;
    const GRec g = p.rec[id];
    const float q = rank_key(px, py, g.a.x, g.a.y, g.a.z, g.a.w, g.b.x);
    if (q < tq[K - 1]) topk_insert<K>(tq, tp, q, id);
  }
  const int n = nchan<NC>(p);
  constexpr int NCR = Chan<NC>::R;
  float cr[NCR];
#pragma unroll
  for (int c = 0; c < NCR; ++c) cr[c] = 0.0f;
  float Z = 0.0f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (tp[k] >= 0) {
      const float w = exp2f((tq[0] - tq[k]) * HALF_LOG2E);
      Z += w;
      const float* col = p.color + (int64_t)tp[k] * n;
#pragma unroll
      for (int c = 0; c < NCR; ++c)
        if (NC > 0 || c < n) cr[c] = fmaf(w, col[c], cr[c]);
    }
  }
  const float iz = Z > 0.0f ? 1.0f / Z : 0.0f;
#pragma unroll
  for (int c = 0; c < NCR; ++c)
    if (NC > 0 || c < n) p.qout[qi * n + c] = cr[c] * iz;
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
