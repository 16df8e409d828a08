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

// K = 0 selects all of S_j (no top-K): arrays keep one slot.
template <int K> struct KS { static constexpr int A = K > 0 ? K : 1; };

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
// Colours of staged candidates live in shared memory, channel-major
// s_col[c * NT + j], when the channel count is a compile-time constant.
template <int NT, int NC>
__device__ __forceinline__ void stage_chunk(const RenderParams& p, int base, int cnt,
                                            float4* s_a, float* s_a11, int* s_gid,
                                            float* s_col) {
  if ((int)threadIdx.x < cnt) {
    const int gid = p.list[base + threadIdx.x];
    if ((unsigned)gid < (unsigned)p.N) {
      const GRec g = p.rec[gid];
      s_a[threadIdx.x] = g.a;
      s_a11[threadIdx.x] = g.b.x;
      s_gid[threadIdx.x] = gid;
      if (NC > 0) {
#pragma unroll
        for (int c = 0; c < (NC > 0 ? NC : 1); ++c)
          s_col[c * NT + threadIdx.x] = p.color[(int64_t)gid * NC + c];
      }
    } else {  // corrupt list entry: a NaN key is never selected
      s_a[threadIdx.x] = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
      s_a11[threadIdx.x] = 0.0f;
      s_gid[threadIdx.x] = -1;
      if (NC > 0) {
#pragma unroll
        for (int c = 0; c < (NC > 0 ? NC : 1); ++c) s_col[c * NT + threadIdx.x] = 0.0f;
      }
      atomicOr(&p.status->flags, FLAG_INTERNAL);
    }
  }
}

// Channel c of staged candidate j (shared memory if staged, else global).
template <int NT, int NC>
__device__ __forceinline__ float staged_colour(const RenderParams& p, const float* s_col,
                                               const int* s_gid, int j, int c) {
  if (NC > 0) return s_col[c * NT + j];
  return p.color[(int64_t)s_gid[j] * p.n + c];
}

// Pass A: the K smallest keys at (px, py), ascending. CH list entries are
// staged per round ("Gaussians per stage", CH <= TILE*TILE).
template <int TILE, int K, int CH>
__device__ __forceinline__ void select_keys(const RenderParams& p, int2 range, float px,
                                            float py, float (&tq)[KS<K>::A], float4* s_a,
                                            float* s_a11, int* s_gid) {
#pragma unroll
  for (int k = 0; k < KS<K>::A; ++k) tq[k] = F_INF;
  if (K == 0 && !p.normalize) return;  // every candidate wins, no shift needed
  for (int base = range.x; base < range.y; base += CH) {
    const int cnt = min(CH, range.y - base);
    __syncthreads();
    stage_chunk<CH, 0>(p, base, cnt, s_a, s_a11, s_gid, nullptr);
    __syncthreads();
#pragma unroll 4
    for (int j = 0; j < cnt; ++j) {
      const float4 a = s_a[j];
      const float q = rank_key(px, py, a.x, a.y, a.z, a.w, s_a11[j]);
      if (K == 0) {  // all of S_j: only the smallest key is needed
        tq[0] = fminf(tq[0], q);
        continue;
      }
      const bool better = q < tq[KS<K>::A - 1];
      if (__any_sync(FULL_MASK, better)) {
        float x = better ? q : F_INF;  // +inf (and NaN) insert nothing
#pragma unroll
        for (int k = 0; k < KS<K>::A; ++k) {
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
                                           float py, const float (&tq)[KS<K>::A],
                                           PixelBlend<Chan<NC>::R>& r, float4* s_a,
                                           float* s_a11, int* s_gid, float* s_col) {
  constexpr int NCR = Chan<NC>::R;
  const int n = nchan<NC>(p);
  r.q0 = p.normalize ? tq[0] : 0.0f;  // unnormalised: w = exp(-q/2) itself
  r.tau = K == 0 ? F_INF : tq[KS<K>::A - 1];
  int lt = 0;
#pragma unroll
  for (int k = 0; k < KS<K>::A; ++k) lt += tq[k] < r.tau ? 1 : 0;
  int eq_left = K - lt;  // tau-valued slots still open
  r.posK = -1;
  r.Z = 0.0f;
#pragma unroll
  for (int c = 0; c < NCR; ++c) r.cr[c] = 0.0f;
  for (int base = range.x; base < range.y; base += CH) {
    const int cnt = min(CH, range.y - base);
    __syncthreads();
    stage_chunk<CH, NC>(p, base, cnt, s_a, s_a11, s_gid, s_col);
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
          const float w = blend_weight(r.q0, q);  // exactly 1 at q = q_min
          r.Z += w;
#pragma unroll
          for (int c = 0; c < NCR; ++c)
            if (NC > 0 || c < n)
              r.cr[c] = fmaf(w, staged_colour<CH, NC>(p, s_col, s_gid, j, c), r.cr[c]);
        }
      }
    }
  }
  const float iz = p.normalize ? (r.Z > 0.0f ? 1.0f / r.Z : 0.0f) : 1.0f;
#pragma unroll
  for (int c = 0; c < NCR; ++c) r.cr[c] *= iz;
}

// ---------------------------------------------------------------------------
// Adjoint fast path for tiles whose whole list fits one stage (the common
// case): the list is staged once, passes A and B run warp-locally over it in
// list order, and pass B's ballots record, per (warp block, candidate), the
// mask of pixels where the candidate is a winner. Pass C then walks only the
// winning (candidate, pixel) pairs, split evenly over the CTA's threads.
// ---------------------------------------------------------------------------

// Pass A over the staged list (list order, keys only).
template <int K>
__device__ __forceinline__ void staged_keys(const RenderParams& p, int cnt, float px, float py,
                                            const float4* s_a, const float* s_a11,
                                            float (&tq)[KS<K>::A]) {
#pragma unroll
  for (int k = 0; k < KS<K>::A; ++k) tq[k] = F_INF;
  if (K == 0 && !p.normalize) return;
#pragma unroll 4
  for (int j = 0; j < cnt; ++j) {
    const float4 a = s_a[j];
    const float q = rank_key(px, py, a.x, a.y, a.z, a.w, s_a11[j]);
    if (K == 0) {
      tq[0] = fminf(tq[0], q);
      continue;
    }
    const bool better = q < tq[KS<K>::A - 1];
    if (__any_sync(FULL_MASK, better)) {
      float x = better ? q : F_INF;
#pragma unroll
      for (int k = 0; k < KS<K>::A; ++k) {
        const float lo = fminf(tq[k], x);
        x = fmaxf(tq[k], x);
        tq[k] = lo;
      }
    }
  }
}

// Pass B over the staged list: exact (q, index) membership, blend, and the
// ballot of winning live pixels of this warp per candidate into mask_w[].
template <int K, int NC, int CH>
__device__ __forceinline__ void staged_blend(const RenderParams& p, int cnt, float px, float py,
                                             bool live, const float (&tq)[KS<K>::A],
                                             const float4* s_a, const float* s_a11,
                                             const int* s_gid, const float* s_col,
                                             unsigned* mask_w, PixelBlend<Chan<NC>::R>& r) {
  constexpr int NCR = Chan<NC>::R;
  const int n = nchan<NC>(p);
  const int lane = threadIdx.x & 31;
  r.q0 = p.normalize ? tq[0] : 0.0f;
  r.tau = K == 0 ? F_INF : tq[KS<K>::A - 1];
  r.posK = -1;
  r.Z = 0.0f;
#pragma unroll
  for (int c = 0; c < NCR; ++c) r.cr[c] = 0.0f;
  int lt = 0;
#pragma unroll
  for (int k = 0; k < KS<K>::A; ++k) lt += tq[k] < r.tau ? 1 : 0;
  int eq_left = K - lt;
#pragma unroll 2
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
    if (lane == 0) mask_w[j] = bal;
    if (win) {
      const float w = blend_weight(r.q0, q);
      r.Z += w;
#pragma unroll
      for (int c = 0; c < NCR; ++c)
        if (NC > 0 || c < n)
          r.cr[c] = fmaf(w, staged_colour<CH, NC>(p, s_col, s_gid, j, c), r.cr[c]);
    }
  }
  const float iz = p.normalize ? (r.Z > 0.0f ? 1.0f / r.Z : 0.0f) : 1.0f;
#pragma unroll
  for (int c = 0; c < NCR; ++c) r.cr[c] *= iz;
}

template <int TILE, int K, int NC>
__global__ void __launch_bounds__(TILE * TILE) k_render_fwd(RenderParams p) {
  constexpr int NT = TILE * TILE;
  __shared__ float4 s_a[NT];
  __shared__ float s_a11[NT];
  __shared__ int s_gid[NT];
  __shared__ float s_col[NT * (NC > 0 ? NC : 1)];
  const int tile_id = blockIdx.x;
  const int tx = tile_id % p.tiles_x, ty = tile_id / p.tiles_x;
  const int2 lp = pixel_of<TILE>(threadIdx.x);
  const int x = tx * TILE + lp.x, y = ty * TILE + lp.y;
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const int2 range = p.range[tile_id];
  float tq[KS<K>::A];
  select_keys<TILE, K, NT>(p, range, px, py, tq, s_a, s_a11, s_gid);
  PixelBlend<Chan<NC>::R> r;
  blend_pass<TILE, K, NC, NT>(p, range, px, py, tq, r, s_a, s_a11, s_gid, s_col);
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
  int a, a11, gid, col, ps0, ps1, gh, part, slotj, loss, scan, start, mask, off, total;
};
__host__ __device__ inline BwdSmem bwd_smem(int NT, int n, int CH) {
  const int NWB = NT / 32;
  BwdSmem L;
  int o = 0;
  L.a = o;     o += 4 * NT;            // float4 staged geometry
  L.a11 = o;   o += NT;
  L.gid = o;   o += NT;
  L.col = o;   o += n * CH;            // staged colours, channel-major
  L.ps0 = o;   o += 4 * NT;            // float4 (px, py, tau, q0)
  L.ps1 = o;   o += 2 * NT;            // float2 (posK bits, beta)
  L.gh = o;    o += n * NT;            // per-pixel -g/(2Z), channel-major
  L.part = o;  o += 2 * (5 + n) * NT;  // pass C partial sums (two slots per thread)
  L.slotj = o; o += 2 * NT;            // candidate held by each slot
  L.loss = o;  o += 2 * (NT / 32) + 2; // doubles
  L.scan = o;  o += 34;                // integer block-scan scratch
  L.start = o; o += NT / 2;            // shorts: item where each thread's pair range starts
  L.mask = o;  o += NWB * CH;          // winner masks [warp block][candidate]
  L.off = o;   o += (NWB * CH + 2) / 2;  // shorts: pair offsets of (candidate, block) items
  L.total = o;
  return L;
}

// Converts a candidate's moment sums into parameter gradients and adds them.
// T = sum over its winning pixels of G*(dx, dy, dx^2, dx dy, dy^2) with
// G = dL/dq; Tc = sum of w * (-g/(2Z)) per channel.
template <int NC>
__device__ __forceinline__ void emit_grad(const RenderParams& p, const TileCtx& t, int gid,
                                          const float (&T)[5],
                                          const float (&Tc)[Chan<NC>::R]) {
  constexpr int NCR = Chan<NC>::R;
  const int n = nchan<NC>(p);
  const GRec rc = p.rec[gid];
  const float2 cs = p.trig[gid];
  const float A00 = rc.a.z, B = rc.a.w, A11 = rc.b.x, t1 = rc.b.z, t2 = rc.b.w;
  const float T1 = t1 * t1, T2 = t2 * t2;
  const float c2 = cs.x * cs.x, s2 = cs.y * cs.y, sc = cs.x * cs.y;
  // q = A00 dx^2 + B dx dy + A11 dy^2 with d = x - mu_px
  const float d_mx = -(2.0f * A00 * T[0] + B * T[1]);
  const float d_my = -(B * T[0] + 2.0f * A11 * T[1]);
  const float dT1 = T[2] * c2 + T[4] * s2 + 2.0f * T[3] * sc;
  const float dT2 = T[2] * s2 + T[4] * c2 - 2.0f * T[3] * sc;
  const float d_th = (T1 - T2) * (2.0f * sc * (T[4] - T[2]) + 2.0f * (c2 - s2) * T[3]);
  float* gdst = p.grad + (int64_t)gid * (5 + n);
  atomicAdd(gdst + 0, d_mx * (float)t.W);
  atomicAdd(gdst + 1, d_my * (float)t.H);
  atomicAdd(gdst + 2, d_th);
  atomicAdd(gdst + 3, 2.0f * t1 * dT1);
  atomicAdd(gdst + 4, 2.0f * t2 * dT2);
#pragma unroll
  for (int c = 0; c < NCR; ++c)
    if (NC > 0 || c < n) atomicAdd(gdst + 5 + c, -2.0f * Tc[c]);  // w g / Z
}

__device__ __forceinline__ int block_scan_int(int v, int* scratch, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(FULL_MASK, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    const int wv = lane < nw ? scratch[lane] : 0;
    int wi = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(FULL_MASK, wi, o);
      if (lane >= o) wi += u;
    }
    if (lane < nw) scratch[lane] = wi - wv;
    if (lane == nw - 1) scratch[32] = wi;
  }
  __syncthreads();
  const int r = scratch[warp] + incl - v;
  total = scratch[32];
  __syncthreads();
  return r;
}

// Pass C of the fast path. The winning (candidate, pixel) pairs, in
// (candidate, warp block, pixel) order, are split into equal contiguous
// ranges, one per thread. A thread accumulates the candidates of its range
// in registers; a candidate whose pairs all lie inside one range is finished
// by that thread, the first and last candidates of every range go to two
// slots, and each candidate's owner thread adds up the slots that hold it.
template <int TILE, int NC, int CH>
__device__ __forceinline__ void flat_pass_c(const RenderParams& p, const TileCtx& t, int cnt,
                                            const float4* s_a, const float* s_a11,
                                            const int* s_gid, const float* s_col,
                                            const unsigned* s_mask, const float4* s_ps0,
                                            const float2* s_ps1, const float* s_gh,
                                            float* s_slot, int* s_slotj, short* s_off,
                                            int* s_scan, short* s_start) {
  constexpr int NT = TILE * TILE;
  constexpr int NWB = NT / 32;
  constexpr int NCR = Chan<NC>::R;
  const int n = nchan<NC>(p);
  const int np = 5 + n;
  const int nit = cnt * NWB;
  auto mask_of = [&](int it) { return s_mask[(it % NWB) * CH + it / NWB]; };
  // exclusive offsets of the items' pair counts
  const int per_it = (nit + NT - 1) / NT;
  const int i0 = (int)threadIdx.x * per_it;
  int loc = 0;
  for (int k = 0; k < per_it; ++k)
    if (i0 + k < nit) loc += __popc(mask_of(i0 + k));
  int P;
  int run = block_scan_int(loc, s_scan, P);
  const int per = (P + NT - 1) / NT;  // pairs per thread
  for (int k = 0; k < per_it; ++k)
    if (i0 + k < nit) {
      const int c = __popc(mask_of(i0 + k));
      s_off[i0 + k] = (short)run;
      // the threads whose range starts inside this item begin here
      for (int th = (run + per - 1) / max(per, 1); per > 0 && th * per < run + c; ++th)
        s_start[th] = i0 + k;
      run += c;
    }
  if (threadIdx.x == 0) s_off[nit] = (short)P;  // P <= pixels * K <= 4096
  s_slotj[2 * threadIdx.x] = -1;
  s_slotj[2 * threadIdx.x + 1] = -1;
  __syncthreads();

  const int r0 = (int)threadIdx.x * per;
  const int r1 = min(P, r0 + per);
  if (r0 < r1) {
    int it = s_start[threadIdx.x];
    const int j_first = it / NWB;
    unsigned m = mask_of(it);
    for (int k = r0 - s_off[it]; k > 0; --k) m &= m - 1;
    int j = j_first, wb = it - j * NWB;
    float4 a = s_a[j];
    float a11 = s_a11[j];
    float cc[NCR];
    auto load_colour = [&](int jj) {
#pragma unroll
      for (int c = 0; c < NCR; ++c)
        cc[c] = (NC > 0 || c < n) ? staged_colour<CH, NC>(p, s_col, s_gid, jj, c) : 0.0f;
    };
    load_colour(j);
    float T[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    float Tc[NCR];
#pragma unroll
    for (int c = 0; c < NCR; ++c) Tc[c] = 0.0f;
    // A candidate of a thread's range gets a slot if the range may not hold
    // all of its pairs: the first one, and the one open when the range ends.
    auto flush = [&](int jj, bool at_end) {
      if (jj == j_first || at_end) {
        const int slot = 2 * (int)threadIdx.x + (jj == j_first ? 0 : 1);
        float* dst = s_slot + slot * np;
#pragma unroll
        for (int k = 0; k < 5; ++k) dst[k] = T[k];
#pragma unroll
        for (int c = 0; c < NCR; ++c)
          if (NC > 0 || c < n) dst[5 + c] = Tc[c];
        s_slotj[slot] = jj;
      } else {
        const int gid = s_gid[jj];
        if ((unsigned)gid < (unsigned)p.N) emit_grad<NC>(p, t, gid, T, Tc);
      }
#pragma unroll
      for (int k = 0; k < 5; ++k) T[k] = 0.0f;
#pragma unroll
      for (int c = 0; c < NCR; ++c) Tc[c] = 0.0f;
    };
    for (int e = r0; e < r1; ++e) {
      const int i = wb * 32 + (__ffs(m) - 1);
      m &= m - 1;
      const float4 s0 = s_ps0[i];
      const float beta = s_ps1[i].y;
      // the ranking key of pass A, recomputed bit for bit (same sequence)
      const float dx = __fsub_rn(s0.x, a.x);
      const float dy = __fsub_rn(s0.y, a.y);
      const float h = __fmaf_rn(a.w, dy, __fmul_rn(a.z, dx));
      const float q = __fmaf_rn(h, dx, __fmul_rn(__fmul_rn(a11, dy), dy));
      const float w = blend_weight(s0.w, q);
      float gd = -beta;
#pragma unroll
      for (int c = 0; c < NCR; ++c)
        if (NC > 0 || c < n) gd = fmaf(s_gh[c * NT + i], cc[c], gd);
      const float Gq = w * gd;
      const float e1 = Gq * dx, e2 = Gq * dy;
      T[0] += e1;
      T[1] += e2;
      T[2] = fmaf(e1, dx, T[2]);
      T[3] = fmaf(e1, dy, T[3]);
      T[4] = fmaf(e2, dy, T[4]);
#pragma unroll
      for (int c = 0; c < NCR; ++c)
        if (NC > 0 || c < n) Tc[c] = fmaf(w, s_gh[c * NT + i], Tc[c]);
      if (m == 0 && e + 1 < r1) {
        do {
          ++it;
          m = mask_of(it);
        } while (m == 0);
        const int nj = it / NWB;
        wb = it - nj * NWB;
        if (nj != j) {
          flush(j, false);
          j = nj;
          a = s_a[j];
          a11 = s_a11[j];
          load_colour(j);
        }
      }
    }
    flush(j, true);
  }
  __syncthreads();
  if ((int)threadIdx.x < cnt) {
    const int j = threadIdx.x;
    const int e0 = s_off[j * NWB], e1 = s_off[(j + 1) * NWB];
    if (e1 > e0) {
      float T[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
      float Tc[NCR];
#pragma unroll
      for (int c = 0; c < NCR; ++c) Tc[c] = 0.0f;
      bool held = false;
      for (int th = e0 / per; th <= (e1 - 1) / per; ++th) {
        for (int sl = 0; sl < 2; ++sl) {
          if (s_slotj[2 * th + sl] != j) continue;
          held = true;
          const float* src = s_slot + (2 * th + sl) * np;
#pragma unroll
          for (int k = 0; k < 5; ++k) T[k] += src[k];
#pragma unroll
          for (int c = 0; c < NCR; ++c)
            if (NC > 0 || c < n) Tc[c] += src[5 + c];
        }
      }
      const int gid = s_gid[j];
      if (held && (unsigned)gid < (unsigned)p.N) emit_grad<NC>(p, t, gid, T, Tc);
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
  float* s_col = smem + SL.col;
  float4* s_ps0 = reinterpret_cast<float4*>(smem + SL.ps0);
  float2* s_ps1 = reinterpret_cast<float2*>(smem + SL.ps1);
  float* s_gh = smem + SL.gh;
  float* s_part = smem + SL.part;
  double* s_loss = reinterpret_cast<double*>(smem + SL.loss);
  unsigned* s_mask = reinterpret_cast<unsigned*>(smem + SL.mask);
  short* s_off = reinterpret_cast<short*>(smem + SL.off);
  int* s_slotj = reinterpret_cast<int*>(smem + SL.slotj);

  const int2 lp = pixel_of<TILE>(threadIdx.x);
  const int x = t.x0 + lp.x, y = t.y0 + lp.y;
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const int2 range = t.range;

  // ---- passes A and B: per-pixel forward values and upstream gradient
  const int len = range.y - range.x;
  const bool fast = len <= CH;
  float tq[KS<K>::A];
  PixelBlend<NCR> r;
  if (fast) {
    __syncthreads();  // the previous tile of a persistent CTA is done with smem
    stage_chunk<CH, NC>(p, range.x, len, s_a, s_a11, s_gid, s_col);
    __syncthreads();
    const int w = threadIdx.x >> 5;
    staged_keys<K>(p, len, px, py, s_a, s_a11, tq);
    staged_blend<K, NC, CH>(p, len, px, py, x < t.W && y < t.H, tq, s_a, s_a11, s_gid, s_col,
                            s_mask + w * CH, r);
  } else {
    select_keys<TILE, K, CH>(p, range, px, py, tq, s_a, s_a11, s_gid);
    blend_pass<TILE, K, NC, CH>(p, range, px, py, tq, r, s_a, s_a11, s_gid, s_col);
  }

  float loss = 0.0f;
  const bool live = x < t.W && y < t.H && r.Z > 0.0f;
  float beta = 0.0f;
  const float iz = live ? (p.normalize ? 1.0f / r.Z : 1.0f) : 0.0f;
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
      if (p.normalize) beta = fmaf(gh, r.cr[c], beta);
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
    flat_pass_c<TILE, NC, CH>(p, t, len, s_a, s_a11, s_gid, s_col, s_mask, s_ps0, s_ps1, s_gh,
                              s_part,
                              s_slotj, s_off, reinterpret_cast<int*>(smem + SL.scan),
                              reinterpret_cast<short*>(smem + SL.start));
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
          const float w = blend_weight(s0.w, q);
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
  bwd_tile<TILE, K, NC, TILE * TILE / 2>(p, t, smem);  // 128 Gaussians per stage at 16x16
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
  const int n = nchan<NC>(p);
  constexpr int NCR = Chan<NC>::R;
  float cr[NCR];
#pragma unroll
  for (int c = 0; c < NCR; ++c) cr[c] = 0.0f;
  float Z = 0.0f;
  if (K == 0) {  // all of S_j
    float q0 = 0.0f;
    if (p.normalize) {
      q0 = F_INF;
      for (int j = range.x; j < range.y; ++j) {
        const int id = p.list[j];
        if ((unsigned)id >= (unsigned)p.N) continue;
        const GRec g = p.rec[id];
        q0 = fminf(q0, rank_key(px, py, g.a.x, g.a.y, g.a.z, g.a.w, g.b.x));
      }
    }
    for (int j = range.x; j < range.y; ++j) {
      const int id = p.list[j];
      if ((unsigned)id >= (unsigned)p.N) continue;
      const GRec g = p.rec[id];
      const float w = blend_weight(q0, rank_key(px, py, g.a.x, g.a.y, g.a.z, g.a.w, g.b.x));
      Z += w;
      const float* col = p.color + (int64_t)id * n;
#pragma unroll
      for (int c = 0; c < NCR; ++c)
        if (NC > 0 || c < n) cr[c] = fmaf(w, col[c], cr[c]);
    }
  } else {
    float tq[KS<K>::A];
    int tp[KS<K>::A];
#pragma unroll
    for (int k = 0; k < KS<K>::A; ++k) {
      tq[k] = F_INF;
      tp[k] = -1;
    }
    for (int j = range.x; j < range.y; ++j) {
      const int id = p.list[j];
      if ((unsigned)id >= (unsigned)p.N) continue;
      const GRec g = p.rec[id];
      const float q = rank_key(px, py, g.a.x, g.a.y, g.a.z, g.a.w, g.b.x);
      if (q < tq[KS<K>::A - 1]) topk_insert<KS<K>::A>(tq, tp, q, id);
    }
    const float q0 = p.normalize ? tq[0] : 0.0f;
#pragma unroll
    for (int k = 0; k < KS<K>::A; ++k) {
      if (tp[k] >= 0) {
        const float w = blend_weight(q0, tq[k]);
        Z += w;
        const float* col = p.color + (int64_t)tp[k] * n;
#pragma unroll
        for (int c = 0; c < NCR; ++c)
          if (NC > 0 || c < n) cr[c] = fmaf(w, col[c], cr[c]);
      }
    }
  }
  const float iz = p.normalize ? (Z > 0.0f ? 1.0f / Z : 0.0f) : 1.0f;
#pragma unroll
  for (int c = 0; c < NCR; ++c)
    if (NC > 0 || c < n) p.qout[qi * n + c] = cr[c] * iz;
}

// Dispatch over the supported K and channel counts.
#define IGS_FOR_K(M, ...)                          \
  switch (K) {                                     \
    case 0: M(0, __VA_ARGS__); break;              \
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
  return K == 0 || K == 1 || K == 2 || K == 3 || K == 4 || K == 8 || K == 10 || K == 16;
}

}  // namespace igs
