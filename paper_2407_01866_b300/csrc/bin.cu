// Per-Gaussian preprocessing and tile binning (Sec. 3.2: 3-sigma enclosing
// circles, tile-circle intersection, per-tile sets S_j).
//
// Pipeline (all stream-ordered, no host synchronisation, graph-capturable):
//   k_preprocess   one thread per Gaussian: mu in pixels, inverse covariance
//                  (Eq. 2), radius 3*max(s); every exact tile hit increments
//                  that tile's counter
//   scan           exclusive prefix sum of the tile counters -> list offsets, M
//                  (for one image its last pass also writes the tile ranges
//                  and the evaluation count)
//   k_emit         every hit takes a slot of its tile's segment (atomic cursor)
//   k_wide_tiles   Gaussians whose tile box exceeds 64 tiles (one image):
//                  counted and emitted tile-major by 8 x 8 tile blocks
//                  (k_wide, one CTA per such Gaussian, for a batch)
//   k_segsort_long a CTA sorts each tile's segment by Gaussian index when it
//                  is longer than the renderer's one-stage list (longer lists
//                  are streamed in index order, which is the tie-break order
//                  of the top-K ranking; shorter ones are ranked by the
//                  renderer itself)
//   k_ranges       [start, end) of every tile from the offsets, and the sum
//                  over tiles of |S_j| * pixels(j)
#include <algorithm>

#include "internal.h"

namespace igs {

namespace {

__device__ __forceinline__ void tile_span(float m, float r, int tile, int tiles, int& lo,
                                          int& hi) {
  // One tile of margin each side: membership itself is decided by the exact
  // circle-rectangle test, the span only has to contain every hit tile.
  const float inv = 1.0f / (float)tile;  // tile is a power of two: exact
  float a = floorf((m - r) * inv) - 1.0f;
  float b = floorf((m + r) * inv) + 1.0f;
  a = fminf(fmaxf(a, 0.0f), (float)(tiles - 1));
  b = fminf(fmaxf(b, -1.0f), (float)(tiles - 1));
  lo = (int)a;
  hi = (int)b;
}

// A Gaussian whose tile box has more tiles than this is binned by a whole CTA
// (threads stride over the box) instead of one thread.
constexpr int WIDE_TILES = 64;
// CTAs of the wide-Gaussian passes (they stride over the wide Gaussians)
constexpr int WIDE_GRID = 148 * 16;

// Image geometry of Gaussian i: the single image, or its image in a batch.
struct ImgGeo {
  int H, W, tiles_x, tiles_y, tile_base;
};
template <bool BATCH>
__device__ __forceinline__ ImgGeo image_geo(const PrepParams& p, int64_t i) {
  if (!BATCH) return ImgGeo{p.H, p.W, p.tiles_x, p.tiles_y, 0};
  const int b = p.img_of[i];
  const int4 d = p.img_dims[b];
  return ImgGeo{d.x, d.y, d.z, d.w, p.tile_off[b]};
}

template <typename T, bool BATCH>
__global__ void __launch_bounds__(256) k_preprocess(PrepParams p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.N) return;
  const ImgGeo ig = image_geo<BATCH>(p, i);
  const T* xy = static_cast<const T*>(p.xy) + i * p.xy_stride;
  const T* ts = static_cast<const T*>(p.inv_scale) + i * p.inv_scale_stride;
  const T* cp = static_cast<const T*>(p.color) + i * p.color_stride;
  const float mux = to_f32(xy[0]), muy = to_f32(xy[1]);
  const float th = to_f32(static_cast<const T*>(p.theta)[i * p.theta_stride]);
  const float t1 = to_f32(ts[0]), t2 = to_f32(ts[1]);
  bool ok = isfinite(mux) && isfinite(muy) && isfinite(th) && isfinite(t1) && isfinite(t2) &&
            t1 > 0.0f && t2 > 0.0f;
  bool cok = true;
  for (int c = 0; c < p.n; ++c) {
    const float v = to_f32(cp[c]);
    cok = cok && isfinite(v);
    p.color_out[i * p.n + c] = v;
  }
  if (!(ok && cok)) atomicOr(&p.status->flags, FLAG_NONFINITE);

  const float mx = __fmul_rn(mux, (float)ig.W);
  const float my = __fmul_rn(muy, (float)ig.H);
  double sd, cd;
  sincos((double)th, &sd, &cd);
  const float c = __double2float_rn(cd), s = __double2float_rn(sd);
  float A00, B, A11;
  conic_from(c, s, t1, t2, A00, B, A11);
  float r = __fdiv_rn(3.0f, fminf(t1, t2));
  if (ok && isfinite(mx) && isfinite(my) && isfinite(r)) {
    int x0, x1, y0, y1;
    tile_span(mx, r, p.tile, ig.tiles_x, x0, x1);
    tile_span(my, r, p.tile, ig.tiles_y, y0, y1);
    const float r2 = __fmul_rn(r, r);
    if ((x1 - x0 + 1) * (y1 - y0 + 1) > WIDE_TILES) {
      const unsigned slot = atomicAdd(&p.status->wide_cnt, 1u);
      p.wide[slot] = (int)i;
      p.wide_geo[slot] = make_float4(mx, my, r, __int_as_float((int)i));
      y1 = y0 - 1;  // counted by k_count_wide
    }
    for (int ty = y0; ty <= y1; ++ty) {
      const float Y0 = (float)(ty * p.tile), Y1 = (float)min((ty + 1) * p.tile, ig.H);
      for (int tx = x0; tx <= x1; ++tx) {
        const float X0 = (float)(tx * p.tile), X1 = (float)min((tx + 1) * p.tile, ig.W);
        if (circle_hits_rect(mx, my, r2, X0, X1, Y0, Y1))
          atomicAdd(p.tcnt + ig.tile_base + ty * ig.tiles_x + tx, 1u);
      }
    }
  } else {
    r = -1.0f;  // binned nowhere
  }
  GRec g;
  g.a = make_float4(mx, my, A00, B);
  g.b = make_float4(A11, r, t1, t2);
  p.rec[i] = g;
  p.trig[i] = make_float2(c, s);
  if constexpr (sizeof(T) == 2) {
    if (p.rec16) {
      HRec h;
      h.mu = (unsigned)reinterpret_cast<const unsigned short&>(xy[0]) |
             ((unsigned)reinterpret_cast<const unsigned short&>(xy[1]) << 16);
      h.A00 = A00;
      h.B = B;
      h.A11 = A11;
      p.rec16[i] = h;
      for (int ch = 0; ch < p.n; ++ch)
        p.col16[i * p.n + ch] = reinterpret_cast<const unsigned short&>(cp[ch]);
    }
  }
}

template <bool BATCH>
__global__ void __launch_bounds__(256) k_emit(PrepParams p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && p.status->m_needed > (unsigned long long)p.m_cap)
    atomicOr(&p.status->flags, FLAG_CAPACITY);
  if (i >= p.N) return;
  const ImgGeo ig = image_geo<BATCH>(p, i);
  const GRec g = p.rec[i];
  const float mx = g.a.x, my = g.a.y, r = g.b.y;
  if (!(r >= 0.0f) || !isfinite(mx) || !isfinite(my) || !isfinite(r)) return;
  int x0, x1, y0, y1;
  tile_span(mx, r, p.tile, ig.tiles_x, x0, x1);
  tile_span(my, r, p.tile, ig.tiles_y, y0, y1);
  if ((x1 - x0 + 1) * (y1 - y0 + 1) > WIDE_TILES) return;  // emitted by k_emit_wide
  const float r2 = __fmul_rn(r, r);
  const unsigned long long cap = (unsigned long long)p.m_cap;
  for (int ty = y0; ty <= y1; ++ty) {
    const float Y0 = (float)(ty * p.tile), Y1 = (float)min((ty + 1) * p.tile, ig.H);
    for (int tx = x0; tx <= x1; ++tx) {
      const float X0 = (float)(tx * p.tile), X1 = (float)min((tx + 1) * p.tile, ig.W);
      if (circle_hits_rect(mx, my, r2, X0, X1, Y0, Y1)) {
        const int t = ig.tile_base + ty * ig.tiles_x + tx;
        // the counter runs back down from the tile's count: one slot per hit
        const unsigned long long pos = p.toff[t] + (atomicSub(p.tcnt + t, 1u) - 1u);
        if (pos < cap) p.vals[pos] = (unsigned int)i;
      }
    }
  }
}

// Wide Gaussians, one CTA each (CTA cta of ncta): threads stride over the
// tile box and apply the same circle-rectangle test. COUNT: increment the
// tiles' counters; otherwise: take the tiles' slots (after the scan).
template <bool BATCH, bool COUNT>
__device__ __forceinline__ void wide_by_gaussian(const PrepParams& p, unsigned cta,
                                                 unsigned ncta) {
  const unsigned int nw = p.status->wide_cnt;
  const unsigned long long cap = (unsigned long long)p.m_cap;
  for (unsigned int wi = cta; wi < nw; wi += ncta) {
    const int i = p.wide[wi];
    const ImgGeo ig = image_geo<BATCH>(p, i);
    const GRec g = p.rec[i];
    const float mx = g.a.x, my = g.a.y, r = g.b.y;
    int x0, x1, y0, y1;
    tile_span(mx, r, p.tile, ig.tiles_x, x0, x1);
    tile_span(my, r, p.tile, ig.tiles_y, y0, y1);
    const float r2 = __fmul_rn(r, r);
    const int bw = x1 - x0 + 1;
    const int area = bw * (y1 - y0 + 1);
    for (int k = threadIdx.x; k < area; k += blockDim.x) {
      const int ty = y0 + k / bw, tx = x0 + k % bw;
      const float Y0 = (float)(ty * p.tile), Y1 = (float)min((ty + 1) * p.tile, ig.H);
      const float X0 = (float)(tx * p.tile), X1 = (float)min((tx + 1) * p.tile, ig.W);
      if (!circle_hits_rect(mx, my, r2, X0, X1, Y0, Y1)) continue;
      const int t = ig.tile_base + ty * ig.tiles_x + tx;
      if (COUNT) {
        atomicAdd(p.tcnt + t, 1u);
      } else {
        const unsigned long long pos = p.toff[t] + (atomicSub(p.tcnt + t, 1u) - 1u);
        if (pos < cap) p.vals[pos] = (unsigned int)i;
      }
    }
  }
}

template <bool BATCH, bool COUNT>
__global__ void __launch_bounds__(256) k_wide(PrepParams p) {
  wide_by_gaussian<BATCH, COUNT>(p, blockIdx.x, gridDim.x);
}

constexpr int WT_BLOCK = 8;              // tiles per side of k_wide_tiles' tile block
constexpr int WT_CHUNK = 256;            // wide Gaussians filtered per round
constexpr unsigned WT_MAX_WIDE = 1u << 14;  // beyond this, one CTA per wide Gaussian

// Wide Gaussians of one image, tile-major: each CTA owns a block of 8 x 8
// tiles, keeps the wide Gaussians whose circle meets the block's rectangle
// (a circle that meets a tile meets the block that holds it) and tests them
// against each of its tiles with the same circle-rectangle test, 4 threads
// per tile. No tile counter is shared with another CTA. COUNT adds each
// tile's hits to its counter (after k_preprocess's narrow hits); otherwise
// the hits take the first slots of the tile's segment from on-chip counters
// (k_emit fills the segment down from its top, so the two never meet). With
// more than WT_MAX_WIDE wide Gaussians, where testing every block against
// every Gaussian would cost more than their hits, the CTAs take one Gaussian
// each (k_wide's scheme).
template <bool COUNT>
__global__ void __launch_bounds__(256) k_wide_tiles(PrepParams p) {
  const unsigned nw = p.status->wide_cnt;
  if (nw == 0) return;
  if (nw > WT_MAX_WIDE) {
    wide_by_gaussian<false, COUNT>(p, blockIdx.x, gridDim.x);
    return;
  }
  const int bxs = (p.tiles_x + WT_BLOCK - 1) / WT_BLOCK;
  const int bys = (p.tiles_y + WT_BLOCK - 1) / WT_BLOCK;
  if ((int)blockIdx.x >= bxs * bys) return;  // the grid also serves the other scheme
  const int bx = (int)blockIdx.x % bxs, by = (int)blockIdx.x / bxs;
  __shared__ float4 s_g[WT_CHUNK];  // (mx, my, r^2, index bits) meeting the block
  __shared__ int s_n;
  __shared__ int s_slot[WT_BLOCK * WT_BLOCK];
  const int tid = threadIdx.x;
  const int tl = tid >> 2, q = tid & 3;  // tile of the block, thread within the tile
  const int tx = bx * WT_BLOCK + (tl % WT_BLOCK);
  const int ty = by * WT_BLOCK + (tl / WT_BLOCK);
  const bool tile_ok = tx < p.tiles_x && ty < p.tiles_y;
  const float X0 = (float)(tx * p.tile), X1 = (float)min((tx + 1) * p.tile, p.W);
  const float Y0 = (float)(ty * p.tile), Y1 = (float)min((ty + 1) * p.tile, p.H);
  const int bx0 = bx * WT_BLOCK * p.tile, by0 = by * WT_BLOCK * p.tile;
  const float BX0 = (float)bx0, BX1 = (float)min(bx0 + WT_BLOCK * p.tile, p.W);
  const float BY0 = (float)by0, BY1 = (float)min(by0 + WT_BLOCK * p.tile, p.H);
  const int t = ty * p.tiles_x + tx;
  const unsigned long long cap = (unsigned long long)p.m_cap;
  const unsigned long long seg = COUNT || !tile_ok ? 0ull : p.toff[t];
  if (tid < WT_BLOCK * WT_BLOCK) s_slot[tid] = 0;
  int hits = 0;
  float4 nxt = (unsigned)tid < nw ? p.wide_geo[tid] : make_float4(0.f, 0.f, -1.f, 0.f);
  for (unsigned base = 0; base < nw; base += WT_CHUNK) {
    __syncthreads();  // the previous round is done with s_g
    if (tid == 0) s_n = 0;
    __syncthreads();
    const float4 g = nxt;  // (mx, my, r, index bits) of wide Gaussian base + tid
    if (base + tid < nw) {
      const float r2 = __fmul_rn(g.z, g.z);
      if (circle_hits_rect(g.x, g.y, r2, BX0, BX1, BY0, BY1))
        s_g[atomicAdd(&s_n, 1)] = make_float4(g.x, g.y, r2, g.w);
    }
    // the next round's record, in flight during this round's tests
    if (base + WT_CHUNK + tid < nw) nxt = p.wide_geo[base + WT_CHUNK + tid];
    __syncthreads();
    const int n = s_n;
    if (!tile_ok) continue;
    for (int k = q; k < n; k += 4) {
      const float4 c = s_g[k];
      if (!circle_hits_rect(c.x, c.y, c.z, X0, X1, Y0, Y1)) continue;
      if (COUNT) {
        ++hits;
      } else {
        const unsigned long long pos = seg + (unsigned)atomicAdd(&s_slot[tl], 1);
        if (pos < cap) p.vals[pos] = (unsigned int)__float_as_int(c.w);
      }
    }
  }
  if (COUNT) {
    hits += __shfl_down_sync(FULL_MASK, hits, 2, 4);
    hits += __shfl_down_sync(FULL_MASK, hits, 1, 4);
    if (q == 0 && tile_ok && hits) p.tcnt[t] += (unsigned)hits;
  }
}

// ---------------------------------------------------------------- scan

template <typename Out>
__device__ __forceinline__ Out block_exclusive_scan(Out v, Out* s_warp, Out& block_total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Out incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const Out t = __shfl_up_sync(FULL_MASK, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    Out w = lane < nw ? s_warp[lane] : Out(0);
    Out wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const Out t = __shfl_up_sync(FULL_MASK, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < nw) s_warp[lane] = wi - w;
    if (lane == nw - 1) s_warp[32] = wi;
  }
  __syncthreads();
  const Out res = s_warp[warp] + incl - v;
  block_total = s_warp[32];
  __syncthreads();
  return res;
}

template <typename In, typename Out>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const In* in, int64_t n,
                                                              unsigned long long* part) {
  __shared__ unsigned long long s_warp[33];
  const int64_t base = (int64_t)blockIdx.x * SCAN_ITEMS;
  unsigned long long sum = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    const int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
    if (i < n) sum += (unsigned long long)in[i];
  }
  unsigned long long tot;
  block_exclusive_scan<unsigned long long>(sum, s_warp, tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_partials(unsigned long long* part, int64_t nb,
                                                        unsigned long long* total) {
  __shared__ unsigned long long s_warp[33];
  unsigned long long carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
    const int64_t b = b0 + threadIdx.x;
    const unsigned long long v = b < nb ? part[b] : 0ull;
    unsigned long long tot;
    const unsigned long long ex = block_exclusive_scan<unsigned long long>(v, s_warp, tot);
    if (b < nb) part[b] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

template <typename In, typename Out>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const In* in, Out* out, int64_t n,
                                                            const unsigned long long* part) {
  __shared__ unsigned long long s_warp[33];
  const int64_t base = (int64_t)blockIdx.x * SCAN_ITEMS + (int64_t)threadIdx.x * SCAN_PER_THREAD;
  unsigned long long v[SCAN_PER_THREAD];
  unsigned long long sum = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    const int64_t i = base + k;
    v[k] = i < n ? (unsigned long long)in[i] : 0ull;
    sum += v[k];
  }
  unsigned long long tot;
  unsigned long long run = block_exclusive_scan<unsigned long long>(sum, s_warp, tot) +
                           part[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    const int64_t i = base + k;
    if (i < n) out[i] = (Out)run;
    run += v[k];
  }
}

// Last pass of the tile-count scan of one image: the list offsets, and with
// them each tile's [start, end) clipped to the stored intersections and the
// evaluation count sum_j |S_j| * pixels(j) (k_ranges and k_tile_evals folded
// in). M comes from the partials pass (status->m_needed).
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down_tiles(
    const unsigned int* in, unsigned long long* out, int64_t n, const unsigned long long* part,
    int2* range, int64_t m_cap, int H, int W, int tile, int tiles_x, DevStatus* st) {
  __shared__ unsigned long long s_warp[33];
  const int64_t base = (int64_t)blockIdx.x * SCAN_ITEMS + (int64_t)threadIdx.x * SCAN_PER_THREAD;
  unsigned int v[SCAN_PER_THREAD];
  unsigned long long sum = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    const int64_t i = base + k;
    v[k] = i < n ? in[i] : 0u;
    sum += v[k];
  }
  unsigned long long tot;
  unsigned long long run = block_exclusive_scan<unsigned long long>(sum, s_warp, tot) +
                           part[blockIdx.x];
  const unsigned long long M = st->m_needed;
  const unsigned long long live = M < (unsigned long long)m_cap ? M : (unsigned long long)m_cap;
  unsigned long long evals = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    const int64_t i = base + k;
    if (i < n) {
      out[i] = run;
      const unsigned long long a = run < live ? run : live;
      const unsigned long long b = run + v[k] < live ? run + v[k] : live;
      range[i] = make_int2((int)a, (int)b);
      const int tx = (int)(i % tiles_x), ty = (int)(i / tiles_x);
      const int w = min((tx + 1) * tile, W) - tx * tile;
      const int h = min((ty + 1) * tile, H) - ty * tile;
      evals += (unsigned long long)v[k] * (unsigned long long)(w * h);
    }
    run += v[k];
  }
  unsigned long long etot;
  block_exclusive_scan<unsigned long long>(evals, s_warp, etot);
  if (threadIdx.x == 0 && etot) atomicAdd(&st->evals, etot);
}

template <typename In, typename Out>
cudaError_t scan_exclusive(const In* in, Out* out, int64_t n, unsigned long long* part,
                           unsigned long long* total, cudaStream_t s) {
  const int64_t nb = (n + SCAN_ITEMS - 1) / SCAN_ITEMS;
  if (nb == 0) {
    if (total) return cudaMemsetAsync(total, 0, sizeof(*total), s);
    return cudaSuccess;
  }
  k_scan_reduce<In, Out><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, part);
  k_scan_partials<<<1, 1024, 0, s>>>(part, nb, total);
  k_scan_down<In, Out><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, part);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- segment sort

__device__ __forceinline__ int64_t live_items(const DevStatus* st, int64_t m_cap) {
  const unsigned long long m = st->m_needed;
  return m < (unsigned long long)m_cap ? (int64_t)m : m_cap;
}

// [a, b) of tile t in the list, clipped to the stored intersections.
__device__ __forceinline__ void tile_segment(const unsigned long long* toff, int t, int T,
                                             const DevStatus* st, int64_t m_cap, int64_t& a,
                                             int64_t& b) {
  const int64_t M = live_items(st, m_cap);
  a = (int64_t)toff[t];
  b = t + 1 < T ? (int64_t)toff[t + 1] : (int64_t)st->m_needed;
  a = a < M ? a : M;
  b = b < M ? b : M;
}

constexpr int SEG_BIG_CHUNK = 4096; // run length a CTA sorts in shared memory

// Ascending sort of tile t's segment by the calling CTA: runs of up to
// SEG_BIG_CHUNK sorted in shared memory (a rank sort up to 512 entries, a
// bitonic network over the run rounded up to a power of two beyond), then
// pairwise merges between vals and tmp, each element placed by its rank (its
// index in its own run plus a binary search in the other run; indices are
// distinct, so the ranks are a permutation).
__device__ void sort_segment_cta(unsigned int* vals, unsigned int* tmp,
                                 const unsigned long long* toff, int t, int T,
                                 const DevStatus* st, int64_t m_cap, unsigned int* sh) {
  int64_t a, b;
  tile_segment(toff, t, T, st, m_cap, a, b);
  const int L = (int)(b - a);
  for (int c0 = 0; c0 < L; c0 += SEG_BIG_CHUNK) {
    const int n = min(SEG_BIG_CHUNK, L - c0);
    if (n <= 2 * 256) {
      // rank sort, two entries per thread: an entry's place is the number
      // of smaller entries (equal ones, only in a corrupt list, by position)
      __syncthreads();
      const int i0 = threadIdx.x, i1 = threadIdx.x + 256;
      const unsigned int v0 = i0 < n ? vals[a + c0 + i0] : 0u;
      const unsigned int v1 = i1 < n ? vals[a + c0 + i1] : 0u;
      if (i0 < n) sh[i0] = v0;
      if (i1 < n) sh[i1] = v1;
      __syncthreads();
      int r0 = 0, r1 = 0;
      for (int j = 0; j < n; ++j) {
        const unsigned int x = sh[j];
        r0 += (x < v0 || (x == v0 && j < i0)) ? 1 : 0;
        r1 += (x < v1 || (x == v1 && j < i1)) ? 1 : 0;
      }
      if (i0 < n) vals[a + c0 + r0] = v0;
      if (i1 < n) vals[a + c0 + r1] = v1;
      continue;
    }
    int P = 64;  // bitonic width: the chunk rounded up to a power of two
    while (P < n) P <<= 1;
    __syncthreads();
    for (int i = threadIdx.x; i < P; i += blockDim.x)
      sh[i] = i < n ? vals[a + c0 + i] : 0xffffffffu;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
          const int l = i ^ j;
          if (l > i) {
            const unsigned int x = sh[i], y = sh[l];
            if ((x > y) == ((i & k) == 0)) {
              sh[i] = y;
              sh[l] = x;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) vals[a + c0 + i] = sh[i];
  }
  __syncthreads();
  unsigned int* src = vals + a;
  unsigned int* dst = tmp + a;
  for (int run = SEG_BIG_CHUNK; run < L; run <<= 1) {
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
      const int r0 = (i / (2 * run)) * (2 * run);
      const bool first = i - r0 < run;
      const int o0 = first ? r0 + run : r0;          // the other run
      const int o1 = first ? min(r0 + 2 * run, L) : r0 + run;
      const unsigned int v = src[i];
      int lo = o0, hi = o1;                          // elements of the other run below v
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (src[mid] < v) lo = mid + 1; else hi = mid;
      }
      const int own = first ? i - r0 : i - (r0 + run);
      dst[r0 + own + (lo - o0)] = v;
    }
    __syncthreads();
    unsigned int* x = src;
    src = dst;
    dst = x;
  }
  if (src != vals + a)
    for (int i = threadIdx.x; i < L; i += blockDim.x) vals[a + i] = src[i];
  __syncthreads();
}

// Every tile segment longer than sort_min, sorted by Gaussian index, one CTA
// per segment: each CTA looks at 32 tiles at a time (one warp reads their
// offsets), collects the long ones in shared memory and sorts them in turn.
__global__ void __launch_bounds__(256) k_segsort_long(unsigned int* vals, unsigned int* tmp,
                                                      const unsigned long long* toff, int T,
                                                      const DevStatus* st, int64_t m_cap,
                                                      int sort_min) {
  __shared__ unsigned int sh[SEG_BIG_CHUNK];
  __shared__ int s_long[32];
  __shared__ int s_n;
  for (int t0 = blockIdx.x * 32; t0 < T; t0 += gridDim.x * 32) {
    __syncthreads();  // the previous round is done with s_long
    if (threadIdx.x < 32) {
      const int t = t0 + (int)threadIdx.x;
      int64_t a = 0, b = 0;
      if (t < T) tile_segment(toff, t, T, st, m_cap, a, b);
      const int L = (int)(b - a);
      const unsigned m = __ballot_sync(FULL_MASK, t < T && L > 1 && L > sort_min);
      if (m & (1u << threadIdx.x)) s_long[__popc(m & ((1u << threadIdx.x) - 1u))] = t;
      if (threadIdx.x == 0) s_n = __popc(m);
    }
    __syncthreads();
    const int nl = s_n;
    for (int q = 0; q < nl; ++q) sort_segment_cta(vals, tmp, toff, s_long[q], T, st, m_cap, sh);
  }
}

// ---------------------------------------------------------------- ranges

__global__ void __launch_bounds__(256) k_ranges(const unsigned long long* toff, int2* range,
                                                int T, const DevStatus* st, int64_t m_cap) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
    int64_t a, b;
    tile_segment(toff, t, T, st, m_cap, a, b);
    range[t] = make_int2((int)a, (int)b);
  }
}

__global__ void __launch_bounds__(256) k_tile_evals(const int2* range, int T, int H, int W,
                                                    int tile, int tiles_x, DevStatus* st) {
  __shared__ unsigned long long s_warp[33];
  unsigned long long acc = 0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < T; j += gridDim.x * blockDim.x) {
    const int tx = j % tiles_x, ty = j / tiles_x;
    const int w = min((tx + 1) * tile, W) - tx * tile;
    const int h = min((ty + 1) * tile, H) - ty * tile;
    const int2 r = range[j];
    acc += (unsigned long long)(r.y - r.x) * (unsigned long long)(w * h);
  }
  unsigned long long tot;
  block_exclusive_scan<unsigned long long>(acc, s_warp, tot);
  if (threadIdx.x == 0 && tot) atomicAdd(&st->evals, tot);
}

__global__ void __launch_bounds__(256) k_fill_image_of(int* img_of, const long long* off,
                                                       int B, int64_t N) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = B - 1;  // largest b with off[b] <= i
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    img_of[i] = lo;
  }
}

__global__ void __launch_bounds__(256) k_tile_evals_batch(const int2* range, int T,
                                                          const int4* dims, const int* tile_off,
                                                          int B, int tile, DevStatus* st) {
  __shared__ unsigned long long s_warp[33];
  unsigned long long acc = 0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < T; j += gridDim.x * blockDim.x) {
    int lo = 0, hi = B - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile_off[mid] <= j) lo = mid; else hi = mid - 1;
    }
    const int4 d = dims[lo];
    const int local = j - tile_off[lo];
    const int tx = local % d.z, ty = local / d.z;
    const int w = min((tx + 1) * tile, d.y) - tx * tile;
    const int h = min((ty + 1) * tile, d.x) - ty * tile;
    const int2 r = range[j];
    acc += (unsigned long long)(r.y - r.x) * (unsigned long long)(w * h);
  }
  unsigned long long tot;
  block_exclusive_scan<unsigned long long>(acc, s_warp, tot);
  if (threadIdx.x == 0 && tot) atomicAdd(&st->evals, tot);
}

}  // namespace

cudaError_t launch_preprocess(const PrepParams& p, int dtype, cudaStream_t s) {
  if (p.N == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((p.N + 255) / 256);
  const bool batch = p.img_of != nullptr;
  switch (dtype * 2 + (batch ? 1 : 0)) {
    case 0: k_preprocess<float, false><<<grid, 256, 0, s>>>(p); break;
    case 1: k_preprocess<float, true><<<grid, 256, 0, s>>>(p); break;
    case 2: k_preprocess<__half, false><<<grid, 256, 0, s>>>(p); break;
    case 3: k_preprocess<__half, true><<<grid, 256, 0, s>>>(p); break;
    case 4: k_preprocess<__nv_bfloat16, false><<<grid, 256, 0, s>>>(p); break;
    case 5: k_preprocess<__nv_bfloat16, true><<<grid, 256, 0, s>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_emit(const PrepParams& p, cudaStream_t s) {
  const unsigned grid = (unsigned)((p.N + 255) / 256);
  if (p.img_of)
    k_emit<true><<<grid > 0 ? grid : 1, 256, 0, s>>>(p);
  else
    k_emit<false><<<grid > 0 ? grid : 1, 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_fill_image_of(int* img_of, const long long* gauss_off, int B, int64_t N,
                                 cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  const int64_t want = (N + 255) / 256;
  k_fill_image_of<<<(unsigned)std::min<int64_t>(want, 148 * 16), 256, 0, s>>>(img_of, gauss_off,
                                                                              B, N);
  return cudaGetLastError();
}

cudaError_t launch_tile_evals_batch(const int2* range, int T, const int4* dims,
                                    const int* tile_off, int B, int tile, DevStatus* status,
                                    cudaStream_t s) {
  const unsigned g = (unsigned)std::min<int64_t>((T + 255) / 256, 148 * 4);
  k_tile_evals_batch<<<g > 0 ? g : 1, 256, 0, s>>>(range, T, dims, tile_off, B, tile, status);
  return cudaGetLastError();
}

cudaError_t launch_scan_u32_to_u64(const unsigned int* in, unsigned long long* out, int64_t n,
                                   unsigned long long* part, unsigned long long* total,
                                   cudaStream_t s) {
  return scan_exclusive<unsigned int, unsigned long long>(in, out, n, part, total, s);
}

cudaError_t launch_scan_u64(const unsigned long long* in, unsigned long long* out, int64_t n,
                            unsigned long long* part, unsigned long long* total,
                            cudaStream_t s) {
  return scan_exclusive<unsigned long long, unsigned long long>(in, out, n, part, total, s);
}

cudaError_t run_binning(const PrepParams& p, int dtype, int T, unsigned long long* part,
                        int2* range, int sort_min, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(p.tcnt, 0, sizeof(unsigned int) * (size_t)T, s);
  if (e != cudaSuccess) return e;
  if ((e = launch_preprocess(p, dtype, s)) != cudaSuccess) return e;
  const bool batch = p.img_of != nullptr;
  // one image: tile blocks own their tiles' wide hits; a batch: one CTA per
  // wide Gaussian (up to WIDE_GRID at a time)
  const int64_t wt_blocks = (int64_t)((p.tiles_x + WT_BLOCK - 1) / WT_BLOCK) *
                            ((p.tiles_y + WT_BLOCK - 1) / WT_BLOCK);
  const unsigned wt_grid = (unsigned)std::max<int64_t>(wt_blocks, 148 * 4);
  if (batch) k_wide<true, true><<<WIDE_GRID, 256, 0, s>>>(p);
  else if (T > 0) k_wide_tiles<true><<<wt_grid, 256, 0, s>>>(p);
  // the tile scan; for one image its last pass also writes the tile ranges
  // and the evaluation count (the batch gets them from k_ranges and its own
  // evaluation kernel after the emission)
  if (batch) {
    if ((e = launch_scan_u32_to_u64(p.tcnt, p.toff, T, part, &p.status->m_needed, s)) !=
        cudaSuccess)
      return e;
  } else if (T > 0) {
    const int64_t nb = ((int64_t)T + SCAN_ITEMS - 1) / SCAN_ITEMS;
    k_scan_reduce<unsigned int, unsigned long long><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(
        p.tcnt, T, part);
    k_scan_partials<<<1, 1024, 0, s>>>(part, nb, &p.status->m_needed);
    k_scan_down_tiles<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(p.tcnt, p.toff, T, part, range,
                                                            p.m_cap, p.H, p.W, p.tile,
                                                            p.tiles_x, p.status);
  }
  if ((e = launch_emit(p, s)) != cudaSuccess) return e;
  if (batch) k_wide<true, false><<<WIDE_GRID, 256, 0, s>>>(p);
  else if (T > 0) k_wide_tiles<false><<<wt_grid, 256, 0, s>>>(p);
  if ((e = launch_segsort(p.vals, p.tmp, p.toff, T, p.status, p.m_cap, sort_min, s)) !=
      cudaSuccess)
    return e;
  if (!batch) return cudaGetLastError();
  return launch_ranges(p.toff, range, T, p.m_cap, p.H, p.W, p.tile,
                       p.img_of ? 0 : p.tiles_x, p.status, s);
}

cudaError_t launch_segsort(unsigned int* vals, unsigned int* tmp,
                           const unsigned long long* toff, int T, DevStatus* status,
                           int64_t m_cap, int sort_min, cudaStream_t s) {
  if (T == 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>(((int64_t)T + 31) / 32, 148 * 8);
  k_segsort_long<<<grid, 256, 0, s>>>(vals, tmp, toff, T, status, m_cap, sort_min);
  return cudaGetLastError();
}

cudaError_t launch_ranges(const unsigned long long* toff, int2* range, int T, int64_t m_cap,
                          int H, int W, int tile, int tiles_x, DevStatus* status,
                          cudaStream_t s) {
  if (T == 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>((T + 255) / 256, 148 * 8);
  k_ranges<<<grid, 256, 0, s>>>(toff, range, T, status, m_cap);
  if (tiles_x > 0) {  // single image; the batched form counts its evaluations itself
    const unsigned g2 = (unsigned)std::min<int64_t>((T + 255) / 256, 148 * 4);
    k_tile_evals<<<g2 > 0 ? g2 : 1, 256, 0, s>>>(range, T, H, W, tile, tiles_x, status);
  }
  return cudaGetLastError();
}

}  // namespace igs
