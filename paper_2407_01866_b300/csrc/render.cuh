// Per-tile forward render (Eq. 5 with top-K, Sec. 3.2), its adjoint
// (Sec. 3.3: gradients through the K retained Gaussians) fused with the L1
// loss, and random-access decode. Included by the translation units that
// instantiate and dispatch them.
//
// One CTA renders one logical tile of TILE x TILE pixels, one pixel per
// thread; each warp owns a compact 8 x 4 block of pixels.
//
// Fast path (the tile's list S_j fits one stage of CH records, the common
// case): the list is staged once into shared memory, ordered by each
// candidate's ranking key at the tile centre, nearest first. The order
// decides only how much work is skipped, never which Gaussians win.
//
//   pass A  each pixel keeps the K smallest packed keys (the binary32
//           ranking key with its low 8 bits replaced by the staged slot):
//           the first K candidates fill the top K through a sorting network,
//           later ones enter through a min/max insertion network, run only
//           when some lane of the warp improves (warp vote). Before
//           candidates are evaluated per pixel, the warp tests them
//           lane-parallel against a lower bound of the key over its 8 x 4
//           block, and re-tests the survivors as the threshold falls: a
//           candidate whose bound exceeds the K-th key of every pixel of the
//           block cannot enter any top K and is skipped. The packed top K is
//           the exact (key, index) top K unless the K-th and (K+1)-th packed
//           keys share their upper 24 bits (or the K-th is negative); a warp
//           with such a pixel recomputes its selection exactly (the float
//           pass A, the tie cut-off and a membership pass).
//   blend   the winners' slots come out of pass A: their keys are recomputed
//           exactly and blended with w = exp(-(q - q_min)/2) (Eq. 5). The
//           adjoint also records each winner as (slot, rank of the pixel
//           among its half-warp's pixels that won the slot): each pixel ORs
//           its lane bit into its half-warp's mask of the slot, and the rank
//           is the number of bits set before its own.
//   pass C  (adjoint only) a counting sort of those records lays out the
//           winning (candidate, pixel) pairs candidate-major; the pairs are
//           split evenly over the CTA's threads; each accumulates dL/dq
//           moments in registers and leaves one partial sum per candidate it
//           touched in a shared-memory slot with a single writer; one thread
//           per candidate adds its slots and turns them into parameter
//           gradients with global (vector) atomics.
//
// K = 0 (every candidate of S_j wins) keeps float keys: pass A finds q_min
// and pass B blends every candidate. Longer lists take the chunked path:
// passes A and B stream the list in ascending index order (equal keys at tau
// are admitted in that order), and pass C re-tests membership per
// (candidate, pixel). Nothing is stored between forward and adjoint.
#pragma once
#include <utility>
#include <type_traits>

#include "internal.h"

namespace igs {

// K = 0 selects all of S_j (no top-K): arrays keep one slot.
template <int K> struct KS { static constexpr int A = K > 0 ? K : 1; };

// Pass C's winner masks: for each warp block and staged candidate j, one
// 32-bit word that lanes 0-15 set their bits in (at warp * CH + j) and one for
// lanes 16-31 (rec_upper(NWB, CH) words further on, in the bank 16 away), so
// that at most 16 lanes' atomics meet at one address.
__host__ __device__ constexpr int rec_upper(int nwb, int ch) { return nwb * ch + 16; }

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

// Pixel centres of the calling warp's 8 x 4 block: (x_lo, x_hi, y_lo, y_hi).
template <int TILE>
__device__ __forceinline__ float4 block_rect(int x0, int y0) {
  constexpr int BPR = TILE / 8;
  const int w = threadIdx.x >> 5;
  const float bx = (float)(x0 + (w % BPR) * 8) + 0.5f;
  const float by = (float)(y0 + (w / BPR) * 4) + 0.5f;
  return make_float4(bx, bx + 7.0f, by, by + 3.0f);
}

constexpr float F_INF = __builtin_huge_valf();
constexpr int GID_NONE = 0x7fffffff;  // tie cut-off that admits every index


// Staged candidate record in shared memory:
//   a = (mx, my, A00, B)   geometry of the ranking key
//   b = (A11, index as int bits)
//   e = (1/(2 A00), 1/(2 A11)), the minimiser of q along one axis for a
//       fixed displacement along the other (fast path only).

// Lower bound of the ranking key of staged record (a, a11, e) at every pixel
// centre of the rectangle R = [x_lo, x_hi] x [y_lo, y_hi], valid for the
// float32 evaluation of rank_key. q is a convex quadratic of the
// displacement d = p - mu; unless mu lies in R, its minimum over R lies on a
// face of R that faces mu, and on such a face (dx fixed) the minimum is at
// dy = -B dx / (2 A11) clamped to the face. The smaller of the (at most two)
// facing faces' minima is reduced by a relative 1e-5 and by 2e-6 times the
// largest sum of term magnitudes |A00| dx^2 + |B dx dy| + A11 dy^2 over R
// (float32 rounding of the key, of the staged conic and of this bound are
// each a few 2^-24 of those).
__device__ __forceinline__ float key_lower_bound(const float4& a, float a11, const float2& e,
                                                 const float4& R) {
  const float ux0 = R.x - a.x, ux1 = R.y - a.x;  // range of dx over R
  const float uy0 = R.z - a.y, uy1 = R.w - a.y;  // range of dy over R
  // face facing mu in x (dx fixed to the near edge), dy minimising, clamped
  const float fdx = ux0 > 0.0f ? ux0 : ux1;
  const float fdy = fminf(fmaxf(-a.w * fdx * e.y, uy0), uy1);
  const float qx = fmaf(fmaf(a.z, fdx, a.w * fdy), fdx, a11 * fdy * fdy);
  // face facing mu in y
  const float gdy = uy0 > 0.0f ? uy0 : uy1;
  const float gdx = fminf(fmaxf(-a.w * gdy * e.x, ux0), ux1);
  const float qy = fmaf(fmaf(a11, gdy, a.w * gdx), gdy, a.z * gdx * gdx);
  const bool xin = ux0 <= 0.0f && ux1 >= 0.0f;
  const bool yin = uy0 <= 0.0f && uy1 >= 0.0f;
  const float L = (xin && yin) ? 0.0f : fminf(xin ? F_INF : qx, yin ? F_INF : qy);
  const float fx = fmaxf(fabsf(ux0), fabsf(ux1));
  const float fy = fmaxf(fabsf(uy0), fabsf(uy1));
  const float hb = 0.5f * fabsf(a.w);
  const float M = (fabsf(a.z) + hb) * fx * fx + (a11 + hb) * fy * fy;
  return fmaf(L, 1.0f - 1e-5f, -2e-6f * M);
}

// Largest value of v over the warp for non-negative keys (negative rounding
// residues count as 0, which only loosens a cull threshold).
__device__ __forceinline__ float warp_max_key(float v) {
  return __uint_as_float(__reduce_max_sync(FULL_MASK, __float_as_uint(fmaxf(v, 0.0f))));
}

// Ranking geometry of Gaussian gid, a = (mx, my, A00, B) and A11, from the
// records the launch reads: the 16-byte hot record of half-precision storage
// (mu in pixels recomputed with preprocessing's binary32 product), else the
// float32 record. Both give the same binary32 values.
__device__ __forceinline__ void load_geom(const RenderParams& p, int gid, float4& a, float& a11) {
  if (p.hdt) {
    const HRec h = p.rec16[gid];
    a = make_float4(__fmul_rn(half_bits_to_f32((unsigned short)(h.mu & 0xffffu), p.hdt),
                              (float)p.W),
                    __fmul_rn(half_bits_to_f32((unsigned short)(h.mu >> 16), p.hdt),
                              (float)p.H),
                    h.A00, h.B);
    a11 = h.A11;
  } else {
    const GRec g = p.rec[gid];
    a = g.a;
    a11 = g.b.x;
  }
}

// Channel c of Gaussian gid's colour (stored half-precision bits, or float32).
__device__ __forceinline__ float load_colour(const RenderParams& p, int gid, int c, int n) {
  return p.hdt ? half_bits_to_f32(p.col16[(int64_t)gid * n + c], p.hdt)
               : p.color[(int64_t)gid * n + c];
}

// Colours of staged candidates live in shared memory, candidate-major
// s_col[j * col_stride(NC) + c], when the channel count is a compile-time
// constant; three channels are padded to a float4 (one 16-byte load).
__host__ __device__ constexpr int col_stride(int nc) { return nc == 3 ? 4 : (nc > 0 ? nc : 1); }

// Chunked path: stage list entries [base, base+cnt) in list order.
template <int NT, int NC>
__device__ __forceinline__ void stage_chunk(const RenderParams& p, int base, int cnt,
                                            float4* s_a, float2* s_b, float* s_col) {
  const int j = threadIdx.x;
  if (j < cnt) {
    const int gid = p.list[base + j];
    if ((unsigned)gid < (unsigned)p.N) {
      float4 a;
      float a11;
      load_geom(p, gid, a, a11);
      s_a[j] = a;
      s_b[j] = make_float2(a11, __int_as_float(gid));
      if (NC > 0) {
#pragma unroll
        for (int c = 0; c < (NC > 0 ? NC : 1); ++c)
          s_col[j * col_stride(NC) + c] = load_colour(p, gid, c, NC);
      }
    } else {  // corrupt list entry: a NaN key is never selected
      s_a[j] = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
      s_b[j] = make_float2(0.f, __int_as_float(-1));
      if (NC > 0) {
#pragma unroll
        for (int c = 0; c < (NC > 0 ? NC : 1); ++c) s_col[j * col_stride(NC) + c] = 0.0f;
      }
      atomicOr(&p.status->flags, FLAG_INTERNAL);
    }
  }
}

// Fast path: stage the whole list (cnt <= NT <= blockDim.x), each record at
// its rank in the (key at (cx, cy), index) order, which does not depend on
// the order of the list. s_key holds 2 NT words (16-byte aligned) of scratch
// that must not overlap the staged arrays.
template <int NT, int NC>
__device__ __forceinline__ void stage_sorted(const RenderParams& p, int base, int cnt, float cx,
                                             float cy, float4* s_a, float2* s_b, float2* s_e,
                                             float* s_col, unsigned* s_key) {
  constexpr int NCS = NC > 0 ? NC : 1;
  const int j = threadIdx.x;
  float4 ga;
  float ga11 = 0.0f;
  float col[NCS];
  int gid = -1;
  unsigned key = 0xffffffffu, kid = 0xffffffffu;  // padding: after every real entry
  if (j < cnt) {
    const int e = p.list[base + j];
    kid = 0x80000000u | (unsigned)j;  // a corrupt entry: unique, after every index
    if ((unsigned)e < (unsigned)p.N) {
      kid = (unsigned)e;
      gid = e;
      load_geom(p, gid, ga, ga11);
      if (NC > 0) {
#pragma unroll
        for (int c = 0; c < NCS; ++c) col[c] = load_colour(p, gid, c, NC);
      }
      key = __float_as_uint(fmaxf(rank_key(cx, cy, ga.x, ga.y, ga.z, ga.w, ga11), 0.0f));
    }
  }
  // 64-bit (key, index) words: one unsigned compare orders them
  const unsigned long long mine = ((unsigned long long)key << 32) | kid;
  const int cnt2 = (cnt + 1) & ~1;
  if (j < cnt2) reinterpret_cast<unsigned long long*>(s_key)[j] = mine;
  __syncthreads();
  if (j < cnt) {
    int r = 0;
    const ulonglong2* k2 = reinterpret_cast<const ulonglong2*>(s_key);
    for (int i = 0; i < cnt2 / 2; ++i) {
      const ulonglong2 v = k2[i];
      r += (v.x < mine ? 1 : 0) + (v.y < mine ? 1 : 0);
    }
    if (gid >= 0) {
      s_a[r] = ga;
      s_b[r] = make_float2(ga11, __int_as_float(gid));
      s_e[r] = make_float2(0.5f * rcp_approx(ga.z), 0.5f * rcp_approx(ga11));
      if (NC > 0) {
#pragma unroll
        for (int c = 0; c < NCS; ++c) s_col[r * col_stride(NC) + c] = col[c];
      }
    } else {  // corrupt list entry: key +inf at every pixel (weight 0 if kept)
      s_a[r] = make_float4(F_INF, 0.f, 1.f, 0.f);
      s_b[r] = make_float2(0.f, __int_as_float(-1));
      s_e[r] = make_float2(0.f, 0.f);
      if (NC > 0) {
#pragma unroll
        for (int c = 0; c < NCS; ++c) s_col[r * col_stride(NC) + c] = 0.0f;
      }
      atomicOr(&p.status->flags, FLAG_INTERNAL);
    }
  }
}

// Channel c of staged candidate j (shared memory if staged, else global).
template <int NT, int NC>
__device__ __forceinline__ float staged_colour(const RenderParams& p, const float* s_col,
                                               const float2* s_b, int j, int c) {
  if (NC > 0) return s_col[j * col_stride(NC) + c];
  return p.color[(int64_t)__float_as_int(s_b[j].y) * p.n + c];
}

// Per-pixel factors -g/(2Z) of the adjoint in shared memory: pixel-major,
// one float4 per pixel, for 3 or 4 channels; channel-major otherwise.
template <int NC>
__device__ __forceinline__ int gh_at(int i, int c, int NT) {
  return (NC == 3 || NC == 4) ? i * 4 + c : c * NT + i;
}
template <int NC>
__device__ __forceinline__ void pixel_gh(const float* s_gh, int i, int n, int NT,
                                         float (&gh)[Chan<NC>::R]) {
  if (NC == 3 || NC == 4) {
    const float4 v = reinterpret_cast<const float4*>(s_gh)[i];
    gh[0] = v.x;
    gh[1] = v.y;
    gh[2] = v.z;
    if (NC == 4) gh[NC == 4 ? 3 : 0] = v.w;
  } else {
#pragma unroll
    for (int c = 0; c < Chan<NC>::R; ++c) gh[c] = (NC > 0 || c < n) ? s_gh[c * NT + i] : 0.0f;
  }
}

// All channels of staged candidate j (one 16-byte load for 3 or 4 channels).
template <int NT, int NC>
__device__ __forceinline__ void staged_colours(const RenderParams& p, const float* s_col,
                                               const float2* s_b, int j,
                                               float (&cc)[Chan<NC>::R]) {
  if (NC == 3 || NC == 4) {
    const float4 v = reinterpret_cast<const float4*>(s_col)[j];
    cc[0] = v.x;
    cc[1] = v.y;
    cc[2] = v.z;
    if (NC == 4) cc[NC == 4 ? 3 : 0] = v.w;
  } else {
    const int n = nchan<NC>(p);
#pragma unroll
    for (int c = 0; c < Chan<NC>::R; ++c)
      cc[c] = (NC > 0 || c < n) ? staged_colour<NT, NC>(p, s_col, s_b, j, c) : 0.0f;
  }
}

// Sorted insertion of key x into tq[0..A-1] (ascending), the largest key
// dropping out into x. +inf inserts nothing.
template <int A>
__device__ __forceinline__ void insert_key(float (&tq)[A], float& x) {
#pragma unroll
  for (int k = 0; k < A; ++k) {
    const float lo = fminf(tq[k], x);
    x = fmaxf(tq[k], x);
    tq[k] = lo;
  }
}

// Ascending sort of v[0..A-1]: Batcher's odd-even merge network for the next
// power of two, without the comparators that meet a wire >= A (those wires
// would hold +inf and never move). The comparator table is built at compile
// time and applied by a fold, so every index is a constant (registers only).
struct SortNet {
  int lo[64], hi[64], n;
};
__host__ __device__ constexpr SortNet make_sort_net(int A) {
  SortNet t{};
  t.n = 0;
  for (int p = 1; p < A; p *= 2)
    for (int k = p; k >= 1; k /= 2)
      for (int j = k % p; j + k < A; j += 2 * k)
        for (int i = 0; i < k; ++i)
          if (i + j + k < A && (i + j) / (2 * p) == (i + j + k) / (2 * p)) {
            t.lo[t.n] = i + j;
            t.hi[t.n] = i + j + k;
            ++t.n;
          }
  return t;
}
template <int A, size_t... C>
__device__ __forceinline__ void apply_sort_net(float (&v)[A], std::index_sequence<C...>) {
  constexpr SortNet t = make_sort_net(A);
  auto cx = [](float& x, float& y) {
    const float lo = fminf(x, y);
    y = fmaxf(x, y);
    x = lo;
  };
  (cx(v[t.lo[C]], v[t.hi[C]]), ...);
}
template <int A>
__device__ __forceinline__ void sort_network(float (&v)[A]) {
  static_assert(A <= 16, "at most 63 comparators are tabulated");
  apply_sort_net<A>(v, std::make_index_sequence<make_sort_net(A).n>{});
}

// Per-pixel result of pass B.
template <int NCR>
struct PixelBlend {
  float Z;          // sum of winner weights (0 if the pixel has none)
  float cr[NCR];    // blended colour
  float tau;        // K-th key (+inf if |S_j| < K)
  float q0;         // smallest key (0 when unnormalised)
  float iz;         // 1 / Z (normalised, Z > 0), 1 (unnormalised) or 0
  int gcut;         // largest index admitted among winners whose key equals tau
  int nw;           // winners recorded by pass B for pass C (fast path adjoint)
};

// ---------------------------------------------------------------------------
// Chunked path (lists longer than one stage), list order.
// ---------------------------------------------------------------------------

// Pass A: the K smallest keys at (px, py), ascending.
template <int TILE, int K, int CH>
__device__ __forceinline__ void select_keys(const RenderParams& p, int2 range, float px,
                                            float py, float (&tq)[KS<K>::A], float4* s_a,
                                            float2* s_b) {
#pragma unroll
  for (int k = 0; k < KS<K>::A; ++k) tq[k] = F_INF;
  if (K == 0 && !p.normalize) return;  // every candidate wins, no shift needed
  for (int base = range.x; base < range.y; base += CH) {
    const int cnt = min(CH, range.y - base);
    __syncthreads();
    stage_chunk<CH, 0>(p, base, cnt, s_a, s_b, nullptr);
    __syncthreads();
#pragma unroll 4
    for (int j = 0; j < cnt; ++j) {
      const float4 a = s_a[j];
      const float q = rank_key(px, py, a.x, a.y, a.z, a.w, s_b[j].x);
      if (K == 0) {  // all of S_j: only the smallest key is needed
        tq[0] = fminf(tq[0], q);
        continue;
      }
      const bool better = q < tq[KS<K>::A - 1];
      if (__any_sync(FULL_MASK, better)) {
        float x = better ? q : F_INF;  // +inf (and NaN) insert nothing
        insert_key<KS<K>::A>(tq, x);
      }
    }
  }
}

// Pass B: exact top-K membership in list (index) order and the blend of Eq. 5.
template <int TILE, int K, int NC, int CH>
__device__ __forceinline__ void blend_pass(const RenderParams& p, int2 range, float px,
                                           float py, const float (&tq)[KS<K>::A],
                                           PixelBlend<Chan<NC>::R>& r, float4* s_a,
                                           float2* s_b, float* s_col) {
  constexpr int NCR = Chan<NC>::R;
  const int n = nchan<NC>(p);
  r.q0 = p.normalize ? tq[0] : 0.0f;  // unnormalised: w = exp(-q/2) itself
  r.tau = K == 0 ? F_INF : tq[KS<K>::A - 1];
  int lt = 0;
#pragma unroll
  for (int k = 0; k < KS<K>::A; ++k) lt += tq[k] < r.tau ? 1 : 0;
  int eq_left = K - lt;  // tau-valued slots still open
  r.gcut = -1;
  r.Z = 0.0f;
#pragma unroll
  for (int c = 0; c < NCR; ++c) r.cr[c] = 0.0f;
  for (int base = range.x; base < range.y; base += CH) {
    const int cnt = min(CH, range.y - base);
    __syncthreads();
    stage_chunk<CH, NC>(p, base, cnt, s_a, s_b, s_col);
    __syncthreads();
#pragma unroll 2
    for (int j = 0; j < cnt; ++j) {
      const float4 a = s_a[j];
      const float q = rank_key(px, py, a.x, a.y, a.z, a.w, s_b[j].x);
      bool win = q < r.tau;
      if (q == r.tau && eq_left > 0) {
        win = true;
        --eq_left;
        r.gcut = __float_as_int(s_b[j].y);
      }
      if (__any_sync(FULL_MASK, win)) {
        if (win) {
          const float w = blend_weight(r.q0, q);  // exactly 1 at q = q_min
          r.Z += w;
          float cc[NCR];
          staged_colours<CH, NC>(p, s_col, s_b, j, cc);
#pragma unroll
          for (int c = 0; c < NCR; ++c)
            if (NC > 0 || c < n) r.cr[c] = fmaf(w, cc[c], r.cr[c]);
        }
      }
    }
  }
  r.iz = p.normalize ? (r.Z > 0.0f ? rcp_approx(r.Z) : 0.0f) : 1.0f;
#pragma unroll
  for (int c = 0; c < NCR; ++c) r.cr[c] *= r.iz;
}

// ---------------------------------------------------------------------------
// Fast path: one staged, key-ordered list; per-warp culling.
// ---------------------------------------------------------------------------

// Pass A over the staged list. mdrop receives the smallest evaluated key
// that did not stay in the top K (+inf if none): a key equal to tau left out.
template <int K>
__device__ __forceinline__ void culled_keys(const RenderParams& p, int cnt, float px, float py,
                                            bool live, const float4& R, const float4* s_a,
                                            const float2* s_b, const float2* s_e,
                                            float (&tq)[KS<K>::A], float& mdrop) {
  constexpr int A = KS<K>::A;
#pragma unroll
  for (int k = 0; k < A; ++k) tq[k] = F_INF;
  mdrop = F_INF;
  if (K == 0 && !p.normalize) return;
  const int lane = threadIdx.x & 31;
  float thr = F_INF;  // no lane of the block can use a key above this
  int c0 = 0, gw = 16;
  if (K > 0) {
    // the first A candidates (nearest first) fill the empty top K, sorted by
    // a network; nothing drops (a NaN key from a corrupt entry counts as +inf)
#pragma unroll
    for (int k = 0; k < A; ++k) {
      const float4 a = s_a[k];
      const float q = k < cnt ? rank_key(px, py, a.x, a.y, a.z, a.w, s_b[k].x) : F_INF;
      tq[k] = q < F_INF ? q : F_INF;
    }
    sort_network<A>(tq);
    c0 = A;
    gw = 32;
    thr = warp_max_key(live ? tq[A - 1] : 0.0f);
  }
  // (K = 0: a first group of 16 then groups of 32). A lane holds the bound of
  // one candidate of the group; the survivors are re-tested against the
  // threshold after every pair, as it only falls.
  for (; c0 < cnt; c0 += gw, gw = 32) {
    const int jl = c0 + lane;
    const float bnd = (lane < gw && jl < cnt) ? key_lower_bound(s_a[jl], s_b[jl].x, s_e[jl], R)
                                              : F_INF;
    unsigned m = __ballot_sync(FULL_MASK, !(bnd > thr));
    auto take = [&](float q) {
      if (K == 0) {  // all of S_j: only the smallest key is needed
        tq[0] = fminf(tq[0], q);
        return;
      }
      const bool better = q < tq[A - 1];
      float out = q;
      if (__any_sync(FULL_MASK, better)) {
        float x = better ? q : F_INF;
        insert_key<A>(tq, x);
        out = better ? x : q;
      }
      mdrop = fminf(mdrop, out);
    };
    while (m) {
      const int j0 = c0 + __ffs(m) - 1;
      m &= m - 1;
      const bool two = m != 0;
      const int j1 = two ? c0 + __ffs(m) - 1 : j0;
      m &= m - 1;
      const float4 a0 = s_a[j0], a1 = s_a[j1];
      const float b0 = s_b[j0].x, b1 = s_b[j1].x;
      const float q0 = rank_key(px, py, a0.x, a0.y, a0.z, a0.w, b0);
      const float q1 = rank_key(px, py, a1.x, a1.y, a1.z, a1.w, b1);
      take(q0);
      if (two) take(q1);
      if (K > 0) {
        thr = warp_max_key(live ? tq[A - 1] : 0.0f);
        m &= __ballot_sync(FULL_MASK, !(bnd > thr));
      }
    }
    thr = warp_max_key(live ? tq[A - 1] : 0.0f);
  }
}

// Index cut-off of a pixel whose tau ties with a key left out: the eq_left-th
// smallest index among candidates with key tau, eq_left = K minus the number
// of keys below tau. Rare; every candidate is re-evaluated once per round.
template <int K>
__device__ __forceinline__ int tie_cutoff(int cnt, float px, float py, bool tie, float tau,
                                          const float (&tq)[KS<K>::A], const float4* s_a,
                                          const float2* s_b) {
  int lt = 0;
#pragma unroll
  for (int k = 0; k < KS<K>::A; ++k) lt += tq[k] < tau ? 1 : 0;
  const int eq_left = K - lt;
  int gc = -1;
  for (int round = 0;; ++round) {
    const bool need = tie && round < eq_left;
    if (!__any_sync(FULL_MASK, need)) break;
    int gmin = GID_NONE;
    for (int j = 0; j < cnt; ++j) {
      const float4 a = s_a[j];
      const float2 b = s_b[j];
      const float q = rank_key(px, py, a.x, a.y, a.z, a.w, b.x);
      const int gid = __float_as_int(b.y);
      if (need && q == tau && gid > gc && gid < gmin) gmin = gid;
    }
    if (need) gc = gmin;
  }
  return tie ? gc : GID_NONE;
}

// Pass B over the staged list where there are no packed keys (K = 0, where
// every candidate is kept): membership against (tau, tie cut-off) and blend.
template <int K, int NC, int CH>
__device__ __forceinline__ void culled_blend(const RenderParams& p, int cnt, float px, float py,
                                             bool live, const float4& R,
                                             const float (&tq)[KS<K>::A], float mdrop,
                                             const float4* s_a, const float2* s_b,
                                             const float2* s_e, const float* s_col,
                                             PixelBlend<Chan<NC>::R>& r) {
  constexpr int NCR = Chan<NC>::R;
  constexpr int A = KS<K>::A;
  const int n = nchan<NC>(p);
  const int lane = threadIdx.x & 31;
  r.nw = 0;
  r.q0 = p.normalize ? tq[0] : 0.0f;
  r.tau = K == 0 ? F_INF : tq[A - 1];
  r.gcut = GID_NONE;
  if (K > 0) {
    const bool tie = mdrop == r.tau && r.tau < F_INF;
    if (__any_sync(FULL_MASK, tie))
      r.gcut = tie_cutoff<K>(cnt, px, py, tie, r.tau, tq, s_a, s_b);
  }
  r.Z = 0.0f;
#pragma unroll
  for (int c = 0; c < NCR; ++c) r.cr[c] = 0.0f;
  const float T = K == 0 ? F_INF : warp_max_key(live ? r.tau : 0.0f);
  for (int c0 = 0; c0 < cnt; c0 += 32) {
    const int jl = c0 + lane;
    const bool in = jl < cnt;
    const bool surv = in && !(key_lower_bound(s_a[jl], s_b[jl].x, s_e[jl], R) > T);
    unsigned m = __ballot_sync(FULL_MASK, surv);
    auto take = [&](int j, float q, int gid) {
      const bool win = q < r.tau || (q == r.tau && gid <= r.gcut);
      if (win) {
        const float w = blend_weight(r.q0, q);  // exactly 1 at q = q_min
        r.Z += w;
        float cc[NCR];
        staged_colours<CH, NC>(p, s_col, s_b, j, cc);
#pragma unroll
        for (int c = 0; c < NCR; ++c)
          if (NC > 0 || c < n) r.cr[c] = fmaf(w, cc[c], r.cr[c]);
      }
    };
    while (m) {
      const int j0 = c0 + __ffs(m) - 1;
      m &= m - 1;
      const bool two = m != 0;
      const int j1 = two ? c0 + __ffs(m) - 1 : j0;
      m &= m - 1;
      const float4 a0 = s_a[j0], a1 = s_a[j1];
      const float2 b0 = s_b[j0], b1 = s_b[j1];
      const float q0 = rank_key(px, py, a0.x, a0.y, a0.z, a0.w, b0.x);
      const float q1 = rank_key(px, py, a1.x, a1.y, a1.z, a1.w, b1.x);
      take(j0, q0, __float_as_int(b0.y));
      if (two) take(j1, q1, __float_as_int(b1.y));
    }
  }
  r.iz = p.normalize ? (r.Z > 0.0f ? rcp_approx(r.Z) : 0.0f) : 1.0f;
#pragma unroll
  for (int c = 0; c < NCR; ++c) r.cr[c] *= r.iz;
}

// ---------------------------------------------------------------------------
// Fast path with packed keys (K > 0). Pass A keeps, per pixel, the K smallest
// packed keys: the binary32 ranking key's bits with the low 8 bits replaced
// by the candidate's staged slot, compared as signed integers. Within one
// bucket of equal upper 24 bits the packed order is the slot order instead
// of the (key, index) order; outside it the two orders agree (keys >= 0
// order like their bits). So the K smallest packed keys are exactly the top K
// unless the K-th and the (K+1)-th smallest fall in one bucket, or the K-th is
// negative (a key below 0 from rounding; negative keys order in reverse as
// integers). The warp then takes the exact path instead: the float pass A,
// the tie cut-off and a membership pass. Otherwise the winners' slots come
// straight out of pass A and no candidate is evaluated a second time to find
// them; only the K winners' keys are recomputed exactly for the blend.
// ---------------------------------------------------------------------------
constexpr int PK_NONE = 0x7fffffff;  // empty slot: after every packed key

__device__ __forceinline__ int pack_key(float q, int slot) {
  return (__float_as_int(q) & ~0xff) | slot;
}

// Sorted insertion of packed key x into tq[0..A-1] (ascending); the largest
// drops out into x. PK_NONE inserts nothing.
template <int A>
__device__ __forceinline__ void insert_pk(int (&tq)[A], int& x) {
#pragma unroll
  for (int k = 0; k < A; ++k) {
    const int lo = min(tq[k], x);
    x = max(tq[k], x);
    tq[k] = lo;
  }
}

template <int A, size_t... C>
__device__ __forceinline__ void apply_sort_net_pk(int (&v)[A], std::index_sequence<C...>) {
  constexpr SortNet t = make_sort_net(A);
  auto cx = [](int& x, int& y) {
    const int lo = min(x, y);
    y = max(x, y);
    x = lo;
  };
  (cx(v[t.lo[C]], v[t.hi[C]]), ...);
}
template <int A>
__device__ __forceinline__ void sort_network_pk(int (&v)[A]) {
  static_assert(A <= 16, "at most 63 comparators are tabulated");
  apply_sort_net_pk<A>(v, std::make_index_sequence<make_sort_net(A).n>{});
}

// Cull threshold of the packed pass A: the upper end of the bucket of the
// largest K-th packed key over the warp's live lanes, as a float. A candidate
// whose key lower bound exceeds it lies in a later bucket than every live
// lane's K-th packed key, so it can neither enter a top K nor share the K-th
// bucket.
__device__ __forceinline__ float pk_threshold(int tk, bool live) {
  return __int_as_float(__reduce_max_sync(FULL_MASK, live ? (tk | 0xff) : INT_MIN));
}

// Pass A with packed keys. tq receives the K smallest packed keys (ascending,
// PK_NONE beyond the list's length), mdrop the smallest packed key evaluated
// but not kept (PK_NONE if none).
template <int K>
__device__ __forceinline__ void packed_keys(int cnt, float px, float py, bool live,
                                            const float4& R, const float4* s_a,
                                            const float2* s_b, const float2* s_e, int (&tq)[K],
                                            int& mdrop) {
  const int lane = threadIdx.x & 31;
  // the first K candidates (nearest first) fill the top K through a network
  if (cnt >= K) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float4 a = s_a[k];
      tq[k] = pack_key(rank_key(px, py, a.x, a.y, a.z, a.w, s_b[k].x), k);
    }
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float4 a = s_a[k];
      tq[k] = k < cnt ? pack_key(rank_key(px, py, a.x, a.y, a.z, a.w, s_b[k].x), k) : PK_NONE;
    }
  }
  sort_network_pk<K>(tq);
  mdrop = PK_NONE;
  float thr = pk_threshold(tq[K - 1], live);
  for (int c0 = K; c0 < cnt; c0 += 32) {
    const int jl = c0 + lane;
    const float bnd = jl < cnt ? key_lower_bound(s_a[jl], s_b[jl].x, s_e[jl], R) : F_INF;
    unsigned m = __ballot_sync(FULL_MASK, !(bnd > thr));
    // a lane whose key is not better passes it through the network
    // unchanged (it is at least every kept key) and drops it
    auto take = [&](int pk) {
      int x = pk;
      if (__any_sync(FULL_MASK, pk < tq[K - 1])) insert_pk<K>(tq, x);
      mdrop = min(mdrop, x);
    };
    while (m) {
      const int j0 = c0 + __ffs(m) - 1;
      m &= m - 1;
      const bool two = m != 0;
      const int j1 = two ? c0 + __ffs(m) - 1 : j0;
      m &= m - 1;
      const float4 a0 = s_a[j0], a1 = s_a[j1];
      const float b0 = s_b[j0].x, b1 = s_b[j1].x;
      const int p0 = pack_key(rank_key(px, py, a0.x, a0.y, a0.z, a0.w, b0), j0);
      const int p1 = pack_key(rank_key(px, py, a1.x, a1.y, a1.z, a1.w, b1), j1);
      take(p0);
      if (two) take(p1);
      // the threshold only falls: survivors are re-tested after every pair
      thr = pk_threshold(tq[K - 1], live);
      m &= __ballot_sync(FULL_MASK, !(bnd > thr));
    }
  }
}

// True when pass A's packed top K may differ from the exact (key, index) top
// K at this pixel (see above).
__device__ __forceinline__ bool pk_ambiguous(int tk, int mdrop) {
  return tk < 0 || (tk != PK_NONE && (tk >> 8) == (mdrop >> 8));
}

// Exact selection for a warp with an ambiguous lane: the float pass A, the
// tie cut-off, then every winner (q < tau, or q == tau and index <= the
// cut-off) packed into tq, in ascending packed order.
template <int K>
__device__ __forceinline__ void exact_winners(const RenderParams& p, int cnt, float px,
                                              float py, bool live, const float4& R,
                                              const float4* s_a, const float2* s_b,
                                              const float2* s_e, int (&tq)[K]) {
  float tf[K];
  float md;
  culled_keys<K>(p, cnt, px, py, live, R, s_a, s_b, s_e, tf, md);
  const float tau = tf[K - 1];
  const bool tie = md == tau && tau < F_INF;
  const int gcut =
      __any_sync(FULL_MASK, tie) ? tie_cutoff<K>(cnt, px, py, tie, tau, tf, s_a, s_b) : GID_NONE;
#pragma unroll
  for (int k = 0; k < K; ++k) tq[k] = PK_NONE;
  const float T = warp_max_key(live ? tau : 0.0f);
  const int lane = threadIdx.x & 31;
  for (int c0 = 0; c0 < cnt; c0 += 32) {
    const int jl = c0 + lane;
    const bool surv = jl < cnt && !(key_lower_bound(s_a[jl], s_b[jl].x, s_e[jl], R) > T);
    unsigned m = __ballot_sync(FULL_MASK, surv);
    while (m) {
      const int j = c0 + __ffs(m) - 1;
      m &= m - 1;
      const float4 a = s_a[j];
      const float2 b = s_b[j];
      const float q = rank_key(px, py, a.x, a.y, a.z, a.w, b.x);
      const bool win = q < tau || (q == tau && __float_as_int(b.y) <= gcut);
      if (__any_sync(FULL_MASK, win)) {
        int x = win ? pack_key(q, j) : PK_NONE;
        insert_pk<K>(tq, x);
      }
    }
  }
}

// A pixel's winner records for pass C, in registers: one per register, or
// (PACK, where registers are scarcer) two 16-bit records per register.
template <int A, bool PACK>
struct WinRecs {
  int v[PACK ? (A + 1) / 2 : A];
  __device__ __forceinline__ void set(int k, int rec) {
    if (!PACK) v[k] = rec;
    else if (k & 1) v[k >> 1] |= rec << 16;
    else v[k >> 1] = rec;
  }
  __device__ __forceinline__ unsigned get(int k) const {
    return PACK ? (((unsigned)v[k >> 1] >> ((k & 1) * 16)) & 0xffffu) : (unsigned)v[k];
  }
};

// Eq. 5 over the winners whose slots are in tq: their keys are recomputed
// exactly, q_min is the smallest of them, and the winners are blended in the
// packed order with w = exp(-(q - q_min)/2). ALL: every entry of tq holds a
// winner (lists of at least K entries), so no entry is tested. REC: each
// winner of a live pixel also sets the lane's bit in its half-warp's mask of
// the slot (cnt_w: this lane's half's masks, as rec_upper describes), and ew
// receives pass C's record of the k-th winner, (slot << 5) | the number of
// lanes of its half that set the mask before it (the popcount of the value
// the OR returns: unique within the half, in no fixed order).
template <int K, int NC, int CH, bool ALL, bool REC, bool PACK>
__device__ __forceinline__ void blend_winners(const RenderParams& p, float px, float py,
                                              const int (&tq)[K], bool live,
                                              const float4* s_a, const float2* s_b,
                                              const float* s_col, unsigned* cnt_w,
                                              PixelBlend<Chan<NC>::R>& r,
                                              WinRecs<K, PACK>* ew) {
  constexpr int NCR = Chan<NC>::R;
  const int n = nchan<NC>(p);
  const unsigned bit = 1u << (threadIdx.x & 31);
  float qe[K];
  float q0 = F_INF;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (ALL || tq[k] != PK_NONE) {
      const int j = tq[k] & 0xff;
      const float4 a = s_a[j];
      qe[k] = rank_key(px, py, a.x, a.y, a.z, a.w, s_b[j].x);
      q0 = fminf(q0, qe[k]);
    }
  }
  r.q0 = p.normalize ? q0 : 0.0f;
  r.Z = 0.0f;
#pragma unroll
  for (int c = 0; c < NCR; ++c) r.cr[c] = 0.0f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (ALL || tq[k] != PK_NONE) {
      const float w = blend_weight(r.q0, qe[k]);  // exactly 1 at q = q_min
      if (REC) {
        const int j = tq[k] & 0xff;
        ew->set(k, live ? (j << 5) | __popc(atomicOr(&cnt_w[j], bit)) : 0);
      }
      r.Z += w;
      float cc[NCR];
      staged_colours<CH, NC>(p, s_col, s_b, tq[k] & 0xff, cc);
#pragma unroll
      for (int c = 0; c < NCR; ++c)
        if (NC > 0 || c < n) r.cr[c] = fmaf(w, cc[c], r.cr[c]);
    }
  }
  r.iz = p.normalize ? (r.Z > 0.0f ? rcp_approx(r.Z) : 0.0f) : 1.0f;
#pragma unroll
  for (int c = 0; c < NCR; ++c) r.cr[c] *= r.iz;
  r.tau = F_INF;
  r.gcut = GID_NONE;
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

// Forward render of one tile (its pixels' Eq. 5 colours into p.img at the
// tile's image offset), with the staged arrays in shared memory.
template <int TILE, int K, int NC>
__device__ __forceinline__ void fwd_tile(const RenderParams& p, const TileCtx& t, float4* s_a,
                                         float2* s_b, float2* s_e, unsigned* s_key,
                                         float* s_col) {
  constexpr int NT = TILE * TILE;
  const int2 lp = pixel_of<TILE>(threadIdx.x);
  const int x = t.x0 + lp.x, y = t.y0 + lp.y;
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const bool in_img = x < t.W && y < t.H;
  const int len = t.range.y - t.range.x;
  float tq[KS<K>::A];
  PixelBlend<Chan<NC>::R> r;
  if (len <= NT) {
    stage_sorted<NT, NC>(p, t.range.x, len, (float)t.x0 + 0.5f * TILE,
                         (float)t.y0 + 0.5f * TILE, s_a, s_b, s_e, s_col, s_key);
    __syncthreads();
    const float4 R = block_rect<TILE>(t.x0, t.y0);
    if constexpr (K > 0) {
      int tk[K];
      int md;
      packed_keys<K>(len, px, py, in_img, R, s_a, s_b, s_e, tk, md);
      if (__any_sync(FULL_MASK, in_img && pk_ambiguous(tk[K - 1], md)))
        exact_winners<K>(p, len, px, py, in_img, R, s_a, s_b, s_e, tk);
      if (len >= K)
        blend_winners<K, NC, NT, true, false, false>(p, px, py, tk, in_img, s_a, s_b, s_col,
                                                     nullptr, r, nullptr);
      else
        blend_winners<K, NC, NT, false, false, false>(p, px, py, tk, in_img, s_a, s_b, s_col,
                                                      nullptr, r, nullptr);
    } else {
      float mdrop;
      culled_keys<K>(p, len, px, py, in_img, R, s_a, s_b, s_e, tq, mdrop);
      culled_blend<K, NC, NT>(p, len, px, py, in_img, R, tq, mdrop, s_a, s_b, s_e, s_col, r);
    }
  } else {
    select_keys<TILE, K, NT>(p, t.range, px, py, tq, s_a, s_b);
    blend_pass<TILE, K, NC, NT>(p, t.range, px, py, tq, r, s_a, s_b, s_col);
  }
  if (!in_img) return;
  const int n = nchan<NC>(p);
  const int64_t plane = (int64_t)t.H * t.W;
  const int64_t o = t.off + (int64_t)y * t.W + x;
#pragma unroll
  for (int c = 0; c < Chan<NC>::R; ++c)
    if (NC > 0 || c < n) p.img[c * plane + o] = r.cr[c];
}

template <int TILE, int K, int NC>
__global__ void __launch_bounds__(TILE * TILE, TILE == 16 ? 6 : 16) k_render_fwd(RenderParams p) {
  constexpr int NT = TILE * TILE;
  __shared__ float4 s_a[NT];
  __shared__ float2 s_b[NT];
  __shared__ float2 s_e[NT];
  __shared__ __align__(16) unsigned s_key[2 * NT];
  __shared__ __align__(16) float s_col[NT * col_stride(NC)];
  const int tile_id = blockIdx.y * p.tiles_x + blockIdx.x;  // grid (tiles_x, tiles_y)
  TileCtx t;
  t.range = p.range[tile_id];
  t.x0 = blockIdx.x * TILE;
  t.y0 = blockIdx.y * TILE;
  t.H = p.H;
  t.W = p.W;
  t.off = 0;
  t.inv_count = p.inv_count;
  t.loss_acc = nullptr;
  fwd_tile<TILE, K, NC>(p, t, s_a, s_b, s_e, s_key, s_col);
}

// Dynamic shared-memory layout of the adjoint kernel (in 4-byte words), for
// NT pixels, n channels and CH Gaussians per stage (64 <= CH <= NT).
struct BwdSmem {
  int a, b, col, ps0, gh, slot_a, slot_b, win, coff, loss, scan, total;
};
__host__ __device__ inline BwdSmem bwd_smem(int NT, int n, int CH) {
  const int NWB = NT / 32;
  const int np = 5 + n;
  auto al4 = [](int v) { return (v + 3) & ~3; };
  BwdSmem L;
  int o = 0;
  L.a = o;      o += 4 * CH;              // float4 (mx, my, A00, B)
  L.b = o;      o += 2 * CH;              // float2 (A11, index)
  L.col = o;    o = al4(o + col_stride(n) * CH);  // staged colours (16-byte aligned)
  L.ps0 = o;    o += 4 * NT;              // float4 (px, py, q0, beta) per pixel
  L.gh = o;     o = al4(o + col_stride(n) * NT);  // per-pixel -g/(2Z) (16-byte aligned)
  // pass C per-candidate sums A_j; before them (ex, ey) of the staged
  // candidates, followed by pass B's winner masks of lanes 0-15 (NWB CH
  // words, later the first slots: they end inside slot_a and slot_b, 2 + NWB
  // <= 10 <= 2 np words per candidate as np >= 6 and CH <= NT) and, 16 words
  // on, those of lanes 16-31 (at most 18 CH + 16 words from slot_a in all:
  // inside slot_a, slot_b and win, at least 6 CH + 14 NT words; win is free
  // until pass C's table is written, after these masks are last read)
  L.slot_a = o; o = al4(o + np * CH);
  L.slot_b = o; o = al4(o + np * NT);     // pass C per-thread sums B_t; rank keys before
  // pass C's table of 16-bit (candidate, pixel) pairs (<= 16 NT entries);
  // the chunked path's (tau, cut-off) per pixel
  L.win = o;    o += 8 * NT;
  L.coff = o;   o += CH + 1;              // first pair of every candidate
  L.loss = o;   o += NWB;               // per-warp loss partials
  L.scan = o;   o += 34;                  // integer block-scan scratch
  L.total = o;
  return L;
}

// Converts a candidate's moment sums into parameter gradients and adds them.
// T = sum over its winning pixels of G*(dx, dy, dx^2, dx dy, dy^2) with
// G = dL/dq; Tc = sum of w * (-g/(2Z)) per channel. The geometry comes from
// the candidate's record: the conic (A00, B, A11), (t1, t2) and (cos, sin).
template <int NC>
__device__ __forceinline__ void emit_grad(const RenderParams& p, const TileCtx& t, int gid,
                                          float A00, float B, float A11, float t1, float t2,
                                          const float2& cs, const float (&T)[5],
                                          const float (&Tc)[Chan<NC>::R]) {
  constexpr int NCR = Chan<NC>::R;
  const int n = nchan<NC>(p);
  const float T1 = t1 * t1, T2 = t2 * t2;
  const float c2 = cs.x * cs.x, s2 = cs.y * cs.y, sc = cs.x * cs.y;
  // q = A00 dx^2 + B dx dy + A11 dy^2 with d = x - mu_px
  const float d_mx = -(2.0f * A00 * T[0] + B * T[1]);
  const float d_my = -(B * T[0] + 2.0f * A11 * T[1]);
  const float dT1 = T[2] * c2 + T[4] * s2 + 2.0f * T[3] * sc;
  const float dT2 = T[2] * s2 + T[4] * c2 - 2.0f * T[3] * sc;
  const float d_th = (T1 - T2) * (2.0f * sc * (T[4] - T[2]) + 2.0f * (c2 - s2) * T[3]);
  float v[5 + NCR];
  v[0] = d_mx * (float)t.W;
  v[1] = d_my * (float)t.H;
  v[2] = d_th;
  v[3] = 2.0f * t1 * dT1;
  v[4] = 2.0f * t2 * dT2;
#pragma unroll
  for (int c = 0; c < NCR; ++c) v[5 + c] = -2.0f * Tc[c];  // w g / Z
  float* gdst = p.grad + (int64_t)gid * (5 + n);
  // a fixed row of 4m (2m) floats on a 16 (8) byte aligned array takes
  // vector atomics (sm_90+); anything else one float at a time
  constexpr int NP = 5 + NCR;
  const uintptr_t al = reinterpret_cast<uintptr_t>(p.grad);
  if (NC > 0 && NP % 4 == 0 && (al & 15u) == 0) {
#pragma unroll
    for (int k = 0; k < NP; k += 4)
      atomicAdd(reinterpret_cast<float4*>(gdst + k), make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]));
  } else if (NC > 0 && NP % 2 == 0 && (al & 7u) == 0) {
#pragma unroll
    for (int k = 0; k < NP; k += 2)
      atomicAdd(reinterpret_cast<float2*>(gdst + k), make_float2(v[k], v[k + 1]));
  } else {
#pragma unroll
    for (int k = 0; k < NP; ++k)
      if (NC > 0 || k < 5 + n) atomicAdd(gdst + k, v[k]);
  }
}

// Exclusive scan of v over the CTA (NWB warps); total receives the sum. One
// barrier: every thread adds the totals of the warps before its own. The
// caller keeps scratch (NWB words) unwritten until a later barrier.
template <int NWB>
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
  int before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < NWB; ++w) {
    const int tw = scratch[w];
    before += w < warp ? tw : 0;
    all += tw;
  }
  total = all;
  return before + incl - v;
}

// floor(a / d) for 0 <= a < 2^22 and d >= 1, given inv = 1/d in float32: the
// float quotient is within one of the exact one, which the checks correct.
__device__ __forceinline__ int div_small(int a, int d, float inv) {
  int q = (int)((float)a * inv);
  if (q * d > a) --q;
  else if ((q + 1) * d <= a) ++q;
  return q;
}

// Pass C of the fast path. The winning (candidate, pixel) pairs, in
// (candidate, warp block) order, are first written out as a table of 16-bit
// entries (candidate << 8 | pixel) by a counting sort of the winner records
// (ew, in each pixel's registers): a scan over candidates of their
// per-half-warp counts (the popcounts of the half-warps' slot masks) gives
// every (candidate, half of a warp block) its first slot (both halves' as
// 16-bit fields of the lower half's mask word), and each pixel stores its own
// winners at that slot plus its rank (within a half, the order in which the
// lanes' mask ORs were served). The
// table is split into equal contiguous ranges, one per thread; a thread
// accumulates the candidates of its range in registers. A candidate's partial
// sums go to the candidate's slot A_j, written by the one thread whose range
// holds the candidate's first pair, or, for the candidate a range opens with
// when it began in an earlier range, to that thread's slot B_t. After a
// barrier, the thread of candidate j adds A_j and the B_t of the later
// threads its pairs reach, and turns the sums into parameter gradients.
// Needs at most NT * 16 pairs (K <= 16): s_win / s_pair hold 16 NT entries.
template <int TILE, int K, int NC, int CH, bool PACK>
__device__ __forceinline__ void flat_pass_c(const RenderParams& p, const TileCtx& t, int cnt,
                                            int nw, const WinRecs<KS<K>::A, PACK>& ew,
                                            const float4* s_a, const float2* s_b,
                                            const float* s_col, unsigned short* s_win,
                                            unsigned* s_cnt, const float4* s_ps0,
                                            const float* s_gh, float* s_slot_a, float* s_slot_b,
                                            int* s_coff, int* s_scan) {
  constexpr int NT = TILE * TILE;
  constexpr int NWB = NT / 32;
  constexpr int NCR = Chan<NC>::R;
  constexpr int A = KS<K>::A;
  const int n = nchan<NC>(p);
  constexpr int U = rec_upper(NWB, CH);
  static_assert(16 * NT < 65536, "first slots are 16-bit fields");
  const int tid = threadIdx.x;
  // candidate tid's counts per half of each warp block (words wb CH + tid and
  // U + wb CH + tid). Thread tid alone reads these words and then overwrites
  // the first (with the first slots), so the counts can be read again after
  // the scan.
  int tot = 0;
  if (tid < cnt) {
#pragma unroll
    for (int wb = 0; wb < NWB; ++wb)
      tot += __popc(s_cnt[wb * CH + tid]) + __popc(s_cnt[U + wb * CH + tid]);
  }
  int P;
  const int base = block_scan_int<NWB>(tid < cnt ? tot : 0, s_scan, P);
  if (tid < cnt) {
    int run = base;
#pragma unroll
    for (int wb = 0; wb < NWB; ++wb) {
      const int lo = __popc(s_cnt[wb * CH + tid]);
      const int hi = __popc(s_cnt[U + wb * CH + tid]);
      s_cnt[wb * CH + tid] = (unsigned)run | ((unsigned)(run + lo) << 16);
      run += lo + hi;
    }
    s_coff[tid] = base;
  }
  if (tid == 0) s_coff[cnt] = P;
  __syncthreads();
  unsigned short* s_pair = s_win;
  // first slots of (candidate, my warp block): my half's 16-bit field
  const unsigned* s_first = s_cnt + (tid >> 5) * CH;
  const unsigned half_sel = (tid & 16) ? 0x4432u : 0x4410u;  // high / low field, zero-extended
  auto put = [&](int k) {
    const unsigned rec = ew.get(k);
    const int j = (int)(rec >> 5);
    s_pair[__byte_perm(s_first[j], 0u, half_sel) + (rec & 31u)] = (unsigned short)((j << 8) | tid);
  };
  if (__all_sync(FULL_MASK, nw == A)) {
#pragma unroll
    for (int k = 0; k < A; ++k) put(k);
  } else {
#pragma unroll
    for (int k = 0; k < A; ++k)
      if (k < nw) put(k);
  }
  const int per = (P + NT - 1) / NT;  // pairs per thread
  const float inv_per = per > 0 ? 1.0f / (float)per : 0.0f;
  // the epilogue's per-candidate geometry, requested now so that it arrives
  // during the accumulation loop
  int egid = -1;
  float4 erb = make_float4(0.f, 0.f, 0.f, 0.f);
  float2 ecs = make_float2(0.f, 0.f);
  if (tid < cnt && s_coff[tid + 1] > s_coff[tid]) {
    egid = __float_as_int(s_b[tid].y);
    if ((unsigned)egid < (unsigned)p.N) {
      erb = p.rec[egid].b;
      ecs = p.trig[egid];
    }
  }
  __syncthreads();

  const int r0 = (int)threadIdx.x * per;
  const int r1 = min(P, r0 + per);
  if (r0 < r1) {
    int e = r0;
    unsigned ent = s_pair[e];
    int j = (int)(ent >> 8);
    const int j_first = j;
    const bool cont = s_coff[j] < r0;  // the first candidate began in an earlier range
    float4 a = s_a[j];
    float a11 = s_b[j].x;
    float cc[NCR];
    auto load_colour = [&](int jj) { staged_colours<CH, NC>(p, s_col, s_b, jj, cc); };
    load_colour(j);
    float T[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    float Tc[NCR];
#pragma unroll
    for (int c = 0; c < NCR; ++c) Tc[c] = 0.0f;
    auto flush = [&](int jj) {
      const bool to_b = cont && jj == j_first;
      float* dst = to_b ? s_slot_b + threadIdx.x : s_slot_a + jj;
      const int stride = to_b ? NT : CH;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        dst[k * stride] = T[k];
        T[k] = 0.0f;
      }
#pragma unroll
      for (int c = 0; c < NCR; ++c) {
        if (NC > 0 || c < n) dst[(5 + c) * stride] = Tc[c];
        Tc[c] = 0.0f;
      }
    };
    for (;;) {
      const int i = (int)(ent & 255u);
      const float4 s0 = s_ps0[i];  // (px, py, q0, beta)
      // the ranking key of pass A, recomputed bit for bit (same sequence)
      const float dx = __fsub_rn(s0.x, a.x);
      const float dy = __fsub_rn(s0.y, a.y);
      const float h = __fmaf_rn(a.w, dy, __fmul_rn(a.z, dx));
      const float q = __fmaf_rn(h, dx, __fmul_rn(__fmul_rn(a11, dy), dy));
      const float w = blend_weight(s0.z, q);
      float gh[NCR];
      pixel_gh<NC>(s_gh, i, n, NT, gh);
      float gd = -s0.w;
#pragma unroll
      for (int c = 0; c < NCR; ++c)
        if (NC > 0 || c < n) gd = fmaf(gh[c], cc[c], gd);
      const float Gq = w * gd;
      const float e1 = Gq * dx, e2 = Gq * dy;
      T[0] += e1;
      T[1] += e2;
      T[2] = fmaf(e1, dx, T[2]);
      T[3] = fmaf(e1, dy, T[3]);
      T[4] = fmaf(e2, dy, T[4]);
#pragma unroll
      for (int c = 0; c < NCR; ++c)
        if (NC > 0 || c < n) Tc[c] = fmaf(w, gh[c], Tc[c]);
      if (++e >= r1) break;
      ent = s_pair[e];
      const int nj = (int)(ent >> 8);
      if (nj != j) {
        flush(j);
        j = nj;
        a = s_a[j];
        a11 = s_b[j].x;
        load_colour(j);
      }
    }
    flush(j);
  }
  __syncthreads();
  if ((int)threadIdx.x < cnt) {
    const int j = threadIdx.x;
    const int e0 = s_coff[j], e1 = s_coff[j + 1];
    if (e1 > e0) {
      float T[5];
      float Tc[NCR];
#pragma unroll
      for (int k = 0; k < 5; ++k) T[k] = s_slot_a[k * CH + j];
#pragma unroll
      for (int c = 0; c < NCR; ++c)
        Tc[c] = (NC > 0 || c < n) ? s_slot_a[(5 + c) * CH + j] : 0.0f;
      const int th1 = div_small(e1 - 1, per, inv_per);
      for (int th = div_small(e0, per, inv_per) + 1; th <= th1; ++th) {
#pragma unroll
        for (int k = 0; k < 5; ++k) T[k] += s_slot_b[k * NT + th];
#pragma unroll
        for (int c = 0; c < NCR; ++c)
          if (NC > 0 || c < n) Tc[c] += s_slot_b[(5 + c) * NT + th];
      }
      if ((unsigned)egid < (unsigned)p.N)
        emit_grad<NC>(p, t, egid, s_a[j].z, s_a[j].w, erb.x, erb.z, erb.w, ecs, T, Tc);
    }
  }
}

// Pass C of the chunked path: threads own (candidate, group of pixels) and
// re-test membership from each pixel's (tau, tie cut-off).
template <int TILE, int NC, int CH>
__device__ __forceinline__ void chunked_pass_c(const RenderParams& p, const TileCtx& t,
                                               const float4* s_ps0, const float2* s_ps1,
                                               const float* s_gh, float* s_part) {
  constexpr int NT = TILE * TILE;
  constexpr int NCR = Chan<NC>::R;
  const int n = nchan<NC>(p);
  const int np = 5 + n;
  const int2 range = t.range;
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
        const bool win = q < s1.x || (q == s1.x && gid <= __float_as_int(s1.y));
        if (win) {
          const float w = blend_weight(s0.z, q);
          float gd = -s0.w;
#pragma unroll
          for (int c = 0; c < NCR; ++c)
            if (NC > 0 || c < n) gd = fmaf(s_gh[gh_at<NC>(i, c, NT)], cc[c], gd);
          const float Gq = w * gd;
          const float e1 = Gq * dx, e2 = Gq * dy;
          S1 += e1;
          S2 += e2;
          S11 = fmaf(e1, dx, S11);
          S12 = fmaf(e1, dy, S12);
          S22 = fmaf(e2, dy, S22);
#pragma unroll
          for (int c = 0; c < NCR; ++c)
            if (NC > 0 || c < n) Sc[c] = fmaf(w, s_gh[gh_at<NC>(i, c, NT)], Sc[c]);
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
      float Tc[NCR];
#pragma unroll
      for (int c = 0; c < NCR; ++c) Tc[c] = 0.0f;
      for (int g2 = 0; g2 < G; ++g2) {
        const float* src = s_part + (g2 * C + j) * np;
#pragma unroll
        for (int k = 0; k < 5; ++k) T[k] += src[k];
#pragma unroll
        for (int c = 0; c < NCR; ++c)
          if (NC > 0 || c < n) Tc[c] += src[5 + c];
      }
      const GRec rc = p.rec[gid];
      emit_grad<NC>(p, t, gid, rc.a.z, rc.a.w, rc.b.x, rc.b.z, rc.b.w, p.trig[gid], T, Tc);
    }
    __syncthreads();
  }
}

// Adjoint of one tile: passes A and B per pixel, then pass C per candidate.
// PACK: winner records two per register (the persistent batched kernel).
template <int TILE, int K, int NC, int CH, bool PACK>
__device__ __forceinline__ void bwd_tile(const RenderParams& p, const TileCtx& t, float* smem) {
  constexpr int NT = TILE * TILE;
  constexpr int NCR = Chan<NC>::R;
  const int n = nchan<NC>(p);
  const BwdSmem SL = bwd_smem(NT, n, CH);
  float4* s_a = reinterpret_cast<float4*>(smem + SL.a);
  float2* s_b = reinterpret_cast<float2*>(smem + SL.b);
  float* s_col = smem + SL.col;
  float4* s_ps0 = reinterpret_cast<float4*>(smem + SL.ps0);
  float* s_gh = smem + SL.gh;
  float* s_slot_a = smem + SL.slot_a;
  float* s_slot_b = smem + SL.slot_b;
  float2* s_e = reinterpret_cast<float2*>(s_slot_a);      // until pass C
  unsigned* s_key = reinterpret_cast<unsigned*>(s_slot_b);  // while staging
  // pass C's pair table (fast path)
  unsigned short* s_win = reinterpret_cast<unsigned short*>(smem + SL.win);
  float2* s_ps1 = reinterpret_cast<float2*>(smem + SL.win);  // chunked path only
  // per (warp block, candidate) counts of pass B, then first pair slots; after
  // (ex, ey), in pass C's sums' storage, which is free until its loop
  unsigned* s_cnt = reinterpret_cast<unsigned*>(s_slot_a) + 2 * CH;
  float* s_loss = smem + SL.loss;

  const int2 lp = pixel_of<TILE>(threadIdx.x);
  const int x = t.x0 + lp.x, y = t.y0 + lp.y;
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const bool in_img = x < t.W && y < t.H;
  const int64_t plane = (int64_t)t.H * t.W;
  const int64_t o = t.off + (int64_t)y * t.W + x;
  // the pixel's target (or upstream gradient) is read now so that its HBM
  // latency hides behind passes A and B (fixed channel counts only)
  const float* src = p.grad_img ? p.grad_img : p.target;
  constexpr int NUP = NC > 0 ? NC : 1;
  float up[NUP];
#pragma unroll
  for (int c = 0; c < NUP; ++c) up[c] = (NC > 0 && in_img) ? src[c * plane + o] : 0.0f;

  // ---- passes A and B: per-pixel forward values and upstream gradient
  const int len = t.range.y - t.range.x;
  const bool fast = len <= CH;
  float tq[KS<K>::A];
  WinRecs<KS<K>::A, PACK> ew;  // fast path: this pixel's winner records
  PixelBlend<NCR> r;
  __syncthreads();  // the previous tile of a persistent CTA is done with smem
  if (fast) {
    stage_sorted<CH, NC>(p, t.range.x, len, (float)t.x0 + 0.5f * TILE,
                         (float)t.y0 + 0.5f * TILE, s_a, s_b, s_e, s_col, s_key);
    __syncthreads();
    const float4 R = block_rect<TILE>(t.x0, t.y0);
    if constexpr (K > 0) {
      constexpr int U = rec_upper(NT / 32, CH);
      // the masks start 2 CH words into slot_a (np = 5 + n >= 6 words per
      // candidate there, per pixel in slot_b; win holds 8 NT words): the lower
      // half's end inside slot_a and slot_b, the upper half's inside win
      static_assert(2 * CH + (NT / 32) * CH <= 6 * CH + 6 * NT, "lower masks outgrow the sums");
      static_assert(2 * CH + U + (NT / 32) * CH <= 6 * CH + 14 * NT, "upper masks outgrow win");
      unsigned* cnt_w = s_cnt + (threadIdx.x >> 5) * CH;  // this warp's winner masks
      for (int j = threadIdx.x & 31; j < len; j += 32) {
        cnt_w[j] = 0u;
        cnt_w[U + j] = 0u;
      }
      cnt_w += (threadIdx.x & 16) ? U : 0;  // this lane's half's
      int tk[K];
      int md;
      packed_keys<K>(len, px, py, in_img, R, s_a, s_b, s_e, tk, md);
      if (__any_sync(FULL_MASK, in_img && pk_ambiguous(tk[K - 1], md)))
        exact_winners<K>(p, len, px, py, in_img, R, s_a, s_b, s_e, tk);
      if (len >= K)
        blend_winners<K, NC, CH, true, true, PACK>(p, px, py, tk, in_img, s_a, s_b, s_col,
                                                   cnt_w, r, &ew);
      else
        blend_winners<K, NC, CH, false, true, PACK>(p, px, py, tk, in_img, s_a, s_b, s_col,
                                                    cnt_w, r, &ew);
      // winners in ascending packed order (PK_NONE entries come last): pass C
      // reads the first nw records
      r.nw = 0;
#pragma unroll
      for (int k = 0; k < K; ++k) r.nw += (in_img && tk[k] != PK_NONE) ? 1 : 0;
    } else {
      float mdrop;
      culled_keys<K>(p, len, px, py, in_img, R, s_a, s_b, s_e, tq, mdrop);
      culled_blend<K, NC, CH>(p, len, px, py, in_img, R, tq, mdrop, s_a, s_b, s_e, s_col, r);
    }
  } else {
    select_keys<TILE, K, CH>(p, t.range, px, py, tq, s_a, s_b);
    blend_pass<TILE, K, NC, CH>(p, t.range, px, py, tq, r, s_a, s_b, s_col);
  }

  // per-pixel factors gh_c = -g_c / (2 Z), so that dL/dq_k = w_k (sum_c
  // gh_c c_k,c - beta) with beta = sum_c gh_c c_r,c; g_c is the upstream
  // gradient, or sign(c_r,c - c_t,c) / (H W n) for the L1 loss. Pixels
  // without weight (no winners) get none, but their |c_r - c_t| (c_r = 0)
  // still counts in the loss.
  const bool live = in_img && r.Z > 0.0f;
  const float hz = live ? -0.5f * r.iz : 0.0f;
  const float hl = hz * t.inv_count;
  float loss = 0.0f;
  float beta = 0.0f;
  float gh[NCR];
#pragma unroll
  for (int c = 0; c < NCR; ++c) {
    gh[c] = 0.0f;
    if (NC > 0 || c < n) {
      const float u = NC > 0 ? up[NC > 0 ? c : 0] : (in_img ? src[c * plane + o] : 0.0f);
      if (p.grad_img) {
        gh[c] = hz * u;
      } else {
        const float d = r.cr[c] - u;
        loss += fabsf(d);
        gh[c] = d > 0.0f ? hl : (d < 0.0f ? -hl : 0.0f);
      }
      if (p.normalize) beta = fmaf(gh[c], r.cr[c], beta);
    }
  }
  if (!in_img) loss = 0.0f;
  if (NC == 3 || NC == 4) {
    reinterpret_cast<float4*>(s_gh)[threadIdx.x] =
        make_float4(gh[0], gh[1], gh[2], NC == 4 ? gh[NC == 4 ? 3 : 0] : 0.0f);
  } else {
#pragma unroll
    for (int c = 0; c < NCR; ++c)
      if (NC > 0 || c < n) s_gh[gh_at<NC>(threadIdx.x, c, NT)] = gh[c];
  }
  s_ps0[threadIdx.x] = make_float4(px, py, r.q0, beta);
  // the chunked pass C (long lists; K = 0, where every candidate wins) re-tests
  // membership from (tau, cut-off)
  const bool flat = fast && K > 0;
  if (!flat) s_ps1[threadIdx.x] = make_float2(live ? r.tau : -F_INF, __int_as_float(r.gcut));
  // per-warp and per-tile partial sums (at most 32 and 256 n terms |d| <= 1)
  // in float32, one float64 atomic per tile (FP64 arithmetic is slow here)
  if (!p.grad_img) {
    const float l = warp_sum<float>(loss);
    if ((threadIdx.x & 31) == 0) s_loss[threadIdx.x >> 5] = l;
  }
  __syncthreads();
  // the tile's loss is added after pass C, away from its barriers
  float tile_loss = 0.0f;
  if (!p.grad_img && threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) tile_loss += s_loss[i];
  }

  // ---- pass C: candidate-major accumulation of the adjoint
  if (flat) {
    flat_pass_c<TILE, K, NC, CH, PACK>(p, t, len, r.nw, ew, s_a, s_b, s_col, s_win, s_cnt, s_ps0, s_gh,
                                 s_slot_a, s_slot_b, reinterpret_cast<int*>(smem + SL.coff),
                                 reinterpret_cast<int*>(smem + SL.scan));
  } else {
    chunked_pass_c<TILE, NC, CH>(p, t, s_ps0, s_ps1, s_gh, s_slot_a);
  }
  if (tile_loss != 0.0f) atomicAdd(t.loss_acc, (double)tile_loss);
}

template <int TILE, int K, int NC>
__global__ void __launch_bounds__(TILE * TILE, TILE == 16 ? 5 : 16) k_render_bwd(RenderParams p) {
  extern __shared__ __align__(16) float smem[];
  const int tile_id = blockIdx.y * p.tiles_x + blockIdx.x;  // grid (tiles_x, tiles_y)
  TileCtx t;
  t.range = p.range[tile_id];
  t.x0 = blockIdx.x * TILE;
  t.y0 = blockIdx.y * TILE;
  t.H = p.H;
  t.W = p.W;
  t.off = 0;
  t.inv_count = p.inv_count;
  t.loss_acc = &p.status->loss_sum;
  bwd_tile<TILE, K, NC, TILE * TILE, false>(p, t, smem);  // the whole tile's pixels per stage
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
__global__ void __launch_bounds__(TILE * TILE, 5) k_render_bwd_batch(RenderParams p,
                                                                  BatchTables bt) {
  extern __shared__ __align__(16) float smem[];
  // the current tile's context lives in shared memory and is read where it
  // is used (in registers it would hold about a dozen through the tile)
  __shared__ TileCtx s_tc;
  __shared__ int s_item;
  int it = blockIdx.x;
  for (;;) {
    __syncthreads();  // every thread is done with the previous tile's context
    if (threadIdx.x == 0) {
      if (bt.order == 0) it = (int)atomicAdd(bt.work, 1u);
      s_item = it;
      if (it < bt.T) {
        const int b = image_of_tile(bt, it);
        const int4 dm = bt.dims[b];
        const int local = it - bt.tile_off[b];
        s_tc.range = p.range[it];
        s_tc.x0 = (local % dm.z) * TILE;
        s_tc.y0 = (local / dm.z) * TILE;
        s_tc.H = dm.x;
        s_tc.W = dm.y;
        s_tc.off = bt.pix_off[b];
        s_tc.inv_count = 1.0f / ((float)dm.x * (float)dm.y * (float)nchan<NC>(p));
        s_tc.loss_acc = bt.loss + b;
      }
    }
    __syncthreads();
    it = s_item;
    if (it >= bt.T) break;
    bwd_tile<TILE, K, NC, CH, true>(p, s_tc, smem);
    if (bt.order != 0) it += gridDim.x;
  }
}

// Forward render of the concatenated tiles of many images, one CTA per tile.
template <int TILE, int K, int NC>
__global__ void __launch_bounds__(TILE * TILE, 6) k_render_fwd_batch(RenderParams p,
                                                                    BatchTables bt) {
  constexpr int NT = TILE * TILE;
  __shared__ float4 s_a[NT];
  __shared__ float2 s_b[NT];
  __shared__ float2 s_e[NT];
  __shared__ __align__(16) unsigned s_key[2 * NT];
  __shared__ __align__(16) float s_col[NT * col_stride(NC)];
  const int it = blockIdx.x;
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
  t.inv_count = 0.0f;
  t.loss_acc = nullptr;
  fwd_tile<TILE, K, NC>(p, t, s_a, s_b, s_e, s_key, s_col);
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
        float4 a;
        float a11;
        load_geom(p, id, a, a11);
        q0 = fminf(q0, rank_key(px, py, a.x, a.y, a.z, a.w, a11));
      }
    }
    for (int j = range.x; j < range.y; ++j) {
      const int id = p.list[j];
      if ((unsigned)id >= (unsigned)p.N) continue;
      float4 a;
      float a11;
      load_geom(p, id, a, a11);
      const float w = blend_weight(q0, rank_key(px, py, a.x, a.y, a.z, a.w, a11));
      Z += w;
#pragma unroll
      for (int c = 0; c < NCR; ++c)
        if (NC > 0 || c < n) cr[c] = fmaf(w, load_colour(p, id, c, n), cr[c]);
    }
  } else {
    float tq[KS<K>::A];
    int tp[KS<K>::A];
#pragma unroll
    for (int k = 0; k < KS<K>::A; ++k) {
      tq[k] = F_INF;
      tp[k] = -1;
    }
    // DU candidates per round: their index and record loads are in flight
    // together (the walk is bound by dependent L2 latencies)
    constexpr int DU = 4;
    for (int j0 = range.x; j0 < range.y; j0 += DU) {
      int id[DU];
      float q[DU];
#pragma unroll
      for (int u = 0; u < DU; ++u) id[u] = j0 + u < range.y ? p.list[j0 + u] : -1;
#pragma unroll
      for (int u = 0; u < DU; ++u) {
        const bool ok = (unsigned)id[u] < (unsigned)p.N;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        float a11 = 0.0f;
        if (ok) load_geom(p, id[u], a, a11);
        q[u] = ok ? rank_key(px, py, a.x, a.y, a.z, a.w, a11) : F_INF;
        if (!ok) id[u] = -1;
      }
#pragma unroll
      for (int u = 0; u < DU; ++u) {
        if (id[u] < 0) continue;
        if (q[u] < tq[KS<K>::A - 1] || (q[u] == tq[KS<K>::A - 1] && id[u] < tp[KS<K>::A - 1]))
          topk_insert<KS<K>::A>(tq, tp, q[u], id[u]);
      }
    }
    const float q0 = p.normalize ? tq[0] : 0.0f;
#pragma unroll
    for (int k = 0; k < KS<K>::A; ++k) {
      if (tp[k] >= 0) {
        const float w = blend_weight(q0, tq[k]);
        Z += w;
#pragma unroll
        for (int c = 0; c < NCR; ++c)
          if (NC > 0 || c < n) cr[c] = fmaf(w, load_colour(p, tp[k], c, n), cr[c]);
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
