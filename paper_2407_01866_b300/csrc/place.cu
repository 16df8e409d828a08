// Content-adaptive placement (Sec. 3.3): Eq. 6 draws initial Gaussian
// positions from image-gradient magnitudes mixed with a uniform share;
// Eq. 7 draws added Gaussians from the per-pixel error of a rendering.
//
// Both draws are decided exactly (the sequence is fixed in include/imgs.h):
//   weight    binary32: gradient s += gx*gx, s += gy*gy over channels (central
//             differences inside, one-sided at the borders), sqrt; or the sum
//             of the channels' |c_r - c_t|
//   integer   floor(min(w, 4096) * 2^24), non-finite -> 0
//   cdf       exclusive prefix sum of the integers (64-bit)
//   draw      53-bit input integers r1, r2: the uniform part (r1 < floor(lambda
//             2^53), or all weights zero) takes pixel floor(r2 HW / 2^53); the
//             weighted part the last pixel whose prefix is <= floor(r2 total / 2^53)
#include "internal.h"

namespace igs {

namespace {

constexpr float W_CAP = 4096.0f;
constexpr float W_SCALE = 16777216.0f;  // 2^24
constexpr unsigned long long R_MASK = (1ull << 53) - 1ull;

__device__ __forceinline__ unsigned long long quantise(float w) {
  const float c = isfinite(w) ? fminf(w, W_CAP) : 0.0f;
  return (unsigned long long)(c * W_SCALE);  // exact scaling; truncation = floor
}

// Binary32 difference of channel plane I [H][W] at (y, x) along x or y.
__device__ __forceinline__ float plane_diff(const float* I, int H, int W, int y, int x, bool along_x) {
  const int L = along_x ? W : H;
  const int k = along_x ? x : y;
  if (L == 1) return 0.0f;
  auto at = [&](int kk) { return along_x ? I[(int64_t)y * W + kk] : I[(int64_t)kk * W + x]; };
  if (k == 0) return __fsub_rn(at(1), at(0));
  if (k == L - 1) return __fsub_rn(at(L - 1), at(L - 2));
  return __fmul_rn(__fsub_rn(at(k + 1), at(k - 1)), 0.5f);
}

__global__ void __launch_bounds__(256) k_grad_weight(const float* target, int H, int W, int n,
                                                     unsigned long long* w) {
  const int64_t HW = (int64_t)H * W;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < HW;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(p / W), x = (int)(p % W);
    float s = 0.0f;
    for (int c = 0; c < n; ++c) {
      const float* I = target + (int64_t)c * HW;
      const float gx = plane_diff(I, H, W, y, x, true);
      const float gy = plane_diff(I, H, W, y, x, false);
      s = __fadd_rn(s, __fmul_rn(gx, gx));
      s = __fadd_rn(s, __fmul_rn(gy, gy));
    }
    w[p] = quantise(__fsqrt_rn(s));
  }
}

__global__ void __launch_bounds__(256) k_error_weight(const float* render, const float* target,
                                                      int64_t HW, int n, unsigned long long* w) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < HW;
       p += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int c = 0; c < n; ++c)
      s = __fadd_rn(s, fabsf(__fsub_rn(render[c * HW + p], target[c * HW + p])));
    w[p] = quantise(s);
  }
}

// New Gaussians at drawn pixels: rows [row0, row0 + count) of params (and
// zero rows of the optional grad / Adam moments).
__global__ void __launch_bounds__(256) k_place(const unsigned long long* excl,
                                               const unsigned long long* total_p, int H, int W,
                                               int n, const float* target,
                                               const unsigned long long* rnd, int64_t count,
                                               unsigned long long thr, float* params,
                                               int64_t row0, float* grad, float* m, float* v) {
  const int64_t HW = (int64_t)H * W;
  const unsigned long long total = *total_p;
  const int np = 5 + n;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
       k += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long r1 = rnd[2 * k] & R_MASK, r2 = rnd[2 * k + 1] & R_MASK;
    int64_t p;
    if (r1 < thr || total == 0) {
      p = (int64_t)__umul64hi(r2 << 11, (unsigned long long)HW);
    } else {
      const unsigned long long t = __umul64hi(r2 << 11, total);
      int64_t lo = 0, hi = HW - 1;  // the last pixel whose exclusive prefix is <= t
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (excl[mid] <= t) lo = mid; else hi = mid - 1;
      }
      p = lo;
    }
    const int y = (int)(p / W), x = (int)(p % W);
    float* row = params + (row0 + k) * np;
    row[0] = __fdiv_rn(__fadd_rn((float)x, 0.5f), (float)W);
    row[1] = __fdiv_rn(__fadd_rn((float)y, 0.5f), (float)H);
    row[2] = 0.0f;
    row[3] = row[4] = 0.2f;  // inverse of the 5 px initial scale (Sec. 4.1)
    for (int c = 0; c < n; ++c) row[5 + c] = target[c * HW + p];
    if (grad) {
      for (int c = 0; c < np; ++c) {
        grad[(row0 + k) * np + c] = 0.0f;
        m[(row0 + k) * np + c] = 0.0f;
        v[(row0 + k) * np + c] = 0.0f;
      }
    }
  }
}

unsigned grid_for(int64_t items) {
  const int64_t b = (items + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 148 * 16 ? 148 * 16 : b));
}

}  // namespace

PlaceLayout place_layout(int64_t HW) {
  PlaceLayout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = (o + bytes + 255) & ~(size_t)255;
    return at;
  };
  L.weights = take(sizeof(unsigned long long) * (size_t)HW);
  L.excl = take(sizeof(unsigned long long) * (size_t)HW);
  L.part = take(sizeof(unsigned long long) * (size_t)((HW + SCAN_ITEMS - 1) / SCAN_ITEMS + 1));
  L.total = take(sizeof(unsigned long long));
  L.bytes = o;
  return L;
}

cudaError_t launch_place(const float* target, const float* render, int H, int W, int n,
                         const unsigned long long* rnd, int64_t count, double lambda,
                         float* params, int64_t row0, float* grad, float* m, float* v,
                         char* ws, cudaStream_t s) {
  const int64_t HW = (int64_t)H * W;
  const PlaceLayout L = place_layout(HW);
  unsigned long long* w = reinterpret_cast<unsigned long long*>(ws + L.weights);
  unsigned long long* excl = reinterpret_cast<unsigned long long*>(ws + L.excl);
  unsigned long long* part = reinterpret_cast<unsigned long long*>(ws + L.part);
  unsigned long long* total = reinterpret_cast<unsigned long long*>(ws + L.total);
  if (render)
    k_error_weight<<<grid_for(HW), 256, 0, s>>>(render, target, HW, n, w);
  else
    k_grad_weight<<<grid_for(HW), 256, 0, s>>>(target, H, W, n, w);
  cudaError_t e = launch_scan_u64(w, excl, HW, part, total, s);
  if (e != cudaSuccess) return e;
  if (count == 0) return cudaGetLastError();
  // branch threshold floor(lambda 2^53), exact in double
  const unsigned long long thr = (unsigned long long)(lambda * 9007199254740992.0);
  k_place<<<grid_for(count), 256, 0, s>>>(excl, total, H, W, n, target, rnd, count, thr, params,
                                          row0, grad, m, v);
  return cudaGetLastError();
}

}  // namespace igs
