// Image-space fitting loss L1 + w (1 - SSIM) (Sec. 3.3 and Sec. 4.1, which
// fits against L1 + 0.1 L_SSIM) and its gradient with respect to the
// rendering, for the fit steps that include the SSIM term.
//
// SSIM is computed per channel with an 11 x 11 Gaussian window (sigma 1.5,
// normalised, zero-padded "same" correlation) and C1 = 0.01^2, C2 = 0.03^2;
// L_SSIM = 1 - mean SSIM over channels and pixels. Four passes, float32;
// the horizontal ones stage row segments in shared memory, the vertical ones
// take one thread per (channel, column, strip of RS rows):
//   h5  horizontal window sums of x, y, x^2, y^2, x y
//   v5  vertical sums -> mu_x, mu_y, E[x^2], E[y^2], E[xy] -> SSIM and its
//       partials G1 = dS/dmu_x, G2 = dS/dE[x^2], G3 = dS/dE[xy]; the loss sum
//       |x - y| + w (1 - S) is reduced into a double
//   h3  horizontal window sums of G1..G3
//   v3  vertical sums, then dL/dx = sign(x - y)/M - (w/M)(bG1 + 2x bG2 + y bG3)
// (the window is symmetric: the transposed correlation is the same one).
#include <cmath>

#include "internal.h"

namespace igs {

namespace {

constexpr int WR = 5;  // window radius
constexpr float C1 = 1e-4f, C2 = 9e-4f;

struct Win {
  float g[2 * WR + 1];
};

// Horizontal passes: a CTA takes a row segment of HSEG outputs, stages it
// with its halo in shared memory once, and every thread sums its taps there.
constexpr int HSEG = 256;

__global__ void __launch_bounds__(HSEG) k_h5(const float* x, const float* y, int64_t rows,
                                             int W, Win w, int64_t total, float* out) {
  __shared__ float sx[HSEG + 2 * WR], sy[HSEG + 2 * WR];
  const int segs = (W + HSEG - 1) / HSEG;
  for (int64_t b = blockIdx.x; b < rows * segs; b += gridDim.x) {
    const int64_t row = (b / segs) * W;  // start of the (channel, row) in the planes
    const int x0 = (int)(b % segs) * HSEG;
    __syncthreads();
    for (int k = threadIdx.x; k < HSEG + 2 * WR; k += blockDim.x) {
      const int xs = x0 - WR + k;
      const bool in = xs >= 0 && xs < W;
      sx[k] = in ? x[row + xs] : 0.0f;
      sy[k] = in ? y[row + xs] : 0.0f;
    }
    __syncthreads();
    const int xx = x0 + threadIdx.x;
    if (xx >= W) continue;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
#pragma unroll
    for (int i = 0; i <= 2 * WR; ++i) {
      const float a = sx[threadIdx.x + i], c = sy[threadIdx.x + i], g = w.g[i];
      s0 = fmaf(g, a, s0);
      s1 = fmaf(g, c, s1);
      s2 = fmaf(g, a * a, s2);
      s3 = fmaf(g, c * c, s3);
      s4 = fmaf(g, a * c, s4);
    }
    const int64_t p = row + xx;
    out[p] = s0;
    out[total + p] = s1;
    out[2 * total + p] = s2;
    out[3 * total + p] = s3;
    out[4 * total + p] = s4;
  }
}

// Vertical passes: a thread covers RS consecutive rows of one column and
// slides down them, so every loaded row feeds up to 2 WR + 1 outputs.
constexpr int RS = 8;

__global__ void __launch_bounds__(256) k_v5(const float* hm, const float* x, const float* y,
                                            int64_t total, int n, int H, int W, Win w,
                                            float w_ssim, float* G, double* acc) {
  const int64_t HW = (int64_t)H * W;
  const int strips = (H + RS - 1) / RS;
  const int64_t items = (int64_t)n * strips * W;
  double part = 0.0;
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int xx = (int)(it % W);
    const int64_t cs = it / W;
    const int y0 = (int)(cs % strips) * RS;
    const int64_t cbase = (cs / strips) * HW;
    float m[5][RS];
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
      for (int j = 0; j < RS; ++j) m[k][j] = 0.0f;
#pragma unroll
    for (int rr = 0; rr < RS + 2 * WR; ++rr) {
      const int r = y0 - WR + rr;
      if (r < 0 || r >= H) continue;
      const int64_t o = cbase + (int64_t)r * W + xx;
      float v[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) v[k] = hm[k * total + o];
#pragma unroll
      for (int j = 0; j < RS; ++j) {
        const int i = rr - WR - j;  // tap offset of row r for output row y0 + j
        if (i < -WR || i > WR) continue;
#pragma unroll
        for (int k = 0; k < 5; ++k) m[k][j] = fmaf(w.g[i + WR], v[k], m[k][j]);
      }
    }
#pragma unroll
    for (int j = 0; j < RS; ++j) {
      if (y0 + j >= H) break;
      const int64_t p = cbase + (int64_t)(y0 + j) * W + xx;
      const float mx = m[0][j], my = m[1][j];
      const float vx = m[2][j] - mx * mx, vy = m[3][j] - my * my, cxy = m[4][j] - mx * my;
      const float A1 = 2.f * mx * my + C1, A2 = 2.f * cxy + C2;
      const float B1 = mx * mx + my * my + C1, B2 = vx + vy + C2;
      const float iB = 1.f / (B1 * B2);
      const float S = A1 * A2 * iB;
      const float dS_dvx = -S / B2;
      const float dS_dcxy = 2.f * A1 * iB;
      const float dmx = 2.f * my * A2 * iB - S * 2.f * mx / B1;
      G[p] = dmx - 2.f * mx * dS_dvx - my * dS_dcxy;
      G[total + p] = dS_dvx;
      G[2 * total + p] = dS_dcxy;
      part += (double)fabsf(x[p] - y[p]) + (double)w_ssim * (1.0 - (double)S);
    }
  }
  part = warp_sum<double>(part);
  if ((threadIdx.x & 31) == 0 && part != 0.0) atomicAdd(acc, part);
}

__global__ void __launch_bounds__(HSEG) k_h3(const float* G, int64_t rows, int W, Win w,
                                             int64_t total, float* out) {
  __shared__ float sg[3][HSEG + 2 * WR];
  const int segs = (W + HSEG - 1) / HSEG;
  for (int64_t b = blockIdx.x; b < rows * segs; b += gridDim.x) {
    const int64_t row = (b / segs) * W;
    const int x0 = (int)(b % segs) * HSEG;
    __syncthreads();
    for (int k = threadIdx.x; k < HSEG + 2 * WR; k += blockDim.x) {
      const int xs = x0 - WR + k;
      const bool in = xs >= 0 && xs < W;
#pragma unroll
      for (int m = 0; m < 3; ++m) sg[m][k] = in ? G[m * total + row + xs] : 0.0f;
    }
    __syncthreads();
    const int xx = x0 + threadIdx.x;
    if (xx >= W) continue;
    float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i <= 2 * WR; ++i) {
#pragma unroll
      for (int m = 0; m < 3; ++m) acc[m] = fmaf(w.g[i], sg[m][threadIdx.x + i], acc[m]);
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) out[m * total + row + xx] = acc[m];
  }
}

__global__ void __launch_bounds__(256) k_v3(const float* hg, const float* x, const float* y,
                                            int64_t total, int n, int H, int W, Win w,
                                            float w_ssim, float inv_m, float* grad) {
  const int64_t HW = (int64_t)H * W;
  const int strips = (H + RS - 1) / RS;
  const int64_t items = (int64_t)n * strips * W;
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int xx = (int)(it % W);
    const int64_t cs = it / W;
    const int y0 = (int)(cs % strips) * RS;
    const int64_t cbase = (cs / strips) * HW;
    float b[3][RS];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int j = 0; j < RS; ++j) b[k][j] = 0.0f;
#pragma unroll
    for (int rr = 0; rr < RS + 2 * WR; ++rr) {
      const int r = y0 - WR + rr;
      if (r < 0 || r >= H) continue;
      const int64_t o = cbase + (int64_t)r * W + xx;
      float v[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) v[k] = hg[k * total + o];
#pragma unroll
      for (int j = 0; j < RS; ++j) {
        const int i = rr - WR - j;
        if (i < -WR || i > WR) continue;
#pragma unroll
        for (int k = 0; k < 3; ++k) b[k][j] = fmaf(w.g[i + WR], v[k], b[k][j]);
      }
    }
#pragma unroll
    for (int j = 0; j < RS; ++j) {
      if (y0 + j >= H) break;
      const int64_t p = cbase + (int64_t)(y0 + j) * W + xx;
      const float xv = x[p], yv = y[p];
      const float d = xv - yv;
      const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
      grad[p] = sgn * inv_m - w_ssim * inv_m * (b[0][j] + 2.f * xv * b[1][j] + yv * b[2][j]);
    }
  }
}

// L1 only: gradient and loss sum.
__global__ void __launch_bounds__(256) k_l1(const float* x, const float* y, int64_t total,
                                            float inv_m, float* grad, double* acc) {
  double part = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const float d = x[p] - y[p];
    grad[p] = (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) * inv_m;
    part += (double)fabsf(d);
  }
  part = warp_sum<double>(part);
  if ((threadIdx.x & 31) == 0 && part != 0.0) atomicAdd(acc, part);
}

__global__ void k_loss_out(const double* acc, float inv_m, float* out) {
  if (threadIdx.x == 0) *out = (float)(*acc * (double)inv_m);
}

unsigned grid_for(int64_t items) {
  const int64_t b = (items + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 148 * 16 ? 148 * 16 : b));
}

Win window() {
  Win w;
  double g[2 * WR + 1], s = 0.0;
  for (int i = -WR; i <= WR; ++i) {
    g[i + WR] = std::exp(-(double)(i * i) / (2.0 * 1.5 * 1.5));
    s += g[i + WR];
  }
  for (int i = 0; i < 2 * WR + 1; ++i) w.g[i] = (float)(g[i] / s);
  return w;
}

}  // namespace

size_t image_loss_scratch_bytes(int n, int H, int W) {
  const size_t total = (size_t)n * H * W;
  return 256 + ((sizeof(float) * 8 * total + 255) & ~(size_t)255);
}

cudaError_t launch_image_loss(const float* x, const float* y, int n, int H, int W,
                              float w_ssim, float* grad, double* acc, float* loss_out,
                              char* scratch, cudaStream_t s) {
  const int64_t total = (int64_t)n * H * W;
  if (total == 0) return cudaSuccess;
  const float inv_m = (float)(1.0 / (double)total);
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  if (w_ssim == 0.0f) {
    k_l1<<<grid_for(total), 256, 0, s>>>(x, y, total, inv_m, grad, acc);
  } else {
    const Win w = window();
    float* hm = reinterpret_cast<float*>(scratch + 256);  // [5][total], then [3][total]
    float* G = hm + 5 * total;                             // [3][total]
    const int64_t rows = (int64_t)n * H;
    const int64_t segs = rows * ((W + HSEG - 1) / HSEG);
    const unsigned hgrid = (unsigned)(segs < 148 * 16 ? segs : 148 * 16);
    k_h5<<<hgrid, HSEG, 0, s>>>(x, y, rows, W, w, total, hm);
    const int64_t strips = (int64_t)n * ((H + RS - 1) / RS) * W;
    k_v5<<<grid_for(strips), 256, 0, s>>>(hm, x, y, total, n, H, W, w, w_ssim, G, acc);
    k_h3<<<hgrid, HSEG, 0, s>>>(G, rows, W, w, total, hm);
    k_v3<<<grid_for(strips), 256, 0, s>>>(hm, x, y, total, n, H, W, w, w_ssim, inv_m, grad);
  }
  if (loss_out) k_loss_out<<<1, 32, 0, s>>>(acc, inv_m, loss_out);
  return cudaGetLastError();
}

}  // namespace igs
