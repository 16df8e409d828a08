// Image-space fitting loss L1 + w (1 - SSIM) (Sec. 3.3 and Sec. 4.1, which
// fits against L1 + 0.1 L_SSIM) and its gradient with respect to the
// rendering, for the fit steps that include the SSIM term.
//
// SSIM is computed per channel with an 11 x 11 Gaussian window (sigma 1.5,
// normalised, zero-padded "same" correlation) and C1 = 0.01^2, C2 = 0.03^2;
// L_SSIM = 1 - mean SSIM over channels and pixels. The gradient is
//   dL/dx = sign(x - y)/M - (w/M)(bG1 + 2x bG2 + y bG3),
// where G1 = dS/dmu_x, G2 = dS/dE[x^2], G3 = dS/dE[xy] are the SSIM partials
// with respect to the raw window moments at each pixel (zero outside the
// image) and bG their window sums (the window is symmetric: the transposed
// correlation is the same one). One kernel does it per 32 x 32 tile of
// output pixels with a halo, float32, for one image or every image of a
// batch in one launch.
#include <cmath>

#include "internal.h"

namespace igs {

namespace {

constexpr int WR = 5;  // window radius
constexpr float C1 = 1e-4f, C2 = 9e-4f;

struct Win {
  float g[2 * WR + 1];
};

// One pass per 32 x 32 output tile: the tile's x and y with a 10-pixel halo
// are staged in shared memory; the window moments and SSIM partials are
// formed over the tile plus a 5-pixel ring, window-summed again over the
// tile, and turned into the gradient. Each thread takes several consecutive
// outputs of a row or column (3, VB, HB, 4 in the four passes), so that
// staged values are reused across taps.
constexpr int TO = 32;           // output tile edge
constexpr int TM = TO + 2 * WR;  // 42: window moments and SSIM partials
constexpr int VB = 7;            // moment rows per thread: 252 tasks, one CTA round
constexpr int HB = 4;            // partial-sum columns per thread (divides TO)
constexpr int TI = TO + 4 * WR;  // 52: staged x and y
constexpr int SSIM_THREADS = 256;
// shared memory (floats): [x | y] staged (2 TI^2), later the partials G
// (3 TM^2); the horizontal sums of the 5 moments (5 TI TM), later those of
// the 3 partials (3 TM TO)
constexpr int SSIM_SA = 2 * TI * TI;
constexpr int SSIM_SB = 5 * TI * TM;
constexpr size_t SSIM_SMEM = sizeof(float) * (SSIM_SA + SSIM_SB);
static_assert(3 * TM * TM <= SSIM_SA && 3 * TM * TO <= SSIM_SB, "ssim smem reuse");

// The images a launch covers: one (dims == nullptr: H, W) or a batch's
// per-image (H, W, 32-tiles across) with first 32-tile and plane offsets.
struct SsimImages {
  int B;
  const int4* dims;
  const int* tile_off;
  const long long* pix_off;
  int H, W;
};

__global__ void __launch_bounds__(SSIM_THREADS, 3) k_ssim_tile(const float* x, const float* y,
                                                            SsimImages im, int n, Win w,
                                                            float w_ssim, float* grad,
                                                            double* acc) {
  extern __shared__ __align__(16) float smem[];
  float* sA = smem;
  float* sB = smem + SSIM_SA;
  const int tid = threadIdx.x;
  // this tile's image and origin
  int b = 0, H = im.H, W = im.W, t = blockIdx.x;
  long long off = 0;
  if (im.dims) {
    int lo = 0, hi = im.B - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (im.tile_off[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    b = lo;
    const int4 d = im.dims[b];
    H = d.x;
    W = d.y;
    t = (int)blockIdx.x - im.tile_off[b];
    off = im.pix_off[b];
  }
  const int tx = (W + TO - 1) / TO;
  const int x0 = (t % tx) * TO, y0 = (t / tx) * TO;
  const int64_t HW = (int64_t)H * W;
  const float inv_m = 1.0f / ((float)n * (float)H * (float)W);
  // this thread's share of the loss: at most a few dozen terms of magnitude
  // <= max(1, w_ssim) per channel, summed in float32; one float64 atomic per
  // warp (FP64 arithmetic runs at a small fraction of the FP32 rate)
  float part = 0.0f;
  for (int c = 0; c < n; ++c) {
    const float* xc = x + off + c * HW;
    const float* yc = y + off + c * HW;
    __syncthreads();  // the previous channel is done with the staged arrays
    for (int k = tid; k < TI * TI; k += SSIM_THREADS) {
      const int r = y0 - 2 * WR + k / TI, q = x0 - 2 * WR + k % TI;
      const bool in = r >= 0 && r < H && q >= 0 && q < W;
      sA[k] = in ? xc[(int64_t)r * W + q] : 0.0f;
      sA[TI * TI + k] = in ? yc[(int64_t)r * W + q] : 0.0f;
    }
    __syncthreads();
    // horizontal window sums of x, y, x^2, y^2, x y: rows TI, columns TM
    for (int task = tid; task < TI * (TM / 3); task += SSIM_THREADS) {
      const int r = task / (TM / 3), j0 = (task % (TM / 3)) * 3;
      float s[5][3];
#pragma unroll
      for (int m = 0; m < 5; ++m)
#pragma unroll
        for (int o = 0; o < 3; ++o) s[m][o] = 0.0f;
#pragma unroll
      for (int e = 0; e < 2 * WR + 3; ++e) {
        const float a = sA[r * TI + j0 + e], d = sA[TI * TI + r * TI + j0 + e];
        const float aa = a * a, dd = d * d, ad = a * d;
#pragma unroll
        for (int o = 0; o < 3; ++o) {
          const int i = e - o;  // tap of input e for output j0 + o
          if (i < 0 || i > 2 * WR) continue;
          const float g = w.g[i];
          s[0][o] = fmaf(g, a, s[0][o]);
          s[1][o] = fmaf(g, d, s[1][o]);
          s[2][o] = fmaf(g, aa, s[2][o]);
          s[3][o] = fmaf(g, dd, s[3][o]);
          s[4][o] = fmaf(g, ad, s[4][o]);
        }
      }
#pragma unroll
      for (int m = 0; m < 5; ++m)
#pragma unroll
        for (int o = 0; o < 3; ++o) sB[(m * TI + r) * TM + j0 + o] = s[m][o];
    }
    __syncthreads();
    // vertical sums -> moments -> SSIM and its partials over the TM x TM
    // ring region (zero outside the image); the loss's SSIM term over the
    // tile's own pixels
    // (VB rows per task: TM * TM / VB = 252 tasks, one round of the CTA)
    for (int task = tid; task < TM * (TM / VB); task += SSIM_THREADS) {
      const int jm = task % TM, i0 = (task / TM) * VB;
      float m[5][VB];
#pragma unroll
      for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int o = 0; o < VB; ++o) m[k][o] = 0.0f;
#pragma unroll
      for (int e = 0; e < 2 * WR + VB; ++e) {
        float v[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) v[k] = sB[(k * TI + i0 + e) * TM + jm];
#pragma unroll
        for (int o = 0; o < VB; ++o) {
          const int i = e - o;
          if (i < 0 || i > 2 * WR) continue;
#pragma unroll
          for (int k = 0; k < 5; ++k) m[k][o] = fmaf(w.g[i], v[k], m[k][o]);
        }
      }
#pragma unroll
      for (int o = 0; o < VB; ++o) {
        const int ii = i0 + o;
        const int py = y0 - WR + ii, px = x0 - WR + jm;
        float g1 = 0.0f, g2 = 0.0f, g3 = 0.0f;
        if (py >= 0 && py < H && px >= 0 && px < W) {
          const float mx = m[0][o], my = m[1][o];
          const float vx = m[2][o] - mx * mx, vy = m[3][o] - my * my, cxy = m[4][o] - mx * my;
          const float A1 = 2.f * mx * my + C1, A2 = 2.f * cxy + C2;
          const float B1 = mx * mx + my * my + C1, B2 = vx + vy + C2;
          const float iB = rcp_approx(B1 * B2);
          const float S = A1 * A2 * iB;
          const float dS_dvx = -S * (B1 * iB);   // -S / B2
          const float dS_dcxy = 2.f * A1 * iB;
          const float dmx = 2.f * my * A2 * iB - S * 2.f * mx * (B2 * iB);  // ... / B1
          g1 = dmx - 2.f * mx * dS_dvx - my * dS_dcxy;
          g2 = dS_dvx;
          g3 = dS_dcxy;
          if (ii >= WR && ii < WR + TO && jm >= WR && jm < WR + TO)
            part += w_ssim * (1.0f - S);
        }
        sA[(0 * TM + ii) * TM + jm] = g1;
        sA[(1 * TM + ii) * TM + jm] = g2;
        sA[(2 * TM + ii) * TM + jm] = g3;
      }
    }
    __syncthreads();
    // horizontal window sums of the partials: rows TM, columns TO
    // (HB columns per task; 8 was no faster)
    for (int task = tid; task < TM * (TO / HB); task += SSIM_THREADS) {
      const int r = task / (TO / HB), j0 = (task % (TO / HB)) * HB;
      float s[3][HB];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int o = 0; o < HB; ++o) s[k][o] = 0.0f;
#pragma unroll
      for (int e = 0; e < 2 * WR + HB; ++e) {
        float v[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] = sA[(k * TM + r) * TM + j0 + e];
#pragma unroll
        for (int o = 0; o < HB; ++o) {
          const int i = e - o;
          if (i < 0 || i > 2 * WR) continue;
#pragma unroll
          for (int k = 0; k < 3; ++k) s[k][o] = fmaf(w.g[i], v[k], s[k][o]);
        }
      }
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int o = 0; o < HB; ++o) sB[(k * TM + r) * TO + j0 + o] = s[k][o];
    }
    __syncthreads();
    // vertical sums -> dL/dx over the tile: sign(x - y)/M - (w/M)(bG1 + 2x bG2 + y bG3)
    {
      const int jo = tid % TO, i0 = (tid / TO) * 4;  // 256 threads: 32 columns x 8 row blocks
      float s[3][4];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int o = 0; o < 4; ++o) s[k][o] = 0.0f;
#pragma unroll
      for (int e = 0; e < 2 * WR + 4; ++e) {
        float v[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] = sB[(k * TM + i0 + e) * TO + jo];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          const int i = e - o;
          if (i < 0 || i > 2 * WR) continue;
#pragma unroll
          for (int k = 0; k < 3; ++k) s[k][o] = fmaf(w.g[i], v[k], s[k][o]);
        }
      }
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const int py = y0 + i0 + o, px = x0 + jo;
        if (py >= H || px >= W) continue;
        const int64_t p = (int64_t)py * W + px;
        const float xv = xc[p], yv = yc[p];
        const float d = xv - yv;
        const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        grad[off + c * HW + p] =
            sgn * inv_m - w_ssim * inv_m * (s[0][o] + 2.f * xv * s[1][o] + yv * s[2][o]);
        part += fabsf(d);
      }
    }
  }
  part = warp_sum<float>(part);
  if ((tid & 31) == 0 && part != 0.0f) atomicAdd(acc + b, (double)part);
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

size_t image_loss_scratch_bytes(int, int, int) { return 256; }

cudaError_t launch_image_loss(const float* x, const float* y, int n, int H, int W,
                              float w_ssim, float* grad, double* acc, float* loss_out,
                              char* scratch, cudaStream_t s) {
  (void)scratch;
  const int64_t total = (int64_t)n * H * W;
  if (total == 0) return cudaSuccess;
  const float inv_m = (float)(1.0 / (double)total);
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  if (w_ssim == 0.0f) {
    k_l1<<<grid_for(total), 256, 0, s>>>(x, y, total, inv_m, grad, acc);
  } else {
    SsimImages im;
    im.B = 1;
    im.dims = nullptr;
    im.tile_off = nullptr;
    im.pix_off = nullptr;
    im.H = H;
    im.W = W;
    e = cudaFuncSetAttribute(k_ssim_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SSIM_SMEM);
    if (e != cudaSuccess) return e;
    const unsigned tiles = (unsigned)(((W + TO - 1) / TO) * ((H + TO - 1) / TO));
    k_ssim_tile<<<tiles, SSIM_THREADS, SSIM_SMEM, s>>>(x, y, im, n, window(), w_ssim, grad,
                                                       acc);
  }
  if (loss_out) k_loss_out<<<1, 32, 0, s>>>(acc, inv_m, loss_out);
  return cudaGetLastError();
}

int ssim_tiles_of(int H, int W) { return ((W + TO - 1) / TO) * ((H + TO - 1) / TO); }

cudaError_t launch_image_loss_batch(const float* x, const float* y, int B, const int4* dims,
                                    const int* tile_off, const long long* pix_off, int tiles,
                                    int n, float w_ssim, float* grad, double* acc,
                                    cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * B, s);
  if (e != cudaSuccess || tiles == 0) return e;
  SsimImages im;
  im.B = B;
  im.dims = dims;
  im.tile_off = tile_off;
  im.pix_off = pix_off;
  im.H = im.W = 0;
  e = cudaFuncSetAttribute(k_ssim_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)SSIM_SMEM);
  if (e != cudaSuccess) return e;
  k_ssim_tile<<<(unsigned)tiles, SSIM_THREADS, SSIM_SMEM, s>>>(x, y, im, n, window(), w_ssim,
                                                               grad, acc);
  return cudaGetLastError();
}

}  // namespace igs
