// Adam update with per-group learning rates and range clamps (Sec. 4.1
// optimiser and learning rates; Sec. 3.1 clipping of theta and the scales),
// and the per-step finalisation (step counter, mean loss).
#include <cmath>

#include "internal.h"

namespace igs {

namespace {

// Adam's bias correction 1 - beta^t in float32, from omb = 1 - beta: it is
// -expm1(t log1p(-omb)), within a few ulp of the float64 value. Every thread
// computes it (no float64 pow: on this part the FP64 pipe is narrow, and a
// per-CTA float64 pow behind a barrier stalled every CTA of the update).
__device__ __forceinline__ float one_minus_pow(float omb, int t) {
  return -expm1f((float)t * log1pf(-omb));
}

// The fit step's finalisation by the Adam launch's last CTA to finish: every
// CTA has read *a.step (at its start) before it counts itself done, so the
// increment is seen by none of them. fin->adam_done starts at 0 (binning
// resets the status block every step).
__device__ __forceinline__ void finalize_last(const AdamParams& a) {
  __syncthreads();  // every thread of this CTA has read *a.step
  if (threadIdx.x == 0 && atomicAdd(&a.fin->adam_done, 1u) == gridDim.x - 1) {
    *a.step += 1;
    if (a.fin_loss) *a.fin_loss = (float)(a.fin->loss_sum * (double)a.fin_inv_count);
  }
}

// One thread per Gaussian row: the column of each element (and so its learning
// rate and clamp) is known without a division, and a row's 5+n floats are
// contiguous, so a warp touches 32 consecutive rows.
template <int NP>
__global__ void __launch_bounds__(256) k_adam(AdamParams a) {
  const int step = *a.step + 1;
  const float inv_bc1 = 1.0f / one_minus_pow(a.omb1, step);
  const float inv_bc2 = 1.0f / one_minus_pow(a.omb2, step);
  const int np = NP > 0 ? NP : 5 + a.n;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.N;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t base = r * np;
#pragma unroll
    for (int col = 0; col < (NP > 0 ? NP : 64); ++col) {
      if (NP == 0 && col >= np) break;
      const int64_t i = base + col;
      const float g = a.G[i];
      const float m = a.b1 * a.m[i] + a.omb1 * g;
      const float v = a.b2 * a.v[i] + a.omb2 * g * g;
      const float lr = col < 2 ? a.lr_mu : col == 2 ? a.lr_theta : col < 5 ? a.lr_t : a.lr_c;
      float p = a.P[i] - lr * (m * inv_bc1) / (sqrtf(v * inv_bc2) + a.eps);
      if (col < 2) p = fminf(fmaxf(p, a.mu_min), a.mu_max);
      else if (col == 2) p = fminf(fmaxf(p, a.theta_min), a.theta_max);
      else if (col < 5) p = fminf(fmaxf(p, a.t_min), a.t_max);
      a.P[i] = p;
      a.m[i] = m;
      a.v[i] = v;
    }
  }
  if (a.fin) finalize_last(a);
}

// Rows of a multiple of 4 floats: consecutive threads take consecutive float4
// of the flattened arrays (coalesced), the columns follow from the index.
template <int NP>
__global__ void __launch_bounds__(256) k_adam_v4(AdamParams a) {
  static_assert(NP % 4 == 0, "float4 rows");
  const int step = *a.step + 1;
  const float inv_bc1 = 1.0f / one_minus_pow(a.omb1, step);
  const float inv_bc2 = 1.0f / one_minus_pow(a.omb2, step);
  const int64_t n4 = a.N * NP / 4;
  float4* P4 = reinterpret_cast<float4*>(a.P);
  const float4* G4 = reinterpret_cast<const float4*>(a.G);
  float4* M4 = reinterpret_cast<float4*>(a.m);
  float4* V4 = reinterpret_cast<float4*>(a.v);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int col0 = (int)((q * 4) % NP);
    float4 p = P4[q], g = G4[q], m = M4[q], v = V4[q];
    float* pp = &p.x;
    const float* gp = &g.x;
    float* mp = &m.x;
    float* vp = &v.x;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int col = col0 + k;
      mp[k] = a.b1 * mp[k] + a.omb1 * gp[k];
      vp[k] = a.b2 * vp[k] + a.omb2 * gp[k] * gp[k];
      const float lr = col < 2 ? a.lr_mu : col == 2 ? a.lr_theta : col < 5 ? a.lr_t : a.lr_c;
      float x = pp[k] - lr * (mp[k] * inv_bc1) / (sqrtf(vp[k] * inv_bc2) + a.eps);
      if (col < 2) x = fminf(fmaxf(x, a.mu_min), a.mu_max);
      else if (col == 2) x = fminf(fmaxf(x, a.theta_min), a.theta_max);
      else if (col < 5) x = fminf(fmaxf(x, a.t_min), a.t_max);
      pp[k] = x;
    }
    P4[q] = p;
    M4[q] = m;
    V4[q] = v;
  }
  if (a.fin) finalize_last(a);
}

__global__ void k_finalize(int32_t* step, DevStatus* st, float inv_count, float* loss_out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *step += 1;
    if (loss_out) *loss_out = (float)(st->loss_sum * (double)inv_count);
  }
}

__global__ void k_finalize_batch(int32_t* step, const double* loss, const int4* dims, int B, int n,
                                 float* loss_out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b == 0) *step += 1;
  if (loss_out && b < B) {
    const int4 d = dims[b];
    loss_out[b] = (float)(loss[b] / ((double)d.x * d.y * n));
  }
}

}  // namespace

cudaError_t launch_finalize_batch(int32_t* step, const double* loss, const int4* dims, int B,
                                  int n, float* loss_out, cudaStream_t s) {
  k_finalize_batch<<<(B + 255) / 256, 256, 0, s>>>(step, loss, dims, B, n, loss_out);
  return cudaGetLastError();
}

cudaError_t launch_adam(const AdamParams& a, cudaStream_t s) {
  if (a.N == 0) {  // no update; a fit step still advances
    if (a.fin) k_finalize<<<1, 32, 0, s>>>(a.step, a.fin, a.fin_inv_count, a.fin_loss);
    return cudaGetLastError();
  }
  int64_t blocks = (a.N + 255) / 256;
  if (blocks > 148 * 16) blocks = 148 * 16;
  switch (a.n) {
    case 1: k_adam<6><<<(unsigned)blocks, 256, 0, s>>>(a); break;
    case 3: {
      const bool aligned16 = ((uintptr_t)a.P | (uintptr_t)a.G | (uintptr_t)a.m |
                              (uintptr_t)a.v) % 16 == 0;
      if (aligned16) {
        int64_t b4 = (a.N * 2 + 255) / 256;
        if (b4 > 148 * 16) b4 = 148 * 16;
        k_adam_v4<8><<<(unsigned)b4, 256, 0, s>>>(a);
      } else {
        k_adam<8><<<(unsigned)blocks, 256, 0, s>>>(a);
      }
      break;
    }
    case 4: k_adam<9><<<(unsigned)blocks, 256, 0, s>>>(a); break;
    case 9: k_adam<14><<<(unsigned)blocks, 256, 0, s>>>(a); break;
    default: k_adam<0><<<(unsigned)blocks, 256, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

namespace {

// Round-to-nearest-even copy of float32 parameters into half storage.
template <typename T>
__global__ void __launch_bounds__(256) k_round_params(const float* src, T* dst, int64_t count);

template <>
__global__ void __launch_bounds__(256) k_round_params<__half>(const float* src, __half* dst,
                                                              int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __float2half_rn(src[i]);
}

template <>
__global__ void __launch_bounds__(256) k_round_params<__nv_bfloat16>(const float* src,
                                                                     __nv_bfloat16* dst,
                                                                     int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

}  // namespace

cudaError_t launch_round_params(const float* src, void* dst, bool bf16, int64_t count,
                                cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  if (bf16)
    k_round_params<__nv_bfloat16><<<(unsigned)blocks, 256, 0, s>>>(
        src, static_cast<__nv_bfloat16*>(dst), count);
  else
    k_round_params<__half><<<(unsigned)blocks, 256, 0, s>>>(src, static_cast<__half*>(dst),
                                                            count);
  return cudaGetLastError();
}

}  // namespace igs
