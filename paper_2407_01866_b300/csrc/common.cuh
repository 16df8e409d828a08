// Device-side building blocks shared by the rasteriser kernels.
//
// The binary32 decision formulas here (conic, 3-sigma radius, tile-circle
// test, ranking key) are the ones fixed in include/imgs.h. They use the _rn
// intrinsics so that the compiler cannot contract or reorder them: the
// selected sets must not depend on code generation.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace igs {

constexpr unsigned FULL_MASK = 0xffffffffu;
// 0.5 * log2(e): exp(-x/2) = exp2(-x * HALF_LOG2E)
constexpr float HALF_LOG2E = 0.72134752044448170368f;

// Preprocessed geometry, two float4 per Gaussian:
//   a = (mx, my, A00, B = 2*A01), b = (A11, r, t1, t2)
struct __align__(16) GRec {
  float4 a;
  float4 b;
};

// Hot record of a Gaussian stored in float16 or bfloat16: the stored bits of
// mu (x low, y high) and the binary32 conic. mu in pixels is recomputed with
// the same binary32 product as preprocessing, so the ranking key is the one
// computed from a GRec, from half the bytes.
struct __align__(16) HRec {
  unsigned int mu;
  float A00, B, A11;
};

// Binary32 value of a stored half-precision bit pattern (hdt 1: float16,
// 2: bfloat16); both convert exactly.
__device__ __forceinline__ float half_bits_to_f32(unsigned short h, int hdt) {
  return hdt == 2 ? __uint_as_float((unsigned)h << 16) : __half2float(__ushort_as_half(h));
}

// Device status block at the head of every workspace. The first 32 bytes
// have the layout of igs_stats in include/imgs.h.
struct DevStatus {
  unsigned int flags;
  unsigned int adam_done;       // CTAs of a fit step's Adam launch that are done
  unsigned long long m_needed;  // total intersections M
  unsigned long long evals;     // sum_j |S_j| * pixels(j)
  double loss_sum;              // sum |c_r - c_t| of the fused backward
  unsigned int reserved2;
  unsigned int wide_cnt;        // Gaussians whose tile box is binned by whole CTAs
  unsigned int pad[6];
};
static_assert(sizeof(DevStatus) == 64, "status block is 64 bytes");

enum : unsigned { FLAG_CAPACITY = 1u, FLAG_NONFINITE = 2u, FLAG_TIMEOUT = 4u, FLAG_INTERNAL = 8u };

template <typename T> __device__ __forceinline__ float to_f32(T v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

// Inverse covariance (Eq. 2 inverted) in the header's binary32 sequence.
__device__ __forceinline__ void conic_from(float c, float s, float t1, float t2,
                                           float& A00, float& B, float& A11) {
  const float T1 = __fmul_rn(t1, t1), T2 = __fmul_rn(t2, t2);
  const float cc = __fmul_rn(c, c), ss = __fmul_rn(s, s), cs = __fmul_rn(c, s);
  A00 = __fadd_rn(__fmul_rn(T1, cc), __fmul_rn(T2, ss));
  A11 = __fadd_rn(__fmul_rn(T1, ss), __fmul_rn(T2, cc));
  const float A01 = __fmul_rn(__fsub_rn(T1, T2), cs);
  B = __fadd_rn(A01, A01);
}

// Tile-circle test of Sec. 3.2 on the closed rect [X0,X1]x[Y0,Y1].
__device__ __forceinline__ bool circle_hits_rect(float mx, float my, float r2, float X0,
                                                 float X1, float Y0, float Y1) {
  const float ex = fmaxf(fmaxf(__fsub_rn(X0, mx), __fsub_rn(mx, X1)), 0.0f);
  const float ey = fmaxf(fmaxf(__fsub_rn(Y0, my), __fsub_rn(my, Y1)), 0.0f);
  const float d2 = __fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey));
  return d2 <= r2;
}

// Ranking key q = d^T Sigma^-1 d at (px, py) (Eq. 1 exponent times -2).
__device__ __forceinline__ float rank_key(float px, float py, float mx, float my, float A00,
                                          float B, float A11) {
  const float dx = __fsub_rn(px, mx);
  const float dy = __fsub_rn(py, my);
  const float h = __fmaf_rn(B, dy, __fmul_rn(A00, dx));
  return __fmaf_rn(h, dx, __fmul_rn(__fmul_rn(A11, dy), dy));
}

// Sorted insertion of (q, id) into tq[0..K-1] / tid[0..K-1], ascending in
// the (key, index) order, dropping the largest: the candidate bubbles down
// the list, swapping with every entry that follows it in that order. The
// result does not depend on the order candidates arrive in.
template <int K>
__device__ __forceinline__ void topk_insert(float (&tq)[K], int (&tid)[K], float q, int id) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float oq = tq[k];
    const int oi = tid[k];
    const bool sw = q < oq || (q == oq && id < oi);
    tq[k] = sw ? q : oq;
    tid[k] = sw ? id : oi;
    q = sw ? oq : q;
    id = sw ? oi : id;
  }
}

// Blend weight exp(-(q - q_min)/2) = 2^((q_min - q) log2(e)/2) on the special
// function unit (ex2.approx, relative error a few 2^-23; 2^0 is exactly 1;
// weights below 2^-126 flush to zero, where they are negligible in the blend).
__device__ __forceinline__ float blend_weight(float q0, float q) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"((q0 - q) * HALF_LOG2E));
  return y;
}

// Reciprocal on the MUFU (rcp.approx: within one ulp).
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float sign_f(float x) {
  return x > 0.0f ? 1.0f : (x < 0.0f ? -1.0f : 0.0f);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
  return v;
}

}  // namespace igs
