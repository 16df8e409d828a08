// Throughput probes for the roofline denominators: FP32 fused multiply-add
// (scalar and packed pairs), the special-function unit's exp2, float and
// integer min/max (the top-K selection's comparators) and warp match.
// Each probe runs independent dependency chains in every thread of a grid
// that fills the GPU, timed with CUDA events; the instructions are inline PTX
// so that the compiler can neither fold nor drop them. Measurement only: the
// rasteriser does not call this library.
#include <cuda_runtime.h>
#include <stdint.h>

#include "igs_peaks.h"

namespace {

constexpr int CHAINS = 8;
constexpr int UNROLL = 16;

template <int KIND>
__global__ void __launch_bounds__(512) k_probe(float* out, int iters, float seed) {
  float a[CHAINS];
  unsigned u[CHAINS];
  unsigned long long p[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) {
    a[c] = seed + 0.001f * (float)(threadIdx.x + c);
    u[c] = threadIdx.x * 2654435761u + c;
    const float lo = a[c], hi = a[c] + 0.5f;
    p[c] = ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
  }
  const float m = 0.999f, b = 0.001f;
  const unsigned long long m2 = ((unsigned long long)__float_as_uint(m) << 32) | __float_as_uint(m);
  const unsigned long long b2 = ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(b);
  const float lim = seed * 0.5f;
  const unsigned ulim = 0x9e3779b9u ^ threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < UNROLL; ++r) {
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) {
        if (KIND == IGS_PEAK_FFMA) {
          asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[c]) : "f"(m), "f"(b));
        } else if (KIND == IGS_PEAK_FFMA2) {
          asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(p[c]) : "l"(m2), "l"(b2));
        } else if (KIND == IGS_PEAK_EX2) {
          asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(a[c]));
        } else if (KIND == IGS_PEAK_FMNMX) {
          asm volatile("min.f32 %0, %0, %1;" : "+f"(a[c]) : "f"(lim));
        } else if (KIND == IGS_PEAK_FMNMX3) {
          asm volatile("min.f32 %0, %0, %1, %2;" : "+f"(a[c]) : "f"(lim), "f"(b));
        } else if (KIND == IGS_PEAK_IMNMX) {
          asm volatile("min.u32 %0, %0, %1;" : "+r"(u[c]) : "r"(ulim));
        } else if (KIND == IGS_PEAK_MATCH) {
          asm volatile("match.any.sync.b32 %0, %0, 0xffffffff;" : "+r"(u[c]));
        }
      }
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c)
    s += a[c] + __uint_as_float(u[c] & 0x3fffffffu) + __uint_as_float((unsigned)p[c]);
  if (s == 1.2345f) out[blockIdx.x] = s;  // keeps every chain live
}

template <int KIND>
cudaError_t launch(int blocks, int threads, int iters, float* out, cudaStream_t st) {
  k_probe<KIND><<<blocks, threads, 0, st>>>(out, iters, 1.5f);
  return cudaGetLastError();
}

cudaError_t launch_kind(int kind, int blocks, int threads, int iters, float* out,
                        cudaStream_t st) {
  switch (kind) {
    case IGS_PEAK_FFMA: return launch<IGS_PEAK_FFMA>(blocks, threads, iters, out, st);
    case IGS_PEAK_FFMA2: return launch<IGS_PEAK_FFMA2>(blocks, threads, iters, out, st);
    case IGS_PEAK_EX2: return launch<IGS_PEAK_EX2>(blocks, threads, iters, out, st);
    case IGS_PEAK_FMNMX: return launch<IGS_PEAK_FMNMX>(blocks, threads, iters, out, st);
    case IGS_PEAK_FMNMX3: return launch<IGS_PEAK_FMNMX3>(blocks, threads, iters, out, st);
    case IGS_PEAK_IMNMX: return launch<IGS_PEAK_IMNMX>(blocks, threads, iters, out, st);
    case IGS_PEAK_MATCH: return launch<IGS_PEAK_MATCH>(blocks, threads, iters, out, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

extern "C" int igs_peak_probe(int kind, int iters, int reps, double* ops_per_s,
                              double* instr_per_s, float* best_ms) {
  if (kind < 0 || kind >= IGS_PEAK_KINDS || iters <= 0 || reps <= 0 || !ops_per_s ||
      !instr_per_s || !best_ms)
    return 1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 2;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 2;
  const int threads = 512, blocks = sms * 4;  // 64 warps per SM: enough chains in flight
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float) * blocks) != cudaSuccess) return 2;
  cudaStream_t st;
  cudaEvent_t e0, e1;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = 0;
  float best = 0.0f;
  if (launch_kind(kind, blocks, threads, 1, out, st) != cudaSuccess) rc = 2;  // warm-up
  for (int r = 0; r < reps && rc == 0; ++r) {
    cudaEventRecord(e0, st);
    if (launch_kind(kind, blocks, threads, iters, out, st) != cudaSuccess) rc = 2;
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = 2;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r == 0 || ms < best) best = ms;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) rc = 2;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  cudaFree(out);
  if (rc) return rc;
  // instructions per thread: iters * UNROLL * CHAINS; packed pairs do two lane-ops each
  const double thr = (double)blocks * threads;
  const double inst = thr * (double)iters * UNROLL * CHAINS;
  *best_ms = best;
  *instr_per_s = (kind == IGS_PEAK_MATCH ? inst / 32.0 : inst) / (best * 1e-3);
  *ops_per_s = (kind == IGS_PEAK_FFMA2 ? 2.0 * inst : inst) / (best * 1e-3);
  return 0;
}
