// Instantiations and dispatch of the random-access decode kernel.
#include "render.cuh"

namespace igs {

#define IGS_DEC_NC(KK, nc)                                            \
  switch (nc) {                                                       \
    case 1: k_decode<KK, 1><<<grid, 256, 0, s>>>(p); break;           \
    case 3: k_decode<KK, 3><<<grid, 256, 0, s>>>(p); break;           \
    case 4: k_decode<KK, 4><<<grid, 256, 0, s>>>(p); break;           \
    case 9: k_decode<KK, 9><<<grid, 256, 0, s>>>(p); break;           \
    default: k_decode<KK, 0><<<grid, 256, 0, s>>>(p); break;          \
  }

cudaError_t launch_render_fwd_t8(const RenderParams& p, int K, cudaStream_t s);
cudaError_t launch_render_fwd_t16(const RenderParams& p, int K, cudaStream_t s);
cudaError_t launch_render_bwd_t8(const RenderParams& p, int K, cudaStream_t s);
cudaError_t launch_render_bwd_t16(const RenderParams& p, int K, cudaStream_t s);

cudaError_t launch_decode(const RenderParams& p, int K, cudaStream_t s) {
  if (p.Q == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((p.Q + 255) / 256);
  const int nc = IGS_NC_OF(p.n);
  IGS_FOR_K(IGS_DEC_NC, nc)
  return cudaGetLastError();
}

bool render_supported(int tile, int K, int n) {
  return (tile == 8 || tile == 16) && k_supported(K) && n >= 1 && n <= 32;
}

cudaError_t launch_render_fwd(const RenderParams& p, int tile, int K, cudaStream_t s) {
  if (tile == 16) return launch_render_fwd_t16(p, K, s);
  if (tile == 8) return launch_render_fwd_t8(p, K, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_render_bwd(const RenderParams& p, int tile, int K, cudaStream_t s) {
  if (tile == 16) return launch_render_bwd_t16(p, K, s);
  if (tile == 8) return launch_render_bwd_t8(p, K, s);
  return cudaErrorInvalidValue;
}

}  // namespace igs
