// Instantiations and dispatch of the per-tile render kernels for 16x16 tiles.
#include "render.cuh"

namespace igs {

#define IGS_FWD_NC(KK, nc)                                                                 \
  switch (nc) {                                                                            \
    case 1: k_render_fwd<16, KK, 1><<<grid, 16 * 16, 0, s>>>(p); break;                    \
    case 3: k_render_fwd<16, KK, 3><<<grid, 16 * 16, 0, s>>>(p); break;                    \
    case 4: k_render_fwd<16, KK, 4><<<grid, 16 * 16, 0, s>>>(p); break;                    \
    case 9: k_render_fwd<16, KK, 9><<<grid, 16 * 16, 0, s>>>(p); break;                    \
    default: k_render_fwd<16, KK, 0><<<grid, 16 * 16, 0, s>>>(p); break;                   \
  }

#define IGS_BWD_NC(KK, nc)                                                                 \
  switch (nc) {                                                                            \
    case 1: k_render_bwd<16, KK, 1><<<grid, 16 * 16, 0, s>>>(p); break;                    \
    case 3: k_render_bwd<16, KK, 3><<<grid, 16 * 16, 0, s>>>(p); break;                    \
    case 4: k_render_bwd<16, KK, 4><<<grid, 16 * 16, 0, s>>>(p); break;                    \
    case 9: k_render_bwd<16, KK, 9><<<grid, 16 * 16, 0, s>>>(p); break;                    \
    default: k_render_bwd<16, KK, 0><<<grid, 16 * 16, 0, s>>>(p); break;                   \
  }

cudaError_t launch_render_fwd_t16(const RenderParams& p, int K, cudaStream_t s) {
  const unsigned grid = (unsigned)(p.tiles_x * p.tiles_y);
  if (grid == 0) return cudaSuccess;
  const int nc = IGS_NC_OF(p.n);
  IGS_FOR_K(IGS_FWD_NC, nc)
  return cudaGetLastError();
}

cudaError_t launch_render_bwd_t16(const RenderParams& p, int K, cudaStream_t s) {
  const unsigned grid = (unsigned)(p.tiles_x * p.tiles_y);
  if (grid == 0) return cudaSuccess;
  const int nc = IGS_NC_OF(p.n);
  IGS_FOR_K(IGS_BWD_NC, nc)
  return cudaGetLastError();
}

}  // namespace igs
