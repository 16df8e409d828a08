// Instantiations and dispatch of the per-tile render kernels for 16x16 tiles.
#include "render.cuh"

namespace igs {

namespace {

template <int KK, int NCC>
cudaError_t fwd_inst(const RenderParams& p, dim3 grid, cudaStream_t s) {
  k_render_fwd<16, KK, NCC><<<grid, 16 * 16, 0, s>>>(p);
  return cudaGetLastError();
}

template <int KK, int NCC>
cudaError_t bwd_inst(const RenderParams& p, dim3 grid, cudaStream_t s) {
  const size_t bytes = sizeof(float) * (size_t)bwd_smem(16 * 16, NCC > 0 ? NCC : p.n, 16 * 16).total;
  if (bytes > 48 * 1024) {
    // the limit is a per-device attribute of the kernel: set on every launch
    // (idempotent, and right for whichever device and thread launches)
    cudaError_t e = cudaFuncSetAttribute(k_render_bwd<16, KK, NCC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
  }
  k_render_bwd<16, KK, NCC><<<grid, 16 * 16, bytes, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

#define IGS_NC_SWITCH(KK, FN)                                  \
  switch (IGS_NC_OF(p.n)) {                                    \
    case 1: return FN<KK, 1>(p, grid, s);                      \
    case 3: return FN<KK, 3>(p, grid, s);                      \
    case 4: return FN<KK, 4>(p, grid, s);                      \
    case 9: return FN<KK, 9>(p, grid, s);                      \
    default: return FN<KK, 0>(p, grid, s);                     \
  }

cudaError_t launch_render_fwd_t16(const RenderParams& p, int K, cudaStream_t s) {
  if (p.tiles_x * p.tiles_y == 0) return cudaSuccess;
  const dim3 grid((unsigned)p.tiles_x, (unsigned)p.tiles_y);  // one CTA per tile
  IGS_FOR_K(IGS_NC_SWITCH, fwd_inst)
  return cudaSuccess;
}

cudaError_t launch_render_bwd_t16(const RenderParams& p, int K, cudaStream_t s) {
  if (p.tiles_x * p.tiles_y == 0) return cudaSuccess;
  const dim3 grid((unsigned)p.tiles_x, (unsigned)p.tiles_y);  // one CTA per tile
  IGS_FOR_K(IGS_NC_SWITCH, bwd_inst)
  return cudaSuccess;
}

}  // namespace igs
