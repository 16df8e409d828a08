// Instantiations and dispatch of the batched render kernels (16x16 tiles):
// the persistent fused forward + L1 + adjoint and the forward render over the
// concatenated tiles of many images.
#include "render.cuh"

namespace igs {

namespace {

template <int KK, int NCC, int CH>
cudaError_t bwd_batch_inst(const RenderParams& p, const BatchTables& bt, int grid,
                           cudaStream_t s) {
  const size_t bytes = sizeof(float) * (size_t)bwd_smem(16 * 16, NCC > 0 ? NCC : p.n, CH).total;
  if (bytes > 48 * 1024) {
    // the limit is a per-device attribute of the kernel: set on every launch
    // (idempotent, and right for whichever device and thread launches)
    cudaError_t e = cudaFuncSetAttribute(k_render_bwd_batch<16, KK, NCC, CH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
  }
  k_render_bwd_batch<16, KK, NCC, CH><<<grid, 256, bytes, s>>>(p, bt);
  return cudaGetLastError();
}

template <int KK, int NCC>
cudaError_t bwd_batch_stage(const RenderParams& p, const BatchTables& bt, int stage, int grid,
                            cudaStream_t s) {
  switch (stage) {
    case 64: return bwd_batch_inst<KK, NCC, 64>(p, bt, grid, s);
    case 128: return bwd_batch_inst<KK, NCC, 128>(p, bt, grid, s);
    case 256: return bwd_batch_inst<KK, NCC, 256>(p, bt, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

#define IGS_BATCH_NC(KK, unused)                                              \
  switch (IGS_NC_OF(p.n)) {                                                   \
    case 1: return bwd_batch_stage<KK, 1>(p, bt, stage, grid, s);             \
    case 3: return bwd_batch_stage<KK, 3>(p, bt, stage, grid, s);             \
    case 4: return bwd_batch_stage<KK, 4>(p, bt, stage, grid, s);             \
    case 9: return bwd_batch_stage<KK, 9>(p, bt, stage, grid, s);             \
    default: return bwd_batch_stage<KK, 0>(p, bt, stage, grid, s);            \
  }

cudaError_t launch_render_bwd_batch(const RenderParams& p, const BatchTables& bt, int K,
                                    int stage, int grid, cudaStream_t s) {
  if (bt.T == 0) return cudaSuccess;
  IGS_FOR_K(IGS_BATCH_NC, 0)
  return cudaSuccess;
}

namespace {

template <int KK, int NCC>
cudaError_t fwd_batch_inst(const RenderParams& p, const BatchTables& bt, cudaStream_t s) {
  k_render_fwd_batch<16, KK, NCC><<<bt.T, 256, 0, s>>>(p, bt);
  return cudaGetLastError();
}

}  // namespace

#define IGS_FWD_BATCH_NC(KK, unused)                                          \
  switch (IGS_NC_OF(p.n)) {                                                   \
    case 1: return fwd_batch_inst<KK, 1>(p, bt, s);                           \
    case 3: return fwd_batch_inst<KK, 3>(p, bt, s);                           \
    case 4: return fwd_batch_inst<KK, 4>(p, bt, s);                           \
    case 9: return fwd_batch_inst<KK, 9>(p, bt, s);                           \
    default: return fwd_batch_inst<KK, 0>(p, bt, s);                          \
  }

cudaError_t launch_render_fwd_batch(const RenderParams& p, const BatchTables& bt, int K,
                                    cudaStream_t s) {
  if (bt.T == 0) return cudaSuccess;
  IGS_FOR_K(IGS_FWD_BATCH_NC, 0)
  return cudaSuccess;
}

}  // namespace igs
