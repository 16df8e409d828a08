// Forward render for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: a
// plug-in running inside a host application that owns every allocation, a
// real-time thread where an allocation could block or fail, or code that
// must keep a fixed, audited device-memory budget. igs_render_forward_static
// serves them: it bins and renders like igs_preprocess_bin followed by
// igs_render_forward, but its scratch lives in one fixed-size array in this
// file, which every GPU that loads the library holds until the process exits.
#include <cstdio>

#include "imgs.h"
#include "internal.h"

namespace igs {

// Fixed scratch for the no-allocation render: IGS_STATIC_SCRATCH_BYTES
// (32 MiB) per device.
constexpr size_t STATIC_SCRATCH_BYTES = IGS_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

namespace {

// Device address of the scratch on the current device. In host code the
// array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress with that device current. It is looked up on every
// call (a cheap query next to a bin and render), so it stays right when the
// device's context is torn down and created again (cudaDeviceReset) and the
// module is loaded at another address. The first call on a device also loads
// the module there.
cudaError_t scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

}  // namespace

}  // namespace igs

using namespace igs;

extern "C" int igs_static_scratch_bytes(size_t* bytes) {
  if (bytes) *bytes = STATIC_SCRATCH_BYTES;
  return IGS_OK;
}

extern "C" int igs_render_forward_static(const igs_gaussians* g, int32_t H, int32_t W,
                                         const igs_config* cfg, float* d_img,
                                         igs_stream stream) {
  char msg[256];
  if (!g || !cfg || !d_img) {
    snprintf(msg, sizeof(msg), "igs_render_forward_static: NULL argument");
    set_last_error(msg);
    return IGS_ERR_INVALID_ARG;
  }
  // Room for the intersections: the largest capacity whose binning sections
  // fit. A render needs only those (igs_preprocess_bin checks the same
  // size); the fit-step images that igs_workspace_size adds for a config with
  // an SSIM term are not used here.
  igs_config bin_cfg = *cfg;
  bin_cfg.ssim_weight = 0.0f;
  size_t fixed = 0;
  if (int r = igs_workspace_size(g->N, g->n, H, W, &bin_cfg, 1, &fixed)) return r;
  if (fixed > STATIC_SCRATCH_BYTES) {
    snprintf(msg, sizeof(msg),
             "igs_render_forward_static: N=%lld, n=%d, %dx%d needs %zu bytes before any "
             "intersection; the static scratch holds %zu",
             (long long)g->N, g->n, H, W, fixed, STATIC_SCRATCH_BYTES);
    set_last_error(msg);
    return IGS_ERR_CAPACITY;
  }
  // Each intersection costs 8 bytes: its list entry and a merge slot.
  int64_t m_cap = (int64_t)((STATIC_SCRATCH_BYTES - fixed) / 8);
  size_t need = 0;
  while (m_cap > 1) {
    if (int r = igs_workspace_size(g->N, g->n, H, W, &bin_cfg, m_cap, &need)) return r;
    if (need <= STATIC_SCRATCH_BYTES) break;
    m_cap -= m_cap / 64 + 1;
  }
  if (m_cap < 1) m_cap = 1;
  void* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "igs_render_forward_static: scratch address: %s",
             cudaGetErrorString(e));
    set_last_error(msg);
    return IGS_ERR_CUDA;
  }
  igs_bins bins;
  // igs_preprocess_bin clears the status block and the tile ranges, and
  // writes every other scratch word it later reads.
  if (int r = igs_preprocess_bin(g, H, W, cfg, scratch, STATIC_SCRATCH_BYTES, m_cap, &bins,
                                 stream))
    return r;
  if (int r = igs_render_forward(&bins, cfg, d_img, stream)) return r;
  igs_stats st;
  if (int r = igs_read_stats(&bins, &st, stream)) return r;  // synchronises `stream`
  if (st.flags & IGS_FLAG_CAPACITY) {
    snprintf(msg, sizeof(msg),
             "igs_render_forward_static: %lld tile-Gaussian intersections exceed the %lld "
             "that fit in the static scratch; the image is incomplete",
             (long long)st.m_needed, (long long)m_cap);
    set_last_error(msg);
    return IGS_ERR_CAPACITY;
  }
  return IGS_OK;
}
