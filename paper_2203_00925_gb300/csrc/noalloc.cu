// fvgb_fv_residual_noalloc: the transport residual with its scratch in a fixed,
// library-owned device array instead of buffers allocated for the mesh.
//
// Some callers cannot allocate device memory at the point where they need a residual:
// a host program whose device memory is handed out by its own pool (a stray cudaMalloc
// can fail or fragment it), or a time-critical loop where cudaMalloc / cudaFree would
// add latency and implicit synchronisation. This entry point allocates nothing: the
// face fluxes and vertex values it needs live in g_noalloc_scratch below, a file-scope
// device array that every GPU loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace fvgb {
namespace {

// 8 MiB: room for n_face + n_vert reals (1,048,576 doubles or 2,097,152 floats), plus
// alignment of the vertex part to 256 bytes.
constexpr size_t kNoAllocBytes = size_t(8) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
struct ScratchSlot {
  unsigned long long ctx_id = 0;   // unique id of the context the address belongs to
  void* addr = nullptr;
};
ScratchSlot g_scratch[kMaxDevices];

// Driver entry points for the current context and its process-unique id, fetched through
// the runtime (no link-time dependency on the driver library). A context id is never
// reused, so a context that was destroyed (cudaDeviceReset) and re-created gets a new id.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_entry_looked_up = false;

// id of the current context, 0 when it cannot be determined
unsigned long long current_ctx_id() {
  if (!g_entry_looked_up) {
    g_entry_looked_up = true;
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      g_ctx_current = (CtxGetCurrentFn)f1;
      g_ctx_id = (CtxGetIdFn)f2;
    }
  }
  if (!g_ctx_current || !g_ctx_id) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_current(&ctx) != 0 || !ctx || g_ctx_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch array in the current context. Set-up happens once per
// device and context: the address is looked up with cudaGetSymbolAddress (with the
// device current) and cached together with the context's id; a later call in another
// context of the same device (after cudaDeviceReset) looks it up again. When the context
// id cannot be read, the address is looked up on every call (a host-side table lookup
// that allocates nothing).
cudaError_t scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  const unsigned long long id = current_ctx_id();
  ScratchSlot& slot = g_scratch[dev];
  if (id == 0 || slot.ctx_id != id || !slot.addr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    // the lookup itself creates the context if there was none: read the id again
    slot.ctx_id = id != 0 ? id : current_ctx_id();
    slot.addr = p;
  }
  *out = slot.addr;
  return cudaSuccess;
}

template <typename T>
fvgb_status residual_noalloc(fvgb_mesh m, const fvgb_tcoef* tc, const T* u, T* res,
                             cudaStream_t s) {
  const TopoDev& t = m->topo;
  const size_t flux_bytes = ((size_t)t.F * sizeof(T) + 255) / 256 * 256;
  const size_t need = flux_bytes + (size_t)t.V * sizeof(T);
  if (need > kNoAllocBytes) {
    set_error("fvgb_fv_residual_noalloc: mesh needs " + std::to_string(need) +
              " bytes of scratch (n_face + n_vert reals), more than the fixed " +
              std::to_string(kNoAllocBytes) + "; use fvgb_fv_residual");
    return FVGB_EINVAL;
  }
  int dev = -1;
  fvgb_status st = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
  if (st) return st;
  if (dev != m->device) {
    set_error("fvgb_fv_residual_noalloc: the mesh's device must be current");
    return FVGB_EINVAL;
  }
  void* base = nullptr;
  st = cuda_status(scratch_address(dev, &base), "cudaGetSymbolAddress");
  if (st) return st;
  T* flux = (T*)base;
  T* uv = (T*)((unsigned char*)base + flux_bytes);
  // every kernel below writes its whole scratch range before reading it, so nothing
  // left by an earlier call is ever read
  if (tc->diff != 0.0) {
    st = cuda_status(launch_vertex<T>(m, tc->bcset, u, uv, false, s), "vertex kernel");
    if (st) return st;
  }
  st = cuda_status(launch_face<T>(m, tc->bcset, u, uv, (const T*)tc->vel_dev, tc->vel_const, true,
                                  tc->diff, false, flux, s), "face kernel");
  if (st) return st;
  return cuda_status(launch_update<T>(m, kResidual, flux, (const T*)tc->src_dev, nullptr, 0.0,
                                      nullptr, res, nullptr, s), "update kernel");
}

}  // namespace
}  // namespace fvgb

using namespace fvgb;

extern "C" fvgb_status fvgb_fv_residual_noalloc(fvgb_mesh m, const fvgb_tcoef* tc,
                                                const void* u, void* res, void* stream) {
  if (!m) { set_error("null mesh handle"); return FVGB_EINVAL; }
  if (!tc) { set_error("tcoef is null"); return FVGB_EINVAL; }
  if (tc->recon != 0 && tc->recon != 1) { set_error("recon must be 0 (upwind) or 1 (MUSCL + Barth-Jespersen)"); return FVGB_EINVAL; }
  if (tc->recon == 1) { set_error("the allocation-free residual is first-order upwind only (recon = 0)"); return FVGB_EUNSUPPORTED; }
  if (!(tc->diff >= 0.0)) { set_error("diffusivity must be >= 0"); return FVGB_EINVAL; }
  if (tc->bcset < 0 || tc->bcset >= (int32_t)m->g64.bc.size()) { set_error("bcset index out of range"); return FVGB_EINVAL; }
  if (!u || !res || u == res) { set_error("u and res must be distinct device arrays"); return FVGB_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  if (m->prec != FVGB_FP64) return residual_noalloc<float>(m, tc, (const float*)u, (float*)res, s);
  return residual_noalloc<double>(m, tc, (const double*)u, (double*)res, s);
}
