// Autotuner for the launch shapes of the gather kernels (least-squares gradient, vertex
// values, face fluxes, face-to-cell update): threads per block x elements per thread,
// chosen by timing every candidate with CUDA events on the mesh's own data, cached per
// device and mesh class (dimension, precision, size bucket). Every shape computes each
// output element with the same thread-local arithmetic, so results do not depend on it.
#include <cuda_runtime.h>

#include <array>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "internal.h"

namespace fvgb {
namespace {

std::mutex g_tune_mutex;
// (device, dim, prec, floor(log2 N)) -> shapes
std::map<std::tuple<int, int, int, int>, std::array<LaunchShape, kTuneCount>> g_tune_cache;

constexpr int kThreadCands[] = {128, 256, 512, 1024};
constexpr int kIptCands[] = {1, 2, 4};

template <typename T>
cudaError_t run_kernel(fvgb_mesh_s* m, int k, cudaStream_t s) {
  Work<T>& w = work_of<T>(m);
  switch (k) {
    case kTuneGrad: return launch_gradient<T>(m, 0, w.tmp, w.grad, s);
    case kTuneVertex: return launch_vertex<T>(m, 0, w.tmp, w.uv, false, s);
    case kTuneFace: return launch_face<T>(m, 0, w.tmp, w.uv, w.vel, nullptr, true, 0.1, false, w.flux, s);
    default: return launch_update<T>(m, kStep, w.flux, w.src, w.tmp, 1e-3, nullptr, w.stage, nullptr, s);
  }
}

template <typename T>
cudaError_t tune_all(fvgb_mesh_s* m, cudaStream_t s) {
  Work<T>& w = work_of<T>(m);
  const TopoDev& t = m->topo;
  cudaError_t e;
  if ((e = cudaMemsetAsync(w.tmp, 0, t.N * sizeof(T), s))) return e;
  if ((e = cudaMemsetAsync(w.vel, 0, t.dim * t.N * sizeof(T), s))) return e;
  if ((e = cudaMemsetAsync(w.src, 0, t.N * sizeof(T), s))) return e;
  if ((e = cudaMemsetAsync(w.uv, 0, t.V * sizeof(T), s))) return e;
  if ((e = cudaMemsetAsync(w.flux, 0, t.F * sizeof(T), s))) return e;
  cudaEvent_t a, b;
  if ((e = cudaEventCreate(&a))) return e;
  if ((e = cudaEventCreate(&b))) { cudaEventDestroy(a); return e; }
  for (int k = 0; k < kTuneCount && e == cudaSuccess; ++k) {
    float best = 1e30f;
    LaunchShape best_shape = m->tune[k];
    for (int th : kThreadCands)
      for (int ipt : kIptCands) {
        m->tune[k] = LaunchShape{th, ipt};
        if ((e = run_kernel<T>(m, k, s))) break;
        if ((e = cudaEventRecord(a, s))) break;
        for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = run_kernel<T>(m, k, s);
        if (e || (e = cudaEventRecord(b, s)) || (e = cudaEventSynchronize(b))) break;
        float ms = 0.0f;
        if ((e = cudaEventElapsedTime(&ms, a, b))) break;
        if (ms < best) { best = ms; best_shape = m->tune[k]; }
      }
    m->tune[k] = best_shape;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return e;
}

void drop_graph(fvgb_mesh_s* m) {
  // a captured step graph holds the old launch shapes
  graph_invalidate(m);
}

}  // namespace
}  // namespace fvgb

using namespace fvgb;

extern "C" fvgb_status fvgb_autotune(fvgb_mesh m, int32_t force, int32_t* shapes_out, void* stream) {
  if (!m) { set_error("null mesh handle"); return FVGB_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  const auto key = std::make_tuple(m->device, m->topo.dim, (int)m->prec,
                                   (int)std::floor(std::log2((double)m->topo.N)));
  bool cached = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end() && !force) {
      for (int k = 0; k < kTuneCount; ++k) m->tune[k] = it->second[k];
      cached = true;
    }
  }
  if (!cached) {
    const long long before = g_kernel_launches.load();
    cudaError_t e = m->prec == FVGB_FP64 ? tune_all<double>(m, s) : tune_all<float>(m, s);
    g_kernel_launches.store(before);   // tuning launches are not part of the work
    if (fvgb_status st = cuda_status(e, "autotune")) return st;
    std::array<LaunchShape, kTuneCount> sh;
    for (int k = 0; k < kTuneCount; ++k) sh[k] = m->tune[k];
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = sh;
  }
  drop_graph(m);
  if (shapes_out)
    for (int k = 0; k < kTuneCount; ++k) {
      shapes_out[2 * k] = m->tune[k].threads;
      shapes_out[2 * k + 1] = m->tune[k].ipt;
    }
  return FVGB_OK;
}

extern "C" fvgb_status fvgb_set_launch_shape(fvgb_mesh m, int32_t kernel, int32_t threads, int32_t ipt) {
  if (!m) { set_error("null mesh handle"); return FVGB_EINVAL; }
  if (kernel < 0 || kernel >= kTuneCount || threads < 32 || threads > 1024 || threads % 32 != 0 ||
      ipt < 1 || ipt > 64) {
    set_error("bad launch shape");
    return FVGB_EINVAL;
  }
  m->tune[kernel] = LaunchShape{threads, ipt};
  drop_graph(m);
  return FVGB_OK;
}
