// C ABI of libfvgb (declared in include/fvgb.h): mesh upload to the device, the
// finite-volume operators, the Poisson refinement loop and the streamer step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "internal.h"
#include "mesh_host.h"

namespace fvgb {

std::atomic<long long> g_kernel_launches{0};

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

fvgb_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return FVGB_OK;
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FVGB_ENOMEM : FVGB_ECUDA;
}

namespace {

#define FVGB_TRY(expr, what)                                   \
  do {                                                         \
    fvgb_status st_ = cuda_status((expr), (what));             \
    if (st_ != FVGB_OK) return st_;                            \
  } while (0)

template <typename T>
cudaError_t dalloc(fvgb_mesh_s* m, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e == cudaSuccess) m->allocs.push_back(q);
  *p = (T*)q;
  return e;
}

template <typename T>
cudaError_t dupload(fvgb_mesh_s* m, T** p, const std::vector<T>& h, cudaStream_t s) {
  cudaError_t e = dalloc(m, p, h.size());
  if (e != cudaSuccess || h.empty()) return e;
  return cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

template <typename T>
std::vector<T> cast(const std::vector<double>& v) {
  return std::vector<T>(v.begin(), v.end());
}

// Sliced ELL with 32-row slices; missing entries repeat pad_self ? the row itself : the
// row's first entry, with weight 0.
void build_sell(const std::vector<int32_t>& ptr, const std::vector<int32_t>& idx,
                const std::vector<double>* w, int64_t nrows, bool pad_self,
                std::vector<int64_t>& sptr, std::vector<int32_t>& sidx, std::vector<double>* sw) {
  const int64_t ns = (nrows + 31) / 32;
  sptr.assign(ns + 1, 0);
  for (int64_t s = 0; s < ns; ++s) {
    int64_t width = 0;
    for (int64_t r = s * 32; r < std::min(nrows, s * 32 + 32); ++r)
      width = std::max<int64_t>(width, ptr[r + 1] - ptr[r]);
    sptr[s + 1] = sptr[s] + width * 32;
  }
  sidx.assign(sptr[ns], 0);
  if (sw) sw->assign(sptr[ns], 0.0);
  for (int64_t s = 0; s < ns; ++s) {
    const int64_t width = (sptr[s + 1] - sptr[s]) / 32;
    for (int64_t r = s * 32; r < std::min(nrows, s * 32 + 32); ++r) {
      const int lane = (int)(r - s * 32);
      const int64_t cnt = ptr[r + 1] - ptr[r];
      for (int64_t k = 0; k < width; ++k) {
        const int64_t pos = sptr[s] + k * 32 + lane;
        if (k < cnt) {
          sidx[pos] = idx[ptr[r] + k];
          if (sw) (*sw)[pos] = (*w)[ptr[r] + k];
        } else {
          sidx[pos] = pad_self ? (int32_t)r : idx[ptr[r]];
        }
      }
    }
  }
}

template <typename T>
cudaError_t upload_geo(fvgb_mesh_s* m, const HostMesh& h, const std::vector<double>& sw,
                       GeoDev<T>& g, cudaStream_t s) {
  cudaError_t e;
  const bool lo = sizeof(T) == 4;
  auto hi_part = [&](const std::vector<double>& v) { return cast<T>(v); };
  auto lo_part = [&](const std::vector<double>& v) {
    std::vector<T> out(v.size());
    for (size_t i = 0; i < v.size(); ++i) out[i] = (T)(v[i] - (double)(T)v[i]);
    return out;
  };
  std::vector<double> inv_vol(h.vol.size());
  for (size_t i = 0; i < h.vol.size(); ++i) inv_vol[i] = 1.0 / h.vol[i];
  if ((e = dupload(m, &g.cen, hi_part(h.cen), s))) return e;
  if (lo && (e = dupload(m, &g.cen_lo, lo_part(h.cen), s))) return e;
  if ((e = dupload(m, &g.vol, cast<T>(h.vol), s))) return e;
  if ((e = dupload(m, &g.inv_vol, cast<T>(inv_vol), s))) return e;
  if ((e = dupload(m, &g.S, cast<T>(h.S), s))) return e;
  if ((e = dupload(m, &g.xf, hi_part(h.xf), s))) return e;
  if (lo && (e = dupload(m, &g.xf_lo, lo_part(h.xf), s))) return e;
  if ((e = dupload(m, &g.coef, cast<T>(h.coef), s))) return e;
  if ((e = dupload(m, &g.valpha, cast<T>(sw), s))) return e;
  g.bc.resize(h.bcs.size());
  for (size_t k = 0; k < h.bcs.size(); ++k) {
    const BCSetHost& b = h.bcs[k];
    BCDev<T>& d = g.bc[k];
    if ((e = dupload(m, &d.bkind, b.bkind, s))) return e;
    if ((e = dupload(m, &d.bval, cast<T>(b.bval), s))) return e;
    if ((e = dupload(m, &d.minv, cast<T>(b.minv), s))) return e;
    if ((e = dupload(m, &d.gptr, b.gptr, s))) return e;
    if ((e = dupload(m, &d.gface, b.gface, s))) return e;
    if ((e = dupload(m, &d.vdir, cast<T>(b.vdir), s))) return e;
    if ((e = dupload(m, &d.at_nbr, b.at_nbr, s))) return e;
    if ((e = dupload(m, &d.at_coef, cast<T>(b.at_coef), s))) return e;
    if ((e = dupload(m, &d.at_diag, cast<T>(b.at_diag), s))) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t alloc_work(fvgb_mesh_s* m, Work<T>& w) {
  const TopoDev& t = m->topo;
  cudaError_t e;
  if ((e = dalloc(m, &w.flux, t.F))) return e;
  if ((e = dalloc(m, &w.uv, t.V))) return e;
  if ((e = dalloc(m, &w.stage, t.N))) return e;
  if ((e = dalloc(m, &w.tmp, t.N))) return e;
  if ((e = dalloc(m, &w.vel, t.dim * t.N))) return e;
  if ((e = dalloc(m, &w.src, t.N))) return e;
  if ((e = dalloc(m, &w.grad, t.dim * t.N))) return e;
  if ((e = dalloc(m, &w.cg_r, t.N))) return e;
  if ((e = dalloc(m, &w.cg_p, t.N))) return e;
  if ((e = dalloc(m, &w.cg_q, t.N))) return e;
  if ((e = dalloc(m, &w.cg_x, t.N))) return e;
  return cudaSuccess;
}

void release(fvgb_mesh_s* m) {
  if (m->ev_cg0) cudaEventDestroy(m->ev_cg0);
  if (m->ev_cg1) cudaEventDestroy(m->ev_cg1);
  for (void* p : m->allocs) cudaFree(p);
  m->allocs.clear();
  if (m->h_scal) cudaFreeHost(m->h_scal);
  m->h_scal = nullptr;
  delete m;
}

fvgb_status check_mesh(fvgb_mesh m) {
  if (!m) { set_error("null mesh handle"); return FVGB_EINVAL; }
  return FVGB_OK;
}

fvgb_status check_bcset(fvgb_mesh m, int32_t k) {
  if (k < 0 || k >= (int32_t)m->g64.bc.size()) { set_error("bcset index out of range"); return FVGB_EINVAL; }
  return FVGB_OK;
}

bool is_fp32(fvgb_mesh m) { return m->prec != FVGB_FP64; }

// ---- transport residual / step in precision T --------------------------------------------
template <typename T>
fvgb_status residual_T(fvgb_mesh m, const fvgb_tcoef* tc, const T* u, T* res, cudaStream_t s) {
  Work<T>& w = work_of<T>(m);
  const bool diff = tc->diff != 0.0;
  if (diff) FVGB_TRY(launch_vertex<T>(m, tc->bcset, u, w.uv, false, s), "vertex kernel");
  FVGB_TRY(launch_face<T>(m, tc->bcset, u, w.uv, (const T*)tc->vel_dev, tc->vel_const, true,
                          tc->diff, false, w.flux, s), "face kernel");
  FVGB_TRY(launch_update<T>(m, kResidual, w.flux, (const T*)tc->src_dev, nullptr, 0.0, nullptr,
                            res, nullptr, s), "update kernel");
  return FVGB_OK;
}

template <typename T>
fvgb_status step_T(fvgb_mesh m, const fvgb_tcoef* tc, T* u, double dt, int nsteps,
                   const double* alpha, int nstage, T* ni_out, cudaStream_t s) {
  Work<T>& w = work_of<T>(m);
  const bool diff = tc->diff != 0.0;
  for (int n = 0; n < nsteps; ++n) {
    const T* in = u;
    for (int k = 0; k < nstage; ++k) {
      const bool last = k == nstage - 1;
      T* out = last ? u : (k % 2 == 0 ? w.stage : w.tmp);
      if (diff) FVGB_TRY(launch_vertex<T>(m, tc->bcset, in, w.uv, false, s), "vertex kernel");
      FVGB_TRY(launch_face<T>(m, tc->bcset, in, w.uv, (const T*)tc->vel_dev, tc->vel_const, true,
                              tc->diff, false, w.flux, s), "face kernel");
      FVGB_TRY(launch_update<T>(m, kStep, w.flux, (const T*)tc->src_dev, u, alpha[k] * dt, nullptr,
                                out, last ? ni_out : nullptr, s), "update kernel");
      in = out;
    }
  }
  return FVGB_OK;
}

// FP64 full diamond operator pieces
fvgb_status poisson_residual(fvgb_mesh m, int bcset, const double* x, const double* b, double* r,
                             cudaStream_t s) {
  Work<double>& w = m->w64;
  FVGB_TRY(launch_vertex<double>(m, bcset, x, w.uv, true, s), "vertex kernel");
  FVGB_TRY(launch_face<double>(m, bcset, x, w.uv, nullptr, nullptr, false, -1.0, true, w.flux, s), "face kernel");
  FVGB_TRY(launch_update<double>(m, b ? kPoissonResidual : kPoissonApply, w.flux, nullptr, nullptr,
                                 0.0, b, r, nullptr, s), "update kernel");
  return FVGB_OK;
}

fvgb_status poisson_rhs_impl(fvgb_mesh m, int bcset, const double* f, double* b, cudaStream_t s) {
  Work<double>& w = m->w64;
  FVGB_TRY(launch_vertex<double>(m, bcset, m->dzero, w.uv, false, s), "vertex kernel");
  FVGB_TRY(launch_face<double>(m, bcset, m->dzero, w.uv, nullptr, nullptr, false, -1.0, false, w.flux, s), "face kernel");
  FVGB_TRY(launch_update<double>(m, kPoissonRhs, w.flux, nullptr, nullptr, 0.0, f, b, nullptr, s), "update kernel");
  return FVGB_OK;
}

fvgb_status solve_impl(fvgb_mesh m, int bcset, const double* f, double* phi,
                       const fvgb_solve_opts* o, fvgb_solve_info* info, cudaStream_t s) {
  fvgb_solve_info loc{0, 0, 0.0, 0.0};
  const int64_t N = m->topo.N;
  m->stats.solves++;
  double* b = m->dphi_tmp2;
  double* r = m->dphi_tmp;
  fvgb_status st = poisson_rhs_impl(m, bcset, f, b, s);
  if (st) return st;
  FVGB_TRY(launch_sumsq(m, b, N, m->d_scal + 0, s), "reduction");
  FVGB_TRY(cudaMemcpyAsync(m->h_scal, m->d_scal, sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
  FVGB_TRY(cudaStreamSynchronize(s), "synchronize");
  const double bnorm = std::sqrt(m->h_scal[0]);
  loc.bnorm = bnorm;
  if (!std::isfinite(bnorm)) { set_error("non-finite right-hand side"); if (info) *info = loc; return FVGB_ENONFINITE; }
  if (bnorm == 0.0) {
    FVGB_TRY(cudaMemsetAsync(phi, 0, N * sizeof(double), s), "memset");
    if (info) *info = loc;
    return FVGB_OK;
  }
  const bool fp32 = o->prec == FVGB_FP32 || o->prec == FVGB_MIXED;
  if (fp32 && !is_fp32(m)) { set_error("FP32 inner solve needs a mesh uploaded with FVGB_FP32 or FVGB_MIXED"); return FVGB_EINVAL; }
  int* hinfo = (int*)(m->h_scal + 4);
  for (int outer = 0;; ++outer) {
    st = poisson_residual(m, bcset, phi, b, r, s);
    if (st) return st;
    FVGB_TRY(launch_sumsq(m, r, N, m->d_scal + 0, s), "reduction");
    FVGB_TRY(cudaMemcpyAsync(m->h_scal, m->d_scal, sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
    if (outer > 0) {
      FVGB_TRY(cudaMemcpyAsync(hinfo, m->d_cg_info, 2 * sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
      FVGB_TRY(cudaMemcpyAsync(hinfo + 2, &m->barrier->status, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
    }
    FVGB_TRY(cudaStreamSynchronize(s), "synchronize");
    if (m->cg_pending) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, m->ev_cg0, m->ev_cg1) == cudaSuccess) m->stats.cg_ms += ms;
      m->cg_pending = false;
    }
    if (outer > 0) {
      loc.inner_its_total += hinfo[0];
      m->stats.cg_iterations += hinfo[0];
      if (hinfo[2] != 0) { set_error("grid barrier of the CG kernel timed out"); if (info) *info = loc; return FVGB_ETIMEOUT; }
      if (hinfo[1] != 0) { set_error("CG breakdown or non-finite value"); if (info) *info = loc; return FVGB_ENONFINITE; }
    }
    loc.rel_res = std::sqrt(m->h_scal[0]) / bnorm;
    loc.outer_its = outer;
    if (outer > 0) m->stats.outer_its++;
    if (!std::isfinite(loc.rel_res)) { set_error("non-finite residual"); if (info) *info = loc; return FVGB_ENONFINITE; }
    if (loc.rel_res <= o->rtol) break;
    if (outer >= o->maxit_outer) {
      set_error("Poisson refinement did not reach rtol within maxit_outer");
      if (info) *info = loc;
      return FVGB_ENOCONV;
    }
    if (m->time_cg) FVGB_TRY(cudaEventRecord(m->ev_cg0, s), "event");
    if (fp32) FVGB_TRY(launch_cg<float>(m, bcset, r, o->inner_rtol, o->maxit_inner, s), "CG launch");
    else FVGB_TRY(launch_cg<double>(m, bcset, r, o->inner_rtol, o->maxit_inner, s), "CG launch");
    if (m->time_cg) {
      FVGB_TRY(cudaEventRecord(m->ev_cg1, s), "event");
      m->cg_pending = true;
    }
    m->stats.cg_launches++;
    if (fp32) FVGB_TRY(launch_add_to_double(m->w32.cg_x, true, phi, N, s), "update");
    else FVGB_TRY(launch_add_to_double(m->w64.cg_x, false, phi, N, s), "update");
  }
  if (info) *info = loc;
  return FVGB_OK;
}

bool opts_ok(const fvgb_solve_opts* o) {
  return o && o->rtol > 0.0 && o->inner_rtol > 0.0 && o->inner_rtol < 1.0 && o->maxit_inner > 0 &&
         o->maxit_outer >= 0 && (o->prec == FVGB_FP64 || o->prec == FVGB_FP32 || o->prec == FVGB_MIXED);
}

}  // namespace
}  // namespace fvgb

using namespace fvgb;

extern "C" {

const char* fvgb_last_error(void) { return g_last_error.c_str(); }

fvgb_status fvgb_mesh_upload(int32_t dim, int64_t n_vert, const double* xyz, int64_t n_cell,
                             const int32_t* cell_vert, int64_t n_bface, const int32_t* bface_vert,
                             const int32_t* bface_tag, int32_t n_bcset, const fvgb_bcset* bcsets,
                             int32_t reorder, int32_t prec, void* stream, fvgb_mesh* out) {
  set_error("");
  if (!out) { set_error("out is null"); return FVGB_EINVAL; }
  *out = nullptr;
  if (n_bcset < 1 || !bcsets) { set_error("at least one boundary-condition set is required"); return FVGB_EINVAL; }
  if (prec != FVGB_FP64 && prec != FVGB_FP32 && prec != FVGB_MIXED) { set_error("bad precision"); return FVGB_EINVAL; }
  std::vector<std::vector<BCInput>> sets(n_bcset);
  for (int k = 0; k < n_bcset; ++k) {
    if (bcsets[k].n_bc < 0 || (bcsets[k].n_bc > 0 && !bcsets[k].bc)) { set_error("bad bcset"); return FVGB_EINVAL; }
    for (int j = 0; j < bcsets[k].n_bc; ++j)
      sets[k].push_back(BCInput{bcsets[k].bc[j].tag, bcsets[k].bc[j].kind, bcsets[k].bc[j].value});
  }
  HostMesh h;
  std::string err;
  int rc = build_host_mesh(dim, n_vert, xyz, n_cell, cell_vert, n_bface, bface_vert, bface_tag,
                           sets, reorder, h, err);
  if (rc) { set_error(err); return (fvgb_status)rc; }

  cudaStream_t s = (cudaStream_t)stream;
  fvgb_mesh_s* m = new fvgb_mesh_s();
  m->prec = (fvgb_prec)prec;
  fvgb_status st = FVGB_OK;
  auto fail = [&](cudaError_t e, const char* what) {
    st = cuda_status(e, what);
    release(m);
    return st;
  };
  cudaError_t e;
  if ((e = cudaGetDevice(&m->device))) return fail(e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device))) return fail(e, "device attribute");
  TopoDev& t = m->topo;
  t.dim = h.dim; t.N = h.N; t.V = h.V; t.F = h.F; t.Fi = h.Fi; t.n_nbr = h.nptr[h.N];
  m->cell_perm_host = h.cell_perm;
  m->vert_perm_host = h.vert_perm;
  if ((e = dupload(m, &t.fL, h.fL, s))) return fail(e, "upload");
  if ((e = dupload(m, &t.fR, h.fR, s))) return fail(e, "upload");
  if ((e = dupload(m, &t.fvert, h.fvert, s))) return fail(e, "upload");
  if ((e = dupload(m, &t.cell_face, h.cell_face, s))) return fail(e, "upload");
  if ((e = dupload(m, &t.cell_perm, h.cell_perm, s))) return fail(e, "upload");
  std::vector<int64_t> sptr;
  std::vector<int32_t> sidx;
  build_sell(h.nptr, h.nidx, nullptr, h.N, true, sptr, sidx, nullptr);
  if ((e = dupload(m, &t.nsell.ptr, sptr, s))) return fail(e, "upload");
  if ((e = dupload(m, &t.nsell.idx, sidx, s))) return fail(e, "upload");
  std::vector<double> sw;
  build_sell(h.vptr, h.vcell, &h.valpha, h.V, false, sptr, sidx, &sw);
  if ((e = dupload(m, &t.vsell.ptr, sptr, s))) return fail(e, "upload");
  if ((e = dupload(m, &t.vsell.idx, sidx, s))) return fail(e, "upload");
  if ((e = upload_geo<double>(m, h, sw, m->g64, s))) return fail(e, "upload");
  if ((e = alloc_work<double>(m, m->w64))) return fail(e, "allocation");
  if (prec != FVGB_FP64) {
    if ((e = upload_geo<float>(m, h, sw, m->g32, s))) return fail(e, "upload");
    if ((e = alloc_work<float>(m, m->w32))) return fail(e, "allocation");
  }
  if ((e = dalloc(m, &m->d_scal, 8 + kRedBlocks + 2 * 8 * 1024))) return fail(e, "allocation");
  if ((e = dalloc(m, &m->dphi_tmp, h.N))) return fail(e, "allocation");
  if ((e = dalloc(m, &m->dphi_tmp2, h.N))) return fail(e, "allocation");
  if ((e = dalloc(m, &m->dzero, h.N))) return fail(e, "allocation");
  if ((e = cudaMemsetAsync(m->dzero, 0, h.N * sizeof(double), s))) return fail(e, "memset");
  if ((e = dalloc(m, &m->barrier, 1))) return fail(e, "allocation");
  if ((e = dalloc(m, &m->d_cg_info, 4))) return fail(e, "allocation");
  if ((e = cudaMallocHost((void**)&m->h_scal, 64 * sizeof(double)))) return fail(e, "pinned allocation");
  m->cg_grid64 = cg_grid_size(m, false);
  m->cg_grid32 = prec != FVGB_FP64 ? cg_grid_size(m, true) : 0;
  if (m->cg_grid64 <= 0 || (prec != FVGB_FP64 && m->cg_grid32 <= 0)) {
    set_error("this device cannot run the library's kernels (built for sm_103a)");
    release(m);
    return FVGB_EUNSUPPORTED;
  }
  if (m->cg_grid64 > 8 * 1024 || m->cg_grid32 > 8 * 1024) { set_error("too many SMs"); release(m); return FVGB_EUNSUPPORTED; }
  if ((e = cudaStreamSynchronize(s))) return fail(e, "synchronize");
  *out = m;
  return FVGB_OK;
}

fvgb_status fvgb_mesh_free(fvgb_mesh m) {
  if (!m) return FVGB_OK;
  cudaDeviceSynchronize();
  release(m);
  return FVGB_OK;
}

fvgb_status fvgb_stats_enable(fvgb_mesh m, int32_t time_cg) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (time_cg && !m->ev_cg0) {
    FVGB_TRY(cudaEventCreate(&m->ev_cg0), "event create");
    FVGB_TRY(cudaEventCreate(&m->ev_cg1), "event create");
  }
  m->time_cg = time_cg ? 1 : 0;
  return FVGB_OK;
}

fvgb_status fvgb_stats_get(fvgb_mesh m, fvgb_stats* out, int32_t reset) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (!out) { set_error("out is null"); return FVGB_EINVAL; }
  *out = m->stats;
  out->kernel_launches = g_kernel_launches.load();
  if (reset) {
    m->stats = fvgb_stats{};
    g_kernel_launches.store(0);
  }
  return FVGB_OK;
}

fvgb_status fvgb_mesh_info(fvgb_mesh m, int64_t* n_cell, int64_t* n_face, int64_t* n_vert,
                           int64_t* n_nbr) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (n_cell) *n_cell = m->topo.N;
  if (n_face) *n_face = m->topo.F;
  if (n_vert) *n_vert = m->topo.V;
  if (n_nbr) *n_nbr = m->topo.n_nbr;
  return FVGB_OK;
}

fvgb_status fvgb_mesh_cell_perm(fvgb_mesh m, int32_t* perm_host) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (!perm_host) { set_error("perm_host is null"); return FVGB_EINVAL; }
  std::memcpy(perm_host, m->cell_perm_host.data(), m->cell_perm_host.size() * sizeof(int32_t));
  return FVGB_OK;
}

fvgb_status fvgb_mesh_vert_perm(fvgb_mesh m, int32_t* perm_host) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (!perm_host) { set_error("perm_host is null"); return FVGB_EINVAL; }
  std::memcpy(perm_host, m->vert_perm_host.data(), m->vert_perm_host.size() * sizeof(int32_t));
  return FVGB_OK;
}

fvgb_status fvgb_permute(fvgb_mesh m, const void* src, void* dst, int32_t n_comp, int32_t elem_bytes,
                         int32_t to_internal, void* stream) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (!src || !dst || src == dst || n_comp < 1 || (elem_bytes != 4 && elem_bytes != 8)) {
    set_error("bad permute arguments");
    return FVGB_EINVAL;
  }
  return cuda_status(launch_permute(src, dst, m->topo.cell_perm, m->topo.N, n_comp, elem_bytes,
                                    to_internal != 0, (cudaStream_t)stream), "permute kernel");
}

fvgb_status fvgb_gradient(fvgb_mesh m, int32_t bcset, const void* u, void* grad, void* stream) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (fvgb_status st = check_bcset(m, bcset)) return st;
  if (!u || !grad) { set_error("null array"); return FVGB_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  if (is_fp32(m)) return cuda_status(launch_gradient<float>(m, bcset, (const float*)u, (float*)grad, s), "gradient kernel");
  return cuda_status(launch_gradient<double>(m, bcset, (const double*)u, (double*)grad, s), "gradient kernel");
}

fvgb_status fvgb_vertex_values(fvgb_mesh m, int32_t bcset, const void* u, void* uv, void* stream) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (fvgb_status st = check_bcset(m, bcset)) return st;
  if (!u || !uv) { set_error("null array"); return FVGB_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  if (is_fp32(m)) return cuda_status(launch_vertex<float>(m, bcset, (const float*)u, (float*)uv, false, s), "vertex kernel");
  return cuda_status(launch_vertex<double>(m, bcset, (const double*)u, (double*)uv, false, s), "vertex kernel");
}

static fvgb_status check_tcoef(fvgb_mesh m, const fvgb_tcoef* tc) {
  if (!tc) { set_error("tcoef is null"); return FVGB_EINVAL; }
  if (tc->recon != 0) { set_error("only first-order upwind (recon = 0) is implemented"); return FVGB_EUNSUPPORTED; }
  if (!(tc->diff >= 0.0)) { set_error("diffusivity must be >= 0"); return FVGB_EINVAL; }
  return check_bcset(m, tc->bcset);
}

fvgb_status fvgb_fv_residual(fvgb_mesh m, const fvgb_tcoef* tc, const void* u, void* res, void* stream) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (fvgb_status st = check_tcoef(m, tc)) return st;
  if (!u || !res || u == res) { set_error("u and res must be distinct device arrays"); return FVGB_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  if (is_fp32(m)) return residual_T<float>(m, tc, (const float*)u, (float*)res, s);
  return residual_T<double>(m, tc, (const double*)u, (double*)res, s);
}

fvgb_status fvgb_fv_step(fvgb_mesh m, const fvgb_tcoef* tc, void* u, double dt, int32_t nsteps,
                         const double* stage_alpha, int32_t nstage, void* stream) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (fvgb_status st = check_tcoef(m, tc)) return st;
  static const double euler[1] = {1.0};
  if (!stage_alpha) { stage_alpha = euler; nstage = 1; }
  if (!u || nsteps < 0 || nstage < 1 || nstage > 8 || !std::isfinite(dt)) { set_error("bad step arguments"); return FVGB_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  if (is_fp32(m)) return step_T<float>(m, tc, (float*)u, dt, nsteps, stage_alpha, nstage, nullptr, s);
  return step_T<double>(m, tc, (double*)u, dt, nsteps, stage_alpha, nstage, nullptr, s);
}

fvgb_status fvgb_poisson_apply(fvgb_mesh m, int32_t bcset, const double* x, double* y, void* stream) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (fvgb_status st = check_bcset(m, bcset)) return st;
  if (!x || !y || x == y) { set_error("x and y must be distinct device arrays"); return FVGB_EINVAL; }
  return poisson_residual(m, bcset, x, nullptr, y, (cudaStream_t)stream);
}

fvgb_status fvgb_poisson_rhs(fvgb_mesh m, int32_t bcset, const double* f, double* b, void* stream) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (fvgb_status st = check_bcset(m, bcset)) return st;
  if (!b) { set_error("b is null"); return FVGB_EINVAL; }
  return poisson_rhs_impl(m, bcset, f, b, (cudaStream_t)stream);
}

fvgb_status fvgb_poisson_solve(fvgb_mesh m, int32_t bcset, const double* f, double* phi,
                               const fvgb_solve_opts* o, fvgb_solve_info* info, void* stream) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (fvgb_status st = check_bcset(m, bcset)) return st;
  if (!phi || !opts_ok(o)) { set_error("bad solve arguments"); return FVGB_EINVAL; }
  return solve_impl(m, bcset, f, phi, o, info, (cudaStream_t)stream);
}

fvgb_status fvgb_streamer_step(fvgb_mesh m, const fvgb_streamer_params* p, void* ne, void* ni,
                               double* phi, void* E, int32_t nsteps, fvgb_solve_info* info,
                               void* stream) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (!p || !ne || !ni || !phi || nsteps < 0 || !opts_ok(&p->solve)) { set_error("bad streamer arguments"); return FVGB_EINVAL; }
  if (fvgb_status st = check_bcset(m, p->bcset_ne)) return st;
  if (fvgb_status st = check_bcset(m, p->bcset_phi)) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = m->topo.N;
  const bool fp32 = is_fp32(m);
  double* f = m->w64.tmp;   // FP64 scratch of the mesh (unused by the FP64 transport path)
  for (int n = 0; n < nsteps; ++n) {
    fvgb_status st = cuda_status(launch_poisson_source(m, ne, ni, fp32, f, s), "source kernel");
    if (st) return st;
    st = solve_impl(m, p->bcset_phi, f, phi, &p->solve, info ? info + n : nullptr, s);
    if (st) return st;
    fvgb_tcoef tc;
    std::memset(&tc, 0, sizeof(tc));
    tc.diff = p->De;
    tc.bcset = p->bcset_ne;
    static const double euler[1] = {1.0};
    if (fp32) {
      Work<float>& w = m->w32;
      FVGB_TRY(launch_convert(phi, w.tmp, N, s), "convert");
      FVGB_TRY(launch_gradient<float>(m, p->bcset_phi, w.tmp, w.grad, s), "gradient kernel");
      FVGB_TRY(launch_cell_physics<float>(m, w.grad, (const float*)ne, p->mu, p->A, p->B, (float*)E,
                                          w.vel, w.src, s), "cell kernel");
      tc.vel_dev = w.vel;
      tc.src_dev = w.src;
      st = step_T<float>(m, &tc, (float*)ne, p->dt, 1, euler, 1, (float*)ni, s);
    } else {
      Work<double>& w = m->w64;
      FVGB_TRY(launch_gradient<double>(m, p->bcset_phi, phi, w.grad, s), "gradient kernel");
      FVGB_TRY(launch_cell_physics<double>(m, w.grad, (const double*)ne, p->mu, p->A, p->B,
                                           (double*)E, w.vel, w.src, s), "cell kernel");
      tc.vel_dev = w.vel;
      tc.src_dev = w.src;
      st = step_T<double>(m, &tc, (double*)ne, p->dt, 1, euler, 1, (double*)ni, s);
    }
    if (st) return st;
  }
  return FVGB_OK;
}

}  // extern "C"
