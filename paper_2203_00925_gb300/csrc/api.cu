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

// Halo lists of the shared-memory gradient (see TopoDev): per tile of kGradTile rows, its
// own rows, then every other cell met in the rows' padded node-neighbour lists (sorted);
// lidx[pos] is the position of sidx[pos] in its row's tile list. Returns the longest list.
// Order each lane's neighbour entries of a SELL-32 slice so that, column by column, the
// eight lanes of a quarter warp read records in different shared-memory bank groups
// (record k of 16 bytes sits in group k % 8; a quarter warp's 16-byte reads are served in
// one pass when their groups differ, or when they read the same record). Greedy: per
// column and quarter, each lane takes an entry of the least used group it still has. The
// least-squares sum is the same set of terms in another order.
void order_slice_for_banks(int16_t* lid, int width) {
  thread_local std::vector<int16_t> bucket[32][8];   // reused across slices
  for (int lane = 0; lane < 32; ++lane) {
    for (int g = 0; g < 8; ++g) bucket[lane][g].clear();
    for (int c = width - 1; c >= 0; --c) {            // popped from the back: original order
      const int16_t v = lid[32 * c + lane];
      bucket[lane][v & 7].push_back(v);
    }
  }
  for (int c = 0; c < width; ++c) {
    for (int qw = 0; qw < 4; ++qw) {
      int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};          // distinct records read in each group
      int first[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
      for (int lane = 8 * qw; lane < 8 * qw + 8; ++lane) {
        int best = -1, best_cost = 1 << 30;
        for (int g = 0; g < 8; ++g) {
          if (bucket[lane][g].empty()) continue;
          // a record another lane of the quarter already reads costs nothing
          const int cost = bucket[lane][g].back() == first[g] ? 0 : cnt[g] + 1;
          if (cost < best_cost) { best = g; best_cost = cost; }
        }
        const int16_t v = bucket[lane][best].back();
        bucket[lane][best].pop_back();
        if (first[best] < 0) first[best] = v;
        if (best_cost > 0) cnt[best] += 1;
        lid[32 * c + lane] = v;
      }
    }
  }
}

int build_grad_tiles(int64_t N, const std::vector<int64_t>& sptr, const std::vector<int32_t>& sidx,
                     std::vector<int32_t>& tptr, std::vector<int32_t>& tidx, std::vector<int16_t>& lidx) {
  const int64_t ntile = (N + kGradTile - 1) / kGradTile;
  std::vector<std::vector<int32_t>> lists(ntile);
  lidx.assign(sidx.size(), 0);
  int max_len = 0;
#pragma omp parallel reduction(max : max_len)
  {
    std::vector<int32_t> stamp(N, -1), pos(N, 0);
#pragma omp for schedule(dynamic, 64)
    for (int64_t t = 0; t < ntile; ++t) {
      const int64_t r0 = t * kGradTile, r1 = std::min<int64_t>(N, r0 + kGradTile);
      std::vector<int32_t>& L = lists[t];
      for (int64_t r = r0; r < r1; ++r) { stamp[r] = (int32_t)t; L.push_back((int32_t)r); }
      const int64_t s0 = r0 / 32, s1 = (r1 + 31) / 32;
      const size_t own = L.size();
      for (int64_t q = sptr[s0]; q < sptr[s1]; ++q) {
        const int32_t j = sidx[q];
        if (stamp[j] != (int32_t)t) { stamp[j] = (int32_t)t; L.push_back(j); }
      }
      std::sort(L.begin() + own, L.end());
      for (size_t k = 0; k < L.size(); ++k) pos[L[k]] = (int32_t)k;
      if (L.size() <= 32767) {
        for (int64_t q = sptr[s0]; q < sptr[s1]; ++q) lidx[q] = (int16_t)pos[sidx[q]];
        for (int64_t sl = s0; sl < s1; ++sl)
          order_slice_for_banks(lidx.data() + sptr[sl], (int)((sptr[sl + 1] - sptr[sl]) / 32));
      }
      max_len = std::max(max_len, (int)L.size());
    }
  }
  tptr.assign(ntile + 1, 0);
  for (int64_t t = 0; t < ntile; ++t) tptr[t + 1] = tptr[t] + (int32_t)lists[t].size();
  tidx.resize(tptr[ntile]);
  for (int64_t t = 0; t < ntile; ++t) std::copy(lists[t].begin(), lists[t].end(), tidx.begin() + tptr[t]);
  return max_len;
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
  {
    const int d = h.dim;
    std::vector<double> xv((size_t)d * h.V);
    for (int64_t v = 0; v < h.V; ++v)
      for (int a = 0; a < d; ++a) xv[a * h.V + v] = h.xyz[v * d + a];
    if ((e = dupload(m, &g.xv, hi_part(xv), s))) return e;
    if (lo && (e = dupload(m, &g.xv_lo, lo_part(xv), s))) return e;
    if ((e = dupload(m, &g.vs1, cast<T>(h.vs1), s))) return e;
  }
  g.bc.resize(h.bcs.size());
  for (size_t k = 0; k < h.bcs.size(); ++k) {
    const BCSetHost& b = h.bcs[k];
    BCDev<T>& d = g.bc[k];
    if ((e = dupload(m, &d.bkind, b.bkind, s))) return e;
    if ((e = dupload(m, &d.bval, cast<T>(b.bval), s))) return e;
    if ((e = dupload(m, &d.minv, cast<T>(b.minv), s))) return e;
    if ((e = dupload(m, &d.gptr, b.gptr, s))) return e;
    if ((e = dupload(m, &d.gface, b.gface, s))) return e;
    if ((e = dupload(m, &d.gmult, b.gmult, s))) return e;
    if ((e = dupload(m, &d.minv_v, cast<T>(b.minv_v), s))) return e;
    if ((e = dupload(m, &d.vdir, cast<T>(b.vdir), s))) return e;
    if ((e = dupload(m, &d.at_nbr, b.at_nbr, s))) return e;
    if ((e = dupload(m, &d.at_coef, cast<T>(b.at_coef), s))) return e;
    if ((e = dupload(m, &d.at_diag, cast<T>(b.at_diag), s))) return e;
    if ((e = dupload(m, &d.at_scoef, cast<T>(b.at_scoef), s))) return e;
    if ((e = dupload(m, &d.at_isd, cast<T>(b.at_isd), s))) return e;
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
  if ((e = dalloc(m, &w.grec, (sizeof(T) == 4 ? 8 : 4) * t.N))) return e;
  if ((e = dalloc(m, &w.vsum, 5 * t.V))) return e;
  if ((e = dalloc(m, &w.cg_r, t.N))) return e;
  if ((e = dalloc(m, &w.cg_p, t.N))) return e;
  if ((e = dalloc(m, &w.cg_q, t.N))) return e;
  if ((e = dalloc(m, &w.cg_x, t.N))) return e;
  return cudaSuccess;
}

// Sub-chunks of the persistent solve: block b owns rows [b N / G, (b+1) N / G), cut at
// part boundaries; parts are contiguous ranges of internal cells.
cudaError_t setup_parts(fvgb_mesh_s* m, const std::vector<int64_t>& part_begin, cudaStream_t s) {
  const int64_t N = m->topo.N;
  const int G = m->solve_grid;
  const int P = (int)part_begin.size() - 1;
  m->part_cell_begin = part_begin;
  std::vector<int32_t> blk_sc(G + 1, 0), sc_part, part_sc(P + 1, 0);
  std::vector<int64_t> sc_begin;
  int p = 0;
  for (int b = 0; b < G; ++b) {
    blk_sc[b] = (int32_t)sc_part.size();
    const int64_t lo = (int64_t)b * N / G, hi = (int64_t)(b + 1) * N / G;
    int64_t i = lo;
    while (i < hi) {
      while (part_begin[p + 1] <= i) ++p;
      sc_begin.push_back(i);
      sc_part.push_back(p);
      i = std::min(hi, part_begin[p + 1]);
    }
  }
  blk_sc[G] = (int32_t)sc_part.size();
  sc_begin.push_back(N);
  const int n_sc = (int)sc_part.size();
  for (int q = 0, sc = 0; q <= P; ++q) {
    while (sc < n_sc && sc_part[sc] < q) ++sc;
    part_sc[q] = sc;
  }
  PartsDev& pd = m->parts;
  pd.n_part = P;
  pd.n_sc = n_sc;
  cudaError_t e;
  if ((e = dupload(m, &pd.blk_sc, blk_sc, s))) return e;
  if ((e = dupload(m, &pd.sc_begin, sc_begin, s))) return e;
  if ((e = dupload(m, &pd.sc_part, sc_part, s))) return e;
  if ((e = dupload(m, &pd.part_sc, part_sc, s))) return e;
  if ((e = dalloc(m, &pd.buf, 4 * (size_t)n_sc))) return e;
  if ((e = dalloc(m, &pd.active, P))) return e;
  if ((e = dalloc(m, &pd.out_inner, P))) return e;
  if ((e = dalloc(m, &pd.norms, P))) return e;
  return cudaSuccess;
}

void release(fvgb_mesh_s* m) {
  graph_release(m);
  amg_release(m);
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

}  // namespace
bool is_fp32(fvgb_mesh m) { return m->prec != FVGB_FP64; }
namespace {

// ---- transport residual / step in precision T --------------------------------------------
// MUSCL (eq. 15): least-squares gradient of u, limited in place
template <typename T>
fvgb_status limited_gradient(fvgb_mesh m, const fvgb_tcoef* tc, const T* u, cudaStream_t s) {
  Work<T>& w = work_of<T>(m);
  FVGB_TRY(launch_gradient<T>(m, tc->bcset, u, w.grad, s), "gradient kernel");
  FVGB_TRY(launch_bj_limit<T>(m, tc->bcset, u, w.grad, s), "limiter kernel");
  return FVGB_OK;
}

template <typename T>
fvgb_status residual_T(fvgb_mesh m, const fvgb_tcoef* tc, const T* u, T* res, cudaStream_t s) {
  Work<T>& w = work_of<T>(m);
  const bool diff = tc->diff != 0.0;
  if (tc->recon) FVGB_TRY_ST(limited_gradient<T>(m, tc, u, s));
  if (diff) FVGB_TRY(launch_vertex<T>(m, tc->bcset, u, w.uv, false, s), "vertex kernel");
  FVGB_TRY(launch_face<T>(m, tc->bcset, u, w.uv, (const T*)tc->vel_dev, tc->vel_const, true,
                          tc->diff, false, w.flux, s, tc->recon ? w.grad : nullptr), "face kernel");
  FVGB_TRY(launch_update<T>(m, kResidual, w.flux, (const T*)tc->src_dev, nullptr, 0.0, nullptr,
                            res, nullptr, s), "update kernel");
  return FVGB_OK;
}

}  // namespace
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
      if (tc->recon) FVGB_TRY_ST(limited_gradient<T>(m, tc, in, s));
      if (diff) FVGB_TRY(launch_vertex<T>(m, tc->bcset, in, w.uv, false, s), "vertex kernel");
      FVGB_TRY(launch_face<T>(m, tc->bcset, in, w.uv, (const T*)tc->vel_dev, tc->vel_const, true,
                              tc->diff, false, w.flux, s, tc->recon ? w.grad : nullptr), "face kernel");
      FVGB_TRY(launch_update<T>(m, kStep, w.flux, (const T*)tc->src_dev, u, alpha[k] * dt, nullptr,
                                out, last ? ni_out : nullptr, s), "update kernel");
      in = out;
    }
  }
  return FVGB_OK;
}
template fvgb_status step_T<float>(fvgb_mesh, const fvgb_tcoef*, float*, double, int, const double*, int, float*, cudaStream_t);
template fvgb_status step_T<double>(fvgb_mesh, const fvgb_tcoef*, double*, double, int, const double*, int, double*, cudaStream_t);

namespace {
// One stage of eq. 6 for the transport: u = base + adt Res(u) (the residual at the current
// u; the update reads base, so u may be overwritten in place) and ni += adt S.
template <typename T>
fvgb_status transport_stage(fvgb_mesh m, const fvgb_tcoef* tc, const T* base, T* u, T* ni, double adt,
                            cudaStream_t s) {
  Work<T>& w = work_of<T>(m);
  if (tc->recon) FVGB_TRY_ST(limited_gradient<T>(m, tc, u, s));
  if (tc->diff != 0.0) FVGB_TRY(launch_vertex<T>(m, tc->bcset, u, w.uv, false, s), "vertex kernel");
  FVGB_TRY(launch_face<T>(m, tc->bcset, u, w.uv, (const T*)tc->vel_dev, tc->vel_const, true,
                          tc->diff, false, w.flux, s, tc->recon ? w.grad : nullptr), "face kernel");
  FVGB_TRY(launch_update<T>(m, kStep, w.flux, (const T*)tc->src_dev, base, adt, nullptr, u, ni, s),
           "update kernel");
  return FVGB_OK;
}
}  // namespace

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

namespace {
// Outer FP64 refinement loop, per part: r = b - A phi, stop a part when
// ||r_p|| <= rtol ||b_p||, otherwise one inner CG solve of A_T delta = r on the parts
// still active and phi += delta. One host synchronisation per outer step.
fvgb_status solve_impl(fvgb_mesh m, int bcset, const double* f, double* phi,
                       const fvgb_solve_opts* o, fvgb_solve_info* info, cudaStream_t s) {
  fvgb_solve_info loc{0, 0, 0.0, 0.0};
  m->stats.solves++;
  const int64_t N = m->topo.N;
  const int P = m->parts.n_part;
  const bool fp32 = o->prec == FVGB_FP32 || o->prec == FVGB_MIXED;
  if (fp32 && !is_fp32(m)) { set_error("FP32 inner solve needs a mesh uploaded with FVGB_FP32 or FVGB_MIXED"); return FVGB_EINVAL; }
  double* b = m->dphi_tmp2;
  double* r = m->dphi_tmp;
  // after a learned start of a streamer step, b and the start's residual are already formed
  const bool primed = m->solve_primed == bcset;
  m->solve_primed = -1;
  if (o->inner > 0) FVGB_TRY_ST(amg_ensure(m, bcset, fp32, s));
  fvgb_status st = primed ? FVGB_OK : poisson_rhs_impl(m, bcset, f, b, s);
  if (st) return st;
  // host staging in pinned memory: [0, P) norms, [P, 2P) ints (active flags, inner its)
  double* hn = m->h_scal + 8;
  int* hact = (int*)(m->h_scal + 8 + P);
  int* hinner = hact + P;
  int* hst = hinner + P;                    // [0] CG status, [1] CG its, [2] barrier status,
                                            // [3] latched transport status
  FVGB_TRY(launch_part_sumsq(m, b, m->parts.norms, s), "norm kernel");
  FVGB_TRY(cudaMemcpyAsync(hn, m->parts.norms, P * sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
  FVGB_TRY(cudaMemcpyAsync(hst + 3, m->d_status, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
  const bool count_warm = m->warm_check_pending;
  if (count_warm) FVGB_TRY(cudaMemcpyAsync(hact, m->warm_used, P * sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
  m->warm_check_pending = false;
  FVGB_TRY(cudaStreamSynchronize(s), "synchronize");
  if (count_warm) {
    m->stats.learned_starts += P;
    for (int p = 0; p < P; ++p) m->stats.learned_kept += hact[p] ? 1 : 0;
  }
  if (hst[3] != 0) {
    FVGB_TRY(cudaMemsetAsync(m->d_status, 0, sizeof(int), s), "memset");
    if (info) *info = loc;
    if (hst[3] & 2) {
      set_error("a tensor-core wait of the learned start timed out (latched status)");
      return FVGB_ETIMEOUT;
    }
    set_error("an earlier transport call produced a non-finite value (latched status)");
    return FVGB_ENONFINITE;
  }
  std::vector<double> bn2(hn, hn + P);
  double bsum = 0.0;
  bool any_zero = false;
  for (int p = 0; p < P; ++p) {
    bsum += bn2[p];
    if (!std::isfinite(bn2[p])) { set_error("non-finite right-hand side"); if (info) *info = loc; return FVGB_ENONFINITE; }
    if (bn2[p] == 0.0) any_zero = true;
  }
  loc.bnorm = std::sqrt(bsum);
  if (any_zero) {   // a part with b = 0 has the solution 0 (and then the residual 0)
    for (int p = 0; p < P; ++p)
      if (bn2[p] == 0.0) {
        const size_t bytes = (m->part_cell_begin[p + 1] - m->part_cell_begin[p]) * sizeof(double);
        FVGB_TRY(cudaMemsetAsync(phi + m->part_cell_begin[p], 0, bytes, s), "memset");
        if (primed) FVGB_TRY(cudaMemsetAsync(r + m->part_cell_begin[p], 0, bytes, s), "memset");
      }
  }
  m->last_outer.assign(P, 0);
  m->last_inner.assign(P, 0);
  m->last_rel.assign(P, 0.0);
  for (int outer = 0;; ++outer) {
    if (!(primed && outer == 0)) {
      st = poisson_residual(m, bcset, phi, b, r, s);
      if (st) return st;
    }
    FVGB_TRY(launch_part_sumsq(m, r, m->parts.norms, s), "norm kernel");
    FVGB_TRY(cudaMemcpyAsync(hn, m->parts.norms, P * sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
    if (outer > 0) {
      FVGB_TRY(cudaMemcpyAsync(hinner, m->parts.out_inner, P * sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
      FVGB_TRY(cudaMemcpyAsync(hst, m->d_cg_info, 2 * sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
      FVGB_TRY(cudaMemcpyAsync(hst + 2, &m->barrier->status, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
    }
    FVGB_TRY(cudaStreamSynchronize(s), "synchronize");
    if (m->cg_pending) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, m->ev_cg0, m->ev_cg1) == cudaSuccess) m->stats.cg_ms += ms;
      m->cg_pending = false;
    }
    if (outer > 0) {
      m->stats.cg_iterations += hst[1];
      int mx = 0;
      for (int p = 0; p < P; ++p) {
        m->last_inner[p] += hinner[p];
        mx = std::max(mx, m->last_inner[p]);
      }
      loc.inner_its_total = mx;
      if (hst[2] != 0) { set_error("a grid barrier of the CG kernel timed out"); if (info) *info = loc; return FVGB_ETIMEOUT; }
      if (hst[0] != 0) { set_error("CG breakdown or non-finite value"); if (info) *info = loc; return FVGB_ENONFINITE; }
    }
    int n_active = 0;
    loc.rel_res = 0.0;
    for (int p = 0; p < P; ++p) {
      const double rel = bn2[p] > 0.0 ? std::sqrt(hn[p] / bn2[p]) : 0.0;
      if (!std::isfinite(rel)) { set_error("non-finite residual"); if (info) *info = loc; return FVGB_ENONFINITE; }
      m->last_rel[p] = rel;
      loc.rel_res = std::max(loc.rel_res, rel);
      hact[p] = rel > o->rtol ? 1 : 0;
      n_active += hact[p];
    }
    loc.outer_its = outer;
    if (n_active == 0) break;
    if (outer >= o->maxit_outer) {
      set_error("Poisson refinement did not reach rtol within maxit_outer");
      if (info) *info = loc;
      return FVGB_ENOCONV;
    }
    for (int p = 0; p < P; ++p) m->last_outer[p] += hact[p];
    m->stats.outer_its++;
    FVGB_TRY(cudaMemcpyAsync(m->parts.active, hact, P * sizeof(int), cudaMemcpyHostToDevice, s), "copy");
    if (m->time_cg) FVGB_TRY(cudaEventRecord(m->ev_cg0, s), "event");
    if (fp32) FVGB_TRY(launch_inner<float>(m, bcset, r, o, s), "inner solve");
    else FVGB_TRY(launch_inner<double>(m, bcset, r, o, s), "inner solve");
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

}  // namespace

bool warm_requested(const fvgb_streamer_params* p) { return p->warm || p->extrapolate; }

// Warm start of the Poisson solve of a streamer step, given ``hist`` earlier steps:
//  - charge history: dq = change of n_i - n_e since the previous step, d2q its change;
//  - base start: phi (the previous potential), or with extrapolation and two earlier
//    steps 2 phi - phi_old (linear in time);
//  - learned correction (when p->warm): the network's increment pred from dq (base = phi)
//    or from d2q (base = extrapolation, whose error is the increment's change), added per
//    part in full where phi + pred has the smaller FP64 residual (r1 = b - A (phi + pred)
//    against r0 = b - A phi), elsewhere scaled by s = <r0, A pred> / ||A pred||^2 (with
//    A pred = r0 - r1), the scale that minimises ||b - A (phi + s pred)||. Either way the
//    start's residual is not larger than without the network.
fvgb_status warm_start(fvgb_mesh m, const fvgb_streamer_params* p, void* ne, void* ni, double* phi,
                       int hist, cudaStream_t s) {
  const int64_t N = m->topo.N;
  const int P = m->parts.n_part;
  m->solve_primed = -1;
  if (!m->q_prev) {
    FVGB_TRY(dalloc(m, &m->q_prev, N), "allocation");
    FVGB_TRY(dalloc(m, &m->dq, N), "allocation");
    FVGB_TRY(dalloc(m, &m->d2q, N), "allocation");
    FVGB_TRY(dalloc(m, &m->phi_old, N), "allocation");
    FVGB_TRY(dalloc(m, &m->phi_old2, N), "allocation");
    FVGB_TRY(dalloc(m, &m->dphi_pred, N), "allocation");
    FVGB_TRY(dalloc(m, &m->phi_save, N), "allocation");
    FVGB_TRY(dalloc(m, &m->warm_norms, 4 * P), "allocation");
    FVGB_TRY(dalloc(m, &m->warm_used, P), "allocation");
    FVGB_TRY(dalloc(m, &m->warm_scale, P), "allocation");
  }
  FVGB_TRY(launch_charge_hist(m, ne, ni, is_fp32(m), hist, m->q_prev, m->dq, m->d2q, s), "charge kernel");
  const bool extrap = p->extrapolate && hist >= 2;
  FVGB_TRY(launch_extrapolate(m, extrap, phi, m->phi_old, m->phi_old2, s), "extrapolation kernel");
  const bool learn = p->warm && hist >= (p->extrapolate ? 2 : 1);
  if (!learn) return FVGB_OK;
  double* f = m->w64.tmp;
  double* b = m->dphi_tmp2;
  double* r0 = m->dphi_tmp;
  FVGB_TRY(launch_poisson_source(m, ne, ni, is_fp32(m), f, s), "source kernel");
  if (fvgb_status st = poisson_rhs_impl(m, p->bcset_phi, f, b, s)) return st;
  double* r1 = f;                      // the source is no longer needed once b is formed
  FVGB_TRY(cudaMemcpyAsync(m->phi_save, phi, N * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
  if (fvgb_status st = poisson_residual(m, p->bcset_phi, phi, b, r0, s)) return st;
  if (fvgb_status st = fvgb_mpnn_predict(p->warm, p->extrapolate ? m->d2q : m->dq, m->phi_old,
                                         m->dphi_pred, s)) return st;
  FVGB_TRY(launch_axpy_d(m->dphi_pred, 1.0, phi, N, s), "update");
  if (fvgb_status st = poisson_residual(m, p->bcset_phi, phi, b, r1, s)) return st;
  // r0 - r1 = A pred: the residual-minimising scale of the correction, per part
  FVGB_TRY(launch_part_dots(m, r0, r1, m->warm_norms, s), "dot kernel");
  m->warm_check_pending = true;
  FVGB_TRY(launch_scale_start(m, m->warm_norms, m->phi_save, m->dphi_pred, phi, m->warm_used, m->warm_scale,
                              r0, r1, s), "start kernel");
  // b and the start's residual are in place for this step's solve (same source, same set)
  m->solve_primed = p->bcset_phi;
  return FVGB_OK;
}

// Field, cell physics and one transport stage of eq. 6 (after the stage's solve):
// ne = ne0 + alpha dt Res(ne), ni = ni0 + alpha dt S, with the field from phi and the
// source from the current ne.
fvgb_status streamer_transport_stage(fvgb_mesh m, const fvgb_streamer_params* p, const void* ne0,
                                     const void* ni0, void* ne, void* ni, const double* phi, void* E,
                                     double alpha, cudaStream_t s) {
  const int64_t N = m->topo.N;
  fvgb_tcoef tc;
  std::memset(&tc, 0, sizeof(tc));
  tc.diff = p->De;
  tc.bcset = p->bcset_ne;
  tc.recon = p->recon;
  if (is_fp32(m)) {
    Work<float>& w = m->w32;
    FVGB_TRY(launch_convert(phi, w.tmp, N, s), "convert");
    FVGB_TRY(launch_gradient<float>(m, p->bcset_phi, w.tmp, w.grad, s), "gradient kernel");
    FVGB_TRY(launch_cell_physics<float>(m, w.grad, (const float*)ne, p->mu, p->A, p->B, (float*)E,
                                        w.vel, w.src, spot_args(m, p), s), "cell kernel");
    FVGB_TRY(cudaMemcpyAsync(ni, ni0, N * sizeof(float), cudaMemcpyDeviceToDevice, s), "copy");
    tc.vel_dev = w.vel;
    tc.src_dev = w.src;
    return transport_stage<float>(m, &tc, (const float*)ne0, (float*)ne, (float*)ni, alpha * p->dt, s);
  }
  Work<double>& w = m->w64;
  FVGB_TRY(launch_gradient<double>(m, p->bcset_phi, phi, w.grad, s), "gradient kernel");
  FVGB_TRY(launch_cell_physics<double>(m, w.grad, (const double*)ne, p->mu, p->A, p->B, (double*)E,
                                       w.vel, w.src, spot_args(m, p), s), "cell kernel");
  FVGB_TRY(cudaMemcpyAsync(ni, ni0, N * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
  tc.vel_dev = w.vel;
  tc.src_dev = w.src;
  return transport_stage<double>(m, &tc, (const double*)ne0, (double*)ne, (double*)ni, alpha * p->dt, s);
}

// Field, cell physics and the transport update of one streamer step (after the solve).
fvgb_status streamer_transport(fvgb_mesh m, const fvgb_streamer_params* p, void* ne, void* ni,
                               const double* phi, void* E, cudaStream_t s) {
  const int64_t N = m->topo.N;
  fvgb_tcoef tc;
  std::memset(&tc, 0, sizeof(tc));
  tc.diff = p->De;
  tc.bcset = p->bcset_ne;
  tc.recon = p->recon;
  static const double euler[1] = {1.0};
  if (is_fp32(m)) {
    Work<float>& w = m->w32;
    FVGB_TRY(launch_convert(phi, w.tmp, N, s), "convert");
    FVGB_TRY(launch_gradient<float>(m, p->bcset_phi, w.tmp, w.grad, s), "gradient kernel");
    FVGB_TRY(launch_cell_physics<float>(m, w.grad, (const float*)ne, p->mu, p->A, p->B, (float*)E,
                                        w.vel, w.src, spot_args(m, p), s), "cell kernel");
    tc.vel_dev = w.vel;
    tc.src_dev = w.src;
    return step_T<float>(m, &tc, (float*)ne, p->dt, 1, euler, 1, (float*)ni, s);
  }
  Work<double>& w = m->w64;
  FVGB_TRY(launch_gradient<double>(m, p->bcset_phi, phi, w.grad, s), "gradient kernel");
  FVGB_TRY(launch_cell_physics<double>(m, w.grad, (const double*)ne, p->mu, p->A, p->B,
                                       (double*)E, w.vel, w.src, spot_args(m, p), s), "cell kernel");
  tc.vel_dev = w.vel;
  tc.src_dev = w.src;
  return step_T<double>(m, &tc, (double*)ne, p->dt, 1, euler, 1, (double*)ni, s);
}

namespace {

bool opts_ok(const fvgb_solve_opts* o) {
  return o && o->rtol > 0.0 && o->inner_rtol > 0.0 && o->inner_rtol < 1.0 && o->maxit_inner > 0 &&
         o->maxit_outer >= 0 && (o->prec == FVGB_FP64 || o->prec == FVGB_FP32 || o->prec == FVGB_MIXED) &&
         o->inner >= 0 && o->inner <= 8;
}

}  // namespace
}  // namespace fvgb

using namespace fvgb;

extern "C" {

const char* fvgb_last_error(void) { return g_last_error.c_str(); }

static fvgb_status upload_impl(int32_t dim, int64_t n_vert, const double* xyz, int64_t n_cell,
                               const int32_t* cell_vert, int64_t n_bface, const int32_t* bface_vert,
                               const int32_t* bface_tag, const std::vector<std::vector<BCInput>>& sets,
                               int32_t reorder, int32_t prec, void* stream, fvgb_mesh* out,
                               const int32_t* cell_part, int n_part);

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
  return upload_impl(dim, n_vert, xyz, n_cell, cell_vert, n_bface, bface_vert, bface_tag, sets,
                     reorder, prec, stream, out, nullptr, 1);
}

fvgb_status fvgb_mesh_upload_ensemble(int32_t dim, int32_t n_part, const fvgb_mesh_part* parts,
                                      int32_t n_bcset, int32_t reorder, int32_t prec,
                                      void* stream, fvgb_mesh* out) {
  set_error("");
  if (!out) { set_error("out is null"); return FVGB_EINVAL; }
  *out = nullptr;
  if (n_part < 1 || n_part > kMaxParts || !parts) { set_error("n_part must be in [1, 128]"); return FVGB_EINVAL; }
  if (n_bcset < 1) { set_error("at least one boundary-condition set is required"); return FVGB_EINVAL; }
  if (dim != 2 && dim != 3) { set_error("dim must be 2 or 3"); return FVGB_EINVAL; }
  constexpr int32_t kTagStride = 65536;
  int64_t nv = 0, nc = 0, nb = 0;
  for (int p = 0; p < n_part; ++p) {
    const fvgb_mesh_part& q = parts[p];
    if (q.n_vert <= 0 || q.n_cell <= 0 || q.n_bface <= 0 || !q.xyz || !q.cell_vert || !q.bface_vert ||
        !q.bface_tag || !q.bcsets) {
      set_error("part " + std::to_string(p) + ": empty mesh or null array");
      return FVGB_EINVAL;
    }
    nv += q.n_vert; nc += q.n_cell; nb += q.n_bface;
  }
  if (nv > (int64_t)INT32_MAX || nc > (int64_t)INT32_MAX / 4) { set_error("ensemble too large for int32 indices"); return FVGB_EINVAL; }
  std::vector<double> xyz((size_t)nv * dim);
  std::vector<int32_t> cv((size_t)nc * (dim + 1)), bfv((size_t)nb * dim), bft(nb), cpart(nc);
  std::vector<std::vector<BCInput>> sets(n_bcset);
  int64_t ov = 0, oc = 0, ob = 0;
  for (int p = 0; p < n_part; ++p) {
    const fvgb_mesh_part& q = parts[p];
    std::copy(q.xyz, q.xyz + q.n_vert * dim, xyz.begin() + ov * dim);
    for (int64_t i = 0; i < q.n_cell * (dim + 1); ++i) {
      const int32_t v = q.cell_vert[i];
      if (v < 0 || v >= q.n_vert) { set_error("part " + std::to_string(p) + ": cell vertex index out of range"); return FVGB_EMESH; }
      cv[oc * (dim + 1) + i] = (int32_t)(v + ov);
    }
    for (int64_t i = 0; i < q.n_cell; ++i) cpart[oc + i] = p;
    for (int64_t i = 0; i < q.n_bface * dim; ++i) {
      const int32_t v = q.bface_vert[i];
      if (v < 0 || v >= q.n_vert) { set_error("part " + std::to_string(p) + ": boundary vertex index out of range"); return FVGB_EMESH; }
      bfv[ob * dim + i] = (int32_t)(v + ov);
    }
    for (int64_t i = 0; i < q.n_bface; ++i) {
      const int32_t t = q.bface_tag[i];
      if (t <= 0 || t >= kTagStride) { set_error("part " + std::to_string(p) + ": boundary tags must be in [1, 65535]"); return FVGB_EMESH; }
      bft[ob + i] = p * kTagStride + t;
    }
    for (int k = 0; k < n_bcset; ++k) {
      const fvgb_bcset& bs = q.bcsets[k];
      if (bs.n_bc < 0 || (bs.n_bc > 0 && !bs.bc)) { set_error("bad bcset"); return FVGB_EINVAL; }
      for (int j = 0; j < bs.n_bc; ++j) {
        if (bs.bc[j].tag <= 0 || bs.bc[j].tag >= kTagStride) { set_error("bc tags must be in [1, 65535]"); return FVGB_EINVAL; }
        sets[k].push_back(BCInput{p * kTagStride + bs.bc[j].tag, bs.bc[j].kind, bs.bc[j].value});
      }
    }
    ov += q.n_vert; oc += q.n_cell; ob += q.n_bface;
  }
  return upload_impl(dim, nv, xyz.data(), nc, cv.data(), nb, bfv.data(), bft.data(), sets, reorder,
                     prec, stream, out, cpart.data(), n_part);
}

static fvgb_status upload_impl(int32_t dim, int64_t n_vert, const double* xyz, int64_t n_cell,
                               const int32_t* cell_vert, int64_t n_bface, const int32_t* bface_vert,
                               const int32_t* bface_tag, const std::vector<std::vector<BCInput>>& sets,
                               int32_t reorder, int32_t prec, void* stream, fvgb_mesh* out,
                               const int32_t* cell_part, int n_part) {
  if (prec != FVGB_FP64 && prec != FVGB_FP32 && prec != FVGB_MIXED) { set_error("bad precision"); return FVGB_EINVAL; }
  HostMesh h;
  std::string err;
  int rc = build_host_mesh(dim, n_vert, xyz, n_cell, cell_vert, n_bface, bface_vert, bface_tag,
                           sets, reorder, h, err, cell_part, n_part);
  if (rc) { set_error(err); return (fvgb_status)rc; }

  cudaStream_t s = (cudaStream_t)stream;
  fvgb_mesh_s* m = new fvgb_mesh_s();
  m->prec = (fvgb_prec)prec;
  // default launch shapes (measured on 6M-cell tetrahedral meshes): FP32 face fluxes two
  // faces per thread in 128-thread blocks; everything else one element per thread
  if (m->prec != FVGB_FP64) m->tune[kTuneFace] = LaunchShape{128, 2};
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
  if ((e = dupload(m, &t.cverts, h.cells, s))) return fail(e, "upload");
  {
    std::vector<int32_t> vc(h.V);
    for (int64_t v = 0; v < h.V; ++v) vc[v] = h.vptr[v + 1] - h.vptr[v];
    if ((e = dupload(m, &t.vcount, vc, s))) return fail(e, "upload");
  }
  std::vector<int64_t> sptr;
  std::vector<int32_t> sidx;
  build_sell(h.nptr, h.nidx, nullptr, h.N, true, sptr, sidx, nullptr);
  if ((e = dupload(m, &t.nsell.ptr, sptr, s))) return fail(e, "upload");
  if ((e = dupload(m, &t.nsell.idx, sidx, s))) return fail(e, "upload");
  if (prec != FVGB_FP64 && h.dim == 3 && h.N >= kGradTile &&
      (int64_t)h.nptr[h.N] < (int64_t)INT32_MAX / 2) {   // the FP32 shared-memory gradient
    std::vector<int32_t> tptr, tidx;
    std::vector<int16_t> lidx;
    const int mx = build_grad_tiles(h.N, sptr, sidx, tptr, tidx, lidx);
    if (mx <= kGradTileMaxHalo) {
      t.tile_max = mx;
      if ((e = dupload(m, &t.tile_ptr, tptr, s))) return fail(e, "upload");
      if ((e = dupload(m, &t.tile_idx, tidx, s))) return fail(e, "upload");
      if ((e = dupload(m, &t.tile_lidx, lidx, s))) return fail(e, "upload");
    }
  }
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
  // zeroed here: solves whose inner solve is not the CG (which resets it per launch) still
  // read its status word
  if ((e = cudaMemsetAsync(m->barrier, 0, sizeof(Barrier), s))) return fail(e, "memset");
  if ((e = dalloc(m, &m->d_cg_info, 4))) return fail(e, "allocation");
  if ((e = cudaMemsetAsync(m->d_cg_info, 0, 4 * sizeof(int), s))) return fail(e, "memset");
  if ((e = dalloc(m, &m->d_status, 1))) return fail(e, "allocation");
  if ((e = cudaMemsetAsync(m->d_status, 0, sizeof(int), s))) return fail(e, "memset");
  if ((e = dalloc(m, &m->d_time, 1))) return fail(e, "allocation");
  if ((e = cudaMemsetAsync(m->d_time, 0, sizeof(double), s))) return fail(e, "memset");
  if ((e = cudaMallocHost((void**)&m->h_scal, (16 + 4 * kMaxParts) * sizeof(double)))) return fail(e, "pinned allocation");
  m->solve_grid = solve_grid_size(m);
  if (m->solve_grid <= 0) {
    set_error("this device cannot run the library's kernels (built for sm_103a)");
    release(m);
    return FVGB_EUNSUPPORTED;
  }
  if ((e = setup_parts(m, h.part_cell_begin, s))) return fail(e, "parts setup");
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

fvgb_status fvgb_integral(fvgb_mesh m, const void* u, double* out, void* stream) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (!u || !out) { set_error("null argument"); return FVGB_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  FVGB_TRY(launch_integral(m, u, is_fp32(m), m->d_scal + 1, s), "integral kernel");
  FVGB_TRY(cudaMemcpyAsync(m->h_scal + 1, m->d_scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
  FVGB_TRY(cudaStreamSynchronize(s), "synchronize");
  *out = m->h_scal[1];
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

fvgb_status fvgb_mesh_parts(fvgb_mesh m, int32_t* n_part, int64_t* cell_begin) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (n_part) *n_part = m->parts.n_part;
  if (cell_begin) std::copy(m->part_cell_begin.begin(), m->part_cell_begin.end(), cell_begin);
  return FVGB_OK;
}

int32_t fvgb_amg_levels(fvgb_mesh m, int32_t bcset, int32_t prec, int64_t* sizes, int32_t cap) {
  if (check_mesh(m) || !sizes || cap < 0) return 0;
  return amg_levels(m, bcset, prec != FVGB_FP64, sizes, cap);
}

fvgb_status fvgb_solve_parts(fvgb_mesh m, double* rel_res, int32_t* outer_its, int32_t* inner_its) {
  if (fvgb_status st = check_mesh(m)) return st;
  const size_t P = (size_t)m->parts.n_part;
  if (m->last_rel.size() != P) { set_error("no solve has run on this mesh"); return FVGB_EINVAL; }
  if (rel_res) std::copy(m->last_rel.begin(), m->last_rel.end(), rel_res);
  if (outer_its) std::copy(m->last_outer.begin(), m->last_outer.end(), outer_its);
  if (inner_its) std::copy(m->last_inner.begin(), m->last_inner.end(), inner_its);
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

fvgb_status fvgb_gradient_vertex(fvgb_mesh m, int32_t bcset, const void* u, void* grad, void* stream) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (fvgb_status st = check_bcset(m, bcset)) return st;
  if (!u || !grad) { set_error("null array"); return FVGB_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  if (is_fp32(m))
    return cuda_status(launch_gradient_vertex<float>(m, bcset, (const float*)u, (float*)grad, s), "gradient kernels");
  return cuda_status(launch_gradient_vertex<double>(m, bcset, (const double*)u, (double*)grad, s), "gradient kernels");
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
  if (tc->recon != 0 && tc->recon != 1) { set_error("recon must be 0 (upwind) or 1 (MUSCL + Barth-Jespersen)"); return FVGB_EINVAL; }
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
  m->solve_primed = -1;   // a caller's own right-hand side: nothing left by a streamer step applies
  return solve_impl(m, bcset, f, phi, o, info, (cudaStream_t)stream);
}

fvgb_status fvgb_streamer_step(fvgb_mesh m, const fvgb_streamer_params* p, void* ne, void* ni,
                               double* phi, void* E, int32_t nsteps, fvgb_solve_info* info,
                               void* stream) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (!p || !ne || !ni || !phi || nsteps < 0 || !opts_ok(&p->solve) || (p->recon != 0 && p->recon != 1) ||
      (p->stages != 0 && p->stages != 1 && p->stages != 3)) { set_error("bad streamer arguments"); return FVGB_EINVAL; }
  if (fvgb_status st = check_bcset(m, p->bcset_ne)) return st;
  if (fvgb_status st = check_bcset(m, p->bcset_phi)) return st;
  if (p->n_spot < 0 || p->n_spot > kMaxSpots || (p->n_spot > 0 && !p->spots) || !std::isfinite(p->t0) ||
      !(p->dt > 0.0)) {
    set_error("bad streamer arguments: n_spot must be in [0, 4] with a spot array, t0 finite, dt > 0");
    return FVGB_EINVAL;
  }
  for (int k = 0; k < p->n_spot; ++k) {
    const fvgb_spot& q = p->spots[k];
    if (!(q.amplitude > 0.0) || !std::isfinite(q.amplitude) || !(q.sigma > 0.0) || !(q.duration >= 0.0) ||
        !std::isfinite(q.t_on) || !std::isfinite(q.duration) || !std::isfinite(q.centre[0]) ||
        !std::isfinite(q.centre[1]) || !std::isfinite(q.centre[2])) {
      set_error("bad plasma spot " + std::to_string(k));
      return FVGB_EINVAL;
    }
  }
  const bool fp32_solve = p->solve.prec == FVGB_FP32 || p->solve.prec == FVGB_MIXED;
  if (fp32_solve && !is_fp32(m)) { set_error("FP32 inner solve needs a mesh uploaded with FVGB_FP32 or FVGB_MIXED"); return FVGB_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  // the step time lives on the device (read by the spot source, advanced after each step)
  if (p->n_spot > 0) FVGB_TRY(launch_time(m, true, p->t0, s), "time kernel");
  int n0 = 0;
  const bool warm = warm_requested(p);
  const int stages = p->stages == 3 ? 3 : 1;
  m->solve_primed = -1;     // only a learned start of this call primes a solve
  if (m->use_graph && stages == 1) {
    // a captured step assumes a full warm-start history: build it with host-driven steps
    const int need = warm ? std::max(0, 2 - m->warm_hist) : 0;
    if (need == 0) return streamer_graph_steps(m, p, ne, ni, phi, E, nsteps, info, s);
    n0 = std::max(0, nsteps - need);
    nsteps = std::min(nsteps, need);
  }
  const bool fp32 = is_fp32(m);
  double* f = m->w64.tmp;   // FP64 scratch of the mesh (unused by the FP64 transport path)
  for (int n = 0; n < nsteps; ++n) {
    m->solve_primed = -1;
    if (warm) {
      fvgb_status st = warm_start(m, p, ne, ni, phi, m->warm_hist, s);
      if (st) return st;
      m->warm_hist = std::min(3, m->warm_hist + 1);
    }
    if (stages == 1) {
      fvgb_status st = cuda_status(launch_poisson_source(m, ne, ni, fp32, f, s), "source kernel");
      if (st) return st;
      st = solve_impl(m, p->bcset_phi, f, phi, &p->solve, info ? info + n : nullptr, s);
      if (st) return st;
      st = streamer_transport(m, p, ne, ni, phi, E, s);
      if (st) return st;
      if (p->n_spot > 0) FVGB_TRY(launch_time(m, false, p->dt, s), "time kernel");
      continue;
    }
    // three stages of eq. 6, each with its own Poisson solve (from the previous stage's phi)
    const size_t bytes = (size_t)m->topo.N * (fp32 ? sizeof(float) : sizeof(double));
    if (!m->rk_ne0) {
      FVGB_TRY(dalloc(m, (unsigned char**)&m->rk_ne0, bytes), "allocation");
      FVGB_TRY(dalloc(m, (unsigned char**)&m->rk_ni0, bytes), "allocation");
    }
    FVGB_TRY(cudaMemcpyAsync(m->rk_ne0, ne, bytes, cudaMemcpyDeviceToDevice, s), "copy");
    FVGB_TRY(cudaMemcpyAsync(m->rk_ni0, ni, bytes, cudaMemcpyDeviceToDevice, s), "copy");
    static const double kAlpha[3] = {0.5, 0.5, 1.0};
    fvgb_solve_info acc{0, 0, 0.0, 0.0};
    for (int k = 0; k < 3; ++k) {
      fvgb_solve_info si{0, 0, 0.0, 0.0};
      fvgb_status st = cuda_status(launch_poisson_source(m, ne, ni, fp32, f, s), "source kernel");
      if (!st) st = solve_impl(m, p->bcset_phi, f, phi, &p->solve, &si, s);
      acc.outer_its += si.outer_its;
      acc.inner_its_total += si.inner_its_total;
      acc.rel_res = std::max(acc.rel_res, si.rel_res);
      acc.bnorm = si.bnorm;
      if (info) info[n] = acc;
      if (st) return st;
      st = streamer_transport_stage(m, p, m->rk_ne0, m->rk_ni0, ne, ni, phi, E, kAlpha[k], s);
      if (st) return st;
    }
    if (p->n_spot > 0) FVGB_TRY(launch_time(m, false, p->dt, s), "time kernel");
  }
  if (n0 > 0) return streamer_graph_steps(m, p, ne, ni, phi, E, n0, info ? info + nsteps : nullptr, s);
  return FVGB_OK;
}

fvgb_status fvgb_streamer_pair(fvgb_mesh m, int32_t which, const double* phi, double* dq_out,
                               double* phi_prev_out, double* dphi_out, void* stream) {
  if (fvgb_status st = check_mesh(m)) return st;
  if ((which != 0 && which != 1) || !phi || !dq_out || !phi_prev_out || !dphi_out) {
    set_error("bad pair arguments");
    return FVGB_EINVAL;
  }
  if (!m->phi_old || m->warm_hist < 2 + which) {
    set_error(which ? "the pair of the extrapolated start needs three streamer steps with a warm start"
                    : "the pair needs two streamer steps with a warm start");
    return FVGB_EINVAL;
  }
  return cuda_status(launch_history_pair(m, which, phi, dq_out, phi_prev_out, dphi_out, (cudaStream_t)stream),
                     "pair kernel");
}

fvgb_status fvgb_sync(fvgb_mesh m, void* stream) {
  if (fvgb_status st = check_mesh(m)) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int* h = (int*)(m->h_scal + 2);
  FVGB_TRY(cudaMemcpyAsync(h, m->d_status, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
  FVGB_TRY(cudaStreamSynchronize(s), "synchronize");
  if (*h != 0) {
    const int v = *h;
    FVGB_TRY(cudaMemsetAsync(m->d_status, 0, sizeof(int), s), "memset");
    FVGB_TRY(cudaStreamSynchronize(s), "synchronize");
    if (v & 2) {
      set_error("a tensor-core wait of the network kernels timed out (latched status, now cleared)");
      return FVGB_ETIMEOUT;
    }
    set_error("a transport call produced a non-finite value (latched status, now cleared)");
    return FVGB_ENONFINITE;
  }
  return FVGB_OK;
}

fvgb_status fvgb_test_barrier(fvgb_mesh m, int32_t skip_block, double timeout_ms) {
  if (fvgb_status st = check_mesh(m)) return st;
  if (skip_block < -1 || skip_block >= m->solve_grid || !(timeout_ms >= 0.0) || timeout_ms > 1000.0) {
    set_error("skip_block must be in [-1, grid) and timeout_ms in [0, 1000]");
    return FVGB_EINVAL;
  }
  m->test_skip_block = skip_block;
  m->test_barrier_ns = (unsigned long long)(timeout_ms * 1e6);
  graph_invalidate(m);
  return FVGB_OK;
}

fvgb_status fvgb_streamer_reset(fvgb_mesh m) {
  if (fvgb_status st = check_mesh(m)) return st;
  m->warm_hist = 0;
  graph_invalidate(m);
  return FVGB_OK;
}

fvgb_status fvgb_set_graph_mode(fvgb_mesh m, int32_t on) {
  if (fvgb_status st = check_mesh(m)) return st;
  m->use_graph = on ? 1 : 0;
  return FVGB_OK;
}

}  // extern "C"
