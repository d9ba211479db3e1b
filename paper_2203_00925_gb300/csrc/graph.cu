// Streamer steps as CUDA graphs: one captured graph per mesh holds a whole step of
// eq. 10 - Poisson source, right-hand side, the FP64 outer refinement loop of the
// Poisson solve as a conditional WHILE node (body: cooperative inner CG, phi update,
// FP64 residual, per-part norms, decision), then the least-squares field, cell physics
// and the transport update. The outer-loop decision is taken on the device
// (k_decide sets the loop condition), so a batch of steps runs without any host
// synchronisation; per-step solve results are copied to pinned host memory in stream
// order and checked once at the end of the batch.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace fvgb {

struct StepInfoDev {
  int outer;      // outer steps (max over parts)
  int inner;      // inner CG iterations (max over parts)
  int status;     // 0 ok, 5 not converged, 6 non-finite / breakdown, 7 barrier timeout
  int pad;
  double rel;     // final relative residual (max over parts)
  double bn2;     // sum over parts of ||b_p||^2
};

struct GraphState {
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr, cs2 = nullptr;
  // what the graph was captured for
  void* ne = nullptr;
  void* ni = nullptr;
  double* phi = nullptr;
  void* E = nullptr;
  fvgb_streamer_params params{};
  std::vector<fvgb_spot> spots;   // copy of the captured step's plasma spots
  // device state
  double* bn2 = nullptr;        // [P]
  double* rel = nullptr;        // [P]
  int* outer = nullptr;         // [P]
  int* inner = nullptr;         // [P]
  int* ctl = nullptr;           // [0] outer steps taken, [1] status
  StepInfoDev* info = nullptr;
  StepInfoDev* h_info = nullptr;  // pinned ring, cap entries
  int cap = 0;
  long long k_pre = 0, k_body = 0, k_post = 0;  // kernels per part of the graph
};

namespace {

// Per-part decision of the outer loop (one block): accumulate the inner iterations of
// the CG launch that just ran (when accumulate), relative residuals, active flags, the
// loop condition and, when the loop ends, the step's summary.
__global__ void k_decide(int P, const double* __restrict__ norms, const double* __restrict__ bn2,
                         double rtol, int maxit_outer, int accumulate, const int* __restrict__ cg_inner,
                         const int* __restrict__ cg_status, const Barrier* __restrict__ bar,
                         int* __restrict__ ctl, int* __restrict__ active, int* __restrict__ outer,
                         int* __restrict__ inner, double* __restrict__ rel,
                         StepInfoDev* __restrict__ info, cudaGraphConditionalHandle handle) {
  __shared__ int s_any, s_bad, s_go;
  if (threadIdx.x == 0) { s_any = 0; s_bad = 0; }
  __syncthreads();
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    if (accumulate) inner[p] += cg_inner[p];
    const double r = bn2[p] > 0.0 ? sqrt(norms[p] / bn2[p]) : (bn2[p] == 0.0 ? 0.0 : bn2[p]);
    rel[p] = r;
    if (!isfinite(r)) atomicOr(&s_bad, 1);
    else if (r > rtol) atomicOr(&s_any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int go = 0;
    if (accumulate && bar->status != 0) ctl[1] = 7;
    else if (accumulate && cg_status[0] != 0) ctl[1] = 6;
    else if (s_bad) ctl[1] = 6;
    else if (s_any && ctl[0] < maxit_outer) { go = 1; ctl[0] += 1; }
    else if (s_any) ctl[1] = 5;
    s_go = go;
    cudaGraphSetConditional(handle, go ? 1u : 0u);
  }
  __syncthreads();
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    const int act = s_go && rel[p] > rtol;
    active[p] = act;
    outer[p] += act;
  }
  if (!s_go && threadIdx.x == 0) {
    int mo = 0, mi = 0;
    double mr = 0.0, b2 = 0.0;
    for (int p = 0; p < P; ++p) {
      mo = max(mo, outer[p]);
      mi = max(mi, inner[p]);
      mr = fmax(mr, rel[p]);
      b2 += bn2[p];
    }
    info->outer = mo;
    info->inner = mi;
    info->status = ctl[1];
    info->rel = mr;
    info->bn2 = b2;
  }
}

__global__ void k_graph_init(int P, int* __restrict__ ctl, int* __restrict__ outer,
                             int* __restrict__ inner) {
  if (threadIdx.x == 0) { ctl[0] = 0; ctl[1] = 0; }
  for (int p = threadIdx.x; p < P; p += blockDim.x) { outer[p] = 0; inner[p] = 0; }
}

// A part whose right-hand side is zero has the solution zero (block p handles part p).
__global__ void k_zero_parts(const double* __restrict__ bn2, const int32_t* __restrict__ part_sc,
                             const int64_t* __restrict__ sc_begin, double* __restrict__ phi, double* __restrict__ r) {
  const int p = blockIdx.y;
  if (bn2[p] != 0.0) return;
  const int64_t lo = sc_begin[part_sc[p]], hi = sc_begin[part_sc[p + 1]];
  for (int64_t i = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < hi; i += (int64_t)gridDim.x * blockDim.x) {
    phi[i] = 0.0;
    if (r) r[i] = 0.0;
  }
}

bool same_spots(const std::vector<fvgb_spot>& a, const fvgb_streamer_params& b) {
  if ((int)a.size() != b.n_spot) return false;
  for (int k = 0; k < b.n_spot; ++k) {
    const fvgb_spot& x = a[k];
    const fvgb_spot& y = b.spots[k];
    if (x.centre[0] != y.centre[0] || x.centre[1] != y.centre[1] || x.centre[2] != y.centre[2] ||
        x.amplitude != y.amplitude || x.sigma != y.sigma || x.t_on != y.t_on || x.duration != y.duration)
      return false;
  }
  return true;
}

// field by field (padding bytes of a caller's struct may hold anything); the start time t0
// is not part of the graph (the step time lives on the device)
bool same_params(const fvgb_streamer_params& a, const fvgb_streamer_params& b) {
  return a.mu == b.mu && a.A == b.A && a.B == b.B && a.De == b.De && a.dt == b.dt &&
         a.bcset_ne == b.bcset_ne && a.bcset_phi == b.bcset_phi && a.solve.rtol == b.solve.rtol &&
         a.solve.inner_rtol == b.solve.inner_rtol && a.solve.maxit_inner == b.solve.maxit_inner &&
         a.solve.maxit_outer == b.solve.maxit_outer && a.solve.prec == b.solve.prec &&
         a.warm == b.warm && a.extrapolate == b.extrapolate && a.recon == b.recon &&
         a.stages == b.stages;
}

cudaError_t capture_error(cudaError_t e) { return e; }

// Capture the whole step into a graph (see file comment).
fvgb_status build_graph(fvgb_mesh m, GraphState& g, const fvgb_streamer_params* p, void* ne,
                        void* ni, double* phi, void* E) {
  const int P = m->parts.n_part;
  const bool fp32_solve = p->solve.prec == FVGB_FP32 || p->solve.prec == FVGB_MIXED;
  double* f = m->w64.tmp;
  double* b = m->dphi_tmp2;
  double* r = m->dphi_tmp;
  // the multigrid hierarchy is built (with host synchronisation) before the capture
  if (p->solve.inner > 0) FVGB_TRY_ST(amg_ensure(m, p->bcset_phi, fp32_solve, g.cs));
  const long long k0 = g_kernel_launches.load();
  cudaGraph_t graph = nullptr;
  FVGB_TRY(cudaGraphCreate(&graph, 0), "graph create");
  cudaGraphConditionalHandle handle;
  FVGB_TRY(cudaGraphConditionalHandleCreate(&handle, graph, 0, 0), "conditional handle");
  FVGB_TRY(cudaStreamBeginCaptureToGraph(g.cs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed),
           "begin capture");
  fvgb_status st = FVGB_OK;
  auto bail = [&](fvgb_status s2) {
    cudaGraph_t dummy = nullptr;
    cudaStreamEndCapture(g.cs, &dummy);
    cudaGraphDestroy(graph);
    cudaGetLastError();
    return s2;
  };
  // ---- before the loop
  if (warm_requested(p) && (st = warm_start(m, p, ne, ni, phi, 2, g.cs))) return bail(st);
  m->warm_check_pending = false;   // captured, not run: graph steps are not counted
  // after a learned start, b and the start's residual are already formed (as in solve_impl)
  const bool primed = m->solve_primed == p->bcset_phi;
  m->solve_primed = -1;
  if (!primed) {
    if ((st = cuda_status(launch_poisson_source(m, ne, ni, is_fp32(m), f, g.cs), "source kernel"))) return bail(st);
    if ((st = poisson_rhs_impl(m, p->bcset_phi, f, b, g.cs))) return bail(st);
  }
  if ((st = cuda_status(launch_part_sumsq(m, b, g.bn2, g.cs), "norm kernel"))) return bail(st);
  k_graph_init<<<1, 128, 0, g.cs>>>(P, g.ctl, g.outer, g.inner);
  k_zero_parts<<<part_grid(m), 256, 0, g.cs>>>(g.bn2, m->parts.part_sc, m->parts.sc_begin, phi,
                                               primed ? r : nullptr);
  count_launch(2);
  if (!primed && (st = poisson_residual(m, p->bcset_phi, phi, b, r, g.cs))) return bail(st);
  if ((st = cuda_status(launch_part_sumsq(m, r, m->parts.norms, g.cs), "norm kernel"))) return bail(st);
  k_decide<<<1, 128, 0, g.cs>>>(P, m->parts.norms, g.bn2, p->solve.rtol, p->solve.maxit_outer, 0,
                                m->parts.out_inner, m->d_cg_info, m->barrier, g.ctl, m->parts.active,
                                g.outer, g.inner, g.rel, g.info, handle);
  count_launch();
  const long long k1 = g_kernel_launches.load();
  // ---- the conditional WHILE node
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  if ((st = cuda_status(cudaStreamGetCaptureInfo(g.cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps),
                        "capture info"))) return bail(st);
  alignas(cudaGraphNodeParams) unsigned char cp_mem[sizeof(cudaGraphNodeParams)];
  std::memset(cp_mem, 0, sizeof(cp_mem));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_mem);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  if ((st = cuda_status(cudaGraphAddNode(&cnode, graph, deps, nullptr, ndeps, &cp), "conditional node")))
    return bail(st);
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if ((st = cuda_status(cudaStreamUpdateCaptureDependencies(g.cs, &cnode, nullptr, 1,
                                                            cudaStreamSetCaptureDependencies),
                        "capture dependencies"))) return bail(st);
  // ---- after the loop: field, cell physics, transport
  if ((st = streamer_transport(m, p, ne, ni, phi, E, g.cs))) return bail(st);
  if (p->n_spot > 0 && (st = cuda_status(launch_time(m, false, p->dt, g.cs), "time kernel"))) return bail(st);
  const long long k2 = g_kernel_launches.load();
  cudaGraph_t out = nullptr;
  if ((st = cuda_status(cudaStreamEndCapture(g.cs, &out), "end capture"))) { cudaGraphDestroy(graph); return st; }
  // ---- the loop body
  if ((st = cuda_status(cudaStreamBeginCaptureToGraph(g.cs2, body, nullptr, nullptr, 0,
                                                      cudaStreamCaptureModeRelaxed), "begin body capture"))) {
    cudaGraphDestroy(graph);
    return st;
  }
  auto bail2 = [&](fvgb_status s2) {
    cudaGraph_t dummy = nullptr;
    cudaStreamEndCapture(g.cs2, &dummy);
    cudaGraphDestroy(graph);
    cudaGetLastError();
    return s2;
  };
  const int64_t N = m->topo.N;
  if (fp32_solve) {
    if ((st = cuda_status(launch_inner<float>(m, p->bcset_phi, r, &p->solve, g.cs2), "inner solve"))) return bail2(st);
    if ((st = cuda_status(launch_add_to_double(m->w32.cg_x, true, phi, N, g.cs2), "update"))) return bail2(st);
  } else {
    if ((st = cuda_status(launch_inner<double>(m, p->bcset_phi, r, &p->solve, g.cs2), "inner solve"))) return bail2(st);
    if ((st = cuda_status(launch_add_to_double(m->w64.cg_x, false, phi, N, g.cs2), "update"))) return bail2(st);
  }
  if ((st = poisson_residual(m, p->bcset_phi, phi, b, r, g.cs2))) return bail2(st);
  if ((st = cuda_status(launch_part_sumsq(m, r, m->parts.norms, g.cs2), "norm kernel"))) return bail2(st);
  k_decide<<<1, 128, 0, g.cs2>>>(P, m->parts.norms, g.bn2, p->solve.rtol, p->solve.maxit_outer, 1,
                                 m->parts.out_inner, m->d_cg_info, m->barrier, g.ctl, m->parts.active,
                                 g.outer, g.inner, g.rel, g.info, handle);
  count_launch();
  const long long k3 = g_kernel_launches.load();
  cudaGraph_t body_out = nullptr;
  if ((st = cuda_status(cudaStreamEndCapture(g.cs2, &body_out), "end body capture"))) { cudaGraphDestroy(graph); return st; }
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if ((st = cuda_status(e, "graph instantiate"))) return st;
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = exec;
  g.ne = ne; g.ni = ni; g.phi = phi; g.E = E; g.params = *p;
  g.spots.assign(p->spots, p->spots + p->n_spot);
  g.params.spots = nullptr;
  g.k_pre = k1 - k0;
  g.k_post = k2 - k1;
  g.k_body = k3 - k2;
  // captured launches do not run: count them when the graph executes
  g_kernel_launches.fetch_sub(k3 - k0);
  return FVGB_OK;
}

}  // namespace

void graph_invalidate(fvgb_mesh m) {
  if (m->graph && m->graph->exec) {
    cudaGraphExecDestroy(m->graph->exec);
    m->graph->exec = nullptr;
  }
}

void graph_release(fvgb_mesh m) {
  GraphState* g = m->graph;
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->cs) cudaStreamDestroy(g->cs);
  if (g->cs2) cudaStreamDestroy(g->cs2);
  if (g->h_info) cudaFreeHost(g->h_info);
  delete g;
  m->graph = nullptr;
}

fvgb_status streamer_graph_steps(fvgb_mesh m, const fvgb_streamer_params* p, void* ne, void* ni,
                                 double* phi, void* E, int nsteps, fvgb_solve_info* info,
                                 cudaStream_t s) {
  if (nsteps == 0) return FVGB_OK;
  const int P = m->parts.n_part;
  if (!m->graph) {
    GraphState* g = new GraphState();
    m->graph = g;
    FVGB_TRY(cudaStreamCreateWithFlags(&g->cs, cudaStreamNonBlocking), "stream create");
    FVGB_TRY(cudaStreamCreateWithFlags(&g->cs2, cudaStreamNonBlocking), "stream create");
    void* q = nullptr;
    FVGB_TRY(cudaMalloc(&q, 2 * P * sizeof(double) + 2 * P * sizeof(int) + 4 * sizeof(int) + sizeof(StepInfoDev) + 256), "allocation");
    m->allocs.push_back(q);
    char* c = (char*)q;
    g->info = (StepInfoDev*)c; c += (sizeof(StepInfoDev) + 15) / 16 * 16;
    g->bn2 = (double*)c; c += P * sizeof(double);
    g->rel = (double*)c; c += P * sizeof(double);
    g->outer = (int*)c; c += P * sizeof(int);
    g->inner = (int*)c; c += P * sizeof(int);
    g->ctl = (int*)c;
  }
  GraphState& g = *m->graph;
  if (!g.exec || g.ne != ne || g.ni != ni || g.phi != phi || g.E != E || !same_params(g.params, *p) || !same_spots(g.spots, *p)) {
    FVGB_TRY(cudaStreamSynchronize(s), "synchronize");
    if (fvgb_status st = build_graph(m, g, p, ne, ni, phi, E)) return st;
  }
  if (g.cap < nsteps) {
    if (g.h_info) cudaFreeHost(g.h_info);
    g.h_info = nullptr;
    g.cap = 0;
    FVGB_TRY(cudaMallocHost((void**)&g.h_info, nsteps * sizeof(StepInfoDev)), "pinned allocation");
    g.cap = nsteps;
  }
  for (int n = 0; n < nsteps; ++n) {
    FVGB_TRY(cudaGraphLaunch(g.exec, s), "graph launch");
    FVGB_TRY(cudaMemcpyAsync(g.h_info + n, g.info, sizeof(StepInfoDev), cudaMemcpyDeviceToHost, s), "copy");
  }
  // a captured step updates the warm-start history like a host-driven one
  if (warm_requested(p)) m->warm_hist = std::min(3, m->warm_hist + nsteps);
  // per-part results of the last solve, for fvgb_solve_parts
  m->last_rel.assign(P, 0.0);
  m->last_outer.assign(P, 0);
  m->last_inner.assign(P, 0);
  FVGB_TRY(cudaMemcpyAsync(m->last_rel.data(), g.rel, P * sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
  FVGB_TRY(cudaMemcpyAsync(m->last_outer.data(), g.outer, P * sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
  FVGB_TRY(cudaMemcpyAsync(m->last_inner.data(), g.inner, P * sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
  int* hlatch = (int*)(m->h_scal + 3);
  FVGB_TRY(cudaMemcpyAsync(hlatch, m->d_status, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
  FVGB_TRY(cudaStreamSynchronize(s), "synchronize");
  fvgb_status first = FVGB_OK;
  for (int n = 0; n < nsteps; ++n) {
    const StepInfoDev& d = g.h_info[n];
    if (info) info[n] = fvgb_solve_info{d.outer, d.inner, d.rel, std::sqrt(d.bn2)};
    count_launch((int)(g.k_pre + g.k_post + g.k_body * d.outer));
    m->stats.solves++;
    m->stats.outer_its += d.outer;
    m->stats.cg_launches += d.outer;
    m->stats.cg_iterations += d.inner;
    if (first == FVGB_OK && d.status != 0) {
      first = d.status == 5 ? FVGB_ENOCONV : d.status == 7 ? FVGB_ETIMEOUT : FVGB_ENONFINITE;
      set_error("streamer step " + std::to_string(n) + ": Poisson solve failed (status " + std::to_string(d.status) + ")");
    }
  }
  if (first == FVGB_OK && *hlatch != 0) {
    FVGB_TRY(cudaMemsetAsync(m->d_status, 0, sizeof(int), s), "memset");
    set_error("a transport update of a graph step produced a non-finite value (latched status)");
    first = FVGB_ENONFINITE;
  }
  return first;
}

}  // namespace fvgb
