// Internal declarations shared by the CUDA translation units of libfvgb.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fvgb.h"

namespace fvgb {

// Sliced-ELL (SELL-32) list: rows grouped in slices of 32 consecutive rows; slice s
// stores its entries column-major from ptr[s], width ptr[s+1]-ptr[s] over 32, so one
// warp reads 128 contiguous bytes per column.
struct Sell {
  int64_t* ptr = nullptr;   // [n_slice + 1] element offsets
  int32_t* idx = nullptr;   // padded entries
};

template <typename T>
struct BCDev {
  int8_t* bkind = nullptr;   // [Fb]
  T* bval = nullptr;         // [Fb]
  T* minv = nullptr;         // [nsym][N]
  int32_t* gptr = nullptr;   // [N+1]
  int32_t* gface = nullptr;  // ghost faces
  int32_t* gmult = nullptr;  // vertices each ghost face shares with the cell
  T* minv_v = nullptr;       // [nsym][N] inverse of the multiplicity-weighted normal matrix
  T* vdir = nullptr;         // [V] NaN = not Dirichlet
  int32_t* at_nbr = nullptr; // [N][4] (unused slot: the cell itself)
  T* at_coef = nullptr;      // [N][4] (unused slot: 0)
  T* at_diag = nullptr;      // [N]
  T* at_scoef = nullptr;     // [N][4] coefficients of D^-1/2 A_T D^-1/2 (the inner CG's operator)
  T* at_isd = nullptr;       // [N] D^-1/2
};

// Real-valued geometry in one precision.
template <typename T>
struct GeoDev {
  T* cen = nullptr;      // [d][N] (high part in FP32)
  T* cen_lo = nullptr;   // [d][N] low part (FP32 only): cen_true = cen + cen_lo
  T* vol = nullptr;      // [N]
  T* inv_vol = nullptr;  // [N]
  T* S = nullptr;        // [d][F]
  T* xf = nullptr;       // [d][F]
  T* xf_lo = nullptr;    // [d][F] (FP32 only)
  T* coef = nullptr;     // [d][F]
  T* valpha = nullptr;   // SELL-padded weights, aligned with vsell.idx
  T* xv = nullptr;       // [d][V] vertex coordinates (high part in FP32)
  T* xv_lo = nullptr;    // [d][V] low part (FP32 only)
  T* vs1 = nullptr;      // [d][V] sum over the cells around A of (x_c - x_A)
  std::vector<BCDev<T>> bc;
};

struct TopoDev {
  int dim = 0;
  int64_t N = 0, V = 0, F = 0, Fi = 0, n_nbr = 0;
  int32_t* fL = nullptr;
  int32_t* fR = nullptr;
  int32_t* fvert = nullptr;      // [d][F]
  int32_t* cell_face = nullptr;  // [d+1][N]
  int32_t* cell_perm = nullptr;  // [N] internal -> caller
  int32_t* cverts = nullptr;     // [N][d+1] vertices of each cell
  int32_t* vcount = nullptr;     // [V] cells around each vertex
  Sell nsell;                    // node neighbours of each cell (padded with the cell)
  Sell vsell;                    // cells around each vertex (padded, weight 0)
  // Tiles of kGradTile consecutive cells for the shared-memory gradient: per tile its
  // halo list (the tile's own cells in order, then the other node neighbours of its cells,
  // sorted) and, aligned with nsell.idx, each entry's position in its tile's list.
  int32_t* tile_ptr = nullptr;   // [n_tile + 1]
  int32_t* tile_idx = nullptr;   // halo lists
  int16_t* tile_lidx = nullptr;  // [size of nsell.idx]
  int tile_max = 0;              // longest halo list (0: tiles not built)
};

constexpr int kGradTile = 128;      // cells per tile of the shared-memory gradient
constexpr int kGradTileMaxHalo = 3072;  // longest halo list the FP32 tiled kernel stages (48 KB)

// Scratch of one precision.
template <typename T>
struct Work {
  T* flux = nullptr;   // [F]
  T* uv = nullptr;     // [V]
  T* stage = nullptr;  // [N] Runge-Kutta stage value
  T* tmp = nullptr;    // [N]
  T* vel = nullptr;    // [d][N]
  T* src = nullptr;    // [N]
  T* grad = nullptr;   // [d][N]
  T* grec = nullptr;   // [N] packed gradient records (FP64: 4 words, FP32: 8 words)
  T* vsum = nullptr;   // [5][V] per-vertex sums of the multiplicity-weighted gradient
  T* cg_r = nullptr;   // [N]
  T* cg_p = nullptr;
  T* cg_q = nullptr;
  T* cg_x = nullptr;
};

// Parts of a mesh (an ensemble of independent meshes packed into one index space) and
// the sub-chunks of the persistent solve: block b owns rows [b N / G, (b+1) N / G) cut at
// part boundaries.
struct PartsDev {
  int n_part = 1;
  int n_sc = 0;
  int32_t* blk_sc = nullptr;    // [G+1] first sub-chunk of each block
  int64_t* sc_begin = nullptr;  // [n_sc+1] first row of each sub-chunk
  int32_t* sc_part = nullptr;   // [n_sc] part of each sub-chunk
  int32_t* part_sc = nullptr;   // [P+1] first sub-chunk of each part
  double* buf = nullptr;        // [2][2][n_sc] partial sums
  int* active = nullptr;        // [P] parts the inner solve works on
  int* out_inner = nullptr;     // [P] inner iterations of the last CG launch
  double* norms = nullptr;      // [P] per-part sums of squares
};

struct Barrier {
  unsigned int count;  // arrivals since the launch (zeroed before every launch)
  int status;          // 0 ok, 1 timeout
  int pad[2];
};

struct GraphState;
struct AmgState;

// Launch shape of a tunable kernel: threads per block and elements per thread.
struct LaunchShape {
  int threads = 256;
  int ipt = 1;
};
enum TuneKernel { kTuneGrad = 0, kTuneVertex = 1, kTuneFace = 2, kTuneUpdate = 3, kTuneCount = 4 };

}  // namespace fvgb

struct fvgb_mesh_s {
  int device = 0;
  int num_sms = 0;
  fvgb_prec prec = FVGB_FP64;
  fvgb::TopoDev topo;
  fvgb::GeoDev<double> g64;
  fvgb::GeoDev<float> g32;
  fvgb::Work<double> w64;
  fvgb::Work<float> w32;
  std::vector<int32_t> cell_perm_host;
  std::vector<int32_t> vert_perm_host;
  double* d_scal = nullptr;             // reduction partials / results (FP64)
  double* h_scal = nullptr;             // pinned host mirror
  double* dphi_tmp = nullptr;           // [N] FP64 scratch (residual r)
  double* dphi_tmp2 = nullptr;          // [N] FP64 scratch (rhs b)
  double* dzero = nullptr;              // [N] zeros
  fvgb::Barrier* barrier = nullptr;
  int* d_cg_info = nullptr;             // [4] iterations, status
  int* d_status = nullptr;              // latched asynchronous errors, cleared when reported:
                                        // bit 0 (1) non-finite transport output, bit 1 (2) a
                                        // tensor-core wait of the network kernels timed out
  double* d_time = nullptr;             // start time of the current streamer step
  int test_skip_block = -1;             // test hook of the CG barrier (fvgb_test_barrier)
  unsigned long long test_barrier_ns = 0;  // barrier wait limit (0: the default 1 s)
  int solve_grid = 0;                   // cooperative grid of the Poisson kernel
  fvgb::PartsDev parts;
  std::vector<int64_t> part_cell_begin; // [P+1] internal cell range of each part
  std::vector<int32_t> last_outer, last_inner;  // per-part results of the last solve
  std::vector<double> last_rel;
  fvgb_stats stats{};                   // counters (kernel_launches is library-wide)
  int time_cg = 0;                      // record CUDA events around CG launches
  cudaEvent_t ev_cg0 = nullptr, ev_cg1 = nullptr;
  bool cg_pending = false;              // events recorded, elapsed time not yet read
  int use_graph = 0;                    // run streamer steps as one CUDA graph each
  fvgb::LaunchShape tune[fvgb::kTuneCount];  // launch shapes (autotuned or default)
  // warm-start history of the streamer (allocated when a warm start is requested)
  double* q_prev = nullptr;             // [N] n_i - n_e of the previous step
  double* dq = nullptr;                 // [N] latest change of n_i - n_e
  double* d2q = nullptr;                // [N] its change since the step before
  double* phi_old = nullptr;            // [N] potential at the start of the last step
  double* phi_old2 = nullptr;           // [N] potential at the start of the step before
  double* dphi_pred = nullptr;          // [N] learned correction
  double* phi_save = nullptr;           // [N] start without the learned correction
  double* warm_norms = nullptr;         // [4][P] per part <r0, A pred>, ||A pred||^2, ||r0||^2, ||r1||^2
  int* warm_used = nullptr;             // [P] 1 where the learned correction was used (scale > 0)
  double* warm_scale = nullptr;         // [P] scale of the learned correction in the start
  bool warm_check_pending = false;      // warm_used of a host-driven step not yet counted
  int solve_primed = -1;                // boundary set whose next solve finds its b and its start's
                                        // residual already in dphi_tmp2 / dphi_tmp (left by the
                                        // learned start); -1: none
  int warm_hist = 0;                    // streamer steps recorded in the history (capped at 3)
  fvgb::GraphState* graph = nullptr;    // captured step graph (graph.cu)
  fvgb::AmgState* amg = nullptr;        // multigrid hierarchies per boundary set (amg.cu)
  void* rk_ne0 = nullptr;               // [N] n_e, n_i at the start of a three-stage streamer step
  void* rk_ni0 = nullptr;
  std::vector<void*> allocs;
};

namespace fvgb {

template <typename T>
inline GeoDev<T>& geo_of(fvgb_mesh_s* m);
template <>
inline GeoDev<double>& geo_of<double>(fvgb_mesh_s* m) { return m->g64; }
template <>
inline GeoDev<float>& geo_of<float>(fvgb_mesh_s* m) { return m->g32; }
template <typename T>
inline Work<T>& work_of(fvgb_mesh_s* m);
template <>
inline Work<double>& work_of<double>(fvgb_mesh_s* m) { return m->w64; }
template <>
inline Work<float>& work_of<float>(fvgb_mesh_s* m) { return m->w32; }

constexpr int kRedBlocks = 1024;   // fixed grid of the deterministic reductions
constexpr int kCgThreads = 512;    // threads per block of the persistent Poisson kernel
constexpr int kCgBlocksPerSm = 1;  // resident blocks per SM of that kernel
constexpr int kMaxParts = 128;     // parts of an ensemble mesh handled by one solve

extern std::atomic<long long> g_kernel_launches;
inline void count_launch(int n = 1) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const std::string& msg);
fvgb_status cuda_status(cudaError_t e, const char* what);

// ops.cu -------------------------------------------------------------------------------
template <typename T>
cudaError_t launch_gradient(fvgb_mesh_s* m, int bcset, const T* u, T* grad, cudaStream_t s);
// multiplicity-weighted (vertex-factorised) variant of the least-squares gradient
template <typename T>
cudaError_t launch_gradient_vertex(fvgb_mesh_s* m, int bcset, const T* u, T* grad, cudaStream_t s);
template <typename T>
cudaError_t launch_vertex(fvgb_mesh_s* m, int bcset, const T* u, T* uv, bool homog, cudaStream_t s);
// face kernel: conv (use velocity), D (diffusion coefficient; -1 gives F = q); lgrad
// (optional, with conv): limited gradient for the MUSCL reconstruction of eq. 15
template <typename T>
cudaError_t launch_face(fvgb_mesh_s* m, int bcset, const T* u, const T* uv, const T* vel,
                        const double* vel_const, bool conv, double D, bool homog, T* flux,
                        cudaStream_t s, const T* lgrad = nullptr);
// Barth-Jespersen limiter: grad <- psi grad (eq. 15)
template <typename T>
cudaError_t launch_bj_limit(fvgb_mesh_s* m, int bcset, const T* u, T* grad, cudaStream_t s);
enum UpdateMode { kResidual = 0, kStep = 1, kPoissonApply = 2, kPoissonResidual = 3, kPoissonRhs = 4 };
template <typename T>
cudaError_t launch_update(fvgb_mesh_s* m, int mode, const T* flux, const T* src, const T* base,
                          double adt, const T* aux, T* out, T* out2, cudaStream_t s);
// Plasma spots of a streamer step (fvgb_spot), passed to the cell-physics kernel by value;
// the step's start time is read from the device (m->d_time).
constexpr int kMaxSpots = 4;
struct SpotArgs {
  int n = 0;
  double cx[kMaxSpots], cy[kMaxSpots], cz[kMaxSpots];
  double amp[kMaxSpots], s2[kMaxSpots], t_on[kMaxSpots], t_off[kMaxSpots];
  double dt = 0.0;
  const double* t = nullptr;
};
SpotArgs spot_args(fvgb_mesh_s* m, const fvgb_streamer_params* p);
template <typename T>
cudaError_t launch_cell_physics(fvgb_mesh_s* m, const T* grad, const T* ne, double mu, double A,
                                double B, T* E, T* vel, T* src, const SpotArgs& sp, cudaStream_t s);
// device time of the streamer steps: set, or advanced by dt
cudaError_t launch_time(fvgb_mesh_s* m, bool set, double v, cudaStream_t s);
cudaError_t launch_poisson_source(fvgb_mesh_s* m, const void* ne, const void* ni, bool fp32,
                                  double* f, cudaStream_t s);
cudaError_t launch_sumsq(fvgb_mesh_s* m, const double* x, int64_t n, double* out, cudaStream_t s);
cudaError_t launch_integral(fvgb_mesh_s* m, const void* u, bool fp32, double* out, cudaStream_t s);
cudaError_t launch_charge_hist(fvgb_mesh_s* m, const void* ne, const void* ni, bool fp32, int hist,
                               double* q_prev, double* dq, double* d2q, cudaStream_t s);
cudaError_t launch_extrapolate(fvgb_mesh_s* m, bool extrap, double* phi, double* phi_old, double* phi_old2,
                               cudaStream_t s);
cudaError_t launch_history_pair(fvgb_mesh_s* m, int which, const double* phi, double* q_out, double* p_out,
                                double* d_out, cudaStream_t s);
dim3 part_grid(const fvgb_mesh_s* m);   // blocks per part x parts of per-part elementwise kernels
cudaError_t launch_scale_start(fvgb_mesh_s* m, const double* dots, const double* saved, const double* pred,
                               double* phi, int* used, double* scale, double* r0, const double* r1,
                               cudaStream_t s);
cudaError_t launch_axpy_d(const double* x, double a, double* y, int64_t n, cudaStream_t s);
cudaError_t launch_add_to_double(const void* x, bool fp32, double* y, int64_t n, cudaStream_t s);
cudaError_t launch_convert(const double* x, float* y, int64_t n, cudaStream_t s);
cudaError_t launch_convert_back(const float* x, double* y, int64_t n, cudaStream_t s);
cudaError_t launch_permute(const void* src, void* dst, const int32_t* perm, int64_t n, int ncomp,
                           int elem_bytes, bool to_internal, cudaStream_t s);
cudaError_t launch_nonfinite_check(const double* x, int64_t n, int* flag, cudaStream_t s);

// api.cu -------------------------------------------------------------------------------
bool is_fp32(fvgb_mesh m);
#define FVGB_TRY(expr, what)                                   \
  do {                                                         \
    fvgb_status st_ = cuda_status((expr), (what));             \
    if (st_ != FVGB_OK) return st_;                            \
  } while (0)
// the same for an expression that already yields an fvgb_status
#define FVGB_TRY_ST(expr)                                      \
  do {                                                         \
    fvgb_status st_ = (expr);                                  \
    if (st_ != FVGB_OK) return st_;                            \
  } while (0)

// Device allocation owned by the mesh (freed with it), and an upload of a host vector.
template <typename T>
cudaError_t dalloc(fvgb_mesh_s* m, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, (count > 0 ? count : 1) * sizeof(T));
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

// amg.cu: multigrid inner solve (hierarchy built on first use per boundary set and
// precision; host synchronisation, so not during stream capture)
fvgb_status amg_ensure(fvgb_mesh m, int bcset, bool fp32, cudaStream_t s);
void amg_release(fvgb_mesh m);
int amg_levels(fvgb_mesh m, int bcset, bool fp32, int64_t* sizes, int cap);
template <typename T>
cudaError_t launch_amg_inner(fvgb_mesh_s* m, int bcset, const double* r, int cycles, cudaStream_t s);

fvgb_status poisson_residual(fvgb_mesh m, int bcset, const double* x, const double* b, double* r,
                             cudaStream_t s);
fvgb_status poisson_rhs_impl(fvgb_mesh m, int bcset, const double* f, double* b, cudaStream_t s);
template <typename T>
fvgb_status step_T(fvgb_mesh m, const fvgb_tcoef* tc, T* u, double dt, int nsteps,
                   const double* alpha, int nstage, T* ni_out, cudaStream_t s);
fvgb_status warm_start(fvgb_mesh m, const fvgb_streamer_params* p, void* ne, void* ni, double* phi,
                       int hist, cudaStream_t s);
bool warm_requested(const fvgb_streamer_params* p);
fvgb_status streamer_transport(fvgb_mesh m, const fvgb_streamer_params* p, void* ne, void* ni,
                               const double* phi, void* E, cudaStream_t s);

// graph.cu -----------------------------------------------------------------------------
fvgb_status streamer_graph_steps(fvgb_mesh m, const fvgb_streamer_params* p, void* ne, void* ni,
                                 double* phi, void* E, int nsteps, fvgb_solve_info* info,
                                 cudaStream_t s);
void graph_release(fvgb_mesh m);
void graph_invalidate(fvgb_mesh m);

// solver.cu ----------------------------------------------------------------------------
int solve_grid_size(fvgb_mesh_s* m);
template <typename T>
cudaError_t launch_cg(fvgb_mesh_s* m, int bcset, const double* r, double inner_rtol, int maxit,
                      cudaStream_t s);

// the inner solve of the Poisson refinement loop selected by o->inner (result in
// work_of<T>(m).cg_x, bookkeeping in parts.out_inner / d_cg_info)
template <typename T>
cudaError_t launch_inner(fvgb_mesh_s* m, int bcset, const double* r, const fvgb_solve_opts* o,
                         cudaStream_t s) {
  if (o->inner > 0) return launch_amg_inner<T>(m, bcset, r, o->inner, s);
  return launch_cg<T>(m, bcset, r, o->inner_rtol, o->maxit_inner, s);
}

cudaError_t launch_part_sumsq(fvgb_mesh_s* m, const double* v, double* out, cudaStream_t s);
// per part <r0, r0 - r1>, ||r0 - r1||^2, ||r0||^2, ||r1||^2 into out[k P, (k + 1) P), k = 0..3
cudaError_t launch_part_dots(fvgb_mesh_s* m, const double* r0, const double* r1, double* out, cudaStream_t s);

}  // namespace fvgb
