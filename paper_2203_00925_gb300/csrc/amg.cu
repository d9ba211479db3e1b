// Multigrid inner solve of the Poisson refinement loop: k V-cycles of smoothed-
// aggregation multigrid on the two-point operator A_T (hierarchy built on the host by
// amg_host.cpp the first time a solve of that boundary set asks for it), replacing the
// inner conjugate-gradient solve when fvgb_solve_opts.inner = k > 0. The outer FP64
// refinement on the full diamond operator, its per-part stopping test and every result
// check are unchanged.
//
// V-cycle on level l with right-hand side b (zero initial guess), damped Jacobi w = 2/3:
//   x = w D^-1 b;  r = b - A x;  b_{l+1} = R r;  x_{l+1} = V-cycle(l+1);  x += P x_{l+1};
//   x_out = x + w D^-1 (b - A x);   on the coarsest level x = A^-1 b (dense inverse).
// Every kernel writes each output element from one thread or one lane group summing in a
// fixed order, so the cycle is bitwise reproducible and can be captured in a graph.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "amg_host.h"
#include "internal.h"

namespace fvgb {

template <typename T>
struct CsrDev {
  int64_t n = 0, m = 0, nnz = 0;
  int64_t* ptr = nullptr;
  int32_t* idx = nullptr;
  T* val = nullptr;
  int lanes = 1;            // threads per row: 1, 4, 8 or 32 (from the mean row length)
};

template <typename T>
struct AmgLevelDev {
  CsrDev<T> A, P, R;
  T* dinv = nullptr;
  T* b = nullptr;    // right-hand side (levels >= 1)
  T* x = nullptr;    // iterate
  T* xo = nullptr;   // smoothed output
  T* r = nullptr;    // residual
};

template <typename T>
struct AmgDev {
  bool built = false;
  std::vector<AmgLevelDev<T>> lv;
  int64_t nco = 0;
  T* cinv = nullptr;
  T* cb = nullptr;
  T* cx = nullptr;
  T* t0 = nullptr;   // level-0 scratch: masked right-hand side
  T* t1 = nullptr;   // level-0 scratch: residual of the current correction
  T* t2 = nullptr;   // level-0 scratch: one cycle's correction
};

struct AmgState {
  std::vector<AmgDev<double>> d64;   // per boundary set
  std::vector<AmgDev<float>> d32;
};

namespace {

constexpr int kAmgThreads = 256;

inline unsigned blocks_for(int64_t n, int per_block) {
  return (unsigned)((n + per_block - 1) / per_block);
}

template <typename T>
__global__ void k_amg_jacobi0(int64_t n, const T* __restrict__ dinv, const T* __restrict__ b,
                              T* __restrict__ x, T w) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] = w * dinv[i] * b[i];
}

// mode 0: y = M v; 1: y += M v; 2: y = b - M v (residual); 3: y = x + w dinv (b - M x).
// LANES consecutive threads share a row: lane l sums entries l, l + LANES, ..., then a
// shuffle tree over the group (fixed order).
template <typename T, int LANES>
__global__ void __launch_bounds__(kAmgThreads)
k_amg_csr(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ idx,
          const T* __restrict__ val, const T* __restrict__ v, const T* __restrict__ b,
          const T* __restrict__ dinv, T w, int mode, T* __restrict__ y) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t i = t / LANES;
  const int lane = (int)(t % LANES);
  const bool valid = i < n;
  T s = T(0);
  if (valid)
    for (int64_t a = ptr[i] + lane; a < ptr[i + 1]; a += LANES) s += val[a] * v[idx[a]];
  if (LANES > 1) {
    // every lane of the warp takes part in the shuffles (rows past n contribute 0)
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, LANES);
  }
  if (!valid || lane != 0) return;
  if (mode == 0) y[i] = s;
  else if (mode == 1) y[i] += s;
  else if (mode == 2) y[i] = b[i] - s;
  else y[i] = v[i] + w * dinv[i] * (b[i] - s);
}

// x = inv b, one warp per row of the dense row-major inverse
template <typename T>
__global__ void __launch_bounds__(kAmgThreads)
k_amg_dense(int64_t n, const T* __restrict__ inv, const T* __restrict__ b, T* __restrict__ x) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  T s = T(0);
  for (int64_t a = lane; a < n; a += 32) s += inv[i * n + a] * b[a];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) x[i] = s;
}

// right-hand side in T, zero on the parts that are not active (one block per sub-chunk)
template <typename T>
__global__ void k_amg_rhs(const double* __restrict__ r, const int64_t* __restrict__ sc_begin,
                          const int32_t* __restrict__ sc_part, const int* __restrict__ active,
                          T* __restrict__ b) {
  const int sc = blockIdx.x;
  const bool act = active[sc_part[sc]] != 0;
  for (int64_t i = sc_begin[sc] + threadIdx.x; i < sc_begin[sc + 1]; i += blockDim.x)
    b[i] = act ? (T)r[i] : T(0);
}

template <typename T>
__global__ void k_amg_add(int64_t n, const T* __restrict__ a, T* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] += a[i];
}

// inner-solve bookkeeping read by the outer loop: cycles per active part, status ok
__global__ void k_amg_info(int P, const int* __restrict__ active, int cycles, int* __restrict__ out_inner,
                           int* __restrict__ cg_info) {
  for (int p = threadIdx.x; p < P; p += blockDim.x) out_inner[p] = active[p] ? cycles : 0;
  if (threadIdx.x == 0) { cg_info[0] = 0; cg_info[1] = cycles; }
}

template <typename T>
cudaError_t csr_launch(const CsrDev<T>& M, const T* v, const T* b, const T* dinv, T w, int mode, T* y,
                       cudaStream_t s) {
  if (M.n == 0) return cudaSuccess;
  const unsigned g = blocks_for(M.n * M.lanes, kAmgThreads);
  switch (M.lanes) {
    case 32: k_amg_csr<T, 32><<<g, kAmgThreads, 0, s>>>(M.n, M.ptr, M.idx, M.val, v, b, dinv, w, mode, y); break;
    case 8: k_amg_csr<T, 8><<<g, kAmgThreads, 0, s>>>(M.n, M.ptr, M.idx, M.val, v, b, dinv, w, mode, y); break;
    case 4: k_amg_csr<T, 4><<<g, kAmgThreads, 0, s>>>(M.n, M.ptr, M.idx, M.val, v, b, dinv, w, mode, y); break;
    default: k_amg_csr<T, 1><<<g, kAmgThreads, 0, s>>>(M.n, M.ptr, M.idx, M.val, v, b, dinv, w, mode, y); break;
  }
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t upload_csr(fvgb_mesh_s* m, const HostCsr& h, CsrDev<T>& d, cudaStream_t s) {
  d.n = h.n;
  d.m = h.m;
  d.nnz = (int64_t)h.idx.size();
  const double mean = h.n > 0 ? (double)d.nnz / (double)h.n : 0.0;
  d.lanes = mean <= 6.0 ? 1 : mean <= 24.0 ? 4 : mean <= 64.0 ? 8 : 32;
  cudaError_t e;
  if ((e = dupload(m, &d.ptr, h.ptr, s))) return e;
  if ((e = dupload(m, &d.idx, h.idx, s))) return e;
  return dupload(m, &d.val, std::vector<T>(h.val.begin(), h.val.end()), s);
}

template <typename T>
std::vector<AmgDev<T>>& amg_of(AmgState* st);
template <>
std::vector<AmgDev<double>>& amg_of<double>(AmgState* st) { return st->d64; }
template <>
std::vector<AmgDev<float>>& amg_of<float>(AmgState* st) { return st->d32; }

template <typename T>
fvgb_status amg_upload(fvgb_mesh m, const AmgHost& H, AmgDev<T>& a, cudaStream_t s) {
  const int L = (int)H.levels.size();
  a.lv.resize(L);
  for (int l = 0; l < L; ++l) {
    const AmgHostLevel& h = H.levels[l];
    AmgLevelDev<T>& d = a.lv[l];
    FVGB_TRY(upload_csr<T>(m, h.A, d.A, s), "upload");
    FVGB_TRY(upload_csr<T>(m, h.P, d.P, s), "upload");
    FVGB_TRY(upload_csr<T>(m, h.R, d.R, s), "upload");
    FVGB_TRY(dupload(m, &d.dinv, std::vector<T>(h.dinv.begin(), h.dinv.end()), s), "upload");
    const int64_t n = h.A.n;
    if (l > 0) FVGB_TRY(dalloc(m, &d.b, n), "allocation");
    FVGB_TRY(dalloc(m, &d.x, n), "allocation");
    FVGB_TRY(dalloc(m, &d.xo, n), "allocation");
    FVGB_TRY(dalloc(m, &d.r, n), "allocation");
  }
  a.nco = H.coarse.n;
  FVGB_TRY(dupload(m, &a.cinv, std::vector<T>(H.coarse_inv.begin(), H.coarse_inv.end()), s), "upload");
  FVGB_TRY(dalloc(m, &a.cb, a.nco), "allocation");
  FVGB_TRY(dalloc(m, &a.cx, a.nco), "allocation");
  const int64_t N = m->topo.N;
  FVGB_TRY(dalloc(m, &a.t0, N), "allocation");
  FVGB_TRY(dalloc(m, &a.t1, N), "allocation");
  FVGB_TRY(dalloc(m, &a.t2, N), "allocation");
  a.built = true;
  return FVGB_OK;
}

// One V-cycle on level l: b -> out (zero initial guess).
template <typename T>
cudaError_t vcycle(AmgDev<T>& a, int l, const T* b, T* out, cudaStream_t s) {
  const T w = T(2.0 / 3.0);
  if (l == (int)a.lv.size()) {
    k_amg_dense<T><<<blocks_for(a.nco * 32, kAmgThreads), kAmgThreads, 0, s>>>(a.nco, a.cinv, b, out);
    count_launch();
    return cudaGetLastError();
  }
  AmgLevelDev<T>& L = a.lv[l];
  const bool last = l + 1 == (int)a.lv.size();
  T* nb = last ? a.cb : a.lv[l + 1].b;
  T* nx = last ? a.cx : a.lv[l + 1].xo;
  cudaError_t e;
  k_amg_jacobi0<T><<<blocks_for(L.A.n, kAmgThreads), kAmgThreads, 0, s>>>(L.A.n, L.dinv, b, L.x, w);
  count_launch();
  if ((e = cudaGetLastError())) return e;
  if ((e = csr_launch(L.A, L.x, b, L.dinv, w, 2, L.r, s))) return e;          // r = b - A x
  if ((e = csr_launch(L.R, L.r, (const T*)nullptr, L.dinv, w, 0, nb, s))) return e;   // b' = R r
  if ((e = vcycle(a, l + 1, nb, nx, s))) return e;
  if ((e = csr_launch(L.P, nx, (const T*)nullptr, L.dinv, w, 1, L.x, s))) return e;   // x += P x'
  return csr_launch(L.A, L.x, b, L.dinv, w, 3, out, s);                        // smoothing
}

}  // namespace

fvgb_status amg_ensure(fvgb_mesh m, int bcset, bool fp32, cudaStream_t s) {
  if (!m->amg) m->amg = new AmgState();
  AmgState* st = m->amg;
  const size_t nb = m->g64.bc.size();
  if (st->d64.size() != nb) st->d64.resize(nb);
  if (st->d32.size() != nb) st->d32.resize(nb);
  if (fp32 ? st->d32[bcset].built : st->d64[bcset].built) return FVGB_OK;
  const TopoDev& t = m->topo;
  const int64_t N = t.N;
  const BCDev<double>& b = m->g64.bc[bcset];
  std::vector<int32_t> nbr(4 * N);
  std::vector<double> coef(4 * N), diag(N), cen(t.dim * N), vol(N);
  FVGB_TRY(cudaStreamSynchronize(s), "synchronize");
  FVGB_TRY(cudaMemcpy(nbr.data(), b.at_nbr, nbr.size() * sizeof(int32_t), cudaMemcpyDeviceToHost), "copy");
  FVGB_TRY(cudaMemcpy(coef.data(), b.at_coef, coef.size() * sizeof(double), cudaMemcpyDeviceToHost), "copy");
  FVGB_TRY(cudaMemcpy(diag.data(), b.at_diag, N * sizeof(double), cudaMemcpyDeviceToHost), "copy");
  FVGB_TRY(cudaMemcpy(cen.data(), m->g64.cen, cen.size() * sizeof(double), cudaMemcpyDeviceToHost), "copy");
  FVGB_TRY(cudaMemcpy(vol.data(), m->g64.vol, N * sizeof(double), cudaMemcpyDeviceToHost), "copy");
  AmgHost H;
  const std::string err = amg_build(t.dim, N, nbr.data(), coef.data(), diag.data(), cen.data(), vol.data(),
                                    m->part_cell_begin, H);
  if (!err.empty()) { set_error("multigrid setup: " + err); return FVGB_EMESH; }
  fvgb_status r = fp32 ? amg_upload<float>(m, H, st->d32[bcset], s) : amg_upload<double>(m, H, st->d64[bcset], s);
  if (r) return r;
  FVGB_TRY(cudaStreamSynchronize(s), "synchronize");
  return FVGB_OK;
}

void amg_release(fvgb_mesh m) {
  delete m->amg;   // device memory is in m->allocs
  m->amg = nullptr;
}

int amg_levels(fvgb_mesh m, int bcset, bool fp32, int64_t* sizes, int cap) {
  if (!m->amg || bcset < 0 || (size_t)bcset >= m->amg->d64.size()) return 0;
  auto fill = [&](auto& a) {
    if (!a.built) return 0;
    int k = 0;
    for (auto& L : a.lv) { if (k < cap) sizes[k] = L.A.n; ++k; }
    if (k < cap) sizes[k] = a.nco;
    return k + 1;
  };
  return fp32 ? fill(m->amg->d32[bcset]) : fill(m->amg->d64[bcset]);
}

// delta (work_of<T>(m).cg_x) = `cycles` V-cycles on A_T delta = r (masked to the active
// parts); the outer loop's inner bookkeeping is filled as for the CG.
template <typename T>
cudaError_t launch_amg_inner(fvgb_mesh_s* m, int bcset, const double* r, int cycles, cudaStream_t s) {
  AmgDev<T>& a = amg_of<T>(m->amg)[bcset];
  Work<T>& w = work_of<T>(m);
  const PartsDev& pd = m->parts;
  const int64_t N = m->topo.N;
  cudaError_t e;
  k_amg_rhs<T><<<pd.n_sc, 256, 0, s>>>(r, pd.sc_begin, pd.sc_part, pd.active, a.t0);
  count_launch();
  if ((e = cudaGetLastError())) return e;
  if ((e = vcycle(a, 0, a.t0, w.cg_x, s))) return e;
  // with no levels (a mesh of at most kAmgCoarseMax cells) the dense solve is exact
  for (int c = 1; c < cycles && !a.lv.empty(); ++c) {
    if ((e = csr_launch(a.lv[0].A, w.cg_x, a.t0, a.lv[0].dinv, T(0), 2, a.t1, s))) return e;
    if ((e = vcycle(a, 0, a.t1, a.t2, s))) return e;
    k_amg_add<T><<<blocks_for(N, kAmgThreads), kAmgThreads, 0, s>>>(N, a.t2, w.cg_x);
    count_launch();
    if ((e = cudaGetLastError())) return e;
  }
  k_amg_info<<<1, 128, 0, s>>>(pd.n_part, pd.active, cycles, pd.out_inner, m->d_cg_info);
  count_launch();
  return cudaGetLastError();
}

template cudaError_t launch_amg_inner<float>(fvgb_mesh_s*, int, const double*, int, cudaStream_t);
template cudaError_t launch_amg_inner<double>(fvgb_mesh_s*, int, const double*, int, cudaStream_t);

}  // namespace fvgb
