// Inner conjugate-gradient solve of the Poisson refinement loop: A_T delta = r on the
// symmetric positive definite two-point part A_T of the diamond operator (eq.
// "laplace" keeps, per face, the term |S_f|^2 / ((x_R - x_L) . S_f) (P_R - P_L)).
//
// One persistent cooperative launch runs the whole CG loop: each block owns a
// contiguous range of cells, vectors are in T (float or double), every dot product is
// accumulated in FP64 and reduced in a fixed order (block partials -> every block sums
// all partials in the same order), so all blocks take the same decisions and the
// result is bitwise reproducible for a given grid size. Grid-wide barriers are
// bounded: a barrier that waits longer than one second sets a status word and every
// block leaves the loop; the host reports FVGB_ETIMEOUT.
#include <cuda_runtime.h>

#include "internal.h"

namespace fvgb {
namespace {

constexpr unsigned long long kBarrierTimeoutNs = 1000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Sense-by-generation grid barrier with a bounded wait. Returns false when any block
// gave up (status set), in which case the caller leaves its loop.
__device__ bool grid_barrier(Barrier* bar, unsigned nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &bar->gen;
    volatile int* vstatus = &bar->status;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&bar->count, 1u);
    int good = 1;
    if (arrived == nblocks - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*vgen == g) {
        if (*vstatus != 0) { good = 0; break; }
        if (global_ns() - t0 > kBarrierTimeoutNs) { atomicExch(&bar->status, 1); good = 0; break; }
        __nanosleep(32);
      }
    }
    if (*vstatus != 0) good = 0;
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

// Grid-wide FP64 sums of NV values in a fixed order; ``part`` alternates between two
// halves so that a fast block never overwrites partials a slow block is still reading.
template <int K>
__device__ bool grid_sum(const double (&v)[K], double* part, int parity, Barrier* bar,
                         double* sh, double (&out)[K]) {
  const unsigned nb = gridDim.x;
  __shared__ double result[K];
  static_assert(K <= 2, "at most two sums per reduction");
  double* base = part + (size_t)parity * nb * 2;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double t = block_sum(v[k], sh);
    if (threadIdx.x == 0) base[k * nb + blockIdx.x] = t;
  }
  if (!grid_barrier(bar, nb)) return false;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
    for (unsigned b = threadIdx.x; b < nb; b += blockDim.x) s += __ldcg(base + k * nb + b);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) result[k] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = result[k];
  return true;
}

template <typename T>
struct CgArgs {
  int64_t N;
  const int32_t* nbr;   // [NV][N]
  const T* coef;        // [NV][N]
  const T* diag;        // [N]
  const double* rhs;    // [N]
  T* x;
  T* r;
  T* p;
  T* q;
  double* part;         // [2][2][grid]
  Barrier* bar;
  int* info;            // [0] iterations, [1] 0 ok / 2 non-finite or breakdown
  double* res;          // [0] rr0, [1] final rr
  double tol2;
  int maxit;
};

// y_i = (A_T v)_i for one row; neighbours' v are read through L2 (other blocks wrote them).
template <typename T, int NV>
__device__ __forceinline__ T at_row(const CgArgs<T>& a, const T* v, int64_t i, T vi) {
  T y = a.diag[i] * vi;
#pragma unroll
  for (int s = 0; s < NV; ++s) {
    const int32_t n = a.nbr[s * a.N + i];
    if (n >= 0) y -= a.coef[s * a.N + i] * __ldcg(v + n);
  }
  return y;
}

// Conjugate gradients with two grid barriers per iteration: after the residual update
// (and its norm) every block forms p = r + beta p and q = A_T r + beta q = A_T p from the
// finished r, so no barrier is needed between the p update and the operator.
template <typename T, int NV>
__global__ void __launch_bounds__(kCgThreads) k_cg(CgArgs<T> a) {
  __shared__ double sh[32];
  const int64_t N = a.N;
  const unsigned nb = gridDim.x;
  const int64_t chunk = (N + nb - 1) / nb;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < N ? lo + chunk : N;
  int parity = 0;
  int its = 0, bad = 0;
  double rr = 0.0, rr0 = 0.0;

  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const T ri = (T)a.rhs[i];
    a.r[i] = ri;
    a.p[i] = ri;
    a.x[i] = T(0);
  }
  if (!grid_barrier(a.bar, nb)) goto done;
  {
    double loc[2] = {0.0, 0.0}, tot[2];
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const T pi = a.p[i];
      const T y = at_row<T, NV>(a, a.p, i, pi);
      a.q[i] = y;
      loc[0] += (double)pi * (double)pi;
      loc[1] += (double)pi * (double)y;
    }
    if (!grid_sum<2>(loc, a.part, parity, a.bar, sh, tot)) goto done;
    rr = rr0 = tot[0];
    double pq = tot[1];
    if (!(rr0 > 0.0)) { bad = rr0 == 0.0 ? 0 : 2; goto done; }
    while (its < a.maxit) {
      if (!(pq > 0.0) || !isfinite(pq)) { bad = 2; break; }
      const T alpha = (T)(rr / pq);
      double l1[1] = {0.0}, t1[1];
      for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        a.x[i] += alpha * a.p[i];
        const T ri = a.r[i] - alpha * a.q[i];
        a.r[i] = ri;
        l1[0] += (double)ri * (double)ri;
      }
      parity ^= 1;
      if (!grid_sum<1>(l1, a.part, parity, a.bar, sh, t1)) goto done;
      const double rrn = t1[0];
      ++its;
      if (!isfinite(rrn)) { bad = 2; break; }
      if (rrn <= a.tol2 * rr0) { rr = rrn; break; }
      const T beta = (T)(rrn / rr);
      rr = rrn;
      double l2[1] = {0.0}, t2[1];
      for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const T ri = a.r[i];
        const T pi = ri + beta * a.p[i];
        const T qi = at_row<T, NV>(a, a.r, i, ri) + beta * a.q[i];
        a.p[i] = pi;
        a.q[i] = qi;
        l2[0] += (double)pi * (double)qi;
      }
      parity ^= 1;
      if (!grid_sum<1>(l2, a.part, parity, a.bar, sh, t2)) goto done;
      pq = t2[0];
    }
  }
done:
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.info[0] = its;
    a.info[1] = bad;
    a.res[0] = rr0;
    a.res[1] = rr;
  }
}

template <typename T>
const void* cg_kernel(int nv) {
  return nv == 4 ? (const void*)k_cg<T, 4> : (const void*)k_cg<T, 3>;
}

}  // namespace

int cg_grid_size(fvgb_mesh_s* m, bool fp32) {
  int per_sm = 0;
  const void* k = fp32 ? cg_kernel<float>(m->topo.dim + 1) : cg_kernel<double>(m->topo.dim + 1);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kCgThreads, 0) != cudaSuccess)
    return 0;
  if (per_sm > 2) per_sm = 2;
  int grid = per_sm * m->num_sms;
  // no more blocks than there are cells to own
  const int64_t need = (m->topo.N + kCgThreads - 1) / kCgThreads;
  if (need < grid) grid = need > 0 ? (int)need : 1;
  return grid;
}

template <typename T>
cudaError_t launch_cg(fvgb_mesh_s* m, int bcset, const double* rhs, double rtol, int maxit,
                      cudaStream_t s) {
  GeoDev<T>& g = geo_of<T>(m);
  Work<T>& w = work_of<T>(m);
  const BCDev<T>& b = g.bc[bcset];
  CgArgs<T> a;
  a.N = m->topo.N;
  a.nbr = b.at_nbr;
  a.coef = b.at_coef;
  a.diag = b.at_diag;
  a.rhs = rhs;
  a.x = w.cg_x;
  a.r = w.cg_r;
  a.p = w.cg_p;
  a.q = w.cg_q;
  a.part = m->d_scal + 8 + kRedBlocks;
  a.bar = m->barrier;
  a.info = m->d_cg_info;
  a.res = m->d_scal + 2;
  a.tol2 = rtol * rtol;
  a.maxit = maxit;
  const int grid = sizeof(T) == 4 ? m->cg_grid32 : m->cg_grid64;
  cudaError_t e = cudaMemsetAsync(m->barrier, 0, sizeof(Barrier), s);
  if (e != cudaSuccess) return e;
  void* args[] = {&a};
  count_launch();
  return cudaLaunchCooperativeKernel(cg_kernel<T>(m->topo.dim + 1), dim3(grid), dim3(kCgThreads),
                                     args, 0, s);
}

template cudaError_t launch_cg<double>(fvgb_mesh_s*, int, const double*, double, int, cudaStream_t);
template cudaError_t launch_cg<float>(fvgb_mesh_s*, int, const double*, double, int, cudaStream_t);

}  // namespace fvgb
