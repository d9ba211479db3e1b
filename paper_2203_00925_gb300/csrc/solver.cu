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

// Block-wide FP64 sum in a fixed order: a shared-memory tree over the block's threads,
// finished by warp 0. Few FP64 instructions per thread (GB300's FP64 rate is low).
__device__ __forceinline__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (unsigned s = blockDim.x >> 1; s >= 32; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = sh[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// Grid-wide FP64 sums of K values in a fixed order (block tree, then warp 0 of every
// block sums the block partials in the same order); ``part`` alternates between two
// halves so that a fast block never overwrites partials a slow block is still reading.
// Returns false when the grid barrier gave up. The sums land in out (shared memory).
template <int K>
__device__ bool grid_sum(const double (&v)[K], double* part, int parity, Barrier* bar,
                         double* sh, double* out) {
  static_assert(K <= 2, "at most two sums per reduction");
  const unsigned nb = gridDim.x;
  double* base = part + (size_t)parity * nb * 2;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double t = block_sum(v[k], sh);
    if (threadIdx.x == 0) base[k * nb + blockIdx.x] = t;
    __syncthreads();
  }
  if (!grid_barrier(bar, nb)) return false;
  if (threadIdx.x < 32) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double t = 0.0;
      for (unsigned b = threadIdx.x; b < nb; b += 32) t += __ldcg(base + k * nb + b);
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (threadIdx.x == 0) out[k] = t;
    }
  }
  __syncthreads();
  return true;
}

template <typename T>
struct CgArgs {
  int64_t N;
  const int32_t* nbr;   // [N][4]
  const T* coef;        // [N][4]
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

// Four operator coefficients of one row, loaded with vector loads.
template <typename T>
struct Coef4;
template <>
struct Coef4<float> {
  float c[4];
  __device__ __forceinline__ void load(const float* p, int64_t i) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p) + i);
    c[0] = v.x; c[1] = v.y; c[2] = v.z; c[3] = v.w;
  }
};
template <>
struct Coef4<double> {
  double c[4];
  __device__ __forceinline__ void load(const double* p, int64_t i) {
    const double2 v0 = __ldg(reinterpret_cast<const double2*>(p) + 2 * i);
    const double2 v1 = __ldg(reinterpret_cast<const double2*>(p) + 2 * i + 1);
    c[0] = v0.x; c[1] = v0.y; c[2] = v1.x; c[3] = v1.y;
  }
};

// Rows per thread per trip through a phase: all loads of the trip are issued before any
// store so that the gathers of several rows are in flight together.
template <typename T>
__host__ __device__ constexpr int unroll_rows() { return sizeof(T) == 4 ? 4 : 2; }

// Phase 1: x += alpha p, r -= alpha q (own rows); returns this thread's sum of r^2.
template <typename T>
__device__ __forceinline__ T cg_phase_xr(const CgArgs<T>& a, int64_t lo, int64_t hi, T alpha) {
  T* __restrict__ X = a.x;
  T* __restrict__ R = a.r;
  const T* __restrict__ P = a.p;
  const T* __restrict__ Q = a.q;
  constexpr int kUnroll = unroll_rows<T>();
  T acc = T(0);
  const int64_t bd = blockDim.x;
  for (int64_t b = lo + threadIdx.x; b < hi; b += kUnroll * bd) {
    T x[kUnroll], p[kUnroll], r[kUnroll], q[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t i = b + u * bd;
      if (i < hi) { x[u] = X[i]; p[u] = P[i]; r[u] = R[i]; q[u] = Q[i]; }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t i = b + u * bd;
      if (i < hi) {
        const T rn = r[u] - alpha * q[u];
        X[i] = x[u] + alpha * p[u];
        R[i] = rn;
        acc += rn * rn;
      }
    }
  }
  return acc;
}

// Phase 2: p = r + beta p, q = A_T r + beta q (= A_T p); returns this thread's sum of
// p.q. Neighbours' r are read through L2 (other blocks wrote them this iteration).
template <typename T>
__device__ __forceinline__ T cg_phase_pq(const CgArgs<T>& a, int64_t lo, int64_t hi, T beta,
                                         const T* v_src) {
  T* __restrict__ P = a.p;
  T* __restrict__ Q = a.q;
  const T* __restrict__ R = v_src;
  const int4* __restrict__ NB = reinterpret_cast<const int4*>(a.nbr);
  constexpr int kUnroll = unroll_rows<T>();
  T acc = T(0);
  const int64_t bd = blockDim.x;
  for (int64_t b = lo + threadIdx.x; b < hi; b += kUnroll * bd) {
    T r[kUnroll], p[kUnroll], q[kUnroll], d[kUnroll], g[kUnroll][4];
    int4 nb[kUnroll];
    Coef4<T> c[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t i = b + u * bd;
      if (i < hi) {
        nb[u] = __ldg(NB + i);
        r[u] = R[i]; p[u] = P[i]; q[u] = Q[i];
        d[u] = __ldg(a.diag + i);
        c[u].load(a.coef, i);
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t i = b + u * bd;
      if (i < hi) {
        g[u][0] = __ldcg(R + nb[u].x);
        g[u][1] = __ldcg(R + nb[u].y);
        g[u][2] = __ldcg(R + nb[u].z);
        g[u][3] = __ldcg(R + nb[u].w);
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t i = b + u * bd;
      if (i < hi) {
        T y = d[u] * r[u];
        y -= c[u].c[0] * g[u][0];
        y -= c[u].c[1] * g[u][1];
        y -= c[u].c[2] * g[u][2];
        y -= c[u].c[3] * g[u][3];
        const T pn = r[u] + beta * p[u];
        const T qn = y + beta * q[u];
        P[i] = pn;
        Q[i] = qn;
        acc += pn * qn;
      }
    }
  }
  return acc;
}

// Conjugate gradients with two grid barriers per iteration: after the residual update
// (and its norm) every block forms p = r + beta p and q = A_T r + beta q = A_T p from the
// finished r, so no barrier is needed between the p update and the operator.
// Dot products: each thread accumulates its own rows in T, the sums across threads and
// blocks are FP64 in a fixed order. The scalars alpha, beta and the stopping test are
// computed once per block (thread 0) and broadcast through shared memory.
template <typename T>
__global__ void __launch_bounds__(kCgThreads) k_cg(CgArgs<T> a) {
  __shared__ double sh[kCgThreads];
  __shared__ double tot[2];
  __shared__ T s_alpha, s_beta;
  __shared__ int s_state;   // 0 continue, 1 converged, 2 breakdown / non-finite, 3 zero rhs
  const int64_t N = a.N;
  const unsigned nb = gridDim.x;
  const int64_t chunk = (N + nb - 1) / nb;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < N ? lo + chunk : N;
  int parity = 0;
  int its = 0;
  double rr = 0.0, rr0 = 0.0;   // meaningful in thread 0
  if (threadIdx.x == 0) s_state = 0;

  // r = rhs, p = 0, q = 0, x = 0: the first p/q phase (beta = 0) then gives p = r, q = A_T r
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const T ri = (T)a.rhs[i];
    a.r[i] = ri;
    a.p[i] = T(0);
    a.q[i] = T(0);
    a.x[i] = T(0);
  }
  if (!grid_barrier(a.bar, nb)) goto done;
  {
    T l0 = T(0);
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const T ri = a.r[i];
      l0 += ri * ri;
    }
    const T l1 = cg_phase_pq<T>(a, lo, hi, T(0), a.r);
    const double loc[2] = {(double)l0, (double)l1};
    if (!grid_sum<2>(loc, a.part, parity, a.bar, sh, tot)) goto done;
    if (threadIdx.x == 0) {
      rr = rr0 = tot[0];
      const double pq = tot[1];
      s_state = !(rr0 > 0.0) ? (rr0 == 0.0 ? 3 : 2) : (!(pq > 0.0) || !isfinite(pq) ? 2 : 0);
      s_alpha = (T)(rr / pq);
    }
    __syncthreads();
    while (s_state == 0 && its < a.maxit) {
      const T lr = cg_phase_xr<T>(a, lo, hi, s_alpha);
      parity ^= 1;
      const double l1v[1] = {(double)lr};
      if (!grid_sum<1>(l1v, a.part, parity, a.bar, sh, tot)) goto done;
      ++its;
      if (threadIdx.x == 0) {
        const double rrn = tot[0];
        if (!isfinite(rrn)) s_state = 2;
        else if (rrn <= a.tol2 * rr0) s_state = 1;
        s_beta = (T)(rrn / rr);
        rr = rrn;
      }
      __syncthreads();
      if (s_state != 0) break;
      const T lpq = cg_phase_pq<T>(a, lo, hi, s_beta, a.r);
      parity ^= 1;
      const double l2v[1] = {(double)lpq};
      if (!grid_sum<1>(l2v, a.part, parity, a.bar, sh, tot)) goto done;
      if (threadIdx.x == 0) {
        const double pq = tot[0];
        if (!(pq > 0.0) || !isfinite(pq)) s_state = 2;
        s_alpha = (T)(rr / pq);
      }
      __syncthreads();
    }
  }
done:
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.info[0] = its;
    a.info[1] = s_state == 2 ? 2 : 0;
    a.res[0] = rr0;
    a.res[1] = rr;
  }
}

template <typename T>
const void* cg_kernel(int) {
  return (const void*)k_cg<T>;
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
