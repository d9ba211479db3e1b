// Inner solve of the Poisson refinement loop (eq. 1.1 discretised by eq. 7 /
// eq. "laplace"): conjugate gradients on the SPD two-point part A_T of the diamond
// operator (per face the term |S_f|^2 / ((x_R - x_L) . S_f) (P_R - P_L)), A_T delta = r,
// in T = float or double with FP64 dot products, as ONE persistent cooperative kernel.
//
// A mesh may hold several independent parts (an ensemble of meshes packed into one
// index space); every part has its own CG scalars and stopping test, and only the parts
// flagged active by the outer loop are solved (delta = 0 elsewhere).
//
// Work split: block b owns the contiguous cell range [b N / G, (b+1) N / G), cut at part
// boundaries into "sub-chunks" (one part each). Every sum is formed per sub-chunk (block
// tree), then per part over its sub-chunks in a fixed order by every block, so all
// blocks take the same decisions and results are bitwise reproducible for a given grid.
// The same decomposition gives the per-part norms of the outer loop (k_part_sumsq).
//
// Grid-wide barriers are bounded: a wait longer than one second (or the limit set by the
// test hook fvgb_test_barrier) sets a status word and every block leaves; the host
// reports FVGB_ETIMEOUT.
#include <cuda_runtime.h>

#include "internal.h"

namespace fvgb {
namespace {

constexpr unsigned long long kBarrierTimeoutNs = 1000000000ull;   // default wait limit

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier on a monotone arrival counter with a bounded wait: the r-th barrier of a
// launch is passed once the counter (zeroed before the launch) reaches r * nblocks, so
// the last arrival itself releases the waiting blocks (no reset, no second word).
// ``target`` is the caller's running count. Returns false when any block gave up
// (status set), in which case the caller leaves. ``skip`` (test hook only) leaves out this
// block's arrival, so that the other blocks' waits run out.
__device__ bool grid_barrier(Barrier* bar, unsigned nblocks, unsigned& target, bool skip,
                             unsigned long long limit_ns) {
  __shared__ int ok;
  __syncthreads();
  target += nblocks;
  if (threadIdx.x == 0) {
    volatile unsigned* vcount = &bar->count;
    volatile int* vstatus = &bar->status;
    __threadfence();
    if (!skip) atomicAdd(&bar->count, 1u);
    int good = 1;
    if ((int)(*vcount - target) < 0) {
      const unsigned long long t0 = global_ns();
      while ((int)(*vcount - target) < 0) {
        if (*vstatus != 0) { good = 0; break; }
        if (global_ns() - t0 > limit_ns) { atomicExch(&bar->status, 1); good = 0; break; }
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

// Block-wide FP64 sum in a fixed order, valid in thread 0. Every thread's value goes to
// shared memory; four warps (one per SM sub-partition) each add a quarter of them, lane
// by lane in index order and then by a shuffle tree, and thread 0 adds the four results.
// GB300 issues FP64 adds at a small fraction of the FP32 rate, so the sum keeps the FP64
// instructions on its critical path few and spread over the four sub-partitions.
// sh holds blockDim.x doubles (blockDim.x a multiple of 128).
__device__ __forceinline__ double block_sum(double v, double* sh) {
  __syncthreads();                      // the previous call's readers are done with sh
  sh[threadIdx.x] = v;
  __syncthreads();
  double t = 0.0;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int quarter = blockDim.x >> 2;
  if (w < 4) {
    const double* q = sh + w * quarter;
    t = q[l];
    for (int j = l + 32; j < quarter; j += 32) t += q[j];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  __syncthreads();                      // every quarter read before the results overwrite sh
  if (w < 4 && l == 0) sh[w] = t;
  __syncthreads();
  if (threadIdx.x == 0) t = (sh[0] + sh[1]) + (sh[2] + sh[3]);
  return t;
}

// Block-wide FP64 sum in a fixed order for launches over many parts: a shuffle tree inside
// each warp, then warp 0 sums the warp totals in warp order. Valid in thread 0. Measured
// faster than block_sum on the 64-mesh ensemble, whose short inner solves leave most
// blocks summing finished or tiny sub-chunks; block_sum is faster on a single mesh.
__device__ __forceinline__ double block_sum_tree(double v, double* sh) {
  __syncthreads();                      // the previous call's readers are done with sh
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;
}

// the block sum of the CG kernel: by part count (uniform over the grid)
__device__ __forceinline__ double cg_block_sum(double v, double* sh, bool many_parts) {
  return many_parts ? block_sum_tree(v, sh) : block_sum(v, sh);
}

template <typename T>
struct SolveArgs {
  int64_t N;
  // two-point operator scaled to unit diagonal, D^-1/2 A_T D^-1/2, in T, cell-major [N][4]
  const int32_t* at_nbr;
  const T* at_scoef;
  const T* at_isd;          // [N] D^-1/2: the CG solves for D^1/2 x from D^-1/2 r
  const double* r_in;       // [N] right-hand side (FP64 outer residual)
  T* cx;
  T* cr;
  T* cp;
  T* cq;
  // parts
  int n_part;
  int n_sc;
  const int32_t* blk_sc;    // [G+1]
  const int64_t* sc_begin;  // [n_sc+1]
  const int32_t* sc_part;   // [n_sc]
  const int32_t* part_sc;   // [P+1]
  const int* active;        // [P] parts to solve
  double* buf;              // [2][2][n_sc] partial sums
  Barrier* bar;
  double inner_tol2;
  int maxit_inner;
  int* out_inner;           // [P] iterations per part
  int* out_status;          // [0]: 0 ok, 6 non-finite / breakdown; [1]: iterations run
  int skip_block;           // test hook: this block never arrives at a barrier (-1: none)
  unsigned long long barrier_ns;  // limit of a barrier wait
};

// Sum the per-sub-chunk partials of K quantities into per-part totals (shared memory
// tot[k * P + p]), every part in sub-chunk order. Call after a grid barrier. The partials
// are first staged in shared memory with one load per thread (one L2 round trip). A part
// of at most kSeqSubChunks sub-chunks is summed by one thread, left to right; a longer
// one by one warp: lanes stride 32 over its sub-chunks, then a shuffle tree. (A warp-wide
// FP64 add costs the same whatever its active lanes, so the few adds of the short parts
// of an ensemble are cheaper in one thread than in a five-level shuffle tree.)
constexpr int kSeqSubChunks = 8;

template <typename T, int K>
__device__ void part_totals(const SolveArgs<T>& a, const double* buf, double* tot,
                            double (*stage)[kCgThreads]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const bool staged = a.n_sc <= (int)blockDim.x;
  if (staged) {
#pragma unroll
    for (int k = 0; k < K; ++k)
      if ((int)threadIdx.x < a.n_sc) stage[k][threadIdx.x] = __ldcg(buf + (size_t)k * a.n_sc + threadIdx.x);
    __syncthreads();
  }
  for (int p = threadIdx.x; p < a.n_part; p += blockDim.x) {
    const int s0 = a.part_sc[p], s1 = a.part_sc[p + 1];
    if (s1 - s0 > kSeqSubChunks) continue;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double t = 0.0;
      for (int sc = s0; sc < s1; ++sc) t += staged ? stage[k][sc] : __ldcg(buf + (size_t)k * a.n_sc + sc);
      tot[k * a.n_part + p] = t;
    }
  }
  for (int p = warp; p < a.n_part; p += nw) {
    if (a.part_sc[p + 1] - a.part_sc[p] <= kSeqSubChunks) continue;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double t = 0.0;
      for (int sc = a.part_sc[p] + lane; sc < a.part_sc[p + 1]; sc += 32)
        t += staged ? stage[k][sc] : __ldcg(buf + (size_t)k * a.n_sc + sc);
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0) tot[k * a.n_part + p] = t;
    }
  }
  __syncthreads();
}

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

// Rows per thread per trip: all loads of a trip are issued before any store so that the
// gathers of several rows are in flight together.
template <typename T>
__host__ __device__ constexpr int unroll_rows() { return sizeof(T) == 4 ? 4 : 2; }
// the x/r phase holds four values a row: more FP64 rows per trip (measured: four FP32 rows
// a trip beat eight on the 64-mesh ensemble and on the 750,000-cell mixed step)
template <typename T>
__host__ __device__ constexpr int unroll_rows_xr() { return 4; }

// CG phase 1 on rows [lo, hi): r -= alpha q; returns the thread's sum of r^2. (The matching
// x += alpha p is deferred to the next phase 2, which reads p anyway, or to the final pass:
// the same additions in the same order, without streaming x and p through this phase.)
template <typename T>
__device__ __forceinline__ T cg_phase_r(const SolveArgs<T>& a, int64_t lo, int64_t hi, T alpha) {
  constexpr int U = unroll_rows_xr<T>();
  T* __restrict__ R = a.cr;
  const T* __restrict__ Q = a.cq;
  T acc = T(0);
  const int64_t bd = blockDim.x;
  for (int64_t b = lo + threadIdx.x; b < hi; b += U * bd) {
    T r[U], q[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = b + u * bd;
      if (i < hi) { r[u] = R[i]; q[u] = Q[i]; }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = b + u * bd;
      if (i < hi) {
        const T rn = r[u] - alpha * q[u];
        R[i] = rn;
        acc += rn * rn;
      }
    }
  }
  return acc;
}

// The final pass on rows [lo, hi): the deferred x += alpha p of the part's last phase 1
// (pending), then back from the scaled unknowns, x = D^-1/2 x.
template <typename T>
__device__ __forceinline__ void cg_phase_x(const SolveArgs<T>& a, int64_t lo, int64_t hi, bool pending, T alpha) {
  T* __restrict__ X = a.cx;
  const T* __restrict__ P = a.cp;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const T x = pending ? X[i] + alpha * P[i] : X[i];
    X[i] = x * __ldg(a.at_isd + i);
  }
}

// CG phase 2 on rows [lo, hi): x += alpha p (the previous phase 1's update, with the old p),
// p = r + beta p, q = S r + beta q (= S p, S = D^-1/2 A_T D^-1/2 with unit diagonal);
// returns the thread's sum of p.q. Neighbours' r are read through L2 (other blocks wrote
// them).
template <typename T>
__device__ __forceinline__ T cg_phase_pq(const SolveArgs<T>& a, int64_t lo, int64_t hi, T beta, T alpha) {
  constexpr int U = unroll_rows<T>();
  T* __restrict__ P = a.cp;
  T* __restrict__ Q = a.cq;
  T* __restrict__ X = a.cx;
  const T* __restrict__ R = a.cr;
  const int4* __restrict__ NB = reinterpret_cast<const int4*>(a.at_nbr);
  T acc = T(0);
  const int64_t bd = blockDim.x;
  for (int64_t b = lo + threadIdx.x; b < hi; b += U * bd) {
    T r[U], p[U], q[U], x[U], g[U][4];
    int4 nb[U];
    Coef4<T> c[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = b + u * bd;
      if (i < hi) {
        nb[u] = __ldg(NB + i);
        r[u] = R[i]; p[u] = P[i]; q[u] = Q[i]; x[u] = X[i];
        c[u].load(a.at_scoef, i);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = b + u * bd;
      if (i < hi) {
        g[u][0] = __ldcg(R + nb[u].x);
        g[u][1] = __ldcg(R + nb[u].y);
        g[u][2] = __ldcg(R + nb[u].z);
        g[u][3] = __ldcg(R + nb[u].w);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = b + u * bd;
      if (i < hi) {
        T y = r[u];                     // unit diagonal
        y -= c[u].c[0] * g[u][0];
        y -= c[u].c[1] * g[u][1];
        y -= c[u].c[2] * g[u][2];
        y -= c[u].c[3] * g[u][3];
        const T pn = r[u] + beta * p[u];
        const T qn = y + beta * q[u];
        X[i] = x[u] + alpha * p[u];
        P[i] = pn;
        Q[i] = qn;
        acc += pn * qn;
      }
    }
  }
  return acc;
}

// One 512-thread block per SM (measured faster than two smaller-register blocks: fewer
// grid-barrier arrivals and partial sums, more rows in flight per thread).
template <typename T>
__global__ void __launch_bounds__(kCgThreads, kCgBlocksPerSm) k_cg(SolveArgs<T> a) {
  __shared__ double sh[kCgThreads];
  __shared__ double stage[2][kCgThreads];
  __shared__ double tot[2 * kMaxParts];
  __shared__ double s_rr[kMaxParts], s_rr0[kMaxParts];
  __shared__ T s_alpha[kMaxParts], s_beta[kMaxParts];
  __shared__ int s_cg[kMaxParts];      // 0 running, 1 converged, 2 breakdown, 3 idle
  __shared__ int s_inner[kMaxParts];
  __shared__ int s_pend[kMaxParts];    // x += alpha p of the part's last phase 1 not yet applied
  __shared__ int s_flag, s_status;
  const unsigned G = gridDim.x;
  const int P = a.n_part;
  const bool many = P > 1;
  const int sc0 = a.blk_sc[blockIdx.x], sc1 = a.blk_sc[blockIdx.x + 1];
  int parity = 0;
  int total_its = 0;
  unsigned target = 0;
  if (threadIdx.x == 0) s_status = 0;
  for (int p = threadIdx.x; p < P; p += blockDim.x) { s_inner[p] = 0; s_pend[p] = 0; }

  // r = D^-1/2 rhs on active parts (0 elsewhere), p = q = x = 0; the first p/q phase
  // (beta = 0) then gives p = r, q = S r
  for (int sc = sc0; sc < sc1; ++sc) {
    const bool act = a.active[a.sc_part[sc]] != 0;
    for (int64_t i = a.sc_begin[sc] + threadIdx.x; i < a.sc_begin[sc + 1]; i += blockDim.x) {
      a.cr[i] = act ? (T)(a.r_in[i] * (double)__ldg(a.at_isd + i)) : T(0);
      a.cp[i] = T(0);
      a.cq[i] = T(0);
      a.cx[i] = T(0);
    }
  }
  if (!grid_barrier(a.bar, G, target, a.skip_block == (int)blockIdx.x, a.barrier_ns)) goto done;
  for (int sc = sc0; sc < sc1; ++sc) {
    const int p = a.sc_part[sc];
    T l0 = T(0), l1 = T(0);
    if (a.active[p]) {
      for (int64_t i = a.sc_begin[sc] + threadIdx.x; i < a.sc_begin[sc + 1]; i += blockDim.x) {
        const T ri = a.cr[i];
        l0 += ri * ri;
      }
      l1 = cg_phase_pq<T>(a, a.sc_begin[sc], a.sc_begin[sc + 1], T(0), T(0));
    }
    const double t0 = cg_block_sum((double)l0, sh, many);
    const double t1 = cg_block_sum((double)l1, sh, many);
    if (threadIdx.x == 0) { a.buf[sc] = t0; a.buf[a.n_sc + sc] = t1; }
  }
  if (!grid_barrier(a.bar, G, target, a.skip_block == (int)blockIdx.x, a.barrier_ns)) goto done;
  part_totals<T, 2>(a, a.buf, tot, stage);
  if (threadIdx.x == 0) s_flag = 0;
  __syncthreads();
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    const double rr0 = tot[p], pq = tot[P + p];
    s_rr[p] = s_rr0[p] = rr0;
    int st = 3;
    if (a.active[p]) {
      if (!(rr0 > 0.0)) st = rr0 == 0.0 ? 3 : 2;
      else st = (!(pq > 0.0) || !isfinite(pq)) ? 2 : 0;
    }
    s_cg[p] = st;
    s_alpha[p] = st == 0 ? (T)(rr0 / pq) : T(0);
    if (st == 0) atomicOr(&s_flag, 1);
  }
  __syncthreads();
  for (int its = 0; s_flag != 0 && its < a.maxit_inner; ++its) {
    parity ^= 1;
    double* buf = a.buf + (size_t)parity * 2 * a.n_sc;
    for (int sc = sc0; sc < sc1; ++sc) {
      const int p = a.sc_part[sc];
      if (s_cg[p] == 0) {             // uniform in the block
        const double t = cg_block_sum((double)cg_phase_r<T>(a, a.sc_begin[sc], a.sc_begin[sc + 1], s_alpha[p]), sh, many);
        if (threadIdx.x == 0) buf[sc] = t;
      } else if (threadIdx.x == 0) {
        buf[sc] = 0.0;
      }
    }
    if (!grid_barrier(a.bar, G, target, a.skip_block == (int)blockIdx.x, a.barrier_ns)) goto done;
    part_totals<T, 1>(a, buf, tot, stage);
    ++total_its;
    if (threadIdx.x == 0) s_flag = 0;
    __syncthreads();
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
      if (s_cg[p] != 0) continue;
      s_pend[p] = 1;
      s_inner[p] += 1;
      const double rrn = tot[p];
      if (!isfinite(rrn)) { s_cg[p] = 2; continue; }
      if (rrn <= a.inner_tol2 * s_rr0[p]) { s_cg[p] = 1; continue; }
      s_beta[p] = (T)(rrn / s_rr[p]);
      s_rr[p] = rrn;
      atomicOr(&s_flag, 1);
    }
    __syncthreads();
    if (s_flag == 0) break;
    parity ^= 1;
    buf = a.buf + (size_t)parity * 2 * a.n_sc;
    for (int sc = sc0; sc < sc1; ++sc) {
      const int p = a.sc_part[sc];
      if (s_cg[p] == 0) {             // uniform in the block
        const double t = cg_block_sum((double)cg_phase_pq<T>(a, a.sc_begin[sc], a.sc_begin[sc + 1], s_beta[p],
                                                             s_alpha[p]), sh, many);
        if (threadIdx.x == 0) buf[sc] = t;
      } else if (threadIdx.x == 0) {
        buf[sc] = 0.0;
      }
    }
    if (!grid_barrier(a.bar, G, target, a.skip_block == (int)blockIdx.x, a.barrier_ns)) goto done;
    part_totals<T, 1>(a, buf, tot, stage);
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
      if (s_cg[p] != 0) continue;
      s_pend[p] = 0;                  // phase 2 applied the pending x update
      const double pq = tot[p];
      if (!(pq > 0.0) || !isfinite(pq)) { s_cg[p] = 2; continue; }
      s_alpha[p] = (T)(s_rr[p] / pq);
    }
    __syncthreads();
  }
  // own rows: the deferred x += alpha p of the parts whose last phase was a phase 1, and
  // every row back to the unscaled correction
  __syncthreads();
  for (int sc = sc0; sc < sc1; ++sc) {
    const int p = a.sc_part[sc];
    cg_phase_x<T>(a, a.sc_begin[sc], a.sc_begin[sc + 1], s_pend[p] != 0, s_alpha[p]);
  }
  for (int p = threadIdx.x; p < P; p += blockDim.x)
    if (s_cg[p] == 2) s_status = 6;
done:
  __syncthreads();
  if (blockIdx.x == 0) {
    for (int p = threadIdx.x; p < P; p += blockDim.x) a.out_inner[p] = s_inner[p];
    if (threadIdx.x == 0) {
      a.out_status[0] = s_status;
      a.out_status[1] = total_its;
    }
  }
}

// Per-part sum of squares of an FP64 vector over the same sub-chunks (one block per
// range of the persistent grid): partials per sub-chunk, then one block sums each part's
// sub-chunks in order.
__global__ void __launch_bounds__(kCgThreads) k_part_sumsq_partial(const double* __restrict__ v,
    const int32_t* __restrict__ blk_sc, const int64_t* __restrict__ sc_begin, double* __restrict__ buf) {
  __shared__ double sh[kCgThreads];
  for (int sc = blk_sc[blockIdx.x]; sc < blk_sc[blockIdx.x + 1]; ++sc) {
    double l = 0.0;
    for (int64_t i = sc_begin[sc] + threadIdx.x; i < sc_begin[sc + 1]; i += blockDim.x) l += v[i] * v[i];
    l = block_sum(l, sh);
    if (threadIdx.x == 0) buf[sc] = l;
  }
}

__global__ void __launch_bounds__(kCgThreads) k_part_sumsq_final(const double* __restrict__ buf,
    const int32_t* __restrict__ part_sc, int n_part, double* __restrict__ out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int p = warp; p < n_part; p += nw) {
    double t = 0.0;
    for (int sc = part_sc[p] + lane; sc < part_sc[p + 1]; sc += 32) t += buf[sc];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) out[p] = t;
  }
}

// Per-part sums of r0 (r0 - r1), (r0 - r1)^2, r0^2 and r1^2 over the same sub-chunks, for
// the scale of a correction whose operator image is r0 - r1 (partials per sub-chunk: four
// block sums, in buf[k * n_sc + sc]).
__global__ void __launch_bounds__(kCgThreads) k_part_dots_partial(const double* __restrict__ r0,
    const double* __restrict__ r1, const int32_t* __restrict__ blk_sc, const int64_t* __restrict__ sc_begin,
    int n_sc, double* __restrict__ buf) {
  __shared__ double sh[kCgThreads];
  for (int sc = blk_sc[blockIdx.x]; sc < blk_sc[blockIdx.x + 1]; ++sc) {
    double a = 0.0, b = 0.0, c0 = 0.0, c1 = 0.0;
    for (int64_t i = sc_begin[sc] + threadIdx.x; i < sc_begin[sc + 1]; i += blockDim.x) {
      const double x = r0[i], y = r1[i];
      const double d = x - y;
      a += x * d;
      b += d * d;
      c0 += x * x;
      c1 += y * y;
    }
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    c0 = block_sum(c0, sh);
    c1 = block_sum(c1, sh);
    if (threadIdx.x == 0) {
      buf[sc] = a;
      buf[n_sc + sc] = b;
      buf[2 * n_sc + sc] = c0;
      buf[3 * n_sc + sc] = c1;
    }
  }
}

}  // namespace

int solve_grid_size(fvgb_mesh_s* m) {
  int a = 0, b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, (const void*)k_cg<float>, kCgThreads, 0) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, (const void*)k_cg<double>, kCgThreads, 0) != cudaSuccess)
    return 0;
  const int per_sm = a < b ? a : b;
  if (per_sm < 1) return 0;
  return (per_sm < kCgBlocksPerSm ? per_sm : kCgBlocksPerSm) * m->num_sms;
}

cudaError_t launch_part_sumsq(fvgb_mesh_s* m, const double* v, double* out, cudaStream_t s) {
  const PartsDev& pd = m->parts;
  k_part_sumsq_partial<<<m->solve_grid, kCgThreads, 0, s>>>(v, pd.blk_sc, pd.sc_begin, pd.buf);
  k_part_sumsq_final<<<1, kCgThreads, 0, s>>>(pd.buf, pd.part_sc, pd.n_part, out);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_part_dots(fvgb_mesh_s* m, const double* r0, const double* r1, double* out, cudaStream_t s) {
  const PartsDev& pd = m->parts;
  k_part_dots_partial<<<m->solve_grid, kCgThreads, 0, s>>>(r0, r1, pd.blk_sc, pd.sc_begin, pd.n_sc, pd.buf);
  for (int k = 0; k < 4; ++k)
    k_part_sumsq_final<<<1, kCgThreads, 0, s>>>(pd.buf + k * pd.n_sc, pd.part_sc, pd.n_part, out + k * pd.n_part);
  count_launch(5);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg(fvgb_mesh_s* m, int bcset, const double* r, double inner_rtol, int maxit,
                      cudaStream_t s) {
  GeoDev<T>& g = geo_of<T>(m);
  Work<T>& w = work_of<T>(m);
  SolveArgs<T> a;
  a.N = m->topo.N;
  a.at_nbr = g.bc[bcset].at_nbr; a.at_scoef = g.bc[bcset].at_scoef; a.at_isd = g.bc[bcset].at_isd;
  a.r_in = r;
  a.cx = w.cg_x; a.cr = w.cg_r; a.cp = w.cg_p; a.cq = w.cg_q;
  const PartsDev& pd = m->parts;
  a.n_part = pd.n_part; a.n_sc = pd.n_sc;
  a.blk_sc = pd.blk_sc; a.sc_begin = pd.sc_begin; a.sc_part = pd.sc_part;
  a.part_sc = pd.part_sc; a.active = pd.active; a.buf = pd.buf;
  a.bar = m->barrier;
  a.inner_tol2 = inner_rtol * inner_rtol;
  a.maxit_inner = maxit;
  a.out_inner = pd.out_inner;
  a.out_status = m->d_cg_info;
  a.skip_block = m->test_skip_block;
  a.barrier_ns = m->test_barrier_ns > 0 ? m->test_barrier_ns : kBarrierTimeoutNs;
  cudaError_t e = cudaMemsetAsync(m->barrier, 0, sizeof(Barrier), s);
  if (e != cudaSuccess) return e;
  void* args[] = {&a};
  count_launch();
  return cudaLaunchCooperativeKernel((const void*)k_cg<T>, dim3(m->solve_grid), dim3(kCgThreads),
                                     args, 0, s);
}

template cudaError_t launch_cg<double>(fvgb_mesh_s*, int, const double*, double, int, cudaStream_t);
template cudaError_t launch_cg<float>(fvgb_mesh_s*, int, const double*, double, int, cudaStream_t);

}  // namespace fvgb
