// Finite-volume kernels of the hot path (Section 2.1 of arXiv 2203.00925):
// least-squares cell gradient (Algorithm "grad"), least-squares vertex values
// (Algorithm "ls"), face fluxes (eq. 4, eq. 15 with psi = 0, eq. "diamond"), the
// face-to-cell gather with the explicit update (eq. 4, eq. 6), and the same face
// operator in the integrated Poisson form (eq. 7 / eq. "laplace").
//
// Every kernel is a gather: each output element is written by one thread that sums
// its inputs in a fixed order, so results are bitwise reproducible run to run (no
// floating-point atomics).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.h"

namespace fvgb {
namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(int64_t n, int threads = kThreads) {
  return (unsigned)((n + threads - 1) / threads);
}

// Grid of a tunable kernel: threads x items per thread cover n elements (grid-stride).
inline unsigned shape_grid(const fvgb_mesh_s* m, int k, int64_t n) {
  const int64_t per_block = (int64_t)m->tune[k].threads * m->tune[k].ipt;
  const int64_t g = (n + per_block - 1) / per_block;
  return (unsigned)(g > 0 ? g : 1);
}

// Difference of two centre coordinates. FP32 keeps each coordinate as a (high, low)
// pair of floats so that the difference of nearby centres keeps FP32 relative accuracy.
__device__ __forceinline__ double cdiff(const double* a, const double*, int64_t ia,
                                        const double* b, const double*, int64_t ib) {
  return a[ia] - b[ib];
}
__device__ __forceinline__ float cdiff(const float* a, const float* alo, int64_t ia,
                                       const float* b, const float* blo, int64_t ib) {
  return (a[ia] - b[ib]) + (alo[ia] - blo[ib]);
}

// Explicitly rounded operations: the face flux is written with them so that its rounding
// sequence (which products are fused) is fixed by the source, not by how the compiler
// schedules a particular instantiation; every launch shape then gives the same bits.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// ---- Algorithm "grad": grad u_i = M_i^{-1} sum_j d_ij (u_j - u_i) ------------------------
// The neighbour loop reads, per neighbour j, one packed 32-byte record (one memory sector)
// holding u_j and the centre of j, written by k_grad_pack for this call:
//   FP64: {u, x, y, z};  FP32: {u, x_hi, y_hi, z_hi, x_lo, y_lo, z_lo, 0}
// (FP32 keeps each coordinate as a high + low float pair so that differences of nearby
// centres keep FP32 relative accuracy). Unused components (2D) are 0.
template <int D>
__global__ void __launch_bounds__(1024)
k_grad_pack(int64_t N, const double* __restrict__ cen, const double* __restrict__,
            const double* __restrict__ u, double* __restrict__ rec) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double2* o = reinterpret_cast<double2*>(rec) + 2 * i;
    o[0] = make_double2(u[i], cen[i]);
    o[1] = make_double2(cen[N + i], D == 3 ? cen[2 * N + i] : 0.0);
  }
}
template <int D>
__global__ void __launch_bounds__(1024)
k_grad_pack(int64_t N, const float* __restrict__ cen, const float* __restrict__ lo,
            const float* __restrict__ u, float* __restrict__ rec) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    float4* o = reinterpret_cast<float4*>(rec) + 2 * i;
    o[0] = make_float4(u[i], cen[i], cen[N + i], D == 3 ? cen[2 * N + i] : 0.0f);
    o[1] = make_float4(lo[i], lo[N + i], D == 3 ? lo[2 * N + i] : 0.0f, 0.0f);
  }
}

// A neighbour's record, and its contribution d_ij (u_j - u_i) to J (the centre
// difference from high and low parts in FP32).
__device__ __forceinline__ void grad_load(const double* rec, int64_t j, double2& a, double2& b) {
  const double2* r = reinterpret_cast<const double2*>(rec) + 2 * j;
  a = __ldg(r);
  b = __ldg(r + 1);
}
__device__ __forceinline__ void grad_load(const float* rec, int64_t j, float4& a, float4& b) {
  const float4* r = reinterpret_cast<const float4*>(rec) + 2 * j;
  a = __ldg(r);
  b = __ldg(r + 1);
}
template <int D>
__device__ __forceinline__ void grad_acc(const double2& a, const double2& b, const double2& ia,
                                         const double2& ib, double* J) {
  const double du = a.x - ia.x;
  J[0] += (a.y - ia.y) * du;
  J[1] += (b.x - ib.x) * du;
  if (D == 3) J[2] += (b.y - ib.y) * du;
}
template <int D>
__device__ __forceinline__ void grad_acc(const float4& a, const float4& b, const float4& ia,
                                         const float4& ib, float* J) {
  const float du = a.x - ia.x;
  J[0] += ((a.y - ia.y) + (b.x - ib.x)) * du;
  J[1] += ((a.z - ia.z) + (b.y - ib.y)) * du;
  if (D == 3) J[2] += ((a.w - ia.w) + (b.z - ib.z)) * du;
}

template <typename T> struct GradVec;
template <> struct GradVec<double> { using type = double2; };
template <> struct GradVec<float> { using type = float4; };

template <typename T, int D>
__global__ void __launch_bounds__(1024)
k_gradient(int64_t N, int64_t F, int64_t Fi, const int64_t* __restrict__ sptr,
           const int32_t* __restrict__ sidx, const T* __restrict__ rec,
           const T* __restrict__ cen, const T* __restrict__ cen_lo, const T* __restrict__ xf,
           const T* __restrict__ xf_lo, const T* __restrict__ u, const T* __restrict__ minv,
           const int32_t* __restrict__ gptr, const int32_t* __restrict__ gface,
           const T* __restrict__ bval, T* __restrict__ grad) {
  using Vec = typename GradVec<T>::type;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = i >> 5;
    const int lane = (int)(i & 31);
    const int64_t b0 = sptr[sl];
    const int width = (int)((sptr[sl + 1] - b0) >> 5);   // every row of a slice has it
    const int32_t* col = sidx + b0 + lane;
    Vec ia, ib;
    grad_load(rec, i, ia, ib);
    T J[3] = {T(0), T(0), T(0)};
    int c = 0;
    for (; c + 4 <= width; c += 4) {      // four independent gathers in flight
      const int32_t j0 = __ldg(col + 32 * c), j1 = __ldg(col + 32 * (c + 1)),
                    j2 = __ldg(col + 32 * (c + 2)), j3 = __ldg(col + 32 * (c + 3));
      Vec a0, b0v, a1, b1v, a2, b2v, a3, b3v;
      grad_load(rec, j0, a0, b0v);
      grad_load(rec, j1, a1, b1v);
      grad_load(rec, j2, a2, b2v);
      grad_load(rec, j3, a3, b3v);
      grad_acc<D>(a0, b0v, ia, ib, J);
      grad_acc<D>(a1, b1v, ia, ib, J);
      grad_acc<D>(a2, b2v, ia, ib, J);
      grad_acc<D>(a3, b3v, ia, ib, J);
    }
    for (; c < width; ++c) {
      const int32_t j = __ldg(col + 32 * c);
      Vec a, b;
      grad_load(rec, j, a, b);
      grad_acc<D>(a, b, ia, ib, J);
    }
    const T ui = u[i];
    for (int32_t t = gptr[i]; t < gptr[i + 1]; ++t) {
      const int32_t f = gface[t];
      const T du = bval[f - Fi] - ui;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const T dx = cdiff(xf + a * F, xf_lo ? xf_lo + a * F : nullptr, f, cen + a * N,
                           cen_lo ? cen_lo + a * N : nullptr, i);
        J[a] += dx * du;
      }
    }
    if constexpr (D == 3) {
      const T m0 = minv[i], m1 = minv[N + i], m2 = minv[2 * N + i], m3 = minv[3 * N + i],
              m4 = minv[4 * N + i], m5 = minv[5 * N + i];
      grad[i] = m0 * J[0] + m1 * J[1] + m2 * J[2];
      grad[N + i] = m1 * J[0] + m3 * J[1] + m4 * J[2];
      grad[2 * N + i] = m2 * J[0] + m4 * J[1] + m5 * J[2];
    } else {
      const T m0 = minv[i], m1 = minv[N + i], m2 = minv[2 * N + i];
      grad[i] = m0 * J[0] + m1 * J[1];
      grad[N + i] = m1 * J[0] + m2 * J[1];
    }
  }
}

// FP32, 3D, shared-memory form of k_gradient: one block per tile of kGradTile consecutive
// cells. The block first stages its tile's halo list (own cells, then their other node
// neighbours) as 16-byte records {u, x - o, y - o, z - o} with coordinates relative to the
// tile's first centre o (high + low parts combined there, so the small differences keep
// FP32 accuracy); each neighbour entry is then one shared-memory read at its int16 local
// position instead of a 32-byte gather from L1/L2. Same sum order as k_gradient.
__global__ void __launch_bounds__(kGradTile)
k_gradient_tiled(int64_t N, int64_t F, int64_t Fi, const int64_t* __restrict__ sptr,
                 const int16_t* __restrict__ lidx, const int32_t* __restrict__ tptr,
                 const int32_t* __restrict__ tidx, const float* __restrict__ rec,
                 const float* __restrict__ cen, const float* __restrict__ cen_lo, const float* __restrict__ xf,
                 const float* __restrict__ xf_lo, const float* __restrict__ minv,
                 const int32_t* __restrict__ gptr, const int32_t* __restrict__ gface,
                 const float* __restrict__ bval, float* __restrict__ grad) {
  extern __shared__ float4 hrec[];
  const int64_t tile = blockIdx.x;
  const int64_t r0 = tile * kGradTile;
  const int32_t h0 = tptr[tile], nh = tptr[tile + 1] - h0;
  const float4* R = reinterpret_cast<const float4*>(rec);
  const float4 oa = __ldg(R + 2 * r0), ob = __ldg(R + 2 * r0 + 1);   // origin: the first own centre
  for (int k = threadIdx.x; k < nh; k += blockDim.x) {
    const int32_t j = __ldg(tidx + h0 + k);
    const float4 a = __ldg(R + 2 * (int64_t)j), b = __ldg(R + 2 * (int64_t)j + 1);
    hrec[k] = make_float4(a.x, (a.y - oa.y) + (b.x - ob.x), (a.z - oa.z) + (b.y - ob.y), (a.w - oa.w) + (b.z - ob.z));
  }
  __syncthreads();
  const int64_t i = r0 + threadIdx.x;
  if (i >= N) return;
  const int64_t sl = i >> 5;
  const int lane = (int)(i & 31);
  const int64_t b0 = sptr[sl];
  const int width = (int)((sptr[sl + 1] - b0) >> 5);
  const int16_t* col = lidx + b0 + lane;
  const float4 me = hrec[threadIdx.x];
  float J[3] = {0.0f, 0.0f, 0.0f};
  int c = 0;
  for (; c + 4 <= width; c += 4) {
    const float4 n0 = hrec[__ldg(col + 32 * c)], n1 = hrec[__ldg(col + 32 * (c + 1))],
                 n2 = hrec[__ldg(col + 32 * (c + 2))], n3 = hrec[__ldg(col + 32 * (c + 3))];
    const float4 nn[4] = {n0, n1, n2, n3};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float du = nn[q].x - me.x;
      J[0] += (nn[q].y - me.y) * du;
      J[1] += (nn[q].z - me.z) * du;
      J[2] += (nn[q].w - me.w) * du;
    }
  }
  for (; c < width; ++c) {
    const float4 nq = hrec[__ldg(col + 32 * c)];
    const float du = nq.x - me.x;
    J[0] += (nq.y - me.y) * du;
    J[1] += (nq.z - me.z) * du;
    J[2] += (nq.w - me.w) * du;
  }
  const float ui = me.x;
  for (int32_t t = gptr[i]; t < gptr[i + 1]; ++t) {
    const int32_t f = gface[t];
    const float du = bval[f - Fi] - ui;
#pragma unroll
    for (int a = 0; a < 3; ++a) J[a] += cdiff(xf + a * F, xf_lo + a * F, f, cen + a * N, cen_lo + a * N, i) * du;
  }
  const float m0 = minv[i], m1 = minv[N + i], m2 = minv[2 * N + i], m3 = minv[3 * N + i], m4 = minv[4 * N + i],
              m5 = minv[5 * N + i];
  grad[i] = m0 * J[0] + m1 * J[1] + m2 * J[2];
  grad[N + i] = m1 * J[0] + m3 * J[1] + m4 * J[2];
  grad[2 * N + i] = m2 * J[0] + m4 * J[1] + m5 * J[2];
}

// ---- multiplicity-weighted least-squares gradient (vertex-factorised variant) ---------------
// grad u_i = Mv_i^{-1} J_i, J_i = sum over the vertices A of T_i, over the cells c around A,
// of (x_c - x_i)(u_c - u_i), plus each Dirichlet ghost point once per shared vertex. Per
// vertex, with y_c = x_c - x_A and a reference value u0 (the first cell around A):
//   S2 = sum (u_c - u0), S3 = sum y_c (u_c - u0)   (pass 1, over the vertex's star),
//   S1 = sum y_c, n = #cells                       (geometry, uploaded),
// and per cell, with y = x_i - x_A, delta = u_i - u0 (pass 2):
//   J_i += S3 - delta S1 - y S2 + n y delta.
// The offsets x_A and u0 keep every term of the size of the differences it stands for.
__device__ __forceinline__ void vdiff(const double2& a, const double2& b, const double* xa, double* y) {
  y[0] = a.y - xa[0]; y[1] = b.x - xa[1]; y[2] = b.y - xa[2];
}
__device__ __forceinline__ void vdiff(const float4& a, const float4& b, const float* xa, float* y) {
  y[0] = (a.y - xa[0]) + (b.x - xa[3]); y[1] = (a.z - xa[1]) + (b.y - xa[4]); y[2] = (a.w - xa[2]) + (b.z - xa[5]);
}

template <typename T, int D>
__global__ void __launch_bounds__(256)
k_vgrad_vertex(int64_t V, const int64_t* __restrict__ sptr, const int32_t* __restrict__ sidx,
               const int32_t* __restrict__ vcount, const T* __restrict__ rec, const T* __restrict__ xv,
               const T* __restrict__ xv_lo, T* __restrict__ vsum) {
  using Vec = typename GradVec<T>::type;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = v >> 5;
    const int lane = (int)(v & 31);
    const int32_t* col = sidx + sptr[sl] + lane;
    const int n = vcount[v];
    T xa[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int a = 0; a < D; ++a) {
      xa[a] = xv[a * V + v];
      if (xv_lo) xa[3 + a] = xv_lo[a * V + v];
    }
    Vec a0, b0;
    grad_load(rec, __ldg(col), a0, b0);
    const T u0 = a0.x;
    T s2 = T(0), s3[3] = {T(0), T(0), T(0)};
    for (int k = 0; k < n; ++k) {
      Vec a, b;
      grad_load(rec, __ldg(col + 32 * k), a, b);
      T y[3];
      vdiff(a, b, xa, y);
      const T du = a.x - u0;
      s2 += du;
#pragma unroll
      for (int c = 0; c < D; ++c) s3[c] += y[c] * du;
    }
    vsum[v] = u0;
    vsum[V + v] = s2;
#pragma unroll
    for (int c = 0; c < D; ++c) vsum[(2 + c) * V + v] = s3[c];
  }
}

template <typename T, int D>
__global__ void __launch_bounds__(256)
k_vgrad_cell(int64_t N, int64_t V, int64_t F, int64_t Fi, const int32_t* __restrict__ cverts,
             const T* __restrict__ rec, const T* __restrict__ xv, const T* __restrict__ xv_lo,
             const int32_t* __restrict__ vcount, const T* __restrict__ vs1, const T* __restrict__ vsum,
             const T* __restrict__ minv, const int32_t* __restrict__ gptr,
             const int32_t* __restrict__ gface, const int32_t* __restrict__ gmult,
             const T* __restrict__ cen, const T* __restrict__ cen_lo, const T* __restrict__ xf,
             const T* __restrict__ xf_lo, const T* __restrict__ bval, T* __restrict__ grad) {
  using Vec = typename GradVec<T>::type;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    Vec ia, ib;
    grad_load(rec, i, ia, ib);
    const T ui = ia.x;
    T J[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int k = 0; k <= D; ++k) {
      const int32_t A = cverts[i * (D + 1) + k];
      T xa[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int a = 0; a < D; ++a) {
        xa[a] = xv[a * V + A];
        if (xv_lo) xa[3 + a] = xv_lo[a * V + A];
      }
      T y[3];
      vdiff(ia, ib, xa, y);
      const T n = (T)vcount[A];
      const T delta = ui - vsum[A];
      const T s2 = vsum[V + A];
#pragma unroll
      for (int a = 0; a < D; ++a)
        J[a] += vsum[(2 + a) * V + A] - delta * vs1[a * V + A] - y[a] * s2 + n * y[a] * delta;
    }
    for (int32_t t = gptr[i]; t < gptr[i + 1]; ++t) {
      const int32_t f = gface[t];
      const T du = (T)gmult[t] * (bval[f - Fi] - ui);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const T dx = cdiff(xf + a * F, xf_lo ? xf_lo + a * F : nullptr, f, cen + a * N,
                           cen_lo ? cen_lo + a * N : nullptr, i);
        J[a] += dx * du;
      }
    }
    if constexpr (D == 3) {
      const T m0 = minv[i], m1 = minv[N + i], m2 = minv[2 * N + i], m3 = minv[3 * N + i],
              m4 = minv[4 * N + i], m5 = minv[5 * N + i];
      grad[i] = m0 * J[0] + m1 * J[1] + m2 * J[2];
      grad[N + i] = m1 * J[0] + m3 * J[1] + m4 * J[2];
      grad[2 * N + i] = m2 * J[0] + m4 * J[1] + m5 * J[2];
    } else {
      const T m0 = minv[i], m1 = minv[N + i], m2 = minv[2 * N + i];
      grad[i] = m0 * J[0] + m1 * J[1];
      grad[N + i] = m1 * J[0] + m2 * J[1];
    }
  }
}

// ---- Algorithm "ls": u_A = sum_c alpha_{A,c} u_c; Dirichlet vertices take g --------------
template <typename T>
__global__ void __launch_bounds__(1024)
k_vertex(int64_t V, const int64_t* __restrict__ sptr, const int32_t* __restrict__ sidx,
         const T* __restrict__ alpha, const T* __restrict__ u, const T* __restrict__ vdir,
         int homog, T* __restrict__ uv) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = v >> 5;
    const int lane = (int)(v & 31);
    const int64_t b0 = sptr[sl];
    const int width = (int)((sptr[sl + 1] - b0) >> 5);   // every row of a slice has it
    const int32_t* col = sidx + b0 + lane;
    const T* wcol = alpha + b0 + lane;
    T s = T(0);
    int c = 0;
    for (; c + 4 <= width; c += 4) {      // four independent gathers in flight
      const int32_t j0 = __ldg(col + 32 * c), j1 = __ldg(col + 32 * (c + 1)),
                    j2 = __ldg(col + 32 * (c + 2)), j3 = __ldg(col + 32 * (c + 3));
      const T w0 = wcol[32 * c], w1 = wcol[32 * (c + 1)], w2 = wcol[32 * (c + 2)],
              w3 = wcol[32 * (c + 3)];
      const T u0 = u[j0], u1 = u[j1], u2 = u[j2], u3 = u[j3];
      s = fma_rn(w0, u0, s);
      s = fma_rn(w1, u1, s);
      s = fma_rn(w2, u2, s);
      s = fma_rn(w3, u3, s);
    }
    for (; c < width; ++c) s = fma_rn(wcol[32 * c], u[__ldg(col + 32 * c)], s);
    const T g = vdir[v];
    if (g == g) s = homog ? T(0) : g;  // Dirichlet vertex (vdir is NaN elsewhere)
    uv[v] = s;
  }
}

// ---- Barth-Jespersen limiter of eq. 15: grad u_i <- psi_i grad u_i ------------------------
// Bounds over u_i, the face neighbours' values and the Dirichlet values of the cell's
// boundary faces; psi_i = min over the cell's faces of min(1, (bound - u_i) / d_f) with
// d_f = grad u_i . (x_f - x_i) (the upper bound where d_f > 0, the lower where d_f < 0).
template <typename T, int D>
__global__ void __launch_bounds__(256)
k_bj_limit(int64_t N, int64_t F, int64_t Fi, const int32_t* __restrict__ cell_face,
           const int32_t* __restrict__ fL, const int32_t* __restrict__ fR,
           const T* __restrict__ u, const T* __restrict__ cen, const T* __restrict__ cen_lo,
           const T* __restrict__ xf, const T* __restrict__ xf_lo,
           const int8_t* __restrict__ bkind, const T* __restrict__ bval, T* __restrict__ grad) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const T ui = u[i];
  T gi[3] = {grad[i], grad[N + i], D == 3 ? grad[2 * N + i] : T(0)};
  T umax = ui, umin = ui;
  int32_t fc[D + 1];
#pragma unroll
  for (int k = 0; k <= D; ++k) {
    const int32_t e = cell_face[k * N + i];
    const int32_t f = e >= 0 ? e : ~e;
    fc[k] = f;
    if (f < Fi) {
      const T uj = u[e >= 0 ? fR[f] : fL[f]];
      umax = fmax(umax, uj);
      umin = fmin(umin, uj);
    } else if (bkind[f - Fi] == FVGB_BC_DIRICHLET) {
      const T g = bval[f - Fi];
      umax = fmax(umax, g);
      umin = fmin(umin, g);
    }
  }
  // psi = min(1, min over faces of (bound - u_i) / d_f). The smallest ratio is tracked as
  // a fraction num / den (both >= 0); in FP64 (costly division) the comparison is by
  // cross-multiplication and the winner is divided once.
  T num = T(1), den = T(1);
#pragma unroll
  for (int k = 0; k <= D; ++k) {
    const int32_t f = fc[k];
    T d = mul_rn(gi[0], cdiff(xf, xf_lo, f, cen, cen_lo, i));
    d = fma_rn(gi[1], cdiff(xf + F, xf_lo ? xf_lo + F : nullptr, f, cen + N, cen_lo ? cen_lo + N : nullptr, i), d);
    if (D == 3)
      d = fma_rn(gi[2], cdiff(xf + 2 * F, xf_lo ? xf_lo + 2 * F : nullptr, f, cen + 2 * N,
                              cen_lo ? cen_lo + 2 * N : nullptr, i), d);
    if (d != T(0)) {
      const T a = d > T(0) ? umax - ui : ui - umin;   // >= 0
      const T b = fabs(d);
      if constexpr (sizeof(T) == 8) {
        if (a * den < num * b) { num = a; den = b; }
      } else {                                           // FP32: products could overflow
        if (a / b < num / den) { num = a; den = b; }
      }
    }
  }
  const T psi = num == T(1) && den == T(1) ? T(1) : num / den;
#pragma unroll
  for (int a = 0; a < D; ++a) grad[a * N + i] = mul_rn(psi, gi[a]);
}

// ---- face flux: F = (V_f . S_f) u_up - D grad u_f . S_f (eq. 4, eq. 15, eq. "diamond") ----
// Each thread takes K faces (block-contiguous, stride blockDim): it issues the streamed
// face data of all K first, then all their gathers, then computes, so that K faces'
// loads are in flight together. The arithmetic of one face does not depend on K.
// With RECON (MUSCL, eq. 15) the upwind cell's value is reconstructed at the face
// centroid with the limited gradient lg: u_c + lg_c . (x_f - x_c); a boundary ghost on
// the upwind side keeps its first-order value.
struct Recon {
  const void* lg = nullptr;      // [d][N] limited gradient
  const void* cen = nullptr;     // [d][N]
  const void* cen_lo = nullptr;  // [d][N] (FP32)
  const void* xf = nullptr;      // [d][F]
  const void* xf_lo = nullptr;   // [d][F] (FP32)
};

template <typename T, int D>
__device__ __forceinline__ T recon_value(const Recon& rc, int64_t N, int64_t F, int64_t f,
                                         int32_t c, T uc) {
  const T* lg = (const T*)rc.lg;
  const T* cen = (const T*)rc.cen;
  const T* clo = (const T*)rc.cen_lo;
  const T* xf = (const T*)rc.xf;
  const T* xlo = (const T*)rc.xf_lo;
  T t = mul_rn(lg[c], cdiff(xf, xlo, f, cen, clo, c));
  t = fma_rn(lg[N + c], cdiff(xf + F, xlo ? xlo + F : nullptr, f, cen + N, clo ? clo + N : nullptr, c), t);
  if (D == 3)
    t = fma_rn(lg[2 * N + c], cdiff(xf + 2 * F, xlo ? xlo + 2 * F : nullptr, f, cen + 2 * N,
                                    clo ? clo + 2 * N : nullptr, c), t);
  return add_rn(uc, t);
}

template <typename T, int D, bool CONV, bool VFIELD, int K, bool RECON = false>
__global__ void __launch_bounds__(1024 / K)
k_face(int64_t F, int64_t Fi, int64_t N, const int32_t* __restrict__ fL,
       const int32_t* __restrict__ fR, const int32_t* __restrict__ fvert,
       const T* __restrict__ S, const T* __restrict__ coef, const T* __restrict__ u,
       const T* __restrict__ uv, const T* __restrict__ vel, T vc0, T vc1, T vc2, T Dcoef,
       const int8_t* __restrict__ bkind, const T* __restrict__ bval, int homog,
       T* __restrict__ flux, Recon rc) {
  constexpr int kInterior = 3;
  const int64_t per_block = (int64_t)blockDim.x * K;
  for (int64_t base = blockIdx.x * per_block + threadIdx.x; base < F;
       base += (int64_t)gridDim.x * per_block) {
    int32_t L[K], R[K], vA[K], vB[K], vC[K];
    int kind[K];
    T s0[K], s1[K], s2[K], c0[K], c1[K], c2[K], gb[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {           // streamed face data (in bounds: clamped)
      const int64_t f = min(base + (int64_t)k * blockDim.x, F - 1);
      L[k] = fL[f];
      if (f < Fi) {
        R[k] = fR[f];
        kind[k] = kInterior;
        gb[k] = T(0);
      } else {
        R[k] = -1;
        kind[k] = bkind[f - Fi];
        gb[k] = homog ? T(0) : bval[f - Fi];
      }
      if (CONV) {
        s0[k] = S[f]; s1[k] = S[F + f];
        s2[k] = D == 3 ? S[2 * F + f] : T(0);
      }
      c0[k] = coef[f]; c1[k] = coef[F + f];
      c2[k] = D == 3 ? coef[2 * F + f] : T(0);
      vA[k] = fvert[f]; vB[k] = fvert[F + f];
      vC[k] = D == 3 ? fvert[2 * F + f] : 0;
    }
    T uL[K], uR[K], ua[K], ub[K], uc[K], vl[K][3], vr[K][3];
    const bool diff = Dcoef != T(0);
#pragma unroll
    for (int k = 0; k < K; ++k) {           // gathers
      uL[k] = u[L[k]];
      uR[k] = R[k] >= 0 ? u[R[k]] : T(0);
      if (CONV && VFIELD) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          vl[k][a] = vel[a * N + L[k]];
          vr[k][a] = R[k] >= 0 ? vel[a * N + R[k]] : vl[k][a];
        }
      }
      const bool need_uv = diff && (kind[k] == kInterior || kind[k] == FVGB_BC_DIRICHLET);
      ua[k] = need_uv ? uv[vA[k]] : T(0);
      ub[k] = need_uv ? uv[vB[k]] : T(0);
      uc[k] = need_uv && D == 3 ? uv[vC[k]] : T(0);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int64_t f = base + (int64_t)k * blockDim.x;
      if (f >= F) break;
      if (kind[k] == FVGB_BC_WALL) { flux[f] = T(0); continue; }
      const T ul = uL[k];
      const T ur = kind[k] == kInterior ? uR[k] : (kind[k] == FVGB_BC_DIRICHLET ? gb[k] : ul);
      T Ff = T(0);
      if (CONV) {
        T vf[3];
        if (VFIELD) {
#pragma unroll
          for (int a = 0; a < D; ++a) vf[a] = mul_rn(T(0.5), add_rn(vl[k][a], vr[k][a]));
        } else {
          vf[0] = vc0; vf[1] = vc1; vf[2] = vc2;
        }
        T vn = fma_rn(vf[1], s1[k], mul_rn(vf[0], s0[k]));
        if (D == 3) vn = fma_rn(vf[2], s2[k], vn);
        T up = vn >= T(0) ? ul : ur;
        if (RECON) {
          if (vn >= T(0)) up = recon_value<T, D>(rc, N, F, f, L[k], ul);
          else if (kind[k] == kInterior) up = recon_value<T, D>(rc, N, F, f, R[k], ur);
        }
        Ff = mul_rn(vn, up);
      }
      if (diff && (kind[k] == kInterior || kind[k] == FVGB_BC_DIRICHLET)) {
        T q = mul_rn(c0[k], sub_rn(ur, ul));
        if constexpr (D == 3) {
          q = fma_rn(c1[k], sub_rn(ua[k], uc[k]), q);
          q = fma_rn(c2[k], sub_rn(ub[k], uc[k]), q);
        } else {
          q = fma_rn(c1[k], sub_rn(ub[k], ua[k]), q);
        }
        Ff = fma_rn(-Dcoef, q, Ff);
      }
      flux[f] = Ff;
    }
  }
}

// ---- gather of the face fluxes of every cell (eq. 4) and what follows from it ---------------
template <typename T, int NV, int MODE>
__global__ void __launch_bounds__(1024)
k_update(int64_t N, const int32_t* __restrict__ cell_face, const T* __restrict__ flux,
         const T* __restrict__ inv_vol, const T* __restrict__ vol, const T* __restrict__ src,
         const T* base, T adt, const T* __restrict__ aux, T* out, T* out2, int* __restrict__ status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    T acc = T(0);  // sum over faces entering i minus faces leaving i
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const int32_t e = cell_face[k * N + i];
      acc += e >= 0 ? -flux[e] : flux[~e];
    }
    if constexpr (MODE == kResidual) {
      const T r = acc * inv_vol[i] + (src ? src[i] : T(0));
      out[i] = r;
      if (!isfinite(r)) atomicOr(status, 1);     // latched for fvgb_sync
    } else if constexpr (MODE == kStep) {
      const T s = src ? src[i] : T(0);
      const T r = acc * inv_vol[i] + s;
      const T v = base[i] + adt * r;
      out[i] = v;
      if (out2) {
        const T w = out2[i] + adt * s;
        out2[i] = w;
        if (!isfinite(w)) atomicOr(status, 1);
      }
      if (!isfinite(v)) atomicOr(status, 1);
    } else if constexpr (MODE == kPoissonApply) {
      out[i] = acc;                       // A x = -mu Lap_h x
    } else if constexpr (MODE == kPoissonResidual) {
      out[i] = aux[i] - acc;              // r = b - A x
    } else {
      out[i] = -vol[i] * (aux ? aux[i] : T(0)) - acc;   // b = -mu f + mu Lap_h(0; g)
    }
  }
}

// ---- streamer cell physics (eq. 10 with v = -mu E, alpha = A exp(-B/|E|)) --------------------
// Plasma spots (Section 4, "Streamer Branching"): the source of the spots averaged over
// the step [t, t + dt], sum_k S_k exp(-|x - c_k|^2 / sigma_k^2) |[t, t + dt] n window_k| / dt,
// in FP64 at the cell centre (FP32 meshes: high + low parts of the centre).
template <typename T, int D>
__device__ __forceinline__ double spot_term(const SpotArgs& sp, const T* __restrict__ cen,
                                            const T* __restrict__ cen_lo, int64_t N, int64_t i) {
  const double t = *sp.t;
  double add = 0.0;
  for (int k = 0; k < sp.n; ++k) {
    const double lo = fmax(t, sp.t_on[k]);
    const double hi = fmin(t + sp.dt, sp.t_off[k]);
    if (!(hi > lo)) continue;
    const double c[3] = {sp.cx[k], sp.cy[k], sp.cz[k]};
    double r2 = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const double x = (double)cen[a * N + i] + (cen_lo ? (double)cen_lo[a * N + i] : 0.0);
      const double d = x - c[a];
      r2 += d * d;
    }
    add += sp.amp[k] * exp(-r2 / sp.s2[k]) * ((hi - lo) / sp.dt);
  }
  return add;
}

template <typename T, int D>
__global__ void __launch_bounds__(kThreads)
k_cell_physics(int64_t N, const T* __restrict__ grad, const T* __restrict__ ne, T mu, T A, T B,
               T* __restrict__ E, T* __restrict__ vel, T* __restrict__ src, const T* __restrict__ cen,
               const T* __restrict__ cen_lo, const SpotArgs sp) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  T e[3], en2 = T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) { e[a] = -grad[a * N + i]; en2 += e[a] * e[a]; }
  const T en = sqrt(en2);
  const T alpha = en > T(0) ? A * exp(-B / en) : T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    vel[a * N + i] = -mu * e[a];
    if (E) E[a * N + i] = e[a];
  }
  T S = alpha * mu * en * ne[i];
  if (sp.n > 0) S += (T)spot_term<T, D>(sp, cen, cen_lo, N, i);
  src[i] = S;
}

__global__ void k_time(double* __restrict__ t, int set, double v) {
  if (threadIdx.x == 0) t[0] = set ? v : t[0] + v;
}

template <typename T>
__global__ void k_poisson_source(int64_t N, const T* __restrict__ ne, const T* __restrict__ ni,
                                 double* __restrict__ f) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  constexpr double kEoverEps0 = 1.602176634e-19 / 8.8541878128e-12;
  f[i] = -kEoverEps0 * ((double)ni[i] - (double)ne[i]);
}

// ---- deterministic FP64 reduction: fixed grid, fixed per-thread order, fixed tree ----------
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

__global__ void __launch_bounds__(256) k_sumsq_partial(const double* __restrict__ x, int64_t n,
                                                       double* __restrict__ part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += x[i] * x[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <typename T>
__global__ void __launch_bounds__(256) k_wsum_partial(const T* __restrict__ u,
                                                      const double* __restrict__ vol, int64_t n,
                                                      double* __restrict__ part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += vol[i] * (double)u[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_sum_final(const double* __restrict__ part, int n,
                                                    double* __restrict__ out) {
  __shared__ double sh[32];
  double s = threadIdx.x < n ? part[threadIdx.x] : 0.0;
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[0] = s;
}

__global__ void k_axpy_d(const double* __restrict__ x, double a, double* __restrict__ y, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

template <typename T>
__global__ void k_add_to_double(const T* __restrict__ x, double* __restrict__ y, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] += (double)x[i];
}

__global__ void k_convert(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}

__global__ void k_convert_back(const float* __restrict__ x, double* __restrict__ y, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = (double)x[i];
}

template <typename E>
__global__ void k_permute(const E* __restrict__ src, E* __restrict__ dst,
                          const int32_t* __restrict__ perm, int64_t n, int ncomp, int to_internal) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t p = perm[i];
  for (int c = 0; c < ncomp; ++c) {
    if (to_internal) dst[c * n + i] = src[c * n + p];
    else dst[c * n + p] = src[c * n + i];
  }
}

__global__ void k_nonfinite(const double* __restrict__ x, int64_t n, int* flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && !isfinite(x[i])) *flag = 1;  // benign race: every writer stores 1
}

}  // namespace

// ---- launchers -------------------------------------------------------------------------------
template <typename T>
cudaError_t launch_gradient(fvgb_mesh_s* m, int bcset, const T* u, T* grad, cudaStream_t s) {
  const TopoDev& t = m->topo;
  GeoDev<T>& g = geo_of<T>(m);
  const BCDev<T>& b = g.bc[bcset];
  T* rec = work_of<T>(m).grec;
  const unsigned gp = grid_for(t.N);
  const unsigned gg = shape_grid(m, kTuneGrad, t.N);
  const int tg = m->tune[kTuneGrad].threads;
  if (t.dim == 3) {
    k_grad_pack<3><<<gp, kThreads, 0, s>>>(t.N, g.cen, g.cen_lo, u, rec);
    if constexpr (sizeof(T) == 4) {
      if (t.tile_max > 0) {      // FP32: the shared-memory form
        const int64_t ntile = (t.N + kGradTile - 1) / kGradTile;
        k_gradient_tiled<<<(unsigned)ntile, kGradTile, t.tile_max * sizeof(float4), s>>>(
            t.N, t.F, t.Fi, t.nsell.ptr, t.tile_lidx, t.tile_ptr, t.tile_idx, (const float*)rec,
            (const float*)g.cen, (const float*)g.cen_lo, (const float*)g.xf, (const float*)g.xf_lo,
            (const float*)b.minv, b.gptr, b.gface, (const float*)b.bval, (float*)grad);
        count_launch(2);
        return cudaGetLastError();
      }
    }
    k_gradient<T, 3><<<gg, tg, 0, s>>>(t.N, t.F, t.Fi, t.nsell.ptr, t.nsell.idx, rec, g.cen,
        g.cen_lo, g.xf, g.xf_lo, u, b.minv, b.gptr, b.gface, b.bval, grad);
  } else {
    k_grad_pack<2><<<gp, kThreads, 0, s>>>(t.N, g.cen, g.cen_lo, u, rec);
    k_gradient<T, 2><<<gg, tg, 0, s>>>(t.N, t.F, t.Fi, t.nsell.ptr, t.nsell.idx, rec, g.cen,
        g.cen_lo, g.xf, g.xf_lo, u, b.minv, b.gptr, b.gface, b.bval, grad);
  }
  count_launch(2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gradient_vertex(fvgb_mesh_s* m, int bcset, const T* u, T* grad, cudaStream_t s) {
  const TopoDev& t = m->topo;
  GeoDev<T>& g = geo_of<T>(m);
  const BCDev<T>& b = g.bc[bcset];
  Work<T>& w = work_of<T>(m);
  const unsigned gv = grid_for(t.V), gc = grid_for(t.N);
  if (t.dim == 3) {
    k_grad_pack<3><<<grid_for(t.N), kThreads, 0, s>>>(t.N, g.cen, g.cen_lo, u, w.grec);
    k_vgrad_vertex<T, 3><<<gv, kThreads, 0, s>>>(t.V, t.vsell.ptr, t.vsell.idx, t.vcount, w.grec, g.xv,
                                                 g.xv_lo, w.vsum);
    k_vgrad_cell<T, 3><<<gc, kThreads, 0, s>>>(t.N, t.V, t.F, t.Fi, t.cverts, w.grec, g.xv, g.xv_lo, t.vcount,
        g.vs1, w.vsum, b.minv_v, b.gptr, b.gface, b.gmult, g.cen, g.cen_lo, g.xf, g.xf_lo, b.bval, grad);
  } else {
    k_grad_pack<2><<<grid_for(t.N), kThreads, 0, s>>>(t.N, g.cen, g.cen_lo, u, w.grec);
    k_vgrad_vertex<T, 2><<<gv, kThreads, 0, s>>>(t.V, t.vsell.ptr, t.vsell.idx, t.vcount, w.grec, g.xv,
                                                 g.xv_lo, w.vsum);
    k_vgrad_cell<T, 2><<<gc, kThreads, 0, s>>>(t.N, t.V, t.F, t.Fi, t.cverts, w.grec, g.xv, g.xv_lo, t.vcount,
        g.vs1, w.vsum, b.minv_v, b.gptr, b.gface, b.gmult, g.cen, g.cen_lo, g.xf, g.xf_lo, b.bval, grad);
  }
  count_launch(3);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_vertex(fvgb_mesh_s* m, int bcset, const T* u, T* uv, bool homog, cudaStream_t s) {
  const TopoDev& t = m->topo;
  GeoDev<T>& g = geo_of<T>(m);
  k_vertex<T><<<shape_grid(m, kTuneVertex, t.V), m->tune[kTuneVertex].threads, 0, s>>>(t.V, t.vsell.ptr, t.vsell.idx, g.valpha, u,
                                                  g.bc[bcset].vdir, homog ? 1 : 0, uv);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bj_limit(fvgb_mesh_s* m, int bcset, const T* u, T* grad, cudaStream_t s) {
  const TopoDev& t = m->topo;
  GeoDev<T>& g = geo_of<T>(m);
  const BCDev<T>& b = g.bc[bcset];
  if (t.dim == 3)
    k_bj_limit<T, 3><<<grid_for(t.N), kThreads, 0, s>>>(t.N, t.F, t.Fi, t.cell_face, t.fL, t.fR, u,
        g.cen, g.cen_lo, g.xf, g.xf_lo, b.bkind, b.bval, grad);
  else
    k_bj_limit<T, 2><<<grid_for(t.N), kThreads, 0, s>>>(t.N, t.F, t.Fi, t.cell_face, t.fL, t.fR, u,
        g.cen, g.cen_lo, g.xf, g.xf_lo, b.bkind, b.bval, grad);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_face(fvgb_mesh_s* m, int bcset, const T* u, const T* uv, const T* vel,
                        const double* vc, bool conv, double D, bool homog, T* flux, cudaStream_t s,
                        const T* lgrad) {
  const TopoDev& t = m->topo;
  GeoDev<T>& g = geo_of<T>(m);
  const BCDev<T>& b = g.bc[bcset];
  Recon rc;
  if (lgrad) rc = Recon{lgrad, g.cen, g.cen_lo, g.xf, g.xf_lo};
  const T v0 = vc ? (T)vc[0] : T(0), v1 = vc ? (T)vc[1] : T(0), v2 = vc ? (T)vc[2] : T(0);
  // K faces per thread (FP64 face fluxes of an FP32 mesh, the Poisson residual, are bound
  // by the FP64 pipe and take K = 1); blocks of at most 1024 / K threads (the kernel's launch bound)
  auto face_grid = [&](int K, int& tb) {
    tb = std::min(m->tune[kTuneFace].threads, 1024 / K);
    return (unsigned)std::max<int64_t>(1, (t.F + (int64_t)tb * K - 1) / ((int64_t)tb * K));
  };
  const int ipt = sizeof(T) == 8 && is_fp32(m) ? 1 : m->tune[kTuneFace].ipt;
  int tb = 0;
#define FVGB_FACE_K(DD, CV, VF, KK)                                                         \
  do {                                                                                      \
    const unsigned gr_ = face_grid(KK, tb);                                                 \
    k_face<T, DD, CV, VF, KK><<<gr_, tb, 0, s>>>(t.F, t.Fi, t.N, t.fL, t.fR, t.fvert, g.S,  \
                                                 g.coef, u, uv, vel, v0, v1, v2, (T)D,      \
                                                 b.bkind, b.bval, homog ? 1 : 0, flux, rc); \
  } while (0)
#define FVGB_FACE_RECON(DD, VF)                                                            \
  do {                                                                                     \
    const unsigned gr_ = face_grid(1, tb);                                                 \
    k_face<T, DD, true, VF, 1, true><<<gr_, tb, 0, s>>>(t.F, t.Fi, t.N, t.fL, t.fR, t.fvert, \
        g.S, g.coef, u, uv, vel, v0, v1, v2, (T)D, b.bkind, b.bval, homog ? 1 : 0, flux, rc); \
  } while (0)
#define FVGB_FACE(DD, CV, VF)                                          \
  do {                                                                 \
    if (ipt >= 4) FVGB_FACE_K(DD, CV, VF, 4);                          \
    else if (ipt == 2) FVGB_FACE_K(DD, CV, VF, 2);                     \
    else FVGB_FACE_K(DD, CV, VF, 1);                                   \
  } while (0)
  if (lgrad && conv) {
    if (t.dim == 3) {
      if (vel) FVGB_FACE_RECON(3, true);
      else FVGB_FACE_RECON(3, false);
    } else {
      if (vel) FVGB_FACE_RECON(2, true);
      else FVGB_FACE_RECON(2, false);
    }
  } else if (t.dim == 3) {
    if (!conv) FVGB_FACE(3, false, false);
    else if (vel) FVGB_FACE(3, true, true);
    else FVGB_FACE(3, true, false);
  } else {
    if (!conv) FVGB_FACE(2, false, false);
    else if (vel) FVGB_FACE(2, true, true);
    else FVGB_FACE(2, true, false);
  }
#undef FVGB_FACE
#undef FVGB_FACE_K
#undef FVGB_FACE_RECON
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update(fvgb_mesh_s* m, int mode, const T* flux, const T* src, const T* base,
                          double adt, const T* aux, T* out, T* out2, cudaStream_t s) {
  const TopoDev& t = m->topo;
  GeoDev<T>& g = geo_of<T>(m);
  const unsigned gr = shape_grid(m, kTuneUpdate, t.N);
  const int tb = m->tune[kTuneUpdate].threads;
#define FVGB_UPD(NV, MD)                                                                 \
  k_update<T, NV, MD><<<gr, tb, 0, s>>>(t.N, t.cell_face, flux, g.inv_vol, g.vol, src, \
                                              base, (T)adt, aux, out, out2, m->d_status)
#define FVGB_UPD_MODES(NV)                                       \
  switch (mode) {                                                \
    case kResidual: FVGB_UPD(NV, kResidual); break;              \
    case kStep: FVGB_UPD(NV, kStep); break;                      \
    case kPoissonApply: FVGB_UPD(NV, kPoissonApply); break;      \
    case kPoissonResidual: FVGB_UPD(NV, kPoissonResidual); break; \
    default: FVGB_UPD(NV, kPoissonRhs); break;                   \
  }
  if (t.dim == 3) { FVGB_UPD_MODES(4) } else { FVGB_UPD_MODES(3) }
#undef FVGB_UPD_MODES
#undef FVGB_UPD
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cell_physics(fvgb_mesh_s* m, const T* grad, const T* ne, double mu, double A,
                                double B, T* E, T* vel, T* src, const SpotArgs& sp, cudaStream_t s) {
  const TopoDev& t = m->topo;
  const GeoDev<T>& g = geo_of<T>(m);
  if (t.dim == 3)
    k_cell_physics<T, 3><<<grid_for(t.N), kThreads, 0, s>>>(t.N, grad, ne, (T)mu, (T)A, (T)B, E, vel, src,
                                                            g.cen, g.cen_lo, sp);
  else
    k_cell_physics<T, 2><<<grid_for(t.N), kThreads, 0, s>>>(t.N, grad, ne, (T)mu, (T)A, (T)B, E, vel, src,
                                                            g.cen, g.cen_lo, sp);
  count_launch();
  return cudaGetLastError();
}

SpotArgs spot_args(fvgb_mesh_s* m, const fvgb_streamer_params* p) {
  SpotArgs a;
  a.n = p->n_spot;
  for (int k = 0; k < p->n_spot; ++k) {
    const fvgb_spot& q = p->spots[k];
    a.cx[k] = q.centre[0]; a.cy[k] = q.centre[1]; a.cz[k] = q.centre[2];
    a.amp[k] = q.amplitude;
    a.s2[k] = q.sigma * q.sigma;
    a.t_on[k] = q.t_on;
    a.t_off[k] = q.t_on + q.duration;
  }
  a.dt = p->dt;
  a.t = m->d_time;
  return a;
}

cudaError_t launch_time(fvgb_mesh_s* m, bool set, double v, cudaStream_t s) {
  k_time<<<1, 32, 0, s>>>(m->d_time, set ? 1 : 0, v);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_poisson_source(fvgb_mesh_s* m, const void* ne, const void* ni, bool fp32,
                                  double* f, cudaStream_t s) {
  const int64_t N = m->topo.N;
  if (fp32)
    k_poisson_source<float><<<grid_for(N), kThreads, 0, s>>>(N, (const float*)ne, (const float*)ni, f);
  else
    k_poisson_source<double><<<grid_for(N), kThreads, 0, s>>>(N, (const double*)ne, (const double*)ni, f);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_sumsq(fvgb_mesh_s* m, const double* x, int64_t n, double* out, cudaStream_t s) {
  k_sumsq_partial<<<kRedBlocks, 256, 0, s>>>(x, n, m->d_scal + 8);
  k_sum_final<<<1, 1024, 0, s>>>(m->d_scal + 8, kRedBlocks, out);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_integral(fvgb_mesh_s* m, const void* u, bool fp32, double* out, cudaStream_t s) {
  const int64_t n = m->topo.N;
  if (fp32) k_wsum_partial<float><<<kRedBlocks, 256, 0, s>>>((const float*)u, m->g64.vol, n, m->d_scal + 8);
  else k_wsum_partial<double><<<kRedBlocks, 256, 0, s>>>((const double*)u, m->g64.vol, n, m->d_scal + 8);
  k_sum_final<<<1, 1024, 0, s>>>(m->d_scal + 8, kRedBlocks, out);
  count_launch(2);
  return cudaGetLastError();
}

// Charge history of the warm start: q = n_i - n_e; with one earlier step dq = q - q_prev,
// with two d2q = dq - dq_prev; then q_prev = q, dq_prev = dq (dq holds both).
template <typename T>
__global__ void k_charge_hist(int64_t N, const T* __restrict__ ne, const T* __restrict__ ni, int hist,
                              double* __restrict__ q_prev, double* __restrict__ dq, double* __restrict__ d2q) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double q = (double)ni[i] - (double)ne[i];
    if (hist >= 1) {
      const double d = q - q_prev[i];
      if (hist >= 2) d2q[i] = d - dq[i];
      dq[i] = d;
    }
    q_prev[i] = q;
  }
}

cudaError_t launch_charge_hist(fvgb_mesh_s* m, const void* ne, const void* ni, bool fp32, int hist,
                               double* q_prev, double* dq, double* d2q, cudaStream_t s) {
  const int64_t N = m->topo.N;
  if (fp32) k_charge_hist<float><<<grid_for(N), kThreads, 0, s>>>(N, (const float*)ne, (const float*)ni, hist, q_prev, dq, d2q);
  else k_charge_hist<double><<<grid_for(N), kThreads, 0, s>>>(N, (const double*)ne, (const double*)ni, hist, q_prev, dq, d2q);
  count_launch();
  return cudaGetLastError();
}

// phi_old2 <- phi_old, phi_old <- phi and, when extrapolating, phi <- 2 phi - phi_old
// (linear in time)
__global__ void k_extrapolate(int64_t N, int extrap, double* __restrict__ phi, double* __restrict__ phi_old,
                              double* __restrict__ phi_old2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double o = phi[i];
    const double po = phi_old[i];
    if (extrap) phi[i] = 2.0 * o - po;
    phi_old2[i] = po;
    phi_old[i] = o;
  }
}

cudaError_t launch_extrapolate(fvgb_mesh_s* m, bool extrap, double* phi, double* phi_old, double* phi_old2,
                               cudaStream_t s) {
  const int64_t N = m->topo.N;
  k_extrapolate<<<grid_for(N), kThreads, 0, s>>>(N, extrap ? 1 : 0, phi, phi_old, phi_old2);
  count_launch();
  return cudaGetLastError();
}

// Training pair of the last streamer step from the warm-start history: which = 0 gives
// (dq, phi^n, phi^{n+1} - phi^n), which = 1 gives (d2q, phi^n, phi^{n+1} - 2 phi^n + phi^{n-1}).
__global__ void k_history_pair(int64_t N, int which, const double* __restrict__ phi,
                               const double* __restrict__ phi_old, const double* __restrict__ phi_old2,
                               const double* __restrict__ dq, const double* __restrict__ d2q,
                               double* __restrict__ q_out, double* __restrict__ p_out, double* __restrict__ d_out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double po = phi_old[i];
    q_out[i] = which ? d2q[i] : dq[i];
    p_out[i] = po;
    d_out[i] = which ? (phi[i] - po) - (po - phi_old2[i]) : phi[i] - po;
  }
}

cudaError_t launch_history_pair(fvgb_mesh_s* m, int which, const double* phi, double* q_out, double* p_out,
                                double* d_out, cudaStream_t s) {
  const int64_t N = m->topo.N;
  k_history_pair<<<grid_for(N), kThreads, 0, s>>>(N, which, phi, m->phi_old, m->phi_old2, m->dq, m->d2q,
                                                  q_out, p_out, d_out);
  count_launch();
  return cudaGetLastError();
}

// per part p (block p): phi = saved + s pred. dots: per part <r0, A pred>, ||A pred||^2,
// ||r0||^2, ||r1||^2 (r1 the residual of saved + pred). s = 1 where ||r1|| < ||r0||, else
// s = <r0, A pred> / ||A pred||^2, the scale that minimises the FP64 residual
// ||r0 - s A pred|| along the prediction; s = 0 where that is undefined. used[p] = (s > 0).
// The start's residual follows from the two residuals already formed (A is linear):
// r = b - A (saved + s pred) = r0 + s (r1 - r0), written over r0.
__global__ void k_scale_start(const double* __restrict__ dots, int P, const int32_t* __restrict__ part_sc,
                              const int64_t* __restrict__ sc_begin, const double* __restrict__ saved,
                              const double* __restrict__ pred, double* __restrict__ phi, int* __restrict__ used,
                              double* __restrict__ scale, double* __restrict__ r0, const double* __restrict__ r1) {
  const int p = blockIdx.y;              // gridDim.x blocks share each part's cell range
  const double num = dots[p], den = dots[P + p], n0 = dots[2 * P + p], n1 = dots[3 * P + p];
  double sc = n1 < n0 ? 1.0 : (den > 0.0 ? num / den : 0.0);
  if (!isfinite(sc)) sc = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    used[p] = sc > 0.0 ? 1 : 0;
    scale[p] = sc;
  }
  const int64_t lo = sc_begin[part_sc[p]], hi = sc_begin[part_sc[p + 1]];
  for (int64_t i = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < hi; i += (int64_t)gridDim.x * blockDim.x) {
    phi[i] = saved[i] + sc * pred[i];
    const double a = r0[i];
    r0[i] = a + sc * (r1[i] - a);
  }
}

// blocks per part of the per-part elementwise kernels: about four an SM in all
dim3 part_grid(const fvgb_mesh_s* m) {
  const int P = m->parts.n_part;
  return dim3((unsigned)std::max(1, (4 * m->num_sms + P - 1) / P), (unsigned)P);
}

cudaError_t launch_scale_start(fvgb_mesh_s* m, const double* dots, const double* saved, const double* pred,
                               double* phi, int* used, double* scale, double* r0, const double* r1,
                               cudaStream_t s) {
  k_scale_start<<<part_grid(m), 256, 0, s>>>(dots, m->parts.n_part, m->parts.part_sc, m->parts.sc_begin,
                                             saved, pred, phi, used, scale, r0, r1);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_axpy_d(const double* x, double a, double* y, int64_t n, cudaStream_t s) {
  k_axpy_d<<<grid_for(n), kThreads, 0, s>>>(x, a, y, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_add_to_double(const void* x, bool fp32, double* y, int64_t n, cudaStream_t s) {
  if (fp32) k_add_to_double<float><<<grid_for(n), kThreads, 0, s>>>((const float*)x, y, n);
  else k_add_to_double<double><<<grid_for(n), kThreads, 0, s>>>((const double*)x, y, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_convert(const double* x, float* y, int64_t n, cudaStream_t s) {
  k_convert<<<grid_for(n), kThreads, 0, s>>>(x, y, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_convert_back(const float* x, double* y, int64_t n, cudaStream_t s) {
  k_convert_back<<<grid_for(n), kThreads, 0, s>>>(x, y, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_permute(const void* src, void* dst, const int32_t* perm, int64_t n, int ncomp,
                           int elem_bytes, bool to_internal, cudaStream_t s) {
  if (elem_bytes == 8)
    k_permute<double><<<grid_for(n), kThreads, 0, s>>>((const double*)src, (double*)dst, perm, n,
                                                        ncomp, to_internal ? 1 : 0);
  else
    k_permute<float><<<grid_for(n), kThreads, 0, s>>>((const float*)src, (float*)dst, perm, n,
                                                       ncomp, to_internal ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_nonfinite_check(const double* x, int64_t n, int* flag, cudaStream_t s) {
  k_nonfinite<<<grid_for(n), kThreads, 0, s>>>(x, n, flag);
  count_launch();
  return cudaGetLastError();
}

#define FVGB_INST(T)                                                                          \
  template cudaError_t launch_gradient<T>(fvgb_mesh_s*, int, const T*, T*, cudaStream_t);     \
  template cudaError_t launch_gradient_vertex<T>(fvgb_mesh_s*, int, const T*, T*, cudaStream_t); \
  template cudaError_t launch_vertex<T>(fvgb_mesh_s*, int, const T*, T*, bool, cudaStream_t); \
  template cudaError_t launch_face<T>(fvgb_mesh_s*, int, const T*, const T*, const T*,        \
                                      const double*, bool, double, bool, T*, cudaStream_t,   \
                                      const T*);                                              \
  template cudaError_t launch_bj_limit<T>(fvgb_mesh_s*, int, const T*, T*, cudaStream_t);     \
  template cudaError_t launch_update<T>(fvgb_mesh_s*, int, const T*, const T*, const T*,      \
                                        double, const T*, T*, T*, cudaStream_t);              \
  template cudaError_t launch_cell_physics<T>(fvgb_mesh_s*, const T*, const T*, double,       \
                                              double, double, T*, T*, T*, const SpotArgs&,    \
                                              cudaStream_t);
FVGB_INST(double)
FVGB_INST(float)
#undef FVGB_INST

}  // namespace fvgb
