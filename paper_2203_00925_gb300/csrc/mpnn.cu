// Message-passing warm start for the Poisson solve (not in the paper; the learned part
// of the synthetic workloads): inference and training kernels.
//
//   f_i   = [ (e/eps0) dq_i mu_i^(2/3) / (V s0),  phi_prev_i / (V s1) ]
//   h0    = relu(W_enc f + b_enc)                                  (hidden 64)
//   3 x:  m_i = sum_j w_ij (h_j - h_i)   (interior faces, w = c1 / max c1)
//         z   = W_l [h ; m] + b_l,   h = h + relu(z)
//   out   = w_dec . h + b_dec,  predicted potential increment V s2 out
//
// The layer products [h ; m] W_l^T (16 cells x 128 inputs x 64 outputs per warp tile)
// and their backward dz W_l run on the tensor cores with mma.sync m16n8k16 (BF16
// operands, FP32 accumulation); hidden states, messages and pre-activations are kept in
// FP32. Weight gradients are FP32 outer-product sums per block, reduced over blocks in
// FP64 in a fixed order (deterministic). Adam updates FP32 master weights and refreshes
// their BF16 copies.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace fvgb {

constexpr int kHid = 64;
constexpr int kIn = 2 * kHid;          // [h ; m]
constexpr int kLayers = 3;
constexpr int kOffWenc = 0, kOffBenc = 128, kOffLayer0 = 192, kLayerSize = kHid * kIn + kHid;
constexpr int kOffWdec = kOffLayer0 + kLayers * kLayerSize;   // 24960
constexpr int kOffBdec = kOffWdec + kHid;                       // 25024
constexpr int kNParams = kOffBdec + 1;                          // 25025
constexpr int kApad = kIn + 8;         // padded bf16 row of an A tile / W row
constexpr int kTpad = kHid + 8;        // padded bf16 row of a transposed W / dz tile
constexpr int kWarps = 4;              // warps per block of the tensor-core kernels
constexpr int kGradBlocks = 304;       // blocks of the gradient reductions

}  // namespace fvgb

struct fvgb_mpnn_s {
  fvgb_mesh m = nullptr;
  int bcset = 0;
  int64_t N = 0;
  double V = 1.0, s0 = 1.0, s1 = 1.0, s2 = 1.0;
  float* theta = nullptr;              // [fvgb::kNParams] FP32 master
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float* grad = nullptr;               // [params]
  __nv_bfloat16* wbf = nullptr;        // [3][64][128]
  float* wn = nullptr;                 // [N][4] message weights
  // activations of the two evaluations N(f) and N(f0 = 0) (set 0 and set 1)
  float* F[2] = {};                    // [N][2]
  float* Z0[2] = {};                   // [N][64]
  float* H[2][4] = {};                 // [N][64], layers 0..3
  float* M[2][3] = {};
  float* Z[2][3] = {};
  float* dout = nullptr;               // [N]
  float* dH = nullptr;                 // [N][64]
  float* dHb = nullptr;                // [N][64]
  float* G = nullptr;                  // [N][64] message part of dz W
  float* dZ = nullptr;                 // [N][64]
  float* part = nullptr;               // [blocks][params] gradient partials
  double* dpart = nullptr;             // [kGradBlocks] loss partials
  double* dloss = nullptr;             // [1]
  double* hloss = nullptr;             // pinned [1]
  int step = 0;
  bool train_buffers = false;
  std::vector<void*> allocs;
};

namespace fvgb {
using MpnnNet = ::fvgb_mpnn_s;

namespace {

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ void st_pair(__nv_bfloat16* p, float a, float b) {
  __nv_bfloat162 v;
  v.x = __float2bfloat16_rn(a);
  v.y = __float2bfloat16_rn(b);
  *reinterpret_cast<__nv_bfloat162*>(p) = v;
}

// ---- features and message weights ---------------------------------------------------------
__global__ void k_features(int64_t N, const double* __restrict__ dq, const double* __restrict__ phi,
                           const double* __restrict__ vol, double c0, double c1, int zero_charge,
                           float* __restrict__ F) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double h = cbrt(vol[i]);
    F[2 * i] = zero_charge ? 0.0f : (float)(c0 * dq[i] * h * h);
    F[2 * i + 1] = (float)(c1 * phi[i]);
  }
}

__global__ void k_max_coef(int64_t n, const double* __restrict__ coef, double* __restrict__ out) {
  __shared__ double sh[256];
  double mx = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, coef[i]);
  sh[threadIdx.x] = mx;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

__global__ void k_msg_weights(int64_t n, const double* __restrict__ coef, const double* __restrict__ cmax,
                              float* __restrict__ w) {
  const double inv = 1.0 / cmax[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w[i] = (float)(coef[i] * inv);
}

// ---- encoder ---------------------------------------------------------------------------------
__global__ void k_encode(int64_t N, const float* __restrict__ F, const float* __restrict__ theta,
                         float* __restrict__ Z0, float* __restrict__ H0) {
  __shared__ float W[3 * kHid];
  for (int k = threadIdx.x; k < 3 * kHid; k += blockDim.x) W[k] = theta[kOffWenc + k];  // W_enc, b_enc
  __syncthreads();
  const int64_t total = N * kHid;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / kHid;
    const int o = (int)(e % kHid);
    const float z = W[2 * o] * F[2 * i] + W[2 * o + 1] * F[2 * i + 1] + W[kOffBenc + o];
    if (Z0) Z0[e] = z;
    H0[e] = fmaxf(z, 0.0f);
  }
}

// ---- one message-passing layer, forward (tensor cores) ---------------------------------------
// Warp w of a block handles tiles of 16 cells: A = [h ; m] (16 x 128, BF16 in shared
// memory), Z = A W^T + b by 8 n-tiles x 8 k-steps of m16n8k16, H_out = H + relu(Z).
__global__ void __launch_bounds__(32 * kWarps)
k_layer_fwd(int64_t N, const float* __restrict__ H, const int4* __restrict__ nbr, const float4* __restrict__ wn,
            const __nv_bfloat16* __restrict__ Wg, const float* __restrict__ bias, float* __restrict__ Mout,
            float* __restrict__ Zout, float* __restrict__ Hout) {
  __shared__ __align__(16) __nv_bfloat16 Ws[kHid * kApad];
  __shared__ __align__(16) __nv_bfloat16 As[kWarps][16 * kApad];
  __shared__ float bs[kHid];
  for (int k = threadIdx.x; k < kHid * kIn; k += blockDim.x) Ws[(k / kIn) * kApad + (k % kIn)] = Wg[k];
  for (int k = threadIdx.x; k < kHid; k += blockDim.x) bs[k] = bias[k];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t4 = lane & 3;
  __nv_bfloat16* A = As[warp];
  const int64_t ntiles = (N + 15) / 16;
  for (int64_t tile = blockIdx.x * (int64_t)kWarps + warp; tile < ntiles; tile += (int64_t)gridDim.x * kWarps) {
    const int64_t c0 = tile * 16;
    for (int r = 0; r < 16; ++r) {
      const int64_t c = c0 + r;
      float hx = 0.0f, hy = 0.0f, mx = 0.0f, my = 0.0f;
      if (c < N) {
        const float2 h = *reinterpret_cast<const float2*>(H + c * kHid + 2 * lane);
        hx = h.x; hy = h.y;
        const int4 nb = nbr[c];
        const float4 w = wn[c];
        const int ns[4] = {nb.x, nb.y, nb.z, nb.w};
        const float ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const float2 hn = *reinterpret_cast<const float2*>(H + (int64_t)ns[s] * kHid + 2 * lane);
          mx += ws[s] * (hn.x - hx);
          my += ws[s] * (hn.y - hy);
        }
        if (Mout) *reinterpret_cast<float2*>(Mout + c * kHid + 2 * lane) = make_float2(mx, my);
      }
      st_pair(A + r * kApad + 2 * lane, hx, hy);
      st_pair(A + r * kApad + kHid + 2 * lane, mx, my);
    }
    __syncwarp();
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < kIn / 16; ++kk) {
      uint32_t a[4];
      a[0] = ld_pair(A + g * kApad + kk * 16 + 2 * t4);
      a[1] = ld_pair(A + (g + 8) * kApad + kk * 16 + 2 * t4);
      a[2] = ld_pair(A + g * kApad + kk * 16 + 8 + 2 * t4);
      a[3] = ld_pair(A + (g + 8) * kApad + kk * 16 + 8 + 2 * t4);
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const __nv_bfloat16* Bc = Ws + (nt * 8 + g) * kApad + kk * 16 + 2 * t4;
        mma16816(acc[nt], a, ld_pair(Bc), ld_pair(Bc + 8));
      }
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int col = nt * 8 + 2 * t4;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int64_t c = c0 + g + 8 * half;
        if (c >= N) continue;
        const float z0 = acc[nt][2 * half] + bs[col], z1 = acc[nt][2 * half + 1] + bs[col + 1];
        if (Zout) *reinterpret_cast<float2*>(Zout + c * kHid + col) = make_float2(z0, z1);
        const float2 h = *reinterpret_cast<const float2*>(H + c * kHid + col);
        *reinterpret_cast<float2*>(Hout + c * kHid + col) = make_float2(h.x + fmaxf(z0, 0.0f), h.y + fmaxf(z1, 0.0f));
      }
    }
    __syncwarp();
  }
}

// ---- decoder: out = w_dec . h + b_dec ----------------------------------------------------------
// mode 0: pred = scale out; mode 1: pred -= scale out (second evaluation, f0 = 0)
__global__ void k_decode(int64_t N, const float* __restrict__ H, const float* __restrict__ theta,
                         double scale, int mode, double* __restrict__ pred) {
  __shared__ float w[kHid + 1];
  for (int k = threadIdx.x; k <= kHid; k += blockDim.x) w[k] = theta[kOffWdec + k];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const float4* h = reinterpret_cast<const float4*>(H + i * kHid);
    float o = w[kHid];
#pragma unroll
    for (int q = 0; q < kHid / 4; ++q) {
      const float4 v = h[q];
      o += w[4 * q] * v.x + w[4 * q + 1] * v.y + w[4 * q + 2] * v.z + w[4 * q + 3] * v.w;
    }
    // separately rounded product and difference: equal outputs cancel exactly
    const double v = __dmul_rn(scale, (double)o);
    if (mode == 0) pred[i] = v;
    else pred[i] = __dsub_rn(pred[i], v);
  }
}

// Training head: pred = N(f) - N(f0 = 0) from the two last hidden states (b_dec cancels),
// dout = 2 (pred - t) / N, per-block loss partials, and the decoder gradient partials
// sum dout (h_a - h_b) (b_dec: 0).
__global__ void k_head_train(int64_t N, const float* __restrict__ Ha, const float* __restrict__ Hb,
                             const float* __restrict__ theta, double scale, const double* __restrict__ target,
                             float* __restrict__ dout, double* __restrict__ lpart) {
  __shared__ float w[kHid];
  __shared__ double sh[256];
  for (int k = threadIdx.x; k < kHid; k += blockDim.x) w[k] = theta[kOffWdec + k];
  __syncthreads();
  double l = 0.0;
  const double invN = 1.0 / (double)N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const float4* ha = reinterpret_cast<const float4*>(Ha + i * kHid);
    const float4* hb = reinterpret_cast<const float4*>(Hb + i * kHid);
    float o = 0.0f;
#pragma unroll
    for (int q = 0; q < kHid / 4; ++q) {
      const float4 a = ha[q], b = hb[q];
      o += w[4 * q] * (a.x - b.x) + w[4 * q + 1] * (a.y - b.y) + w[4 * q + 2] * (a.z - b.z) +
           w[4 * q + 3] * (a.w - b.w);
    }
    const double d = (double)o - target[i] / scale;
    l += d * d;
    dout[i] = (float)(2.0 * d * invN);
  }
  sh[threadIdx.x] = l;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) lpart[blockIdx.x] = sh[0];
}

// dH = sign dout w_dec for one evaluation
__global__ void k_head_dh(int64_t N, const float* __restrict__ dout, const float* __restrict__ theta,
                          float sign, float* __restrict__ dH) {
  const int64_t total = N * kHid;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    dH[e] = sign * dout[e / kHid] * theta[kOffWdec + (int)(e % kHid)];
}

// decoder gradient partials: part[b][w_dec] = sum dout (h_a - h_b); part[b][b_dec] = 0
__global__ void k_decode_grad(int64_t N, const float* __restrict__ Ha, const float* __restrict__ Hb,
                              const float* __restrict__ dout, float* __restrict__ part) {
  const int64_t per = (N + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * per, hi = lo + per < N ? lo + per : N;
  float* p = part + (size_t)blockIdx.x * kNParams;
  if (threadIdx.x < kHid) {
    float acc = 0.0f;
    for (int64_t i = lo; i < hi; ++i) acc += dout[i] * (Ha[i * kHid + threadIdx.x] - Hb[i * kHid + threadIdx.x]);
    p[kOffWdec + threadIdx.x] = acc;
  } else if (threadIdx.x == kHid) {
    p[kOffBdec] = 0.0f;
  }
}

// ---- one layer, backward (tensor cores) --------------------------------------------------------
// dz = dH_next * (z > 0);  [g_h ; g_m] = dz W_l  (16 cells x 64 x 128 per warp tile);
// dH = dH_next + g_h;  G = g_m (its message is added by k_msg_add);  dZ = dz (FP32, for the
// weight gradients).
__global__ void __launch_bounds__(32 * kWarps)
k_layer_bwd(int64_t N, const float* __restrict__ dHn, const float* __restrict__ Z,
            const __nv_bfloat16* __restrict__ Wg, float* __restrict__ dZ, float* __restrict__ dH,
            float* __restrict__ G) {
  __shared__ __align__(16) __nv_bfloat16 WT[kIn * kTpad];   // W^T: [in][out]
  __shared__ __align__(16) __nv_bfloat16 Ds[kWarps][16 * kTpad];
  for (int k = threadIdx.x; k < kHid * kIn; k += blockDim.x) {
    const int o = k / kIn, i = k % kIn;
    WT[i * kTpad + o] = Wg[k];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t4 = lane & 3;
  __nv_bfloat16* D = Ds[warp];
  const int64_t ntiles = (N + 15) / 16;
  for (int64_t tile = blockIdx.x * (int64_t)kWarps + warp; tile < ntiles; tile += (int64_t)gridDim.x * kWarps) {
    const int64_t c0 = tile * 16;
    for (int r = 0; r < 16; ++r) {
      const int64_t c = c0 + r;
      float dx = 0.0f, dy = 0.0f;
      if (c < N) {
        const float2 d = *reinterpret_cast<const float2*>(dHn + c * kHid + 2 * lane);
        const float2 z = *reinterpret_cast<const float2*>(Z + c * kHid + 2 * lane);
        dx = z.x > 0.0f ? d.x : 0.0f;
        dy = z.y > 0.0f ? d.y : 0.0f;
        *reinterpret_cast<float2*>(dZ + c * kHid + 2 * lane) = make_float2(dx, dy);
      }
      st_pair(D + r * kTpad + 2 * lane, dx, dy);
    }
    __syncwarp();
    float acc[16][4];
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < kHid / 16; ++kk) {
      uint32_t a[4];
      a[0] = ld_pair(D + g * kTpad + kk * 16 + 2 * t4);
      a[1] = ld_pair(D + (g + 8) * kTpad + kk * 16 + 2 * t4);
      a[2] = ld_pair(D + g * kTpad + kk * 16 + 8 + 2 * t4);
      a[3] = ld_pair(D + (g + 8) * kTpad + kk * 16 + 8 + 2 * t4);
#pragma unroll
      for (int nt = 0; nt < 16; ++nt) {
        const __nv_bfloat16* Bc = WT + (nt * 8 + g) * kTpad + kk * 16 + 2 * t4;
        mma16816(acc[nt], a, ld_pair(Bc), ld_pair(Bc + 8));
      }
    }
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
      const int col = nt * 8 + 2 * t4;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int64_t c = c0 + g + 8 * half;
        if (c >= N) continue;
        const float v0 = acc[nt][2 * half], v1 = acc[nt][2 * half + 1];
        if (col < kHid) {
          const float2 d = *reinterpret_cast<const float2*>(dHn + c * kHid + col);
          *reinterpret_cast<float2*>(dH + c * kHid + col) = make_float2(d.x + v0, d.y + v1);
        } else {
          *reinterpret_cast<float2*>(G + c * kHid + col - kHid) = make_float2(v0, v1);
        }
      }
    }
    __syncwarp();
  }
}

// dH_i += sum_j w_ij (G_j - G_i): the adjoint of the (symmetric) message operator
__global__ void k_msg_add(int64_t N, const float* __restrict__ Gm, const int4* __restrict__ nbr,
                          const float4* __restrict__ wn, float* __restrict__ dH) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < N; c += nwarps) {
    const float2 gi = *reinterpret_cast<const float2*>(Gm + c * kHid + 2 * lane);
    const int4 nb = nbr[c];
    const float4 w = wn[c];
    const int ns[4] = {nb.x, nb.y, nb.z, nb.w};
    const float ws[4] = {w.x, w.y, w.z, w.w};
    float mx = 0.0f, my = 0.0f;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const float2 gn = *reinterpret_cast<const float2*>(Gm + (int64_t)ns[s] * kHid + 2 * lane);
      mx += ws[s] * (gn.x - gi.x);
      my += ws[s] * (gn.y - gi.y);
    }
    float2* d = reinterpret_cast<float2*>(dH + c * kHid + 2 * lane);
    const float2 dv = *d;
    *d = make_float2(dv.x + mx, dv.y + my);
  }
}

// Weight gradients of one layer: part[b][W_l] = sum over the block's cells of dz (x) [h ; m],
// part[b][b_l] = sum dz. Thread t owns input feature t % 128 and 32 outputs.
__global__ void __launch_bounds__(256) k_layer_wgrad(int64_t N, const float* __restrict__ dZ,
                                                     const float* __restrict__ H, const float* __restrict__ Mm,
                                                     int off, float* __restrict__ part) {
  __shared__ float dz[16][kHid];
  __shared__ float hm[16][kIn];
  const int i = threadIdx.x % kIn, og = threadIdx.x / kIn;
  float acc[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) acc[j] = 0.0f;
  float accb = 0.0f;
  const int64_t per = (N + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * per, hi = lo + per < N ? lo + per : N;
  for (int64_t c0 = lo; c0 < hi; c0 += 16) {
    const int nc = (int)(hi - c0 < 16 ? hi - c0 : 16);
    for (int k = threadIdx.x; k < 16 * kHid; k += blockDim.x) {
      const int r = k / kHid, o = k % kHid;
      dz[r][o] = r < nc ? dZ[(c0 + r) * kHid + o] : 0.0f;
      hm[r][o] = r < nc ? H[(c0 + r) * kHid + o] : 0.0f;
      hm[r][kHid + o] = r < nc ? Mm[(c0 + r) * kHid + o] : 0.0f;
    }
    __syncthreads();
    for (int r = 0; r < nc; ++r) {
      const float v = hm[r][i];
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] += dz[r][og * 32 + j] * v;
      if (threadIdx.x < kHid) accb += dz[r][threadIdx.x];
    }
    __syncthreads();
  }
  float* p = part + (size_t)blockIdx.x * kNParams + off;
#pragma unroll
  for (int j = 0; j < 32; ++j) p[(og * 32 + j) * kIn + i] = acc[j];
  if (threadIdx.x < kHid) p[kHid * kIn + threadIdx.x] = accb;
}

// encoder gradients: dz0 = dH0 * (z0 > 0); part[b][W_enc] = sum dz0 (x) f, part[b][b_enc] = sum dz0
__global__ void k_encode_grad(int64_t N, const float* __restrict__ dH, const float* __restrict__ Z0,
                              const float* __restrict__ F, float* __restrict__ part) {
  const int o = threadIdx.x;
  if (o >= kHid) return;
  const int64_t per = (N + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * per, hi = lo + per < N ? lo + per : N;
  float a0 = 0.0f, a1 = 0.0f, ab = 0.0f;
  for (int64_t c = lo; c < hi; ++c) {
    const float d = Z0[c * kHid + o] > 0.0f ? dH[c * kHid + o] : 0.0f;
    a0 += d * F[2 * c];
    a1 += d * F[2 * c + 1];
    ab += d;
  }
  float* p = part + (size_t)blockIdx.x * kNParams;
  p[kOffWenc + 2 * o] = a0;
  p[kOffWenc + 2 * o + 1] = a1;
  p[kOffBenc + o] = ab;
}

// grad[k] = sum over blocks of part[b][k] in block order (FP64 accumulation)
__global__ void k_reduce_grad(int nblocks, const float* __restrict__ part, float* __restrict__ grad) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kNParams; k += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += (double)part[(size_t)b * kNParams + k];
    grad[k] = (float)s;
  }
}

__global__ void k_reduce_loss(int n, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < n; ++b) s += part[b];
    out[0] = s;
  }
}

// Adam on the FP32 master weights; refresh the BF16 copies of the layer matrices
__global__ void k_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float b1, float b2, float c1, float c2,
                       float eps, __nv_bfloat16* __restrict__ wbf) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kNParams; k += gridDim.x * blockDim.x) {
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.0f - b1) * gk;
    const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float t = theta[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    theta[k] = t;
    const int l = (k - kOffLayer0) / kLayerSize, r = (k - kOffLayer0) % kLayerSize;
    if (k >= kOffLayer0 && k < kOffWdec && r < kHid * kIn) wbf[l * kHid * kIn + r] = __float2bfloat16_rn(t);
  }
}

__global__ void k_refresh_bf16(const float* __restrict__ theta, __nv_bfloat16* __restrict__ wbf) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kLayers * kHid * kIn; k += gridDim.x * blockDim.x) {
    const int l = k / (kHid * kIn), r = k % (kHid * kIn);
    wbf[k] = __float2bfloat16_rn(theta[kOffLayer0 + l * kLayerSize + r]);
  }
}

template <typename T>
cudaError_t nalloc(MpnnNet* n, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e == cudaSuccess) n->allocs.push_back(q);
  *p = (T*)q;
  return e;
}

void net_release(MpnnNet* n) {
  for (void* p : n->allocs) cudaFree(p);
  if (n->hloss) cudaFreeHost(n->hloss);
  delete n;
}

unsigned grid_n(int64_t n, int t = 256) {
  int64_t g = (n + t - 1) / t;
  if (g > 65535 * 8) g = 65535 * 8;
  return (unsigned)(g > 0 ? g : 1);
}

cudaError_t alloc_train(MpnnNet* n) {
  if (n->train_buffers) return cudaSuccess;
  const size_t NH = (size_t)n->N * kHid;
  cudaError_t e;
  for (int set = 0; set < 2; ++set) {
    if (set == 1 && (e = nalloc(n, &n->F[1], (size_t)n->N * 2))) return e;
    if ((e = nalloc(n, &n->Z0[set], NH))) return e;
    for (int l = 0; l < kLayers; ++l) {
      if ((e = nalloc(n, &n->M[set][l], NH))) return e;
      if ((e = nalloc(n, &n->Z[set][l], NH))) return e;
    }
    for (int l = set == 0 ? 2 : 0; l <= kLayers; ++l)
      if ((e = nalloc(n, &n->H[set][l], NH))) return e;
  }
  if ((e = nalloc(n, &n->dH, NH))) return e;
  if ((e = nalloc(n, &n->dHb, NH))) return e;
  if ((e = nalloc(n, &n->G, NH))) return e;
  if ((e = nalloc(n, &n->dZ, NH))) return e;
  if ((e = nalloc(n, &n->dout, n->N))) return e;
  if ((e = nalloc(n, &n->part, (size_t)2 * kGradBlocks * kNParams))) return e;
  if ((e = nalloc(n, &n->dpart, kGradBlocks))) return e;
  n->train_buffers = true;
  return cudaSuccess;
}

unsigned layer_grid(MpnnNet* n) {
  return (unsigned)std::min<int64_t>((n->N + 16 * kWarps - 1) / (16 * kWarps), (int64_t)n->m->num_sms * 16);
}

// One evaluation of the network. train: activation set ``set`` keeps every layer;
// otherwise hidden states ping-pong in H[0][0..1]. zero_charge: f0 = 0.
cudaError_t forward(MpnnNet* n, int set, const double* dq, const double* phi, bool train,
                    bool zero_charge, cudaStream_t s) {
  fvgb_mesh m = n->m;
  const int64_t N = n->N;
  constexpr double kEoverEps0 = 1.602176634e-19 / 8.8541878128e-12;
  float* F = n->F[train ? set : 0];
  k_features<<<grid_n(N), 256, 0, s>>>(N, dq, phi, m->g64.vol, kEoverEps0 / (n->V * n->s0),
                                       1.0 / (n->V * n->s1), zero_charge ? 1 : 0, F);
  k_encode<<<grid_n(N * kHid), 256, 0, s>>>(N, F, n->theta, train ? n->Z0[set] : nullptr, n->H[train ? set : 0][0]);
  count_launch(2);
  const int4* nbr = reinterpret_cast<const int4*>(m->g64.bc[n->bcset].at_nbr);
  const float4* wn = reinterpret_cast<const float4*>(n->wn);
  for (int l = 0; l < kLayers; ++l) {
    const float* Hin = train ? n->H[set][l] : n->H[0][l % 2];
    float* Hout = train ? n->H[set][l + 1] : n->H[0][(l + 1) % 2];
    k_layer_fwd<<<layer_grid(n), 32 * kWarps, 0, s>>>(N, Hin, nbr, wn, n->wbf + (size_t)l * kHid * kIn,
                                                      n->theta + kOffLayer0 + l * kLayerSize + kHid * kIn,
                                                      train ? n->M[set][l] : nullptr,
                                                      train ? n->Z[set][l] : nullptr, Hout);
    count_launch();
  }
  return cudaGetLastError();
}

// prediction dphi = V s2 (N(f) - N(f0 = 0))
cudaError_t predict(MpnnNet* n, const double* dq, const double* phi, double* dphi, cudaStream_t s) {
  cudaError_t e;
  const double scale = n->V * n->s2;
  const float* last = n->H[0][kLayers % 2];
  if ((e = forward(n, 0, dq, phi, false, false, s))) return e;
  k_decode<<<grid_n(n->N), 256, 0, s>>>(n->N, last, n->theta, scale, 0, dphi);
  if ((e = forward(n, 0, dq, phi, false, true, s))) return e;
  k_decode<<<grid_n(n->N), 256, 0, s>>>(n->N, last, n->theta, scale, 1, dphi);
  count_launch(2);
  return cudaGetLastError();
}

// backward of sum_i dout_i sign N_set(f)_i through the layers and the encoder into the
// gradient partial rows [row0, row0 + kGradBlocks)
void backward_set(MpnnNet* n, int set, float sign, int row0, cudaStream_t s) {
  const int64_t N = n->N;
  const int G = kGradBlocks;
  float* part = n->part + (size_t)row0 * kNParams;
  k_head_dh<<<grid_n(N * kHid), 256, 0, s>>>(N, n->dout, n->theta, sign, n->dH);
  count_launch();
  float* dHn = n->dH;
  float* dHo = n->dHb;
  const int4* nbr = reinterpret_cast<const int4*>(n->m->g64.bc[n->bcset].at_nbr);
  const float4* wn = reinterpret_cast<const float4*>(n->wn);
  for (int l = kLayers - 1; l >= 0; --l) {
    k_layer_bwd<<<layer_grid(n), 32 * kWarps, 0, s>>>(N, dHn, n->Z[set][l], n->wbf + (size_t)l * kHid * kIn,
                                                      n->dZ, dHo, n->G);
    k_msg_add<<<grid_n(N * 32), 256, 0, s>>>(N, n->G, nbr, wn, dHo);
    k_layer_wgrad<<<G, 256, 0, s>>>(N, n->dZ, n->H[set][l], n->M[set][l], kOffLayer0 + l * kLayerSize, part);
    count_launch(3);
    std::swap(dHn, dHo);
  }
  k_encode_grad<<<G, kHid, 0, s>>>(N, dHn, n->Z0[set], n->F[set], part);
  count_launch();
}

// loss and gradient into n->grad (and n->dloss)
cudaError_t loss_grad(MpnnNet* n, const double* dq, const double* phi, const double* target, cudaStream_t s) {
  cudaError_t e;
  if ((e = alloc_train(n))) return e;
  if ((e = forward(n, 0, dq, phi, true, false, s))) return e;
  if ((e = forward(n, 1, dq, phi, true, true, s))) return e;
  const int64_t N = n->N;
  const int G = kGradBlocks;
  if ((e = cudaMemsetAsync(n->part, 0, (size_t)2 * G * kNParams * sizeof(float), s))) return e;
  k_head_train<<<G, 256, 0, s>>>(N, n->H[0][kLayers], n->H[1][kLayers], n->theta, n->V * n->s2, target,
                                 n->dout, n->dpart);
  k_reduce_loss<<<1, 32, 0, s>>>(G, n->dpart, n->dloss);
  k_decode_grad<<<G, 96, 0, s>>>(N, n->H[0][kLayers], n->H[1][kLayers], n->dout, n->part);
  count_launch(3);
  backward_set(n, 0, 1.0f, 0, s);
  backward_set(n, 1, -1.0f, G, s);
  k_reduce_grad<<<grid_n(kNParams), 256, 0, s>>>(2 * G, n->part, n->grad);
  count_launch();
  return cudaGetLastError();
}

}  // namespace
}  // namespace fvgb

using namespace fvgb;

extern "C" {

fvgb_status fvgb_mpnn_create(fvgb_mesh m, int32_t bcset, fvgb_mpnn* out) {
  if (!m || !out) { set_error("null argument"); return FVGB_EINVAL; }
  *out = nullptr;
  if (bcset < 0 || bcset >= (int32_t)m->g64.bc.size()) { set_error("bcset index out of range"); return FVGB_EINVAL; }
  fvgb_mpnn_s* n = new fvgb_mpnn_s();
  n->m = m;
  n->bcset = bcset;
  n->N = m->topo.N;
  const size_t NH = (size_t)n->N * kHid;
  cudaError_t e = cudaSuccess;
  auto fail = [&](const char* what) {
    fvgb_status st = cuda_status(e, what);
    net_release(n);
    return st;
  };
  if ((e = nalloc(n, &n->theta, kNParams))) return fail("allocation");
  if ((e = nalloc(n, &n->adam_m, kNParams))) return fail("allocation");
  if ((e = nalloc(n, &n->adam_v, kNParams))) return fail("allocation");
  if ((e = nalloc(n, &n->grad, kNParams))) return fail("allocation");
  if ((e = nalloc(n, &n->wbf, (size_t)kLayers * kHid * kIn))) return fail("allocation");
  if ((e = nalloc(n, &n->wn, (size_t)n->N * 4))) return fail("allocation");
  if ((e = nalloc(n, &n->F[0], (size_t)n->N * 2))) return fail("allocation");
  if ((e = nalloc(n, &n->H[0][0], NH))) return fail("allocation");
  if ((e = nalloc(n, &n->H[0][1], NH))) return fail("allocation");
  if ((e = nalloc(n, &n->dloss, 2))) return fail("allocation");
  if ((e = cudaMallocHost((void**)&n->hloss, sizeof(double)))) return fail("pinned allocation");
  if ((e = cudaMemset(n->theta, 0, kNParams * sizeof(float)))) return fail("memset");
  if ((e = cudaMemset(n->adam_m, 0, kNParams * sizeof(float)))) return fail("memset");
  if ((e = cudaMemset(n->adam_v, 0, kNParams * sizeof(float)))) return fail("memset");
  if ((e = cudaMemset(n->wbf, 0, (size_t)kLayers * kHid * kIn * sizeof(__nv_bfloat16)))) return fail("memset");
  // message weights: c1 of the interior faces (two-point coefficients of bcset), / max
  const double* coef = m->g64.bc[bcset].at_coef;
  k_max_coef<<<1, 256>>>(4 * n->N, coef, n->dloss + 1);
  k_msg_weights<<<grid_n(4 * n->N), 256>>>(4 * n->N, coef, n->dloss + 1, n->wn);
  count_launch(2);
  if ((e = cudaDeviceSynchronize())) return fail("message weights");
  *out = n;
  return FVGB_OK;
}

fvgb_status fvgb_mpnn_free(fvgb_mpnn net) {
  if (!net) return FVGB_OK;
  cudaDeviceSynchronize();
  net_release(net);
  return FVGB_OK;
}

int64_t fvgb_mpnn_param_count(void) { return kNParams; }

fvgb_status fvgb_mpnn_set_params(fvgb_mpnn net, const float* theta_host) {
  if (!net || !theta_host) { set_error("null argument"); return FVGB_EINVAL; }
  FVGB_TRY(cudaMemcpy(net->theta, theta_host, kNParams * sizeof(float), cudaMemcpyHostToDevice), "copy");
  FVGB_TRY(cudaMemset(net->adam_m, 0, kNParams * sizeof(float)), "memset");
  FVGB_TRY(cudaMemset(net->adam_v, 0, kNParams * sizeof(float)), "memset");
  net->step = 0;
  k_refresh_bf16<<<grid_n(kLayers * kHid * kIn), 256>>>(net->theta, net->wbf);
  count_launch();
  return cuda_status(cudaDeviceSynchronize(), "refresh");
}

fvgb_status fvgb_mpnn_get_params(fvgb_mpnn net, float* theta_host) {
  if (!net || !theta_host) { set_error("null argument"); return FVGB_EINVAL; }
  return cuda_status(cudaMemcpy(theta_host, net->theta, kNParams * sizeof(float), cudaMemcpyDeviceToHost), "copy");
}

fvgb_status fvgb_mpnn_set_scales(fvgb_mpnn net, double V, double s0, double s1, double s2) {
  if (!net || !(V > 0) || !(s0 > 0) || !(s1 > 0) || !(s2 > 0)) { set_error("scales must be positive"); return FVGB_EINVAL; }
  net->V = V; net->s0 = s0; net->s1 = s1; net->s2 = s2;
  return FVGB_OK;
}

fvgb_status fvgb_mpnn_predict(fvgb_mpnn net, const double* dq, const double* phi_prev, double* dphi,
                              void* stream) {
  if (!net || !dq || !phi_prev || !dphi) { set_error("null argument"); return FVGB_EINVAL; }
  return cuda_status(predict(net, dq, phi_prev, dphi, (cudaStream_t)stream), "forward");
}

fvgb_status fvgb_mpnn_loss_grad(fvgb_mpnn net, const double* dq, const double* phi_prev,
                                const double* target, double* loss_host, float* grad_host, void* stream) {
  if (!net || !dq || !phi_prev || !target) { set_error("null argument"); return FVGB_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  FVGB_TRY(loss_grad(net, dq, phi_prev, target, s), "loss/gradient");
  if (grad_host) FVGB_TRY(cudaMemcpyAsync(grad_host, net->grad, kNParams * sizeof(float), cudaMemcpyDeviceToHost, s), "copy");
  FVGB_TRY(cudaMemcpyAsync(net->hloss, net->dloss, sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
  FVGB_TRY(cudaStreamSynchronize(s), "synchronize");
  if (loss_host) *loss_host = net->hloss[0] / (double)net->N;
  return FVGB_OK;
}

fvgb_status fvgb_mpnn_train_step(fvgb_mpnn net, const double* dq, const double* phi_prev,
                                 const double* target, float lr, double* loss_host, void* stream) {
  if (!net || !dq || !phi_prev || !target || !(lr > 0.0f)) { set_error("bad arguments"); return FVGB_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  FVGB_TRY(loss_grad(net, dq, phi_prev, target, s), "loss/gradient");
  net->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, (float)net->step), c2 = 1.0f - std::pow(b2, (float)net->step);
  k_adam<<<grid_n(kNParams), 256, 0, s>>>(net->theta, net->adam_m, net->adam_v, net->grad, lr, b1, b2, c1, c2,
                                          1e-8f, net->wbf);
  count_launch();
  if (loss_host) {
    FVGB_TRY(cudaMemcpyAsync(net->hloss, net->dloss, sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
    FVGB_TRY(cudaStreamSynchronize(s), "synchronize");
    *loss_host = net->hloss[0] / (double)net->N;
  }
  return cuda_status(cudaGetLastError(), "adam");
}

}  // extern "C"
