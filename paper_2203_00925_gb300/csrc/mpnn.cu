// Message-passing warm start for the Poisson solve (not in the paper; the learned part
// of the synthetic workloads): inference and training kernels.
//
//   f_i   = [ (e/eps0) dq_i mu_i^(2/3) / (V s0),  phi_prev_i / (V s1) ]
//   h0    = relu(W_enc f + b_enc)                                  (hidden 64)
//   layer(l, h; graph): m_i = sum_j w_ij (h_j - h_i), z = W_l [h ; m] + b_l, h + relu(z)
//   h1    = layer(0, h0; interior faces, w = c1 / max c1)
//   middle layer on a hierarchy of cubic aggregates of the cells (built on the host when
//   the network is created): at every level the mean over each aggregate of the level
//   below, then kHops times layer(1, c; face-adjacent aggregates, w = 1/6); back up, every
//   level adds its aggregate's value, down to h2 = h1 + c_1 of the cell's aggregate
//   h3    = layer(2, h2; interior faces)
//   out   = w_dec . h3 + b_dec,  predicted potential increment V s2 out
//
// The layer products [h ; m] W_l^T (128 rows x 128 inputs x 64 outputs per tile) and
// their backward dz W_l (128 rows x 64 x 128) run on the fifth-generation tensor cores:
// the block gathers a tile of BF16 operands into shared memory (128-byte swizzled K-major
// layout), one thread issues tcgen05.mma (kind::f16, FP32 accumulators in tensor memory),
// completion is signalled through an mbarrier, and the warps read the accumulator with
// tcgen05.ld for the fused epilogue (bias, ReLU, residual). The same kernels run the fine
// layers (rows = cells, four face neighbours with weights) and the aggregate layers (rows =
// aggregates, up to six neighbours of weight 1/6). Training keeps hidden states, messages
// and pre-activations in FP32; the inference path writes the cells' hidden states once, as
// BF16 (the tensor-core operands are BF16 anyway), with the encoder, the hierarchy's copy
// back and the decoder fused into the layers. Weight gradients are per-block sums accumulated in
// tensor memory, reduced over blocks in FP64 in a fixed order (deterministic). Adam updates
// FP32 master weights and refreshes their BF16 copies.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
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
constexpr int kTile = 128;             // cells per tensor-core tile (the MMA's M)
constexpr int kTileThreads = 256;      // threads of the layer kernels: two per cell row
constexpr int kGradBlocks = 304;       // blocks of the gradient reductions (and of the backward)
constexpr int kHops = 2;               // applications of the middle layer per aggregate level
constexpr int kMaxLevels = 16;
// dynamic shared memory of the layer kernels: forward A = [h ; m] (128 x 128 BF16, 32 KB)
// and W (64 x 128, 16 KB): up to four blocks an SM, 4 x 64 tensor-memory columns.
// Backward: B1 = W^T (128 x 64, 16 KB), A1 = dz (128 cells x 64, 16 KB), A2 = [h ; m]^T
// (128 inputs x 128 cells, 32 KB), B2 = dz^T (64 outputs x 128 cells, 16 KB); the last three
// are reused as the 64 KB staging of the data product: at most two blocks an SM,
// 2 x 256 tensor-memory columns.
constexpr uint32_t kFwdB = 32768, kFwdSmem = 49152;
constexpr uint32_t kBwdA1 = 16384, kBwdA2 = 32768, kBwdB2 = 65536, kBwdSmem = 81920;

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
  double* hcell = nullptr;             // [N] mu^(1/3)
  __nv_bfloat16* Hb[2] = {};           // [N][64] BF16 hidden states of the inference path
  // aggregate hierarchy (multilevel architecture; n_lev = 0: the middle layer runs on the
  // faces): level k (0-based) has lev_n[k] nodes, rows [lev_off[k], + lev_n[k]) of the
  // coarse arrays; the nodes below it are the cells (k = 0) or level k - 1's
  int n_lev = 0;
  int64_t lev_n[fvgb::kMaxLevels] = {};
  int64_t lev_off[fvgb::kMaxLevels + 1] = {};
  int64_t below_off[fvgb::kMaxLevels + 1] = {};   // offsets into parent / child_idx
  int64_t ptr_off[fvgb::kMaxLevels] = {};         // offsets into child_ptr
  int32_t* parent = nullptr;           // per level: aggregate of each node below (level-local)
  int32_t* child_ptr = nullptr;        // per level: [lev_n + 1] CSR of the nodes below
  int32_t* child_idx = nullptr;        // per level: nodes below, by aggregate, ascending
  float* inv_count = nullptr;          // [coarse rows] 1 / nodes in the aggregate
  int32_t* cnbr = nullptr;             // [coarse rows][8] face-adjacent aggregates, padded with self
  int32_t* nparent = nullptr;          // [N][4] level-1 aggregate of each face-neighbour slot
  int64_t n_coarse = 0;
  // activations of the two evaluations N(f) and N(f0 = 0) (set 0 and set 1)
  float* F[2] = {};                    // [N][2]
  float* Z0[2] = {};                   // [N][64]
  float* H[2][4] = {};                 // [N][64]: h0, h1, h2, h3
  float* M[2][3] = {};                 // fine layers (0 and 2; 1 too when local)
  float* Z[2][3] = {};
  float* Hc[2][fvgb::kHops + 1] = {};  // [coarse rows][64]: hop inputs, last = level output
  float* Mc[2][fvgb::kHops] = {};
  float* Zc[2][fvgb::kHops] = {};
  float* dout = nullptr;               // [N]
  float* dH = nullptr;                 // [N][64]
  float* dHb = nullptr;                // [N][64]
  float* G = nullptr;                  // [N][64] message part of dz W
  float* dC = nullptr;                 // [coarse rows][64] gradients of the level outputs
  float* cP = nullptr;                 // [lev_n[0]][64] gradient ping-pong of the hops
  float* cQ = nullptr;
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

// ---- tcgen05 helpers -------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 128-byte swizzled K-major layout: K in slabs of 64 elements, a slab of R rows taking
// R x 128 bytes (1024-byte aligned); the 16-byte chunk c of row r sits at chunk c ^ (r % 8)
// of the row (the hardware's swizzle of address bits [4, 7) by bits [7, 10)), so the eight
// chunks of a row, and one chunk of eight consecutive rows, fall in different banks.
__device__ __forceinline__ uint32_t sw_off(int r, int k, int R) {
  return (uint32_t)((k >> 6) * R * 128 + r * 128 + ((((k >> 3) & 7) ^ (r & 7)) << 4) + (k & 7) * 2);
}
// descriptor of such an operand: start address (slab base + 32 bytes per K step of 16 inside
// the slab), stride byte offset 1024 (8-row groups), version 1, swizzle mode 128 bytes
__device__ __forceinline__ uint64_t sw_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}
// address of the K step kk (16 elements) of a swizzled operand of R rows
__device__ __forceinline__ uint32_t sw_kstep(uint32_t base, int kk, int R) {
  return base + (uint32_t)((kk >> 2) * R * 128 + (kk & 3) * 32);
}

// Instruction descriptor of kind::f16: BF16 A and B (both K-major), FP32 accumulator, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// make the block's st.shared of an operand tile visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {   // one warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {      // the same warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// D (tensor memory) = A B^T (+ D when accumulate), one thread issues
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       int accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
// arrive on the mbarrier once every MMA issued so far by this thread has completed
__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ unsigned long long mp_global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase ``parity`` of the mbarrier, for at most one second; false on timeout.
constexpr unsigned long long kMbarTimeoutNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
  const uint32_t a = smem_u32(mbar);
  const unsigned long long t0 = mp_global_ns();
  for (;;) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(a), "r"(parity) : "memory");
    if (done) return true;
    if (mp_global_ns() - t0 > kMbarTimeoutNs) return false;
  }
}

// 32 consecutive FP32 accumulator columns of this thread's lane (its warp's 32 lanes)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 v;
  v.x = __float2bfloat16_rn(a);
  v.y = __float2bfloat16_rn(b);
  return *reinterpret_cast<uint32_t*>(&v);
}
// eight values as BF16 into one 16-byte row of a core matrix
__device__ __forceinline__ void st_bf16x8(unsigned char* p, const float (&v)[8]) {
  *reinterpret_cast<uint4*>(p) = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]),
                                            pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
}
__device__ __forceinline__ void st_bf16x4(unsigned char* p, const float4& v) {
  *reinterpret_cast<uint2*>(p) = make_uint2(pack_bf16(v.x, v.y), pack_bf16(v.z, v.w));
}
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
// four BF16 values (8 bytes) widened to FP32
__device__ __forceinline__ float4 ld_bf16x4(const __nv_bfloat16* p) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&v.x);
  const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&v.y);
  return make_float4(__bfloat162float(a.x), __bfloat162float(a.y), __bfloat162float(b.x), __bfloat162float(b.y));
}
__device__ __forceinline__ void st4(float* p, const float4& v) { *reinterpret_cast<float4*>(p) = v; }
// staging of a row-per-thread accumulator: float4 q of row r at q ^ (r % Q) (Q = float4s
// per row), so that 32 rows writing one quad, or one row read by quads, hit distinct banks
template <int Q>
__device__ __forceinline__ float* stage_at(float* S, int r, int q) {
  return S + r * (4 * Q) + 4 * (q ^ (r % Q));
}

// ---- features and message weights ---------------------------------------------------------
// hcell = mu^(1/3) of every cell, once per network (the features' length scale)
__global__ void k_cell_size(int64_t N, const double* __restrict__ vol, double* __restrict__ hcell) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    hcell[i] = cbrt(vol[i]);
}

__global__ void k_features(int64_t N, const double* __restrict__ dq, const double* __restrict__ phi,
                           const double* __restrict__ hcell, double c0, double c1, int zero_charge,
                           float* __restrict__ F) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double h = hcell[i];
    F[2 * i] = zero_charge ? 0.0f : (float)(c0 * dq[i] * h * h);
    F[2 * i + 1] = (float)(c1 * phi[i]);
  }
}

// maximum of n coefficients: per-block maxima into part[blockIdx.x], then (nblocks = 1,
// n = grid of the first pass) the maximum of those
__global__ void k_max_coef(int64_t n, const double* __restrict__ coef, double* __restrict__ part) {
  __shared__ double sh[256];
  double mx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    mx = fmax(mx, coef[i]);
  sh[threadIdx.x] = mx;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
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
// Where the layer's input rows come from and where its output goes:
//  kInH:      h_j = H[j]
//  kInEncode: h_j = relu(W_enc F[j] + b_enc), the encoder recomputed from the two features
//             (inference: the encoder's 256-byte rows are never written)
//  kInHb:     h_j = Hb[j], a BF16 copy (inference, where the cells' hidden states are
//             written once and read by the next layer: half the bytes)
//  kInParentB: h_j = Hb[j] + U[parent[j]], the copy back of the aggregate hierarchy applied
//             on the fly (inference)
// Output: Hout = h + relu(z) (and M, Z when given), or with dec set the decoder on the fly,
// o = w_dec . (h + relu(z)) + b_dec, pred = scale o (mode 0) or pred - scale o (mode 1).
enum LayerIn { kInH = 0, kInEncode = 1, kInHb = 2, kInParentB = 3 };

struct LayerArgs {
  const float* H = nullptr;          // [rows][64] (kInH)
  const __nv_bfloat16* Hb = nullptr; // [rows][64] BF16 (kInHb, kInParentB)
  const float* F = nullptr;          // [rows][2] features (kInEncode)
  const float* enc = nullptr;        // W_enc [64][2], b_enc [64] (kInEncode)
  const float* U = nullptr;          // [aggregates][64] (kInParentB)
  const int32_t* parent = nullptr;   // [rows] (kInParentB)
  const int4* nparent = nullptr;     // [rows] parents of the four face-neighbour slots (kInParentB)
  float* M = nullptr;                // outputs: messages, pre-activations, hidden state
  float* Z = nullptr;
  float* Hout = nullptr;
  __nv_bfloat16* Houtb = nullptr;    // or the hidden state as BF16
  const float* dec = nullptr;        // w_dec [64], b_dec: decode instead of writing Hout
  double scale = 1.0;
  int mode = 0;
  double* pred = nullptr;
};

// Persistent over tiles of 128 rows. The block's eight warps gather the tile's rows
// A_c = [h ; m] into the BF16 operand tile (fine layers: rows are cells, m = sum_j w_j (h_j - h)
// over four face neighbours, nbr [N] int4 and wn [N] float4; aggregate layers: rows are
// aggregates, m = (1/6) sum_j (h_j - h) over six slots nbr [2 N] int4 padded with the row
// itself), 16 lanes a row (a float4 of features each: whole 256-byte rows per load), two
// rows a step, warp w taking rows [16 w, 16 w + 16); the tile is in the 128-byte swizzled
// K-major layout (h in the first slab, m in the second), so a row's stores are
// bank-conflict-free. Thread 0 issues Z = A W^T as 8 tcgen05.mma of K = 16 into 64
// tensor-memory columns; after the mbarrier signals completion warp w reads lanes
// 32 (w % 4) .. + 31 and columns 32 (w / 4) .. + 31, adds the bias and stages Z in shared
// memory (over the consumed A tile); the warps then write Z (training) and H_out = H + relu(Z)
// row by row, coalesced, or decode the rows. A wait that runs out sets bit 2 of *err and the
// block leaves.
// es: the encoder in shared memory, [w_0 of the 64 features][w_1][b] (kInEncode)
template <int kSrc>
__device__ __forceinline__ float4 layer_row(const LayerArgs& a, int64_t j, int q, const float* es, int32_t pj = -1) {
  if constexpr (kSrc == kInEncode) {
    const float2 f = *reinterpret_cast<const float2*>(a.F + 2 * j);
    const float4 w0 = *reinterpret_cast<const float4*>(es + 4 * q);
    const float4 w1 = *reinterpret_cast<const float4*>(es + kHid + 4 * q);
    const float4 b = *reinterpret_cast<const float4*>(es + 2 * kHid + 4 * q);
    return make_float4(fmaxf(w0.x * f.x + w1.x * f.y + b.x, 0.0f), fmaxf(w0.y * f.x + w1.y * f.y + b.y, 0.0f),
                       fmaxf(w0.z * f.x + w1.z * f.y + b.z, 0.0f), fmaxf(w0.w * f.x + w1.w * f.y + b.w, 0.0f));
  } else if constexpr (kSrc == kInParentB) {
    const float4 h = ld_bf16x4(a.Hb + j * kHid + 4 * q);
    const float4 u = ld4(a.U + (int64_t)(pj >= 0 ? pj : a.parent[j]) * kHid + 4 * q);
    return make_float4(h.x + u.x, h.y + u.y, h.z + u.z, h.w + u.w);
  } else if constexpr (kSrc == kInHb) {
    return ld_bf16x4(a.Hb + j * kHid + 4 * q);
  } else {
    return ld4(a.H + j * kHid + 4 * q);
  }
}

// (ptxas holds these at 64 registers a thread: four blocks an SM)
template <bool kCoarse, int kSrc>
__global__ void __launch_bounds__(kTileThreads)
k_layer_fwd(int64_t N, LayerArgs a, const int4* __restrict__ nbr, const float4* __restrict__ wn,
            const __nv_bfloat16* __restrict__ Wg, const float* __restrict__ bias, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ float bs[kHid];
  __shared__ float ds[kHid + 1];
  __shared__ __align__(16) float es[3 * kHid];
  __shared__ int4 snbr[2 * kTile];              // the tile's neighbour lists (fine: + the neighbours' parents)
  __shared__ int32_t sparent[kTile];             // the tile's rows' parents (kInParentB)
  __shared__ int s_fail;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  unsigned char* As = smem;
  unsigned char* Bs = smem + kFwdB;
  float* S = reinterpret_cast<float*>(smem);      // Z staging (128 x 64), over the A tile
  // W (the B operand: 64 outputs x 128 inputs), once per block
  for (int e = t; e < kHid * (kIn / 8); e += kTileThreads) {
    const int r = e / (kIn / 8), kc = e % (kIn / 8);
    *reinterpret_cast<uint4*>(Bs + sw_off(r, kc * 8, kHid)) =
        *reinterpret_cast<const uint4*>(Wg + r * kIn + kc * 8);
  }
  if (t < kHid) bs[t] = bias[t];
  if (a.dec && t <= kHid) ds[t] = a.dec[t];
  if (kSrc == kInEncode && t < kHid) {
    es[t] = a.enc[2 * t];
    es[kHid + t] = a.enc[2 * t + 1];
    es[2 * kHid + t] = a.enc[2 * kHid + t];
  }
  if (t == 0) {
    s_fail = 0;
    mbar_init(&mbar, 1);
  }
  if (warp == 0) tmem_alloc(&tmem_base, kHid);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const int erow = 32 * (warp & 3) + lane, ecol = 32 * (warp >> 2);   // epilogue: row, first column
  const uint32_t tld = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + ecol;
  const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
  const int q = lane & 15;                       // this lane's float4 of a row
  const int64_t ntiles = (N + kTile - 1) / kTile;
  uint32_t phase = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // the tile's neighbour lists (and parents) into shared memory in one coalesced pass, so
    // that each gather below waits on one global load (the rows) instead of an index first
    {
      const int64_t r0 = tile * kTile;
      if constexpr (kCoarse) {
        if (r0 + t / 2 < N) snbr[t] = nbr[2 * r0 + t];
      } else if (t < kTile) {
        if (r0 + t < N) snbr[t] = nbr[r0 + t];
      } else if constexpr (kSrc == kInParentB) {
        if (r0 + t - kTile < N) {
          snbr[t] = a.nparent[r0 + t - kTile];
          sparent[t - kTile] = a.parent[r0 + t - kTile];
        }
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int st = 0; st < 8; ++st) {
      const int r = 16 * warp + 2 * st + (lane >> 4);
      const int64_t cr = tile * kTile + r;
      float4 h = make_float4(0.f, 0.f, 0.f, 0.f), m = h;
      if (cr < N) {
        h = layer_row<kSrc>(a, cr, q, es, kSrc == kInParentB ? sparent[r] : -1);
        if constexpr (kCoarse) {
          const int4 na = snbr[2 * r], nb = snbr[2 * r + 1];
          const int ns[6] = {na.x, na.y, na.z, na.w, nb.x, nb.y};
#pragma unroll
          for (int j = 0; j < 6; ++j) {
            const float4 g = layer_row<kSrc>(a, ns[j], q, es);
            m.x += g.x - h.x; m.y += g.y - h.y; m.z += g.z - h.z; m.w += g.w - h.w;
          }
          const float sixth = 1.0f / 6.0f;
          m.x *= sixth; m.y *= sixth; m.z *= sixth; m.w *= sixth;
        } else {
          const int4 nb = snbr[r];
          const float4 w4 = wn[cr];
          const int4 np = kSrc == kInParentB ? snbr[kTile + r] : make_int4(-1, -1, -1, -1);
          const float4 g0 = layer_row<kSrc>(a, nb.x, q, es, np.x), g1 = layer_row<kSrc>(a, nb.y, q, es, np.y),
                       g2 = layer_row<kSrc>(a, nb.z, q, es, np.z), g3 = layer_row<kSrc>(a, nb.w, q, es, np.w);
          m.x = w4.x * (g0.x - h.x) + w4.y * (g1.x - h.x) + w4.z * (g2.x - h.x) + w4.w * (g3.x - h.x);
          m.y = w4.x * (g0.y - h.y) + w4.y * (g1.y - h.y) + w4.z * (g2.y - h.y) + w4.w * (g3.y - h.y);
          m.z = w4.x * (g0.z - h.z) + w4.y * (g1.z - h.z) + w4.z * (g2.z - h.z) + w4.w * (g3.z - h.z);
          m.w = w4.x * (g0.w - h.w) + w4.y * (g1.w - h.w) + w4.z * (g2.w - h.w) + w4.w * (g3.w - h.w);
        }
        if (a.M) st4(a.M + cr * kHid + 4 * q, m);
      }
      st_bf16x4(As + sw_off(r, 4 * q, kTile), h);
      st_bf16x4(As + sw_off(r, kHid + 4 * q, kTile), m);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < kIn / 16; ++kk)
        tc_mma(tmem, sw_desc(sw_kstep(a0, kk, kTile)), sw_desc(sw_kstep(b0, kk, kHid)), idesc_bf16(kTile, kHid),
               kk > 0);
      tc_commit(&mbar);
    }
    if (!mbar_wait(&mbar, phase)) s_fail = 1;
    phase ^= 1;
    __syncthreads();
    if (s_fail) break;
    tc_fence_after();
    {
      float z[32];
      tmem_ld32(tld, z);
#pragma unroll
      for (int j = 0; j < 32; j += 4) {
        const int col = ecol + j;
        st4(stage_at<16>(S, erow, col >> 2),
            make_float4(z[j] + bs[col], z[j + 1] + bs[col + 1], z[j + 2] + bs[col + 2], z[j + 3] + bs[col + 3]));
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int st = 0; st < 8; ++st) {
      const int r = 16 * warp + 2 * st + (lane >> 4);
      const int64_t cr = tile * kTile + r;
      float4 ho = make_float4(0.f, 0.f, 0.f, 0.f);
      if (cr < N) {
        const float4 zz = *reinterpret_cast<const float4*>(stage_at<16>(S, r, q));
        if (a.Z) st4(a.Z + cr * kHid + 4 * q, zz);
        const float4 hv = layer_row<kSrc>(a, cr, q, es, kSrc == kInParentB ? sparent[r] : -1);
        ho = make_float4(hv.x + fmaxf(zz.x, 0.0f), hv.y + fmaxf(zz.y, 0.0f), hv.z + fmaxf(zz.z, 0.0f),
                         hv.w + fmaxf(zz.w, 0.0f));
        if (!a.dec) {
          if (a.Houtb) st_bf16x4(reinterpret_cast<unsigned char*>(a.Houtb + cr * kHid + 4 * q), ho);
          else st4(a.Hout + cr * kHid + 4 * q, ho);
        }
      }
      if (a.dec) {                    // uniform over the block: every lane takes part
        float o = ds[4 * q] * ho.x + ds[4 * q + 1] * ho.y + ds[4 * q + 2] * ho.z + ds[4 * q + 3] * ho.w;
        o += __shfl_xor_sync(0xffffffffu, o, 8);
        o += __shfl_xor_sync(0xffffffffu, o, 4);
        o += __shfl_xor_sync(0xffffffffu, o, 2);
        o += __shfl_xor_sync(0xffffffffu, o, 1);
        if (q == 0 && cr < N) {
          // separately rounded product and difference: equal outputs cancel exactly
          const double v = __dmul_rn(a.scale, (double)(o + ds[kHid]));
          a.pred[cr] = a.mode == 0 ? v : __dsub_rn(a.pred[cr], v);
        }
      }
    }
    tc_fence_before();
    __syncthreads();      // accumulator read and staging consumed before the next tile
  }
  if (s_fail) {
    if (t == 0) atomicOr(err, 2);
    mbar_wait(&mbar, phase ^ 1);       // the tensor cores may still be writing: wait once more
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, kHid);
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

// Per-block sums over the block's cell range for the gradient partials: kRowGroups groups of
// 64 threads (one feature each) take every kRowGroups-th cell, then the group sums are
// added in group order.
constexpr int kRowGroups = 8;

// decoder gradient partials: part[b][w_dec] = sum dout (h_a - h_b); part[b][b_dec] = 0
__global__ void __launch_bounds__(kRowGroups * kHid)
k_decode_grad(int64_t N, const float* __restrict__ Ha, const float* __restrict__ Hb,
              const float* __restrict__ dout, float* __restrict__ part) {
  __shared__ float red[kRowGroups][kHid];
  const int64_t per = (N + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * per, hi = lo + per < N ? lo + per : N;
  const int g = threadIdx.x / kHid, o = threadIdx.x % kHid;
  float acc = 0.0f;
#pragma unroll 4
  for (int64_t i = lo + g; i < hi; i += kRowGroups) acc += dout[i] * (Ha[i * kHid + o] - Hb[i * kHid + o]);
  red[g][o] = acc;
  __syncthreads();
  float* p = part + (size_t)blockIdx.x * kNParams;
  if (threadIdx.x < kHid) {
    float t = 0.0f;
#pragma unroll
    for (int q = 0; q < kRowGroups; ++q) t += red[q][o];
    p[kOffWdec + o] = t;
  } else if (threadIdx.x == kHid) {
    p[kOffBdec] = 0.0f;
  }
}

// ---- one layer, backward with its weight gradients (tensor cores) ------------------------------
// Persistent: up to kGradBlocks blocks take tiles of 128 rows in turn (the same kernel for
// the fine and the aggregate layers: it reads only its tile's rows). Per tile, with
// dz = dH_next * (z > 0):
//  - data product [g_h ; g_m] = dz W_l (4 tcgen05.mma of K = 16 into tensor-memory columns
//    [0, 128)): dH = dH_next + g_h, G = g_m (its message is added by k_msg_add), written
//    row by row through a shared-memory staging of the accumulator;
//  - weight gradient dW_l^T += [h ; m]^T dz over the tile's cells (8 tcgen05.mma of K = 16 into
//    columns [128, 192), accumulated over all tiles of the block): both operands have the
//    cells as K, a lane per feature packing eight cells into one 16-byte row;
//  - bias gradient: sums of dz kept per lane in registers over the block's tiles.
// Operands are in the 128-byte swizzled K-major layout. At the end the block adds its
// partials to part[blockIdx.x] (weights [out][in], bias; zeroed before the backward, so the
// middle layer's applications at every level and hop accumulate there in launch order); the
// partials are summed over blocks in a fixed order later.
__global__ void __launch_bounds__(kTileThreads)
k_layer_bwd(int64_t N, const float* __restrict__ dHn, const float* __restrict__ Z,
            const float* __restrict__ Hin, const float* __restrict__ Min,
            const __nv_bfloat16* __restrict__ Wg, float* __restrict__ dH, float* __restrict__ G,
            float* __restrict__ part, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  __shared__ float red[16][kHid];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  unsigned char* B1 = smem;
  unsigned char* A1 = smem + kBwdA1;
  unsigned char* A2 = smem + kBwdA2;
  unsigned char* B2 = smem + kBwdB2;
  float* S = reinterpret_cast<float*>(smem + kBwdA1);   // 128 x 128 staging over A1, A2, B2
  // W^T (the data product's B operand: 128 inputs x 64 outputs): (n, k) = W[k][n]
  for (int e = t; e < kHid * kIn; e += kTileThreads) {
    const int k = e / kIn, n = e % kIn;
    *reinterpret_cast<__nv_bfloat16*>(B1 + sw_off(n, k, kIn)) = Wg[e];
  }
  if (t == 0) {
    s_fail = 0;
    mbar_init(&mbar, 1);
  }
  if (warp == 0) tmem_alloc(&tmem_base, 256);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t lanebase = (uint32_t)(32 * (warp & 3)) << 16;
  const int erow = 32 * (warp & 3) + lane;
  const uint32_t a1 = smem_u32(A1), b1 = smem_u32(B1), a2 = smem_u32(A2), b2 = smem_u32(B2);
  const int q = lane & 15;
  const int64_t ntiles = (N + kTile - 1) / kTile;
  float4 bacc = make_float4(0.f, 0.f, 0.f, 0.f);   // bias sums of features 4 q .. 4 q + 3
  uint32_t phase = 0;
  int ntile_done = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++ntile_done) {
    const int64_t c0 = tile * kTile;
    // A1 = dz (rows = cells): 16 lanes a row, two rows a step
#pragma unroll 4
    for (int st = 0; st < 8; ++st) {
      const int r = 16 * warp + 2 * st + (lane >> 4);
      const int64_t cr = c0 + r;
      float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
      if (cr < N) {
        const float4 dd = ld4(dHn + cr * kHid + 4 * q), z = ld4(Z + cr * kHid + 4 * q);
        d = make_float4(z.x > 0.0f ? dd.x : 0.0f, z.y > 0.0f ? dd.y : 0.0f, z.z > 0.0f ? dd.z : 0.0f,
                        z.w > 0.0f ? dd.w : 0.0f);
      }
      bacc.x += d.x; bacc.y += d.y; bacc.z += d.z; bacc.w += d.w;
      st_bf16x4(A1 + sw_off(r, 4 * q, kTile), d);
    }
    // A2 = [h ; m]^T and B2 = dz^T (rows = features, K = cells): a lane per feature, eight
    // cells packed into one 16-byte row; items (feature block of 32, group of 8 cells)
#pragma unroll 1
    for (int it = warp; it < 6 * 16; it += 8) {
      const int fb = it >> 4, cg = it & 15;      // fb 0..3: [h ; m] features, 4..5: dz outputs
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int64_t c = c0 + 8 * cg + j;
        float x = 0.0f;
        if (c < N) {
          if (fb < 2) x = Hin[c * kHid + 32 * fb + lane];
          else if (fb < 4) x = Min[c * kHid + 32 * (fb - 2) + lane];
          else {
            const int o = 32 * (fb - 4) + lane;
            const float dd = dHn[c * kHid + o];
            x = Z[c * kHid + o] > 0.0f ? dd : 0.0f;
          }
        }
        v[j] = x;
      }
      if (fb < 4) st_bf16x8(A2 + sw_off(32 * fb + lane, 8 * cg, kIn), v);
      else st_bf16x8(B2 + sw_off(32 * (fb - 4) + lane, 8 * cg, kHid), v);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < kHid / 16; ++kk)
        tc_mma(tmem, sw_desc(sw_kstep(a1, kk, kTile)), sw_desc(sw_kstep(b1, kk, kIn)), idesc_bf16(kTile, kIn),
               kk > 0);
#pragma unroll
      for (int kk = 0; kk < kTile / 16; ++kk)
        tc_mma(tmem + kIn, sw_desc(sw_kstep(a2, kk, kIn)), sw_desc(sw_kstep(b2, kk, kHid)), idesc_bf16(kIn, kHid),
               (ntile_done > 0 || kk > 0) ? 1 : 0);
      tc_commit(&mbar);
    }
    if (!mbar_wait(&mbar, phase)) s_fail = 1;
    phase ^= 1;
    __syncthreads();
    if (s_fail) break;
    tc_fence_after();
    // stage the data product (row per thread, warp halves: columns 0-63 / 64-127)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int col0 = 64 * (warp >> 2) + 32 * h;
      float v[32];
      tmem_ld32(tmem + lanebase + col0, v);
#pragma unroll
      for (int j = 0; j < 32; j += 4)
        st4(stage_at<32>(S, erow, (col0 + j) >> 2), make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]));
    }
    __syncthreads();
    // write back row by row: lanes 0-15 dH (= dH_next + g_h), lanes 16-31 G (= g_m)
#pragma unroll 4
    for (int st = 0; st < 16; ++st) {
      const int r = 16 * warp + st;
      const int64_t cr = c0 + r;
      if (cr < N) {
        const float4 v = *reinterpret_cast<const float4*>(stage_at<32>(S, r, lane));
        if (lane < 16) {
          const float4 dv = ld4(dHn + cr * kHid + 4 * lane);
          st4(dH + cr * kHid + 4 * lane, make_float4(dv.x + v.x, dv.y + v.y, dv.z + v.z, dv.w + v.w));
        } else {
          st4(G + cr * kHid + 4 * (lane - 16), v);
        }
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  if (s_fail) {
    if (t == 0) atomicOr(err, 2);
    mbar_wait(&mbar, phase ^ 1);
  }
  __syncthreads();
  tc_fence_after();
  // the block's partials: dW^T in columns [128, 192) (lane = input, column = output)
  float* p = part + (size_t)blockIdx.x * kNParams;
  if (!s_fail) {
    const int in = 32 * (warp & 3) + lane;
    const int o0 = 32 * (warp >> 2);
    float v[32];
    tmem_ld32(tmem + lanebase + kIn + o0, v);
    if (ntile_done > 0) {
#pragma unroll
      for (int j = 0; j < 32; ++j) p[(o0 + j) * kIn + in] += v[j];
    }
  }
  // bias: lanes q and q + 16 hold the same features for different rows
  bacc.x += __shfl_xor_sync(0xffffffffu, bacc.x, 16);
  bacc.y += __shfl_xor_sync(0xffffffffu, bacc.y, 16);
  bacc.z += __shfl_xor_sync(0xffffffffu, bacc.z, 16);
  bacc.w += __shfl_xor_sync(0xffffffffu, bacc.w, 16);
  if (lane < 16) {
    red[warp][4 * lane] = bacc.x;
    red[warp][4 * lane + 1] = bacc.y;
    red[warp][4 * lane + 2] = bacc.z;
    red[warp][4 * lane + 3] = bacc.w;
  }
  __syncthreads();
  if (t < kHid) {
    float b = 0.0f;
#pragma unroll
    for (int w = 0; w < 8; ++w) b += red[w][t];
    p[kHid * kIn + t] += b;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 256);
}

// dH_i += sum_j w_ij (G_j - G_i): the adjoint of the (symmetric) message operator; fine
// rows (four weighted face neighbours) or aggregate rows (six slots of weight 1/6, padded
// with the row itself)
template <bool kCoarse>
__global__ void k_msg_add(int64_t N, const float* __restrict__ Gm, const int4* __restrict__ nbr,
                          const float4* __restrict__ wn, float* __restrict__ dH) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < N; c += nwarps) {
    const float2 gi = *reinterpret_cast<const float2*>(Gm + c * kHid + 2 * lane);
    float mx = 0.0f, my = 0.0f;
    if constexpr (kCoarse) {
      const int4 na = nbr[2 * c], nb = nbr[2 * c + 1];
      const int ns[6] = {na.x, na.y, na.z, na.w, nb.x, nb.y};
#pragma unroll
      for (int s = 0; s < 6; ++s) {
        const float2 gn = *reinterpret_cast<const float2*>(Gm + (int64_t)ns[s] * kHid + 2 * lane);
        mx += gn.x - gi.x;
        my += gn.y - gi.y;
      }
      mx *= 1.0f / 6.0f;
      my *= 1.0f / 6.0f;
    } else {
      const int4 nb = nbr[c];
      const float4 w = wn[c];
      const int ns[4] = {nb.x, nb.y, nb.z, nb.w};
      const float ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const float2 gn = *reinterpret_cast<const float2*>(Gm + (int64_t)ns[s] * kHid + 2 * lane);
        mx += ws[s] * (gn.x - gi.x);
        my += ws[s] * (gn.y - gi.y);
      }
    }
    float2* d = reinterpret_cast<float2*>(dH + c * kHid + 2 * lane);
    const float2 dv = *d;
    *d = make_float2(dv.x + mx, dv.y + my);
  }
}

// ---- aggregate hierarchy: mean over aggregates, copy back ----------------------------------
// nparent[i][s] = parent[nbr[i][s]]: the level-1 aggregates of a cell's four neighbour slots
__global__ void k_neighbour_parents(int64_t n, const int4* __restrict__ nbr, const int32_t* __restrict__ parent,
                                    int4* __restrict__ nparent) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int4 b = nbr[i];
    nparent[i] = make_int4(parent[b.x], parent[b.y], parent[b.z], parent[b.w]);
  }
}


// out[a] = s_a sum over the nodes below of aggregate a (child_ptr / child_idx, ascending) of
// in[child], s_a = inv_count[a] (the mean) or 1 (inv_count null: the adjoint of the copy
// back); 16 lanes a row, a float4 of features each. The first kChildBatch child indices are
// read before any child's row, so those rows' loads are in flight together.
constexpr int kChildBatch = 8;
__device__ __forceinline__ float4 ld_row4(const float* p) { return ld4(p); }
__device__ __forceinline__ float4 ld_row4(const __nv_bfloat16* p) { return ld_bf16x4(p); }
template <typename Tin>
__global__ void k_child_sum(int64_t n, const int32_t* __restrict__ child_ptr, const int32_t* __restrict__ child_idx,
                            const Tin* __restrict__ in, const float* __restrict__ inv_count,
                            float* __restrict__ out) {
  const int q = threadIdx.x & 15;
  const int64_t row0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 4;
  const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 4;
  for (int64_t a = row0; a < n; a += stride) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const int32_t b = child_ptr[a], e = child_ptr[a + 1];
    for (int32_t k0 = b; k0 < e; k0 += kChildBatch) {
      int32_t c[kChildBatch];
#pragma unroll
      for (int j = 0; j < kChildBatch; ++j) c[j] = k0 + j < e ? child_idx[k0 + j] : -1;
      float4 v[kChildBatch];
#pragma unroll
      for (int j = 0; j < kChildBatch; ++j)
        v[j] = c[j] >= 0 ? ld_row4(in + (int64_t)c[j] * kHid + 4 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int j = 0; j < kChildBatch; ++j) {     // in child order
        acc.x += v[j].x; acc.y += v[j].y; acc.z += v[j].z; acc.w += v[j].w;
      }
    }
    if (inv_count) {
      const float s = inv_count[a];
      acc.x *= s; acc.y *= s; acc.z *= s; acc.w *= s;
    }
    st4(out + a * kHid + 4 * q, acc);
  }
}

// out[i] = a[i] + s_p b[p], p = parent[i], s_p = inv_count[p] or 1 (inv_count null): the copy
// back of the way up, and the adjoint of the mean; out may be a (same row, same thread).
// 16 lanes a row; each thread takes kParentRows rows, their loads issued together.
constexpr int kParentRows = 4;
__global__ void k_add_parent(int64_t n, const float* a, const float* __restrict__ b,
                             const int32_t* __restrict__ parent, const float* __restrict__ inv_count,
                             float* out) {
  const int q = threadIdx.x & 15;
  const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 4;   // row group
  const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x) >> 4;
  for (int64_t i0 = g; i0 < n; i0 += ngroups * kParentRows) {
    int32_t p[kParentRows];
    float4 x[kParentRows], y[kParentRows];
#pragma unroll
    for (int j = 0; j < kParentRows; ++j) {
      const int64_t i = i0 + j * ngroups;
      p[j] = i < n ? parent[i] : -1;
      x[j] = i < n ? ld4(a + i * kHid + 4 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < kParentRows; ++j)
      y[j] = p[j] >= 0 ? ld4(b + (int64_t)p[j] * kHid + 4 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < kParentRows; ++j) {
      const int64_t i = i0 + j * ngroups;
      if (i >= n) continue;
      const float sc = inv_count ? inv_count[p[j]] : 1.0f;
      st4(out + i * kHid + 4 * q, make_float4(x[j].x + sc * y[j].x, x[j].y + sc * y[j].y, x[j].z + sc * y[j].z,
                                             x[j].w + sc * y[j].w));
    }
  }
}

// encoder gradients: dz0 = dH0 * (z0 > 0); part[b][W_enc] = sum dz0 (x) f, part[b][b_enc] = sum dz0
__global__ void __launch_bounds__(kRowGroups * kHid)
k_encode_grad(int64_t N, const float* __restrict__ dH, const float* __restrict__ Z0,
              const float* __restrict__ F, float* __restrict__ part) {
  __shared__ float red[3][kRowGroups][kHid];
  const int64_t per = (N + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * per, hi = lo + per < N ? lo + per : N;
  const int g = threadIdx.x / kHid, o = threadIdx.x % kHid;
  float a0 = 0.0f, a1 = 0.0f, ab = 0.0f;
#pragma unroll 4
  for (int64_t c = lo + g; c < hi; c += kRowGroups) {
    const float d = Z0[c * kHid + o] > 0.0f ? dH[c * kHid + o] : 0.0f;
    const float2 f = *reinterpret_cast<const float2*>(F + 2 * c);
    a0 += d * f.x;
    a1 += d * f.y;
    ab += d;
  }
  red[0][g][o] = a0;
  red[1][g][o] = a1;
  red[2][g][o] = ab;
  __syncthreads();
  if (threadIdx.x < kHid) {
    float t0 = 0.0f, t1 = 0.0f, tb = 0.0f;
#pragma unroll
    for (int q = 0; q < kRowGroups; ++q) { t0 += red[0][q][o]; t1 += red[1][q][o]; tb += red[2][q][o]; }
    float* p = part + (size_t)blockIdx.x * kNParams;
    p[kOffWenc + 2 * o] = t0;
    p[kOffWenc + 2 * o + 1] = t1;
    p[kOffBenc + o] = tb;
  }
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
  const size_t NH = (size_t)n->N * kHid, CH = (size_t)n->n_coarse * kHid;
  cudaError_t e;
  for (int set = 0; set < 2; ++set) {
    if (set == 1 && (e = nalloc(n, &n->F[1], (size_t)n->N * 2))) return e;
    if ((e = nalloc(n, &n->Z0[set], NH))) return e;
    for (int l = 0; l < kLayers; l += n->n_lev > 0 ? 2 : 1) {   // the fine layers
      if ((e = nalloc(n, &n->M[set][l], NH))) return e;
      if ((e = nalloc(n, &n->Z[set][l], NH))) return e;
    }
    for (int l = 0; l <= kLayers; ++l)
      if ((e = nalloc(n, &n->H[set][l], NH))) return e;
    for (int j = 0; j < kHops && n->n_lev > 0; ++j) {
      if ((e = nalloc(n, &n->Mc[set][j], CH))) return e;
      if ((e = nalloc(n, &n->Zc[set][j], CH))) return e;
    }
    if (set == 1 && n->n_lev > 0)
      for (int j = 0; j <= kHops; ++j)
        if ((e = nalloc(n, &n->Hc[1][j], CH))) return e;
  }
  if ((e = nalloc(n, &n->dH, NH))) return e;
  if ((e = nalloc(n, &n->dHb, NH))) return e;
  if ((e = nalloc(n, &n->G, NH))) return e;
  if (n->n_lev > 0) {
    if ((e = nalloc(n, &n->dC, CH))) return e;
    if ((e = nalloc(n, &n->cP, (size_t)n->lev_n[0] * kHid))) return e;
    if ((e = nalloc(n, &n->cQ, (size_t)n->lev_n[0] * kHid))) return e;
  }
  if ((e = nalloc(n, &n->dout, n->N))) return e;
  if ((e = nalloc(n, &n->part, (size_t)2 * kGradBlocks * kNParams))) return e;
  n->train_buffers = true;
  return cudaSuccess;
}

// ---- aggregate hierarchy (host, at creation) ---------------------------------------------
// Per part, with [lo, hi] the bounding box of the part's cell centres and r_1 =
// max(1, round((n / 6)^(1/3))) boxes per axis, a cell's level-1 box index per axis is
// min(r_1 - 1, floor((x - lo) / (hi - lo) r_1)) (0 when hi = lo). Level k + 1 halves the box
// indices (r_{k+1} = ceil(r_k / 2)); levels continue while some part has r_k > 2, and stop
// early once every part is one box. Aggregates are the non-empty boxes, numbered part by
// part in increasing (x, y, z) index order; neighbours are the non-empty boxes sharing a
// face. The same FP64 operations as the oracle's rule, so both build the same hierarchy.
struct HostHierarchy {
  std::vector<int64_t> n;                      // nodes per level
  std::vector<std::vector<int32_t>> parent;    // per level: aggregate of each node below
  std::vector<std::vector<int32_t>> nbr;       // per level: [n][8] neighbours, padded with self
};

HostHierarchy build_hierarchy(const double* cen, int64_t N, const std::vector<int64_t>& pb) {
  const int P = (int)pb.size() - 1;
  HostHierarchy out;
  std::vector<int32_t> kc(3 * (size_t)N);      // box coordinates of the nodes below
  std::vector<int64_t> rad(P), below_begin(pb.begin(), pb.end());
  for (int p = 0; p < P; ++p) {
    const int64_t b = pb[p], e = pb[p + 1], np = e - b;
    const int64_t r = std::max<int64_t>(1, (int64_t)std::nearbyint(std::pow((double)np / 6.0, 1.0 / 3.0)));
    rad[p] = r;
    for (int a = 0; a < 3; ++a) {
      const double* x = cen + (size_t)a * N;
      double lo = x[b], hi = x[b];
      for (int64_t i = b; i < e; ++i) { lo = std::min(lo, x[i]); hi = std::max(hi, x[i]); }
      for (int64_t i = b; i < e; ++i) {
        int64_t k = 0;
        if (hi > lo) k = std::min<int64_t>(r - 1, (int64_t)std::floor((x[i] - lo) / (hi - lo) * (double)r));
        kc[3 * i + a] = (int32_t)k;
      }
    }
  }
  int64_t n_below = N;
  for (bool first = true;; first = false) {
    if (!first) {
      bool more = false;
      for (int p = 0; p < P; ++p) more |= rad[p] > 2;
      if (!more) break;
      for (auto& k : kc) k >>= 1;
      for (auto& r : rad) r = (r + 1) / 2;
    }
    std::vector<int32_t> parent(n_below), nbr;
    std::vector<int32_t> next_kc;
    std::vector<int64_t> next_begin(P + 1, 0);
    int64_t offset = 0;
    for (int p = 0; p < P; ++p) {
      const int64_t r = rad[p];
      std::vector<int64_t> rank((size_t)(r * r * r), -1);
      for (int64_t i = below_begin[p]; i < below_begin[p + 1]; ++i)
        rank[(size_t)((kc[3 * i] * r + kc[3 * i + 1]) * r + kc[3 * i + 2])] = 0;
      int64_t nb = 0;                              // present keys get ranks in key order
      for (auto& v : rank)
        if (v == 0) v = nb++;
      for (int64_t i = below_begin[p]; i < below_begin[p + 1]; ++i)
        parent[i] = (int32_t)(offset + rank[(size_t)((kc[3 * i] * r + kc[3 * i + 1]) * r + kc[3 * i + 2])]);
      for (int64_t key = 0; key < r * r * r; ++key) {
        if (rank[key] < 0) continue;
        const int64_t x = key / (r * r), y = (key / r) % r, z = key % r;
        const int64_t self = offset + rank[key];
        int32_t slots[8];
        int ns = 0;
        const int64_t d[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
        for (int q = 0; q < 6; ++q) {
          const int64_t nx = x + d[q][0], ny = y + d[q][1], nz = z + d[q][2];
          if (nx < 0 || ny < 0 || nz < 0 || nx >= r || ny >= r || nz >= r) continue;
          const int64_t rk = rank[(size_t)((nx * r + ny) * r + nz)];
          if (rk >= 0) slots[ns++] = (int32_t)(offset + rk);
        }
        while (ns < 8) slots[ns++] = (int32_t)self;
        nbr.insert(nbr.end(), slots, slots + 8);
        next_kc.push_back((int32_t)x);
        next_kc.push_back((int32_t)y);
        next_kc.push_back((int32_t)z);
      }
      next_begin[p] = offset;
      offset += nb;
    }
    next_begin[P] = offset;
    out.n.push_back(offset);
    out.parent.push_back(std::move(parent));
    out.nbr.push_back(std::move(nbr));
    kc = std::move(next_kc);
    below_begin = next_begin;
    n_below = offset;
    if (offset <= P || (int)out.n.size() == kMaxLevels) break;
  }
  return out;
}

// upload the hierarchy: parents, children (CSR, ascending), 1 / counts, neighbours
cudaError_t upload_hierarchy(MpnnNet* n, const HostHierarchy& h) {
  const int L = (int)h.n.size();
  n->n_lev = L;
  std::vector<int32_t> parent, cptr, cidx, nbr;
  std::vector<float> inv;
  int64_t off = 0, boff = 0, poff = 0;
  for (int k = 0; k < L; ++k) {
    const int64_t nk = h.n[k];
    const std::vector<int32_t>& par = h.parent[k];
    n->lev_n[k] = nk;
    n->lev_off[k] = off;
    n->below_off[k] = boff;
    n->ptr_off[k] = poff;
    std::vector<int32_t> cnt(nk + 1, 0);
    for (int32_t a : par) cnt[a + 1] += 1;
    for (int64_t a = 0; a < nk; ++a) {
      inv.push_back(1.0f / (float)cnt[a + 1]);
      cnt[a + 1] += cnt[a];
    }
    std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1), idx(par.size());
    for (size_t i = 0; i < par.size(); ++i) idx[fill[par[i]]++] = (int32_t)i;
    parent.insert(parent.end(), par.begin(), par.end());   // level-local aggregate indices
    cptr.insert(cptr.end(), cnt.begin(), cnt.end());
    cidx.insert(cidx.end(), idx.begin(), idx.end());
    nbr.insert(nbr.end(), h.nbr[k].begin(), h.nbr[k].end());
    off += nk;
    boff += (int64_t)par.size();
    poff += nk + 1;
  }
  n->lev_off[L] = off;
  n->below_off[L] = boff;
  n->n_coarse = off;
  cudaError_t e;
  if ((e = nalloc(n, &n->parent, parent.size()))) return e;
  if ((e = nalloc(n, &n->child_ptr, cptr.size()))) return e;
  if ((e = nalloc(n, &n->child_idx, cidx.size()))) return e;
  if ((e = nalloc(n, &n->inv_count, inv.size()))) return e;
  if ((e = nalloc(n, &n->cnbr, nbr.size()))) return e;
  if ((e = cudaMemcpy(n->parent, parent.data(), parent.size() * 4, cudaMemcpyHostToDevice))) return e;
  if ((e = cudaMemcpy(n->child_ptr, cptr.data(), cptr.size() * 4, cudaMemcpyHostToDevice))) return e;
  if ((e = cudaMemcpy(n->child_idx, cidx.data(), cidx.size() * 4, cudaMemcpyHostToDevice))) return e;
  if ((e = cudaMemcpy(n->inv_count, inv.data(), inv.size() * 4, cudaMemcpyHostToDevice))) return e;
  return cudaMemcpy(n->cnbr, nbr.data(), nbr.size() * 4, cudaMemcpyHostToDevice);
}

// grid of the forward layer kernel over ``rows``: persistent over 128-row tiles, as many
// blocks as fit on the SMs (48 KB shared memory and 64 tensor-memory columns a block, up to
// four an SM); the backward runs up to kGradBlocks blocks (80 KB and 256 columns a block,
// two an SM)
unsigned fwd_grid(const MpnnNet* n, int64_t rows) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((rows + kTile - 1) / kTile, (int64_t)n->m->num_sms * 4));
}
unsigned bwd_grid(int64_t rows) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((rows + kTile - 1) / kTile, kGradBlocks));
}
unsigned row16_grid(int64_t rows) { return grid_n(rows * 16); }
// k_add_parent: kParentRows rows a 16-lane group, about eight 256-thread blocks an SM at most
unsigned parent_grid(const MpnnNet* n, int64_t rows) {
  const int64_t groups = (rows + kParentRows - 1) / kParentRows;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((groups * 16 + 255) / 256, (int64_t)n->m->num_sms * 8));
}

// dynamic shared memory above 48 KB must be enabled per kernel (current device)
cudaError_t layer_kernels_setup() {
  const void* fwd[] = {(const void*)k_layer_fwd<false, kInH>, (const void*)k_layer_fwd<true, kInH>,
                       (const void*)k_layer_fwd<false, kInEncode>, (const void*)k_layer_fwd<false, kInHb>,
                       (const void*)k_layer_fwd<false, kInParentB>};
  for (const void* f : fwd) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
    if (e != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute(k_layer_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem);
}

// level-local views of the hierarchy arrays
const int32_t* lev_parent(const MpnnNet* n, int k) { return n->parent + n->below_off[k]; }
const int32_t* lev_child_ptr(const MpnnNet* n, int k) { return n->child_ptr + n->ptr_off[k]; }
const int32_t* lev_child_idx(const MpnnNet* n, int k) { return n->child_idx + n->below_off[k]; }
const float* lev_inv(const MpnnNet* n, int k) { return n->inv_count + n->lev_off[k]; }
const int4* lev_nbr(const MpnnNet* n, int k) {
  return reinterpret_cast<const int4*>(n->cnbr + (size_t)8 * n->lev_off[k]);
}
float* rows_at(float* base, const MpnnNet* n, int k) { return base ? base + (size_t)n->lev_off[k] * kHid : nullptr; }

// one forward layer launch over ``rows`` rows (fine: face neighbours and weights; coarse:
// the level's aggregate neighbours)
template <bool kCoarse, int kSrc>
void launch_layer(MpnnNet* n, int l, int64_t rows, const LayerArgs& a, const int4* nb, cudaStream_t s) {
  const __nv_bfloat16* W = n->wbf + (size_t)l * kHid * kIn;
  const float* b = n->theta + kOffLayer0 + l * kLayerSize + kHid * kIn;
  const float4* wn = kCoarse ? nullptr : reinterpret_cast<const float4*>(n->wn);
  k_layer_fwd<kCoarse, kSrc><<<fwd_grid(n, rows), kTileThreads, kFwdSmem, s>>>(rows, a, nb, wn, W, b, n->m->d_status);
  count_launch();
}

LayerArgs hidden_io(const float* H, float* M, float* Z, float* Hout) {
  LayerArgs a;
  a.H = H;
  a.M = M;
  a.Z = Z;
  a.Hout = Hout;
  return a;
}

// the aggregate levels of one evaluation: down (mean of the level below, then kHops middle
// layers, keeping messages and pre-activations when M / Z are given), then up to level 0:
// every level's output adds its aggregate's (the cells' copy back is left to the caller)
void levels_forward(MpnnNet* n, const float* h1, const __nv_bfloat16* h1b, float* const* Hc, float* const* Mc,
                    float* const* Zc, cudaStream_t s) {
  for (int k = 0; k < n->n_lev; ++k) {
    const int64_t nk = n->lev_n[k];
    if (k == 0 && h1b)
      k_child_sum<__nv_bfloat16><<<row16_grid(nk), 256, 0, s>>>(nk, lev_child_ptr(n, k), lev_child_idx(n, k), h1b,
                                                                lev_inv(n, k), rows_at(Hc[0], n, k));
    else
      k_child_sum<float><<<row16_grid(nk), 256, 0, s>>>(nk, lev_child_ptr(n, k), lev_child_idx(n, k),
                                                        k == 0 ? h1 : rows_at(Hc[kHops], n, k - 1), lev_inv(n, k),
                                                        rows_at(Hc[0], n, k));
    count_launch();
    for (int j = 0; j < kHops; ++j)
      launch_layer<true, kInH>(n, 1, nk,
                               hidden_io(rows_at(Hc[j], n, k), Mc ? rows_at(Mc[j], n, k) : nullptr,
                                         Zc ? rows_at(Zc[j], n, k) : nullptr, rows_at(Hc[j + 1], n, k)),
                               lev_nbr(n, k), s);
  }
  for (int k = n->n_lev - 1; k >= 1; --k) {
    float* up = rows_at(Hc[kHops], n, k - 1);
    k_add_parent<<<parent_grid(n, n->lev_n[k - 1]), 256, 0, s>>>(n->lev_n[k - 1], up, rows_at(Hc[kHops], n, k),
                                                            lev_parent(n, k), nullptr, up);
    count_launch();
  }
}

// One training evaluation of the network into activation set ``set`` (every layer's input,
// messages and pre-activations kept for the backward: H[set][0..3], Hc/Mc/Zc[set]).
// zero_charge: f0 = 0.
cudaError_t forward(MpnnNet* n, int set, const double* dq, const double* phi, bool zero_charge, cudaStream_t s) {
  fvgb_mesh m = n->m;
  const int64_t N = n->N;
  constexpr double kEoverEps0 = 1.602176634e-19 / 8.8541878128e-12;
  float** H = n->H[set];
  k_features<<<grid_n(N), 256, 0, s>>>(N, dq, phi, n->hcell, kEoverEps0 / (n->V * n->s0),
                                       1.0 / (n->V * n->s1), zero_charge ? 1 : 0, n->F[set]);
  k_encode<<<grid_n(N * kHid), 256, 0, s>>>(N, n->F[set], n->theta, n->Z0[set], H[0]);
  count_launch(2);
  const int4* nbr = reinterpret_cast<const int4*>(m->g64.bc[n->bcset].at_nbr);
  launch_layer<false, kInH>(n, 0, N, hidden_io(H[0], n->M[set][0], n->Z[set][0], H[1]), nbr, s);
  if (n->n_lev == 0) {
    launch_layer<false, kInH>(n, 1, N, hidden_io(H[1], n->M[set][1], n->Z[set][1], H[2]), nbr, s);
  } else {
    levels_forward(n, H[1], nullptr, n->Hc[set], n->Mc[set], n->Zc[set], s);
    k_add_parent<<<parent_grid(n, N), 256, 0, s>>>(N, H[1], rows_at(n->Hc[set][kHops], n, 0), lev_parent(n, 0), nullptr,
                                               H[2]);
    count_launch();
  }
  launch_layer<false, kInH>(n, 2, N, hidden_io(H[2], n->M[set][2], n->Z[set][2], H[3]), nbr, s);
  return cudaGetLastError();
}

// One inference evaluation, decoded into pred (mode 0: pred = V s2 N(f); mode 1: pred -=
// V s2 N(f)). The encoder runs inside layer 0's gathers, the cells' copy back of the
// hierarchy inside layer 2's, and the decoder in layer 2's epilogue: the cells' hidden
// states are written once, as BF16 (h1; h2 too for the local architecture).
cudaError_t forward_infer(MpnnNet* n, const double* dq, const double* phi, bool zero_charge, double* pred,
                          int mode, cudaStream_t s) {
  fvgb_mesh m = n->m;
  const int64_t N = n->N;
  constexpr double kEoverEps0 = 1.602176634e-19 / 8.8541878128e-12;
  k_features<<<grid_n(N), 256, 0, s>>>(N, dq, phi, n->hcell, kEoverEps0 / (n->V * n->s0),
                                       1.0 / (n->V * n->s1), zero_charge ? 1 : 0, n->F[0]);
  count_launch();
  const int4* nbr = reinterpret_cast<const int4*>(m->g64.bc[n->bcset].at_nbr);
  __nv_bfloat16* h1 = n->Hb[0];
  LayerArgs a0;
  a0.F = n->F[0];
  a0.enc = n->theta + kOffWenc;
  a0.Houtb = h1;
  launch_layer<false, kInEncode>(n, 0, N, a0, nbr, s);
  LayerArgs a2;
  a2.dec = n->theta + kOffWdec;
  a2.scale = n->V * n->s2;
  a2.mode = mode;
  a2.pred = pred;
  if (n->n_lev == 0) {
    LayerArgs a1;
    a1.Hb = h1;
    a1.Houtb = n->Hb[1];
    launch_layer<false, kInHb>(n, 1, N, a1, nbr, s);
    a2.Hb = n->Hb[1];
    launch_layer<false, kInHb>(n, 2, N, a2, nbr, s);
  } else {
    levels_forward(n, nullptr, h1, n->Hc[0], nullptr, nullptr, s);
    a2.Hb = h1;
    a2.U = rows_at(n->Hc[0][kHops], n, 0);
    a2.parent = lev_parent(n, 0);
    a2.nparent = reinterpret_cast<const int4*>(n->nparent);
    launch_layer<false, kInParentB>(n, 2, N, a2, nbr, s);
  }
  return cudaGetLastError();
}

// prediction dphi = V s2 (N(f) - N(f0 = 0))
cudaError_t predict(MpnnNet* n, const double* dq, const double* phi, double* dphi, cudaStream_t s) {
  cudaError_t e;
  if ((e = forward_infer(n, dq, phi, false, dphi, 0, s))) return e;
  return forward_infer(n, dq, phi, true, dphi, 1, s);
}

// backward of sum_i dout_i sign N_set(f)_i through the layers, the hierarchy and the encoder
// into the gradient partial rows [row0, row0 + kGradBlocks) (zeroed by the caller)
void backward_set(MpnnNet* n, int set, float sign, int row0, cudaStream_t s) {
  const int64_t N = n->N;
  float* part = n->part + (size_t)row0 * kNParams;
  const int4* nbr = reinterpret_cast<const int4*>(n->m->g64.bc[n->bcset].at_nbr);
  const float4* wn = reinterpret_cast<const float4*>(n->wn);
  int* err = n->m->d_status;
  auto layer_back = [&](int l, int64_t rows, const float* dHn, const float* Z, const float* Hin, const float* Min,
                        float* dHo, bool coarse, const int4* nb) {
    k_layer_bwd<<<bwd_grid(rows), kTileThreads, kBwdSmem, s>>>(rows, dHn, Z, Hin, Min, n->wbf + (size_t)l * kHid * kIn,
                                                               dHo, n->G, part + kOffLayer0 + l * kLayerSize, err);
    if (coarse) k_msg_add<true><<<grid_n(rows * 32), 256, 0, s>>>(rows, n->G, nb, nullptr, dHo);
    else k_msg_add<false><<<grid_n(rows * 32), 256, 0, s>>>(rows, n->G, nb, wn, dHo);
    count_launch(2);
  };
  k_head_dh<<<grid_n(N * kHid), 256, 0, s>>>(N, n->dout, n->theta, sign, n->dH);
  count_launch();
  // layer 2: d h3 (dH) -> d h2 (dHb)
  layer_back(2, N, n->dH, n->Z[set][2], n->H[set][2], n->M[set][2], n->dHb, false, nbr);
  float* X = n->dHb;
  if (n->n_lev == 0) {
    // local: layer 1, d h2 (dHb) -> d h1 (dH); layer 0, -> d h0 (dHb)
    layer_back(1, N, X, n->Z[set][1], n->H[set][1], n->M[set][1], n->dH, false, nbr);
    layer_back(0, N, n->dH, n->Z[set][0], n->H[set][0], n->M[set][0], n->dHb, false, nbr);
    k_encode_grad<<<kGradBlocks, kRowGroups * kHid, 0, s>>>(N, n->dHb, n->Z0[set], n->F[set], part);
    count_launch();
    return;
  }
  // adjoint of the way up: the output of level k receives the sum over its nodes of theirs
  const int L = n->n_lev;
  k_child_sum<float><<<row16_grid(n->lev_n[0]), 256, 0, s>>>(n->lev_n[0], lev_child_ptr(n, 0), lev_child_idx(n, 0), X,
                                                      nullptr, rows_at(n->dC, n, 0));
  count_launch();
  for (int k = 1; k < L; ++k) {
    k_child_sum<float><<<row16_grid(n->lev_n[k]), 256, 0, s>>>(n->lev_n[k], lev_child_ptr(n, k), lev_child_idx(n, k),
                                                        rows_at(n->dC, n, k - 1), nullptr, rows_at(n->dC, n, k));
    count_launch();
  }
  // adjoint of the way down, coarsest level first: the hops in reverse, then the mean
  for (int k = L - 1; k >= 0; --k) {
    const int64_t nk = n->lev_n[k];
    const float* cur = rows_at(n->dC, n, k);
    for (int j = kHops - 1; j >= 0; --j) {
      float* nxt = (j % 2 == (kHops - 1) % 2) ? n->cP : n->cQ;
      layer_back(1, nk, cur, rows_at(n->Zc[set][j], n, k), rows_at(n->Hc[set][j], n, k), rows_at(n->Mc[set][j], n, k),
                 nxt, true, lev_nbr(n, k));
      cur = nxt;
    }
    float* down = k > 0 ? rows_at(n->dC, n, k - 1) : X;
    const int64_t nb = k > 0 ? n->lev_n[k - 1] : N;
    k_add_parent<<<parent_grid(n, nb), 256, 0, s>>>(nb, down, cur, lev_parent(n, k), lev_inv(n, k), down);
    count_launch();
  }
  // layer 0: d h1 (dHb) -> d h0 (dH)
  layer_back(0, N, X, n->Z[set][0], n->H[set][0], n->M[set][0], n->dH, false, nbr);
  k_encode_grad<<<kGradBlocks, kRowGroups * kHid, 0, s>>>(N, n->dH, n->Z0[set], n->F[set], part);
  count_launch();
}

// loss and gradient into n->grad (and n->dloss)
cudaError_t loss_grad(MpnnNet* n, const double* dq, const double* phi, const double* target, cudaStream_t s) {
  cudaError_t e;
  if ((e = alloc_train(n))) return e;
  if ((e = forward(n, 0, dq, phi, false, s))) return e;
  if ((e = forward(n, 1, dq, phi, true, s))) return e;
  const int64_t N = n->N;
  const int G = kGradBlocks;
  if ((e = cudaMemsetAsync(n->part, 0, (size_t)2 * G * kNParams * sizeof(float), s))) return e;
  k_head_train<<<G, 256, 0, s>>>(N, n->H[0][kLayers], n->H[1][kLayers], n->theta, n->V * n->s2, target,
                                 n->dout, n->dpart);
  k_reduce_loss<<<1, 32, 0, s>>>(G, n->dpart, n->dloss);
  k_decode_grad<<<G, kRowGroups * kHid, 0, s>>>(N, n->H[0][kLayers], n->H[1][kLayers], n->dout, n->part);
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

fvgb_status fvgb_mpnn_create(fvgb_mesh m, int32_t bcset, int32_t multilevel, fvgb_mpnn* out) {
  if (!m || !out) { set_error("null argument"); return FVGB_EINVAL; }
  *out = nullptr;
  if (bcset < 0 || bcset >= (int32_t)m->g64.bc.size()) { set_error("bcset index out of range"); return FVGB_EINVAL; }
  if (m->topo.dim != 3 || m->topo.N < 1) { set_error("the network needs a non-empty 3D mesh"); return FVGB_EINVAL; }
  if (multilevel != 0 && multilevel != 1) { set_error("multilevel must be 0 or 1"); return FVGB_EINVAL; }
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
  if ((e = layer_kernels_setup())) return fail("tensor-core kernel attributes");
  if ((e = nalloc(n, &n->theta, kNParams))) return fail("allocation");
  if ((e = nalloc(n, &n->adam_m, kNParams))) return fail("allocation");
  if ((e = nalloc(n, &n->adam_v, kNParams))) return fail("allocation");
  if ((e = nalloc(n, &n->grad, kNParams))) return fail("allocation");
  if ((e = nalloc(n, &n->wbf, (size_t)kLayers * kHid * kIn))) return fail("allocation");
  if ((e = nalloc(n, &n->wn, (size_t)n->N * 4))) return fail("allocation");
  if ((e = nalloc(n, &n->F[0], (size_t)n->N * 2))) return fail("allocation");
  if ((e = nalloc(n, &n->hcell, (size_t)n->N))) return fail("allocation");
  if ((e = nalloc(n, &n->Hb[0], NH))) return fail("allocation");
  if (!multilevel && (e = nalloc(n, &n->Hb[1], NH))) return fail("allocation");
  k_cell_size<<<grid_n(n->N), 256>>>(n->N, m->g64.vol, n->hcell);
  count_launch();
  if (multilevel) {
    std::vector<double> cen((size_t)3 * n->N);
    if ((e = cudaMemcpy(cen.data(), m->g64.cen, cen.size() * sizeof(double), cudaMemcpyDeviceToHost)))
      return fail("centre copy");
    if ((e = upload_hierarchy(n, build_hierarchy(cen.data(), n->N, m->part_cell_begin))))
      return fail("aggregate hierarchy");
  }
  for (int j = 0; j <= kHops && n->n_lev > 0; ++j)
    if ((e = nalloc(n, &n->Hc[0][j], (size_t)n->n_coarse * kHid))) return fail("allocation");
  if (n->n_lev > 0) {
    if ((e = nalloc(n, &n->nparent, (size_t)4 * n->N))) return fail("allocation");
    k_neighbour_parents<<<grid_n(n->N), 256>>>(n->N, reinterpret_cast<const int4*>(m->g64.bc[bcset].at_nbr),
                                               n->parent, reinterpret_cast<int4*>(n->nparent));
    count_launch();
  }
  if ((e = nalloc(n, &n->dloss, 2))) return fail("allocation");
  if ((e = cudaMallocHost((void**)&n->hloss, sizeof(double)))) return fail("pinned allocation");
  if ((e = cudaMemset(n->theta, 0, kNParams * sizeof(float)))) return fail("memset");
  if ((e = cudaMemset(n->adam_m, 0, kNParams * sizeof(float)))) return fail("memset");
  if ((e = cudaMemset(n->adam_v, 0, kNParams * sizeof(float)))) return fail("memset");
  if ((e = cudaMemset(n->wbf, 0, (size_t)kLayers * kHid * kIn * sizeof(__nv_bfloat16)))) return fail("memset");
  // message weights: c1 of the interior faces (two-point coefficients of bcset), / max
  const double* coef = m->g64.bc[bcset].at_coef;
  if ((e = nalloc(n, &n->dpart, kGradBlocks))) return fail("allocation");
  k_max_coef<<<kGradBlocks, 256>>>(4 * n->N, coef, n->dpart);
  k_max_coef<<<1, 256>>>(kGradBlocks, n->dpart, n->dloss + 1);
  k_msg_weights<<<grid_n(4 * n->N), 256>>>(4 * n->N, coef, n->dloss + 1, n->wn);
  count_launch(3);
  if ((e = cudaDeviceSynchronize())) return fail("message weights");
  *out = n;
  return FVGB_OK;
}

fvgb_status fvgb_mpnn_hierarchy(int64_t n_cell, const double* cen, int32_t n_part, const int64_t* part_begin,
                                int32_t* n_levels, int64_t* level_n, int32_t* parent, int32_t* nbr) {
  if (n_cell < 1 || !cen || n_part < 1 || !part_begin || !n_levels || !level_n) {
    set_error("bad arguments");
    return FVGB_EINVAL;
  }
  std::vector<int64_t> pb(part_begin, part_begin + n_part + 1);
  if (pb[0] != 0 || pb[n_part] != n_cell) { set_error("part ranges must cover the cells"); return FVGB_EINVAL; }
  for (int p = 0; p < n_part; ++p)
    if (pb[p + 1] <= pb[p]) { set_error("empty or decreasing part range"); return FVGB_EINVAL; }
  for (int64_t i = 0; i < 3 * n_cell; ++i)
    if (!std::isfinite(cen[i])) { set_error("non-finite centre"); return FVGB_EINVAL; }
  const HostHierarchy h = build_hierarchy(cen, n_cell, pb);
  *n_levels = (int32_t)h.n.size();
  for (size_t k = 0; k < h.n.size(); ++k) level_n[k] = h.n[k];
  for (size_t k = 0; k < h.n.size(); ++k) {
    if (parent) parent = std::copy(h.parent[k].begin(), h.parent[k].end(), parent);
    if (nbr) nbr = std::copy(h.nbr[k].begin(), h.nbr[k].end(), nbr);
  }
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
