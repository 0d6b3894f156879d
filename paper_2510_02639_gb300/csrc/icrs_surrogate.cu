// Learned surrogate of the finite-source correction, gated back to ICRS.
//
// Not in the paper: a small MLP predicts the part of y = 1e4 log(A_ICRS/A_PS)
// that a second-order finite-source estimate b (from point-source
// magnifications on the source limb) misses, from 7 features of an epoch,
// with a log-variance output; an error gate sends every epoch whose predicted
// uncertainty, correction size or caustic proximity is too large (or whose
// point-source solves are flagged) back to full ICRS.
//
//   network   7 -> 128 -> 128 -> 128 -> 128 -> 2, SiLU on the hidden layers
//   numerics  BF16 weights, inputs and inter-layer activations; FP32
//             accumulation in tensor memory (tcgen05.mma kind::f16); FP32
//             master weights and Adam moments; in the backward pass each
//             layer's upstream gradient dZ is rounded to BF16 before its
//             three contractions (dW = dZ^T X, db = sum dZ, dX = dZ W)
//   loss      Gaussian NLL 1/2 [(y - mu)^2 e^{-s} + s], mean over the batch
//   features  (w_c.x, w_c.y, log10 s, (log10 q + 3)/2, log10 rho + 3,
//             4 (u1 - 0.55), clamp(log10 min_j |det J(z_j)|, -6, 1)), the
//             minimum over the point-source images z_j at the source centre
//             and at eight points of the source limb
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "icrs.h"
#include "icrs_common.cuh"
#include "icrs_ps.cuh"
#include "icrs_tc.cuh"

namespace icrs {
namespace sg {

constexpr int NIN = 7, H = 128, NOUT = 2;
constexpr int KIN = 16;    // layer-0 contraction, padded (one MMA K-step)
constexpr int NOUTP = 16;  // layer-4 outputs, padded (smallest N for M = 128)
constexpr int TM = 128;    // samples per tile (the MMA M)
constexpr int NT = 128;    // threads: one per tile row / TMEM lane
constexpr int NPARAM = ICRS_MLP_NPARAM;

// offsets in the FP32 parameter vector (row-major [out][in] weights)
constexpr int OW0 = 0, OB0 = OW0 + H * NIN;
constexpr int OW1 = OB0 + H, OB1 = OW1 + H * H;
constexpr int OW2 = OB1 + H, OB2 = OW2 + H * H;
constexpr int OW3 = OB2 + H, OB3 = OW3 + H * H;
constexpr int OW4 = OB3 + H, OB4 = OW4 + NOUT * H;
static_assert(OB4 + NOUT == NPARAM, "parameter count");

__host__ __device__ constexpr int w_off(int l) { return l == 0 ? OW0 : l == 1 ? OW1 : l == 2 ? OW2 : l == 3 ? OW3 : OW4; }
__host__ __device__ constexpr int b_off(int l) { return l == 0 ? OB0 : l == 1 ? OB1 : l == 2 ? OB2 : l == 3 ? OB3 : OB4; }

// packed BF16 operand tiles (bytes), each in the K-major no-swizzle layout
constexpr int PB_W0 = 0;                       // W0   [128][16]
constexpr int PB_W1 = PB_W0 + H * KIN * 2;     // W1..W3 [128][128]
constexpr int PB_W4 = PB_W1 + 3 * H * H * 2;   // W4   [16][128]
constexpr int PB_FWD = PB_W4 + NOUTP * H * 2;  // end of the forward tiles
constexpr int PB_W1T = PB_FWD;                 // W1^T..W3^T [128][128]
constexpr int PB_W4T = PB_W1T + 3 * H * H * 2; // W4^T [128][16]
constexpr int PACK_BYTES = PB_W4T + H * NOUTP * 2;
static_assert(PACK_BYTES == ICRS_MLP_PACK_BYTES, "pack size");

constexpr int WAIT_TRIES = 1 << 20;  // bounded mbarrier waits

// ---------------------------------------------------------------- packing
// One thread per 16-byte chunk (8 BF16 of one tile row).
__global__ void pack_kernel(const float* __restrict__ theta, uint8_t* __restrict__ pack) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= PACK_BYTES / 16) return;
  const int byte = c * 16;
  int base, K, l;
  bool tr;
  if (byte < PB_W1) { base = PB_W0; K = KIN; l = 0; tr = false; }
  else if (byte < PB_W4) { int j = (byte - PB_W1) / (H * H * 2); base = PB_W1 + j * H * H * 2; K = H; l = 1 + j; tr = false; }
  else if (byte < PB_W1T) { base = PB_W4; K = H; l = 4; tr = false; }
  else if (byte < PB_W4T) { int j = (byte - PB_W1T) / (H * H * 2); base = PB_W1T + j * H * H * 2; K = H; l = 1 + j; tr = true; }
  else { base = PB_W4T; K = NOUTP; l = 4; tr = true; }
  const int o = byte - base;
  const int rg = o / (16 * K), rem = o % (16 * K);
  const int r = rg * 8 + (rem % 128) / 16, k0 = (rem / 128) * 8;
  const int nout = l == 4 ? NOUT : H, nin = l == 0 ? NIN : H;
  __align__(16) __nv_bfloat16 v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int k = k0 + i;
    const int no = tr ? k : r;  // output neuron
    const int ni = tr ? r : k;  // input index
    const float x = (no < nout && ni < nin) ? theta[w_off(l) + no * nin + ni] : 0.0f;
    v[i] = __float2bfloat16_rn(x);
  }
  *reinterpret_cast<uint4*>(pack + byte) = *reinterpret_cast<const uint4*>(v);
}

__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float silu_prime(float z) {
  const float sg = 1.0f / (1.0f + expf(-z));
  return sg * (1.0f + z * (1.0f - sg));
}

__device__ __forceinline__ void store8(uint8_t* dst, const float* x) {
  __align__(16) __nv_bfloat16 h[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) h[i] = __float2bfloat16_rn(x[i]);
  *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(h);
}

__device__ __forceinline__ void copy16(uint8_t* dst, const uint8_t* src, int bytes, int tid) {
  for (int i = tid; i < bytes / 16; i += NT)
    reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(src)[i];
}

// Issue D = A B^T over K (multiple of 16) from K-major tiles: thread 0 only.
__device__ __forceinline__ void issue_gemm(uint32_t d_tmem, uint32_t a_smem, uint32_t b_smem, int K, int N, bool acc0) {
  const uint32_t id = tc::idesc_bf16(TM, N);
  for (int ks = 0; ks < K / 16; ++ks) {
    const uint64_t ad = tc::smem_desc(a_smem + ks * 256, 128, 16 * K);
    const uint64_t bd = tc::smem_desc(b_smem + ks * 256, 128, 16 * K);
    tc::mma_bf16(d_tmem, ad, bd, id, (ks > 0 || acc0) ? 1u : 0u);
  }
}

// Layer-0 input row: the 7 features rounded to BF16, zero padded to 16.
__device__ __forceinline__ void load_input_row(const float* __restrict__ feat, int q, int n, float* f) {
#pragma unroll
  for (int i = 0; i < 16; ++i) f[i] = 0.0f;
  if (q < n) {
    const float4 a = reinterpret_cast<const float4*>(feat + (size_t)q * 8)[0];
    const float4 b = reinterpret_cast<const float4*>(feat + (size_t)q * 8)[1];
    f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w; f[4] = b.x; f[5] = b.y; f[6] = b.z;
  }
}

// ---------------------------------------------------------------- inference
// Persistent: every CTA keeps the forward tiles (106,496 B) in shared memory
// and walks tiles of 128 queries.  Per layer: one thread issues the MMAs,
// all 128 threads read their row from TMEM, add the bias, apply SiLU and
// write the next layer's BF16 operand.
constexpr int INF_SMEM = PB_FWD + H * KIN * 2 + H * H * 2;

__global__ void __launch_bounds__(NT, 1)
mlp_infer_kernel(const uint8_t* __restrict__ pack, const float* __restrict__ theta, const float* __restrict__ feat,
                 int n, float* __restrict__ out, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t* Wf = sm;                    // W0 | W1 | W2 | W3 | W4 as packed
  uint8_t* X0 = sm + PB_FWD;           // [128][16]
  uint8_t* X = X0 + H * KIN * 2;       // [128][128]
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_sh;
  const int tid = threadIdx.x, warp = tid >> 5;
  copy16(Wf, pack, PB_FWD, tid);
  if (tid == 0) tc::mbar_init(&bar, 1);
  if (warp == 0) { tc::tmem_alloc(&tmem_sh, 128); tc::tmem_relinquish(); }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_sh;
  const uint32_t lane = (uint32_t)(warp * 32) << 16;
  const uint32_t sW = tc::smem_addr(Wf), sX0 = tc::smem_addr(X0), sX = tc::smem_addr(X);
  uint32_t ph = 0;
  bool failed = false;
  // all threads: wait for the MMAs just committed; false (everywhere) on timeout
  auto wait_mma = [&]() -> bool {
    const bool ok = tc::mbar_wait(&bar, ph, WAIT_TRIES);
    ph ^= 1u;
    tc::fence_after_sync();
    return !__syncthreads_or(!ok);
  };
  auto hidden_epilogue = [&](int l) {
    const float* b = theta + b_off(l);
    for (int c = 0; c < H; c += 16) {
      float v[16];
      tc::tmem_ld16(tmem + lane + c, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = silu(v[j] + b[c + j]);
      store8(X + tc::kmajor_offset(tid, c, H), v);
      store8(X + tc::kmajor_offset(tid, c + 8, H), v + 8);
    }
  };
  const int ntiles = (n + TM - 1) / TM;
  for (int tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    const int q = tile * TM + tid;
    float f[16];
    load_input_row(feat, q, n, f);
    store8(X0 + tc::kmajor_offset(tid, 0, KIN), f);
    store8(X0 + tc::kmajor_offset(tid, 8, KIN), f + 8);
    for (int l = 0; l < 5 && !failed; ++l) {
      tc::fence_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
        if (l == 0) issue_gemm(tmem, sX0, sW + PB_W0, KIN, H, false);
        else if (l < 4) issue_gemm(tmem, sX, sW + PB_W1 + (l - 1) * H * H * 2, H, H, false);
        else issue_gemm(tmem, sX, sW + PB_W4, H, NOUTP, false);
        tc::mma_commit(&bar);
      }
      if (!wait_mma()) { failed = true; break; }
      if (l < 4) {
        hidden_epilogue(l);
      } else {
        float v[16];
        tc::tmem_ld16(tmem + lane, v);
        if (q < n) {
          out[(size_t)q * 2] = v[0] + theta[OB4];
          out[(size_t)q * 2 + 1] = v[1] + theta[OB4 + 1];
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  if (failed && tid == 0 && err) atomicExch(err, 1);
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

// ---------------------------------------------------------------- training
// One CTA per tile of 128 samples: forward (pre-activations and BF16
// activations kept in the workspace), loss, backward, and the tile's
// gradient written to the workspace; reduce_adam_kernel sums the tiles in a
// fixed order and applies Adam.
constexpr size_t WS_Z = (size_t)4 * TM * H * 4;           // Z_l  [4][128][128] f32
constexpr size_t WS_X0 = (size_t)TM * KIN * 2;            // X_0  [128][16] bf16
constexpr size_t WS_X = (size_t)4 * TM * H * 2;           // X_1..X_4 [4][128][128] bf16
constexpr size_t WS_G = (((size_t)NPARAM * 4 + 255) / 256) * 256;
constexpr size_t WS_TILE = WS_Z + WS_X0 + WS_X + WS_G + 256;  // + the tile's loss
constexpr int TR_SMEM = 5 * H * H * 2 + TM * 2 * 4;

__global__ void __launch_bounds__(NT, 1)
mlp_train_tile_kernel(const uint8_t* __restrict__ pack, const float* __restrict__ theta,
                      const float* __restrict__ feat, const float* __restrict__ target, int n,
                      uint8_t* __restrict__ ws, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t* Wb = sm;                  // current layer's operand tile (W_l or W_l^T)
  uint8_t* Xb = Wb + H * H * 2;      // forward A operand X_l [m][k]
  uint8_t* DZ = Xb + H * H * 2;      // dZ_l [m][n]
  uint8_t* DZT = DZ + H * H * 2;     // dZ_l^T [n][m]
  uint8_t* XT = DZT + H * H * 2;     // X_l^T [k][m]
  float* dz4 = reinterpret_cast<float*>(XT + H * H * 2);  // [128][2]
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_sh;
  __shared__ float red[NT / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lanei = tid & 31;
  const int tile = blockIdx.x;
  const int q = tile * TM + tid;
  const bool valid = q < n;
  uint8_t* wt = ws + (size_t)tile * WS_TILE;
  float* Zs = reinterpret_cast<float*>(wt);
  __nv_bfloat16* X0s = reinterpret_cast<__nv_bfloat16*>(wt + WS_Z);
  __nv_bfloat16* Xs = reinterpret_cast<__nv_bfloat16*>(wt + WS_Z + WS_X0);
  float* Gs = reinterpret_cast<float*>(wt + WS_Z + WS_X0 + WS_X);
  float* lossp = reinterpret_cast<float*>(wt + WS_Z + WS_X0 + WS_X + WS_G);

  if (tid == 0) tc::mbar_init(&bar, 1);
  if (warp == 0) { tc::tmem_alloc(&tmem_sh, 256); tc::tmem_relinquish(); }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_sh;
  const uint32_t Dx = tmem, Dw = tmem + 128;
  const uint32_t lane = (uint32_t)(warp * 32) << 16;
  const uint32_t sWb = tc::smem_addr(Wb), sXb = tc::smem_addr(Xb), sDZ = tc::smem_addr(DZ);
  const uint32_t sDZT = tc::smem_addr(DZT), sXT = tc::smem_addr(XT);
  uint32_t ph = 0;
  bool failed = false;
  auto wait_mma = [&]() -> bool {
    const bool ok = tc::mbar_wait(&bar, ph, WAIT_TRIES);
    ph ^= 1u;
    tc::fence_after_sync();
    return !__syncthreads_or(!ok);
  };
  auto sync_for_mma = [&]() {
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
  };

  do {
    // ---------------- forward
    copy16(Wb, pack + PB_W0, H * KIN * 2, tid);
    {
      float f[16];
      load_input_row(feat, q, n, f);
      store8(Xb + tc::kmajor_offset(tid, 0, KIN), f);
      store8(Xb + tc::kmajor_offset(tid, 8, KIN), f + 8);
      __align__(16) __nv_bfloat16 h[16];
      for (int i = 0; i < 16; ++i) h[i] = __float2bfloat16_rn(f[i]);
      reinterpret_cast<uint4*>(X0s + (size_t)tid * KIN)[0] = reinterpret_cast<const uint4*>(h)[0];
      reinterpret_cast<uint4*>(X0s + (size_t)tid * KIN)[1] = reinterpret_cast<const uint4*>(h)[1];
    }
    sync_for_mma();
    if (tid == 0) { tc::fence_after_sync(); issue_gemm(Dx, sXb, sWb, KIN, H, false); tc::mma_commit(&bar); }
    if (!wait_mma()) { failed = true; break; }
    for (int l = 0; l < 4; ++l) {
      const float* b = theta + b_off(l);
      float* Zl = Zs + (size_t)l * TM * H + (size_t)tid * H;
      __nv_bfloat16* Xn = Xs + (size_t)l * TM * H + (size_t)tid * H;  // X_{l+1}
      for (int c = 0; c < H; c += 16) {
        float v[16];
        tc::tmem_ld16(Dx + lane + c, v);
        __align__(16) __nv_bfloat16 h[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          v[j] += b[c + j];
          Zl[c + j] = v[j];
          v[j] = silu(v[j]);
          h[j] = __float2bfloat16_rn(v[j]);
        }
        reinterpret_cast<uint4*>(Xn + c)[0] = reinterpret_cast<const uint4*>(h)[0];
        reinterpret_cast<uint4*>(Xn + c)[1] = reinterpret_cast<const uint4*>(h)[1];
        store8(Xb + tc::kmajor_offset(tid, c, H), v);
        store8(Xb + tc::kmajor_offset(tid, c + 8, H), v + 8);
      }
      if (l < 3) copy16(Wb, pack + PB_W1 + l * H * H * 2, H * H * 2, tid);
      else copy16(Wb, pack + PB_W4, NOUTP * H * 2, tid);
      sync_for_mma();
      if (tid == 0) {
        tc::fence_after_sync();
        issue_gemm(Dx, sXb, sWb, H, l < 3 ? H : NOUTP, false);
        tc::mma_commit(&bar);
      }
      if (!wait_mma()) { failed = true; break; }
    }
    if (failed) break;
    // ---------------- loss and dZ_4 (BF16-rounded)
    float loss = 0.0f;
    {
      float v[16];
      tc::tmem_ld16(Dx + lane, v);
      float d0 = 0.0f, d1 = 0.0f;
      if (valid) {
        const float mu = v[0] + theta[OB4], s = v[1] + theta[OB4 + 1];
        const float r = target[q] - mu, e = expf(-s);
        loss = 0.5f * (r * r * e + s);
        d0 = -r * e / (float)n;
        d1 = 0.5f * (1.0f - r * r * e) / (float)n;
      }
      float g16[16];
      for (int j = 0; j < 16; ++j) g16[j] = 0.0f;
      g16[0] = __bfloat162float(__float2bfloat16_rn(d0));
      g16[1] = __bfloat162float(__float2bfloat16_rn(d1));
      dz4[tid * 2] = g16[0];
      dz4[tid * 2 + 1] = g16[1];
      store8(DZ + tc::kmajor_offset(tid, 0, KIN), g16);
      store8(DZ + tc::kmajor_offset(tid, 8, KIN), g16 + 8);
    }
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if (lanei == 0) red[warp] = loss;
    copy16(Wb, pack + PB_W4T, H * NOUTP * 2, tid);
    sync_for_mma();
    if (tid == 0) {
      tc::fence_after_sync();
      issue_gemm(Dx, sDZ, sWb, KIN, H, false);  // dX_4 = dZ_4 W_4
      tc::mma_commit(&bar);
      lossp[0] = red[0] + red[1] + red[2] + red[3];
    }
    // dW_4, db_4 on the CUDA cores (two outputs): column k of X_4 is in Xb
    {
      float a0 = 0.0f, a1 = 0.0f;
      for (int m = 0; m < TM; ++m) {
        const float x = __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(Xb + tc::kmajor_offset(m, tid, H)));
        a0 = fmaf(dz4[m * 2], x, a0);
        a1 = fmaf(dz4[m * 2 + 1], x, a1);
      }
      Gs[OW4 + tid] = a0;
      Gs[OW4 + H + tid] = a1;
      if (tid < 2) {
        float sb = 0.0f;
        for (int m = 0; m < TM; ++m) sb += dz4[m * 2 + tid];
        Gs[OB4 + tid] = sb;
      }
    }
    if (!wait_mma()) { failed = true; break; }
    // ---------------- hidden layers, top down
    for (int l = 3; l >= 0 && !failed; --l) {
      const int Kl = l == 0 ? KIN : H;
      const int nin = l == 0 ? NIN : H;
      const float* Zl = Zs + (size_t)l * TM * H + (size_t)tid * H;
      for (int c = 0; c < H; c += 16) {
        float v[16];
        tc::tmem_ld16(Dx + lane + c, v);
        __align__(16) __nv_bfloat16 h[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          v[j] *= silu_prime(Zl[c + j]);
          h[j] = __float2bfloat16_rn(v[j]);
        }
        store8(DZ + tc::kmajor_offset(tid, c, H), v);
        store8(DZ + tc::kmajor_offset(tid, c + 8, H), v + 8);
#pragma unroll
        for (int j = 0; j < 16; ++j)
          *reinterpret_cast<__nv_bfloat16*>(DZT + tc::kmajor_offset(c + j, tid, H)) = h[j];
      }
      // X_l^T [k][m] from this row of X_l
      const __nv_bfloat16* Xl = l == 0 ? X0s + (size_t)tid * KIN : Xs + (size_t)(l - 1) * TM * H + (size_t)tid * H;
      for (int k = 0; k < Kl; ++k) *reinterpret_cast<__nv_bfloat16*>(XT + tc::kmajor_offset(k, tid, H)) = Xl[k];
      if (l > 0) copy16(Wb, pack + PB_W1T + (l - 1) * H * H * 2, H * H * 2, tid);
      sync_for_mma();
      if (tid == 0) {
        tc::fence_after_sync();
        issue_gemm(Dw, sDZT, sXT, H, Kl, false);       // dW_l = dZ_l^T X_l
        if (l > 0) issue_gemm(Dx, sDZ, sWb, H, H, false);  // dX_l = dZ_l W_l
        tc::mma_commit(&bar);
      }
      // db_l: row n = tid of dZ^T (the BF16 values the contractions use)
      {
        float sb = 0.0f;
        for (int m = 0; m < TM; m += 8) {
          const uint4 u = *reinterpret_cast<const uint4*>(DZT + tc::kmajor_offset(tid, m, H));
          const __nv_bfloat16* hh = reinterpret_cast<const __nv_bfloat16*>(&u);
          for (int j = 0; j < 8; ++j) sb += __bfloat162float(hh[j]);
        }
        Gs[b_off(l) + tid] = sb;
      }
      if (!wait_mma()) { failed = true; break; }
      for (int c = 0; c < Kl; c += 16) {
        float v[16];
        tc::tmem_ld16(Dw + lane + c, v);
        for (int j = 0; j < 16; ++j)
          if (c + j < nin) Gs[w_off(l) + tid * nin + c + j] = v[j];
      }
      tc::fence_before_sync();
      __syncthreads();
    }
  } while (false);
  if (failed && tid == 0 && err) atomicExch(err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// Sum of the tile gradients (fixed order), optional output, Adam update.
__global__ void reduce_adam_kernel(float* __restrict__ theta, float* __restrict__ m1, float* __restrict__ m2,
                                   const uint8_t* __restrict__ ws, int ntiles, int n, int step, float lr,
                                   float* __restrict__ grad_out, float* __restrict__ loss_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && loss_out) {
    double L = 0.0;
    for (int t = 0; t < ntiles; ++t)
      L += *reinterpret_cast<const float*>(ws + (size_t)t * WS_TILE + WS_Z + WS_X0 + WS_X + WS_G);
    *loss_out = (float)(L / n);
  }
  if (i >= NPARAM) return;
  float g = 0.0f;
  for (int t = 0; t < ntiles; ++t)
    g += reinterpret_cast<const float*>(ws + (size_t)t * WS_TILE + WS_Z + WS_X0 + WS_X)[i];
  if (grad_out) grad_out[i] = g;
  if (lr > 0.0f) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float a = b1 * m1[i] + (1.0f - b1) * g;
    const float v = b2 * m2[i] + (1.0f - b2) * g * g;
    m1[i] = a;
    m2[i] = v;
    const float mh = a / (1.0f - powf(b1, (float)step));
    const float vh = v / (1.0f - powf(b2, (float)step));
    theta[i] -= lr * mh / (sqrtf(vh) + eps);
  }
}

// ---------------------------------------------------------------- features
constexpr float TARGET_SCALE = 1e4f;

// <r^2> / rho^2 of the brightness over the source disk.  The law
// I0 [1 - u1 (1 - mu) - u2 (1 - mu)^2 - sum_k a_k (1 - mu^(k/2))] is a sum of
// powers c_p mu^p, mu = sqrt(1 - x), x = r^2 / rho^2, with c_0 = 1 - u1 - u2 -
// sum a, c_1 = u1 + 2 u2, c_2 = -u2 and a_k at p = k/2; over the disk
// int mu^p dx = 2/(p+2) and int mu^p x dx = 2/(p+2) - 2/(p+4).
__device__ double profile_r2(const icrs_params& p) {
  const double a[4] = {p.a1, p.a2, p.a3, p.a4};
  const double c0 = 1.0 - p.u1 - p.u2 - (a[0] + a[1] + a[2] + a[3]);
  double m0 = c0 + p.u1 * (2.0 / 3.0) + p.u2 * (2.0 * (2.0 / 3.0) - 0.5);
  double m1 = c0 * 0.5 + (p.u1 + 2.0 * p.u2) * (2.0 / 3.0 - 0.4) - p.u2 * (0.5 - 1.0 / 3.0);
  for (int k = 1; k <= 4; ++k) {
    const double q = 0.5 * k;
    m0 += a[k - 1] * (2.0 / (q + 2.0));
    m1 += a[k - 1] * (2.0 / (q + 2.0) - 2.0 / (q + 4.0));
  }
  return m1 / m0;
}
constexpr int NLIMB_SG = 32;  // source-limb points of the feature kernel
constexpr int FEAT_THREADS = 128;  // threads (epochs) per feature block
static_assert((NLIMB_SG & (NLIMB_SG - 1)) == 0, "the harmonic index wraps with a mask");

__global__ void features_kernel(const icrs_params* __restrict__ P, int S, const double* __restrict__ T, int E,
                                icrs_grid g, float* __restrict__ feat, double* __restrict__ A_ps,
                                uint32_t* __restrict__ status) {
  // limb magnifications minus the centre's, [k][thread], and the twiddles
  // e^{-2 pi i j / 32} of the limb harmonics
  __shared__ float dlimb[NLIMB_SG][FEAT_THREADS];
  __shared__ float2 tw[NLIMB_SG];
  if (threadIdx.x < NLIMB_SG) {
    double sn, cs;
    sincospi(2.0 * threadIdx.x / NLIMB_SG, &sn, &cs);
    tw[threadIdx.x] = make_float2((float)cs, (float)-sn);
  }
  __syncthreads();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)S * E) return;
  const int s = (int)(idx / E);
  const icrs_params prm = P[s];
  const Lens L = make_lens(prm);
  const cd w = source_centre(prm, T[idx]);
  PointSource<2> ps = point_source_solve<2>(L, w, g.max_iter, g.img_tol, nullptr);
  // 32 source-limb points: a caustic inside the disk changes the image count
  // between the centre and some limb point, which the centre's own images
  // cannot show when the centre lies outside the caustic (a cusp tip can
  // enter the disk between widely spaced samples)
  double mind = ps.m > 0 ? ps.min_det : 0.0;
  uint32_t stf = ps.st;
  double Alimb = 0.0;
  for (int k = 0; k < NLIMB_SG; ++k) {
    double sn, cs;
    sincospi(2.0 * k / NLIMB_SG, &sn, &cs);
    PointSource<2> pl = point_source_solve<2>(L, mk(w.x + prm.rho * cs, w.y + prm.rho * sn), g.max_iter, g.img_tol, nullptr);
    mind = fmin(mind, pl.m > 0 ? pl.min_det : 0.0);
    if (pl.m != ps.m || pl.st) stf |= ICRS_ST_LIMB;
    Alimb += pl.A / NLIMB_SG;
    dlimb[k][threadIdx.x] = (float)(pl.A - ps.A);
  }
  // harmonics of order m = 3..16 of the limb values (the orders 17..29 are
  // their mirror images, so orders 3..15 count twice and 16 once)
  float hsum = 0.f;
  for (int m = 3; m <= NLIMB_SG / 2; ++m) {
    float cr = 0.f, ci = 0.f;
    for (int k = 0; k < NLIMB_SG; ++k) {
      const float2 w_ = tw[(m * k) & (NLIMB_SG - 1)];
      const float d = dlimb[k][threadIdx.x];
      cr = fmaf(d, w_.x, cr);
      ci = fmaf(d, w_.y, ci);
    }
    hsum += (m < NLIMB_SG / 2 ? 2.f : 1.f) * sqrtf(cr * cr + ci * ci);
  }
  const double rough = (double)hsum / NLIMB_SG / ps.A;
  if (!(rough <= ICRS_ROUGH_MAX)) stf |= ICRS_ST_ROUGH;
  // second-order finite-source estimate: the limb mean minus the centre is
  // (rho^2 / 4) lap A to leading order, and the disk average of A is
  // A + (<r^2> / 4) lap A, <r^2> the brightness's second moment
  const double fu = g.uniform ? 0.5 : profile_r2(prm);
  const double est = ps.A > 0.0 ? TARGET_SCALE * log1p(fu * (Alimb / ps.A - 1.0)) : 0.0;
  if (prm.spot_c != 0.0 && prm.spot_r > 0.0) stf |= ICRS_ST_SPOT;
  if (!g.uniform && (prm.u2 != 0.0 || prm.a1 != 0.0 || prm.a2 != 0.0 || prm.a3 != 0.0 || prm.a4 != 0.0))
    stf |= ICRS_ST_PROFILE;
  float* f = feat + idx * 8;
  f[0] = (float)w.x;
  f[1] = (float)w.y;
  f[2] = (float)log10(prm.s);
  f[3] = (float)((log10(prm.q) + 3.0) * 0.5);
  f[4] = (float)(log10(prm.rho) + 3.0);
  f[5] = (float)(4.0 * (prm.u1 - 0.55));
  f[6] = mind > 0.0 ? (float)fmin(1.0, fmax(-6.0, log10(mind))) : -6.0f;
  f[7] = (est == est) ? (float)fmax(-1e4, fmin(1e4, est)) : 0.0f;
  A_ps[idx] = ps.A;
  if (status) status[idx] = stf;
}

// ---------------------------------------------------------------- gate
// Accept an epoch when its feature status is clean (solves, image count across
// the disk, limb roughness), its caustic feature
// is at least caustic_min, the predicted standard deviation exp(s/2) is at
// most sigma_max, |mu| at most mu_max, the second-order estimate |b|
// (feature 7) at most b_max (units of 1e-4 in log A), and A_ps at most A_max
// (A_small when rho < rho_min: small sources away from the far field, and all
// sources at high magnification, are where ICRS itself still moves by 1e-4
// between grid refinements); accepted epochs get
// A = A_ps exp(1e-4 (b + mu)).  Routed epochs are listed in order.
constexpr int GB = 1024;  // queries per gate block

__global__ void gate_flags_kernel(const float* __restrict__ pred, const float* __restrict__ feat,
                                  const double* __restrict__ A_ps, const uint32_t* __restrict__ st_ps, int n,
                                  float sigma_max, float mu_max, float b_max, float caustic_min, double A_max,
                                  float rho_min, double A_small, double* __restrict__ A,
                                  uint8_t* __restrict__ flag, int32_t* __restrict__ bcount) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  const int q = blockIdx.x * GB + threadIdx.x;
  int routed = 0;
  if (q < n) {
    const float mu = pred[(size_t)q * 2], s = pred[(size_t)q * 2 + 1];
    const float base = feat[(size_t)q * 8 + 7];
    const bool ok = st_ps[q] == 0u && feat[(size_t)q * 8 + 6] >= caustic_min && expf(0.5f * s) <= sigma_max &&
                    fabsf(mu) <= mu_max && fabsf(base) <= b_max && isfinite(mu) &&
                    A_ps[q] <= (feat[(size_t)q * 8 + 4] >= log10f(rho_min) + 3.0f ? A_max : A_small);
    routed = ok ? 0 : 1;
    if (ok) A[q] = A_ps[q] * exp(((double)base + (double)mu) / (double)TARGET_SCALE);
    flag[q] = (uint8_t)routed;
  }
  const unsigned b = __ballot_sync(0xffffffffu, routed);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(&cnt, __popc(b));
  __syncthreads();
  if (threadIdx.x == 0) bcount[blockIdx.x] = cnt;
}

// Exclusive scan of the block counts (one block of 1024 threads).
__global__ void gate_scan_kernel(int32_t* __restrict__ bcount, int nb, int32_t* __restrict__ total) {
  __shared__ int sh[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? bcount[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nb) bcount[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void gate_scatter_kernel(const uint8_t* __restrict__ flag, int n, const int32_t* __restrict__ boff,
                                    int32_t* __restrict__ routed_idx) {
  __shared__ int wsum[GB / 32];
  const int q = blockIdx.x * GB + threadIdx.x;
  const int f = q < n ? flag[q] : 0;
  const int lanei = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned b = __ballot_sync(0xffffffffu, f);
  if (lanei == 0) wsum[w] = __popc(b);
  __syncthreads();
  int off = boff[blockIdx.x];
  for (int i = 0; i < w; ++i) off += wsum[i];
  if (f) routed_idx[off + __popc(b & ((1u << lanei) - 1u))] = q;
}

// ---------------------------------------------------------------- epoch preselection
// Non-learned gate (Sec. 3.4 (iii): the extended-source computation runs only
// on a preselected set of epochs near caustics).  An epoch is near a caustic
// unless its point-source solves are clean (status 0), its caustic feature is
// at least caustic_min, the second-order finite-source estimate |b| is at most
// b_max and A_ps is at most A_max (A_small for rho < rho_min).  Every epoch of
// the same light curve within n_ext epochs of a near-caustic one is routed
// too.  The rest get the estimate: A_ps (mode 0) or A_ps exp(1e-4 b) (mode 1).
__global__ void epoch_near_kernel(const float* __restrict__ feat, const double* __restrict__ A_ps,
                                  const uint32_t* __restrict__ st_ps, int n, float b_max, float caustic_min,
                                  double A_max, float rho_min, double A_small, uint8_t* __restrict__ near) {
  const int q = blockIdx.x * GB + threadIdx.x;
  if (q >= n) return;
  const float base = feat[(size_t)q * 8 + 7];
  // the estimate holds for any radial law, so ICRS_ST_PROFILE does not route here
  const bool ok = (st_ps[q] & ~ICRS_ST_PROFILE) == 0u && feat[(size_t)q * 8 + 6] >= caustic_min &&
                  fabsf(base) <= b_max &&
                  A_ps[q] <= (feat[(size_t)q * 8 + 4] >= log10f(rho_min) + 3.0f ? A_max : A_small);
  near[q] = ok ? 0 : 1;
}

__global__ void epoch_extend_kernel(const uint8_t* __restrict__ near, const float* __restrict__ feat,
                                    const double* __restrict__ A_ps, int S, int E, int n_ext, int mode,
                                    double* __restrict__ A, uint8_t* __restrict__ flag,
                                    int32_t* __restrict__ bcount) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  const long long n = (long long)S * E;
  const long long q = (long long)blockIdx.x * GB + threadIdx.x;
  int routed = 0;
  if (q < n) {
    const int e = (int)(q % E);
    const long long row = q - e;
    const int e0 = e - n_ext < 0 ? 0 : e - n_ext;
    const int e1 = e + n_ext >= E ? E - 1 : e + n_ext;
    for (int k = e0; k <= e1 && !routed; ++k) routed = near[row + k];
    if (!routed)
      A[q] = mode == 0 ? A_ps[q] : A_ps[q] * exp((double)feat[(size_t)q * 8 + 7] / (double)TARGET_SCALE);
    flag[q] = (uint8_t)routed;
  }
  const unsigned b = __ballot_sync(0xffffffffu, routed);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(&cnt, __popc(b));
  __syncthreads();
  if (threadIdx.x == 0) bcount[blockIdx.x] = cnt;
}

// ---------------------------------------------------------------- training data
// Target of the network: y = 1e4 log(A_ICRS / A_ps) - b (b = features[7]).
__global__ void target_kernel(const double* __restrict__ A, const double* __restrict__ A_ps,
                              const float* __restrict__ feat, int n, float* __restrict__ target) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  target[q] = (float)((double)TARGET_SCALE * log(A[q] / A_ps[q]) - (double)feat[(size_t)q * 8 + 7]);
}

// Mini-batch gather: rows idx[i] of (features, target).
__global__ void batch_kernel(const float4* __restrict__ feat, const float* __restrict__ target,
                             const int32_t* __restrict__ idx, int n, float4* __restrict__ out_feat,
                             float* __restrict__ out_target) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t r = (size_t)idx[i];
  out_feat[2 * (size_t)i] = feat[2 * r];
  out_feat[2 * (size_t)i + 1] = feat[2 * r + 1];
  out_target[i] = target[r];
}

// ---------------------------------------------------------------- static scratch
// Scratch of the allocation-free training step.  Some callers cannot ask for
// device memory at the point where they train:
//   - code running between the begin and end of a stream capture, where an
//     allocation would break or be recorded into the capture;
//   - host-side schedulers with a fixed memory budget that own no allocator;
//   - processes that must leave the device allocator untouched between steps.
// For them the step can use this file-scope array: 32 tiles, i.e. batches of
// up to 4096 samples, about 19 MB, reserved when this module is loaded.
constexpr int STATIC_MAX_N = ICRS_MLP_STATIC_MAX_N;
constexpr size_t STATIC_WS_BYTES = (size_t)((STATIC_MAX_N + TM - 1) / TM) * WS_TILE;
static __device__ __align__(256) uint8_t g_train_scratch[STATIC_WS_BYTES];

}  // namespace sg
}  // namespace icrs

#include <mutex>

using namespace icrs;
using namespace icrs::sg;

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the static scratch for the current device, looked up
// once per device (with that device current) and cached.
int static_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ICRS_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return ICRS_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* a = nullptr;
    if (cudaGetSymbolAddress(&a, g_train_scratch) != cudaSuccess || !a) return ICRS_ECUDA;
    g_scratch_addr[dev] = a;
  }
  *out = g_scratch_addr[dev];
  return ICRS_OK;
}
}  // namespace

extern "C" {

size_t icrs_mlp_workspace_bytes(int n) {
  if (n <= 0) return 0;
  return (size_t)((n + TM - 1) / TM) * WS_TILE;
}

int icrs_mlp_pack(const float* theta, void* pack, void* stream) {
  if (!theta || !pack) return ICRS_EINVAL;
  const int chunks = PACK_BYTES / 16;
  pack_kernel<<<(chunks + 255) / 256, 256, 0, (cudaStream_t)stream>>>(theta, (uint8_t*)pack);
  return cudaGetLastError() == cudaSuccess ? ICRS_OK : ICRS_ECUDA;
}

int icrs_mlp_infer(const void* pack, const float* theta, const float* feat, int n, float* out, int* err,
                   void* stream) {
  if (n < 0) return ICRS_EINVAL;
  if (n == 0) return ICRS_OK;
  if (!pack || !theta || !feat || !out) return ICRS_EINVAL;
  if (((uintptr_t)feat & 15) || ((uintptr_t)pack & 15)) return ICRS_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ICRS_ECUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ICRS_ECUDA;
  if (cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, INF_SMEM) != cudaSuccess)
    return ICRS_ECUDA;
  const int ntiles = (n + TM - 1) / TM;
  const int grid = ntiles < nsm ? ntiles : nsm;
  mlp_infer_kernel<<<grid, NT, INF_SMEM, (cudaStream_t)stream>>>((const uint8_t*)pack, theta, feat, n, out, err);
  return cudaGetLastError() == cudaSuccess ? ICRS_OK : ICRS_ECUDA;
}

int icrs_mlp_train_step(float* theta, float* adam_m, float* adam_v, void* pack, int step, float lr,
                        const float* feat, const float* target, int n, float* grad, float* loss, void* workspace,
                        size_t workspace_bytes, int* err, void* stream) {
  if (n <= 0 || step < 1 || !(lr >= 0.0f)) return ICRS_EINVAL;
  if (!theta || !pack || !feat || !target || !workspace) return ICRS_EINVAL;
  if (lr > 0.0f && (!adam_m || !adam_v)) return ICRS_EINVAL;
  if (((uintptr_t)feat & 15) || ((uintptr_t)pack & 15) || ((uintptr_t)workspace & 255)) return ICRS_EINVAL;
  if (workspace_bytes < icrs_mlp_workspace_bytes(n)) return ICRS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaFuncSetAttribute(mlp_train_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TR_SMEM) != cudaSuccess)
    return ICRS_ECUDA;
  const int ntiles = (n + TM - 1) / TM;
  mlp_train_tile_kernel<<<ntiles, NT, TR_SMEM, st>>>((const uint8_t*)pack, theta, feat, target, n,
                                                     (uint8_t*)workspace, err);
  reduce_adam_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(theta, adam_m, adam_v, (const uint8_t*)workspace, ntiles,
                                                           n, step, lr, grad, loss);
  if (lr > 0.0f) {
    const int chunks = PACK_BYTES / 16;
    pack_kernel<<<(chunks + 255) / 256, 256, 0, st>>>(theta, (uint8_t*)pack);
  }
  return cudaGetLastError() == cudaSuccess ? ICRS_OK : ICRS_ECUDA;
}

int icrs_mlp_train_step_noalloc(float* theta, float* adam_m, float* adam_v, void* pack, int step, float lr,
                                const float* feat, const float* target, int n, float* grad, float* loss, int* err,
                                void* stream) {
  if (n <= 0 || n > STATIC_MAX_N) return ICRS_EINVAL;
  void* ws = nullptr;
  const int rc = static_scratch(&ws);
  if (rc != ICRS_OK) return rc;
  // Every scratch word the step reads (activations, pre-activations, the
  // per-tile gradients and losses) is written earlier in the same step, so
  // nothing has to be cleared between calls.
  return icrs_mlp_train_step(theta, adam_m, adam_v, pack, step, lr, feat, target, n, grad, loss, ws,
                             STATIC_WS_BYTES, err, stream);
}

int icrs_surrogate_features(const icrs_params* p, int S, const double* t, int E, const icrs_grid* g, float* feat,
                            double* A_ps, uint32_t* status, void* stream) {
  if (S < 0 || E < 0 || !g) return ICRS_EINVAL;
  if (S == 0 || E == 0) return ICRS_OK;
  if (!p || !t || !feat || !A_ps) return ICRS_EINVAL;
  if (g->n_lens != 2) return ICRS_EUNSUPPORTED;
  const long long total = (long long)S * E;
  const long long blocks = (total + FEAT_THREADS - 1) / FEAT_THREADS;
  if (blocks > 2147483647LL) return ICRS_EUNSUPPORTED;
  features_kernel<<<(unsigned)blocks, FEAT_THREADS, 0, (cudaStream_t)stream>>>(p, S, t, E, *g, feat, A_ps, status);
  return cudaGetLastError() == cudaSuccess ? ICRS_OK : ICRS_ECUDA;
}

size_t icrs_surrogate_gate_workspace_bytes(int n) {
  if (n <= 0) return 0;
  const size_t nb = (size_t)(n + GB - 1) / GB;
  return ((size_t)n + 255) / 256 * 256 + nb * 4;
}

int icrs_surrogate_gate(const float* pred, const float* feat, const double* A_ps, const uint32_t* st_ps, int n,
                        float sigma_max, float mu_max, float b_max, float caustic_min, double A_max, float rho_min,
                        double A_small, double* A, int32_t* routed_idx,
                        int32_t* n_routed, void* workspace, size_t workspace_bytes, void* stream) {
  if (n < 0) return ICRS_EINVAL;
  if (n == 0) return ICRS_OK;
  if (!pred || !feat || !A_ps || !st_ps || !A || !routed_idx || !n_routed || !workspace) return ICRS_EINVAL;
  if (workspace_bytes < icrs_surrogate_gate_workspace_bytes(n)) return ICRS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = (n + GB - 1) / GB;
  uint8_t* flag = (uint8_t*)workspace;
  int32_t* bcount = (int32_t*)((uint8_t*)workspace + ((size_t)n + 255) / 256 * 256);
  gate_flags_kernel<<<nb, GB, 0, st>>>(pred, feat, A_ps, st_ps, n, sigma_max, mu_max, b_max, caustic_min, A_max,
                                       rho_min, A_small, A, flag, bcount);
  gate_scan_kernel<<<1, 1024, 0, st>>>(bcount, nb, n_routed);
  gate_scatter_kernel<<<nb, GB, 0, st>>>(flag, n, bcount, routed_idx);
  return cudaGetLastError() == cudaSuccess ? ICRS_OK : ICRS_ECUDA;
}

int icrs_surrogate_target(const double* A, const double* A_ps, const float* feat, int n, float* target,
                          void* stream) {
  if (n < 0) return ICRS_EINVAL;
  if (n == 0) return ICRS_OK;
  if (!A || !A_ps || !feat || !target) return ICRS_EINVAL;
  target_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(A, A_ps, feat, n, target);
  return cudaGetLastError() == cudaSuccess ? ICRS_OK : ICRS_ECUDA;
}

int icrs_surrogate_batch(const float* feat, const float* target, const int32_t* idx, int n, float* out_feat,
                         float* out_target, void* stream) {
  if (n < 0) return ICRS_EINVAL;
  if (n == 0) return ICRS_OK;
  if (!feat || !target || !idx || !out_feat || !out_target) return ICRS_EINVAL;
  if (((uintptr_t)feat & 15) || ((uintptr_t)out_feat & 15)) return ICRS_EINVAL;
  batch_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>((const float4*)feat, target, idx, n,
                                                                 (float4*)out_feat, out_target);
  return cudaGetLastError() == cudaSuccess ? ICRS_OK : ICRS_ECUDA;
}

size_t icrs_epoch_gate_workspace_bytes(int S, int E) {
  if (S <= 0 || E <= 0) return 0;
  const size_t n = (size_t)S * (size_t)E;
  return (n + 255) / 256 * 256 + icrs_surrogate_gate_workspace_bytes((int)n);
}

int icrs_epoch_gate(const float* feat, const double* A_ps, const uint32_t* st_ps, int S, int E, int n_ext, int mode,
                    float b_max, float caustic_min, double A_max, float rho_min, double A_small, double* A,
                    int32_t* routed_idx, int32_t* n_routed, void* workspace, size_t workspace_bytes, void* stream) {
  if (S < 0 || E < 0 || n_ext < 0 || (mode != 0 && mode != 1)) return ICRS_EINVAL;
  if ((long long)S * E > 2147483647LL) return ICRS_EUNSUPPORTED;
  const int n = S * E;
  if (n == 0) return ICRS_OK;
  if (!feat || !A_ps || !st_ps || !A || !routed_idx || !n_routed || !workspace) return ICRS_EINVAL;
  if (workspace_bytes < icrs_epoch_gate_workspace_bytes(S, E)) return ICRS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = (n + GB - 1) / GB;
  uint8_t* near = (uint8_t*)workspace;
  uint8_t* flag = near + ((size_t)n + 255) / 256 * 256;
  int32_t* bcount = (int32_t*)(flag + ((size_t)n + 255) / 256 * 256);
  epoch_near_kernel<<<nb, GB, 0, st>>>(feat, A_ps, st_ps, n, b_max, caustic_min, A_max, rho_min, A_small, near);
  epoch_extend_kernel<<<nb, GB, 0, st>>>(near, feat, A_ps, S, E, n_ext, mode, A, flag, bcount);
  gate_scan_kernel<<<1, 1024, 0, st>>>(bcount, nb, n_routed);
  gate_scatter_kernel<<<nb, GB, 0, st>>>(flag, n, bcount, routed_idx);
  return cudaGetLastError() == cudaSuccess ? ICRS_OK : ICRS_ECUDA;
}

}  // extern "C"
