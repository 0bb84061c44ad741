// Learned warm start: a per-column MLP 16 -> 128 -> 128 -> 128 -> 32 on the 5th-generation tensor
// cores.  Every GEMM is a tcgen05.mma (kind::f16, BF16 operands from shared memory, FP32
// accumulators in tensor memory), issued by one thread, completed through an mbarrier, and read
// back with tcgen05.ld.  Operands sit in shared memory in the canonical no-swizzle K-major layout:
// 8 x 16-byte core matrices, core matrices adjacent along K at 128 B (leading byte offset) and
// 8-row groups at K x 16 B (stride byte offset).  The packed weights are kept in global memory
// already in that layout, so a CTA brings them in with one cp.async.bulk copy.
//
// Forward (persistent, 1 CTA = 4 warps per SM): per 128-row tile, X -> smem, then four
// MMA -> TMEM -> bias/ReLU/BF16 -> smem rounds; the last layer writes FP32 outputs.
// Backward (one CTA per 128-row tile): per layer, dW = dZ^T H (contraction over the tile's rows,
// reduced across tiles with FP32 atomics) and dH = dZ W on the tensor cores, ReLU masks and bias
// gradients on the CUDA cores.  Adam updates FP32 master weights and repacks the BF16 operands.
//
// Every wait on an mbarrier is bounded; on time-out the kernel records an error flag, skips the
// tensor-memory reads, releases its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bp_internal.cuh"

namespace {

constexpr int IN = BP_MLP_IN, HID = BP_MLP_HIDDEN, OUT = BP_MLP_OUT, OUT_USED = BP_MLP_OUT_USED;
constexpr int64_t OW1 = 0, OB1 = OW1 + HID * IN, OW2 = OB1 + HID, OB2 = OW2 + HID * HID, OW3 = OB2 + HID,
                  OB3 = OW3 + HID * HID, OW4 = OB3 + HID, OB4 = OW4 + OUT * HID, NPARAM = OB4 + OUT;
// packed BF16 operands (bytes): forward B operands W_l (n = out, k = in), then W_l^T (n = in, k = out)
constexpr uint32_t PF1 = 0, PF2 = PF1 + HID * IN * 2, PF3 = PF2 + HID * HID * 2, PF4 = PF3 + HID * HID * 2,
                   PF_END = PF4 + OUT * HID * 2;
constexpr uint32_t PT2 = PF_END, PT3 = PT2 + HID * HID * 2, PT4 = PT3 + HID * HID * 2, PT_END = PT4 + HID * OUT * 2;
constexpr uint32_t ACT_BYTES = 128 * HID * 2;           // one 128 x 128 BF16 operand tile
constexpr uint32_t FWD_SMEM = PF_END + ACT_BYTES + 4 * 128 * 4;
constexpr uint32_t BWD_SMEM = 4 * ACT_BYTES;
constexpr int WAIT_SPINS = 1 << 22;

__host__ __device__ __forceinline__ uint32_t kmaj(int row, int k, int K) {
  return (uint32_t)((row >> 3) * (K * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t K) {
  uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;             // leading byte offset: next core matrix along K
  d |= (uint64_t)(((uint32_t)K * 16) >> 4) << 32;  // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                      // descriptor version (sm_100 family), no swizzle
  return d;
}

// kind::f16 instruction descriptor: FP32 accumulate, BF16 A and B, both K-major, N >> 3, M >> 4
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[M x K] B[N x K]^T, K a multiple of 16, issued by one thread
__device__ __forceinline__ void gemm(uint32_t tmem_d, const uint8_t* sA, const uint8_t* sB, int M, int N, int K) {
  const uint32_t id = idesc_bf16(M, N);
  for (int ks = 0; ks < K / 16; ++ks) {
    const uint64_t a = sdesc(smem_u32(sA) + ks * 256, K), b = sdesc(smem_u32(sB) + ks * 256, K);
    const uint32_t acc = ks > 0;
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)));
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  for (int it = 0; it < WAIT_SPINS; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase));
    if (done) return true;
    if (it > 32) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tc_sync() {  // smem writes visible to the tensor cores, TMEM ordered
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
}

__device__ __forceinline__ uint32_t tmem_alloc_warp0(uint32_t* slot, uint32_t ncols) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  return 0;
}

__device__ __forceinline__ void tmem_free_warp0(uint32_t tmem, uint32_t ncols) {
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

__device__ __forceinline__ uint16_t bf16_bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float bf16_val(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

// ------------------------------------------------------------------ forward
struct FwdArgs {
  const uint8_t* wpack;
  const float* params;
  const uint16_t* X;
  int64_t n;
  float* Y;
  uint16_t *H1, *H2, *H3;  // nullable: activations kept for the backward pass
  int* err;
};

__global__ void __launch_bounds__(128, 1) k_mlp_forward(const FwdArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t* sW = sm;
  uint8_t* sA = sm + PF_END;
  float* sBias = reinterpret_cast<float*>(sm + PF_END + ACT_BYTES);
  __shared__ __align__(8) uint64_t bar_w, bar_mma;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t ntiles = (a.n + 127) / 128;
  if (blockIdx.x >= ntiles) return;
  for (int i = tid; i < 3 * HID + OUT; i += 128) {
    const int64_t off = i < HID ? OB1 + i : (i < 2 * HID ? OB2 + i - HID : (i < 3 * HID ? OB3 + i - 2 * HID : OB4 + i - 3 * HID));
    sBias[i] = a.params[off];
  }
  tmem_alloc_warp0(&tmem_slot, 128);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_w)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_mma)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  tc_sync();
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {  // TMA bulk copy of all packed forward weights
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar_w)), "r"(PF_END));
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(sW)),
                 "l"(a.wpack), "r"(PF_END), "r"(smem_u32(&bar_w)));
  }
  bool ok = __syncthreads_and(mbar_wait(&bar_w, 0));
  uint32_t phase = 0;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
    const int64_t row = tile * 128 + tid;
    const bool valid = row < a.n;
    uint4 x0 = make_uint4(0, 0, 0, 0), x1 = x0;
    if (valid) {
      x0 = reinterpret_cast<const uint4*>(a.X + row * IN)[0];
      x1 = reinterpret_cast<const uint4*>(a.X + row * IN)[1];
    }
    *reinterpret_cast<uint4*>(sA + kmaj(tid, 0, IN)) = x0;
    *reinterpret_cast<uint4*>(sA + kmaj(tid, 8, IN)) = x1;
    tc_sync();
    for (int layer = 0; layer < 4 && ok; ++layer) {
      const int K = layer == 0 ? IN : HID, N = layer == 3 ? OUT : HID;
      const uint32_t woff = layer == 0 ? PF1 : (layer == 1 ? PF2 : (layer == 2 ? PF3 : PF4));
      if (tid == 0) {
        gemm(tmem, sA, sW + woff, 128, N, K);
        mma_commit(&bar_mma);
      }
      ok = __syncthreads_and(mbar_wait(&bar_mma, phase));
      phase ^= 1;
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (!ok) break;
      if (layer < 3) {
        uint16_t* Hg = layer == 0 ? a.H1 : (layer == 1 ? a.H2 : a.H3);
        for (int c0 = 0; c0 < HID; c0 += 32) {
          float v[32];
          tmem_ld32(tmem + lane_base + c0, v);
          uint32_t pk[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float h0 = fmaxf(v[2 * j] + sBias[layer * HID + c0 + 2 * j], 0.f);
            const float h1 = fmaxf(v[2 * j + 1] + sBias[layer * HID + c0 + 2 * j + 1], 0.f);
            pk[j] = (uint32_t)bf16_bits(h0) | ((uint32_t)bf16_bits(h1) << 16);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint4 w = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
            *reinterpret_cast<uint4*>(sA + kmaj(tid, c0 + 8 * q, HID)) = w;
            if (Hg && valid) reinterpret_cast<uint4*>(Hg + row * HID + c0)[q] = w;
          }
        }
        tc_sync();
      } else {
        float v[32];
        tmem_ld32(tmem + lane_base, v);
        if (valid) {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            reinterpret_cast<float4*>(a.Y + row * OUT)[q] =
                make_float4(v[4 * q] + sBias[3 * HID + 4 * q], v[4 * q + 1] + sBias[3 * HID + 4 * q + 1],
                            v[4 * q + 2] + sBias[3 * HID + 4 * q + 2], v[4 * q + 3] + sBias[3 * HID + 4 * q + 3]);
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
      }
    }
  }
  if (!ok && tid == 0) atomicExch(a.err, 1);
  if (!ok) {  // give an MMA that might still be in flight a bounded chance to land before freeing TMEM
    mbar_wait(&bar_mma, phase);
  }
  tmem_free_warp0(tmem, 128);
}

// ------------------------------------------------------------------ backward
struct BwdArgs {
  const uint8_t* wpack;
  const uint16_t *X, *H1, *H2, *H3;
  const float *Y, *T;
  int64_t n;
  float scale;  // 2 / n
  float* grad;
  double* loss;
  int* err;
};

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reads the dH accumulator of the tile (row = thread), applies the ReLU mask of H_in (the layer's
// input activations), accumulates the bias gradient of that layer and writes dZ = dH * mask as the
// next step's operands: natural (row, feature) into sHA and transposed (feature, row) into sWA.
__device__ __forceinline__ void relu_back(uint32_t tmem_h, const uint16_t* Hrow, bool valid, uint8_t* sHA,
                                          uint8_t* sWA, float* gbias, int tid) {
  const uint32_t lane_base = (uint32_t)((tid >> 5) * 32) << 16;
  for (int c0 = 0; c0 < HID; c0 += 32) {
    float v[32];
    tmem_ld32(tmem_h + lane_base + c0, v);
    uint32_t pk[16];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float hin = valid ? bf16_val(Hrow[c0 + j]) : 0.f;
      const float dz = (valid && hin > 0.f) ? v[j] : 0.f;
      v[j] = dz;
      const uint16_t b = bf16_bits(dz);
      if (j & 1)
        pk[j >> 1] |= (uint32_t)b << 16;
      else
        pk[j >> 1] = b;
      *reinterpret_cast<uint16_t*>(sWA + kmaj(c0 + j, tid, 128)) = b;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      *reinterpret_cast<uint4*>(sHA + kmaj(tid, c0 + 8 * q, HID)) =
          make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float s = warp_sum_f(v[j]);
      if ((tid & 31) == 0) atomicAdd(gbias + c0 + j, s);
    }
  }
}

// transposed write of a BF16 row (length len) of the tile: element (feature f, row tid) of a K-major
// operand whose K is the tile's 128 rows
__device__ __forceinline__ void write_rowT(uint8_t* s, const uint16_t* src, bool valid, int len, int tid) {
  for (int f = 0; f < len; ++f)
    *reinterpret_cast<uint16_t*>(s + kmaj(f, tid, 128)) = valid ? src[f] : (uint16_t)0;
}

__device__ __forceinline__ void copy_operand(uint8_t* dst, const uint8_t* src, uint32_t bytes, int tid) {
  for (uint32_t i = tid * 16; i < bytes; i += 128 * 16)
    *reinterpret_cast<uint4*>(dst + i) = *reinterpret_cast<const uint4*>(src + i);
}

__global__ void __launch_bounds__(128, 1) k_mlp_backward(const BwdArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t* sWA = sm;                   // A of the dW GEMM (dZ^T: features x rows)
  uint8_t* sWB = sm + ACT_BYTES;       // B of the dW GEMM (H^T: features x rows)
  uint8_t* sHA = sm + 2 * ACT_BYTES;   // A of the dH GEMM (dZ: rows x features)
  uint8_t* sHB = sm + 3 * ACT_BYTES;   // B of the dH GEMM (W^T: in x out)
  __shared__ __align__(8) uint64_t bar_mma;
  __shared__ uint32_t tmem_slot;
  __shared__ float s_loss[4];
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t row = blockIdx.x * 128LL + tid;
  const bool valid = row < a.n;
  tmem_alloc_warp0(&tmem_slot, 256);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_mma)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // output gradient dY4 = (2/n)(Y - T) on the used outputs; loss
  float dy[OUT];
  float lsum = 0.f;
#pragma unroll
  for (int o = 0; o < OUT; ++o) {
    float d = 0.f;
    if (valid && o < OUT_USED) {
      d = a.Y[row * OUT + o] - a.T[row * OUT + o];
      lsum += d * d;
    }
    dy[o] = a.scale * d;
  }
  lsum = warp_sum_f(lsum);
  if (lane == 0) s_loss[tid >> 5] = lsum;
#pragma unroll
  for (int o = 0; o < OUT; ++o) {
    const float s = warp_sum_f(dy[o]);
    if (lane == 0) atomicAdd(a.grad + OB4 + o, s);
  }
  // layer 4 operands: dW4^T = H3^T dY4 (M = 128 in, N = 32 out), dH3 = dY4 W4 (M = rows, N = 128, K = 32)
  write_rowT(sWA, a.H3 + row * HID, valid, HID, tid);
  for (int o = 0; o < OUT; ++o) *reinterpret_cast<uint16_t*>(sWB + kmaj(o, tid, 128)) = bf16_bits(dy[o]);
  for (int q = 0; q < OUT / 8; ++q) {
    uint32_t pk[4];
    for (int j = 0; j < 4; ++j)
      pk[j] = (uint32_t)bf16_bits(dy[8 * q + 2 * j]) | ((uint32_t)bf16_bits(dy[8 * q + 2 * j + 1]) << 16);
    *reinterpret_cast<uint4*>(sHA + kmaj(tid, 8 * q, OUT)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
  copy_operand(sHB, a.wpack + PT4, HID * OUT * 2, tid);
  tc_sync();
  if (tid == 0) atomicAdd(a.loss, (double)(s_loss[0] + s_loss[1] + s_loss[2] + s_loss[3]) / (double)a.n);
  const uint32_t tmem = tmem_slot;
  const uint32_t lane_base = (uint32_t)((tid >> 5) * 32) << 16;
  uint32_t phase = 0;
  bool ok = true;
  if (tid == 0) {
    gemm(tmem, sWA, sWB, 128, OUT, 128);
    gemm(tmem + 128, sHA, sHB, 128, HID, OUT);
    mma_commit(&bar_mma);
  }
  ok = __syncthreads_and(mbar_wait(&bar_mma, phase));
  phase ^= 1;
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    float v[32];
    tmem_ld32(tmem + lane_base, v);  // dW4^T[f = tid][o]
    for (int o = 0; o < OUT; ++o) atomicAdd(a.grad + OW4 + (int64_t)o * HID + tid, v[o]);
    relu_back(tmem + 128, a.H3 + row * HID, valid, sHA, sWA, a.grad + OB3, tid);
  }
  // layers 3 and 2: dW = dZ^T H_in (M = out, N = in, K = rows), dH_in = dZ W (B = W^T)
  for (int layer = 3; layer >= 2 && ok; --layer) {
    const uint16_t* Hin = layer == 3 ? a.H2 : a.H1;
    write_rowT(sWB, Hin + row * HID, valid, HID, tid);
    copy_operand(sHB, a.wpack + (layer == 3 ? PT3 : PT2), HID * HID * 2, tid);
    tc_sync();
    if (tid == 0) {
      gemm(tmem, sWA, sWB, 128, HID, 128);
      gemm(tmem + 128, sHA, sHB, 128, HID, HID);
      mma_commit(&bar_mma);
    }
    ok = __syncthreads_and(mbar_wait(&bar_mma, phase));
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!ok) break;
    const int64_t OW = layer == 3 ? OW3 : OW2;
    for (int c0 = 0; c0 < HID; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + lane_base + c0, v);  // dW[o = tid][i = c0 + j]
      for (int j = 0; j < 32; ++j) atomicAdd(a.grad + OW + (int64_t)tid * HID + c0 + j, v[j]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // all reads of sWA / sHA by the MMAs are complete; rewrite them
    asm volatile("tcgen05.fence::after_thread_sync;");
    relu_back(tmem + 128, Hin + row * HID, valid, sHA, sWA, a.grad + (layer == 3 ? OB2 : OB1), tid);
  }
  // layer 1: dW1 = dZ1^T X (M = 128 out, N = 16 in, K = rows)
  if (ok) {
    write_rowT(sWB, a.X + row * IN, valid, IN, tid);
    tc_sync();
    if (tid == 0) {
      gemm(tmem, sWA, sWB, 128, IN, 128);
      mma_commit(&bar_mma);
    }
    ok = __syncthreads_and(mbar_wait(&bar_mma, phase));
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
      float v[32];
      tmem_ld32(tmem + lane_base, v);  // columns 0..15 hold dW1[o = tid][i]
      for (int i = 0; i < IN; ++i) atomicAdd(a.grad + OW1 + (int64_t)tid * IN + i, v[i]);
    }
  }
  if (!ok) {
    if (tid == 0) atomicExch(a.err, 1);
    mbar_wait(&bar_mma, phase);
  }
  tmem_free_warp0(tmem, 256);
}

// ------------------------------------------------------------------ Adam + operand packing
__device__ __forceinline__ void pack_param(int64_t i, float p, uint8_t* wpack) {
  int layer = -1, o = 0, in = 0, nin = 0, nout = 0;
  if (i < OB1) {
    layer = 0, nin = IN, nout = HID, o = (int)(i / IN), in = (int)(i % IN);
  } else if (i >= OW2 && i < OB2) {
    layer = 1, nin = HID, nout = HID, o = (int)((i - OW2) / HID), in = (int)((i - OW2) % HID);
  } else if (i >= OW3 && i < OB3) {
    layer = 2, nin = HID, nout = HID, o = (int)((i - OW3) / HID), in = (int)((i - OW3) % HID);
  } else if (i >= OW4 && i < OB4) {
    layer = 3, nin = HID, nout = OUT, o = (int)((i - OW4) / HID), in = (int)((i - OW4) % HID);
  }
  if (layer < 0) return;
  const uint16_t b = bf16_bits(p);
  const uint32_t pf[4] = {PF1, PF2, PF3, PF4};
  *reinterpret_cast<uint16_t*>(wpack + pf[layer] + kmaj(o, in, nin)) = b;
  if (layer > 0) {
    const uint32_t pt[4] = {0, PT2, PT3, PT4};
    *reinterpret_cast<uint16_t*>(wpack + pt[layer] + kmaj(in, o, nout)) = b;
  }
}

__global__ void k_pack(const float* __restrict__ params, uint8_t* __restrict__ wpack) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < NPARAM; i += (int64_t)gridDim.x * blockDim.x)
    pack_param(i, params[i], wpack);
}

__global__ void k_adam(float* __restrict__ params, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ grad, float lr, float c1, float c2, uint8_t* __restrict__ wpack) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < NPARAM; i += (int64_t)gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float mi = 0.9f * m[i] + 0.1f * g;
    const float vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    const float p = params[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    params[i] = p;
    pack_param(i, p, wpack);
  }
}

// ------------------------------------------------------------------ mesh features / prediction
// Base column quantities q = (ln(H/1000), asinh(1000 s_x)/4, asinh(1000 s_y)/4, ln(beta/1000)), [4][nv].
__global__ void k_feature_base(const double* __restrict__ acc, const double* __restrict__ thick,
                               const double* __restrict__ beta, int nv, double* __restrict__ q) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nv) return;
  const double w = acc[2 * nv + a];
  q[a] = log(thick[a] / 1000.0);
  q[nv + a] = 0.25 * asinh(1000.0 * acc[a] / w);
  q[2 * nv + a] = 0.25 * asinh(1000.0 * acc[nv + a] / w);
  q[3 * nv + a] = log(fmax(beta[a], 1e-30) / 1000.0);
}

// One Jacobi smoothing sweep of the 4 quantities: mean over the closed neighbourhood of each vertex.
__global__ void k_feature_smooth(const int32_t* __restrict__ nbr_ptr, const int32_t* __restrict__ nbr_idx, int nv,
                                 const double* __restrict__ in, double* __restrict__ out) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nv) return;
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  const int b0 = nbr_ptr[a], b1 = nbr_ptr[a + 1];
  for (int k = b0; k < b1; ++k) {
    const int b = nbr_idx[k];
    s0 += in[b];
    s1 += in[nv + b];
    s2 += in[2 * nv + b];
    s3 += in[3 * nv + b];
  }
  const double inv = 1.0 / (b1 - b0);
  out[a] = s0 * inv;
  out[nv + a] = s1 * inv;
  out[2 * nv + a] = s2 * inv;
  out[3 * nv + a] = s3 * inv;
}

// 16 BF16 features: hi/lo BF16 splits of the 4 local quantities (about 16 significant bits each),
// the 4 quantities averaged over ~5 km (8 sweeps), ln beta and the surface slope averaged over ~15 km
// (40 sweeps), and sigma_1 (the layering).
__global__ void k_feature_pack(const double* __restrict__ q, const double* __restrict__ q8,
                               const double* __restrict__ q40, const double* __restrict__ sigma, int nv,
                               uint16_t* __restrict__ X) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nv) return;
  uint16_t* x = X + (int64_t)a * IN;
  for (int k = 0; k < 4; ++k) {
    const float v = (float)q[k * nv + a];
    const uint16_t hi = bf16_bits(v);
    x[2 * k] = hi;
    x[2 * k + 1] = bf16_bits(v - bf16_val(hi));
  }
  for (int k = 0; k < 4; ++k) x[8 + k] = bf16_bits((float)q8[k * nv + a]);
  x[12] = bf16_bits((float)q40[3 * nv + a]);
  x[13] = bf16_bits((float)q40[nv + a]);
  x[14] = bf16_bits((float)q40[2 * nv + a]);
  x[15] = bf16_bits((float)sigma[1]);
}

// Structured decoder: per component c the network scales the sliding part b_c = u_sia,c(bed) and the
// deformation part d_c(sigma) = u_sia,c(sigma) - b_c of the shallow-ice profile,
//   u_c(sigma_l) = (1 + y[2c]) b_c + (1 + y[2c + 1]) d_c(sigma_l),
// so the predicted column keeps a physically consistent vertical profile.
__global__ void k_scatter_prediction(const float* __restrict__ Y, const double* __restrict__ Usia, int nv, int L,
                                     double* __restrict__ U) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nv) return;
  const int64_t base = 2LL * a * (L + 1);
  for (int c = 0; c < 2; ++c) {
    const double sb = 1.0 + (double)Y[(int64_t)a * OUT + 2 * c], sd = 1.0 + (double)Y[(int64_t)a * OUT + 2 * c + 1];
    const double b = Usia[base + c];
    for (int l = 0; l <= L; ++l) U[base + 2 * l + c] = sb * b + sd * (Usia[base + 2 * l + c] - b);
  }
}

// Decoder training targets: per column and component, the scales (s_b, s_d) of the shallow-ice
// sliding part b (the bed value, at every level) and deformation part d = u_sia - b that minimise
//   |s_b b + s_d d - u|^2 + reg^2 (|b|^2 (s_b - 1)^2 + |d|^2 (s_d - 1)^2)
// (2 x 2 normal equations, solved in FP64 by Cramer's rule; a numerically singular system keeps
// s = 1), written as y = s - 1 clipped to [-5, 5] in T[a][0..3]; T[a][4..31] = 0.
// d = a - b (the step from the shallow-ice guess to the network's, for the energy judge)
__global__ void k_diff(const double* __restrict__ a, const double* __restrict__ b, int64_t n, double* __restrict__ d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = a[i] - b[i];
}

__global__ void k_profile_scales(const double* __restrict__ U, const double* __restrict__ Usia, int nv, int L,
                                 double reg2, float* __restrict__ T) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nv) return;
  const int64_t base = 2LL * a * (L + 1);
  float* t = T + (int64_t)a * OUT;
  for (int c = 0; c < 2; ++c) {
    const double b = Usia[base + c];
    double bb = 0.0, dd = 0.0, bd = 0.0, ub = 0.0, ud = 0.0;
    for (int l = 0; l <= L; ++l) {
      const double d = Usia[base + 2 * l + c] - b, u = U[base + 2 * l + c];
      bb += b * b;
      dd += d * d;
      bd += b * d;
      ub += u * b;
      ud += u * d;
    }
    const double a11 = (1.0 + reg2) * bb, a22 = (1.0 + reg2) * dd, a12 = bd;
    const double r1 = ub + reg2 * bb, r2 = ud + reg2 * dd;
    const double det = a11 * a22 - a12 * a12;
    double sb = 1.0, sd = 1.0;
    if (det > 1e-30 * (a11 * a22 + 1e-300)) {
      sb = (r1 * a22 - r2 * a12) / det;
      sd = (a11 * r2 - a12 * r1) / det;
    }
    t[2 * c] = (float)fmin(fmax(sb - 1.0, -5.0), 5.0);
    t[2 * c + 1] = (float)fmin(fmax(sd - 1.0, -5.0), 5.0);
  }
  for (int j = 4; j < OUT; ++j) t[j] = 0.f;
}

uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

}  // namespace

struct bp_mlp {
  int device = 0;
  float *params = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  uint8_t* wpack = nullptr;
  int64_t step = 0;
  int64_t cap = 0;  // rows of the activation buffers
  uint16_t *H1 = nullptr, *H2 = nullptr, *H3 = nullptr;
  float* Y = nullptr;
  double* loss = nullptr;
  int* err = nullptr;
  double* host = nullptr;
  std::vector<void*> allocs;
};

namespace {

template <class T>
int mlp_alloc(bp_mlp* n, T** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return BP_ENOMEM;
  }
  n->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return BP_OK;
}

int ensure_rows(bp_mlp* net, int64_t n) {
  if (n <= net->cap) return BP_OK;
  for (void* p : {(void*)net->H1, (void*)net->H2, (void*)net->H3, (void*)net->Y}) {
    if (!p) continue;
    auto it = std::find(net->allocs.begin(), net->allocs.end(), p);
    if (it != net->allocs.end()) net->allocs.erase(it);
    cudaFree(p);
  }
  net->H1 = net->H2 = net->H3 = nullptr;
  net->Y = nullptr;
  net->cap = 0;
  int rc;
  if ((rc = mlp_alloc(net, &net->H1, n * HID)) || (rc = mlp_alloc(net, &net->H2, n * HID)) ||
      (rc = mlp_alloc(net, &net->H3, n * HID)) || (rc = mlp_alloc(net, &net->Y, n * OUT)))
    return rc;
  net->cap = n;
  return BP_OK;
}

int launch_forward(bp_mlp* net, const uint16_t* X, int64_t n, float* Y, bool keep, cudaStream_t s) {
  BP_CUDA_TRY(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, FWD_SMEM));
  BP_CUDA_TRY(cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, BWD_SMEM));
  FwdArgs a{net->wpack, net->params, X, n, Y, keep ? net->H1 : nullptr, keep ? net->H2 : nullptr,
            keep ? net->H3 : nullptr, net->err};
  const int64_t ntiles = (n + 127) / 128;
  int nsm = 148;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, net->device);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, nsm));
  k_mlp_forward<<<grid, 128, FWD_SMEM, s>>>(a);
  BP_CUDA_TRY(cudaGetLastError());
  return BP_OK;
}

int gradient(bp_mlp* net, const uint16_t* X, const float* T, int64_t n, float* grad, cudaStream_t s) {
  int rc = ensure_rows(net, n);
  if (rc) return rc;
  if ((rc = launch_forward(net, X, n, net->Y, true, s))) return rc;
  BP_CUDA_TRY(cudaMemsetAsync(grad, 0, NPARAM * sizeof(float), s));
  BP_CUDA_TRY(cudaMemsetAsync(net->loss, 0, sizeof(double), s));
  BwdArgs b{net->wpack, X, net->H1, net->H2, net->H3, net->Y, T, n, 2.0f / (float)n, grad, net->loss, net->err};
  k_mlp_backward<<<(unsigned)((n + 127) / 128), 128, BWD_SMEM, s>>>(b);
  BP_CUDA_TRY(cudaGetLastError());
  return BP_OK;
}

int check_err(bp_mlp* net, cudaStream_t s) {
  int e = 0;
  BP_CUDA_TRY(cudaMemcpyAsync(net->host, net->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  BP_CUDA_TRY(cudaStreamSynchronize(s));
  std::memcpy(&e, net->host, sizeof(int));
  if (e) {
    bp_set_last_cuda_error(cudaErrorLaunchTimeout, "tensor-core wait timed out", __LINE__);
    return BP_ECUDA;
  }
  return BP_OK;
}

}  // namespace

extern "C" int64_t bp_mlp_param_count(void) { return NPARAM; }

extern "C" void bp_mlp_free(bp_mlp* net) {
  if (!net) return;
  bp_device_guard g(net->device);
  cudaDeviceSynchronize();
  for (void* p : net->allocs) cudaFree(p);
  if (net->host) cudaFreeHost(net->host);
  delete net;
}

extern "C" int bp_mlp_set_params(bp_mlp* net, const float* host, int64_t n, void* stream) {
  if (!net || !host || n != NPARAM) return BP_EINVAL;
  bp_device_guard g(net->device);
  cudaStream_t s = (cudaStream_t)stream;
  BP_CUDA_TRY(cudaMemcpyAsync(net->params, host, NPARAM * sizeof(float), cudaMemcpyHostToDevice, s));
  BP_CUDA_TRY(cudaMemsetAsync(net->m, 0, NPARAM * sizeof(float), s));
  BP_CUDA_TRY(cudaMemsetAsync(net->v, 0, NPARAM * sizeof(float), s));
  BP_CUDA_TRY(cudaMemsetAsync(net->wpack, 0, PT_END, s));
  k_pack<<<(NPARAM + 255) / 256, 256, 0, s>>>(net->params, net->wpack);
  BP_CUDA_TRY(cudaGetLastError());
  net->step = 0;
  BP_CUDA_TRY(cudaStreamSynchronize(s));
  return BP_OK;
}

extern "C" int bp_mlp_get_params(const bp_mlp* net, float* host, int64_t n, void* stream) {
  if (!net || !host || n != NPARAM) return BP_EINVAL;
  bp_device_guard g(net->device);
  cudaStream_t s = (cudaStream_t)stream;
  BP_CUDA_TRY(cudaMemcpyAsync(host, net->params, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, s));
  BP_CUDA_TRY(cudaStreamSynchronize(s));
  return BP_OK;
}

// Parameters on disk: the NumPy .npy format (version 1.0) of a little-endian float32 vector of
// NPARAM entries, so that numpy.save / numpy.load read and write the same files.
namespace {
std::string npy_header() {
  std::string h = "{'descr': '<f4', 'fortran_order': False, 'shape': (" + std::to_string(NPARAM) + ",), }";
  const size_t pre = 10;  // magic (6), version (2), header length (2)
  while ((pre + h.size() + 1) % 64 != 0) h.push_back(' ');
  h.push_back('\n');
  return h;
}
}  // namespace

extern "C" int bp_mlp_save(const bp_mlp* net, const char* path) {
  if (!net || !path) return BP_EINVAL;
  std::vector<float> p(NPARAM);
  int rc = bp_mlp_get_params(net, p.data(), NPARAM, nullptr);
  if (rc) return rc;
  const std::string h = npy_header();
  FILE* f = std::fopen(path, "wb");
  if (!f) return BP_EIO;
  const unsigned char magic[8] = {0x93, 'N', 'U', 'M', 'P', 'Y', 1, 0};
  const unsigned char hl[2] = {(unsigned char)(h.size() & 0xFF), (unsigned char)(h.size() >> 8)};
  bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hl, 1, 2, f) == 2 &&
            std::fwrite(h.data(), 1, h.size(), f) == h.size() &&
            std::fwrite(p.data(), sizeof(float), NPARAM, f) == (size_t)NPARAM;  // little-endian host
  ok = (std::fclose(f) == 0) && ok;
  return ok ? BP_OK : BP_EIO;
}

extern "C" int bp_mlp_load(bp_mlp* net, const char* path) {
  if (!net || !path) return BP_EINVAL;
  FILE* f = std::fopen(path, "rb");
  if (!f) return BP_EIO;
  struct Closer {
    FILE* f;
    ~Closer() { std::fclose(f); }
  } closer{f};
  unsigned char pre[8];
  if (std::fread(pre, 1, 8, f) != 8 || pre[0] != 0x93 || std::memcmp(pre + 1, "NUMPY", 5) != 0) return BP_EIO;
  size_t hlen = 0;
  if (pre[6] == 1) {
    unsigned char b[2];
    if (std::fread(b, 1, 2, f) != 2) return BP_EIO;
    hlen = b[0] | ((size_t)b[1] << 8);
  } else if (pre[6] == 2 || pre[6] == 3) {
    unsigned char b[4];
    if (std::fread(b, 1, 4, f) != 4) return BP_EIO;
    hlen = b[0] | ((size_t)b[1] << 8) | ((size_t)b[2] << 16) | ((size_t)b[3] << 24);
  } else {
    return BP_EIO;
  }
  if (hlen > 4096) return BP_EIO;
  std::string h(hlen, '\0');
  if (std::fread(&h[0], 1, hlen, f) != hlen) return BP_EIO;
  // the header must describe a C-ordered little-endian float32 vector of exactly NPARAM entries
  const std::string shape = "(" + std::to_string(NPARAM) + ",)";
  if (h.find("'<f4'") == std::string::npos || h.find("'fortran_order': False") == std::string::npos ||
      h.find(shape) == std::string::npos)
    return BP_EIO;
  std::vector<float> p(NPARAM);
  if (std::fread(p.data(), sizeof(float), NPARAM, f) != (size_t)NPARAM) return BP_EIO;
  return bp_mlp_set_params(net, p.data(), NPARAM, nullptr);
}

extern "C" int bp_mlp_create(uint64_t seed, bp_mlp** out) {
  if (!out) return BP_EINVAL;
  *out = nullptr;
  auto* net = new bp_mlp();
  BP_CUDA_TRY(cudaGetDevice(&net->device));
  int rc;
  if ((rc = mlp_alloc(net, &net->params, NPARAM)) || (rc = mlp_alloc(net, &net->m, NPARAM)) ||
      (rc = mlp_alloc(net, &net->v, NPARAM)) || (rc = mlp_alloc(net, &net->grad, NPARAM)) ||
      (rc = mlp_alloc(net, &net->wpack, PT_END)) || (rc = mlp_alloc(net, &net->loss, 1)) ||
      (rc = mlp_alloc(net, &net->err, 1))) {
    bp_mlp_free(net);
    return rc;
  }
  if (cudaMallocHost(&net->host, 64) != cudaSuccess) {
    cudaGetLastError();
    bp_mlp_free(net);
    return BP_ENOMEM;
  }
  if (cudaMemset(net->err, 0, sizeof(int)) != cudaSuccess) {
    bp_mlp_free(net);
    return BP_ECUDA;
  }
  // He-uniform weights U(-sqrt(6 / fan_in), +sqrt(6 / fan_in)) from SplitMix64(seed, index); zero biases
  std::vector<float> p(NPARAM, 0.f);
  auto fill = [&](int64_t off, int64_t count, int fan_in) {
    const double lim = std::sqrt(6.0 / fan_in);
    for (int64_t i = 0; i < count; ++i) {
      const uint64_t r = splitmix64(seed * 0x100000001B3ull + (uint64_t)(off + i));
      const double u = (double)(r >> 11) * (1.0 / 9007199254740992.0);
      p[off + i] = (float)((2.0 * u - 1.0) * lim);
    }
  };
  fill(OW1, HID * IN, IN);
  fill(OW2, HID * HID, HID);
  fill(OW3, HID * HID, HID);
  fill(OW4, OUT * HID, HID);
  rc = bp_mlp_set_params(net, p.data(), NPARAM, nullptr);
  if (rc) {
    bp_mlp_free(net);
    return rc;
  }
  *out = net;
  return BP_OK;
}

extern "C" int bp_mlp_forward(bp_mlp* net, const uint16_t* X, int64_t n, float* Y, void* stream) {
  if (!net || !X || !Y || n < 1 || !bp_aligned16(X) || !bp_aligned16(Y)) return BP_EINVAL;
  bp_device_guard g(net->device);
  return launch_forward(net, X, n, Y, false, (cudaStream_t)stream);
}

extern "C" int bp_mlp_gradient(bp_mlp* net, const uint16_t* X, const float* T, int64_t n, float* grad,
                               double* loss_host, void* stream) {
  if (!net || !X || !T || !grad || n < 1 || !bp_aligned16(X)) return BP_EINVAL;
  bp_device_guard g(net->device);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = gradient(net, X, T, n, grad, s);
  if (rc) return rc;
  if (loss_host) {
    BP_CUDA_TRY(cudaMemcpyAsync(net->host + 1, net->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    if ((rc = check_err(net, s))) return rc;
    *loss_host = net->host[1];
  }
  return BP_OK;
}

extern "C" int bp_mlp_train_step(bp_mlp* net, const uint16_t* X, const float* T, int64_t n, float lr, void* stream) {
  if (!net || !X || !T || n < 1 || !bp_aligned16(X) || !(lr > 0)) return BP_EINVAL;
  bp_device_guard g(net->device);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = gradient(net, X, T, n, net->grad, s);
  if (rc) return rc;
  net->step += 1;
  const float c1 = 1.f - std::pow(0.9f, (float)net->step), c2 = 1.f - std::pow(0.999f, (float)net->step);
  k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(net->params, net->m, net->v, net->grad, lr, c1, c2, net->wpack);
  BP_CUDA_TRY(cudaGetLastError());
  return BP_OK;
}

extern "C" int bp_mlp_features(bp_mesh* m, uint16_t* X, void* stream) {
  if (!m || !X) return BP_EINVAL;
  if (m->nl != BP_MLP_LEVELS - 1) return BP_EUNSUP;
  bp_device_guard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  double* acc = nullptr;
  int rc = bp_nodal_surface_gradient(m, &acc, s);
  if (rc) return rc;
  if (!m->mlp_q) {
    if ((rc = bp_alloc(m, &m->mlp_q, 16 * (size_t)m->nv))) return rc;
  }
  double *q = m->mlp_q, *q8 = q + 4 * (size_t)m->nv, *q40 = q + 8 * (size_t)m->nv, *tmp = q + 12 * (size_t)m->nv;
  const int gb = (m->nv + 127) / 128;
  k_feature_base<<<gb, 128, 0, s>>>(acc, m->thick, m->beta, m->nv, q);
  const double* src = q;
  for (int it = 0; it < 40; ++it) {  // ping-pong between q8/q40 and tmp; after 8 sweeps keep a copy in q8
    double* dst = (it % 2 == 0) ? tmp : q40;
    k_feature_smooth<<<gb, 128, 0, s>>>(m->nbr_ptr, m->nbr_idx, m->nv, src, dst);
    src = dst;
    if (it == 7) BP_CUDA_TRY(cudaMemcpyAsync(q8, dst, 4 * (size_t)m->nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  k_feature_pack<<<gb, 128, 0, s>>>(q, q8, q40, m->sigma, m->nv, X);
  BP_CUDA_TRY(cudaGetLastError());
  return BP_OK;
}

namespace {
// U = decoder(Y, shallow-ice guess), the guess computed into Usia (workspace)
int decode_with_sia(bp_mesh* m, const float* Y, double* Usia, double* U, cudaStream_t s) {
  int rc = bp_initial_guess(m, BP_GUESS_SIA, Usia, s);
  if (rc) return rc;
  k_scatter_prediction<<<(m->nv + 127) / 128, 128, 0, s>>>(Y, Usia, m->nv, m->nl, U);
  BP_CUDA_TRY(cudaGetLastError());
  return BP_OK;
}
}  // namespace

extern "C" int bp_learned_decode(bp_mesh* m, const float* Y, double* U, void* stream) {
  if (!m || !Y || !U || !bp_aligned16(U)) return BP_EINVAL;
  bp_device_guard g(m->device);
  uint16_t* X = nullptr;
  float* Yw = nullptr;
  double *Usia = nullptr, *R = nullptr, *red = nullptr;
  int rc = bp_learned_scratch(m, &X, &Yw, &Usia, &R, &red);
  if (rc) return rc;
  return decode_with_sia(m, Y, Usia, U, (cudaStream_t)stream);
}

extern "C" int bp_learned_targets(bp_mesh* m, const double* U, double reg, float* T, void* stream) {
  if (!m || !U || !T || !bp_aligned16(U) || !(reg >= 0) || !std::isfinite(reg)) return BP_EINVAL;
  bp_device_guard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  uint16_t* X = nullptr;
  float* Yw = nullptr;
  double *Usia = nullptr, *R = nullptr, *red = nullptr;
  int rc = bp_learned_scratch(m, &X, &Yw, &Usia, &R, &red);
  if (rc) return rc;
  if ((rc = bp_initial_guess(m, BP_GUESS_SIA, Usia, s))) return rc;
  k_profile_scales<<<(m->nv + 127) / 128, 128, 0, s>>>(U, Usia, m->nv, m->nl, reg * reg, T);
  BP_CUDA_TRY(cudaGetLastError());
  return BP_OK;
}

extern "C" int bp_initial_guess_learned(bp_mesh* m, bp_mlp* net, double* U, int judge, int* used, void* stream) {
  if (!m || !net || !U || !bp_aligned16(U)) return BP_EINVAL;
  if (judge < BP_JUDGE_RESIDUAL || judge > BP_JUDGE_NONE) return BP_EINVAL;
  if (m->nl != BP_MLP_LEVELS - 1) return BP_EUNSUP;
  bp_device_guard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  uint16_t* X = nullptr;
  float* Y = nullptr;
  double *Usia = nullptr, *R = nullptr, *red = nullptr;
  int rc = bp_learned_scratch(m, &X, &Y, &Usia, &R, &red);
  if (rc) return rc;
  if ((rc = bp_mlp_features(m, X, s))) return rc;
  if ((rc = launch_forward(net, X, m->nv, Y, false, s))) return rc;
  if ((rc = decode_with_sia(m, Y, Usia, U, s))) return rc;
  if ((rc = check_err(net, s))) return rc;
  // the FP64 residual norm (or the FP64 energy) judges the prediction against the shallow-ice guess
  bool keep = true;
  if (judge == BP_JUDGE_RESIDUAL) {
    double f_mlp, f_sia;
    if ((rc = bp_assemble_residual(m, U, R, s)) || (rc = bp_norm2_host(m, R, s, &f_mlp))) return rc;
    if ((rc = bp_assemble_residual(m, Usia, R, s)) || (rc = bp_norm2_host(m, R, s, &f_sia))) return rc;
    keep = std::isfinite(f_mlp) && f_mlp <= f_sia;
  } else if (judge == BP_JUDGE_ENERGY) {
    // Pi_h(U_net) <= Pi_h(U_sia) decided by the sign of the energy change from the shallow-ice guess
    // to the network's, formed term by term in FP64-accurate pairs (one pass instead of two full
    // energies, and exact where the two energies agree to many digits)
    k_diff<<<(int)std::min<int64_t>((m->ndof + 255) / 256, 148 * 16), 256, 0, s>>>(U, Usia, m->ndof, R);
    BP_CUDA_TRY(cudaGetLastError());
    double dE;
    if ((rc = bp_energy_change_ex(m, Usia, R, 1.0, BP_F64X2_DS, &dE, s))) return rc;
    keep = std::isfinite(dE) && dE <= 0.0;
  }
  if (!keep) BP_CUDA_TRY(cudaMemcpyAsync(U, Usia, m->ndof * sizeof(double), cudaMemcpyDeviceToDevice, s));
  BP_CUDA_TRY(cudaStreamSynchronize(s));
  if (used) *used = keep ? 1 : 0;
  return BP_OK;
}
