// Inference of the interpolation network on the fifth-generation tensor
// cores (tcgen05): Y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for every row x
// of a BF16 feature matrix X [M x 64], FP32 accumulation, Y [M x 16] FP32.
// The network proposes the P-row and Q-column weights of a fine point in
// place of the least-squares fit of eq. ls_interpolation (not in the paper).
//
// Mapping (one CTA of 8 warps, persistent over 128-row tiles, four CTAs per
// SM):
//  * the three weight matrices are converted to BF16 once per CTA and kept
//    in shared memory in the 128-byte-swizzled K-major layout of the MMA
//    operands (a row of 64 BF16 = 128 bytes, 8-row groups 1024 bytes apart,
//    the 16-byte chunk c of row r stored at chunk c ^ (r mod 8));
//  * the feature tile [128 x 64] is brought in by TMA (cp.async.bulk.tensor,
//    same swizzle, rows past M zero-filled), double buffered so the next
//    tile loads while the current one is computed; once the first layer has
//    consumed it, the same buffer holds the hidden activations of the tile;
//  * one thread issues the MMAs (M = 128, K = 16 per instruction, four per
//    layer) with the accumulators in tensor memory: layer 1 in columns
//    0-63, layer 2 in 64-127, layer 3 (N = 16) again in 0-15;
//  * after each MMA group completes (tcgen05.commit on an mbarrier), the
//    threads read the accumulator (tcgen05.ld; warps w and w + 4 share the
//    TMEM lanes 32(w mod 4).., one half of the columns each), add the bias,
//    apply ReLU and write BF16 rows into the swizzled A-operand tile of the
//    next layer; the last layer's row goes straight to global memory.
// Every wait is bounded (2 s of globaltimer); a CTA that gives up sets
// *err, waits (bounded) for its copies and MMAs in flight, frees its tensor
// memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <atomic>
#include <mutex>

#include "internal.cuh"
#include "mlp_layout.cuh"

namespace bamg {

namespace {

constexpr int kTileM = 128;
constexpr int kTcThreads = 256;
constexpr uint32_t kTmemCols = 128;
constexpr uint32_t kTileBytes = kTileM * 128;            // 128 rows of 64 BF16
// shared memory map (byte offsets from a 1024-byte aligned base)
constexpr uint32_t kOffW1 = 0;                           // 64 rows
constexpr uint32_t kOffW2 = kOffW1 + 64 * 128;           // 64 rows
constexpr uint32_t kOffW3 = kOffW2 + 64 * 128;           // 16 rows
constexpr uint32_t kOffX0 = kOffW3 + 16 * 128;           // feature / activation tile, buffer 0
constexpr uint32_t kOffX1 = kOffX0 + kTileBytes;         // buffer 1
constexpr uint32_t kOffBias = kOffX1 + kTileBytes;       // b1, b2, b3 (FP32)
constexpr uint32_t kOffBar = kOffBias + 1024;            // mbarriers, TMEM address
constexpr uint32_t kSmemUsed = kOffBar + 64;
constexpr uint32_t kSmemAlloc = kSmemUsed + 1024;        // slack for the 1024-byte alignment
static_assert(kOffX0 % 1024 == 0 && kOffX1 % 1024 == 0, "operand tiles 1024-aligned");

constexpr unsigned long long kWaitNs = 2000000000ull;    // bound of every wait

__device__ inline unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of the 16-byte chunk c (0..7) of row r in a swizzled tile
__device__ inline uint32_t sw128(int r, int c) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}

// shared-memory matrix descriptor of a K-major, 128-byte-swizzled operand
// tile at shared address a: start address, leading byte offset 16 (unused
// when K fits one swizzle row), stride byte offset 1024 (8-row groups),
// descriptor version 1, swizzle mode 2 (128 bytes)
__device__ inline uint64_t sdesc(uint32_t a) {
  return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ inline void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ inline void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// true once the phase with the given parity has completed; false after kWaitNs
__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = now_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (now_ns() - t0 > kWaitNs) return false;
  }
}

__device__ inline void tma_load_tile(uint32_t dst, const CUtensorMap* map, int row0, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(row0), "r"(bar)
      : "memory");
}

__device__ inline void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      ::"r"(d), "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ inline void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ inline void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ inline void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ inline void tmem_ld16(uint32_t ta, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
}
__device__ inline void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ inline uint32_t pack2(float lo, float hi) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16(lo)) |
         ((uint32_t)__bfloat16_as_ushort(__float2bfloat16(hi)) << 16);
}

// rows x 64 FP32 weights (row-major, output-major) -> swizzled BF16 operand
__device__ inline void stage_weights(uint8_t* base, uint32_t off, const float* __restrict__ W, int rows) {
  for (int e = threadIdx.x; e < rows * 8; e += blockDim.x) {
    const int r = e >> 3, c = e & 7;
    const float* w = W + r * 64 + c * 8;
    uint4 v = make_uint4(pack2(w[0], w[1]), pack2(w[2], w[3]), pack2(w[4], w[5]), pack2(w[6], w[7]));
    *reinterpret_cast<uint4*>(base + off + sw128(r, c)) = v;
  }
}

// accumulator columns [32 h, 32 h + 32) of this thread's row, + bias, ReLU,
// BF16 into row `row` of the swizzled tile at `off`
__device__ inline void hidden_epilogue(uint8_t* base, uint32_t off, uint32_t tacc, const float* bias, int row,
                                       int h) {
  uint32_t r[32];
  tmem_ld16(tacc + 32 * h, *reinterpret_cast<uint32_t(*)[16]>(r + 0));
  tmem_ld16(tacc + 32 * h + 16, *reinterpret_cast<uint32_t(*)[16]>(r + 16));
  tmem_wait_ld();
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = fmaxf(__uint_as_float(r[8 * c + q]) + bias[32 * h + 8 * c + q], 0.f);
    *reinterpret_cast<uint4*>(base + off + sw128(row, 4 * h + c)) =
        make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
  }
}

// four K = 16 steps of one layer: D[tmem] (+)= A[a_off] B[b_off]^T
__device__ inline void issue_layer(uint32_t sbase, uint32_t a_off, uint32_t b_off, uint32_t dtm, uint32_t id) {
  const uint64_t a = sdesc(sbase + a_off), b = sdesc(sbase + b_off);
#pragma unroll
  for (int k = 0; k < 4; ++k) mma_bf16(dtm, a + 2 * k, b + 2 * k, id, k > 0 ? 1u : 0u);   // +32 bytes per step
}

}  // namespace

__global__ void __launch_bounds__(kTcThreads, 4)
mlp_forward_tc_kernel(const __grid_constant__ CUtensorMap xmap, int M, const float* __restrict__ P,
                      float* __restrict__ Y, int* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ uint8_t dyn_smem[];
  uint8_t* base = dyn_smem + ((1024 - (smem_u32(dyn_smem) & 1023)) & 1023);
  const uint32_t sbase = smem_u32(base);
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t bar_x0 = sbase + kOffBar, bar_x1 = bar_x0 + 8, bar_mma = bar_x0 + 16;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + kOffBar + 24);
  float* bias = reinterpret_cast<float*>(base + kOffBias);

  if (tid == 0) {
    mbar_init(bar_x0, 1);
    mbar_init(bar_x1, 1);
    mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  stage_weights(base, kOffW1, P + kW1, 64);
  stage_weights(base, kOffW2, P + kW2, 64);
  stage_weights(base, kOffW3, P + kW3, 16);
  for (int i = tid; i < kH; i += blockDim.x) {
    bias[i] = P[kB1 + i];
    bias[64 + i] = P[kB2 + i];
  }
  if (tid < kO) bias[128 + tid] = P[kB3 + tid];
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const int row = tid & (kTileM - 1), half = tid >> 7;
  const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;   // this warp's TMEM lanes
  const uint32_t id64 = idesc_bf16(kTileM, 64), id16 = idesc_bf16(kTileM, 16);

  const int ntiles = (M + kTileM - 1) / kTileM;
  uint32_t par_x[2] = {0u, 0u};   // thread 0: next parity of each feature buffer
  bool pend[2] = {false, false};  // thread 0: a copy into that buffer is in flight
  uint32_t par_m = 0u;            // parity of the next MMA completion
  bool mma_pending = false;
  bool ok = true;
  if (tid == 0 && (int)blockIdx.x < ntiles) {
    mbar_expect_tx(bar_x0, kTileBytes);
    tma_load_tile(sbase + kOffX0, &xmap, (int)blockIdx.x * kTileM, bar_x0);
    pend[0] = true;
  }
  int it = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int b = it & 1;
    const uint32_t offx = b ? kOffX1 : kOffX0;
    const uint32_t barx = b ? bar_x1 : bar_x0;
    bool mine = true;
    if (tid == 0) {
      const int tn = t + (int)gridDim.x;
      if (tn < ntiles) {                 // prefetch the next tile into the other buffer
        const uint32_t bo = b ? bar_x0 : bar_x1;
        mbar_expect_tx(bo, kTileBytes);
        tma_load_tile(sbase + (b ? kOffX0 : kOffX1), &xmap, tn * kTileM, bo);
        pend[b ^ 1] = true;
      }
      mine = mbar_wait(barx, par_x[b]);
      if (mine) {
        pend[b] = false;
        par_x[b] ^= 1u;
        fence_after_sync();
        issue_layer(sbase, offx, kOffW1, tmem + 0, id64);
        mma_commit(bar_mma);
        mma_pending = true;
      }
    }
    // layer 1 -> H1
    if (!__syncthreads_and(mine)) { ok = false; break; }
    mine = mbar_wait(bar_mma, par_m);
    if (!__syncthreads_and(mine)) { ok = false; break; }
    par_m ^= 1u;
    mma_pending = false;
    fence_after_sync();
    hidden_epilogue(base, offx, tmem + lane_off + 0, bias, row, half);
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      issue_layer(sbase, offx, kOffW2, tmem + 64, id64);
      mma_commit(bar_mma);
      mma_pending = true;
    }
    // layer 2 -> H2
    mine = mbar_wait(bar_mma, par_m);
    if (!__syncthreads_and(mine)) { ok = false; break; }
    par_m ^= 1u;
    mma_pending = false;
    fence_after_sync();
    hidden_epilogue(base, offx, tmem + lane_off + 64, bias + 64, row, half);
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      issue_layer(sbase, offx, kOffW3, tmem + 0, id16);
      mma_commit(bar_mma);
      mma_pending = true;
    }
    // layer 3 -> Y
    mine = mbar_wait(bar_mma, par_m);
    if (!__syncthreads_and(mine)) { ok = false; break; }
    par_m ^= 1u;
    mma_pending = false;
    fence_after_sync();
    if (half == 0) {
      uint32_t r[16];
      tmem_ld16(tmem + lane_off + 0, r);
      tmem_wait_ld();
      const int grow = t * kTileM + row;
      if (grow < M) {
        float4* y = reinterpret_cast<float4*>(Y + (size_t)grow * kO);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          y[q] = make_float4(__uint_as_float(r[4 * q + 0]) + bias[128 + 4 * q + 0],
                             __uint_as_float(r[4 * q + 1]) + bias[128 + 4 * q + 1],
                             __uint_as_float(r[4 * q + 2]) + bias[128 + 4 * q + 2],
                             __uint_as_float(r[4 * q + 3]) + bias[128 + 4 * q + 3]);
      }
    }
    fence_before_sync();
    __syncthreads();
  }
  // drain: copies and MMAs still in flight (only after a timeout), bounded
  if (tid == 0) {
    if (!ok) atomicExch(err, 1);
    for (int q = 0; q < 2; ++q)
      if (pend[q]) mbar_wait(q ? bar_x1 : bar_x0, par_x[q]);
    if (mma_pending) mbar_wait(bar_mma, par_m);
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry points (the
// library does not link the driver library itself)
EncodeTiledFn encode_tiled() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

std::atomic<uint64_t> g_tc_attr{0};

}  // namespace

// Y[M x 16] = network(X[M x 64] BF16) on the tensor cores; err_dev: one
// device int, set to 1 when a CTA gave up waiting (left 0 otherwise).
bamg_status mlp_forward_tc(int M, const float* P, const void* X, float* Y, int* err_dev, cudaStream_t s) {
  if (M <= 0) return BAMG_OK;
  if ((reinterpret_cast<uintptr_t>(X) & 15u) != 0 || (reinterpret_cast<uintptr_t>(Y) & 15u) != 0) {
    set_error("network features and outputs must be 16-byte aligned");
    return BAMG_ERR_ARG;
  }
  EncodeTiledFn enc = encode_tiled();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return BAMG_ERR_UNSUPPORTED;
  }
  CUtensorMap map;
  const cuuint64_t gdim[2] = {(cuuint64_t)kF, (cuuint64_t)M};
  const cuuint64_t gstride[1] = {(cuuint64_t)kF * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kF, (cuuint32_t)kTileM};
  const cuuint32_t estride[2] = {1, 1};
  CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(X), gdim, gstride, box, estride,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return BAMG_ERR_CUDA;
  }
  int max_dyn = 0;
  BAMG_TRY(allow_max_smem((const void*)mlp_forward_tc_kernel, g_tc_attr, &max_dyn));
  if ((int)kSmemAlloc > max_dyn) {
    set_error("network kernel needs %u bytes of shared memory, %d available", kSmemAlloc, max_dyn);
    return BAMG_ERR_UNSUPPORTED;
  }
  const int ntiles = (M + kTileM - 1) / kTileM;
  int grid = 4 * num_sms();
  if (grid > ntiles) grid = ntiles;
  return launch(mlp_forward_tc_kernel, dim3(grid), dim3(kTcThreads), (size_t)kSmemAlloc, s, map, M, P, Y, err_dev);
}

}  // namespace bamg
