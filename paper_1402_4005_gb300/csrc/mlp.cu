// Learned interpolation: a 3-layer MLP that proposes the weights of a fine
// point's row of P and column of Q from its local stencil (an extension to
// the least-squares fit of eq. ls_interpolation / Section 5, which produces
// its training targets and stays the fallback).
//
// Features of a fine point i on a grid level (64, stored as BF16):
//   [0, 25)  b_{i, i+o} / b_ii  for the 25 offsets o of the 5x5 box (row of B)
//   [25, 50) b_{i+o, i} / b_ii  (column of B, read from B^T)
//   [50, 58) 1 where the neighbour at the k-th offset of the 3x3 box is coarse
//   58       1 (constant), [59, 64) 0
// Outputs (16): slots 0..7 = P weights, 8..15 = Q weights, slot k for the
// k-th offset of the 3x3 box without its centre (row-major order), i.e. the
// order of J_i.  Q weights are shifted to sum to one (Section 5 constraint).
//
// Network 64 -> 64 -> 64 -> 16, ReLU, weights and activations BF16,
// products accumulated in FP32.  Inference runs on the tcgen05 tensor cores
// with TMEM accumulators (mlp_tc.cu).  The training kernel here uses
// mma.sync m16n8k16 tiles: one warp handles 16 points, layer outputs are
// handed to the next layer through shared memory.  Training: mean squared error on
// the used slots, gradients of all layers by the same warp tiles (block-local
// FP32 accumulation, one global add per block), Adam on FP32 master weights.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "hierarchy.cuh"
#include "mlp_layout.cuh"

namespace bamg {

constexpr int kMlpWarps = 4;
constexpr int kMlpThreads = kMlpWarps * 32;

__device__ inline uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ inline void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[16 x 8NT] += A[16 x K] B[K x 8NT]; A(i, k) and B(k, n) return BF16.
// Accumulator c[nt]: (g, 8nt+2t), (g, 8nt+2t+1), (g+8, 8nt+2t), (g+8, 8nt+2t+1)
// with g = lane / 4, t = lane % 4.
template <int K, int NT, typename FA, typename FB>
__device__ inline void warp_gemm(float (&c)[NT][4], FA A, FB B) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int ks = 0; ks < K / 16; ++ks) {
    const int k0 = ks * 16 + 2 * t;
    uint32_t a[4];
    a[0] = pack_bf16(A(g, k0), A(g, k0 + 1));
    a[1] = pack_bf16(A(g + 8, k0), A(g + 8, k0 + 1));
    a[2] = pack_bf16(A(g, k0 + 8), A(g, k0 + 9));
    a[3] = pack_bf16(A(g + 8, k0 + 8), A(g + 8, k0 + 9));
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      uint32_t b[2];
      b[0] = pack_bf16(B(k0, nt * 8 + g), B(k0 + 1, nt * 8 + g));
      b[1] = pack_bf16(B(k0 + 8, nt * 8 + g), B(k0 + 9, nt * 8 + g));
      mma16816(c[nt], a, b);
    }
  }
}

template <int NT>
__device__ inline void zero_acc(float (&c)[NT][4]) {
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.f;
}

// store an accumulator tile (16 x 8NT) with bias and optional ReLU into a
// row-major BF16 buffer (ld elements per row)
template <int NT>
__device__ inline void store_act(const float (&c)[NT][4], const float* bias, bool relu, __nv_bfloat16* out, int ld) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int row = g + (q >> 1) * 8, col = nt * 8 + 2 * t + (q & 1);
      float v = c[nt][q] + (bias ? bias[col] : 0.f);
      if (relu) v = fmaxf(v, 0.f);
      out[row * ld + col] = __float2bfloat16(v);
    }
}

struct MlpSmem {
  __nv_bfloat16 w1[kH * kF], w2[kH * kH], w3[kO * kH];
  float b1[kH], b2[kH], b3[kO];
};

__device__ inline void load_weights(MlpSmem& S, const float* __restrict__ P) {
  for (int i = threadIdx.x; i < kH * kF; i += blockDim.x) S.w1[i] = __float2bfloat16(P[kW1 + i]);
  for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) S.w2[i] = __float2bfloat16(P[kW2 + i]);
  for (int i = threadIdx.x; i < kO * kH; i += blockDim.x) S.w3[i] = __float2bfloat16(P[kW3 + i]);
  for (int i = threadIdx.x; i < kH; i += blockDim.x) { S.b1[i] = P[kB1 + i]; S.b2[i] = P[kB2 + i]; }
  for (int i = threadIdx.x; i < kO; i += blockDim.x) S.b3[i] = P[kB3 + i];
  __syncthreads();
}

struct WarpTile {
  __nv_bfloat16 x[16 * kF], h1[16 * kH], h2[16 * kH];
};

// Forward of one 16-point tile: x -> h1 -> h2 (BF16, shared) -> y (FP32 regs).
__device__ inline void forward_tile(const MlpSmem& S, WarpTile& T, float (&y)[2][4]) {
  float c[8][4];
  zero_acc(c);
  warp_gemm<kF, 8>(c, [&](int i, int k) { return T.x[i * kF + k]; },
                   [&](int k, int n) { return S.w1[n * kF + k]; });
  store_act(c, S.b1, true, T.h1, kH);
  __syncwarp();
  zero_acc(c);
  warp_gemm<kH, 8>(c, [&](int i, int k) { return T.h1[i * kH + k]; },
                   [&](int k, int n) { return S.w2[n * kH + k]; });
  store_act(c, S.b2, true, T.h2, kH);
  __syncwarp();
  zero_acc(y);
  warp_gemm<kH, 2>(y, [&](int i, int k) { return T.h2[i * kH + k]; },
                   [&](int k, int n) { return S.w3[n * kH + k]; });
  const int lane = threadIdx.x & 31, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) y[nt][q] += S.b3[nt * 8 + 2 * t + (q & 1)];
}

__device__ inline void load_tile_x(WarpTile& T, const __nv_bfloat16* __restrict__ X, int row0, int M) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < 16 * kF; e += 32) {
    int r = e / kF, k = e % kF;
    T.x[e] = row0 + r < M ? X[(size_t)(row0 + r) * kF + k] : __float2bfloat16(0.f);
  }
  __syncwarp();
}

struct GradSmem {
  float w1[kH * kF], w2[kH * kH], w3[kO * kH], b1[kH], b2[kH], b3[kO];
};

struct BackTile {
  __nv_bfloat16 d3[16 * kO], d2[16 * kH], d1[16 * kH];
};

// Sum over the lanes of one bias column: the two row halves in the lane,
// then the eight row groups g (lanes differing in bits 2-4), fixed order.
__device__ inline float bias_col_sum(float lo, float hi) {
  float v = lo + hi;
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 16);
  return v;
}

// Forward + backward on rows [0, M): writes this block's d(loss)/d(params)
// to part[blockIdx.x] (FP32, parameter layout) and adds the loss sum to
// loss[0].  loss = sum mask (y - t)^2 / count.  Each warp accumulates its
// tiles into its own shared copy without atomics and the block sums the
// copies in warp order, so the gradient does not depend on scheduling.
__global__ void __launch_bounds__(kMlpThreads) mlp_grad_kernel(int M, float inv_count, const float* __restrict__ P,
                                                               const __nv_bfloat16* __restrict__ X,
                                                               const float* __restrict__ Tg,
                                                               const float* __restrict__ mask,
                                                               float* __restrict__ part, float* __restrict__ loss) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ unsigned char dyn[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(dyn);
  GradSmem* Dall = reinterpret_cast<GradSmem*>(dyn + sizeof(MlpSmem));
  WarpTile* tiles = reinterpret_cast<WarpTile*>(dyn + sizeof(MlpSmem) + kMlpWarps * sizeof(GradSmem));
  BackTile* btiles =
      reinterpret_cast<BackTile*>(dyn + sizeof(MlpSmem) + kMlpWarps * sizeof(GradSmem) + kMlpWarps * sizeof(WarpTile));
  load_weights(S, P);
  for (int i = threadIdx.x; i < (int)(kMlpWarps * sizeof(GradSmem) / sizeof(float)); i += blockDim.x)
    reinterpret_cast<float*>(Dall)[i] = 0.f;
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  GradSmem& D = Dall[w];
  WarpTile& T = tiles[w];
  BackTile& Bk = btiles[w];
  float lsum = 0.f;
  const int ntiles = (M + 15) / 16;
  for (int tile = blockIdx.x * kMlpWarps + w; tile < ntiles; tile += gridDim.x * kMlpWarps) {
    const int row0 = tile * 16;
    load_tile_x(T, X, row0, M);
    float y[2][4];
    forward_tile(S, T, y);
    // dL/dy = 2 mask (y - t) / count
    {
      float dv[2][4];
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int r = g + (q >> 1) * 8, col = nt * 8 + 2 * t + (q & 1);
          int row = row0 + r;
          float d = 0.f;
          if (row < M) {
            float m = mask[(size_t)row * kO + col];
            float e = y[nt][q] - Tg[(size_t)row * kO + col];
            lsum += m * e * e;
            d = 2.f * m * e * inv_count;
          }
          Bk.d3[r * kO + col] = __float2bfloat16(d);
          dv[nt][q] = d;
        }
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float v = bias_col_sum(dv[nt][h], dv[nt][2 + h]);
          if (g == 0) D.b3[nt * 8 + 2 * t + h] += v;
        }
    }
    __syncwarp();
    // dW3 (16 x 64) += d3^T h2
    {
      float c[8][4];
      zero_acc(c);
      warp_gemm<16, 8>(c, [&](int i, int k) { return Bk.d3[k * kO + i]; },
                       [&](int k, int n) { return T.h2[k * kH + n]; });
#pragma unroll
      for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int i = g + (q >> 1) * 8, n = nt * 8 + 2 * t + (q & 1);
          D.w3[i * kH + n] += c[nt][q];
        }
    }
    // d2 = (d3 W3) * relu'(h2)
    {
      float c[8][4];
      zero_acc(c);
      warp_gemm<16, 8>(c, [&](int i, int k) { return Bk.d3[i * kO + k]; },
                       [&](int k, int n) { return S.w3[k * kH + n]; });
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        float vv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int r = g + (q >> 1) * 8, col = nt * 8 + 2 * t + (q & 1);
          float v = __bfloat162float(T.h2[r * kH + col]) > 0.f ? c[nt][q] : 0.f;
          Bk.d2[r * kH + col] = __float2bfloat16(v);
          vv[q] = v;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float v = bias_col_sum(vv[h], vv[2 + h]);
          if (g == 0) D.b2[nt * 8 + 2 * t + h] += v;
        }
      }
    }
    __syncwarp();
    // dW2 (64 x 64) += d2^T h1, four row tiles
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
      float c[8][4];
      zero_acc(c);
      warp_gemm<16, 8>(c, [&](int i, int k) { return Bk.d2[k * kH + mt * 16 + i]; },
                       [&](int k, int n) { return T.h1[k * kH + n]; });
#pragma unroll
      for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int i = mt * 16 + g + (q >> 1) * 8, n = nt * 8 + 2 * t + (q & 1);
          D.w2[i * kH + n] += c[nt][q];
        }
    }
    // d1 = (d2 W2) * relu'(h1)
    {
      float c[8][4];
      zero_acc(c);
      warp_gemm<kH, 8>(c, [&](int i, int k) { return Bk.d2[i * kH + k]; },
                       [&](int k, int n) { return S.w2[k * kH + n]; });
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        float vv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int r = g + (q >> 1) * 8, col = nt * 8 + 2 * t + (q & 1);
          float v = __bfloat162float(T.h1[r * kH + col]) > 0.f ? c[nt][q] : 0.f;
          Bk.d1[r * kH + col] = __float2bfloat16(v);
          vv[q] = v;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float v = bias_col_sum(vv[h], vv[2 + h]);
          if (g == 0) D.b1[nt * 8 + 2 * t + h] += v;
        }
      }
    }
    __syncwarp();
    // dW1 (64 x 64) += d1^T x
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
      float c[8][4];
      zero_acc(c);
      warp_gemm<16, 8>(c, [&](int i, int k) { return Bk.d1[k * kH + mt * 16 + i]; },
                       [&](int k, int n) { return T.x[k * kF + n]; });
#pragma unroll
      for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int i = mt * 16 + g + (q >> 1) * 8, n = nt * 8 + 2 * t + (q & 1);
          D.w1[i * kF + n] += c[nt][q];
        }
    }
    __syncwarp();
  }
  lsum = warp_sum(lsum);
  if (lane == 0) atomicAdd(loss, lsum * inv_count);   // reported only
  __syncthreads();
  float* out = part + (size_t)blockIdx.x * kNParam;
  auto wsum = [&](const float* (&src)[kMlpWarps], int i) {
    float v = 0.f;
#pragma unroll
    for (int k = 0; k < kMlpWarps; ++k) v += src[k][i];
    return v;
  };
  const float* s1[kMlpWarps];
  const float* s2[kMlpWarps];
  const float* s3[kMlpWarps];
  const float* c1[kMlpWarps];
  const float* c2[kMlpWarps];
  const float* c3[kMlpWarps];
#pragma unroll
  for (int k = 0; k < kMlpWarps; ++k) {
    s1[k] = Dall[k].w1; s2[k] = Dall[k].w2; s3[k] = Dall[k].w3;
    c1[k] = Dall[k].b1; c2[k] = Dall[k].b2; c3[k] = Dall[k].b3;
  }
  for (int i = threadIdx.x; i < kH * kF; i += blockDim.x) out[kW1 + i] = wsum(s1, i);
  for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) out[kW2 + i] = wsum(s2, i);
  for (int i = threadIdx.x; i < kO * kH; i += blockDim.x) out[kW3 + i] = wsum(s3, i);
  for (int i = threadIdx.x; i < kH; i += blockDim.x) { out[kB1 + i] = wsum(c1, i); out[kB2 + i] = wsum(c2, i); }
  for (int i = threadIdx.x; i < kO; i += blockDim.x) out[kB3 + i] = wsum(c3, i);
}

// G[i] += sum over the blocks of part[b][i], blocks in order.
__global__ void grad_reduce_kernel(int nb, const float* __restrict__ part, float* __restrict__ G) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNParam) return;
  float v = 0.f;
  for (int b = 0; b < nb; ++b) v += part[(size_t)b * kNParam + i];
  G[i] += v;
}

__global__ void adam_kernel(int np, float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ G, float lr, float b1, float b2, float eps, float c1, float c2) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  float gr = G[i];
  float mi = b1 * m[i] + (1.f - b1) * gr;
  float vi = b2 * v[i] + (1.f - b2) * gr * gr;
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// He initialisation from SplitMix64 (stream 8192): uniform(-a, a), a = sqrt(6 / fan_in); biases 0.
__global__ void mlp_init_kernel(float* __restrict__ P, uint64_t seed) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNParam) return;
  float a = 0.f;
  if (i < kB1) a = sqrtf(6.f / kF);
  else if (i >= kW2 && i < kB2) a = sqrtf(6.f / kH);
  else if (i >= kW3 && i < kB3) a = sqrtf(6.f / kH);
  P[i] = a == 0.f ? 0.f : (float)(a * splitmix_pm1(seed, 8192, (uint64_t)i));
}

// ------------------------------------------------------------ features
__device__ inline double find_entry(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                    const double* __restrict__ va, int i, int j) {
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] == j) return va[p];
  return 0.0;
}

// slot of the offset (di, dj) in the 3x3 box without its centre
__device__ inline int box_slot(int di, int dj) {
  int s = (di + 1) * 3 + (dj + 1);
  return s > 4 ? s - 1 : s;
}

__global__ void mlp_features_kernel(int n, int nx, int ny, const int32_t* __restrict__ brp, const int32_t* __restrict__ bci,
                                    const double* __restrict__ bva, const int32_t* __restrict__ trp,
                                    const int32_t* __restrict__ tci, const double* __restrict__ tva,
                                    const int8_t* __restrict__ cf, const int32_t* __restrict__ fidx,
                                    __nv_bfloat16* __restrict__ X) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || cf[i]) return;
  int row = fidx[i];
  int gi = i / ny, gj = i % ny;
  double dii = find_entry(brp, bci, bva, i, i);
  double inv = dii != 0.0 ? 1.0 / dii : 0.0;
  __nv_bfloat16* x = X + (size_t)row * kF;
  int k = 0;
  for (int di = -2; di <= 2; ++di)
    for (int dj = -2; dj <= 2; ++dj, ++k) {
      int a = gi + di, b = gj + dj;
      double rv = 0.0, cv = 0.0;
      if (a >= 0 && a < nx && b >= 0 && b < ny) {
        int j = a * ny + b;
        rv = find_entry(brp, bci, bva, i, j) * inv;
        cv = find_entry(trp, tci, tva, i, j) * inv;
      }
      x[k] = __float2bfloat16((float)rv);
      x[25 + k] = __float2bfloat16((float)cv);
    }
  for (int di = -1; di <= 1; ++di)
    for (int dj = -1; dj <= 1; ++dj) {
      if (di == 0 && dj == 0) continue;
      int a = gi + di, b = gj + dj;
      bool c = a >= 0 && a < nx && b >= 0 && b < ny && cf[a * ny + b];
      x[50 + box_slot(di, dj)] = __float2bfloat16(c ? 1.f : 0.f);
    }
  x[58] = __float2bfloat16(1.f);
  for (int q = 59; q < kF; ++q) x[q] = __float2bfloat16(0.f);
}

// Training targets: the LS weights of the level in slots, with a mask.
__global__ void mlp_targets_kernel(int n, int ny, const int8_t* __restrict__ cf, const int32_t* __restrict__ fidx,
                                   const int32_t* __restrict__ jrp, const int32_t* __restrict__ jci,
                                   const int32_t* __restrict__ prp, const double* __restrict__ pva,
                                   const double* __restrict__ qva, float* __restrict__ T, float* __restrict__ mask) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || cf[i]) return;
  int row = fidx[i];
  float* t = T + (size_t)row * kO;
  float* m = mask + (size_t)row * kO;
  for (int q = 0; q < kO; ++q) { t[q] = 0.f; m[q] = 0.f; }
  int gi = i / ny, gj = i % ny;
  int pq = prp[i];
  for (int e = jrp[i]; e < jrp[i + 1]; ++e, ++pq) {
    int j = jci[e];
    int di = j / ny - gi, dj = j % ny - gj;
    if (di < -1 || di > 1 || dj < -1 || dj > 1 || (di == 0 && dj == 0)) continue;
    int s = box_slot(di, dj);
    t[s] = (float)pva[pq];
    t[8 + s] = (float)qva[pq];
    m[s] = 1.f;
    m[8 + s] = 1.f;
  }
}

// Inference results back into the fits: P rows as predicted, Q columns
// shifted to sum to one over J_i.
__global__ void mlp_scatter_kernel(int n, int ny, const int8_t* __restrict__ cf, const int32_t* __restrict__ fidx,
                                   const int32_t* __restrict__ jrp, const int32_t* __restrict__ jci,
                                   const float* __restrict__ Y, double* __restrict__ fitP, double* __restrict__ fitQ) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || cf[i]) return;
  const float* y = Y + (size_t)fidx[i] * kO;
  int gi = i / ny, gj = i % ny;
  int c = jrp[i + 1] - jrp[i];
  double sq = 0.0;
  for (int e = jrp[i]; e < jrp[i + 1]; ++e) {
    int j = jci[e];
    int di = j / ny - gi, dj = j % ny - gj;
    bool in_box = di >= -1 && di <= 1 && dj >= -1 && dj <= 1 && !(di == 0 && dj == 0);
    int s = in_box ? box_slot(di, dj) : 0;
    fitP[e] = in_box ? (double)y[s] : 0.0;
    fitQ[e] = in_box ? (double)y[8 + s] : 0.0;
    sq += fitQ[e];
  }
  double shift = c > 0 ? (1.0 - sq) / c : 0.0;
  for (int e = jrp[i]; e < jrp[i + 1]; ++e) fitQ[e] += shift;
}

__global__ void fine_index_kernel(int n, const int8_t* __restrict__ cf, const int32_t* __restrict__ pre,
                                  int32_t* __restrict__ fidx) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) fidx[i] = cf[i] ? -1 : i - pre[i];
}

__global__ void cf_count_kernel(int n, const int8_t* __restrict__ cf, int32_t* __restrict__ c) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] = cf[i] ? 1 : 0;
}

// ============================================================ host side
static std::atomic<uint64_t> g_grad_attr{0};
static size_t grad_smem() {
  return sizeof(MlpSmem) + kMlpWarps * (sizeof(GradSmem) + sizeof(WarpTile) + sizeof(BackTile));
}

// Inference on the tcgen05 tensor cores (mlp_tc.cu); synchronises the
// stream to read the kernel's timeout flag.
bamg_status mlp_forward(int M, const float* P, const void* X, float* Y, cudaStream_t s) {
  if (M <= 0) return BAMG_OK;
  DevMem err;
  BAMG_TRY(err.alloc(sizeof(int), s));
  BAMG_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  BAMG_TRY(mlp_forward_tc(M, P, X, Y, err.as<int>(), s));
  int h = 0;
  BAMG_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  if (h) {
    set_error("network inference kernel gave up waiting for its copies or tensor-core operations");
    return BAMG_ERR_TIMEOUT;
  }
  return BAMG_OK;
}

bamg_status mlp_grad(int M, float inv_count, const float* P, const void* X, const float* T, const float* mask,
                     float* G, float* loss, cudaStream_t s) {
  if (M <= 0) return BAMG_OK;
  size_t sm = grad_smem();
  int max_dyn = 0;
  BAMG_TRY(allow_max_smem((const void*)mlp_grad_kernel, g_grad_attr, &max_dyn));
  int tiles = (M + 15) / 16;
  int grid = (int)cdiv(tiles, kMlpWarps * 4);   // each warp takes a few tiles: fewer partial gradients
  if (grid > num_sms()) grid = num_sms();
  DevMem part;
  BAMG_TRY(part.alloc(sizeof(float) * (size_t)grid * kNParam, s));
  BAMG_TRY(launch(mlp_grad_kernel, dim3(grid), dim3(kMlpThreads), sm, s, M, inv_count, P,
                  (const __nv_bfloat16*)X, T, mask, part.as<float>(), loss));
  return launch(grad_reduce_kernel, dim3(cdiv(kNParam, 256)), dim3(256), 0, s, grid, (const float*)part.as<float>(),
                G);
}

// Features of the fine points of a geometric level, in ascending fine index.
bamg_status mlp_level_features(const Level& L, void* X, int32_t* fidx, int* nf_host, cudaStream_t s) {
  DevMem cnt, pre;
  BAMG_TRY(cnt.alloc(sizeof(int32_t) * (L.n + 1), s));
  BAMG_TRY(pre.alloc(sizeof(int32_t) * (L.n + 1), s));
  BAMG_TRY(launch(cf_count_kernel, dim3(cdiv(L.n, 256)), dim3(256), 0, s, L.n, L.cf.as<int8_t>(), cnt.as<int32_t>()));
  int64_t nc = 0;
  BAMG_TRY(scan_counts(cnt.as<int32_t>(), pre.as<int32_t>(), L.n, s, &nc));
  BAMG_TRY(launch(fine_index_kernel, dim3(cdiv(L.n, 256)), dim3(256), 0, s, L.n, L.cf.as<int8_t>(),
                  (const int32_t*)pre.as<int32_t>(), fidx));
  *nf_host = L.n - (int)nc;
  if (X)
    BAMG_TRY(launch(mlp_features_kernel, dim3(cdiv(L.n, 128)), dim3(128), 0, s, L.n, L.nx, L.ny, L.B.r(), L.B.c(),
                    L.B.v(), L.Bt.r(), L.Bt.c(), L.Bt.v(), L.cf.as<int8_t>(), (const int32_t*)fidx,
                    (__nv_bfloat16*)X));
  return BAMG_OK;
}

// Setup hook: P and Q weights of level L from the network (geometric levels).
bamg_status mlp_fits(const Level& L, const float* P, double* fitP, double* fitQ, cudaStream_t s) {
  DevMem fidx, X, Y;
  BAMG_TRY(fidx.alloc(sizeof(int32_t) * L.n, s));
  int nf = 0;
  BAMG_TRY(mlp_level_features(L, nullptr, fidx.as<int32_t>(), &nf, s));
  BAMG_TRY(X.alloc(sizeof(__nv_bfloat16) * (size_t)(nf > 0 ? nf : 1) * kF, s));
  BAMG_TRY(Y.alloc(sizeof(float) * (size_t)(nf > 0 ? nf : 1) * kO, s));
  BAMG_TRY(launch(mlp_features_kernel, dim3(cdiv(L.n, 128)), dim3(128), 0, s, L.n, L.nx, L.ny, L.B.r(), L.B.c(),
                  L.B.v(), L.Bt.r(), L.Bt.c(), L.Bt.v(), L.cf.as<int8_t>(), (const int32_t*)fidx.as<int32_t>(),
                  X.as<__nv_bfloat16>()));
  BAMG_TRY(mlp_forward(nf, P, X.p, Y.as<float>(), s));
  return launch(mlp_scatter_kernel, dim3(cdiv(L.n, 256)), dim3(256), 0, s, L.n, L.ny, L.cf.as<int8_t>(),
                (const int32_t*)fidx.as<int32_t>(), L.Jrp.as<int32_t>(), L.Jci.as<int32_t>(),
                (const float*)Y.as<float>(), fitP, fitQ);
}

int mlp_num_params() { return kNParam; }

}  // namespace bamg

using namespace bamg;

extern "C" int bamg_mlp_num_params(void) { return kNParam; }

extern "C" bamg_status bamg_mlp_init(float* params, uint64_t seed, void* stream) {
  BAMG_CHECK_ARG(params);
  return launch(mlp_init_kernel, dim3(cdiv(kNParam, 256)), dim3(256), 0, reinterpret_cast<cudaStream_t>(stream),
                params, seed);
}

// Parameter files: tag, entry count, FNV-1a hash (Fowler, Noll and Vo; 32-bit
// offset basis 2166136261, prime 16777619) of the entry bytes, entries; all
// fields little-endian, written byte by byte so the host's order is irrelevant.
namespace {
const unsigned char kMlpTag[8] = {'B', 'A', 'M', 'G', 'M', 'L', 'P', '1'};
constexpr size_t kMlpHead = 16;

void put_u32(unsigned char* b, uint32_t v) {
  for (int k = 0; k < 4; ++k) b[k] = (unsigned char)(v >> (8 * k));
}
uint32_t get_u32(const unsigned char* b) {
  uint32_t v = 0;
  for (int k = 0; k < 4; ++k) v |= (uint32_t)b[k] << (8 * k);
  return v;
}
uint32_t fnv1a32(const unsigned char* b, size_t n) {
  uint32_t h = 2166136261u;
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 16777619u;
  }
  return h;
}
bool all_finite(const std::vector<float>& w) {
  for (float v : w)
    if (!std::isfinite(v)) return false;
  return true;
}
}  // namespace

extern "C" bamg_status bamg_mlp_save(const char* path, const float* params, int on_device, void* stream) {
  BAMG_CHECK_ARG(path && params);
  std::vector<float> w(kNParam);
  if (on_device) {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    BAMG_CUDA(cudaMemcpyAsync(w.data(), params, sizeof(float) * kNParam, cudaMemcpyDeviceToHost, s));
    BAMG_CUDA(cudaStreamSynchronize(s));
  } else {
    std::memcpy(w.data(), params, sizeof(float) * kNParam);
  }
  if (!all_finite(w)) {
    set_error("network parameters to save hold a non-finite entry");
    return BAMG_ERR_NUMERIC;
  }
  std::vector<unsigned char> buf(kMlpHead + 4 * (size_t)kNParam);
  for (int i = 0; i < kNParam; ++i) {
    uint32_t u;
    std::memcpy(&u, &w[i], 4);
    put_u32(&buf[kMlpHead + 4 * (size_t)i], u);
  }
  std::memcpy(buf.data(), kMlpTag, 8);
  put_u32(&buf[8], (uint32_t)kNParam);
  put_u32(&buf[12], fnv1a32(&buf[kMlpHead], 4 * (size_t)kNParam));
  FILE* f = std::fopen(path, "wb");
  if (!f) {
    set_error("cannot open %s for writing", path);
    return BAMG_ERR_IO;
  }
  bool ok = std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) {
    set_error("writing %s failed", path);
    return BAMG_ERR_IO;
  }
  return BAMG_OK;
}

extern "C" bamg_status bamg_mlp_load(const char* path, float* params, int on_device, void* stream) {
  BAMG_CHECK_ARG(path && params);
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    set_error("cannot open %s for reading", path);
    return BAMG_ERR_IO;
  }
  const size_t len = kMlpHead + 4 * (size_t)kNParam;
  std::vector<unsigned char> buf(len + 1);
  const size_t got = std::fread(buf.data(), 1, len + 1, f);   // one byte more detects trailing data
  const bool rd_err = std::ferror(f) != 0;
  std::fclose(f);
  if (rd_err) {
    set_error("reading %s failed", path);
    return BAMG_ERR_IO;
  }
  if (got < kMlpHead || std::memcmp(buf.data(), kMlpTag, 8) != 0) {
    set_error("%s is not a network parameter file", path);
    return BAMG_ERR_IO;
  }
  const uint32_t count = get_u32(&buf[8]);
  if (count != (uint32_t)kNParam) {
    set_error("%s holds %u parameters, the network has %d", path, count, kNParam);
    return BAMG_ERR_IO;
  }
  if (got != len) {
    set_error("%s is %s", path, got < len ? "truncated" : "longer than its entries");
    return BAMG_ERR_IO;
  }
  if (get_u32(&buf[12]) != fnv1a32(&buf[kMlpHead], 4 * (size_t)kNParam)) {
    set_error("%s: hash of the entries does not match", path);
    return BAMG_ERR_IO;
  }
  std::vector<float> w(kNParam);
  for (int i = 0; i < kNParam; ++i) {
    const uint32_t u = get_u32(&buf[kMlpHead + 4 * (size_t)i]);
    std::memcpy(&w[i], &u, 4);
  }
  if (!all_finite(w)) {
    set_error("%s holds a non-finite parameter", path);
    return BAMG_ERR_NUMERIC;
  }
  if (on_device) {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    BAMG_CUDA(cudaMemcpyAsync(params, w.data(), sizeof(float) * kNParam, cudaMemcpyHostToDevice, s));
    BAMG_CUDA(cudaStreamSynchronize(s));
  } else {
    std::memcpy(params, w.data(), sizeof(float) * kNParam);
  }
  return BAMG_OK;
}

extern "C" bamg_status bamg_mlp_forward(const float* params, int M, const void* X_bf16, float* Y, void* stream) {
  BAMG_CHECK_ARG(params && M >= 0 && (M == 0 || (X_bf16 && Y)));
  return mlp_forward(M, params, X_bf16, Y, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" bamg_status bamg_mlp_grad(const float* params, int M, const void* X_bf16, const float* T,
                                     const float* mask, float* grad, float* loss_dev, void* stream) {
  BAMG_CHECK_ARG(params && X_bf16 && T && mask && grad && loss_dev && M >= 1);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  DevMem cnt;
  // count of used outputs (mean over the mask)
  std::vector<float> hm;
  BAMG_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * kNParam, s));
  BAMG_CUDA(cudaMemsetAsync(loss_dev, 0, sizeof(float), s));
  hm.resize((size_t)M * kO);
  BAMG_CUDA(cudaMemcpyAsync(hm.data(), mask, sizeof(float) * hm.size(), cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  double c = 0;
  for (float v : hm) c += v;
  float inv = c > 0 ? (float)(1.0 / c) : 0.f;
  return mlp_grad(M, inv, params, X_bf16, T, mask, grad, loss_dev, s);
}

extern "C" bamg_status bamg_mlp_train(float* params, int M, const void* X_bf16, const float* T, const float* mask,
                                      int epochs, int batch, float lr, float* loss_host, void* stream) {
  BAMG_CHECK_ARG(params && X_bf16 && T && mask && M >= 1 && epochs >= 1 && batch >= 16);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  DevMem G, m1, m2, loss;
  BAMG_TRY(G.alloc(sizeof(float) * kNParam, s));
  BAMG_TRY(m1.alloc(sizeof(float) * kNParam, s));
  BAMG_TRY(m2.alloc(sizeof(float) * kNParam, s));
  BAMG_TRY(loss.alloc(sizeof(float), s));
  BAMG_CUDA(cudaMemsetAsync(m1.p, 0, sizeof(float) * kNParam, s));
  BAMG_CUDA(cudaMemsetAsync(m2.p, 0, sizeof(float) * kNParam, s));
  // per-batch normaliser: number of used outputs in the batch
  std::vector<float> hm((size_t)M * kO);
  BAMG_CUDA(cudaMemcpyAsync(hm.data(), mask, sizeof(float) * hm.size(), cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  const int nb = (M + batch - 1) / batch;
  std::vector<float> inv(nb);
  for (int b = 0; b < nb; ++b) {
    double c = 0;
    for (size_t k = (size_t)b * batch * kO; k < std::min((size_t)M, (size_t)(b + 1) * batch) * kO; ++k) c += hm[k];
    inv[b] = c > 0 ? (float)(1.0 / c) : 0.f;
  }
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  long long step = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    BAMG_CUDA(cudaMemsetAsync(loss.p, 0, sizeof(float), s));
    for (int b = 0; b < nb; ++b) {
      int r0 = b * batch, mb = std::min(batch, M - r0);
      BAMG_CUDA(cudaMemsetAsync(G.p, 0, sizeof(float) * kNParam, s));
      BAMG_TRY(mlp_grad(mb, inv[b], params, (const __nv_bfloat16*)X_bf16 + (size_t)r0 * kF, T + (size_t)r0 * kO,
                        mask + (size_t)r0 * kO, G.as<float>(), loss.as<float>(), s));
      ++step;
      float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
      BAMG_TRY(launch(adam_kernel, dim3(cdiv(kNParam, 256)), dim3(256), 0, s, kNParam, params, m1.as<float>(),
                      m2.as<float>(), (const float*)G.as<float>(), lr, b1, b2, eps, c1, c2));
    }
    if (loss_host) {
      float l = 0;
      BAMG_CUDA(cudaMemcpyAsync(&l, loss.p, sizeof(float), cudaMemcpyDeviceToHost, s));
      BAMG_CUDA(cudaStreamSynchronize(s));
      loss_host[ep] = l / nb;
    }
  }
  return BAMG_OK;
}

// Harvest (features, LS targets, mask) from a level of a hierarchy built
// with least-squares fits; rows in ascending fine index.
extern "C" bamg_status bamg_mlp_harvest(const bamg_hierarchy* h, int level, void* X_bf16, float* T, float* mask,
                                        int capacity, int* count, void* stream) {
  BAMG_CHECK_ARG(h && count && level >= 0 && level + 1 < (int)h->lv.size());
  const Level& L = h->lv[level];
  if (h->p.coarsening != BAMG_COARSEN_GEOMETRIC || L.nx <= 0 || L.ny <= 0) {
    set_error("feature extraction needs a geometric level (grid shape)");
    return BAMG_ERR_UNSUPPORTED;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  DevMem fidx;
  BAMG_TRY(fidx.alloc(sizeof(int32_t) * L.n, s));
  int nf = 0;
  BAMG_TRY(mlp_level_features(L, nullptr, fidx.as<int32_t>(), &nf, s));
  *count = nf;
  if (!X_bf16) return BAMG_OK;   // size query
  BAMG_CHECK_ARG(T && mask && capacity >= nf);
  BAMG_TRY(launch(mlp_features_kernel, dim3(cdiv(L.n, 128)), dim3(128), 0, s, L.n, L.nx, L.ny, L.B.r(), L.B.c(),
                  L.B.v(), L.Bt.r(), L.Bt.c(), L.Bt.v(), L.cf.as<int8_t>(), (const int32_t*)fidx.as<int32_t>(),
                  (__nv_bfloat16*)X_bf16));
  return launch(mlp_targets_kernel, dim3(cdiv(L.n, 256)), dim3(256), 0, s, L.n, L.ny, L.cf.as<int8_t>(),
                (const int32_t*)fidx.as<int32_t>(), L.Jrp.as<int32_t>(), L.Jci.as<int32_t>(), L.P.r(), L.P.v(),
                L.Qt.v(), T, mask);
}
