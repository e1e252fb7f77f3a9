// Kernels over blocks of test vectors (n x LD, row-major) and vectors.
//
// Layout: a row of a block is LD contiguous values (LD*sizeof(T) bytes); a
// group of LPR = LD / VW lanes owns one matrix row and each lane one 16-byte
// vector of VW values, so the gather of a neighbour's row is one coalesced
// LD*sizeof(T)-byte transaction.  CSR column/value of a nonzero is read once
// per row group (broadcast to its lanes).
#include "internal.cuh"

namespace bamg {

template <typename T, int LD>
struct Blk {
  static constexpr int VW = Vec16<T>::W;
  static constexpr int LPR = LD / VW;
  static constexpr int RPW = 32 / LPR;
  static_assert(LD % VW == 0 && LPR >= 1 && LPR <= 32, "bad block width");
};

// Layout of the row kernels (relaxation, block SpMM): on large levels
// (W = 2) rows of 64 bytes or more are split into NV = 2 interleaved 16-byte
// vectors per lane (lane q of the row group holds vectors q and q + LPR), so
// a row group has half the lanes, a warp twice the rows, and each gather
// instruction of the group covers contiguous 32-byte sectors; small levels
// (W = 1) keep one vector per lane and twice the warps.
constexpr int kRowPairMin = 1 << 17;               // rows from which W = 2
template <typename T, int LD, int W = 2>
struct RowBlk {
  static constexpr int VW = Vec16<T>::W;
  static constexpr int NVR = LD / VW;              // 16-byte vectors per row
  static constexpr int NV = (NVR >= 4 && W == 2) ? 2 : 1;   // vectors per lane
  static constexpr int LPR = NVR / NV;             // lanes per row
  static constexpr int RPW = 32 / LPR;             // rows per warp
  static_assert(LD % VW == 0 && LPR >= 1 && LPR <= 32, "bad block width");
  __device__ static int col(int q, int v) { return (q + v * LPR) * VW; }
};

// acc = (A X)_row for the lane's NV vectors; the nonzeros are taken four at
// a time (indices and values first, then the row gathers) so that more loads
// are in flight per row group.
template <typename T, int LD, int W>
__device__ inline void row_times_block(int i, int q, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                       const T* __restrict__ va, const T* __restrict__ X,
                                       T (&acc)[RowBlk<T, LD, W>::NV][RowBlk<T, LD, W>::VW]) {
  using C = RowBlk<T, LD, W>;
#pragma unroll
  for (int v = 0; v < C::NV; ++v)
#pragma unroll
    for (int w = 0; w < C::VW; ++w) acc[v][w] = T(0);
  const int p0 = __ldg(rp + i), p1 = __ldg(rp + i + 1);
  int p = p0;
  for (; p + 4 <= p1; p += 4) {
    int j[4];
    T a[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      j[u] = __ldg(ci + p + u);
      a[u] = __ldg(va + p + u);
    }
    T xv[4][C::NV][C::VW];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < C::NV; ++v) vload_ro(X + (size_t)j[u] * LD + C::col(q, v), xv[u][v]);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < C::NV; ++v)
#pragma unroll
        for (int w = 0; w < C::VW; ++w) acc[v][w] = fma(a[u], xv[u][v][w], acc[v][w]);
  }
  for (; p < p1; ++p) {
    const int j = __ldg(ci + p);
    const T a = __ldg(va + p);
    T xv[C::NV][C::VW];
#pragma unroll
    for (int v = 0; v < C::NV; ++v) vload_ro(X + (size_t)j * LD + C::col(q, v), xv[v]);
#pragma unroll
    for (int v = 0; v < C::NV; ++v)
#pragma unroll
      for (int w = 0; w < C::VW; ++w) acc[v][w] = fma(a, xv[v][w], acc[v][w]);
  }
}

// Y = X + omega D^{-1} (sigma .* R - B X)   (Algorithm 1 smoothing loops;
// weighted Jacobi, Section 3).  keep0: column 0 copied unchanged.  Two
// independent jobs (the V and U relaxations) share one launch: blockIdx.y
// selects the job.
template <typename T, int LD, int W>
__global__ void __launch_bounds__(256, 6) relax_block_kernel(RelaxJob<T> j0, RelaxJob<T> j1) {
  pdl_wait();
  pdl_trigger();
  using C = RowBlk<T, LD, W>;
  const RelaxJob<T>& a = blockIdx.y ? j1 : j0;
  int lane = threadIdx.x & 31;
  int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int i = gw * C::RPW + lane / C::LPR;
  int q = lane % C::LPR;
  if (i >= a.n) return;
  T acc[C::NV][C::VW];
  row_times_block<T, LD, W>(i, q, a.rp, a.ci, a.va, a.X, acc);
  const T di = __ldg(a.dinv + i);
#pragma unroll
  for (int v = 0; v < C::NV; ++v) {
    const size_t o = (size_t)i * LD + C::col(q, v);
    T xi[C::VW], y[C::VW];
    vload_ro(a.X + o, xi);
    if (a.R) {
      T rv[C::VW];
      vload_ro(a.R + o, rv);
#pragma unroll
      for (int w = 0; w < C::VW; ++w) {
        T s = a.sig ? __ldg(a.sig + C::col(q, v) + w) : T(1);
        y[w] = xi[w] + (a.omega * (s * rv[w] - acc[v][w])) * di;
      }
    } else {
#pragma unroll
      for (int w = 0; w < C::VW; ++w) y[w] = xi[w] + (a.omega * (-acc[v][w])) * di;
    }
    if (a.keep0 && q == 0 && v == 0) y[0] = xi[0];
    vstore(a.Y + o, y);
  }
}

// Y = A X  (rows x LD) for a CSR A; up to three independent products per
// launch (blockIdx.y selects one).
template <typename T, int LD, int W>
__global__ void __launch_bounds__(256, 6) spmm_block_kernel(SpmmJob<T> j0, SpmmJob<T> j1, SpmmJob<T> j2) {
  pdl_wait();
  pdl_trigger();
  using C = RowBlk<T, LD, W>;
  const SpmmJob<T>& a = blockIdx.y == 0 ? j0 : (blockIdx.y == 1 ? j1 : j2);
  int lane = threadIdx.x & 31;
  int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int i = gw * C::RPW + lane / C::LPR;
  int q = lane % C::LPR;
  if (i >= a.rows) return;
  T acc[C::NV][C::VW];
  row_times_block<T, LD, W>(i, q, a.rp, a.ci, a.va, a.X, acc);
#pragma unroll
  for (int v = 0; v < C::NV; ++v) vstore(a.Y + (size_t)i * LD + C::col(q, v), acc[v]);
}

// Per-block column sums of K products, written to part[block][K*LD].
// mode 0 (norms): pair 0 = x.x, pair 1 = (Bx).(Bx) with Bx formed on the fly.
// mode 1 (dots):  pair k = A_k . B_k for the supplied block pairs.
template <typename T, int LD, int MODE>
__global__ void __launch_bounds__(256)
coldot_kernel(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
              const T* __restrict__ va, const T* __restrict__ X, const T* __restrict__ A0,
              const T* __restrict__ B0, const T* __restrict__ A1, const T* __restrict__ B1,
              const T* __restrict__ A2, const T* __restrict__ B2, int npairs,
              double* __restrict__ part) {
  pdl_wait();
  pdl_trigger();
  using C = Blk<T, LD>;
  // per-thread sums in the block precision (a thread covers a few rows; the
  // FP64 pipes of GB300 are narrow), block and grid sums in FP64
  using Acc = T;
  constexpr int K = 3;
  __shared__ double sh[8][K * LD];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int q = lane % C::LPR;
  Acc acc[K][C::VW];
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int v = 0; v < C::VW; ++v) acc[k][v] = Acc(0);
  int rows_per_block = (blockDim.x >> 5) * C::RPW;
  for (int i = blockIdx.x * rows_per_block + w * C::RPW + lane / C::LPR; i < n;
       i += gridDim.x * rows_per_block) {
    size_t o = (size_t)i * LD + q * C::VW;
    if (MODE == 0) {
      T bx[C::VW], xi[C::VW];
#pragma unroll
      for (int v = 0; v < C::VW; ++v) bx[v] = T(0);
      for (int p = __ldg(rp + i); p < __ldg(rp + i + 1); ++p) {
        int j = __ldg(ci + p);
        T a = __ldg(va + p);
        T xv[C::VW];
        vload_ro(X + (size_t)j * LD + q * C::VW, xv);
#pragma unroll
        for (int v = 0; v < C::VW; ++v) bx[v] = fma(a, xv[v], bx[v]);
      }
      vload_ro(X + o, xi);
#pragma unroll
      for (int v = 0; v < C::VW; ++v) {
        acc[0][v] = fma(xi[v], xi[v], acc[0][v]);
        acc[1][v] = fma(bx[v], bx[v], acc[1][v]);
      }
    } else {
      const T* As[3] = {A0, A1, A2};
      const T* Bs[3] = {B0, B1, B2};
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (k < npairs) {
          T a[C::VW], b[C::VW];
          vload_ro(As[k] + o, a);
          vload_ro(Bs[k] + o, b);
#pragma unroll
          for (int v = 0; v < C::VW; ++v) acc[k][v] = fma(a[v], b[v], acc[k][v]);
        }
      }
    }
  }
  // lanes with equal q hold the same columns: reduce over the row groups
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int v = 0; v < C::VW; ++v)
      for (int o = 16; o >= C::LPR; o >>= 1) acc[k][v] += __shfl_xor_sync(0xffffffffu, acc[k][v], o);
  if (lane < C::LPR) {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int v = 0; v < C::VW; ++v) sh[w][k * LD + lane * C::VW + v] = (double)acc[k][v];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < K * LD; t += blockDim.x) {
    double s = 0.0;
    for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) s += sh[ww][t];
    part[(size_t)blockIdx.x * K * LD + t] = s;
  }
}

// From sums [x.x | Bx.Bx]: scale_k = 1/||x_k||, w_k = ||x_k|| / ||B x_k||
// (eq. ls_weights for the normalised vector).
template <typename T, int LD>
__global__ void weights_finalize_kernel(const double* __restrict__ sums, int r, int skip0,
                                        T* __restrict__ scale, double* __restrict__ w,
                                        double* __restrict__ norms) {
  pdl_wait();
  pdl_trigger();
  int k = threadIdx.x;
  if (k >= LD) return;
  double xx = sums[k], bb = sums[LD + k];
  bool active = k < r && !(skip0 && k == 0);
  double nx = sqrt(xx);
  norms[k] = nx;
  if (active && xx > 0.0 && bb > 0.0) {
    scale[k] = T(1.0 / nx);
    w[k] = nx / sqrt(bb);
  } else {
    scale[k] = T(1);
    w[k] = 0.0;
  }
}

template <typename T, int LD>
__global__ void scale_cols_kernel(int n, T* __restrict__ X, const T* __restrict__ scale) {
  pdl_wait();
  pdl_trigger();
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * LD) return;
  X[t] *= scale[t % LD];
}

// eq. singular_value: sigma_k = u.Bv / (sqrt(u.Mu) sqrt(v.Nv)).
template <typename T>
__global__ void rayleigh_finalize_kernel(const double* __restrict__ sums, int LD, int r,
                                         T* __restrict__ sig, double* __restrict__ sig64) {
  pdl_wait();
  pdl_trigger();
  int k = threadIdx.x;
  if (k >= LD) return;
  double num = sums[k], um = sums[LD + k], vn = sums[2 * LD + k];
  double s = (k < r && um > 0.0 && vn > 0.0) ? num / (sqrt(um) * sqrt(vn)) : 0.0;
  sig[k] = T(s);
  if (sig64) sig64[k] = s;
}

// Test vectors (Section 4.2 random start, Section 5 u^(1) = 1): SplitMix64
// uniform(-1,1), V column k from stream 2k, U column k from stream 2k+1.
template <typename T, int LD>
__global__ void init_vectors_kernel(int n, int r, uint64_t seed, T* __restrict__ U, T* __restrict__ V) {
  pdl_wait();
  pdl_trigger();
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * LD) return;
  int i = (int)(t / LD), k = (int)(t % LD);
  if (k >= r) {
    U[t] = T(0); V[t] = T(0);
    return;
  }
  V[t] = T(splitmix_pm1(seed, 2ull * k, (uint64_t)i));
  U[t] = k == 0 ? T(1) : T(splitmix_pm1(seed, 2ull * k + 1, (uint64_t)i));
}

// Canonical injection R (Algorithm 1): Xc[I, :] = X[cpt[I], :].
template <typename T, int LD>
__global__ void inject_kernel(int nc, const int32_t* __restrict__ cpt, const T* __restrict__ X,
                              T* __restrict__ Xc) {
  pdl_wait();
  pdl_trigger();
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)nc * LD) return;
  int I = (int)(t / LD), k = (int)(t % LD);
  Xc[t] = X[(size_t)cpt[I] * LD + k];
}

// ------------------------------------------------------- vector kernels
// One group of G lanes per row, RU consecutive rows per group; modes of the
// V-cycle and GMRES.  The loads of the RU rows are issued together (column
// indices and values, then the gathers of x) so that RU times more memory
// requests are in flight per lane than with one row per group; each row
// still sums its products lane by lane in the order p0 + g, p0 + g + G, ...
// and then across the group, so the result does not depend on RU.
// kJacobiZero2: the first two sweeps from zero in one pass.  The first
// sweep's value at a neighbour, (omega b_j) dinv_j, is recomputed from b and
// dinv with the same two rounded products, so the result is bit for bit that
// of kJacobiZero followed by kJacobi.
enum VecMode { kJacobi = 0, kJacobiZero = 1, kResid = 2, kSpmv = 3, kSpmvAdd = 4, kJacobiZero2 = 5 };

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <typename T, int G, int MODE, int RU>
__global__ void __launch_bounds__(256)
csr_vec_kernel(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
               const T* __restrict__ va, const T* __restrict__ dinv, T omega, const T* __restrict__ x,
               const T* __restrict__ b, T* __restrict__ y) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const size_t grp = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int g = lane % G;
  const long long i0 = (long long)grp * RU;   // every lane joins the shuffles below
  T acc[RU];
#pragma unroll
  for (int u = 0; u < RU; ++u) acc[u] = T(0);
  if (MODE != kJacobiZero) {
    int p0[RU], p1[RU];
    int len = 0;
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const bool v = i0 + u < n;
      p0[u] = v ? __ldg(rp + i0 + u) : 0;
      p1[u] = v ? __ldg(rp + i0 + u + 1) : 0;
      len = max(len, p1[u] - p0[u]);
    }
    for (int off = g; off < len; off += G) {
      int c[RU];
      T a[RU];
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        const int p = p0[u] + off;
        const bool in = p < p1[u];
        c[u] = in ? __ldg(ci + p) : -1;
        a[u] = in ? __ldg(va + p) : T(0);
      }
      T xv[RU];
      if (MODE == kJacobiZero2) {
#pragma unroll
        for (int u = 0; u < RU; ++u)
          xv[u] = c[u] >= 0 ? mul_rn(mul_rn(omega, __ldg(b + c[u])), __ldg(dinv + c[u])) : T(0);
      } else {
#pragma unroll
        for (int u = 0; u < RU; ++u) xv[u] = c[u] >= 0 ? __ldg(x + c[u]) : T(0);
      }
#pragma unroll
      for (int u = 0; u < RU; ++u)
        if (c[u] >= 0) acc[u] = fma(a[u], xv[u], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < RU; ++u) acc[u] = group_sum<G>(acc[u]);
  }
  if (g != 0) return;
#pragma unroll
  for (int u = 0; u < RU; ++u) {
    const long long i = i0 + u;
    if (i >= n) break;
    if (MODE == kJacobi) y[i] = x[i] + (omega * (b[i] - acc[u])) * dinv[i];
    else if (MODE == kJacobiZero2) y[i] = mul_rn(mul_rn(omega, b[i]), dinv[i]) + (omega * (b[i] - acc[u])) * dinv[i];
    else if (MODE == kJacobiZero) y[i] = (omega * b[i]) * dinv[i];
    else if (MODE == kResid) y[i] = b[i] - acc[u];
    else if (MODE == kSpmv) y[i] = acc[u];
    else y[i] = y[i] + acc[u];
  }
}

template <typename T>
__global__ void dense_gemv_kernel(int n, const T* __restrict__ A, const T* __restrict__ x, T* __restrict__ y) {
  pdl_wait();
  pdl_trigger();
  int lane = threadIdx.x & 31;
  int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (i >= n) return;
  T acc = T(0);
  for (int j = lane; j < n; j += 32) acc = fma(A[(size_t)i * n + j], x[j], acc);
  acc = warp_sum(acc);
  if (lane == 0) y[i] = acc;
}

template <typename S, typename D>
__global__ void convert_kernel(size_t n, const S* __restrict__ a, D* __restrict__ b) {
  pdl_wait();
  pdl_trigger();
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = D(a[t]);
}

// up to kConvMany double arrays to float in one launch (blockIdx.y = array)
__global__ void convert_many_kernel(ConvMany job) {
  pdl_wait();
  pdl_trigger();
  const int q = blockIdx.y;
  const size_t n = job.n[q];
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    job.dst[q][t] = float(job.src[q][t]);
}

// Jacobi divisor of row i (Section 3: x <- x + omega D^{-1} (b - B x)).
// d_i = b_ii when b_ii > 0.  A coarse Petrov-Galerkin operator Q B P may have
// b_ii <= 0, where that step is undefined; there d_i is the larger of the l1
// norms of row i and of column i of B (an l1-Jacobi row, usable for the
// relaxations with B and with B^T alike) and the row is counted in *nsafe.
// A row whose row and column are both zero is reported in *bad_row.
template <typename T>
__global__ void diag_inv_kernel(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const double* __restrict__ va, const int32_t* __restrict__ trp,
                                const double* __restrict__ tva, T* __restrict__ dinv,
                                int* __restrict__ bad_row, int* __restrict__ nsafe) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 0.0, l1r = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    if (ci[p] == i) d = va[p];
    l1r += fabs(va[p]);
  }
  if (d > 0.0) {
    dinv[i] = T(1.0 / d);
    return;
  }
  double l1c = 0.0;
  for (int p = trp[i]; p < trp[i + 1]; ++p) l1c += fabs(tva[p]);
  const double m = fmax(l1r, l1c);
  if (m > 0.0) {
    dinv[i] = T(1.0 / m);
    atomicAdd(nsafe, 1);
  } else {
    dinv[i] = T(0);
    atomicMin(bad_row, i);
  }
}

// =================================================================== host
template <typename T, int LD, int W>
static bamg_status relax_lw(int n, const RelaxJob<T>& j0, const RelaxJob<T>* j1, cudaStream_t s) {
  using C = RowBlk<T, LD, W>;
  unsigned blocks = cdiv(n, 8 * C::RPW);
  return launch(relax_block_kernel<T, LD, W>, dim3(blocks, j1 ? 2 : 1), dim3(256), 0, s, j0, j1 ? *j1 : j0);
}

template <typename T, int LD>
static bamg_status relax_ld(const RelaxJob<T>& j0, const RelaxJob<T>* j1, cudaStream_t s) {
  const int n = j1 && j1->n > j0.n ? j1->n : j0.n;
  return n >= kRowPairMin ? relax_lw<T, LD, 2>(n, j0, j1, s) : relax_lw<T, LD, 1>(n, j0, j1, s);
}

template <typename T, int LD, int W>
static bamg_status spmm_lw(int rows, const SpmmJob<T>* jobs, int k, cudaStream_t s) {
  using C = RowBlk<T, LD, W>;
  return launch(spmm_block_kernel<T, LD, W>, dim3(cdiv(rows, 8 * C::RPW), k), dim3(256), 0, s, jobs[0],
                jobs[k > 1 ? 1 : 0], jobs[k > 2 ? 2 : 0]);
}

template <typename T, int LD>
static bamg_status spmm_ld(const SpmmJob<T>* jobs, int k, cudaStream_t s) {
  int rows = 0;
  for (int q = 0; q < k; ++q) rows = jobs[q].rows > rows ? jobs[q].rows : rows;
  return rows >= kRowPairMin ? spmm_lw<T, LD, 2>(rows, jobs, k, s) : spmm_lw<T, LD, 1>(rows, jobs, k, s);
}

#define BAMG_LD_DISPATCH(ld, CALL)                 \
  switch (ld) {                                    \
    case 4: { constexpr int LDC = 4; CALL; }       \
    case 8: { constexpr int LDC = 8; CALL; }       \
    case 16: { constexpr int LDC = 16; CALL; }     \
    case 32: { constexpr int LDC = 32; CALL; }     \
    default: set_error("block width %d not in {4,8,16,32}", ld); return BAMG_ERR_ARG; \
  }

template <typename T>
bamg_status relax_block(int n, int ld, const int32_t* rp, const int32_t* ci, const T* va, const T* dinv,
                        const T* X, T* Y, const T* R, const T* sig, T omega, int keep0, cudaStream_t s) {
  RelaxJob<T> j{n, rp, ci, va, dinv, X, Y, R, sig, omega, keep0};
  BAMG_LD_DISPATCH(ld, return (relax_ld<T, LDC>(j, nullptr, s)));
}

// The V relaxation with B and the U relaxation with B^T in one launch.
template <typename T>
bamg_status relax_block2(int n, int ld, const int32_t* rp, const int32_t* ci, const T* va, const int32_t* trp,
                         const int32_t* tci, const T* tva, const T* dinv, const T* V, T* Vn, const T* U, T* Un,
                         const T* RV, const T* RU, const T* sig, T omega, int keepU0, cudaStream_t s) {
  RelaxJob<T> jv{n, rp, ci, va, dinv, V, Vn, RV, sig, omega, 0};
  RelaxJob<T> ju{n, trp, tci, tva, dinv, U, Un, RU, sig, omega, keepU0};
  BAMG_LD_DISPATCH(ld, return (relax_ld<T, LDC>(jv, &ju, s)));
}

template <typename T>
bamg_status spmm_block(int rows, int ld, const int32_t* rp, const int32_t* ci, const T* va, const T* X,
                       T* Y, cudaStream_t s) {
  SpmmJob<T> j{rows, rp, ci, va, X, Y};
  BAMG_LD_DISPATCH(ld, return (spmm_ld<T, LDC>(&j, 1, s)));
}

// Up to three independent products Y_q = A_q X_q in one launch.
template <typename T>
bamg_status spmm_block_multi(int ld, const SpmmJob<T>* jobs, int k, cudaStream_t s) {
  if (k < 1 || k > 3) {
    set_error("spmm_block_multi takes 1 to 3 products");
    return BAMG_ERR_ARG;
  }
  BAMG_LD_DISPATCH(ld, return (spmm_ld<T, LDC>(jobs, k, s)));
}

static int reduce_blocks(int n, int rows_per_block) {
  int nb = (int)cdiv(n, rows_per_block);
  int cap = 4 * num_sms();
  return nb < cap ? (nb > 0 ? nb : 1) : cap;
}

template <typename T, int LD>
static bamg_status norms_ld(int n, int r, const int32_t* rp, const int32_t* ci, const T* va, T* X,
                            int normalise, int skip0, T* scale, double* w, double* norms, cudaStream_t s) {
  using C = Blk<T, LD>;
  int nb = reduce_blocks(n, 8 * C::RPW);
  DevMem part, sums;
  BAMG_TRY(part.alloc(sizeof(double) * nb * 3 * LD, s));
  BAMG_TRY(sums.alloc(sizeof(double) * 3 * LD, s));
  BAMG_TRY(launch(coldot_kernel<T, LD, 0>, dim3(nb), dim3(256), 0, s, n, rp, ci, va, (const T*)X,
                  (const T*)nullptr, (const T*)nullptr, (const T*)nullptr, (const T*)nullptr,
                  (const T*)nullptr, (const T*)nullptr, 0, part.as<double>()));
  BAMG_TRY(reduce_partials(part.as<double>(), nb, 3 * LD, sums.as<double>(), s));
  BAMG_TRY(launch(weights_finalize_kernel<T, LD>, dim3(1), dim3(32), 0, s, (const double*)sums.as<double>(),
                  r, skip0, scale, w, norms));
  if (normalise)
    BAMG_TRY(launch(scale_cols_kernel<T, LD>, dim3(cdiv((long long)n * LD, 256)), dim3(256), 0, s, n, X,
                    (const T*)scale));
  return BAMG_OK;
}

template <typename T>
bamg_status norms_weights(int n, int ld, int r, const int32_t* rp, const int32_t* ci, const T* va, T* X,
                          int normalise, int skip0, T* scale, double* w, double* norms, cudaStream_t s) {
  BAMG_LD_DISPATCH(ld, return (norms_ld<T, LDC>(n, r, rp, ci, va, X, normalise, skip0, scale, w, norms, s)));
}

// Same launches as norms_ld, with every buffer supplied by the caller:
// part[max_blocks * 3 * LD], sums[3 * LD], scale[LD], w[LD], norms[LD].
template <typename T, int LD>
static bamg_status norms_ws_ld(int n, int r, const int32_t* rp, const int32_t* ci, const T* va, T* X,
                               int normalise, int skip0, double* part, int max_blocks, double* sums, T* scale,
                               double* w, double* norms, cudaStream_t s) {
  using C = Blk<T, LD>;
  int nb = reduce_blocks(n, 8 * C::RPW);
  if (nb > max_blocks) nb = max_blocks;
  BAMG_TRY(launch(coldot_kernel<T, LD, 0>, dim3(nb), dim3(256), 0, s, n, rp, ci, va, (const T*)X,
                  (const T*)nullptr, (const T*)nullptr, (const T*)nullptr, (const T*)nullptr,
                  (const T*)nullptr, (const T*)nullptr, 0, part));
  BAMG_TRY(reduce_partials(part, nb, 3 * LD, sums, s));
  BAMG_TRY(launch(weights_finalize_kernel<T, LD>, dim3(1), dim3(32), 0, s, (const double*)sums, r, skip0,
                  scale, w, norms));
  if (normalise)
    BAMG_TRY(launch(scale_cols_kernel<T, LD>, dim3(cdiv((long long)n * LD, 256)), dim3(256), 0, s, n, X,
                    (const T*)scale));
  return BAMG_OK;
}

template <typename T>
bamg_status norms_weights_ws(int n, int ld, int r, const int32_t* rp, const int32_t* ci, const T* va, T* X,
                             int normalise, int skip0, double* part, int max_blocks, double* sums, T* scale,
                             double* w, double* norms, cudaStream_t s) {
  BAMG_LD_DISPATCH(ld, return (norms_ws_ld<T, LDC>(n, r, rp, ci, va, X, normalise, skip0, part, max_blocks,
                                                   sums, scale, w, norms, s)));
}

template <typename T, int LD>
static bamg_status dots_ld(int n, int npairs, const T* A0, const T* B0, const T* A1, const T* B1,
                           const T* A2, const T* B2, double* sums, cudaStream_t s) {
  using C = Blk<T, LD>;
  int nb = reduce_blocks(n, 8 * C::RPW);
  DevMem part;
  BAMG_TRY(part.alloc(sizeof(double) * nb * 3 * LD, s));
  BAMG_TRY(launch(coldot_kernel<T, LD, 1>, dim3(nb), dim3(256), 0, s, n, (const int32_t*)nullptr,
                  (const int32_t*)nullptr, (const T*)nullptr, (const T*)nullptr, A0, B0, A1, B1, A2, B2,
                  npairs, part.as<double>()));
  return reduce_partials(part.as<double>(), nb, 3 * LD, sums, s);
}

template <typename T>
bamg_status col_dots(int n, int ld, int npairs, const T* A0, const T* B0, const T* A1, const T* B1,
                     const T* A2, const T* B2, double* sums, cudaStream_t s) {
  BAMG_LD_DISPATCH(ld, return (dots_ld<T, LDC>(n, npairs, A0, B0, A1, B1, A2, B2, sums, s)));
}

template <typename T>
bamg_status rayleigh_finalize(const double* sums, int ld, int r, T* sig, double* sig64, cudaStream_t s) {
  return launch(rayleigh_finalize_kernel<T>, dim3(1), dim3(32), 0, s, sums, ld, r, sig, sig64);
}

template <typename T>
bamg_status init_vectors(int n, int ld, int r, uint64_t seed, T* U, T* V, cudaStream_t s) {
  unsigned g = cdiv((long long)n * ld, 256);
  BAMG_LD_DISPATCH(ld, return launch(init_vectors_kernel<T, LDC>, dim3(g), dim3(256), 0, s, n, r, seed, U, V));
}

template <typename T>
bamg_status inject(int nc, int ld, const int32_t* cpt, const T* X, T* Xc, cudaStream_t s) {
  unsigned g = cdiv((long long)nc * ld, 256);
  BAMG_LD_DISPATCH(ld, return launch(inject_kernel<T, LDC>, dim3(g), dim3(256), 0, s, nc, cpt, X, Xc));
}

// rows per lane group: short rows take several per group
template <int G> constexpr int vec_rows() { return G <= 4 ? 4 : G == 8 ? 2 : 1; }

template <typename T, int G, int MODE>
static bamg_status vec_launch(int n, const int32_t* rp, const int32_t* ci, const T* va, const T* dinv, T omega,
                              const T* x, const T* b, T* y, cudaStream_t s) {
  constexpr int RU = vec_rows<G>();
  const unsigned g = cdiv((long long)cdiv(n, RU) * G, 256);
  return launch(csr_vec_kernel<T, G, MODE, RU>, dim3(g), dim3(256), 0, s, n, rp, ci, va, dinv, omega, x, b, y);
}

template <typename T, int MODE>
static bamg_status vec_g(int n, int G, const int32_t* rp, const int32_t* ci, const T* va, const T* dinv,
                         T omega, const T* x, const T* b, T* y, cudaStream_t s) {
  switch (G) {
    case 2: return vec_launch<T, 2, MODE>(n, rp, ci, va, dinv, omega, x, b, y, s);
    case 4: return vec_launch<T, 4, MODE>(n, rp, ci, va, dinv, omega, x, b, y, s);
    case 8: return vec_launch<T, 8, MODE>(n, rp, ci, va, dinv, omega, x, b, y, s);
    case 16: return vec_launch<T, 16, MODE>(n, rp, ci, va, dinv, omega, x, b, y, s);
    default: return vec_launch<T, 32, MODE>(n, rp, ci, va, dinv, omega, x, b, y, s);
  }
}

template <typename T>
bamg_status csr_vec(int mode, int n, int G, const int32_t* rp, const int32_t* ci, const T* va, const T* dinv,
                    T omega, const T* x, const T* b, T* y, cudaStream_t s) {
  switch (mode) {
    case kJacobi: return vec_g<T, kJacobi>(n, G, rp, ci, va, dinv, omega, x, b, y, s);
    case kJacobiZero: return vec_g<T, kJacobiZero>(n, G, rp, ci, va, dinv, omega, x, b, y, s);
    case kResid: return vec_g<T, kResid>(n, G, rp, ci, va, dinv, omega, x, b, y, s);
    case kSpmv: return vec_g<T, kSpmv>(n, G, rp, ci, va, dinv, omega, x, b, y, s);
    case kJacobiZero2: return vec_g<T, kJacobiZero2>(n, G, rp, ci, va, dinv, omega, x, b, y, s);
    default: return vec_g<T, kSpmvAdd>(n, G, rp, ci, va, dinv, omega, x, b, y, s);
  }
}

template <typename T>
bamg_status dense_gemv(int n, const T* A, const T* x, T* y, cudaStream_t s) {
  return launch(dense_gemv_kernel<T>, dim3(cdiv((long long)n * 32, 256)), dim3(256), 0, s, n, A, x, y);
}

template <typename S, typename D>
bamg_status convert(size_t n, const S* a, D* b, cudaStream_t s) {
  return launch(convert_kernel<S, D>, dim3(cdiv((long long)n, 256)), dim3(256), 0, s, n, a, b);
}

bamg_status convert_many(const ConvMany& job, cudaStream_t s) {
  if (job.k <= 0) return BAMG_OK;
  size_t mx = 0;
  for (int q = 0; q < job.k; ++q) mx = job.n[q] > mx ? job.n[q] : mx;
  unsigned g = cdiv((long long)(mx > 0 ? mx : 1), 256);
  if (g > 4096u) g = 4096u;
  return launch(convert_many_kernel, dim3(g, job.k), dim3(256), 0, s, job);
}

template <typename T>
bamg_status diag_inv(int n, const int32_t* rp, const int32_t* ci, const double* va, const int32_t* trp,
                     const double* tva, T* dinv, int* bad_row, int* nsafe, cudaStream_t s) {
  return launch(diag_inv_kernel<T>, dim3(cdiv(n, 256)), dim3(256), 0, s, n, rp, ci, va, trp, tva, dinv, bad_row,
                nsafe);
}

// Prolongation and the first post-smoothing sweep in one pass:
// y = z1 + omega dinv .* (b - B z1) with z1 = z0 + P e.  A row's group of G
// lanes forms the z1 entries its B entries need from P's rows (the
// prolongation is never stored), so the V-cycle takes one pass instead of
// two.
template <typename T, int G>
__global__ void __launch_bounds__(256)
prolong_jacobi_kernel(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                      const T* __restrict__ va, const T* __restrict__ dinv, T omega,
                      const int32_t* __restrict__ prp, const int32_t* __restrict__ pci, const T* __restrict__ pva,
                      const T* __restrict__ e, const T* __restrict__ z0, const T* __restrict__ b,
                      T* __restrict__ y) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;   // every lane joins the shuffles
  const int g = lane % G;
  auto z1 = [&](int k) {
    T v = T(0);
    for (int p = __ldg(prp + k); p < __ldg(prp + k + 1); ++p) v = fma(__ldg(pva + p), __ldg(e + __ldg(pci + p)), v);
    return z0[k] + v;
  };
  T acc = T(0);
  if (i < n) {
    const int p0 = __ldg(rp + i), p1 = __ldg(rp + i + 1);
    for (int p = p0 + g; p < p1; p += G) acc = fma(__ldg(va + p), z1(__ldg(ci + p)), acc);
  }
  acc = group_sum<G>(acc);
  if (g == 0 && i < n) y[i] = z1((int)i) + (omega * (b[i] - acc)) * dinv[i];
}

template <typename T>
bamg_status prolong_jacobi(int n, int G, const int32_t* rp, const int32_t* ci, const T* va, const T* dinv,
                           T omega, const int32_t* prp, const int32_t* pci, const T* pva, const T* e,
                           const T* z0, const T* b, T* y, cudaStream_t s) {
  auto go = [&](auto kern, int g) {
    return launch(kern, dim3(cdiv((long long)n * g, 256)), dim3(256), 0, s, n, rp, ci, va, dinv, omega, prp, pci,
                  pva, e, z0, b, y);
  };
  switch (G) {
    case 2: return go(prolong_jacobi_kernel<T, 2>, 2);
    case 4: return go(prolong_jacobi_kernel<T, 4>, 4);
    case 8: return go(prolong_jacobi_kernel<T, 8>, 8);
    case 16: return go(prolong_jacobi_kernel<T, 16>, 16);
    default: return go(prolong_jacobi_kernel<T, 32>, 32);
  }
}

#define BAMG_INST(T)                                                                                       \
  template bamg_status prolong_jacobi<T>(int, int, const int32_t*, const int32_t*, const T*, const T*, T,  \
                                         const int32_t*, const int32_t*, const T*, const T*, const T*,     \
                                         const T*, T*, cudaStream_t);                                      \
  template bamg_status relax_block<T>(int, int, const int32_t*, const int32_t*, const T*, const T*,       \
                                      const T*, T*, const T*, const T*, T, int, cudaStream_t);           \
  template bamg_status spmm_block<T>(int, int, const int32_t*, const int32_t*, const T*, const T*, T*,    \
                                     cudaStream_t);                                                     \
  template bamg_status norms_weights<T>(int, int, int, const int32_t*, const int32_t*, const T*, T*, int, \
                                        int, T*, double*, double*, cudaStream_t);                       \
  template bamg_status col_dots<T>(int, int, int, const T*, const T*, const T*, const T*, const T*,       \
                                   const T*, double*, cudaStream_t);                                    \
  template bamg_status rayleigh_finalize<T>(const double*, int, int, T*, double*, cudaStream_t);         \
  template bamg_status init_vectors<T>(int, int, int, uint64_t, T*, T*, cudaStream_t);                   \
  template bamg_status inject<T>(int, int, const int32_t*, const T*, T*, cudaStream_t);                  \
  template bamg_status csr_vec<T>(int, int, int, const int32_t*, const int32_t*, const T*, const T*, T,   \
                                  const T*, const T*, T*, cudaStream_t);                                \
  template bamg_status dense_gemv<T>(int, const T*, const T*, T*, cudaStream_t);                         \
  template bamg_status diag_inv<T>(int, const int32_t*, const int32_t*, const double*, const int32_t*,  \
                                   const double*, T*, int*, int*, cudaStream_t);                        \
  template bamg_status relax_block2<T>(int, int, const int32_t*, const int32_t*, const T*, const int32_t*, \
                                       const int32_t*, const T*, const T*, const T*, T*, const T*, T*,    \
                                       const T*, const T*, const T*, T, int, cudaStream_t);              \
  template bamg_status spmm_block_multi<T>(int, const SpmmJob<T>*, int, cudaStream_t);

BAMG_INST(float)
BAMG_INST(double)
template bamg_status norms_weights_ws<float>(int, int, int, const int32_t*, const int32_t*, const float*, float*,
                                             int, int, double*, int, double*, float*, double*, double*,
                                             cudaStream_t);
template bamg_status norms_weights_ws<double>(int, int, int, const int32_t*, const int32_t*, const double*,
                                              double*, int, int, double*, int, double*, double*, double*, double*,
                                              cudaStream_t);
template bamg_status convert<double, float>(size_t, const double*, float*, cudaStream_t);
template bamg_status convert<float, double>(size_t, const float*, double*, cudaStream_t);
template bamg_status convert<double, double>(size_t, const double*, double*, cudaStream_t);
template bamg_status convert<float, float>(size_t, const float*, float*, cudaStream_t);

}  // namespace bamg
