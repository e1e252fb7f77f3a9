// Coarsest-level dense problems, one cooperative kernel.
//
// eq. generalized_eigenvalue: the r smallest generalized singular triplets of
// (B, M, N): B v = sigma M u, B^T u = sigma N v.  With Cholesky factors
// M = L_M L_M^T, N = L_N L_N^T they are the singular triplets of
// C = L_M^{-1} B L_N^{-T}; u = L_M^{-T} u~, v = L_N^{-T} v~.  The SVD of C is
// the one-sided Jacobi method (Hestenes 1958) with the round-robin parallel
// ordering, accumulating the right vectors (accurate also for the null
// triplet).  For the zero singular value the left vector is known in closed
// form: 1^T B = 0 makes u proportional to 1 (Section 5).
//
// Section 3, eq. coarse_grid_correction: the V-cycle uses the pseudo-inverse
// of B.  With unit left/right null vectors e = 1/sqrt(n) and w,
// B^+ = (B + e w^T)^{-1} - w e^T; the inverse is Gauss-Jordan elimination
// with partial pivoting.
//
// Phases are separated by a grid-wide barrier whose waits are bounded: a
// block that waits longer than the limit raises an error flag and every
// block leaves the kernel; the host reports BAMG_ERR_TIMEOUT.
#include <cfloat>

#include "internal.cuh"

namespace bamg {

constexpr int kDenseThreads = 256;
constexpr int kDenseMaxN = 1024;
constexpr int kMaxSweeps = 40;

struct DenseCtl {
  unsigned int count;
  unsigned int gen;
  int err;            // 1 = barrier timeout, 2 = M or N not positive definite
  int pad;
  unsigned int rot[kMaxSweeps];
};

__device__ inline unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Returns false when the kernel must stop (timeout or error flag).
__device__ bool grid_barrier(DenseCtl* ctl) {
  __syncthreads();
  __shared__ int stop;
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = &ctl->gen;
    volatile int* err = &ctl->err;
    unsigned int g = *gen;
    __threadfence();
    unsigned int arrived = atomicAdd(&ctl->count, 1u);
    if (arrived == gridDim.x - 1) {
      ctl->count = 0;
      __threadfence();
      atomicAdd(&ctl->gen, 1u);
    } else {
      unsigned long long t0 = gtimer();
      while (*gen == g && *err == 0) {
        if (gtimer() - t0 > 2000000000ull) {  // 2 s
          atomicCAS(&ctl->err, 0, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    stop = *err != 0;
  }
  __syncthreads();
  return !stop;
}

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr double v = FLT_EPSILON; };
template <> struct Eps<double> { static constexpr double v = DBL_EPSILON; };

template <typename T>
struct DenseArgs {
  int n, r;
  const double *B, *M, *N;
  double *sigma, *U, *V, *Bpinv;
  T *LM, *LN;       // n x n: Cholesky factor in the lower triangle, its transpose above
  T *C, *W;         // n x n column-major: Jacobi iterate and accumulated rotations
  T *G;             // n x 2n row-major Gauss-Jordan tableau
  T *sig_all;       // n column norms
  int *order;       // r selected columns
  T *unull;         // n: normalised null vector w (Euclidean) of B
  DenseCtl* ctl;
};

template <typename T>
__device__ T block_sum3(T& a, T& b, T& c, T* red) {
  // reduces a, b, c over the block; results broadcast in a, b, c
  a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) { red[w] = a; red[32 + w] = b; red[64 + w] = c; }
  __syncthreads();
  if (threadIdx.x < 32) {
    int nw = blockDim.x >> 5;
    T x = lane < nw ? red[lane] : T(0), y = lane < nw ? red[32 + lane] : T(0),
      z = lane < nw ? red[64 + lane] : T(0);
    x = warp_sum(x); y = warp_sum(y); z = warp_sum(z);
    if (lane == 0) { red[0] = x; red[32] = y; red[64] = z; }
  }
  __syncthreads();
  a = red[0]; b = red[32]; c = red[64];
  __syncthreads();
  return a;
}

// ------------------------------------------------------------ phase helpers
template <typename T>
__device__ bool cholesky2(const DenseArgs<T>& A) {
  const int n = A.n;
  size_t gt = (size_t)blockIdx.x * blockDim.x + threadIdx.x, GT = (size_t)gridDim.x * blockDim.x;
  for (size_t t = gt; t < (size_t)n * n; t += GT) {
    A.LM[t] = T(A.M[t]);
    A.LN[t] = T(A.N[t]);
  }
  if (!grid_barrier(A.ctl)) return false;
  for (int k = 0; k < n; ++k) {
    T dm = A.LM[(size_t)k * n + k], dn = A.LN[(size_t)k * n + k];
    if (!(dm > T(0)) || !(dn > T(0))) {
      if (gt == 0) atomicCAS(&A.ctl->err, 0, 2);
      grid_barrier(A.ctl);
      return false;
    }
    T sm = sqrt(dm), sn = sqrt(dn);
    for (size_t t = gt; t < (size_t)2 * (n - k - 1); t += GT) {
      int which = (int)(t / (n - k - 1));
      int i = k + 1 + (int)(t % (n - k - 1));
      T* L = which ? A.LN : A.LM;
      T l = L[(size_t)i * n + k] / (which ? sn : sm);
      L[(size_t)i * n + k] = l;
      L[(size_t)k * n + i] = l;
    }
    if (!grid_barrier(A.ctl)) return false;
    int m = n - k - 1;
    for (size_t t = gt; t < (size_t)2 * m * m; t += GT) {
      int which = (int)(t / ((size_t)m * m));
      size_t u = t % ((size_t)m * m);
      int i = k + 1 + (int)(u / m), j = k + 1 + (int)(u % m);
      T* L = which ? A.LN : A.LM;
      L[(size_t)i * n + j] -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
    }
    if (gt == 0) { A.LM[(size_t)k * n + k] = sm; A.LN[(size_t)k * n + k] = sn; }
    if (!grid_barrier(A.ctl)) return false;
  }
  return true;
}

// Forward substitution L y = b with L stored as its transpose above the
// diagonal (row m of the upper part = column m of L, contiguous); one warp,
// b in shared memory, overwritten by y.
template <typename T>
__device__ void warp_lower_solve(const T* LT, int n, T* b) {
  int lane = threadIdx.x & 31;
  for (int m = 0; m < n; ++m) {
    T xm = b[m] / LT[(size_t)m * n + m];
    __syncwarp();
    for (int i = m + 1 + lane; i < n; i += 32) b[i] -= LT[(size_t)m * n + i] * xm;
    if (lane == 0) b[m] = xm;
    __syncwarp();
  }
}

// Back substitution L^T u = b with L lower (row m of L contiguous).
template <typename T>
__device__ void warp_upper_solve(const T* L, int n, T* b) {
  int lane = threadIdx.x & 31;
  for (int m = n - 1; m >= 0; --m) {
    T um = b[m] / L[(size_t)m * n + m];
    __syncwarp();
    for (int i = lane; i < m; i += 32) b[i] -= L[(size_t)m * n + i] * um;
    if (lane == 0) b[m] = um;
    __syncwarp();
  }
}

// C = L_M^{-1} B L_N^{-T}, stored column-major; W = I.
template <typename T>
__device__ bool form_C(const DenseArgs<T>& A, T* smem) {
  const int n = A.n;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T* b = smem + (size_t)w * n;
  int gw = blockIdx.x * nw + w, GW = gridDim.x * nw;
  // X = L_M^{-1} B, column j of B -> column j of X (kept in W, column-major)
  for (int j = gw; j < n; j += GW) {
    for (int i = lane; i < n; i += 32) b[i] = T(A.B[(size_t)i * n + j]);
    __syncwarp();
    warp_lower_solve(A.LM, n, b);
    for (int i = lane; i < n; i += 32) A.W[(size_t)j * n + i] = b[i];
    __syncwarp();
  }
  if (!grid_barrier(A.ctl)) return false;
  // row i of C = L_N^{-1} (row i of X)
  for (int i = gw; i < n; i += GW) {
    for (int j = lane; j < n; j += 32) b[j] = A.W[(size_t)j * n + i];
    __syncwarp();
    warp_lower_solve(A.LN, n, b);
    for (int j = lane; j < n; j += 32) A.C[(size_t)j * n + i] = b[j];
    __syncwarp();
  }
  if (!grid_barrier(A.ctl)) return false;
  size_t gt = (size_t)blockIdx.x * blockDim.x + threadIdx.x, GT = (size_t)gridDim.x * blockDim.x;
  for (size_t t = gt; t < (size_t)n * n; t += GT) A.W[t] = (t / n == t % n) ? T(1) : T(0);
  return grid_barrier(A.ctl);
}

__device__ inline void rr_pair(int N2, int t, int k, int& p, int& q) {
  int M = N2 - 1;
  if (k == 0) { p = t; q = N2 - 1; }
  else { p = (t + k) % M; q = (t - k + M) % M; }
  if (p > q) { int s = p; p = q; q = s; }
}

template <typename T>
__device__ bool jacobi_svd(const DenseArgs<T>& A, T* red) {
  const int n = A.n;
  const int N2 = n + (n & 1);
  const double tol = Eps<T>::v * sqrt((double)n);
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    for (int t = 0; t < N2 - 1; ++t) {
      for (int k = blockIdx.x; k < N2 / 2; k += gridDim.x) {
        int p, q;
        rr_pair(N2, t, k, p, q);
        if (q >= n) continue;  // padding column of an odd n
        T* cp = A.C + (size_t)p * n;
        T* cq = A.C + (size_t)q * n;
        T al = 0, be = 0, ga = 0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
          T x = cp[i], y = cq[i];
          al += x * x; be += y * y; ga += x * y;
        }
        block_sum3(al, be, ga, red);
        if (!(al > T(0) && be > T(0))) continue;
        if (!(fabs((double)ga) > tol * sqrt((double)al * (double)be))) continue;
        T zeta = (be - al) / (T(2) * ga);
        T tt = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
        T cs = T(1) / sqrt(T(1) + tt * tt), sn = cs * tt;
        T* wp = A.W + (size_t)p * n;
        T* wq = A.W + (size_t)q * n;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
          T x = cp[i], y = cq[i];
          cp[i] = cs * x - sn * y;
          cq[i] = sn * x + cs * y;
          T u = wp[i], v = wq[i];
          wp[i] = cs * u - sn * v;
          wq[i] = sn * u + cs * v;
        }
        if (threadIdx.x == 0) atomicAdd(&A.ctl->rot[sweep], 1u);
      }
      if (!grid_barrier(A.ctl)) return false;
    }
    if (*(volatile unsigned int*)&A.ctl->rot[sweep] == 0) break;
  }
  return true;
}

// sigma_j = ||C e_j||; the r smallest (ties by index) become order[0..r).
template <typename T>
__device__ bool select_smallest(const DenseArgs<T>& A, T* red) {
  const int n = A.n;
  for (int j = blockIdx.x; j < n; j += gridDim.x) {
    T a = 0, b = 0, c = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      T x = A.C[(size_t)j * n + i];
      a += x * x;
    }
    block_sum3(a, b, c, red);
    if (threadIdx.x == 0) A.sig_all[j] = sqrt(a);
  }
  if (!grid_barrier(A.ctl)) return false;
  size_t gt = (size_t)blockIdx.x * blockDim.x + threadIdx.x, GT = (size_t)gridDim.x * blockDim.x;
  for (size_t j = gt; j < (size_t)n; j += GT) {
    T sj = A.sig_all[j];
    int rank = 0;
    for (int m = 0; m < n; ++m) {
      T sm = A.sig_all[m];
      rank += (sm < sj || (sm == sj && m < (int)j)) ? 1 : 0;
    }
    if (rank < A.r) A.order[rank] = (int)j;
  }
  return grid_barrier(A.ctl);
}

// u = L_M^{-T} (C e_j / sigma_j), v = L_N^{-T} W e_j; sign of v fixed by its
// largest-magnitude entry (lowest index on ties); for the null triplet u is
// the positive constant 1/sqrt(1^T M 1).  Also stores the unit null vector w.
template <typename T>
__device__ bool triplets(const DenseArgs<T>& A, T* smem) {
  const int n = A.n, r = A.r;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int gw = blockIdx.x * nw + w, GW = gridDim.x * nw;
  T smax = 0;
  for (int m = 0; m < n; ++m) smax = fmax(smax, A.sig_all[m]);
  T null_tol = T(n * Eps<T>::v) * smax;
  T* b = smem + (size_t)w * n;
  for (int a = gw; a < r; a += GW) {
    int j = A.order[a];
    T sj = A.sig_all[j];
    bool is_null = sj <= null_tol;
    // v = L_N^{-T} W e_j
    for (int i = lane; i < n; i += 32) b[i] = A.W[(size_t)j * n + i];
    __syncwarp();
    warp_upper_solve(A.LN, n, b);
    // sign: largest |v_i|, lowest index on ties
    T best = -1; int bi = n;
    for (int i = lane; i < n; i += 32) {
      T av = fabs(b[i]);
      if (av > best || (av == best && i < bi)) { best = av; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      T ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    T sgn = b[bi] < T(0) ? T(-1) : T(1);
    T nv = 0;
    for (int i = lane; i < n; i += 32) {
      T v = sgn * b[i];
      A.V[(size_t)i * r + a] = double(v);
      nv += v * v;
    }
    nv = warp_sum(nv);
    if (is_null && a == 0) {
      T inv = T(1) / sqrt(nv);
      for (int i = lane; i < n; i += 32) A.unull[i] = sgn * b[i] * inv;
    }
    __syncwarp();
    if (is_null) {
      // 1^T M 1 = ||L_M^T 1||^2 ; u = 1 / sqrt(1^T M 1)
      T s = 0;
      for (int i = lane; i < n; i += 32)
        for (int m = 0; m < n; ++m) s += T(A.M[(size_t)i * n + m]);
      s = warp_sum(s);
      T u = T(1) / sqrt(s);
      for (int i = lane; i < n; i += 32) A.U[(size_t)i * r + a] = double(u);
    } else {
      for (int i = lane; i < n; i += 32) b[i] = A.C[(size_t)j * n + i] / sj;
      __syncwarp();
      warp_upper_solve(A.LM, n, b);
      for (int i = lane; i < n; i += 32) A.U[(size_t)i * r + a] = double(sgn * b[i]);
    }
    if (lane == 0) A.sigma[a] = double(sj);
    __syncwarp();
  }
  return grid_barrier(A.ctl);
}

// B^+ = (B + e w^T)^{-1} - w e^T, e = 1/sqrt(n), Gauss-Jordan with partial
// pivoting on the n x 2n tableau [B + e w^T | I].
template <typename T>
__device__ bool pseudo_inverse(const DenseArgs<T>& A, T* smem, T* red) {
  const int n = A.n, n2 = 2 * n;
  const T e = T(1) / sqrt(T(n));
  size_t gt = (size_t)blockIdx.x * blockDim.x + threadIdx.x, GT = (size_t)gridDim.x * blockDim.x;
  for (size_t t = gt; t < (size_t)n * n2; t += GT) {
    int i = (int)(t / n2), j = (int)(t % n2);
    A.G[t] = j < n ? T(A.B[(size_t)i * n + j]) + e * A.unull[j] : (j - n == i ? T(1) : T(0));
  }
  if (!grid_barrier(A.ctl)) return false;
  T* prow = smem;
  T* krow = smem + n2;
  __shared__ T pv[kDenseThreads];
  __shared__ int pi[kDenseThreads];
  for (int k = 0; k < n; ++k) {
    // pivot: largest |G[i][k]|, i >= k, lowest index on ties (every block)
    T best = -1; int bi = n;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
      T a = fabs(A.G[(size_t)i * n2 + k]);
      if (a > best) { best = a; bi = i; }
    }
    pv[threadIdx.x] = best; pi[threadIdx.x] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) {
        T ob = pv[threadIdx.x + o]; int oi = pi[threadIdx.x + o];
        if (ob > pv[threadIdx.x] || (ob == pv[threadIdx.x] && oi < pi[threadIdx.x])) {
          pv[threadIdx.x] = ob; pi[threadIdx.x] = oi;
        }
      }
      __syncthreads();
    }
    int p = pi[0];
    for (int j = threadIdx.x; j < n2; j += blockDim.x) {
      prow[j] = A.G[(size_t)p * n2 + j];
      krow[j] = A.G[(size_t)k * n2 + j];
    }
    __syncthreads();
    T piv = prow[k];
    if (!grid_barrier(A.ctl)) return false;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
      T* gi = A.G + (size_t)i * n2;
      const T* src = (i == p) ? krow : gi;
      T f = (i == k) ? T(0) : src[k];
      __syncthreads();
      for (int j = threadIdx.x; j < n2; j += blockDim.x) {
        if (j < k) continue;
        T pj = prow[j] / piv;
        gi[j] = (i == k) ? pj : src[j] - f * pj;
      }
      __syncthreads();
    }
    if (!grid_barrier(A.ctl)) return false;
  }
  for (size_t t = gt; t < (size_t)n * n; t += GT) {
    int i = (int)(t / n), j = (int)(t % n);
    A.Bpinv[t] = double(A.G[(size_t)i * n2 + n + j] - A.unull[i] * e);
  }
  return true;
}

template <typename T>
__global__ void __launch_bounds__(kDenseThreads) coarsest_kernel(DenseArgs<T> A) {
  extern __shared__ unsigned char dyn[];
  T* smem = reinterpret_cast<T*>(dyn);
  __shared__ T red[96];
  if (!cholesky2(A)) return;
  if (!form_C(A, smem)) return;
  if (!jacobi_svd(A, red)) return;
  if (!select_smallest(A, red)) return;
  if (!triplets(A, smem)) return;
  if (A.Bpinv) pseudo_inverse(A, smem, red);
}

__global__ void csr_to_dense_kernel(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                    const double* __restrict__ va, double* __restrict__ D) {
  int i = blockIdx.x;
  for (int p = rp[i] + threadIdx.x; p < rp[i + 1]; p += blockDim.x) D[(size_t)i * n + ci[p]] = va[p];
}

bamg_status csr_to_dense(int n, const int32_t* rp, const int32_t* ci, const double* va, double* D,
                         cudaStream_t s) {
  BAMG_CUDA(cudaMemsetAsync(D, 0, sizeof(double) * (size_t)n * n, s));
  return launch(csr_to_dense_kernel, dim3(n), dim3(64), 0, s, n, rp, ci, va, D);
}

template <typename T>
static bamg_status coarsest_t(int n, int r, const double* B, const double* M, const double* N, double* sigma,
                              double* U, double* V, double* Bpinv, cudaStream_t s) {
  DevMem lm, ln, c, w, g, sg, ord, un, ctl;
  size_t nn = (size_t)n * n;
  BAMG_TRY(lm.alloc(sizeof(T) * nn, s));
  BAMG_TRY(ln.alloc(sizeof(T) * nn, s));
  BAMG_TRY(c.alloc(sizeof(T) * nn, s));
  BAMG_TRY(w.alloc(sizeof(T) * nn, s));
  BAMG_TRY(g.alloc(Bpinv ? sizeof(T) * 2 * nn : 16, s));
  BAMG_TRY(sg.alloc(sizeof(T) * n, s));
  BAMG_TRY(ord.alloc(sizeof(int) * (r + 1), s));
  BAMG_TRY(un.alloc(sizeof(T) * n, s));
  BAMG_TRY(ctl.alloc(sizeof(DenseCtl), s));
  BAMG_CUDA(cudaMemsetAsync(ctl.p, 0, sizeof(DenseCtl), s));
  BAMG_CUDA(cudaMemsetAsync(un.p, 0, sizeof(T) * n, s));
  DenseArgs<T> a;
  a.n = n; a.r = r; a.B = B; a.M = M; a.N = N;
  a.sigma = sigma; a.U = U; a.V = V; a.Bpinv = Bpinv;
  a.LM = lm.as<T>(); a.LN = ln.as<T>(); a.C = c.as<T>(); a.W = w.as<T>(); a.G = g.as<T>();
  a.sig_all = sg.as<T>(); a.order = ord.as<int>(); a.unull = un.as<T>(); a.ctl = ctl.as<DenseCtl>();
  size_t smem = sizeof(T) * (size_t)(kDenseThreads / 32) * n;
  if (smem < sizeof(T) * 2 * 2 * (size_t)n) smem = sizeof(T) * 4 * (size_t)n;
  auto kern = coarsest_kernel<T>;
  BAMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, per_sm = 0;
  BAMG_CUDA(cudaGetDevice(&dev));
  BAMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kDenseThreads, smem));
  if (per_sm < 1) {
    set_error("coarsest kernel cannot be resident (shared memory %zu B)", smem);
    return BAMG_ERR_UNSUPPORTED;
  }
  int grid = num_sms();  // one block per SM: co-resident by the cooperative launch
  int want = (n + 1) / 2;
  if (grid > want) grid = want;
  if (grid < 1) grid = 1;
  void* args[] = {&a};
  BAMG_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(kDenseThreads), args, smem, s));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  DenseCtl h;
  BAMG_CUDA(cudaMemcpyAsync(&h, ctl.p, sizeof(DenseCtl), cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  if (h.err == 1) {
    set_error("coarsest kernel: grid barrier wait exceeded its limit");
    return BAMG_ERR_TIMEOUT;
  }
  if (h.err == 2) {
    set_error("coarsest level: M or N is not positive definite");
    return BAMG_ERR_NUMERIC;
  }
  return BAMG_OK;
}

bamg_status coarsest_solve(int prec, int n, int r, const double* B, const double* M, const double* N,
                           double* sigma, double* U, double* V, double* Bpinv, cudaStream_t s) {
  if (n < 1 || n > kDenseMaxN || r < 1 || r > n) {
    set_error("coarsest solve needs 1 <= r <= n <= %d (n = %d, r = %d)", kDenseMaxN, n, r);
    return BAMG_ERR_UNSUPPORTED;
  }
  if (prec == 1) return coarsest_t<float>(n, r, B, M, N, sigma, U, V, Bpinv, s);
  return coarsest_t<double>(n, r, B, M, N, sigma, U, V, Bpinv, s);
}

}  // namespace bamg
