// Coarsest-level dense problems in one thread-block cluster.
//
// eq. generalized_eigenvalue: the r smallest generalized singular triplets of
// (B, M, N): B v = sigma M u, B^T u = sigma N v.  With Cholesky factors
// M = L_M L_M^T and N = L_N L_N^T they are the singular triplets of
// C = L_M^{-1} B L_N^{-T}; u = L_M^{-T} u~, v = L_N^{-T} v~.
//
// Only the r smallest triplets are needed, so the SVD of C goes through
// Householder bidiagonalization C = Q_B D P_B^T (Golub-Kahan), the r
// smallest singular values of the bidiagonal D by multisection on its
// Golub-Kahan tridiagonal form (Sturm counts), their right vectors by
// inverse iteration on that tridiagonal (orthogonalised within clusters of
// close values), and v~ = P_B v_D.  The left vector is u~ = C v~ / ||C v~||;
// for the zero singular value it is known in closed form, because 1^T B = 0
// makes u proportional to 1 (Section 5).
//
// Section 3, eq. coarse_grid_correction: the V-cycle applies the
// pseudo-inverse of B.  With the unit null vectors e = 1/sqrt(n) (left) and w
// (right), B^+ = (B + e w^T)^{-1} - w e^T; the inverse is Gauss-Jordan
// elimination with partial pivoting.
//
// Mapping: one cluster of up to 16 blocks.  Every n x n matrix is row-major
// and its rows are owned cyclically (row i by block i mod NB); a block only
// writes its own rows, so they stay in its L1.  The sequential algorithms
// (Cholesky, triangular solves, bidiagonalization, Gauss-Jordan) advance one
// index per step: the owner of the next pivot row publishes the vector all
// blocks need, then a hardware cluster barrier, then every block updates its
// own rows.  Published vectors are read through L2 (__ldcg).
#include <cooperative_groups.h>

#include <cfloat>
#include <cstdio>
#include <cstdlib>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace bamg {

constexpr int kDenseThreads = 256;
constexpr int kWarps = kDenseThreads / 32;
constexpr int kDenseMaxN = 1024;
constexpr int kMaxR = 32;
constexpr int kMaxNB = 16;

struct DenseCtl {
  int err;                    // 2 = M or N not positive definite
  int pad;
  unsigned long long tp[10];  // globaltimer at phase ends (block 0), for tracing
};

__device__ inline unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr double v = FLT_EPSILON; static constexpr double tiny = FLT_MIN; };
template <> struct Eps<double> { static constexpr double v = DBL_EPSILON; static constexpr double tiny = DBL_MIN; };

template <typename T>
struct DenseArgs {
  int n, r;
  const double *B, *M, *N;
  double *sigma, *U, *V, *Bpinv;
  T *LM, *LN;      // n x n: Cholesky factor L below the diagonal, L^T above
  T *X;            // n x n work (L_M^{-1} B, then its transpose solved with L_N)
  T *C;            // n x n: C = L_M^{-1} B L_N^{-T}
  T *W;            // n x n: bidiagonalization work
  T *Pr;           // n x n: right Householder vectors (row k = reflector k)
  T *G;            // n x 2n: Gauss-Jordan tableau
  T *R;            // n x 2r: right-hand sides of the triplet solves
  T *pub;          // 4 slots of 2n: published vectors (double buffered)
  T *part;         // kMaxNB x (n + 2 kMaxR + 2): per-block partial sums
  T *cval;         // kMaxNB: pivot candidates (value)
  int *cidx;       // kMaxNB: pivot candidates (row)
  int *pcol;       // n: pivot column assigned to each row (-1 = none yet)
  T *d, *e, *taup; // bidiagonal and right reflector scalars
  T *sig;          // r selected singular values
  T *vb;           // r x n: right vectors of the bidiagonal, then of C
  T *z;            // r x (6 * 2n): inverse iteration work, one slice per value
  T *unull;        // n: unit right null vector of B
  DenseCtl* ctl;
};

__device__ inline void csync() { cg::this_cluster().sync(); }

template <typename T> __device__ inline T ldcg(const T* p) { return __ldcg(p); }

// first index i >= from owned by block b (i mod NB == b)
__device__ inline int first_own(int b, int NB, int from) {
  int q = from - b;
  return q <= 0 ? b : b + ((q + NB - 1) / NB) * NB;
}

template <typename T>
__device__ T block_sum(T a, T* red) {
  a = warp_sum(a);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = a;
  __syncthreads();
  T s = 0;
  for (int k = 0; k < kWarps; ++k) s += red[k];
  __syncthreads();
  return s;
}

// ------------------------------------------------------------ Cholesky x 2
// Right-looking on the full symmetric trailing matrix.  The owner of row k
// publishes column k of L (row k of the trailing matrix over sqrt(a_kk));
// every block subtracts l l^T from its own rows.  On exit the lower triangle
// holds L and the upper triangle L^T.
template <typename T>
__device__ void chol_publish(const DenseArgs<T>& A, int m) {
  const int n = A.n;
  for (int f = 0; f < 2; ++f) {
    const T* L = f ? A.LN : A.LM;
    T* pb = A.pub + (size_t)(2 * f + (m & 1)) * n;
    T a = L[(size_t)m * n + m];
    T l = a > T(0) ? sqrt(a) : a;
    T inv = a > T(0) ? T(1) / l : T(0);
    for (int j = m + 1 + threadIdx.x; j < n; j += blockDim.x) pb[j] = L[(size_t)m * n + j] * inv;
    if (threadIdx.x == 0) pb[m] = l;
  }
}

template <typename T>
__device__ bool cholesky_rows(const DenseArgs<T>& A, int NB, T* sv) {
  const int n = A.n, b = blockIdx.x;
  for (int i = b; i < n; i += NB)
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      A.LM[(size_t)i * n + j] = T(A.M[(size_t)i * n + j]);
      A.LN[(size_t)i * n + j] = T(A.N[(size_t)i * n + j]);
    }
  __syncthreads();
  if (b == 0) chol_publish(A, 0);
  csync();
  T* sm = sv;
  T* sn = sv + n;
  for (int k = 0; k < n; ++k) {
    const T* pm = A.pub + (size_t)(k & 1) * n;
    const T* pn = A.pub + (size_t)(2 + (k & 1)) * n;
    for (int j = k + threadIdx.x; j < n; j += blockDim.x) {
      sm[j] = ldcg(pm + j);
      sn[j] = ldcg(pn + j);
    }
    __syncthreads();
    if (!(sm[k] > T(0)) || !(sn[k] > T(0))) {
      if (b == 0 && threadIdx.x == 0) A.ctl->err = 2;
      return false;  // every block reads the same pivots and leaves here
    }
    if (k % NB == b)
      for (int j = k + threadIdx.x; j < n; j += blockDim.x) {
        A.LM[(size_t)k * n + j] = sm[j];
        A.LN[(size_t)k * n + j] = sn[j];
      }
    for (int i = first_own(b, NB, k + 1); i < n; i += NB) {
      const T lm = sm[i], ln = sn[i];
      for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) {
        A.LM[(size_t)i * n + j] -= lm * sm[j];
        A.LN[(size_t)i * n + j] -= ln * sn[j];
      }
      if (threadIdx.x == 0) {
        A.LM[(size_t)i * n + k] = lm;
        A.LN[(size_t)i * n + k] = ln;
      }
    }
    __syncthreads();
    if (k + 1 < n && (k + 1) % NB == b) chol_publish(A, k + 1);
    csync();
  }
  return true;
}

// ------------------------------------------------ row triangular solves
// F holds L below and L^T above the diagonal.  X (n x ncol, row stride ld,
// own rows) is overwritten by L^{-1} X (FORWARD) or L^{-T} X (backward).  A
// second factor F2 may serve the columns from split on (F2 = nullptr: none).
template <typename T, bool FORWARD>
__device__ void row_solve(const DenseArgs<T>& A, int NB, const T* F, const T* F2, int split, T* X, int ld,
                          int ncol, T* sv) {
  const int n = A.n, b = blockIdx.x;
  auto pivot_row = [&](int m) {
    T* pb = A.pub + (size_t)(m & 1) * 2 * n;
    T* xm = X + (size_t)m * ld;
    const T d1 = F[(size_t)m * n + m];
    const T d2 = F2 ? F2[(size_t)m * n + m] : d1;
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
      T v = xm[c] / (c < split ? d1 : d2);
      xm[c] = v;
      pb[c] = v;
    }
  };
  int m = FORWARD ? 0 : n - 1;
  if (m % NB == b) pivot_row(m);
  csync();
  for (int s = 0; s < n; ++s, m += FORWARD ? 1 : -1) {
    const T* pb = A.pub + (size_t)(m & 1) * 2 * n;
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) sv[c] = ldcg(pb + c);
    __syncthreads();
    int i0 = FORWARD ? first_own(b, NB, m + 1) : b;
    for (int i = i0; FORWARD ? i < n : i < m; i += NB) {
      // forward: L[i][m] (below diagonal of row i); backward: L^T[i][m] (above)
      const T f1 = F[(size_t)i * n + m];
      const T f2 = F2 ? F2[(size_t)i * n + m] : f1;
      T* xi = X + (size_t)i * ld;
      for (int c = threadIdx.x; c < ncol; c += blockDim.x) xi[c] -= (c < split ? f1 : f2) * sv[c];
    }
    __syncthreads();
    int mn = FORWARD ? m + 1 : m - 1;
    if (s + 1 < n && mn % NB == b) pivot_row(mn);
    csync();
  }
}

// C = L_M^{-1} B L_N^{-T}; W = C for the bidiagonalization.
template <typename T>
__device__ void form_C(const DenseArgs<T>& A, int NB, T* sv) {
  const int n = A.n, b = blockIdx.x;
  for (int i = b; i < n; i += NB)
    for (int j = threadIdx.x; j < n; j += blockDim.x) A.X[(size_t)i * n + j] = T(A.B[(size_t)i * n + j]);
  __syncthreads();
  row_solve<T, true>(A, NB, A.LM, (const T*)nullptr, n, A.X, n, n, sv);   // X = L_M^{-1} B
  for (int i = b; i < n; i += NB)                                        // W = X^T (own rows)
    for (int j = threadIdx.x; j < n; j += blockDim.x) A.W[(size_t)i * n + j] = ldcg(A.X + (size_t)j * n + i);
  __syncthreads();
  row_solve<T, true>(A, NB, A.LN, (const T*)nullptr, n, A.W, n, n, sv);   // W = C^T
  for (int i = b; i < n; i += NB)                                        // C = W^T
    for (int j = threadIdx.x; j < n; j += blockDim.x) A.C[(size_t)i * n + j] = ldcg(A.W + (size_t)j * n + i);
  csync();  // all of W read before any block overwrites its rows
  for (int i = b; i < n; i += NB)
    for (int j = threadIdx.x; j < n; j += blockDim.x) A.W[(size_t)i * n + j] = A.C[(size_t)i * n + j];
  csync();
}

template <typename T>
__device__ void householder(T alpha, T s2, T& beta, T& tau, T& scale) {
  beta = alpha; tau = T(0); scale = T(0);
  if (s2 > T(0)) {
    T nrm = sqrt(alpha * alpha + s2);
    beta = alpha >= T(0) ? -nrm : nrm;
    tau = (beta - alpha) / beta;
    scale = T(1) / (alpha - beta);
  }
}


// ------------------------------------------------- Householder bidiagonalization
// W = Q_B D P_B^T, d[k] on the diagonal and e[k] above it; right reflectors
// I - taup[k] p_k p_k^T (p_k[k+1] = 1, support k+1..n-1) kept in row k of Pr
// (the left ones are not needed).  Left reflector of column k: each block
// sums x_i W[i][j] and x_i^2 over its own rows i > k into partials; after the
// barrier every block forms s_j = tau (W[k][j] + scale * sum_b partial_b[j])
// and updates its rows.  Right reflector of row k: built and published by
// the owner of row k, applied by every block to its own rows.
template <typename T>
__device__ void bidiag_partials(const DenseArgs<T>& A, int NB, int k) {
  const int n = A.n, b = blockIdx.x;
  const int stride = n + 2 * kMaxR + 2;
  T* part = A.part + (size_t)b * stride;
  const int i0 = first_own(b, NB, k + 1);
  for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) {
    T t = 0;
    for (int i = i0; i < n; i += NB) t += A.W[(size_t)i * n + k] * A.W[(size_t)i * n + j];
    part[j] = t;
  }
  if (threadIdx.x == 0) {
    T s2 = 0;
    for (int i = i0; i < n; i += NB) s2 += A.W[(size_t)i * n + k] * A.W[(size_t)i * n + k];
    part[n] = s2;
  }
  if (k % NB == b) {                       // publish row k for the other blocks
    T* rowk = A.pub;
    for (int j = k + threadIdx.x; j < n; j += blockDim.x) rowk[j] = A.W[(size_t)k * n + j];
  }
}

template <typename T>
__device__ void bidiagonalize(const DenseArgs<T>& A, int NB, T* sv, T* red) {
  const int n = A.n, b = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int stride = n + 2 * kMaxR + 2;
  T* s_vec = sv;          // n: s_j of the left reflector
  T* p_vec = sv + n;      // n: right reflector
  __shared__ T sc[4];
  bidiag_partials(A, NB, 0);
  csync();
  for (int k = 0; k < n; ++k) {
    // left reflector of column k
    if (threadIdx.x == 0) {
      T s2 = 0;
      for (int q = 0; q < NB; ++q) s2 += ldcg(A.part + (size_t)q * stride + n);
      T beta, tau, scale;
      householder(ldcg(A.pub + k), s2, beta, tau, scale);
      sc[0] = tau; sc[1] = scale;
      if (b == 0) A.d[k] = beta;
    }
    __syncthreads();
    const T tau = sc[0], scale = sc[1];
    for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) {
      T t = 0;
      for (int q = 0; q < NB; ++q) t += ldcg(A.part + (size_t)q * stride + j);
      s_vec[j] = tau * (ldcg(A.pub + j) + scale * t);
    }
    __syncthreads();
    if (tau != T(0)) {
      for (int i = first_own(b, NB, k); i < n; i += NB) {
        const T vi = (i == k) ? T(1) : A.W[(size_t)i * n + k] * scale;
        for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) A.W[(size_t)i * n + j] -= vi * s_vec[j];
      }
    }
    __syncthreads();
    if (k == n - 1) break;
    // right reflector of row k (owner builds and publishes it)
    T* pub_p = A.pub + 2 * n;
    if (k % NB == b) {
      const T* wk = A.W + (size_t)k * n;
      T s2 = 0;
      for (int j = k + 2 + threadIdx.x; j < n; j += blockDim.x) s2 += wk[j] * wk[j];
      s2 = block_sum(s2, red);
      T beta, taup, scp;
      householder(wk[k + 1], s2, beta, taup, scp);
      for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) {
        T pj = (j == k + 1) ? T(1) : wk[j] * scp;
        pub_p[j] = pj;
        A.Pr[(size_t)k * n + j] = pj;
      }
      for (int j = threadIdx.x; j <= k; j += blockDim.x) A.Pr[(size_t)k * n + j] = T(0);
      if (threadIdx.x == 0) {
        pub_p[n] = taup;
        A.e[k] = beta;
        A.taup[k] = taup;
      }
    }
    csync();
    const T taup = ldcg(pub_p + n);
    for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) p_vec[j] = ldcg(pub_p + j);
    __syncthreads();
    if (taup != T(0)) {
      for (int i = first_own(b, NB, k + 1) + NB * w; i < n; i += NB * kWarps) {   // one warp per row
        T* wi = A.W + (size_t)i * n;
        T sdot = 0;
        for (int j = k + 1 + lane; j < n; j += 32) sdot += wi[j] * p_vec[j];
        sdot = warp_sum(sdot) * taup;
        for (int j = k + 1 + lane; j < n; j += 32) wi[j] -= sdot * p_vec[j];
      }
    }
    __syncthreads();
    bidiag_partials(A, NB, k + 1);
    csync();
  }
  csync();
}

// ------------------------------------------------ bidiagonal singular values
// Golub-Kahan tridiagonal: zero diagonal, off-diagonals d0, e0, d1, e1, ...,
// d_{n-1}; its eigenvalues are +-sigma.  off(k) couples positions k-1 and k.
template <typename T>
__device__ inline T gk_off(const T* d, const T* e, int k) {
  return (k & 1) ? d[k >> 1] : e[(k >> 1) - 1];
}

// Number of eigenvalues of the tridiagonal below x (LDL^T Sturm count).
template <typename T>
__device__ int gk_count(const T* d, const T* e, int n, T x, T pivmin) {
  int cnt = 0;
  T q = -x;
  if (fabs(q) < pivmin) q = -pivmin;
  cnt += q < T(0);
  for (int k = 1; k < 2 * n; ++k) {
    T o = gk_off(d, e, k);
    q = -x - o * o / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < T(0);
  }
  return cnt;
}

template <typename T>
__device__ T gk_bound(const T* d, const T* e, int n) {
  T g = 0;
  for (int k = 0; k < 2 * n; ++k) {
    T a = k > 0 ? fabs(gk_off(d, e, k)) : T(0);
    T b = k + 1 < 2 * n ? fabs(gk_off(d, e, k + 1)) : T(0);
    g = fmax(g, a + b);
  }
  return g;
}

// sigma_a (a-th smallest, from 0) by 33-way multisection, one warp.
template <typename T>
__device__ T gk_sigma(const T* d, const T* e, int n, int a, T gmax, T pivmin) {
  const int lane = threadIdx.x & 31;
  T lo = 0, hi = gmax;
  const T eps = T(Eps<T>::v);
  for (int it = 0; it < 64; ++it) {
    if (hi - lo <= T(2) * eps * hi + T(2) * eps * gmax * T(1e-3)) break;
    T step = (hi - lo) / T(33);
    T x = lo + T(lane + 1) * step;
    int c = gk_count(d, e, n, x, pivmin) - n;
    unsigned bal = __ballot_sync(0xffffffffu, c >= a + 1);
    T nl, nh;
    if (bal) {
      int j = __ffs(bal) - 1;
      nh = lo + T(j + 1) * step;
      nl = j > 0 ? lo + T(j) * step : lo;
    } else {
      nl = lo + T(32) * step;
      nh = hi;
    }
    lo = nl;
    hi = nh;
  }
  return T(0.5) * (lo + hi);
}


// One lane: LU with partial pivoting of the tridiagonal T - sigma I (size m),
// storing reciprocal pivots for the solves.
template <typename T>
__device__ void gk_factor(const T* d, const T* e, int m, T sigma, T pert, T* dd, T* du, T* du2, T* dl,
                          T* piv) {
  for (int k = 0; k < m; ++k) {
    dd[k] = -sigma;
    du[k] = k + 1 < m ? gk_off(d, e, k + 1) : T(0);
    dl[k] = du[k];
    du2[k] = T(0);
  }
  for (int k = 0; k + 1 < m; ++k) {
    if (fabs(dd[k]) >= fabs(dl[k])) {
      piv[k] = T(0);
      if (dd[k] == T(0)) dd[k] = pert;
      T f = dl[k] / dd[k];
      dl[k] = f;
      dd[k + 1] -= f * du[k];
    } else {
      piv[k] = T(1);
      T f = dd[k] / dl[k];
      dd[k] = dl[k];
      dl[k] = f;
      T t = du[k];
      du[k] = dd[k + 1];
      dd[k + 1] = t - f * dd[k + 1];
      if (k + 2 < m) {
        du2[k] = du[k + 1];
        du[k + 1] = -f * du[k + 1];
      }
    }
  }
  if (dd[m - 1] == T(0)) dd[m - 1] = pert;
  for (int k = 0; k < m; ++k) dd[k] = T(1) / dd[k];   // reciprocal pivots
}

template <typename T>
__device__ void gk_solve(int m, const T* rdd, const T* du, const T* du2, const T* dl, const T* piv, T* b) {
  for (int k = 0; k + 1 < m; ++k) {
    if (piv[k] == T(0)) {
      b[k + 1] -= dl[k] * b[k];
    } else {
      T t = b[k];
      b[k] = b[k + 1];
      b[k + 1] = t - dl[k] * b[k];
    }
  }
  b[m - 1] *= rdd[m - 1];
  if (m > 1) b[m - 2] = (b[m - 2] - du[m - 2] * b[m - 1]) * rdd[m - 2];
  for (int k = m - 3; k >= 0; --k) b[k] = (b[k] - du[k] * b[k + 1] - du2[k] * b[k + 2]) * rdd[k];
}

// The r smallest singular values and right vectors of the bidiagonal, then
// v~ = P_B v_D.  sigma: one warp per value.  Values closer than
// sqrt(eps) * bound form a cluster; one warp per cluster runs inverse
// iteration on the Golub-Kahan tridiagonal, orthogonalising each member
// against the earlier ones.
template <typename T>
__device__ void bidiag_triplets(const DenseArgs<T>& A) {
  const int n = A.n, r = A.r, m = 2 * n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int gw = blockIdx.x * kWarps + w, GW = gridDim.x * kWarps;
  const T gmax = gk_bound(A.d, A.e, n);
  const T pivmin = T(Eps<T>::tiny) * fmax(T(1), gmax * gmax);
  for (int a = gw; a < r; a += GW) {
    T s = gk_sigma(A.d, A.e, n, a, gmax, pivmin);
    if (lane == 0) A.sig[a] = s;
  }
  csync();
  const T ortol = T(sqrt(Eps<T>::v)) * gmax;
  const T pert = T(Eps<T>::v) * gmax;
  int c = 0;
  for (int a0 = 0; a0 < r; ++a0) {
    if (a0 > 0 && ldcg(A.sig + a0) - ldcg(A.sig + a0 - 1) <= ortol) continue;
    int a1 = a0 + 1;
    while (a1 < r && ldcg(A.sig + a1) - ldcg(A.sig + a1 - 1) <= ortol) ++a1;
    if (c++ % GW != gw) continue;
    for (int a = a0; a < a1; ++a) {
      T* base = A.z + (size_t)a * 6 * m;
      T *dd = base, *du = base + m, *du2 = base + 2 * m, *dl = base + 3 * m, *pv = base + 4 * m;
      T* zv = base + 5 * m;
      if (lane == 0) gk_factor(A.d, A.e, m, ldcg(A.sig + a), pert, dd, du, du2, dl, pv);
      for (int k = lane; k < m; k += 32)
        zv[k] = T(1) + T(0.5) * T((unsigned)(k * 2654435761u) % 1000u) / T(1000) + T(a);
      __syncwarp();
      for (int it = 0; it < 4; ++it) {
        if (lane == 0) gk_solve(m, dd, du, du2, dl, pv, zv);
        __syncwarp();
        for (int q = a0; q < a; ++q) {           // orthogonalise within the cluster
          const T* zq = A.z + (size_t)q * 6 * m + 5 * m;
          T dot = 0;
          for (int k = lane; k < m; k += 32) dot += zq[k] * zv[k];
          dot = warp_sum(dot);
          for (int k = lane; k < m; k += 32) zv[k] -= dot * zq[k];
          __syncwarp();
        }
        T nrm = 0;
        for (int k = lane; k < m; k += 32) nrm += zv[k] * zv[k];
        nrm = warp_sum(nrm);
        T inv = nrm > T(0) ? T(1) / sqrt(nrm) : T(0);
        for (int k = lane; k < m; k += 32) zv[k] *= inv;
        __syncwarp();
      }
      T nv = 0;                                   // right vector: even positions
      for (int i = lane; i < n; i += 32) nv += zv[2 * i] * zv[2 * i];
      nv = warp_sum(nv);
      T inv = nv > T(0) ? T(1) / sqrt(nv) : T(0);
      for (int i = lane; i < n; i += 32) A.vb[(size_t)a * n + i] = zv[2 * i] * inv;
      __syncwarp();
    }
  }
  csync();
  for (int a = gw; a < r; a += GW) {              // v~ = P_B v_D, last reflector first
    T* y = A.vb + (size_t)a * n;
    for (int k = n - 2; k >= 0; --k) {
      const T tau = ldcg(A.taup + k);
      if (tau == T(0)) continue;
      const T* p = A.Pr + (size_t)k * n;
      T s = 0;
      for (int j = k + 1 + lane; j < n; j += 32) s += ldcg(p + j) * y[j];
      s = warp_sum(s) * tau;
      for (int j = k + 1 + lane; j < n; j += 32) y[j] -= s * ldcg(p + j);
      __syncwarp();
    }
  }
  csync();
}

// ------------------------------------------------------------- triplets
// Right-hand sides [v~_a | C v~_a / ||C v~_a||] in the own rows of R; both
// back substitutions (L_N^T for v, L_M^T for u) in one sweep; sign: largest
// |v_i| positive (lowest index on ties).  For a zero singular value (below
// n * eps * bound) u = 1 / sqrt(1^T M 1) and v normalised in the 2-norm is the
// right null vector w of B.
template <typename T>
__device__ void triplets(const DenseArgs<T>& A, int NB, T* sv, T* red) {
  const int n = A.n, r = A.r, r2 = 2 * r, b = blockIdx.x;
  const int stride = n + 2 * kMaxR + 2;
  T* part = A.part + (size_t)b * stride;
  const T gmax = gk_bound(A.d, A.e, n);
  const T null_tol = T(n * Eps<T>::v) * gmax;
  for (int i = b; i < n; i += NB)
    for (int c = threadIdx.x; c < r2; c += blockDim.x) {
      T val;
      if (c < r) {
        val = ldcg(A.vb + (size_t)c * n + i);
      } else {
        const T* va = A.vb + (size_t)(c - r) * n;
        const T* ci = A.C + (size_t)i * n;
        T acc = 0;
        for (int j = 0; j < n; ++j) acc += ci[j] * ldcg(va + j);
        val = acc;
      }
      A.R[(size_t)i * r2 + c] = val;
    }
  __syncthreads();
  for (int a = threadIdx.x; a < r; a += blockDim.x) {
    T s = 0;
    for (int i = b; i < n; i += NB) s += A.R[(size_t)i * r2 + r + a] * A.R[(size_t)i * r2 + r + a];
    part[a] = s;
  }
  {
    T s = 0;                                       // partial 1^T M 1 over own rows
    for (int i = b; i < n; i += NB)
      for (int j = threadIdx.x; j < n; j += blockDim.x) s += T(A.M[(size_t)i * n + j]);
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[n + r2 + 1] = s;
  }
  csync();
  for (int a = threadIdx.x; a < r; a += blockDim.x) {
    T s = 0;
    for (int q = 0; q < NB; ++q) s += ldcg(A.part + (size_t)q * stride + a);
    sv[a] = s > T(0) ? T(1) / sqrt(s) : T(0);
  }
  __syncthreads();
  for (int i = b; i < n; i += NB)
    for (int a = threadIdx.x; a < r; a += blockDim.x) A.R[(size_t)i * r2 + r + a] *= sv[a];
  __syncthreads();
  row_solve<T, false>(A, NB, A.LN, A.LM, r, A.R, r2, r2, sv);
  // sign candidates per value and the norm of v_0
  for (int a = threadIdx.x; a < r; a += blockDim.x) {
    T best = -1, bi = T(n), s0 = 0;
    for (int i = b; i < n; i += NB) {
      T v = A.R[(size_t)i * r2 + a];
      if (fabs(v) > best) { best = fabs(v); bi = T(i); }
      if (a == 0) s0 += v * v;
    }
    part[n + 2 * a] = best;
    part[n + 2 * a + 1] = bi;
    if (a == 0) part[n + r2] = s0;
  }
  csync();
  T* sgn = sv;          // r signs
  T* uconst = sv + r;   // 1 / sqrt(1^T M 1) and 1/||v_0||
  for (int a = threadIdx.x; a < r; a += blockDim.x) {
    T best = -1, bi = T(n);
    for (int q = 0; q < NB; ++q) {
      T v = ldcg(A.part + (size_t)q * stride + n + 2 * a);
      T ix = ldcg(A.part + (size_t)q * stride + n + 2 * a + 1);
      if (v > best || (v == best && ix < bi)) { best = v; bi = ix; }
    }
    T vv = A.R[(size_t)(int)bi * r2 + a];  // read through L2: row bi may belong to another block
    vv = ldcg(A.R + (size_t)(int)bi * r2 + a);
    sgn[a] = vv < T(0) ? T(-1) : T(1);
  }
  if (threadIdx.x == 0) {
    T s1 = 0, s0 = 0;
    for (int q = 0; q < NB; ++q) {
      s1 += ldcg(A.part + (size_t)q * stride + n + r2 + 1);
      s0 += ldcg(A.part + (size_t)q * stride + n + r2);
    }
    uconst[0] = T(1) / sqrt(s1);
    uconst[1] = s0 > T(0) ? T(1) / sqrt(s0) : T(0);
  }
  __syncthreads();
  const bool null0 = ldcg(A.sig) <= null_tol;
  for (int i = b; i < n; i += NB) {
    for (int a = threadIdx.x; a < r; a += blockDim.x) {
      const bool is_null = ldcg(A.sig + a) <= null_tol;
      T v = sgn[a] * A.R[(size_t)i * r2 + a];
      A.V[(size_t)i * r + a] = double(v);
      A.U[(size_t)i * r + a] = double(is_null ? uconst[0] : sgn[a] * A.R[(size_t)i * r2 + r + a]);
    }
    if (threadIdx.x == 0) A.unull[i] = null0 ? sgn[0] * A.R[(size_t)i * r2] * uconst[1] : T(0);
  }
  if (b == 0)
    for (int a = threadIdx.x; a < r; a += blockDim.x) A.sigma[a] = double(ldcg(A.sig + a));
  csync();
}

// ------------------------------------------------------------ pseudo-inverse
// B^+ = (B + e w^T)^{-1} - w e^T by Gauss-Jordan on [B + e w^T | I] with
// partial pivoting and no row exchanges: the row chosen for column k keeps
// its place and records k; at the end row i holds row pcol[i] of the inverse.
template <typename T>
__device__ void gj_candidate(const DenseArgs<T>& A, int NB, int k, T* red) {
  const int n = A.n, n2 = 2 * n, b = blockIdx.x;
  __shared__ T cv[kWarps];
  __shared__ int ci[kWarps];
  T best = -1;
  int bi = n;
  for (int i = b + NB * threadIdx.x; i < n; i += NB * blockDim.x) {
    if (A.pcol[i] >= 0) continue;
    T v = fabs(A.G[(size_t)i * n2 + k]);
    if (v > best) { best = v; bi = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    T ob = __shfl_xor_sync(0xffffffffu, best, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { cv[w] = best; ci[w] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < kWarps; ++q)
      if (cv[q] > best || (cv[q] == best && ci[q] < bi)) { best = cv[q]; bi = ci[q]; }
    A.cval[b] = best;
    A.cidx[b] = bi;
  }
  (void)red;
}

template <typename T>
__device__ void pseudo_inverse(const DenseArgs<T>& A, int NB, T* sv, T* red) {
  const int n = A.n, n2 = 2 * n, b = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const T e = T(1) / sqrt(T(n));
  for (int i = b; i < n; i += NB) {
    for (int j = threadIdx.x; j < n2; j += blockDim.x)
      A.G[(size_t)i * n2 + j] = j < n ? T(A.B[(size_t)i * n + j]) + e * ldcg(A.unull + j) : (j - n == i ? T(1) : T(0));
    if (threadIdx.x == 0) A.pcol[i] = -1;
  }
  __syncthreads();
  gj_candidate(A, NB, 0, red);
  csync();
  __shared__ int sp;
  T* prow = sv;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      T best = -1;
      int bi = n;
      for (int q = 0; q < NB; ++q) {
        T v = ldcg(A.cval + q);
        int ix = __ldcg(A.cidx + q);
        if (v > best || (v == best && ix < bi)) { best = v; bi = ix; }
      }
      sp = bi;
    }
    __syncthreads();
    const int p = sp;
    if (p % NB == b) {                          // normalise and publish the pivot row
      T* gp = A.G + (size_t)p * n2;
      const T inv = T(1) / gp[k];
      __syncthreads();
      for (int j = k + threadIdx.x; j < n2; j += blockDim.x) {
        T v = gp[j] * inv;
        gp[j] = v;
        A.pub[j] = v;
      }
      if (threadIdx.x == 0) A.pcol[p] = k;
    }
    csync();
    for (int j = k + threadIdx.x; j < n2; j += blockDim.x) prow[j] = ldcg(A.pub + j);
    __syncthreads();
    for (int i = b + NB * w; i < n; i += NB * kWarps) {   // one warp per own row
      if (i == p) continue;
      T* gi = A.G + (size_t)i * n2;
      const T f = gi[k];
      __syncwarp();
      if (f != T(0))
        for (int j = k + lane; j < n2; j += 32) gi[j] -= f * prow[j];
      __syncwarp();
    }
    __syncthreads();
    if (k + 1 < n) gj_candidate(A, NB, k + 1, red);
    csync();
  }
  for (int i = b; i < n; i += NB) {
    const int c = A.pcol[i];
    for (int j = threadIdx.x; j < n; j += blockDim.x)
      A.Bpinv[(size_t)c * n + j] = double(A.G[(size_t)i * n2 + n + j] - ldcg(A.unull + c) * e);
  }
}

template <typename T>
__global__ void __launch_bounds__(kDenseThreads, 1) coarsest_kernel(DenseArgs<T> A) {
  extern __shared__ unsigned char dyn[];
  T* sv = reinterpret_cast<T*>(dyn);
  __shared__ T red[kWarps];
  const int NB = gridDim.x;
  const bool b0 = blockIdx.x == 0 && threadIdx.x == 0;
  if (b0) A.ctl->tp[0] = gtimer();
  if (!cholesky_rows(A, NB, sv)) return;
  if (b0) A.ctl->tp[1] = gtimer();
  form_C(A, NB, sv);
  if (b0) A.ctl->tp[2] = gtimer();
  bidiagonalize(A, NB, sv, red);
  if (b0) A.ctl->tp[3] = gtimer();
  bidiag_triplets(A);
  if (b0) A.ctl->tp[4] = gtimer();
  triplets(A, NB, sv, red);
  if (b0) A.ctl->tp[5] = gtimer();
  if (A.Bpinv) pseudo_inverse(A, NB, sv, red);
  if (b0) A.ctl->tp[6] = gtimer();
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
  DevMem lm, ln, x, c, w, pr, g, rr, pub, part, cv, ci, pc, de, sg, vb, z, un, ctl;
  size_t nn = (size_t)n * n;
  BAMG_TRY(lm.alloc(sizeof(T) * nn, s));
  BAMG_TRY(ln.alloc(sizeof(T) * nn, s));
  BAMG_TRY(x.alloc(sizeof(T) * nn, s));
  BAMG_TRY(c.alloc(sizeof(T) * nn, s));
  BAMG_TRY(w.alloc(sizeof(T) * nn, s));
  BAMG_TRY(pr.alloc(sizeof(T) * nn, s));
  BAMG_TRY(g.alloc(Bpinv ? sizeof(T) * 2 * nn : 16, s));
  BAMG_TRY(rr.alloc(sizeof(T) * (size_t)n * 2 * r, s));
  BAMG_TRY(pub.alloc(sizeof(T) * 8 * (size_t)n + 64, s));
  BAMG_TRY(part.alloc(sizeof(T) * kMaxNB * (size_t)(n + 2 * kMaxR + 2), s));
  BAMG_TRY(cv.alloc(sizeof(T) * kMaxNB, s));
  BAMG_TRY(ci.alloc(sizeof(int) * kMaxNB, s));
  BAMG_TRY(pc.alloc(sizeof(int) * n, s));
  BAMG_TRY(de.alloc(sizeof(T) * 3 * n, s));
  BAMG_TRY(sg.alloc(sizeof(T) * r, s));
  BAMG_TRY(vb.alloc(sizeof(T) * (size_t)r * n, s));
  BAMG_TRY(z.alloc(sizeof(T) * (size_t)r * 12 * n, s));
  BAMG_TRY(un.alloc(sizeof(T) * n, s));
  BAMG_TRY(ctl.alloc(sizeof(DenseCtl), s));
  BAMG_CUDA(cudaMemsetAsync(ctl.p, 0, sizeof(DenseCtl), s));
  BAMG_CUDA(cudaMemsetAsync(un.p, 0, sizeof(T) * n, s));
  BAMG_CUDA(cudaMemsetAsync(de.p, 0, sizeof(T) * 3 * n, s));
  DenseArgs<T> a;
  a.n = n; a.r = r; a.B = B; a.M = M; a.N = N;
  a.sigma = sigma; a.U = U; a.V = V; a.Bpinv = Bpinv;
  a.LM = lm.as<T>(); a.LN = ln.as<T>(); a.X = x.as<T>(); a.C = c.as<T>(); a.W = w.as<T>(); a.Pr = pr.as<T>();
  a.G = g.as<T>(); a.R = rr.as<T>(); a.pub = pub.as<T>(); a.part = part.as<T>();
  a.cval = cv.as<T>(); a.cidx = ci.as<int>(); a.pcol = pc.as<int>();
  a.d = de.as<T>(); a.e = a.d + n; a.taup = a.e + n;
  a.sig = sg.as<T>(); a.vb = vb.as<T>(); a.z = z.as<T>(); a.unull = un.as<T>(); a.ctl = ctl.as<DenseCtl>();
  // at most 2 * 1024 doubles: below the default dynamic shared memory limit,
  // so no per-call attribute (a per-function setting would race between
  // threads that set up different chains concurrently)
  size_t smem = sizeof(T) * 2 * (size_t)n + 64;
  auto kern = coarsest_kernel<T>;
  BAMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.blockDim = dim3(kDenseThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.gridDim = dim3(kMaxNB);
  int csize = 8;
  {
    int maxc = 0;
    cfg.numAttrs = 0;
    if (cudaOccupancyMaxPotentialClusterSize(&maxc, (void*)kern, &cfg) == cudaSuccess && maxc >= 1)
      csize = maxc < kMaxNB ? maxc : kMaxNB;
    cudaGetLastError();
  }
  cfg.gridDim = dim3(csize);
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  BAMG_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  DenseCtl h;
  BAMG_CUDA(cudaMemcpyAsync(&h, ctl.p, sizeof(DenseCtl), cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  if (std::getenv("BAMG_TRACE")) {
    const char* nm[6] = {"cholesky", "form_C", "bidiag", "bidiag_svd", "triplets", "pinv"};
    fprintf(stderr, "[bamg] coarsest n=%d prec=%s cluster=%d:", n, sizeof(T) == 4 ? "f32" : "f64", csize);
    for (int k = 0; k < 6; ++k)
      if (h.tp[k + 1] >= h.tp[k] && h.tp[k + 1]) fprintf(stderr, " %s=%.1fus", nm[k], (h.tp[k + 1] - h.tp[k]) / 1e3);
    fprintf(stderr, "\n");
  }
  if (h.err == 2) {
    set_error("coarsest level: M or N is not positive definite");
    return BAMG_ERR_NUMERIC;
  }
  return BAMG_OK;
}

bamg_status coarsest_solve(int prec, int n, int r, const double* B, const double* M, const double* N,
                           double* sigma, double* U, double* V, double* Bpinv, cudaStream_t s) {
  if (n < 2 || n > kDenseMaxN || r < 1 || r > n || r > kMaxR) {
    set_error("coarsest solve needs 1 <= r <= min(n, %d), 2 <= n <= %d (n = %d, r = %d)", kMaxR, kDenseMaxN, n, r);
    return BAMG_ERR_UNSUPPORTED;
  }
  if (prec == 1) return coarsest_t<float>(n, r, B, M, N, sigma, U, V, Bpinv, s);
  return coarsest_t<double>(n, r, B, M, N, sigma, U, V, Bpinv, s);
}

}  // namespace bamg
