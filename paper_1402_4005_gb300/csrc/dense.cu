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
// pseudo-inverse of B.  With e = 1/sqrt(n) 1 (the unit left null vector,
// 1^T B = 0) the matrix B + e e^T is nonsingular and X = (B + e e^T)^{-1}
// satisfies e^T X = e^T and X e = w / (e^T w) for the right null vector w;
// then B^+ = (I - w w^T) X (I - e e^T) (B B^+ = I - e e^T, B^+ B = I - w w^T).
// None of this needs the singular triplets, so X (Gauss-Jordan with partial
// pivoting) runs in a second cluster concurrently with the triplets.
//
// Mapping: one cluster of up to 16 blocks.  Rows of every n x n matrix are
// owned cyclically (row i by block i mod NB) and only their owner writes
// them.  The sequential algorithms (Cholesky, triangular solves,
// bidiagonalization, Gauss-Jordan) advance one index per step: the owner of
// the next pivot row publishes the vector all blocks need, a hardware
// cluster barrier follows, then every block updates its own rows.
//
// Two storage policies share this code.  Shared (SM = true, when the own
// rows of all matrices fit): each block keeps its own rows, its published
// vectors and its partial sums in shared memory, and the other blocks read
// them through distributed shared memory, so a step costs a barrier and one
// remote read.  Global (SM = false, larger n): the same arrays live in global
// memory and remote reads go through L2 (__ldcg).  Reductions over the NB
// blocks load the NB partials in parallel (unrolled to the cluster limit).
#include <cooperative_groups.h>

#include <atomic>
#include <cfloat>
#include <cstddef>
#include <chrono>
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

// Row-owned arrays (LM ... pcol) are, under the shared policy, the compact
// own rows of the block (local row i / NB); under the global policy, the
// full arrays.  The remaining arrays are global under both policies.
template <typename T>
struct DenseArgs {
  int n, r, NB, RP;      // size, triplets, cluster blocks, own rows per block
  const double *B, *M, *N;
  double *sigma, *U, *V, *Bpinv;
  T *LM, *LN;      // Cholesky factor L below the diagonal, L^T above
  T *S1;           // X = L_M^{-1} B, then C = L_M^{-1} B L_N^{-T}
  T *S2;           // W: C^T during the solves, then C for the bidiagonalization
  T *S3;           // right Householder vectors (row k = reflector k)
                   // S2 and S3 are adjacent: Gauss-Jordan tableau G (2n per row)
  T *R;            // n x 2r: right-hand sides of the triplet solves
  T *pub;          // published vectors: 4 slots of 2n (+ 64)
  T *part;         // partial sums of a block: part_stride(n) entries
  int *pcol;       // pivot column assigned to each row (-1 = none yet)
  T *d, *e, *taup; // bidiagonal and right reflector scalars
  T *sig;          // r selected singular values
  T *vb;           // r x n: right vectors of the bidiagonal, then of C
  T *z;            // r x (6 * 2n): inverse iteration work, one slice per value
  T *unull;        // n: unit right null vector of B
  DenseCtl* ctl;
};

// partial sums of a block: [0, n) a vector, then scalars, per-value slots and
// two pivot slots; the bidiagonalization double-buffers its column partials
// (n + 1 entries at offset (k & 1) * (n + 1)), hence the 2n.
__host__ __device__ inline int part_stride(int n) { return 2 * n + 2 * kMaxR + 8; }

__device__ inline void csync() { cg::this_cluster().sync(); }

template <bool SM, typename T> __device__ inline T rd(const T* p) {
  if constexpr (SM) return *p;
  else return __ldcg(p);
}

// blocks of the cluster: a compile-time 16 under the shared policy (index
// arithmetic by shifts), the launched cluster size otherwise
template <bool SM, typename T> __device__ inline int nblocks(const DenseArgs<T>& A) {
  if constexpr (SM) return kMaxNB;
  else return A.NB;
}

// own row i of a row-owned array with row length ld
template <bool SM, typename T>
__device__ inline T* own(const DenseArgs<T>& A, T* base, int i, int ld) {
  if constexpr (SM) return base + (size_t)(i / kMaxNB) * ld;
  else return base + (size_t)i * ld;
}
// row i of a row-owned array, possibly owned by another block
template <bool SM, typename T>
__device__ inline const T* any(const DenseArgs<T>& A, T* base, int i, int ld) {
  if constexpr (SM) return cg::this_cluster().map_shared_rank(base + (size_t)(i / kMaxNB) * ld, i % kMaxNB);
  else return base + (size_t)i * ld;
}
template <bool SM, typename T>
__device__ inline int* own_pcol(const DenseArgs<T>& A, int i) {
  if constexpr (SM) return A.pcol + i / kMaxNB;
  else return A.pcol + i;
}
// publication buffer: written by its owner, read by everyone
template <bool SM, typename T> __device__ inline T* pub_w(const DenseArgs<T>& A) { return A.pub; }
template <bool SM, typename T> __device__ inline const T* pub_r(const DenseArgs<T>& A, int owner) {
  if constexpr (SM) return cg::this_cluster().map_shared_rank(A.pub, owner);
  else return A.pub;
}
template <bool SM, typename T> __device__ inline T* part_w(const DenseArgs<T>& A) {
  if constexpr (SM) return A.part;
  else return A.part + (size_t)blockIdx.x * part_stride(A.n);
}
template <bool SM, typename T> __device__ inline const T* part_r(const DenseArgs<T>& A, int q) {
  if constexpr (SM) return cg::this_cluster().map_shared_rank(A.part, q);
  else return A.part + (size_t)q * part_stride(A.n);
}
// sum over the blocks of partial slot k (the loads are issued together)
template <bool SM, typename T>
__device__ inline T part_sum(const DenseArgs<T>& A, int k) {
  T v[kMaxNB];
#pragma unroll
  for (int q = 0; q < kMaxNB; ++q) v[q] = q < nblocks<SM>(A) ? rd<SM>(part_r<SM>(A, q) + k) : T(0);
  T s = 0;
#pragma unroll
  for (int q = 0; q < kMaxNB; ++q) s += v[q];
  return s;
}

// first index i >= from owned by block b (i mod NB == b)
__device__ inline int first_own(int b, int NB, int from) {
  int q = from - b;
  return q <= 0 ? b : b + ((q + NB - 1) / NB) * NB;
}

// store(e, load(e)) for e in [0, count) over the block's threads, eight
// loads per thread issued before their stores: loads from another block's
// shared memory (or L2) then overlap, where a store between them (which the
// compiler must assume may alias the next load) would serialise them.
template <typename T, typename Load, typename Store>
__device__ inline void batched_copy(int count, Load load, Store store) {
  constexpr int kB = 8;
  for (int e0 = threadIdx.x; e0 < count; e0 += kB * blockDim.x) {
    T v[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      v[u] = e < count ? load(e) : T(0);
    }
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      if (e < count) store(e, v[u]);
    }
  }
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
// Right-looking blocked Cholesky of M and N together, on the full symmetric
// trailing matrices, kCholK columns per cluster step.  Every block fetches
// the step's panel rows from their owners, factors the kCholK x kCholK
// diagonal block and forms the panel rows of L^T itself (the same arithmetic
// in every block), then subtracts the panel's rank-kCholK product from its
// own trailing rows.  The owners store the finished panel rows after the
// step's barrier, when no block reads them any more.  On exit the lower
// triangle holds L and the upper triangle L^T.
constexpr int kCholK = 4;

template <bool SM, typename T>
__device__ bool cholesky_rows(const DenseArgs<T>& A, T* sv) {
  const int n = A.n, NB = nblocks<SM>(A), b = blockIdx.x;
  // 2 kCholK panel rows of length n (M rows, then N rows): the block's own
  // publication buffer under the shared policy (no block publishes during
  // the factorization), its dynamic shared memory after the 3n scratch
  // otherwise
  T* stage = SM ? A.pub : sv + 3 * n;
  __shared__ T pinv[2 * kCholK];
  __shared__ int bad;
  for (int i = b; i < n; i += NB) {
    T* lm = own<SM>(A, A.LM, i, n);
    T* ln = own<SM>(A, A.LN, i, n);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      lm[j] = T(A.M[(size_t)i * n + j]);
      ln[j] = T(A.N[(size_t)i * n + j]);
    }
  }
  if (threadIdx.x == 0) bad = 0;
  csync();
  // owner rows of the panel starting at p0 (pk rows) from the staged L^T rows
  auto store_panel = [&](int p0, int pk) {
    for (int p = 0; p < pk; ++p) {
      const int m = p0 + p;
      if (m % NB != b) continue;
      T* lm = own<SM>(A, A.LM, m, n);
      T* ln = own<SM>(A, A.LN, m, n);
      for (int j = p0 + threadIdx.x; j < n; j += blockDim.x) {
        // left of the diagonal: L[m][j] = (L^T)[j][m], a staged panel row
        const int pr = j < m ? j - p0 : p, col = j < m ? m : j;
        lm[j] = stage[(size_t)pr * n + col];
        ln[j] = stage[(size_t)(kCholK + pr) * n + col];
      }
    }
  };
  for (int k0 = 0; k0 < n; k0 += kCholK) {
    const int kk = min(kCholK, n - k0);
    if (k0 > 0) {
      store_panel(k0 - kCholK, kCholK);
      __syncthreads();
    }
    for (int j = k0 + threadIdx.x; j < n; j += blockDim.x) {   // loads batched across the rows
      T x[2 * kCholK];
#pragma unroll
      for (int u = 0; u < 2 * kCholK; ++u) {
        const int f = u / kCholK, p = u % kCholK;
        x[u] = p < kk ? rd<SM>(any<SM>(A, f ? A.LN : A.LM, k0 + p, n) + j) : T(0);
      }
#pragma unroll
      for (int u = 0; u < 2 * kCholK; ++u)
        if (u % kCholK < kk) stage[(size_t)u * n + j] = x[u];
    }
    __syncthreads();
    // diagonal blocks: thread 0 (M) and thread 32 (N), in registers, in
    // place: U = L^T
    if ((threadIdx.x & 31) == 0 && threadIdx.x < 64) {
      const int f = threadIdx.x >> 5;
      T* U = stage + (size_t)f * kCholK * n + k0;
      T a[kCholK][kCholK];
#pragma unroll
      for (int p = 0; p < kCholK; ++p)
#pragma unroll
        for (int c = 0; c < kCholK; ++c) a[p][c] = (c >= p && c < kk) ? U[(size_t)p * n + c] : T(0);
      bool ok = true;
#pragma unroll
      for (int p = 0; p < kCholK; ++p) {
        if (p < kk) {
          T d = a[p][p];
#pragma unroll
          for (int q = 0; q < p; ++q) d -= a[q][p] * a[q][p];
          ok = ok && d > T(0);
          const T l = sqrt(d), inv = T(1) / l;
          a[p][p] = l;
          pinv[f * kCholK + p] = inv;
#pragma unroll
          for (int c = p + 1; c < kCholK; ++c) {
            T t = a[p][c];
#pragma unroll
            for (int q = 0; q < p; ++q) t -= a[q][p] * a[q][c];
            a[p][c] = t * inv;
          }
        }
      }
#pragma unroll
      for (int p = 0; p < kCholK; ++p)
#pragma unroll
        for (int c = 0; c < kCholK; ++c)
          if (c >= p && c < kk) U[(size_t)p * n + c] = a[p][c];
      if (!ok) bad = 1;
    }
    __syncthreads();
    if (bad) {
      if (b == 0 && threadIdx.x == 0) A.ctl->err = 2;
      csync();       // every block reaches the same verdict at the same step
      return false;
    }
    // the panel rows of L^T right of the diagonal block: a thread per column
    const int w2 = n - k0 - kk;
    for (int e = threadIdx.x; e < 2 * w2; e += blockDim.x) {
      const int f = e / w2, j = k0 + kk + (e - f * w2);
      T* U = stage + (size_t)f * kCholK * n;
      T u[kCholK];
#pragma unroll
      for (int p = 0; p < kCholK; ++p) {
        if (p < kk) {
          T t = U[(size_t)p * n + j];
#pragma unroll
          for (int q = 0; q < p; ++q) t -= U[(size_t)q * n + k0 + p] * u[q];
          u[p] = t * pinv[f * kCholK + p];
          U[(size_t)p * n + j] = u[p];
        }
      }
    }
    __syncthreads();
    // own trailing rows: subtract the panel product (column-major sweep, a
    // thread owns column j of every own row) and store the L entries
    const int i0 = first_own(b, NB, k0 + kk);
    for (int j = k0 + kk + threadIdx.x; j < n; j += blockDim.x) {
      T um[kCholK], un[kCholK];
#pragma unroll
      for (int p = 0; p < kCholK; ++p) {
        um[p] = p < kk ? stage[(size_t)p * n + j] : T(0);
        un[p] = p < kk ? stage[(size_t)(kCholK + p) * n + j] : T(0);
      }
#pragma unroll 2
      for (int i = i0; i < n; i += NB) {
        T* __restrict__ lmi = own<SM>(A, A.LM, i, n);
        T* __restrict__ lni = own<SM>(A, A.LN, i, n);
        T xm = lmi[j], xn = lni[j];
#pragma unroll
        for (int p = 0; p < kCholK; ++p) {
          if (p < kk) {                 // rows p >= kk of the stage are stale
            xm -= stage[(size_t)p * n + i] * um[p];
            xn -= stage[(size_t)(kCholK + p) * n + i] * un[p];
          }
        }
        lmi[j] = xm;
        lni[j] = xn;
      }
    }
    for (int e = threadIdx.x; e < kCholK * ((n - i0 + NB - 1) / NB); e += blockDim.x) {
      const int p = e % kCholK, i = i0 + (e / kCholK) * NB;
      if (p < kk) {
        own<SM>(A, A.LM, i, n)[k0 + p] = stage[(size_t)p * n + i];
        own<SM>(A, A.LN, i, n)[k0 + p] = stage[(size_t)(kCholK + p) * n + i];
      }
    }
    csync();
  }
  store_panel(((n - 1) / kCholK) * kCholK, n - ((n - 1) / kCholK) * kCholK);
  csync();
  return true;
}

// ------------------------------------------------ row triangular solves
// F holds L below and L^T above the diagonal (row-owned, length n).  X
// (row-owned, row length ld, ncol used) is overwritten by L^{-1} X (FORWARD)
// or L^{-T} X (backward).  A second factor F2 may serve the columns from
// split on (F2 = nullptr: none).
template <bool SM, bool FORWARD, typename T>
__device__ void row_solve(const DenseArgs<T>& A, T* F, T* F2, int split, T* X, int ld, int ncol, T* sv) {
  const int n = A.n, NB = nblocks<SM>(A), b = blockIdx.x;
  auto pivot_row = [&](int m) {
    T* pb = pub_w<SM>(A) + (size_t)(m & 1) * 2 * n;
    T* xm = own<SM>(A, X, m, ld);
    const T d1 = own<SM>(A, F, m, n)[m];
    const T d2 = F2 ? own<SM>(A, F2, m, n)[m] : d1;
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
    const T* pb = pub_r<SM>(A, m % NB) + (size_t)(m & 1) * 2 * n;
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) sv[c] = rd<SM>(pb + c);
    __syncthreads();
    int i0 = FORWARD ? first_own(b, NB, m + 1) : b;
    for (int i = i0; FORWARD ? i < n : i < m; i += NB) {
      // forward: L[i][m] (below diagonal of row i); backward: L^T[i][m] (above)
      const T f1 = own<SM>(A, F, i, n)[m];
      const T f2 = F2 ? own<SM>(A, F2, i, n)[m] : f1;
      T* xi = own<SM>(A, X, i, ld);
      for (int c = threadIdx.x; c < ncol; c += blockDim.x) xi[c] -= (c < split ? f1 : f2) * sv[c];
    }
    __syncthreads();
    int mn = FORWARD ? m + 1 : m - 1;
    if (s + 1 < n && mn % NB == b) pivot_row(mn);
    csync();
  }
}

// Solves in place, for the block's own vectors z_c (c = b mod NB, c in
// [c_lo, c_hi), stored as the own rows c of the row-owned array Z, length
// n), L z = z (UPPER = false: forward substitution) or L^T z = z (UPPER:
// backward), with L lower triangular stored in the rows of F (row t holds
// L[t][0..t] and L^T[t][t..n-1]).  Rows of F are staged kStage at a time
// (any block's rows, loads batched across the rows) with no cluster
// barrier.  Per chunk, a group of g lanes per vector first forms the kStage
// dot products with the entries already solved (independent sums, one pass
// over them), then resolves the chunk's triangle serially in registers:
// the serial chain per row is at most kStage - 1 terms long.
constexpr int kStage = 8;
static_assert(2 * kCholK <= kStage, "the Cholesky panels share the staging buffer");
template <bool SM, bool UPPER, typename T>
__device__ void local_solve(const DenseArgs<T>& A, T* F, T* Z, int c_lo, int c_hi, T* stage) {
  const int n = A.n, NB = nblocks<SM>(A), b = blockIdx.x;
  const int v0 = c_lo <= b ? 0 : (c_lo - b + NB - 1) / NB;        // first own c >= c_lo
  const int nvec = b < c_hi ? max(0, (c_hi - b + NB - 1) / NB - v0) : 0;
  int g = 32;                                     // lanes per vector (power of two)
  while (g > 1 && nvec * g > (int)blockDim.x) g >>= 1;
  const int grp = threadIdx.x / g, gl = threadIdx.x % g;
  const int ngrp = blockDim.x / g;
  const int vmax = ((nvec + ngrp - 1) / ngrp) * ngrp;
  __shared__ T rdiag[kStage];
  for (int k0 = 0; k0 < n; k0 += kStage) {
    const int rows = min(kStage, n - k0);
    const int c0 = UPPER ? n - k0 - rows : k0;     // first row of the chunk
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      T x[kStage];
#pragma unroll
      for (int u = 0; u < kStage; ++u) {
        const int t = c0 + u;
        x[u] = (u < rows && (UPPER ? q >= t : q <= t)) ? rd<SM>(any<SM>(A, F, t, n) + q) : T(0);
      }
#pragma unroll
      for (int u = 0; u < kStage; ++u)
        if (u < rows) {
          stage[(size_t)u * n + q] = x[u];
          if (q == c0 + u) rdiag[u] = T(1) / x[u];   // reciprocal pivots, off the chain
        }
    }
    __syncthreads();
    const int qa = UPPER ? c0 + rows : 0, qb = UPPER ? n : c0;   // entries already solved
    for (int v = grp; v < vmax; v += ngrp) {
      const bool act = v < nvec;
      T* z = act ? own<SM>(A, Z, b + (v0 + v) * NB, n) : nullptr;
      T part[kStage];
#pragma unroll
      for (int u = 0; u < kStage; ++u) part[u] = T(0);
      if (act)
        for (int q = qa + gl; q < qb; q += g) {
          const T zq = z[q];
#pragma unroll
          for (int u = 0; u < kStage; ++u) part[u] += stage[(size_t)u * n + q] * zq;
        }
#pragma unroll
      for (int u = 0; u < kStage; ++u)
        for (int o = g / 2; o > 0; o >>= 1) part[u] += __shfl_xor_sync(0xffffffffu, part[u], o, g);
      if (act) {                                  // the chunk's triangle, every lane alike
        T zc[kStage];
#pragma unroll
        for (int u = 0; u < kStage; ++u) zc[u] = u < rows ? z[c0 + u] : T(0);
#pragma unroll
        for (int s = 0; s < kStage; ++s) {
          const int u = UPPER ? kStage - 1 - s : s;
          if (u < rows) {
            T acc = part[u];
            if (UPPER) {
#pragma unroll
              for (int w = u + 1; w < kStage; ++w)
                if (w < rows) acc += stage[(size_t)u * n + c0 + w] * zc[w];
            } else {
#pragma unroll
              for (int w = 0; w < u; ++w) acc += stage[(size_t)u * n + c0 + w] * zc[w];
            }
            zc[u] = (zc[u] - acc) * rdiag[u];
          }
        }
        if (gl == 0)
#pragma unroll
          for (int u = 0; u < kStage; ++u)
            if (u < rows) z[c0 + u] = zc[u];
      }
      __syncwarp();
    }
    __syncthreads();
  }
}

// C = L_M^{-1} B L_N^{-T} in S1; W = C in S2 for the bidiagonalization.
// X = L_M^{-1} B column by column (block b solves the columns j = b mod NB,
// kept as the own rows j of S2 = X^T), then X's rows gathered into S1, then
// each row of C solves L_N c^T = x^T: two local solves, two barriers.
template <bool SM, typename T>
__device__ void form_C(const DenseArgs<T>& A, T* sv) {
  const int n = A.n, NB = nblocks<SM>(A), b = blockIdx.x;
  // staging rows: the block's own publication buffer under the shared policy
  // (no block publishes during the local solves), its dynamic shared memory
  // after the 3n scratch otherwise (the global publication buffer is common)
  T* stage = SM ? A.pub : sv + 3 * n;
  for (int j = b; j < n; j += NB) {                 // own rows j of S2: column j of B
    T* x = own<SM>(A, A.S2, j, n);
    for (int t = threadIdx.x; t < n; t += blockDim.x) x[t] = T(A.B[(size_t)t * n + j]);
  }
  __syncthreads();
  local_solve<SM, false>(A, A.LM, A.S2, 0, n, stage);   // S2 rows: columns of X
  csync();
  batched_copy<T>(                                  // X rows into S1
      ((n - b + NB - 1) / NB) * n,
      [&](int e) { return rd<SM>(any<SM>(A, A.S2, e - (e / n) * n, n) + b + (e / n) * NB); },
      [&](int e, T v) { own<SM>(A, A.S1, b + (e / n) * NB, n)[e - (e / n) * n] = v; });
  __syncthreads();
  local_solve<SM, false>(A, A.LN, A.S1, 0, n, stage);   // S1 rows: rows of C
  csync();  // every block done reading S2 before it becomes W
  for (int i = b; i < n; i += NB) {
    T* w = own<SM>(A, A.S2, i, n);
    const T* c = own<SM>(A, A.S1, i, n);
    for (int j = threadIdx.x; j < n; j += blockDim.x) w[j] = c[j];
  }
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
// I - taup[k] p_k p_k^T (p_k[k+1] = 1, support k+1..n-1) kept in row k of S3
// (the left ones are not needed).  Left reflector of column k: each block
// sums x_i W[i][j] and x_i^2 over its own rows i > k into partials; after the
// barrier every block forms s_j = tau (W[k][j] + scale * sum_b partial_b[j])
// and updates its rows.  Right reflector of row k: built and published by
// the owner of row k, applied by every block to its own rows.
// Partials and published row of step k go to the buffers of parity k & 1:
// with one cluster barrier per step a block may start writing step k + 1
// while another still reads step k.
template <bool SM, typename T>
__device__ void bidiag_partials(const DenseArgs<T>& A, int k) {
  const int n = A.n, NB = nblocks<SM>(A), b = blockIdx.x;
  T* part = part_w<SM>(A) + (k & 1) * (n + 1);
  const int i0 = first_own(b, NB, k + 1);
  for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) {
    T t = 0;
    for (int i = i0; i < n; i += NB) {
      const T* wi = own<SM>(A, A.S2, i, n);
      t += wi[k] * wi[j];
    }
    part[j] = t;
  }
  if (threadIdx.x == 0) {
    T s2 = 0;
    for (int i = i0; i < n; i += NB) {
      const T x = own<SM>(A, A.S2, i, n)[k];
      s2 += x * x;
    }
    part[n] = s2;
  }
  if (k % NB == b) {                       // publish row k for the other blocks
    T* rowk = pub_w<SM>(A) + (k & 1) * n;
    const T* wk = own<SM>(A, A.S2, k, n);
    for (int j = k + threadIdx.x; j < n; j += blockDim.x) rowk[j] = wk[j];
  }
}

template <bool SM, typename T>
__device__ void bidiagonalize(const DenseArgs<T>& A, T* sv, T* red) {
  const int n = A.n, NB = nblocks<SM>(A), b = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T* s_vec = sv;          // n: s_j of the left reflector
  T* p_vec = sv + n;      // n: row k after the left reflector, then the right reflector
  T* rowk = sv + 2 * n;   // n: row k as published at the end of the previous step
  __shared__ T sc[2];
  bidiag_partials<SM>(A, 0);
  csync();
  for (int k = 0; k < n; ++k) {
    const int po = (k & 1) * (n + 1);            // this step's partial buffer
    const T* pk_pub = pub_r<SM>(A, k % NB) + (k & 1) * n;
    // left reflector of column k: thread 0 forms tau while every thread
    // fetches its entries of row k and of the column sums (s_vec holds the
    // sums until tau is known)
    if (threadIdx.x == 0) {
      T beta, tau, scale;
      householder(rd<SM>(pk_pub + k), part_sum<SM>(A, po + n), beta, tau, scale);
      sc[0] = tau; sc[1] = scale;
      if (b == 0) A.d[k] = beta;
    }
    for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) {
      rowk[j] = rd<SM>(pk_pub + j);
      s_vec[j] = part_sum<SM>(A, po + j);
    }
    __syncthreads();
    const T tau = sc[0], scale = sc[1];
    for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) s_vec[j] = tau * (rowk[j] + scale * s_vec[j]);
    __syncthreads();
    if (tau != T(0)) {
      for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x) {
        const T sj = s_vec[j];
#pragma unroll 4
        for (int i = first_own(b, NB, k); i < n; i += NB) {
          T* __restrict__ wi = own<SM>(A, A.S2, i, n);
          const T vi = (i == k) ? T(1) : wi[k] * scale;
          wi[j] -= vi * sj;
        }
      }
    }
    if (k == n - 1) break;
    // right reflector of row k, formed by every block from the published row
    // and s (the owner's updated row k is exactly rowk - s)
    for (int j = k + 1 + threadIdx.x; j < n; j += blockDim.x)
      p_vec[j] = tau != T(0) ? rowk[j] - s_vec[j] : rowk[j];
    __syncthreads();
    T s2r = 0;
    for (int j = k + 2 + threadIdx.x; j < n; j += blockDim.x) s2r += p_vec[j] * p_vec[j];
    s2r = block_sum(s2r, red);
    T betar, taup, scp;
    householder(p_vec[k + 1], s2r, betar, taup, scp);
    __syncthreads();
    const bool owner = k % NB == b;
    T* pk = owner ? own<SM>(A, A.S3, k, n) : nullptr;   // the owner keeps the reflector
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      if (j > k) {
        const T pj = (j == k + 1) ? T(1) : p_vec[j] * scp;
        p_vec[j] = pj;
        if (owner) pk[j] = pj;
      } else if (owner) {
        pk[j] = T(0);
      }
    }
    if (owner && threadIdx.x == 0) {
      A.e[k] = betar;
      A.taup[k] = taup;
    }
    __syncthreads();
    if (taup != T(0)) {
      for (int i = first_own(b, NB, k + 1) + NB * w; i < n; i += NB * kWarps) {   // one warp per row
        T* wi = own<SM>(A, A.S2, i, n);
        T sdot = 0;
        for (int j = k + 1 + lane; j < n; j += 32) sdot += wi[j] * p_vec[j];
        sdot = warp_sum(sdot) * taup;
        for (int j = k + 1 + lane; j < n; j += 32) wi[j] -= sdot * p_vec[j];
      }
    }
    __syncthreads();
    bidiag_partials<SM>(A, k + 1);
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

// Number of eigenvalues of the tridiagonal below x (Sturm count).  In FP64
// the sign changes of the leading principal minors p_k(x) are counted with
// the three-term recurrence p_k = -x p_{k-1} - off(k)^2 p_{k-2} (no FP64
// division, narrow on GB300), rescaled by exact powers of two to stay in
// range; a ratio p_k / p_{k-1} below pivmin in magnitude is replaced by
// -pivmin, as in the LDL^T ratio form used in FP32.
template <typename T> struct GkRange;
template <> struct GkRange<double> { static constexpr double big = 0x1p+256, small = 0x1p-256; };
template <> struct GkRange<float> { static constexpr float big = 0x1p+48f, small = 0x1p-48f; };

template <typename T>
__device__ int gk_count(const T* d, const T* e, int n, T x, T pivmin) {
  if constexpr (sizeof(T) == 4) {
    // FP32: the LDL^T ratios q_k = -x - off(k)^2 / q_{k-1}
    int cnt = 0;
    T q = -x;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < T(0);
    for (int k = 1; k < 2 * n; ++k) {
      T o = gk_off(d, e, k);
      q = -x - __fdividef(o * o, q);   // fast division: a 2-ulp error is a tiny perturbation of off(k)^2
      if (fabs(q) < pivmin) q = -pivmin;
      cnt += q < T(0);
    }
    return cnt;
  }
  T pprev = T(1), p = -x;
  if (fabs(p) < pivmin) p = -pivmin;
  int cnt = p < T(0);
  for (int k = 1; k < 2 * n; ++k) {
    const T o = gk_off(d, e, k);
    T pn = -x * p - (o * o) * pprev;
    if (fabs(pn) < pivmin * fabs(p)) pn = -pivmin * p;
    cnt += (pn < T(0)) != (p < T(0));
    pprev = p;
    p = pn;
    if (fabs(p) > GkRange<T>::big) {
      p *= GkRange<T>::small;
      pprev *= GkRange<T>::small;
    } else if (fabs(p) < GkRange<T>::small && fabs(pprev) < GkRange<T>::small) {
      p *= GkRange<T>::big;
      pprev *= GkRange<T>::big;
    }
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

// One lane: LU with partial pivoting of the tridiagonal T - sigma I (size m);
// the warp then replaces the pivots by their reciprocals for the solves.
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
template <bool SM, typename T>
__device__ void bidiag_triplets(const DenseArgs<T>& A, T* sv) {
  const int n = A.n, r = A.r, m = 2 * n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // consecutive values on different blocks: one warp per SM while r <= NB,
  // so the per-value work does not share an SM's FP64 units
  const int gw = w * gridDim.x + blockIdx.x, GW = gridDim.x * kWarps;
  // the bidiagonal and the reflector scalars, staged in shared memory
  T* d = sv;
  T* e = sv + n;
  T* taup = sv + 2 * n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    d[k] = __ldcg(A.d + k);
    e[k] = __ldcg(A.e + k);
    taup[k] = __ldcg(A.taup + k);
  }
  __syncthreads();
  const T gmax = gk_bound(d, e, n);
  const T pivmin = T(Eps<T>::tiny) * fmax(T(1), gmax * gmax);
  for (int a = gw; a < r; a += GW) {
    T s = gk_sigma(d, e, n, a, gmax, pivmin);
    if (lane == 0) A.sig[a] = s;
  }
  csync();
  const T ortol = T(sqrt(Eps<T>::v)) * gmax;
  const T pert = T(Eps<T>::v) * gmax;
  int c = 0;
  for (int a0 = 0; a0 < r; ++a0) {
    if (a0 > 0 && __ldcg(A.sig + a0) - __ldcg(A.sig + a0 - 1) <= ortol) continue;
    int a1 = a0 + 1;
    while (a1 < r && __ldcg(A.sig + a1) - __ldcg(A.sig + a1 - 1) <= ortol) ++a1;
    if (c++ % GW != gw) continue;
    // the factors and the iterate of the serial solves in shared memory (the
    // block's rows of S2, free in this phase) when they fit, else in the
    // global scratch; the converged iterate is kept in the global scratch for
    // the later members of the cluster
    const bool wsm = SM && (w + 1) * 6 * m <= A.RP * n;
    for (int a = a0; a < a1; ++a) {
      T* base = wsm ? A.S2 + (size_t)w * 6 * m : A.z + (size_t)a * 6 * m;
      T *dd = base, *du = base + m, *du2 = base + 2 * m, *dl = base + 3 * m, *pv = base + 4 * m;
      T* zv = base + 5 * m;
      if (lane == 0) gk_factor(d, e, m, __ldcg(A.sig + a), pert, dd, du, du2, dl, pv);
      __syncwarp();
      for (int k = lane; k < m; k += 32) {
        dd[k] = T(1) / dd[k];                       // reciprocal pivots
        zv[k] = T(1) + T(0.5) * T((unsigned)(k * 2654435761u) % 1000u) / T(1000) + T(a);
      }
      __syncwarp();
      // an isolated value converges in two steps from an accurate shift;
      // members of a cluster take four, with orthogonalisation
      const int iters = (a1 - a0 > 1) ? 4 : 2;
      for (int it = 0; it < iters; ++it) {
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
      if (wsm && a + 1 < a1)
        for (int k = lane; k < m; k += 32) A.z[(size_t)a * 6 * m + 5 * m + k] = zv[k];
      T nv = 0;                                   // right vector: even positions
      for (int i = lane; i < n; i += 32) nv += zv[2 * i] * zv[2 * i];
      nv = warp_sum(nv);
      T inv = nv > T(0) ? T(1) / sqrt(nv) : T(0);
      for (int i = lane; i < n; i += 32) A.vb[(size_t)a * n + i] = zv[2 * i] * inv;
      __syncwarp();
    }
  }
  csync();
  constexpr int kReg = 8;                         // vector / reflector entries per lane
  for (int a = gw; a < r; a += GW) {              // v~ = P_B v_D, last reflector first
    T* y = A.vb + (size_t)a * n;
    if (n <= 32 * kReg) {
      // y and the reflectors in registers at the absolute positions
      // lane + 32 q; reflector k - 1 is fetched while reflector k is applied
      T yr[kReg], pr[kReg], nx[kReg];
      auto fetch = [&](int k, T (&dst)[kReg]) {
        const T* p = any<SM>(A, A.S3, k, n);
#pragma unroll
        for (int q = 0; q < kReg; ++q) {
          const int j = lane + 32 * q;
          dst[q] = (j > k && j < n) ? rd<SM>(p + j) : T(0);
        }
      };
#pragma unroll
      for (int q = 0; q < kReg; ++q) yr[q] = lane + 32 * q < n ? y[lane + 32 * q] : T(0);
      if (n >= 2) fetch(n - 2, pr);
      for (int k = n - 2; k >= 0; --k) {
        if (k > 0) fetch(k - 1, nx);
        const T tau = taup[k];
        if (tau != T(0)) {
          T s = 0;
#pragma unroll
          for (int q = 0; q < kReg; ++q) s += pr[q] * yr[q];
          s = warp_sum(s) * tau;
#pragma unroll
          for (int q = 0; q < kReg; ++q) yr[q] -= s * pr[q];
        }
#pragma unroll
        for (int q = 0; q < kReg; ++q) pr[q] = nx[q];
      }
#pragma unroll
      for (int q = 0; q < kReg; ++q)
        if (lane + 32 * q < n) y[lane + 32 * q] = yr[q];
    } else {
      for (int k = n - 2; k >= 0; --k) {
        const T tau = taup[k];
        if (tau == T(0)) continue;
        const T* p = any<SM>(A, A.S3, k, n);
        T s = 0;
        for (int j = k + 1 + lane; j < n; j += 32) s += rd<SM>(p + j) * y[j];
        s = warp_sum(s) * tau;
        for (int j = k + 1 + lane; j < n; j += 32) y[j] -= s * rd<SM>(p + j);
        __syncwarp();
      }
    }
  }
  csync();
}

// ------------------------------------------------------------- triplets
// Right-hand sides [v~_a | C v~_a / ||C v~_a||] in the own rows of R; both
// back substitutions (L_N^T for v, L_M^T for u) in one sweep; sign: largest
// |v_i| positive (lowest index on ties).  For a zero singular value (below
// n * eps * bound) u = 1 / sqrt(1^T M 1) and v normalised in the 2-norm is the
// right null vector w of B.  Row-sweep form (a cluster barrier per row), for
// the small sizes where the 2r vectors do not fit the rows of S2.
template <bool SM, typename T>
__device__ void triplets_rows(const DenseArgs<T>& A, T* sv, T* red) {
  const int n = A.n, r = A.r, r2 = 2 * r, NB = nblocks<SM>(A), b = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T* part = part_w<SM>(A);
  const T gmax = gk_bound(A.d, A.e, n);
  const T null_tol = T(n * Eps<T>::v) * gmax;
  for (int i = b; i < n; i += NB) {
    T* ri = own<SM>(A, A.R, i, r2);
    for (int c = threadIdx.x; c < r; c += blockDim.x) ri[c] = __ldcg(A.vb + (size_t)c * n + i);
  }
  {
    // C v~_a for the own rows: one warp per (row, value) pair
    const int npair = ((n - b + NB - 1) / NB) * r;
    for (int q = w; q < npair; q += kWarps) {
      const int i = b + (q / r) * NB, a = q % r;
      const T* ci = own<SM>(A, A.S1, i, n);
      const T* va = A.vb + (size_t)a * n;
      T acc = 0;
      for (int j = lane; j < n; j += 32) acc += ci[j] * __ldcg(va + j);
      acc = warp_sum(acc);
      if (lane == 0) own<SM>(A, A.R, i, r2)[r + a] = acc;
    }
  }
  __syncthreads();
  for (int a = threadIdx.x; a < r; a += blockDim.x) {
    T s = 0;
    for (int i = b; i < n; i += NB) {
      const T x = own<SM>(A, A.R, i, r2)[r + a];
      s += x * x;
    }
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
    T s = part_sum<SM>(A, a);
    sv[a] = s > T(0) ? T(1) / sqrt(s) : T(0);
  }
  __syncthreads();
  for (int i = b; i < n; i += NB) {
    T* ri = own<SM>(A, A.R, i, r2);
    for (int a = threadIdx.x; a < r; a += blockDim.x) ri[r + a] *= sv[a];
  }
  __syncthreads();
  row_solve<SM, false>(A, A.LN, A.LM, r, A.R, r2, r2, sv);
  // sign candidates per value and the norm of v_0
  for (int a = threadIdx.x; a < r; a += blockDim.x) {
    T best = -1, bi = T(n), s0 = 0;
    for (int i = b; i < n; i += NB) {
      T v = own<SM>(A, A.R, i, r2)[a];
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
    T vals[kMaxNB], idx[kMaxNB];
#pragma unroll
    for (int q = 0; q < kMaxNB; ++q) {
      vals[q] = q < NB ? rd<SM>(part_r<SM>(A, q) + n + 2 * a) : T(-2);
      idx[q] = q < NB ? rd<SM>(part_r<SM>(A, q) + n + 2 * a + 1) : T(n);
    }
    T best = -1, bi = T(n);
#pragma unroll
    for (int q = 0; q < kMaxNB; ++q)
      if (vals[q] > best || (vals[q] == best && idx[q] < bi)) { best = vals[q]; bi = idx[q]; }
    const T vv = rd<SM>(any<SM>(A, A.R, (int)bi, r2) + a);
    sgn[a] = vv < T(0) ? T(-1) : T(1);
  }
  if (threadIdx.x == 0) {
    const T s1 = part_sum<SM>(A, n + r2 + 1);
    const T s0 = part_sum<SM>(A, n + r2);
    uconst[0] = T(1) / sqrt(s1);
    uconst[1] = s0 > T(0) ? T(1) / sqrt(s0) : T(0);
  }
  __syncthreads();
  const bool null0 = __ldcg(A.sig) <= null_tol;
  for (int i = b; i < n; i += NB) {
    const T* ri = own<SM>(A, A.R, i, r2);
    for (int a = threadIdx.x; a < r; a += blockDim.x) {
      const bool is_null = __ldcg(A.sig + a) <= null_tol;
      A.V[(size_t)i * r + a] = double(sgn[a] * ri[a]);
      A.U[(size_t)i * r + a] = double(is_null ? uconst[0] : sgn[a] * ri[r + a]);
    }
    if (threadIdx.x == 0) A.unull[i] = null0 ? sgn[0] * ri[0] * uconst[1] : T(0);
  }
  if (b == 0)
    for (int a = threadIdx.x; a < r; a += blockDim.x) A.sigma[a] = double(__ldcg(A.sig + a));
  csync();
}

// The same triplets with the 2r back substitutions as local solves, with no
// cluster barrier: the v~_a on the first half of the blocks (L_N^T), the u~_a
// on the second half (L_M^T); the owner of v_a also takes its sign and
// publishes it for the owner of u_a.
template <bool SM, typename T>
__device__ void triplets_local(const DenseArgs<T>& A, T* sv, T* red) {
  const int n = A.n, r = A.r, r2 = 2 * r, NB = nblocks<SM>(A), b = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T* part = part_w<SM>(A);
  const T gmax = gk_bound(A.d, A.e, n);
  const T null_tol = T(n * Eps<T>::v) * gmax;
  {
    // C v~_a for the own rows: one warp per (row, value) pair
    const int npair = ((n - b + NB - 1) / NB) * r;
    for (int q = w; q < npair; q += kWarps) {
      const int i = b + (q / r) * NB, a = q % r;
      const T* ci = own<SM>(A, A.S1, i, n);
      const T* va = A.vb + (size_t)a * n;
      T acc = 0;
      for (int j = lane; j < n; j += 32) acc += ci[j] * __ldcg(va + j);
      acc = warp_sum(acc);
      if (lane == 0) own<SM>(A, A.R, i, r2)[r + a] = acc;
    }
  }
  __syncthreads();
  for (int a = threadIdx.x; a < r; a += blockDim.x) {
    T s = 0;
    for (int i = b; i < n; i += NB) {
      const T x = own<SM>(A, A.R, i, r2)[r + a];
      s += x * x;
    }
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
  // v~_a on the first half of the blocks, u~_a on the second, vpb per block:
  // vector a of kind f (0: v, 1: u) is the own row b + slot NB of S2 of block
  // b = f half + a / vpb (slot = a mod vpb), so each block solves with one
  // factor only and both kinds advance together
  const int half = NB / 2, vpb = (r + half - 1) / half;
  const int f = b < half ? 0 : 1, a_lo = (b - f * half) * vpb;
  const int nv = b < 2 * half ? max(0, min(vpb, r - a_lo)) : 0;
  for (int v = 0; v < nv; ++v) {
    const int a = a_lo + v;
    T* z = own<SM>(A, A.S2, b + v * NB, n);
    if (f == 0) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) z[i] = __ldcg(A.vb + (size_t)a * n + i);
    } else {
      const T s = part_sum<SM>(A, a);
      const T sc = s > T(0) ? T(1) / sqrt(s) : T(0);
      batched_copy<T>(
          n, [&](int i) { return rd<SM>(any<SM>(A, A.R, i, r2) + r + a); }, [&](int i, T x) { z[i] = x * sc; });
    }
  }
  __syncthreads();
  T* stage = SM ? A.pub : sv + 3 * n;
  if (nv > 0) {
    if (f == 0)
      local_solve<SM, true>(A, A.LN, A.S2, b, b + nv * NB, stage);
    else
      local_solve<SM, true>(A, A.LM, A.S2, b, b + nv * NB, stage);
  }
  // signs of the own v_a (largest |v_i| positive, lowest index on ties) and
  // ||v_0||^2, published in the partial slots n + 2a and n + 2r
  __shared__ int redi[kWarps];
  for (int v = 0; v < (f == 0 ? nv : 0); ++v) {
    const int a = a_lo + v;
    const T* z = own<SM>(A, A.S2, b + v * NB, n);
    T best = T(-1);
    int bi = n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const T x = fabs(z[i]);
      if (x > best) { best = x; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    __syncthreads();
    if (lane == 0) { red[w] = best; redi[w] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int k = 1; k < kWarps; ++k)
        if (red[k] > best || (red[k] == best && redi[k] < bi)) { best = red[k]; bi = redi[k]; }
      part[n + 2 * a] = (bi < n && z[bi] < T(0)) ? T(-1) : T(1);
    }
    __syncthreads();
    if (a == 0) {
      T s0 = 0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) s0 += z[i] * z[i];
      s0 = block_sum(s0, red);
      if (threadIdx.x == 0) part[n + r2] = s0;
    }
  }
  csync();
  const T uconst = T(1) / sqrt(part_sum<SM>(A, n + r2 + 1));   // 1 / sqrt(1^T M 1)
  const bool null0 = __ldcg(A.sig) <= null_tol;
  for (int v = 0; v < nv; ++v) {
    const int a = a_lo + v;
    const T* z = own<SM>(A, A.S2, b + v * NB, n);
    const T sg = rd<SM>(part_r<SM>(A, a / vpb) + n + 2 * a);   // from the owner of v_a
    if (f == 0) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) A.V[(size_t)i * r + a] = double(sg * z[i]);
      if (a == 0) {
        const T s0 = part[n + r2];
        const T inv0 = s0 > T(0) ? T(1) / sqrt(s0) : T(0);
        for (int i = threadIdx.x; i < n; i += blockDim.x) A.unull[i] = null0 ? sg * z[i] * inv0 : T(0);
      }
    } else {
      const bool is_null = __ldcg(A.sig + a) <= null_tol;
      for (int i = threadIdx.x; i < n; i += blockDim.x)
        A.U[(size_t)i * r + a] = double(is_null ? uconst : sg * z[i]);
    }
  }
  if (b == 0)
    for (int a = threadIdx.x; a < r; a += blockDim.x) A.sigma[a] = double(__ldcg(A.sig + a));
  csync();
}

template <bool SM, typename T>
__device__ void triplets(const DenseArgs<T>& A, T* sv, T* red) {
  const int NB = nblocks<SM>(A), half = NB / 2;
  // the vpb vectors of a block are its own rows b + v NB of S2
  const int vpb = half > 0 ? (A.r + half - 1) / half : A.n + 1;
  const bool fits = half > 0 && (SM ? vpb <= A.RP : NB - 1 + (vpb - 1) * NB < A.n);
  if (fits)
    triplets_local<SM>(A, sv, red);
  else
    triplets_rows<SM>(A, sv, red);
}

// ------------------------------------------------------------ pseudo-inverse
// X = (B + e e^T)^{-1} by Gauss-Jordan on [B + e e^T | I] with partial
// pivoting and no row exchanges: the row chosen for column k keeps its place
// and records k; at the end row i holds row pcol[i] of X.  The tableau G
// (2n per row) is the row-owned array S2.
template <bool SM, typename T>
__device__ void gj_candidate(const DenseArgs<T>& A, int k) {
  const int n = A.n, n2 = 2 * n, NB = nblocks<SM>(A), b = blockIdx.x;
  __shared__ T cv[kWarps];
  __shared__ int ci[kWarps];
  T best = -1;
  int bi = n;
  for (int i = b + NB * threadIdx.x; i < n; i += NB * blockDim.x) {
    if (*own_pcol<SM>(A, i) >= 0) continue;
    T v = fabs(own<SM>(A, A.S2, i, n2)[k]);
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
    T* part = part_w<SM>(A);
    part[n + 2 * kMaxR + 2] = best;
    part[n + 2 * kMaxR + 3] = T(bi);
  }
}

// sv: 2n scratch; A.unull: global n-vector for X e (any values on entry).
template <bool SM, typename T>
__device__ void pseudo_inverse(const DenseArgs<T>& A, T* sv, T* red) {
  const int n = A.n, n2 = 2 * n, NB = nblocks<SM>(A), b = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const T e = T(1) / sqrt(T(n));
  const T ee = T(1) / T(n);                      // every entry of e e^T
  T* G = A.S2;
  for (int i = b; i < n; i += NB) {
    T* gi = own<SM>(A, G, i, n2);
    for (int j = threadIdx.x; j < n2; j += blockDim.x)
      gi[j] = j < n ? T(A.B[(size_t)i * n + j]) + ee : (j - n == i ? T(1) : T(0));
    if (threadIdx.x == 0) *own_pcol<SM>(A, i) = -1;
  }
  __syncthreads();
  gj_candidate<SM>(A, 0);
  csync();
  __shared__ int sp;
  T* prow = sv;
  for (int k = 0; k < n; ++k) {
    if (w == 0) {                               // best candidate over the blocks
      T best = -1;
      int bi = n;
      if (lane < NB) {
        const T* pq = part_r<SM>(A, lane);
        best = rd<SM>(pq + n + 2 * kMaxR + 2);
        bi = (int)rd<SM>(pq + n + 2 * kMaxR + 3);
      }
      for (int o = 16; o > 0; o >>= 1) {
        T ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) sp = bi;
    }
    __syncthreads();
    const int p = sp;
    if (p % NB == b) {                          // normalise and publish the pivot row
      T* gp = own<SM>(A, G, p, n2);
      T* pw = pub_w<SM>(A);
      const T inv = T(1) / gp[k];
      __syncthreads();
      for (int j = k + threadIdx.x; j < n2; j += blockDim.x) {
        T v = gp[j] * inv;
        gp[j] = v;
        pw[j] = v;
      }
      if (threadIdx.x == 0) *own_pcol<SM>(A, p) = k;
    }
    csync();
    const T* pr = pub_r<SM>(A, p % NB);
    for (int j = k + threadIdx.x; j < n2; j += blockDim.x) prow[j] = rd<SM>(pr + j);
    __syncthreads();
    for (int i = b + NB * w; i < n; i += NB * kWarps) {   // one warp per own row
      if (i == p) continue;
      T* gi = own<SM>(A, G, i, n2);
      const T f = gi[k];
      __syncwarp();
      if (f != T(0))
        for (int j = k + lane; j < n2; j += 32) gi[j] -= f * prow[j];
      __syncwarp();
    }
    __syncthreads();
    if (k + 1 < n) gj_candidate<SM>(A, k + 1);
    csync();
  }
  // s = X e (s_c = e * row sum of X's row c), w = s / ||s||
  T* part = part_w<SM>(A);
  T* xs = A.unull;
  T ps2 = 0;
  for (int i = b; i < n; i += NB) {
    const int c = *own_pcol<SM>(A, i);
    const T* gi = own<SM>(A, G, i, n2);
    T t = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) t += gi[n + j];
    t = block_sum(t, red) * e;
    if (threadIdx.x == 0) {
      xs[c] = t;
      ps2 += t * t;
    }
  }
  if (threadIdx.x == 0) part[n] = ps2;
  __syncthreads();
  csync();
  const T nrm = sqrt(part_sum<SM>(A, n));
  // partial w^T X over the own rows
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    T t = 0;
    for (int i = b; i < n; i += NB) {
      const int c = *own_pcol<SM>(A, i);
      t += (xs[c] / nrm) * own<SM>(A, G, i, n2)[n + j];
    }
    part[j] = t;
  }
  csync();
  T* wtx = sv;                                    // w^T X
  for (int j = threadIdx.x; j < n; j += blockDim.x) wtx[j] = part_sum<SM>(A, j);
  __syncthreads();
  // B^+ = X - w (w^T X) - (X e) e^T + w (w^T X e) e^T, with w^T X e = ||s||
  for (int i = b; i < n; i += NB) {
    const int c = *own_pcol<SM>(A, i);
    const T* gi = own<SM>(A, G, i, n2);
    const T sc = xs[c], wc = sc / nrm;
    for (int j = threadIdx.x; j < n; j += blockDim.x)
      A.Bpinv[(size_t)c * n + j] = double(gi[n + j] - wc * wtx[j] - sc * e + wc * nrm * e);
  }
}

// Shared-policy layout of one block's dynamic shared memory, in elements of
// T after the 3n scratch vector: pub, part, LM, LN, S1, S2, S3, R, then pcol.
__host__ __device__ inline size_t smem_elems(int n, int r, int RP) {
  return (size_t)3 * n + (size_t)8 * n + 64 + part_stride(n) + (size_t)5 * RP * n + (size_t)RP * 2 * r;
}

template <typename T, bool SM>
__global__ void __launch_bounds__(kDenseThreads, 1) coarsest_kernel(DenseArgs<T> A) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char dyn[];
  T* sv = reinterpret_cast<T*>(dyn);
  __shared__ T red[kWarps];
  const int n = A.n;
  A.NB = gridDim.x;
  if constexpr (SM) {
    T* p = sv + 3 * n;
    A.pub = p;  p += 8 * n + 64;
    A.part = p; p += part_stride(n);
    A.LM = p;   p += (size_t)A.RP * n;
    A.LN = p;   p += (size_t)A.RP * n;
    A.S1 = p;   p += (size_t)A.RP * n;
    A.S2 = p;   p += (size_t)A.RP * n;
    A.S3 = p;   p += (size_t)A.RP * n;
    A.R = p;    p += (size_t)A.RP * 2 * A.r;
    A.pcol = reinterpret_cast<int*>(p);
  }
  const bool b0 = blockIdx.x == 0 && threadIdx.x == 0;
  if (b0) A.ctl->tp[0] = gtimer();
  if (!cholesky_rows<SM>(A, sv)) return;
  if (b0) A.ctl->tp[1] = gtimer();
  form_C<SM>(A, sv);
  if (b0) A.ctl->tp[2] = gtimer();
  bidiagonalize<SM>(A, sv, red);
  if (b0) A.ctl->tp[3] = gtimer();
  bidiag_triplets<SM>(A, sv);
  if (b0) A.ctl->tp[4] = gtimer();
  triplets<SM>(A, sv, red);
  if (b0) A.ctl->tp[5] = gtimer();
  csync();   // no block leaves while another may still read its shared memory
}

// Shared-policy layout of the pseudo-inverse kernel, in elements of T: 2n
// scratch, pub (2n + 64), part, the tableau rows (RP x 2n), then pcol.
__host__ __device__ inline size_t pinv_smem_elems(int n, int RP) {
  return (size_t)2 * n + (size_t)2 * n + 64 + part_stride(n) + (size_t)RP * 2 * n;
}

template <typename T, bool SM>
__global__ void __launch_bounds__(kDenseThreads, 1) pinv_kernel(DenseArgs<T> A) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char dyn[];
  T* sv = reinterpret_cast<T*>(dyn);
  __shared__ T red[kWarps];
  const int n = A.n;
  A.NB = gridDim.x;
  if constexpr (SM) {
    T* p = sv + 2 * n;
    A.pub = p;  p += 2 * n + 64;
    A.part = p; p += part_stride(n);
    A.S2 = p;   p += (size_t)A.RP * 2 * n;
    A.pcol = reinterpret_cast<int*>(p);
  }
  const bool b0 = blockIdx.x == 0 && threadIdx.x == 0;
  if (b0) A.ctl->tp[0] = gtimer();
  pseudo_inverse<SM>(A, sv, red);
  if (b0) A.ctl->tp[1] = gtimer();
  csync();
}

__global__ void csr_to_dense_kernel(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                    const double* __restrict__ va, double* __restrict__ D) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x;
  for (int p = rp[i] + threadIdx.x; p < rp[i + 1]; p += blockDim.x) D[(size_t)i * n + ci[p]] = va[p];
}

bamg_status csr_to_dense(int n, const int32_t* rp, const int32_t* ci, const double* va, double* D,
                         cudaStream_t s) {
  BAMG_CUDA(cudaMemsetAsync(D, 0, sizeof(double) * (size_t)n * n, s));
  return launch(csr_to_dense_kernel, dim3(n), dim3(64), 0, s, n, rp, ci, va, D);
}

static int max_cluster(const void* kern, cudaLaunchConfig_t cfg, int want) {
  int maxc = 0;
  cfg.gridDim = dim3(want);
  cfg.numAttrs = 0;
  if (cudaOccupancyMaxPotentialClusterSize(&maxc, kern, &cfg) != cudaSuccess) maxc = 0;
  cudaGetLastError();
  return maxc < want ? maxc : want;
}

// Cluster launch of kern with csize blocks and smem bytes on stream s.
template <typename T>
static bamg_status cluster_launch(void (*kern)(DenseArgs<T>), int csize, size_t smem, cudaStream_t s,
                                  const DenseArgs<T>& a) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.blockDim = dim3(kDenseThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.gridDim = dim3(csize);
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  BAMG_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
  return BAMG_OK;
}

// Storage policy and cluster size for a kernel: shared rows with 16 blocks
// when smem_sm bytes fit and such a cluster can be placed, else global rows
// with the largest placeable cluster and smem_gl bytes.
template <typename T>
static bamg_status choose_policy(void (*ksm)(DenseArgs<T>), void (*kgl)(DenseArgs<T>), size_t smem_sm,
                                 size_t smem_gl, std::atomic<uint64_t>& sm_attr, std::atomic<uint64_t>& gl_attr,
                                 bool* use_sm, int* csize) {
  int max_sm = 0, max_gl = 0;
  BAMG_TRY(allow_max_smem((const void*)ksm, sm_attr, &max_sm));
  BAMG_TRY(allow_max_smem((const void*)kgl, gl_attr, &max_gl));
  BAMG_CUDA(cudaFuncSetAttribute(ksm, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  BAMG_CUDA(cudaFuncSetAttribute(kgl, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kDenseThreads);
  *use_sm = false;
  if (smem_sm <= (size_t)max_sm) {
    cfg.dynamicSmemBytes = smem_sm;
    *use_sm = max_cluster((const void*)ksm, cfg, kMaxNB) == kMaxNB;
  }
  if (*use_sm) {
    *csize = kMaxNB;
    return BAMG_OK;
  }
  if (smem_gl > (size_t)max_gl) {
    set_error("dense coarsest kernel needs %zu bytes of shared memory", smem_gl);
    return BAMG_ERR_UNSUPPORTED;
  }
  cfg.dynamicSmemBytes = smem_gl;
  *csize = max_cluster((const void*)kgl, cfg, kMaxNB);
  if (*csize < 1) *csize = 1;
  return BAMG_OK;
}

template <typename T> struct DenseAttrs {
  static std::atomic<uint64_t> tsm, tgl, psm, pgl;
};
template <typename T> std::atomic<uint64_t> DenseAttrs<T>::tsm{0};
template <typename T> std::atomic<uint64_t> DenseAttrs<T>::tgl{0};
template <typename T> std::atomic<uint64_t> DenseAttrs<T>::psm{0};
template <typename T> std::atomic<uint64_t> DenseAttrs<T>::pgl{0};

// A side stream per host thread and device for the pseudo-inverse cluster.
static bamg_status side_stream(cudaStream_t* out) {
  thread_local cudaStream_t streams[64] = {};
  int dev = 0;
  BAMG_CUDA(cudaGetDevice(&dev));
  cudaStream_t& st = streams[dev & 63];
  if (!st) BAMG_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  *out = st;
  return BAMG_OK;
}

template <typename T>
static bamg_status coarsest_t(int n, int r, const double* B, const double* M, const double* N, double* sigma,
                              double* U, double* V, double* Bpinv, cudaStream_t s, HostWork during,
                              int* err_out) {
  // ---- triplets: Cholesky, C, bidiagonalization, SVD, back-transform
  DenseArgs<T> a = {};
  a.n = n; a.r = r; a.B = B; a.M = M; a.N = N;
  a.sigma = sigma; a.U = U; a.V = V; a.Bpinv = nullptr;
  auto ksm = coarsest_kernel<T, true>;
  auto kgl = coarsest_kernel<T, false>;
  const int rp16 = (n + kMaxNB - 1) / kMaxNB;
  const size_t smem16 = sizeof(T) * smem_elems(n, r, rp16) + sizeof(int) * rp16;
  const size_t smemg = sizeof(T) * (3 + kStage) * (size_t)n + 64;
  bool use_sm = false;
  int csize = 0;
  BAMG_TRY(choose_policy<T>(ksm, kgl, smem16, smemg, DenseAttrs<T>::tsm, DenseAttrs<T>::tgl, &use_sm, &csize));
  DevMem big, glob, de, sg, vb, z, un, ctl;
  if (use_sm) {
    a.RP = rp16;
  } else {
    size_t nn = (size_t)n * n;
    size_t elems = 5 * nn + (size_t)n * 2 * r + 8 * (size_t)n + 64 + kMaxNB * (size_t)part_stride(n);
    BAMG_TRY(big.alloc(sizeof(T) * elems, s));
    BAMG_TRY(glob.alloc(sizeof(int) * n, s));
    T* p = big.as<T>();
    a.LM = p; p += nn;
    a.LN = p; p += nn;
    a.S1 = p; p += nn;
    a.S2 = p; p += nn;
    a.S3 = p; p += nn;
    a.R = p; p += (size_t)n * 2 * r;
    a.pub = p; p += 8 * (size_t)n + 64;
    a.part = p;
    a.pcol = glob.as<int>();
    a.RP = (n + csize - 1) / csize;
  }
  BAMG_TRY(de.alloc(sizeof(T) * 3 * n, s));
  BAMG_TRY(sg.alloc(sizeof(T) * r, s));
  BAMG_TRY(vb.alloc(sizeof(T) * (size_t)r * n, s));
  BAMG_TRY(z.alloc(sizeof(T) * (size_t)r * 12 * n, s));
  BAMG_TRY(un.alloc(sizeof(T) * n, s));
  BAMG_TRY(ctl.alloc(2 * sizeof(DenseCtl), s));
  BAMG_CUDA(cudaMemsetAsync(ctl.p, 0, 2 * sizeof(DenseCtl), s));
  BAMG_CUDA(cudaMemsetAsync(un.p, 0, sizeof(T) * n, s));
  BAMG_CUDA(cudaMemsetAsync(de.p, 0, sizeof(T) * 3 * n, s));
  a.d = de.as<T>(); a.e = a.d + n; a.taup = a.e + n;
  a.sig = sg.as<T>(); a.vb = vb.as<T>(); a.z = z.as<T>(); a.unull = un.as<T>(); a.ctl = ctl.as<DenseCtl>();
  a.NB = csize;

  // ---- pseudo-inverse (independent of the triplets) on a side stream
  DenseArgs<T> q = {};
  bool p_sm = false;
  int p_csize = 0;
  DevMem pbig, pglob, pxs;
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  auto psm = pinv_kernel<T, true>;
  auto pgl = pinv_kernel<T, false>;
  size_t psmem16 = 0, psmemg = sizeof(T) * 2 * (size_t)n + 64;
  if (Bpinv) {
    q.n = n; q.r = r; q.B = B; q.Bpinv = Bpinv;
    psmem16 = sizeof(T) * pinv_smem_elems(n, rp16) + sizeof(int) * rp16;
    BAMG_TRY(choose_policy<T>(psm, pgl, psmem16, psmemg, DenseAttrs<T>::psm, DenseAttrs<T>::pgl, &p_sm, &p_csize));
    if (p_sm) {
      q.RP = rp16;
    } else {
      BAMG_TRY(pbig.alloc(sizeof(T) * ((size_t)2 * n * n + 2 * (size_t)n + 64 + kMaxNB * (size_t)part_stride(n)), s));
      BAMG_TRY(pglob.alloc(sizeof(int) * n, s));
      T* p = pbig.as<T>();
      q.S2 = p; p += (size_t)2 * n * n;
      q.pub = p; p += 2 * (size_t)n + 64;
      q.part = p;
      q.pcol = pglob.as<int>();
      q.RP = (n + p_csize - 1) / p_csize;
    }
    BAMG_TRY(pxs.alloc(sizeof(T) * n, s));
    q.unull = pxs.as<T>();
    q.ctl = ctl.as<DenseCtl>() + 1;
    q.NB = p_csize;
    BAMG_TRY(side_stream(&s2));
    BAMG_CUDA(cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming));
    BAMG_CUDA(cudaEventCreateWithFlags(&ev1, cudaEventDisableTiming));
    BAMG_CUDA(cudaEventRecord(ev0, s));
    BAMG_CUDA(cudaStreamWaitEvent(s2, ev0, 0));
    BAMG_TRY(cluster_launch<T>(p_sm ? psm : pgl, p_csize, p_sm ? psmem16 : psmemg, s2, q));
    BAMG_CUDA(cudaEventRecord(ev1, s2));
  }
  bamg_status st = cluster_launch<T>(use_sm ? ksm : kgl, csize, use_sm ? smem16 : smemg, s, a);
  if (Bpinv) {
    // the caller's stream waits for the pseudo-inverse (also before any
    // buffer of this call is released on it)
    cudaStreamWaitEvent(s, ev1, 0);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
  }
  BAMG_TRY(st);
  // (before the status read below: a copy into pageable memory returns only
  // when the stream has drained)
  const auto t_hw0 = std::chrono::steady_clock::now();
  const bamg_status hw = during.fn ? during.fn(during.ctx) : BAMG_OK;
  const auto t_hw1 = std::chrono::steady_clock::now();
  if (err_out && !std::getenv("BAMG_TRACE")) {
    // status for the caller's later read; this call's buffers are released
    // on the stream after the kernels (and after the side stream's event)
    static_assert(offsetof(DenseCtl, err) == 0, "status word first");
    BAMG_CUDA(cudaMemcpyAsync(err_out, ctl.p, sizeof(int), cudaMemcpyDeviceToDevice, s));
    return hw;
  }
  DenseCtl h[2];
  BAMG_CUDA(cudaMemcpyAsync(h, ctl.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  const auto t_hw2 = std::chrono::steady_clock::now();
  if (std::getenv("BAMG_TRACE")) {
    const char* nm[5] = {"cholesky", "form_C", "bidiag", "bidiag_svd", "triplets"};
    fprintf(stderr, "[bamg] coarsest n=%d prec=%s cluster=%d %s:", n, sizeof(T) == 4 ? "f32" : "f64", csize,
            use_sm ? "smem" : "global");
    for (int k = 0; k < 5; ++k)
      if (h[0].tp[k + 1] >= h[0].tp[k] && h[0].tp[k + 1])
        fprintf(stderr, " %s=%.1fus", nm[k], (h[0].tp[k + 1] - h[0].tp[k]) / 1e3);
    if (Bpinv && h[1].tp[1] >= h[1].tp[0])
      fprintf(stderr, " | pinv (%s, concurrent)=%.1fus", p_sm ? "smem" : "global", (h[1].tp[1] - h[1].tp[0]) / 1e3);
    if (during.fn)
      fprintf(stderr, " | host work meanwhile %.1fus, then waited %.1fus",
              std::chrono::duration<double, std::micro>(t_hw1 - t_hw0).count(),
              std::chrono::duration<double, std::micro>(t_hw2 - t_hw1).count());
    fprintf(stderr, "\n");
  }
  if (h[0].err == 2) {
    set_error("coarsest level: M or N is not positive definite");
    return BAMG_ERR_NUMERIC;
  }
  if (err_out) BAMG_CUDA(cudaMemsetAsync(err_out, 0, sizeof(int), s));
  return hw;
}

bamg_status coarsest_solve(int prec, int n, int r, const double* B, const double* M, const double* N,
                           double* sigma, double* U, double* V, double* Bpinv, cudaStream_t s, HostWork during,
                           int* err_out) {
  if (n < 2 || n > kDenseMaxN || r < 1 || r > n || r > kMaxR) {
    set_error("coarsest solve needs 1 <= r <= min(n, %d), 2 <= n <= %d (n = %d, r = %d)", kMaxR, kDenseMaxN, n, r);
    return BAMG_ERR_UNSUPPORTED;
  }
  if (prec == 1) return coarsest_t<float>(n, r, B, M, N, sigma, U, V, Bpinv, s, during, err_out);
  return coarsest_t<double>(n, r, B, M, N, sigma, U, V, Bpinv, s, during, err_out);
}

}  // namespace bamg
