// Batched least-squares fits of interpolation rows and restriction columns.
//
// eq. ls_interpolation / eq. ls_weights: for a fine point i with set J_i
// (c = |J_i| <= 8) and test vectors x^(k), k < r, the weights minimise
//   sum_k ( w_k x_i^(k) - sum_{j in J_i} p_j w_k x_j^(k) )^2 ,
// w_k = sqrt(omega_k).  Section 5 (restriction): rows k >= 1 only (u^(1) = 1
// enters as the constraint) and sum_j p_j = 1.
//
// GPU mapping: one segment of LD lanes per fine point, lane k = test vector
// k, so the r x c system lives one row per lane and every gather of x_j is a
// coalesced LD-element row read.  Householder QR with segment shuffles, then
// back substitution.  FP64 test vectors are fitted in FP64.  FP32 test
// vectors (mixed precision) are fitted in FP32 first; a point whose
// triangular factor has min |r_jj| < 1e-3 max |r_jj| (an ill-conditioned
// neighbourhood) is flagged and fitted again in FP64 by a second launch that
// skips every other point.  The constraint is removed by the
// null-space method: p = 1/c + Z y with Z the last c-1 columns of the
// Householder reflector H = I - 2 h h^T / h^T h, h = 1 + sqrt(c) e_1, which
// maps the ones vector to a multiple of e_1 (so those columns are an
// orthonormal basis of the complement of 1).
//
// Optional Tikhonov term (ridge = delta > 0, not in the paper): the fit also
// penalises lambda ||p - 1/c||^2 with lambda = delta * trace(G) / c, G the
// weighted Gram matrix of the c neighbour columns, i.e. it pulls the
// directions the test vectors leave ill-determined towards the equal weights
// of the simple-averaging operator (Section 5).  Solved as least squares
// with sqrt(lambda) I appended below the test-vector rows: lane k keeps, next
// to its test-vector row, the appended rows k, k + S, ... of that identity,
// and the same Householder sweep reduces both.  The unconstrained fit is
// shifted to the prior first (y <- y - X 1/c, p = 1/c + d); the constrained
// one already works around q0 = 1/c, whose null-space coordinates are zero.
#include "internal.cuh"

namespace bamg {

constexpr int kCMax = 8;

template <int S, typename R>
__device__ inline R seg_sum(R v) {
#pragma unroll
  for (int o = S / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int S, typename R>
__device__ inline R seg_get(R v, int src) {
  return __shfl_sync(0xffffffffu, v, src, S);
}

// R: arithmetic type.  only != nullptr: fit just the points with only[i] != 0.
// flag != nullptr: set flag[i] = 1 where min |r_jj| < cond_tol * max |r_jj|.
// AUG: with the Tikhonov rows of weight ridge (> 0).
// A set larger than min(S, 8) cannot be held by the segment: the row is
// skipped (nothing written) and counted in *oversize.
template <typename T, typename R, int S, bool CONSTR, bool AUG>
__global__ void __launch_bounds__(256)
ls_fit_kernel(int n, int r, const int32_t* __restrict__ jrp, const int32_t* __restrict__ jci,
              const T* __restrict__ X, const double* __restrict__ w, double* __restrict__ out,
              int* __restrict__ rankdef, const int8_t* __restrict__ only, int8_t* __restrict__ flag,
              R cond_tol, R ridge, int* __restrict__ oversize) {
  pdl_wait();
  pdl_trigger();
  constexpr int PPW = 32 / S;
  int lane = threadIdx.x & 31;
  int gw = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  int i = gw * PPW + lane / S;
  int k = lane % S;
  bool valid = i < n && (only == nullptr || only[i] != 0);
  int c = valid ? jrp[i + 1] - jrp[i] : 0;
  int base = valid ? jrp[i] : 0;
  if (c > (S < kCMax ? S : kCMax)) {
    if (k == 0) atomicAdd(oversize, 1);
    c = 0;
  }
  if (__reduce_max_sync(0xffffffffu, c) == 0) return;  // warp-uniform exit

  bool row_on = valid && c > 0 && k < r && !(CONSTR && k == 0);
  R wk = row_on ? R(w[k]) : R(0);
  R y = row_on ? wk * R(X[(size_t)i * S + k]) : R(0);
  R a[kCMax];
#pragma unroll
  for (int m = 0; m < kCMax; ++m)
    a[m] = (row_on && m < c) ? wk * R(X[(size_t)jci[base + m] * S + k]) : R(0);

  // Tikhonov rows: sqrt(lambda), lambda = ridge * trace(G) / c
  constexpr int NB = AUG ? (kCMax + S - 1) / S : 1;
  R sq_lam = R(0);
  if constexpr (AUG) {
    R loc = R(0);
#pragma unroll
    for (int m = 0; m < kCMax; ++m) loc += a[m] * a[m];
    const R tr = seg_sum<S>(loc);
    sq_lam = c > 0 ? sqrt(ridge * tr / R(c)) : R(0);
    if (!CONSTR && c > 0) {  // shift to the prior p0 = 1/c
      R sa = R(0);
#pragma unroll
      for (int m = 0; m < kCMax; ++m) sa += a[m];
      y -= sa / R(c);
    }
  }

  // Section 5 constraint: substitute p = 1/c + Z y~
  int cc = c;
  R sqc = 0, hh = 1;
  if (CONSTR && c >= 2) {
    sqc = sqrt(R(c));
    hh = R(2) * R(c) + R(2) * sqc;
    R inv_c = R(1) / R(c);
    R t = (R(1) + sqc) * a[0];
    R sa = a[0];
#pragma unroll
    for (int m = 1; m < kCMax; ++m) {
      if (m < c) { t += a[m]; sa += a[m]; }
    }
    y -= sa * inv_c;
    R g = R(2) * t / hh;
#pragma unroll
    for (int m = 0; m < kCMax - 1; ++m) a[m] = (m < c - 1) ? a[m + 1] - g : R(0);
    a[kCMax - 1] = R(0);
    cc = c - 1;
  } else if (CONSTR) {
    cc = 0;  // c == 1: p = 1
  }
  int ccw = __reduce_max_sync(0xffffffffu, cc);

  // appended rows: lane k holds rows k + t*S of sqrt(lambda) I (cc x cc),
  // right-hand side zero; they sit below every test-vector row
  R b[NB][kCMax], y2[NB];
#pragma unroll
  for (int t = 0; t < NB; ++t) {
    y2[t] = R(0);
#pragma unroll
    for (int m = 0; m < kCMax; ++m) b[t][m] = (AUG && k + t * S == m && m < cc) ? sq_lam : R(0);
  }

  // Householder QR of the S x cc system (plus the appended rows), right-hand side y.
  R rdiag[kCMax];
  R rmax = 0, rmin = R(1e30);
#pragma unroll
  for (int j = 0; j < kCMax; ++j) {
    rdiag[j] = R(0);
    if (j < ccw) {
      bool act = j < cc;
      R xj = (k >= j) ? a[j] : R(0);
      R loc2 = xj * xj;
      if constexpr (AUG) {
#pragma unroll
        for (int t = 0; t < NB; ++t) loc2 += b[t][j] * b[t][j];
      }
      R s2 = seg_sum<S>(loc2);
      R ajj = seg_get<S>(a[j], j);
      R nrm = sqrt(s2);
      R alpha = ajj > R(0) ? -nrm : nrm;
      R v = (k == j) ? ajj - alpha : xj;
      R vtv = R(2) * nrm * (nrm + fabs(ajj));
      bool go = act && nrm > R(0);
      R inv = go ? R(2) / vtv : R(0);
#pragma unroll
      for (int m = j + 1; m < kCMax; ++m) {
        if (m < ccw) {
          R dl = v * a[m];
          if constexpr (AUG) {
#pragma unroll
            for (int t = 0; t < NB; ++t) dl += b[t][j] * b[t][m];
          }
          R d = seg_sum<S>(dl);
          if (go) a[m] -= v * (d * inv);
          if constexpr (AUG) {
#pragma unroll
            for (int t = 0; t < NB; ++t)
              if (go) b[t][m] -= b[t][j] * (d * inv);
          }
        }
      }
      R dyl = v * y;
      if constexpr (AUG) {
#pragma unroll
        for (int t = 0; t < NB; ++t) dyl += b[t][j] * y2[t];
      }
      R dy = seg_sum<S>(dyl);
      if (go) y -= v * (dy * inv);
      if constexpr (AUG) {
#pragma unroll
        for (int t = 0; t < NB; ++t) {
          if (go) y2[t] -= b[t][j] * (dy * inv);
          if (go) b[t][j] = R(0);
        }
      }
      if (go) a[j] = (k == j) ? alpha : (k > j ? R(0) : a[j]);
      rdiag[j] = go ? alpha : R(0);
      rmax = fmax(rmax, fabs(rdiag[j]));
      if (act) rmin = fmin(rmin, fabs(rdiag[j]));
    }
  }
  // back substitution; pivots below 1e-13 relative are dropped
  R p[kCMax];
  int dropped = 0;
#pragma unroll
  for (int j = kCMax - 1; j >= 0; --j) {
    p[j] = R(0);
    if (j < ccw) {
      R num = y;
#pragma unroll
      for (int m = j + 1; m < kCMax; ++m) num -= a[m] * p[m];
      bool keep = j < cc && fabs(rdiag[j]) > R(1e-13) * rmax;
      if (j < cc && !keep) dropped = 1;
      R pj = (k == j && keep) ? num / a[j] : R(0);
      p[j] = seg_get<S>(pj, j);
    }
  }
  // the constrained weights from the null-space coordinates: in FP64 for an
  // FP64 fit; in FP32 for an FP32 fit (FP64 division and square root are
  // costly on this part), after which the entry of the last lane is moved
  // by 1 - (the FP64 sum of the segment's weights), so that the weights
  // still sum to one to FP64 rounding
  double val = 0.0;
  if (CONSTR) {
    if constexpr (sizeof(R) == 4) {
      float vf = 1.0f;
      if (c > 1) {
        const float sq = sqrtf((float)c), h2 = 2.0f * c + 2.0f * sq;
        float sy = 0.0f;
#pragma unroll
        for (int m = 0; m < kCMax - 1; ++m) sy += (m < c - 1) ? (float)p[m] : 0.0f;
        const float g = 2.0f * sy / h2;
        float ym = 0.0f;
#pragma unroll
        for (int m = 1; m < kCMax; ++m) if (m == k) ym = (float)p[m - 1];
        vf = 1.0f / (float)c + (k == 0 ? -(1.0f + sq) * g : ym - g);
      }
      const double tot = seg_sum<S>((valid && k < c) ? (double)vf : 0.0);   // every lane shuffles
      val = (double)vf;
      if (c > 1 && k == c - 1) val += 1.0 - tot;
      if (c == 1) val = 1.0;
    } else if (c == 1) {
      val = 1.0;
    } else {
      const double sq = sqrt((double)c), h2 = 2.0 * c + 2.0 * sq;
      double sy = 0.0;
#pragma unroll
      for (int m = 0; m < kCMax - 1; ++m) sy += (m < c - 1) ? (double)p[m] : 0.0;
      double g = 2.0 * sy / h2;
      double ym = 0.0;
#pragma unroll
      for (int m = 1; m < kCMax; ++m) if (m == k) ym = (double)p[m - 1];
      val = 1.0 / c + (k == 0 ? -(1.0 + sq) * g : ym - g);
    }
  } else {
#pragma unroll
    for (int m = 0; m < kCMax; ++m) if (m == k) val = (double)p[m];
    if (AUG) val += 1.0 / c;
  }
  if (!valid || c == 0) return;
  // a row flagged for the FP64 refit is counted by that refit alone
  const bool refit = flag != nullptr && cc > 0 && rmin < cond_tol * rmax;
  if (refit && k == 0) flag[i] = 1;
  if (k < c) out[base + k] = val;
  if (k == 0 && dropped && !refit) atomicAdd(rankdef, 1);
}

template <typename T, typename R, int S>
static bamg_status ls_fit_launch(int n, int r, const int32_t* J_rp, const int32_t* J_ci, const T* X,
                                 const double* w, int constrained, double ridge, double* out, int* rankdef,
                                 const int8_t* only, int8_t* flag, int* oversize, cudaStream_t s) {
  constexpr int PPW = 32 / S;
  unsigned grid = cdiv(n, 8 * PPW);
  const R tol = R(1e-3), rg = R(ridge);
  if (ridge > 0.0) {
    if (constrained)
      return launch(ls_fit_kernel<T, R, S, true, true>, dim3(grid), dim3(256), 0, s, n, r, J_rp, J_ci, X, w, out,
                    rankdef, only, flag, tol, rg, oversize);
    return launch(ls_fit_kernel<T, R, S, false, true>, dim3(grid), dim3(256), 0, s, n, r, J_rp, J_ci, X, w, out,
                  rankdef, only, flag, tol, rg, oversize);
  }
  if (constrained)
    return launch(ls_fit_kernel<T, R, S, true, false>, dim3(grid), dim3(256), 0, s, n, r, J_rp, J_ci, X, w, out,
                  rankdef, only, flag, tol, rg, oversize);
  return launch(ls_fit_kernel<T, R, S, false, false>, dim3(grid), dim3(256), 0, s, n, r, J_rp, J_ci, X, w, out,
                rankdef, only, flag, tol, rg, oversize);
}

template <typename T, int S>
static bamg_status ls_fit_s(int n, int r, const int32_t* J_rp, const int32_t* J_ci, const T* X,
                            const double* w, int constrained, double ridge, double* out, int* rankdef,
                            int* oversize, cudaStream_t s) {
  if (sizeof(T) == 8)
    return ls_fit_launch<T, double, S>(n, r, J_rp, J_ci, X, w, constrained, ridge, out, rankdef, nullptr, nullptr,
                                       oversize, s);
  // FP32 pass, then FP64 on the flagged (ill-conditioned) points only
  DevMem flag;
  BAMG_TRY(flag.alloc((size_t)n, s));
  BAMG_CUDA(cudaMemsetAsync(flag.p, 0, (size_t)n, s));
  BAMG_TRY(ls_fit_launch<T, float, S>(n, r, J_rp, J_ci, X, w, constrained, ridge, out, rankdef, nullptr,
                                      flag.as<int8_t>(), oversize, s));
  return ls_fit_launch<T, double, S>(n, r, J_rp, J_ci, X, w, constrained, ridge, out, rankdef,
                                     (const int8_t*)flag.as<int8_t>(), nullptr, oversize, s);
}

template <typename T>
bamg_status ls_fit(int n, int ld, int r, const int32_t* J_rp, const int32_t* J_ci, const T* X,
                   const double* w, int constrained, double* out, int* rankdef_dev, cudaStream_t s, double ridge) {
  // rankdef_dev[0]: rank-deficient rows; rankdef_dev[1]: rows whose set exceeds min(ld, 8)
  if (!(ridge >= 0.0 && ridge < 1e300)) {
    set_error("ridge weight %g must be finite and >= 0", ridge);
    return BAMG_ERR_ARG;
  }
  switch (ld) {
    case 4: return ls_fit_s<T, 4>(n, r, J_rp, J_ci, X, w, constrained, ridge, out, rankdef_dev, rankdef_dev + 1, s);
    case 8: return ls_fit_s<T, 8>(n, r, J_rp, J_ci, X, w, constrained, ridge, out, rankdef_dev, rankdef_dev + 1, s);
    case 16: return ls_fit_s<T, 16>(n, r, J_rp, J_ci, X, w, constrained, ridge, out, rankdef_dev, rankdef_dev + 1, s);
    case 32: return ls_fit_s<T, 32>(n, r, J_rp, J_ci, X, w, constrained, ridge, out, rankdef_dev, rankdef_dev + 1, s);
    default: set_error("block width %d not in {4,8,16,32}", ld); return BAMG_ERR_ARG;
  }
}

template bamg_status ls_fit<float>(int, int, int, const int32_t*, const int32_t*, const float*, const double*,
                                   int, double*, int*, cudaStream_t, double);
template bamg_status ls_fit<double>(int, int, int, const int32_t*, const int32_t*, const double*,
                                    const double*, int, double*, int*, cudaStream_t, double);

}  // namespace bamg
