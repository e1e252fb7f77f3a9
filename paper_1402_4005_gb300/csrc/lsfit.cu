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
// coalesced LD-element row read.  Householder QR in FP64 with segment
// shuffles, then back substitution.  The constraint is removed by the
// null-space method: p = 1/c + Z y with Z the last c-1 columns of the
// Householder reflector H = I - 2 h h^T / h^T h, h = 1 + sqrt(c) e_1, which
// maps the ones vector to a multiple of e_1 (so those columns are an
// orthonormal basis of the complement of 1).
#include "internal.cuh"

namespace bamg {

constexpr int kCMax = 8;

template <int S>
__device__ inline double seg_sum(double v) {
#pragma unroll
  for (int o = S / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int S>
__device__ inline double seg_get(double v, int src) {
  return __shfl_sync(0xffffffffu, v, src, S);
}

template <typename T, int S, bool CONSTR>
__global__ void __launch_bounds__(256)
ls_fit_kernel(int n, int r, const int32_t* __restrict__ jrp, const int32_t* __restrict__ jci,
              const T* __restrict__ X, const double* __restrict__ w, double* __restrict__ out,
              int* __restrict__ rankdef) {
  constexpr int PPW = 32 / S;
  int lane = threadIdx.x & 31;
  int gw = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  int i = gw * PPW + lane / S;
  int k = lane % S;
  bool valid = i < n;
  int c = valid ? jrp[i + 1] - jrp[i] : 0;
  int base = valid ? jrp[i] : 0;
  if (__reduce_max_sync(0xffffffffu, c) == 0) return;  // warp-uniform exit

  bool row_on = valid && c > 0 && k < r && !(CONSTR && k == 0);
  double wk = row_on ? w[k] : 0.0;
  double y = row_on ? wk * (double)X[(size_t)i * S + k] : 0.0;
  double a[kCMax];
#pragma unroll
  for (int m = 0; m < kCMax; ++m)
    a[m] = (row_on && m < c) ? wk * (double)X[(size_t)jci[base + m] * S + k] : 0.0;

  // Section 5 constraint: substitute p = 1/c + Z y~
  int cc = c;
  double sqc = 0.0, hh = 1.0;
  if (CONSTR && c >= 2) {
    sqc = sqrt((double)c);
    hh = 2.0 * c + 2.0 * sqc;
    double inv_c = 1.0 / c;
    double t = (1.0 + sqc) * a[0];
    double sa = a[0];
#pragma unroll
    for (int m = 1; m < kCMax; ++m) {
      if (m < c) { t += a[m]; sa += a[m]; }
    }
    y -= sa * inv_c;
    double g = 2.0 * t / hh;
#pragma unroll
    for (int m = 0; m < kCMax - 1; ++m) a[m] = (m < c - 1) ? a[m + 1] - g : 0.0;
    a[kCMax - 1] = 0.0;
    cc = c - 1;
  } else if (CONSTR) {
    cc = 0;  // c == 1: p = 1
  }
  int ccw = __reduce_max_sync(0xffffffffu, cc);

  // Householder QR of the S x cc system, right-hand side y.
  double rdiag[kCMax];
  double rmax = 0.0;
#pragma unroll
  for (int j = 0; j < kCMax; ++j) {
    rdiag[j] = 0.0;
    if (j < ccw) {
      bool act = j < cc;
      double xj = (k >= j) ? a[j] : 0.0;
      double s2 = seg_sum<S>(xj * xj);
      double ajj = seg_get<S>(a[j], j);
      double nrm = sqrt(s2);
      double alpha = ajj > 0.0 ? -nrm : nrm;
      double v = (k == j) ? ajj - alpha : xj;
      double vtv = 2.0 * nrm * (nrm + fabs(ajj));
      bool go = act && nrm > 0.0;
      double inv = go ? 2.0 / vtv : 0.0;
#pragma unroll
      for (int m = j + 1; m < kCMax; ++m) {
        if (m < ccw) {
          double d = seg_sum<S>(v * a[m]);
          if (go) a[m] -= v * (d * inv);
        }
      }
      double dy = seg_sum<S>(v * y);
      if (go) y -= v * (dy * inv);
      if (go) a[j] = (k == j) ? alpha : (k > j ? 0.0 : a[j]);
      rdiag[j] = go ? alpha : 0.0;
      rmax = fmax(rmax, fabs(rdiag[j]));
    }
  }
  // back substitution; pivots below 1e-13 relative are dropped
  double p[kCMax];
  int dropped = 0;
#pragma unroll
  for (int j = kCMax - 1; j >= 0; --j) {
    p[j] = 0.0;
    if (j < ccw) {
      double num = y;
#pragma unroll
      for (int m = j + 1; m < kCMax; ++m) num -= a[m] * p[m];
      bool keep = j < cc && fabs(rdiag[j]) > 1e-13 * rmax;
      if (j < cc && !keep) dropped = 1;
      double pj = (k == j && keep) ? num / a[j] : 0.0;
      p[j] = seg_get<S>(pj, j);
    }
  }
  if (!valid || c == 0) return;
  double val;
  if (CONSTR) {
    if (c == 1) {
      val = 1.0;
    } else {
      double sy = 0.0;
#pragma unroll
      for (int m = 0; m < kCMax - 1; ++m) sy += (m < c - 1) ? p[m] : 0.0;
      double g = 2.0 * sy / hh;
      double ym = 0.0;
#pragma unroll
      for (int m = 1; m < kCMax; ++m) if (m == k) ym = p[m - 1];
      val = 1.0 / c + (k == 0 ? -(1.0 + sqc) * g : ym - g);
    }
  } else {
    val = 0.0;
#pragma unroll
    for (int m = 0; m < kCMax; ++m) if (m == k) val = p[m];
  }
  if (k < c) out[base + k] = val;
  if (k == 0 && dropped) atomicAdd(rankdef, 1);
}

template <typename T, int S>
static bamg_status ls_fit_s(int n, int r, const int32_t* J_rp, const int32_t* J_ci, const T* X,
                            const double* w, int constrained, double* out, int* rankdef, cudaStream_t s) {
  constexpr int PPW = 32 / S;
  unsigned grid = cdiv(n, 8 * PPW);
  if (constrained)
    return launch(ls_fit_kernel<T, S, true>, dim3(grid), dim3(256), 0, s, n, r, J_rp, J_ci, X, w, out, rankdef);
  return launch(ls_fit_kernel<T, S, false>, dim3(grid), dim3(256), 0, s, n, r, J_rp, J_ci, X, w, out, rankdef);
}

template <typename T>
bamg_status ls_fit(int n, int ld, int r, const int32_t* J_rp, const int32_t* J_ci, const T* X,
                   const double* w, int constrained, double* out, int* rankdef_dev, cudaStream_t s) {
  switch (ld) {
    case 4: return ls_fit_s<T, 4>(n, r, J_rp, J_ci, X, w, constrained, out, rankdef_dev, s);
    case 8: return ls_fit_s<T, 8>(n, r, J_rp, J_ci, X, w, constrained, out, rankdef_dev, s);
    case 16: return ls_fit_s<T, 16>(n, r, J_rp, J_ci, X, w, constrained, out, rankdef_dev, s);
    case 32: return ls_fit_s<T, 32>(n, r, J_rp, J_ci, X, w, constrained, out, rankdef_dev, s);
    default: set_error("block width %d not in {4,8,16,32}", ld); return BAMG_ERR_ARG;
  }
}

template bamg_status ls_fit<float>(int, int, int, const int32_t*, const int32_t*, const float*, const double*,
                                   int, double*, int*, cudaStream_t);
template bamg_status ls_fit<double>(int, int, int, const int32_t*, const int32_t*, const double*,
                                    const double*, int, double*, int*, cudaStream_t);

}  // namespace bamg
