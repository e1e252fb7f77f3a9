// Host-side launchers shared between the translation units of libbamg.
#pragma once

#include "common.cuh"

namespace bamg {

enum VecModeHost { VEC_JACOBI = 0, VEC_JACOBI_ZERO = 1, VEC_RESID = 2, VEC_SPMV = 3, VEC_SPMV_ADD = 4,
                   VEC_JACOBI_ZERO2 = 5 };

// Several double -> float conversions in one launch.
constexpr int kConvMany = 8;
struct ConvMany {
  int k = 0;
  const double* src[kConvMany];
  float* dst[kConvMany];
  size_t n[kConvMany];
};
bamg_status convert_many(const ConvMany& job, cudaStream_t s);

// Several exclusive scans (out[q][0..n[q]], out[q][n[q]] = total), one
// launch when every array is short enough for one block.
constexpr int kScanMany = 4;
struct ScanMany {
  int k = 0;
  const int32_t* in[kScanMany];
  int32_t* out[kScanMany];
  int n[kScanMany];
};
bamg_status scan_many(const ScanMany& job, cudaStream_t s);

// Lanes per row of the vector kernels for a matrix with `avg` entries per row.
inline int vec_lanes(double avg) { return avg <= 3 ? 2 : avg <= 6 ? 4 : avg <= 12 ? 8 : avg <= 24 ? 16 : 32; }

// sparse.cu
bamg_status check_rowptr(int n, const int32_t* rp, int64_t nnz, cudaStream_t s);
bamg_status transpose_csr(int rows, int cols, int nnz, const int32_t* rp, const int32_t* ci,
                          const double* va, int32_t* trp, int32_t* tci, double* tva, cudaStream_t s);
bamg_status build_B_count(int n, const int32_t* rp, const int32_t* ci, int32_t* cnt, cudaStream_t s);
bamg_status build_B_fill(int n, const int32_t* rp, const int32_t* ci, const double* va,
                         const int32_t* brp, int32_t* bci, double* bva, cudaStream_t s);
bamg_status check_stochastic(int n, const int32_t* rp, const int32_t* ci, const double* va, double tol,
                             int64_t* bad_host, cudaStream_t s);

// spgemm.cu
bamg_status spgemm_symbolic(int m, const int32_t* arp, const int32_t* aci, const int32_t* brp,
                            const int32_t* bci, int32_t* crp, int64_t* nnz_host, cudaStream_t s);
bamg_status spgemm_numeric(int m, const int32_t* arp, const int32_t* aci, const double* ava,
                           const int32_t* brp, const int32_t* bci, const double* bva,
                           const int32_t* crp, int32_t* cci, double* cva, cudaStream_t s);
// Independent products C_q = A_q B_q.  With annz (entries of A) and
// maxrow_b (an upper bound on the entries of a row of B) given for every job,
// the scratch is sized by annz * maxrow_b and one host read per call returns
// nnz(C) and maxrow_c (entries of C's longest row); otherwise two host reads.
struct SpgemmJob {
  int m;
  const int32_t *arp, *aci;
  const double* ava;
  const int32_t *brp, *bci;
  const double* bva;
  DevMem *crp, *cci, *cva;   // allocated on the stream
  int64_t nnz;
  int64_t annz = -1;
  int maxrow_b = -1;
  int maxrow_c = -1;          // out (bounded path)
};
bamg_status spgemm_multi(SpgemmJob* jobs, int k, cudaStream_t s);
// C = A B in one expansion pass; allocates C's arrays on s, nnz(C) to the host
bamg_status spgemm(int m, const int32_t* arp, const int32_t* aci, const double* ava, const int32_t* brp,
                   const int32_t* bci, const double* bva, DevMem& crp, DevMem& cci, DevMem& cva, int64_t* nnz_host,
                   cudaStream_t s);

// blockops.cu
template <typename T>
struct RelaxJob {          // Y = X + omega D^{-1}(sig .* R - A X), keep0: column 0 kept
  int n;
  const int32_t *rp, *ci;
  const T *va, *dinv, *X;
  T* Y;
  const T *R, *sig;
  T omega;
  int keep0;
};
template <typename T>
struct SpmmJob {           // Y = A X for a rows x cols CSR A and a block X
  int rows;
  const int32_t *rp, *ci;
  const T *va, *X;
  T* Y;
};
template <typename T>
bamg_status relax_block2(int n, int ld, const int32_t* rp, const int32_t* ci, const T* va, const int32_t* trp,
                         const int32_t* tci, const T* tva, const T* dinv, const T* V, T* Vn, const T* U, T* Un,
                         const T* RV, const T* RU, const T* sig, T omega, int keepU0, cudaStream_t s);
template <typename T>
bamg_status spmm_block_multi(int ld, const SpmmJob<T>* jobs, int k, cudaStream_t s);
template <typename T>
bamg_status relax_block(int n, int ld, const int32_t* rp, const int32_t* ci, const T* va, const T* dinv,
                        const T* X, T* Y, const T* R, const T* sig, T omega, int keep0, cudaStream_t s);
template <typename T>
bamg_status spmm_block(int rows, int ld, const int32_t* rp, const int32_t* ci, const T* va, const T* X,
                       T* Y, cudaStream_t s);
template <typename T>
bamg_status norms_weights(int n, int ld, int r, const int32_t* rp, const int32_t* ci, const T* va, T* X,
                          int normalise, int skip0, T* scale, double* w, double* norms, cudaStream_t s);
template <typename T>
bamg_status norms_weights_ws(int n, int ld, int r, const int32_t* rp, const int32_t* ci, const T* va, T* X,
                             int normalise, int skip0, double* part, int max_blocks, double* sums, T* scale,
                             double* w, double* norms, cudaStream_t s);
template <typename T>
bamg_status col_dots(int n, int ld, int npairs, const T* A0, const T* B0, const T* A1, const T* B1,
                     const T* A2, const T* B2, double* sums, cudaStream_t s);
template <typename T>
bamg_status rayleigh_finalize(const double* sums, int ld, int r, T* sig, double* sig64, cudaStream_t s);
template <typename T>
bamg_status init_vectors(int n, int ld, int r, uint64_t seed, T* U, T* V, cudaStream_t s);
template <typename T>
bamg_status inject(int nc, int ld, const int32_t* cpt, const T* X, T* Xc, cudaStream_t s);
template <typename T>
bamg_status csr_vec(int mode, int n, int G, const int32_t* rp, const int32_t* ci, const T* va, const T* dinv,
                    T omega, const T* x, const T* b, T* y, cudaStream_t s);
template <typename T>
bamg_status dense_gemv(int n, const T* A, const T* x, T* y, cudaStream_t s);
// y = z1 + omega dinv .* (b - B z1), z1 = z0 + P e: the prolongation and the
// first post-smoothing sweep in one pass (B: rp, ci, va with G lanes per row)
template <typename T>
bamg_status prolong_jacobi(int n, int G, const int32_t* rp, const int32_t* ci, const T* va, const T* dinv,
                           T omega, const int32_t* prp, const int32_t* pci, const T* pva, const T* e,
                           const T* z0, const T* b, T* y, cudaStream_t s);

// smooth.cu: multicolour Gauss-Seidel (greedy colouring of the symmetrised
// graph of B in SplitMix64 priority order, rows by colour, sweeps)
bamg_status colour_graph(int n, const int32_t* brp, const int32_t* bci, const int32_t* trp, const int32_t* tci,
                         uint64_t seed, int level, int32_t* colour, int* ncolours, cudaStream_t s);
bamg_status colour_rows(int n, const int32_t* colour, int ncolours, int32_t* colour_rp_host, int32_t* rows,
                        cudaStream_t s);
template <typename T>
bamg_status mcgs_sweep(int G, int ncolours, const int32_t* crp, const int32_t* rows, const int32_t* rp,
                       const int32_t* ci, const T* va, const T* dinv, const T* b, T* x, cudaStream_t s);
template <typename S, typename D>
bamg_status convert(size_t n, const S* a, D* b, cudaStream_t s);
template <typename T>
bamg_status diag_inv(int n, const int32_t* rp, const int32_t* ci, const double* va, const int32_t* trp,
                     const double* tva, T* dinv, int* bad_row, int* nsafe, cudaStream_t s);

// hierarchy.cu: out[0] = sum x, out[1] = sum |x|
bamg_status abs_sums(int n, const double* x, double* out, cudaStream_t s);
bamg_status orient_normalise(int n, double* x, cudaStream_t s);

// coarsen.cu
bamg_status coarsen_geometric(int nx, int ny, int8_t* cf, int32_t* cmap, int32_t* J_rp, int32_t* J_ci,
                              int* nc_host, cudaStream_t s);
bamg_status coarsen_mis(int n, const int32_t* brp, const int32_t* bci, const int32_t* trp,
                        const int32_t* tci, uint64_t seed, int level, int8_t* cf, int32_t* cmap,
                        int* nc_host, cudaStream_t s);
bamg_status graph_sets(int n, const int32_t* brp, const int32_t* bci, const double* bva,
                       const int32_t* trp, const int32_t* tci, const double* tva, const int8_t* cf,
                       int c_min, int c_max, int32_t* J_rp, int32_t* J_ci, cudaStream_t s);
bamg_status coarse_points(int n, const int8_t* cf, const int32_t* cmap, int32_t* cpt, cudaStream_t s);
bamg_status transfer_pattern(int n, const int8_t* cf, const int32_t* cmap, const int32_t* J_rp,
                             const int32_t* J_ci, int32_t* P_rp, int32_t* P_ci, double* P_val,
                             cudaStream_t s);
bamg_status scatter_fits(int n, const int8_t* cf, const int32_t* J_rp, const double* fit,
                         const int32_t* P_rp, double* P_val, cudaStream_t s);
bamg_status average_fits(int n, const int32_t* J_rp, double* fit, cudaStream_t s);

// lsfit.cu
// ridge > 0: Tikhonov term ridge * trace(G) / c * ||p - 1/c||^2 (0 = plain fit).
// rankdef_dev points to two counters: rank-deficient rows, and rows whose set
// exceeds min(ld, 8) (skipped, nothing written).
template <typename T>
bamg_status ls_fit(int n, int ld, int r, const int32_t* J_rp, const int32_t* J_ci, const T* X,
                   const double* w, int constrained, double* out, int* rankdef_dev, cudaStream_t s,
                   double ridge = 0.0);

// mlp_tc.cu: network inference on the tensor cores (err_dev: timeout flag)
bamg_status mlp_forward_tc(int M, const float* P, const void* X, float* Y, int* err_dev, cudaStream_t s);

// dense.cu.  during (optional): host work run while the coarsest kernels
// execute (after their launch, before the call waits for them); its status
// is returned when the solve itself succeeds.
struct HostWork {
  bamg_status (*fn)(void* ctx) = nullptr;
  void* ctx = nullptr;
};
// err_out (optional, device int): the call returns without waiting for the
// kernels and leaves their status there (2 = M or N not positive definite).
bamg_status coarsest_solve(int prec, int n, int r, const double* B, const double* M, const double* N,
                           double* sigma, double* U, double* V, double* Bpinv, cudaStream_t s,
                           HostWork during = HostWork(), int* err_out = nullptr);
bamg_status csr_to_dense(int n, const int32_t* rp, const int32_t* ci, const double* va, double* D,
                         cudaStream_t s);

}  // namespace bamg
