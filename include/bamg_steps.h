/*
 * bamg_steps.h - the individual device steps of the bootstrap-AMG hot path,
 * exported for callers that assemble their own pipeline and for
 * step-by-step verification.
 *
 * All pointers are device pointers unless named *_host.  Blocks of test
 * vectors are n x ld row-major (row i holds its ld entries contiguously;
 * columns >= r are padding); ld must be 4, 8, 16 or 32.  CSR arrays are int32
 * row_ptr[rows+1] and int32 col[nnz] sorted ascending within each row.
 * `prec` selects the value type of matrices and blocks: 0 = double,
 * 1 = float.  Steps that size their output in two calls (count, then fill)
 * read the count back to the host and synchronise `stream`.  Scratch space,
 * where a step needs it, is taken from the stream-ordered device pool and
 * returned before the call ends.  Errors: BAMG_ERR_ARG for bad sizes or
 * null pointers, BAMG_ERR_CUDA for launch failures, the step-specific codes
 * documented below.
 */
#ifndef BAMG_STEPS_H
#define BAMG_STEPS_H

#include "bamg.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Section 2, eq. steadystatesystemlinear: B = I - A with the diagonal always
 * stored.  Count pass: *nnzB = nnz(A) + number of rows of A without a
 * diagonal entry.  Fill pass writes B_row_ptr[n+1], B_col[nnzB], B_val. */
bamg_status bamg_step_build_B_count(int n, const int32_t* A_rp, const int32_t* A_ci,
                                    int64_t* nnzB, void* stream);
bamg_status bamg_step_build_B(int n, const int32_t* A_rp, const int32_t* A_ci,
                              const double* A_val, int32_t* B_rp, int32_t* B_ci,
                              double* B_val, void* stream);

/* Section 2: validation of a column-stochastic A (a_ij >= 0 and
 * |sum_i a_ij - 1| <= tol).  *bad_host = number of offending columns plus
 * entries (0 = valid). */
bamg_status bamg_step_check_stochastic(int n, const int32_t* A_rp, const int32_t* A_ci,
                                       const double* A_val, double tol,
                                       int64_t* bad_host, void* stream);

/* Transpose of a rows x cols CSR (values double).  Output row_ptr[cols+1],
 * columns ascending. */
bamg_status bamg_step_transpose(int rows, int cols, int nnz, const int32_t* rp,
                                const int32_t* ci, const double* val, int32_t* t_rp,
                                int32_t* t_ci, double* t_val, void* stream);

/* Algorithm 1 smoothing loops with weighted Jacobi (Section 3; F = D/omega):
 * Y = X + omega D^{-1} (R .* sigma - B X), sweep by sweep, where D is the
 * diagonal of B, R is an optional right-hand side block (NULL = 0) scaled per
 * column by sigma (NULL = 1), and keep_col0 = 1 leaves column 0 unchanged
 * (the fixed left null vector u^(1) = 1 of Section 5).  dinv[i] = 1/b_ii.
 * X and Y may not alias. */
bamg_status bamg_step_relax_block(int prec, int n, int ld, const int32_t* rp,
                                  const int32_t* ci, const void* val, const void* dinv,
                                  const void* X, void* Y, const void* R,
                                  const void* sigma, double omega, int keep_col0,
                                  void* stream);

/* Reciprocal Jacobi divisors (Section 3, weighted Jacobi): dinv[i] = 1/b_ii
 * where b_ii > 0; where b_ii <= 0 (possible on coarse Petrov-Galerkin levels,
 * which the paper does not treat) 1/max(||row i||_1, ||column i||_1).  B and
 * its transpose (trp, tva: CSR of B^T) are device CSR arrays of an n x n
 * matrix; dinv: device, n doubles; *nsafe_host receives the number of rows
 * that took the l1 divisor.  BAMG_ERR_NUMERIC when a row and its column are
 * both zero. */
bamg_status bamg_step_jacobi_divisor(int n, const int32_t* rp, const int32_t* ci, const double* val,
                                     const int32_t* trp, const double* tval, double* dinv,
                                     int* nsafe_host, void* stream);

/* Y = A X for a rows x cols CSR A and a cols x ld block X (Y rows x ld). */
bamg_status bamg_step_spmm_block(int prec, int rows, int ld, const int32_t* rp,
                                 const int32_t* ci, const void* val, const void* X,
                                 void* Y, void* stream);

/* The vector kernel of the V-cycle (Section 3, eq. error_propagator_twogrid)
 * and of GMRES (Section 6): one group of lanes per row of the n x n CSR
 * matrix B with nnz entries (the group width follows nnz / n, as in the
 * solver).  mode 0: y = x + omega dinv .* (b - B x), a weighted Jacobi sweep;
 * mode 1: y = omega dinv .* b, the first sweep from zero; mode 2:
 * y = b - B x, the residual; mode 3: y = B x; mode 4: y += B x; mode 5:
 * the first two sweeps from zero in one pass, bit for bit mode 1 followed by
 * mode 0.  x, b, y, dinv: device vectors of n values in the precision prec
 * (0 = double, 1 = float); b is not read in modes 3 and 4, x not in modes 1
 * and 5, dinv only in modes 0, 1 and 5 (NULL allowed otherwise).  y may not
 * alias x or b.
 * BAMG_ERR_ARG for a missing argument or an unknown mode. */
bamg_status bamg_step_csr_vec(int prec, int mode, int n, int64_t nnz, const int32_t* rp,
                              const int32_t* ci, const void* val, const void* dinv,
                              double omega, const void* x, const void* b, void* y,
                              void* stream);

/* eq. ls_weights with unit test vectors: for each column k < r,
 * norm_host[k] = ||x_k||_2 and w_host[k] = ||x_k||_2 / ||B x_k||_2 (the
 * square root of omega_k after normalising x_k).  When normalise = 1 the
 * columns of X are scaled to unit norm in place (skip_col0 = 1 leaves
 * column 0 alone and reports w_host[0] = 0).  FP64 accumulation. */
bamg_status bamg_step_norms_weights(int prec, int n, int ld, int r, const int32_t* rp,
                                    const int32_t* ci, const void* val, void* X,
                                    int normalise, int skip_col0, double* norm_host,
                                    double* w_host, void* stream);

/* bamg_step_norms_weights without any device allocation (the paper has no
 * counterpart; this is a service for callers).  For callers that must not
 * allocate device memory once running - for example a service whose device
 * memory is planned up front by its own allocator or a fixed budget, where a
 * cudaMalloc or cudaMallocAsync mid-run could fail, stall or fragment that
 * plan.  Arguments, results and tolerances are those of
 * bamg_step_norms_weights; scratch lives in a fixed ~0.8 MB device array
 * that each GPU loading the library keeps until the process exits.  The
 * first call on a device looks up that array's address (make it before any
 * stream capture); after a cudaDeviceReset the next call looks it up again
 * in the new context.  ld must be 4, 8, 16 or 32 and r <= ld, else
 * BAMG_ERR_ARG.  All calls share the array: calls that overlap on the GPU
 * race and must be serialised by the caller. */
bamg_status bamg_step_norms_weights_noalloc(int prec, int n, int ld, int r, const int32_t* rp,
                                            const int32_t* ci, const void* val, void* X,
                                            int normalise, int skip_col0, double* norm_host,
                                            double* w_host, void* stream);

/* Geometric C/F splitting (Section 7): coarse = (i even, j even) on an
 * nx x ny grid.  cf[n] int8 (1 = C), cmap[n] int32 coarse index or -1,
 * and the interpolation sets J_i (C points of the 3x3 box, ascending) as a
 * CSR over all n rows (coarse rows empty): J_rp[n+1], J_ci[<= 4n] with fine
 * indices.  *nc_host = number of coarse points. */
bamg_status bamg_step_coarsen_geometric(int nx, int ny, int8_t* cf, int32_t* cmap,
                                        int32_t* J_rp, int32_t* J_ci, int* nc_host,
                                        void* stream);

/* Greedy maximal independent set on the symmetrised graph of B, vertices
 * in decreasing SplitMix64 priority (seed, stream 4096 + level), equal
 * priorities by increasing index; computed by parallel rounds that reach the
 * same set.  Needs the patterns of B and B^T.  Writes cf, cmap. */
bamg_status bamg_step_coarsen_mis(int n, const int32_t* B_rp, const int32_t* B_ci,
                                  const int32_t* Bt_rp, const int32_t* Bt_ci,
                                  uint64_t seed, int level, int8_t* cf, int32_t* cmap,
                                  int* nc_host, void* stream);

/* Greedy colouring of the symmetrised graph of B (Section 3: Gauss-Seidel is
 * an admissible splitting; rows of one colour are updated together): the
 * vertices in decreasing SplitMix64 priority (seed, stream 6144 + level,
 * ties by lower index), each taking the smallest colour absent from its
 * neighbours taken before it; computed in parallel rounds with the same
 * result bit for bit.  B and B^T as CSR (device, int32); colour[n] (device,
 * caller-owned) receives colours 0 .. *ncolours_host - 1.  Synchronises the
 * stream.  BAMG_ERR_NUMERIC if the rounds do not finish within n + 1 (not
 * reachable on valid input: each round colours at least the highest-priority
 * uncoloured vertex). */
bamg_status bamg_step_colour(int n, const int32_t* B_rp, const int32_t* B_ci, const int32_t* Bt_rp,
                             const int32_t* Bt_ci, uint64_t seed, int level, int32_t* colour, int* ncolours_host,
                             void* stream);

/* Rows grouped by colour, ascending inside a colour: rows[n] (device) and
 * colour_rp_host[ncolours + 1] (host) with the rows of colour c at
 * rows[colour_rp_host[c] .. colour_rp_host[c + 1]).  Synchronises the
 * stream. */
bamg_status bamg_step_colour_rows(int n, const int32_t* colour, int ncolours, int32_t* colour_rp_host,
                                  int32_t* rows, void* stream);

/* One forward multicolour Gauss-Seidel sweep in place on x[n] (device):
 * colour by colour, x_i <- x_i + (b_i - (B x)_i) * dinv_i over the rows of
 * the colour (unweighted; dinv = 1 / Jacobi divisor).  val, dinv, b, x are
 * double (prec = 0) or float (prec = 1); colour_rp_host and rows as from
 * bamg_step_colour_rows (BAMG_ERR_ARG unless colour_rp_host runs from 0 to n
 * without decreasing).  Stream-ordered; x is updated in place, so rows of one
 * colour must not be coupled by B (true for the colouring above). */
bamg_status bamg_step_mcgs_sweep(int prec, int n, const int32_t* rp, const int32_t* ci, const void* val,
                                 const void* dinv, int ncolours, const int32_t* colour_rp_host, const int32_t* rows,
                                 const void* b, void* x, void* stream);

/* Interpolation sets on a graph: per fine point, coarse neighbours ranked by
 * strength |b_ij| + |b_ji| (descending, ties by index), at most c_max, topped
 * up to c_min from distance two by the largest strength product.  Output J
 * CSR over all n rows (coarse rows empty), fine indices ascending; J_ci must
 * hold n * c_max entries. */
bamg_status bamg_step_graph_sets(int n, const int32_t* B_rp, const int32_t* B_ci,
                                 const double* B_val, const int32_t* Bt_rp,
                                 const int32_t* Bt_ci, const double* Bt_val,
                                 const int8_t* cf, int c_min, int c_max, int32_t* J_rp,
                                 int32_t* J_ci, void* stream);

/* eq. ls_interpolation: for every fine row i with J_i non-empty, the weights
 * p_i = argmin sum_{k<r} (w_k (v_i^(k) - sum_{j in J_i} p_ij v_j^(k)))^2, by
 * Householder QR in FP64 (w = sqrt of the LS weights).  Output row-wise into
 * out[J_rp[i] .. J_rp[i+1]).  constrained = 1 solves the restriction
 * problem of Section 5 instead: rows k >= 1 only, subject to sum_j p_ij = 1.
 * ridge = delta > 0 adds lambda ||p_i - 1/c||^2 to each fit, lambda = delta *
 * trace(G_i) / c with G_i the weighted Gram matrix of the c = |J_i| neighbour
 * columns (bamg_params.ls_ridge; 0 = the plain fit, a negative or non-finite
 * delta is BAMG_ERR_ARG).
 * Sets must satisfy |J_i| <= min(ld, 8) (bamg_setup guarantees it through
 * c_max <= 8 and c_max <= block width); rows with larger sets are left
 * unwritten and the call returns BAMG_ERR_ARG (the other rows are fitted).
 * *rankdef_host = number of rows whose fit was rank deficient (pivots below
 * 1e-13 relative were dropped); in FP32 (prec = 1) a row that is refitted in
 * FP64 is counted by the FP64 fit only. */
bamg_status bamg_step_ls_fit(int prec, int n, int ld, int r, const int32_t* J_rp,
                             const int32_t* J_ci, const void* X, const double* w,
                             int constrained, double ridge, double* out,
                             int* rankdef_host, void* stream);

/* Two-phase sparse product C = A B (A: m x k, B: k x p, values double) on the
 * structural pattern (entries that cancel are kept).  Symbolic pass writes
 * C_rp[m+1] and *nnzC_host; numeric pass fills C_ci (ascending) and C_val.
 * BAMG_ERR_NUMERIC if a row has more than 8192 products. */
bamg_status bamg_step_spgemm_symbolic(int m, const int32_t* A_rp, const int32_t* A_ci,
                                      const int32_t* B_rp, const int32_t* B_ci,
                                      int32_t* C_rp, int64_t* nnzC_host, void* stream);
bamg_status bamg_step_spgemm_numeric(int m, const int32_t* A_rp, const int32_t* A_ci,
                                     const double* A_val, const int32_t* B_rp,
                                     const int32_t* B_ci, const double* B_val,
                                     const int32_t* C_rp, int32_t* C_ci, double* C_val,
                                     void* stream);

/* eq. generalized_eigenvalue on the coarsest level: the r smallest
 * generalized singular triplets of (B, M, N) (dense n x n row-major, M and N
 * symmetric positive definite), sigma ascending, u^T M u = v^T N v = 1, sign
 * fixed so the largest-magnitude entry of v is positive (for sigma below
 * n*eps*sigma_max the largest entry of u is made positive as well).
 * U, V: n x r row-major.  Bpinv (may be NULL): Moore-Penrose pseudo-inverse
 * of B with its smallest singular value dropped (Section 3), row-major.
 * Computed in the precision `prec` (inputs and outputs stay double).
 * BAMG_ERR_NUMERIC if M or N is not positive definite; n <= 1024. */
bamg_status bamg_step_coarsest(int prec, int n, int r, const double* B, const double* M,
                               const double* N, double* sigma, double* U, double* V,
                               double* Bpinv, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BAMG_STEPS_H */
