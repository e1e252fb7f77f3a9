/*
 * bamg.h - C ABI of the GB300 bootstrap-AMG solver for the stationary vector
 * of an irreducible Markov chain.
 *
 * Problem (Section 2, eq. steadystatesystemlinear): given the column-stochastic
 * transition matrix A (a_ij = probability of the move j -> i, every column
 * sums to one, A irreducible), find x > 0 with B x = 0, B = I - A.  The
 * result is returned with ||x||_1 = 1.
 *
 * Method: one bootstrap setup cycle (Algorithm 1) builds interpolation P by
 * weighted least squares (eq. ls_interpolation, eq. ls_weights), restriction Q
 * by least squares constrained to 1^T Q = 1^T (Section 5), the Petrov-Galerkin
 * coarse operators B_c = Q B P (Section 3) and approximate singular triplets;
 * the solve phase runs GMRES on the residual equation (Section 6, eq.
 * residual) preconditioned by a V-cycle (eq. error_propagator_twogrid).
 *
 * Conventions for every call:
 *  - every function returns a bamg_status and never aborts or throws;
 *    bamg_last_error() gives a one-line description of the last failure on
 *    the calling thread;
 *  - device pointers are CUDA device addresses of the current device;
 *  - `stream` is a cudaStream_t (NULL = legacy default stream); work is
 *    stream-ordered and a hierarchy must be used from one stream at a time;
 *    the hierarchy returns its memory on the stream given to bamg_setup, so
 *    that stream must stay valid until bamg_destroy;
 *  - the caller owns A and every vector passed in; the library owns the
 *    hierarchy until bamg_destroy();
 *  - on error the outputs are unspecified and no memory is leaked.
 */
#ifndef BAMG_H
#define BAMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BAMG_OK = 0,
  BAMG_ERR_ARG = 1,            /* invalid argument (null pointer, size, layout) */
  BAMG_ERR_NOT_STOCHASTIC = 2, /* a_ij < 0 or a column sum differs from 1      */
  BAMG_ERR_CUDA = 3,           /* a CUDA runtime call or launch failed          */
  BAMG_ERR_OOM = 4,            /* device allocation failed                      */
  BAMG_ERR_NOT_CONVERGED = 5,  /* max_iter reached above the tolerance          */
  BAMG_ERR_BREAKDOWN = 6,      /* GMRES breakdown before convergence            */
  BAMG_ERR_NUMERIC = 7,        /* zero row and column in a coarse B, non-SPD M_l/N_l,
                                  singular fit, or a row beyond kernel limits   */
  BAMG_ERR_TIMEOUT = 8,        /* a bounded device-side wait gave up            */
  BAMG_ERR_UNSUPPORTED = 9,    /* valid request outside this build's limits     */
  BAMG_ERR_IO = 10             /* a file could not be read or written, or is
                                  not a well-formed parameter file              */
} bamg_status;

enum { BAMG_COARSEN_GEOMETRIC = 0, BAMG_COARSEN_MIS = 1 };
enum { BAMG_PREC_FP64 = 0, BAMG_PREC_MIXED = 1 };
enum { BAMG_RESTRICT_LS = 0, BAMG_RESTRICT_AVERAGE = 1 };
enum { BAMG_INTERP_LS = 0, BAMG_INTERP_MLP = 1 };
enum { BAMG_SMOOTH_JACOBI = 0, BAMG_SMOOTH_MCGS = 1 };

/* CSR of the column-stochastic A (row i = probabilities of entering state i).
 * row_ptr[n+1], col_idx[nnz] (ascending within each row, 0 <= col < n),
 * val[nnz].  on_device = 0: host pointers (copied at setup); 1: device
 * pointers (read during bamg_setup only).  nx, ny: grid shape for geometric
 * coarsening, state s = i*ny + j (0 when there is no grid). */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const double* val;
  int on_device;
  int nx, ny;
} bamg_csr;

/* Setup parameters.  Defaults (bamg_params_default) follow Section 7:
 * 3+3 weighted Jacobi sweeps with omega = 0.7, r = 8 test vectors, up to
 * c = 4 interpolation points. */
typedef struct {
  int r;             /* test vectors per side, 1 <= r <= 32                   */
  int max_levels;    /* hierarchy depth limit (>= 1)                           */
  int coarse_min;    /* stop coarsening once n_l <= coarse_min                 */
  int nu_setup;      /* Jacobi sweeps per level in each setup relaxation phase */
  int nu_pre, nu_post; /* V-cycle pre/post Jacobi sweeps                       */
  int c_min, c_max;  /* interpolation set size bounds (graph coarsening)       */
  double omega;      /* Jacobi weight: x <- x + omega D^{-1}(b - B x); a coarse
                        row with b_ii <= 0 takes for d_i the larger l1 norm of
                        row i and column i of B                               */
  int coarsening;    /* BAMG_COARSEN_GEOMETRIC (needs nx, ny) or _MIS          */
  int precision;     /* BAMG_PREC_FP64 or BAMG_PREC_MIXED (FP32 V-cycle and
                        setup relaxation inside FP64 GMRES)                    */
  int restriction;   /* BAMG_RESTRICT_LS (Section 5) or _AVERAGE               */
  uint64_t seed;     /* SplitMix64 seed of test vectors and MIS priorities     */
  double stochastic_tol; /* |column sum - 1| allowed at validation (1e-12)     */
  int max_coarse_dense;  /* largest coarsest level solved densely (<= 1024)    */
  int interp;        /* BAMG_INTERP_LS (eq. ls_interpolation, Section 5) or
                        BAMG_INTERP_MLP: P and Q weights proposed by the
                        interpolation network (geometric coarsening only); the
                        setup then relaxes no test-vector blocks and carries
                        only x^(0) up from the coarsest level               */
  const float* mlp_params; /* device, bamg_mlp_num_params() floats, read during
                        bamg_setup when interp = BAMG_INTERP_MLP              */
  int setup_cycles;  /* bootstrap setup cycles, 1..8 (2 = the BAMG^2 variant of
                        Section 7): each later cycle rebuilds the hierarchy from
                        the previous cycle's finest triplets; must be 1 with
                        network fits                                          */
  int smoother;      /* V-cycle smoother: BAMG_SMOOTH_JACOBI (weighted Jacobi,
                        Section 7) or BAMG_SMOOTH_MCGS (Gauss-Seidel, one of
                        the splittings of Section 3, in multicolour order: the
                        greedy colouring of the symmetrised graph of each
                        level's B, SplitMix64 priorities, stream 6144 + level;
                        x_i += (b_i - (Bx)_i) / d_i, unweighted, d the Jacobi
                        divisor).  The setup relaxations stay weighted Jacobi.
                        Not available for batches.                            */
  double ls_ridge;   /* delta >= 0 (default 0, the paper's plain fit): each LS
                        fit of a P row or Q column also penalises
                        lambda ||p - 1/c||^2, lambda = delta * trace(G) / c, G
                        the weighted Gram matrix of the point's c neighbour
                        columns, pulling ill-determined directions towards
                        the equal weights of the simple-averaging operator
                        (Section 5); not in the paper.  delta = 0.03 keeps
                        the coarse diagonals of the deep 2D and planar-graph
                        hierarchies of Section 7 positive with r = 8; a
                        negative or non-finite delta is BAMG_ERR_ARG.       */
} bamg_params;

typedef struct {
  int restart;       /* GMRES restart length m (>= 1)                          */
  int max_iter;      /* total iteration limit                                  */
  double tol;        /* stop when ||B x||_1 / ||x||_1 <= tol                   */
  int plain;         /* 1: GMRES(restart) without the V-cycle (the identity as
                        preconditioner), started from the uniform vector: the
                        unpreconditioned comparator of Section 7; 0: BAMG      */
} bamg_solve_params;

typedef struct {
  int iterations;    /* preconditioned GMRES iterations                        */
  int iters_to_1e7;  /* first iteration with ||Bx||_2/||x||_2 estimate <= 1e-7 */
  int levels;
  double rel_res_1;  /* final true ||B x||_1 / ||x||_1                          */
  double setup_ms, solve_ms;
  double op_cplx, grid_cplx; /* eq. operator_complexity_def; sum n_l / n      */
  double min_x;      /* smallest entry of the normalised x                     */
  int fallback_iterations; /* mixed precision only: iterations with FP32
                        V-cycles before the solve stalled and continued with
                        FP64 V-cycles from the current x (0 = no fallback;
                        the hierarchy then stays FP64)                        */
} bamg_solve_info;

typedef struct bamg_hierarchy bamg_hierarchy;

bamg_status bamg_params_default(bamg_params* p);
bamg_status bamg_solve_params_default(bamg_solve_params* p);

/* Validates A (a_ij >= 0, sorted in-range indices, column sums within
 * stochastic_tol of 1), forms B = I - A and runs one bootstrap setup cycle
 * (Algorithm 1) on the device.  Irreducibility is a precondition that is not
 * checked.  *out receives a library-owned hierarchy. */
bamg_status bamg_setup(const bamg_csr* A, const bamg_params* p, void* stream,
                       bamg_hierarchy** out);

/* z = C r: one V-cycle from a zero initial guess on the finest level
 * (Section 6, eq. iterate_preconditioner with e^(0) = 0).  r_dev, z_dev:
 * device arrays of n doubles; they may not alias. */
bamg_status bamg_vcycle(bamg_hierarchy* h, const double* r_dev, double* z_dev,
                        void* stream);

/* Solves B x = 0 by V-cycle-preconditioned flexible GMRES on the residual
 * equation started from the setup's x^(0) (Section 6).  x_dev: device array
 * of n doubles receiving x > 0 with ||x||_1 = 1.  info may be NULL.
 * In mixed precision, a solve that hits max_iter (or breaks down) with FP32
 * V-cycles switches the hierarchy to FP64 V-cycles (coarsest pseudo-inverse
 * recomputed in FP64) and continues from its current x with a fresh max_iter
 * (info->fallback_iterations > 0).  Returns BAMG_ERR_NOT_CONVERGED (x still
 * written) when max_iter is hit in FP64. */
bamg_status bamg_solve(bamg_hierarchy* h, double* x_dev, const bamg_solve_params* sp,
                       bamg_solve_info* info, void* stream);

/* Host-buffer convenience: bamg_setup + bamg_solve + copy of x to host memory
 * (x_host: n doubles).  Uses the given stream and synchronises it. */
bamg_status bamg_solve_host(const bamg_csr* A, const bamg_params* p,
                            const bamg_solve_params* sp, double* x_host,
                            bamg_solve_info* info, void* stream);

void bamg_destroy(bamg_hierarchy* h);

const char* bamg_status_string(bamg_status s);
const char* bamg_last_error(void);

/* Number of kernels this library has launched in the process so far. */
uint64_t bamg_launch_count(void);

/* -------------------------------------------------------------- batches --
 * Many independent chains solved together.  Each chain gets its own bootstrap
 * setup (run concurrently on `host_threads` host threads, 0 = 4, each with
 * its own stream); the hierarchies are then joined level by level into
 * block-diagonal operators so that one V-cycle (captured as a CUDA graph)
 * and one flexible GMRES run serve all chains, with per-chain dot products,
 * Givens rotations and convergence tests (Section 6).  Vectors are the
 * concatenation of the chains' vectors in input order (offsets from
 * bamg_batch_offsets).  Every chain must satisfy the conditions of
 * bamg_setup. */
typedef struct bamg_batch bamg_batch;

bamg_status bamg_setup_batched(const bamg_csr* As, int nchains, const bamg_params* p, int host_threads,
                               void* stream, bamg_batch** out);
/* x_dev: concatenated device vector (sum of n_c doubles) receiving every
 * chain's x > 0 with ||x_c||_1 = 1; infos: nchains entries or NULL. */
bamg_status bamg_solve_batched(bamg_batch* b, double* x_dev, const bamg_solve_params* sp,
                               bamg_solve_info* infos, void* stream);
/* z = C r for every chain at once (one batched V-cycle). */
bamg_status bamg_vcycle_batched(bamg_batch* b, const double* r_dev, double* z_dev, void* stream);
/* offsets_host[nchains + 1]: start of chain c in the concatenated vectors. */
bamg_status bamg_batch_offsets(const bamg_batch* b, int64_t* offsets_host);
/* Lanes per row chosen by the autotuner for the batched B, P and Q of a level. */
bamg_status bamg_batch_lanes(const bamg_batch* b, int level, int* lanes_B, int* lanes_P, int* lanes_Q);
/* The hierarchy of chain c (owned by the batch; do not destroy it). */
bamg_hierarchy* bamg_batch_chain(const bamg_batch* b, int c);
void bamg_destroy_batched(bamg_batch* b);

/* ------------------------------------------------ learned interpolation --
 * Not in the paper: a small network proposes the weights that the
 * least-squares fits (eq. ls_interpolation; Section 5) compute, from the
 * local stencil of B.  The LS setup provides its training targets and stays
 * the fallback.
 *
 * Features of a fine point i of a geometric level (64 bf16 per point):
 * [0,25) b_{i,i+o}/b_ii and [25,50) b_{i+o,i}/b_ii over the 25 offsets o of
 * the 5x5 box (row-major, grid state s = gx*ny + gy, 0 outside the grid),
 * [50,58) 1 where the k-th neighbour of the 3x3 box (row-major, centre
 * skipped) is a coarse point, [58] = 1, [59,64) = 0.  Outputs (16 floats per
 * point): [0,8) P weights and [8,16) Q weights in the same 8 neighbour slots;
 * at setup the Q weights of a point are shifted by a common amount so that
 * they sum to one over J_i (the constraint of Section 5).
 * Network: 64 -> 64 -> 64 -> 16, ReLU after the two hidden layers.
 * Parameter vector (float, bamg_mlp_num_params() = 9360 entries):
 * W1[64][64], b1[64], W2[64][64], b2[64], W3[16][64], b3[16]; W[out][in].
 * Products run on the tensor cores with bf16 operands (weights, inputs and
 * hidden activations rounded to bf16) and fp32 accumulation. */
int bamg_mlp_num_params(void);
/* He-uniform weights from SplitMix64(seed, stream 8192), zero biases. */
bamg_status bamg_mlp_init(float* params_dev, uint64_t seed, void* stream);
/* Parameter files.  Layout (every field little-endian): the 8 bytes
 * "BAMGMLP1", the entry count as uint32 (= bamg_mlp_num_params()), the
 * 32-bit FNV-1a hash of the entry bytes as uint32, then the entries as IEEE
 * binary32 in the order above; nothing follows them.  `params` is device
 * memory when on_device != 0 (copied on `stream`, which is synchronised
 * before the call returns), else host memory; the caller owns it.
 * bamg_mlp_save writes (or replaces) the file at `path`.  bamg_mlp_load
 * fills params[0, bamg_mlp_num_params()) and leaves it untouched on any
 * error.  A file that cannot be opened, read or written, a wrong tag, count,
 * length or hash is BAMG_ERR_IO; a non-finite entry (in the file or in the
 * vector to save) is BAMG_ERR_NUMERIC. */
bamg_status bamg_mlp_save(const char* path, const float* params, int on_device, void* stream);
bamg_status bamg_mlp_load(const char* path, float* params, int on_device, void* stream);
/* Y[M][16] = network(X[M][64]); device arrays, X in bf16. */
bamg_status bamg_mlp_forward(const float* params_dev, int M, const void* X_bf16, float* Y, void* stream);
/* Loss = sum(mask * (Y - T)^2) / sum(mask) over the M rows and its gradient:
 * grad[9360] (device, overwritten), *loss_dev (device float, overwritten). */
bamg_status bamg_mlp_grad(const float* params_dev, int M, const void* X_bf16, const float* T,
                          const float* mask, float* grad, float* loss_dev, void* stream);
/* Adam (beta 0.9, 0.999, eps 1e-8) on minibatches of `batch` consecutive
 * rows for `epochs` passes; params updated in place; loss_host[epochs] (may
 * be NULL) receives the mean minibatch loss of each pass. */
bamg_status bamg_mlp_train(float* params_dev, int M, const void* X_bf16, const float* T, const float* mask,
                           int epochs, int batch, float lr, float* loss_host, void* stream);
/* Training rows of level `level` of an LS hierarchy (geometric): features X,
 * targets T (the LS weights of P and Q in the 8 slots) and mask (1 on the
 * slots of J_i), one row per fine point in ascending state order.  With
 * X_bf16 = NULL only *count (the number of fine points) is returned; else
 * capacity >= *count rows are required. */
bamg_status bamg_mlp_harvest(const bamg_hierarchy* h, int level, void* X_bf16, float* T, float* mask,
                             int capacity, int* count, void* stream);

/* Judge: asymptotic convergence factor of the stationary iteration
 * x <- x + C(-B x) with the hierarchy's V-cycle C, from `iters` (>= 2)
 * iterations started at x_i = 1 + 0.5 u_i (u from SplitMix64(seed, stream
 * 8193)): the geometric mean of the residual 1-norm ratios over the second
 * half of the run. */
bamg_status bamg_vcycle_factor(bamg_hierarchy* h, int iters, uint64_t seed, double* factor, void* stream);
/* Learned setup judged against a bound, with the LS setup as fallback:
 * builds the hierarchy with interp = BAMG_INTERP_MLP; if that fails
 * numerically or its V-cycle factor (bamg_vcycle_factor, 12 iterations)
 * exceeds max_factor, builds the LS hierarchy instead.  *used_ls = 1 when
 * the fallback was taken; *factor = the factor of the hierarchy returned
 * (measured for the learned one, -1 when the LS one was not judged). */
bamg_status bamg_setup_judged(const bamg_csr* A, const bamg_params* p, double max_factor, void* stream,
                              bamg_hierarchy** out, double* factor, int* used_ls);

/* ---------------------------------------------------------------- views --
 * Read-only views of the device arrays of a hierarchy, valid until
 * bamg_destroy.  Level 0 is the finest.  CSR arrays are int32 row_ptr[rows+1],
 * int32 col[nnz], double val[nnz]; P and Qt are n_l x n_{l+1} with fine rows
 * (Qt = Q^T), Q is n_{l+1} x n_l; M, N are NULL on level 0 (identity). */
typedef struct {
  int rows, cols, nnz;
  const int32_t* row_ptr;
  const int32_t* col;
  const double* val;
} bamg_csr_view;

typedef struct {
  int n;
  bamg_csr_view B, M, N, P, Qt, Q;   /* P, Qt, Q empty on the coarsest level */
  const int8_t* cf;                 /* 1 = coarse, 0 = fine (NULL on coarsest) */
  const int32_t* cmap;              /* coarse index or -1                      */
  const double* s;                  /* sqrt LS weights of V (r)                */
  const double* t;                  /* sqrt LS weights of U (r, t[0] = 0)      */
  int jacobi_l1_rows;               /* rows with b_ii <= 0 (l1 Jacobi divisor)  */
  const int32_t* colour;            /* multicolour smoother: colour of each row
                                       (NULL unless smoother = MCGS, and on the
                                       coarsest level)                         */
  int ncolours;
} bamg_level_view;

int bamg_num_levels(const bamg_hierarchy* h);
bamg_status bamg_level(const bamg_hierarchy* h, int l, bamg_level_view* out);

/* Setup triplets on the finest level: sigma (host, r doubles), and device
 * views of U, V (n x ld row-major, ld = block stride >= r) and x^(0).  A
 * hierarchy built with network fits carries no test vectors: U and V are
 * NULL and sigma holds the coarsest level's values. */
bamg_status bamg_triplets(const bamg_hierarchy* h, double* sigma_host, int* ld,
                          const double** U_dev, const double** V_dev,
                          const double** x0_dev);

/* Dense pseudo-inverse of the coarsest operator (n_L x n_L, row-major). */
bamg_status bamg_coarse_pinv(const bamg_hierarchy* h, int* nL, const double** Bpinv_dev);

#ifdef __cplusplus
}
#endif
#endif /* BAMG_H */
