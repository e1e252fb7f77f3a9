// C ABI of libbamg: argument checking and dispatch.  No exception crosses
// this boundary and every call returns a bamg_status.
#include <chrono>
#include <cstring>
#include <new>

#include "hierarchy.cuh"

using namespace bamg;

namespace {
thread_local char g_status_buf[8] = "";
inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }
int block_ld(int r) {
  int ld = 4;
  while (ld < r) ld <<= 1;
  return ld;
}
double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
}  // namespace

namespace bamg {
const char* last_error_text();
}

extern "C" {

bamg_status bamg_params_default(bamg_params* p) {
  if (!p) return BAMG_ERR_ARG;
  std::memset(p, 0, sizeof(*p));
  p->r = 8;
  p->max_levels = 25;
  p->coarse_min = 300;
  p->nu_setup = 5;
  p->nu_pre = 3;
  p->nu_post = 3;
  p->c_min = 1;
  p->c_max = 4;
  p->omega = 0.7;
  p->coarsening = BAMG_COARSEN_GEOMETRIC;
  p->precision = BAMG_PREC_FP64;
  p->restriction = BAMG_RESTRICT_LS;
  p->seed = 1;
  p->stochastic_tol = 1e-12;
  p->max_coarse_dense = 1024;
  p->setup_cycles = 1;
  return BAMG_OK;
}

bamg_status bamg_solve_params_default(bamg_solve_params* p) {
  if (!p) return BAMG_ERR_ARG;
  p->restart = 20;
  p->max_iter = 500;
  p->tol = 1e-10;
  p->plain = 0;
  return BAMG_OK;
}

const char* bamg_status_string(bamg_status s) {
  switch (s) {
    case BAMG_OK: return "ok";
    case BAMG_ERR_ARG: return "invalid argument";
    case BAMG_ERR_NOT_STOCHASTIC: return "matrix is not column stochastic";
    case BAMG_ERR_CUDA: return "CUDA error";
    case BAMG_ERR_OOM: return "out of device memory";
    case BAMG_ERR_NOT_CONVERGED: return "not converged";
    case BAMG_ERR_BREAKDOWN: return "GMRES breakdown";
    case BAMG_ERR_NUMERIC: return "numerical failure";
    case BAMG_ERR_TIMEOUT: return "device wait timed out";
    case BAMG_ERR_UNSUPPORTED: return "unsupported request";
    case BAMG_ERR_IO: return "file error";
  }
  return "unknown status";
}

const char* bamg_last_error(void) { return bamg::last_error_text(); }

uint64_t bamg_launch_count(void) { return g_launches.load(); }

static bamg_status check_params(const bamg_csr* A, const bamg_params* p) {
  BAMG_CHECK_ARG(A && p);
  BAMG_CHECK_ARG(A->n >= 1 && A->n <= INT32_MAX - 1 && A->nnz >= 0 && A->nnz <= INT32_MAX);
  BAMG_CHECK_ARG(A->row_ptr && (A->nnz == 0 || (A->col_idx && A->val)));
  BAMG_CHECK_ARG(p->r >= 1 && p->r <= 32);
  BAMG_CHECK_ARG(p->max_levels >= 1 && p->max_levels <= 64 && p->coarse_min >= 1);
  BAMG_CHECK_ARG(p->nu_setup >= 0 && p->nu_pre >= 0 && p->nu_post >= 0);
  BAMG_CHECK_ARG(p->omega > 0.0 && p->omega < 2.0);
  BAMG_CHECK_ARG(p->coarsening == BAMG_COARSEN_GEOMETRIC || p->coarsening == BAMG_COARSEN_MIS);
  BAMG_CHECK_ARG(p->precision == BAMG_PREC_FP64 || p->precision == BAMG_PREC_MIXED);
  BAMG_CHECK_ARG(p->restriction == BAMG_RESTRICT_LS || p->restriction == BAMG_RESTRICT_AVERAGE);
  BAMG_CHECK_ARG(p->c_min >= 1 && p->c_max >= p->c_min && p->c_max <= 8 && p->c_max <= block_ld(p->r));
  BAMG_CHECK_ARG(p->stochastic_tol >= 0.0);
  BAMG_CHECK_ARG(p->max_coarse_dense >= 1 && p->max_coarse_dense <= 1024);
  if (p->coarsening == BAMG_COARSEN_GEOMETRIC)
    BAMG_CHECK_ARG(A->nx >= 1 && A->ny >= 1 && (int64_t)A->nx * A->ny == A->n);
  BAMG_CHECK_ARG(p->interp == BAMG_INTERP_LS || p->interp == BAMG_INTERP_MLP);
  BAMG_CHECK_ARG(p->setup_cycles >= 1 && p->setup_cycles <= 8);
  BAMG_CHECK_ARG(p->interp == BAMG_INTERP_LS || p->setup_cycles == 1);
  BAMG_CHECK_ARG(p->smoother == BAMG_SMOOTH_JACOBI || p->smoother == BAMG_SMOOTH_MCGS);
  BAMG_CHECK_ARG(p->ls_ridge >= 0.0 && p->ls_ridge < 1e300);
  if (p->interp == BAMG_INTERP_MLP) {
    BAMG_CHECK_ARG(p->mlp_params != nullptr);
    if (p->coarsening != BAMG_COARSEN_GEOMETRIC) {
      set_error("network fits need geometric coarsening (grid-offset features)");
      return BAMG_ERR_UNSUPPORTED;
    }
  }
  return BAMG_OK;
}

}  // extern "C"

namespace bamg {
// prepare = false leaves the V-cycle's vectors and graph to the first
// V-cycle, FGMRES or factor call (batched setups, whose chains are solved
// through the batch's own V-cycle)
bamg_status setup_impl(const bamg_csr* A, const bamg_params* p, void* stream, bamg_hierarchy** out, bool prepare) {
  if (!out) return BAMG_ERR_ARG;
  *out = nullptr;
  BAMG_TRY(check_params(A, p));
  bamg_hierarchy* h = new (std::nothrow) bamg_hierarchy();
  if (!h) return BAMG_ERR_OOM;
  h->p = *p;
  h->ld = block_ld(p->r);
  h->mixed = p->precision == BAMG_PREC_MIXED;
  h->lv.reserve(64);
  cudaStream_t s = S(stream);
  double t0 = now_ms();
  bamg_status st = BAMG_OK;
  // every kernel of the library waits for its predecessor before it touches
  // memory (pdl_wait() first, or after loads of data written before the
  // setup), so the setup's chains of small kernels launch with programmatic
  // serialisation and each launch overlaps the previous kernel
  PdlScope pdl;
  // temporaries released during the setup serve its later allocations
  AllocScope cache;
  do {
    if (cudaGetDevice(&h->device) != cudaSuccess) { st = BAMG_ERR_CUDA; break; }
    configure_pool(h->device);
    if (p->interp == BAMG_INTERP_MLP) {
      h->learned = 1;
      size_t bytes = sizeof(float) * mlp_num_params();
      st = h->mlp.alloc(bytes, s);
      if (st != BAMG_OK) break;
      if (cudaMemcpyAsync(h->mlp.p, p->mlp_params, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        set_error("copy of the network parameters failed");
        st = BAMG_ERR_CUDA;
        break;
      }
    }
    h->prep_early = prepare ? 1 : 0;
    st = setup_finest(h, A, s);
    if (st != BAMG_OK) break;
    st = h->mixed ? run_setup<float>(h, s) : run_setup<double>(h, s);
    if (st != BAMG_OK) break;
    if (h->nL > p->max_coarse_dense) {
      set_error("coarsest level has %d points, above max_coarse_dense = %d", h->nL, p->max_coarse_dense);
      st = BAMG_ERR_UNSUPPORTED;
      break;
    }
    if (prepare) {
      st = vcycle_prepare(h, s);
      if (st != BAMG_OK) break;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) { st = BAMG_ERR_CUDA; break; }
  } while (false);
  if (st != BAMG_OK) {
    cudaStreamSynchronize(s);
    bamg_destroy(h);
    return st;
  }
  h->setup_ms = now_ms() - t0;
  *out = h;
  return BAMG_OK;
}
}  // namespace bamg

extern "C" {

bamg_status bamg_setup(const bamg_csr* A, const bamg_params* p, void* stream, bamg_hierarchy** out) {
  return setup_impl(A, p, stream, out, true);
}

bamg_status bamg_vcycle(bamg_hierarchy* h, const double* r_dev, double* z_dev, void* stream) {
  BAMG_CHECK_ARG(h && r_dev && z_dev && r_dev != z_dev);
  cudaStream_t s = S(stream);
  BAMG_TRY(vcycle_prepare(h, s));
  size_t n = h->lv[0].n;
  BAMG_CUDA(cudaMemcpyAsync(h->io_in.p, r_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  BAMG_TRY(vcycle_run(h, s));
  BAMG_CUDA(cudaMemcpyAsync(z_dev, h->io_out.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  return BAMG_OK;
}

bamg_status bamg_vcycle_factor(bamg_hierarchy* h, int iters, uint64_t seed, double* factor, void* stream) {
  BAMG_CHECK_ARG(h && factor && iters >= 2 && iters <= 10000);
  return vcycle_factor(h, iters, seed, factor, S(stream));
}

bamg_status bamg_setup_judged(const bamg_csr* A, const bamg_params* p, double max_factor, void* stream,
                              bamg_hierarchy** out, double* factor, int* used_ls) {
  BAMG_CHECK_ARG(out && p && factor && used_ls && p->interp == BAMG_INTERP_MLP);
  *out = nullptr;
  *used_ls = 0;
  *factor = -1.0;
  bamg_hierarchy* h = nullptr;
  bamg_status st = bamg_setup(A, p, stream, &h);
  if (st == BAMG_OK) {
    double f = 0.0;
    st = vcycle_factor(h, 12, p->seed, &f, S(stream));
    if (st == BAMG_OK && f <= max_factor) {
      *out = h;
      *factor = f;
      return BAMG_OK;
    }
    bamg_destroy(h);
    if (st != BAMG_OK) return st;
  } else if (st != BAMG_ERR_NUMERIC) {
    return st;
  }
  // fallback: the least-squares fits
  bamg_params q = *p;
  q.interp = BAMG_INTERP_LS;
  q.mlp_params = nullptr;
  st = bamg_setup(A, &q, stream, out);
  if (st == BAMG_OK) *used_ls = 1;
  return st;
}

bamg_status bamg_solve(bamg_hierarchy* h, double* x_dev, const bamg_solve_params* sp, bamg_solve_info* info,
                       void* stream) {
  BAMG_CHECK_ARG(h && x_dev && sp);
  BAMG_CHECK_ARG(sp->restart >= 1 && sp->restart <= 64 && sp->max_iter >= 1 && sp->tol > 0.0);
  double t0 = now_ms();
  bamg_solve_info tmp;
  std::memset(&tmp, 0, sizeof(tmp));
  bamg_status st = fgmres(h, x_dev, sp, &tmp, S(stream));
  if ((st == BAMG_ERR_NOT_CONVERGED || st == BAMG_ERR_BREAKDOWN) && h->mixed && !sp->plain) {
    // the FP32 V-cycle stalled: continue from the current x with FP64 V-cycles
    const int mixed_its = tmp.iterations;
    bamg_status pr = promote_fp64(h, S(stream));
    if (pr == BAMG_OK)
      pr = cudaMemcpyAsync(h->x0.p, x_dev, sizeof(double) * h->lv[0].n, cudaMemcpyDeviceToDevice, S(stream)) ==
                   cudaSuccess
               ? BAMG_OK
               : BAMG_ERR_CUDA;
    if (pr != BAMG_OK) {
      st = pr;
    } else {
      st = fgmres(h, x_dev, sp, &tmp, S(stream));
      tmp.iterations += mixed_its;
      tmp.fallback_iterations = mixed_its;
      if (tmp.iters_to_1e7 >= 0) tmp.iters_to_1e7 += mixed_its;
    }
  }
  cudaStreamSynchronize(S(stream));
  tmp.solve_ms = now_ms() - t0;
  tmp.setup_ms = h->setup_ms;
  tmp.levels = (int)h->lv.size();
  tmp.op_cplx = h->op_cplx;
  tmp.grid_cplx = h->grid_cplx;
  if (info) *info = tmp;
  return st;
}

bamg_status bamg_solve_host(const bamg_csr* A, const bamg_params* p, const bamg_solve_params* sp,
                            double* x_host, bamg_solve_info* info, void* stream) {
  BAMG_CHECK_ARG(A && p && sp && x_host);
  bamg_hierarchy* h = nullptr;
  BAMG_TRY(bamg_setup(A, p, stream, &h));
  cudaStream_t s = S(stream);
  DevMem x;
  bamg_status st = x.alloc(sizeof(double) * A->n, s);
  if (st == BAMG_OK) {
    st = bamg_solve(h, x.as<double>(), sp, info, stream);
    if (st == BAMG_OK || st == BAMG_ERR_NOT_CONVERGED) {
      cudaError_t e = cudaMemcpyAsync(x_host, x.p, sizeof(double) * A->n, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        set_error("copy of x to the host failed: %s", cudaGetErrorString(e));
        st = BAMG_ERR_CUDA;
      }
    }
  }
  x.release();
  bamg_destroy(h);
  return st;
}

void bamg_destroy(bamg_hierarchy* h) {
  if (!h) return;
  gmres_release(h);
  if (h->vexec) cudaGraphExecDestroy(h->vexec);
  if (h->vgraph) cudaGraphDestroy(h->vgraph);
  if (h->cap_stream) {
    cudaStreamSynchronize(h->cap_stream);
    cudaStreamDestroy(h->cap_stream);
  }
  delete h;
}

int bamg_num_levels(const bamg_hierarchy* h) { return h ? (int)h->lv.size() : 0; }

static bamg_csr_view view_of(const Csr& A) {
  bamg_csr_view v;
  v.rows = A.rows; v.cols = A.cols; v.nnz = A.nnz;
  v.row_ptr = A.rows ? A.r() : nullptr;
  v.col = A.rows ? A.c() : nullptr;
  v.val = A.rows ? A.v() : nullptr;
  return v;
}

bamg_status bamg_level(const bamg_hierarchy* h, int l, bamg_level_view* out) {
  BAMG_CHECK_ARG(h && out && l >= 0 && l < (int)h->lv.size());
  const Level& L = h->lv[l];
  out->n = L.n;
  out->B = view_of(L.B);
  out->M = view_of(L.M);
  out->N = view_of(L.N);
  out->P = view_of(L.P);
  out->Qt = view_of(L.Qt);
  out->Q = view_of(L.Q);
  out->cf = L.cf.as<int8_t>();
  out->cmap = L.cmap.as<int32_t>();
  out->s = L.s.as<double>();
  out->t = L.t.as<double>();
  out->jacobi_l1_rows = L.nsafe;
  out->colour = L.ncol > 0 ? L.colour.as<int32_t>() : nullptr;
  out->ncolours = L.ncol;
  return BAMG_OK;
}

bamg_status bamg_triplets(const bamg_hierarchy* h, double* sigma_host, int* ld, const double** U_dev,
                          const double** V_dev, const double** x0_dev) {
  BAMG_CHECK_ARG(h);
  if (sigma_host) std::memcpy(sigma_host, h->sigma.data(), sizeof(double) * h->sigma.size());
  if (ld) *ld = h->ld;
  if (U_dev) *U_dev = h->U64.as<double>();
  if (V_dev) *V_dev = h->V64.as<double>();
  if (x0_dev) *x0_dev = h->x0.as<double>();
  return BAMG_OK;
}

bamg_status bamg_coarse_pinv(const bamg_hierarchy* h, int* nL, const double** Bpinv_dev) {
  BAMG_CHECK_ARG(h && nL && Bpinv_dev);
  *nL = h->nL;
  *Bpinv_dev = h->Bpinv.as<double>();
  return BAMG_OK;
}

// ------------------------------------------------------------------- steps
bamg_status bamg_step_build_B_count(int n, const int32_t* A_rp, const int32_t* A_ci, int64_t* nnzB,
                                    void* stream) {
  BAMG_CHECK_ARG(n >= 1 && A_rp && A_ci && nnzB);
  cudaStream_t s = S(stream);
  DevMem cnt, rp;
  BAMG_TRY(cnt.alloc(sizeof(int32_t) * (n + 1), s));
  BAMG_TRY(rp.alloc(sizeof(int32_t) * (n + 1), s));
  BAMG_TRY(build_B_count(n, A_rp, A_ci, cnt.as<int32_t>(), s));
  return scan_counts(cnt.as<int32_t>(), rp.as<int32_t>(), n, s, nnzB);
}

bamg_status bamg_step_build_B(int n, const int32_t* A_rp, const int32_t* A_ci, const double* A_val,
                              int32_t* B_rp, int32_t* B_ci, double* B_val, void* stream) {
  BAMG_CHECK_ARG(n >= 1 && A_rp && A_ci && A_val && B_rp && B_ci && B_val);
  cudaStream_t s = S(stream);
  DevMem cnt;
  BAMG_TRY(cnt.alloc(sizeof(int32_t) * (n + 1), s));
  BAMG_TRY(build_B_count(n, A_rp, A_ci, cnt.as<int32_t>(), s));
  BAMG_TRY(scan_counts(cnt.as<int32_t>(), B_rp, n, s, nullptr));
  return build_B_fill(n, A_rp, A_ci, A_val, B_rp, B_ci, B_val, s);
}

bamg_status bamg_step_check_stochastic(int n, const int32_t* A_rp, const int32_t* A_ci, const double* A_val,
                                       double tol, int64_t* bad_host, void* stream) {
  BAMG_CHECK_ARG(n >= 1 && A_rp && A_ci && A_val && bad_host);
  return check_stochastic(n, A_rp, A_ci, A_val, tol, bad_host, S(stream));
}

bamg_status bamg_step_transpose(int rows, int cols, int nnz, const int32_t* rp, const int32_t* ci,
                                const double* val, int32_t* t_rp, int32_t* t_ci, double* t_val, void* stream) {
  BAMG_CHECK_ARG(rows >= 1 && cols >= 1 && nnz >= 0 && rp && ci && t_rp && t_ci);
  return transpose_csr(rows, cols, nnz, rp, ci, val, t_rp, t_ci, t_val, S(stream));
}

bamg_status bamg_step_relax_block(int prec, int n, int ld, const int32_t* rp, const int32_t* ci, const void* val,
                                  const void* dinv, const void* X, void* Y, const void* R, const void* sigma,
                                  double omega, int keep_col0, void* stream) {
  BAMG_CHECK_ARG(n >= 1 && rp && ci && val && dinv && X && Y && X != Y && (prec == 0 || prec == 1));
  if (prec == 1)
    return relax_block<float>(n, ld, rp, ci, (const float*)val, (const float*)dinv, (const float*)X, (float*)Y,
                              (const float*)R, (const float*)sigma, (float)omega, keep_col0, S(stream));
  return relax_block<double>(n, ld, rp, ci, (const double*)val, (const double*)dinv, (const double*)X,
                             (double*)Y, (const double*)R, (const double*)sigma, omega, keep_col0, S(stream));
}

bamg_status bamg_step_jacobi_divisor(int n, const int32_t* rp, const int32_t* ci, const double* val,
                                     const int32_t* trp, const double* tval, double* dinv, int* nsafe_host,
                                     void* stream) {
  BAMG_CHECK_ARG(n >= 1 && rp && ci && val && trp && tval && dinv && nsafe_host);
  cudaStream_t s = S(stream);
  DevMem flags;
  BAMG_TRY(flags.alloc(2 * sizeof(int), s));
  int init[2] = {INT32_MAX, 0};
  BAMG_CUDA(cudaMemcpyAsync(flags.p, init, sizeof(init), cudaMemcpyHostToDevice, s));
  BAMG_TRY(diag_inv<double>(n, rp, ci, val, trp, tval, dinv, flags.as<int>(), flags.as<int>() + 1, s));
  int hf[2] = {0, 0};
  BAMG_CUDA(cudaMemcpyAsync(hf, flags.p, sizeof(hf), cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  *nsafe_host = hf[1];
  if (hf[0] != INT32_MAX) {
    set_error("row and column %d are zero", hf[0]);
    return BAMG_ERR_NUMERIC;
  }
  return BAMG_OK;
}

bamg_status bamg_step_spmm_block(int prec, int rows, int ld, const int32_t* rp, const int32_t* ci,
                                 const void* val, const void* X, void* Y, void* stream) {
  BAMG_CHECK_ARG(rows >= 1 && rp && ci && val && X && Y && (prec == 0 || prec == 1));
  if (prec == 1)
    return spmm_block<float>(rows, ld, rp, ci, (const float*)val, (const float*)X, (float*)Y, S(stream));
  return spmm_block<double>(rows, ld, rp, ci, (const double*)val, (const double*)X, (double*)Y, S(stream));
}

bamg_status bamg_step_csr_vec(int prec, int mode, int n, int64_t nnz, const int32_t* rp, const int32_t* ci,
                              const void* val, const void* dinv, double omega, const void* x, const void* b,
                              void* y, void* stream) {
  BAMG_CHECK_ARG(n >= 1 && nnz >= 0 && rp && ci && val && y && (prec == 0 || prec == 1));
  BAMG_CHECK_ARG(mode >= VEC_JACOBI && mode <= VEC_JACOBI_ZERO2);
  BAMG_CHECK_ARG(mode == VEC_SPMV || mode == VEC_SPMV_ADD || b);
  BAMG_CHECK_ARG(mode == VEC_JACOBI_ZERO || mode == VEC_JACOBI_ZERO2 || x);
  BAMG_CHECK_ARG((mode != VEC_JACOBI && mode != VEC_JACOBI_ZERO && mode != VEC_JACOBI_ZERO2) || dinv);
  const int G = vec_lanes((double)nnz / n);
  if (prec == 1)
    return csr_vec<float>(mode, n, G, rp, ci, (const float*)val, (const float*)dinv, (float)omega,
                          (const float*)x, (const float*)b, (float*)y, S(stream));
  return csr_vec<double>(mode, n, G, rp, ci, (const double*)val, (const double*)dinv, omega, (const double*)x,
                         (const double*)b, (double*)y, S(stream));
}

bamg_status bamg_step_norms_weights(int prec, int n, int ld, int r, const int32_t* rp, const int32_t* ci,
                                    const void* val, void* X, int normalise, int skip_col0, double* norm_host,
                                    double* w_host, void* stream) {
  BAMG_CHECK_ARG(n >= 1 && r >= 1 && r <= ld && rp && ci && val && X && norm_host && w_host);
  cudaStream_t s = S(stream);
  DevMem scale, w, nr;
  BAMG_TRY(scale.alloc(sizeof(double) * ld, s));
  BAMG_TRY(w.alloc(sizeof(double) * ld, s));
  BAMG_TRY(nr.alloc(sizeof(double) * ld, s));
  if (prec == 1)
    BAMG_TRY(norms_weights<float>(n, ld, r, rp, ci, (const float*)val, (float*)X, normalise, skip_col0,
                                  scale.as<float>(), w.as<double>(), nr.as<double>(), s));
  else
    BAMG_TRY(norms_weights<double>(n, ld, r, rp, ci, (const double*)val, (double*)X, normalise, skip_col0,
                                   scale.as<double>(), w.as<double>(), nr.as<double>(), s));
  BAMG_CUDA(cudaMemcpyAsync(norm_host, nr.p, sizeof(double) * r, cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaMemcpyAsync(w_host, w.p, sizeof(double) * r, cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  return BAMG_OK;
}

bamg_status bamg_step_coarsen_geometric(int nx, int ny, int8_t* cf, int32_t* cmap, int32_t* J_rp, int32_t* J_ci,
                                        int* nc_host, void* stream) {
  BAMG_CHECK_ARG(nx >= 1 && ny >= 1 && cf && cmap && J_rp && J_ci);
  return coarsen_geometric(nx, ny, cf, cmap, J_rp, J_ci, nc_host, S(stream));
}

bamg_status bamg_step_coarsen_mis(int n, const int32_t* B_rp, const int32_t* B_ci, const int32_t* Bt_rp,
                                  const int32_t* Bt_ci, uint64_t seed, int level, int8_t* cf, int32_t* cmap,
                                  int* nc_host, void* stream) {
  BAMG_CHECK_ARG(n >= 1 && B_rp && B_ci && Bt_rp && Bt_ci && cf && cmap && level >= 0);
  return coarsen_mis(n, B_rp, B_ci, Bt_rp, Bt_ci, seed, level, cf, cmap, nc_host, S(stream));
}

bamg_status bamg_step_colour(int n, const int32_t* B_rp, const int32_t* B_ci, const int32_t* Bt_rp,
                             const int32_t* Bt_ci, uint64_t seed, int level, int32_t* colour, int* ncolours_host,
                             void* stream) {
  BAMG_CHECK_ARG(n >= 1 && B_rp && B_ci && Bt_rp && Bt_ci && colour && ncolours_host && level >= 0);
  return colour_graph(n, B_rp, B_ci, Bt_rp, Bt_ci, seed, level, colour, ncolours_host, S(stream));
}

bamg_status bamg_step_colour_rows(int n, const int32_t* colour, int ncolours, int32_t* colour_rp_host,
                                  int32_t* rows, void* stream) {
  BAMG_CHECK_ARG(n >= 1 && colour && ncolours >= 1 && colour_rp_host && rows);
  bamg_status st = colour_rows(n, colour, ncolours, colour_rp_host, rows, S(stream));
  if (st == BAMG_OK && cudaStreamSynchronize(S(stream)) != cudaSuccess) return BAMG_ERR_CUDA;
  return st;
}

bamg_status bamg_step_mcgs_sweep(int prec, int n, const int32_t* rp, const int32_t* ci, const void* val,
                                 const void* dinv, int ncolours, const int32_t* colour_rp_host, const int32_t* rows,
                                 const void* b, void* x, void* stream) {
  BAMG_CHECK_ARG(n >= 1 && rp && ci && val && dinv && ncolours >= 1 && colour_rp_host && rows && b && x);
  BAMG_CHECK_ARG(colour_rp_host[0] == 0 && colour_rp_host[ncolours] == n && (prec == 0 || prec == 1));
  for (int c = 0; c < ncolours; ++c) BAMG_CHECK_ARG(colour_rp_host[c + 1] >= colour_rp_host[c]);
  const int G = 4;
  if (prec == 1)
    return mcgs_sweep<float>(G, ncolours, colour_rp_host, rows, rp, ci, (const float*)val, (const float*)dinv,
                             (const float*)b, (float*)x, S(stream));
  return mcgs_sweep<double>(G, ncolours, colour_rp_host, rows, rp, ci, (const double*)val, (const double*)dinv,
                            (const double*)b, (double*)x, S(stream));
}

bamg_status bamg_step_graph_sets(int n, const int32_t* B_rp, const int32_t* B_ci, const double* B_val,
                                 const int32_t* Bt_rp, const int32_t* Bt_ci, const double* Bt_val, const int8_t* cf,
                                 int c_min, int c_max, int32_t* J_rp, int32_t* J_ci, void* stream) {
  BAMG_CHECK_ARG(n >= 1 && B_rp && B_ci && B_val && Bt_rp && Bt_ci && Bt_val && cf && J_rp && J_ci);
  return graph_sets(n, B_rp, B_ci, B_val, Bt_rp, Bt_ci, Bt_val, cf, c_min, c_max, J_rp, J_ci, S(stream));
}

bamg_status bamg_step_ls_fit(int prec, int n, int ld, int r, const int32_t* J_rp, const int32_t* J_ci,
                             const void* X, const double* w, int constrained, double ridge, double* out,
                             int* rankdef_host, void* stream) {
  BAMG_CHECK_ARG(n >= 1 && r >= 1 && r <= ld && J_rp && J_ci && X && w && out);
  BAMG_CHECK_ARG(ridge >= 0.0 && ridge < 1e300);
  cudaStream_t s = S(stream);
  DevMem rk;
  BAMG_TRY(rk.alloc(2 * sizeof(int), s));
  BAMG_CUDA(cudaMemsetAsync(rk.p, 0, 2 * sizeof(int), s));
  if (prec == 1)
    BAMG_TRY(ls_fit<float>(n, ld, r, J_rp, J_ci, (const float*)X, w, constrained, out, rk.as<int>(), s, ridge));
  else
    BAMG_TRY(ls_fit<double>(n, ld, r, J_rp, J_ci, (const double*)X, w, constrained, out, rk.as<int>(), s, ridge));
  int h[2] = {0, 0};
  BAMG_CUDA(cudaMemcpyAsync(h, rk.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  if (rankdef_host) *rankdef_host = h[0];
  if (h[1] > 0) {
    set_error("%d interpolation sets exceed min(ld, 8) = %d entries", h[1], ld < 8 ? ld : 8);
    return BAMG_ERR_ARG;
  }
  return BAMG_OK;
}

bamg_status bamg_step_spgemm_symbolic(int m, const int32_t* A_rp, const int32_t* A_ci, const int32_t* B_rp,
                                      const int32_t* B_ci, int32_t* C_rp, int64_t* nnzC_host, void* stream) {
  BAMG_CHECK_ARG(m >= 1 && A_rp && A_ci && B_rp && B_ci && C_rp && nnzC_host);
  return spgemm_symbolic(m, A_rp, A_ci, B_rp, B_ci, C_rp, nnzC_host, S(stream));
}

bamg_status bamg_step_spgemm_numeric(int m, const int32_t* A_rp, const int32_t* A_ci, const double* A_val,
                                     const int32_t* B_rp, const int32_t* B_ci, const double* B_val,
                                     const int32_t* C_rp, int32_t* C_ci, double* C_val, void* stream) {
  BAMG_CHECK_ARG(m >= 1 && A_rp && A_ci && A_val && B_rp && B_ci && B_val && C_rp && C_ci && C_val);
  return spgemm_numeric(m, A_rp, A_ci, A_val, B_rp, B_ci, B_val, C_rp, C_ci, C_val, S(stream));
}

bamg_status bamg_step_coarsest(int prec, int n, int r, const double* B, const double* M, const double* N,
                               double* sigma, double* U, double* V, double* Bpinv, void* stream) {
  BAMG_CHECK_ARG(B && M && N && sigma && U && V && (prec == 0 || prec == 1));
  return coarsest_solve(prec, n, r, B, M, N, sigma, U, V, Bpinv, S(stream));
}

}  // extern "C"
