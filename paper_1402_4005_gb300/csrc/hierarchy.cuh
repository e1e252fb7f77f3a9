// The multigrid hierarchy owned by a bamg_hierarchy handle.
#pragma once

#include <vector>

#include "internal.cuh"

namespace bamg {

struct Csr {
  int rows = 0, cols = 0, nnz = 0;
  int maxrow = -1;          // upper bound on the entries of a row (-1: unknown)
  DevMem rp, ci, va, va32;  // va32: float copy of the values (mixed precision)
  const int32_t* r() const { return rp.as<int32_t>(); }
  const int32_t* c() const { return ci.as<int32_t>(); }
  const double* v() const { return va.as<double>(); }
  template <typename T> const T* vals() const;
  bamg_status alloc(int rows_, int cols_, int nnz_, cudaStream_t s) {
    rows = rows_; cols = cols_; nnz = nnz_;
    BAMG_TRY(rp.alloc(sizeof(int32_t) * (rows + 1), s));
    BAMG_TRY(ci.alloc(sizeof(int32_t) * (nnz > 0 ? nnz : 1), s));
    return va.alloc(sizeof(double) * (nnz > 0 ? nnz : 1), s);
  }
  bamg_status make32(cudaStream_t s) {
    BAMG_TRY(va32.alloc(sizeof(float) * (nnz > 0 ? nnz : 1), s));
    return convert<double, float>((size_t)nnz, v(), va32.as<float>(), s);
  }
  // allocate the float copy and queue its conversion in `job` (one launch
  // for several matrices)
  bamg_status add32(ConvMany& job, cudaStream_t s) {
    BAMG_TRY(va32.alloc(sizeof(float) * (nnz > 0 ? nnz : 1), s));
    job.src[job.k] = v();
    job.dst[job.k] = va32.as<float>();
    job.n[job.k] = (size_t)nnz;
    ++job.k;
    return BAMG_OK;
  }
  bool empty() const { return rows == 0; }
};
template <> inline const double* Csr::vals<double>() const { return va.as<double>(); }
template <> inline const float* Csr::vals<float>() const { return va32.as<float>(); }

struct Level {
  int n = 0;
  int nx = 0, ny = 0;
  int nc = 0;             // coarse size (0 on the coarsest level)
  int vec_g = 4;          // lanes per row in the vector kernels (chosen from nnz/row)
  int nsafe = 0;          // rows with b_ii <= 0 whose Jacobi divisor is an l1 norm
  Csr B, Bt, M, N, P, Qt, Q, Pt;
  DevMem dinv, dinv32, dflags;
  DevMem cf, cmap, cpt, Jrp, Jci;
  DevMem s, t;            // sqrt LS weights (double[ld])
  // V-cycle vectors in the V-cycle precision
  DevMem vb, vz, vt, vr;
  // multicolour Gauss-Seidel smoother: colours, rows by colour, and the
  // colour offsets (host copy, ncol + 1 entries)
  DevMem colour, crows;
  std::vector<int32_t> crp;
  int ncol = 0;
};

}  // namespace bamg

namespace bamg {
struct GmresState;   // solve.cu: persistent FGMRES workspace and captured step
}

struct bamg_hierarchy {
  bamg_params p;
  int ld = 8;             // block stride (power of two >= r)
  int mixed = 0;
  int device = 0;
  cudaStream_t cap_stream = nullptr;   // private stream for graph capture
  std::vector<bamg::Level> lv;
  int nL = 0;
  bamg::DevMem Bpinv, Bpinv32;
  std::vector<double> sigma;            // setup triplets (finest level)
  bamg::DevMem U64, V64, x0;            // n x ld, n x ld, n
  bamg::DevMem io_in, io_out;           // V-cycle entry/exit (double)
  cudaGraph_t vgraph = nullptr;
  cudaGraphExec_t vexec = nullptr;
  uint64_t vgraph_kernels = 0;          // kernels per V-cycle graph launch
  double setup_ms = 0.0;
  double op_cplx = 0.0, grid_cplx = 0.0;
  int rankdef = 0;
  bamg::GmresState* gm = nullptr;       // FGMRES workspace (first solve)
  int prep_early = 0;                   // capture the V-cycle and Arnoldi graphs during the coarsest solve
  int learned = 0;                      // fits from the interpolation network
  bamg::DevMem mlp;                     // its parameters (float, copied at setup)
};

namespace bamg {
// z = C in (in: n doubles, or the column j = col[0] of an n-row array when col
// is given; with w given and j > 0 that column is first formed as w * rinv[0]
// and stored); z is written to out and, with out_col, to its column j.
template <typename T>
bamg_status vcycle_body(bamg_hierarchy* h, cudaStream_t s, double* in, const int* col, double* out,
                        double* out_col, const double* w, const double* rinv);
bamg_status vcycle_prepare(bamg_hierarchy* h, cudaStream_t s);
// solve.cu: FGMRES workspace and Arnoldi graph for the default restart
// (20), unpreconditioned = false; a solve with other settings re-captures
bamg_status gmres_prepare_default(bamg_hierarchy* h);
bamg_status vcycle_run(bamg_hierarchy* h, cudaStream_t s);
bamg_status promote_fp64(bamg_hierarchy* h, cudaStream_t s);
bamg_status fgmres(bamg_hierarchy* h, double* x, const bamg_solve_params* sp, bamg_solve_info* info,
                   cudaStream_t s);
bamg_status setup_finest(bamg_hierarchy* h, const bamg_csr* A, cudaStream_t s);
// abi.cu: bamg_setup, optionally without preparing the V-cycle (done lazily)
bamg_status setup_impl(const bamg_csr* A, const bamg_params* p, void* stream, bamg_hierarchy** out, bool prepare);
template <typename T> bamg_status run_setup(bamg_hierarchy* h, cudaStream_t s);
void gmres_release(bamg_hierarchy* h);
// mlp.cu: P rows and Q columns of a geometric level from the network
int mlp_num_params();
bamg_status mlp_fits(const Level& L, const float* params, double* fitP, double* fitQ, cudaStream_t s);
// solve.cu: asymptotic factor of the stationary iteration x <- x - C B x
bamg_status vcycle_factor(bamg_hierarchy* h, int iters, uint64_t seed, double* factor, cudaStream_t s);
}  // namespace bamg
