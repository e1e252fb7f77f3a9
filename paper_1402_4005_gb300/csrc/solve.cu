// Solve phase (Section 6): V-cycle preconditioner and flexible GMRES.
//
// V-cycle (Section 3, eq. error_propagator_twogrid): from z = 0, nu_pre
// weighted-Jacobi sweeps (or multicolour Gauss-Seidel sweeps), residual,
// r_c = Q r, recursion (B_L^+ r_L on the coarsest level), z += P e_c,
// nu_post sweeps.  It runs in the hierarchy's V-cycle precision (FP64, or
// FP32 in mixed mode) and is captured once into a CUDA graph that reads a
// fixed FP64 input buffer and writes a fixed FP64 output buffer.  A mixed
// hierarchy can be switched to FP64 V-cycles (promote_fp64) when its solve
// stalls.
//
// GMRES on the residual equation B e = -B x^(0) (eq. residual), written as
// B x = 0 from x^(0).  The V-cycle is applied on the right (flexible GMRES,
// which admits a preconditioner computed in lower precision); Arnoldi uses
// classical Gram-Schmidt with one re-orthogonalisation, Givens rotations and
// the small triangular solve run on the device in FP64.  The stopping rule
// is the true ||B x||_1 / ||x||_1, evaluated whenever the 2-norm estimate
// allows it to hold.  With the identity in place of the V-cycle and the
// uniform start vector the same code is the unpreconditioned GMRES(m) the
// paper compares against (Section 7).
#include <chrono>
#include <cmath>
#include <new>
#include <vector>

#include "hierarchy.cuh"

namespace bamg {

static int lanes_for(const Csr& A) {
  return vec_lanes(A.rows ? (double)A.nnz / A.rows : 1.0);
}

template <typename T> static const T* dinv_t(const Level& L);
template <> const double* dinv_t<double>(const Level& L) { return L.dinv.as<double>(); }
template <> const float* dinv_t<float>(const Level& L) { return L.dinv32.as<float>(); }
template <typename T> static const T* pinv_t(const bamg_hierarchy* h);
template <> const double* pinv_t<double>(const bamg_hierarchy* h) { return h->Bpinv.as<double>(); }
template <> const float* pinv_t<float>(const bamg_hierarchy* h) { return h->Bpinv32.as<float>(); }

template <typename T>
static bamg_status vcycle_level(bamg_hierarchy* h, int l, cudaStream_t s) {
  Level& L = h->lv[l];
  T* b = L.vb.as<T>();
  T* z = L.vz.as<T>();
  if (l == (int)h->lv.size() - 1) return dense_gemv<T>(L.n, pinv_t<T>(h), b, z, s);
  const bamg_params& p = h->p;
  const T om = T(p.omega);
  const T* dv = dinv_t<T>(L);
  const T* bv = L.B.vals<T>();
  T* cur = z;
  T* alt = L.vt.as<T>();
  if (p.smoother == BAMG_SMOOTH_MCGS) {
    // multicolour Gauss-Seidel, in place (Section 3 splitting)
    auto sweep = [&](T* x) {
      return mcgs_sweep<T>(L.vec_g, L.ncol, L.crp.data(), L.crows.as<int32_t>(), L.B.r(), L.B.c(), bv, dv, b, x, s);
    };
    BAMG_CUDA(cudaMemsetAsync(z, 0, sizeof(T) * L.n, s));
    for (int it = 0; it < p.nu_pre; ++it) BAMG_TRY(sweep(z));
    BAMG_TRY(csr_vec<T>(VEC_RESID, L.n, L.vec_g, L.B.r(), L.B.c(), bv, dv, om, z, b, L.vr.as<T>(), s));
    Level& C = h->lv[l + 1];
    BAMG_TRY(csr_vec<T>(VEC_SPMV, L.nc, lanes_for(L.Q), L.Q.r(), L.Q.c(), L.Q.vals<T>(), dv, om, L.vr.as<T>(),
                        nullptr, C.vb.as<T>(), s));
    BAMG_TRY(vcycle_level<T>(h, l + 1, s));
    BAMG_TRY(csr_vec<T>(VEC_SPMV_ADD, L.n, lanes_for(L.P), L.P.r(), L.P.c(), L.P.vals<T>(), dv, om,
                        C.vz.as<T>(), nullptr, z, s));
    for (int it = 0; it < p.nu_post; ++it) BAMG_TRY(sweep(z));
    return BAMG_OK;
  }
  if (p.nu_pre == 0) {
    BAMG_CUDA(cudaMemsetAsync(cur, 0, sizeof(T) * L.n, s));
  } else {
    BAMG_TRY(csr_vec<T>(VEC_JACOBI_ZERO, L.n, L.vec_g, L.B.r(), L.B.c(), bv, dv, om, nullptr, b, cur, s));
    for (int it = 1; it < p.nu_pre; ++it) {
      BAMG_TRY(csr_vec<T>(VEC_JACOBI, L.n, L.vec_g, L.B.r(), L.B.c(), bv, dv, om, cur, b, alt, s));
      std::swap(cur, alt);
    }
  }
  BAMG_TRY(csr_vec<T>(VEC_RESID, L.n, L.vec_g, L.B.r(), L.B.c(), bv, dv, om, cur, b, L.vr.as<T>(), s));
  Level& C = h->lv[l + 1];
  BAMG_TRY(csr_vec<T>(VEC_SPMV, L.nc, lanes_for(L.Q), L.Q.r(), L.Q.c(), L.Q.vals<T>(), dv, om, L.vr.as<T>(),
                      nullptr, C.vb.as<T>(), s));
  BAMG_TRY(vcycle_level<T>(h, l + 1, s));
  BAMG_TRY(csr_vec<T>(VEC_SPMV_ADD, L.n, lanes_for(L.P), L.P.r(), L.P.c(), L.P.vals<T>(), dv, om,
                      C.vz.as<T>(), nullptr, cur, s));
  for (int it = 0; it < p.nu_post; ++it) {
    BAMG_TRY(csr_vec<T>(VEC_JACOBI, L.n, L.vec_g, L.B.r(), L.B.c(), bv, dv, om, cur, b, alt, s));
    std::swap(cur, alt);
  }
  if (cur != z) BAMG_CUDA(cudaMemcpyAsync(z, cur, sizeof(T) * L.n, cudaMemcpyDeviceToDevice, s));
  return BAMG_OK;
}

__global__ void copy_d_kernel(size_t n, const double* __restrict__ a, double* __restrict__ b) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = a[t];
}

__global__ void fill_kernel(size_t n, double v, double* __restrict__ b) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = v;
}

template <typename T>
bamg_status vcycle_body(bamg_hierarchy* h, cudaStream_t s) {
  Level& L0 = h->lv[0];
  size_t n = L0.n;
  if (sizeof(T) == 4) {
    BAMG_TRY(convert<double, float>(n, h->io_in.as<double>(), (float*)L0.vb.p, s));
  } else {
    BAMG_TRY(launch(copy_d_kernel, dim3(cdiv((long long)n, 256)), dim3(256), 0, s, n,
                    (const double*)h->io_in.as<double>(), (double*)L0.vb.p));
  }
  BAMG_TRY(vcycle_level<T>(h, 0, s));
  if (sizeof(T) == 4) {
    BAMG_TRY(convert<float, double>(n, (const float*)L0.vz.p, h->io_out.as<double>(), s));
  } else {
    BAMG_TRY(launch(copy_d_kernel, dim3(cdiv((long long)n, 256)), dim3(256), 0, s, n,
                    (const double*)L0.vz.p, h->io_out.as<double>()));
  }
  return BAMG_OK;
}

// Allocates the V-cycle vectors and captures the V-cycle into a graph.
bamg_status vcycle_prepare(bamg_hierarchy* h, cudaStream_t s) {
  if (h->vexec) return BAMG_OK;
  size_t es = h->mixed ? sizeof(float) : sizeof(double);
  for (auto& L : h->lv) {
    BAMG_TRY(L.vb.alloc(es * L.n, s));
    BAMG_TRY(L.vz.alloc(es * L.n, s));
    BAMG_TRY(L.vt.alloc(es * L.n, s));
    BAMG_TRY(L.vr.alloc(es * L.n, s));
  }
  BAMG_TRY(h->io_in.alloc(sizeof(double) * h->lv[0].n, s));
  BAMG_TRY(h->io_out.alloc(sizeof(double) * h->lv[0].n, s));
  if (h->p.smoother == BAMG_SMOOTH_MCGS)
    for (size_t l = 0; l + 1 < h->lv.size(); ++l) {     // colourings of the smoothed levels
      Level& L = h->lv[l];
      BAMG_TRY(L.colour.alloc(sizeof(int32_t) * L.n, s));
      BAMG_TRY(L.crows.alloc(sizeof(int32_t) * L.n, s));
      BAMG_TRY(colour_graph(L.n, L.B.r(), L.B.c(), L.Bt.r(), L.Bt.c(), h->p.seed, (int)l, L.colour.as<int32_t>(),
                            &L.ncol, s));
      L.crp.assign(L.ncol + 1, 0);
      BAMG_TRY(colour_rows(L.n, L.colour.as<int32_t>(), L.ncol, L.crp.data(), L.crows.as<int32_t>(), s));
    }
  BAMG_CUDA(cudaStreamSynchronize(s));
  if (!h->cap_stream) BAMG_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  uint64_t before = t_launches;
  BAMG_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  bamg_status st = h->mixed ? vcycle_body<float>(h, h->cap_stream) : vcycle_body<double>(h, h->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  if (st != BAMG_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  BAMG_CUDA(e);
  h->vgraph = g;
  BAMG_CUDA(cudaGraphInstantiate(&h->vexec, g, 0));
  h->vgraph_kernels = t_launches - before;
  g_launches.fetch_sub(h->vgraph_kernels);  // counted again at each replay
  return BAMG_OK;
}

// Switches a mixed-precision hierarchy to FP64 V-cycles: the coarsest
// pseudo-inverse recomputed in FP64 (one triplet, discarded), the V-cycle
// vectors reallocated in FP64, the V-cycle and Arnoldi graphs captured again.
bamg_status promote_fp64(bamg_hierarchy* h, cudaStream_t s) {
  if (!h->mixed) return BAMG_OK;
  Level& LL = h->lv.back();
  const int nL = LL.n;
  const size_t nn = (size_t)nL * nL;
  DevMem Bd, Md, Nd, sg, Ud, Vd;
  BAMG_TRY(Bd.alloc(sizeof(double) * nn, s));
  BAMG_TRY(Md.alloc(sizeof(double) * nn, s));
  BAMG_TRY(Nd.alloc(sizeof(double) * nn, s));
  BAMG_TRY(sg.alloc(sizeof(double), s));
  BAMG_TRY(Ud.alloc(sizeof(double) * nL, s));
  BAMG_TRY(Vd.alloc(sizeof(double) * nL, s));
  BAMG_TRY(csr_to_dense(nL, LL.B.r(), LL.B.c(), LL.B.v(), Bd.as<double>(), s));
  if (LL.M.empty()) {
    std::vector<double> I(nn, 0.0);
    for (int i = 0; i < nL; ++i) I[(size_t)i * nL + i] = 1.0;
    BAMG_CUDA(cudaMemcpyAsync(Md.p, I.data(), sizeof(double) * nn, cudaMemcpyHostToDevice, s));
    BAMG_CUDA(cudaMemcpyAsync(Nd.p, I.data(), sizeof(double) * nn, cudaMemcpyHostToDevice, s));
    BAMG_CUDA(cudaStreamSynchronize(s));
  } else {
    BAMG_TRY(csr_to_dense(nL, LL.M.r(), LL.M.c(), LL.M.v(), Md.as<double>(), s));
    BAMG_TRY(csr_to_dense(nL, LL.N.r(), LL.N.c(), LL.N.v(), Nd.as<double>(), s));
  }
  BAMG_TRY(coarsest_solve(0, nL, 1, Bd.as<double>(), Md.as<double>(), Nd.as<double>(), sg.as<double>(),
                          Ud.as<double>(), Vd.as<double>(), h->Bpinv.as<double>(), s));
  h->mixed = 0;
  gmres_release(h);
  if (h->vexec) cudaGraphExecDestroy(h->vexec);
  if (h->vgraph) cudaGraphDestroy(h->vgraph);
  h->vexec = nullptr;
  h->vgraph = nullptr;
  return vcycle_prepare(h, s);
}

bamg_status vcycle_run(bamg_hierarchy* h, cudaStream_t s) {
  BAMG_CUDA(cudaGraphLaunch(h->vexec, s));
  g_launches.fetch_add(h->vgraph_kernels);
  return BAMG_OK;
}

// ------------------------------------------------------------- FGMRES kernels
constexpr int kRedBlocks = 256;

// The Arnoldi step of FGMRES runs as one captured graph; its kernels read
// the step index j (basis vectors 0..j in use) from device memory, so the
// same graph serves every step.  Partial sums use the fixed row stride m+1.

// part[b * (m+1) + k] = block b's share of V_k . w for k <= j
// part[b * (m+1) + k] = the block's share of V_k . w for k <= j: every block
// takes all j + 1 columns over its rows (one wave of blocks, w read once
// per column from L2), warp sums kept per warp and added in warp order.
constexpr int kMultidotMax = 65;   // m + 1 <= 65 (restart <= 64)
__global__ void __launch_bounds__(256) multidot_kernel(int n, int m, const int* __restrict__ dj,
                                                       const double* __restrict__ V, size_t ldv,
                                                       const double* __restrict__ w, double* __restrict__ part) {
  __shared__ double sh[8][kMultidotMax];
  const int K = dj[0] + 1, lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int k = 0; k < K; ++k) {
    const double* v = V + (size_t)k * ldv;
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += v[i] * w[i];
    s = warp_sum(s);
    if (lane == 0) sh[wp][k] = s;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q][k];
    part[(size_t)blockIdx.x * (m + 1) + k] = t;
  }
}

// out[k] = sum over the nb blocks of part[b * (m+1) + k], k <= j (fixed order)
__global__ void multidot_reduce_kernel(int nb, int m, const int* __restrict__ dj, const double* __restrict__ part,
                                       double* __restrict__ out) {
  __shared__ double sh[8];
  const int k = blockIdx.x;
  if (k > dj[0]) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(size_t)b * (m + 1) + k];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
    out[k] = t;
  }
}

// w -= sum_{k <= j} h[k] V_k
__global__ void orth_update_kernel(int n, const int* __restrict__ dj, const double* __restrict__ V, size_t ldv,
                                   const double* __restrict__ h, double* __restrict__ w) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int K = dj[0] + 1;
  double acc = w[i];
  for (int k = 0; k < K; ++k) acc -= h[k] * V[(size_t)k * ldv + i];
  w[i] = acc;
}

// out = V_j (get = 1) or V_j = in (get = 0)
__global__ void column_io_kernel(int n, const int* __restrict__ dj, int get, double* __restrict__ V,
                                 double* __restrict__ io) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double* v = V + (size_t)dj[0] * n;
  if (get) io[i] = v[i];
  else v[i] = io[i];
}

// V_{j+1} = w / ||w||
__global__ void next_basis_kernel(int n, const int* __restrict__ dj, const double* __restrict__ w,
                                  const double* __restrict__ nrm, double* __restrict__ V) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  V[(size_t)(dj[0] + 1) * n + i] = w[i] / nrm[0];
}

__global__ void step_kernel(int* dj) { dj[0] += 1; }

// y = x + sum_k c[k] Z_k
__global__ void combine_kernel(int n, int K, const double* __restrict__ Z, size_t ldz,
                               const double* __restrict__ c, const double* __restrict__ x, double* __restrict__ y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = x[i];
  for (int k = 0; k < K; ++k) acc += c[k] * Z[(size_t)k * ldz + i];
  y[i] = acc;
}

__global__ void scale_by_kernel(int n, const double* __restrict__ a, const double* __restrict__ f, int inv,
                                double* __restrict__ b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = inv ? 1.0 / f[0] : f[0];
  b[i] = a[i] * s;
}

__global__ void sumsq_kernel(int n, const double* __restrict__ x, double* __restrict__ part) {
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += x[i] * x[i];
  s = warp_sum(s);
  __shared__ double sh[8];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
    part[blockIdx.x] = t;
  }
}

__global__ void sqrt_kernel(double* v) { v[0] = sqrt(v[0]); }

// Arnoldi column j: H(:, j) = h1 + h2 (two CGS passes), H(j+1, j) = ||w||.
// Applies the previous Givens rotations, forms the new one, updates g, and
// solves R y = g(0..j).  st[0] = |g(j+1)| (residual 2-norm estimate),
// st[1] = H(j+1, j) before rotation.
// Column j of the Hessenberg matrix (h1 + h2 from the two Gram-Schmidt
// passes, then ||w||) through the previous rotations into R, a new rotation,
// the rotated right-hand side g; st = {|g_{j+1}|, ||w||}.  One thread; the
// column is streamed (each rotation only needs the entry carried from the
// previous one).
__global__ void givens_kernel(const int* __restrict__ dj, int m, const double* __restrict__ h1,
                              const double* __restrict__ h2, const double* __restrict__ wnorm,
                              double* __restrict__ R, double* __restrict__ cs, double* __restrict__ sn,
                              double* __restrict__ g, double* __restrict__ st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int j = dj[0];
  const double hn = wnorm[0];
  double carry = h1[0] + h2[0];
  for (int k = 0; k < j; ++k) {
    const double next = h1[k + 1] + h2[k + 1];
    const double c = cs[k], sk = sn[k];
    R[(size_t)k * m + j] = c * carry + sk * next;
    carry = -sk * carry + c * next;
  }
  const double a = carry, b = hn;
  const double d = hypot(a, b);
  const double c = d > 0.0 ? a / d : 1.0, sk = d > 0.0 ? b / d : 0.0;
  cs[j] = c; sn[j] = sk;
  R[(size_t)j * m + j] = d;
  g[j + 1] = -sk * g[j];
  g[j] = c * g[j];
  st[0] = fabs(g[j + 1]);
  st[1] = hn;
}

// y = R^{-1} g for the leading (j+1) x (j+1) block (back substitution).
__global__ void ysolve_kernel(int j, int m, const double* __restrict__ R, const double* __restrict__ g,
                              double* __restrict__ y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int k = j; k >= 0; --k) {
    double acc = g[k];
    for (int q = k + 1; q <= j; ++q) acc -= R[(size_t)k * m + q] * y[q];
    const double rkk = R[(size_t)k * m + k];
    y[k] = rkk != 0.0 ? acc / rkk : 0.0;
  }
}

__global__ void init_g_kernel(int m, const double* __restrict__ beta, double* __restrict__ g) {
  int k = threadIdx.x;
  if (k <= m) g[k] = k == 0 ? beta[0] : 0.0;
}

// Smallest entry: per-block minima, then one block over them.
__global__ void min_part_kernel(int n, const double* __restrict__ x, double* __restrict__ part) {
  __shared__ double sh[256];
  double m = INFINITY;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = fmin(m, x[i]);
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

bamg_status orient_normalise(int n, double* x, cudaStream_t s);

struct Gm {
  int n, m;
  DevMem V, Z, w, w2, xj, zeros, h1, h2, part, R, cs, sn, g, y, st, scal, sums;
};

static int red_blocks(int n) {
  int nb = (int)cdiv(n, 256);
  return nb < kRedBlocks ? (nb > 0 ? nb : 1) : kRedBlocks;
}

static bamg_status norm2_dev(Gm& G, const double* x, double* out, cudaStream_t s) {
  int nb = red_blocks(G.n);
  BAMG_TRY(launch(sumsq_kernel, dim3(nb), dim3(256), 0, s, G.n, x, G.part.as<double>()));
  BAMG_TRY(reduce_partials(G.part.as<double>(), nb, 1, out, s));
  return launch(sqrt_kernel, dim3(1), dim3(1), 0, s, out);
}


// rel = ||B x||_1 / ||x||_1 (read back to the host); xn1 = ||x||_1
static bamg_status true_residual(bamg_hierarchy* h, Gm& G, const double* x, double* rel, double* xn1,
                                 cudaStream_t s) {
  Level& L = h->lv[0];
  BAMG_TRY(csr_vec<double>(VEC_SPMV, L.n, L.vec_g, L.B.r(), L.B.c(), L.B.v(), L.dinv.as<double>(), 1.0, x,
                           nullptr, G.w2.as<double>(), s));
  double* sm = G.sums.as<double>();
  BAMG_TRY(abs_sums(L.n, G.w2.as<double>(), sm, s));
  BAMG_TRY(abs_sums(L.n, x, sm + 2, s));
  double hs[4];
  BAMG_CUDA(cudaMemcpyAsync(hs, sm, sizeof(hs), cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  *xn1 = hs[3];
  *rel = hs[3] > 0.0 ? hs[1] / hs[3] : INFINITY;
  return BAMG_OK;
}

// Persistent FGMRES workspace of a hierarchy and the captured Arnoldi step
// (rebuilt when the restart length changes).  Buffers live on the
// hierarchy's private stream, which outlives them.
struct GmresState {
  int m = 0;
  int plain = 0;             // 1: the identity instead of the V-cycle
  Gm G;
  DevMem dj;                 // step index j of the current restart cycle
  double* st_host = nullptr; // pinned: {|g_{j+1}|, ||w||} of the last step
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;
  ~GmresState() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (st_host) cudaFreeHost(st_host);
  }
};

void gmres_release(bamg_hierarchy* h) {
  delete h->gm;
  h->gm = nullptr;
}

// One Arnoldi step j (read from the device): z_j = C v_j (V-cycle), w = B z_j,
// two classical Gram-Schmidt passes, ||w||, the Givens update of column j,
// v_{j+1} = w / ||w||, j <- j + 1, and {|g_{j+1}|, ||w||} to pinned memory.
static bamg_status arnoldi_body(bamg_hierarchy* h, GmresState& S, cudaStream_t s) {
  Level& L = h->lv[0];
  Gm& G = S.G;
  const int n = G.n, m = G.m;
  const unsigned gv = cdiv(n, 256);
  const int nb = red_blocks(n);
  const int* dj = S.dj.as<int>();
  double* V = G.V.as<double>();
  BAMG_TRY(launch(column_io_kernel, dim3(gv), dim3(256), 0, s, n, dj, 1, V, h->io_in.as<double>()));
  if (S.plain)
    BAMG_TRY(launch(copy_d_kernel, dim3(gv), dim3(256), 0, s, (size_t)n, (const double*)h->io_in.as<double>(),
                    h->io_out.as<double>()));
  else
    BAMG_TRY(h->mixed ? vcycle_body<float>(h, s) : vcycle_body<double>(h, s));
  BAMG_TRY(launch(column_io_kernel, dim3(gv), dim3(256), 0, s, n, dj, 0, G.Z.as<double>(), h->io_out.as<double>()));
  BAMG_TRY(csr_vec<double>(VEC_SPMV, n, L.vec_g, L.B.r(), L.B.c(), L.B.v(), L.dinv.as<double>(), 1.0,
                           (const double*)h->io_out.as<double>(), nullptr, G.w.as<double>(), s));
  for (int pass = 0; pass < 2; ++pass) {       // classical Gram-Schmidt, twice
    double* hc = pass ? G.h2.as<double>() : G.h1.as<double>();
    BAMG_TRY(launch(multidot_kernel, dim3(nb), dim3(256), 0, s, n, m, dj, (const double*)V, (size_t)n,
                    (const double*)G.w.as<double>(), G.part.as<double>()));
    BAMG_TRY(launch(multidot_reduce_kernel, dim3(m + 1), dim3(256), 0, s, nb, m, dj,
                    (const double*)G.part.as<double>(), hc));
    BAMG_TRY(launch(orth_update_kernel, dim3(gv), dim3(256), 0, s, n, dj, (const double*)V, (size_t)n,
                    (const double*)hc, G.w.as<double>()));
  }
  BAMG_TRY(norm2_dev(G, G.w.as<double>(), G.scal.as<double>(), s));
  BAMG_TRY(launch(givens_kernel, dim3(1), dim3(32), 0, s, dj, m, (const double*)G.h1.as<double>(),
                  (const double*)G.h2.as<double>(), (const double*)G.scal.as<double>(), G.R.as<double>(),
                  G.cs.as<double>(), G.sn.as<double>(), G.g.as<double>(), G.st.as<double>()));
  BAMG_TRY(launch(next_basis_kernel, dim3(gv), dim3(256), 0, s, n, dj, (const double*)G.w.as<double>(),
                  (const double*)G.scal.as<double>(), V));
  BAMG_TRY(launch(step_kernel, dim3(1), dim3(1), 0, s, S.dj.as<int>()));
  BAMG_CUDA(cudaMemcpyAsync(S.st_host, G.st.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  return BAMG_OK;
}

static bamg_status gmres_prepare(bamg_hierarchy* h, int m, int plain) {
  if (h->gm && h->gm->m == m && h->gm->plain == plain) return BAMG_OK;
  gmres_release(h);
  cudaStream_t cs = h->cap_stream;
  GmresState* S = new (std::nothrow) GmresState();
  if (!S) return BAMG_ERR_OOM;
  h->gm = S;
  S->plain = plain;
  const int n = h->lv[0].n;
  Gm& G = S->G;
  S->m = m;
  G.n = n;
  G.m = m;
  BAMG_TRY(G.V.alloc(sizeof(double) * (size_t)(m + 1) * n, cs));
  BAMG_TRY(G.Z.alloc(sizeof(double) * (size_t)m * n, cs));
  BAMG_TRY(G.w.alloc(sizeof(double) * n, cs));
  BAMG_TRY(G.w2.alloc(sizeof(double) * n, cs));
  BAMG_TRY(G.xj.alloc(sizeof(double) * n, cs));
  BAMG_TRY(G.zeros.alloc(sizeof(double) * n, cs));
  BAMG_TRY(G.h1.alloc(sizeof(double) * (m + 1), cs));
  BAMG_TRY(G.h2.alloc(sizeof(double) * (m + 1), cs));
  BAMG_TRY(G.part.alloc(sizeof(double) * kRedBlocks * (m + 1), cs));
  BAMG_TRY(G.R.alloc(sizeof(double) * (size_t)(m + 1) * m, cs));
  BAMG_TRY(G.cs.alloc(sizeof(double) * m, cs));
  BAMG_TRY(G.sn.alloc(sizeof(double) * m, cs));
  BAMG_TRY(G.g.alloc(sizeof(double) * (m + 1), cs));
  BAMG_TRY(G.y.alloc(sizeof(double) * m, cs));
  BAMG_TRY(G.st.alloc(sizeof(double) * 2, cs));
  BAMG_TRY(G.scal.alloc(sizeof(double) * 2, cs));
  BAMG_TRY(G.sums.alloc(sizeof(double) * 4, cs));
  BAMG_TRY(S->dj.alloc(sizeof(int), cs));
  BAMG_CUDA(cudaMemsetAsync(G.zeros.p, 0, sizeof(double) * n, cs));
  BAMG_CUDA(cudaHostAlloc(&S->st_host, 2 * sizeof(double), cudaHostAllocDefault));
  BAMG_CUDA(cudaStreamSynchronize(cs));
  uint64_t before = t_launches;
  BAMG_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  bamg_status st = arnoldi_body(h, *S, cs);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  if (st != BAMG_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  BAMG_CUDA(e);
  S->graph = g;
  BAMG_CUDA(cudaGraphInstantiate(&S->exec, g, 0));
  S->kernels = t_launches - before;
  g_launches.fetch_sub(S->kernels);  // counted at each replay
  return BAMG_OK;
}

bamg_status fgmres(bamg_hierarchy* h, double* x, const bamg_solve_params* sp, bamg_solve_info* info,
                   cudaStream_t s) {
  Level& L = h->lv[0];
  const int n = L.n, m = sp->restart;
  BAMG_TRY(vcycle_prepare(h, s));
  BAMG_TRY(gmres_prepare(h, m, sp->plain ? 1 : 0));
  GmresState& S = *h->gm;
  Gm& G = S.G;
  if (sp->plain)        // unpreconditioned comparator: from the uniform vector
    BAMG_TRY(launch(fill_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, (size_t)n, 1.0 / n, x));
  else
    BAMG_CUDA(cudaMemcpyAsync(x, h->x0.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));

  double rel = 0.0, xn1 = 1.0;
  BAMG_TRY(true_residual(h, G, x, &rel, &xn1, s));
  const double xn1_0 = xn1;
  double xn2_0 = 0.0;
  BAMG_TRY(norm2_dev(G, x, G.scal.as<double>() + 1, s));
  BAMG_CUDA(cudaMemcpyAsync(&xn2_0, G.scal.as<double>() + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  int its = 0, it7 = -1;
  bool done = rel <= sp->tol;
  bool breakdown = false, stalled = false;
  // with the FP32 V-cycle, a true residual that falls by less than half over
  // two restart cycles in a row marks a stall (the caller continues in FP64)
  const bool stall_check = h->mixed && !sp->plain;
  double prev_rel = rel;
  int slow = 0;
  double* V = G.V.as<double>();
  double* Z = G.Z.as<double>();
  const unsigned gv = cdiv(n, 256);
  while (!done && its < sp->max_iter) {
    // r = -B x, beta = ||r||, v_0 = r / beta, g = beta e_1, j = 0
    BAMG_TRY(csr_vec<double>(VEC_RESID, n, L.vec_g, L.B.r(), L.B.c(), L.B.v(), L.dinv.as<double>(), 1.0, x,
                             G.zeros.as<double>(), G.w.as<double>(), s));
    BAMG_TRY(norm2_dev(G, G.w.as<double>(), G.scal.as<double>(), s));
    BAMG_TRY(launch(scale_by_kernel, dim3(gv), dim3(256), 0, s, n, (const double*)G.w.as<double>(),
                    (const double*)G.scal.as<double>(), 1, V));
    BAMG_TRY(launch(init_g_kernel, dim3(1), dim3(128), 0, s, m, (const double*)G.scal.as<double>(),
                    G.g.as<double>()));
    BAMG_CUDA(cudaMemsetAsync(S.dj.p, 0, sizeof(int), s));
    for (int j = 0; j < m && !done; ++j) {
      BAMG_CUDA(cudaGraphLaunch(S.exec, s));
      g_launches.fetch_add(S.kernels);
      BAMG_CUDA(cudaStreamSynchronize(s));
      const double st0 = S.st_host[0], st1 = S.st_host[1];
      const int K = j + 1;
      ++its;
      if (it7 < 0 && st0 <= 1e-7 * xn2_0) it7 = its;
      breakdown = !(st1 > 0.0);
      bool last = (j == m - 1) || its >= sp->max_iter || breakdown;
      if (st0 <= 2.0 * sp->tol * xn1_0 || last) {
        BAMG_TRY(launch(ysolve_kernel, dim3(1), dim3(32), 0, s, j, m, (const double*)G.R.as<double>(),
                        (const double*)G.g.as<double>(), G.y.as<double>()));
        BAMG_TRY(launch(combine_kernel, dim3(gv), dim3(256), 0, s, n, K, (const double*)Z, (size_t)n,
                        (const double*)G.y.as<double>(), (const double*)x, G.xj.as<double>()));
        BAMG_TRY(true_residual(h, G, G.xj.as<double>(), &rel, &xn1, s));
        if (rel <= sp->tol || last) {
          BAMG_CUDA(cudaMemcpyAsync(x, G.xj.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
          done = rel <= sp->tol;
          break;
        }
      }
    }
    if (breakdown && !done) break;
    if (stall_check && !done) {
      slow = rel > 0.5 * prev_rel ? slow + 1 : 0;
      prev_rel = rel;
      if (slow >= 2) { stalled = true; break; }
    }
  }
  BAMG_TRY(orient_normalise(n, x, s));
  double fin[2] = {0, 0};
  {
    const int nb = red_blocks(n);
    BAMG_TRY(launch(min_part_kernel, dim3(nb), dim3(256), 0, s, n, (const double*)x, G.part.as<double>()));
    BAMG_TRY(launch(min_part_kernel, dim3(1), dim3(256), 0, s, nb, (const double*)G.part.as<double>(),
                    G.scal.as<double>()));
  }
  BAMG_CUDA(cudaMemcpyAsync(fin, G.scal.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  BAMG_TRY(true_residual(h, G, x, &rel, &xn1, s));
  if (info) {
    info->iterations = its;
    info->iters_to_1e7 = it7;
    info->rel_res_1 = rel;
    info->min_x = fin[0];
  }
  if (!done) {
    set_error("GMRES %s after %d iterations at ||Bx||_1/||x||_1 = %.3e", stalled ? "stalled" : "stopped", its,
              rel);
    return breakdown ? BAMG_ERR_BREAKDOWN : BAMG_ERR_NOT_CONVERGED;
  }
  return BAMG_OK;
}

// ------------------------------------------------- V-cycle convergence factor
// x_i = 1 + 0.5 * u_i with u_i uniform in [-1, 1) (SplitMix64 stream 8193)
__global__ void factor_start_kernel(int n, uint64_t seed, double* __restrict__ x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = 1.0 + 0.5 * splitmix_pm1(seed, 8193, (uint64_t)i);
}

__global__ void add_kernel(int n, const double* __restrict__ z, double* __restrict__ x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] += z[i];
}

// Stationary iteration x <- x + C(0 - B x) with the V-cycle C: the residual
// obeys r <- (I - B C) r (eq. error_propagator_twogrid moved to the residual
// side), so the ratio of its 1-norms over the second half of the run
// estimates the asymptotic convergence factor on the range of B.
bamg_status vcycle_factor(bamg_hierarchy* h, int iters, uint64_t seed, double* factor, cudaStream_t s) {
  BAMG_TRY(vcycle_prepare(h, s));
  Level& L = h->lv[0];
  const int n = L.n;
  DevMem x, r, zero, sums;
  BAMG_TRY(x.alloc(sizeof(double) * n, s));
  BAMG_TRY(r.alloc(sizeof(double) * n, s));
  BAMG_TRY(zero.alloc(sizeof(double) * n, s));
  BAMG_TRY(sums.alloc(sizeof(double) * 2 * (iters + 1), s));
  BAMG_CUDA(cudaMemsetAsync(zero.p, 0, sizeof(double) * n, s));
  unsigned g = cdiv(n, 256);
  BAMG_TRY(launch(factor_start_kernel, dim3(g), dim3(256), 0, s, n, seed, x.as<double>()));
  const int G = lanes_for(L.B);
  for (int k = 0; k <= iters; ++k) {
    BAMG_TRY(csr_vec<double>(VEC_RESID, n, G, L.B.r(), L.B.c(), L.B.v(), nullptr, 0.0, x.as<double>(),
                             zero.as<double>(), r.as<double>(), s));
    BAMG_TRY(abs_sums(n, r.as<double>(), sums.as<double>() + 2 * k, s));
    if (k == iters) break;
    BAMG_CUDA(cudaMemcpyAsync(h->io_in.p, r.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    BAMG_TRY(vcycle_run(h, s));
    BAMG_TRY(launch(add_kernel, dim3(g), dim3(256), 0, s, n, (const double*)h->io_out.as<double>(), x.as<double>()));
  }
  std::vector<double> hs(2 * (iters + 1));
  BAMG_CUDA(cudaMemcpyAsync(hs.data(), sums.p, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  const int k0 = iters / 2;
  double a = hs[2 * k0 + 1], b = hs[2 * iters + 1];
  if (!(a > 0.0) || !std::isfinite(b)) {
    *factor = std::isfinite(b) ? 0.0 : INFINITY;
    return BAMG_OK;
  }
  *factor = std::pow(b / a, 1.0 / (iters - k0));
  return BAMG_OK;
}

template bamg_status vcycle_body<double>(bamg_hierarchy*, cudaStream_t);
template bamg_status vcycle_body<float>(bamg_hierarchy*, cudaStream_t);

}  // namespace bamg
