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
#include <cuda.h>

#include <chrono>
#include <cstdlib>
#include <cmath>
#include <mutex>
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
__global__ void zero_kernel(size_t n, T* __restrict__ y) {
  pdl_wait();
  pdl_trigger();
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) y[t] = T(0);
}

// Levels of at most this many rows take the prolongation and the first
// post-sweep in one pass: there a pass costs its launch and latency, not its
// bytes (on a 2^20-row level the fused pass, which gathers P's rows for every
// neighbour, made the Delaunay solve 15 % slower).
constexpr int kFuseProlongRows = 65536;

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
  const unsigned gn = cdiv(L.n, 256);
  if (p.smoother == BAMG_SMOOTH_MCGS) {
    // multicolour Gauss-Seidel, in place (Section 3 splitting)
    auto sweep = [&](T* x) {
      return mcgs_sweep<T>(L.vec_g, L.ncol, L.crp.data(), L.crows.as<int32_t>(), L.B.r(), L.B.c(), bv, dv, b, x, s);
    };
    BAMG_TRY(launch(zero_kernel<T>, dim3(gn), dim3(256), 0, s, (size_t)L.n, z));
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
  // Jacobi sweeps alternate between z and the scratch vt; the first two
  // pre-sweeps from zero take one pass.  The start buffer is chosen so that
  // the last sweep writes z.
  const int swaps = (p.nu_pre >= 2 ? p.nu_pre - 2 : 0) + p.nu_post;
  T* cur = swaps % 2 == 0 ? z : L.vt.as<T>();
  T* alt = cur == z ? L.vt.as<T>() : z;
  if (p.nu_pre == 0) {
    BAMG_TRY(launch(zero_kernel<T>, dim3(gn), dim3(256), 0, s, (size_t)L.n, cur));
  } else if (p.nu_pre == 1) {
    BAMG_TRY(csr_vec<T>(VEC_JACOBI_ZERO, L.n, L.vec_g, L.B.r(), L.B.c(), bv, dv, om, nullptr, b, cur, s));
  } else {
    BAMG_TRY(csr_vec<T>(VEC_JACOBI_ZERO2, L.n, L.vec_g, L.B.r(), L.B.c(), bv, dv, om, nullptr, b, cur, s));
    for (int it = 2; it < p.nu_pre; ++it) {
      BAMG_TRY(csr_vec<T>(VEC_JACOBI, L.n, L.vec_g, L.B.r(), L.B.c(), bv, dv, om, cur, b, alt, s));
      std::swap(cur, alt);
    }
  }
  BAMG_TRY(csr_vec<T>(VEC_RESID, L.n, L.vec_g, L.B.r(), L.B.c(), bv, dv, om, cur, b, L.vr.as<T>(), s));
  Level& C = h->lv[l + 1];
  BAMG_TRY(csr_vec<T>(VEC_SPMV, L.nc, lanes_for(L.Q), L.Q.r(), L.Q.c(), L.Q.vals<T>(), dv, om, L.vr.as<T>(),
                      nullptr, C.vb.as<T>(), s));
  BAMG_TRY(vcycle_level<T>(h, l + 1, s));
  int post = p.nu_post;
  if (post > 0 && L.n <= kFuseProlongRows) {
    // z += P e_c and the first post-sweep in one pass (writes alt, as the
    // sweep did); on larger levels the separate passes move fewer bytes
    BAMG_TRY(prolong_jacobi<T>(L.n, L.vec_g, L.B.r(), L.B.c(), bv, dv, om, L.P.r(), L.P.c(), L.P.vals<T>(),
                               C.vz.as<T>(), cur, b, alt, s));
    std::swap(cur, alt);
    --post;
  } else {
    BAMG_TRY(csr_vec<T>(VEC_SPMV_ADD, L.n, lanes_for(L.P), L.P.r(), L.P.c(), L.P.vals<T>(), dv, om,
                        C.vz.as<T>(), nullptr, cur, s));
  }
  for (int it = 0; it < post; ++it) {
    BAMG_TRY(csr_vec<T>(VEC_JACOBI, L.n, L.vec_g, L.B.r(), L.B.c(), bv, dv, om, cur, b, alt, s));
    std::swap(cur, alt);
  }
  if (cur != z) {
    set_error("V-cycle level %d: the last sweep did not write z", l);
    return BAMG_ERR_CUDA;
  }
  return BAMG_OK;
}

__global__ void fill_kernel(size_t n, double v, double* __restrict__ b) {
  pdl_wait();
  pdl_trigger();
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = v;
}

// V-cycle input: b = in, or the column j = col[0] of the n-row array in,
// converted to the V-cycle precision.  With w given and j > 0 the column is
// first formed as w * rinv[0] (the previous Arnoldi step's w / ||w||) and
// stored.
template <typename T>
__global__ void vc_in_kernel(int n, double* __restrict__ in, const int* __restrict__ col, const double* __restrict__ w,
                             const double* __restrict__ rinv, T* __restrict__ b) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v;
  if (col) {
    const int j = col[0];
    double* vc = in + (size_t)j * n;
    if (w && j > 0) {
      v = w[i] * rinv[0];
      vc[i] = v;
    } else {
      v = vc[i];
    }
  } else {
    v = in[i];
  }
  b[i] = T(v);
}

// V-cycle output: out = z in FP64, and the same values into the column
// col[0] of out_col when out_col is given.
template <typename T>
__global__ void vc_out_kernel(int n, const T* __restrict__ z, double* __restrict__ out, const int* __restrict__ col,
                              double* __restrict__ out_col) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = double(z[i]);
  out[i] = v;
  if (out_col) out_col[(size_t)col[0] * n + i] = v;
}

// z = C in (in: n doubles, or the column j = col[0] of an n-row array, formed
// from w and rinv first when w is given and j > 0); z goes to out and, with
// out_col, also to the column j of out_col.
template <typename T>
bamg_status vcycle_body(bamg_hierarchy* h, cudaStream_t s, double* in, const int* col, double* out,
                        double* out_col, const double* w, const double* rinv) {
  Level& L0 = h->lv[0];
  const int n = L0.n;
  BAMG_TRY(launch(vc_in_kernel<T>, dim3(cdiv(n, 256)), dim3(256), 0, s, n, in, col, w, rinv, L0.vb.as<T>()));
  BAMG_TRY(vcycle_level<T>(h, 0, s));
  return launch(vc_out_kernel<T>, dim3(cdiv(n, 256)), dim3(256), 0, s, n, (const T*)L0.vz.as<T>(), out, col,
                out_col);
}

// BAMG_TRACE: nodes of a captured graph and how many of its edges are
// programmatic (kernel-to-kernel overlap) rather than full dependencies.
static void trace_edges(const char* what, cudaGraph_t g) {
  size_t nn = 0, ne = 0;
  cudaGraphGetNodes(g, nullptr, &nn);
  cudaGraphGetEdges(g, nullptr, nullptr, nullptr, &ne);
  std::vector<cudaGraphNode_t> from(ne), to(ne);
  std::vector<cudaGraphEdgeData> ed(ne);
  size_t prog = 0;
  if (ne && cudaGraphGetEdges(g, from.data(), to.data(), ed.data(), &ne) == cudaSuccess)
    for (size_t e = 0; e < ne; ++e) prog += ed[e].type == cudaGraphDependencyTypeProgrammatic;
  cudaGetLastError();
  fprintf(stderr, "[bamg] %s graph: %zu nodes, %zu edges, %zu programmatic\n", what, nn, ne, prog);
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
  const bool mcgs = h->p.smoother == BAMG_SMOOTH_MCGS;
  if (mcgs)
    for (size_t l = 0; l + 1 < h->lv.size(); ++l) {     // colourings of the smoothed levels
      Level& L = h->lv[l];
      BAMG_TRY(L.colour.alloc(sizeof(int32_t) * L.n, s));
      BAMG_TRY(L.crows.alloc(sizeof(int32_t) * L.n, s));
      BAMG_TRY(colour_graph(L.n, L.B.r(), L.B.c(), L.Bt.r(), L.Bt.c(), h->p.seed, (int)l, L.colour.as<int32_t>(),
                            &L.ncol, s));
      L.crp.assign(L.ncol + 1, 0);
      BAMG_TRY(colour_rows(L.n, L.colour.as<int32_t>(), L.ncol, L.crp.data(), L.crows.as<int32_t>(), s));
    }
  // (the Jacobi V-cycle needs no result of the stream's pending work: the
  // capture only records pointers, and the graph runs after the setup)
  if (mcgs) BAMG_CUDA(cudaStreamSynchronize(s));
  if (!h->cap_stream) BAMG_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  uint64_t before = t_launches;
  BAMG_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  bamg_status st;
  {
    PdlScope pdl;
    double* in = h->io_in.as<double>();
    double* out = h->io_out.as<double>();
    st = h->mixed ? vcycle_body<float>(h, h->cap_stream, in, nullptr, out, nullptr, nullptr, nullptr)
                  : vcycle_body<double>(h, h->cap_stream, in, nullptr, out, nullptr, nullptr, nullptr);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  if (st != BAMG_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  BAMG_CUDA(e);
  h->vgraph = g;
  if (std::getenv("BAMG_TRACE")) trace_edges("V-cycle", g);
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

// The Arnoldi step of FGMRES runs as one captured graph; its kernels read
// the step index j (basis vectors 0..j in use) from device memory, so the
// same graph serves every step.  Partial sums use the fixed row stride m+1.

// Classical Gram-Schmidt against the basis V_0 .. V_j (K = j + 1 columns of
// n rows, stride ldv), three fused forms:
//   kGsDots:   out[k] = V_k . w;
//   kGsUpDots: w -= sum_k hin[k] V_k, then out[k] = V_k . w (the first pass's
//              update and the second pass's products: V read once for both);
//   kGsUpNorm: w -= sum_k hin[k] V_k, then out[0] = ||w||_2, out[1] = 1 / out[0].
// One wave of at most kRedBlocks blocks; each thread takes the rows
// tid, tid + stride, ...; loads of eight columns are issued together.
// FP64 arithmetic is the scarce resource here, so the eight per-lane sums of
// a chunk are reduced over the warp by a reduce-scatter (nine additions per
// lane instead of five per column).  A block adds its warps' totals in warp
// order into part (row stride m + 1); the last block to finish reduces the
// blocks' shares the same way (thread t takes block t) and resets the
// arrival counter.  The order is fixed, so every run gives the same result.
constexpr int kMultidotMax = 65;   // m + 1 <= 65 (restart <= 64)
constexpr int kRedBlocks = 256;
enum { kGsDots = 0, kGsUpDots = 1, kGsUpNorm = 2 };

// The Givens update of column j (kGsUpNorm, by its last block once ||w|| is
// known): column j of the Hessenberg matrix, h1 + h2 from the two passes and
// then ||w||, goes through the previous rotations into R (row stride m), a new
// rotation (cs, sn) zeroes ||w||, the right-hand side g is rotated, the
// status slot st[2 (j mod 2) + {0, 1}] = {|g_{j+1}|, ||w||} is written (two
// slots, so that step j + 1 may run while the host reads step j) and j
// advances.
struct GivensArgs {
  const double* h1;
  double *R, *cs, *sn, *g, *st;
  int* dj;
};

// Warp reduce-scatter of eight per-lane values a[0..7]: returns, in every
// lane, the warp total of column rs8_col(lane) (the four lanes that differ
// only in bits 0 and 1 hold the same column).
__device__ __forceinline__ int rs8_col(int lane) { return (lane >> 2) & 7; }
__device__ __forceinline__ double rs8(const double (&a)[8], int lane) {
  const unsigned full = 0xffffffffu;
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
  double b[4];
#pragma unroll
  for (int q = 0; q < 4; ++q)      // lanes without bit 4 keep columns 0..3, the others 4..7
    b[q] = (h16 ? a[q + 4] : a[q]) + __shfl_xor_sync(full, h16 ? a[q] : a[q + 4], 16);
  double c[2];
#pragma unroll
  for (int q = 0; q < 2; ++q)
    c[q] = (h8 ? b[q + 2] : b[q]) + __shfl_xor_sync(full, h8 ? b[q] : b[q + 2], 8);
  double d = (h4 ? c[1] : c[0]) + __shfl_xor_sync(full, h4 ? c[0] : c[1], 4);
  d += __shfl_xor_sync(full, d, 2);
  d += __shfl_xor_sync(full, d, 1);
  return d;
}

template <int MODE>
__global__ void __launch_bounds__(256) gs_kernel(int n, int m, const int* __restrict__ dj,
                                                 const double* __restrict__ V, size_t ldv,
                                                 const double* __restrict__ hin, double* __restrict__ w,
                                                 double* __restrict__ part, unsigned* __restrict__ arrived,
                                                 double* __restrict__ out, GivensArgs ga) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[8][kMultidotMax];
  __shared__ double hs[kMultidotMax];
  __shared__ double gc[kMultidotMax], gsn[kMultidotMax];
  __shared__ bool last;
  const int K = dj[0] + 1, lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int col = rs8_col(lane);
  const int stride = gridDim.x * blockDim.x, i0 = blockIdx.x * blockDim.x + threadIdx.x;
  double ss = 0.0;
  if (MODE != kGsDots) {
    for (int k = threadIdx.x; k < K; k += blockDim.x) hs[k] = hin[k];
    __syncthreads();
    for (int i = i0; i < n; i += stride) {
      double acc = w[i];
      for (int kc = 0; kc < K; kc += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = kc + u < K ? V[(size_t)(kc + u) * ldv + i] : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (kc + u < K) acc -= hs[kc + u] * v[u];
      }
      w[i] = acc;
      if (MODE == kGsUpNorm) ss += acc * acc;
    }
  }
  if (MODE == kGsUpNorm) {
    ss = warp_sum(ss);
    if (lane == 0) sh[wp][0] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < 8; ++q) t += sh[q][0];
      part[blockIdx.x] = t;
    }
  } else {
    for (int kc = 0; kc < K; kc += 8) {
      double sd[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) sd[u] = 0.0;
      for (int i = i0; i < n; i += stride) {
        const double wi = w[i];
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = kc + u < K ? V[(size_t)(kc + u) * ldv + i] : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (kc + u < K) sd[u] += v[u] * wi;
      }
      const double r = rs8(sd, lane);
      if ((lane & 3) == 0 && kc + col < K) sh[wp][kc + col] = r;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      double t = 0.0;
      for (int q = 0; q < 8; ++q) t += sh[q][k];
      part[(size_t)blockIdx.x * (m + 1) + k] = t;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(arrived, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int t = threadIdx.x, nb = gridDim.x;
  if (MODE == kGsUpNorm) {
    double r = t < nb ? __ldcg(part + t) : 0.0;
    r = warp_sum(r);
    if (lane == 0) sh[wp][0] = r;
    // column j of the Hessenberg matrix and the earlier rotations, staged
    const int j = K - 1;
    for (int k = t; k <= j; k += blockDim.x) hs[k] = ga.h1[k] + hs[k];
    for (int k = t; k < j; k += blockDim.x) {
      gc[k] = ga.cs[k];
      gsn[k] = ga.sn[k];
    }
    __syncthreads();
    if (t == 0) {
      double a = 0.0;
      for (int q = 0; q < 8; ++q) a += sh[q][0];
      const double nrm = sqrt(a);
      out[0] = nrm;
      out[1] = 1.0 / nrm;
      *arrived = 0u;
      // the rotations stream the column (each needs only the carried entry)
      double carry = hs[0];
      for (int k = 0; k < j; ++k) {
        const double next = hs[k + 1];
        const double c = gc[k], sk = gsn[k];
        ga.R[(size_t)k * m + j] = c * carry + sk * next;
        carry = -sk * carry + c * next;
      }
      const double d = hypot(carry, nrm);
      const double c = d > 0.0 ? carry / d : 1.0, sk = d > 0.0 ? nrm / d : 0.0;
      ga.cs[j] = c;
      ga.sn[j] = sk;
      ga.R[(size_t)j * m + j] = d;
      ga.g[j + 1] = -sk * ga.g[j];
      ga.g[j] = c * ga.g[j];
      ga.st[2 * (j & 1)] = fabs(ga.g[j + 1]);
      ga.st[2 * (j & 1) + 1] = nrm;
      ga.dj[0] = j + 1;   // every block has read j (the arrival count is complete)
    }
    return;
  }
  for (int kc = 0; kc < K; kc += 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = (kc + u < K && t < nb) ? __ldcg(part + (size_t)t * (m + 1) + kc + u) : 0.0;
    const double r = rs8(v, lane);
    if ((lane & 3) == 0 && kc + col < K) sh[wp][kc + col] = r;
  }
  __syncthreads();
  for (int k = t; k < K; k += blockDim.x) {
    double a = 0.0;
    for (int q = 0; q < 8; ++q) a += sh[q][k];
    out[k] = a;
  }
  if (t == 0) *arrived = 0u;
}

// Unpreconditioned step: V_j = w * rinv[0] for j > 0 (the previous step's
// w / ||w||), then out = V_j and Z_j = V_j.
__global__ void plain_io_kernel(int n, const int* __restrict__ dj, double* __restrict__ V,
                                const double* __restrict__ w, const double* __restrict__ rinv,
                                double* __restrict__ out, double* __restrict__ Z) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int j = dj[0];
  const size_t o = (size_t)j * n + i;
  double v;
  if (j > 0) {
    v = w[i] * rinv[0];
    V[o] = v;
  } else {
    v = V[o];
  }
  out[i] = v;
  Z[o] = v;
}

// y = x + sum_k c[k] Z_k
__global__ void combine_kernel(int n, int K, const double* __restrict__ Z, size_t ldz,
                               const double* __restrict__ c, const double* __restrict__ x, double* __restrict__ y) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = x[i];
  for (int kc = 0; kc < K; kc += 8) {       // eight column loads in flight
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = kc + u < K ? Z[(size_t)(kc + u) * ldz + i] : 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (kc + u < K) acc += c[kc + u] * v[u];
  }
  y[i] = acc;
}

__global__ void scale_by_kernel(int n, const double* __restrict__ a, const double* __restrict__ f, int inv,
                                double* __restrict__ b) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = inv ? 1.0 / f[0] : f[0];
  b[i] = a[i] * s;
}

// out[0] = ||x||_2: per-block sums of squares (warp sums added in warp
// order), then the last block to finish adds the nb block sums in a fixed
// order (thread t takes blocks t, t + 256, ..., then warp sums in warp
// order), takes the square root and resets the arrival counter.
__global__ void __launch_bounds__(256) norm2_kernel(int n, const double* __restrict__ x, double* __restrict__ part,
                                                   unsigned* __restrict__ arrived, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[8];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += x[i] * x[i];
  s = warp_sum(s);
  if (lane == 0) sh[wp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += sh[q];
    part[blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(arrived, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double r = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += 256) r += __ldcg(part + b);
  r = warp_sum(r);
  if (lane == 0) sh[wp] = r;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += sh[q];
    out[0] = sqrt(t);
    *arrived = 0u;
  }
}

// y = R^{-1} g for the leading (j+1) x (j+1) block (back substitution).  A
// warp stages the upper triangle in shared memory (at most 64 x 64, stride
// kYsolveLd), one thread substitutes.
constexpr int kYsolveLd = 65;
__global__ void ysolve_kernel(int j, int m, const double* __restrict__ R, const double* __restrict__ g,
                              double* __restrict__ y) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ double rs[];      // (j + 1) x kYsolveLd, then g and y
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  double* gs = rs + (size_t)(j + 1) * kYsolveLd;
  double* ys = gs + (j + 1);
  for (int k = 0; k <= j; ++k)
    for (int q = k + (int)threadIdx.x; q <= j; q += 32) rs[k * kYsolveLd + q] = R[(size_t)k * m + q];
  for (int k = threadIdx.x; k <= j; k += 32) gs[k] = g[k];
  __syncwarp();
  if (threadIdx.x != 0) return;
  for (int k = j; k >= 0; --k) {
    double acc = gs[k];
    for (int q = k + 1; q <= j; ++q) acc -= rs[k * kYsolveLd + q] * ys[q];
    const double rkk = rs[k * kYsolveLd + k];
    ys[k] = rkk != 0.0 ? acc / rkk : 0.0;
    y[k] = ys[k];
  }
}

__global__ void init_g_kernel(int m, const double* __restrict__ beta, double* __restrict__ g) {
  pdl_wait();
  pdl_trigger();
  int k = threadIdx.x;
  if (k <= m) g[k] = k == 0 ? beta[0] : 0.0;
}

// Smallest entry: per-block minima, then one block over them.
__global__ void min_part_kernel(int n, const double* __restrict__ x, double* __restrict__ part) {
  pdl_wait();
  pdl_trigger();
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
  DevMem V, Z, w, w2, xj, zeros, h1, h2, part, R, cs, sn, g, y, scal, sums;
  DevMem arrived;   // arrival counters of the last-block reductions
};

static int red_blocks(int n) {
  int nb = (int)cdiv(n, 256);
  return nb < kRedBlocks ? (nb > 0 ? nb : 1) : kRedBlocks;
}

enum { kArrMultidot = 0, kArrNorm = 1, kArrCount = 2 };

static bamg_status norm2_dev(Gm& G, const double* x, double* out, cudaStream_t s) {
  return launch(norm2_kernel, dim3(red_blocks(G.n)), dim3(256), 0, s, G.n, x, G.part.as<double>(),
                G.arrived.as<unsigned>() + kArrNorm, out);
}


// rel = ||B x||_1 / ||x||_1 (read back to the host); xn1 = ||x||_1; with
// xn2 given also ||x||_2, in the same read
static bamg_status true_residual(bamg_hierarchy* h, Gm& G, const double* x, double* rel, double* xn1,
                                 cudaStream_t s, double* xn2 = nullptr) {
  Level& L = h->lv[0];
  BAMG_TRY(csr_vec<double>(VEC_SPMV, L.n, L.vec_g, L.B.r(), L.B.c(), L.B.v(), L.dinv.as<double>(), 1.0, x,
                           nullptr, G.w2.as<double>(), s));
  double* sm = G.sums.as<double>();
  BAMG_TRY(abs_sums(L.n, G.w2.as<double>(), sm, s));
  BAMG_TRY(abs_sums(L.n, x, sm + 2, s));
  if (xn2) BAMG_TRY(norm2_dev(G, x, sm + 4, s));
  double hs[5];
  BAMG_CUDA(cudaMemcpyAsync(hs, sm, sizeof(double) * (xn2 ? 5 : 4), cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  *xn1 = hs[3];
  *rel = hs[3] > 0.0 ? hs[1] / hs[3] : INFINITY;
  if (xn2) *xn2 = hs[4];
  return BAMG_OK;
}

// Persistent FGMRES workspace of a hierarchy and the captured Arnoldi step
// (rebuilt when the restart length changes).  Buffers live on the
// hierarchy's private stream, which outlives them.
// Pinned, mapped host slots (four doubles) for the per-step Arnoldi status.
// A pinned allocation per workspace may synchronise with the device (and a
// pinned free does), so slots come from chunks allocated once per CUDA
// context and kept for its life.  Slots are keyed by the context id: after a
// device reset (a new context) the old chunks are gone, their slots are
// dropped and never handed out again.
namespace {
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
constexpr int kSlotDoubles = 4, kSlotsPerChunk = 256;
std::mutex g_slot_mu;
unsigned long long g_slot_ctx = 0;
std::vector<double*> g_slot_free;

unsigned long long slot_ctx_id() {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
  });
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (!get_cur || !get_id || get_cur(&c) != CUDA_SUCCESS || c == nullptr || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}
}  // namespace

// A slot of the current context (*ctx receives its id); nullptr on failure.
static double* slot_get(unsigned long long* ctx) {
  const unsigned long long id = slot_ctx_id();
  std::lock_guard<std::mutex> lk(g_slot_mu);
  if (id == 0 || id != g_slot_ctx) {
    g_slot_free.clear();
    g_slot_ctx = id;
  }
  if (id == 0) {   // no context id: a slot of its own, freed with the workspace
    void* p = nullptr;
    if (cudaHostAlloc(&p, sizeof(double) * kSlotDoubles, cudaHostAllocMapped) != cudaSuccess) return nullptr;
    *ctx = 0;
    return static_cast<double*>(p);
  }
  if (g_slot_free.empty()) {
    void* c = nullptr;
    if (cudaHostAlloc(&c, sizeof(double) * kSlotDoubles * kSlotsPerChunk, cudaHostAllocMapped | cudaHostAllocPortable) !=
        cudaSuccess)
      return nullptr;
    for (int i = kSlotsPerChunk - 1; i >= 0; --i) g_slot_free.push_back(static_cast<double*>(c) + i * kSlotDoubles);
  }
  double* p = g_slot_free.back();
  g_slot_free.pop_back();
  *ctx = id;
  return p;
}

static void slot_put(double* p, unsigned long long ctx) {
  if (!p) return;
  if (ctx == 0) {
    cudaFreeHost(p);
    return;
  }
  std::lock_guard<std::mutex> lk(g_slot_mu);
  if (ctx == g_slot_ctx) g_slot_free.push_back(p);
}

struct GmresState {
  int m = 0;
  int plain = 0;             // 1: the identity instead of the V-cycle
  Gm G;
  DevMem dj;                 // step index j of the current restart cycle
  double* st_host = nullptr; // pinned, mapped slot: {|g_{j+1}|, ||w||} of steps j even / odd
  double* st_dev = nullptr;  // the same memory as the device sees it
  unsigned long long st_ctx = 0;
  cudaEvent_t done[2] = {nullptr, nullptr};   // recorded after steps j even / odd
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;
  ~GmresState() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (cudaEvent_t e : done)
      if (e) cudaEventDestroy(e);
    slot_put(st_host, st_ctx);
  }
};

void gmres_release(bamg_hierarchy* h) {
  delete h->gm;
  h->gm = nullptr;
}

// One Arnoldi step j (read from the device): for j > 0 v_j = w / ||w|| from
// the previous step, z_j = C v_j (V-cycle, into Z_j and io_out), w = B z_j,
// two classical Gram-Schmidt passes, ||w|| and the Givens update of column j
// with {|g_{j+1}|, ||w||} to pinned memory, j <- j + 1.  Kernel nodes only
// (programmatic dependent launches).
static bamg_status arnoldi_body(bamg_hierarchy* h, GmresState& S, cudaStream_t s) {
  Level& L = h->lv[0];
  Gm& G = S.G;
  const int n = G.n, m = G.m;
  const unsigned gv = cdiv(n, 256);
  const int nb = red_blocks(n);
  int* dj = S.dj.as<int>();
  double* V = G.V.as<double>();
  double* Z = G.Z.as<double>();
  double* zo = h->io_out.as<double>();
  unsigned* arr = G.arrived.as<unsigned>();
  // for j > 0 the input kernel first forms v_j = w / ||w|| from the previous
  // step's w and reciprocal norm (scal[1])
  const double* wprev = G.w.as<double>();
  const double* rinv = G.scal.as<double>() + 1;
  if (S.plain)
    BAMG_TRY(launch(plain_io_kernel, dim3(gv), dim3(256), 0, s, n, (const int*)dj, V, wprev, rinv, zo, Z));
  else
    BAMG_TRY(h->mixed ? vcycle_body<float>(h, s, V, dj, zo, Z, wprev, rinv)
                      : vcycle_body<double>(h, s, V, dj, zo, Z, wprev, rinv));
  BAMG_TRY(csr_vec<double>(VEC_SPMV, n, L.vec_g, L.B.r(), L.B.c(), L.B.v(), L.dinv.as<double>(), 1.0,
                           (const double*)zo, nullptr, G.w.as<double>(), s));
  // classical Gram-Schmidt, twice: h1 = V^T w; w -= V h1, h2 = V^T w;
  // w -= V h2, ||w||
  double* h1 = G.h1.as<double>();
  double* h2 = G.h2.as<double>();
  const double* Vc = V;
  const GivensArgs none{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  const GivensArgs ga{h1, G.R.as<double>(), G.cs.as<double>(), G.sn.as<double>(), G.g.as<double>(), S.st_dev, dj};
  BAMG_TRY(launch(gs_kernel<kGsDots>, dim3(nb), dim3(256), 0, s, n, m, (const int*)dj, Vc, (size_t)n,
                  (const double*)nullptr, G.w.as<double>(), G.part.as<double>(), arr + kArrMultidot, h1, none));
  BAMG_TRY(launch(gs_kernel<kGsUpDots>, dim3(nb), dim3(256), 0, s, n, m, (const int*)dj, Vc, (size_t)n,
                  (const double*)h1, G.w.as<double>(), G.part.as<double>(), arr + kArrMultidot, h2, none));
  // the update, ||w||, the Givens update of column j and j <- j + 1
  return launch(gs_kernel<kGsUpNorm>, dim3(nb), dim3(256), 0, s, n, m, (const int*)dj, Vc, (size_t)n,
                (const double*)h2, G.w.as<double>(), G.part.as<double>(), arr + kArrNorm, G.scal.as<double>(), ga);
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
  BAMG_TRY(G.scal.alloc(sizeof(double) * 2, cs));
  BAMG_TRY(G.sums.alloc(sizeof(double) * 5, cs));
  BAMG_TRY(G.arrived.alloc(sizeof(unsigned) * kArrCount, cs));
  BAMG_TRY(S->dj.alloc(sizeof(int), cs));
  BAMG_CUDA(cudaMemsetAsync(G.zeros.p, 0, sizeof(double) * n, cs));
  BAMG_CUDA(cudaMemsetAsync(G.arrived.p, 0, sizeof(unsigned) * kArrCount, cs));
  S->st_host = slot_get(&S->st_ctx);
  if (!S->st_host) {
    set_error("pinned host memory for the Arnoldi status could not be allocated");
    return BAMG_ERR_OOM;
  }
  BAMG_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&S->st_dev), S->st_host, 0));
  for (cudaEvent_t& e : S->done) BAMG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  BAMG_CUDA(cudaStreamSynchronize(cs));
  uint64_t before = t_launches;
  BAMG_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  bamg_status st;
  {
    PdlScope pdl;
    st = arnoldi_body(h, *S, cs);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  if (st != BAMG_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  BAMG_CUDA(e);
  S->graph = g;
  if (std::getenv("BAMG_TRACE")) trace_edges("Arnoldi", g);
  BAMG_CUDA(cudaGraphInstantiate(&S->exec, g, 0));
  S->kernels = t_launches - before;
  g_launches.fetch_sub(S->kernels);  // counted at each replay
  return BAMG_OK;
}

bamg_status gmres_prepare_default(bamg_hierarchy* h) { return gmres_prepare(h, 20, 0); }

// Launches the next Arnoldi step (the graph) and records its event.
static bamg_status step_launch(GmresState& S, int& launched, cudaStream_t s) {
  BAMG_CUDA(cudaGraphLaunch(S.exec, s));
  g_launches.fetch_add(S.kernels);
  BAMG_CUDA(cudaEventRecord(S.done[launched & 1], s));
  ++launched;
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

  double rel = 0.0, xn1 = 1.0, xn2_0 = 0.0;
  BAMG_TRY(true_residual(h, G, x, &rel, &xn1, s, &xn2_0));
  const double xn1_0 = xn1;
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
    // Step j + 1 is launched before the host waits for step j, so the GPU is
    // not idle while the host reads the estimate, unless step j + 1 cannot be
    // used (end of the cycle or of max_iter) or the estimates so far predict
    // that step j meets the stopping test.  A step launched ahead and not
    // used writes only the column j + 1 entries of the Arnoldi state, which
    // the solution of step j does not read.
    int launched = 0;
    double est1 = -1.0, est2 = -1.0;   // estimates of the last two steps
    for (int j = 0; j < m && !done; ++j) {
      if (launched == j) BAMG_TRY(step_launch(S, launched, s));
      bool ahead = j + 1 < m && its + 1 < sp->max_iter;
      if (ahead && est1 > 0.0 && est2 > 0.0 && est1 * (est1 / est2) <= 2.0 * sp->tol * xn1_0) ahead = false;
      if (ahead) BAMG_TRY(step_launch(S, launched, s));
      BAMG_CUDA(cudaEventSynchronize(S.done[j & 1]));
      const volatile double* sh = S.st_host + 2 * (j & 1);
      const double st0 = sh[0], st1 = sh[1];
      est2 = est1;
      est1 = st0;
      const int K = j + 1;
      ++its;
      if (it7 < 0 && st0 <= 1e-7 * xn2_0) it7 = its;
      breakdown = !(st1 > 0.0);
      bool last = (j == m - 1) || its >= sp->max_iter || breakdown;
      if (st0 <= 2.0 * sp->tol * xn1_0 || last) {
        BAMG_TRY(launch(ysolve_kernel, dim3(1), dim3(32), sizeof(double) * ((size_t)(j + 1) * (kYsolveLd + 2)), s, j, m, (const double*)G.R.as<double>(),
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
  BAMG_CUDA(cudaStreamSynchronize(s));
  // rel is that of the final iterate before orient_normalise, which only
  // rescales it: ||B x||_1 / ||x||_1 does not change under scaling
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
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = 1.0 + 0.5 * splitmix_pm1(seed, 8193, (uint64_t)i);
}

__global__ void add_kernel(int n, const double* __restrict__ z, double* __restrict__ x) {
  pdl_wait();
  pdl_trigger();
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

template bamg_status vcycle_body<double>(bamg_hierarchy*, cudaStream_t, double*, const int*, double*, double*,
                                         const double*, const double*);
template bamg_status vcycle_body<float>(bamg_hierarchy*, cudaStream_t, double*, const int*, double*, double*,
                                        const double*, const double*);

}  // namespace bamg
