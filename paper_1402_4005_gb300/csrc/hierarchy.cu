// Setup phase: B = I - A and one bootstrap cycle (Algorithm 1) on the device.
//
// Top-down, level by level: relax the test-vector blocks V (with B) and U
// (with B^T, u^(1) = 1 fixed), normalise and weight them (eq. ls_weights),
// split C/F, fit P rows and Q columns (eq. ls_interpolation, Section 5),
// form B_{l+1} = Q B P, M_{l+1} = Q M Q^T, N_{l+1} = P^T N P, inject.  On the
// coarsest level, the r smallest generalized singular triplets and B_L^+.
// Bottom-up: interpolate the triplets (Q^T u, P v) and relax the
// inhomogeneous systems B v = sigma M u, B^T u = sigma N v with the Rayleigh
// quotient update (eq. singular_value).  Only sizes are read back to the
// host; all arithmetic runs in the kernels.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "hierarchy.cuh"

namespace bamg {

// Optional phase timing (BAMG_TRACE set): synchronises the stream at each
// mark and prints the elapsed host time to stderr.
struct Trace {
  bool on = std::getenv("BAMG_TRACE") != nullptr;
  std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
  void mark(cudaStream_t s, const char* what, int level) {
    if (!on) return;
    cudaStreamSynchronize(s);
    auto now = std::chrono::steady_clock::now();
    fprintf(stderr, "[bamg] L%d %-18s %8.3f ms\n", level, what,
            std::chrono::duration<double, std::milli>(now - t).count());
    t = now;
  }
};

// ------------------------------------------------------------ small kernels
__global__ void pad_block_kernel(int n, int r, int ld, const double* __restrict__ src, float* __restrict__ d32,
                                 double* __restrict__ d64) {
  pdl_wait();
  pdl_trigger();
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * ld) return;
  int i = (int)(t / ld), k = (int)(t % ld);
  double v = k < r ? src[(size_t)i * r + k] : 0.0;
  if (d32) d32[t] = (float)v;
  if (d64) d64[t] = v;
}

__global__ void column_kernel(int n, int ld, int k, const double* __restrict__ X, double* __restrict__ x) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = X[(size_t)i * ld + k];
}

// partial sums of x and |x| per block
__global__ void sum_abs_kernel(int n, const double* __restrict__ x, double* __restrict__ part) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[2][8];
  double s = 0.0, a = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    s += x[i];
    a += fabs(x[i]);
  }
  s = warp_sum(s); a = warp_sum(a);
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sh[0][w] = s; sh[1][w] = a; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ts = 0, ta = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { ts += sh[0][k]; ta += sh[1][k]; }
    part[2 * blockIdx.x] = ts;
    part[2 * blockIdx.x + 1] = ta;
  }
}

// x <- x * sign(sum) / ||x||_1  (positive orientation, unit 1-norm)
__global__ void orient_kernel(int n, const double* __restrict__ sums, double* __restrict__ x) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double f = (sums[0] < 0.0 ? -1.0 : 1.0) / sums[1];
  x[i] *= f;
}

bamg_status abs_sums(int n, const double* x, double* out, cudaStream_t s) {
  int nb = (int)cdiv(n, 256);
  if (nb > 4 * num_sms()) nb = 4 * num_sms();
  DevMem part;
  BAMG_TRY(part.alloc(sizeof(double) * 2 * nb, s));
  BAMG_TRY(launch(sum_abs_kernel, dim3(nb), dim3(256), 0, s, n, x, part.as<double>()));
  return reduce_partials(part.as<double>(), nb, 2, out, s);
}

bamg_status orient_normalise(int n, double* x, cudaStream_t s) {
  DevMem sums;
  BAMG_TRY(sums.alloc(sizeof(double) * 2, s));
  BAMG_TRY(abs_sums(n, x, sums.as<double>(), s));
  return launch(orient_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n, (const double*)sums.as<double>(), x);
}

// ------------------------------------------------------------ csr helpers
static bamg_status csr_transpose(const Csr& A, Csr& T, cudaStream_t s) {
  BAMG_TRY(T.alloc(A.cols, A.rows, A.nnz, s));
  return transpose_csr(A.rows, A.cols, A.nnz, A.r(), A.c(), A.v(), T.rp.as<int32_t>(), T.ci.as<int32_t>(),
                       T.va.as<double>(), s);
}

static bamg_status csr_products(const std::vector<std::pair<const Csr*, const Csr*>>& ab,
                                const std::vector<Csr*>& out, cudaStream_t s) {
  std::vector<SpgemmJob> jobs(ab.size());
  for (size_t q = 0; q < ab.size(); ++q) {
    const Csr& A = *ab[q].first;
    const Csr& B = *ab[q].second;
    Csr& C = *out[q];
    jobs[q] = SpgemmJob{A.rows, A.r(), A.c(), A.v(), B.r(), B.c(), B.v(), &C.rp, &C.ci, &C.va, 0};
    jobs[q].annz = A.nnz;
    jobs[q].maxrow_b = B.maxrow;
  }
  BAMG_TRY(spgemm_multi(jobs.data(), (int)jobs.size(), s));
  for (size_t q = 0; q < ab.size(); ++q) {
    Csr& C = *out[q];
    C.rows = ab[q].first->rows;
    C.cols = ab[q].second->cols;
    C.nnz = (int)jobs[q].nnz;
    C.maxrow = jobs[q].maxrow_c;
  }
  return BAMG_OK;
}

// B^T, 1/diag(B) (Jacobi needs b_ii > 0: Section 3 / coarse levels), lanes.
static bamg_status finish_level(bamg_hierarchy* h, Level& L, int l, cudaStream_t s) {
  L.n = L.B.rows;
  BAMG_TRY(csr_transpose(L.B, L.Bt, s));
  BAMG_TRY(L.dinv.alloc(sizeof(double) * L.n, s));
  // flags: {first row whose row and column are zero (0x7F7F7F7F = none),
  // rows with the l1 divisor}; read for all levels at the end of the setup
  BAMG_TRY(L.dflags.alloc(2 * sizeof(int), s));
  BAMG_CUDA(cudaMemsetAsync(L.dflags.p, 0x7F, sizeof(int), s));
  BAMG_CUDA(cudaMemsetAsync(L.dflags.as<int>() + 1, 0, sizeof(int), s));
  BAMG_TRY(diag_inv<double>(L.n, L.B.r(), L.B.c(), L.B.v(), L.Bt.r(), L.Bt.v(), L.dinv.as<double>(),
                            L.dflags.as<int>(), L.dflags.as<int>() + 1, s));
  (void)l;
  double avg = L.n ? (double)L.B.nnz / L.n : 1.0;
  L.vec_g = vec_lanes(avg);
  if (h->mixed) {
    ConvMany job;
    BAMG_TRY(L.B.add32(job, s));
    BAMG_TRY(L.Bt.add32(job, s));
    BAMG_TRY(L.dinv32.alloc(sizeof(float) * L.n, s));
    job.src[job.k] = L.dinv.as<double>();
    job.dst[job.k] = L.dinv32.as<float>();
    job.n[job.k++] = (size_t)L.n;
    if (!L.M.empty()) BAMG_TRY(L.M.add32(job, s));
    if (!L.N.empty()) BAMG_TRY(L.N.add32(job, s));
    BAMG_TRY(convert_many(job, s));
  }
  return BAMG_OK;
}

template <typename T> static const T* dinv_of(const Level& L);
template <> const double* dinv_of<double>(const Level& L) { return L.dinv.as<double>(); }
template <> const float* dinv_of<float>(const Level& L) { return L.dinv32.as<float>(); }

static bool is_coarsest(const bamg_hierarchy* h, const Level& L, int l) {
  const bamg_params& p = h->p;
  if (l + 1 >= p.max_levels || L.n <= p.coarse_min) return true;
  if (p.coarsening == BAMG_COARSEN_GEOMETRIC && (L.nx < 3 && L.ny < 3)) return true;
  return false;
}

template <typename T>
static bamg_status relax_triplets(bamg_hierarchy* h, int l, DevMem& U, DevMem& V, DevMem& sig, DevMem& sig64,
                                  cudaStream_t s);

// ------------------------------------------------------------ one level down
// inhomog: a subsequent bootstrap cycle, whose first smoothing is the
// inhomogeneous one with the sigma update (the smoothing of the last loop
// of Algorithm 1) on the carried triplets.
template <typename T>
static bamg_status coarsen_level(bamg_hierarchy* h, int l, DevMem& U, DevMem& V, DevMem& Uc, DevMem& Vc,
                                 DevMem& tmpU, DevMem& tmpV, DevMem& scale, DevMem& norms, DevMem& rkd,
                                 DevMem& sig, DevMem& sig64, bool inhomog, cudaStream_t s) {
  const bamg_params& p = h->p;
  const int ld = h->ld, r = p.r;
  Level& L = h->lv[l];
  const T om = T(p.omega);
  const T* Bv = L.B.vals<T>();
  const T* Btv = L.Bt.vals<T>();
  const T* dv = dinv_of<T>(L);
  Trace tr;
  const bool learned = h->learned != 0;
  // Algorithm 1, first smoothing loop: relax V with B and U with B^T
  // (not needed when the network proposes the fits)
  if (inhomog && !learned) BAMG_TRY(relax_triplets<T>(h, l, U, V, sig, sig64, s));
  {
    PdlScope pdl;   // block relaxations only, each waiting for its predecessor
    for (int it = 0; !learned && !inhomog && it < p.nu_setup; ++it) {
      BAMG_TRY(relax_block2<T>(L.n, ld, L.B.r(), L.B.c(), Bv, L.Bt.r(), L.Bt.c(), Btv, dv, V.as<T>(),
                               tmpV.as<T>(), U.as<T>(), tmpU.as<T>(), nullptr, nullptr, nullptr, om, 1, s));
      std::swap(V, tmpV);
      std::swap(U, tmpU);
    }
  }
  tr.mark(s, "relax", l);
  // eq. ls_weights with unit vectors
  if (!learned) {
    BAMG_TRY(L.s.alloc(sizeof(double) * ld, s));
    BAMG_TRY(L.t.alloc(sizeof(double) * ld, s));
    BAMG_TRY(norms_weights<T>(L.n, ld, r, L.B.r(), L.B.c(), Bv, V.as<T>(), 1, 0, scale.as<T>(),
                              L.s.as<double>(), norms.as<double>(), s));
    BAMG_TRY(norms_weights<T>(L.n, ld, r, L.Bt.r(), L.Bt.c(), Btv, U.as<T>(), 1, 1, scale.as<T>(),
                              L.t.as<double>(), norms.as<double>(), s));
    tr.mark(s, "weights", l);
  }
  // C/F splitting and interpolation sets
  BAMG_TRY(L.cf.alloc(L.n, s));
  BAMG_TRY(L.cmap.alloc(sizeof(int32_t) * L.n, s));
  BAMG_TRY(L.Jrp.alloc(sizeof(int32_t) * (L.n + 1), s));
  int nc = 0;
  int cgx = 0, cgy = 0;
  if (p.coarsening == BAMG_COARSEN_GEOMETRIC) {
    BAMG_TRY(L.Jci.alloc(sizeof(int32_t) * 4 * (size_t)L.n, s));
    BAMG_TRY(coarsen_geometric(L.nx, L.ny, L.cf.as<int8_t>(), L.cmap.as<int32_t>(), L.Jrp.as<int32_t>(),
                               L.Jci.as<int32_t>(), &nc, s));
    cgx = (L.nx + 1) / 2;
    cgy = (L.ny + 1) / 2;
  } else {
    BAMG_TRY(coarsen_mis(L.n, L.B.r(), L.B.c(), L.Bt.r(), L.Bt.c(), p.seed, l, L.cf.as<int8_t>(),
                         L.cmap.as<int32_t>(), &nc, s));
    BAMG_TRY(L.Jci.alloc(sizeof(int32_t) * (size_t)p.c_max * L.n, s));
    BAMG_TRY(graph_sets(L.n, L.B.r(), L.B.c(), L.B.v(), L.Bt.r(), L.Bt.c(), L.Bt.v(), L.cf.as<int8_t>(),
                        p.c_min, p.c_max, L.Jrp.as<int32_t>(), L.Jci.as<int32_t>(), s));
  }
  if (nc < 1 || nc >= L.n) {
    set_error("level %d: coarsening produced %d coarse points of %d", l, nc, L.n);
    return BAMG_ERR_NUMERIC;
  }
  L.nc = nc;
  BAMG_TRY(L.cpt.alloc(sizeof(int32_t) * nc, s));
  BAMG_TRY(coarse_points(L.n, L.cf.as<int8_t>(), L.cmap.as<int32_t>(), L.cpt.as<int32_t>(), s));
  int32_t njz = 0;
  if (p.coarsening == BAMG_COARSEN_GEOMETRIC) {
    // |J_i| summed over the fine points in closed form: per dimension of
    // size N the odd indices contribute 2 coarse neighbours each, the last
    // one only 1 when N is even (S_N), and E_N = ceil(N / 2) indices are even
    auto S = [](int N) { return 2 * (N / 2) - (N % 2 == 0 ? 1 : 0); };
    auto E = [](int N) { return (N + 1) / 2; };
    njz = S(L.nx) * E(L.ny) + E(L.nx) * S(L.ny) + S(L.nx) * S(L.ny);
  } else {
    BAMG_CUDA(cudaMemcpyAsync(&njz, L.Jrp.as<int32_t>() + L.n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    BAMG_CUDA(cudaStreamSynchronize(s));
  }
  tr.mark(s, "split+sets", l);
  // P rows and Q columns (eq. ls_interpolation; Section 5)
  DevMem fitP, fitQ;
  BAMG_TRY(fitP.alloc(sizeof(double) * (njz > 0 ? njz : 1), s));
  BAMG_TRY(fitQ.alloc(sizeof(double) * (njz > 0 ? njz : 1), s));
  if (learned) {
    BAMG_TRY(mlp_fits(L, h->mlp.as<float>(), fitP.as<double>(), fitQ.as<double>(), s));
    if (p.restriction == BAMG_RESTRICT_AVERAGE) BAMG_TRY(average_fits(L.n, L.Jrp.as<int32_t>(), fitQ.as<double>(), s));
  } else {
    BAMG_TRY(ls_fit<T>(L.n, ld, r, L.Jrp.as<int32_t>(), L.Jci.as<int32_t>(), V.as<T>(), L.s.as<double>(), 0,
                       fitP.as<double>(), rkd.as<int>(), s, p.ls_ridge));
    if (p.restriction == BAMG_RESTRICT_AVERAGE)
      BAMG_TRY(average_fits(L.n, L.Jrp.as<int32_t>(), fitQ.as<double>(), s));
    else
      BAMG_TRY(ls_fit<T>(L.n, ld, r, L.Jrp.as<int32_t>(), L.Jci.as<int32_t>(), U.as<T>(), L.t.as<double>(), 1,
                         fitQ.as<double>(), rkd.as<int>(), s, p.ls_ridge));
  }
  int nnzP = njz + nc;
  // rows of P and Q^T: |J_i| entries for an F point (at most 4 for the
  // geometric sets, c_max for the graph sets), one for a C point
  const int set_max = p.coarsening == BAMG_COARSEN_GEOMETRIC ? 4 : (p.c_max > 1 ? p.c_max : 1);
  for (Csr* X : {&L.P, &L.Qt}) {
    BAMG_TRY(X->alloc(L.n, nc, nnzP, s));
    X->maxrow = set_max;
    BAMG_TRY(transfer_pattern(L.n, L.cf.as<int8_t>(), L.cmap.as<int32_t>(), L.Jrp.as<int32_t>(),
                              L.Jci.as<int32_t>(), X->rp.as<int32_t>(), X->ci.as<int32_t>(),
                              X->va.as<double>(), s));
  }
  BAMG_TRY(scatter_fits(L.n, L.cf.as<int8_t>(), L.Jrp.as<int32_t>(), fitP.as<double>(), L.P.r(),
                        L.P.va.as<double>(), s));
  BAMG_TRY(scatter_fits(L.n, L.cf.as<int8_t>(), L.Jrp.as<int32_t>(), fitQ.as<double>(), L.Qt.r(),
                        L.Qt.va.as<double>(), s));
  tr.mark(s, "ls fits", l);
  BAMG_TRY(csr_transpose(L.Qt, L.Q, s));
  BAMG_TRY(csr_transpose(L.P, L.Pt, s));
  tr.mark(s, "transposes", l);
  // Petrov-Galerkin operators (Section 3; Algorithm 1)
  h->lv.emplace_back();
  Level& Lc = h->lv[l + 1];
  Level& Lf = h->lv[l];
  {
    // two rounds of independent products: B P, M Q^T (or Q Q^T), N P (or
    // P^T P); then Q (B P), Q (M Q^T), P^T (N P)
    Csr BP, MQt, NP;
    std::vector<std::pair<const Csr*, const Csr*>> ab;
    std::vector<Csr*> out;
    ab.push_back({&Lf.B, &Lf.P}); out.push_back(&BP);
    if (Lf.M.empty()) { ab.push_back({&Lf.Q, &Lf.Qt}); out.push_back(&Lc.M); }
    else { ab.push_back({&Lf.M, &Lf.Qt}); out.push_back(&MQt); }
    if (Lf.N.empty()) { ab.push_back({&Lf.Pt, &Lf.P}); out.push_back(&Lc.N); }
    else { ab.push_back({&Lf.N, &Lf.P}); out.push_back(&NP); }
    BAMG_TRY(csr_products(ab, out, s));
    ab.clear();
    out.clear();
    ab.push_back({&Lf.Q, &BP}); out.push_back(&Lc.B);
    if (!Lf.M.empty()) { ab.push_back({&Lf.Q, &MQt}); out.push_back(&Lc.M); }
    if (!Lf.N.empty()) { ab.push_back({&Lf.Pt, &NP}); out.push_back(&Lc.N); }
    BAMG_TRY(csr_products(ab, out, s));
  }
  tr.mark(s, "galerkin spgemm", l);
  Lc.nx = cgx;
  Lc.ny = cgy;
  BAMG_TRY(finish_level(h, Lc, l + 1, s));
  tr.mark(s, "finish coarse", l);
  if (h->mixed) {
    ConvMany job;
    BAMG_TRY(Lf.P.add32(job, s));
    BAMG_TRY(Lf.Qt.add32(job, s));
    BAMG_TRY(Lf.Q.add32(job, s));
    BAMG_TRY(convert_many(job, s));
  }
  if (learned) return BAMG_OK;
  // injection of the test vectors
  BAMG_TRY(Uc.alloc(sizeof(T) * (size_t)nc * ld, s));
  BAMG_TRY(Vc.alloc(sizeof(T) * (size_t)nc * ld, s));
  BAMG_TRY(inject<T>(nc, ld, Lf.cpt.as<int32_t>(), U.as<T>(), Uc.as<T>(), s));
  BAMG_TRY(inject<T>(nc, ld, Lf.cpt.as<int32_t>(), V.as<T>(), Vc.as<T>(), s));
  tr.mark(s, "inject", l);
  return BAMG_OK;
}

// Inhomogeneous relaxation with the Rayleigh update on level l.
template <typename T>
static bamg_status relax_triplets(bamg_hierarchy* h, int l, DevMem& U, DevMem& V, DevMem& sig, DevMem& sig64,
                                  cudaStream_t s) {
  // a chain of small dependent kernels (block relaxation, block products,
  // column dots, partial sums, Rayleigh quotients), each of which waits for
  // its predecessor first: launched with programmatic serialisation
  PdlScope pdl;
  const bamg_params& p = h->p;
  const int ld = h->ld, r = p.r;
  Level& L = h->lv[l];
  size_t bytes = sizeof(T) * (size_t)L.n * ld;
  DevMem tU, tV, MU, NV, BV, sums;
  BAMG_TRY(tU.alloc(bytes, s));
  BAMG_TRY(tV.alloc(bytes, s));
  BAMG_TRY(BV.alloc(bytes, s));
  if (!L.M.empty()) BAMG_TRY(MU.alloc(bytes, s));
  if (!L.N.empty()) BAMG_TRY(NV.alloc(bytes, s));
  BAMG_TRY(sums.alloc(sizeof(double) * 3 * ld, s));
  const T om = T(p.omega);
  const T* dv = dinv_of<T>(L);
  const bool hasM = !L.M.empty(), hasN = !L.N.empty();
  // M U and N V of the current iterates (reused: U and V do not change
  // between the Rayleigh update of one sweep and the relaxation of the next)
  auto mass_products = [&](bool withB) -> bamg_status {
    SpmmJob<T> jobs[3];
    int k = 0;
    if (withB) jobs[k++] = SpmmJob<T>{L.n, L.B.r(), L.B.c(), L.B.vals<T>(), V.as<T>(), BV.as<T>()};
    if (hasM) jobs[k++] = SpmmJob<T>{L.n, L.M.r(), L.M.c(), L.M.vals<T>(), U.as<T>(), MU.as<T>()};
    if (hasN) jobs[k++] = SpmmJob<T>{L.n, L.N.r(), L.N.c(), L.N.vals<T>(), V.as<T>(), NV.as<T>()};
    return k ? spmm_block_multi<T>(ld, jobs, k, s) : BAMG_OK;
  };
  BAMG_TRY(mass_products(false));
  for (int it = 0; it < p.nu_setup; ++it) {
    const T* mu = hasM ? MU.as<T>() : U.as<T>();
    const T* nv = hasN ? NV.as<T>() : V.as<T>();
    // both from the previous iterates (Algorithm 1, second smoothing loop)
    BAMG_TRY(relax_block2<T>(L.n, ld, L.B.r(), L.B.c(), L.B.vals<T>(), L.Bt.r(), L.Bt.c(), L.Bt.vals<T>(), dv,
                             V.as<T>(), tV.as<T>(), U.as<T>(), tU.as<T>(), mu, nv, sig.as<T>(), om, 0, s));
    std::swap(U, tU);
    std::swap(V, tV);
    // eq. singular_value
    BAMG_TRY(mass_products(true));
    mu = hasM ? MU.as<T>() : U.as<T>();
    nv = hasN ? NV.as<T>() : V.as<T>();
    BAMG_TRY(col_dots<T>(L.n, ld, 3, U.as<T>(), BV.as<T>(), U.as<T>(), mu, V.as<T>(), nv, sums.as<double>(), s));
    BAMG_TRY(rayleigh_finalize<T>(sums.as<double>(), ld, r, sig.as<T>(), sig64.as<double>(), s));
  }
  return BAMG_OK;
}

// The divisor flags of every level in one read: rows with the l1 divisor per
// level, and an error for a zero row and column.
static bamg_status check_levels(bamg_hierarchy* h, cudaStream_t s) {
  std::vector<int> f(2 * h->lv.size(), 0);
  for (size_t l = 0; l < h->lv.size(); ++l)
    BAMG_CUDA(cudaMemcpyAsync(&f[2 * l], h->lv[l].dflags.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  for (size_t l = 0; l < h->lv.size(); ++l) {
    if (f[2 * l] != 0x7F7F7F7F) {
      set_error("level %zu: row and column %d of B are zero", l, f[2 * l]);
      return BAMG_ERR_NUMERIC;
    }
    h->lv[l].nsafe = f[2 * l + 1];
  }
  return BAMG_OK;
}

// x = column k of the n x ld block V, k the first index of the smallest
// |sigma_k| among k < rr
__global__ void x0_column_kernel(int n, int ld, int rr, const double* __restrict__ sig,
                                 const double* __restrict__ V, double* __restrict__ x) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int kmin = 0;
  for (int k = 1; k < rr; ++k)
    if (fabs(sig[k]) < fabs(sig[kmin])) kmin = k;
  x[i] = V[(size_t)i * ld + kmin];
}

// out = {dflags of every level (2 each), rankdef, coarsest status, sigma[0..ld)}
constexpr int kFlagLevels = 64;
struct SetupFlags {
  const int* dflags[kFlagLevels];
  int nlev;
  const int* rkd;
  const int* cerr;
  const double* sig;
  int ld;
};
__global__ void setup_flags_kernel(SetupFlags f, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  const int t = threadIdx.x;
  for (int l = t; l < f.nlev; l += blockDim.x) {
    out[2 * l] = f.dflags[l][0];
    out[2 * l + 1] = f.dflags[l][1];
  }
  if (t == 0) {
    out[2 * f.nlev] = f.rkd[0];
    out[2 * f.nlev + 1] = f.cerr ? f.cerr[0] : 0;
  }
  for (int k = t; k < f.ld; k += blockDim.x) out[2 * f.nlev + 2 + k] = f.sig[k];
}

static bamg_status setup_flags(bamg_hierarchy* h, cudaStream_t s, const int* rkd, const int* cerr,
                               const double* sig, int ld) {
  const int nlev = (int)h->lv.size();
  if (nlev > kFlagLevels) {
    set_error("%d levels exceed the %d the setup supports", nlev, kFlagLevels);
    return BAMG_ERR_UNSUPPORTED;
  }
  SetupFlags f = {};
  for (int l = 0; l < nlev; ++l) f.dflags[l] = h->lv[l].dflags.as<int>();
  f.nlev = nlev;
  f.rkd = rkd;
  f.cerr = cerr;
  f.sig = sig;
  f.ld = ld;
  const int total = 2 * nlev + 2 + ld;
  DevMem out;
  BAMG_TRY(out.alloc(sizeof(double) * total, s));
  BAMG_TRY(launch(setup_flags_kernel, dim3(1), dim3(64), 0, s, f, out.as<double>()));
  std::vector<double> hv(total);
  BAMG_CUDA(cudaMemcpyAsync(hv.data(), out.p, sizeof(double) * total, cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  if ((int)hv[2 * nlev + 1] == 2) {
    set_error("coarsest level: M or N is not positive definite");
    return BAMG_ERR_NUMERIC;
  }
  for (int l = 0; l < nlev; ++l) {
    const int zr = (int)hv[2 * l];
    if (zr != 0x7F7F7F7F) {
      set_error("level %d: row and column %d of B are zero", l, zr);
      return BAMG_ERR_NUMERIC;
    }
    h->lv[l].nsafe = (int)hv[2 * l + 1];
  }
  h->rankdef = (int)hv[2 * nlev];
  h->sigma.assign(hv.begin() + 2 * nlev + 2, hv.end());
  return BAMG_OK;
}

static void complexities(bamg_hierarchy* h) {
  // eq. operator_complexity_def; Section 7
  double nnz_sum = 0, n_sum = 0;
  for (auto& L : h->lv) { nnz_sum += L.B.nnz; n_sum += L.n; }
  h->op_cplx = nnz_sum / h->lv[0].B.nnz;
  h->grid_cplx = n_sum / h->lv[0].n;
}

// Setup with network fits: no test vectors to carry up, so only the right
// singular vector of the smallest coarsest |sigma| is interpolated (v <- P v)
// and smoothed towards B v = 0 on each level on the way up (the sigma = 0
// case of the inhomogeneous relaxation); it becomes x^(0).
static bamg_status learned_unwind(bamg_hierarchy* h, int l, int rr, const double* Vd, const double* sg,
                                  cudaStream_t s) {
  std::vector<double> sig(rr);
  BAMG_CUDA(cudaMemcpyAsync(sig.data(), sg, sizeof(double) * rr, cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  int kmin = 0;
  for (int k = 1; k < rr; ++k)
    if (std::fabs(sig[k]) < std::fabs(sig[kmin])) kmin = k;
  h->sigma = sig;
  h->sigma.resize(h->p.r, 0.0);
  const int nL = h->lv[l].n;
  DevMem x, y, zero;
  BAMG_TRY(x.alloc(sizeof(double) * nL, s));
  BAMG_TRY(launch(column_kernel, dim3(cdiv(nL, 256)), dim3(256), 0, s, nL, rr, kmin, Vd, x.as<double>()));
  for (int k = l - 1; k >= 0; --k) {
    Level& L = h->lv[k];
    BAMG_TRY(y.alloc(sizeof(double) * L.n, s));
    BAMG_TRY(zero.alloc(sizeof(double) * L.n, s));
    BAMG_CUDA(cudaMemsetAsync(zero.p, 0, sizeof(double) * L.n, s));
    int gp = (L.P.rows && L.P.nnz / L.P.rows > 2) ? 4 : 2;
    BAMG_TRY(csr_vec<double>(VEC_SPMV, L.n, gp, L.P.r(), L.P.c(), L.P.v(), nullptr, 0.0, x.as<double>(), nullptr,
                             y.as<double>(), s));
    std::swap(x, y);
    BAMG_TRY(y.alloc(sizeof(double) * L.n, s));
    for (int it = 0; it < h->p.nu_setup; ++it) {
      BAMG_TRY(csr_vec<double>(VEC_JACOBI, L.n, L.vec_g, L.B.r(), L.B.c(), L.B.v(), L.dinv.as<double>(),
                               h->p.omega, x.as<double>(), zero.as<double>(), y.as<double>(), s));
      std::swap(x, y);
    }
  }
  h->x0 = std::move(x);
  BAMG_TRY(orient_normalise(h->lv[0].n, h->x0.as<double>(), s));
  BAMG_TRY(check_levels(h, s));
  complexities(h);
  return BAMG_OK;
}

template <typename T>
static bamg_status run_setup(bamg_hierarchy* h, cudaStream_t s) {
  const bamg_params& p = h->p;
  const int ld = h->ld, r = p.r;
  const bool learned = h->learned != 0;
  std::vector<DevMem> U(1), V(1);
  int n0 = h->lv[0].n;
  if (!learned) {
    BAMG_TRY(U[0].alloc(sizeof(T) * (size_t)n0 * ld, s));
    BAMG_TRY(V[0].alloc(sizeof(T) * (size_t)n0 * ld, s));
    BAMG_TRY(init_vectors<T>(n0, ld, r, p.seed, U[0].as<T>(), V[0].as<T>(), s));
  }
  DevMem scale, norms, rkd, sig, sig64, coarse_err;
  BAMG_TRY(scale.alloc(sizeof(T) * ld, s));
  BAMG_TRY(norms.alloc(sizeof(double) * ld, s));
  BAMG_TRY(rkd.alloc(2 * sizeof(int), s));
  BAMG_TRY(sig.alloc(sizeof(T) * ld, s));
  BAMG_TRY(sig64.alloc(sizeof(double) * ld, s));
  BAMG_CUDA(cudaMemsetAsync(rkd.p, 0, 2 * sizeof(int), s));
  // bootstrap cycles: each later cycle rebuilds the hierarchy below the
  // finest level from the previous cycle's finest triplets (Section 4)
  const int cycles = learned ? 1 : p.setup_cycles;
  int rr = r;   // triplets the coarsest level provides (min(r, n_L))
  for (int cyc = 0; cyc < cycles; ++cyc) {
    if (cyc > 0) {
      h->lv.resize(1);
      U.resize(1);
      V.resize(1);
    }
    int l = 0;
    while (!is_coarsest(h, h->lv[l], l)) {
      DevMem tU, tV;
      size_t bytes = sizeof(T) * (size_t)h->lv[l].n * ld;
      if (!learned) {
        BAMG_TRY(tU.alloc(bytes, s));
        BAMG_TRY(tV.alloc(bytes, s));
      }
      U.emplace_back();
      V.emplace_back();
      BAMG_TRY(coarsen_level<T>(h, l, U[l], V[l], U[l + 1], V[l + 1], tU, tV, scale, norms, rkd, sig, sig64,
                                cyc > 0, s));
      ++l;
    }
    // coarsest level: eq. generalized_eigenvalue and the pseudo-inverse
    Trace tr;
    Level& LL = h->lv[l];
    int nL = LL.n;
    h->nL = nL;
    rr = r < nL ? r : nL;
    DevMem Bd, Md, Nd, sg, Ud, Vd;
    size_t nn = (size_t)nL * nL;
    BAMG_TRY(Bd.alloc(sizeof(double) * nn, s));
    BAMG_TRY(Md.alloc(sizeof(double) * nn, s));
    BAMG_TRY(Nd.alloc(sizeof(double) * nn, s));
    BAMG_TRY(sg.alloc(sizeof(double) * r, s));
    BAMG_TRY(Ud.alloc(sizeof(double) * (size_t)nL * r, s));
    BAMG_TRY(Vd.alloc(sizeof(double) * (size_t)nL * r, s));
    BAMG_CUDA(cudaMemsetAsync(sg.p, 0, sizeof(double) * r, s));
    BAMG_CUDA(cudaMemsetAsync(Ud.p, 0, sizeof(double) * (size_t)nL * r, s));
    BAMG_CUDA(cudaMemsetAsync(Vd.p, 0, sizeof(double) * (size_t)nL * r, s));
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
    BAMG_TRY(h->Bpinv.alloc(sizeof(double) * nn, s));
    if (h->mixed) BAMG_TRY(h->Bpinv32.alloc(sizeof(float) * nn, s));
    // In the last bootstrap cycle every level the V-cycle reads exists now:
    // its graph and the Arnoldi graph are captured on the host while the
    // coarsest kernels run (capture records pointers only).
    struct Early {
      bamg_hierarchy* h;
      cudaStream_t s;
    } early{h, s};
    HostWork during;
    if (h->prep_early && cyc == cycles - 1 && p.smoother == BAMG_SMOOTH_JACOBI) {
      during.ctx = &early;
      during.fn = [](void* c) -> bamg_status {
        Early* e = static_cast<Early*>(c);
        BAMG_TRY(vcycle_prepare(e->h, e->s));
        return gmres_prepare_default(e->h);
      };
    }
    // Ud/Vd are nL x rr row-major (rr <= r).  The coarsest kernels' status is
    // read with the setup's final flags (LS setups): the host queues the
    // bottom-up work while they run.
    if (!learned) {
      BAMG_TRY(coarse_err.alloc(sizeof(int), s));
      BAMG_CUDA(cudaMemsetAsync(coarse_err.p, 0, sizeof(int), s));
    }
    BAMG_TRY(coarsest_solve(h->mixed ? 1 : 0, nL, rr, Bd.as<double>(), Md.as<double>(), Nd.as<double>(),
                            sg.as<double>(), Ud.as<double>(), Vd.as<double>(), h->Bpinv.as<double>(), s, during,
                            learned ? nullptr : coarse_err.as<int>()));
    if (h->mixed) BAMG_TRY(convert<double, float>(nn, h->Bpinv.as<double>(), h->Bpinv32.as<float>(), s));
    tr.mark(s, "coarsest solve", l);
    if (learned) return learned_unwind(h, l, rr, Vd.as<double>(), sg.as<double>(), s);
    // triplets into padded blocks
    BAMG_TRY(U[l].alloc(sizeof(T) * (size_t)nL * ld, s));
    BAMG_TRY(V[l].alloc(sizeof(T) * (size_t)nL * ld, s));
    unsigned g = cdiv((long long)nL * ld, 256);
    float* f32 = nullptr;
    double* f64 = nullptr;
    if (sizeof(T) == 4) f32 = (float*)U[l].p; else f64 = (double*)U[l].p;
    BAMG_TRY(launch(pad_block_kernel, dim3(g), dim3(256), 0, s, nL, rr, ld, (const double*)Ud.as<double>(), f32, f64));
    if (sizeof(T) == 4) f32 = (float*)V[l].p; else f64 = (double*)V[l].p;
    BAMG_TRY(launch(pad_block_kernel, dim3(g), dim3(256), 0, s, nL, rr, ld, (const double*)Vd.as<double>(), f32, f64));
    {
      unsigned g1 = cdiv(ld, 256);
      if (sizeof(T) == 4) { f32 = (float*)sig.p; f64 = nullptr; } else { f64 = (double*)sig.p; f32 = nullptr; }
      BAMG_TRY(launch(pad_block_kernel, dim3(g1), dim3(256), 0, s, 1, rr, ld, (const double*)sg.as<double>(), f32, f64));
      BAMG_TRY(launch(pad_block_kernel, dim3(g1), dim3(256), 0, s, 1, rr, ld, (const double*)sg.as<double>(),
                      (float*)nullptr, sig64.as<double>()));
    }
    // bottom-up: interpolate and relax (Algorithm 1, last loop)
    for (int k = l - 1; k >= 0; --k) {
      Level& L = h->lv[k];
      {
        PdlScope pdl;
        BAMG_TRY(spmm_block<T>(L.n, ld, L.Qt.r(), L.Qt.c(), L.Qt.vals<T>(), U[k + 1].as<T>(), U[k].as<T>(), s));
        BAMG_TRY(spmm_block<T>(L.n, ld, L.P.r(), L.P.c(), L.P.vals<T>(), V[k + 1].as<T>(), V[k].as<T>(), s));
      }
      BAMG_TRY(relax_triplets<T>(h, k, U[k], V[k], sig, sig64, s));
      tr.mark(s, "bottom-up relax", k);
      U[k + 1].release();
      V[k + 1].release();
    }
  }
  // finest triplets, x^(0) = v of the smallest |sigma| (chosen on the device)
  BAMG_TRY(h->U64.alloc(sizeof(double) * (size_t)n0 * ld, s));
  BAMG_TRY(h->V64.alloc(sizeof(double) * (size_t)n0 * ld, s));
  BAMG_TRY(convert<T, double>((size_t)n0 * ld, U[0].as<T>(), h->U64.as<double>(), s));
  BAMG_TRY(convert<T, double>((size_t)n0 * ld, V[0].as<T>(), h->V64.as<double>(), s));
  BAMG_TRY(h->x0.alloc(sizeof(double) * n0, s));
  BAMG_TRY(launch(x0_column_kernel, dim3(cdiv(n0, 256)), dim3(256), 0, s, n0, ld, rr,
                  (const double*)sig64.as<double>(), (const double*)h->V64.as<double>(), h->x0.as<double>()));
  BAMG_TRY(orient_normalise(n0, h->x0.as<double>(), s));
  // the setup's one closing host read: divisor flags of every level, fits
  // refitted or rank deficient, the coarsest status, the finest sigma
  BAMG_TRY(setup_flags(h, s, rkd.as<int>(), coarse_err.p ? coarse_err.as<int>() : nullptr,
                       sig64.as<double>(), ld));
  h->sigma.resize(r);
  complexities(h);
  return BAMG_OK;
}

template bamg_status run_setup<double>(bamg_hierarchy*, cudaStream_t);
template bamg_status run_setup<float>(bamg_hierarchy*, cudaStream_t);

// --------------------------------------------------------------- level 0
bamg_status setup_finest(bamg_hierarchy* h, const bamg_csr* A, cudaStream_t s) {
  int n = (int)A->n;
  int nnz = (int)A->nnz;
  DevMem arp, aci, ava;
  const int32_t *rp = A->row_ptr, *ci = A->col_idx;
  const double* va = A->val;
  if (!A->on_device) {
    BAMG_TRY(arp.alloc(sizeof(int32_t) * (n + 1), s));
    BAMG_TRY(aci.alloc(sizeof(int32_t) * (nnz > 0 ? nnz : 1), s));
    BAMG_TRY(ava.alloc(sizeof(double) * (nnz > 0 ? nnz : 1), s));
    BAMG_CUDA(cudaMemcpyAsync(arp.p, rp, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s));
    BAMG_CUDA(cudaMemcpyAsync(aci.p, ci, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s));
    BAMG_CUDA(cudaMemcpyAsync(ava.p, va, sizeof(double) * nnz, cudaMemcpyHostToDevice, s));
    rp = arp.as<int32_t>(); ci = aci.as<int32_t>(); va = ava.as<double>();
  }
  BAMG_TRY(check_rowptr(n, rp, nnz, s));
  int64_t bad = 0;
  BAMG_TRY(check_stochastic(n, rp, ci, va, h->p.stochastic_tol, &bad, s));
  if (bad) {
    set_error("A is not column stochastic: %lld offending entries or columns", (long long)bad);
    return BAMG_ERR_NOT_STOCHASTIC;
  }
  h->lv.emplace_back();
  Level& L = h->lv[0];
  DevMem cnt;
  BAMG_TRY(cnt.alloc(sizeof(int32_t) * (n + 1), s));
  BAMG_TRY(build_B_count(n, rp, ci, cnt.as<int32_t>(), s));
  DevMem brp;
  BAMG_TRY(brp.alloc(sizeof(int32_t) * (n + 1), s));
  int64_t nnzB = 0;
  BAMG_TRY(scan_counts(cnt.as<int32_t>(), brp.as<int32_t>(), n, s, &nnzB));
  L.B.rows = L.B.cols = n;
  L.B.nnz = (int)nnzB;
  L.B.rp = std::move(brp);
  BAMG_TRY(L.B.ci.alloc(sizeof(int32_t) * nnzB, s));
  BAMG_TRY(L.B.va.alloc(sizeof(double) * nnzB, s));
  BAMG_TRY(build_B_fill(n, rp, ci, va, L.B.r(), L.B.ci.as<int32_t>(), L.B.va.as<double>(), s));
  L.nx = A->nx;
  L.ny = A->ny;
  BAMG_TRY(finish_level(h, L, 0, s));
  BAMG_CUDA(cudaStreamSynchronize(s));  // A's copies are released on return
  return BAMG_OK;
}

}  // namespace bamg
