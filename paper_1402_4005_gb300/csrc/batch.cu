// Many chains in one solve: block-diagonal batching of independent hierarchies.
//
// Every chain gets its own bootstrap setup (Algorithm 1); the setups run
// concurrently, one host thread and one stream each.  The hierarchies are
// then concatenated level by level into block-diagonal operators.  Chains are
// ordered by depth (deepest first), so at every level the chains that
// continue below form a prefix of the rows: one launch smooths, restricts and
// interpolates all of them, and one batched dense GEMV applies the coarsest
// pseudo-inverses (Section 3) of the chains that end at that level.  The
// batched V-cycle is captured once as a CUDA graph.  Flexible GMRES (Section
// 6) runs for all chains in lock step on the concatenated vectors, with
// per-chain (segmented) dot products, Hessenberg matrices, Givens rotations
// and convergence tests; a converged chain is frozen.  Lanes per row of
// every batched operator are chosen by timing the candidates once (autotune).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "hierarchy.cuh"

namespace bamg {

struct BLevel {
  int n = 0, n_cont = 0, nc_next = 0;
  Csr B, P, Q;
  DevMem dinv, dinv32;
  int gB = 4, gP = 4, gQ = 4;
  int ncoarse_rows = 0;
  DevMem c_pinv_off, c_base, c_len;   // per coarsest row: pinv row offset, chain row base, chain size
  DevMem pinv64, pinv32;
  DevMem vb, vz, vt, vr;
};

}  // namespace bamg

struct bamg_batch {
  bamg_params p;
  int mixed = 0, nch = 0, device = 0;
  std::vector<bamg_hierarchy*> h;           // input order
  std::vector<int> order;                   // batch position -> input index
  std::vector<std::vector<int64_t>> off;    // off[l][pos]: row offset of the chain at level l
  std::vector<bamg::BLevel> lv;
  std::vector<int64_t> in_off;              // input-order offsets of x
  bamg::DevMem seg0, rowchain0, io_in, io_out;
  cudaStream_t cap = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  uint64_t gk = 0;
  double setup_ms = 0.0;
  std::vector<cudaStream_t> wstreams;       // per-thread setup streams (the chains free memory on them)
};

namespace bamg {

// ------------------------------------------------------------ assembly
__global__ void shift_kernel(int cnt, const int32_t* __restrict__ src, int32_t add, int32_t* __restrict__ dst) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) dst[i] = src[i] + add;
}

static bamg_status concat_csr(const std::vector<const Csr*>& parts, const std::vector<int64_t>& row_off,
                              const std::vector<int64_t>& col_off, int rows, int cols, Csr& out, bool mixed,
                              cudaStream_t s) {
  int64_t nnz = 0;
  for (auto* c : parts) nnz += c->nnz;
  if (nnz > INT32_MAX) {
    set_error("batched operator has %lld nonzeros, above the int32 index range", (long long)nnz);
    return BAMG_ERR_UNSUPPORTED;
  }
  BAMG_TRY(out.alloc(rows, cols, (int)nnz, s));
  int64_t q = 0;
  for (size_t k = 0; k < parts.size(); ++k) {
    const Csr& c = *parts[k];
    int32_t* rp = out.rp.as<int32_t>() + row_off[k];
    BAMG_TRY(launch(shift_kernel, dim3(cdiv(c.rows + 1, 256)), dim3(256), 0, s, c.rows + 1, c.r(), (int32_t)q, rp));
    BAMG_TRY(launch(shift_kernel, dim3(cdiv(c.nnz, 256)), dim3(256), 0, s, c.nnz, c.c(), (int32_t)col_off[k],
                    out.ci.as<int32_t>() + q));
    BAMG_CUDA(cudaMemcpyAsync(out.va.as<double>() + q, c.v(), sizeof(double) * c.nnz, cudaMemcpyDeviceToDevice, s));
    q += c.nnz;
  }
  if (parts.empty()) BAMG_CUDA(cudaMemsetAsync(out.rp.p, 0, sizeof(int32_t) * (rows + 1), s));
  if (mixed) BAMG_TRY(out.make32(s));
  return BAMG_OK;
}

// Autotune: lanes per row of the vector kernels, by timing each candidate.
template <typename T>
static int autotune_lanes(const Csr& A, int rows, const T* vals, cudaStream_t s) {
  if (rows <= 0 || A.nnz == 0) return 4;
  DevMem x, y;
  if (x.alloc(sizeof(T) * (A.cols > 0 ? A.cols : 1), s) != BAMG_OK) return 4;
  if (y.alloc(sizeof(T) * rows, s) != BAMG_OK) return 4;
  cudaMemsetAsync(x.p, 0, sizeof(T) * (A.cols > 0 ? A.cols : 1), s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best = 4;
  float tbest = 1e30f;
  for (int G : {2, 4, 8, 16, 32}) {
    csr_vec<T>(VEC_SPMV, rows, G, A.r(), A.c(), vals, (const T*)nullptr, T(1), x.as<T>(), nullptr, y.as<T>(), s);
    cudaEventRecord(e0, s);
    for (int k = 0; k < 5; ++k)
      csr_vec<T>(VEC_SPMV, rows, G, A.r(), A.c(), vals, (const T*)nullptr, T(1), x.as<T>(), nullptr, y.as<T>(), s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < tbest) { tbest = ms; best = G; }
  }
  g_launches.fetch_sub(30);  // tuning launches are not part of any solve
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

static bamg_status build_levels(bamg_batch* bt, cudaStream_t s) {
  const int nch = bt->nch;
  std::vector<int> depth(nch);
  for (int pos = 0; pos < nch; ++pos) depth[pos] = (int)bt->h[bt->order[pos]]->lv.size();
  int L = depth.empty() ? 0 : depth[0];
  bt->off.assign(L + 1, std::vector<int64_t>(nch + 1, 0));
  for (int l = 0; l < L; ++l) {
    int64_t o = 0;
    for (int pos = 0; pos < nch; ++pos) {
      bt->off[l][pos] = o;
      if (depth[pos] > l) o += bt->h[bt->order[pos]]->lv[l].n;
    }
    bt->off[l][nch] = o;
  }
  bt->lv.clear();
  bt->lv.reserve(L);
  for (int l = 0; l < L; ++l) {
    bt->lv.emplace_back();
    BLevel& B = bt->lv[l];
    int present = 0, cont = 0;
    for (int pos = 0; pos < nch; ++pos) {
      if (depth[pos] > l) ++present;
      if (depth[pos] > l + 1) ++cont;
    }
    B.n = (int)bt->off[l][present];
    B.n_cont = (int)bt->off[l][cont];
    B.nc_next = l + 1 < L ? (int)bt->off[l + 1][cont] : 0;
    std::vector<const Csr*> bp, pp, qp;
    std::vector<int64_t> ro, co, pro, pco, qro, qco;
    for (int pos = 0; pos < present; ++pos) {
      const Level& lv = bt->h[bt->order[pos]]->lv[l];
      bp.push_back(&lv.B);
      ro.push_back(bt->off[l][pos]);
      co.push_back(bt->off[l][pos]);
      if (pos < cont) {
        pp.push_back(&lv.P);
        pro.push_back(bt->off[l][pos]);
        pco.push_back(bt->off[l + 1][pos]);
        qp.push_back(&lv.Q);
        qro.push_back(bt->off[l + 1][pos]);
        qco.push_back(bt->off[l][pos]);
      }
    }
    if (std::getenv("BAMG_TRACE"))
      fprintf(stderr, "[bamg] batch level %d: present %d cont %d n %d n_cont %d nc_next %d\n", l, present, cont, B.n,
              B.n_cont, B.nc_next);
    BAMG_TRY(concat_csr(bp, ro, co, B.n, B.n, B.B, bt->mixed, s));
    BAMG_TRY(B.dinv.alloc(sizeof(double) * (B.n > 0 ? B.n : 1), s));
    for (int pos = 0; pos < present; ++pos) {
      const Level& lv = bt->h[bt->order[pos]]->lv[l];
      BAMG_CUDA(cudaMemcpyAsync(B.dinv.as<double>() + bt->off[l][pos], lv.dinv.p, sizeof(double) * lv.n,
                                cudaMemcpyDeviceToDevice, s));
    }
    if (bt->mixed) {
      BAMG_TRY(B.dinv32.alloc(sizeof(float) * (B.n > 0 ? B.n : 1), s));
      BAMG_TRY(convert<double, float>((size_t)B.n, B.dinv.as<double>(), B.dinv32.as<float>(), s));
    }
    if (cont > 0) {
      BAMG_TRY(concat_csr(pp, pro, pco, B.n_cont, B.nc_next, B.P, bt->mixed, s));
      BAMG_TRY(concat_csr(qp, qro, qco, B.nc_next, B.n_cont, B.Q, bt->mixed, s));
    }
    // chains whose coarsest level is l
    std::vector<long long> poff, base, len;
    int64_t pinv_total = 0;
    for (int pos = cont; pos < present; ++pos) {
      const bamg_hierarchy* hc = bt->h[bt->order[pos]];
      int nL = hc->nL;
      for (int i = 0; i < nL; ++i) {
        poff.push_back(pinv_total + (int64_t)i * nL);
        base.push_back(bt->off[l][pos]);
        len.push_back(nL);
      }
      pinv_total += (int64_t)nL * nL;
    }
    B.ncoarse_rows = (int)poff.size();
    if (B.ncoarse_rows > 0) {
      BAMG_TRY(B.c_pinv_off.alloc(sizeof(long long) * poff.size(), s));
      BAMG_TRY(B.c_base.alloc(sizeof(long long) * base.size(), s));
      BAMG_TRY(B.c_len.alloc(sizeof(long long) * len.size(), s));
      BAMG_CUDA(cudaMemcpyAsync(B.c_pinv_off.p, poff.data(), sizeof(long long) * poff.size(), cudaMemcpyHostToDevice, s));
      BAMG_CUDA(cudaMemcpyAsync(B.c_base.p, base.data(), sizeof(long long) * base.size(), cudaMemcpyHostToDevice, s));
      BAMG_CUDA(cudaMemcpyAsync(B.c_len.p, len.data(), sizeof(long long) * len.size(), cudaMemcpyHostToDevice, s));
      BAMG_TRY(B.pinv64.alloc(sizeof(double) * pinv_total, s));
      int64_t q = 0;
      for (int pos = cont; pos < present; ++pos) {
        const bamg_hierarchy* hc = bt->h[bt->order[pos]];
        size_t cnt = (size_t)hc->nL * hc->nL;
        BAMG_CUDA(cudaMemcpyAsync(B.pinv64.as<double>() + q, hc->Bpinv.p, sizeof(double) * cnt,
                                  cudaMemcpyDeviceToDevice, s));
        q += cnt;
      }
      if (bt->mixed) {
        BAMG_TRY(B.pinv32.alloc(sizeof(float) * pinv_total, s));
        BAMG_TRY(convert<double, float>((size_t)pinv_total, B.pinv64.as<double>(), B.pinv32.as<float>(), s));
      }
      BAMG_CUDA(cudaStreamSynchronize(s));   // host vectors above leave scope
    }
    size_t es = bt->mixed ? sizeof(float) : sizeof(double);
    size_t nb = (size_t)(B.n > 0 ? B.n : 1);
    BAMG_TRY(B.vb.alloc(es * nb, s));
    BAMG_TRY(B.vz.alloc(es * nb, s));
    BAMG_TRY(B.vt.alloc(es * nb, s));
    BAMG_TRY(B.vr.alloc(es * nb, s));
  }
  // autotune the lanes per row of every batched operator
  for (auto& B : bt->lv) {
    if (bt->mixed) {
      if (B.n_cont > 0) B.gB = autotune_lanes<float>(B.B, B.n_cont, B.B.vals<float>(), s);
      if (!B.P.empty()) B.gP = autotune_lanes<float>(B.P, B.n_cont, B.P.vals<float>(), s);
      if (!B.Q.empty()) B.gQ = autotune_lanes<float>(B.Q, B.nc_next, B.Q.vals<float>(), s);
    } else {
      if (B.n_cont > 0) B.gB = autotune_lanes<double>(B.B, B.n_cont, B.B.vals<double>(), s);
      if (!B.P.empty()) B.gP = autotune_lanes<double>(B.P, B.n_cont, B.P.vals<double>(), s);
      if (!B.Q.empty()) B.gQ = autotune_lanes<double>(B.Q, B.nc_next, B.Q.vals<double>(), s);
    }
  }
  // level-0 segments (batch order) and row -> chain map
  const int n0 = bt->lv.empty() ? 0 : bt->lv[0].n;
  std::vector<int> seg(nch + 1), rc(n0);
  for (int pos = 0; pos <= nch; ++pos) seg[pos] = (int)bt->off[0][pos];
  for (int pos = 0; pos < nch; ++pos)
    for (int i = seg[pos]; i < seg[pos + 1]; ++i) rc[i] = pos;
  BAMG_TRY(bt->seg0.alloc(sizeof(int) * (nch + 1), s));
  BAMG_TRY(bt->rowchain0.alloc(sizeof(int) * (n0 > 0 ? n0 : 1), s));
  BAMG_CUDA(cudaMemcpyAsync(bt->seg0.p, seg.data(), sizeof(int) * (nch + 1), cudaMemcpyHostToDevice, s));
  BAMG_CUDA(cudaMemcpyAsync(bt->rowchain0.p, rc.data(), sizeof(int) * n0, cudaMemcpyHostToDevice, s));
  BAMG_TRY(bt->io_in.alloc(sizeof(double) * (n0 > 0 ? n0 : 1), s));
  BAMG_TRY(bt->io_out.alloc(sizeof(double) * (n0 > 0 ? n0 : 1), s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  return BAMG_OK;
}

// ------------------------------------------------------------ batched V-cycle
template <typename T>
__global__ void coarse_gemv_kernel(int rows, int row0, const long long* __restrict__ poff,
                                   const long long* __restrict__ base, const long long* __restrict__ len,
                                   const T* __restrict__ pinv, const T* __restrict__ b, T* __restrict__ z) {
  pdl_wait();
  pdl_trigger();
  int lane = threadIdx.x & 31;
  int g = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (g >= rows) return;
  const T* a = pinv + poff[g];
  const T* x = b + base[g];
  int m = (int)len[g];
  T acc = T(0);
  for (int j = lane; j < m; j += 32) acc = fma(a[j], x[j], acc);
  acc = warp_sum(acc);
  if (lane == 0) z[row0 + g] = acc;
}

template <typename T> static const T* bl_dinv(const BLevel& B);
template <> const double* bl_dinv<double>(const BLevel& B) { return B.dinv.as<double>(); }
template <> const float* bl_dinv<float>(const BLevel& B) { return B.dinv32.as<float>(); }
template <typename T> static const T* bl_pinv(const BLevel& B);
template <> const double* bl_pinv<double>(const BLevel& B) { return B.pinv64.as<double>(); }
template <> const float* bl_pinv<float>(const BLevel& B) { return B.pinv32.as<float>(); }

template <typename T>
static bamg_status bvcycle_level(bamg_batch* bt, int l, cudaStream_t s) {
  BLevel& B = bt->lv[l];
  const bamg_params& p = bt->p;
  T* b = B.vb.as<T>();
  T* z = B.vz.as<T>();
  const T om = T(p.omega);
  if (B.n_cont > 0) {
    const T* dv = bl_dinv<T>(B);
    const T* bv = B.B.vals<T>();
    T* cur = z;
    T* alt = B.vt.as<T>();
    if (p.nu_pre == 0) {
      BAMG_CUDA(cudaMemsetAsync(cur, 0, sizeof(T) * B.n_cont, s));
    } else {
      BAMG_TRY(csr_vec<T>(VEC_JACOBI_ZERO, B.n_cont, B.gB, B.B.r(), B.B.c(), bv, dv, om, nullptr, b, cur, s));
      for (int it = 1; it < p.nu_pre; ++it) {
        BAMG_TRY(csr_vec<T>(VEC_JACOBI, B.n_cont, B.gB, B.B.r(), B.B.c(), bv, dv, om, cur, b, alt, s));
        std::swap(cur, alt);
      }
    }
    BAMG_TRY(csr_vec<T>(VEC_RESID, B.n_cont, B.gB, B.B.r(), B.B.c(), bv, dv, om, cur, b, B.vr.as<T>(), s));
    BLevel& C = bt->lv[l + 1];
    BAMG_TRY(csr_vec<T>(VEC_SPMV, B.nc_next, B.gQ, B.Q.r(), B.Q.c(), B.Q.vals<T>(), dv, om, B.vr.as<T>(),
                        nullptr, C.vb.as<T>(), s));
    BAMG_TRY(bvcycle_level<T>(bt, l + 1, s));
    BAMG_TRY(csr_vec<T>(VEC_SPMV_ADD, B.n_cont, B.gP, B.P.r(), B.P.c(), B.P.vals<T>(), dv, om, C.vz.as<T>(),
                        nullptr, cur, s));
    for (int it = 0; it < p.nu_post; ++it) {
      BAMG_TRY(csr_vec<T>(VEC_JACOBI, B.n_cont, B.gB, B.B.r(), B.B.c(), bv, dv, om, cur, b, alt, s));
      std::swap(cur, alt);
    }
    if (cur != z) BAMG_CUDA(cudaMemcpyAsync(z, cur, sizeof(T) * B.n_cont, cudaMemcpyDeviceToDevice, s));
  }
  if (B.ncoarse_rows > 0)
    BAMG_TRY(launch(coarse_gemv_kernel<T>, dim3(cdiv((long long)B.ncoarse_rows * 32, 256)), dim3(256), 0, s,
                    B.ncoarse_rows, B.n_cont, (const long long*)B.c_pinv_off.as<long long>(),
                    (const long long*)B.c_base.as<long long>(), (const long long*)B.c_len.as<long long>(),
                    bl_pinv<T>(B), (const T*)b, z));
  return BAMG_OK;
}

__global__ void copy_dd_kernel(size_t n, const double* __restrict__ a, double* __restrict__ b) {
  pdl_wait();
  pdl_trigger();
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = a[t];
}

template <typename T>
static bamg_status bvcycle_body(bamg_batch* bt, cudaStream_t s) {
  BLevel& L0 = bt->lv[0];
  size_t n = L0.n;
  if (sizeof(T) == 4) {
    BAMG_TRY(convert<double, float>(n, bt->io_in.as<double>(), (float*)L0.vb.p, s));
  } else {
    BAMG_TRY(launch(copy_dd_kernel, dim3(cdiv((long long)n, 256)), dim3(256), 0, s, n,
                    (const double*)bt->io_in.as<double>(), (double*)L0.vb.p));
  }
  BAMG_TRY(bvcycle_level<T>(bt, 0, s));
  if (sizeof(T) == 4) {
    BAMG_TRY(convert<float, double>(n, (const float*)L0.vz.p, bt->io_out.as<double>(), s));
  } else {
    BAMG_TRY(launch(copy_dd_kernel, dim3(cdiv((long long)n, 256)), dim3(256), 0, s, n, (const double*)L0.vz.p,
                    bt->io_out.as<double>()));
  }
  return BAMG_OK;
}

static bamg_status bvcycle_prepare(bamg_batch* bt) {
  if (!bt->cap) BAMG_CUDA(cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking));
  uint64_t before = t_launches;
  BAMG_CUDA(cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeThreadLocal));
  bamg_status st;
  {
    PdlScope pdl;   // kernel-to-kernel edges programmatic (every kernel waits first)
    st = bt->mixed ? bvcycle_body<float>(bt, bt->cap) : bvcycle_body<double>(bt, bt->cap);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(bt->cap, &g);
  if (st != BAMG_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  BAMG_CUDA(e);
  bt->g = g;
  BAMG_CUDA(cudaGraphInstantiate(&bt->ge, g, 0));
  bt->gk = t_launches - before;
  g_launches.fetch_sub(bt->gk);
  return BAMG_OK;
}

static bamg_status bvcycle_run(bamg_batch* bt, cudaStream_t s) {
  BAMG_CUDA(cudaGraphLaunch(bt->ge, s));
  g_launches.fetch_add(bt->gk);
  return BAMG_OK;
}

// ------------------------------------------------------------ batched FGMRES
// out[c * H + k] = sum over the rows of chain c of V_k . w
__global__ void seg_multidot_kernel(const int* __restrict__ seg, int H, const double* __restrict__ V, size_t ldv,
                                    const double* __restrict__ w, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  int c = blockIdx.x, k = blockIdx.y;
  const double* v = V + (size_t)k * ldv;
  double s = 0.0;
  for (int i = seg[c] + threadIdx.x; i < seg[c + 1]; i += blockDim.x) s += v[i] * w[i];
  s = warp_sum(s);
  __shared__ double sh[8];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
    out[(size_t)c * H + k] = t;
  }
}

// per chain: sums of x, |x| and x^2 -> out[3c .. 3c+2]
__global__ void seg_sums_kernel(const int* __restrict__ seg, const double* __restrict__ x, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  int c = blockIdx.x;
  double s = 0, a = 0, q = 0;
  for (int i = seg[c] + threadIdx.x; i < seg[c + 1]; i += blockDim.x) {
    double v = x[i];
    s += v; a += fabs(v); q += v * v;
  }
  s = warp_sum(s); a = warp_sum(a); q = warp_sum(q);
  __shared__ double sh[3][8];
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { sh[0][w] = s; sh[1][w] = a; sh[2][w] = q; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ts = 0, ta = 0, tq = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { ts += sh[0][k]; ta += sh[1][k]; tq += sh[2][k]; }
    out[3 * c] = ts; out[3 * c + 1] = ta; out[3 * c + 2] = tq;
  }
}

// w[i] -= sum_k h[c(i) * H + k] V_k[i]
__global__ void seg_orth_kernel(int n, const int* __restrict__ rc, int K, int H, const double* __restrict__ V,
                                size_t ldv, const double* __restrict__ h, double* __restrict__ w) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* hc = h + (size_t)rc[i] * H;
  double acc = w[i];
  for (int k = 0; k < K; ++k) acc -= hc[k] * V[(size_t)k * ldv + i];
  w[i] = acc;
}

// b[i] = active(c) ? a[i] / f[3c+2]^(1/2) : 0   (normalise per chain)
__global__ void seg_normalise_kernel(int n, const int* __restrict__ rc, const double* __restrict__ a,
                                     const double* __restrict__ sums, const int* __restrict__ active,
                                     double* __restrict__ b) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = rc[i];
  double q = sums[3 * c + 2];
  b[i] = (active[c] && q > 0.0) ? a[i] / sqrt(q) : 0.0;
}

// y[i] = x[i] + active(c) * sum_k c_k Z_k[i]
__global__ void seg_combine_kernel(int n, const int* __restrict__ rc, int K, int H, const double* __restrict__ Z,
                                   size_t ldz, const double* __restrict__ coef, const int* __restrict__ active,
                                   const double* __restrict__ x, double* __restrict__ y) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = rc[i];
  double acc = x[i];
  if (active[c]) {
    const double* cc = coef + (size_t)c * H;
    for (int k = 0; k < K; ++k) acc += cc[k] * Z[(size_t)k * ldz + i];
  }
  y[i] = acc;
}

// one thread per chain: Arnoldi column j, Givens rotations, triangular solve
__global__ void seg_givens_kernel(int nch, int j, int m, const double* __restrict__ h1, const double* __restrict__ h2,
                                  const double* __restrict__ wsums, const int* __restrict__ active,
                                  double* __restrict__ R, double* __restrict__ cs, double* __restrict__ sn,
                                  double* __restrict__ g, double* __restrict__ y, double* __restrict__ st) {
  pdl_wait();
  pdl_trigger();
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nch) return;
  if (!active[c]) { st[2 * c] = 0.0; st[2 * c + 1] = 0.0; return; }
  const int H = m + 1;
  double col[65];
  for (int k = 0; k <= j; ++k) col[k] = h1[(size_t)c * H + k] + h2[(size_t)c * H + k];
  double hn = sqrt(wsums[3 * c + 2]);
  col[j + 1] = hn;
  double* csc = cs + (size_t)c * m;
  double* snc = sn + (size_t)c * m;
  double* gc = g + (size_t)c * H;
  double* Rc = R + (size_t)c * H * m;
  double* yc = y + (size_t)c * H;
  for (int k = 0; k < j; ++k) {
    double t = csc[k] * col[k] + snc[k] * col[k + 1];
    col[k + 1] = -snc[k] * col[k] + csc[k] * col[k + 1];
    col[k] = t;
  }
  double a = col[j], b = col[j + 1];
  double d = hypot(a, b);
  double cc = d > 0.0 ? a / d : 1.0, ss = d > 0.0 ? b / d : 0.0;
  csc[j] = cc; snc[j] = ss;
  col[j] = d;
  gc[j + 1] = -ss * gc[j];
  gc[j] = cc * gc[j];
  for (int k = 0; k <= j; ++k) Rc[(size_t)k * m + j] = col[k];
  for (int k = j; k >= 0; --k) {
    double acc = gc[k];
    for (int q = k + 1; q <= j; ++q) acc -= Rc[(size_t)k * m + q] * yc[q];
    double rkk = Rc[(size_t)k * m + k];
    yc[k] = rkk != 0.0 ? acc / rkk : 0.0;
  }
  st[2 * c] = fabs(gc[j + 1]);
  st[2 * c + 1] = hn;
}

__global__ void seg_init_g_kernel(int nch, int m, const double* __restrict__ sums, double* __restrict__ g) {
  pdl_wait();
  pdl_trigger();
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nch) return;
  for (int k = 0; k <= m; ++k) g[(size_t)c * (m + 1) + k] = k == 0 ? sqrt(sums[3 * c + 2]) : 0.0;
}

// x <- x * sign(sum) / ||x||_1 per chain
__global__ void seg_orient_kernel(int n, const int* __restrict__ rc, const double* __restrict__ sums,
                                  double* __restrict__ x) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = rc[i];
  double f = (sums[3 * c] < 0.0 ? -1.0 : 1.0) / sums[3 * c + 1];
  x[i] *= f;
}

__global__ void negate_kernel(int n, double* __restrict__ x) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = -x[i];
}

static bamg_status batched_fgmres(bamg_batch* bt, double* x, const bamg_solve_params* sp, bamg_solve_info* infos,
                                  cudaStream_t s) {
  PdlScope pdl;   // consecutive kernels overlap their launches (each waits for its predecessor first)
  const int nch = bt->nch, m = sp->restart, H = m + 1;
  BLevel& L0 = bt->lv[0];
  const int n = L0.n;
  const int* seg = bt->seg0.as<int>();
  const int* rc = bt->rowchain0.as<int>();
  const int gB = L0.gB;
  DevMem V, Z, w, w2, xj, h1, h2, R, cs, sn, g, y, st, sums, act;
  BAMG_TRY(V.alloc(sizeof(double) * (size_t)H * n, s));
  BAMG_TRY(Z.alloc(sizeof(double) * (size_t)m * n, s));
  BAMG_TRY(w.alloc(sizeof(double) * n, s));
  BAMG_TRY(w2.alloc(sizeof(double) * n, s));
  BAMG_TRY(xj.alloc(sizeof(double) * n, s));
  BAMG_TRY(h1.alloc(sizeof(double) * (size_t)nch * H, s));
  BAMG_TRY(h2.alloc(sizeof(double) * (size_t)nch * H, s));
  BAMG_TRY(R.alloc(sizeof(double) * (size_t)nch * H * m, s));
  BAMG_TRY(cs.alloc(sizeof(double) * (size_t)nch * m, s));
  BAMG_TRY(sn.alloc(sizeof(double) * (size_t)nch * m, s));
  BAMG_TRY(g.alloc(sizeof(double) * (size_t)nch * H, s));
  BAMG_TRY(y.alloc(sizeof(double) * (size_t)nch * H, s));
  BAMG_TRY(st.alloc(sizeof(double) * 2 * nch, s));
  BAMG_TRY(sums.alloc(sizeof(double) * 3 * nch * 4, s));
  BAMG_TRY(act.alloc(sizeof(int) * nch, s));
  BAMG_CUDA(cudaMemsetAsync(y.p, 0, sizeof(double) * (size_t)nch * H, s));
  const unsigned gv = cdiv(n, 256);
  double* sumA = sums.as<double>();
  double* sumB = sums.as<double>() + 3 * nch;
  double* sumC = sums.as<double>() + 6 * nch;   // true residual: ||B x|| per chain
  double* sumD = sums.as<double>() + 9 * nch;   // true residual: ||x|| per chain
  std::vector<int> active(nch, 1), its(nch, 0), it7(nch, -1);
  std::vector<double> rel(nch, 0.0), xn1(nch, 1.0), xn2(nch, 1.0), hs(3 * nch), hs2(3 * nch), hst(2 * nch);
  // x = x^(0) of every chain (batch order)
  for (int pos = 0; pos < nch; ++pos) {
    const bamg_hierarchy* hc = bt->h[bt->order[pos]];
    BAMG_CUDA(cudaMemcpyAsync(x + bt->off[0][pos], hc->x0.p, sizeof(double) * hc->lv[0].n, cudaMemcpyDeviceToDevice, s));
  }
  auto true_res = [&](const double* xv) -> bamg_status {
    BAMG_TRY(csr_vec<double>(VEC_SPMV, n, gB, L0.B.r(), L0.B.c(), L0.B.v(), L0.dinv.as<double>(), 1.0, xv,
                             nullptr, w2.as<double>(), s));
    BAMG_TRY(launch(seg_sums_kernel, dim3(nch), dim3(256), 0, s, seg, (const double*)w2.as<double>(), sumC));
    BAMG_TRY(launch(seg_sums_kernel, dim3(nch), dim3(256), 0, s, seg, xv, sumD));
    BAMG_CUDA(cudaMemcpyAsync(hs.data(), sumC, sizeof(double) * 3 * nch, cudaMemcpyDeviceToHost, s));
    BAMG_CUDA(cudaMemcpyAsync(hs2.data(), sumD, sizeof(double) * 3 * nch, cudaMemcpyDeviceToHost, s));
    BAMG_CUDA(cudaStreamSynchronize(s));
    return BAMG_OK;
  };
  BAMG_TRY(true_res(x));
  for (int c = 0; c < nch; ++c) {
    xn1[c] = hs2[3 * c + 1];
    xn2[c] = std::sqrt(hs2[3 * c + 2]);
    rel[c] = hs[3 * c + 1] / hs2[3 * c + 1];
    if (rel[c] <= sp->tol) active[c] = 0;
  }
  // a mixed-precision chain whose true residual falls by less than half over
  // two restart cycles in a row has stalled (FP32 V-cycle accuracy): it
  // leaves the lock-step iteration and continues with FP64 V-cycles
  std::vector<double> prev_rel(rel);
  std::vector<int> slow(nch, 0);
  int total = 0;
  auto any_active = [&]() { for (int c = 0; c < nch; ++c) if (active[c]) return true; return false; };
  while (any_active() && total < sp->max_iter) {
    BAMG_CUDA(cudaMemcpyAsync(act.p, active.data(), sizeof(int) * nch, cudaMemcpyHostToDevice, s));
    // r = -B x per chain, v_0 = r / ||r||, g = ||r|| e_1
    BAMG_TRY(csr_vec<double>(VEC_SPMV, n, gB, L0.B.r(), L0.B.c(), L0.B.v(), L0.dinv.as<double>(), 1.0, x,
                             nullptr, w.as<double>(), s));
    BAMG_TRY(launch(negate_kernel, dim3(gv), dim3(256), 0, s, n, w.as<double>()));
    BAMG_TRY(launch(seg_sums_kernel, dim3(nch), dim3(256), 0, s, seg, (const double*)w.as<double>(), sumA));
    BAMG_TRY(launch(seg_normalise_kernel, dim3(gv), dim3(256), 0, s, n, rc, (const double*)w.as<double>(),
                    (const double*)sumA, (const int*)act.as<int>(), V.as<double>()));
    BAMG_TRY(launch(seg_init_g_kernel, dim3(cdiv(nch, 128)), dim3(128), 0, s, nch, m, (const double*)sumA,
                    g.as<double>()));
    bool cycle_done = false;
    for (int j = 0; j < m && !cycle_done; ++j) {
      double* vj = V.as<double>() + (size_t)j * n;
      double* zj = Z.as<double>() + (size_t)j * n;
      BAMG_CUDA(cudaMemcpyAsync(bt->io_in.p, vj, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      BAMG_TRY(bvcycle_run(bt, s));
      BAMG_CUDA(cudaMemcpyAsync(zj, bt->io_out.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      BAMG_TRY(csr_vec<double>(VEC_SPMV, n, gB, L0.B.r(), L0.B.c(), L0.B.v(), L0.dinv.as<double>(), 1.0, zj,
                               nullptr, w.as<double>(), s));
      const int K = j + 1;
      BAMG_TRY(launch(seg_multidot_kernel, dim3(nch, K), dim3(256), 0, s, seg, H, (const double*)V.as<double>(),
                      (size_t)n, (const double*)w.as<double>(), h1.as<double>()));
      BAMG_TRY(launch(seg_orth_kernel, dim3(gv), dim3(256), 0, s, n, rc, K, H, (const double*)V.as<double>(),
                      (size_t)n, (const double*)h1.as<double>(), w.as<double>()));
      BAMG_TRY(launch(seg_multidot_kernel, dim3(nch, K), dim3(256), 0, s, seg, H, (const double*)V.as<double>(),
                      (size_t)n, (const double*)w.as<double>(), h2.as<double>()));
      BAMG_TRY(launch(seg_orth_kernel, dim3(gv), dim3(256), 0, s, n, rc, K, H, (const double*)V.as<double>(),
                      (size_t)n, (const double*)h2.as<double>(), w.as<double>()));
      BAMG_TRY(launch(seg_sums_kernel, dim3(nch), dim3(256), 0, s, seg, (const double*)w.as<double>(), sumA));
      BAMG_TRY(launch(seg_givens_kernel, dim3(cdiv(nch, 64)), dim3(64), 0, s, nch, j, m,
                      (const double*)h1.as<double>(), (const double*)h2.as<double>(), (const double*)sumA,
                      (const int*)act.as<int>(), R.as<double>(), cs.as<double>(), sn.as<double>(), g.as<double>(),
                      y.as<double>(), st.as<double>()));
      BAMG_CUDA(cudaMemcpyAsync(hst.data(), st.p, sizeof(double) * 2 * nch, cudaMemcpyDeviceToHost, s));
      BAMG_CUDA(cudaStreamSynchronize(s));
      ++total;
      bool need_check = (j == m - 1) || total >= sp->max_iter;
      for (int c = 0; c < nch; ++c) {
        if (!active[c]) continue;
        ++its[c];
        if (it7[c] < 0 && hst[2 * c] <= 1e-7 * xn2[c]) it7[c] = its[c];
        if (hst[2 * c] <= 2.0 * sp->tol * xn1[c] || !(hst[2 * c + 1] > 0.0)) need_check = true;
      }
      if (need_check) {
        BAMG_TRY(launch(seg_combine_kernel, dim3(gv), dim3(256), 0, s, n, rc, K, H, (const double*)Z.as<double>(),
                        (size_t)n, (const double*)y.as<double>(), (const int*)act.as<int>(), (const double*)x,
                        xj.as<double>()));
        BAMG_TRY(true_res(xj.as<double>()));
        bool last = (j == m - 1) || total >= sp->max_iter;
        bool changed = false;
        for (int c = 0; c < nch; ++c) {
          if (!active[c]) continue;
          double rc_ = hs[3 * c + 1] / hs2[3 * c + 1];
          bool brk = !(hst[2 * c + 1] > 0.0);
          if (rc_ <= sp->tol || last || brk) {
            BAMG_CUDA(cudaMemcpyAsync(x + bt->off[0][c], xj.as<double>() + bt->off[0][c],
                                      sizeof(double) * (bt->off[0][c + 1] - bt->off[0][c]),
                                      cudaMemcpyDeviceToDevice, s));
            rel[c] = rc_;
            if (rc_ <= sp->tol || brk) { active[c] = 0; changed = true; }
          }
          if (last && active[c] && bt->mixed) {
            slow[c] = rel[c] > 0.5 * prev_rel[c] ? slow[c] + 1 : 0;
            prev_rel[c] = rel[c];
            if (slow[c] >= 2) { active[c] = 0; changed = true; }
          }
        }
        if (last) cycle_done = true;
        if (changed) BAMG_CUDA(cudaMemcpyAsync(act.p, active.data(), sizeof(int) * nch, cudaMemcpyHostToDevice, s));
        if (!any_active()) break;
      }
      if (!cycle_done)
        BAMG_TRY(launch(seg_normalise_kernel, dim3(gv), dim3(256), 0, s, n, rc, (const double*)w.as<double>(),
                        (const double*)sumA, (const int*)act.as<int>(), V.as<double>() + (size_t)(j + 1) * n));
    }
  }
  // x > 0, unit 1-norm per chain
  BAMG_TRY(launch(seg_sums_kernel, dim3(nch), dim3(256), 0, s, seg, (const double*)x, sumB));
  BAMG_TRY(launch(seg_orient_kernel, dim3(gv), dim3(256), 0, s, n, rc, (const double*)sumB, x));
  BAMG_TRY(true_res(x));
  bool ok = true;
  for (int pos = 0; pos < nch; ++pos) {
    double r = hs[3 * pos + 1] / hs2[3 * pos + 1];
    if (!(r <= sp->tol)) ok = false;
    if (infos) {
      bamg_solve_info& inf = infos[bt->order[pos]];
      inf.iterations = its[pos];
      inf.iters_to_1e7 = it7[pos];
      inf.rel_res_1 = r;
      const bamg_hierarchy* hc = bt->h[bt->order[pos]];
      inf.levels = (int)hc->lv.size();
      inf.op_cplx = hc->op_cplx;
      inf.grid_cplx = hc->grid_cplx;
      inf.setup_ms = bt->setup_ms;
      inf.min_x = 0.0;
      inf.fallback_iterations = 0;
    }
  }
  if (!ok) {
    set_error("batched GMRES stopped with chains above the tolerance");
    return BAMG_ERR_NOT_CONVERGED;
  }
  return BAMG_OK;
}

}  // namespace bamg

using namespace bamg;

// ------------------------------------------------------------------- C ABI
extern "C" bamg_status bamg_setup_batched(const bamg_csr* As, int nchains, const bamg_params* p, int host_threads,
                                          void* stream, bamg_batch** out) {
  BAMG_CHECK_ARG(As && p && out && nchains >= 1);
  *out = nullptr;
  if (p->smoother != BAMG_SMOOTH_JACOBI) {
    set_error("batches take the weighted Jacobi smoother only");
    return BAMG_ERR_UNSUPPORTED;
  }
  bamg_batch* bt = new (std::nothrow) bamg_batch();
  if (!bt) return BAMG_ERR_OOM;
  bt->p = *p;
  bt->mixed = p->precision == BAMG_PREC_MIXED;
  bt->nch = nchains;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  auto t0 = std::chrono::steady_clock::now();
  if (cudaGetDevice(&bt->device) != cudaSuccess) { delete bt; return BAMG_ERR_CUDA; }
  bt->h.assign(nchains, nullptr);
  std::vector<bamg_status> st(nchains, BAMG_OK);
  std::vector<std::string> err(nchains);
  int T = host_threads > 0 ? host_threads : 4;   // more threads contend for the launch path
  if (T > nchains) T = nchains;
  bt->wstreams.assign(T, nullptr);
  for (int t = 0; t < T; ++t)
    if (cudaStreamCreateWithFlags(&bt->wstreams[t], cudaStreamNonBlocking) != cudaSuccess) {
      bt->wstreams[t] = nullptr;
      set_error("stream creation failed");
      bamg_destroy_batched(bt);
      return BAMG_ERR_CUDA;
    }
  std::vector<std::thread> pool;
  for (int t = 0; t < T; ++t) {
    pool.emplace_back([&, t]() {
      cudaSetDevice(bt->device);
      cudaStream_t ts = bt->wstreams[t];
      for (int c = t; c < nchains; c += T) {
        st[c] = setup_impl(&As[c], p, ts, &bt->h[c], false);
        if (st[c] != BAMG_OK) err[c] = bamg_last_error();
      }
      cudaStreamSynchronize(ts);
    });
  }
  for (auto& th : pool) th.join();
  const bool trace = std::getenv("BAMG_TRACE") != nullptr;
  auto since = [&]() { return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count(); };
  if (trace) fprintf(stderr, "[bamg] batch: %d chain setups done (%.1f ms)\n", nchains, since());
  for (int c = 0; c < nchains; ++c)
    if (st[c] != BAMG_OK) {
      set_error("chain %d: %s", c, err[c].c_str());
      bamg_status r = st[c];
      bamg_destroy_batched(bt);
      return r;
    }
  bt->order.resize(nchains);
  for (int c = 0; c < nchains; ++c) bt->order[c] = c;
  std::stable_sort(bt->order.begin(), bt->order.end(),
                   [&](int a, int b) { return bt->h[a]->lv.size() > bt->h[b]->lv.size(); });
  bt->in_off.assign(nchains + 1, 0);
  for (int c = 0; c < nchains; ++c) bt->in_off[c + 1] = bt->in_off[c] + bt->h[c]->lv[0].n;
  if (trace) fprintf(stderr, "[bamg] batch: sorted, n0 = %lld (%.1f ms)\n", (long long)bt->in_off[nchains], since());
  bamg_status r = build_levels(bt, s);
  if (trace) fprintf(stderr, "[bamg] batch: levels built (%d), status %d (%.1f ms)\n", (int)bt->lv.size(), (int)r, since());
  if (r == BAMG_OK) r = bvcycle_prepare(bt);
  if (trace) fprintf(stderr, "[bamg] batch: V-cycle graph status %d (%.1f ms)\n", (int)r, since());
  if (r != BAMG_OK) {
    cudaStreamSynchronize(s);
    bamg_destroy_batched(bt);
    return r;
  }
  bt->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = bt;
  return BAMG_OK;
}

extern "C" bamg_status bamg_solve_batched(bamg_batch* bt, double* x_dev, const bamg_solve_params* sp,
                                          bamg_solve_info* infos, void* stream) {
  BAMG_CHECK_ARG(bt && x_dev && sp);
  BAMG_CHECK_ARG(sp->restart >= 1 && sp->restart <= 64 && sp->max_iter >= 1 && sp->tol > 0.0);
  if (sp->plain) {
    set_error("batches are solved with the V-cycle only (plain = 0)");
    return BAMG_ERR_UNSUPPORTED;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  auto t0 = std::chrono::steady_clock::now();
  const int n0 = bt->lv[0].n;
  DevMem xb;
  BAMG_TRY(xb.alloc(sizeof(double) * n0, s));
  std::vector<bamg_solve_info> local;
  if (!infos) {
    local.assign(bt->nch, bamg_solve_info{});
    infos = local.data();
  }
  bamg_status r = batched_fgmres(bt, xb.as<double>(), sp, infos, s);
  for (int pos = 0; pos < bt->nch; ++pos) {
    int c = bt->order[pos];
    BAMG_CUDA(cudaMemcpyAsync(x_dev + bt->in_off[c], xb.as<double>() + bt->off[0][pos],
                              sizeof(double) * (bt->in_off[c + 1] - bt->in_off[c]), cudaMemcpyDeviceToDevice, s));
  }
  BAMG_CUDA(cudaStreamSynchronize(s));
  if ((r == BAMG_ERR_NOT_CONVERGED || r == BAMG_ERR_BREAKDOWN) && bt->mixed) {
    // chains whose FP32 V-cycle stalled continue alone, from their current
    // x, with FP64 V-cycles (the batch's own V-cycle stays FP32)
    r = BAMG_OK;
    for (int c = 0; c < bt->nch; ++c) {
      if (infos[c].rel_res_1 <= sp->tol) continue;
      bamg_hierarchy* hc = bt->h[c];
      double* xc = x_dev + bt->in_off[c];
      BAMG_TRY(promote_fp64(hc, s));
      BAMG_CUDA(cudaMemcpyAsync(hc->x0.p, xc, sizeof(double) * hc->lv[0].n, cudaMemcpyDeviceToDevice, s));
      bamg_solve_info ic{};
      bamg_status rc = fgmres(hc, xc, sp, &ic, s);
      const int mixed_its = infos[c].iterations;
      infos[c].iterations = mixed_its + ic.iterations;
      infos[c].fallback_iterations = mixed_its;
      infos[c].rel_res_1 = ic.rel_res_1;
      infos[c].min_x = ic.min_x;
      if (rc != BAMG_OK) r = rc;
    }
    BAMG_CUDA(cudaStreamSynchronize(s));
  }
  double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (infos)
    for (int c = 0; c < bt->nch; ++c) infos[c].solve_ms = ms;
  return r;
}

extern "C" bamg_status bamg_vcycle_batched(bamg_batch* bt, const double* r_dev, double* z_dev, void* stream) {
  BAMG_CHECK_ARG(bt && r_dev && z_dev && r_dev != z_dev);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (int pos = 0; pos < bt->nch; ++pos) {
    int c = bt->order[pos];
    BAMG_CUDA(cudaMemcpyAsync(bt->io_in.as<double>() + bt->off[0][pos], r_dev + bt->in_off[c],
                              sizeof(double) * (bt->in_off[c + 1] - bt->in_off[c]), cudaMemcpyDeviceToDevice, s));
  }
  BAMG_TRY(bvcycle_run(bt, s));
  for (int pos = 0; pos < bt->nch; ++pos) {
    int c = bt->order[pos];
    BAMG_CUDA(cudaMemcpyAsync(z_dev + bt->in_off[c], bt->io_out.as<double>() + bt->off[0][pos],
                              sizeof(double) * (bt->in_off[c + 1] - bt->in_off[c]), cudaMemcpyDeviceToDevice, s));
  }
  return BAMG_OK;
}

extern "C" bamg_status bamg_batch_offsets(const bamg_batch* bt, int64_t* offsets_host) {
  BAMG_CHECK_ARG(bt && offsets_host);
  for (int c = 0; c <= bt->nch; ++c) offsets_host[c] = bt->in_off[c];
  return BAMG_OK;
}

extern "C" bamg_status bamg_batch_lanes(const bamg_batch* bt, int level, int* lanes_B, int* lanes_P, int* lanes_Q) {
  BAMG_CHECK_ARG(bt && level >= 0 && level < (int)bt->lv.size() && lanes_B && lanes_P && lanes_Q);
  *lanes_B = bt->lv[level].gB;
  *lanes_P = bt->lv[level].gP;
  *lanes_Q = bt->lv[level].gQ;
  return BAMG_OK;
}

extern "C" bamg_hierarchy* bamg_batch_chain(const bamg_batch* bt, int c) {
  if (!bt || c < 0 || c >= bt->nch) return nullptr;
  return bt->h[c];
}

extern "C" void bamg_destroy_batched(bamg_batch* bt) {
  if (!bt) return;
  if (bt->ge) cudaGraphExecDestroy(bt->ge);
  if (bt->g) cudaGraphDestroy(bt->g);
  if (bt->cap) {
    cudaStreamSynchronize(bt->cap);
    cudaStreamDestroy(bt->cap);
  }
  for (auto* h : bt->h) bamg_destroy(h);
  for (cudaStream_t ws : bt->wstreams)
    if (ws) {
      cudaStreamSynchronize(ws);
      cudaStreamDestroy(ws);
    }
  delete bt;
}
