// C/F splitting and interpolation sets (integer work, bit-exact with the
// sequential definitions).
//
// Geometric (Section 7): coarse points are (i even, j even) of an nx x ny
// grid; J_i = coarse points of the 3x3 box around i.
// Graph: the greedy maximal independent set taken in decreasing SplitMix64
// priority (ties by index) stands in for compatible relaxation, which the
// paper cites without giving; it is computed by parallel rounds (a vertex
// joins when it beats every undecided neighbour), which reach exactly the
// sequential greedy set.  J_i = strongest coarse neighbours, topped up from
// distance two.
#include "internal.cuh"

namespace bamg {

constexpr uint64_t kMisStream = 4096;

__global__ void geo_split_kernel(int nx, int ny, int8_t* __restrict__ cf, int32_t* __restrict__ cmap,
                                 int32_t* __restrict__ jcnt) {
  pdl_wait();
  pdl_trigger();
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nx * ny) return;
  int i = s / ny, j = s % ny;
  int cny = (ny + 1) / 2;
  bool c = (i % 2 == 0) && (j % 2 == 0);
  cf[s] = c ? 1 : 0;
  cmap[s] = c ? (i / 2) * cny + j / 2 : -1;
  int cnt = 0;
  if (!c) {
    for (int di = -1; di <= 1; ++di)
      for (int dj = -1; dj <= 1; ++dj) {
        int a = i + di, b = j + dj;
        if (a >= 0 && a < nx && b >= 0 && b < ny && a % 2 == 0 && b % 2 == 0) ++cnt;
      }
  }
  jcnt[s] = cnt;
}

__global__ void geo_sets_kernel(int nx, int ny, const int32_t* __restrict__ jrp, int32_t* __restrict__ jci) {
  pdl_wait();
  pdl_trigger();
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nx * ny) return;
  int i = s / ny, j = s % ny;
  if (i % 2 == 0 && j % 2 == 0) return;
  int q = jrp[s];
  for (int di = -1; di <= 1; ++di)
    for (int dj = -1; dj <= 1; ++dj) {
      int a = i + di, b = j + dj;
      if (a >= 0 && a < nx && b >= 0 && b < ny && a % 2 == 0 && b % 2 == 0) jci[q++] = a * ny + b;
    }
}

bamg_status coarsen_geometric(int nx, int ny, int8_t* cf, int32_t* cmap, int32_t* J_rp, int32_t* J_ci,
                              int* nc_host, cudaStream_t s) {
  int n = nx * ny;
  DevMem cnt;
  BAMG_TRY(cnt.alloc(sizeof(int32_t) * (n + 1), s));
  BAMG_TRY(launch(geo_split_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, nx, ny, cf, cmap,
                  cnt.as<int32_t>()));
  BAMG_TRY(scan_counts(cnt.as<int32_t>(), J_rp, n, s, nullptr));
  BAMG_TRY(launch(geo_sets_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, nx, ny, (const int32_t*)J_rp, J_ci));
  if (nc_host) *nc_host = ((nx + 1) / 2) * ((ny + 1) / 2);
  return BAMG_OK;
}

// ------------------------------------------------------------------- MIS
__device__ inline bool beats(uint64_t ki, int i, uint64_t kj, int j) {
  return ki > kj || (ki == kj && i < j);
}

// state: 0 undecided, 1 coarse, 2 fine, 3 selected in this round.
__global__ void mis_select_kernel(int n, const int32_t* __restrict__ brp, const int32_t* __restrict__ bci,
                                  const int32_t* __restrict__ trp, const int32_t* __restrict__ tci,
                                  uint64_t seed, int level, int8_t* __restrict__ state) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || state[i] != 0) return;
  uint64_t ki = splitmix_draw(seed, kMisStream + level, i);
  const int32_t* rps[2] = {brp, trp};
  const int32_t* cis[2] = {bci, tci};
  for (int m = 0; m < 2; ++m) {
    for (int p = rps[m][i]; p < rps[m][i + 1]; ++p) {
      int j = cis[m][p];
      if (j == i) continue;
      int8_t sj = state[j];
      if (sj == 0 || sj == 3) {
        if (beats(splitmix_draw(seed, kMisStream + level, j), j, ki, i)) return;
      }
    }
  }
  state[i] = 3;
}

__global__ void mis_finalize_kernel(int n, const int32_t* __restrict__ brp, const int32_t* __restrict__ bci,
                                    const int32_t* __restrict__ trp, const int32_t* __restrict__ tci,
                                    int8_t* __restrict__ state, int* __restrict__ undecided) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int8_t si = state[i];
  if (si == 3) {
    state[i] = 1;
    return;
  }
  if (si != 0) return;
  const int32_t* rps[2] = {brp, trp};
  const int32_t* cis[2] = {bci, tci};
  for (int m = 0; m < 2; ++m)
    for (int p = rps[m][i]; p < rps[m][i + 1]; ++p) {
      int j = cis[m][p];
      if (j == i) continue;
      int8_t sj = state[j];
      if (sj == 1 || sj == 3) {
        state[i] = 2;
        return;
      }
    }
  atomicAdd(undecided, 1);
}

__global__ void state_to_cf_kernel(int n, const int8_t* __restrict__ state, int8_t* __restrict__ cf,
                                   int32_t* __restrict__ cnt) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int8_t c = state[i] == 1 ? 1 : 0;
  cf[i] = c;
  cnt[i] = c;
}

__global__ void cmap_kernel(int n, const int8_t* __restrict__ cf, const int32_t* __restrict__ pre,
                            int32_t* __restrict__ cmap) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  cmap[i] = cf[i] ? pre[i] : -1;
}

bamg_status coarsen_mis(int n, const int32_t* brp, const int32_t* bci, const int32_t* trp,
                        const int32_t* tci, uint64_t seed, int level, int8_t* cf, int32_t* cmap,
                        int* nc_host, cudaStream_t s) {
  DevMem state, und, cnt, pre;
  BAMG_TRY(state.alloc(n, s));
  BAMG_TRY(und.alloc(sizeof(int), s));
  BAMG_TRY(cnt.alloc(sizeof(int32_t) * (n + 1), s));
  BAMG_TRY(pre.alloc(sizeof(int32_t) * (n + 1), s));
  BAMG_CUDA(cudaMemsetAsync(state.p, 0, n, s));
  // rounds are queued four at a time before the host reads the count of
  // undecided vertices (a round over a fully decided state changes nothing)
  constexpr int kRoundsPerCheck = 4;
  for (int round = 0;; round += kRoundsPerCheck) {
    if (round > n + 1) {
      set_error("independent-set rounds did not terminate");
      return BAMG_ERR_NUMERIC;
    }
    for (int q = 0; q < kRoundsPerCheck; ++q) {
      BAMG_CUDA(cudaMemsetAsync(und.p, 0, sizeof(int), s));
      BAMG_TRY(launch(mis_select_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n, brp, bci, trp, tci, seed,
                      level, state.as<int8_t>()));
      BAMG_TRY(launch(mis_finalize_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n, brp, bci, trp, tci,
                      state.as<int8_t>(), und.as<int>()));
    }
    int h = 0;
    BAMG_CUDA(cudaMemcpyAsync(&h, und.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    BAMG_CUDA(cudaStreamSynchronize(s));
    if (h == 0) break;
  }
  BAMG_TRY(launch(state_to_cf_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n,
                  (const int8_t*)state.as<int8_t>(), cf, cnt.as<int32_t>()));
  int64_t nc = 0;
  BAMG_TRY(scan_counts(cnt.as<int32_t>(), pre.as<int32_t>(), n, s, &nc));
  BAMG_TRY(launch(cmap_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n, (const int8_t*)cf,
                  (const int32_t*)pre.as<int32_t>(), cmap));
  if (nc_host) *nc_host = (int)nc;
  return BAMG_OK;
}

// ---------------------------------------------------- graph interpolation
constexpr int kMaxC = 8;
constexpr int kMaxCand = 256;

// Symmetrised neighbours of row i: merge of row i of B and of B^T (both
// ascending); strength |b_ij| + |b_ji|.  Calls f(j, s) for j != i.
template <typename F>
__device__ inline void for_sym_neighbours(int i, const int32_t* __restrict__ brp, const int32_t* __restrict__ bci,
                                          const double* __restrict__ bva, const int32_t* __restrict__ trp,
                                          const int32_t* __restrict__ tci, const double* __restrict__ tva, F f) {
  int p = brp[i], pe = brp[i + 1], q = trp[i], qe = trp[i + 1];
  while (p < pe || q < qe) {
    int jb = p < pe ? bci[p] : INT32_MAX;
    int jt = q < qe ? tci[q] : INT32_MAX;
    int j = jb < jt ? jb : jt;
    double sv = 0.0;
    if (jb == j) { sv = sv + fabs(bva[p]); ++p; }
    if (jt == j) { sv = sv + fabs(tva[q]); ++q; }
    if (j != i) f(j, sv);
  }
}

__device__ inline bool better(double sa, int ja, double sb, int jb) {
  return sa > sb || (sa == sb && ja < jb);
}

__global__ void graph_sets_kernel(int n, const int32_t* __restrict__ brp, const int32_t* __restrict__ bci,
                                  const double* __restrict__ bva, const int32_t* __restrict__ trp,
                                  const int32_t* __restrict__ tci, const double* __restrict__ tva,
                                  const int8_t* __restrict__ cf, int c_min, int c_max,
                                  int32_t* __restrict__ cnt, int32_t* __restrict__ tmp,
                                  int* __restrict__ overflow) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (cf[i]) { cnt[i] = 0; return; }
  int sel[kMaxC];
  double ss[kMaxC];
  int ns = 0;
  // distance one: keep the best c_max by (strength desc, index asc)
  for_sym_neighbours(i, brp, bci, bva, trp, tci, tva, [&](int j, double sv) {
    if (!cf[j]) return;
    int pos = ns;
    while (pos > 0 && better(sv, j, ss[pos - 1], sel[pos - 1])) --pos;
    if (pos >= c_max) return;
    int last = ns < c_max ? ns : c_max - 1;
    for (int t = last; t > pos; --t) { sel[t] = sel[t - 1]; ss[t] = ss[t - 1]; }
    sel[pos] = j; ss[pos] = sv;
    if (ns < c_max) ++ns;
  });
  if (ns < c_min) {
    int cj[kMaxCand];
    double cw[kMaxCand];
    int nc = 0;
    for_sym_neighbours(i, brp, bci, bva, trp, tci, tva, [&](int k, double sik) {
      for_sym_neighbours(k, brp, bci, bva, trp, tci, tva, [&](int j, double skj) {
        if (j == i || !cf[j]) return;
        for (int t = 0; t < ns; ++t) if (sel[t] == j) return;
        double w = sik * skj;
        for (int t = 0; t < nc; ++t)
          if (cj[t] == j) { if (w > cw[t]) cw[t] = w; return; }
        if (nc < kMaxCand) { cj[nc] = j; cw[nc] = w; ++nc; } else { atomicAdd(overflow, 1); }
      });
    });
    while (ns < c_min && nc > 0) {
      int b = 0;
      for (int t = 1; t < nc; ++t) if (better(cw[t], cj[t], cw[b], cj[b])) b = t;
      sel[ns] = cj[b]; ss[ns] = cw[b]; ++ns;
      cj[b] = cj[nc - 1]; cw[b] = cw[nc - 1]; --nc;
    }
  }
  // ascending fine index
  for (int a = 1; a < ns; ++a) {
    int v = sel[a], t = a - 1;
    while (t >= 0 && sel[t] > v) { sel[t + 1] = sel[t]; --t; }
    sel[t + 1] = v;
  }
  cnt[i] = ns;
  for (int t = 0; t < ns; ++t) tmp[(size_t)i * c_max + t] = sel[t];
}

__global__ void compact_sets_kernel(int n, int c_max, const int32_t* __restrict__ tmp,
                                    const int32_t* __restrict__ jrp, int32_t* __restrict__ jci) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int q = jrp[i]; q < jrp[i + 1]; ++q) jci[q] = tmp[(size_t)i * c_max + (q - jrp[i])];
}

bamg_status graph_sets(int n, const int32_t* brp, const int32_t* bci, const double* bva,
                       const int32_t* trp, const int32_t* tci, const double* tva, const int8_t* cf,
                       int c_min, int c_max, int32_t* J_rp, int32_t* J_ci, cudaStream_t s) {
  if (c_max < 1 || c_max > kMaxC || c_min < 1 || c_min > c_max) {
    set_error("interpolation set bounds need 1 <= c_min <= c_max <= %d", kMaxC);
    return BAMG_ERR_ARG;
  }
  DevMem cnt, tmp, ovf;
  BAMG_TRY(cnt.alloc(sizeof(int32_t) * (n + 1), s));
  BAMG_TRY(tmp.alloc(sizeof(int32_t) * (size_t)n * c_max, s));
  BAMG_TRY(ovf.alloc(sizeof(int), s));
  BAMG_CUDA(cudaMemsetAsync(ovf.p, 0, sizeof(int), s));
  BAMG_TRY(launch(graph_sets_kernel, dim3(cdiv(n, 128)), dim3(128), 0, s, n, brp, bci, bva, trp, tci, tva, cf,
                  c_min, c_max, cnt.as<int32_t>(), tmp.as<int32_t>(), ovf.as<int>()));
  int h = 0;
  BAMG_CUDA(cudaMemcpyAsync(&h, ovf.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  if (h) {
    set_error("distance-two candidate list exceeded %d entries", kMaxCand);
    return BAMG_ERR_UNSUPPORTED;
  }
  BAMG_TRY(scan_counts(cnt.as<int32_t>(), J_rp, n, s, nullptr));
  return launch(compact_sets_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n, c_max,
                (const int32_t*)tmp.as<int32_t>(), (const int32_t*)J_rp, J_ci);
}

// ------------------------------------------------------- transfer patterns
__global__ void coarse_points_kernel(int n, const int8_t* __restrict__ cf, const int32_t* __restrict__ cmap,
                                     int32_t* __restrict__ cpt) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && cf[i]) cpt[cmap[i]] = i;
}

bamg_status coarse_points(int n, const int8_t* cf, const int32_t* cmap, int32_t* cpt, cudaStream_t s) {
  return launch(coarse_points_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n, cf, cmap, cpt);
}

__global__ void pattern_count_kernel(int n, const int8_t* __restrict__ cf, const int32_t* __restrict__ jrp,
                                     int32_t* __restrict__ cnt) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  cnt[i] = cf[i] ? 1 : jrp[i + 1] - jrp[i];
}

// eq. Pstructure: identity rows on C; F rows on J_i (coarse indices).
__global__ void pattern_fill_kernel(int n, const int8_t* __restrict__ cf, const int32_t* __restrict__ cmap,
                                    const int32_t* __restrict__ jrp, const int32_t* __restrict__ jci,
                                    const int32_t* __restrict__ prp, int32_t* __restrict__ pci,
                                    double* __restrict__ pva) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int q = prp[i];
  if (cf[i]) {
    pci[q] = cmap[i];
    pva[q] = 1.0;
    return;
  }
  for (int t = jrp[i]; t < jrp[i + 1]; ++t, ++q) {
    pci[q] = cmap[jci[t]];
    pva[q] = 0.0;
  }
}

bamg_status transfer_pattern(int n, const int8_t* cf, const int32_t* cmap, const int32_t* J_rp,
                             const int32_t* J_ci, int32_t* P_rp, int32_t* P_ci, double* P_val,
                             cudaStream_t s) {
  DevMem cnt;
  BAMG_TRY(cnt.alloc(sizeof(int32_t) * (n + 1), s));
  BAMG_TRY(launch(pattern_count_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n, cf, J_rp, cnt.as<int32_t>()));
  BAMG_TRY(scan_counts(cnt.as<int32_t>(), P_rp, n, s, nullptr));
  return launch(pattern_fill_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n, cf, cmap, J_rp, J_ci,
                (const int32_t*)P_rp, P_ci, P_val);
}

__global__ void scatter_fits_kernel(int n, const int8_t* __restrict__ cf, const int32_t* __restrict__ jrp,
                                    const double* __restrict__ fit, const int32_t* __restrict__ prp,
                                    double* __restrict__ pva) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || cf[i]) return;
  int q = prp[i];
  for (int t = jrp[i]; t < jrp[i + 1]; ++t, ++q) pva[q] = fit[t];
}

bamg_status scatter_fits(int n, const int8_t* cf, const int32_t* J_rp, const double* fit,
                         const int32_t* P_rp, double* P_val, cudaStream_t s) {
  return launch(scatter_fits_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n, cf, J_rp, fit, P_rp, P_val);
}

// Section 5 comparison: simple averaging, every entry of a column of Q = 1/c.
__global__ void average_fits_kernel(int n, const int32_t* __restrict__ jrp, double* __restrict__ fit) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = jrp[i + 1] - jrp[i];
  for (int t = jrp[i]; t < jrp[i + 1]; ++t) fit[t] = 1.0 / c;
}

bamg_status average_fits(int n, const int32_t* J_rp, double* fit, cudaStream_t s) {
  return launch(average_fits_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n, J_rp, fit);
}

}  // namespace bamg
