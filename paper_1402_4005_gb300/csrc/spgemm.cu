// Two-phase sparse matrix product C = A B by expand-sort-compress.
//
// Row i of C is built by one group of threads (a warp, or a whole block for
// long rows): the products a_ik b_kj of row i are expanded into shared memory
// with key (j << 32 | sequence number), sorted by a bitonic network, and
// compressed.  The symbolic pass counts distinct j; the numeric pass sums each
// run of equal j in sequence order, so results do not depend on scheduling.
// Every structural product keeps its slot (no cancellation drops), which is
// the pattern convention of the Petrov-Galerkin products Q B P, Q M Q^T and
// P^T N P (Section 3, Algorithm 1).
#include <atomic>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace bamg {

constexpr int kWarpCap = 256;      // products per row handled by one warp (20 KB of shared memory per block of 4)
constexpr int kBlockCap = 8192;    // products per row handled by one block
constexpr int kWarpsPerBlock = 4;
constexpr int kBigThreads = 256;

// stats[0] = largest row product count, stats[1..2] = 64-bit total (one
// atomic pair per warp)
__global__ void count_products_kernel(int m, const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                                      const int32_t* __restrict__ brp, int32_t* __restrict__ prod,
                                      int* __restrict__ stats) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  long long c = 0;
  if (i < m) {
    for (int p = arp[i]; p < arp[i + 1]; ++p) {
      int k = aci[p];
      c += brp[k + 1] - brp[k];
    }
    prod[i] = c > INT32_MAX ? INT32_MAX : (int)c;
  }
  int mx = c > INT32_MAX ? INT32_MAX : (int)c;
  unsigned long long sum = (unsigned long long)c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
  }
  if ((threadIdx.x & 31) == 0 && sum > 0) {
    atomicMax(stats, mx);
    atomicAdd(reinterpret_cast<unsigned long long*>(stats + 2), sum);
  }
}

template <int G>
__device__ inline void gsync() {
  if constexpr (G == 32) __syncwarp(); else __syncthreads();
}

// Bitonic sort of m (power of two) keys with attached values by G threads.
template <int G, bool VALS>
__device__ void group_sort(unsigned long long* key, double* val, int m, int lane) {
  for (int k = 2; k <= m; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < m; i += G) {
        int ixj = i ^ j;
        if (ixj > i) {
          bool up = (i & k) == 0;
          unsigned long long a = key[i], b = key[ixj];
          if ((a > b) == up) {
            key[i] = b; key[ixj] = a;
            if (VALS) { double t = val[i]; val[i] = val[ixj]; val[ixj] = t; }
          }
        }
      }
      gsync<G>();
    }
  }
}

// The smem rows key/val of mp (a power of two, 32 E) entries sorted through
// registers by one warp.
template <int E, bool VALS>
__device__ inline void warp_sort_smem(unsigned long long* key, double* val, int lane) {
  unsigned long long k[E];
  double v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    k[e] = key[lane * E + e];
    v[e] = VALS ? val[lane * E + e] : 0.0;
  }
  warp_sort_regs<E, VALS>(k, v, lane);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    key[lane * E + e] = k[e];
    if (VALS) val[lane * E + e] = v[e];
  }
  __syncwarp();
}

// Expand the products of row i into key/val (count entries), pad to pow2.
template <int G, bool VALS>
__device__ int expand_row(int i, const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                          const double* __restrict__ ava, const int32_t* __restrict__ brp,
                          const int32_t* __restrict__ bci, const double* __restrict__ bva,
                          int count, unsigned long long* key, double* val, int lane) {
  // sequential enumeration split across lanes: lane handles A entries
  // p = a0 + lane, a0 + lane + G, ...; the sequence number of a product is
  // its position in the row-major enumeration (A order, then B order).
  int a0 = arp[i], a1 = arp[i + 1];
  // prefix of B-row lengths over A entries, computed redundantly per entry
  for (int p = a0 + lane; p < a1; p += G) {
    int k = aci[p];
    int off = 0;
    for (int q = a0; q < p; ++q) {
      int kk = aci[q];
      off += brp[kk + 1] - brp[kk];
    }
    double av = VALS ? ava[p] : 0.0;
    for (int t = brp[k]; t < brp[k + 1]; ++t, ++off) {
      key[off] = ((unsigned long long)(unsigned)bci[t] << 32) | (unsigned)off;
      if (VALS) val[off] = av * bva[t];
    }
  }
  int mp = 1;
  while (mp < count) mp <<= 1;
  for (int t = count + lane; t < mp; t += G) key[t] = ~0ull;
  gsync<G>();
  return mp;
}

// Symbolic: distinct columns of row i.  Numeric: write sorted columns and
// run sums.  Rows whose product count is outside (lo, hi] are skipped.
template <int G, bool NUMERIC>
__device__ void row_product(int i, int lo, int hi, const int32_t* __restrict__ prod,
                            const int32_t* __restrict__ arp, const int32_t* __restrict__ aci,
                            const double* __restrict__ ava, const int32_t* __restrict__ brp,
                            const int32_t* __restrict__ bci, const double* __restrict__ bva,
                            int32_t* __restrict__ ccount, const int32_t* __restrict__ crp,
                            int32_t* __restrict__ cci, double* __restrict__ cva,
                            unsigned long long* key, double* val, int* flag, int lane) {
  int count = prod[i];
  if (count <= lo || count > hi) return;
  int mp = expand_row<G, NUMERIC>(i, arp, aci, ava, brp, bci, bva, count, key, val, lane);
  if constexpr (G == 32) {
    // rows of up to 256 products: the sort in registers (padding keys ~0
    // fill the row to 32 E entries)
    if (mp <= 256) {
      const int E = mp <= 32 ? 1 : mp <= 64 ? 2 : mp <= 128 ? 4 : 8;
      for (int t = mp + lane; t < 32 * E; t += 32) key[t] = ~0ull;
      __syncwarp();
      if (E == 1) warp_sort_smem<1, NUMERIC>(key, val, lane);
      else if (E == 2) warp_sort_smem<2, NUMERIC>(key, val, lane);
      else if (E == 4) warp_sort_smem<4, NUMERIC>(key, val, lane);
      else warp_sort_smem<8, NUMERIC>(key, val, lane);
    } else {
      group_sort<G, NUMERIC>(key, val, mp, lane);
    }
  } else {
    group_sort<G, NUMERIC>(key, val, mp, lane);
  }
  // segment starts
  for (int t = lane; t < count; t += G) {
    unsigned c = (unsigned)(key[t] >> 32);
    flag[t] = (t == 0 || (unsigned)(key[t - 1] >> 32) != c) ? 1 : 0;
  }
  gsync<G>();
  if (!NUMERIC) {
    int s = 0;
    for (int t = lane; t < count; t += G) s += flag[t];
    // reduce within the group
    if constexpr (G == 32) {
      s = warp_sum(s);
      if (lane == 0) ccount[i] = s;
    } else {
      s = warp_sum(s);
      __shared__ int red[32];
      if ((lane & 31) == 0) red[lane >> 5] = s;
      __syncthreads();
      if (lane == 0) {
        int tot = 0;
        for (int w = 0; w < G / 32; ++w) tot += red[w];
        ccount[i] = tot;
      }
      __syncthreads();
    }
    gsync<G>();
    return;
  }
  // exclusive prefix of flags, sequential chunks per lane
  int chunk = (count + G - 1) / G;
  int b = lane * chunk, e = min(count, b + chunk);
  int local = 0;
  for (int t = b; t < e; ++t) local += flag[t];
  int incl = local;
  if constexpr (G == 32) {
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
  } else {
    __shared__ int sc[kBigThreads];
    sc[lane] = local;
    __syncthreads();
    if (lane == 0) {
      int run = 0;
      for (int w = 0; w < G; ++w) { run += sc[w]; sc[w] = run; }
    }
    __syncthreads();
    incl = sc[lane];
    if (ccount != nullptr && lane == 0) ccount[i] = sc[G - 1];
    __syncthreads();
  }
  if constexpr (G == 32) {
    const int tot = __shfl_sync(0xffffffffu, incl, 31);
    if (ccount != nullptr && lane == 0) ccount[i] = tot;
  }
  int pos = incl - local;
  int base = crp[i];
  for (int t = b; t < e; ++t) {
    if (flag[t]) {
      unsigned c = (unsigned)(key[t] >> 32);
      double sum = 0.0;
      for (int u = t; u < count && (unsigned)(key[u] >> 32) == c; ++u) sum += val[u];
      cci[base + pos] = (int32_t)c;
      cva[base + pos] = sum;
      ++pos;
    }
  }
  gsync<G>();
}

template <bool NUMERIC>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
spgemm_warp_kernel(int m, const int32_t* __restrict__ prod, const int32_t* __restrict__ arp,
                   const int32_t* __restrict__ aci, const double* __restrict__ ava,
                   const int32_t* __restrict__ brp, const int32_t* __restrict__ bci,
                   const double* __restrict__ bva, int32_t* __restrict__ ccount,
                   const int32_t* __restrict__ crp, int32_t* __restrict__ cci, double* __restrict__ cva) {
  pdl_wait();
  pdl_trigger();
  __shared__ unsigned long long skey[kWarpsPerBlock][kWarpCap];
  __shared__ double sval[kWarpsPerBlock][NUMERIC ? kWarpCap : 1];
  __shared__ int sflag[kWarpsPerBlock][kWarpCap];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int i = blockIdx.x * kWarpsPerBlock + w;
  if (i >= m) return;
  row_product<32, NUMERIC>(i, -1, kWarpCap, prod, arp, aci, ava, brp, bci, bva, ccount, crp, cci,
                           cva, skey[w], sval[w], sflag[w], lane);
}

template <bool NUMERIC>
__global__ void __launch_bounds__(kBigThreads)
spgemm_block_kernel(int m, const int32_t* __restrict__ prod, const int32_t* __restrict__ arp,
                    const int32_t* __restrict__ aci, const double* __restrict__ ava,
                    const int32_t* __restrict__ brp, const int32_t* __restrict__ bci,
                    const double* __restrict__ bva, int32_t* __restrict__ ccount,
                    const int32_t* __restrict__ crp, int32_t* __restrict__ cci, double* __restrict__ cva) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ unsigned char dyn[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(dyn);
  double* val = reinterpret_cast<double*>(key + kBlockCap);
  int* flag = reinterpret_cast<int*>(val + (NUMERIC ? kBlockCap : 1));
  int i = blockIdx.x;
  if (prod[i] <= kWarpCap) return;
  row_product<kBigThreads, NUMERIC>(i, kWarpCap, kBlockCap, prod, arp, aci, ava, brp, bci, bva,
                                    ccount, crp, cci, cva, key, val, flag, threadIdx.x);
}

struct SpgemmPlan {
  DevMem prod, stats;
  int maxprod = 0;
  long long total = 0;
};

static bamg_status plan_products(int m, const int32_t* arp, const int32_t* aci, const int32_t* brp,
                                 SpgemmPlan& pl, cudaStream_t s) {
  BAMG_TRY(pl.prod.alloc(sizeof(int32_t) * (m + 1), s));
  BAMG_TRY(pl.stats.alloc(4 * sizeof(int), s));
  BAMG_CUDA(cudaMemsetAsync(pl.stats.p, 0, 4 * sizeof(int), s));
  BAMG_TRY(launch(count_products_kernel, dim3(cdiv(m, 256)), dim3(256), 0, s, m, arp, aci, brp,
                  pl.prod.as<int32_t>(), pl.stats.as<int>()));
  int h[4];
  BAMG_CUDA(cudaMemcpyAsync(h, pl.stats.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  pl.maxprod = h[0];
  unsigned long long t = 0;
  std::memcpy(&t, h + 2, sizeof(t));
  pl.total = (long long)t;
  if (pl.maxprod > kBlockCap) {
    set_error("sparse product row with %d products exceeds the %d limit", pl.maxprod, kBlockCap);
    return BAMG_ERR_NUMERIC;
  }
  if (pl.total > INT32_MAX) {
    set_error("sparse product with %lld products exceeds the int32 index range", pl.total);
    return BAMG_ERR_UNSUPPORTED;
  }
  return BAMG_OK;
}

static size_t big_smem(bool numeric) {
  return sizeof(unsigned long long) * kBlockCap + sizeof(double) * (numeric ? kBlockCap : 1) +
         sizeof(int) * kBlockCap;
}

template <bool NUMERIC>
static bamg_status run_rows(int m, const int32_t* prod, int maxprod, const int32_t* arp, const int32_t* aci,
                            const double* ava, const int32_t* brp, const int32_t* bci,
                            const double* bva, int32_t* ccount, const int32_t* crp, int32_t* cci,
                            double* cva, cudaStream_t s) {
  BAMG_TRY(launch(spgemm_warp_kernel<NUMERIC>, dim3(cdiv(m, kWarpsPerBlock)), dim3(kWarpsPerBlock * 32),
                  0, s, m, prod, arp, aci, ava, brp, bci, bva, ccount, crp, cci, cva));
  if (maxprod > kWarpCap) {
    size_t sm = big_smem(NUMERIC);
    static std::atomic<uint64_t> attr_done{0};
    int max_dyn = 0;
    BAMG_TRY(allow_max_smem((const void*)spgemm_block_kernel<NUMERIC>, attr_done, &max_dyn));
    BAMG_TRY(launch(spgemm_block_kernel<NUMERIC>, dim3(m), dim3(kBigThreads), sm, s, m,
                    prod, arp, aci, ava, brp, bci, bva, ccount, crp,
                    cci, cva));
  }
  return BAMG_OK;
}

bamg_status spgemm_symbolic(int m, const int32_t* arp, const int32_t* aci, const int32_t* brp,
                            const int32_t* bci, int32_t* crp, int64_t* nnz_host, cudaStream_t s) {
  SpgemmPlan pl;
  BAMG_TRY(plan_products(m, arp, aci, brp, pl, s));
  DevMem cnt;
  BAMG_TRY(cnt.alloc(sizeof(int32_t) * (m + 1), s));
  BAMG_TRY(run_rows<false>(m, pl.prod.as<int32_t>(), pl.maxprod, arp, aci, nullptr, brp, bci, nullptr, cnt.as<int32_t>(), nullptr,
                           nullptr, nullptr, s));
  return scan_counts(cnt.as<int32_t>(), crp, m, s, nnz_host);
}

__global__ void compact_rows_kernel(int m, const int32_t* __restrict__ src_rp, const int32_t* __restrict__ cnt,
                                    const int32_t* __restrict__ scol, const double* __restrict__ sval,
                                    const int32_t* __restrict__ crp, int32_t* __restrict__ cci,
                                    double* __restrict__ cva) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (i >= m) return;
  const int a = src_rp[i], b = crp[i], c = cnt[i];
  for (int t = lane; t < c; t += 32) {
    cci[b + t] = scol[a + t];
    cva[b + t] = sval[a + t];
  }
}

// ------------------------------------------------- several products at once
// Up to kMaxJobs independent products share each launch (blockIdx.y = job).
constexpr int kMaxJobs = 4;
struct SpJobs {
  int k = 0;
  int m[kMaxJobs];
  const int32_t *arp[kMaxJobs], *aci[kMaxJobs], *brp[kMaxJobs], *bci[kMaxJobs];
  const double *ava[kMaxJobs], *bva[kMaxJobs];
  int32_t *prod[kMaxJobs], *offs[kMaxJobs], *cnts[kMaxJobs];
  int* stats[kMaxJobs];
  int32_t* scol[kMaxJobs];
  double* sval[kMaxJobs];
  const int32_t* crp[kMaxJobs];
  int32_t* cci[kMaxJobs];
  double* cva[kMaxJobs];
  // bounded path (longl != nullptr): rows of more than kWarpCap products,
  // their count in stats[1]; info = {overflow, nnz(C), entries of C's
  // longest row, 0}; cap = scratch entries
  int32_t* longl[kMaxJobs];
  int* info[kMaxJobs];
  long long cap[kMaxJobs];
};

// products per row, and per job their maximum and total (one atomic pair
// per warp: a million rows updating two counters one by one serialise)
__global__ void count_products_multi(SpJobs J) {
  pdl_wait();
  pdl_trigger();
  const int q = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  long long c = 0;
  if (i < J.m[q]) {
    for (int p = J.arp[q][i]; p < J.arp[q][i + 1]; ++p) {
      const int k = J.aci[q][p];
      c += J.brp[q][k + 1] - J.brp[q][k];
    }
    J.prod[q][i] = c > INT32_MAX ? INT32_MAX : (int)c;
    if (J.longl[q] && c > kWarpCap) {
      if (c > kBlockCap) atomicExch(J.info[q], 1);             // no kernel takes such a row
      else J.longl[q][atomicAdd(J.stats[q] + 1, 1)] = i;
    }
  }
  int mx = c > INT32_MAX ? INT32_MAX : (int)c;
  unsigned long long sum = (unsigned long long)c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
  }
  if ((threadIdx.x & 31) == 0 && sum > 0) {
    atomicMax(J.stats[q], mx);
    atomicAdd(reinterpret_cast<unsigned long long*>(J.stats[q] + 2), sum);
  }
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32) spgemm_warp_multi(SpJobs J) {
  pdl_wait();
  pdl_trigger();
  __shared__ unsigned long long skey[kWarpsPerBlock][kWarpCap];
  __shared__ double sval[kWarpsPerBlock][kWarpCap];
  __shared__ int sflag[kWarpsPerBlock][kWarpCap];
  const int q = blockIdx.y;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kWarpsPerBlock + w;
  if (i >= J.m[q]) return;
  if (J.info[q]) {   // bounded scratch: a row that would not fit is not written
    const int c = J.prod[q][i];
    if (c <= kWarpCap && (long long)J.offs[q][i] + c > J.cap[q]) {
      if (lane == 0) atomicExch(J.info[q], 1);
      return;
    }
  }
  row_product<32, true>(i, -1, kWarpCap, J.prod[q], J.arp[q], J.aci[q], J.ava[q], J.brp[q], J.bci[q], J.bva[q],
                        J.cnts[q], J.offs[q], J.scol[q], J.sval[q], skey[w], sval[w], sflag[w], lane);
}

// Bounded path: the rows of more than kWarpCap products, a block each, from
// the list the count kernel built (blocks stride over it).
__global__ void __launch_bounds__(kBigThreads) spgemm_block_list_multi(SpJobs J) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ unsigned char dyn[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(dyn);
  double* val = reinterpret_cast<double*>(key + kBlockCap);
  int* flag = reinterpret_cast<int*>(val + kBlockCap);
  const int q = blockIdx.y;
  const int nl = J.stats[q][1];
  for (int idx = blockIdx.x; idx < nl; idx += gridDim.x) {
    const int i = J.longl[q][idx];
    const int c = J.prod[q][i];
    if ((long long)J.offs[q][i] + c > J.cap[q]) {
      if (threadIdx.x == 0) atomicExch(J.info[q], 1);
      continue;
    }
    row_product<kBigThreads, true>(i, kWarpCap, kBlockCap, J.prod[q], J.arp[q], J.aci[q], J.ava[q], J.brp[q],
                                   J.bci[q], J.bva[q], J.cnts[q], J.offs[q], J.scol[q], J.sval[q], key, val, flag,
                                   threadIdx.x);
  }
}

// Bounded path: info[1] = nnz(C) = crp[m], info[2] = entries of the longest row.
__global__ void spgemm_info_multi(SpJobs J) {
  pdl_wait();
  pdl_trigger();
  const int q = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int c = i < J.m[q] ? J.cnts[q][i] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c = max(c, __shfl_xor_sync(0xffffffffu, c, o));
  if ((threadIdx.x & 31) == 0 && c > 0) atomicMax(J.info[q] + 2, c);
  if (blockIdx.x == 0 && threadIdx.x == 0) J.info[q][1] = J.crp[q][J.m[q]];
}

__global__ void compact_rows_multi(SpJobs J) {
  pdl_wait();
  pdl_trigger();
  const int q = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (i >= J.m[q]) return;
  const int a = J.offs[q][i], b = J.crp[q][i], c = J.cnts[q][i];
  for (int t = lane; t < c; t += 32) {
    J.cci[q][b + t] = J.scol[q][a + t];
    J.cva[q][b + t] = J.sval[q][a + t];
  }
}

// One expansion pass: each row's sorted, summed entries go to a scratch
// slot of its product count, then the rows are packed into C.  Two host
// reads: the product statistics (buffer sizes) and nnz(C).
bamg_status spgemm(int m, const int32_t* arp, const int32_t* aci, const double* ava, const int32_t* brp,
                   const int32_t* bci, const double* bva, DevMem& crp, DevMem& cci, DevMem& cva, int64_t* nnz_host,
                   cudaStream_t s) {
  SpgemmPlan pl;
  BAMG_TRY(plan_products(m, arp, aci, brp, pl, s));
  DevMem off, cnt, scol, sval;
  BAMG_TRY(off.alloc(sizeof(int32_t) * (m + 1), s));
  BAMG_TRY(scan_counts(pl.prod.as<int32_t>(), off.as<int32_t>(), m, s, nullptr));
  BAMG_TRY(cnt.alloc(sizeof(int32_t) * (m + 1), s));
  BAMG_TRY(scol.alloc(sizeof(int32_t) * (pl.total > 0 ? pl.total : 1), s));
  BAMG_TRY(sval.alloc(sizeof(double) * (pl.total > 0 ? pl.total : 1), s));
  BAMG_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * (m + 1), s));
  BAMG_TRY(run_rows<true>(m, pl.prod.as<int32_t>(), pl.maxprod, arp, aci, ava, brp, bci, bva, cnt.as<int32_t>(), off.as<int32_t>(),
                          scol.as<int32_t>(), sval.as<double>(), s));
  BAMG_TRY(crp.alloc(sizeof(int32_t) * (m + 1), s));
  BAMG_TRY(scan_counts(cnt.as<int32_t>(), crp.as<int32_t>(), m, s, nnz_host));
  BAMG_TRY(cci.alloc(sizeof(int32_t) * (*nnz_host > 0 ? *nnz_host : 1), s));
  BAMG_TRY(cva.alloc(sizeof(double) * (*nnz_host > 0 ? *nnz_host : 1), s));
  return launch(compact_rows_kernel, dim3(cdiv((long long)m * 32, 256)), dim3(256), 0, s, m,
                (const int32_t*)off.as<int32_t>(), (const int32_t*)cnt.as<int32_t>(),
                (const int32_t*)scol.as<int32_t>(), (const double*)sval.as<double>(),
                (const int32_t*)crp.as<int32_t>(), cci.as<int32_t>(), cva.as<double>());
}

// Several independent products at once: each phase is issued for every
// product before the one host read that phase needs (product statistics,
// then the nnz of every result), so k products cost two host reads.
// Bounded: the scratch of job q holds cap_q = annz_q * maxrow_b_q products (at
// least the true count), so the counts need no host read; rows that would not
// fit are not written and raise the overflow flag.  One host read: the flags,
// nnz(C) and the longest row of C.
static bamg_status spgemm_multi_bounded(SpgemmJob* jobs, int k, const long long* cap, cudaStream_t s) {
  // per job: stats(4), info(4); then prod, offs, cnts (m + 1 each), long rows (m)
  std::vector<size_t> ro(k + 1, 0);
  for (int q = 0; q < k; ++q) ro[q + 1] = ro[q] + 3 * (size_t)(jobs[q].m + 1) + (size_t)jobs[q].m;
  DevMem ints;
  const size_t head = 8 * (size_t)k;
  BAMG_TRY(ints.alloc(sizeof(int32_t) * (head + ro[k]), s));
  BAMG_CUDA(cudaMemsetAsync(ints.p, 0, sizeof(int32_t) * (head + ro[k]), s));
  int* hd = ints.as<int>();
  int32_t* rows = ints.as<int32_t>() + head;
  SpJobs J;
  J.k = k;
  int maxm = 0;
  std::vector<size_t> so(k + 1, 0);
  for (int q = 0; q < k; ++q) {
    const SpgemmJob& S = jobs[q];
    J.m[q] = S.m;
    J.arp[q] = S.arp; J.aci[q] = S.aci; J.ava[q] = S.ava;
    J.brp[q] = S.brp; J.bci[q] = S.bci; J.bva[q] = S.bva;
    J.prod[q] = rows + ro[q];
    J.offs[q] = rows + ro[q] + (S.m + 1);
    J.cnts[q] = rows + ro[q] + 2 * (size_t)(S.m + 1);
    J.longl[q] = rows + ro[q] + 3 * (size_t)(S.m + 1);
    J.stats[q] = hd + 8 * q;
    J.info[q] = hd + 8 * q + 4;
    J.cap[q] = cap[q];
    so[q + 1] = so[q] + (size_t)(cap[q] > 0 ? cap[q] : 1);
    maxm = S.m > maxm ? S.m : maxm;
  }
  BAMG_TRY(launch(count_products_multi, dim3(cdiv(maxm, 256), k), dim3(256), 0, s, J));
  DevMem scol, sval;
  BAMG_TRY(scol.alloc(sizeof(int32_t) * so[k], s));
  BAMG_TRY(sval.alloc(sizeof(double) * so[k], s));
  ScanMany sc;
  for (int q = 0; q < k; ++q) {
    J.scol[q] = scol.as<int32_t>() + so[q];
    J.sval[q] = sval.as<double>() + so[q];
    sc.in[sc.k] = J.prod[q];
    sc.out[sc.k] = J.offs[q];
    sc.n[sc.k++] = jobs[q].m;
  }
  BAMG_TRY(scan_many(sc, s));
  BAMG_TRY(launch(spgemm_warp_multi, dim3(cdiv(maxm, kWarpsPerBlock), k), dim3(kWarpsPerBlock * 32), 0, s, J));
  {
    static std::atomic<uint64_t> attr_done{0};
    int max_dyn = 0;
    BAMG_TRY(allow_max_smem((const void*)spgemm_block_list_multi, attr_done, &max_dyn));
    BAMG_TRY(launch(spgemm_block_list_multi, dim3(64, k), dim3(kBigThreads), big_smem(true), s, J));
  }
  ScanMany sc2;
  for (int q = 0; q < k; ++q) {
    BAMG_TRY(jobs[q].crp->alloc(sizeof(int32_t) * (jobs[q].m + 1), s));
    J.crp[q] = jobs[q].crp->as<int32_t>();
    sc2.in[sc2.k] = J.cnts[q];
    sc2.out[sc2.k] = jobs[q].crp->as<int32_t>();
    sc2.n[sc2.k++] = jobs[q].m;
  }
  BAMG_TRY(scan_many(sc2, s));
  BAMG_TRY(launch(spgemm_info_multi, dim3(cdiv(maxm, 256), k), dim3(256), 0, s, J));
  std::vector<int> h(head);
  BAMG_CUDA(cudaMemcpyAsync(h.data(), hd, sizeof(int) * head, cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  for (int q = 0; q < k; ++q) {
    const int* inf = &h[8 * q + 4];
    if (inf[0]) {
      set_error("sparse product: a row exceeds %d products or the products exceed their bound %lld", kBlockCap,
                cap[q]);
      return BAMG_ERR_NUMERIC;
    }
    SpgemmJob& S = jobs[q];
    S.nnz = inf[1];
    S.maxrow_c = inf[2];
    BAMG_TRY(S.cci->alloc(sizeof(int32_t) * (S.nnz > 0 ? S.nnz : 1), s));
    BAMG_TRY(S.cva->alloc(sizeof(double) * (S.nnz > 0 ? S.nnz : 1), s));
    J.cci[q] = S.cci->as<int32_t>();
    J.cva[q] = S.cva->as<double>();
  }
  return launch(compact_rows_multi, dim3(cdiv((long long)maxm * 32, 256), k), dim3(256), 0, s, J);
}

bamg_status spgemm_multi(SpgemmJob* jobs, int k, cudaStream_t s) {
  if (k <= 0) return BAMG_OK;
  if (k > kMaxJobs) {
    for (int q0 = 0; q0 < k; q0 += kMaxJobs)
      BAMG_TRY(spgemm_multi(jobs + q0, k - q0 < kMaxJobs ? k - q0 : kMaxJobs, s));
    return BAMG_OK;
  }
  {
    long long cap[kMaxJobs];
    bool bounded = true;
    for (int q = 0; q < k; ++q) {
      if (jobs[q].annz < 0 || jobs[q].maxrow_b < 0) {
        bounded = false;
        break;
      }
      cap[q] = jobs[q].annz * (long long)jobs[q].maxrow_b;
      bounded = bounded && cap[q] <= INT32_MAX;
    }
    if (bounded) return spgemm_multi_bounded(jobs, k, cap, s);
  }
  // one int32 buffer for the statistics and the per-row arrays of all jobs
  // (product counts, their offsets, entry counts), one pair for the scratch
  std::vector<size_t> ro(k + 1, 0);
  for (int q = 0; q < k; ++q) ro[q + 1] = ro[q] + 3 * (size_t)(jobs[q].m + 1);
  DevMem ints;
  BAMG_TRY(ints.alloc(sizeof(int32_t) * (4 * (size_t)k + ro[k]), s));
  int* stats = ints.as<int>();
  int32_t* rows = ints.as<int32_t>() + 4 * k;
  BAMG_CUDA(cudaMemsetAsync(ints.p, 0, sizeof(int32_t) * (4 * (size_t)k + ro[k]), s));
  SpJobs J;
  J.k = k;
  int maxm = 0;
  for (int q = 0; q < k; ++q) {
    const SpgemmJob& S = jobs[q];
    J.longl[q] = nullptr;
    J.info[q] = nullptr;
    J.cap[q] = 0;
    J.m[q] = S.m;
    J.arp[q] = S.arp; J.aci[q] = S.aci; J.ava[q] = S.ava;
    J.brp[q] = S.brp; J.bci[q] = S.bci; J.bva[q] = S.bva;
    J.prod[q] = rows + ro[q];
    J.offs[q] = rows + ro[q] + (S.m + 1);
    J.cnts[q] = rows + ro[q] + 2 * (size_t)(S.m + 1);
    J.stats[q] = stats + 4 * q;
    maxm = S.m > maxm ? S.m : maxm;
  }
  BAMG_TRY(launch(count_products_multi, dim3(cdiv(maxm, 256), k), dim3(256), 0, s, J));
  std::vector<int> h(4 * k);
  BAMG_CUDA(cudaMemcpyAsync(h.data(), stats, sizeof(int) * 4 * k, cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  std::vector<SpgemmPlan> pl(k);
  std::vector<size_t> so(k + 1, 0);
  for (int q = 0; q < k; ++q) {
    pl[q].maxprod = h[4 * q];
    unsigned long long t = 0;
    std::memcpy(&t, &h[4 * q + 2], sizeof(t));
    pl[q].total = (long long)t;
    if (pl[q].maxprod > kBlockCap) {
      set_error("sparse product row with %d products exceeds the %d limit", pl[q].maxprod, kBlockCap);
      return BAMG_ERR_NUMERIC;
    }
    if (pl[q].total > INT32_MAX) {
      set_error("sparse product with %lld products exceeds the int32 index range", pl[q].total);
      return BAMG_ERR_UNSUPPORTED;
    }
    so[q + 1] = so[q] + (size_t)pl[q].total;
  }
  DevMem scol, sval;
  BAMG_TRY(scol.alloc(sizeof(int32_t) * (so[k] > 0 ? so[k] : 1), s));
  BAMG_TRY(sval.alloc(sizeof(double) * (so[k] > 0 ? so[k] : 1), s));
  ScanMany sc;
  for (int q = 0; q < k; ++q) {
    J.scol[q] = scol.as<int32_t>() + so[q];
    J.sval[q] = sval.as<double>() + so[q];
    sc.in[sc.k] = J.prod[q];
    sc.out[sc.k] = J.offs[q];
    sc.n[sc.k++] = jobs[q].m;
  }
  BAMG_TRY(scan_many(sc, s));
  // rows of up to kWarpCap products: one warp each, all products in one
  // launch; longer rows: a block each, per product
  BAMG_TRY(launch(spgemm_warp_multi, dim3(cdiv(maxm, kWarpsPerBlock), k), dim3(kWarpsPerBlock * 32), 0, s, J));
  for (int q = 0; q < k; ++q)
    if (pl[q].maxprod > kWarpCap) {
      size_t sm = big_smem(true);
      static std::atomic<uint64_t> attr_done{0};
      int max_dyn = 0;
      BAMG_TRY(allow_max_smem((const void*)spgemm_block_kernel<true>, attr_done, &max_dyn));
      BAMG_TRY(launch(spgemm_block_kernel<true>, dim3(J.m[q]), dim3(kBigThreads), sm, s, J.m[q], J.prod[q],
                      J.arp[q], J.aci[q], J.ava[q], J.brp[q], J.bci[q], J.bva[q], J.cnts[q], J.offs[q], J.scol[q],
                      J.sval[q]));
    }
  ScanMany sc2;
  for (int q = 0; q < k; ++q) {
    BAMG_TRY(jobs[q].crp->alloc(sizeof(int32_t) * (jobs[q].m + 1), s));
    J.crp[q] = jobs[q].crp->as<int32_t>();
    sc2.in[sc2.k] = J.cnts[q];
    sc2.out[sc2.k] = jobs[q].crp->as<int32_t>();
    sc2.n[sc2.k++] = jobs[q].m;
  }
  BAMG_TRY(scan_many(sc2, s));
  std::vector<int32_t> nz(k);
  for (int q = 0; q < k; ++q)
    BAMG_CUDA(cudaMemcpyAsync(&nz[q], jobs[q].crp->as<int32_t>() + jobs[q].m, sizeof(int32_t),
                              cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  for (int q = 0; q < k; ++q) {
    SpgemmJob& S = jobs[q];
    S.nnz = nz[q];
    S.maxrow_c = -1;
    BAMG_TRY(S.cci->alloc(sizeof(int32_t) * (S.nnz > 0 ? S.nnz : 1), s));
    BAMG_TRY(S.cva->alloc(sizeof(double) * (S.nnz > 0 ? S.nnz : 1), s));
    J.cci[q] = S.cci->as<int32_t>();
    J.cva[q] = S.cva->as<double>();
  }
  return launch(compact_rows_multi, dim3(cdiv((long long)maxm * 32, 256), k), dim3(256), 0, s, J);
}

bamg_status spgemm_numeric(int m, const int32_t* arp, const int32_t* aci, const double* ava,
                           const int32_t* brp, const int32_t* bci, const double* bva,
                           const int32_t* crp, int32_t* cci, double* cva, cudaStream_t s) {
  SpgemmPlan pl;
  BAMG_TRY(plan_products(m, arp, aci, brp, pl, s));
  return run_rows<true>(m, pl.prod.as<int32_t>(), pl.maxprod, arp, aci, ava, brp, bci, bva, nullptr, crp, cci, cva, s);
}

}  // namespace bamg
