// Structural sparse operations: B = I - A, validation, scan, transpose and
// the two-phase sparse matrix product used for Q B P, Q M Q^T and P^T N P.
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <vector>

#include <map>
#include <array>
#include "internal.cuh"

namespace bamg {

std::atomic<uint64_t> g_launches{0};
thread_local uint64_t t_launches = 0;
thread_local bool t_pdl = false;
static thread_local char t_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_err, sizeof(t_err), fmt, ap);
  va_end(ap);
}

const char* last_error_text() { return t_err; }

// ------------------------------------------------------------ block cache
namespace {
struct ScopeCache {
  // free blocks per stream and size class (256 B << c)
  std::map<cudaStream_t, std::array<std::vector<void*>, 16>> free;
};
thread_local ScopeCache* t_scope = nullptr;
int class_of(size_t bytes) {
  int c = 0;
  for (size_t b = 256; b < bytes; b <<= 1) ++c;
  return c;
}
}  // namespace

AllocScope::AllocScope() : owner(t_scope == nullptr) {
  if (owner) t_scope = new ScopeCache();
}

AllocScope::~AllocScope() {
  if (!owner) return;
  ScopeCache* c = t_scope;
  t_scope = nullptr;
  for (auto& kv : c->free)
    for (auto& v : kv.second)
      for (void* p : v) cudaFreeAsync(p, kv.first);
  delete c;
}

bool scope_active() { return t_scope != nullptr; }

// a free block of this class on stream s, else of the next two larger ones
void* scope_get(size_t bytes, cudaStream_t s, size_t* got) {
  auto it = t_scope->free.find(s);
  if (it == t_scope->free.end()) return nullptr;
  const int c0 = class_of(bytes);
  for (int c = c0; c < c0 + 3 && c < 16; ++c) {
    auto& v = it->second[c];
    if (!v.empty()) {
      void* p = v.back();
      v.pop_back();
      *got = size_t(256) << c;
      return p;
    }
  }
  return nullptr;
}

bool scope_put(void* p, size_t bytes, cudaStream_t s) {
  if (!t_scope) return false;
  const int c = class_of(bytes);
  if (c >= 16 || (size_t(256) << c) != bytes) return false;
  t_scope->free[s][c].push_back(p);
  return true;
}

void configure_pool(int device) {
  static std::mutex mu;
  static bool done[64] = {false};
  std::lock_guard<std::mutex> g(mu);
  if (device < 0 || device >= 64 || done[device]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done[device] = true;
}

int num_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// ------------------------------------------------------------------ scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ inline long long block_excl_scan(long long v, long long* sh, long long* total) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    long long s = lane < (kScanThreads / 32) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < (kScanThreads / 32)) sh[lane] = s;
  }
  __syncthreads();
  long long off = w > 0 ? sh[w - 1] : 0;
  *total = sh[kScanThreads / 32 - 1];
  __syncthreads();
  return off + x - v;
}

__global__ void scan_tile_sums(const int32_t* __restrict__ in, int n, long long* __restrict__ part) {
  pdl_wait();
  pdl_trigger();
  __shared__ long long sh[32];
  long long base = (long long)blockIdx.x * kScanTile;
  long long s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    long long i = base + (long long)threadIdx.x * kScanItems + k;
    if (i < n) s += in[i];
  }
  long long tot;
  block_excl_scan(s, sh, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void scan_partials(long long* part, int nb, long long* total_out) {
  pdl_wait();
  pdl_trigger();
  __shared__ long long sh[32];
  long long carry = 0;
  for (int b0 = 0; b0 < nb; b0 += kScanThreads) {
    int b = b0 + threadIdx.x;
    long long v = b < nb ? part[b] : 0;
    long long tot;
    long long ex = block_excl_scan(v, sh, &tot);
    if (b < nb) part[b] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void scan_apply(const int32_t* __restrict__ in, int n, const long long* __restrict__ part,
                           const long long* __restrict__ total, int32_t* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  __shared__ long long sh[32];
  long long base = (long long)blockIdx.x * kScanTile;
  long long loc[kScanItems];
  long long s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    long long i = base + (long long)threadIdx.x * kScanItems + k;
    loc[k] = i < n ? in[i] : 0;
    s += loc[k];
  }
  long long tot;
  long long ex = block_excl_scan(s, sh, &tot) + part[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k) {
    long long i = base + (long long)threadIdx.x * kScanItems + k;
    if (i < n) out[i] = (int32_t)ex;
    ex += loc[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = (int32_t)*total;
}

// Arrays up to kScanOneBlock entries: one block of 1024 threads, each
// scanning a contiguous chunk of at most 8 (chunk sums, a block scan of
// them, then the chunk prefixes), so the scan is a single launch.  Larger
// arrays take the three-launch tiled scan, which spreads over the SMs (on
// one block, chunks of 64 made the setup of the 256^2 tandem queue 0.2 ms
// slower than the tiled scan's three launches).
constexpr int kScanOneThreads = 1024;
constexpr int kScanOneBlock = 8 * kScanOneThreads;

// Exclusive scan of in[0..n) into out[0..n] by the calling block (1024
// threads, n <= kScanOneBlock).
__device__ void scan_block_body(const int32_t* __restrict__ in, int n, int32_t* __restrict__ out) {
  __shared__ long long sh[kScanOneThreads / 32];
  const int chunk = (n + kScanOneThreads - 1) / kScanOneThreads;
  const int b = threadIdx.x * chunk, e = min(n, b + chunk);
  long long sum = 0;
  for (int i = b; i < e; ++i) sum += in[i];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    long long t = sh[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    sh[lane] = t;
  }
  __syncthreads();
  long long run = (w > 0 ? sh[w - 1] : 0) + x - sum;
  for (int i = b; i < e; ++i) {
    out[i] = (int32_t)run;
    run += in[i];
  }
  if (threadIdx.x == kScanOneThreads - 1) out[n] = (int32_t)sh[kScanOneThreads / 32 - 1];
}

__global__ void __launch_bounds__(kScanOneThreads) scan_one_block(const int32_t* __restrict__ in, int n,
                                                                   int32_t* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  scan_block_body(in, n, out);
}

// several independent scans, one block each (blockIdx.x = array)
__global__ void __launch_bounds__(kScanOneThreads) scan_many_kernel(ScanMany job) {
  pdl_wait();
  pdl_trigger();
  const int q = blockIdx.x;
  scan_block_body(job.in[q], job.n[q], job.out[q]);
}

bamg_status scan_many(const ScanMany& job, cudaStream_t s) {
  bool one = true;
  for (int q = 0; q < job.k; ++q) one = one && job.n[q] <= kScanOneBlock;
  if (one) return job.k > 0 ? launch(scan_many_kernel, dim3(job.k), dim3(kScanOneThreads), 0, s, job) : BAMG_OK;
  for (int q = 0; q < job.k; ++q) BAMG_TRY(scan_counts(job.in[q], job.out[q], job.n[q], s, nullptr));
  return BAMG_OK;
}

bamg_status scan_counts(const int32_t* counts, int32_t* out, int n, cudaStream_t s,
                        int64_t* total_host) {
  if (n <= kScanOneBlock) {
    BAMG_TRY(launch(scan_one_block, dim3(1), dim3(kScanOneThreads), 0, s, counts, n, out));
    if (total_host) {
      int32_t t = 0;
      BAMG_CUDA(cudaMemcpyAsync(&t, out + n, sizeof(t), cudaMemcpyDeviceToHost, s));
      BAMG_CUDA(cudaStreamSynchronize(s));
      *total_host = t;
    }
    return BAMG_OK;
  }
  int nb = (int)cdiv(n > 0 ? n : 1, kScanTile);
  DevMem part;
  BAMG_TRY(part.alloc(sizeof(long long) * (nb + 1), s));
  long long* p = part.as<long long>();
  BAMG_TRY(launch(scan_tile_sums, dim3(nb), dim3(kScanThreads), 0, s, counts, n, p));
  BAMG_TRY(launch(scan_partials, dim3(1), dim3(kScanThreads), 0, s, p, nb, p + nb));
  BAMG_TRY(launch(scan_apply, dim3(nb), dim3(kScanThreads), 0, s, counts, n,
                  (const long long*)p, (const long long*)(p + nb), out));
  if (total_host) {
    long long t = 0;
    BAMG_CUDA(cudaMemcpyAsync(&t, p + nb, sizeof(t), cudaMemcpyDeviceToHost, s));
    BAMG_CUDA(cudaStreamSynchronize(s));
    if (t > INT32_MAX) {
      set_error("scan total %lld exceeds int32 index range", t);
      return BAMG_ERR_UNSUPPORTED;
    }
    *total_host = t;
  }
  return BAMG_OK;
}

// One block per output: each thread sums a strided subset of the nb
// partials, then a fixed-order tree over the block, so the result is the
// same on every run (the order depends on nb only).
constexpr int kReduceThreads = 256;
__global__ void __launch_bounds__(kReduceThreads) reduce_partials_kernel(const double* __restrict__ part, int nb,
                                                                         int K, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[kReduceThreads / 32];
  const int k = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += kReduceThreads) s += part[(size_t)b * K + k];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kReduceThreads / 32; ++w) t += sh[w];
    out[k] = t;
  }
}

bamg_status reduce_partials(const double* partial, int nb, int K, double* out, cudaStream_t s) {
  return launch(reduce_partials_kernel, dim3(K), dim3(kReduceThreads), 0, s, partial, nb, K, out);
}

// ------------------------------------------------------------- B = I - A
__global__ void buildB_count_kernel(int n, const int32_t* __restrict__ rp,
                                    const int32_t* __restrict__ ci, int32_t* __restrict__ cnt) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int has = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) has |= (ci[p] == i);
  cnt[i] = rp[i + 1] - rp[i] + (has ? 0 : 1);
}

__global__ void buildB_fill_kernel(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                   const double* __restrict__ va, const int32_t* __restrict__ brp,
                                   int32_t* __restrict__ bci, double* __restrict__ bva) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int q = brp[i];
  bool placed = false;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int j = ci[p];
    if (!placed && j > i) {
      bci[q] = i; bva[q] = 1.0; ++q; placed = true;
    }
    if (j == i) {
      bci[q] = i; bva[q] = 1.0 + (-va[p]); ++q; placed = true;
    } else {
      bci[q] = j; bva[q] = -va[p]; ++q;
    }
  }
  if (!placed) { bci[q] = i; bva[q] = 1.0; }
}

// Section 2: a_ij >= 0, column sums one; also sorted, in-range indices.
__global__ void check_entries_kernel(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                     const double* __restrict__ va, double* __restrict__ colsum,
                                     unsigned long long* __restrict__ bad) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int prev = -1;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int j = ci[p];
    double a = va[p];
    if (j < 0 || j >= n || j <= prev || !(a >= 0.0)) {
      atomicAdd(bad, 1ull);
      if (j < 0 || j >= n) continue;
    }
    prev = j;
    atomicAdd(&colsum[j], a);
  }
}

__global__ void check_colsum_kernel(int n, const double* __restrict__ colsum, double tol,
                                    unsigned long long* __restrict__ bad) {
  pdl_wait();
  pdl_trigger();
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double c = colsum[j];
  if (!(fabs(c - 1.0) <= tol)) atomicAdd(bad, 1ull);
}

__global__ void check_rowptr_kernel(int n, const int32_t* __restrict__ rp, int64_t nnz,
                                    unsigned long long* __restrict__ bad) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  if (i == 0 && rp[0] != 0) atomicAdd(bad, 1ull);
  if (i == n && rp[n] != nnz) atomicAdd(bad, 1ull);
  if (i < n && rp[i + 1] < rp[i]) atomicAdd(bad, 1ull);
}

bamg_status check_rowptr(int n, const int32_t* rp, int64_t nnz, cudaStream_t s) {
  DevMem bad;
  BAMG_TRY(bad.alloc(sizeof(unsigned long long), s));
  BAMG_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(unsigned long long), s));
  BAMG_TRY(launch(check_rowptr_kernel, dim3(cdiv(n + 1, 256)), dim3(256), 0, s, n, rp, nnz,
                  bad.as<unsigned long long>()));
  unsigned long long h = 0;
  BAMG_CUDA(cudaMemcpyAsync(&h, bad.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  if (h) {
    set_error("row_ptr is not a monotone array from 0 to nnz");
    return BAMG_ERR_ARG;
  }
  return BAMG_OK;
}

// ------------------------------------------------------------ transpose
__global__ void col_count_kernel(int nnz, const int32_t* __restrict__ ci, int32_t* __restrict__ cnt) {
  pdl_wait();
  pdl_trigger();
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nnz) atomicAdd(&cnt[ci[p]], 1);
}

__global__ void transpose_scatter_kernel(int rows, const int32_t* __restrict__ rp,
                                         const int32_t* __restrict__ ci, const double* __restrict__ va,
                                         int32_t* __restrict__ fill, int32_t* __restrict__ tci,
                                         double* __restrict__ tva) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int q = atomicAdd(&fill[ci[p]], 1);
    tci[q] = i;
    if (va) tva[q] = va[p];
  }
}

// Sort each output row by column (the source row), making the result
// independent of the scatter order: one warp per row, rows of up to 32
// entries sorted in registers (the columns of a transposed row are
// distinct), longer rows by insertion on lane 0.
__global__ void sort_rows_warp_kernel(int rows, const int32_t* __restrict__ rp, int32_t* __restrict__ ci,
                                      double* __restrict__ va) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (i >= rows) return;
  const int b = rp[i], e = rp[i + 1], len = e - b;
  if (len <= 1) return;
  if (len > 32) {
    if (lane != 0) return;
    for (int p = b + 1; p < e; ++p) {
      int k = ci[p];
      double v = va ? va[p] : 0.0;
      int q = p - 1;
      while (q >= b && ci[q] > k) {
        ci[q + 1] = ci[q];
        if (va) va[q + 1] = va[q];
        --q;
      }
      ci[q + 1] = k;
      if (va) va[q + 1] = v;
    }
    return;
  }
  unsigned long long key[1] = {lane < len ? (unsigned long long)(unsigned)ci[b + lane] : ~0ull};
  double v[1] = {(va && lane < len) ? va[b + lane] : 0.0};
  warp_sort_regs<1, true>(key, v, lane);
  if (lane < len) {
    ci[b + lane] = (int32_t)key[0];
    if (va) va[b + lane] = v[0];
  }
}

bamg_status transpose_csr(int rows, int cols, int nnz, const int32_t* rp, const int32_t* ci,
                          const double* va, int32_t* trp, int32_t* tci, double* tva, cudaStream_t s) {
  DevMem cnt, fill;
  BAMG_TRY(cnt.alloc(sizeof(int32_t) * (cols + 1), s));
  BAMG_TRY(fill.alloc(sizeof(int32_t) * (cols + 1), s));
  BAMG_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * (cols + 1), s));
  BAMG_TRY(launch(col_count_kernel, dim3(cdiv(nnz, 256)), dim3(256), 0, s, nnz, ci, cnt.as<int32_t>()));
  BAMG_TRY(scan_counts(cnt.as<int32_t>(), trp, cols, s, nullptr));
  BAMG_CUDA(cudaMemcpyAsync(fill.p, trp, sizeof(int32_t) * cols, cudaMemcpyDeviceToDevice, s));
  BAMG_TRY(launch(transpose_scatter_kernel, dim3(cdiv(rows, 256)), dim3(256), 0, s, rows, rp, ci, va,
                  fill.as<int32_t>(), tci, tva));
  BAMG_TRY(launch(sort_rows_warp_kernel, dim3(cdiv((long long)cols * 32, 256)), dim3(256), 0, s, cols,
                  (const int32_t*)trp, tci, tva));
  return BAMG_OK;
}

bamg_status build_B_count(int n, const int32_t* rp, const int32_t* ci, int32_t* cnt, cudaStream_t s) {
  return launch(buildB_count_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n, rp, ci, cnt);
}

bamg_status build_B_fill(int n, const int32_t* rp, const int32_t* ci, const double* va,
                         const int32_t* brp, int32_t* bci, double* bva, cudaStream_t s) {
  return launch(buildB_fill_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n, rp, ci, va, brp, bci, bva);
}

bamg_status check_stochastic(int n, const int32_t* rp, const int32_t* ci, const double* va, double tol,
                             int64_t* bad_host, cudaStream_t s) {
  DevMem colsum, bad;
  BAMG_TRY(colsum.alloc(sizeof(double) * n, s));
  BAMG_TRY(bad.alloc(sizeof(unsigned long long), s));
  BAMG_CUDA(cudaMemsetAsync(colsum.p, 0, sizeof(double) * n, s));
  BAMG_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(unsigned long long), s));
  BAMG_TRY(launch(check_entries_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n, rp, ci, va,
                  colsum.as<double>(), bad.as<unsigned long long>()));
  BAMG_TRY(launch(check_colsum_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n,
                  (const double*)colsum.as<double>(), tol, bad.as<unsigned long long>()));
  unsigned long long h = 0;
  BAMG_CUDA(cudaMemcpyAsync(&h, bad.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  *bad_host = (int64_t)h;
  return BAMG_OK;
}

bamg_status allow_max_smem(const void* fn, std::atomic<uint64_t>& done, int* max_dyn) {
  int dev = 0, optin = 0;
  BAMG_CUDA(cudaGetDevice(&dev));
  BAMG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  BAMG_CUDA(cudaFuncGetAttributes(&fa, fn));
  const int avail = optin - (int)fa.sharedSizeBytes;
  *max_dyn = avail;
  const uint64_t bit = 1ull << (dev & 63);
  if (done.load() & bit) return BAMG_OK;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (done.load() & bit) return BAMG_OK;
  BAMG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, avail));
  done.fetch_or(bit);
  return BAMG_OK;
}

}  // namespace bamg
