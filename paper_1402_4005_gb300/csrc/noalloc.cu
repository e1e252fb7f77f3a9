// bamg_step_norms_weights_noalloc: the norms / least-squares weights step
// with its scratch space in a fixed device array instead of the pool.
//
// Who needs it: callers that must not allocate device memory once they are
// running - services whose device memory is handed out up front by their
// own allocator or a fixed budget, where a cudaMalloc or cudaMallocAsync in
// the middle of a run could fail, stall the stream, or fragment memory the
// caller has already planned.  They pass the block X and read the results as
// with bamg_step_norms_weights; the library touches no allocator.
//
// The scratch is one file-scope __device__ array of about 0.8 MB that every
// GPU which loads this library keeps until the process exits.  Its host-side
// name is only a stand-in, so the device address is looked up once per
// device (cudaGetSymbolAddress, with that device current) at the first call
// on that device; make that first call before any stream capture.  All calls
// share the array: calls that overlap on the GPU (other streams, other host
// threads) race on it and must be serialised by the caller.
//
// cudaDeviceReset loads the module into a new context, where the array may
// sit at another address: the cached address is kept with the identifier of
// the context it was looked up in (cuCtxGetId, reached through the runtime's
// driver entry points, so the library does not link the driver library), and
// a call from a different context looks the address up again.
#include <cuda.h>

#include <mutex>

#include "internal.cuh"

namespace bamg {

constexpr int kNoAllocMaxBlocks = 1024;  // partial-sum rows (grid size cap)
constexpr int kNoAllocMaxLD = 32;        // widest block supported
constexpr size_t kPartDoubles = (size_t)kNoAllocMaxBlocks * 3 * kNoAllocMaxLD;
constexpr size_t kScratchDoubles = kPartDoubles + 3 * kNoAllocMaxLD + 3 * kNoAllocMaxLD;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

static std::mutex g_noalloc_mu;
static double* g_noalloc_addr[256] = {nullptr};
static unsigned long long g_noalloc_ctx[256] = {0};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Identifier of the calling thread's current context, 0 if none or if the
// driver does not provide it.
static unsigned long long current_ctx_id() {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_cur = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
  }
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (!get_cur || !get_id || get_cur(&c) != CUDA_SUCCESS || c == nullptr || get_id(c, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of the scratch array on the current device (looked up once
// per device and context).
static bamg_status noalloc_scratch(double** out) {
  int dev = 0;
  BAMG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) {
    set_error("device index %d out of range", dev);
    return BAMG_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (g_noalloc_addr[dev]) {
    const unsigned long long id = current_ctx_id();
    if (id == 0 || id != g_noalloc_ctx[dev]) g_noalloc_addr[dev] = nullptr;
  }
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("cudaGetSymbolAddress of the fixed scratch failed: %s", cudaGetErrorString(e));
      return BAMG_ERR_CUDA;
    }
    g_noalloc_addr[dev] = static_cast<double*>(p);
    g_noalloc_ctx[dev] = current_ctx_id();
  }
  *out = g_noalloc_addr[dev];
  return BAMG_OK;
}

}  // namespace bamg

using namespace bamg;

extern "C" bamg_status bamg_step_norms_weights_noalloc(int prec, int n, int ld, int r, const int32_t* rp,
                                                       const int32_t* ci, const void* val, void* X,
                                                       int normalise, int skip_col0, double* norm_host,
                                                       double* w_host, void* stream) {
  BAMG_CHECK_ARG(n >= 1 && r >= 1 && rp && ci && val && X && norm_host && w_host && (prec == 0 || prec == 1));
  if (ld != 4 && ld != 8 && ld != 16 && ld != 32) {
    set_error("block width %d is not 4, 8, 16 or 32 (fixed scratch holds ld <= %d)", ld, kNoAllocMaxLD);
    return BAMG_ERR_ARG;
  }
  if (r > ld) {
    set_error("r = %d exceeds the block width %d", r, ld);
    return BAMG_ERR_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double* base = nullptr;
  BAMG_TRY(noalloc_scratch(&base));
  double* part = base;
  double* sums = base + kPartDoubles;
  double* w = sums + 3 * kNoAllocMaxLD;
  double* norms = w + kNoAllocMaxLD;
  double* scale = norms + kNoAllocMaxLD;  // kNoAllocMaxLD doubles, used as T[ld]
  // Every element the launches read is written earlier in the same call
  // (per-block partials, their sums, the per-column factors), so nothing
  // left by a previous call is used and no clearing is needed.
  if (prec == 1)
    BAMG_TRY(norms_weights_ws<float>(n, ld, r, rp, ci, (const float*)val, (float*)X, normalise, skip_col0, part,
                                     kNoAllocMaxBlocks, sums, reinterpret_cast<float*>(scale), w, norms, s));
  else
    BAMG_TRY(norms_weights_ws<double>(n, ld, r, rp, ci, (const double*)val, (double*)X, normalise, skip_col0,
                                      part, kNoAllocMaxBlocks, sums, scale, w, norms, s));
  BAMG_CUDA(cudaMemcpyAsync(norm_host, norms, sizeof(double) * r, cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaMemcpyAsync(w_host, w, sizeof(double) * r, cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  return BAMG_OK;
}
