// Internal helpers shared by the translation units of libbamg.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <utility>

#include "bamg.h"
#include "bamg_steps.h"

namespace bamg {

// ------------------------------------------------------------ status plumbing
void set_error(const char* fmt, ...);
extern std::atomic<uint64_t> g_launches;
// launches issued by the calling thread (used to size captured graphs)
extern thread_local uint64_t t_launches;

#define BAMG_TRY(...)                                    \
  do {                                                   \
    bamg_status s_ = (__VA_ARGS__);                      \
    if (s_ != BAMG_OK) return s_;                        \
  } while (0)

#define BAMG_CUDA(...)                                                          \
  do {                                                                          \
    cudaError_t e_ = (__VA_ARGS__);                                             \
    if (e_ != cudaSuccess) {                                                    \
      bamg::set_error("%s:%d %s: %s", __FILE__, __LINE__, #__VA_ARGS__,         \
                      cudaGetErrorString(e_));                                  \
      return e_ == cudaErrorMemoryAllocation ? BAMG_ERR_OOM : BAMG_ERR_CUDA;    \
    }                                                                           \
  } while (0)

#define BAMG_CHECK_ARG(cond)                                         \
  do {                                                               \
    if (!(cond)) {                                                   \
      bamg::set_error("%s:%d invalid argument: %s", __FILE__, __LINE__, #cond); \
      return BAMG_ERR_ARG;                                           \
    }                                                                \
  } while (0)

// Programmatic dependent launch (sm_90 and later).  While t_pdl is set (the
// captures of the V-cycle and Arnoldi graphs, which hold kernel nodes only),
// launch() gives each kernel the programmatic-serialisation attribute: the
// kernel may start while its predecessor on the stream is still running, so
// its launch latency overlaps the predecessor's work.  Every kernel launched
// that way calls pdl_wait() before its first global memory access; it
// returns once the predecessor grid has completed and its writes are
// visible (at once for a kernel launched normally).  pdl_trigger() then lets
// the successor begin launching; it only schedules, it orders nothing.
extern thread_local bool t_pdl;
struct PdlScope {
  bool prev;
  PdlScope() : prev(t_pdl) { t_pdl = true; }
  ~PdlScope() { t_pdl = prev; }
  PdlScope(const PdlScope&) = delete;
  PdlScope& operator=(const PdlScope&) = delete;
};
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch a kernel, count it and check the launch.
template <typename... KArgs, typename... Args>
inline bamg_status launch(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                          cudaStream_t s, Args&&... args) {
  if (grid.x == 0 || grid.y == 0 || grid.z == 0) return BAMG_OK;
  cudaError_t e;
  if (t_pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
  } else {
    k<<<grid, block, smem, s>>>(std::forward<Args>(args)...);
    e = cudaGetLastError();
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
  if (e != cudaSuccess) {
    set_error("kernel launch failed: %s", cudaGetErrorString(e));
    return BAMG_ERR_CUDA;
  }
  return BAMG_OK;
}

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// --------------------------------------------------- stream-ordered buffers
// Block cache of one call (sparse.cu).  While an AllocScope is active on the
// calling thread (the setup), blocks of at most kScopeMax bytes are rounded
// up to a power of two; those released during the call go to a free list of
// their stream and serve later allocations on the same stream in the same
// call (the stream orders the new uses after the old ones), instead of a
// cudaFreeAsync / cudaMallocAsync pair each.  The rest are returned to the
// pool when the scope ends.
constexpr size_t kScopeMax = size_t(8) << 20;
struct AllocScope {
  AllocScope();
  ~AllocScope();
  AllocScope(const AllocScope&) = delete;
  AllocScope& operator=(const AllocScope&) = delete;
  bool owner;
};
bool scope_active();
void* scope_get(size_t bytes, cudaStream_t s, size_t* got);
bool scope_put(void* p, size_t bytes, cudaStream_t s);

// Device memory from the stream-ordered pool (cudaMallocAsync); freed on the
// same stream.  The pool keeps freed blocks, so repeated setups re-use them.
struct DevMem {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = nullptr;
  bool rounded = false;     // a power-of-two block allocated in a scope
  DevMem() = default;
  DevMem(const DevMem&) = delete;
  DevMem& operator=(const DevMem&) = delete;
  DevMem(DevMem&& o) noexcept { *this = std::move(o); }
  DevMem& operator=(DevMem&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p; bytes = o.bytes; s = o.s; rounded = o.rounded;
      o.p = nullptr; o.bytes = 0; o.rounded = false;
    }
    return *this;
  }
  ~DevMem() { release(); }
  void release() {
    if (p && !(rounded && scope_put(p, bytes, s))) cudaFreeAsync(p, s);
    p = nullptr;
    bytes = 0;
    rounded = false;
  }
  bamg_status alloc(size_t nbytes, cudaStream_t st) {
    release();
    s = st;
    if (nbytes == 0) nbytes = 16;
    if (nbytes <= kScopeMax && scope_active()) {
      size_t cls = 256;
      while (cls < nbytes) cls <<= 1;
      rounded = true;
      size_t got = 0;
      if (void* q = scope_get(cls, st, &got)) {
        p = q;
        bytes = got;
        return BAMG_OK;
      }
      nbytes = cls;
    }
    cudaError_t e = cudaMallocAsync(&p, nbytes, st);
    if (e != cudaSuccess) {
      p = nullptr;
      set_error("cudaMallocAsync(%zu) failed: %s", nbytes, cudaGetErrorString(e));
      return BAMG_ERR_OOM;
    }
    bytes = nbytes;
    return BAMG_OK;
  }
  template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

void configure_pool(int device);

// ------------------------------------------------------------ device helpers
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

// SplitMix64 output function (Steele, Lea, Flood 2014; constants of Vigna's
// public-domain splitmix64.c).  Counter-based: output k of a generator with
// state s is mix(s + (k + 1) * gamma).
__host__ __device__ inline uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t splitmix_draw(uint64_t seed, uint64_t stream, uint64_t i) {
  uint64_t ctr = (stream << 32) + i;
  return splitmix_mix(seed + (ctr + 1ull) * kGamma);
}
// uniform(-1, 1): 53 high bits to [0, 1), then 2u - 1 (exact in double).
__host__ __device__ inline double splitmix_pm1(uint64_t seed, uint64_t stream, uint64_t i) {
  double u = (double)(splitmix_draw(seed, stream, i) >> 11) * 0x1.0p-53;
  return 2.0 * u - 1.0;
}

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int W = 2; };

__device__ inline void vload(const float* p, float (&v)[4]) {
  float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ inline void vload(const double* p, double (&v)[2]) {
  double2 t = *reinterpret_cast<const double2*>(p);
  v[0] = t.x; v[1] = t.y;
}
__device__ inline void vstore(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ inline void vstore(double* p, const double (&v)[2]) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
}
__device__ inline void vload_ro(const float* p, float (&v)[4]) {
  float4 t = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ inline void vload_ro(const double* p, double (&v)[2]) {
  double2 t = __ldg(reinterpret_cast<const double2*>(p));
  v[0] = t.x; v[1] = t.y;
}

template <typename T>
__device__ inline T warp_sum(T v, unsigned mask = 0xffffffffu) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

// Sum over aligned groups of G lanes (G power of two <= 32).
template <int G, typename T>
__device__ inline T group_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Bitonic sort of 32 E keys held in registers by one warp, element
// lane * E + e in key[e] (ascending; keys are distinct).  Partners closer
// than E elements are in the same lane; farther ones are exchanged with
// shuffles.  Values travel with their keys.
template <int E, bool VALS>
__device__ inline void warp_sort_regs(unsigned long long (&key)[E], double (&val)[E], int lane) {
  constexpr int N = 32 * E;
#pragma unroll
  for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= E) {
        const int lm = j / E;
        const bool lower = (lane & lm) == 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const unsigned long long pk = __shfl_xor_sync(0xffffffffu, key[e], lm);
          double pv = 0.0;
          if (VALS) pv = __shfl_xor_sync(0xffffffffu, val[e], lm);
          const bool up = ((lane * E + e) & k) == 0;
          const bool take = (lower == up) ? (pk < key[e]) : (pk > key[e]);
          if (take) {
            key[e] = pk;
            if (VALS) val[e] = pv;
          }
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if ((e & j) == 0) {
            const int f = e | j;
            const bool up = ((lane * E + e) & k) == 0;
            if ((key[e] > key[f]) == up) {
              const unsigned long long t = key[e]; key[e] = key[f]; key[f] = t;
              if (VALS) { const double tv = val[e]; val[e] = val[f]; val[f] = tv; }
            }
          }
        }
      }
    }
  }
}

// ----------------------------------------------------- small internal APIs
// Exclusive scan of n int32 counts into out[0..n] (out[n] = total), int64
// total returned through total_host when non-null (synchronises the stream).
bamg_status scan_counts(const int32_t* counts, int32_t* out, int n, cudaStream_t s,
                        int64_t* total_host);

// Deterministic reduction of per-block partial sums: partial[nb][K] -> out[K].
bamg_status reduce_partials(const double* partial, int nb, int K, double* out,
                            cudaStream_t s);

int num_sms();

// Raises the dynamic shared-memory limit of kernel fn to the device's opt-in
// maximum (less its static shared memory) once per device: setups may run
// concurrently on several host threads, so the attribute is set under a lock
// and never changed afterwards.  *max_dyn receives the usable bytes.
bamg_status allow_max_smem(const void* fn, std::atomic<uint64_t>& done, int* max_dyn);

}  // namespace bamg
