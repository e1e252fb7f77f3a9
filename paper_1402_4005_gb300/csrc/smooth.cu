// Multicolour Gauss-Seidel (Section 3 lists Gauss-Seidel among the admissible
// smoothers; the paper's experiments use weighted Jacobi).
//
// Colouring: greedy colouring of the symmetrised graph of B, vertices taken
// in decreasing SplitMix64 priority (stream 6144 + level, ties by index),
// each taking the smallest colour absent from its neighbours taken before
// it.  Computed by parallel rounds: an uncoloured vertex that beats every
// uncoloured neighbour takes the smallest colour absent from its coloured
// neighbours.  Its higher-priority neighbours are then all coloured and no
// lower-priority one is, so every vertex gets the colour of the sequential
// greedy order, bit for bit.
//
// Sweep: rows of one colour share no edge of the symmetrised graph, so one
// launch updates all of them at once, x_i <- x_i + (b_i - (B x)_i) / d_i with
// d the Jacobi divisor (b_ii where b_ii > 0); colours in increasing order,
// which is the sequential sweep over the rows sorted by (colour, index).
#include "internal.cuh"

namespace bamg {

constexpr uint64_t kColourStream = 6144;

__device__ inline bool prio_beats(uint64_t ki, int i, uint64_t kj, int j) {
  return ki > kj || (ki == kj && i < j);
}

// Smallest colour not used by the coloured neighbours of i (colours >= 64
// by a scan of the neighbours).
__device__ int smallest_free(int i, const int32_t* __restrict__ brp, const int32_t* __restrict__ bci,
                             const int32_t* __restrict__ trp, const int32_t* __restrict__ tci,
                             const int32_t* colour) {
  unsigned long long used = 0;
  const int32_t* rps[2] = {brp, trp};
  const int32_t* cis[2] = {bci, tci};
  for (int m = 0; m < 2; ++m)
    for (int p = rps[m][i]; p < rps[m][i + 1]; ++p) {
      const int j = cis[m][p];
      const int cj = j == i ? -1 : colour[j];
      if (cj >= 0 && cj < 64) used |= 1ull << cj;
    }
  if (~used != 0ull) return __ffsll((long long)~used) - 1;
  for (int c = 64;; ++c) {
    bool taken = false;
    for (int m = 0; m < 2 && !taken; ++m)
      for (int p = rps[m][i]; p < rps[m][i + 1]; ++p) {
        const int j = cis[m][p];
        if (j != i && colour[j] == c) {
          taken = true;
          break;
        }
      }
    if (!taken) return c;
  }
}

// One round.  A colour read while its vertex is being coloured in this round
// is seen either as -1 (the reader waits a round) or as its final value.
__global__ void colour_round_kernel(int n, const int32_t* __restrict__ brp, const int32_t* __restrict__ bci,
                                    const int32_t* __restrict__ trp, const int32_t* __restrict__ tci,
                                    uint64_t seed, int level, int32_t* colour, int* __restrict__ left) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || colour[i] >= 0) return;
  const uint64_t ki = splitmix_draw(seed, kColourStream + level, i);
  const int32_t* rps[2] = {brp, trp};
  const int32_t* cis[2] = {bci, tci};
  for (int m = 0; m < 2; ++m)
    for (int p = rps[m][i]; p < rps[m][i + 1]; ++p) {
      const int j = cis[m][p];
      if (j == i) continue;
      if (colour[j] < 0 && prio_beats(splitmix_draw(seed, kColourStream + level, j), j, ki, i)) {
        atomicAdd(left, 1);
        return;
      }
    }
  colour[i] = smallest_free(i, brp, bci, trp, tci, colour);
}

__global__ void colour_count_kernel(int n, const int32_t* __restrict__ colour, int* __restrict__ maxc) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicMax(maxc, colour[i]);
}

bamg_status colour_graph(int n, const int32_t* brp, const int32_t* bci, const int32_t* trp, const int32_t* tci,
                         uint64_t seed, int level, int32_t* colour, int* ncolours, cudaStream_t s) {
  DevMem left;
  BAMG_TRY(left.alloc(2 * sizeof(int), s));
  BAMG_CUDA(cudaMemsetAsync(colour, 0xFF, sizeof(int32_t) * (size_t)n, s));   // -1
  for (int round = 0;; ++round) {
    if (round > n + 1) {
      set_error("colouring rounds did not terminate");
      return BAMG_ERR_NUMERIC;
    }
    BAMG_CUDA(cudaMemsetAsync(left.p, 0, sizeof(int), s));
    BAMG_TRY(launch(colour_round_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n, brp, bci, trp, tci, seed, level,
                    colour, left.as<int>()));
    int h = 0;
    BAMG_CUDA(cudaMemcpyAsync(&h, left.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    BAMG_CUDA(cudaStreamSynchronize(s));
    if (h == 0) break;
  }
  BAMG_CUDA(cudaMemsetAsync(left.as<int>() + 1, 0xFF, sizeof(int), s));
  BAMG_TRY(launch(colour_count_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n, (const int32_t*)colour,
                  left.as<int>() + 1));
  int mc = -1;
  BAMG_CUDA(cudaMemcpyAsync(&mc, left.as<int>() + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  BAMG_CUDA(cudaStreamSynchronize(s));
  *ncolours = mc + 1;
  return BAMG_OK;
}

// ------------------------------------------------------- rows by colour
__global__ void colour_flag_kernel(int n, const int32_t* __restrict__ colour, int c, int32_t* __restrict__ flag) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = colour[i] == c ? 1 : 0;
}

__global__ void colour_scatter_kernel(int n, const int32_t* __restrict__ colour, int c, int base,
                                      const int32_t* __restrict__ pos, int32_t* __restrict__ rows) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && colour[i] == c) rows[base + pos[i]] = i;
}

// rows[colour_rp[c] .. colour_rp[c + 1]) = rows of colour c, ascending;
// colour_rp is returned on the host (ncolours + 1 entries).
bamg_status colour_rows(int n, const int32_t* colour, int ncolours, int32_t* colour_rp_host, int32_t* rows,
                        cudaStream_t s) {
  DevMem flag, pos;
  BAMG_TRY(flag.alloc(sizeof(int32_t) * (n + 1), s));
  BAMG_TRY(pos.alloc(sizeof(int32_t) * (n + 1), s));
  colour_rp_host[0] = 0;
  for (int c = 0; c < ncolours; ++c) {
    BAMG_TRY(launch(colour_flag_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n, colour, c, flag.as<int32_t>()));
    int64_t cnt = 0;
    BAMG_TRY(scan_counts(flag.as<int32_t>(), pos.as<int32_t>(), n, s, &cnt));
    BAMG_TRY(launch(colour_scatter_kernel, dim3(cdiv(n, 256)), dim3(256), 0, s, n, colour, c, colour_rp_host[c],
                    (const int32_t*)pos.as<int32_t>(), rows));
    colour_rp_host[c + 1] = colour_rp_host[c] + (int32_t)cnt;
  }
  return BAMG_OK;
}

// ----------------------------------------------------------------- sweep
// The rows of one colour, a group of G lanes per row.
template <typename T, int G>
__global__ void __launch_bounds__(256)
mcgs_kernel(int cnt, const int32_t* __restrict__ rows, const int32_t* __restrict__ rp,
            const int32_t* __restrict__ ci, const T* __restrict__ va, const T* __restrict__ dinv,
            const T* __restrict__ b, T* x) {
  pdl_wait();
  pdl_trigger();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = t / G, g = threadIdx.x % G;
  const bool valid = k < cnt;      // every lane joins the shuffles below
  const int i = valid ? __ldg(rows + k) : 0;
  T acc = T(0);
  if (valid) {
    const int p1 = __ldg(rp + i + 1);
    for (int p = __ldg(rp + i) + g; p < p1; p += G) acc = fma(__ldg(va + p), x[__ldg(ci + p)], acc);
  }
  acc = group_sum<G>(acc);
  if (valid && g == 0) x[i] = x[i] + (b[i] - acc) * dinv[i];
}

template <typename T, int G>
static bamg_status mcgs_g(int ncolours, const int32_t* crp, const int32_t* rows, const int32_t* rp,
                          const int32_t* ci, const T* va, const T* dinv, const T* b, T* x, cudaStream_t s) {
  for (int c = 0; c < ncolours; ++c) {
    const int cnt = crp[c + 1] - crp[c];
    BAMG_TRY(launch(mcgs_kernel<T, G>, dim3(cdiv((long long)cnt * G, 256)), dim3(256), 0, s, cnt, rows + crp[c],
                    rp, ci, va, dinv, b, x));
  }
  return BAMG_OK;
}

// One forward multicolour sweep in place on x; crp on the host.
template <typename T>
bamg_status mcgs_sweep(int G, int ncolours, const int32_t* crp, const int32_t* rows, const int32_t* rp,
                       const int32_t* ci, const T* va, const T* dinv, const T* b, T* x, cudaStream_t s) {
  switch (G) {
    case 2: return mcgs_g<T, 2>(ncolours, crp, rows, rp, ci, va, dinv, b, x, s);
    case 4: return mcgs_g<T, 4>(ncolours, crp, rows, rp, ci, va, dinv, b, x, s);
    case 8: return mcgs_g<T, 8>(ncolours, crp, rows, rp, ci, va, dinv, b, x, s);
    case 16: return mcgs_g<T, 16>(ncolours, crp, rows, rp, ci, va, dinv, b, x, s);
    default: return mcgs_g<T, 32>(ncolours, crp, rows, rp, ci, va, dinv, b, x, s);
  }
}

template bamg_status mcgs_sweep<float>(int, int, const int32_t*, const int32_t*, const int32_t*, const int32_t*,
                                       const float*, const float*, const float*, float*, cudaStream_t);
template bamg_status mcgs_sweep<double>(int, int, const int32_t*, const int32_t*, const int32_t*, const int32_t*,
                                        const double*, const double*, const double*, double*, cudaStream_t);

}  // namespace bamg
