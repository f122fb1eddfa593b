// evoke_build_dag_noalloc: the degree-ordered DAG (the same output as
// evoke_build_dag) computed without allocating any device memory.
//
// Who needs this: callers that cannot call cudaMalloc / cudaMallocAsync.
// Typical cases are programs whose device memory is owned up front by their
// own pool or arena (a library allocation then fails, or fragments that
// pool), and code on latency-critical paths that cannot pay for an
// allocation, which may synchronise the device.  Such callers pass every
// input and output buffer themselves; the only scratch this function needs
// (the per-tile partial sums of one prefix sum) lives in the file-scope
// device array below, which every GPU that loads the library holds until the
// process exits.
//
// Limits and sharing:
//  - n <= kNaMaxVertices (8,388,608); larger graphs get EVOKE_ERANGE.
//  - The scratch array is shared by every call on a device and keeps the
//    last call's contents.  Every element a call reads was written earlier by
//    the same call, so nothing has to start at zero.  Calls that overlap on
//    the GPU (concurrent streams, or several host threads) race on the array
//    and must be serialised by the caller.
//  - The first call on a device looks up the array's device address
//    (cudaGetSymbolAddress, once per device, with that device current).  Make
//    that first call before any stream capture on the device.
#include <mutex>

#include "evoke_internal.cuh"
#include "../../include/evoke.h"

namespace {

constexpr u32 kNaThreads = 256;
constexpr u32 kNaItems = 8;
constexpr u32 kNaTile = kNaThreads * kNaItems;  // 2048 vertices per scan tile
constexpr u32 kNaMaxTiles = 4096;
constexpr u32 kNaMaxVertices = kNaMaxTiles * kNaTile;  // 8,388,608

// per-tile sums of the out-degree scan, then their total (entry kNaMaxTiles)
static __device__ __align__(256) u64 g_noalloc_scratch[kNaMaxTiles + 2];

std::mutex g_na_mu;
u64* g_na_addr[64] = {};  // device address of g_noalloc_scratch per device

// degree order of Sec. 2, with degrees read from rowptr
__device__ __forceinline__ bool na_prec(const u32* rowptr, u32 i, u32 j) {
  const u32 di = rowptr[i + 1] - rowptr[i], dj = rowptr[j + 1] - rowptr[j];
  return di < dj || (di == dj && i < j);
}

// out-degree of every vertex, written into dag_rowptr[0..n)
__global__ void na_count_kernel(const u32* __restrict__ rowptr, const u32* __restrict__ col,
                                u32* __restrict__ cnt, u32 n) {
  const u32 u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (u >= n) return;
  u32 c = 0;
  for (u32 s = rowptr[u] + lane; s < rowptr[u + 1]; s += 32) c += na_prec(rowptr, u, col[s]) ? 1u : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) cnt[u] = c;
}

__device__ u32 na_block_exclusive(u32 v, u32* total) {
  __shared__ u32 wt[kNaThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  u32 x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wt[wid] = x;
  __syncthreads();
  if (wid == 0) {
    u32 t = lane < (int)(kNaThreads / 32) ? wt[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < (int)(kNaThreads / 32)) wt[lane] = t;
  }
  __syncthreads();
  const u32 before = wid ? wt[wid - 1] : 0;
  if (total) *total = wt[kNaThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

// scan phase 1: tile sums into the scratch array
__global__ void na_tile_sum_kernel(const u32* __restrict__ cnt, u32 n, u64* __restrict__ sums) {
  const u32 base = blockIdx.x * kNaTile + threadIdx.x * kNaItems;
  u32 s = 0;
  for (u32 i = 0; i < kNaItems; ++i)
    if (base + i < n) s += cnt[base + i];
  u32 tot;
  na_block_exclusive(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// scan phase 2: exclusive prefix of the tile sums; the total goes to sums[nb]
__global__ void na_tile_prefix_kernel(u64* sums, u32 nb) {
  __shared__ u64 carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (u32 b0 = 0; b0 < nb; b0 += kNaThreads) {
    const u32 i = b0 + threadIdx.x;
    const u32 v = i < nb ? (u32)sums[i] : 0;
    u32 tot;
    const u32 ex = na_block_exclusive(v, &tot);
    if (i < nb) sums[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

// scan phase 3: in-place exclusive prefix of the out-degrees -> dag_rowptr
__global__ void na_apply_kernel(u32* data, u32 n, const u64* __restrict__ sums, u32 nb) {
  const u32 base = blockIdx.x * kNaTile + threadIdx.x * kNaItems;
  u32 vals[kNaItems];
  u32 local = 0;
  for (u32 i = 0; i < kNaItems; ++i) {
    vals[i] = base + i < n ? data[base + i] : 0;
    local += vals[i];
  }
  __syncthreads();
  u32 run = na_block_exclusive(local, nullptr) + (u32)sums[blockIdx.x];
  for (u32 i = 0; i < kNaItems; ++i) {
    if (base + i < n) data[base + i] = run;
    run += vals[i];
  }
  if (blockIdx.x == nb - 1 && threadIdx.x == 0) data[n] = (u32)sums[nb];
}

// out-neighbours in ascending id order; writes beyond m entries are dropped
__global__ void na_fill_kernel(const u32* __restrict__ rowptr, const u32* __restrict__ col,
                               const u32* __restrict__ dag_ptr, u32* __restrict__ dag_col, u32 n,
                               u64 m) {
  const u32 u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (u >= n) return;
  u32 base = dag_ptr[u];
  const u32 b = rowptr[u], e = rowptr[u + 1];
  for (u32 s0 = b; s0 < e; s0 += 32) {
    const u32 s = s0 + lane;
    const bool ok = s < e && na_prec(rowptr, u, col[s]);
    const u32 bal = __ballot_sync(0xffffffffu, ok);
    if (ok) {
      const u32 pos = base + __popc(bal & ((1u << lane) - 1u));
      if (pos < m) dag_col[pos] = col[s];
    }
    base += __popc(bal);
  }
}

// device address of the scratch array for the current device (set up once)
int scratch_address(u64** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return EVOKE_ECUDA;
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return EVOKE_ECUDA;
    g_na_addr[dev] = static_cast<u64*>(p);
  }
  *out = g_na_addr[dev];
  return EVOKE_OK;
}

}  // namespace

extern "C" int evoke_build_dag_noalloc(const uint32_t* rowptr, const uint32_t* colidx,
                                       uint32_t n, uint64_t m, uint32_t* dag_rowptr,
                                       uint32_t* dag_colidx, void* stream) {
  if (!rowptr || !dag_rowptr || (m && (!colidx || !dag_colidx))) return EVOKE_EINVAL;
  if (n > kNaMaxVertices || 2 * m >= 0xffffffffull) return EVOKE_ERANGE;
  u64* sums = nullptr;
  int rc = scratch_address(&sums);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n == 0) {
    if (cudaMemsetAsync(dag_rowptr, 0, sizeof(u32), st) != cudaSuccess) return EVOKE_ECUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? EVOKE_OK : EVOKE_ECUDA;
  }
  const u32 nb = (n + kNaTile - 1) / kNaTile;
  const unsigned wblocks = (unsigned)(((u64)n * 32 + 255) / 256);
  na_count_kernel<<<wblocks, 256, 0, st>>>(rowptr, colidx, dag_rowptr, n);
  na_tile_sum_kernel<<<nb, kNaThreads, 0, st>>>(dag_rowptr, n, sums);
  na_tile_prefix_kernel<<<1, kNaThreads, 0, st>>>(sums, nb);
  na_apply_kernel<<<nb, kNaThreads, 0, st>>>(dag_rowptr, n, sums, nb);
  na_fill_kernel<<<wblocks, 256, 0, st>>>(rowptr, colidx, dag_rowptr, dag_colidx, n, m);
  if (cudaGetLastError() != cudaSuccess) return EVOKE_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? EVOKE_OK : EVOKE_ECUDA;
}
