// Graph preparation: degrees, reverse-slot map with input validation, the
// degree-ordered DAG (Sec. 2 "Degree ordering": i precedes j iff d(i) < d(j),
// ties by id; every edge is oriented from the earlier to the later vertex),
// and the prefix sums used to lay out per-slot lists.
#include "evoke_internal.cuh"

namespace {

constexpr int kWarpsPerBlock = 8;

__global__ void degrees_kernel(const u32* __restrict__ rowptr, u32* __restrict__ deg, u32 n) {
  u32 u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < n) deg[u] = rowptr[u + 1] - rowptr[u];
}

// rev[s] = slot of (v,u) for slot s = (u,v); flags rows that are not strictly
// increasing (duplicates / unsorted), self-loops, ids out of range and
// asymmetric edges.
__global__ void rev_kernel(const u32* __restrict__ rowptr, const u32* __restrict__ col,
                           u32* __restrict__ rev, u32 n, int* status) {
  const u32 warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const u32 u = warp;
  const u32 b = rowptr[u], e = rowptr[u + 1];
  for (u32 s = b + lane; s < e; s += 32) {
    const u32 v = col[s];
    if (v >= n) {
      atomicOr(status, ST_RANGE);
      rev[s] = 0;
      continue;
    }
    if (v == u || (s > b && col[s - 1] >= v)) atomicOr(status, ST_NOT_SIMPLE);
    const u32 vb = rowptr[v], ve = rowptr[v + 1];
    const u32 p = lower_bound_u32(col, vb, ve, u);
    if (p >= ve || col[p] != u) {
      atomicOr(status, ST_NOT_SIMPLE);
      rev[s] = s;
    } else {
      rev[s] = p;
    }
  }
}

__global__ void dag_count_kernel(const u32* __restrict__ rowptr, const u32* __restrict__ col,
                                 const u32* __restrict__ deg, u32* __restrict__ cnt,
                                 unsigned char* __restrict__ sin, u32 n) {
  const u32 warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const u32 u = warp;
  u32 c = 0;
  for (u32 s = rowptr[u] + lane; s < rowptr[u + 1]; s += 32) {
    const bool out = prec(deg, u, col[s]);
    c += out ? 1u : 0u;
    if (sin) sin[s] = out ? 0 : 1;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) cnt[u] = c;
}

__global__ void dag_fill_kernel(const u32* __restrict__ rowptr, const u32* __restrict__ col,
                                const u32* __restrict__ deg, const u32* __restrict__ dag_ptr,
                                u32* __restrict__ dag_col, u32* __restrict__ dag_slot, u32 n) {
  const u32 warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const u32 u = warp;
  u32 base = dag_ptr[u];
  const u32 b = rowptr[u], e = rowptr[u + 1];
  for (u32 s0 = b; s0 < e; s0 += 32) {
    const u32 s = s0 + lane;
    const bool ok = s < e && prec(deg, u, col[s]);
    const u32 bal = __ballot_sync(0xffffffffu, ok);
    if (ok) {
      const u32 pos = base + __popc(bal & ((1u << lane) - 1u));
      dag_col[pos] = col[s];
      dag_slot[pos] = s;
    }
    base += __popc(bal);
  }
}

// ---- exclusive scan (three phases) -----------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr u64 kScanTile = (u64)kScanThreads * kScanItems;

template <typename T>
__device__ u64 block_exclusive_scan(u64 v, u64* total) {
  __shared__ u64 warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  u64 x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    u64 y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    u64 w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      u64 y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = w;
  }
  __syncthreads();
  const u64 before = wid ? warp_tot[wid - 1] : 0;
  if (total) *total = warp_tot[kScanThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

template <typename TIn>
__global__ void scan_reduce_kernel(const TIn* __restrict__ in, u64 count, u64* __restrict__ sums) {
  const u64 base = (u64)blockIdx.x * kScanTile;
  u64 s = 0;
  for (int i = 0; i < kScanItems; ++i) {
    const u64 idx = base + (u64)i * kScanThreads + threadIdx.x;
    if (idx < count) s += in[idx];
  }
  u64 tot;
  block_exclusive_scan<u64>(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void scan_sums_kernel(u64* sums, u64 nb) {
  __shared__ u64 carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (u64 base = 0; base < nb; base += kScanThreads) {
    const u64 idx = base + threadIdx.x;
    const u64 v = idx < nb ? sums[idx] : 0;
    u64 tot;
    const u64 ex = block_exclusive_scan<u64>(v, &tot);
    if (idx < nb) sums[idx] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

template <typename TIn, typename TOut>
__global__ void scan_apply_kernel(const TIn* in, u64 count, const u64* __restrict__ sums,
                                  TOut* out) {
  const u64 base = (u64)blockIdx.x * kScanTile + (u64)threadIdx.x * kScanItems;
  u64 vals[kScanItems];
  u64 local = 0;
  for (int i = 0; i < kScanItems; ++i) {
    const u64 idx = base + i;
    vals[i] = idx < count ? (u64)in[idx] : 0;
    local += vals[i];
  }
  __syncthreads();  // `in` may alias `out`: all loads before any store
  u64 run = block_exclusive_scan<u64>(local, nullptr) + sums[blockIdx.x];
  for (int i = 0; i < kScanItems; ++i) {
    const u64 idx = base + i;
    if (idx < count) out[idx] = (TOut)run;
    run += vals[i];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[count] = (TOut)sums[gridDim.x];
}

// ---- batches: concatenated per-graph CSRs -> one CSR of their disjoint union --
__device__ __forceinline__ u32 graph_of(const long long* off, u32 G, u64 x) {
  // largest g < G with off[g] <= x
  u32 lo = 0, hi = G;
  while (hi - lo > 1) {
    u32 mid = lo + ((hi - lo) >> 1);
    if ((u64)off[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void union_rows_kernel(const u32* __restrict__ rowptr_cat, const long long* vtx_off,
                                  const long long* edge_off, u32 G, u32 n, u32* __restrict__ rowptr,
                                  u32* __restrict__ comp_base) {
  const u32 v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v > n) return;
  if (v == n) {
    rowptr[n] = (u32)edge_off[G];
    return;
  }
  const u32 g = graph_of(vtx_off, G, v);
  const u32 local = v - (u32)vtx_off[g];
  // graph g's rowptr occupies entries vtx_off[g] + g .. vtx_off[g+1] + g
  rowptr[v] = (u32)edge_off[g] + rowptr_cat[vtx_off[g] + g + local];
  comp_base[v] = (u32)vtx_off[g];
}

__global__ void union_cols_kernel(const u32* __restrict__ col_cat, const long long* vtx_off,
                                  const long long* edge_off, u32 G, u64 S, u32* __restrict__ col) {
  const u64 s = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const u32 g = graph_of(edge_off, G, s);
  col[s] = col_cat[s] + (u32)vtx_off[g];
}

__global__ void max_component_kernel(const long long* vtx_off, u32 G, u32* out) {
  const u32 g = blockIdx.x * blockDim.x + threadIdx.x;
  u32 v = g < G ? (u32)(vtx_off[g + 1] - vtx_off[g]) : 0;
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v) atomicMax(out, v);
}

}  // namespace

void launch_union_csr(const u32* rowptr_cat, const u32* col_cat, const long long* vtx_off,
                      const long long* edge_off, u32 G, u32 n, u64 S, u32* rowptr, u32* col,
                      u32* comp_base, cudaStream_t st) {
  union_rows_kernel<<<(n + 1 + 255) / 256, 256, 0, st>>>(rowptr_cat, vtx_off, edge_off, G, n,
                                                          rowptr, comp_base);
  if (S) union_cols_kernel<<<(unsigned)((S + 255) / 256), 256, 0, st>>>(col_cat, vtx_off, edge_off, G, S, col);
}

void launch_max_component(const long long* vtx_off, u32 G, u32* out, cudaStream_t st) {
  if (G) max_component_kernel<<<(G + 255) / 256, 256, 0, st>>>(vtx_off, G, out);
}

// the thread-major tile layout of scan_apply (thread t owns items
// [t*8, t*8+8)) differs from scan_reduce's strided layout; both only need the
// per-tile total, which is layout independent.

size_t scan_tmp_bytes(u64 count) {
  const u64 nb = (count + kScanTile - 1) / kScanTile + 1;
  return (size_t)(nb + 1) * sizeof(u64);
}

void launch_scan_u32_to_u64(const u32* in, u64* out, u64 count, void* tmp, cudaStream_t st) {
  u64* sums = static_cast<u64*>(tmp);
  const u64 nb = (count + kScanTile - 1) / kScanTile;
  if (nb == 0) {
    cudaMemsetAsync(out, 0, sizeof(u64), st);
    return;
  }
  scan_reduce_kernel<u32><<<(unsigned)nb, kScanThreads, 0, st>>>(in, count, sums);
  scan_sums_kernel<<<1, kScanThreads, 0, st>>>(sums, nb);
  scan_apply_kernel<u32, u64><<<(unsigned)nb, kScanThreads, 0, st>>>(in, count, sums, out);
}

void launch_scan_u32_inplace(u32* data, u64 count, void* tmp, cudaStream_t st) {
  u64* sums = static_cast<u64*>(tmp);
  const u64 nb = (count + kScanTile - 1) / kScanTile;
  if (nb == 0) {
    cudaMemsetAsync(data, 0, sizeof(u32), st);
    return;
  }
  scan_reduce_kernel<u32><<<(unsigned)nb, kScanThreads, 0, st>>>(data, count, sums);
  scan_sums_kernel<<<1, kScanThreads, 0, st>>>(sums, nb);
  scan_apply_kernel<u32, u32><<<(unsigned)nb, kScanThreads, 0, st>>>(data, count, sums, data);
}

void launch_degrees(const Graph& g, cudaStream_t st) {
  if (!g.n) return;
  degrees_kernel<<<(g.n + 255) / 256, 256, 0, st>>>(g.rowptr, g.deg, g.n);
}

void launch_rev_validate(const Graph& g, int* status, cudaStream_t st) {
  if (!g.n) return;
  const u64 threads = (u64)g.n * 32;
  rev_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(g.rowptr, g.col, g.rev, g.n, status);
}

void launch_dag(const Graph& g, u32* cnt, void* scan_tmp, cudaStream_t st) {
  if (!g.n) {
    cudaMemsetAsync(g.dag_ptr, 0, sizeof(u32), st);
    return;
  }
  const u64 threads = (u64)g.n * 32;
  const unsigned blocks = (unsigned)((threads + kWarpsPerBlock * 32 - 1) / (kWarpsPerBlock * 32));
  dag_count_kernel<<<blocks, kWarpsPerBlock * 32, 0, st>>>(g.rowptr, g.col, g.deg, cnt, g.sin,
                                                           g.n);
  cudaMemcpyAsync(g.dag_ptr, cnt, sizeof(u32) * g.n, cudaMemcpyDeviceToDevice, st);
  launch_scan_u32_inplace(g.dag_ptr, g.n, scan_tmp, st);
  dag_fill_kernel<<<blocks, kWarpsPerBlock * 32, 0, st>>>(g.rowptr, g.col, g.deg, g.dag_ptr,
                                                          g.dag_col, g.dag_slot, g.n);
}
