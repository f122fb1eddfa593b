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

// ---- relabelling by decreasing degree ---------------------------------------
// Vertices are renumbered so that ids ascend as degrees descend; hubs, whose
// 2-hop-map entries every root touches most, then share a small id range.
__global__ void deg_hist_kernel(const u32* __restrict__ rowptr, u32 n, u32* hist) {
  const u32 u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < n) atomicAdd(&hist[rowptr[u + 1] - rowptr[u]], 1u);
}
// exclusive prefix over degrees from the largest down (one block)
__global__ void deg_scan_desc_kernel(u32* hist, u32 dmax) {
  __shared__ u32 carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (u32 b0 = 0; b0 <= dmax; b0 += blockDim.x) {
    const u32 i = b0 + threadIdx.x;  // i-th largest degree
    const u32 dgr = i <= dmax ? dmax - i : 0;
    const u32 v = i <= dmax ? hist[dgr] : 0;
    // block inclusive scan
    __shared__ u32 tmp[1024];
    tmp[threadIdx.x] = v;
    __syncthreads();
    for (u32 o = 1; o < blockDim.x; o <<= 1) {
      const u32 y = threadIdx.x >= o ? tmp[threadIdx.x - o] : 0;
      __syncthreads();
      tmp[threadIdx.x] += y;
      __syncthreads();
    }
    if (i <= dmax) hist[dgr] = carry + tmp[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += tmp[threadIdx.x];
    __syncthreads();
  }
}
__global__ void relabel_scatter_kernel(const u32* __restrict__ rowptr, u32 n, u32* cursor,
                                       u32* __restrict__ new_id, u32* __restrict__ old_of,
                                       u32* __restrict__ new_deg) {
  const u32 u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  const u32 d = rowptr[u + 1] - rowptr[u];
  const u32 k = atomicAdd(&cursor[d], 1u);
  new_id[u] = k;
  old_of[k] = u;
  new_deg[k] = d;
}
// rows of the relabelled graph, unsorted: warp per new row
__global__ void relabel_fill_kernel(const u32* __restrict__ rowptr, const u32* __restrict__ col,
                                    const u32* __restrict__ new_id, const u32* __restrict__ old_of,
                                    const u32* __restrict__ nrow, u32* __restrict__ ncol, u32 n) {
  const u32 w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const u32 u = old_of[w];
  const u32 b = rowptr[u], d = rowptr[u + 1] - b, o = nrow[w];
  for (u32 k = lane; k < d; k += 32) ncol[o + k] = new_id[col[b + k]];
}
// bitonic sort of one row in shared memory (ascending, padded with ~0)
template <bool kBlock>
__device__ void bitonic_sort(u32* a, u32 len, u32 tid, u32 nthreads) {
  for (u32 k = 2; k <= len; k <<= 1)
    for (u32 j = k >> 1; j > 0; j >>= 1) {
      for (u32 i = tid; i < len; i += nthreads) {
        const u32 ixj = i ^ j;
        if (ixj > i) {
          const u32 x = a[i], y = a[ixj];
          const bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[ixj] = x;
          }
        }
      }
      if (kBlock) __syncthreads();
      else __syncwarp();
    }
}
constexpr u32 kWarpSortMax = 1024;
__global__ void row_sort_warp_kernel(const u32* __restrict__ nrow, u32* ncol, u32 first, u32 n) {
  __shared__ u32 buf[8][kWarpSortMax];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const u32 r = first + blockIdx.x * 8 + wid;
  if (r >= n) return;
  const u32 b = nrow[r], d = nrow[r + 1] - b;
  if (d < 2) return;
  u32 len = 1;
  while (len < d) len <<= 1;
  for (u32 k = lane; k < len; k += 32) buf[wid][k] = k < d ? ncol[b + k] : 0xffffffffu;
  __syncwarp();
  bitonic_sort<false>(buf[wid], len, lane, 32);
  for (u32 k = lane; k < d; k += 32) ncol[b + k] = buf[wid][k];
}
__global__ void row_sort_block_kernel(const u32* __restrict__ nrow, u32* ncol) {
  extern __shared__ u32 big[];
  const u32 r = blockIdx.x;
  const u32 b = nrow[r], d = nrow[r + 1] - b;
  u32 len = 1;
  while (len < d) len <<= 1;
  for (u32 k = threadIdx.x; k < len; k += blockDim.x) big[k] = k < d ? ncol[b + k] : 0xffffffffu;
  __syncthreads();
  bitonic_sort<true>(big, len, threadIdx.x, blockDim.x);
  for (u32 k = threadIdx.x; k < d; k += blockDim.x) ncol[b + k] = big[k];
}
// original slot of every relabelled slot (for per-edge outputs)
__global__ void orig_slot_kernel(const u32* __restrict__ rowptr, const u32* __restrict__ col,
                                 const u32* __restrict__ old_of, const u32* __restrict__ nrow,
                                 const u32* __restrict__ ncol, u32 n, u32* __restrict__ orig) {
  const u32 w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const u32 u = old_of[w];
  const u32 b = rowptr[u], e = rowptr[u + 1];
  for (u32 s = nrow[w] + lane; s < nrow[w + 1]; s += 32) {
    const u32 v = old_of[ncol[s]];
    orig[s] = lower_bound_u32(col, b, e, v);
  }
}

}  // namespace

u32 relabel_prepare(const u32* rowptr, u32 n, u32 dmax, u32* hist, u32* new_id, u32* old_of,
                    u32* new_deg, cudaStream_t st) {
  // returns nothing on the host side; the number of long rows is derived later
  cudaMemsetAsync(hist, 0, sizeof(u32) * (dmax + 1), st);
  deg_hist_kernel<<<(n + 255) / 256, 256, 0, st>>>(rowptr, n, hist);
  deg_scan_desc_kernel<<<1, 1024, 0, st>>>(hist, dmax);
  relabel_scatter_kernel<<<(n + 255) / 256, 256, 0, st>>>(rowptr, n, hist, new_id, old_of, new_deg);
  return 0;
}

void relabel_build(const u32* rowptr, const u32* col, const u32* new_id, const u32* old_of,
                   const u32* nrow, u32* ncol, u32 n, u32 long_rows, u32 dmax, cudaStream_t st) {
  if (!n) return;
  relabel_fill_kernel<<<(unsigned)(((u64)n * 32 + 255) / 256), 256, 0, st>>>(rowptr, col, new_id,
                                                                             old_of, nrow, ncol, n);
  if (long_rows) {
    u32 len = 1;
    while (len < dmax) len <<= 1;
    row_sort_block_kernel<<<long_rows, 1024, len * sizeof(u32), st>>>(nrow, ncol);
  }
  if (n > long_rows)
    row_sort_warp_kernel<<<(n - long_rows + 7) / 8, 256, 0, st>>>(nrow, ncol, long_rows, n);
}

void relabel_configure(u32 dmax) {
  u32 len = 1;
  while (len < dmax) len <<= 1;
  cudaFuncSetAttribute(row_sort_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(len * sizeof(u32)));
}

void launch_orig_slot(const u32* rowptr, const u32* col, const u32* old_of, const u32* nrow,
                      const u32* ncol, u32 n, u32* orig, cudaStream_t st) {
  if (n)
    orig_slot_kernel<<<(unsigned)(((u64)n * 32 + 255) / 256), 256, 0, st>>>(rowptr, col, old_of,
                                                                           nrow, ncol, n, orig);
}

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
