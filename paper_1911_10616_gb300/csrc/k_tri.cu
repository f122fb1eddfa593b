// Triangle layer (Thm. 4orbit): per-edge triangle counts T(e) and sorted
// per-edge triangle lists, the triangle-based edge orbits E7 and E9 of
// Lem. 4edgeorbit, per-vertex sums over the edge opposite a vertex in its
// triangles, and the per-triangle 4-clique counts K4(t) that feed E11 = K4(e),
// and orbits 66, 70 and 71 of Thm. 5vertexorbit.
//
// Triangle lists: for the slot s of edge (u,v) in row u, tl[tl_ptr[s] ..
// tl_ptr[s+1]) holds, in ascending order of x, the slot of (u,x) in row u for
// every common neighbour x.  The list of the reverse slot holds the slots of
// (v,x) in row v in the same order, so index k of both lists names the same
// triangle {u,v,x}.
#include "evoke_internal.cuh"

namespace {

__device__ __forceinline__ u32 row_of(const u32* rowptr, u32 n, u32 s) {
  // largest u with rowptr[u] <= s
  u32 lo = 0, hi = n;
  while (hi - lo > 1) {
    u32 mid = lo + ((hi - lo) >> 1);
    if (rowptr[mid] <= s) lo = mid;
    else hi = mid;
  }
  return lo;
}

// one thread per DAG edge (u -> v): u precedes v, so d(u) <= d(v); walk N(u)
// and binary-search each entry in N(v).
template <bool kFill>
__global__ void tri_kernel(Graph g, u32* __restrict__ T, u32 m) {
  const u32 e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  const u32 s = g.dag_slot[e];
  const u32 u = g.col[g.rev[s]];  // the row owning slot s
  const u32 v = g.col[s];
  const u32 ub = g.rowptr[u], ue = g.rowptr[u + 1];
  const u32 vb = g.rowptr[v], ve = g.rowptr[v + 1];
  const u32 r = g.rev[s];
  u32 cnt = 0;
  u64 o1 = 0, o2 = 0;
  if (kFill) {
    o1 = g.tl_ptr[s];
    o2 = g.tl_ptr[r];
  }
  u32 lo = vb;
  for (u32 i = ub; i < ue; ++i) {
    const u32 x = g.col[i];
    lo = lower_bound_u32(g.col, lo, ve, x);
    if (lo >= ve) break;
    if (g.col[lo] == x) {
      if (kFill) {
        g.tl[o1 + cnt] = i;
        g.tl[o2 + cnt] = lo;
        g.tlv[o1 + cnt] = x;
        g.tlv[o2 + cnt] = x;
      }
      ++cnt;
    }
  }
  if (!kFill) {
    T[s] = cnt;
    T[r] = cnt;
  }
}

// per slot (u,v): E7(u,v) = sum_{x in T(u,v)} (d(x)-2);  E9<u,v> = sum (T(u,x)-1);
// and, in DAG order, the triangles whose third vertex x lies between u and v
// (Mmid) or after both (Mtop).
__global__ void tri_edge_kernel(Graph g, SlotArrays sa) {
  const u64 s = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.S) return;
  const u32 u = g.col[g.rev[s]];  // the row owning slot s
  const u32 v = g.col[s];
  u64 e7 = 0, e9 = 0;
  u32 mid = 0, top = 0;
  for (u64 k = g.tl_ptr[s]; k < g.tl_ptr[s + 1]; ++k) {
    const u32 sx = g.tl[k];
    const u32 x = g.col[sx];
    e7 += (u64)((long long)g.deg[x] - 2);
    e9 += (u64)((long long)sa.T[sx] - 1);
    if (prec(g.deg, u, x)) {
      if (prec(g.deg, x, v)) ++mid;
      else ++top;
    }
  }
  sa.E7[s] = e7;
  sa.E9[s] = e9;
  sa.Mmid[s] = mid;
  sa.Mtop[s] = top;
}

// per vertex u: sums over the edges (v,x) opposite u in its triangles, each
// triangle visited twice (through v and through x).
template <int kPass>
__global__ void tri_opp_kernel(Graph g, SlotArrays sa, u64* __restrict__ acc) {
  const u32 u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (u >= g.n) return;
  const u32 n = g.n;
  u64 a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  for (u32 s = g.rowptr[u]; s < g.rowptr[u + 1]; ++s) {
    if (sa.T[s] == 0) continue;
    const u32 r = g.rev[s];
    for (u64 k = g.tl_ptr[r] + lane; k < g.tl_ptr[r + 1]; k += 32) {
      const u32 e = g.tl[k];  // slot (v,x) in row v
      if (kPass == 1) {
        const long long t = sa.T[e];
        a0 += (u64)(t - 1);
        a1 += c2(t - 1);
      } else {
        a0 += sa.E7[e];
        a1 += sa.E5[e];
        a2 += sa.E9[e] + sa.E9[g.rev[e]];
        a3 += sa.K4[e];
      }
    }
  }
  a0 = warp_sum(a0);
  a1 = warp_sum(a1);
  if (kPass == 2) {
    a2 = warp_sum(a2);
    a3 = warp_sum(a3);
  }
  if (lane == 0) {
    if (kPass == 1) {
      acc[(u64)A_S12 * n + u] = a0;
      acc[(u64)A_S54 * n + u] = a1;
    } else {
      acc[(u64)A_S46 * n + u] = a0;
      acc[(u64)A_S52 * n + u] = a1;
      acc[(u64)A_S59 * n + u] = a2;
      acc[(u64)A_S65 * n + u] = a3;
    }
  }
}

// One warp per DAG edge a -> b (slot s of b in row a); lanes take the
// triangle-list entries c of (a,b) with b preceding c, so every triangle
// a < b < c (degree order) is seen once.  K4(t) = |N(a)^N(b)^N(c)| =
// |tl(a,b) ^ tl(a,c)| (both ascending slot lists of row a).  Every apex of
// these triangles lies in tl(a,b): the warp sums the apex credits per list
// position in shared memory and adds them once per apex; the credits of a,
// b and of the edge (a,b) are summed over the warp.
constexpr int kK4Warps = 8;
constexpr u32 kK4Pos = 1024;

__global__ void __launch_bounds__(kK4Warps * 32)
k4_kernel(Graph g, SlotArrays sa, u64* __restrict__ acc, u32 m) {
  __shared__ u32 s70[kK4Warps][kK4Pos];
  __shared__ u32 s66[kK4Warps][kK4Pos];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const u32 e = blockIdx.x * kK4Warps + wid;
  if (e >= m) return;
  const u32 s = g.dag_slot[e];
  const u64 p0 = g.tl_ptr[s], p1 = g.tl_ptr[s + 1];
  if (p1 - p0 < 1) return;
  const u32 b = g.col[s];
  const u32 r = g.rev[s];
  const u32 a = g.col[r];
  const u32 n = g.n;
  const u64 r0 = g.tl_ptr[r];
  const bool local = p1 - p0 <= kK4Pos;
  if (local) {
    for (u32 i = lane; i < p1 - p0; i += 32) s70[wid][i] = s66[wid][i] = 0;
    __syncwarp();
  }
  u64 k4ab = 0, k2ab = 0;
  for (u64 q = p0 + lane; q < p1; q += 32) {
    const u32 c = g.tlv[q];
    if (!prec(g.deg, b, c)) continue;
    const u32 sac = g.tl[q];
    const u32 sbc = g.tl[r0 + (q - p0)];
    const u64 q0 = g.tl_ptr[sac], q1 = g.tl_ptr[sac + 1];
    u64 i = p0, j = q0;
    u32 k4 = 0;
    while (i < p1 && j < q1) {
      const u32 x = g.tl[i], y = g.tl[j];
      if (x < y) ++i;
      else if (y < x) ++j;
      else { ++k4; ++i; ++j; }
    }
    if (!k4) continue;
    k4ab += k4;
    atomicAdd(&sa.K4[sac], (u64)k4);
    atomicAdd(&sa.K4[g.rev[sac]], (u64)k4);
    atomicAdd(&sa.K4[sbc], (u64)k4);
    atomicAdd(&sa.K4[g.rev[sbc]], (u64)k4);
    const u64 k2 = c2(k4);
    if (k2) {
      k2ab += k2;
      atomicAdd(&acc[(u64)A_S71 * n + c], k2);
    }
    const u32 tsum = sa.T[s] + sa.T[sac] + sa.T[sbc];
    i = p0;
    j = q0;
    while (i < p1 && j < q1) {
      const u32 x = g.tl[i], y = g.tl[j];
      if (x < y) ++i;
      else if (y < x) ++j;
      else {
        if (local) {
          if (k4 > 1) atomicAdd(&s70[wid][i - p0], k4 - 1);
          atomicAdd(&s66[wid][i - p0], tsum);
        } else {
          const u32 apex = g.tlv[i];
          if (k4 > 1) atomicAdd(&acc[(u64)A_S70 * n + apex], (u64)(k4 - 1));
          atomicAdd(&acc[(u64)A_S66 * n + apex], (u64)tsum);
        }
        ++i;
        ++j;
      }
    }
  }
  k4ab = warp_sum(k4ab);
  k2ab = warp_sum(k2ab);
  if (lane == 0) {
    if (k4ab) {
      atomicAdd(&sa.K4[s], k4ab);
      atomicAdd(&sa.K4[r], k4ab);
    }
    if (k2ab) {
      atomicAdd(&acc[(u64)A_S71 * n + a], k2ab);
      atomicAdd(&acc[(u64)A_S71 * n + b], k2ab);
    }
  }
  if (local) {
    __syncwarp();
    for (u32 i = lane; i < p1 - p0; i += 32) {
      const u32 v70 = s70[wid][i], v66 = s66[wid][i];
      if (v70 | v66) {
        const u32 apex = g.tlv[p0 + i];
        if (v70) atomicAdd(&acc[(u64)A_S70 * n + apex], (u64)v70);
        if (v66) atomicAdd(&acc[(u64)A_S66 * n + apex], (u64)v66);
      }
    }
  }
}

// every 4-clique on an edge lies in two of the edge's triangles
__global__ void halve_kernel(u64* __restrict__ x, u64 count) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) x[i] >>= 1;
}

inline unsigned blocks_for(u64 threads, unsigned bs) { return (unsigned)((threads + bs - 1) / bs); }

}  // namespace

void launch_tri_count(const Graph& g, u32* T, cudaStream_t st) {
  const u32 m = (u32)(g.S / 2);
  if (!m) return;
  tri_kernel<false><<<blocks_for(m, 256), 256, 0, st>>>(g, T, m);
}

void launch_tri_fill(const Graph& g, const u32* T, cudaStream_t st) {
  const u32 m = (u32)(g.S / 2);
  if (!m) return;
  tri_kernel<true><<<blocks_for(m, 256), 256, 0, st>>>(g, const_cast<u32*>(T), m);
}

void launch_tri_edge(const Graph& g, const SlotArrays& sa, cudaStream_t st) {
  if (!g.S) return;
  tri_edge_kernel<<<blocks_for(g.S, 256), 256, 0, st>>>(g, sa);
}

void launch_tri_opp1(const Graph& g, const SlotArrays& sa, u64* acc, cudaStream_t st) {
  if (!g.n) return;
  tri_opp_kernel<1><<<blocks_for((u64)g.n * 32, 256), 256, 0, st>>>(g, sa, acc);
}

void launch_tri_opp2(const Graph& g, const SlotArrays& sa, u64* acc, cudaStream_t st) {
  if (!g.n) return;
  tri_opp_kernel<2><<<blocks_for((u64)g.n * 32, 256), 256, 0, st>>>(g, sa, acc);
}

void launch_k4_known(const Graph& g, const SlotArrays& sa, u64* acc, u64 total, cudaStream_t st) {
  if (!g.S) return;
  const u32 m = (u32)(g.S / 2);
  if (total) k4_kernel<<<(m + kK4Warps - 1) / kK4Warps, kK4Warps * 32, 0, st>>>(g, sa, acc, m);
  halve_kernel<<<blocks_for(g.S, 256), 256, 0, st>>>(sa.K4, g.S);
}


