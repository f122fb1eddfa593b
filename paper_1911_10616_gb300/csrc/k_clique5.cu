// 5-cliques per vertex (orbit 72, Thm. 5-Cycle-Clique).
#include "evoke_internal.cuh"

namespace {

// --- 5-cliques: per DAG edge (a -> b), triangles inside S = N+(a)^N+(b) ----
// Every 5-clique a<b<c<d<e (DAG order) is seen once, at its lowest edge (a,b),
// as the triangle {c,d,e} of G[S].  One warp per DAG edge: S goes to shared
// memory (ascending ids), the adjacency inside S to bitmap rows, and the
// triangles of G[S] through c are sum_{d in row(c)} popc(row(c) & row(d)) / 2.
// Edges whose S exceeds the shared-memory capacity take a slower path that
// re-derives S on the fly.
constexpr int kK5Warps = 4;

__device__ void k5_slow_edge(const Graph& g, u64* acc, u32 a, u32 b) {
  const int lane = threadIdx.x & 31;
  const u32 n = g.n;
  const u32 ab = g.dag_ptr[a], ae = g.dag_ptr[a + 1];
  const u32 bb = g.dag_ptr[b], be = g.dag_ptr[b + 1];
  u64 cab = 0;
  for (u32 i = ab + lane; i < ae; i += 32) {
    const u32 c = g.dag_col[i];
    if (!contains_u32(g.dag_col, bb, be, c)) continue;
    u64 cc = 0;
    const u32 cb = g.dag_ptr[c], ce = g.dag_ptr[c + 1];
    for (u32 p = cb; p < ce; ++p) {
      const u32 d = g.dag_col[p];
      if (!contains_u32(g.dag_col, ab, ae, d) || !contains_u32(g.dag_col, bb, be, d)) continue;
      u64 cd = 0;
      for (u32 p2 = g.dag_ptr[d]; p2 < g.dag_ptr[d + 1]; ++p2) {
        const u32 f = g.dag_col[p2];
        if (contains_u32(g.dag_col, cb, ce, f) && contains_u32(g.dag_col, ab, ae, f) &&
            contains_u32(g.dag_col, bb, be, f)) {
          ++cd;
          atomicAdd(&acc[(u64)A_K5 * n + f], 1ull);
        }
      }
      if (cd) atomicAdd(&acc[(u64)A_K5 * n + d], cd);
      cc += cd;
    }
    if (cc) atomicAdd(&acc[(u64)A_K5 * n + c], cc);
    cab += cc;
  }
  cab = warp_sum(cab);
  if (lane == 0 && cab) {
    atomicAdd(&acc[(u64)A_K5 * n + a], cab);
    atomicAdd(&acc[(u64)A_K5 * n + b], cab);
  }
}

__global__ void __launch_bounds__(kK5Warps * 32)
k5_kernel(Graph g, u64* __restrict__ acc, u32 m, u32 smax) {
  extern __shared__ u32 k5_smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const u32 words = (smax + 31) / 32;
  u32* S = k5_smem + (size_t)wid * (2 * smax + (size_t)smax * words);
  u32* tcnt = S + smax;
  u32* rows = tcnt + smax;
  const u32 n = g.n;
  const u32 gw = blockIdx.x * kK5Warps + wid;
  const u32 nw = gridDim.x * kK5Warps;
  for (u32 e = gw; e < m; e += nw) {
    const u32 sab = g.dag_slot[e];
    const u32 a = g.col[g.rev[sab]], b = g.dag_col[e];  // source, target of DAG edge e
    if (g.dag_ptr[a + 1] - g.dag_ptr[a] < 3 || g.dag_ptr[b + 1] - g.dag_ptr[b] < 3) continue;
    // S = N+(a) ^ N+(b) = the common neighbours of a and b after b in the
    // degree order (a precedes b): the triangle list of slot (a,b),
    // filtered; ascending by id like the list
    const u64 p0 = g.tl_ptr[sab], p1 = g.tl_ptr[sab + 1];
    if (p1 - p0 < 3) continue;
    u32 s = 0;
    bool over = false;
    for (u64 base = p0; base < p1; base += 32) {
      const u64 i = base + lane;
      const u32 x = i < p1 ? g.tlv[i] : 0;
      const bool hit = i < p1 && prec(g.deg, b, x);
      const u32 bal = __ballot_sync(0xffffffffu, hit);
      const u32 pos = s + __popc(bal & ((1u << lane) - 1u));
      if (hit && pos < smax) S[pos] = x;
      s += __popc(bal);
    }
    if (s < 3) continue;
    if (s > smax) over = true;
    if (over) {
      k5_slow_edge(g, acc, a, b);
      continue;
    }
    const u32 w = (s + 31) / 32;
    for (u32 i = lane; i < s * w; i += 32) rows[i] = 0;
    __syncwarp();
    // adjacency inside S (both directions)
    for (u32 ci = lane; ci < s; ci += 32) {
      const u32 c = S[ci];
      for (u32 p = g.dag_ptr[c]; p < g.dag_ptr[c + 1]; ++p) {
        const u32 d = g.dag_col[p];
        const u32 di = lower_bound_u32(S, 0, s, d);
        if (di < s && S[di] == d) {
          atomicOr(&rows[ci * w + (di >> 5)], 1u << (di & 31));
          atomicOr(&rows[di * w + (ci >> 5)], 1u << (ci & 31));
        }
      }
    }
    __syncwarp();
    // per unordered edge (c,d) of G[S], c < d: k_cd = |N_S(c) ^ N_S(d)|
    // triangles; crediting k_cd to both ends gives each vertex twice its
    // triangle count
    for (u32 ci = lane; ci < s; ci += 32) tcnt[ci] = 0;
    __syncwarp();
    for (u32 ci = lane; ci < s; ci += 32) {
      const u32* rc = rows + ci * w;
      u32 tc = 0;
      for (u32 k = (ci + 1) >> 5; k < w; ++k) {
        u32 bits = rc[k];
        if (k == (ci >> 5)) bits &= ~((2u << (ci & 31)) - 1u);  // partners d > c
        while (bits) {
          const u32 di = k * 32 + __ffs(bits) - 1;
          bits &= bits - 1;
          const u32* rd = rows + di * w;
          u32 kcd = 0;
          for (u32 q = 0; q < w; ++q) kcd += __popc(rc[q] & rd[q]);
          if (kcd) {
            tc += kcd;
            atomicAdd(&tcnt[di], kcd);
          }
        }
      }
      if (tc) atomicAdd(&tcnt[ci], tc);
    }
    __syncwarp();
    u64 tot = 0;
    for (u32 ci = lane; ci < s; ci += 32) {
      const u32 t2 = tcnt[ci];
      const u32 tc = t2 >> 1;
      if (tc) atomicAdd(&acc[(u64)A_K5 * n + S[ci]], (u64)tc);
      tot += tc;
    }
    tot = warp_sum(tot);
    if (lane == 0 && tot) {
      atomicAdd(&acc[(u64)A_K5 * n + a], tot / 3);
      atomicAdd(&acc[(u64)A_K5 * n + b], tot / 3);
    }
    __syncwarp();
  }
}

}  // namespace

K5Config k5_configure(u32 max_outdeg) {
  K5Config c{};
  if (max_outdeg < 3) return c;
  // shared memory per warp: S list + |S| x ceil(|S|/32) bitmap words
  u32 smax = (max_outdeg + 31) / 32 * 32;
  const u32 cap = 640;
  if (smax > cap) smax = cap;
  const size_t per_warp = (2 * (size_t)smax + (size_t)smax * ((smax + 31) / 32)) * sizeof(u32);
  c.smem = per_warp * kK5Warps;
  c.smax = smax;
  cudaFuncSetAttribute(k5_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k5_kernel, kK5Warps * 32, c.smem);
  c.blocks = (u32)sms * (u32)(per_sm > 0 ? per_sm : 1) * 4;
  return c;
}

void launch_k5(const Graph& g, u64* acc, const K5Config& c, cudaStream_t st) {
  const u32 m = (u32)(g.S / 2);
  if (!m || !c.blocks) return;
  k5_kernel<<<c.blocks, kK5Warps * 32, c.smem, st>>>(g, acc, m, c.smax);
}
