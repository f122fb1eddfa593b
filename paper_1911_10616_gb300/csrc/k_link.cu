// The wheel pass (orbits 68 and 69): 4-cycles of each vertex's link graph.
#include "evoke_internal.cuh"

namespace {

// --- wheel pass: 4-cycles inside N(u) per vertex, for every slot (u,a) -------
// (orbits 68 and 69: a wheel is a hub u plus a 4-cycle of the link graph
// G[N(u)], whose edges are the triangle-list entries of u's slots).  Each
// 4-cycle of G[N(u)] is found once, from its top vertex a, the smallest id
// (the highest degree after the relabelling): the wedges a - b - c with b > a
// and c > a give W'(a,c) = |{b > a : b ~ a, b ~ c}|, and C(W'(a,c), 2) cycles
// have top a and opposite vertex c.  They are credited to a and to c, and the
// middle b of each wedge a - b - c gets W'(a,c) - 1 (one per other middle), so
// every slot (u,x) ends with the number of 4-cycles of G[N(u)] through x.
// Ordering the tops by degree is what keeps the wedge count down: a wedge
// through a hub b is walked only from the few tops of still higher degree.
// One warp per slot (u,a): it walks the b > a entries of tl(u,a) 32 at a time
// and, for each, the tail c > a of tl(u,b) (entered by binary search; slot
// order = id order).  Sweep 1 counts W' in 16-bit halves of shared-memory
// words when d(u) <= kLinkSmem (then W' < 2^16), else in 32-bit words of the
// warp's global scratch row, and lists the touched partners; sweep 2 walks
// the same wedges again to credit the middles.
constexpr int kLinkWarps = 8;
constexpr u32 kLinkSmem = 512;

constexpr size_t kLinkDynSmem = (size_t)kLinkWarps * (kLinkSmem / 2 + kLinkSmem) * sizeof(u32);

__global__ void __launch_bounds__(kLinkWarps * 32)
link_kernel(Graph g, SlotArrays sa, u32* __restrict__ scratch, u32 dmax) {
  extern __shared__ u32 link_smem[];
  u32 (*s_map)[kLinkSmem / 2] = reinterpret_cast<u32 (*)[kLinkSmem / 2]>(link_smem);
  u32 (*s_list)[kLinkSmem] =
      reinterpret_cast<u32 (*)[kLinkSmem]>(link_smem + (size_t)kLinkWarps * (kLinkSmem / 2));
  __shared__ u32 s_pref[kLinkWarps][33];
  __shared__ u64 s_start[kLinkWarps][32];
  __shared__ u32 s_sb[kLinkWarps][32];
  __shared__ u32 s_cnt[kLinkWarps];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const u32 gw = blockIdx.x * kLinkWarps + wid;
  const u32 nwarps = gridDim.x * kLinkWarps;
  u32* gmap = scratch + (u64)gw * 2 * dmax;
  u32* glist = gmap + dmax;
  for (u32 i = lane; i < kLinkSmem / 2; i += 32) s_map[wid][i] = 0;
  __syncwarp();
  for (u64 s = gw; s < g.S; s += nwarps) {
    if (sa.T[s] < 2) continue;
    const u64 q1 = g.tl_ptr[s + 1];
    u64 kb = g.tl_ptr[s];
    {  // first entry of tl(u,a) with b > a
      u64 hi = q1;
      while (kb < hi) {
        const u64 mid = kb + ((hi - kb) >> 1);
        if (g.tl[mid] <= (u32)s) kb = mid + 1;
        else hi = mid;
      }
    }
    if (q1 - kb < 2) continue;  // a cycle with top a needs two middles
    const u32 lo = g.col[g.rev[s]];  // the row owning slot s
    const u32 ub = g.rowptr[lo], du = g.rowptr[lo + 1] - ub;
    const bool small = du <= kLinkSmem;
    u32* list = small ? s_list[wid] : glist;
    if (lane == 0) s_cnt[wid] = 0;
    __syncwarp();
    // the wedges of 32 b's at a time: per lane one b (slot sb, tail start
    // and length), then the concatenated tails one entry per lane
    auto load_chunk = [&](u64 k0) -> u32 {
      const u64 k = k0 + lane;
      u32 len = 0, sb = 0;
      u64 st0 = 0;
      if (k < q1) {
        sb = g.tl[k];
        u64 l2 = g.tl_ptr[sb], h2 = g.tl_ptr[sb + 1];
        const u64 end = h2;
        while (l2 < h2) {  // first partner slot > s
          const u64 mid = l2 + ((h2 - l2) >> 1);
          if (g.tl[mid] <= (u32)s) l2 = mid + 1;
          else h2 = mid;
        }
        st0 = l2;
        len = (u32)(end - l2);
      }
      u32 incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      s_pref[wid][lane + 1] = incl;
      if (lane == 0) s_pref[wid][0] = 0;
      s_start[wid][lane] = st0;
      s_sb[wid][lane] = sb;
      __syncwarp();
      return s_pref[wid][32];
    };
    auto next_list = [&](u32 it, u32& l2) {  // l2: list of entry it (non-decreasing)
      if (s_pref[wid][l2 + 1] <= it) {
        u32 h2 = 32;
        ++l2;
        while (h2 - l2 > 1) {
          const u32 mid = (l2 + h2) >> 1;
          if (s_pref[wid][mid] <= it) l2 = mid;
          else h2 = mid;
        }
      }
    };
    // sweep 1: W' per partner c, and the cycles with top a
    u64 c4 = 0;
    u32 tot1 = 0;  // entries of the (last) chunk
    for (u64 k0 = kb; k0 < q1; k0 += 32) {
      const u32 tot = load_chunk(k0);
      tot1 = tot;
      u32 l2 = 0;
      for (u32 it = lane; it < tot; it += 32) {
        next_list(it, l2);
        const u32 pc = g.tl[s_start[wid][l2] + (it - s_pref[wid][l2])] - ub;
        u32 old;
        if (small) {
          const u32 sh = (pc & 1u) * 16u;
          old = (atomicAdd(&s_map[wid][pc >> 1], 1u << sh) >> sh) & 0xffffu;
        } else {
          old = atomicAdd(&gmap[pc], 1u);
        }
        c4 += old;
        if (old == 0) list[atomicAdd(&s_cnt[wid], 1u)] = pc;
      }
      __syncwarp();
    }
    // opposite vertices: C(W'(a,c), 2) each
    const u32 cnt = s_cnt[wid];
    for (u32 i = lane; i < cnt; i += 32) {
      const u32 pc = list[i];
      u32 w;
      if (small) {
        const u32 sh = (pc & 1u) * 16u;
        w = (s_map[wid][pc >> 1] >> sh) & 0xffffu;
      } else {
        w = gmap[pc];
      }
      if (w >= 2) atomicAdd(&sa.b68[ub + pc], (u64)w * (w - 1) / 2);
    }
    // sweep 2: each middle b of a wedge a - b - c gets W'(a,c) - 1.  With one
    // chunk only, its tables are still in shared memory from sweep 1.
    const bool one_chunk = q1 - kb <= 32;
    for (u64 k0 = kb; k0 < q1; k0 += 32) {
      const u32 tot = one_chunk ? tot1 : load_chunk(k0);
      const u32 iters = (tot + 31) & ~31u;
      u32 l2 = 0;
      for (u32 it = lane; it < iters; it += 32) {
        u32 key = 0xffffffffu;
        u64 add = 0;
        if (it < tot) {
          next_list(it, l2);
          const u32 pc = g.tl[s_start[wid][l2] + (it - s_pref[wid][l2])] - ub;
          u32 w;
          if (small) {
            const u32 sh = (pc & 1u) * 16u;
            w = (s_map[wid][pc >> 1] >> sh) & 0xffffu;
          } else {
            w = gmap[pc];
          }
          key = l2;
          add = w - 1;
        }
        bool tail;
        const u64 sum = seg_sum(key, add, &tail);
        if (tail && key != 0xffffffffu && sum) atomicAdd(&sa.b68[s_sb[wid][key]], sum);
      }
      __syncwarp();
    }
    __syncwarp();
    for (u32 i = lane; i < cnt; i += 32) {
      const u32 pc = list[i];
      if (small) s_map[wid][pc >> 1] = 0;
      else gmap[pc] = 0;
    }
    __syncwarp();
    c4 = warp_sum(c4);
    if (lane == 0 && c4) atomicAdd(&sa.b68[s], c4);
  }
}

}  // namespace

void link_configure() {
  cudaFuncSetAttribute(link_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLinkDynSmem);
}

void launch_link(const Graph& g, const SlotArrays& sa, u32* scratch, u32 warps, u32 dmax,
                 cudaStream_t st) {
  if (!g.S || !warps) return;
  link_kernel<<<warps / kLinkWarps, kLinkWarps * 32, kLinkDynSmem, st>>>(g, sa, scratch, dmax);
}
