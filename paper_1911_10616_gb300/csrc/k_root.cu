// Per-root 2-hop pass (Thm. 5vertexorbit, orbits needing W(u,v), TT(u,v) and
// D(u,v); Thm. 5-Cycle-Clique for orbit 34) and the orders of its roots.
//
// One CTA owns one root u at a time (persistent CTAs pull roots from a queue
// ordered by decreasing work, the degree-bucket schedule).  Each CTA has a
// dense map over all vertex ids in global memory (L2 resident for small
// roots) holding, for every x two hops from u:
//   W[x]   = |N(u) ^ N(x)|            (bit 31: x is a neighbour of u)
//   Wn[x]  = wedges u-v-x that are not in-in at v (not u->v<-x in the DAG)
//   TT[x]  = sum over wedges u-v-x of T(v,x)
//   D[x]   = edges inside N(u) ^ N(x)  (diamonds with u, x off the chord)
//   P[x]   = directed 3-paths u<-k->j->x  (k->u, k->j, j->x)
// Phases: (1) wedges -> W, Wn, TT;  (2) diamonds -> D and the orbit-64
// shares of the chord ends;  3-paths ending at u -> 5-cycle credits and P;
// (3) wedges again -> E5 = C4(u,v), orbit-49/62 shares of the centres, and
// the 5-cycle credit of the wedge centre; map scan -> orbits 8, 36, 50, 51, 63.
#include <cstdlib>

#include "evoke_internal.cuh"

namespace {

constexpr u32 kFlag = 0x80000000u;
constexpr u32 kCnt = 0x7fffffffu;

// bring the line holding *p into L2 without waiting for it
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// largest i in [0, len) with pref[i] <= w   (pref ascending, pref[0] = 0)
__device__ __forceinline__ u32 seg_find(const u32* pref, u32 len, u32 w) {
  u32 lo = 0, hi = len;
  while (hi - lo > 1) {
    u32 mid = lo + ((hi - lo) >> 1);
    if (pref[mid] <= w) lo = mid;
    else hi = mid;
  }
  return lo;
}

// sum `val` over runs of equal `key` in consecutive lanes; the last lane of
// each run adds the run total to arr[key].
__device__ __forceinline__ void seg_atomic_add(u64* arr, u32 key, bool valid, u64 val) {
  const int lane = threadIdx.x & 31;
  const u32 k = valid ? key : 0xffffffffu;
  if (!valid) val = 0;
  const u32 prev = __shfl_up_sync(0xffffffffu, k, 1);
  const u32 heads = __ballot_sync(0xffffffffu, lane == 0 || prev != k);
  const u32 upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
  const int start = 31 - __clz(heads & upto);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u64 y = __shfl_up_sync(0xffffffffu, val, o);
    if (lane - o >= start) val += y;
  }
  const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
  if (tail && valid && val) atomicAdd(&arr[k], val);
}

__device__ u64 block_sum(u64 v, u64* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  u64 t = 0;
  if (wid == 0) {
    t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0;
    t = warp_sum(t);
  }
  return t;  // valid in thread 0
}

// exclusive prefix of (deg[col[ub+i]]) for i < du into pref[0..du]
__device__ void neighbour_degree_prefix(const Graph& g, u32 ub, u32 du, u32* pref, u64* red,
                                        u32* s_carry) {
  if (threadIdx.x == 0) *s_carry = 0;
  __syncthreads();
  for (u32 base = 0; base < du; base += blockDim.x) {
    const u32 i = base + threadIdx.x;
    const u32 v = i < du ? g.deg[g.col[ub + i]] : 0;
    // block exclusive scan (32-bit)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    u32 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      u32 y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    u32* wt = reinterpret_cast<u32*>(red);
    if (lane == 31) wt[wid] = x;
    __syncthreads();
    if (wid == 0) {
      u32 t = lane < (int)(blockDim.x >> 5) ? wt[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        u32 y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      if (lane < (int)(blockDim.x >> 5)) wt[lane] = t;
    }
    __syncthreads();
    const u32 before = (wid ? wt[wid - 1] : 0) + *s_carry;
    if (i < du) pref[i] = before + x - v;
    const u32 tot = wt[(blockDim.x >> 5) - 1];
    __syncthreads();
    if (threadIdx.x == 0) *s_carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) pref[du] = *s_carry;
  __syncthreads();
}

// neighbour-degree prefix kept in shared memory for roots of degree below
// this (smaller for the narrow CTAs used on batches of small graphs)
template <int kThreads>
constexpr u32 smem_pref_cap() { return kThreads >= 256 ? 2048u : 512u; }


template <int kThreads>
__global__ void __launch_bounds__(kThreads, 1024 / kThreads)
root_kernel(Graph g, SlotArrays sa, u64* __restrict__ acc, RootScratch rs, u32* pref_all,
            u32 pref_stride) {
  constexpr u32 kCold = 0x40000000u;  // W bit 30: the cold record is in use
  constexpr u32 kW = 0x3fffffffu;
  const u32 n = g.n;
  const u64 off = (u64)blockIdx.x * rs.map_stride;
  MapHot* __restrict__ H = rs.hot + off;
  MapCold* __restrict__ C = rs.cold + off;
  u32* __restrict__ touched = rs.touched + off;
  u32* __restrict__ jlist = rs.jlist + off;
  // the records of the first rs.smem_recs ids live in shared memory instead
  // (after the relabelling by decreasing degree these are the hubs, which
  // most 2-hop walks reach); the global records of those ids stay unused
  extern __shared__ __align__(16) unsigned char root_dyn_smem[];
  MapHot* const s_hot = reinterpret_cast<MapHot*>(root_dyn_smem);
  const u32 K = rs.smem_recs;
  auto HP = [&](u32 lx) -> MapHot* { return lx < K ? s_hot + lx : H + lx; };
  for (u32 i = threadIdx.x; i < K; i += blockDim.x) s_hot[i] = MapHot{};
  __shared__ u32 s_wpref[kThreads / 32][33];
  __shared__ u64 s_wsab[kThreads / 32][32];
  __shared__ u32 s_wsa[kThreads / 32][32];
  __shared__ u32 s_wsb[kThreads / 32][32];
  constexpr u32 kSmemPref = smem_pref_cap<kThreads>();
  __shared__ u32 s_pref[kSmemPref + 1];
  __shared__ u32 s_nrp[kSmemPref];            // rowptr of each neighbour (small roots)
  __shared__ unsigned char s_nout[kSmemPref];  // u -> neighbour in the DAG
  __shared__ u32 s_root, s_nt, s_nj, s_carry, s_next, s_end;
  __shared__ u64 s_red[32];
  __shared__ long long s_t0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  u32* gpref = pref_all + (u64)blockIdx.x * pref_stride;

  if (threadIdx.x == 0) s_next = s_end = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      // roots come from the queue in chunks of rs.chunk consecutive entries
      if (s_next >= s_end) {
        s_next = atomicAdd(rs.head, rs.chunk);
        s_end = min(s_next + rs.chunk, n);
      }
      s_root = s_next < s_end ? s_next++ : n;
      s_nt = 0;
      s_nj = 0;
      s_t0 = clock64();
    }
    __syncthreads();
    const u32 qi = s_root;
    if (qi >= n) {
      if (rs.cta_end && threadIdx.x == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        rs.cta_end[blockIdx.x] = t;
      }
      break;
    }
    const u32 u = rs.order[qi];
    // maps are indexed by id within the root's component (batched graphs)
    const u32 cb = rs.comp_base ? rs.comp_base[u] : 0u;
    const u32 ub = g.rowptr[u], ue = g.rowptr[u + 1], du = ue - ub;
    u32* pref = du + 1 <= kSmemPref ? s_pref : gpref;
    long long tp = 0;
    if (rs.prof && threadIdx.x == 0) tp = clock64();
    u64 a51 = 0, a63 = 0;

    // phase 0: mark the neighbours, prefix of their degrees
    for (u32 i = threadIdx.x; i < du; i += blockDim.x) {
      const u32 v = g.col[ub + i];
      HP(v - cb)->W = kFlag;
      touched[atomicAdd(&s_nt, 1u)] = v;
    }
    const bool small = du + 1 <= kSmemPref;
    if (small)
      for (u32 i = threadIdx.x; i < du; i += blockDim.x) {
        const u32 v = g.col[ub + i];
        s_nrp[i] = g.rowptr[v];
        s_nout[i] = prec(g.deg, u, v) ? 1 : 0;
      }
    neighbour_degree_prefix(g, ub, du, pref, s_red, &s_carry);
    const u32 total = pref[du];
    // wedge w = (u, v_i, x): neighbour index i, slot t of x in row v_i, u -> v_i
    auto wedge = [&](u32 w, u32& i, u32& t, bool& out) {
      i = seg_find(pref, du + 1, w);
      if (small) {
        t = s_nrp[i] + (w - pref[i]);
        out = s_nout[i] != 0;
      } else {
        const u32 v = g.col[ub + i];
        t = g.rowptr[v] + (w - pref[i]);
        out = prec(g.deg, u, v);
      }
    };

    // phase 1: wedges u - v - x.  W (low word) and Wn (high word) of the hot
    // record are bumped by one 64-bit atomic.  An atomic that misses L2 is far
    // slower to serve than a read miss, so each thread prefetches the record
    // of its next wedge into L2 before it performs the current atomic.
    {
      constexpr u32 kNone = 0xffffffffu;
      auto target = [&](u32 w, u32& x, bool& in_in) {
        u32 i, t;
        bool out;
        wedge(w, i, t, out);
        x = g.col[t];
        in_in = out && g.sin[t];  // u -> v <- x
        if (x == u) x = kNone;
        else if (x - cb >= K) prefetch_l2(H + (x - cb));
      };
      u32 x = kNone;
      bool in_in = false;
      if (threadIdx.x < total) target(threadIdx.x, x, in_in);
      for (u32 w = threadIdx.x; w < total; w += blockDim.x) {
        u32 xn = kNone;
        bool inn = false;
        if (w + blockDim.x < total) target(w + blockDim.x, xn, inn);
        if (x != kNone) {
          const u64 old = atomicAdd(reinterpret_cast<u64*>(&HP(x - cb)->W),
                                    in_in ? 1ull : (1ull | (1ull << 32)));
          if ((u32)old == 0) touched[atomicAdd(&s_nt, 1u)] = x;
        }
        x = xn;
        in_in = inn;
      }
    }
    __syncthreads();
    if (rs.prof && threadIdx.x == 0) {
      long long t = clock64();
      atomicAdd(&rs.prof[0], (u64)(t - tp));
      tp = t;
    }

    {
    // phase 2a: diamonds.  Triangle (u,a,b) with a < b; every y in
    // N(a)^N(b) other than u closes a diamond with chord (a,b) and u, y off
    // the chord.  Each warp takes 32 triangle-list entries of u at a time and
    // walks the concatenation of their chord lists, one list entry per lane.
    {
      const u64 q0 = g.tl_ptr[ub], q1 = g.tl_ptr[ue];
      const u64 span = q1 - q0;
      for (u64 base = (u64)wid * 32; base < span; base += (u64)nw * 32) {
        const u64 q = q0 + base + lane;
        u32 len = 0, sab = 0, sa_ = 0, sb = 0;
        if (q < q1) {
          u32 lo = ub, hi = ue;
          while (hi - lo > 1) {
            u32 mid = lo + ((hi - lo) >> 1);
            if (g.tl_ptr[mid] <= q) lo = mid;
            else hi = mid;
          }
          sb = g.tl[q];
          sa_ = lo;
          if (sb > lo) {  // b > a, each triangle at u once
            sab = g.tl[g.tl_ptr[g.rev[lo]] + (q - g.tl_ptr[lo])];
            len = (u32)(g.tl_ptr[sab + 1] - g.tl_ptr[sab]);
          }
        }
        u32 incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        s_wpref[wid][lane + 1] = incl;
        if (lane == 0) s_wpref[wid][0] = 0;
        s_wsab[wid][lane] = len ? g.tl_ptr[sab] : 0;
        s_wsa[wid][lane] = sa_;
        s_wsb[wid][lane] = sb;
        __syncwarp();
        const u32 tot = s_wpref[wid][32];
        u32 lo = 0;  // chord list of entry `it`; non-decreasing as `it` grows
        for (u32 it0 = 0; it0 < tot; it0 += 32) {
          const u32 it = it0 + lane;
          u32 key = 0xffffffffu;
          u64 add = 0;
          if (it < tot) {
            if (s_wpref[wid][lo + 1] <= it) {
              u32 hi = 32;
              ++lo;
              while (hi - lo > 1) {
                const u32 mid = (lo + hi) >> 1;
                if (s_wpref[wid][mid] <= it) lo = mid;
                else hi = mid;
              }
            }
            const u32 y = g.tlv[s_wsab[wid][lo] + (it - s_wpref[wid][lo])];
            if (y != u) {
              const u64 wy2 = (u64)((long long)(HP(y - cb)->W & kW) - 2);
              a63 += wy2;                 // DM63: sum over diamonds of W(u,y) - 2
              if (u < y) {
                atomicAdd(&HP(y - cb)->D, 1u);  // D(u,y), needed for y > u only
                add = wy2;
                key = lo;
              }
            }
          }
          bool tail;
          const u64 sum = seg_sum(key, add, &tail);
          if (tail && key != 0xffffffffu && sum) {  // orbit-64 shares of the chord ends
            atomicAdd(&sa.b64[s_wsa[wid][key]], sum);
            atomicAdd(&sa.b64[s_wsb[wid][key]], sum);
          }
        }
        __syncwarp();
      }
    }
    // phase 2b: directed 3-paths u <- k -> j -> i (Fig. 5cycle with l = u),
    // grouped by the middle vertex j:  R[j] = |N-(u) ^ N-(j)| (out-out
    // wedges u <- k -> j), Y[j] = sum over those k of the triangles k->j->x
    // with k->x, X[x] = sum over k in N-(u) ^ N-(x) of the triangles k->y->x.
    for (u32 idx = wid; idx < du; idx += nw) {
      const u32 k = g.col[ub + idx];
      if (!prec(g.deg, k, u)) continue;  // k -> u
      const u32 pe = g.dag_ptr[k + 1];
      // the cold records are first touched here: prefetch each lane's next one
      if (g.dag_ptr[k] + lane < pe) prefetch_l2(C + (g.dag_col[g.dag_ptr[k] + lane] - cb));
      for (u32 p = g.dag_ptr[k] + lane; p < pe; p += 32) {
        const u32 x = g.dag_col[p];
        if (p + 32 < pe) prefetch_l2(C + (g.dag_col[p + 32] - cb));
        if (x == u) continue;
        const u32 sk = g.dag_slot[p];
        const u64 old = atomicAdd(&C[x - cb].RY, (1ull << 32) | (u64)sa.Mtop[sk]);
        if ((old >> 32) == 0) {
          jlist[atomicAdd(&s_nj, 1u)] = x;
          atomicOr(&HP(x - cb)->W, kCold);
        }
        const u32 mm = sa.Mmid[sk];
        if (mm) atomicAdd(&C[x - cb].X, mm);
      }
    }
    __syncthreads();
    if (rs.prof && threadIdx.x == 0) {
      long long t = clock64();
      atomicAdd(&rs.prof[1], (u64)(t - tp));
      tp = t;
    }
    // phase 2c: per middle vertex j, push R[j] to every end i in N+(j) (the
    // 3-path counts P) and pull Z[j] = sum of Wn over N+(j); credit j.
    {
      const u32 nj = s_nj;
      for (u32 idx = wid; idx < nj; idx += nw) {
        const u32 j = jlist[idx];
        const u64 ry = C[j - cb].RY;
        const u64 R = ry >> 32, Yj = ry & 0xffffffffull;
        const bool jl = (HP(j - cb)->W & kFlag) != 0;
        const bool j_to_u = jl && prec(g.deg, j, u);
        u64 z = 0;
        for (u32 p = g.dag_ptr[j] + lane; p < g.dag_ptr[j + 1]; p += 32) {
          const u32 i = g.dag_col[p];
          if (i == u) continue;
          MapHot* hi = HP(i - cb);
          const u32 wn = hi->Wn;
          if (!wn) continue;
          z += wn;
          const u32 old = atomicAdd(&hi->P, (u32)R);
          if (old + (u32)R < old) *rs.overflow = 1;
          if (jl) {
            atomicAdd(&C[i - cb].Pjl, R);
            if (!(hi->W & kCold)) atomicOr(&hi->W, kCold);
          }
        }
        z = warp_sum(z);
        if (lane == 0) {
          C[j - cb].Z = z;
          const u64 dpj = (u64)(g.dag_ptr[j + 1] - g.dag_ptr[j]) - (j_to_u ? 1 : 0);
          const u64 cj = R * z - Yj + (j_to_u ? R : 0) - (jl ? 2 * R * dpj : 0);
          if (cj) atomicAdd(&acc[(u64)A_C5 * n + j], cj);
        }
      }
    }
    __syncthreads();
    if (rs.prof && threadIdx.x == 0) {
      long long t = clock64();
      atomicAdd(&rs.prof[2], (u64)(t - tp));
      tp = t;
    }

    // phase 3a: wedges again, now that W, D and P are complete: E5 = C4(u,v),
    // orbit-49/62 shares of the centre, 5-cycle credit of the wedge centre,
    // and DM51 = sum over wedges u-v-x of (T(v,x) - [u~x]) (W(u,x) - 1).
    {
      const u32 iters = (total + blockDim.x - 1) / blockDim.x * blockDim.x;
      for (u32 w = threadIdx.x; w < iters; w += blockDim.x) {
        bool valid = w < total;
        u32 s = 0;
        u64 e5 = 0, b49 = 0, b62 = 0, bw = 0;
        if (valid) {
          u32 i, t;
          bool out;
          wedge(w, i, t, out);
          const u32 x = g.col[t];
          s = ub + i;
          if (x == u) {
            valid = false;
          } else {
            const MapHot h = *HP(x - cb);
            const long long wx = h.W & kW;
            e5 = (u64)(wx - 1);
            a51 += ((u64)sa.T[t] - ((h.W & kFlag) ? 1 : 0)) * (u64)(wx - 1);
            if (u < x) {
              b49 = c2(wx - 1);
              b62 = h.D;
            }
            if (!(out && g.sin[t])) bw = h.P;
          }
        }
        seg_atomic_add(sa.E5, s, valid, e5);
        seg_atomic_add(sa.b49, s, valid, b49);
        seg_atomic_add(sa.b62, s, valid, b62);
        seg_atomic_add(sa.bc5, s, valid, bw);
      }
    }
    // phase 3a': 5-cycle credit of each in-neighbour k (the source vertex)
    for (u32 idx = wid; idx < du; idx += nw) {
      const u32 k = g.col[ub + idx];
      if (!prec(g.deg, k, u)) continue;
      u64 zs = 0;
      for (u32 p = g.dag_ptr[k] + lane; p < g.dag_ptr[k + 1]; p += 32) {
        const u32 j = g.dag_col[p];
        if (j == u) continue;
        u64 t = C[j - cb].Z;
        if (HP(j - cb)->W & kFlag) {
          const u64 dpj = (u64)(g.dag_ptr[j + 1] - g.dag_ptr[j]) - (prec(g.deg, j, u) ? 1 : 0);
          t -= dpj;
        }
        zs += t;
      }
      zs = warp_sum(zs);
      if (lane == 0) {
        const u32 rk = g.rev[ub + idx];  // slot of u in row k (a DAG slot)
        const u64 tri = rs.tsrc[k] - sa.Mtop[rk] - sa.Mmid[rk];
        const u64 ck = zs - 2 * tri;
        if (ck) atomicAdd(&sa.bc5[ub + idx], ck);
      }
    }
    __syncthreads();
    if (rs.prof && threadIdx.x == 0) {
      long long t = clock64();
      atomicAdd(&rs.prof[3], (u64)(t - tp));
      tp = t;
    }

    }

    // phase 3b: scan the map (orbits 8, 36, 50; the 5-cycle credits of the
    // path ends), reset it
    {
      u64 a8 = 0, a36 = 0, a50 = 0, a5 = 0;
      const u32 nt = s_nt;
      for (u32 idx = threadIdx.x; idx < nt; idx += blockDim.x) {
        const u32 x = touched[idx];
        const MapHot h = *HP(x - cb);
        const long long w = h.W & kW;
        const u64 cw2 = c2(w);
        a8 += cw2;
        a36 += cw2 * (u64)((long long)g.deg[x] - 2);
        a50 += c3(w);
        if (h.W & kCold) {
          const MapCold c = C[x - cb];
          if (h.P | c.X) {
            const bool u_to_x = (h.W & kFlag) && prec(g.deg, u, x);
            const u64 rx = c.RY >> 32;
            const u64 ci = (u64)h.P * (u64)h.Wn - ((u64)c.X - (u_to_x ? rx : 0)) - c.Pjl;
            if (ci) atomicAdd(&acc[(u64)A_C5 * n + x], ci);
            a5 += ci;
          }
          C[x - cb] = MapCold{};
        } else if (h.P) {
          const u64 ci = (u64)h.P * (u64)h.Wn;
          if (ci) atomicAdd(&acc[(u64)A_C5 * n + x], ci);
          a5 += ci;
        }
        *HP(x - cb) = MapHot{};
      }
      a8 = block_sum(a8, s_red);
      if (threadIdx.x == 0) acc[(u64)A_DM8 * n + u] = a8;
      a36 = block_sum(a36, s_red);
      if (threadIdx.x == 0) acc[(u64)A_S36 * n + u] = a36;
      a50 = block_sum(a50, s_red);
      if (threadIdx.x == 0) acc[(u64)A_S50 * n + u] = a50;
      a51 = block_sum(a51, s_red);
      if (threadIdx.x == 0) acc[(u64)A_S51 * n + u] = a51;
      a63 = block_sum(a63, s_red);
      if (threadIdx.x == 0) acc[(u64)A_S63 * n + u] = a63;
      a5 = block_sum(a5, s_red);
      if (threadIdx.x == 0 && a5) atomicAdd(&acc[(u64)A_C5 * n + u], a5);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const long long t = clock64();
      if (rs.prof) atomicAdd(&rs.prof[4], (u64)(t - tp));
      if (rs.cycles) rs.cycles[u] = (u64)(t - s_t0);
    }
  }
}

// --- degree-bucket schedule: roots by decreasing wedge work ------------------
__device__ __forceinline__ u32 bucket_of(u64 work) { return 63u - (u32)__clzll(work | 1ull); }

__global__ void sched_hist_kernel(const u64* __restrict__ work, u32 n, u32* cnt) {
  const u32 u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < n) atomicAdd(&cnt[63u - bucket_of(work[u])], 1u);
}
__global__ void sched_scan_kernel(u32* cnt, u32* head) {
  u32 run = 0;
  for (int b = 0; b < 64; ++b) {
    const u32 c = cnt[b];
    cnt[b] = run;
    run += c;
  }
  *head = 0;
}
__global__ void sched_scatter_kernel(const u64* __restrict__ work, u32 n, u32* cursor,
                                     u32* order) {
  const u32 u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < n) order[atomicAdd(&cursor[63u - bucket_of(work[u])], 1u)] = u;
}

}  // namespace

u32 root_map_stride(u32 map_n) {
  const u64 lines = ((u64)map_n + 7) / 8 + 3;  // 8 hot records per 128-byte line
  return (u32)((lines | 1) * 8);
}

size_t root_scratch_bytes(u32 map_stride, int ctas) {
  return (size_t)ctas * map_stride * (sizeof(MapHot) + sizeof(MapCold) + 2 * sizeof(u32)) +
         16 * 256;
}

// --- hub-grouped schedule: roots ordered by their highest-degree neighbour --
// After the relabelling by decreasing degree that neighbour is the first entry
// of the row.  Roots that share it have largely the same 2-hop set, so a CTA
// that takes several of them in a row re-touches the same map lines (and the
// same adjacency row) while they are still cached.  Counting sort by that key.
__device__ __forceinline__ u32 hub_key(const Graph& g, u32 u) {
  const u32 b = g.rowptr[u];
  return g.rowptr[u + 1] > b ? g.col[b] : g.n - 1;
}
__global__ void hub_hist_kernel(Graph g, u32* cnt) {
  const u32 u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < g.n) atomicAdd(&cnt[hub_key(g, u)], 1u);
}
__global__ void hub_scatter_kernel(Graph g, u32* cursor, u32* order) {
  const u32 u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < g.n) order[atomicAdd(&cursor[hub_key(g, u)], 1u)] = u;
}

void launch_hub_schedule(const Graph& g, RootScratch& rs, u32* cnt, void* scan_tmp,
                         cudaStream_t st) {
  if (!g.n) return;
  cudaMemsetAsync(cnt, 0, sizeof(u32) * g.n, st);
  hub_hist_kernel<<<(g.n + 255) / 256, 256, 0, st>>>(g, cnt);
  launch_scan_u32_inplace(cnt, g.n, scan_tmp, st);
  hub_scatter_kernel<<<(g.n + 255) / 256, 256, 0, st>>>(g, cnt, rs.order);
}

void launch_schedule(const Graph& g, u64* acc, RootScratch& rs, cudaStream_t st) {
  if (!g.n) return;
  const u64* work = acc + (u64)A_WORK * g.n;
  cudaMemsetAsync(rs.bucket_cnt, 0, 64 * sizeof(u32), st);
  sched_hist_kernel<<<(g.n + 255) / 256, 256, 0, st>>>(work, g.n, rs.bucket_cnt);
  sched_scan_kernel<<<1, 1, 0, st>>>(rs.bucket_cnt, rs.head);
  sched_scatter_kernel<<<(g.n + 255) / 256, 256, 0, st>>>(work, g.n, rs.bucket_cnt, rs.order);
}

namespace {
// Shared memory left for map records when `per_sm` CTAs of root_kernel<T>
// share an SM; sets the kernel's dynamic shared-memory limit once.
template <int T>
size_t root_dyn_smem(int per_sm) {
  static size_t static_smem = 0, per_sm_smem = 0, reserved = 0, optin = 0;
  static bool ready = false;
  if (!ready) {
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, root_kernel<T>);
    int dev = 0, a = 0, b = 0, c = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&a, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&b, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&c, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    static_smem = fa.sharedSizeBytes;
    per_sm_smem = (size_t)a;
    reserved = (size_t)b;
    optin = (size_t)c;
    const size_t cap = optin > static_smem ? optin - static_smem : 0;
    cudaFuncSetAttribute(root_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
    ready = true;
  }
  if (per_sm < 1) per_sm = 1;
  const size_t share = per_sm_smem / (size_t)per_sm;
  if (share <= reserved + static_smem + 1024) return 0;
  size_t dyn = share - reserved - static_smem;
  if (dyn + static_smem > optin) dyn = optin - static_smem;
  return dyn / 512 * 512;
}
}  // namespace

void launch_root_with_pref(const Graph& g, const SlotArrays& sa, u64* acc, RootScratch& rs,
                           u32* pref, u32 pref_stride, cudaStream_t st) {
  if (!g.n) return;
  cudaMemsetAsync(rs.head, 0, sizeof(u32), st);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = (rs.ctas + sms - 1) / sms;
  size_t dyn = 0;
  switch (rs.threads) {
    case 64: dyn = root_dyn_smem<64>(per_sm); break;
    case 128: dyn = root_dyn_smem<128>(per_sm); break;
    case 256: dyn = root_dyn_smem<256>(per_sm); break;
    case 1024: dyn = root_dyn_smem<1024>(per_sm); break;
    default: dyn = root_dyn_smem<512>(per_sm);
  }
  const u64 max_recs = dyn / sizeof(MapHot);
  // more records than this cost the root pass more L1 cache than they save
  // in map traffic (measured on the 1M-vertex Chung-Lu graph: 3,072 records
  // per 512- or 1024-thread CTA, 512 per 256-thread CTA)
  const u64 cap = rs.threads >= 512 ? 3072 : rs.threads == 256 ? 512 : max_recs;
  u64 recs = max_recs < cap ? max_recs : cap;
  if (const char* e = getenv("EVOKE_ROOT_SMEM_RECS")) {  // tuning override
    const long long r = atoll(e);
    if (r >= 0) recs = (u64)r < max_recs ? (u64)r : max_recs;
  }
  if (recs > rs.map_n) recs = rs.map_n;
  rs.smem_recs = (u32)recs;
  dyn = (size_t)recs * sizeof(MapHot);
  switch (rs.threads) {
    case 64: root_kernel<64><<<rs.ctas, 64, dyn, st>>>(g, sa, acc, rs, pref, pref_stride); break;
    case 128: root_kernel<128><<<rs.ctas, 128, dyn, st>>>(g, sa, acc, rs, pref, pref_stride); break;
    case 256: root_kernel<256><<<rs.ctas, 256, dyn, st>>>(g, sa, acc, rs, pref, pref_stride); break;
    case 1024: root_kernel<1024><<<rs.ctas, 1024, dyn, st>>>(g, sa, acc, rs, pref, pref_stride); break;
    default: root_kernel<512><<<rs.ctas, 512, dyn, st>>>(g, sa, acc, rs, pref, pref_stride);
  }
}

void root_configure() {
  root_dyn_smem<64>(16);
  root_dyn_smem<128>(8);
  root_dyn_smem<256>(4);
  root_dyn_smem<512>(2);
  root_dyn_smem<1024>(1);
}

