// Per-root 2-hop pass (Thm. 5vertexorbit, orbits needing W(u,v), TT(u,v) and
// D(u,v); Thm. 5-Cycle-Clique for orbit 34), the wheel pass (orbits 68, 69)
// and 5-cliques (orbit 72).
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
#include "evoke_internal.cuh"

namespace {

constexpr int kRootThreads = 512;
constexpr u32 kFlag = 0x80000000u;
constexpr u32 kCnt = 0x7fffffffu;

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

__global__ void __launch_bounds__(kRootThreads)
root_kernel(Graph g, SlotArrays sa, u64* __restrict__ acc, RootScratch rs, u32* pref_all,
            u32 pref_stride) {
  const u32 n = g.n;
  const u64 off = (u64)blockIdx.x * n;
  u32* __restrict__ W = rs.W + off;
  u32* __restrict__ Wn = rs.Wn + off;
  u32* __restrict__ D = rs.D + off;
  u32* __restrict__ P = rs.P + off;
  u64* __restrict__ TT = rs.TT + off;
  u32* __restrict__ touched = rs.touched + off;
  u32* pref = pref_all + (u64)blockIdx.x * pref_stride;
  __shared__ u32 s_root, s_nt, s_carry;
  __shared__ u64 s_red[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;

  for (;;) {
    if (threadIdx.x == 0) {
      s_root = atomicAdd(rs.head, 1u);
      s_nt = 0;
    }
    __syncthreads();
    const u32 qi = s_root;
    if (qi >= n) break;
    const u32 u = rs.order[qi];
    const u32 ub = g.rowptr[u], ue = g.rowptr[u + 1], du = ue - ub;
    const u32 degu = du;

    // phase 0: mark the neighbours, prefix of their degrees
    for (u32 i = threadIdx.x; i < du; i += blockDim.x) {
      const u32 v = g.col[ub + i];
      W[v] = kFlag;
      touched[atomicAdd(&s_nt, 1u)] = v;
    }
    neighbour_degree_prefix(g, ub, du, pref, s_red, &s_carry);
    const u32 total = pref[du];

    // phase 1: wedges u - v - x
    for (u32 w = threadIdx.x; w < total; w += blockDim.x) {
      const u32 i = seg_find(pref, du + 1, w);
      const u32 v = g.col[ub + i];
      const u32 t = g.rowptr[v] + (w - pref[i]);
      const u32 x = g.col[t];
      if (x == u) continue;
      const u32 old = atomicAdd(&W[x], 1u);
      if (old == 0) touched[atomicAdd(&s_nt, 1u)] = x;
      if (!(prec(g.deg, u, v) && prec(g.deg, x, v))) atomicAdd(&Wn[x], 1u);
      atomicAdd(&TT[x], (u64)sa.T[t]);
    }
    __syncthreads();

    // phase 2a: diamonds.  Triangle (u,a,b) with a < b; every y in
    // N(a)^N(b) other than u closes a diamond with chord (a,b).
    {
      const u64 q0 = g.tl_ptr[ub], q1 = g.tl_ptr[ue];
      for (u64 q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        // owning slot of entry q within row u
        u32 lo = ub, hi = ue;
        while (hi - lo > 1) {
          u32 mid = lo + ((hi - lo) >> 1);
          if (g.tl_ptr[mid] <= q) lo = mid;
          else hi = mid;
        }
        const u32 s = lo;
        const u32 sb = g.tl[q];
        if (sb <= s) continue;  // b > a, each triangle at u once
        const u32 sab = g.tl[g.tl_ptr[g.rev[s]] + (q - g.tl_ptr[s])];
        u64 add64 = 0;
        for (u64 k = g.tl_ptr[sab]; k < g.tl_ptr[sab + 1]; ++k) {
          const u32 y = g.col[g.tl[k]];
          if (y == u) continue;
          atomicAdd(&D[y], 1u);
          if (u < y) add64 += (u64)((long long)(W[y] & kCnt) - 2);
        }
        if (add64) {
          atomicAdd(&sa.b64[s], add64);
          atomicAdd(&sa.b64[sb], add64);
        }
      }
    }
    // phase 2b: directed 3-paths u <- k -> j -> i  (Fig. 5cycle, l = u)
    {
      u64 cl = 0;
      for (u32 idx = wid; idx < du; idx += nw) {
        const u32 k = g.col[ub + idx];
        if (!prec(g.deg, k, u)) continue;  // need k -> u
        const u32 kb = g.dag_ptr[k], ke = g.dag_ptr[k + 1];
        u64 ck = 0;
        for (u32 p = kb + lane; p < ke; p += 32) {
          const u32 j = g.dag_col[p];
          if (j == u) continue;
          const u32 jl = (W[j] & kFlag) ? 1u : 0u;
          u64 cj = 0;
          for (u32 p2 = g.dag_ptr[j]; p2 < g.dag_ptr[j + 1]; ++p2) {
            const u32 i = g.dag_col[p2];
            if (i == u) continue;
            const u32 wn = Wn[i];
            if (!wn) continue;
            const u32 ik = contains_u32(g.dag_col, kb, ke, i) ? 1u : 0u;
            const u64 c = (u64)(wn - ik - jl);
            cl += c;
            ck += c - ik;
            cj += c - jl;
            if (c) atomicAdd(&acc[(u64)A_C5 * n + i], c);
            atomicAdd(&P[i], 1u);
          }
          if (cj) atomicAdd(&acc[(u64)A_C5 * n + j], cj);
        }
        ck = warp_sum(ck);
        if (lane == 0 && ck) atomicAdd(&sa.bc5[ub + idx], ck);
      }
      cl = block_sum(cl, s_red);
      if (threadIdx.x == 0 && cl) atomicAdd(&acc[(u64)A_C5 * n + u], cl);
    }
    __syncthreads();

    // phase 3a: wedges again, now that W, D and P are complete
    {
      const u32 iters = (total + blockDim.x - 1) / blockDim.x * blockDim.x;
      for (u32 w = threadIdx.x; w < iters; w += blockDim.x) {
        bool valid = w < total;
        u32 s = 0;
        u64 e5 = 0, b49 = 0, b62 = 0, bw = 0;
        if (valid) {
          const u32 i = seg_find(pref, du + 1, w);
          const u32 v = g.col[ub + i];
          const u32 t = g.rowptr[v] + (w - pref[i]);
          const u32 x = g.col[t];
          s = ub + i;
          if (x == u) {
            valid = false;
          } else {
            const long long wx = W[x] & kCnt;
            e5 = (u64)(wx - 1);
            if (u < x) {
              b49 = c2(wx - 1);
              b62 = D[x];
            }
            if (!(prec(g.deg, u, v) && prec(g.deg, x, v))) bw = P[x];
          }
        }
        seg_atomic_add(sa.E5, s, valid, e5);
        seg_atomic_add(sa.b49, s, valid, b49);
        seg_atomic_add(sa.b62, s, valid, b62);
        seg_atomic_add(sa.bc5, s, valid, bw);
      }
    }
    __syncthreads();

    // phase 3b: scan the map, reset it
    {
      u64 a8 = 0, a36 = 0, a50 = 0, a51 = 0, a63 = 0;
      const u32 nt = s_nt;
      for (u32 idx = threadIdx.x; idx < nt; idx += blockDim.x) {
        const u32 x = touched[idx];
        const u32 wr = W[x];
        const long long w = wr & kCnt;
        const u64 cw2 = c2(w);
        a8 += cw2;
        a36 += cw2 * (u64)((long long)g.deg[x] - 2);
        a50 += c3(w);
        const u64 tt = TT[x] - ((wr & kFlag) ? (u64)w : 0);
        a51 += tt * (u64)(w - 1);
        a63 += (u64)D[x] * (u64)(w - 2);
        W[x] = 0;
        Wn[x] = 0;
        D[x] = 0;
        P[x] = 0;
        TT[x] = 0;
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
    }
    (void)degu;
    __syncthreads();
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

// --- wheel pass: 4-cycles through a inside N(u), for every slot (u,a) ------
// sum_c C(W_c, 2) is accumulated as the sum of the counter value before each
// increment.
__global__ void link_kernel(Graph g, SlotArrays sa, u32* __restrict__ scratch, u32 dmax) {
  const u32 gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u32 nwarps = (gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  u32* M = scratch + (u64)gw * dmax;
  for (u64 s = gw; s < g.S; s += nwarps) {
    if (sa.T[s] < 2) continue;
    const u32 a = g.col[s];
    (void)a;
    // row of s: the map is indexed by position in that row
    u32 lo = 0, hi = g.n;
    while (hi - lo > 1) {
      u32 mid = lo + ((hi - lo) >> 1);
      if (g.rowptr[mid] <= (u32)s) lo = mid;
      else hi = mid;
    }
    const u32 ub = g.rowptr[lo];
    u64 c4 = 0;
    for (u64 k = g.tl_ptr[s] + lane; k < g.tl_ptr[s + 1]; k += 32) {
      const u32 sb = g.tl[k];
      for (u64 k2 = g.tl_ptr[sb]; k2 < g.tl_ptr[sb + 1]; ++k2) {
        const u32 sc = g.tl[k2];
        if (sc == (u32)s) continue;
        c4 += atomicAdd(&M[sc - ub], 1u);
      }
    }
    __syncwarp();
    for (u64 k = g.tl_ptr[s] + lane; k < g.tl_ptr[s + 1]; k += 32) {
      const u32 sb = g.tl[k];
      for (u64 k2 = g.tl_ptr[sb]; k2 < g.tl_ptr[sb + 1]; ++k2) M[g.tl[k2] - ub] = 0;
    }
    __syncwarp();
    c4 = warp_sum(c4);
    if (lane == 0) sa.b68[s] = c4;
  }
}

// --- 5-cliques: per DAG edge (a -> b), triangles inside N+(a)^N+(b) --------
__global__ void k5_kernel(Graph g, u64* __restrict__ acc, u32 m) {
  const u32 e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  // source of DAG edge e
  u32 lo = 0, hi = g.n;
  while (hi - lo > 1) {
    u32 mid = lo + ((hi - lo) >> 1);
    if (g.dag_ptr[mid] <= e) lo = mid;
    else hi = mid;
  }
  const u32 a = lo, b = g.dag_col[e];
  const u32 ab = g.dag_ptr[a], ae = g.dag_ptr[a + 1];
  const u32 bb = g.dag_ptr[b], be = g.dag_ptr[b + 1];
  if (ae - ab < 3 || be - bb < 3) return;
  const u32 n = g.n;
  u64 cab = 0;
  u32 i = ab, j = bb;
  while (i < ae && j < be) {
    const u32 x = g.dag_col[i], y = g.dag_col[j];
    if (x < y) { ++i; continue; }
    if (y < x) { ++j; continue; }
    const u32 c = x;
    ++i;
    ++j;
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
  if (cab) {
    atomicAdd(&acc[(u64)A_K5 * n + a], cab);
    atomicAdd(&acc[(u64)A_K5 * n + b], cab);
  }
}

}  // namespace

size_t root_scratch_bytes(u32 n, int ctas) {
  return (size_t)ctas * n * (4 * sizeof(u32) + sizeof(u64) + sizeof(u32));
}

void launch_schedule(const Graph& g, u64* acc, RootScratch& rs, cudaStream_t st) {
  if (!g.n) return;
  const u64* work = acc + (u64)A_WORK * g.n;
  cudaMemsetAsync(rs.bucket_cnt, 0, 64 * sizeof(u32), st);
  sched_hist_kernel<<<(g.n + 255) / 256, 256, 0, st>>>(work, g.n, rs.bucket_cnt);
  sched_scan_kernel<<<1, 1, 0, st>>>(rs.bucket_cnt, rs.head);
  sched_scatter_kernel<<<(g.n + 255) / 256, 256, 0, st>>>(work, g.n, rs.bucket_cnt, rs.order);
}

void launch_root_with_pref(const Graph& g, const SlotArrays& sa, u64* acc, RootScratch& rs,
                           u32* pref, u32 pref_stride, cudaStream_t st) {
  if (!g.n) return;
  cudaMemsetAsync(rs.head, 0, sizeof(u32), st);
  root_kernel<<<rs.ctas, kRootThreads, 0, st>>>(g, sa, acc, rs, pref, pref_stride);
}

void launch_link(const Graph& g, const SlotArrays& sa, u32* scratch, u32 warps, u32 dmax,
                 cudaStream_t st) {
  if (!g.S || !warps) return;
  link_kernel<<<(warps * 32 + 255) / 256, 256, 0, st>>>(g, sa, scratch, dmax);
}

void launch_k5(const Graph& g, u64* acc, cudaStream_t st) {
  const u32 m = (u32)(g.S / 2);
  if (!m) return;
  k5_kernel<<<(m + 255) / 256, 256, 0, st>>>(g, acc, m);
}
