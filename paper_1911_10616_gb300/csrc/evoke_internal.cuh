// Internal declarations shared by the translation units of libevoke (the CUDA
// path).  Nothing here is part of the public C ABI (include/evoke.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

typedef unsigned long long u64;
typedef unsigned int u32;

// ---------------------------------------------------------------------------
// Per-vertex accumulators (int64, wrapping arithmetic), structure of arrays:
// acc[A_xxx * n + u].  Each entry is one partial sum of the equations of
// Lem. 4vertexorbit / Thm. 5vertexorbit, named after the orbit it feeds.
// ---------------------------------------------------------------------------
enum AccIndex : int {
  A_T = 0,     // T(u): triangles at u
  A_DM1,       // sum_{v in N(u)} (d(v)-1)
  A_DM6,       // sum C(d(v)-1, 2)
  A_DM10,      // sum T(u,v) (d(v)-2)
  A_DM13,      // sum C(T(u,v), 2)
  A_S22,       // sum C(d(v)-1, 3)
  A_S41,       // sum C(T(u,v),2) (d(v)-3)
  A_S55,       // sum C(T(u,v),3)
  A_S12,       // opposite-edge sum of (T(v,x)-1), each triangle twice
  A_S54,       // opposite-edge sum of C(T(v,x)-1, 2), twice
  A_S46,       // opposite-edge sum of E7(v,x), twice
  A_S52,       // opposite-edge sum of E5(v,x), twice
  A_S59,       // opposite-edge sum of E9<v,x> + E9<x,v>, twice
  A_S65,       // opposite-edge sum of E11(v,x) = K4(v,x), twice
  A_S70,       // sum over 4-cliques at u of (K4(opposite triangle) - 1)
  A_S66,       // sum over 4-cliques at u of T-sum of the opposite triangle
  A_S71,       // sum over triangles at u of C(K4(t), 2)
  A_DM8,       // C4(u)
  A_S36,       // sum_v C(W(u,v),2) (d(v)-2)
  A_S50,       // sum_v C(W(u,v),3)
  A_S51,       // sum_v TT(u,v) (W(u,v)-1)
  A_S63,       // sum_v D(u,v) (W(u,v)-2)
  A_C5,        // 5-cycles through u
  A_K5,        // 5-cliques through u
  A_S4,        // sum DM1(v)
  A_S9,        // sum (T(v) - T(u,v))
  A_S18,       // sum DM6(v)
  A_S19,       // sum DM5(v)
  A_S24,       // sum DM10(v)
  A_S28,       // sum T(v)
  A_S31,       // sum (d(v)-1) T(v)
  A_S35,       // sum DM8(v)
  A_S37,       // sum E5(u,v) (d(v)-2)
  A_S39,       // sum DM13(v)
  A_S40,       // sum E9<v,u> (d(v)-3)
  A_S45,       // sum DM12(v)
  A_S57,       // sum E11(u,v) (d(v)-3)
  A_S60,       // sum E9<v,u> (T(u,v)-1)
  A_S67,       // sum E11(u,v) (T(u,v)-2)
  A_K4X3,      // sum E11(u,v) = 3 K4(u)
  A_S29,       // sum T(u,v) DM1(v)
  A_S32,       // sum T(u,v) C(d(v)-2, 2)
  A_S43,       // sum T(u,v) (T(v)-1)
  A_S48,       // sum (T(u,v)-1) E7(u,v)
  A_S61,       // sum (T(u,v)-1) E9<u,v>   (twice the triangle sum)
  A_S53,       // sum T(u,v) E5(u,v)
  A_S25,       // sum (d(v)-2) E7(u,v)      (twice the triangle sum)
  A_S49,       // sum over neighbour pairs of C(W(v,x)-1, 2)
  A_S62,       // sum over neighbour pairs of D(v,x)
  A_S64,       // sum over diamonds with chord at u of (W(v,x)-2)
  A_S68,       // sum over v in N(u) of 4-cycles through u inside N(v)
  A_S69X4,     // 4 * (4-cycles inside N(u))
  A_DM4,       // DM4(u)  (stored for the next neighbour round)
  A_DM9,       // DM9(u)
  A_DM12,      // DM12(u)
  A_DM14,      // DM14(u)
  A_S15,       // sum DM4(v)
  A_S27,       // sum DM9(v)
  A_S56,       // sum DM14(v)
  A_WORK,      // root work estimate sum_{v in N(u)} d(v) (scheduling)
  A_TSRC,      // DAG triangles with u as the source (u precedes both others)
  NACC
};

// per-slot arrays (slot s = position of v in row u of the CSR, 0..2m-1)
struct SlotArrays {
  u32* T;        // T(u,v)
  u64* E5;       // C4(u,v)
  u64* E7;       // sum_{x in T(u,v)} (d(x)-2)
  u64* E9;       // E9<u,v> = sum_{x in T(u,v)} (T(u,x)-1)
  u64* K4;       // K4(u,v) = E11
  u64* b49;      // root u's share of DM49 for centre v
  u64* b62;      // root u's share of DM62 for centre v
  u64* b64;      // root u's share of DM64 for chord end v
  u64* b68;      // 4-cycles through v inside N(u)
  u64* bc5;      // root u's 5-cycle credits for v
  u32* Mmid;     // triangles on (u,v) whose third vertex lies between u and v
  u32* Mtop;     // triangles on (u,v) whose third vertex follows both
};

struct Graph {
  u32 n;
  u64 S;                 // 2m slots
  const u32* rowptr;     // n+1
  const u32* col;        // S
  u32* deg;              // n
  u32* rev;              // S: slot of (v,u) for slot (u,v)
  unsigned char* sin;    // S: 1 if slot (u,v) is an in-edge of u in the DAG (v precedes u)
  u32* dag_ptr;          // n+1: out-neighbours (u -> v iff u precedes v)
  u32* dag_col;          // m
  u32* dag_slot;         // m: CSR slot of each DAG edge (in the source row)
  u64* tl_ptr;           // S+1: triangle-list offsets per slot
  u32* tl;               // per slot (u,v): slots (u,x) for x in N(u)^N(v), ascending x
  u32* tlv;              // the vertex ids x of the same entries
};

// device helpers ------------------------------------------------------------
// per-warp segmented sum over runs of equal `key` (non-decreasing across the
// lanes, 0xffffffff for idle lanes); returns the run total on the run's last
// lane and sets *is_tail there.
__device__ __forceinline__ u64 seg_sum(u32 key, u64 val, bool* is_tail) {
  const int lane = threadIdx.x & 31;
  const u32 prev = __shfl_up_sync(0xffffffffu, key, 1);
  const u32 heads = __ballot_sync(0xffffffffu, lane == 0 || prev != key);
  const u32 upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
  const int start = 31 - __clz(heads & upto);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u64 y = __shfl_up_sync(0xffffffffu, val, o);
    if (lane - o >= start) val += y;
  }
  *is_tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
  return val;
}

__device__ __forceinline__ bool prec(const u32* deg, u32 i, u32 j) {
  u32 di = deg[i], dj = deg[j];
  return di < dj || (di == dj && i < j);
}

__device__ __forceinline__ u64 c2(long long x) {
  if (x < 2) return 0;
  unsigned __int128 p = (unsigned __int128)x * (unsigned __int128)(x - 1);
  return (u64)(p >> 1);
}
__device__ __forceinline__ u64 c3(long long x) {
  if (x < 3) return 0;
  unsigned __int128 p = (unsigned __int128)x * (unsigned __int128)(x - 1) * (unsigned __int128)(x - 2);
  return (u64)(p / 6);
}
__device__ __forceinline__ u64 c4(long long x) {
  if (x < 4) return 0;
  unsigned __int128 p = (unsigned __int128)x * (unsigned __int128)(x - 1);
  p = p * (unsigned __int128)(x - 2);
  p = p / 6;
  p = p * (unsigned __int128)(x - 3);
  return (u64)(p / 4);
}
// binomial of a count that may already exceed 2^32 (e.g. C(DM1, 2))
__device__ __forceinline__ u64 c2u(u64 x) {
  if ((long long)x < 2) return 0;
  unsigned __int128 p = (unsigned __int128)x * (unsigned __int128)(x - 1);
  return (u64)(p >> 1);
}

// first index i in [lo, hi) with a[i] >= key
__device__ __forceinline__ u32 lower_bound_u32(const u32* a, u32 lo, u32 hi, u32 key) {
  while (lo < hi) {
    u32 mid = lo + ((hi - lo) >> 1);
    if (a[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ bool contains_u32(const u32* a, u32 lo, u32 hi, u32 key) {
  u32 p = lower_bound_u32(a, lo, hi, key);
  return p < hi && a[p] == key;
}

__device__ __forceinline__ u64 warp_sum(u64 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// status word bits written by kernels (read back by the host)
enum DeviceStatus : int {
  ST_OK = 0,
  ST_NOT_SIMPLE = 1,   // unsorted row, duplicate, self-loop or asymmetric edge
  ST_RANGE = 2,        // vertex id >= n
};

// launchers (one per kernel family), all asynchronous on `st`
void launch_degrees(const Graph& g, cudaStream_t st);
void launch_rev_validate(const Graph& g, int* status, cudaStream_t st);
void launch_dag(const Graph& g, u32* tmp_counts, void* scan_tmp, cudaStream_t st);
void launch_scan_u32_to_u64(const u32* in, u64* out, u64 count, void* tmp, cudaStream_t st);
size_t scan_tmp_bytes(u64 count);
void launch_scan_u32_inplace(u32* data, u64 count, void* tmp, cudaStream_t st);
void launch_tri_count(const Graph& g, u32* T, cudaStream_t st);
void launch_tri_fill(const Graph& g, const u32* T, cudaStream_t st);
void launch_tri_edge(const Graph& g, const SlotArrays& sa, cudaStream_t st);
void launch_vsum1(const Graph& g, const SlotArrays& sa, u64* acc, cudaStream_t st);
void launch_tri_opp1(const Graph& g, const SlotArrays& sa, u64* acc, cudaStream_t st);
// A CTA's dense 2-hop map, one entry per vertex id (within a component for
// batches), split by access frequency: every wedge touches the 16-byte hot
// record; only vertices on the root's directed 3-paths touch the cold one.
struct __align__(16) MapHot {
  u32 W;      // |N(root) ^ N(x)| in bits 0..29; bit 31: x ~ root; bit 30: cold record in use
  u32 Wn;     // wedges root-v-x not in-in at v (not root->v<-x)
  u32 D;      // diamonds with root and x off the chord (x > root only)
  u32 P;      // directed 3-paths root <- k -> j -> x
};
struct __align__(32) MapCold {
  u32 X;      // sum over k in N-(root)^N-(x) of #(k -> y -> x)
  u32 pad;
  u64 RY;     // (|N-(root)^N-(x)| << 32) | sum over those k of #(k -> x -> y, k -> y)
  u64 Pjl;    // 3-paths root <- k -> j -> x with j ~ root
  u64 Z;      // sum of Wn over N+(x)
};

struct RootScratch {
  MapHot* hot;   // per CTA: map_n records, zero between roots
  MapCold* cold; // per CTA: map_n records, zero between roots
  int* overflow; // set if a 32-bit 3-path count would wrap
  const u32* comp_base;  // optional [n]: first id of each vertex's component (batches)
  u32 map_n;     // records per CTA: n, or the largest component of a batch
  u32 map_stride;  // records between two CTAs' maps (root_map_stride(map_n))
  int threads;   // 64, 128, 256 or 512 threads per CTA
  u32* touched;  // per CTA: n, ids touched by the current root
  u32* jlist;    // per CTA: n, middle vertices of the current root's 3-paths
  u32* order;    // n: roots in schedule order
  u32* head;     // 1: queue head
  u32* bucket_cnt;  // 64
  u64* tsrc;     // n: DAG triangles with the vertex as source
  u64* prof;     // optional [8]: cycles per phase (summed over roots)
  u64* cycles;   // optional [n]: cycles per root
  u64* cta_end;  // optional [ctas]: global timer (ns) when each CTA ran out of roots
  int ctas;
  u32 chunk;     // roots a CTA takes from the queue at a time (1: one by one)
  u32 smem_recs; // hot records of ids [0, smem_recs) kept in shared memory (set at launch)
};
// per-CTA record stride: at least map_n, an odd number of 128-byte lines of
// hot records, so that the CTAs' records of one vertex do not sit a power
// of two apart (and on the same L2 slice)
u32 root_map_stride(u32 map_n);
size_t root_scratch_bytes(u32 map_stride, int ctas);
void launch_schedule(const Graph& g, u64* acc, RootScratch& rs, cudaStream_t st);
// roots grouped by their highest-degree neighbour (cnt: scratch of n entries)
void launch_hub_schedule(const Graph& g, RootScratch& rs, u32* cnt, void* scan_tmp,
                         cudaStream_t st);
void launch_root_with_pref(const Graph& g, const SlotArrays& sa, u64* acc, RootScratch& rs,
                           u32* pref, u32 pref_stride, cudaStream_t st);
void root_configure();  // host-side set-up (kernel attributes)
void link_configure();  // host-side set-up (kernel attributes)
void launch_link(const Graph& g, const SlotArrays& sa, u32* scratch, u32 warps, u32 dmax,
                 cudaStream_t st);
struct K5Config {
  size_t smem;
  u32 smax;
  u32 blocks;
};
K5Config k5_configure(u32 max_outdeg);  // host-side set-up (kernel attributes)
void launch_k5(const Graph& g, u64* acc, const K5Config& c, cudaStream_t st);
void launch_k4_known(const Graph& g, const SlotArrays& sa, u64* acc, u64 total, cudaStream_t st);
void launch_union_csr(const u32* rowptr_cat, const u32* col_cat, const long long* vtx_off,
                      const long long* edge_off, u32 G, u32 n, u64 S, u32* rowptr, u32* col,
                      u32* comp_base, cudaStream_t st);
// Largest vertex degree accepted.  The per-pair records of the root pass keep
// 32-bit counts whose bounds follow from the degree d: W <= d, D <= C(W, 2)
// and the 3-path sums Y, X <= d^2 all stay below 2^32 for d <= 65,535 (the
// per-pair 3-path count P has its own overflow flag).
constexpr u32 kMaxDegree = 65535;
// relabelling by decreasing degree (single graphs)
constexpr u32 kRelabelMaxDegree = 32768;  // longest row the block sort holds in shared memory
u32 relabel_prepare(const u32* rowptr, u32 n, u32 dmax, u32* hist, u32* new_id, u32* old_of,
                    u32* new_deg, cudaStream_t st);
void relabel_build(const u32* rowptr, const u32* col, const u32* new_id, const u32* old_of,
                   const u32* nrow, u32* ncol, u32 n, u32 long_rows, u32 dmax, cudaStream_t st);
void relabel_configure(u32 dmax);
void launch_orig_slot(const u32* rowptr, const u32* col, const u32* old_of, const u32* nrow,
                      const u32* ncol, u32 n, u32* orig, cudaStream_t st);
void launch_max_component(const long long* vtx_off, u32 G, u32* out, cudaStream_t st);
void launch_tri_opp2(const Graph& g, const SlotArrays& sa, u64* acc, cudaStream_t st);
void launch_vsum2(const Graph& g, const SlotArrays& sa, u64* acc, cudaStream_t st);
void launch_vsum3(const Graph& g, u64* acc, cudaStream_t st);
int upload_transform(const long long* A73x73);
// orbits: 73 (out is n x 73) or 15 (the 4-vertex orbits 0..14 only, out n x 15)
// induced = false writes the non-induced counts DM (A^-1 not applied)
void launch_finalize(const Graph& g, const u64* acc, long long* out, const u32* old_of,
                     int orbits, bool induced, cudaStream_t st);
void launch_column_sums(const long long* counts, u64 rows, int K, u64* sums, int sms,
                        cudaStream_t st);
void launch_vsum2_four(const Graph& g, const SlotArrays& sa, u64* acc, cudaStream_t st);
void launch_edge_orbits12(const Graph& g, const SlotArrays& sa, const u64* acc, long long* out,
                          const u32* orig, cudaStream_t st);
// learned work model
int mlp_param_count();
void launch_features(const Graph& g, const u64* acc, float* X, cudaStream_t st);
void launch_mlp_forward(const float* X, u32 N, const float* params, float* y, cudaStream_t st);
void launch_mlp_grad(const float* X, const float* T, const u32* idx, u32 lo, u32 cnt,
                     const float* params, float* grad, float* loss, cudaStream_t st);
void launch_adam(float* params, const float* grad, float* state, float lr, int step,
                 cudaStream_t st);
void launch_priority_schedule(const float* y, u32 n, u32* bucket_cnt, u32* head, u32* order,
                              cudaStream_t st);
