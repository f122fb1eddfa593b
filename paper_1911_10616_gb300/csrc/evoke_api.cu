// C ABI of libevoke and the host-side orchestration of the orbit-counting
// pass sequence (see include/evoke.h for the contract of every entry point).
//
// The matrix A of App. A (non-induced = A * induced) is derived here at load
// time from the thirty patterns of Fig. node_orbits: A[i][j] is the number of
// connected spanning subgraphs of pattern H(j) in which a vertex of orbit j
// plays orbit i.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "evoke_internal.cuh"
#include "../../include/evoke.h"

namespace {

// ---- patterns of Fig. node_orbits ------------------------------------------
// vertices 0-based in drawing order; `orb` gives the printed orbit number of
// one vertex per orbit (-1 elsewhere); the rest follow by automorphism.
struct Pat {
  int k;
  int ne;
  int e[10][2];
  int orb[5];
};

const Pat kPat[30] = {
    {2, 1, {{0, 1}}, {-1, 0, -1, -1, -1}},
    {3, 2, {{0, 1}, {1, 2}}, {-1, 2, 1, -1, -1}},
    {3, 3, {{0, 1}, {0, 2}, {1, 2}}, {-1, -1, 3, -1, -1}},
    {4, 3, {{0, 1}, {1, 2}, {2, 3}}, {-1, -1, 5, 4, -1}},
    {4, 3, {{0, 2}, {1, 2}, {2, 3}}, {-1, -1, 7, 6, -1}},
    {4, 4, {{0, 1}, {0, 2}, {1, 3}, {2, 3}}, {-1, -1, 8, -1, -1}},
    {4, 4, {{0, 1}, {1, 2}, {1, 3}, {2, 3}}, {9, 11, 10, -1, -1}},
    {4, 5, {{0, 1}, {0, 2}, {0, 3}, {1, 3}, {2, 3}}, {-1, 12, -1, 13, -1}},
    {4, 6, {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}}, {-1, -1, -1, 14, -1}},
    {5, 4, {{0, 1}, {1, 2}, {2, 3}, {3, 4}}, {-1, -1, 17, 16, 15}},
    {5, 4, {{0, 2}, {1, 2}, {2, 3}, {3, 4}}, {19, -1, 21, 20, 18}},
    {5, 4, {{0, 2}, {1, 2}, {2, 3}, {2, 4}}, {-1, -1, 23, -1, 22}},
    {5, 5, {{0, 2}, {1, 3}, {2, 3}, {2, 4}, {3, 4}}, {24, -1, 26, -1, 25}},
    {5, 5, {{0, 1}, {0, 2}, {1, 2}, {2, 3}, {3, 4}}, {29, -1, 30, 28, 27}},
    {5, 5, {{0, 2}, {1, 2}, {2, 3}, {2, 4}, {3, 4}}, {31, -1, 33, 32, -1}},
    {5, 5, {{0, 1}, {0, 2}, {1, 3}, {2, 4}, {3, 4}}, {-1, -1, -1, -1, 34}},
    {5, 5, {{0, 1}, {1, 2}, {1, 3}, {2, 4}, {3, 4}}, {35, 38, 37, -1, 36}},
    {5, 6, {{0, 1}, {1, 2}, {1, 3}, {1, 4}, {2, 4}, {3, 4}}, {39, 42, 40, -1, 41}},
    {5, 6, {{0, 1}, {0, 2}, {1, 2}, {2, 3}, {2, 4}, {3, 4}}, {-1, -1, 44, 43, -1}},
    {5, 6, {{0, 1}, {1, 2}, {1, 3}, {2, 3}, {2, 4}, {3, 4}}, {45, 47, 48, -1, 46}},
    {5, 6, {{0, 1}, {0, 2}, {0, 3}, {1, 4}, {2, 4}, {3, 4}}, {50, 49, -1, -1, -1}},
    {5, 6, {{0, 1}, {0, 2}, {1, 3}, {2, 3}, {2, 4}, {3, 4}}, {51, -1, 53, -1, 52}},
    {5, 7, {{0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}, {2, 4}, {3, 4}}, {54, -1, 55, -1, -1}},
    {5, 7, {{0, 1}, {1, 2}, {1, 3}, {1, 4}, {2, 3}, {2, 4}, {3, 4}}, {56, 58, 57, -1, -1}},
    {5, 7, {{0, 1}, {0, 2}, {1, 2}, {1, 3}, {2, 3}, {2, 4}, {3, 4}}, {59, 60, 61, -1, -1}},
    {5, 7, {{0, 1}, {0, 2}, {0, 3}, {1, 4}, {2, 3}, {2, 4}, {3, 4}}, {-1, 62, 64, -1, 63}},
    {5, 8, {{0, 1}, {0, 2}, {1, 2}, {1, 3}, {1, 4}, {2, 3}, {2, 4}, {3, 4}}, {65, -1, 67, -1, 66}},
    {5, 8, {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 4}, {2, 3}, {2, 4}, {3, 4}}, {-1, -1, 69, 68, -1}},
    {5, 9, {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {1, 4}, {2, 3}, {2, 4}, {3, 4}},
     {70, -1, -1, 71, -1}},
    {5, 10, {{0, 1}, {0, 2}, {0, 3}, {0, 4}, {1, 2}, {1, 3}, {1, 4}, {2, 3}, {2, 4}, {3, 4}},
     {-1, -1, -1, -1, 72}},
};

using Adj = unsigned;  // bit a*5+b set for every ordered adjacent pair

Adj adj_of_edges(const int (*e)[2], int ne, unsigned edge_mask = ~0u) {
  Adj m = 0;
  for (int i = 0; i < ne; ++i)
    if (edge_mask >> i & 1u) m |= (1u << (e[i][0] * 5 + e[i][1])) | (1u << (e[i][1] * 5 + e[i][0]));
  return m;
}
Adj permute(Adj m, const int* p, int k) {
  Adj r = 0;
  for (int a = 0; a < k; ++a)
    for (int b = 0; b < k; ++b)
      if (m >> (a * 5 + b) & 1u) r |= 1u << (p[a] * 5 + p[b]);
  return r;
}
bool spans_connected(Adj m, int k) {
  unsigned reach = 1;
  for (int it = 0; it < k; ++it)
    for (int a = 0; a < k; ++a)
      if (reach >> a & 1u)
        for (int b = 0; b < k; ++b)
          if (m >> (a * 5 + b) & 1u) reach |= 1u << b;
  return reach == (1u << k) - 1u;
}

struct Derived {
  bool ok = false;
  long long A[73 * 73] = {};
  int orbit_pattern[73] = {};  // pattern owning each orbit
  int orbit_size[73] = {};     // vertices of the pattern in the orbit
};

Derived derive() {
  Derived out;
  int full_orb[30][5];
  Adj pat_adj[30];
  for (int j = 0; j < 30; ++j) {
    const Pat& P = kPat[j];
    pat_adj[j] = adj_of_edges(P.e, P.ne);
    for (int a = 0; a < 5; ++a) full_orb[j][a] = P.orb[a];
    // spread each printed label over its automorphism class
    int p[5] = {0, 1, 2, 3, 4};
    bool changed = true;
    while (changed) {
      changed = false;
      std::sort(p, p + P.k);
      do {
        if (permute(pat_adj[j], p, P.k) != pat_adj[j]) continue;
        for (int a = 0; a < P.k; ++a) {
          const int x = full_orb[j][a], y = full_orb[j][p[a]];
          if (x >= 0 && y < 0) { full_orb[j][p[a]] = x; changed = true; }
          if (x >= 0 && y >= 0 && x != y) return out;
        }
      } while (std::next_permutation(p, p + P.k));
    }
    for (int a = 0; a < P.k; ++a) {
      if (full_orb[j][a] < 0) return out;
      out.orbit_pattern[full_orb[j][a]] = j;
      out.orbit_size[full_orb[j][a]]++;
    }
  }
  // A: connected spanning edge subsets of each pattern
  for (int j = 0; j < 30; ++j) {
    const Pat& P = kPat[j];
    for (int v = 0; v < P.k; ++v) {
      for (unsigned sub = 1; sub < (1u << P.ne); ++sub) {
        const Adj m = adj_of_edges(P.e, P.ne, sub);
        if (!spans_connected(m, P.k)) continue;
        const int ecount = __builtin_popcount(sub);
        int hit = -1;
        for (int i = 0; i < 30 && hit < 0; ++i) {
          if (kPat[i].k != P.k || kPat[i].ne != ecount) continue;
          int p[5] = {0, 1, 2, 3, 4};
          do {
            if (permute(m, p, P.k) == pat_adj[i]) { hit = full_orb[i][p[v]]; break; }
          } while (std::next_permutation(p, p + P.k));
        }
        if (hit < 0) return out;
        out.A[hit * 73 + full_orb[j][v]] += 1;  // summed over the orbit's vertices
      }
    }
    // each column was accumulated once per vertex of its orbit
    int cls_size[73] = {};
    for (int v = 0; v < P.k; ++v) cls_size[full_orb[j][v]]++;
    for (int v = 0; v < P.k; ++v) {
      const int o = full_orb[j][v];
      if (cls_size[o] <= 0) continue;
      for (int i = 0; i < 73; ++i) {
        if (out.A[i * 73 + o] % cls_size[o]) return out;
        out.A[i * 73 + o] /= cls_size[o];
      }
      cls_size[o] = -cls_size[o];  // normalised
    }
  }
  out.ok = true;
  return out;
}

const Derived& derived() {
  static const Derived d = derive();
  return d;
}

// ---- phase profiling -------------------------------------------------------
struct PhaseRec {
  const char* name;
  int launches;
  cudaEvent_t a, b;
};
struct PhaseAgg {
  char name[24];
  int launches = 0;
  int calls = 0;
  double ms = 0;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<PhaseRec> g_pending;
std::vector<PhaseAgg> g_agg;
unsigned long long g_launches = 0;

// Runs `fn` (which enqueues `launches` kernels on `st`) as one named phase.
bool debug_sync() {
  static const bool on = [] {
    const char* e = getenv("EVOKE_SYNC_CHECK");
    return e && *e && *e != '0';
  }();
  return on;
}

template <typename F>
void phase(const char* name, int launches, cudaStream_t st, F&& fn) {
  if (debug_sync()) {
    fn();
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e1 != cudaSuccess || e2 != cudaSuccess)
      fprintf(stderr, "evoke: phase %s failed: launch=%s sync=%s\n", name,
              cudaGetErrorString(e1), cudaGetErrorString(e2));
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_launches += (unsigned long long)launches;
    return;
  }
  bool on;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    on = g_prof_on;
    g_launches += (unsigned long long)launches;
  }
  if (!on) {
    fn();
    return;
  }
  PhaseRec r{name, launches, nullptr, nullptr};
  cudaEventCreate(&r.a);
  cudaEventCreate(&r.b);
  cudaEventRecord(r.a, st);
  fn();
  cudaEventRecord(r.b, st);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_pending.push_back(r);
}

void drain_pending() {
  for (PhaseRec& r : g_pending) {
    float ms = 0;
    cudaEventSynchronize(r.b);
    cudaEventElapsedTime(&ms, r.a, r.b);
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
    PhaseAgg* agg = nullptr;
    for (PhaseAgg& x : g_agg)
      if (!strncmp(x.name, r.name, sizeof(x.name) - 1)) agg = &x;
    if (!agg) {
      g_agg.emplace_back();
      agg = &g_agg.back();
      strncpy(agg->name, r.name, sizeof(agg->name) - 1);
      agg->name[sizeof(agg->name) - 1] = 0;
    }
    agg->launches += r.launches;
    agg->calls += 1;
    agg->ms += ms;
  }
  g_pending.clear();
}

std::mutex g_upload_mu;
int g_uploaded_device = -1;

int ensure_transform() {
  const Derived& d = derived();
  if (!d.ok) return EVOKE_ECUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return EVOKE_ECUDA;
  std::lock_guard<std::mutex> lk(g_upload_mu);
  if (g_uploaded_device == dev) return EVOKE_OK;
  if (upload_transform(d.A) < 0) return EVOKE_ECUDA;
  g_uploaded_device = dev;
  return EVOKE_OK;
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// Device memory comes from a pool private to the library, one per device,
// whose release threshold is unlimited: the blocks of a finished call stay
// reserved for the next one instead of being unmapped at every stream
// synchronisation (a 1M-vertex plan holds tens of GB).
cudaMemPool_t library_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = p;
  }
  return pools[dev];
}
template <class T>
cudaError_t dmalloc(T** ptr, size_t bytes, cudaStream_t st) {
  cudaMemPool_t p = library_pool();
  void* v = nullptr;
  const cudaError_t e = p ? cudaMallocFromPoolAsync(&v, bytes, p, st) : cudaMallocAsync(&v, bytes, st);
  *ptr = static_cast<T*>(v);
  return e;
}

// a bump allocator over one cudaMallocAsync block
struct Arena {
  char* base = nullptr;
  size_t cap = 0, used = 0;
  cudaStream_t st = nullptr;
  bool overflow = false;
  template <typename T>
  T* take(size_t count) {
    size_t off = (used + 255) & ~size_t(255);
    size_t end = off + std::max<size_t>(count, 1) * sizeof(T);
    if (end > cap) {
      overflow = true;
      return nullptr;
    }
    used = end;
    return reinterpret_cast<T*>(base + off);
  }
};
template <typename T>
size_t sz(size_t count) {
  return ((std::max<size_t>(count, 1) * sizeof(T)) + 255) & ~size_t(255);
}

// out[0] = max degree, out[1] = max DAG out-degree
__global__ void dmax_kernel(const u32* deg, const u32* dag_ptr, u32 n, u32* out) {
  u32 u = blockIdx.x * blockDim.x + threadIdx.x;
  u32 v = u < n ? deg[u] : 0;
  u32 w = u < n ? dag_ptr[u + 1] - dag_ptr[u] : 0;
  for (int o = 16; o > 0; o >>= 1) {
    v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    w = max(w, __shfl_xor_sync(0xffffffffu, w, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (v) atomicMax(out, v);
    if (w) atomicMax(out + 1, w);
  }
}

__global__ void degree_max_kernel(const u32* rowptr, u32 n, u32* out) {
  const u32 u = blockIdx.x * blockDim.x + threadIdx.x;
  u32 v = u < n ? rowptr[u + 1] - rowptr[u] : 0;
  const u32 l = (u < n && v > 1024u) ? 1u : 0u;
  u32 c = l;
  for (int o = 16; o > 0; o >>= 1) {
    v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (v) atomicMax(out, v);
    if (c) atomicAdd(out + 1, c);
  }
}
template <typename T>
__global__ void unpermute_rows_kernel(const T* in, T* out, const u32* old_of, u32 n, u32 width) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (u64)n * width) return;
  const u32 r = (u32)(i / width), k = (u32)(i % width);
  out[(u64)old_of[r] * width + k] = in[i];
}
__global__ void unpermute_slots_kernel(const long long* in, long long* out, const u32* orig, u64 S) {
  const u64 s = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < S) out[orig[s]] = in[s];
}

__global__ void widen_kernel(const u32* in, long long* out, u64 count) {
  u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = in[i];
}
__global__ void copy_i64_kernel(const u64* in, long long* out, u64 count) {
  u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = (long long)in[i];
}

// ---------------------------------------------------------------------------
// Plans.  A plan owns every device buffer the pass sequence needs for one
// input (one graph, or one batch of graphs as their disjoint union).  Creating
// it runs the sizing passes (DAG, triangle counts) and synchronises the
// stream; executing it enqueues the whole pass sequence, from the CSR to the
// int64[n x 73] counts, with no host synchronisation (so it can be captured
// into a CUDA graph and replayed).
// ---------------------------------------------------------------------------
struct Config {
  int root_threads = 0;   // 0: 512 for single graphs, 64 for batches of small graphs
  bool tunable = true;    // false: one-shot call, no later set_tuning
  int root_ctas = 0;      // 0: 2 per SM (512 threads) / 4 per SM (256)
  u32 link_warps = 0;     // 0: 64 per SM
  int orbits = 73;        // 73, or 15: the 4-vertex orbits only
  bool induced = true;    // false: write the non-induced counts DM
  int schedule = 0;       // 0: degree-bucket; 1: grouped by highest-degree neighbour
  u32 chunk = 8;          // roots per queue grab under schedule 1
};

// evoke_opts.orbits: 0 or 73 -> all orbits, 15 -> orbits 0..14; else -1
int opts_orbits(const evoke_opts* o) {
  if (!o || o->orbits == 0 || o->orbits == 73) return 73;
  return o->orbits == 15 ? 15 : -1;
}

}  // namespace

struct evoke_plan {
  // input
  const u32* rowptr = nullptr;
  const u32* col = nullptr;
  u32 n = 0;
  u64 m = 0;
  // batch input (the union CSR below is rebuilt from it on every execution)
  bool batch = false;
  const u32* rowptr_cat = nullptr;
  const u32* col_cat = nullptr;
  const long long* vtx_off = nullptr;
  const long long* edge_off = nullptr;
  u32 G = 0;
  u32 max_comp = 0;
  // sizes
  u32 dmax = 0, max_outdeg = 0;
  u64 ntri_entries = 0;
  Config cfg;
  K5Config k5{};
  // device memory
  void* block = nullptr;
  size_t bytes = 0;
  void* block2 = nullptr;
  size_t bytes2 = 0;
  Graph g{};
  SlotArrays sa{};
  u64* acc = nullptr;
  RootScratch rs{};
  u32* pref = nullptr;
  u32 pref_stride = 0;
  u32* link_scratch = nullptr;
  u32* cnt = nullptr;
  void* scan_tmp = nullptr;
  int* status = nullptr;
  u32* misc = nullptr;
  u32* union_rowptr = nullptr;
  u32* union_col = nullptr;
  u32* comp_base = nullptr;
  // relabelling by decreasing degree (single graphs): the passes run on the
  // relabelled CSR; outputs are mapped back to the caller's ids
  bool relabel = false;
  const u32* in_rowptr = nullptr;
  const u32* in_col = nullptr;
  u32* rl_new_id = nullptr;
  u32* rl_old_of = nullptr;
  u32* rl_rowptr = nullptr;
  u32* rl_col = nullptr;
  u32* rl_hist = nullptr;
  u32 rl_dmax = 0;
  u32 rl_long_rows = 0;
  void* rl_block = nullptr;
  cudaStream_t st = nullptr;
  int launches_per_exec = 0;
  int ctas_alloc = 0;     // CTAs the root maps were allocated for
  // learned schedule
  const float* model = nullptr;  // device, 1249 floats
  float* feat = nullptr;         // n x 4
  float* prio = nullptr;         // n
  void* model_block = nullptr;
  // CUDA graph of one execution
  cudaGraphExec_t gexec = nullptr;
  long long* gexec_out = nullptr;
};

namespace {

int sm_count_cached() { return sm_count(); }

int check_csr(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
              cudaStream_t st) {
  if (n == 0xffffffffu || 2 * m >= 0xffffffffull) return EVOKE_ERANGE;
  if (!rowptr) return EVOKE_EINVAL;
  if (m > 0 && !colidx) return EVOKE_EINVAL;
  uint32_t last = 0;
  if (cudaMemcpyAsync(&last, rowptr + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) !=
      cudaSuccess)
    return EVOKE_EINVAL;
  if (cudaStreamSynchronize(st) != cudaSuccess) return EVOKE_ECUDA;
  if ((uint64_t)last != 2 * m) return EVOKE_EINVAL;
  return EVOKE_OK;
}

void apply_config(evoke_plan* P, u32 map_n) {
  const int sms = sm_count_cached();
  const int t = P->cfg.root_threads ? P->cfg.root_threads : (P->batch ? 64 : 512);
  P->rs.threads = (t == 64 || t == 128 || t == 256 || t == 1024) ? t : 512;
  P->rs.ctas = P->cfg.root_ctas > 0 ? P->cfg.root_ctas : sms * (1024 / P->rs.threads);
  // maps for up to 16 (small maps) or 4 CTAs per SM when that is cheap, so
  // that tuning can raise the CTA count later
  const size_t per_cta =
      (size_t)root_map_stride(map_n) * (sizeof(MapHot) + sizeof(MapCold) + 2 * sizeof(u32));
  P->ctas_alloc = P->rs.ctas;
  if (!P->cfg.tunable) return;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = (size_t)4 << 30;
  const size_t budget = std::min<size_t>(free_b / 3, (size_t)64 << 30);
  for (int per_sm : {16, 8, 4})
    if ((size_t)sms * per_sm * per_cta <= budget) {
      P->ctas_alloc = std::max(P->ctas_alloc, sms * per_sm);
      break;
    }
}

// the CSR invariants of the caller's graph (simple, symmetric, sorted rows)
int validate_csr(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
                 cudaStream_t st) {
  if (!n) return EVOKE_OK;
  const u64 S = 2 * m;
  size_t bytes = sz<u32>(S) + sz<int>(4);
  void* blk = nullptr;
  if (dmalloc(&blk, bytes, st) != cudaSuccess) return EVOKE_ENOMEM;
  Graph g{};
  g.n = n;
  g.S = S;
  g.rowptr = rowptr;
  g.col = colidx;
  g.rev = static_cast<u32*>(blk);
  int* status = reinterpret_cast<int*>(static_cast<char*>(blk) + sz<u32>(S));
  cudaMemsetAsync(status, 0, sizeof(int), st);
  launch_rev_validate(g, status, st);
  int h = 0;
  cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(blk, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return EVOKE_ECUDA;
  if (h & ST_RANGE) return EVOKE_ERANGE;
  if (h & ST_NOT_SIMPLE) return EVOKE_ENOTSIMPLE;
  return EVOKE_OK;
}

bool relabel_wanted() {
  const char* e = getenv("EVOKE_NO_RELABEL");
  return !(e && *e && *e != '0');
}

void relabel_run(evoke_plan* P, cudaStream_t st) {
  relabel_prepare(P->in_rowptr, P->n, P->rl_dmax, P->rl_hist, P->rl_new_id, P->rl_old_of,
                  P->rl_rowptr, st);
  launch_scan_u32_inplace(P->rl_rowptr, P->n, P->scan_tmp, st);
  relabel_build(P->in_rowptr, P->in_col, P->rl_new_id, P->rl_old_of, P->rl_rowptr, P->rl_col, P->n,
                P->rl_long_rows, P->rl_dmax, st);
}

// decide on relabelling and allocate its buffers (single graphs)
int plan_relabel_setup(evoke_plan* P) {
  if (P->batch || !relabel_wanted() || P->n < 2) return EVOKE_OK;
  cudaStream_t st = P->st;
  u32* d = nullptr;
  if (dmalloc(&d, 2 * sizeof(u32), st) != cudaSuccess) return EVOKE_ENOMEM;
  cudaMemsetAsync(d, 0, 2 * sizeof(u32), st);
  degree_max_kernel<<<(P->n + 255) / 256, 256, 0, st>>>(P->rowptr, P->n, d);
  u32 h[2] = {0, 0};
  cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return EVOKE_ECUDA;
  if (h[0] > kRelabelMaxDegree) return EVOKE_OK;  // rows too long for the in-place sort
  const u64 S = 2 * P->m;
  size_t bytes = 3 * sz<u32>(P->n + 1) + sz<u32>(S) + sz<u32>(h[0] + 1);
  if (dmalloc(&P->rl_block, bytes, st) != cudaSuccess) return EVOKE_ENOMEM;
  Arena ar{static_cast<char*>(P->rl_block), bytes, 0, st};
  P->rl_new_id = ar.take<u32>(P->n + 1);
  P->rl_old_of = ar.take<u32>(P->n + 1);
  P->rl_rowptr = ar.take<u32>(P->n + 1);
  P->rl_col = ar.take<u32>(S);
  P->rl_hist = ar.take<u32>(h[0] + 1);
  if (ar.overflow) return EVOKE_ENOMEM;
  P->rl_dmax = h[0];
  P->rl_long_rows = h[1];
  relabel_configure(h[0]);
  P->in_rowptr = P->rowptr;
  P->in_col = P->col;
  P->rowptr = P->rl_rowptr;
  P->col = P->rl_col;
  P->relabel = true;
  return EVOKE_OK;
}

// stage 1 buffers (graph-sized) and the sizing passes
int plan_stage1(evoke_plan* P, bool validate) {
  cudaStream_t st = P->st;
  const u32 n = P->n;
  const u64 m = P->m, S = 2 * m;
  size_t bytes = sz<u32>(n) + sz<u32>(S) + sz<u32>(n + 1) + 2 * sz<u32>(m) + sz<u32>(n) +
                 sz<char>(scan_tmp_bytes(std::max<u64>(S, n) + 1)) + sz<u32>(S) +
                 sz<u64>(S + 1) + sz<int>(4) + sz<u32>(4) + sz<unsigned char>(S);
  if (P->batch) bytes += sz<u32>(n + 1) + sz<u32>(S) + sz<u32>(n);
  if (dmalloc(&P->block, bytes, st) != cudaSuccess) return EVOKE_ENOMEM;
  P->bytes = bytes;
  Arena ar{static_cast<char*>(P->block), bytes, 0, st};
  Graph& g = P->g;
  if (P->batch) {
    P->union_rowptr = ar.take<u32>(n + 1);
    P->union_col = ar.take<u32>(S);
    P->comp_base = ar.take<u32>(n);
    P->rowptr = P->union_rowptr;
    P->col = P->union_col;
  }
  g.n = n;
  g.S = S;
  g.rowptr = P->rowptr;
  g.col = P->col;
  g.deg = ar.take<u32>(n);
  g.rev = ar.take<u32>(S);
  g.sin = ar.take<unsigned char>(S);
  g.dag_ptr = ar.take<u32>(n + 1);
  g.dag_col = ar.take<u32>(m);
  g.dag_slot = ar.take<u32>(m);
  P->cnt = ar.take<u32>(n);
  P->scan_tmp = ar.take<char>(scan_tmp_bytes(std::max<u64>(S, n) + 1));
  P->sa.T = ar.take<u32>(S);
  g.tl_ptr = ar.take<u64>(S + 1);
  P->status = ar.take<int>(4);
  P->misc = ar.take<u32>(4);
  if (ar.overflow) return EVOKE_ENOMEM;
  cudaMemsetAsync(P->status, 0, sizeof(int) * 4, st);
  cudaMemsetAsync(P->misc, 0, sizeof(u32) * 4, st);
  if (P->batch)
    launch_union_csr(P->rowptr_cat, P->col_cat, P->vtx_off, P->edge_off, P->G, n, S,
                     P->union_rowptr, P->union_col, P->comp_base, st);
  if (P->relabel) relabel_run(P, st);
  launch_degrees(g, st);
  launch_rev_validate(g, P->status, st);
  if (validate) {
    int status = 0;
    cudaMemcpyAsync(&status, P->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return EVOKE_ECUDA;
    if (status & ST_RANGE) return EVOKE_ERANGE;
    if (status & ST_NOT_SIMPLE) return EVOKE_ENOTSIMPLE;
  }
  launch_dag(g, P->cnt, P->scan_tmp, st);
  if (n) dmax_kernel<<<(n + 255) / 256, 256, 0, st>>>(g.deg, g.dag_ptr, n, P->misc);
  launch_tri_count(g, P->sa.T, st);
  launch_scan_u32_to_u64(P->sa.T, g.tl_ptr, S, P->scan_tmp, st);
  u64 total = 0;
  u32 mx[2] = {0, 0};
  cudaMemcpyAsync(&total, g.tl_ptr + S, sizeof(u64), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(mx, P->misc, 2 * sizeof(u32), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return EVOKE_ECUDA;
  P->ntri_entries = total;
  P->dmax = mx[0];
  P->max_outdeg = mx[1];
  if (P->dmax > kMaxDegree) return EVOKE_ERANGE;  // 32-bit per-pair counts could wrap
  return EVOKE_OK;
}

// stage 2 buffers: triangle lists, per-slot arrays, accumulators, scratch
int plan_stage2(evoke_plan* P) {
  cudaStream_t st = P->st;
  const u32 n = P->n;
  const u64 S = P->g.S;
  const u32 map_n = P->batch ? std::max<u32>(P->max_comp, 1) : std::max<u32>(n, 1);
  apply_config(P, map_n);
  const int ctas = P->ctas_alloc;
  const u32 dmax = std::max<u32>(P->dmax, 1);
  P->cfg.link_warps = P->cfg.link_warps ? P->cfg.link_warps : (u32)sm_count_cached() * 64;
  P->cfg.link_warps = (P->cfg.link_warps + 7) / 8 * 8;
  const u32 link_warps = P->cfg.link_warps;
  P->pref_stride = dmax + 1;
  const bool root_profile = [] {
    const char* e = getenv("EVOKE_ROOT_PROFILE");
    return e && *e && *e != '0';
  }();
  size_t bytes = 2 * sz<u32>(P->ntri_entries) + 9 * sz<u64>(S) + 2 * sz<u32>(S) + sz<u64>(8) +
                 sz<u64>((size_t)NACC * n) + root_scratch_bytes(root_map_stride(map_n), ctas) + 256 * 8 +
                 sz<u32>(n) + sz<u32>(256) + sz<u32>(4) +
                 sz<u32>((size_t)ctas * P->pref_stride) + sz<u32>((size_t)link_warps * 2 * dmax);
  if (dmalloc(&P->block2, bytes, st) != cudaSuccess) return EVOKE_ENOMEM;
  P->bytes2 = bytes;
  Arena ar{static_cast<char*>(P->block2), bytes, 0, st};
  P->g.tl = ar.take<u32>(P->ntri_entries);
  P->g.tlv = ar.take<u32>(P->ntri_entries);
  SlotArrays& sa = P->sa;
  sa.E5 = ar.take<u64>(S);
  sa.E7 = ar.take<u64>(S);
  sa.E9 = ar.take<u64>(S);
  sa.K4 = ar.take<u64>(S);
  sa.b49 = ar.take<u64>(S);
  sa.b62 = ar.take<u64>(S);
  sa.b64 = ar.take<u64>(S);
  sa.b68 = ar.take<u64>(S);
  sa.bc5 = ar.take<u64>(S);
  sa.Mmid = ar.take<u32>(S);
  sa.Mtop = ar.take<u32>(S);
  P->acc = ar.take<u64>((size_t)NACC * n);
  RootScratch& rs = P->rs;
  rs.map_n = map_n;
  rs.map_stride = root_map_stride(map_n);
  rs.comp_base = P->batch ? P->comp_base : nullptr;
  rs.hot = ar.take<MapHot>((size_t)ctas * rs.map_stride);
  rs.cold = ar.take<MapCold>((size_t)ctas * rs.map_stride);
  rs.overflow = P->status + 1;
  rs.touched = ar.take<u32>((size_t)ctas * rs.map_stride);
  rs.jlist = ar.take<u32>((size_t)ctas * rs.map_stride);
  rs.order = ar.take<u32>(n);
  rs.bucket_cnt = ar.take<u32>(256);
  rs.head = ar.take<u32>(4);
  rs.tsrc = P->acc + (size_t)A_TSRC * n;
  rs.chunk = 1;
  rs.cta_end = nullptr;
  rs.prof = root_profile ? ar.take<u64>(8) : nullptr;
  rs.cycles = nullptr;
  P->pref = ar.take<u32>((size_t)ctas * P->pref_stride);
  P->link_scratch = ar.take<u32>((size_t)link_warps * 2 * dmax);  // counters + partner list
  if (ar.overflow) return EVOKE_ENOMEM;
  // maps and scratch rows are left zeroed by the kernels that use them
  cudaMemsetAsync(P->block2, 0, ar.used, st);
  P->k5 = k5_configure(P->max_outdeg);
  link_configure();
  root_configure();
  return EVOKE_OK;
}

// zero what is accumulated into during one execution
void clear_accumulators(evoke_plan* P, cudaStream_t st) {
  const u64 S = P->g.S;
  const size_t slot_bytes = (char*)(P->sa.Mmid) - (char*)(P->sa.E5);  // E5 .. bc5 contiguous
  cudaMemsetAsync(P->sa.E5, 0, slot_bytes, st);
  cudaMemsetAsync(P->acc, 0, sizeof(u64) * (size_t)NACC * P->n, st);
  cudaMemsetAsync(P->status + 1, 0, sizeof(int), st);  // 32-bit 3-path count overflow flag
  if (P->rs.prof) cudaMemsetAsync(P->rs.prof, 0, sizeof(u64) * 8, st);
  (void)S;
}

// the whole pass sequence; no host synchronisation
void execute(evoke_plan* P, long long* out, cudaStream_t st, bool timed) {
  Graph& g = P->g;
  SlotArrays& sa = P->sa;
  u64* acc = P->acc;
  const u32 n = P->n;
  const u64 S = g.S;
  const int nl = n ? 1 : 0, sl = S ? 1 : 0;
  auto run = [&](const char* name, int launches, auto&& fn) {
    if (timed) phase(name, launches, st, fn);
    else fn();
  };
  run("memset", 0, [&] { clear_accumulators(P, st); });
  if (P->batch)
    run("union_csr", 1 + sl, [&] {
      launch_union_csr(P->rowptr_cat, P->col_cat, P->vtx_off, P->edge_off, P->G, n, S,
                       P->union_rowptr, P->union_col, P->comp_base, st);
    });
  if (P->relabel)
    run("relabel", 6 + (P->rl_long_rows ? 1 : 0) + (n > P->rl_long_rows ? 1 : 0), [&] {
      relabel_run(P, st);
    });
  run("degrees", nl, [&] { launch_degrees(g, st); });
  run("rev", nl, [&] { launch_rev_validate(g, P->status, st); });
  run("dag", n ? 5 : 0, [&] { launch_dag(g, P->cnt, P->scan_tmp, st); });
  run("tri_count", sl, [&] { launch_tri_count(g, sa.T, st); });
  run("tri_scan", S ? 3 : 0, [&] { launch_scan_u32_to_u64(sa.T, g.tl_ptr, S, P->scan_tmp, st); });
  const bool four = P->cfg.orbits == 15;
  run("tri_fill", sl, [&] { launch_tri_fill(g, sa.T, st); });
  run("tri_edge", sl, [&] { launch_tri_edge(g, sa, st); });
  run("vsum1", nl, [&] { launch_vsum1(g, sa, acc, st); });
  run("tri_opp1", nl, [&] { launch_tri_opp1(g, sa, acc, st); });
  run("k4", (P->ntri_entries ? 1 : 0) + sl, [&] { launch_k4_known(g, sa, acc, P->ntri_entries, st); });
  if (P->model) {
    run("model", 2 * nl, [&] {
      launch_features(g, acc, P->feat, st);
      launch_mlp_forward(P->feat, n, P->model, P->prio, st);
    });
    P->rs.chunk = 1;
    run("schedule", 3 * nl, [&] {
      launch_priority_schedule(P->prio, n, P->rs.bucket_cnt, P->rs.head, P->rs.order, st);
    });
  } else if (P->cfg.schedule == 1) {
    P->rs.chunk = P->cfg.chunk;
    run("schedule", n ? 5 : 0, [&] { launch_hub_schedule(g, P->rs, P->cnt, P->scan_tmp, st); });
  } else {
    run("schedule", 3 * nl, [&] { launch_schedule(g, acc, P->rs, st); });
  }
  run("root", nl, [&] {
    launch_root_with_pref(g, sa, acc, P->rs, P->pref, P->pref_stride, st);
  });
  if (four) {
    run("vsum2", nl, [&] { launch_vsum2_four(g, sa, acc, st); });
  } else {
    run("link", sl, [&] {
      launch_link(g, sa, P->link_scratch, P->cfg.link_warps, std::max<u32>(P->dmax, 1), st);
    });
    run("k5", P->k5.blocks ? 1 : 0, [&] { launch_k5(g, acc, P->k5, st); });
    run("tri_opp2", nl, [&] { launch_tri_opp2(g, sa, acc, st); });
    run("vsum2", nl, [&] { launch_vsum2(g, sa, acc, st); });
    run("vsum3", nl, [&] { launch_vsum3(g, acc, st); });
  }
  if (out)
    run("finalize", nl, [&] {
      launch_finalize(g, acc, out, P->relabel ? P->rl_old_of : nullptr, P->cfg.orbits,
                      P->cfg.induced, st);
    });
}

int count_launches(const evoke_plan* P, bool with_out) {
  const int nl = P->n ? 1 : 0, sl = P->g.S ? 1 : 0;
  int k = 0;
  if (P->batch) k += 1 + sl;
  if (P->relabel) k += 6 + (P->rl_long_rows ? 1 : 0) + (P->n > P->rl_long_rows ? 1 : 0);
  const bool four = P->cfg.orbits == 15;
  // degrees, rev, dag, tri_count, tri_scan, tri_fill, tri_edge, vsum1, tri_opp1
  k += nl + nl + (P->n ? 5 : 0) + sl + (P->g.S ? 3 : 0) + sl + sl + nl + nl;
  // k4, schedule, root
  const int sched = (!P->model && P->cfg.schedule == 1) ? (P->n ? 5 : 0) : 3 * nl;
  k += (P->ntri_entries ? 1 : 0) + sl + sched + nl;
  // [link, k5, tri_opp2], vsum2, [vsum3]
  k += four ? nl : sl + (P->k5.blocks ? 1 : 0) + nl + nl + nl;
  if (P->model) k += 2 * nl;
  if (with_out) k += nl;
  return k;
}

void plan_free(evoke_plan* P) {
  if (!P) return;
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  if (P->model_block) cudaFreeAsync(P->model_block, P->st);
  if (P->rl_block) cudaFreeAsync(P->rl_block, P->st);
  if (P->block) cudaFreeAsync(P->block, P->st);
  if (P->block2) cudaFreeAsync(P->block2, P->st);
  cudaStreamSynchronize(P->st);
  delete P;
}

int plan_finish_create(evoke_plan* P, evoke_plan** out_plan) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    plan_free(P);
    return EVOKE_ECUDA;
  }
  *out_plan = P;
  return EVOKE_OK;
}

int create_single(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
                  const evoke_opts* opts, cudaStream_t st, evoke_plan** out_plan,
                  bool tunable = true) {
  int rc = ensure_transform();
  if (rc) return rc;
  rc = check_csr(rowptr, colidx, n, m, st);
  if (rc) return rc;
  evoke_plan* P = new evoke_plan();
  P->rowptr = rowptr;
  P->col = colidx;
  P->n = n;
  P->m = m;
  P->st = st;
  P->cfg.tunable = tunable;
  if (opts && opts->root_ctas > 0) P->cfg.root_ctas = opts->root_ctas;
  P->cfg.orbits = opts_orbits(opts);
  P->cfg.induced = !(opts && opts->noninduced);
  if (opts && opts->schedule == 1) P->cfg.schedule = 1;
  if (P->cfg.orbits < 0) {
    plan_free(P);
    return EVOKE_EINVAL;
  }
  if (opts && opts->validate) {  // validate the caller's CSR before relabelling it
    rc = validate_csr(rowptr, colidx, n, m, st);
    if (rc) {
      plan_free(P);
      return rc;
    }
  }
  rc = plan_relabel_setup(P);
  if (!rc) rc = plan_stage1(P, false);
  if (!rc) rc = plan_stage2(P);
  if (rc) {
    plan_free(P);
    return rc;
  }
  P->launches_per_exec = count_launches(P, true);
  return plan_finish_create(P, out_plan);
}

// synchronous one-shot run on a plan, with the phase profiler
int run_once(evoke_plan* P, long long* out, cudaStream_t st) {
  execute(P, out, st, /*timed=*/true);  // phase() counts the launches
  if (P->rs.prof) {
    u64 pc[8] = {};
    cudaMemcpyAsync(pc, P->rs.prof, sizeof(pc), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    fprintf(stderr, "evoke root phases (Gcycles summed over CTAs): wedges %.2f, diamonds+R %.2f, "
                    "3-path push %.2f, wedges2+k %.2f, scan %.2f\n",
            pc[0] * 1e-9, pc[1] * 1e-9, pc[2] * 1e-9, pc[3] * 1e-9, pc[4] * 1e-9);
  }
  int ovf = 0;
  cudaMemcpyAsync(&ovf, P->status + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaGetLastError();
  cudaError_t e2 = cudaStreamSynchronize(st);
  if (e != cudaSuccess || e2 != cudaSuccess) return EVOKE_ECUDA;
  return ovf ? EVOKE_EOVERFLOW : EVOKE_OK;
}

}  // namespace

extern "C" {

int evoke_version(void) { return 100; }

int evoke_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
  return EVOKE_OK;
}

int evoke_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  drain_pending();
  g_agg.clear();
  return EVOKE_OK;
}

int evoke_profile_read(evoke_phase_time* out, int cap, int* count) {
  if (!count || (cap > 0 && !out)) return EVOKE_EINVAL;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  drain_pending();
  *count = (int)g_agg.size();
  for (int i = 0; i < cap && i < (int)g_agg.size(); ++i) {
    memcpy(out[i].name, g_agg[i].name, sizeof(out[i].name));
    out[i].launches = g_agg[i].launches;
    out[i].calls = g_agg[i].calls;
    out[i].ms = g_agg[i].ms;
  }
  return EVOKE_OK;
}

unsigned long long evoke_launch_count_impl() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  return g_launches;
}

uint64_t evoke_launch_count(void) { return (uint64_t)evoke_launch_count_impl(); }

const char* evoke_strerror(int code) {
  switch (code) {
    case EVOKE_OK: return "ok";
    case EVOKE_EINVAL: return "invalid argument";
    case EVOKE_ENOTSIMPLE: return "input is not a simple undirected graph";
    case EVOKE_ERANGE: return "vertex id or size out of range";
    case EVOKE_ENOMEM: return "device allocation failed";
    case EVOKE_ECUDA: return "CUDA error";
    case EVOKE_ETIMEOUT: return "bounded device wait timed out";
    case EVOKE_EOVERFLOW: return "count overflow";
    case EVOKE_EINCONSISTENT: return "orbit counts of one pattern disagree";
    default: return "unknown status";
  }
}

int evoke_orbit_matrix(int64_t* A) {
  if (!A) return EVOKE_EINVAL;
  const Derived& d = derived();
  if (!d.ok) return EVOKE_ECUDA;
  for (int i = 0; i < 73 * 73; ++i) A[i] = d.A[i];
  return EVOKE_OK;
}


int evoke_plan_create(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
                      const evoke_opts* opts, void* stream, evoke_plan** plan) {
  if (!plan) return EVOKE_EINVAL;
  *plan = nullptr;
  return create_single(rowptr, colidx, n, m, opts, static_cast<cudaStream_t>(stream), plan);
}

int evoke_plan_create_batch(const uint32_t* rowptr_cat, const uint32_t* colidx_cat,
                            const int64_t* vtx_off, const int64_t* edge_off, uint32_t G,
                            const evoke_opts* opts, void* stream, evoke_plan** plan) {
  if (!plan || !rowptr_cat || !vtx_off || !edge_off) return EVOKE_EINVAL;
  *plan = nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = ensure_transform();
  if (rc) return rc;
  long long tot[2] = {0, 0};
  if (cudaMemcpyAsync(&tot[0], vtx_off + G, sizeof(long long), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(&tot[1], edge_off + G, sizeof(long long), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess)
    return EVOKE_EINVAL;
  if (cudaStreamSynchronize(st) != cudaSuccess) return EVOKE_ECUDA;
  if (tot[0] < 0 || tot[1] < 0 || (tot[1] & 1)) return EVOKE_EINVAL;
  if (tot[0] >= 0xffffffffll || tot[1] >= 0xffffffffll) return EVOKE_ERANGE;
  if (tot[1] && !colidx_cat) return EVOKE_EINVAL;
  evoke_plan* P = new evoke_plan();
  P->batch = true;
  P->rowptr_cat = rowptr_cat;
  P->col_cat = colidx_cat;
  P->vtx_off = reinterpret_cast<const long long*>(vtx_off);
  P->edge_off = reinterpret_cast<const long long*>(edge_off);
  P->G = G;
  P->n = (u32)tot[0];
  P->m = (u64)tot[1] / 2;
  P->st = st;
  if (opts && opts->root_ctas > 0) P->cfg.root_ctas = opts->root_ctas;
  P->cfg.orbits = opts_orbits(opts);
  P->cfg.induced = !(opts && opts->noninduced);
  if (opts && opts->schedule == 1) P->cfg.schedule = 1;
  if (P->cfg.orbits < 0) {
    delete P;
    return EVOKE_EINVAL;
  }
  // the largest component sizes the per-CTA maps of the root pass
  {
    u32* d = nullptr;
    if (dmalloc(&d, sizeof(u32), st) != cudaSuccess) {
      delete P;
      return EVOKE_ENOMEM;
    }
    cudaMemsetAsync(d, 0, sizeof(u32), st);
    launch_max_component(P->vtx_off, G, d, st);
    u32 mc = 0;
    cudaMemcpyAsync(&mc, d, sizeof(u32), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      delete P;
      return EVOKE_ECUDA;
    }
    P->max_comp = mc;
  }
  rc = plan_stage1(P, opts && opts->validate);
  if (!rc) rc = plan_stage2(P);
  if (rc) {
    plan_free(P);
    return rc;
  }
  P->launches_per_exec = count_launches(P, true);
  return plan_finish_create(P, plan);
}

int evoke_plan_execute(evoke_plan* plan, int64_t* out, void* stream) {
  if (!plan || (plan->n && !out)) return EVOKE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_launches += (unsigned long long)plan->launches_per_exec;
  }
  execute(plan, reinterpret_cast<long long*>(out), st, /*timed=*/false);
  return cudaGetLastError() == cudaSuccess ? EVOKE_OK : EVOKE_ECUDA;
}

int evoke_plan_status(const evoke_plan* plan, void* stream) {
  if (!plan) return EVOKE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int ovf = 0;
  cudaMemcpyAsync(&ovf, plan->status + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return EVOKE_ECUDA;
  return ovf ? EVOKE_EOVERFLOW : EVOKE_OK;
}

int evoke_plan_execute_profiled(evoke_plan* plan, int64_t* out, void* stream) {
  if (!plan || (plan->n && !out)) return EVOKE_EINVAL;
  execute(plan, reinterpret_cast<long long*>(out), static_cast<cudaStream_t>(stream),
          /*timed=*/true);
  return cudaGetLastError() == cudaSuccess ? EVOKE_OK : EVOKE_ECUDA;
}

int evoke_plan_launch_graph(evoke_plan* plan, int64_t* out, void* stream) {
  if (!plan || (plan->n && !out)) return EVOKE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  long long* o = reinterpret_cast<long long*>(out);
  if (!plan->gexec || plan->gexec_out != o) {
    if (plan->gexec) {
      cudaGraphExecDestroy(plan->gexec);
      plan->gexec = nullptr;
    }
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return EVOKE_ECUDA;
    cudaGraph_t graph = nullptr;
    int rc = EVOKE_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = EVOKE_ECUDA;
    if (!rc) {
      execute(plan, o, cs, /*timed=*/false);
      if (cudaStreamEndCapture(cs, &graph) != cudaSuccess) rc = EVOKE_ECUDA;
    }
    if (!rc && cudaGraphInstantiate(&plan->gexec, graph, 0) != cudaSuccess) rc = EVOKE_ECUDA;
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (rc) {
      cudaGetLastError();
      return rc;
    }
    plan->gexec_out = o;
  }
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_launches += (unsigned long long)plan->launches_per_exec;
  }
  return cudaGraphLaunch(plan->gexec, st) == cudaSuccess ? EVOKE_OK : EVOKE_ECUDA;
}

int evoke_plan_info(const evoke_plan* plan, evoke_plan_stats* out) {
  if (!plan || !out) return EVOKE_EINVAL;
  out->n = plan->n;
  out->m = plan->m;
  out->triangles = plan->ntri_entries / 6;
  out->max_degree = plan->dmax;
  out->max_out_degree = plan->max_outdeg;
  out->max_component = plan->batch ? plan->max_comp : plan->n;
  out->device_bytes = plan->bytes + plan->bytes2;
  out->kernels_per_execution = plan->launches_per_exec;
  out->root_threads = plan->rs.threads;
  out->root_ctas = plan->rs.ctas;
  out->root_ctas_max = plan->ctas_alloc;
  out->orbits = plan->cfg.orbits;
  out->link_warps = (int32_t)plan->cfg.link_warps;
  return EVOKE_OK;
}

int evoke_plan_set_tuning(evoke_plan* plan, int32_t root_threads, int32_t root_ctas) {
  if (!plan || root_ctas <= 0 ||
      (root_threads != 64 && root_threads != 128 && root_threads != 256 && root_threads != 512 &&
       root_threads != 1024))
    return EVOKE_EINVAL;
  const int per_sm_max = 2048 / root_threads;
  if (root_ctas > sm_count_cached() * per_sm_max * 4) return EVOKE_ERANGE;
  // the per-CTA maps were sized when the plan was created
  if (root_ctas > plan->ctas_alloc) return EVOKE_ERANGE;
  if (plan->gexec) {
    cudaGraphExecDestroy(plan->gexec);
    plan->gexec = nullptr;
  }
  plan->cfg.root_threads = root_threads;
  plan->rs.threads = root_threads;
  plan->rs.ctas = root_ctas;
  return EVOKE_OK;
}

int evoke_plan_set_schedule(evoke_plan* plan, int32_t schedule, int32_t chunk) {
  if (!plan || (schedule != 0 && schedule != 1) || chunk < 1 || chunk > 4096) return EVOKE_EINVAL;
  if (plan->gexec) {
    cudaGraphExecDestroy(plan->gexec);
    plan->gexec = nullptr;
  }
  plan->cfg.schedule = schedule;
  plan->cfg.chunk = (u32)chunk;
  plan->launches_per_exec = count_launches(plan, true);
  return EVOKE_OK;
}

int evoke_plan_set_model(evoke_plan* plan, const float* params) {
  if (!plan) return EVOKE_EINVAL;
  if (plan->gexec) {
    cudaGraphExecDestroy(plan->gexec);
    plan->gexec = nullptr;
  }
  plan->model = params;
  if (params && !plan->model_block && plan->n) {
    if (dmalloc(&plan->model_block, sizeof(float) * 5 * (size_t)plan->n + 256, plan->st) !=
        cudaSuccess)
      return EVOKE_ENOMEM;
    plan->feat = static_cast<float*>(plan->model_block);
    plan->prio = plan->feat + 4 * (size_t)plan->n;
    if (cudaStreamSynchronize(plan->st) != cudaSuccess) return EVOKE_ECUDA;
  }
  plan->launches_per_exec = count_launches(plan, true);
  return EVOKE_OK;
}

int evoke_plan_features(evoke_plan* plan, float* X, void* stream) {
  if (!plan || (plan->n && !X)) return EVOKE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!plan->relabel) {
    launch_features(plan->g, plan->acc, X, st);
  } else if (plan->n) {
    float* tmp = nullptr;
    if (dmalloc(&tmp, sizeof(float) * 4 * (size_t)plan->n, st) != cudaSuccess) return EVOKE_ENOMEM;
    launch_features(plan->g, plan->acc, tmp, st);
    const u64 cnt = 4 * (u64)plan->n;
    unpermute_rows_kernel<float><<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(
        tmp, X, plan->rl_old_of, plan->n, 4);
    cudaFreeAsync(tmp, st);
  }
  return cudaGetLastError() == cudaSuccess ? EVOKE_OK : EVOKE_ECUDA;
}

int evoke_plan_root_timing(evoke_plan* plan, uint64_t* root_cycles, uint64_t* cta_end_ns,
                           int64_t* out, void* stream) {
  if (!plan) return EVOKE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  u64* cyc = reinterpret_cast<u64*>(root_cycles);
  if (root_cycles && plan->relabel && plan->n &&
      dmalloc(&cyc, sizeof(u64) * (size_t)plan->n, st) != cudaSuccess)
    return EVOKE_ENOMEM;
  plan->rs.cycles = cyc;
  plan->rs.cta_end = reinterpret_cast<u64*>(cta_end_ns);
  execute(plan, reinterpret_cast<long long*>(out), st, /*timed=*/false);
  plan->rs.cycles = nullptr;
  plan->rs.cta_end = nullptr;
  if (root_cycles && plan->relabel && plan->n) {
    unpermute_rows_kernel<u64><<<(plan->n + 255) / 256, 256, 0, st>>>(
        cyc, reinterpret_cast<u64*>(root_cycles), plan->rl_old_of, plan->n, 1);
    cudaFreeAsync(cyc, st);
  }
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_launches += (unsigned long long)count_launches(plan, out != nullptr);
  }
  return cudaGetLastError() == cudaSuccess ? EVOKE_OK : EVOKE_ECUDA;
}

int evoke_mlp_forward(const float* X, uint32_t N, const float* params, float* y, void* stream) {
  if ((N && (!X || !y)) || !params) return EVOKE_EINVAL;
  launch_mlp_forward(X, N, params, y, static_cast<cudaStream_t>(stream));
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_launches += N ? 1 : 0;
  }
  return cudaGetLastError() == cudaSuccess ? EVOKE_OK : EVOKE_ECUDA;
}

int evoke_mlp_grad(const float* X, const float* T, uint32_t N, const float* params, float* grad,
                   float* loss, void* stream) {
  if (!params || !grad || !loss || (N && (!X || !T))) return EVOKE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaMemsetAsync(loss, 0, sizeof(float), st);
  launch_mlp_grad(X, T, nullptr, 0, N, params, grad, loss, st);
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_launches += N ? 1 : 0;
  }
  return cudaGetLastError() == cudaSuccess ? EVOKE_OK : EVOKE_ECUDA;
}

int evoke_mlp_train(const float* X, const float* T, uint32_t N, float* params, float* state,
                    int32_t epochs, int32_t batch, float lr, float* loss_out, float* scratch,
                    void* stream) {
  if (!X || !T || !params || !state || !scratch || N == 0 || epochs <= 0 || batch <= 0)
    return EVOKE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* grad = scratch;             // 1249
  float* loss = scratch + 1280;      // epochs
  cudaMemsetAsync(loss, 0, sizeof(float) * epochs, st);
  int step = 0;
  for (int e = 0; e < epochs; ++e) {
    for (u32 lo = 0; lo < N; lo += (u32)batch) {
      const u32 cnt = std::min<u32>((u32)batch, N - lo);
      launch_mlp_grad(X, T, nullptr, lo, cnt, params, grad, loss + e, st);
      launch_adam(params, grad, state, lr, ++step, st);
    }
  }
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_launches += 2ull * (unsigned long long)step;
  }
  if (loss_out) {
    cudaMemcpyAsync(loss_out, loss, sizeof(float) * epochs, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return EVOKE_ECUDA;
  }
  return cudaGetLastError() == cudaSuccess ? EVOKE_OK : EVOKE_ECUDA;
}

int evoke_plan_destroy(evoke_plan* plan) {
  if (!plan) return EVOKE_EINVAL;
  plan_free(plan);
  return EVOKE_OK;
}

int evoke_count_orbits(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
                       int64_t* out, const evoke_opts* opts, void* stream) {
  if (n && !out) return EVOKE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  evoke_plan* P = nullptr;
  int rc = create_single(rowptr, colidx, n, m, opts, st, &P, /*tunable=*/false);
  if (rc) return rc;
  rc = run_once(P, reinterpret_cast<long long*>(out), st);
  plan_free(P);
  return rc;
}

int evoke_count_batch(const uint32_t* rowptr_cat, const uint32_t* colidx_cat,
                      const int64_t* vtx_off, const int64_t* edge_off, uint32_t G, int64_t* out,
                      const evoke_opts* opts, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  evoke_plan* P = nullptr;
  int rc = evoke_plan_create_batch(rowptr_cat, colidx_cat, vtx_off, edge_off, G, opts, stream, &P);
  if (rc) return rc;
  if (P->n && !out) {
    plan_free(P);
    return EVOKE_EINVAL;
  }
  rc = run_once(P, reinterpret_cast<long long*>(out), st);
  plan_free(P);
  return rc;
}

int evoke_edge_orbits(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
                      int64_t* tri, int64_t* c4, int64_t* k4, int64_t* e7, int64_t* e9,
                      void* stream) {
  if (!tri && !c4 && !k4 && !e7 && !e9) return EVOKE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  evoke_plan* P = nullptr;
  int rc = create_single(rowptr, colidx, n, m, nullptr, st, &P, /*tunable=*/false);
  if (rc) return rc;
  rc = run_once(P, nullptr, st);
  const u64 S = P->g.S;
  const unsigned eb = (unsigned)((S + 255) / 256);
  if (!rc && S) {
    // per-slot values in the plan's slot order, then (relabelled plans) in the caller's
    long long* tmp = nullptr;
    u32* orig = nullptr;
    if (P->relabel) {
      if (dmalloc(&tmp, sizeof(long long) * S, st) != cudaSuccess ||
          dmalloc(&orig, sizeof(u32) * S, st) != cudaSuccess)
        rc = EVOKE_ENOMEM;
      else
        launch_orig_slot(P->in_rowptr, P->in_col, P->rl_old_of, P->rl_rowptr, P->rl_col, P->n,
                         orig, st);
    }
    auto emit = [&](auto&& fill, int64_t* dst) {
      if (!dst || rc) return;
      long long* d = reinterpret_cast<long long*>(dst);
      if (!P->relabel) {
        fill(d);
      } else {
        fill(tmp);
        unpermute_slots_kernel<<<eb, 256, 0, st>>>(tmp, d, orig, S);
      }
    };
    emit([&](long long* d) { widen_kernel<<<eb, 256, 0, st>>>(P->sa.T, d, S); }, tri);
    emit([&](long long* d) { copy_i64_kernel<<<eb, 256, 0, st>>>(P->sa.E5, d, S); }, c4);
    emit([&](long long* d) { copy_i64_kernel<<<eb, 256, 0, st>>>(P->sa.K4, d, S); }, k4);
    emit([&](long long* d) { copy_i64_kernel<<<eb, 256, 0, st>>>(P->sa.E7, d, S); }, e7);
    emit([&](long long* d) { copy_i64_kernel<<<eb, 256, 0, st>>>(P->sa.E9, d, S); }, e9);
    if (tmp) cudaFreeAsync(tmp, st);
    if (orig) cudaFreeAsync(orig, st);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) rc = EVOKE_ECUDA;
  }
  plan_free(P);
  return rc;
}

int evoke_edge_orbit_counts(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n,
                            uint64_t m, int64_t* out, void* stream) {
  if (!out && m) return EVOKE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  evoke_plan* P = nullptr;
  int rc = create_single(rowptr, colidx, n, m, nullptr, st, &P, /*tunable=*/false);
  if (rc) return rc;
  rc = run_once(P, nullptr, st);
  const u64 S = P->g.S;
  if (!rc && S) {
    u32* orig = nullptr;
    if (P->relabel && dmalloc(&orig, sizeof(u32) * S, st) != cudaSuccess) rc = EVOKE_ENOMEM;
    if (!rc)
      phase("edge_orbits", orig ? 2 : 1, st, [&] {
        if (orig)
          launch_orig_slot(P->in_rowptr, P->in_col, P->rl_old_of, P->rl_rowptr, P->rl_col, P->n,
                           orig, st);
        launch_edge_orbits12(P->g, P->sa, P->acc, reinterpret_cast<long long*>(out), orig, st);
      });
    if (orig) cudaFreeAsync(orig, st);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) rc = EVOKE_ECUDA;
  }
  plan_free(P);
  return rc;
}

int evoke_graphlet_totals(const int64_t* counts, uint32_t n, int32_t orbits, int64_t* totals,
                          void* stream) {
  if ((n && !counts) || !totals || (orbits != 73 && orbits != 15)) return EVOKE_EINVAL;
  const Derived& d = derived();
  if (!d.ok) return EVOKE_ECUDA;
  const int np = orbits == 73 ? 30 : 9;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  u64 sums[73] = {};
  if (n) {
    u64* dsum = nullptr;
    if (dmalloc(&dsum, sizeof(u64) * orbits, st) != cudaSuccess) return EVOKE_ENOMEM;
    cudaMemsetAsync(dsum, 0, sizeof(u64) * orbits, st);
    launch_column_sums(reinterpret_cast<const long long*>(counts), n, orbits, dsum,
                       sm_count_cached(), st);
    {
      std::lock_guard<std::mutex> lk(g_prof_mu);
      g_launches += 1;
    }
    cudaMemcpyAsync(sums, dsum, sizeof(u64) * orbits, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(dsum, st);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
      return EVOKE_ECUDA;
  }
  // each copy of pattern j puts orbit_size[o] of its vertices in orbit o, so
  // every orbit of j must give the same quotient
  int rc = EVOKE_OK;
  for (int j = 0; j < np; ++j) {
    bool first = true;
    long long t = 0;
    for (int o = 0; o < orbits; ++o) {
      if (d.orbit_pattern[o] != j) continue;
      const u64 sz = (u64)d.orbit_size[o];
      if (sums[o] % sz) rc = EVOKE_EINCONSISTENT;
      const long long q = (long long)(sums[o] / sz);
      if (first) t = q;
      else if (q != t) rc = EVOKE_EINCONSISTENT;
      first = false;
    }
    totals[j] = t;
  }
  return rc;
}

int evoke_build_dag(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
                    uint32_t* dag_rowptr, uint32_t* dag_colidx, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!dag_rowptr || (m && !dag_colidx)) return EVOKE_EINVAL;
  int rc = check_csr(rowptr, colidx, n, m, st);
  if (rc) return rc;
  // the DAG alone: degrees, reverse slots, counts, scan, fill
  const u64 S = 2 * m;
  size_t bytes = sz<u32>(n) + sz<u32>(S) + sz<u32>(n) + sz<char>(scan_tmp_bytes(std::max<u64>(S, n) + 1)) +
                 sz<u32>(m) + sz<int>(4);
  void* blk = nullptr;
  if (dmalloc(&blk, bytes, st) != cudaSuccess) return EVOKE_ENOMEM;
  Arena ar{static_cast<char*>(blk), bytes, 0, st};
  Graph g{};
  g.n = n;
  g.S = S;
  g.rowptr = rowptr;
  g.col = colidx;
  g.deg = ar.take<u32>(n);
  g.rev = ar.take<u32>(S);
  u32* cnt = ar.take<u32>(n);
  void* scan_tmp = ar.take<char>(scan_tmp_bytes(std::max<u64>(S, n) + 1));
  g.dag_slot = ar.take<u32>(m);
  int* status = ar.take<int>(4);
  g.dag_ptr = dag_rowptr;
  g.dag_col = dag_colidx;
  if (ar.overflow) {
    cudaFreeAsync(blk, st);
    return EVOKE_ENOMEM;
  }
  cudaMemsetAsync(status, 0, sizeof(int) * 4, st);
  phase("degrees", n ? 1 : 0, st, [&] { launch_degrees(g, st); });
  phase("dag", n ? 5 : 0, st, [&] { launch_dag(g, cnt, scan_tmp, st); });
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(blk, st);
  cudaError_t e2 = cudaStreamSynchronize(st);
  return (e == cudaSuccess && e2 == cudaSuccess) ? EVOKE_OK : EVOKE_ECUDA;
}

}  // extern "C"
