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
    for (int a = 0; a < P.k; ++a)
      if (full_orb[j][a] < 0) return out;
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

__global__ void widen_kernel(const u32* in, long long* out, u64 count) {
  u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = in[i];
}
__global__ void copy_i64_kernel(const u64* in, long long* out, u64 count) {
  u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = (long long)in[i];
}

// Everything that the passes need, laid out in device memory.
struct Run {
  Graph g{};
  SlotArrays sa{};
  u64* acc = nullptr;
  int* status = nullptr;
  u32* misc = nullptr;  // [0] dmax
  u32* cnt = nullptr;
  void* scan_tmp = nullptr;
  void* block = nullptr;
  void* block2 = nullptr;
  cudaStream_t st = nullptr;
  u32 dmax = 0;
  u32 max_outdeg = 0;
  u64 ntri_entries = 0;
};

int check_args(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
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

// Stages shared by every entry point: degrees, validation, reverse slots,
// DAG, triangle counts and lists.
int prepare(Run& R, const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
            bool validate, bool need_lists, cudaStream_t st) {
  R.st = st;
  const u64 S = 2 * m;
  size_t bytes = sz<u32>(n) + sz<u32>(S) + sz<u32>(n + 1) + 2 * sz<u32>(m) + sz<u32>(n) +
                 sz<char>(scan_tmp_bytes(std::max<u64>(S, n) + 1)) + sz<u32>(S) +
                 sz<u64>(S + 1) + sz<int>(4) + sz<u32>(4);
  if (cudaMallocAsync(&R.block, bytes, st) != cudaSuccess) return EVOKE_ENOMEM;
  Arena ar{static_cast<char*>(R.block), bytes, 0, st};
  Graph& g = R.g;
  g.n = n;
  g.S = S;
  g.rowptr = rowptr;
  g.col = colidx;
  g.deg = ar.take<u32>(n);
  g.rev = ar.take<u32>(S);
  g.dag_ptr = ar.take<u32>(n + 1);
  g.dag_col = ar.take<u32>(m);
  g.dag_slot = ar.take<u32>(m);
  R.cnt = ar.take<u32>(n);
  R.scan_tmp = ar.take<char>(scan_tmp_bytes(std::max<u64>(S, n) + 1));
  R.sa.T = ar.take<u32>(S);
  g.tl_ptr = ar.take<u64>(S + 1);
  R.status = ar.take<int>(4);
  R.misc = ar.take<u32>(4);
  if (ar.overflow) return EVOKE_ENOMEM;
  cudaMemsetAsync(R.status, 0, sizeof(int) * 4, st);
  cudaMemsetAsync(R.misc, 0, sizeof(u32) * 4, st);
  phase("degrees", n ? 1 : 0, st, [&] { launch_degrees(g, st); });
  phase("rev_validate", n ? 1 : 0, st, [&] { launch_rev_validate(g, R.status, st); });
  if (validate) {
    int status = 0;
    cudaMemcpyAsync(&status, R.status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return EVOKE_ECUDA;
    if (status & ST_RANGE) return EVOKE_ERANGE;
    if (status & ST_NOT_SIMPLE) return EVOKE_ENOTSIMPLE;
  }
  phase("dag", n ? 5 : 0, st, [&] { launch_dag(g, R.cnt, R.scan_tmp, st); });
  phase("dmax", n ? 1 : 0, st, [&] {
    if (n) dmax_kernel<<<(n + 255) / 256, 256, 0, st>>>(g.deg, g.dag_ptr, n, R.misc);
  });
  if (!need_lists) return EVOKE_OK;
  phase("tri_count", m ? 1 : 0, st, [&] { launch_tri_count(g, R.sa.T, st); });
  phase("tri_scan", S ? 3 : 0, st, [&] { launch_scan_u32_to_u64(R.sa.T, g.tl_ptr, S, R.scan_tmp, st); });
  u64 total = 0;
  u32 mx[2] = {0, 0};
  cudaMemcpyAsync(&total, g.tl_ptr + S, sizeof(u64), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(mx, R.misc, 2 * sizeof(u32), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return EVOKE_ECUDA;
  R.ntri_entries = total;
  R.dmax = mx[0];
  R.max_outdeg = mx[1];
  if (cudaMallocAsync(&R.block2, sz<u32>(total), st) != cudaSuccess) return EVOKE_ENOMEM;
  g.tl = static_cast<u32*>(R.block2);
  phase("tri_fill", m ? 1 : 0, st, [&] { launch_tri_fill(g, R.sa.T, st); });
  return EVOKE_OK;
}

void release(Run& R) {
  if (R.block) cudaFreeAsync(R.block, R.st);
  if (R.block2) cudaFreeAsync(R.block2, R.st);
  R.block = R.block2 = nullptr;
}

int finish(Run& R, int rc) {
  cudaError_t e = cudaGetLastError();
  release(R);
  cudaError_t e2 = cudaStreamSynchronize(R.st);
  if (rc != EVOKE_OK) return rc;
  if (e != cudaSuccess || e2 != cudaSuccess) return EVOKE_ECUDA;
  return EVOKE_OK;
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

int evoke_build_dag(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
                    uint32_t* dag_rowptr, uint32_t* dag_colidx, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!dag_rowptr || (m && !dag_colidx)) return EVOKE_EINVAL;
  int rc = check_args(rowptr, colidx, n, m, st);
  if (rc) return rc;
  Run R;
  rc = prepare(R, rowptr, colidx, n, m, false, false, st);
  if (rc == EVOKE_OK) {
    cudaMemcpyAsync(dag_rowptr, R.g.dag_ptr, sizeof(u32) * (n + 1), cudaMemcpyDeviceToDevice, st);
    if (m)
      cudaMemcpyAsync(dag_colidx, R.g.dag_col, sizeof(u32) * m, cudaMemcpyDeviceToDevice, st);
  }
  return finish(R, rc);
}

int evoke_edge_orbits(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
                      int64_t* tri, int64_t* c4, int64_t* k4, int64_t* e7, int64_t* e9,
                      void* stream);

int evoke_count_orbits(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
                       int64_t* out, const evoke_opts* opts, void* stream);

}  // extern "C"

namespace {

// The full pass sequence.  `out` may be null (intermediates only).
int run_all(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
            int64_t* out, const evoke_opts* opts, cudaStream_t st, int64_t* e_tri,
            int64_t* e_c4, int64_t* e_k4, int64_t* e_e7, int64_t* e_e9) {
  int rc = ensure_transform();
  if (rc) return rc;
  rc = check_args(rowptr, colidx, n, m, st);
  if (rc) return rc;
  if (n && out == nullptr && !e_tri && !e_c4 && !e_k4 && !e_e7 && !e_e9) return EVOKE_EINVAL;
  Run R;
  rc = prepare(R, rowptr, colidx, n, m, opts && opts->validate, true, st);
  if (rc) return finish(R, rc);
  Graph& g = R.g;
  const u64 S = g.S;
  const int ctas = (opts && opts->root_ctas > 0) ? opts->root_ctas : 2 * sm_count();
  const u32 dmax = std::max<u32>(R.dmax, 1);
  const u32 link_warps = (u32)sm_count() * 64;  // multiple of 8
  const u32 pref_stride = dmax + 1;
  // second arena: slot arrays, accumulators, scratch
  const bool root_profile = [] {
    const char* e = getenv("EVOKE_ROOT_PROFILE");
    return e && *e && *e != '0';
  }();
  size_t bytes = 9 * sz<u64>(S) + 2 * sz<u32>(S) + sz<u64>(8) + sz<u64>((size_t)NACC * n) +
                 root_scratch_bytes(n, ctas) + 256 * 8 + sz<u32>(n) + sz<u32>(64) + sz<u32>(4) +
                 sz<u32>((size_t)ctas * pref_stride) + sz<u32>((size_t)link_warps * dmax);
  void* blk = nullptr;
  if (cudaMallocAsync(&blk, bytes, st) != cudaSuccess) return finish(R, EVOKE_ENOMEM);
  Arena ar{static_cast<char*>(blk), bytes, 0, st};
  SlotArrays& sa = R.sa;
  sa.E5 = ar.take<u64>(S);
  sa.E7 = ar.take<u64>(S);
  sa.E9 = ar.take<u64>(S);
  sa.K4 = ar.take<u64>(S);
  sa.b49 = ar.take<u64>(S);
  sa.b62 = ar.take<u64>(S);
  sa.b64 = ar.take<u64>(S);
  sa.b68 = ar.take<u64>(S);
  sa.bc5 = ar.take<u64>(S);
  u64* acc = ar.take<u64>((size_t)NACC * n);
  RootScratch rs{};
  rs.ctas = ctas;
  rs.map = ar.take<MapRec>((size_t)ctas * n);
  rs.touched = ar.take<u32>((size_t)ctas * n);
  rs.jlist = ar.take<u32>((size_t)ctas * n);
  rs.order = ar.take<u32>(n);
  rs.bucket_cnt = ar.take<u32>(64);
  rs.head = ar.take<u32>(4);
  rs.tsrc = acc + (size_t)A_TSRC * n;
  rs.prof = root_profile ? ar.take<u64>(8) : nullptr;
  rs.cycles = nullptr;
  sa.Mmid = ar.take<u32>(S);
  sa.Mtop = ar.take<u32>(S);
  u32* pref = ar.take<u32>((size_t)ctas * pref_stride);
  u32* link_scratch = ar.take<u32>((size_t)link_warps * dmax);
  if (ar.overflow) {
    cudaFreeAsync(blk, st);
    return finish(R, EVOKE_ENOMEM);
  }
  // zero everything that is accumulated into
  cudaMemsetAsync(blk, 0, ar.used, st);

  const int nl = n ? 1 : 0, sl = S ? 1 : 0;
  phase("tri_edge", sl, st, [&] { launch_tri_edge(g, sa, st); });
  phase("vsum1", nl, st, [&] { launch_vsum1(g, sa, acc, st); });
  phase("tri_opp1", nl, st, [&] { launch_tri_opp1(g, sa, acc, st); });
  phase("k4", (R.ntri_entries ? 1 : 0) + sl, st, [&] { launch_k4(g, sa, acc, st); });
  phase("schedule", 3 * nl, st, [&] { launch_schedule(g, acc, rs, st); });
  phase("root", nl, st, [&] { launch_root_with_pref(g, sa, acc, rs, pref, pref_stride, st); });
  if (rs.prof) {
    u64 pc[8] = {};
    cudaMemcpyAsync(pc, rs.prof, sizeof(pc), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    fprintf(stderr, "evoke root phases (Gcycles summed over CTAs): wedges %.2f, diamonds+R %.2f, "
                    "3-path push %.2f, wedges2+k %.2f, scan %.2f\n",
            pc[0] * 1e-9, pc[1] * 1e-9, pc[2] * 1e-9, pc[3] * 1e-9, pc[4] * 1e-9);
  }
  phase("link", sl, st, [&] { launch_link(g, sa, link_scratch, link_warps, dmax, st); });
  phase("k5", sl, st, [&] { launch_k5(g, acc, R.max_outdeg, st); });
  phase("tri_opp2", nl, st, [&] { launch_tri_opp2(g, sa, acc, st); });
  phase("vsum2", nl, st, [&] { launch_vsum2(g, sa, acc, st); });
  phase("vsum3", nl, st, [&] { launch_vsum3(g, acc, st); });
  if (out) phase("finalize", nl, st, [&] { launch_finalize(g, acc, reinterpret_cast<long long*>(out), st); });
  const unsigned eb = (unsigned)((S + 255) / 256);
  if (S) {
    if (e_tri) widen_kernel<<<eb, 256, 0, st>>>(sa.T, reinterpret_cast<long long*>(e_tri), S);
    if (e_c4) copy_i64_kernel<<<eb, 256, 0, st>>>(sa.E5, reinterpret_cast<long long*>(e_c4), S);
    if (e_k4) copy_i64_kernel<<<eb, 256, 0, st>>>(sa.K4, reinterpret_cast<long long*>(e_k4), S);
    if (e_e7) copy_i64_kernel<<<eb, 256, 0, st>>>(sa.E7, reinterpret_cast<long long*>(e_e7), S);
    if (e_e9) copy_i64_kernel<<<eb, 256, 0, st>>>(sa.E9, reinterpret_cast<long long*>(e_e9), S);
  }
  cudaFreeAsync(blk, st);
  return finish(R, EVOKE_OK);
}

}  // namespace

extern "C" {

int evoke_count_orbits(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
                       int64_t* out, const evoke_opts* opts, void* stream) {
  if (n && !out) return EVOKE_EINVAL;
  return run_all(rowptr, colidx, n, m, out, opts, static_cast<cudaStream_t>(stream), nullptr,
                 nullptr, nullptr, nullptr, nullptr);
}

int evoke_edge_orbits(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
                      int64_t* tri, int64_t* c4, int64_t* k4, int64_t* e7, int64_t* e9,
                      void* stream) {
  if (!tri && !c4 && !k4 && !e7 && !e9) return EVOKE_EINVAL;
  return run_all(rowptr, colidx, n, m, nullptr, nullptr, static_cast<cudaStream_t>(stream), tri,
                 c4, k4, e7, e9);
}

}  // extern "C"
