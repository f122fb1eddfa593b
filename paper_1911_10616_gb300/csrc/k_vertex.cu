// Neighbour-sum passes (the O(m+n) class of Tab. orbits-category) and the
// fused equation + induced-transform kernel: the non-induced counts DM of
// Lem. 4vertexorbit and Thm. 5vertexorbit from the accumulated partial sums,
// then DIM = A^-1 DM (App. A) by back substitution, written as int64[n x 73].
#include "evoke_internal.cuh"

namespace {

constexpr int kFinalThreads = 64;

__device__ __forceinline__ u64 A(const u64* acc, int idx, u32 n, u32 u) {
  return acc[(u64)idx * n + u];
}
__device__ __forceinline__ u64 sgn(long long x) { return (u64)x; }

// neighbour-sum pass 1: sums over N(u) of functions of d(v) and T(u,v)
__global__ void vsum1_kernel(Graph g, SlotArrays sa, u64* __restrict__ acc) {
  const u32 u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (u >= g.n) return;
  const u32 n = g.n;
  u64 t2 = 0, s1 = 0, s6 = 0, s10 = 0, s13 = 0, s22 = 0, s41 = 0, s55 = 0, wk = 0, ts = 0;
  for (u32 s = g.rowptr[u] + lane; s < g.rowptr[u + 1]; s += 32) {
    const u32 v = g.col[s];
    const long long dv = g.deg[v];
    if (prec(g.deg, u, v)) ts += sa.Mtop[s];
    const long long t = sa.T[s];
    t2 += (u64)t;
    s1 += sgn(dv - 1);
    s6 += c2(dv - 1);
    s10 += (u64)t * sgn(dv - 2);
    s13 += c2(t);
    s22 += c3(dv - 1);
    s41 += c2(t) * sgn(dv - 3);
    s55 += c3(t);
    wk += (u64)dv;
  }
  t2 = warp_sum(t2); s1 = warp_sum(s1); s6 = warp_sum(s6); s10 = warp_sum(s10);
  s13 = warp_sum(s13); s22 = warp_sum(s22); s41 = warp_sum(s41); s55 = warp_sum(s55);
  wk = warp_sum(wk);
  ts = warp_sum(ts);
  if (lane == 0) {
    acc[(u64)A_TSRC * n + u] = ts;
    acc[(u64)A_T * n + u] = t2 >> 1;
    acc[(u64)A_DM1 * n + u] = s1;
    acc[(u64)A_DM6 * n + u] = s6;
    acc[(u64)A_DM10 * n + u] = s10;
    acc[(u64)A_DM13 * n + u] = s13;
    acc[(u64)A_S22 * n + u] = s22;
    acc[(u64)A_S41 * n + u] = s41;
    acc[(u64)A_S55 * n + u] = s55;
    acc[(u64)A_WORK * n + u] = wk;
  }
}

// neighbour-sum pass 2: needs the per-vertex values of pass 1, the per-slot edge orbits
// and the root / wheel / 4-clique passes
__global__ void vsum2_kernel(Graph g, SlotArrays sa, u64* __restrict__ acc) {
  const u32 u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (u >= g.n) return;
  const u32 n = g.n;
  enum { kS4, kS9, kS18, kS19, kS24, kS28, kS31, kS35, kS37, kS39, kS40, kS45, kS57, kS60,
         kS67, kK4, kS29, kS32, kS43, kS48, kS61, kS53, kS25, kS49, kS62, kS64, kS68, kC5,
         kS69, kN };
  u64 r[kN];
#pragma unroll
  for (int i = 0; i < kN; ++i) r[i] = 0;
  for (u32 s = g.rowptr[u] + lane; s < g.rowptr[u + 1]; s += 32) {
    const u32 v = g.col[s];
    const u32 rv = g.rev[s];
    const long long dv = g.deg[v];
    const u64 t = sa.T[s];
    const u64 dm1v = A(acc, A_DM1, n, v);
    const u64 tv = A(acc, A_T, n, v);
    r[kS4] += dm1v;
    r[kS9] += tv - t;
    r[kS18] += A(acc, A_DM6, n, v);
    r[kS19] += dm1v * sgn(dv - 1) - 2 * tv;
    r[kS24] += A(acc, A_DM10, n, v);
    r[kS28] += tv;
    r[kS31] += sgn(dv - 1) * tv;
    r[kS35] += A(acc, A_DM8, n, v);
    r[kS37] += sa.E5[s] * sgn(dv - 2);
    r[kS39] += A(acc, A_DM13, n, v);
    r[kS40] += sa.E9[rv] * sgn(dv - 3);
    r[kS45] += A(acc, A_S12, n, v) >> 1;
    r[kS57] += sa.K4[s] * sgn(dv - 3);
    r[kS60] += sa.E9[rv] * (t - 1);
    r[kS67] += sa.K4[s] * (t - 2);
    r[kK4] += sa.K4[s];
    r[kS29] += t * dm1v;
    r[kS32] += t * c2(dv - 2);
    r[kS43] += t * (tv - 1);
    r[kS48] += (t - 1) * sa.E7[s];
    r[kS61] += (t - 1) * sa.E9[s];
    r[kS53] += t * sa.E5[s];
    r[kS25] += sgn(dv - 2) * sa.E7[s];
    r[kS49] += sa.b49[rv];
    r[kS62] += sa.b62[rv];
    r[kS64] += sa.b64[rv];
    r[kS68] += sa.b68[rv];
    r[kC5] += sa.bc5[rv];
    r[kS69] += sa.b68[s];
  }
#pragma unroll
  for (int i = 0; i < kN; ++i) r[i] = warp_sum(r[i]);
  if (lane) return;
  const long long d = g.rowptr[u + 1] - g.rowptr[u];
  const u64 T = A(acc, A_T, n, u);
  auto put = [&](int idx, u64 v) { acc[(u64)idx * n + u] = v; };
  put(A_S4, r[kS4]);
  put(A_S9, r[kS9]);
  put(A_S18, r[kS18]);
  put(A_S19, r[kS19]);
  put(A_S24, r[kS24]);
  put(A_S28, r[kS28]);
  put(A_S31, r[kS31]);
  put(A_S35, r[kS35]);
  put(A_S37, r[kS37]);
  put(A_S39, r[kS39]);
  put(A_S40, r[kS40]);
  put(A_S45, r[kS45]);
  put(A_S57, r[kS57]);
  put(A_S60, r[kS60]);
  put(A_S67, r[kS67]);
  put(A_K4X3, r[kK4]);
  put(A_S29, r[kS29]);
  put(A_S32, r[kS32]);
  put(A_S43, r[kS43]);
  put(A_S48, r[kS48]);
  put(A_S61, r[kS61]);
  put(A_S53, r[kS53]);
  put(A_S25, r[kS25]);
  put(A_S49, r[kS49]);
  put(A_S62, r[kS62]);
  put(A_S64, r[kS64]);
  put(A_S68, r[kS68]);
  put(A_S69X4, r[kS69]);
  put(A_C5, A(acc, A_C5, n, u) + r[kC5]);
  put(A_DM4, r[kS4] - 2 * c2(d) - 2 * T);
  put(A_DM9, r[kS9]);
  put(A_DM12, A(acc, A_S12, n, u) >> 1);
  put(A_DM14, r[kK4] / 3);
}

// neighbour-sum pass 3: sums of pass-2 values over N(u)
__global__ void vsum3_kernel(Graph g, u64* __restrict__ acc) {
  const u32 u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (u >= g.n) return;
  const u32 n = g.n;
  u64 s15 = 0, s27 = 0, s56 = 0;
  for (u32 s = g.rowptr[u] + lane; s < g.rowptr[u + 1]; s += 32) {
    const u32 v = g.col[s];
    s15 += A(acc, A_DM4, n, v);
    s27 += A(acc, A_DM9, n, v);
    s56 += A(acc, A_DM14, n, v);
  }
  s15 = warp_sum(s15);
  s27 = warp_sum(s27);
  s56 = warp_sum(s56);
  if (lane == 0) {
    acc[(u64)A_S15 * n + u] = s15;
    acc[(u64)A_S27 * n + u] = s27;
    acc[(u64)A_S56 * n + u] = s56;
  }
}

// nonzeros of A above the diagonal, grouped by row (row i: entries
// kRowStart[i] .. kRowStart[i+1]); A is unit upper triangular.
constexpr int kMaxNz = 2048;
__constant__ unsigned short kNzCol[kMaxNz];
__constant__ short kNzVal[kMaxNz];
__constant__ unsigned short kRowStart[74];

// kOrb = 73: all orbits; kOrb = 15: the 4-vertex orbits 0..14 only (A is
// block diagonal by pattern size, so their rows of A^-1 stay inside 0..14)
// induced = false: the non-induced counts DM themselves (no A^-1).
template <int kOrb>
__global__ void __launch_bounds__(kFinalThreads)
finalize_kernel(Graph g, const u64* __restrict__ acc, long long* __restrict__ out,
                const u32* __restrict__ old_of, bool induced) {
  __shared__ long long s_out[kFinalThreads * kOrb];
  const u32 n = g.n;
  const u32 u0 = blockIdx.x * kFinalThreads;
  const u32 u = u0 + threadIdx.x;
  if (u < n) {
    u64 M[73];
    const long long d = g.rowptr[u + 1] - g.rowptr[u];
    auto a = [&](int idx) { return acc[(u64)idx * n + u]; };
    const u64 T = a(A_T), DM1 = a(A_DM1), DM4 = a(A_DM4), DM6 = a(A_DM6), DM8 = a(A_DM8);
    const u64 DM9 = a(A_DM9), DM10 = a(A_DM10), DM12 = a(A_DM12), DM13 = a(A_DM13);
    const u64 DM14 = a(A_DM14);
    const u64 DM2 = c2(d), DM3 = T, DM7 = c3(d);
    const u64 DM5 = DM1 * sgn(d - 1) - 2 * T;
    const u64 DM11 = T * sgn(d - 2);
    M[0] = (u64)d;
    M[1] = DM1;
    M[2] = DM2;
    M[3] = DM3;
    M[4] = DM4;
    M[5] = DM5;
    M[6] = DM6;
    M[7] = DM7;
    M[8] = DM8;
    M[9] = DM9;
    M[10] = DM10;
    M[11] = DM11;
    M[12] = DM12;
    M[13] = DM13;
    M[14] = DM14;
    if constexpr (kOrb == 73) {
    M[15] = a(A_S15) - DM5 - 2 * DM11 - 2 * DM8;
    M[16] = DM4 * sgn(d - 1) - DM10 - 2 * DM8;
    M[17] = c2u(DM1) - DM3 - DM6 - DM8 - DM10;
    M[18] = a(A_S18) - 3 * DM7 - DM10;
    M[19] = a(A_S19) - DM4 - DM5 - DM10;
    M[20] = sgn(d - 1) * DM6 - DM10;
    M[21] = DM1 * c2(d - 1) - 2 * DM11;
    M[22] = a(A_S22);
    M[23] = c4(d);
    M[24] = a(A_S24) - DM10 - 2 * DM11 - 2 * DM12;
    M[25] = (a(A_S25) >> 1) - DM12;
    M[26] = sgn(d - 2) * DM10 - 2 * DM13;
    M[27] = a(A_S27) - DM11 - 2 * DM13;
    M[28] = sgn(d - 1) * a(A_S28) - 2 * DM3 - 2 * DM11 - 2 * DM12;
    M[29] = a(A_S29) - 4 * DM3 - DM10 - 2 * DM11 - 2 * DM12 - 2 * DM13;
    M[30] = DM1 * T - 2 * DM3 - DM10 - 2 * DM13;
    M[31] = a(A_S31) - 2 * DM9 - DM10 - 2 * DM3;
    M[32] = a(A_S32);
    M[33] = T * c2(d - 2);
    M[34] = a(A_C5);
    M[35] = a(A_S35) - 2 * DM8 - DM13;
    M[36] = a(A_S36) - DM13;
    M[37] = a(A_S37) - 2 * DM12;
    M[38] = DM8 * sgn(d - 2) - DM13;
    M[39] = a(A_S39) - DM13 - 2 * DM12;
    M[40] = a(A_S40);
    M[41] = a(A_S41);
    M[42] = DM13 * sgn(d - 3);
    M[43] = a(A_S43) - 2 * DM12 - 2 * DM13;
    M[44] = c2u(T) - DM13;
    M[45] = a(A_S45) - 2 * DM13 - 3 * DM14;
    M[46] = (a(A_S46) >> 1) - DM11 - 3 * DM14;
    M[47] = DM12 * sgn(d - 2) - 3 * DM14;
    M[48] = a(A_S48) - 6 * DM14;
    M[49] = a(A_S49);
    M[50] = a(A_S50);
    M[51] = a(A_S51) - 2 * DM12;
    M[52] = (a(A_S52) >> 1) - 2 * DM13;
    M[53] = a(A_S53) - 2 * DM13 - 2 * DM12;
    M[54] = a(A_S54) >> 1;
    M[55] = a(A_S55);
    M[56] = a(A_S56) - 3 * DM14;
    M[57] = a(A_S57);
    M[58] = DM14 * sgn(d - 3);
    M[59] = (a(A_S59) >> 1) - 2 * DM13 - 6 * DM14;
    M[60] = a(A_S60) - 6 * DM14;
    M[61] = (a(A_S61) >> 1) - 3 * DM14;
    M[62] = a(A_S62) - DM13;
    M[63] = a(A_S63);
    M[64] = a(A_S64);
    M[65] = (a(A_S65) >> 1) - 3 * DM14;
    M[66] = a(A_S66) - 6 * DM14;
    M[67] = a(A_S67);
    M[68] = a(A_S68);
    M[69] = a(A_S69X4) >> 2;
    M[70] = a(A_S70);
    M[71] = a(A_S71);
    M[72] = a(A_K5);
    }
    // induced counts: back substitution from the last orbit down
    long long* o = s_out + threadIdx.x * kOrb;
    for (int i = kOrb - 1; i >= 0; --i) {
      u64 v = M[i];
      if (induced)
        for (int k = kRowStart[i]; k < kRowStart[i + 1]; ++k)
          v -= (u64)(long long)kNzVal[k] * (u64)o[kNzCol[k]];
      o[i] = (long long)v;
    }
  }
  __syncthreads();
  const u32 cnt = min((u32)kFinalThreads, n - u0);
  if (!old_of) {
    long long* dst = out + (u64)u0 * kOrb;
    for (u32 i = threadIdx.x; i < cnt * kOrb; i += kFinalThreads) dst[i] = s_out[i];
  } else {  // relabelled graph: row of vertex u0 + r goes to its caller id
    for (u32 i = threadIdx.x; i < cnt * kOrb; i += kFinalThreads) {
      const u32 r = i / kOrb, k = i % kOrb;
      out[(u64)old_of[u0 + r] * kOrb + k] = s_out[i];
    }
  }
}

// neighbour-sum pass 2 of the 4-vertex-orbit mode: DM4, DM9, DM12, DM14 only
__global__ void vsum2_four_kernel(Graph g, SlotArrays sa, u64* __restrict__ acc) {
  const u32 u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (u >= g.n) return;
  const u32 n = g.n;
  u64 s4 = 0, s9 = 0, k4 = 0;
  for (u32 s = g.rowptr[u] + lane; s < g.rowptr[u + 1]; s += 32) {
    const u32 v = g.col[s];
    s4 += A(acc, A_DM1, n, v);
    s9 += A(acc, A_T, n, v) - sa.T[s];
    k4 += sa.K4[s];
  }
  s4 = warp_sum(s4);
  s9 = warp_sum(s9);
  k4 = warp_sum(k4);
  if (lane) return;
  const long long d = g.rowptr[u + 1] - g.rowptr[u];
  const u64 T = A(acc, A_T, n, u);
  acc[(u64)A_DM4 * n + u] = s4 - 2 * c2(d) - 2 * T;
  acc[(u64)A_DM9 * n + u] = s9;
  acc[(u64)A_DM12 * n + u] = A(acc, A_S12, n, u) >> 1;
  acc[(u64)A_DM14 * n + u] = k4 / 3;
}

inline unsigned warp_blocks(u32 n) { return (unsigned)(((u64)n * 32 + 255) / 256); }

}  // namespace

void launch_vsum1(const Graph& g, const SlotArrays& sa, u64* acc, cudaStream_t st) {
  if (!g.n) return;
  vsum1_kernel<<<warp_blocks(g.n), 256, 0, st>>>(g, sa, acc);
}
void launch_vsum2(const Graph& g, const SlotArrays& sa, u64* acc, cudaStream_t st) {
  if (!g.n) return;
  vsum2_kernel<<<warp_blocks(g.n), 256, 0, st>>>(g, sa, acc);
}
void launch_vsum3(const Graph& g, u64* acc, cudaStream_t st) {
  if (!g.n) return;
  vsum3_kernel<<<warp_blocks(g.n), 256, 0, st>>>(g, acc);
}

int upload_transform(const long long* A) {
  unsigned short col[kMaxNz];
  short val[kMaxNz];
  unsigned short start[74];
  int nz = 0;
  for (int i = 0; i < 73; ++i) {
    start[i] = (unsigned short)nz;
    if (A[i * 73 + i] != 1) return -1;
    for (int j = 0; j < 73; ++j) {
      if (j == i || !A[i * 73 + j]) continue;
      if (j < i || nz >= kMaxNz || A[i * 73 + j] > 32767 || A[i * 73 + j] < -32768) return -1;
      col[nz] = (unsigned short)j;
      val[nz] = (short)A[i * 73 + j];
      ++nz;
    }
  }
  start[73] = (unsigned short)nz;
  if (cudaMemcpyToSymbol(kNzCol, col, sizeof(unsigned short) * (nz ? nz : 1)) != cudaSuccess) return -2;
  if (cudaMemcpyToSymbol(kNzVal, val, sizeof(short) * (nz ? nz : 1)) != cudaSuccess) return -2;
  if (cudaMemcpyToSymbol(kRowStart, start, sizeof(start)) != cudaSuccess) return -2;
  return nz;
}

void launch_finalize(const Graph& g, const u64* acc, long long* out, const u32* old_of,
                     int orbits, bool induced, cudaStream_t st) {
  if (!g.n) return;
  const unsigned blocks = (g.n + kFinalThreads - 1) / kFinalThreads;
  if (orbits == 15)
    finalize_kernel<15><<<blocks, kFinalThreads, 0, st>>>(g, acc, out, old_of, induced);
  else
    finalize_kernel<73><<<blocks, kFinalThreads, 0, st>>>(g, acc, out, old_of, induced);
}

// Column sums of an int64[rows x K] count matrix (K = 73 or 15), wrapping
// u64.  Every block has a multiple of K threads and so does the grid, so a
// grid-stride walk keeps each thread on one column.
__global__ void column_sums_kernel(const long long* __restrict__ counts, u64 total, int K,
                                   u64* __restrict__ sums) {
  __shared__ u64 s[73];
  if (threadIdx.x < (unsigned)K) s[threadIdx.x] = 0;
  __syncthreads();
  const u64 stride = (u64)gridDim.x * blockDim.x;
  u64 a = 0;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride)
    a += (u64)counts[i];
  if (a) atomicAdd(&s[threadIdx.x % K], a);
  __syncthreads();
  if (threadIdx.x < (unsigned)K && s[threadIdx.x]) atomicAdd(&sums[threadIdx.x], s[threadIdx.x]);
}

void launch_column_sums(const long long* counts, u64 rows, int K, u64* sums, int sms,
                        cudaStream_t st) {
  if (!rows) return;
  const int threads = 1024 / K * K;
  column_sums_kernel<<<2 * sms, threads, 0, st>>>(counts, rows * (u64)K, K, sums);
}

void launch_vsum2_four(const Graph& g, const SlotArrays& sa, u64* acc, cudaStream_t st) {
  if (!g.n) return;
  vsum2_four_kernel<<<warp_blocks(g.n), 256, 0, st>>>(g, sa, acc);
}

// --- edge orbits of the 3- and 4-vertex patterns (Lem. 4edgeorbit) --------
// One thread per slot s = (u,v); row s (or orig[s] for relabelled plans) of
// `out` receives E0..E11 <u,v>, u on the side of the higher vertex orbit for
// the asymmetric edge orbits (Fig. edge_orbits).  The five edge sums the
// earlier passes keep per slot (T, E5 = C4(u,v), E7, E9, K4) are combined
// with d(u), d(v), T(u) and DM1(u).
__global__ void edge_orbit_kernel(Graph g, SlotArrays sa, const u64* __restrict__ acc,
                                  long long* __restrict__ out, const u32* __restrict__ orig) {
  const u64 s = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.S) return;
  const u32 n = g.n;
  const u32 v = g.col[s], u = g.col[g.rev[s]];
  const long long du = g.deg[u], dv = g.deg[v];
  const long long t = sa.T[s];
  const u64 tu = acc[(u64)A_T * n + u], dm1 = acc[(u64)A_DM1 * n + u];
  u64 e[12];
  e[0] = (u64)(du - 1);
  e[1] = (u64)t;
  e[2] = dm1 - (u64)(dv - 1) - (u64)t;            // 3-paths v-u-x-y, u inner
  e[3] = (u64)((du - 1) * (dv - 1) - t);           // 3-paths with (u,v) in the middle
  e[4] = c2(du - 1);                               // 3-stars centred at u
  e[5] = sa.E5[s];                                 // 4-cycles through (u,v)
  e[6] = tu - (u64)t;                              // paws, u the centre, v the pendant
  e[7] = sa.E7[s];                                 // paws with (u,v) opposite the centre
  e[8] = (u64)(t * (du - 2));                      // paws, u the centre, v on the triangle
  e[9] = sa.E9[s];                                 // diamonds, u a chord end, v a tip
  e[10] = c2(t);                                   // diamonds with chord (u,v)
  e[11] = sa.K4[s];                                // 4-cliques
  const u64 row = orig ? (u64)orig[s] : s;
  long long* o = out + row * 12;
#pragma unroll
  for (int i = 0; i < 12; i += 2)
    *reinterpret_cast<longlong2*>(o + i) = make_longlong2((long long)e[i], (long long)e[i + 1]);
}

void launch_edge_orbits12(const Graph& g, const SlotArrays& sa, const u64* acc, long long* out,
                          const u32* orig, cudaStream_t st) {
  if (!g.S) return;
  edge_orbit_kernel<<<(unsigned)((g.S + 255) / 256), 256, 0, st>>>(g, sa, acc, out, orig);
}
