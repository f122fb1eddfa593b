/*
 * evoke.h -- C ABI of libevoke, a GB300 (sm_103a) implementation of EVOKE's
 * per-vertex orbit counting (Pashanasangi & Seshadhri, "Efficiently Counting
 * Vertex Orbits of All 5-vertex Subgraphs, by EVOKE").
 *
 * For every vertex u of a simple undirected graph the library computes the
 * exact induced counts of the 73 vertex orbits 0..72 of the connected 2- to
 * 5-vertex patterns H0..H29 (Sec. 1.1 "Problem Description", Fig.
 * node_orbits): out[u*73 + k] is the number of vertex sets S containing u,
 * |S| <= 5, whose induced subgraph is the pattern owning orbit k with u in
 * orbit k.  The route is the paper's: base-pattern counts over the degree
 * ordered DAG (Sec. 2 "Degree ordering", Thm. running-time), the non-induced
 * counts of Lem. 4vertexorbit, Lem. 4edgeorbit, Thm. 5vertexorbit and
 * Thm. 5-Cycle-Clique, then the induced transform DIM = A^-1 DM (App. A).
 *
 * Conventions for every entry point:
 *  - Graph input is CSR in DEVICE memory: rowptr[n+1] (uint32, rowptr[0] = 0,
 *    rowptr[n] = 2m) and colidx[2m] (uint32).  Each row must be strictly
 *    increasing, without self-loops, and the graph symmetric (a simple
 *    undirected graph; Sec. 2).  n < 2^32 - 1 and 2m < 2^32.  Isolated
 *    vertices and n = 0 are legal.  The largest degree must be at most
 *    65,535 (EVOKE_ERANGE otherwise): the per-pair counts of the 2-hop pass
 *    are 32-bit, and their bounds (d, d(d-1)/2, d^2) fit only up to there.
 *  - `stream` is a cudaStream_t (0 = legacy default stream).  Work is
 *    enqueued on it; the functions synchronise that stream internally where
 *    noted (to size internal buffers and to read validation results) and
 *    return after the results are written, unless stated otherwise.
 *  - The caller owns every buffer passed in.  The library allocates its
 *    internal workspace on `stream` from a memory pool of its own (one per
 *    device, created on first use) and frees it before returning (plans:
 *    when destroyed).  Freed memory stays reserved by that pool for later
 *    calls rather than being unmapped at each synchronisation.
 *  - Return value: EVOKE_OK or one of the error codes below; nothing throws
 *    across the ABI.  evoke_strerror() names a code.
 *  - Counts are int64 two's-complement; the arithmetic wraps modulo 2^64,
 *    so results are exact whenever the true counts fit in int64.
 */
#ifndef EVOKE_H
#define EVOKE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EVOKE_OK 0
#define EVOKE_EINVAL 1       /* bad argument (null pointer, sizes inconsistent) */
#define EVOKE_ENOTSIMPLE 2   /* input is not a simple undirected graph (validate) */
#define EVOKE_ERANGE 3       /* a vertex id >= n (validate), n / m too large, or a degree > 65,535 */
#define EVOKE_ENOMEM 4       /* internal device allocation failed */
#define EVOKE_ECUDA 5        /* a CUDA call or kernel launch failed */
#define EVOKE_ETIMEOUT 6     /* a bounded device wait gave up */
#define EVOKE_EOVERFLOW 7    /* an internal 32-bit count (3-paths per vertex pair) wrapped */
#define EVOKE_EINCONSISTENT 8 /* counts whose orbits of one pattern disagree (totals) */

typedef struct evoke_opts {
  int32_t validate;   /* nonzero: check the CSR invariants first (syncs the stream) */
  int32_t root_ctas;  /* persistent CTAs of the per-root pass; 0 = 2 per SM */
  int32_t schedule;   /* order of the per-root pass: 0 = degree-bucket schedule
                         (decreasing wedge work); 1 = roots grouped by their
                         highest-degree neighbour, taken by the CTAs in chunks
                         of 8 consecutive roots (see evoke_plan_set_schedule) */
  int32_t orbits;     /* 0 or 73: all 73 orbits, out is int64[n*73];
                         15: the 4-vertex orbits 0..14 only (Thm. 4orbit,
                         Lem. 4vertexorbit), out is int64[n*15]; the passes
                         that feed only 5-vertex orbits (wheels, 5-cliques,
                         their neighbour sums) are skipped; other values:
                         EVOKE_EINVAL */
  int32_t noninduced; /* nonzero: write the non-induced counts DM (Sec. 2
                         "Induced vs non-induced"; A^-1 of App. A not applied) */
} evoke_opts;

/*
 * evoke_count_orbits -- induced orbit counts of all vertices.
 *   rowptr, colidx : device CSR as described above (read only).
 *   n, m           : vertices and undirected edges (colidx has 2m entries).
 *   out            : device int64[n*73] (n*15 with opts->orbits = 15),
 *                    row-major, orbit index = the paper's orbit number
 *                    (Fig. node_orbits); fully written.
 *   opts           : may be NULL (defaults: no validation, 2 CTAs per SM).
 * Synchronises `stream` (buffer sizing).  Errors: EVOKE_EINVAL (null
 * pointers with n > 0, rowptr[n] != 2m), EVOKE_ENOTSIMPLE / EVOKE_ERANGE
 * (validate only), EVOKE_ENOMEM, EVOKE_ECUDA.
 */
int evoke_count_orbits(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
                       int64_t* out, const evoke_opts* opts, void* stream);

/*
 * evoke_count_batch -- induced orbit counts of every vertex of G graphs at
 * once (many small graphs of uneven sizes).  All arrays are DEVICE memory:
 *   rowptr_cat : uint32, the graphs' own rowptr arrays back to back; graph g
 *                occupies entries vtx_off[g] + g .. vtx_off[g+1] + g
 *                (n_g + 1 entries, local offsets starting at 0).
 *   colidx_cat : uint32[edge_off[G]], the graphs' colidx arrays back to back,
 *                local vertex ids (0 .. n_g-1).
 *   vtx_off    : int64[G+1], prefix sums of n_g;  edge_off : int64[G+1],
 *                prefix sums of 2 m_g.
 *   out        : int64[vtx_off[G] * 73]; the rows of graph g start at row
 *                vtx_off[g].  Every graph must itself be simple (see above).
 * The graphs are processed as one disjoint union (counts of connected
 * patterns are per component); the per-root maps are sized by the largest
 * graph.  Limits: vtx_off[G] and edge_off[G] below 2^32 - 1.  Synchronises
 * `stream`.  Errors as evoke_count_orbits.
 */
int evoke_count_batch(const uint32_t* rowptr_cat, const uint32_t* colidx_cat,
                      const int64_t* vtx_off, const int64_t* edge_off, uint32_t G, int64_t* out,
                      const evoke_opts* opts, void* stream);

/*
 * Plans: the same computation split into a sizing step and a replayable
 * execution.  evoke_plan_create / evoke_plan_create_batch take the inputs of
 * evoke_count_orbits / evoke_count_batch (which must stay unchanged and
 * alive while the plan is used), run the sizing passes, allocate every
 * device buffer the execution needs (stream-ordered, on `stream`) and
 * synchronise `stream`.  evoke_plan_execute enqueues the whole pass sequence
 * (CSR to counts) on `stream` without any host synchronisation, so it may be
 * captured into a CUDA graph; evoke_plan_launch_graph captures one execution
 * into a CUDA graph on first use (and again whenever `out` changes) and
 * launches that graph.  evoke_plan_destroy synchronises and frees.  A plan
 * must not be executed concurrently on two streams.
 */
typedef struct evoke_plan evoke_plan;

typedef struct evoke_plan_stats {
  uint32_t n;                 /* vertices (all graphs of a batch) */
  uint64_t m;                 /* undirected edges */
  uint64_t triangles;
  uint32_t max_degree;
  uint32_t max_out_degree;    /* in the degree-ordered DAG */
  uint32_t max_component;     /* largest graph of a batch; n otherwise */
  uint64_t device_bytes;      /* device memory held by the plan */
  int32_t kernels_per_execution;
  int32_t root_threads;       /* threads per CTA of the per-root pass */
  int32_t root_ctas;          /* persistent CTAs of the per-root pass */
  int32_t root_ctas_max;      /* most CTAs evoke_plan_set_tuning accepts */
  int32_t link_warps;
  int32_t orbits;             /* orbits per output row: 73, or 15 */
} evoke_plan_stats;

int evoke_plan_create(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
                      const evoke_opts* opts, void* stream, evoke_plan** plan);
int evoke_plan_create_batch(const uint32_t* rowptr_cat, const uint32_t* colidx_cat,
                            const int64_t* vtx_off, const int64_t* edge_off, uint32_t G,
                            const evoke_opts* opts, void* stream, evoke_plan** plan);
int evoke_plan_execute(evoke_plan* plan, int64_t* out, void* stream);
int evoke_plan_launch_graph(evoke_plan* plan, int64_t* out, void* stream);
/* evoke_plan_execute with every phase bracketed by the profiler's events
 * (when evoke_profile_enable is on); same kernels, same results. */
int evoke_plan_execute_profiled(evoke_plan* plan, int64_t* out, void* stream);
int evoke_plan_info(const evoke_plan* plan, evoke_plan_stats* stats);
/* Device-side status of the plan's latest execution on `stream`: synchronises
 * the stream, then returns EVOKE_EOVERFLOW if a 32-bit per-pair 3-path count
 * of the 5-cycle pass wrapped (the counts of that execution are then not
 * exact), EVOKE_ECUDA if the stream failed, else EVOKE_OK.  Executions are
 * asynchronous, so this is how a caller of evoke_plan_execute or
 * evoke_plan_launch_graph learns of an overflow. */
int evoke_plan_status(const evoke_plan* plan, void* stream);
/* Autotuning hook: threads per CTA (64, 128, 256 or 512; the narrow shapes
 * suit batches of small graphs) and the number of persistent CTAs of the
 * per-root pass, at most root_ctas_max of evoke_plan_info. */
int evoke_plan_set_tuning(evoke_plan* plan, int32_t root_threads, int32_t root_ctas);
/* Root order of later executions: schedule 0 (degree-bucket) or 1 (grouped by
 * highest-degree neighbour, `chunk` consecutive roots per queue grab, 1..4096).
 * Counts do not depend on it.  Errors: EVOKE_EINVAL. */
int evoke_plan_set_schedule(evoke_plan* plan, int32_t schedule, int32_t chunk);
int evoke_plan_destroy(evoke_plan* plan);

/*
 * Learned work model.  The paper has no counterpart: it runs one thread and
 * schedules nothing.  Here a 4 -> 32 -> 32 -> 1 ReLU MLP in FP32 (1249
 * parameters, layout W1[32][4], b1[32], W2[32][32], b2[32], W3[32], b3)
 * predicts log2 of the cycles the per-root pass spends on each vertex from
 * log2(1 + x) of (DAG out-degree, neighbour degree sum = wedges rooted at
 * the vertex, sum of the out-neighbours' out-degrees, triangles at the
 * vertex).  With a model attached, the plan
 * orders its persistent root queue by that prediction (largest first)
 * instead of by the wedge-work estimate sum_{v in N(u)} d(v); the counts are
 * identical either way.  All arrays are DEVICE memory.
 *
 * evoke_plan_set_model  : attach params (1249 floats, must stay alive), or
 *                         NULL to return to the degree-bucket schedule.
 * evoke_plan_features   : X[n*4] features of every vertex (valid after one
 *                         execution of the plan).
 * evoke_plan_root_timing: one execution that also records, per vertex, the
 *                         clock64 cycles the per-root pass spent on it
 *                         (root_cycles[n]) and, per CTA, the global timer
 *                         (ns) when it ran out of roots (cta_end_ns[ctas]);
 *                         either may be NULL; out may be NULL.
 * evoke_mlp_forward     : y[N] = MLP(X[N*4]).
 * evoke_mlp_grad        : grad[1249] of the mean squared error of MLP(X)
 *                         against T[N], and the loss (*loss, device float).
 * evoke_mlp_train       : `epochs` passes of Adam (lr, beta 0.9 / 0.999) over
 *                         contiguous mini-batches of `batch` samples; params
 *                         updated in place, state = 2*1249 floats (zero at
 *                         start), scratch = 1280 + epochs floats, loss_out =
 *                         HOST float[epochs] (mean batch loss summed per
 *                         epoch) or NULL.  Synchronises `stream` if loss_out.
 */
int evoke_plan_set_model(evoke_plan* plan, const float* params);
int evoke_plan_features(evoke_plan* plan, float* X, void* stream);
int evoke_plan_root_timing(evoke_plan* plan, uint64_t* root_cycles, uint64_t* cta_end_ns,
                           int64_t* out, void* stream);
int evoke_mlp_forward(const float* X, uint32_t N, const float* params, float* y, void* stream);
int evoke_mlp_grad(const float* X, const float* T, uint32_t N, const float* params, float* grad,
                   float* loss, void* stream);
int evoke_mlp_train(const float* X, const float* T, uint32_t N, float* params, float* state,
                    int32_t epochs, int32_t batch, float lr, float* loss_out, float* scratch,
                    void* stream);

/*
 * evoke_build_dag -- the degree-ordered DAG of Sec. 2: edge u -> v iff
 * d(u) < d(v), or d(u) = d(v) and u < v.
 *   dag_rowptr : device uint32[n+1] (written), dag_colidx : device
 *   uint32[m] (written), out-neighbours of each vertex ascending by id.
 * Synchronises `stream`.  Errors as evoke_count_orbits.
 */
int evoke_build_dag(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
                    uint32_t* dag_rowptr, uint32_t* dag_colidx, void* stream);

/*
 * evoke_build_dag_noalloc -- the same DAG as evoke_build_dag, for callers
 * that cannot allocate device memory: for example programs whose GPU memory
 * is owned up front by their own pool or arena (an allocation by a library
 * would fail or fragment it), or latency-critical code that cannot afford an
 * allocation, which may synchronise the device.  It allocates nothing: the
 * caller passes every buffer, and the one scratch buffer it needs (partial
 * sums of a prefix sum, about 32 KiB) is a static device array of the
 * library, held by every GPU that loads the library until the process exits.
 * The paper has no counterpart; this is an interface convenience.
 *   rowptr, colidx, n, m : device CSR as above (rowptr[n] must equal 2m; if
 *                          it does not, writes past m entries are dropped).
 *   dag_rowptr : device uint32[n+1], dag_colidx : device uint32[m] (written).
 * Limits: n <= 8,388,608 (EVOKE_ERANGE beyond).  All calls share the static
 * scratch array, so calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  The first call on a
 * device looks up the array's device address once; make it before any
 * stream capture on that device.  Synchronises `stream`.
 * Errors: EVOKE_EINVAL (null pointers), EVOKE_ERANGE, EVOKE_ECUDA.
 */
int evoke_build_dag_noalloc(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n,
                            uint64_t m, uint32_t* dag_rowptr, uint32_t* dag_colidx,
                            void* stream);

/*
 * evoke_edge_orbits -- per-edge counts of Lem. 4edgeorbit and Thm. 4orbit,
 * one entry per CSR slot s (slot of v in row u, 0 <= s < 2m), device int64[2m]
 * each (any may be NULL to skip):
 *   tri[s] = T(u,v) = E1, c4[s] = C4(u,v) = E5, k4[s] = K4(u,v) = E11,
 *   e7[s] = E7(u,v) = sum over x in N(u)^N(v) of (d(x)-2),
 *   e9[s] = E9<u,v> = sum over x in N(u)^N(v) of (T(u,x)-1).
 * Synchronises `stream`.  Errors as evoke_count_orbits.
 */
int evoke_edge_orbits(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n, uint64_t m,
                      int64_t* tri, int64_t* c4, int64_t* k4, int64_t* e7, int64_t* e9,
                      void* stream);

/*
 * evoke_edge_orbit_counts -- the twelve edge orbits E0..E11 of the 3- and
 * 4-vertex patterns (Fig. edge_orbits), non-induced, per Lem. 4edgeorbit.
 * out: device int64[2m * 12], row s = CSR slot s = (u,v) (the slot of v in
 * row u), column i = E_i<u,v>: the number of distinct non-induced copies of
 * the orbit's pattern in which (u,v) lies in edge orbit i and, where the two
 * ends of the edge orbit lie in different vertex orbits, u lies in the one
 * with the larger orbit number (e.g. E0<u,v> = d(u) - 1, u the centre of the
 * 2-path).  Symmetric orbits (E1, E3, E5, E7, E10, E11) give the same value
 * in slots (u,v) and (v,u).  The caller owns `out`.  Synchronises `stream`.
 * Errors as evoke_count_orbits; EVOKE_EINVAL if out is NULL and m > 0.
 */
int evoke_edge_orbit_counts(const uint32_t* rowptr, const uint32_t* colidx, uint32_t n,
                            uint64_t m, int64_t* out, void* stream);

/*
 * evoke_graphlet_totals -- global pattern counts from per-vertex orbit
 * counts: totals[j] = (sum over u of counts[u][o]) / |orbit o| for any
 * orbit o of pattern H_j (each copy of H_j has |orbit o| vertices in o).
 * Induced counts give induced copies, non-induced counts non-induced ones.
 *   counts : device int64[n * orbits], as written by evoke_count_orbits /
 *            evoke_count_batch / evoke_plan_execute (read only).
 *   orbits : 73 (totals of H0..H29, 30 entries) or 15 (H0..H8, 9 entries).
 *   totals : HOST int64[30] or int64[9] (written).
 * Synchronises `stream`.  Errors: EVOKE_EINVAL (null pointers, orbits not
 * 73 or 15), EVOKE_ENOMEM, EVOKE_ECUDA, EVOKE_EINCONSISTENT (a column sum
 * is not a multiple of its orbit size, or two orbits of one pattern give
 * different totals: not an orbit-count matrix; totals are still written).
 */
int evoke_graphlet_totals(const int64_t* counts, uint32_t n, int32_t orbits, int64_t* totals,
                          void* stream);

/*
 * evoke_orbit_matrix -- the library's matrix A of App. A (DM = A * DIM),
 * derived from the patterns at load time, into HOST int64[73*73] row-major.
 * Errors: EVOKE_EINVAL (null), EVOKE_ECUDA (pattern tables inconsistent).
 */
int evoke_orbit_matrix(int64_t* A);

/*
 * Phase profiling.  While enabled, every pass of the entry points above is
 * bracketed by CUDA events recorded on the stream the pass's kernels are
 * launched on (the caller's stream).  evoke_profile_read() synchronises those
 * events and returns, per pass name, the number of kernel launches, the
 * number of executions and the summed device time in milliseconds (host
 * array `out` of `cap` entries; *count receives the number of passes).
 * evoke_launch_count() returns the kernels launched by the library since it
 * was loaded (counted whether or not profiling is enabled).
 */
typedef struct evoke_phase_time {
  char name[24];
  int32_t launches;
  int32_t calls;
  double ms;
} evoke_phase_time;

int evoke_profile_enable(int on);
int evoke_profile_read(evoke_phase_time* out, int cap, int* count);
int evoke_profile_reset(void);
uint64_t evoke_launch_count(void);

/* Human-readable name of a status code (static string). */
const char* evoke_strerror(int code);

/* Library version, major * 10000 + minor * 100 + patch. */
int evoke_version(void);

#ifdef __cplusplus
}
#endif

#endif /* EVOKE_H */
