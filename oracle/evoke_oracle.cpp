// ORACLE -- test infrastructure only.
//
// A plain, slow, single-file CPU implementation of what EVOKE computes
// (Pashanasangi & Seshadhri, "Efficiently Counting Vertex Orbits of All
// 5-vertex Subgraphs, by EVOKE"): for every vertex u of a simple undirected
// graph, the induced counts of the 73 vertex orbits (0..72) of the connected
// 2- to 5-vertex patterns H0..H29 (Fig. node_orbits).
//
// Only tests/, the smoke check and the CPU-baseline leg of the benchmark may
// load this file's library.  It shares no code, table or helper with the CUDA
// path.  Three independent parts:
//
//   (1) patterns and orbits: the 30 patterns transcribed from Fig. node_orbits;
//       orbits are the automorphism classes (Def. auto), computed here by
//       brute force over all vertex permutations, then named by the orbit
//       number the figure prints on one vertex of each class.
//   (2) brute force (the definition): ESU enumeration (Wernicke & Rasche) of
//       every connected induced k-subset, k = 2..5; each subset is classified
//       and every member vertex gets +1 on its orbit.  Also, for tiny graphs,
//       the non-induced counts by enumerating every connected spanning edge
//       subset of every connected induced subset.
//   (3) the paper's method: base counts from plain definitions, then the
//       equations of Lem. 4vertexorbit, Lem. 4edgeorbit and Thm. 5vertexorbit,
//       the 5-cycle counter of Thm. 5-Cycle-Clique (directed 3-paths over the
//       degree-ordered DAG plus non in-in wedges, with the tailed-triangle
//       corrections) and 5-cliques by directed-clique enumeration; finally the
//       induced counts DIM = A^-1 DM (App. A), A derived by brute force over
//       the patterns themselves.
//
// Also: the edge orbits E0..E11 of Fig. edge_orbits, by the Definition that
// follows the figure (brute force over non-induced copies, tiny graphs) and
// by Lem. 4edgeorbit from the base counts; and the 4-vertex orbits alone
// (the method stopped after Lem. 4vertexorbit).
//
// Pins (the tests' CPU suite): the 4-vertex block of A equals Fig. A (but for
// one printed entry, A[5][13], an erratum: the definition gives 4) and its
// inverse Fig. Ainv; the
// orbits equal networkx's automorphism classes; brute force equals an
// independent networkx enumeration and closed forms (cliques, stars, cycles,
// paths); every DM equation equals non-induced brute force; the formula path
// equals brute force on random graphs; edge orbits: hand counts, closed forms,
// brute force = lemma, and totals against the vertex-orbit brute force; the
// 4-vertex-only path equals brute force and the full method's first columns.
//
// Arithmetic is exact: __int128 accumulation; a value outside int64 raises the
// overflow flag (return code 7).  Where the printed equations are garbled the
// reading taken is stated at the equation (see the comments marked READING).
#include <algorithm>
#include <array>
#include <cstdint>
#include <iterator>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;
typedef long long ll;

namespace {

// ---------------------------------------------------------------------------
// (1) Patterns H0..H29 (Fig. node_orbits; vertex ids 1..k as in the drawing)
// ---------------------------------------------------------------------------
struct PatternDef {
  int k;
  const char* edges;   // pairs of digits "12 23 ..."
  const char* labels;  // "vertex:orbit,..." -- the orbit number printed on a vertex
};

const PatternDef kPatterns[30] = {
    {2, "12", "2:0"},                                            // H0
    {3, "12 23", "2:2,3:1"},                                     // H1
    {3, "12 13 23", "3:3"},                                      // H2
    {4, "12 23 34", "3:5,4:4"},                                  // H3
    {4, "13 23 34", "3:7,4:6"},                                  // H4
    {4, "12 13 24 34", "3:8"},                                   // H5
    {4, "12 23 24 34", "1:9,2:11,3:10"},                         // H6
    {4, "12 13 14 24 34", "2:12,4:13"},                          // H7
    {4, "12 13 14 23 24 34", "4:14"},                            // H8
    {5, "12 23 34 45", "3:17,4:16,5:15"},                        // H9
    {5, "13 23 34 45", "1:19,3:21,4:20,5:18"},                   // H10
    {5, "13 23 34 35", "3:23,5:22"},                             // H11
    {5, "13 24 34 35 45", "1:24,3:26,5:25"},                     // H12
    {5, "12 13 23 34 45", "1:29,3:30,4:28,5:27"},                // H13
    {5, "13 23 34 35 45", "1:31,3:33,4:32"},                     // H14
    {5, "12 13 24 35 45", "5:34"},                               // H15
    {5, "12 23 24 35 45", "1:35,2:38,3:37,5:36"},                // H16
    {5, "12 23 24 25 35 45", "1:39,2:42,3:40,5:41"},             // H17
    {5, "12 13 23 34 35 45", "3:44,4:43"},                       // H18
    {5, "12 23 24 34 35 45", "1:45,2:47,3:48,5:46"},             // H19
    {5, "12 13 14 25 35 45", "1:50,2:49"},                       // H20
    {5, "12 13 24 34 35 45", "1:51,3:53,5:52"},                  // H21
    {5, "13 14 23 24 34 35 45", "1:54,3:55"},                    // H22
    {5, "12 23 24 25 34 35 45", "1:56,2:58,3:57"},               // H23
    {5, "12 13 23 24 34 35 45", "1:59,2:60,3:61"},               // H24
    {5, "12 13 14 25 34 35 45", "2:62,3:64,5:63"},               // H25
    {5, "12 13 23 24 25 34 35 45", "1:65,3:67,5:66"},            // H26
    {5, "12 13 14 23 25 34 35 45", "3:69,4:68"},                 // H27
    {5, "12 13 14 23 24 25 34 35 45", "1:70,4:71"},              // H28
    {5, "12 13 14 15 23 24 25 34 35 45", "5:72"},                // H29
};

// Edge orbits of the 3- and 4-vertex patterns (Fig. edge_orbits), numbered as
// in Lem. 4edgeorbit: the pattern and the vertex orbits of the edge's two
// ends, larger first.  READING: the figure's labels sit between edges in the
// extracted text; the numbering is fixed by the lemma's equations instead
// (E0 = d(u)-1 is the 2-path, E2 / E3 the end / middle edges of the 3-path,
// E6 / E7 / E8 the paw's pendant edge / edge opposite the centre / edges at
// the centre on the triangle, E9 / E10 the diamond's outer edges / chord).
struct EdgeOrbitDef {
  int pattern, hi, lo;
};
const EdgeOrbitDef kEdgeOrbits[12] = {
    {1, 2, 1},   {2, 3, 3},   {3, 5, 4},    {3, 5, 5},   {4, 7, 6},    {5, 8, 8},
    {6, 11, 9},  {6, 10, 10}, {6, 11, 10},  {7, 13, 12}, {7, 13, 13},  {8, 14, 14}};

struct Pattern {
  int k = 0;
  int adj[5][5] = {};
  int orbit[5] = {-1, -1, -1, -1, -1};  // orbit number of each vertex
};

struct Tables {
  bool ok = false;
  Pattern pat[30];
  int orbit_size[73] = {};
  int orbit_pattern[73] = {};
  int orbit_k[73] = {};
  // classification of a k-vertex adjacency mask: per position, the orbit, or -1
  std::vector<std::vector<std::array<int, 5>>> cls;  // cls[k][mask]
  ll A[73][73] = {};      // DM = A * DIM (App. A)
  // edge orbit of an edge whose ends have vertex orbits (hi, lo), hi >= lo,
  // in a 3- or 4-vertex pattern; -1 if none
  int edge_orbit[15][15];
};

inline int pair_bit(int i, int j) {  // i < j < 5, bit index among C(5,2) pairs
  static const int idx[5][5] = {{-1, 0, 1, 2, 3},
                                {0, -1, 4, 5, 6},
                                {1, 4, -1, 7, 8},
                                {2, 5, 7, -1, 9},
                                {3, 6, 8, 9, -1}};
  return idx[i][j];
}

bool connected_mask(int k, int mask) {
  int seen = 1, frontier = 1;
  while (frontier) {
    int nxt = 0;
    for (int a = 0; a < k; ++a)
      if (frontier >> a & 1)
        for (int b = 0; b < k; ++b)
          if (a != b && (mask >> pair_bit(std::min(a, b), std::max(a, b)) & 1) && !(seen >> b & 1))
            nxt |= 1 << b;
    seen |= nxt;
    frontier = nxt;
  }
  return seen == (1 << k) - 1;
}

Tables build_tables() {
  Tables t;
  t.cls.assign(6, {});
  for (int k = 2; k <= 5; ++k) {
    std::array<int, 5> none;
    none.fill(-1);
    t.cls[k].assign(1 << 10, none);  // masks use the 5-vertex pair numbering
  }
  for (int o = 0; o < 73; ++o) t.orbit_pattern[o] = -1;
  for (int j = 0; j < 30; ++j) {
    Pattern& p = t.pat[j];
    p.k = kPatterns[j].k;
    for (const char* c = kPatterns[j].edges; *c; ++c) {
      if (*c == ' ') continue;
      int a = c[0] - '1', b = c[1] - '1';
      p.adj[a][b] = p.adj[b][a] = 1;
      ++c;
    }
    // automorphism classes by brute force over permutations (Def. auto)
    int perm[5] = {0, 1, 2, 3, 4};
    int cls_of[5] = {0, 1, 2, 3, 4};
    do {
      bool aut = true;
      for (int a = 0; a < p.k && aut; ++a)
        for (int b = 0; b < p.k; ++b)
          if (p.adj[a][b] != p.adj[perm[a]][perm[b]]) { aut = false; break; }
      if (aut)
        for (int a = 0; a < p.k; ++a) {
          int lo = std::min(cls_of[a], cls_of[perm[a]]);
          int ca = cls_of[a], cb = cls_of[perm[a]];
          for (int x = 0; x < p.k; ++x)
            if (cls_of[x] == ca || cls_of[x] == cb) cls_of[x] = lo;
        }
    } while (std::next_permutation(perm, perm + p.k));
    // name each class by the label printed on one of its vertices
    for (const char* c = kPatterns[j].labels; *c;) {
      int v = c[0] - '1';
      int num = 0;
      c += 2;
      while (*c >= '0' && *c <= '9') num = num * 10 + (*c++ - '0');
      if (*c == ',') ++c;
      for (int x = 0; x < p.k; ++x)
        if (cls_of[x] == cls_of[v]) {
          if (p.orbit[x] != -1 && p.orbit[x] != num) return t;  // two labels on one class
          p.orbit[x] = num;
        }
      if (t.orbit_pattern[num] != -1) return t;
      t.orbit_pattern[num] = j;
    }
    for (int x = 0; x < p.k; ++x) {
      if (p.orbit[x] < 0) return t;  // unlabelled class
      t.orbit_size[p.orbit[x]]++;
      t.orbit_k[p.orbit[x]] = p.k;
    }
    // every relabelling of the pattern -> classification table entry
    int q[5] = {0, 1, 2, 3, 4};
    do {
      int mask = 0;
      for (int a = 0; a < p.k; ++a)
        for (int b = a + 1; b < p.k; ++b)
          if (p.adj[a][b]) mask |= 1 << pair_bit(std::min(q[a], q[b]), std::max(q[a], q[b]));
      auto& e = t.cls[p.k][mask];
      for (int a = 0; a < p.k; ++a) {
        if (e[q[a]] != -1 && e[q[a]] != p.orbit[a]) return t;
        e[q[a]] = p.orbit[a];
      }
    } while (std::next_permutation(q, q + p.k));
  }
  for (int o = 0; o < 73; ++o)
    if (t.orbit_pattern[o] < 0) return t;
  // every connected graph on k vertices must be classified
  for (int k = 2; k <= 5; ++k) {
    int allowed = 0;
    for (int a = 0; a < k; ++a)
      for (int b = a + 1; b < k; ++b) allowed |= 1 << pair_bit(a, b);
    for (int mask = 0; mask < (1 << 10); ++mask) {
      if (mask & ~allowed) continue;
      if (connected_mask(k, mask) != (t.cls[k][mask][0] != -1)) return t;
    }
  }
  // A (App. A): A[i][j] = number of non-induced matches of orbit i that an
  // induced copy of orbit j's pattern contains at a vertex of orbit j, i.e.
  // the connected spanning edge subsets of H_j in which that vertex has orbit i.
  for (int j = 0; j < 30; ++j) {
    const Pattern& p = t.pat[j];
    int pe[10][2], ne = 0;
    for (int a = 0; a < p.k; ++a)
      for (int b = a + 1; b < p.k; ++b)
        if (p.adj[a][b]) { pe[ne][0] = a; pe[ne][1] = b; ++ne; }
    ll cnt[5][73] = {};
    for (int sub = 1; sub < (1 << ne); ++sub) {
      int mask = 0;
      for (int e = 0; e < ne; ++e)
        if (sub >> e & 1) mask |= 1 << pair_bit(pe[e][0], pe[e][1]);
      if (!connected_mask(p.k, mask)) continue;
      const auto& c = t.cls[p.k][mask];
      for (int a = 0; a < p.k; ++a) cnt[a][c[a]]++;
    }
    for (int a = 0; a < p.k; ++a)
      for (int i = 0; i < 73; ++i) t.A[i][p.orbit[a]] = cnt[a][i];
    // the column must not depend on which vertex of the orbit is used
    for (int a = 0; a < p.k; ++a)
      for (int b = 0; b < p.k; ++b)
        if (p.orbit[a] == p.orbit[b])
          for (int i = 0; i < 73; ++i)
            if (cnt[a][i] != cnt[b][i]) return t;
  }
  // edge orbits: every edge of H1..H8 falls in exactly one row of the table,
  // and the rows are the automorphism classes of the edges (Def. auto)
  for (int a = 0; a < 15; ++a)
    for (int b = 0; b < 15; ++b) t.edge_orbit[a][b] = -1;
  for (int r = 0; r < 12; ++r) {
    const EdgeOrbitDef& e = kEdgeOrbits[r];
    if (e.hi < e.lo || e.hi > 14 || t.edge_orbit[e.hi][e.lo] != -1) return t;
    if (t.orbit_pattern[e.hi] != e.pattern || t.orbit_pattern[e.lo] != e.pattern) return t;
    t.edge_orbit[e.hi][e.lo] = r;
  }
  for (int j = 1; j <= 8; ++j) {
    const Pattern& p = t.pat[j];
    int ecls[5][5];
    for (int a = 0; a < 5; ++a)
      for (int b = 0; b < 5; ++b) ecls[a][b] = -1;
    for (int a = 0; a < p.k; ++a)
      for (int b = a + 1; b < p.k; ++b)
        if (p.adj[a][b]) {
          const int r = t.edge_orbit[std::max(p.orbit[a], p.orbit[b])][std::min(p.orbit[a], p.orbit[b])];
          if (r < 0) return t;
          ecls[a][b] = r;
        }
    // edges related by an automorphism share a row; edges sharing a row are
    // related by one
    int perm[5] = {0, 1, 2, 3, 4};
    bool linked[5][5][5][5] = {};
    do {
      bool aut = true;
      for (int a = 0; a < p.k && aut; ++a)
        for (int b = 0; b < p.k; ++b)
          if (p.adj[a][b] != p.adj[perm[a]][perm[b]]) { aut = false; break; }
      if (!aut) continue;
      for (int a = 0; a < p.k; ++a)
        for (int b = a + 1; b < p.k; ++b)
          if (p.adj[a][b]) {
            int c = std::min(perm[a], perm[b]), d = std::max(perm[a], perm[b]);
            if (ecls[a][b] != ecls[c][d]) return t;
            linked[a][b][c][d] = true;
          }
    } while (std::next_permutation(perm, perm + p.k));
    for (int a = 0; a < p.k; ++a)
      for (int b = a + 1; b < p.k; ++b)
        for (int c = 0; c < p.k; ++c)
          for (int d = c + 1; d < p.k; ++d)
            if (p.adj[a][b] && p.adj[c][d] && ecls[a][b] == ecls[c][d] && !linked[a][b][c][d])
              return t;
  }
  t.ok = true;
  return t;
}

const Tables& tables() {
  static const Tables t = build_tables();
  return t;
}

// ---------------------------------------------------------------------------
// graph helpers
// ---------------------------------------------------------------------------
struct G {
  uint32_t n;
  const int64_t* rp;
  const uint32_t* col;
  ll deg(uint32_t u) const { return rp[u + 1] - rp[u]; }
  const uint32_t* nb(uint32_t u) const { return col + rp[u]; }
  bool adj(uint32_t u, uint32_t v) const {
    const uint32_t* b = nb(u);
    const uint32_t* e = b + deg(u);
    return std::binary_search(b, e, v);
  }
  // slot of v in row u (v must be a neighbour)
  int64_t slot(uint32_t u, uint32_t v) const {
    const uint32_t* b = nb(u);
    return rp[u] + (std::lower_bound(b, b + deg(u), v) - b);
  }
  // degree order (Sec. 2 "Degree ordering"): i < j iff d(i) < d(j), ties by id
  bool prec(uint32_t i, uint32_t j) const {
    ll di = deg(i), dj = deg(j);
    return di < dj || (di == dj && i < j);
  }
};

std::vector<uint32_t> common(const G& g, uint32_t a, uint32_t b) {
  std::vector<uint32_t> out;
  const uint32_t *x = g.nb(a), *xe = x + g.deg(a), *y = g.nb(b), *ye = y + g.deg(b);
  while (x < xe && y < ye) {
    if (*x < *y) ++x;
    else if (*y < *x) ++y;
    else { out.push_back(*x); ++x; ++y; }
  }
  return out;
}

ll count_common(const G& g, uint32_t a, uint32_t b) {
  ll c = 0;
  const uint32_t *x = g.nb(a), *xe = x + g.deg(a), *y = g.nb(b), *ye = y + g.deg(b);
  while (x < xe && y < ye) {
    if (*x < *y) ++x;
    else if (*y < *x) ++y;
    else { ++c; ++x; ++y; }
  }
  return c;
}

inline i128 C2(i128 x) { return x < 2 ? 0 : x * (x - 1) / 2; }
inline i128 C3(i128 x) { return x < 3 ? 0 : x * (x - 1) * (x - 2) / 6; }
inline i128 C4(i128 x) { return x < 4 ? 0 : x * (x - 1) * (x - 2) * (x - 3) / 24; }

int nthreads_of(int requested) {
#ifdef _OPENMP
  return requested > 0 ? requested : omp_get_max_threads();
#else
  (void)requested;
  return 1;
#endif
}
int thread_id() {
#ifdef _OPENMP
  return omp_get_thread_num();
#else
  return 0;
#endif
}

// ---------------------------------------------------------------------------
// (2) brute force: ESU over connected induced k-subsets, k = 2..5
// ---------------------------------------------------------------------------
struct Esu {
  const G& g;
  const Tables& t;
  ll* dim;        // n*73, this thread's accumulator
  ll* dm;         // n*73 non-induced accumulator or null
  uint32_t root;
  uint32_t sub[5] = {0, 0, 0, 0, 0};
  int ns = 0;
  ll* eo = nullptr;  // optional [2m*12]: edge-orbit matches per slot (Lem. 4edgeorbit)
  int kmax = 5;      // largest subset enumerated

  bool in_sub(uint32_t x) const {
    for (int i = 0; i < ns; ++i)
      if (sub[i] == x) return true;
    return false;
  }
  bool adj_to_sub(uint32_t x) const {
    for (int i = 0; i < ns; ++i)
      if (g.adj(sub[i], x)) return true;
    return false;
  }
  void report() {
    int mask = 0;
    int pe[10][2], ne = 0;
    for (int a = 0; a < ns; ++a)
      for (int b = a + 1; b < ns; ++b)
        if (g.adj(sub[a], sub[b])) {
          mask |= 1 << pair_bit(a, b);
          pe[ne][0] = a; pe[ne][1] = b; ++ne;
        }
    const auto& c = t.cls[ns][mask];
    for (int a = 0; a < ns; ++a) dim[(size_t)sub[a] * 73 + c[a]]++;
    if (dm) {
      for (int s = 1; s < (1 << ne); ++s) {
        int sm = 0;
        for (int e = 0; e < ne; ++e)
          if (s >> e & 1) sm |= 1 << pair_bit(pe[e][0], pe[e][1]);
        if (!connected_mask(ns, sm)) continue;
        const auto& cc = t.cls[ns][sm];
        for (int a = 0; a < ns; ++a) dm[(size_t)sub[a] * 73 + cc[a]]++;
      }
    }
    if (eo && (ns == 3 || ns == 4)) {
      // every non-induced copy (connected spanning edge subset) and each of
      // its edges: +1 on the edge orbit, in the slot leaving the end with the
      // larger vertex orbit (both slots when the ends share an orbit)
      for (int s = 1; s < (1 << ne); ++s) {
        int sm = 0;
        for (int e = 0; e < ne; ++e)
          if (s >> e & 1) sm |= 1 << pair_bit(pe[e][0], pe[e][1]);
        if (!connected_mask(ns, sm)) continue;
        const auto& cc = t.cls[ns][sm];
        for (int e = 0; e < ne; ++e) {
          if (!(s >> e & 1)) continue;
          const int a = pe[e][0], b = pe[e][1];
          const int oa = cc[a], ob = cc[b];
          const int r = t.edge_orbit[std::max(oa, ob)][std::min(oa, ob)];
          if (oa >= ob) eo[(size_t)g.slot(sub[a], sub[b]) * 12 + r]++;
          if (ob >= oa) eo[(size_t)g.slot(sub[b], sub[a]) * 12 + r]++;
        }
      }
    }
  }
  void extend(std::vector<uint32_t> ext) {
    if (ns >= 2) report();
    if (ns == kmax) return;
    while (!ext.empty()) {
      uint32_t w = ext.back();
      ext.pop_back();
      std::vector<uint32_t> ext2 = ext;
      // exclusive neighbourhood of w w.r.t. the current subset, ids > root
      const uint32_t* nw = g.nb(w);
      for (ll i = 0; i < g.deg(w); ++i) {
        uint32_t u = nw[i];
        if (u <= root || u == w || in_sub(u) || adj_to_sub(u)) continue;
        if (std::find(ext2.begin(), ext2.end(), u) == ext2.end()) ext2.push_back(u);
      }
      sub[ns++] = w;
      extend(ext2);
      --ns;
    }
  }
};

// ---------------------------------------------------------------------------
// (3) the paper's method
// ---------------------------------------------------------------------------
struct Formula {
  const G& g;
  int threads;
  std::vector<i128> DM;        // n*73 non-induced counts, by orbit number
  // per slot (u,v): T(u,v), C4(u,v), K4(u,v), E7, E9<u,v>
  std::vector<ll> Te, C4e, K4e, E7e, E9e;
  bool overflow = false;
  bool four_only = false;      // stop after Lem. 4vertexorbit (orbits 0..14)

  explicit Formula(const G& gg, int th) : g(gg), threads(th) {}

  i128& dm(uint32_t u, int o) { return DM[(size_t)u * 73 + o]; }

  void run();
};

void Formula::run() {
  const uint32_t n = g.n;
  const int64_t S = g.rp[n];
  DM.assign((size_t)n * 73, 0);
  Te.assign(S, 0); C4e.assign(S, 0); K4e.assign(S, 0); E7e.assign(S, 0); E9e.assign(S, 0);
  const int nt = nthreads_of(threads);

  // --- base counts from their plain definitions -----------------------------
  // T(u,v) = |N(u) ^ N(v)| for every edge (triangles on the edge)
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
  for (int64_t u = 0; u < (int64_t)n; ++u)
    for (int64_t s = g.rp[u]; s < g.rp[u + 1]; ++s) Te[s] = count_common(g, (uint32_t)u, g.col[s]);

  // C4(u,v): 4-cycles u-v-b-a-u through the edge, by direct enumeration
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
  for (int64_t u = 0; u < (int64_t)(four_only ? 0 : n); ++u)
    for (int64_t s = g.rp[u]; s < g.rp[u + 1]; ++s) {
      uint32_t v = g.col[s];
      ll c = 0;
      for (int64_t i = g.rp[u]; i < g.rp[u + 1]; ++i) {
        uint32_t a = g.col[i];
        if (a == v) continue;
        // b in N(v) \ {u}, b ~ a  ->  |N(a) ^ N(v)| minus u (a ~ u, v ~ u always)
        c += count_common(g, a, v) - 1;
      }
      C4e[s] = c;
    }

  // K4(u,v): 4-cliques on the edge = edges inside N(u) ^ N(v)
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
  for (int64_t u = 0; u < (int64_t)n; ++u)
    for (int64_t s = g.rp[u]; s < g.rp[u + 1]; ++s) {
      std::vector<uint32_t> cn = common(g, (uint32_t)u, g.col[s]);
      ll c = 0;
      for (size_t i = 0; i < cn.size(); ++i)
        for (size_t j = i + 1; j < cn.size(); ++j)
          if (g.adj(cn[i], cn[j])) ++c;
      K4e[s] = c;
    }

  std::vector<i128> d(n), T(n), C4v(n), K4v(n);
  for (uint32_t u = 0; u < n; ++u) {
    d[u] = g.deg(u);
    i128 t2 = 0, k3 = 0;
    for (int64_t s = g.rp[u]; s < g.rp[u + 1]; ++s) { t2 += Te[s]; k3 += K4e[s]; }
    T[u] = t2 / 2;    // each triangle at u has two edges at u
    K4v[u] = k3 / 3;  // each 4-clique at u has three edges at u
  }
  // C4(u): 4-cycles through u = sum over neighbour pairs {a,b} of (|N(a)^N(b)| - 1)
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
  for (int64_t u = 0; u < (int64_t)n; ++u) {
    i128 c = 0;
    for (int64_t i = g.rp[u]; i < g.rp[u + 1]; ++i)
      for (int64_t j = i + 1; j < g.rp[u + 1]; ++j) c += count_common(g, g.col[i], g.col[j]) - 1;
    C4v[u] = c;
  }
  // triangle-based edge counts E7, E9 (Lem. 4edgeorbit)
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
  for (int64_t u = 0; u < (int64_t)(four_only ? 0 : n); ++u)
    for (int64_t s = g.rp[u]; s < g.rp[u + 1]; ++s) {
      uint32_t v = g.col[s];
      ll e7 = 0, e9 = 0;
      for (uint32_t x : common(g, (uint32_t)u, v)) {
        e7 += g.deg(x) - 2;
        e9 += Te[g.slot((uint32_t)u, x)] - 1;
      }
      E7e[s] = e7;
      E9e[s] = e9;
    }

  auto rev = [&](int64_t s, uint32_t u) { return g.slot(g.col[s], u); };

  // --- Lem. 4vertexorbit ------------------------------------------------------
  for (uint32_t u = 0; u < n; ++u) {
    i128 s1 = 0, s6 = 0, s10 = 0, s13 = 0;
    for (int64_t s = g.rp[u]; s < g.rp[u + 1]; ++s) {
      uint32_t v = g.col[s];
      s1 += d[v] - 1;                 // READING: sum of (d(v) - 1)
      s6 += C2(d[v] - 1);
      s10 += (i128)Te[s] * (d[v] - 2);
      s13 += C2(Te[s]);
    }
    dm(u, 0) = d[u];
    dm(u, 1) = s1;
    dm(u, 2) = C2(d[u]);
    dm(u, 3) = T[u];
    dm(u, 5) = dm(u, 1) * (d[u] - 1) - 2 * dm(u, 3);
    dm(u, 6) = s6;
    dm(u, 7) = C3(d[u]);
    dm(u, 8) = C4v[u];
    dm(u, 10) = s10;
    dm(u, 11) = T[u] * (d[u] - 2);
    dm(u, 13) = s13;
    dm(u, 14) = K4v[u];
  }
  for (uint32_t u = 0; u < n; ++u) {
    i128 s4 = 0, s9 = 0;
    for (int64_t s = g.rp[u]; s < g.rp[u + 1]; ++s) {
      uint32_t v = g.col[s];
      s4 += dm(v, 1);
      s9 += T[v] - Te[s];             // READING: sum of (T(v) - T(u,v))
    }
    dm(u, 4) = s4 - 2 * dm(u, 2) - 2 * dm(u, 3);
    dm(u, 9) = s9;
    // theta_12: triangles t = (u,v,x), sum of (T(v,x) - 1)
    i128 s12 = 0;
    for (int64_t s = g.rp[u]; s < g.rp[u + 1]; ++s) {
      uint32_t v = g.col[s];
      for (uint32_t x : common(g, u, v))
        if (x > v) s12 += Te[g.slot(v, x)] - 1;
    }
    dm(u, 12) = s12;
  }

  if (four_only) return;

  // --- Thm. 5vertexorbit ------------------------------------------------------
  // pair quantities, from plain definitions
  auto W = [&](uint32_t a, uint32_t b) -> i128 { return count_common(g, a, b); };
  auto D3 = [&](uint32_t a, uint32_t b, uint32_t c) -> i128 {
    ll k = 0;
    for (uint32_t x : common(g, a, b))
      if (g.adj(c, x)) ++k;
    return k;
  };
  // D(u,v): diamonds with u, v off the chord = edges inside N(u) ^ N(v)
  auto Dpair = [&](uint32_t a, uint32_t b) -> i128 {
    std::vector<uint32_t> cn = common(g, a, b);
    ll k = 0;
    for (size_t i = 0; i < cn.size(); ++i)
      for (size_t j = i + 1; j < cn.size(); ++j)
        if (g.adj(cn[i], cn[j])) ++k;
    return k;
  };

#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
  for (int64_t uu = 0; uu < (int64_t)n; ++uu) {
    const uint32_t u = (uint32_t)uu;
    const i128 du = d[u];
    auto M = [&](int o) -> i128& { return dm(u, o); };
    // neighbour sums (O(m+n) class)
    i128 n4 = 0, n5 = 0, n6 = 0, n9 = 0, n10 = 0, n8 = 0, n12 = 0, n13 = 0, n14 = 0;
    i128 s20 = 0, s21 = 0, s22 = 0, s28 = 0, s30 = 0, s31 = 0, s37 = 0, s40 = 0, s41 = 0;
    i128 s42 = 0, s55 = 0, s57 = 0, s60 = 0, s67 = 0;
    for (int64_t s = g.rp[u]; s < g.rp[u + 1]; ++s) {
      const uint32_t v = g.col[s];
      const i128 dv = d[v];
      const int64_t r = rev(s, u);
      n4 += dm(v, 4); n5 += dm(v, 5); n6 += dm(v, 6); n8 += dm(v, 8);
      n9 += dm(v, 9); n10 += dm(v, 10); n12 += dm(v, 12); n13 += dm(v, 13); n14 += dm(v, 14);
      s20 += (du - 1) * C2(dv - 1);
      s21 += (dv - 1) * C2(du - 1);
      s22 += C3(dv - 1);
      s28 += (du - 1) * T[v];
      s30 += (dv - 1) * T[u];
      s31 += (dv - 1) * T[v];
      s37 += (i128)C4e[s] * (dv - 2);
      s40 += (i128)E9e[r] * (dv - 3);        // READING: E9<v,u>, v the chord end
      s41 += C2(Te[s]) * (dv - 3);
      s42 += C2(Te[s]) * (du - 3);
      s55 += C3(Te[s]);
      s57 += (i128)K4e[s] * (dv - 3);
      s60 += (i128)E9e[r] * ((i128)Te[s] - 1);
      s67 += (i128)K4e[s] * ((i128)Te[s] - 2);
    }
    M(15) = n4 - M(5) - 2 * M(11) - 2 * M(8);
    M(16) = M(4) * (du - 1) - M(10) - 2 * M(8);
    M(17) = C2(M(1)) - M(3) - M(6) - M(8) - M(10);
    M(18) = n6 - 3 * M(7) - M(10);
    M(19) = n5 - M(4) - M(5) - M(10);      // READING: the garbled term is DM5(u)
    M(20) = s20 - M(10);                   // READING: coefficient 1 on DM10
    M(21) = s21 - 2 * M(11);               // READING: coefficient 2 on DM11
    M(22) = s22;
    M(23) = C4(du);
    M(24) = n10 - M(10) - 2 * M(11) - 2 * M(12);
    M(27) = n9 - M(11) - 2 * M(13);
    M(28) = s28 - 2 * M(3) - 2 * M(11) - 2 * M(12);
    M(30) = s30 - 2 * M(3) - M(10) - 2 * M(13);
    M(31) = s31 - 2 * M(9) - M(10) - 2 * M(3);
    M(33) = M(3) * C2(du - 2);
    M(35) = n8 - 2 * M(8) - M(13);         // READING: R8 = DM8(u), R13 = DM13(u)
    M(37) = s37 - 2 * M(12);
    M(38) = M(8) * (du - 2) - M(13);
    M(39) = n13 - M(13) - 2 * M(12);
    M(40) = s40;
    M(41) = s41;
    M(42) = s42;
    M(44) = C2(M(3)) - M(13);
    M(45) = n12 - 2 * M(13) - 3 * M(14);
    M(47) = M(12) * (du - 2) - 3 * M(14);
    M(55) = s55;
    M(56) = n14 - 3 * M(14);
    M(57) = s57;
    M(58) = M(14) * (du - 3);
    M(60) = s60 - 6 * M(14);
    M(67) = s67;

    // triangle sums t = (u,v,x)  (O(W) class)
    i128 s25 = 0, s26 = 0, s29 = 0, s32 = 0, s43 = 0, s46 = 0, s48 = 0, s52 = 0, s53 = 0;
    i128 s54 = 0, s59 = 0, s61 = 0, s65 = 0, s71 = 0;
    for (int64_t s = g.rp[u]; s < g.rp[u + 1]; ++s) {
      const uint32_t v = g.col[s];
      for (uint32_t x : common(g, u, v)) {
        if (x < v) continue;
        const i128 dv = d[v], dx = d[x];
        const int64_t sux = g.slot(u, x), svx = g.slot(v, x), sxv = g.slot(x, v);
        const i128 Tuv = Te[s], Tux = Te[sux], Tvx = Te[svx];
        s25 += (dv - 2) * (dx - 2);
        s26 += (du - 2) * ((dx - 2) + (dv - 2));
        s29 += dm(v, 1) + dm(x, 1);
        s32 += C2(dv - 2) + C2(dx - 2);
        s43 += (T[v] - 1) + (T[x] - 1);
        s46 += E7e[svx];
        s48 += (Tuv - 1) * (dx - 2) + (Tux - 1) * (dv - 2);
        s52 += C4e[svx];
        s53 += C4e[s] + C4e[sux];
        s54 += C2(Tvx - 1);
        s59 += (i128)E9e[sxv] + E9e[svx];
        s61 += (Tuv - 1) * (Tux - 1);
        s65 += K4e[svx];
        s71 += C2(D3(u, v, x));            // K4(t) = common neighbours of the triangle
      }
    }
    M(25) = s25 - M(12);
    M(26) = s26 - 2 * M(13);
    M(29) = s29 - 4 * M(3) - M(10) - 2 * M(11) - 2 * M(12) - 2 * M(13);
    M(32) = s32;
    M(43) = s43 - 2 * M(12) - 2 * M(13);
    M(46) = s46 - M(11) - 3 * M(14);
    M(48) = s48 - 6 * M(14);
    M(52) = s52 - 2 * M(13);
    M(53) = s53 - 2 * M(13) - 2 * M(12);
    M(54) = s54;
    M(59) = s59 - 2 * M(13) - 6 * M(14);
    M(61) = s61 - 3 * M(14);
    M(65) = s65 - 3 * M(14);
    M(71) = s71;

    // 4-clique sums <u,v,x,y>
    i128 s66 = 0, s70 = 0;
    {
      std::vector<uint32_t> nu(g.nb(u), g.nb(u) + g.deg(u));
      for (size_t a = 0; a < nu.size(); ++a)
        for (size_t b = a + 1; b < nu.size(); ++b) {
          if (!g.adj(nu[a], nu[b])) continue;
          for (size_t c = b + 1; c < nu.size(); ++c) {
            if (!g.adj(nu[a], nu[c]) || !g.adj(nu[b], nu[c])) continue;
            const uint32_t v = nu[a], x = nu[b], y = nu[c];
            s66 += (i128)Te[g.slot(v, x)] + Te[g.slot(v, y)] + Te[g.slot(x, y)];
            s70 += D3(v, x, y) - 1;        // K4(v,x,y) - 1
          }
        }
    }
    M(66) = s66 - 6 * M(14);               // READING: minus 6 DM14(u)
    M(70) = s70;

    // wedge-pair sums
    // 2-hop partners v (all v != u with a common neighbour)
    std::vector<uint32_t> hop2;
    for (int64_t s = g.rp[u]; s < g.rp[u + 1]; ++s)
      for (int64_t t2 = g.rp[g.col[s]]; t2 < g.rp[g.col[s] + 1]; ++t2)
        if (g.col[t2] != u) hop2.push_back(g.col[t2]);
    std::sort(hop2.begin(), hop2.end());
    hop2.erase(std::unique(hop2.begin(), hop2.end()), hop2.end());
    i128 s36 = 0, s50 = 0, s51 = 0, s63 = 0;
    for (uint32_t v : hop2) {
      const i128 w = W(u, v);
      const bool uv = g.adj(u, v);
      // READING: TT(u,v) = sum over x in N(u)^N(v) of (T(x,v) - [u~v])
      i128 tt = 0;
      for (uint32_t x : common(g, u, v)) tt += (i128)Te[g.slot(x, v)] - (uv ? 1 : 0);
      s36 += C2(w) * (d[v] - 2);
      s50 += C3(w);
      s51 += tt * (w - 1);
      s63 += Dpair(u, v) * (w - 2);
    }
    M(36) = s36 - M(13);
    M(50) = s50;
    M(51) = s51 - 2 * M(12);
    M(63) = s63;

    // unordered neighbour pairs {v,x}
    i128 s49 = 0, s62 = 0, s64 = 0, s69 = 0;
    for (int64_t i = g.rp[u]; i < g.rp[u + 1]; ++i)
      for (int64_t j = i + 1; j < g.rp[u + 1]; ++j) {
        const uint32_t v = g.col[i], x = g.col[j];
        const i128 w = W(v, x);
        const i128 d3 = D3(u, v, x);
        s49 += C2(w - 1);
        s62 += Dpair(v, x);
        s64 += d3 * (w - 2);                // READING: D(v,u,x) = |N(v)^N(u)^N(x)|
        s69 += C2(d3);
      }
    M(49) = s49;
    M(62) = s62 - M(13);
    M(64) = s64;
    M(69) = s69 / 2;                        // READING: each wheel counted on both diagonals
    // wedges <u,v,x>: u an end, v the centre, x the other end
    i128 s68 = 0;
    for (int64_t i = g.rp[u]; i < g.rp[u + 1]; ++i) {
      const uint32_t v = g.col[i];
      for (int64_t j = g.rp[v]; j < g.rp[v + 1]; ++j) {
        const uint32_t x = g.col[j];
        if (x == u) continue;
        s68 += C2(D3(u, v, x));
      }
    }
    M(68) = s68;
  }
  // --- Thm. 5-Cycle-Clique: 5-cycles through directed 3-paths ----------------
  // Directed 3-path (Fig. 5cycle, right): k->j, k->l, j->i.  Each 5-cycle has
  // exactly one such path whose closing wedge i-w-l is not in-in at w.
  {
    std::vector<std::vector<ll>> part(nt, std::vector<ll>(n, 0));
    std::vector<std::vector<uint32_t>> outn(n);
    for (uint32_t u = 0; u < n; ++u)
      for (int64_t s = g.rp[u]; s < g.rp[u + 1]; ++s)
        if (g.prec(u, g.col[s])) outn[u].push_back(g.col[s]);
    auto out_adj = [&](uint32_t a, uint32_t b) {  // a -> b
      return std::binary_search(outn[a].begin(), outn[a].end(), b);
    };
    // process the paths grouped by their end l; Wn(i,l) = number of wedges
    // i-w-l that are not in-in (not i->w<-l) -- the directed wedge table.
#pragma omp parallel num_threads(nt)
    {
      ll* acc = part[thread_id()].data();
      std::vector<ll> Wn(n, 0), P(n, 0);
      std::vector<uint32_t> touched;
#pragma omp for schedule(dynamic, 8)
      for (int64_t ll_ = 0; ll_ < (int64_t)n; ++ll_) {
        const uint32_t l = (uint32_t)ll_;
        touched.clear();
        for (int64_t s = g.rp[l]; s < g.rp[l + 1]; ++s) {
          const uint32_t w = g.col[s];
          for (int64_t t2 = g.rp[w]; t2 < g.rp[w + 1]; ++t2) {
            const uint32_t i = g.col[t2];
            if (i == l) continue;
            const bool in_in = g.prec(l, w) && g.prec(i, w);
            if (in_in) continue;
            if (Wn[i] == 0 && P[i] == 0) touched.push_back(i);
            Wn[i]++;
          }
        }
        // enumerate directed 3-paths ending at l: k->l, k->j, j->i
        for (int64_t s = g.rp[l]; s < g.rp[l + 1]; ++s) {
          const uint32_t k = g.col[s];
          if (!g.prec(k, l)) continue;  // need k -> l
          for (uint32_t j : outn[k]) {
            if (j == l) continue;
            for (uint32_t i : outn[j]) {
              if (i == l) continue;
              const bool ik = out_adj(k, i);   // k ~ i (k precedes i)
              const bool jl = g.adj(j, l);
              const ll c = Wn[i] - (ik ? 1 : 0) - (jl ? 1 : 0);
              acc[i] += c; acc[j] += c; acc[k] += c; acc[l] += c;
              if (Wn[i] == 0 && P[i] == 0) touched.push_back(i);
              P[i]++;
              // tailed triangles (Fig. TaileTri): types (1)/(2) put j on the
              // wedge i-j-l, type (3) puts k on the wedge i-k-l
              if (jl) acc[j] -= 1;
              if (ik) acc[k] -= 1;
            }
          }
        }
        // the fifth vertex w: every non in-in wedge i-w-l gains P(i,l)
        for (int64_t s = g.rp[l]; s < g.rp[l + 1]; ++s) {
          const uint32_t w = g.col[s];
          ll add = 0;
          for (int64_t t2 = g.rp[w]; t2 < g.rp[w + 1]; ++t2) {
            const uint32_t i = g.col[t2];
            if (i == l) continue;
            if (g.prec(l, w) && g.prec(i, w)) continue;
            add += P[i];
          }
          acc[w] += add;
        }
        for (uint32_t x : touched) { Wn[x] = 0; P[x] = 0; }
      }
    }
    for (uint32_t u = 0; u < n; ++u) {
      i128 c = 0;
      for (int th = 0; th < nt; ++th) c += part[th][u];
      dm(u, 34) = c;
    }
    // 5-cliques via directed cliques in the DAG (Chiba-Nishizeki)
    for (auto& p : part) std::fill(p.begin(), p.end(), 0);
#pragma omp parallel num_threads(nt)
    {
      ll* acc = part[thread_id()].data();
#pragma omp for schedule(dynamic, 8)
      for (int64_t aa = 0; aa < (int64_t)n; ++aa) {
        const uint32_t a = (uint32_t)aa;
        for (uint32_t b : outn[a]) {
          std::vector<uint32_t> s1;
          std::set_intersection(outn[a].begin(), outn[a].end(), outn[b].begin(), outn[b].end(),
                                std::back_inserter(s1));
          for (uint32_t c : s1) {
            std::vector<uint32_t> s2;
            std::set_intersection(s1.begin(), s1.end(), outn[c].begin(), outn[c].end(),
                                  std::back_inserter(s2));
            for (uint32_t dd : s2)
              for (uint32_t e : outn[dd])
                if (std::binary_search(s2.begin(), s2.end(), e)) {
                  acc[a]++; acc[b]++; acc[c]++; acc[dd]++; acc[e]++;
                }
          }
        }
      }
    }
    for (uint32_t u = 0; u < n; ++u) {
      i128 c = 0;
      for (int th = 0; th < nt; ++th) c += part[th][u];
      dm(u, 72) = c;
    }
  }
  // range check
  for (const i128& x : DM)
    if (x > (i128)INT64_MAX || x < (i128)INT64_MIN) overflow = true;
}

// induced = A^-1 * non-induced; A is unit upper triangular within each
// pattern size (orbits numbered by non-decreasing edge count), so back
// substitution from the highest orbit down is exact in integers.
bool invert_apply(const Tables& t, const i128* dm, i128* dim) {
  for (int i = 72; i >= 0; --i) {
    i128 v = dm[i];
    for (int j = i + 1; j < 73; ++j)
      if (t.A[i][j]) v -= (i128)t.A[i][j] * dim[j];
    dim[i] = v;
  }
  return true;
}

inline int store(const i128* src, int64_t* dst, size_t cnt) {
  int rc = 0;
  for (size_t i = 0; i < cnt; ++i) {
    if (src[i] > (i128)INT64_MAX || src[i] < (i128)INT64_MIN) rc = 7;
    dst[i] = (int64_t)src[i];
  }
  return rc;
}

}  // namespace

extern "C" {

// 0 on success; the pattern/orbit/A tables failed their own consistency checks otherwise.
int oracle_tables_ok() { return tables().ok ? 0 : 1; }

// orbit_of[j*5 + x] = orbit number of vertex x (0-based) of pattern H_j, -1 beyond k
int oracle_pattern_orbits(int* k_of, int* orbit_of, int* orbit_size) {
  const Tables& t = tables();
  if (!t.ok) return 1;
  for (int j = 0; j < 30; ++j) {
    k_of[j] = t.pat[j].k;
    for (int x = 0; x < 5; ++x) orbit_of[j * 5 + x] = x < t.pat[j].k ? t.pat[j].orbit[x] : -1;
  }
  for (int o = 0; o < 73; ++o) orbit_size[o] = t.orbit_size[o];
  return 0;
}

// pattern edges as adjacency matrices adj[j*25 + a*5 + b]
int oracle_pattern_adj(int* adj) {
  const Tables& t = tables();
  if (!t.ok) return 1;
  for (int j = 0; j < 30; ++j)
    for (int a = 0; a < 5; ++a)
      for (int b = 0; b < 5; ++b) adj[j * 25 + a * 5 + b] = t.pat[j].adj[a][b];
  return 0;
}

int oracle_A_matrix(int64_t* A) {
  const Tables& t = tables();
  if (!t.ok) return 1;
  for (int i = 0; i < 73; ++i)
    for (int j = 0; j < 73; ++j) A[i * 73 + j] = t.A[i][j];
  return 0;
}

// Brute force (the definition).  dim: n*73 induced counts.  dm (optional):
// n*73 non-induced counts by enumerating connected spanning edge subsets.
int oracle_brute_force(const int64_t* rowptr, const uint32_t* col, uint32_t n, int64_t* dim,
                       int64_t* dm, int threads) {
  const Tables& t = tables();
  if (!t.ok) return 1;
  G g{n, rowptr, col};
  const int nt = nthreads_of(threads);
  std::vector<std::vector<ll>> pd(nt, std::vector<ll>((size_t)n * 73, 0));
  std::vector<std::vector<ll>> pm(dm ? nt : 0, std::vector<ll>((size_t)n * 73, 0));
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t r = 0; r < (int64_t)n; ++r) {
    int th = thread_id();
    Esu e{g, t, pd[th].data(), dm ? pm[th].data() : nullptr, (uint32_t)r};
    e.sub[0] = (uint32_t)r;
    e.ns = 1;
    std::vector<uint32_t> ext;
    for (int64_t s = rowptr[r]; s < rowptr[r + 1]; ++s)
      if (col[s] > (uint32_t)r) ext.push_back(col[s]);
    e.extend(ext);
  }
  for (size_t i = 0; i < (size_t)n * 73; ++i) {
    ll a = 0, b = 0;
    for (int th = 0; th < nt; ++th) {
      a += pd[th][i];
      if (dm) b += pm[th][i];
    }
    dim[i] = a;
    if (dm) dm[i] = b;
  }
  return 0;
}

// The paper's method.  dm (optional): non-induced counts; dim (optional):
// induced counts.  Returns 7 if any value leaves int64.
int oracle_formulas(const int64_t* rowptr, const uint32_t* col, uint32_t n, int64_t* dm,
                    int64_t* dim, int threads) {
  const Tables& t = tables();
  if (!t.ok) return 1;
  G g{n, rowptr, col};
  Formula f(g, threads);
  f.run();
  int rc = f.overflow ? 7 : 0;
  if (dm) rc |= store(f.DM.data(), dm, (size_t)n * 73);
  if (dim) {
    std::vector<i128> out((size_t)n * 73);
#pragma omp parallel for num_threads(nthreads_of(threads))
    for (int64_t u = 0; u < (int64_t)n; ++u)
      invert_apply(t, &f.DM[(size_t)u * 73], &out[(size_t)u * 73]);
    rc |= store(out.data(), dim, (size_t)n * 73);
  }
  return rc;
}

// The 4-vertex orbits only (Thm. 4orbit: Lem. 4vertexorbit, then the 4-vertex
// block of A^-1).  dim: n*15 induced counts of orbits 0..14.
int oracle_formulas4(const int64_t* rowptr, const uint32_t* col, uint32_t n, int64_t* dim,
                     int threads) {
  const Tables& t = tables();
  if (!t.ok) return 1;
  G g{n, rowptr, col};
  Formula f(g, threads);
  f.four_only = true;
  f.run();
  int rc = f.overflow ? 7 : 0;
  std::vector<i128> out(73);
  for (uint32_t u = 0; u < n; ++u) {
    // orbits 15..72 of f.DM are zero; A is block diagonal by pattern size
    if (!invert_apply(t, &f.DM[(size_t)u * 73], out.data())) rc = 7;
    rc |= store(out.data(), dim + (size_t)u * 15, 15);
  }
  return rc;
}

// Per-slot edge quantities of Lem. 4edgeorbit and per-vertex T, C4, K4, for
// intermediate checks: each output array has rowptr[n] entries (slot (u,v) =
// position of v in row u); E9 is the ordered count E9<u,v>.
int oracle_edge_counts(const int64_t* rowptr, const uint32_t* col, uint32_t n, int64_t* T,
                       int64_t* C4, int64_t* K4, int64_t* E7, int64_t* E9, int threads) {
  const Tables& t = tables();
  if (!t.ok) return 1;
  G g{n, rowptr, col};
  Formula f(g, threads);
  f.run();
  const int64_t S = rowptr[n];
  for (int64_t s = 0; s < S; ++s) {
    T[s] = f.Te[s]; C4[s] = f.C4e[s]; K4[s] = f.K4e[s]; E7[s] = f.E7e[s]; E9[s] = f.E9e[s];
  }
  return f.overflow ? 7 : 0;
}

// Edge orbits by the definition: out [rowptr[n] * 12], row = slot (u,v),
// column i = E_i<u,v> (Fig. edge_orbits, the Definition after it), by
// enumerating every connected 3- and 4-vertex subset and its connected
// spanning edge subsets.  Tiny graphs only.
int oracle_edge_orbits_brute(const int64_t* rowptr, const uint32_t* col, uint32_t n, int64_t* out,
                             int threads) {
  const Tables& t = tables();
  if (!t.ok) return 1;
  G g{n, rowptr, col};
  const int nt = nthreads_of(threads);
  const size_t S = (size_t)rowptr[n];
  std::vector<std::vector<ll>> pe(nt, std::vector<ll>(S * 12, 0));
  std::vector<std::vector<ll>> pd(nt, std::vector<ll>((size_t)n * 73, 0));
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t r = 0; r < (int64_t)n; ++r) {
    int th = thread_id();
    Esu e{g, t, pd[th].data(), nullptr, (uint32_t)r};
    e.eo = pe[th].data();
    e.kmax = 4;
    e.sub[0] = (uint32_t)r;
    e.ns = 1;
    std::vector<uint32_t> ext;
    for (int64_t s = rowptr[r]; s < rowptr[r + 1]; ++s)
      if (col[s] > (uint32_t)r) ext.push_back(col[s]);
    e.extend(ext);
  }
  for (size_t i = 0; i < S * 12; ++i) {
    ll a = 0;
    for (int th = 0; th < nt; ++th) a += pe[th][i];
    out[i] = a;
  }
  return 0;
}

// Edge orbits by Lem. 4edgeorbit, from the base counts of the paper's method.
int oracle_edge_orbits_formula(const int64_t* rowptr, const uint32_t* col, uint32_t n,
                               int64_t* out, int threads) {
  const Tables& t = tables();
  if (!t.ok) return 1;
  G g{n, rowptr, col};
  Formula f(g, threads);
  f.run();
  std::vector<i128> Tu(n, 0), dm1(n, 0);  // T(u) and DM1(u) = sum over N(u) of d(v)-1
  for (uint32_t u = 0; u < n; ++u)
    for (int64_t s = rowptr[u]; s < rowptr[u + 1]; ++s) {
      Tu[u] += f.Te[s];
      dm1[u] += g.deg(col[s]) - 1;
    }
  for (uint32_t u = 0; u < n; ++u) Tu[u] /= 2;
  int rc = f.overflow ? 7 : 0;
  for (uint32_t u = 0; u < n; ++u)
    for (int64_t s = rowptr[u]; s < rowptr[u + 1]; ++s) {
      const uint32_t v = col[s];
      const i128 du = g.deg(u), dv = g.deg(v), T = f.Te[s];
      i128 e[12];
      e[0] = du - 1;
      e[1] = T;
      e[2] = (dm1[u] - (dv - 1)) - T;  // sum over x in N(u)\v of (d(x)-1), minus E1
      e[3] = (du - 1) * (dv - 1) - T;
      e[4] = C2(du - 1);
      e[5] = f.C4e[s];
      e[6] = Tu[u] - T;                 // r(theta_3) matches at u, minus E1
      e[7] = f.E7e[s];
      e[8] = T * (du - 2);
      e[9] = f.E9e[s];
      e[10] = C2(T);
      e[11] = f.K4e[s];
      rc |= store(e, out + (size_t)s * 12, 12);
    }
  return rc;
}

int oracle_max_threads() { return nthreads_of(0); }

}  // extern "C"
