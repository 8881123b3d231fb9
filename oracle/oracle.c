/*
 * CPU ORACLE -- test infrastructure only.
 *
 * A plain, slow, single-threaded C restatement of what the graph-pattern-
 * mining hot path computes. Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load it; the library's product path never
 * does. It shares no code, header, table or helper with the CUDA library.
 *
 * Every count is an exact unsigned integer. Sums are accumulated in 128-bit
 * integers and a result that does not fit in 64 bits is reported as an error
 * (return value ORC_E_OVERFLOW) instead of wrapping.
 *
 * Graph input: undirected simple graph, symmetric CSR with sorted neighbour
 * lists, no self-loops, no duplicates (the paper's input convention, Section 6).
 *
 * Two tiers:
 *  tier 1 (brute force, tiny graphs): the definitions of Section 2 and the
 *    appendix "Subgraphs, Subgraph Trees and Patterns" written out: every
 *    k-subset (vertex-induced) or every injective map (edge-induced).
 *  tier 2 (exact plain algorithms, any size): the paper's own search
 *    decompositions (orientation, matching order, local counting) with plain
 *    merge intersections and no blocking or reordering; each is pinned by
 *    tier 1 and by closed forms in the tests.
 *
 * Order used for orientation (appendix "Orientation (Total Order)"):
 *   a < b  iff  (deg a, a) < (deg b, b)    -- edges point to the higher degree,
 *                                            ties to the larger vertex id.
 * Root conventions for root-range restricted counts (so that a count over a
 * range of root vertices can be compared piece by piece):
 *   k-clique : the clique vertex that is minimal in the order above;
 *   diamond  : the order-minimal endpoint of the edge shared by both triangles;
 *   4-cycle  : the cycle vertex that is maximal in the order above.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_E_ARG -1
#define ORC_E_OOM -2
#define ORC_E_OVERFLOW -3
#define ORC_E_CAP -4

typedef unsigned __int128 u128;
typedef __int128 i128;

static const u128 U64_LIMIT = ((u128)1) << 64;

/* ------------------------------------------------------------------ */
/* basic graph queries                                                 */
/* ------------------------------------------------------------------ */

static uint64_t deg_of(const uint64_t *rp, uint32_t v) { return rp[v + 1] - rp[v]; }

/* binary search for v in the sorted neighbour list of u */
static int adjacent(const uint64_t *rp, const uint32_t *col, uint32_t u, uint32_t v) {
  uint64_t lo = rp[u], hi = rp[u + 1];
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (col[mid] < v)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo < rp[u + 1] && col[lo] == v;
}

/* a precedes b in the degree order (appendix "Orientation (Total Order)") */
static int precedes(const uint64_t *rp, uint32_t a, uint32_t b) {
  uint64_t da = deg_of(rp, a), db = deg_of(rp, b);
  return da < db || (da == db && a < b);
}

/* |A ∩ B| of two ascending arrays, by merging */
static uint64_t merge_count(const uint32_t *a, uint64_t na, const uint32_t *b, uint64_t nb) {
  uint64_t i = 0, j = 0, c = 0;
  while (i < na && j < nb) {
    if (a[i] < b[j])
      ++i;
    else if (a[i] > b[j])
      ++j;
    else {
      ++c;
      ++i;
      ++j;
    }
  }
  return c;
}

/* A ∩ B written to out (ascending); returns its size */
static uint64_t merge_into(const uint32_t *a, uint64_t na, const uint32_t *b, uint64_t nb, uint32_t *out) {
  uint64_t i = 0, j = 0, c = 0;
  while (i < na && j < nb) {
    if (a[i] < b[j])
      ++i;
    else if (a[i] > b[j])
      ++j;
    else {
      out[c++] = a[i];
      ++i;
      ++j;
    }
  }
  return c;
}

/* ------------------------------------------------------------------ */
/* patterns: automorphisms and isomorphism (tier 1 helpers)            */
/* ------------------------------------------------------------------ */

/* next permutation of p[0..k-1] in lexicographic order; 0 when done */
static int next_perm(uint32_t *p, uint32_t k) {
  if (k < 2) return 0;
  int32_t i = (int32_t)k - 2;
  while (i >= 0 && p[i] >= p[i + 1]) --i;
  if (i < 0) return 0;
  int32_t j = (int32_t)k - 1;
  while (p[j] <= p[i]) --j;
  uint32_t t = p[i];
  p[i] = p[j];
  p[j] = t;
  for (uint32_t a = (uint32_t)i + 1, b = k - 1; a < b; ++a, --b) {
    t = p[a];
    p[a] = p[b];
    p[b] = t;
  }
  return 1;
}

/* Number of automorphisms of the k-vertex pattern with adjacency padj
 * (k*k row-major 0/1): permutations s with padj[s(i)][s(j)] == padj[i][j]. */
uint64_t orc_automorphisms(uint32_t k, const uint8_t *padj) {
  uint32_t p[16];
  for (uint32_t i = 0; i < k; ++i) p[i] = i;
  uint64_t count = 0;
  do {
    int ok = 1;
    for (uint32_t i = 0; i < k && ok; ++i)
      for (uint32_t j = 0; j < k; ++j)
        if ((padj[p[i] * k + p[j]] != 0) != (padj[i * k + j] != 0)) {
          ok = 0;
          break;
        }
    count += ok;
  } while (next_perm(p, k));
  return count;
}

/* ------------------------------------------------------------------ */
/* tier 1: brute force over k-subsets and injective maps               */
/* ------------------------------------------------------------------ */

/* Vertex-induced count (Section 2, k-MC, TC and k-CL use vertex-induced
 * subgraphs): number of k-subsets W of V with G[W] isomorphic to P, decided by
 * trying all k! bijections. Intended for n <= ~40. */
int orc_bf_induced(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t k, const uint8_t *padj,
                   uint64_t *out) {
  if (k < 1 || k > 8) return ORC_E_ARG;
  if (k > n) {
    *out = 0;
    return ORC_OK;
  }
  uint32_t w[16], p[16];
  uint8_t g[64];
  for (uint32_t i = 0; i < k; ++i) w[i] = i;
  u128 count = 0;
  for (;;) {
    for (uint32_t i = 0; i < k; ++i)
      for (uint32_t j = 0; j < k; ++j) g[i * k + j] = (i != j) && adjacent(rp, col, w[i], w[j]);
    for (uint32_t i = 0; i < k; ++i) p[i] = i;
    int iso = 0;
    do {
      int ok = 1;
      for (uint32_t i = 0; i < k && ok; ++i)
        for (uint32_t j = 0; j < k; ++j)
          if ((padj[i * k + j] != 0) != (g[p[i] * k + p[j]] != 0)) {
            ok = 0;
            break;
          }
      if (ok) {
        iso = 1;
        break;
      }
    } while (next_perm(p, k));
    count += (u128)iso;
    /* next k-combination of 0..n-1 */
    int32_t i = (int32_t)k - 1;
    while (i >= 0 && w[i] == n - k + (uint32_t)i) --i;
    if (i < 0) break;
    w[i]++;
    for (uint32_t j = (uint32_t)i + 1; j < k; ++j) w[j] = w[j - 1] + 1;
  }
  *out = (uint64_t)count;
  return ORC_OK;
}

/* Edge-induced (non-induced) count (Section 2, SL): the number of subgraphs
 * of G isomorphic to P = #{injective f: V_P -> V, every pattern edge maps to a
 * graph edge} / |Aut(P)|. Intended for n <= ~40, k <= 5. */
int orc_bf_noninduced(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t k, const uint8_t *padj,
                      uint64_t *out) {
  if (k < 1 || k > 8) return ORC_E_ARG;
  if (k > n) {
    *out = 0;
    return ORC_OK;
  }
  uint32_t f[16];
  u128 maps = 0;
  /* depth-first over injective maps, checking pattern edges to earlier positions */
  int32_t depth = 0;
  f[0] = 0;
  for (;;) {
    if (f[depth] >= n) {
      if (depth == 0) break;
      --depth;
      f[depth]++;
      continue;
    }
    int ok = 1;
    for (int32_t j = 0; j < depth && ok; ++j) {
      if (f[j] == f[depth]) ok = 0;
      else if (padj[(uint32_t)depth * k + (uint32_t)j] && !adjacent(rp, col, f[depth], f[j]))
        ok = 0;
    }
    if (!ok) {
      f[depth]++;
      continue;
    }
    if ((uint32_t)depth == k - 1) {
      maps++;
      f[depth]++;
      continue;
    }
    ++depth;
    f[depth] = 0;
  }
  uint64_t aut = orc_automorphisms(k, padj);
  if (aut == 0 || maps % aut != 0) return ORC_E_ARG;
  u128 c = maps / aut;
  if (c >= U64_LIMIT) return ORC_E_OVERFLOW;
  *out = (uint64_t)c;
  return ORC_OK;
}

/* All injective maps f (as k-tuples, pattern vertex order) of P into G with
 * every pattern edge on a graph edge; tuples written to out (k*cap). Returns
 * the number of maps in *nmaps (even beyond cap). Used by the tests to form
 * the set of distinct embeddings (edge sets) for listing parity. */
int orc_bf_maps(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t k, const uint8_t *padj, uint32_t *out,
                uint64_t cap, uint64_t *nmaps) {
  if (k < 1 || k > 8) return ORC_E_ARG;
  *nmaps = 0;
  if (k > n) return ORC_OK;
  uint32_t f[16];
  int32_t depth = 0;
  f[0] = 0;
  uint64_t cnt = 0;
  for (;;) {
    if (f[depth] >= n) {
      if (depth == 0) break;
      --depth;
      f[depth]++;
      continue;
    }
    int ok = 1;
    for (int32_t j = 0; j < depth && ok; ++j) {
      if (f[j] == f[depth]) ok = 0;
      else if (padj[(uint32_t)depth * k + (uint32_t)j] && !adjacent(rp, col, f[depth], f[j]))
        ok = 0;
    }
    if (!ok) {
      f[depth]++;
      continue;
    }
    if ((uint32_t)depth == k - 1) {
      if (cnt < cap)
        for (uint32_t i = 0; i < k; ++i) out[cnt * k + i] = f[i];
      cnt++;
      f[depth]++;
      continue;
    }
    ++depth;
    f[depth] = 0;
  }
  *nmaps = cnt;
  return cnt > cap ? ORC_E_CAP : ORC_OK;
}

/* ------------------------------------------------------------------ */
/* tier 2: orientation (appendix "Orientation (Total Order)")          */
/* ------------------------------------------------------------------ */

typedef struct {
  uint64_t *rp; /* n+1 */
  uint32_t *col;
} out_csr;

/* N+(v) = { w in N(v) : v precedes w }, kept in ascending id order */
static int orient(uint32_t n, const uint64_t *rp, const uint32_t *col, out_csr *o) {
  o->rp = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
  if (!o->rp) return ORC_E_OOM;
  for (uint32_t v = 0; v < n; ++v) {
    uint64_t c = 0;
    for (uint64_t e = rp[v]; e < rp[v + 1]; ++e) c += precedes(rp, v, col[e]);
    o->rp[v + 1] = o->rp[v] + c;
  }
  o->col = (uint32_t *)malloc((o->rp[n] ? o->rp[n] : 1) * sizeof(uint32_t));
  if (!o->col) {
    free(o->rp);
    return ORC_E_OOM;
  }
  for (uint32_t v = 0; v < n; ++v) {
    uint64_t w = o->rp[v];
    for (uint64_t e = rp[v]; e < rp[v + 1]; ++e)
      if (precedes(rp, v, col[e])) o->col[w++] = col[e];
  }
  return ORC_OK;
}

static void free_out(out_csr *o) {
  free(o->rp);
  free(o->col);
}

/* Out-degree of every vertex in the oriented graph (for the tests). */
int orc_out_degrees(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t *outdeg) {
  for (uint32_t v = 0; v < n; ++v) {
    uint32_t c = 0;
    for (uint64_t e = rp[v]; e < rp[v + 1]; ++e) c += precedes(rp, v, col[e]);
    outdeg[v] = c;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* tier 2: k-cliques over the orientation (Section 2 k-CL; the local   */
/* graph search of Section 5 "Search on Local Graph" in set form)      */
/* ------------------------------------------------------------------ */

/* number of ways to complete a clique with `need` more vertices, all drawn
 * from the candidate set cand (every member adjacent to all chosen ones) */
static u128 extend_clique(const out_csr *o, const uint32_t *cand, uint64_t nc, uint32_t need, uint32_t *scratch,
                          uint64_t stride) {
  if (need == 1) return nc;
  u128 total = 0;
  uint32_t *next = scratch;
  for (uint64_t i = 0; i < nc; ++i) {
    uint32_t x = cand[i];
    uint64_t nn = merge_into(cand, nc, o->col + o->rp[x], o->rp[x + 1] - o->rp[x], next);
    if (nn + 1 >= need) total += extend_clique(o, next, nn, need - 1, scratch + stride, stride);
  }
  return total;
}

/* k-cliques whose order-minimal vertex lies in [root_lo, root_hi). k >= 1. */
int orc_cliques(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t k, uint32_t root_lo, uint32_t root_hi,
                uint64_t *out) {
  if (k < 1 || k > 16 || root_lo > root_hi || root_hi > n) return ORC_E_ARG;
  if (k == 1) {
    *out = root_hi - root_lo;
    return ORC_OK;
  }
  out_csr o;
  int rc = orient(n, rp, col, &o);
  if (rc) return rc;
  uint64_t maxd = 0;
  for (uint32_t v = 0; v < n; ++v)
    if (o.rp[v + 1] - o.rp[v] > maxd) maxd = o.rp[v + 1] - o.rp[v];
  uint64_t stride = maxd + 1;
  uint32_t *scratch = (uint32_t *)malloc(stride * (k + 1) * sizeof(uint32_t));
  if (!scratch) {
    free_out(&o);
    return ORC_E_OOM;
  }
  u128 total = 0;
  for (uint32_t u = root_lo; u < root_hi; ++u)
    total += extend_clique(&o, o.col + o.rp[u], o.rp[u + 1] - o.rp[u], k - 1, scratch, stride);
  free(scratch);
  free_out(&o);
  if (total >= U64_LIMIT) return ORC_E_OVERFLOW;
  *out = (uint64_t)total;
  return ORC_OK;
}

/* Core numbers (appendix "Orientation (Total Order)", the core value based
 * order): core[v] is the largest c such that v belongs to a subgraph whose
 * every vertex has degree >= c in it. Textbook peeling with a bucket queue
 * (Batagelj and Zaversnik 2003): take a vertex of minimum remaining degree,
 * fix its core number, lower the remaining degree of its neighbours that
 * are still present (never below the current core number). */
int orc_core_numbers(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t *core) {
  uint32_t md = 0;
  for (uint32_t v = 0; v < n; ++v)
    if (deg_of(rp, v) > md) md = (uint32_t)deg_of(rp, v);
  uint32_t *d = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
  uint32_t *bin = (uint32_t *)calloc((size_t)md + 2, sizeof(uint32_t));
  uint32_t *pos = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
  uint32_t *vert = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
  if (!d || !bin || !pos || !vert) {
    free(d), free(bin), free(pos), free(vert);
    return ORC_E_OOM;
  }
  for (uint32_t v = 0; v < n; ++v) {
    d[v] = (uint32_t)deg_of(rp, v);
    bin[d[v]]++;
  }
  uint32_t start = 0; /* bin[x] = first slot of degree x in vert */
  for (uint32_t x = 0; x <= md; ++x) {
    uint32_t c = bin[x];
    bin[x] = start;
    start += c;
  }
  for (uint32_t v = 0; v < n; ++v) {
    pos[v] = bin[d[v]];
    vert[pos[v]] = v;
    bin[d[v]]++;
  }
  for (uint32_t x = md; x > 0; --x) bin[x] = bin[x - 1];
  bin[0] = 0;
  for (uint32_t i = 0; i < n; ++i) {
    uint32_t v = vert[i];
    for (uint64_t e = rp[v]; e < rp[v + 1]; ++e) {
      uint32_t u = col[e];
      if (d[u] > d[v]) {
        /* move u to the front of its bucket, then one bucket down */
        uint32_t du = d[u], pu = pos[u], pw = bin[du], w = vert[pw];
        if (u != w) {
          pos[u] = pw;
          vert[pu] = w;
          pos[w] = pu;
          vert[pw] = u;
        }
        bin[du]++;
        d[u]--;
      }
    }
  }
  for (uint32_t v = 0; v < n; ++v) core[v] = d[v];
  free(d), free(bin), free(pos), free(vert);
  return ORC_OK;
}

/* The degeneracy order of level-synchronous peeling (the reading taken of the
 * core value based order): at level k, every vertex still present with
 * remaining degree <= k is taken in round r; taking a round's vertices lowers
 * the remaining degree of their neighbours still present, and those that
 * drop to k are taken in round r + 1 (same level); an empty level moves to
 * the smallest remaining degree. order[v] = the round that took v. Written
 * as plain sequential loops over whole rounds, so the rounds are the sets the
 * definition gives whatever the processing order within a round. */
int orc_core_order(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t *order) {
  uint32_t *d = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
  unsigned char *taken = (unsigned char *)calloc((size_t)n + 1, 1);
  uint32_t *cur = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
  uint32_t *nxt = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
  if (!d || !taken || !cur || !nxt) {
    free(d), free(taken), free(cur), free(nxt);
    return ORC_E_OOM;
  }
  for (uint32_t v = 0; v < n; ++v) d[v] = (uint32_t)deg_of(rp, v);
  uint64_t left = n;
  uint32_t k = 0, round = 0;
  while (left > 0) {
    uint32_t nc = 0, mn = UINT32_MAX;
    for (uint32_t v = 0; v < n; ++v) {
      if (taken[v]) continue;
      if (d[v] <= k) {
        taken[v] = 1;
        order[v] = round;
        cur[nc++] = v;
      } else if (d[v] < mn) {
        mn = d[v];
      }
    }
    if (nc == 0) {
      k = mn;
      continue;
    }
    while (nc > 0) {
      left -= nc;
      uint32_t nn = 0;
      for (uint32_t i = 0; i < nc; ++i) {
        uint32_t v = cur[i];
        for (uint64_t e = rp[v]; e < rp[v + 1]; ++e) {
          uint32_t w = col[e];
          if (taken[w]) continue;
          if (--d[w] == k) {
            taken[w] = 1;
            order[w] = round + 1;
            nxt[nn++] = w;
          }
        }
      }
      uint32_t *t = cur;
      cur = nxt;
      nxt = t;
      nc = nn;
      ++round;
    }
    ++k;
  }
  free(d), free(taken), free(cur), free(nxt);
  return ORC_OK;
}

/* k-cliques whose first vertex in the order (key, id) lies in [root_lo,
 * root_hi): the same search over the orientation v -> w iff (key v, v) <
 * (key w, w). With key = the core numbers this is the core value based
 * orientation of the appendix; the total over all roots does not depend on
 * the order. */
int orc_cliques_keyed(uint32_t n, const uint64_t *rp, const uint32_t *col, const uint32_t *key, uint32_t k,
                      uint32_t root_lo, uint32_t root_hi, uint64_t *out) {
  if (k < 2 || k > 16 || root_lo > root_hi || root_hi > n) return ORC_E_ARG;
  out_csr o;
  o.rp = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
  if (!o.rp) return ORC_E_OOM;
  for (uint32_t v = 0; v < n; ++v) {
    uint64_t c = 0;
    for (uint64_t e = rp[v]; e < rp[v + 1]; ++e) {
      uint32_t w = col[e];
      c += key[v] < key[w] || (key[v] == key[w] && v < w);
    }
    o.rp[v + 1] = o.rp[v] + c;
  }
  o.col = (uint32_t *)malloc((o.rp[n] ? o.rp[n] : 1) * sizeof(uint32_t));
  if (!o.col) {
    free(o.rp);
    return ORC_E_OOM;
  }
  uint64_t maxd = 0;
  for (uint32_t v = 0; v < n; ++v) {
    uint64_t w = o.rp[v];
    for (uint64_t e = rp[v]; e < rp[v + 1]; ++e) {
      uint32_t x = col[e];
      if (key[v] < key[x] || (key[v] == key[x] && v < x)) o.col[w++] = x;
    }
    if (o.rp[v + 1] - o.rp[v] > maxd) maxd = o.rp[v + 1] - o.rp[v];
  }
  uint64_t stride = maxd + 1;
  uint32_t *scratch = (uint32_t *)malloc(stride * (k + 1) * sizeof(uint32_t));
  if (!scratch) {
    free_out(&o);
    return ORC_E_OOM;
  }
  u128 total = 0;
  for (uint32_t u = root_lo; u < root_hi; ++u)
    total += extend_clique(&o, o.col + o.rp[u], o.rp[u + 1] - o.rp[u], k - 1, scratch, stride);
  free(scratch);
  free_out(&o);
  if (total >= U64_LIMIT) return ORC_E_OVERFLOW;
  *out = (uint64_t)total;
  return ORC_OK;
}

/* Triangles (Section 2, TC): 3-cliques. */
int orc_triangles(uint32_t n, const uint64_t *rp, const uint32_t *col, uint64_t *out) {
  return orc_cliques(n, rp, col, 3, 0, n, out);
}

/* ------------------------------------------------------------------ */
/* tier 2: edge-induced diamonds by local counting (Section 5 "Local   */
/* Counting": sum over edges of C(n_t, 2), n_t = triangles on the edge) */
/* ------------------------------------------------------------------ */

/* diamonds whose shared edge has its order-minimal endpoint in [lo, hi) */
int orc_diamonds(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t root_lo, uint32_t root_hi,
                 uint64_t *out) {
  if (root_lo > root_hi || root_hi > n) return ORC_E_ARG;
  u128 total = 0;
  for (uint32_t a = root_lo; a < root_hi; ++a)
    for (uint64_t e = rp[a]; e < rp[a + 1]; ++e) {
      uint32_t b = col[e];
      if (!precedes(rp, a, b)) continue;
      uint64_t t = merge_count(col + rp[a], rp[a + 1] - rp[a], col + rp[b], rp[b + 1] - rp[b]);
      if (t >= 2) total += (u128)t * (t - 1) / 2;
    }
  if (total >= U64_LIMIT) return ORC_E_OVERFLOW;
  *out = (uint64_t)total;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* tier 2: edge-induced 4-cycles (Section 2 SL)                         */
/* ------------------------------------------------------------------ */

/* 4-cycles whose order-maximal vertex v0 lies in [lo, hi). For each v0, every
 * wedge v0 - x - w with x and w both preceding v0 is tallied at w; a 4-cycle
 * with maximal vertex v0 and opposite vertex w is exactly a pair of such
 * wedges, so it is counted once by C(tally(w), 2). */
int orc_cycles4(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t root_lo, uint32_t root_hi,
                uint64_t *out) {
  if (root_lo > root_hi || root_hi > n) return ORC_E_ARG;
  uint64_t *tally = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
  uint32_t *touched = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
  if (!tally || !touched) {
    free(tally);
    free(touched);
    return ORC_E_OOM;
  }
  u128 total = 0;
  for (uint32_t v0 = root_lo; v0 < root_hi; ++v0) {
    uint64_t nt = 0;
    for (uint64_t e = rp[v0]; e < rp[v0 + 1]; ++e) {
      uint32_t x = col[e];
      if (!precedes(rp, x, v0)) continue;
      for (uint64_t f = rp[x]; f < rp[x + 1]; ++f) {
        uint32_t w = col[f];
        if (!precedes(rp, w, v0)) continue;
        if (tally[w]++ == 0) touched[nt++] = w;
      }
    }
    for (uint64_t i = 0; i < nt; ++i) {
      uint64_t c = tally[touched[i]];
      total += (u128)c * (c - 1) / 2;
      tally[touched[i]] = 0;
    }
  }
  free(tally);
  free(touched);
  if (total >= U64_LIMIT) return ORC_E_OVERFLOW;
  *out = (uint64_t)total;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* tier 2: motif counting by local counting (Section 5 "Local Counting",*/
/* Eq. 1, the 3-MC and 4-MC local-count listings of the appendix)       */
/* ------------------------------------------------------------------ */

/* Non-induced (edge-induced) counts of the connected 4-vertex patterns,
 * order: [3-star, 4-path, tailed-triangle, 4-cycle, diamond, 4-clique].
 *   3-star          = sum_v C(d_v, 3)
 *   4-path          = sum_{uv in E} (d_u - 1)(d_v - 1) - 3 T
 *   tailed triangle = sum_v t_v (d_v - 2),  t_v = triangles through v
 *   4-cycle         = orc_cycles4
 *   diamond         = sum_e C(t_e, 2),      t_e = triangles on edge e
 *   4-clique        = orc_cliques(k = 4)
 * 3-vertex order: [wedge (2-path), triangle]: sum_v C(d_v, 2) and T. */
int orc_noninduced_terms(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t k, uint64_t *out) {
  if (k != 3 && k != 4) return ORC_E_ARG;
  u128 s2 = 0, s3 = 0;
  for (uint32_t v = 0; v < n; ++v) {
    u128 d = deg_of(rp, v);
    if (d >= 2) s2 += d * (d - 1) / 2;
    if (d >= 3) s3 += d * (d - 1) * (d - 2) / 6;
  }
  /* per-edge triangle counts by merging full neighbour lists */
  u128 tri3 = 0, paths = 0, diam = 0;
  uint64_t *tv = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
  if (!tv) return ORC_E_OOM;
  for (uint32_t u = 0; u < n; ++u)
    for (uint64_t e = rp[u]; e < rp[u + 1]; ++e) {
      uint32_t v = col[e];
      if (v <= u) continue;
      uint64_t t = merge_count(col + rp[u], rp[u + 1] - rp[u], col + rp[v], rp[v + 1] - rp[v]);
      tri3 += t;
      tv[u] += t;
      tv[v] += t;
      paths += (u128)(deg_of(rp, u) - 1) * (deg_of(rp, v) - 1);
      if (t >= 2) diam += (u128)t * (t - 1) / 2;
    }
  if (tri3 % 3 != 0) {
    free(tv);
    return ORC_E_ARG;
  }
  u128 T = tri3 / 3;
  if (k == 3) {
    free(tv);
    if (s2 >= U64_LIMIT || T >= U64_LIMIT) return ORC_E_OVERFLOW;
    out[0] = (uint64_t)s2;
    out[1] = (uint64_t)T;
    return ORC_OK;
  }
  u128 tailed = 0;
  for (uint32_t v = 0; v < n; ++v) {
    /* tv[v] counts each triangle through v twice (once per incident edge) */
    u128 t = tv[v] / 2;
    uint64_t d = deg_of(rp, v);
    if (d >= 2) tailed += t * (d - 2);
  }
  free(tv);
  u128 p4 = paths - 3 * T;
  uint64_t c4, k4;
  int rc = orc_cycles4(n, rp, col, 0, n, &c4);
  if (rc) return rc;
  rc = orc_cliques(n, rp, col, 4, 0, n, &k4);
  if (rc) return rc;
  if (s3 >= U64_LIMIT || p4 >= U64_LIMIT || tailed >= U64_LIMIT || diam >= U64_LIMIT) return ORC_E_OVERFLOW;
  out[0] = (uint64_t)s3;
  out[1] = (uint64_t)p4;
  out[2] = (uint64_t)tailed;
  out[3] = c4;
  out[4] = (uint64_t)diam;
  out[5] = k4;
  return ORC_OK;
}

/* Induced motif counts from the non-induced ones. A non-induced count of
 * pattern X is the sum over patterns Y of (induced count of Y) times the
 * number of spanning copies of X inside Y; the matrix is unitriangular in the
 * order 4-clique, diamond, 4-cycle, tailed triangle, 4-path, 3-star, so it is
 * solved from the densest pattern down:
 *   K4 in K4: 1          D in K4: 6            C4 in K4: 3, in D: 1
 *   TT in K4: 12, D: 4   P in K4: 12, D: 6, C4: 4, TT: 2
 *   S in K4: 4, D: 2, TT: 1
 * 3-vertex: triangle = T, open wedge = sum C(d,2) - 3 T (appendix 3-MC listing). */
int orc_motifs(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t k, uint64_t *out) {
  uint64_t N[6];
  int rc = orc_noninduced_terms(n, rp, col, k, N);
  if (rc) return rc;
  if (k == 3) {
    i128 wedge = (i128)N[0] - 3 * (i128)N[1];
    if (wedge < 0) return ORC_E_ARG;
    out[0] = (uint64_t)wedge;
    out[1] = N[1];
    return ORC_OK;
  }
  i128 S = N[0], P = N[1], TT = N[2], C4 = N[3], D = N[4], K4 = N[5];
  i128 iK4 = K4;
  i128 iD = D - 6 * iK4;
  i128 iC4 = C4 - iD - 3 * iK4;
  i128 iTT = TT - 4 * iD - 12 * iK4;
  i128 iP = P - 2 * iTT - 4 * iC4 - 6 * iD - 12 * iK4;
  i128 iS = S - iTT - 2 * iD - 4 * iK4;
  i128 v[6] = {iS, iP, iTT, iC4, iD, iK4};
  for (int i = 0; i < 6; ++i) {
    if (v[i] < 0 || v[i] >= (i128)U64_LIMIT) return ORC_E_ARG;
    out[i] = (uint64_t)v[i];
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* 5-vertex motifs (Section 2 k-MC for k = 5): every connected induced   */
/* 5-vertex subgraph, enumerated once by ESU (Wernicke 2006: extend a   */
/* connected set only by vertices after its first vertex and outside   */
/* the neighbourhood of the set so far), classified by isomorphism     */
/* class through a canonical adjacency mask (minimum over the 120      */
/* vertex permutations).                                                */
/* ------------------------------------------------------------------ */

/* pair (i, j), i < j, of 5 vertices -> bit index 0..9 in lexicographic order */
static int pair_bit5(int i, int j) {
  static const int base[4] = {0, 4, 7, 9};
  if (i > j) {
    int t = i;
    i = j;
    j = t;
  }
  return base[i] + (j - i - 1);
}

static uint32_t canon5(uint32_t mask) {
  uint32_t best = 0xffffffffu;
  int p[5];
  /* the 120 permutations p of {0..4}: vertex i of the mask becomes p[i] */
  for (p[0] = 0; p[0] < 5; ++p[0])
    for (p[1] = 0; p[1] < 5; ++p[1])
      for (p[2] = 0; p[2] < 5; ++p[2])
        for (p[3] = 0; p[3] < 5; ++p[3])
          for (p[4] = 0; p[4] < 5; ++p[4]) {
            int used = (1 << p[0]) | (1 << p[1]) | (1 << p[2]) | (1 << p[3]) | (1 << p[4]);
            if (used != 31) continue;
            uint32_t m = 0;
            for (int i = 0; i < 5; ++i)
              for (int j = i + 1; j < 5; ++j)
                if (mask >> pair_bit5(i, j) & 1u) m |= 1u << pair_bit5(p[i], p[j]);
            if (m < best) best = m;
          }
  return best;
}

static int connected5(uint32_t mask) {
  uint32_t seen = 1u, grow = 1u;
  while (grow) {
    uint32_t next = 0;
    for (int i = 0; i < 5; ++i)
      if (grow >> i & 1u)
        for (int j = 0; j < 5; ++j)
          if (j != i && (mask >> pair_bit5(i, j) & 1u) && !(seen >> j & 1u)) next |= 1u << j;
    seen |= next;
    grow = next;
  }
  return seen == 31u;
}

/* class index of every 10-bit mask (255 = not connected); classes ordered
 * by edge count, then by canonical mask */
static int motif5_table(uint8_t *cls, uint32_t *class_mask) {
  uint32_t canon[1024];
  int nc = 0;
  for (uint32_t m = 0; m < 1024; ++m) canon[m] = connected5(m) ? canon5(m) : 0xffffffffu;
  for (uint32_t m = 0; m < 1024; ++m) {
    if (canon[m] != m) continue; /* m is canonical and connected */
    class_mask[nc++] = m;
  }
  for (int i = 1; i < nc; ++i) /* insertion sort by (edges, mask) */
    for (int j = i; j > 0; --j) {
      uint32_t a = class_mask[j - 1], b = class_mask[j];
      int ea = __builtin_popcount(a), eb = __builtin_popcount(b);
      if (ea < eb || (ea == eb && a < b)) break;
      class_mask[j - 1] = b;
      class_mask[j] = a;
    }
  for (uint32_t m = 0; m < 1024; ++m) {
    cls[m] = 255;
    if (canon[m] == 0xffffffffu) continue;
    for (int i = 0; i < nc; ++i)
      if (class_mask[i] == canon[m]) cls[m] = (uint8_t)i;
  }
  return nc;
}

typedef struct {
  const uint64_t *rp;
  const uint32_t *col;
  const uint8_t *cls;
  uint64_t *cnt;
  uint32_t *ext_pool; /* 5 levels */
  uint64_t level_cap;
  uint32_t v;
} esu_ctx;

static void esu_extend(esu_ctx *x, uint32_t *sub, int ns, const uint32_t *ext, uint64_t next, int level) {
  if (ns == 5) {
    uint32_t mask = 0;
    for (int i = 0; i < 5; ++i)
      for (int j = i + 1; j < 5; ++j)
        if (adjacent(x->rp, x->col, sub[i], sub[j])) mask |= 1u << pair_bit5(i, j);
    x->cnt[x->cls[mask]]++;
    return;
  }
  uint32_t *ext2 = x->ext_pool + (uint64_t)level * x->level_cap;
  while (next > 0) {
    uint32_t w = ext[--next];
    uint64_t n2 = 0;
    for (uint64_t i = 0; i < next; ++i) ext2[n2++] = ext[i];
    for (uint64_t e = x->rp[w]; e < x->rp[w + 1]; ++e) {
      uint32_t u = x->col[e];
      if (u <= x->v) continue;
      int excl = 1;
      for (int i = 0; i < ns && excl; ++i)
        if (u == sub[i] || adjacent(x->rp, x->col, sub[i], u)) excl = 0;
      if (excl) ext2[n2++] = u;
    }
    sub[ns] = w;
    esu_extend(x, sub, ns + 1, ext2, n2, level + 1);
  }
}

/* Induced counts of the 21 connected 5-vertex patterns; class_mask[i] is the
 * canonical adjacency mask of class i (edge {a, b} of vertices 0..4 at the
 * bit pair_bit5(a, b) gives: pairs in lexicographic order (0,1) = bit 0 ...
 * (3,4) = bit 9); classes ordered by edge count, then by mask. */
int orc_motifs5_roots(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t root_lo, uint32_t root_hi,
                      uint64_t *out, uint32_t *class_mask);
int orc_motifs5(uint32_t n, const uint64_t *rp, const uint32_t *col, uint64_t *out, uint32_t *class_mask) {
  return orc_motifs5_roots(n, rp, col, 0, n, out, class_mask);
}

/* As orc_motifs5, restricted to the subgraphs whose smallest vertex (the
 * root ESU extends from) lies in [root_lo, root_hi). */
int orc_motifs5_roots(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t root_lo, uint32_t root_hi,
                      uint64_t *out, uint32_t *class_mask) {
  uint8_t cls[1024];
  uint32_t cm[32];
  int nc = motif5_table(cls, cm);
  if (nc != 21) return ORC_E_ARG;
  uint64_t maxd = 0;
  for (uint32_t v = 0; v < n; ++v)
    if (deg_of(rp, v) > maxd) maxd = deg_of(rp, v);
  esu_ctx x;
  x.rp = rp;
  x.col = col;
  x.cls = cls;
  x.cnt = out;
  x.level_cap = 5 * maxd + 1;
  x.ext_pool = (uint32_t *)malloc(6 * x.level_cap * sizeof(uint32_t));
  if (!x.ext_pool) return ORC_E_OOM;
  for (int i = 0; i < 21; ++i) {
    out[i] = 0;
    if (class_mask) class_mask[i] = cm[i];
  }
  uint32_t sub[5];
  if (root_hi > n) root_hi = n;
  for (uint32_t v = root_lo; v < root_hi; ++v) {
    x.v = v;
    uint32_t *ext = x.ext_pool;
    uint64_t ne = 0;
    for (uint64_t e = rp[v]; e < rp[v + 1]; ++e)
      if (col[e] > v) ext[ne++] = col[e];
    sub[0] = v;
    esu_extend(&x, sub, 1, ext, ne, 1);
  }
  free(x.ext_pool);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* worked examples of the paper                                        */
/* ------------------------------------------------------------------ */

/* Eq. 1: local wedge count of edge (u,v) from its local triangle count. */
int64_t orc_eq1_local_wedges(int64_t deg_u, int64_t deg_v, int64_t c_tri) {
  return (deg_u - c_tri - 1) + (deg_v - c_tri - 1);
}

/* Induced wedges (open 2-paths) that contain edge (u,v), counted directly:
 * vertices adjacent to exactly one of u, v (other than u and v). */
int orc_edge_wedges_direct(const uint64_t *rp, const uint32_t *col, uint32_t u, uint32_t v, uint64_t *out) {
  uint64_t c = 0;
  for (uint64_t e = rp[u]; e < rp[u + 1]; ++e)
    if (col[e] != v && !adjacent(rp, col, v, col[e])) ++c;
  for (uint64_t e = rp[v]; e < rp[v + 1]; ++e)
    if (col[e] != u && !adjacent(rp, col, u, col[e])) ++c;
  *out = c;
  return ORC_OK;
}

/* Memoization of embedding connectivity (Section 4.2, appendix "Example for
 * Connectivity Code"): for an embedding emb[0..len-1] the code of the vertex
 * at level l has bit i set iff it is adjacent to emb[i], i < l. The codes are
 * concatenated level by level (level 1 first), most significant bit first.
 * Returns the number of code bits; the code itself is written to *code. */
int orc_connectivity_code(const uint64_t *rp, const uint32_t *col, const uint32_t *emb, uint32_t len,
                          uint64_t *code) {
  uint64_t c = 0;
  int nbits = 0;
  for (uint32_t l = 1; l < len; ++l)
    for (uint32_t i = 0; i < l; ++i) {
      c = (c << 1) | (uint64_t)adjacent(rp, col, emb[l], emb[i]);
      ++nbits;
    }
  *code = c;
  return nbits;
}

/* Rebuild the k x k adjacency of an embedding from its connectivity code. */
int orc_code_to_adjacency(uint32_t k, uint64_t code, uint8_t *adj) {
  int nbits = (int)(k * (k - 1) / 2);
  memset(adj, 0, (size_t)k * k);
  int pos = nbits - 1;
  for (uint32_t l = 1; l < k; ++l)
    for (uint32_t i = 0; i < l; ++i) {
      uint8_t b = (uint8_t)((code >> pos) & 1u);
      adj[l * k + i] = adj[i * k + l] = b;
      --pos;
    }
  return ORC_OK;
}

/* Memoization of neighbourhood connectivity (Section 4.3, MNC): the bit-vector
 * of embedding positions whose vertex is adjacent to v. */
uint64_t orc_connectivity_map_lookup(const uint64_t *rp, const uint32_t *col, const uint32_t *emb, uint32_t len,
                                     uint32_t v) {
  uint64_t bits = 0;
  for (uint32_t i = 0; i < len; ++i)
    if (emb[i] != v && adjacent(rp, col, v, emb[i])) bits |= 1ULL << i;
  return bits;
}

/* Symmetry breaking (appendix "Symmetry Breaking (Partial Order)"): given a
 * list of pairs (a_i, b_i) meaning f(a_i) < f(b_i), count the permutations of
 * 0..k-1 (as vertex id assignments) satisfying all of them. With correct
 * constraints this times |Aut(P)| equals k!. */
uint64_t orc_orders_satisfying(uint32_t k, const uint32_t *pairs, uint32_t npairs) {
  uint32_t p[16];
  for (uint32_t i = 0; i < k; ++i) p[i] = i;
  uint64_t c = 0;
  do {
    int ok = 1;
    for (uint32_t i = 0; i < npairs; ++i)
      if (!(p[pairs[2 * i]] < p[pairs[2 * i + 1]])) {
        ok = 0;
        break;
      }
    c += ok;
  } while (next_perm(p, k));
  return c;
}
