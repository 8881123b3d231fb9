/*
 * Seeded synthetic graph generators: the INPUT side of every test and
 * benchmark. Both the CPU oracle and the CUDA path consume what this file
 * produces; it holds none of the mining arithmetic (no intersections, no
 * counting, no orientation), only graph sampling and CSR assembly.
 *
 * Output format (the paper's input convention, Section 6 "Input graphs"):
 * an undirected simple graph as a symmetric CSR with no self-loops, no
 * duplicate edges and every neighbour list sorted ascending.
 *   rowptr: uint64[n+1], col: uint32[rowptr[n]].
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * SplitMix64 (Steele, Lea & Flood, 2014), both written from their published
 * definitions. Every generator is single-threaded and therefore bit-for-bit
 * reproducible on any x86-64 host for a given seed.
 *
 * Generators:
 *   R-MAT     Chakrabarti, Zhan & Faloutsos (SDM 2004): ef * 2^scale edge
 *             samples, recursive quadrant choice with probabilities
 *             (a,b,c,d), no per-level noise, then a seeded random vertex
 *             permutation (counts are invariant under it).
 *   Chung-Lu  expected-degree model with power-law weights, sampled with the
 *             O(n+m) skipping method of Miller & Hagberg (WAW 2011).
 *   G(n,p)    Erdos-Renyi via geometric skipping (Batagelj & Brandes 2005).
 *
 * Ownership: every *_out array is malloc'd here and released by gg_free().
 * Return value: 0 on success, -1 on invalid arguments, -2 on allocation
 * failure.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------- PRNG ---------------- */

typedef struct {
  uint64_t s[4];
} gg_rng;

static uint64_t splitmix64(uint64_t *x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static void rng_seed(gg_rng *r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(gg_rng *r) {
  uint64_t *s = r->s;
  uint64_t out = rotl64(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
  return out;
}

/* uniform double in [0,1) with 53 random bits */
static inline double rng_unif(gg_rng *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0, bound) by Lemire's multiply-shift with rejection */
static uint64_t rng_below(gg_rng *r, uint64_t bound) {
  for (;;) {
    uint64_t x = rng_next(r);
    __uint128_t m = (__uint128_t)x * bound;
    uint64_t lo = (uint64_t)m;
    if (lo >= bound || lo >= (uint64_t)(-bound) % bound) return (uint64_t)(m >> 64);
  }
}

/* seeded Fisher-Yates permutation of 0..n-1 */
static uint32_t *random_permutation(uint32_t n, gg_rng *r) {
  uint32_t *p = (uint32_t *)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
  if (!p) return NULL;
  for (uint32_t i = 0; i < n; ++i) p[i] = i;
  for (uint32_t i = n; i > 1; --i) {
    uint32_t j = (uint32_t)rng_below(r, i);
    uint32_t t = p[i - 1];
    p[i - 1] = p[j];
    p[j] = t;
  }
  return p;
}

/* ---------------- edge buffer ---------------- */

typedef struct {
  uint32_t *u, *v;
  uint64_t len, cap;
} edge_buf;

static int eb_push(edge_buf *b, uint32_t u, uint32_t v) {
  if (b->len == b->cap) {
    uint64_t nc = b->cap ? b->cap * 2 : 1024;
    uint32_t *nu = (uint32_t *)realloc(b->u, nc * sizeof(uint32_t));
    if (!nu) return -2;
    b->u = nu;
    uint32_t *nv = (uint32_t *)realloc(b->v, nc * sizeof(uint32_t));
    if (!nv) return -2;
    b->v = nv;
    b->cap = nc;
  }
  b->u[b->len] = u;
  b->v[b->len] = v;
  b->len++;
  return 0;
}

static void eb_free(edge_buf *b) {
  free(b->u);
  free(b->v);
  b->u = b->v = NULL;
  b->len = b->cap = 0;
}

/* ---------------- CSR assembly ---------------- */

static unsigned bits_for(uint64_t n) {
  unsigned b = 1;
  while (b < 64 && (1ULL << b) < n) ++b;
  return b;
}

/* LSD radix sort of 64-bit keys on their low `nbits` bits, 16 bits per pass */
static int radix_sort_u64(uint64_t *a, uint64_t len, unsigned nbits) {
  if (len < 2) return 0;
  uint64_t *tmp = (uint64_t *)malloc(len * sizeof(uint64_t));
  if (!tmp) return -2;
  uint64_t *cnt = (uint64_t *)malloc(65536 * sizeof(uint64_t));
  if (!cnt) {
    free(tmp);
    return -2;
  }
  uint64_t *src = a, *dst = tmp;
  for (unsigned shift = 0; shift < nbits; shift += 16) {
    memset(cnt, 0, 65536 * sizeof(uint64_t));
    for (uint64_t i = 0; i < len; ++i) cnt[(src[i] >> shift) & 0xFFFF]++;
    uint64_t sum = 0;
    for (int d = 0; d < 65536; ++d) {
      uint64_t c = cnt[d];
      cnt[d] = sum;
      sum += c;
    }
    for (uint64_t i = 0; i < len; ++i) dst[cnt[(src[i] >> shift) & 0xFFFF]++] = src[i];
    uint64_t *t = src;
    src = dst;
    dst = t;
  }
  if (src != a) memcpy(a, src, len * sizeof(uint64_t));
  free(cnt);
  free(tmp);
  return 0;
}

/* Symmetrise, drop self-loops and duplicates, sort: edge list -> CSR. */
static int build_csr(uint32_t n, const uint32_t *eu, const uint32_t *ev, uint64_t ne, uint64_t **rowptr_out,
                     uint32_t **col_out, uint64_t *nnz_out) {
  unsigned b = bits_for((uint64_t)n);
  uint64_t *keys = (uint64_t *)malloc((2 * ne + 1) * sizeof(uint64_t));
  if (!keys) return -2;
  uint64_t k = 0;
  for (uint64_t i = 0; i < ne; ++i) {
    uint32_t u = eu[i], v = ev[i];
    if (u == v) continue;
    keys[k++] = ((uint64_t)u << b) | v;
    keys[k++] = ((uint64_t)v << b) | u;
  }
  if (radix_sort_u64(keys, k, 2 * b)) {
    free(keys);
    return -2;
  }
  uint64_t w = 0;
  for (uint64_t i = 0; i < k; ++i)
    if (i == 0 || keys[i] != keys[i - 1]) keys[w++] = keys[i];
  uint64_t *rowptr = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
  uint32_t *col = (uint32_t *)malloc((w ? w : 1) * sizeof(uint32_t));
  if (!rowptr || !col) {
    free(keys);
    free(rowptr);
    free(col);
    return -2;
  }
  uint64_t mask = (b >= 64) ? ~0ULL : ((1ULL << b) - 1);
  for (uint64_t i = 0; i < w; ++i) {
    rowptr[(keys[i] >> b) + 1]++;
    col[i] = (uint32_t)(keys[i] & mask);
  }
  for (uint32_t i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
  free(keys);
  *rowptr_out = rowptr;
  *col_out = col;
  *nnz_out = w;
  return 0;
}

/* ---------------- public entry points ---------------- */

void gg_free(void *p) { free(p); }

int gg_csr_from_edges(uint32_t n, const uint32_t *src, const uint32_t *dst, uint64_t ne, uint64_t **rowptr_out,
                      uint32_t **col_out, uint64_t *nnz_out) {
  if (!rowptr_out || !col_out || !nnz_out) return -1;
  for (uint64_t i = 0; i < ne; ++i)
    if (src[i] >= n || dst[i] >= n) return -1;
  return build_csr(n, src, dst, ne, rowptr_out, col_out, nnz_out);
}

int gg_rmat(uint32_t scale, double edge_factor, double a, double b, double c, uint64_t seed, int permute,
            uint64_t **rowptr_out, uint32_t **col_out, uint64_t *nnz_out) {
  if (scale < 1 || scale > 30 || edge_factor <= 0.0 || a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return -1;
  uint32_t n = 1u << scale;
  uint64_t ns = (uint64_t)llround(edge_factor * (double)n);
  gg_rng r;
  rng_seed(&r, seed);
  uint32_t *eu = (uint32_t *)malloc((ns ? ns : 1) * sizeof(uint32_t));
  uint32_t *ev = (uint32_t *)malloc((ns ? ns : 1) * sizeof(uint32_t));
  if (!eu || !ev) {
    free(eu);
    free(ev);
    return -2;
  }
  const double ab = a + b, abc = a + b + c;
  for (uint64_t i = 0; i < ns; ++i) {
    uint32_t u = 0, v = 0;
    for (uint32_t lvl = 0; lvl < scale; ++lvl) {
      double x = rng_unif(&r);
      uint32_t bit = 1u << (scale - 1 - lvl);
      if (x < a) {
      } else if (x < ab) {
        v |= bit;
      } else if (x < abc) {
        u |= bit;
      } else {
        u |= bit;
        v |= bit;
      }
    }
    eu[i] = u;
    ev[i] = v;
  }
  if (permute) {
    uint32_t *p = random_permutation(n, &r);
    if (!p) {
      free(eu);
      free(ev);
      return -2;
    }
    for (uint64_t i = 0; i < ns; ++i) {
      eu[i] = p[eu[i]];
      ev[i] = p[ev[i]];
    }
    free(p);
  }
  int rc = build_csr(n, eu, ev, ns, rowptr_out, col_out, nnz_out);
  free(eu);
  free(ev);
  return rc;
}

/* Chung-Lu weights: w_i proportional to (i + i0)^(-1/(gamma-1)), scaled so
 * that the mean weight is dbar, with the offset i0 chosen so that the largest
 * weight equals the structural cutoff sqrt(sum w). Then every pair
 * probability w_i w_j / sum(w) is at most 1 and no probability is clipped. */
static double *chung_lu_weights(uint32_t n, double dbar, double gamma) {
  double *w = (double *)malloc((size_t)n * sizeof(double));
  if (!w) return NULL;
  const double alpha = 1.0 / (gamma - 1.0);
  const double S = dbar * (double)n;
  const double target = sqrt(S);
  double lo = log(1e-3), hi = log((double)n);
  for (int it = 0; it < 48; ++it) {
    double i0 = exp(0.5 * (lo + hi));
    double sum = 0.0;
    for (uint32_t i = 0; i < n; ++i) sum += pow((double)i + i0, -alpha);
    double w0 = S * pow(i0, -alpha) / sum;
    if (w0 > target)
      lo = log(i0); /* largest weight too big: move the offset up */
    else
      hi = log(i0);
  }
  double i0 = exp(hi);
  double sum = 0.0;
  for (uint32_t i = 0; i < n; ++i) {
    w[i] = pow((double)i + i0, -alpha);
    sum += w[i];
  }
  for (uint32_t i = 0; i < n; ++i) w[i] *= S / sum;
  return w;
}

int gg_chung_lu(uint32_t n, double dbar, double gamma, uint64_t seed, int permute, uint64_t **rowptr_out,
                uint32_t **col_out, uint64_t *nnz_out, double *max_weight_out) {
  if (n < 2 || dbar <= 0.0 || gamma <= 2.0) return -1;
  double *w = chung_lu_weights(n, dbar, gamma);
  if (!w) return -2;
  double S = 0.0;
  for (uint32_t i = 0; i < n; ++i) S += w[i];
  if (max_weight_out) *max_weight_out = w[0];
  gg_rng r;
  rng_seed(&r, seed);
  edge_buf eb = {0};
  /* Miller-Hagberg: weights are non-increasing in i, so for a fixed u the
   * pair probability is non-increasing in v; skip geometrically with the
   * current upper bound p and accept with q/p. */
  for (uint32_t u = 0; u + 1 < n; ++u) {
    uint64_t v = (uint64_t)u + 1;
    double p = w[u] * w[v] / S;
    if (p > 1.0) p = 1.0;
    while (v < n && p > 0.0) {
      if (p < 1.0) {
        double x = 1.0 - rng_unif(&r); /* (0,1] */
        double skip = floor(log(x) / log1p(-p));
        if (skip > (double)n) break;
        v += (uint64_t)skip;
      }
      if (v < n) {
        double q = w[u] * w[v] / S;
        if (q > 1.0) q = 1.0;
        double x = rng_unif(&r);
        if (x < q / p) {
          if (eb_push(&eb, u, (uint32_t)v)) {
            eb_free(&eb);
            free(w);
            return -2;
          }
        }
        p = q;
        v += 1;
      }
    }
  }
  free(w);
  if (permute) {
    uint32_t *p = random_permutation(n, &r);
    if (!p) {
      eb_free(&eb);
      return -2;
    }
    for (uint64_t i = 0; i < eb.len; ++i) {
      eb.u[i] = p[eb.u[i]];
      eb.v[i] = p[eb.v[i]];
    }
    free(p);
  }
  int rc = build_csr(n, eb.u, eb.v, eb.len, rowptr_out, col_out, nnz_out);
  eb_free(&eb);
  return rc;
}

int gg_erdos_renyi(uint32_t n, double p, uint64_t seed, int permute, uint64_t **rowptr_out, uint32_t **col_out,
                   uint64_t *nnz_out) {
  if (n < 1 || p < 0.0 || p > 1.0) return -1;
  gg_rng r;
  rng_seed(&r, seed);
  edge_buf eb = {0};
  if (p > 0.0) {
    /* Batagelj-Brandes: walk the strictly lower triangle (v > w) in row-major
     * order, jumping geometric gaps between successive edges. */
    int64_t v = 1, w = -1;
    const double lq = log1p(-p);
    while (v < (int64_t)n) {
      if (p < 1.0) {
        double x = 1.0 - rng_unif(&r);
        double skip = floor(log(x) / lq);
        if (skip > 4.0 * (double)n * (double)n) break;
        w += 1 + (int64_t)skip;
      } else {
        w += 1;
      }
      while (w >= v && v < (int64_t)n) {
        w -= v;
        v += 1;
      }
      if (v < (int64_t)n) {
        if (eb_push(&eb, (uint32_t)v, (uint32_t)w)) {
          eb_free(&eb);
          return -2;
        }
      }
    }
  }
  if (permute) {
    uint32_t *pp = random_permutation(n, &r);
    if (!pp) {
      eb_free(&eb);
      return -2;
    }
    for (uint64_t i = 0; i < eb.len; ++i) {
      eb.u[i] = pp[eb.u[i]];
      eb.v[i] = pp[eb.v[i]];
    }
    free(pp);
  }
  int rc = build_csr(n, eb.u, eb.v, eb.len, rowptr_out, col_out, nnz_out);
  eb_free(&eb);
  return rc;
}
