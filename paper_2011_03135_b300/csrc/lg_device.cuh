// Device building blocks of the local-graph clique search, shared by the
// per-class kernels (clique.cu) and the batched persistent kernel (batch.cu).
// See clique.cu for the method.
#pragma once

#include <stdint.h>

namespace gpm_dev {

// Bitmap rows are stored with an odd stride (words + 1 when the word count is
// even) so that rows read by different lanes fall in different shared-memory
// banks.
__host__ __device__ constexpr uint32_t row_stride(uint32_t words) { return words | 1u; }

__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t *a, uint32_t n, uint32_t x) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// largest i in [0, n) with pre[i] <= f (pre ascending, pre[0] = 0 <= f)
__device__ __forceinline__ uint32_t row_of(const uint32_t *pre, uint32_t n, uint32_t f) {
  uint32_t lo = 0, hi = n;  // invariant: pre[lo] <= f, answer in [lo, hi)
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (pre[mid] <= f) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Flat expansion of one root's local graph. Threads [t0, t0 + nt) of the
// calling group cooperate; the caller synchronises before and after.
// perm (optional): row and bit positions of L[i] (see rank_local); the
// triangle-count scatter keeps id positions.
// ROWS = false (triangles only): the bitmap is not written.
template <bool SCATTER, bool ROWS = true>
__device__ __forceinline__ uint32_t build_rows(const uint32_t *__restrict__ dcol, uint32_t *t_edge, const uint32_t *L,
                                               const uint32_t *pre,
                                               const uint64_t *xb, uint32_t *R, uint32_t *tc, uint32_t d,
                                               uint32_t rs, uint32_t t, uint32_t nt, const uint32_t *perm = nullptr) {
  const uint32_t E = pre[d];
  uint32_t found = 0;
  const uint32_t lo_id = L[0], hi_id = L[d - 1];
  for (uint32_t f = t; f < E; f += nt) {
    const uint32_t i = row_of(pre, d, f);
    const uint32_t p = f - pre[i];
    const uint64_t arc = xb[i] + p;
    const uint32_t y = __ldg(dcol + arc);
    if (y < lo_id || y > hi_id) continue;
    const uint32_t j = lower_bound_u32(L, d, y);
    if (j < d && L[j] == y) {
      const uint32_t ri = perm ? perm[i] : i, rj = perm ? perm[j] : j;
      if (ROWS) atomicOr(&R[(size_t)ri * rs + (rj >> 5)], 1u << (rj & 31));
      ++found;
      if (SCATTER) {
        atomicAdd(&tc[i], 1u);
        atomicAdd(&tc[j], 1u);
        atomicAdd(&t_edge[arc], 1u);
      }
    }
  }
  return found;
}

// Position table of L for build_rows_runs: open addressing on the vertex id
// with 2^hbits >= 4d slots (keys, then values). Built by the whole CTA; the
// caller synchronises before and after.
constexpr uint32_t kPosEmpty = 0xffffffffu;
__device__ __forceinline__ uint32_t pos_hash(uint32_t y, uint32_t hbits) { return (y * 0x9E3779B1u) >> (32 - hbits); }

__device__ __forceinline__ void build_pos_table(const uint32_t *L, uint32_t d, uint32_t *hk, uint32_t hbits,
                                                uint32_t t, uint32_t nt) {
  const uint32_t ns = 1u << hbits, mask = ns - 1;
  uint32_t *hv = hk + ns;
  for (uint32_t i = t; i < ns; i += nt) hk[i] = kPosEmpty;
  __syncthreads();
  for (uint32_t i = t; i < d; i += nt) {
    const uint32_t y = L[i];
    uint32_t h = pos_hash(y, hbits);
    while (atomicCAS(&hk[h], kPosEmpty, y) != kPosEmpty) h = (h + 1) & mask;  // ids in L are distinct
    hv[h] = i;
  }
}

// build_rows with four consecutive elements per thread (one search for the
// row of the first, then a forward step) and, given a position table hk, the
// element lookup in it (about two probes instead of a binary search over L).
template <bool SCATTER, bool ROWS = true>
__device__ __forceinline__ uint32_t build_rows_runs(const uint32_t *__restrict__ dcol, uint32_t *t_edge,
                                                      const uint32_t *L, const uint32_t *pre, const uint64_t *xb,
                                                      uint32_t *R, uint32_t *tc, uint32_t d, uint32_t rs, uint32_t t,
                                                      uint32_t nt, const uint32_t *perm, const uint32_t *hk,
                                                      uint32_t hbits) {
  const uint32_t E = pre[d], mask = (1u << hbits) - 1;
  const uint32_t *hv = hk ? hk + (1u << hbits) : nullptr;
  uint32_t found = 0;
  const uint32_t lo_id = L[0], hi_id = L[d - 1];
  for (uint32_t f0 = 4 * t; f0 < E; f0 += 4 * nt) {
    uint32_t i = row_of(pre, d, f0);
    uint32_t rowi[4];
    uint64_t arc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t f = f0 + q;
      if (f < E) {
        while (pre[i + 1] <= f) ++i;
        rowi[q] = i;
        arc[q] = xb[i] + (f - pre[i]);
      } else {
        rowi[q] = 0xffffffffu;
        arc[q] = 0;
      }
    }
    uint32_t y[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) y[q] = (rowi[q] != 0xffffffffu) ? __ldg(dcol + arc[q]) : 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (rowi[q] == 0xffffffffu || y[q] < lo_id || y[q] > hi_id) continue;
      uint32_t j = kPosEmpty;
      if (hk) {
        uint32_t h = pos_hash(y[q], hbits);
        for (;;) {
          const uint32_t k = hk[h];
          if (k == y[q]) {
            j = hv[h];
            break;
          }
          if (k == kPosEmpty) break;
          h = (h + 1) & mask;
        }
      } else {
        const uint32_t jj = lower_bound_u32(L, d, y[q]);
        if (jj < d && L[jj] == y[q]) j = jj;
      }
      if (j == kPosEmpty) continue;
      const uint32_t ii = rowi[q];
      const uint32_t ri = perm ? perm[ii] : ii, rj = perm ? perm[j] : j;
      if (ROWS) atomicOr(&R[(size_t)ri * rs + (rj >> 5)], 1u << (rj & 31));
      ++found;
      if (SCATTER) {
        atomicAdd(&tc[ii], 1u);
        atomicAdd(&tc[j], 1u);
        atomicAdd(&t_edge[arc[q]], 1u);
      }
    }
  }
  return found;
}

// Enumerate pairs (i, j in R_i), triples and (KMAX 6) quadruples for the 4-,
// 5- and 6-clique terms. A group of G lanes handles one row at a time; lane gl
// of the group holds word gl of the row (W <= G), so every AND is one word
// per lane.
template <int G, int KMAX>
__device__ __forceinline__ void enumerate_rows(const uint32_t *R, uint32_t d, uint32_t W, uint32_t rs, uint32_t row0,
                                               uint32_t row_step, uint32_t gl, unsigned long long &a4,
                                               unsigned long long &a5, unsigned long long &a6) {
  for (uint32_t i = row0; i < d; i += row_step) {
    const uint32_t *ri = R + (size_t)i * rs;
    const uint32_t riw = (gl < W) ? ri[gl] : 0u;
    for (uint32_t t = 0; t < W; ++t) {
      uint32_t bits = ri[t];
      while (bits) {
        const uint32_t j = t * 32 + __ffs(bits) - 1;
        bits &= bits - 1;
        const uint32_t *rj = R + (size_t)j * rs;
        const uint32_t mw = (gl < W) ? (riw & rj[gl]) : 0u;
        a4 += __popc(mw);
        if (KMAX >= 5) {
          for (uint32_t t2 = 0; t2 < W; ++t2) {
            uint32_t b2 = ri[t2] & rj[t2];
            while (b2) {
              const uint32_t l = t2 * 32 + __ffs(b2) - 1;
              b2 &= b2 - 1;
              const uint32_t *rl = R + (size_t)l * rs;
              const uint32_t m5 = (gl < W) ? (mw & rl[gl]) : 0u;
              a5 += __popc(m5);
              if (KMAX >= 6) {
                for (uint32_t t3 = 0; t3 < W; ++t3) {
                  uint32_t b3 = ri[t3] & rj[t3] & rl[t3];
                  while (b3) {
                    const uint32_t y = t3 * 32 + __ffs(b3) - 1;
                    b3 &= b3 - 1;
                    if (gl < W) a6 += __popc(m5 & R[(size_t)y * rs + gl]);
                  }
                }
              }
            }
          }
        }
      }
    }
  }
}

// Same for W > 32 (global-memory class): lane gl holds words gl, gl+G, ...
template <int KMAX>
__device__ inline void enumerate_rows_wide(const uint32_t *R, uint32_t d, uint32_t W, uint32_t rs, uint32_t row0,
                                           uint32_t row_step, uint32_t gl, unsigned long long &a4,
                                           unsigned long long &a5, unsigned long long &a6) {
  constexpr uint32_t G = 32;
  for (uint32_t i = row0; i < d; i += row_step) {
    const uint32_t *ri = R + (size_t)i * rs;
    for (uint32_t t = 0; t < W; ++t) {
      uint32_t bits = ri[t];
      while (bits) {
        const uint32_t j = t * 32 + __ffs(bits) - 1;
        bits &= bits - 1;
        const uint32_t *rj = R + (size_t)j * rs;
        for (uint32_t w = gl; w < W; w += G) a4 += __popc(ri[w] & rj[w]);
        if (KMAX >= 5) {
          for (uint32_t t2 = 0; t2 < W; ++t2) {
            uint32_t b2 = ri[t2] & rj[t2];
            while (b2) {
              const uint32_t l = t2 * 32 + __ffs(b2) - 1;
              b2 &= b2 - 1;
              const uint32_t *rl = R + (size_t)l * rs;
              for (uint32_t w = gl; w < W; w += G) a5 += __popc(ri[w] & rj[w] & rl[w]);
              if (KMAX >= 6) {
                for (uint32_t t3 = 0; t3 < W; ++t3) {
                  uint32_t b3 = ri[t3] & rj[t3] & rl[t3];
                  while (b3) {
                    const uint32_t y = t3 * 32 + __ffs(b3) - 1;
                    b3 &= b3 - 1;
                    const uint32_t *ry = R + (size_t)y * rs;
                    for (uint32_t w = gl; w < W; w += G) a6 += __popc(ri[w] & rj[w] & rl[w] & ry[w]);
                  }
                }
              }
            }
          }
        }
      }
    }
  }
}



// ---------------------------------------------------------------------------
// Nested local graph for the 5-clique level (CTA roots).
//
// For row i of the root's local graph, the candidates of the next level are
// S = R_i (c vertices). Compacting every row R_j, j in S, to the positions of
// S (a bit-gather) gives the local graph of the next level, C (c rows of
// W' = ceil(c/32) words), on which
//   4-cliques through (u, L[i]) = sum_a |C_a|
//   5-cliques through (u, L[i]) = sum_a sum_{b in C_a} |C_a & C_b|
// -- the paper's shrinking local graph, one more level down. A row of width
// W' is far narrower than W for most i, so the last level costs W' words per
// visited 4-clique instead of W, and one thread walks one compacted row.
// ---------------------------------------------------------------------------
// Rows with c <= wcap (64 or 128) are nested by one warp; a warp's buffer holds
// S[wcap] pref[32] C[wcap rows of row_stride(wcap/32) words].
constexpr uint32_t kNestWarpC = 128;  // largest wcap
__host__ __device__ constexpr uint32_t nest_warp_words(uint32_t wcap) {
  return wcap + 32 + wcap * row_stride(wcap / 32);
}

__host__ __device__ constexpr uint64_t nest_words(uint32_t maxd, uint32_t nwarps, uint32_t big_cap,
                                                  uint32_t wcap = kNestWarpC) {
  // counters[4], big-row list[maxd], wide-row list[maxd], then a pool that
  // holds the warps' buffers in the warp phase, and the groups' (or the
  // CTA's) S[maxd] pref[32] C[...] in the big-row phases
  return 4ull + 2ull * maxd + (uint64_t)nwarps * nest_warp_words(wcap) + maxd + 32 + big_cap;
}

// named barrier over `nthreads` threads (a multiple of 32) of the CTA
__device__ __forceinline__ void group_bar(uint32_t id, uint32_t nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Number of set bits of row ri (W <= 32 words); when it is at most cap, their
// positions go to S (ascending) and per-word prefix counts to pref. Called by
// one whole warp.
__device__ __forceinline__ uint32_t list_bits_warp(const uint32_t *ri, uint32_t W, uint32_t *S, uint32_t *pref,
                                                   uint32_t cap) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t x = (lane < W) ? ri[lane] : 0u;
  const uint32_t cnt = __popc(x);
  uint32_t incl = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
  if (total > cap) return total;
  uint32_t k = incl - cnt;
  if (lane < W) pref[lane] = k;
  while (x) {
    const uint32_t p = __ffs(x) - 1;
    x &= x - 1;
    S[k++] = lane * 32 + p;
  }
  __syncwarp();
  return total;
}

// Gather the bits of x (a subset of riw) to the low popc(riw) positions, in
// order: the bits of one input word land in one contiguous output range.
__device__ __forceinline__ uint32_t gather_bits(uint32_t x, uint32_t riw) {
  uint32_t out = 0;
  while (x) {
    const uint32_t p = __ffs(x) - 1;
    x &= x - 1;
    out |= 1u << __popc(riw & ((1u << p) - 1u));
  }
  return out;
}

// compact row R_j (j = S[a]) onto the positions of ri into crow (Wp words,
// zeroed here); returns |R_j & R_i|
// (words of rj below w0 are known to be zero)
__device__ __forceinline__ uint32_t compact_row(const uint32_t *rj, const uint32_t *ri, const uint32_t *pref, uint32_t W,
                                                uint32_t *crow, uint32_t Wp, uint32_t w0 = 0) {
  for (uint32_t k = 0; k < Wp; ++k) crow[k] = 0u;
  uint32_t bits = 0;
  for (uint32_t w = w0; w < W; ++w) {
    const uint32_t riw = ri[w];
    const uint32_t x = rj[w] & riw;
    if (!x) continue;
    const uint32_t out = gather_bits(x, riw);
    bits += __popc(x);
    const uint32_t base = pref[w], wi = base >> 5, lo = base & 31;
    crow[wi] |= out << lo;
    if (lo && lo + __popc(riw) > 32) crow[wi + 1] |= out >> (32 - lo);
  }
  return bits;
}

// sum over the set bits b in word k of row a of |C_a & C_b| (rows of Wp words,
// stride Wp); one (a, k) unit bounds a thread's loop to 32 bits
// (with tri, C is strictly upper triangular: C_b has no bit below b + 1).
// With K6, s6 also gets sum over x in C_a & C_b of |C_a & C_b & C_x|.
template <bool K6 = false>
__device__ __forceinline__ unsigned long long nested_pairs_unit(const uint32_t *C, uint32_t a, uint32_t k,
                                                                uint32_t Wp, uint32_t cs, bool tri,
                                                                unsigned long long &s6) {
  const uint32_t *ca = C + (size_t)a * cs;
  uint32_t s = 0;  // at most 32 x 32 x Wp
  uint32_t bits = ca[k];
  while (bits) {
    const uint32_t b = k * 32 + __ffs(bits) - 1;
    bits &= bits - 1;
    const uint32_t *cb = C + (size_t)b * cs;
    for (uint32_t k2 = tri ? (b + 1) >> 5 : 0; k2 < Wp; ++k2) {
      const uint32_t m = ca[k2] & cb[k2];
      s += __popc(m);
      if (K6) {
        uint32_t mx = m;
        while (mx) {
          const uint32_t x = k2 * 32 + __ffs(mx) - 1;
          mx &= mx - 1;
          const uint32_t *cx = C + (size_t)x * cs;
          for (uint32_t k3 = tri ? (x + 1) >> 5 : 0; k3 < Wp; ++k3) s6 += __popc(ca[k3] & cb[k3] & cx[k3]);
        }
      }
    }
  }
  return s;
}

// Rows with c <= 32: lane a keeps compacted row C_a in a register; the pairs
// (a, b) are visited with one shuffle of C_b per b (no shared memory).
// With K6, Cs (32 words of the warp's buffer) holds the rows for the 6-clique
// level: sum over b in C_a, x in C_a & C_b of |C_a & C_b & C_x|.
template <bool K6 = false>
__device__ __forceinline__ void nested_row_reg32(const uint32_t *R, uint32_t W, uint32_t rs, const uint32_t *ri,
                                                 uint32_t c, const uint32_t *S, const uint32_t *pref,
                                                 unsigned long long &a4, unsigned long long &a5, bool tri,
                                                 unsigned long long &a6, uint32_t *Cs) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t ca = 0;
  if (lane < c) {
    const uint32_t *rj = R + (size_t)S[lane] * rs;
    for (uint32_t w = tri ? (S[lane] + 1) >> 5 : 0; w < W; ++w) {
      const uint32_t riw = ri[w];
      const uint32_t x = rj[w] & riw;
      if (x) ca |= gather_bits(x, riw) << pref[w];  // c <= 32: every output bit is in word 0
    }
  }
  a4 += __popc(ca);
  if (K6) {
    Cs[lane] = ca;
    __syncwarp();
  }
  for (uint32_t b = 0; b < c; ++b) {
    const uint32_t cb = __shfl_sync(0xffffffffu, ca, b);
    if ((ca >> b) & 1u) {
      const uint32_t m = ca & cb;
      a5 += __popc(m);
      if (K6) {
        uint32_t mx = m;
        while (mx) {
          const uint32_t x = __ffs(mx) - 1;
          mx &= mx - 1;
          a6 += __popc(m & Cs[x]);
        }
      }
    }
  }
  if (K6) __syncwarp();
}

// Row i by a group of lanes without nesting (fallback for rows too wide to
// compact): the group takes every `ng`-th bit j of R_i.
template <bool K6 = false>
__device__ __forceinline__ void row_k45_groups(const uint32_t *R, uint32_t W, uint32_t rs, uint32_t i, uint32_t g,
                                               uint32_t ng, uint32_t gl, uint32_t G, unsigned long long &a4,
                                               unsigned long long &a5, unsigned long long &a6) {
  const uint32_t *ri = R + (size_t)i * rs;
  uint32_t seen = 0;
  for (uint32_t t = 0; t < W; ++t) {
    uint32_t bits = ri[t];
    while (bits) {
      const uint32_t j = t * 32 + __ffs(bits) - 1;
      bits &= bits - 1;
      if ((seen++ % ng) != g) continue;
      const uint32_t *rj = R + (size_t)j * rs;
      for (uint32_t w = gl; w < W; w += G) {
        const uint32_t mw = ri[w] & rj[w];
        a4 += __popc(mw);
      }
      for (uint32_t t2 = 0; t2 < W; ++t2) {
        uint32_t b2 = ri[t2] & rj[t2];
        while (b2) {
          const uint32_t l = t2 * 32 + __ffs(b2) - 1;
          b2 &= b2 - 1;
          const uint32_t *rl = R + (size_t)l * rs;
          for (uint32_t w = gl; w < W; w += G) a5 += __popc(ri[w] & rj[w] & rl[w]);
          if (K6) {
            for (uint32_t t3 = 0; t3 < W; ++t3) {
              uint32_t b3 = ri[t3] & rj[t3] & rl[t3];
              while (b3) {
                const uint32_t y = t3 * 32 + __ffs(b3) - 1;
                b3 &= b3 - 1;
                const uint32_t *ry = R + (size_t)y * rs;
                for (uint32_t w = gl; w < W; w += G) a6 += __popc(ri[w] & rj[w] & rl[w] & ry[w]);
              }
            }
          }
        }
      }
    }
  }
}

// 4- and 5-cliques of one root's local graph R (d rows, W <= 32 words) by the
// whole CTA with nesting. nest: nest_words(maxd, blockDim/32, big_cap, wcap)
// words. Rows with c <= wcap are nested by one warp each; larger rows by four
// groups of warps (one row per group at a time, named barriers, so groups do
// not wait for each other); rows too large for a group's share of the pool by
// the whole CTA at the end.
// With tri, R is strictly upper triangular (positions in the orientation's
// order), and so is every nested C: the word loops start at the pivot.
template <bool K6 = false>
__device__ inline void enumerate_nested_cta(const uint32_t *R, uint32_t d, uint32_t W, uint32_t rs, uint32_t *nest,
                                            uint32_t maxd, uint32_t big_cap, unsigned long long &a4,
                                            unsigned long long &a5, unsigned long long &a6, bool tri = false,
                                            uint32_t wcap = kNestWarpC) {
  const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  uint32_t *ctr = nest;  // [0] next row, [1] big rows, [2] next big row, [3] wide rows
  uint32_t *big_list = nest + 4;
  uint32_t *wide_list = big_list + maxd;
  uint32_t *pool = wide_list + maxd;
  const uint32_t wwords = nest_warp_words(wcap);
  const uint32_t pool_words = nw * wwords + maxd + 32 + big_cap;
  if (tid == 0) {
    ctr[0] = 0;
    ctr[1] = 0;
    ctr[2] = 0;
    ctr[3] = 0;
  }
  __syncthreads();
  // rows with c <= kNestWarpC: one warp each, pulled dynamically
  {
    uint32_t *wbuf = pool + (size_t)wid * wwords;
    uint32_t *S = wbuf, *pref = wbuf + wcap, *C = wbuf + wcap + 32;
    for (;;) {
      uint32_t i = 0;
      if (lane == 0) i = atomicAdd(&ctr[0], 1u);
      i = __shfl_sync(0xffffffffu, i, 0);
      if (i >= d) break;
      const uint32_t *ri = R + (size_t)i * rs;
      const uint32_t c = list_bits_warp(ri, W, S, pref, wcap);
      if (c < 2) continue;
      if (c > wcap) {
        if (lane == 0) big_list[atomicAdd(&ctr[1], 1u)] = i;
        continue;
      }
      if (c <= 32) {
        nested_row_reg32<K6>(R, W, rs, ri, c, S, pref, a4, a5, tri, a6, C);
        __syncwarp();
        continue;
      }
      const uint32_t Wp = (c + 31) / 32, cs = row_stride(Wp);
      for (uint32_t a = lane; a < c; a += 32) {
        const uint32_t bits =
            compact_row(R + (size_t)S[a] * rs, ri, pref, W, C + (size_t)a * cs, Wp, tri ? (S[a] + 1) >> 5 : 0);
        a4 += bits;
      }
      __syncwarp();
      // units in word-major order: a round of lanes takes neighbouring rows, word k alike
      for (uint32_t u = lane; u < c * Wp; u += 32) a5 += nested_pairs_unit<K6>(C, u % c, u / c, Wp, cs, tri, a6);
      __syncwarp();
    }
  }
  __syncthreads();
  const uint32_t nbig = ctr[1];
  // rows with larger c: groups of four warps, one row per group at a time
  if (nbig) {
    const uint32_t gwarps = nw >= 32 ? 8u : 4u;  // four groups for 16 or 32 warps
    const uint32_t ng = nw >= gwarps ? nw / gwarps : 1u;
    const uint32_t gthreads = (ng > 1) ? gwarps * 32 : nt;
    const uint32_t g = (ng > 1) ? wid / gwarps : 0u;
    if (g < ng) {  // warps beyond ng groups (nw not a multiple of 4) sit this phase out
      const uint32_t gt = tid - g * gthreads, gw = gt >> 5;
      const uint32_t share = pool_words / ng;
      uint32_t *S = pool + (size_t)g * share, *pref = S + maxd, *hdr = pref + 32, *C = hdr + 4;
      const uint32_t cap = share > maxd + 36 ? share - maxd - 36 : 0u;
      for (;;) {
        if (gt == 0) hdr[0] = atomicAdd(&ctr[2], 1u);
        group_bar(1 + g, gthreads);
        const uint32_t q = hdr[0];
        if (q >= nbig) break;
        const uint32_t i = big_list[q];
        const uint32_t *ri = R + (size_t)i * rs;
        if (gw == 0) {
          const uint32_t c = list_bits_warp(ri, W, S, pref, maxd);
          if (lane == 0) hdr[1] = c;
        }
        group_bar(1 + g, gthreads);
        const uint32_t c = hdr[1];
        const uint32_t Wp = (c + 31) / 32, cs = row_stride(Wp);
        if ((uint64_t)c * cs > cap) {
          if (gt == 0) wide_list[atomicAdd(&ctr[3], 1u)] = i;
          continue;
        }
        // one thread per compacted row: no write sharing
        if (gt == 0) hdr[2] = 0;
        for (uint32_t a = gt; a < c; a += gthreads)
          a4 += compact_row(R + (size_t)S[a] * rs, ri, pref, W, C + (size_t)a * cs, Wp, tri ? (S[a] + 1) >> 5 : 0);
        group_bar(1 + g, gthreads);
        // pair units in word-major order, 32 at a time per warp (with tri the
        // work per unit falls steeply with the row and the word)
        for (;;) {
          uint32_t u0 = 0;
          if (lane == 0) u0 = atomicAdd(&hdr[2], 32u);
          u0 = __shfl_sync(0xffffffffu, u0, 0);
          if (u0 >= c * Wp) break;
          const uint32_t u = u0 + lane;
          if (u < c * Wp) a5 += nested_pairs_unit<K6>(C, u % c, u / c, Wp, cs, tri, a6);
        }
        group_bar(1 + g, gthreads);
      }
    }
  }
  __syncthreads();
  // rows too large for a group: the whole CTA with the whole pool
  const uint32_t nwide = ctr[3];
  uint32_t *S = pool, *pref = pool + maxd, *C = pref + 32;
  const uint32_t cap = pool_words - maxd - 32;
  for (uint32_t r = 0; r < nwide; ++r) {
    const uint32_t i = wide_list[r];
    const uint32_t *ri = R + (size_t)i * rs;
    if (wid == 0) {
      const uint32_t c = list_bits_warp(ri, W, S, pref, maxd);
      if (lane == 0) {
        ctr[0] = c;
        ctr[2] = 0;
      }
    }
    __syncthreads();
    const uint32_t c = ctr[0];
    const uint32_t Wp = (c + 31) / 32, cs = row_stride(Wp);
    if ((uint64_t)c * cs <= cap) {
      for (uint32_t u = tid; u < c * cs; u += nt) C[u] = 0u;
      __syncthreads();
      // (row, word) units: every thread works on the wide row
      for (uint32_t u = tid; u < c * W; u += nt) {
        const uint32_t a = u / W, w = u % W;
        if (tri && w < ((S[a] + 1) >> 5)) continue;
        const uint32_t riw = ri[w];
        const uint32_t x = R[(size_t)S[a] * rs + w] & riw;
        if (!x) continue;
        a4 += __popc(x);
        const uint32_t out = gather_bits(x, riw);
        const uint32_t base = pref[w], wi = base >> 5, lo = base & 31;
        uint32_t *crow = C + (size_t)a * cs;
        atomicOr(&crow[wi], out << lo);
        if (lo && lo + __popc(riw) > 32) atomicOr(&crow[wi + 1], out >> (32 - lo));
      }
      __syncthreads();
      for (;;) {
        uint32_t u0 = 0;
        if (lane == 0) u0 = atomicAdd(&ctr[2], 32u);
        u0 = __shfl_sync(0xffffffffu, u0, 0);
        if (u0 >= c * Wp) break;
        const uint32_t u = u0 + lane;
        if (u < c * Wp) a5 += nested_pairs_unit<K6>(C, u % c, u / c, Wp, cs, tri, a6);
      }
    } else {
      row_k45_groups<K6>(R, W, rs, i, tid >> 5, nt >> 5, lane, 32, a4, a5, a6);
    }
    __syncthreads();
  }
}

// Words of shared memory one warp needs for a root of out-degree <= maxd:
// xb[maxd] (uint64) | L[maxd] | pre[maxd+1] | R[maxd*W] | tc[maxd] (scatter)
__host__ __device__ constexpr uint32_t warp_words(uint32_t maxd, bool scatter) {
  return ((2 * maxd + maxd + (maxd + 1) + maxd * row_stride((maxd + 31) / 32) + (scatter ? maxd : 0)) + 1) & ~1u;
}

// Same layout for one CTA-wide root with W words per row, plus perm[maxd]
// (positions in the orientation's order, see rank_local).
__host__ __device__ constexpr uint64_t cta_words(uint32_t maxd, uint32_t W) {
  return 2ull * maxd + maxd + (maxd + 1) + (uint64_t)maxd * row_stride(W) + maxd + maxd + 2;
}

// Ranks of the local vertices in the orientation's order (degree, then id):
// perm[i] = #{i' : (deg L[i'], L[i']) < (deg L[i], L[i])}. Since L is sorted by
// id, the key (deg << 32 | i) orders like (deg, id). Bitonic sort of the padded
// keys in `keys` (nextpow2(d) words x 2) by the whole CTA; every thread calls.
__device__ __forceinline__ void rank_local(const uint32_t *__restrict__ deg, const uint32_t *L, uint32_t d,
                                           uint64_t *keys, uint32_t *perm) {
  const uint32_t tid = threadIdx.x, nt = blockDim.x;
  uint32_t n2 = 2;
  while (n2 < d) n2 <<= 1;
  for (uint32_t i = tid; i < n2; i += nt) keys[i] = (i < d) ? (((uint64_t)__ldg(deg + L[i]) << 32) | i) : ~0ull;
  __syncthreads();
  for (uint32_t k = 2; k <= n2; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t t = tid; t < n2 / 2; t += nt) {
        const uint32_t lo = 2 * j * (t / j) + (t % j), hi = lo + j;
        const bool up = (lo & k) == 0;
        const uint64_t x = keys[lo], y = keys[hi];
        if ((x > y) == up) {
          keys[lo] = y;
          keys[hi] = x;
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t p = tid; p < d; p += nt) perm[(uint32_t)keys[p]] = p;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Cliques of any size k >= 7: the shrinking candidate set of the local-graph
// search (k-CL on the local graph, one level per clique vertex) with the set
// held as a bitmap over the root's local vertices, distributed over a warp
// (lane l keeps words l, l + 32, ... of it: NWL words per lane). Once a set
// has at most 32 members it is compacted into a register graph (lane b keeps
// row b of the induced 32-vertex DAG) and the remaining levels run as per-lane
// loops over single words.
// ---------------------------------------------------------------------------

// Per-warp scratch (words) of the generic search: Mw[32 NWL] | pref[32 NWL] | S[32] | Ds[32]
__host__ __device__ constexpr uint32_t gen_warp_words(uint32_t nwl) { return 64 * nwl + 64; }

// r-cliques (r >= 1) among the members m of the register graph (rows Ds in
// shared memory; lane x also holds its own row dl = Ds[x]). The graph is a
// DAG: row x holds x's successors, so each clique is met once, through its
// first vertex; successors are taken from all of m, since the DAG order need
// not follow the bit order. The whole warp walks the first r - 3 levels
// together (m is warp-uniform); then lane x takes the third-last vertex x, a
// loop the second-last and a popcount the last, so lanes diverge over one
// level only. Returns this lane's share (at most C(32, r) < 2^32 in all).
template <int r>
__device__ __forceinline__ uint32_t reg_cliques_warp(uint32_t m, uint32_t dl, const uint32_t *Ds) {
  const uint32_t lane = threadIdx.x & 31;
  if constexpr (r == 1) {
    return lane == 0 ? __popc(m) : 0u;
  } else if constexpr (r == 2) {
    return ((m >> lane) & 1u) ? __popc(m & dl) : 0u;
  } else if constexpr (r == 3) {
    uint32_t s = 0;
    if ((m >> lane) & 1u) {
      const uint32_t m1 = m & dl;
      uint32_t rest = m1;
      while (rest) {
        const uint32_t z = __ffs(rest) - 1;
        rest &= rest - 1;
        s += __popc(m1 & Ds[z]);
      }
    }
    return s;
  } else {
    uint32_t s = 0, rest = m;
    while (rest) {
      const uint32_t x = __ffs(rest) - 1;
      rest &= rest - 1;
      const uint32_t m2 = m & Ds[x];
      if (__popc(m2) >= (uint32_t)(r - 1)) s += reg_cliques_warp<r - 1>(m2, dl, Ds);
    }
    return s;
  }
}

// position of the j-th (from 0) set bit of v (j < popc(v)), by halving
__device__ __forceinline__ uint32_t select_bit(uint32_t v, uint32_t j) {
  uint32_t pos = 0, c = __popc(v & 0xffffu);
  if (j >= c) { j -= c; v >>= 16; pos += 16; }
  c = __popc(v & 0xffu);
  if (j >= c) { j -= c; v >>= 8; pos += 8; }
  c = __popc(v & 0xfu);
  if (j >= c) { j -= c; v >>= 4; pos += 4; }
  c = __popc(v & 0x3u);
  if (j >= c) { j -= c; v >>= 2; pos += 2; }
  if (j >= (v & 1u)) pos += 1;
  return pos;
}

// r-cliques (r >= 1) of the register graph among the members c, counted by
// one lane on its own (rows Ds in shared memory)
template <int r>
__device__ __forceinline__ uint32_t seq_cliques(uint32_t c, const uint32_t *Ds) {
  if constexpr (r == 1) {
    return __popc(c);
  } else {
    uint32_t s = 0, rest = c;
    while (rest) {
      const uint32_t z = __ffs(rest) - 1;
      rest &= rest - 1;
      const uint32_t c2 = c & Ds[z];
      if constexpr (r == 2) s += __popc(c2);
      else if (__popc(c2) >= (uint32_t)(r - 1)) s += seq_cliques<r - 1>(c2, Ds);
    }
    return s;
  }
}

// r-cliques (r >= 4) among the members m of the register graph, with the
// pairs (x, y) of a member and one of its successors spread over the lanes:
// an inclusive scan of the successor counts numbers the pairs, lane p takes
// pairs p, p + 32, ... (x by a binary search of the scan, y by bit selection)
// and counts the (r - 2)-cliques among the common successors of x and y on
// its own. All lanes work as long as there are 32 pairs, where walking the
// first levels warp-uniformly leaves every lane outside the current set idle.
// tmp: 64 words of the warp's scratch. Returns this lane's share.
template <int r>
__device__ __forceinline__ uint32_t reg_cliques_pairs(uint32_t m, const uint32_t *Ds, uint32_t *tmp) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t *succ = tmp, *upto = tmp + 32;
  const uint32_t mx = ((m >> lane) & 1u) ? (m & Ds[lane]) : 0u;
  uint32_t incl = __popc(mx);
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  succ[lane] = mx;
  upto[lane] = incl;
  __syncwarp();
  const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
  uint32_t s = 0;
  for (uint32_t p = lane; p < total; p += 32) {
    uint32_t lo = 0, hi = 31;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (upto[mid] > p) hi = mid;
      else lo = mid + 1;
    }
    const uint32_t sx = succ[lo];
    const uint32_t y = select_bit(sx, p - (upto[lo] - __popc(sx)));
    const uint32_t c = sx & Ds[y];
    if (__popc(c) >= (uint32_t)(r - 2)) s += seq_cliques<r - 2>(c, Ds);
  }
  __syncwarp();
  return s;
}

// Q-cliques (Q >= 1) among the members of the set m (NWL words per lane) of
// the local-graph DAG R (W words per row, stride rs). Called by a whole warp
// with warp-uniform arguments; returns this lane's share (the warp sum is the
// count). With tri, row j of R has no bit at or below j.
template <int Q, int NWL>
__device__ unsigned long long set_cliques(const uint32_t *R, uint32_t W, uint32_t rs, const uint32_t (&m)[NWL],
                                          uint32_t *scr, bool tri) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t cnt = 0;
#pragma unroll
  for (int j = 0; j < NWL; ++j) cnt += __popc(m[j]);
  if constexpr (Q == 1) {
    return cnt;
  } else {
    const uint32_t c = __reduce_add_sync(0xffffffffu, cnt);
    if (c < (uint32_t)Q) return 0;
    if (c <= 32) {
      // compact onto a register graph: S lists the members in order, pref[w]
      // counts the members in words before w
      uint32_t *Mw = scr, *pref = scr + 32 * NWL, *S = scr + 64 * NWL, *Ds = S + 32;
      uint32_t run = 0;
#pragma unroll
      for (int j = 0; j < NWL; ++j) {
        const uint32_t x0 = m[j], k0 = __popc(x0);
        uint32_t incl = k0;
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= (uint32_t)o) incl += y;
        }
        const uint32_t w = j * 32 + lane;
        uint32_t k = run + incl - k0, x = x0;
        Mw[w] = x0;
        pref[w] = k;
        while (x) {
          S[k++] = w * 32 + __ffs(x) - 1;
          x &= x - 1;
        }
        run += __shfl_sync(0xffffffffu, incl, 31);
      }
      __syncwarp();
      uint32_t db = 0;
      if (lane < c) {
        const uint32_t v = S[lane];
        const uint32_t *rv = R + (size_t)v * rs;
        for (uint32_t w = tri ? (v + 1) >> 5 : 0; w < W; ++w) {
          const uint32_t mw = Mw[w];
          const uint32_t x = rv[w] & mw;
          if (x) db |= gather_bits(x, mw) << pref[w];  // c <= 32: every output bit is in word 0
        }
      }
      Ds[lane] = db;
      __syncwarp();
      const uint32_t all = c == 32 ? ~0u : (1u << c) - 1u;
      unsigned long long s;
      if constexpr (Q >= 4) s = reg_cliques_pairs<Q>(all, Ds, scr);  // Mw and pref are free again
      else s = reg_cliques_warp<Q>(all, db, Ds);
      __syncwarp();
      return s;
    } else if constexpr (Q <= 3) {
      // more than 32 members, two or three levels left: lane l takes the
      // member at bit l of each word (a uniform loop over the words), then
      // loops over the members after it; the set stays in shared memory
      uint32_t *Mw = scr;
#pragma unroll
      for (int j = 0; j < NWL; ++j) Mw[j * 32 + lane] = m[j];
      __syncwarp();
      unsigned long long s = 0;
      for (uint32_t w = 0; w < W; ++w) {
        const uint32_t mw = Mw[w];
        if (!((mw >> lane) & 1u)) continue;
        const uint32_t a = w * 32 + lane;
        const uint32_t *ra = R + (size_t)a * rs;
        const uint32_t w0 = tri ? (a + 1) >> 5 : 0u;
        if constexpr (Q == 2) {
          uint32_t t = 0;
          for (uint32_t w2 = w0; w2 < W; ++w2) t += __popc(Mw[w2] & ra[w2]);
          s += t;
        } else {
          for (uint32_t w1 = w0; w1 < W; ++w1) {
            uint32_t x = Mw[w1] & ra[w1];
            while (x) {
              const uint32_t b = w1 * 32 + __ffs(x) - 1;
              x &= x - 1;
              const uint32_t *rb = R + (size_t)b * rs;
              uint32_t t = 0;
              for (uint32_t w2 = tri ? (b + 1) >> 5 : 0u; w2 < W; ++w2) t += __popc(Mw[w2] & ra[w2] & rb[w2]);
              s += t;
            }
          }
        }
      }
      __syncwarp();
      return s;
    } else {
      // first member a, then (Q-1)-cliques among a's successors in the set
      unsigned long long s = 0;
#pragma unroll 1
      for (int j = 0; j < NWL && (uint32_t)j * 32 < W; ++j) {
        const uint32_t tw = min(32u, W - (uint32_t)j * 32);
#pragma unroll 1
        for (uint32_t t = 0; t < tw; ++t) {
          uint32_t word = __shfl_sync(0xffffffffu, m[j], t);
          const uint32_t w = j * 32 + t;
          while (word) {
            const uint32_t a = w * 32 + __ffs(word) - 1;
            word &= word - 1;
            const uint32_t *ra = R + (size_t)a * rs;
            uint32_t m2[NWL];
#pragma unroll
            for (int jj = 0; jj < NWL; ++jj) {
              const uint32_t ww = jj * 32 + lane;
              m2[jj] = (ww < W) ? (m[jj] & ra[ww]) : 0u;
            }
            s += set_cliques<Q - 1, NWL>(R, W, rs, m2, scr, tri);
          }
        }
      }
      return s;
    }
  }
}

// k-cliques (KMAX = k >= 7) through the root of the CTA's local graph. The
// work is cut into (row i, word w) units, claimed dynamically by warps in
// word-major order, so that the rows of a heavy local graph spread over the
// CTA: a unit takes each member a in word w of R_i and counts the
// (k-3)-cliques among R_i & R_a. A root may be split over nslices CTAs, each
// building the local graph: with a global counter gctr (zero before the
// launch) their warps claim the root's units from it, so the CTAs of a root
// finish together; without it (ctr: a shared counter) each takes the units
// congruent to its slice. Every thread of the CTA calls it.
template <int KMAX, int NWL>
__device__ __forceinline__ void rows_generic_cta(const uint32_t *R, uint32_t d, uint32_t W, uint32_t rs,
                                                 uint32_t *ctr, uint32_t *scr, bool tri, unsigned long long &ak,
                                                 uint32_t slice, uint32_t nslices, unsigned int *gctr = nullptr) {
  const uint32_t lane = threadIdx.x & 31;
  if (threadIdx.x == 0) *ctr = 0;
  __syncthreads();
  const uint32_t units = d * W;
  for (;;) {
    uint32_t q = 0;
    if (lane == 0) q = atomicAdd(gctr ? gctr : ctr, 1u);
    q = __shfl_sync(0xffffffffu, q, 0);
    const uint32_t u = gctr ? q : q * nslices + slice;
    if (u >= units) break;
    const uint32_t i = u % d, w = u / d;
    const uint32_t *ri = R + (size_t)i * rs;
    uint32_t word = ri[w];
    if (!word) continue;
    uint32_t mi[NWL];
#pragma unroll
    for (int j = 0; j < NWL; ++j) {
      const uint32_t ww = j * 32 + lane;
      mi[j] = (ww < W) ? ri[ww] : 0u;
    }
    while (word) {
      const uint32_t a = w * 32 + __ffs(word) - 1;
      word &= word - 1;
      const uint32_t *ra = R + (size_t)a * rs;
      uint32_t m2[NWL];
#pragma unroll
      for (int j = 0; j < NWL; ++j) {
        const uint32_t ww = j * 32 + lane;
        m2[j] = (ww < W) ? (mi[j] & ra[ww]) : 0u;
      }
      ak += set_cliques<KMAX - 3, NWL>(R, W, rs, m2, scr, tri);
    }
  }
}

// One root u (2 <= d+(u) <= MAXD) processed by the calling warp. `base` is
// the warp's shared-memory region of warp_words(MAXD, SCATTER) words.
template <int MAXD, int G, int KMAX, bool SCATTER>
__device__ __forceinline__ void lg_root_warp(const uint64_t *__restrict__ drow, const uint32_t *__restrict__ dcol,
                                             uint32_t *t_edge, uint32_t u, uint32_t *base, unsigned long long &a3,
                                             unsigned long long &a4, unsigned long long &a5, unsigned long long &a6,
                                             uint32_t *gen = nullptr) {
  const uint32_t lane = threadIdx.x & 31;
  uint64_t *xb = reinterpret_cast<uint64_t *>(base);
  uint32_t *L = base + 2 * MAXD;
  uint32_t *pre = L + MAXD;
  uint32_t *R = pre + MAXD + 1;
  uint32_t *tc = R + MAXD * row_stride((MAXD + 31) / 32);
  const uint64_t ub = drow[u];
  const uint32_t d = (uint32_t)(drow[u + 1] - ub);
  const uint32_t w_used = (d + 31) / 32, rs = row_stride(w_used);
  for (uint32_t i = lane; i < d; i += 32) {
    const uint32_t x = __ldg(dcol + ub + i);
    L[i] = x;
    const uint64_t xs = __ldg(drow + x), xe = __ldg(drow + x + 1);
    xb[i] = xs;
    pre[i + 1] = (uint32_t)(xe - xs);
    if (SCATTER) tc[i] = 0;
  }
  if (KMAX >= 4)
    for (uint32_t i = lane; i < d * rs; i += 32) R[i] = 0;
  if (lane == 0) pre[0] = 0;
  __syncwarp();
  uint32_t carry = 0;
  for (uint32_t c0 = 0; c0 < d; c0 += 32) {
    const uint32_t i = c0 + lane;
    uint32_t v = (i < d) ? pre[i + 1] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= (uint32_t)o) v += y;
    }
    if (i < d) pre[i + 1] = v + carry;
    carry += __shfl_sync(0xffffffffu, v, 31);
  }
  __syncwarp();
  a3 += build_rows_runs<SCATTER, (KMAX >= 4)>(dcol, t_edge, L, pre, xb, R, tc, d, rs, lane, 32, nullptr, nullptr, 0);
  __syncwarp();
  if (SCATTER) {
    for (uint32_t i = lane; i < d; i += 32)
      if (tc[i]) atomicAdd(&t_edge[ub + i], tc[i]);
  }
  if constexpr (KMAX >= 7) {
    // (k-1)-cliques among all of L; a6 carries the k-clique count
    uint32_t m[1];
    m[0] = (lane < w_used) ? ((lane + 1) * 32 <= d ? ~0u : (1u << (d & 31)) - 1u) : 0u;
    a6 += set_cliques<KMAX - 1, 1>(R, w_used, rs, m, gen, false);
  } else if (KMAX >= 4) {
    enumerate_rows<G, KMAX>(R, d, w_used, rs, lane / G, 32 / G, lane % G, a4, a5, a6);
  }
  __syncwarp();
}

// One root u (2 <= d+(u) <= maxd) processed by the whole CTA. `base` holds
// cta_words(maxd, W) words (shared or global memory); W >= ceil(maxd / 32).
// Every thread of the CTA must call it.
template <int G, int KMAX, bool SCATTER, int NWL = 1>
__device__ __forceinline__ void lg_root_cta(const uint64_t *__restrict__ drow, const uint32_t *__restrict__ dcol,
                                            uint32_t *t_edge, uint32_t u, uint32_t maxd, uint32_t W, uint32_t *base,
                                            unsigned long long &a3, unsigned long long &a4, unsigned long long &a5,
                                            unsigned long long &a6, uint32_t *nest = nullptr, uint32_t big_cap = 0,
                                            const uint32_t *__restrict__ deg = nullptr, uint32_t wcap = kNestWarpC,
                                            uint32_t *gen = nullptr, uint32_t slice = 0, uint32_t nslices = 1,
                                            unsigned int *gctr = nullptr) {
  const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
  uint64_t *xb = reinterpret_cast<uint64_t *>(base);
  uint32_t *L = base + 2 * (size_t)maxd;
  uint32_t *pre = L + maxd;
  uint32_t *R = pre + maxd + 1;
  uint32_t *tc = R + (size_t)maxd * row_stride(W);
  uint32_t *perm = tc + maxd;
  const uint64_t ub = drow[u];
  const uint32_t d = (uint32_t)(drow[u + 1] - ub);
  const uint32_t w_used = (d + 31) / 32, rs = row_stride(w_used);
  // the nested 5-clique search runs on positions in the orientation's order;
  // the sort keys borrow R's space (8-byte aligned) before R is cleared
  uint32_t n2 = 2;
  while (n2 < d) n2 <<= 1;
  uint64_t *keys = reinterpret_cast<uint64_t *>((reinterpret_cast<uintptr_t>(R) + 7) & ~(uintptr_t)7);
  const bool tri = KMAX >= 5 && nest != nullptr && deg != nullptr && w_used <= 32 &&
                   (uint64_t)maxd * row_stride(W) >= 2ull * n2 + 1;
  for (uint32_t i = tid; i < d; i += nt) {
    const uint32_t x = __ldg(dcol + ub + i);
    L[i] = x;
    const uint64_t xs = __ldg(drow + x), xe = __ldg(drow + x + 1);
    xb[i] = xs;
    pre[i + 1] = (uint32_t)(xe - xs);
    if (SCATTER) tc[i] = 0;
  }
  if (tri) {
    __syncthreads();
    rank_local(deg, L, d, keys, perm);
  }
  if (KMAX >= 4)
    for (size_t i = tid; i < (size_t)d * rs; i += nt) R[i] = 0;
  if (tid == 0) pre[0] = 0;
  // with the nested-search region present, its pool holds L's position table
  // until the enumeration starts (2^hbits >= 4d slots, keys and values: most
  // lookups miss, and a table a quarter full ends a miss in about 1.4 probes)
  uint32_t hbits = 1;
  while ((1u << hbits) < 4 * d) ++hbits;
  uint32_t *hk = nest ? nest + 4 + 2 * (size_t)maxd : nullptr;
  if (hk) build_pos_table(L, d, hk, hbits, tid, nt);
  __syncthreads();
  if (tid < 32) {
    uint32_t carry = 0;
    for (uint32_t c0 = 0; c0 < d; c0 += 32) {
      const uint32_t i = c0 + lane;
      uint32_t v = (i < d) ? pre[i + 1] : 0u;
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= (uint32_t)o) v += y;
      }
      if (i < d) pre[i + 1] = v + carry;
      carry += __shfl_sync(0xffffffffu, v, 31);
    }
  }
  __syncthreads();
  if (hk)
    a3 += build_rows_runs<SCATTER, (KMAX >= 4)>(dcol, t_edge, L, pre, xb, R, tc, d, rs, tid, nt, tri ? perm : nullptr,
                                                hk, hbits);
  else
    a3 += build_rows<SCATTER, (KMAX >= 4)>(dcol, t_edge, L, pre, xb, R, tc, d, rs, tid, nt, tri ? perm : nullptr);
  __syncthreads();
  if (SCATTER) {
    for (uint32_t i = tid; i < d; i += nt)
      if (tc[i]) atomicAdd(&t_edge[ub + i], tc[i]);
  }
  if constexpr (KMAX >= 7) {
    // gen: a counter word, then one scratch region per warp (the nested pool
    // is free again once the rows are built); a6 carries the k-clique count
    uint32_t *g = gen ? gen : nest + 4 + 2 * (size_t)maxd;
    rows_generic_cta<KMAX, NWL>(R, d, w_used, rs, g, g + 4 + (size_t)(tid >> 5) * gen_warp_words(NWL), tri, a6,
                                slice, nslices, gctr);
  } else if (KMAX >= 5 && nest != nullptr && w_used <= 32) {
    enumerate_nested_cta<(KMAX >= 6)>(R, d, w_used, rs, nest, maxd, big_cap, a4, a5, a6, tri, wcap);
  } else if (KMAX >= 4) {
    if (w_used > 32)
      enumerate_rows_wide<KMAX>(R, d, w_used, rs, tid / 32, nt / 32, lane, a4, a5, a6);
    else
      enumerate_rows<G, KMAX>(R, d, w_used, rs, tid / G, nt / G, tid % G, a4, a5, a6);
  }
  __syncthreads();
}

}  // namespace gpm_dev
