// Work items of the batched and served forms: per-root tasks of many
// queries over many graphs, processed by one CTA each in a persistent kernel.
// See batch.cu for the method.
#pragma once

#include <algorithm>
#include <string>
#include <vector>

#include "gpm_internal.h"
#include "lg_device.cuh"
#include "motif_device.cuh"

namespace gpm_item {

enum ItemType : uint32_t {
  IT_LG_WARP = 0, IT_LG_CTA = 1, IT_C4_SMALL = 2, IT_C4_BIG = 3, IT_EDGE = 4, IT_C4_BUCKET = 5,
  IT_C4_HUBPART = 6, IT_C4_HUBSUM = 7
};

// a, b, c, d: hub items only (served form). A hub 4-cycle root is counted by
// several PART items, each tallying the wedges of a range [lo, hi) of the
// root's work units into a shared slot of the hub pool with fire-and-forget
// increments, then by SUM items, each summing C(c,2) over words [lo, hi) of
// the slot while clearing them. a = hub root index, b = slot, c = the value
// the slot's SUM counter (PART) or PART counter (SUM) must reach first, d =
// the number of PART (or SUM) items of this root. Every wait points at items
// earlier in the same queue.
struct Item {
  uint32_t type, q, lo, hi;
  uint32_t a, b, c, d;
};

struct QDesc {
  uint64_t tag;              // caller's request tag (served form)
  const uint64_t *rowptr;
  const uint32_t *col;
  const uint32_t *deg;
  const uint64_t *drow;
  const uint32_t *dcol;
  uint32_t *t_edge;
  const uint32_t *tasks;     // LG root tasks of the graph (class order)
  const uint32_t *c4_tasks;  // 4-cycle roots
  const uint32_t *edeg;      // degree of col[e] per CSR entry (4-cycle wedge walks)
  const uint2 *hub_units;    // {x, chunk} work units of the hub-class 4-cycle roots
  uint32_t hub_base;         // hub root j is c4_tasks[hub_base + j]
  unsigned long long *acc;   // ACC_WORDS accumulators
  unsigned long long *out;   // 6 results
  unsigned int *left;        // [0] scatter items left, [1] items left
  uint32_t n, kind;
  uint64_t m;
  uint32_t nformula;
  uint32_t formula[6];
  uint32_t scatter_items, all_items;
};

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kWarpMaxD = 128;
constexpr uint64_t kWaitLimit = 1ull << 26;

// CTA roots with out-degree above this build their bitmap in a per-CTA
// global-memory slot, so the persistent kernel's shared memory stays small
constexpr uint32_t kItemCtaSmemMaxD = 384;

struct ItemEnv {
  uint32_t *tally_pool;
  uint64_t tally_slot_words;
  unsigned int *status;
  uint32_t cta_maxd, cta_W;  // shared-memory CTA roots (out-degree <= cta_maxd)
  uint32_t *lg_pool;         // global-memory bitmap slots, one per CTA
  uint64_t lg_slot_words;
  uint32_t lg_maxd, lg_W;    // larger roots
  uint32_t *c4_buf;          // bucketed 4-cycle buffers, one slot per CTA
  uint64_t c4_buf_words;
  uint32_t *hub_pool;        // hub tallies: slots of hub_slot_words words, zero between uses
  uint64_t hub_slot_words;
  unsigned int *hub_done;    // per slot: [2s] PART items done, [2s+1] SUM items done
};

constexpr uint32_t kHubItemUnits = 128;         // work units per PART item
constexpr uint32_t kHubItemWords = 1u << 18;    // tally words per SUM item
constexpr uint32_t kHubUnitChunk = gpm_dev::kC4HubChunk;  // adjacency entries per work unit

// Bounded wait of thread 0 until counter reaches target (modulo 2^32).
__device__ __forceinline__ void wait_counter(const unsigned int *counter, uint32_t target, unsigned int *status) {
  uint64_t n = 0;
  while ((int)(*(volatile const unsigned int *)counter - target) < 0) {
    __nanosleep(200);
    if (++n > kWaitLimit) {
      atomicOr(status, ST_TIMEOUT);
      break;
    }
  }
  __threadfence();
}

// shared memory carve-up: the union of the item types' needs
__host__ __device__ constexpr size_t warp_region_words() { return gpm_dev::warp_words(kWarpMaxD, true); }

template <int KMAX, bool SCATTER>
__device__ void lg_warp_item(const QDesc &q, const Item &it, uint32_t *smem, unsigned long long &a3,
                             unsigned long long &a4, unsigned long long &a5) {
  unsigned long long a6_unused = 0;  // items count at most 5-cliques
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t *base = smem + (size_t)wid * warp_region_words();
  for (uint32_t t = it.lo + wid; t < it.hi; t += kWarps) {
    const uint32_t u = q.tasks[t];
    const uint32_t d = (uint32_t)(q.drow[u + 1] - q.drow[u]);
    if (d < 2) continue;
    if (d <= 32)
      gpm_dev::lg_root_warp<32, 1, KMAX, SCATTER>(q.drow, q.dcol, q.t_edge, u, base, a3, a4, a5, a6_unused);
    else
      gpm_dev::lg_root_warp<kWarpMaxD, 4, KMAX, SCATTER>(q.drow, q.dcol, q.t_edge, u, base, a3, a4, a5, a6_unused);
  }
  (void)lane;
}

template <int KMAX, bool SCATTER>
__device__ void lg_cta_item(const ItemEnv &a, const QDesc &q, const Item &it, uint32_t *smem,
                            unsigned long long &a3, unsigned long long &a4, unsigned long long &a5) {
  unsigned long long a6_unused = 0;  // items count at most 5-cliques
  const uint32_t u = q.tasks[it.lo];
  const uint32_t d = (uint32_t)(q.drow[u + 1] - q.drow[u]);
  if (d > a.cta_maxd) {
    uint32_t *slot = a.lg_pool + (size_t)blockIdx.x * a.lg_slot_words;
    gpm_dev::lg_root_cta<32, KMAX, SCATTER>(q.drow, q.dcol, q.t_edge, u, a.lg_maxd, a.lg_W, slot, a3, a4, a5, a6_unused);
  } else if (a.cta_W <= 8) {
    gpm_dev::lg_root_cta<8, KMAX, SCATTER>(q.drow, q.dcol, q.t_edge, u, a.cta_maxd, a.cta_W, smem, a3, a4, a5, a6_unused);
  } else if (a.cta_W <= 16) {
    gpm_dev::lg_root_cta<16, KMAX, SCATTER>(q.drow, q.dcol, q.t_edge, u, a.cta_maxd, a.cta_W, smem, a3, a4, a5, a6_unused);
  } else {
    gpm_dev::lg_root_cta<32, KMAX, SCATTER>(q.drow, q.dcol, q.t_edge, u, a.cta_maxd, a.cta_W, smem, a3, a4, a5, a6_unused);
  }
}

__device__ __forceinline__ void block_add(unsigned long long *dst, unsigned long long v) {
  v = gpm_dev::warp_sum(v);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}


// Process one item with the whole CTA and fold its partial sums into the
// query's accumulators. q must be readable by every thread (shared memory).
// s_pre (kThreads + 33 words) and s_rp (kThreads entries): scratch of the
// bucketed 4-cycle walk.
__device__ __forceinline__ void run_item(const ItemEnv &a, const QDesc &q, const Item &it, uint32_t *smem,
                                         uint32_t *s_x, uint32_t *s_cnt, uint32_t *s_nt, uint32_t *s_pre,
                                         uint64_t *s_rp) {
  const uint32_t tid = threadIdx.x;
  unsigned long long a3 = 0, a4 = 0, a5 = 0, c4 = 0;
  gpm_dev::EdgeTerms et;
  bool overflow = false;
  const uint32_t kind = q.kind;
  switch (it.type) {
    case IT_LG_WARP:
      if (kind == GPM_QUERY_MOTIF4) lg_warp_item<4, true>(q, it, smem, a3, a4, a5);
      else if (kind == GPM_QUERY_CLIQUE5) lg_warp_item<5, false>(q, it, smem, a3, a4, a5);
      else if (kind == GPM_QUERY_CLIQUE4) lg_warp_item<4, false>(q, it, smem, a3, a4, a5);
      else lg_warp_item<3, false>(q, it, smem, a3, a4, a5);
      break;
    case IT_LG_CTA:
      if (kind == GPM_QUERY_MOTIF4) lg_cta_item<4, true>(a, q, it, smem, a3, a4, a5);
      else if (kind == GPM_QUERY_CLIQUE5) lg_cta_item<5, false>(a, q, it, smem, a3, a4, a5);
      else if (kind == GPM_QUERY_CLIQUE4) lg_cta_item<4, false>(a, q, it, smem, a3, a4, a5);
      else lg_cta_item<3, false>(a, q, it, smem, a3, a4, a5);
      break;
    case IT_C4_SMALL: {
      const uint32_t wid = tid >> 5;
      uint32_t *keys = smem + (size_t)wid * 2 * gpm_dev::kC4HashSlots;
      uint32_t *cnt = keys + gpm_dev::kC4HashSlots;
      for (uint32_t t = it.lo + wid; t < it.hi; t += kWarps)
        c4 += gpm_dev::c4_root_warp(q.rowptr, q.col, q.deg, q.edeg, q.c4_tasks[t], keys, cnt, overflow);
      break;
    }
    case IT_C4_BUCKET: {
      uint32_t *lin = a.c4_buf + (size_t)blockIdx.x * a.c4_buf_words;
      c4 += gpm_dev::c4_root_bucketed(q.rowptr, q.col, q.deg, q.edeg, q.c4_tasks[it.lo], lin, lin + a.c4_buf_words / 2,
                                      smem, s_x, s_cnt, overflow, s_pre, s_rp);
      break;
    }
    case IT_C4_BIG: {
      uint32_t *tally = a.tally_pool + (size_t)blockIdx.x * a.tally_slot_words;
      // the slot holds the tally in its first half and the touched list in its
      // second half for every query size: a smaller query's touched entries
      // must never land in a larger query's tally range
      c4 += gpm_dev::c4_root_cta(q.rowptr, q.col, q.deg, q.edeg, q.c4_tasks[it.lo], tally, tally + a.tally_slot_words / 2,
                                 s_x, s_cnt, s_nt);
      break;
    }
    case IT_C4_HUBPART: {
      if (tid == 0) wait_counter(&a.hub_done[2 * it.b + 1], it.c, a.status);
      __syncthreads();
      const uint32_t v0 = q.c4_tasks[q.hub_base + it.a], d0 = q.deg[v0];
      uint32_t *tally = a.hub_pool + (size_t)it.b * a.hub_slot_words;
      const uint32_t lane = tid & 31, wid = tid >> 5;
      for (uint32_t u = it.lo + wid; u < it.hi; u += kWarps) {
        const uint2 unit = q.hub_units[u];
        const uint64_t e0 = q.rowptr[unit.x] + (uint64_t)unit.y * kHubUnitChunk;
        const uint64_t e1 = min(q.rowptr[unit.x + 1], e0 + kHubUnitChunk);
        for (uint64_t base = e0; base < e1; base += 128) {
          uint32_t w[4], dw[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint64_t e = base + 32 * k + lane;
            w[k] = (e < e1) ? q.col[e] : 0u;
            dw[k] = (e < e1) ? q.edeg[e] : 0xffffffffu;
          }
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (gpm_dev::precedes(dw[k], w[k], d0, v0)) atomicAdd(&tally[w[k]], 1u);
        }
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) atomicAdd(&a.hub_done[2 * it.b], 1u);
      break;
    }
    case IT_C4_HUBSUM: {
      if (tid == 0) wait_counter(&a.hub_done[2 * it.b], it.c, a.status);
      __syncthreads();
      uint4 *T4 = reinterpret_cast<uint4 *>(a.hub_pool + (size_t)it.b * a.hub_slot_words);
      for (uint32_t i = it.lo / 4 + tid; i < it.hi / 4; i += kThreads) {
        const uint4 v = __ldcg(T4 + i);
        if (v.x | v.y | v.z | v.w) {
          c4 += (unsigned long long)v.x * (v.x - (v.x > 0)) / 2 + (unsigned long long)v.y * (v.y - (v.y > 0)) / 2 +
                (unsigned long long)v.z * (v.z - (v.z > 0)) / 2 + (unsigned long long)v.w * (v.w - (v.w > 0)) / 2;
          __stcg(T4 + i, make_uint4(0u, 0u, 0u, 0u));
        }
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) atomicAdd(&a.hub_done[2 * it.b + 1], 1u);
      break;
    }
    case IT_EDGE: {
      const uint32_t wid = tid >> 5;
      if (kind == GPM_QUERY_MOTIF4) {
        // wait until every triangle-scatter item of this query has finished
        if (tid == 0) {
          uint64_t it_wait = 0;
          while (*(volatile unsigned int *)&q.left[0] != 0u) {
            __nanosleep(200);
            if (++it_wait > kWaitLimit) {
              atomicOr(a.status, ST_TIMEOUT);
              break;
            }
          }
          __threadfence();
        }
        __syncthreads();
        for (uint64_t u = it.lo + wid; u < it.hi; u += kWarps)
          gpm_dev::edge_terms_vertex<true, true>(q.drow, q.dcol, q.deg, q.t_edge, u, true, et);
      } else {
        for (uint64_t u = it.lo + wid; u < it.hi; u += kWarps)
          gpm_dev::edge_terms_vertex<false, false>(q.drow, q.dcol, q.deg, nullptr, u, true, et);
      }
      break;
    }
    default: break;
  }
  block_add(&q.acc[ACC_T], a3);
  block_add(&q.acc[ACC_K4], a4);
  block_add(&q.acc[ACC_K5], a5);
  block_add(&q.acc[ACC_C4], c4);
  block_add(&q.acc[ACC_D], et.D);
  block_add(&q.acc[ACC_P], et.P);
  block_add(&q.acc[ACC_S], et.S);
  block_add(&q.acc[ACC_W], et.W);
  block_add(&q.acc[ACC_TT2], et.TT);
  block_add(&q.acc[ACC_T3], et.T3);
  // Every thread's atomics (partial sums, per-arc triangle counts) must be
  // performed device-wide before thread 0 counts this item as done: another
  // CTA may read them as soon as the counter drops.
  __threadfence();
  if (__syncthreads_or(overflow) && tid == 0) atomicOr(a.status, ST_CAPACITY);
}

// Called by thread 0 after run_item: counts the item as done; returns true
// when it was the query's last item.
__device__ __forceinline__ bool item_done(const QDesc &q, const Item &it) {
  __threadfence();
  if (q.kind == GPM_QUERY_MOTIF4 && (it.type == IT_LG_WARP || it.type == IT_LG_CTA)) atomicSub(&q.left[0], 1u);
  const unsigned int before = atomicSub(&q.left[1], 1u);
  if (before != 1u) return false;
  __threadfence();
  return true;
}

// The query's counts from its accumulators (thread 0, after its last item).
__device__ __forceinline__ unsigned int finalize_query(const QDesc &q, unsigned long long *out6) {
  unsigned long long acc[ACC_WORDS];
  for (int i = 0; i < ACC_WORDS; ++i) acc[i] = atomicAdd(&q.acc[i], 0ull);
  bool bad = false;
  for (uint32_t i = 0; i < 6; ++i)
    out6[i] = (i < q.nformula) ? gpm_dev::finalize_formula(q.formula[i], acc, q.n, q.m, bad) : 0ull;
  return bad ? ST_CAPACITY : 0u;
}

// Host side: cut one query (graph g, kind) into items for query slot qi.
// Heavy items (one CTA root each) go to `heavy`, ranges of warp roots to
// `light`, vertex ranges of local-count terms to `edge`. Returns the number
// of items and of triangle-scatter items through *all and *scatter.
// With hub_phase, the hub-class 4-cycle roots get no items: they are counted
// by separate whole-GPU launches ahead of the persistent kernel.
// With hub_items (served form), hub-class roots whose tally is dense (n <= 4
// x their wedge bound) become PART and SUM items (slot and wait targets are
// filled in at admission by assign_hub_slots); the others keep one CTA item.
inline void append_query_items(const gpm_graph *g, uint32_t kind, uint32_t qi, uint32_t roots_per_item,
                               uint32_t verts_per_item, std::vector<Item> &heavy, std::vector<Item> &light,
                               std::vector<Item> &edge, uint32_t *scatter, uint32_t *all, bool hub_phase = false,
                               bool hub_items = false, uint64_t hub_slot_words = 0) {
  uint32_t sc = 0, al = 0;
  const uint32_t warp_end = g->cls_begin[CLS_WARP + 1];
  for (uint32_t t = 0; t < warp_end; t += roots_per_item) {
    light.push_back({IT_LG_WARP, qi, t, std::min(warp_end, t + roots_per_item)});
    ++al;
    ++sc;
  }
  for (uint32_t t = g->cls_begin[CLS_CTA]; t < g->cls_begin[CLS_XL + 1]; ++t) {
    heavy.push_back({IT_LG_CTA, qi, t, t + 1});
    ++al;
    ++sc;
  }
  if (kind == GPM_QUERY_MOTIF4) {
    for (uint32_t t = g->c4_begin[0]; t < g->c4_begin[1]; t += roots_per_item) {
      light.push_back({IT_C4_SMALL, qi, t, std::min(g->c4_begin[1], t + roots_per_item)});
      ++al;
    }
    for (uint32_t t = g->c4_begin[1]; t < g->c4_begin[2]; ++t) {
      heavy.push_back({IT_C4_BUCKET, qi, t, t + 1});
      ++al;
    }
    for (uint32_t t = g->c4_begin[2]; t < (hub_phase ? g->c4_begin[2] : g->c4_begin[3]); ++t) {
      const uint32_t j = t - g->c4_begin[2];
      if (hub_items && j < g->c4_hub_bnd.size() && (uint64_t)g->n <= 4ull * g->c4_hub_bnd[j]) {
        const uint64_t u0 = g->c4_hub_uoff[j], u1 = g->c4_hub_uoff[j + 1];
        const uint32_t P = (uint32_t)((u1 - u0 + kHubItemUnits - 1) / kHubItemUnits);
        const uint64_t words = ((uint64_t)std::max<uint32_t>(g->n, 1) + 3) & ~3ull;
        const uint32_t Q = (uint32_t)((words + kHubItemWords - 1) / kHubItemWords);
        for (uint64_t u = u0; u < u1; u += kHubItemUnits)
          heavy.push_back({IT_C4_HUBPART, qi, (uint32_t)u, (uint32_t)std::min<uint64_t>(u1, u + kHubItemUnits), j, 0, 0, P});
        for (uint64_t w = 0; w < words; w += kHubItemWords)
          heavy.push_back({IT_C4_HUBSUM, qi, (uint32_t)w, (uint32_t)std::min<uint64_t>(words, w + kHubItemWords), j, 0, 0, Q});
        al += P + Q;
        (void)hub_slot_words;
        continue;
      }
      heavy.push_back({IT_C4_BIG, qi, t, t + 1});
      ++al;
    }
  }
  if (kind == GPM_QUERY_MOTIF3 || kind == GPM_QUERY_MOTIF4) {
    for (uint32_t v = 0; v < g->n; v += verts_per_item) {
      edge.push_back({IT_EDGE, qi, v, std::min(g->n, v + verts_per_item)});
      ++al;
    }
  }
  *scatter = (kind == GPM_QUERY_MOTIF4) ? sc : 0u;
  *all = al;
}

// Slot and wait targets of hub items, in queue order. next_slot, parts and
// sums (per slot, counting every PART / SUM item ever issued for it) carry
// over between calls; each root takes the next slot round robin.
inline void assign_hub_slots(Item *items, size_t n, uint32_t nslots, uint32_t *next_slot, uint32_t *parts,
                             uint32_t *sums) {
  for (size_t i = 0; i < n;) {
    if (items[i].type != IT_C4_HUBPART) {
      ++i;
      continue;
    }
    const uint32_t P = items[i].d;
    const uint32_t Q = items[i + P].d;
    const uint32_t s = (*next_slot)++ % nslots;
    const uint32_t wait_sum = sums[s];
    parts[s] += P;
    for (uint32_t k = 0; k < P; ++k) {
      items[i + k].b = s;
      items[i + k].c = wait_sum;
    }
    for (uint32_t k = 0; k < Q; ++k) {
      items[i + P + k].b = s;
      items[i + P + k].c = parts[s];
    }
    sums[s] += Q;
    i += P + Q;
  }
}

inline int formulas_for(uint32_t kind, uint32_t *f, uint32_t *nf) {
  switch (kind) {
    case GPM_QUERY_MOTIF3: f[0] = F_WEDGE_I; f[1] = F_TRI; *nf = 2; return GPM_OK;
    case GPM_QUERY_MOTIF4:
      f[0] = F_STAR_I; f[1] = F_PATH_I; f[2] = F_TT_I; f[3] = F_C4_I; f[4] = F_D_I; f[5] = F_K4_I;
      *nf = 6;
      return GPM_OK;
    case GPM_QUERY_TC: f[0] = F_TRI; *nf = 1; return GPM_OK;
    case GPM_QUERY_CLIQUE4: f[0] = F_K4; *nf = 1; return GPM_OK;
    case GPM_QUERY_CLIQUE5: f[0] = F_K5; *nf = 1; return GPM_OK;
    default: return gpm_fail(GPM_E_INVALID_ARG, "unknown query kind " + std::to_string(kind));
  }
}

// Prepare a graph for item processing: orientation, root classes with the
// item bound on warp roots, and (for 4-motif queries) the 4-cycle root lists.
// hub_phase: the batched form's whole-GPU hub launches (units and tallies);
// hub_items: the served form's hub items (units only).
inline int prepare_for_items(gpm_graph *g, bool need_c4, cudaStream_t st, bool hub_phase = false,
                             bool hub_items = false) {
  int rc = gpm_prepare_graph(g, st);
  if (rc) return rc;
  const gpm_tuning &t = gpm_tune();
  if (g->cls_maxdeg[CLS_WARP] > kWarpMaxD || t.warp_max_degree > kWarpMaxD) {
    const uint32_t old_w = t.warp_max_degree;
    gpm_tune().warp_max_degree = std::min<uint32_t>(old_w, kWarpMaxD);
    g->tune_warp_max = 0;
    rc = gpm_ensure_classes(g, st);
    gpm_tune().warp_max_degree = old_w;
    if (rc) return rc;
  }
  if (need_c4) {
    rc = (hub_phase || hub_items) ? gpm_c4_hub_prepare(g, st, hub_phase) : gpm_build_c4_tasks(g, st);
    if (rc) return rc;
  }
  return GPM_OK;
}

// Shared memory of the item kernels: the largest of the item types' needs.
inline size_t item_smem_bytes(uint32_t smem_cta_maxd, bool need_c4) {
  const uint32_t W = std::max<uint32_t>(1, (smem_cta_maxd + 31) / 32);
  const size_t warp_bytes = (size_t)gpm_dev::warp_words(kWarpMaxD, true) * 4 * kWarps;
  const size_t cta_bytes = smem_cta_maxd ? gpm_dev::cta_words(smem_cta_maxd, W) * 4 : 0;
  const size_t c4_bytes = need_c4 ? std::max<size_t>((size_t)kWarps * 2 * gpm_dev::kC4HashSlots * 4,
                                                     (size_t)gpm_dev::c4_bucket_smem_words(kWarps) * 4)
                                  : 0;
  return std::max(warp_bytes, std::max(cta_bytes, c4_bytes));
}

// Largest CTA-root out-degree of a prepared graph (CTA and global classes).
inline uint32_t cta_root_maxd(const gpm_graph *g) {
  return std::max(g->cls_maxdeg[CLS_CTA], g->cls_maxdeg[CLS_XL]);
}

// Shared-memory and global-slot shapes of CTA items for roots up to maxd_all;
// allocates the global slots (one per CTA of the grid) when needed.
inline int setup_cta_items(ItemEnv &env, uint32_t maxd_all, int grid, uint32_t **pool_out) {
  env.cta_maxd = std::min(maxd_all, kItemCtaSmemMaxD);
  env.cta_W = std::max<uint32_t>(1, (env.cta_maxd + 31) / 32);
  env.lg_pool = nullptr;
  env.lg_slot_words = 0;
  env.lg_maxd = 0;
  env.lg_W = 1;
  if (maxd_all > kItemCtaSmemMaxD) {
    env.lg_maxd = maxd_all;
    env.lg_W = (maxd_all + 31) / 32;
    env.lg_slot_words = (gpm_dev::cta_words(maxd_all, env.lg_W) + 63) & ~63ull;
    if (cudaMalloc(pool_out, sizeof(uint32_t) * env.lg_slot_words * (size_t)grid) != cudaSuccess) {
      cudaGetLastError();
      return gpm_fail(GPM_E_OOM, "bitmap slot allocation failed");
    }
    env.lg_pool = *pool_out;
  }
  return GPM_OK;
}

}  // namespace gpm_item
