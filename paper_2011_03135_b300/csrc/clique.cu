// k-clique counting (k = 3, 4, 5 in one pass) over the degree-ordered
// orientation, by search on the local graph.
//
// Method (Section 5 "Search on Local Graph" and the k-CL local-graph listing
// of the appendix; orientation per appendix "Orientation (Total Order)"):
// every k-clique has exactly one order-first vertex u (its root), and its
// other k-1 vertices lie in L = N+(u). For root u the kernel builds the
// local graph on L as a bitmap adjacency R (row i = the positions j in L with
// an arc L[i] -> L[j]), i.e. the intersections N+(L[i]) ∩ L, and then
//   triangles rooted at u = sum_i |R_i|
//   4-cliques            = sum_i sum_{j in R_i} |R_i & R_j|
//   5-cliques            = sum_i sum_{j in R_i} sum_{l in R_i & R_j} |R_i & R_j & R_l|
// so each deeper DFS level of the paper's shrinking local graph becomes an
// AND of bit rows and the last level is counted with popc, not enumerated.
//
// Work distribution (replaces the paper's per-thread tasks with work
// stealing): roots are grouped by out-degree d into classes
//   d <= 32        one warp per root, one 32-bit word per row
//   d <= warp_max  one warp per root, W = ceil(d/32) words per row
//   d <= cta_max   one CTA per root, bitmap in shared memory
//   larger         one CTA per root, bitmap in a global-memory slot
// and every persistent warp/CTA pulls roots from a global atomic queue; the
// large classes are ordered by decreasing d (largest first).
//
// Building R is a load-balanced flat expansion: the concatenation of the
// lists N+(L[i]) is split evenly over the lanes (coalesced reads), each
// element is looked up in L by binary search in shared memory and sets one
// bit with a shared-memory atomicOr.
//
// Scatter mode (motif counting, Section 5 "Local Counting"): each triangle
// (u, L[i], L[j]) found while building also adds 1 to the triangle count of
// its three arcs, t_edge[u->L[i]], t_edge[u->L[j]] and t_edge[L[i]->L[j]].
#include <algorithm>

#include "gpm_internal.h"

namespace {

struct LGArgs {
  const uint64_t *__restrict__ drow;
  const uint32_t *__restrict__ dcol;
  const uint32_t *__restrict__ tasks;
  uint32_t ntasks;
  uint32_t root_lo, root_hi;
  uint32_t W;  // words per bitmap row (CTA / global classes)
  unsigned int *queue;
  unsigned long long *acc;  // acc[3] triangles, acc[4] 4-cliques, acc[5] 5-cliques
  uint32_t *t_edge;         // scatter mode
  uint32_t *pool;           // global-memory slots (XL class)
  uint64_t slot_words;
  unsigned int *status;
};

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
template <bool SCATTER>
__device__ __forceinline__ uint32_t build_rows(const LGArgs &a, const uint32_t *L, const uint32_t *pre,
                                               const uint64_t *xb, uint32_t *R, uint32_t *tc, uint32_t d,
                                               uint32_t W, uint32_t t, uint32_t nt) {
  const uint32_t E = pre[d];
  uint32_t found = 0;
  const uint32_t lo_id = L[0], hi_id = L[d - 1];
  for (uint32_t f = t; f < E; f += nt) {
    const uint32_t i = row_of(pre, d, f);
    const uint32_t p = f - pre[i];
    const uint64_t arc = xb[i] + p;
    const uint32_t y = __ldg(a.dcol + arc);
    if (y < lo_id || y > hi_id) continue;
    const uint32_t j = lower_bound_u32(L, d, y);
    if (j < d && L[j] == y) {
      atomicOr(&R[(size_t)i * W + (j >> 5)], 1u << (j & 31));
      ++found;
      if (SCATTER) {
        atomicAdd(&tc[i], 1u);
        atomicAdd(&tc[j], 1u);
        atomicAdd(&a.t_edge[arc], 1u);
      }
    }
  }
  return found;
}

// Enumerate pairs (i, j in R_i) and triples for the 4- and 5-clique terms.
// A group of G lanes handles one row at a time; lane gl of the group holds
// word gl of the row (W <= G), so every AND is one word per lane.
template <int G, int KMAX>
__device__ __forceinline__ void enumerate_rows(const uint32_t *R, uint32_t d, uint32_t W, uint32_t row0,
                                               uint32_t row_step, uint32_t gl, unsigned long long &a4,
                                               unsigned long long &a5) {
  for (uint32_t i = row0; i < d; i += row_step) {
    const uint32_t *ri = R + (size_t)i * W;
    const uint32_t riw = (gl < W) ? ri[gl] : 0u;
    for (uint32_t t = 0; t < W; ++t) {
      uint32_t bits = ri[t];
      while (bits) {
        const uint32_t j = t * 32 + __ffs(bits) - 1;
        bits &= bits - 1;
        const uint32_t *rj = R + (size_t)j * W;
        const uint32_t mw = (gl < W) ? (riw & rj[gl]) : 0u;
        a4 += __popc(mw);
        if (KMAX >= 5) {
          for (uint32_t t2 = 0; t2 < W; ++t2) {
            uint32_t b2 = ri[t2] & rj[t2];
            while (b2) {
              const uint32_t l = t2 * 32 + __ffs(b2) - 1;
              b2 &= b2 - 1;
              if (gl < W) a5 += __popc(mw & R[(size_t)l * W + gl]);
            }
          }
        }
      }
    }
  }
}

// Same for W > 32 (global-memory class): lane gl holds words gl, gl+G, ...
template <int KMAX>
__device__ void enumerate_rows_wide(const uint32_t *R, uint32_t d, uint32_t W, uint32_t row0, uint32_t row_step,
                                    uint32_t gl, unsigned long long &a4, unsigned long long &a5) {
  constexpr uint32_t G = 32;
  for (uint32_t i = row0; i < d; i += row_step) {
    const uint32_t *ri = R + (size_t)i * W;
    for (uint32_t t = 0; t < W; ++t) {
      uint32_t bits = ri[t];
      while (bits) {
        const uint32_t j = t * 32 + __ffs(bits) - 1;
        bits &= bits - 1;
        const uint32_t *rj = R + (size_t)j * W;
        for (uint32_t w = gl; w < W; w += G) a4 += __popc(ri[w] & rj[w]);
        if (KMAX >= 5) {
          for (uint32_t t2 = 0; t2 < W; ++t2) {
            uint32_t b2 = ri[t2] & rj[t2];
            while (b2) {
              const uint32_t l = t2 * 32 + __ffs(b2) - 1;
              b2 &= b2 - 1;
              const uint32_t *rl = R + (size_t)l * W;
              for (uint32_t w = gl; w < W; w += G) a5 += __popc(ri[w] & rj[w] & rl[w]);
            }
          }
        }
      }
    }
  }
}

__device__ __forceinline__ void flush_acc(const LGArgs &a, unsigned long long a3, unsigned long long a4,
                                          unsigned long long a5, int kmax) {
  for (int o = 16; o > 0; o >>= 1) {
    a3 += __shfl_down_sync(0xffffffffu, a3, o);
    a4 += __shfl_down_sync(0xffffffffu, a4, o);
    a5 += __shfl_down_sync(0xffffffffu, a5, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (a3) atomicAdd(&a.acc[3], a3);
    if (kmax >= 4 && a4) atomicAdd(&a.acc[4], a4);
    if (kmax >= 5 && a5) atomicAdd(&a.acc[5], a5);
  }
}

// ---------------------------------------------------------------------------
// one warp per root, bitmap in shared memory
// ---------------------------------------------------------------------------
template <int MAXD, int G, int KMAX, bool SCATTER>
__global__ void __launch_bounds__(256) lg_warp_kernel(LGArgs a) {
  constexpr uint32_t W = (MAXD + 31) / 32;
  // per-warp region: xb[MAXD] (uint64) | L[MAXD] | pre[MAXD+1] | R[MAXD*W] | tc[MAXD]
  constexpr uint32_t kWords = 2 * MAXD + MAXD + (MAXD + 1) + MAXD * W + (SCATTER ? MAXD : 0);
  constexpr uint32_t kStride = (kWords + 1) & ~1u;  // keep 8-byte alignment per warp
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t *base = smem + (size_t)wid * kStride;
  uint64_t *xb = reinterpret_cast<uint64_t *>(base);
  uint32_t *L = base + 2 * MAXD;
  uint32_t *pre = L + MAXD;
  uint32_t *R = pre + MAXD + 1;
  uint32_t *tc = R + MAXD * W;

  unsigned long long a3 = 0, a4 = 0, a5 = 0;
  for (;;) {
    uint32_t task = 0;
    if (lane == 0) task = atomicAdd(a.queue, 1u);
    task = __shfl_sync(0xffffffffu, task, 0);
    if (task >= a.ntasks) break;
    const uint32_t u = a.tasks[task];
    if (u < a.root_lo || u >= a.root_hi) continue;
    const uint64_t ub = a.drow[u];
    const uint32_t d = (uint32_t)(a.drow[u + 1] - ub);
    if (d < 2 || d > MAXD) continue;
    const uint32_t w_used = (d + 31) / 32;
    // stage L = N+(u), the row bases and the out-degrees of its members
    for (uint32_t i = lane; i < d; i += 32) {
      const uint32_t x = __ldg(a.dcol + ub + i);
      L[i] = x;
      const uint64_t xs = __ldg(a.drow + x), xe = __ldg(a.drow + x + 1);
      xb[i] = xs;
      pre[i + 1] = (uint32_t)(xe - xs);
      if (SCATTER) tc[i] = 0;
    }
    for (uint32_t i = lane; i < d * w_used; i += 32) R[i] = 0;
    if (lane == 0) pre[0] = 0;
    __syncwarp();
    // inclusive scan of pre[1..d] in chunks of 32
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
    a3 += build_rows<SCATTER>(a, L, pre, xb, R, tc, d, w_used, lane, 32);
    __syncwarp();
    if (SCATTER) {
      for (uint32_t i = lane; i < d; i += 32)
        if (tc[i]) atomicAdd(&a.t_edge[ub + i], tc[i]);
    }
    if (KMAX >= 4) enumerate_rows<G, KMAX>(R, d, w_used, lane / G, 32 / G, lane % G, a4, a5);
    __syncwarp();
  }
  (void)W;
  flush_acc(a, a3, a4, a5, KMAX);
}

// ---------------------------------------------------------------------------
// one CTA per root; bitmap in shared memory (GLOBAL = false) or in this
// CTA's global-memory slot (GLOBAL = true)
// ---------------------------------------------------------------------------
template <int G, int KMAX, bool SCATTER, bool GLOBAL>
__global__ void __launch_bounds__(512) lg_cta_kernel(LGArgs a, uint32_t maxd) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_task;
  const uint32_t W = a.W;
  uint32_t *base = GLOBAL ? a.pool + (size_t)blockIdx.x * a.slot_words : smem;
  uint64_t *xb = reinterpret_cast<uint64_t *>(base);
  uint32_t *L = base + 2 * (size_t)maxd;
  uint32_t *pre = L + maxd;
  uint32_t *R = pre + maxd + 1;
  uint32_t *tc = R + (size_t)maxd * W;
  const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;

  unsigned long long a3 = 0, a4 = 0, a5 = 0;
  for (;;) {
    if (tid == 0) s_task = atomicAdd(a.queue, 1u);
    __syncthreads();
    const uint32_t task = s_task;
    __syncthreads();
    if (task >= a.ntasks) break;
    const uint32_t u = a.tasks[task];
    if (u < a.root_lo || u >= a.root_hi) continue;
    const uint64_t ub = a.drow[u];
    const uint32_t d = (uint32_t)(a.drow[u + 1] - ub);
    if (d < 2 || d > maxd) continue;
    const uint32_t w_used = (d + 31) / 32;
    for (uint32_t i = tid; i < d; i += nt) {
      const uint32_t x = __ldg(a.dcol + ub + i);
      L[i] = x;
      const uint64_t xs = __ldg(a.drow + x), xe = __ldg(a.drow + x + 1);
      xb[i] = xs;
      pre[i + 1] = (uint32_t)(xe - xs);
      if (SCATTER) tc[i] = 0;
    }
    for (size_t i = tid; i < (size_t)d * w_used; i += nt) R[i] = 0;
    if (tid == 0) pre[0] = 0;
    __syncthreads();
    // inclusive scan of pre[1..d] by warp 0
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
    a3 += build_rows<SCATTER>(a, L, pre, xb, R, tc, d, w_used, tid, nt);
    __syncthreads();
    if (SCATTER) {
      for (uint32_t i = tid; i < d; i += nt)
        if (tc[i]) atomicAdd(&a.t_edge[ub + i], tc[i]);
    }
    if (KMAX >= 4) {
      if (GLOBAL && w_used > 32)
        enumerate_rows_wide<KMAX>(R, d, w_used, tid / 32, nt / 32, lane, a4, a5);
      else
        enumerate_rows<G, KMAX>(R, d, w_used, tid / G, nt / G, tid % G, a4, a5);
    }
    __syncthreads();
  }
  flush_acc(a, a3, a4, a5, KMAX);
}

constexpr uint32_t warp_words(uint32_t maxd, bool scatter) {
  return ((2 * maxd + maxd + (maxd + 1) + maxd * ((maxd + 31) / 32) + (scatter ? maxd : 0)) + 1) & ~1u;
}

uint64_t cta_words(uint32_t maxd, uint32_t W) {
  return 2ull * maxd + maxd + (maxd + 1) + (uint64_t)maxd * W + maxd + 2;
}

template <int MAXD, int G, int KMAX, bool SCATTER>
int launch_warp(const LGArgs &a, int device, cudaStream_t st) {
  constexpr int kThreads = 256;
  const size_t smem = (size_t)warp_words(MAXD, SCATTER) * 4 * (kThreads / 32);
  auto kern = lg_warp_kernel<MAXD, G, KMAX, SCATTER>;
  GPM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
  if (per_sm < 1) per_sm = 1;
  if (gpm_tune().blocks_per_sm) per_sm = std::min<int>(per_sm, gpm_tune().blocks_per_sm);
  int blocks = gpm_num_sms(device) * per_sm;
  const int need = (int)((a.ntasks + (kThreads / 32) - 1) / (kThreads / 32));
  blocks = std::max(1, std::min(blocks, need));
  GPM_LAUNCH(MAXD <= 32 ? "lg_warp_d32" : "lg_warp", st, kern<<<blocks, kThreads, smem, st>>>(a));
  GPM_CUDA(cudaGetLastError());
  return GPM_OK;
}

template <int G, int KMAX, bool SCATTER, bool GLOBAL>
int launch_cta(const LGArgs &a, uint32_t maxd, int blocks_cap, int device, cudaStream_t st) {
  constexpr int kThreads = 512;
  const size_t smem = GLOBAL ? 0 : (size_t)cta_words(maxd, a.W) * 4;
  auto kern = lg_cta_kernel<G, KMAX, SCATTER, GLOBAL>;
  if (!GLOBAL) GPM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
  if (per_sm < 1) per_sm = 1;
  int blocks = gpm_num_sms(device) * per_sm;
  blocks = std::max(1, std::min<int>(blocks, (int)a.ntasks));
  if (blocks_cap > 0) blocks = std::min(blocks, blocks_cap);
  GPM_LAUNCH(GLOBAL ? "lg_cta_global" : "lg_cta", st, kern<<<blocks, kThreads, smem, st>>>(a, maxd));
  GPM_CUDA(cudaGetLastError());
  return GPM_OK;
}

template <int KMAX, bool SCATTER>
int launch_all(gpm_graph *g, LGArgs base, unsigned int *queues, cudaStream_t st) {
  const int dev = g->device;
  // class W32: d <= 32
  {
    LGArgs a = base;
    a.tasks = g->tasks + g->cls_begin[CLS_W32];
    a.ntasks = g->cls_begin[CLS_W32 + 1] - g->cls_begin[CLS_W32];
    a.queue = queues + 0;
    if (a.ntasks) GPM_TRY((launch_warp<32, 1, KMAX, SCATTER>(a, dev, st)));
  }
  // class WARP: 32 < d <= warp_max (<= 256)
  {
    LGArgs a = base;
    a.tasks = g->tasks + g->cls_begin[CLS_WARP];
    a.ntasks = g->cls_begin[CLS_WARP + 1] - g->cls_begin[CLS_WARP];
    a.queue = queues + 1;
    const uint32_t md = g->cls_maxdeg[CLS_WARP];
    if (a.ntasks) {
      if (md <= 64) GPM_TRY((launch_warp<64, 2, KMAX, SCATTER>(a, dev, st)));
      else if (md <= 128) GPM_TRY((launch_warp<128, 4, KMAX, SCATTER>(a, dev, st)));
      else GPM_TRY((launch_warp<256, 8, KMAX, SCATTER>(a, dev, st)));
    }
  }
  // class CTA: shared-memory bitmap
  {
    LGArgs a = base;
    a.tasks = g->tasks + g->cls_begin[CLS_CTA];
    a.ntasks = g->cls_begin[CLS_CTA + 1] - g->cls_begin[CLS_CTA];
    a.queue = queues + 2;
    const uint32_t md = g->cls_maxdeg[CLS_CTA];
    a.W = (md + 31) / 32;
    if (a.ntasks) {
      if (a.W <= 8) GPM_TRY((launch_cta<8, KMAX, SCATTER, false>(a, md, 0, dev, st)));
      else if (a.W <= 16) GPM_TRY((launch_cta<16, KMAX, SCATTER, false>(a, md, 0, dev, st)));
      else GPM_TRY((launch_cta<32, KMAX, SCATTER, false>(a, md, 0, dev, st)));
    }
  }
  // class XL: global-memory bitmaps, one slot per resident CTA
  {
    LGArgs a = base;
    a.tasks = g->tasks + g->cls_begin[CLS_XL];
    a.ntasks = g->cls_begin[CLS_XL + 1] - g->cls_begin[CLS_XL];
    a.queue = queues + 3;
    const uint32_t md = g->cls_maxdeg[CLS_XL];
    if (a.ntasks) {
      a.W = (md + 31) / 32;
      a.slot_words = (cta_words(md, a.W) + 63) & ~63ull;
      const size_t slot_bytes = a.slot_words * 4;
      const size_t budget = (size_t)4 << 30;
      int slots = (int)std::min<size_t>(std::min<size_t>(budget / slot_bytes, (size_t)gpm_num_sms(dev)),
                                        (size_t)a.ntasks);
      if (slots < 1)
        return gpm_fail(GPM_E_UNSUPPORTED, "root out-degree " + std::to_string(md) +
                                               " needs a local-graph bitmap larger than the 4 GiB slot budget");
      if (g->xl_pool_bytes < (size_t)slots * slot_bytes) {
        if (g->xl_pool) {
          cudaFree(g->xl_pool);
          g->device_bytes -= g->xl_pool_bytes;
          g->xl_pool = nullptr;
          g->xl_pool_bytes = 0;
        }
        GPM_TRY(gpm_graph_alloc(g, (void **)&g->xl_pool, (size_t)slots * slot_bytes));
        g->xl_pool_bytes = (size_t)slots * slot_bytes;
      }
      a.pool = g->xl_pool;
      if (a.W <= 8) GPM_TRY((launch_cta<8, KMAX, SCATTER, true>(a, md, slots, dev, st)));
      else if (a.W <= 16) GPM_TRY((launch_cta<16, KMAX, SCATTER, true>(a, md, slots, dev, st)));
      else GPM_TRY((launch_cta<32, KMAX, SCATTER, true>(a, md, slots, dev, st)));
    }
  }
  return GPM_OK;
}

}  // namespace

int gpm_launch_cliques(gpm_graph *g, int kmax, bool scatter, uint32_t root_lo, uint32_t root_hi,
                       unsigned long long *acc, cudaStream_t st) {
  if (kmax < 3 || kmax > 5) return gpm_fail(GPM_E_UNSUPPORTED, "clique pass supports k = 3..5");
  unsigned int *queues = reinterpret_cast<unsigned int *>(g->work + WK_QUEUE0);
  GPM_CUDA(cudaMemsetAsync(queues, 0, 8 * sizeof(unsigned int), st));
  LGArgs a{};
  a.drow = g->drow;
  a.dcol = g->dcol;
  a.root_lo = root_lo;
  a.root_hi = root_hi;
  a.acc = acc;
  a.t_edge = g->t_edge;
  a.status = reinterpret_cast<unsigned int *>(g->work + WK_STATUS);
  if (scatter && !g->t_edge) return gpm_fail(GPM_E_INVALID_ARG, "scatter pass without a per-arc buffer");
  if (scatter) {
    if (kmax == 3) return launch_all<3, true>(g, a, queues, st);
    return launch_all<4, true>(g, a, queues, st);
  }
  if (kmax == 3) return launch_all<3, false>(g, a, queues, st);
  if (kmax == 4) return launch_all<4, false>(g, a, queues, st);
  return launch_all<5, false>(g, a, queues, st);
}
