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
#include "lg_device.cuh"

namespace {

struct LGArgs {
  const uint64_t *__restrict__ drow;
  const uint32_t *__restrict__ dcol;
  const uint32_t *__restrict__ deg;  // undirected degrees (orientation order of local vertices)
  const uint32_t *__restrict__ tasks;
  uint32_t ntasks;
  uint32_t root_lo, root_hi;
  uint32_t W;  // words per bitmap row (CTA / global classes)
  unsigned int *queue;
  unsigned long long *acc;  // acc[3] triangles, acc[4..6] 4- to 6-cliques; k >= 7: acc[k - 7]
  uint32_t *t_edge;         // scatter mode
  uint32_t *pool;           // global-memory slots (XL class)
  uint64_t slot_words;
  uint32_t slices;          // CTAs per root (k >= 7: a root's units are split over them)
  unsigned int *ucount;     // k >= 7: per-task unit counters shared by a root's CTAs (zero at launch)
  unsigned int *status;
};

__device__ __forceinline__ void flush_acc(const LGArgs &a, unsigned long long a3, unsigned long long a4,
                                          unsigned long long a5, unsigned long long a6, int kmax) {
  bool c3 = false, c4 = false, c5 = false, c6 = false;
  if (kmax >= 7) {
    // the generic pass adds only its own clique size (a6 carries it)
    a6 = warp_sum_checked(a6, c6);
    if ((threadIdx.x & 31) == 0) acc_add_checked(&a.acc[kmax - 7], a6, c6, a.status, kmax - 7);
    return;
  }
  a3 = warp_sum_checked(a3, c3);
  a4 = warp_sum_checked(a4, c4);
  a5 = warp_sum_checked(a5, c5);
  if (kmax >= 6) a6 = warp_sum_checked(a6, c6);
  if ((threadIdx.x & 31) == 0) {
    acc_add_checked(&a.acc[3], a3, c3, a.status, ACC_T);
    if (kmax >= 4) acc_add_checked(&a.acc[4], a4, c4, a.status, ACC_K4);
    if (kmax >= 5) acc_add_checked(&a.acc[5], a5, c5, a.status, ACC_K5);
    if (kmax >= 6) acc_add_checked(&a.acc[ACC_K6], a6, c6, a.status, ACC_K6);
  }
}

// ---------------------------------------------------------------------------
// one warp per root, bitmap in shared memory
// ---------------------------------------------------------------------------
// per-warp shared words: the local graph, then (k >= 7) the generic search's scratch
template <int MAXD, int KMAX, bool SCATTER>
__host__ __device__ constexpr uint32_t warp_stride() {
  return gpm_dev::warp_words(MAXD, SCATTER) + (KMAX >= 7 ? gpm_dev::gen_warp_words(1) : 0);
}

template <int MAXD, int G, int KMAX, bool SCATTER>
__global__ void __launch_bounds__(256) lg_warp_kernel(LGArgs a) {
  constexpr uint32_t kStride = warp_stride<MAXD, KMAX, SCATTER>();
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t *base = smem + (size_t)wid * kStride;
  unsigned long long a3 = 0, a4 = 0, a5 = 0, a6 = 0;
  // roots are claimed kClaim at a time: the warp classes hold most of the
  // vertices, and one atomic per root on a single counter would serialise
  // the warps
  constexpr uint32_t kClaim = 4;
  for (;;) {
    uint32_t first = 0;
    if (lane == 0) first = atomicAdd(a.queue, kClaim);
    first = __shfl_sync(0xffffffffu, first, 0);
    if (first >= a.ntasks) break;
    const uint32_t last = first + kClaim < a.ntasks ? first + kClaim : a.ntasks;
    for (uint32_t task = first; task < last; ++task) {
      const uint32_t u = a.tasks[task];
      if (u < a.root_lo || u >= a.root_hi) continue;
      const uint32_t d = (uint32_t)(a.drow[u + 1] - a.drow[u]);
      if (d < 2 || d > MAXD) continue;
      gpm_dev::lg_root_warp<MAXD, G, KMAX, SCATTER>(a.drow, a.dcol, a.t_edge, u, base, a3, a4, a5, a6,
                                                    base + gpm_dev::warp_words(MAXD, SCATTER));
    }
  }
  flush_acc(a, a3, a4, a5, a6, KMAX);
}

// ---------------------------------------------------------------------------
// one CTA per root; bitmap in shared memory (GLOBAL = false) or in this
// CTA's global-memory slot (GLOBAL = true)
// ---------------------------------------------------------------------------
template <int G, int KMAX, bool SCATTER, bool GLOBAL, int THREADS, int NWLG = 4>
__global__ void __launch_bounds__(THREADS) lg_cta_kernel(LGArgs a, uint32_t maxd, uint32_t big_cap, uint32_t wcap) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_task;
  uint32_t *base = GLOBAL ? a.pool + (size_t)blockIdx.x * a.slot_words : smem;
  // nested local graphs for the 5-clique level live after the bitmap (shared memory only)
  uint32_t *nest = (!GLOBAL && KMAX >= 5 && big_cap) ? smem + gpm_dev::cta_words(maxd, a.W) : nullptr;
  // k >= 7 with global-memory bitmaps: the generic search's counter and
  // per-warp scratch, for rows of up to 32 NWLG words: in static shared memory
  // (NWLG = 4), or in the dynamic shared memory, which global-memory bitmaps
  // leave unused (NWLG = 16)
  constexpr int kNwl = (GLOBAL && KMAX >= 7) ? NWLG : 1;
  __shared__ uint32_t gen_s[(GLOBAL && KMAX >= 7 && NWLG <= 4) ? 4 + (THREADS / 32) * gpm_dev::gen_warp_words(4) : 1];
  uint32_t *gen = (GLOBAL && KMAX >= 7) ? (NWLG <= 4 ? gen_s : smem) : nullptr;
  unsigned long long a3 = 0, a4 = 0, a5 = 0, a6 = 0;
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(a.queue, 1u);
    __syncthreads();
    const uint32_t task = s_task;
    __syncthreads();
    if (task >= a.ntasks * a.slices) break;
    const uint32_t u = a.tasks[task / a.slices];
    if (u < a.root_lo || u >= a.root_hi) continue;
    const uint32_t d = (uint32_t)(a.drow[u + 1] - a.drow[u]);
    if (d < 2 || d > maxd) continue;
    gpm_dev::lg_root_cta<G, KMAX, SCATTER, kNwl>(a.drow, a.dcol, a.t_edge, u, maxd, a.W, base, a3, a4, a5, a6,
                                                 nest, big_cap, a.deg, wcap, gen, task % a.slices, a.slices,
                                                 a.ucount ? a.ucount + task / a.slices : nullptr);
  }
  flush_acc(a, a3, a4, a5, a6, KMAX);
}

using gpm_dev::cta_words;
using gpm_dev::warp_words;

template <int MAXD, int G, int KMAX, bool SCATTER>
int launch_warp(const LGArgs &a, int device, cudaStream_t st) {
  constexpr int kThreads = 256;
  const size_t smem = (size_t)warp_stride<MAXD, KMAX, SCATTER>() * 4 * (kThreads / 32);
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

int max_smem_optin(int device) {
  static int cached[64] = {0};
  if (device < 0 || device >= 64) return 227 * 1024;
  if (!cached[device]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 227 * 1024;
    }
    cached[device] = v;
  }
  return cached[device];
}

// THREADS = 1024 (32 warps, one CTA per SM) for the largest shared-memory
// roots with the nested 5-clique search: 32 warp buffers for rows of up to
// 128 candidates fit beside a bitmap of up to 1024 rows, and the big-row
// groups reuse the same pool afterwards.
template <int G, int KMAX, bool SCATTER, bool GLOBAL, int THREADS, int NWLG = 4>
int launch_cta_t(const LGArgs &a, uint32_t maxd, int blocks_cap, int device, cudaStream_t st, size_t smem_limit,
                 const char *name) {
  size_t smem = GLOBAL ? 0 : (size_t)cta_words(maxd, a.W) * 4;
  if (GLOBAL && KMAX >= 7 && NWLG > 4) smem = (4 + (size_t)(THREADS / 32) * gpm_dev::gen_warp_words(NWLG)) * 4;
  const size_t limit = smem_limit ? smem_limit : (size_t)max_smem_optin(device);
  // one-warp rows of up to 128 candidates when their buffers fit, else 64
  uint32_t wcap = gpm_dev::kNestWarpC;
  if (smem + (size_t)gpm_dev::nest_words(maxd, THREADS / 32, 0, wcap) * 4 + 2048 + 4 * 1024 > limit) wcap = 64;
  uint32_t big_cap = 0;
  if (!GLOBAL && KMAX >= 5) {
    // room left after the bitmap and the per-warp nested buffers goes to the CTA-wide nested buffer
    const size_t fixed = smem + (size_t)gpm_dev::nest_words(maxd, THREADS / 32, 0, wcap) * 4 + 2048;
    if (fixed + 4 * 1024 <= limit) {
      big_cap = (uint32_t)std::min<size_t>((limit - fixed) / 4, 32768);
      smem += (size_t)gpm_dev::nest_words(maxd, THREADS / 32, big_cap, wcap) * 4;
    }
  }
  if (KMAX >= 7 && !GLOBAL &&
      (big_cap == 0 || gpm_dev::nest_warp_words(wcap) < gpm_dev::gen_warp_words(1) + 4))
    return gpm_fail(GPM_E_UNSUPPORTED, "no shared memory left for the generic clique search's scratch");
  auto kern = lg_cta_kernel<G, KMAX, SCATTER, GLOBAL, THREADS, NWLG>;
  if (smem) GPM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, smem));
  if (per_sm < 1) per_sm = 1;
  int blocks = gpm_num_sms(device) * per_sm;
  blocks = std::max(1, std::min<int>(blocks, (int)(a.ntasks * a.slices)));
  if (blocks_cap > 0) blocks = std::min(blocks, blocks_cap);
  GPM_LAUNCH(name ? name : (GLOBAL ? "lg_cta_global" : "lg_cta"), st,
             kern<<<blocks, THREADS, smem, st>>>(a, maxd, big_cap, wcap));
  GPM_CUDA(cudaGetLastError());
  return GPM_OK;
}

template <int G, int KMAX, bool SCATTER, bool GLOBAL, int NWLG = 4>
int launch_cta(const LGArgs &a, uint32_t maxd, int blocks_cap, int device, cudaStream_t st,
               size_t smem_limit = 0, const char *name = nullptr, bool wide = false) {
  if (KMAX >= 5 && !GLOBAL && wide)
    return launch_cta_t<G, KMAX, SCATTER, GLOBAL, 1024>(a, maxd, blocks_cap, device, st, smem_limit, name);
  return launch_cta_t<G, KMAX, SCATTER, GLOBAL, 512, NWLG>(a, maxd, blocks_cap, device, st, smem_limit, name);
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
    if (KMAX >= 7 && a.ntasks) {
      // the generic search spreads a root over a CTA (a heavy local graph in
      // one warp would be the last to finish)
      a.W = (md + 31) / 32;
      a.slices = 2;  // lighter roots than the CTA class: two CTAs each (measured best of 2, 4, 8, 16)
      if (base.ucount) a.ucount = base.ucount + g->cls_begin[CLS_WARP];
      GPM_TRY((launch_cta<32, KMAX, SCATTER, false>(a, md, 0, dev, st, (size_t)(max_smem_optin(dev) / 2 - 1024),
                                                    "lg_cta_mid")));
    } else if (a.ntasks) {
      if (md <= 64) GPM_TRY((launch_warp<64, 2, KMAX, SCATTER>(a, dev, st)));
      else if (md <= 128) GPM_TRY((launch_warp<128, 4, KMAX, SCATTER>(a, dev, st)));
      else GPM_TRY((launch_warp<256, 8, KMAX, SCATTER>(a, dev, st)));
    }
  }
  // class CTA: shared-memory bitmap; roots above the split degree with the
  // largest footprint, the rest sized for two CTAs per SM
  for (int part = 0; part < 2; ++part) {
    LGArgs a = base;
    const uint32_t b0 = part == 0 ? g->cls_begin[CLS_CTA] : g->cta_split;
    const uint32_t b1 = part == 0 ? g->cta_split : g->cls_begin[CLS_CTA + 1];
    a.tasks = g->tasks + b0;
    a.ntasks = b1 - b0;
    a.queue = queues + (part == 0 ? 2 : 6);
    if (base.ucount) a.ucount = base.ucount + b0;
    const uint32_t md = part == 0 ? g->cls_maxdeg[CLS_CTA] : g->cta_lo_maxd;
    a.W = (md + 31) / 32;
    const size_t limit = part == 0 ? 0 : (size_t)(max_smem_optin(dev) / 2 - 1024);
    const char *nm = part == 0 ? "lg_cta_hi" : "lg_cta_lo";
    if (a.ntasks) {
      const bool wide = part == 0;
      if constexpr (KMAX >= 7) {
        // the generic search does not use the row-group width
        GPM_TRY((launch_cta<32, KMAX, SCATTER, false>(a, md, 0, dev, st, limit, nm, wide && a.W > 8)));
      } else {
        if (a.W <= 8) GPM_TRY((launch_cta<8, KMAX, SCATTER, false>(a, md, 0, dev, st, limit, nm)));
        else if (a.W <= 16) GPM_TRY((launch_cta<16, KMAX, SCATTER, false>(a, md, 0, dev, st, limit, nm, wide)));
        else GPM_TRY((launch_cta<32, KMAX, SCATTER, false>(a, md, 0, dev, st, limit, nm, wide)));
      }
    }
  }
  // class XL: global-memory bitmaps, one slot per resident CTA
  {
    LGArgs a = base;
    a.tasks = g->tasks + g->cls_begin[CLS_XL];
    a.ntasks = g->cls_begin[CLS_XL + 1] - g->cls_begin[CLS_XL];
    a.queue = queues + 3;
    if (base.ucount) a.ucount = base.ucount + g->cls_begin[CLS_XL];
    const uint32_t md = g->cls_maxdeg[CLS_XL];
    if (a.ntasks) {
      a.W = (md + 31) / 32;
      if (KMAX >= 7 && a.W > 512)
        return gpm_fail(GPM_E_UNSUPPORTED, "k-clique counting for k >= 7 supports root out-degrees up to 16384 "
                                           "(this graph has " + std::to_string(md) + ")");
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
      if constexpr (KMAX >= 7) {
        if (a.W > 128) GPM_TRY((launch_cta<32, KMAX, SCATTER, true, 16>(a, md, slots, dev, st)));
        else GPM_TRY((launch_cta<32, KMAX, SCATTER, true>(a, md, slots, dev, st)));
      } else {
        if (a.W <= 8) GPM_TRY((launch_cta<8, KMAX, SCATTER, true>(a, md, slots, dev, st)));
        else if (a.W <= 16) GPM_TRY((launch_cta<16, KMAX, SCATTER, true>(a, md, slots, dev, st)));
        else GPM_TRY((launch_cta<32, KMAX, SCATTER, true>(a, md, slots, dev, st)));
      }
    }
  }
  return GPM_OK;
}

}  // namespace

int gpm_launch_cliques(gpm_graph *g, int kmax, bool scatter, uint32_t root_lo, uint32_t root_hi,
                       unsigned long long *acc, cudaStream_t st) {
  if (kmax < 3 || kmax > 9) return gpm_fail(GPM_E_UNSUPPORTED, "clique pass supports k = 3..9");
  if (kmax >= 7 && scatter) return gpm_fail(GPM_E_INVALID_ARG, "the per-arc scatter pass runs with k <= 4");
  unsigned int *queues = reinterpret_cast<unsigned int *>(g->work + WK_QUEUE0);
  GPM_CUDA(cudaMemsetAsync(queues, 0, 8 * sizeof(unsigned int), st));
  LGArgs a{};
  a.slices = kmax >= 7 ? 4u : 1u;
  if (kmax >= 7) {
    // one unit counter per root task of the CTA classes, shared by the root's CTAs
    const size_t words = std::max<uint32_t>(g->n, 1);
    if (!g->gen_ucount) GPM_TRY(gpm_graph_alloc(g, (void **)&g->gen_ucount, sizeof(unsigned int) * words));
    GPM_CUDA(cudaMemsetAsync(g->gen_ucount, 0, sizeof(unsigned int) * words, st));
    a.ucount = g->gen_ucount;
  }
  a.drow = g->drow;
  a.dcol = g->dcol;
  a.deg = g->okey ? g->okey : g->deg;  // the key of the orientation order
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
  if (kmax == 5) return launch_all<5, false>(g, a, queues, st);
  if (kmax == 7) return launch_all<7, false>(g, a, queues, st);
  if (kmax == 8) return launch_all<8, false>(g, a, queues, st);
  if (kmax == 9) return launch_all<9, false>(g, a, queues, st);
  return launch_all<6, false>(g, a, queues, st);
}
