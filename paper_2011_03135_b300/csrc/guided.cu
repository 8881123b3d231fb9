// Pattern-guided search for any connected pattern of up to 8 vertices
// (explicit-pattern problems of Section 2: counting, listing, existence),
// driven by the planner's output (plan.cpp):
//   - the matching order (appendix "Pattern-Guided Search (Matching Order)"):
//     pattern vertex order[j] is matched at level j; every level is adjacent
//     in the pattern to an earlier one;
//   - the symmetry-breaking partial order (appendix "Symmetry Breaking
//     (Partial Order)"): a pair (a, b) requires id(f(a)) < id(f(b)), which
//     becomes a lower or an upper id bound on the candidates of the later
//     level; it leaves one match per distinct subgraph, so counting matches
//     counts subgraphs;
//   - the degree filter (Section 4.3): a candidate for pattern vertex v needs
//     graph degree >= the degree of v in the pattern.
// The candidates of level j are the neighbours of one matched vertex adjacent
// to order[j] in the pattern (the one of smallest graph degree), kept if they
// are adjacent to the other matched vertices adjacent to order[j] (set
// intersection by binary search in the sorted lists), not adjacent to the
// non-adjacent ones when the pattern is vertex-induced (set difference),
// distinct from the matched vertices, within the id bounds and the degree
// filter.
//
// GPU mapping: a work item is an arc (u0, u1) matched to the first two
// pattern vertices of the order; warps claim chunks of adjacency positions
// from a global counter and walk each item's search tree depth first, the
// lanes sharing the filtering of one candidate list (compacted with a
// ballot). Levels 2 .. k-2 keep their candidate lists in per-warp scratch;
// the last level is counted (or its matches written) without being stored.
#include <algorithm>
#include <cstring>
#include <vector>

#include "gpm_internal.h"

namespace {

constexpr int kGuidedThreads = 256;
constexpr int kGuidedWarps = kGuidedThreads / 32;
constexpr uint32_t kGuidedChunk = 32;

struct GuidedArgs {
  const uint64_t *__restrict__ rowptr;
  const uint32_t *__restrict__ col;
  const uint32_t *__restrict__ deg;
  uint32_t n;
  uint64_t nnz;
  GuidedPlan plan;
  unsigned long long *queue;   // adjacency positions claimed so far
  uint32_t *scratch;           // per warp: levels 2 .. k-2, `cap` words each
  uint64_t cap;
  unsigned long long *acc;     // count (when out == nullptr)
  uint32_t *out;               // listing: tuples of k vertices in pattern order
  uint64_t out_cap;
  unsigned long long *counter; // listing: slots reserved so far
  unsigned int *status;
};

__device__ __forceinline__ bool adjacent(const uint64_t *__restrict__ rowptr, const uint32_t *__restrict__ col,
                                         uint32_t x, uint32_t u) {
  uint64_t lo = rowptr[x], hi = rowptr[x + 1];
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    const uint32_t c = __ldg(col + mid);
    if (c == u) return true;
    if (c < u) lo = mid + 1;
    else hi = mid;
  }
  return false;
}

__device__ __forceinline__ bool listing_full(const GuidedArgs &a) {
  return a.out && *(volatile const unsigned long long *)a.counter >= a.out_cap;
}

// Does x pass the tests of level j against the matched vertices M[0 .. j-1]
// (the pivot's adjacency is implied by x coming from its list)?
__device__ __forceinline__ bool candidate_ok(const GuidedArgs &a, const uint32_t *M, uint32_t j, uint32_t piv,
                                             uint32_t x) {
  const GuidedPlan &p = a.plan;
  if (__ldg(a.deg + x) < p.mindeg[j]) return false;
  for (uint32_t i = 0; i < j; ++i) {
    const uint32_t mi = M[i];
    if (x == mi) return false;
    if ((p.lower[j] >> i & 1u) && !(mi < x)) return false;
    if ((p.upper[j] >> i & 1u) && !(x < mi)) return false;
  }
  for (uint32_t i = 0; i < j; ++i) {
    if (i == piv) continue;
    const bool c = p.conn[j] >> i & 1u;
    if (c) {
      if (!adjacent(a.rowptr, a.col, M[i], x)) return false;
    } else if (p.induced) {
      if (adjacent(a.rowptr, a.col, M[i], x)) return false;
    }
  }
  return true;
}

__global__ void __launch_bounds__(kGuidedThreads) guided_kernel(GuidedArgs a) {
  __shared__ uint32_t s_M[kGuidedWarps][8], s_n[kGuidedWarps][8], s_i[kGuidedWarps][8];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint64_t gw = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint32_t k = a.plan.k;
  uint32_t *M = s_M[wid], *N = s_n[wid], *I = s_i[wid];
  uint32_t *lists = a.scratch + gw * a.cap * 8;  // level j at lists + j * cap
  unsigned long long cnt = 0;
  bool stop = false;
  while (!stop) {
    unsigned long long p0 = 0;
    if (lane == 0) p0 = atomicAdd(a.queue, (unsigned long long)kGuidedChunk);
    p0 = __shfl_sync(0xffffffffu, p0, 0);
    if (p0 >= a.nnz) break;
    const uint64_t p1 = min((uint64_t)p0 + kGuidedChunk, a.nnz);
    uint32_t u0;
    {
      uint32_t lo = 0, hi = a.n;  // largest v with rowptr[v] <= p0
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a.rowptr[mid] <= p0) lo = mid;
        else hi = mid;
      }
      u0 = lo;
    }
    for (uint64_t q = p0; q < p1; ++q) {
      while (a.rowptr[u0 + 1] <= q) ++u0;
      if (listing_full(a)) {
        stop = true;
        break;
      }
      const uint32_t u1 = __ldg(a.col + q);
      // levels 0 and 1: the arc (u0, u1)
      if (__ldg(a.deg + u0) < a.plan.mindeg[0] || __ldg(a.deg + u1) < a.plan.mindeg[1]) continue;
      if ((a.plan.lower[1] & 1u) && !(u0 < u1)) continue;
      if ((a.plan.upper[1] & 1u) && !(u1 < u0)) continue;
      if (lane == 0) {
        M[0] = u0;
        M[1] = u1;
      }
      __syncwarp();
      uint32_t j = 2;
      bool build = true;
      for (;;) {
        if (build) {
          // candidates of level j: the list of the adjacent matched vertex of smallest degree
          uint32_t piv = 0, pd = 0xffffffffu;
          for (uint32_t i = 0; i < j; ++i)
            if (a.plan.conn[j] >> i & 1u) {
              const uint32_t d = __ldg(a.deg + M[i]);
              if (d < pd) {
                pd = d;
                piv = i;
              }
            }
          const uint64_t b = a.rowptr[M[piv]], e = a.rowptr[M[piv] + 1];
          const bool last = (j + 1 == k);
          uint32_t *L = lists + (uint64_t)j * a.cap;
          uint32_t nl = 0;
          for (uint64_t t0 = b; t0 < e; t0 += 32) {
            const uint64_t t = t0 + lane;
            uint32_t x = 0;
            bool ok = false;
            if (t < e) {
              x = __ldg(a.col + t);
              ok = candidate_ok(a, M, j, piv, x);
            }
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            if (!m) continue;
            if (!last) {
              if (ok) L[nl + __popc(m & ((1u << lane) - 1u))] = x;
            } else if (!a.out) {
              if (lane == 0) cnt += __popc(m);
            } else {
              uint64_t slot = 0;
              if (lane == 0) slot = atomicAdd(a.counter, (unsigned long long)__popc(m));
              slot = __shfl_sync(0xffffffffu, slot, 0) + __popc(m & ((1u << lane) - 1u));
              if (ok && slot < a.out_cap) {
                uint32_t *row = a.out + slot * k;
                for (uint32_t i = 0; i < j; ++i) row[a.plan.order[i]] = M[i];
                row[a.plan.order[j]] = x;
              }
            }
            nl += __popc(m);
          }
          __syncwarp();
          if (lane == 0) {
            N[j] = last ? 0u : nl;
            I[j] = 0;
          }
          __syncwarp();
          build = false;
        }
        // next candidate of level j, or back up
        if (I[j] < N[j]) {
          if (lane == 0) {
            M[j] = lists[(uint64_t)j * a.cap + I[j]];
            I[j] = I[j] + 1;
          }
          __syncwarp();
          ++j;
          build = true;
          continue;
        }
        if (j == 2) break;
        --j;
      }
    }
  }
  cnt = __shfl_sync(0xffffffffu, cnt, 0);
  if (lane == 0 && !a.out) acc_add_checked(a.acc, cnt, false, a.status, -1);
}

}  // namespace

int gpm_guided_plan(const gpm_pattern &p, GuidedPlan *plan) {
  const gpm_pattern_info_t &info = p.info;
  const uint32_t k = p.k;
  if (k < 3 || k > 8) return gpm_fail(GPM_E_UNSUPPORTED, "the pattern-guided search covers patterns with 3..8 vertices");
  std::memset(plan, 0, sizeof(*plan));
  plan->k = k;
  plan->induced = p.induced ? 1u : 0u;
  uint32_t level_of[8];
  for (uint32_t j = 0; j < k; ++j) {
    plan->order[j] = info.matching_order[j];
    level_of[info.matching_order[j]] = j;
  }
  for (uint32_t j = 0; j < k; ++j) {
    const uint32_t v = plan->order[j];
    plan->mindeg[j] = info.min_degree[v];
    for (uint32_t i = 0; i < j; ++i)
      if (p.adj[plan->order[i] * k + v]) plan->conn[j] |= 1u << i;
    if (j > 0 && !plan->conn[j]) return gpm_fail(GPM_E_INVALID_ARG, "internal: matching order is not connected");
  }
  for (uint32_t s = 0; s < info.n_sb_pairs; ++s) {
    const uint32_t a = info.sb_pairs[2 * s], b = info.sb_pairs[2 * s + 1];  // id(f(a)) < id(f(b))
    const uint32_t la = level_of[a], lb = level_of[b];
    if (la < lb) plan->lower[lb] |= 1u << la;  // f(b) > f(a), a matched first
    else plan->upper[la] |= 1u << lb;          // f(a) < f(b), b matched first
  }
  return GPM_OK;
}

int gpm_launch_guided(gpm_graph *g, const GuidedPlan &plan, unsigned long long *acc, uint32_t *out, uint64_t out_cap,
                      unsigned long long *counter, cudaStream_t st) {
  if (g->nnz == 0) return GPM_OK;
  int per_sm = 0;
  GPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, guided_kernel, kGuidedThreads, 0));
  // at most 4 CTAs per SM: the candidate lists of a warp take 8 x (max degree) words
  const uint32_t blocks = (uint32_t)gpm_num_sms(g->device) * (uint32_t)std::min(std::max(per_sm, 1), 4);
  const uint64_t warps = (uint64_t)blocks * kGuidedWarps;
  const uint64_t cap = (uint64_t)g->max_degree + 32;
  const size_t need = sizeof(uint32_t) * warps * cap * 8;
  if (g->guided_scratch_bytes < need) {
    if (g->guided_scratch) {
      cudaFree(g->guided_scratch);
      g->device_bytes -= g->guided_scratch_bytes;
      g->guided_scratch = nullptr;
      g->guided_scratch_bytes = 0;
    }
    GPM_TRY(gpm_graph_alloc(g, (void **)&g->guided_scratch, need));
    g->guided_scratch_bytes = need;
  }
  unsigned long long *queue = reinterpret_cast<unsigned long long *>(g->work + WK_MISC) + 5;
  GPM_CUDA(cudaMemsetAsync(queue, 0, sizeof(unsigned long long), st));
  GuidedArgs a{};
  a.rowptr = g->rowptr;
  a.col = g->col;
  a.deg = g->deg;
  a.n = g->n;
  a.nnz = g->nnz;
  a.plan = plan;
  a.queue = queue;
  a.scratch = g->guided_scratch;
  a.cap = cap;
  a.acc = acc;
  a.out = out;
  a.out_cap = out_cap;
  a.counter = counter;
  a.status = reinterpret_cast<unsigned int *>(g->work + WK_STATUS);
  GPM_LAUNCH("guided_kernel", st, guided_kernel<<<blocks, kGuidedThreads, 0, st>>>(a));
  GPM_CUDA(cudaGetLastError());
  return GPM_OK;
}
