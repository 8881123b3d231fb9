// Motif counting by local counting, and 4-cycle counting.
//
// Local counting (Section 5 "Local Counting", Eq. 1 and the 3-MC / 4-MC
// local-count listings of the appendix): the non-induced (edge-induced)
// counts of the connected 4-vertex patterns follow from per-vertex degrees
// and per-edge triangle counts t_e, except the 4-cycle and the 4-clique,
// which are enumerated (as the paper's 4-MC code does):
//   3-star          N_S  = sum_v C(d_v, 3)
//   4-path          N_P  = sum_{uv} (d_u - 1)(d_v - 1) - 3T
//   tailed triangle N_TT = sum_v t_v (d_v - 2) = 1/2 sum_{uv} t_uv (d_u + d_v - 4)
//   diamond         N_D  = sum_{uv} C(t_uv, 2)   (the diamond example of Section 5)
//   4-cycle         N_C4 (enumerated below)
//   4-clique        N_K4 (clique pass)
// The induced counts then follow by inverting the unitriangular relation
// N_X = sum_Y (copies of X spanning Y) I_Y, densest pattern first.
// For 3 vertices: induced triangle = T, induced (open) wedge = sum_v C(d_v,2) - 3T.
//
// 4-cycles: a cycle is rooted at its order-last vertex v0 (order = degree,
// then id). All wedges v0 - x - w with x and w before v0 in the order are
// tallied by their far end w; a cycle rooted at v0 with opposite vertex w is a
// pair of such wedges, so the count is sum_w C(tally(w), 2). Roots are split
// by their wedge bound B(v0) = sum of d_x over x before v0:
//   small  (B <= 512): one warp, shared-memory hash table;
//   bucketed (B <= 2M): one CTA, wedge ends scattered into hash buckets in a
//           global buffer, each bucket aggregated in shared memory;
//   hub    (larger): all CTAs of the GPU on a few roots at a time, each root
//           with a dense tally of n words that stays in L2. A tally increment
//           that returns c adds c to the count (the pairs it closes), so
//           sum_w C(tally(w), 2) is formed without a second pass; the touched
//           entries are listed and reset by the next launch.
// The wedge walks read the neighbour's degree from a per-entry copy (edeg)
// beside col instead of gathering deg[w].
#include <algorithm>
#include <vector>

#include "gpm_internal.h"
#include "motif_device.cuh"

namespace {

using gpm_dev::precedes;
using gpm_dev::warp_sum;

// ---------------------------------------------------------------------------
// per-arc / per-vertex local-count terms
// ---------------------------------------------------------------------------
template <bool USE_T>
__global__ void edge_terms_kernel(const uint64_t *__restrict__ drow, const uint32_t *__restrict__ dcol,
                                  const uint32_t *__restrict__ deg, uint32_t *__restrict__ t_edge, uint32_t n,
                                  uint32_t root_lo, uint32_t root_hi, unsigned long long *__restrict__ acc,
                                  unsigned int *__restrict__ status) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  gpm_dev::EdgeTerms s;
  for (uint64_t u = warp; u < n; u += nwarps)
    gpm_dev::edge_terms_vertex<USE_T, false>(drow, dcol, deg, t_edge, u, u >= root_lo && u < root_hi, s);
  bool cD = s.ovf, cP = s.ovf, cS = s.ovf, cW = s.ovf, cTT = s.ovf, cT3 = s.ovf;
  s.D = warp_sum_checked(s.D, cD);
  s.P = warp_sum_checked(s.P, cP);
  s.S = warp_sum_checked(s.S, cS);
  s.W = warp_sum_checked(s.W, cW);
  s.TT = warp_sum_checked(s.TT, cTT);
  s.T3 = warp_sum_checked(s.T3, cT3);
  if (lane == 0) {
    acc_add_checked(&acc[ACC_P], s.P, cP, status, ACC_P);
    acc_add_checked(&acc[ACC_S], s.S, cS, status, ACC_S);
    acc_add_checked(&acc[ACC_W], s.W, cW, status, ACC_W);
    if (USE_T) {
      acc_add_checked(&acc[ACC_D], s.D, cD, status, ACC_D);
      acc_add_checked(&acc[ACC_TT2], s.TT, cTT, status, ACC_TT2);
      acc_add_checked(&acc[ACC_T3], s.T3, cT3, status, ACC_T3);
    }
  }
}

// ---------------------------------------------------------------------------
// 4-cycles
// ---------------------------------------------------------------------------
constexpr uint32_t kSmallBound = gpm_dev::kC4SmallBound;
constexpr uint32_t kHashSlots = gpm_dev::kC4HashSlots;

// wedge bound B(v0) = sum of d_x over neighbours x before v0; class 0 small
// (warp hash), 1 bucketed, 2 hub
__global__ void c4_bound_kernel(const uint64_t *__restrict__ rowptr, const uint32_t *__restrict__ col,
                                const uint32_t *__restrict__ deg, const uint32_t *__restrict__ edeg, uint32_t n,
                                uint32_t hub_bound, uint32_t *__restrict__ counts, uint32_t *__restrict__ tasks,
                                uint32_t *__restrict__ cursors, int fill, uint32_t *__restrict__ bvals = nullptr) {
  // a warp takes 32 consecutive vertices: lane k sums the list of vertex k
  // on its own when it has at most kBoundLane entries (four loads in flight),
  // and the warp then walks the longer lists one at a time (lanes over the
  // neighbours); lane k keeps vertex k's class, and the 32 outcomes are
  // counted / placed with one atomic per class
  constexpr uint32_t kBoundLane = 64;
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t g0 = warp * 32; g0 < n; g0 += nwarps * 32) {
    int my_c = -1;
    uint32_t my_b = 0;
    const uint64_t vl = g0 + lane;
    const bool on = vl < n;
    const uint32_t dl = on ? deg[vl] : 0u;
    unsigned long long bl = 0;
    if (on && dl <= kBoundLane) {
      const uint64_t rb = rowptr[vl];
      uint32_t i = 0;
      for (; i + 4 <= dl; i += 4) {
        const uint32_t x0 = col[rb + i], x1 = col[rb + i + 1], x2 = col[rb + i + 2], x3 = col[rb + i + 3];
        const uint32_t d0 = edeg[rb + i], d1 = edeg[rb + i + 1], d2 = edeg[rb + i + 2], d3 = edeg[rb + i + 3];
        if (precedes(d0, x0, dl, (uint32_t)vl)) bl += d0;
        if (precedes(d1, x1, dl, (uint32_t)vl)) bl += d1;
        if (precedes(d2, x2, dl, (uint32_t)vl)) bl += d2;
        if (precedes(d3, x3, dl, (uint32_t)vl)) bl += d3;
      }
      for (; i < dl; ++i) {
        const uint32_t x = col[rb + i], dx = edeg[rb + i];
        if (precedes(dx, x, dl, (uint32_t)vl)) bl += dx;
      }
    }
    uint32_t longm = __ballot_sync(0xffffffffu, on && dl > kBoundLane);
    while (longm) {
      const uint32_t k = __ffs(longm) - 1;
      longm &= longm - 1;
      const uint64_t v = g0 + k;
      const uint32_t dv = __shfl_sync(0xffffffffu, dl, k);
      unsigned long long b = 0;
      for (uint64_t e = rowptr[v] + lane; e < rowptr[v + 1]; e += 32) {
        const uint32_t x = col[e];
        const uint32_t dx = edeg[e];
        if (precedes(dx, x, dv, (uint32_t)v)) b += dx;
      }
      b = __shfl_sync(0xffffffffu, warp_sum(b), 0);
      if (lane == k) bl = b;
    }
    if (on && bl >= 3) {  // a cycle needs two wedges, each scanning v0 itself plus w
      my_c = (bl <= kSmallBound) ? 0 : (bl <= hub_bound ? 1 : 2);
      my_b = (uint32_t)(bl > 0xffffffffull ? 0xffffffffull : bl);
    }
    for (int c = 0; c < 3; ++c) {
      const uint32_t m = __ballot_sync(0xffffffffu, my_c == c);
      if (!m) continue;
      if (fill) {
        const int leader = __ffs(m) - 1;
        uint32_t pos = 0;
        if ((int)lane == leader) pos = atomicAdd(&cursors[c], (uint32_t)__popc(m));
        pos = __shfl_sync(0xffffffffu, pos, leader);
        if (my_c == c) {
          const uint32_t at = pos + __popc(m & ((1u << lane) - 1u));
          tasks[at] = (uint32_t)(g0 + lane);
          if (c >= 1 && bvals) bvals[at] = my_b;
        }
      } else {
        const uint32_t mb = __reduce_max_sync(0xffffffffu, my_c == 1 ? my_b : 0u);
        if (lane == 0) {
          atomicAdd(&counts[c], (uint32_t)__popc(m));
          if (c == 1) atomicMax(&counts[3], mb);
        }
      }
    }
  }
}

// edeg[e] = deg[col[e]]
__global__ void c4_edeg_kernel(const uint32_t *__restrict__ col, const uint32_t *__restrict__ deg, uint64_t nnz,
                               uint32_t *__restrict__ edeg) {
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < nnz; e += nth) edeg[e] = deg[col[e]];
}

struct C4Args {
  const uint64_t *__restrict__ rowptr;
  const uint32_t *__restrict__ col;
  const uint32_t *__restrict__ deg;
  const uint32_t *__restrict__ edeg;
  const uint32_t *__restrict__ tasks;
  uint32_t ntasks;
  uint32_t root_lo, root_hi;
  unsigned int *queue;
  unsigned long long *acc;
  unsigned int *status;
  uint32_t *pool;  // bucketed class: per-CTA bucket buffers
  const uint32_t *bvals;  // wedge bound of every task (plain path), or null
  uint32_t n;
};

// one warp per root, shared-memory hash table
__global__ void __launch_bounds__(256) c4_small_kernel(C4Args a) {
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t *keys = smem + (size_t)wid * 2 * kHashSlots;
  uint32_t *cnt = keys + kHashSlots;
  unsigned long long acc = 0;
  bool overflow = false;
  // roots are claimed 8 at a time: most roots of this class are a few
  // microseconds of work, and one atomic per root on a single counter would
  // serialise the warps
  constexpr uint32_t kClaim = 8;
  for (;;) {
    uint32_t first = 0;
    if (lane == 0) first = atomicAdd(a.queue, kClaim);
    first = __shfl_sync(0xffffffffu, first, 0);
    if (first >= a.ntasks) break;
    const uint32_t last = first + kClaim < a.ntasks ? first + kClaim : a.ntasks;
    for (uint32_t task = first; task < last; ++task) {
      const uint32_t v0 = a.tasks[task];
      if (v0 < a.root_lo || v0 >= a.root_hi) continue;
      acc += gpm_dev::c4_root_warp(a.rowptr, a.col, a.deg, a.edeg, v0, keys, cnt, overflow);
    }
  }
  bool carry = false;
  acc = warp_sum_checked(acc, carry);
  if (lane == 0) acc_add_checked(&a.acc[ACC_C4], acc, carry, a.status, ACC_C4);
  if (__any_sync(0xffffffffu, overflow) && lane == 0) atomicOr(a.status, ST_CAPACITY);
}

// ---------------------------------------------------------------------------
// hub roots: the whole grid on up to kHubMaxR roots per launch
// ---------------------------------------------------------------------------
constexpr uint32_t kHubChunk = gpm_dev::kC4HubChunk;  // adjacency entries of x per work unit
constexpr int kHubMaxR = 4;
constexpr int kHubThreads = 256;

// count pass (units == nullptr): info[3j] = work units of hub root j (one per
// kHubChunk entries of every x before v0), info[3j+1] = deg(v0), info[3j+2] =
// wedge bound. Fill pass: units[uoff[j] ..] = {x, chunk}, x in adjacency
// order. One warp per root.
__global__ void c4_hub_units_kernel(const uint64_t *__restrict__ rowptr, const uint32_t *__restrict__ col,
                                    const uint32_t *__restrict__ deg, const uint32_t *__restrict__ edeg,
                                    const uint32_t *__restrict__ roots, uint32_t nroots,
                                    unsigned long long *__restrict__ info, const unsigned long long *__restrict__ uoff,
                                    uint32_t *__restrict__ units) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t j = warp; j < nroots; j += nwarps) {
    const uint32_t v0 = roots[j], d0 = deg[v0];
    const uint64_t b0 = rowptr[v0], e0 = rowptr[v0 + 1];
    unsigned long long run = units ? uoff[j] : 0ull, bound = 0;
    for (uint64_t cb = b0; cb < e0; cb += 32) {
      const uint64_t e = cb + lane;
      uint32_t x = 0, k = 0;
      if (e < e0) {
        x = col[e];
        const uint32_t dx = edeg[e];
        if (precedes(dx, x, d0, v0)) {
          k = (dx + kHubChunk - 1) / kHubChunk;
          bound += dx;
        }
      }
      uint32_t incl = k;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += y;
      }
      if (units)
        for (uint32_t c = 0; c < k; ++c) {
          const unsigned long long u = run + incl - k + c;
          units[2 * u] = x;
          units[2 * u + 1] = c;
        }
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    bound = warp_sum(bound);
    if (!units && lane == 0) {
      info[3 * j] = run;
      info[3 * j + 1] = d0;
      info[3 * j + 2] = bound;
    }
  }
}

// A root's tally is "dense" when n is small against its wedge bound: its
// wedges are counted with fire-and-forget increments and the next launch sums
// C(c,2) over the whole tally while clearing it. Otherwise ("sparse") every
// increment returns the old value c, which is added to the count (the pairs
// the new wedge closes), and first touches are listed for the reset.
struct HubGroup {
  uint32_t nr, prev_nr;
  uint32_t dense, prev_dense;            // bit r: root r is dense
  uint32_t v0[kHubMaxR], d0[kHubMaxR];
  unsigned long long ub[kHubMaxR];       // first unit of root r
  unsigned long long cum[kHubMaxR + 1];  // flattened unit index where root r starts
  uint32_t *tally, *touched;             // nr slots of npad words each (this launch's set)
  unsigned int *ntouched;                // nr counters, zero on entry
  uint32_t *prev_tally, *prev_touched;   // previous launch's set: summed / reset here
  const unsigned int *prev_ntouched;
};

__device__ __forceinline__ unsigned long long pairs_of(uint32_t c) { return (unsigned long long)c * (c - (c > 0)) / 2; }

// ---- bulk asynchronous copies (TMA engine) into shared memory, per warp ----
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// bytes and both addresses are multiples of 16
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// shared memory read by ordinary loads is about to be overwritten by a bulk copy
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// bounded wait for the completion of phase `parity`; false if the limit was hit
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 20); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

constexpr uint32_t kHubStage = kHubChunk + 8;  // words per staged array: a unit plus 16-byte rounding

struct HubUnit {
  uint32_t r, off, n;  // group root, first entry within the staged range, entries
  uint64_t a0;         // first staged word (16-byte aligned)
  uint32_t words;      // staged words (multiple of 4)
};

__device__ __forceinline__ HubUnit hub_unit(const uint64_t *__restrict__ rowptr, const uint2 *__restrict__ units,
                                            const HubGroup &grp, unsigned long long f) {
  HubUnit h;
  h.r = 0;
  while (h.r + 1 < grp.nr && f >= grp.cum[h.r + 1]) ++h.r;
  const uint2 unit = units[grp.ub[h.r] + (f - grp.cum[h.r])];
  const uint64_t e0 = rowptr[unit.x] + (uint64_t)unit.y * kHubChunk;
  const uint64_t e1 = min(rowptr[unit.x + 1], e0 + kHubChunk);
  h.a0 = e0 & ~3ull;
  h.off = (uint32_t)(e0 - h.a0);
  h.n = (uint32_t)(e1 - e0);
  h.words = (uint32_t)(((e1 + 3) & ~3ull) - h.a0);
  return h;
}

// Finishes the previous group's tallies, then tallies the wedges of this
// group's roots. Each warp takes whole units (x, chunk) and stages each unit's
// col and edeg ranges in shared memory with bulk asynchronous copies, two
// units in flight per warp (the next one is copied while the current one is
// tallied). Waits are bounded: on a timeout the warp records ST_TIMEOUT,
// waits (bounded) for its copies still in flight and stops.
__global__ void __launch_bounds__(kHubThreads) c4_hub_kernel(const uint64_t *__restrict__ rowptr,
                                                             const uint32_t *__restrict__ col,
                                                             const uint32_t *__restrict__ edeg,
                                                             const uint2 *__restrict__ units, uint64_t npad,
                                                             HubGroup grp, unsigned long long *__restrict__ acc_out,
                                                             unsigned int *__restrict__ status) {
  constexpr uint32_t kW = kHubThreads / 32;
  __shared__ unsigned long long s_acc[kW];
  __shared__ __align__(16) uint32_t s_stage[kW][2][2][kHubStage];  // [warp][buffer][col, edeg][words]
  __shared__ __align__(8) uint64_t s_bar[kW][2];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint64_t gtid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  unsigned long long acc = 0;
  for (uint32_t r = 0; r < grp.prev_nr; ++r) {
    uint32_t *T = grp.prev_tally + (size_t)r * npad;
    if ((grp.prev_dense >> r) & 1u) {
      uint4 *T4 = reinterpret_cast<uint4 *>(T);
      for (uint64_t i = gtid; i < npad / 4; i += nth) {
        const uint4 v = __ldcg(T4 + i);
        if (v.x | v.y | v.z | v.w) {
          acc += pairs_of(v.x) + pairs_of(v.y) + pairs_of(v.z) + pairs_of(v.w);
          __stcg(T4 + i, make_uint4(0u, 0u, 0u, 0u));
        }
      }
    } else {
      const uint32_t cnt = grp.prev_ntouched[r];
      const uint32_t *L = grp.prev_touched + (size_t)r * npad;
      for (uint64_t i = gtid; i < cnt; i += nth) T[__ldcg(L + i)] = 0u;
    }
  }
  if (lane == 0) {
    mbar_init(&s_bar[wid][0], 1);
    mbar_init(&s_bar[wid][1], 1);
    mbar_fence_init();
  }
  __syncwarp();
  const unsigned long long total = grp.cum[grp.nr];
  const unsigned long long stride = nth >> 5;
  auto issue = [&](const HubUnit &h, uint32_t b) {
    if (lane == 0) {
      fence_proxy_async();
      mbar_expect_tx(&s_bar[wid][b], 8u * h.words);
      bulk_copy_g2s(s_stage[wid][b][0], col + h.a0, 4u * h.words, &s_bar[wid][b]);
      bulk_copy_g2s(s_stage[wid][b][1], edeg + h.a0, 4u * h.words, &s_bar[wid][b]);
    }
  };
  uint32_t phase = 0u, pending = 0u;  // bit b: parity to wait for / a copy in flight, buffer b
  unsigned long long f = gtid >> 5;
  HubUnit cur{};
  if (f < total) {
    cur = hub_unit(rowptr, units, grp, f);
    issue(cur, 0);
    pending |= 1u;
  }
  bool timed_out = false;
  for (uint32_t k = 0; f < total; ++k, f += stride) {
    const uint32_t b = k & 1u;
    HubUnit nxt{};
    if (f + stride < total) {
      nxt = hub_unit(rowptr, units, grp, f + stride);
      issue(nxt, b ^ 1u);
      pending |= 2u >> b;
    }
    if (!mbar_wait(&s_bar[wid][b], (phase >> b) & 1u)) {
      timed_out = true;
      break;
    }
    phase ^= 1u << b;
    pending &= ~(1u << b);
    const uint32_t *sc = s_stage[wid][b][0] + cur.off;
    const uint32_t *sd = s_stage[wid][b][1] + cur.off;
    const uint32_t v0 = grp.v0[cur.r], d0 = grp.d0[cur.r];
    uint32_t *tally = grp.tally + (size_t)cur.r * npad;
    if ((grp.dense >> cur.r) & 1u) {
      for (uint32_t i = lane; i < cur.n; i += 32) {
        const uint32_t w = sc[i];
        if (precedes(sd[i], w, d0, v0)) atomicAdd(&tally[w], 1u);
      }
    } else {
      uint32_t *touched = grp.touched + (size_t)cur.r * npad;
      for (uint32_t base = 0; base < cur.n; base += 32) {
        const uint32_t i = base + lane;
        const uint32_t w = (i < cur.n) ? sc[i] : 0u;
        const bool v = (i < cur.n) && precedes(sd[i], w, d0, v0);
        const uint32_t old = v ? atomicAdd(&tally[w], 1u) : 1u;
        acc += v ? old : 0u;
        const bool first = v && old == 0u;
        const uint32_t m = __ballot_sync(0xffffffffu, first);
        if (m) {
          const int leader = __ffs(m) - 1;
          uint32_t pos = 0;
          if ((int)lane == leader) pos = atomicAdd(&grp.ntouched[cur.r], (uint32_t)__popc(m));
          pos = __shfl_sync(0xffffffffu, pos, leader);
          if (first) touched[pos + __popc(m & ((1u << lane) - 1u))] = w;
        }
      }
    }
    __syncwarp();  // every lane is done with buffer b before it is refilled
    cur = nxt;
  }
  if (timed_out) {
    if (lane == 0) atomicOr(status, ST_TIMEOUT);
    for (uint32_t b = 0; b < 2; ++b)
      if ((pending >> b) & 1u) mbar_wait(&s_bar[wid][b], (phase >> b) & 1u);
  }
  bool wcarry = false;
  acc = warp_sum_checked(acc, wcarry);
  if (wcarry && lane == 0) atomicOr(status + 1, 1u << ACC_C4);
  if (lane == 0) s_acc[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    bool carry = false;
    for (uint32_t i = 0; i < kW; ++i) {
      carry |= (t + s_acc[i] < t);
      t += s_acc[i];
    }
    acc_add_checked(&acc_out[ACC_C4], t, carry, status, ACC_C4);
  }
}

// one CTA per large root, bucketed aggregation (buffer slot per CTA) with
// tables of kC4PlainTable slots per warp, so that three CTAs fit an SM
// (roots above c4_bucket_narrow_bound<kC4PlainTable>() take wider tables in
// half of the warps); roots whose wedge bound is at most 3/4 of
// kC4DirectSlots are counted in one shared-memory table instead (the whole
// dynamic shared memory)
constexpr int kC4BucketThreads = 512;
constexpr uint32_t kC4PlainTable = 256;
constexpr uint32_t kC4DirectSlots = 1u << (31 - __builtin_clz(gpm_dev::c4_bucket_smem_words<kC4PlainTable>(
                                                              kC4BucketThreads / 32) / 2));
static_assert((kC4DirectSlots & (kC4DirectSlots - 1)) == 0, "direct table slots: a power of two");
__global__ void __launch_bounds__(kC4BucketThreads) c4_bucket_kernel(C4Args a, uint64_t slot_words) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_task, s_cnt;
  __shared__ uint32_t s_x[kC4BucketThreads];
  __shared__ uint32_t s_pre[kC4BucketThreads + 33];
  __shared__ uint64_t s_rp[kC4BucketThreads];
  uint32_t *buf = a.pool + (size_t)blockIdx.x * slot_words;
  unsigned long long acc = 0;
  bool overflow = false;
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(a.queue, 1u);
    __syncthreads();
    const uint32_t task = s_task;
    __syncthreads();
    if (task >= a.ntasks) break;
    const uint32_t v0 = a.tasks[task];
    if (v0 < a.root_lo || v0 >= a.root_hi) continue;
    acc += gpm_dev::c4_root_bucketed<kC4PlainTable>(a.rowptr, a.col, a.deg, a.edeg, v0, buf, buf + slot_words / 2,
                                                    smem, s_x, &s_cnt, overflow, s_pre, s_rp, kC4DirectSlots,
                                                    a.bvals ? a.bvals[task] : 0u);
  }
  bool carry = false;
  acc = warp_sum_checked(acc, carry);
  if ((threadIdx.x & 31) == 0) acc_add_checked(&a.acc[ACC_C4], acc, carry, a.status, ACC_C4);
  if (__syncthreads_or(overflow) && threadIdx.x == 0) atomicOr(a.status, ST_CAPACITY);
}

// ---------------------------------------------------------------------------
// large roots, plain count path: range-partitioned tallies in shared memory.
// The wedge ends w of a root lie in [0, n); the id space is cut into ranges of
// `width` ids, and a CTA takes the ranges of a root one after the other,
// keeping a dense tally of the current range in shared memory (16-bit
// counters, two per word: a count is at most the root's degree, < 65536).
// For range r the wedges with an end in it are the segments of the lists
// N(x), x before v0, between the precomputed offsets roff[x][r] and
// roff[x][r+1] (lists are sorted by id), so every wedge is read once and
// counted once in shared memory; C(c,2) is summed over the range's tally while
// it is cleared for the next range.
// ---------------------------------------------------------------------------
constexpr int kRangeThreads = 1024;
constexpr uint32_t kRangeMaxWidth = 98304;
constexpr uint32_t kRangeTallyWords = kRangeMaxWidth / 2;  // 192 KB, a multiple of 4 words
constexpr int kRangeRun = 4;  // wedge ends per lane in flight in the walk
// dynamic shared memory: tally, segment prefix (threads + 1), warp sums (32),
// segment starts (threads)
constexpr size_t kRangeSmemBytes = 4ull * (kRangeTallyWords + kRangeThreads + 1 + 32 + kRangeThreads);

// roff[x * nr1 + r] = rowptr[x] + (number of entries of N(x) with id < r *
// width), for r = 0 .. nr1 - 1 (absolute positions in col; the last one is
// rowptr[x + 1]). One warp per vertex; entry p writes the offsets of the
// ranges that begin after its predecessor and at or before it, so every
// offset is written once.
__global__ void c4_roff_kernel(const uint64_t *__restrict__ rowptr, const uint32_t *__restrict__ col, uint32_t n,
                               uint32_t width, uint32_t nr1, uint32_t *__restrict__ roff) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t x = warp; x < n; x += nwarps) {
    const uint64_t b = rowptr[x];
    const uint32_t d = (uint32_t)(rowptr[x + 1] - b);
    uint32_t *row = roff + x * nr1;
    for (uint32_t p = lane; p <= d; p += 32) {
      const uint32_t lo = (p == 0) ? 0u : col[b + p - 1] / width + 1u;
      const uint32_t hi = (p == d) ? nr1 - 1u : col[b + p] / width;
      for (uint32_t r = lo; r <= hi; ++r) row[r] = (uint32_t)(b + p);
    }
  }
}

struct C4RangeArgs {
  const uint64_t *__restrict__ rowptr;
  const uint32_t *__restrict__ col;
  const uint32_t *__restrict__ deg;
  const uint32_t *__restrict__ edeg;
  const uint32_t *__restrict__ roff;  // absolute positions in col
  uint32_t nr1, width;
  const uint4 *__restrict__ items;  // {v0, first range, end range, 0}
  uint32_t nitems;
  uint32_t root_lo, root_hi;
  unsigned int *queue;
  unsigned long long *acc;
  unsigned int *status;
};

// C(a,2) + C(b,2) for the two 16-bit counters of a tally word
__device__ __forceinline__ unsigned long long pairs16(uint32_t v) {
  const unsigned long long a = v & 0xffffu, b = v >> 16;
  return (a * (a - (a > 0)) + b * (b - (b > 0))) >> 1;
}

__global__ void __launch_bounds__(kRangeThreads, 1) c4_range_kernel(C4RangeArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t *T = smem;
  uint32_t *s_pre = T + kRangeTallyWords;        // kRangeThreads + 1
  uint32_t *s_wsum = s_pre + kRangeThreads + 1;  // 32
  uint32_t *s_base = s_wsum + 32;                // kRangeThreads
  __shared__ uint4 s_item;
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  uint4 *T4 = reinterpret_cast<uint4 *>(T);
  for (uint32_t i = tid; i < kRangeTallyWords / 4; i += kRangeThreads) T4[i] = make_uint4(0u, 0u, 0u, 0u);
  const uint32_t tw4 = (a.width / 2 + 3) / 4;  // uint4 words of one range's tally
  unsigned long long acc = 0;
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      const uint32_t it = atomicAdd(a.queue, 1u);
      s_item = it < a.nitems ? a.items[it] : make_uint4(0xffffffffu, 0u, 0u, 0u);
    }
    __syncthreads();
    const uint4 item = s_item;
    if (item.x == 0xffffffffu) break;
    const uint32_t v0 = item.x;
    if (v0 < a.root_lo || v0 >= a.root_hi) continue;
    const uint32_t d0 = a.deg[v0];
    const uint64_t b0 = a.rowptr[v0], e0 = a.rowptr[v0 + 1];
    for (uint32_t r = item.y; r < item.z; ++r) {
      const uint32_t wbase = r * a.width;
      for (uint64_t cb = b0; cb < e0; cb += kRangeThreads) {
        // segment of N(x) in range r for this thread's x (length 0 unless x precedes v0)
        const uint64_t e = cb + tid;
        uint32_t len = 0, start = 0;
        if (e < e0) {
          const uint32_t x = a.col[e];
          if (precedes(a.edeg[e], x, d0, v0)) {
            const uint32_t *ro = a.roff + (uint64_t)x * a.nr1 + r;
            const uint32_t o0 = ro[0];
            len = ro[1] - o0;
            start = o0;
          }
        }
        const uint32_t cnt = (e0 - cb < (uint64_t)kRangeThreads) ? (uint32_t)(e0 - cb) : (uint32_t)kRangeThreads;
        uint32_t incl = len;
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= (uint32_t)o) incl += y;
        }
        if (lane == 31) s_wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
          const uint32_t v = s_wsum[lane];
          uint32_t wi = v;
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= (uint32_t)o) wi += y;
          }
          s_wsum[lane] = wi - v;
        }
        __syncthreads();
        const uint32_t excl = incl - len + s_wsum[wid];
        s_pre[tid] = excl;
        if (tid == kRangeThreads - 1) s_pre[kRangeThreads] = excl + len;
        s_base[tid] = start;
        __syncthreads();
        const uint32_t total = s_pre[cnt];
        // blocks of kRangeRun * 32 wedge ends per warp, 32 consecutive ends per
        // load (coalesced); the segment of an end is searched among the rows
        // that the block's first and last ends fall in
        for (uint32_t blk = wid * (32u * kRangeRun); blk < total; blk += kRangeThreads * kRangeRun) {
          const uint32_t flast = min(blk + 32u * kRangeRun - 1u, total - 1u);
          uint32_t ib = 0;
          if (lane < 2) ib = gpm_dev::c4_row_of(s_pre, cnt, lane ? flast : blk);
          const uint32_t ilo = __shfl_sync(0xffffffffu, ib, 0), ihi = __shfl_sync(0xffffffffu, ib, 1);
          uint32_t wv[kRangeRun];
          bool ok[kRangeRun];
#pragma unroll
          for (int q = 0; q < kRangeRun; ++q) {
            const uint32_t f = blk + 32u * q + lane;
            ok[q] = false;
            wv[q] = 0;
            if (f < total) {
              uint32_t lo = ilo, hi = ihi + 1;  // largest i in [lo, hi) with s_pre[i] <= f
              while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (s_pre[mid] <= f) lo = mid;
                else hi = mid;
              }
              const uint32_t ee = s_base[lo] + (f - s_pre[lo]);
              wv[q] = __ldg(a.col + ee);
              ok[q] = precedes(__ldg(a.edeg + ee), wv[q], d0, v0);
            }
          }
#pragma unroll
          for (int q = 0; q < kRangeRun; ++q)
            if (ok[q]) {
              const uint32_t t = wv[q] - wbase;
              atomicAdd(&T[t >> 1], 1u << ((t & 1u) << 4));
            }
        }
        __syncthreads();
      }
      // C(c,2) over the range's tally, clearing it for the next range
      for (uint32_t i = tid; i < tw4; i += kRangeThreads) {
        const uint4 v = T4[i];
        if (v.x | v.y | v.z | v.w) {
          acc += pairs16(v.x) + pairs16(v.y) + pairs16(v.z) + pairs16(v.w);
          T4[i] = make_uint4(0u, 0u, 0u, 0u);
        }
      }
      __syncthreads();
    }
  }
  bool carry = false;
  acc = warp_sum_checked(acc, carry);
  if (lane == 0) acc_add_checked(&a.acc[ACC_C4], acc, carry, a.status, ACC_C4);
}

// ---------------------------------------------------------------------------
// finalize: requested counts from the accumulators (one thread)
// ---------------------------------------------------------------------------
// accumulator slots a formula reads (their 64-bit overflow makes its count invalid)
__device__ __forceinline__ uint32_t formula_slots(uint32_t f) {
  const uint32_t inv = (1u << ACC_T) | (1u << ACC_K4) | (1u << ACC_D) | (1u << ACC_P) | (1u << ACC_S) |
                       (1u << ACC_TT2) | (1u << ACC_C4);  // the 4-motif inversion reads all six terms
  switch (f) {
    case F_TRI: return 1u << ACC_T;
    case F_K4: return 1u << ACC_K4;
    case F_K5: return 1u << ACC_K5;
    case F_K6: return 1u << ACC_K6;
    case F_K7: return 1u << 0;
    case F_K8: return 1u << 1;
    case F_K9: return 1u << 2;
    case F_WEDGE_NI: return 1u << ACC_W;
    case F_WEDGE_I: return (1u << ACC_W) | (1u << ACC_T);
    case F_STAR_NI: return 1u << ACC_S;
    case F_PATH_NI: return (1u << ACC_P) | (1u << ACC_T);
    case F_TT_NI: return 1u << ACC_TT2;
    case F_C4_NI: return 1u << ACC_C4;
    case F_D_NI: return 1u << ACC_D;
    case F_STAR_I: case F_PATH_I: case F_TT_I: case F_C4_I: case F_D_I: case F_K4_I: return inv;
    default: return 0u;
  }
}

__global__ void finalize_kernel(FinalizeSpec spec, const unsigned long long *__restrict__ acc, uint64_t n, uint64_t m,
                                unsigned long long *__restrict__ out, unsigned int *__restrict__ status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  bool bad = false;
  const uint32_t over = status[1];
  for (uint32_t i = 0; i < spec.npat; ++i) {
    out[i] = gpm_dev::finalize_formula(spec.formula[i], acc, n, m, bad);
    bad |= (formula_slots(spec.formula[i]) & over) != 0;
  }
  if (bad) atomicOr(status, ST_CAPACITY);
}

}  // namespace

int gpm_launch_edge_terms(gpm_graph *g, bool use_t_edge, uint32_t root_lo, uint32_t root_hi,
                          unsigned long long *acc, cudaStream_t st) {
  const int blocks = gpm_num_sms(g->device) * 8;
  if (g->n == 0) return GPM_OK;
  unsigned int *status = reinterpret_cast<unsigned int *>(g->work + WK_STATUS);
  if (use_t_edge)
    GPM_LAUNCH("edge_terms_kernel", st, edge_terms_kernel<true><<<blocks, 256, 0, st>>>(g->drow, g->dcol, g->deg, g->t_edge, g->n, root_lo, root_hi, acc, status));
  else
    GPM_LAUNCH("edge_terms_kernel", st, edge_terms_kernel<false><<<blocks, 256, 0, st>>>(g->drow, g->dcol, g->deg, nullptr, g->n, root_lo, root_hi, acc, status));
  GPM_CUDA(cudaGetLastError());
  return GPM_OK;
}

// a hub root's tally is summed densely when n <= 4 x its wedge bound
static inline bool hub_dense(uint32_t n, uint64_t bound) { return (uint64_t)n <= 4ull * bound; }

// edeg[e] = deg(col[e]), built once per graph
static int ensure_edeg(gpm_graph *g, cudaStream_t st) {
  if (g->edeg) return GPM_OK;
  const int blocks = gpm_num_sms(g->device) * 8;
  GPM_TRY(gpm_graph_alloc(g, (void **)&g->edeg, sizeof(uint32_t) * (std::max<uint64_t>(g->nnz, 1) + kCsrPadWords)));
  if (g->nnz) {
    GPM_LAUNCH("c4_edeg_kernel", st, c4_edeg_kernel<<<blocks, 256, 0, st>>>(g->col, g->deg, g->nnz, g->edeg));
    GPM_CUDA(cudaGetLastError());
  }
  return GPM_OK;
}

static int ensure_c4_tasks(gpm_graph *g, cudaStream_t st) {
  const uint32_t hub_bound = std::min(gpm_tune().c4_hub_bound, gpm_dev::kC4BucketMaxBound);
  if (g->c4_ready && g->c4_hub_bound == hub_bound) return GPM_OK;
  if (!g->c4_tasks) GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4_tasks, sizeof(uint32_t) * std::max<uint32_t>(g->n, 1)));
  const int blocks = gpm_num_sms(g->device) * 8;
  GPM_TRY(ensure_edeg(g, st));
  uint32_t *tmp = reinterpret_cast<uint32_t *>(g->work + WK_MISC);  // counts[3], max bound, cursors[3]
  GPM_CUDA(cudaMemsetAsync(tmp, 0, 8 * sizeof(uint32_t), st));
  if (g->n) {
    GPM_LAUNCH("c4_bound_kernel", st,
               c4_bound_kernel<<<blocks, 256, 0, st>>>(g->rowptr, g->col, g->deg, g->edeg, g->n, hub_bound, tmp,
                                                        nullptr, nullptr, 0));
    GPM_CUDA(cudaGetLastError());
  }
  uint32_t h[4];
  GPM_CUDA(cudaMemcpyAsync(h, tmp, sizeof(h), cudaMemcpyDeviceToHost, st));
  GPM_CUDA(cudaStreamSynchronize(st));
  g->c4_begin[0] = 0;
  g->c4_begin[1] = h[0];
  g->c4_begin[2] = h[0] + h[1];
  g->c4_begin[3] = h[0] + h[1] + h[2];
  g->c4_bucket_maxb = h[3];
  uint32_t cur[3] = {0, h[0], h[0] + h[1]};
  GPM_CUDA(cudaMemcpyAsync(tmp + 4, cur, sizeof(cur), cudaMemcpyHostToDevice, st));
  if (g->n) {
    GPM_LAUNCH("c4_bound_kernel", st,
               c4_bound_kernel<<<blocks, 256, 0, st>>>(g->rowptr, g->col, g->deg, g->edeg, g->n, hub_bound,
                                                        nullptr, g->c4_tasks, tmp + 4, 1));
    GPM_CUDA(cudaGetLastError());
  }
  GPM_CUDA(cudaStreamSynchronize(st));
  g->c4_ready = true;
  g->c4_hub_bound = hub_bound;
  g->c4_hub_ready = false;
  return GPM_OK;
}

// Work units and (with tallies) tally sets of the hub roots (class 2), built
// once per task list.
static int ensure_c4_hub(gpm_graph *g, cudaStream_t st, bool tallies = true) {
  const uint32_t nhub = g->c4_begin[3] - g->c4_begin[2];
  if (g->c4_hub_ready && (!tallies || !nhub || g->c4_hub_tally)) return GPM_OK;
  const uint32_t *roots = g->c4_tasks + g->c4_begin[2];
  if (!g->c4_hub_ready) {
    if (g->c4_hub_units) {
      cudaFree(g->c4_hub_units);
      g->c4_hub_units = nullptr;
    }
    g->c4_hub_root.assign(nhub, 0);
    g->c4_hub_deg.assign(nhub, 0);
    g->c4_hub_bnd.assign(nhub, 0);
    g->c4_hub_uoff.assign((size_t)nhub + 1, 0);
  }
  if (nhub && !g->c4_hub_ready) {
    const int blocks = gpm_num_sms(g->device) * 8;
    unsigned long long *info = nullptr;
    GPM_CUDA(cudaMalloc(&info, sizeof(unsigned long long) * (3 * (size_t)nhub + (size_t)nhub + 1)));
    unsigned long long *d_uoff = info + 3 * (size_t)nhub;
    std::vector<unsigned long long> h(3 * (size_t)nhub);
    int rc = GPM_OK;
    do {
      GPM_LAUNCH("c4_hub_units_kernel", st,
                 c4_hub_units_kernel<<<blocks, 256, 0, st>>>(g->rowptr, g->col, g->deg, g->edeg, roots, nhub, info,
                                                              nullptr, nullptr));
      if (cudaGetLastError() != cudaSuccess ||
          cudaMemcpyAsync(h.data(), info, sizeof(unsigned long long) * 3 * nhub, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaMemcpyAsync(g->c4_hub_root.data(), roots, sizeof(uint32_t) * nhub, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        rc = gpm_fail(GPM_E_DEVICE, "4-cycle hub unit count failed");
        break;
      }
      for (uint32_t j = 0; j < nhub; ++j) {
        g->c4_hub_uoff[j + 1] = g->c4_hub_uoff[j] + h[3 * j];
        g->c4_hub_deg[j] = (uint32_t)h[3 * j + 1];
        g->c4_hub_bnd[j] = h[3 * j + 2];
      }
      const uint64_t U = g->c4_hub_uoff[nhub];
      rc = gpm_graph_alloc(g, (void **)&g->c4_hub_units, sizeof(uint32_t) * 2 * std::max<uint64_t>(U, 1));
      if (rc) break;
      if (cudaMemcpyAsync(d_uoff, g->c4_hub_uoff.data(), sizeof(unsigned long long) * ((size_t)nhub + 1),
                          cudaMemcpyHostToDevice, st) != cudaSuccess) {
        rc = gpm_fail(GPM_E_DEVICE, "4-cycle hub offsets upload failed");
        break;
      }
      GPM_LAUNCH("c4_hub_units_kernel", st,
                 c4_hub_units_kernel<<<blocks, 256, 0, st>>>(g->rowptr, g->col, g->deg, g->edeg, roots, nhub, nullptr,
                                                              d_uoff, g->c4_hub_units));
      if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        rc = gpm_fail(GPM_E_DEVICE, "4-cycle hub unit fill failed");
    } while (0);
    cudaFree(info);
    if (rc) return rc;
  }
  g->c4_hub_ready = true;
  if (nhub && tallies) {
    // tallies: as many roots per launch as keep one set of tallies within 32 MiB
    const uint64_t npad = ((uint64_t)std::max<uint32_t>(g->n, 1) + 3) & ~3ull;
    const uint32_t R = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(kHubMaxR, (32ull << 20) / (4ull * npad)));
    bool any_sparse = false;
    for (uint32_t j = 0; j < nhub; ++j) any_sparse |= !hub_dense(g->n, g->c4_hub_bnd[j]);
    const size_t words = 2 * (size_t)R * npad;
    if (!g->c4_hub_tally || g->c4_hub_R != R) {
      if (g->c4_hub_tally) cudaFree(g->c4_hub_tally);
      if (g->c4_hub_touched) cudaFree(g->c4_hub_touched);
      g->c4_hub_tally = g->c4_hub_touched = nullptr;
      GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4_hub_tally, sizeof(uint32_t) * words));
      GPM_CUDA(cudaMemsetAsync(g->c4_hub_tally, 0, sizeof(uint32_t) * words, st));
      g->c4_hub_R = R;
    }
    if (any_sparse && !g->c4_hub_touched)
      GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4_hub_touched, sizeof(uint32_t) * words));
    const size_t ctr_words = ((size_t)nhub + 2) * R;
    if (g->c4_hub_ctr_words < ctr_words) {
      if (g->c4_hub_ctr) cudaFree(g->c4_hub_ctr);
      g->c4_hub_ctr = nullptr;
      GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4_hub_ctr, sizeof(unsigned int) * ctr_words));
      g->c4_hub_ctr_words = ctr_words;
    }
  }
  return GPM_OK;
}

// Hub roots in [root_lo, root_hi): one launch per group of c4_hub_R roots,
// each also finishing the previous group's tallies, and a final launch that
// finishes the last group. Only enqueues work (capturable in a CUDA graph).
static int launch_c4_hub(gpm_graph *g, uint32_t root_lo, uint32_t root_hi, unsigned long long *acc, cudaStream_t st,
                         uint32_t *nlaunch) {
  std::vector<uint32_t> J;
  for (uint32_t j = 0; j < (uint32_t)g->c4_hub_root.size(); ++j)
    if (g->c4_hub_root[j] >= root_lo && g->c4_hub_root[j] < root_hi) J.push_back(j);
  if (nlaunch) *nlaunch = 0;
  if (J.empty()) return GPM_OK;
  const uint32_t R = g->c4_hub_R;
  const uint64_t npad = ((uint64_t)std::max<uint32_t>(g->n, 1) + 3) & ~3ull;
  const size_t set_words = (size_t)R * npad;
  const uint32_t ngroups = (uint32_t)((J.size() + R - 1) / R);
  GPM_CUDA(cudaMemsetAsync(g->c4_hub_ctr, 0, sizeof(unsigned int) * (size_t)(ngroups + 1) * R, st));
  int per_sm = 0;
  GPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c4_hub_kernel, kHubThreads, 0));
  const unsigned blocks = (unsigned)(gpm_num_sms(g->device) * std::max(per_sm, 1));
  const uint2 *units = reinterpret_cast<const uint2 *>(g->c4_hub_units);
  HubGroup prev{};
  for (uint32_t gi = 0; gi <= ngroups; ++gi) {
    HubGroup grp{};
    const size_t set = gi & 1u;
    grp.tally = g->c4_hub_tally + set * set_words;
    grp.touched = g->c4_hub_touched ? g->c4_hub_touched + set * set_words : nullptr;
    grp.ntouched = g->c4_hub_ctr + (size_t)gi * R;
    if (gi < ngroups) {
      for (uint32_t k = gi * R; k < std::min<uint32_t>((gi + 1) * R, (uint32_t)J.size()); ++k) {
        const uint32_t j = J[k], r = grp.nr++;
        grp.v0[r] = g->c4_hub_root[j];
        grp.d0[r] = g->c4_hub_deg[j];
        grp.ub[r] = g->c4_hub_uoff[j];
        grp.cum[r + 1] = grp.cum[r] + (g->c4_hub_uoff[j + 1] - g->c4_hub_uoff[j]);
        if (hub_dense(g->n, g->c4_hub_bnd[j])) grp.dense |= 1u << r;
      }
    }
    if (gi > 0) {
      grp.prev_nr = prev.nr;
      grp.prev_dense = prev.dense;
      grp.prev_tally = prev.tally;
      grp.prev_touched = prev.touched;
      grp.prev_ntouched = prev.ntouched;
    }
    GPM_LAUNCH("c4_hub_kernel", st,
               c4_hub_kernel<<<blocks, kHubThreads, 0, st>>>(g->rowptr, g->col, g->edeg, units, npad, grp, acc,
                                                             reinterpret_cast<unsigned int *>(g->work + WK_STATUS)));
    GPM_CUDA(cudaGetLastError());
    prev = grp;
  }
  if (nlaunch) *nlaunch = ngroups + 1;
  return GPM_OK;
}

int gpm_c4_hub_prepare(gpm_graph *g, cudaStream_t st, bool tallies) {
  GPM_TRY(ensure_c4_tasks(g, st));
  return ensure_c4_hub(g, st, tallies);
}

int gpm_c4_hub_enqueue(gpm_graph *g, uint32_t root_lo, uint32_t root_hi, unsigned long long *acc, cudaStream_t st,
                       uint32_t *nlaunch) {
  if (!g->c4_ready || !g->c4_hub_ready || (!g->c4_hub_tally && !g->c4_hub_root.empty()))
    return gpm_fail(GPM_E_INVALID_ARG, "4-cycle hub roots are not prepared");
  return launch_c4_hub(g, root_lo, root_hi, acc, st, nlaunch);
}

int gpm_build_c4_tasks(gpm_graph *g, cudaStream_t st) { return ensure_c4_tasks(g, st); }


// ---------------------------------------------------------------------------
// plain count path with range tallies for the large roots
// ---------------------------------------------------------------------------
// the range tallies use 16-bit counters (a count is at most the root's
// degree) and 32-bit positions in col
static bool c4_use_range(const gpm_graph *g) {
  const gpm_tuning &t = gpm_tune();
  return (t.c4_range_bound != 0xffffffffu || t.c4_pull_bound != 0xffffffffu) && g->max_degree <= 0xffffu &&
         g->nnz < (1ull << 32);
}

// range offsets of every list for ranges of `width` ids, built once per graph and width
static int ensure_c4_roff(gpm_graph *g, uint32_t width, cudaStream_t st) {
  if (g->c4_roff && g->c4_roff_width == width) return GPM_OK;
  if (g->c4_roff) {
    cudaFree(g->c4_roff);
    g->device_bytes -= sizeof(uint32_t) * (size_t)g->c4_nr1 * std::max<uint32_t>(g->n, 1);
    g->c4_roff = nullptr;
  }
  const uint32_t nr = std::max<uint32_t>(1, (uint32_t)(((uint64_t)g->n + width - 1) / width));
  const uint32_t nr1 = nr + 1;
  GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4_roff, sizeof(uint32_t) * (size_t)nr1 * std::max<uint32_t>(g->n, 1)));
  g->c4_roff_width = width;
  g->c4_nr1 = nr1;
  if (g->n) {
    const int blocks = gpm_num_sms(g->device) * 8;
    GPM_LAUNCH("c4_roff_kernel", st,
               c4_roff_kernel<<<blocks, 256, 0, st>>>(g->rowptr, g->col, g->n, width, nr1, g->c4_roff));
    GPM_CUDA(cudaGetLastError());
  }
  return GPM_OK;
}

// Root classes of the plain path by wedge bound B: small (B <= 512),
// bucketed, range (c4_range_bound < B <= c4_pull_bound) and pull (B >
// c4_pull_bound). Range items: one per (root, range), roots in order of
// decreasing wedge bound and the ranges of a root consecutive, so that the
// items running at the same time belong to a few roots whose neighbour lists
// stay in L2 while every range of those roots is tallied. Pull roots: in
// order of decreasing wedge bound, 128 per pass.
static int ensure_c4_plain(gpm_graph *g, cudaStream_t st) {
  const uint32_t pull = std::max<uint32_t>(gpm_tune().c4_pull_bound, kSmallBound);
  // the bucketed class takes bounds up to kC4BucketMaxBound; larger roots
  // below the pull bound become range items
  const uint32_t bound = std::min<uint32_t>(
      std::min<uint32_t>(std::max<uint32_t>(gpm_tune().c4_range_bound, kSmallBound), pull), gpm_dev::kC4BucketMaxBound);
  const uint32_t width = gpm_tune().c4_range_width;
  if (g->c4p_ready && g->c4p_bound == bound && g->c4p_pull == pull && g->c4p_width == width) return GPM_OK;
  GPM_TRY(ensure_edeg(g, st));
  const size_t nw = std::max<uint32_t>(g->n, 1);
  if (!g->c4p_tasks) GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4p_tasks, sizeof(uint32_t) * nw));
  if (!g->c4p_bval) GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4p_bval, sizeof(uint32_t) * nw));
  const int blocks = gpm_num_sms(g->device) * 8;
  uint32_t *tmp = reinterpret_cast<uint32_t *>(g->work + WK_MISC);  // counts[3], max bound, cursors[3]
  GPM_CUDA(cudaMemsetAsync(tmp, 0, 8 * sizeof(uint32_t), st));
  if (g->n) {
    GPM_LAUNCH("c4_bound_kernel", st,
               c4_bound_kernel<<<blocks, 256, 0, st>>>(g->rowptr, g->col, g->deg, g->edeg, g->n, bound, tmp, nullptr,
                                                        nullptr, 0));
    GPM_CUDA(cudaGetLastError());
  }
  uint32_t h[4];
  GPM_CUDA(cudaMemcpyAsync(h, tmp, sizeof(h), cudaMemcpyDeviceToHost, st));
  GPM_CUDA(cudaStreamSynchronize(st));
  g->c4p_begin[0] = 0;
  g->c4p_begin[1] = h[0];
  g->c4p_begin[2] = h[0] + h[1];
  g->c4p_begin[3] = h[0] + h[1] + h[2];
  g->c4p_bucket_maxb = h[3];
  const uint32_t cur[3] = {0, h[0], h[0] + h[1]};
  GPM_CUDA(cudaMemcpyAsync(tmp + 4, cur, sizeof(cur), cudaMemcpyHostToDevice, st));
  if (g->n) {
    GPM_LAUNCH("c4_bound_kernel", st,
               c4_bound_kernel<<<blocks, 256, 0, st>>>(g->rowptr, g->col, g->deg, g->edeg, g->n, bound, nullptr,
                                                        g->c4p_tasks, tmp + 4, 1, g->c4p_bval));
    GPM_CUDA(cudaGetLastError());
  }
  const uint32_t nbig = h[2];
  std::vector<uint32_t> roots(nbig), bv(nbig);
  if (nbig) {
    GPM_CUDA(cudaMemcpyAsync(roots.data(), g->c4p_tasks + g->c4p_begin[2], sizeof(uint32_t) * nbig,
                             cudaMemcpyDeviceToHost, st));
    GPM_CUDA(cudaMemcpyAsync(bv.data(), g->c4p_bval + g->c4p_begin[2], sizeof(uint32_t) * nbig,
                             cudaMemcpyDeviceToHost, st));
  }
  GPM_CUDA(cudaStreamSynchronize(st));
  std::vector<uint32_t> ord(nbig);
  for (uint32_t i = 0; i < nbig; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](uint32_t x, uint32_t y) {
    return bv[x] != bv[y] ? bv[x] > bv[y] : roots[x] < roots[y];
  });
  std::vector<uint32_t> pull_roots;
  uint32_t nrange = 0;
  for (uint32_t i : ord) {
    if (bv[i] > pull) pull_roots.push_back(roots[i]);
    else ++nrange;
  }
  GPM_TRY(gpm_c4_pull_prepare(g, pull_roots, st));
  if (nrange) GPM_TRY(ensure_c4_roff(g, width, st));
  const uint32_t nr = nrange ? g->c4_nr1 - 1 : 0;
  std::vector<uint32_t> items;
  items.reserve(4 * (size_t)nrange * nr);
  for (uint32_t i : ord) {
    if (bv[i] > pull) continue;
    for (uint32_t r = 0; r < nr; ++r) {
      items.push_back(roots[i]);
      items.push_back(r);
      items.push_back(r + 1);
      items.push_back(0u);
    }
  }
  g->c4p_nitems = (uint32_t)(items.size() / 4);
  const size_t bytes = sizeof(uint32_t) * std::max<size_t>(items.size(), 4);
  if (g->c4p_items_cap < bytes) {
    if (g->c4p_items) {
      cudaFree(g->c4p_items);
      g->device_bytes -= g->c4p_items_cap;
      g->c4p_items = nullptr;
      g->c4p_items_cap = 0;
    }
    GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4p_items, bytes));
    g->c4p_items_cap = bytes;
  }
  if (!items.empty())
    GPM_CUDA(cudaMemcpyAsync(g->c4p_items, items.data(), sizeof(uint32_t) * items.size(), cudaMemcpyHostToDevice, st));
  GPM_CUDA(cudaStreamSynchronize(st));
  g->c4p_ready = true;
  g->c4p_bound = bound;
  g->c4p_pull = pull;
  g->c4p_width = width;
  return GPM_OK;
}

bool gpm_c4_plain_ready(const gpm_graph *g) { return c4_use_range(g) ? g->c4p_ready : g->c4_ready; }

static int launch_c4_bucketed(gpm_graph *g, const C4Args &a, const uint32_t *tasks, uint32_t ntasks, uint32_t maxb,
                              unsigned int *queue, cudaStream_t st) {
  const int sms = gpm_num_sms(g->device);
  C4Args b = a;
  b.tasks = tasks;
  b.ntasks = ntasks;
  b.queue = queue;
  const size_t smem = (size_t)gpm_dev::c4_bucket_smem_words<kC4PlainTable>(kC4BucketThreads / 32) * 4;
  GPM_CUDA(cudaFuncSetAttribute(c4_bucket_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c4_bucket_kernel, kC4BucketThreads, smem));
  const uint64_t slot_words = gpm_dev::c4_bucket_slot_words(std::max<uint32_t>(maxb, 1));
  size_t slots = (size_t)sms * (size_t)std::max(per_sm, 1);
  slots = std::min<size_t>(slots, ntasks);
  const size_t need = slots * slot_words * 4;
  if (g->c4_bucket_bytes < need) {
    if (g->c4_bucket_buf) {
      cudaFree(g->c4_bucket_buf);
      g->device_bytes -= g->c4_bucket_bytes;
      g->c4_bucket_buf = nullptr;
      g->c4_bucket_bytes = 0;
    }
    GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4_bucket_buf, need));
    g->c4_bucket_bytes = need;
  }
  b.pool = g->c4_bucket_buf;
  GPM_LAUNCH("c4_bucket_kernel", st, c4_bucket_kernel<<<(unsigned)slots, kC4BucketThreads, smem, st>>>(b, slot_words));
  GPM_CUDA(cudaGetLastError());
  return GPM_OK;
}

static int launch_c4_small(gpm_graph *g, const C4Args &a, const uint32_t *tasks, uint32_t ntasks, unsigned int *queue,
                           cudaStream_t st) {
  const int sms = gpm_num_sms(g->device);
  C4Args s = a;
  s.tasks = tasks;
  s.ntasks = ntasks;
  s.queue = queue;
  const size_t smem = (size_t)8 * 2 * kHashSlots * 4;
  GPM_CUDA(cudaFuncSetAttribute(c4_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c4_small_kernel, 256, smem));
  int blocks = std::max(1, std::min<int>(sms * std::max(per_sm, 1), (int)((ntasks + 7) / 8)));
  GPM_LAUNCH("c4_small_kernel", st, c4_small_kernel<<<blocks, 256, smem, st>>>(s));
  GPM_CUDA(cudaGetLastError());
  return GPM_OK;
}

static int launch_cycles4_range(gpm_graph *g, uint32_t root_lo, uint32_t root_hi, unsigned long long *acc,
                                cudaStream_t st) {
  GPM_TRY(ensure_c4_plain(g, st));
  unsigned int *queues = reinterpret_cast<unsigned int *>(g->work + WK_QUEUE0) + 4;
  GPM_CUDA(cudaMemsetAsync(queues, 0, 3 * sizeof(unsigned int), st));
  C4Args a{};
  a.rowptr = g->rowptr;
  a.col = g->col;
  a.deg = g->deg;
  a.edeg = g->edeg;
  a.root_lo = root_lo;
  a.root_hi = root_hi;
  a.acc = acc;
  a.status = reinterpret_cast<unsigned int *>(g->work + WK_STATUS);
  a.n = g->n;
  GPM_TRY(gpm_launch_c4_pull(g, root_lo, root_hi, acc, st));
  if (g->c4p_nitems) {
    C4RangeArgs r{};
    r.rowptr = g->rowptr;
    r.col = g->col;
    r.deg = g->deg;
    r.edeg = g->edeg;
    r.roff = g->c4_roff;
    r.nr1 = g->c4_nr1;
    r.width = g->c4_roff_width;
    r.items = reinterpret_cast<const uint4 *>(g->c4p_items);
    r.nitems = g->c4p_nitems;
    r.root_lo = root_lo;
    r.root_hi = root_hi;
    r.queue = queues + 1;
    r.acc = acc;
    r.status = reinterpret_cast<unsigned int *>(g->work + WK_STATUS);
    GPM_CUDA(cudaFuncSetAttribute(c4_range_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRangeSmemBytes));
    int per_sm = 0;
    GPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c4_range_kernel, kRangeThreads, kRangeSmemBytes));
    const unsigned blocks = (unsigned)std::min<uint64_t>((uint64_t)gpm_num_sms(g->device) * std::max(per_sm, 1),
                                                         g->c4p_nitems);
    GPM_LAUNCH("c4_range_kernel", st, c4_range_kernel<<<blocks, kRangeThreads, kRangeSmemBytes, st>>>(r));
    GPM_CUDA(cudaGetLastError());
  }
  const uint32_t nsmall = g->c4p_begin[1], nbucket = g->c4p_begin[2] - g->c4p_begin[1];
  if (nbucket) {
    C4Args ab = a;
    ab.bvals = g->c4p_bval + g->c4p_begin[1];  // the bounds computed when the classes were built
    GPM_TRY(launch_c4_bucketed(g, ab, g->c4p_tasks + g->c4p_begin[1], nbucket, g->c4p_bucket_maxb, queues + 2, st));
  }
  if (nsmall) GPM_TRY(launch_c4_small(g, a, g->c4p_tasks, nsmall, queues, st));
  return GPM_OK;
}

int gpm_launch_cycles4(gpm_graph *g, uint32_t root_lo, uint32_t root_hi, unsigned long long *acc, cudaStream_t st) {
  if (c4_use_range(g)) return launch_cycles4_range(g, root_lo, root_hi, acc, st);
  GPM_TRY(ensure_c4_tasks(g, st));
  unsigned int *queues = reinterpret_cast<unsigned int *>(g->work + WK_QUEUE0) + 4;
  GPM_CUDA(cudaMemsetAsync(queues, 0, 3 * sizeof(unsigned int), st));
  C4Args a{};
  a.rowptr = g->rowptr;
  a.col = g->col;
  a.deg = g->deg;
  a.edeg = g->edeg;
  a.root_lo = root_lo;
  a.root_hi = root_hi;
  a.acc = acc;
  a.status = reinterpret_cast<unsigned int *>(g->work + WK_STATUS);
  a.n = g->n;
  const uint32_t nsmall = g->c4_begin[1] - g->c4_begin[0];
  const uint32_t nbucket = g->c4_begin[2] - g->c4_begin[1];
  const uint32_t nbig = g->c4_begin[3] - g->c4_begin[2];
  if (nsmall) GPM_TRY(launch_c4_small(g, a, g->c4_tasks, nsmall, queues, st));
  if (nbucket)
    GPM_TRY(launch_c4_bucketed(g, a, g->c4_tasks + g->c4_begin[1], nbucket, g->c4_bucket_maxb, queues + 2, st));
  if (nbig) {
    GPM_TRY(ensure_c4_hub(g, st));
    GPM_TRY(launch_c4_hub(g, root_lo, root_hi, acc, st, nullptr));
  }
  return GPM_OK;
}

int gpm_launch_finalize(const FinalizeSpec &spec, const unsigned long long *acc, uint64_t n, uint64_t m,
                        unsigned long long *out, unsigned int *status, cudaStream_t st) {
  GPM_LAUNCH("finalize_kernel", st, finalize_kernel<<<1, 32, 0, st>>>(spec, acc, n, m, out, status));
  GPM_CUDA(cudaGetLastError());
  return GPM_OK;
}
