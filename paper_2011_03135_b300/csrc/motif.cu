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
// pair of such wedges, so the count is sum_w C(tally(w), 2). Roots with a
// small wedge bound tally in a per-warp shared-memory hash table, the others
// in a dense per-CTA tally array in global memory.
#include <algorithm>

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
                                  uint32_t root_lo, uint32_t root_hi, unsigned long long *__restrict__ acc) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  gpm_dev::EdgeTerms s;
  for (uint64_t u = warp; u < n; u += nwarps)
    gpm_dev::edge_terms_vertex<USE_T, false>(drow, dcol, deg, t_edge, u, u >= root_lo && u < root_hi, s);
  s.D = warp_sum(s.D);
  s.P = warp_sum(s.P);
  s.S = warp_sum(s.S);
  s.W = warp_sum(s.W);
  s.TT = warp_sum(s.TT);
  s.T3 = warp_sum(s.T3);
  if (lane == 0) {
    atomicAdd(&acc[ACC_P], s.P);
    atomicAdd(&acc[ACC_S], s.S);
    atomicAdd(&acc[ACC_W], s.W);
    if (USE_T) {
      atomicAdd(&acc[ACC_D], s.D);
      atomicAdd(&acc[ACC_TT2], s.TT);
      atomicAdd(&acc[ACC_T3], s.T3);
    }
  }
}

// ---------------------------------------------------------------------------
// 4-cycles
// ---------------------------------------------------------------------------
constexpr uint32_t kSmallBound = gpm_dev::kC4SmallBound;
constexpr uint32_t kHashSlots = gpm_dev::kC4HashSlots;

// wedge bound B(v0) = sum of d_x over neighbours x before v0; class 0 small
// (warp hash), 1 bucketed, 2 dense tally
__global__ void c4_bound_kernel(const uint64_t *__restrict__ rowptr, const uint32_t *__restrict__ col,
                                const uint32_t *__restrict__ deg, uint32_t n, uint32_t *__restrict__ counts,
                                uint32_t *__restrict__ tasks, uint32_t *__restrict__ cursors, int fill) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t v = warp; v < n; v += nwarps) {
    const uint32_t dv = deg[v];
    unsigned long long b = 0;
    for (uint64_t e = rowptr[v] + lane; e < rowptr[v + 1]; e += 32) {
      const uint32_t x = col[e];
      const uint32_t dx = deg[x];
      if (precedes(dx, x, dv, (uint32_t)v)) b += dx;
    }
    b = warp_sum(b);
    if (lane == 0 && b >= 3) {  // a cycle needs two wedges, each scanning v0 itself plus w
      const int c = (b <= kSmallBound) ? 0 : (b <= gpm_dev::kC4BucketMaxBound ? 1 : 2);
      if (fill) {
        tasks[atomicAdd(&cursors[c], 1u)] = (uint32_t)v;
      } else {
        atomicAdd(&counts[c], 1u);
        if (c == 1) atomicMax(&counts[3], (uint32_t)b);
      }
    }
  }
}

struct C4Args {
  const uint64_t *__restrict__ rowptr;
  const uint32_t *__restrict__ col;
  const uint32_t *__restrict__ deg;
  const uint32_t *__restrict__ tasks;
  uint32_t ntasks;
  uint32_t root_lo, root_hi;
  unsigned int *queue;
  unsigned long long *acc;
  unsigned int *status;
  uint32_t *pool;  // big class: per CTA, tally[n] then touched[n]
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
  for (;;) {
    uint32_t task = 0;
    if (lane == 0) task = atomicAdd(a.queue, 1u);
    task = __shfl_sync(0xffffffffu, task, 0);
    if (task >= a.ntasks) break;
    const uint32_t v0 = a.tasks[task];
    if (v0 < a.root_lo || v0 >= a.root_hi) continue;
    acc += gpm_dev::c4_root_warp(a.rowptr, a.col, a.deg, v0, keys, cnt, overflow);
  }
  acc = warp_sum(acc);
  if (lane == 0 && acc) atomicAdd(&a.acc[ACC_C4], acc);
  if (__any_sync(0xffffffffu, overflow) && lane == 0) atomicOr(a.status, ST_CAPACITY);
}

// one CTA per root, dense tally in this CTA's global-memory slot
constexpr int kC4BigThreads = 256;
__global__ void __launch_bounds__(kC4BigThreads) c4_big_kernel(C4Args a) {
  __shared__ uint32_t s_task, s_nt, s_cnt;
  __shared__ uint32_t s_x[kC4BigThreads];
  const uint32_t tid = threadIdx.x, lane = tid & 31;
  uint32_t *tally = a.pool + (size_t)blockIdx.x * 2 * a.n;
  uint32_t *touched = tally + a.n;
  unsigned long long acc = 0;
  for (;;) {
    if (tid == 0) s_task = atomicAdd(a.queue, 1u);
    __syncthreads();
    const uint32_t task = s_task;
    __syncthreads();
    if (task >= a.ntasks) break;
    const uint32_t v0 = a.tasks[task];
    if (v0 < a.root_lo || v0 >= a.root_hi) continue;
    acc += gpm_dev::c4_root_cta(a.rowptr, a.col, a.deg, v0, tally, touched, s_x, &s_cnt, &s_nt);
  }
  acc = warp_sum(acc);
  if (lane == 0 && acc) atomicAdd(&a.acc[ACC_C4], acc);
}

// one CTA per large root, bucketed aggregation (buffer slot per CTA)
constexpr int kC4BucketThreads = 512;
__global__ void __launch_bounds__(kC4BucketThreads) c4_bucket_kernel(C4Args a, uint64_t slot_words) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_task, s_cnt;
  __shared__ uint32_t s_x[kC4BucketThreads];
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
    acc += gpm_dev::c4_root_bucketed(a.rowptr, a.col, a.deg, v0, buf, smem, s_x, &s_cnt, overflow);
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(&a.acc[ACC_C4], acc);
  if (__syncthreads_or(overflow) && threadIdx.x == 0) atomicOr(a.status, ST_CAPACITY);
}

// ---------------------------------------------------------------------------
// finalize: requested counts from the accumulators (one thread)
// ---------------------------------------------------------------------------
__global__ void finalize_kernel(FinalizeSpec spec, const unsigned long long *__restrict__ acc, uint64_t n, uint64_t m,
                                unsigned long long *__restrict__ out, unsigned int *__restrict__ status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  bool bad = false;
  for (uint32_t i = 0; i < spec.npat; ++i) out[i] = gpm_dev::finalize_formula(spec.formula[i], acc, n, m, bad);
  if (bad) atomicOr(status, ST_CAPACITY);
}

}  // namespace

int gpm_launch_edge_terms(gpm_graph *g, bool use_t_edge, uint32_t root_lo, uint32_t root_hi,
                          unsigned long long *acc, cudaStream_t st) {
  const int blocks = gpm_num_sms(g->device) * 8;
  if (g->n == 0) return GPM_OK;
  if (use_t_edge)
    GPM_LAUNCH("edge_terms_kernel", st, edge_terms_kernel<true><<<blocks, 256, 0, st>>>(g->drow, g->dcol, g->deg, g->t_edge, g->n, root_lo, root_hi, acc));
  else
    GPM_LAUNCH("edge_terms_kernel", st, edge_terms_kernel<false><<<blocks, 256, 0, st>>>(g->drow, g->dcol, g->deg, nullptr, g->n, root_lo, root_hi, acc));
  GPM_CUDA(cudaGetLastError());
  return GPM_OK;
}

static int ensure_c4_tasks(gpm_graph *g, cudaStream_t st) {
  if (g->c4_ready) return GPM_OK;
  if (!g->c4_tasks) GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4_tasks, sizeof(uint32_t) * std::max<uint32_t>(g->n, 1)));
  uint32_t *tmp = reinterpret_cast<uint32_t *>(g->work + WK_MISC);  // counts[3], max bound, cursors[3]
  GPM_CUDA(cudaMemsetAsync(tmp, 0, 8 * sizeof(uint32_t), st));
  const int blocks = gpm_num_sms(g->device) * 8;
  if (g->n) {
    GPM_LAUNCH("c4_bound_kernel", st,
               c4_bound_kernel<<<blocks, 256, 0, st>>>(g->rowptr, g->col, g->deg, g->n, tmp, nullptr, nullptr, 0));
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
               c4_bound_kernel<<<blocks, 256, 0, st>>>(g->rowptr, g->col, g->deg, g->n, nullptr, g->c4_tasks, tmp + 4, 1));
    GPM_CUDA(cudaGetLastError());
  }
  GPM_CUDA(cudaStreamSynchronize(st));
  g->c4_ready = true;
  return GPM_OK;
}

int gpm_build_c4_tasks(gpm_graph *g, cudaStream_t st) { return ensure_c4_tasks(g, st); }

int gpm_launch_cycles4(gpm_graph *g, uint32_t root_lo, uint32_t root_hi, unsigned long long *acc, cudaStream_t st) {
  GPM_TRY(ensure_c4_tasks(g, st));
  unsigned int *queues = reinterpret_cast<unsigned int *>(g->work + WK_QUEUE0) + 4;
  GPM_CUDA(cudaMemsetAsync(queues, 0, 3 * sizeof(unsigned int), st));
  C4Args a{};
  a.rowptr = g->rowptr;
  a.col = g->col;
  a.deg = g->deg;
  a.root_lo = root_lo;
  a.root_hi = root_hi;
  a.acc = acc;
  a.status = reinterpret_cast<unsigned int *>(g->work + WK_STATUS);
  a.n = g->n;
  const int sms = gpm_num_sms(g->device);
  const uint32_t nsmall = g->c4_begin[1] - g->c4_begin[0];
  const uint32_t nbucket = g->c4_begin[2] - g->c4_begin[1];
  const uint32_t nbig = g->c4_begin[3] - g->c4_begin[2];
  if (nsmall) {
    C4Args s = a;
    s.tasks = g->c4_tasks;
    s.ntasks = nsmall;
    s.queue = queues;
    const size_t smem = (size_t)8 * 2 * kHashSlots * 4;
    GPM_CUDA(cudaFuncSetAttribute(c4_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c4_small_kernel, 256, smem));
    int blocks = std::max(1, std::min<int>(sms * std::max(per_sm, 1), (int)((nsmall + 7) / 8)));
    GPM_LAUNCH("c4_small_kernel", st, c4_small_kernel<<<blocks, 256, smem, st>>>(s));
    GPM_CUDA(cudaGetLastError());
  }
  if (nbucket) {
    C4Args b = a;
    b.tasks = g->c4_tasks + g->c4_begin[1];
    b.ntasks = nbucket;
    b.queue = queues + 2;
    const size_t smem = (size_t)gpm_dev::c4_bucket_smem_words(kC4BucketThreads / 32) * 4;
    GPM_CUDA(cudaFuncSetAttribute(c4_bucket_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c4_bucket_kernel, kC4BucketThreads, smem));
    const uint64_t slot_words = ((uint64_t)std::max<uint32_t>(g->c4_bucket_maxb, 1) + 63) & ~63ull;
    size_t slots = (size_t)sms * (size_t)std::max(per_sm, 1);
    slots = std::min<size_t>(slots, nbucket);
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
    GPM_LAUNCH("c4_bucket_kernel", st,
               c4_bucket_kernel<<<(unsigned)slots, kC4BucketThreads, smem, st>>>(b, slot_words));
    GPM_CUDA(cudaGetLastError());
  }
  if (nbig) {
    C4Args b = a;
    b.tasks = g->c4_tasks + g->c4_begin[2];
    b.ntasks = nbig;
    b.queue = queues + 1;
    // hub roots are bound by the latency of their global tally atomics: keep many
    // CTAs resident (each with its own tally slot), within a memory budget
    int per_sm = 0;
    GPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c4_big_kernel, kC4BigThreads, 0));
    const size_t slot_bytes = 2 * (size_t)std::max<uint32_t>(g->n, 1) * 4;
    const size_t budget = (size_t)16 << 30;
    size_t slots = (size_t)sms * (size_t)std::max(1, std::min(per_sm, 8));
    slots = std::min(slots, std::max<size_t>(1, budget / slot_bytes));
    slots = std::min(slots, (size_t)nbig);
    if (g->tally_slots < slots) {
      if (g->tally_pool) {
        cudaFree(g->tally_pool);
        g->device_bytes -= g->tally_slots * slot_bytes;
        g->tally_pool = nullptr;
        g->tally_slots = 0;
      }
      GPM_TRY(gpm_graph_alloc(g, (void **)&g->tally_pool, slots * slot_bytes));
      GPM_CUDA(cudaMemsetAsync(g->tally_pool, 0, slots * slot_bytes, st));
      g->tally_slots = slots;
    }
    b.pool = g->tally_pool;
    GPM_LAUNCH("c4_big_kernel", st, c4_big_kernel<<<(unsigned)slots, kC4BigThreads, 0, st>>>(b));
    GPM_CUDA(cudaGetLastError());
  }
  return GPM_OK;
}

int gpm_launch_finalize(const FinalizeSpec &spec, const unsigned long long *acc, uint64_t n, uint64_t m,
                        unsigned long long *out, unsigned int *status, cudaStream_t st) {
  GPM_LAUNCH("finalize_kernel", st, finalize_kernel<<<1, 32, 0, st>>>(spec, acc, n, m, out, status));
  GPM_CUDA(cudaGetLastError());
  return GPM_OK;
}
