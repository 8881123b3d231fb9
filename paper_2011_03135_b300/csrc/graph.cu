// Graph ingest on the device: CSR validation, degrees, the degree-ordered
// orientation and the root-task classes.
//
// Orientation (appendix "Orientation (Total Order)"): arc u -> v iff
// (deg u, u) < (deg v, v), i.e. each edge points to the endpoint of higher
// degree and ties point to the larger id. Every row of the oriented CSR keeps
// the ascending id order of the symmetric CSR.
#include <algorithm>
#include <vector>

#include "gpm_internal.h"

namespace {


__device__ __forceinline__ bool precedes(uint32_t du, uint32_t u, uint32_t dv, uint32_t v) {
  return du < dv || (du == dv && u < v);
}

// ---------------------------------------------------------------------------
// validation: one warp per vertex; rows longer than kValidateSplit entries
// are listed and checked by validate_long_kernel, one CTA per row, so that a
// hub's row does not leave one warp working after all others are done
// ---------------------------------------------------------------------------
constexpr uint32_t kValidateSplit = 2048;

// the checks of entry i of the row [b, e) of v (b <= i < e <= nnz, checked by
// the caller): id range, loop, ascending order, mirror arc
__device__ __forceinline__ uint32_t validate_entry(const uint64_t *__restrict__ rowptr,
                                                   const uint32_t *__restrict__ col, uint32_t n, uint64_t nnz,
                                                   uint64_t v, uint64_t b, uint64_t i) {
  uint32_t bad = 0;
  const uint32_t c = col[i];
  if (c >= n) return ST_OUT_OF_RANGE;
  if (c == v) bad |= ST_SELF_LOOP;
  if (i > b) {
    const uint32_t p = col[i - 1];
    if (p == c) bad |= ST_DUPLICATE;
    else if (p > c) bad |= ST_NOT_SORTED;
  }
  // symmetric: v must be in N(c) (binary search; rows may be unsorted if
  // the input is bad, in which case NOT_SORTED is reported as well)
  uint64_t lo = rowptr[c], hi = rowptr[c + 1];
  if (hi < lo || hi > nnz) return bad | ST_BAD_ROWPTR;
  const uint64_t end = hi;
  while (lo < hi) {
    uint64_t mid = lo + ((hi - lo) >> 1);
    if (col[mid] < (uint32_t)v) lo = mid + 1;
    else hi = mid;
  }
  if (lo >= end || col[lo] != (uint32_t)v) bad |= ST_ASYMMETRIC;
  return bad;
}

// longv (room for n ids) and *nlong (zero at launch) collect the rows longer
// than kValidateSplit; with longv null every row is checked here
__global__ void validate_kernel(const uint64_t *__restrict__ rowptr, const uint32_t *__restrict__ col, uint32_t n,
                                uint64_t nnz, uint32_t *__restrict__ status, uint32_t *__restrict__ longv,
                                uint32_t *__restrict__ nlong) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t bad = 0;
  if (warp == 0 && lane == 0) {
    if (rowptr[0] != 0 || rowptr[n] != nnz) bad |= ST_BAD_ROWPTR;
  }
  for (uint64_t v = warp; v < n; v += nwarps) {
    const uint64_t b = rowptr[v], e = rowptr[v + 1];
    if (e < b || e > nnz) {
      bad |= ST_BAD_ROWPTR;
      continue;
    }
    if (longv && e - b > kValidateSplit) {
      if (lane == 0) longv[atomicAdd(nlong, 1u)] = (uint32_t)v;
      continue;
    }
    for (uint64_t i = b + lane; i < e; i += 32) bad |= validate_entry(rowptr, col, n, nnz, v, b, i);
  }
  bad = __reduce_or_sync(0xffffffffu, bad);
  if (lane == 0 && bad) atomicOr(status, bad);
}

// the rows listed by validate_kernel (whose offsets it has checked), one CTA
// per row at a time
__global__ void validate_long_kernel(const uint64_t *__restrict__ rowptr, const uint32_t *__restrict__ col,
                                     uint32_t n, uint64_t nnz, uint32_t *__restrict__ status,
                                     const uint32_t *__restrict__ longv, const uint32_t *__restrict__ nlong) {
  const uint32_t count = *nlong;
  uint32_t bad = 0;
  for (uint32_t l = blockIdx.x; l < count; l += gridDim.x) {
    const uint32_t v = longv[l];
    const uint64_t b = rowptr[v], e = rowptr[v + 1];
    for (uint64_t i = b + threadIdx.x; i < e; i += blockDim.x) bad |= validate_entry(rowptr, col, n, nnz, v, b, i);
  }
  bad = __reduce_or_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicOr(status, bad);
}

// degrees and the largest degree
__global__ void degree_kernel(const uint64_t *__restrict__ rowptr, uint32_t n, uint32_t *__restrict__ deg,
                              uint32_t *__restrict__ maxdeg) {
  uint32_t mx = 0;
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t d = (uint32_t)(rowptr[v + 1] - rowptr[v]);
    deg[v] = d;
    mx = max(mx, d);
  }
  mx = __reduce_max_sync(0xffffffffu, mx);
  if ((threadIdx.x & 31) == 0) atomicMax(maxdeg, mx);
}

// out-degree of every vertex in the orientation: one warp per vertex
__global__ void outdeg_kernel(const uint64_t *__restrict__ rowptr, const uint32_t *__restrict__ col,
                              const uint32_t *__restrict__ deg, uint32_t n, uint32_t *__restrict__ outdeg,
                              uint32_t *__restrict__ maxout) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t mx = 0;
  for (uint64_t v = warp; v < n; v += nwarps) {
    const uint64_t b = rowptr[v], e = rowptr[v + 1];
    const uint32_t dv = deg[v];
    uint32_t c = 0;
    for (uint64_t i = b + lane; i < e; i += 32) {
      const uint32_t w = col[i];
      c += precedes(dv, (uint32_t)v, deg[w], w);
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) outdeg[v] = c;
    mx = max(mx, c);
  }
  if (lane == 0) atomicMax(maxout, mx);
}

// write the kept neighbours of every vertex, order preserved (warp ballot)
__global__ void fill_dag_kernel(const uint64_t *__restrict__ rowptr, const uint32_t *__restrict__ col,
                                const uint32_t *__restrict__ deg, uint32_t n, const uint64_t *__restrict__ drow,
                                uint32_t *__restrict__ dcol) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t v = warp; v < n; v += nwarps) {
    const uint64_t b = rowptr[v], e = rowptr[v + 1];
    const uint32_t dv = deg[v];
    uint64_t out = drow[v];
    for (uint64_t base = b; base < e; base += 32) {
      const uint64_t i = base + lane;
      uint32_t w = 0;
      bool keep = false;
      if (i < e) {
        w = col[i];
        keep = precedes(dv, (uint32_t)v, deg[w], w);
      }
      const uint32_t mask = __ballot_sync(0xffffffffu, keep);
      if (keep) dcol[out + __popc(mask & ((1u << lane) - 1u))] = w;
      out += __popc(mask);
    }
  }
}

// ---------------------------------------------------------------------------
// exclusive scan of uint32 counts into uint64 offsets (three passes)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t *total) {
  __shared__ uint64_t warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint64_t s = (lane < kScanThreads / 32) ? warp_sums[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  uint64_t before = (wid > 0) ? warp_sums[wid - 1] : 0;
  *total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void scan_tiles_kernel(const uint32_t *__restrict__ in, uint64_t n, uint64_t *__restrict__ out,
                                  uint64_t *__restrict__ tile_sums) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint32_t vals[kScanItems];
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    vals[k] = (base + k < n) ? in[base + k] : 0u;
    s += vals[k];
  }
  uint64_t total;
  uint64_t pre = block_exclusive_scan(s, &total);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = pre;
    pre += vals[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void scan_sums_kernel(uint64_t *__restrict__ tile_sums, uint64_t ntiles) {
  uint64_t carry = 0;
  for (uint64_t b = 0; b < ntiles; b += kScanThreads) {
    uint64_t i = b + threadIdx.x;
    uint64_t v = (i < ntiles) ? tile_sums[i] : 0;
    uint64_t total;
    uint64_t pre = block_exclusive_scan(v, &total);
    if (i < ntiles) tile_sums[i] = carry + pre;
    carry += total;
  }
}

__global__ void scan_add_kernel(uint64_t *__restrict__ out, uint64_t n, const uint64_t *__restrict__ tile_sums,
                                const uint32_t *__restrict__ in) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    out[i] += tile_sums[i / kScanTile];
    if (i == n - 1) out[n] = out[i] + in[i];
  }
}

// ---------------------------------------------------------------------------
// root-task classes by out-degree
// ---------------------------------------------------------------------------
__device__ __forceinline__ int task_class(uint32_t d, uint32_t warp_max, uint32_t cta_max) {
  if (d < 2) return -1;
  if (d <= 32) return CLS_W32;
  if (d <= warp_max) return CLS_WARP;
  if (d <= cta_max) return CLS_CTA;
  return CLS_XL;
}

__global__ void class_count_kernel(const uint64_t *__restrict__ drow, uint32_t n, uint32_t warp_max,
                                   uint32_t cta_max, uint32_t *__restrict__ counts, uint32_t *__restrict__ maxd) {
  // per-thread tallies, one warp reduction and one atomic per class and warp
  uint32_t cnt[NUM_CLS] = {0, 0, 0, 0}, mx[NUM_CLS] = {0, 0, 0, 0};
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t d = (uint32_t)(drow[v + 1] - drow[v]);
    int c = task_class(d, warp_max, cta_max);
#pragma unroll
    for (int k = 0; k < NUM_CLS; ++k)
      if (c == k) {
        ++cnt[k];
        mx[k] = max(mx[k], d);
      }
  }
#pragma unroll
  for (int k = 0; k < NUM_CLS; ++k) {
    const uint32_t tc = __reduce_add_sync(0xffffffffu, cnt[k]);
    const uint32_t tm = __reduce_max_sync(0xffffffffu, mx[k]);
    if ((threadIdx.x & 31) == 0 && tc) {
      atomicAdd(&counts[k], tc);
      atomicMax(&maxd[k], tm);
    }
  }
}

// Scatter roots into their class segment, one cursor reservation per class
// and warp step. Within a segment, order is unspecified.
__global__ void class_fill_kernel(const uint64_t *__restrict__ drow, uint32_t n, uint32_t warp_max, uint32_t cta_max,
                                  uint32_t *__restrict__ cursors, uint32_t *__restrict__ tasks) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t base = blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u); base < n; base += stride) {
    const uint64_t v = base + lane;
    int c = -1;
    if (v < n) c = task_class((uint32_t)(drow[v + 1] - drow[v]), warp_max, cta_max);
#pragma unroll
    for (int k = 0; k < NUM_CLS; ++k) {
      const uint32_t m = __ballot_sync(0xffffffffu, c == k);
      if (!m) continue;
      const int leader = __ffs(m) - 1;
      uint32_t pos = 0;
      if ((int)lane == leader) pos = atomicAdd(&cursors[k], (uint32_t)__popc(m));
      pos = __shfl_sync(0xffffffffu, pos, leader);
      if (c == k) tasks[pos + __popc(m & ((1u << lane) - 1u))] = (uint32_t)v;
    }
  }
}

// Sort keys for ordering the CTA and XL classes by decreasing out-degree so
// that the largest roots start first (longest-processing-time-first).
__global__ void class_keys_kernel(const uint32_t *__restrict__ tasks, uint32_t count,
                                  const uint64_t *__restrict__ drow, uint64_t *__restrict__ keys) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    uint32_t v = tasks[i];
    keys[i] = ((uint64_t)(drow[v + 1] - drow[v]) << 32) | v;
  }
}

}  // namespace

int gpm_num_sms(int device) {
  static int cached[64] = {0};
  if (device < 0 || device >= 64) return 148;
  if (!cached[device]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0) v = 148;
    cached[device] = v;
  }
  return cached[device];
}

int gpm_launch_validate(gpm_graph *g, cudaStream_t st, uint32_t *d_status, uint32_t *d_longv, uint32_t *d_nlong) {
  const int sms = gpm_num_sms(g->device);
  GPM_LAUNCH("validate_kernel", st,
             validate_kernel<<<sms * 8, 256, 0, st>>>(g->rowptr, g->col, g->n, g->nnz, d_status, d_longv, d_nlong));
  GPM_CUDA(cudaGetLastError());
  if (d_longv) {
    GPM_LAUNCH("validate_long_kernel", st,
               validate_long_kernel<<<sms * 2, 1024, 0, st>>>(g->rowptr, g->col, g->n, g->nnz, d_status, d_longv,
                                                              d_nlong));
    GPM_CUDA(cudaGetLastError());
  }
  return GPM_OK;
}

int gpm_graph_alloc(gpm_graph *g, void **ptr, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return gpm_fail(GPM_E_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  g->device_bytes += bytes;
  return GPM_OK;
}

int gpm_ensure_classes(gpm_graph *g, cudaStream_t st) {
  const gpm_tuning &t = gpm_tune();
  if (g->tune_warp_max == t.warp_max_degree && g->tune_cta_max == t.cta_max_degree) return GPM_OK;
  if (!g->tasks) GPM_TRY(gpm_graph_alloc(g, (void **)&g->tasks, sizeof(uint32_t) * (size_t)std::max<uint32_t>(g->n, 1)));
  uint32_t *dtmp = reinterpret_cast<uint32_t *>(g->work + WK_MISC);  // 4 counts + 4 maxd = 8 words = 4 uint64
  GPM_CUDA(cudaMemsetAsync(dtmp, 0, 8 * sizeof(uint32_t), st));
  const int blocks = gpm_num_sms(g->device) * 4;
  GPM_LAUNCH("class_count_kernel", st, class_count_kernel<<<blocks, 256, 0, st>>>(g->drow, g->n, t.warp_max_degree, t.cta_max_degree, dtmp, dtmp + 4));
  GPM_CUDA(cudaGetLastError());
  uint32_t h[8];
  GPM_CUDA(cudaMemcpyAsync(h, dtmp, sizeof(h), cudaMemcpyDeviceToHost, st));
  GPM_CUDA(cudaStreamSynchronize(st));
  g->cls_begin[0] = 0;
  for (int c = 0; c < NUM_CLS; ++c) {
    g->cls_begin[c + 1] = g->cls_begin[c] + h[c];
    g->cls_maxdeg[c] = h[4 + c];
  }
  uint32_t cur[4] = {g->cls_begin[0], g->cls_begin[1], g->cls_begin[2], g->cls_begin[3]};
  GPM_CUDA(cudaMemcpyAsync(dtmp, cur, sizeof(cur), cudaMemcpyHostToDevice, st));
  GPM_LAUNCH("class_fill_kernel", st, class_fill_kernel<<<blocks, 256, 0, st>>>(g->drow, g->n, t.warp_max_degree, t.cta_max_degree, dtmp, g->tasks));
  GPM_CUDA(cudaGetLastError());
  const uint32_t big = g->cls_begin[NUM_CLS] - g->cls_begin[CLS_CTA];
  if (big > 1) {
    if (!g->prep_keys)
      GPM_TRY(gpm_graph_alloc(g, (void **)&g->prep_keys, sizeof(uint64_t) * (size_t)std::max<uint32_t>(g->n, 1)));
    uint64_t *dkeys = g->prep_keys;
    GPM_LAUNCH("class_keys_kernel", st, class_keys_kernel<<<(big + 255) / 256, 256, 0, st>>>(g->tasks + g->cls_begin[CLS_CTA], big, g->drow, dkeys));
    std::vector<uint64_t> keys(big);
    GPM_CUDA(cudaGetLastError());
    GPM_CUDA(cudaMemcpyAsync(keys.data(), dkeys, sizeof(uint64_t) * big, cudaMemcpyDeviceToHost, st));
    GPM_CUDA(cudaStreamSynchronize(st));
    std::vector<uint32_t> order(big);
    for (int c = CLS_CTA; c <= CLS_XL; ++c) {
      const uint32_t b = g->cls_begin[c] - g->cls_begin[CLS_CTA], en = g->cls_begin[c + 1] - g->cls_begin[CLS_CTA];
      std::sort(keys.begin() + b, keys.begin() + en, [](uint64_t x, uint64_t y) {
        return (x >> 32) != (y >> 32) ? (x >> 32) > (y >> 32) : (uint32_t)x < (uint32_t)y;
      });
    }
    for (uint32_t i = 0; i < big; ++i) order[i] = (uint32_t)keys[i];
    GPM_CUDA(cudaMemcpyAsync(g->tasks + g->cls_begin[CLS_CTA], order.data(), sizeof(uint32_t) * big,
                             cudaMemcpyHostToDevice, st));
    // split of the CTA class (keys of the class are sorted by decreasing out-degree)
    const uint32_t ncta = g->cls_begin[CLS_CTA + 1] - g->cls_begin[CLS_CTA];
    uint32_t k = 0;
    while (k < ncta && (uint32_t)(keys[k] >> 32) > kCtaSplitDegree) ++k;
    g->cta_split = g->cls_begin[CLS_CTA] + k;
    g->cta_lo_maxd = (k < ncta) ? (uint32_t)(keys[k] >> 32) : 0;
  } else {
    const uint32_t ncta = g->cls_begin[CLS_CTA + 1] - g->cls_begin[CLS_CTA];
    const bool hi = ncta > 0 && g->cls_maxdeg[CLS_CTA] > kCtaSplitDegree;
    g->cta_split = hi ? g->cls_begin[CLS_CTA + 1] : g->cls_begin[CLS_CTA];
    g->cta_lo_maxd = (ncta > 0 && !hi) ? g->cls_maxdeg[CLS_CTA] : 0;
  }
  GPM_CUDA(cudaStreamSynchronize(st));
  g->tune_warp_max = t.warp_max_degree;
  g->tune_cta_max = t.cta_max_degree;
  return GPM_OK;
}

// ---------------------------------------------------------------------------
// Core numbers by level-synchronous peeling (the core value based order of
// the appendix "Orientation (Total Order)"). At level k every vertex still
// present whose remaining degree is <= k gets core number k and is peeled;
// peeling lowers the remaining degree of the neighbours still present, and a
// neighbour whose degree drops to k joins the next frontier of the same
// level. When a level's frontier empties, the next level is the smallest
// remaining degree (at least k + 1). Each vertex also records the round in
// which it is peeled (rounds count across levels): ordered by (round, id),
// every vertex has at most core-number many successors, since its successors
// were all still present, and its remaining degree was at most k, when it
// was taken.
// ---------------------------------------------------------------------------
namespace {

constexpr uint32_t kCoreUnset = 0xffffffffu;

__global__ void core_init_kernel(const uint32_t *__restrict__ deg, uint32_t n, uint32_t *__restrict__ cdeg,
                                 uint32_t *__restrict__ core) {
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
    cdeg[v] = deg[v];
    core[v] = kCoreUnset;
  }
}

// Level-synchronous k-core peel in one cooperative launch (every block is
// resident, so blocks may wait for one another). Phases alternate:
//   scan at level k over the active list (vertices not yet taken when the
//     previous scan ran): every vertex still present with remaining degree
//     <= k is taken in the current round (frontier); the others form the next
//     active list, and the smallest remaining degree among them is kept (to
//     jump over empty levels);
//   peel: the neighbours still present of every frontier vertex lose one
//     remaining degree; a neighbour that drops to k is taken in the next round
//     (claimed once) and forms the next frontier. A frontier holds work items
//     {vertex, piece}: the list of a taken vertex is cut into pieces of
//     kCorePiece entries when it is taken, and a warp walks one piece, so the
//     high-degree vertices of the late rounds spread over the grid;
// peel rounds repeat until a frontier is empty, then k grows. Phase P counts
// into counter slot P % 3 ({frontier items, smallest degree left, unused,
// active list}); block 0 clears slot (P + 1) % 3 at the start of
// phase P, a slot every block has finished reading one phase earlier. Phases
// end at a grid barrier whose waits are bounded: on a timeout the kernel
// records ST_TIMEOUT and stops.
constexpr uint32_t kBarrierSpins = 1u << 24;
constexpr uint32_t kCorePiece = 32;  // list entries per frontier item: one per lane

__device__ __forceinline__ bool grid_barrier(unsigned int *bar, uint32_t nblocks, uint32_t &gen) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const uint32_t target = gen + 1;
    __threadfence();  // this block's writes before its arrival
    if (atomicAdd(&bar[0], 1u) == nblocks - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicExch(&bar[1], target);
    } else {
      uint32_t it = 0;
      while (*(volatile unsigned int *)&bar[1] != target) {
        if (++it > kBarrierSpins) {
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    gen = target;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

struct CoreArgs {
  const uint64_t *__restrict__ rowptr;
  const uint32_t *__restrict__ col;
  const uint32_t *__restrict__ deg;
  uint32_t n;
  uint32_t *cdeg, *core, *order;
  uint2 *fa, *fb;          // frontiers: {vertex, piece} items (n + nnz / kCorePiece each)
  uint32_t *act0, *act1;   // active lists (n words each; act0 = 0..n-1 at launch)
  unsigned int *ctr;       // 3 slots x 4 words
  unsigned int *bar;       // grid barrier {arrivals, generation}, zero at launch
  unsigned int *status;
  uint32_t max_phases;
};

// the pieces of w's list as items of frontier F (item counter *c)
__device__ __forceinline__ void push_pieces(const CoreArgs &a, uint32_t w, uint2 *F, unsigned int *c) {
  const uint32_t np = (__ldg(a.deg + w) + kCorePiece - 1) / kCorePiece;
  if (!np) return;
  const uint32_t at = atomicAdd(c, np);
  for (uint32_t p = 0; p < np; ++p) F[at + p] = make_uint2(w, p);
}

// warp-aggregated append of v to list L with counter *c (lanes with `join`)
__device__ __forceinline__ void warp_append(bool join, uint32_t v, uint32_t *L, unsigned int *c) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t m = __ballot_sync(0xffffffffu, join);
  uint32_t at = 0;
  if (m && lane == 0) at = atomicAdd(c, (uint32_t)__popc(m));
  at = __shfl_sync(0xffffffffu, at, 0);
  if (join) L[at + __popc(m & ((1u << lane) - 1u))] = v;
}

// one neighbour w of a peeled vertex at level k (the remaining degree of a
// vertex already taken may drop further; it is never read again, and the
// claim below fails for it)
__device__ __forceinline__ void core_lower(const CoreArgs &a, uint32_t w, uint32_t k, uint32_t next_round, uint2 *fout,
                                           unsigned int *pc) {
  const uint32_t old = atomicSub(&a.cdeg[w], 1u);
  if (old == k + 1 && atomicCAS(&a.core[w], kCoreUnset, k) == kCoreUnset) {
    a.order[w] = next_round;
    push_pieces(a, w, fout, &pc[0]);
  }
}

__global__ void __launch_bounds__(1024) core_peel_all_kernel(CoreArgs a) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t gtid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t first = blockIdx.x * (uint64_t)blockDim.x;  // this block's first index of a strided loop
  const uint64_t warp = gtid >> 5, nwarps = nth >> 5;
  uint32_t gen = 0, phase = 0, k = 0, round = 0, na = a.n;
  uint32_t *ain = a.act0, *aout = a.act1;
  bool ok = true;
  auto barrier = [&]() -> bool { return grid_barrier(a.bar, gridDim.x, gen); };
  auto clear_next = [&]() {
    if (gtid == 0) {
      unsigned int *nxt = a.ctr + 4 * ((phase + 1) % 3);
      nxt[0] = 0u;
      nxt[1] = kCoreUnset;
      nxt[2] = 0u;
      nxt[3] = 0u;
    }
  };
  for (;;) {
    // ---- scan phase at level k ----
    if (phase >= a.max_phases) {
      ok = false;
      break;
    }
    unsigned int *cnt = a.ctr + 4 * (phase % 3);
    clear_next();
    {
      uint32_t mn = kCoreUnset;
      for (uint64_t base = first; base < na; base += nth) {
        const uint64_t i = base + threadIdx.x;
        bool take = false, keep = false;
        uint32_t v = 0;
        if (i < na) {
          v = ain[i];
          if (a.core[v] == kCoreUnset) {
            const uint32_t c = a.cdeg[v];
            if (c <= k) {
              a.core[v] = k;
              a.order[v] = round;
              take = true;
            } else {
              keep = true;
              mn = min(mn, c);
            }
          }
        }
        if (take) push_pieces(a, v, a.fa, &cnt[0]);
        warp_append(keep, v, aout, &cnt[3]);
      }
      mn = __reduce_min_sync(0xffffffffu, mn);
      if (lane == 0 && mn != kCoreUnset) atomicMin(&cnt[1], mn);
    }
    if (!barrier()) {
      ok = false;
      break;
    }
    ++phase;
    uint32_t nin = *(volatile unsigned int *)&cnt[0];
    const uint32_t mn = *(volatile unsigned int *)&cnt[1];
    na = *(volatile unsigned int *)&cnt[3];
    {
      uint32_t *t = ain;
      ain = aout;
      aout = t;
    }
    if (nin == 0) {
      if (mn == kCoreUnset) break;  // every vertex has been taken
      if (mn <= k) {
        ok = false;
        break;
      }
      k = mn;  // no vertex left at this level: jump to the smallest remaining degree
      continue;
    }
    // ---- peel rounds at level k ----
    uint2 *fin = a.fa, *fout = a.fb;
    while (nin > 0) {
      if (phase >= a.max_phases) {
        ok = false;
        break;
      }
      unsigned int *pc = a.ctr + 4 * (phase % 3);
      clear_next();
      for (uint64_t i = warp; i < nin; i += nwarps) {
        const uint2 it = fin[i];
        const uint64_t e = a.rowptr[it.x + 1];
        const uint64_t b = a.rowptr[it.x] + (uint64_t)it.y * kCorePiece;
        const uint64_t pe = b + kCorePiece < e ? b + kCorePiece : e;
        for (uint64_t j = b + lane; j < pe; j += 32) core_lower(a, a.col[j], k, round + 1, fout, pc);
      }
      if (!barrier()) {
        ok = false;
        break;
      }
      ++phase;
      nin = *(volatile unsigned int *)&pc[0];
      uint2 *t = fin;
      fin = fout;
      fout = t;
      ++round;
    }
    if (!ok) break;
    ++k;
  }
  if (!ok && gtid == 0) atomicOr(a.status, ST_TIMEOUT);
}

__global__ void core_iota_kernel(uint32_t n, uint32_t *__restrict__ act) {
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
    act[v] = (uint32_t)v;
}

}  // namespace

int gpm_core_numbers(gpm_graph *g, cudaStream_t st) {
  const uint32_t n = g->n;
  const size_t nw = std::max<uint32_t>(n, 1);
  if (!g->core) GPM_TRY(gpm_graph_alloc(g, (void **)&g->core, sizeof(uint32_t) * nw));
  // remaining degrees, two active lists, the peel round of every vertex,
  // counters and the grid barrier, then two frontiers of items
  const size_t fcap = nw + g->nnz / kCorePiece + 1;
  if (!g->core_work)
    GPM_TRY(gpm_graph_alloc(g, (void **)&g->core_work, sizeof(uint32_t) * (4 * nw + 16 + 4 * fcap)));
  g->core_order = g->core_work + 3 * nw;
  if (n == 0) return GPM_OK;
  uint32_t *w = g->core_work;
  unsigned int *ctr = g->core_order + nw, *bar = ctr + 12;
  unsigned int *status = reinterpret_cast<unsigned int *>(g->work + WK_STATUS);
  const int sms = gpm_num_sms(g->device);
  GPM_LAUNCH("core_init_kernel", st, core_init_kernel<<<sms * 4, 256, 0, st>>>(g->deg, n, w, g->core));
  GPM_LAUNCH("core_iota_kernel", st, core_iota_kernel<<<sms * 4, 256, 0, st>>>(n, w + nw));
  GPM_CUDA(cudaGetLastError());
  unsigned int init[14] = {0u, kCoreUnset, 0u, 0u, 0u, kCoreUnset, 0u, 0u, 0u, kCoreUnset, 0u, 0u, 0u, 0u};
  GPM_CUDA(cudaMemcpyAsync(ctr, init, sizeof(init), cudaMemcpyHostToDevice, st));
  GPM_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned int), st));
  // one 1024-thread block per SM: the grid barriers between phases cost one
  // arrival per block
  int per_sm = 0;
  GPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, core_peel_all_kernel, 1024, 0));
  if (per_sm < 1) return gpm_fail(GPM_E_DEVICE, "core peel kernel does not fit an SM");
  const unsigned blocks = (unsigned)sms;
  CoreArgs a{};
  a.rowptr = g->rowptr;
  a.col = g->col;
  a.deg = g->deg;
  a.n = n;
  a.cdeg = w;
  a.act0 = w + nw;
  a.act1 = w + 2 * nw;
  a.fa = reinterpret_cast<uint2 *>(w + 4 * nw + 16);
  a.fb = a.fa + fcap;
  a.core = g->core;
  a.order = g->core_order;
  a.ctr = ctr;
  a.bar = bar;
  a.status = status;
  // every round takes at least one vertex, every scan without one raises k:
  // at most n rounds and n + 1 scans
  a.max_phases = (uint32_t)std::min<uint64_t>(0xffffffffull, 2ull * n + 4);
  void *args[] = {&a};
  GPM_LAUNCH("core_peel_all_kernel", st,
             GPM_CUDA(cudaLaunchCooperativeKernel((const void *)core_peel_all_kernel, dim3(blocks), dim3(1024), args, 0,
                                                  st)));
  GPM_CUDA(cudaGetLastError());
  unsigned int s = 0;
  GPM_CUDA(cudaMemcpyAsync(&s, status, sizeof(s), cudaMemcpyDeviceToHost, st));
  GPM_CUDA(cudaStreamSynchronize(st));
  if (s & ST_TIMEOUT) return gpm_fail(GPM_E_TIMEOUT, "core peel: a grid barrier wait or the phase limit ran out");
  return GPM_OK;
}

int gpm_prepare_graph(gpm_graph *g, cudaStream_t st) {
  if (g->prepared) return gpm_ensure_classes(g, st);
  const uint32_t n = g->n;
  g->m = g->nnz / 2;
  if (!g->drow) GPM_TRY(gpm_graph_alloc(g, (void **)&g->drow, sizeof(uint64_t) * ((size_t)n + 1)));
  if (!g->dcol) GPM_TRY(gpm_graph_alloc(g, (void **)&g->dcol, sizeof(uint32_t) * (size_t)std::max<uint64_t>(g->m, 1)));
  const uint64_t ntiles = ((uint64_t)n + kScanTile - 1) / kScanTile;
  if (!g->prep_outdeg)
    GPM_TRY(gpm_graph_alloc(g, (void **)&g->prep_outdeg, sizeof(uint32_t) * (size_t)std::max<uint32_t>(n, 1)));
  if (!g->prep_tiles)
    GPM_TRY(gpm_graph_alloc(g, (void **)&g->prep_tiles, sizeof(uint64_t) * (size_t)std::max<uint64_t>(ntiles, 1)));
  uint32_t *outdeg = g->prep_outdeg;
  uint64_t *tile_sums = g->prep_tiles;
  uint32_t *dmax = reinterpret_cast<uint32_t *>(g->work + WK_MISC);
  cudaError_t e = cudaMemsetAsync(dmax, 0, 2 * sizeof(uint32_t), st);
  const int sms = gpm_num_sms(g->device);
  if (e == cudaSuccess && n > 0) {
    GPM_LAUNCH("degree_kernel", st, degree_kernel<<<sms * 4, 256, 0, st>>>(g->rowptr, n, g->deg, dmax));
    g->okey = g->deg;
    if (g->orient_mode == GPM_ORIENT_CORE) {
      GPM_TRY(gpm_core_numbers(g, st));
      g->okey = g->core_order;
    }
    GPM_LAUNCH("outdeg_kernel", st, outdeg_kernel<<<sms * 8, 256, 0, st>>>(g->rowptr, g->col, g->okey, n, outdeg, dmax + 1));
    GPM_LAUNCH("scan_tiles_kernel", st, scan_tiles_kernel<<<(unsigned)ntiles, kScanThreads, 0, st>>>(outdeg, n, g->drow, tile_sums));
    GPM_LAUNCH("scan_sums_kernel", st, scan_sums_kernel<<<1, kScanThreads, 0, st>>>(tile_sums, ntiles));
    GPM_LAUNCH("scan_add_kernel", st, scan_add_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g->drow, n, tile_sums, outdeg));
    GPM_LAUNCH("fill_dag_kernel", st, fill_dag_kernel<<<sms * 8, 256, 0, st>>>(g->rowptr, g->col, g->okey, n, g->drow, g->dcol));
    e = cudaGetLastError();
  } else if (e == cudaSuccess) {
    e = cudaMemsetAsync(g->drow, 0, sizeof(uint64_t), st);
  }
  uint32_t h[2] = {0, 0};
  uint64_t arcs = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, dmax, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&arcs, g->drow + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return gpm_cuda_fail(e, "orientation");
  g->max_degree = h[0];
  g->max_outdeg = h[1];
  if (arcs != g->m) return gpm_fail(GPM_E_ASYMMETRIC, "orientation produced " + std::to_string(arcs) +
                                                          " arcs for " + std::to_string(g->m) + " edges");
  g->prepared = true;
  return gpm_ensure_classes(g, st);
}
