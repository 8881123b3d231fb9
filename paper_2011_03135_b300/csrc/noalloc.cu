// 4-cycle counting that allocates nothing.
//
// Some callers cannot allocate device memory while they run: frameworks that
// hand all device memory to their own arena and forbid outside allocations,
// jobs with a hard memory budget where an allocation could fail half-way
// through, or latency-sensitive loops where cudaMalloc/cudaFree would
// synchronise the whole device. For them gpm_count_cycles4_noalloc counts
// the edge-induced 4-cycles of a CSR that the caller already holds in device
// memory, writing the count to a device word the caller provides, with every
// intermediate buffer carved from one fixed array that is part of the loaded
// library image (kNoAllocWords 32-bit words = 64 MiB, held by every GPU that
// loads the library until the process exits).
//
// The kernels are a variant of the 4-cycle pass of motif.cu whose degree
// array, tallies, work counters and accumulator live in that array instead of
// buffers owned by a graph handle: roots whose wedge bound is at most 512 are
// counted first by warps with a shared-memory hash (as the small class, every
// SM busy whatever n is); the larger roots then by CTAs with a dense wedge
// tally of n words each (as many CTAs as tallies fit next to the degrees),
// which pick them out of batches of 512 roots.
#include <mutex>

#include "gpm_internal.h"
#include "motif_device.cuh"

namespace {

constexpr uint64_t kNoAllocWords = 16ull << 20;  // 64 MiB
constexpr uint32_t kNoAllocThreads = 512;
constexpr uint32_t kCtrWords = 64;  // [0], [1] claim counters of the two kernels, [2..3] count (uint64)
constexpr uint32_t kSmallWarps = 4;  // 8 KB of hash per warp, 32 KB of static shared memory per block

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

// device address of g_noalloc_scratch, per device (set up once, with the device current)
std::mutex g_mu;
void *g_scratch_addr[64] = {nullptr};

int scratch_address(int device, uint32_t **out) {
  if (device < 0 || device >= 64) return gpm_fail(GPM_E_DEVICE, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return gpm_cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
    g_scratch_addr[device] = p;
  }
  *out = static_cast<uint32_t *>(g_scratch_addr[device]);
  return GPM_OK;
}

__global__ void noalloc_degree_kernel(const uint64_t *__restrict__ rowptr, uint32_t n, uint32_t *__restrict__ deg) {
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
    deg[v] = (uint32_t)(rowptr[v + 1] - rowptr[v]);
}

// wedge bound of root v0: the degrees of its neighbours before it (degree, then id)
__device__ __forceinline__ unsigned long long wedge_bound_thread(const uint64_t *__restrict__ rowptr,
                                                               const uint32_t *__restrict__ col,
                                                               const uint32_t *__restrict__ deg, uint32_t v0) {
  const uint32_t d0 = deg[v0];
  unsigned long long b = 0;
  for (uint64_t e = rowptr[v0]; e < rowptr[v0 + 1]; ++e) {
    const uint32_t x = col[e], dx = deg[x];
    if (gpm_dev::precedes(dx, x, d0, v0)) b += dx;
  }
  return b;
}

// roots with wedge bound in [3, kC4SmallBound]: one warp each, shared-memory hash
__global__ void __launch_bounds__(kSmallWarps * 32) noalloc_small_kernel(const uint64_t *__restrict__ rowptr,
                                                                          const uint32_t *__restrict__ col,
                                                                          const uint32_t *__restrict__ deg, uint32_t n,
                                                                          uint32_t *ctr) {
  __shared__ uint32_t s_hash[kSmallWarps][2 * gpm_dev::kC4HashSlots];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t *keys = s_hash[wid], *cnt = keys + gpm_dev::kC4HashSlots;
  unsigned long long acc = 0;
  bool overflow = false;
  for (;;) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&ctr[0], 32u);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= n) break;
    // lane k finds the bound of root base + k; then the warp takes the small ones in turn
    const uint32_t mine = base + lane;
    const unsigned long long b = mine < n ? wedge_bound_thread(rowptr, col, deg, mine) : 0ull;
    uint32_t small = __ballot_sync(0xffffffffu, b >= 3 && b <= gpm_dev::kC4SmallBound);
    while (small) {
      const uint32_t k = __ffs(small) - 1;
      small &= small - 1;
      acc += gpm_dev::c4_root_warp(rowptr, col, deg, nullptr, base + k, keys, cnt, overflow);
    }
  }
  acc = gpm_dev::warp_sum(acc);
  if (lane == 0 && acc) atomicAdd(reinterpret_cast<unsigned long long *>(ctr + 2), acc);
}

// roots with wedge bound above kC4SmallBound: each CTA takes batches of
// kNoAllocThreads roots, keeps the large ones, and counts each with the whole
// CTA on the dense tally + touched list of its slot
__global__ void __launch_bounds__(kNoAllocThreads) noalloc_c4_kernel(const uint64_t *__restrict__ rowptr,
                                                                      const uint32_t *__restrict__ col,
                                                                      const uint32_t *__restrict__ deg, uint32_t n,
                                                                      uint32_t *slots, uint32_t *ctr) {
  __shared__ uint32_t s_base, s_nbig, s_nt, s_cnt;
  __shared__ uint32_t s_x[kNoAllocThreads], s_big[kNoAllocThreads];
  uint32_t *tally = slots + (size_t)blockIdx.x * 2 * n;
  uint32_t *touched = tally + n;
  unsigned long long acc = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      s_base = atomicAdd(&ctr[1], kNoAllocThreads);
      s_nbig = 0;
    }
    __syncthreads();
    const uint32_t base = s_base;
    if (base >= n) break;
    const uint32_t v = base + threadIdx.x;
    if (v < n && wedge_bound_thread(rowptr, col, deg, v) > gpm_dev::kC4SmallBound) s_big[atomicAdd(&s_nbig, 1u)] = v;
    __syncthreads();
    const uint32_t nbig = s_nbig;
    for (uint32_t i = 0; i < nbig; ++i)
      acc += gpm_dev::c4_root_cta(rowptr, col, deg, nullptr, s_big[i], tally, touched, s_x, &s_cnt, &s_nt);
    __syncthreads();
  }
  acc = gpm_dev::warp_sum(acc);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(reinterpret_cast<unsigned long long *>(ctr + 2), acc);
}

__global__ void noalloc_store_kernel(const uint32_t *ctr, unsigned long long *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = *reinterpret_cast<const unsigned long long *>(ctr + 2);
}

}  // namespace

extern "C" int gpm_count_cycles4_noalloc(const uint64_t *rowptr, const uint32_t *col, uint32_t n, uint64_t *count,
                                         void *stream) {
  if (!rowptr || !count || (n > 0 && !col)) return gpm_fail(GPM_E_INVALID_ARG, "null argument");
  // degrees (n) + at least one slot (2n) + counters must fit in the fixed array
  const uint64_t need_one = (uint64_t)n + 2ull * n + kCtrWords;
  if (need_one > kNoAllocWords)
    return gpm_fail(GPM_E_INVALID_ARG, "graph too large for the no-allocation entry point: n = " + std::to_string(n) +
                                           " needs " + std::to_string(need_one) + " scratch words, the fixed array has " +
                                           std::to_string(kNoAllocWords) + " (n <= " +
                                           std::to_string((kNoAllocWords - kCtrWords) / 3) + ")");
  int device = 0;
  GPM_CUDA(cudaGetDevice(&device));
  uint32_t *base = nullptr;
  GPM_TRY(scratch_address(device, &base));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint32_t *ctr = base;
  uint32_t *deg = base + kCtrWords;
  uint32_t *slots = deg + n;
  const uint64_t slot_words = 2ull * std::max<uint32_t>(n, 1);
  uint64_t nslots = (kNoAllocWords - kCtrWords - n) / slot_words;
  nslots = std::min<uint64_t>(nslots, (uint64_t)gpm_num_sms(device));
  nslots = std::max<uint64_t>(1, std::min<uint64_t>(nslots, std::max<uint32_t>(n, 1)));
  // the array keeps the previous call's contents (possibly laid out for
  // another n): clear what must start at zero -- the counters and the tally
  // half of every slot (the touched half is written before it is read)
  GPM_CUDA(cudaMemsetAsync(ctr, 0, kCtrWords * sizeof(uint32_t), st));
  for (uint64_t s = 0; s < nslots; ++s)
    GPM_CUDA(cudaMemsetAsync(slots + s * slot_words, 0, sizeof(uint32_t) * std::max<uint32_t>(n, 1), st));
  if (n > 0) {
    const int sms = gpm_num_sms(device);
    GPM_LAUNCH("noalloc_degree_kernel", st, noalloc_degree_kernel<<<sms * 4, 256, 0, st>>>(rowptr, n, deg));
    GPM_LAUNCH("noalloc_small_kernel", st,
               noalloc_small_kernel<<<(unsigned)sms * 8, kSmallWarps * 32, 0, st>>>(rowptr, col, deg, n, ctr));
    GPM_LAUNCH("noalloc_c4_kernel", st,
               noalloc_c4_kernel<<<(unsigned)nslots, kNoAllocThreads, 0, st>>>(rowptr, col, deg, n, slots, ctr));
  }
  GPM_LAUNCH("noalloc_store_kernel", st,
             noalloc_store_kernel<<<1, 32, 0, st>>>(ctr, reinterpret_cast<unsigned long long *>(count)));
  GPM_CUDA(cudaGetLastError());
  return GPM_OK;
}
