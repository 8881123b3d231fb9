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
// The kernel is a variant of the 4-cycle pass (one CTA per root, dense wedge
// tally per CTA, as in motif.cu) whose tallies, degree array, work queue and
// accumulator live in that array instead of buffers owned by a graph handle.
#include <mutex>

#include "gpm_internal.h"
#include "motif_device.cuh"

namespace {

constexpr uint64_t kNoAllocWords = 16ull << 20;  // 64 MiB
constexpr uint32_t kNoAllocThreads = 512;
constexpr uint32_t kCtrWords = 64;  // [0] queue head, [1] status, [2..3] count (uint64)

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

// every vertex is a candidate root (order-last vertex of its cycles); one CTA
// per root, tally + touched list in this CTA's slot of the scratch
__global__ void __launch_bounds__(kNoAllocThreads) noalloc_c4_kernel(const uint64_t *__restrict__ rowptr,
                                                                      const uint32_t *__restrict__ col,
                                                                      const uint32_t *__restrict__ deg, uint32_t n,
                                                                      uint32_t *slots, uint32_t *ctr) {
  __shared__ uint32_t s_root, s_nt, s_cnt;
  __shared__ uint32_t s_x[kNoAllocThreads];
  uint32_t *tally = slots + (size_t)blockIdx.x * 2 * n;
  uint32_t *touched = tally + n;
  unsigned long long acc = 0;
  for (;;) {
    if (threadIdx.x == 0) s_root = atomicAdd(&ctr[0], 1u);
    __syncthreads();
    const uint32_t v0 = s_root;
    __syncthreads();
    if (v0 >= n) break;
    acc += gpm_dev::c4_root_cta(rowptr, col, deg, nullptr, v0, tally, touched, s_x, &s_cnt, &s_nt);
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
  // the array keeps the previous call's contents: clear what must start at zero
  GPM_CUDA(cudaMemsetAsync(ctr, 0, kCtrWords * sizeof(uint32_t), st));
  GPM_CUDA(cudaMemsetAsync(slots, 0, nslots * slot_words * sizeof(uint32_t), st));
  if (n > 0) {
    GPM_LAUNCH("noalloc_degree_kernel", st, noalloc_degree_kernel<<<gpm_num_sms(device) * 4, 256, 0, st>>>(rowptr, n, deg));
    GPM_LAUNCH("noalloc_c4_kernel", st,
               noalloc_c4_kernel<<<(unsigned)nslots, kNoAllocThreads, 0, st>>>(rowptr, col, deg, n, slots, ctr));
  }
  GPM_LAUNCH("noalloc_store_kernel", st,
             noalloc_store_kernel<<<1, 32, 0, st>>>(ctr, reinterpret_cast<unsigned long long *>(count)));
  GPM_CUDA(cudaGetLastError());
  return GPM_OK;
}
