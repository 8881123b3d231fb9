// Subgraph listing (Section 2, SL; listing requires enumerating every
// embedding that is written, counting does not). Each kernel writes tuples in
// the order of its pattern TEMPLATE, each one the representative that
// satisfies the template's symmetry-breaking constraints (appendix "Symmetry
// Breaking (Partial Order)"); the caller permutes template positions to the
// user's pattern numbering.
//
// Output slots are reserved with one atomicAdd per group of matches; a kernel
// stops enumerating once the counter reaches the capacity, so writing the
// first `cap` matches costs far less than a full enumeration.
//
// Templates:
//   diamond  (a, b, c, d): shared edge {a, b} with a < b, c < d both adjacent
//            to a and b (matching order: triangle first, appendix "Pattern-
//            Guided Search (Matching Order)", the order the paper selects)
//   4-cycle  (v0, w, x, y): cycle v0-x-w-y-v0, v0 the smallest id, w opposite
//            to v0, x < y
//   k-clique ascending ids (k = 3..5 with unrolled levels, 6..8 with a
//            per-warp stack of candidate levels)
#include <algorithm>

#include "gpm_internal.h"

namespace {

__device__ __forceinline__ bool stop_now(const unsigned long long *counter, uint64_t cap) {
  return *(volatile const unsigned long long *)counter >= cap;
}

__device__ __forceinline__ bool bsearch_u32(const uint32_t *a, uint64_t n, uint32_t x) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    uint64_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo < n && a[lo] == x;
}

// Warp-cooperative A ∩ B of two ascending lists into out (ascending); every
// lane returns the size. Elements of the shorter list are searched in the
// longer one.
__device__ uint32_t warp_intersect(const uint32_t *A, uint64_t na, const uint32_t *B, uint64_t nb, uint32_t *out) {
  const uint32_t lane = threadIdx.x & 31;
  if (na > nb) {
    const uint32_t *t = A;
    A = B;
    B = t;
    uint64_t tn = na;
    na = nb;
    nb = tn;
  }
  uint32_t cnt = 0;
  for (uint64_t b = 0; b < na; b += 32) {
    const uint64_t i = b + lane;
    uint32_t x = 0;
    bool hit = false;
    if (i < na) {
      x = A[i];
      hit = bsearch_u32(B, nb, x);
    }
    const uint32_t m = __ballot_sync(0xffffffffu, hit);
    if (hit) out[cnt + __popc(m & ((1u << lane) - 1u))] = x;
    cnt += __popc(m);
  }
  __syncwarp();
  return cnt;
}

__global__ void list_diamond_kernel(const uint64_t *__restrict__ rowptr, const uint32_t *__restrict__ col,
                                    const uint64_t *__restrict__ drow, const uint32_t *__restrict__ dcol, uint32_t n,
                                    uint32_t *__restrict__ buf, uint64_t cap, unsigned long long *counter,
                                    uint32_t *__restrict__ scratch, uint64_t scratch_words) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t *T = scratch + warp * scratch_words;
  for (uint64_t u = warp; u < n; u += nwarps) {
    if (stop_now(counter, cap)) return;
    for (uint64_t e = drow[u]; e < drow[u + 1]; ++e) {
      if (stop_now(counter, cap)) return;
      const uint32_t v = dcol[e];
      const uint32_t a = min((uint32_t)u, v), b = max((uint32_t)u, v);
      const uint32_t t = warp_intersect(col + rowptr[u], rowptr[u + 1] - rowptr[u], col + rowptr[v],
                                        rowptr[v + 1] - rowptr[v], T);
      if (t < 2) continue;
      const unsigned long long P = (unsigned long long)t * (t - 1) / 2;
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(counter, P);
      base = __shfl_sync(0xffffffffu, base, 0);
      if (base >= cap) return;
      const unsigned long long lim = min(P, (unsigned long long)(cap - base));
      for (uint32_t ci = 0; ci + 1 < t; ++ci) {
        const unsigned long long off = (unsigned long long)ci * (2ull * t - ci - 1) / 2;
        if (off >= lim) break;
        for (uint32_t dj = ci + 1 + lane; dj < t; dj += 32) {
          const unsigned long long q = off + (dj - ci - 1);
          if (q < lim) {
            uint4 tup = make_uint4(a, b, T[ci], T[dj]);
            *reinterpret_cast<uint4 *>(buf + (base + q) * 4) = tup;
          }
        }
      }
      __syncwarp();
    }
  }
}

__global__ void list_cycle4_kernel(const uint64_t *__restrict__ rowptr, const uint32_t *__restrict__ col, uint32_t n,
                                   uint32_t *__restrict__ buf, uint64_t cap, unsigned long long *counter) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t v0 = warp; v0 < n; v0 += nwarps) {
    const uint64_t b0 = rowptr[v0], e0 = rowptr[v0 + 1];
    for (uint64_t ix = b0; ix < e0; ++ix) {
      if (stop_now(counter, cap)) return;
      const uint32_t x = col[ix];
      if (x <= v0) continue;
      // lanes over w in N(x), w > v0; y in N(v0) ∩ N(w) with y > x
      for (uint64_t f = rowptr[x] + lane; f < rowptr[x + 1]; f += 32) {
        const uint32_t w = col[f];
        if (w <= v0) continue;
        const uint64_t bw = rowptr[w], ew = rowptr[w + 1];
        uint64_t i = ix + 1, j = bw;
        while (i < e0 && j < ew) {
          const uint32_t yi = col[i], yj = col[j];
          if (yi < yj) ++i;
          else if (yi > yj) ++j;
          else {
            const unsigned long long slot = atomicAdd(counter, 1ull);
            if (slot >= cap) break;
            *reinterpret_cast<uint4 *>(buf + slot * 4) = make_uint4((uint32_t)v0, w, x, yi);
            ++i;
            ++j;
          }
        }
      }
    }
  }
}

__device__ __forceinline__ void sort_small(uint32_t *v, int k) {
  for (int i = 1; i < k; ++i) {
    uint32_t x = v[i];
    int j = i - 1;
    while (j >= 0 && v[j] > x) {
      v[j + 1] = v[j];
      --j;
    }
    v[j + 1] = x;
  }
}

// k-cliques, k = 3..5: one warp per root u, arcs u -> x, candidate sets of
// successive levels in the warp's scratch (the per-level candidate stack).
__global__ void list_cliques_kernel(const uint64_t *__restrict__ drow, const uint32_t *__restrict__ dcol, uint32_t n,
                                    int k, uint32_t *__restrict__ buf, uint64_t cap, unsigned long long *counter,
                                    uint32_t *__restrict__ scratch, uint64_t level_words) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t *C1 = scratch + warp * 3 * level_words;
  uint32_t *C2 = C1 + level_words;
  uint32_t *C3 = C2 + level_words;
  for (uint64_t u = warp; u < n; u += nwarps) {
    const uint64_t ub = drow[u], ue = drow[u + 1];
    if (ue - ub < (uint64_t)(k - 1)) continue;
    for (uint64_t e = ub; e < ue; ++e) {
      if (stop_now(counter, cap)) return;
      const uint32_t x = dcol[e];
      const uint32_t c1 = warp_intersect(dcol + ub, ue - ub, dcol + drow[x], drow[x + 1] - drow[x], C1);
      if (k == 3) {
        if (!c1) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(counter, (unsigned long long)c1);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (uint32_t i = lane; i < c1; i += 32)
          if (base + i < cap) {
            uint32_t t[3] = {(uint32_t)u, x, C1[i]};
            sort_small(t, 3);
            for (int q = 0; q < 3; ++q) buf[(base + i) * 3 + q] = t[q];
          }
        continue;
      }
      for (uint32_t a = 0; a < c1; ++a) {
        const uint32_t y = C1[a];
        const uint32_t c2 = warp_intersect(C1, c1, dcol + drow[y], drow[y + 1] - drow[y], C2);
        if (k == 4) {
          if (!c2) continue;
          unsigned long long base = 0;
          if (lane == 0) base = atomicAdd(counter, (unsigned long long)c2);
          base = __shfl_sync(0xffffffffu, base, 0);
          for (uint32_t i = lane; i < c2; i += 32)
            if (base + i < cap) {
              uint32_t t[4] = {(uint32_t)u, x, y, C2[i]};
              sort_small(t, 4);
              for (int q = 0; q < 4; ++q) buf[(base + i) * 4 + q] = t[q];
            }
          continue;
        }
        for (uint32_t b = 0; b < c2; ++b) {
          const uint32_t z = C2[b];
          const uint32_t c3 = warp_intersect(C2, c2, dcol + drow[z], drow[z + 1] - drow[z], C3);
          if (!c3) continue;
          unsigned long long base = 0;
          if (lane == 0) base = atomicAdd(counter, (unsigned long long)c3);
          base = __shfl_sync(0xffffffffu, base, 0);
          for (uint32_t i = lane; i < c3; i += 32)
            if (base + i < cap) {
              uint32_t t[5] = {(uint32_t)u, x, y, z, C3[i]};
              sort_small(t, 5);
              for (int q = 0; q < 5; ++q) buf[(base + i) * 5 + q] = t[q];
            }
        }
        if (stop_now(counter, cap)) return;
      }
    }
  }
}

// k-cliques, k = 6..8: the same per-root search with the candidate sets of
// all k - 2 levels on a per-warp stack in scratch, walked depth first by the
// whole warp (the position in every level is warp-uniform). Level l holds the
// candidates for the next vertex after u, x and the picks of levels 1..l-1;
// the last level is written out.
__global__ void list_cliques_deep_kernel(const uint64_t *__restrict__ drow, const uint32_t *__restrict__ dcol,
                                         uint32_t n, int k, uint32_t *__restrict__ buf, uint64_t cap,
                                         unsigned long long *counter, uint32_t *__restrict__ scratch,
                                         uint64_t level_words) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t *stack = scratch + warp * (uint64_t)(k - 2) * level_words;
  const int last = k - 2;
  for (uint64_t u = warp; u < n; u += nwarps) {
    const uint64_t ub = drow[u], ue = drow[u + 1];
    if (ue - ub < (uint64_t)(k - 1)) continue;
    for (uint64_t e = ub; e < ue; ++e) {
      if (stop_now(counter, cap)) return;
      const uint32_t x = dcol[e];
      uint32_t cnt[8], pos[8], pick[8];
      cnt[1] = warp_intersect(dcol + ub, ue - ub, dcol + drow[x], drow[x + 1] - drow[x], stack);
      pos[1] = 0;
      int l = 1;
      while (l >= 1) {
        const uint32_t *Cl = stack + (uint64_t)(l - 1) * level_words;
        if (l == last) {
          const uint32_t c = cnt[l];
          if (c) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(counter, (unsigned long long)c);
            base = __shfl_sync(0xffffffffu, base, 0);
            for (uint32_t i = lane; i < c; i += 32)
              if (base + i < cap) {
                uint32_t t[8];
                t[0] = (uint32_t)u;
                t[1] = x;
                for (int q = 1; q < l; ++q) t[1 + q] = pick[q];
                t[k - 1] = Cl[i];
                sort_small(t, k);
                for (int q = 0; q < k; ++q) buf[(base + i) * k + q] = t[q];
              }
          }
          --l;
          continue;
        }
        if (pos[l] >= cnt[l]) {
          --l;
          continue;
        }
        if (stop_now(counter, cap)) return;
        const uint32_t y = Cl[pos[l]++];
        pick[l] = y;
        cnt[l + 1] = warp_intersect(Cl, cnt[l], dcol + drow[y], drow[y + 1] - drow[y],
                                    stack + (uint64_t)l * level_words);
        pos[l + 1] = 0;
        ++l;
      }
    }
  }
}

struct Perm8 {
  uint32_t p[8];
};

__global__ void permute_kernel(uint32_t *__restrict__ buf, uint64_t count, int k, Perm8 perm) {
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < count; t += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t tmp[8];
    for (int j = 0; j < k; ++j) tmp[j] = buf[t * k + j];
    for (int j = 0; j < k; ++j) buf[t * k + perm.p[j]] = tmp[j];
  }
}

int listing_grid(gpm_graph *g, int *blocks) {
  *blocks = gpm_num_sms(g->device) * 4;
  return GPM_OK;
}

int ensure_list_scratch(gpm_graph *g, size_t bytes) {
  if (g->list_scratch_bytes >= bytes) return GPM_OK;
  if (g->list_scratch) {
    cudaFree(g->list_scratch);
    g->device_bytes -= g->list_scratch_bytes;
    g->list_scratch = nullptr;
    g->list_scratch_bytes = 0;
  }
  GPM_TRY(gpm_graph_alloc(g, (void **)&g->list_scratch, bytes));
  g->list_scratch_bytes = bytes;
  return GPM_OK;
}

}  // namespace

int gpm_launch_list_diamond(gpm_graph *g, uint32_t *buf, uint64_t cap, unsigned long long *counter,
                            cudaStream_t st) {
  int blocks;
  listing_grid(g, &blocks);
  const uint64_t warps = (uint64_t)blocks * 8;
  const uint64_t words = std::max<uint64_t>(g->max_degree, 1);
  GPM_TRY(ensure_list_scratch(g, warps * words * 4));
  if (g->n) GPM_LAUNCH("list_diamond_kernel", st, list_diamond_kernel<<<blocks, 256, 0, st>>>(g->rowptr, g->col, g->drow, g->dcol, g->n, buf, cap, counter,
                                                        g->list_scratch, words));
  GPM_CUDA(cudaGetLastError());
  return GPM_OK;
}

int gpm_launch_list_cycle4(gpm_graph *g, uint32_t *buf, uint64_t cap, unsigned long long *counter, cudaStream_t st) {
  int blocks;
  listing_grid(g, &blocks);
  if (g->n) GPM_LAUNCH("list_cycle4_kernel", st, list_cycle4_kernel<<<blocks, 256, 0, st>>>(g->rowptr, g->col, g->n, buf, cap, counter));
  GPM_CUDA(cudaGetLastError());
  return GPM_OK;
}

int gpm_launch_list_cliques(gpm_graph *g, int k, uint32_t *buf, uint64_t cap, unsigned long long *counter,
                            cudaStream_t st) {
  if (k < 3 || k > 8) return gpm_fail(GPM_E_UNSUPPORTED, "clique listing supports k = 3..8");
  int blocks;
  listing_grid(g, &blocks);
  const uint64_t warps = (uint64_t)blocks * 8;
  const uint64_t words = std::max<uint64_t>(g->max_outdeg, 1);
  if (k >= 6) {
    GPM_TRY(ensure_list_scratch(g, warps * (uint64_t)(k - 2) * words * 4));
    if (g->n)
      GPM_LAUNCH("list_cliques_deep_kernel", st,
                 list_cliques_deep_kernel<<<blocks, 256, 0, st>>>(g->drow, g->dcol, g->n, k, buf, cap, counter,
                                                                  g->list_scratch, words));
    GPM_CUDA(cudaGetLastError());
    return GPM_OK;
  }
  GPM_TRY(ensure_list_scratch(g, warps * 3 * words * 4));
  if (g->n) GPM_LAUNCH("list_cliques_kernel", st, list_cliques_kernel<<<blocks, 256, 0, st>>>(g->drow, g->dcol, g->n, k, buf, cap, counter, g->list_scratch,
                                                        words));
  GPM_CUDA(cudaGetLastError());
  return GPM_OK;
}

int gpm_launch_permute_tuples(uint32_t *buf, uint64_t count, int k, const uint32_t *perm, cudaStream_t st) {
  Perm8 p{};
  for (int j = 0; j < k; ++j) p.p[j] = perm[j];
  if (count) GPM_LAUNCH("permute_kernel", st, permute_kernel<<<std::max<uint64_t>(1, std::min<uint64_t>((count + 255) / 256, 4096)), 256, 0, st>>>(
      buf, count, k, p));
  GPM_CUDA(cudaGetLastError());
  return GPM_OK;
}
