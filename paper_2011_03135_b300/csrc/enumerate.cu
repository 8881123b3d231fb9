// Pattern-oblivious enumeration of connected k-vertex induced subgraphs
// (k = 3, 4, 5) with classification by connectivity code.
//
// This is the paper's high-level path for k-motif counting without local
// counting (Section 4.2 "Memoization of Embedding Connectivity" and the
// appendix "Example for Connectivity Code"; k-MC as defined in Section 2):
// embeddings are grown by vertex extension, every vertex added at level l
// carries a connectivity code of l bits (bit i set when it is adjacent to the
// vertex added at level i), and the concatenation of the codes of a complete
// embedding (1 + 2 + ... + (k-1) bits) identifies its pattern through a table
// built once on the host.
//
// Each connected k-set is generated exactly once by the extension rule of
// ESU (Wernicke, "Efficient detection of network motifs", IEEE/ACM TCBB 2006):
// the set's smallest vertex v is its root; a candidate list holds vertices
// larger than v that are neighbours of the set; choosing candidate w keeps the
// candidates after w and adds the neighbours of w that are larger than v and
// adjacent to no earlier member (their code is the single bit of w). The
// codes of carried-over candidates gain one bit (adjacency to w), so the
// connectivity of every candidate to the whole embedding is known without
// looking it up again -- the memoization the paper describes.
//
// GPU mapping: a work item is a first extension, i.e. an arc (v, w1) with
// w1 > v; warps claim chunks of adjacency positions from a global counter.
// A warp walks the item's subtree depth first: lanes share the work of one
// extension (candidates carried over in parallel, neighbours of w filtered in
// parallel and compacted with a ballot). The last level is not stored: each
// lane forms the full code of its leaf and the warp adds equal codes with one
// shared-memory atomic per distinct code into a per-CTA histogram over all
// codes, flushed to the class counts when the CTA finishes.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "gpm_internal.h"

namespace {

constexpr int kEnumThreads = 256;
constexpr uint32_t kEnumChunk = 32;  // adjacency positions claimed at a time by a warp

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

// Leaves of the warp: lanes with `valid` add code `full` to the histogram,
// one shared-memory atomic per distinct code.
__device__ __forceinline__ void count_leaves(unsigned long long *hist, bool valid, uint32_t full) {
  const unsigned act = __ballot_sync(0xffffffffu, valid);
  if (!valid) return;
  const unsigned grp = __match_any_sync(act, full);
  if ((threadIdx.x & 31) == (uint32_t)(__ffs(grp) - 1)) atomicAdd(&hist[full], (unsigned long long)__popc(grp));
}

struct EnumArgs {
  const uint64_t *__restrict__ rowptr;
  const uint32_t *__restrict__ col;
  uint32_t n;
  uint32_t root_lo, root_hi;       // roots (smallest vertices) counted
  unsigned long long *queue;       // adjacency positions claimed so far
  uint32_t *scratch;               // per warp: candidate lists E2, E3 (vertices), codes after them
  uint64_t warp_words;             // words of scratch per warp
  uint64_t cap2, cap3;             // capacities of E2 and E3
  const uint8_t *__restrict__ cls; // class of every full code (255: none)
  unsigned long long *counts;      // per class
  unsigned int *status;
};

// Candidates for level l + 1 after choosing w = E[i] at level l: the
// candidates after i with one more code bit (part A), then the neighbours
// of w that are larger than v, are not members and are adjacent to no
// earlier member (part B, code = bit l). `excl` tests the earlier members.
// At the last level the leaves are counted instead of stored.
template <int K, int L, typename Excl>
__device__ __forceinline__ uint32_t extend(const EnumArgs &a, uint32_t v, uint32_t w, const uint32_t *E,
                                           const uint8_t *C, uint32_t i, uint32_t nE, uint32_t *E2, uint8_t *C2,
                                           uint32_t sub_code, unsigned long long *hist, Excl excl) {
  const uint32_t lane = threadIdx.x & 31;
  constexpr uint32_t off = L * (L + 1) / 2;  // bits of the codes of levels 1 .. L (the leaf's code follows)
  constexpr bool leaf = (L + 1 == K - 1);  // the candidates complete k-vertex sets (vertex levels 0 .. K-1)
  uint32_t n2 = 0;
  // part A: order kept, every candidate carried over
  for (uint32_t t0 = i + 1; t0 < nE; t0 += 32) {
    const uint32_t t = t0 + lane;
    bool valid = false;
    uint32_t code = 0, u = 0;
    if (t < nE) {
      u = E[t];
      code = (uint32_t)C[t] | ((uint32_t)adjacent(a.rowptr, a.col, w, u) << L);
      valid = true;
    }
    if (leaf) {
      count_leaves(hist, valid, sub_code | (code << off));
    } else if (valid) {
      E2[t - (i + 1)] = u;
      C2[t - (i + 1)] = (uint8_t)code;
    }
  }
  if (!leaf) n2 = nE - (i + 1);
  // part B: exclusive neighbours of w
  const uint64_t b = a.rowptr[w], e = a.rowptr[w + 1];
  for (uint64_t p0 = b; p0 < e; p0 += 32) {
    const uint64_t p = p0 + lane;
    bool keep = false;
    if (p < e) {
      const uint32_t u = __ldg(a.col + p);
      keep = u > v && excl(u);
    }
    if (leaf) {
      count_leaves(hist, keep, sub_code | ((1u << L) << off));
    } else {
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const uint32_t pos = n2 + __popc(m & ((1u << lane) - 1u));
        E2[pos] = __ldg(a.col + p);
        C2[pos] = (uint8_t)(1u << L);
      }
      n2 += __popc(m);
    }
  }
  __syncwarp();
  return n2;
}

template <int K>
__global__ void __launch_bounds__(kEnumThreads) enum_kernel(EnumArgs a) {
  constexpr uint32_t kCodes = 1u << (K * (K - 1) / 2);
  __shared__ unsigned long long hist[kCodes];
  for (uint32_t i = threadIdx.x; i < kCodes; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t gw = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  uint32_t *E2 = a.scratch + gw * a.warp_words;
  uint32_t *E3 = E2 + a.cap2;
  uint8_t *C2 = reinterpret_cast<uint8_t *>(E3 + a.cap3);
  uint8_t *C3 = C2 + a.cap2;
  // items: the adjacency positions of the roots in [root_lo, root_hi)
  const uint64_t qbase = a.rowptr[a.root_lo], qend = a.rowptr[a.root_hi];
  for (;;) {
    unsigned long long p0 = 0;
    if (lane == 0) p0 = qbase + atomicAdd(a.queue, (unsigned long long)kEnumChunk);
    p0 = __shfl_sync(0xffffffffu, p0, 0);
    if (p0 >= qend) break;
    const uint64_t p1 = min((uint64_t)p0 + kEnumChunk, qend);
    // row of position p0
    uint32_t v;
    {
      uint32_t lo = 0, hi = a.n;  // largest v with rowptr[v] <= p0
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a.rowptr[mid] <= p0) lo = mid;
        else hi = mid;
      }
      v = lo;
    }
    for (uint64_t p = p0; p < p1; ++p) {
      while (a.rowptr[v + 1] <= p) ++v;
      const uint32_t w1 = __ldg(a.col + p);
      if (w1 <= v) continue;
      // level 2 candidates: N(v) after w1 (code: adjacent to v, and to w1 or
      // not), then neighbours of w1 above v that are not adjacent to v
      const uint64_t ve = a.rowptr[v + 1];
      uint32_t n2 = 0;
      constexpr bool leaf2 = (K == 3);
      for (uint64_t t0 = p + 1; t0 < ve; t0 += 32) {
        const uint64_t t = t0 + lane;
        bool valid = false;
        uint32_t code = 0, u = 0;
        if (t < ve) {
          u = __ldg(a.col + t);
          code = 1u | ((uint32_t)adjacent(a.rowptr, a.col, w1, u) << 1);
          valid = true;
        }
        if (leaf2) {
          count_leaves(hist, valid, 1u | (code << 1));
        } else if (valid) {
          E2[t - (p + 1)] = u;
          C2[t - (p + 1)] = (uint8_t)code;
        }
      }
      if (!leaf2) n2 = (uint32_t)(ve - (p + 1));
      {
        const uint64_t b = a.rowptr[w1], e = a.rowptr[w1 + 1];
        for (uint64_t q0 = b; q0 < e; q0 += 32) {
          const uint64_t q = q0 + lane;
          bool keep = false;
          uint32_t u = 0;
          if (q < e) {
            u = __ldg(a.col + q);
            keep = u > v && !adjacent(a.rowptr, a.col, v, u);
          }
          if (leaf2) {
            count_leaves(hist, keep, 1u | (2u << 1));
          } else {
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) {
              const uint32_t pos = n2 + __popc(m & ((1u << lane) - 1u));
              E2[pos] = u;
              C2[pos] = 2u;
            }
            n2 += __popc(m);
          }
        }
      }
      __syncwarp();
      if (K == 3) continue;
      // level 3: choose w2 among E2
      for (uint32_t i2 = 0; i2 < n2; ++i2) {
        const uint32_t w2 = E2[i2];
        const uint32_t s2 = 1u | ((uint32_t)C2[i2] << 1);  // codes of levels 1, 2
        auto excl2 = [&](uint32_t u) {
          return u != w1 && !adjacent(a.rowptr, a.col, v, u) && !adjacent(a.rowptr, a.col, w1, u);
        };
        if (K == 4) {
          extend<K, 2>(a, v, w2, E2, C2, i2, n2, E3, C3, s2, hist, excl2);
          continue;
        }
        const uint32_t n3 = extend<K, 2>(a, v, w2, E2, C2, i2, n2, E3, C3, s2, hist, excl2);
        for (uint32_t i3 = 0; i3 < n3; ++i3) {
          const uint32_t w3 = E3[i3];
          const uint32_t s3 = s2 | ((uint32_t)C3[i3] << 3);  // codes of levels 1, 2, 3
          auto excl3 = [&](uint32_t u) {
            return u != w1 && u != w2 && !adjacent(a.rowptr, a.col, v, u) && !adjacent(a.rowptr, a.col, w1, u) &&
                   !adjacent(a.rowptr, a.col, w2, u);
          };
          extend<K, 3>(a, v, w3, E3, C3, i3, n3, E3, C3, s3, hist, excl3);  // leaf level: nothing is stored
        }
      }
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < kCodes; i += blockDim.x) {
    const unsigned long long c = hist[i];
    if (c && a.cls[i] != 255) acc_add_checked(&a.counts[a.cls[i]], c, false, a.status, -1);
  }
}

// ---------------------------------------------------------------------------
// host: class tables
// ---------------------------------------------------------------------------
// A k-vertex graph (k <= 5) is held as a pair mask: bit pair_index(i, j) for
// the edge {i, j}, pairs (0,1), (0,2), ..., (k-2,k-1) in lexicographic order.
// Its class is its smallest pair mask over all vertex orders; classes of
// connected graphs are numbered by edge count, then by that smallest mask.
uint32_t pair_index(uint32_t k, uint32_t i, uint32_t j) {
  if (i > j) std::swap(i, j);
  uint32_t idx = 0;
  for (uint32_t r = 0; r < i; ++r) idx += k - 1 - r;
  return idx + (j - i - 1);
}

uint32_t smallest_mask(uint32_t k, uint32_t mask) {
  uint32_t perm[5] = {0, 1, 2, 3, 4};
  uint32_t best = 0xffffffffu;
  do {
    uint32_t m = 0;
    for (uint32_t i = 0; i < k; ++i)
      for (uint32_t j = i + 1; j < k; ++j)
        if (mask >> pair_index(k, i, j) & 1u) m |= 1u << pair_index(k, perm[i], perm[j]);
    best = std::min(best, m);
  } while (std::next_permutation(perm, perm + k));
  return best;
}

bool mask_connected(uint32_t k, uint32_t mask) {
  uint32_t reach = 1u;
  for (uint32_t round = 0; round < k; ++round)
    for (uint32_t i = 0; i < k; ++i)
      for (uint32_t j = 0; j < k; ++j)
        if (i != j && (reach >> i & 1u) && (mask >> pair_index(k, i, j) & 1u)) reach |= 1u << j;
  return reach == (1u << k) - 1u;
}

struct ClassTable {
  std::vector<uint32_t> class_mask;  // smallest pair mask of each class, in class order
  std::vector<uint8_t> by_code;      // concatenated connectivity code -> class (255: disconnected)
};

const ClassTable &class_table(uint32_t k) {
  static ClassTable tables[6];
  static std::once_flag once[6];
  std::call_once(once[k], [k] {
    ClassTable &t = tables[k];
    const uint32_t L = k * (k - 1) / 2;
    std::vector<uint32_t> canon(1u << L);
    for (uint32_t m = 0; m < (1u << L); ++m) {
      canon[m] = mask_connected(k, m) ? smallest_mask(k, m) : 0xffffffffu;
      if (canon[m] == m) t.class_mask.push_back(m);
    }
    std::stable_sort(t.class_mask.begin(), t.class_mask.end(), [](uint32_t x, uint32_t y) {
      return __builtin_popcount(x) != __builtin_popcount(y) ? __builtin_popcount(x) < __builtin_popcount(y) : x < y;
    });
    // concatenated code: vertex j's code (bit i = adjacent to vertex i < j)
    // at bits j(j-1)/2 .. j(j-1)/2 + j - 1
    t.by_code.assign(1u << L, 255);
    for (uint32_t c = 0; c < (1u << L); ++c) {
      uint32_t m = 0;
      for (uint32_t j = 1; j < k; ++j)
        for (uint32_t i = 0; i < j; ++i)
          if (c >> (j * (j - 1) / 2 + i) & 1u) m |= 1u << pair_index(k, i, j);
      if (canon[m] == 0xffffffffu) continue;
      for (size_t q = 0; q < t.class_mask.size(); ++q)
        if (t.class_mask[q] == canon[m]) t.by_code[c] = (uint8_t)q;
    }
  });
  return tables[k];
}

uint32_t pattern_mask(const gpm_pattern &p) {
  uint32_t m = 0;
  for (uint32_t i = 0; i < p.k; ++i)
    for (uint32_t j = i + 1; j < p.k; ++j)
      if (p.adj[i * p.k + j]) m |= 1u << pair_index(p.k, i, j);
  return m;
}

__global__ void enum_finalize_kernel(EnumFinalize spec, const unsigned long long *__restrict__ cnt,
                                     unsigned long long *__restrict__ out, unsigned int *__restrict__ status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  bool over = false;
  for (uint32_t i = 0; i < spec.npat; ++i) {
    unsigned long long s = 0;
    for (uint32_t c = 0; c < spec.nclass; ++c) {
      const unsigned long long f = spec.coef[i][c];
      if (!f) continue;
      const unsigned long long x = cnt[c];
      const unsigned long long hi = __umul64hi(x, f), lo = x * f;
      over |= hi != 0 || s + lo < s;
      s += lo;
    }
    out[spec.slot[i]] = s;
  }
  if (over) atomicOr(status, ST_CAPACITY);
}

}  // namespace

int gpm_enum_classes(uint32_t k, uint32_t *class_mask, uint32_t cap) {
  if (k < 3 || k > 5) return 0;
  const ClassTable &t = class_table(k);
  for (size_t i = 0; i < t.class_mask.size() && i < cap; ++i) class_mask[i] = t.class_mask[i];
  return (int)t.class_mask.size();
}

uint32_t gpm_enum_pair_index(uint32_t k, uint32_t i, uint32_t j) { return pair_index(k, i, j); }

int gpm_enum_class_of(const gpm_pattern &p) {
  if (p.k < 3 || p.k > 5) return -1;
  const ClassTable &t = class_table(p.k);
  const uint32_t want = smallest_mask(p.k, pattern_mask(p));
  for (size_t c = 0; c < t.class_mask.size(); ++c)
    if (t.class_mask[c] == want) return (int)c;
  return -1;
}

int gpm_enum_coefficients(const gpm_pattern &p, uint16_t *coef, uint32_t *nclass) {
  if (p.k < 3 || p.k > 5) return gpm_fail(GPM_E_UNSUPPORTED, "pattern-oblivious enumeration covers k = 3, 4, 5");
  const ClassTable &t = class_table(p.k);
  *nclass = (uint32_t)t.class_mask.size();
  const uint32_t want = smallest_mask(p.k, pattern_mask(p));
  for (size_t c = 0; c < t.class_mask.size(); ++c) {
    uint32_t f = 0;
    const uint32_t cm = t.class_mask[c];
    if (p.induced) {
      f = (cm == want) ? 1u : 0u;
    } else {
      // spanning subgraphs of the class graph isomorphic to the pattern: its
      // non-induced copies inside one vertex set of that class
      for (uint32_t s = cm;; s = (s - 1) & cm) {
        if ((uint32_t)__builtin_popcount(s) == p.info.n_edges && mask_connected(p.k, s) && smallest_mask(p.k, s) == want)
          ++f;
        if (s == 0) break;
      }
    }
    coef[c] = (uint16_t)f;
  }
  return GPM_OK;
}

int gpm_launch_enumerate(gpm_graph *g, uint32_t k, uint32_t root_lo, uint32_t root_hi, unsigned long long *counts,
                         cudaStream_t st) {
  if (k < 3 || k > 5) return gpm_fail(GPM_E_UNSUPPORTED, "pattern-oblivious enumeration covers k = 3, 4, 5");
  const ClassTable &t = class_table(k);
  const uint32_t L = k * (k - 1) / 2;
  if (!g->enum_cls[k]) {
    GPM_TRY(gpm_graph_alloc(g, (void **)&g->enum_cls[k], 1u << L));
    GPM_CUDA(cudaMemcpyAsync(g->enum_cls[k], t.by_code.data(), 1u << L, cudaMemcpyHostToDevice, st));
  }
  GPM_CUDA(cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * 32, st));
  if (g->nnz == 0 || root_lo >= root_hi) return GPM_OK;
  int per_sm = 0;
  cudaError_t e;
  if (k == 3) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, enum_kernel<3>, kEnumThreads, 0);
  else if (k == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, enum_kernel<4>, kEnumThreads, 0);
  else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, enum_kernel<5>, kEnumThreads, 0);
  GPM_CUDA(e);
  const uint32_t blocks = (uint32_t)gpm_num_sms(g->device) * (uint32_t)std::max(per_sm, 1);
  const uint64_t warps = (uint64_t)blocks * (kEnumThreads / 32);
  // candidate lists: E2 <= d(v) + d(w1), E3 <= |E2| + d(w2)
  const uint64_t cap2 = 2ull * g->max_degree + 32, cap3 = 3ull * g->max_degree + 32;
  const uint64_t warp_words = cap2 + cap3 + (cap2 + cap3 + 3) / 4;
  const size_t need = sizeof(uint32_t) * warps * warp_words;
  if (g->enum_scratch_bytes < need) {
    if (g->enum_scratch) {
      cudaFree(g->enum_scratch);
      g->device_bytes -= g->enum_scratch_bytes;
      g->enum_scratch = nullptr;
      g->enum_scratch_bytes = 0;
    }
    GPM_TRY(gpm_graph_alloc(g, (void **)&g->enum_scratch, need));
    g->enum_scratch_bytes = need;
  }
  unsigned long long *queue = reinterpret_cast<unsigned long long *>(g->work + WK_MISC) + 6;
  GPM_CUDA(cudaMemsetAsync(queue, 0, sizeof(unsigned long long), st));
  EnumArgs a{};
  a.rowptr = g->rowptr;
  a.col = g->col;
  a.n = g->n;
  a.root_lo = root_lo;
  a.root_hi = root_hi;
  a.queue = queue;
  a.scratch = g->enum_scratch;
  a.warp_words = warp_words;
  a.cap2 = cap2;
  a.cap3 = cap3;
  a.cls = g->enum_cls[k];
  a.counts = counts;
  a.status = reinterpret_cast<unsigned int *>(g->work + WK_STATUS);
  if (k == 3) GPM_LAUNCH("enum_kernel_k3", st, enum_kernel<3><<<blocks, kEnumThreads, 0, st>>>(a));
  else if (k == 4) GPM_LAUNCH("enum_kernel_k4", st, enum_kernel<4><<<blocks, kEnumThreads, 0, st>>>(a));
  else GPM_LAUNCH("enum_kernel_k5", st, enum_kernel<5><<<blocks, kEnumThreads, 0, st>>>(a));
  GPM_CUDA(cudaGetLastError());
  return GPM_OK;
}

int gpm_launch_enum_finalize(const EnumFinalize &spec, const unsigned long long *cnt, unsigned long long *out,
                             unsigned int *status, cudaStream_t st) {
  GPM_LAUNCH("enum_finalize_kernel", st, enum_finalize_kernel<<<1, 32, 0, st>>>(spec, cnt, out, status));
  GPM_CUDA(cudaGetLastError());
  return GPM_OK;
}
