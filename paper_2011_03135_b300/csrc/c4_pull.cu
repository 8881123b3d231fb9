// 4-cycles of the roots with the largest wedge bounds, 128 roots per pass.
//
// The count of 4-cycles rooted at v0 (its order-last vertex; order = degree,
// then id) is sum_w C(c(w), 2) over vertices w before v0, where c(w) is the
// number of neighbours x of v0 that precede v0 and are adjacent to w (the
// wedges v0 - x - w; the 4-cycle problem of Section 2, rooted as in the
// symmetry-breaking order of the appendix). For a root whose neighbours'
// lists together hold millions of entries, c(w) is nonzero for most w, so
// instead of walking the wedges of each root (pushing every wedge end into a
// tally) this pass pulls, for up to 128 roots at once:
//
//   * mark: bit r of M[y] (4 words per vertex) is set for every neighbour y
//     of root r that precedes it;
//   * pull: for every vertex w, c_r(w) = number of y in N(w) with bit r of
//     M[y] set (and w before root r), for all 128 r at once with bit-sliced
//     counters: plane j of a lane's counters holds bit j of 32 roots' counts;
//     the words M[y] of 8 entries are summed by a carry-save adder tree and
//     the 4-bit sums added into the planes;
//     sum_r C(c_r(w), 2) is read off the planes with popcounts:
//       C(c, 2) summed over 32 counters
//         = sum_{j>=1} 2^(j-1) (2^j - 1) popc(P_j) + sum_{j<k} 2^(j+k) popc(P_j & P_k);
//   * clear: the marked words are reset to zero.
//
// One pass reads every adjacency list once (the same for any number of
// roots up to 128), where the wedge walk reads every list of every root's
// neighbours. The lists are read from a copy of the CSR in order of
// decreasing degree (built once per graph, 32-bit offsets), so that the
// vertices a warp holds have similar degrees. Vertices of degree <= kTinyMax
// take one lane each (a kernel of their own); for the others, work items are
// taken 8 per warp claim, one per group of 4 lanes (lane l of a group owns
// roots 32l..32l+31): a vertex of degree <= kPullChunk is one item, whose
// counts are finished in registers; a larger vertex is cut into items of
// kPullChunk entries, whose per-root counts are added into a counter row of
// that vertex (128 words in global memory), finished by a third kernel.
#include <algorithm>
#include <vector>

#include "gpm_internal.h"
#include "motif_device.cuh"

namespace {

using gpm_dev::precedes;

constexpr int kPullThreads = 256;
constexpr uint32_t kPullRoots = 128;   // roots per pass (4 words of M per vertex)
constexpr uint32_t kPullChunk = 1024;  // entries per item
constexpr int kPlanes = 11;            // counters up to 2047 >= kPullChunk
constexpr int kBatch = 8;              // entries summed by one carry-save tree
constexpr int kLoad = 16;              // entries loaded together by a lane (main kernel)
constexpr int kPad = 16;               // entries of padding after the last list
constexpr uint32_t kTinyMax = 15;      // vertices of degree <= 15: one per lane, all 128 roots

struct C4PullArgs {
  const uint32_t *__restrict__ deg;
  const uint32_t *__restrict__ ord;    // vertices by decreasing degree
  const uint32_t *__restrict__ prow;   // list of ord[i]: pcol[prow[i], prow[i + 1])
  const uint32_t *__restrict__ pcol;
  const uint2 *__restrict__ chunks;    // items of the large vertices: {position, first entry}
  uint32_t nchunks;                    // ord[0, n_big) are cut into chunks
  uint32_t n_big, n_act;               // ord[0, n_act): degree >= 2
  uint32_t n_tiny;                     // ord[n_tiny, n_act): degree <= kTinyMax
  const uint32_t *__restrict__ M;      // 4 words per vertex
  uint32_t *__restrict__ cntb;         // kPullRoots counters per large vertex (zero)
  const uint32_t *__restrict__ roots;  // the pass's roots
  uint32_t nb;                         // <= kPullRoots
  unsigned int *queue;
  unsigned long long *acc;
  unsigned int *status;
};

// full adder over 32 bit positions: s = a + b + c (mod 2), k = carry
__device__ __forceinline__ void fadd(uint32_t a, uint32_t b, uint32_t c, uint32_t &s, uint32_t &k) {
  s = a ^ b ^ c;
  k = (a & b) | (c & (a ^ b));
}

// adds kBatch = 8 words of one-bit inputs x (bit position b of every word
// belongs to counter b), restricted to the bits of mask, to the bit-sliced
// counters p: a carry-save tree forms the 4-bit sums (b3 b2 b1 b0) of the 8
// inputs per bit position, which are then added into the planes
__device__ __forceinline__ void plane_add8(uint32_t (&p)[kPlanes], const uint32_t (&x)[8], uint32_t mask) {
  uint32_t s1, c1, s2, c2, s3, c3, s5, d1;
  fadd(x[0], x[1], x[2], s1, c1);
  fadd(x[3], x[4], x[5], s2, c2);
  fadd(s1, s2, x[6], s3, c3);
  const uint32_t b0 = (s3 ^ x[7]) & mask, c4 = s3 & x[7];
  fadd(c1, c2, c3, s5, d1);
  const uint32_t b1 = (s5 ^ c4) & mask, d2 = s5 & c4;
  const uint32_t b2 = (d1 ^ d2) & mask, b3 = d1 & d2 & mask;
  uint32_t c = p[0] & b0, t;
  p[0] ^= b0;
  fadd(p[1], b1, c, t, c);
  p[1] = t;
  fadd(p[2], b2, c, t, c);
  p[2] = t;
  fadd(p[3], b3, c, t, c);
  p[3] = t;
#pragma unroll
  for (int j = 4; j < kPlanes; ++j) {
    if (!c) break;
    t = p[j] & c;
    p[j] ^= c;
    c = t;
  }
}

// sum of C(c, 2) over the 32 counters, planes [0, T) nonzero
template <int T>
__device__ __forceinline__ unsigned long long plane_pairs_t(const uint32_t (&p)[kPlanes]) {
  unsigned long long s = 0;
#pragma unroll
  for (int j = 1; j < T; ++j) s += (unsigned long long)(((1u << j) - 1u) << (j - 1)) * (uint32_t)__popc(p[j]);
#pragma unroll
  for (int j = 0; j < T; ++j)
#pragma unroll
    for (int k = j + 1; k < T; ++k) s += (unsigned long long)(uint32_t)__popc(p[j] & p[k]) << (j + k);
  return s;
}

// counters of at most `walked` additions: planes [0, bits(walked))
__device__ __forceinline__ unsigned long long plane_pairs(const uint32_t (&p)[kPlanes], uint32_t walked) {
  switch (32 - __clz(walked)) {
    case 0:
    case 1: return 0;  // every counter <= 1
    case 2: return plane_pairs_t<2>(p);
    case 3: return plane_pairs_t<3>(p);
    case 4: return plane_pairs_t<4>(p);
    case 5: return plane_pairs_t<5>(p);
    case 6: return plane_pairs_t<6>(p);
    case 7: return plane_pairs_t<7>(p);
    case 8: return plane_pairs_t<8>(p);
    case 9: return plane_pairs_t<9>(p);
    case 10: return plane_pairs_t<10>(p);
    default: return plane_pairs_t<11>(p);
  }
}

// bits of lane word lw: roots r = 32 lw + b that w precedes (key order)
__device__ __forceinline__ uint32_t before_mask(const unsigned long long *s_key, unsigned long long minkey,
                                                uint32_t nb, unsigned long long kw, uint32_t lw) {
  if (kw < minkey) return 0xffffffffu;
  uint32_t m = 0;
  for (uint32_t b = 0; b < 32; ++b) {
    const uint32_t r = 32 * lw + b;
    if (r < nb && s_key[r] > kw) m |= 1u << b;
  }
  return m;
}

// adjacency data read once per pass is loaded with an L2 evict-first policy,
// so that the membership words (16 bytes per vertex, gathered once per
// entry) keep their place in L2
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint32_t ld_once(const uint32_t *p, uint64_t pol) {
  uint32_t v;
  asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}

__global__ void __launch_bounds__(kPullThreads, 4) c4_pull_kernel(C4PullArgs a) {
  __shared__ unsigned long long s_key[kPullRoots];
  __shared__ unsigned long long s_min;
  const uint32_t tid = threadIdx.x, lane = tid & 31;
  const uint32_t lw = lane & 3;  // word of M (roots 32 lw .. 32 lw + 31)
  const uint64_t pol = evict_first_policy();
  for (uint32_t r = tid; r < kPullRoots; r += kPullThreads)
    s_key[r] = r < a.nb ? ((unsigned long long)a.deg[a.roots[r]] << 32) | a.roots[r] : ~0ull;
  __syncthreads();
  if (tid == 0) {
    unsigned long long mk = ~0ull;
    for (uint32_t r = 0; r < a.nb; ++r) mk = s_key[r] < mk ? s_key[r] : mk;
    s_min = mk;
  }
  __syncthreads();
  const unsigned long long minkey = s_min;
  const uint32_t nitems = a.nchunks + (a.n_tiny - a.n_big);
  unsigned long long acc = 0;
  bool carry = false;
  for (;;) {
    uint32_t first = 0;
    if (lane == 0) first = atomicAdd(a.queue, 8u);
    first = __shfl_sync(0xffffffffu, first, 0);
    if (first >= nitems) break;
    const uint32_t item = first + (lane >> 2);
    if (item >= nitems) continue;
    // the item's entries [e0, e1) of the list of the vertex at position pos
    uint32_t pos, e0, e1;
    if (item < a.nchunks) {
      const uint2 c = a.chunks[item];
      pos = c.x;
      e0 = c.y;
      const uint32_t end = ld_once(a.prow + pos + 1, pol);
      e1 = end - e0 > kPullChunk ? e0 + kPullChunk : end;
    } else {
      pos = a.n_big + (item - a.nchunks);
      e0 = ld_once(a.prow + pos, pol);
      e1 = ld_once(a.prow + pos + 1, pol);
    }
    const uint32_t w = ld_once(a.ord + pos, pol);
    const uint32_t dw = pos < a.n_big ? a.deg[w] : e1 - e0;
    const uint32_t mask = before_mask(s_key, minkey, a.nb, ((unsigned long long)dw << 32) | w, lw);
    if (!mask) continue;
    uint32_t p[kPlanes];
#pragma unroll
    for (int j = 0; j < kPlanes; ++j) p[j] = 0;
    // batches of kLoad entries; pcol has kPad entries of padding, so the
    // loads past e1 stay in bounds and only their membership words are skipped
    // the next batch's entries are loaded before this batch's words are
    // gathered (software pipelining over the batches of a long list)
    uint32_t yn[kLoad];
#pragma unroll
    for (int i = 0; i < kLoad; ++i) yn[i] = ld_once(a.pcol + e0 + i, pol);
    for (uint32_t e = e0; e < e1; e += kLoad) {
      const uint32_t left = e1 - e;
      uint32_t y[kLoad], m[kBatch], m2[kBatch];
#pragma unroll
      for (int i = 0; i < kLoad; ++i) y[i] = yn[i];
      if (left > kLoad) {
#pragma unroll
        for (int i = 0; i < kLoad; ++i) yn[i] = ld_once(a.pcol + e + kLoad + i, pol);
      }
#pragma unroll
      for (int i = 0; i < kBatch; ++i) m[i] = (uint32_t)i < left ? __ldg(a.M + 4ull * y[i] + lw) : 0u;
#pragma unroll
      for (int i = 0; i < kBatch; ++i)
        m2[i] = (uint32_t)(i + kBatch) < left ? __ldg(a.M + 4ull * y[i + kBatch] + lw) : 0u;
      plane_add8(p, m, mask);
      plane_add8(p, m2, mask);
    }
    if (item >= a.nchunks) {
      acc += plane_pairs(p, e1 - e0);
    } else {
      // a chunk of a large vertex: its per-root counts into the vertex's row
      uint32_t *row = a.cntb + (size_t)pos * kPullRoots + 32 * lw;
      for (uint32_t r = 0; r < 32; ++r) {
        uint32_t c = 0;
#pragma unroll
        for (int j = 0; j < kPlanes; ++j) c |= ((p[j] >> r) & 1u) << j;
        if (c) atomicAdd(row + r, c);
      }
    }
  }
  // per-thread sums are far below 2^64; the warp sums and the accumulator
  // additions are checked
  acc = warp_sum_checked(acc, carry);
  if (lane == 0) acc_add_checked(&a.acc[ACC_C4], acc, carry, a.status, ACC_C4);
}

// 4-bit counters (at most 15 additions): the carry-save sum of 8 inputs added into 4 planes
__device__ __forceinline__ void plane_add8_4(uint32_t (&p)[4], const uint32_t (&x)[8], uint32_t mask) {
  uint32_t s1, c1, s2, c2, s3, c3, s5, d1;
  fadd(x[0], x[1], x[2], s1, c1);
  fadd(x[3], x[4], x[5], s2, c2);
  fadd(s1, s2, x[6], s3, c3);
  const uint32_t b0 = (s3 ^ x[7]) & mask, c4 = s3 & x[7];
  fadd(c1, c2, c3, s5, d1);
  const uint32_t b1 = (s5 ^ c4) & mask, d2 = s5 & c4;
  const uint32_t b2 = (d1 ^ d2) & mask, b3 = d1 & d2 & mask;
  uint32_t c = p[0] & b0, t;
  p[0] ^= b0;
  fadd(p[1], b1, c, t, c);
  p[1] = t;
  fadd(p[2], b2, c, t, c);
  p[2] = t;
  p[3] ^= b3 ^ c;  // no carry out of plane 3: every counter stays <= 15
}

__device__ __forceinline__ unsigned long long pairs4(const uint32_t (&p)[4], uint32_t walked) {
  // plane_pairs_t over 4 planes, read through an 11-plane view
  uint32_t q[kPlanes];
#pragma unroll
  for (int j = 0; j < kPlanes; ++j) q[j] = j < 4 ? p[j] : 0u;
  switch (32 - __clz(walked)) {
    case 0:
    case 1: return 0;
    case 2: return plane_pairs_t<2>(q);
    case 3: return plane_pairs_t<3>(q);
    default: return plane_pairs_t<4>(q);
  }
}

// Vertices of degree 2..kTinyMax (ord[n_tiny, n_act)), one per lane: a warp
// claims 32 consecutive positions (adjacent lists of similar length), each
// lane gathers the whole 16-byte membership word of its entries and keeps
// 4 x 4 planes (all 128 roots); the latency of each vertex's dependent loads
// is shared by 32 vertices instead of 8.
__global__ void __launch_bounds__(kPullThreads, 3) c4_pull_tiny_kernel(C4PullArgs a) {
  __shared__ unsigned long long s_key[kPullRoots];
  __shared__ unsigned long long s_min;
  const uint32_t tid = threadIdx.x, lane = tid & 31;
  const uint64_t pol = evict_first_policy();
  for (uint32_t r = tid; r < kPullRoots; r += kPullThreads)
    s_key[r] = r < a.nb ? ((unsigned long long)a.deg[a.roots[r]] << 32) | a.roots[r] : ~0ull;
  __syncthreads();
  if (tid == 0) {
    unsigned long long mk = ~0ull;
    for (uint32_t r = 0; r < a.nb; ++r) mk = s_key[r] < mk ? s_key[r] : mk;
    s_min = mk;
  }
  __syncthreads();
  const unsigned long long minkey = s_min;
  const uint32_t ntiny = a.n_act - a.n_tiny;
  const uint4 *M4 = reinterpret_cast<const uint4 *>(a.M);
  unsigned long long acc = 0;
  bool carry = false;
  for (;;) {
    uint32_t first = 0;
    if (lane == 0) first = atomicAdd(a.queue + 1, 32u);
    first = __shfl_sync(0xffffffffu, first, 0);
    if (first >= ntiny) break;
    if (first + lane >= ntiny) continue;
    const uint32_t pos = a.n_tiny + first + lane;
    const uint32_t e0 = ld_once(a.prow + pos, pol), e1 = ld_once(a.prow + pos + 1, pol);
    const uint32_t dw = e1 - e0;
    uint32_t mk[4] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu};
    if (((unsigned long long)dw << 32 | 0xffffffffull) >= minkey) {
      // w may follow some roots of the pass: exact key comparisons
      const unsigned long long kw = ((unsigned long long)dw << 32) | ld_once(a.ord + pos, pol);
#pragma unroll
      for (uint32_t k = 0; k < 4; ++k) mk[k] = before_mask(s_key, minkey, a.nb, kw, k);
      if (!(mk[0] | mk[1] | mk[2] | mk[3])) continue;
    }
    uint32_t p[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int j = 0; j < 4; ++j) p[k][j] = 0;
    for (uint32_t e = e0; e < e1; e += kBatch) {
      const uint32_t *src = a.pcol + e;
      const uint32_t left = e1 - e;
      uint32_t y[kBatch];
      uint4 m[kBatch];
#pragma unroll
      for (int i = 0; i < kBatch; ++i) y[i] = ld_once(src + i, pol);
#pragma unroll
      for (int i = 0; i < kBatch; ++i) m[i] = (uint32_t)i < left ? __ldg(M4 + y[i]) : make_uint4(0, 0, 0, 0);
      uint32_t x[kBatch];
#pragma unroll
      for (int i = 0; i < kBatch; ++i) x[i] = m[i].x;
      plane_add8_4(p[0], x, mk[0]);
#pragma unroll
      for (int i = 0; i < kBatch; ++i) x[i] = m[i].y;
      plane_add8_4(p[1], x, mk[1]);
#pragma unroll
      for (int i = 0; i < kBatch; ++i) x[i] = m[i].z;
      plane_add8_4(p[2], x, mk[2]);
#pragma unroll
      for (int i = 0; i < kBatch; ++i) x[i] = m[i].w;
      plane_add8_4(p[3], x, mk[3]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) acc += pairs4(p[k], dw);
  }
  acc = warp_sum_checked(acc, carry);
  if (lane == 0) acc_add_checked(&a.acc[ACC_C4], acc, carry, a.status, ACC_C4);
}

// sum of C(c, 2) over the counter rows of the large vertices, which are
// reset to zero
__global__ void c4_pull_rows_kernel(uint32_t *__restrict__ cntb, uint64_t nwords, unsigned long long *acc,
                                    unsigned int *status) {
  unsigned long long s = 0;
  bool carry = false;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nwords; i += nth) {
    const uint32_t c = cntb[i];
    if (c) {
      s += (unsigned long long)c * (c - 1) / 2;
      cntb[i] = 0;
    }
  }
  s = warp_sum_checked(s, carry);
  if ((threadIdx.x & 31) == 0) acc_add_checked(&acc[ACC_C4], s, carry, status, ACC_C4);
}

// bit r of M[y] for the neighbours y of root r that precede it (set), or the
// same words reset to zero (!set); one CTA per root, roots outside
// [root_lo, root_hi) left out
__global__ void c4_pull_mark_kernel(const uint64_t *__restrict__ rowptr, const uint32_t *__restrict__ col,
                                    const uint32_t *__restrict__ deg, const uint32_t *__restrict__ edeg,
                                    const uint32_t *__restrict__ inv, const uint32_t *__restrict__ roots,
                                    uint32_t root_lo, uint32_t root_hi, uint32_t *__restrict__ M, int set) {
  const uint32_t r = blockIdx.x;
  const uint32_t v0 = roots[r];
  if (v0 < root_lo || v0 >= root_hi) return;
  const uint32_t d0 = deg[v0];
  const uint32_t word = r >> 5, bit = 1u << (r & 31);
  for (uint64_t e = rowptr[v0] + threadIdx.x; e < rowptr[v0 + 1]; e += blockDim.x) {
    const uint32_t y = col[e];
    if (!precedes(edeg[e], y, d0, v0)) continue;
    const uint32_t q = inv[y];
    if (set) atomicOr(&M[4ull * q + word], bit);
    else M[4ull * q + word] = 0u;
  }
}

// position of every vertex in the order ord
__global__ void c4_pull_inv_kernel(const uint32_t *__restrict__ ord, uint32_t n, uint32_t *__restrict__ inv) {
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += nth) inv[ord[i]] = (uint32_t)i;
}

// vertices by decreasing degree: a histogram of the degrees, then a scatter
// with one atomic per group of lanes holding the same degree
__global__ void c4_deg_hist_kernel(const uint32_t *__restrict__ deg, uint32_t n, uint32_t *__restrict__ hist) {
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += nth) atomicAdd(&hist[deg[v]], 1u);
}

__global__ void c4_deg_scatter_kernel(const uint32_t *__restrict__ deg, uint32_t n, uint32_t *__restrict__ cursor,
                                      uint32_t *__restrict__ ord) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t base = blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u); base < n; base += nth) {
    const uint64_t v = base + lane;
    const bool on = v < n;
    const uint32_t d = on ? deg[v] : 0xffffffffu;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const int leader = __ffs(peers) - 1;
    uint32_t at = 0;
    if ((int)lane == leader && on) at = atomicAdd(&cursor[d], (uint32_t)__popc(peers));
    at = __shfl_sync(0xffffffffu, at, leader);
    if (on) ord[at + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)v;
  }
}

// the CSR in the order ord (positions [0, n_act)): prow[i] = base[d] + (i -
// first[d]) d for the vertex of degree d at position i (positions of equal
// degree are consecutive), and its list copied to pcol[prow[i] ..]; one warp
// per position
__global__ void c4_pull_csr_kernel(const uint64_t *__restrict__ rowptr, const uint32_t *__restrict__ col,
                                   const uint32_t *__restrict__ deg, const uint32_t *__restrict__ ord,
                                   const uint32_t *__restrict__ inv, uint32_t n_act, const uint32_t *__restrict__ first,
                                   const uint64_t *__restrict__ base, uint32_t *__restrict__ prow,
                                   uint32_t *__restrict__ pcol) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = warp; i < n_act; i += nwarps) {
    const uint32_t w = ord[i];
    const uint32_t d = deg[w];
    const uint64_t at = base[d] + (i - first[d]) * (uint64_t)d;
    if (lane == 0) {
      prow[i] = (uint32_t)at;
      if (i + 1 == n_act) prow[n_act] = (uint32_t)(at + d);
    }
    const uint64_t src = rowptr[w];
    for (uint32_t k = lane; k < d; k += 32) pcol[at + k] = inv[col[src + k]];
  }
}

}  // namespace

// vertices by decreasing degree and their lists in that order, the chunks of
// the large vertices, the membership words and counter rows (zero) and the
// queue counters; built once per graph (the graph's nnz is below 2^32 on
// this path)
static int ensure_c4_pull(gpm_graph *g, uint32_t npass, cudaStream_t st) {
  const size_t nw = std::max<uint32_t>(g->n, 1);
  if (!g->c4q_ord) {
    GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4q_ord, sizeof(uint32_t) * nw));
    const uint32_t nbin = g->max_degree + 1;
    uint32_t *hist = nullptr;
    GPM_TRY(gpm_graph_alloc(g, (void **)&hist, sizeof(uint32_t) * nbin));
    GPM_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * nbin, st));
    const int blocks = gpm_num_sms(g->device) * 8;
    if (g->n) {
      GPM_LAUNCH("c4_deg_hist_kernel", st, c4_deg_hist_kernel<<<blocks, 256, 0, st>>>(g->deg, g->n, hist));
      GPM_CUDA(cudaGetLastError());
    }
    std::vector<uint32_t> h(nbin);
    GPM_CUDA(cudaMemcpyAsync(h.data(), hist, sizeof(uint32_t) * nbin, cudaMemcpyDeviceToHost, st));
    GPM_CUDA(cudaStreamSynchronize(st));
    // cur[d] = vertices of degree > d (the first position of degree d),
    // base[d] = entries of the vertices of degree > d
    std::vector<uint32_t> cur(nbin);
    std::vector<uint64_t> base(nbin);
    uint32_t above = 0;
    uint64_t ent = 0;
    for (uint32_t d = nbin; d-- > 0;) {
      cur[d] = above;
      base[d] = ent;
      above += h[d];
      ent += (uint64_t)h[d] * d;
    }
    g->c4q_nbig = nbin > kPullChunk + 1 ? cur[kPullChunk] : 0;
    g->c4q_nact = nbin > 2 ? cur[1] : 0;
    g->c4q_ntiny = nbin > kTinyMax ? cur[kTinyMax] : 0;
    const uint64_t pnnz = nbin > 2 ? base[1] : 0;
    // chunks of the vertices of degree > kPullChunk, in position order
    std::vector<uint2> chunks;
    for (uint32_t d = nbin; d-- > kPullChunk + 1;)
      for (uint32_t i = cur[d]; i < cur[d] + h[d]; ++i)
        for (uint32_t off = 0; off < d; off += kPullChunk)
          chunks.push_back(make_uint2(i, (uint32_t)(base[d] + (uint64_t)(i - cur[d]) * d + off)));
    uint64_t *dbase = nullptr;
    GPM_TRY(gpm_graph_alloc(g, (void **)&dbase, sizeof(uint64_t) * nbin));
    GPM_CUDA(cudaMemcpyAsync(dbase, base.data(), sizeof(uint64_t) * nbin, cudaMemcpyHostToDevice, st));
    GPM_CUDA(cudaMemcpyAsync(hist, cur.data(), sizeof(uint32_t) * nbin, cudaMemcpyHostToDevice, st));
    if (g->n) {
      GPM_LAUNCH("c4_deg_scatter_kernel", st, c4_deg_scatter_kernel<<<blocks, 256, 0, st>>>(g->deg, g->n, hist,
                                                                                            g->c4q_ord));
      GPM_CUDA(cudaGetLastError());
    }
    // the scatter advanced every cursor to the end of its degree's
    // positions: reload the first positions
    GPM_CUDA(cudaMemcpyAsync(hist, cur.data(), sizeof(uint32_t) * nbin, cudaMemcpyHostToDevice, st));
    GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4q_inv, sizeof(uint32_t) * nw));
    if (g->n) {
      GPM_LAUNCH("c4_pull_inv_kernel", st, c4_pull_inv_kernel<<<blocks, 256, 0, st>>>(g->c4q_ord, g->n, g->c4q_inv));
      GPM_CUDA(cudaGetLastError());
    }
    GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4q_prow, sizeof(uint32_t) * ((size_t)g->c4q_nact + 1)));
    GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4q_pcol, sizeof(uint32_t) * (pnnz + kPad)));
    GPM_CUDA(cudaMemsetAsync(g->c4q_pcol + pnnz, 0, sizeof(uint32_t) * kPad, st));
    GPM_CUDA(cudaMemsetAsync(g->c4q_prow, 0, sizeof(uint32_t), st));
    if (g->c4q_nact) {
      GPM_LAUNCH("c4_pull_csr_kernel", st,
                 c4_pull_csr_kernel<<<blocks, 256, 0, st>>>(g->rowptr, g->col, g->deg, g->c4q_ord, g->c4q_inv,
                                                            g->c4q_nact, hist, dbase, g->c4q_prow, g->c4q_pcol));
      GPM_CUDA(cudaGetLastError());
    }
    g->c4q_nchunks = (uint32_t)chunks.size();
    GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4q_chunks, sizeof(uint2) * std::max<size_t>(chunks.size(), 1)));
    if (!chunks.empty())
      GPM_CUDA(cudaMemcpyAsync(g->c4q_chunks, chunks.data(), sizeof(uint2) * chunks.size(), cudaMemcpyHostToDevice,
                               st));
    const size_t rows = sizeof(uint32_t) * kPullRoots * std::max<size_t>(g->c4q_nbig, 1);
    GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4q_cntb, rows));
    GPM_CUDA(cudaMemsetAsync(g->c4q_cntb, 0, rows, st));
    GPM_CUDA(cudaStreamSynchronize(st));
    cudaFree(hist);
    cudaFree(dbase);
    g->device_bytes -= sizeof(uint32_t) * nbin + sizeof(uint64_t) * nbin;
  }
  if (!g->c4q_M) {
    GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4q_M, 4 * sizeof(uint32_t) * nw));
    GPM_CUDA(cudaMemsetAsync(g->c4q_M, 0, 4 * sizeof(uint32_t) * nw, st));
  }
  if (g->c4q_queue_words < 2 * npass) {
    if (g->c4q_queue) {
      cudaFree(g->c4q_queue);
      g->device_bytes -= sizeof(unsigned int) * g->c4q_queue_words;
      g->c4q_queue = nullptr;
      g->c4q_queue_words = 0;
    }
    GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4q_queue, sizeof(unsigned int) * 2 * npass));
    g->c4q_queue_words = 2 * npass;
  }
  return GPM_OK;
}

int gpm_c4_pull_prepare(gpm_graph *g, const std::vector<uint32_t> &roots, cudaStream_t st) {
  const uint32_t npass = (uint32_t)((roots.size() + kPullRoots - 1) / kPullRoots);
  g->c4q_hroots = roots;
  if (roots.empty()) return GPM_OK;
  GPM_TRY(ensure_c4_pull(g, npass, st));
  if (g->c4q_roots_cap < roots.size()) {
    if (g->c4q_roots) {
      cudaFree(g->c4q_roots);
      g->device_bytes -= sizeof(uint32_t) * g->c4q_roots_cap;
      g->c4q_roots = nullptr;
      g->c4q_roots_cap = 0;
    }
    GPM_TRY(gpm_graph_alloc(g, (void **)&g->c4q_roots, sizeof(uint32_t) * roots.size()));
    g->c4q_roots_cap = roots.size();
  }
  GPM_CUDA(cudaMemcpyAsync(g->c4q_roots, roots.data(), sizeof(uint32_t) * roots.size(), cudaMemcpyHostToDevice, st));
  GPM_CUDA(cudaStreamSynchronize(st));
  return GPM_OK;
}

int gpm_launch_c4_pull(gpm_graph *g, uint32_t root_lo, uint32_t root_hi, unsigned long long *acc, cudaStream_t st) {
  const std::vector<uint32_t> &hr = g->c4q_hroots;
  if (hr.empty()) return GPM_OK;
  const uint32_t npass = (uint32_t)((hr.size() + kPullRoots - 1) / kPullRoots);
  GPM_CUDA(cudaMemsetAsync(g->c4q_queue, 0, sizeof(unsigned int) * 2 * npass, st));
  int per_sm = 0, per_sm_tiny = 0;
  GPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c4_pull_kernel, kPullThreads, 0));
  GPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_tiny, c4_pull_tiny_kernel, kPullThreads, 0));
  const int sms = gpm_num_sms(g->device);
  const unsigned blocks = (unsigned)sms * (unsigned)std::max(per_sm, 1);
  const unsigned blocks_tiny = (unsigned)sms * (unsigned)std::max(per_sm_tiny, 1);
  unsigned int *status = reinterpret_cast<unsigned int *>(g->work + WK_STATUS);
  for (uint32_t p = 0; p < npass; ++p) {
    const uint32_t r0 = p * kPullRoots;
    const uint32_t nb = std::min<uint32_t>(kPullRoots, (uint32_t)hr.size() - r0);
    bool any = false;
    for (uint32_t i = r0; i < r0 + nb && !any; ++i) any = hr[i] >= root_lo && hr[i] < root_hi;
    if (!any) continue;  // no root of this pass in the requested range
    const uint32_t *roots = g->c4q_roots + r0;
    GPM_LAUNCH("c4_pull_mark_kernel", st,
               c4_pull_mark_kernel<<<nb, 256, 0, st>>>(g->rowptr, g->col, g->deg, g->edeg, g->c4q_inv, roots,
                                                       root_lo, root_hi, g->c4q_M, 1));
    GPM_CUDA(cudaGetLastError());
    C4PullArgs a{};
    a.deg = g->deg;
    a.ord = g->c4q_ord;
    a.prow = g->c4q_prow;
    a.pcol = g->c4q_pcol;
    a.chunks = reinterpret_cast<const uint2 *>(g->c4q_chunks);
    a.nchunks = g->c4q_nchunks;
    a.n_big = g->c4q_nbig;
    a.n_act = g->c4q_nact;
    a.n_tiny = g->c4q_ntiny;
    a.M = g->c4q_M;
    a.cntb = g->c4q_cntb;
    a.roots = roots;
    a.nb = nb;
    a.queue = g->c4q_queue + 2 * p;
    a.acc = acc;
    a.status = status;
    if (a.nchunks + (a.n_tiny - a.n_big)) {
      GPM_LAUNCH("c4_pull_kernel", st, c4_pull_kernel<<<blocks, kPullThreads, 0, st>>>(a));
      GPM_CUDA(cudaGetLastError());
    }
    if (a.n_act > a.n_tiny) {
      GPM_LAUNCH("c4_pull_tiny_kernel", st, c4_pull_tiny_kernel<<<blocks_tiny, kPullThreads, 0, st>>>(a));
      GPM_CUDA(cudaGetLastError());
    }
    if (g->c4q_nbig) {
      const uint64_t nwords = (uint64_t)g->c4q_nbig * kPullRoots;
      const unsigned rb = (unsigned)std::min<uint64_t>((nwords + 255) / 256, (uint64_t)sms * 8);
      GPM_LAUNCH("c4_pull_rows_kernel", st,
                 c4_pull_rows_kernel<<<rb, 256, 0, st>>>(g->c4q_cntb, nwords, acc, status));
      GPM_CUDA(cudaGetLastError());
    }
    GPM_LAUNCH("c4_pull_mark_kernel", st,
               c4_pull_mark_kernel<<<nb, 256, 0, st>>>(g->rowptr, g->col, g->deg, g->edeg, g->c4q_inv, roots,
                                                       root_lo, root_hi, g->c4q_M, 0));
    GPM_CUDA(cudaGetLastError());
  }
  return GPM_OK;
}
