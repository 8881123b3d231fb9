// Device building blocks of the local-graph clique search, shared by the
// per-class kernels (clique.cu) and the batched persistent kernel (batch.cu).
// See clique.cu for the method.
#pragma once

#include <stdint.h>

namespace gpm_dev {

__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t *a, uint32_t n, uint32_t x) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// largest i in [0, n) with pre[i] <= f (pre ascending, pre[0] = 0 <= f)
__device__ __forceinline__ uint32_t row_of(const uint32_t *pre, uint32_t n, uint32_t f) {
  uint32_t lo = 0, hi = n;  // invariant: pre[lo] <= f, answer in [lo, hi)
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (pre[mid] <= f) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Flat expansion of one root's local graph. Threads [t0, t0 + nt) of the
// calling group cooperate; the caller synchronises before and after.
template <bool SCATTER>
__device__ __forceinline__ uint32_t build_rows(const uint32_t *__restrict__ dcol, uint32_t *t_edge, const uint32_t *L,
                                               const uint32_t *pre,
                                               const uint64_t *xb, uint32_t *R, uint32_t *tc, uint32_t d,
                                               uint32_t W, uint32_t t, uint32_t nt) {
  const uint32_t E = pre[d];
  uint32_t found = 0;
  const uint32_t lo_id = L[0], hi_id = L[d - 1];
  for (uint32_t f = t; f < E; f += nt) {
    const uint32_t i = row_of(pre, d, f);
    const uint32_t p = f - pre[i];
    const uint64_t arc = xb[i] + p;
    const uint32_t y = __ldg(dcol + arc);
    if (y < lo_id || y > hi_id) continue;
    const uint32_t j = lower_bound_u32(L, d, y);
    if (j < d && L[j] == y) {
      atomicOr(&R[(size_t)i * W + (j >> 5)], 1u << (j & 31));
      ++found;
      if (SCATTER) {
        atomicAdd(&tc[i], 1u);
        atomicAdd(&tc[j], 1u);
        atomicAdd(&t_edge[arc], 1u);
      }
    }
  }
  return found;
}

// Enumerate pairs (i, j in R_i) and triples for the 4- and 5-clique terms.
// A group of G lanes handles one row at a time; lane gl of the group holds
// word gl of the row (W <= G), so every AND is one word per lane.
template <int G, int KMAX>
__device__ __forceinline__ void enumerate_rows(const uint32_t *R, uint32_t d, uint32_t W, uint32_t row0,
                                               uint32_t row_step, uint32_t gl, unsigned long long &a4,
                                               unsigned long long &a5) {
  for (uint32_t i = row0; i < d; i += row_step) {
    const uint32_t *ri = R + (size_t)i * W;
    const uint32_t riw = (gl < W) ? ri[gl] : 0u;
    for (uint32_t t = 0; t < W; ++t) {
      uint32_t bits = ri[t];
      while (bits) {
        const uint32_t j = t * 32 + __ffs(bits) - 1;
        bits &= bits - 1;
        const uint32_t *rj = R + (size_t)j * W;
        const uint32_t mw = (gl < W) ? (riw & rj[gl]) : 0u;
        a4 += __popc(mw);
        if (KMAX >= 5) {
          for (uint32_t t2 = 0; t2 < W; ++t2) {
            uint32_t b2 = ri[t2] & rj[t2];
            while (b2) {
              const uint32_t l = t2 * 32 + __ffs(b2) - 1;
              b2 &= b2 - 1;
              if (gl < W) a5 += __popc(mw & R[(size_t)l * W + gl]);
            }
          }
        }
      }
    }
  }
}

// Same for W > 32 (global-memory class): lane gl holds words gl, gl+G, ...
template <int KMAX>
__device__ void enumerate_rows_wide(const uint32_t *R, uint32_t d, uint32_t W, uint32_t row0, uint32_t row_step,
                                    uint32_t gl, unsigned long long &a4, unsigned long long &a5) {
  constexpr uint32_t G = 32;
  for (uint32_t i = row0; i < d; i += row_step) {
    const uint32_t *ri = R + (size_t)i * W;
    for (uint32_t t = 0; t < W; ++t) {
      uint32_t bits = ri[t];
      while (bits) {
        const uint32_t j = t * 32 + __ffs(bits) - 1;
        bits &= bits - 1;
        const uint32_t *rj = R + (size_t)j * W;
        for (uint32_t w = gl; w < W; w += G) a4 += __popc(ri[w] & rj[w]);
        if (KMAX >= 5) {
          for (uint32_t t2 = 0; t2 < W; ++t2) {
            uint32_t b2 = ri[t2] & rj[t2];
            while (b2) {
              const uint32_t l = t2 * 32 + __ffs(b2) - 1;
              b2 &= b2 - 1;
              const uint32_t *rl = R + (size_t)l * W;
              for (uint32_t w = gl; w < W; w += G) a5 += __popc(ri[w] & rj[w] & rl[w]);
            }
          }
        }
      }
    }
  }
}


// Words of shared memory one warp needs for a root of out-degree <= maxd:
// xb[maxd] (uint64) | L[maxd] | pre[maxd+1] | R[maxd*W] | tc[maxd] (scatter)
__host__ __device__ constexpr uint32_t warp_words(uint32_t maxd, bool scatter) {
  return ((2 * maxd + maxd + (maxd + 1) + maxd * ((maxd + 31) / 32) + (scatter ? maxd : 0)) + 1) & ~1u;
}

// Same layout for one CTA-wide root with W words per row.
__host__ __device__ constexpr uint64_t cta_words(uint32_t maxd, uint32_t W) {
  return 2ull * maxd + maxd + (maxd + 1) + (uint64_t)maxd * W + maxd + 2;
}

// One root u (2 <= d+(u) <= MAXD) processed by the calling warp. `base` is
// the warp's shared-memory region of warp_words(MAXD, SCATTER) words.
template <int MAXD, int G, int KMAX, bool SCATTER>
__device__ __forceinline__ void lg_root_warp(const uint64_t *__restrict__ drow, const uint32_t *__restrict__ dcol,
                                             uint32_t *t_edge, uint32_t u, uint32_t *base, unsigned long long &a3,
                                             unsigned long long &a4, unsigned long long &a5) {
  const uint32_t lane = threadIdx.x & 31;
  uint64_t *xb = reinterpret_cast<uint64_t *>(base);
  uint32_t *L = base + 2 * MAXD;
  uint32_t *pre = L + MAXD;
  uint32_t *R = pre + MAXD + 1;
  uint32_t *tc = R + MAXD * ((MAXD + 31) / 32);
  const uint64_t ub = drow[u];
  const uint32_t d = (uint32_t)(drow[u + 1] - ub);
  const uint32_t w_used = (d + 31) / 32;
  for (uint32_t i = lane; i < d; i += 32) {
    const uint32_t x = __ldg(dcol + ub + i);
    L[i] = x;
    const uint64_t xs = __ldg(drow + x), xe = __ldg(drow + x + 1);
    xb[i] = xs;
    pre[i + 1] = (uint32_t)(xe - xs);
    if (SCATTER) tc[i] = 0;
  }
  for (uint32_t i = lane; i < d * w_used; i += 32) R[i] = 0;
  if (lane == 0) pre[0] = 0;
  __syncwarp();
  uint32_t carry = 0;
  for (uint32_t c0 = 0; c0 < d; c0 += 32) {
    const uint32_t i = c0 + lane;
    uint32_t v = (i < d) ? pre[i + 1] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= (uint32_t)o) v += y;
    }
    if (i < d) pre[i + 1] = v + carry;
    carry += __shfl_sync(0xffffffffu, v, 31);
  }
  __syncwarp();
  a3 += build_rows<SCATTER>(dcol, t_edge, L, pre, xb, R, tc, d, w_used, lane, 32);
  __syncwarp();
  if (SCATTER) {
    for (uint32_t i = lane; i < d; i += 32)
      if (tc[i]) atomicAdd(&t_edge[ub + i], tc[i]);
  }
  if (KMAX >= 4) enumerate_rows<G, KMAX>(R, d, w_used, lane / G, 32 / G, lane % G, a4, a5);
  __syncwarp();
}

// One root u (2 <= d+(u) <= maxd) processed by the whole CTA. `base` holds
// cta_words(maxd, W) words (shared or global memory); W >= ceil(maxd / 32).
// Every thread of the CTA must call it.
template <int G, int KMAX, bool SCATTER>
__device__ __forceinline__ void lg_root_cta(const uint64_t *__restrict__ drow, const uint32_t *__restrict__ dcol,
                                            uint32_t *t_edge, uint32_t u, uint32_t maxd, uint32_t W, uint32_t *base,
                                            unsigned long long &a3, unsigned long long &a4, unsigned long long &a5) {
  const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
  uint64_t *xb = reinterpret_cast<uint64_t *>(base);
  uint32_t *L = base + 2 * (size_t)maxd;
  uint32_t *pre = L + maxd;
  uint32_t *R = pre + maxd + 1;
  uint32_t *tc = R + (size_t)maxd * W;
  const uint64_t ub = drow[u];
  const uint32_t d = (uint32_t)(drow[u + 1] - ub);
  const uint32_t w_used = (d + 31) / 32;
  for (uint32_t i = tid; i < d; i += nt) {
    const uint32_t x = __ldg(dcol + ub + i);
    L[i] = x;
    const uint64_t xs = __ldg(drow + x), xe = __ldg(drow + x + 1);
    xb[i] = xs;
    pre[i + 1] = (uint32_t)(xe - xs);
    if (SCATTER) tc[i] = 0;
  }
  for (size_t i = tid; i < (size_t)d * w_used; i += nt) R[i] = 0;
  if (tid == 0) pre[0] = 0;
  __syncthreads();
  if (tid < 32) {
    uint32_t carry = 0;
    for (uint32_t c0 = 0; c0 < d; c0 += 32) {
      const uint32_t i = c0 + lane;
      uint32_t v = (i < d) ? pre[i + 1] : 0u;
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= (uint32_t)o) v += y;
      }
      if (i < d) pre[i + 1] = v + carry;
      carry += __shfl_sync(0xffffffffu, v, 31);
    }
  }
  __syncthreads();
  a3 += build_rows<SCATTER>(dcol, t_edge, L, pre, xb, R, tc, d, w_used, tid, nt);
  __syncthreads();
  if (SCATTER) {
    for (uint32_t i = tid; i < d; i += nt)
      if (tc[i]) atomicAdd(&t_edge[ub + i], tc[i]);
  }
  if (KMAX >= 4) {
    if (w_used > 32)
      enumerate_rows_wide<KMAX>(R, d, w_used, tid / 32, nt / 32, lane, a4, a5);
    else
      enumerate_rows<G, KMAX>(R, d, w_used, tid / G, nt / G, tid % G, a4, a5);
  }
  __syncthreads();
}

}  // namespace gpm_dev
