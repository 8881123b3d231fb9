// Device building blocks of 4-cycle counting and the local-count terms,
// shared by the per-pass kernels (motif.cu) and the batched persistent kernel
// (batch.cu). See motif.cu for the method.
#pragma once

#include <stdint.h>

namespace gpm_dev {

constexpr uint32_t kC4SmallBound = 512;  // wedge bound for the shared-memory class
constexpr uint32_t kC4HubChunk = 256;    // adjacency entries of x per hub work unit
constexpr uint32_t kC4HashSlots = 1024;  // per warp, load factor <= 1/2
constexpr uint32_t kC4Empty = 0xffffffffu;

__device__ __forceinline__ bool precedes(uint32_t da, uint32_t a, uint32_t db, uint32_t b) {
  return da < db || (da == db && a < b);
}

// Degree of the neighbour col[e] = w: from the per-entry copy edeg when the
// graph has one (a coalesced load beside col), else gathered from deg.
__device__ __forceinline__ uint32_t nbr_deg(const uint32_t *__restrict__ edeg, const uint32_t *__restrict__ deg,
                                            uint64_t e, uint32_t w) {
  return edeg ? __ldg(edeg + e) : __ldg(deg + w);
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// 4-cycles rooted at v0 (its order-last vertex) by the calling warp, with a
// shared-memory hash table keys/cnt of kC4HashSlots entries each. The wedge
// bound of v0 must be <= kC4SmallBound. Returns this lane's part of the count.
__device__ __forceinline__ unsigned long long c4_root_warp(const uint64_t *__restrict__ rowptr,
                                                           const uint32_t *__restrict__ col,
                                                           const uint32_t *__restrict__ deg,
                                                           const uint32_t *__restrict__ edeg, uint32_t v0,
                                                           uint32_t *keys, uint32_t *cnt, bool &overflow) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t d0 = deg[v0];
  const uint64_t b0 = rowptr[v0], e0 = rowptr[v0 + 1];
  // a root with at most 32 neighbours has at most its one chunk's total of
  // wedge ends: its table is the smallest power of two >= twice that (32 ..
  // kC4HashSlots slots), cleared and summed at that size; larger roots use
  // every slot
  uint32_t bits = 10;  // log2(kC4HashSlots)
  bool cleared = false;
  if (e0 - b0 > 32) {
    for (uint32_t i = lane; i < kC4HashSlots; i += 32) {
      keys[i] = kC4Empty;
      cnt[i] = 0;
    }
    __syncwarp();
    cleared = true;
  }
  for (uint64_t cb = b0; cb < e0; cb += 32) {
    // up to 32 neighbours x of v0 at a time; the lists of those before v0
    // are walked as one concatenated run, 32 entries per step, each lane
    // finding its entry's list by a binary search (over the lanes, by
    // shuffles) of the inclusive scan of the list lengths
    const uint64_t ex = cb + lane;
    uint32_t len = 0;
    uint64_t xs = 0;
    if (ex < e0) {
      const uint32_t x = col[ex];
      if (precedes(nbr_deg(edeg, deg, ex, x), x, d0, v0)) {
        xs = rowptr[x];
        len = (uint32_t)(rowptr[x + 1] - xs);
      }
    }
    uint32_t incl = len;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (uint32_t)o) incl += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (!cleared) {
      bits = 5;
      while (bits < 10 && (1u << bits) < 2 * total) ++bits;
      for (uint32_t i = lane; i < (1u << bits); i += 32) {
        keys[i] = kC4Empty;
        cnt[i] = 0;
      }
      __syncwarp();
      cleared = true;
    }
    const uint32_t tmask = (1u << bits) - 1;
    for (uint32_t fb = 0; fb < total; fb += 32) {
      const uint32_t f = fb + lane;
      // first lane whose inclusive sum exceeds f (lane 31 for every f < total:
      // five halvings of [0, 31])
      uint32_t lo = 0, hi = 31;
#pragma unroll
      for (int step = 0; step < 5; ++step) {
        const uint32_t mid = (lo + hi) >> 1;
        const uint32_t v = __shfl_sync(0xffffffffu, incl, mid);
        if (lo < hi) {
          if (v <= f) lo = mid + 1;
          else hi = mid;
        }
      }
      const uint32_t src = lo;
      const uint64_t st = __shfl_sync(0xffffffffu, xs, src);
      const uint32_t before = __shfl_sync(0xffffffffu, incl - len, src);
      if (f >= total) continue;
      const uint64_t e = st + (f - before);
      const uint32_t w = col[e];
      if (!precedes(nbr_deg(edeg, deg, e, w), w, d0, v0)) continue;
      uint32_t h = (w * 2654435761u) >> (32 - bits);
      uint32_t probes = 0;
      for (;;) {
        const uint32_t k = atomicCAS(&keys[h], kC4Empty, w);
        if (k == kC4Empty || k == w) {
          atomicAdd(&cnt[h], 1u);
          break;
        }
        h = (h + 1) & tmask;
        if (++probes > tmask) {
          overflow = true;
          break;
        }
      }
    }
  }
  __syncwarp();
  unsigned long long acc = 0;
  if (cleared) {
    for (uint32_t i = lane; i < (1u << bits); i += 32) {
      const unsigned long long c = cnt[i];
      acc += c * (c - (c > 0)) / 2;
    }
  }
  __syncwarp();
  return acc;
}

// 4-cycles rooted at v0 by the whole CTA with a dense tally (n words, all
// zero on entry and on exit) and a touched list (n words) in global memory.
// s_x is a shared buffer of blockDim.x words. Every thread must call it.
// Returns this thread's part of the count.
__device__ __forceinline__ unsigned long long c4_root_cta(const uint64_t *__restrict__ rowptr,
                                                          const uint32_t *__restrict__ col,
                                                          const uint32_t *__restrict__ deg,
                                                          const uint32_t *__restrict__ edeg, uint32_t v0,
                                                          uint32_t *tally, uint32_t *touched, uint32_t *s_x,
                                                          uint32_t *s_cnt, uint32_t *s_nt) {
  const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  if (tid == 0) *s_nt = 0;
  const uint32_t d0 = deg[v0];
  const uint64_t b0 = rowptr[v0], e0 = rowptr[v0 + 1];
  for (uint64_t cb = b0; cb < e0; cb += nt) {
    if (tid == 0) *s_cnt = 0;
    __syncthreads();
    const uint64_t ex = cb + tid;
    if (ex < e0) {
      const uint32_t x = col[ex];
      if (precedes(nbr_deg(edeg, deg, ex, x), x, d0, v0)) s_x[atomicAdd(s_cnt, 1u)] = x;
    }
    __syncthreads();
    const uint32_t cnt = *s_cnt;
    for (uint32_t xi = wid; xi < cnt; xi += nw) {
      const uint32_t x = s_x[xi];
      for (uint64_t f = rowptr[x] + lane; f < rowptr[x + 1]; f += 32) {
        const uint32_t w = col[f];
        if (!precedes(nbr_deg(edeg, deg, f, w), w, d0, v0)) continue;
        if (atomicAdd(&tally[w], 1u) == 0u) touched[atomicAdd(s_nt, 1u)] = w;
      }
    }
    __syncthreads();
  }
  // the touched list is read below past L1 (ld.cg): make every thread's
  // entries reach L2 before the barrier
  __threadfence();
  __syncthreads();
  const uint32_t ntouched = *s_nt;
  unsigned long long acc = 0;
  for (uint32_t i = tid; i < ntouched; i += nt) {
    const uint32_t w = __ldcg(touched + i);
    // read-and-reset at L2: the tally was built by other threads' atomics
    const unsigned long long c = atomicExch(&tally[w], 0u);
    acc += c * (c - 1) / 2;
  }
  __syncthreads();
  return acc;
}

// ---------------------------------------------------------------------------
// 4-cycles of a large root by bucketed aggregation. The wedge ends w of root
// v0 are first scattered into P hash buckets in a per-CTA global buffer
// (streaming writes and reads, instead of random read-modify-writes on a dense
// tally that does not fit in L2); then every warp aggregates whole buckets in a
// private shared-memory hash table. P is chosen so that a bucket holds about
// kC4BucketTarget entries on average.
// ---------------------------------------------------------------------------
constexpr uint32_t kC4BucketTarget = 128;
constexpr uint32_t kC4BucketTable = 512;    // per-warp hash slots (two CTAs of 16 warps fit an SM)
constexpr uint32_t kC4MaxBuckets = 4096;
constexpr uint32_t kC4BucketMaxBound = kC4MaxBuckets * 2 * kC4BucketTarget;  // larger roots: hub class

__device__ __forceinline__ uint32_t c4_bucket_hash(uint32_t w) { return (w * 0x9E3779B1u) >> 7; }
// slot of w in a table of 2^bits slots
__device__ __forceinline__ uint32_t c4_slot_hash(uint32_t w, uint32_t bits) { return (w * 0x85EBCA77u) >> (32 - bits); }

// shared memory words for c4_root_bucketed<TABLE> with nwarps warps
template <uint32_t TABLE = kC4BucketTable>
__host__ __device__ constexpr uint32_t c4_bucket_smem_words(uint32_t nwarps) {
  return 2 * kC4MaxBuckets + 4 + nwarps * 2 * TABLE;
}
// largest wedge bound c4_root_bucketed<TABLE> takes with one table of TABLE
// slots per warp (buckets of TABLE / 4 entries on average, at most 2x that)
template <uint32_t TABLE>
__host__ __device__ constexpr uint32_t c4_bucket_narrow_bound() {
  return kC4MaxBuckets * 2 * (TABLE / 4);
}

// words of one CTA's bucket buffer (lin, then buf) for wedge bounds <= maxb
__host__ __device__ constexpr uint64_t c4_bucket_slot_words(uint64_t maxb) {
  return 2 * ((maxb + 63) & ~63ull);
}

// largest i in [0, n) with pre[i] <= f (pre ascending, pre[0] = 0 <= f)
__device__ __forceinline__ uint32_t c4_row_of(const uint32_t *pre, uint32_t n, uint32_t f) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (pre[mid] <= f) lo = mid;
    else hi = mid;
  }
  return lo;
}

// One chunk of the bucketed walk over the concatenated lists N(x), x in
// s_x[0..cnt): the CTA takes the entries in blocks of 128 per warp, four
// consecutive entries per lane (one row search for the first), so short
// lists do not leave lanes idle. s_pre holds blockDim.x + 33 words, s_rp
// blockDim.x entries. Every thread calls it; the caller synchronises after.
// sink(w, v) is called by every lane for every slot of the walk (v: w is
// a wedge end before v0), warp-synchronously.
template <class Sink>
__device__ __forceinline__ void c4_walk_flat(const uint64_t *__restrict__ rowptr, const uint32_t *__restrict__ col,
                                             const uint32_t *__restrict__ deg, const uint32_t *__restrict__ edeg,
                                             uint32_t v0, uint32_t d0, const uint32_t *s_x, uint32_t cnt,
                                             uint32_t *s_pre, uint64_t *s_rp, Sink &&sink) {
  const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  uint32_t *s_wsum = s_pre + nt + 1;
  uint32_t len = 0;
  if (tid < cnt) {
    const uint32_t x = s_x[tid];
    const uint64_t rb = rowptr[x];
    s_rp[tid] = rb;
    len = (uint32_t)(rowptr[x + 1] - rb);
  }
  uint32_t incl = len;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  if (lane == 31) s_wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const uint32_t v = (lane < nw) ? s_wsum[lane] : 0u;
    uint32_t wi = v;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= (uint32_t)o) wi += y;
    }
    if (lane < nw) s_wsum[lane] = wi - v;
  }
  __syncthreads();
  const uint32_t excl = incl - len + s_wsum[wid];
  if (tid < cnt) s_pre[tid] = excl;
  if (tid + 1 == cnt) s_pre[cnt] = excl + len;
  if (cnt == 0 && tid == 0) s_pre[0] = 0;
  __syncthreads();
  const uint32_t total = s_pre[cnt];
  for (uint32_t start = wid * 128; start < total; start += nw * 128) {
    const uint32_t f0 = start + 4 * lane;
    uint32_t i = (f0 < total) ? c4_row_of(s_pre, cnt, f0) : 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t f = f0 + q;
      uint32_t w = 0;
      bool v = false;
      if (f < total) {
        while (s_pre[i + 1] <= f) ++i;
        const uint64_t e = s_rp[i] + (f - s_pre[i]);
        w = col[e];
        v = precedes(nbr_deg(edeg, deg, e, w), w, d0, v0);
      }
      sink(w, v);
    }
  }
}

// counts wedge end w in a shared-memory table of tmask + 1 slots (linear
// probing); a full table sets overflow
__device__ __forceinline__ void c4_table_add(uint32_t *keys, uint32_t *vals, uint32_t tmask, uint32_t bits,
                                             uint32_t w, bool &overflow) {
  uint32_t h = c4_slot_hash(w, bits);
  for (uint32_t probes = 0;; ++probes) {
    const uint32_t k = atomicCAS(&keys[h], kC4Empty, w);
    if (k == kC4Empty || k == w) {
      atomicAdd(&vals[h], 1u);
      return;
    }
    h = (h + 1) & tmask;
    if (probes >= tmask) {
      overflow = true;
      return;
    }
  }
}

// 4-cycles rooted at v0 with bucketed aggregation. One walk over the wedges
// v0 - x - w appends every wedge end to `lin` (warp-aggregated) and counts it
// in its hash bucket; a streaming pass then scatters `lin` into `buf` by
// bucket. lin and buf hold at least the root's wedge bound entries each;
// sm = c4_bucket_smem_words<TABLE>(blockDim.x / 32) words of shared memory;
// s_x holds blockDim.x words. Each warp aggregates buckets in a table of
// TABLE slots; a root whose bound exceeds c4_bucket_narrow_bound<TABLE>() uses
// tables of 2 TABLE slots (two warps' space) in half of the warps, so every
// TABLE takes bounds up to c4_bucket_narrow_bound<2 TABLE>() (up to
// kC4BucketMaxBound for TABLE >= kC4BucketTable / 2). Every thread must call
// it; returns this thread's part.
template <uint32_t TABLE = kC4BucketTable>
__device__ __forceinline__ unsigned long long c4_root_bucketed(const uint64_t *__restrict__ rowptr,
                                                               const uint32_t *__restrict__ col,
                                                               const uint32_t *__restrict__ deg,
                                                               const uint32_t *__restrict__ edeg, uint32_t v0,
                                                               uint32_t *lin, uint32_t *buf, uint32_t *sm,
                                                               uint32_t *s_x, uint32_t *s_cnt, bool &overflow,
                                                               uint32_t *s_pre = nullptr, uint64_t *s_rp = nullptr,
                                                               uint32_t direct_slots = 0, uint32_t known_bound = 0) {
  const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  uint32_t *bcnt = sm;                       // [kC4MaxBuckets]: counts, then write cursors
  uint32_t *boff = sm + kC4MaxBuckets;       // [kC4MaxBuckets + 1]
  uint32_t *ctl = boff + kC4MaxBuckets + 1;  // [0] bound, [1] next bucket, [2] wedges in lin
  uint32_t *const tables = sm + 2 * kC4MaxBuckets + 4;
  const uint32_t d0 = deg[v0];
  const uint64_t b0 = rowptr[v0], e0 = rowptr[v0 + 1];
  // wedge bound (known from the class split, else summed here) -> bucket
  // count P (a power of two)
  if (tid == 0) {
    ctl[0] = 0;
    ctl[2] = 0;
  }
  __syncthreads();
  uint32_t bound = known_bound;
  if (!bound) {
    unsigned long long b = 0;
    for (uint64_t e = b0 + tid; e < e0; e += nt) {
      const uint32_t x = col[e];
      const uint32_t dx = nbr_deg(edeg, deg, e, x);
      if (precedes(dx, x, d0, v0)) b += dx;
    }
    b = warp_sum(b);
    if (lane == 0 && b) atomicAdd(&ctl[0], (uint32_t)(b > 0xffffffffull ? 0xffffffffull : b));
    __syncthreads();
    bound = ctl[0];
  }
  if (direct_slots && s_pre && 4ull * bound <= 3ull * direct_slots) {
    // every wedge end fits a table of direct_slots slots (at most 3/4 full)
    // in the whole shared-memory region: counted there directly, no bucket
    // buffers (every thread has read the bound before the region is reused)
    __syncthreads();
    uint32_t bits = 6;
    while ((1u << bits) < 2 * bound && (1u << bits) < direct_slots) ++bits;
    const uint32_t tmask = (1u << bits) - 1;
    uint32_t *dkeys = sm, *dvals = dkeys + direct_slots;
    for (uint32_t i = tid; i <= tmask; i += nt) {
      dkeys[i] = kC4Empty;
      dvals[i] = 0;
    }
    for (uint64_t cb = b0; cb < e0; cb += nt) {
      if (tid == 0) *s_cnt = 0;
      __syncthreads();
      const uint64_t ex = cb + tid;
      if (ex < e0) {
        const uint32_t x = col[ex];
        if (precedes(nbr_deg(edeg, deg, ex, x), x, d0, v0)) s_x[atomicAdd(s_cnt, 1u)] = x;
      }
      __syncthreads();
      c4_walk_flat(rowptr, col, deg, edeg, v0, d0, s_x, *s_cnt, s_pre, s_rp, [&](uint32_t w, bool v) {
        if (v) c4_table_add(dkeys, dvals, tmask, bits, w, overflow);
      });
      __syncthreads();
    }
    unsigned long long acc = 0;
    for (uint32_t i = tid; i <= tmask; i += nt) {
      const unsigned long long c = dvals[i];
      acc += c * (c - (c > 0)) / 2;
    }
    __syncthreads();
    return acc;
  }
  // table slots per aggregating warp, buckets of a quarter of that on average
  const bool wide = bound > c4_bucket_narrow_bound<TABLE>();
  const uint32_t tslots = wide ? 2 * TABLE : TABLE;
  uint32_t *keys = tables + (size_t)wid * 2 * tslots;
  uint32_t *vals = keys + tslots;
  uint32_t P = 1;
  while (P < kC4MaxBuckets && (unsigned long long)P * (tslots / 4) < bound) P <<= 1;
  const uint32_t pmask = P - 1;
  for (uint32_t b = tid; b < P; b += nt) bcnt[b] = 0;
  __syncthreads();
  // the walk: x before v0 collected per chunk of v0's list, then each warp
  // takes an x and its lanes walk N(x) in rounds of 32
  for (uint64_t cb = b0; cb < e0; cb += nt) {
    if (tid == 0) *s_cnt = 0;
    __syncthreads();
    const uint64_t ex = cb + tid;
    if (ex < e0) {
      const uint32_t x = col[ex];
      if (precedes(nbr_deg(edeg, deg, ex, x), x, d0, v0)) s_x[atomicAdd(s_cnt, 1u)] = x;
    }
    __syncthreads();
    const uint32_t cnt = *s_cnt;
    if (s_pre) {
      c4_walk_flat(rowptr, col, deg, edeg, v0, d0, s_x, cnt, s_pre, s_rp, [&](uint32_t w, bool v) {
        if (v) atomicAdd(&bcnt[c4_bucket_hash(w) & pmask], 1u);
        const uint32_t m = __ballot_sync(0xffffffffu, v);
        if (m) {
          const int leader = __ffs(m) - 1;
          uint32_t pos = 0;
          if ((int)lane == leader) pos = atomicAdd(&ctl[2], (uint32_t)__popc(m));
          pos = __shfl_sync(0xffffffffu, pos, leader);
          if (v) lin[pos + __popc(m & ((1u << lane) - 1u))] = w;
        }
      });
      __syncthreads();
      continue;
    }
    for (uint32_t xi = wid; xi < cnt; xi += nw) {
      const uint32_t x = s_x[xi];
      const uint64_t xe = rowptr[x + 1];
      for (uint64_t base = rowptr[x]; base < xe; base += 32) {
        const uint64_t e = base + lane;
        uint32_t w = 0;
        bool v = false;
        if (e < xe) {
          w = col[e];
          v = precedes(nbr_deg(edeg, deg, e, w), w, d0, v0);
        }
        if (v) atomicAdd(&bcnt[c4_bucket_hash(w) & pmask], 1u);
        const uint32_t m = __ballot_sync(0xffffffffu, v);
        if (m) {
          const int leader = __ffs(m) - 1;
          uint32_t pos = 0;
          if ((int)lane == leader) pos = atomicAdd(&ctl[2], (uint32_t)__popc(m));
          pos = __shfl_sync(0xffffffffu, pos, leader);
          if (v) lin[pos + __popc(m & ((1u << lane) - 1u))] = w;
        }
      }
    }
    __syncthreads();
  }
  const uint32_t total = ctl[2];
  // exclusive scan of the bucket counts (one warp), cursors = offsets
  if (wid == 0) {
    uint32_t carry = 0;
    for (uint32_t c0 = 0; c0 < P; c0 += 32) {
      const uint32_t i = c0 + lane;
      const uint32_t v = (i < P) ? bcnt[i] : 0u;
      uint32_t incl = v;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += y;
      }
      if (i < P) {
        boff[i] = carry + incl - v;
        bcnt[i] = carry + incl - v;
      }
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) {
      boff[P] = carry;
      ctl[1] = 0;
    }
  }
  __syncthreads();
  // streaming scatter by bucket (lin was written by other threads of this CTA)
  for (uint32_t i = tid; i < total; i += nt) {
    const uint32_t w = lin[i];
    buf[atomicAdd(&bcnt[c4_bucket_hash(w) & pmask], 1u)] = w;
  }
  // the buffer is read below by other warps of this CTA (plain loads, CTA scope)
  __syncthreads();
  // each warp aggregates whole buckets in its hash table (with wide tables,
  // the warps of the first half only)
  unsigned long long acc = 0;
  if (wide && wid >= nw / 2) {
    __syncthreads();
    return acc;
  }
  for (uint32_t i = lane; i < tslots; i += 32) {
    keys[i] = kC4Empty;
    vals[i] = 0;
  }
  __syncwarp();
  for (;;) {
    uint32_t b = 0;
    if (lane == 0) b = atomicAdd(&ctl[1], 1u);
    b = __shfl_sync(0xffffffffu, b, 0);
    if (b >= P) break;
    const uint32_t e0 = boff[b], e1 = boff[b + 1];
    if (e1 - e0 < 2) continue;  // a single wedge closes no cycle
    // table of the smallest power of two >= 2 x entries (32 .. tslots
    // slots): clearing and summing it costs at most twice the bucket
    uint32_t bits = 5;
    while (bits < 31 && (1u << bits) < 2 * (e1 - e0) && (1u << bits) < tslots) ++bits;
    const uint32_t tmask = (1u << bits) - 1;
    for (uint32_t e = e0 + lane; e < e1; e += 32) {
      const uint32_t w = buf[e];
      uint32_t h = c4_slot_hash(w, bits);
      uint32_t probes = 0;
      for (;;) {
        const uint32_t k = atomicCAS(&keys[h], kC4Empty, w);
        if (k == kC4Empty || k == w) {
          atomicAdd(&vals[h], 1u);
          break;
        }
        h = (h + 1) & tmask;
        if (++probes > tmask) {
          overflow = true;
          break;
        }
      }
    }
    __syncwarp();
    for (uint32_t i = lane; i <= tmask; i += 32) {
      const unsigned long long c = vals[i];
      acc += c * (c - (c > 0)) / 2;
      keys[i] = kC4Empty;
      vals[i] = 0;
    }
    __syncwarp();
  }
  __syncthreads();
  return acc;
}

// Local-count terms of vertex u (degree terms by lane 0; arc terms over the
// out-arcs of u in the orientation, lane-strided). With USE_T the per-arc
// triangle counts are read (and, with CLEAR_T, reset to zero afterwards).
struct EdgeTerms {
  unsigned long long D = 0, P = 0, S = 0, W = 0, TT = 0, T3 = 0;
  bool ovf = false;  // a term or a per-thread sum went past 64 bits
};

// C(d, 3) for d >= 3 without an intermediate past 64 bits: the factor
// divisible by 2 and the one divisible by 3 are divided first; ovf is set
// when C(d, 3) itself does not fit (d above about 4.8 million)
__device__ __forceinline__ unsigned long long choose3(unsigned long long d, bool &ovf) {
  unsigned long long x = d, y = d - 1, z = d - 2;
  if (x % 2 == 0) x /= 2;
  else y /= 2;
  if (x % 3 == 0) x /= 3;
  else if (y % 3 == 0) y /= 3;
  else z /= 3;
  const unsigned long long xy = x * y;  // d < 2^32: below 2^64
  ovf |= __umul64hi(xy, z) != 0;
  return xy * z;
}

__device__ __forceinline__ void add_checked(unsigned long long &s, unsigned long long v, bool &ovf) {
  ovf |= (s + v < s);
  s += v;
}

template <bool USE_T, bool CLEAR_T>
__device__ __forceinline__ void edge_terms_vertex(const uint64_t *__restrict__ drow, const uint32_t *__restrict__ dcol,
                                                  const uint32_t *__restrict__ deg, uint32_t *t_edge, uint64_t u,
                                                  bool in_range, EdgeTerms &s) {
  const uint32_t lane = threadIdx.x & 31;
  const unsigned long long du = deg[u];
  if (lane == 0) {
    if (du >= 3) add_checked(s.S, choose3(du, s.ovf), s.ovf);
    if (du >= 2) add_checked(s.W, du * (du - 1) / 2, s.ovf);
  }
  for (uint64_t e = drow[u] + lane; e < drow[u + 1]; e += 32) {
    const unsigned long long dv = deg[dcol[e]];
    add_checked(s.P, (du - 1) * (dv - 1), s.ovf);
    if (USE_T) {
      const unsigned long long t = CLEAR_T ? __ldcg(t_edge + e) : t_edge[e];
      if (t) {
        if (in_range) add_checked(s.D, t * (t - 1) / 2, s.ovf);
        s.ovf |= __umul64hi(t, du + dv - 4) != 0;
        add_checked(s.TT, t * (du + dv - 4), s.ovf);
        s.T3 += t;
        if (CLEAR_T) t_edge[e] = 0;
      }
    }
  }
}

// Requested count from the accumulators (layout ACC_* of gpm_internal.h).
// Induced 4-vertex counts are formed modulo 2^64 (exact when the true values
// fit); `bad` is set when an induced count exceeds its non-induced bound.
__device__ __forceinline__ unsigned long long finalize_formula(uint32_t f, const unsigned long long *acc, uint64_t n,
                                                               uint64_t m, bool &bad) {
  const unsigned long long T = acc[3];
  const unsigned long long NS = acc[10], NP = acc[9] - 3ull * T, NTT = acc[12] / 2ull, NC4 = acc[14], ND = acc[8],
                           NK4 = acc[4];
  const unsigned long long iK4 = NK4;
  const unsigned long long iD = ND - 6ull * iK4;
  const unsigned long long iC4 = NC4 - iD - 3ull * iK4;
  const unsigned long long iTT = NTT - 4ull * iD - 12ull * iK4;
  const unsigned long long iP = NP - 2ull * iTT - 4ull * iC4 - 6ull * iD - 12ull * iK4;
  const unsigned long long iS = NS - iTT - 2ull * iD - 4ull * iK4;
  unsigned long long v = 0;
  switch (f) {
    case 0: v = n; break;                 // F_VERTEX
    case 1: v = m; break;                 // F_EDGE
    case 2: v = T; break;                 // F_TRI
    case 3: v = acc[4]; break;            // F_K4
    case 4: v = acc[5]; break;            // F_K5
    case 5: v = acc[11]; break;           // F_WEDGE_NI
    case 6: v = acc[11] - 3ull * T; bad |= (v > acc[11]); break;  // F_WEDGE_I
    case 7: v = NS; break;
    case 8: v = NP; break;
    case 9: v = NTT; break;
    case 10: v = NC4; break;
    case 11: v = ND; break;
    case 12: v = iS; bad |= (iS > NS); break;
    case 13: v = iP; bad |= (iP > NP); break;
    case 14: v = iTT; bad |= (iTT > NTT); break;
    case 15: v = iC4; bad |= (iC4 > NC4); break;
    case 16: v = iD; bad |= (iD > ND); break;
    case 17: v = iK4; break;
    case 18: v = acc[6]; break;           // F_K6
    case 19: v = acc[0]; break;           // F_K7
    case 20: v = acc[1]; break;           // F_K8
    case 21: v = acc[2]; break;           // F_K9
    default: bad = true; break;
  }
  return v;
}

}  // namespace gpm_dev
