// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/gpm.h"

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
void gpm_set_error(const std::string &msg);
int gpm_fail(int code, const std::string &msg);
int gpm_cuda_fail(cudaError_t e, const char *what);

#define GPM_CUDA(call)                                  \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return gpm_cuda_fail(_e, #call); \
  } while (0)

#define GPM_TRY(expr)          \
  do {                         \
    int _rc = (expr);          \
    if (_rc != GPM_OK) return _rc; \
  } while (0)

// ---------------------------------------------------------------------------
// device status word bits (validation)
// ---------------------------------------------------------------------------
enum : uint32_t {
  ST_OUT_OF_RANGE = 1u,
  ST_NOT_SORTED = 2u,
  ST_DUPLICATE = 4u,
  ST_SELF_LOOP = 8u,
  ST_ASYMMETRIC = 16u,
  ST_BAD_ROWPTR = 32u,
  ST_TIMEOUT = 64u,
  ST_CAPACITY = 128u,
};

#ifdef __CUDACC__
// Exact 64-bit count accumulation. Per-thread sums cannot wrap in any feasible
// run (that takes ~2^64 additions); the sums of a warp and the additions into
// the device accumulators are checked: a carry out of 64 bits sets
// ST_CAPACITY in *status, which the host turns into GPM_E_OVERFLOW.
__device__ __forceinline__ unsigned long long warp_sum_checked(unsigned long long v, bool &carry) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_down_sync(0xffffffffu, v, o);
    carry |= (v + y < v);
    v += y;
  }
  return v;
}
// status[0]: error bits; status[1] bit s: accumulator slot s went past 64
// bits (the finalize step turns that into ST_CAPACITY for the counts that
// use slot s); slot < 0: report ST_CAPACITY directly
__device__ __forceinline__ void acc_add_checked(unsigned long long *acc, unsigned long long v, bool carry,
                                                unsigned int *status, int slot) {
  const unsigned long long old = v ? atomicAdd(acc, v) : 0ull;
  if ((carry || old + v < old) && status) {
    if (slot >= 0) atomicOr(status + 1, 1u << slot);
    else atomicOr(status, 128u);  // ST_CAPACITY
  }
}
#endif

// Out-degree classes of root vertices in the orientation. A root with
// out-degree d < 2 roots no triangle and is never a task.
enum { CLS_W32 = 0, CLS_WARP = 1, CLS_CTA = 2, CLS_XL = 3, NUM_CLS = 4 };

constexpr uint32_t kCtaSplitDegree = 384;

struct gpm_tuning {
  uint32_t warp_max_degree = 128;  // class CLS_WARP upper bound (<= 256)
  uint32_t cta_max_degree = 1024;  // class CLS_CTA upper bound (<= 1024)
  uint32_t blocks_per_sm = 0;      // 0 = occupancy-derived
  uint32_t c4_hub_bound = 1048576; // 4-cycle roots above this wedge bound: hub path
  uint32_t batch_direct_us = 1000;  // batched queries at least this slow run their plain path
  // plain count path: 4-cycle roots whose wedge bound exceeds this are counted
  // by range-partitioned shared-memory tallies (0xffffffff: never; then the
  // bucketed and hub classes above take them)
  uint32_t c4_range_bound = 1048576;
  uint32_t c4_range_width = 98304;  // vertex ids per tally range (even, <= 98304)
  // plain count path: roots whose wedge bound exceeds this (and c4_range_bound)
  // are counted 128 at a time by a pull over every vertex with bit-sliced
  // counters (0xffffffff: never)
  uint32_t c4_pull_bound = 262144;
};
gpm_tuning &gpm_tune();

// ---------------------------------------------------------------------------
// graph handle
// ---------------------------------------------------------------------------
struct gpm_graph {
  int device = 0;
  uint32_t n = 0;
  uint64_t nnz = 0;
  uint32_t max_degree = 0;

  // symmetric CSR and degrees
  uint64_t *rowptr = nullptr;  // n+1
  uint32_t *col = nullptr;     // nnz
  uint32_t *deg = nullptr;     // n

  // orientation: by degree (default) or by core number, ties to the larger id
  // in both; okey points at the key array of the order in use
  uint32_t orient_mode = 0;      // GPM_ORIENT_DEGREE or GPM_ORIENT_CORE
  uint32_t *core = nullptr;      // n core numbers (core order only)
  uint32_t *core_work = nullptr; // remaining degrees, active lists, peel rounds, counters, frontier items
  uint32_t *core_order = nullptr; // n (inside core_work): round of the peel that took each vertex
  uint32_t *okey = nullptr;
  bool prepared = false;
  uint64_t m = 0;                // arcs = nnz/2
  uint64_t *drow = nullptr;      // n+1
  uint32_t *dcol = nullptr;      // m, ascending ids per row
  uint32_t max_outdeg = 0;

  // root tasks grouped by out-degree class; class c occupies
  // tasks[cls_begin[c] .. cls_begin[c+1]) (host copy of the offsets)
  uint32_t *tasks = nullptr;
  uint32_t cls_begin[NUM_CLS + 1] = {0, 0, 0, 0, 0};
  uint32_t cls_maxdeg[NUM_CLS] = {0, 0, 0, 0};
  uint32_t tune_warp_max = 0, tune_cta_max = 0;  // thresholds the classes were built with
  // the CTA class is ordered by decreasing out-degree; roots from cta_split on
  // have out-degree <= kCtaSplitDegree (max cta_lo_maxd) and run with smaller
  // shared-memory footprints, two CTAs per SM
  uint32_t cta_split = 0, cta_lo_maxd = 0;

  // preparation scratch, kept for re-orientation
  uint32_t *prep_outdeg = nullptr;  // n
  uint64_t *prep_tiles = nullptr;   // scan tile sums
  uint64_t *prep_keys = nullptr;    // n, sort keys of the CTA/XL classes

  // small device work area: queue heads, accumulators, status
  uint64_t *work = nullptr;  // WORK_WORDS words
  // scratch pools, grown on demand
  uint32_t *t_edge = nullptr;   // per-arc triangle counts (m)
  uint32_t *xl_pool = nullptr;  // global-memory bitmaps for CLS_XL roots
  unsigned int *gen_ucount = nullptr;  // k >= 7: unit counter per root task (n words)
  size_t xl_pool_bytes = 0;
  uint32_t *tally_pool = nullptr;  // 4-cycle wedge tallies, n words per slot
  size_t tally_slots = 0;
  uint32_t *list_scratch = nullptr;
  size_t list_scratch_bytes = 0;
  // 4-cycle roots grouped by wedge bound; classes: [0,1) small (warp hash),
  // [1,2) bucketed, [2,3) hub roots (whole-GPU tallies in the plain and
  // batched forms, PART/SUM items in the served form; a per-CTA dense tally
  // item where a hub root's tally would be sparse)
  uint32_t *c4_tasks = nullptr;
  uint32_t c4_begin[4] = {0, 0, 0, 0};
  uint32_t c4_bucket_maxb = 0;  // largest wedge bound among bucketed roots
  uint32_t *c4_bucket_buf = nullptr;
  size_t c4_bucket_bytes = 0;
  uint32_t *edeg = nullptr;     // nnz: deg(col[e]), read beside col by the wedge walks
  bool c4_ready = false;
  uint32_t c4_hub_bound = 0;    // threshold the classes were built with
  // hub roots: host copies of the roots and their degrees, work units
  // {x, chunk} (unit offsets per root in c4_hub_uoff), and two sets of
  // c4_hub_R tallies + touched lists of n words each (tallies zero between calls)
  bool c4_hub_ready = false;
  std::vector<uint32_t> c4_hub_root, c4_hub_deg;
  std::vector<uint64_t> c4_hub_uoff, c4_hub_bnd;
  uint32_t *c4_hub_units = nullptr;
  uint32_t *c4_hub_tally = nullptr;
  uint32_t *c4_hub_touched = nullptr;
  uint32_t c4_hub_R = 0;
  unsigned int *c4_hub_ctr = nullptr;
  size_t c4_hub_ctr_words = 0;
  // plain count path with range tallies: its own root classes [0,1) small,
  // [1,2) bucketed, [2,3) range roots; range roots become items
  // {v0, first range, end range} ordered by decreasing wedge bound.
  // c4_roff: per vertex, c4_nr1 = ranges + 1 positions in col (32-bit) where
  // the ids of each range of c4_roff_width ids begin in its list (built once
  // per graph and width, like edeg)
  uint32_t *c4p_tasks = nullptr;
  uint32_t *c4p_bval = nullptr;
  uint32_t c4p_begin[4] = {0, 0, 0, 0};
  uint32_t c4p_bucket_maxb = 0;
  uint32_t c4p_bound = 0, c4p_pull = 0, c4p_width = 0;
  bool c4p_ready = false;
  uint32_t *c4p_items = nullptr;  // uint4 per item
  size_t c4p_items_cap = 0;
  uint32_t c4p_nitems = 0;
  uint32_t *c4_roff = nullptr;
  uint32_t c4_roff_width = 0, c4_nr1 = 0;
  // plain count path, pull class (roots above c4_pull_bound, 128 per pass):
  // vertices by decreasing degree (c4q_ord; the first c4q_nbig have degree
  // > 1024, the first c4q_nact degree >= 2) and their lists in that order,
  // membership bits of a pass's roots
  // (c4q_M, 4 words per vertex, zero between passes), the pull roots by
  // decreasing wedge bound (device c4q_roots, host c4q_hroots), one queue
  // counter per pass
  uint32_t *c4q_ord = nullptr;
  uint32_t c4q_nbig = 0, c4q_nact = 0, c4q_ntiny = 0;  // ord[c4q_ntiny, c4q_nact): degree 2..15
  uint32_t *c4q_prow = nullptr;  // the lists in the order c4q_ord: c4q_pcol[prow[i] .. prow[i + 1])
  uint32_t *c4q_pcol = nullptr;
  uint32_t *c4q_chunks = nullptr;  // {position, first entry} of each 1024-entry chunk of the first c4q_nbig
  uint32_t c4q_nchunks = 0;
  uint32_t *c4q_cntb = nullptr;  // 128 counters per vertex of degree > 1024 (zero between passes)
  uint32_t *c4q_inv = nullptr;   // position of every vertex in c4q_ord (c4q_pcol and c4q_M use positions)
  uint32_t *c4q_M = nullptr;
  uint32_t *c4q_roots = nullptr;
  size_t c4q_roots_cap = 0;
  std::vector<uint32_t> c4q_hroots;
  unsigned int *c4q_queue = nullptr;
  size_t c4q_queue_words = 0;
  // pattern-oblivious enumeration: class of every connectivity code (k = 3..5),
  // per-warp candidate lists, class counts (32 words)
  uint8_t *enum_cls[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  uint32_t *enum_scratch = nullptr;
  size_t enum_scratch_bytes = 0;
  unsigned long long *enum_counts = nullptr;
  // pattern-guided search: per-warp candidate lists
  uint32_t *guided_scratch = nullptr;
  size_t guided_scratch_bytes = 0;

  size_t device_bytes = 0;
  std::mutex mu;
};

// patterns per count call
constexpr uint32_t kMaxPatterns = 32;

// layout of gpm_graph::work (uint64 words)
enum {
  WK_QUEUE0 = 0,   // 16 uint32 queue heads
  WK_ACC = 8,      // 16 accumulators
  WK_ACC2 = 24,    // 16 accumulators of a second pass
  WK_STATUS = 56,  // status bits
  WK_MISC = 57,    // 7 misc words
  WK_OUT = 64,     // kMaxPatterns results
  WORK_WORDS = 96,
};

// ---------------------------------------------------------------------------
// pattern handle
// ---------------------------------------------------------------------------
enum PatternClass : uint32_t {
  PC_VERTEX = 0,      // k = 1
  PC_EDGE,            // k = 2
  PC_CLIQUE,          // k >= 3, complete
  PC_WEDGE,           // 3 vertices, 2 edges
  PC_STAR3,           // 4 vertices
  PC_PATH4,
  PC_TAILED,
  PC_CYCLE4,
  PC_DIAMOND,
  PC_OTHER,
};

struct gpm_pattern {
  uint32_t k = 0;
  uint8_t adj[64] = {0};
  int induced = 1;
  PatternClass cls = PC_OTHER;
  gpm_pattern_info_t info{};
  // isomorphism from the class template to this pattern's numbering:
  // template vertex t is pattern vertex tmpl_to_pat[t]
  uint32_t tmpl_to_pat[8] = {0, 1, 2, 3, 4, 5, 6, 7};
};

int gpm_plan_pattern(gpm_pattern *p);  // fills cls, info, tmpl_to_pat

// ---------------------------------------------------------------------------
// device entry points (launchers), all asynchronous on `st`
// ---------------------------------------------------------------------------
// CSR checks into *d_status; d_longv (room for n ids, e.g. the not yet
// filled degree array) and d_nlong (zero) let rows above 2048 entries be
// checked one CTA per row
int gpm_launch_validate(gpm_graph *g, cudaStream_t st, uint32_t *d_status, uint32_t *d_longv = nullptr,
                        uint32_t *d_nlong = nullptr);
int gpm_prepare_graph(gpm_graph *g, cudaStream_t st);
int gpm_ensure_classes(gpm_graph *g, cudaStream_t st);
// core numbers of every vertex into g->core and the peel round of every
// vertex into g->core_order (k-core peeling on the device); needs g->deg
int gpm_core_numbers(gpm_graph *g, cudaStream_t st);

// persistent grid size for a kernel
int gpm_num_sms(int device);

// Clique counts for k = 3..kmax (kmax <= 6), or for k = kmax alone (7..9, into
// acc[kmax - 7]), over roots in [root_lo, root_hi).
// Adds to acc[ACC_T .. kmax] (uint64, device). scatter: additionally adds
// every triangle to the per-arc counts g->t_edge (zeroed by the caller).
int gpm_launch_cliques(gpm_graph *g, int kmax, bool scatter, uint32_t root_lo, uint32_t root_hi,
                       unsigned long long *acc, cudaStream_t st);

// 4-cycle root lists (wedge-bound classes), built once per graph.
int gpm_build_c4_tasks(gpm_graph *g, cudaStream_t st);

// Hub-class 4-cycle roots (wedge bound above the hub threshold) on their own:
// prepare builds the task lists, work units and tallies (host synchronisations);
// enqueue only launches (capturable), adding their 4-cycles to acc[ACC_C4].
int gpm_c4_hub_prepare(gpm_graph *g, cudaStream_t st, bool tallies = true);
int gpm_c4_hub_enqueue(gpm_graph *g, uint32_t root_lo, uint32_t root_hi, unsigned long long *acc, cudaStream_t st,
                       uint32_t *nlaunch);

// 4-cycles whose order-last vertex lies in [root_lo, root_hi): acc[ACC_C4] += count.
// The first call per graph builds the root classes with host synchronisations;
// gpm_c4_plain_ready tells whether they exist (later calls only enqueue).
bool gpm_c4_plain_ready(const gpm_graph *g);
// pull class of the plain path: roots (by decreasing wedge bound) set up once,
// then every pass with a root in [root_lo, root_hi) enqueued
int gpm_c4_pull_prepare(gpm_graph *g, const std::vector<uint32_t> &roots, cudaStream_t st);
int gpm_launch_c4_pull(gpm_graph *g, uint32_t root_lo, uint32_t root_hi, unsigned long long *acc, cudaStream_t st);
int gpm_launch_cycles4(gpm_graph *g, uint32_t root_lo, uint32_t root_hi, unsigned long long *acc, cudaStream_t st);

// Per-arc and per-vertex local-count terms (ACC_D .. ACC_T3). With
// use_t_edge = false only the degree terms (ACC_P, ACC_S, ACC_W) are formed.
// ACC_D only counts arcs whose tail lies in [root_lo, root_hi).
int gpm_launch_edge_terms(gpm_graph *g, bool use_t_edge, uint32_t root_lo, uint32_t root_hi,
                          unsigned long long *acc, cudaStream_t st);

// Accumulator slots (uint64) filled by the passes above.
enum {
  ACC_K7 = 0,    // 7-, 8- and 9-cliques (slots 0..2: k - 7)
  ACC_T = 3,     // triangles
  ACC_K4 = 4,    // 4-cliques
  ACC_K5 = 5,    // 5-cliques
  ACC_K6 = 6,    // 6-cliques
  ACC_D = 8,     // sum over arcs C(t_e, 2)   (edge-induced diamonds)
  ACC_P = 9,     // sum over arcs (d_u-1)(d_v-1)
  ACC_S = 10,    // sum_v C(d_v, 3)
  ACC_W = 11,    // sum_v C(d_v, 2)
  ACC_TT2 = 12,  // sum over arcs t_e (d_u + d_v - 4)  (= 2 x tailed triangles)
  ACC_T3 = 13,   // sum over arcs t_e (= 3 x triangles)
  ACC_C4 = 14,   // 4-cycles
  ACC_WORDS = 16,
};

// output formulas for gpm_launch_finalize
enum Formula : uint32_t {
  F_VERTEX = 0, F_EDGE, F_TRI, F_K4, F_K5, F_WEDGE_NI, F_WEDGE_I,
  F_STAR_NI, F_PATH_NI, F_TT_NI, F_C4_NI, F_D_NI,
  F_STAR_I, F_PATH_I, F_TT_I, F_C4_I, F_D_I, F_K4_I, F_K6, F_K7, F_K8, F_K9,
};
struct FinalizeSpec {
  uint32_t npat;
  uint32_t formula[32];
};
// out[i] = formula[i](acc); status |= ST_CAPACITY when an induced count is
// inconsistent (a term overflowed 64 bits).
int gpm_launch_finalize(const FinalizeSpec &spec, const unsigned long long *acc, uint64_t n, uint64_t m,
                        unsigned long long *out, unsigned int *status, cudaStream_t st);

// Pattern-oblivious enumeration of connected k-vertex induced subgraphs
// (k = 3, 4, 5) classified by connectivity code: counts[c] (32 words, zeroed
// here) = induced count of class c; classes of connected k-vertex graphs are
// numbered by edge count, then by the smallest pair mask over vertex orders
// (pairs (0,1), (0,2), ..., (k-2,k-1) as bits 0, 1, ...).
// Only subgraphs whose smallest vertex lies in [root_lo, root_hi) are counted.
int gpm_launch_enumerate(gpm_graph *g, uint32_t k, uint32_t root_lo, uint32_t root_hi, unsigned long long *counts,
                         cudaStream_t st);
int gpm_enum_classes(uint32_t k, uint32_t *class_mask, uint32_t cap);  // number of classes
uint32_t gpm_enum_pair_index(uint32_t k, uint32_t i, uint32_t j);
int gpm_enum_class_of(const gpm_pattern &p);  // class of an induced pattern, -1 outside k = 3..5
// coef[c] = copies of pattern p (induced: 1 for its own class; edge-induced:
// spanning subgraphs of class c isomorphic to p) for every class c
int gpm_enum_coefficients(const gpm_pattern &p, uint16_t *coef, uint32_t *nclass);
struct EnumFinalize {
  uint32_t npat, nclass;
  uint32_t slot[32];       // output position of each enumerated pattern
  uint16_t coef[32][32];   // out[slot[i]] = sum_c coef[i][c] * counts[c]
};
int gpm_launch_enum_finalize(const EnumFinalize &spec, const unsigned long long *cnt, unsigned long long *out,
                             unsigned int *status, cudaStream_t st);

// Pattern-guided search for a connected pattern of 3..8 vertices, planned
// from the pattern's matching order, symmetry-breaking pairs and degree
// filter: level j matches pattern vertex order[j]; conn[j] bit i: adjacent in
// the pattern to order[i]; lower[j] / upper[j] bit i: the candidate's id must
// be above / below the vertex matched at level i; mindeg[j]: degree filter.
struct GuidedPlan {
  uint32_t k, induced;
  uint32_t order[8], conn[8], lower[8], upper[8], mindeg[8];
};
int gpm_guided_plan(const gpm_pattern &p, GuidedPlan *plan);
// Counting (out == nullptr): *acc += number of distinct subgraphs (acc zeroed
// by the caller). Listing: matches written to out (tuples of k vertices in
// pattern vertex order) while *counter < out_cap, every warp stopping at its
// next work item once the counter reaches out_cap.
int gpm_launch_guided(gpm_graph *g, const GuidedPlan &plan, unsigned long long *acc, uint32_t *out, uint64_t out_cap,
                      unsigned long long *counter, cudaStream_t st);

// Listing.
int gpm_launch_list_diamond(gpm_graph *g, uint32_t *buf, uint64_t cap, unsigned long long *counter,
                            cudaStream_t st);
int gpm_launch_list_cycle4(gpm_graph *g, uint32_t *buf, uint64_t cap, unsigned long long *counter,
                           cudaStream_t st);
int gpm_launch_list_cliques(gpm_graph *g, int k, uint32_t *buf, uint64_t cap, unsigned long long *counter,
                            cudaStream_t st);
int gpm_launch_permute_tuples(uint32_t *buf, uint64_t count, int k, const uint32_t *perm, cudaStream_t st);

// launch accounting / per-kernel event timing (profile.cpp)
void gpm_prof_begin(const char *name, cudaStream_t st);
void gpm_prof_end(cudaStream_t st);
void gpm_note_launches(uint64_t k);  // kernels launched by a CUDA-graph replay
uint64_t gpm_captured_launches();    // kernels this thread has launched into stream captures
#define GPM_LAUNCH(name, st, ...)  \
  do {                             \
    gpm_prof_begin(name, st);      \
    __VA_ARGS__;                   \
    gpm_prof_end(st);              \
  } while (0)

// The plain count path of a prepared graph, enqueued on `st` without host
// synchronisation (the 4-cycle task lists must exist when the patterns need
// them); out_dev receives npat counts, the graph's status word its error bits.
int gpm_enqueue_count(gpm_graph *g, const gpm_pattern_t *pats, uint32_t npat, unsigned long long *out_dev,
                      cudaStream_t st);
const unsigned int *gpm_graph_status(const gpm_graph *g);

// col and edeg are allocated with this many extra words: 16-byte bulk copies
// of an adjacency range may round its end up past the last entry
constexpr size_t kCsrPadWords = 16;

// grow-on-demand device allocation owned by the graph
int gpm_graph_alloc(gpm_graph *g, void **ptr, size_t bytes);
