// C-ABI of libgpm.so: graph handles, patterns, counting, listing.
// Argument checking and pass scheduling live here; every step of a count or
// a listing runs in the library's own CUDA kernels.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "gpm_internal.h"

// ---------------------------------------------------------------------------
// errors and tuning
// ---------------------------------------------------------------------------
static thread_local std::string t_last_error;

void gpm_set_error(const std::string &msg) { t_last_error = msg; }

int gpm_fail(int code, const std::string &msg) {
  t_last_error = msg;
  return code;
}

int gpm_cuda_fail(cudaError_t e, const char *what) {
  t_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return (e == cudaErrorMemoryAllocation) ? GPM_E_OOM : GPM_E_DEVICE;
}

gpm_tuning &gpm_tune() {
  static gpm_tuning t;
  return t;
}

namespace {

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

unsigned long long *acc_of(gpm_graph *g) { return reinterpret_cast<unsigned long long *>(g->work + WK_ACC); }
unsigned long long *acc2_of(gpm_graph *g) { return reinterpret_cast<unsigned long long *>(g->work + WK_ACC2); }
unsigned long long *out_of(gpm_graph *g) { return reinterpret_cast<unsigned long long *>(g->work + WK_OUT); }
unsigned int *status_of(gpm_graph *g) { return reinterpret_cast<unsigned int *>(g->work + WK_STATUS); }

void free_graph(gpm_graph *g) {
  void *ptrs[] = {g->rowptr, g->col,   g->deg,        g->drow,       g->dcol,     g->tasks,
                  g->work,   g->t_edge, g->xl_pool, g->tally_pool, g->list_scratch, g->c4_tasks, g->c4_bucket_buf,
                  g->prep_outdeg, g->prep_tiles, g->prep_keys, g->edeg, g->c4_hub_units, g->c4_hub_tally,
                  g->c4_hub_touched, g->c4_hub_ctr, g->core, g->core_work, g->c4p_tasks, g->c4p_bval,
                  g->c4p_items, g->c4_roff, g->c4q_ord, g->c4q_M, g->c4q_roots, g->c4q_queue,
                  g->c4q_prow, g->c4q_pcol, g->c4q_chunks, g->c4q_cntb, g->gen_ucount,
                  g->c4q_inv};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  delete g;
}

int status_to_code(uint32_t s) {
  if (s & ST_BAD_ROWPTR) return gpm_fail(GPM_E_INVALID_ARG, "rowptr is not a valid offset array (rowptr[0] != 0, "
                                                            "decreasing, or rowptr[n] != nnz)");
  if (s & ST_OUT_OF_RANGE) return gpm_fail(GPM_E_OUT_OF_RANGE, "a neighbour id is >= n");
  if (s & ST_NOT_SORTED) return gpm_fail(GPM_E_NOT_SORTED, "a neighbour list is not sorted ascending");
  if (s & ST_DUPLICATE) return gpm_fail(GPM_E_DUPLICATE, "a neighbour list contains a duplicate");
  if (s & ST_SELF_LOOP) return gpm_fail(GPM_E_SELF_LOOP, "the graph has a self-loop");
  if (s & ST_ASYMMETRIC) return gpm_fail(GPM_E_ASYMMETRIC, "the CSR is not symmetric");
  if (s & ST_TIMEOUT) return gpm_fail(GPM_E_TIMEOUT, "a bounded device wait gave up");
  if (s & ST_CAPACITY) return gpm_fail(GPM_E_OVERFLOW, "a count does not fit the device accumulators");
  return GPM_OK;
}

int check_graph(gpm_graph_t g) {
  if (!g) return gpm_fail(GPM_E_INVALID_ARG, "null graph handle");
  return GPM_OK;
}

int prepare_locked(gpm_graph *g, cudaStream_t st) {
  int cur = 0;
  GPM_CUDA(cudaGetDevice(&cur));
  if (cur != g->device) GPM_CUDA(cudaSetDevice(g->device));
  return gpm_prepare_graph(g, st);
}

// Pass schedule for a set of patterns.
struct Passes {
  int clique_kmax = 0;     // largest clique size needed (0 = none), from the non-scatter pass
  uint32_t gen_k = 0;      // bit k set: a pass of the generic search for k-cliques (k = 7..9)
  bool scatter = false;    // per-arc triangle counts needed
  bool edge_terms = false; // degree terms (P, S, W)
  bool cycles4 = false;
  bool tri = false;        // triangles needed (from any clique pass)
  uint32_t enum_k = 0;     // pattern-oblivious enumeration of k-vertex subgraphs (0 = none)
  FinalizeSpec spec{};
  EnumFinalize espec{};
  std::vector<std::pair<uint32_t, GuidedPlan>> guided;  // patterns counted by the pattern-guided search
};

// Pattern i counted from the class counts of the enumeration.
int schedule_enum(const gpm_pattern *p, uint32_t i, Passes *ps) {
  if (ps->enum_k && ps->enum_k != p->k)
    return gpm_fail(GPM_E_UNSUPPORTED, "enumerated patterns of one call must have the same number of vertices");
  ps->enum_k = p->k;
  const uint32_t j = ps->espec.npat++;
  ps->espec.slot[j] = i;
  uint32_t nc = 0;
  GPM_TRY(gpm_enum_coefficients(*p, ps->espec.coef[j], &nc));
  ps->espec.nclass = nc;
  ps->spec.formula[i] = F_VERTEX;  // placeholder, overwritten by the enumeration's finalize
  return GPM_OK;
}

enum Force { FORCE_NONE = 0, FORCE_ENUMERATE, FORCE_GUIDED };

int schedule(const gpm_pattern_t *pats, uint32_t npat, bool ranged, Passes *ps, Force force = FORCE_NONE) {
  if (npat > kMaxPatterns) return gpm_fail(GPM_E_INVALID_ARG, "at most 32 patterns per call");
  ps->spec.npat = npat;
  const bool enumerate_all = force == FORCE_ENUMERATE;
  for (uint32_t i = 0; i < npat; ++i) {
    const gpm_pattern *p = pats[i];
    if (!p) return gpm_fail(GPM_E_INVALID_ARG, "null pattern handle");
    if (force == FORCE_GUIDED || (p->cls == PC_OTHER && p->k >= 6)) {
      if (ranged) return gpm_fail(GPM_E_UNSUPPORTED, "root-range counts are not defined for the pattern-guided search");
      GuidedPlan plan;
      GPM_TRY(gpm_guided_plan(*p, &plan));
      ps->guided.emplace_back(i, plan);
      ps->spec.formula[i] = F_VERTEX;  // placeholder, replaced by the search's count
      continue;
    }
    if (enumerate_all || (p->cls == PC_OTHER && p->k == 5)) {
      GPM_TRY(schedule_enum(p, i, ps));  // root: the smallest vertex of the subgraph
      continue;
    }
    uint32_t f = 0;
    const bool ind = p->induced != 0;
    switch (p->cls) {
      case PC_VERTEX: f = F_VERTEX; break;
      case PC_EDGE: f = F_EDGE; break;
      case PC_CLIQUE:
        if (p->k > 9) return gpm_fail(GPM_E_UNSUPPORTED, "k-clique counting is implemented for k <= 9");
        if (p->k >= 7) {
          ps->gen_k |= 1u << p->k;
          f = F_K7 + (p->k - 7);
          break;
        }
        ps->clique_kmax = std::max<int>(ps->clique_kmax, (int)p->k);
        f = p->k == 3 ? F_TRI : (p->k == 4 ? F_K4 : (p->k == 5 ? F_K5 : F_K6));
        break;
      case PC_WEDGE:
        ps->edge_terms = true;
        if (ind) {
          ps->tri = true;
          f = F_WEDGE_I;
        } else {
          f = F_WEDGE_NI;
        }
        break;
      case PC_STAR3:
      case PC_PATH4:
      case PC_TAILED:
      case PC_CYCLE4:
      case PC_DIAMOND:
        if (ind) {
          // all six non-induced terms are needed for the inversion
          ps->scatter = ps->edge_terms = ps->cycles4 = ps->tri = true;
          ps->clique_kmax = std::max(ps->clique_kmax, 4);
          f = p->cls == PC_STAR3 ? F_STAR_I
            : p->cls == PC_PATH4 ? F_PATH_I
            : p->cls == PC_TAILED ? F_TT_I
            : p->cls == PC_CYCLE4 ? F_C4_I : F_D_I;
        } else if (p->cls == PC_STAR3) {
          ps->edge_terms = true;
          f = F_STAR_NI;
        } else if (p->cls == PC_PATH4) {
          ps->edge_terms = ps->tri = true;
          f = F_PATH_NI;
        } else if (p->cls == PC_TAILED) {
          ps->edge_terms = ps->scatter = true;
          f = F_TT_NI;
        } else if (p->cls == PC_CYCLE4) {
          ps->cycles4 = true;
          f = F_C4_NI;
        } else {
          ps->edge_terms = ps->scatter = true;
          f = F_D_NI;
        }
        break;
      default: return gpm_fail(GPM_E_UNSUPPORTED, "no GPU kernel for this pattern (supported: cliques k <= 9 and "
                                                  "connected patterns with 3, 4 or 5 vertices)");
    }
    if (ranged && !(p->cls == PC_CLIQUE || (p->cls == PC_DIAMOND && !ind) || (p->cls == PC_CYCLE4 && !ind)))
      return gpm_fail(GPM_E_UNSUPPORTED, "root-range counts are defined for cliques, diamonds, 4-cycles and 5-vertex "
                                         "patterns");
    ps->spec.formula[i] = f;
  }
  if (ps->tri) ps->clique_kmax = std::max(ps->clique_kmax, 3);
  return GPM_OK;
}

// Enqueue every pass and the finalize kernel; results in out_dev[0..npat).
int enqueue_count(gpm_graph *g, const gpm_pattern_t *pats, uint32_t npat, uint32_t lo, uint32_t hi, bool ranged,
                  unsigned long long *out_dev, cudaStream_t st, Force force = FORCE_NONE) {
  Passes ps;
  GPM_TRY(schedule(pats, npat, ranged, &ps, force));
  unsigned long long *acc = acc_of(g);
  GPM_CUDA(cudaMemsetAsync(acc, 0, ACC_WORDS * sizeof(unsigned long long), st));
  GPM_CUDA(cudaMemsetAsync(status_of(g), 0, sizeof(uint64_t), st));
  if (ps.scatter) {
    if (!g->t_edge) GPM_TRY(gpm_graph_alloc(g, (void **)&g->t_edge, sizeof(uint32_t) * std::max<uint64_t>(g->m, 1)));
    GPM_CUDA(cudaMemsetAsync(g->t_edge, 0, sizeof(uint32_t) * std::max<uint64_t>(g->m, 1), st));
    // the scatter pass covers every root (per-arc counts must be complete)
    const int k1 = std::min(ps.clique_kmax, 4);
    GPM_TRY(gpm_launch_cliques(g, std::max(k1, 3), true, 0, g->n, acc, st));
    if (ps.clique_kmax >= 5 || (ranged && ps.clique_kmax > 0)) {
      // 5- and 6-cliques (or range-restricted cliques) from a separate pass
      unsigned long long *acc2 = acc2_of(g);
      GPM_CUDA(cudaMemsetAsync(acc2, 0, ACC_WORDS * sizeof(unsigned long long), st));
      GPM_TRY(gpm_launch_cliques(g, ps.clique_kmax, false, lo, hi, acc2, st));
      GPM_CUDA(cudaMemcpyAsync(acc + ACC_T, acc2 + ACC_T, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                               st));
    }
  } else if (ps.clique_kmax >= 3) {
    GPM_TRY(gpm_launch_cliques(g, ps.clique_kmax, false, lo, hi, acc, st));
  }
  for (int k = 7; k <= 9; ++k)
    if (ps.gen_k & (1u << k)) GPM_TRY(gpm_launch_cliques(g, k, false, lo, hi, acc, st));
  if (ps.edge_terms) GPM_TRY(gpm_launch_edge_terms(g, ps.scatter, lo, hi, acc, st));
  if (ps.cycles4) GPM_TRY(gpm_launch_cycles4(g, lo, hi, acc, st));
  if (ps.enum_k) {
    if (!g->enum_counts) GPM_TRY(gpm_graph_alloc(g, (void **)&g->enum_counts, 32 * sizeof(unsigned long long)));
    GPM_TRY(gpm_launch_enumerate(g, ps.enum_k, lo, hi, g->enum_counts, st));
  }
  GPM_TRY(gpm_launch_finalize(ps.spec, acc, g->n, g->m, out_dev, status_of(g), st));
  if (ps.enum_k) GPM_TRY(gpm_launch_enum_finalize(ps.espec, g->enum_counts, out_dev, status_of(g), st));
  for (auto &gp : ps.guided) {
    GPM_CUDA(cudaMemsetAsync(out_dev + gp.first, 0, sizeof(unsigned long long), st));
    GPM_TRY(gpm_launch_guided(g, gp.second, out_dev + gp.first, nullptr, 0, nullptr, st));
  }
  return GPM_OK;
}

int count_to_host(gpm_graph *g, const gpm_pattern_t *pats, uint32_t npat, uint32_t lo, uint32_t hi, bool ranged,
                  uint64_t *counts, cudaStream_t st, Force force = FORCE_NONE) {
  unsigned long long *out = out_of(g);
  GPM_TRY(enqueue_count(g, pats, npat, lo, hi, ranged, out, st, force));
  uint64_t h[kMaxPatterns];
  uint64_t status = 0;
  GPM_CUDA(cudaMemcpyAsync(h, out, npat * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  GPM_CUDA(cudaMemcpyAsync(&status, status_of(g), sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  GPM_CUDA(cudaStreamSynchronize(st));
  GPM_TRY(status_to_code((uint32_t)status));
  std::memcpy(counts, h, npat * sizeof(uint64_t));
  return GPM_OK;
}

bool is_device_pointer(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

int gpm_enqueue_count(gpm_graph *g, const gpm_pattern_t *pats, uint32_t npat, unsigned long long *out_dev,
                      cudaStream_t st) {
  return enqueue_count(g, pats, npat, 0, g->n, false, out_dev, st);
}

const unsigned int *gpm_graph_status(const gpm_graph *g) {
  return reinterpret_cast<const unsigned int *>(g->work + WK_STATUS);
}

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *gpm_last_error(void) { return t_last_error.c_str(); }

const char *gpm_version(void) { return "gpm-b300 0.1 (sm_103a)"; }

int gpm_set_options(const gpm_options_t *opt) {
  if (!opt) return gpm_fail(GPM_E_INVALID_ARG, "null options");
  // checked and applied on a copy: an invalid field leaves every option as it was
  gpm_tuning t = gpm_tune();
  if (opt->warp_max_degree) {
    if (opt->warp_max_degree < 32 || opt->warp_max_degree > 256)
      return gpm_fail(GPM_E_INVALID_ARG, "warp_max_degree must be in [32, 256]");
    t.warp_max_degree = opt->warp_max_degree;
  }
  if (opt->cta_max_degree) {
    if (opt->cta_max_degree < t.warp_max_degree || opt->cta_max_degree > 1024)
      return gpm_fail(GPM_E_INVALID_ARG, "cta_max_degree must be in [warp_max_degree, 1024]");
    t.cta_max_degree = opt->cta_max_degree;
  }
  if (opt->blocks_per_sm) t.blocks_per_sm = opt->blocks_per_sm;
  if (opt->c4_hub_bound) {
    if (opt->c4_hub_bound <= 512 || opt->c4_hub_bound > 1048576)
      return gpm_fail(GPM_E_INVALID_ARG, "c4_hub_bound must be in [513, 1048576]");
    t.c4_hub_bound = opt->c4_hub_bound;
  }
  if (opt->batch_direct_us) t.batch_direct_us = opt->batch_direct_us;
  if (opt->c4_range_bound) {
    if (opt->c4_range_bound < 512) return gpm_fail(GPM_E_INVALID_ARG, "c4_range_bound must be >= 512");
    t.c4_range_bound = opt->c4_range_bound;
  }
  if (opt->c4_range_width) {
    if (opt->c4_range_width < 64 || opt->c4_range_width > 98304 || (opt->c4_range_width & 1u))
      return gpm_fail(GPM_E_INVALID_ARG, "c4_range_width must be even and in [64, 98304]");
    t.c4_range_width = opt->c4_range_width;
  }
  if (opt->c4_pull_bound) {
    if (opt->c4_pull_bound < 512) return gpm_fail(GPM_E_INVALID_ARG, "c4_pull_bound must be >= 512");
    t.c4_pull_bound = opt->c4_pull_bound;
  }
  gpm_tune() = t;
  return GPM_OK;
}

int gpm_get_options(gpm_options_t *opt) {
  if (!opt) return gpm_fail(GPM_E_INVALID_ARG, "null options");
  std::memset(opt, 0, sizeof(*opt));
  opt->warp_max_degree = gpm_tune().warp_max_degree;
  opt->cta_max_degree = gpm_tune().cta_max_degree;
  opt->blocks_per_sm = gpm_tune().blocks_per_sm;
  opt->c4_hub_bound = gpm_tune().c4_hub_bound;
  opt->batch_direct_us = gpm_tune().batch_direct_us;
  opt->c4_range_bound = gpm_tune().c4_range_bound;
  opt->c4_range_width = gpm_tune().c4_range_width;
  opt->c4_pull_bound = gpm_tune().c4_pull_bound;
  return GPM_OK;
}

int gpm_graph_create(const uint64_t *rowptr, const uint32_t *col, uint32_t n, uint64_t nnz, uint32_t flags,
                     void *stream, gpm_graph_t *out) {
  if (!out || !rowptr || (nnz && !col)) return gpm_fail(GPM_E_INVALID_ARG, "null argument");
  if (nnz % 2) return gpm_fail(GPM_E_ASYMMETRIC, "nnz is odd, the CSR cannot be symmetric");
  cudaStream_t st = as_stream(stream);
  const bool dev_in = (flags & GPM_GRAPH_DEVICE_INPUT) != 0;
  if (!dev_in) {
    if (rowptr[0] != 0 || rowptr[n] != nnz)
      return gpm_fail(GPM_E_INVALID_ARG, "rowptr[0] must be 0 and rowptr[n] must equal nnz");
  }
  gpm_graph *g = new gpm_graph();
  g->n = n;
  g->nnz = nnz;
  int rc = GPM_OK;
  auto fail = [&](int code) {
    free_graph(g);
    return code;
  };
  if (cudaGetDevice(&g->device) != cudaSuccess) {
    cudaGetLastError();
    return fail(gpm_fail(GPM_E_DEVICE, "no CUDA device"));
  }
  if ((rc = gpm_graph_alloc(g, (void **)&g->rowptr, sizeof(uint64_t) * ((size_t)n + 1)))) return fail(rc);
  if ((rc = gpm_graph_alloc(g, (void **)&g->col, sizeof(uint32_t) * (std::max<uint64_t>(nnz, 1) + kCsrPadWords))))
    return fail(rc);
  if ((rc = gpm_graph_alloc(g, (void **)&g->deg, sizeof(uint32_t) * std::max<uint32_t>(n, 1)))) return fail(rc);
  if ((rc = gpm_graph_alloc(g, (void **)&g->work, sizeof(uint64_t) * WORK_WORDS))) return fail(rc);
  const cudaMemcpyKind kind = dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMemcpyAsync(g->rowptr, rowptr, sizeof(uint64_t) * ((size_t)n + 1), kind, st);
  if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(g->col, col, sizeof(uint32_t) * nnz, kind, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->work, 0, sizeof(uint64_t) * WORK_WORDS, st);
  if (e != cudaSuccess) return fail(gpm_cuda_fail(e, "graph upload"));
  if (flags & GPM_GRAPH_VALIDATE) {
    uint32_t *dst = reinterpret_cast<uint32_t *>(g->work + WK_STATUS);
    // the degree array (filled only when the graph is prepared) lists the
    // long rows; WK_MISC (cleared above) counts them
    if ((rc = gpm_launch_validate(g, st, dst, g->deg, reinterpret_cast<uint32_t *>(g->work + WK_MISC)))) return fail(rc);
    uint32_t s = 0;
    e = cudaMemcpyAsync(&s, dst, sizeof(s), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(gpm_cuda_fail(e, "validation"));
    if (s) return fail(status_to_code(s));
  } else {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(gpm_cuda_fail(e, "graph upload"));
  }
  *out = g;
  return GPM_OK;
}

int gpm_graph_destroy(gpm_graph_t g) {
  if (!g) return gpm_fail(GPM_E_INVALID_ARG, "null graph handle");
  cudaDeviceSynchronize();
  free_graph(g);
  return GPM_OK;
}

int gpm_graph_prepare(gpm_graph_t g, void *stream) {
  GPM_TRY(check_graph(g));
  std::lock_guard<std::mutex> lk(g->mu);
  return prepare_locked(g, as_stream(stream));
}

int gpm_graph_reset(gpm_graph_t g) {
  GPM_TRY(check_graph(g));
  std::lock_guard<std::mutex> lk(g->mu);
  g->prepared = false;
  g->c4_ready = false;
  g->c4p_ready = false;
  g->tune_warp_max = g->tune_cta_max = 0;
  return GPM_OK;
}

int gpm_graph_set_orientation(gpm_graph_t g, uint32_t mode) {
  GPM_TRY(check_graph(g));
  if (mode != GPM_ORIENT_DEGREE && mode != GPM_ORIENT_CORE)
    return gpm_fail(GPM_E_INVALID_ARG, "orientation must be GPM_ORIENT_DEGREE or GPM_ORIENT_CORE");
  std::lock_guard<std::mutex> lk(g->mu);
  if (g->orient_mode != mode) {
    g->orient_mode = mode;
    g->prepared = false;
    g->tune_warp_max = g->tune_cta_max = 0;
  }
  return GPM_OK;
}

int gpm_graph_core_numbers(gpm_graph_t g, uint32_t *core, void *stream) {
  GPM_TRY(check_graph(g));
  if (!core && g->n) return gpm_fail(GPM_E_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = as_stream(stream);
  GPM_TRY(prepare_locked(g, st));
  if (g->orient_mode != GPM_ORIENT_CORE) GPM_TRY(gpm_core_numbers(g, st));
  if (g->n) GPM_CUDA(cudaMemcpyAsync(core, g->core, sizeof(uint32_t) * g->n, cudaMemcpyDefault, st));
  GPM_CUDA(cudaStreamSynchronize(st));
  return GPM_OK;
}

int gpm_graph_info(gpm_graph_t g, gpm_graph_info_t *info) {
  GPM_TRY(check_graph(g));
  if (!info) return gpm_fail(GPM_E_INVALID_ARG, "null info");
  std::lock_guard<std::mutex> lk(g->mu);
  std::memset(info, 0, sizeof(*info));
  info->n = g->n;
  info->nnz = g->nnz;
  info->max_degree = g->max_degree;
  info->prepared = g->prepared ? 1u : 0u;
  info->dag_arcs = g->prepared ? g->m : 0;
  info->max_out_degree = g->max_outdeg;
  info->device_bytes = g->device_bytes;
  return GPM_OK;
}

int gpm_pattern_spec(uint32_t k, const uint8_t *adj, int induced, gpm_pattern_t *out) {
  if (!out || (!adj && k > 1)) return gpm_fail(GPM_E_INVALID_ARG, "null argument");
  if (k > 8) return gpm_fail(GPM_E_K_TOO_LARGE, "pattern has more than 8 vertices");
  gpm_pattern *p = new gpm_pattern();
  p->k = k;
  if (k > 1) std::memcpy(p->adj, adj, (size_t)k * k);
  p->induced = induced ? 1 : 0;
  int rc = gpm_plan_pattern(p);
  if (rc) {
    delete p;
    return rc;
  }
  *out = p;
  return GPM_OK;
}

int gpm_pattern_clique(uint32_t k, gpm_pattern_t *out) {
  if (k < 1) return gpm_fail(GPM_E_INVALID_ARG, "clique needs k >= 1");
  if (k > 8) return gpm_fail(GPM_E_K_TOO_LARGE, "pattern has more than 8 vertices");
  uint8_t a[64] = {0};
  for (uint32_t i = 0; i < k; ++i)
    for (uint32_t j = 0; j < k; ++j) a[i * k + j] = (i != j);
  return gpm_pattern_spec(k, a, 1, out);
}

int gpm_pattern_motifs(uint32_t k, gpm_pattern_t *out, uint32_t *npat) {
  if (!out || !npat) return gpm_fail(GPM_E_INVALID_ARG, "null argument");
  std::vector<std::vector<std::pair<int, int>>> pats;
  if (k == 3) {
    pats = {{{0, 1}, {0, 2}}, {{0, 1}, {0, 2}, {1, 2}}};
  } else if (k == 4) {
    pats = {
        {{0, 1}, {0, 2}, {0, 3}},                  // 3-star
        {{0, 1}, {1, 2}, {2, 3}},                  // 4-path
        {{0, 1}, {0, 2}, {1, 2}, {2, 3}},          // tailed triangle
        {{0, 2}, {2, 1}, {1, 3}, {3, 0}},          // 4-cycle
        {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}},  // diamond
        {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}},
    };
  } else if (k == 5) {
    // the 21 connected 5-vertex graphs, by edge count, then smallest pair mask
    uint32_t cm[32];
    const int nc = gpm_enum_classes(5, cm, 32);
    for (int c = 0; c < nc; ++c) {
      std::vector<std::pair<int, int>> es;
      for (uint32_t i = 0; i < 5; ++i)
        for (uint32_t j = i + 1; j < 5; ++j)
          if (cm[c] >> gpm_enum_pair_index(5, i, j) & 1u) es.emplace_back((int)i, (int)j);
      pats.push_back(es);
    }
  } else {
    return gpm_fail(GPM_E_UNSUPPORTED, "motif sets are provided for k = 3, 4 and 5");
  }
  std::vector<gpm_pattern_t> made;
  for (auto &es : pats) {
    uint8_t a[64] = {0};
    for (auto &e : es) a[e.first * k + e.second] = a[e.second * k + e.first] = 1;
    gpm_pattern_t p = nullptr;
    int rc = gpm_pattern_spec(k, a, 1, &p);
    if (rc) {
      for (auto q : made) delete q;
      return rc;
    }
    made.push_back(p);
  }
  for (size_t i = 0; i < made.size(); ++i) out[i] = made[i];
  *npat = (uint32_t)made.size();
  return GPM_OK;
}

int gpm_pattern_destroy(gpm_pattern_t p) {
  if (!p) return gpm_fail(GPM_E_INVALID_ARG, "null pattern handle");
  delete p;
  return GPM_OK;
}

int gpm_pattern_info(gpm_pattern_t p, gpm_pattern_info_t *info) {
  if (!p || !info) return gpm_fail(GPM_E_INVALID_ARG, "null argument");
  *info = p->info;
  return GPM_OK;
}

int gpm_count(gpm_graph_t g, const gpm_pattern_t *pats, uint32_t npat, uint64_t *counts, void *stream) {
  GPM_TRY(check_graph(g));
  if (!pats || !counts || npat == 0) return gpm_fail(GPM_E_INVALID_ARG, "null argument or no patterns");
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = as_stream(stream);
  GPM_TRY(prepare_locked(g, st));
  return count_to_host(g, pats, npat, 0, g->n, false, counts, st);
}

int gpm_count_async(gpm_graph_t g, const gpm_pattern_t *pats, uint32_t npat, uint64_t *counts_dev, void *stream) {
  GPM_TRY(check_graph(g));
  if (!pats || !counts_dev || npat == 0) return gpm_fail(GPM_E_INVALID_ARG, "null argument or no patterns");
  std::lock_guard<std::mutex> lk(g->mu);
  if (!g->prepared) return gpm_fail(GPM_E_INVALID_ARG, "graph is not prepared (call gpm_graph_prepare first)");
  for (uint32_t i = 0; i < npat; ++i)
    if (pats[i] && pats[i]->cls == PC_CYCLE4 && !gpm_c4_plain_ready(g)) {
      // the 4-cycle task lists are built (with a host synchronisation) on first use
      uint64_t tmp[kMaxPatterns];
      GPM_TRY(count_to_host(g, pats, npat, 0, g->n, false, tmp, as_stream(stream)));
      break;
    }
  return enqueue_count(g, pats, npat, 0, g->n, false, reinterpret_cast<unsigned long long *>(counts_dev),
                       as_stream(stream));
}

int gpm_count_enumerate(gpm_graph_t g, const gpm_pattern_t *pats, uint32_t npat, uint64_t *counts, void *stream) {
  GPM_TRY(check_graph(g));
  if (!pats || !counts || npat == 0) return gpm_fail(GPM_E_INVALID_ARG, "null argument or no patterns");
  for (uint32_t i = 0; i < npat; ++i) {
    if (!pats[i]) return gpm_fail(GPM_E_INVALID_ARG, "null pattern handle");
    if (pats[i]->k < 3 || pats[i]->k > 5)
      return gpm_fail(GPM_E_UNSUPPORTED, "pattern-oblivious enumeration covers patterns with 3, 4 or 5 vertices");
  }
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = as_stream(stream);
  GPM_TRY(prepare_locked(g, st));
  return count_to_host(g, pats, npat, 0, g->n, false, counts, st, FORCE_ENUMERATE);
}

int gpm_count_guided(gpm_graph_t g, const gpm_pattern_t *pats, uint32_t npat, uint64_t *counts, void *stream) {
  GPM_TRY(check_graph(g));
  if (!pats || !counts || npat == 0) return gpm_fail(GPM_E_INVALID_ARG, "null argument or no patterns");
  for (uint32_t i = 0; i < npat; ++i) {
    if (!pats[i]) return gpm_fail(GPM_E_INVALID_ARG, "null pattern handle");
    if (pats[i]->k < 3)
      return gpm_fail(GPM_E_UNSUPPORTED, "the pattern-guided search covers patterns with 3..8 vertices");
  }
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = as_stream(stream);
  GPM_TRY(prepare_locked(g, st));
  return count_to_host(g, pats, npat, 0, g->n, false, counts, st, FORCE_GUIDED);
}

int gpm_count_roots(gpm_graph_t g, const gpm_pattern_t *pats, uint32_t npat, uint32_t root_lo, uint32_t root_hi,
                    uint64_t *counts, void *stream) {
  GPM_TRY(check_graph(g));
  if (!pats || !counts || npat == 0) return gpm_fail(GPM_E_INVALID_ARG, "null argument or no patterns");
  if (root_lo > root_hi || root_hi > g->n) return gpm_fail(GPM_E_INVALID_ARG, "root range outside [0, n]");
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = as_stream(stream);
  GPM_TRY(prepare_locked(g, st));
  return count_to_host(g, pats, npat, root_lo, root_hi, true, counts, st);
}

int gpm_count_cliques(gpm_graph_t g, uint32_t k, uint32_t root_lo, uint32_t root_hi, uint64_t *count,
                      void *stream) {
  GPM_TRY(check_graph(g));
  if (!count) return gpm_fail(GPM_E_INVALID_ARG, "null argument");
  if (k < 3 || k > 9) return gpm_fail(GPM_E_INVALID_ARG, "gpm_count_cliques takes k = 3..9");
  if (root_lo > root_hi || root_hi > g->n) return gpm_fail(GPM_E_INVALID_ARG, "root range outside [0, n]");
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = as_stream(stream);
  GPM_TRY(prepare_locked(g, st));
  unsigned long long *acc = acc_of(g);
  GPM_CUDA(cudaMemsetAsync(acc, 0, ACC_WORDS * sizeof(unsigned long long), st));
  GPM_CUDA(cudaMemsetAsync(status_of(g), 0, sizeof(uint64_t), st));
  GPM_TRY(gpm_launch_cliques(g, (int)k, false, root_lo, root_hi, acc, st));
  const int slot = k >= 7 ? ACC_K7 + (int)(k - 7) : (int)k;
  uint64_t h = 0, status = 0;
  GPM_CUDA(cudaMemcpyAsync(&h, acc + slot, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  GPM_CUDA(cudaMemcpyAsync(&status, status_of(g), sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  GPM_CUDA(cudaStreamSynchronize(st));
  GPM_TRY(status_to_code((uint32_t)status));
  // the high word holds one bit per accumulator slot that went past 64 bits
  if (((status >> 32) >> slot) & 1ull) return gpm_fail(GPM_E_OVERFLOW, "the clique count does not fit in 64 bits");
  *count = h;
  return GPM_OK;
}

int gpm_exists(gpm_graph_t g, gpm_pattern_t p, int *found, uint32_t *witness, void *stream) {
  GPM_TRY(check_graph(g));
  if (!p || !found) return gpm_fail(GPM_E_INVALID_ARG, "null argument");
  const bool clique = p->cls == PC_CLIQUE && p->k >= 3 && p->k <= 8;
  const bool sl = !p->induced && (p->cls == PC_DIAMOND || p->cls == PC_CYCLE4);
  GuidedPlan plan{};
  const bool guided = !clique && !sl;  // every other connected pattern of 3..8 vertices
  if (guided) GPM_TRY(gpm_guided_plan(*p, &plan));
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = as_stream(stream);
  GPM_TRY(prepare_locked(g, st));
  // the listing kernels with room for one match: every warp stops at its next
  // check once the slot counter is non-zero (no counting pass)
  uint32_t *dbuf = reinterpret_cast<uint32_t *>(out_of(g));  // 128 bytes, 16-byte aligned
  unsigned long long *counter = reinterpret_cast<unsigned long long *>(g->work + WK_MISC);
  GPM_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
  const uint32_t k = p->k;
  if (guided) GPM_TRY(gpm_launch_guided(g, plan, nullptr, dbuf, 1, counter, st));
  else if (p->cls == PC_DIAMOND) GPM_TRY(gpm_launch_list_diamond(g, dbuf, 1, counter, st));
  else if (p->cls == PC_CYCLE4) GPM_TRY(gpm_launch_list_cycle4(g, dbuf, 1, counter, st));
  else GPM_TRY(gpm_launch_list_cliques(g, (int)k, dbuf, 1, counter, st));
  unsigned long long c = 0;
  uint32_t t[8] = {0};
  GPM_CUDA(cudaMemcpyAsync(&c, counter, sizeof(c), cudaMemcpyDeviceToHost, st));
  GPM_CUDA(cudaMemcpyAsync(t, dbuf, k * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  GPM_CUDA(cudaStreamSynchronize(st));
  *found = c > 0 ? 1 : 0;
  if (witness && c > 0)  // template order -> pattern numbering (the guided search writes pattern order)
    for (uint32_t j = 0; j < k; ++j) witness[guided ? j : p->tmpl_to_pat[j]] = t[j];
  return GPM_OK;
}

int gpm_list(gpm_graph_t g, gpm_pattern_t p, uint32_t *buf, uint64_t cap, uint64_t *written, uint64_t *total,
             void *stream) {
  GPM_TRY(check_graph(g));
  if (!p || !written || !total || (cap && !buf)) return gpm_fail(GPM_E_INVALID_ARG, "null argument");
  const bool clique = p->cls == PC_CLIQUE && p->k >= 3 && p->k <= 8;
  const bool sl = !p->induced && (p->cls == PC_DIAMOND || p->cls == PC_CYCLE4);
  GuidedPlan plan{};
  const bool guided = !clique && !sl;  // every other connected pattern of 3..8 vertices
  if (guided) GPM_TRY(gpm_guided_plan(*p, &plan));
  std::lock_guard<std::mutex> lk(g->mu);
  cudaStream_t st = as_stream(stream);
  GPM_TRY(prepare_locked(g, st));
  uint64_t tot = 0;
  GPM_TRY(count_to_host(g, &p, 1, 0, g->n, false, &tot, st));
  const uint32_t k = p->k;
  uint64_t nw = 0;
  if (cap > 0 && tot > 0) {
    const bool direct = is_device_pointer(buf) && (reinterpret_cast<uintptr_t>(buf) % 16 == 0);
    uint32_t *dbuf = buf;
    if (!direct) {
      cudaError_t e = cudaMalloc(&dbuf, (size_t)std::min(cap, tot) * k * sizeof(uint32_t) + 16);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return gpm_fail(GPM_E_OOM, "listing buffer allocation failed");
      }
    }
    const uint64_t dcap = std::min(cap, tot);
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(g->work + WK_MISC);
    int rc = GPM_OK;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) rc = gpm_cuda_fail(e, "listing");
    if (!rc) {
      if (guided) rc = gpm_launch_guided(g, plan, nullptr, dbuf, dcap, counter, st);
      else if (p->cls == PC_DIAMOND) rc = gpm_launch_list_diamond(g, dbuf, dcap, counter, st);
      else if (p->cls == PC_CYCLE4) rc = gpm_launch_list_cycle4(g, dbuf, dcap, counter, st);
      else rc = gpm_launch_list_cliques(g, (int)k, dbuf, dcap, counter, st);
    }
    unsigned long long c = 0;
    if (!rc) {
      e = cudaMemcpyAsync(&c, counter, sizeof(c), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) rc = gpm_cuda_fail(e, "listing");
    }
    if (!rc) {
      nw = std::min<uint64_t>(c, dcap);
      bool ident = true;
      for (uint32_t j = 0; j < k && !guided; ++j) ident &= (p->tmpl_to_pat[j] == j);
      if (!ident) rc = gpm_launch_permute_tuples(dbuf, nw, (int)k, p->tmpl_to_pat, st);
    }
    if (!rc && !direct && nw) {
      e = cudaMemcpyAsync(buf, dbuf, nw * k * sizeof(uint32_t), cudaMemcpyDefault, st);
      if (e != cudaSuccess) rc = gpm_cuda_fail(e, "listing copy");
    }
    if (!rc) {
      e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) rc = gpm_cuda_fail(e, "listing");
    }
    if (!direct) cudaFree(dbuf);
    if (rc) return rc;
  }
  *written = nw;
  *total = tot;
  return GPM_OK;
}

}  // extern "C"
