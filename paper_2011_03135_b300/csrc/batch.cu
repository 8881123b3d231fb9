// Batched form: many count queries over many resident graphs in ONE
// persistent fused kernel, replayed from a CUDA graph.
//
// Each query (a graph and a kind: 3-/4-motifs, triangles, 4- or 5-cliques)
// is cut into work items of the same per-root routines the per-class kernels
// use (lg_device.cuh, motif_device.cuh):
//   LG_WARP  a range of roots with out-degree <= 128, one root per warp
//   LG_CTA   one root with a larger out-degree, the whole CTA
//   C4_SMALL  a range of 4-cycle roots with a small wedge bound, one per warp
//   C4_BUCKET one 4-cycle root with a larger bound, bucketed by the whole CTA
//   EDGE      a range of vertices: local-count terms (4-motif queries wait
//             until all of the query's triangle-scatter items are done)
// Items sit in one global queue, heavy items first and EDGE items last; every
// CTA pulls the next item with one atomicAdd. A query's last finished item
// computes its counts (motif inversion included) on the device. Nothing
// synchronises the host between queries, so small queries overlap with large
// ones instead of each paying a launch sequence and a host round trip.
// Hub-class 4-cycle roots are counted by whole-GPU launches captured ahead of
// the persistent kernel, and the heaviest queries (timed at creation) run
// their plain count path there too.
//
// The EDGE items' wait is bounded (a spin with __nanosleep and an iteration
// cap); on timeout the kernel sets a status bit, the host reports
// GPM_E_TIMEOUT and re-zeroes the per-arc buffers.
//
// The per-query schedule (roots per warp item, vertices per EDGE item, the
// warp/CTA split) is chosen by a small autotuner: each candidate is timed by
// one replay on the first run and the fastest is kept.
#include <algorithm>
#include <cstring>
#include <vector>

#include "batch_device.cuh"

using namespace gpm_item;

namespace {

struct BatchArgs {
  const QDesc *qs;
  const Item *items;
  uint32_t nitems;
  unsigned int *head;
  ItemEnv env;
};

__global__ void __launch_bounds__(kThreads) batch_kernel(BatchArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ Item s_item;
  __shared__ uint32_t s_idx, s_cnt, s_nt;
  __shared__ uint32_t s_x[kThreads];
  __shared__ uint32_t s_pre[kThreads + 33];
  __shared__ uint64_t s_rp[kThreads];
  const uint32_t tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      s_idx = atomicAdd(a.head, 1u);
      if (s_idx < a.nitems) s_item = a.items[s_idx];
    }
    __syncthreads();
    if (s_idx >= a.nitems) break;
    const Item it = s_item;
    __syncthreads();
    const QDesc &q = a.qs[it.q];
    run_item(a.env, q, it, smem, s_x, &s_cnt, &s_nt, s_pre, s_rp);
    if (tid == 0 && item_done(q, it)) {
      // last item of this query: its counts, then re-arm it for the next replay
      const unsigned int bad = finalize_query(q, q.out);
      if (bad) atomicOr(a.env.status, bad);
      for (int i = 0; i < ACC_WORDS; ++i) q.acc[i] = 0ull;
      q.left[0] = q.scatter_items;
      __threadfence();
      q.left[1] = q.all_items;
    }
    __syncthreads();
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct gpm_batch {
  int device = 0;
  std::vector<gpm_query_t> queries;
  cudaStream_t stream = nullptr;
  QDesc *d_qs = nullptr;
  Item *d_items = nullptr;
  uint32_t nitems = 0, items_cap = 0;
  unsigned long long *d_acc = nullptr;  // nq * ACC_WORDS
  unsigned long long *d_out = nullptr;  // nq * 6
  unsigned int *d_left = nullptr;       // nq * 2
  unsigned int *d_head = nullptr;       // head, status
  uint32_t *tally_pool = nullptr;
  uint64_t tally_slot_words = 0;
  uint32_t *lg_pool = nullptr;
  uint32_t *c4_buf = nullptr;
  uint32_t c4_maxb = 0;
  ItemEnv env{};
  uint64_t *h_out = nullptr;  // pinned
  std::vector<uint32_t *> own_t_edge;  // per-arc buffers of repeated motif-4 graphs
  uint32_t cta_maxd = 0, cta_W = 0;
  size_t smem = 0;
  int grid = 0;
  uint32_t roots_per_item = 64, verts_per_item = 8192;
  bool tuned = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t graph_kernels = 1;  // kernels one replay launches
  std::vector<QDesc> qs;
  // queries run as their plain count path inside the captured graph (heavy
  // queries, measured at creation), with their patterns and status words
  std::vector<uint8_t> direct;
  std::vector<gpm_pattern_t> kind_pats[8];
  unsigned int *d_dstatus = nullptr;  // one word per query (the direct ones use the first ndirect)
  unsigned int *h_dstatus = nullptr;
  uint32_t ndirect = 0;
  double tuned_ms = 0.0;
  std::vector<float> qms;     // plain-path device time of every query (ms), measured at creation
  float direct_ms = 0.0f;     // threshold in use
};

namespace {

void free_batch(gpm_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  void *dev[] = {b->d_qs,       b->d_items, b->d_acc,  b->d_out,     b->d_left, b->d_head,
                 b->tally_pool, b->lg_pool, b->c4_buf, b->d_dstatus};
  for (void *p : dev)
    if (p) cudaFree(p);
  if (b->h_out) cudaFreeHost(b->h_out);
  if (b->h_dstatus) cudaFreeHost(b->h_dstatus);
  for (auto &v : b->kind_pats)
    for (gpm_pattern_t p : v) gpm_pattern_destroy(p);
  for (uint32_t *p : b->own_t_edge) cudaFree(p);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

// Work items for the current schedule; heavy items first, EDGE items last.
void make_items(gpm_batch *b, std::vector<Item> &items) {
  items.clear();
  std::vector<Item> heavy, light, edge;
  const uint32_t nq = (uint32_t)b->queries.size();
  for (uint32_t qi = 0; qi < nq; ++qi) {
    QDesc &q = b->qs[qi];
    if (b->direct[qi]) {
      q.scatter_items = q.all_items = 0;
      continue;
    }
    append_query_items(b->queries[qi].graph, q.kind, qi, b->roots_per_item, b->verts_per_item, heavy, light, edge,
                       &q.scatter_items, &q.all_items, true);
  }
  items.insert(items.end(), heavy.begin(), heavy.end());
  items.insert(items.end(), light.begin(), light.end());
  items.insert(items.end(), edge.begin(), edge.end());
}

int upload_schedule(gpm_batch *b) {
  std::vector<Item> items;
  make_items(b, items);
  const uint32_t nq = (uint32_t)b->queries.size();
  if (items.size() > b->items_cap) {
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    GPM_CUDA(cudaMalloc(&b->d_items, sizeof(Item) * std::max<size_t>(items.size(), 1)));
    b->items_cap = (uint32_t)items.size();
  }
  b->nitems = (uint32_t)items.size();
  std::vector<unsigned int> left(2 * nq);
  for (uint32_t i = 0; i < nq; ++i) {
    left[2 * i] = b->qs[i].scatter_items;
    left[2 * i + 1] = b->qs[i].all_items;
  }
  GPM_CUDA(cudaMemcpyAsync(b->d_items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice, b->stream));
  GPM_CUDA(cudaMemcpyAsync(b->d_qs, b->qs.data(), sizeof(QDesc) * nq, cudaMemcpyHostToDevice, b->stream));
  GPM_CUDA(cudaMemcpyAsync(b->d_left, left.data(), sizeof(unsigned int) * 2 * nq, cudaMemcpyHostToDevice,
                           b->stream));
  GPM_CUDA(cudaMemsetAsync(b->d_acc, 0, sizeof(unsigned long long) * ACC_WORDS * nq, b->stream));
  GPM_CUDA(cudaStreamSynchronize(b->stream));
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  return GPM_OK;
}

int capture(gpm_batch *b) {
  BatchArgs a{};
  a.qs = b->d_qs;
  a.items = b->d_items;
  a.nitems = b->nitems;
  a.head = b->d_head;
  a.env = b->env;
  a.env.status = b->d_head + 1;
  a.env.tally_pool = b->tally_pool;
  a.env.tally_slot_words = b->tally_slot_words;
  const uint32_t nq = (uint32_t)b->queries.size();
  GPM_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  cudaMemsetAsync(b->d_head, 0, sizeof(unsigned int), b->stream);
  // hub-class 4-cycle roots first: whole-GPU launches per query, adding to the
  // query's accumulator before the persistent kernel finalises it
  b->graph_kernels = 1;
  const uint64_t captured0 = gpm_captured_launches();
  int hub_rc = GPM_OK;
  // heavy queries: their plain count path, outputs straight to their slots
  for (uint32_t qi = 0, k = 0; qi < nq && hub_rc == GPM_OK; ++qi) {
    if (!b->direct[qi]) continue;
    const std::vector<gpm_pattern_t> &pats = b->kind_pats[b->qs[qi].kind];
    gpm_graph *g = b->queries[qi].graph;
    hub_rc = gpm_enqueue_count(g, pats.data(), (uint32_t)pats.size(), b->d_out + (size_t)6 * qi, b->stream);
    if (hub_rc == GPM_OK &&
        cudaMemcpyAsync(b->d_dstatus + k++, gpm_graph_status(g), sizeof(unsigned int), cudaMemcpyDeviceToDevice,
                        b->stream) != cudaSuccess)
      hub_rc = gpm_fail(GPM_E_DEVICE, "batch capture (status copy)");
  }
  b->graph_kernels += gpm_captured_launches() - captured0;
  for (uint32_t qi = 0; qi < nq && hub_rc == GPM_OK; ++qi) {
    gpm_graph *g = b->queries[qi].graph;
    if (b->direct[qi] || b->qs[qi].kind != GPM_QUERY_MOTIF4 || g->c4_begin[3] == g->c4_begin[2]) continue;
    uint32_t nl = 0;
    hub_rc = gpm_c4_hub_enqueue(g, 0, g->n, b->d_acc + (size_t)qi * ACC_WORDS, b->stream, &nl);
    b->graph_kernels += nl;
  }
  GPM_LAUNCH("batch_kernel", b->stream, batch_kernel<<<b->grid, kThreads, b->smem, b->stream>>>(a));
  cudaMemcpyAsync(b->h_out, b->d_out, sizeof(uint64_t) * 6 * nq, cudaMemcpyDeviceToHost, b->stream);
  if (b->ndirect)
    cudaMemcpyAsync(b->h_dstatus, b->d_dstatus, sizeof(unsigned int) * b->ndirect, cudaMemcpyDeviceToHost, b->stream);
  cudaError_t e = cudaStreamEndCapture(b->stream, &b->graph);
  if (hub_rc != GPM_OK) return hub_rc;
  if (e != cudaSuccess) return gpm_cuda_fail(e, "batch capture");
  GPM_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
  return GPM_OK;
}

int replay(gpm_batch *b, float *ms) {
  if (!b->exec) GPM_TRY(capture(b));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ms) {
    GPM_CUDA(cudaEventCreate(&e0));
    GPM_CUDA(cudaEventCreate(&e1));
    GPM_CUDA(cudaEventRecord(e0, b->stream));
  }
  GPM_CUDA(cudaGraphLaunch(b->exec, b->stream));
  gpm_note_launches(b->graph_kernels);
  if (ms) GPM_CUDA(cudaEventRecord(e1, b->stream));
  GPM_CUDA(cudaStreamSynchronize(b->stream));
  if (ms) {
    cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  unsigned int status = 0;
  GPM_CUDA(cudaMemcpy(&status, b->d_head + 1, sizeof(status), cudaMemcpyDeviceToHost));
  if (status) {
    // a timed-out or overflowing run leaves partial state: re-arm everything
    GPM_CUDA(cudaMemset(b->d_head + 1, 0, sizeof(unsigned int)));
    for (size_t i = 0; i < b->queries.size(); ++i)
      if (b->qs[i].t_edge)
        GPM_CUDA(cudaMemset(b->qs[i].t_edge, 0, sizeof(uint32_t) * std::max<uint64_t>(b->qs[i].m, 1)));
    GPM_TRY(upload_schedule(b));
    if (status & ST_TIMEOUT) return gpm_fail(GPM_E_TIMEOUT, "batched kernel: a bounded wait gave up");
    return gpm_fail(GPM_E_OVERFLOW, "batched kernel: a motif count does not fit in 64 bits");
  }
  for (uint32_t k = 0; k < b->ndirect; ++k)
    if (b->h_dstatus[k]) return gpm_fail(GPM_E_OVERFLOW, "batched plain-path query: a count does not fit in 64 bits");
  return GPM_OK;
}

// Heavy queries run their plain count path inside the captured graph: a
// query whose plain path takes at least the direct threshold on the device is
// marked direct, together with every other query on the same graph (they
// share its per-arc buffer). Small queries become items of the persistent
// kernel, where they overlap instead of paying a launch sequence each. The
// plain-path time of every query is measured once, when the batch is created
// (a first run also sizes every lazily grown buffer); the autotuner then
// tries several thresholds on these times.
int measure_plain(gpm_batch *b) {
  const uint32_t nq = (uint32_t)b->queries.size();
  for (uint32_t i = 0; i < nq; ++i) {
    const uint32_t kind = b->qs[i].kind;
    std::vector<gpm_pattern_t> &v = b->kind_pats[kind];
    if (!v.empty()) continue;
    if (kind == GPM_QUERY_MOTIF3 || kind == GPM_QUERY_MOTIF4) {
      gpm_pattern_t p[8];
      uint32_t np = 0;
      GPM_TRY(gpm_pattern_motifs(kind == GPM_QUERY_MOTIF3 ? 3 : 4, p, &np));
      v.assign(p, p + np);
    } else {
      gpm_pattern_t p = nullptr;
      GPM_TRY(gpm_pattern_clique(kind == GPM_QUERY_TC ? 3 : kind == GPM_QUERY_CLIQUE4 ? 4 : 5, &p));
      v.push_back(p);
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  GPM_CUDA(cudaEventCreate(&e0));
  GPM_CUDA(cudaEventCreate(&e1));
  b->qms.assign(nq, 0.0f);
  int rc = GPM_OK;
  for (uint32_t i = 0; i < nq && rc == GPM_OK; ++i) {
    gpm_graph *g = b->queries[i].graph;
    const std::vector<gpm_pattern_t> &pats = b->kind_pats[b->qs[i].kind];
    std::lock_guard<std::mutex> lk(g->mu);
    float ms = 0.0f;
    for (int rep = 0; rep < 2 && rc == GPM_OK; ++rep) {
      if (cudaEventRecord(e0, b->stream) != cudaSuccess) rc = gpm_fail(GPM_E_DEVICE, "event record");
      if (rc == GPM_OK) rc = gpm_enqueue_count(g, pats.data(), (uint32_t)pats.size(), b->d_out + (size_t)6 * i, b->stream);
      if (rc == GPM_OK && (cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                           cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = gpm_fail(GPM_E_DEVICE, "timing a batched query's plain path");
      if (rep == 0 && ms < 0.05f) break;  // clearly small: no second run needed
    }
    b->qms[i] = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (cudaMalloc(&b->d_dstatus, sizeof(unsigned int) * nq) != cudaSuccess ||
      cudaMallocHost(&b->h_dstatus, sizeof(unsigned int) * nq) != cudaSuccess) {
    cudaGetLastError();
    return gpm_fail(GPM_E_OOM, "batch status allocation failed");
  }
  return GPM_OK;
}

// Direct queries for threshold `ms` (3.4e38: none); resets what the item
// queries expect at the start of a run and drops the captured graph.
int set_direct(gpm_batch *b, float ms) {
  const uint32_t nq = (uint32_t)b->queries.size();
  std::vector<gpm_graph *> heavy_graphs;
  for (uint32_t i = 0; i < nq; ++i)
    if (b->qms[i] >= ms) heavy_graphs.push_back(b->queries[i].graph);
  b->direct.assign(nq, 0);
  for (uint32_t i = 0; i < nq; ++i)
    b->direct[i] = std::find(heavy_graphs.begin(), heavy_graphs.end(), b->queries[i].graph) != heavy_graphs.end();
  b->ndirect = (uint32_t)std::count(b->direct.begin(), b->direct.end(), (uint8_t)1);
  b->direct_ms = ms;
  // plain runs leave per-arc triangle counts in the graphs' buffers, which
  // item queries expect zero at the start of a run; and counts in the output slots
  for (uint32_t i = 0; i < nq; ++i)
    if (!b->direct[i] && b->qs[i].t_edge)
      GPM_CUDA(cudaMemsetAsync(b->qs[i].t_edge, 0, sizeof(uint32_t) * std::max<uint64_t>(b->qs[i].m, 1), b->stream));
  GPM_CUDA(cudaMemsetAsync(b->d_out, 0, sizeof(unsigned long long) * 6 * nq, b->stream));
  GPM_CUDA(cudaStreamSynchronize(b->stream));
  return GPM_OK;
}

// Autotuner: which queries run their plain path (threshold 1/4, 1 and 4
// times batch_direct_us on their measured plain time) x the item schedule
// (roots per warp item, vertices per EDGE item); each candidate is captured
// and timed by one replay after a warm one, the fastest is kept.
int autotune(gpm_batch *b) {
  struct Cand {
    uint32_t roots, verts;
  };
  const Cand cands[] = {{64, 8192}, {16, 4096}, {256, 32768}};
  const uint32_t direct_us = gpm_tune().batch_direct_us;
  std::vector<float> thresholds;
  if (direct_us == 0xffffffffu) thresholds = {3.4e38f};
  else thresholds = {0.25e-3f * direct_us, 1e-3f * direct_us, 4e-3f * direct_us};
  float best = 1e30f, best_thr = thresholds[0];
  Cand bestc = cands[0];
  for (float thr : thresholds) {
    GPM_TRY(set_direct(b, thr));
    for (const Cand &c : cands) {
      b->roots_per_item = c.roots;
      b->verts_per_item = c.verts;
      GPM_TRY(upload_schedule(b));
      float ms = 0.f;
      GPM_TRY(replay(b, nullptr));  // warm
      GPM_TRY(replay(b, &ms));
      if (ms < best) {
        best = ms;
        bestc = c;
        best_thr = thr;
      }
    }
  }
  GPM_TRY(set_direct(b, best_thr));
  b->roots_per_item = bestc.roots;
  b->verts_per_item = bestc.verts;
  b->tuned_ms = best;
  GPM_TRY(upload_schedule(b));
  b->tuned = true;
  return GPM_OK;
}

}  // namespace

extern "C" {

int gpm_batch_create(const gpm_query_t *queries, uint32_t nq, gpm_batch_t *out) {
  if (!queries || !out || nq == 0) return gpm_fail(GPM_E_INVALID_ARG, "null argument or empty batch");
  gpm_batch *b = new gpm_batch();
  auto fail = [&](int code) {
    free_batch(b);
    return code;
  };
  b->queries.assign(queries, queries + nq);
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    cudaGetLastError();
    return fail(gpm_fail(GPM_E_DEVICE, "no CUDA device"));
  }
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(gpm_fail(GPM_E_DEVICE, "stream creation failed"));
  uint32_t nmax = 1;
  bool need_c4 = false;
  b->qs.resize(nq);
  std::vector<gpm_graph *> m4_graphs;
  for (uint32_t i = 0; i < nq; ++i) {
    gpm_graph *g = queries[i].graph;
    if (!g) return fail(gpm_fail(GPM_E_INVALID_ARG, "null graph in batch"));
    std::lock_guard<std::mutex> lk(g->mu);
    int rc = prepare_for_items(g, queries[i].kind == GPM_QUERY_MOTIF4, b->stream, true);
    if (rc) return fail(rc);
    QDesc &q = b->qs[i];
    std::memset(&q, 0, sizeof(q));
    q.kind = queries[i].kind;
    rc = formulas_for(q.kind, q.formula, &q.nformula);
    if (rc) return fail(rc);
    if (q.kind == GPM_QUERY_MOTIF4) {
      if (!g->t_edge) {
        rc = gpm_graph_alloc(g, (void **)&g->t_edge, sizeof(uint32_t) * std::max<uint64_t>(g->m, 1));
        if (rc) return fail(rc);
      }
      if (cudaMemsetAsync(g->t_edge, 0, sizeof(uint32_t) * std::max<uint64_t>(g->m, 1), b->stream) != cudaSuccess)
        return fail(gpm_fail(GPM_E_DEVICE, "t_edge reset failed"));
      need_c4 = true;
    }
    q.rowptr = g->rowptr;
    q.col = g->col;
    q.deg = g->deg;
    q.drow = g->drow;
    q.dcol = g->dcol;
    q.t_edge = g->t_edge;
    if (q.kind == GPM_QUERY_MOTIF4) {
      if (std::find(m4_graphs.begin(), m4_graphs.end(), g) != m4_graphs.end()) {
        // the same graph in several motif-4 queries: each needs its own per-arc counts
        uint32_t *p = nullptr;
        if (cudaMalloc(&p, sizeof(uint32_t) * std::max<uint64_t>(g->m, 1)) != cudaSuccess) {
          cudaGetLastError();
          return fail(gpm_fail(GPM_E_OOM, "per-query arc buffer allocation failed"));
        }
        b->own_t_edge.push_back(p);
        cudaMemsetAsync(p, 0, sizeof(uint32_t) * std::max<uint64_t>(g->m, 1), b->stream);
        q.t_edge = p;
      }
      m4_graphs.push_back(g);
    }
    q.tasks = g->tasks;
    q.c4_tasks = g->c4_tasks;
    q.edeg = g->edeg;
    q.n = g->n;
    q.m = g->m;
    nmax = std::max(nmax, g->n);
    b->cta_maxd = std::max(b->cta_maxd, cta_root_maxd(g));
    if (q.kind == GPM_QUERY_MOTIF4) b->c4_maxb = std::max(b->c4_maxb, g->c4_bucket_maxb);
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fail(gpm_fail(GPM_E_DEVICE, "batch preparation"));
  // arenas
  int rc = GPM_OK;
  if (cudaMalloc(&b->d_qs, sizeof(QDesc) * nq) != cudaSuccess ||
      cudaMalloc(&b->d_acc, sizeof(unsigned long long) * ACC_WORDS * nq) != cudaSuccess ||
      cudaMalloc(&b->d_out, sizeof(unsigned long long) * 6 * nq) != cudaSuccess ||
      cudaMalloc(&b->d_left, sizeof(unsigned int) * 2 * nq) != cudaSuccess ||
      cudaMalloc(&b->d_head, sizeof(unsigned int) * 4) != cudaSuccess ||
      cudaMallocHost(&b->h_out, sizeof(uint64_t) * 6 * nq) != cudaSuccess) {
    cudaGetLastError();
    return fail(gpm_fail(GPM_E_OOM, "batch arena allocation failed"));
  }
  cudaMemset(b->d_head, 0, sizeof(unsigned int) * 4);
  cudaMemset(b->d_out, 0, sizeof(unsigned long long) * 6 * nq);
  for (uint32_t i = 0; i < nq; ++i) {
    b->qs[i].acc = b->d_acc + (size_t)ACC_WORDS * i;
    b->qs[i].out = b->d_out + (size_t)6 * i;
    b->qs[i].left = b->d_left + 2 * i;
  }
  // shared memory: the largest of the item types' needs (CTA roots above the
  // shared-memory bound use global slots)
  b->smem = item_smem_bytes(std::min(b->cta_maxd, kItemCtaSmemMaxD), need_c4);
  if (cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem) != cudaSuccess)
    return fail(gpm_fail(GPM_E_DEVICE, "shared memory attribute"));
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, kThreads, b->smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  b->grid = gpm_num_sms(b->device) * per_sm;
  rc = setup_cta_items(b->env, b->cta_maxd, b->grid, &b->lg_pool);
  if (rc) return fail(rc);
  if (need_c4 && b->c4_maxb) {
    b->env.c4_buf_words = gpm_dev::c4_bucket_slot_words(b->c4_maxb);
    if (cudaMalloc(&b->c4_buf, sizeof(uint32_t) * b->env.c4_buf_words * b->grid) != cudaSuccess) {
      cudaGetLastError();
      return fail(gpm_fail(GPM_E_OOM, "4-cycle bucket buffer allocation failed"));
    }
    b->env.c4_buf = b->c4_buf;
  }
  if (need_c4) {
    b->tally_slot_words = 2 * (uint64_t)nmax;
    if (cudaMalloc(&b->tally_pool, sizeof(uint32_t) * b->tally_slot_words * b->grid) != cudaSuccess) {
      cudaGetLastError();
      return fail(gpm_fail(GPM_E_OOM, "batch tally pool allocation failed"));
    }
    cudaMemset(b->tally_pool, 0, sizeof(uint32_t) * b->tally_slot_words * b->grid);
  }
  rc = measure_plain(b);
  if (rc) return fail(rc);
  {
    const uint32_t direct_us = gpm_tune().batch_direct_us;
    rc = set_direct(b, direct_us == 0xffffffffu ? 3.4e38f : 1e-3f * direct_us);
  }
  if (rc) return fail(rc);
  rc = upload_schedule(b);
  if (rc) return fail(rc);
  *out = b;
  return GPM_OK;
}

int gpm_batch_run(gpm_batch_t b, uint64_t *counts, void *stream) {
  if (!b || !counts) return gpm_fail(GPM_E_INVALID_ARG, "null argument");
  cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
  // order after the caller's stream
  cudaEvent_t ev;
  GPM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  GPM_CUDA(cudaEventRecord(ev, user));
  GPM_CUDA(cudaStreamWaitEvent(b->stream, ev, 0));
  cudaEventDestroy(ev);
  if (!b->tuned) GPM_TRY(autotune(b));
  GPM_TRY(replay(b, nullptr));
  std::memcpy(counts, b->h_out, sizeof(uint64_t) * 6 * b->queries.size());
  return GPM_OK;
}

int gpm_batch_info(gpm_batch_t b, uint32_t *nitems, uint32_t *roots_per_item, uint32_t *verts_per_item,
                   uint32_t *grid) {
  if (!b) return gpm_fail(GPM_E_INVALID_ARG, "null batch");
  if (nitems) *nitems = b->nitems;
  if (roots_per_item) *roots_per_item = b->roots_per_item;
  if (verts_per_item) *verts_per_item = b->verts_per_item;
  if (grid) *grid = (uint32_t)b->grid;
  return GPM_OK;
}

int gpm_batch_direct(gpm_batch_t b, uint32_t *ndirect, uint64_t *graph_kernels) {
  if (!b) return gpm_fail(GPM_E_INVALID_ARG, "null batch");
  if (ndirect) *ndirect = b->ndirect;
  if (graph_kernels) *graph_kernels = b->graph_kernels;
  return GPM_OK;
}

int gpm_batch_destroy(gpm_batch_t b) {
  if (!b) return gpm_fail(GPM_E_INVALID_ARG, "null batch");
  cudaStreamSynchronize(b->stream);
  free_batch(b);
  return GPM_OK;
}

int gpm_count_batch(const gpm_query_t *queries, uint32_t nq, uint64_t *counts, void *stream) {
  gpm_batch_t b = nullptr;
  GPM_TRY(gpm_batch_create(queries, nq, &b));
  int rc = gpm_batch_run(b, counts, stream);
  gpm_batch_destroy(b);
  return rc;
}

}  // extern "C"
