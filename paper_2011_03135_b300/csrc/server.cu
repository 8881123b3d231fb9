// Served form: a request loop with continuous batching over device-resident
// graphs.
//
// A persistent serving kernel pulls work items from a ring in device memory
// that the host keeps appending to while the kernel runs. Each admitted
// request (a graph and a query kind: triangles, 4-/5-cliques, 3-/4-motifs)
// occupies a request slot (its query descriptor, accumulators and item
// counters) and is cut into the same per-root items as the batched form
// (batch_device.cuh). Items of requests admitted while others are on the GPU
// land behind them in the ring, so their work overlaps on the device with the
// requests already running. When a request's last item finishes, the CTA that
// ran it forms the counts and writes a completion record to a ring in mapped
// host memory; the host polls that ring.
//
// Two rings: requests with at most kExpressItems items go to an express ring
// that the kernel drains first, so small requests are not queued behind the
// thousands of items of a large one (each request stays in one ring, which
// keeps its triangle items ahead of its edge-term items).
//
// Admission is by memory footprint: a request needs a free slot, room in the
// item ring and, for 4-motif queries, a per-arc triangle-count block (4 bytes
// per edge) from a fixed device arena; otherwise it waits in a host FIFO and
// is admitted when completions free resources. Express and bulk requests wait
// in separate FIFOs, and bulk requests may hold at most three quarters of the
// slots, so a blocked large request never holds back small ones.
//
// Every wait is bounded: the kernel's idle poll exits after about 20 ms
// without work (the host relaunches it when work arrives), and the 4-motif
// edge items' wait on their request's triangle items gives up with a status
// bit after a fixed number of polls.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <deque>
#include <map>
#include <vector>

#include "batch_device.cuh"

using namespace gpm_item;

namespace {

struct SlotState {
  QDesc q;
  unsigned long long acc[ACC_WORDS];
  unsigned int left[2];
  unsigned int pad[2];
};

struct Completion {
  unsigned long long seq;  // position + 1 once written
  unsigned long long tag;
  unsigned int slot;
  unsigned int status;
  unsigned long long counts[6];
};

constexpr uint64_t kExpressItems = 64;
constexpr uint32_t kHubSlots = 16;  // hub-class 4-cycle roots in flight at once

struct Ctl {
  unsigned long long head[2];  // next item position to claim, per ring (0 express, 1 bulk)
  unsigned long long tail[2];  // items published by the host, per ring
  unsigned long long comp_tail;
  unsigned int stop;
  unsigned int status;
};

struct ServeArgs {
  SlotState *slots;
  const Item *ring[2];
  unsigned long long ring_cap[2];
  Ctl *ctl;
  Completion *comp;  // mapped host memory
  unsigned int comp_cap;
  unsigned long long idle_limit;
  ItemEnv env;
};

__global__ void __launch_bounds__(kThreads) serve_kernel(ServeArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ Item s_item;
  __shared__ QDesc s_q;
  __shared__ int s_ok;
  __shared__ uint32_t s_cnt, s_nt;
  __shared__ uint32_t s_x[kThreads];
  __shared__ uint32_t s_pre[kThreads + 33];
  __shared__ uint64_t s_rp[kThreads];
  const uint32_t tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      s_ok = 0;
      unsigned long long idle = 0;
      for (;;) {
        if (*(volatile unsigned int *)&a.ctl->stop) break;
        bool busy = false;
        for (int r = 0; r < 2 && !s_ok; ++r) {
          const unsigned long long h = *(volatile unsigned long long *)&a.ctl->head[r];
          const unsigned long long t = *(volatile unsigned long long *)&a.ctl->tail[r];
          if (h < t) {
            busy = true;
            if (atomicCAS(&a.ctl->head[r], h, h + 1) == h) {
              const volatile uint32_t *src =
                  reinterpret_cast<const volatile uint32_t *>(a.ring[r] + (h % a.ring_cap[r]));
              uint32_t *dst = reinterpret_cast<uint32_t *>(&s_item);
              for (int w = 0; w < (int)(sizeof(Item) / 4); ++w) dst[w] = src[w];
              s_ok = 1;
            }
          }
        }
        if (s_ok) break;
        if (busy) continue;  // lost a race: retry at once
        __nanosleep(2000);
        if (++idle > a.idle_limit) break;
      }
    }
    __syncthreads();
    if (!s_ok) break;
    // the slot's descriptor is rewritten for every request that reuses it: read it past L1
    {
      const volatile uint32_t *src = reinterpret_cast<const volatile uint32_t *>(&a.slots[s_item.q].q);
      uint32_t *dst = reinterpret_cast<uint32_t *>(&s_q);
      for (uint32_t w = tid; w < sizeof(QDesc) / 4; w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    const Item it = s_item;
    run_item(a.env, s_q, it, smem, s_x, &s_cnt, &s_nt, s_pre, s_rp);
    if (tid == 0 && item_done(s_q, it)) {
      unsigned long long out6[6];
      const unsigned int bad = finalize_query(s_q, out6);
      const unsigned long long pos = atomicAdd(&a.ctl->comp_tail, 1ull);
      Completion *c = a.comp + (pos % a.comp_cap);
      c->tag = s_q.tag;
      c->slot = it.q;
      c->status = bad | (*(volatile unsigned int *)&a.ctl->status & ST_TIMEOUT);
      for (int i = 0; i < 6; ++i) c->counts[i] = out6[i];
      __threadfence_system();
      *(volatile unsigned long long *)&c->seq = pos + 1;
    }
    __syncthreads();
  }
}

}  // namespace

struct gpm_server {
  int device = 0;
  std::vector<gpm_graph *> graphs;
  cudaStream_t exec = nullptr, copy = nullptr;
  cudaEvent_t kernel_done = nullptr;
  bool launched = false;
  // device state
  SlotState *d_slots = nullptr;
  Item *d_ring[2] = {nullptr, nullptr};
  Ctl *d_ctl = nullptr;
  uint32_t *d_arena = nullptr;
  uint32_t *tally_pool = nullptr;
  uint64_t tally_slot_words = 0;
  uint32_t *lg_pool = nullptr;
  uint32_t *c4_buf = nullptr;
  uint32_t c4_maxb = 0;
  // hub-class 4-cycle roots: slots of the hub pool, per-slot item counters, and
  // the host's running totals of PART / SUM items issued per slot
  uint32_t *hub_pool = nullptr;
  unsigned int *hub_done = nullptr;
  uint32_t hub_slots = 0, hub_next = 0;
  std::vector<uint32_t> hub_parts, hub_sums;
  std::vector<Item> admit_items;  // staging of one request's items
  ItemEnv env{};
  // host mapped / pinned
  Completion *h_comp = nullptr;
  Completion *d_comp = nullptr;
  Item *h_stage = nullptr;
  SlotState *h_slot_stage = nullptr;
  unsigned long long *h_tail = nullptr;  // 2 words
  // sizes
  uint32_t nslots = 0, comp_cap = 0;
  uint64_t ring_cap[2] = {0, 0}, stage_cap = 0, arena_words = 0;
  size_t smem = 0;
  int grid = 0;
  uint32_t cta_maxd = 0, cta_W = 0;
  // host bookkeeping
  struct Req {
    uint32_t graph, kind;
    uint64_t tag;
  };
  struct Live {
    bool busy = false;
    Req req;
    int ring = 0;
    uint64_t ring_begin = 0, ring_end = 0;
    uint64_t arena_off = 0, arena_len = 0;
  };
  std::vector<Live> live;
  std::vector<uint32_t> free_slots;
  std::deque<Req> pending[2];  // 0 express, 1 bulk
  uint32_t bulk_live = 0, bulk_max = 0;
  std::deque<gpm_completion_t> instant;  // requests with no device work (empty task sets)
  uint32_t max_pending = 1u << 20;
  std::map<uint64_t, uint64_t> arena_free;  // offset -> length (words)
  uint64_t tail[2] = {0, 0};
  uint64_t comp_read = 0;
  uint32_t roots_per_item = 64, verts_per_item = 8192;
  // per (graph, kind) item templates with q = 0
  std::map<std::pair<uint32_t, uint32_t>, std::vector<Item>> templates;
  std::map<std::pair<uint32_t, uint32_t>, std::pair<uint32_t, uint32_t>> tmpl_counts;  // (scatter, all)
  std::map<std::pair<uint32_t, uint32_t>, bool> tmpl_hub;  // template holds hub items
  std::mutex mu;
};

namespace {

int arena_take(gpm_server *s, uint64_t words, uint64_t *off) {
  for (auto it = s->arena_free.begin(); it != s->arena_free.end(); ++it) {
    if (it->second >= words) {
      *off = it->first;
      const uint64_t rest = it->second - words;
      const uint64_t roff = it->first + words;
      s->arena_free.erase(it);
      if (rest) s->arena_free[roff] = rest;
      return 1;
    }
  }
  return 0;
}

void arena_give(gpm_server *s, uint64_t off, uint64_t words) {
  auto it = s->arena_free.emplace(off, words).first;
  auto next = std::next(it);
  if (next != s->arena_free.end() && it->first + it->second == next->first) {
    it->second += next->second;
    s->arena_free.erase(next);
  }
  if (it != s->arena_free.begin()) {
    auto prev = std::prev(it);
    if (prev->first + prev->second == it->first) {
      prev->second += it->second;
      s->arena_free.erase(it);
    }
  }
}

uint64_t oldest_ring_begin(gpm_server *s, int r) {
  uint64_t m = s->tail[r];
  for (auto &l : s->live)
    if (l.busy && l.ring == r) m = std::min(m, l.ring_begin);
  return m;
}

const std::vector<Item> &items_for(gpm_server *s, uint32_t gi, uint32_t kind, uint32_t *scatter, uint32_t *all) {
  auto key = std::make_pair(gi, kind);
  auto it = s->templates.find(key);
  if (it == s->templates.end()) {
    std::vector<Item> heavy, light, edge, all_items;
    uint32_t sc = 0, al = 0;
    append_query_items(s->graphs[gi], kind, 0, s->roots_per_item, s->verts_per_item, heavy, light, edge, &sc, &al,
                       false, true);
    bool hub = false;
    for (const Item &x : heavy) hub |= x.type == IT_C4_HUBPART;
    s->tmpl_hub[key] = hub;
    all_items.insert(all_items.end(), heavy.begin(), heavy.end());
    all_items.insert(all_items.end(), light.begin(), light.end());
    all_items.insert(all_items.end(), edge.begin(), edge.end());
    it = s->templates.emplace(key, std::move(all_items)).first;
    s->tmpl_counts[key] = {sc, al};
  }
  *scatter = s->tmpl_counts[key].first;
  *all = s->tmpl_counts[key].second;
  return it->second;
}

int ensure_running(gpm_server *s) {
  bool running = false;
  if (s->launched) {
    cudaError_t q = cudaEventQuery(s->kernel_done);
    if (q == cudaErrorNotReady) running = true;
    else if (q != cudaSuccess) return gpm_cuda_fail(q, "serving kernel");
  }
  if (running) return GPM_OK;
  ServeArgs a{};
  a.slots = s->d_slots;
  for (int r = 0; r < 2; ++r) {
    a.ring[r] = s->d_ring[r];
    a.ring_cap[r] = s->ring_cap[r];
  }
  a.ctl = s->d_ctl;
  a.comp = s->d_comp;
  a.comp_cap = s->comp_cap;
  a.idle_limit = 10000;  // about 20 ms of 2 us polls without work
  a.env = s->env;
  a.env.status = &s->d_ctl->status;
  a.env.tally_pool = s->tally_pool;
  a.env.tally_slot_words = s->tally_slot_words;
  GPM_LAUNCH("serve_kernel", s->exec, serve_kernel<<<s->grid, kThreads, s->smem, s->exec>>>(a));
  GPM_CUDA(cudaGetLastError());
  GPM_CUDA(cudaEventRecord(s->kernel_done, s->exec));
  s->launched = true;
  return GPM_OK;
}

// Try to admit the request; returns 1 when admitted, 0 when resources are short.
int try_admit(gpm_server *s, const gpm_server::Req &r, int *rc) {
  *rc = GPM_OK;
  if (s->free_slots.empty()) return 0;
  uint32_t sc = 0, al = 0;
  const std::vector<Item> &tmpl = items_for(s, r.graph, r.kind, &sc, &al);
  const uint64_t nitems = tmpl.size();
  gpm_graph *g = s->graphs[r.graph];
  if (nitems > kExpressItems && s->bulk_live >= s->bulk_max) return 0;
  if (nitems == 0) {
    // nothing rooted anywhere (no root has two out-neighbours): every count is 0
    gpm_completion_t c{};
    c.tag = r.tag;
    c.graph = r.graph;
    c.kind = r.kind;
    c.status = GPM_OK;
    uint32_t f[6];
    formulas_for(r.kind, f, &c.ncounts);
    s->instant.push_back(c);
    return 1;
  }
  // requests with hub items use the bulk ring: their items wait on each other
  // (and on earlier hub items), which must all be claimed in one order
  const bool hub = s->tmpl_hub[std::make_pair(r.graph, r.kind)];
  const int ring = (nitems <= kExpressItems && !hub) ? 0 : 1;
  if (s->tail[ring] + nitems - oldest_ring_begin(s, ring) > s->ring_cap[ring]) return 0;
  uint64_t off = 0, words = 0;
  if (r.kind == GPM_QUERY_MOTIF4) {
    words = (std::max<uint64_t>(g->m, 1) + 63) & ~63ull;
    if (!arena_take(s, words, &off)) return 0;
  }
  const uint32_t slot = s->free_slots.back();
  s->free_slots.pop_back();
  if (ring == 1) ++s->bulk_live;
  gpm_server::Live &l = s->live[slot];
  l.busy = true;
  l.req = r;
  l.arena_off = off;
  l.arena_len = words;
  l.ring = ring;
  l.ring_begin = s->tail[ring];
  l.ring_end = s->tail[ring] + nitems;
  // slot state: descriptor, zero accumulators, item counters
  SlotState &st = s->h_slot_stage[slot];
  std::memset(&st, 0, sizeof(st));
  QDesc &q = st.q;
  q.tag = r.tag;
  q.kind = r.kind;
  formulas_for(r.kind, q.formula, &q.nformula);
  q.rowptr = g->rowptr;
  q.col = g->col;
  q.deg = g->deg;
  q.drow = g->drow;
  q.dcol = g->dcol;
  q.t_edge = (r.kind == GPM_QUERY_MOTIF4) ? s->d_arena + off : nullptr;
  q.tasks = g->tasks;
  q.c4_tasks = g->c4_tasks;
  q.edeg = g->edeg;
  q.hub_units = reinterpret_cast<const uint2 *>(g->c4_hub_units);
  q.hub_base = g->c4_begin[2];
  q.n = g->n;
  q.m = g->m;
  SlotState *dslot = s->d_slots + slot;
  q.acc = dslot->acc;
  q.out = nullptr;
  q.left = dslot->left;
  q.scatter_items = sc;
  q.all_items = al;
  st.left[0] = sc;
  st.left[1] = al;
  cudaError_t e = cudaMemcpyAsync(dslot, &st, sizeof(SlotState), cudaMemcpyHostToDevice, s->copy);
  // this request's items: the slot, and the hub items' pool slots and wait targets
  s->admit_items.assign(tmpl.begin(), tmpl.end());
  for (Item &x : s->admit_items) x.q = slot;
  if (hub)
    assign_hub_slots(s->admit_items.data(), s->admit_items.size(), s->hub_slots, &s->hub_next, s->hub_parts.data(),
                     s->hub_sums.data());
  // items into the ring (two pieces when it wraps)
  uint64_t done = 0;
  while (e == cudaSuccess && done < nitems) {
    const uint64_t pos = s->tail[ring] + done;
    const uint64_t ring_i = pos % s->ring_cap[ring];
    const uint64_t chunk = std::min<uint64_t>({nitems - done, s->ring_cap[ring] - ring_i, s->stage_cap});
    for (uint64_t k = 0; k < chunk; ++k) s->h_stage[k] = s->admit_items[done + k];
    e = cudaMemcpyAsync(s->d_ring[ring] + ring_i, s->h_stage, sizeof(Item) * chunk, cudaMemcpyHostToDevice,
                        s->copy);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy);  // the staging buffer is reused
    done += chunk;
  }
  s->tail[ring] += nitems;
  s->h_tail[ring] = s->tail[ring];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&s->d_ctl->tail[ring], &s->h_tail[ring], sizeof(unsigned long long), cudaMemcpyHostToDevice,
                        s->copy);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy);
  if (e != cudaSuccess) {
    *rc = gpm_cuda_fail(e, "server admission");
    return 0;
  }
  *rc = ensure_running(s);
  return 1;
}

// Express FIFO first, then bulk FIFO; each stops at its first request that
// does not fit.
int admit_pending(gpm_server *s) {
  for (int q = 0; q < 2; ++q) {
    while (!s->pending[q].empty()) {
      int rc = GPM_OK;
      if (!try_admit(s, s->pending[q].front(), &rc)) {
        if (rc) return rc;
        break;
      }
      s->pending[q].pop_front();
    }
  }
  return GPM_OK;
}

int express_request(gpm_server *s, uint32_t graph, uint32_t kind) {
  uint32_t sc, al;
  return items_for(s, graph, kind, &sc, &al).size() <= kExpressItems ? 0 : 1;
}

void free_server(gpm_server *s) {
  if (s->exec) cudaStreamSynchronize(s->exec);
  void *dev[] = {s->hub_pool, s->hub_done, s->d_slots, s->d_ring[0], s->d_ring[1], s->d_ctl, s->d_arena, s->tally_pool, s->lg_pool,
                 s->c4_buf};
  for (void *p : dev)
    if (p) cudaFree(p);
  if (s->h_comp) cudaFreeHost(s->h_comp);
  if (s->h_stage) cudaFreeHost(s->h_stage);
  if (s->h_slot_stage) cudaFreeHost(s->h_slot_stage);
  if (s->h_tail) cudaFreeHost(s->h_tail);
  if (s->kernel_done) cudaEventDestroy(s->kernel_done);
  if (s->exec) cudaStreamDestroy(s->exec);
  if (s->copy) cudaStreamDestroy(s->copy);
  delete s;
}

}  // namespace

extern "C" {

int gpm_server_start(const gpm_graph_t *graphs, uint32_t ngraphs, const gpm_server_opts_t *opts,
                     gpm_server_t *out) {
  if (!graphs || !out || ngraphs == 0) return gpm_fail(GPM_E_INVALID_ARG, "null argument or no graphs");
  gpm_server *s = new gpm_server();
  auto fail = [&](int code) {
    free_server(s);
    return code;
  };
  const uint32_t nslots = (opts && opts->max_inflight) ? opts->max_inflight : 256;
  s->bulk_max = std::max<uint32_t>(1, nslots - nslots / 4);
  const uint64_t arena_bytes = (opts && opts->arena_bytes) ? opts->arena_bytes : (4ull << 30);
  const uint64_t ring_items = (opts && opts->ring_items) ? opts->ring_items : (8ull << 20);
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    return fail(gpm_fail(GPM_E_DEVICE, "no CUDA device"));
  }
  if (cudaStreamCreateWithFlags(&s->exec, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->kernel_done, cudaEventDisableTiming) != cudaSuccess)
    return fail(gpm_fail(GPM_E_DEVICE, "stream creation failed"));
  uint32_t nmax = 1;
  for (uint32_t i = 0; i < ngraphs; ++i) {
    gpm_graph *g = graphs[i];
    if (!g) return fail(gpm_fail(GPM_E_INVALID_ARG, "null graph"));
    std::lock_guard<std::mutex> lk(g->mu);
    int rc = prepare_for_items(g, true, s->copy, false, true);
    if (rc) return fail(rc);
    s->graphs.push_back(g);
    nmax = std::max(nmax, g->n);
    s->cta_maxd = std::max(s->cta_maxd, cta_root_maxd(g));
    s->c4_maxb = std::max(s->c4_maxb, g->c4_bucket_maxb);
  }
  if (cudaStreamSynchronize(s->copy) != cudaSuccess) return fail(gpm_fail(GPM_E_DEVICE, "graph preparation"));
  s->nslots = nslots;
  s->comp_cap = nslots;
  s->ring_cap[0] = 1u << 20;
  s->ring_cap[1] = ring_items;
  s->stage_cap = 1u << 16;
  s->arena_words = arena_bytes / 4;
  if (cudaMalloc(&s->d_slots, sizeof(SlotState) * nslots) != cudaSuccess ||
      cudaMalloc(&s->d_ring[0], sizeof(Item) * s->ring_cap[0]) != cudaSuccess ||
      cudaMalloc(&s->d_ring[1], sizeof(Item) * s->ring_cap[1]) != cudaSuccess ||
      cudaMalloc(&s->d_ctl, sizeof(Ctl)) != cudaSuccess ||
      cudaMalloc(&s->d_arena, sizeof(uint32_t) * std::max<uint64_t>(s->arena_words, 1)) != cudaSuccess ||
      cudaHostAlloc(&s->h_comp, sizeof(Completion) * s->comp_cap, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc(&s->h_stage, sizeof(Item) * s->stage_cap, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(&s->h_slot_stage, sizeof(SlotState) * nslots, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(&s->h_tail, 2 * sizeof(unsigned long long), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return fail(gpm_fail(GPM_E_OOM, "server allocation failed"));
  }
  if (cudaHostGetDevicePointer(reinterpret_cast<void **>(&s->d_comp), s->h_comp, 0) != cudaSuccess)
    return fail(gpm_fail(GPM_E_DEVICE, "mapped completion ring"));
  std::memset(s->h_comp, 0, sizeof(Completion) * s->comp_cap);
  cudaMemset(s->d_ctl, 0, sizeof(Ctl));
  cudaMemset(s->d_arena, 0, sizeof(uint32_t) * std::max<uint64_t>(s->arena_words, 1));
  s->arena_free[0] = s->arena_words;
  s->live.resize(nslots);
  for (uint32_t i = 0; i < nslots; ++i) s->free_slots.push_back(nslots - 1 - i);
  // kernel shape: the union of the item types' shared memory needs (CTA roots
  // above the shared-memory bound use global slots)
  s->smem = item_smem_bytes(std::min(s->cta_maxd, kItemCtaSmemMaxD), true);
  if (cudaFuncSetAttribute(serve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem) != cudaSuccess)
    return fail(gpm_fail(GPM_E_DEVICE, "shared memory attribute"));
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, serve_kernel, kThreads, s->smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  s->grid = gpm_num_sms(s->device) * per_sm;
  {
    int rc = setup_cta_items(s->env, s->cta_maxd, s->grid, &s->lg_pool);
    if (rc) return fail(rc);
  }
  if (s->c4_maxb) {
    s->env.c4_buf_words = gpm_dev::c4_bucket_slot_words(s->c4_maxb);
    if (cudaMalloc(&s->c4_buf, sizeof(uint32_t) * s->env.c4_buf_words * s->grid) != cudaSuccess) {
      cudaGetLastError();
      return fail(gpm_fail(GPM_E_OOM, "4-cycle bucket buffer allocation failed"));
    }
    s->env.c4_buf = s->c4_buf;
  }
  s->tally_slot_words = 2 * (uint64_t)nmax;
  if (cudaMalloc(&s->tally_pool, sizeof(uint32_t) * s->tally_slot_words * s->grid) != cudaSuccess) {
    cudaGetLastError();
    return fail(gpm_fail(GPM_E_OOM, "server tally pool allocation failed"));
  }
  cudaMemset(s->tally_pool, 0, sizeof(uint32_t) * s->tally_slot_words * s->grid);
  // hub pool: kHubSlots tallies of the largest graph's n words (rounded to 4)
  s->hub_slots = kHubSlots;
  s->env.hub_slot_words = ((uint64_t)nmax + 3) & ~3ull;
  s->hub_parts.assign(s->hub_slots, 0);
  s->hub_sums.assign(s->hub_slots, 0);
  if (cudaMalloc(&s->hub_pool, sizeof(uint32_t) * s->env.hub_slot_words * s->hub_slots) != cudaSuccess ||
      cudaMalloc(&s->hub_done, sizeof(unsigned int) * 2 * s->hub_slots) != cudaSuccess) {
    cudaGetLastError();
    return fail(gpm_fail(GPM_E_OOM, "server hub pool allocation failed"));
  }
  cudaMemset(s->hub_pool, 0, sizeof(uint32_t) * s->env.hub_slot_words * s->hub_slots);
  cudaMemset(s->hub_done, 0, sizeof(unsigned int) * 2 * s->hub_slots);
  s->env.hub_pool = s->hub_pool;
  s->env.hub_done = s->hub_done;
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(gpm_fail(GPM_E_DEVICE, "server set-up"));
  *out = s;
  return GPM_OK;
}

int gpm_server_submit(gpm_server_t s, uint32_t graph, uint32_t kind, uint64_t tag) {
  if (!s) return gpm_fail(GPM_E_INVALID_ARG, "null server");
  if (graph >= s->graphs.size()) return gpm_fail(GPM_E_INVALID_ARG, "graph index out of range");
  uint32_t f[6], nf;
  GPM_TRY(formulas_for(kind, f, &nf));
  std::lock_guard<std::mutex> lk(s->mu);
  gpm_server::Req r{graph, kind, tag};
  // a request that can never fit is refused outright
  uint32_t sc, al;
  const uint64_t nitems = items_for(s, graph, kind, &sc, &al).size();
  if (nitems > s->ring_cap[1]) return gpm_fail(GPM_E_INVALID_ARG, "request needs more items than the ring holds");
  if (kind == GPM_QUERY_MOTIF4 && ((std::max<uint64_t>(s->graphs[graph]->m, 1) + 63) & ~63ull) > s->arena_words)
    return gpm_fail(GPM_E_INVALID_ARG, "request needs more arena memory than the server has");
  const int q = express_request(s, graph, kind);
  if (s->pending[q].empty()) {
    int rc = GPM_OK;
    if (try_admit(s, r, &rc)) return GPM_OK;
    if (rc) return rc;
  }
  if (s->pending[0].size() + s->pending[1].size() >= s->max_pending)
    return gpm_fail(GPM_E_BUSY, "server queue is full");
  s->pending[q].push_back(r);
  return GPM_OK;
}

int gpm_server_poll(gpm_server_t s, gpm_completion_t *out, uint32_t max, uint32_t *n) {
  if (!s || !n || (max && !out)) return gpm_fail(GPM_E_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  uint32_t got = 0;
  while (got < max && !s->instant.empty()) {
    out[got++] = s->instant.front();
    s->instant.pop_front();
  }
  while (got < max) {
    Completion *c = s->h_comp + (s->comp_read % s->comp_cap);
    if (*(volatile unsigned long long *)&c->seq != s->comp_read + 1) break;
    std::atomic_thread_fence(std::memory_order_acquire);
    const uint32_t slot = c->slot;
    gpm_server::Live &l = s->live[slot];
    gpm_completion_t &o = out[got++];
    std::memset(&o, 0, sizeof(o));
    o.tag = c->tag;
    o.graph = l.req.graph;
    o.kind = l.req.kind;
    o.status = (c->status & ST_TIMEOUT) ? GPM_E_TIMEOUT : ((c->status & ST_CAPACITY) ? GPM_E_OVERFLOW : GPM_OK);
    uint32_t f[6];
    formulas_for(l.req.kind, f, &o.ncounts);
    for (int i = 0; i < 6; ++i) o.counts[i] = c->counts[i];
    if (o.status != GPM_OK && l.arena_len)
      cudaMemsetAsync(s->d_arena + l.arena_off, 0, l.arena_len * 4, s->copy);  // re-zero a dirty block
    if (l.arena_len) arena_give(s, l.arena_off, l.arena_len);
    if (l.ring == 1) --s->bulk_live;
    l.busy = false;
    s->free_slots.push_back(slot);
    s->comp_read++;
  }
  cudaStreamSynchronize(s->copy);
  GPM_TRY(admit_pending(s));
  bool outstanding = false;
  for (auto &l : s->live) outstanding |= l.busy;
  if (outstanding) GPM_TRY(ensure_running(s));
  *n = got;
  return GPM_OK;
}

int gpm_server_stats(gpm_server_t s, uint32_t *inflight, uint32_t *pending) {
  if (!s) return gpm_fail(GPM_E_INVALID_ARG, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  uint32_t busy = 0;
  for (auto &l : s->live) busy += l.busy;
  if (inflight) *inflight = busy;
  if (pending) *pending = (uint32_t)(s->pending[0].size() + s->pending[1].size());
  return GPM_OK;
}

int gpm_server_stop(gpm_server_t s) {
  if (!s) return gpm_fail(GPM_E_INVALID_ARG, "null server");
  unsigned int one = 1;
  cudaMemcpyAsync(&s->d_ctl->stop, &one, sizeof(one), cudaMemcpyHostToDevice, s->copy);
  cudaStreamSynchronize(s->copy);
  cudaError_t e = cudaStreamSynchronize(s->exec);
  free_server(s);
  if (e != cudaSuccess) return gpm_cuda_fail(e, "serving kernel");
  return GPM_OK;
}

}  // extern "C"
