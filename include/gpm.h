/*
 * gpm.h -- C-ABI of the B300 graph-pattern-mining library (libgpm.so).
 *
 * The library counts and lists embeddings of small connected patterns in a
 * large undirected graph on one GPU, following the problem statement of
 * Sandslash (arxiv 2011.03135): Section 2 "Problem Definition" (embeddings,
 * vertex- vs edge-induced subgraphs, counting vs listing, the GPM problems
 * TC, k-CL, SL, k-MC) and Section 3.1 "High-Level API" (a pattern given
 * explicitly by its edges plus an induced/non-induced flag; a clique
 * generator; all k-vertex motifs).
 *
 * Conventions shared by every entry point
 *  - Return value: GPM_OK (0) on success, a negative GPM_E_* code on error.
 *    On error no output argument is modified and gpm_last_error() returns a
 *    message for the calling host thread.
 *  - Counts are exact unsigned 64-bit integers. A count that does not fit in
 *    64 bits is reported as GPM_E_OVERFLOW: every warp's partial sum and
 *    every addition into the device accumulators is checked for a carry out
 *    of 64 bits (a single thread's running sum could only wrap after ~2^64
 *    additions), and the motif inversion checks its terms. The batched and
 *    served forms report an overflow of the motif inversion only.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Calls that return results in host memory synchronise that
 *    stream before returning; *_async calls do not.
 *  - Handles are owned by the library; a handle must not be used after it
 *    has been destroyed. Calls on one graph handle are serialised on the
 *    host, and their device work must not overlap: a graph keeps one set of
 *    accumulators and scratch buffers, so asynchronous counts on the same
 *    graph belong on one stream. Different graphs are independent.
 *  - Vertex ids are uint32 (n < 2^32); CSR offsets are uint64.
 */
#ifndef GPM_H_
#define GPM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------- status codes ---------------- */
#define GPM_OK 0
#define GPM_E_INVALID_ARG (-1)
#define GPM_E_NOT_SORTED (-2)        /* a neighbour list is not strictly ascending */
#define GPM_E_SELF_LOOP (-3)         /* v appears in its own neighbour list */
#define GPM_E_DUPLICATE (-4)         /* a neighbour appears twice in one list */
#define GPM_E_ASYMMETRIC (-5)        /* u in N(v) but v not in N(u) */
#define GPM_E_DISCONNECTED_PATTERN (-6)
#define GPM_E_K_TOO_LARGE (-7)
#define GPM_E_OOM (-8)               /* device allocation failed */
#define GPM_E_DEVICE (-9)            /* a CUDA call failed */
#define GPM_E_TIMEOUT (-10)          /* a bounded device-side wait gave up */
#define GPM_E_BUSY (-11)             /* admission refused (server) */
#define GPM_E_UNSUPPORTED (-12)      /* outside a kernel's limits (pattern size, root out-degree, root ranges) */
#define GPM_E_OVERFLOW (-13)         /* a result does not fit in 64 bits */
#define GPM_E_OUT_OF_RANGE (-14)     /* vertex id >= n in the CSR */

/* ---------------- handles ---------------- */
typedef struct gpm_graph *gpm_graph_t;
typedef struct gpm_pattern *gpm_pattern_t;

/* ---------------- graphs ---------------- */

/* gpm_graph_create flags */
#define GPM_GRAPH_VALIDATE 1u     /* check sorted / no loop / no duplicate / symmetric on the GPU */
#define GPM_GRAPH_DEVICE_INPUT 2u /* rowptr/col are device pointers (copied device-to-device) */

/*
 * Upload an undirected simple graph given as a symmetric CSR (Section 6: the
 * inputs are symmetric, without self-loops or duplicate edges, with sorted
 * neighbour lists).
 *   rowptr : uint64[n+1], rowptr[0] = 0, rowptr[n] = nnz (host memory unless
 *            GPM_GRAPH_DEVICE_INPUT)
 *   col    : uint32[nnz], neighbours of v in col[rowptr[v] .. rowptr[v+1])
 *   nnz    : 2 x (number of undirected edges)
 * The library copies both arrays; the caller keeps ownership of its buffers.
 * With GPM_GRAPH_VALIDATE, a malformed CSR returns GPM_E_NOT_SORTED,
 * GPM_E_SELF_LOOP, GPM_E_DUPLICATE, GPM_E_ASYMMETRIC or GPM_E_OUT_OF_RANGE and
 * no handle is created; an input with several faults reports the first of
 * GPM_E_INVALID_ARG (offsets that decrease or run past nnz),
 * GPM_E_OUT_OF_RANGE, GPM_E_NOT_SORTED, GPM_E_DUPLICATE, GPM_E_SELF_LOOP,
 * GPM_E_ASYMMETRIC. Without the flag the input is trusted. In both cases an
 * odd nnz (GPM_E_ASYMMETRIC) and, for host input, rowptr[0] != 0 or
 * rowptr[n] != nnz (GPM_E_INVALID_ARG) are rejected before any device work.
 * Synchronises `stream`.
 */
int gpm_graph_create(const uint64_t *rowptr, const uint32_t *col, uint32_t n, uint64_t nnz, uint32_t flags,
                     void *stream, gpm_graph_t *out);

/* Release every device buffer of the graph (synchronises the device). */
int gpm_graph_destroy(gpm_graph_t g);

/*
 * Build the orientation (appendix "Orientation (Total Order)": by default
 * every edge points to the endpoint of higher degree, ties to the larger id;
 * see gpm_graph_set_orientation) and the task lists used by the kernels.
 * Idempotent; called implicitly by the first count. Synchronises `stream`.
 */
int gpm_graph_prepare(gpm_graph_t g, void *stream);

/*
 * Drop the orientation and task lists so that the next prepare (or count)
 * rebuilds them from the resident CSR; device buffers are kept for reuse.
 * Used to time the whole path, orientation included, on a resident graph.
 */
int gpm_graph_reset(gpm_graph_t g);

#define GPM_ORIENT_DEGREE 0u /* edges point to the endpoint of higher degree (default) */
#define GPM_ORIENT_CORE 1u   /* core value based: the degeneracy (peeling) order */

/*
 * Choose the total order of the orientation (appendix "Orientation (Total
 * Order)": degree based, ties to the larger id; or core value based, read as
 * the degeneracy order of k-core peeling: vertices in the order the
 * level-synchronous peel removes them (by round, ties to the larger id), so
 * that no vertex has more successors than its core number). Takes effect
 * at the next prepare (the current orientation is dropped when the mode
 * changes). Totals do not depend on the order; the root of a clique or of a
 * diamond in gpm_count_roots / gpm_count_cliques follows it. The core order
 * costs a k-core peel on the device at prepare time.
 * Errors: GPM_E_INVALID_ARG for an unknown mode.
 */
int gpm_graph_set_orientation(gpm_graph_t g, uint32_t mode);

/*
 * Core number of every vertex (the largest c such that the vertex lies in a
 * subgraph of minimum degree >= c), by level-synchronous k-core peeling on
 * the device. core: uint32[n], host or device memory. Prepares the graph if
 * needed. Synchronises `stream`.
 */
int gpm_graph_core_numbers(gpm_graph_t g, uint32_t *core, void *stream);

typedef struct {
  uint32_t n;
  uint32_t max_degree;
  uint64_t nnz;
  uint64_t dag_arcs;        /* = nnz / 2 once prepared, else 0 */
  uint32_t max_out_degree;  /* largest out-degree in the orientation */
  uint32_t prepared;
  uint64_t device_bytes;    /* device memory held by the handle */
} gpm_graph_info_t;

/* Facts of a graph handle into *info (host memory, written only on success);
 * GPM_E_INVALID_ARG for a null handle or output. No device work. */
int gpm_graph_info(gpm_graph_t g, gpm_graph_info_t *info);

/* ---------------- patterns ---------------- */

/*
 * A pattern given explicitly by its k x k adjacency matrix (Section 3.1: a
 * pattern is defined by its vertices and edges; Section 2: vertex-induced or
 * edge-induced embeddings).
 *   k       : 1..8 vertices (GPM_E_K_TOO_LARGE above 8)
 *   adj     : uint8[k*k], row-major, 0/1, symmetric, zero diagonal
 *   induced : 1 = count vertex-induced embeddings (TC, k-CL, k-MC),
 *             0 = edge-induced (non-induced) embeddings (SL)
 * The pattern must be connected (GPM_E_DISCONNECTED_PATTERN). The planner
 * computes |Aut(P)|, the symmetry-breaking partial order, a matching order
 * and the execution strategy (appendix "Symmetry Breaking", "Pattern-Guided
 * Search (Matching Order)").
 */
int gpm_pattern_spec(uint32_t k, const uint8_t *adj, int induced, gpm_pattern_t *out);

/* The k-clique, k in 1..8 (Section 3.1 helper "generate clique"). */
int gpm_pattern_clique(uint32_t k, gpm_pattern_t *out);

/*
 * All connected k-vertex patterns, vertex-induced (Section 2, k-MC; the
 * helper "generate all k-vertex patterns" of Section 3.1), k = 3, 4 or 5.
 * Writes *npat handles to out[] (room for 21 must be provided), in the fixed
 * order  k=3: wedge, triangle;
 *        k=4: 3-star, 4-path, tailed triangle, 4-cycle, diamond, 4-clique;
 *        k=5: the 21 connected 5-vertex graphs by number of edges, then by
 *             their smallest pair mask over the 120 vertex orders, where the
 *             pair mask of a 5-vertex graph has bit b set for the b-th pair
 *             of (0,1), (0,2), (0,3), (0,4), (1,2), (1,3), (1,4), (2,3), (2,4),
 *             (3,4) that is an edge (so 0: 4-path, ..., 20: 5-clique).
 */
int gpm_pattern_motifs(uint32_t k, gpm_pattern_t *out, uint32_t *npat);

/* Release a pattern handle (host memory only); GPM_E_INVALID_ARG for null. */
int gpm_pattern_destroy(gpm_pattern_t p);

/* strategy chosen by the planner */
#define GPM_STRATEGY_CLIQUE_DAG 1    /* orientation + local-graph bitmap search */
#define GPM_STRATEGY_LOCAL_COUNT 2   /* local counting (Section 5) for 3/4-vertex patterns */
#define GPM_STRATEGY_EDGE 3          /* single edge / vertex: closed form */
#define GPM_STRATEGY_ENUMERATE 4     /* pattern-oblivious enumeration with connectivity codes (5 vertices) */
#define GPM_STRATEGY_GUIDED 5        /* pattern-guided search from the matching order (6..8 vertices) */

typedef struct {
  uint32_t k;
  uint32_t n_edges;
  uint32_t induced;
  uint32_t is_clique;
  uint32_t strategy;           /* GPM_STRATEGY_* */
  uint32_t motif_index;        /* position in the k = 3, 4, 5 motif order, or UINT32_MAX */
  uint64_t automorphisms;      /* |Aut(P)| */
  uint32_t n_sb_pairs;         /* symmetry-breaking constraints id(f(a)) < id(f(b)) */
  uint32_t sb_pairs[2 * 28];   /* (a_0, b_0, a_1, b_1, ...) in pattern vertex numbering */
  uint32_t matching_order[8];  /* pattern vertices in the order they are matched */
  uint32_t min_degree[8];      /* degree filter per pattern vertex (its pattern degree) */
} gpm_pattern_info_t;

/* The planner's facts of a pattern into *info (host memory, written only on
 * success); GPM_E_INVALID_ARG for a null handle or output. No device work. */
int gpm_pattern_info(gpm_pattern_t p, gpm_pattern_info_t *info);

/* ---------------- counting ---------------- */

/*
 * Exact counts of npat patterns in g (Section 2: the support of a pattern is
 * its number of embeddings; each distinct subgraph is counted once, i.e. the
 * count of maps divided by |Aut(P)|).
 *   counts : host uint64[npat]
 * Supported on the GPU: every connected pattern with up to 8 vertices,
 * induced or not (k-cliques to k = 9 through gpm_count_cliques); at most 32
 * patterns per call. Cliques run the orientation and local-graph search,
 * other 3- and 4-vertex patterns local counting, other 5-vertex patterns the
 * pattern-oblivious enumeration, other 6- to 8-vertex patterns the
 * pattern-guided search.
 * Patterns that share work are computed together (e.g. all 4-vertex motifs
 * by local counting, Section 5; 3-, 4- and 5-cliques in one pass; every
 * non-clique 5-vertex pattern of a call from one enumeration, as
 * gpm_count_enumerate). Synchronises `stream`.
 */
int gpm_count(gpm_graph_t g, const gpm_pattern_t *pats, uint32_t npat, uint64_t *counts, void *stream);

/*
 * Counts by pattern-oblivious enumeration (Section 4.2, "Memoization of
 * Embedding Connectivity"; appendix "Example for Connectivity Code"): every
 * connected induced k-vertex subgraph of g is generated once by vertex
 * extension from its smallest vertex, each added vertex carries its
 * connectivity code to the vertices before it, and the concatenated code of
 * a complete embedding selects its pattern class. An induced pattern gets
 * its class count; an edge-induced pattern gets the sum over classes of the
 * class count times the number of spanning subgraphs of the class graph that
 * are copies of the pattern. All patterns must have the same k = 3, 4 or 5
 * (GPM_E_UNSUPPORTED otherwise); the results equal gpm_count's, which for
 * k = 3, 4 takes local counting instead, so this call is an independent
 * check of it. The work grows with the number of connected k-vertex subsets,
 * which is large around high-degree vertices. counts: host uint64[npat];
 * a sum beyond 2^64 returns GPM_E_OVERFLOW. Synchronises `stream`.
 */
int gpm_count_enumerate(gpm_graph_t g, const gpm_pattern_t *pats, uint32_t npat, uint64_t *counts, void *stream);

/*
 * Counts by the pattern-guided search (appendix "Pattern-Guided Search
 * (Matching Order)", "Symmetry Breaking (Partial Order)"; Section 4.3 degree
 * filtering), for any connected pattern with 3..8 vertices, induced or not:
 * the pattern's vertices are matched in the planner's matching order
 * (gpm_pattern_info), each candidate list is the neighbour list of one
 * matched pattern neighbour intersected with the lists of the others (and
 * differenced with the non-neighbours' lists for induced patterns), bounded
 * by the symmetry-breaking id constraints and the degree filter, so each
 * distinct subgraph is matched once. gpm_count takes this path for patterns
 * with 6..8 vertices that are not cliques; this call forces it for any
 * pattern (a second, independent path for the others). One search per
 * pattern. counts: host uint64[npat]. Synchronises `stream`.
 */
int gpm_count_guided(gpm_graph_t g, const gpm_pattern_t *pats, uint32_t npat, uint64_t *counts, void *stream);

/* As gpm_count, but writes the counts to DEVICE memory `counts_dev`
 * (uint64[npat]) and does not synchronise. The graph must be prepared. */
int gpm_count_async(gpm_graph_t g, const gpm_pattern_t *pats, uint32_t npat, uint64_t *counts_dev, void *stream);

/*
 * Counts restricted to embeddings whose ROOT vertex id lies in [root_lo,
 * root_hi). Summing over a partition of [0, n) gives gpm_count's result, so a
 * root range is the unit of sharding across GPUs. Roots, with "order" the
 * orientation order (degree, id):
 *   k-clique : the clique vertex that is first in the order;
 *   diamond (edge-induced): the order-first endpoint of the shared edge;
 *   4-cycle (edge-induced): the cycle vertex that is last in the order;
 *   other 5-vertex patterns (counted by enumeration): the smallest vertex id.
 * Other patterns return GPM_E_UNSUPPORTED. counts: host uint64[npat].
 */
int gpm_count_roots(gpm_graph_t g, const gpm_pattern_t *pats, uint32_t npat, uint32_t root_lo, uint32_t root_hi,
                    uint64_t *counts, void *stream);

/*
 * k-clique count for one k = 3..9 over the roots in [root_lo, root_hi) (the
 * root of a clique is its vertex that is first in the orientation order; the
 * full range [0, n) gives the total). Section 2 k-CL with the local-graph
 * search of Section 5 ("search on local graph"): for k <= 6 the fused pass of
 * gpm_count; for k >= 7 the generic search, which keeps the shrinking
 * candidate set as a bitmap over the root's out-neighbours and switches to
 * register graphs once it has at most 32 members (their (member, successor)
 * pairs spread over the lanes). k >= 7 needs root out-degrees <= 16384
 * (GPM_E_UNSUPPORTED otherwise; every out-degree of the degree order is at
 * most sqrt(2m), so graphs of up to 134 M edges always qualify).
 *   *count : host uint64
 * Errors: GPM_E_INVALID_ARG for k outside 3..9, a bad range or a null
 * pointer. The count is accumulated in uint64 (exact below 2^64).
 * Synchronises `stream`.
 */
int gpm_count_cliques(gpm_graph_t g, uint32_t k, uint32_t root_lo, uint32_t root_hi, uint64_t *count,
                      void *stream);

/* ---------------- listing ---------------- */

/*
 * Subgraph listing (Section 2, SL): writes up to `cap` embeddings of p as
 * k-tuples, tuple t = (f(0), ..., f(k-1)) in PATTERN vertex order, into buf
 * (uint32[k*cap], host or device memory). Every written tuple is a valid
 * embedding (each pattern edge maps to a graph edge), satisfies the pattern's
 * symmetry-breaking constraints (gpm_pattern_info) and stands for a distinct
 * subgraph. Which min(total, cap) embeddings are written is unspecified.
 *   *written : number of tuples written = min(total, cap)
 *   *total   : exact number of embeddings (= gpm_count of p)
 * Supported: every connected pattern with 3..8 vertices, induced or not.
 * The edge-induced diamond and 4-cycle and the k-cliques have their own
 * kernels; every other pattern runs the pattern-guided search (see
 * gpm_count_guided). Synchronises `stream`.
 */
int gpm_list(gpm_graph_t g, gpm_pattern_t p, uint32_t *buf, uint64_t cap, uint64_t *written, uint64_t *total,
             void *stream);

/*
 * Existence query (Section 3.1: the optional early-termination condition of
 * the API, used for pattern existence): *found = 1 if g holds at least one
 * embedding of p, else 0. Runs the listing search with room for one match and
 * no counting pass, so every warp stops at its next check once a match is
 * written. witness (host uint32[k], may be NULL): on *found = 1, one
 * embedding in PATTERN vertex order, as gpm_list writes it.
 * Supported: as gpm_list (every connected pattern with 3..8 vertices).
 * Synchronises `stream`.
 */
int gpm_exists(gpm_graph_t g, gpm_pattern_t p, int *found, uint32_t *witness, void *stream);

/* ---------------- batched form ---------------- */

#define GPM_QUERY_MOTIF3 3u  /* 2 induced counts: wedge, triangle */
#define GPM_QUERY_MOTIF4 4u  /* 6 induced counts, order of gpm_pattern_motifs(4) */
#define GPM_QUERY_TC 5u      /* 1 count: triangles */
#define GPM_QUERY_CLIQUE4 6u /* 1 count: 4-cliques */
#define GPM_QUERY_CLIQUE5 7u /* 1 count: 5-cliques */

typedef struct {
  gpm_graph_t graph; /* the library prepares it if needed */
  uint32_t kind;     /* GPM_QUERY_* */
  uint32_t reserved;
} gpm_query_t;

typedef struct gpm_batch *gpm_batch_t;

/*
 * Plan a batch of queries over resident graphs (the paper's k-MC and k-CL
 * problems, Section 2, for many inputs at once). Every query is cut into work
 * items of per-root tasks; all items of all queries run in ONE persistent
 * kernel captured in a CUDA graph, pulling items from a global atomic queue,
 * so small and large queries overlap on the device. Heavy queries (plain
 * count path at least batch_direct_us on the device, timed here) instead run
 * that path inside the same captured graph, ahead of the persistent kernel;
 * so do the whole-GPU launches of hub-class 4-cycle roots of item queries.
 * The graphs must outlive the batch and must not be counted concurrently by
 * other calls while the batch runs. Roots with out-degree above 1024 are not
 * supported in item queries (GPM_E_UNSUPPORTED). Synchronises the device.
 */
int gpm_batch_create(const gpm_query_t *queries, uint32_t nq, gpm_batch_t *out);

/*
 * Run the batch: counts is host uint64[6*nq]; query i writes counts[6i ..]
 * (2, 6 or 1 values by kind, the rest 0). The first run autotunes the item
 * schedule (roots per warp item, vertices per edge item) by timing each
 * candidate once; later runs replay the captured graph. Results equal
 * gpm_count of each query alone. Ordered after `stream`; returns when done.
 */
int gpm_batch_run(gpm_batch_t b, uint64_t *counts, void *stream);

/* Schedule chosen by the autotuner and the persistent grid size. */
int gpm_batch_info(gpm_batch_t b, uint32_t *nitems, uint32_t *roots_per_item, uint32_t *verts_per_item,
                   uint32_t *grid);

/* Number of queries that run their plain count path inside the graph, and
 * kernels one replay launches. */
int gpm_batch_direct(gpm_batch_t b, uint32_t *ndirect, uint64_t *graph_kernels);

/* Release a batch and its captured graph and device buffers (synchronises
 * the batch's stream); the graphs it counts stay owned by the caller. */
int gpm_batch_destroy(gpm_batch_t b);

/* create + run + destroy. */
int gpm_count_batch(const gpm_query_t *queries, uint32_t nq, uint64_t *counts, void *stream);

/* ---------------- served form ---------------- */

typedef struct gpm_server *gpm_server_t;

typedef struct {
  uint32_t max_inflight;  /* request slots running at once (default 256) */
  uint32_t reserved0;
  uint64_t arena_bytes;   /* device arena for per-request buffers (default 4 GiB) */
  uint64_t ring_items;    /* capacity of the device work-item ring (default 8 Mi items) */
  uint64_t reserved[4];
} gpm_server_opts_t;

typedef struct {
  uint64_t tag;        /* the tag given to gpm_server_submit */
  uint32_t graph;      /* index into the server's graph list */
  uint32_t kind;       /* GPM_QUERY_* */
  int32_t status;      /* GPM_OK, GPM_E_TIMEOUT or GPM_E_OVERFLOW */
  uint32_t ncounts;    /* 1, 2 or 6 */
  uint64_t counts[6];  /* as gpm_count_batch */
} gpm_completion_t;

/*
 * Start a request loop over resident graphs (the GPM problems of Section 2
 * served continuously). A persistent kernel pulls per-root work items of all
 * admitted requests from a device ring that the host appends to while it
 * runs, so requests that arrive while others are on the GPU overlap with
 * them (continuous batching). A request is admitted when a request slot, room
 * in the item ring and, for 4-motif queries, 4 bytes per edge of the device
 * arena are free; otherwise it waits in a host FIFO. Requests of at most 64
 * items use an express ring that the kernel drains first and an express FIFO;
 * larger ones may hold at most three quarters of the slots. Hub-class 4-cycle
 * roots run as many short items over a pool of 16 shared tally slots (the
 * pool holds 16 x the largest n words). Every device-side wait is bounded; the
 * kernel exits after ~20 ms without work and is relaunched by the next submit
 * or poll. The graphs must outlive the server and must not be used by other
 * calls while it runs. Synchronises the device.
 */
int gpm_server_start(const gpm_graph_t *graphs, uint32_t ngraphs, const gpm_server_opts_t *opts,
                     gpm_server_t *out);

/* Queue a count request (kind GPM_QUERY_*) on graph index `graph`; it is
 * admitted at once when resources allow. GPM_E_BUSY: the host FIFO is full. */
int gpm_server_submit(gpm_server_t s, uint32_t graph, uint32_t kind, uint64_t tag);

/* Collect up to max finished requests (non-blocking), admit waiting requests
 * whose resources have been freed, and keep the serving kernel running while
 * work is outstanding. *n = number written to out. */
int gpm_server_poll(gpm_server_t s, gpm_completion_t *out, uint32_t max, uint32_t *n);

/* Requests in flight on the device and waiting in the host FIFO. */
int gpm_server_stats(gpm_server_t s, uint32_t *inflight, uint32_t *pending);

/* Stop the serving kernel (bounded) and release the server. */
int gpm_server_stop(gpm_server_t s);

/* ---------------- counting without device allocation ---------------- */

/*
 * Edge-induced 4-cycles of a CSR that already lives in device memory, for
 * callers that must not allocate device memory while they run: frameworks
 * whose own arena owns all device memory, jobs with a hard memory budget where
 * an allocation could fail half-way through, or latency-critical loops where
 * cudaMalloc or cudaFree would synchronise the whole device. The paper has no
 * counterpart; this entry point exists for those callers.
 *   rowptr, col : DEVICE pointers, symmetric sorted CSR as for gpm_graph_create
 *                 (trusted: not validated)
 *   count       : DEVICE pointer to one uint64 that receives the count
 * Every intermediate buffer is carved from one fixed array that is part of the
 * library image: 64 MiB per GPU, held by every GPU that loads the library until
 * the process exits. A graph needs 3n + 64 words of it, so n is limited to
 * 5,592,384 vertices; a larger n returns GPM_E_INVALID_ARG with a message and
 * launches nothing. No cudaMalloc, cudaFree or other allocating call is made.
 * The first call on a device looks up the array's device address (with that
 * device current), so make that first call before any stream capture begins.
 * All calls share the one array and the array keeps the previous call's
 * contents (the entry point clears what must start at zero): calls whose work
 * overlaps on the GPU, from any stream or thread, race and give wrong counts.
 * Asynchronous on `stream`; the result equals gpm_count of the edge-induced
 * 4-cycle pattern.
 */
int gpm_count_cycles4_noalloc(const uint64_t *rowptr, const uint32_t *col, uint32_t n, uint64_t *count, void *stream);

/* ---------------- diagnostics ---------------- */

/* Message for the last error on the calling host thread ("" if none). */
const char *gpm_last_error(void);

/* Library version string. */
const char *gpm_version(void);

/* Number of kernels this library has launched in this process. */
uint64_t gpm_kernel_launches(void);

/*
 * Per-kernel timing: while enabled, every kernel launch of the library is
 * bracketed by CUDA events on its launching stream. gpm_profile_report()
 * writes {"<kernel>": {"launches": L, "ms": T}, ...} (JSON, NUL-terminated,
 * truncated to len; *needed = full size) summed since the last reset; call it
 * after synchronising the streams involved.
 */
int gpm_profile_enable(int on);
int gpm_profile_reset(void);
int gpm_profile_report(char *buf, size_t len, size_t *needed);

/* Tuning knobs for tests and the autotuner (0 = leave unchanged). */
typedef struct {
  uint32_t warp_max_degree; /* roots with out-degree <= this run one per warp */
  uint32_t cta_max_degree;  /* ... <= this one per CTA in shared memory; larger: global-memory bitmaps */
  uint32_t blocks_per_sm;   /* persistent grid size multiplier */
  uint32_t c4_hub_bound;    /* 4-cycle roots whose wedge bound (sum of the degrees of their neighbours
                               before them) exceeds this are counted by the whole GPU a few at a time;
                               range [513, 1048576], default 1048576. The batched and served forms use it
                               always, the plain count path only with c4_range_bound and c4_pull_bound
                               both 0xffffffff */
  uint32_t batch_direct_us; /* batched form: a query whose plain count path takes at least this many
                               microseconds on the device (timed when the batch is created) runs that
                               path inside the captured graph instead of as items; default 1000,
                               0xffffffff = never */
  uint32_t c4_range_bound;  /* plain count path (graphs of maximum degree <= 65535 and fewer than 2^32
                               adjacency entries): 4-cycle roots whose wedge bound exceeds this, up to
                               c4_pull_bound, are counted range by range over vertex ids with a dense
                               shared-memory tally; roots between 512 and the smaller of the two bounds
                               are bucketed; range [512, 0xfffffffe], default 1048576; 0xffffffff = never */
  uint32_t c4_range_width;  /* vertex ids per tally range of that path: even, in [64, 98304], default 98304 */
  uint32_t c4_pull_bound;   /* plain count path: 4-cycle roots whose wedge bound exceeds this are counted
                               128 at a time by one pass over every adjacency list with bit-sliced
                               counters; range [512, 0xfffffffe], default 262144; 0xffffffff = never.
                               With both bounds 0xffffffff the bucketed class goes up to c4_hub_bound and
                               the hub class takes the larger roots */
} gpm_options_t;

/* Process-wide: gpm_set_options applies every non-zero field (GPM_E_INVALID_ARG,
 * and nothing applied, when a field is outside its range); graphs rebuild the
 * task classes that depend on a changed field at their next count.
 * gpm_get_options writes the values in force. */
int gpm_set_options(const gpm_options_t *opt);
int gpm_get_options(gpm_options_t *opt);

#ifdef __cplusplus
}
#endif
#endif /* GPM_H_ */
