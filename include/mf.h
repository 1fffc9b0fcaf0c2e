/*
 * mf.h -- C ABI of the GB300 dynamic max-flow library (libmfgpu.so).
 *
 * The library keeps one flow network resident in GPU memory and maintains its
 * maximum s-t flow under batches of edge-capacity changes, by the Dynamic Push
 * Relabel method of "Efficient Dynamic MaxFlow Computation on GPUs"
 * (arXiv 2511.05895): Algorithm 5 (updates processing), Algorithm 4 (dynamic
 * push-relabel: source re-saturation, deficient vertices as extra sinks, loop
 * of backward BFS / PushRelabel / RemoveInvalidEdges), Algorithms 2 and 3
 * (the two kernels), and Algorithm 1 (static solve from zero flow).
 *
 * Conventions for every function:
 *  - Return value: MF_OK (0) or one of the MF_E* codes below; mf_strerror()
 *    names it.  A NULL graph or output pointer gives MF_EINVAL.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Work is enqueued on it and the call returns without
 *    waiting, except where a function says it synchronises.
 *  - Integer widths: vertex ids int32, edge ids int32 (m < 2^31), edge
 *    capacities int32 >= 0, excess and flow values int64.
 *  - Ownership: the library copies every input array; the caller keeps its
 *    buffers.  Output buffers are allocated by the caller.  The graph owns
 *    its device memory until mf_destroy().
 *  - Thread safety: calls on one graph must not run concurrently from several
 *    host threads; distinct graphs are independent.
 */
#ifndef MF_H
#define MF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes -------------------------------------------------------- */
#define MF_OK          0
#define MF_EINVAL      1  /* bad argument or bad batch content (state unchanged) */
#define MF_ENOMEM      2  /* device or host allocation failed                     */
#define MF_ECUDA       3  /* a CUDA runtime call failed                            */
#define MF_ENOTSOLVED  4  /* updates or queries before a successful mf_solve       */
#define MF_ETIMEOUT    5  /* the device loop reached max_iters or a device wait
                             reached its time limit; state invalid until mf_solve */

/* ---- flags of mf_apply_updates / mf_min_cut / export / import ------------ */
#define MF_HOST_PTRS    0x0  /* pointer arguments are host memory (default)      */
#define MF_DEVICE_PTRS  0x1  /* pointer arguments are device memory              */
#define MF_DELTA        0x2  /* new_cap[i] is a signed change; the new capacity
                                is max(0, old + new_cap[i])                      */
#define MF_RECOMPUTE    0x4  /* write the new capacities, then solve from zero
                                flow (the static recompute of Sec. 6.1) instead
                                of the dynamic repair                            */

/* ---- processing modes (Sec. 5.2 / 5.3) ---------------------------------- */
#define MF_MODE_DATA_DRIVEN 0  /* worklist of active vertices (Sec. 5.3)         */

typedef struct mf_graph mf_graph;

/* Options.  Initialise with mf_options_default() and override fields.
 *  kernel_cycles  KERNELCYCLES of Algorithm 2: push/relabel steps per active
 *                 vertex between two global relabels.  0 = max(1, round(m/n)),
 *                 the average degree used in Sec. 6.1.
 *  mode           MF_MODE_DATA_DRIVEN.
 *  max_iters      cap on loop iterations (one BFS + PushRelabel +
 *                 RemoveInvalidEdges round) of one solve or repair; reaching
 *                 it reports MF_ETIMEOUT.  0 = 4 * n + 1000.
 *  grid_blocks    CTAs of the persistent solver kernel; 0 = one full wave
 *                 (co-resident CTAs per SM x SM count).  Larger values are
 *                 clamped to one full wave.
 *  time_limit_ms  wall-clock limit of one solve/repair kernel, checked once
 *                 per loop iteration; passing it reports MF_ETIMEOUT.
 *                 0 = 60000.
 *  alloc / free   device allocator callbacks (both NULL = cudaMalloc/cudaFree).
 *                 alloc(bytes, ctx) returns a device pointer or NULL. */
typedef struct mf_options {
    int32_t kernel_cycles;
    int32_t mode;
    int64_t max_iters;
    int32_t grid_blocks;
    int32_t time_limit_ms;
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *alloc_ctx;
} mf_options;

/* Counters of the last mf_solve / mf_apply_updates (device-side counts).
 *  iterations   BFS + push/relabel rounds of the device loop (Alg. 1/4 while)
 *  bfs_levels   BFS levels over all iterations
 *  bfs_vertices vertices reached by the BFS (sum over iterations)
 *  bfs_arcs     arcs scanned by the BFS
 *  worklist     active vertices processed (sum of worklist sizes)
 *  pr_arcs      arcs scanned by PushRelabel (Alg. 2)
 *  pushes, relabels   Alg. 2 operations
 *  ri_arcs, ri_moves  arcs scanned / saturated by RemoveInvalidEdges (Alg. 3)
 *  batch        entries of the last batch (0 for mf_solve)
 *  clamped      arcs whose residual went negative and was clamped (Alg. 5)
 *  resat_arcs   source arcs scanned by the re-saturation step (Alg. 4)
 *  t_*_ns       device time per phase (globaltimer between grid barriers):
 *               batch + re-saturation, height init, BFS, warp PushRelabel,
 *               hub PushRelabel cycles, RemoveInvalidEdges
 *  hub_cycles   cooperative PushRelabel cycles of high-degree vertices
 *  barriers     grid barriers passed
 *  bfs_bottom_up_levels  BFS levels run bottom-up (direction-optimising)
 *  pr_rounds    PushRelabel activation rounds (vertices made active by a push
 *               are processed in the next round of the same iteration) */
typedef struct mf_stats {
    int64_t flow;
    int64_t iterations;
    int64_t bfs_levels;
    int64_t bfs_vertices;
    int64_t bfs_arcs;
    int64_t worklist;
    int64_t pr_arcs;
    int64_t pushes;
    int64_t relabels;
    int64_t ri_arcs;
    int64_t ri_moves;
    int64_t batch;
    int64_t clamped;
    int64_t resat_arcs;
    int64_t n;
    int64_t m;
    int64_t arcs;
    int64_t t_batch_ns;
    int64_t t_reset_ns;
    int64_t t_bfs_ns;
    int64_t t_pr_ns;
    int64_t t_hub_ns;
    int64_t t_ri_ns;
    int64_t hub_cycles;
    int64_t barriers;
    int64_t bfs_bottom_up_levels;
    int64_t pr_rounds;
    int32_t status;
    int32_t kernel_cycles;
    int32_t grid_blocks;
    int32_t block_threads;
} mf_stats;

/* Fill *opt with the defaults described above. */
int mf_options_default(mf_options *opt);

/* Build the resident graph (Bi-CSR of Sec. 5.1: for every vertex one arc per
 * distinct neighbour in either direction, with the paired reverse arc; a
 * missing direction gets capacity 0; parallel edges share their arc and
 * their capacities add).
 *   n        vertices, >= 2
 *   m        edges; edge id = position in the CSR below, 0 <= m < 2^31
 *   row_ptr  [n+1] int64, edges of vertex u are row_ptr[u] .. row_ptr[u+1]-1
 *   col      [m] int32 head of each edge, 0 <= col < n; self-loops are kept
 *            as edge ids but carry no flow
 *   cap      [m] int32 capacity >= 0
 *   s, t     source and sink, s != t
 *   opt      options or NULL for the defaults
 *   stream   stream for the uploads
 *   out      receives the graph handle
 * Host or device pointers are both accepted for row_ptr/col/cap.  The sum of
 * the capacities sharing one arc pair must stay below 2^31 for every capacity
 * up to the limit that mf_cap_limit() reports; larger capacities are rejected
 * here and in mf_apply_updates.  Synchronises `stream` before returning.  The
 * graph starts unsolved (call mf_solve). */
int mf_create(int32_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
              const int32_t *cap, int32_t s, int32_t t, const mf_options *opt,
              void *stream, mf_graph **out);

/* Largest capacity a single edge may take in this graph. */
int mf_cap_limit(const mf_graph *g, int32_t *out);

/* Static max-flow from zero flow on the current capacities (Algorithm 1:
 * residuals reset to the capacities, source arcs saturated, then the device
 * loop).  Asynchronous; read the result with mf_flow_value. */
int mf_solve(mf_graph *g, void *stream);

/* Apply a batch of capacity changes and repair the max flow (Algorithms 5
 * and 4), or recompute it from zero flow when flags has MF_RECOMPUTE.
 *   k         batch entries, 0 <= k <= m
 *   edge_id   [k] int32 distinct edge ids in [0, m)
 *   new_cap   [k] int32 new capacity >= 0 (or signed change with MF_DELTA)
 *   flags     MF_HOST_PTRS or MF_DEVICE_PTRS, optionally | MF_DELTA, MF_RECOMPUTE
 * Asynchronous.  Host batches are copied to the device on `stream` first.
 * Batch contents (id range, duplicate ids, capacity range) are validated on
 * the device before anything changes; a bad batch leaves the state unchanged
 * and the next mf_flow_value / mf_sync reports MF_EINVAL.  Requires a solved
 * graph (MF_ENOTSOLVED otherwise). */
int mf_apply_updates(mf_graph *g, int64_t k, const int32_t *edge_id, const int32_t *new_cap,
                     int32_t flags, void *stream);

/* Wait for the graph's work and report the status of the last solve/repair:
 * MF_OK, MF_EINVAL (rejected batch, reported once), MF_ETIMEOUT. */
int mf_sync(mf_graph *g);

/* Max-flow value of the current state (Algorithm 4's final sum: excess of t
 * plus the excess of every deficient vertex; Algorithm 1: e(t)).
 * Synchronises; returns the status of the last solve/repair like mf_sync. */
int mf_flow_value(mf_graph *g, int64_t *out);

/* Minimum cut: side[v] = 1 if v is on the source side S = {h(v) >= n}
 * (Note 1 of Sec. 3), else 0.  side is [n] bytes, host or device per flags.
 * Synchronises. */
int mf_min_cut(mf_graph *g, uint8_t *side, int32_t flags);

/* Counters of the last solve/repair.  Synchronises. */
int mf_stats_get(mf_graph *g, mf_stats *out);

/* Sizes of the resident structure: vertices, edges, arcs. */
int mf_sizes(const mf_graph *g, int32_t *n, int64_t *m, int64_t *arcs);

/* Copy the resident Bi-CSR out (host buffers, any may be NULL):
 * arc_row [n+1] int64, head/rev/cap [arcs] int32 (cap = current arc
 * capacity, the sum of the edges it carries).  Synchronises. */
int mf_export_graph(mf_graph *g, int64_t *arc_row, int32_t *head, int32_t *rev, int32_t *cap);

/* Checkpoint: copy residuals r [arcs] int32, excess [n] int64 and heights
 * [n] int32 out (host or device buffers per flags; any may be NULL).
 * Synchronises. */
int mf_export_state(mf_graph *g, int32_t *r, int64_t *excess, int32_t *height, int32_t flags);

/* Resume: load residuals, excess and heights previously exported from a
 * graph built from the same inputs with the same current capacities.  The
 * graph is then treated as solved.  Synchronises. */
int mf_import_state(mf_graph *g, const int32_t *r, const int64_t *excess, const int32_t *height,
                    int32_t flags);

/* Free all device memory of the graph (synchronises first).  NULL is a no-op. */
void mf_destroy(mf_graph *g);

/* Allocation-free static max-flow on a Bi-CSR that the caller already holds in
 * device memory.  The paper has no counterpart: it is for callers that must
 * not allocate GPU memory themselves -- for example a plugin that runs inside
 * another framework which owns all device memory through its own pool, or a
 * service path where allocations are forbidden after start-up -- and so
 * cannot use mf_create.  Instead of allocating, it works in one static
 * device array of 12,943,872 bytes (about 12.3 MiB) that every GPU which
 * loads this library holds until the process exits.
 *   n, arcs        vertices (2 .. 131072) and Bi-CSR arcs (0 .. 2097152);
 *                  larger graphs are rejected with MF_EINVAL
 *   row [n+1], head/rev/cap [arcs]   the Bi-CSR of mf_bicsr_host, int32,
 *                  device memory, read only
 *   s, t           source and sink
 *   kernel_cycles  as mf_options (0 = default)
 *   r [arcs] int32, excess [n] int64, height [n] int32: device outputs --
 *                  the final residuals, excesses and heights (the min cut is
 *                  {v : height[v] >= n})
 *   flow           HOST int64 receiving the max-flow value
 *   stream         stream for the work (NULL = legacy default stream)
 * Synchronises `stream` and returns MF_OK, MF_EINVAL, MF_ECUDA or
 * MF_ETIMEOUT.  It calls no cudaMalloc or cudaFree.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) and the
 * kernel's grid size; make that first call before any stream capture.  All
 * calls share the one array and it keeps the last call's contents (each call
 * clears what must start at zero): calls that overlap on the GPU -- from
 * several host threads or on several streams -- race and must be serialised
 * by the caller. */
int mf_solve_bicsr_noalloc(int32_t n, int64_t arcs, const int32_t *row, const int32_t *head,
                           const int32_t *rev, const int32_t *cap, int32_t s, int32_t t,
                           int32_t kernel_cycles, int32_t *r, int64_t *excess, int32_t *height,
                           int64_t *flow, void *stream);

/* Static string naming an error code. */
const char *mf_strerror(int code);

/* Detail of the last failure reported to the calling host thread (a CUDA
 * error string, the rejected argument, ...).  Valid until the next call. */
const char *mf_last_error(void);

/* Host-only construction of the Bi-CSR that mf_create uploads (Sec. 5.1);
 * needs no GPU.  Call once with all output pointers NULL to learn *arcs,
 * then again with buffers: arc_row [n+1] int64, head/rev/arc_cap [arcs]
 * int32, arc_of_edge [m] int32 (-1 for a self-loop), *cap_limit as
 * mf_cap_limit.  Inputs as mf_create (host pointers only). */
int mf_bicsr_host(int32_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                  const int32_t *cap, int32_t s, int32_t t, int64_t *arcs, int64_t *arc_row,
                  int32_t *head, int32_t *rev, int32_t *arc_cap, int32_t *arc_of_edge,
                  int32_t *cap_limit);

/* Library version, e.g. "0.1.0". */
const char *mf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MF_H */
