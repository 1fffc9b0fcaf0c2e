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
#define MF_ECHECK      6  /* a device-side consistency check of debug_checks
                             failed (an out-of-range list entry, or an excess,
                             residual pair or residual mirror that disagrees
                             with the arcs); state invalid until mf_solve    */

/* ---- flags of mf_apply_updates / mf_min_cut / export / import ------------ */
#define MF_HOST_PTRS    0x0  /* pointer arguments are host memory (default)      */
#define MF_DEVICE_PTRS  0x1  /* pointer arguments are device memory              */
#define MF_DELTA        0x2  /* new_cap[i] is a signed change; the new capacity
                                is max(0, old + new_cap[i])                      */
#define MF_RECOMPUTE    0x4  /* write the new capacities, then solve from zero
                                flow (the static recompute of Sec. 6.1) instead
                                of the dynamic repair                            */

/* ---- batch policies (mf_set_policy) ----------------------------------------
 * FIXED    always the dynamic repair with the graph's KERNELCYCLES (default)
 * PLAIN    dynamic repair when the batch holds at most 1 % of the edges,
 *          else a static recompute; KERNELCYCLES = average degree (Sec. 6.1)
 * LEARNED  the policy network (mf_mlp_*) chooses repair or recompute,
 *          KERNELCYCLES and the processing mode of the repair (data-driven,
 *          topology-driven, or -- on a graph created with MF_MODE_PUSH_PULL,
 *          which keeps the exact cut that Alg. 8 starts from -- Dynamic
 *          Push-Pull; on other graphs a push-pull choice runs data-driven)
 *          from 12 batch features; it falls back to PLAIN (and the graph's
 *          own mode) on any non-finite or out-of-range input */
#define MF_POLICY_FIXED   0
#define MF_POLICY_PLAIN   1
#define MF_POLICY_LEARNED 2

/* ---- processing modes (Sec. 5.2 / 5.3) ---------------------------------- */
#define MF_MODE_DATA_DRIVEN 0  /* worklist of active vertices (Sec. 5.3)         */
#define MF_MODE_TOPOLOGY    1  /* every push/relabel round visits every vertex
                                  id and serves the active ones, with no
                                  worklist (Sec. 5.2)                          */
#define MF_MODE_PUSH_PULL   2  /* repairs by Dynamic Push-Pull (Alg. 8, Sec. 4.2):
                                  saturate the arcs across the previous cut,
                                  push on its sink side and pull on its source
                                  side concurrently, then push on the leftover
                                  subgraph P.  Needs the exact cut of the
                                  previous state, which every job of such a
                                  graph keeps by ending on a BFS.  exit_kind 3
                                  marks a push-pull repair.  Solves from zero
                                  flow (mf_solve, MF_RECOMPUTE) use static
                                  push-pull (Sec. 4.2): the arcs into t are
                                  saturated too and the vertices left deficient
                                  are sinks of the loop.                       */

typedef struct mf_graph mf_graph;

/* Options.  Initialise with mf_options_default() and override fields.
 *  kernel_cycles  KERNELCYCLES of Algorithm 2: push/relabel steps per active
 *                 vertex between two global relabels.  0 = max(1, round(m/n)),
 *                 the average degree used in Sec. 6.1.
 *  mode           MF_MODE_DATA_DRIVEN (default), MF_MODE_TOPOLOGY or
 *                 MF_MODE_PUSH_PULL.
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
 *                 alloc(bytes, ctx) returns a device pointer or NULL.
 *  debug_checks   non-zero: every solve/repair kernel checks the vertex ids it
 *                 reads from its lists and queues (out of range: the entry is
 *                 skipped) and, at its end, re-derives the state's invariants
 *                 over all arcs -- e(v) = sum over v's arcs of (r - cap) (the
 *                 incremental excess of the repair equals the full recount of
 *                 Alg. 4 line 2), r >= 0, r(a) + r(rev a) = cap(a) + cap(rev a),
 *                 and the residual mirror; a failure sets a status bit that
 *                 mf_flow_value reports as MF_ECHECK.  Never traps.  Costs one
 *                 O(arcs) pass per kernel.  0 = off. */
typedef struct mf_options {
    int32_t kernel_cycles;
    int32_t mode;
    int64_t max_iters;
    int32_t grid_blocks;
    int32_t time_limit_ms;
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *alloc_ctx;
    int32_t debug_checks;
} mf_options;

/* Counters of the last mf_solve / mf_apply_updates (device-side counts).
 *  iterations   loop iterations that ran PushRelabel (Alg. 1/4 while loop)
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
 *  pr_rounds    PushRelabel activation generations: in the topology-driven
 *               mode the rounds (a vertex made active by a push is served in
 *               the next round of the same iteration); in the data-driven and
 *               push-pull modes the highest generation of the activation
 *               queue (a vertex made active is queued at once with the
 *               pusher's generation + 1) plus one, summed over the phases
 *  policy_*     last policy decision: kind 0 = repair, 1 = recompute; the
 *               KERNELCYCLES chosen; 1 if the learned policy fell back
 *  exit_kind    how the loop ended: 0 = a BFS found no active vertex; 1 = the
 *               last PushRelabel/RemoveInvalidEdges round left no active
 *               vertex under its own (valid) heights, so no final BFS ran;
 *               2 = the batch only raised capacities of arcs that do not
 *               cross the last exact cut, so the flow value cannot change
 *               and no loop ran; 3 = a Dynamic Push-Pull repair
 *               (MF_MODE_PUSH_PULL).  After 1, 2 or 3 the heights are not the
 *               BFS fixed point; mf_min_cut and mf_export_state recompute
 *               them first (one BFS). */
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
    int32_t policy_kind;
    int32_t policy_kernel_cycles;
    int32_t policy_fallback;
    int32_t exit_kind;
    int32_t status;
    int32_t kernel_cycles;
    int32_t grid_blocks;
    int32_t block_threads;
    int32_t policy_mode;      /* processing mode the policy chose for the last
                                 batch (MF_MODE_*; the graph's own without a
                                 learned policy)                             */
    int32_t reserved0;
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

/* mf_apply_updates for a batch whose size lives in device memory (*k_dev,
 * int32, at most k_max) with device arrays edge_id / new_cap: nothing in the
 * call depends on host values, so it can be captured in a CUDA graph and
 * replayed for every batch (the batch-sequence stamps are kept on the
 * device).  Size the staging first with one call outside the capture (or a
 * call of mf_apply_updates with k >= k_max).  Flags: MF_DELTA,
 * MF_RECOMPUTE. */
int mf_apply_updates_dev(mf_graph *g, const int32_t *k_dev, int64_t k_max, const int32_t *edge_id,
                         const int32_t *new_cap, int32_t flags, void *stream);

/* Enqueue on `stream` the copy of the last solve/repair's status and value
 * into result[0..1] (host memory, preferably pinned): result[0] low 32 bits =
 * status bits (1 rejected batch, 2 iteration cap, 4 device wait limit,
 * 8 wall-clock limit; 0 = success), result[1] = flow value.  Does not wait. */
int mf_flow_value_async(mf_graph *g, int64_t *result, void *stream);

/* Wait for the graph's work, then make `stream` (NULL = legacy default
 * stream) the stream that later synchronising calls wait on.  Call it before
 * destroying a stream the graph last ran on. */
int mf_set_stream(mf_graph *g, void *stream);

/* Device memory the graph holds (bytes). */
int mf_device_bytes(const mf_graph *g, int64_t *bytes);

/* CTAs of the graph's persistent kernel (options.grid_blocks after clamping). */
int mf_grid_blocks(const mf_graph *g, int32_t *blocks);

/* CTAs of the graph's following solve/repair launches (clamped to one full
 * wave; a launch captured in a CUDA graph keeps the size it was captured
 * with).  Any size gives the same results; fewer CTAs leave SMs to other
 * graphs' repairs.  Does not synchronise.  MF_EINVAL if blocks < 1. */
int mf_set_grid_blocks(mf_graph *g, int32_t blocks);

/* Wait for the graph's work and report the status of the last solve/repair:
 * MF_OK, MF_EINVAL (rejected batch, reported once), MF_ETIMEOUT. */
int mf_sync(mf_graph *g);

/* Max-flow value of the current state (Algorithm 4's final sum: excess of t
 * plus the excess of every deficient vertex; Algorithm 1: e(t)).
 * Synchronises; returns the status of the last solve/repair like mf_sync. */
int mf_flow_value(mf_graph *g, int64_t *out);

/* Minimum cut: side[v] = 1 if v is on the source side S = {h(v) >= n}
 * (Note 1 of Sec. 3), else 0, with h the exact BFS heights (recomputed by one
 * device BFS if the last solve stopped without one; see exit_kind).  side is
 * [n] bytes, host or device per flags.  Synchronises. */
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
 * [n] int32 out (host or device buffers per flags; any may be NULL).  The
 * heights are the exact BFS heights (recomputed first when needed, as for
 * mf_min_cut).  Synchronises. */
int mf_export_state(mf_graph *g, int32_t *r, int64_t *excess, int32_t *height, int32_t flags);

/* Resume: load residuals, excess and heights previously exported from a
 * graph built from the same inputs with the same current capacities.  The
 * graph is then treated as solved.  Synchronises. */
int mf_import_state(mf_graph *g, const int32_t *r, const int64_t *excess, const int32_t *height,
                    int32_t flags);

/* Change the wall-clock limit of the graph's following solve/repair kernels
 * (time_limit_ms of mf_options; 0 = 60000).  Takes effect at the next launch;
 * does not synchronise.  Returns MF_EINVAL for a negative value. */
int mf_set_time_limit(mf_graph *g, int32_t time_limit_ms);

/* Free all device memory of the graph (synchronises first).  NULL is a no-op. */
void mf_destroy(mf_graph *g);

/* Allocation-free static max-flow on a Bi-CSR that the caller already holds in
 * device memory.  The paper has no counterpart: it is for callers that must
 * not allocate GPU memory themselves -- for example a plugin that runs inside
 * another framework which owns all device memory through its own pool, or a
 * service path where allocations are forbidden after start-up -- and so
 * cannot use mf_create.  Instead of allocating, it works in one static
 * device array of 14,288,384 bytes (about 13.6 MiB) that every GPU which
 * loads this library holds until the process exits.
 *   n, arcs        vertices (2 .. 131072) and Bi-CSR arcs (0 .. 2097152);
 *                  larger graphs are rejected with MF_EINVAL
 *   row [n+1], head/rev/cap [arcs]   the Bi-CSR of mf_bicsr_host, int32,
 *                  device memory, read only, head and r 16-byte aligned for
 *                  the fastest path (any alignment works).  mf_bicsr_host
 *                  returns the offsets arc_row as int64: the caller narrows
 *                  them to int32 for row (they fit, arcs <= 2097152).  The
 *                  arrays must be mf_bicsr_host's output unchanged (row[n] ==
 *                  arcs, heads in range, rev an involution pairing u -> v with
 *                  v -> u): they are not validated, and inconsistent arrays
 *                  make the kernel read out of bounds.
 *   s, t           source and sink
 *   kernel_cycles  as mf_options; 0 = the average Bi-CSR degree
 *                  max(1, round((arcs / 2) / n)), computed from arcs because
 *                  the input edge count is not passed: where the Bi-CSR merged
 *                  antiparallel edges it can differ from mf_create's default
 *                  (same values, other timings) -- pass it explicitly to match
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

/* Choose how mf_apply_updates handles batches (MF_POLICY_*).  params: host
 * array of the network (mf_mlp_sizes' n_total floats, layout in
 * csrc/mf_mlp.cuh), required the first time LEARNED is set, copied; NULL
 * keeps the loaded one.  MF_RECOMPUTE in a call's flags still forces a
 * static recompute.  Synchronises when params is given. */
int mf_set_policy(mf_graph *g, int32_t mode, const float *params);

/* The 12 policy features of a batch for this graph (what the network sees):
 * log2 n, log2 m, log2(1+k), k/m, share of increments, share of edges out of
 * s or into t, log2(1 + sum |change|), log2(1 + last flow value), average
 * Bi-CSR degree, log2(1 + largest degree), loop iterations of the last
 * solve/repair, share of vertices its BFS reached per iteration.  Batch as in
 * mf_apply_updates (flags MF_DEVICE_PTRS, MF_DELTA); features: host [12].
 * Changes nothing.  Synchronises. */
int mf_policy_features(mf_graph *g, int64_t k, const int32_t *edge_id, const int32_t *new_cap,
                       int32_t flags, float *features);

/* ---- the policy network (device arrays, float32, stream-ordered) -------
 * Sizes: inputs 12, outputs 5 (repair-vs-recompute logit, log2
 * KERNELCYCLES, and the logits of the processing modes data-driven,
 * topology-driven, push-pull), trained parameters, all parameters (with the
 * input normalisation mu[12], sd[12] at the end). */
int mf_mlp_sizes(int32_t *n_in, int32_t *n_out, int32_t *n_trained, int32_t *n_total);

/* Bytes of the caller-provided workspace for mini-batches of `batch`. */
int64_t mf_mlp_workspace_bytes(int32_t batch);

/* Y[n x 5] = network(X[n x 12]); P: n_total parameters. */
int mf_mlp_forward(const float *P, const float *X, int32_t n, float *Y, void *stream);

/* Gradient (grad [n_trained]) and value (loss [1]) over all n samples of the
 * mean loss BCE(y0, t0) + wkc * (y1 - t1)^2 / 2 + wmode * CE(softmax(y2..y4),
 * t2), t2 the index 0/1/2 of the target mode stored as a float.  workspace:
 * mf_mlp_workspace_bytes(n). */
int mf_mlp_grad(const float *P, const float *X, const float *T0, const float *T1, const float *T2, int32_t n,
                float wkc, float wmode, float *grad, float *loss, void *workspace, void *stream);

/* `steps` Adam steps (lr; betas 0.9, 0.999) on mini-batches of `batch`
 * consecutive samples taken cyclically from X/T0/T1/T2 (shuffle beforehand).
 * M, V: Adam moments [n_trained] (zero before the first step); step0: steps
 * taken before (for the bias correction).  loss_hist [steps] or NULL receives
 * each mini-batch loss.  workspace: mf_mlp_workspace_bytes(batch). */
int mf_mlp_train(float *P, float *M, float *V, const float *X, const float *T0, const float *T1, const float *T2,
                 int32_t n, int32_t steps, int32_t batch, float lr, float wkc, float wmode, int32_t step0,
                 float *loss_hist, void *workspace, void *stream);

/* ---- serving several resident graphs (continuous batching) --------------
 * A server owns a scheduler thread.  Graphs (created, policy set and solved
 * beforehand; each with its own grid size, mf_options.grid_blocks) are added
 * to it; batches are submitted from host arrays and complete asynchronously.
 * A request is admitted when its graph has no repair in flight, the CTAs of
 * all repairs in flight stay within sm_slots (so that their persistent grids
 * are co-resident and overlap), and their device staging fits the HBM budget
 * left after the resident graphs; requests that do not fit wait while later
 * ones for other graphs may start (a graph's own requests keep their
 * order).  A request's repair runs on a grid sized to its batch: the graph's
 * full grid for batches above 20,000 entries and for recomputes, half of it
 * above 2,000 entries, a quarter below (at least one CTA), so that small
 * repairs are admitted beside large ones -- but graphs of 2^21 vertices or
 * more always take their full grid and graphs of 2^19 or more at least half
 * (every repair runs a BFS over the whole graph).  Each
 * graph's repair and recompute are captured once per grid size in CUDA
 * graphs and replayed (use_cuda_graphs; if a capture fails the server
 * launches that case directly and reports fewer captured graphs; up to six
 * per graph).  A graph belongs to the server once added: call nothing else
 * on it until mf_server_destroy, and destroy the server before its graphs. */
typedef struct mf_server mf_server;
typedef struct mf_server_options {
    int64_t hbm_budget_bytes;   /* 0 = the device's total memory                  */
    int32_t sm_slots;           /* CTAs of all repairs in flight; 0 = SM count    */
    int32_t use_cuda_graphs;    /* 1 (default) = replay captured repairs          */
} mf_server_options;
typedef struct mf_server_stats {
    int64_t submitted, completed, failed;
    int32_t max_inflight;       /* most repairs in flight at once                 */
    int32_t graphs, captured_graphs;  /* captured: CUDA graphs instantiated      */
    int32_t reserved;
    double p50_us, p99_us, mean_us;  /* submit-to-completion latency             */
    double makespan_s;          /* first submit to last completion                */
    int64_t replays;            /* requests served by replaying a captured graph  */
    int64_t direct_launches;    /* requests launched without a captured graph     */
} mf_server_stats;

int mf_server_options_default(mf_server_options *opt);
int mf_server_create(const mf_server_options *opt, mf_server **out);
/* Add a solved graph; max_batch bounds its batches.  MF_ENOMEM if it does not
 * fit the HBM budget, MF_EINVAL if its grid exceeds sm_slots.  *index
 * receives the graph's number for mf_server_submit.  Synchronises. */
int mf_server_add_graph(mf_server *s, mf_graph *g, int64_t max_batch, int32_t *index);
/* Queue a batch (host arrays, copied) for graph `graph`; flags MF_DELTA,
 * MF_RECOMPUTE.  *ticket identifies the request. */
int mf_server_submit(mf_server *s, int32_t graph, int64_t k, const int32_t *edge_id, const int32_t *new_cap,
                     int32_t flags, int64_t *ticket);
/* *done = 1 once the request completed; then *flow, *code (MF_OK, MF_EINVAL,
 * MF_ETIMEOUT, MF_ECUDA) and *latency_us (submit to completion) are set. */
int mf_server_poll(mf_server *s, int64_t ticket, int32_t *done, int64_t *flow, int32_t *code,
                   double *latency_us);
/* Wait until every submitted request completed.  Returns MF_OK once they
 * have, whether or not they succeeded: each request's code comes from
 * mf_server_poll, and mf_server_stats counts the failed ones. */
int mf_server_drain(mf_server *s);
int mf_server_stats_get(mf_server *s, mf_server_stats *out);
/* Forget the latencies and counts of completed requests. */
void mf_server_reset_stats(mf_server *s);
/* Wait for all requests, stop the thread, free the server's resources (the
 * graphs stay; destroy them afterwards). */
void mf_server_destroy(mf_server *s);

/* Tracing: one record per grid barrier of the solve/repair kernel, and one
 * per BFS level that CTA 0 ran alone (no grid barrier).
 *   phase  MF_PHASE_*; mode: BFS 0 top-down frontier, 1 top-down items of
 *          high-degree vertices, 2 bottom-up groups, 3 bottom-up items,
 *          4 a level of a small frontier run by CTA 0 alone (not a barrier),
 *          6 / 5 the barriers before and after such a run; hub
 *          cycles 0 set-up, 1 lowest-neighbour scan, 3 pushes;
 *          RemoveInvalidEdges: why the loop went on to another BFS, bits
 *          1 the activation rounds or generations reached their cap (or
 *          the activation queue was full), 2 the hub cycles
 *          reached theirs, 4 an arc was saturated, 8 a push re-activated a
 *          high-degree vertex (0: it stopped; a height-init record of step 1,
 *          the recount of the deficits, follows)
 *   iter   loop iteration (-1 before the loop), step: BFS level, activation
 *          round (0 for a queue phase) or hub cycle, count: frontier size,
 *          list size (queued entries for a queue phase) or items
 *   ns     device time since the previous barrier (globaltimer of CTA 0) */
#define MF_PHASE_BATCH          0  /* batch, capacity apply, clamp, re-saturation */
#define MF_PHASE_HEIGHT_INIT    1
#define MF_PHASE_BFS            2
#define MF_PHASE_PUSH_RELABEL   3  /* activation queue or rounds, a warp per vertex */
#define MF_PHASE_HUB            4  /* cooperative cycles of high-degree vertices    */
#define MF_PHASE_REMOVE_INVALID 5
typedef struct mf_trace_rec {
    int16_t phase;
    int16_t mode;
    int32_t iter;
    int32_t step;
    int32_t count;
    int64_t ns;
} mf_trace_rec;

/* Keep the records of each following solve/repair in a device buffer of
 * `capacity` records (0 turns tracing off and frees the buffer).  Records past
 * the capacity are counted but dropped.  Synchronises. */
int mf_trace_enable(mf_graph *g, int32_t capacity);

/* Copy up to max_records records of the last solve/repair to `out` (host);
 * *count receives how many the launch produced.  Synchronises. */
int mf_trace_read(mf_graph *g, mf_trace_rec *out, int32_t max_records, int32_t *count);

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
