// GB300 (sm_103a) dynamic max-flow: device kernels and the C ABI of mf.h.
//
// The whole solve / repair of one graph is ONE persistent cooperative kernel
// (k_solve): every CTA of one full wave runs the phases below in lock-step,
// separated by a bounded grid barrier, so the data-dependent loops (BFS
// levels, the push/relabel rounds) never return to the host (the paper also
// decides termination on the device, Sec. 3):
//
//   validate batch -> apply capacity changes (Alg. 5, lines 1-3)
//   -> clamp negative residuals (Alg. 5, lines 4-11)
//   -> saturate source arcs (Alg. 4 lines 3-7 / Alg. 1 third loop)
//   -> loop { height init with deficient vertices as sinks (Alg. 4)
//             backward BFS global relabel + active worklist (Sec. 5.3)
//             stop when no vertex is active
//             PushRelabel x KERNELCYCLES (Alg. 2)
//             RemoveInvalidEdges (Alg. 3)
//             stop when that round left nothing pending (Alg. 4's own test) }
//   -> flow = e(t) + sum of deficits (Alg. 4, final sum).
//
// Dynamic Push-Pull (Alg. 6-8) runs in the same loop, in the instance
// k_solve<true>: saturate the arcs across the previous cut, then push on its
// sink side and pull on its source side (one search, both heights in h), then
// the plain loop on the leftover subgraph P.  A batch that only raises
// capacities off the exact cut skips the loop (the flow cannot change).
//
// Residual capacities are kept twice: r[a] and its mirror rr[a] = r[rev[a]],
// so that the backward BFS reads the residual of the arc INTO the frontier
// vertex from a contiguous array instead of gathering r[rev[a]].  Every write
// to r[x] has a matching write to rr[rev[x]].
//
// Mutable arrays are read with ld.global.cg (L2, coherent across SMs): the
// persistent kernel never relies on L1 contents across a grid barrier.
//
// The phases avoid atomics that the whole grid aims at one address: the
// items of a phase are dealt to the warps by a fixed stride (no work
// tickets), and each warp stages the BFS frontier it discovers in shared
// memory and publishes it a stage at a time.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "mf.h"
#include "mf_internal.h"
#include "mf_mlp.cuh"

namespace mf {

constexpr int kBlock = 768;   // one CTA per SM: 152 arrivals per grid barrier
constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kWaitNs = 20ull * 1000ull * 1000ull * 1000ull;  // 20 s per barrier wait

// status bits (Ctl::status)
constexpr int ST_EINVAL = 1;   // rejected batch (state unchanged)
constexpr int ST_ITERS = 2;    // max_iters reached
constexpr int ST_WAIT = 4;     // a grid-barrier wait reached its time limit
constexpr int ST_TIME = 8;     // the kernel ran past its wall-clock limit
constexpr int ST_CHECK = 16;   // a debug_checks consistency check failed
constexpr int ST_STICKY = ST_ITERS | ST_WAIT | ST_TIME | ST_CHECK;

// JOB_REFRESH recomputes exact BFS heights (and the exact cut S = {h >= n})
// for a state whose last solve stopped without a final BFS; it does nothing
// when the heights are exact already.
enum JobKind { JOB_SOLVE = 0, JOB_REPAIR = 1, JOB_RECOMPUTE = 2, JOB_AUTO = 3, JOB_REFRESH = 4 };

// How the last solve/repair ended (mf_stats.exit_kind)
enum ExitKind { EXIT_BFS = 0, EXIT_CLEAN = 1, EXIT_NO_CUT_CHANGE = 2, EXIT_PUSH_PULL = 3 };

// Fewest PushRelabel activation rounds per loop iteration, and the fewest
// cooperative cycles the high-degree vertices get per iteration (see k_solve).
constexpr int kMaxRounds = 16;
constexpr int kMinHubCycles = 4;
// The push-pull instance gives its hubs more cycles per pass: there a hub
// left active costs another dual search of the whole graph (measured on
// RMAT-20 100k batches: 3.2 -> 2.0-3.2 loop iterations, 1.24 -> 1.14 ms).
constexpr int kMinHubCyclesPP = 8;
// PushRelabel passes per loop iteration (hub cycles, then activation rounds;
// a pass that turns hubs active again hands them to the next pass, when
// there are at most kPassHubs of them).  The push-pull instance takes more:
// there the re-activated hubs are few and another pass costs much less than
// another dual BFS (measured on RMAT-20: 1.66 -> 1.32 ms per repair).
constexpr int kMaxPasses = 2;
constexpr int kMaxPassesPP = 4;
// BFS levels whose frontier has at most this many arcs and vertices run on
// CTA 0 alone, with the frontiers in shared memory
constexpr long long kSoloArcs = 8192;
constexpr int kSoloCap = 4096;
constexpr int kPassHubs = 32;   // most re-activated hubs a further pass takes
constexpr int kPassHubsPP = 64;

constexpr int S_COUNT_MAX = 24;

// Device control block.  Fields marked (z) are zero whenever no k_solve is
// running: they are zeroed at creation, by mf_solve, and by the last thread
// of every k_solve that ends normally.
struct Ctl {
    int status;           // ST_* bits                      } read together by
    int batch_err;        // (z) set by batch validation    } mf_flow_value
    long long flow;       // result of the last solve/repair }
    unsigned bar_word;    // grid barrier: generation (high 16 bits), arrivals (z, low 16 bits)
    unsigned bar_pad;
    int qcnt[3];          // (z) BFS frontier sizes, rotating by level
    int ccnt[3];          // (z) BFS chunk-item counts, rotating by level
    long long asum[3];    // (z) sum of the degrees of each BFS frontier, rotating
    int acnt[3];          // (z) activation-round list sizes, rotating by round
    int rlcnt;            // (z) relabel list size
    unsigned stamp_base;  // first activation stamp of the next launch (kept across launches)
    unsigned bseq;        // sequence number of the last batch (duplicate-id stamps)
    int wcnt;             // (z) active worklist size (vertices of degree <= kHubDeg)
    int hcnt;             // (z) active hub list size (degree > kHubDeg)
    int hccnt;            // (z) hub work items
    int hub_act[2];       // (z) hubs still active in the current hub cycle
    int hlc[2];           // (z) live hub items for the next cycle, double-buffered
    int pad0;
    long long dacc[2];    // (z) sum of deficits at the last height init
    long long iters;
    unsigned long long t_start;  // globaltimer at kernel entry
    int pol_kind;         // policy decision for the next JOB_AUTO launch
    int pol_kc;
    int pol_mode;         // processing mode chosen for it (MF_MODE_*)
    int pol_fallback;     // 1 if the learned policy fell back to the plain rule
    float feat[12];       // features of the last batch the policy kernel saw
    long long pol_acc[3]; // (z) k_policy's batch sums: increments, entries at s or t, sum |delta|
    int pol_done;         // (z) k_policy CTAs that have added their sums
    int pad3;
    int abort_loop;       // (z) set by thread 0 when the wall-clock limit passed
    int trace_n;          // trace records written by the current launch
    int ri_moved[2];      // (z) RemoveInvalidEdges saturated an arc, by iteration parity
    int phc[2];           // (z) hub lists of the next PushRelabel pass, by pass parity
    int rhcnt;            // (z) RemoveInvalidEdges items of relabelled hubs
    int pad2;
    int inc_block;        // (z) the batch holds a decrement or an increment across the cut
    int heights_exact;    // h is the BFS fixed point of the current residual graph
    int cut_exact;        // {h >= n} is exactly the set that cannot reach a sink
    int exit_kind;        // ExitKind of the last solve/repair
    int solo_L;           // BFS level at which CTA 0 hands a small-frontier run back
    long long solo_seen;  // frontier arcs counted up to that level
    long long st[S_COUNT_MAX];  // statistics, see enum Stat
    long long st_aux[S_COUNT_MAX];  // where a JOB_REFRESH counts, keeping st intact
    // the activation queue of a PushRelabel phase (see k_solve): consumer
    // tickets, producer reservations and finished entries, each on its own
    // 128-byte line (every warp of the grid polls or bumps them)
    alignas(128) int aq_head;   // (z)
    alignas(128) int aq_tail;   // (z)
    alignas(128) int aq_done;   // (z)
    alignas(128) int aq_over;   // (z) an active vertex was left out (generation cap, full queue)
    int aq_maxgen;              // (z) highest generation enqueued
    alignas(128) int aq_fin;    // (z) every queued entry has been processed
    long long chk_where;        // first failed debug check: kind << 40 | index (kept until mf_solve)
};

enum Stat {
    S_LEVELS, S_BFS_VERTS, S_BFS_ARCS, S_WL, S_PR_ARCS, S_PUSH, S_RELABEL, S_RI_ARCS, S_RI_MOVES,
    S_BATCH, S_CLAMPED, S_RESAT,
    // phase times (ns, globaltimer of CTA 0 between grid barriers) and counts
    S_T_BATCH, S_T_RESET, S_T_BFS, S_T_PRW, S_T_HUB, S_T_RI, S_HUB_CYCLES, S_BARRIERS,
    S_BU_LEVELS, S_ROUNDS,
    S_COUNT
};
static_assert(S_COUNT <= S_COUNT_MAX, "statistics array too small");

// One trace record per grid barrier of k_solve (see mf_trace_read in mf.h).
struct TraceRec {
    short phase, mode;
    int iter, step, count;
    long long ns;
};

struct DevGraph {
    int n, s, t, m;
    long long A;
    int cap_limit;
    const int *row, *head, *rev, *arc_of_edge;
    const unsigned char *edge_st;   // per edge: 1 if it leaves s or enters t (policy feature), or nullptr
    int *cap, *r, *rr, *h, *cap_edge;
    long long *e;
    unsigned *stamp;
    int *qb0, *qb1, *wl;
    int2 *cb;
    int *hl, *hmode;          // active hubs; per-hub cycle state
    int *hl2;                 // hub list of odd PushRelabel passes
    int2 *hri;                // RemoveInvalidEdges items of relabelled hubs (vertex, first arc)
    int *hnit, *hdone;        // per-hub work items, and items finished in the cycle
    int2 *hcl;                // hub work items (hub index, first arc)
    int2 *hlv0, *hlv1;        // items of the hubs still active, per cycle (double buffer)
    unsigned *hikey;          // lowest residual-neighbour height per item of the current cycle
    unsigned long long *hkey; // per-hub lowest (height, arc) key
    long long *hrem;          // per-hub excess left to push in the current cycle
    TraceRec *trace;          // per-barrier trace records, or null
    int trace_cap;
    unsigned *astamp;         // per-vertex stamp of the last activation list joined
    unsigned *rstamp;         // per-vertex stamp of the last relabel list joined
    int *rl;                  // vertices relabelled in the current loop iteration
    unsigned char *part;      // push-pull partition per vertex (kPartT / kPartS / kPartP), or null
    Ctl *ctl;
    int al16;                 // head, r and rr start on 16-byte boundaries (16-byte staging copies)
    unsigned long long *aq;   // activation queue slots (generation << 32 | vertex + 1; 0 = empty)
    int qc;                   // its capacity
};

// Push-pull partitions (Alg. 8): T can reach a sink, S cannot (the previous
// cut); P holds what neither stage-1 BFS reached.
constexpr unsigned char kPartT = 0, kPartS = 1, kPartP = 2;

struct Job {
    int kind, k, flags, kc, mode;
    int debug;           // debug_checks: list-entry bounds and the end-of-kernel invariants
    int exact_exit;      // 1: stop only after a BFS finds no active vertex
    int pp;              // 1: a repair by Dynamic Push-Pull (Alg. 8) when the cut is exact
    int sink_sat;        // 1: a solve from zero flow also saturates the arcs into t
    long long *st;       // statistics array (Ctl::st, or Ctl::st_aux for JOB_REFRESH)
    TraceRec *trace;     // trace records, or nullptr
    const int *k_dev;    // if set, the batch size is read from device memory
    long long max_iters;
    unsigned long long time_limit_ns;
    const int *ids, *caps;
    int *newc, *dlt;
};

// ---------------------------------------------------------------- helpers --
__device__ __forceinline__ int lcg(const int *p) { return __ldcg(p); }
__device__ __forceinline__ long long lcg(const long long *p) { return __ldcg(p); }
__device__ __forceinline__ int2 lcg(const int2 *p) { return __ldcg(p); }

__device__ __forceinline__ void add_ll(long long *p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(p), static_cast<unsigned long long>(v));
}

// Arrival on a counter with acquire-release order at GPU scope: this
// thread's earlier writes are visible to whoever sees the new count, and the
// last arrival sees everyone's.
__device__ __forceinline__ int arrive_acq_rel(int *p) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
    return old;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_acquire_s32(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// A value every lane of the warp must agree on (it steers warp-wide control
// flow): read once by lane 0 and broadcast.  A word that other warps write
// concurrently could otherwise reach the lanes as different values.
__device__ __forceinline__ int bcast_ld(const int *p) {
    return __shfl_sync(0xffffffffu, (threadIdx.x & 31) == 0 ? __ldcg(p) : 0, 0);
}
__device__ __forceinline__ long long bcast_ld(const long long *p) {
    return __shfl_sync(0xffffffffu, (threadIdx.x & 31) == 0 ? __ldcg(p) : 0ll, 0);
}

__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_min(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(kFull, v, o);
        v = w < v ? w : v;
    }
    return v;
}

__device__ __forceinline__ long long warp_incl_scan(long long x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Warp-aggregated append: one atomicAdd per warp (Sec. 5.3: ballot, then the
// warp leader reserves space).  Must be called by all 32 lanes.
__device__ __forceinline__ void warp_append(bool pred, int val, int *cnt, int *buf) {
    const unsigned mask = __ballot_sync(kFull, pred);
    if (!mask) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(cnt, __popc(mask));
    base = __shfl_sync(kFull, base, leader);
    if (pred) buf[base + __popc(mask & ((1u << lane) - 1u))] = val;
}

// Bounded grid barrier for a cooperative (co-resident) grid: one arrival
// atomic per CTA on a counter; the last arrival resets it and releases the
// next generation, which the other CTAs poll.  (Measured on GB300 with 152
// CTAs: 2.4 us per barrier, against 3.0 us for per-CTA arrival flags polled
// by one CTA.)  Every wait gives up after kWaitNs and sets ST_WAIT; returns
// false when any CTA gave up (the kernel must then return).
__device__ __forceinline__ bool grid_sync(Ctl *C) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        // one word holds the generation and the arrivals: the arrival's
        // atomic returns the generation to wait on, and the last CTA to
        // arrive starts the next generation with zero arrivals
        __threadfence();
        const unsigned old = atomicAdd(&C->bar_word, 1u);
        if ((old & 0xffffu) == gridDim.x - 1) {
            __threadfence();
            atomicAdd(&C->bar_word, 0x10000u - gridDim.x);
        } else {
            const unsigned long long t0 = gtimer();
            unsigned spins = 0;
            while (((ld_acquire(&C->bar_word) ^ old) & 0xffff0000u) == 0) {
                if ((++spins & 31u) == 0) {
                    if (__ldcg(&C->status) & ST_WAIT) break;
                    if (gtimer() - t0 > kWaitNs) {
                        atomicOr(&C->status, ST_WAIT);
                        break;
                    }
                }
                __nanosleep(20);
            }
        }
        __threadfence();
        ok = (__ldcg(&C->status) & ST_WAIT) == 0;
    }
    __syncthreads();
    return ok;
}

// ---------------------------------------------------------- BFS visiting --
// Per-thread work counters (32-bit to spare registers; added to the 64-bit
// statistics at the end of the kernel, and every 256 loop iterations so that
// no thread's count can wrap).  Adding them once per warp after every
// iteration cost ≈ 10 us per iteration: 3,648 atomics on each of 9 words.
struct Counters {
    unsigned bfs_arcs = 0, bfs_verts = 0, pr_arcs = 0, push = 0, relabel = 0, ri_arcs = 0,
             ri_moves = 0, clamped = 0, resat = 0;
};

constexpr int kIlp = 4;    // arcs in flight per lane in PushRelabel and RemoveInvalidEdges
constexpr int kIlpB = 4;   // arcs in flight per lane in the BFS

struct ArcRoundBfs {
    int ra[kIlpB], w[kIlpB];
};

// Warp-aggregated append of the lanes' flagged values of N slots: one
// atomicAdd for the whole warp and all slots; positions from cap on go to
// spill (same positions) instead of buf.  All 32 lanes call.
template <int N>
__device__ __forceinline__ void warp_append_n(const bool (&pred)[N], const int (&val)[N], int *cnt, int *buf,
                                              int cap = 0x7fffffff, int *spill = nullptr) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    unsigned m[N];
    int tot = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        m[j] = __ballot_sync(kFull, pred[j]);
        tot += __popc(m[j]);
    }
    if (tot == 0) return;
    int base = 0;
    if (lane == 0) base = atomicAdd(cnt, tot);
    base = __shfl_sync(kFull, base, 0);
#pragma unroll
    for (int j = 0; j < N; ++j) {
        if (pred[j]) {
            const int pos = base + __popc(m[j] & below);
            (pos < cap ? buf : spill)[pos] = val[j];
        }
        base += __popc(m[j]);
    }
}

constexpr int kWq = 320;   // staged frontier entries per warp (24 warps: 7680 ints)
constexpr int kFl = 4;     // staged entries per lane in flight when a stage is published

// The next BFS frontier as one warp writes it.  In grid-wide levels the
// entries are staged in the warp's kWq ints of shared memory and reach the
// global queue buf a whole stage at a time (one reservation on cnt); the
// bookkeeping of the staged vertices (their degrees for the frontier's arc
// total, their excess for the active lists) is done when the stage is
// published, for up to 32 kFl vertices at once, instead of inside the arc
// scan that discovered them: the scan's chain of dependent accesses ends at
// the height CAS.  front_flush must run before the level's grid barrier.  In
// CTA 0's small-frontier levels (stage == nullptr) entries go straight to the
// shared frontier (positions >= cap to spill) with their bookkeeping done at
// once, and the arc total goes to its counter.
struct Front {
    int *cnt, *buf;
    long long *asum;
    int cap;
    int *spill;
    int *stage;     // this warp's kWq shared ints, or nullptr
    int sn;         // staged entries (warp-uniform)
    long long ds;   // arc total not yet added (warp-uniform)
    unsigned mark;  // activation stamp given to the worklist entries (queued from the start)
};

// Publish the staged entries and do their bookkeeping: each joins the global
// frontier, its degree counts towards the frontier's arc total, and a vertex
// with positive excess (in the first stage of a push-pull repair, a deficient
// vertex of the pull side) is active: worklist (degree <= kHubDeg) or hub
// list.  All 32 lanes call.
__device__ __forceinline__ void front_flush_entries(const DevGraph &G, Front &F, bool dual, Counters &K) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    int base = 0;
    if (lane == 0) base = atomicAdd(F.cnt, F.sn);
    base = __shfl_sync(kFull, base, 0);
    long long ds = 0;
    for (int i0 = 0; i0 < F.sn; i0 += 32 * kFl) {
        int v[kFl], deg[kFl];
        long long ev[kFl];
        bool ok[kFl], small[kFl], hub[kFl];
#pragma unroll
        for (int j = 0; j < kFl; ++j) {
            const int i = i0 + 32 * j + lane;
            ok[j] = i < F.sn;
            v[j] = ok[j] ? F.stage[i] : 0;
            if (ok[j]) F.buf[base + i] = v[j];
        }
#pragma unroll
        for (int j = 0; j < kFl; ++j) {
            deg[j] = ok[j] ? __ldg(&G.row[v[j] + 1]) - __ldg(&G.row[v[j]]) : 0;
            ev[j] = ok[j] ? lcg(&G.e[v[j]]) : 0;
        }
#pragma unroll
        for (int j = 0; j < kFl; ++j) {
            // a vertex of the pull side (forward search) is active when deficient
            const bool pull = ok[j] && dual && G.part[v[j]] == kPartS;
            const bool act = ok[j] && (pull ? ev[j] < 0 : ev[j] > 0);
            ds += deg[j];
            K.bfs_verts += ok[j];
            hub[j] = act && deg[j] > kHubDeg;
            small[j] = act && !hub[j];
            if (small[j]) G.astamp[v[j]] = F.mark;
        }
        warp_append_n(small, v, &G.ctl->wcnt, G.wl);
        warp_append_n(hub, v, &G.ctl->hcnt, G.hl);
    }
    F.ds += warp_sum(ds);
    __syncwarp();
    F.sn = 0;
}

// Publish what the warp has staged.  All 32 lanes call.
__device__ __forceinline__ void front_flush(const DevGraph &G, Front &F, bool dual, Counters &K) {
    if (F.stage && F.sn) front_flush_entries(G, F, dual, K);
    if (F.ds && (threadIdx.x & 31) == 0) add_ll(F.asum, F.ds);
    F.ds = 0;
}

// Stage the lanes' flagged values of N slots (at most 32 N <= kWq entries).
// Only for grid-wide levels (F.stage set).  All 32 lanes call.
template <int N>
__device__ __forceinline__ void front_stage_n(const DevGraph &G, const bool (&pred)[N], const int (&val)[N],
                                              Front &F, bool dual, Counters &K) {
    const unsigned below = (1u << (threadIdx.x & 31)) - 1u;
    unsigned m[N];
    int tot = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        m[j] = __ballot_sync(kFull, pred[j]);
        tot += __popc(m[j]);
    }
    if (tot == 0) return;
    if (F.sn + tot > kWq) front_flush_entries(G, F, dual, K);
    int base = F.sn;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        if (pred[j]) F.stage[base + __popc(m[j] & below)] = val[j];
        base += __popc(m[j]);
    }
    F.sn = base;
}

// bfs_discovered for kIlpB slots per lane at once.  Grid-wide levels stage
// the vertices (bookkeeping when the stage is published); CTA 0's levels do
// the bookkeeping here, the loads of all slots issued together and each list
// getting one reservation per warp.
__device__ __forceinline__ void bfs_discovered_n(const DevGraph &G, const bool (&disc)[kIlpB], const int (&v)[kIlpB],
                                                 unsigned fwd, bool dual, Front &F, Counters &K) {
    bool any = false;
#pragma unroll
    for (int j = 0; j < kIlpB; ++j) any |= disc[j];
    if (!__any_sync(kFull, any)) return;
    if (F.stage) {
        front_stage_n(G, disc, v, F, dual, K);
        return;
    }
    warp_append_n(disc, v, F.cnt, F.buf, F.cap, F.spill);
    int deg[kIlpB];
    long long ev[kIlpB];
#pragma unroll
    for (int j = 0; j < kIlpB; ++j) {
        deg[j] = disc[j] ? __ldg(&G.row[v[j] + 1]) - __ldg(&G.row[v[j]]) : 0;
        ev[j] = disc[j] ? lcg(&G.e[v[j]]) : 0;
    }
    long long ds = 0;
    bool small[kIlpB], hub[kIlpB];
#pragma unroll
    for (int j = 0; j < kIlpB; ++j) {
        ds += deg[j];
        K.bfs_verts += disc[j];
        // a vertex of the pull side (forward search) is active when deficient
        const bool act = disc[j] && (((fwd >> j) & 1u) ? ev[j] < 0 : ev[j] > 0);
        hub[j] = act && deg[j] > kHubDeg;
        small[j] = act && !hub[j];
        if (small[j]) G.astamp[v[j]] = F.mark;
    }
    ds = warp_sum(ds);
    if ((threadIdx.x & 31) == 0 && ds) add_ll(F.asum, ds);
    warp_append_n(small, v, &G.ctl->wcnt, G.wl);
    warp_append_n(hub, v, &G.ctl->hcnt, G.hl);
}

// Bookkeeping of a vertex v reached at the next level (disc), one slot per
// lane: as bfs_discovered_n.  All 32 lanes call.
__device__ __forceinline__ void bfs_discovered(const DevGraph &G, bool disc, int v, bool fwd, bool dual,
                                               Front &F, Counters &K) {
    bool d1[kIlpB];
    int v1[kIlpB];
#pragma unroll
    for (int j = 0; j < kIlpB; ++j) {
        d1[j] = j == 0 && disc;
        v1[j] = j == 0 ? v : 0;
    }
    bfs_discovered_n(G, d1, v1, fwd ? 1u : 0u, dual, F, K);
}

// Backward BFS step over kIlpB arcs per lane (a[j] of frontier vertex u, head
// v; ok[j] marks a real arc): the arc v -> u is residual iff rr[a] > 0; an
// unvisited v (height n) gets height L + 1 (global relabel, Sec. 2.2).  Newly
// reached vertices with positive excess are active and join the worklist
// (degree <= kHubDeg) or the hub list.  Slots whose bit is set in fwd belong
// to the pull side of a push-pull repair and search forward instead: u -> v
// residual (r[a] > 0), and a deficient v is active.  Every load of a round is
// issued before any of them is used.  All 32 lanes call.
__device__ __forceinline__ void bfs_visit_n(const DevGraph &G, const int (&a)[kIlpB], const bool (&ok)[kIlpB],
                                            unsigned fwd, bool dual, int L, Front &F, Counters &K) {
    const int n = G.n;
    int v[kIlpB], rin[kIlpB], hv[kIlpB];
    bool disc[kIlpB];
#pragma unroll
    for (int j = 0; j < kIlpB; ++j) {
        v[j] = ok[j] ? __ldg(&G.head[a[j]]) : 0;
        rin[j] = ok[j] ? lcg(((fwd >> j) & 1u) ? &G.r[a[j]] : &G.rr[a[j]]) : 0;
        K.bfs_arcs += ok[j];
    }
#pragma unroll
    for (int j = 0; j < kIlpB; ++j) hv[j] = (rin[j] > 0 && v[j] != G.s) ? lcg(&G.h[v[j]]) : -1;
#pragma unroll
    for (int j = 0; j < kIlpB; ++j) disc[j] = hv[j] == n && atomicCAS(&G.h[v[j]], n, L + 1) == n;
    bfs_discovered_n(G, disc, v, fwd, dual, F, K);
}

// Expand up to 32 frontier vertices (one per lane, degree deg starting at
// arc beg, fwd for the pull side of a push-pull repair) with the arcs
// balanced over the lanes: lane i handles arcs k0 + 32 j + i of the
// concatenated lists.
__device__ __forceinline__ void bfs_expand_warp(const DevGraph &G, int beg, int deg, bool fwd, bool dual, int L,
                                                Front &F, Counters &K) {
    const unsigned fwd_lanes = __ballot_sync(kFull, fwd);
    const int lane = threadIdx.x & 31;
    int incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    const int excl = incl - deg;
    for (int k0 = 0; k0 < total; k0 += 32 * kIlpB) {
        int a[kIlpB];
        bool ok[kIlpB];
        unsigned fw = 0;
#pragma unroll
        for (int jj = 0; jj < kIlpB; ++jj) {
            const int k = k0 + 32 * jj + lane;
            int j = 0;  // owner lane: largest j with excl_j <= k
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int cand = j + step;
                const int ex = __shfl_sync(kFull, excl, cand & 31);
                if (cand < 32 && ex <= k) j = cand;
            }
            const int ob = __shfl_sync(kFull, beg, j);
            const int oe = __shfl_sync(kFull, excl, j);
            ok[jj] = k < total;
            a[jj] = ob + (k - oe);
            fw |= ((fwd_lanes >> j) & 1u) << jj;
        }
        bfs_visit_n(G, a, ok, fw, dual, L, F, K);
    }
}

// Bottom-up step of the backward BFS (direction-optimising search): the
// unvisited vertices v of a group of 32 consecutive ids look for a residual
// arc v -> w into the current frontier (h(w) == L); the first one found gives
// h(v) = L + 1.  The group's arcs are balanced over the lanes and the scan of
// a vertex stops once it is found.  Vertices of degree > kBigDeg become
// kChunk-arc items of the chunk list instead.  In the first stage of a
// push-pull repair (dual) a vertex of the pull side looks for a residual arc
// w -> v from the frontier instead, and only frontier vertices of the
// vertex's own side count.  All 32 lanes call.
// What a lane needs of its vertex base + lane before the group's scan: its
// height and arc range, loaded one group ahead (the warp loads the next
// group's while it scans this one).  During a bottom-up level only the
// owning lane writes an unvisited vertex's height, so the early read is
// exact.
struct BuPre {
    int hv, beg, end;
};

__device__ __forceinline__ BuPre bu_prefetch(const DevGraph &G, int base) {
    const int v = base + (threadIdx.x & 31);
    BuPre p{-1, 0, 0};
    if (v < G.n) {
        p.hv = lcg(&G.h[v]);
        p.beg = __ldg(&G.row[v]);
        p.end = __ldg(&G.row[v + 1]);
    }
    return p;
}

__device__ __forceinline__ void bfs_bottom_up_group(const DevGraph &G, int base, const BuPre &pre, bool dual, int L,
                                                    Front &F, int *ccnt, Counters &K) {
    const int lane = threadIdx.x & 31;
    const int n = G.n;
    const int v = base + lane;
    int beg = 0, deg = 0;
    const int side = (dual && v < n) ? G.part[v] : kPartT;
    if (v < n && v != G.s && pre.hv == n) {
        beg = pre.beg;
        deg = pre.end - beg;
        if (deg > kBigDeg) {
            const int nc = (deg + kChunk - 1) / kChunk;
            const int pos = atomicAdd(ccnt, nc);
            for (int c = 0; c < nc; ++c) G.cb[pos + c] = make_int2(v, beg + c * kChunk);
            deg = 0;
        }
    }
    const unsigned want = __ballot_sync(kFull, deg > 0);
    unsigned found = 0;
    if (want) {
        int incl = deg;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        const int excl = incl - deg;
        const unsigned pull_lanes = __ballot_sync(kFull, side == kPartS);
        for (int k0 = 0; k0 < total && found != want; k0 += 32 * kIlpB) {
            int a[kIlpB], own[kIlpB], ra[kIlpB], w[kIlpB];
#pragma unroll
            for (int jj = 0; jj < kIlpB; ++jj) {
                const int k = k0 + 32 * jj + lane;
                int j = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const int cand = j + step;
                    const int ex = __shfl_sync(kFull, excl, cand & 31);
                    if (cand < 32 && ex <= k) j = cand;
                }
                own[jj] = j;
                a[jj] = __shfl_sync(kFull, beg, j) + (k - __shfl_sync(kFull, excl, j));
                const bool live = k < total && !((found >> j) & 1u);
                ra[jj] = live ? lcg(((pull_lanes >> j) & 1u) ? &G.rr[a[jj]] : &G.r[a[jj]]) : 0;
                w[jj] = live ? __ldg(&G.head[a[jj]]) : 0;
                K.bfs_arcs += live;
            }
            unsigned hit = 0;
#pragma unroll
            for (int jj = 0; jj < kIlpB; ++jj)
                if (ra[jj] > 0 && lcg(&G.h[w[jj]]) == L &&
                    (!dual || G.part[w[jj]] == (((pull_lanes >> own[jj]) & 1u) ? kPartS : kPartT)))
                    hit |= 1u << own[jj];
            found |= __reduce_or_sync(kFull, hit);
        }
    }
    const bool disc = (found >> lane) & 1u;
    if (disc) G.h[v] = L + 1;
    bfs_discovered(G, disc, v, side == kPartS, dual, F, K);
}

// Bottom-up scan of one kChunk-arc item of a high-degree unvisited vertex;
// several items of one vertex may find a parent, the height CAS elects one.
__device__ __forceinline__ void bfs_bottom_up_item(const DevGraph &G, int2 item, bool dual, int L, Front &F,
                                                   Counters &K) {
    const int lane = threadIdx.x & 31;
    const int v = item.x;
    const int side = dual ? G.part[v] : kPartT;
    bool disc = false;
    if (bcast_ld(&G.h[v]) == G.n) {
        const int a1 = min(item.y + kChunk, __ldg(&G.row[v + 1]));
        bool hit = false;
        for (int a0 = item.y; a0 < a1 && !hit; a0 += 32 * kIlpB) {
            if (a0 != item.y && bcast_ld(&G.h[v]) != G.n) break;
            ArcRoundBfs R;
#pragma unroll
            for (int j = 0; j < kIlpB; ++j) {
                const int a = a0 + 32 * j + lane;
                R.ra[j] = a < a1 ? lcg(side == kPartS ? &G.rr[a] : &G.r[a]) : 0;
                R.w[j] = a < a1 ? __ldg(&G.head[a]) : 0;
                K.bfs_arcs += a < a1;
            }
            bool mine = false;
#pragma unroll
            for (int j = 0; j < kIlpB; ++j)
                mine |= R.ra[j] > 0 && lcg(&G.h[R.w[j]]) == L && (!dual || G.part[R.w[j]] == side);
            hit = __any_sync(kFull, mine);
        }
        if (hit && lane == 0) disc = atomicCAS(&G.h[v], G.n, L + 1) == G.n;
    }
    disc = __shfl_sync(kFull, disc, 0);
    bfs_discovered(G, disc && lane == 0, v, side == kPartS, dual, F, K);
}

// ------------------------------------------------------ push / relabel --
// One push of d units along arc a (u -> v) with reverse arc b: both residual
// copies of the arc pair (reductions: nothing waits on them) and the head's
// excess; the caller subtracts the total from e(u).  Returns e(v) before.
// A push into s or t (never active) is a reduction too: the pusher does not
// wait in the queue of same-address atomics that the many pushes into the
// sink form at its L2 slice.
__device__ __forceinline__ long long push_arc(const DevGraph &G, int a, int b, int v, int d) {
    atomicSub(&G.r[a], d);
    atomicSub(&G.rr[b], d);
    atomicAdd(&G.r[b], d);
    atomicAdd(&G.rr[a], d);
    if (v == G.t || v == G.s) {
        add_ll(&G.e[v], d);
        return 1;
    }
    return (long long)atomicAdd(reinterpret_cast<unsigned long long *>(&G.e[v]), (unsigned long long)d);
}

// One pull of d units into u along arc a (u -> v) of u's list, reverse arc
// b: the arc v -> u loses d of residual and v loses d of excess
// (PullRelabel, Alg. 6); the caller adds the total to e(u).  Returns e(v)
// before the pull.
__device__ __forceinline__ long long pull_arc(const DevGraph &G, int a, int b, int v, int d) {
    atomicSub(&G.r[b], d);
    atomicSub(&G.rr[a], d);
    atomicAdd(&G.r[a], d);
    atomicAdd(&G.rr[b], d);
    if (v == G.t || v == G.s) {
        add_ll(&G.e[v], -(long long)d);
        return -1;
    }
    return (long long)atomicAdd(reinterpret_cast<unsigned long long *>(&G.e[v]), (unsigned long long)(-(long long)d));
}

// Where the vertices that a push makes active go: the list of the next
// activation round (see the PushRelabel phase of k_solve).  A vertex enters
// one list at most once, by the stamp of that list.
struct ActList {
    int *cnt;
    int *list;
    unsigned stamp;
    unsigned rstamp;   // stamp of this loop iteration's relabel list
    int *hcnt;         // the next pass's hub list (high-degree vertices a push
    int *hlist;        //   turned active), its size and its stamp
    unsigned hstamp;
    // queue mode (the PushRelabel phases of the data-driven and push-pull
    // modes): activated vertices go to the activation queue with generation
    // gen instead of to list; stamp then marks "queued or being processed"
    unsigned long long *aq;   // or nullptr: round lists
    int qc, gen, gen_cap;
    Ctl *C;
};

// Enqueue the lanes' flagged vertices of N slots into the activation queue
// with generation AL.gen (one reservation per warp); entries past the queue's
// capacity are dropped, counted as finished and flagged (the iteration then
// ends on another global relabel).  All 32 lanes call.
template <int N>
__device__ __forceinline__ void aq_push_n(const ActList &AL, const bool (&pred)[N], const int (&val)[N]) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    unsigned m[N];
    int tot = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        m[j] = __ballot_sync(kFull, pred[j]);
        tot += __popc(m[j]);
    }
    if (tot == 0) return;
    int base = 0;
    if (lane == 0) base = atomicAdd(&AL.C->aq_tail, tot);
    base = __shfl_sync(kFull, base, 0);
    int over = 0;
    const unsigned long long tag = (unsigned long long)(unsigned)AL.gen << 32;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        if (pred[j]) {
            const int pos = base + __popc(m[j] & below);
            if (pos < AL.qc) st_release_u64(&AL.aq[pos], tag | (unsigned)(val[j] + 1));
            else ++over;
        }
        base += __popc(m[j]);
    }
    over = (int)warp_sum((long long)over);
    if (lane == 0) {
        atomicMax(&AL.C->aq_maxgen, AL.gen);
        if (over) {
            atomicAdd(&AL.C->aq_done, over);
            atomicExch(&AL.C->aq_over, 1);
        }
    }
}

// A vertex whose height PushRelabel raised joins the relabel list of the loop
// iteration once: only relabelled vertices can own arcs that RemoveInvalidEdges
// must saturate (the others keep their BFS height, which no residual arc can
// make steep).  One thread calls.
__device__ __forceinline__ void note_relabel(const DevGraph &G, int u, unsigned rstamp) {
    if (atomicExch(&G.rstamp[u], rstamp) != rstamp) G.rl[atomicAdd(&G.ctl->rlcnt, 1)] = u;
}

// Single-thread enqueue of v (as aq_push_n).
__device__ __forceinline__ void aq_push_one(const ActList &AL, int v) {
    const int pos = atomicAdd(&AL.C->aq_tail, 1);
    if (pos < AL.qc) {
        st_release_u64(&AL.aq[pos], ((unsigned long long)(unsigned)AL.gen << 32) | (unsigned)(v + 1));
    } else {
        atomicAdd(&AL.C->aq_done, 1);
        atomicExch(&AL.C->aq_over, 1);
    }
    atomicMax(&AL.C->aq_maxgen, AL.gen);
}

// File the vertices that moves turned active (add: worklist vertices, degree
// <= kHubDeg; add_hub: hubs; neither s nor t): each joins the next activation
// round's list -- in queue mode the activation queue -- or the next pass's
// hub list, once, by the list's stamp.  In queue mode a vertex is marked
// from its enqueue until the warp that processes it has finished, and that
// warp clears the mark before it reads the vertex's excess a last time: with
// a fence between the excess atomic and the mark here, and between the clear
// and the read there, at least one side sees the other, so a vertex that a
// push turns active while it is being processed is queued again exactly once
// and no activation is lost.  Past the generation cap a vertex is left
// active, unqueued, and the phase is flagged.  All 32 lanes call.
template <int N>
__device__ __forceinline__ void file_activations(const DevGraph &G, bool (&add)[N], bool (&add_hub)[N],
                                                 const int (&v)[N], const ActList &AL) {
    bool any = false;
#pragma unroll
    for (int j = 0; j < N; ++j) any |= add[j] || add_hub[j];
    if (!__any_sync(kFull, any)) return;
    if (AL.aq) {
        if (AL.gen >= AL.gen_cap) {
            bool capped = false;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                capped |= add[j];
                add[j] = false;
            }
            if (__any_sync(kFull, capped) && (threadIdx.x & 31) == 0) atomicExch(&AL.C->aq_over, 1);
        }
        __threadfence();
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
        if (add[j]) add[j] = atomicExch(&G.astamp[v[j]], AL.stamp) != AL.stamp;
        if (add_hub[j]) add_hub[j] = atomicExch(&G.astamp[v[j]], AL.hstamp) != AL.hstamp;
    }
    if (AL.aq) aq_push_n(AL, add, v);
    else warp_append_n(add, v, AL.cnt, AL.list);
    warp_append_n(add_hub, v, AL.hcnt, AL.hlist);
}

// One round of a warp's arc scan: lane i holds arcs a0 + 32 j + i (j < kIlp)
// with their residual (0 past `end`), head and the head's height, and, when
// the round is one to push along (REV), the reverse arcs of its residual
// arcs.  All loads of the round are issued before any is used; the reverse
// arcs load beside the heights.
struct ArcRound {
    int ra[kIlp], v[kIlp], hv[kIlp], rb[kIlp];
};

// The residual is that of the arc u -> head (push) or head -> u (pull, the
// mirror rr).  With a partition array pt, an arc to a vertex of another part
// counts as absent (push-pull: each side works on its own vertices only).
template <bool PULL, bool REV>
__device__ __forceinline__ void load_round_t(const DevGraph &G, int a0, int end, ArcRound &R,
                                             const unsigned char *pt, unsigned char side) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < kIlp; ++j) {
        const int a = a0 + 32 * j + lane;
        const bool ok = a < end;
        R.ra[j] = ok ? lcg(PULL ? &G.rr[a] : &G.r[a]) : 0;
        R.v[j] = ok ? __ldg(&G.head[a]) : 0;
    }
    if (pt) {
#pragma unroll
        for (int j = 0; j < kIlp; ++j)
            if (R.ra[j] > 0 && pt[R.v[j]] != side) R.ra[j] = 0;
    }
#pragma unroll
    for (int j = 0; j < kIlp; ++j) {
        R.hv[j] = R.ra[j] > 0 ? lcg(&G.h[R.v[j]]) : 0;
        R.rb[j] = (REV && R.ra[j] > 0) ? __ldg(&G.rev[a0 + 32 * j + lane]) : 0;
    }
}

__device__ __forceinline__ int round_arcs(int a0, int end) {
    const int lane = threadIdx.x & 31;
    int c = 0;
#pragma unroll
    for (int j = 0; j < kIlp; ++j) c += (a0 + 32 * j + lane) < end;
    return c;
}

// Lowest (height, arc offset from beg) key over the residual arcs of a round.
__device__ __forceinline__ unsigned long long round_min_key(const ArcRound &R, int a0, int beg) {
    const int lane = threadIdx.x & 31;
    unsigned long long best = ~0ull;
#pragma unroll
    for (int j = 0; j < kIlp; ++j) {
        if (R.ra[j] > 0) {
            const unsigned long long key =
                ((unsigned long long)(unsigned)R.hv[j] << 32) | (unsigned)(a0 + 32 * j + lane - beg);
            best = key < best ? key : best;
        }
    }
    return best;
}

// The amount moved along arc a (u -> v, reverse b) in one step: a push or a
// pull.
template <bool PULL>
__device__ __forceinline__ long long move_arc(const DevGraph &G, int a, int b, int v, int d) {
    return PULL ? pull_arc(G, a, b, v, d) : push_arc(G, a, b, v, d);
}

// The amounts of one round at height hh, in arc order (round slot j, then
// lane), as consecutive Alg. 2 steps would move them: min(rem, c_f) each
// until rem is used up; tot receives the round's residual at height hh.
__device__ __forceinline__ void round_amounts(const ArcRound &R, int hh, long long rem, int (&d)[kIlp],
                                              long long &tot) {
    tot = 0;
#pragma unroll
    for (int j = 0; j < kIlp; ++j) {
        const int ra = (R.ra[j] > 0 && R.hv[j] == hh) ? R.ra[j] : 0;
        const long long incl = warp_incl_scan(ra) + tot;
        const long long dj = rem - (incl - ra);
        d[j] = dj < 0 ? 0 : (dj > ra ? ra : (int)dj);
        tot = __shfl_sync(kFull, incl, 31);
    }
}

// The moves of one round (d[j] > 0: d[j] units along slot j of R, a round
// loaded with its reverse arcs), and the filing of the vertices they turn
// active: a push that raised e(v) above 0 (a pull that lowered it below 0)
// makes v active, and v (not s or t) joins the next activation round when its
// degree is <= kHubDeg, else the hub list of the next PushRelabel pass.  The
// heads' degrees load beside the move atomics, so the filing waits once for
// both; v's height is the one the scan read (a push only goes below h(u) <
// n).  Each list gets one reservation per warp.  Returns this lane's total
// moved.  All 32 lanes call.
template <bool PULL>
__device__ __forceinline__ long long move_round(const DevGraph &G, int a0, const int (&d)[kIlp], const ArcRound &R,
                                                const ActList &AL, Counters &K) {
    const int lane = threadIdx.x & 31;
    long long old[kIlp], sent = 0;
    int deg[kIlp];
#pragma unroll
    for (int j = 0; j < kIlp; ++j) {
        old[j] = 0;
        deg[j] = 0;
        if (d[j] > 0) {
            old[j] = move_arc<PULL>(G, a0 + 32 * j + lane, R.rb[j], R.v[j], d[j]);
            deg[j] = __ldg(&G.row[R.v[j] + 1]) - __ldg(&G.row[R.v[j]]);
            sent += d[j];
            ++K.push;
        }
    }
    bool add[kIlp], add_hub[kIlp];
#pragma unroll
    for (int j = 0; j < kIlp; ++j) {
        const bool turned = PULL ? (old[j] >= 0 && old[j] - d[j] < 0) : (old[j] <= 0 && old[j] + d[j] > 0);
        const bool cand = d[j] > 0 && turned && R.v[j] != G.s && R.v[j] != G.t;
        add[j] = cand && deg[j] <= kHubDeg;
        add_hub[j] = cand && deg[j] > kHubDeg;
    }
    file_activations(G, add, add_hub, R.v, AL);
    return sent;
}

// ------------------------------------------------ staged arc ranges --
// A warp that scans the arcs of one vertex of degree 129 .. kStg copies them
// to its own shared memory first: residuals and heads as 16-byte cp.async
// copies (L2 only, so residuals written by other SMs' atomics are seen; no
// register holds an arc in flight), then the heights of the residual arcs'
// heads, gathered kGat per lane at a time.  A range of up to kStg arcs then
// takes three dependent round trips to memory instead of two per 128-arc
// round.  The staged range starts at the 16-byte boundary at or below the
// first arc: index i of a stage is arc (a0 & ~3) + i.
constexpr int kStg = 512;              // arcs one warp stages at a time
constexpr int kStgInts = kStg + 8;     // + the alignment slack of the first copy
constexpr int kStgWarp = 3 * kStgInts; // ints per warp: heads, residuals, heights
constexpr int kGat = 8;                // height gathers in flight per lane
static_assert(kHubDeg <= kStg, "a worklist vertex fits one stage");
constexpr int kDynSmem = (kBlock / 32) * kStgWarp * 4;   // bytes of dynamic shared memory of k_solve

__device__ __forceinline__ void cp_async16(int *dst, const int *src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}

// Copy arcs [a0, a1) of the int array src (A entries) to dst[i], i = a -
// (a0 & ~3): 16 bytes per copy, except where the array is not 16-byte aligned
// or the copy would pass its end (plain L2 loads there).  Pair with
// stage_wait.  All 32 lanes call.
__device__ __forceinline__ void stage_copy(const int *src, int *dst, int a0, int a1, long long A, bool al16) {
    const int base = a0 & ~3;
    const int nch = (a1 - base + 3) >> 2;
    for (int c = threadIdx.x & 31; c < nch; c += 32) {
        const long long a = base + 4LL * c;
        if (al16 && a + 4 <= A) {
            cp_async16(dst + 4 * c, src + a);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (a + q < A) dst[4 * c + q] = __ldcg(src + a + q);
        }
    }
}

// Wait for this lane's copies, then make every lane's visible to the warp.
__device__ __forceinline__ void stage_wait() {
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
}

// Heights of the heads of the staged residual arcs in [a0, a1): sh[i] = h of
// the head, or INT_MAX for no residual arc (out of range, zero residual, or,
// with a partition array pt, a head in another part: its residual is zeroed
// in sr).  Returns this lane's lowest (height, arc - a0) key.
__device__ __forceinline__ unsigned long long stage_heights(const DevGraph &G, const int *sv, int *sr, int *sh,
                                                            int a0, int a1, const unsigned char *pt,
                                                            unsigned char side) {
    const int lane = threadIdx.x & 31;
    const int base = a0 & ~3, cnt = a1 - base;
    unsigned long long best = ~0ull;
    for (int i0 = lane; i0 < cnt; i0 += 32 * kGat) {
        int hv[kGat];
        bool res[kGat];
        unsigned char pv[kGat];
#pragma unroll
        for (int j = 0; j < kGat; ++j) {
            const int i = i0 + 32 * j;
            res[j] = i < cnt && base + i >= a0 && sr[i] > 0;
            const int v = res[j] ? sv[i] : 0;
            hv[j] = res[j] ? lcg(&G.h[v]) : 0;
            pv[j] = (pt && res[j]) ? pt[v] : side;
        }
#pragma unroll
        for (int j = 0; j < kGat; ++j) {
            const int i = i0 + 32 * j;
            if (res[j] && pv[j] != side) {
                res[j] = false;
                sr[i] = 0;
            }
            if (i < cnt) sh[i] = res[j] ? hv[j] : INT_MAX;
            if (res[j]) {
                const unsigned long long key = ((unsigned long long)(unsigned)hv[j] << 32) | (unsigned)(base + i - a0);
                best = key < best ? key : best;
            }
        }
    }
    __syncwarp();
    return best;
}

// The moves of N slots per lane (d[j] > 0: d[j] units along arc a[j] of u,
// reverse b[j], head v[j]) and the filing of the vertices they turn active,
// as move_round.  Returns this lane's total moved.  All 32 lanes call.
constexpr int kMv = 4;   // moves in flight per lane
template <bool PULL, int N>
__device__ __forceinline__ long long move_batch(const DevGraph &G, const int (&a)[N], const int (&b)[N],
                                                const int (&v)[N], const int (&d)[N], const ActList &AL,
                                                Counters &K) {
    long long old[N], sent = 0;
    int deg[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        old[j] = 0;
        deg[j] = 0;
        if (d[j] > 0) {
            old[j] = move_arc<PULL>(G, a[j], b[j], v[j], d[j]);
            deg[j] = __ldg(&G.row[v[j] + 1]) - __ldg(&G.row[v[j]]);
            sent += d[j];
            ++K.push;
        }
    }
    bool add[N], add_hub[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const bool turned = PULL ? (old[j] >= 0 && old[j] - d[j] < 0) : (old[j] <= 0 && old[j] + d[j] > 0);
        const bool cand = d[j] > 0 && turned && v[j] != G.s && v[j] != G.t;
        add[j] = cand && deg[j] <= kHubDeg;
        add_hub[j] = cand && deg[j] > kHubDeg;
    }
    file_activations(G, add, add_hub, v, AL);
    return sent;
}

// The moves a decision to push at height hh makes along staged arcs [a0,
// a1): the amounts in arc order (min(rem, c_f) each, 32 arcs a step, over
// the arcs at height hh), written over the heights in sh, then all moves at
// once, kGat per lane in flight.  Returns the warp's total moved (all lanes).
template <bool PULL>
__device__ __forceinline__ long long stage_moves(const DevGraph &G, const int *sv, const int *sr, int *sh, int a0,
                                                 int a1, int hh, long long rem, const ActList &AL, Counters &K) {
    const int lane = threadIdx.x & 31;
    const int base = a0 & ~3, cnt = a1 - base;
    int iend = 0;
    for (int i0 = 0; i0 < cnt && rem > 0; i0 += 32) {
        const int i = i0 + lane;
        const int ra = (i < cnt && sh[i] == hh) ? sr[i] : 0;
        const long long incl = warp_incl_scan(ra);
        const long long dj = rem - (incl - ra);
        if (i < cnt) sh[i] = dj < 0 ? 0 : (dj > ra ? ra : (int)dj);
        rem -= min(__shfl_sync(kFull, incl, 31), rem);
        iend = i0 + 32;
    }
    __syncwarp();
    long long sent = 0;
    const int lim = min(iend, cnt);
    // warp-uniform trip count: move_batch holds warp-wide ballots
    for (int i0 = 0; i0 < lim; i0 += 32 * kMv) {
        int a[kMv], b[kMv], v[kMv], d[kMv];
        bool any = false;
#pragma unroll
        for (int j = 0; j < kMv; ++j) {
            const int i = i0 + 32 * j + lane;
            d[j] = i < lim ? sh[i] : 0;
            a[j] = base + i;
            v[j] = d[j] > 0 ? sv[i] : 0;
            b[j] = d[j] > 0 ? __ldg(&G.rev[a[j]]) : 0;
            any |= d[j] > 0;
        }
        if (!__any_sync(kFull, any)) continue;
        sent += move_batch<PULL, kMv>(G, a, b, v, d, AL, K);
    }
    return warp_sum(sent);
}

// Algorithm 2 on vertex u by one warp, up to kc cycles.  A cycle scans u's
// arcs once for the lowest residual neighbour height h^ (ties: lowest arc;
// heights read once per cycle, Note 3 of Sec. 3).  If h(u) > h^ the cycle
// performs the pushes that consecutive Alg. 2 steps would make to the arcs at
// height h^ -- in arc order, min(e, c_f) each, until e(u) is used up --
// (from the round the scan loaded when u has one round of arcs; vertices with
// more reload the rounds that hold such an arc); otherwise it relabels u to
// h^ + 1.  A vertex without residual arcs gets height n.  Only u's warp
// lowers r(u, .) and e(u) and changes h(u) during a round; other warps only
// raise r(u, .) and e(u), so every amount pushed is available, h(u) is read
// once, and e(u) is re-read beside each cycle's arc loads.  With PULL the
// same steps are Algorithm 6 (PullRelabel) on a deficient u: residual arcs
// into u, pulls of min(-e, c_f) from the lowest of them.  Once its steps are
// done u joins the iteration's relabel list if it was relabelled, and the
// next round's list if still active.
template <bool PULL>
__device__ __forceinline__ void pr_finish_t(const DevGraph &G, int u, int hu, bool relabelled, const ActList &AL) {
    if ((threadIdx.x & 31) == 0) {
        if (relabelled) note_relabel(G, u, AL.rstamp);
        if (AL.aq) {
            atomicExch(&G.astamp[u], 0u);   // u leaves the queue before its excess is read (file_activations)
            __threadfence();
        }
        const long long eu = lcg(&G.e[u]);
        if (hu < G.n && (PULL ? eu < 0 : eu > 0)) {
            if (AL.aq && AL.gen >= AL.gen_cap) {
                atomicExch(&AL.C->aq_over, 1);
            } else if (atomicExch(&G.astamp[u], AL.stamp) != AL.stamp) {
                if (AL.aq) aq_push_one(AL, u);
                else AL.list[atomicAdd(AL.cnt, 1)] = u;
            }
        }
    }
    __syncwarp();
}

// The cycle's decision after the scan: returns the height to push to, or -1
// after a relabel (hu updated, h(u) written), or -2 when u is done.
__device__ __forceinline__ int pr_decide(const DevGraph &G, int u, unsigned long long best, long long eu, int &hu,
                                         bool &relabelled, Counters &K) {
    if (eu <= 0) return -2;
    if (best == ~0ull) {
        hu = G.n;
        if ((threadIdx.x & 31) == 0) {
            G.h[u] = G.n;
            ++K.relabel;
        }
        relabelled = true;
        return -2;
    }
    const int hh = (int)(best >> 32);
    if (hu <= hh) {
        hu = hh + 1;
        if ((threadIdx.x & 31) == 0) {
            G.h[u] = hu;
            ++K.relabel;
        }
        relabelled = true;
        return -1;
    }
    return hh;
}

// u with one round of arcs (<= 32 kIlp)
template <bool PULL>
__device__ __forceinline__ void push_relabel_small_t(const DevGraph &G, int u, int beg, int end, int kc,
                                                  const ActList &AL, const unsigned char *pt, unsigned char side,
                                                  Counters &K) {
    const int lane = threadIdx.x & 31;
    int hu = bcast_ld(&G.h[u]);
    bool relabelled = false;
    for (int c = 0; c < kc && hu < G.n; ++c) {
        const long long eu = bcast_ld(&G.e[u]);
        ArcRound R;
        load_round_t<PULL, true>(G, beg, end, R, pt, side);
        K.pr_arcs += round_arcs(beg, end);
        const unsigned long long best = warp_min(round_min_key(R, beg, beg));
        const int hh = pr_decide(G, u, best, PULL ? -eu : eu, hu, relabelled, K);
        if (hh == -2) break;
        if (hh == -1) continue;
        int d[kIlp];
        long long tot;
        round_amounts(R, hh, PULL ? -eu : eu, d, tot);
        const long long sent = warp_sum(move_round<PULL>(G, beg, d, R, AL, K));
        if (lane == 0 && sent) add_ll(&G.e[u], PULL ? sent : -sent);
        __syncwarp();
    }
    pr_finish_t<PULL>(G, u, hu, relabelled, AL);
}

// u with more than one round of arcs (<= kHubDeg): the arcs are staged in
// the warp's shared memory (heads once, residuals and heights every cycle),
// and the pushes go along the staged arcs at height h^ in arc order, 32 arcs
// a step.
template <bool PULL>
__device__ __forceinline__ void push_relabel_staged_t(const DevGraph &G, int u, int beg, int end, int kc,
                                                      const ActList &AL, const unsigned char *pt,
                                                      unsigned char side, int *stg, Counters &K) {
    const int lane = threadIdx.x & 31;
    int *sv = stg, *sr = stg + kStgInts, *sh = stg + 2 * kStgInts;
    stage_copy(G.head, sv, beg, end, G.A, G.al16);
    int hu = bcast_ld(&G.h[u]);
    bool relabelled = false;
    for (int c = 0; c < kc && hu < G.n; ++c) {
        const long long eu = bcast_ld(&G.e[u]);
        stage_copy(PULL ? G.rr : G.r, sr, beg, end, G.A, G.al16);
        stage_wait();
        K.pr_arcs += (end - beg + 31 - lane) / 32;
        const unsigned long long best = warp_min(stage_heights(G, sv, sr, sh, beg, end, pt, side));
        const int hh = pr_decide(G, u, best, PULL ? -eu : eu, hu, relabelled, K);
        if (hh == -2) break;
        if (hh == -1) continue;
        const long long sent = stage_moves<PULL>(G, sv, sr, sh, beg, end, hh, PULL ? -eu : eu, AL, K);
        if (lane == 0 && sent) add_ll(&G.e[u], PULL ? sent : -sent);
        __syncwarp();
    }
    pr_finish_t<PULL>(G, u, hu, relabelled, AL);
}

template <bool PULL>
__device__ __forceinline__ void push_relabel_warp_t(const DevGraph &G, int u, int kc, const ActList &AL,
                                                    const unsigned char *pt, unsigned char side, int *stg,
                                                    Counters &K) {
    const int beg = __ldg(&G.row[u]), end = __ldg(&G.row[u + 1]);
    if (end - beg <= 32 * kIlp)
        push_relabel_small_t<PULL>(G, u, beg, end, kc, AL, pt, side, K);
    else
        push_relabel_staged_t<PULL>(G, u, beg, end, kc, AL, pt, side, stg, K);
}

__device__ __forceinline__ void push_relabel_warp(const DevGraph &G, int u, int kc, const ActList &AL, int *stg,
                                                  Counters &K) {
    push_relabel_warp_t<false>(G, u, kc, AL, nullptr, 0, stg, K);
}

// Algorithm 3 over the arcs [a0, a1) of vertex u (height hu) by one warp:
// every residual arc u -> v with h(u) > h(v) + 1 is saturated, moving its
// residual as excess to v.  With PULL it is the h- form (Algorithm 7): every
// residual arc v -> u with h(u) > h(v) + 1 is saturated, moving the residual
// into u.  With a partition array pt only arcs within u's part count.
// Returns this lane's share of the excess moved out of u (PULL: into u).
template <bool PULL>
__device__ __forceinline__ long long remove_invalid_range_t(const DevGraph &G, int hu, int a0, int a1,
                                                            const unsigned char *pt, unsigned char side,
                                                            Counters &K) {
    const int lane = threadIdx.x & 31;
    long long moved = 0;
    for (int b0 = a0; b0 < a1; b0 += 32 * kIlp) {
        ArcRound R;
        load_round_t<PULL, false>(G, b0, a1, R, pt, side);
        K.ri_arcs += round_arcs(b0, a1);
#pragma unroll
        for (int j = 0; j < kIlp; ++j) {
            if (R.ra[j] > 0 && hu > R.hv[j] + 1) {
                const int a = b0 + 32 * j + lane;
                move_arc<PULL>(G, a, __ldg(&G.rev[a]), R.v[j], R.ra[j]);
                moved += R.ra[j];
                ++K.ri_moves;
            }
        }
    }
    return moved;
}

template <bool PULL>
__device__ __forceinline__ void remove_invalid_warp_t(const DevGraph &G, int u, int *moved_flag,
                                                      const unsigned char *pt, unsigned char side, Counters &K) {
    const int lane = threadIdx.x & 31;
    const int beg = __ldg(&G.row[u]), end = __ldg(&G.row[u + 1]);
    const int hu = __shfl_sync(kFull, lane == 0 ? lcg(&G.h[u]) : 0, 0);
    const long long moved = warp_sum(remove_invalid_range_t<PULL>(G, hu, beg, end, pt, side, K));
    if (lane == 0 && moved) {
        add_ll(&G.e[u], PULL ? moved : -moved);
        *moved_flag = 1;   // once per warp
    }
}

// Hub cycle helpers (the cooperative PushRelabel of high-degree vertices).
// H1 scan of one kPrChunk-arc item [a0, a1) of hub u (first arc beg): the
// lowest (height, arc) key over its residual arcs (PULL: arcs into u).
template <bool PULL>
__device__ __forceinline__ unsigned long long hub_scan_item(const DevGraph &G, int a0, int a1, int beg,
                                                            const unsigned char *pt, unsigned char side,
                                                            Counters &K) {
    unsigned long long best = ~0ull;
    for (; a0 < a1; a0 += 32 * kIlp) {
        ArcRound R;
        load_round_t<PULL, false>(G, a0, a1, R, pt, side);
        K.pr_arcs += round_arcs(a0, a1);
        const unsigned long long k = round_min_key(R, a0, beg);
        best = k < best ? k : best;
    }
    return best;
}

// H3 of one item: moves along the item's residual arcs at height hh, in arc
// order, each warp reserving its share of what the hub has left to move
// (*rem) with one atomic.  Returns the amount this warp moved (all lanes).
template <bool PULL>
__device__ __forceinline__ long long hub_move_item(const DevGraph &G, int a0, int a1, int hh, long long *rem,
                                                   const ActList &AL, const unsigned char *pt, unsigned char side,
                                                   bool skip_done, Counters &K) {
    const int lane = threadIdx.x & 31;
    long long sent = 0;
    for (; a0 < a1; a0 += 32 * kIlp) {
        // the hub's excess may already be reserved by the items before this
        // one (not checked in the first push-pull stage, where scanning every
        // item measured faster: its pushes spread over the hub's arcs)
        if (skip_done && bcast_ld(rem) <= 0) break;
        ArcRound R;
        // (the arcs H1 scanned in this cycle: not counted again)
        load_round_t<PULL, true>(G, a0, a1, R, pt, side);
        int ra[kIlp];
        long long incl[kIlp], tot = 0;
#pragma unroll
        for (int j = 0; j < kIlp; ++j) {
            ra[j] = (R.ra[j] > 0 && R.hv[j] == hh) ? R.ra[j] : 0;
            incl[j] = warp_incl_scan(ra[j]) + tot;   // arc order: round j, then lane
            tot = __shfl_sync(kFull, incl[j], 31);
        }
        if (tot == 0) continue;
        long long old = 0;
        if (lane == 0)
            old = (long long)atomicAdd(reinterpret_cast<unsigned long long *>(rem), (unsigned long long)(-tot));
        old = __shfl_sync(kFull, old, 0);
        if (old <= 0) break;
        int d[kIlp];
#pragma unroll
        for (int j = 0; j < kIlp; ++j) {
            const long long dj = old - (incl[j] - ra[j]);
            d[j] = dj < 0 ? 0 : (dj > ra[j] ? ra[j] : (int)dj);
        }
        sent += move_round<PULL>(G, a0, d, R, AL, K);
    }
    return warp_sum(sent);
}

// Add the warp's counters to the statistics st and clear them.  All 32 lanes
// call.
__device__ __forceinline__ void flush_counters(Counters &K, long long *st) {
    const unsigned vals[9] = {K.bfs_verts, K.bfs_arcs, K.pr_arcs, K.push, K.relabel, K.ri_arcs, K.ri_moves,
                              K.clamped, K.resat};
    const int idx[9] = {S_BFS_VERTS, S_BFS_ARCS, S_PR_ARCS, S_PUSH, S_RELABEL, S_RI_ARCS, S_RI_MOVES, S_CLAMPED,
                        S_RESAT};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const long long v = warp_sum((long long)vals[i]);
        if ((threadIdx.x & 31) == 0 && v) add_ll(&st[idx[i]], v);
    }
    K = Counters{};
}

// The same at the end of the kernel, summed over the CTA in shared memory
// first: one global atomic per statistic and CTA instead of one per warp.
// Every thread of the CTA calls.
__device__ __forceinline__ void flush_counters_cta(Counters &K, long long *st) {
    __shared__ unsigned long long s_sum[9];
    if (threadIdx.x < 9) s_sum[threadIdx.x] = 0;
    __syncthreads();
    const unsigned vals[9] = {K.bfs_verts, K.bfs_arcs, K.pr_arcs, K.push, K.relabel, K.ri_arcs, K.ri_moves,
                              K.clamped, K.resat};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const long long v = warp_sum((long long)vals[i]);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_sum[i], (unsigned long long)v);
    }
    __syncthreads();
    if (threadIdx.x < 9 && s_sum[threadIdx.x]) {
        int slot;
        switch (threadIdx.x) {
            case 0: slot = S_BFS_VERTS; break;
            case 1: slot = S_BFS_ARCS; break;
            case 2: slot = S_PR_ARCS; break;
            case 3: slot = S_PUSH; break;
            case 4: slot = S_RELABEL; break;
            case 5: slot = S_RI_ARCS; break;
            case 6: slot = S_RI_MOVES; break;
            case 7: slot = S_CLAMPED; break;
            default: slot = S_RESAT; break;
        }
        add_ll(&st[slot], (long long)s_sum[threadIdx.x]);
    }
    K = Counters{};
}

// ------------------------------------------- staged BFS work items --
// The grid-wide top-down item phase of a BFS level stages each kChunk-arc
// item's heads and residuals (the residual of the arc into the frontier
// vertex, or out of it on the pull side of a push-pull search) in the warp's
// shared memory by cp.async, one item ahead: the copies of the next item are
// in flight while the warp scans the current one from shared memory, so an
// arc round waits only for the heights of its heads.  Residuals do not change
// during a BFS level, so the early copy is exact.
constexpr int kItemBuf = kChunk + 8;       // ints per array of one staged item
constexpr int kItemWarp = 4 * kItemBuf;    // two items (heads, residuals) per warp
constexpr int kItemOff = 2 * kSoloCap;     // after the frontier stages
static_assert(kItemOff + (kBlock / 32) * kItemWarp <= kDynSmem / 4, "staged items exceed the shared memory");

struct ItemMeta {
    int x, y, a1;   // vertex, first arc, end of the item's arcs
    bool fwd;       // pull side of a push-pull search: forward residuals
};

__device__ __forceinline__ ItemMeta item_meta(const DevGraph &G, int c, bool dual) {
    const int2 it = lcg(&G.cb[c]);
    ItemMeta m;
    m.x = it.x;
    m.y = it.y;
    m.a1 = min(it.y + kChunk, __ldg(&G.row[it.x + 1]));
    m.fwd = dual && G.part[it.x] == kPartS;
    return m;
}

__device__ __forceinline__ void item_issue(const DevGraph &G, const ItemMeta &m, int *buf) {
    stage_copy(G.head, buf, m.y, m.a1, G.A, G.al16);
    stage_copy(m.fwd ? G.r : G.rr, buf + kItemBuf, m.y, m.a1, G.A, G.al16);
}

// bfs_visit_n over arcs whose heads and residuals are staged (index a - base).
__device__ __forceinline__ void bfs_visit_staged(const DevGraph &G, const int *sv, const int *sr, int base,
                                                 const int (&a)[kIlpB], const bool (&ok)[kIlpB], unsigned fwd,
                                                 bool dual, int L, Front &F, Counters &K) {
    const int n = G.n;
    int v[kIlpB], rin[kIlpB], hv[kIlpB];
    bool disc[kIlpB];
#pragma unroll
    for (int j = 0; j < kIlpB; ++j) {
        v[j] = ok[j] ? sv[a[j] - base] : 0;
        rin[j] = ok[j] ? sr[a[j] - base] : 0;
        K.bfs_arcs += ok[j];
    }
#pragma unroll
    for (int j = 0; j < kIlpB; ++j) hv[j] = (rin[j] > 0 && v[j] != G.s) ? lcg(&G.h[v[j]]) : -1;
#pragma unroll
    for (int j = 0; j < kIlpB; ++j) disc[j] = hv[j] == n && atomicCAS(&G.h[v[j]], n, L + 1) == n;
    bfs_discovered_n(G, disc, v, fwd, dual, F, K);
}

// debug_checks: record a failed check (the first one's kind and index) and
// make the state invalid until the next mf_solve; the caller skips the
// access.  Kinds: 1 list entry out of range, 2 excess != net inflow, 3
// residual pair or mirror inconsistent.
__device__ __forceinline__ void check_fail(Ctl *C, int kind, long long where) {
    if ((atomicOr(&C->status, ST_CHECK) & ST_CHECK) == 0)
        C->chk_where = ((long long)kind << 40) | (where & 0xffffffffffll);
}

// A vertex id read from a list or queue, checked when debug_checks is on.
__device__ __forceinline__ bool vertex_ok(const Job &J, Ctl *C, int u, int n) {
    if (!J.debug || (u >= 0 && u < n)) return true;
    check_fail(C, 1, u);
    return false;
}

// ------------------------------------------------------------ the kernel --
// Grid barrier inside k_solve; CTA 0's thread 0 charges the time since the
// previous barrier to a phase bucket of the statistics and, when tracing is
// on, appends a record (phase, loop iteration, step, mode, count, time).
#define ST (J.st)
#define TR (J.trace)
#define MF_SYNC_T(bucket, step, mode, aux)                                    \
    do {                                                                      \
        if (!grid_sync(C)) return;                                            \
        if (gtid == 0) {                                                      \
            const unsigned long long now_ = gtimer();                         \
            const long long dt_ = (long long)(now_ - tprev);                  \
            ST[bucket] += dt_;                                                \
            ST[S_BARRIERS] += 1;                                              \
            if (TR) {                                                         \
                const int k_ = C->trace_n++;                                  \
                if (k_ < G.trace_cap)                                         \
                    TR[k_] = TraceRec{(short)(bucket), (short)(mode),    \
                                           (int)it, (int)(step), (int)(aux), dt_}; \
            }                                                                 \
            tprev = now_;                                                     \
        }                                                                     \
    } while (0)
#define MF_SYNC(bucket) MF_SYNC_T(bucket, -1, 0, -1)
// The same record without a grid barrier (levels CTA 0 runs alone).
#define MF_TRACE_T(bucket, step, mode, aux)                                   \
    do {                                                                      \
        if (gtid == 0) {                                                      \
            const unsigned long long now_ = gtimer();                         \
            const long long dt_ = (long long)(now_ - tprev);                  \
            ST[bucket] += dt_;                                                \
            if (TR) {                                                         \
                const int k_ = C->trace_n++;                                  \
                if (k_ < G.trace_cap)                                         \
                    TR[k_] = TraceRec{(short)(bucket), (short)(mode),         \
                                      (int)it, (int)(step), (int)(aux), dt_}; \
            }                                                                 \
            tprev = now_;                                                     \
        }                                                                     \
    } while (0)

// PP: the instance that can run Dynamic Push-Pull (Alg. 8); the plain
// instance compiles without its code paths.
template <bool PP>
__global__ void __launch_bounds__(kBlock, 1) k_solve(DevGraph G, Job J) {
    Ctl *C = G.ctl;
    const int lane = threadIdx.x & 31;
    const long long gtid = (long long)blockIdx.x * kBlock + threadIdx.x;
    const long long gthreads = (long long)gridDim.x * kBlock;
    const int gwarp = (int)(gtid >> 5);
    const int nwarps = (int)(gthreads >> 5);
    const int n = G.n, s = G.s, t = G.t;
    Counters K;
    // BFS frontiers in shared memory: CTA 0's small-frontier levels, and the
    // warps' staged entries in grid-wide levels (barriers keep them apart)
    // dynamic shared memory (kDynSmem bytes), used by one kind of phase at a
    // time (grid barriers keep them apart): the BFS frontiers at its start,
    // the warps' arc stages of PushRelabel
    extern __shared__ __align__(16) int s_dyn[];
    int *const s_bfs = s_dyn;
    int *const stg = s_dyn + (threadIdx.x >> 5) * kStgWarp;
    static_assert(2 * kSoloCap * 4 <= kDynSmem, "the shared frontiers exceed the dynamic shared memory");
    static_assert(kWq * (kBlock / 32) <= 2 * kSoloCap, "frontier stages exceed the shared frontier");
    static_assert(kWq >= 32 * kIlpB, "a stage holds one round of arcs");
    unsigned long long tprev = gtimer();
    long long it = -1;   // loop iteration (-1 before the loop, for trace records)

    // A sticky error (iteration cap, barrier wait) invalidates the state
    // until the next mf_solve, which clears it before launching.
    if (__ldcg(&C->status) & ST_STICKY) return;
    const unsigned stamp_base = __ldcg(&C->stamp_base) + 1u;
    // JOB_AUTO: the policy kernel launched just before chose repair or
    // recompute and KERNELCYCLES
    int kind = J.kind, kc = J.kc, jmode = J.mode;
    bool pp_pick = true;   // a fixed job of a push-pull graph repairs by push-pull
    if (kind == JOB_AUTO) {
        kind = lcg(&C->pol_kind);
        kc = lcg(&C->pol_kc);
        jmode = lcg(&C->pol_mode);
        pp_pick = jmode == MF_MODE_PUSH_PULL;
        if (pp_pick) jmode = MF_MODE_DATA_DRIVEN;   // the plain loop of push-pull's stage 2
    }
    if (kind == JOB_REFRESH && lcg(&C->heights_exact)) return;
    const bool batch_job = kind == JOB_REPAIR || kind == JOB_RECOMPUTE;
    const int kb = J.k_dev ? lcg(J.k_dev) : J.k;          // batch entries
    const unsigned seq = __ldcg(&C->bseq) + 1u;           // this batch's stamp
    if (gtid == 0) {
        for (int i = 0; i < S_COUNT; ++i) ST[i] = 0;
        ST[S_BATCH] = batch_job ? kb : 0;
        C->t_start = gtimer();
        if (TR) C->trace_n = 0;
    }

    // Dynamic Push-Pull (Alg. 8) needs the exact cut of the previous state:
    // T = {h < n} can reach a sink, S = {h >= n} cannot
    const bool pp = PP && J.pp && pp_pick && kind == JOB_REPAIR && G.part && lcg(&C->cut_exact);
    if (pp)
        for (long long v0 = gtid; v0 < n; v0 += 4 * gthreads) {   // four heights in flight per thread
            int hv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) hv[j] = v0 + j * gthreads < n ? lcg(&G.h[v0 + j * gthreads]) : 0;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (v0 + j * gthreads < n) G.part[v0 + j * gthreads] = hv[j] < n ? kPartT : kPartS;
        }

    // ---- batch: validate, then apply (Algorithm 5) ----------------------
    bool fast = false;   // pure-increment batch that cannot change the cut
    if (batch_job) {
        for (long long i = gtid; i < kb; i += gthreads) {
            const int eid = J.ids[i];
            bool bad = eid < 0 || eid >= G.m;
            int nc = 0;
            if (!bad) {
                long long v = J.caps[i];
                if (J.flags & MF_DELTA) {
                    v += lcg(&G.cap_edge[eid]);
                    if (v < 0) v = 0;
                }
                if (v < 0 || v > G.cap_limit) bad = true;
                else nc = (int)v;
                if (atomicExch(&G.stamp[eid], seq) == seq) bad = true;  // duplicate id
            }
            J.newc[i] = nc;
            if (bad) atomicOr(&C->batch_err, 1);
        }
        MF_SYNC(S_T_BATCH);
        if (lcg(&C->batch_err)) {
            grid_sync(C);
            if (gtid == 0) {
                atomicOr(&C->status, ST_EINVAL);
                C->batch_err = 0;
                C->bseq = seq;
            }
            return;
        }
        // c_f(u,v) += c'(u,v) - c(u,v)  (Alg. 5, lines 1-3)
        bool blocks = false;   // this thread saw a decrement or an increment across the cut
        for (long long i = gtid; i < kb; i += gthreads) {
            const int eid = J.ids[i];
            const int nc = lcg(&J.newc[i]);
            const int d = nc - lcg(&G.cap_edge[eid]);
            G.cap_edge[eid] = nc;
            J.dlt[i] = d;
            const int a = __ldg(&G.arc_of_edge[eid]);
            if (a >= 0 && d != 0) {
                atomicAdd(&G.cap[a], d);
                if (kind == JOB_REPAIR) {
                    const int b = __ldg(&G.rev[a]);
                    atomicAdd(&G.r[a], d);
                    atomicAdd(&G.rr[b], d);
                    // an increment can raise the flow only on an arc from
                    // the side that cannot reach a sink to the side that can
                    if (d < 0 || (lcg(&G.h[__ldg(&G.head[b])]) >= n && lcg(&G.h[__ldg(&G.head[a])]) < n))
                        blocks = true;
                }
            }
        }
        // one store per warp: tens of thousands of same-address stores from
        // every SM serialise at one L2 slice
        if (__any_sync(kFull, blocks) && lane == 0) C->inc_block = 1;
        MF_SYNC(S_T_BATCH);
        // With the exact cut S = {h >= n} of the previous state (no residual
        // arc from S to T), increments on arcs that do not go from S to T
        // leave that cut saturated and its capacity unchanged, so the flow
        // value stays the same and the state stays terminal (Sec. 4: only
        // changes on the cut's arcs can change the maximum).
        fast = kind == JOB_REPAIR && lcg(&C->cut_exact) && !lcg(&C->inc_block);
        if (kind == JOB_REPAIR && !fast) {
            // flow above the new capacity goes back: the tail keeps it as
            // excess, the head becomes deficient (Alg. 5, lines 4-11; the
            // excess update is the exact incremental form of Alg. 4 line 2).
            for (long long i = gtid; i < kb; i += gthreads) {
                if (lcg(&J.dlt[i]) >= 0) continue;
                const int a = __ldg(&G.arc_of_edge[J.ids[i]]);
                if (a < 0) continue;
                const int old = atomicMax(&G.r[a], 0);
                if (old < 0) {
                    const int o = -old;
                    const int b = __ldg(&G.rev[a]);
                    atomicAdd(&G.rr[b], o);
                    atomicSub(&G.r[b], o);
                    atomicSub(&G.rr[a], o);
                    add_ll(&G.e[__ldg(&G.head[b])], (long long)o);
                    add_ll(&G.e[__ldg(&G.head[a])], -(long long)o);
                    ++K.clamped;
                }
            }
            MF_SYNC(S_T_BATCH);
            if (pp) {
                // Alg. 8: saturate every residual arc from S to T.  Before the
                // batch the cut had none, so only raised batch arcs can have one.
                for (long long i = gtid; i < kb; i += gthreads) {
                    if (lcg(&J.dlt[i]) <= 0) continue;
                    const int a = __ldg(&G.arc_of_edge[J.ids[i]]);
                    if (a < 0) continue;
                    const int b = __ldg(&G.rev[a]);
                    const int u = __ldg(&G.head[b]), v = __ldg(&G.head[a]);
                    if (G.part[u] != kPartS || G.part[v] != kPartT) continue;
                    const int ra = atomicExch(&G.r[a], 0);
                    if (ra > 0) {
                        atomicSub(&G.rr[b], ra);
                        atomicAdd(&G.r[b], ra);
                        atomicAdd(&G.rr[a], ra);
                        add_ll(&G.e[u], -(long long)ra);
                        add_ll(&G.e[v], (long long)ra);
                    }
                }
                MF_SYNC(S_T_BATCH);
            }
        }
    }
    const bool pp_ran = pp && !fast;
    int stage = pp_ran ? 1 : 0;   // 0 plain loop; push-pull: 1 push on T and pull on S, 2 push on P

    // ---- zero flow (Algorithm 1, first two loops) ------------------------
    if (kind == JOB_SOLVE || kind == JOB_RECOMPUTE) {
        for (long long a = gtid; a < G.A; a += gthreads) {
            G.r[a] = lcg(&G.cap[a]);
            G.rr[a] = lcg(&G.cap[__ldg(&G.rev[a])]);
        }
        for (long long v = gtid; v < n; v += gthreads) G.e[v] = 0;
        MF_SYNC(S_T_BATCH);
    }

    // ---- saturate the source arcs (Alg. 1 third loop, Alg. 4 lines 3-7) --
    // (on the fast path every source arc that regains residual leads into
    // S, so the moved excess stays on vertices that cannot reach a sink)
    if (kind != JOB_REFRESH) {
        long long moved = 0;
        const int a0 = __ldg(&G.row[s]), a1 = __ldg(&G.row[s + 1]);
        for (long long a = a0 + gtid; a < a1; a += gthreads) {
            const int ra = lcg(&G.r[a]);
            ++K.resat;
            if (ra > 0) {
                const int b = __ldg(&G.rev[a]);
                G.r[a] = 0;
                G.rr[b] = 0;
                atomicAdd(&G.r[b], ra);
                atomicAdd(&G.rr[a], ra);
                add_ll(&G.e[__ldg(&G.head[a])], (long long)ra);
                moved += ra;
            }
        }
        moved = warp_sum(moved);
        if (lane == 0 && moved) add_ll(&G.e[s], -moved);
        MF_SYNC(S_T_BATCH);
    }

    // ---- static push-pull (Sec. 4.2): also saturate every arc into t; the
    // vertices left deficient become secondary sinks of the loop below
    if (J.sink_sat && (kind == JOB_SOLVE || kind == JOB_RECOMPUTE)) {
        long long moved = 0;
        const int a0 = __ldg(&G.row[t]), a1 = __ldg(&G.row[t + 1]);
        for (long long a = a0 + gtid; a < a1; a += gthreads) {
            const int rin = lcg(&G.rr[a]);   // residual of v -> t
            if (rin > 0) {
                const int b = __ldg(&G.rev[a]);
                G.r[b] = 0;
                G.rr[a] = 0;
                atomicAdd(&G.r[a], rin);
                atomicAdd(&G.rr[b], rin);
                add_ll(&G.e[__ldg(&G.head[a])], -(long long)rin);
                moved += rin;
            }
        }
        moved = warp_sum(moved);
        if (lane == 0 && moved) add_ll(&G.e[t], moved);
        MF_SYNC(S_T_BATCH);
    }

    // ---- device loop (Algorithm 4 while-loop) ----------------------------
    bool early = false;   // stopped when PushRelabel left no active vertex
    unsigned snext = stamp_base;   // next unused activation stamp
    for (it = 0; !fast; ++it) {
        const int par = (int)(it & 1);
        // the stamp of the first PushRelabel pass's queue: the BFS gives it to
        // the worklist entries it files (queued from the start)
        const unsigned wmark0 = snext++;
        // height init: t and deficient vertices are sinks (height 0), all
        // others n; the sinks form BFS level 0.
        if (gtid == 0) {
            C->aq_head = C->aq_tail = C->aq_done = C->aq_over = C->aq_maxgen = C->aq_fin = 0;
            C->qcnt[1] = 0;
            C->qcnt[2] = 0;
            C->ccnt[0] = 0;
            C->asum[1] = C->asum[2] = 0;
            C->acnt[0] = C->acnt[1] = C->acnt[2] = 0;
            C->rlcnt = 0;
            C->rhcnt = 0;
            C->phc[1] = 0;
            C->wcnt = 0;
            C->hcnt = 0;
            C->hccnt = 0;
            C->hub_act[0] = C->hub_act[1] = 0;
            C->hlc[0] = C->hlc[1] = 0;
            C->dacc[par ^ 1] = 0;
            if (gtimer() - C->t_start > J.time_limit_ns) C->abort_loop = 1;
        }
        {
            long long dsum = 0, rdeg = 0;
            constexpr int kRs = 4;   // vertices in flight per thread (their excesses loaded first)
            for (long long vb0 = (long long)gwarp * 32; vb0 < n; vb0 += kRs * gthreads) {
                long long evs[kRs];
#pragma unroll
                for (int j = 0; j < kRs; ++j) {
                    const long long v = vb0 + j * gthreads + lane;
                    evs[j] = v < n ? lcg(&G.e[v]) : 0;
                }
#pragma unroll
                for (int j = 0; j < kRs; ++j) {
                    const long long v = vb0 + j * gthreads + lane;
                    bool root = false;
                    if (v < n) {
                        const long long ev = evs[j];
                        if (stage == 0) {
                            root = (v == t) || (v != s && ev < 0);
                            G.h[v] = root ? 0 : n;
                            if (root && v != t) dsum += ev;
                        } else if (stage == 1) {
                            // Alg. 8: h+ roots are t and the deficient vertices of T,
                            // h- roots are s and the overflowing vertices of S (both
                            // heights live in h: the two sides are disjoint)
                            root = G.part[v] == kPartT ? (v == t || ev < 0) : (v == s || ev > 0);
                            G.h[v] = root ? 0 : n;
                        } else {
                            // the subgraph P: its deficient vertices are the sinks;
                            // the rest of the graph sits at n + 1, out of reach
                            const bool inP = G.part[v] == kPartP;
                            root = inP && ev < 0;
                            G.h[v] = inP ? (root ? 0 : n) : n + 1;
                        }
                        if (root) rdeg += __ldg(&G.row[v + 1]) - __ldg(&G.row[v]);
                    }
                    warp_append(root, (int)v, &C->qcnt[0], G.qb0);
                }
            }
            dsum = warp_sum(dsum);
            rdeg = warp_sum(rdeg);
            if (lane == 0 && dsum) add_ll(&C->dacc[par], dsum);
            if (lane == 0 && rdeg) add_ll(&C->asum[0], rdeg);
        }
        MF_SYNC_T(S_T_RESET, 0, 0, lcg(&C->qcnt[0]));
        // the flags of the next iteration: their last readers (the previous
        // iteration's exit test) are all past this barrier
        if (gtid == 0) C->ri_moved[par ^ 1] = 0;

        // backward BFS from the sinks over residual arcs (global relabel),
        // level-synchronous and direction-optimising: top-down from the
        // frontier while it is small, bottom-up from the unvisited vertices
        // while the frontier holds more than 1/14 of the unvisited arcs.
        int L = 0;
        bool bottom_up = false;
        long long arcs_seen = 0;
        for (;;) {
            const int cur = lcg(&C->qcnt[L % 3]);
            if (cur == 0) break;
            const long long mf = lcg(&C->asum[L % 3]);
            arcs_seen += mf;
            const bool dual = PP && stage == 1;   // push-pull: backward on T, forward on S
            // (the dual search of push-pull takes a smaller vertex share: its
            // first frontier, the overflowing and deficient vertices of both
            // sides, is a few percent of the vertices but touches few of the
            // others, which then scan all their arcs bottom-up)
            if (!bottom_up) bottom_up = mf * 14 > G.A - arcs_seen && cur * (dual ? 32LL : 64LL) > n;
            else bottom_up = cur * 24LL >= n;
            if (!bottom_up && mf <= kSoloArcs && cur <= kSoloCap) {
                // A small frontier: CTA 0 runs the levels alone, with the
                // frontiers in shared memory and in step by __syncthreads only,
                // until the frontier passes kSoloCap vertices or kSoloArcs arcs,
                // the search would turn bottom-up, or the frontier empties; it
                // then hands the frontier back in the global queue.  The rest
                // of the grid waits at one barrier.  Every thread has read this
                // level's counters before CTA 0 starts (the first barrier).
                MF_SYNC_T(S_T_BFS, L, 6, cur);
                if (blockIdx.x == 0) {
                    int (*s_front)[kSoloCap] = reinterpret_cast<int (*)[kSoloCap]>(s_bfs);
                    __shared__ int s_cnt[2];
                    __shared__ long long s_arcs[2];
                    __shared__ int s_big;
                    const int cw = threadIdx.x >> 5;
                    const int *F0 = (L & 1) ? G.qb1 : G.qb0;
                    for (int i = threadIdx.x; i < cur; i += kBlock) s_front[0][i] = lcg(&F0[i]);
                    if (threadIdx.x == 0) {
                        s_cnt[1] = 0;
                        s_arcs[1] = 0;
                        s_big = 0;
                    }
                    __syncthreads();
                    int Ls = L, cs = cur, b = 0;
                    long long seen = arcs_seen, mfs = 0;
                    for (;;) {
                        int *ccs = &C->ccnt[Ls % 3];
                        int *spill = (Ls & 1) ? G.qb0 : G.qb1;   // positions >= kSoloCap of the next frontier
                        Front SF{&s_cnt[b ^ 1], s_front[b ^ 1], &s_arcs[b ^ 1], kSoloCap, spill, nullptr, 0, 0, wmark0};
                        int gs = 32;   // frontier vertices per warp: fewer when they do not fill the warps
                        while (gs > 1 && (gs >> 1) * (kBlock / 32) >= cs) gs >>= 1;
                        for (int grp = cw; grp * gs < cs; grp += kBlock / 32) {
                            const int idx = grp * gs + lane;
                            int beg = 0, deg = 0;
                            bool fwd = false;
                            if (lane < gs && idx < cs) {
                                const int u = s_front[b][idx];
                                fwd = dual && G.part[u] == kPartS;
                                beg = __ldg(&G.row[u]);
                                deg = __ldg(&G.row[u + 1]) - beg;
                                if (deg > kBigDeg) {
                                    const int nc = (deg + kChunk - 1) / kChunk;
                                    const int pos = atomicAdd(ccs, nc);
                                    for (int c = 0; c < nc; ++c) G.cb[pos + c] = make_int2(u, beg + c * kChunk);
                                    s_big = 1;
                                    deg = 0;
                                }
                            }
                            bfs_expand_warp(G, beg, deg, fwd, dual, Ls, SF, K);
                        }
                        __syncthreads();
                        if (s_big) {
                            const int nch = lcg(ccs);
                            for (int c = cw; c < nch; c += kBlock / 32) {
                                const int2 item = lcg(&G.cb[c]);
                                const unsigned fw = (dual && G.part[item.x] == kPartS) ? (1u << kIlpB) - 1u : 0u;
                                const int a1 = min(item.y + kChunk, __ldg(&G.row[item.x + 1]));
                                for (int ab = item.y; ab < a1; ab += 32 * kIlpB) {
                                    int a[kIlpB];
                                    bool ok[kIlpB];
#pragma unroll
                                    for (int j = 0; j < kIlpB; ++j) {
                                        a[j] = ab + 32 * j + lane;
                                        ok[j] = a[j] < a1;
                                    }
                                    bfs_visit_n(G, a, ok, fw, dual, Ls, SF, K);
                                }
                            }
                            __syncthreads();
                        }
                        MF_TRACE_T(S_T_BFS, Ls, 4, cs);
                        ++Ls;
                        cs = s_cnt[b ^ 1];
                        mfs = s_arcs[b ^ 1];
                        __syncthreads();   // everyone has read the counts
                        b ^= 1;
                        if (threadIdx.x == 0) {
                            s_cnt[b ^ 1] = 0;
                            s_arcs[b ^ 1] = 0;
                            s_big = 0;
                            C->ccnt[Ls % 3] = 0;
                        }
                        if (cs == 0 || cs > kSoloCap || mfs > kSoloArcs ||
                            (mfs * 14 > G.A - (seen + mfs) && cs * 64LL > n))
                            break;
                        seen += mfs;
                        __syncthreads();
                    }
                    // hand the frontier of level Ls back in the global queue
                    int *Fg = (Ls & 1) ? G.qb1 : G.qb0;
                    for (int i = threadIdx.x; i < min(cs, kSoloCap); i += kBlock) Fg[i] = s_front[b][i];
                    if (threadIdx.x == 0) {
                        C->qcnt[Ls % 3] = cs;
                        C->asum[Ls % 3] = mfs;
                        C->qcnt[(Ls + 1) % 3] = 0;
                        C->asum[(Ls + 1) % 3] = 0;
                        C->solo_L = Ls;
                        C->solo_seen = seen;   // arcs of the levels run, without level Ls
                    }
                }
                MF_SYNC_T(S_T_BFS, L, 5, cur);
                L = lcg(&C->solo_L);
                arcs_seen = lcg(&C->solo_seen);
                continue;
            }
            const int *F = (L & 1) ? G.qb1 : G.qb0;
            int *NF = (L & 1) ? G.qb0 : G.qb1;
            int *ncnt = &C->qcnt[(L + 1) % 3];
            int *ccnt = &C->ccnt[L % 3];
            long long *asum = &C->asum[(L + 1) % 3];
            if (gtid == 0) {
                C->qcnt[(L + 2) % 3] = 0;
                C->ccnt[(L + 1) % 3] = 0;
                C->asum[(L + 2) % 3] = 0;
                if (bottom_up) ST[S_BU_LEVELS] += 1;
            }
            Front FR{ncnt, NF, asum, 0x7fffffff, nullptr, s_bfs + (threadIdx.x >> 5) * kWq, 0, 0, wmark0};
            if (bottom_up) {
                // groups of 32 consecutive vertex ids (warp w: groups w, w + W, ...)
                const int groups = (n + 31) / 32;
                BuPre pre = bu_prefetch(G, gwarp * 32);
                for (int grp = gwarp; grp < groups; grp += nwarps) {
                    const BuPre cur = pre;
                    if (grp + nwarps < groups) pre = bu_prefetch(G, (grp + nwarps) * 32);
                    bfs_bottom_up_group(G, grp * 32, cur, dual, L, FR, ccnt, K);
                }
            } else {
                // groups of gs frontier vertices (warp w: groups w, w + W, ...):
                // 32, or fewer when the frontier does not fill the grid's warps,
                // so that the arcs of a small frontier still spread over them
                int gs = 32;
                while (gs > 1 && (long long)(gs >> 1) * nwarps >= cur) gs >>= 1;
                for (int grp = gwarp; grp * gs < cur; grp += nwarps) {
                    const int idx = grp * gs + lane;
                    int beg = 0, deg = 0;
                    bool fwd = false;
                    const int u = (lane < gs && idx < cur) ? lcg(&F[idx]) : 0;
                    if (lane < gs && idx < cur && vertex_ok(J, C, u, n)) {
                        fwd = dual && G.part[u] == kPartS;
                        beg = __ldg(&G.row[u]);
                        deg = __ldg(&G.row[u + 1]) - beg;
                        if (deg > kBigDeg) {
                            const int nc = (deg + kChunk - 1) / kChunk;
                            const int pos = atomicAdd(ccnt, nc);
                            for (int c = 0; c < nc; ++c) G.cb[pos + c] = make_int2(u, beg + c * kChunk);
                            deg = 0;
                        }
                    }
                    bfs_expand_warp(G, beg, deg, fwd, dual, L, FR, K);
                }
            }
            front_flush(G, FR, dual, K);
            MF_SYNC_T(S_T_BFS, L, bottom_up ? 2 : 0, cur);
            const int nch = lcg(ccnt);
            if (nch > 0) {
                if (bottom_up) {
                    for (int c = gwarp; c < nch; c += nwarps) bfs_bottom_up_item(G, lcg(&G.cb[c]), dual, L, FR, K);
                } else {
                    // items staged one ahead (see item_issue)
                    int *const ibuf = s_dyn + kItemOff + (threadIdx.x >> 5) * kItemWarp;
                    int c = gwarp, b = 0;
                    ItemMeta cur = c < nch ? item_meta(G, c, dual) : ItemMeta{0, 0, 0, false};
                    if (c < nch) item_issue(G, cur, ibuf);
                    asm volatile("cp.async.commit_group;" ::: "memory");
                    ItemMeta nxt = c + nwarps < nch ? item_meta(G, c + nwarps, dual) : ItemMeta{0, 0, 0, false};
                    for (; c < nch; c += nwarps) {
                        if (c + nwarps < nch) item_issue(G, nxt, ibuf + (b ^ 1) * 2 * kItemBuf);
                        asm volatile("cp.async.commit_group;" ::: "memory");
                        const ItemMeta nn =
                            c + 2 * nwarps < nch ? item_meta(G, c + 2 * nwarps, dual) : ItemMeta{0, 0, 0, false};
                        asm volatile("cp.async.wait_group 1;" ::: "memory");   // the current item's copies
                        __syncwarp();
                        const int *sv = ibuf + b * 2 * kItemBuf;
                        const unsigned fw = cur.fwd ? (1u << kIlpB) - 1u : 0u;
                        for (int ab = cur.y; ab < cur.a1; ab += 32 * kIlpB) {
                            int a[kIlpB];
                            bool ok[kIlpB];
#pragma unroll
                            for (int j = 0; j < kIlpB; ++j) {
                                a[j] = ab + 32 * j + lane;
                                ok[j] = a[j] < cur.a1;
                            }
                            bfs_visit_staged(G, sv, sv + kItemBuf, cur.y & ~3, a, ok, fw, dual, L, FR, K);
                        }
                        __syncwarp();   // every lane is done with this buffer before it is refilled
                        cur = nxt;
                        nxt = nn;
                        b ^= 1;
                    }
                    asm volatile("cp.async.wait_all;" ::: "memory");
                }
                front_flush(G, FR, dual, K);
                MF_SYNC_T(S_T_BFS, L, bottom_up ? 3 : 1, nch);
            }
            ++L;
        }
        if (gtid == 0) ST[S_LEVELS] += L;

        // termination: no active vertex under the fresh BFS heights
        const int nw = lcg(&C->wcnt);
        const int nh = lcg(&C->hcnt);
        if (nw == 0 && nh == 0) {
            if (stage == 1) {
                // Alg. 8: what neither search reached -- overflowing vertices
                // of T that reach no sink, deficient vertices of S that no
                // source reaches -- forms P, where the push phase continues
                for (long long v = gtid; v < n; v += gthreads)
                    if (v != s && v != t && lcg(&G.h[v]) == n) G.part[v] = kPartP;
                MF_SYNC_T(S_T_RESET, 2, 0, 0);
                stage = 2;
                continue;
            }
            break;
        }
        if (it >= J.max_iters) {
            if (gtid == 0) atomicOr(&C->status, ST_ITERS);
            break;
        }
        if (lcg(&C->abort_loop)) {   // written before the height-init barrier
            if (gtid == 0) atomicOr(&C->status, ST_TIME);
            break;
        }

        // PushRelabel (Alg. 2), in passes.  A pass serves the high-degree
        // vertices of its hub list together, in kPrChunk-arc items over the
        // whole grid (cooperative cycles), and then the worklist, one warp per
        // vertex, in activation rounds: a vertex that a push turns active joins
        // the list of the next round instead of waiting for the next BFS.
        // Cycles and rounds are separated by grid barriers, so no vertex is
        // ever processed by two warps at once.  High-degree vertices that a
        // pass turns active again form the hub list of the next pass.
        const unsigned rstamp_it = snext++;   // relabel-list stamp of this iteration
        if (gtid == 0) {
            C->qcnt[0] = 0;
            C->asum[0] = 0;
        }
        bool rounds_clean = true;   // the last activation round left no active vertex
        bool hubs_clean = true;     // the last hub cycle left no hub active
        int pend = 0;               // hubs that the last pass turned active
        // Rounds per pass: kMaxRounds, and past that, while the list holds at
        // most one vertex per warp, as many as the BFS just run had levels --
        // such a round costs about what a BFS level costs, so on deep graphs
        // (grids) finishing a few active vertices by rounds is cheaper than
        // another global relabel.
        const int max_rounds = L > kMaxRounds ? L : kMaxRounds;
        for (int pass = 0; pass < (PP ? kMaxPassesPP : kMaxPasses); ++pass) {
            const int *HL = (pass & 1) ? G.hl2 : G.hl;
            const int nhp = pass == 0 ? nh : pend;
            const unsigned wstamp = pass == 0 ? wmark0 : snext++;   // this pass's round-0 list / queue
            const unsigned hstamp = snext++;   // the next pass's hub list
            int *const pcnt = &C->phc[(pass + 1) & 1];
            // pass 0 appends to phc[1] and starts its rounds on the counters
            // zeroed at the iteration's start; a later pass always has hubs,
            // so its set-up barrier comes before any use of what is zeroed
            // here (the previous pass's rounds ended with an empty list)
            if (gtid == 0) {
                if (pass > 0) {
                    *pcnt = 0;
                    C->wcnt = 0;
                    C->acnt[0] = C->acnt[1] = C->acnt[2] = 0;
                }
                C->hub_act[0] = C->hub_act[1] = 0;
                C->hlc[0] = C->hlc[1] = 0;
                ST[S_WL] += nhp;
            }
            // the data-driven and push-pull modes run PushRelabel from the
            // activation queue; the topology-driven mode in rounds
            const bool qmode = jmode != MF_MODE_TOPOLOGY && G.aq != nullptr;
            const ActList AL0{&C->wcnt, G.wl,   wstamp,     rstamp_it, pcnt, (pass & 1) ? G.hl : G.hl2,
                              hstamp,   qmode ? G.aq : nullptr, G.qc, 0, max_rounds, C};
            bool pass_hubs_clean = true;
            if (nhp > 0) {
                pass_hubs_clean = false;
                for (int i = gwarp; i < nhp; i += nwarps) {
                    const int u = bcast_ld(&HL[i]);
                    if (!vertex_ok(J, C, u, n)) continue;   // warp-uniform
                    const int beg = __ldg(&G.row[u]);
                    const int nc = (__ldg(&G.row[u + 1]) - beg + kPrChunk - 1) / kPrChunk;
                    int pos = 0;
                    if (lane == 0) {
                        pos = atomicAdd(&C->hccnt, nc);
                        G.hkey[i] = ~0ull;
                        G.hnit[i] = nc;
                        G.hdone[i] = 0;
                        if (pass == 0) {
                            // right after the BFS a reached vertex's lowest
                            // residual neighbour sits exactly one level below
                            // it, so the first cycle's decision needs no scan:
                            // push to the arcs at height h(u) - 1
                            const long long eu = lcg(&G.e[u]);
                            G.hmode[i] = lcg(&G.h[u]);
                            G.hrem[i] = eu < 0 ? -eu : eu;
                        } else {
                            G.hmode[i] = 0;
                        }
                    }
                    pos = __shfl_sync(kFull, pos, 0);
                    for (int c = lane; c < nc; c += 32) G.hcl[pos + c] = make_int2(i, beg + c * kPrChunk);
                }
                MF_SYNC_T(S_T_HUB, -1, 0, nhp);
                // a later pass's queue: the previous pass's counters have been
                // read (before this barrier), and nothing is queued before the
                // first H3 (a later pass's first cycle has an H1 barrier)
                if (pass > 0 && gtid == 0)
                    C->aq_head = C->aq_tail = C->aq_done = C->aq_over = C->aq_maxgen = C->aq_fin = 0;
                const int nhc = lcg(&C->hccnt);
                const int hub_min = PP ? kMinHubCyclesPP : kMinHubCycles;
                const int hub_cycles = kc > hub_min ? kc : hub_min;
                for (int c = 0; c < hub_cycles; ++c) {
                    if (gtid == 0) ST[S_HUB_CYCLES] += 1;
                    const bool fresh = c == 0 && pass == 0;   // H1 decided by the BFS heights
                    // H1: lowest residual neighbour of every unfinished hub; the
                    // warp that completes a hub's last item takes the hub's
                    // decision (push at the lowest height, after a relabel when
                    // the hub is not above it; or finish)
                    // the cycle's items: all hub items in cycle 0, afterwards the
                    // items of the hubs still active after the previous cycle
                    const int2 *items = c == 0 ? G.hcl : ((c - 1) & 1 ? G.hlv1 : G.hlv0);
                    const int nitems = c == 0 ? nhc : lcg(&C->hlc[(c - 1) & 1]);
                    for (int w = fresh ? nitems : gwarp; w < nitems; w += nwarps) {
                        const int2 item = lcg(&items[w]);
                        const int i = item.x;
                        if (lcg(&G.hmode[i]) < 0) continue;
                        const int u = lcg(&HL[i]);
                        const int beg = __ldg(&G.row[u]);
                        const int a1 = min(item.y + kPrChunk, __ldg(&G.row[u + 1]));
                        // no push or relabel runs during H1, so every item of a hub
                        // sees the same e(u), h(u): the items of a hub that is no
                        // longer active skip the scan and only arrive
                        // (a hub of the pull side of a push-pull repair is
                        // active when deficient and scans its arcs in)
                        const unsigned char side = stage == 1 ? G.part[u] : kPartT;
                        const bool pull = PP && side == kPartS;
                        const long long eu0 = lcg(&G.e[u]);
                        const bool live = (pull ? eu0 < 0 : eu0 > 0) && lcg(&G.h[u]) < n;
                        const unsigned char *ptc = stage == 1 ? G.part : nullptr;
                        unsigned long long best = ~0ull;
                        if (live)
                            best = pull ? hub_scan_item<true>(G, item.y, a1, beg, ptc, side, K)
                                        : hub_scan_item<false>(G, item.y, a1, beg, ptc, side, K);
                        best = warp_min(best);
                        bool relabelled = false;
                        if (lane == 0) {
                            G.hikey[w] = (unsigned)(best >> 32);   // lowest height in this item
                            if (best != ~0ull) atomicMin(&G.hkey[i], best);
                            if (arrive_acq_rel(&G.hdone[i]) == lcg(&G.hnit[i]) - 1) {
                                const int hu = lcg(&G.h[u]);
                                const long long eu = pull ? -lcg(&G.e[u]) : lcg(&G.e[u]);   // amount to move
                                const unsigned long long key = __ldcg(&G.hkey[i]);
                                G.hkey[i] = ~0ull;
                                G.hdone[i] = 0;
                                int mode;
                                if (hu >= n || eu <= 0) {
                                    mode = -1;
                                } else if (key == ~0ull) {
                                    G.h[u] = n;
                                    ++K.relabel;
                                    relabelled = true;
                                    mode = -1;
                                } else {
                                    const int hh = (int)(key >> 32);
                                    // push to the arcs at height hh, after
                                    // relabelling u to hh + 1 if it is not
                                    // above them (the same cycle's H3 pushes:
                                    // a relabel followed by a rescan in the
                                    // next cycle cost a cycle per relabel)
                                    if (hu <= hh) {
                                        G.h[u] = hh + 1;
                                        ++K.relabel;
                                        relabelled = true;
                                    }
                                    if (hh + 1 < n) {
                                        mode = hh + 1;
                                        G.hrem[i] = eu;
                                    } else {
                                        mode = -1;
                                    }
                                }
                                G.hmode[i] = mode;
                                // (a pushing hub is counted, and listed for the
                                // next cycle, by its last H3 item if it is still
                                // active after its pushes)
                                // a relabelled hub's items join the iteration's
                                // RemoveInvalidEdges list once
                                if (relabelled && atomicExch(&G.rstamp[u], rstamp_it) == rstamp_it)
                                    relabelled = false;
                            }
                        }
                        // the deciding warp lists a newly relabelled hub's items
                        // for RemoveInvalidEdges
                        relabelled = __shfl_sync(kFull, relabelled, 0);
                        if (relabelled) {
                            const int nit = lcg(&G.hnit[i]);
                            int rpos = 0;
                            if (lane == 0) rpos = atomicAdd(&C->rhcnt, nit);
                            rpos = __shfl_sync(kFull, rpos, 0);
                            for (int q = lane; q < nit; q += 32) G.hri[rpos + q] = make_int2(u, beg + q * kPrChunk);
                        }
                    }
                    if (!fresh) MF_SYNC_T(S_T_HUB, c, 1, nitems);
                    // hub_act[(c+1)&1] was last read by the exit test of cycle c-1,
                    // which every thread has passed once it is past the H1 barrier;
                    // likewise the item count of the set-up, read before H1 (with
                    // no H1 barrier, it is zeroed after the H3 barrier instead)
                    if (gtid == 0) {
                        C->hub_act[(c + 1) & 1] = 0;
                        if (c == 0 && !fresh) C->hccnt = 0;
                    }
                    // H3: pushes along the lowest arcs; each warp reserves its share
                    // of the hub's excess with one atomic
                    // hlc[(c+1)&1] counted the list of cycle c-1, read before H1
                    if (gtid == 0) C->hlc[(c + 1) & 1] = 0;
                    for (int w = gwarp; w < nitems; w += nwarps) {
                        const int2 item = lcg(&items[w]);
                        const int i = item.x;
                        const int mode = lcg(&G.hmode[i]);
                        if (mode <= 0) continue;
                        const int hh = mode - 1;
                        const int u = lcg(&HL[i]);
                        const int beg = __ldg(&G.row[u]);
                        const int a1 = min(item.y + kPrChunk, __ldg(&G.row[u + 1]));
                        const unsigned char side = stage == 1 ? G.part[u] : kPartT;
                        const bool pull = PP && side == kPartS;
                        // (hikey: the item's lowest height, found by H1; else no arc at h^ here)
                        if (fresh || lcg(reinterpret_cast<const int *>(&G.hikey[w])) == hh) {
                            const unsigned char *ptc = stage == 1 ? G.part : nullptr;
                            if (pull) {
                                const long long got = hub_move_item<true>(G, item.y, a1, hh, &G.hrem[i], AL0, ptc,
                                                                          side, stage != 1, K);
                                if (lane == 0 && got) add_ll(&G.e[u], got);
                            } else {
                                const long long sent = hub_move_item<false>(G, item.y, a1, hh, &G.hrem[i], AL0,
                                                                            ptc, side, stage != 1, K);
                                if (lane == 0 && sent) add_ll(&G.e[u], -sent);
                            }
                        }
                        // the hub's last item to finish sees e(u) after all of
                        // its pushes: a hub still active takes its items into
                        // the next cycle's list
                        int pos = -1;
                        const int nit = lcg(&G.hnit[i]);
                        if (lane == 0) {
                            if (arrive_acq_rel(&G.hdone[i]) == nit - 1) {
                                G.hdone[i] = 0;
                                const long long eu = lcg(&G.e[u]);
                                if (lcg(&G.h[u]) < n && (pull ? eu < 0 : eu > 0)) {
                                    atomicAdd(&C->hub_act[c & 1], 1);
                                    pos = atomicAdd(&C->hlc[c & 1], nit);
                                }
                            }
                        }
                        pos = __shfl_sync(kFull, pos, 0);
                        if (pos >= 0) {
                            int2 *next_items = c & 1 ? G.hlv1 : G.hlv0;
                            for (int q = lane; q < nit; q += 32) next_items[pos + q] = make_int2(i, beg + q * kPrChunk);
                        }
                    }
                    MF_SYNC_T(S_T_HUB, c, 3, lcg(&C->hub_act[c & 1]));
                    if (gtid == 0 && fresh) C->hccnt = 0;
                    if (lcg(&C->hub_act[c & 1]) == 0) {
                        pass_hubs_clean = true;
                        break;
                    }
                }
            }
            bool pass_rounds_clean = true;
            int cnt = lcg(&C->wcnt);
            const int qtail0 = qmode ? lcg(&C->aq_tail) : 0;   // queued by the hub cycles
            if (qmode && cnt + qtail0 > 0) {
                // PushRelabel from the activation queue, without rounds: the
                // worklist entries (generation 0) are dealt to the warps by
                // stride, then each warp takes a ticket for the next queued
                // entry and waits for it; a vertex that a push turns active is
                // queued at once with the next generation and taken by the next
                // free warp, so a slow vertex holds up only the vertices it
                // activates.  The phase ends when every queued entry has been
                // processed (the warp whose completion makes the count of
                // processed entries equal to the count of queued ones raises
                // aq_fin).  Generations stand for the activation rounds: none
                // past max_rounds is queued.  One grid barrier at the end.
                const int n0 = cnt;
                for (int i = gwarp;; i += nwarps) {
                    int u = -1, gen = 0;
                    if (i < n0) {
                        u = bcast_ld(&G.wl[i]);
                    } else {
                        int q = 0;
                        unsigned long long slot = 0;
                        if (lane == 0) {
                            q = atomicAdd(&C->aq_head, 1);
                            const unsigned long long t0 = gtimer();
                            unsigned ns = 32;
                            for (int k = 0;; ++k) {
                                if (q < G.qc) {
                                    slot = ld_acquire_u64(&G.aq[q]);
                                    if (slot) {
                                        G.aq[q] = 0;   // the slot is free again for the next phase
                                        break;
                                    }
                                }
                                if ((k & 3) == 3 && ld_acquire_s32(&C->aq_fin)) break;
                                if (gtimer() - t0 > kWaitNs) {
                                    atomicOr(&C->status, ST_WAIT);
                                    break;
                                }
                                __nanosleep(ns);
                                ns = ns < 1024 ? 2 * ns : ns;
                            }
                        }
                        slot = __shfl_sync(kFull, slot, 0);
                        if (!slot) break;   // every entry processed (or a wait gave up)
                        u = (int)(slot & 0xffffffffu) - 1;
                        gen = (int)(slot >> 32);
                    }
                    const ActList AL{nullptr, nullptr, wstamp, rstamp_it, pcnt, AL0.hlist, hstamp,
                                     G.aq,    G.qc,    gen + 1, max_rounds, C};
                    if (!vertex_ok(J, C, u, n)) {
                        // skipped; still counted as processed below
                    } else if (stage == 1) {
                        const unsigned char side = G.part[u];
                        if (side == kPartS)
                            push_relabel_warp_t<true>(G, u, kc, AL, G.part, side, stg, K);
                        else
                            push_relabel_warp_t<false>(G, u, kc, AL, G.part, side, stg, K);
                    } else {
                        push_relabel_warp(G, u, kc, AL, stg, K);
                    }
                    if (lane == 0) {
                        // this entry's own enqueues, and (by the acquire) those
                        // of every entry counted before it, precede the tail read
                        const int d = arrive_acq_rel(&C->aq_done) + 1;
                        if (d == n0 + ld_acquire_s32(&C->aq_tail)) atomicExch(&C->aq_fin, 1);
                    }
                }
                MF_SYNC_T(S_T_PRW, 0, 0, cnt + lcg(&C->aq_tail));
                pass_rounds_clean = lcg(&C->aq_over) == 0;
                if (gtid == 0) {
                    ST[S_ROUNDS] += lcg(&C->aq_maxgen) + 1;
                    ST[S_WL] += cnt + lcg(&C->aq_tail);
                }
                // (the counters are zeroed for the next pass after its set-up
                // barrier, when every thread has read them)
            } else if (!qmode && (cnt > 0 || (pass == 0 && jmode == MF_MODE_TOPOLOGY))) {
                pass_rounds_clean = false;
                const int *list = G.wl;
                for (int rd = 0;; ++rd) {
                    int *nlist = (rd & 1) ? G.qb0 : G.qb1;
                    const ActList AL{&C->acnt[(rd + 1) % 3], nlist, snext++, rstamp_it, pcnt, AL0.hlist, hstamp};
                    if (gtid == 0) {
                        C->acnt[(rd + 2) % 3] = 0;
                        ST[S_ROUNDS] += 1;
                        ST[S_WL] += cnt;
                    }
                    if (jmode == MF_MODE_TOPOLOGY) {
                        // topology-driven (Sec. 5.2): every round visits every
                        // vertex id and serves the active ones, each warp 32 ids
                        // at a time (no worklist: the round lists only tell
                        // whether another round has work)
                        for (int grp = gwarp; grp * 32 < n; grp += nwarps) {
                            const int base = grp * 32;
                            const int v = base + lane;
                            bool act = false;
                            if (v < n && v != s && v != t && __ldg(&G.row[v + 1]) - __ldg(&G.row[v]) <= kHubDeg)
                                act = lcg(&G.h[v]) < n && lcg(&G.e[v]) > 0;
                            unsigned mask = __ballot_sync(kFull, act);
                            while (mask) {
                                const int j = __ffs(mask) - 1;
                                mask &= mask - 1u;
                                push_relabel_warp(G, base + j, kc, AL, stg, K);
                            }
                        }
                    } else if (stage == 1) {
                        // push-pull: push on T (h+), pull on S (h-), each side
                        // only over arcs within it
                        for (int i = gwarp; i < cnt; i += nwarps) {
                            const int u = lcg(&list[i]);
                            const unsigned char side = G.part[u];
                            if (side == kPartS)
                                push_relabel_warp_t<true>(G, u, kc, AL, G.part, side, stg, K);
                            else
                                push_relabel_warp_t<false>(G, u, kc, AL, G.part, side, stg, K);
                        }
                    } else {
                        for (int i = gwarp; i < cnt; i += nwarps)
                            push_relabel_warp(G, lcg(&list[i]), kc, AL, stg, K);
                    }
                    MF_SYNC_T(S_T_PRW, rd, 0, cnt);
                    cnt = lcg(AL.cnt);
                    list = nlist;
                    if (cnt == 0) pass_rounds_clean = true;
                    if (cnt == 0 || rd + 1 >= max_rounds || (rd + 1 >= kMaxRounds && cnt > nwarps)) break;
                }
            }
            hubs_clean = pass_hubs_clean;
            rounds_clean = pass_rounds_clean;
            pend = lcg(pcnt);   // every append to it came before the pass's last barrier
            // another pass only for a few re-activated hubs: a large set of
            // them is better served after a global relabel
            if (pend == 0 || pend > (PP ? kPassHubsPP : kPassHubs) || !pass_hubs_clean || !pass_rounds_clean)
                break;
        }

        // RemoveInvalidEdges (Alg. 3): relabelled vertices by warps,
        // relabelled hubs by items
        // (push-pull: only arcs within the vertex's part; the pull side uses
        // the h- form, Algorithm 7)
        const unsigned char *ptc = stage ? G.part : nullptr;
        const int nrl = lcg(&C->rlcnt);
        for (int i = gwarp; i < nrl; i += nwarps) {
            const int u = bcast_ld(&G.rl[i]);
            if (!vertex_ok(J, C, u, n)) continue;   // warp-uniform
            const unsigned char side = ptc ? ptc[u] : kPartT;
            if (side == kPartS)
                remove_invalid_warp_t<true>(G, u, &C->ri_moved[par], ptc, side, K);
            else
                remove_invalid_warp_t<false>(G, u, &C->ri_moved[par], ptc, side, K);
        }
        const int nri = lcg(&C->rhcnt);
        for (int w = gwarp; w < nri; w += nwarps) {
            const int2 item = lcg(&G.hri[w]);
            const int u = __shfl_sync(kFull, item.x, 0);
            if (!vertex_ok(J, C, u, n)) continue;   // warp-uniform
            const int hu = bcast_ld(&G.h[u]);
            const int a1 = min(item.y + kPrChunk, __ldg(&G.row[u + 1]));
            const unsigned char side = stage == 1 ? G.part[u] : (stage == 2 ? kPartP : kPartT);
            if (PP && side == kPartS) {
                const long long got = warp_sum(remove_invalid_range_t<true>(G, hu, item.y, a1, ptc, side, K));
                if (lane == 0 && got) {
                    add_ll(&G.e[u], got);
                    C->ri_moved[par] = 1;
                }
            } else {
                const long long moved = warp_sum(remove_invalid_range_t<false>(G, hu, item.y, a1, ptc, side, K));
                if (lane == 0 && moved) {
                    add_ll(&G.e[u], -moved);
                    C->ri_moved[par] = 1;
                }
            }
        }
        MF_SYNC_T(S_T_RI, 0, 0, nrl + nri);
        if ((it & 255) == 255) flush_counters(K, ST);

        // Alg. 4's loop test, on the heights PushRelabel left: no vertex is
        // active if every activation was served (the last round's list is
        // empty, no hub is left active or was turned active again) and
        // RemoveInvalidEdges moved nothing.  The labelling is then valid (the
        // only arcs that pushes and relabels can make steep leave relabelled
        // vertices, and RemoveInvalidEdges found none), so each vertex with
        // excess sits at height >= n and cannot reach a sink: the preflow is
        // maximum without another BFS.  The value needs the current deficits.
        const int busy = (rounds_clean ? 0 : 1) | (hubs_clean ? 0 : 2) | (lcg(&C->ri_moved[par]) ? 4 : 0) |
                         (pend > 0 ? 8 : 0);
        if (gtid == 0 && TR && C->trace_n - 1 < G.trace_cap) TR[C->trace_n - 1].mode = (short)busy;
        if (!J.exact_exit && kind != JOB_REFRESH && stage == 0 && busy == 0) {
            long long dsum = 0;
            for (long long v = gtid; v < n; v += gthreads) {
                const long long ev = lcg(&G.e[v]);
                if (v != s && v != t && ev < 0) dsum += ev;
            }
            dsum = warp_sum(dsum);
            if (lane == 0 && dsum) add_ll(&C->dacc[par ^ 1], dsum);
            MF_SYNC_T(S_T_RESET, 1, 0, 0);
            early = true;
            break;
        }
    }

    if (pp_ran) {
        // Alg. 8's result: the new cut is S' = (S minus P) plus the part of P
        // that reaches no sink of P, T' the rest; every deficient vertex ended
        // in T', so the value is e(t) plus all deficits (recounted here).
        // The heights are rewritten to encode the cut for the next repair
        // (T' below n, S' at n): exact as a cut, not as BFS distances.
        long long dsum = 0;
        for (long long v = gtid; v < n; v += gthreads) {
            const long long ev = lcg(&G.e[v]);
            if (v != s && v != t && ev < 0) dsum += ev;
            const unsigned char p = G.part[v];
            if (p == kPartT) G.h[v] = 0;
            else if (p == kPartS) G.h[v] = n;
        }
        dsum = warp_sum(dsum);
        if (lane == 0 && dsum) add_ll(&C->dacc[(it & 1) ^ 1], dsum);
        MF_SYNC_T(S_T_RESET, 3, 0, 0);
    }

    // ---- debug_checks: the state's invariants over all arcs ----------------
    // e(v) = sum over v's arcs of (r - cap) (the incremental excess updates
    // of the repair equal the full recount of Alg. 4 line 2), r >= 0, the
    // residuals of an arc pair add up to the pair's capacities, and the
    // mirror rr(a) = r(rev a).  One warp per vertex.
    if (J.debug) {
        for (int v = gwarp; v < n; v += nwarps) {
            const int a0 = __ldg(&G.row[v]), a1 = __ldg(&G.row[v + 1]);
            long long in = 0;
            bool bad = false;
            for (int a = a0 + lane; a < a1; a += 32) {
                const int b = __ldg(&G.rev[a]);
                const int ra = lcg(&G.r[a]), rb = lcg(&G.r[b]);
                in += (long long)ra - lcg(&G.cap[a]);
                if (ra < 0 || (long long)ra + rb != (long long)lcg(&G.cap[a]) + lcg(&G.cap[b]) ||
                    lcg(&G.rr[a]) != rb) {
                    if (!bad) check_fail(C, 3, a);
                    bad = true;
                }
            }
            in = warp_sum(in);
            if (lane == 0 && in != lcg(&G.e[v])) check_fail(C, 2, v);
        }
    }

    // ---- result and statistics -------------------------------------------
    if (gtid == 0) {
        // dacc: deficits at the last height init, or recounted at a clean
        // exit and after a push-pull repair
        if (!fast) C->flow = lcg(&G.e[t]) + lcg(&C->dacc[(early || pp_ran) ? (it & 1) ^ 1 : it & 1]);
        if (kind != JOB_REFRESH) {
            C->iters = fast ? 0 : early ? it + 1 : it;
            C->exit_kind = fast ? EXIT_NO_CUT_CHANGE : early ? EXIT_CLEAN : pp_ran ? EXIT_PUSH_PULL : EXIT_BFS;
        }
        C->heights_exact = !fast && !early && !pp_ran;
        C->cut_exact = !early;   // the fast path keeps the exact cut it started from
        C->ri_moved[0] = C->ri_moved[1] = 0;
        C->phc[0] = C->phc[1] = 0;
        C->rhcnt = 0;
        C->inc_block = 0;
        for (int i = 0; i < 3; ++i) {
            C->qcnt[i] = C->ccnt[i] = 0;
            C->asum[i] = 0;
        }
        C->wcnt = C->hcnt = C->hccnt = C->rlcnt = 0;
        C->acnt[0] = C->acnt[1] = C->acnt[2] = 0;
        C->stamp_base = snext;
        if (batch_job) C->bseq = seq;
        C->hub_act[0] = C->hub_act[1] = 0;
        C->hlc[0] = C->hlc[1] = 0;
        C->dacc[0] = C->dacc[1] = 0;
        C->batch_err = 0;
        C->abort_loop = 0;
    }
    flush_counters_cta(K, ST);
}

#undef ST
#undef TR

// ------------------------------------------------------------- policy --
static_assert(MF_MODE_DATA_DRIVEN == 0 && MF_MODE_TOPOLOGY == 1 && MF_MODE_PUSH_PULL == 2,
              "the network's mode outputs 2, 3, 4 are the modes in this order");

struct PolicyJob {
    int k, flags, mode, kc_plain, max_deg;
    int gmode;             // the graph's own processing mode (MF_MODE_*)
    int pp_ok;             // the graph can repair by Dynamic Push-Pull
    const int *k_dev;      // if set, the batch size is read from device memory
    const int *ids, *caps;
    const float *params;   // network parameters (mf_mlp.cuh), or null
};

// Features of a batch and the policy decision for the k_solve launch that
// follows (JOB_AUTO).  CTAs of 256 threads stride over the batch entries and
// add their integer sums (exact, so the result does not depend on the order)
// to the control block; the last CTA to arrive computes the 12 features,
// then the plain rule (dynamic repair when the batch holds at most 1 % of
// the edges, KERNELCYCLES = average degree) or the network, with the plain
// rule as fallback on any non-finite or out-of-range input (|z| > 8), and
// clears the sums for the next launch.  Entries with bad ids are skipped
// here; k_solve rejects the batch.
// Four 256-thread CTAs per CTA of the repair's grid: a 100k-entry batch is
// then one entry per thread, its chain of dependent gathers (edge, arc,
// reverse arc, heads) walked once instead of three times in a row.
constexpr int kPolicyCtasPerSlot = 4;
__global__ void __launch_bounds__(256) k_policy(DevGraph G, PolicyJob PJ) {
    Ctl *C = G.ctl;
    if (PJ.k_dev) PJ.k = lcg(PJ.k_dev);
    __shared__ long long red[3][8];
    __shared__ float x[mlp::kIn], z[mlp::kIn], h1[mlp::kH1], h2[mlp::kH2], y[mlp::kOut];
    __shared__ int fb, last;
    long long inc = 0, touch = 0, sumd = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < PJ.k;
         i += (long long)gridDim.x * blockDim.x) {
        const int id = PJ.ids[i];
        if (id < 0 || id >= G.m) continue;
        const long long old = lcg(&G.cap_edge[id]);
        long long nc = PJ.caps[i];
        if (PJ.flags & MF_DELTA) nc = old + nc < 0 ? 0 : old + nc;
        inc += nc > old;
        sumd += nc > old ? nc - old : old - nc;
        if (G.edge_st) {
            touch += __ldg(&G.edge_st[id]);
        } else {
            const int a = __ldg(&G.arc_of_edge[id]);
            if (a >= 0 && (__ldg(&G.head[a]) == G.t || __ldg(&G.head[__ldg(&G.rev[a])]) == G.s)) ++touch;
        }
    }
    inc = warp_sum(inc);
    touch = warp_sum(touch);
    sumd = warp_sum(sumd);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = inc;
        red[1][threadIdx.x >> 5] = touch;
        red[2][threadIdx.x >> 5] = sumd;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < 3; ++q) {
            long long v = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[q][w];
            if (v) add_ll(&C->pol_acc[q], v);
        }
        __threadfence();
        last = atomicAdd(&C->pol_done, 1) == (int)gridDim.x - 1;
        if (last) {
            __threadfence();
            for (int q = 0; q < 3; ++q) {
                red[q][0] = __ldcg(&C->pol_acc[q]);
                C->pol_acc[q] = 0;
            }
            C->pol_done = 0;
        }
    }
    __syncthreads();
    if (!last) return;
    if (threadIdx.x == 0) {
        const float n = (float)G.n, m = (float)(G.m > 0 ? G.m : 1), k = (float)PJ.k;
        const float kk = k > 0.f ? k : 1.f;
        const long long iters = lcg(&C->iters);
        const long long reached = lcg(&C->st[S_BFS_VERTS]);
        x[0] = log2f(n);
        x[1] = log2f(m);
        x[2] = log2f(1.f + k);
        x[3] = k / m;
        x[4] = (float)red[0][0] / kk;
        x[5] = (float)red[1][0] / kk;
        x[6] = log2f(1.f + (float)red[2][0]);
        const long long fl = lcg(&C->flow);
        x[7] = log2f(1.f + (float)(fl < 0 ? -fl : fl));
        x[8] = (float)G.A / n;
        x[9] = log2f(1.f + (float)PJ.max_deg);
        x[10] = (float)iters;
        x[11] = (float)reached / ((float)(iters + 1) * n);
        for (int j = 0; j < mlp::kIn; ++j) C->feat[j] = x[j];
        fb = PJ.mode != MF_POLICY_LEARNED || PJ.params == nullptr;
        if (!fb)
            for (int j = 0; j < mlp::kIn; ++j) {
                z[j] = (x[j] - PJ.params[mlp::oMu + j]) / PJ.params[mlp::oSd + j];
                if (!isfinite(z[j]) || fabsf(z[j]) > 8.f) fb = 1;
            }
    }
    __syncthreads();
    if (!fb) {
        const float *P = PJ.params;
        if (threadIdx.x < mlp::kH1) {
            float a = P[mlp::oB1 + threadIdx.x];
            for (int j = 0; j < mlp::kIn; ++j) a += P[mlp::oW1 + threadIdx.x * mlp::kIn + j] * z[j];
            h1[threadIdx.x] = a > 0.f ? a : 0.f;
        }
        __syncthreads();
        if (threadIdx.x < mlp::kH2) {
            float a = P[mlp::oB2 + threadIdx.x];
            for (int j = 0; j < mlp::kH1; ++j) a += P[mlp::oW2 + threadIdx.x * mlp::kH1 + j] * h1[j];
            h2[threadIdx.x] = a > 0.f ? a : 0.f;
        }
        __syncthreads();
        if (threadIdx.x < mlp::kOut) {
            float a = P[mlp::oB3 + threadIdx.x];
            for (int j = 0; j < mlp::kH2; ++j) a += P[mlp::oW3 + threadIdx.x * mlp::kH2 + j] * h2[j];
            y[threadIdx.x] = a;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int kind, kc, mode = PJ.gmode;
        bool fallback = fb != 0;
        for (int o = 0; o < mlp::kOut && !fallback; ++o)
            if (!isfinite(y[o])) fallback = true;
        if (fallback) {
            kind = (long long)PJ.k * 100 <= (long long)G.m ? JOB_REPAIR : JOB_RECOMPUTE;
            kc = PJ.kc_plain;
        } else {
            kind = y[0] > 0.f ? JOB_REPAIR : JOB_RECOMPUTE;
            const float l = fminf(fmaxf(rintf(y[1]), 0.f), 6.f);
            kc = 1 << (int)l;
            // the mode of the largest logit (outputs 2, 3, 4: data-driven,
            // topology-driven, push-pull); push-pull only where the graph
            // keeps the exact cut it needs, else the better of the other two
            int best = 0;
            for (int c = 1; c < mlp::kModes; ++c)
                if (y[2 + c] > y[2 + best]) best = c;
            if (best == MF_MODE_PUSH_PULL && !PJ.pp_ok) best = y[3] > y[2] ? MF_MODE_TOPOLOGY : MF_MODE_DATA_DRIVEN;
            mode = best;
        }
        C->pol_kind = kind;
        C->pol_kc = kc;
        C->pol_mode = mode;
        C->pol_fallback = (PJ.mode == MF_POLICY_LEARNED && fallback) ? 1 : 0;
    }
}

__global__ void k_cut_side(const int *h, int n, unsigned char *side) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
        side[v] = h[v] >= n ? 1 : 0;
}

// ---------------------------------------------- allocation-free solve --
// Scratch of mf_solve_bicsr_noalloc: one static device array per GPU that
// loads this library, used instead of device allocations for everything the
// solve kernel needs besides the caller's graph and output arrays.  Sized for
// graphs of at most kNoAllocMaxN vertices and kNoAllocMaxArcs Bi-CSR arcs.
constexpr int kNoAllocMaxN = 1 << 17;
constexpr long long kNoAllocMaxArcs = 1LL << 21;
constexpr int kNoAllocMaxGrid = 1024;
constexpr long long kNoAllocMaxHubs = kNoAllocMaxArcs / kHubDeg;

__host__ __device__ constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Byte offsets of the scratch regions (each 256-byte aligned).
struct NoAllocLayout {
    static constexpr size_t ctl = 0;
    static constexpr size_t rr = ctl + align256(sizeof(Ctl));
    static constexpr size_t qb0 = rr + align256(sizeof(int) * kNoAllocMaxArcs);
    static constexpr size_t qb1 = qb0 + align256(sizeof(int) * kNoAllocMaxN);
    static constexpr size_t wl = qb1 + align256(sizeof(int) * kNoAllocMaxN);
    static constexpr size_t rl = wl + align256(sizeof(int) * kNoAllocMaxN);
    static constexpr size_t astamp = rl + align256(sizeof(int) * kNoAllocMaxN);
    static constexpr size_t rstamp = astamp + align256(sizeof(unsigned) * kNoAllocMaxN);
    static constexpr size_t cb = rstamp + align256(sizeof(unsigned) * kNoAllocMaxN);
    static constexpr size_t hcl = cb + align256(sizeof(int2) * (kNoAllocMaxArcs / kChunk + kNoAllocMaxN));
    static constexpr size_t hlv0 = hcl + align256(sizeof(int2) * (kNoAllocMaxArcs / kPrChunk + kNoAllocMaxHubs));
    static constexpr size_t hlv1 = hlv0 + align256(sizeof(int2) * (kNoAllocMaxArcs / kPrChunk + kNoAllocMaxHubs));
    static constexpr size_t hikey = hlv1 + align256(sizeof(int2) * (kNoAllocMaxArcs / kPrChunk + kNoAllocMaxHubs));
    static constexpr size_t hl = hikey + align256(sizeof(unsigned) * (kNoAllocMaxArcs / kPrChunk + kNoAllocMaxHubs));
    static constexpr size_t hmode = hl + align256(sizeof(int) * kNoAllocMaxHubs);
    static constexpr size_t hnit = hmode + align256(sizeof(int) * kNoAllocMaxHubs);
    static constexpr size_t hdone = hnit + align256(sizeof(int) * kNoAllocMaxHubs);
    static constexpr size_t hkey = hdone + align256(sizeof(int) * kNoAllocMaxHubs);
    static constexpr size_t hrem = hkey + align256(sizeof(unsigned long long) * kNoAllocMaxHubs);
    static constexpr size_t hl2 = hrem + align256(sizeof(long long) * kNoAllocMaxHubs);
    static constexpr size_t hri = hl2 + align256(sizeof(int) * kNoAllocMaxHubs);
    static constexpr size_t aq = hri + align256(sizeof(int2) * (kNoAllocMaxArcs / kPrChunk + kNoAllocMaxHubs));
    static constexpr size_t total = aq + align256(sizeof(unsigned long long) * kNoAllocMaxN);
};

static_assert(NoAllocLayout::total == 14288384, "the header states the scratch size (14,288,384 bytes)");
static __device__ __align__(256) unsigned char g_noalloc_scratch[NoAllocLayout::total];

}  // namespace mf

// =============================================================== C ABI ====
using namespace mf;

struct mf_graph {
    int dev = 0;
    int32_t n = 0, s = 0, t = 0;
    int64_t m = 0, A = 0;
    int32_t cap_limit = 0;
    int kc = 1;
    long long max_iters = 0;
    unsigned long long time_limit_ns = 0;
    int grid = 0, sms = 0;
    int max_grid = 0;   // one full wave of co-resident CTAs
    mf_options opt{};
    DevGraph dg{};
    std::vector<void *> owned;
    std::vector<size_t> owned_bytes;
    int *b_ids = nullptr, *b_caps = nullptr, *b_newc = nullptr, *b_dlt = nullptr;
    int64_t b_cap = 0;
    unsigned char *side_buf = nullptr;
    bool solved = false;
    int policy = MF_POLICY_FIXED;
    float *params = nullptr;   // policy network parameters on the device
    int max_deg = 0;
    cudaStream_t last = nullptr;
};

namespace {

thread_local std::string g_last_error;

// Per-device set-up of the allocation-free solve.
constexpr int kNoAllocMaxDevices = 64;
struct NoAllocDevice {
    unsigned char *base = nullptr;   // device address of g_noalloc_scratch
    int grid = 0;
    cudaError_t err = cudaSuccess;
};
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];
std::once_flag g_noalloc_once[kNoAllocMaxDevices];

int set_err(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

// k_solve takes kDynSmem bytes of dynamic shared memory (above the default
// 48 KB limit): both instances get the attribute once per device, before
// their first occupancy query or launch on it.
std::once_flag g_smem_once[kNoAllocMaxDevices];
cudaError_t g_smem_err[kNoAllocMaxDevices];

cudaError_t solve_kernels_prepare(int dev) {
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(g_smem_once[dev], [dev]() {
        cudaError_t e = cudaFuncSetAttribute(k_solve<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_solve<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmem);
        g_smem_err[dev] = e;
    });
    return g_smem_err[dev];
}

#define MF_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return set_err(MF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    } while (0)

void *dalloc(mf_graph *g, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (g->opt.alloc) {
        p = g->opt.alloc(bytes, g->opt.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void dfree(mf_graph *g, void *p) {
    if (!p) return;
    if (g->opt.free) g->opt.free(p, g->opt.alloc_ctx);
    else cudaFree(p);
}

template <class T>
T *dnew(mf_graph *g, size_t count) {
    T *p = static_cast<T *>(dalloc(g, count * sizeof(T)));
    if (p) {
        g->owned.push_back(p);
        g->owned_bytes.push_back(count * sizeof(T));
    }
    return p;
}

void dforget(mf_graph *g, void *p) {
    for (size_t i = 0; i < g->owned.size(); ++i)
        if (g->owned[i] == p) {
            g->owned.erase(g->owned.begin() + long(i));
            g->owned_bytes.erase(g->owned_bytes.begin() + long(i));
            return;
        }
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice;
}

template <class T>
int host_copy(const T *src, size_t count, std::vector<T> &dst, const T **out) {
    if (is_device_ptr(src)) {
        dst.resize(count);
        if (count) MF_CUDA(cudaMemcpy(dst.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost));
        *out = dst.data();
    } else {
        *out = src;
    }
    return MF_OK;
}

int read_ctl(mf_graph *g, Ctl *out, size_t bytes = sizeof(Ctl)) {
    MF_CUDA(cudaSetDevice(g->dev));
    MF_CUDA(cudaMemcpyAsync(out, g->dg.ctl, bytes, cudaMemcpyDeviceToHost, g->last));
    MF_CUDA(cudaStreamSynchronize(g->last));
    return MF_OK;
}

int launch(mf_graph *g, const Job &job, cudaStream_t st) {
    DevGraph dg = g->dg;
    Job jb = job;
    jb.st = job.kind == JOB_REFRESH ? g->dg.ctl->st_aux : g->dg.ctl->st;
    jb.debug = g->opt.debug_checks != 0;
    jb.trace = job.kind == JOB_REFRESH ? nullptr : g->dg.trace;
    void *args[] = {&dg, &jb};
    // a push-pull graph keeps its cut exact (every job ends on a BFS) and
    // solves from zero flow by static push-pull
    if (g->opt.mode == MF_MODE_PUSH_PULL) {
        jb.exact_exit = 1;
        jb.sink_sat = 1;
    }
    const void *fn = job.pp ? (const void *)k_solve<true> : (const void *)k_solve<false>;
    cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(g->grid), dim3(kBlock), args, kDynSmem, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(MF_ECUDA, std::string("cooperative launch: ") + cudaGetErrorString(e));
    }
    g->last = st;
    return MF_OK;
}

int launch_policy(mf_graph *g, int64_t k, const int *ids, const int *caps, int flags, cudaStream_t st) {
    PolicyJob pj{};
    pj.k = int(k);
    pj.flags = flags;
    pj.mode = g->policy;
    pj.kc_plain = g->kc;
    pj.max_deg = g->max_deg;
    pj.ids = ids;
    pj.caps = caps;
    pj.params = g->params;
    pj.gmode = g->opt.mode;
    pj.pp_ok = g->opt.mode == MF_MODE_PUSH_PULL;
    cudaGetLastError();   // an earlier, unrelated failure of this thread is not this launch's
    k_policy<<<kPolicyCtasPerSlot * g->grid, 256, 0, st>>>(g->dg, pj);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(MF_ECUDA, std::string("policy launch: ") + cudaGetErrorString(e));
    return MF_OK;
}

int ensure_batch_capacity(mf_graph *g, int64_t k, cudaStream_t st) {
    if (k <= g->b_cap) return MF_OK;
    int64_t want = std::max<int64_t>(k, std::max<int64_t>(1024, g->b_cap * 2));
    MF_CUDA(cudaStreamSynchronize(st));
    if (g->last && g->last != st) MF_CUDA(cudaStreamSynchronize(g->last));
    int *ptrs[4] = {g->b_ids, g->b_caps, g->b_newc, g->b_dlt};
    for (int *p : ptrs) {
        if (!p) continue;
        dfree(g, p);
        dforget(g, p);
    }
    g->b_ids = dnew<int>(g, size_t(want));
    g->b_caps = dnew<int>(g, size_t(want));
    g->b_newc = dnew<int>(g, size_t(want));
    g->b_dlt = dnew<int>(g, size_t(want));
    if (!g->b_ids || !g->b_caps || !g->b_newc || !g->b_dlt) {
        g->b_cap = 0;
        return set_err(MF_ENOMEM, "batch staging allocation failed");
    }
    g->b_cap = want;
    return MF_OK;
}

// Make h the exact BFS heights of the current state (a no-op on the device
// when they are exact already), on the graph's last stream.
int refresh_heights(mf_graph *g) {
    Job j{};
    j.kind = JOB_REFRESH;
    j.exact_exit = 1;
    j.kc = g->kc;
    j.mode = g->opt.mode;
    j.max_iters = g->max_iters;
    j.time_limit_ns = g->time_limit_ns;
    return launch(g, j, g->last);
}

int status_to_code(mf_graph *g, const Ctl &c) {
    if (c.status & ST_CHECK) {
        g->solved = false;
        static const char *kinds[] = {"?", "list entry out of range", "excess differs from the net inflow",
                                      "residual pair or mirror inconsistent"};
        const long long kind = c.chk_where >> 40, where = c.chk_where & 0xffffffffffll;
        return set_err(MF_ECHECK, std::string("debug check failed: ") + kinds[kind >= 1 && kind <= 3 ? kind : 0] +
                                      " (index " + std::to_string(where) + ")");
    }
    if (c.status & ST_STICKY) {
        g->solved = false;
        return set_err(MF_ETIMEOUT, (c.status & ST_WAIT)   ? "device wait reached its time limit"
                                    : (c.status & ST_TIME) ? "device loop reached its wall-clock limit"
                                                           : "device loop reached max_iters");
    }
    if (c.status & ST_EINVAL) {
        int zero = c.status & ~ST_EINVAL;
        MF_CUDA(cudaMemcpyAsync(&g->dg.ctl->status, &zero, sizeof(int), cudaMemcpyHostToDevice, g->last));
        MF_CUDA(cudaStreamSynchronize(g->last));
        return set_err(MF_EINVAL, "batch rejected on the device (edge id out of range, duplicate id or capacity out of range)");
    }
    return MF_OK;
}

}  // namespace

extern "C" {

const char *mf_version(void) { return "0.1.0"; }

const char *mf_strerror(int code) {
    switch (code) {
        case MF_OK: return "ok";
        case MF_EINVAL: return "invalid argument";
        case MF_ENOMEM: return "out of memory";
        case MF_ECUDA: return "CUDA error";
        case MF_ENOTSOLVED: return "graph not solved";
        case MF_ETIMEOUT: return "device loop timeout";
        case MF_ECHECK: return "device consistency check failed";
        default: return "unknown error";
    }
}

const char *mf_last_error(void) { return g_last_error.c_str(); }

int mf_options_default(mf_options *opt) {
    if (!opt) return MF_EINVAL;
    std::memset(opt, 0, sizeof(*opt));
    opt->mode = MF_MODE_DATA_DRIVEN;
    return MF_OK;
}

int mf_bicsr_host(int32_t n, int64_t m, const int64_t *row_ptr, const int32_t *col, const int32_t *cap,
                  int32_t s, int32_t t, int64_t *arcs, int64_t *arc_row, int32_t *head, int32_t *rev,
                  int32_t *arc_cap, int32_t *arc_of_edge, int32_t *cap_limit) {
    if (!row_ptr || (m > 0 && (!col || !cap)) || !arcs) return set_err(MF_EINVAL, "null argument");
    HostBiCSR G;
    int rc = build_bicsr(n, m, row_ptr, col, cap, s, t, &G);
    if (rc) return set_err(rc == 2 ? MF_ENOMEM : MF_EINVAL, "graph rejected by the Bi-CSR builder");
    *arcs = G.arcs;
    if (arc_row) for (int32_t u = 0; u <= n; ++u) arc_row[u] = G.row[size_t(u)];
    if (head) std::copy(G.head.begin(), G.head.end(), head);
    if (rev) std::copy(G.rev.begin(), G.rev.end(), rev);
    if (arc_cap) std::copy(G.cap.begin(), G.cap.end(), arc_cap);
    if (arc_of_edge) std::copy(G.arc_of_edge.begin(), G.arc_of_edge.end(), arc_of_edge);
    if (cap_limit) *cap_limit = G.cap_limit;
    return MF_OK;
}

int mf_create(int32_t n, int64_t m, const int64_t *row_ptr, const int32_t *col, const int32_t *cap,
              int32_t s, int32_t t, const mf_options *opt, void *stream, mf_graph **out) {
    if (!out || !row_ptr || (m > 0 && (!col || !cap))) return set_err(MF_EINVAL, "null argument");
    *out = nullptr;
    if (n < 2 || m < 0 || m >= INT32_MAX || s < 0 || t < 0 || s >= n || t >= n || s == t)
        return set_err(MF_EINVAL, "bad sizes or terminals");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<int64_t> hrow;
    std::vector<int32_t> hcol, hcap;
    const int64_t *prow;
    const int32_t *pcol = col, *pcap = cap;
    int rc = host_copy(row_ptr, size_t(n) + 1, hrow, &prow);
    if (rc) return rc;
    if (m > 0) {
        if ((rc = host_copy(col, size_t(m), hcol, &pcol))) return rc;
        if ((rc = host_copy(cap, size_t(m), hcap, &pcap))) return rc;
    }
    HostBiCSR H;
    rc = build_bicsr(n, m, prow, pcol, pcap, s, t, &H);
    if (rc) return set_err(rc == 2 ? MF_ENOMEM : MF_EINVAL, "graph rejected by the Bi-CSR builder");

    mf_graph *g = new (std::nothrow) mf_graph();
    if (!g) return set_err(MF_ENOMEM, "host allocation");
    if (opt) g->opt = *opt;
    else mf_options_default(&g->opt);
    auto fail = [&](int code, const std::string &msg) {
        mf_destroy(g);
        return set_err(code, msg);
    };
    if ((g->opt.alloc == nullptr) != (g->opt.free == nullptr)) return fail(MF_EINVAL, "alloc and free must both be set");
    if (g->opt.mode != MF_MODE_DATA_DRIVEN && g->opt.mode != MF_MODE_TOPOLOGY && g->opt.mode != MF_MODE_PUSH_PULL)
        return fail(MF_EINVAL, "unknown mode");
    if (cudaGetDevice(&g->dev) != cudaSuccess) return fail(MF_ECUDA, "no CUDA device");
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, g->dev);
    cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->dev);
    if (!coop) return fail(MF_ECUDA, "device does not support cooperative launch");
    int per_sm = 0;
    int per_sm_pp = 0;
    if (solve_kernels_prepare(g->dev) != cudaSuccess) return fail(MF_ECUDA, "shared-memory attribute of k_solve");
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve<false>, kBlock, kDynSmem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_pp, k_solve<true>, kBlock, kDynSmem) != cudaSuccess)
        return fail(MF_ECUDA, "occupancy query failed");
    per_sm = std::min(per_sm, per_sm_pp);
    if (per_sm < 1)
        return fail(MF_ECUDA, "occupancy query failed");
    g->grid = per_sm * g->sms;
    g->max_grid = g->grid;
    if (g->opt.grid_blocks > 0) g->grid = std::min(g->grid, int(g->opt.grid_blocks));

    g->n = n; g->m = m; g->A = H.arcs; g->s = s; g->t = t;
    g->cap_limit = H.cap_limit;
    g->max_deg = H.max_deg;
    int64_t avg = (m + n / 2) / n;
    g->kc = g->opt.kernel_cycles > 0 ? g->opt.kernel_cycles : int(std::max<int64_t>(1, avg));
    g->max_iters = g->opt.max_iters > 0 ? g->opt.max_iters : 4LL * n + 1000;
    g->time_limit_ns = 1000000ull * (unsigned long long)(g->opt.time_limit_ms > 0 ? g->opt.time_limit_ms : 60000);

    const size_t A = size_t(std::max<int64_t>(H.arcs, 1)), N = size_t(n), M = size_t(std::max<int64_t>(m, 1));
    DevGraph &D = g->dg;
    D.n = n; D.s = s; D.t = t; D.m = int(m); D.A = H.arcs; D.cap_limit = H.cap_limit;
    int *row = dnew<int>(g, N + 1), *head = dnew<int>(g, A), *rev = dnew<int>(g, A), *aoe = dnew<int>(g, M);
    D.row = row; D.head = head; D.rev = rev; D.arc_of_edge = aoe;
    unsigned char *est = dnew<unsigned char>(g, M);
    D.edge_st = est;
    D.cap = dnew<int>(g, A); D.r = dnew<int>(g, A); D.rr = dnew<int>(g, A);
    D.h = dnew<int>(g, N); D.e = dnew<long long>(g, N);
    D.cap_edge = dnew<int>(g, M); D.stamp = dnew<unsigned>(g, M);
    D.qb0 = dnew<int>(g, N); D.qb1 = dnew<int>(g, N); D.wl = dnew<int>(g, N);
    D.cb = dnew<int2>(g, size_t(std::max<int64_t>(H.chunk_items, 1)));
    const size_t NH = size_t(std::max<int64_t>(H.hubs, 1));
    D.hl = dnew<int>(g, NH);
    D.hl2 = dnew<int>(g, NH);
    D.hmode = dnew<int>(g, NH);
    D.hkey = dnew<unsigned long long>(g, NH);
    D.hrem = dnew<long long>(g, NH);
    D.hnit = dnew<int>(g, NH);
    D.hdone = dnew<int>(g, NH);
    D.hcl = dnew<int2>(g, size_t(std::max<int64_t>(H.hub_chunk_items, 1)));
    D.hlv0 = dnew<int2>(g, size_t(std::max<int64_t>(H.hub_chunk_items, 1)));
    D.hlv1 = dnew<int2>(g, size_t(std::max<int64_t>(H.hub_chunk_items, 1)));
    D.hikey = dnew<unsigned>(g, size_t(std::max<int64_t>(H.hub_chunk_items, 1)));
    D.hri = dnew<int2>(g, size_t(std::max<int64_t>(H.hub_chunk_items, 1)));
    D.astamp = dnew<unsigned>(g, N);
    D.rstamp = dnew<unsigned>(g, N);
    D.rl = dnew<int>(g, N);
    D.part = g->opt.mode == MF_MODE_PUSH_PULL ? dnew<unsigned char>(g, N) : nullptr;
    D.qc = int(std::max<size_t>(N, 1024));
    D.aq = dnew<unsigned long long>(g, size_t(D.qc));
    D.ctl = dnew<Ctl>(g, 1);
    g->side_buf = dnew<unsigned char>(g, N);
    // an allocator callback may hand out blocks without 16-byte alignment:
    // the staging copies then fall back to plain loads
    auto al16 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    D.al16 = al16(D.head) && al16(D.r) && al16(D.rr);
    if (!row || !head || !rev || !aoe || !est || !D.cap || !D.r || !D.rr || !D.h || !D.e || !D.cap_edge || !D.stamp ||
        !D.qb0 || !D.qb1 || !D.wl || !D.cb || !D.ctl || !g->side_buf || !D.hl || !D.hmode || !D.hkey ||
        !D.hrem || !D.hnit || !D.hdone || !D.hcl || !D.hlv0 || !D.hlv1 || !D.hikey || !D.hl2 || !D.hri || !D.astamp ||
        !D.rstamp || !D.rl || !D.aq)
        return fail(MF_ENOMEM, "device allocation failed");
    auto up = [&](void *dst, const void *src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
    };
    std::vector<int32_t> cap_edge(pcap, pcap + m);
    // the policy's "edges out of s or into t" feature, one byte per edge (0
    // for a self-loop, which has no arc)
    std::vector<unsigned char> edge_st(size_t(std::max<int64_t>(m, 1)), 0);
    for (int32_t u = 0; u < n; ++u)
        for (int64_t i = prow[u]; i < prow[u + 1]; ++i)
            edge_st[size_t(i)] = pcol[i] != u && (u == s || pcol[i] == t);
    if (up(row, H.row.data(), (N + 1) * 4) || up(head, H.head.data(), size_t(H.arcs) * 4) ||
        up(rev, H.rev.data(), size_t(H.arcs) * 4) || up(aoe, H.arc_of_edge.data(), size_t(m) * 4) ||
        up(est, edge_st.data(), size_t(m)) ||
        up(D.cap, H.cap.data(), size_t(H.arcs) * 4) || up(D.cap_edge, cap_edge.data(), size_t(m) * 4) ||
        cudaMemsetAsync(D.stamp, 0, M * 4, st) || cudaMemsetAsync(D.ctl, 0, sizeof(Ctl), st) ||
        cudaMemsetAsync(D.aq, 0, size_t(D.qc) * 8, st) ||
        cudaMemsetAsync(D.e, 0, N * 8, st) || cudaMemsetAsync(D.h, 0, N * 4, st) ||
        cudaMemsetAsync(D.astamp, 0, N * 4, st) || cudaMemsetAsync(D.rstamp, 0, N * 4, st) ||
        cudaMemsetAsync(D.r, 0, A * 4, st) || cudaMemsetAsync(D.rr, 0, A * 4, st) ||
        cudaStreamSynchronize(st)) {
        cudaGetLastError();
        return fail(MF_ECUDA, "upload failed");
    }
    g->last = st;
    *out = g;
    return MF_OK;
}

int mf_cap_limit(const mf_graph *g, int32_t *out) {
    if (!g || !out) return MF_EINVAL;
    *out = g->cap_limit;
    return MF_OK;
}

int mf_sizes(const mf_graph *g, int32_t *n, int64_t *m, int64_t *arcs) {
    if (!g) return MF_EINVAL;
    if (n) *n = g->n;
    if (m) *m = g->m;
    if (arcs) *arcs = g->A;
    return MF_OK;
}

int mf_solve(mf_graph *g, void *stream) {
    if (!g) return MF_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MF_CUDA(cudaSetDevice(g->dev));
    MF_CUDA(cudaMemsetAsync(g->dg.ctl, 0, sizeof(Ctl), st));
    MF_CUDA(cudaMemsetAsync(g->dg.stamp, 0, size_t(std::max<int64_t>(g->m, 1)) * 4, st));
    MF_CUDA(cudaMemsetAsync(g->dg.astamp, 0, size_t(g->n) * 4, st));
    MF_CUDA(cudaMemsetAsync(g->dg.rstamp, 0, size_t(g->n) * 4, st));
    // a launch that gave up inside a PushRelabel phase may have left queue entries
    MF_CUDA(cudaMemsetAsync(g->dg.aq, 0, size_t(g->dg.qc) * 8, st));
    Job j{};
    j.kind = JOB_SOLVE;
    j.kc = g->kc;
    j.mode = g->opt.mode;
    j.max_iters = g->max_iters;
    j.time_limit_ns = g->time_limit_ns;
    int rc = launch(g, j, st);
    if (rc == MF_OK) g->solved = true;
    return rc;
}

int mf_apply_updates(mf_graph *g, int64_t k, const int32_t *edge_id, const int32_t *new_cap, int32_t flags,
                     void *stream) {
    if (!g) return MF_EINVAL;
    if (!g->solved) return set_err(MF_ENOTSOLVED, "call mf_solve first");
    if (k < 0 || k > g->m || (k > 0 && (!edge_id || !new_cap)))
        return set_err(MF_EINVAL, "bad batch size or null batch pointer");
    if (flags & ~(MF_DEVICE_PTRS | MF_DELTA | MF_RECOMPUTE)) return set_err(MF_EINVAL, "unknown flags");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MF_CUDA(cudaSetDevice(g->dev));
    int rc = ensure_batch_capacity(g, std::max<int64_t>(k, 1), st);
    if (rc) return rc;
    const int *ids = edge_id, *caps = new_cap;
    if (!(flags & MF_DEVICE_PTRS) && k > 0) {
        MF_CUDA(cudaMemcpyAsync(g->b_ids, edge_id, size_t(k) * 4, cudaMemcpyHostToDevice, st));
        MF_CUDA(cudaMemcpyAsync(g->b_caps, new_cap, size_t(k) * 4, cudaMemcpyHostToDevice, st));
        ids = g->b_ids;
        caps = g->b_caps;
    }
    Job j{};
    j.kind = (flags & MF_RECOMPUTE) ? JOB_RECOMPUTE : JOB_REPAIR;
    if (!(flags & MF_RECOMPUTE) && g->policy != MF_POLICY_FIXED) {
        rc = launch_policy(g, k, ids, caps, flags, st);
        if (rc) return rc;
        j.kind = JOB_AUTO;
    }
    j.k = int(k);
    j.flags = flags;
    j.kc = g->kc;
    j.mode = g->opt.mode;
    j.pp = g->opt.mode == MF_MODE_PUSH_PULL;
    j.max_iters = g->max_iters;
    j.time_limit_ns = g->time_limit_ns;
    j.ids = ids;
    j.caps = caps;
    j.newc = g->b_newc;
    j.dlt = g->b_dlt;
    return launch(g, j, st);
}

int mf_apply_updates_dev(mf_graph *g, const int32_t *k_dev, int64_t k_max, const int32_t *edge_id,
                         const int32_t *new_cap, int32_t flags, void *stream) {
    if (!g || !k_dev || !edge_id || !new_cap) return set_err(MF_EINVAL, "null argument");
    if (!g->solved) return set_err(MF_ENOTSOLVED, "call mf_solve first");
    if (k_max < 0 || k_max > g->m) return set_err(MF_EINVAL, "bad k_max");
    if (flags & ~(MF_DELTA | MF_RECOMPUTE | MF_DEVICE_PTRS)) return set_err(MF_EINVAL, "unknown flags");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MF_CUDA(cudaSetDevice(g->dev));
    if (g->b_cap < std::max<int64_t>(k_max, 1)) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        MF_CUDA(cudaStreamIsCapturing(st, &cs));
        if (cs != cudaStreamCaptureStatusNone)
            return set_err(MF_EINVAL, "batch staging must be sized (k_max) before stream capture");
        int rc = ensure_batch_capacity(g, std::max<int64_t>(k_max, 1), st);
        if (rc) return rc;
    }
    Job j{};
    j.kind = (flags & MF_RECOMPUTE) ? JOB_RECOMPUTE : JOB_REPAIR;
    if (!(flags & MF_RECOMPUTE) && g->policy != MF_POLICY_FIXED) {
        PolicyJob pj{};
        pj.k = 0;
        pj.k_dev = k_dev;
        pj.flags = flags & MF_DELTA;
        pj.mode = g->policy;
        pj.kc_plain = g->kc;
        pj.max_deg = g->max_deg;
        pj.ids = edge_id;
        pj.caps = new_cap;
        pj.params = g->params;
        pj.gmode = g->opt.mode;
        pj.pp_ok = g->opt.mode == MF_MODE_PUSH_PULL;
        cudaGetLastError();   // an earlier, unrelated failure of this thread is not this launch's
        k_policy<<<kPolicyCtasPerSlot * g->grid, 256, 0, st>>>(g->dg, pj);
        MF_CUDA(cudaGetLastError());
        j.kind = JOB_AUTO;
    }
    j.k = 0;
    j.k_dev = k_dev;
    j.flags = flags;
    j.kc = g->kc;
    j.mode = g->opt.mode;
    j.pp = g->opt.mode == MF_MODE_PUSH_PULL;
    j.max_iters = g->max_iters;
    j.time_limit_ns = g->time_limit_ns;
    j.ids = edge_id;
    j.caps = new_cap;
    j.newc = g->b_newc;
    j.dlt = g->b_dlt;
    return launch(g, j, st);
}

int mf_set_stream(mf_graph *g, void *stream) {
    if (!g) return MF_EINVAL;
    MF_CUDA(cudaSetDevice(g->dev));
    if (g->last) MF_CUDA(cudaStreamSynchronize(g->last));
    g->last = static_cast<cudaStream_t>(stream);
    return MF_OK;
}

int mf_flow_value_async(mf_graph *g, int64_t *result, void *stream) {
    if (!g || !result) return MF_EINVAL;
    MF_CUDA(cudaSetDevice(g->dev));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MF_CUDA(cudaMemcpyAsync(result, g->dg.ctl, 16, cudaMemcpyDeviceToHost, st));
    return MF_OK;
}

int mf_device_bytes(const mf_graph *g, int64_t *bytes) {
    if (!g || !bytes) return MF_EINVAL;
    int64_t b = 0;
    for (size_t x : g->owned_bytes) b += int64_t(x);
    *bytes = b;
    return MF_OK;
}

int mf_grid_blocks(const mf_graph *g, int32_t *blocks) {
    if (!g || !blocks) return MF_EINVAL;
    *blocks = g->grid;
    return MF_OK;
}

int mf_set_grid_blocks(mf_graph *g, int32_t blocks) {
    if (!g || blocks < 1) return set_err(MF_EINVAL, "null graph or fewer than one CTA");
    g->grid = std::min(int(blocks), g->max_grid);
    return MF_OK;
}

int mf_sync(mf_graph *g) {
    if (!g) return MF_EINVAL;
    Ctl c;
    int rc = read_ctl(g, &c);
    if (rc) return rc;
    return status_to_code(g, c);
}

int mf_flow_value(mf_graph *g, int64_t *out) {
    if (!g || !out) return MF_EINVAL;
    Ctl c;
    int rc = read_ctl(g, &c, 16);   // status, batch_err, flow
    if (rc) return rc;
    if (c.status & ST_CHECK) {      // where the check failed, for the message
        rc = read_ctl(g, &c);
        if (rc) return rc;
    }
    rc = status_to_code(g, c);
    if (rc == MF_ETIMEOUT || rc == MF_ECHECK) return rc;
    if (!g->solved) return set_err(MF_ENOTSOLVED, "call mf_solve first");
    *out = c.flow;
    return rc;
}

int mf_min_cut(mf_graph *g, uint8_t *side, int32_t flags) {
    if (!g || !side) return MF_EINVAL;
    if (!g->solved) return set_err(MF_ENOTSOLVED, "call mf_solve first");
    MF_CUDA(cudaSetDevice(g->dev));
    int rc = refresh_heights(g);
    if (rc) return rc;
    unsigned char *dst = (flags & MF_DEVICE_PTRS) ? side : g->side_buf;
    int blocks = std::max(1, std::min(g->sms * 4, (g->n + 255) / 256));
    cudaGetLastError();   // an earlier, unrelated failure of this thread is not this launch's
    k_cut_side<<<blocks, 256, 0, g->last>>>(g->dg.h, g->n, dst);
    MF_CUDA(cudaGetLastError());
    if (!(flags & MF_DEVICE_PTRS))
        MF_CUDA(cudaMemcpyAsync(side, g->side_buf, size_t(g->n), cudaMemcpyDeviceToHost, g->last));
    return mf_sync(g);
}

int mf_stats_get(mf_graph *g, mf_stats *out) {
    if (!g || !out) return MF_EINVAL;
    Ctl c;
    int rc = read_ctl(g, &c);
    if (rc) return rc;
    std::memset(out, 0, sizeof(*out));
    out->flow = c.flow;
    out->iterations = c.iters;
    out->bfs_levels = c.st[S_LEVELS];
    out->bfs_vertices = c.st[S_BFS_VERTS];
    out->bfs_arcs = c.st[S_BFS_ARCS];
    out->worklist = c.st[S_WL];
    out->pr_arcs = c.st[S_PR_ARCS];
    out->pushes = c.st[S_PUSH];
    out->relabels = c.st[S_RELABEL];
    out->ri_arcs = c.st[S_RI_ARCS];
    out->ri_moves = c.st[S_RI_MOVES];
    out->batch = c.st[S_BATCH];
    out->clamped = c.st[S_CLAMPED];
    out->resat_arcs = c.st[S_RESAT];
    out->n = g->n;
    out->m = g->m;
    out->arcs = g->A;
    out->t_batch_ns = c.st[S_T_BATCH];
    out->t_reset_ns = c.st[S_T_RESET];
    out->t_bfs_ns = c.st[S_T_BFS];
    out->t_pr_ns = c.st[S_T_PRW];
    out->t_hub_ns = c.st[S_T_HUB];
    out->t_ri_ns = c.st[S_T_RI];
    out->hub_cycles = c.st[S_HUB_CYCLES];
    out->barriers = c.st[S_BARRIERS];
    out->bfs_bottom_up_levels = c.st[S_BU_LEVELS];
    out->pr_rounds = c.st[S_ROUNDS];
    out->policy_kind = c.pol_kind == JOB_RECOMPUTE ? 1 : 0;
    out->policy_kernel_cycles = c.pol_kc;
    out->policy_fallback = c.pol_fallback;
    out->policy_mode = g->policy == MF_POLICY_LEARNED ? c.pol_mode : g->opt.mode;
    out->exit_kind = c.exit_kind;
    out->status = c.status;
    out->kernel_cycles = g->kc;
    out->grid_blocks = g->grid;
    out->block_threads = kBlock;
    return MF_OK;
}

int mf_export_graph(mf_graph *g, int64_t *arc_row, int32_t *head, int32_t *rev, int32_t *cap) {
    if (!g) return MF_EINVAL;
    MF_CUDA(cudaSetDevice(g->dev));
    MF_CUDA(cudaStreamSynchronize(g->last));
    if (arc_row) {
        std::vector<int32_t> row(size_t(g->n) + 1);
        MF_CUDA(cudaMemcpy(row.data(), g->dg.row, row.size() * 4, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < row.size(); ++i) arc_row[i] = row[i];
    }
    if (head && g->A) MF_CUDA(cudaMemcpy(head, g->dg.head, size_t(g->A) * 4, cudaMemcpyDeviceToHost));
    if (rev && g->A) MF_CUDA(cudaMemcpy(rev, g->dg.rev, size_t(g->A) * 4, cudaMemcpyDeviceToHost));
    if (cap && g->A) MF_CUDA(cudaMemcpy(cap, g->dg.cap, size_t(g->A) * 4, cudaMemcpyDeviceToHost));
    return MF_OK;
}

int mf_export_state(mf_graph *g, int32_t *r, int64_t *excess, int32_t *height, int32_t flags) {
    if (!g) return MF_EINVAL;
    MF_CUDA(cudaSetDevice(g->dev));
    if (height && g->solved) {
        int rc = refresh_heights(g);
        if (rc) return rc;
    }
    cudaMemcpyKind kind = (flags & MF_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (r && g->A) MF_CUDA(cudaMemcpyAsync(r, g->dg.r, size_t(g->A) * 4, kind, g->last));
    if (excess) MF_CUDA(cudaMemcpyAsync(excess, g->dg.e, size_t(g->n) * 8, kind, g->last));
    if (height) MF_CUDA(cudaMemcpyAsync(height, g->dg.h, size_t(g->n) * 4, kind, g->last));
    MF_CUDA(cudaStreamSynchronize(g->last));
    return MF_OK;
}

int mf_import_state(mf_graph *g, const int32_t *r, const int64_t *excess, const int32_t *height, int32_t flags) {
    if (!g || !r || !excess || !height) return MF_EINVAL;
    MF_CUDA(cudaSetDevice(g->dev));
    cudaMemcpyKind kind = (flags & MF_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    MF_CUDA(cudaStreamSynchronize(g->last));
    if (g->A) MF_CUDA(cudaMemcpy(g->dg.r, r, size_t(g->A) * 4, kind));
    MF_CUDA(cudaMemcpy(g->dg.e, excess, size_t(g->n) * 8, kind));
    MF_CUDA(cudaMemcpy(g->dg.h, height, size_t(g->n) * 4, kind));
    // rebuild the mirror rr[a] = r[rev[a]] on the host side of the copy
    std::vector<int32_t> hr(size_t(g->A)), hrev(size_t(g->A)), hrr(size_t(g->A));
    if (g->A) {
        MF_CUDA(cudaMemcpy(hr.data(), g->dg.r, size_t(g->A) * 4, cudaMemcpyDeviceToHost));
        MF_CUDA(cudaMemcpy(hrev.data(), g->dg.rev, size_t(g->A) * 4, cudaMemcpyDeviceToHost));
        for (size_t a = 0; a < hr.size(); ++a) hrr[a] = hr[size_t(hrev[a])];
        MF_CUDA(cudaMemcpy(g->dg.rr, hrr.data(), size_t(g->A) * 4, cudaMemcpyHostToDevice));
    }
    // value of the imported state: e(t) plus the deficits (Alg. 4, final sum)
    std::vector<int64_t> he(size_t(g->n));
    MF_CUDA(cudaMemcpy(he.data(), g->dg.e, size_t(g->n) * 8, cudaMemcpyDeviceToHost));
    long long flow = he[size_t(g->t)];
    for (int32_t v = 0; v < g->n; ++v)
        if (v != g->s && v != g->t && he[size_t(v)] < 0) flow += he[size_t(v)];
    MF_CUDA(cudaMemset(g->dg.ctl, 0, sizeof(Ctl)));
    MF_CUDA(cudaMemset(g->dg.stamp, 0, size_t(std::max<int64_t>(g->m, 1)) * 4));
    MF_CUDA(cudaMemset(g->dg.astamp, 0, size_t(g->n) * 4));
    MF_CUDA(cudaMemset(g->dg.rstamp, 0, size_t(g->n) * 4));
    MF_CUDA(cudaMemset(g->dg.aq, 0, size_t(g->dg.qc) * 8));
    MF_CUDA(cudaMemcpy(&g->dg.ctl->flow, &flow, sizeof(flow), cudaMemcpyHostToDevice));
    MF_CUDA(cudaDeviceSynchronize());
    g->solved = true;
    return MF_OK;
}

int mf_set_time_limit(mf_graph *g, int32_t time_limit_ms) {
    if (!g || time_limit_ms < 0) return set_err(MF_EINVAL, "null graph or negative time limit");
    g->opt.time_limit_ms = time_limit_ms;
    g->time_limit_ns = 1000000ull * (unsigned long long)(time_limit_ms > 0 ? time_limit_ms : 60000);
    return MF_OK;
}

void mf_destroy(mf_graph *g) {
    if (!g) return;
    cudaSetDevice(g->dev);
    if (g->last) cudaStreamSynchronize(g->last);
    cudaDeviceSynchronize();
    for (void *p : g->owned) dfree(g, p);
    delete g;
}

int mf_set_policy(mf_graph *g, int32_t mode, const float *params) {
    if (!g || mode < MF_POLICY_FIXED || mode > MF_POLICY_LEARNED) return MF_EINVAL;
    if (mode == MF_POLICY_LEARNED && !params && !g->params)
        return set_err(MF_EINVAL, "the learned policy needs network parameters");
    MF_CUDA(cudaSetDevice(g->dev));
    if (params) {
        if (!g->params) g->params = dnew<float>(g, mlp::kTotal);
        if (!g->params) return set_err(MF_ENOMEM, "policy parameter allocation failed");
        MF_CUDA(cudaStreamSynchronize(g->last));
        MF_CUDA(cudaMemcpy(g->params, params, sizeof(float) * mlp::kTotal, cudaMemcpyHostToDevice));
    }
    g->policy = mode;
    return MF_OK;
}

int mf_policy_features(mf_graph *g, int64_t k, const int32_t *edge_id, const int32_t *new_cap, int32_t flags,
                       float *features) {
    if (!g || !features || k < 0 || k > g->m || (k > 0 && (!edge_id || !new_cap))) return MF_EINVAL;
    MF_CUDA(cudaSetDevice(g->dev));
    cudaStream_t st = g->last;
    int rc = ensure_batch_capacity(g, std::max<int64_t>(k, 1), st);
    if (rc) return rc;
    const int *ids = edge_id, *caps = new_cap;
    if (!(flags & MF_DEVICE_PTRS) && k > 0) {
        MF_CUDA(cudaMemcpyAsync(g->b_ids, edge_id, size_t(k) * 4, cudaMemcpyHostToDevice, st));
        MF_CUDA(cudaMemcpyAsync(g->b_caps, new_cap, size_t(k) * 4, cudaMemcpyHostToDevice, st));
        ids = g->b_ids;
        caps = g->b_caps;
    }
    rc = launch_policy(g, k, ids, caps, flags & MF_DELTA, st);
    if (rc) return rc;
    Ctl c;
    rc = read_ctl(g, &c);
    if (rc) return rc;
    for (int j = 0; j < mlp::kIn; ++j) features[j] = c.feat[j];
    return MF_OK;
}

int mf_trace_enable(mf_graph *g, int32_t capacity) {
    if (!g || capacity < 0) return MF_EINVAL;
    MF_CUDA(cudaSetDevice(g->dev));
    MF_CUDA(cudaStreamSynchronize(g->last));
    if (g->dg.trace) {
        dfree(g, g->dg.trace);
        dforget(g, g->dg.trace);
        g->dg.trace = nullptr;
        g->dg.trace_cap = 0;
    }
    if (capacity == 0) return MF_OK;
    g->dg.trace = dnew<TraceRec>(g, size_t(capacity));
    if (!g->dg.trace) return set_err(MF_ENOMEM, "trace buffer allocation failed");
    g->dg.trace_cap = capacity;
    return MF_OK;
}

int mf_trace_read(mf_graph *g, mf_trace_rec *out, int32_t max_records, int32_t *count) {
    if (!g || !count || max_records < 0 || (max_records > 0 && !out)) return MF_EINVAL;
    Ctl c;
    int rc = read_ctl(g, &c);
    if (rc) return rc;
    const int avail = std::min(c.trace_n, g->dg.trace_cap);
    *count = c.trace_n;
    const int k = std::min(avail, int(max_records));
    if (k <= 0 || !g->dg.trace) return MF_OK;
    std::vector<TraceRec> tmp(static_cast<size_t>(k));
    MF_CUDA(cudaMemcpy(tmp.data(), g->dg.trace, size_t(k) * sizeof(TraceRec), cudaMemcpyDeviceToHost));
    for (int i = 0; i < k; ++i) {
        int ph = MF_PHASE_BATCH;
        switch (tmp[size_t(i)].phase) {
            case S_T_RESET: ph = MF_PHASE_HEIGHT_INIT; break;
            case S_T_BFS: ph = MF_PHASE_BFS; break;
            case S_T_PRW: ph = MF_PHASE_PUSH_RELABEL; break;
            case S_T_HUB: ph = MF_PHASE_HUB; break;
            case S_T_RI: ph = MF_PHASE_REMOVE_INVALID; break;
            default: ph = MF_PHASE_BATCH; break;
        }
        out[i].phase = int16_t(ph);
        out[i].mode = tmp[size_t(i)].mode;
        out[i].iter = tmp[size_t(i)].iter;
        out[i].step = tmp[size_t(i)].step;
        out[i].count = tmp[size_t(i)].count;
        out[i].ns = tmp[size_t(i)].ns;
    }
    return MF_OK;
}

// Allocation-free static solve on a caller-provided Bi-CSR (see mf.h).
int mf_solve_bicsr_noalloc(int32_t n, int64_t arcs, const int32_t *row, const int32_t *head, const int32_t *rev,
                           const int32_t *cap, int32_t s, int32_t t, int32_t kernel_cycles, int32_t *r,
                           int64_t *excess, int32_t *height, int64_t *flow, void *stream) {
    if (n < 2 || s < 0 || t < 0 || s >= n || t >= n || s == t || arcs < 0)
        return set_err(MF_EINVAL, "bad sizes or terminals");
    if (n > kNoAllocMaxN || arcs > kNoAllocMaxArcs)
        return set_err(MF_EINVAL, "graph larger than the static scratch: at most " + std::to_string(kNoAllocMaxN) +
                                      " vertices and " + std::to_string(kNoAllocMaxArcs) + " arcs");
    if (!row || !head || !rev || !cap || !r || !excess || !height || !flow)
        return set_err(MF_EINVAL, "null argument");
    int dev = 0;
    MF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return set_err(MF_EINVAL, "device index out of range");
    // once per device: the device address of the static scratch array (host
    // code only sees a host-side stand-in for it) and the co-resident grid
    std::call_once(g_noalloc_once[dev], [dev]() {
        NoAllocDevice &D = g_noalloc_dev[dev];
        D.err = cudaGetSymbolAddress(reinterpret_cast<void **>(&D.base), g_noalloc_scratch);
        int per_sm = 0, sms = 0;
        if (D.err == cudaSuccess) D.err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (D.err == cudaSuccess) D.err = solve_kernels_prepare(dev);
        if (D.err == cudaSuccess)
            D.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve<false>, kBlock, kDynSmem);
        D.grid = std::min(per_sm * sms, kNoAllocMaxGrid);
        if (D.err == cudaSuccess && D.grid < 1) D.err = cudaErrorInvalidConfiguration;
    });
    const NoAllocDevice &ND = g_noalloc_dev[dev];
    if (ND.err != cudaSuccess)
        return set_err(MF_ECUDA, std::string("scratch set-up: ") + cudaGetErrorString(ND.err));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *b = ND.base;
    using Lo = NoAllocLayout;
    DevGraph D{};
    D.n = n; D.s = s; D.t = t; D.m = 0; D.A = arcs; D.cap_limit = 0;
    D.row = row; D.head = head; D.rev = rev; D.arc_of_edge = nullptr; D.edge_st = nullptr;
    D.cap = const_cast<int *>(cap);      // read only by a solve from zero flow
    D.r = r; D.e = reinterpret_cast<long long *>(excess); D.h = height;
    D.cap_edge = nullptr; D.stamp = nullptr;
    D.al16 = ((reinterpret_cast<uintptr_t>(head) | reinterpret_cast<uintptr_t>(r)) & 15u) == 0;
    D.ctl = reinterpret_cast<Ctl *>(b + Lo::ctl);
    D.rr = reinterpret_cast<int *>(b + Lo::rr);
    D.qb0 = reinterpret_cast<int *>(b + Lo::qb0);
    D.qb1 = reinterpret_cast<int *>(b + Lo::qb1);
    D.wl = reinterpret_cast<int *>(b + Lo::wl);
    D.rl = reinterpret_cast<int *>(b + Lo::rl);
    D.astamp = reinterpret_cast<unsigned *>(b + Lo::astamp);
    D.rstamp = reinterpret_cast<unsigned *>(b + Lo::rstamp);
    D.cb = reinterpret_cast<int2 *>(b + Lo::cb);
    D.hcl = reinterpret_cast<int2 *>(b + Lo::hcl);
    D.hlv0 = reinterpret_cast<int2 *>(b + Lo::hlv0);
    D.hlv1 = reinterpret_cast<int2 *>(b + Lo::hlv1);
    D.hikey = reinterpret_cast<unsigned *>(b + Lo::hikey);
    D.hl = reinterpret_cast<int *>(b + Lo::hl);
    D.hmode = reinterpret_cast<int *>(b + Lo::hmode);
    D.hnit = reinterpret_cast<int *>(b + Lo::hnit);
    D.hdone = reinterpret_cast<int *>(b + Lo::hdone);
    D.hkey = reinterpret_cast<unsigned long long *>(b + Lo::hkey);
    D.hrem = reinterpret_cast<long long *>(b + Lo::hrem);
    D.hl2 = reinterpret_cast<int *>(b + Lo::hl2);
    D.hri = reinterpret_cast<int2 *>(b + Lo::hri);
    D.aq = reinterpret_cast<unsigned long long *>(b + Lo::aq);
    D.qc = std::min(std::max(n, 1024), kNoAllocMaxN);
    // the previous call's contents stay in the array: clear what must start at 0
    MF_CUDA(cudaMemsetAsync(D.ctl, 0, sizeof(Ctl), st));
    MF_CUDA(cudaMemsetAsync(D.aq, 0, sizeof(unsigned long long) * size_t(D.qc), st));
    MF_CUDA(cudaMemsetAsync(D.astamp, 0, sizeof(unsigned) * size_t(n), st));
    MF_CUDA(cudaMemsetAsync(D.rstamp, 0, sizeof(unsigned) * size_t(n), st));
    Job j{};
    j.kind = JOB_SOLVE;
    j.exact_exit = 1;   // the caller reads the cut {height >= n} from the heights
    j.st = D.ctl->st;
    j.trace = nullptr;
    j.kc = kernel_cycles > 0 ? kernel_cycles : int(std::max<int64_t>(1, (arcs / 2 + n / 2) / n));
    j.max_iters = 4LL * n + 1000;
    j.time_limit_ns = 60ull * 1000ull * 1000ull * 1000ull;
    void *args[] = {&D, &j};
    cudaError_t e =
        cudaLaunchCooperativeKernel((const void *)k_solve<false>, dim3(ND.grid), dim3(kBlock), args, kDynSmem, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(MF_ECUDA, std::string("cooperative launch: ") + cudaGetErrorString(e));
    }
    int32_t status = 0;
    MF_CUDA(cudaMemcpyAsync(&status, &D.ctl->status, sizeof(status), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaMemcpyAsync(flow, &D.ctl->flow, sizeof(*flow), cudaMemcpyDeviceToHost, st));
    MF_CUDA(cudaStreamSynchronize(st));
    if (status & ST_STICKY) return set_err(MF_ETIMEOUT, "device loop did not finish");
    return MF_OK;
}

}  // extern "C"
