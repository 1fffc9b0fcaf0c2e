/*
 * CPU oracle for the dynamic max-flow path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark load this file's shared library.  The CUDA library never links,
 * includes or calls it, and it shares no code with the CUDA library.
 *
 * What the method computes has a plain definition: the value of a maximum
 * s-t flow of the graph with its current capacities (Sec. 2.1, the problem
 * statement: capacity constraint 0 <= f(u,v) <= c(u,v) and conservation at
 * every vertex other than s and t).  The dynamic method of Sec. 4.1 reaches
 * exactly that value (its closing theorem), so the oracle does not imitate the
 * dynamic method: after every batch the test rebuilds the capacities and calls
 * orc_maxflow_fifo() from scratch.
 *
 *   orc_maxflow_fifo   sequential FIFO push-relabel (Goldberg-Tarjan, the
 *                      algorithm recalled in Sec. 2.2) with exact global
 *                      relabelling by backward BFS from t (Sec. 2.2's global
 *                      relabelling heuristic).  Residual network with one
 *                      forward arc per input edge and one paired reverse arc
 *                      of capacity 0 -- no merging of parallel or antiparallel
 *                      edges; self-loops are dropped.  64-bit residuals.
 *   orc_maxflow_ek     Edmonds-Karp shortest augmenting paths (Sec. 2.2), an
 *                      independent cross-check for small graphs.
 *   orc_mincut_brute   minimum over all s-t cuts by enumeration (max-flow =
 *                      min-cut), for n <= 26.
 *   orc_certify        checks that a claimed max-flow state of ANY solver is
 *                      optimal: capacity feasibility, excess bookkeeping, a
 *                      cut with no residual arc crossing it, sign conditions
 *                      and value = cut capacity (Theorem 3.2's cut argument
 *                      and the pseudo-flow theorem of Sec. 4.1).  It derives
 *                      no expected value from the state it checks.
 *   orc_bfs_heights    exact backward BFS distances to a root set in a given
 *                      residual graph (the global relabel of Sec. 2.2 / Alg. 4).
 *
 * Return codes: 0 = success, negative = bad arguments / out of memory.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

/* ------------------------------------------------------------------------ */
/* Residual network with explicit paired arcs                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t n;
    int64_t na;          /* number of arcs (2 per non-loop edge)           */
    int64_t *first;      /* [n+1] arcs of u are first[u] .. first[u+1]-1   */
    int32_t *to;         /* [na] head of each arc                          */
    int64_t *mate;       /* [na] position of the paired arc                */
    int64_t *res;        /* [na] residual capacity                         */
    int64_t *cap;        /* [na] original capacity (0 for reverse arcs)    */
    int64_t *edge_arc;   /* [m]  position of each edge's forward arc or -1 */
} net_t;

static void net_free(net_t *g) {
    free(g->first); free(g->to); free(g->mate); free(g->res); free(g->cap); free(g->edge_arc);
    memset(g, 0, sizeof(*g));
}

static int net_build(net_t *g, int32_t n, int64_t m, const int64_t *row_ptr,
                     const int32_t *col, const int32_t *cap) {
    memset(g, 0, sizeof(*g));
    g->n = n;
    int64_t loops = 0;
    for (int32_t u = 0; u < n; ++u)
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            if (col[e] < 0 || col[e] >= n || cap[e] < 0) return ORC_EINVAL;
            if (col[e] == u) ++loops;
        }
    int64_t na = 2 * (m - loops);
    g->na = na;
    g->first = calloc((size_t)n + 1, sizeof(int64_t));
    g->to = malloc(sizeof(int32_t) * (size_t)(na ? na : 1));
    g->mate = malloc(sizeof(int64_t) * (size_t)(na ? na : 1));
    g->res = malloc(sizeof(int64_t) * (size_t)(na ? na : 1));
    g->cap = malloc(sizeof(int64_t) * (size_t)(na ? na : 1));
    g->edge_arc = malloc(sizeof(int64_t) * (size_t)(m ? m : 1));
    int64_t *fill = calloc((size_t)n + 1, sizeof(int64_t));
    if (!g->first || !g->to || !g->mate || !g->res || !g->cap || !g->edge_arc || !fill) {
        free(fill); net_free(g); return ORC_ENOMEM;
    }
    /* out-degree in the residual network: each edge gives its tail one arc
       and its head one arc */
    for (int32_t u = 0; u < n; ++u)
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col[e];
            if (v == u) continue;
            g->first[u + 1]++;
            g->first[v + 1]++;
        }
    for (int32_t u = 0; u < n; ++u) g->first[u + 1] += g->first[u];
    memcpy(fill, g->first, sizeof(int64_t) * ((size_t)n + 1));
    for (int32_t u = 0; u < n; ++u)
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col[e];
            if (v == u) { g->edge_arc[e] = -1; continue; }
            int64_t a = fill[u]++, b = fill[v]++;
            g->to[a] = v; g->res[a] = cap[e]; g->cap[a] = cap[e]; g->mate[a] = b;
            g->to[b] = u; g->res[b] = 0;      g->cap[b] = 0;      g->mate[b] = a;
            g->edge_arc[e] = a;
        }
    free(fill);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* FIFO push-relabel with global relabelling                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    net_t *g;
    int32_t s, t, n;
    int32_t *d;        /* height (distance label)                        */
    int64_t *ex;       /* excess                                         */
    int64_t *cur;      /* current-arc pointer                            */
    int32_t *q;        /* FIFO of active vertices, circular, capacity n  */
    int64_t qh, qt;    /* head / tail counters                           */
    uint8_t *inq;
    int32_t *bfs;      /* BFS queue                                      */
} fifo_t;

static void fifo_push_q(fifo_t *F, int32_t v) {
    if (F->inq[v]) return;
    F->inq[v] = 1;
    F->q[F->qt % F->n] = v;
    F->qt++;
}

/* Exact heights: d(v) = residual distance from v to t; unreachable -> n.
   Rebuilds the FIFO from the active vertices (e > 0, d < n). */
static void fifo_global_relabel(fifo_t *F) {
    net_t *g = F->g;
    int32_t n = F->n;
    for (int32_t v = 0; v < n; ++v) F->d[v] = n;
    int64_t head = 0, tail = 0;
    F->d[F->t] = 0;
    F->bfs[tail++] = F->t;
    while (head < tail) {
        int32_t u = F->bfs[head++];
        for (int64_t a = g->first[u]; a < g->first[u + 1]; ++a) {
            int32_t w = g->to[a];
            /* the paired arc w -> u is residual: w reaches u */
            if (w != F->s && F->d[w] == n && g->res[g->mate[a]] > 0) {
                F->d[w] = F->d[u] + 1;
                F->bfs[tail++] = w;
            }
        }
    }
    F->d[F->s] = n;
    F->qh = F->qt = 0;
    memset(F->inq, 0, (size_t)n);
    for (int32_t v = 0; v < n; ++v) {
        F->cur[v] = g->first[v];
        if (v != F->s && v != F->t && F->ex[v] > 0 && F->d[v] < n) fifo_push_q(F, v);
    }
}

int orc_maxflow_fifo(int32_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                     const int32_t *cap, int32_t s, int32_t t, int64_t *flow_out,
                     /* optional final state (any may be NULL); arrays sized as
                        orc_arc_count() reports */
                     int64_t *arc_first, int32_t *arc_head, int64_t *arc_mate,
                     int64_t *arc_cap, int64_t *arc_res, int64_t *excess, int32_t *height) {
    if (n < 2 || s < 0 || t < 0 || s >= n || t >= n || s == t || m < 0 || !flow_out)
        return ORC_EINVAL;
    net_t g;
    int rc = net_build(&g, n, m, row_ptr, col, cap);
    if (rc) return rc;
    fifo_t F;
    memset(&F, 0, sizeof(F));
    F.g = &g; F.s = s; F.t = t; F.n = n;
    F.d = calloc((size_t)n, sizeof(int32_t));
    F.ex = calloc((size_t)n, sizeof(int64_t));
    F.cur = calloc((size_t)n, sizeof(int64_t));
    F.q = calloc((size_t)n, sizeof(int32_t));
    F.inq = calloc((size_t)n, 1);
    F.bfs = calloc((size_t)n, sizeof(int32_t));
    if (!F.d || !F.ex || !F.cur || !F.q || !F.inq || !F.bfs) { rc = ORC_ENOMEM; goto done; }

    /* saturate every arc leaving s */
    for (int64_t a = g.first[s]; a < g.first[s + 1]; ++a) {
        int64_t c = g.res[a];
        if (c <= 0) continue;
        g.res[a] = 0;
        g.res[g.mate[a]] += c;
        F.ex[g.to[a]] += c;
        F.ex[s] -= c;
    }
    fifo_global_relabel(&F);
    int64_t relabels = 0;
    while (F.qh < F.qt) {
        int32_t u = F.q[F.qh % n];
        F.qh++;
        F.inq[u] = 0;
        /* discharge u */
        while (F.ex[u] > 0 && F.d[u] < n) {
            if (F.cur[u] == g.first[u + 1]) {
                /* relabel: one above the lowest residual neighbour */
                int32_t best = 2 * n;
                for (int64_t a = g.first[u]; a < g.first[u + 1]; ++a)
                    if (g.res[a] > 0 && F.d[g.to[a]] < best) best = F.d[g.to[a]];
                F.d[u] = (best + 1 < n) ? best + 1 : n;
                F.cur[u] = g.first[u];
                ++relabels;
                continue;
            }
            int64_t a = F.cur[u];
            int32_t w = g.to[a];
            if (g.res[a] > 0 && F.d[u] == F.d[w] + 1) {
                int64_t delta = F.ex[u] < g.res[a] ? F.ex[u] : g.res[a];
                g.res[a] -= delta;
                g.res[g.mate[a]] += delta;
                F.ex[u] -= delta;
                F.ex[w] += delta;
                if (w != s && w != t) fifo_push_q(&F, w);
            } else {
                F.cur[u]++;
            }
        }
        if (relabels >= n) {
            relabels = 0;
            fifo_global_relabel(&F);
        }
    }
    *flow_out = F.ex[t];
    if (arc_first) memcpy(arc_first, g.first, sizeof(int64_t) * ((size_t)n + 1));
    if (arc_head) memcpy(arc_head, g.to, sizeof(int32_t) * (size_t)g.na);
    if (arc_mate) memcpy(arc_mate, g.mate, sizeof(int64_t) * (size_t)g.na);
    if (arc_cap) memcpy(arc_cap, g.cap, sizeof(int64_t) * (size_t)g.na);
    if (arc_res) memcpy(arc_res, g.res, sizeof(int64_t) * (size_t)g.na);
    if (excess) memcpy(excess, F.ex, sizeof(int64_t) * (size_t)n);
    if (height) {
        /* final exact distances to t, so that {d >= n} is the source side */
        fifo_global_relabel(&F);
        memcpy(height, F.d, sizeof(int32_t) * (size_t)n);
    }
done:
    free(F.d); free(F.ex); free(F.cur); free(F.q); free(F.inq); free(F.bfs);
    net_free(&g);
    return rc;
}

/* number of residual arcs orc_maxflow_fifo() uses for this graph */
int64_t orc_arc_count(int32_t n, const int64_t *row_ptr, const int32_t *col) {
    int64_t na = 0;
    for (int32_t u = 0; u < n; ++u)
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
            if (col[e] != u) na += 2;
    return na;
}

/* ------------------------------------------------------------------------ */
/* Edmonds-Karp                                                             */
/* ------------------------------------------------------------------------ */
int orc_maxflow_ek(int32_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                   const int32_t *cap, int32_t s, int32_t t, int64_t *flow_out) {
    if (n < 2 || s < 0 || t < 0 || s >= n || t >= n || s == t || m < 0 || !flow_out)
        return ORC_EINVAL;
    net_t g;
    int rc = net_build(&g, n, m, row_ptr, col, cap);
    if (rc) return rc;
    int64_t *parc = malloc(sizeof(int64_t) * (size_t)n);
    int32_t *q = malloc(sizeof(int32_t) * (size_t)n);
    if (!parc || !q) { free(parc); free(q); net_free(&g); return ORC_ENOMEM; }
    int64_t flow = 0;
    for (;;) {
        for (int32_t v = 0; v < n; ++v) parc[v] = -2;   /* -2: unvisited */
        parc[s] = -1;
        int64_t head = 0, tail = 0;
        q[tail++] = s;
        while (head < tail && parc[t] == -2) {
            int32_t u = q[head++];
            for (int64_t a = g.first[u]; a < g.first[u + 1]; ++a) {
                int32_t w = g.to[a];
                if (g.res[a] > 0 && parc[w] == -2) { parc[w] = a; q[tail++] = w; }
            }
        }
        if (parc[t] == -2) break;
        int64_t bott = INT64_MAX;
        for (int32_t v = t; v != s; ) {
            int64_t a = parc[v];
            if (g.res[a] < bott) bott = g.res[a];
            v = g.to[g.mate[a]];
        }
        for (int32_t v = t; v != s; ) {
            int64_t a = parc[v];
            g.res[a] -= bott;
            g.res[g.mate[a]] += bott;
            v = g.to[g.mate[a]];
        }
        flow += bott;
    }
    *flow_out = flow;
    free(parc); free(q); net_free(&g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Minimum s-t cut by enumeration                                            */
/* ------------------------------------------------------------------------ */
int orc_mincut_brute(int32_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                     const int32_t *cap, int32_t s, int32_t t, int64_t *cut_out) {
    if (n < 2 || n > 26 || s < 0 || t < 0 || s >= n || t >= n || s == t || !cut_out)
        return ORC_EINVAL;
    int32_t others[32];
    int k = 0;
    for (int32_t v = 0; v < n; ++v) if (v != s && v != t) others[k++] = v;
    int64_t best = INT64_MAX;
    uint8_t side[32];
    for (uint64_t mask = 0; mask < (1ull << k); ++mask) {
        memset(side, 0, sizeof(side));
        side[s] = 1;
        for (int i = 0; i < k; ++i) if (mask >> i & 1) side[others[i]] = 1;
        int64_t c = 0;
        for (int32_t u = 0; u < n; ++u)
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
                if (side[u] && !side[col[e]]) c += cap[e];
        if (c < best) best = c;
    }
    (void)m;
    *cut_out = best;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Backward BFS distances                                                   */
/* ------------------------------------------------------------------------ */
/* h[v] = length of the shortest residual path from v to any root
   (root[v] != 0), n if there is none; s is never relabelled (h[s] = n).
   Arcs are grouped by tail: arc a of row u goes u -> head[a]; rev[a] is its
   paired arc head[a] -> u; r[] are residual capacities. */
int orc_bfs_heights(int32_t n, const int64_t *arc_row, const int32_t *head, const int64_t *rev,
                    const int64_t *r, const uint8_t *root, int32_t s, int32_t *h) {
    int32_t *q = malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!q) return ORC_ENOMEM;
    int64_t qh = 0, qt = 0;
    for (int32_t v = 0; v < n; ++v) {
        h[v] = n;
        if (v != s && root[v]) { h[v] = 0; q[qt++] = v; }
    }
    while (qh < qt) {
        int32_t u = q[qh++];
        for (int64_t a = arc_row[u]; a < arc_row[u + 1]; ++a) {
            int32_t w = head[a];
            if (w != s && h[w] == n && r[rev[a]] > 0) { h[w] = h[u] + 1; q[qt++] = w; }
        }
    }
    free(q);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Optimality certificate of a claimed max-flow state                       */
/* ------------------------------------------------------------------------ */
/* Failure bits returned through *fail_bits (0 = certified). */
#define CERT_STRUCT   (1u << 0)   /* rev / head / tail inconsistent            */
#define CERT_CAPS     (1u << 1)   /* arc capacities != current edge capacities */
#define CERT_RESID    (1u << 2)   /* r < 0 or r + r_rev != c + c_rev           */
#define CERT_EXCESS   (1u << 3)   /* e(v) != net inflow, or sum e != 0         */
#define CERT_CUT      (1u << 4)   /* s not in S, t in S, or residual arc S->T  */
#define CERT_SIGNS    (1u << 5)   /* e < 0 in S-{s} or e > 0 in T-{t}          */
#define CERT_VALUE    (1u << 6)   /* value != sum_T e or != C(S, T)            */
#define CERT_HEIGHTS  (1u << 7)   /* h is not the BFS fixed point / side       */

static int cmp_pair(const void *x, const void *y) {
    const int64_t *a = x, *b = y;
    return (a[0] > b[0]) - (a[0] < b[0]);
}

/* State layout (any solver): vertex u's arcs are arc_row[u] .. arc_row[u+1]-1,
   arc a goes u -> head[a] with paired arc rev[a], capacity arc_cap[a] and
   residual r[a]; excess[v]; side[v] = 1 for the source side S.  Several input
   edges may share one arc (parallel edges), and both directions of a vertex
   pair share one arc pair.  height may be NULL; if given, it must equal the
   exact backward BFS distance to the roots {t} U {v != s : e(v) < 0} with n
   for unreachable vertices, and side must equal (height >= n).
   Edges: current capacities in CSR (row_ptr, col, cap).  flow: the claimed
   max-flow value. */
int orc_certify(int32_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                const int32_t *cap, int32_t s, int32_t t,
                const int64_t *arc_row, const int32_t *head, const int64_t *rev,
                const int64_t *arc_cap, const int64_t *r, const int64_t *excess,
                const uint8_t *side, const int32_t *height, int64_t flow,
                uint32_t *fail_bits, int64_t *fail_where) {
    if (n < 2 || !fail_bits || !fail_where) return ORC_EINVAL;
    uint32_t bad = 0;
    int64_t where = -1;
#define FAIL(bit, w) do { if (!(bad & (bit))) { if (where < 0) where = (w); } bad |= (bit); } while (0)
    int64_t A = arc_row[n];
    /* structure */
    for (int32_t u = 0; u < n; ++u)
        for (int64_t a = arc_row[u]; a < arc_row[u + 1]; ++a) {
            int64_t b = rev[a];
            if (head[a] < 0 || head[a] >= n || head[a] == u || b < 0 || b >= A || rev[b] != a ||
                head[b] != u || !(arc_row[head[a]] <= b && b < arc_row[head[a] + 1]))
                FAIL(CERT_STRUCT, a);
        }
    if (bad) { *fail_bits = bad; *fail_where = where; return 0; }
    /* capacities: per tail u, sum of edge caps per head == sum of arc caps per head */
    int64_t maxdeg = 0;
    for (int32_t u = 0; u < n; ++u) {
        int64_t d = (row_ptr[u + 1] - row_ptr[u]) + (arc_row[u + 1] - arc_row[u]);
        if (d > maxdeg) maxdeg = d;
    }
    int64_t *buf = malloc(sizeof(int64_t) * 2 * (size_t)(maxdeg ? maxdeg : 1));
    if (!buf) return ORC_ENOMEM;
    for (int32_t u = 0; u < n && !(bad & CERT_CAPS); ++u) {
        int64_t k = 0;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            if (col[e] == u) continue;
            buf[2 * k] = col[e]; buf[2 * k + 1] = cap[e]; ++k;
        }
        for (int64_t a = arc_row[u]; a < arc_row[u + 1]; ++a) {
            buf[2 * k] = head[a]; buf[2 * k + 1] = -arc_cap[a]; ++k;
        }
        qsort(buf, (size_t)k, 2 * sizeof(int64_t), cmp_pair);
        for (int64_t i = 0; i < k; ) {
            int64_t j = i, sum = 0;
            while (j < k && buf[2 * j] == buf[2 * i]) { sum += buf[2 * j + 1]; ++j; }
            if (sum != 0) { FAIL(CERT_CAPS, u); break; }
            i = j;
        }
    }
    free(buf);
    /* residuals */
    for (int64_t a = 0; a < A; ++a)
        if (r[a] < 0 || r[a] + r[rev[a]] != arc_cap[a] + arc_cap[rev[a]]) FAIL(CERT_RESID, a);
    /* excess = net inflow; flow on arc a is arc_cap[a] - r[a] (net, pair-wise) */
    int64_t total = 0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t inflow = 0;
        for (int64_t a = arc_row[v]; a < arc_row[v + 1]; ++a) inflow += r[a] - arc_cap[a];
        if (inflow != excess[v]) FAIL(CERT_EXCESS, v);
        total += excess[v];
    }
    if (total != 0) FAIL(CERT_EXCESS, -2);
    /* cut */
    if (!side[s] || side[t]) FAIL(CERT_CUT, -3);
    for (int32_t u = 0; u < n; ++u) {
        if (!side[u]) continue;
        for (int64_t a = arc_row[u]; a < arc_row[u + 1]; ++a)
            if (!side[head[a]] && r[a] > 0) FAIL(CERT_CUT, a);
    }
    /* signs */
    for (int32_t v = 0; v < n; ++v) {
        if (v == s || v == t) continue;
        if (side[v] && excess[v] < 0) FAIL(CERT_SIGNS, v);
        if (!side[v] && excess[v] > 0) FAIL(CERT_SIGNS, v);
    }
    /* value: sum of excess over T, and the capacity of the cut from the input edges */
    int64_t sumT = 0, cut = 0;
    for (int32_t v = 0; v < n; ++v) if (!side[v]) sumT += excess[v];
    for (int32_t u = 0; u < n; ++u) {
        if (!side[u]) continue;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
            if (!side[col[e]]) cut += cap[e];
    }
    if (sumT != flow || cut != flow) FAIL(CERT_VALUE, -4);
    /* heights: BFS fixed point */
    if (height) {
        uint8_t *root = malloc((size_t)n);
        int32_t *hb = malloc(sizeof(int32_t) * (size_t)n);
        if (!root || !hb) { free(root); free(hb); return ORC_ENOMEM; }
        for (int32_t v = 0; v < n; ++v) root[v] = (v == t) || (v != s && excess[v] < 0);
        orc_bfs_heights(n, arc_row, head, rev, r, root, s, hb);
        for (int32_t v = 0; v < n; ++v)
            if (hb[v] != height[v] || (height[v] >= n) != (side[v] != 0)) { FAIL(CERT_HEIGHTS, v); break; }
        free(root); free(hb);
    }
#undef FAIL
    *fail_bits = bad;
    *fail_where = where;
    return 0;
}
