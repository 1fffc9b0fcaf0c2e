// Host construction of the Bi-CSR graph representation (Sec. 5.1 of the
// paper: outgoing and incoming edges of every vertex in one list, zero-
// capacity entries for missing reverse edges, and an array giving the
// position of each arc's reverse in the neighbour's list, so that a push
// touches both directions in O(1)).
//
// Parallel edges u -> v share one arc (capacities add) and both directions of
// a vertex pair form one arc pair; this changes no max-flow value.  The work
// is split over host threads by vertex ranges.
#include <algorithm>
#include <atomic>
#include <climits>
#include <new>
#include <thread>

#include "mf_internal.h"

namespace mf {
namespace {

template <class F>
void parallel_for(int64_t count, F &&fn) {
    unsigned hw = std::thread::hardware_concurrency();
    int64_t nth = std::max<int64_t>(1, std::min<int64_t>(hw ? hw : 1, 64));
    if (count < (1 << 15) || nth == 1) {
        fn(int64_t(0), count);
        return;
    }
    const int64_t grain = std::max<int64_t>(4096, count / (nth * 16));
    std::atomic<int64_t> next(0);
    std::vector<std::thread> pool;
    for (int64_t i = 0; i < nth; ++i)
        pool.emplace_back([&]() {
            for (;;) {
                int64_t b = next.fetch_add(grain);
                if (b >= count) break;
                fn(b, std::min(count, b + grain));
            }
        });
    for (auto &th : pool) th.join();
}

inline int64_t find_sorted(const int32_t *a, int64_t lo, int64_t hi, int32_t key) {
    const int32_t *p = std::lower_bound(a + lo, a + hi, key);
    return (p != a + hi && *p == key) ? (p - a) : -1;
}

}  // namespace

int build_bicsr(int32_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                const int32_t *cap, int32_t s, int32_t t, HostBiCSR *out) {
    if (n < 2 || m < 0 || m >= INT32_MAX || s < 0 || t < 0 || s >= n || t >= n || s == t)
        return 1;
    if (row_ptr[0] != 0 || row_ptr[n] != m) return 1;
    for (int32_t u = 0; u < n; ++u)
        if (row_ptr[u + 1] < row_ptr[u]) return 1;
    std::atomic<int> bad(0);
    parallel_for(m, [&](int64_t b, int64_t e) {
        for (int64_t i = b; i < e; ++i)
            if (col[i] < 0 || col[i] >= n || cap[i] < 0) bad.store(1);
    });
    if (bad.load()) return 1;
    try {
        HostBiCSR &G = *out;
        G.n = n; G.m = m; G.s = s; G.t = t;
        // 1. every vertex's neighbour multiset (out-heads and in-tails)
        std::vector<int64_t> deg2(size_t(n) + 1, 0);
        for (int32_t u = 0; u < n; ++u)
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                int32_t v = col[e];
                if (v == u) continue;
                deg2[u + 1]++;
                deg2[v + 1]++;
            }
        for (int32_t u = 0; u < n; ++u) deg2[u + 1] += deg2[u];
        std::vector<int32_t> nb(size_t(deg2[n]));
        {
            std::vector<int64_t> fill(deg2.begin(), deg2.end() - 1);
            for (int32_t u = 0; u < n; ++u)
                for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                    int32_t v = col[e];
                    if (v == u) continue;
                    nb[size_t(fill[u]++)] = v;
                    nb[size_t(fill[v]++)] = u;
                }
        }
        // 2. sort + unique per vertex
        std::vector<int32_t> dcount(size_t(n), 0);
        parallel_for(n, [&](int64_t b, int64_t e) {
            for (int64_t u = b; u < e; ++u) {
                int32_t *p = nb.data() + deg2[u], *q = nb.data() + deg2[u + 1];
                std::sort(p, q);
                dcount[size_t(u)] = int32_t(std::unique(p, q) - p);
            }
        });
        int64_t A = 0;
        for (int32_t u = 0; u < n; ++u) A += dcount[size_t(u)];
        if (A >= INT32_MAX) return 1;
        G.arcs = A;
        G.row.assign(size_t(n) + 1, 0);
        for (int32_t u = 0; u < n; ++u) G.row[size_t(u) + 1] = G.row[size_t(u)] + dcount[size_t(u)];
        G.head.resize(size_t(A));
        parallel_for(n, [&](int64_t b, int64_t e) {
            for (int64_t u = b; u < e; ++u)
                std::copy(nb.data() + deg2[u], nb.data() + deg2[u] + dcount[size_t(u)],
                          G.head.data() + G.row[size_t(u)]);
        });
        std::vector<int32_t>().swap(nb);
        // 3. reverse arcs
        G.rev.resize(size_t(A));
        parallel_for(n, [&](int64_t b, int64_t e) {
            for (int64_t u = b; u < e; ++u)
                for (int32_t a = G.row[size_t(u)]; a < G.row[size_t(u) + 1]; ++a) {
                    int32_t v = G.head[size_t(a)];
                    G.rev[size_t(a)] = int32_t(find_sorted(G.head.data(), G.row[size_t(v)],
                                                           G.row[size_t(v) + 1], int32_t(u)));
                }
        });
        // 4. edge -> arc map, arc capacities, pair multiplicities
        G.arc_of_edge.assign(size_t(m), -1);
        G.cap.assign(size_t(A), 0);
        std::vector<int32_t> mult(size_t(A), 0);
        std::atomic<int> overflow(0);
        parallel_for(n, [&](int64_t b, int64_t e) {
            for (int64_t u = b; u < e; ++u)
                for (int64_t i = row_ptr[u]; i < row_ptr[u + 1]; ++i) {
                    if (col[i] == u) continue;
                    int64_t a = find_sorted(G.head.data(), G.row[size_t(u)], G.row[size_t(u) + 1], col[i]);
                    G.arc_of_edge[size_t(i)] = int32_t(a);
                    int64_t c = int64_t(G.cap[size_t(a)]) + cap[i];
                    if (c > INT32_MAX) { overflow.store(1); c = INT32_MAX; }
                    G.cap[size_t(a)] = int32_t(c);
                    mult[size_t(a)]++;
                }
        });
        int64_t maxmult = 1;
        for (int64_t a = 0; a < A; ++a) {
            int64_t pm = int64_t(mult[size_t(a)]) + mult[size_t(G.rev[size_t(a)])];
            if (pm > maxmult) maxmult = pm;
        }
        G.cap_limit = int32_t(INT32_MAX / maxmult);
        if (overflow.load()) return 1;
        for (int64_t i = 0; i < m; ++i)
            if (cap[i] > G.cap_limit) return 1;
        // 5. work-item bound for big vertices
        G.chunk_items = 0;
        G.hubs = 0;
        G.hub_chunk_items = 0;
        G.max_deg = 0;
        for (int32_t u = 0; u < n; ++u) {
            int32_t d = G.row[size_t(u) + 1] - G.row[size_t(u)];
            G.max_deg = std::max(G.max_deg, d);
            if (d > kBigDeg) G.chunk_items += (d + kChunk - 1) / kChunk;
            if (d > kHubDeg) {
                G.hubs += 1;
                G.hub_chunk_items += (d + kPrChunk - 1) / kPrChunk;
            }
        }
    } catch (const std::bad_alloc &) {
        return 2;
    }
    return 0;
}

}  // namespace mf
