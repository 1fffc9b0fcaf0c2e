// Internal declarations shared by the host graph builder (mf_build.cpp) and
// the CUDA library (mf_gpu.cu).  Not part of the public ABI (include/mf.h).
#pragma once

#include <cstdint>
#include <vector>

namespace mf {

// Frontier vertices whose Bi-CSR degree exceeds kBigDeg are expanded by the
// BFS as kChunk-arc work items spread over all warps instead of inside their
// 32-vertex group, so that no warp holds more than 32 x kBigDeg arcs of a
// level.
constexpr int kBigDeg = 64;
constexpr int kChunk = 256;
// Active vertices whose degree exceeds kHubDeg ("hubs") run PushRelabel and
// RemoveInvalidEdges cooperatively over the whole grid, in kPrChunk-arc work
// items; smaller ones are handled by one warp each.
constexpr int kHubDeg = 512;
constexpr int kPrChunk = 256;

// Host image of the Bi-CSR of Sec. 5.1.  Vertex u owns arcs row[u] ..
// row[u+1]-1, one per distinct neighbour v (u -> v edge, v -> u edge, or
// both), sorted by v.  rev[a] is the arc of the opposite direction in the
// neighbour's list.  cap[a] is the sum of the capacities of the input edges
// u -> v (0 when there is none).  arc_of_edge[e] is the arc that carries input
// edge e, or -1 for a self-loop.
struct HostBiCSR {
    int32_t n = 0;
    int64_t m = 0;
    int64_t arcs = 0;
    int32_t s = 0, t = 0;
    std::vector<int32_t> row;
    std::vector<int32_t> head, rev, cap;
    std::vector<int32_t> arc_of_edge;
    int32_t cap_limit = 0;      // largest capacity one edge may take
    int64_t chunk_items = 0;    // sum over big vertices of ceil(deg / kChunk)
    int64_t hubs = 0;           // vertices with degree > kHubDeg
    int64_t hub_chunk_items = 0;  // sum over hubs of ceil(deg / kPrChunk)
    int32_t max_deg = 0;
};

// Returns 0 on success, 1 (MF_EINVAL) on bad input, 2 (MF_ENOMEM) on
// allocation failure.  Inputs are host pointers.
int build_bicsr(int32_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                const int32_t *cap, int32_t s, int32_t t, HostBiCSR *out);

}  // namespace mf
