// Internal definitions shared by the CUDA translation units of libtc.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "tc.h"

namespace tc {

// Sentinel adjacency word: larger than every real entry (id < 2^30 - 1
// gives (id << 2) | 3 <= 0xFFFFFFFB).
constexpr uint32_t SENT = 0xFFFFFFFFu;
// Sentinel words stored after the adjacency array so that vector loads of a
// merge window may run past the last row.
constexpr int64_t ADJ_PAD = 8192;

// Whether the sorted adjacency row l[0..n) holds neighbour id `key`
// (binary search on the id bits of the tagged words).
__device__ __forceinline__ bool list_has(const uint32_t* l, int n, uint32_t key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((l[mid] >> 2) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo < n && (l[lo] >> 2) == key;
}
// Accumulator slots per graph: 64 triad codes, then the dyadic sums
// n - |N(u)| - |N(v)| over the dyads with pre = 1, 2, 3 (slots 64, 65, 66).
constexpr int ACC = 67;

// ---------------------------------------------------------------- errors --
tc_status fail(tc_status s, const std::string& msg);
tc_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define TC_CUDA(call)                                                      \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return ::tc::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

// Stream-ordered allocation from the library's own memory pool (kept
// resident between calls, so repeated builds/censuses do not remap memory).
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

// -------------------------------------------------------------- graph set --
// Device storage for G >= 1 graphs built together.  Vertices of all graphs
// are concatenated: graph g owns global rows voff[g] .. voff[g+1]-1, while the
// neighbour ids stored in adj are LOCAL to the graph.
struct GraphSet {
    int32_t G = 0;
    int64_t total_n = 0;
    int64_t nnz = 0;           // adjacency entries (2 * dyads over all graphs)
    int64_t adj_cap = 0;       // allocated entries excluding the padding
    int64_t* row_ptr = nullptr;    // [total_n + 1], global offsets into adj
    uint32_t* adj = nullptr;       // [adj_cap + ADJ_PAD]
    int32_t* deg = nullptr;        // [total_n]
    int32_t* vtag = nullptr;       // [3 * total_n]: per vertex #out-only, #in-only, #mutual nbrs
    int32_t* split = nullptr;      // [total_n]: entries of row x below x (its first entry above x)
    int32_t* arow = nullptr;       // [adj_cap]: global row of each adjacency entry
    int32_t max_deg = 0;           // largest degree over all graphs
    std::vector<int64_t> voff;     // host [G+1]
    std::vector<tc_graph_stats_t> stats;  // host [G]
    int64_t max_n = 0;

    // census work space, grown on demand
    void* ws = nullptr;
    size_t ws_bytes = 0;

    ~GraphSet();
};

// Packed FP16 cost-model weights installed on the current device (or null).
const void* cost_model_weights();

// tri_path = TC_TRI_AUTO: for each graph of gidx, merge[i] = 1 when it takes
// the merge path, 0 the forward path (installed path model, else the
// degree-skew rule).
tc_status path_route(const GraphSet& set, const std::vector<int32_t>& gidx, std::vector<uint8_t>& merge,
                     cudaStream_t st);

}  // namespace tc

struct tc_graph_s {
    std::shared_ptr<tc::GraphSet> set;
    int32_t index = 0;
};
