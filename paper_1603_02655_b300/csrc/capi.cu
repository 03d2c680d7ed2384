// C-ABI plumbing: status strings, the thread-local last error, the device
// memory pool, graph handles.
#include <cstdio>
#include <mutex>

#include "tc_internal.cuh"

namespace tc {

static thread_local std::string g_last_error;

tc_status fail(tc_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

tc_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s failed: %s (%s) at %s:%d", what, cudaGetErrorName(e),
             cudaGetErrorString(e), file, line);
    g_last_error = buf;
    cudaGetLastError();  // clear a non-sticky error
    return e == cudaErrorMemoryAllocation ? TC_ERR_OOM : TC_ERR_CUDA;
}

// One pool per device, owned by the library, with an unlimited release
// threshold so freed blocks stay mapped for the next call.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];
static bool g_pool_ok[64];

static cudaMemPool_t pool_for_current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool_ok[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
        g_pool[dev] = p;
        g_pool_ok[dev] = true;
    }
    return g_pool[dev];
}

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    cudaMemPool_t pool = pool_for_current_device();
    if (!pool) return cudaErrorInitializationError;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

void dev_free(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

GraphSet::~GraphSet() {
    // the caller of tc_graph_free has synchronised the device
    dev_free(row_ptr, 0);
    dev_free(adj, 0);
    dev_free(deg, 0);
    dev_free(vtag, 0);
    dev_free(split, 0);
    dev_free(arow, 0);
    dev_free(ws, 0);
    cudaStreamSynchronize(0);
}

}  // namespace tc

extern "C" {

const char* tc_status_str(tc_status s) {
    switch (s) {
        case TC_OK: return "TC_OK";
        case TC_ERR_ARG: return "TC_ERR_ARG: invalid argument";
        case TC_ERR_ID_RANGE: return "TC_ERR_ID_RANGE: arc endpoint outside [0, n)";
        case TC_ERR_OOM: return "TC_ERR_OOM: device allocation failed";
        case TC_ERR_CUDA: return "TC_ERR_CUDA: CUDA runtime error";
        case TC_ERR_TIMEOUT: return "TC_ERR_TIMEOUT: bounded device wait ran out";
        case TC_ERR_UNSUPPORTED: return "TC_ERR_UNSUPPORTED: size or feature not supported";
    }
    return "unknown tc_status";
}

const char* tc_last_error(void) { return tc::g_last_error.c_str(); }

tc_status tc_opts_default(tc_opts* o) {
    if (!o) return tc::fail(TC_ERR_ARG, "tc_opts_default: null");
    *o = tc_opts{};
    o->bin_mode = TC_BIN_HEURISTIC;
    o->thr_thread = 192;
    o->thr_warp = 256;
    o->chunk = 1024;
    o->stream_max = 1 << 30;
    o->persistent = 0;
    o->hub_ratio = 1;
    o->own_min = 128;
    o->tri_path = TC_TRI_AUTO;
    o->fwd_big = 64;
    return TC_OK;
}

tc_status tc_graph_stats(tc_graph g, tc_graph_stats_t* out) {
    if (!g || !out) return tc::fail(TC_ERR_ARG, "tc_graph_stats: null argument");
    *out = g->set->stats[(size_t)g->index];
    return TC_OK;
}

tc_status tc_graph_export(tc_graph g, int64_t* row_ptr, uint32_t* adj) {
    if (!g || !row_ptr || !adj) return tc::fail(TC_ERR_ARG, "tc_graph_export: null argument");
    const tc::GraphSet& s = *g->set;
    const int64_t v0 = s.voff[(size_t)g->index], v1 = s.voff[(size_t)g->index + 1];
    TC_CUDA(cudaDeviceSynchronize());
    TC_CUDA(cudaMemcpy(row_ptr, s.row_ptr + v0, sizeof(int64_t) * (size_t)(v1 - v0 + 1),
                       cudaMemcpyDeviceToHost));
    const int64_t base = row_ptr[0];
    for (int64_t i = 0; i <= v1 - v0; ++i) row_ptr[i] -= base;
    const int64_t cnt = row_ptr[v1 - v0];
    if (cnt > 0)
        TC_CUDA(cudaMemcpy(adj, s.adj + base, sizeof(uint32_t) * (size_t)cnt,
                           cudaMemcpyDeviceToHost));
    return TC_OK;
}

void tc_graph_free(tc_graph g) {
    if (!g) return;
    cudaDeviceSynchronize();
    delete g;
}

}  // extern "C"
