// tc_graph_build / tc_graph_build_batched: arc lists -> tagged combined CRS.
//
// The thesis builds, on the host, one CRS for out-arcs E(u) and one for the
// undirected neighbourhoods N(u) (Sec. 5.1.1).  Here both are one device
// array: row x holds every neighbour y of x once, as (y << 2) | tag with tag
// bit0 = arc x->y and bit1 = arc y->x, sorted by y.  The census then reads
// IsEdge and IsNeighbour from the tags of the merge instead of searching.
//
// Steps (all on the device, on the caller's stream):
//   1 keys: each arc x->y emits one canonical key (row min(x,y), nbr
//     max(x,y), tag seen from the lower endpoint); self-loops emit a sentinel
//     key that sorts last; ids are range-checked.
//   2 a radix sort of the 64-bit keys (library primitive: CUB): each dyad
//     once, in (lower, higher) order.
//   3 run heads over (lower, higher); an exclusive scan numbers the dyads.
//   4 each run is a dyad (the OR of its tags): its upper entry (row lower) in
//     dyad order, its lower entry (row higher) for the next sort; per-row
//     counts of upper and lower entries and of tags.
//   5 a stable radix sort of the lower entries by row (32-bit keys, the
//     library again): each row's lower entries by ascending neighbour.
//   6 scans of the counts -> row_ptr; each row is its lower entries, then its
//     upper ones (so a row's split point is its lower count); per-graph
//     statistics (arcs, dyads, mutual, merged entries = sum d^2, max degree).
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <cstring>

#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr uint64_t KEY_SENT = ~0ull;

__device__ __forceinline__ int find_graph(const int64_t* off, int G, int64_t i) {
    // largest g with off[g] <= i
    int lo = 0, hi = G - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_dyad_keys(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                            const int64_t* __restrict__ arc_off, const int64_t* __restrict__ voff, int G, int sh,
                            bool undirected, uint64_t* __restrict__ keys, int* __restrict__ err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int g = G == 1 ? 0 : find_graph(arc_off, G, i);
        const int64_t base = voff[g], n = voff[g + 1] - base;
        const int32_t s = src[i], d = dst[i];
        uint64_t k = KEY_SENT;
        if (s < 0 || s >= n || d < 0 || d >= n) {
            atomicOr(err, 1);
        } else if (s != d) {
            const int32_t lo = min(s, d), hi = max(s, d);
            // tag seen from the lower endpoint: bit0 = arc lo->hi, bit1 = hi->lo
            const uint32_t tag = undirected ? 3u : (s < d ? 1u : 2u);
            k = ((uint64_t)(base + lo) << sh) | ((uint64_t)hi << 2) | tag;
        }
        keys[i] = k;
    }
}

__global__ void k_heads(const uint64_t* __restrict__ k, int64_t N, int32_t* __restrict__ head) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t a = k[i];
        head[i] = (a != KEY_SENT) && (i == 0 || (k[i - 1] >> 2) != (a >> 2));
    }
}

__device__ __forceinline__ uint32_t tag_swap(uint32_t t) { return ((t & 1u) << 1) | (t >> 1); }

// One thread per sorted key; the first key of each (lower, higher) run is a
// dyad <u,v> with the OR of the run's tags: dyad j gets the upper entry
// (row u, v << 2 | tag) and the lower entry (row v, u << 2 | swapped tag).
// Counts per row: upper and lower entries, entries of each tag (atomics
// aggregated over a warp's lanes with the same row u, resp. row u and tag:
// sorted keys keep them in neighbouring lanes).
__global__ void k_dyads(const uint64_t* __restrict__ k, int64_t M, const int32_t* __restrict__ head,
                        const int32_t* __restrict__ dpos, int sh, uint32_t nbr_mask, const int64_t* __restrict__ voff,
                        int G, int32_t* __restrict__ up_row, uint32_t* __restrict__ up_val,
                        uint32_t* __restrict__ lo_key, uint32_t* __restrict__ lo_val, int32_t* __restrict__ cnt_up,
                        int32_t* __restrict__ cnt_lo, int32_t* __restrict__ vtag) {
    const int lane = threadIdx.x & 31;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < M; i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;  // whole warps iterate together
        const bool is_head = i < M && head[i];
        uint64_t u = ~0ull;
        uint32_t tag = 0;
        if (is_head) {
            const uint64_t key = k[i] >> 2;
            for (int64_t j = i; j < M && (k[j] >> 2) == key; ++j) tag |= (uint32_t)(k[j] & 3u);
            u = k[i] >> sh;
            const uint32_t vl = (uint32_t)(key & nbr_mask);
            const int64_t base = G == 1 ? 0 : voff[find_graph(voff, G, (int64_t)u)];
            const uint64_t v = (uint64_t)base + vl;
            const uint32_t ul = (uint32_t)(u - (uint64_t)base);
            const int32_t j = dpos[i];
            up_row[j] = (int32_t)u;
            up_val[j] = (vl << 2) | tag;
            lo_key[j] = (uint32_t)v;
            lo_val[j] = (ul << 2) | tag_swap(tag);
            atomicAdd(&cnt_lo[v], 1);
            atomicAdd(&vtag[3 * v + tag_swap(tag) - 1], 1);
        }
        const unsigned same_row = __match_any_sync(0xffffffffu, u);
        const unsigned same_tag = __match_any_sync(0xffffffffu, (u << 2) | tag);
        if (is_head && lane == __ffs(same_row) - 1) atomicAdd(&cnt_up[u], __popc(same_row));
        if (is_head && lane == __ffs(same_tag) - 1) atomicAdd(&vtag[3 * u + tag - 1], __popc(same_tag));
    }
}

__global__ void k_row_counts(const int32_t* __restrict__ cnt_lo, const int32_t* __restrict__ cnt_up, int64_t n,
                             unsigned long long* __restrict__ cnt) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        cnt[x] = (unsigned long long)(cnt_lo[x] + cnt_up[x]);
}

// Lower entries (sorted by row, then neighbour) to the front of their rows;
// lpre = exclusive scan of the lower counts (each row's first sorted entry).
__global__ void k_place_lo(const uint32_t* __restrict__ key, const uint32_t* __restrict__ val, int64_t D,
                           const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ lpre,
                           uint32_t* __restrict__ adj, int32_t* __restrict__ arow) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < D; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = key[j];
        const int64_t p = row_ptr[v] + (j - lpre[v]);
        adj[p] = val[j];
        arow[p] = (int32_t)v;
    }
}

// Upper entries (in dyad order: by row, then neighbour) after the lower ones.
__global__ void k_place_up(const int32_t* __restrict__ row, const uint32_t* __restrict__ val, int64_t D,
                           const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ cnt_lo,
                           const int32_t* __restrict__ upre, uint32_t* __restrict__ adj, int32_t* __restrict__ arow) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < D; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = row[j];
        const int64_t p = row_ptr[u] + cnt_lo[u] + (j - upre[u]);
        adj[p] = val[j];
        arow[p] = u;
    }
}

__global__ void k_fill_sent(uint32_t* __restrict__ p, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = SENT;
}

// Thread per row: degree, and per-graph statistics from the row's degree and tag
// counts (k_dyads counted the tags); a warp whose rows lie in one graph adds
// its sums with one atomic each (one graph: a block adds its sums once).
__global__ void k_rowstats(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ vtag,
                           const int64_t* __restrict__ voff, int G, int64_t total_n, int32_t* __restrict__ deg,
                           unsigned long long* __restrict__ gstat /* [G][6] */) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    if (G == 1) {  // one graph: per-thread sums, then one atomic per block and statistic
        unsigned long long v[5] = {0, 0, 0, 0, 0};  // arcs, degree, 2 x mutual, degree^2, max degree
        for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total_n;
             x += (int64_t)gridDim.x * blockDim.x) {
            const int64_t b = row_ptr[x];
            const unsigned long long d = (unsigned long long)(row_ptr[x + 1] - b);
            deg[x] = (int32_t)d;
            const int c1 = vtag[3 * x], c3 = vtag[3 * x + 2];
            v[0] += (unsigned long long)(c1 + c3);
            v[1] += d;
            v[2] += (unsigned long long)c3;
            v[3] += d * d;
            v[4] = v[4] > d ? v[4] : d;
        }
        __shared__ unsigned long long part[5][32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            for (int q = 0; q < 4; ++q) v[q] += __shfl_xor_sync(full, v[q], o);
            const unsigned long long t = __shfl_xor_sync(full, v[4], o);
            v[4] = v[4] > t ? v[4] : t;
        }
        const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        if (lane == 0)
            for (int q = 0; q < 5; ++q) part[q][warp] = v[q];
        __syncthreads();
        if (threadIdx.x < 5) {
            const int q = threadIdx.x;
            unsigned long long a = 0;
            for (int w = 0; w < nw; ++w) a = q == 4 ? (a > part[q][w] ? a : part[q][w]) : a + part[q][w];
            if (a) {
                if (q == 4) atomicMax(gstat + 4, a);
                else atomicAdd(gstat + q, a);
            }
        }
        return;
    }
    for (int64_t x0 = blockIdx.x * (int64_t)blockDim.x; x0 < total_n; x0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = x0 + threadIdx.x;
        const bool valid = x < total_n;
        unsigned long long v[5] = {0, 0, 0, 0, 0};  // arcs, degree, 2 x mutual, degree^2, max degree
        int g = 0;
        if (valid) {
            const int64_t b = row_ptr[x];
            const unsigned long long d = (unsigned long long)(row_ptr[x + 1] - b);
            deg[x] = (int32_t)d;
            g = G == 1 ? 0 : find_graph(voff, G, x);
            const int c1 = vtag[3 * x], c3 = vtag[3 * x + 2];
            v[0] = (unsigned long long)(c1 + c3);
            v[1] = d;
            v[2] = (unsigned long long)c3;
            v[3] = d * d;
            v[4] = d;
        }
        const int g0 = __shfl_sync(full, g, 0);
        if (__all_sync(full, !valid || g == g0)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                for (int q = 0; q < 4; ++q) v[q] += __shfl_xor_sync(full, v[q], o);
                const unsigned long long t = __shfl_xor_sync(full, v[4], o);
                v[4] = v[4] > t ? v[4] : t;
            }
            if (lane == 0) {
                unsigned long long* st = gstat + 6 * (size_t)g0;
                for (int q = 0; q < 4; ++q)
                    if (v[q]) atomicAdd(st + q, v[q]);
                if (v[4]) atomicMax(st + 4, v[4]);
            }
        } else if (valid) {
            unsigned long long* st = gstat + 6 * (size_t)g;
            for (int q = 0; q < 4; ++q)
                if (v[q]) atomicAdd(st + q, v[q]);
            if (v[4]) atomicMax(st + 4, v[4]);
        }
    }
}

int bits_for(uint64_t x) {  // smallest b with x < 2^b
    int b = 0;
    while (b < 64 && (x >> b) != 0) ++b;
    return b;
}

struct Scratch {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit Scratch(cudaStream_t st) : s(st) {}
    template <class T>
    cudaError_t get(T** p, size_t count) {
        void* q = nullptr;
        cudaError_t e = dev_alloc(&q, count * sizeof(T), s);
        if (e == cudaSuccess) ptrs.push_back(q);
        *p = (T*)q;
        return e;
    }
    ~Scratch() {
        for (void* p : ptrs) dev_free(p, s);
    }
};

// out = exclusive scan of in (count < 2^31 items, sums < 2^31).
tc_status scan_i32(Scratch& S, const int32_t* in, int32_t* out, int64_t count, cudaStream_t st) {
    if (count <= 0) return TC_OK;
    size_t bytes = 0;
    TC_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, bytes, in, out, (int)count, st));
    void* tmp = nullptr;
    TC_CUDA(S.get((char**)&tmp, bytes));
    TC_CUDA(cub::DeviceScan::ExclusiveSum(tmp, bytes, in, out, (int)count, st));
    return TC_OK;
}

int grid_for(int64_t work, int threads) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t g = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)sms * 16));
}

tc_status build_impl(int32_t G, const int32_t* ns, const int64_t* arc_off, const int32_t* src,
                     const int32_t* dst, uint32_t flags, cudaStream_t st, tc_graph* outs) {
    if (G < 1 || !ns || !arc_off || !outs) return fail(TC_ERR_ARG, "graph build: null argument or G < 1");
    if (flags & ~(TC_DEVICE_PTRS | TC_UNDIRECTED)) return fail(TC_ERR_ARG, "graph build: unknown flag");
    const bool undirected = (flags & TC_UNDIRECTED) != 0;  // an edge is both arcs
    std::vector<int64_t> voff((size_t)G + 1, 0), aoff((size_t)G + 1, 0);
    int64_t max_n = 0;
    for (int32_t g = 0; g < G; ++g) {
        if (ns[g] < 0) return fail(TC_ERR_ARG, "graph build: n < 0");
        if (ns[g] >= (1 << 30)) return fail(TC_ERR_UNSUPPORTED, "graph build: n must be < 2^30");
        voff[g + 1] = voff[g] + ns[g];
        max_n = std::max<int64_t>(max_n, ns[g]);
    }
    std::memcpy(aoff.data(), arc_off, sizeof(int64_t) * ((size_t)G + 1));
    if (aoff[0] != 0) return fail(TC_ERR_ARG, "graph build: arc_off[0] must be 0");
    for (int32_t g = 0; g < G; ++g)
        if (aoff[g + 1] < aoff[g]) return fail(TC_ERR_ARG, "graph build: arc offsets decrease");
    const int64_t m = aoff[G];
    const int64_t total_n = voff[G];
    if (total_n >= ((int64_t)1 << 31)) return fail(TC_ERR_UNSUPPORTED, "graph build: total vertices must be < 2^31");
    if (m > 0 && (!src || !dst)) return fail(TC_ERR_ARG, "graph build: null arc arrays");
    if (2 * m >= ((int64_t)1 << 31) - 1) return fail(TC_ERR_UNSUPPORTED, "graph build: m must be < 2^30");
    const int nb = std::max(1, bits_for((uint64_t)std::max<int64_t>(max_n - 1, 0)));
    const int rb = std::max(1, bits_for((uint64_t)total_n));  // total_n itself < 2^rb: no real key is all ones
    const int sh = nb + 2;
    if (sh + rb > 64) return fail(TC_ERR_UNSUPPORTED, "graph build: key does not fit 64 bits");

    auto set = std::make_shared<GraphSet>();
    set->G = G;
    set->total_n = total_n;
    set->voff = voff;
    set->max_n = max_n;
    set->stats.assign((size_t)G, tc_graph_stats_t{});
    const int64_t N = 2 * m;
    set->adj_cap = N;
    TC_CUDA(dev_alloc((void**)&set->row_ptr, sizeof(int64_t) * (size_t)(total_n + 1), st));
    TC_CUDA(dev_alloc((void**)&set->adj, sizeof(uint32_t) * (size_t)(N + ADJ_PAD), st));
    TC_CUDA(dev_alloc((void**)&set->deg, sizeof(int32_t) * (size_t)std::max<int64_t>(total_n, 1), st));
    TC_CUDA(dev_alloc((void**)&set->vtag, sizeof(int32_t) * 3 * (size_t)std::max<int64_t>(total_n, 1), st));
    TC_CUDA(cudaMemsetAsync(set->vtag, 0, sizeof(int32_t) * 3 * (size_t)std::max<int64_t>(total_n, 1), st));
    TC_CUDA(dev_alloc((void**)&set->split, sizeof(int32_t) * (size_t)std::max<int64_t>(total_n, 1), st));
    // split = the row's lower count, counted by k_dyads
    TC_CUDA(cudaMemsetAsync(set->split, 0, sizeof(int32_t) * (size_t)std::max<int64_t>(total_n, 1), st));
    TC_CUDA(dev_alloc((void**)&set->arow, sizeof(int32_t) * (size_t)std::max<int64_t>(N, 1), st));

    Scratch S(st);
    int32_t *d_src = nullptr, *d_dst = nullptr;
    if (m > 0) {
        if (flags & TC_DEVICE_PTRS) {
            d_src = const_cast<int32_t*>(src);
            d_dst = const_cast<int32_t*>(dst);
        } else {
            TC_CUDA(S.get(&d_src, (size_t)m));
            TC_CUDA(S.get(&d_dst, (size_t)m));
            TC_CUDA(cudaMemcpyAsync(d_src, src, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, st));
            TC_CUDA(cudaMemcpyAsync(d_dst, dst, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, st));
        }
    }
    int64_t *d_aoff = nullptr, *d_voff = nullptr;
    int* d_err = nullptr;
    unsigned long long *d_cnt = nullptr, *d_gstat = nullptr;
    TC_CUDA(S.get(&d_aoff, (size_t)G + 1));
    TC_CUDA(S.get(&d_voff, (size_t)G + 1));
    TC_CUDA(S.get(&d_err, 1));
    TC_CUDA(S.get(&d_cnt, (size_t)total_n + 1));
    TC_CUDA(S.get(&d_gstat, 6 * (size_t)G + 8));
    TC_CUDA(cudaMemcpyAsync(d_aoff, aoff.data(), sizeof(int64_t) * ((size_t)G + 1), cudaMemcpyHostToDevice, st));
    TC_CUDA(cudaMemcpyAsync(d_voff, voff.data(), sizeof(int64_t) * ((size_t)G + 1), cudaMemcpyHostToDevice, st));
    TC_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    TC_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long) * ((size_t)total_n + 1), st));
    TC_CUDA(cudaMemsetAsync(d_gstat, 0, sizeof(unsigned long long) * (6 * (size_t)G + 8), st));

    int64_t nnz_host = 0;
    int32_t* cnt_up = nullptr;
    TC_CUDA(S.get(&cnt_up, (size_t)std::max<int64_t>(total_n, 1)));
    TC_CUDA(cudaMemsetAsync(cnt_up, 0, sizeof(int32_t) * (size_t)std::max<int64_t>(total_n, 1), st));
    int64_t D = 0;
    int32_t* up_row = nullptr;
    uint32_t *up_val = nullptr, *lk[2] = {nullptr, nullptr}, *lv[2] = {nullptr, nullptr};
    if (m > 0) {
        uint64_t *k0 = nullptr, *k1 = nullptr;
        int32_t *head = nullptr, *dpos = nullptr;
        TC_CUDA(S.get(&k0, (size_t)m));
        TC_CUDA(S.get(&k1, (size_t)m));
        TC_CUDA(S.get(&head, (size_t)m));
        TC_CUDA(S.get(&dpos, (size_t)m));
        k_dyad_keys<<<grid_for(m, 256), 256, 0, st>>>(d_src, d_dst, m, d_aoff, d_voff, G, sh, undirected, k0, d_err);
        TC_CUDA(cudaGetLastError());
        cub::DoubleBuffer<uint64_t> db(k0, k1);
        size_t tmp_bytes = 0;
        TC_CUDA(cub::DeviceRadixSort::SortKeys(nullptr, tmp_bytes, db, (int)m, 2, sh + rb, st));
        void* tmp = nullptr;
        TC_CUDA(S.get((char**)&tmp, tmp_bytes));
        TC_CUDA(cub::DeviceRadixSort::SortKeys(tmp, tmp_bytes, db, (int)m, 2, sh + rb, st));
        const uint64_t* ks = db.Current();
        k_heads<<<grid_for(m, 256), 256, 0, st>>>(ks, m, head);
        TC_CUDA(cudaGetLastError());
        if (tc_status s2 = scan_i32(S, head, dpos, m, st); s2 != TC_OK) return s2;
        int32_t last_pos = 0, last_head = 0;
        TC_CUDA(cudaMemcpyAsync(&last_pos, dpos + m - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaMemcpyAsync(&last_head, head + m - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
        D = (int64_t)last_pos + last_head;
        TC_CUDA(S.get(&up_row, (size_t)D));
        TC_CUDA(S.get(&up_val, (size_t)D));
        for (int b = 0; b < 2; ++b) {
            TC_CUDA(S.get(&lk[b], (size_t)D));
            TC_CUDA(S.get(&lv[b], (size_t)D));
        }
        k_dyads<<<grid_for(m, 256), 256, 0, st>>>(ks, m, head, dpos, sh, (uint32_t)((1ull << nb) - 1), d_voff, G,
                                                  up_row, up_val, lk[0], lv[0], cnt_up, set->split, set->vtag);
        TC_CUDA(cudaGetLastError());
    }
    nnz_host = 2 * D;
    set->nnz = nnz_host;
    // row_ptr = exclusive scan of the row counts (total_n + 1 items, last count 0)
    if (total_n > 0) {
        k_row_counts<<<grid_for(total_n, 256), 256, 0, st>>>(set->split, cnt_up, total_n, d_cnt);
        TC_CUDA(cudaGetLastError());
    }
    {
        size_t scan_bytes = 0;
        TC_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, d_cnt,
                                              (unsigned long long*)set->row_ptr, (int)(total_n + 1), st));
        void* tmp = nullptr;
        TC_CUDA(S.get((char**)&tmp, scan_bytes));
        TC_CUDA(cub::DeviceScan::ExclusiveSum(tmp, scan_bytes, d_cnt,
                                              (unsigned long long*)set->row_ptr, (int)(total_n + 1), st));
    }
    if (D > 0) {
        // lower entries sorted by row (stable: the dyad order keeps each row's
        // lower neighbours ascending)
        cub::DoubleBuffer<uint32_t> dk(lk[0], lk[1]), dv(lv[0], lv[1]);
        size_t tmp_bytes = 0;
        TC_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, dk, dv, (int)D, 0, rb, st));
        void* tmp = nullptr;
        TC_CUDA(S.get((char**)&tmp, tmp_bytes));
        TC_CUDA(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, dk, dv, (int)D, 0, rb, st));
        int32_t *lpre = nullptr, *upre = nullptr;
        TC_CUDA(S.get(&lpre, (size_t)total_n));
        TC_CUDA(S.get(&upre, (size_t)total_n));
        if (tc_status s2 = scan_i32(S, set->split, lpre, total_n, st); s2 != TC_OK) return s2;
        if (tc_status s2 = scan_i32(S, cnt_up, upre, total_n, st); s2 != TC_OK) return s2;
        k_place_lo<<<grid_for(D, 256), 256, 0, st>>>(dk.Current(), dv.Current(), D, set->row_ptr, lpre, set->adj,
                                                     set->arow);
        TC_CUDA(cudaGetLastError());
        k_place_up<<<grid_for(D, 256), 256, 0, st>>>(up_row, up_val, D, set->row_ptr, set->split, upre, set->adj,
                                                     set->arow);
        TC_CUDA(cudaGetLastError());
    }
    k_fill_sent<<<grid_for(ADJ_PAD + (N - nnz_host), 256), 256, 0, st>>>(set->adj + nnz_host,
                                                                        ADJ_PAD + (N - nnz_host));
    TC_CUDA(cudaGetLastError());
    if (total_n > 0) {
        k_rowstats<<<grid_for(total_n, 256), 256, 0, st>>>(set->row_ptr, set->vtag, d_voff, G, total_n, set->deg,
                                                          d_gstat);
        TC_CUDA(cudaGetLastError());
    }
    std::vector<unsigned long long> gstat(6 * (size_t)G);
    int err = 0;
    TC_CUDA(cudaMemcpyAsync(gstat.data(), d_gstat, sizeof(unsigned long long) * 6 * (size_t)G,
                            cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    if (err) return fail(TC_ERR_ID_RANGE, "graph build: an arc endpoint lies outside [0, n)");
    for (int32_t g = 0; g < G; ++g) {
        tc_graph_stats_t& s = set->stats[(size_t)g];
        const unsigned long long* x = gstat.data() + 6 * (size_t)g;
        s.n = ns[g];
        s.arcs = (int64_t)x[0];
        s.dyads = (int64_t)(x[1] / 2);
        s.mutual = (int64_t)(x[2] / 2);
        s.asym = s.dyads - s.mutual;
        s.merged_entries = (int64_t)x[3];
        s.max_degree = (int64_t)x[4];
        set->max_deg = std::max<int32_t>(set->max_deg, (int32_t)x[4]);
    }
    for (int32_t g = 0; g < G; ++g) {
        outs[g] = new tc_graph_s;
        outs[g]->set = set;
        outs[g]->index = g;
    }
    return TC_OK;
}

}  // namespace
}  // namespace tc

extern "C" {

tc_status tc_graph_build(int32_t n, const int32_t* src, const int32_t* dst, int64_t m, uint32_t flags,
                         void* stream, tc_graph* out) {
    if (!out) return tc::fail(TC_ERR_ARG, "tc_graph_build: out is null");
    *out = nullptr;
    if (n < 0 || m < 0) return tc::fail(TC_ERR_ARG, "tc_graph_build: negative size");
    int64_t off[2] = {0, m};
    try {
        return tc::build_impl(1, &n, off, src, dst, flags, (cudaStream_t)stream, out);
    } catch (const std::bad_alloc&) {
        return tc::fail(TC_ERR_OOM, "tc_graph_build: host allocation failed");
    } catch (...) {
        return tc::fail(TC_ERR_CUDA, "tc_graph_build: unexpected exception");
    }
}

tc_status tc_graph_build_batched(int32_t G, const int32_t* ns, const int64_t* arc_off, const int32_t* src,
                                 const int32_t* dst, uint32_t flags, void* stream, tc_graph* outs) {
    if (!outs) return tc::fail(TC_ERR_ARG, "tc_graph_build_batched: outs is null");
    try {
        return tc::build_impl(G, ns, arc_off, src, dst, flags, (cudaStream_t)stream, outs);
    } catch (const std::bad_alloc&) {
        return tc::fail(TC_ERR_OOM, "tc_graph_build_batched: host allocation failed");
    } catch (...) {
        return tc::fail(TC_ERR_CUDA, "tc_graph_build_batched: unexpected exception");
    }
}

}  // extern "C"
