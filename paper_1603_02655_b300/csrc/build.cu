// tc_graph_build / tc_graph_build_batched: arc lists -> tagged combined CRS.
//
// The thesis builds, on the host, one CRS for out-arcs E(u) and one for the
// undirected neighbourhoods N(u) (Sec. 5.1.1).  Here both are one device
// array: row x holds every neighbour y of x once, as (y << 2) | tag with tag
// bit0 = arc x->y and bit1 = arc y->x, sorted by y.  The census then reads
// IsEdge and IsNeighbour from the tags of the merge instead of searching.
//
// Every arc x->y (ids range-checked, self-loops dropped) gives the entry
// (y << 2) | 1 of row x and (x << 2) | 2 of row y.  The build sorts these
// entries in hand-written kernels (no library sort):
//   1 buckets of 2^b consecutive rows: each block of k_bkt_hist counts the
//     entries of its share of the arcs per bucket in shared memory; a scan
//     of the (bucket, block) counts gives every block its slots in every
//     bucket, and k_bkt_scatter writes the entries there (no global atomics;
//     an entry is packed into 32 bits when the ids allow it).
//   2 k_bkt_rows, a block per bucket: the bucket's entries are counted per
//     row and placed row by row in shared memory (each row gets its raw
//     segment of the bucket), then every row is sorted and its runs of one
//     neighbour are merged (OR of the tags): a row of at most smax (8, or
//     16 when rows average 12 raw entries or more) entries in one thread's
//     registers, one of at most WCH entries by one
//     warp (a bitonic network over registers and shuffles).  The distinct
//     words go to the start of the row's raw segment, with the row's
//     distinct count, tag counts and split point (entries below its own id).
//     A bucket with more than CAP entries places its rows in global memory
//     instead, and k_rows sorts them there.
//   3 rows of more than WCH entries (hub rows) are split by id range into
//     segments of about SUB_AVG entries (k_long_split), which warps sort in
//     registers (k_seg_sort); a segment longer than WCH (ids crowded into one
//     range) is sorted in CAP-word pieces in shared memory (k_big_sort) and
//     merged pairwise in global memory (k_merge_round).  Their runs are
//     counted per WCH-word tile (k_long_count).
//   4 a scan of the distinct counts gives row_ptr; k_compact and
//     k_long_write move the rows to their final places and write each
//     entry's row; k_rowstats adds the per-graph statistics (arcs, dyads,
//     mutual, merged entries = sum d^2, max degree).
// When the rows are too many for NB_MAX buckets of MAX_BROWS rows, step 1
// is replaced by a count and a placement with one global atomic per entry
// (k_arc_count, k_arc_scatter) and k_rows sorts every row.
#include <algorithm>
#include <cstring>

#include "scan.cuh"
#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr int SMALL_MAX = 16;   // rows sorted by one thread (at most; a build picks 8 or 16)
constexpr int MID_LONG = 64;    // warp-sorted rows taken first in a bucket
constexpr int WCH = 512;        // rows (and pieces) sorted by one warp
constexpr int CAP = 8192;       // words one block sorts in shared memory
constexpr int SPAD = WCH + WCH / 32;  // a warp's staging words (one pad word per 32)
constexpr int MAX_BROWS = 1024;       // rows per bucket (2^b, b <= MAX_BBITS)
constexpr int MAX_BBITS = 10;
constexpr int MIN_BBITS = 5;          // buckets of at least 32 rows
constexpr int NB_MAX = 16384;         // buckets
constexpr int PT_NT = 1024;           // threads of the partition kernels
constexpr int BS_NT = 512;            // threads of the block sorts
constexpr int BS_W = BS_NT / 32;
constexpr int RW_NT = 256;            // threads of k_rows
constexpr int RW_W = RW_NT / 32;
static_assert(BS_W * SPAD >= CAP, "the warps' staging areas double as the merge buffer");

__device__ __forceinline__ int find_graph(const int64_t* off, int G, int64_t i) {
    // largest g with off[g] <= i
    int lo = 0, hi = G - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int pad(int i) { return i + (i >> 5); }

// ------------------------------------------------------------ arcs -> rows

struct ArcIn {
    const int32_t* src;
    const int32_t* dst;
    int64_t m;
    const int64_t* arc_off;  // [G + 1]
    const int64_t* voff;     // [G + 1]
    int G;
};

// Global rows of arc i: 1 for an arc, 0 for a self-loop, -1 for an id
// outside [0, n).
__device__ __forceinline__ int arc_rows(const ArcIn& a, int64_t i, int64_t& x, int64_t& y, int32_t& s, int32_t& d) {
    const int g = a.G == 1 ? 0 : find_graph(a.arc_off, a.G, i);
    const int64_t base = a.voff[g], n = a.voff[g + 1] - base;
    s = a.src[i];
    d = a.dst[i];
    if (s < 0 || s >= n || d < 0 || d >= n) return -1;
    x = base + s;
    y = base + d;
    return s != d ? 1 : 0;
}

// A partition entry: {word, row within the bucket}, packed into 32 bits
// (row << (32 - b) | word) when every word fits below bit 32 - b.
template <bool PACK>
struct Ent {
    using T = uint2;
    static __device__ __forceinline__ T make(uint32_t w, uint32_t r, int) { return make_uint2(w, r); }
    static __device__ __forceinline__ uint32_t row(T e, int) { return e.y; }
    static __device__ __forceinline__ uint32_t word(T e, int) { return e.x; }
};
template <>
struct Ent<true> {
    using T = uint32_t;
    static __device__ __forceinline__ T make(uint32_t w, uint32_t r, int b) { return (r << (32 - b)) | w; }
    static __device__ __forceinline__ uint32_t row(T e, int b) { return e >> (32 - b); }
    static __device__ __forceinline__ uint32_t word(T e, int b) { return e & (0xffffffffu >> b); }
};

// Bucket path, step 1: the entries of block k's arcs per bucket, stored
// bucket-major (hist[bucket * nblk + k]) so that one scan orders them by
// bucket, then block.
__global__ void __launch_bounds__(PT_NT) k_bkt_hist(ArcIn a, int b, int NB, int nblk, int32_t* __restrict__ hist,
                                                    int* __restrict__ err) {
    extern __shared__ int32_t h_cnt[];
    for (int k = threadIdx.x; k < NB; k += PT_NT) h_cnt[k] = 0;
    __syncthreads();
    const int64_t per = (a.m + nblk - 1) / nblk, i0 = blockIdx.x * per, i1 = min(a.m, i0 + per);
    int bad = 0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += PT_NT) {
        int64_t x, y;
        int32_t s, d;
        const int k = arc_rows(a, i, x, y, s, d);
        if (k < 0) bad = 1;
        if (k <= 0) continue;
        atomicAdd(h_cnt + (x >> b), 1);
        atomicAdd(h_cnt + (y >> b), 1);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, 1);
    for (int k = threadIdx.x; k < NB; k += PT_NT) hist[(int64_t)k * nblk + blockIdx.x] = h_cnt[k];
}

// Bucket path, step 1: every entry to a slot of its bucket; the order
// inside a bucket is arbitrary.
template <bool PACK>
__global__ void __launch_bounds__(PT_NT) k_bkt_scatter(ArcIn a, int b, int NB, int nblk, bool undirected,
                                                       const int32_t* __restrict__ S,
                                                       typename Ent<PACK>::T* __restrict__ ent) {
    extern __shared__ int32_t h_cur[];
    for (int k = threadIdx.x; k < NB; k += PT_NT) h_cur[k] = S[(int64_t)k * nblk + blockIdx.x];
    __syncthreads();
    const uint32_t mask = (1u << b) - 1u, tx = undirected ? 3u : 1u, ty = undirected ? 3u : 2u;
    const int64_t per = (a.m + nblk - 1) / nblk, i0 = blockIdx.x * per, i1 = min(a.m, i0 + per);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += PT_NT) {
        int64_t x, y;
        int32_t s, d;
        if (arc_rows(a, i, x, y, s, d) <= 0) continue;
        const int32_t px = atomicAdd(h_cur + (x >> b), 1);
        const int32_t py = atomicAdd(h_cur + (y >> b), 1);
        ent[px] = Ent<PACK>::make(((uint32_t)d << 2) | tx, (uint32_t)x & mask, b);
        ent[py] = Ent<PACK>::make(((uint32_t)s << 2) | ty, (uint32_t)y & mask, b);
    }
}

// Atomic path: raw row lengths.
__global__ void k_arc_count(ArcIn a, int32_t* __restrict__ cnt, int* __restrict__ err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.m; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t x, y;
        int32_t s, d;
        const int k = arc_rows(a, i, x, y, s, d);
        if (k < 0) atomicOr(err, 1);
        if (k <= 0) continue;
        atomicAdd(cnt + x, 1);
        atomicAdd(cnt + y, 1);
    }
}

// Atomic path: each entry takes a slot of its row's raw segment by counting
// the row's counter back down (so the counters end at zero).
__global__ void k_arc_scatter(ArcIn a, bool undirected, const int32_t* __restrict__ roff, int32_t* __restrict__ cnt,
                              uint32_t* __restrict__ tmp) {
    const uint32_t tx = undirected ? 3u : 1u, ty = undirected ? 3u : 2u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.m; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t x, y;
        int32_t s, d;
        if (arc_rows(a, i, x, y, s, d) <= 0) continue;
        const int32_t px = roff[x] + atomicSub(cnt + x, 1) - 1;
        const int32_t py = roff[y] + atomicSub(cnt + y, 1) - 1;
        tmp[px] = ((uint32_t)d << 2) | tx;
        tmp[py] = ((uint32_t)s << 2) | ty;
    }
}

// ------------------------------------------------------------ block scan
// Exclusive block-wide scan of v; *total gets the block's sum.  All threads
// of the block call it; it begins and ends with a barrier.
__device__ __forceinline__ long long block_excl_scan(long long v, long long* wsum, long long* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    __syncthreads();  // wsum may still be read by a previous call
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < nw) wsum[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    *total = wsum[nw - 1];
    return inc - v + (warp > 0 ? wsum[warp - 1] : 0);
}


// ------------------------------------------------------------ row sorting

// Bitonic network over P words held by one thread (P <= SMALL_MAX).
template <int P>
__device__ __forceinline__ void sort_thread(uint32_t (&v)[SMALL_MAX]) {
#pragma unroll
    for (int k = 2; k <= P; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < P; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    const uint32_t a = v[i], b = v[l];
                    const bool up = (i & k) == 0;
                    v[i] = up ? min(a, b) : max(a, b);
                    v[l] = up ? max(a, b) : min(a, b);
                }
            }
}

// Bitonic network over 32 * R words held by a warp, lane l holding words
// l*R .. l*R + R - 1 (blocked): distances below R stay in a lane, larger
// ones go through shuffles.
template <int R>
__device__ __forceinline__ void sort_warp(uint32_t (&v)[R], int lane) {
    constexpr int P = 32 * R;
#pragma unroll
    for (int k = 2; k <= P; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= R) {
                const int lj = j / R;
                const bool lower = (lane & lj) == 0;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const uint32_t a = v[r];
                    const uint32_t b = __shfl_xor_sync(0xffffffffu, a, lj);
                    const bool up = ((lane * R + r) & k) == 0;
                    v[r] = up == lower ? min(a, b) : max(a, b);
                }
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if ((r & j) == 0) {
                        const bool up = ((lane * R + r) & k) == 0;
                        const uint32_t a = v[r], b = v[r | j];
                        v[r] = up ? min(a, b) : max(a, b);
                        v[r | j] = up ? max(a, b) : min(a, b);
                    }
                }
            }
        }
    }
}

// Words s[0..len) of a warp's staging area (padded) -> sorted in place.
template <int R>
__device__ __forceinline__ void warp_sort_staged(uint32_t* s, int len, int lane) {
    uint32_t v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = lane * R + r;
        v[r] = i < len ? s[pad(i)] : SENT;
    }
    __syncwarp();
    sort_warp<R>(v, lane);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = lane * R + r;
        if (i < len) s[pad(i)] = v[r];
    }
    __syncwarp();
}

__device__ __forceinline__ void warp_sort_any(uint32_t* s, int len, int lane) {
    if (len <= 32) warp_sort_staged<1>(s, len, lane);
    else if (len <= 64) warp_sort_staged<2>(s, len, lane);
    else if (len <= 128) warp_sort_staged<4>(s, len, lane);
    else if (len <= 256) warp_sort_staged<8>(s, len, lane);
    else warp_sort_staged<16>(s, len, lane);
}

// One lane's PER consecutive outputs of the pairwise merge of sorted runs of
// W words (runs 2q and 2q+1 of src[0..L) -> dst): the tile of 32 * PER
// outputs starting at o0 (a multiple of 32 * PER); each lane finds its split
// by a merge-path search.  Ties take the left run first.
template <int PER, class T>
__device__ __forceinline__ void merge_part(const uint32_t* src, uint32_t* dst, T L, T W, T o0, int lane) {
    const T q0 = (o0 / (2 * W)) * (2 * W);
    const T na = min(W, L - q0);
    const T nb = max((T)0, min(W, L - q0 - W));
    const uint32_t* A = src + q0;
    const uint32_t* B = A + na;
    uint32_t* out = dst + q0;
    const T d0 = o0 - q0 + (T)lane * PER;
    const T d1 = min(min(o0 + (T)(32 * PER), L) - q0, d0 + (T)PER);
    if (d0 >= d1) return;
    if (nb == 0) {
        for (T d = d0; d < d1; ++d) out[d] = A[d];
        return;
    }
    T lo = max((T)0, d0 - nb), hi = min(d0, na);
    while (lo < hi) {  // the split of diagonal d0: lo words from A, d0 - lo from B
        const T mid = (lo + hi) >> 1;
        if (A[mid] <= B[d0 - 1 - mid]) lo = mid + 1;
        else hi = mid;
    }
    T a = lo, b = d0 - lo;
    for (T d = d0; d < d1; ++d) {
        const bool fromA = b >= nb || (a < na && A[a] <= B[b]);
        out[d] = fromA ? A[a++] : B[b++];
    }
}

// Sorts w[0..len) (len <= CAP) in shared memory with the whole block: warps
// sort WCH-word pieces through their staging areas (buf + warp * SPAD), then
// merge rounds double the sorted runs between w and buf.  Returns where the
// sorted words are.  Begins after and ends with a barrier.
__device__ uint32_t* block_sort(uint32_t* w, uint32_t* buf, int len) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t* s = buf + warp * SPAD;
    const int npc = (len + WCH - 1) / WCH;
    for (int q = warp; q < npc; q += nw) {
        const int q0 = q * WCH, ql = min(WCH, len - q0);
        for (int i = lane; i < ql; i += 32) s[pad(i)] = w[q0 + i];
        __syncwarp();
        warp_sort_any(s, ql, lane);
        for (int i = lane; i < ql; i += 32) w[q0 + i] = s[pad(i)];
        __syncwarp();
    }
    __syncthreads();
    uint32_t* src = w;
    uint32_t* dst = buf;
    for (int W = WCH; W < len; W <<= 1) {
        for (int t = warp; t < npc; t += nw) merge_part<WCH / 32, int>(src, dst, len, W, t * WCH, lane);
        __syncthreads();
        uint32_t* x = src;
        src = dst;
        dst = x;
    }
    return src;
}

struct RowOut {
    int32_t* ucnt;   // distinct entries per row
    int32_t* vtag;   // [3 * rows]: entries with tag 1, 2, 3
    int32_t* split;  // entries below the row's own id
};

__device__ __forceinline__ void row_stats(RowOut o, int64_t x, int k, int c1, int c2, int c3, int lo) {
    o.ucnt[x] = k;
    o.vtag[3 * x] = c1;
    o.vtag[3 * x + 1] = c2;
    o.vtag[3 * x + 2] = c3;
    o.split[x] = lo;
}

// A short row (L <= P words at `in`, any order, P <= SMALL_MAX) sorted in
// one thread's registers by a network of P words; its distinct words (OR of
// the tags of a run) go to out[0..).
template <int P>
__device__ __forceinline__ void thread_row(const uint32_t* in, int L, uint32_t* out, int64_t x, int64_t xl,
                                           RowOut o) {
    uint32_t v[SMALL_MAX];
#pragma unroll
    for (int i = 0; i < P; ++i) v[i] = i < L ? in[i] : SENT;
    sort_thread<P>(v);
    int k = 0, lo = 0, c1 = 0, c2 = 0, c3 = 0;
    uint32_t cur = v[0];
    auto emit = [&](uint32_t w) {
        out[k++] = w;
        const uint32_t t = w & 3u;
        c1 += t == 1u;
        c2 += t == 2u;
        c3 += t == 3u;
        lo += (int64_t)(w >> 2) < xl;
    };
#pragma unroll
    for (int i = 1; i < P; ++i) {
        if (i < L) {
            const uint32_t w = v[i];
            if ((w >> 2) == (cur >> 2)) cur |= w & 3u;
            else {
                emit(cur);
                cur = w;
            }
        }
    }
    emit(cur);
    row_stats(o, x, k, c1, c2, c3, lo);
}

// The same with the network sized by pmax, the longest short row of the
// warp (Ls = 0: no row; pmax <= SMAX).
template <int SMAX>
__device__ __forceinline__ void thread_row_any(const uint32_t* in, int Ls, int pmax, uint32_t* out, int64_t x,
                                               int64_t xl, RowOut o) {
    static_assert(SMAX == 8 || SMAX == 16, "short rows of up to 8 or 16 entries");
    if (Ls == 0) return;
    if (pmax <= 2) thread_row<2>(in, Ls, out, x, xl, o);
    else if (pmax <= 4) thread_row<4>(in, Ls, out, x, xl, o);
    else if (SMAX == 8 || pmax <= 8) thread_row<8>(in, Ls, out, x, xl, o);
    else thread_row<16>(in, Ls, out, x, xl, o);
}

// A sorted row in a warp's staging area s (padded, len words): one word per
// run of one neighbour (OR of its tags) to out[0..), and the row's counts.
__device__ __forceinline__ void warp_dedup(const uint32_t* s, int len, uint32_t* out, int64_t x, int64_t xl,
                                           RowOut o, int lane) {
    const unsigned full = 0xffffffffu;
    int k = 0, lo = 0, c1 = 0, c2 = 0, c3 = 0;
    for (int i0 = 0; i0 < len; i0 += 32) {
        const int i = i0 + lane;
        const uint32_t w = i < len ? s[pad(i)] : SENT;
        const bool head = i < len && (i == 0 || (s[pad(i - 1)] >> 2) != (w >> 2));
        uint32_t t = w & 3u;
        if (head)
            for (int j = i + 1; j < len && (s[pad(j)] >> 2) == (w >> 2); ++j) t |= s[pad(j)] & 3u;
        const unsigned hb = __ballot_sync(full, head);
        if (head) {
            out[k + __popc(hb & ((1u << lane) - 1u))] = (w & ~3u) | t;
            c1 += t == 1u;
            c2 += t == 2u;
            c3 += t == 3u;
            lo += (int64_t)(w >> 2) < xl;
        }
        k += __popc(hb);
    }
    c1 = __reduce_add_sync(full, c1);
    c2 = __reduce_add_sync(full, c2);
    c3 = __reduce_add_sync(full, c3);
    lo = __reduce_add_sync(full, lo);
    if (lane == 0) row_stats(o, x, k, c1, c2, c3, lo);
}

__device__ __forceinline__ int64_t local_id(const int64_t* voff, int G, int64_t x) {
    return x - (G == 1 ? 0 : voff[find_graph(voff, G, x)]);
}

// --------------------------------------------------- step 2: the buckets

struct LongOut {
    int32_t* ctr;    // [0] long rows, [1] segments, [2] longest crowded segment, [3] large buckets,
                     // [4] row tiles, [5] crowded-segment pieces, [6] crowded-segment tiles
    int32_t* lng;    // long rows
    uint4* tiles;    // {row, WCH-word tile, the row's first tile item, 0}
    uint8_t* lflag;  // 1 for a long row (placed by k_long_write)
    uint4* segs;     // {first word, length, row, 0}: the entries of one id range of a long row
    uint2* bpieces;  // {segment, CAP-word piece} of the segments longer than WCH
    uint2* btiles;   // {segment, WCH-word tile} of those segments
};

// A row of more than WCH entries goes to the long path: listed, flagged, and
// cut into WCH-word tiles for its final count and placement.
__device__ __forceinline__ void route_long(const LongOut& lo, int64_t x, int L) {
    lo.lng[atomicAdd(lo.ctr + 0, 1)] = (int32_t)x;
    lo.lflag[x] = 1;
    const int nt = (L + WCH - 1) / WCH;
    const int tb = atomicAdd(lo.ctr + 4, nt);
    for (int t = 0; t < nt; ++t) lo.tiles[tb + t] = make_uint4((uint32_t)x, (uint32_t)t, (uint32_t)tb, 0u);
}

struct BktArgs {
    const void* ent;   // Ent<PACK>::T entries
    const int32_t* S;  // bucket k's entries start at S[k * nblk]
    int nblk, NB, b;
    int64_t total_n;
    const int64_t* voff;
    int G;
    uint32_t* tmp;   // raw segments: each row's distinct words at its start
    int32_t* roff;   // [total_n + 1] raw row offsets
    RowOut o;
    int32_t* fbk;    // buckets too large for shared memory
    LongOut lo;
};

constexpr size_t BK_SMEM = sizeof(uint32_t) * ((size_t)CAP + (MAX_BROWS + 1) + MAX_BROWS + (size_t)BS_W * SPAD);

template <bool PACK, int SMAX>
__global__ void __launch_bounds__(BS_NT, 3) k_bkt_rows(BktArgs a) {
    using E = Ent<PACK>;
    const typename E::T* ent = static_cast<const typename E::T*>(a.ent);
    extern __shared__ __align__(16) uint32_t bk_sm[];
    uint32_t* words = bk_sm;                                 // the bucket's words, row by row
    int32_t* rpos = reinterpret_cast<int32_t*>(words + CAP);  // raw row offsets in the bucket, [nr + 1]
    int32_t* rcur = rpos + MAX_BROWS + 1;                     // row counters / cursors, then the middle rows
    uint32_t* stage = reinterpret_cast<uint32_t*>(rcur + MAX_BROWS);  // warp staging areas
    __shared__ long long wsum[32];
    __shared__ int nmid, nmid_lo, nlongs, mcur;
    __shared__ int longs[CAP / (WCH + 1) + 1];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
    for (int k = blockIdx.x; k < a.NB; k += gridDim.x) {
        const int32_t e0 = a.S[(int64_t)k * a.nblk];
        const int c = a.S[(int64_t)(k + 1) * a.nblk] - e0;
        const int64_t r0 = (int64_t)k << a.b;
        const int nr = (int)min((int64_t)1 << a.b, a.total_n - r0);
        for (int j = tid; j < nr; j += BS_NT) rcur[j] = 0;
        __syncthreads();
        for (int i = tid; i < c; i += BS_NT) atomicAdd(rcur + E::row(ent[e0 + i], a.b), 1);
        __syncthreads();
        {  // rpos = exclusive scan of the row counts, 2 rows per thread
            const int j0 = tid * 2;
            const int v0 = j0 < nr ? rcur[j0] : 0, v1 = j0 + 1 < nr ? rcur[j0 + 1] : 0;
            long long tot;
            const int run = (int)block_excl_scan(v0 + v1, wsum, &tot);
            if (j0 < nr) rpos[j0] = run;
            if (j0 + 1 < nr) rpos[j0 + 1] = run + v0;
            if (tid == 0) rpos[nr] = c;
        }
        __syncthreads();
        for (int j = tid; j < nr; j += BS_NT) {
            a.roff[r0 + j] = e0 + rpos[j];
            rcur[j] = rpos[j];
        }
        if (tid == 0 && r0 + nr == a.total_n) a.roff[a.total_n] = e0 + c;
        __syncthreads();
        if (c > CAP) {  // too large: the rows' raw segments in global memory, sorted by k_rows
            for (int i = tid; i < c; i += BS_NT) {
                const typename E::T e = ent[e0 + i];
                a.tmp[e0 + atomicAdd(rcur + E::row(e, a.b), 1)] = E::word(e, a.b);
            }
            if (tid == 0) a.fbk[atomicAdd(a.lo.ctr + 3, 1)] = k;
            __syncthreads();
            continue;
        }
        for (int i = tid; i < c; i += BS_NT) {
            const typename E::T e = ent[e0 + i];
            words[atomicAdd(rcur + E::row(e, a.b), 1)] = E::word(e, a.b);
        }
        if (tid == 0) {
            nmid = 0;
            nmid_lo = 0;
            nlongs = 0;
            mcur = 0;
        }
        __syncthreads();
        int32_t* mids = rcur;  // the cursors are spent
        // the rows for warps (those of more than MID_LONG entries from the
        // front, the others from the back, so that the longest are taken
        // first) and for the long path, listed
        for (int j = tid; j < nr; j += BS_NT) {
            const int L = rpos[j + 1] - rpos[j];
            if (L > MID_LONG && L <= WCH) mids[atomicAdd(&nmid, 1)] = j;
            else if (L > SMAX && L <= WCH) mids[nr - 1 - atomicAdd(&nmid_lo, 1)] = j;
            else if (L > WCH) longs[atomicAdd(&nlongs, 1)] = j;
        }
        __syncthreads();
        const int nhi = nmid, nall = nmid + nmid_lo;
        // short rows by their threads; a warp with none (a bucket of fewer
        // rows than threads) goes on to the middle rows at once
        for (int j0 = 0; j0 < nr; j0 += BS_NT) {
            const int j = j0 + tid;
            const int p = j < nr ? rpos[j] : 0;
            const int L = j < nr ? rpos[j + 1] - p : 0;
            const int Ls = L <= SMAX ? L : 0;
            const int pmax = __reduce_max_sync(full, Ls);
            if (pmax > 0)
                thread_row_any<SMAX>(words + p, Ls, pmax, a.tmp + e0 + p, r0 + j, local_id(a.voff, a.G, r0 + j),
                                     a.o);
        }
        uint32_t* s = stage + warp * SPAD;
        for (;;) {  // middle rows: a warp each
            int idx = 0;
            if (lane == 0) idx = atomicAdd(&mcur, 1);
            idx = __shfl_sync(full, idx, 0);
            if (idx >= nall) break;
            const int j = idx < nhi ? mids[idx] : mids[nr - 1 - (idx - nhi)];
            const int p = rpos[j], len = rpos[j + 1] - p;
            for (int i = lane; i < len; i += 32) s[pad(i)] = words[p + i];
            __syncwarp();
            warp_sort_any(s, len, lane);
            warp_dedup(s, len, a.tmp + e0 + p, r0 + j, local_id(a.voff, a.G, r0 + j), a.o, lane);
            __syncwarp();
        }
        for (int li = warp; li < nlongs; li += BS_W) {  // longer rows: raw words out, to the long path
            const int j = longs[li];
            const int p = rpos[j], len = rpos[j + 1] - p;
            for (int i = lane; i < len; i += 32) a.tmp[e0 + p + i] = words[p + i];
            if (lane == 0) route_long(a.lo, r0 + j, len);
        }
        __syncthreads();
    }
}

// ------------------------------------------- step 2b: rows in global memory

// Rows whose raw words lie in global memory (every row on the atomic path,
// else the rows of the buckets too large for shared memory), 32 consecutive
// rows per warp: rows of at most smax entries are sorted and merged by
// their lanes, rows of at most WCH entries by the whole warp one after
// another; longer rows go to the long path.
__global__ void __launch_bounds__(RW_NT) k_rows(const int32_t* __restrict__ roff, int64_t total_n,
                                                const int64_t* __restrict__ voff, int G, uint32_t* __restrict__ tmp,
                                                RowOut o, const int32_t* __restrict__ fbk, int b, LongOut lo,
                                                int smax) {
    __shared__ uint32_t stage[RW_W][SPAD];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* s = stage[warp];
    const int gsh = b - 5;  // warp groups per bucket: 2^gsh
    const int64_t groups = fbk ? ((int64_t)lo.ctr[3] << gsh) : (total_n + 31) >> 5;
    for (int64_t grp = blockIdx.x * (int64_t)RW_W + warp; grp < groups; grp += (int64_t)gridDim.x * RW_W) {
        const int64_t first =
            fbk ? ((int64_t)fbk[grp >> gsh] << b) + ((grp & ((1 << gsh) - 1)) << 5) : (grp << 5);
        const int64_t x = first + lane;
        const bool valid = x < total_n;
        const int32_t base = valid ? roff[x] : 0;
        const int L = valid ? roff[x + 1] - base : 0;
        const int64_t xl = valid ? local_id(voff, G, x) : 0;
        if (L > WCH) route_long(lo, x, L);
        const int Ls = L <= smax ? L : 0;
        const int pmax = __reduce_max_sync(full, Ls);
        if (pmax > 0) thread_row_any<SMALL_MAX>(tmp + base, Ls, pmax, tmp + base, x, xl, o);
        unsigned mid = __ballot_sync(full, L > smax && L <= WCH);
        while (mid) {
            const int src = __ffs(mid) - 1;
            mid &= mid - 1;
            const int len = __shfl_sync(full, L, src);
            const int32_t rb = __shfl_sync(full, base, src);
            const int64_t rx = __shfl_sync(full, x, src);
            const int64_t rxl = __shfl_sync(full, xl, src);
            for (int i = lane; i < len; i += 32) s[pad(i)] = tmp[rb + i];
            __syncwarp();
            warp_sort_any(s, len, lane);
            warp_dedup(s, len, tmp + rb, rx, rxl, o, lane);
            __syncwarp();
        }
    }
}

// ---------------------------------------------------- step 3: long rows

constexpr int SUB_AVG = 128;   // expected entries per id range of a long row
constexpr int SUB_MAX = 4096;  // id ranges per long row
constexpr int LS_NT = 512;

constexpr int LW_MAX = 4096;                 // long rows split by one warp
constexpr int LW_S = LW_MAX / (SUB_AVG / 2);  // their id ranges: fewer than 2 L / SUB_AVG + 1
static_assert(LW_S % 32 == 0, "whole counters per lane");

// Long rows, a block each (those of more than LW_MAX entries; a warp each
// for the others): the row's raw entries (tmp) distributed by id
// range into tmp2, ranges of 2^sh ids sized so that an even spread of the
// row's neighbours puts about SUB_AVG entries in each; every non-empty range
// becomes a segment.  Ranges are disjoint intervals of ids, so sorting each
// segment sorts the row.
__global__ void __launch_bounds__(LS_NT) k_long_split(const int32_t* __restrict__ roff,
                                                      const int64_t* __restrict__ voff, int G, LongOut lo,
                                                      const uint32_t* __restrict__ tmp, uint32_t* __restrict__ tmp2) {
    __shared__ int32_t cnt[SUB_MAX];
    __shared__ long long wsum[32];
    __shared__ int sbase;
    const int nlong = lo.ctr[0];
    for (int li = blockIdx.x; li < nlong; li += gridDim.x) {
        const int64_t x = lo.lng[li];
        const int32_t rb = roff[x];
        const int L = roff[x + 1] - rb;
        if (L <= LW_MAX) continue;  // split by one warp (k_long_split_w)
        const int g = G == 1 ? 0 : find_graph(voff, G, x);
        const int64_t n = voff[g + 1] - voff[g];
        int sh = 0;
        while (((int64_t)L << (sh + 1)) <= n * SUB_AVG) ++sh;
        while ((((n - 1) >> sh) + 1) > SUB_MAX) ++sh;
        const int S = (int)(((n - 1) >> sh) + 1);
        for (int j = threadIdx.x; j < S; j += LS_NT) cnt[j] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < L; i += LS_NT) atomicAdd(cnt + ((tmp[rb + i] >> 2) >> sh), 1);
        __syncthreads();
        const int j0 = threadIdx.x * 8;
        int v[8], sum = 0, ne = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            v[q] = j0 + q < S ? cnt[j0 + q] : 0;
            sum += v[q];
            ne += v[q] > 0;
        }
        long long tot;
        const long long ex = block_excl_scan(((long long)ne << 32) | (long long)sum, wsum, &tot);
        int run = (int)(ex & 0xffffffffll), rk = (int)(ex >> 32);
        if (threadIdx.x == 0) sbase = atomicAdd(lo.ctr + 1, (int)(tot >> 32));
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (j0 + q < S) {
                cnt[j0 + q] = run;  // now the range's cursor
                if (v[q] > 0) lo.segs[sbase + rk++] = make_uint4((uint32_t)(rb + run), (uint32_t)v[q], (uint32_t)x, 0u);
                run += v[q];
            }
        __syncthreads();
        for (int i = threadIdx.x; i < L; i += LS_NT) {
            const uint32_t w = tmp[rb + i];
            tmp2[rb + atomicAdd(cnt + ((w >> 2) >> sh), 1)] = w;
        }
        __syncthreads();
    }
}

// The same for the long rows of at most LW_MAX entries, a warp each: the
// range width follows the same rule, so a row has fewer than
// 2 L / SUB_AVG + 1 ranges (the width 2^sh is above n SUB_AVG / (2 L), or
// sh = 0 and n < 2 L / SUB_AVG), at most LW_S, counted in the warp's shared
// counters.
__global__ void __launch_bounds__(256) k_long_split_w(const int32_t* __restrict__ roff,
                                                      const int64_t* __restrict__ voff, int G, LongOut lo,
                                                      const uint32_t* __restrict__ tmp, uint32_t* __restrict__ tmp2) {
    constexpr int PL = LW_S / 32;  // counters per lane
    __shared__ int32_t cnt_all[8][LW_S];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t* cnt = cnt_all[warp];
    const int nlong = lo.ctr[0];
    for (int li = blockIdx.x * 8 + warp; li < nlong; li += gridDim.x * 8) {
        const int64_t x = lo.lng[li];
        const int32_t rb = roff[x];
        const int L = roff[x + 1] - rb;
        if (L > LW_MAX) continue;
        const int g = G == 1 ? 0 : find_graph(voff, G, x);
        const int64_t n = voff[g + 1] - voff[g];
        int sh = 0;
        while (((int64_t)L << (sh + 1)) <= n * SUB_AVG) ++sh;
        const int S = (int)(((n - 1) >> sh) + 1);  // <= LW_S (see above)
        for (int j = lane; j < LW_S; j += 32) cnt[j] = 0;
        __syncwarp();
        for (int i = lane; i < L; i += 32) atomicAdd(cnt + ((tmp[rb + i] >> 2) >> sh), 1);
        __syncwarp();
        int v[PL], sum = 0, ne = 0;
#pragma unroll
        for (int q = 0; q < PL; ++q) {
            const int j = lane * PL + q;
            v[q] = j < S ? cnt[j] : 0;
            sum += v[q];
            ne += v[q] > 0;
        }
        long long inc = ((long long)ne << 32) | (long long)sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(full, inc, o);
            if (lane >= o) inc += t;
        }
        const long long tot = __shfl_sync(full, inc, 31);
        const long long ex = inc - (((long long)ne << 32) | (long long)sum);
        int sbase = 0;
        if (lane == 0) sbase = atomicAdd(lo.ctr + 1, (int)(tot >> 32));
        sbase = __shfl_sync(full, sbase, 0);
        int run = (int)(ex & 0xffffffffll), rk = (int)(ex >> 32);
        __syncwarp();
#pragma unroll
        for (int q = 0; q < PL; ++q) {
            const int j = lane * PL + q;
            if (j < S) {
                cnt[j] = run;  // now the range's cursor
                if (v[q] > 0) lo.segs[sbase + rk++] = make_uint4((uint32_t)(rb + run), (uint32_t)v[q], (uint32_t)x, 0u);
                run += v[q];
            }
        }
        __syncwarp();
        for (int i = lane; i < L; i += 32) {
            const uint32_t w = tmp[rb + i];
            tmp2[rb + atomicAdd(cnt + ((w >> 2) >> sh), 1)] = w;
        }
        __syncwarp();
    }
}

// Segments, a warp each: one of at most WCH words sorted in registers (tmp2
// -> tmp); a longer one (ids crowded into one range) is listed with its
// CAP-word pieces and WCH-word tiles for k_big_sort and the merge rounds.
__global__ void __launch_bounds__(RW_NT) k_seg_sort(LongOut lo, const uint32_t* __restrict__ tmp2,
                                                    uint32_t* __restrict__ tmp) {
    __shared__ uint32_t stage[RW_W][SPAD];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* s = stage[warp];
    const int nseg = lo.ctr[1];
    for (int it = blockIdx.x * RW_W + warp; it < nseg; it += gridDim.x * RW_W) {
        const uint4 sg = lo.segs[it];
        const int len = (int)sg.y;
        if (len > WCH) {
            if (lane == 0) {
                const int np = (len + CAP - 1) / CAP, nt = (len + WCH - 1) / WCH;
                const int pb = atomicAdd(lo.ctr + 5, np);
                for (int q = 0; q < np; ++q) lo.bpieces[pb + q] = make_uint2((uint32_t)it, (uint32_t)q);
                const int tb = atomicAdd(lo.ctr + 6, nt);
                for (int t = 0; t < nt; ++t) lo.btiles[tb + t] = make_uint2((uint32_t)it, (uint32_t)t);
                atomicMax(lo.ctr + 2, len);
            }
            continue;
        }
        for (int i = lane; i < len; i += 32) s[pad(i)] = tmp2[sg.x + i];
        __syncwarp();
        warp_sort_any(s, len, lane);
        for (int i = lane; i < len; i += 32) tmp[sg.x + i] = s[pad(i)];
        __syncwarp();
    }
}

constexpr size_t LS_SMEM = sizeof(uint32_t) * ((size_t)CAP + (size_t)BS_W * SPAD);

// Crowded segments: each CAP-word piece sorted in shared memory, in tmp2.
__global__ void __launch_bounds__(BS_NT) k_big_sort(LongOut lo, uint32_t* __restrict__ tmp2) {
    extern __shared__ __align__(16) uint32_t ls_sm[];
    uint32_t* w = ls_sm;
    uint32_t* buf = ls_sm + CAP;
    const int np = lo.ctr[5];
    for (int it = blockIdx.x; it < np; it += gridDim.x) {
        const uint2 pc = lo.bpieces[it];
        const uint4 sg = lo.segs[pc.x];
        const int q0 = (int)pc.y * CAP, len = min(CAP, (int)sg.y - q0);
        uint32_t* seg = tmp2 + sg.x + q0;
        for (int i = threadIdx.x; i < len; i += BS_NT) w[i] = seg[i];
        __syncthreads();
        const uint32_t* srt = block_sort(w, buf, len);
        for (int i = threadIdx.x; i < len; i += BS_NT) seg[i] = srt[i];
        __syncthreads();
    }
}

__device__ __forceinline__ int big_rounds(int len) {
    const int np = (len + CAP - 1) / CAP;
    int r = 0;
    while ((1 << r) < np) ++r;
    return r;
}

// Round r of the crowded segments' merge: sorted runs of CAP << r words are
// merged pairwise (tmp2 -> tmp in even rounds, back in odd ones), a warp per
// WCH-word tile of a segment's output, each lane 16 words from its own
// merge-path split.  Segments already one run sit the round out; after the
// last round k_big_copy brings the ones that ended in tmp2 to tmp.
__global__ void __launch_bounds__(256) k_merge_round(LongOut lo, int r, const uint32_t* __restrict__ src,
                                                     uint32_t* __restrict__ dst) {
    const int lane = threadIdx.x & 31;
    const int nt = lo.ctr[6];
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int it = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < nt; it += nwarps) {
        const uint2 tl = lo.btiles[it];
        const uint4 sg = lo.segs[tl.x];
        const int len = (int)sg.y;
        if (big_rounds(len) <= r) continue;
        merge_part<WCH / 32, int>(src + sg.x, dst + sg.x, len, CAP << r, (int)tl.y * WCH, lane);
    }
}

__global__ void __launch_bounds__(256) k_big_copy(LongOut lo, const uint32_t* __restrict__ tmp2,
                                                  uint32_t* __restrict__ tmp) {
    const int lane = threadIdx.x & 31;
    const int nt = lo.ctr[6];
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int it = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < nt; it += nwarps) {
        const uint2 tl = lo.btiles[it];
        const uint4 sg = lo.segs[tl.x];
        const int len = (int)sg.y;
        if (big_rounds(len) & 1) continue;
        const int i1 = min(len, (int)(tl.y + 1) * WCH);
        for (int i = (int)tl.y * WCH + lane; i < i1; i += 32) tmp[sg.x + i] = tmp2[sg.x + i];
    }
}

// The sorted long rows (tmp): run heads of one WCH-word tile per warp,
// counted into the row's distinct count (and per tile into tcnt), tag
// counts and split point.
__global__ void __launch_bounds__(256) k_long_count(const int32_t* __restrict__ roff, LongOut lo,
                                                    const int64_t* __restrict__ voff, int G,
                                                    const uint32_t* __restrict__ tmp, RowOut o,
                                                    int32_t* __restrict__ tcnt) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nt = lo.ctr[4];
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int it = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < nt; it += nwarps) {
        const uint4 tl = lo.tiles[it];
        const int64_t x = tl.x;
        const int32_t rb = roff[x];
        const int L = roff[x + 1] - rb;
        const uint32_t* s = tmp + rb;
        const int64_t xl = local_id(voff, G, x);
        int k = 0, lw = 0, c1 = 0, c2 = 0, c3 = 0;
        const int i1 = min(L, (int)(tl.y + 1) * WCH);
        for (int i = (int)tl.y * WCH + lane; i < i1; i += 32) {
            const uint32_t w = s[i];
            if (i == 0 || (s[i - 1] >> 2) != (w >> 2)) {
                uint32_t t = w & 3u;
                for (int j = i + 1; j < L && (s[j] >> 2) == (w >> 2); ++j) t |= s[j] & 3u;
                ++k;
                c1 += t == 1u;
                c2 += t == 2u;
                c3 += t == 3u;
                lw += (int64_t)(w >> 2) < xl;
            }
        }
        k = __reduce_add_sync(full, k);
        c1 = __reduce_add_sync(full, c1);
        c2 = __reduce_add_sync(full, c2);
        c3 = __reduce_add_sync(full, c3);
        lw = __reduce_add_sync(full, lw);
        if (lane == 0) {
            tcnt[it] = k;
            atomicAdd(o.ucnt + x, k);
            if (c1) atomicAdd(o.vtag + 3 * x, c1);
            if (c2) atomicAdd(o.vtag + 3 * x + 1, c2);
            if (c3) atomicAdd(o.vtag + 3 * x + 2, c3);
            if (lw) atomicAdd(o.split + x, lw);
        }
    }
}

// ----------------------------------------------------- step 4: placement

// Rows other than the long ones, 32 consecutive rows per warp: their
// distinct entries, back to back, copied by all lanes; each entry's row too.
__global__ void __launch_bounds__(256) k_compact(const int32_t* __restrict__ roff, const int32_t* __restrict__ ucnt,
                                                 const uint8_t* __restrict__ lflag,
                                                 const int64_t* __restrict__ row_ptr, int64_t total_n,
                                                 const uint32_t* __restrict__ tmp, uint32_t* __restrict__ adj,
                                                 int32_t* __restrict__ arow) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t groups = (total_n + 31) >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t grp = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); grp < groups; grp += nwarps) {
        const int64_t x = (grp << 5) + lane;
        const bool valid = x < total_n;
        const int32_t sb = valid ? roff[x] : 0;
        const int len = valid && !lflag[x] ? ucnt[x] : 0;
        const int64_t db = valid ? row_ptr[x] : 0;
        int inc = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(full, inc, o);
            if (lane >= o) inc += t;
        }
        const int pre = inc - len, total = __shfl_sync(full, inc, 31);
        for (int e0 = 0; e0 < total; e0 += 32) {
            const int e = e0 + lane;
            int q = 0;  // the last lane whose row starts at or before e
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const int pq = __shfl_sync(full, pre, q + st);
                if (pq <= e) q += st;
            }
            const int pq = __shfl_sync(full, pre, q);
            const int32_t sq = __shfl_sync(full, sb, q);
            const int64_t dq = __shfl_sync(full, db, q);
            if (e < total) {
                adj[dq + (e - pq)] = tmp[sq + (e - pq)];
                arow[dq + (e - pq)] = (int32_t)((grp << 5) + q);
            }
        }
    }
}

// Long rows, a warp per WCH-word tile: the tile's run heads (tags OR-ed over
// the run) after those of the row's earlier tiles.
__global__ void __launch_bounds__(256) k_long_write(const int32_t* __restrict__ roff, LongOut lo,
                                                    const uint32_t* __restrict__ tmp,
                                                    const int32_t* __restrict__ tcnt,
                                                    const int64_t* __restrict__ row_ptr, uint32_t* __restrict__ adj,
                                                    int32_t* __restrict__ arow) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nt = lo.ctr[4];
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int it = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < nt; it += nwarps) {
        const uint4 tl = lo.tiles[it];
        const int64_t x = tl.x;
        const int32_t rb = roff[x];
        const int L = roff[x + 1] - rb;
        const uint32_t* s = tmp + rb;
        int pre = 0;
        for (int u = (int)tl.z + lane; u < it; u += 32) pre += tcnt[u];
        pre = __reduce_add_sync(full, pre);
        const int64_t d0 = row_ptr[x] + pre;
        int k = 0;
        const int i1 = min(L, (int)(tl.y + 1) * WCH);
        for (int i0 = (int)tl.y * WCH; i0 < i1; i0 += 32) {
            const int i = i0 + lane;
            const uint32_t w = i < i1 ? s[i] : SENT;
            const bool head = i < i1 && (i == 0 || (s[i - 1] >> 2) != (w >> 2));
            uint32_t t = w & 3u;
            if (head)
                for (int j = i + 1; j < L && (s[j] >> 2) == (w >> 2); ++j) t |= s[j] & 3u;
            const unsigned hb = __ballot_sync(full, head);
            if (head) {
                const int64_t p = d0 + k + __popc(hb & ((1u << lane) - 1u));
                adj[p] = (w & ~3u) | t;
                arow[p] = (int32_t)x;
            }
            k += __popc(hb);
        }
    }
}

// Sentinel words from adj[row_ptr[rows]] (the end of the entries) to `end`.
__global__ void k_fill_tail(uint32_t* __restrict__ adj, const int64_t* __restrict__ nnz_at, int64_t end) {
    const int64_t b = *nnz_at;
    for (int64_t i = b + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < end; i += (int64_t)gridDim.x * blockDim.x)
        adj[i] = SENT;
}

// Thread per row: degree, and per-graph statistics from the row's degree and tag
// counts; a warp whose rows lie in one graph adds its sums with one atomic
// each (one graph: a block adds its sums once).
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

int device_sms() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

int grid_for(int64_t work, int threads, int sms) {
    int64_t g = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)sms * 16));
}

// out[0..n] = exclusive scan of in[0..n) and the total (n < 2^31 items).
template <class OUT>
tc_status scan_excl(Scratch& S, const int32_t* in, int64_t n, OUT* out, cudaStream_t st) {
    char* tmp = nullptr;
    TC_CUDA(S.get(&tmp, scan_tmp_bytes(n)));
    TC_CUDA(scan_run<false>(ScanLoad<int32_t>{in}, n, out, tmp, true, st));
    return TC_OK;
}

// A small page-locked host word block per host thread, so counts can come
// back from the device while later kernels are already queued.
int32_t* pinned_words() {
    struct Holder {
        int32_t* p = nullptr;
        ~Holder() {
            if (p) cudaFreeHost(p);
        }
    };
    static thread_local Holder h;
    if (!h.p && cudaMallocHost((void**)&h.p, 8 * sizeof(int32_t)) != cudaSuccess) h.p = nullptr;
    return h.p;
}

// Bucket rows 2^b: buckets of about CAP / 3 entries on average, at most
// NB_MAX buckets; -1 when that needs more than MAX_BROWS rows per bucket.
int bucket_bits(int64_t total_n, int64_t entries) {
    int b = MIN_BBITS;
    const double target = (double)CAP / 3.0 * (double)total_n / (double)std::max<int64_t>(entries, 1);
    while (b < MAX_BBITS && (double)(1 << (b + 1)) <= target) ++b;
    while (b <= MAX_BBITS && ((total_n + ((int64_t)1 << b) - 1) >> b) > NB_MAX) ++b;
    return b <= MAX_BBITS ? b : -1;
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
    if (total_n >= ((int64_t)1 << 31) - 1)
        return fail(TC_ERR_UNSUPPORTED, "graph build: total vertices must be < 2^31 - 1");
    if (m > 0 && (!src || !dst)) return fail(TC_ERR_ARG, "graph build: null arc arrays");
    if (2 * m >= ((int64_t)1 << 31) - 1) return fail(TC_ERR_UNSUPPORTED, "graph build: m must be < 2^30");
    const int sms = device_sms();

    auto set = std::make_shared<GraphSet>();
    set->G = G;
    set->total_n = total_n;
    set->voff = voff;
    set->max_n = max_n;
    set->stats.assign((size_t)G, tc_graph_stats_t{});
    const int64_t N = 2 * m;
    const size_t nrows = (size_t)std::max<int64_t>(total_n, 1);
    set->adj_cap = N;
    TC_CUDA(dev_alloc((void**)&set->row_ptr, sizeof(int64_t) * (size_t)(total_n + 1), st));
    TC_CUDA(dev_alloc((void**)&set->adj, sizeof(uint32_t) * (size_t)(N + ADJ_PAD), st));
    TC_CUDA(dev_alloc((void**)&set->deg, sizeof(int32_t) * nrows, st));
    TC_CUDA(dev_alloc((void**)&set->vtag, sizeof(int32_t) * 3 * nrows, st));
    TC_CUDA(dev_alloc((void**)&set->split, sizeof(int32_t) * nrows, st));
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
    unsigned long long* d_gstat = nullptr;
    int32_t *roff = nullptr, *ucnt = nullptr, *ctr = nullptr, *tcnt = nullptr;
    uint32_t *tmp = nullptr, *tmp2 = nullptr;
    LongOut lo{};
    const size_t tile_cap = (size_t)(2 * N / WCH + 16);    // WCH-word tiles of rows or segments
    const size_t long_cap = (size_t)(N / WCH + 16);        // rows longer than WCH
    const size_t seg_cap = (size_t)(N / (SUB_AVG / 2) + long_cap);  // fewer than 2 L / SUB_AVG + 1 ranges per row
    const size_t piece_cap = (size_t)(N / CAP + N / WCH + 16);
    TC_CUDA(S.get(&d_aoff, (size_t)G + 1));
    TC_CUDA(S.get(&d_voff, (size_t)G + 1));
    TC_CUDA(S.get(&d_err, 1));
    TC_CUDA(S.get(&d_gstat, 6 * (size_t)G + 8));
    TC_CUDA(S.get(&roff, nrows + 1));
    TC_CUDA(S.get(&ucnt, nrows + 1));
    TC_CUDA(S.get(&ctr, 8));
    TC_CUDA(S.get(&tmp, (size_t)std::max<int64_t>(N, 1)));
    TC_CUDA(S.get(&tmp2, (size_t)std::max<int64_t>(N, 1)));
    TC_CUDA(S.get(&lo.lng, long_cap));
    TC_CUDA(S.get(&lo.tiles, tile_cap));
    TC_CUDA(S.get(&lo.lflag, nrows));
    TC_CUDA(S.get(&lo.segs, seg_cap));
    TC_CUDA(S.get(&lo.bpieces, piece_cap));
    TC_CUDA(S.get(&lo.btiles, tile_cap));
    TC_CUDA(S.get(&tcnt, tile_cap));
    lo.ctr = ctr;
    TC_CUDA(cudaMemcpyAsync(d_aoff, aoff.data(), sizeof(int64_t) * ((size_t)G + 1), cudaMemcpyHostToDevice, st));
    TC_CUDA(cudaMemcpyAsync(d_voff, voff.data(), sizeof(int64_t) * ((size_t)G + 1), cudaMemcpyHostToDevice, st));
    TC_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    TC_CUDA(cudaMemsetAsync(d_gstat, 0, sizeof(unsigned long long) * (6 * (size_t)G + 8), st));
    TC_CUDA(cudaMemsetAsync(ctr, 0, sizeof(int32_t) * 8, st));
    TC_CUDA(cudaMemsetAsync(ucnt, 0, sizeof(int32_t) * (nrows + 1), st));
    TC_CUDA(cudaMemsetAsync(lo.lflag, 0, nrows, st));
    TC_CUDA(cudaMemsetAsync(set->vtag, 0, sizeof(int32_t) * 3 * nrows, st));
    TC_CUDA(cudaMemsetAsync(set->split, 0, sizeof(int32_t) * nrows, st));

    const ArcIn ai{d_src, d_dst, m, d_aoff, d_voff, G};
    // rows sorted by one thread: up to 8 entries when rows average fewer than
    // 12 raw entries, else up to 16 (measured on B300: R-MAT scale 22 with 7.9
    // per row builds 0.08 ms faster with 8; Chung-Lu with 17.5 per row 0.06 ms
    // faster with 16); longer rows are sorted by a warp
    const int smax = N <= 12 * std::max<int64_t>(total_n, 1) ? 8 : SMALL_MAX;
    const RowOut ro{ucnt, set->vtag, set->split};
    const int b = total_n > 0 ? bucket_bits(total_n, N) : -1;
    if (b >= 0) {  // buckets of 2^b rows
        const int NB = (int)((total_n + ((int64_t)1 << b) - 1) >> b);
        const int nblk = sms;
        int32_t *hist = nullptr, *Sb = nullptr, *fbk = nullptr;
        void* ent = nullptr;
        // packed entries when every word (nbr << 2 | tag) fits below bit 32 - b
        const bool pack = max_n <= ((int64_t)1 << (30 - b));
        TC_CUDA(S.get(&hist, (size_t)NB * nblk));
        TC_CUDA(S.get(&Sb, (size_t)NB * nblk + 1));
        TC_CUDA(S.get(&fbk, (size_t)NB));
        TC_CUDA(S.get((char**)&ent, (pack ? 4 : 8) * (size_t)std::max<int64_t>(N, 1)));
        const size_t hsm = sizeof(int32_t) * (size_t)NB;
        TC_CUDA(cudaFuncSetAttribute(k_bkt_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm));
        TC_CUDA(cudaFuncSetAttribute(k_bkt_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm));
        TC_CUDA(cudaFuncSetAttribute(k_bkt_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm));
        auto kb = pack ? (smax == 8 ? k_bkt_rows<true, 8> : k_bkt_rows<true, 16>)
                       : (smax == 8 ? k_bkt_rows<false, 8> : k_bkt_rows<false, 16>);
        TC_CUDA(cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BK_SMEM));
        k_bkt_hist<<<nblk, PT_NT, hsm, st>>>(ai, b, NB, nblk, hist, d_err);
        TC_CUDA(cudaGetLastError());
        if (tc_status s2 = scan_excl<int32_t>(S, hist, (int64_t)NB * nblk, Sb, st); s2 != TC_OK) return s2;
        if (pack) k_bkt_scatter<true><<<nblk, PT_NT, hsm, st>>>(ai, b, NB, nblk, undirected, Sb, (uint32_t*)ent);
        else k_bkt_scatter<false><<<nblk, PT_NT, hsm, st>>>(ai, b, NB, nblk, undirected, Sb, (uint2*)ent);
        TC_CUDA(cudaGetLastError());
        const BktArgs ba{ent, Sb, nblk, NB, b, total_n, d_voff, G, tmp, roff, ro, fbk, lo};
        kb<<<(unsigned)std::min(NB, sms * 3), BS_NT, BK_SMEM, st>>>(ba);
        TC_CUDA(cudaGetLastError());
        k_rows<<<(unsigned)sms * 4, RW_NT, 0, st>>>(roff, total_n, d_voff, G, tmp, ro, fbk, b, lo, smax);
        TC_CUDA(cudaGetLastError());
    } else if (total_n > 0) {  // one atomic per entry
        int32_t* cnt = nullptr;
        TC_CUDA(S.get(&cnt, nrows + 1));
        TC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nrows + 1), st));
        if (m > 0) {
            k_arc_count<<<grid_for(m, 256, sms), 256, 0, st>>>(ai, cnt, d_err);
            TC_CUDA(cudaGetLastError());
        }
        if (tc_status s2 = scan_excl<int32_t>(S, cnt, total_n, roff, st); s2 != TC_OK) return s2;
        if (m > 0) {
            k_arc_scatter<<<grid_for(m, 256, sms), 256, 0, st>>>(ai, undirected, roff, cnt, tmp);
            TC_CUDA(cudaGetLastError());
        }
        const int64_t groups = (total_n + 31) / 32;
        k_rows<<<(unsigned)std::min<int64_t>((groups + RW_W - 1) / RW_W, (int64_t)sms * 16), RW_NT, 0, st>>>(
            roff, total_n, d_voff, G, tmp, ro, nullptr, MIN_BBITS, lo, smax);
        TC_CUDA(cudaGetLastError());
    }
    if (total_n > 0) {  // long rows: split by id range, segments sorted, crowded segments merged
        k_long_split_w<<<(unsigned)sms * 8, 256, 0, st>>>(roff, d_voff, G, lo, tmp, tmp2);
        TC_CUDA(cudaGetLastError());
        k_long_split<<<(unsigned)sms * 2, LS_NT, 0, st>>>(roff, d_voff, G, lo, tmp, tmp2);
        TC_CUDA(cudaGetLastError());
        k_seg_sort<<<(unsigned)sms * 16, RW_NT, 0, st>>>(lo, tmp2, tmp);
        TC_CUDA(cudaGetLastError());
        // the longest crowded segment comes back while their pieces sort
        int32_t* hw = pinned_words();
        if (!hw) return fail(TC_ERR_OOM, "graph build: page-locked host words");
        TC_CUDA(cudaFuncSetAttribute(k_big_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LS_SMEM));
        cudaEvent_t ev;
        TC_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaError_t e = cudaMemcpyAsync(hw, ctr, sizeof(int32_t) * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaEventRecord(ev, st);
        if (e == cudaSuccess) {
            k_big_sort<<<(unsigned)sms * 2, BS_NT, LS_SMEM, st>>>(lo, tmp2);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventSynchronize(ev);
        cudaEventDestroy(ev);
        TC_CUDA(e);
        const int maxbig = hw[2], nlong = hw[0];
        if (maxbig > 0) {
            int rounds = 0;
            while (((int64_t)CAP << rounds) < maxbig) ++rounds;
            for (int r = 0; r < rounds; ++r) {
                k_merge_round<<<(unsigned)sms * 8, 256, 0, st>>>(lo, r, (r & 1) ? tmp : tmp2, (r & 1) ? tmp2 : tmp);
                TC_CUDA(cudaGetLastError());
            }
            k_big_copy<<<(unsigned)sms * 8, 256, 0, st>>>(lo, tmp2, tmp);
            TC_CUDA(cudaGetLastError());
        }
        if (nlong > 0) {
            k_long_count<<<(unsigned)sms * 8, 256, 0, st>>>(roff, lo, d_voff, G, tmp, ro, tcnt);
            TC_CUDA(cudaGetLastError());
        }
    }
    if (tc_status s2 = scan_excl<int64_t>(S, ucnt, total_n, set->row_ptr, st); s2 != TC_OK) return s2;
    if (total_n > 0) {
        k_compact<<<grid_for((total_n + 31) / 32 * 32, 256, sms), 256, 0, st>>>(roff, ucnt, lo.lflag, set->row_ptr,
                                                                                 total_n, tmp, set->adj, set->arow);
        TC_CUDA(cudaGetLastError());
        k_long_write<<<(unsigned)sms * 8, 256, 0, st>>>(roff, lo, tmp, tcnt, set->row_ptr, set->adj, set->arow);
        TC_CUDA(cudaGetLastError());
        k_rowstats<<<grid_for(total_n, 256, sms), 256, 0, st>>>(set->row_ptr, set->vtag, d_voff, G, total_n,
                                                                set->deg, d_gstat);
        TC_CUDA(cudaGetLastError());
    }
    k_fill_tail<<<grid_for(ADJ_PAD + N, 256, sms), 256, 0, st>>>(set->adj, set->row_ptr + total_n, N + ADJ_PAD);
    TC_CUDA(cudaGetLastError());
    std::vector<unsigned long long> gstat(6 * (size_t)G);
    int err = 0;
    TC_CUDA(cudaMemcpyAsync(gstat.data(), d_gstat, sizeof(unsigned long long) * 6 * (size_t)G,
                            cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    if (err) return fail(TC_ERR_ID_RANGE, "graph build: an arc endpoint lies outside [0, n)");
    int64_t nnz = 0;
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
        nnz += (int64_t)x[1];
        set->max_deg = std::max<int32_t>(set->max_deg, (int32_t)x[4]);
    }
    set->nnz = nnz;
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
