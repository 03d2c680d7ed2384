// tc_census / tc_census_batched: the per-canonical-dyad merge/classify pass.
//
// Method (Sec. 2.2, Fig. "Subquadratic Triad Census Algorithm", with the v0.4
// pre-computed dyad code of Sec. 4.2.4 and the canonical-dyad task queues of
// Sec. 4.3.1 / 5.1.1).  For every canonical dyad <u,v>, u < v adjacent, with
// pre = e(u,v) + 2e(v,u), A = N(u), B = N(v) (tagged, sorted):
//   dyadic term   Census[pre==3 ? 102 : 012] += n - |S| - 2,
//                 S = A u B \ {u,v},  |S| = |A| + |B| - 2 - |A n B|;
//   connected     every w in S with  v < w  or  (u < w < v and w not in N(u))
//                 adds 1 to code pre + 4*tag_u(w) + 16*tag_v(w)
//                 (tag_x(w) = e(x,w) + 2e(w,x), 0 when w is not a neighbour).
// 003 = C(n,3) - sum of the other fifteen (128-bit).
//
// How the work is split across kernels (the result is the same integer sum,
// regrouped; every per-dyad contribution is counted exactly once):
//  * w only in A (tag_v = 0) is counted iff w > v, i.e. it is one of the
//    entries of row u after v; w only in B (tag_u = 0) is counted iff w > u,
//    i.e. one of the entries of row v after u.  The task pass (k_tasks_flat,
//    one thread per adjacency entry, suffix counts from a tag scan; or
//    k_tasks, one warp per row) adds, per dyad, the counts of A after v into
//    codes pre+4t and the counts of B after u into codes pre+16t, as if no
//    element were shared, plus n - |A| - |B| into the dyadic slot.  It emits
//    the dyad as a task binned by |A|+|B|, unless its higher-degree endpoint
//    owns it (owner lookups below).
//  * The shared elements w correct the classification: if w > v the triad
//    was counted as pre+4tu and pre+16tv and is moved to pre+4tu+16tv; if
//    u < w < v it was counted as pre+16tv and must not count at all; a w
//    below u changes nothing.  In a triangle a < b < c the first case is
//    dyad <a,b> with w = c, the second dyad <a,c> with w = b, both fixed by
//    the three tags of the triangle, so both corrections are made when dyad
//    <a,b> finds c: only shared elements above v are searched for.  They are
//    found by k_owner (the shorter list's entries above v looked up in an
//    index of the owner's list) or by the merge kernels (k_merge, k_hub and
//    the separate-launch items: both lists streamed).
//  * |A n B| itself is never counted: summed over the dyads it is fixed by
//    the closed-triad counts, which k_fold adds to the dyadic slots after
//    mapping the 64 codes onto the 16 MAN types; k_fold closes 003.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "mlp.cuh"
#include "scan.cuh"
#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr int WARPS = 8;  // warps per 256-thread block

// Per-task timing records of an instrumented census: tasks whose endpoint
// hash has (hash & mask) == 0 append {u, v, bin, cycles}.
struct Instr {
    int4* buf;
    unsigned int* count;
    unsigned int cap;
    unsigned int mask;
};

__device__ __forceinline__ bool sampled(const Instr* ins, uint32_t u, uint32_t v) {
    uint32_t h = u * 0x9E3779B1u ^ (v * 0x85EBCA77u + 0x27d4eb2fu);
    h ^= h >> 15;
    h *= 0x2c1b3c6du;
    h ^= h >> 12;
    return (h & ins->mask) == 0;
}

__device__ __forceinline__ void record(const Instr* ins, uint32_t u, uint32_t v, int bin, long long cycles) {
    const unsigned slot = atomicAdd(ins->count, 1u);
    if (slot < ins->cap)
        ins->buf[slot] = make_int4((int)u, (int)v, bin, (int)min(cycles, (long long)0x7fffffff));
}

thread_local tc_profile_t g_profile;
thread_local bool g_profile_valid = false;

// profile marks: start, after the task pass, k_split (forward path: the
// forward lists), the owner prep (k_tri_big), k_owner (k_tri_small), the
// four merge kernels, k_fold
constexpr int NEV = 10;

struct ProfileEvents {
    cudaEvent_t ev[NEV + 1];  // ev[NEV]: before the exact-cost pass (TC_BIN_EXACT)
};

tc_status profile_events(ProfileEvents** out) {
    static thread_local ProfileEvents pe[64];
    static thread_local bool made[64];
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    dev &= 63;
    if (!made[dev]) {
        for (int k = 0; k <= NEV; ++k) TC_CUDA(cudaEventCreate(&pe[dev].ev[k]));
        made[dev] = true;
    }
    *out = &pe[dev];
    return TC_OK;
}

// ------------------------------------------------------------ type table --
// MAN type of the labelled triad with 6-bit code (bit order of Fig. "Triad
// Code Algorithm": e(u,v)=1, e(v,u)=2, e(u,w)=4, e(w,u)=8, e(v,w)=16,
// e(w,v)=32), decided from the mutual/asymmetric dyad counts and the vertex
// degree signatures of the triad.
__host__ __device__ __forceinline__ int triad_type(int code) {
    const int e01 = code & 1, e10 = (code >> 1) & 1, e02 = (code >> 2) & 1;
    const int e20 = (code >> 3) & 1, e12 = (code >> 4) & 1, e21 = (code >> 5) & 1;
    const int od[3] = {e01 + e02, e10 + e12, e20 + e21};
    const int id[3] = {e10 + e20, e01 + e21, e02 + e12};
    const int M = (e01 & e10) + (e02 & e20) + (e12 & e21);
    const int A = (e01 ^ e10) + (e02 ^ e20) + (e12 ^ e21);
    bool out2 = false, in2 = false, src2 = false, snk2 = false;
    for (int x = 0; x < 3; ++x) {
        out2 |= od[x] == 2;
        in2 |= id[x] == 2;
        src2 |= od[x] == 2 && id[x] == 0;  // sends two arcs, receives none
        snk2 |= id[x] == 2 && od[x] == 0;  // receives two arcs, sends none
    }
    if (M == 0 && A == 0) return 0;                 // 003
    if (M == 0 && A == 1) return 1;                 // 012
    if (M == 1 && A == 0) return 2;                 // 102
    if (M == 0 && A == 2) return out2 ? 3 : (in2 ? 4 : 5);  // 021D 021U 021C
    if (M == 1 && A == 1) return in2 ? 6 : 7;       // 111D (arc into the pair) 111U
    if (M == 0 && A == 3) return out2 ? 8 : 9;      // 030T 030C
    if (M == 2 && A == 0) return 10;                // 201
    if (M == 1 && A == 2) return src2 ? 11 : (snk2 ? 12 : 13);  // 120D 120U 120C
    if (M == 2 && A == 1) return 14;                // 210
    return 15;                                      // 300
}

// ---------------------------------------------------------- device types --
struct SegDev {
    int64_t rb;    // first global row of the graph (local id = global - rb)
    int64_t n;     // vertices
    int64_t eb;    // first global adjacency entry of the graph
    int32_t slot;  // output index
    int32_t pad;
};

// Task bins: 0 thread per task, 1 warp per task, 2 split into tiles,
// 3 stream (warp per task, short list staged, long list streamed).
constexpr int NBIN = 4;

struct Bins {
    uint4* rec[NBIN];     // {u global, v global, seg<<2 | pre, position in u's list after v}
    uint32_t cap[NBIN];
    unsigned int* cnt;    // [NBIN] records appended per bin
    int* overflow;
    unsigned long long* entries;  // [NBIN] merged entries per bin
    uint4* own;           // owner pieces {row, seg, piece, 0}: owners up to
                          // OWN_CAP from the front, larger ones from the back
    uint32_t own_cap;
    unsigned int* own_cnt;        // [2] larger owners, smaller owners
    unsigned long long* own_stat; // [4] tasks, merged entries, probes, staged entries
};

// Longest shorter list a streamed task stages whole in shared memory; longer
// ones (hub tasks) run in a separate launch that stages it in pieces.
constexpr int STREAM_SMAX = 1024;

// Owner tasks: a dyad whose higher-degree endpoint (the owner; equal degrees:
// the larger id) has degree in [own_min, OWN_MAX] is not merged; k_owner
// indexes the owner's list in shared memory and looks the other endpoint's
// list up in it.
constexpr int OWN_CAP = 512;     // owners up to this degree are staged whole
constexpr int OWN_MAX = 131072;  // larger ones: bucket starts only
// an owner's dyads are cut into pieces of this many list positions, one work
// item each (so that several CTAs share a large owner)
constexpr int OWN_PIECE = 1024;

struct BinParams {
    int thr_thread, thr_warp, stream_max, own_min;
    const __half2* mlp;     // packed FP16 cost model, or null for the degree-sum rule
    const int32_t* vtag;    // per-vertex tag counts (model features)
    int fwd;                // 1: the triangles come from the forward lists: emit no task
    const uint32_t* exact;  // TC_BIN_EXACT: |S| of each canonical dyad at its adjacency
                            // position in row u (k_union_entries), else null
    // shard of the work (tc_census_shard; everything when unsharded): the task
    // terms of the selection's entries [e_lo, e_hi) (k_tasks_flat) or of its
    // rows [r_lo, r_hi) (k_tasks), and the dyads owned by rows [r_lo, r_hi)
    int64_t e_lo, e_hi, r_lo, r_hi;
};

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int seg_of(const int64_t* pfx, int nseg, int64_t r) {
    int lo = 0, hi = nseg - 1;  // largest s with pfx[s] <= r
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pfx[mid] <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// --------------------------------------------------------------- k_tasks --
// One warp per row x (rows pulled in blocks from a global cursor).  For each
// entry (y, t) of row x at position k: suffix counts S1..S3 of the tags of
// entries after k.  y > x: canonical dyad <x,y> (pre = t): add S into codes
// pre+4t', n-|A|-|B| into the dyadic slot, emit the task.  y < x: row x is
// B of dyad <y,x> (pre = swapped t): add S into codes pre+16t'.
__global__ void __launch_bounds__(256) k_tasks(const int64_t* __restrict__ row_ptr,
                                               const uint32_t* __restrict__ adj,
                                               const int32_t* __restrict__ deg,
                                               const SegDev* __restrict__ seg,
                                               const int64_t* __restrict__ pfx, int nseg,
                                               int64_t total_rows, BinParams bp, Bins bins,
                                               unsigned long long* __restrict__ acc,
                                               unsigned long long* __restrict__ cursor) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    const unsigned above = lane == 31 ? 0u : (full << (lane + 1));
    const unsigned below = (1u << lane) - 1u;
    constexpr int ROWS = 32;

    int s = -1;
    int64_t rb = 0, n = 0, sp = 0;
    unsigned long long Aa[3][3], Bb[3][3], Dd[3], Ee[NBIN], Os[4] = {0, 0, 0, 0};
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) Aa[p][q] = Bb[p][q] = 0;
    Dd[0] = Dd[1] = Dd[2] = 0;
#pragma unroll
    for (int b = 0; b < NBIN; ++b) Ee[b] = 0;

    auto flush = [&]() {
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                unsigned long long a = warp_sum64(Aa[p][q]), b = warp_sum64(Bb[p][q]);
                if (lane == 0 && s >= 0) {
                    if (a) atomicAdd(acc + (size_t)s * ACC + (p + 1) + 4 * (q + 1), a);
                    if (b) atomicAdd(acc + (size_t)s * ACC + (p + 1) + 16 * (q + 1), b);
                }
                Aa[p][q] = Bb[p][q] = 0;
            }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            unsigned long long d = warp_sum64(Dd[q]);
            if (lane == 0 && s >= 0 && d) atomicAdd(acc + (size_t)s * ACC + 64 + q, d);
            Dd[q] = 0;
        }
    };

    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(cursor, (unsigned long long)ROWS);
        base = __shfl_sync(full, base, 0);
        if ((int64_t)base >= total_rows) break;
        const int64_t rend = min((int64_t)base + ROWS, total_rows);
        for (int64_t r = (int64_t)base; r < rend; ++r) {
            const int sr = nseg == 1 ? 0 : seg_of(pfx, nseg, r);
            if (sr != s) {
                flush();
                s = sr;
                rb = seg[s].rb;
                n = seg[s].n;
                sp = pfx[s];
            }
            if (r < bp.r_lo || r >= bp.r_hi) continue;  // another shard's row
            const int64_t xl = r - sp;
            const int64_t x = rb + xl;
            const int64_t beg = row_ptr[x];
            const int d = deg[x];
            if (!bp.fwd && bp.own_min > 0 && d >= bp.own_min && d <= OWN_MAX) {  // an owner: append its pieces
                const bool large = d > OWN_CAP;
                const int np = (d + OWN_PIECE - 1) / OWN_PIECE;
                unsigned k = 0;
                if (lane == 0) k = atomicAdd(bins.own_cnt + (large ? 0 : 1), (unsigned)np);
                k = __shfl_sync(full, k, 0);
                for (int p = lane; p < np; p += 32) {
                    const unsigned i = k + (unsigned)p;
                    if (i < bins.own_cap) bins.own[large ? bins.own_cap - 1 - i : i] =
                        make_uint4((uint32_t)x, (uint32_t)s, (uint32_t)p, 0u);
                    else atomicOr(bins.overflow, 1);
                }
                if (lane == 0) Os[3] += (unsigned long long)d * (unsigned long long)np;
            }
            int c1 = 0, c2 = 0, c3 = 0;
            for (int cb = ((d - 1) >> 5) << 5; cb >= 0; cb -= 32) {
                const int k = cb + lane;
                const bool valid = k < d;
                const uint32_t e = valid ? __ldg(adj + beg + k) : 0u;
                const uint32_t y = e >> 2;
                const int t = (int)(e & 3u);
                const unsigned m1 = __ballot_sync(full, valid && t == 1);
                const unsigned m2 = __ballot_sync(full, valid && t == 2);
                const unsigned m3 = __ballot_sync(full, valid && t == 3);
                const unsigned long long S1 = (unsigned)(c1 + __popc(m1 & above));
                const unsigned long long S2 = (unsigned)(c2 + __popc(m2 & above));
                const unsigned long long S3 = (unsigned)(c3 + __popc(m3 & above));
                c1 += __popc(m1);
                c2 += __popc(m2);
                c3 += __popc(m3);
                const bool is_task = valid && (int64_t)y > xl;
                const bool is_twin = valid && (int64_t)y < xl;
                const int pre_task = t;
                const int pre_twin = ((t & 1) << 1) | (t >> 1);
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    const bool ta = is_task && pre_task == p + 1;
                    const bool tb = is_twin && pre_twin == p + 1;
                    Aa[p][0] += ta ? S1 : 0ull;
                    Aa[p][1] += ta ? S2 : 0ull;
                    Aa[p][2] += ta ? S3 : 0ull;
                    Bb[p][0] += tb ? S1 : 0ull;
                    Bb[p][1] += tb ? S2 : 0ull;
                    Bb[p][2] += tb ? S3 : 0ull;
                }
                int L = 0;
                int bin = -1;
                if (is_task) {
                    const int dv = deg[rb + y];
                    L = d + dv;
                    const unsigned long long dy = (unsigned long long)(n - (int64_t)d - (int64_t)dv);
#pragma unroll
                    for (int q = 0; q < 3; ++q) Dd[q] += pre_task == q + 1 ? dy : 0ull;
                    const int dh = max(d, dv);
                    if (bp.fwd) {
                    } else if (bp.own_min > 0 && dh >= bp.own_min && dh <= OWN_MAX) {  // owner task
                        Os[0] += 1;
                        Os[1] += (unsigned long long)L;

                    } else {
                        const int c = bp.exact ? (int)bp.exact[beg + k] + 2 : L;  // |S| + 2 = L - c_uv
                        bin = c <= bp.thr_thread ? 0
                              : c <= bp.thr_warp ? 1
                              : min(d, dv) <= min(bp.stream_max, STREAM_SMAX) ? 3 : 2;
                    }
                }
#pragma unroll
                for (int b = 0; b < NBIN; ++b) Ee[b] += bin == b ? (unsigned long long)L : 0ull;
                const uint4 rec = make_uint4((uint32_t)x, (uint32_t)(rb + y),
                                             ((uint32_t)s << 2) | (uint32_t)pre_task, (uint32_t)(k + 1));
#pragma unroll
                for (int b = 0; b < NBIN; ++b) {
                    const bool mine = bin == b;
                    const unsigned mask = __ballot_sync(full, mine);
                    if (mask) {
                        const int leader = __ffs(mask) - 1;
                        unsigned int at = 0;
                        if (lane == leader) at = atomicAdd(bins.cnt + b, (unsigned)__popc(mask));
                        at = __shfl_sync(full, at, leader);
                        if (mine) {
                            const unsigned idx = at + __popc(mask & below);
                            if (idx < bins.cap[b]) bins.rec[b][idx] = rec;
                            else atomicOr(bins.overflow, 1);
                        }
                    }
                }
            }
        }
    }
    flush();
#pragma unroll
    for (int b = 0; b < NBIN; ++b) {
        const unsigned long long e = warp_sum64(Ee[b]);
        if (lane == 0 && e) atomicAdd(bins.entries + b, e);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned long long e = warp_sum64(Os[k]);
        if (lane == 0 && e) atomicAdd(bins.own_stat + k, e);
    }
}

// ---------------------------------------------------------- k_tasks_flat --
// The same per-dyad terms as k_tasks, one adjacency entry per thread.  The
// suffix counts of entry k in row x (entries after k with each tag) are the
// row's tag totals (vtag, from the build) minus the row-local inclusive prefix
// of one-hot tag words, itself the difference of a global inclusive scan at k
// and before the row's first entry; the scan packs the three tags in 21-bit
// fields, exact while every row has fewer than 2^21 entries (the difference
// is taken modulo 2^64, so carries out of earlier rows cancel).
constexpr int TAG_BITS = 21;
constexpr unsigned long long TAG_MASK = (1ull << TAG_BITS) - 1;

// The one-hot tag word of entry f of the selected graphs' entries (in the
// order of their concatenation; entry k = the graph's first entry + offset),
// computed as the scan reads it (no array of words is written).
struct OneHot {
    const uint32_t* adj;
    const SegDev* seg;
    const int64_t* epfx;
    int nseg;
    __device__ unsigned long long operator()(int64_t f) const {
        const int s = nseg == 1 ? 0 : seg_of(epfx, nseg, f);
        const uint32_t t = __ldg(adj + seg[s].eb + (f - epfx[s])) & 3u;  // 1, 2 or 3
        return 1ull << (TAG_BITS * (t - 1));
    }
};

// Thread per row of the selected graphs: register each owner's work items.
__global__ void k_owner_rows(const int32_t* __restrict__ deg, const SegDev* __restrict__ seg,
                             const int64_t* __restrict__ pfx, int nseg, int64_t total_rows, int own_min,
                             Bins bins, int64_t r_lo, int64_t r_hi) {
    const int64_t r_end = min(total_rows, r_hi);
    for (int64_t r = r_lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < r_end;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int s = nseg == 1 ? 0 : seg_of(pfx, nseg, r);
        const int64_t x = seg[s].rb + (r - pfx[s]);
        const int d = deg[x];
        if (d < own_min || d > OWN_MAX) continue;
        const bool large = d > OWN_CAP;
        const int np = (d + OWN_PIECE - 1) / OWN_PIECE;
        const unsigned k = atomicAdd(bins.own_cnt + (large ? 0 : 1), (unsigned)np);
        for (int p = 0; p < np; ++p) {
            const unsigned i = k + (unsigned)p;
            if (i < bins.own_cap) bins.own[large ? bins.own_cap - 1 - i : i] =
                make_uint4((uint32_t)x, (uint32_t)s, (uint32_t)p, 0u);
            else atomicOr(bins.overflow, 1);
        }
        atomicAdd(bins.own_stat + 3, (unsigned long long)d * (unsigned long long)np);
    }
}

// Forward flags of the forward path, written by the task pass as it reads
// each entry (flag null: none).
struct FlagOut {
    uint8_t* flag;         // [entries] 1 when the entry's neighbour ranks above its row
    const int32_t* rank;   // per selected row
    const int64_t* pfx;    // first selected row of each graph
};

// Warps take runs of FLAT_RUN entries of the selected graphs' concatenated
// adjacency (graph boundaries rarely fall inside one); lanes whose entry lies
// in another graph than the warp's accumulators add directly.
constexpr int FLAT_RUN = 1024;

__global__ void __launch_bounds__(256, 4) k_tasks_flat(const int64_t* __restrict__ row_ptr,
                                                    const uint32_t* __restrict__ adj,
                                                    const int32_t* __restrict__ arow,
                                                    const int32_t* __restrict__ deg,
                                                    const int32_t* __restrict__ vtag,
                                                    const unsigned long long* __restrict__ scan,
                                                    const SegDev* __restrict__ seg,
                                                    const int64_t* __restrict__ epfx, int nseg,
                                                    int64_t total_entries, BinParams bp, Bins bins,
                                                    unsigned long long* __restrict__ acc,
                                                    unsigned long long* __restrict__ cursor, FlagOut fo) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    const unsigned below = (1u << lane) - 1u;
    int s = -1;  // graph of the warp's accumulators
    unsigned long long Aa[3][3], Bb[3][3], Dd[3], Ee[NBIN], Os[2] = {0, 0};
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) Aa[p][q] = Bb[p][q] = 0;
    Dd[0] = Dd[1] = Dd[2] = 0;
#pragma unroll
    for (int b = 0; b < NBIN; ++b) Ee[b] = 0;
    auto flush = [&]() {
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const unsigned long long a = warp_sum64(Aa[p][q]), b = warp_sum64(Bb[p][q]);
                if (lane == 0 && s >= 0) {
                    if (a) atomicAdd(acc + (size_t)s * ACC + (p + 1) + 4 * (q + 1), a);
                    if (b) atomicAdd(acc + (size_t)s * ACC + (p + 1) + 16 * (q + 1), b);
                }
                Aa[p][q] = Bb[p][q] = 0;
            }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const unsigned long long d = warp_sum64(Dd[q]);
            if (lane == 0 && s >= 0 && d) atomicAdd(acc + (size_t)s * ACC + 64 + q, d);
            Dd[q] = 0;
        }
    };
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(cursor, (unsigned long long)FLAT_RUN);
        base = __shfl_sync(full, base, 0);
        if ((int64_t)base >= total_entries) break;
        const int64_t fend = min((int64_t)base + FLAT_RUN, total_entries);
        int ls = nseg == 1 ? 0 : seg_of(epfx, nseg, (int64_t)base);  // lane's graph, stepped forward
        for (int64_t f0 = (int64_t)base; f0 < fend; f0 += 32) {
            const int64_t f = f0 + lane;
            const bool valid = f < fend;
            while (valid && ls + 1 < nseg && epfx[ls + 1] <= f) ++ls;
            const int ws = __shfl_sync(full, ls, 0);
            if (ws != s) {
                flush();
                s = ws;
            }
            const bool mine = ls == s;  // else this lane's entry belongs to a later graph
            const SegDev sg = seg[ls];
            const int64_t k = valid ? sg.eb + (f - epfx[ls]) : 0;
            const uint32_t e = valid ? __ldg(adj + k) : 0u;
            const int64_t x = valid ? (int64_t)arow[k] : 0;
            const int64_t xl = x - sg.rb;
            const uint32_t y = e >> 2;
            const int t = (int)(e & 3u);
            uint32_t S1 = 0, S2 = 0, S3 = 0;
            int d = 0;
            int64_t rp = 0;
            if (fo.flag && valid) {  // forward entry: its neighbour ranks above its row
                const int64_t p = fo.pfx[ls];
                fo.flag[f] = fo.rank[p + y] > fo.rank[p + xl] ? 1 : 0;
            }
            if (valid) {
                rp = row_ptr[x];
                const int64_t frs = epfx[ls] + (rp - sg.eb);  // the row's first entry, in scan order
                const unsigned long long I = scan[f] - (frs > 0 ? scan[frs - 1] : 0ull);
                S1 = (uint32_t)vtag[3 * x] - (uint32_t)(I & TAG_MASK);
                S2 = (uint32_t)vtag[3 * x + 1] - (uint32_t)((I >> TAG_BITS) & TAG_MASK);
                S3 = (uint32_t)vtag[3 * x + 2] - (uint32_t)((I >> (2 * TAG_BITS)) & TAG_MASK);
                d = deg[x];
            }
            const bool part = valid && f >= bp.e_lo && f < bp.e_hi;  // this shard's entry
            const bool is_task = part && (int64_t)y > xl;
            const bool is_twin = part && (int64_t)y < xl;
            const int pre_task = t;
            const int pre_twin = ((t & 1) << 1) | (t >> 1);
            int L = 0;
            int bin = -1;
            unsigned long long dy = 0;
            if (is_task) {
                const int dv = deg[sg.rb + y];
                L = d + dv;
                dy = (unsigned long long)(sg.n - (int64_t)d - (int64_t)dv);
                const int dh = max(d, dv);
                if (bp.fwd) {
                } else if (bp.own_min > 0 && dh >= bp.own_min && dh <= OWN_MAX) {  // owner task
                    Os[0] += 1;
                    Os[1] += (unsigned long long)L;
                } else {
                    const int c = bp.exact ? (int)bp.exact[k] + 2 : L;  // |S| + 2 = L - c_uv
                    bin = c <= bp.thr_thread ? 0
                          : c <= bp.thr_warp ? 1
                          : min(d, dv) <= min(bp.stream_max, STREAM_SMAX) ? 3 : 2;
                }
            }
            if (mine) {
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    const bool ta = is_task && pre_task == p + 1;
                    const bool tb = is_twin && pre_twin == p + 1;
                    Aa[p][0] += ta ? S1 : 0u;
                    Aa[p][1] += ta ? S2 : 0u;
                    Aa[p][2] += ta ? S3 : 0u;
                    Bb[p][0] += tb ? S1 : 0u;
                    Bb[p][1] += tb ? S2 : 0u;
                    Bb[p][2] += tb ? S3 : 0u;
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) Dd[q] += (is_task && pre_task == q + 1) ? dy : 0ull;
            } else if (valid && (is_task || is_twin)) {  // an entry of a later graph: add directly
                unsigned long long* h = acc + (size_t)ls * ACC;
                const int p = (is_task ? pre_task : pre_twin) - 1;
                const int sh4 = is_task ? 4 : 16;
                if (S1) atomicAdd(h + (p + 1) + sh4 * 1, (unsigned long long)S1);
                if (S2) atomicAdd(h + (p + 1) + sh4 * 2, (unsigned long long)S2);
                if (S3) atomicAdd(h + (p + 1) + sh4 * 3, (unsigned long long)S3);
                if (dy) atomicAdd(h + 63 + pre_task, dy);
            }
#pragma unroll
            for (int b = 0; b < NBIN; ++b) Ee[b] += bin == b ? (unsigned long long)L : 0ull;
            const uint4 rec = make_uint4((uint32_t)x, (uint32_t)(sg.rb + y), ((uint32_t)ls << 2) | (uint32_t)pre_task,
                                         (uint32_t)(k - rp + 1));
#pragma unroll
            for (int b = 0; b < NBIN; ++b) {
                const bool in = bin == b;
                const unsigned mask = __ballot_sync(full, in);
                if (mask) {
                    const int leader = __ffs(mask) - 1;
                    unsigned int at = 0;
                    if (lane == leader) at = atomicAdd(bins.cnt + b, (unsigned)__popc(mask));
                    at = __shfl_sync(full, at, leader);
                    if (in) {
                        const unsigned idx = at + __popc(mask & below);
                        if (idx < bins.cap[b]) bins.rec[b][idx] = rec;
                        else atomicOr(bins.overflow, 1);
                    }
                }
            }
        }
    }
    flush();
#pragma unroll
    for (int b = 0; b < NBIN; ++b) {
        const unsigned long long e = warp_sum64(Ee[b]);
        if (lane == 0 && e) atomicAdd(bins.entries + b, e);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const unsigned long long e = warp_sum64(Os[k]);
        if (lane == 0 && e) atomicAdd(bins.own_stat + k, e);
    }
}

// ------------------------------------------------------- k_union_entries --
// Exact task cost for bin_mode = TC_BIN_EXACT: |S| = |N(u) u N(v) \ {u, v}|
// of every canonical dyad <u, v> of the selection (the W3 workload of a task,
// Sec. 4.3: the cost the non-uniform distribution of Sec. 4.3.2 balances),
// written at the dyad's adjacency position in row u.  |S| = d_u + d_v - 2 -
// c_uv, with c_uv the common neighbours.  Warps take 32 entries at a time;
// the canonical ones (neighbour above the row) are done one after the other,
// the lanes binary-searching the shorter list's entries in the longer one.
__global__ void __launch_bounds__(256) k_union_entries(const int64_t* __restrict__ row_ptr,
                                                       const uint32_t* __restrict__ adj,
                                                       const int32_t* __restrict__ arow,
                                                       const int32_t* __restrict__ deg,
                                                       const SegDev* __restrict__ seg,
                                                       const int64_t* __restrict__ epfx, int nseg,
                                                       int64_t entries, uint32_t* __restrict__ usz) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t f0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; f0 < entries;
         f0 += warps * 32) {
        const int64_t f = f0 + lane;
        int64_t k = 0, x = 0, y = 0;
        bool canon = false;
        if (f < entries) {
            const int s = nseg == 1 ? 0 : seg_of(epfx, nseg, f);
            const SegDev& g = seg[s];
            k = g.eb + (f - epfx[s]);
            x = arow[k];
            y = g.rb + (int64_t)(__ldg(adj + k) >> 2);
            canon = y > x;
        }
        for (unsigned m = __ballot_sync(full, canon); m; m &= m - 1) {
            const int src = __ffs(m) - 1;
            const int64_t kk = __shfl_sync(full, k, src), u = __shfl_sync(full, x, src),
                          v = __shfl_sync(full, y, src);
            const int du = deg[u], dv = deg[v];
            const bool u_short = du <= dv;
            const uint32_t* sl = adj + row_ptr[u_short ? u : v];
            const uint32_t* gl = adj + row_ptr[u_short ? v : u];
            const int ns = u_short ? du : dv, ng = u_short ? dv : du;
            int common = 0;
            for (int i = lane; i < ns; i += 32) common += list_has(gl, ng, __ldg(sl + i) >> 2) ? 1 : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) common += __shfl_xor_sync(full, common, o);
            if (lane == 0) usz[kk] = (uint32_t)(du + dv - 2 - common);
        }
    }
}

// --------------------------------------------------------------- k_route --
// Learned hub splitting: each task above the warp bin (collected in `cand`)
// goes to the stream bin or is split into tiles, whichever the FP16 cost
// model predicts cheaper (stream only when the shorter list fits a warp's
// shared memory).
__global__ void __launch_bounds__(256) k_route(const __half2* __restrict__ mlp, const int32_t* __restrict__ deg,
                                               const int32_t* __restrict__ vtag, const uint4* __restrict__ cand,
                                               const unsigned int* __restrict__ ncand_p, uint32_t cand_cap,
                                               uint4* __restrict__ tiles_task, unsigned int* __restrict__ ntiles_task,
                                               uint4* __restrict__ stream_task, unsigned int* __restrict__ nstream,
                                               uint32_t cap, int stream_max, int* __restrict__ overflow) {
    __shared__ __align__(16) __half2 w[MLPH_N + 2];
    for (int k = threadIdx.x; k < MLPH_N; k += blockDim.x) w[k] = mlp[k];
    __syncthreads();
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const unsigned n = min(*ncand_p, cand_cap);
    for (unsigned base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const unsigned i = base + threadIdx.x;
        const bool has = i < n;
        uint4 r = make_uint4(0, 0, 0, 0);
        bool to_stream = false;
        if (has) {
            r = cand[i];
            const int du = deg[r.x], dv = deg[r.y];
            const int ds = min(du, dv), dg = max(du, dv);
            const bool us = du <= dv;
            float f[MLP_IN], pr[MLP_OUT];
            task_features(ds, dg, vtag + 3 * (size_t)(us ? r.x : r.y), vtag + 3 * (size_t)(us ? r.y : r.x), f);
            mlp_predict_h(w, f, pr);
            to_stream = ds <= min(stream_max, STREAM_SMAX) && pr[3] < pr[2];
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const bool mine = has && (k == 0 ? to_stream : !to_stream);
            const unsigned m = __ballot_sync(full, mine);
            if (!m) continue;
            const int leader = __ffs(m) - 1;
            unsigned at = 0;
            if (lane == leader) at = atomicAdd(k == 0 ? nstream : ntiles_task, (unsigned)__popc(m));
            at = __shfl_sync(full, at, leader);
            if (mine) {
                const unsigned idx = at + __popc(m & below);
                if (idx < cap) (k == 0 ? stream_task : tiles_task)[idx] = r;
                else atomicOr(overflow, 1);
            }
        }
    }
}

// --------------------------------------------------------------- k_split --
// Tasks of the split bin, 32 per warp: cut each task's merge of A and B into
// tiles of `tile` outputs, reserve consecutive tile records, and find each
// tile's start on the merge path -- the number of A entries among the first d
// outputs, ties taken from A first -- by binary search.  The tiles of the 32
// tasks are spread over the lanes so that 32 searches are in flight.
__global__ void __launch_bounds__(256) k_split(const int64_t* __restrict__ row_ptr,
                                               const uint32_t* __restrict__ adj,
                                               const uint4* __restrict__ task,
                                               const unsigned int* __restrict__ ntask_p, uint32_t task_cap,
                                               int tile, uint4* __restrict__ tiles,
                                               int32_t* __restrict__ ia_out,
                                               unsigned int* __restrict__ ntile_p, uint32_t tile_cap,
                                               int* __restrict__ overflow, int stream_max, int hub_ratio,
                                               uint4* __restrict__ hub,
                                               uint32_t hub_cap, const unsigned int* __restrict__ nstream_p,
                                               unsigned int* __restrict__ nhub,
                                               unsigned long long* __restrict__ hub_entries) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const unsigned nt = min(*ntask_p, task_cap);
    // hub tasks fill the stream-bin array from its end, below the streamed
    // tasks already there (the two are disjoint sets of dyads)
    const unsigned hub_room = hub_cap - min(*nstream_p, hub_cap);
    unsigned long long he = 0;
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    for (unsigned w0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32u; w0 < nt; w0 += warps * 32u) {
        const unsigned i = w0 + lane;
        const bool has = i < nt;
        const uint4 r = has ? task[i] : make_uint4(0, 0, 0, 0);
        int64_t ab = 0, a = 0, bb = 0, b = 0;
        if (has) {
            ab = row_ptr[r.x];
            a = row_ptr[r.x + 1] - ab;
            bb = row_ptr[r.y];
            b = row_ptr[r.y + 1] - bb;
        }
        // a hub task (shorter list within stream_max, longer list at least
        // hub_ratio times longer) is streamed whole by the hub launch instead
        // of being cut into tiles
        const int64_t sh = min(a, b);
        const bool to_hub = has && sh <= (int64_t)stream_max && max(a, b) >= (int64_t)hub_ratio * sh;
        {
            const unsigned m = __ballot_sync(full, to_hub);
            if (m) {
                const int leader = __ffs(m) - 1;
                unsigned at = 0;
                if (lane == leader) at = atomicAdd(nhub, (unsigned)__popc(m));
                at = __shfl_sync(full, at, leader);
                if (to_hub) {
                    const unsigned idx = at + __popc(m & below);
                    if (idx < hub_room) hub[hub_cap - 1 - idx] = r;
                    else atomicOr(overflow, 1);
                    he += (unsigned long long)(a + b);
                }
            }
        }
        const unsigned ntl = (has && !to_hub) ? (unsigned)((a + b + tile - 1) / tile) : 0u;
        unsigned incl = ntl;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(full, incl, o);
            if (lane >= o) incl += v;
        }
        const unsigned total = __shfl_sync(full, incl, 31);
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(ntile_p, total);
        base = __shfl_sync(full, base, 0);
        for (unsigned k0 = 0; k0 < total; k0 += 32) {
            const unsigned k = k0 + lane;
            // owner lane: the first lane whose inclusive tile count exceeds k
            int lo = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const unsigned v = __shfl_sync(full, incl, lo + step - 1);
                if (v <= k) lo += step;
            }
            const int own = min(lo, 31);
            const unsigned first = __shfl_sync(full, incl - ntl, own);
            const uint32_t ox = __shfl_sync(full, r.x, own), oy = __shfl_sync(full, r.y, own);
            const uint32_t oz = __shfl_sync(full, r.z, own);
            const int64_t oab = __shfl_sync(full, ab, own), oa = __shfl_sync(full, a, own);
            const int64_t obb = __shfl_sync(full, bb, own), ob = __shfl_sync(full, b, own);
            if (k < total) {
                const int64_t d = (int64_t)(k - first) * tile;
                int64_t l2 = max((int64_t)0, d - ob), hi = min(d, oa);
                while (l2 < hi) {
                    const int64_t mid = (l2 + hi) >> 1;
                    if ((__ldg(adj + oab + mid) | 3u) <= (__ldg(adj + obb + d - 1 - mid) | 3u)) l2 = mid + 1;
                    else hi = mid;
                }
                if (base + k < tile_cap) {
                    tiles[base + k] = make_uint4(ox, oy, oz, (uint32_t)d);
                    ia_out[base + k] = (int32_t)l2;
                } else {
                    atomicOr(overflow, 1);
                }
            }
        }
    }
    he = warp_sum64(he);
    if (lane == 0 && he) atomicAdd(hub_entries, he);
}

// ----------------------------------------------------- shared-element fix --
// w is in both N(u) and N(v) (tags tu, tv), u < v < w: the triangle {u,v,w}
// is handled once, by its lowest dyad <u,v>.  For <u,v> its contribution
// moves from the single-list codes pre+4tu and pre+16tv to the joint code;
// for <u,w>, whose middle vertex is v, the single-list code tu + 16 tag_w(v)
// (tag_w(v): tv with its two bits swapped) must not count.  A shared w below
// v is left to the dyad of the triangle's two lowest vertices.
__device__ __forceinline__ uint32_t tag_swap(uint32_t t) { return ((t & 1u) << 1) | (t >> 1); }

__device__ __forceinline__ void on_shared(unsigned long long* h, uint32_t w, uint32_t ul, uint32_t vl,
                                          uint32_t pre, uint32_t tu, uint32_t tv) {
    (void)ul;
    if (w > vl) {
        atomicAdd(h + pre + 4 * tu, ~0ull);
        atomicAdd(h + pre + 16 * tv, ~0ull);
        atomicAdd(h + pre + 4 * tu + 16 * tv, 1ull);
        atomicAdd(h + tu + 16 * tag_swap(tv), ~0ull);
    }
}

template <int WPB>
__device__ __forceinline__ void flush_hist(unsigned long long* hs, unsigned long long* acc, int tag, int lane) {
    if (tag >= 0)
        for (int j = lane; j < ACC; j += 32) {
            const unsigned long long v = hs[j];
            if (v) atomicAdd(acc + (size_t)tag * ACC + j, v);
            hs[j] = 0;
        }
    else
        for (int j = lane; j < ACC; j += 32) hs[j] = 0;
}

// --------------------------------------------------------- per-warp state --
// Each warp accumulates into its own 66-slot histogram in shared memory,
// tagged with the graph (segment) it currently counts for; when the graph
// changes the histogram is flushed into that graph's accumulators.
struct WarpHist {
    unsigned long long* hs;
    unsigned long long* acc;
    int tag;
    int lane;
    const Instr* ins = nullptr;
    __device__ __forceinline__ void retag(int s) {
        if (s != tag) {
            flush_hist<WARPS>(hs, acc, tag, lane);
            __syncwarp();
            tag = s;
        }
    }
};

// ---------------------------------------------------------- thread items --
// One thread per small task (32 consecutive tasks per warp item): a plain
// two-pointer merge from global memory.  A lane whose task belongs to
// another graph than the warp's histogram adds into global memory directly.
// Only shared elements above v change a code through this dyad (on_shared),
// so with `split` (entries of each row below its own id) both lists start
// above v: v's own split point, and in u's list the entry after v, whose
// position the task record carries in .w (the task pass knows it).
template <bool INS>
__device__ __forceinline__ void thread_item(WarpHist& w, const int64_t* __restrict__ row_ptr,
                                            const uint32_t* __restrict__ adj, const SegDev* __restrict__ seg,
                                            const int32_t* __restrict__ split, const uint4* __restrict__ rec,
                                            unsigned base, unsigned ntask) {
    const unsigned ti = base + w.lane;
    const bool has = ti < ntask;
    const uint4 r = has ? rec[ti] : make_uint4(0, 0, 0, 0);
    const int s = (int)(r.z >> 2);
    w.retag(__shfl_sync(0xffffffffu, s, 0));
    unsigned long long* h = (s == w.tag) ? w.hs : w.acc + (size_t)s * ACC;
    if (has) {
        const long long t0 = INS ? clock64() : 0;
        uint32_t c = 0;
        const uint32_t pre = r.z & 3u;
        const int64_t rb = seg[s].rb;
        const uint32_t ul = (uint32_t)(r.x - rb), vl = (uint32_t)(r.y - rb);
        int64_t ia = row_ptr[r.x], ib = row_ptr[r.y];
        const int64_t ae = row_ptr[r.x + 1], be = row_ptr[r.y + 1];
        if (split) {
            ia += r.w;
            ib += split[r.y];
        }
        uint32_t eA = ia < ae ? __ldg(adj + ia) : SENT;
        uint32_t eB = ib < be ? __ldg(adj + ib) : SENT;
        for (;;) {
            const uint32_t kA = eA | 3u, kB = eB | 3u;
            if (kA == SENT && kB == SENT) break;
            if (kA == kB) {
                ++c;
                on_shared(h, kA >> 2, ul, vl, pre, eA & 3u, eB & 3u);
                ++ia;
                ++ib;
                eA = ia < ae ? __ldg(adj + ia) : SENT;
                eB = ib < be ? __ldg(adj + ib) : SENT;
            } else if (kA < kB) {
                ++ia;
                eA = ia < ae ? __ldg(adj + ia) : SENT;
            } else {
                ++ib;
                eB = ib < be ? __ldg(adj + ib) : SENT;
            }
        }
        (void)c;  // shared elements: their dyadic share comes from the closed-triad counts (k_fold)
        if (INS && sampled(w.ins, r.x, r.y)) record(w.ins, r.x, r.y, 0, clock64() - t0);
    }
    __syncwarp();
}

__global__ void __launch_bounds__(256) k_thread(const int64_t* __restrict__ row_ptr,
                                                const uint32_t* __restrict__ adj,
                                                const SegDev* __restrict__ seg,
                                                const int32_t* __restrict__ split,
                                                const uint4* __restrict__ rec,
                                                const unsigned int* __restrict__ cnt, uint32_t cap,
                                                unsigned long long* __restrict__ acc) {
    __shared__ unsigned long long hs_all[WARPS][ACC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpHist w{hs_all[warp], acc, -1, lane};
    for (int j = lane; j < ACC; j += 32) w.hs[j] = 0;
    __syncwarp();
    const unsigned ntask = min(*cnt, cap);
    for (unsigned base = (blockIdx.x * WARPS + warp) * 32u; base < ntask; base += gridDim.x * WARPS * 32u)
        thread_item<false>(w, row_ptr, adj, seg, split, rec, base, ntask);
    __syncwarp();
    flush_hist<WARPS>(w.hs, acc, w.tag, lane);
}

// ------------------------------------------------------- merge spans (a3) --
// A span of a neighbour list is copied to shared memory with 16-byte loads
// from the 16-byte boundary at or below its start; the returned offset is
// where the span begins in `raw`.  Words at absolute positions >= lim are
// stored as the sentinel.  `count` words after the start are guaranteed.
template <int NT>
__device__ __forceinline__ int load_span(uint32_t* __restrict__ raw, const uint32_t* __restrict__ adj,
                                         int64_t p, int count, int64_t lim, int tid) {
    const int64_t q = p & ~(int64_t)3;
    const int o = (int)(p - q);
    const int nq = (o + count + 3) >> 2;
    const uint4* src = reinterpret_cast<const uint4*>(adj + q);
    uint4* dst = reinterpret_cast<uint4*>(raw);
    for (int m = tid; m < nq; m += NT) {
        uint4 x = __ldg(src + m);
        const int64_t a = q + 4 * (int64_t)m;
        if (a + 3 >= lim) {
            x.x = a < lim ? x.x : SENT;
            x.y = a + 1 < lim ? x.y : SENT;
            x.z = a + 2 < lim ? x.z : SENT;
            x.w = a + 3 < lim ? x.w : SENT;
        }
        dst[m] = x;
    }
    return o;
}

// load_span for a list addressed by pointer, with 32-bit positions relative
// to it: `count` words from p, those at relative index >= lim stored as the
// sentinel.  Returns the span's offset in `raw`.
__device__ __forceinline__ int load_span_p(uint32_t* __restrict__ raw, const uint32_t* __restrict__ p, int count,
                                           int lim, int lane) {
    const int o = (int)(((uintptr_t)p >> 2) & 3);
    const uint4* src = reinterpret_cast<const uint4*>(p - o);
    uint4* dst = reinterpret_cast<uint4*>(raw);
    const int nq = (o + count + 3) >> 2;
    const int lo = lim + o;  // limit relative to the aligned start
    for (int m = lane; m < nq; m += 32) {
        uint4 x = __ldg(src + m);
        const int a = 4 * m;
        if (a + 3 >= lo) {
            x.x = a < lo ? x.x : SENT;
            x.y = a + 1 < lo ? x.y : SENT;
            x.z = a + 2 < lo ? x.z : SENT;
            x.w = a + 3 < lo ? x.w : SENT;
        }
        dst[m] = x;
    }
    return o;
}

__device__ __forceinline__ int ceil_log2(int x) {  // smallest k with 2^k >= x (x >= 1)
    return 32 - __clz(max(x, 1) - 1);
}

// Shared elements of A[0..na) and B[0..nb) (sorted spans in shared memory),
// found by one of two exact strategies over the same data:
//  * search: every element of the shorter span is located in the longer one
//    by binary search (cheap when one span is much shorter: hub vs leaf);
//  * merge: the merge path of the two spans is cut at equal diagonals, one
//    cut per thread (binary search), and each thread takes its steps of the
//    two-pointer merge; an element of A taken while the equal element of B
//    is at the B head is a shared element (ties are taken from A first).
// A[na] must be the sentinel and B[nb] must be the element that follows the
// span in B (or the sentinel): the merge then also reports the pair
// (A[na-1], B[nb]) -- an element shared across the span boundary -- and the
// search strategy checks that pair explicitly when `boundary` is set.
template <int NT>
__device__ __forceinline__ uint32_t shared_elements(const uint32_t* sA, int na, const uint32_t* sB, int nb,
                                                    bool boundary, uint32_t ul, uint32_t vl, uint32_t pre,
                                                    unsigned long long* h, int tid) {
    uint32_t c = 0;
    const int tot = na + nb;
    const int ns = min(na, nb), nl = max(na, nb);
    if (ns == 0 && !boundary) return 0;
    // issue-slot estimates of the two strategies (per thread: a search step
    // ~7 instructions, a merge step ~12)
    const int search_cost = ((ns + NT - 1) / NT) * (ceil_log2(nl + 1) + 1) * 7;
    const int merge_cost = ((tot + NT - 1) / NT) * 12 + ceil_log2(tot + 1) * 9;
    if (search_cost <= merge_cost) {
        const bool small_is_A = na <= nb;
        const uint32_t* sm = small_is_A ? sA : sB;
        const uint32_t* lg = small_is_A ? sB : sA;
        for (int k = tid; k < ns; k += NT) {
            const uint32_t x = sm[k];
            const uint32_t key = x | 3u;
            int lo = 0, hi = nl;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((lg[mid] | 3u) < key) lo = mid + 1;
                else hi = mid;
            }
            if (lo < nl) {
                const uint32_t y = lg[lo];
                if ((y | 3u) == key) {
                    ++c;
                    on_shared(h, key >> 2, ul, vl, pre, small_is_A ? (x & 3u) : (y & 3u),
                              small_is_A ? (y & 3u) : (x & 3u));
                }
            }
        }
        if (boundary && tid == 0 && na > 0) {
            const uint32_t x = sA[na - 1], y = sB[nb];
            if ((x | 3u) == (y | 3u)) {
                ++c;
                on_shared(h, x >> 2, ul, vl, pre, x & 3u, y & 3u);
            }
        }
    } else {
        // odd step count: balanced lanes start an odd stride apart, spreading
        // their shared-memory reads over the banks
        const int K = ((tot + NT - 1) / NT) | 1;
        const int dl = min(tid * K, tot);
        const int steps = min(K, tot - dl);
        int lo = max(0, dl - nb), hi = min(dl, na);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((sA[mid] | 3u) <= (sB[dl - 1 - mid] | 3u)) lo = mid + 1;
            else hi = mid;
        }
        int ia = lo, ib = dl - lo;
        uint32_t eA = sA[ia], eB = sB[ib];
        for (int s = 0; s < steps; ++s) {
            const uint32_t kA = eA | 3u, kB = eB | 3u;
            const bool takeA = kA <= kB;
            if (kA == kB) {
                ++c;
                on_shared(h, kA >> 2, ul, vl, pre, eA & 3u, eB & 3u);
            }
            ia += takeA;
            ib += !takeA;
            const uint32_t nx = takeA ? sA[ia] : sB[ib];
            eA = takeA ? nx : eA;
            eB = takeA ? eB : nx;
        }
    }
    return c;
}

// ------------------------------------------------------------ warp items --
// One warp per record.  Without ia_start a record is a whole task with
// |A|+|B| <= WARP_LMAX: both lists, each followed by a sentinel, are copied
// into the warp's shared memory.  With ia_start a record is one tile of at
// most `tile` merge outputs of a larger task: it starts where k_split put it
// on the merge path and ends where the task's next tile starts (or at the end
// of both lists), so exactly the spans A[is..ie) and B[js..je) are loaded,
// plus B[je] for the pair that straddles the tile boundary.
constexpr int WARP_LMAX = 1024;
constexpr int WARP_BUF = WARP_LMAX + 16;  // words of shared memory per warp

template <bool INS>
__device__ __forceinline__ void warp_item(WarpHist& w, uint32_t* raw, const int64_t* __restrict__ row_ptr,
                                          const uint32_t* __restrict__ adj, const SegDev* __restrict__ seg,
                                          const int32_t* __restrict__ split, const uint4* __restrict__ rec,
                                          const int32_t* __restrict__ ia_start, unsigned i, unsigned nrec,
                                          int tile) {
    const int lane = w.lane;
    const long long t0 = INS ? clock64() : 0;
    const uint4 r = rec[i];
    const int s = (int)(r.z >> 2);
    const uint32_t pre = r.z & 3u;
    w.retag(s);
    const int64_t rb = seg[s].rb;
    const int64_t ab = row_ptr[r.x], ae = row_ptr[r.x + 1];
    const int64_t bb = row_ptr[r.y], be = row_ptr[r.y + 1];
    int64_t is = 0, ie = ae - ab, js = 0, je = be - bb;
    if (ia_start) {
        const int64_t L = ie + je, d0 = r.w, d1 = min(d0 + (int64_t)tile, L);
        is = ia_start[i];
        ie = d1 == L ? ie : (int64_t)ia_start[min(i + 1, nrec - 1)];
        js = d0 - is;
        je = d1 - ie;
    } else if (split) {  // a whole task: both lists from above v (see thread_item)
        is = r.w;
        js = split[r.y];
    }
    const int na = (int)(ie - is), nb = (int)(je - js);
    const int oA = load_span<32>(raw, adj, ab + is, na + 1, ab + ie, lane);
    uint32_t* rawB = raw + ((oA + na + 1 + 3) & ~3);
    const int oB = load_span<32>(rawB, adj, bb + js, nb + 1, min(bb + je + 1, be), lane);
    __syncwarp();
    shared_elements<32>(raw + oA, na, rawB + oB, nb, ia_start != nullptr, (uint32_t)(r.x - rb), (uint32_t)(r.y - rb),
                        pre, w.hs, lane);
    __syncwarp();
    if (INS && lane == 0 && sampled(w.ins, r.x, r.y))
        record(w.ins, r.x, r.y, ia_start ? 2 : 1, clock64() - t0);
}

__global__ void __launch_bounds__(256) k_warp(const int64_t* __restrict__ row_ptr,
                                              const uint32_t* __restrict__ adj,
                                              const SegDev* __restrict__ seg,
                                              const int32_t* __restrict__ split,
                                              const uint4* __restrict__ rec,
                                              const int32_t* __restrict__ ia_start,
                                              const unsigned int* __restrict__ cnt, uint32_t cap,
                                              int tile, unsigned long long* __restrict__ acc) {
    __shared__ __align__(16) uint32_t sbuf[WARPS][WARP_BUF];
    __shared__ unsigned long long hs_all[WARPS][ACC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpHist w{hs_all[warp], acc, -1, lane};
    for (int j = lane; j < ACC; j += 32) w.hs[j] = 0;
    __syncwarp();
    const unsigned ntask = min(*cnt, cap);
    for (unsigned i = blockIdx.x * WARPS + warp; i < ntask; i += gridDim.x * WARPS)
        warp_item<false>(w, sbuf[warp], row_ptr, adj, seg, split, rec, ia_start, i, ntask, tile);
    __syncwarp();
    flush_hist<WARPS>(w.hs, acc, w.tag, lane);
}

// ---------------------------------------------------------- stream items --
// One warp per task whose shorter list S has at most STREAM_SMAX entries
// (the longer list G may be a hub's).  S is copied to shared memory (followed
// by a sentinel); G is streamed through registers in steps of 32*EPL entries
// (EPL consecutive entries per lane, 16-byte loads), every entry of G being
// read once.  At each step the entries of S whose keys do not exceed the
// step's last key are located: with few of them, each is broadcast and every
// lane compares it with its own entries; otherwise the lane holding a key is
// the first lane whose last key is not smaller (a 5-step search over the
// lanes by shuffles).  Both lists are sorted, so each entry of S is placed in
// exactly one step and every shared element is found once.
static_assert(STREAM_SMAX + 8 <= WARP_BUF, "stream buffer fits the warp buffer");

template <int EPL, bool INS>
__device__ __forceinline__ void stream_item(WarpHist& w, uint32_t* buf, const int64_t* __restrict__ row_ptr,
                                            const uint32_t* __restrict__ adj, const SegDev* __restrict__ seg,
                                            const int32_t* __restrict__ split, const uint4 r) {
    constexpr int STEP = 32 * EPL;
    constexpr int NQ = EPL / 4;  // 16-byte loads per lane per step
    const unsigned full = 0xffffffffu;
    const int lane = w.lane;
    const long long t0 = INS ? clock64() : 0;
    const int s = (int)(r.z >> 2);
    const uint32_t pre = r.z & 3u;
    w.retag(s);
    const int64_t rb = seg[s].rb;
    const uint32_t ul = (uint32_t)(r.x - rb), vl = (uint32_t)(r.y - rb);
    // both lists from above v (see thread_item)
    const int64_t ab = row_ptr[r.x] + (split ? r.w : 0), ae = row_ptr[r.x + 1];
    const int64_t bb = row_ptr[r.y] + (split ? split[r.y] : 0), be = row_ptr[r.y + 1];
    const bool s_is_A = (ae - ab) <= (be - bb);
    const int64_t pS = s_is_A ? ab : bb;
    const int nS = (int)(s_is_A ? ae - ab : be - bb);
    const int64_t pG = s_is_A ? bb : ab, gend = s_is_A ? be : ae;
    const int oS = load_span<32>(buf, adj, pS, nS + 1, pS + nS, lane);
    const uint32_t* sS = buf + oS;
    __syncwarp();
    int js = 0;
    uint32_t c = 0;
    for (int64_t base = pG & ~(int64_t)3; base < gend; base += STEP) {
        const int64_t e0 = base + EPL * lane;
        uint32_t v[EPL];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const uint4 x = __ldg(reinterpret_cast<const uint4*>(adj + e0) + q);
            v[4 * q] = x.x;
            v[4 * q + 1] = x.y;
            v[4 * q + 2] = x.z;
            v[4 * q + 3] = x.w;
        }
        uint32_t lane_last;
        if (base < pG || base + STEP > gend) {  // first or last step: mask foreign entries
#pragma unroll
            for (int j = 0; j < EPL; ++j) {
                const int64_t idx = e0 + j;
                v[j] = (idx >= pG && idx < gend) ? v[j] : SENT;  // never equal to a real key
            }
            lane_last = e0 + EPL - 1 < pG ? 0u : (e0 + EPL - 1 >= gend ? SENT : (v[EPL - 1] | 3u));
        } else {
            lane_last = v[EPL - 1] | 3u;
        }
        const uint32_t step_last = __shfl_sync(full, lane_last, 31);
        for (;;) {
            const int jj = js + lane;
            const uint32_t t = sS[min(jj, nS)];  // sS[nS] is the sentinel
            const uint32_t tkey = t | 3u;
            const bool inr = jj < nS && tkey <= step_last;
            const unsigned m = __ballot_sync(full, inr);
            if (m == 0) break;
            const int k = __popc(m);
            if (k <= 3) {
                for (int q = 0; q < k; ++q) {
                    const uint32_t tq = __shfl_sync(full, t, q);
                    const uint32_t qkey = tq | 3u;
                    uint32_t hit = SENT;
#pragma unroll
                    for (int j = 0; j < EPL; ++j) hit = (v[j] | 3u) == qkey ? v[j] : hit;
                    if (hit != SENT) {
                        ++c;
                        on_shared(w.hs, qkey >> 2, ul, vl, pre, s_is_A ? (tq & 3u) : (hit & 3u),
                                  s_is_A ? (hit & 3u) : (tq & 3u));
                    }
                }
                js += k;
                break;  // k < 32: the rest of S lies beyond this step
            }
            int own = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const uint32_t x = __shfl_sync(full, lane_last, own + step - 1);
                if (x < tkey) own += step;
            }
            own = min(own, 31);
            uint32_t hit = SENT;
#pragma unroll
            for (int j = 0; j < EPL; ++j) {
                const uint32_t x = __shfl_sync(full, v[j], own);
                hit = (x | 3u) == tkey ? x : hit;
            }
            if (inr && hit != SENT) {
                ++c;
                on_shared(w.hs, tkey >> 2, ul, vl, pre, s_is_A ? (t & 3u) : (hit & 3u),
                          s_is_A ? (hit & 3u) : (t & 3u));
            }
            js += k;
            if (k < 32) break;
        }
    }
    (void)c;
    __syncwarp();
    if (INS && lane == 0 && sampled(w.ins, r.x, r.y)) record(w.ins, r.x, r.y, 3, clock64() - t0);
}

// Stream-bin tasks, one per warp.
template <int EPL>
__global__ void __launch_bounds__(256) k_stream(const int64_t* __restrict__ row_ptr,
                                                const uint32_t* __restrict__ adj,
                                                const SegDev* __restrict__ seg,
                                                const int32_t* __restrict__ split,
                                                const uint4* __restrict__ rec,
                                                const unsigned int* __restrict__ cnt, uint32_t cap,
                                                unsigned long long* __restrict__ acc) {
    __shared__ __align__(16) uint32_t sbuf[WARPS][WARP_BUF];
    __shared__ unsigned long long hs_all[WARPS][ACC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpHist w{hs_all[warp], acc, -1, lane};
    for (int j = lane; j < ACC; j += 32) w.hs[j] = 0;
    __syncwarp();
    const unsigned ntask = min(*cnt, cap);
    for (unsigned i = blockIdx.x * WARPS + warp; i < ntask; i += gridDim.x * WARPS)
        stream_item<EPL, false>(w, sbuf[warp], row_ptr, adj, seg, split, rec[i]);
    __syncwarp();
    flush_hist<WARPS>(w.hs, acc, w.tag, lane);
}

// ------------------------------------------------------------ hub items --
// A streamed task whose shorter list S is longer than STREAM_SMAX (both
// endpoints are hubs).  As a stream item, but S is staged STREAM_SMAX entries
// at a time, each piece followed by a sentinel; when a piece is used up inside
// a step of G the next one is staged and the same step is matched again.  Kept
// out of the persistent merge so that its extra state does not cost that
// kernel registers (occupancy).
template <int EPL>
__device__ __forceinline__ void hub_item(WarpHist& w, uint32_t* buf, const int64_t* __restrict__ row_ptr,
                                            const uint32_t* __restrict__ adj, const SegDev* __restrict__ seg,
                                            const int32_t* __restrict__ split, const uint4 r) {
    constexpr int STEP = 32 * EPL;
    constexpr int NQ = EPL / 4;  // 16-byte loads per lane per step
    const unsigned full = 0xffffffffu;
    const int lane = w.lane;
    const int s = (int)(r.z >> 2);
    const uint32_t pre = r.z & 3u;
    w.retag(s);
    const int64_t rb = seg[s].rb;
    const uint32_t ul = (uint32_t)(r.x - rb), vl = (uint32_t)(r.y - rb);
    // both lists from above v (see thread_item)
    const int64_t ab = row_ptr[r.x] + (split ? r.w : 0), ae = row_ptr[r.x + 1];
    const int64_t bb = row_ptr[r.y] + (split ? split[r.y] : 0), be = row_ptr[r.y + 1];
    const bool s_is_A = (ae - ab) <= (be - bb);
    const uint32_t* Sp = adj + (s_is_A ? ab : bb);
    const int nS = (int)(s_is_A ? ae - ab : be - bb);
    // G from its 16-byte boundary: valid relative offsets [lead, glen)
    const int64_t pG = s_is_A ? bb : ab;
    const int lead = (int)(pG & 3);
    const uint32_t* Gp = adj + (pG - lead);
    const int glen = (int)((s_is_A ? be : ae) - (pG - lead));
    // S is staged STREAM_SMAX entries at a time; chunk [sc, sc+cs) is followed
    // by the sentinel in shared memory
    int sc = 0, cs = min(nS, STREAM_SMAX);
    const uint32_t* sS = buf + load_span_p(buf, Sp, cs + 1, cs, lane);
    __syncwarp();
    int js = 0;
    uint32_t c = 0;
    for (int off = 0; off < glen; off += STEP) {
        const int e0 = off + EPL * lane;
        uint32_t v[EPL];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const uint4 x = __ldg(reinterpret_cast<const uint4*>(Gp + e0) + q);
            v[4 * q] = x.x;
            v[4 * q + 1] = x.y;
            v[4 * q + 2] = x.z;
            v[4 * q + 3] = x.w;
        }
        uint32_t lane_last;
        if (off < lead || off + STEP > glen) {  // first or last step: mask foreign entries
#pragma unroll
            for (int j = 0; j < EPL; ++j) v[j] = (e0 + j >= lead && e0 + j < glen) ? v[j] : SENT;
            lane_last = e0 + EPL - 1 < lead ? 0u : (e0 + EPL - 1 >= glen ? SENT : (v[EPL - 1] | 3u));
        } else {
            lane_last = v[EPL - 1] | 3u;
        }
        const uint32_t step_last = __shfl_sync(full, lane_last, 31);
        for (;;) {
            if (js == cs && sc + cs < nS) {  // chunk used up: stage the next, same step
                __syncwarp();
                sc += cs;
                cs = min(nS - sc, STREAM_SMAX);
                js = 0;
                sS = buf + load_span_p(buf, Sp + sc, cs + 1, cs, lane);
                __syncwarp();
            }
            const int jj = js + lane;
            const uint32_t t = sS[min(jj, cs)];  // sS[cs] is the sentinel
            const uint32_t tkey = t | 3u;
            const bool inr = jj < cs && tkey <= step_last;
            const unsigned m = __ballot_sync(full, inr);
            if (m == 0) break;
            const int k = __popc(m);
            if (k <= 3) {
                for (int q = 0; q < k; ++q) {
                    const uint32_t tq = __shfl_sync(full, t, q);
                    const uint32_t qkey = tq | 3u;
                    uint32_t hit = SENT;
#pragma unroll
                    for (int j = 0; j < EPL; ++j) hit = (v[j] | 3u) == qkey ? v[j] : hit;
                    if (hit != SENT) {
                        ++c;
                        on_shared(w.hs, qkey >> 2, ul, vl, pre, s_is_A ? (tq & 3u) : (hit & 3u),
                                  s_is_A ? (hit & 3u) : (tq & 3u));
                    }
                }
                js += k;
                if (js == cs && sc + cs < nS) continue;  // next chunk may lie in this step
                break;  // the rest of S lies beyond this step
            }
            int own = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const uint32_t x = __shfl_sync(full, lane_last, own + step - 1);
                if (x < tkey) own += step;
            }
            own = min(own, 31);
            uint32_t hit = SENT;
#pragma unroll
            for (int j = 0; j < EPL; ++j) {
                const uint32_t x = __shfl_sync(full, v[j], own);
                hit = (x | 3u) == tkey ? x : hit;
            }
            if (inr && hit != SENT) {
                ++c;
                on_shared(w.hs, tkey >> 2, ul, vl, pre, s_is_A ? (t & 3u) : (hit & 3u),
                          s_is_A ? (hit & 3u) : (t & 3u));
            }
            js += k;
            if (k < 32 && !(js == cs && sc + cs < nS)) break;
        }
    }
    (void)c;
    __syncwarp();
}


// Hub tasks, one per warp; k_split stores them from the end of the
// stream-bin array.
template <int EPL>
__global__ void __launch_bounds__(256) k_hub(const int64_t* __restrict__ row_ptr,
                                             const uint32_t* __restrict__ adj,
                                             const SegDev* __restrict__ seg,
                                             const int32_t* __restrict__ split,
                                             const uint4* __restrict__ rec,
                                             const unsigned int* __restrict__ cnt, uint32_t cap,
                                             unsigned long long* __restrict__ acc) {
    __shared__ __align__(16) uint32_t sbuf[WARPS][WARP_BUF];
    __shared__ unsigned long long hs_all[WARPS][ACC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpHist w{hs_all[warp], acc, -1, lane};
    for (int j = lane; j < ACC; j += 32) w.hs[j] = 0;
    __syncwarp();
    const unsigned ntask = min(*cnt, cap);
    for (unsigned i = blockIdx.x * WARPS + warp; i < ntask; i += gridDim.x * WARPS)
        hub_item<EPL>(w, sbuf[warp], row_ptr, adj, seg, split, rec[cap - 1 - i]);
    __syncwarp();
    flush_hist<WARPS>(w.hs, acc, w.tag, lane);
}

// ---------------------------------------------------------------- k_merge --
// The whole merge phase in one persistent launch: warps pull work from the
// four bins in decreasing order of task size (streamed tasks, tiles of split
// tasks, whole warp tasks, groups of 32 thread tasks), each bin through its
// own atomic cursor, so no bin waits for another kernel's tail.
struct MergeQueues {
    const uint4* rec[NBIN];       // bin records (rec[2] unused: tiles below)
    const unsigned int* cnt;      // records per bin
    uint32_t cap[NBIN];
    const uint4* tiles;           // tile records of split tasks
    const int32_t* ia;            // their merge-path starts
    const unsigned int* ntile;
    uint32_t tile_cap;
    int tile;
    unsigned int* cursor;         // [4] per-queue cursors, zeroed before launch
    const int32_t* split;         // per row: entries below its own id (whole tasks start above v)
    Instr ins;                    // per-task timing (ins.buf null: off)
};

template <int EPL, bool INS>
__global__ void __launch_bounds__(256) k_merge(const int64_t* __restrict__ row_ptr,
                                               const uint32_t* __restrict__ adj,
                                               const SegDev* __restrict__ seg, MergeQueues q,
                                               unsigned long long* __restrict__ acc) {
    __shared__ __align__(16) uint32_t sbuf[WARPS][WARP_BUF];
    __shared__ unsigned long long hs_all[WARPS][ACC];
    const unsigned full = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpHist w{hs_all[warp], acc, -1, lane, INS ? &q.ins : nullptr};
    for (int j = lane; j < ACC; j += 32) w.hs[j] = 0;
    __syncwarp();
    const unsigned n3 = min(q.cnt[3], q.cap[3]);
    const unsigned nt = min(*q.ntile, q.tile_cap);
    const unsigned n1 = min(q.cnt[1], q.cap[1]);
    const unsigned n0 = min(q.cnt[0], q.cap[0]);
    const unsigned n0g = (n0 + 31) / 32;
    // queue k: items, items taken per cursor step
    const unsigned items[4] = {n3, nt, n1, n0g};
    const unsigned grab[4] = {1, 2, 4, 2};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        for (;;) {
            unsigned at = 0;
            if (lane == 0) at = atomicAdd(q.cursor + k, grab[k]);
            at = __shfl_sync(full, at, 0);
            if (at >= items[k]) break;
            const unsigned end = min(at + grab[k], items[k]);
            for (unsigned i = at; i < end; ++i) {
                if (k == 0) stream_item<EPL, INS>(w, sbuf[warp], row_ptr, adj, seg, q.split, q.rec[3][i]);
                else if (k == 1)
                    warp_item<INS>(w, sbuf[warp], row_ptr, adj, seg, q.split, q.tiles, q.ia, i, nt, q.tile);
                else if (k == 2)
                    warp_item<INS>(w, sbuf[warp], row_ptr, adj, seg, q.split, q.rec[1], nullptr, i, n1, 0);
                else thread_item<INS>(w, row_ptr, adj, seg, q.split, q.rec[0], i * 32u, n0);
            }
        }
    }
    __syncwarp();
    flush_hist<WARPS>(w.hs, acc, w.tag, lane);
}

// ---------------------------------------------------------------- k_cta --
// One CTA per tile of at most TILE merge outputs of a large task.  The tile
// starts where k_split put it on the merge path and ends where the task's
// next tile starts (or at the end of both lists), so exactly the tile's spans
// A[is..ie) and B[js..je) are loaded, plus B[je] for the boundary pair.
constexpr int CTA_NT = 256;
constexpr int TILE = 3840;

__global__ void __launch_bounds__(CTA_NT) k_cta(const int64_t* __restrict__ row_ptr,
                                                const uint32_t* __restrict__ adj,
                                                const SegDev* __restrict__ seg,
                                                const uint4* __restrict__ rec,
                                                const int32_t* __restrict__ ia_start,
                                                const unsigned int* __restrict__ cnt, uint32_t cap,
                                                int tile, unsigned long long* __restrict__ acc) {
    __shared__ __align__(16) uint32_t rawA[TILE + 8];
    __shared__ __align__(16) uint32_t rawB[TILE + 8];
    __shared__ unsigned long long hs[ACC];
    const int tid = threadIdx.x, lane = tid & 31;
    for (int j = tid; j < ACC; j += CTA_NT) hs[j] = 0;
    __syncthreads();
    int tag = -1;
    const unsigned n2 = min(*cnt, cap);
    for (unsigned i = blockIdx.x; i < n2; i += gridDim.x) {
        const uint4 r = rec[i];
        const int s = (int)(r.z >> 2);
        const uint32_t pre = r.z & 3u;
        __syncthreads();  // the previous tile's shared-memory reads are done
        if (s != tag) {
            if (tid < 32) flush_hist<1>(hs, acc, tag, lane);
            __syncthreads();
            tag = s;
        }
        const int64_t rb = seg[s].rb;
        const int64_t ab = row_ptr[r.x], ae = row_ptr[r.x + 1];
        const int64_t bb = row_ptr[r.y], be = row_ptr[r.y + 1];
        const int64_t a = ae - ab, L = a + (be - bb);
        const int64_t d0 = r.w, d1 = min(d0 + (int64_t)tile, L);
        const int64_t is = ia_start[i];
        const int64_t ie = d1 == L ? a : (int64_t)ia_start[min(i + 1, n2 - 1)];
        const int64_t js = d0 - is, je = d1 - ie;
        const int na = (int)(ie - is), nb = (int)(je - js);
        const int oA = load_span<CTA_NT>(rawA, adj, ab + is, na + 1, ab + ie, tid);
        const int oB = load_span<CTA_NT>(rawB, adj, bb + js, nb + 1, min(bb + je + 1, be), tid);
        __syncthreads();
        shared_elements<CTA_NT>(rawA + oA, na, rawB + oB, nb, true, (uint32_t)(r.x - rb), (uint32_t)(r.y - rb), pre,
                                hs, tid);
    }
    __syncthreads();
    if (tid < 32) flush_hist<1>(hs, acc, tag, lane);
}

// ---------------------------------------------------------------- k_fold --
// 64 codes -> 16 MAN types; 003 = C(n,3) - the rest, in 128-bit (Sec. 2.2).
// With raw non-null (a shard of the census) the accumulators themselves go
// to raw[slot]: shards are summed word by word before they are folded.
__global__ void k_fold(const unsigned long long* __restrict__ acc, const SegDev* __restrict__ seg, int nseg,
                       tc_census_t* __restrict__ out, tc_census64_t* __restrict__ codes,
                       unsigned long long* __restrict__ raw) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const unsigned long long* h = acc + (size_t)s * ACC;
    if (raw) {
        for (int w = 0; w < ACC; ++w) raw[(size_t)seg[s].slot * ACC + w] = h[w];
        return;
    }
    unsigned long long cnt[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) cnt[t] = 0;
    for (int code = 0; code < 64; ++code) cnt[triad_type(code)] += h[code];
    // Slots 64..66 hold sum (n - |N(u)| - |N(v)|) over the dyads with
    // pre = 1, 2, 3; the dyadic term n - |S| - 2 adds c_uv = |N(u) n N(v)|
    // per dyad.  A triad whose three pairs are all adjacent adds 1 to c_uv of
    // each of its dyads, so sum_asym c_uv = 3(030T + 030C) + 2(120D + 120U +
    // 120C) + 210 and sum_mutual c_uv = (120D + 120U + 120C) + 2 * 210 + 3 * 300.
    const unsigned long long c120 = cnt[11] + cnt[12] + cnt[13];
    cnt[1] += h[64] + h[65] + 3 * (cnt[8] + cnt[9]) + 2 * c120 + cnt[14];
    cnt[2] += h[66] + c120 + 2 * cnt[14] + 3 * cnt[15];
    const unsigned __int128 n = (unsigned __int128)(unsigned long long)seg[s].n;
    unsigned __int128 all = n >= 3 ? n * (n - 1) * (n - 2) / 6 : 0;
    for (int t = 1; t < 16; ++t) all -= cnt[t];
    tc_census_t o;
    o.count[0] = (uint64_t)all;
    o.count003_hi = (uint64_t)(all >> 64);
    for (int t = 1; t < 16; ++t) o.count[t] = cnt[t];
    out[seg[s].slot] = o;
    if (codes) {
        // the 64 labelled codes (Fig. "Triad Code Algorithm" without the
        // TriadTable step): a connected triad keeps the code of the dyad that
        // counts it; a triad with one adjacent pair has code pre, counted by
        // the dyadic term.  Its c_uv share per pre value: a closed triad is
        // counted with u < v < w, so its three dyads, in canonical order, have
        // pre values pre, t_u(w), t_v(w).
        tc_census64_t c;
        unsigned long long dy[3] = {h[64], h[65], h[66]};
        for (int code = 0; code < 64; ++code) {
            c.count[code] = h[code];
            const int p = code & 3, tu = (code >> 2) & 3, tv = (code >> 4) & 3;
            if (tu && tv)
                for (int q = 1; q <= 3; ++q)
                    dy[q - 1] += h[code] * (unsigned long long)((p == q) + (tu == q) + (tv == q));
        }
        for (int q = 1; q <= 3; ++q) c.count[q] += dy[q - 1];
        c.count[0] = (uint64_t)all;
        c.count0_hi = (uint64_t)(all >> 64);
        codes[seg[s].slot] = c;
    }
}

// ---------------------------------------------------------------- owners --
// Owner tasks (the IsNeighbour query of the method answered by a lookup in
// the owner's list instead of a merge).  For an owner h of degree D the
// neighbour ids are cut into 2^lB buckets by their high bits (2^lB ~ D), and
// each bucket into 16 (owners up to OWN_CAP, whose list is also copied to
// shared memory) or 32 (larger owners) sub-buckets by the next bits.  Shared
// memory holds, per bucket, the start of its entries in h's list and a mask of
// the sub-buckets that hold one.  A key whose sub-bucket bit is clear is
// absent (one shared load, the common case); the others are queued per warp
// and, 32 at a time, looked up by scanning their bucket's few entries (in
// shared memory, or in the list in global memory for larger owners).  The dyads of h are the entries x of h's list that h owns
// (deg x < D, or deg x = D and x < h); every entry w of x's list is looked
// up, and each hit is a shared element of the dyad {h, x}.  Only the shared
// elements are handled here: the per-dyad suffix and dyadic terms of every
// dyad come from k_tasks.
//
// Work item: a piece of at most OWN_PIECE positions of h's list, taken
// OWN_NT positions at a time.  Their owned dyads are compacted into a task
// table (list start, id and tag, running offset of the concatenated lists),
// and each warp takes an equal range of the concatenation, OWN_UNIT entries
// at a time, so a long list is shared by several warps.
constexpr int OWN_NT = 512;
constexpr int OWN_WARPS = OWN_NT / 32;
constexpr int OWN_LBS = 9;   // staged owners: at most 2^9 buckets
constexpr int OWN_LBL = 13;  // larger owners: at most 2^13 buckets
constexpr int OWN_G = 2;     // aligned 16-byte groups per lane per unit
constexpr int OWN_UNIT = 32 * 4 * OWN_G;
// consecutive items a CTA takes at a time from the larger owners (pieces of
// one owner are consecutive, so the CTA indexes it once for all of them)
constexpr unsigned OWN_GRAB = 2;
constexpr size_t own_pad(size_t b) { return (b + 15) / 16 * 16; }
constexpr size_t OWN_T_BYTES = sizeof(uint32_t) * OWN_CAP;
constexpr size_t OWN_ST_BYTES = own_pad(sizeof(uint32_t) * ((1 << OWN_LBS) + 1));
constexpr size_t OWN_HS_BYTES = sizeof(int32_t) * OWN_WARPS * ACC;
constexpr size_t OWN_SB_BYTES = sizeof(int64_t) * OWN_NT;
constexpr size_t OWN_XE_BYTES = sizeof(uint32_t) * OWN_NT;
constexpr size_t OWN_PP_BYTES = own_pad(sizeof(int32_t) * (OWN_NT + 1));
constexpr int OWN_QN = 64;  // per-warp queue of keys that passed the mask test
constexpr size_t OWN_Q_BYTES = (sizeof(uint32_t) + sizeof(uint16_t)) * OWN_QN * OWN_WARPS;
// the index region holds either a staged owner (list T, then its table st)
// or a larger owner (32-bit starts ls, then masks lm)
constexpr size_t OWN_LS_BYTES = own_pad(sizeof(uint32_t) * ((1 << OWN_LBL) + 1));
constexpr size_t OWN_STAGED_BYTES = OWN_T_BYTES + OWN_ST_BYTES;
constexpr size_t OWN_LARGE_BYTES = OWN_LS_BYTES + sizeof(uint32_t) * (1 << OWN_LBL);
constexpr size_t OWN_IDX_BYTES = OWN_STAGED_BYTES > OWN_LARGE_BYTES ? OWN_STAGED_BYTES : OWN_LARGE_BYTES;
constexpr size_t OWN_SMEM =
    OWN_IDX_BYTES + OWN_HS_BYTES + OWN_SB_BYTES + OWN_XE_BYTES + OWN_PP_BYTES + OWN_Q_BYTES;
static_assert(OWN_NT <= 65536, "queued task indices are 16-bit");
// staged owner: st[b] = start << 16 | sub-bucket mask, b in [0, 2^lB]
static_assert(OWN_CAP <= 65535, "staged bucket starts are 16-bit");
// larger owner: 32-bit starts [0, 2^lB] and 32-bit masks [0, 2^lB) in the
// space of the staged list and table
static_assert(OWN_CAP <= (1 << OWN_LBS), "a staged owner has at most one entry per bucket on average");
static_assert(OWN_PIECE % OWN_NT == 0, "an item is a whole number of task tables");

struct OwnArgs {
    const int64_t* row_ptr;
    const uint32_t* adj;
    const int32_t* deg;
    const int32_t* split;    // per row: entries below the row's own id
    const SegDev* seg;
    const uint4* list;       // Bins::own
    uint32_t cap;            // Bins::own_cap
    const unsigned* cnt;     // [2] pieces of larger, smaller owners
    unsigned* cursor;        // [2]
    unsigned long long* acc;
    unsigned long long* lookups;  // keys looked up (profile)
    int64_t* psb;            // per adjacency entry of an owner (k_owner_prep): start of the
    int32_t* plen;           // other endpoint's list part above min(u, v), and its length
};

struct Owner {
    int64_t rb, beg;      // graph's first row; start of the owner's list
    uint32_t hl;          // owner's local id
    uint32_t row;         // owner's global row
    int D, lB, shift, s;  // degree, log2 buckets, key >> shift = bucket, graph
    int fsh, fmask;       // sub-bucket = (key >> fsh) & fmask
    int p0, p1;           // list positions [p0, p1) whose dyads this item handles
};

__device__ __forceinline__ Owner owner_setup(const OwnArgs& a, uint4 rec, int lbmax, int lsub) {
    Owner o;
    o.s = (int)rec.y;
    o.rb = a.seg[o.s].rb;
    const int64_t n = a.seg[o.s].n;
    o.row = rec.x;
    o.hl = (uint32_t)(rec.x - o.rb);
    o.beg = a.row_ptr[rec.x];
    o.D = (int)(a.row_ptr[rec.x + 1] - o.beg);
    const int nbits = ceil_log2((int)min(n, (int64_t)1 << 30));
    o.lB = min(ceil_log2(o.D), lbmax);
    o.shift = max(0, nbits - o.lB);  // key >> shift < 2^lB
    const int sb = min(o.shift, lsub);
    o.fsh = o.shift - sb;
    o.fmask = (1 << sb) - 1;
    o.p0 = (int)rec.z * OWN_PIECE;
    o.p1 = min(o.D, o.p0 + OWN_PIECE);
    return o;
}

// Index of the owner: bucket starts and sub-bucket masks (and, for a staged
// owner, the list).  Starts first (every bucket b in [0, 2^lB] is written by
// exactly one thread), then the masks by atomic OR.
__device__ __forceinline__ int owner_sub(const Owner& o, uint32_t key) { return (int)((key >> o.fsh) & o.fmask); }

template <bool STAGED>
__device__ __forceinline__ void owner_index(const Owner& o, const uint32_t* __restrict__ G, uint32_t* T,
                                            uint32_t* st, uint32_t* ls, uint32_t* lm) {
    const int nb = 1 << o.lB;
    if (!STAGED)
        for (int b = threadIdx.x; b < nb; b += OWN_NT) lm[b] = 0;
    for (int j = threadIdx.x; j < o.D; j += OWN_NT) {
        const uint32_t e = __ldg(G + j);
        if (STAGED) T[j] = e;
        const int bj = (int)((e >> 2) >> o.shift);
        const int bp = j == 0 ? -1 : (int)((__ldg(G + j - 1) >> 2) >> o.shift);
        for (int b = bp + 1; b <= bj; ++b) {
            if (STAGED) st[b] = (uint32_t)j << 16;
            else ls[b] = (uint32_t)j;
        }
        if (j == o.D - 1)
            for (int b = bj + 1; b <= nb; ++b) {
                if (STAGED) st[b] = (uint32_t)o.D << 16;
                else ls[b] = (uint32_t)o.D;
            }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < o.D; j += OWN_NT) {
        const uint32_t key = __ldg(G + j) >> 2;
        const int b = (int)(key >> o.shift);
        const uint32_t bit = 1u << owner_sub(o, key);
        atomicOr((STAGED ? st : lm) + b, bit);
    }
}

// Entry of the owner's list with key `key`, or SENT.
template <bool STAGED>
__device__ __forceinline__ bool owner_maybe(const Owner& o, const uint32_t* st, const uint32_t* lm, uint32_t key) {
    const uint32_t b = key >> o.shift;
    return ((STAGED ? st[b] : lm[b]) >> owner_sub(o, key)) & 1u;
}

template <bool STAGED>
__device__ __forceinline__ uint32_t owner_find(const Owner& o, const uint32_t* L, const uint32_t* st,
                                               const uint32_t* ls, uint32_t key) {
    const uint32_t b = key >> o.shift;
    const int j0 = STAGED ? (int)(st[b] >> 16) : (int)ls[b];
    const int j1 = STAGED ? (int)(st[b + 1] >> 16) : (int)ls[b + 1];
    if (STAGED) {  // the list is in shared memory: scan
        for (int j = j0; j < j1; ++j) {
            const uint32_t e = L[j];
            if ((e >> 2) >= key) return (e >> 2) == key ? e : SENT;
        }
        return SENT;
    }
    // the list is in global memory: up to 8 independent loads per round
    uint32_t hit = SENT;
    for (int j = j0; j < j1; j += 8) {
        uint32_t e[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) e[k] = j + k < j1 ? __ldg(L + j + k) : SENT;
#pragma unroll
        for (int k = 0; k < 8; ++k) hit = (e[k] >> 2) == key ? e[k] : hit;
    }
    return hit;
}

// A shared element w > v of dyad <u,v> (see on_shared): corrections of the
// suffix terms of <u,v> and <u,w>, into the warp's 32-bit histogram.
__device__ __forceinline__ void on_shared32(int32_t* h, uint32_t w, uint32_t vl, uint32_t pre, uint32_t tu,
                                            uint32_t tv) {
    if (w > vl) {
        atomicAdd(h + pre + 4 * tu, -1);
        atomicAdd(h + pre + 16 * tv, -1);
        atomicAdd(h + pre + 4 * tu + 16 * tv, 1);
        atomicAdd(h + tu + 16 * tag_swap(tv), -1);
    }
}

// Per-warp 32-bit histogram for one graph, added (sign-extended) into that
// graph's 64-bit accumulators when the graph changes, at the end, and before
// any slot could leave the int32 range (each shared element moves a slot by
// at most 2, and a work item adds fewer than 2^28 shared elements per warp).
struct OwnHist {
    int32_t* hs;
    unsigned long long* acc;
    int tag;
    int lane;
    unsigned pending;  // shared elements since the last flush
    __device__ __forceinline__ void flush() {
        if (tag >= 0)
            for (int j = lane; j < ACC; j += 32) {
                const int32_t v = hs[j];
                if (v) atomicAdd(acc + (size_t)tag * ACC + j, (unsigned long long)(long long)v);
                hs[j] = 0;
            }
        __syncwarp();
        pending = 0;
    }
    __device__ __forceinline__ void retag(int s) {
        if (s != tag || pending > (1u << 29)) {
            flush();
            tag = s;
        }
    }
};

struct OwnCtl {
    unsigned idx;   // item being processed
    uint32_t row;   // owner indexed in shared memory (~0: none)
    int seg;
    int ntask, total;
    unsigned long long wsum[OWN_WARPS];
};

// For every position of every owner work item (a warp per item): whether the
// owner owns the dyad with that neighbour x and, if so, where the part of x's
// list above v = max(h, x) starts and how long it is (x's split when h < x,
// else found by binary search above the split: h > x is one of x's upper
// neighbours).  A flat pass, so these dependent loads overlap freely instead
// of stalling k_owner between its barriers.
__global__ void __launch_bounds__(256) k_owner_prep(OwnArgs a) {
    const int lane = threadIdx.x & 31;
    const unsigned nlarge = min(a.cnt[0], a.cap), nsmall = min(a.cnt[1], a.cap - nlarge);
    const unsigned nitems = nlarge + nsmall;
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    for (unsigned i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < nitems; i += warps) {
        const uint4 rec = i < nsmall ? a.list[i] : a.list[a.cap - 1 - (i - nsmall)];
        const int64_t rb = a.seg[rec.y].rb;
        const uint32_t hl = (uint32_t)(rec.x - rb);
        const int64_t beg = a.row_ptr[rec.x];
        const int D = (int)(a.row_ptr[rec.x + 1] - beg);
        const int p0 = (int)rec.z * OWN_PIECE, p1 = min(D, p0 + OWN_PIECE);
        for (int pos = p0 + lane; pos < p1; pos += 32) {
            const uint32_t x = __ldg(a.adj + beg + pos) >> 2;
            const int dx = a.deg[rb + x];
            int len = 0;
            int64_t sb = 0;
            if (dx < D || (dx == D && x < hl)) {
                sb = a.row_ptr[rb + x];
                int lo = a.split[rb + x], hi = dx;
                if (hl > x)  // h is one of x's upper neighbours: start after it
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if ((__ldg(a.adj + sb + mid) >> 2) <= hl) lo = mid + 1;
                        else hi = mid;
                    }
                len = dx - lo;
                sb += lo;
            }
            a.psb[beg + pos] = sb;
            a.plen[beg + pos] = len;
        }
    }
}

// The same, one thread per adjacency entry of the census's graphs (entry k
// of row h, found from the per-entry rows of the build): entries of rows that
// are not owners are skipped.  Every lookup range is independent, so the
// dependent loads of all of them overlap.
__global__ void __launch_bounds__(256) k_owner_prep_flat(OwnArgs a, const int32_t* __restrict__ arow,
                                                         const int64_t* __restrict__ epfx, int nseg,
                                                         int64_t total, int own_min) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < total; f += (int64_t)gridDim.x * blockDim.x) {
        const int s = nseg == 1 ? 0 : seg_of(epfx, nseg, f);
        const int64_t k = a.seg[s].eb + (f - epfx[s]);
        const int64_t h = arow[k];
        const int D = a.deg[h];
        if (D < own_min || D > OWN_MAX) continue;
        const int64_t rb = a.seg[s].rb;
        const uint32_t hl = (uint32_t)(h - rb);
        const uint32_t x = __ldg(a.adj + k) >> 2;
        const int dx = a.deg[rb + x];
        int len = 0;
        int64_t sb = 0;
        if (dx < D || (dx == D && x < hl)) {
            sb = a.row_ptr[rb + x];
            int lo = a.split[rb + x], hi = dx;
            if (hl > x)  // h is one of x's upper neighbours: start after it
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if ((__ldg(a.adj + sb + mid) >> 2) <= hl) lo = mid + 1;
                    else hi = mid;
                }
            len = dx - lo;
            sb += lo;
        }
        a.psb[k] = sb;
        a.plen[k] = len;
    }
}

// The task table of positions [q0, q0 + OWN_NT) of the item: for each owned
// dyad {h, x}, in list order, the part of x's list above v = max(h, x) (a
// shared element below v is handled by another dyad of its triangle, see
// on_shared; its share of the dyadic term comes from the closed-triad counts
// in k_fold).  The parts are
// concatenated in "slots", each part widened to whole aligned 16-byte groups
// of x's list (lead entries before it, trail after it, both < 4), so that
// every 4 slots from a multiple of 4 are one aligned 16-byte load of one
// list.  tsb = aligned word index << 4 | trail << 2 | lead, txe = x << 2 | the
// owner's tag for x, tpp = first slot (tpp[ntask] = total slots).  One
// position per thread; one block-wide scan of
// (count << 54 | slots << 27 | lookups).
__device__ __forceinline__ void owner_table(const OwnArgs& a, const Owner& o, int q0, const uint32_t* L,
                                            int64_t* tsb, uint32_t* txe, int32_t* tpp, OwnCtl& ctl) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pos = q0 + (int)threadIdx.x;
    const bool valid = pos < o.p1;
    const uint32_t e = valid ? L[pos] : 0u;
    const uint32_t x = e >> 2;
    const int len = valid ? a.plen[o.beg + pos] : 0;
    const int64_t sb = len > 0 ? a.psb[o.beg + pos] : 0;
    const int lead = (int)(sb & 3);
    const int slots = len > 0 ? (lead + len + 3) & ~3 : 0;
    const unsigned long long v =
        len > 0 ? ((1ull << 54) | ((unsigned long long)slots << 27) | (unsigned long long)len) : 0ull;
    unsigned long long incl = v;
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
        const unsigned long long t = __shfl_up_sync(full, incl, k);
        if (lane >= k) incl += t;
    }
    if (lane == 31) ctl.wsum[warp] = incl;
    __syncthreads();
    unsigned long long ex = incl - v;
    for (int w = 0; w < warp; ++w) ex += ctl.wsum[w];
    if (len > 0) {
        const int t = (int)(ex >> 54);
        const int trail = slots - lead - len;
        tsb[t] = ((sb - lead) << 4) | (int64_t)(trail << 2) | lead;
        txe[t] = (x << 2) | (e & 3u);
        tpp[t] = (int)((ex >> 27) & 0x7ffffff);
    }
    if (threadIdx.x == OWN_NT - 1) {
        ex += v;
        ctl.ntask = (int)(ex >> 54);
        ctl.total = (int)((ex >> 27) & 0x7ffffff);
        tpp[ctl.ntask] = ctl.total;
        const unsigned long long lookups = ex & 0x7ffffff;
        if (lookups) atomicAdd(a.lookups, lookups);
    }
}

// Per-warp queue of keys that passed the mask test: the list entry and its
// task-table index, OWN_QN slots used as a ring.
struct OwnQueue {
    uint32_t* se;
    uint16_t* q;
    int head, n;  // warp-uniform
};

// Look up the 32 queued keys at the head (or the first `cnt`), one per lane.
template <bool STAGED>
__device__ __forceinline__ void owner_drain(OwnHist& w, OwnQueue& Q, int cnt, const Owner& o, const uint32_t* L,
                                            const uint32_t* st, const uint32_t* ls, const uint32_t* txe,
                                            uint32_t& c012, uint32_t& c102) {
    __syncwarp();
    const int lane = w.lane;
    if (lane < cnt) {
        const int slot = (Q.head + lane) & (OWN_QN - 1);
        const uint32_t se = Q.se[slot];
        const uint32_t key = se >> 2;
        const uint32_t hit = owner_find<STAGED>(o, L, st, ls, key);
        if (hit != SENT) {
            const uint32_t xe = txe[Q.q[slot]];
            const uint32_t xt = xe >> 2, et = xe & 3u;
            const bool h_is_u = o.hl < xt;
            const uint32_t pre = h_is_u ? et : (((et & 1u) << 1) | (et >> 1));
            const uint32_t th = hit & 3u, tx = se & 3u;
            on_shared32(w.hs, key, h_is_u ? xt : o.hl, pre, h_is_u ? th : tx, h_is_u ? tx : th);
            ++c012;  // shared elements (for the flush bound)
        }
    }
    __syncwarp();
    Q.head = (Q.head + cnt) & (OWN_QN - 1);
    Q.n -= cnt;
}

// Issue this lane's loads for the unit of OWN_UNIT slots at f0 of the warp's
// range [f0, hi): 4 * OWN_G slots from s0 in aligned 16-byte groups, each
// inside one dyad's part (parts are whole groups, at least one each).  keep
// has bit i set for slot i when it lies inside its part (not the lead of the
// part's first group or the trail of its last); tqp holds the group's task
// index in 16-bit fields.  t is the lane's task: the last dyad whose first
// slot is <= the lane's previous group, advanced here (slots only grow).
__device__ __forceinline__ void owner_issue(const OwnArgs& a, const int64_t* tsb, const int32_t* tpp, int f0, int hi,
                                            int lane, int& t, uint4 (&g)[OWN_G], uint32_t& tqp, uint32_t& keep) {
    const int s0 = f0 + 4 * OWN_G * lane;
    tqp = 0;
    keep = 0;
#pragma unroll
    for (int k = 0; k < OWN_G; ++k) g[k] = make_uint4(SENT, SENT, SENT, SENT);
#pragma unroll
    for (int k = 0; k < OWN_G; ++k) {
        const int sk = s0 + 4 * k;
        if (sk < hi) {
            while (tpp[t + 1] <= sk) ++t;  // ends below ntask: tpp[ntask] = total > sk
            const int64_t d = tsb[t];
            const int p = tpp[t];
            const int rel = sk - p;
            g[k] = __ldg(reinterpret_cast<const uint4*>(a.adj + (d >> 4) + rel));
            const int lead = (int)(d & 3), end = tpp[t + 1] - p - (int)((d >> 2) & 3);
            // slots rel .. rel+3 inside [lead, end)
            const int lo4 = max(lead - rel, 0), hi4 = min(end - rel, 4);
            const uint32_t bits = hi4 > lo4 ? ((1u << hi4) - 1u) & ~((1u << lo4) - 1u) : 0u;
            keep |= bits << (4 * k);
            tqp |= (uint32_t)t << (16 * k);
        }
    }
}

// Units of the current task table.  Each warp takes an equal range of the
// table's slots (whole groups), a unit of OWN_UNIT slots at a time; a lane
// finds its first dyad by binary search and then only steps forward.  The
// next unit's loads are issued before the current unit is filtered, so they
// are in flight meanwhile.
template <bool STAGED>
__device__ __forceinline__ void owner_units(OwnHist& w, OwnQueue& Q, const OwnArgs& a, const Owner& o,
                                            const uint32_t* L, const uint32_t* st, const uint32_t* ls,
                                            const uint32_t* lm, const int64_t* tsb, const uint32_t* txe,
                                            const int32_t* tpp, int ntask, int total) {
    static_assert(OWN_G <= 2, "task indices of a lane's groups are packed in 16-bit fields of one word");
    const unsigned full = 0xffffffffu;
    const int lane = w.lane;
    const unsigned upto = 0xffffffffu >> (31 - lane);  // bits 0..lane
    uint32_t c012 = 0, c102 = 0;
    const int warp = (int)(threadIdx.x >> 5);
    const int lo = (int)(((int64_t)total * warp / OWN_WARPS) & ~(int64_t)3);
    const int hi = warp == OWN_WARPS - 1 ? total : (int)(((int64_t)total * (warp + 1) / OWN_WARPS) & ~(int64_t)3);
    int t = 0;
    {
        const int s0 = lo + 4 * OWN_G * lane;
        if (s0 < hi) {
            int l = 0, h = ntask - 1;  // last dyad whose first slot is <= s0
            while (l < h) {
                const int mid = (l + h + 1) >> 1;
                if (tpp[mid] <= s0) l = mid;
                else h = mid - 1;
            }
            t = l;
        }
    }
    uint4 g[OWN_G];
    uint32_t tqp, keep;
    int f0 = lo;
    owner_issue(a, tsb, tpp, f0, hi, lane, t, g, tqp, keep);
    while (f0 < hi) {
        uint4 gn[OWN_G];
        uint32_t tqn, keepn;
        const int f0n = f0 + OWN_UNIT;
        owner_issue(a, tsb, tpp, f0n, hi, lane, t, gn, tqn, keepn);
        uint32_t se[4 * OWN_G];
#pragma unroll
        for (int k = 0; k < OWN_G; ++k) {
            se[4 * k] = g[k].x;
            se[4 * k + 1] = g[k].y;
            se[4 * k + 2] = g[k].z;
            se[4 * k + 3] = g[k].w;
        }
#pragma unroll
        for (int j = 0; j < 4 * OWN_G; ++j) {
            const bool pass = ((keep >> j) & 1u) && owner_maybe<STAGED>(o, st, lm, se[j] >> 2);
            const unsigned m = __ballot_sync(full, pass);
            if (pass) {
                const int slot = (Q.head + Q.n + __popc(m & (upto >> 1))) & (OWN_QN - 1);
                Q.se[slot] = se[j];
                Q.q[slot] = (uint16_t)(tqp >> (16 * (j >> 2)));
            }
            Q.n += __popc(m);
            if (Q.n >= 32) owner_drain<STAGED>(w, Q, 32, o, L, st, ls, txe, c012, c102);
        }
#pragma unroll
        for (int k = 0; k < OWN_G; ++k) g[k] = gn[k];
        tqp = tqn;
        keep = keepn;
        f0 = f0n;
    }
    if (Q.n > 0) owner_drain<STAGED>(w, Q, Q.n, o, L, st, ls, txe, c012, c102);  // the table changes next
    w.pending += __reduce_add_sync(full, c012 + c102);
    __syncwarp();
}

// Persistent: first the pieces of owners above OWN_CAP (bucket starts in
// shared memory, the list read from global memory), then the others (list
// staged).  Consecutive pieces of one owner on a CTA reuse its index.
__global__ void __launch_bounds__(OWN_NT, 2) k_owner(OwnArgs a) {
    extern __shared__ __align__(16) unsigned char own_smem[];
    uint32_t* T = reinterpret_cast<uint32_t*>(own_smem);
    uint32_t* st = reinterpret_cast<uint32_t*>(own_smem + OWN_T_BYTES);
    uint32_t* ls = reinterpret_cast<uint32_t*>(own_smem);
    uint32_t* lm = reinterpret_cast<uint32_t*>(own_smem + OWN_LS_BYTES);
    unsigned char* p = own_smem + OWN_IDX_BYTES;
    int32_t* hs_all = reinterpret_cast<int32_t*>(p);
    p += OWN_HS_BYTES;
    int64_t* tsb = reinterpret_cast<int64_t*>(p);
    p += OWN_SB_BYTES;
    uint32_t* txe = reinterpret_cast<uint32_t*>(p);
    p += OWN_XE_BYTES;
    int32_t* tpp = reinterpret_cast<int32_t*>(p);
    p += OWN_PP_BYTES;
    __shared__ OwnCtl ctl;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    OwnHist w{hs_all + (size_t)warp * ACC, a.acc, -1, lane, 0u};
    OwnQueue Q{reinterpret_cast<uint32_t*>(p) + warp * OWN_QN,
               reinterpret_cast<uint16_t*>(p + sizeof(uint32_t) * OWN_QN * OWN_WARPS) + warp * OWN_QN, 0, 0};
    for (int j = lane; j < ACC; j += 32) w.hs[j] = 0;
    __syncwarp();
    const unsigned nlarge = min(a.cnt[0], a.cap), nsmall = min(a.cnt[1], a.cap - nlarge);
    for (int phase = 0; phase < 2; ++phase) {
        const unsigned nitems = phase == 0 ? nlarge : nsmall;
        if (threadIdx.x == 0) {  // the index in shared memory changes form between phases
            ctl.row = ~0u;
            ctl.seg = -1;
        }
        const unsigned grab = phase == 0 ? OWN_GRAB : 1u;
        for (;;) {
            if (threadIdx.x == 0) {
                ctl.idx = atomicAdd(a.cursor + phase, grab);
            }
            __syncthreads();
            const unsigned idx0 = ctl.idx;
            if (idx0 >= nitems) break;
            for (unsigned idx = idx0; idx < min(idx0 + grab, nitems); ++idx) {
            const Owner o = phase == 0 ? owner_setup(a, a.list[a.cap - 1 - idx], OWN_LBL, 5)
                                       : owner_setup(a, a.list[idx], OWN_LBS, 4);
            const uint32_t* G = a.adj + o.beg;
            const bool restage = o.row != ctl.row || o.s != ctl.seg;
            if (restage) {  // index the owner (unless the last item had it)
                if (phase == 0) owner_index<false>(o, G, T, st, ls, lm);
                else owner_index<true>(o, G, T, st, ls, lm);
                __syncthreads();
            }
            if (threadIdx.x == 0 && restage) {  // all threads have compared
                ctl.row = o.row;
                ctl.seg = o.s;
            }
            w.retag(o.s);
            for (int q0 = o.p0; q0 < o.p1; q0 += OWN_NT) {
                if (phase == 0) owner_table(a, o, q0, G, tsb, txe, tpp, ctl);
                else owner_table(a, o, q0, T, tsb, txe, tpp, ctl);
                __syncthreads();
                const int ntask = ctl.ntask, total = ctl.total;
                if (phase == 0) owner_units<false>(w, Q, a, o, G, st, ls, lm, tsb, txe, tpp, ntask, total);
                else owner_units<true>(w, Q, a, o, T, st, ls, lm, tsb, txe, tpp, ntask, total);
                __syncthreads();
            }
            }
        }
    }
    w.flush();
}

#include "forward.cuh"

// ------------------------------------------------------------- host side --
constexpr int STREAM_EPL = 8;

struct Launch {
    int sms = 148;
    int occ_tasks = 1, occ_thread = 1, occ_warp = 1, occ_cta = 1, occ_stream = 1, occ_merge = 1, occ_flat = 1;
    int occ_owner = 1, occ_tri_big = 1, occ_tri_small = 1, occ_tri_big_ids = 1, occ_tri_small_ids = 1;
    bool ready = false;
};

tc_status launch_info(Launch& L) {
    static Launch cache[64];
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    Launch& c = cache[dev & 63];
    if (!c.ready) {
        TC_CUDA(cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev));
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ_tasks, k_tasks, 256, 0));
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ_thread, k_thread, 256, 0));
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ_warp, k_warp, 256, 0));
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ_cta, k_cta, CTA_NT, 0));
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ_stream, k_stream<STREAM_EPL>, 256, 0));
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ_merge, k_merge<STREAM_EPL, false>, 256, 0));
        c.occ_tasks = std::max(1, c.occ_tasks);
        c.occ_thread = std::max(1, c.occ_thread);
        c.occ_warp = std::max(1, c.occ_warp);
        c.occ_cta = std::max(1, c.occ_cta);
        c.occ_stream = std::max(1, c.occ_stream);
        c.occ_merge = std::max(1, c.occ_merge);
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ_flat, k_tasks_flat, 256, 0));
        c.occ_flat = std::max(1, c.occ_flat);
        TC_CUDA(cudaFuncSetAttribute(k_owner, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OWN_SMEM));
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ_owner, k_owner, OWN_NT, OWN_SMEM));
        c.occ_owner = std::max(1, c.occ_owner);
        TC_CUDA(cudaFuncSetAttribute(k_tri_big<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TB_SMEM));
        TC_CUDA(cudaFuncSetAttribute(k_tri_big<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TB_SMEM));
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ_tri_big, k_tri_big<false>, TB_NT, TB_SMEM));
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ_tri_big_ids, k_tri_big<true>, TB_NT, TB_SMEM));
        c.occ_tri_big = std::max(1, c.occ_tri_big);
        c.occ_tri_big_ids = std::max(1, c.occ_tri_big_ids);
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ_tri_small, k_tri_small<false>, 256, 0));
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ_tri_small_ids, k_tri_small<true>, 256, 0));
        c.occ_tri_small = std::max(1, c.occ_tri_small);
        c.occ_tri_small_ids = std::max(1, c.occ_tri_small_ids);
        c.ready = true;
    }
    L = c;
    return TC_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Everything a census of a list of graphs needs that can be decided on the
// host: resolved options, the graph (segment) table, capacities and the work
// space layout.
struct Layout {
    tc_opts o;
    int nseg = 0;
    int64_t rows = 0;
    uint64_t cap01 = 0, cap2 = 0;
    std::vector<SegDev> segs;
    std::vector<int64_t> pfx;
    std::vector<int64_t> epfx;  // adjacency entries of the selected graphs, running
    bool flat = false;          // per-entry task terms (k_tasks_flat)
    int64_t entries = 0;
    size_t scan_bytes = 0;      // scan work space (scan_tmp_bytes)
    size_t o_acc, o_ctr, o_seg, o_pfx, o_out, o_codes, o_r[NBIN], o_rt, o_tl, o_ia, o_own, o_psb, o_plen, o_epfx,
        o_scan, o_scantmp, need;
    uint32_t own_cap = 0;
    bool exact = false;  // TC_BIN_EXACT on the merge path: |S| per canonical dyad first
    size_t o_usz = 0;
    // tc_census_shard: this call does shard `shard` of `nshards` and writes the
    // raw accumulators of each graph to raw[slot] instead of folding them
    int32_t shard = 0, nshards = 1;
    unsigned long long* raw = nullptr;
    // triangles classified in id order (the 64-code census, shards), else in
    // rank order (the 16-type census)
    bool ids = false;
    // forward path (tri_path = TC_TRI_FORWARD)
    bool fwd = false;
    int nb = 0;            // blocks of the rank computation
    int64_t dyads = 0;     // canonical dyads of the selection
    uint32_t item_cap = 0;
    size_t fscan_bytes = 0;
    size_t o_hist, o_hex, o_co, o_clsb, o_rank, o_perm, o_flag, o_fs, o_fptr, o_kind, o_tcnt, o_tpre, o_longs,
        o_fid, o_fwd, o_trec, o_items, o_fscantmp, o_tp, o_tpc;
    uint32_t piece_cap = 0;  // pieces of the longer rows in the row-wise task pass
};

// counters (uint32 words): [0..3] records per bin, [4] overflow flag,
// [5] tile records, [8..9] row cursor (u64), [10..17] merged entries per bin
// (u64), [20..23] cursors of the persistent merge queues
// Counter words: 0-3 bin records, 4 overflow, 5 tiles, 6 routed split tasks,
// 7 hub tasks, 8-9 task-build row cursor, 10-17 bin entries, 20-23 merge
// cursors, 24-25 hub entries, 26-27 owner cursors, 28-29 owner rows (larger,
// smaller), 32-39 owner tasks, merged entries, probes, staged entries.
// Forward path: 40 tag-map items, 41 long rows, 42-43 work cursors, 44-51
// lookups and triangles of each lookup form (u64), 52-53 forward-list
// entries the tag-map items stage (u64), 54 pieces of the row-wise task pass.
constexpr int CTR_WORDS = 64;

tc_status make_layout(const GraphSet& set, const std::vector<int32_t>& gidx, const tc_opts* opts_in,
                      Layout& Lo, const std::vector<int32_t>* slots = nullptr) {
    tc_opts o;
    tc_opts_default(&o);
    if (opts_in) o = *opts_in;
    if (o.bin_mode != TC_BIN_HEURISTIC && o.bin_mode != TC_BIN_MLP && o.bin_mode != TC_BIN_EXACT)
        return fail(TC_ERR_ARG, "census: unknown bin_mode");
    if (o.thr_thread < 0 || o.thr_warp < o.thr_thread || o.chunk < 256 ||
        o.chunk > (o.split_cta ? TILE : WARP_LMAX))
        return fail(TC_ERR_ARG, "census: need 0 <= thr_thread <= thr_warp and 256 <= chunk <= "
                                "1024 (warp tiles) or 3840 (split_cta = 1)");
    if (o.stream_max < 0) return fail(TC_ERR_ARG, "census: stream_max < 0");
    if (o.hub_ratio < 0) return fail(TC_ERR_ARG, "census: hub_ratio < 0");
    if (o.own_min < 0) return fail(TC_ERR_ARG, "census: own_min < 0");
    if (o.persistent && o.split_cta)
        return fail(TC_ERR_ARG, "census: the persistent merge runs warp tiles (split_cta must be 0)");
    if (o.tri_path != TC_TRI_FORWARD && o.tri_path != TC_TRI_MERGE) return fail(TC_ERR_ARG, "census: unknown tri_path");
    // (TC_TRI_AUTO is resolved per graph before a layout is made)
    if (o.fwd_big < 1) return fail(TC_ERR_ARG, "census: fwd_big < 1");
    // a warp holds both lists (or the short list) in shared memory
    o.thr_warp = std::min(o.thr_warp, WARP_LMAX);

    const int nseg = (int)gidx.size();
    Lo.segs.assign((size_t)nseg, SegDev{});
    Lo.pfx.assign((size_t)nseg + 1, 0);
    Lo.epfx.assign((size_t)nseg + 1, 0);
    std::vector<int64_t> gent((size_t)set.G + 1, 0);  // first adjacency entry of each graph
    for (int32_t g = 0; g < set.G; ++g) gent[(size_t)g + 1] = gent[(size_t)g] + 2 * set.stats[(size_t)g].dyads;
    int64_t dyads = 0, merged = 0;
    for (int i = 0; i < nseg; ++i) {
        const int g = gidx[(size_t)i];
        Lo.segs[(size_t)i].rb = set.voff[(size_t)g];
        Lo.segs[(size_t)i].n = set.voff[(size_t)g + 1] - set.voff[(size_t)g];
        Lo.segs[(size_t)i].eb = gent[(size_t)g];
        Lo.epfx[(size_t)i + 1] = Lo.epfx[(size_t)i] + 2 * set.stats[(size_t)g].dyads;
        Lo.segs[(size_t)i].slot = slots ? (*slots)[(size_t)i] : i;
        Lo.segs[(size_t)i].pad = 0;
        Lo.pfx[(size_t)i + 1] = Lo.pfx[(size_t)i] + Lo.segs[(size_t)i].n;
        dyads += set.stats[(size_t)g].dyads;
        merged += set.stats[(size_t)g].merged_entries;
    }
    Lo.o = o;
    Lo.nseg = nseg;
    Lo.rows = Lo.pfx[(size_t)nseg];
    Lo.cap01 = (uint64_t)dyads + 1;
    Lo.cap2 = (uint64_t)(merged / o.chunk) + (uint64_t)dyads + 1;
    if (Lo.cap01 >= 0xffffffffull || Lo.cap2 >= 0xffffffffull)
        return fail(TC_ERR_UNSUPPORTED, "census: more than 2^32 tasks");
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off = align256(off + bytes); return at; };
    Lo.o_acc = take(sizeof(unsigned long long) * ACC * (size_t)nseg);
    Lo.o_ctr = take(sizeof(unsigned int) * CTR_WORDS);
    Lo.o_seg = take(sizeof(SegDev) * (size_t)nseg);
    Lo.o_pfx = take(sizeof(int64_t) * ((size_t)nseg + 1));
    Lo.o_out = take(sizeof(tc_census_t) * (size_t)nseg);
    Lo.o_codes = take(sizeof(tc_census64_t) * (size_t)nseg);
    // per-entry task terms need every row below 2^21 entries (packed tag scan)
    Lo.entries = Lo.epfx[(size_t)nseg];
    // the forward path needs the per-entry rows and fewer than 2^31 entries
    // (its scans count in int32); otherwise the merge path runs
    Lo.fwd = o.tri_path == TC_TRI_FORWARD && set.arow != nullptr && Lo.rows > 0 && Lo.entries > 0 &&
             Lo.entries < ((int64_t)1 << 31);
    Lo.dyads = dyads;
    // merge-path bins, tiles and owner tables (one record each when unused)
    const uint64_t c01 = Lo.fwd ? 1 : Lo.cap01, c2 = Lo.fwd ? 1 : Lo.cap2;
    for (int b = 0; b < NBIN; ++b) Lo.o_r[b] = take(sizeof(uint4) * c01);
    Lo.o_rt = o.bin_mode == TC_BIN_MLP ? take(sizeof(uint4) * c01) : Lo.o_r[2];
    Lo.o_tl = take(sizeof(uint4) * c2);
    Lo.o_ia = take(sizeof(int32_t) * c2);
    // exact task costs, one word per adjacency entry of the build
    Lo.exact = o.bin_mode == TC_BIN_EXACT && !Lo.fwd && set.arow != nullptr && Lo.entries > 0;
    Lo.o_usz = take(sizeof(uint32_t) * (Lo.exact ? (size_t)set.nnz : 1));
    if (Lo.fwd) {
        Lo.cap01 = Lo.cap2 = 1;
        o.own_min = 0;
        Lo.o.own_min = 0;
    }
    // pieces: sum over owners of ceil(d / OWN_PIECE) <= rows + 2|U| / OWN_PIECE
    Lo.own_cap = (uint32_t)std::min<int64_t>(Lo.rows + 2 * dyads / OWN_PIECE + 1, 0xffffffffll);
    Lo.o_own = take(sizeof(uint4) * (o.own_min > 0 ? Lo.own_cap : 1));
    // per adjacency entry of an owner: start and length of the other
    // endpoint's list part (k_owner_prep)
    const size_t nprep = o.own_min > 0 ? (size_t)std::max<int64_t>(set.nnz, 1) : 1;
    Lo.o_psb = take(sizeof(int64_t) * nprep);
    Lo.o_plen = take(sizeof(int32_t) * nprep);
    Lo.flat = !o.row_tasks && set.arow != nullptr && set.max_deg < (1 << TAG_BITS) && set.nnz > 0;
    Lo.o_epfx = take(sizeof(int64_t) * ((size_t)nseg + 1));
    Lo.scan_bytes = 0;
    Lo.flat = Lo.flat && Lo.entries > 0;
    if (Lo.flat) Lo.scan_bytes = scan_tmp_bytes(Lo.entries);
    Lo.o_scan = take(sizeof(unsigned long long) * (Lo.flat && !Lo.fwd ? (size_t)Lo.entries : 1));
    Lo.o_scantmp = take(std::max<size_t>(Lo.scan_bytes, 16));
    // forward lists: ranks, forward entries, dyad records by owner
    if (Lo.fwd) {
        const size_t rows = (size_t)Lo.rows, D = (size_t)std::max<int64_t>(dyads, 1);
        Lo.nb = (int)((Lo.rows + RK_B - 1) / RK_B);
        Lo.item_cap = (uint32_t)std::min<int64_t>(Lo.rows + dyads / TRI_PIECE + 1, 0xffffffffll);
        Lo.fscan_bytes = std::max(scan_tmp_bytes((int64_t)NCLS * Lo.nb),
                                  std::max(scan_tmp_bytes(Lo.entries), scan_tmp_bytes((int64_t)rows + 1)));
        Lo.o_hist = take(sizeof(uint32_t) * NCLS * (size_t)Lo.nb);
        Lo.o_hex = take(sizeof(uint32_t) * NCLS * (size_t)Lo.nb);
        Lo.o_co = take(sizeof(int64_t) * NCLS * (size_t)nseg);
        Lo.o_clsb = take(sizeof(int32_t) * NCLS * (size_t)nseg);
        Lo.o_rank = take(sizeof(int32_t) * rows);
        Lo.o_perm = take(sizeof(int32_t) * rows);
        Lo.o_flag = take(sizeof(uint8_t) * (size_t)Lo.entries);
        Lo.o_fs = take(sizeof(int32_t) * (size_t)Lo.entries);
        Lo.o_fptr = take(sizeof(uint32_t) * (rows + 1));
        Lo.o_kind = take(sizeof(uint8_t) * rows);
        Lo.o_tcnt = take(sizeof(unsigned long long) * (rows + 1));
        Lo.o_tpre = take(sizeof(unsigned long long) * (rows + 1));
        Lo.o_longs = take(sizeof(uint32_t) * rows);
        Lo.o_fid = take(sizeof(uint32_t) * D);
        Lo.o_fwd = take(sizeof(uint32_t) * D);
        Lo.o_trec = take(sizeof(uint4) * D);
        Lo.o_items = take(sizeof(uint4) * 2 * (size_t)Lo.item_cap);
        Lo.o_fscantmp = take(std::max<size_t>(Lo.fscan_bytes, 16));
        Lo.piece_cap = (uint32_t)std::min<int64_t>(Lo.rows + Lo.entries / TR_PIECE + 1, 0xffffffffll);
        Lo.o_tp = take(sizeof(uint4) * 3 * (size_t)Lo.piece_cap);
        Lo.o_tpc = take(sizeof(uint4) * (size_t)Lo.piece_cap);
    }
    Lo.need = off;
    return TC_OK;
}

// The graph table goes to the device once (a pageable copy: not part of a
// captured graph).
tc_status upload_layout(const Layout& Lo, char* ws, cudaStream_t st) {
    TC_CUDA(cudaMemcpyAsync(ws + Lo.o_seg, Lo.segs.data(), sizeof(SegDev) * (size_t)Lo.nseg,
                            cudaMemcpyHostToDevice, st));
    TC_CUDA(cudaMemcpyAsync(ws + Lo.o_pfx, Lo.pfx.data(), sizeof(int64_t) * ((size_t)Lo.nseg + 1),
                            cudaMemcpyHostToDevice, st));
    TC_CUDA(cudaMemcpyAsync(ws + Lo.o_epfx, Lo.epfx.data(), sizeof(int64_t) * ((size_t)Lo.nseg + 1),
                            cudaMemcpyHostToDevice, st));
    return TC_OK;
}

// The forward path (tri_path = TC_TRI_FORWARD): the vertex ranks; the task
// pass adds every dyad's suffix and dyadic terms, emits no task and flags
// the forward entries; the forward lists and the dyad records are built;
// the two lookup kernels apply each triangle's correction once.  Marks 1
// (ranks + task pass), 2 (forward lists), 3 (tag-map owners), 4..8 (the
// other owners).
template <class Mark>
tc_status enqueue_forward(const GraphSet& set, const Layout& Lo, char* ws, cudaStream_t st, const Launch& L,
                          const BinParams& bp, const Bins& bins, Mark& mark) {
    unsigned long long* acc = (unsigned long long*)(ws + Lo.o_acc);
    unsigned int* ctr = (unsigned int*)(ws + Lo.o_ctr);
    const SegDev* d_seg = (const SegDev*)(ws + Lo.o_seg);
    const int64_t* d_pfx = (const int64_t*)(ws + Lo.o_pfx);
    const int64_t* d_epfx = (const int64_t*)(ws + Lo.o_epfx);
    unsigned long long* cursor = (unsigned long long*)(ctr + 8);
    uint32_t* hist = (uint32_t*)(ws + Lo.o_hist);
    uint32_t* hex = (uint32_t*)(ws + Lo.o_hex);
    int64_t* co = (int64_t*)(ws + Lo.o_co);
    int32_t* clsb = (int32_t*)(ws + Lo.o_clsb);
    int32_t* rank = (int32_t*)(ws + Lo.o_rank);
    int32_t* perm = (int32_t*)(ws + Lo.o_perm);
    uint8_t* flag = (uint8_t*)(ws + Lo.o_flag);
    void* tmp = ws + Lo.o_fscantmp;
    // vertex ranks: (floor(log2 d), id) per graph
    k_rank_hist<<<Lo.nb, RK_B, 0, st>>>(set.deg, d_seg, d_pfx, Lo.nseg, Lo.rows, Lo.nb, hist);
    TC_CUDA(cudaGetLastError());
    TC_CUDA(scan_run<false>(ScanLoad<uint32_t>{hist}, (int64_t)NCLS * Lo.nb, hex, tmp, false, st));
    k_rank_seg<<<std::min(Lo.nseg, L.sms * 16), 32, 0, st>>>(set.deg, d_seg, d_pfx, Lo.nseg, Lo.rows, Lo.nb, hex, co,
                                                             clsb);
    TC_CUDA(cudaGetLastError());
    k_rank_assign<<<Lo.nb, RK_B, 0, st>>>(set.deg, d_seg, d_pfx, Lo.nseg, Lo.rows, Lo.nb, hex, co, rank, perm,
                                          bins.overflow);
    TC_CUDA(cudaGetLastError());
    // the task pass, with the forward flags
    if (Lo.flat) {  // row-wise: a thread per short row, a warp per piece of a longer one
        TermArgs ta;
        ta.row_ptr = set.row_ptr;
        ta.adj = set.adj;
        ta.seg = d_seg;
        ta.pfx = d_pfx;
        ta.epfx = d_epfx;
        ta.nseg = Lo.nseg;
        ta.rows = Lo.rows;
        ta.r_lo = bp.r_lo;
        ta.r_hi = bp.r_hi;
        ta.rank = rank;
        ta.perm = perm;
        ta.flag = flag;
        ta.acc = acc;
        ta.pieces = (uint4*)(ws + Lo.o_tp);
        ta.npieces = ctr + 54;
        ta.piece_cap = Lo.piece_cap;
        ta.pcnt = (uint4*)(ws + Lo.o_tpc);
        k_terms_rows<<<L.sms * 8, 256, 0, st>>>(ta);
        TC_CUDA(cudaGetLastError());
        k_piece_counts<<<L.sms * 4, 256, 0, st>>>(ta);
        TC_CUDA(cudaGetLastError());
        k_terms_pieces<<<L.sms * 8, 256, 0, st>>>(ta);
    } else {
        k_tasks<<<L.sms * L.occ_tasks, 256, 0, st>>>(set.row_ptr, set.adj, set.deg, d_seg, d_pfx, Lo.nseg, Lo.rows,
                                                     bp, bins, acc, cursor);
        TC_CUDA(cudaGetLastError());
        k_fwd_flags<<<L.sms * 16, 256, 0, st>>>(set.adj, set.arow, d_seg, d_pfx, d_epfx, Lo.nseg, Lo.entries, rank,
                                                flag);
    }
    TC_CUDA(cudaGetLastError());
    mark(1);
    // forward lists and the dyad records
    FwdLayout F;
    F.fs = (const int32_t*)(ws + Lo.o_fs);
    F.fptr = (uint32_t*)(ws + Lo.o_fptr);
    F.kind = (uint8_t*)(ws + Lo.o_kind);
    F.tcnt = (unsigned long long*)(ws + Lo.o_tcnt);
    F.tpre = (unsigned long long*)(ws + Lo.o_tpre);
    F.fid = (uint32_t*)(ws + Lo.o_fid);
    F.fwd = (uint32_t*)(ws + Lo.o_fwd);
    F.trec = (uint4*)(ws + Lo.o_trec);
    F.items = (uint4*)(ws + Lo.o_items);
    F.item_cap = Lo.item_cap;
    F.longs = (uint32_t*)(ws + Lo.o_longs);
    F.nitems = ctr + 40;
    F.nlong = ctr + 41;
    F.cursor = ctr + 42;
    F.stat = (unsigned long long*)(ctr + 44);
    F.rank = rank;
    F.perm = perm;
    F.clsb = clsb;
    TC_CUDA(scan_run<true>(ScanLoad<uint8_t>{flag}, Lo.entries, (int32_t*)(ws + Lo.o_fs), tmp, false, st));
    k_fwd_rows<<<L.sms * 8, FR_NT, 0, st>>>(set.row_ptr, set.deg, d_seg, d_pfx, d_epfx, Lo.nseg, Lo.rows, Lo.o.fwd_big,
                                           F, bp.r_lo, bp.r_hi);
    TC_CUDA(cudaGetLastError());
    TC_CUDA(scan_run<false>(ScanLoad<unsigned long long>{F.tcnt}, Lo.rows + 1, F.tpre, tmp, false, st));
    k_fwd_items<<<L.sms * 4, 256, 0, st>>>(d_pfx, Lo.nseg, F);
    TC_CUDA(cudaGetLastError());
    k_fwd_fill<<<L.sms * 16, 256, 0, st>>>(set.adj, set.arow, d_seg, d_pfx, d_epfx, Lo.nseg, Lo.entries, F);
    TC_CUDA(cudaGetLastError());
    k_fwd_sort_short<<<L.sms * 8, 256, 0, st>>>(Lo.rows, F);
    TC_CUDA(cudaGetLastError());
    k_fwd_sort<<<L.sms * 8, 256, 0, st>>>(set.deg, d_seg, d_pfx, Lo.nseg, F);
    TC_CUDA(cudaGetLastError());
    k_fwd_recs<<<L.sms * 16, 256, 0, st>>>(set.row_ptr, set.adj, set.arow, d_seg, d_pfx, d_epfx, Lo.nseg,
                                           Lo.entries, Lo.rows, F);
    TC_CUDA(cudaGetLastError());
    mark(2);
    TriArgs ta;
    ta.seg = d_seg;
    ta.pfx = d_pfx;
    ta.nseg = Lo.nseg;
    ta.rows = Lo.rows;
    ta.fptr = F.fptr;
    ta.tpre = F.tpre;
    ta.fwd = F.fwd;
    ta.trec = F.trec;
    ta.items = F.items;
    ta.nitems = F.nitems;
    ta.item_cap = F.item_cap;
    ta.cursor = F.cursor;
    ta.rank = rank;
    ta.perm = perm;
    ta.acc = acc;
    ta.stat = F.stat;
    // the 64-code census and shards need each triangle in id order; the
    // 16-type census takes it in rank order
    if (Lo.ids) k_tri_big<true><<<L.sms * L.occ_tri_big_ids, TB_NT, TB_SMEM, st>>>(ta);
    else k_tri_big<false><<<L.sms * L.occ_tri_big, TB_NT, TB_SMEM, st>>>(ta);
    TC_CUDA(cudaGetLastError());
    mark(3);
    if (Lo.ids) k_tri_small<true><<<L.sms * L.occ_tri_small_ids, 256, 0, st>>>(ta);
    else k_tri_small<false><<<L.sms * L.occ_tri_small, 256, 0, st>>>(ta);
    TC_CUDA(cudaGetLastError());
    for (int k = 4; k <= 7; ++k) mark(k);
    return TC_OK;
}

// The census itself: one memset and the kernels, all on `st` (capturable).
tc_status enqueue_census(const GraphSet& set, const Layout& Lo, char* ws, tc_census_t* d_out, cudaStream_t st,
                         ProfileEvents* pe, const Instr* ins = nullptr, tc_census64_t* d_codes = nullptr) {
    const tc_opts& o = Lo.o;
    unsigned long long* acc = (unsigned long long*)(ws + Lo.o_acc);
    unsigned int* ctr = (unsigned int*)(ws + Lo.o_ctr);
    const SegDev* d_seg = (const SegDev*)(ws + Lo.o_seg);
    const int64_t* d_pfx = (const int64_t*)(ws + Lo.o_pfx);
    Bins bins;
    for (int b = 0; b < NBIN; ++b) {
        bins.rec[b] = (uint4*)(ws + Lo.o_r[b]);
        bins.cap[b] = (uint32_t)Lo.cap01;
    }
    bins.cnt = ctr;
    bins.overflow = (int*)(ctr + 4);
    bins.entries = (unsigned long long*)(ctr + 10);
    bins.own = (uint4*)(ws + Lo.o_own);
    bins.own_cap = Lo.own_cap;
    bins.own_cnt = ctr + 28;
    bins.own_stat = (unsigned long long*)(ctr + 32);
    unsigned long long* cursor = (unsigned long long*)(ctr + 8);
    uint4* d_tiles = (uint4*)(ws + Lo.o_tl);
    int32_t* d_ia = (int32_t*)(ws + Lo.o_ia);
    const uint32_t cap2 = (uint32_t)Lo.cap2;
    Launch L;
    if (tc_status s = launch_info(L); s != TC_OK) return s;
    const __half2* mlp = o.bin_mode == TC_BIN_MLP ? (const __half2*)cost_model_weights() : nullptr;
    // with a cost model, every task above the warp bin is first collected in
    // bin 2 and then routed by k_route (stream bin or tiles)
    const uint32_t* exact = Lo.exact ? (const uint32_t*)(ws + Lo.o_usz) : nullptr;
    // shard k of N: entries [k E / N, (k+1) E / N) for the task terms, rows
    // [k R / N, (k+1) R / N) for the owned dyads (the ids are arbitrary, so
    // an even cut of the rows spreads the owners' work)
    const auto cut = [&](int64_t total, int32_t k) {
        return (int64_t)((unsigned __int128)(uint64_t)total * (uint64_t)k / (uint64_t)Lo.nshards);
    };
    const BinParams bp{o.thr_thread, o.thr_warp, mlp ? 0 : o.stream_max, o.own_min, mlp, set.vtag, Lo.fwd ? 1 : 0,
                       exact, cut(Lo.entries, Lo.shard), cut(Lo.entries, Lo.shard + 1), cut(Lo.rows, Lo.shard),
                       cut(Lo.rows, Lo.shard + 1)};
    uint4* split_tasks = (uint4*)(ws + Lo.o_rt);
    auto mark = [&](int k) {
        if (pe) cudaEventRecord(pe->ev[k], st);
    };
    if (Lo.exact) {  // the exact costs first (timed apart from the census kernels)
        if (pe) cudaEventRecord(pe->ev[NEV], st);
        k_union_entries<<<L.sms * 8, 256, 0, st>>>(set.row_ptr, set.adj, set.arow, set.deg, d_seg,
                                                   (const int64_t*)(ws + Lo.o_epfx), Lo.nseg, Lo.entries,
                                                   (uint32_t*)(ws + Lo.o_usz));
        TC_CUDA(cudaGetLastError());
    }
    TC_CUDA(cudaMemsetAsync(ws, 0, Lo.o_seg, st));  // accumulators + counters
    mark(0);
    if (Lo.fwd) {
        if (tc_status r = enqueue_forward(set, Lo, ws, st, L, bp, bins, mark); r != TC_OK) return r;
    } else if (Lo.rows > 0) {
        if (Lo.flat) {
            unsigned long long* scan = (unsigned long long*)(ws + Lo.o_scan);
            const int64_t* d_epfx = (const int64_t*)(ws + Lo.o_epfx);
            TC_CUDA(scan_run<true>(OneHot{set.adj, d_seg, d_epfx, Lo.nseg}, Lo.entries, scan, ws + Lo.o_scantmp,
                                   false, st));
            if (bp.own_min > 0) {
                k_owner_rows<<<L.sms * 8, 256, 0, st>>>(set.deg, d_seg, d_pfx, Lo.nseg, Lo.rows, bp.own_min, bins,
                                                        bp.r_lo, bp.r_hi);
                TC_CUDA(cudaGetLastError());
            }
            k_tasks_flat<<<L.sms * L.occ_flat, 256, 0, st>>>(set.row_ptr, set.adj, set.arow, set.deg, set.vtag, scan,
                                                             d_seg, (const int64_t*)(ws + Lo.o_epfx), Lo.nseg,
                                                             Lo.entries, bp, bins, acc, cursor,
                                                             FlagOut{nullptr, nullptr, nullptr});
        } else {
            k_tasks<<<L.sms * L.occ_tasks, 256, 0, st>>>(set.row_ptr, set.adj, set.deg, d_seg, d_pfx, Lo.nseg,
                                                         Lo.rows, bp, bins, acc, cursor);
        }
        TC_CUDA(cudaGetLastError());
        const unsigned int* nsplit = ctr + 2;
        if (mlp) {
            k_route<<<L.sms * 4, 256, 0, st>>>(mlp, set.deg, set.vtag, bins.rec[2], ctr + 2, bins.cap[2], split_tasks,
                                               ctr + 6, bins.rec[3], ctr + 3, (uint32_t)Lo.cap01,
                                               o.stream_max, bins.overflow);
            TC_CUDA(cudaGetLastError());
            nsplit = ctr + 6;
        }
        mark(1);
        // hub tasks: counted in ctr[7], entries in ctr[24..25], records at the
        // end of the stream-bin array (with a cost model, what it sent to
        // tiles stays there)
        unsigned long long* hub_entries = (unsigned long long*)(ctr + 24);
        k_split<<<L.sms * 8, 256, 0, st>>>(set.row_ptr, set.adj, split_tasks, nsplit, bins.cap[2], o.chunk,
                                            d_tiles, d_ia, ctr + 5, cap2, bins.overflow, mlp ? 0 : o.stream_max,
                                            o.hub_ratio,
                                            bins.rec[3], bins.cap[3], ctr + 3, ctr + 7, hub_entries);
        TC_CUDA(cudaGetLastError());
        mark(2);
        if (o.own_min > 0) {
            const OwnArgs oa{set.row_ptr, set.adj, set.deg, set.split, d_seg, bins.own, bins.own_cap, ctr + 28,
                             ctr + 26, acc, bins.own_stat + 2, (int64_t*)(ws + Lo.o_psb),
                             (int32_t*)(ws + Lo.o_plen)};
            if (Lo.flat)
                k_owner_prep_flat<<<L.sms * 16, 256, 0, st>>>(oa, set.arow, (const int64_t*)(ws + Lo.o_epfx), Lo.nseg,
                                                              Lo.entries, o.own_min);
            else
                k_owner_prep<<<L.sms * 8, 256, 0, st>>>(oa);
            TC_CUDA(cudaGetLastError());
            mark(3);
            k_owner<<<L.sms * L.occ_owner, OWN_NT, OWN_SMEM, st>>>(oa);
            TC_CUDA(cudaGetLastError());
        } else {
            mark(3);
        }
        mark(4);
        auto hub_launch = [&]() {
            k_hub<STREAM_EPL><<<L.sms * L.occ_stream, 256, 0, st>>>(set.row_ptr, set.adj, d_seg, set.split,
                                                                              bins.rec[3], ctr + 7, bins.cap[3],
                                                                              acc);
            return cudaGetLastError();
        };
        if (o.persistent) {
            MergeQueues q;
            for (int b = 0; b < NBIN; ++b) {
                q.rec[b] = bins.rec[b];
                q.cap[b] = bins.cap[b];
            }
            q.cnt = ctr;
            q.tiles = d_tiles;
            q.ia = d_ia;
            q.ntile = ctr + 5;
            q.tile_cap = cap2;
            q.tile = o.chunk;
            q.cursor = ctr + 20;
            q.split = set.split;
            q.ins = ins ? *ins : Instr{nullptr, nullptr, 0, 0};
            TC_CUDA(hub_launch());
            mark(5);
            if (ins)
                k_merge<STREAM_EPL, true><<<L.sms * L.occ_merge, 256, 0, st>>>(set.row_ptr, set.adj, d_seg, q, acc);
            else
                k_merge<STREAM_EPL, false><<<L.sms * L.occ_merge, 256, 0, st>>>(set.row_ptr, set.adj, d_seg, q, acc);
            TC_CUDA(cudaGetLastError());
            mark(6);
            mark(7);
            mark(8);
        } else {
            if (o.split_cta)
                k_cta<<<L.sms * L.occ_cta, CTA_NT, 0, st>>>(set.row_ptr, set.adj, d_seg, d_tiles, d_ia, ctr + 5, cap2,
                                                            o.chunk, acc);
            else
                k_warp<<<L.sms * L.occ_warp, 256, 0, st>>>(set.row_ptr, set.adj, d_seg, set.split, d_tiles, d_ia,
                                                            ctr + 5, cap2, o.chunk, acc);
            TC_CUDA(cudaGetLastError());
            mark(5);
            k_stream<STREAM_EPL><<<L.sms * L.occ_stream, 256, 0, st>>>(set.row_ptr, set.adj, d_seg, set.split,
                                                                               bins.rec[3], ctr + 3, bins.cap[3], acc);
            TC_CUDA(cudaGetLastError());
            TC_CUDA(hub_launch());
            mark(6);
            k_warp<<<L.sms * L.occ_warp, 256, 0, st>>>(set.row_ptr, set.adj, d_seg, set.split, bins.rec[1], nullptr,
                                                        ctr + 1, bins.cap[1], 0, acc);
            TC_CUDA(cudaGetLastError());
            mark(7);
            k_thread<<<L.sms * L.occ_thread, 256, 0, st>>>(set.row_ptr, set.adj, d_seg, set.split, bins.rec[0],
                                                            ctr + 0, bins.cap[0], acc);
            TC_CUDA(cudaGetLastError());
        }
    } else {
        for (int k = 1; k <= 7; ++k) mark(k);
    }
    mark(8);
    k_fold<<<(Lo.nseg + 127) / 128, 128, 0, st>>>(acc, d_seg, Lo.nseg, d_out, d_codes, Lo.raw);
    TC_CUDA(cudaGetLastError());
    mark(9);
    return TC_OK;
}

// Kernels of this library a census launches (a prefix scan is 3 kernels).
int census_launches(const Layout& Lo) {
    if (Lo.rows == 0) return 1;
    // 3 rank kernels, the task pass (3 row-wise kernels, or k_tasks +
    // k_fwd_flags), 6 forward-list kernels, 2 lookup kernels, k_fold, and
    // the scans of the rank classes, the forward flags and the owned dyads
    if (Lo.fwd) return (Lo.flat ? 15 : 14) + 9;
    const int route = Lo.o.bin_mode == TC_BIN_MLP && cost_model_weights() ? 1 : 0;
    const int tasks = Lo.flat ? (Lo.o.own_min > 0 ? 2 : 1) + 3 : 1;  // the tag scan, k_owner_rows, k_tasks_flat
    return (Lo.o.persistent ? 4 : 7) + tasks + route + (Lo.o.own_min > 0 ? 2 : 0) + (Lo.exact ? 1 : 0);
}

tc_status read_profile(const Layout& Lo, const char* ws, ProfileEvents* pe, cudaStream_t st) {
    unsigned int c[CTR_WORDS];
    TC_CUDA(cudaMemcpyAsync(c, ws + Lo.o_ctr, sizeof c, cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    tc_profile_t& P = g_profile;
    P = tc_profile_t{};
    // marks: 0 start, 1 tasks, 2 split (forward lists), 3 owner prep
    // (tag-map owners), 4 owners (the other owners), 5..8 merge kernels, 9 fold
    float ms[NEV] = {0};
    for (int k = 0; k + 1 < NEV; ++k) TC_CUDA(cudaEventElapsedTime(&ms[k], pe->ev[k], pe->ev[k + 1]));
    float total = 0;
    TC_CUDA(cudaEventElapsedTime(&total, pe->ev[0], pe->ev[NEV - 1]));
    P.ms_tasks = ms[0];
    if (Lo.fwd) {
        P.ms_forward = ms[1];
        P.ms_tri_map = ms[2];
        P.ms_tri_search = ms[3];
    } else {
        P.ms_split = ms[1];
        P.ms_owner_prep = ms[2];
        P.ms_owner = ms[3];
        if (Lo.o.persistent) {
            P.ms_stream = ms[4];          // hub tasks
            P.ms_merge = ms[4] + ms[5];   // hub tasks + k_merge
        } else {
            P.ms_tiles = ms[4];
            P.ms_stream = ms[5];
            P.ms_warp = ms[6];
            P.ms_thread = ms[7];
            P.ms_merge = ms[4] + ms[5] + ms[6] + ms[7];
        }
    }
    P.ms_fold = ms[8];
    P.ms_total = total;
    if (Lo.exact) TC_CUDA(cudaEventElapsedTime(&P.ms_exact_cost, pe->ev[NEV], pe->ev[0]));
    P.launches = census_launches(Lo);
    const bool routed = Lo.o.bin_mode == TC_BIN_MLP && cost_model_weights();
    auto u64 = [&](int w) { return (int64_t)(((unsigned long long)c[w + 1] << 32) | c[w]); };
    for (int b = 0; b < NBIN; ++b) {
        P.bin_tasks[b] = (b == 2 && routed) ? c[6] : c[b];
        P.bin_entries[b] = u64(10 + 2 * b);
    }
    P.chunks = c[5];
    P.hub_tasks = c[7];
    P.hub_entries = u64(24);
    P.owner_items = (int64_t)c[28] + c[29];
    P.owner_tasks = u64(32);
    P.owner_entries = u64(34);
    P.owner_probes = u64(36);
    P.owner_staged = u64(38);
    if (Lo.fwd) {
        P.fwd_entries = Lo.dyads;
        P.map_items = std::min<int64_t>(c[40], Lo.item_cap);
        P.map_lookups = u64(44);
        P.map_triangles = u64(46);
        P.search_lookups = u64(48);
        P.search_triangles = u64(50);
        unsigned long long tot = 0;  // records: tag-map owners << 32 | the others
        TC_CUDA(cudaMemcpyAsync(&tot, ws + Lo.o_tpre + sizeof(unsigned long long) * (size_t)Lo.rows,
                                sizeof tot, cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
        P.map_dyads = (int64_t)(tot >> 32);
        P.search_dyads = (int64_t)(tot & 0xffffffffull);
        P.map_list_entries = u64(52);
    }
    g_profile_valid = true;
    return TC_OK;
}

// A shard of the census (tc_census_shard): shard `shard` of `nshards`, the
// raw accumulators of graph i written to raw[slot(i)] (device).
struct Shard {
    int32_t shard = 0, nshards = 1;
    unsigned long long* raw = nullptr;
};

// One census over the graphs gidx with a resolved tri_path; with slots,
// graph i's record goes to out[slots[i]] (device output only).
tc_status census_part(GraphSet& set, const std::vector<int32_t>& gidx, const tc_opts* opts_in,
                      tc_census_t* out, uint32_t flags, cudaStream_t st, const Instr* ins = nullptr,
                      tc_census64_t* codes = nullptr, const std::vector<int32_t>* slots = nullptr,
                      const Shard* sh = nullptr) {
    Layout Lo;
    if (tc_status s = make_layout(set, gidx, opts_in, Lo, slots); s != TC_OK) return s;
    if (sh) {
        Lo.shard = sh->shard;
        Lo.nshards = sh->nshards;
        Lo.raw = sh->raw;
    }
    Lo.ids = codes != nullptr || sh != nullptr;
    if (set.ws_bytes < Lo.need) {
        dev_free(set.ws, st);
        set.ws = nullptr;
        set.ws_bytes = 0;
        TC_CUDA(dev_alloc(&set.ws, Lo.need, st));
        set.ws_bytes = Lo.need;
    }
    char* ws = (char*)set.ws;
    const bool dev = (flags & TC_OUT_DEVICE) != 0;
    tc_census_t* d_out = dev && out ? out : (tc_census_t*)(ws + Lo.o_out);
    tc_census64_t* d_codes = !codes ? nullptr : dev ? codes : (tc_census64_t*)(ws + Lo.o_codes);
    ProfileEvents* pe = nullptr;
    if (Lo.o.profile) {
        if (tc_status s = profile_events(&pe); s != TC_OK) return s;
    }
    if (tc_status s = upload_layout(Lo, ws, st); s != TC_OK) return s;
    if (tc_status s = enqueue_census(set, Lo, ws, d_out, st, pe, ins, d_codes); s != TC_OK) return s;
    if (pe) {
        if (tc_status s = read_profile(Lo, ws, pe, st); s != TC_OK) return s;
    }
    if (!dev) {
        int ovf = 0;
        if (out)
            TC_CUDA(cudaMemcpyAsync(out, d_out, sizeof(tc_census_t) * (size_t)Lo.nseg, cudaMemcpyDeviceToHost, st));
        if (codes)
            TC_CUDA(cudaMemcpyAsync(codes, d_codes, sizeof(tc_census64_t) * (size_t)Lo.nseg, cudaMemcpyDeviceToHost,
                                    st));
        TC_CUDA(cudaMemcpyAsync(&ovf, ws + Lo.o_ctr + 4 * sizeof(unsigned int), sizeof(int),
                                cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
        if (ovf) return fail(TC_ERR_CUDA, "census: task bin overflow (internal error)");
    }
    return TC_OK;
}

// tri_path = TC_TRI_AUTO: the graphs routed to each path (path_route), with
// their positions in the caller's list.
struct Parts {
    std::vector<int32_t> gidx[2], slots[2];  // [0] forward, [1] merge
};

tc_status split_parts(const GraphSet& set, const std::vector<int32_t>& gidx, cudaStream_t st, Parts& P) {
    std::vector<uint8_t> merge;
    if (tc_status s = path_route(set, gidx, merge, st); s != TC_OK) return s;
    for (size_t i = 0; i < gidx.size(); ++i) {
        P.gidx[merge[i]].push_back(gidx[i]);
        P.slots[merge[i]].push_back((int32_t)i);
    }
    return TC_OK;
}

// out and/or codes (either may be null): one record per graph, host memory
// or, with TC_OUT_DEVICE, device memory.  With tri_path = TC_TRI_AUTO each
// graph is censused on the path the router picks (two censuses, records in
// the caller's order; a profiled call profiles the second).
tc_status census_impl(GraphSet& set, const std::vector<int32_t>& gidx, const tc_opts* opts_in,
                      tc_census_t* out, uint32_t flags, cudaStream_t st, const Instr* ins = nullptr,
                      tc_census64_t* codes = nullptr, const Shard* sh = nullptr) {
    if (flags & ~TC_OUT_DEVICE) return fail(TC_ERR_ARG, "census: unknown flag");
    tc_opts resolved;
    if (!opts_in) {  // the defaults (tri_path TC_TRI_AUTO)
        tc_opts_default(&resolved);
        opts_in = &resolved;
    }
    if (opts_in->tri_path != TC_TRI_AUTO)
        return census_part(set, gidx, opts_in, out, flags, st, ins, codes, nullptr, sh);
    Parts P;
    if (tc_status s = split_parts(set, gidx, st, P); s != TC_OK) return s;
    const bool dev = (flags & TC_OUT_DEVICE) != 0;
    const size_t G = gidx.size();
    tc_census_t* d_out = dev ? out : nullptr;
    tc_census64_t* d_codes = dev ? codes : nullptr;
    if (!dev && !sh) {  // device staging for the records, copied back at the end
        if (out) TC_CUDA(dev_alloc((void**)&d_out, sizeof(tc_census_t) * std::max<size_t>(G, 1), st));
        if (codes) TC_CUDA(dev_alloc((void**)&d_codes, sizeof(tc_census64_t) * std::max<size_t>(G, 1), st));
    }
    tc_status r = TC_OK;
    for (int k = 0; k < 2 && r == TC_OK; ++k) {
        if (P.gidx[k].empty()) continue;
        tc_opts o = *opts_in;
        o.tri_path = k == 0 ? TC_TRI_FORWARD : TC_TRI_MERGE;
        r = census_part(set, P.gidx[k], &o, d_out, TC_OUT_DEVICE, st, ins, d_codes, &P.slots[k], sh);
    }
    if (!dev && !sh) {
        if (r == TC_OK && out)
            r = cudaMemcpyAsync(out, d_out, sizeof(tc_census_t) * G, cudaMemcpyDeviceToHost, st) == cudaSuccess
                    ? TC_OK : fail(TC_ERR_CUDA, "census: copy of the records");
        if (r == TC_OK && codes)
            r = cudaMemcpyAsync(codes, d_codes, sizeof(tc_census64_t) * G, cudaMemcpyDeviceToHost, st) == cudaSuccess
                    ? TC_OK : fail(TC_ERR_CUDA, "census: copy of the records");
        if (r == TC_OK && cudaStreamSynchronize(st) != cudaSuccess) r = fail(TC_ERR_CUDA, "census: synchronise");
        if (d_out) dev_free(d_out, st);
        if (d_codes) dev_free(d_codes, st);
    }
    return r;
}

std::vector<int32_t> handle_indices(int32_t G, const tc_graph* gs) {
    std::vector<int32_t> idx((size_t)G);
    for (int32_t i = 0; i < G; ++i) idx[(size_t)i] = gs[i]->index;
    return idx;
}

tc_status check_handles(int32_t G, const tc_graph* gs, const char* who) {
    if (G < 0 || (G > 0 && !gs)) return fail(TC_ERR_ARG, std::string(who) + ": bad arguments");
    for (int32_t i = 0; i < G; ++i) {
        if (!gs[i]) return fail(TC_ERR_ARG, std::string(who) + ": null handle");
        if (gs[i]->set != gs[0]->set)
            return fail(TC_ERR_UNSUPPORTED, std::string(who) + ": handles come from different builds");
    }
    return TC_OK;
}

}  // namespace
}  // namespace tc

extern "C" {

tc_status tc_census_profile(tc_profile_t* out) {
    if (!out) return tc::fail(TC_ERR_ARG, "tc_census_profile: null");
    if (!tc::g_profile_valid) return tc::fail(TC_ERR_ARG, "tc_census_profile: no profiled census on this thread");
    *out = tc::g_profile;
    return TC_OK;
}

int tc_triad_type(int code) { return (code < 0 || code > 63) ? -1 : tc::triad_type(code); }

tc_status tc_census(tc_graph g, const tc_opts* opts, tc_census_t* out, uint32_t flags, void* stream) {
    if (!g || !out) return tc::fail(TC_ERR_ARG, "tc_census: null argument");
    try {
        std::vector<int32_t> idx{g->index};
        return tc::census_impl(*g->set, idx, opts, out, flags, (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        return tc::fail(TC_ERR_OOM, "tc_census: host allocation failed");
    } catch (...) {
        return tc::fail(TC_ERR_CUDA, "tc_census: unexpected exception");
    }
}

tc_status tc_census_batched(int32_t G, const tc_graph* gs, const tc_opts* opts, tc_census_t* out,
                            uint32_t flags, void* stream) {
    if (G < 0 || (G > 0 && (!gs || !out))) return tc::fail(TC_ERR_ARG, "tc_census_batched: bad arguments");
    if (G == 0) return TC_OK;
    try {
        if (tc_status s = tc::check_handles(G, gs, "tc_census_batched"); s != TC_OK) return s;
        return tc::census_impl(*gs[0]->set, tc::handle_indices(G, gs), opts, out, flags, (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        return tc::fail(TC_ERR_OOM, "tc_census_batched: host allocation failed");
    } catch (...) {
        return tc::fail(TC_ERR_CUDA, "tc_census_batched: unexpected exception");
    }
}

tc_status tc_census_shard(int32_t G, const tc_graph* gs, const tc_opts* opts, int32_t shard, int32_t nshards,
                          uint64_t* acc, void* stream) {
    if (G < 0 || (G > 0 && (!gs || !acc)) || nshards < 1 || shard < 0 || shard >= nshards)
        return tc::fail(TC_ERR_ARG, "tc_census_shard: bad arguments");
    if (G == 0) return TC_OK;
    try {
        if (tc_status s = tc::check_handles(G, gs, "tc_census_shard"); s != TC_OK) return s;
        tc::Shard sh;
        sh.shard = shard;
        sh.nshards = nshards;
        sh.raw = (unsigned long long*)acc;
        return tc::census_impl(*gs[0]->set, tc::handle_indices(G, gs), opts, nullptr, TC_OUT_DEVICE,
                               (cudaStream_t)stream, nullptr, nullptr, &sh);
    } catch (const std::bad_alloc&) {
        return tc::fail(TC_ERR_OOM, "tc_census_shard: host allocation failed");
    } catch (...) {
        return tc::fail(TC_ERR_CUDA, "tc_census_shard: unexpected exception");
    }
}

tc_status tc_census_fold(int32_t G, const tc_graph* gs, const uint64_t* acc, tc_census_t* out,
                         tc_census64_t* codes, uint32_t flags, void* stream) {
    if (G < 0 || (G > 0 && (!gs || !acc || (!out && !codes))))
        return tc::fail(TC_ERR_ARG, "tc_census_fold: bad arguments");
    if (flags & ~TC_OUT_DEVICE) return tc::fail(TC_ERR_ARG, "tc_census_fold: unknown flag");
    if (G == 0) return TC_OK;
    try {
        if (tc_status s = tc::check_handles(G, gs, "tc_census_fold"); s != TC_OK) return s;
        const tc::GraphSet& set = *gs[0]->set;
        cudaStream_t st = (cudaStream_t)stream;
        std::vector<tc::SegDev> seg((size_t)G);
        for (int32_t i = 0; i < G; ++i) {
            const int32_t g = gs[i]->index;
            seg[(size_t)i].rb = set.voff[(size_t)g];
            seg[(size_t)i].n = set.voff[(size_t)g + 1] - set.voff[(size_t)g];
            seg[(size_t)i].eb = 0;
            seg[(size_t)i].slot = i;
            seg[(size_t)i].pad = 0;
        }
        const bool dev = (flags & TC_OUT_DEVICE) != 0;
        const size_t so = sizeof(tc_census_t) * (size_t)G, sc = sizeof(tc_census64_t) * (size_t)G;
        const size_t bytes = sizeof(tc::SegDev) * (size_t)G + (dev ? 0 : (out ? so : 0) + (codes ? sc : 0));
        char* buf = nullptr;
        TC_CUDA(tc::dev_alloc((void**)&buf, bytes, st));
        tc::SegDev* d_seg = (tc::SegDev*)buf;
        tc_census_t* d_out = !out ? nullptr : dev ? out : (tc_census_t*)(buf + sizeof(tc::SegDev) * (size_t)G);
        tc_census64_t* d_codes = !codes ? nullptr : dev ? codes
                                 : (tc_census64_t*)(buf + sizeof(tc::SegDev) * (size_t)G + (out ? so : 0));
        cudaError_t e = cudaMemcpyAsync(d_seg, seg.data(), sizeof(tc::SegDev) * (size_t)G, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            tc::k_fold<<<(G + 127) / 128, 128, 0, st>>>((const unsigned long long*)acc, d_seg, G, d_out, d_codes,
                                                         nullptr);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && !dev && out) e = cudaMemcpyAsync(out, d_out, so, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && !dev && codes) e = cudaMemcpyAsync(codes, d_codes, sc, cudaMemcpyDeviceToHost, st);
        // the segment table is a pageable upload: wait for it before release
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        tc::dev_free(buf, st);
        if (e != cudaSuccess) return tc::cuda_fail(e, "tc_census_fold", __FILE__, __LINE__);
        return TC_OK;
    } catch (const std::bad_alloc&) {
        return tc::fail(TC_ERR_OOM, "tc_census_fold: host allocation failed");
    } catch (...) {
        return tc::fail(TC_ERR_CUDA, "tc_census_fold: unexpected exception");
    }
}

tc_status tc_census_codes(tc_graph g, const tc_opts* opts, tc_census64_t* out, uint32_t flags, void* stream) {
    if (!g || !out) return tc::fail(TC_ERR_ARG, "tc_census_codes: null argument");
    try {
        std::vector<int32_t> idx{g->index};
        return tc::census_impl(*g->set, idx, opts, nullptr, flags, (cudaStream_t)stream, nullptr, out);
    } catch (const std::bad_alloc&) {
        return tc::fail(TC_ERR_OOM, "tc_census_codes: host allocation failed");
    } catch (...) {
        return tc::fail(TC_ERR_CUDA, "tc_census_codes: unexpected exception");
    }
}

tc_status tc_census_codes_batched(int32_t G, const tc_graph* gs, const tc_opts* opts, tc_census64_t* out,
                                  uint32_t flags, void* stream) {
    if (G < 0 || (G > 0 && (!gs || !out))) return tc::fail(TC_ERR_ARG, "tc_census_codes_batched: bad arguments");
    if (G == 0) return TC_OK;
    try {
        if (tc_status s = tc::check_handles(G, gs, "tc_census_codes_batched"); s != TC_OK) return s;
        return tc::census_impl(*gs[0]->set, tc::handle_indices(G, gs), opts, nullptr, flags, (cudaStream_t)stream,
                               nullptr, out);
    } catch (const std::bad_alloc&) {
        return tc::fail(TC_ERR_OOM, "tc_census_codes_batched: host allocation failed");
    } catch (...) {
        return tc::fail(TC_ERR_CUDA, "tc_census_codes_batched: unexpected exception");
    }
}

}  // extern "C"

// ------------------------------------------------ allocation-free census --
// tc_census_csr_noalloc: the census of a caller-held device CSR using only a
// fixed scratch area compiled into the library (see tc.h for who needs it).
// It runs the same task-build, per-thread merge and fold kernels as
// tc_census, with every dyad routed to the thread-per-task merge, which reads
// no word past the end of a neighbour list, so the caller's adjacency needs
// no padding.
namespace tc {
namespace {

constexpr int64_t NOALLOC_MAX_N = TC_NOALLOC_MAX_N;
constexpr int64_t NOALLOC_MAX_DYADS = TC_NOALLOC_MAX_DYADS;

struct NoallocLayout {
    unsigned long long acc[ACC];  // per-code accumulators + dyadic slots
    unsigned int ctr[32];         // bin counters, capacity flag, row cursor, bin sums
    unsigned int bad[4];          // CSR checks: [0] row offsets, [1] neighbour id outside [0, n)
    SegDev seg;                   // the single graph
    int64_t pfx[2];
    int32_t deg[NOALLOC_MAX_N];
    uint4 rec[NOALLOC_MAX_DYADS];
};

// The scratch itself.  In host code this name is only a stand-in for the
// device object: kernels receive the address looked up below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocLayout)];

// The device address of the scratch on the current device.  Looked up on
// every call: cudaGetSymbolAddress allocates nothing once the module is
// loaded on the device (the first call on a device loads it), and a fresh
// lookup stays right after the caller resets the device, when the module is
// loaded again and the array may sit elsewhere.
tc_status noalloc_scratch(NoallocLayout** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(scratch)", __FILE__, __LINE__);
    *out = (NoallocLayout*)p;
    return TC_OK;
}

// Clears the accumulators and counters left by the previous call, fills the
// graph descriptor and the degree array, and checks the caller's CSR: row
// offsets from 0 to nnz without decreasing, every neighbour id in [0, n).
__global__ void k_noalloc_init(NoallocLayout* s, const int64_t* __restrict__ row_ptr,
                               const uint32_t* __restrict__ adj, int32_t n, int64_t nnz) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    if (tid < ACC) s->acc[tid] = 0;
    if (tid < 32) s->ctr[tid] = 0;
    if (tid == 0) {
        s->seg.rb = 0;
        s->seg.n = n;
        s->seg.eb = 0;
        s->seg.slot = 0;
        s->seg.pad = 0;
        s->pfx[0] = 0;
        s->pfx[1] = n;
        if (row_ptr[0] != 0 || row_ptr[n] != nnz) s->bad[0] = 1;
    }
    for (int64_t x = tid; x < n; x += step) {
        const int64_t d = row_ptr[x + 1] - row_ptr[x];
        if (d < 0) s->bad[0] = 1;
        s->deg[x] = (int32_t)d;
    }
    for (int64_t k = tid; k < nnz; k += step)
        if ((adj[k] >> 2) >= (uint32_t)n) s->bad[1] = 1;
}

tc_status census_noalloc(int32_t n, const int64_t* row_ptr, const uint32_t* adj, int64_t nnz,
                         tc_census_t* out, cudaStream_t st) {
    if (n < 0 || nnz < 0 || (nnz & 1)) return fail(TC_ERR_ARG, "tc_census_csr_noalloc: negative or odd size");
    if (!row_ptr || !out || (nnz > 0 && !adj)) return fail(TC_ERR_ARG, "tc_census_csr_noalloc: null pointer");
    if (n > NOALLOC_MAX_N)
        return fail(TC_ERR_UNSUPPORTED, "tc_census_csr_noalloc: n exceeds TC_NOALLOC_MAX_N (262144)");
    if (nnz / 2 > NOALLOC_MAX_DYADS)
        return fail(TC_ERR_UNSUPPORTED, "tc_census_csr_noalloc: nnz/2 exceeds TC_NOALLOC_MAX_DYADS (262144)");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    TC_CUDA(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone)
        return fail(TC_ERR_ARG, "tc_census_csr_noalloc: the stream is capturing (the call synchronises it)");
    NoallocLayout* s = nullptr;
    if (tc_status r = noalloc_scratch(&s); r != TC_OK) return r;
    Launch L;
    if (tc_status r = launch_info(L); r != TC_OK) return r;
    TC_CUDA(cudaMemsetAsync(s->bad, 0, sizeof(s->bad), st));
    const int64_t span = std::max<int64_t>(n, nnz);
    k_noalloc_init<<<std::max(1, (int)std::min<int64_t>((span + 255) / 256, (int64_t)L.sms * 8)), 256, 0, st>>>(
        s, row_ptr, adj, n, nnz);
    TC_CUDA(cudaGetLastError());
    unsigned int bad[2] = {0, 0};
    TC_CUDA(cudaMemcpyAsync(bad, s->bad, sizeof(bad), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    if (bad[0])
        return fail(TC_ERR_ARG, "tc_census_csr_noalloc: row_ptr does not run from 0 to nnz without decreasing");
    if (bad[1]) return fail(TC_ERR_ID_RANGE, "tc_census_csr_noalloc: a neighbour id outside [0, n)");
    Bins bins;
    bins.rec[0] = bins.rec[1] = bins.rec[2] = bins.rec[3] = s->rec;
    // a well-formed CSR lists each dyad in both rows, so it has nnz/2 dyads
    bins.cap[0] = (uint32_t)(nnz / 2);
    bins.cap[1] = bins.cap[2] = bins.cap[3] = 0;
    bins.cnt = s->ctr;
    bins.overflow = (int*)(s->ctr + 4);
    bins.entries = (unsigned long long*)(s->ctr + 10);
    unsigned long long* cursor = (unsigned long long*)(s->ctr + 8);
    bins.own = nullptr;
    bins.own_cap = 0;
    bins.own_cnt = nullptr;
    bins.own_stat = nullptr;
    const BinParams bp{0x7fffffff, 0x7fffffff, 0, 0, nullptr, nullptr, 0, nullptr, 0, INT64_MAX, 0, INT64_MAX};
    if (n > 0) {
        k_tasks<<<L.sms * L.occ_tasks, 256, 0, st>>>(row_ptr, adj, s->deg, &s->seg, s->pfx, 1, n, bp, bins,
                                                     s->acc, cursor);
        TC_CUDA(cudaGetLastError());
        k_thread<<<L.sms * L.occ_thread, 256, 0, st>>>(row_ptr, adj, &s->seg, nullptr, s->rec, s->ctr + 0,
                                                        bins.cap[0], s->acc);
        TC_CUDA(cudaGetLastError());
    }
    k_fold<<<1, 128, 0, st>>>(s->acc, &s->seg, 1, out, nullptr, nullptr);
    TC_CUDA(cudaGetLastError());
    int ovf = 0;
    TC_CUDA(cudaMemcpyAsync(&ovf, s->ctr + 4, sizeof(int), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    if (ovf)
        return fail(TC_ERR_UNSUPPORTED, "tc_census_csr_noalloc: the CSR holds more dyads than nnz/2 "
                                        "(not symmetric; result invalid)");
    return TC_OK;
}

}  // namespace
}  // namespace tc

extern "C" tc_status tc_census_csr_noalloc(int32_t n, const int64_t* row_ptr, const uint32_t* adj, int64_t nnz,
                                           tc_census_t* out, void* stream) {
    try {
        return tc::census_noalloc(n, row_ptr, adj, nnz, out, (cudaStream_t)stream);
    } catch (...) {
        return tc::fail(TC_ERR_CUDA, "tc_census_csr_noalloc: unexpected exception");
    }
}

// ------------------------------------------------------------ batch plans --
struct tc_plan_s {
    std::shared_ptr<tc::GraphSet> set;
    tc::Layout lo[2];        // one census, or (TC_TRI_AUTO) the forward and the merge part
    char* ws[2] = {nullptr, nullptr};
    int parts = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace tc {
namespace {

tc_status plan_create(int32_t G, const tc_graph* gs, const tc_opts* opts, tc_census_t* out, cudaStream_t st,
                      tc_plan* result) {
    if (G < 1 || !gs || !out || !result) return fail(TC_ERR_ARG, "tc_plan_create: bad arguments");
    if (tc_status s = check_handles(G, gs, "tc_plan_create"); s != TC_OK) return s;
    if (opts && opts->profile) return fail(TC_ERR_ARG, "tc_plan_create: profile must be 0 in a plan");
    std::unique_ptr<tc_plan_s> p(new tc_plan_s);
    p->set = gs[0]->set;
    const std::vector<int32_t> idx = handle_indices(G, gs);
    tc_opts resolved;
    if (!opts) {  // the defaults (tri_path TC_TRI_AUTO)
        tc_opts_default(&resolved);
        opts = &resolved;
    }
    Parts P;
    tc_opts po[2];
    if (opts && opts->tri_path == TC_TRI_AUTO) {  // a census per path, records in the caller's order
        if (tc_status s = split_parts(*p->set, idx, st, P); s != TC_OK) return s;
        for (int k = 0; k < 2; ++k) {
            if (P.gidx[k].empty()) continue;
            po[p->parts] = *opts;
            po[p->parts].tri_path = k == 0 ? TC_TRI_FORWARD : TC_TRI_MERGE;
            if (tc_status s = make_layout(*p->set, P.gidx[k], &po[p->parts], p->lo[p->parts], &P.slots[k]);
                s != TC_OK)
                return s;
            ++p->parts;
        }
    } else {
        if (tc_status s = make_layout(*p->set, idx, opts, p->lo[0]); s != TC_OK) return s;
        p->parts = 1;
    }
    Launch L;
    if (tc_status s = launch_info(L); s != TC_OK) return s;
    struct Guard {
        tc_plan_s* p;
        cudaStream_t st;
        bool ok = false;
        ~Guard() {
            if (!ok) {
                cudaStreamSynchronize(st);
                if (p->exec) cudaGraphExecDestroy(p->exec);
                if (p->graph) cudaGraphDestroy(p->graph);
                for (int k = 0; k < 2; ++k) dev_free(p->ws[k], st);
                cudaStreamSynchronize(st);
            }
        }
    } guard{p.get(), st};
    for (int k = 0; k < p->parts; ++k) {
        TC_CUDA(dev_alloc((void**)&p->ws[k], p->lo[k].need, st));
        if (tc_status s = upload_layout(p->lo[k], p->ws[k], st); s != TC_OK) return s;
    }
    TC_CUDA(cudaStreamSynchronize(st));
    cudaStream_t cap = nullptr;
    TC_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    tc_status s = TC_OK;
    if (e == cudaSuccess) {
        for (int k = 0; k < p->parts && s == TC_OK; ++k)
            s = enqueue_census(*p->set, p->lo[k], p->ws[k], out, cap, nullptr);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (s == TC_OK && e2 != cudaSuccess) s = cuda_fail(e2, "cudaStreamEndCapture", __FILE__, __LINE__);
        p->graph = g;
    } else {
        s = cuda_fail(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
    }
    cudaStreamDestroy(cap);
    if (s != TC_OK) return s;
    TC_CUDA(cudaGraphInstantiate(&p->exec, p->graph, 0));
    guard.ok = true;
    *result = p.release();
    return TC_OK;
}

}  // namespace
}  // namespace tc

extern "C" {

tc_status tc_plan_create(int32_t G, const tc_graph* gs, const tc_opts* opts, tc_census_t* out, void* stream,
                         tc_plan* plan) {
    if (plan) *plan = nullptr;
    try {
        return tc::plan_create(G, gs, opts, out, (cudaStream_t)stream, plan);
    } catch (const std::bad_alloc&) {
        return tc::fail(TC_ERR_OOM, "tc_plan_create: host allocation failed");
    } catch (...) {
        return tc::fail(TC_ERR_CUDA, "tc_plan_create: unexpected exception");
    }
}

tc_status tc_plan_run(tc_plan plan, void* stream) {
    if (!plan) return tc::fail(TC_ERR_ARG, "tc_plan_run: null plan");
    TC_CUDA(cudaGraphLaunch(plan->exec, (cudaStream_t)stream));
    return TC_OK;
}

void tc_plan_free(tc_plan plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    for (int k = 0; k < 2; ++k) tc::dev_free(plan->ws[k], 0);
    cudaStreamSynchronize(0);
    delete plan;
}

}  // extern "C"

// -------------------------------------------------------------- autotuner --
// Coordinate descent over the binning and launch options: starting from
// `base`, each option in turn takes the candidate value with the smallest
// measured census time (CUDA events, best of two runs after one warm-up),
// the others held at their current best.  Every trial computes the full
// census; the counts do not depend on the options.
namespace tc {
namespace {

tc_status autotune(int32_t G, const tc_graph* gs, const tc_opts* base, int32_t max_trials, cudaStream_t st,
                   tc_opts* best, float* best_ms, int32_t* trials_out) {
    if (G < 1 || !gs || !best) return fail(TC_ERR_ARG, "tc_autotune: bad arguments");
    if (tc_status s = check_handles(G, gs, "tc_autotune"); s != TC_OK) return s;
    GraphSet& set = *gs[0]->set;
    const std::vector<int32_t> idx = handle_indices(G, gs);
    tc_opts cur;
    tc_opts_default(&cur);
    if (base) cur = *base;
    cur.profile = 0;
    tc_census_t* d_out = nullptr;
    TC_CUDA(dev_alloc((void**)&d_out, sizeof(tc_census_t) * (size_t)G, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TC_CUDA(cudaEventCreate(&e0));
    TC_CUDA(cudaEventCreate(&e1));
    struct Cleanup {
        cudaEvent_t a, b;
        tc_census_t* p;
        cudaStream_t s;
        ~Cleanup() {
            cudaStreamSynchronize(s);
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            dev_free(p, s);
        }
    } cleanup{e0, e1, d_out, st};
    int trials = 0;
    auto timeit = [&](const tc_opts& o, float& ms) -> tc_status {
        float bestv = 3.4e38f;
        for (int r = 0; r < 3; ++r) {
            TC_CUDA(cudaEventRecord(e0, st));
            if (tc_status s = census_impl(set, idx, &o, d_out, TC_OUT_DEVICE, st); s != TC_OK) return s;
            TC_CUDA(cudaEventRecord(e1, st));
            TC_CUDA(cudaEventSynchronize(e1));
            float t = 0;
            TC_CUDA(cudaEventElapsedTime(&t, e0, e1));
            if (r > 0) bestv = std::min(bestv, t);
        }
        ms = bestv;
        ++trials;
        return TC_OK;
    };
    float cur_ms = 0;
    if (tc_status s = timeit(cur, cur_ms); s != TC_OK) return s;
    // coordinate descent over these fields, two passes: first how triangles
    // are found, then that path's own settings (the tag-map threshold of the
    // forward path; for the merge path the owner threshold first, since it
    // decides which dyads reach the merge bins at all)
    const int32_t path_c[] = {TC_TRI_FORWARD, TC_TRI_MERGE, TC_TRI_AUTO};
    const int32_t big_c[] = {8, 16, 32, 64, 128, 256};
    const int32_t own_c[] = {0, 64, 128, 256, 512, 1024, 4096};
    const int32_t thr_thread_c[] = {0, 16, 32, 48, 64, 96, 128, 192};
    const int32_t thr_warp_c[] = {64, 128, 256, 512, 1024};
    const int32_t stream_c[] = {0, 256, 1024, 1 << 30};
    const int32_t chunk_c[] = {256, 512, 1024};
    const int32_t pers_c[] = {0, 1};
    struct Field {
        int32_t tc_opts::*f;
        const int32_t* cand;
        int nc;
    };
    const Field fields[] = {{&tc_opts::tri_path, path_c, 3},     {&tc_opts::fwd_big, big_c, 6},
                            {&tc_opts::own_min, own_c, 7},       {&tc_opts::thr_thread, thr_thread_c, 8},
                            {&tc_opts::thr_warp, thr_warp_c, 5}, {&tc_opts::stream_max, stream_c, 4},
                            {&tc_opts::chunk, chunk_c, 3},       {&tc_opts::persistent, pers_c, 2}};
    for (int pass = 0; pass < 2; ++pass) {
        for (const Field& fd : fields) {
            const int32_t* cand = fd.cand;
            const int nc = fd.nc;
            // a field of the other path changes nothing: skip it
            const bool fwd_field = fd.f == &tc_opts::fwd_big, path_field = fd.f == &tc_opts::tri_path;
            const bool uses_fwd = cur.tri_path != TC_TRI_MERGE, uses_merge = cur.tri_path != TC_TRI_FORWARD;
            if (!path_field && (fwd_field ? !uses_fwd : !uses_merge)) continue;
            for (int k = 0; k < nc; ++k) {
                if (max_trials > 0 && trials >= max_trials) break;
                tc_opts o = cur;
                int32_t* f = &(o.*fd.f);
                if (*f == cand[k]) continue;
                *f = cand[k];
                if (o.thr_thread > o.thr_warp) continue;
                if (o.persistent) o.split_cta = 0;
                float ms = 0;
                if (tc_status s = timeit(o, ms); s != TC_OK) return s;
                if (ms < cur_ms) {
                    cur = o;
                    cur_ms = ms;
                }
            }
        }
    }
    *best = cur;
    if (best_ms) *best_ms = cur_ms;
    if (trials_out) *trials_out = trials;
    return TC_OK;
}

}  // namespace
}  // namespace tc

extern "C" tc_status tc_autotune(int32_t G, const tc_graph* gs, const tc_opts* base, int32_t max_trials, void* stream,
                                 tc_opts* best, float* best_ms, int32_t* trials) {
    try {
        return tc::autotune(G, gs, base, max_trials, (cudaStream_t)stream, best, best_ms, trials);
    } catch (...) {
        return tc::fail(TC_ERR_CUDA, "tc_autotune: unexpected exception");
    }
}

// ------------------------------------------------------- cost sampling --
namespace tc {
namespace {

tc_status cost_sample(int32_t G, const tc_graph* gs, int32_t bin, int32_t mask, int32_t cap, int32_t* samples,
                      int32_t* n_out, cudaStream_t st) {
    if (G < 1 || !gs || bin < 0 || bin > 3 || mask < 0 || cap < 0 || (cap > 0 && !samples) || !n_out)
        return fail(TC_ERR_ARG, "tc_cost_sample: bad arguments");
    if (tc_status s = check_handles(G, gs, "tc_cost_sample"); s != TC_OK) return s;
    tc_opts o;
    tc_opts_default(&o);
    o.tri_path = TC_TRI_MERGE;  // per-task timings come from the merge bins
    o.persistent = 1;
    o.split_cta = 0;
    if (bin == 0) {
        o.thr_thread = 0x3fffffff;
        o.thr_warp = 0x3fffffff;
    } else if (bin == 1) {
        o.thr_thread = 0;
        o.thr_warp = WARP_LMAX;
        o.stream_max = 0;
    } else {
        o.thr_thread = 0;
        o.thr_warp = 0;
        o.stream_max = bin == 3 ? (1 << 30) : 0;
    }
    unsigned int* count = nullptr;
    TC_CUDA(dev_alloc((void**)&count, sizeof(unsigned int), st));
    TC_CUDA(cudaMemsetAsync(count, 0, sizeof(unsigned int), st));
    Instr ins{(int4*)samples, count, (unsigned)cap, (unsigned)mask};
    tc_census_t* out = nullptr;
    TC_CUDA(dev_alloc((void**)&out, sizeof(tc_census_t) * (size_t)G, st));
    tc_status s = census_impl(*gs[0]->set, handle_indices(G, gs), &o, out, TC_OUT_DEVICE, st, &ins);
    unsigned int n = 0;
    if (s == TC_OK) {
        TC_CUDA(cudaMemcpyAsync(&n, count, sizeof n, cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
    }
    dev_free(out, st);
    dev_free(count, st);
    *n_out = (int32_t)std::min<unsigned>(n, (unsigned)cap);
    return s;
}

}  // namespace
}  // namespace tc

extern "C" tc_status tc_cost_sample(int32_t G, const tc_graph* gs, int32_t bin, int32_t mask, int32_t cap,
                                    int32_t* samples, int32_t* n, void* stream) {
    try {
        return tc::cost_sample(G, gs, bin, mask, cap, samples, n, (cudaStream_t)stream);
    } catch (...) {
        return tc::fail(TC_ERR_CUDA, "tc_cost_sample: unexpected exception");
    }
}
