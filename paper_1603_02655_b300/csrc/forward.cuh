// Triangle corrections by degree-ranked forward lists (the census's default
// way of finding the shared neighbours of canonical dyads).
//
// Included by census.cu inside its anonymous namespace, after SegDev,
// seg_of, tag_swap, warp_sum64, ceil_log2 and ACC.
//
// What is computed.  The task pass (k_tasks_flat / k_tasks) adds every
// dyad's suffix terms as if no neighbour were shared (Sec. 2.2, Fig.
// "Subquadratic Triad Census Algorithm", regrouped).  A shared neighbour w
// of a dyad <u,v> changes the classification only through the triangle
// {u, v, w}: with its vertices a < b < c and tags t_ab, t_ac, t_bc, dyad <a,b>
// moves one count from codes t_ab + 4 t_ac and t_ab + 16 t_bc to
// t_ab + 4 t_ac + 16 t_bc, and dyad <a,c> drops the count t_ac + 16 t_cb it
// added for b (the canonical test rejects b there, since b is a neighbour
// of a).  So the census needs each triangle exactly once, with its three
// tags, and nothing else from the shared neighbours (their share of the
// dyadic term comes from the closed-triad counts in k_fold).
//
// How triangles are found.  Vertices are ranked by (floor(log2 d), id) per
// graph (rank R, 0 .. n-1).  The forward list F(x) holds the neighbours of x
// of higher rank, sorted by rank, as R << 2 | tag seen from x.  A triangle
// x, h, w with R(x) < R(h) < R(w) is found exactly once: at the dyad {x, h},
// owned by h, as an element w of the suffix of F(x) after h that also lies
// in F(h).  Because high-degree vertices rank last, every F(h) is short (at
// most a few hundred entries on the power-law workloads), and the suffixes
// sum to about half the lookups of an id-ordered search (R-MAT scale 22:
// 5.3e8 instead of 1.1e9 for the hub dyads alone).
//
// Two lookup forms:
//  * k_tri_big: an owner with many forward neighbours and few vertices
//    ranked above it gets a CTA: a 2-bit tag map over the ranks above R(h)
//    in shared memory (0 = not in F(h), else the tag t_h(w)) answers every
//    lookup exactly with one shared load.  The owner's dyads, one piece of
//    at most TRI_PIECE at a time, are laid out as concatenated suffixes that
//    the warps split evenly.
//  * k_tri_small: every other owner: warps take runs of dyad records; a
//    lookup is a binary search of F(h) (global memory, cached: a run's dyads
//    share few owners).
// Hits (triangles) are queued per warp and applied 32 at a time: the third
// vertex's id is read from the rank permutation, the three vertices are
// ordered by id, and the four histogram updates are made.

constexpr int RK_B = 1024;  // rows per block of the rank computation
constexpr int NCLS = 32;    // degree classes floor(log2 d), d = 0 in class 0

__device__ __forceinline__ int deg_class(int d) { return d > 0 ? 31 - __clz(d) : 0; }

// Row r of the census's selection (graphs concatenated) and its segment.
__device__ __forceinline__ int row_seg(const int64_t* pfx, int nseg, int64_t r) {
    return nseg == 1 ? 0 : seg_of(pfx, nseg, r);
}

// ------------------------------------------------------------ vertex ranks --
// Class counts of each block of RK_B rows, class-major: hist[c * nb + b].
__global__ void __launch_bounds__(RK_B) k_rank_hist(const int32_t* __restrict__ deg, const SegDev* __restrict__ seg,
                                                    const int64_t* __restrict__ pfx, int nseg, int64_t rows, int nb,
                                                    uint32_t* __restrict__ hist) {
    __shared__ unsigned cnt[NCLS];
    if (threadIdx.x < NCLS) cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * RK_B + threadIdx.x;
    if (r < rows) {
        const int s = row_seg(pfx, nseg, r);
        atomicAdd(&cnt[deg_class(deg[seg[s].rb + (r - pfx[s])])], 1u);
    }
    __syncthreads();
    if (threadIdx.x < NCLS) hist[(size_t)threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

// Rows of class c below row p, counted from the class-major exclusive scan
// hex of the block counts (relative to the class's first block) and the rows
// of p's block before p.  One warp; cnt is its shared counter array.
__device__ __forceinline__ unsigned rank_below(const int32_t* deg, const SegDev* seg, const int64_t* pfx, int nseg,
                                               int64_t rows, int nb, const uint32_t* hex, int64_t p, unsigned* cnt,
                                               int lane) {
    const int b = (int)min(p / RK_B, (int64_t)nb - 1);
    cnt[lane] = 0;
    __syncwarp();
    for (int64_t q = (int64_t)b * RK_B + lane; q < p; q += 32) {
        const int s = row_seg(pfx, nseg, q);
        atomicAdd(&cnt[deg_class(deg[seg[s].rb + (q - pfx[s])])], 1u);
    }
    __syncwarp();
    const unsigned v = hex[(size_t)lane * nb + b] - hex[(size_t)lane * nb] + cnt[lane];
    __syncwarp();
    return v;  // for class = lane
}

// Per graph s: co[s][c] = (ranks before class c in the graph) - (rows of
// class c before the graph's first row).  One warp per graph.
__global__ void k_rank_seg(const int32_t* __restrict__ deg, const SegDev* __restrict__ seg,
                           const int64_t* __restrict__ pfx, int nseg, int64_t rows, int nb,
                           const uint32_t* __restrict__ hex, int64_t* __restrict__ co) {
    __shared__ unsigned cnt[NCLS];
    const int lane = threadIdx.x & 31;
    for (int s = blockIdx.x; s < nseg; s += gridDim.x) {
        const unsigned p0 = rank_below(deg, seg, pfx, nseg, rows, nb, hex, pfx[s], cnt, lane);
        const unsigned p1 = rank_below(deg, seg, pfx, nseg, rows, nb, hex, pfx[s + 1], cnt, lane);
        unsigned in = p1 - p0, ex = in;  // class sizes in the graph -> exclusive prefix over classes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, ex, o);
            if (lane >= o) ex += t;
        }
        ex -= in;
        co[(size_t)s * NCLS + lane] = (int64_t)ex - (int64_t)p0;
    }
}

// Rank of every row: its class's first rank in the graph plus the rows of
// the same class before it (stable in id order); perm is the inverse.
__global__ void __launch_bounds__(RK_B) k_rank_assign(const int32_t* __restrict__ deg,
                                                      const SegDev* __restrict__ seg,
                                                      const int64_t* __restrict__ pfx, int nseg, int64_t rows,
                                                      int nb, const uint32_t* __restrict__ hex,
                                                      const int64_t* __restrict__ co, int32_t* __restrict__ rank,
                                                      int32_t* __restrict__ perm, int* __restrict__ err) {
    __shared__ unsigned cw[RK_B / 32][NCLS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = threadIdx.x; c < (RK_B / 32) * NCLS; c += RK_B) (&cw[0][0])[c] = 0;
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * RK_B + threadIdx.x;
    const bool valid = r < rows;
    int s = 0, c = NCLS;  // NCLS: no class (past the last row)
    if (valid) {
        s = row_seg(pfx, nseg, r);
        c = deg_class(deg[seg[s].rb + (r - pfx[s])]);
    }
    const unsigned same = __match_any_sync(0xffffffffu, c);
    const unsigned before = __popc(same & ((1u << lane) - 1u));
    if (valid && before == 0) cw[warp][c] = __popc(same);
    __syncthreads();
    if (threadIdx.x < NCLS) {  // exclusive prefix over the warps, per class
        unsigned run = 0;
        for (int w = 0; w < RK_B / 32; ++w) {
            const unsigned t = cw[w][threadIdx.x];
            cw[w][threadIdx.x] = run;
            run += t;
        }
    }
    __syncthreads();
    if (valid) {
        const int b = blockIdx.x;
        const int64_t P = (int64_t)(hex[(size_t)c * nb + b] - hex[(size_t)c * nb]) + cw[warp][c] + before;
        const int64_t R = co[(size_t)s * NCLS + c] + P;
        if (R >= 0 && R < seg[s].n) {  // always, by construction; checked before it indexes perm
            rank[r] = (int32_t)R;
            perm[pfx[s] + R] = (int32_t)(r - pfx[s]);
        } else {
            rank[r] = 0;
            atomicOr(err, 2);
        }
    }
}

// -------------------------------------------------------- forward lists --
// Entry f of the selection (graphs' adjacency concatenated) is forward when
// its neighbour ranks above its row.
struct FwdFlag {
    const uint32_t* adj;
    const int32_t* arow;
    const SegDev* seg;
    const int64_t* pfx;
    const int64_t* epfx;
    const int32_t* rank;
    int nseg;
    __device__ int operator()(int64_t f) const {
        const int s = nseg == 1 ? 0 : seg_of(epfx, nseg, f);
        const SegDev& g = seg[s];
        const int64_t k = g.eb + (f - epfx[s]);
        const int64_t rx = pfx[s] + ((int64_t)arow[k] - g.rb);
        const int64_t ry = pfx[s] + (int64_t)(__ldg(adj + k) >> 2);
        return rank[ry] > rank[rx] ? 1 : 0;
    }
};
using FwdFlagIt = thrust::transform_iterator<FwdFlag, thrust::counting_iterator<int64_t>, int>;

// Per row: the start of its forward list (from the inclusive scan fs of the
// forward flags), its number of lower-ranked neighbours (the dyads it owns),
// and, for an owner that takes the tag-map path, its work items (pieces of
// TRI_PIECE dyads).
constexpr int TRI_PIECE = 1024;
constexpr int MAP_KEYS = 1 << 17;  // ranks a tag map covers (2 bits each: 32 KB)

struct FwdLayout {
    const int32_t* fs;     // [entries] inclusive count of forward entries
    uint32_t* fptr;        // [rows + 1] forward list start
    uint32_t* nown;        // [rows + 1] dyads owned (lower-ranked neighbours); nown[rows] = 0
    uint32_t* tptr;        // [rows + 1] exclusive scan of nown
    uint32_t* tcur;        // [rows] fill cursors of the dyad records
    uint32_t* fid;         // [dyads] forward entries in id order
    uint32_t* fwd;         // [dyads] forward entries in rank order: R << 2 | tag
    uint4* trec;           // [dyads] dyad records by owner
    uint4* items;          // tag-map work items {owner row, piece, 0, 0}
    uint32_t item_cap;
    unsigned* nitems;      // [1]
    unsigned* cursor;      // [2] work cursors (tag-map items, record runs)
    unsigned long long* stat;  // [4] lookups and triangles of each path
    const int32_t* rank;
    const int32_t* perm;
};

__device__ __forceinline__ bool map_owner(int nplus, int64_t n, int32_t R, int big_min) {
    return nplus >= big_min && nplus > 0 && n - (int64_t)R - 1 <= MAP_KEYS;
}

__global__ void k_fwd_rows(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ deg,
                           const SegDev* __restrict__ seg, const int64_t* __restrict__ pfx,
                           const int64_t* __restrict__ epfx, int nseg, int64_t rows, int big_min, FwdLayout F) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int s = row_seg(pfx, nseg, r);
        const SegDev& g = seg[s];
        const int64_t x = g.rb + (r - pfx[s]);
        const int64_t f0 = epfx[s] + (row_ptr[x] - g.eb), f1 = epfx[s] + (row_ptr[x + 1] - g.eb);
        const uint32_t a = f0 > 0 ? (uint32_t)F.fs[f0 - 1] : 0u, b = f1 > 0 ? (uint32_t)F.fs[f1 - 1] : 0u;
        F.fptr[r] = a;
        const uint32_t own = (uint32_t)deg[x] - (b - a);
        F.nown[r] = own;
        if (r == rows - 1) {
            F.fptr[rows] = b;
            F.nown[rows] = 0;
        }
        if (own > 0 && map_owner((int)(b - a), g.n, F.rank[r], big_min)) {
            const unsigned np = (own + TRI_PIECE - 1) / TRI_PIECE;
            const unsigned k = atomicAdd(F.nitems, np);
            for (unsigned p = 0; p < np; ++p)
                if (k + p < F.item_cap) F.items[k + p] = make_uint4((uint32_t)r, p, 0u, 0u);
        }
    }
}

// Forward entries in id order (a flat pass over the selection's entries).
__global__ void k_fwd_ids(const uint32_t* __restrict__ adj, const SegDev* __restrict__ seg,
                          const int64_t* __restrict__ epfx, int nseg, int64_t entries, FwdLayout F) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < entries;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int32_t here = F.fs[f];
        if (here > (f > 0 ? F.fs[f - 1] : 0)) {
            const int s = nseg == 1 ? 0 : seg_of(epfx, nseg, f);
            F.fid[here - 1] = __ldg(adj + seg[s].eb + (f - epfx[s]));
        }
    }
}

// One warp per row with a forward list: a stable partition of the list (in
// id order) by degree class gives rank order; each entry is written as
// R << 2 | tag, and its dyad {x, y} (owned by y) gets a record in y's part
// of trec: {first entry of the suffix after y, suffix length, x << 2 | tag
// of y seen from x, owner row}.
__global__ void __launch_bounds__(256) k_fwd_sort(const int32_t* __restrict__ deg, const SegDev* __restrict__ seg,
                                                  const int64_t* __restrict__ pfx, int nseg, int64_t rows,
                                                  FwdLayout F) {
    __shared__ unsigned cnt_all[8][NCLS + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned* cnt = cnt_all[warp];
    const unsigned full = 0xffffffffu, lt = (1u << lane) - 1u;
    const int64_t nwarps = (int64_t)gridDim.x * 8;
    for (int64_t r = blockIdx.x * 8 + warp; r < rows; r += nwarps) {
        const uint32_t b0 = F.fptr[r], m = F.fptr[r + 1] - b0;
        if (m == 0) continue;
        const int s = row_seg(pfx, nseg, r);
        const int64_t rb = seg[s].rb, p0 = pfx[s];
        const uint32_t xl = (uint32_t)(r - p0);
        cnt[lane] = 0;
        __syncwarp();
        for (uint32_t i0 = 0; i0 < m; i0 += 32) {
            const uint32_t i = i0 + lane;
            const int c = i < m ? deg_class(deg[rb + (F.fid[b0 + i] >> 2)]) : NCLS;
            const unsigned same = __match_any_sync(full, c);
            if (c < NCLS && (same & lt) == 0) cnt[c] += __popc(same);
            __syncwarp();
        }
        {  // class counts -> exclusive starts
            const unsigned v = cnt[lane];
            unsigned ex = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(full, ex, o);
                if (lane >= o) ex += t;
            }
            __syncwarp();
            cnt[lane] = ex - v;
            __syncwarp();
        }
        for (uint32_t i0 = 0; i0 < m; i0 += 32) {
            const uint32_t i = i0 + lane;
            const uint32_t e = i < m ? F.fid[b0 + i] : 0u;
            const int c = i < m ? deg_class(deg[rb + (e >> 2)]) : NCLS;
            const unsigned same = __match_any_sync(full, c);
            const uint32_t pos = c < NCLS ? cnt[c] + __popc(same & lt) : 0u;
            __syncwarp();
            if (c < NCLS && (same & lt) == 0) cnt[c] += __popc(same);
            __syncwarp();
            if (i < m) {
                const int64_t ry = p0 + (e >> 2);
                F.fwd[b0 + pos] = ((uint32_t)F.rank[ry] << 2) | (e & 3u);
                const uint32_t slot = F.tptr[ry] + atomicAdd(F.tcur + ry, 1u);
                F.trec[slot] = make_uint4(b0 + pos + 1, m - pos - 1, (xl << 2) | (e & 3u), (uint32_t)ry);
            }
        }
    }
}

// ------------------------------------------------------------ triangles --
// The four updates a triangle makes, its vertices given in any order with
// the tags between them (t_pq = e(p,q) + 2 e(q,p)).
__device__ __forceinline__ void tri_correct(int32_t* h, uint32_t a, uint32_t b, uint32_t c, uint32_t t_ab,
                                            uint32_t t_ac, uint32_t t_bc) {
    uint32_t t;
    if (a > b) {
        t = a; a = b; b = t;
        t_ab = tag_swap(t_ab);
        t = t_ac; t_ac = t_bc; t_bc = t;
    }
    if (b > c) {
        t = b; b = c; c = t;
        t_bc = tag_swap(t_bc);
        t = t_ab; t_ab = t_ac; t_ac = t;
    }
    if (a > b) {
        t = a; a = b; b = t;
        t_ab = tag_swap(t_ab);
        t = t_ac; t_ac = t_bc; t_bc = t;
    }
    atomicAdd(h + t_ab + 4 * t_ac, -1);
    atomicAdd(h + t_ab + 16 * t_bc, -1);
    atomicAdd(h + t_ab + 4 * t_ac + 16 * t_bc, 1);
    atomicAdd(h + t_ac + 16 * tag_swap(t_bc), -1);
}

// Per-warp 32-bit histogram of the 64 codes for one graph, added into the
// graph's 64-bit accumulators when the graph changes and at the end, and
// before a slot could leave the int32 range (a triangle moves a slot by at
// most 4).
struct TriHist {
    int32_t* hs;
    unsigned long long* acc;
    int tag;
    int lane;
    unsigned pending;
    __device__ __forceinline__ void flush() {
        if (tag >= 0)
            for (int j = lane; j < 64; j += 32) {
                const int32_t v = hs[j];
                if (v) atomicAdd(acc + (size_t)tag * ACC + j, (unsigned long long)(long long)v);
                hs[j] = 0;
            }
        __syncwarp();
        pending = 0;
    }
    __device__ __forceinline__ void retag(int s) {
        if (s != tag || pending > (1u << 28)) {
            flush();
            tag = s;
        }
    }
};

constexpr int TQN = 64;  // per-warp queue of hits (ring)

struct TriQueue {
    uint2* q;   // {R << 2 | t_h(w), dyad << 2 | t_x(w)}
    int head, n;
};

// Shared-memory layout of k_tri_big.
constexpr int TB_NT = 512;
constexpr int TB_W = TB_NT / 32;
constexpr size_t TB_MAP_BYTES = sizeof(uint32_t) * (MAP_KEYS / 16);
constexpr size_t TB_OFF_BYTES = sizeof(uint32_t) * (TRI_PIECE + 32);
constexpr size_t TB_FST_BYTES = sizeof(uint32_t) * TRI_PIECE;
constexpr size_t TB_XIN_BYTES = sizeof(uint32_t) * TRI_PIECE;
constexpr size_t TB_HS_BYTES = sizeof(int32_t) * 64 * TB_W;
constexpr size_t TB_Q_BYTES = sizeof(uint2) * TQN * TB_W;
constexpr size_t TB_SMEM = TB_MAP_BYTES + TB_OFF_BYTES + TB_FST_BYTES + TB_XIN_BYTES + TB_HS_BYTES + TB_Q_BYTES;
static_assert(TRI_PIECE == 2 * TB_NT, "a piece's records are read two per thread");

struct TriArgs {
    const SegDev* seg;
    const int64_t* pfx;
    int nseg;
    int64_t rows;
    int big_min;
    const uint32_t* fptr;
    const uint32_t* tptr;
    const uint32_t* nown;
    const uint32_t* fwd;
    const uint4* trec;
    const uint4* items;
    const unsigned* nitems;
    uint32_t item_cap;
    unsigned* cursor;
    const int32_t* rank;
    const int32_t* perm;
    unsigned long long* acc;
    unsigned long long* stat;  // [0] tag-map lookups, [1] their triangles, [2] search lookups, [3] triangles
    uint32_t ntrec;            // records (dyads of the selection)
    int* err;                  // set when a rank lies outside the range its construction gives it
};

struct TbCtl {
    unsigned item;
    int64_t mapped;  // owner whose tag map is in shared memory (-1: none)
    uint32_t mb, mn;  // its forward list
    int32_t mR;
    int ntask, total;
    unsigned long long wsum[TB_W];
};

// Apply the queued hits at the head (cnt of them, one per lane): the third
// vertex's id from the rank permutation, x and t_x(h) from the dyad table.
__device__ __forceinline__ void big_drain(TriHist& H, TriQueue& Q, int cnt, const uint32_t* txin, const int32_t* perm,
                                          int64_t p0, int64_t n, uint32_t hl, unsigned& hits) {
    __syncwarp();
    const int lane = H.lane;
    if (lane < cnt) {
        const uint2 e = Q.q[(Q.head + lane) & (TQN - 1)];
        const uint32_t R = e.x >> 2, th = e.x & 3u;
        const uint32_t xin = txin[e.y >> 2];
        if (R < n) {  // ranks of the graph lie in [0, n)
            const uint32_t w = (uint32_t)perm[p0 + R];
            tri_correct(H.hs, xin >> 2, hl, w, xin & 3u, e.y & 3u, th);
            ++hits;
        }
    }
    __syncwarp();
    Q.head = (Q.head + cnt) & (TQN - 1);
    Q.n -= cnt;
}

// Owners with a tag map: persistent CTAs take work items (pieces of one
// owner's dyad records); consecutive pieces of one owner reuse its map.
__global__ void __launch_bounds__(TB_NT, 2) k_tri_big(TriArgs a) {
    extern __shared__ __align__(16) unsigned char tb_smem[];
    uint32_t* map = reinterpret_cast<uint32_t*>(tb_smem);
    uint32_t* toff = reinterpret_cast<uint32_t*>(tb_smem + TB_MAP_BYTES);
    uint32_t* tfst = reinterpret_cast<uint32_t*>(tb_smem + TB_MAP_BYTES + TB_OFF_BYTES);
    uint32_t* txin = reinterpret_cast<uint32_t*>(tb_smem + TB_MAP_BYTES + TB_OFF_BYTES + TB_FST_BYTES);
    int32_t* hs_all = reinterpret_cast<int32_t*>(tb_smem + TB_MAP_BYTES + TB_OFF_BYTES + TB_FST_BYTES + TB_XIN_BYTES);
    uint2* q_all = reinterpret_cast<uint2*>(tb_smem + TB_MAP_BYTES + TB_OFF_BYTES + TB_FST_BYTES + TB_XIN_BYTES +
                                            TB_HS_BYTES);
    __shared__ TbCtl ctl;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int j = threadIdx.x; j < MAP_KEYS / 16; j += TB_NT) map[j] = 0;
    TriHist H{hs_all + warp * 64, a.acc, -1, lane, 0u};
    for (int j = lane; j < 64; j += 32) H.hs[j] = 0;
    TriQueue Q{q_all + warp * TQN, 0, 0};
    if (threadIdx.x == 0) ctl.mapped = -1;
    unsigned long long looked = 0, tri = 0;
    unsigned hits = 0;
    const unsigned nitems = min(*a.nitems, a.item_cap);
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) ctl.item = atomicAdd(a.cursor, 1u);
        __syncthreads();
        const unsigned it = ctl.item;
        if (it >= nitems) break;
        const uint4 rec = a.items[it];
        const int64_t rh = rec.x;
        const int s = row_seg(a.pfx, a.nseg, rh);
        const int64_t p0 = a.pfx[s], ns = a.seg[s].n;
        const uint32_t hl = (uint32_t)(rh - p0);
        const int32_t Rh = a.rank[rh];
        if (rh != ctl.mapped) {  // clear the previous owner's map entries, then map this owner
            if (ctl.mapped >= 0)
                for (uint32_t i = threadIdx.x; i < ctl.mn; i += TB_NT) {
                    const uint32_t k = (a.fwd[ctl.mb + i] >> 2) - (uint32_t)ctl.mR - 1u;
                    if (k < (uint32_t)MAP_KEYS) map[k >> 4] = 0;
                }
            __syncthreads();
            const uint32_t mb = a.fptr[rh], mn = a.fptr[rh + 1] - mb;
            for (uint32_t i = threadIdx.x; i < mn; i += TB_NT) {
                const uint32_t e = a.fwd[mb + i];
                const uint32_t k = (e >> 2) - (uint32_t)Rh - 1u;
                if (k < (uint32_t)MAP_KEYS) atomicOr(map + (k >> 4), (e & 3u) << (2 * (k & 15u)));
                else atomicOr(a.err, 2);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                ctl.mapped = rh;
                ctl.mb = mb;
                ctl.mn = mn;
                ctl.mR = Rh;
            }
        }
        H.retag(s);
        // the piece's dyads with a non-empty suffix, in record order: first
        // suffix entry, running slot offset, x << 2 | t_x(h)
        const uint32_t t0 = a.tptr[rh] + rec.y * TRI_PIECE;
        const uint32_t t1 = min(a.tptr[rh] + a.nown[rh], t0 + TRI_PIECE);
        uint4 r0 = make_uint4(0, 0, 0, 0), r1 = make_uint4(0, 0, 0, 0);
        const uint32_t i0 = t0 + 2 * threadIdx.x;
        if (i0 < t1) r0 = a.trec[i0];
        if (i0 + 1 < t1) r1 = a.trec[i0 + 1];
        const unsigned long long v = ((unsigned long long)((r0.y > 0) + (r1.y > 0)) << 40) | (r0.y + r1.y);
        unsigned long long incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(full, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) ctl.wsum[warp] = incl;
        __syncthreads();
        unsigned long long ex = incl - v;
        for (int w = 0; w < warp; ++w) ex += ctl.wsum[w];
        {
            int d = (int)(ex >> 40);
            uint32_t off = (uint32_t)(ex & 0xffffffffffull);
            if (r0.y > 0) {
                toff[d] = off;
                tfst[d] = r0.x;
                txin[d] = r0.z;
                ++d;
                off += r0.y;
            }
            if (r1.y > 0) {
                toff[d] = off;
                tfst[d] = r1.x;
                txin[d] = r1.z;
            }
        }
        if (threadIdx.x == TB_NT - 1) {
            ex += v;
            ctl.ntask = (int)(ex >> 40);
            ctl.total = (int)(ex & 0xffffffffffull);
        }
        __syncthreads();
        const int ntask = ctl.ntask, total = ctl.total;
        for (int j = threadIdx.x; j < 32; j += TB_NT) toff[ntask + j] = 0xffffffffu;  // no start past the end
        __syncthreads();
        // this warp's equal share of the concatenated suffixes
        const int lo = (int)((int64_t)total * warp / TB_W), hi = (int)((int64_t)total * (warp + 1) / TB_W);
        if (lo < hi) {
            int before;  // dyads starting below lo
            {
                int l = 0, h = ntask;  // first d with toff[d] >= lo
                while (l < h) {
                    const int mid = (l + h) >> 1;
                    if ((int)toff[mid] < lo) l = mid + 1;
                    else h = mid;
                }
                before = l;
            }
            // slot -> (valid, entry index, dyad) for the chunk at c; advances `before`
            auto locate = [&](int c, bool& ok, uint32_t& fi, int& d) {
                const uint32_t st = before + lane < ntask + 32 ? toff[before + lane] : 0xffffffffu;
                const bool in = st != 0xffffffffu && (int)st < c + 32;
                // dyads starting in [c, c + 32): their start bits
                const unsigned bits = __reduce_or_sync(full, in ? 1u << ((int)st - c) : 0u);
                const int sl = c + lane;
                ok = sl < hi;
                d = before + __popc(bits & (lt | (1u << lane))) - 1;
                before += __popc(bits);
                fi = ok ? tfst[d] + (uint32_t)(sl - (int)toff[d]) : 0u;
            };
            bool ok0;
            uint32_t fi0;
            int d0;
            locate(lo, ok0, fi0, d0);
            uint32_t k0 = ok0 ? __ldg(a.fwd + fi0) : 0u;
            for (int c = lo; c < hi; c += 32) {
                bool ok1 = false;
                uint32_t fi1 = 0, k1 = 0;
                int d1 = 0;
                if (c + 32 < hi) {
                    locate(c + 32, ok1, fi1, d1);
                    k1 = ok1 ? __ldg(a.fwd + fi1) : 0u;
                }
                const uint32_t kk = (k0 >> 2) - (uint32_t)Rh - 1u;  // < MAP_KEYS: the suffix ranks above h
                const uint32_t th = ok0 && kk < (uint32_t)MAP_KEYS ? (map[kk >> 4] >> (2 * (kk & 15u))) & 3u : 0u;
                const bool hit = th != 0;
                const unsigned m = __ballot_sync(full, hit);
                if (hit) Q.q[(Q.head + Q.n + __popc(m & lt)) & (TQN - 1)] =
                    make_uint2(((k0 >> 2) << 2) | th, ((uint32_t)d0 << 2) | (k0 & 3u));
                Q.n += __popc(m);
                if (Q.n >= 32) big_drain(H, Q, 32, txin, a.perm, p0, ns, hl, hits);
                looked += ok0 ? 1 : 0;
                ok0 = ok1;
                fi0 = fi1;
                k0 = k1;
                d0 = d1;
            }
        }
        if (Q.n > 0) big_drain(H, Q, Q.n, txin, a.perm, p0, ns, hl, hits);  // the table changes next
        const unsigned wh = __reduce_add_sync(full, hits);
        H.pending += wh;
        tri += wh;
        hits = 0;
        __syncthreads();
    }
    H.flush();
    looked = warp_sum64(looked);
    if (lane == 0 && looked) atomicAdd(a.stat + 0, looked);
    if (lane == 0 && tri) atomicAdd(a.stat + 1, tri);
}

// Every other owner: warps take runs of TS_RUN dyad records (in owner
// order) and, 32 records at a time, search each suffix entry in its owner's
// forward list.  Records of tag-map owners, of owners without forward
// neighbours and with empty suffixes are skipped.
constexpr int TS_RUN = 1024;

__global__ void __launch_bounds__(256) k_tri_small(TriArgs a) {
    __shared__ int32_t hs_all[8][64];
    __shared__ uint2 q_all[8][TQN];
    __shared__ uint4 cr_all[8][32];   // compacted records
    __shared__ uint2 co_all[8][32];   // their owners' forward lists
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    TriHist H{hs_all[warp], a.acc, -1, lane, 0u};
    for (int j = lane; j < 64; j += 32) H.hs[j] = 0;
    TriQueue Q{q_all[warp], 0, 0};
    __syncwarp();
    unsigned long long looked = 0, tri = 0;
    unsigned hits = 0;
    for (;;) {
        unsigned run = 0;
        if (lane == 0) run = atomicAdd(a.cursor + 1, (unsigned)TS_RUN);
        run = __shfl_sync(full, run, 0);
        if (run >= a.ntrec) break;
        const uint32_t rend = min(a.ntrec, run + TS_RUN);
        for (uint32_t g0 = run; g0 < rend;) {
            const uint32_t t = g0 + lane;
            const bool valid = t < rend;
            const uint4 rec = valid ? a.trec[t] : make_uint4(0, 0, 0, 0);
            const int64_t rh = rec.w;
            int s = valid ? row_seg(a.pfx, a.nseg, rh) : -1;
            const int s0 = __shfl_sync(full, s, 0);
            // a group stays within one graph (records are in owner order)
            const unsigned other = __ballot_sync(full, !valid || s != s0);
            const int take = other ? __ffs(other) - 1 : 32;
            const bool in = lane < take;
            uint32_t hb = 0, hn = 0;
            bool use = false;
            if (in && rec.y > 0) {
                hb = a.fptr[rh];
                hn = a.fptr[rh + 1] - hb;
                use = hn > 0 && !map_owner((int)hn, a.seg[s].n, a.rank[rh], a.big_min);
            }
            const int64_t p0 = a.pfx[s0], ns0 = a.seg[s0].n;
            H.retag(s0);
            // compact the used records into lanes 0 .. ng-1
            const unsigned um = __ballot_sync(full, use);
            const int ng = __popc(um);
            if (use) {
                const int at = __popc(um & lt);
                cr_all[warp][at] = make_uint4(rec.x, rec.y, rec.z, (uint32_t)(rh - p0));
                co_all[warp][at] = make_uint2(hb, hn);
            }
            __syncwarp();
            uint32_t fst = 0, len = 0, xin = 0, ob = 0, on = 0, hl = 0;
            if (lane < ng) {
                const uint4 c = cr_all[warp][lane];
                const uint2 o = co_all[warp][lane];
                fst = c.x;
                len = c.y;
                xin = c.z;
                hl = c.w;
                ob = o.x;
                on = o.y;
            }
            __syncwarp();
            uint32_t off = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(full, off, o);
                if (lane >= o) off += v;
            }
            const uint32_t total = __shfl_sync(full, off, 31);
            off -= len;  // exclusive start of this lane's dyad
            int before = 0;
            for (uint32_t c = 0; c < total; c += 32) {
                const bool st_in = lane < ng && off >= c && off < c + 32;
                const unsigned bits = __reduce_or_sync(full, st_in ? 1u << (off - c) : 0u);
                const int d = before + __popc(bits & (lt | (1u << lane))) - 1;
                before += __popc(bits);
                const uint32_t sl = c + lane;
                const bool ok = sl < total;
                const int dd = ok ? d : 0;
                const uint32_t f_st = __shfl_sync(full, fst, dd), f_off = __shfl_sync(full, off, dd);
                const uint32_t h_b = __shfl_sync(full, ob, dd), h_n = __shfl_sync(full, on, dd);
                uint32_t th = 0, kv = 0;
                if (ok) {
                    kv = __ldg(a.fwd + f_st + (sl - f_off));
                    const uint32_t key = kv & ~3u;  // R << 2
                    uint32_t lo = h_b, n = h_n;
                    while (n > 0) {
                        const uint32_t half = n >> 1;
                        if ((__ldg(a.fwd + lo + half) & ~3u) < key) {
                            lo += half + 1;
                            n -= half + 1;
                        } else {
                            n = half;
                        }
                    }
                    if (lo < h_b + h_n) {
                        const uint32_t e = __ldg(a.fwd + lo);
                        if ((e & ~3u) == key) th = e & 3u;
                    }
                    ++looked;
                }
                const bool hit = th != 0;
                const unsigned m = __ballot_sync(full, hit);
                if (hit) Q.q[(Q.head + Q.n + __popc(m & lt)) & (TQN - 1)] =
                    make_uint2((kv & ~3u) | th, ((uint32_t)d << 2) | (kv & 3u));
                Q.n += __popc(m);
                while (Q.n >= 32 || (Q.n > 0 && c + 32 >= total)) {  // drain (all before the group changes)
                    const int cnt = min(Q.n, 32);
                    __syncwarp();
                    const uint2 e = Q.q[(Q.head + (lane < cnt ? lane : 0)) & (TQN - 1)];
                    const int dq = lane < cnt ? (int)(e.y >> 2) : 0;
                    const uint32_t qx = __shfl_sync(full, xin, dq), qh = __shfl_sync(full, hl, dq);
                    if (lane < cnt && (e.x >> 2) < ns0) {  // ranks of the graph lie in [0, n)
                        const uint32_t w = (uint32_t)a.perm[p0 + (e.x >> 2)];
                        tri_correct(H.hs, qx >> 2, qh, w, qx & 3u, e.y & 3u, e.x & 3u);
                        ++hits;
                    }
                    __syncwarp();
                    Q.head = (Q.head + cnt) & (TQN - 1);
                    Q.n -= cnt;
                }
            }
            const unsigned wh = __reduce_add_sync(full, hits);
            H.pending += wh;
            tri += wh;
            hits = 0;
            g0 += (uint32_t)take;
        }
    }
    H.flush();
    looked = warp_sum64(looked);
    if (lane == 0 && looked) atomicAdd(a.stat + 2, looked);
    if (lane == 0 && tri) atomicAdd(a.stat + 3, tri);
}
