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
// of higher rank, as R << 2 | tag seen from x, in rank order.  A triangle
// x, h, w with R(x) < R(h) < R(w) is found exactly once: at the dyad {x, h},
// owned by h, as an element w of F(x) ranked above h (the suffix after h of
// a list of more than FWD_SHORT entries, the whole of a shorter one) that
// also lies in F(h).  Because high-degree vertices rank last, every F(h) is
// short (at most a few hundred entries on the power-law workloads), and the
// suffixes sum to about half the lookups of an id-ordered search (R-MAT
// scale 22: 5.3e8 instead of 1.1e9 for the hub dyads alone).
//
// Two lookup forms:
//  * k_tri_big: an owner with many forward neighbours and few vertices
//    ranked above it gets a CTA: a 2-bit tag map over the ranks above R(h)
//    in shared memory (0 = not in F(h), else the tag t_h(w)) answers every
//    lookup exactly with one shared load.  The owner's dyads, one piece of
//    at most TRI_PIECE at a time, are laid out as concatenated suffixes that
//    the warps split evenly.
//  * k_tri_small: every other owner: warps take runs of dyad records; a
//    lookup binary-searches F(h) (global memory, cached: a run's dyads
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
// class c before the graph's first row), and clsb[s][c] = the ranks before
// class c in the graph (its first rank).  One warp per graph.
__global__ void k_rank_seg(const int32_t* __restrict__ deg, const SegDev* __restrict__ seg,
                           const int64_t* __restrict__ pfx, int nseg, int64_t rows, int nb,
                           const uint32_t* __restrict__ hex, int64_t* __restrict__ co,
                           int32_t* __restrict__ clsb) {
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
        clsb[(size_t)s * NCLS + lane] = (int32_t)ex;
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
// its neighbour ranks above its row: flag[f] = 1.  The task pass writes the
// flags as it reads each entry (k_tasks_flat); k_fwd_flags does the same for
// the row-per-warp task pass.
__global__ void k_fwd_flags(const uint32_t* __restrict__ adj, const int32_t* __restrict__ arow,
                            const SegDev* __restrict__ seg, const int64_t* __restrict__ pfx,
                            const int64_t* __restrict__ epfx, int nseg, int64_t entries,
                            const int32_t* __restrict__ rank, uint8_t* __restrict__ flag) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < entries;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int s = nseg == 1 ? 0 : seg_of(epfx, nseg, f);
        const SegDev& g = seg[s];
        const int64_t k = g.eb + (f - epfx[s]);
        const int64_t p = pfx[s];
        flag[f] = rank[p + (__ldg(adj + k) >> 2)] > rank[p + ((int64_t)arow[k] - g.rb)] ? 1 : 0;
    }
}

// ------------------------------------------------------ row-wise terms --
// The forward path's task pass, row by row instead of entry by entry (no
// global scan of tag words).  In row x (sorted by neighbour id) every pair of
// entries i < j counts once: when y_i lies above x (the dyad <x, y_i>) as code
// t_i + 4 t_j (an entry of row u after v), when y_i lies below x (the dyad
// <y_i, x>) as code swap(t_i) + 16 t_j (an entry of row v after u).  And each
// entry adds, to the dyadic sum of its dyad's pre value (t_i above x,
// swap(t_i) below), n when it lies above x and -d_x always: summed over both
// entries of a dyad <u, v> that is n - d_u - d_v.  (The same terms k_tasks
// adds per canonical dyad, Sec. 2.2 regrouped.)  Each entry also gets its
// forward flag.  Rows of at most TR_SHORT entries are done by one thread;
// longer rows are cut into pieces of TR_PIECE entries, one warp each
// (k_terms_pieces), the counts of later pieces of the same row carried in
// (k_piece_counts).
constexpr int TR_SHORT = 32;
constexpr int TR_PIECE = 2048;
constexpr int TR_ILP = 4;  // chunks of 32 entries a piece's warp has in flight
constexpr int TR_RUN = 1;  // 32-row groups a warp takes at a time (more per take measured slower)

// Per-thread term sums for one graph: the pair counts A[p][q], B[p][q]
// (p, q = tag - 1) in 32-bit counters in shared memory, [18][32] per warp
// (word (pair * 32 + lane): no bank conflicts), flushed before they could
// wrap; the dyadic sums D[p] in registers.  flush() adds the warp's sums to
// the graph's accumulators.
struct TermSums {
    uint32_t* sm;  // this warp's [18][32] counters
    int lane;
    unsigned long long D[3];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < 18; ++i) sm[i * 32 + lane] = 0;
        D[0] = D[1] = D[2] = 0;
    }
    // one entry of tag t (1..3) with c[q] entries of tag q + 1 after it in its row
    __device__ __forceinline__ void add(bool on, bool up, uint32_t t, const uint32_t c[3], unsigned long long dy) {
        const uint32_t pa = up ? t : tag_swap(t);  // the dyad's pre value
        if (on) {
            uint32_t* b = sm + ((up ? 0u : 9u) + 3u * (pa - 1u)) * 32u + lane;
            b[0] += c[0];
            b[32] += c[1];
            b[64] += c[2];
        }
#pragma unroll
        for (int p = 0; p < 3; ++p) D[p] += (on && pa == (uint32_t)(p + 1)) ? dy : 0ull;
    }
    // warp sums into graph s's accumulators (lane 0 adds)
    __device__ __forceinline__ void flush(unsigned long long* acc, int s) {
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 18; ++i) {
            const unsigned long long v = warp_sum64(sm[i * 32 + lane]);
            const int p = (i % 9) / 3, q = i % 3;
            if (lane == 0 && s >= 0 && v)
                atomicAdd(acc + (size_t)s * ACC + (p + 1) + (i < 9 ? 4 : 16) * (q + 1), v);
        }
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const unsigned long long dd = warp_sum64(D[p]);
            if (lane == 0 && s >= 0 && dd) atomicAdd(acc + (size_t)s * ACC + 64 + p, dd);
        }
        __syncwarp();
        zero();
        __syncwarp();
    }
    // one lane's sums straight into graph s's accumulators
    __device__ __forceinline__ void add_direct(unsigned long long* acc, int s) {
#pragma unroll
        for (int i = 0; i < 18; ++i) {
            const uint32_t v = sm[i * 32 + lane];
            const int p = (i % 9) / 3, q = i % 3;
            if (v) atomicAdd(acc + (size_t)s * ACC + (p + 1) + (i < 9 ? 4 : 16) * (q + 1), (unsigned long long)v);
            sm[i * 32 + lane] = 0;
        }
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            if (D[p]) atomicAdd(acc + (size_t)s * ACC + 64 + p, D[p]);
            D[p] = 0;
        }
    }
};

struct TermArgs {
    const int64_t* row_ptr;
    const uint32_t* adj;
    const SegDev* seg;
    const int64_t* pfx;
    const int64_t* epfx;
    int nseg;
    int64_t rows;
    int64_t r_lo, r_hi;   // the rows whose terms this call adds (a shard), all flags regardless
    const int32_t* rank;  // per selected row
    const int32_t* perm;  // rank -> local row, per graph
    uint8_t* flag;        // [entries] forward flags
    unsigned long long* acc;
    uint4* pieces;        // [3 * piece_cap] piece records of the longer rows (Piece)
    unsigned* npieces;
    uint32_t piece_cap;
    uint4* pcnt;          // [piece_cap] tag counts of the pieces of rows of several pieces
};

// A piece of a longer row, everything its warp needs: the row's first
// adjacency entry and first selection entry, the graph's first selected
// row, the row's length and rank, the row, the piece and the row's pieces,
// the graph.
struct Piece {
    int64_t beg, f0, p0;
    int32_t d, R;
    uint32_t r, k, np;
    int32_t s;
};

__device__ __forceinline__ void put_piece(uint4* q, const Piece& P) {
    q[0] = make_uint4((uint32_t)P.beg, (uint32_t)((uint64_t)P.beg >> 32), (uint32_t)P.f0,
                      (uint32_t)((uint64_t)P.f0 >> 32));
    q[1] = make_uint4((uint32_t)P.p0, (uint32_t)((uint64_t)P.p0 >> 32), (uint32_t)P.d, (uint32_t)P.R);
    q[2] = make_uint4(P.r, P.k, P.np, (uint32_t)P.s);
}

__device__ __forceinline__ Piece get_piece(const uint4& a, const uint4& b, const uint4& c) {
    Piece P;
    P.beg = (int64_t)(((uint64_t)a.y << 32) | a.x);
    P.f0 = (int64_t)(((uint64_t)a.w << 32) | a.z);
    P.p0 = (int64_t)(((uint64_t)b.y << 32) | b.x);
    P.d = (int32_t)b.z;
    P.R = (int32_t)b.w;
    P.r = c.x;
    P.k = c.y;
    P.np = c.z;
    P.s = (int32_t)c.w;
    return P;
}

// One thread per row of at most TR_SHORT entries, the rows taken in rank
// order (a warp takes TR_RUN groups of 32 consecutive ranks at a time: rows
// of one degree class, so the lanes' rows are about as long), in batches of 16
// entries from the row's end up to the longest row of the group, each
// batch's loads issued before its entries are counted; longer rows are
// listed as pieces.
__global__ void __launch_bounds__(256, 3) k_terms_rows(TermArgs a) {
    __shared__ uint32_t tsm[8][18 * 32];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    TermSums T;
    T.sm = tsm[threadIdx.x >> 5];
    T.lane = lane;
    T.zero();
    int cur = -1;  // the graph of the warp's sums
    unsigned groups = 0;  // 32-row groups since the last flush (a lane adds < 2^10 per group)
    for (int64_t g0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32 * TR_RUN; g0 < a.rows;
         g0 += warps * 32 * TR_RUN) {
        for (int it = 0; it < TR_RUN; ++it) {
            const int64_t i = g0 + 32 * it + lane;  // rank position: graph s's ranks start at pfx[s]
            const bool valid = i < a.rows;
            const int s = valid ? row_seg(a.pfx, a.nseg, i) : -1;
            const int s0 = __shfl_sync(full, s, 0);
            if (s0 < 0) break;
            // rows of two graphs in one group: each lane adds its own row's
            // terms to its graph directly (after the warp's sums are flushed)
            const bool mixed = __any_sync(full, valid && s != s0);
            if (s0 != cur || mixed || ++groups >= (1u << 20)) {
                T.flush(a.acc, cur);
                cur = s0;
                groups = 0;
            }
            unsigned np = 0;
            Piece P;
            int64_t p0 = 0, xl = 0, r = 0, beg = 0, f0 = 0;
            int d = 0;
            int32_t R = 0;
            if (valid) {
                const SegDev& g = a.seg[s];
                p0 = a.pfx[s];
                xl = a.perm[i];
                r = p0 + xl;
                const int64_t x = g.rb + xl;
                beg = a.row_ptr[x];
                d = (int)(a.row_ptr[x + 1] - beg);
                R = (int32_t)(i - p0);
                f0 = a.epfx[s] + (beg - g.eb);
                if (d > TR_SHORT) {
                    np = (unsigned)((d + TR_PIECE - 1) / TR_PIECE);
                    P.beg = beg;
                    P.f0 = f0;
                    P.p0 = p0;
                    P.d = d;
                    P.R = R;
                    P.r = (uint32_t)r;
                    P.np = np;
                    P.s = s;
                }
            }
            // the group's short rows, up to its longest one (warp-uniform bounds)
            const int ds = (valid && d <= TR_SHORT) ? d : 0;
            const int dm = __reduce_max_sync(full, ds);
            if (dm > 0) {
                const bool terms = valid && r >= a.r_lo && r < a.r_hi;
                const unsigned long long n = valid ? (unsigned long long)a.seg[s].n : 0ull;
                const unsigned long long dx = (unsigned long long)ds;
                uint32_t c[3] = {0, 0, 0};
                for (int kb = dm > 16 ? 16 : 0; kb >= 0; kb -= 16) {
                    const int nb = min(dm - kb, 16);
                    uint32_t e[16];
                    int32_t rk[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) e[k] = (k < nb && kb + k < ds) ? __ldg(a.adj + beg + kb + k) : 0u;
#pragma unroll
                    for (int k = 0; k < 16; ++k) rk[k] = e[k] ? a.rank[p0 + (e[k] >> 2)] : 0;
#pragma unroll
                    for (int k = 15; k >= 0; --k) {
                        if (k < nb && e[k]) {
                            const uint32_t y = e[k] >> 2, t = e[k] & 3u;
                            a.flag[f0 + kb + k] = rk[k] > R ? 1 : 0;
                            const bool up = (int64_t)y > xl;
                            T.add(terms, up, t, c, (up ? n : 0ull) - dx);
                            c[0] += t == 1u;
                            c[1] += t == 2u;
                            c[2] += t == 3u;
                        }
                    }
                }
            }
            if (mixed && valid) T.add_direct(a.acc, s);
            // the pieces of the longer rows: one atomic per warp
            unsigned incl = np;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_up_sync(full, incl, o);
                if (lane >= o) incl += v;
            }
            const unsigned tot = __shfl_sync(full, incl, 31);
            unsigned at = 0;
            if (lane == 31 && tot) at = atomicAdd(a.npieces, tot);
            at = __shfl_sync(full, at, 31) + incl - np;
            for (unsigned q = 0; q < np; ++q)
                if (at + q < a.piece_cap) {
                    P.k = q;
                    put_piece(a.pieces + 3 * (size_t)(at + q), P);
                }
        }
    }
    T.flush(a.acc, cur);
}

// Tag counts of every piece of a row of several pieces (one warp per piece).
__global__ void __launch_bounds__(256) k_piece_counts(TermArgs a) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const uint32_t np_all = min(*a.npieces, a.piece_cap);
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < np_all; w += warps) {
        const uint4 q2 = a.pieces[3 * w + 2];
        if (q2.z < 2) continue;
        const Piece P = get_piece(a.pieces[3 * w], a.pieces[3 * w + 1], q2);
        const int k0 = (int)P.k * TR_PIECE, k1 = min(P.d, k0 + TR_PIECE);
        uint32_t c1 = 0, c2 = 0, c3 = 0;
        for (int k = k0 + lane; k < k1; k += 32) {
            const uint32_t t = __ldg(a.adj + P.beg + k) & 3u;
            c1 += t == 1u;
            c2 += t == 2u;
            c3 += t == 3u;
        }
        c1 = __reduce_add_sync(full, c1);
        c2 = __reduce_add_sync(full, c2);
        c3 = __reduce_add_sync(full, c3);
        if (lane == 0) a.pcnt[w] = make_uint4(c1, c2, c3, 0u);
    }
}

// One warp per piece of a longer row: TR_ILP chunks of 32 entries at a time
// from the piece's end, the counts after each entry from ballots plus those
// carried from the later entries (and the later pieces of the row).  The
// next piece's record loads while this one runs.
__global__ void __launch_bounds__(256, 3) k_terms_pieces(TermArgs a) {
    __shared__ uint32_t tsm[8][18 * 32];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned after = ~((2u << lane) - 1u);  // lanes above this one
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const uint32_t np_all = min(*a.npieces, a.piece_cap);
    TermSums T;
    T.sm = tsm[threadIdx.x >> 5];
    T.lane = lane;
    T.zero();
    int cur = -1;
    unsigned since = 0;  // pieces since the last flush (a lane adds < 64 * 2^21 per piece)
    int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    uint4 n0 = make_uint4(0, 0, 0, 0), n1 = n0, n2 = n0;
    if (w < np_all) {
        n0 = a.pieces[3 * w];
        n1 = a.pieces[3 * w + 1];
        n2 = a.pieces[3 * w + 2];
    }
    for (; w < np_all; w += warps) {
        const Piece P = get_piece(n0, n1, n2);
        if (w + warps < np_all) {
            n0 = a.pieces[3 * (w + warps)];
            n1 = a.pieces[3 * (w + warps) + 1];
            n2 = a.pieces[3 * (w + warps) + 2];
        }
        if (P.s != cur || ++since >= 16) {
            T.flush(a.acc, cur);
            cur = P.s;
            since = 0;
        }
        const int64_t xl = (int64_t)P.r - P.p0;
        const int k0 = (int)P.k * TR_PIECE, k1 = min(P.d, k0 + TR_PIECE);
        const bool terms = (int64_t)P.r >= a.r_lo && (int64_t)P.r < a.r_hi;
        const unsigned long long n = (unsigned long long)a.seg[P.s].n, dx = (unsigned long long)P.d;
        uint32_t cc[3] = {0, 0, 0};  // entries of each tag after the current chunk
        for (uint32_t q = P.k + 1; q < P.np; ++q) {  // the row's later pieces
            const uint4 c = a.pcnt[w - P.k + q];
            cc[0] += c.x;
            cc[1] += c.y;
            cc[2] += c.z;
        }
        // TR_ILP chunks at a time from the piece's end: loads first, then the
        // chunks in order from the last
        for (int top = k0 + ((k1 - k0 - 1) & ~31); top >= k0; top -= 32 * TR_ILP) {
            uint32_t e[TR_ILP];
            int32_t rk[TR_ILP];
#pragma unroll
            for (int u = 0; u < TR_ILP; ++u) {
                const int k = top - 32 * u + lane;
                e[u] = (k >= k0 && k < k1) ? __ldg(a.adj + P.beg + k) : 0u;
            }
#pragma unroll
            for (int u = 0; u < TR_ILP; ++u) rk[u] = e[u] ? a.rank[P.p0 + (e[u] >> 2)] : 0;
#pragma unroll
            for (int u = 0; u < TR_ILP; ++u) {
                const int k = top - 32 * u + lane;
                const bool valid = e[u] != 0u;
                const uint32_t y = e[u] >> 2, t = e[u] & 3u;
                if (valid) a.flag[P.f0 + k] = rk[u] > P.R ? 1 : 0;
                const unsigned m1 = __ballot_sync(full, t == 1u), m2 = __ballot_sync(full, t == 2u),
                               m3 = __ballot_sync(full, t == 3u);
                const uint32_t c[3] = {cc[0] + __popc(m1 & after), cc[1] + __popc(m2 & after),
                                       cc[2] + __popc(m3 & after)};
                const bool up = (int64_t)y > xl;
                T.add(terms && valid, up, t, c, (up ? n : 0ull) - dx);
                cc[0] += __popc(m1);
                cc[1] += __popc(m2);
                cc[2] += __popc(m3);
            }
        }
    }
    T.flush(a.acc, cur);
}

// Rows whose forward list has at most FWD_SHORT entries are sorted in
// registers (k_fwd_sort_short) and a dyad of such a row looks up its whole
// forward list instead of the part ranked above the owner (an entry ranked
// below the owner cannot lie in the owner's forward list, so the result is
// the same, and no search for the suffix is needed); R-MAT scale 22: +3%
// lookups, 15x fewer rows for the warp-per-row sort.
constexpr int FWD_SHORT = 16;
constexpr int TRI_PIECE = 512;     // dyad records per tag-map work item
constexpr int MAP_KEYS = 1 << 17;  // ranks a tag map covers (2 bits each: 32 KB)
constexpr int MLIST = 1024;        // longest forward list of a tag-map owner

// Dyad records (one per dyad whose owner has a forward list), in two parts:
// first the tag-map owners' records, grouped by owner (their work items
// refer to these ranges), then the other owners', grouped by owner.  A
// record is {first entry of the lookup list, its length, x << 2 | t_x(h),
// owner row h}.
struct FwdLayout {
    const int32_t* fs;         // [entries] inclusive count of forward entries
    uint32_t* fptr;            // [rows + 1] forward list start
    uint8_t* kind;             // [rows] owner kind: 0 no records, 1 tag map, 2 search
    unsigned long long* tcnt;  // [rows + 1] records per owner: map << 32 | search
    unsigned long long* tpre;  // [rows + 1] exclusive scan of tcnt
    uint32_t* fid;             // [dyads] forward entries in id order (adjacency words)
    uint32_t* fwd;             // [dyads] forward entries: R << 2 | tag, rank order in long rows
    uint4* trec;               // [dyads] dyad records
    uint4* items;              // tag-map work items, two words each (see k_fwd_items)
    uint32_t item_cap;
    uint32_t* longs;           // rows whose forward list is sorted (more than FWD_SHORT entries)
    unsigned* nitems;          // [1]
    unsigned* nlong;           // [1]
    unsigned* cursor;          // [2] work cursors (tag-map items, search records)
    unsigned long long* stat;  // [5] lookups and triangles of each lookup form, staged list entries
    const int32_t* rank;
    const int32_t* perm;
    const int32_t* clsb;       // [graphs][NCLS] first rank of each degree class
};

// Tag-map owners: a forward list of at least big_min entries, or of at
// least big_min / MID_DIV entries when the owner also owns at least OWN_MID
// dyads (its list is then probed often enough to pay for the map; measured
// on B300 against thresholds of 2-8 and 16-256: R-MAT scale 22 census 3.245
// -> 3.213 ms, Chung-Lu 2^22 5.450 -> 5.343 ms); and a list and a rank
// range the map holds.
constexpr int MID_DIV = 8;
constexpr uint32_t OWN_MID = 128;
__device__ __forceinline__ bool map_owner(int nplus, int64_t n, int32_t R, int big_min, uint32_t own) {
    const bool wide = nplus >= big_min || (nplus >= big_min / MID_DIV && own >= OWN_MID);
    return wide && nplus > 0 && nplus <= MLIST && n - (int64_t)R - 1 <= MAP_KEYS;
}

// Per row: its forward list (start from the flag scan), the dyads it owns
// (lower-ranked neighbours) and which lookup form they take, its tag-map
// work items, and whether its forward list is sorted.  The two lists are
// appended with one atomic per block and list.
constexpr int FR_NT = 256;

__global__ void __launch_bounds__(FR_NT) k_fwd_rows(const int64_t* __restrict__ row_ptr,
                                                    const int32_t* __restrict__ deg, const SegDev* __restrict__ seg,
                                                    const int64_t* __restrict__ pfx, const int64_t* __restrict__ epfx,
                                                    int nseg, int64_t rows, int big_min, FwdLayout F,
                                                    int64_t r_lo, int64_t r_hi) {
    __shared__ unsigned wsum[2][FR_NT / 32];
    __shared__ unsigned base[2];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t b0 = (int64_t)blockIdx.x * FR_NT; b0 < rows; b0 += (int64_t)gridDim.x * FR_NT) {
        const int64_t r = b0 + threadIdx.x;
        unsigned np = 0, lng = 0;
        if (r < rows) {
            const int s = row_seg(pfx, nseg, r);
            const SegDev& g = seg[s];
            const int64_t x = g.rb + (r - pfx[s]);
            const int64_t f0 = epfx[s] + (row_ptr[x] - g.eb), f1 = epfx[s] + (row_ptr[x + 1] - g.eb);
            const uint32_t a = f0 > 0 ? (uint32_t)F.fs[f0 - 1] : 0u, b = f1 > 0 ? (uint32_t)F.fs[f1 - 1] : 0u;
            // dyads owned by r: its neighbours ranked below it (none when the
            // row belongs to another shard)
            const uint32_t m = b - a, own = r >= r_lo && r < r_hi ? (uint32_t)deg[x] - m : 0u;
            F.fptr[r] = a;
            if (r == rows - 1) {
                F.fptr[rows] = b;
                F.tcnt[rows] = 0;
            }
            const bool big = own > 0 && map_owner((int)m, g.n, F.rank[r], big_min, own);
            const bool search = !big && own > 0 && m > 0;
            F.kind[r] = big ? 1 : search ? 2 : 0;
            F.tcnt[r] = big ? (unsigned long long)own << 32 : search ? (unsigned long long)own : 0ull;
            if (big) np = (own + TRI_PIECE - 1) / TRI_PIECE;
            lng = m > FWD_SHORT ? 1u : 0u;
        }
        // block-wide exclusive offsets of the work items and the long rows
        unsigned ip = np, lp = lng;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t1 = __shfl_up_sync(full, ip, o), t2 = __shfl_up_sync(full, lp, o);
            if (lane >= o) {
                ip += t1;
                lp += t2;
            }
        }
        if (lane == 31) {
            wsum[0][warp] = ip;
            wsum[1][warp] = lp;
        }
        __syncthreads();
        if (threadIdx.x < 2) {
            unsigned tot = 0;
            for (int w = 0; w < FR_NT / 32; ++w) {
                const unsigned t = wsum[threadIdx.x][w];
                wsum[threadIdx.x][w] = tot;
                tot += t;
            }
            base[threadIdx.x] = tot ? atomicAdd(threadIdx.x == 0 ? F.nitems : F.nlong, tot) : 0u;
        }
        __syncthreads();
        const unsigned at = base[0] + wsum[0][warp] + ip - np;
        for (unsigned p = 0; p < np; ++p)
            if (at + p < F.item_cap) F.items[2 * (at + p)] = make_uint4((uint32_t)r, p, 0u, 0u);
        if (lng) F.longs[base[1] + wsum[1][warp] + lp - 1] = (uint32_t)r;
        __syncthreads();
    }
}

// Forward entries, one thread per entry of the selection: in a short row
// the entry R << 2 | tag (in id order until k_fwd_sort_short), in a long row
// the adjacency word for k_fwd_sort.
__global__ void k_fwd_fill(const uint32_t* __restrict__ adj, const int32_t* __restrict__ arow,
                           const SegDev* __restrict__ seg, const int64_t* __restrict__ pfx,
                           const int64_t* __restrict__ epfx, int nseg, int64_t entries, FwdLayout F) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < entries;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int32_t here = F.fs[f];
        if (here == (f > 0 ? F.fs[f - 1] : 0)) continue;
        const int s = nseg == 1 ? 0 : seg_of(epfx, nseg, f);
        const SegDev& g = seg[s];
        const int64_t k = g.eb + (f - epfx[s]);
        const uint32_t e = __ldg(adj + k);
        const uint32_t p = (uint32_t)here - 1u;
        const int64_t p0 = pfx[s], rx = p0 + ((int64_t)arow[k] - g.rb);
        if (F.fptr[rx + 1] - F.fptr[rx] > FWD_SHORT) F.fid[p] = e;
        else F.fwd[p] = ((uint32_t)F.rank[p0 + (e >> 2)] << 2) | (e & 3u);
    }
}

// One thread per short row (2 .. FWD_SHORT entries): its entries sorted by
// rank in registers (a bitonic network over 16 words, unused ones padded
// with the largest word), so that every forward list is in rank order.
__global__ void k_fwd_sort_short(int64_t rows, FwdLayout F) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b0 = F.fptr[r], m = F.fptr[r + 1] - b0;
        if (m < 2 || m > FWD_SHORT) continue;
        uint32_t e[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) e[i] = i < (int)m ? F.fwd[b0 + i] : 0xffffffffu;
#pragma unroll
        for (int k = 2; k <= 16; k <<= 1)
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int l = i ^ j;
                    if (l > i) {
                        const uint32_t a = e[i], b = e[l];
                        const bool sw = ((i & k) == 0) ? a > b : a < b;
                        e[i] = sw ? b : a;
                        e[l] = sw ? a : b;
                    }
                }
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (i < (int)m) F.fwd[b0 + i] = e[i];
    }
}
static_assert(FWD_SHORT <= 16, "short rows are sorted in a 16-word network");

// One warp per long row: a stable partition of the forward list (in id
// order) by degree class gives rank order.  The first pass looks up each
// entry's rank, writes R << 2 | tag over the id-order word and counts the
// classes; the second reads those words back and places them.  An entry's
// class comes from its rank (the last class whose first rank is at most R,
// searched in the graph's NCLS class starts), so each entry costs one random
// load.
__global__ void __launch_bounds__(256) k_fwd_sort(const int32_t* __restrict__ deg, const SegDev* __restrict__ seg,
                                                  const int64_t* __restrict__ pfx, int nseg, FwdLayout F) {
    __shared__ unsigned cnt_all[8][NCLS + 1];
    __shared__ int32_t cb_all[8][NCLS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned* cnt = cnt_all[warp];
    int32_t* cb = cb_all[warp];
    const unsigned full = 0xffffffffu, lt = (1u << lane) - 1u;
    const unsigned nlong = *F.nlong;
    auto cls_of = [&](uint32_t R) {  // cb[0] = 0 <= R
        int c = 0;
#pragma unroll
        for (int st = NCLS / 2; st > 0; st >>= 1)
            if ((uint32_t)cb[c + st] <= R) c += st;
        return c;
    };
    for (unsigned li = blockIdx.x * 8 + warp; li < nlong; li += gridDim.x * 8) {
        const int64_t r = F.longs[li];
        const uint32_t b0 = F.fptr[r], m = F.fptr[r + 1] - b0;
        const int s = row_seg(pfx, nseg, r);
        const int64_t p0 = pfx[s];
        cnt[lane] = 0;
        cb[lane] = F.clsb[(size_t)s * NCLS + lane];
        __syncwarp();
        for (uint32_t i0 = 0; i0 < m; i0 += 32) {
            const uint32_t i = i0 + lane;
            int c = NCLS;
            if (i < m) {
                const uint32_t e = F.fid[b0 + i];
                const uint32_t R = (uint32_t)F.rank[p0 + (e >> 2)];
                F.fid[b0 + i] = (R << 2) | (e & 3u);
                c = cls_of(R);
            }
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
            const uint32_t w = i < m ? F.fid[b0 + i] : 0u;
            const int c = i < m ? cls_of(w >> 2) : NCLS;
            const unsigned same = __match_any_sync(full, c);
            const uint32_t pos = c < NCLS ? cnt[c] + __popc(same & lt) : 0u;
            __syncwarp();
            if (c < NCLS && (same & lt) == 0) cnt[c] += __popc(same);
            __syncwarp();
            if (i < m) F.fwd[b0 + pos] = w;
        }
        __syncwarp();  // cb and cnt are rewritten for the next row
    }
}

// Dyad records, written from the owner's side with no atomics: entry f of
// row y whose neighbour x ranks below y is the dyad {x, y} owned by y, and
// its index among row y's such entries (the entries before it minus the
// forward ones, from the flag scan) is its slot in y's records.  Its lookup
// list is x's whole forward list when that is short, else the part of it
// ranked above y (found by binary search of the sorted list).
__global__ void k_fwd_recs(const int64_t* __restrict__ row_ptr, const uint32_t* __restrict__ adj,
                           const int32_t* __restrict__ arow, const SegDev* __restrict__ seg,
                           const int64_t* __restrict__ pfx, const int64_t* __restrict__ epfx, int nseg,
                           int64_t entries, int64_t rows, FwdLayout F) {
    const unsigned long long tot = F.tpre[rows];
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < entries;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int32_t here = F.fs[f];
        if (here != (f > 0 ? F.fs[f - 1] : 0)) continue;  // forward: not owned by this row
        const int s = nseg == 1 ? 0 : seg_of(epfx, nseg, f);
        const SegDev& g = seg[s];
        const int64_t k = g.eb + (f - epfx[s]);
        const int64_t p0 = pfx[s], y = arow[k], ry = p0 + (y - g.rb);
        const uint8_t kd = F.kind[ry];
        if (kd == 0) continue;
        const int64_t f0 = epfx[s] + (row_ptr[y] - g.eb);  // the row's first entry
        const uint32_t fwd_before = (uint32_t)here - (f0 > 0 ? (uint32_t)F.fs[f0 - 1] : 0u);
        const uint32_t j = (uint32_t)(f - f0) - fwd_before;
        const unsigned long long pre = F.tpre[ry];
        const uint32_t slot = (kd == 1 ? (uint32_t)(pre >> 32) : (uint32_t)(tot >> 32) + (uint32_t)pre) + j;
        const uint32_t e = __ldg(adj + k);
        const int64_t rx = p0 + (e >> 2);
        uint32_t a = F.fptr[rx], m = F.fptr[rx + 1] - a;
        if (m > FWD_SHORT) {  // the part of the sorted list ranked above y
            const uint32_t key = (uint32_t)F.rank[ry] << 2;
            uint32_t lo = a, n = m;
            while (n > 0) {
                const uint32_t half = n >> 1;
                if ((F.fwd[lo + half] & ~3u) <= key) {
                    lo += half + 1;
                    n -= half + 1;
                } else {
                    n = half;
                }
            }
            m -= lo - a;
            a = lo;
        }
        F.trec[slot] = make_uint4(a, m, ((e >> 2) << 2) | tag_swap(e & 3u), (uint32_t)ry);
    }
}

// ------------------------------------------------------------ triangles --
// A triangle's correction depends only on its three tags in the id order of
// its vertices a < b < c: t_ab, t_ac, t_bc in {1, 2, 3} (27 triangle
// types).  Dyad <a,b> moves one count from codes t_ab + 4 t_ac and
// t_ab + 16 t_bc to t_ab + 4 t_ac + 16 t_bc, and dyad <a,c> drops the count
// t_ac + 16 t_cb it added for b.  The lookups count triangles per type; the
// four code updates per type are applied when the counts are flushed.
//
// Seen by type rather than by code, the correction is symmetric in the three
// vertices: the suffix terms counted the triad once as each of the three
// two-edge triads (edges ab, ac; ab, bc; ac, cb: one per vertex as the
// centre), and it is one full triangle.  So for the 16-type census any order
// of a, b, c gives the same counts after the fold, and the lookups take them
// in rank order (x, h, w: no id needed, tags straight from the lookup); the
// 64-code census (and a shard, whose accumulators may be folded to codes)
// needs the id order, which costs a gather of w's id per triangle.
__device__ __forceinline__ int tri_type(uint32_t a, uint32_t b, uint32_t c, uint32_t t_ab, uint32_t t_ac,
                                        uint32_t t_bc) {
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
        t_ab = tag_swap(t_ab);
        t = t_ac; t_ac = t_bc; t_bc = t;
    }
    return (int)(9 * (t_ab - 1) + 3 * (t_ac - 1) + (t_bc - 1));
}

// Per-warp triangle counts by type for one graph; the code updates go into
// the graph's 64-bit accumulators when the graph changes, at the end, and
// before a count could wrap.
struct TriHist {
    uint32_t* hs;  // [2][32]: types 0..26, one copy per lane parity
    unsigned long long* acc;
    int tag;
    int lane;
    unsigned pending;
    unsigned long long seen;  // triangles flushed by this lane's counter
    __device__ __forceinline__ void flush() {
        if (tag >= 0 && lane < 27) {
            const unsigned long long c = (unsigned long long)hs[lane] + hs[32 + lane];
            seen += c;
            if (c) {
                unsigned long long* h = acc + (size_t)tag * ACC;
                const uint32_t t_ab = lane / 9 + 1, t_ac = (lane / 3) % 3 + 1, t_bc = lane % 3 + 1;
                atomicAdd(h + t_ab + 4 * t_ac, 0ull - c);
                atomicAdd(h + t_ab + 16 * t_bc, 0ull - c);
                atomicAdd(h + t_ab + 4 * t_ac + 16 * t_bc, c);
                atomicAdd(h + t_ac + 16 * tag_swap(t_bc), 0ull - c);
            }
        }
        hs[lane] = 0;
        hs[32 + lane] = 0;
        __syncwarp();
        pending = 0;
    }
    __device__ __forceinline__ void retag(int s) {
        if (s != tag || pending > (1u << 30)) {
            flush();
            tag = s;
        }
    }
    // one triangle per active lane (shared-memory atomics; the two copies
    // halve the lanes that meet on one counter)
    __device__ __forceinline__ void add(bool active, int type) {
        if (active) atomicAdd(hs + ((lane & 1) << 5) + type, 1u);
    }
    // the same at base = hs + ((lane & 1) << 5) - 13, type + 13 given: a
    // predicated shared-memory reduction (no branch around it)
    __device__ __forceinline__ static void add_at(uint32_t* base, bool active, uint32_t type13) {
        const unsigned addr = (unsigned)__cvta_generic_to_shared(base + type13);
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %0, 0;\n\t@p red.shared.add.u32 [%1], 1;\n\t}"
                     :: "r"((unsigned)active), "r"(addr) : "memory");
    }
};

constexpr int TQN = 64;  // per-warp queue of hits (ring)

struct TriArgs {
    const SegDev* seg;
    const int64_t* pfx;
    int nseg;
    int64_t rows;
    const uint32_t* fptr;
    const unsigned long long* tpre;
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
};

// Lookup lists are cut into pieces of at most PIECE entries: a warp locates
// 32 pieces at a time from the start bits of the dyads whose pieces begin in
// that chunk (one piece per lane), then looks them up two at a time, one per
// half-warp, each lane one entry (coalesced loads).  R-MAT scale 22: 82% of
// the lanes' entry slots are used.
constexpr int PIECE = 16;
constexpr int HW_ILP = 4;  // piece pairs whose entries a warp loads together (searches)
constexpr int TB_ILP = 8;  // the same for the tag-map lookups (a chunk's 32 pieces in two steps)

// Pieces of the dyads begun before chunk c: `before` is advanced past the
// dyads whose first piece lies in [c, c + 32); returns this lane's dyad.
// `start` is the dyad's first piece (ignored for lanes without one).
__device__ __forceinline__ int chunk_dyad(bool has, uint32_t start, uint32_t c, int& before, int lane) {
    const bool in = has && start >= c && start < c + 32;
    const unsigned bits = __reduce_or_sync(0xffffffffu, in ? 1u << (start - c) : 0u);
    const int d = before + __popc(bits & (0xffffffffu >> (31 - lane))) - 1;
    before += __popc(bits);
    return d;
}

// Queue a chunk-iteration's hits (one lookup per lane): {R << 2 | t_h(w),
// dyad << 2 | t_x(w)}.
__device__ __forceinline__ void enqueue(uint2* q, int qh, int& qn, bool hit, uint32_t kv, uint32_t th, int d, int lane) {
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (hit) q[(qh + qn + __popc(m & ((1u << lane) - 1u))) & (TQN - 1)] = make_uint2((kv & ~3u) | th, ((uint32_t)d << 2) | (kv & 3u));
    qn += __popc(m);
}

// Apply cnt queued hits (one per lane): the third vertex's id from the rank
// permutation; x and t_x(h) from xin of the hit's dyad; the owner h.
// Queued hits are applied in two steps, so that the gather of the third
// vertex's id overlaps the following lookups: drain() takes cnt entries off
// the queue (one per lane), reads x, t_x(h) and the owner from the hit's
// dyad, issues the gather and keeps the batch pending; the pending batch is
// counted when the next one is taken (or by finish(), before the dyad table
// changes).
struct Pending {
    uint32_t w, x, h, tags;  // third vertex (loading), x << 2 | t_x(h), owner, t_x(w) << 2 | t_h(w)
    bool on;
};

__device__ __forceinline__ void finish(TriHist& H, Pending& P, unsigned& hits) {
    int type = 0;
    if (P.on) {
        type = tri_type(P.x >> 2, P.h, P.w, P.x & 3u, P.tags >> 2, P.tags & 3u);
        ++hits;
    }
    H.add(P.on, type);
    P.on = false;
}

template <class XinOf, class OwnerOf>
__device__ __forceinline__ void drain(TriHist& H, Pending& P, uint2* q, int& head, int& n, int cnt, XinOf xin_of,
                                      OwnerOf owner_of, const int32_t* perm, int64_t p0, int64_t ns,
                                      unsigned& hits) {
    const int lane = H.lane;
    finish(H, P, hits);
    __syncwarp();
    const uint2 e = q[(head + (lane < cnt ? lane : 0)) & (TQN - 1)];
    const int dq = lane < cnt ? (int)(e.y >> 2) : 0;
    const uint32_t qx = xin_of(dq), qh = owner_of(dq);
    P.on = lane < cnt && (e.x >> 2) < ns;  // ranks of the graph lie in [0, n)
    if (P.on) {
        P.w = (uint32_t)perm[p0 + (e.x >> 2)];
        P.x = qx;
        P.h = qh;
        P.tags = ((e.y & 3u) << 2) | (e.x & 3u);
    }
    __syncwarp();
    head = (head + cnt) & (TQN - 1);
    n -= cnt;
}

// Shared-memory layout of k_tri_big.
constexpr int TB_NT = 256;
constexpr int TB_W = TB_NT / 32;
constexpr int TB_REC = TRI_PIECE;  // records per work item, two per thread
constexpr size_t TB_MAP_BYTES = sizeof(uint32_t) * (MAP_KEYS / 16);
constexpr size_t TB_LIST_BYTES = sizeof(uint32_t) * 2 * MLIST;
constexpr size_t TB_TAB_BYTES = sizeof(uint32_t) * 4 * TB_REC;
constexpr size_t TB_HS_BYTES = sizeof(uint32_t) * 64 * TB_W;
constexpr size_t TB_Q_BYTES = sizeof(uint2) * TQN * TB_W;
constexpr size_t TB_SMEM = TB_MAP_BYTES + TB_LIST_BYTES + TB_TAB_BYTES + TB_HS_BYTES + TB_Q_BYTES;
static_assert(TB_REC == 2 * TB_NT, "a work item's records are read two per thread");
// chunk counts the queue area holds: items of more pieces (lookup lists
// longer than 2,048 entries on average) find their chunks' dyads by search
constexpr int TB_CB_CAP = (int)(TB_Q_BYTES / sizeof(uint16_t));

// Tag-map work items: two words each, {owner row, owner rank, forward list
// start, its length} and {first record, end of records, graph, 0}
// (k_fwd_rows writes {owner row, piece}; k_fwd_items completes them once the
// record offsets are known).
__global__ void k_fwd_items(const int64_t* __restrict__ pfx, int nseg, FwdLayout F) {
    const unsigned n = min(*F.nitems, F.item_cap);
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint4 it = F.items[2 * k];
        const int64_t rh = it.x;
        const uint32_t tb = (uint32_t)(F.tpre[rh] >> 32), te = (uint32_t)(F.tpre[rh + 1] >> 32);
        const uint32_t t0 = tb + it.y * TB_REC, t1 = min(te, t0 + (uint32_t)TB_REC);
        const uint32_t mb = F.fptr[rh], mn = F.fptr[rh + 1] - mb;
        F.items[2 * k] = make_uint4(it.x, (uint32_t)F.rank[rh], mb, mn);
        F.items[2 * k + 1] = make_uint4(t0, t1, (uint32_t)row_seg(pfx, nseg, rh), 0u);
        atomicAdd(F.stat + 4, (unsigned long long)mn);  // forward-list entries the items stage
    }
}

__device__ __forceinline__ void cp_async4(uint32_t* dst, const uint32_t* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Owners with a tag map: persistent CTAs take work items (up to TB_REC of
// one owner's records each) from a global cursor, two items ahead: the
// descriptor of the item after next is fetched while this one runs, and
// warp 0 copies the next owner's forward list asynchronously.  The item's
// dyads with a non-empty lookup list are compacted into a table (first
// entry, length, x << 2 | t_x(h), first piece), and the warps take its
// pieces 32 at a time from a shared cursor.  The item's records load while
// the map changes owner.
template <bool IDS>
__global__ void __launch_bounds__(TB_NT, 4) k_tri_big(TriArgs a) {
    extern __shared__ __align__(16) unsigned char tb_smem[];
    uint32_t* map = reinterpret_cast<uint32_t*>(tb_smem);
    uint32_t* mlist = reinterpret_cast<uint32_t*>(tb_smem + TB_MAP_BYTES);
    uint32_t* pof = reinterpret_cast<uint32_t*>(tb_smem + TB_MAP_BYTES + TB_LIST_BYTES);
    uint32_t* tfst = pof + TB_REC;
    uint32_t* tlen = tfst + TB_REC;
    uint32_t* txin = tlen + TB_REC;
    uint32_t* hs_all = reinterpret_cast<uint32_t*>(tb_smem + TB_MAP_BYTES + TB_LIST_BYTES + TB_TAB_BYTES);
    uint2* q_all = reinterpret_cast<uint2*>(tb_smem + TB_MAP_BYTES + TB_LIST_BYTES + TB_TAB_BYTES + TB_HS_BYTES);
    // rank-order counting (no hit queues): the queue area holds, per 32-piece
    // chunk of the item, the number of the item's dyads begun before it
    uint16_t* cbefore = reinterpret_cast<uint16_t*>(q_all);
    __shared__ unsigned long long wsum[TB_W];
    __shared__ int ctl_ntask, ctl_total;
    __shared__ unsigned ccur;  // next 32-piece chunk of the item
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = threadIdx.x; j < MAP_KEYS / 16; j += TB_NT) map[j] = 0;
    TriHist H{hs_all + warp * 64, a.acc, -1, lane, 0u};
    uint32_t* const hbase = H.hs + ((lane & 1) << 5) - 13;
    H.hs[lane] = 0;
    H.hs[32 + lane] = 0;
    uint2* q = q_all + warp * TQN;
    int qh = 0, qn = 0;
    Pending P{0, 0, 0, 0, false};
    unsigned long long looked = 0, tri = 0;
    unsigned hits = 0;
    const unsigned nitems = min(*a.nitems, a.item_cap);
    // descriptors of this item and the next two (slot i % 3); y = 0xffffffff
    // in the second word's z marks "no item"
    __shared__ uint4 dring[3][2];
    const uint4 none = make_uint4(0, 0, 0xffffffffu, 0);
    auto fetch = [&](uint4& A, uint4& B) {  // lane 0 of warp 0
        const unsigned k = atomicAdd(a.cursor, 1u);
        if (k < nitems) {
            A = a.items[2 * k];
            B = a.items[2 * k + 1];
        } else {
            A = make_uint4(0, 0, 0, 0);
            B = none;
        }
    };
    uint4 fA = make_uint4(0, 0, 0, 0), fB = none;  // the item after next, in flight (warp 0 lane 0)
    if (threadIdx.x == 0) {
        uint4 A, B;
        fetch(A, B);
        dring[0][0] = A;
        dring[0][1] = B;
        fetch(A, B);
        dring[1][0] = A;
        dring[1][1] = B;
    }
    __syncthreads();
    if (warp == 0 && dring[0][1].z != 0xffffffffu) {
        for (uint32_t i = lane; i < dring[0][0].w; i += 32) cp_async4(mlist + i, a.fwd + dring[0][0].z + i);
        cp_async_commit();
    }
    int64_t prev_rh = -1;
    int32_t prev_R = 0;
    uint32_t prev_n = 0;
    for (int b = 0, slot = 0;; b ^= 1, slot = slot == 2 ? 0 : slot + 1) {
        const uint4 dA = dring[slot][0], dB = dring[slot][1];
        if (dB.z == 0xffffffffu) break;
        const uint4 nA = dring[slot == 2 ? 0 : slot + 1][0], nB = dring[slot == 2 ? 0 : slot + 1][1];
        if (threadIdx.x == 0) fetch(fA, fB);  // consumed at the end of this item
        const int64_t rh = dA.x;
        const int32_t Rh = (int32_t)dA.y;
        const uint32_t mn = dA.w, t0 = dB.x, t1 = dB.y;
        const int sg = (int)dB.z;
        const int64_t p0 = a.pfx[sg], ns = a.seg[sg].n;
        // the item's records, two per thread, in flight while the map changes
        uint4 r0 = make_uint4(0, 0, 0, 0), r1 = make_uint4(0, 0, 0, 0);
        const uint32_t i0 = t0 + 2 * threadIdx.x;
        if (i0 < t1) r0 = a.trec[i0];
        if (i0 + 1 < t1) r1 = a.trec[i0 + 1];
        if (warp == 0) cp_async_wait_all();  // this owner's list is in mlist[b]
        if (rh != prev_rh) {  // clear the previous owner's entries, then map this owner
            const uint32_t* old = mlist + (b ^ 1) * MLIST;
            for (uint32_t i = threadIdx.x; i < prev_n; i += TB_NT) {
                const uint32_t k = (old[i] >> 2) - (uint32_t)prev_R - 1u;
                if (k < (uint32_t)MAP_KEYS) map[k >> 4] = 0;
            }
            __syncthreads();
            const uint32_t* cur = mlist + b * MLIST;
            for (uint32_t i = threadIdx.x; i < mn; i += TB_NT) {
                const uint32_t e = cur[i];
                const uint32_t k = (e >> 2) - (uint32_t)Rh - 1u;
                if (k < (uint32_t)MAP_KEYS) atomicOr(map + (k >> 4), (e & 3u) << (2 * (k & 15u)));
            }
        }
        // the item's table: one block-wide scan of (dyads << 40 | pieces)
        const uint32_t np0 = (r0.y + PIECE - 1) / PIECE, np1 = (r1.y + PIECE - 1) / PIECE;
        const unsigned long long v = ((unsigned long long)((np0 > 0) + (np1 > 0)) << 40) | (np0 + np1);
        unsigned long long incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(full, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        if (threadIdx.x == 0) ccur = 0;
        __syncthreads();
        unsigned long long ex = incl - v;
        for (int w = 0; w < warp; ++w) ex += wsum[w];
        {
            int d = (int)(ex >> 40);
            uint32_t po = (uint32_t)(ex & 0xffffffffffull);
            // chunk ch (pieces from 32 ch) begins inside exactly one dyad's
            // pieces [po, po + np): the dyads begun before it are that dyad's
            // index, plus one when the dyad began in an earlier chunk
            auto mark = [&](int dd, uint32_t p0, uint32_t np) {
                if constexpr (!IDS) {
                    for (uint32_t ch = (p0 + 31) >> 5; (ch << 5) < p0 + np && ch < (uint32_t)TB_CB_CAP; ++ch)
                        cbefore[ch] = (uint16_t)((ch << 5) == p0 ? dd : dd + 1);
                }
            };
            if (np0 > 0) {
                pof[d] = po;
                tfst[d] = r0.x;
                tlen[d] = r0.y;
                txin[d] = r0.z;
                mark(d, po, np0);
                ++d;
                po += np0;
            }
            if (np1 > 0) {
                pof[d] = po;
                tfst[d] = r1.x;
                tlen[d] = r1.y;
                txin[d] = r1.z;
                mark(d, po, np1);
            }
        }
        if (threadIdx.x == TB_NT - 1) {
            ex += v;
            ctl_ntask = (int)(ex >> 40);
            ctl_total = (int)(ex & 0xffffffffffull);
        }
        __syncthreads();
        const int ntask = ctl_ntask, total = ctl_total;
        if (warp == 0 && nB.z != 0xffffffffu) {  // the next owner's list, asynchronously
            uint32_t* nl = mlist + (b ^ 1) * MLIST;
            for (uint32_t i = lane; i < nA.w; i += 32) cp_async4(nl + i, a.fwd + nA.z + i);
            cp_async_commit();
        }
        H.retag(sg);
        const uint32_t Rh1 = (uint32_t)Rh + 1u, hl = (uint32_t)(rh - p0);
        // 32-piece chunks of the item, taken dynamically by the warps
        for (;;) {
            int c = 0;
            if (lane == 0) c = (int)atomicAdd(&ccur, 32u);
            c = __shfl_sync(full, c, 0);
            if (c >= total) break;
            int before;  // dyads whose first piece lies below c
            if (!IDS && total <= TB_CB_CAP * 32) {  // c < total: an index below TB_CB_CAP
                before = cbefore[c >> 5];
            } else {
                int l = 0, h = ntask;
                while (l < h) {
                    const int mid = (l + h) >> 1;
                    if ((int)pof[mid] < c) l = mid + 1;
                    else h = mid;
                }
                before = l;
            }
            const bool has = before + lane < ntask;
            const uint32_t st = has ? pof[before + lane] : 0u;
            const int d = chunk_dyad(has, st, (uint32_t)c, before, lane);
            const bool ok = c + lane < total;
            uint32_t base = 0, cnt = 0;  // cnt: entries | 9 t_x(h) << 8
            if (ok) {
                const uint32_t pq = (uint32_t)(c + lane) - pof[d];
                base = tfst[d] + PIECE * pq;
                cnt = min((uint32_t)PIECE, tlen[d] - PIECE * pq) | ((9u * (txin[d] & 3u)) << 8);
            }
            // the chunk's pieces two at a time, one per half-warp (lane & 15
            // is the entry), TB_ILP pairs loaded together
            const int npc = min(32, total - c), e = lane & 15, half = lane >> 4;
            for (int u0 = 0; u0 < npc; u0 += 2 * TB_ILP) {
                uint32_t kv[TB_ILP], xt[TB_ILP];
                int dv[TB_ILP];
                bool vv[TB_ILP];
#pragma unroll
                for (int u = 0; u < TB_ILP; ++u) {
                    const int src = u0 + 2 * u + half;
                    const uint32_t pb = __shfl_sync(full, base, src & 31), pc = __shfl_sync(full, cnt, src & 31);
                    if (IDS) dv[u] = __shfl_sync(full, d, src & 31);
                    vv[u] = src < npc && (uint32_t)e < (pc & 0xffu);
                    xt[u] = pc >> 8;
                    kv[u] = vv[u] ? __ldg(a.fwd + pb + e) : 0u;
                }
#pragma unroll
                for (int u = 0; u < TB_ILP; ++u) {
                    // ranks at or below h, and the zero word of an idle lane,
                    // fall outside the map
                    const uint32_t kk = (kv[u] >> 2) - Rh1;
                    const uint32_t mw = map[(kk >> 4) & (MAP_KEYS / 16 - 1)];  // always in range
                    const uint32_t th = kk < (uint32_t)MAP_KEYS ? (mw >> (2 * (kk & 15u))) & 3u : 0u;
                    if (IDS) {
                        enqueue(q, qh, qn, th != 0, kv[u], th, dv[u], lane);
                        if (qn >= 32)
                            drain(H, P, q, qh, qn, 32, [&](int dq) { return txin[dq]; }, [&](int) { return hl; },
                                  a.perm, p0, ns, hits);
                    } else {  // rank order x < h < w: the type from the three tags (counted at flush)
                        TriHist::add_at(hbase, th != 0, xt[u] + 3u * (kv[u] & 3u) + th);
                    }
                }
            }
            looked += cnt & 0xffu;
        }
        if (IDS) {
            if (qn > 0)  // the table changes next
                drain(H, P, q, qh, qn, qn, [&](int dq) { return txin[dq]; }, [&](int) { return hl; }, a.perm, p0,
                      ns, hits);
            finish(H, P, hits);
        }
        // hits bound the histogram's growth: counted in IDS mode, else the
        // item's entry slots (its triangles are counted at flush)
        const unsigned wh = IDS ? __reduce_add_sync(full, hits) : 0u;
        H.pending += IDS ? wh : (unsigned)total * PIECE;
        tri += wh;
        hits = 0;
        prev_rh = rh;
        prev_R = Rh;
        prev_n = mn;
        if (threadIdx.x == 0) {
            const int s2 = slot == 0 ? 2 : slot - 1;  // (slot + 2) % 3
            dring[s2][0] = fA;
            dring[s2][1] = fB;
        }
        __syncthreads();
    }
    if (warp == 0) cp_async_wait_all();
    H.flush();
    if (!IDS) tri = warp_sum64(H.seen);
    looked = warp_sum64(looked);
    if (lane == 0 && looked) atomicAdd(a.stat + 0, looked);
    if (lane == 0 && tri) atomicAdd(a.stat + 1, tri);
}

// Every other owner: warps take runs of TS_RUN records of the search part
// (grouped by owner) and, 32 records at a time, look each piece's entries up
// in its owner's forward list (sorted by rank) by binary search, the piece's
// searches in lockstep (a run's dyads share few owners, so their lists stay
// in cache).
constexpr int TS_RUN = 128;

template <bool IDS>
__global__ void __launch_bounds__(256) k_tri_small(TriArgs a) {
    __shared__ uint32_t hs_all[8][64];
    __shared__ uint2 q_all[8][TQN];
    __shared__ uint4 st_all[8][32];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    TriHist H{hs_all[warp], a.acc, -1, lane, 0u};
    uint32_t* const hbase = H.hs + ((lane & 1) << 5) - 13;
    H.hs[lane] = 0;
    H.hs[32 + lane] = 0;
    uint2* q = q_all[warp];
    uint4* stage = st_all[warp];
    int qh = 0, qn = 0;
    Pending P{0, 0, 0, 0, false};
    __syncwarp();
    unsigned long long looked = 0, tri = 0;
    unsigned hits = 0;
    const unsigned long long tot = a.tpre[a.rows];
    const uint32_t r0 = (uint32_t)(tot >> 32), r1 = r0 + (uint32_t)(tot & 0xffffffffull);
    for (;;) {
        unsigned run = 0;
        if (lane == 0) run = r0 + atomicAdd(a.cursor + 1, (unsigned)TS_RUN);
        run = __shfl_sync(full, run, 0);
        if (run >= r1) break;
        const uint32_t rend = min(r1, run + TS_RUN);
        for (uint32_t g0 = run; g0 < rend;) {
            const uint32_t t = g0 + lane;
            const bool valid = t < rend;
            const uint4 rec = valid ? a.trec[t] : make_uint4(0, 0, 0, 0);
            const int s = valid ? row_seg(a.pfx, a.nseg, (int64_t)rec.w) : -1;
            const int s0 = __shfl_sync(full, s, 0);
            // a group stays within one graph (records are grouped by owner)
            const unsigned other = __ballot_sync(full, !valid || s != s0);
            const int take = other ? __ffs(other) - 1 : 32;
            const int64_t p0 = a.pfx[s0], ns0 = a.seg[s0].n;
            H.retag(s0);
            // the group's dyads with a non-empty lookup list, compacted
            const bool use = lane < take && rec.y > 0;
            const unsigned um = __ballot_sync(full, use);
            const int ng = __popc(um);
            if (use) stage[__popc(um & lt)] = rec;
            __syncwarp();
            uint32_t fst = 0, len = 0, xin = 0, hl = 0, hb = 0, hn = 0;
            if (lane < ng) {
                const uint4 c = stage[lane];
                fst = c.x;
                len = c.y;
                xin = c.z;
                hl = (uint32_t)((int64_t)c.w - p0);
                hb = a.fptr[c.w];
                hn = a.fptr[c.w + 1] - hb;
            }
            __syncwarp();
            const uint32_t np = (len + PIECE - 1) / PIECE;
            uint32_t poff = np;  // first piece of this lane's dyad
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(full, poff, o);
                if (lane >= o) poff += v;
            }
            const uint32_t total = __shfl_sync(full, poff, 31);
            poff -= np;
            int before = 0;
            for (uint32_t c = 0; c < total; c += 32) {
                const int d = chunk_dyad(lane < ng, poff, c, before, lane);
                const bool ok = c + lane < total;
                const int dd = ok ? d : 0;
                const uint32_t d_fst = __shfl_sync(full, fst, dd), d_len = __shfl_sync(full, len, dd);
                const uint32_t d_off = __shfl_sync(full, poff, dd);
                const uint32_t d_xin = __shfl_sync(full, xin, dd);
                uint32_t cnt = 0, base = 0;  // cnt: entries | 9 t_x(h) << 8
                if (ok) {
                    const uint32_t pq = c + lane - d_off;
                    base = d_fst + PIECE * pq;
                    cnt = min((uint32_t)PIECE, d_len - PIECE * pq) | ((9u * (d_xin & 3u)) << 8);
                }
                // the chunk's pieces two at a time, one per half-warp (lane & 15
                // is the entry): each lane searches its key in the piece's
                // owner list, HW_ILP pairs in lockstep
                const int npc = (int)min(32u, total - c), e = lane & 15, half = lane >> 4;
                for (int t0 = 0; t0 < npc; t0 += 2 * HW_ILP) {
                    uint32_t kv[HW_ILP], ob[HW_ILP], on[HW_ILP], pos[HW_ILP], xt[HW_ILP];
                    int dv[HW_ILP];
                    bool vv[HW_ILP];
                    uint32_t maxn = 0;
#pragma unroll
                    for (int u = 0; u < HW_ILP; ++u) {
                        const int src = t0 + 2 * u + half;
                        const uint32_t pb = __shfl_sync(full, base, src & 31), pc = __shfl_sync(full, cnt, src & 31);
                        dv[u] = __shfl_sync(full, d, src & 31);
                        const int od = dv[u] < 0 ? 0 : dv[u];
                        ob[u] = __shfl_sync(full, hb, od & 31);
                        on[u] = __shfl_sync(full, hn, od & 31);
                        vv[u] = src < npc && (uint32_t)e < (pc & 0xffu);
                        xt[u] = pc >> 8;
                        kv[u] = vv[u] ? __ldg(a.fwd + pb + e) : 0u;
                        if (!vv[u]) on[u] = 0;
                        pos[u] = 0;
                        maxn = max(maxn, on[u]);
                    }
                    // lower bound of each key in its owner's sorted list
                    for (uint32_t step = maxn ? 1u << (31 - __clz(maxn)) : 0u; step > 0; step >>= 1) {
#pragma unroll
                        for (int u = 0; u < HW_ILP; ++u)
                            if (pos[u] + step <= on[u] &&
                                (__ldg(a.fwd + ob[u] + pos[u] + step - 1) & ~3u) < (kv[u] & ~3u))
                                pos[u] += step;
                    }
#pragma unroll
                    for (int u = 0; u < HW_ILP; ++u) {
                        uint32_t th = 0;
                        if (vv[u] && pos[u] < on[u]) {
                            const uint32_t w = __ldg(a.fwd + ob[u] + pos[u]);
                            if ((w & ~3u) == (kv[u] & ~3u)) th = w & 3u;
                        }
                        if (IDS) {
                            enqueue(q, qh, qn, th != 0, kv[u], th, dv[u], lane);
                            if (qn >= 32)
                                drain(H, P, q, qh, qn, 32, [&](int dq) { return __shfl_sync(full, xin, dq); },
                                      [&](int dq) { return __shfl_sync(full, hl, dq); }, a.perm, p0, ns0, hits);
                        } else {  // rank order x < h < w: the type from the three tags (counted at flush)
                            TriHist::add_at(hbase, th != 0, xt[u] + 3u * (kv[u] & 3u) + th);
                        }
                    }
                }
                looked += cnt & 0xffu;
            }
            if (IDS) {
                if (qn > 0)  // the group changes next
                    drain(H, P, q, qh, qn, qn, [&](int dq) { return __shfl_sync(full, xin, dq); },
                          [&](int dq) { return __shfl_sync(full, hl, dq); }, a.perm, p0, ns0, hits);
                finish(H, P, hits);
            }
            // hits bound the histogram's growth: counted in IDS mode, else
            // the group's entry slots (its triangles are counted at flush)
            const unsigned wh = IDS ? __reduce_add_sync(full, hits) : 0u;
            H.pending += IDS ? wh : total * PIECE;
            tri += wh;
            hits = 0;
            g0 += (uint32_t)take;
        }
    }
    H.flush();
    if (!IDS) tri = warp_sum64(H.seen);
    looked = warp_sum64(looked);
    if (lane == 0 && looked) atomicAdd(a.stat + 2, looked);
    if (lane == 0 && tri) atomicAdd(a.stat + 3, tri);
}
