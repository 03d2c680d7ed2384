/*
 * Triad-census ORACLE -- test infrastructure only.
 *
 * This file is a plain, slow, obviously-correct CPU restatement of the
 * subquadratic triad census described in the thesis "Study and evaluation of
 * an Irregular Graph Algorithm on Multicore and GPU Processor Architectures"
 * (arXiv 1603.02655).  It exists so that tests, the smoke check and the
 * benchmark's CPU-baseline leg can check and time the CUDA library against an
 * independent implementation.  The product path never calls it, and it shares
 * no code, header, table or constant with the CUDA library.
 *
 * Contents
 *   oracle_triad_table  64 -> 16 isomorphism table, DERIVED here from the MAN
 *                       naming rules of Sec. 2.2 (the thesis does not print
 *                       the table; its figure of the 16 types is lost).
 *   oracle_brute        O(n^3) definition: classify every vertex triple.
 *   oracle_brute_codes  O(n^3) 64-code census: each triple given to the dyad
 *                       and third vertex that count it (canonical test).
 *   oracle_census_codes the 64-code (non-isomorphic) census of the same loop.
 *   oracle_census_*     the algorithm of Sec. 2.2, Fig. "Subquadratic Triad
 *                       Census Algorithm", with the v0.4 pre-computed dyad part
 *                       of Sec. 4.2.4 (Fig. "Modified TriadCode Algorithm").
 *                       Set union S = N(u) u N(v) \ {u,v} is built explicitly;
 *                       IsEdge / IsNeighbour are binary searches.
 *   multithreaded run   std::thread over canonical-dyad task queues cut with
 *                       the uniform-distribution cost |N(u)|+|N(v)|-2 of
 *                       Sec. 4.3.1 (Fig. "... Canonical Dyad(uniform distr.)"),
 *                       one private census per thread, summed after the join
 *                       (the decoupled per-thread arrays of Sec. 4.3.2).
 *
 * Type indices are 0-based in MAN order: 0=003 1=012 2=102 3=021D 4=021U
 * 5=021C 6=111D 7=111U 8=030T 9=030C 10=201 11=120D 12=120U 13=120C 14=210
 * 15=300 (the thesis numbers them 1..16, Sec. 2.2).
 *
 * Readings of points where the thesis is silent or garbled:
 *   - self-loops are dropped and duplicate arcs collapse (it assumes a strict
 *     digraph, Sec. 2.2);
 *   - the null-triad line "T1 = T - T1 - T2" is read as
 *     003 = C(n,3) - (all other counts), computed in 128-bit arithmetic because
 *     n(n-1)(n-2) overflows 64 bits for n > ~2.6M;
 *   - the 6-bit code is 0-based: code = pre + 4e(u,w) + 8e(w,u) + 16e(v,w)
 *     + 32e(w,v) with pre = e(u,v) + 2e(v,u) (Fig. "Modified TriadCode").
 *
 * Parity pins (tests/test_oracle.py): all 64 three-vertex digraphs, all 4096
 * four-vertex digraphs against brute force, closed forms, invariants, an
 * external black-box census routine, and G(n,p) expected counts.
 */
#include <algorithm>
#include <array>
#include <atomic>
#include <iterator>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

typedef unsigned __int128 u128;

namespace {

/* ---------------------------------------------------------------- table -- */

/* Arc e(a,b) of the three-vertex digraph encoded by a 6-bit code; vertex 0 is
 * u, 1 is v, 2 is w (bit order of Fig. "Triad Code Algorithm"). */
bool code_arc(int code, int a, int b) {
    if (a == 0 && b == 1) return code & 1;
    if (a == 1 && b == 0) return code & 2;
    if (a == 0 && b == 2) return code & 4;
    if (a == 2 && b == 0) return code & 8;
    if (a == 1 && b == 2) return code & 16;
    if (a == 2 && b == 1) return code & 32;
    return false;
}

/* Classify one labelled triad by the MAN rules of Sec. 2.2:
 * M mutual, A asymmetric, N null dyads, plus the U/D/C/T property. */
int classify_man(int code) {
    int M = 0, A = 0;
    int asym_out[3] = {0, 0, 0}, asym_in[3] = {0, 0, 0};
    int mutual_pair_other = -1; /* for M==1: the vertex outside the mutual pair */
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
    for (int k = 0; k < 3; ++k) {
        int a = pa[k], b = pb[k];
        bool ab = code_arc(code, a, b), ba = code_arc(code, b, a);
        if (ab && ba) {
            ++M;
            mutual_pair_other = 3 - a - b;
        } else if (ab) {
            ++A; asym_out[a]++; asym_in[b]++;
        } else if (ba) {
            ++A; asym_out[b]++; asym_in[a]++;
        }
    }
    bool some_out2 = asym_out[0] == 2 || asym_out[1] == 2 || asym_out[2] == 2;
    bool some_in2 = asym_in[0] == 2 || asym_in[1] == 2 || asym_in[2] == 2;
    if (M == 0 && A == 0) return 0;                   /* 003 */
    if (M == 0 && A == 1) return 1;                   /* 012 */
    if (M == 1 && A == 0) return 2;                   /* 102 */
    if (M == 0 && A == 2) {                           /* 021 */
        if (some_out2) return 3;                      /* 021D: one vertex sends both */
        if (some_in2) return 4;                       /* 021U: one vertex receives both */
        return 5;                                     /* 021C: a 2-path */
    }
    if (M == 1 && A == 1) {                           /* 111 */
        int r = mutual_pair_other;
        /* D: the lone asymmetric arc runs from the outside vertex into the pair */
        return asym_out[r] == 1 ? 6 : 7;
    }
    if (M == 0 && A == 3) return some_out2 ? 8 : 9;   /* 030T transitive, 030C cycle */
    if (M == 2 && A == 0) return 10;                  /* 201 */
    if (M == 1 && A == 2) {                           /* 120 */
        int r = mutual_pair_other;
        if (asym_out[r] == 2) return 11;              /* 120D: outside vertex sends both */
        if (asym_in[r] == 2) return 12;               /* 120U: outside vertex receives both */
        return 13;                                    /* 120C */
    }
    if (M == 2 && A == 1) return 14;                  /* 210 */
    return 15;                                        /* 300 */
}

struct Table {
    int t[64];
    Table() { for (int c = 0; c < 64; ++c) t[c] = classify_man(c); }
};
const Table& table() { static Table tb; return tb; }

u128 choose3(int64_t n) {
    if (n < 3) return 0;
    u128 x = (u128)(uint64_t)n * (u128)(uint64_t)(n - 1) * (u128)(uint64_t)(n - 2);
    return x / 6;
}

/* ---------------------------------------------------------------- graph -- */

/* Sorted adjacency in CRS form (Sec. 2.5.1, Fig. "Adjacency array representation"):
 * N(u) the undirected open neighbourhood, E(u) the out-arcs. */
struct OGraph {
    int32_t n = 0;
    std::vector<int64_t> nptr, eptr;
    std::vector<int32_t> nbr, out;
};

void build_crs(int32_t n, std::vector<uint64_t>& keys, std::vector<int64_t>& ptr,
               std::vector<int32_t>& col) {
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    ptr.assign((size_t)n + 1, 0);
    col.resize(keys.size());
    for (size_t i = 0; i < keys.size(); ++i) {
        ptr[(keys[i] >> 32) + 1]++;
        col[i] = (int32_t)(keys[i] & 0xffffffffu);
    }
    for (int64_t v = 0; v < n; ++v) ptr[v + 1] += ptr[v];
}

OGraph* graph_new(int32_t n, int64_t m, const int32_t* src, const int32_t* dst) {
    if (n < 0 || m < 0) return nullptr;
    std::vector<uint64_t> ek, nk;
    ek.reserve((size_t)m);
    nk.reserve(2 * (size_t)m);
    for (int64_t i = 0; i < m; ++i) {
        int32_t s = src[i], d = dst[i];
        if (s < 0 || s >= n || d < 0 || d >= n) return nullptr;
        if (s == d) continue; /* strict digraph: loops dropped */
        ek.push_back(((uint64_t)s << 32) | (uint32_t)d);
        nk.push_back(((uint64_t)s << 32) | (uint32_t)d);
        nk.push_back(((uint64_t)d << 32) | (uint32_t)s);
    }
    OGraph* g = new OGraph;
    g->n = n;
    build_crs(n, ek, g->eptr, g->out);
    build_crs(n, nk, g->nptr, g->nbr);
    return g;
}

bool is_edge(const OGraph& g, int32_t a, int32_t b) {
    return std::binary_search(g.out.begin() + g.eptr[a], g.out.begin() + g.eptr[a + 1], b);
}
bool is_neighbour(const OGraph& g, int32_t a, int32_t b) {
    return std::binary_search(g.nbr.begin() + g.nptr[a], g.nbr.begin() + g.nptr[a + 1], b);
}
int64_t deg(const OGraph& g, int32_t a) { return g.nptr[a + 1] - g.nptr[a]; }

/* The dyad loop of Fig. "Subquadratic Triad Census Algorithm" for u in
 * [ub, ue): dyadic term, canonical test, TriadCode.  Adds into cnt[16]
 * (index 0 untouched) and returns the merged-entry count sum(|N(u)|+|N(v)|). */
uint64_t census_range(const OGraph& g, int32_t ub, int32_t ue, u128 cnt[16]) {
    const int* T = table().t;
    const int64_t n = g.n;
    std::vector<int32_t> S;
    uint64_t entries = 0;
    for (int32_t u = ub; u < ue; ++u) {
        auto nu_b = g.nbr.begin() + g.nptr[u], nu_e = g.nbr.begin() + g.nptr[u + 1];
        for (auto it = nu_b; it != nu_e; ++it) {
            const int32_t v = *it;
            if (!(u < v)) continue;                         /* canonical dyad */
            auto nv_b = g.nbr.begin() + g.nptr[v], nv_e = g.nbr.begin() + g.nptr[v + 1];
            entries += (uint64_t)(deg(g, u) + deg(g, v));
            /* S = N(u) u N(v) \ {u, v} */
            S.clear();
            std::set_union(nu_b, nu_e, nv_b, nv_e, std::back_inserter(S));
            S.erase(std::remove_if(S.begin(), S.end(),
                                   [&](int32_t x) { return x == u || x == v; }),
                    S.end());
            /* pre-computed dyad part (v0.4) */
            const int e0 = is_edge(g, u, v) ? 1 : 0;
            const int e1 = is_edge(g, v, u) ? 1 : 0;
            const int pre = e0 + 2 * e1;
            const int dyadic_type = (e0 && e1) ? 2 /* 102 */ : 1 /* 012 */;
            cnt[dyadic_type] += (u128)(uint64_t)(n - (int64_t)S.size() - 2);
            for (int32_t w : S) {
                if (v < w || (w < v && u < w && !is_neighbour(g, u, w))) {
                    int code = pre;
                    code += 4 * (is_edge(g, u, w) ? 1 : 0);
                    code += 8 * (is_edge(g, w, u) ? 1 : 0);
                    code += 16 * (is_edge(g, v, w) ? 1 : 0);
                    code += 32 * (is_edge(g, w, v) ? 1 : 0);
                    cnt[T[code]] += 1;
                }
            }
        }
    }
    return entries;
}

/* The same loop in the non-isomorphic mode of Fig. "Triad Code Algorithm"
 * (the code itself, no TriadTable): the dyadic term goes to code pre (a
 * triad whose only arcs join u and v), every counted w to its 6-bit code.
 * Adds into c[64] (index 0 untouched). */
void census_codes_range(const OGraph& g, int32_t ub, int32_t ue, u128 c[64]) {
    const int64_t n = g.n;
    std::vector<int32_t> S;
    for (int32_t u = ub; u < ue; ++u) {
        auto nu_b = g.nbr.begin() + g.nptr[u], nu_e = g.nbr.begin() + g.nptr[u + 1];
        for (auto it = nu_b; it != nu_e; ++it) {
            const int32_t v = *it;
            if (!(u < v)) continue;                         /* canonical dyad */
            auto nv_b = g.nbr.begin() + g.nptr[v], nv_e = g.nbr.begin() + g.nptr[v + 1];
            S.clear();
            std::set_union(nu_b, nu_e, nv_b, nv_e, std::back_inserter(S));
            S.erase(std::remove_if(S.begin(), S.end(),
                                   [&](int32_t x) { return x == u || x == v; }),
                    S.end());
            const int pre = (is_edge(g, u, v) ? 1 : 0) + 2 * (is_edge(g, v, u) ? 1 : 0);
            c[pre] += (u128)(uint64_t)(n - (int64_t)S.size() - 2);
            for (int32_t w : S) {
                if (v < w || (w < v && u < w && !is_neighbour(g, u, w))) {
                    int code = pre;
                    code += 4 * (is_edge(g, u, w) ? 1 : 0);
                    code += 8 * (is_edge(g, w, u) ? 1 : 0);
                    code += 16 * (is_edge(g, v, w) ? 1 : 0);
                    code += 32 * (is_edge(g, w, v) ? 1 : 0);
                    c[code] += 1;
                }
            }
        }
    }
}

void close_null(int64_t n, u128 cnt[16]) {
    u128 sum = 0;
    for (int t = 1; t < 16; ++t) sum += cnt[t];
    cnt[0] = choose3(n) - sum;
}

void store(const u128 cnt[16], uint64_t* lo, uint64_t* hi) {
    for (int t = 0; t < 16; ++t) {
        lo[t] = (uint64_t)cnt[t];
        hi[t] = (uint64_t)(cnt[t] >> 64);
    }
}

} // namespace

extern "C" {

/* 64 -> 16 table, derived from the MAN rules. */
void oracle_triad_table(int32_t out[64]) {
    for (int c = 0; c < 64; ++c) out[c] = table().t[c];
}

/* O(n^3) census by definition: every triple i<j<k, code of (i,j,k).
 * Returns 0, or -1 on bad arguments (n > 4096, id out of range). */
int oracle_brute(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                 uint64_t out[16]) {
    if (n < 0 || n > 4096 || m < 0) return -1;
    std::vector<uint8_t> adj((size_t)n * (size_t)n, 0);
    for (int64_t i = 0; i < m; ++i) {
        int32_t s = src[i], d = dst[i];
        if (s < 0 || s >= n || d < 0 || d >= n) return -1;
        if (s != d) adj[(size_t)s * n + d] = 1;
    }
    auto e = [&](int a, int b) { return (int)adj[(size_t)a * n + b]; };
    const int* T = table().t;
    for (int t = 0; t < 16; ++t) out[t] = 0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            for (int k = j + 1; k < n; ++k) {
                int code = e(i, j) + 2 * e(j, i) + 4 * e(i, k) + 8 * e(k, i) +
                           16 * e(j, k) + 32 * e(k, j);
                out[T[code]]++;
            }
    return 0;
}

/* O(n^3) 64-code census by definition: every triple i<j<k is given to the
 * canonical dyad <u,v> (u < v adjacent) and third vertex w that count it --
 * the only adjacent pair when w is isolated from both (code pre), else the
 * pair for which w passes the canonical test v < w or (u < w < v and w not
 * a neighbour of u) -- and its code is taken with that labelling; a triple
 * without arcs has code 0.  Returns 0, -1 on bad arguments (n > 4096, id out
 * of range), -2 if some triple is counted other than exactly once. */
int oracle_brute_codes(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, uint64_t out[64]) {
    if (n < 0 || n > 4096 || m < 0) return -1;
    std::vector<uint8_t> adj((size_t)n * (size_t)n, 0);
    for (int64_t i = 0; i < m; ++i) {
        int32_t s = src[i], d = dst[i];
        if (s < 0 || s >= n || d < 0 || d >= n) return -1;
        if (s != d) adj[(size_t)s * n + d] = 1;
    }
    auto e = [&](int a, int b) { return (int)adj[(size_t)a * n + b]; };
    auto nb = [&](int a, int b) { return e(a, b) || e(b, a); };
    for (int t = 0; t < 64; ++t) out[t] = 0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            for (int k = j + 1; k < n; ++k) {
                const int uvw[3][3] = {{i, j, k}, {i, k, j}, {j, k, i}};
                int counted = 0, any = 0;
                for (const auto& t : uvw) {
                    const int u = t[0], v = t[1], w = t[2];
                    if (!nb(u, v)) continue;
                    any = 1;
                    const int pre = e(u, v) + 2 * e(v, u);
                    if (!nb(u, w) && !nb(v, w)) {
                        out[pre]++;
                        ++counted;
                    } else if (v < w || (u < w && w < v && !nb(u, w))) {
                        out[pre + 4 * e(u, w) + 8 * e(w, u) + 16 * e(v, w) + 32 * e(w, v)]++;
                        ++counted;
                    }
                }
                if (!any) {
                    out[0]++;
                    ++counted;
                }
                if (counted != 1) return -2;
            }
    return 0;
}

void* oracle_graph_new(int32_t n, int64_t m, const int32_t* src, const int32_t* dst) {
    return graph_new(n, m, src, dst);
}

void oracle_graph_free(void* g) { delete (OGraph*)g; }

/* stats[0] n, [1] arcs, [2] canonical dyads |U|, [3] mutual dyads,
 * [4] asymmetric dyads, [5] merged entries sum over canonical dyads of
 * |N(u)|+|N(v)|, [6] max undirected degree. */
void oracle_graph_stats(const void* gp, int64_t stats[7]) {
    const OGraph& g = *(const OGraph*)gp;
    int64_t dyads = 0, mutual = 0, merged = 0, maxd = 0;
    for (int32_t u = 0; u < g.n; ++u) {
        maxd = std::max(maxd, deg(g, u));
        for (int64_t k = g.nptr[u]; k < g.nptr[u + 1]; ++k) {
            int32_t v = g.nbr[k];
            if (u < v) {
                ++dyads;
                merged += deg(g, u) + deg(g, v);
                if (is_edge(g, u, v) && is_edge(g, v, u)) ++mutual;
            }
        }
    }
    stats[0] = g.n;
    stats[1] = (int64_t)g.out.size();
    stats[2] = dyads;
    stats[3] = mutual;
    stats[4] = dyads - mutual;
    stats[5] = merged;
    stats[6] = maxd;
}

/* |N(u) n N(v)| for one pair (sampled checks at sizes the full census is too
 * slow for). */
int64_t oracle_common(const void* gp, int32_t u, int32_t v) {
    const OGraph& g = *(const OGraph*)gp;
    int64_t c = 0;
    int64_t i = g.nptr[u], ie = g.nptr[u + 1], j = g.nptr[v], je = g.nptr[v + 1];
    while (i < ie && j < je) {
        if (g.nbr[i] < g.nbr[j]) ++i;
        else if (g.nbr[j] < g.nbr[i]) ++j;
        else { ++c; ++i; ++j; }
    }
    return c;
}

/* Partial census over canonical dyads with u in [ub, ue): types 1..15 only
 * (no 003 closure).  Returns the merged entries processed. */
uint64_t oracle_census_range(const void* gp, int32_t ub, int32_t ue, uint64_t lo[16],
                             uint64_t hi[16]) {
    const OGraph& g = *(const OGraph*)gp;
    u128 cnt[16] = {0};
    ub = std::max(ub, 0);
    ue = std::min(ue, g.n);
    uint64_t entries = ub < ue ? census_range(g, ub, ue, cnt) : 0;
    store(cnt, lo, hi);
    return entries;
}

/* Full census with `threads` worker threads (1 = the sequential algorithm).
 * lo/hi receive the 128-bit count of each of the 16 types. */
void oracle_census(const void* gp, int32_t threads, uint64_t lo[16], uint64_t hi[16]) {
    const OGraph& g = *(const OGraph*)gp;
    if (threads < 1) threads = 1;
    /* Task queues over canonical dyads, uniform-distribution cost
     * |N(u)|+|N(v)|-2, cut at vertex boundaries once a queue exceeds
     * MaxNsetSize = total / (64 * threads). */
    std::vector<int32_t> cuts{0};
    {
        uint64_t total = 0;
        std::vector<uint64_t> cost((size_t)g.n, 0);
        for (int32_t u = 0; u < g.n; ++u) {
            for (int64_t k = g.nptr[u]; k < g.nptr[u + 1]; ++k) {
                int32_t v = g.nbr[k];
                if (u < v) cost[u] += (uint64_t)(deg(g, u) + deg(g, v) - 2) + 1;
            }
            total += cost[u];
        }
        uint64_t max_nset = total / (64ull * (uint64_t)threads) + 1, acc = 0;
        for (int32_t u = 0; u < g.n; ++u) {
            acc += cost[u];
            if (acc > max_nset) { cuts.push_back(u + 1); acc = 0; }
        }
        if (cuts.back() != g.n) cuts.push_back(g.n);
    }
    const int nq = (int)cuts.size() - 1;
    std::vector<std::array<u128, 16>> local((size_t)threads);
    std::atomic<int> next{0};
    auto worker = [&](int t) {
        u128* c = local[(size_t)t].data();
        for (int k = 0; k < 16; ++k) c[k] = 0;
        for (;;) {
            int q = next.fetch_add(1);
            if (q >= nq) break;
            census_range(g, cuts[q], cuts[q + 1], c);
        }
    };
    if (threads == 1) {
        worker(0);
    } else {
        std::vector<std::thread> pool;
        for (int t = 0; t < threads; ++t) pool.emplace_back(worker, t);
        for (auto& th : pool) th.join();
    }
    u128 cnt[16] = {0};
    for (int t = 0; t < threads; ++t)
        for (int k = 0; k < 16; ++k) cnt[k] += local[(size_t)t][k];
    close_null(g.n, cnt);
    store(cnt, lo, hi);
}

/* 64-code census (sequential), 128-bit per code; code 0 = C(n,3) minus all
 * others. */
void oracle_census_codes(const void* gp, uint64_t lo[64], uint64_t hi[64]) {
    const OGraph& g = *(const OGraph*)gp;
    u128 c[64] = {0};
    census_codes_range(g, 0, g.n, c);
    u128 sum = 0;
    for (int t = 1; t < 64; ++t) sum += c[t];
    c[0] = choose3(g.n) - sum;
    for (int t = 0; t < 64; ++t) {
        lo[t] = (uint64_t)c[t];
        hi[t] = (uint64_t)(c[t] >> 64);
    }
}

} // extern "C"
