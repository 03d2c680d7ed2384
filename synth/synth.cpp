/*
 * Seeded synthetic digraph generators.
 *
 * These produce the directed graphs that stand in for the thesis's real
 * datasets (Sec. 4.1: Actors, Patents, Amazon, Slashdot, Google, ... -- sparse,
 * power-law, mean degree ~4-12), which are not available.  The same arc lists
 * feed the CUDA library, the CPU oracle and the benchmark.  Nothing here
 * computes any part of the triad census: the module only draws arcs, removes
 * self-loops and duplicate arcs, adds reciprocal arcs and relabels vertices.
 *
 * Random numbers: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator: the k-th value of stream `key` is mix64(key + (k+1)*GAMMA).  Every
 * draw is addressed by (stream, counter), so results do not depend on the
 * number of host threads.
 *
 * Generators
 *   gnp        directed G(n,p) over ordered pairs (geometric skipping), then each
 *              first-stage arc's reverse added with probability `recip`.
 *   rmat       R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with quadrant
 *              probabilities (a,b,c,1-a-b-c); optional rejection of endpoints
 *              >= n, optional orientation from higher to lower generator id,
 *              reciprocation and a random relabelling of vertex ids.
 *   chung_lu   directed Chung-Lu: tail and head of each arc drawn in proportion
 *              to power-law weights w_i = (i + i0)^(-1/(gamma-1)), i0 chosen so
 *              the largest expected total degree is `max_deg` (Walker/Vose alias
 *              sampling), then reciprocation and relabelling.
 *   batch      many independent graphs of log-uniform size, alternating G(n,p)
 *              and R-MAT, each with its own reciprocity.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <thread>
#include <vector>

namespace {

const uint64_t GAMMA = 0x9E3779B97F4A7C15ull;

inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
inline uint64_t draw(uint64_t key, uint64_t ctr) { return mix64(key + (ctr + 1) * GAMMA); }
inline double u01(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }
inline uint64_t stream(uint64_t seed, uint64_t tag) { return mix64(seed * GAMMA + mix64(tag)); }
inline uint64_t bounded(uint64_t x, uint64_t range) {
    return (uint64_t)(((unsigned __int128)x * range) >> 64);
}

/* stream tags */
enum : uint64_t { T_GNP = 1, T_RECIP = 2, T_RMAT = 3, T_PERM = 4, T_CL = 5, T_BATCH = 6 };

struct Arcs {
    std::vector<int32_t> src, dst;
    std::vector<int64_t> goff; /* graph offsets (batch) */
    std::vector<int32_t> gn;   /* vertex count per graph */
};

int host_threads() {
    unsigned t = std::thread::hardware_concurrency();
    return t == 0 ? 1 : (int)std::min(t, 64u);
}

template <class F>
void parallel_for(int64_t count, F f) {
    int nt = host_threads();
    if (count < 65536 || nt == 1) { f(0, count); return; }
    std::vector<std::thread> pool;
    int64_t chunk = (count + nt - 1) / nt;
    for (int t = 0; t < nt; ++t) {
        int64_t b = t * chunk, e = std::min(count, b + chunk);
        if (b >= e) break;
        pool.emplace_back([=] { f(b, e); });
    }
    for (auto& th : pool) th.join();
}

/* Sorted, duplicate-free arc keys (src<<32 | dst) without self-loops. */
void dedup(std::vector<uint64_t>& keys) {
    keys.erase(std::remove_if(keys.begin(), keys.end(),
                              [](uint64_t k) { return (k >> 32) == (k & 0xffffffffu); }),
               keys.end());
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
}

/* Add the reverse of each arc with probability r, then dedup again. */
void reciprocate(std::vector<uint64_t>& keys, double r, uint64_t key) {
    if (r <= 0) return;
    size_t m = keys.size();
    for (size_t e = 0; e < m; ++e)
        if (u01(draw(key, e)) < r) {
            uint64_t s = keys[e] >> 32, d = keys[e] & 0xffffffffu;
            keys.push_back((d << 32) | s);
        }
    dedup(keys);
}

/* Fisher-Yates relabelling of vertex ids. */
void permute(std::vector<uint64_t>& keys, int64_t n, uint64_t key) {
    std::vector<uint32_t> pi((size_t)n);
    for (int64_t i = 0; i < n; ++i) pi[i] = (uint32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)bounded(draw(key, (uint64_t)i), (uint64_t)i + 1);
        std::swap(pi[i], pi[j]);
    }
    for (auto& k : keys) k = ((uint64_t)pi[k >> 32] << 32) | pi[k & 0xffffffffu];
}

void append(Arcs& out, const std::vector<uint64_t>& keys) {
    size_t base = out.src.size();
    out.src.resize(base + keys.size());
    out.dst.resize(base + keys.size());
    for (size_t i = 0; i < keys.size(); ++i) {
        out.src[base + i] = (int32_t)(keys[i] >> 32);
        out.dst[base + i] = (int32_t)(keys[i] & 0xffffffffu);
    }
}

/* G(n,p) over the n(n-1) ordered pairs, visiting only the chosen pairs by
 * geometric skips (Batagelj & Brandes 2005). */
void gen_gnp(std::vector<uint64_t>& keys, int64_t n, double p, uint64_t key) {
    if (n < 2 || p <= 0) return;
    const uint64_t P = (uint64_t)n * (uint64_t)(n - 1);
    if (p >= 1) {
        for (uint64_t k = 0; k < P; ++k) {
            uint64_t i = k / (uint64_t)(n - 1), r = k % (uint64_t)(n - 1);
            uint64_t j = r < i ? r : r + 1;
            keys.push_back((i << 32) | j);
        }
        return;
    }
    const double lq = std::log1p(-p);
    uint64_t ctr = 0;
    double k = -1;
    for (;;) {
        double u = u01(draw(key, ctr++));
        k += 1 + std::floor(std::log1p(-u) / lq);
        if (k >= (double)P) break;
        uint64_t kk = (uint64_t)k;
        uint64_t i = kk / (uint64_t)(n - 1), r = kk % (uint64_t)(n - 1);
        uint64_t j = r < i ? r : r + 1;
        keys.push_back((i << 32) | j);
    }
}

/* One R-MAT endpoint pair at `scale` levels, from the draw stream of (e, attempt). */
inline void rmat_pair(uint64_t key, uint64_t e, uint64_t attempt, int scale, double a,
                      double ab, double abc, uint64_t& s, uint64_t& d) {
    uint64_t h = mix64(key ^ mix64(e * 64 + attempt));
    s = 0; d = 0;
    for (int l = 0; l < scale; ++l) {
        double r = u01(draw(h, (uint64_t)l));
        uint64_t sb = 0, db = 0;
        if (r < a) {
        } else if (r < ab) {
            db = 1;
        } else if (r < abc) {
            sb = 1;
        } else {
            sb = 1; db = 1;
        }
        s = (s << 1) | sb;
        d = (d << 1) | db;
    }
}

void gen_rmat(std::vector<uint64_t>& keys, int scale, int64_t n, int64_t draws, double a,
              double b, double c, bool orient_down, uint64_t key) {
    size_t base = keys.size();
    keys.resize(base + (size_t)draws);
    const double ab = a + b, abc = a + b + c;
    parallel_for(draws, [&](int64_t lo, int64_t hi) {
        for (int64_t e = lo; e < hi; ++e) {
            uint64_t s = 0, d = 0;
            for (uint64_t att = 0;; ++att) {
                rmat_pair(key, (uint64_t)e, att, scale, a, ab, abc, s, d);
                if ((int64_t)s < n && (int64_t)d < n) break;
            }
            if (orient_down && s < d) std::swap(s, d);
            keys[base + (size_t)e] = (s << 32) | d;
        }
    });
}

/* Walker alias table (Vose's construction) for sampling index i with
 * probability w_i / sum(w). */
struct Alias {
    std::vector<double> prob;
    std::vector<uint32_t> alias;
    explicit Alias(const std::vector<double>& w) {
        size_t n = w.size();
        prob.assign(n, 0);
        alias.assign(n, 0);
        double sum = 0;
        for (double x : w) sum += x;
        std::vector<double> q(n);
        std::vector<uint32_t> small, large;
        for (size_t i = 0; i < n; ++i) {
            q[i] = w[i] * (double)n / sum;
            (q[i] < 1.0 ? small : large).push_back((uint32_t)i);
        }
        while (!small.empty() && !large.empty()) {
            uint32_t s = small.back(); small.pop_back();
            uint32_t l = large.back(); large.pop_back();
            prob[s] = q[s];
            alias[s] = l;
            q[l] = (q[l] + q[s]) - 1.0;
            (q[l] < 1.0 ? small : large).push_back(l);
        }
        for (uint32_t i : large) prob[i] = 1.0;
        for (uint32_t i : small) prob[i] = 1.0;
    }
    uint32_t sample(uint64_t x, uint64_t y) const {
        uint64_t col = bounded(x, prob.size());
        return u01(y) < prob[col] ? (uint32_t)col : alias[col];
    }
};

void gen_chung_lu(std::vector<uint64_t>& keys, int64_t n, double gamma, double mean_total,
                  double max_deg, uint64_t key) {
    const double alpha = 1.0 / (gamma - 1.0);
    const double arcs = 0.5 * mean_total * (double)n;
    /* expected total degree of vertex 0 = 2*arcs*w_0/W; choose i0 by bisection
     * (midpoint-rule W) so that it equals max_deg */
    auto top = [&](double i0) {
        double W = (std::pow(n - 0.5 + i0, 1 - alpha) - std::pow(i0 - 0.5, 1 - alpha)) /
                   (1 - alpha);
        return 2.0 * arcs * std::pow(i0, -alpha) / W;
    };
    double lo = 0.5 + 1e-9, hi = (double)n;
    for (int it = 0; it < 200; ++it) {
        double mid = std::sqrt(lo * hi);
        if (top(mid) > max_deg) lo = mid; else hi = mid;
    }
    const double i0 = hi;
    std::vector<double> w((size_t)n);
    for (int64_t i = 0; i < n; ++i) w[i] = std::pow((double)i + i0, -alpha);
    Alias al(w);
    const int64_t m = (int64_t)std::llround(arcs);
    size_t base = keys.size();
    keys.resize(base + (size_t)m);
    parallel_for(m, [&](int64_t b, int64_t e) {
        for (int64_t k = b; k < e; ++k) {
            uint64_t c = 4 * (uint64_t)k;
            uint64_t s = al.sample(draw(key, c), draw(key, c + 1));
            uint64_t d = al.sample(draw(key, c + 2), draw(key, c + 3));
            keys[base + (size_t)k] = (s << 32) | d;
        }
    });
}

} // namespace

extern "C" {

void* synth_gnp(int32_t n, double p, double recip, uint64_t seed) {
    std::vector<uint64_t> keys;
    gen_gnp(keys, n, p, stream(seed, T_GNP));
    dedup(keys);
    reciprocate(keys, recip, stream(seed, T_RECIP));
    Arcs* a = new Arcs;
    append(*a, keys);
    a->goff = {0, (int64_t)a->src.size()};
    a->gn = {n};
    return a;
}

/* R-MAT with edge_factor * 2^scale draws.  orient_down: every arc from the
 * higher to the lower generator id.  permute: random relabelling at the end. */
void* synth_rmat(int32_t scale, int32_t edge_factor, double a, double b, double c,
                 double recip, int32_t orient_down, int32_t do_permute, uint64_t seed) {
    const int64_t n = (int64_t)1 << scale;
    std::vector<uint64_t> keys;
    gen_rmat(keys, scale, n, (int64_t)edge_factor * n, a, b, c, orient_down != 0,
             stream(seed, T_RMAT));
    dedup(keys);
    reciprocate(keys, recip, stream(seed, T_RECIP));
    if (do_permute) permute(keys, n, stream(seed, T_PERM));
    Arcs* out = new Arcs;
    append(*out, keys);
    out->goff = {0, (int64_t)out->src.size()};
    out->gn = {(int32_t)n};
    return out;
}

void* synth_chung_lu(int32_t n, double gamma, double mean_total_degree, double max_degree,
                     double recip, uint64_t seed) {
    std::vector<uint64_t> keys;
    gen_chung_lu(keys, n, gamma, mean_total_degree, max_degree, stream(seed, T_CL));
    dedup(keys);
    reciprocate(keys, recip, stream(seed, T_RECIP));
    permute(keys, n, stream(seed, T_PERM));
    Arcs* out = new Arcs;
    append(*out, keys);
    out->goff = {0, (int64_t)out->src.size()};
    out->gn = {n};
    return out;
}

/* G independent graphs: n log-uniform in [n_lo, n_hi]; even index G(n,p) with
 * mean out-degree uniform in [deg_lo, deg_hi]; odd index R-MAT with
 * edge_factor*n draws at scale ceil(log2 n) (endpoints >= n redrawn);
 * reciprocity uniform in [0, recip_hi].  Vertex ids are local to each graph. */
void* synth_batch(int32_t G, int32_t n_lo, int32_t n_hi, double deg_lo, double deg_hi,
                  int32_t edge_factor, double recip_hi, uint64_t seed) {
    std::vector<std::vector<uint64_t>> per((size_t)G);
    std::vector<int32_t> ns((size_t)G);
    const uint64_t bkey = stream(seed, T_BATCH);
    for (int32_t g = 0; g < G; ++g) {
        double x = u01(draw(bkey, 4 * (uint64_t)g));
        double nn = std::exp(std::log((double)n_lo) +
                             x * (std::log((double)n_hi) - std::log((double)n_lo)));
        ns[g] = std::max(3, std::min(n_hi, (int32_t)std::floor(nn)));
    }
    auto one = [&](int32_t g) {
        const int64_t n = ns[g];
        const uint64_t gseed = mix64(seed ^ mix64(0x5bd1e995ull + (uint64_t)g));
        const double r = recip_hi * u01(draw(bkey, 4 * (uint64_t)g + 1));
        std::vector<uint64_t>& keys = per[g];
        if ((g & 1) == 0) {
            double deg = deg_lo + (deg_hi - deg_lo) * u01(draw(bkey, 4 * (uint64_t)g + 2));
            gen_gnp(keys, n, std::min(1.0, deg / (double)(n - 1)), stream(gseed, T_GNP));
        } else {
            int scale = 0;
            while (((int64_t)1 << scale) < n) ++scale;
            std::vector<uint64_t> tmp;
            /* serial draws inside one graph; graphs run in parallel below */
            const double a = 0.57, b = 0.19, c = 0.19;
            const uint64_t key = stream(gseed, T_RMAT);
            int64_t draws = (int64_t)edge_factor * n;
            keys.resize((size_t)draws);
            for (int64_t e = 0; e < draws; ++e) {
                uint64_t s = 0, d = 0;
                for (uint64_t att = 0;; ++att) {
                    rmat_pair(key, (uint64_t)e, att, scale, a, a + b, a + b + c, s, d);
                    if ((int64_t)s < n && (int64_t)d < n) break;
                }
                keys[(size_t)e] = (s << 32) | d;
            }
        }
        dedup(keys);
        reciprocate(keys, r, stream(gseed, T_RECIP));
    };
    int nt = host_threads();
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t)
        pool.emplace_back([&, t] {
            for (int32_t g = t; g < G; g += nt) one(g);
        });
    for (auto& th : pool) th.join();
    Arcs* out = new Arcs;
    out->goff.push_back(0);
    size_t total = 0;
    for (auto& k : per) total += k.size();
    out->src.reserve(total);
    out->dst.reserve(total);
    for (int32_t g = 0; g < G; ++g) {
        append(*out, per[g]);
        out->goff.push_back((int64_t)out->src.size());
        std::vector<uint64_t>().swap(per[g]);
    }
    out->gn = ns;
    return out;
}

void synth_size(const void* h, int64_t* m, int32_t* graphs) {
    const Arcs* a = (const Arcs*)h;
    *m = (int64_t)a->src.size();
    *graphs = (int32_t)a->gn.size();
}

void synth_copy(const void* h, int32_t* src, int32_t* dst, int64_t* goff, int32_t* gn) {
    const Arcs* a = (const Arcs*)h;
    std::copy(a->src.begin(), a->src.end(), src);
    std::copy(a->dst.begin(), a->dst.end(), dst);
    std::copy(a->goff.begin(), a->goff.end(), goff);
    std::copy(a->gn.begin(), a->gn.end(), gn);
}

void synth_free(void* h) { delete (Arcs*)h; }

} // extern "C"
