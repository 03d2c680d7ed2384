// tc_graph_build_text: a network file in the Pajek-style text format the
// thesis reads (Sec. 4.2.1 "Implementation details": the order of the graph,
// optional vertex lines with labels, then the arcs of a directed or the
// edges of an undirected graph, told apart by their section keyword; Sec.
// 5.1.1: 0- or 1-based vertex ids) parsed on the device and built into a
// graph (tc_graph_build).
//
// Steps (all on the device except the section table, a handful of lines):
//   1 line starts: a byte after '\n' (or the first byte) starts a line; an
//     exclusive scan of the flags numbers the lines.
//   2 line kinds: header ('*' first), data (anything else but a comment '%'
//     or a blank line); the header lines are compacted and their first bytes
//     read back; the host turns them into sections (keyword, first line).
//   3 arcs per data line (its section decides: 1 per *Arcs line, 2 per
//     *Edges line, one or two per further id of an *Arcslist / *Edgeslist
//     line, none in *Vertices); an exclusive scan gives each line its slot.
//   4 each data line writes its arcs (ids minus the base); tc_graph_build
//     range-checks them.

#include <algorithm>
#include <cctype>
#include <cstring>

#include "scan.cuh"
#include "tc_internal.cuh"

namespace tc {
namespace {

enum SectionKind : int32_t { SEC_VERTICES = 0, SEC_ARCS = 1, SEC_EDGES = 2, SEC_ARCSLIST = 3, SEC_EDGESLIST = 4 };

constexpr int HDR_BYTES = 64;  // bytes of a header line read back to the host

__device__ __forceinline__ bool is_blank(char c) { return c == ' ' || c == '\t' || c == '\r'; }

__global__ void k_line_flags(const char* __restrict__ t, int64_t bytes, int32_t* __restrict__ flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < bytes; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || t[i - 1] == '\n') ? 1 : 0;
}

__global__ void k_line_starts(const int32_t* __restrict__ flag, const int32_t* __restrict__ idx, int64_t bytes,
                              int64_t* __restrict__ start) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < bytes; i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) start[idx[i]] = i;
}

// 1 for a header line ('*' after leading blanks), else 0; data lines are
// told apart later.
__global__ void k_line_headers(const char* __restrict__ t, int64_t bytes, const int64_t* __restrict__ start,
                               int32_t L, int32_t* __restrict__ hdr) {
    for (int32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < L; l += gridDim.x * blockDim.x) {
        int64_t p = start[l];
        while (p < bytes && is_blank(t[p])) ++p;
        hdr[l] = (p < bytes && t[p] == '*') ? 1 : 0;
    }
}

__global__ void k_header_lines(const int32_t* __restrict__ hdr, const int32_t* __restrict__ hidx, int32_t L,
                               const char* __restrict__ t, int64_t bytes, const int64_t* __restrict__ start,
                               int32_t* __restrict__ hline, char* __restrict__ htext) {
    for (int32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < L; l += gridDim.x * blockDim.x) {
        if (!hdr[l]) continue;
        const int32_t k = hidx[l];
        hline[k] = l;
        for (int j = 0; j < HDR_BYTES; ++j) {
            const int64_t p = start[l] + j;
            const char c = p < bytes ? t[p] : '\n';
            htext[(size_t)k * HDR_BYTES + j] = c;
            if (c == '\n') break;
        }
    }
}

// Consume the next whitespace-separated token of the line from p: false at
// the end of the line; else num = its value when it is a decimal integer
// below 2^31, -1 otherwise.
__device__ bool next_token(const char* t, int64_t bytes, int64_t& p, int64_t& num) {
    while (p < bytes && is_blank(t[p])) ++p;
    if (p >= bytes || t[p] == '\n') return false;
    int64_t v = 0;
    bool digits = true;
    int nd = 0;
    while (p < bytes && t[p] != '\n' && !is_blank(t[p])) {
        const char c = t[p];
        if (c >= '0' && c <= '9' && nd < 11) {
            v = v * 10 + (c - '0');
            ++nd;
        } else {
            digits = false;
        }
        ++p;
    }
    num = (digits && nd > 0 && v < ((int64_t)1 << 31)) ? v : -1;
    return true;
}

struct Sections {
    const int32_t* first;  // first line of each section (after its header)
    const int32_t* kind;
    int32_t count;
};

// Section of line l: the last one whose header precedes it (-1: none).
__device__ __forceinline__ int section_of(const Sections& s, int32_t l) {
    int lo = 0, hi = s.count - 1, at = -1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        if (s.first[mid] <= l) {
            at = mid;
            lo = mid + 1;
        } else {
            hi = mid - 1;
        }
    }
    return at;
}

// Arcs of line l (EMIT: also write them from slot off).  Error codes in
// *err: 1 data before any section, 2 a malformed line.
template <bool EMIT>
__global__ void k_line_arcs(const char* __restrict__ t, int64_t bytes, const int64_t* __restrict__ start, int32_t L,
                            Sections sec, int32_t base, int64_t* __restrict__ cnt, const int64_t* __restrict__ off,
                            int32_t* __restrict__ src, int32_t* __restrict__ dst, int* __restrict__ err) {
    for (int32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < L; l += gridDim.x * blockDim.x) {
        int64_t p = start[l];
        while (p < bytes && is_blank(t[p])) ++p;
        int64_t c = 0;
        const bool data = p < bytes && t[p] != '\n' && t[p] != '*' && t[p] != '%';
        if (data) {
            const int s = section_of(sec, l);
            const int kind = s < 0 ? -1 : sec.kind[s];
            if (kind < 0) {
                atomicOr(err, 1);
            } else if (kind == SEC_ARCS || kind == SEC_EDGES) {
                int64_t a = -1, b = -1;
                const bool ok = next_token(t, bytes, p, a) && next_token(t, bytes, p, b) && a >= 0 && b >= 0;
                if (!ok) {
                    atomicOr(err, 2);
                } else {
                    c = kind == SEC_EDGES ? 2 : 1;
                    if (EMIT) {
                        const int64_t o = off[l];
                        src[o] = (int32_t)(a - base);
                        dst[o] = (int32_t)(b - base);
                        if (kind == SEC_EDGES) {
                            src[o + 1] = (int32_t)(b - base);
                            dst[o + 1] = (int32_t)(a - base);
                        }
                    }
                }
            } else if (kind == SEC_ARCSLIST || kind == SEC_EDGESLIST) {
                int64_t a = -1, b = -1;
                if (!next_token(t, bytes, p, a) || a < 0) {
                    atomicOr(err, 2);
                } else {
                    const int per = kind == SEC_EDGESLIST ? 2 : 1;
                    int64_t o = EMIT ? off[l] : 0;
                    while (next_token(t, bytes, p, b)) {
                        if (b < 0) {
                            atomicOr(err, 2);
                            break;
                        }
                        if (EMIT) {
                            src[o] = (int32_t)(a - base);
                            dst[o] = (int32_t)(b - base);
                            if (per == 2) {
                                src[o + 1] = (int32_t)(b - base);
                                dst[o + 1] = (int32_t)(a - base);
                            }
                            o += per;
                        }
                        c += per;
                    }
                }
            }
        }
        if (!EMIT) cnt[l] = c;
    }
}

int grid_of(int64_t work) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t g = (work + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)sms * 16));
}

// Keyword of a header line (case-insensitive), and for *Vertices the order.
bool parse_header(const char* h, int* kind, int64_t* order) {
    int j = 0;
    while (j < HDR_BYTES && (h[j] == ' ' || h[j] == '\t')) ++j;
    if (j >= HDR_BYTES || h[j] != '*') return false;
    ++j;
    char word[16] = {0};
    int w = 0;
    while (j < HDR_BYTES && std::isalpha((unsigned char)h[j]) && w < 15) word[w++] = (char)std::tolower((unsigned char)h[j++]);
    *order = -1;
    if (!std::strcmp(word, "vertices")) {
        *kind = SEC_VERTICES;
        while (j < HDR_BYTES && (h[j] == ' ' || h[j] == '\t')) ++j;
        int64_t v = 0;
        int nd = 0;
        while (j < HDR_BYTES && h[j] >= '0' && h[j] <= '9' && nd < 11) v = v * 10 + (h[j++] - '0'), ++nd;
        if (nd == 0) return false;
        *order = v;
        return true;
    }
    if (!std::strcmp(word, "arcs")) return *kind = SEC_ARCS, true;
    if (!std::strcmp(word, "edges")) return *kind = SEC_EDGES, true;
    if (!std::strcmp(word, "arcslist")) return *kind = SEC_ARCSLIST, true;
    if (!std::strcmp(word, "edgeslist")) return *kind = SEC_EDGESLIST, true;
    *kind = -1;  // *Matrix, *Network, ...: recognised as a header, not supported
    return true;
}

struct Scratch {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit Scratch(cudaStream_t st) : s(st) {}
    template <class T>
    cudaError_t get(T** p, size_t count) {
        void* q = nullptr;
        cudaError_t e = dev_alloc(&q, std::max<size_t>(count, 1) * sizeof(T), s);
        if (e == cudaSuccess) ptrs.push_back(q);
        *p = (T*)q;
        return e;
    }
    ~Scratch() {
        for (void* p : ptrs) dev_free(p, s);
    }
};

template <class T>
tc_status exclusive_scan(Scratch& S, const T* in, T* out, int64_t count, cudaStream_t st) {
    void* tmp = nullptr;
    TC_CUDA(S.get((char**)&tmp, scan_tmp_bytes(count)));
    TC_CUDA(scan_run<false>(ScanLoad<T>{in}, count, out, tmp, false, st));
    return TC_OK;
}

tc_status build_text(const char* text, int64_t bytes, int32_t base, uint32_t flags, cudaStream_t st, tc_graph* out) {
    if (flags & ~TC_DEVICE_PTRS) return fail(TC_ERR_ARG, "graph build (text): unknown flag");
    if (base != 0 && base != 1) return fail(TC_ERR_ARG, "graph build (text): id base must be 0 or 1");
    if (bytes < 0 || (bytes > 0 && !text)) return fail(TC_ERR_ARG, "graph build (text): bad text");
    if (bytes >= ((int64_t)1 << 31) - 1) return fail(TC_ERR_UNSUPPORTED, "graph build (text): text must be < 2 GB");
    if (bytes == 0) return fail(TC_ERR_ARG, "graph build (text): no *Vertices header (the order of the graph)");
    Scratch S(st);
    const char* t = text;
    if (!(flags & TC_DEVICE_PTRS) && bytes > 0) {
        char* d = nullptr;
        TC_CUDA(S.get(&d, (size_t)bytes));
        TC_CUDA(cudaMemcpyAsync(d, text, (size_t)bytes, cudaMemcpyHostToDevice, st));
        t = d;
    }
    // 1 line starts
    int32_t *flag = nullptr, *lidx = nullptr;
    TC_CUDA(S.get(&flag, (size_t)bytes));
    TC_CUDA(S.get(&lidx, (size_t)bytes));
    int32_t L = 0;
    int64_t* start = nullptr;
    if (bytes > 0) {
        k_line_flags<<<grid_of(bytes), 256, 0, st>>>(t, bytes, flag);
        TC_CUDA(cudaGetLastError());
        if (tc_status s = exclusive_scan(S, flag, lidx, bytes, st); s != TC_OK) return s;
        int32_t last[2] = {0, 0};
        TC_CUDA(cudaMemcpyAsync(&last[0], lidx + bytes - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaMemcpyAsync(&last[1], flag + bytes - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
        L = last[0] + last[1];
        TC_CUDA(S.get(&start, (size_t)L));
        k_line_starts<<<grid_of(bytes), 256, 0, st>>>(flag, lidx, bytes, start);
        TC_CUDA(cudaGetLastError());
    }
    // 2 header lines -> sections (host)
    std::vector<int32_t> sec_first, sec_kind;
    int64_t order = -1;
    if (L > 0) {
        int32_t *hdr = nullptr, *hidx = nullptr;
        TC_CUDA(S.get(&hdr, (size_t)L));
        TC_CUDA(S.get(&hidx, (size_t)L));
        k_line_headers<<<grid_of(L), 256, 0, st>>>(t, bytes, start, L, hdr);
        TC_CUDA(cudaGetLastError());
        if (tc_status s = exclusive_scan(S, hdr, hidx, L, st); s != TC_OK) return s;
        int32_t last[2] = {0, 0};
        TC_CUDA(cudaMemcpyAsync(&last[0], hidx + L - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaMemcpyAsync(&last[1], hdr + L - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
        const int32_t H = last[0] + last[1];
        if (H > 0) {
            int32_t* hline = nullptr;
            char* htext = nullptr;
            TC_CUDA(S.get(&hline, (size_t)H));
            TC_CUDA(S.get(&htext, (size_t)H * HDR_BYTES));
            TC_CUDA(cudaMemsetAsync(htext, '\n', (size_t)H * HDR_BYTES, st));
            k_header_lines<<<grid_of(L), 256, 0, st>>>(hdr, hidx, L, t, bytes, start, hline, htext);
            TC_CUDA(cudaGetLastError());
            std::vector<int32_t> hl((size_t)H);
            std::vector<char> ht((size_t)H * HDR_BYTES);
            TC_CUDA(cudaMemcpyAsync(hl.data(), hline, sizeof(int32_t) * (size_t)H, cudaMemcpyDeviceToHost, st));
            TC_CUDA(cudaMemcpyAsync(ht.data(), htext, (size_t)H * HDR_BYTES, cudaMemcpyDeviceToHost, st));
            TC_CUDA(cudaStreamSynchronize(st));
            for (int32_t k = 0; k < H; ++k) {
                int kind = -1;
                int64_t v = -1;
                if (!parse_header(ht.data() + (size_t)k * HDR_BYTES, &kind, &v))
                    return fail(TC_ERR_ARG, "graph build (text): malformed section header");
                if (kind < 0)
                    return fail(TC_ERR_UNSUPPORTED, "graph build (text): only *Vertices, *Arcs, *Edges, *Arcslist "
                                                    "and *Edgeslist sections are read");
                if (kind == SEC_VERTICES) {
                    if (order >= 0) return fail(TC_ERR_ARG, "graph build (text): more than one *Vertices header");
                    order = v;
                }
                sec_first.push_back(hl[(size_t)k] + 1);
                sec_kind.push_back(kind);
            }
        }
    }
    if (order < 0) return fail(TC_ERR_ARG, "graph build (text): no *Vertices header (the order of the graph)");
    if (order >= (1 << 30)) return fail(TC_ERR_UNSUPPORTED, "graph build (text): n must be < 2^30");
    // 3 arcs per line, 4 the arcs
    int32_t *d_first = nullptr, *d_kind = nullptr, *src = nullptr, *dst = nullptr;
    int64_t *cnt = nullptr, *off = nullptr;
    int* err = nullptr;
    const int32_t nsec = (int32_t)sec_first.size();
    TC_CUDA(S.get(&d_first, (size_t)nsec));
    TC_CUDA(S.get(&d_kind, (size_t)nsec));
    TC_CUDA(S.get(&cnt, (size_t)L));
    TC_CUDA(S.get(&off, (size_t)L));
    TC_CUDA(S.get(&err, 1));
    TC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    if (nsec > 0) {
        TC_CUDA(cudaMemcpyAsync(d_first, sec_first.data(), sizeof(int32_t) * (size_t)nsec, cudaMemcpyHostToDevice, st));
        TC_CUDA(cudaMemcpyAsync(d_kind, sec_kind.data(), sizeof(int32_t) * (size_t)nsec, cudaMemcpyHostToDevice, st));
    }
    const Sections sec{d_first, d_kind, nsec};
    int64_t M = 0;
    if (L > 0) {
        k_line_arcs<false><<<grid_of(L), 256, 0, st>>>(t, bytes, start, L, sec, base, cnt, nullptr, nullptr, nullptr,
                                                       err);
        TC_CUDA(cudaGetLastError());
        if (tc_status s = exclusive_scan(S, cnt, off, L, st); s != TC_OK) return s;
        int64_t last[2] = {0, 0};
        int e = 0;
        TC_CUDA(cudaMemcpyAsync(&last[0], off + L - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaMemcpyAsync(&last[1], cnt + L - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
        if (e & 1) return fail(TC_ERR_ARG, "graph build (text): data line before any section header");
        if (e & 2) return fail(TC_ERR_ARG, "graph build (text): malformed arc or edge line");
        M = last[0] + last[1];
        if (M >= ((int64_t)1 << 30)) return fail(TC_ERR_UNSUPPORTED, "graph build (text): more than 2^30 arcs");
        TC_CUDA(S.get(&src, (size_t)M));
        TC_CUDA(S.get(&dst, (size_t)M));
        if (M > 0) {
            k_line_arcs<true><<<grid_of(L), 256, 0, st>>>(t, bytes, start, L, sec, base, cnt, off, src, dst, err);
            TC_CUDA(cudaGetLastError());
        }
    }
    return tc_graph_build((int32_t)order, M ? src : nullptr, M ? dst : nullptr, M, TC_DEVICE_PTRS, st, out);
}

}  // namespace
}  // namespace tc

extern "C" tc_status tc_graph_build_text(const char* text, int64_t bytes, int32_t id_base, uint32_t flags,
                                         void* stream, tc_graph* out) {
    if (!out) return tc::fail(TC_ERR_ARG, "tc_graph_build_text: out is null");
    *out = nullptr;
    try {
        return tc::build_text(text, bytes, id_base, flags, (cudaStream_t)stream, out);
    } catch (const std::bad_alloc&) {
        return tc::fail(TC_ERR_OOM, "tc_graph_build_text: host allocation failed");
    } catch (...) {
        return tc::fail(TC_ERR_CUDA, "tc_graph_build_text: unexpected exception");
    }
}
