// Learned cost model for task binning: an 8-32-32-4 MLP (ReLU) that predicts
// log2 of the cycles a canonical-dyad task takes in each of the four bins,
// trained on timings the census records (tc_cost_sample).  Training runs in
// FP32 kernels (forward, backward, Adam); binning runs the network in FP16.
// The thesis bins tasks by the degree sum |N(u)|+|N(v)|-2 (Sec. 4.3.1); that
// heuristic stays the fallback when no model is installed.
#include <cstring>
#include <cmath>
#include <mutex>
#include <vector>

#include <algorithm>

#include "mlp.cuh"
#include "tc_internal.cuh"

namespace tc {
namespace {

// ------------------------------------------------------------- features --
__global__ void k_features(const int32_t* __restrict__ deg, const int32_t* __restrict__ vtag,
                           const int32_t* __restrict__ uv, int32_t n, int64_t total_rows,
                           float* __restrict__ feat, int* __restrict__ err) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int64_t u = uv[2 * i], v = uv[2 * i + 1];
        float f[MLP_IN];
        if (u < 0 || u >= total_rows || v < 0 || v >= total_rows) {
            atomicOr(err, 1);
            for (int k = 0; k < MLP_IN; ++k) f[k] = 0.0f;
        } else {
            task_features_uv(u, v, deg, vtag, f);
        }
        for (int k = 0; k < MLP_IN; ++k) feat[(size_t)i * MLP_IN + k] = f[k];
    }
}

// |S| = |N(u) u N(v) \ {u, v}| of pairs of vertices of one graph each (the
// graph's global rows [voff[g], voff[g+1]), local ids = row - voff[g]): the
// exact task cost of Sec. 4.3.1 (workload W3).
// One warp per pair: lanes take the shorter list's entries in turn and
// binary-search them in the longer one; |S| = d_u + d_v - |common| - 2 when
// u and v are adjacent (each list then holds the other endpoint).

__global__ void k_union_sizes(const int64_t* __restrict__ row_ptr, const uint32_t* __restrict__ adj,
                              const int64_t* __restrict__ voff, int G, const int32_t* __restrict__ uv, int32_t n,
                              int32_t* __restrict__ out, int* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const int64_t u = uv[2 * i], v = uv[2 * i + 1];
        int lo_g = 0, hi_g = G - 1;  // graph of u: last g with voff[g] <= u
        while (lo_g < hi_g) {
            const int mid = (lo_g + hi_g + 1) >> 1;
            if (voff[mid] <= u) lo_g = mid;
            else hi_g = mid - 1;
        }
        const int64_t r0 = voff[lo_g], r1 = voff[lo_g + 1];
        if (u < r0 || u >= r1 || v < r0 || v >= r1) {
            if (lane == 0) {
                atomicOr(err, 1);
                out[i] = 0;
            }
            continue;
        }
        const int64_t ub = row_ptr[u], vb = row_ptr[v];
        const int du = (int)(row_ptr[u + 1] - ub), dv = (int)(row_ptr[v + 1] - vb);
        const bool u_short = du <= dv;
        const uint32_t* sl = adj + (u_short ? ub : vb);
        const uint32_t* gl = adj + (u_short ? vb : ub);
        const int ns = u_short ? du : dv, ng = u_short ? dv : du;
        int common = 0;
        for (int k = lane; k < ns; k += 32) common += list_has(gl, ng, sl[k] >> 2) ? 1 : 0;
        for (int o = 16; o > 0; o >>= 1) common += __shfl_xor_sync(0xffffffffu, common, o);
        if (lane == 0) {
            const bool adjacent = u != v && list_has(adj + ub, du, (uint32_t)(v - r0));
            out[i] = du + dv - common - (adjacent ? 2 : 0);
        }
    }
}

// ------------------------------------------------------- FP32 training --
// Sample b of the batch is sample idx(b) of the data set: all samples in
// order when the batch is the whole set (step < 0), else a SplitMix64 draw.
__device__ __forceinline__ int32_t batch_index(uint64_t seed, int64_t step, int b, int32_t n, int32_t nb) {
    if (step < 0) return b;
    uint64_t z = seed + ((uint64_t)step * (uint64_t)nb + (uint64_t)b + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (int32_t)(((unsigned __int128)z * (uint64_t)n) >> 64);
}

// Forward and backward of one sample per thread.  Loss of a sample: half the
// squared error of the head of the bin it was measured in, averaged over the
// batch.  Stores the batch's inputs, activations and pre-activation gradients
// for the weight-gradient kernel, and a per-block partial loss.
__global__ void __launch_bounds__(128) k_mlp_fwd_bwd(const float* __restrict__ prm, const float* __restrict__ feat,
                                                     const int32_t* __restrict__ bin,
                                                     const float* __restrict__ target, int32_t n, int32_t nb,
                                                     uint64_t seed, int64_t step, float* __restrict__ X,
                                                     float* __restrict__ H1, float* __restrict__ H2,
                                                     float* __restrict__ D1, float* __restrict__ D2,
                                                     float* __restrict__ D3, double* __restrict__ loss_part) {
    __shared__ float w[MLP_NPARAM];
    __shared__ double red[128];
    for (int k = threadIdx.x; k < MLP_NPARAM; k += blockDim.x) w[k] = prm[k];
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (b < nb) {
        const int32_t s = batch_index(seed, step, b, n, nb);
        float x[MLP_IN], z1[MLP_H], h1[MLP_H], z2[MLP_H], h2[MLP_H], o[MLP_OUT];
        for (int i = 0; i < MLP_IN; ++i) x[i] = feat[(size_t)s * MLP_IN + i];
        for (int j = 0; j < MLP_H; ++j) {
            float a = w[MLP_B1 + j];
            for (int i = 0; i < MLP_IN; ++i) a += w[MLP_W1 + j * MLP_IN + i] * x[i];
            z1[j] = a;
            h1[j] = a > 0.0f ? a : 0.0f;
        }
        for (int j = 0; j < MLP_H; ++j) {
            float a = w[MLP_B2 + j];
            for (int i = 0; i < MLP_H; ++i) a += w[MLP_W2 + j * MLP_H + i] * h1[i];
            z2[j] = a;
            h2[j] = a > 0.0f ? a : 0.0f;
        }
        for (int k = 0; k < MLP_OUT; ++k) {
            float a = w[MLP_B3 + k];
            for (int i = 0; i < MLP_H; ++i) a += w[MLP_W3 + k * MLP_H + i] * h2[i];
            o[k] = a;
        }
        const int t = bin[s];
        float d3[MLP_OUT];
        for (int k = 0; k < MLP_OUT; ++k) d3[k] = 0.0f;
        const float err = o[t] - target[s];
        d3[t] = err / (float)nb;
        l = 0.5 * (double)err * (double)err / (double)nb;
        float d2[MLP_H], d1[MLP_H];
        for (int i = 0; i < MLP_H; ++i) {
            float a = 0.0f;
            for (int k = 0; k < MLP_OUT; ++k) a += w[MLP_W3 + k * MLP_H + i] * d3[k];
            d2[i] = z2[i] > 0.0f ? a : 0.0f;
        }
        for (int i = 0; i < MLP_H; ++i) {
            float a = 0.0f;
            for (int j = 0; j < MLP_H; ++j) a += w[MLP_W2 + j * MLP_H + i] * d2[j];
            d1[i] = z1[i] > 0.0f ? a : 0.0f;
        }
        for (int i = 0; i < MLP_IN; ++i) X[(size_t)b * MLP_IN + i] = x[i];
        for (int j = 0; j < MLP_H; ++j) {
            H1[(size_t)b * MLP_H + j] = h1[j];
            H2[(size_t)b * MLP_H + j] = h2[j];
            D1[(size_t)b * MLP_H + j] = d1[j];
            D2[(size_t)b * MLP_H + j] = d2[j];
        }
        for (int k = 0; k < MLP_OUT; ++k) D3[(size_t)b * MLP_OUT + k] = d3[k];
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

// One thread per parameter: its gradient summed over the batch in a fixed
// order (no atomics, so the result is deterministic).
__global__ void k_mlp_wgrad(int32_t nb, const float* __restrict__ X, const float* __restrict__ H1,
                            const float* __restrict__ H2, const float* __restrict__ D1,
                            const float* __restrict__ D2, const float* __restrict__ D3,
                            float* __restrict__ grad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= MLP_NPARAM) return;
    const float *A, *B;
    int sa, sb, ia, ib;
    if (p < MLP_B1) {
        A = D1; sa = MLP_H; ia = (p - MLP_W1) / MLP_IN; B = X; sb = MLP_IN; ib = (p - MLP_W1) % MLP_IN;
    } else if (p < MLP_W2) {
        A = D1; sa = MLP_H; ia = p - MLP_B1; B = nullptr; sb = 0; ib = 0;
    } else if (p < MLP_B2) {
        A = D2; sa = MLP_H; ia = (p - MLP_W2) / MLP_H; B = H1; sb = MLP_H; ib = (p - MLP_W2) % MLP_H;
    } else if (p < MLP_W3) {
        A = D2; sa = MLP_H; ia = p - MLP_B2; B = nullptr; sb = 0; ib = 0;
    } else if (p < MLP_B3) {
        A = D3; sa = MLP_OUT; ia = (p - MLP_W3) / MLP_H; B = H2; sb = MLP_H; ib = (p - MLP_W3) % MLP_H;
    } else {
        A = D3; sa = MLP_OUT; ia = p - MLP_B3; B = nullptr; sb = 0; ib = 0;
    }
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) {
        const float a = A[(size_t)b * sa + ia];
        acc += B ? (double)a * (double)B[(size_t)b * sb + ib] : (double)a;
    }
    grad[p] = (float)acc;
}

__global__ void k_sum_loss(const double* __restrict__ part, int np, float* __restrict__ loss) {
    double s = 0.0;
    for (int i = 0; i < np; ++i) s += part[i];
    *loss = (float)s;
}

__global__ void k_adam(float* __restrict__ prm, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, int64_t t) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= MLP_NPARAM) return;
    const float g = grad[p];
    const float mm = b1 * m[p] + (1.0f - b1) * g;
    const float vv = b2 * v[p] + (1.0f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float mh = mm / (1.0f - powf(b1, (float)t));
    const float vh = vv / (1.0f - powf(b2, (float)t));
    prm[p] -= lr * mh / (sqrtf(vh) + eps);
}

// ------------------------------------------------------------ prediction --
__global__ void k_mlp_predict32(const float* __restrict__ prm, const float* __restrict__ feat, int32_t n,
                                float* __restrict__ out) {
    __shared__ float w[MLP_NPARAM];
    for (int k = threadIdx.x; k < MLP_NPARAM; k += blockDim.x) w[k] = prm[k];
    __syncthreads();
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        float h1[MLP_H], h2[MLP_H];
        for (int j = 0; j < MLP_H; ++j) {
            float a = w[MLP_B1 + j];
            for (int i = 0; i < MLP_IN; ++i) a += w[MLP_W1 + j * MLP_IN + i] * feat[(size_t)s * MLP_IN + i];
            h1[j] = a > 0.0f ? a : 0.0f;
        }
        for (int j = 0; j < MLP_H; ++j) {
            float a = w[MLP_B2 + j];
            for (int i = 0; i < MLP_H; ++i) a += w[MLP_W2 + j * MLP_H + i] * h1[i];
            h2[j] = a > 0.0f ? a : 0.0f;
        }
        for (int k = 0; k < MLP_OUT; ++k) {
            float a = w[MLP_B3 + k];
            for (int i = 0; i < MLP_H; ++i) a += w[MLP_W3 + k * MLP_H + i] * h2[i];
            out[(size_t)s * MLP_OUT + k] = a;
        }
    }
}

__global__ void k_mlp_predict16(const __half2* __restrict__ packed, const float* __restrict__ feat, int32_t n,
                                float* __restrict__ out) {
    __shared__ __align__(16) __half2 P[MLPH_N + 2];
    for (int k = threadIdx.x; k < MLPH_N; k += blockDim.x) P[k] = packed[k];
    __syncthreads();
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // one sample per thread
    if (s < n) {
        float x[MLP_IN], o[MLP_OUT];
        for (int i = 0; i < MLP_IN; ++i) x[i] = feat[(size_t)s * MLP_IN + i];
        mlp_predict_h(P, x, o);
        for (int k = 0; k < MLP_OUT; ++k) out[(size_t)s * MLP_OUT + k] = o[k];
    }
}

// FP32 parameters -> packed FP16 pairs (host side).
void pack_half(const float* prm, std::vector<__half2>& P) {
    P.assign(MLPH_N, __floats2half2_rn(0.0f, 0.0f));
    for (int p = 0; p < MLP_H / 2; ++p) {
        for (int i = 0; i < MLP_IN; ++i)
            P[MLPH_L1 + p * MLP_IN + i] = __floats2half2_rn(prm[MLP_W1 + 2 * p * MLP_IN + i],
                                                             prm[MLP_W1 + (2 * p + 1) * MLP_IN + i]);
        P[MLPH_B1 + p] = __floats2half2_rn(prm[MLP_B1 + 2 * p], prm[MLP_B1 + 2 * p + 1]);
        for (int i = 0; i < MLP_H; ++i)
            P[MLPH_L2 + p * MLP_H + i] = __floats2half2_rn(prm[MLP_W2 + 2 * p * MLP_H + i],
                                                            prm[MLP_W2 + (2 * p + 1) * MLP_H + i]);
        P[MLPH_B2 + p] = __floats2half2_rn(prm[MLP_B2 + 2 * p], prm[MLP_B2 + 2 * p + 1]);
    }
    for (int p = 0; p < MLP_OUT / 2; ++p) {
        for (int i = 0; i < MLP_H; ++i)
            P[MLPH_L3 + p * MLP_H + i] = __floats2half2_rn(prm[MLP_W3 + 2 * p * MLP_H + i],
                                                            prm[MLP_W3 + (2 * p + 1) * MLP_H + i]);
        P[MLPH_B3 + p] = __floats2half2_rn(prm[MLP_B3 + 2 * p], prm[MLP_B3 + 2 * p + 1]);
    }
}

std::mutex g_model_mu;
__half2* g_model[64];  // installed packed weights per device (library-owned)

__half2* g_path_model[64];  // installed path-routing model per device (library-owned)

// Routing features of one graph (host, from its build statistics), the
// inputs of the path model: log2(1+n)/32, log2(1+dyads)/32,
// log2(1+mean degree)/8, log2(1+max degree)/20, log2(max/mean degree)/8,
// log2(1+merged entries/dyads)/20, mutual fraction, log2(1+merged)/40.
void path_features(const tc_graph_stats_t& s, float f[MLP_IN]) {
    const double n = (double)s.n, dy = (double)s.dyads, mean = n > 0 ? 2.0 * dy / n : 0.0;
    const double mx = (double)s.max_degree, merged = (double)s.merged_entries;
    f[0] = (float)(std::log2(1.0 + n) / 32.0);
    f[1] = (float)(std::log2(1.0 + dy) / 32.0);
    f[2] = (float)(std::log2(1.0 + mean) / 8.0);
    f[3] = (float)(std::log2(1.0 + mx) / 20.0);
    f[4] = (float)(mean > 0 ? std::log2(std::max(1.0, mx / mean)) / 8.0 : 0.0);
    f[5] = (float)(std::log2(1.0 + merged / std::max(1.0, dy)) / 20.0);
    f[6] = (float)(dy > 0 ? (double)s.mutual / dy : 0.0);
    f[7] = (float)(std::log2(1.0 + merged) / 40.0);
}

// The degree-skew rule: the forward path when the largest degree is at
// least PATH_SKEW times the mean degree (hubs: the forward lists stay short
// and the merge path's hub dyads are long), else the merge path.
constexpr double PATH_SKEW = 8.0;

tc_status path_route_impl(const GraphSet& set, const std::vector<int32_t>& gidx, std::vector<uint8_t>& merge,
                          cudaStream_t st) {
    const size_t G = gidx.size();
    merge.assign(G, 0);
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    __half2* model = (dev >= 0 && dev < 64) ? g_path_model[dev] : nullptr;
    if (!model) {
        for (size_t i = 0; i < G; ++i) {
            const tc_graph_stats_t& s = set.stats[(size_t)gidx[i]];
            const double mean = s.n > 0 ? 2.0 * (double)s.dyads / (double)s.n : 0.0;
            merge[i] = (double)s.max_degree < PATH_SKEW * mean ? 1 : 0;
        }
        return TC_OK;
    }
    // the installed network, FP16 as in binning: output 0 = log2 cost of the
    // forward path, 1 = of the merge path
    std::vector<float> f(G * MLP_IN), o(G * MLP_OUT);
    for (size_t i = 0; i < G; ++i) path_features(set.stats[(size_t)gidx[i]], f.data() + i * MLP_IN);
    float* d = nullptr;
    TC_CUDA(dev_alloc((void**)&d, sizeof(float) * G * (MLP_IN + MLP_OUT), st));
    cudaError_t e = cudaMemcpyAsync(d, f.data(), sizeof(float) * G * MLP_IN, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        k_mlp_predict16<<<(int)((G + 255) / 256), 256, 0, st>>>(model, d, (int32_t)G, d + G * MLP_IN);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(o.data(), d + G * MLP_IN, sizeof(float) * G * MLP_OUT, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(d, st);
    if (e != cudaSuccess) return cuda_fail(e, "path model inference", __FILE__, __LINE__);
    for (size_t i = 0; i < G; ++i) merge[i] = o[i * MLP_OUT + 1] < o[i * MLP_OUT + 0] ? 1 : 0;
    return TC_OK;
}

struct TrainBuffers {
    float *X = nullptr, *H1 = nullptr, *H2 = nullptr, *D1 = nullptr, *D2 = nullptr, *D3 = nullptr;
    double* part = nullptr;
    cudaStream_t st;
    ~TrainBuffers() {
        dev_free(X, st);
        dev_free(H1, st);
        dev_free(H2, st);
        dev_free(D1, st);
        dev_free(D2, st);
        dev_free(D3, st);
        dev_free(part, st);
    }
};

tc_status alloc_train(TrainBuffers& B, int32_t nb, cudaStream_t st) {
    B.st = st;
    const size_t n = (size_t)nb;
    TC_CUDA(dev_alloc((void**)&B.X, sizeof(float) * n * MLP_IN, st));
    TC_CUDA(dev_alloc((void**)&B.H1, sizeof(float) * n * MLP_H, st));
    TC_CUDA(dev_alloc((void**)&B.H2, sizeof(float) * n * MLP_H, st));
    TC_CUDA(dev_alloc((void**)&B.D1, sizeof(float) * n * MLP_H, st));
    TC_CUDA(dev_alloc((void**)&B.D2, sizeof(float) * n * MLP_H, st));
    TC_CUDA(dev_alloc((void**)&B.D3, sizeof(float) * n * MLP_OUT, st));
    TC_CUDA(dev_alloc((void**)&B.part, sizeof(double) * (n / 128 + 1), st));
    return TC_OK;
}

tc_status grad_step(const float* prm, const float* feat, const int32_t* bin, const float* target, int32_t n,
                    int32_t nb, uint64_t seed, int64_t step, TrainBuffers& B, float* grad, float* loss,
                    cudaStream_t st) {
    const int blocks = (nb + 127) / 128;
    k_mlp_fwd_bwd<<<blocks, 128, 0, st>>>(prm, feat, bin, target, n, nb, seed, step, B.X, B.H1, B.H2, B.D1, B.D2,
                                         B.D3, B.part);
    TC_CUDA(cudaGetLastError());
    k_mlp_wgrad<<<(MLP_NPARAM + 127) / 128, 128, 0, st>>>(nb, B.X, B.H1, B.H2, B.D1, B.D2, B.D3, grad);
    TC_CUDA(cudaGetLastError());
    if (loss) {
        k_sum_loss<<<1, 1, 0, st>>>(B.part, blocks, loss);
        TC_CUDA(cudaGetLastError());
    }
    return TC_OK;
}

}  // namespace

tc_status path_route(const GraphSet& set, const std::vector<int32_t>& gidx, std::vector<uint8_t>& merge,
                     cudaStream_t st) {
    return path_route_impl(set, gidx, merge, st);
}

// Installed FP16 weights of the current device, or nullptr.
const void* cost_model_weights() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_model_mu);
    return g_model[dev];
}

}  // namespace tc

extern "C" {

tc_status tc_cost_features(tc_graph g, const int32_t* uv, int32_t n, float* feat, void* stream) {
    if (!g || n < 0 || (n > 0 && (!uv || !feat))) return tc::fail(TC_ERR_ARG, "tc_cost_features: bad arguments");
    if (n == 0) return TC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int* err = nullptr;
    TC_CUDA(tc::dev_alloc((void**)&err, sizeof(int), st));
    TC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    const tc::GraphSet& s = *g->set;
    tc::k_features<<<(n + 255) / 256, 256, 0, st>>>(s.deg, s.vtag, uv, n, s.total_n, feat, err);
    TC_CUDA(cudaGetLastError());
    int h = 0;
    TC_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    tc::dev_free(err, st);
    if (h) return tc::fail(TC_ERR_ID_RANGE, "tc_cost_features: a vertex outside the graph set");
    return TC_OK;
}

tc_status tc_union_sizes(tc_graph g, const int32_t* uv, int32_t n, int32_t* out, void* stream) {
    if (!g || n < 0 || (n > 0 && (!uv || !out))) return tc::fail(TC_ERR_ARG, "tc_union_sizes: bad arguments");
    if (n == 0) return TC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int* err = nullptr;
    TC_CUDA(tc::dev_alloc((void**)&err, sizeof(int), st));
    TC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    const tc::GraphSet& s = *g->set;
    int64_t* voff = nullptr;
    TC_CUDA(tc::dev_alloc((void**)&voff, sizeof(int64_t) * s.voff.size(), st));
    TC_CUDA(cudaMemcpyAsync(voff, s.voff.data(), sizeof(int64_t) * s.voff.size(), cudaMemcpyHostToDevice, st));
    tc::k_union_sizes<<<(int)std::min<int64_t>(((int64_t)n + 7) / 8, 1 << 20), 256, 0, st>>>(
        s.row_ptr, s.adj, voff, (int)s.G, uv, n, out, err);
    TC_CUDA(cudaGetLastError());
    int h = 0;
    TC_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TC_CUDA(cudaStreamSynchronize(st));
    tc::dev_free(err, st);
    tc::dev_free(voff, st);
    if (h) return tc::fail(TC_ERR_ID_RANGE, "tc_union_sizes: a pair not within one graph of the build");
    return TC_OK;
}

tc_status tc_mlp_loss_grad(const float* params, const float* feat, const int32_t* bin, const float* target,
                           int32_t n, float* grad, float* loss, void* stream) {
    if (!params || !feat || !bin || !target || !grad || n < 1)
        return tc::fail(TC_ERR_ARG, "tc_mlp_loss_grad: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    tc::TrainBuffers B;
    if (tc_status s = tc::alloc_train(B, n, st); s != TC_OK) return s;
    if (tc_status s = tc::grad_step(params, feat, bin, target, n, n, 0, -1, B, grad, loss, st); s != TC_OK)
        return s;
    TC_CUDA(cudaStreamSynchronize(st));
    return TC_OK;
}

tc_status tc_mlp_train(float* params, const float* feat, const int32_t* bin, const float* target, int32_t n,
                       int32_t steps, int32_t batch, float lr, uint64_t seed, float* loss, void* stream) {
    if (!params || !feat || !bin || !target || n < 1 || steps < 0 || batch < 1 || !(lr > 0))
        return tc::fail(TC_ERR_ARG, "tc_mlp_train: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    tc::TrainBuffers B;
    if (tc_status s = tc::alloc_train(B, batch, st); s != TC_OK) return s;
    float *grad = nullptr, *m = nullptr, *v = nullptr;
    TC_CUDA(tc::dev_alloc((void**)&grad, sizeof(float) * tc::MLP_NPARAM, st));
    TC_CUDA(tc::dev_alloc((void**)&m, sizeof(float) * tc::MLP_NPARAM, st));
    TC_CUDA(tc::dev_alloc((void**)&v, sizeof(float) * tc::MLP_NPARAM, st));
    TC_CUDA(cudaMemsetAsync(m, 0, sizeof(float) * tc::MLP_NPARAM, st));
    TC_CUDA(cudaMemsetAsync(v, 0, sizeof(float) * tc::MLP_NPARAM, st));
    for (int32_t t = 0; t < steps; ++t) {
        if (tc_status s = tc::grad_step(params, feat, bin, target, n, batch, seed, t, B, grad, nullptr, st);
            s != TC_OK)
            return s;
        tc::k_adam<<<(tc::MLP_NPARAM + 127) / 128, 128, 0, st>>>(params, grad, m, v, lr, 0.9f, 0.999f, 1e-8f,
                                                                 (int64_t)t + 1);
        TC_CUDA(cudaGetLastError());
    }
    if (loss) {  // loss over the whole data set after training
        tc::TrainBuffers F;
        if (tc_status s = tc::alloc_train(F, n, st); s != TC_OK) return s;
        if (tc_status s = tc::grad_step(params, feat, bin, target, n, n, 0, -1, F, grad, loss, st); s != TC_OK)
            return s;
        TC_CUDA(cudaStreamSynchronize(st));
    }
    tc::dev_free(grad, st);
    tc::dev_free(m, st);
    tc::dev_free(v, st);
    TC_CUDA(cudaStreamSynchronize(st));
    return TC_OK;
}

tc_status tc_mlp_predict(const float* params, const float* feat, int32_t n, int32_t half_precision, float* out,
                         void* stream) {
    if (!params || !feat || !out || n < 0) return tc::fail(TC_ERR_ARG, "tc_mlp_predict: bad arguments");
    if (n == 0) return TC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    if (half_precision) {
        std::vector<float> h(tc::MLP_NPARAM);
        TC_CUDA(cudaMemcpyAsync(h.data(), params, sizeof(float) * tc::MLP_NPARAM, cudaMemcpyDeviceToHost, st));
        TC_CUDA(cudaStreamSynchronize(st));
        std::vector<__half2> P;
        tc::pack_half(h.data(), P);
        __half2* d = nullptr;
        TC_CUDA(tc::dev_alloc((void**)&d, sizeof(__half2) * P.size(), st));
        TC_CUDA(cudaMemcpyAsync(d, P.data(), sizeof(__half2) * P.size(), cudaMemcpyHostToDevice, st));
        tc::k_mlp_predict16<<<(n + 255) / 256, 256, 0, st>>>(d, feat, n, out);
        TC_CUDA(cudaGetLastError());
        TC_CUDA(cudaStreamSynchronize(st));
        tc::dev_free(d, st);
    } else {
        tc::k_mlp_predict32<<<blocks, 256, 0, st>>>(params, feat, n, out);
        TC_CUDA(cudaGetLastError());
        TC_CUDA(cudaStreamSynchronize(st));
    }
    return TC_OK;
}

tc_status tc_cost_model_load(const float* params) {
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return tc::fail(TC_ERR_UNSUPPORTED, "tc_cost_model_load: device index >= 64");
    std::lock_guard<std::mutex> lk(tc::g_model_mu);
    if (!params) {  // uninstall: binning falls back to the degree-sum heuristic
        if (tc::g_model[dev]) {
            TC_CUDA(cudaDeviceSynchronize());
            TC_CUDA(cudaFree(tc::g_model[dev]));
            tc::g_model[dev] = nullptr;
        }
        return TC_OK;
    }
    std::vector<__half2> P;
    tc::pack_half(params, P);
    if (!tc::g_model[dev]) TC_CUDA(cudaMalloc((void**)&tc::g_model[dev], sizeof(__half2) * tc::MLPH_N));
    TC_CUDA(cudaMemcpy(tc::g_model[dev], P.data(), sizeof(__half2) * P.size(), cudaMemcpyHostToDevice));
    return TC_OK;
}

tc_status tc_path_features(int32_t G, const tc_graph* gs, float* feat) {
    if (G < 0 || (G > 0 && (!gs || !feat))) return tc::fail(TC_ERR_ARG, "tc_path_features: bad arguments");
    for (int32_t i = 0; i < G; ++i) {
        if (!gs[i]) return tc::fail(TC_ERR_ARG, "tc_path_features: null handle");
        tc::path_features(gs[i]->set->stats[(size_t)gs[i]->index], feat + (size_t)i * tc::MLP_IN);
    }
    return TC_OK;
}

tc_status tc_path_model_load(const float* params) {
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return tc::fail(TC_ERR_UNSUPPORTED, "tc_path_model_load: device index >= 64");
    std::lock_guard<std::mutex> lk(tc::g_model_mu);
    if (!params) {  // uninstall: routing falls back to the degree-skew rule
        if (tc::g_path_model[dev]) {
            TC_CUDA(cudaDeviceSynchronize());
            TC_CUDA(cudaFree(tc::g_path_model[dev]));
            tc::g_path_model[dev] = nullptr;
        }
        return TC_OK;
    }
    std::vector<__half2> P;
    tc::pack_half(params, P);
    if (!tc::g_path_model[dev]) TC_CUDA(cudaMalloc((void**)&tc::g_path_model[dev], sizeof(__half2) * tc::MLPH_N));
    TC_CUDA(cudaMemcpy(tc::g_path_model[dev], P.data(), sizeof(__half2) * P.size(), cudaMemcpyHostToDevice));
    return TC_OK;
}

tc_status tc_path_route(int32_t G, const tc_graph* gs, int32_t* path, void* stream) {
    if (G < 0 || (G > 0 && (!gs || !path))) return tc::fail(TC_ERR_ARG, "tc_path_route: bad arguments");
    if (G == 0) return TC_OK;
    for (int32_t i = 0; i < G; ++i) {
        if (!gs[i]) return tc::fail(TC_ERR_ARG, "tc_path_route: null handle");
        if (gs[i]->set != gs[0]->set) return tc::fail(TC_ERR_UNSUPPORTED, "tc_path_route: handles of different builds");
    }
    std::vector<int32_t> idx((size_t)G);
    for (int32_t i = 0; i < G; ++i) idx[(size_t)i] = gs[i]->index;
    std::vector<uint8_t> merge;
    try {
        if (tc_status s = tc::path_route(*gs[0]->set, idx, merge, (cudaStream_t)stream); s != TC_OK) return s;
    } catch (...) {
        return tc::fail(TC_ERR_CUDA, "tc_path_route: unexpected exception");
    }
    for (int32_t i = 0; i < G; ++i) path[i] = merge[(size_t)i] ? TC_TRI_MERGE : TC_TRI_FORWARD;
    return TC_OK;
}

}  // extern "C"
