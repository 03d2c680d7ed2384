// Device-wide prefix sums used by the graph build and the census: tiles of
// SCN_TILE items, a sum per tile (k_scn_part), a scan of the tile sums by
// one block (k_scn_top), then each tile rescanned from its offset
// (k_scn_down).  Three launches, no block waits on another.  The items are
// f(i) for a functor f (an array load, or a value computed from an index),
// summed as 64-bit unsigned words and converted to OUT on the way out.
// Each translation unit gets its own copy (anonymous namespace).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

namespace tc {
namespace {

constexpr int SCN_NT = 512;
constexpr int SCN_IT = 8;
constexpr int SCN_TILE = SCN_NT * SCN_IT;

// f(i) = p[i]
template <class T>
struct ScanLoad {
    const T* p;
    __device__ __forceinline__ unsigned long long operator()(int64_t i) const { return (unsigned long long)p[i]; }
};

// A thread's SCN_IT consecutive items from b0: f(i) one by one, or for an
// array in whole 16-byte (or 8-byte) loads when aligned and inside the array.
template <class F>
__device__ __forceinline__ void scn_load(const F& f, int64_t b0, int64_t n, unsigned long long (&v)[SCN_IT]) {
#pragma unroll
    for (int k = 0; k < SCN_IT; ++k) v[k] = b0 + k < n ? f(b0 + k) : 0ull;
}
template <class T>
__device__ __forceinline__ void scn_load(const ScanLoad<T>& f, int64_t b0, int64_t n,
                                         unsigned long long (&v)[SCN_IT]) {
    constexpr int BYTES = (int)sizeof(T) * SCN_IT;
    const T* q = f.p + b0;
    const uintptr_t al = BYTES >= 16 ? 15 : BYTES - 1;
    if (b0 + SCN_IT <= n && (reinterpret_cast<uintptr_t>(q) & al) == 0) {
        T x[SCN_IT];
        if constexpr (BYTES >= 16) {
#pragma unroll
            for (int k = 0; k < BYTES / 16; ++k)
                reinterpret_cast<uint4*>(x)[k] = reinterpret_cast<const uint4*>(q)[k];
        } else if constexpr (BYTES == 8) {
            *reinterpret_cast<uint2*>(x) = *reinterpret_cast<const uint2*>(q);
        } else {
#pragma unroll
            for (int k = 0; k < SCN_IT; ++k) x[k] = q[k];
        }
#pragma unroll
        for (int k = 0; k < SCN_IT; ++k) v[k] = (unsigned long long)x[k];
    } else {
#pragma unroll
        for (int k = 0; k < SCN_IT; ++k) v[k] = b0 + k < n ? (unsigned long long)f.p[b0 + k] : 0ull;
    }
}

// Exclusive block-wide scan of v; *total gets the block's sum.  Begins and
// ends with a barrier.
__device__ __forceinline__ unsigned long long scn_block(unsigned long long v, unsigned long long* wsum,
                                                        unsigned long long* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    __syncthreads();
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < nw ? wsum[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < nw) wsum[lane] = w;
    }
    __syncthreads();
    *total = wsum[nw - 1];
    return inc - v + (warp > 0 ? wsum[warp - 1] : 0ull);
}

template <class F>
__global__ void __launch_bounds__(SCN_NT) k_scn_part(F f, int64_t n, unsigned long long* __restrict__ part) {
    __shared__ unsigned long long wsum[32];
    const int64_t b0 = (int64_t)blockIdx.x * SCN_TILE + (int64_t)threadIdx.x * SCN_IT;
    unsigned long long v[SCN_IT];
    scn_load(f, b0, n, v);
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < SCN_IT; ++k) s += v[k];
    unsigned long long total;
    scn_block(s, wsum, &total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// One block: part[0..np) -> exclusive prefixes, part[np] = the total.
__global__ void __launch_bounds__(SCN_NT) k_scn_top(unsigned long long* __restrict__ part, int64_t np) {
    __shared__ unsigned long long wsum[32];
    unsigned long long carry = 0;
    for (int64_t b = 0; b < np; b += SCN_NT) {
        const int64_t i = b + threadIdx.x;
        const unsigned long long v = i < np ? part[i] : 0ull;
        unsigned long long total;
        const unsigned long long ex = scn_block(v, wsum, &total);
        if (i < np) part[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) part[np] = carry;
}

// out[i] = sum of f(0..i) (INCL) or f(0..i-1); with_total: out[n] = the sum.
template <class F, class OUT, bool INCL>
__global__ void __launch_bounds__(SCN_NT) k_scn_down(F f, int64_t n, const unsigned long long* __restrict__ part,
                                                     int64_t np, OUT* __restrict__ out, bool with_total) {
    __shared__ unsigned long long wsum[32];
    const int64_t b0 = (int64_t)blockIdx.x * SCN_TILE + (int64_t)threadIdx.x * SCN_IT;
    unsigned long long v[SCN_IT];
    scn_load(f, b0, n, v);
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < SCN_IT; ++k) s += v[k];
    unsigned long long total;
    unsigned long long run = part[blockIdx.x] + scn_block(s, wsum, &total);
    OUT o[SCN_IT];
#pragma unroll
    for (int k = 0; k < SCN_IT; ++k) {
        if (INCL) run += v[k];
        o[k] = (OUT)run;
        if (!INCL) run += v[k];
    }
    constexpr int OB = (int)sizeof(OUT) * SCN_IT;
    OUT* q = out + b0;
    if (OB % 16 == 0 && b0 + SCN_IT <= n && (reinterpret_cast<uintptr_t>(q) & 15) == 0) {
#pragma unroll
        for (int k = 0; k < OB / 16; ++k) reinterpret_cast<uint4*>(q)[k] = reinterpret_cast<const uint4*>(o)[k];
    } else {
#pragma unroll
        for (int k = 0; k < SCN_IT; ++k)
            if (b0 + k < n) q[k] = o[k];
    }
    if (with_total && blockIdx.x == 0 && threadIdx.x == 0) out[n] = (OUT)part[np];
}

// Work space (bytes) of a scan of n items.
inline size_t scan_tmp_bytes(int64_t n) {
    return sizeof(unsigned long long) * (size_t)(std::max<int64_t>(1, (n + SCN_TILE - 1) / SCN_TILE) + 1);
}

// out[0..n) = inclusive (INCL) or exclusive prefix sums of f(0..n); with
// with_total, out[n] = the sum (out then has n + 1 items).  tmp holds at
// least scan_tmp_bytes(n) bytes.
template <bool INCL, class F, class OUT>
cudaError_t scan_run(F f, int64_t n, OUT* out, void* tmp, bool with_total, cudaStream_t st) {
    const int64_t np = std::max<int64_t>(1, (n + SCN_TILE - 1) / SCN_TILE);
    unsigned long long* part = static_cast<unsigned long long*>(tmp);
    k_scn_part<F><<<(unsigned)np, SCN_NT, 0, st>>>(f, n, part);
    k_scn_top<<<1, SCN_NT, 0, st>>>(part, np);
    k_scn_down<F, OUT, INCL><<<(unsigned)np, SCN_NT, 0, st>>>(f, n, part, np, out, with_total);
    return cudaGetLastError();
}

}  // namespace
}  // namespace tc
