// Cost model shared by the census (FP16 inference in task binning) and the
// training kernels: features of a canonical-dyad task and the 8-32-32-4 MLP.
#pragma once

#include <cuda_fp16.h>

#include <cstdint>

namespace tc {

constexpr int MLP_IN = 8;
constexpr int MLP_H = 32;
constexpr int MLP_OUT = 4;  // predicted log2(cycles) of the task in bins 0..3
// parameter layout (floats): W1[H][IN] b1[H] W2[H][H] b2[H] W3[OUT][H] b3[OUT]
constexpr int MLP_W1 = 0;
constexpr int MLP_B1 = MLP_W1 + MLP_H * MLP_IN;
constexpr int MLP_W2 = MLP_B1 + MLP_H;
constexpr int MLP_B2 = MLP_W2 + MLP_H * MLP_H;
constexpr int MLP_W3 = MLP_B2 + MLP_H;
constexpr int MLP_B3 = MLP_W3 + MLP_OUT * MLP_H;
constexpr int MLP_NPARAM = MLP_B3 + MLP_OUT;  // 1476

// Features of task <u,v> from the undirected degrees and the per-vertex tag
// counts (out-only, in-only, mutual neighbours), ordered shorter list first:
// log2 sizes scaled by 1/20, their difference, and tag fractions.
__device__ __forceinline__ void task_features(int ds, int dg, const int32_t* ts, const int32_t* tg,
                                              float f[MLP_IN]) {
    const float ls = log2f(1.0f + (float)ds), lg = log2f(1.0f + (float)dg);
    const float is = ds > 0 ? 1.0f / (float)ds : 0.0f, ig = dg > 0 ? 1.0f / (float)dg : 0.0f;
    f[0] = ls * 0.05f;
    f[1] = lg * 0.05f;
    f[2] = (lg - ls) * 0.05f;
    f[3] = log2f(1.0f + (float)(ds + dg)) * 0.05f;
    f[4] = (float)ts[2] * is;
    f[5] = (float)tg[2] * ig;
    f[6] = (float)ts[0] * is;
    f[7] = (float)tg[0] * ig;
}

// Same features for a task given its two endpoints (global rows).
__device__ __forceinline__ void task_features_uv(int64_t u, int64_t v, const int32_t* deg, const int32_t* vtag,
                                                 float f[MLP_IN]) {
    const int du = deg[u], dv = deg[v];
    const bool us = du <= dv;
    task_features(us ? du : dv, us ? dv : du, vtag + 3 * (us ? u : v), vtag + 3 * (us ? v : u), f);
}

// FP16 inference.  The weights are packed as half2 pairs of consecutive
// output neurons, (W[2p][i], W[2p+1][i]) for each input i, so every half2
// fused multiply-add advances two neurons:
//   L1[16][8] B1[16] L2[16][32] B2[16] L3[2][32] B3[2]   (738 half2)
constexpr int MLPH_L1 = 0;
constexpr int MLPH_B1 = MLPH_L1 + (MLP_H / 2) * MLP_IN;
constexpr int MLPH_L2 = MLPH_B1 + MLP_H / 2;
constexpr int MLPH_B2 = MLPH_L2 + (MLP_H / 2) * MLP_H;
constexpr int MLPH_L3 = MLPH_B2 + MLP_H / 2;
constexpr int MLPH_B3 = MLPH_L3 + (MLP_OUT / 2) * MLP_H;
constexpr int MLPH_N = MLPH_B3 + MLP_OUT / 2;  // 738 half2

__device__ __forceinline__ void mlp_predict_h(const __half2* __restrict__ P, const float x[MLP_IN],
                                              float out[MLP_OUT]) {
    const __half2 zero = __float2half2_rn(0.0f);
    __half2 h1[MLP_H / 2];
#pragma unroll
    for (int p = 0; p < MLP_H / 2; ++p) {
        __half2 acc = P[MLPH_B1 + p];
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) acc = __hfma2(P[MLPH_L1 + p * MLP_IN + i], __float2half2_rn(x[i]), acc);
        h1[p] = __hmax2(acc, zero);
        asm volatile("" ::: "memory");  // keep the weight loads of one pair at a time
    }
    __half2 h2[MLP_H / 2];
#pragma unroll
    for (int p = 0; p < MLP_H / 2; ++p) {
        __half2 acc = P[MLPH_B2 + p];
        const __half2* row = P + MLPH_L2 + p * MLP_H;
#pragma unroll
        for (int i = 0; i < MLP_H; i += 2) {
            const __half2 a = h1[i / 2];
            acc = __hfma2(row[i], __low2half2(a), acc);
            acc = __hfma2(row[i + 1], __high2half2(a), acc);
        }
        h2[p] = __hmax2(acc, zero);
        asm volatile("" ::: "memory");
    }
#pragma unroll
    for (int p = 0; p < MLP_OUT / 2; ++p) {
        __half2 acc = P[MLPH_B3 + p];
#pragma unroll
        for (int i = 0; i < MLP_H; i += 2) {
            const __half2 a = h2[i / 2];
            acc = __hfma2(P[MLPH_L3 + p * MLP_H + i], __low2half2(a), acc);
            acc = __hfma2(P[MLPH_L3 + p * MLP_H + i + 1], __high2half2(a), acc);
        }
        out[2 * p] = __low2float(acc);
        out[2 * p + 1] = __high2float(acc);
    }
}

}  // namespace tc
