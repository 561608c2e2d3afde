// Layout of the learned scheduler's parameters and the feature function
// shared by the trainer (sched.cu) and the persistent kernel (peel.cu).
#pragma once
#include <math.h>

#include "common.cuh"

constexpr int SF = TRUSS_SCHED_FEATURES;  // inputs
constexpr int SH = 32;                    // hidden width (two layers)
constexpr int SV = TRUSS_SCHED_VARIANTS;  // outputs: one per variant

enum {
    SP_MU = 0,                // [SF] feature means
    SP_ISD = SP_MU + SF,      // [SF] feature inverse standard deviations
    SP_W1 = SP_ISD + SF,      // [SH][SF]
    SP_B1 = SP_W1 + SH * SF,  // [SH]
    SP_W2 = SP_B1 + SH,       // [SH][SH]
    SP_B2 = SP_W2 + SH * SH,  // [SH]
    SP_W3 = SP_B2 + SH,       // [SV][SH]
    SP_B3 = SP_W3 + SV * SH,  // [SV]
    SP_COUNT = SP_B3 + SV
};
static_assert(SP_COUNT == TRUSS_SCHED_PARAMS, "parameter count in truss.h");

// log2 of frontier size, shorter-row sum and max, level, edges left (+1)
__host__ __device__ __forceinline__ void sched_features(int64_t size, int64_t dsum, int64_t dmax, int64_t level,
                                                        int64_t todo, float* x) {
    x[0] = log2f(1.f + (float)size);
    x[1] = log2f(1.f + (float)dsum);
    x[2] = log2f(1.f + (float)dmax);
    x[3] = log2f(1.f + (float)level);
    x[4] = log2f(1.f + (float)todo);
}

// A sub-level whose normalised features lie further than this many standard
// deviations from the training mean is outside what the model was fitted
// on: the fixed heuristic decides it.
constexpr float SCHED_Z_MAX = 4.f;

// Warp-cooperative inference (all 32 lanes call): lane j computes hidden unit
// j of each layer; returns the variant with the smallest predicted time, or
// -1 (the heuristic decides) when a feature is out of the training range or
// the model yields a non-finite value.
__device__ __forceinline__ int sched_pick(const float* __restrict__ p, const float* x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < SF; i++)
        if (fabsf((x[i] - __ldg(p + SP_MU + i)) * __ldg(p + SP_ISD + i)) > SCHED_Z_MAX) return -1;
    float a = __ldg(p + SP_B1 + lane);
#pragma unroll
    for (int i = 0; i < SF; i++) a = fmaf(__ldg(p + SP_W1 + lane * SF + i), (x[i] - __ldg(p + SP_MU + i)) * __ldg(p + SP_ISD + i), a);
    const float h1 = a > 0.f ? a : 0.f;
    float b = __ldg(p + SP_B2 + lane);
#pragma unroll
    for (int k = 0; k < SH; k++) b = fmaf(__ldg(p + SP_W2 + lane * SH + k), __shfl_sync(0xffffffffu, h1, k), b);
    const float h2 = b > 0.f ? b : 0.f;
    int best = -1;
    float bo = 0.f;
#pragma unroll
    for (int v = 0; v < SV; v++) {
        float o = __ldg(p + SP_W3 + v * SH + lane) * h2;
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) o += __shfl_xor_sync(0xffffffffu, o, s);
        o += __ldg(p + SP_B3 + v);
        if (!isfinite(o)) return -1;
        if (best < 0 || o < bo) {
            best = v;
            bo = o;
        }
    }
    return best;
}
