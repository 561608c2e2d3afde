// Learned sub-level scheduler: a small FP32 MLP cost model (project
// addition; the paper schedules with OpenMP's dynamic loop scheduling).
//
// Model: 5 frontier features -> 32 -> 32 -> TRUSS_SCHED_VARIANTS predicted
// log2 device times of a sub-level, one per ProcessSubLevel variant; ReLU
// hidden layers; the decision is the argmin.  Features are normalised by a
// per-feature mean and inverse standard deviation stored with the weights.
// Training minimises the mean squared error of the log2 times over logged
// sub-levels (every variant's time is known for every sub-level, because the
// frontier sequence does not depend on the variant) with full-batch Adam,
// entirely on the device: a partial-gradient kernel per block of samples,
// then one reduction + Adam kernel.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "graph.cuh"
#include "sched.cuh"

namespace {

constexpr int ST = 256;  // threads per block for the sample-parallel kernels

struct Model {
    const float* p;
    __device__ __forceinline__ float w1(int j, int i) const { return p[SP_W1 + j * SF + i]; }
    __device__ __forceinline__ float b1(int j) const { return p[SP_B1 + j]; }
    __device__ __forceinline__ float w2(int j, int k) const { return p[SP_W2 + j * SH + k]; }
    __device__ __forceinline__ float b2(int j) const { return p[SP_B2 + j]; }
    __device__ __forceinline__ float w3(int v, int j) const { return p[SP_W3 + v * SH + j]; }
    __device__ __forceinline__ float b3(int v) const { return p[SP_B3 + v]; }
};

// Forward pass of one sample by one thread; the outputs go to out.
__device__ void sample_forward(const Model& M, const float* x, float* out) {
    float xn[SF];
#pragma unroll
    for (int i = 0; i < SF; i++) xn[i] = (x[i] - M.p[SP_MU + i]) * M.p[SP_ISD + i];
    float h1[SH];
#pragma unroll
    for (int j = 0; j < SH; j++) {
        float a = M.b1(j);
#pragma unroll
        for (int i = 0; i < SF; i++) a = fmaf(M.w1(j, i), xn[i], a);
        h1[j] = a > 0.f ? a : 0.f;
    }
    float h2[SH];
    for (int j = 0; j < SH; j++) {
        float a = M.b2(j);
#pragma unroll
        for (int k = 0; k < SH; k++) a = fmaf(M.w2(j, k), h1[k], a);
        h2[j] = a > 0.f ? a : 0.f;
    }
#pragma unroll
    for (int v = 0; v < SV; v++) {
        float a = M.b3(v);
#pragma unroll
        for (int j = 0; j < SH; j++) a = fmaf(M.w3(v, j), h2[j], a);
        out[v] = a;
    }
}

// 32 samples, one per lane (lanes without a sample pass valid = false):
// forward and backward passes of scale * sum_v (o_v - y_v)^2.  Each
// parameter's gradient is summed over the warp with shuffles and added once
// to g (shared memory).  Returns the warp's loss (on every lane).
__device__ float warp_fwd_bwd(const Model& M, const float* x, const float* y, bool valid, float scale, float* g) {
    const int lane = threadIdx.x & 31;
    auto add = [&](int idx, float v) {
        v = warp_sum(v);
        if (lane == 0) atomicAdd(g + idx, v);
    };
    float xn[SF];
#pragma unroll
    for (int i = 0; i < SF; i++) xn[i] = valid ? (x[i] - M.p[SP_MU + i]) * M.p[SP_ISD + i] : 0.f;
    float z1[SH], h1[SH];
#pragma unroll
    for (int j = 0; j < SH; j++) {
        float a = M.b1(j);
#pragma unroll
        for (int i = 0; i < SF; i++) a = fmaf(M.w1(j, i), xn[i], a);
        z1[j] = a;
        h1[j] = a > 0.f ? a : 0.f;
    }
    float z2[SH], h2[SH];
    for (int j = 0; j < SH; j++) {
        float a = M.b2(j);
#pragma unroll
        for (int k = 0; k < SH; k++) a = fmaf(M.w2(j, k), h1[k], a);
        z2[j] = a;
        h2[j] = a > 0.f ? a : 0.f;
    }
    float dov[SV], loss = 0.f;
#pragma unroll
    for (int v = 0; v < SV; v++) {
        float a = M.b3(v);
#pragma unroll
        for (int j = 0; j < SH; j++) a = fmaf(M.w3(v, j), h2[j], a);
        const float d = valid ? a - y[v] : 0.f;
        loss += d * d * scale;
        dov[v] = 2.f * d * scale;
        add(SP_B3 + v, dov[v]);
    }
    float dz2[SH];
    for (int j = 0; j < SH; j++) {
        float a = 0.f;
#pragma unroll
        for (int v = 0; v < SV; v++) {
            add(SP_W3 + v * SH + j, dov[v] * h2[j]);
            a = fmaf(M.w3(v, j), dov[v], a);
        }
        dz2[j] = z2[j] > 0.f ? a : 0.f;
        add(SP_B2 + j, dz2[j]);
    }
    float dh1[SH];
#pragma unroll
    for (int k = 0; k < SH; k++) dh1[k] = 0.f;
    for (int j = 0; j < SH; j++)
        for (int k = 0; k < SH; k++) {
            add(SP_W2 + j * SH + k, dz2[j] * h1[k]);
            dh1[k] = fmaf(M.w2(j, k), dz2[j], dh1[k]);
        }
    float dxn[SF];
#pragma unroll
    for (int i = 0; i < SF; i++) dxn[i] = 0.f;
    for (int j = 0; j < SH; j++) {
        const float dz1 = z1[j] > 0.f ? dh1[j] : 0.f;
        add(SP_B1 + j, dz1);
#pragma unroll
        for (int i = 0; i < SF; i++) {
            add(SP_W1 + j * SF + i, dz1 * xn[i]);
            dxn[i] = fmaf(M.w1(j, i), dz1, dxn[i]);
        }
    }
    // normalisation: xn = (x - mu) * isd
#pragma unroll
    for (int i = 0; i < SF; i++) {
        add(SP_ISD + i, valid ? dxn[i] * (x[i] - M.p[SP_MU + i]) : 0.f);
        add(SP_MU + i, -dxn[i] * M.p[SP_ISD + i]);
    }
    return warp_sum(loss);
}

// per-block partial gradients of the mean loss (row blockIdx.x of partial)
__global__ void __launch_bounds__(ST) k_sched_grad(const float* __restrict__ params, const float* __restrict__ x,
                                                   const float* __restrict__ y, int64_t n, float* __restrict__ partial,
                                                   float* __restrict__ partial_loss) {
    __shared__ float g[SP_COUNT];
    __shared__ float lsum[ST / 32];
    for (int i = threadIdx.x; i < SP_COUNT; i += blockDim.x) g[i] = 0.f;
    __syncthreads();
    const Model M{params};
    const float scale = 1.f / (float)(n * SV);
    const int lane = threadIdx.x & 31;
    float loss = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t s = base + lane;
        const bool valid = s < n;
        loss += warp_fwd_bwd(M, x + (valid ? s : 0) * SF, y + (valid ? s : 0) * SV, valid, scale, g);
    }
    if (lane == 0) lsum[threadIdx.x >> 5] = loss;
    __syncthreads();
    for (int i = threadIdx.x; i < SP_COUNT; i += blockDim.x) partial[(int64_t)blockIdx.x * SP_COUNT + i] = g[i];
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < ST / 32; w++) t += lsum[w];
        partial_loss[blockIdx.x] = t;
    }
}

// sum the partial gradients; optionally write them out and/or take one Adam step
__global__ void __launch_bounds__(ST) k_sched_reduce(const float* __restrict__ partial,
                                                     const float* __restrict__ partial_loss, int nparts,
                                                     float* __restrict__ grad, float* __restrict__ params,
                                                     float* __restrict__ adam, float* __restrict__ loss_out,
                                                     int step, float lr) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int i = threadIdx.x; i < SP_COUNT; i += blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < nparts; b++) s += partial[(int64_t)b * SP_COUNT + i];
        if (grad) grad[i] = s;
        if (params && i >= SP_W1) {  // normalisation constants are not trained
            float* mo = adam + i;
            float* ve = adam + SP_COUNT + i;
            *mo = b1 * *mo + (1.f - b1) * s;
            *ve = b2 * *ve + (1.f - b2) * s * s;
            const float mh = *mo / (1.f - powf(b1, (float)step));
            const float vh = *ve / (1.f - powf(b2, (float)step));
            params[i] -= lr * mh / (sqrtf(vh) + eps);
        }
    }
    if (threadIdx.x == 0 && loss_out) {
        float t = 0.f;
        for (int b = 0; b < nparts; b++) t += partial_loss[b];
        *loss_out = t;
    }
}

__global__ void k_sched_predict(const float* __restrict__ params, const float* __restrict__ x, int64_t n,
                                float* __restrict__ out) {
    const Model M{params};
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        sample_forward(M, x + s * SF, out + s * SV);
}

// per-feature mean and inverse standard deviation of the training inputs
__global__ void k_sched_norm(const float* __restrict__ x, int64_t n, float* __restrict__ params) {
    __shared__ double acc[2 * SF][ST / 32];
    double s[SF], q[SF];
#pragma unroll
    for (int i = 0; i < SF; i++) s[i] = q[i] = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x)
#pragma unroll
        for (int i = 0; i < SF; i++) {
            const double v = x[k * SF + i];
            s[i] += v;
            q[i] += v * v;
        }
#pragma unroll
    for (int i = 0; i < SF; i++) {
        s[i] = warp_sum(s[i]);
        q[i] = warp_sum(q[i]);
        if ((threadIdx.x & 31) == 0) {
            acc[i][threadIdx.x >> 5] = s[i];
            acc[SF + i][threadIdx.x >> 5] = q[i];
        }
    }
    __syncthreads();
    if (threadIdx.x < SF) {
        const int i = threadIdx.x;
        double S = 0, Q = 0;
        for (int w = 0; w < ST / 32; w++) {
            S += acc[i][w];
            Q += acc[SF + i][w];
        }
        const double mu = n ? S / (double)n : 0.0;
        const double var = n ? Q / (double)n - mu * mu : 1.0;
        params[SP_MU + i] = (float)mu;
        params[SP_ISD + i] = (float)(1.0 / sqrt(var > 1e-12 ? var : 1.0));
    }
}

int partial_blocks(int64_t n, int sms) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + ST - 1) / ST, sms)); }

}  // namespace

// Features of a sub-level: log2 of frontier size, shorter-row sum and max,
// level and edges left (each + 1).  Shared by the host and the device.
extern "C" void truss_sched_features(const truss_sublevel_trace* tr, int64_t n, float* x) {
    for (int64_t k = 0; k < n; k++) sched_features(tr[k].n_light + tr[k].n_heavy, tr[k].dsum, tr[k].dmax, tr[k].level,
                                                   tr[k].todo, x + k * SF);
}

extern "C" int truss_sched_init(float* d_params, uint64_t seed, void* stream) {
    if (!d_params) return TRUSS_EINVAL;
    float h[SP_COUNT];
    // He-style uniform initialisation from a counter-based SplitMix64 stream
    uint64_t state = seed;
    auto next = [&]() {
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (float)((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;
    };
    for (int i = 0; i < SF; i++) {
        h[SP_MU + i] = 0.f;
        h[SP_ISD + i] = 1.f;
    }
    const float a1 = sqrtf(6.f / SF), a2 = sqrtf(6.f / SH);
    for (int i = 0; i < SH * SF; i++) h[SP_W1 + i] = a1 * next();
    for (int i = 0; i < SH; i++) h[SP_B1 + i] = 0.f;
    for (int i = 0; i < SH * SH; i++) h[SP_W2 + i] = a2 * next();
    for (int i = 0; i < SH; i++) h[SP_B2 + i] = 0.f;
    for (int i = 0; i < SV * SH; i++) h[SP_W3 + i] = a2 * next() * 0.5f;
    for (int i = 0; i < SV; i++) h[SP_B3 + i] = 0.f;
    CU(cudaMemcpyAsync(d_params, h, sizeof(h), cudaMemcpyHostToDevice, (cudaStream_t)stream));
    CU(cudaStreamSynchronize((cudaStream_t)stream));
    return TRUSS_OK;
}

extern "C" int truss_sched_grad(const float* d_params, const float* d_x, const float* d_y, int64_t n, float* d_grad,
                                float* h_loss, void* stream) {
    if (!d_params || n < 0 || (n > 0 && (!d_x || !d_y)) || !d_grad) return TRUSS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int nb = partial_blocks(n, sms);
    float *part = nullptr, *pl = nullptr, *dl = nullptr;
    CU(cudaMallocAsync((void**)&part, sizeof(float) * (size_t)nb * SP_COUNT, s));
    CU(cudaMallocAsync((void**)&pl, sizeof(float) * (size_t)nb, s));
    CU(cudaMallocAsync((void**)&dl, sizeof(float), s));
    k_sched_grad<<<nb, ST, 0, s>>>(d_params, d_x, d_y, n, part, pl);
    k_sched_reduce<<<1, ST, 0, s>>>(part, pl, nb, d_grad, nullptr, nullptr, dl, 0, 0.f);
    CU(cudaGetLastError());
    float loss = 0.f;
    CU(cudaMemcpyAsync(&loss, dl, sizeof(float), cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(part, s);
    cudaFreeAsync(pl, s);
    cudaFreeAsync(dl, s);
    CU(cudaStreamSynchronize(s));
    if (h_loss) *h_loss = loss;
    return TRUSS_OK;
}

extern "C" int truss_sched_train(float* d_params, const float* d_x, const float* d_y, int64_t n, int32_t epochs,
                                 float lr, float* h_loss, void* stream) {
    if (!d_params || n <= 0 || !d_x || !d_y || epochs < 0 || !(lr > 0.f)) return TRUSS_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int nb = partial_blocks(n, sms);
    float *part = nullptr, *pl = nullptr, *dl = nullptr, *adam = nullptr;
    CU(cudaMallocAsync((void**)&part, sizeof(float) * (size_t)nb * SP_COUNT, s));
    CU(cudaMallocAsync((void**)&pl, sizeof(float) * (size_t)nb, s));
    CU(cudaMallocAsync((void**)&dl, sizeof(float), s));
    CU(cudaMallocAsync((void**)&adam, sizeof(float) * 2 * SP_COUNT, s));
    CU(cudaMemsetAsync(adam, 0, sizeof(float) * 2 * SP_COUNT, s));
    k_sched_norm<<<1, ST, 0, s>>>(d_x, n, d_params);
    for (int e = 1; e <= epochs; e++) {
        k_sched_grad<<<nb, ST, 0, s>>>(d_params, d_x, d_y, n, part, pl);
        k_sched_reduce<<<1, ST, 0, s>>>(part, pl, nb, nullptr, d_params, adam, dl, e, lr);
    }
    // loss of the final model
    k_sched_grad<<<nb, ST, 0, s>>>(d_params, d_x, d_y, n, part, pl);
    k_sched_reduce<<<1, ST, 0, s>>>(part, pl, nb, nullptr, nullptr, nullptr, dl, 0, 0.f);
    CU(cudaGetLastError());
    float loss = 0.f;
    CU(cudaMemcpyAsync(&loss, dl, sizeof(float), cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(part, s);
    cudaFreeAsync(pl, s);
    cudaFreeAsync(dl, s);
    cudaFreeAsync(adam, s);
    CU(cudaStreamSynchronize(s));
    if (h_loss) *h_loss = loss;
    return TRUSS_OK;
}

extern "C" int truss_sched_predict(const float* d_params, const float* d_x, int64_t n, float* d_out, void* stream) {
    if (!d_params || n < 0 || (n > 0 && (!d_x || !d_out))) return TRUSS_EINVAL;
    if (n == 0) return TRUSS_OK;
    k_sched_predict<<<grid_for(n, 128), 128, 0, (cudaStream_t)stream>>>(d_params, d_x, n, d_out);
    CU(cudaGetLastError());
    return TRUSS_OK;
}
