// The sigma policy network: an MLP with three hidden layers of 64 ReLU units over a
// 64-value history of the solver's checks, five outputs (one predicted outcome per
// sigma multiplier).  Weights are stored in BF16 for the forward and backward passes,
// with FP32 accumulation and FP32 master weights updated by Adam.  Forward, backward
// (per-CTA partial gradients), the fixed-order gradient reduction and the optimiser step
// are the kernels below; everything is deterministic.
//
// Parameter layout (row-major W[out][in]):  W1 64x64, b1 64, W2 64x64, b2 64, W3 64x64,
// b3 64, W4 5x64, b4 5: 12,805 values.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace hprmlp {

constexpr int IN = 64, H = 64, OUT = 5;
constexpr int OW1 = 0, OB1 = OW1 + H * IN, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H,
              OB3 = OW3 + H * H, OW4 = OB3 + H, OB4 = OW4 + OUT * H, P = OB4 + OUT;
constexpr int TPB = 64;   // threads per CTA: thread j owns hidden unit j of every layer

__device__ __forceinline__ float wf(const __nv_bfloat16 *w, int i) { return __bfloat162float(w[i]); }

// one sample's forward pass, activations kept in shared memory; returns q in q[0..OUT)
__device__ __forceinline__ void forward(const __nv_bfloat16 *w, const float *x, float *a0, float *z1,
                                        float *z2, float *z3, float *q)
{
    const int j = threadIdx.x;
    a0[j] = x[j];
    __syncthreads();
    float s = wf(w, OB1 + j);
    for (int k = 0; k < IN; ++k) s = fmaf(wf(w, OW1 + j * IN + k), a0[k], s);
    z1[j] = s;
    __syncthreads();
    s = wf(w, OB2 + j);
    for (int k = 0; k < H; ++k) s = fmaf(wf(w, OW2 + j * H + k), fmaxf(z1[k], 0.f), s);
    z2[j] = s;
    __syncthreads();
    s = wf(w, OB3 + j);
    for (int k = 0; k < H; ++k) s = fmaf(wf(w, OW3 + j * H + k), fmaxf(z2[k], 0.f), s);
    z3[j] = s;
    __syncthreads();
    if (j < OUT) {
        float t = wf(w, OB4 + j);
        for (int k = 0; k < H; ++k) t = fmaf(wf(w, OW4 + j * H + k), fmaxf(z3[k], 0.f), t);
        q[j] = t;
    }
    __syncthreads();
}

// outputs for n samples (one CTA per sample)
__global__ void __launch_bounds__(TPB) k_infer(const __nv_bfloat16 *__restrict__ w, const float *__restrict__ X,
                                               int n, float *Q)
{
    __shared__ float a0[IN], z1[H], z2[H], z3[H], q[OUT];
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        forward(w, X + (size_t)i * IN, a0, z1, z2, z3, q);
        if (threadIdx.x < OUT) Q[(size_t)i * OUT + threadIdx.x] = q[threadIdx.x];
        __syncthreads();
    }
}

// Loss 1/2 (q[a_i] - y_i)^2 summed over samples idx[lo .. hi) of CTA c (chunk samples
// each), and its gradient with respect to the BF16 weights, as CTA partials:
// gpart[c * P + p] and lpart[c].  The gradient rows of thread j are its own; its
// updates walk the columns in a rotated order so the 64 threads hit distinct banks.
__global__ void __launch_bounds__(TPB) k_grad(const __nv_bfloat16 *__restrict__ w, const float *__restrict__ X,
                                              const int *__restrict__ act, const float *__restrict__ y,
                                              const int *__restrict__ idx, int n, int chunk, float *gpart,
                                              double *lpart)
{
    extern __shared__ float g[];          // P accumulators
    __shared__ float a0[IN], z1[H], z2[H], z3[H], q[OUT], d3[H], d2[H], d1[H];
    __shared__ float err;
    const int j = threadIdx.x;
    for (int p = j; p < P; p += TPB) g[p] = 0.f;
    double loss = 0.0;
    __syncthreads();
    const int lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    for (int s = lo; s < hi; ++s) {
        const int i = idx ? idx[s] : s;
        forward(w, X + (size_t)i * IN, a0, z1, z2, z3, q);
        const int a = act[i];
        if (j == 0) {
            err = q[a] - y[i];
            loss += 0.5 * (double)err * (double)err;
        }
        __syncthreads();
        const float e = err;
        // output layer: dq = e at output a
        const float r3 = fmaxf(z3[j], 0.f);
        g[OW4 + a * H + j] += e * r3;
        if (j == 0) g[OB4 + a] += e;
        d3[j] = z3[j] > 0.f ? e * wf(w, OW4 + a * H + j) : 0.f;
        __syncthreads();
        // layer 3: W3 gradient row j, delta of layer 2 (column j of W3)
        {
            const float dj = d3[j];
            for (int t = 0; t < H; ++t) {
                const int k = (j + t) & (H - 1);
                g[OW3 + j * H + k] += dj * fmaxf(z2[k], 0.f);
            }
            g[OB3 + j] += dj;
            float s2 = 0.f;
            for (int r = 0; r < H; ++r) s2 = fmaf(wf(w, OW3 + r * H + j), d3[r], s2);
            d2[j] = z2[j] > 0.f ? s2 : 0.f;
        }
        __syncthreads();
        {
            const float dj = d2[j];
            for (int t = 0; t < H; ++t) {
                const int k = (j + t) & (H - 1);
                g[OW2 + j * H + k] += dj * fmaxf(z1[k], 0.f);
            }
            g[OB2 + j] += dj;
            float s1 = 0.f;
            for (int r = 0; r < H; ++r) s1 = fmaf(wf(w, OW2 + r * H + j), d2[r], s1);
            d1[j] = z1[j] > 0.f ? s1 : 0.f;
        }
        __syncthreads();
        {
            const float dj = d1[j];
            for (int t = 0; t < IN; ++t) {
                const int k = (j + t) & (IN - 1);
                g[OW1 + j * IN + k] += dj * a0[k];
            }
            g[OB1 + j] += dj;
        }
        __syncthreads();
    }
    for (int p = j; p < P; p += TPB) gpart[(size_t)blockIdx.x * P + p] = g[p];
    if (j == 0) lpart[blockIdx.x] = loss;
}

// gradient and loss means over the batch: CTA partials summed in CTA order
__global__ void k_reduce_grad(const float *__restrict__ gpart, const double *__restrict__ lpart, int ctas,
                              double inv_n, float *grad, double *loss)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < ctas; ++c) s += (double)gpart[(size_t)c * P + p];
        grad[p] = (float)(s * inv_n);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int c = 0; c < ctas; ++c) s += lpart[c];
        *loss = s * inv_n;
    }
}

// Adam (Kingma & Ba, 2015) on the FP32 masters, then their BF16 copy
__global__ void k_adam(float *w, float *m, float *v, const float *__restrict__ g, float lr, float b1, float b2,
                       float eps, float c1, float c2, __nv_bfloat16 *wb)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        const float gp = g[p];
        const float mp = b1 * m[p] + (1.f - b1) * gp;
        const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
        m[p] = mp;
        v[p] = vp;
        const float wp = w[p] - lr * (mp / c1) / (sqrtf(vp / c2) + eps);
        w[p] = wp;
        wb[p] = __float2bfloat16_rn(wp);
    }
}

__global__ void k_to_bf16(const float *__restrict__ w, __nv_bfloat16 *wb)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x)
        wb[p] = __float2bfloat16_rn(w[p]);
}

constexpr size_t GRAD_SMEM = sizeof(float) * P;

}  // namespace hprmlp
