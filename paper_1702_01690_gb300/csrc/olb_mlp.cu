// olb_mlp.cu -- training and inference of the learned WENO-5 weight network
// (olb_mlp.cuh) on the GPU with hand-written kernels.
//
// Objective (per sample s): the interface value v2 + sum_q w_q G_q should be
// the target t; in normalised units the loss is the mean over samples of
// (sum_q w_q Gn_q - tn)^2 with Gn = G / r, tn = (t - v2) / r, r = max - min of
// the stencil.  Inputs: x [S][5] normalised stencils, Gn [S][3], tn [S].
//
// k_mlp_grad: one CTA per 128 samples.  Each thread runs the forward and
// backward pass of one sample, keeping the activations of the CTA's samples
// in shared memory; the weight gradients are then sums over those samples
// (small matrix products), one atomicAdd per parameter per CTA.
// k_adam: the Adam update of Kingma & Ba (2015), elementwise.
#include <cmath>
#include <algorithm>
#include <vector>

#include "../../include/olb.h"
#include "olb_mlp.cuh"

using namespace olb;

namespace {

constexpr int GB = 128;  // samples per CTA of k_mlp_grad

struct GradSmem {
    float th[MLP_P + 1];
    float x[GB][MLP_IN];
    float h1[GB][MLP_H + 1];
    float h2[GB][MLP_H + 1];
    float dz[GB][MLP_OUT];
    float da2[GB][MLP_H + 1];
    float da1[GB][MLP_H + 1];
    float red[GB / 32];
};

__global__ void __launch_bounds__(GB)
k_mlp_grad(const float *__restrict__ theta, const float *__restrict__ X, const float *__restrict__ Gn,
           const float *__restrict__ tn, int S, float inv_S, float *__restrict__ grad, float *__restrict__ loss)
{
    extern __shared__ __align__(16) unsigned char raw[];
    GradSmem &sm = *reinterpret_cast<GradSmem *>(raw);
    const int tid = threadIdx.x;
    for (int p = tid; p < MLP_P; p += GB) sm.th[p] = theta[p];
    const int s = blockIdx.x * GB + tid;
    const bool valid = s < S;
    for (int q = 0; q < MLP_IN; ++q) sm.x[tid][q] = valid ? X[(long long)s * MLP_IN + q] : 0.f;
    __syncthreads();
    const float *th = sm.th;
    // forward
    for (int j = 0; j < MLP_H; ++j) {
        float a = th[MLP_B1 + j];
        for (int q = 0; q < MLP_IN; ++q) a = fmaf(th[MLP_W1 + j * MLP_IN + q], sm.x[tid][q], a);
        sm.h1[tid][j] = tanhf(a);
    }
    for (int j = 0; j < MLP_H; ++j) {
        float a = th[MLP_B2 + j];
        for (int k = 0; k < MLP_H; ++k) a = fmaf(th[MLP_W2 + j * MLP_H + k], sm.h1[tid][k], a);
        sm.h2[tid][j] = tanhf(a);
    }
    float z[MLP_OUT], w[MLP_OUT];
    for (int q = 0; q < MLP_OUT; ++q) {
        float a = th[MLP_B3 + q];
        for (int j = 0; j < MLP_H; ++j) a = fmaf(th[MLP_W3 + q * MLP_H + j], sm.h2[tid][j], a);
        z[q] = a;
    }
    const float zm = fmaxf(z[0], fmaxf(z[1], z[2]));
    float se = 0.f;
    for (int q = 0; q < MLP_OUT; ++q) {
        w[q] = expf(z[q] - zm);
        se += w[q];
    }
    float g[MLP_OUT] = {0.f, 0.f, 0.f};
    float res = 0.f;
    if (valid) {
        for (int q = 0; q < MLP_OUT; ++q) {
            w[q] /= se;
            g[q] = Gn[(long long)s * MLP_OUT + q];
        }
        res = fmaf(w[0], g[0], fmaf(w[1], g[1], fmaf(w[2], g[2], -tn[s])));
    }
    // backward: dL/dw = 2 res G / S; softmax; tanh layers
    float dw[MLP_OUT], wdw = 0.f;
    for (int q = 0; q < MLP_OUT; ++q) {
        dw[q] = valid ? 2.f * inv_S * res * g[q] : 0.f;
        wdw = fmaf(valid ? w[q] : 0.f, dw[q], wdw);
    }
    for (int q = 0; q < MLP_OUT; ++q) sm.dz[tid][q] = valid ? w[q] * (dw[q] - wdw) : 0.f;
    for (int j = 0; j < MLP_H; ++j) {
        float a = 0.f;
        for (int q = 0; q < MLP_OUT; ++q) a = fmaf(sm.dz[tid][q], th[MLP_W3 + q * MLP_H + j], a);
        const float h = sm.h2[tid][j];
        sm.da2[tid][j] = a * (1.f - h * h);
    }
    for (int k = 0; k < MLP_H; ++k) {
        float a = 0.f;
        for (int j = 0; j < MLP_H; ++j) a = fmaf(sm.da2[tid][j], th[MLP_W2 + j * MLP_H + k], a);
        const float h = sm.h1[tid][k];
        sm.da1[tid][k] = a * (1.f - h * h);
    }
    // loss of the CTA's samples
    float l2 = res * res;
    for (int off = 16; off > 0; off >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, off);
    if ((tid & 31) == 0) sm.red[tid >> 5] = l2;
    __syncthreads();
    if (tid == 0) {
        float acc = 0.f;
        for (int k = 0; k < GB / 32; ++k) acc += sm.red[k];
        atomicAdd(loss, acc * inv_S);
    }
    // weight gradients: sums over the CTA's samples
    const int ns = min(GB, S - blockIdx.x * GB);
    for (int p = tid; p < MLP_P; p += GB) {
        float acc = 0.f;
        if (p < MLP_B1) {
            const int j = p / MLP_IN, q = p - j * MLP_IN;
            for (int t = 0; t < ns; ++t) acc = fmaf(sm.da1[t][j], sm.x[t][q], acc);
        } else if (p < MLP_W2) {
            const int j = p - MLP_B1;
            for (int t = 0; t < ns; ++t) acc += sm.da1[t][j];
        } else if (p < MLP_B2) {
            const int j = (p - MLP_W2) / MLP_H, k = (p - MLP_W2) - j * MLP_H;
            for (int t = 0; t < ns; ++t) acc = fmaf(sm.da2[t][j], sm.h1[t][k], acc);
        } else if (p < MLP_W3) {
            const int j = p - MLP_B2;
            for (int t = 0; t < ns; ++t) acc += sm.da2[t][j];
        } else if (p < MLP_B3) {
            const int q = (p - MLP_W3) / MLP_H, j = (p - MLP_W3) - q * MLP_H;
            for (int t = 0; t < ns; ++t) acc = fmaf(sm.dz[t][q], sm.h2[t][j], acc);
        } else {
            const int q = p - MLP_B3;
            for (int t = 0; t < ns; ++t) acc += sm.dz[t][q];
        }
        atomicAdd(grad + p, acc);
    }
}

__global__ void k_adam(float *__restrict__ theta, const float *__restrict__ grad, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= MLP_P) return;
    const float g = grad[p];
    const float mm = fmaf(b1, m[p], (1.f - b1) * g);
    const float vv = fmaf(b2, v[p], (1.f - b2) * g * g);
    m[p] = mm;
    v[p] = vv;
    theta[p] -= lr * (mm * c1) / (sqrtf(vv * c2) + eps);
}

__global__ void k_mlp_forward(const float *__restrict__ theta, const float *__restrict__ X, int S,
                              float *__restrict__ W)
{
    __shared__ __align__(16) float th[MLP_P + 1];
    for (int p = threadIdx.x; p < MLP_P; p += blockDim.x) th[p] = theta[p];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    float x[MLP_IN], w[MLP_OUT];
    for (int q = 0; q < MLP_IN; ++q) x[q] = X[(long long)s * MLP_IN + q];
    mlp_weights(th, x, w);
    for (int q = 0; q < MLP_OUT; ++q) W[(long long)s * MLP_OUT + q] = w[q];
}

cudaError_t grad_launch(const float *theta, const float *x, const float *g, const float *t, int n, float *grad,
                        float *loss, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(GradSmem));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_mlp_grad<<<(n + GB - 1) / GB, GB, sizeof(GradSmem), s>>>(theta, x, g, t, n, 1.0f / (float)n, grad, loss);
    return cudaGetLastError();
}

}  // namespace

extern "C" int olb_mlp_forward(const float *theta, const float *x, int n, float *w, void *stream)
{
    if (!theta || !x || !w || n < 0) return OLB_ERR_ARG;
    if (n == 0) return OLB_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_mlp_forward<<<(n + 127) / 128, 128, 0, s>>>(theta, x, n, w);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return cuda_status(e);
}

extern "C" int olb_mlp_grad(const float *theta, const float *x, const float *g, const float *t, int n, float *grad,
                            float *loss, void *stream)
{
    if (!theta || !x || !g || !t || !grad || !loss || n < 1) return OLB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(grad, 0, MLP_P * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (e == cudaSuccess) e = grad_launch(theta, x, g, t, n, grad, loss, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return cuda_status(e);
}

extern "C" int olb_mlp_train(float *theta, const float *x, const float *g, const float *t, int n, int epochs,
                             int batch, float lr, void *stream, float *loss_history)
{
    if (!theta || !x || !g || !t || n < 1 || epochs < 1 || batch < 1 || !(lr > 0.f)) return OLB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float *work = nullptr;  // grad, m, v, per-epoch loss
    cudaError_t e = cudaMalloc((void **)&work, (3 * MLP_P + epochs + 8) * sizeof(float));
    if (e != cudaSuccess) return cuda_status(e);
    float *grad = work, *m = work + MLP_P, *v = work + 2 * MLP_P, *lhist = work + 3 * MLP_P;
    e = cudaMemsetAsync(work, 0, (3 * MLP_P + epochs + 8) * sizeof(float), s);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    long long step = 0;
    const int nb = (n + batch - 1) / batch;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        for (int b = 0; b < nb && e == cudaSuccess; ++b) {
            const int off = b * batch, cnt = std::min(batch, n - off);
            ++step;
            e = cudaMemsetAsync(grad, 0, MLP_P * sizeof(float), s);
            // the loss of minibatch b is weighted by its share of the epoch
            if (e == cudaSuccess)
                e = grad_launch(theta, x + (long long)off * MLP_IN, g + (long long)off * MLP_OUT, t + off, cnt, grad,
                                lhist + ep, s);
            if (e == cudaSuccess) {
                const float c1 = 1.f / (1.f - powf(b1, (float)step)), c2 = 1.f / (1.f - powf(b2, (float)step));
                k_adam<<<(MLP_P + 255) / 256, 256, 0, s>>>(theta, grad, m, v, lr, b1, b2, eps, c1, c2);
                e = cudaGetLastError();
            }
        }
    }
    std::vector<float> h(epochs, 0.f);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), lhist, epochs * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(work);
    if (e != cudaSuccess) return cuda_status(e);
    if (loss_history)
        for (int ep = 0; ep < epochs; ++ep) loss_history[ep] = h[ep] / (float)nb;
    return OLB_OK;
}
