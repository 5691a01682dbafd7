// olb_mlp.cuh -- the learned WENO-5 weight network on the device.
//
// A 5-32-32-3 MLP (tanh, tanh, softmax) maps the normalised stencil
// x = (v - mean v) / (max v - min v) of an interface to three convex weights
// that replace the Jiang-Shu weights of Eq. weno5_omega.  Parameters, 1347
// floats: W1 [32][5], b1 [32], W2 [32][32], b2 [32], W3 [3][32], b3 [3]
// (row-major, concatenated).
#pragma once

#include "olb_kernels.cuh"

namespace olb {

constexpr int MLP_IN = 5, MLP_H = 32, MLP_OUT = 3;
constexpr int MLP_W1 = 0, MLP_B1 = 160, MLP_W2 = 192, MLP_B2 = 1216, MLP_W3 = 1248, MLP_B3 = 1344;
constexpr int MLP_P = 1347;
// The network acts only where the stencil is not smooth in the Jiang-Shu
// sense: min sigma_q < MLP_GUARD max sigma_q.  Where the three indicators are
// within that factor (smooth data, for which the Jiang-Shu weights approach
// the ideal weights and keep 5th order) the Jiang-Shu weights are used.
constexpr double MLP_GUARD = 0.9;

// tanh(x) = sign(x) (1 - 2 / (exp(2 |x|) + 1)), with exp(2 |x|) = 2^(2 |x| / ln 2)
// and the reciprocal from the special-function unit (ex2.approx.ftz.f32,
// rcp.approx.ftz.f32): 6 instructions instead of an accurate tanhf, with an
// absolute error of ~1e-7 (the network's forward pass is checked against the
// FP64 network at 2e-6 in the tests); exp overflowing to +inf gives 1.
__device__ __forceinline__ float tanh_fast(float x)
{
    float e, r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(fabsf(x) * 2.8853900817779268f));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(e + 1.0f));
    return copysignf(fmaf(-2.0f, r, 1.0f), x);
}

// Weights of one stencil; th points to the parameters (shared memory in the
// stage kernel).  x: normalised stencil.
__device__ __forceinline__ void mlp_weights(const float *__restrict__ th, const float x[MLP_IN], float w[MLP_OUT])
{
    float h1[MLP_H];
#pragma unroll
    for (int j = 0; j < MLP_H; ++j) {
        float a = th[MLP_B1 + j];
#pragma unroll
        for (int q = 0; q < MLP_IN; ++q) a = fmaf(th[MLP_W1 + j * MLP_IN + q], x[q], a);
        h1[j] = tanh_fast(a);
    }
    float z0 = th[MLP_B3 + 0], z1 = th[MLP_B3 + 1], z2 = th[MLP_B3 + 2];
#pragma unroll 4
    for (int j = 0; j < MLP_H; ++j) {
        const float4 *row = reinterpret_cast<const float4 *>(th + MLP_W2 + j * MLP_H);
        float a = th[MLP_B2 + j];
#pragma unroll
        for (int k4 = 0; k4 < MLP_H / 4; ++k4) {
            const float4 r = row[k4];
            a = fmaf(r.x, h1[4 * k4 + 0], a);
            a = fmaf(r.y, h1[4 * k4 + 1], a);
            a = fmaf(r.z, h1[4 * k4 + 2], a);
            a = fmaf(r.w, h1[4 * k4 + 3], a);
        }
        const float h2 = tanh_fast(a);
        z0 = fmaf(th[MLP_W3 + 0 * MLP_H + j], h2, z0);
        z1 = fmaf(th[MLP_W3 + 1 * MLP_H + j], h2, z1);
        z2 = fmaf(th[MLP_W3 + 2 * MLP_H + j], h2, z2);
    }
    const float zm = fmaxf(z0, fmaxf(z1, z2));
    const float e0 = expf(z0 - zm), e1 = expf(z1 - zm), e2 = expf(z2 - zm);
    const float inv = 1.0f / (e0 + e1 + e2);
    w[0] = e0 * inv;
    w[1] = e1 * inv;
    w[2] = e2 * inv;
}

// Learned WENO-5 interface value (without p/m) of the upwind-ordered stencil:
// where any smoothness indicator vanishes the Jiang-Shu weights with Table
// tab:weno apply (constant ghost layers keep their exact flux), and so do
// they where the stencil is smooth (min sigma_q >= MLP_GUARD max sigma_q);
// otherwise v2 + sum_q w_q G_q with the network's weights.  The network runs
// in FP32; the candidates are combined in the population precision.
template <typename real>
__device__ __forceinline__ real weno5_learned(const float *__restrict__ th, real v0, real v1, real v2, real v3,
                                              real v4)
{
    const real d01 = v1 - v0, d12 = v2 - v1, d23 = v3 - v2, d34 = v4 - v3;
    const real a1 = d12 - d01, b1 = fma(real(3), d12, -d01);
    const real a2 = d23 - d12, b2 = d12 + d23;
    const real a3 = d34 - d23, b3 = fma(real(-3), d23, d34);
    const real s1 = fma(real(13) * a1, a1, real(3) * b1 * b1);
    const real s2 = fma(real(13) * a2, a2, real(3) * b2 * b2);
    const real s3 = fma(real(13) * a3, a3, real(3) * b3 * b3);
    const real smin = s1 < s2 ? (s1 < s3 ? s1 : s3) : (s2 < s3 ? s2 : s3);
    const real smax = s1 > s2 ? (s1 > s3 ? s1 : s3) : (s2 > s3 ? s2 : s3);
    const bool zero = (a1 == real(0) && b1 == real(0)) || (a2 == real(0) && b2 == real(0)) ||
                      (a3 == real(0) && b3 == real(0));
    if (zero || smin >= real(MLP_GUARD) * smax) return weno5(v0, v1, v2, v3, v4);
    real mx = v0, mn = v0;
    mx = v1 > mx ? v1 : mx;
    mn = v1 < mn ? v1 : mn;
    mx = v2 > mx ? v2 : mx;
    mn = v2 < mn ? v2 : mn;
    mx = v3 > mx ? v3 : mx;
    mn = v3 < mn ? v3 : mn;
    mx = v4 > mx ? v4 : mx;
    mn = v4 < mn ? v4 : mn;
    const real mean = (v0 + v1 + v2 + v3 + v4) * real(0.2);
    const real ir = real(1) / (mx - mn);
    const float x[MLP_IN] = {(float)((v0 - mean) * ir), (float)((v1 - mean) * ir), (float)((v2 - mean) * ir),
                             (float)((v3 - mean) * ir), (float)((v4 - mean) * ir)};
    float w[MLP_OUT];
    mlp_weights(th, x, w);
    const real G1 = fma(real(5.0 / 6.0), d12, real(-1.0 / 3.0) * d01);
    const real G2 = fma(real(1.0 / 3.0), d23, real(1.0 / 6.0) * d12);
    const real G3 = fma(real(2.0 / 3.0), d23, real(-1.0 / 6.0) * d34);
    return fma((real)w[0], G1, fma((real)w[1], G2, fma((real)w[2], G3, v2)));
}

// The same for the compensated FP32 storage: the correction sum_q w_q G_q (the
// interface value minus v2) from the stencil's first differences d01 .. d34,
// which fix the normalised stencil (shift invariant) and the candidates.
__device__ __forceinline__ float weno5_learned_corr(const float *__restrict__ th, float d01, float d12, float d23,
                                                   float d34)
{
    const float a1 = d12 - d01, b1 = fmaf(3.0f, d12, -d01);
    const float a2 = d23 - d12, b2 = d12 + d23;
    const float a3 = d34 - d23, b3 = fmaf(-3.0f, d23, d34);
    const float s1 = fmaf(13.0f * a1, a1, 3.0f * b1 * b1);
    const float s2 = fmaf(13.0f * a2, a2, 3.0f * b2 * b2);
    const float s3 = fmaf(13.0f * a3, a3, 3.0f * b3 * b3);
    const float smin = fminf(s1, fminf(s2, s3)), smax = fmaxf(s1, fmaxf(s2, s3));
    const bool zero = (a1 == 0.0f && b1 == 0.0f) || (a2 == 0.0f && b2 == 0.0f) || (a3 == 0.0f && b3 == 0.0f);
    if (zero || smin >= (float)MLP_GUARD * smax) return weno5_corr(d01, d12, d23, d34);
    // the stencil relative to v0
    const float w1 = d01, w2 = w1 + d12, w3 = w2 + d23, w4 = w3 + d34;
    const float mx = fmaxf(fmaxf(0.0f, w1), fmaxf(fmaxf(w2, w3), w4));
    const float mn = fminf(fminf(0.0f, w1), fminf(fminf(w2, w3), w4));
    const float mean = (((w1 + w2) + w3) + w4) * 0.2f;
    const float ir = 1.0f / (mx - mn);
    const float x[MLP_IN] = {(0.0f - mean) * ir, (w1 - mean) * ir, (w2 - mean) * ir, (w3 - mean) * ir,
                             (w4 - mean) * ir};
    float w[MLP_OUT];
    mlp_weights(th, x, w);
    const float G1 = fmaf(5.0f / 6.0f, d12, (-1.0f / 3.0f) * d01);
    const float G2 = fmaf(1.0f / 3.0f, d23, (1.0f / 6.0f) * d12);
    const float G3 = fmaf(2.0f / 3.0f, d23, (-1.0f / 6.0f) * d34);
    return fmaf(w[0], G1, fmaf(w[1], G2, w[2] * G3));
}

}  // namespace olb
