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

// Whether the network acts on the stencil with first differences d01 .. d34:
// no smoothness indicator vanishes and min sigma_q < MLP_GUARD max sigma_q
// (otherwise Jiang-Shu with Table tab:weno applies).  The decision is that of
// the population precision.  FP64 spares its FP64 pipe (which bounds that
// kernel): the zero test is on the differences' bits, an FP32 pre-check
// decides away from the threshold, and the FP64 indicators that remain are
// compared on the integer pipe (they are >= 0, and their bit patterns order
// like their values; x == 0 of either sign is a zero pattern without the sign
// bit).
template <typename real>
__device__ __forceinline__ bool learned_guard(real d01, real d12, real d23, real d34)
{
    if constexpr (sizeof(real) == 8) {
        // a_q = b_q = 0 exactly when both differences of sub-stencil q are 0
        // (a difference of two numbers is 0 only when they are equal, and an
        // FMA is exact before its one rounding)
        auto z = [](double v) { return (__double_as_longlong(v) << 1) == 0; };
        if ((z(d01) && z(d12)) || (z(d12) && z(d23)) || (z(d23) && z(d34))) return false;
        // FP32 pre-check: each sigma_q is a positive-definite quadratic form in
        // two differences (condition number ~18), so from the differences
        // rounded to FP32 it carries a relative error below ~3e-6; outside a
        // band of 1e-4 around the threshold the FP32 comparison is the FP64
        // one.  Inside the band, or with squares near FP32's range limits,
        // the FP64 test below decides.
        const float e01 = (float)d01, e12 = (float)d12, e23 = (float)d23, e34 = (float)d34;
        const float fa1 = e12 - e01, fb1 = fmaf(3.0f, e12, -e01);
        const float fa2 = e23 - e12, fb2 = e12 + e23;
        const float fa3 = e34 - e23, fb3 = fmaf(-3.0f, e23, e34);
        const float f1 = fmaf(13.0f * fa1, fa1, 3.0f * fb1 * fb1);
        const float f2v = fmaf(13.0f * fa2, fa2, 3.0f * fb2 * fb2);
        const float f3 = fmaf(13.0f * fa3, fa3, 3.0f * fb3 * fb3);
        const float fmn = fminf(f1, fminf(f2v, f3)), fmx = fmaxf(f1, fmaxf(f2v, f3));
        if (fmx > 1e-30f && fmx < 1e30f) {
            if (fmn < (float)(MLP_GUARD * (1.0 - 1e-4)) * fmx) return true;
            if (fmn > (float)(MLP_GUARD * (1.0 + 1e-4)) * fmx) return false;
        }
    }
    const real a1 = d12 - d01, b1 = fma(real(3), d12, -d01);
    const real a2 = d23 - d12, b2 = d12 + d23;
    const real a3 = d34 - d23, b3 = fma(real(-3), d23, d34);
    const real s1 = fma(real(13) * a1, a1, real(3) * b1 * b1);
    const real s2 = fma(real(13) * a2, a2, real(3) * b2 * b2);
    const real s3 = fma(real(13) * a3, a3, real(3) * b3 * b3);
    real smin, smax;
    bool zero;
    if constexpr (sizeof(real) == 8) {
        const long long i1 = __double_as_longlong(s1), i2 = __double_as_longlong(s2), i3 = __double_as_longlong(s3);
        smin = i1 < i2 ? (i1 < i3 ? s1 : s3) : (i2 < i3 ? s2 : s3);
        smax = i1 > i2 ? (i1 > i3 ? s1 : s3) : (i2 > i3 ? s2 : s3);
        auto z = [](real v) { return (__double_as_longlong(v) << 1) == 0; };
        zero = (z(a1) && z(b1)) || (z(a2) && z(b2)) || (z(a3) && z(b3));
    } else {
        smin = fminf(s1, fminf(s2, s3));
        smax = fmaxf(s1, fmaxf(s2, s3));
        zero = (a1 == 0.0f && b1 == 0.0f) || (a2 == 0.0f && b2 == 0.0f) || (a3 == 0.0f && b3 == 0.0f);
    }
    return !zero && smin < real(MLP_GUARD) * smax;
}

// The network's input from the stencil's first differences in FP32: the
// normalised stencil x = (v - mean) / (max - min), taken relative to v0
// (shift invariant); all zero where the network does not act.
__device__ __forceinline__ void learned_input_x(const float e[4], bool acts, float x[MLP_IN])
{
    const float w1 = e[0], w2 = w1 + e[1], w3 = w2 + e[2], w4 = w3 + e[3];
    const float mx = fmaxf(fmaxf(0.0f, w1), fmaxf(fmaxf(w2, w3), w4));
    const float mn = fminf(fminf(0.0f, w1), fminf(fminf(w2, w3), w4));
    const float mean = (((w1 + w2) + w3) + w4) * 0.2f;
    const float ir = acts ? 1.0f / (mx - mn) : 0.0f;
    x[0] = (0.0f - mean) * ir;
    x[1] = (w1 - mean) * ir;
    x[2] = (w2 - mean) * ir;
    x[3] = (w3 - mean) * ir;
    x[4] = (w4 - mean) * ir;
}

// The correction sum_q w_q G_q (the interface value minus v2, Eq. weno5_flux)
// from the network's weights and the first differences, in FP32 (the weights
// carry FP32 error anyway).
__device__ __forceinline__ float learned_corr_from(const float w[MLP_OUT], const float e[4])
{
    const float G1 = fmaf(5.0f / 6.0f, e[1], (-1.0f / 3.0f) * e[0]);
    const float G2 = fmaf(1.0f / 3.0f, e[2], (1.0f / 6.0f) * e[1]);
    const float G3 = fmaf(2.0f / 3.0f, e[2], (-1.0f / 6.0f) * e[3]);
    return fmaf(w[0], G1, fmaf(w[1], G2, w[2] * G3));
}

// The network's correction of a stencil it acts on (per thread).
__device__ __forceinline__ float learned_corr_net(const float *__restrict__ th, const float e[4])
{
    float x[MLP_IN], w[MLP_OUT];
    learned_input_x(e, true, x);
    mlp_weights(th, x, w);
    return learned_corr_from(w, e);
}

// Learned WENO-5 interface value (without p/m) of the upwind-ordered stencil:
// where any smoothness indicator vanishes the Jiang-Shu weights with Table
// tab:weno apply (constant ghost layers keep their exact flux), and so do
// they where the stencil is smooth (min sigma_q >= MLP_GUARD max sigma_q);
// otherwise v2 + sum_q w_q G_q with the network's weights.  The guard is
// taken in the population precision; the network and the correction
// sum_q w_q G_q run in FP32 (the weights carry FP32 error anyway), and the
// correction is added to v2 in the population precision.
template <typename real>
__device__ __forceinline__ real weno5_learned(const float *__restrict__ th, real v0, real v1, real v2, real v3,
                                              real v4)
{
    const real d01 = v1 - v0, d12 = v2 - v1, d23 = v3 - v2, d34 = v4 - v3;
    if (!learned_guard<real>(d01, d12, d23, d34)) {
        // Jiang-Shu on the same differences (the operations of weno5)
        const real q12 = d12 * d12, q23 = d23 * d23;
        return weno5_core(d01, d12, d23, d34, q23, real(2.5) * q12, real(2.5) * q23, v2);
    }
    const float e[4] = {(float)d01, (float)d12, (float)d23, (float)d34};
    return v2 + (real)learned_corr_net(th, e);
}

// The same for the compensated FP32 storage: the correction sum_q w_q G_q (the
// interface value minus v2) from the stencil's first differences d01 .. d34,
// which fix the normalised stencil (shift invariant) and the candidates.
__device__ __forceinline__ float weno5_learned_corr(const float *__restrict__ th, float d01, float d12, float d23,
                                                   float d34)
{
    if (!learned_guard<float>(d01, d12, d23, d34)) return weno5_corr(d01, d12, d23, d34);
    const float e[4] = {d01, d12, d23, d34};
    return learned_corr_net(th, e);
}

// ---------------------------------------------------------------- the network on the tensor pipe
// Inside the stage kernel the 32 lanes of a warp evaluate the network for 32
// stencils at once: layer 1 per lane, the 32 x 32 layer as a matrix product
// on the tensor pipe (mma.sync m16n8k8 with TF32 operands; each operand
// split into a TF32 high part and a TF32 remainder and the product taken as
// hi hi + hi lo + lo hi, accurate to ~2^-21 like an FP32 dot product), layer 3
// and the softmax per stencil.

// scratch floats per warp: one 16 x 8 block of layer-1 outputs (row stride 9)
constexpr int MLP_WARP_SCRATCH = 16 * 9;
// shared memory after the parameters (1348 floats): W2 split into TF32 high
// parts and remainders (2 x 1024 words), then the warps' scratch
constexpr int MLP_W2HI_OFF = 1348, MLP_W2LO_OFF = 1348 + 1024, MLP_SCRATCH_OFF = 1348 + 2048;

__device__ __forceinline__ void tf32_split(float v, unsigned &hi, unsigned &lo)
{
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(v));
    const float r = v - __uint_as_float(hi);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}

// Fill the split copies of W2 after the parameters (all threads of the CTA).
__device__ __forceinline__ void mlp_split_w2(float *th)
{
    unsigned *w2h = reinterpret_cast<unsigned *>(th + MLP_W2HI_OFF);
    unsigned *w2l = reinterpret_cast<unsigned *>(th + MLP_W2LO_OFF);
    for (int i = threadIdx.x; i < MLP_H * MLP_H; i += blockDim.x) tf32_split(th[MLP_W2 + i], w2h[i], w2l[i]);
}

// c += a b for one m16n8k8 tile (row-major A, column-major B, FP32 accumulators).
__device__ __forceinline__ void mma_tf32(float c[4], const unsigned a[4], const unsigned b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Weights w of this lane's stencil x; every lane of the warp must call it,
// from one call site (mma.sync.aligned needs the whole warp at the same
// instruction; lanes whose stencil the network does not act on pass any x and
// ignore w).
// th: parameters in shared memory; sc: this warp's MLP_WARP_SCRATCH floats.
__device__ __forceinline__ void mlp_weights_warp(const float *__restrict__ th, const float x[MLP_IN],
                                                 float w[MLP_OUT], float *sc)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    // layer 2 accumulators: rows = stencils (lanes), 16 per m-tile mt;
    // columns = outputs, 8 per n-tile nt; k = the 32 layer-1 outputs, 8 per
    // step ks, each step's layer-1 outputs computed just before it
    float acc[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.0f;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        float hc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = 8 * ks + q;
            float a = th[MLP_B1 + j];
#pragma unroll
            for (int i = 0; i < MLP_IN; ++i) a = fmaf(th[MLP_W1 + j * MLP_IN + i], x[i], a);
            hc[q] = tanh_fast(a);
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            // the m-tile's 16 lanes put their 8 layer-1 outputs in the scratch
            __syncwarp();
            if ((lane >> 4) == mt)
#pragma unroll
                for (int q = 0; q < 8; ++q) sc[(lane & 15) * 9 + q] = hc[q];
            __syncwarp();
            unsigned ah[4], al[4];
            tf32_split(sc[g * 9 + t], ah[0], al[0]);
            tf32_split(sc[(g + 8) * 9 + t], ah[1], al[1]);
            tf32_split(sc[g * 9 + t + 4], ah[2], al[2]);
            tf32_split(sc[(g + 8) * 9 + t + 4], ah[3], al[3]);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                // B[k][n] = W2[n][k]: k = 8 ks + t (+4), n = 8 nt + g
                const unsigned *w2h = reinterpret_cast<const unsigned *>(th + MLP_W2HI_OFF);
                const unsigned *w2l = reinterpret_cast<const unsigned *>(th + MLP_W2LO_OFF);
                const int i0 = (8 * nt + g) * MLP_H + 8 * ks + t;
                const unsigned bh[2] = {w2h[i0], w2h[i0 + 4]}, bl[2] = {w2l[i0], w2l[i0 + 4]};
                mma_tf32(acc[mt][nt], al, bh);
                mma_tf32(acc[mt][nt], ah, bl);
                mma_tf32(acc[mt][nt], ah, bh);
            }
        }
    }
    // h2 = tanh(acc + b2) and layer 3: accumulator q of (mt, nt) holds stencil
    // 16 mt + g + 8 (q >> 1) = g + 8 m, output 8 nt + 2 t + (q & 1)
    float z[4][MLP_OUT];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int o = 0; o < MLP_OUT; ++o) z[m][o] = 0.0f;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = 8 * nt + 2 * t + (q & 1), m = 2 * mt + (q >> 1);
                const float h2 = tanh_fast(acc[mt][nt][q] + th[MLP_B2 + j]);
#pragma unroll
                for (int o = 0; o < MLP_OUT; ++o) z[m][o] = fmaf(th[MLP_W3 + o * MLP_H + j], h2, z[m][o]);
            }
    // sum over the four lanes of a row group (t = 0..3): every one gets the total
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int o = 0; o < MLP_OUT; ++o) {
            z[m][o] += __shfl_xor_sync(0xffffffffu, z[m][o], 1);
            z[m][o] += __shfl_xor_sync(0xffffffffu, z[m][o], 2);
        }
    // lane (g, t) finishes stencil g + 8 t
    float zz[MLP_OUT];
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) {
        float v = z[0][o];
        v = t == 1 ? z[1][o] : v;
        v = t == 2 ? z[2][o] : v;
        v = t == 3 ? z[3][o] : v;
        zz[o] = v + th[MLP_B3 + o];
    }
    const float zm = fmaxf(zz[0], fmaxf(zz[1], zz[2]));
    const float e0 = expf(zz[0] - zm), e1 = expf(zz[1] - zm), e2 = expf(zz[2] - zm);
    const float inv = 1.0f / (e0 + e1 + e2);
    // stencil F sits in lane F; lane 4 (F mod 8) + F / 8 finished it
    const int src = 4 * (lane & 7) + (lane >> 3);
    w[0] = __shfl_sync(0xffffffffu, e0 * inv, src);
    w[1] = __shfl_sync(0xffffffffu, e1 * inv, src);
    w[2] = __shfl_sync(0xffffffffu, e2 * inv, src);
}

}  // namespace olb
