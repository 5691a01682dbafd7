// olb_kernels.cuh -- device building blocks shared by the stage kernel
// (olb_fused.cuh): stencil coefficients, WENO-5, equilibrium factors, Kahan
// sums, and the initialisation / moment-output / conversion kernels,
// templated on the population precision (double, or float with
// Kahan-compensated moments).
#pragma once

#include "olb_internal.cuh"

namespace olb {

// ---------------------------------------------------------------- stencils
// Weights w^{|l|,|m|} of the 49-point gradient (Eq. stencil_grad).
__host__ __device__ constexpr double grad_w(int l, int m)
{
    return (l == 1 && m == 0) || (l == 0 && m == 1) ? 31.0 / 70.0
         : (l == 1 && m == 1)                       ? 27.0 / 140.0
         : (l == 2 && m == 1) || (l == 1 && m == 2) ? -3.0 / 70.0
         : (l == 2 && m == 2)                       ? 3.0 / 560.0
         : (l == 3 && m == 0) || (l == 0 && m == 3) ? -1.0 / 630.0
         : (l == 3 && m == 1) || (l == 1 && m == 3) ? 1.0 / 280.0
                                                    : 0.0;
}

// Coefficient of n_{i+l, j+m}, l > 0, in d/dx (Laplacian n) (Eq. stencil_glap,
// the entry in row |m| and column |l| of the printed matrix, with the
// 4th-order-consistent c1 = -17/2160 and c4 = -59/540); n_{i-l, j+m} takes
// the opposite sign.
__host__ __device__ constexpr double glap_c(int am, int l)
{
    return (am == 3 && l == 3) ? -17.0 / 2160.0   // c1
         : (am == 0 && l == 3) ? -59.0 / 540.0    // c4
         : (am == 2 && l == 2) ? 13.0 / 120.0     // c6
         : (am == 1 && l == 2) ? -7.0 / 30.0      // c7
         : (am == 0 && l == 2) ? 5.0 / 4.0        // c8
         : (am == 2 && l == 1) ? -7.0 / 60.0      // c10
         : (am == 1 && l == 1) ? 187.0 / 240.0    // c11
         : (am == 0 && l == 1) ? -59.0 / 20.0     // c12
                               : 0.0;
}

// ---------------------------------------------------------------- WENO-5
// Reciprocal of d > 0 in FP64: the hardware approximation rcp.approx.ftz.f64
// as a seed, refined by two Newton-Raphson steps r <- r (2 - d r) (each
// doubles the number of correct bits), written as fused multiply-adds.
// Flushes subnormal d to zero (d < 2.2e-308 gives +inf).
__device__ __forceinline__ double recip_nr(double d)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    return fma(r, e, r);
}

// v0..v4 = f_{i-2} .. f_{i+2} in the upwind orientation; returns the WENO-5
// interface value sum_q wbar_q Fhat^q (without p/m).
//
// In terms of the first differences d01 = v1 - v0, ..., d34 = v4 - v3, the
// indicators of Eq. weno5_sigma (13/12 a_q^2 + 1/4 b_q^2, a_q and b_q linear
// in two neighbouring differences) are positive-definite quadratic forms:
//   12 sigma_1 / 16 = d01^2 - 11/4 d01 d12 + 5/2 d12^2
//   12 sigma_2 / 16 = d12^2 + d23^2 - 5/4 d12 d23 = d12 (d12 - 5/4 d23) + d23^2
//   12 sigma_3 / 16 = d34^2 - 11/4 d23 d34 + 5/2 d23^2
// (the weights only depend on ratios of the sigma_q, so the common factor
// 12/16 is dropped), and 6 (Fhat^q - v2) of Eq. weno5_flux are
//   6 G_1 = 5 d12 - 2 d01,  6 G_2 = d12 + 2 d23,  6 G_3 = 4 d23 - d34.
// A form vanishes exactly when both of its differences do (the case of
// Table tab:weno).
//
// Weights: wbar_q is proportional to delta_q / sigma_q^2.  Multiplying every
// term by 10 (sigma_1 sigma_2 sigma_3)^2 gives weights proportional to
// A_q = 10 delta_q (prod_{r != q} sigma_r)^2, which needs one reciprocal,
// equals the table row for a single vanishing indicator, and is 0/0 only when
// two or three vanish; those cases take Table tab:weno (the ideal weights of
// the vanishing set).  If the products underflow without an exact zero the
// min-scaled form delta_q (s/sigma_q)^2 is used instead.
//
// weno5_core takes the first differences, q23 = d23^2 and h12 = 2.5 d12^2,
// h23 = 2.5 d23^2; weno5 (one face) and weno5_strip
// (consecutive faces, carrying those values from face to face) both end in
// it, with the same operations on the same operands, so they agree bit for bit.
__device__ __forceinline__ double weno5_core(double d01, double d12, double d23, double d34, double q23, double h12,
                                             double h23, double v2)
{
    const double s1 = fma(d01, fma(-2.75, d12, d01), h12);
    const double s2 = fma(d12, fma(-1.25, d23, d12), q23);
    const double s3 = fma(d34, fma(-2.75, d23, d34), h23);
    const double G1 = fma(5.0, d12, -2.0 * d01);
    const double G2 = fma(2.0, d23, d12);
    const double G3 = fma(4.0, d23, -d34);
    const double p1 = s2 * s3, p2 = s1 * s3, p3 = s1 * s2;
    double A1 = p1 * p1, A2 = (6.0 * p2) * p2, A3 = (3.0 * p3) * p3;
    double den = A1 + A2 + A3;
    // den >= 0 (or NaN): its bit pattern orders like its value, so the test
    // for a normal den runs on the integer pipe
    if (__double_as_longlong(den) <= 0x0010000000000000LL) {
        // two or three indicators vanish (Table tab:weno: the ideal weights of
        // the vanishing set), or the products underflow (min-scaled weights);
        // only the weights diverge, the combination below is shared
        if (s1 == 0.0 || s2 == 0.0 || s3 == 0.0) {
            A1 = (s1 == 0.0) ? 1.0 : 0.0;
            A2 = (s2 == 0.0) ? 6.0 : 0.0;
            A3 = (s3 == 0.0) ? 3.0 : 0.0;
        } else {
            const double s = fmin(s1, fmin(s2, s3));
            const double r1 = s / s1, r2 = s / s2, r3 = s / s3;
            A1 = r1 * r1;
            A2 = (6.0 * r2) * r2;
            A3 = (3.0 * r3) * r3;
        }
        den = A1 + A2 + A3;
    }
    return fma(fma(A1, G1, fma(A2, G2, A3 * G3)), recip_nr(6.0 * den), v2);
}
__device__ __forceinline__ double weno5(double v0, double v1, double v2, double v3, double v4)
{
    const double d01 = v1 - v0, d12 = v2 - v1, d23 = v3 - v2, d34 = v4 - v3;
    const double q12 = d12 * d12, q23 = d23 * d23;
    return weno5_core(d01, d12, d23, d34, q23, 2.5 * q12, 2.5 * q23, v2);
}

// FP32 form (same forms and candidates): the products of four squared
// indicators underflow in single precision, so the weights are always the
// min-scaled 10 delta_q (s/sigma_q)^2 (same normalised weights), with Table
// tab:weno when an indicator vanishes.
__device__ __forceinline__ float weno5_core(float d01, float d12, float d23, float d34, float q23, float h12, float h23,
                                            float v2)
{
    const float s1 = fmaf(d01, fmaf(-2.75f, d12, d01), h12);
    const float s2 = fmaf(d12, fmaf(-1.25f, d23, d12), q23);
    const float s3 = fmaf(d34, fmaf(-2.75f, d23, d34), h23);
    const float G1 = fmaf(5.0f, d12, -2.0f * d01);
    const float G2 = fmaf(2.0f, d23, d12);
    const float G3 = fmaf(4.0f, d23, -d34);
    float w1, w2, w3;
    const float s = fminf(s1, fminf(s2, s3));
    if (s > 0.0f) {
        const float r1 = __fdividef(s, s1), r2 = __fdividef(s, s2), r3 = __fdividef(s, s3);
        w1 = r1 * r1;
        w2 = (6.0f * r2) * r2;
        w3 = (3.0f * r3) * r3;
    } else {
        w1 = (s1 == 0.0f) ? 1.0f : 0.0f;
        w2 = (s2 == 0.0f) ? 6.0f : 0.0f;
        w3 = (s3 == 0.0f) ? 3.0f : 0.0f;
    }
    return fmaf(fmaf(w1, G1, fmaf(w2, G2, w3 * G3)), __fdividef(1.0f, 6.0f * (w1 + w2 + w3)), v2);
}
__device__ __forceinline__ float weno5(float v0, float v1, float v2, float v3, float v4)
{
    const float d01 = v1 - v0, d12 = v2 - v1, d23 = v3 - v2, d34 = v4 - v3;
    const float q12 = d12 * d12, q23 = d23 * d23;
    return weno5_core(d01, d12, d23, d34, q23, 2.5f * q12, 2.5f * q23, v2);
}

// S consecutive faces along a row or column, in the upwind direction: the
// stencil v_0 .. v_4 of face j is p[(j + m) step], m = 0..4, and its value
// goes to out[j ostep].  Neighbouring faces share three first differences
// and one scaled square, which are carried instead of recomputed (4 fewer
// operations per face after the first).
template <int S, typename real>
__device__ __forceinline__ void weno5_strip(const real *p, int step, real *out, int ostep)
{
    real v2 = p[2 * step], v3 = p[3 * step];
    const real v1 = p[step];
    real d01 = v1 - p[0], d12 = v2 - v1, d23 = v3 - v2;
    real h12 = real(2.5) * (d12 * d12);
#pragma unroll
    for (int j = 0; j < S; ++j) {
        const real v4 = p[(j + 4) * step];
        const real d34 = v4 - v3;
        const real q23 = d23 * d23, h23 = real(2.5) * q23;
        out[j * ostep] = weno5_core(d01, d12, d23, d34, q23, h12, h23, v2);
        d01 = d12;
        d12 = d23;
        d23 = d34;
        h12 = h23;
        v2 = v3;
        v3 = v4;
    }
}

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ int wrap(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

// Even extension of a field about both wall faces (Sec. 3.4.3): period 2 nx.
__device__ __forceinline__ int reflect(int i, int n)
{
    int r = wrap(i, 2 * n);
    return r >= n ? 2 * n - 1 - r : r;
}

// Equilibrium factors g_k(u, T), k = 0..4 (Eq. g_alpha with m = 1):
// g_k = sum_l w_k He_l(p_k) c_l with c_l = sum_s (T-1)^s u^(l-2s)/(2^s s!(l-2s)!).
template <typename real>
__device__ __forceinline__ void eq_factors(const Tab<real> &t, real u, real T, real g[NQ])
{
    const real th = T - real(1);
    const real u2 = u * u;
    const real c1 = u;
    const real c2 = real(0.5) * (u2 + th);
    const real c3 = u * fma(u2, real(1.0 / 6.0), real(0.5) * th);
    const real c4 = fma(u2 * u2, real(1.0 / 24.0), fma(real(0.25) * th, u2, real(0.125) * th * th));
#pragma unroll
    for (int k = 0; k < NQ; ++k)
        g[k] = fma(t.wHe[k][4], c4, fma(t.wHe[k][3], c3, fma(t.wHe[k][2], c2, fma(t.wHe[k][1], c1, t.wHe[k][0]))));
}

// Kahan-compensated accumulation (FP32 variant).
struct Kahan {
    float s, c;
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// ---------------------------------------------------------------- double-float
// A value held as the unevaluated sum hi + lo of two floats (~44 significant
// bits), built from error-free transformations: Knuth's TwoSum (a + b = s + e
// exactly), Dekker's Fast2Sum (the same for |a| >= |b|) and the exact product
// a b = p + e with e = fma(a, b, -p).  Division takes one correction step
// with the exact residual.  Used for the FP32 variant's moment recovery, so
// that the low-rate FP64 pipe stays out of the FP32 stage kernel.  Relies on
// the build's -fmad=false: no product or sum here may be contracted.
struct f2 {
    float hi, lo;
};
__device__ __forceinline__ f2 two_sum(float a, float b)
{
    const float s = a + b, bv = s - a;
    return {s, (a - (s - bv)) + (b - bv)};
}
__device__ __forceinline__ f2 fast_two_sum(float a, float b)
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ f2 f2_from_kahan(const Kahan &k) { return fast_two_sum(k.s, -k.c); }
__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    // both parts summed exactly, then renormalised (accurate under cancellation)
    f2 s = two_sum(a.hi, b.hi);
    const f2 t = two_sum(a.lo, b.lo);
    s = fast_two_sum(s.hi, s.lo + t.hi);
    return fast_two_sum(s.hi, s.lo + t.lo);
}
__device__ __forceinline__ f2 f2_neg(f2 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.hi, -p);
    return fast_two_sum(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}
__device__ __forceinline__ f2 f2_scale(f2 a, float s) { return {a.hi * s, a.lo * s}; }  // s a power of 2
__device__ __forceinline__ f2 f2_div(f2 a, f2 b)
{
    const float r = __frcp_rn(b.hi);
    const float q1 = a.hi * r;
    // residual a - b q1 (b.hi q1 exactly by fma), then q2 = residual / b
    const float p = b.hi * q1;
    const float pe = fmaf(b.hi, q1, -p);
    const f2 res = f2_add(a, f2_neg(fast_two_sum(p, fmaf(b.lo, q1, pe))));
    return fast_two_sum(q1, res.hi * r);
}
__device__ __forceinline__ f2 f2_of(double v)
{
    const float hi = __double2float_rn(v);
    return {hi, __double2float_rn(v - (double)hi)};
}

// Moments of the 25 populations at one node in FP64: n, jx, jy, e.
template <typename real>
__device__ __forceinline__ void node_sums(const real *__restrict__ f, long long plane, long long o,
                                          const Tab<real> &t, double &n, double &jx, double &jy, double &e);

template <>
__device__ __forceinline__ void node_sums<double>(const double *__restrict__ f, long long plane, long long o,
                                                  const Tab<double> &t, double &n, double &jx, double &jy,
                                                  double &e)
{
    double sx[NQ], sy[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) sy[k] = 0.0;
#pragma unroll
    for (int k1 = 0; k1 < NQ; ++k1) {
        double r = 0.0;
#pragma unroll
        for (int k2 = 0; k2 < NQ; ++k2) {
            const double v = __ldg(f + (NQ * k1 + k2) * plane + o);
            r += v;
            sy[k2] += v;
        }
        sx[k1] = r;
    }
    n = jx = jy = e = 0.0;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        n += sx[k];
        jx = fma(t.R[k], sx[k], jx);
        jy = fma(t.R[k], sy[k], jy);
        e = fma(t.R2[k], sx[k] + sy[k], e);
    }
}

template <>
__device__ __forceinline__ void node_sums<float>(const float *__restrict__ f, long long plane, long long o,
                                                 const Tab<float> &t, double &n, double &jx, double &jy,
                                                 double &e)
{
    Kahan kn{0.f, 0.f}, kx{0.f, 0.f}, ky{0.f, 0.f}, ke{0.f, 0.f};
#pragma unroll
    for (int k1 = 0; k1 < NQ; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < NQ; ++k2) {
            const float v = __ldg(f + (NQ * k1 + k2) * plane + o);
            kn.add(v);
            kx.add(t.R[k1] * v);
            ky.add(t.R[k2] * v);
            ke.add((t.R2[k1] + t.R2[k2]) * v);
        }
    n = kn.value();
    jx = kx.value();
    jy = ky.value();
    e = ke.value();
}

// ---------------------------------------------------------------- init / output
template <typename real>
__global__ void k_init(real *__restrict__ f, const double *__restrict__ n, const double *__restrict__ ux,
                       const double *__restrict__ uy, const double *__restrict__ T, Geo g, Tab<real> t)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)g.nx * g.ny) return;
    const int j = (int)(idx / g.nx), i = (int)(idx - (long long)j * g.nx);
    const long long o = (long long)j * g.pitch + i;
    real gx[NQ], gy[NQ];
    eq_factors<real>(t, (real)ux[idx], (real)T[idx], gx);
    eq_factors<real>(t, (real)uy[idx], (real)T[idx], gy);
    const real nn = (real)n[idx];
#pragma unroll
    for (int k1 = 0; k1 < NQ; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < NQ; ++k2) f[(NQ * k1 + k2) * g.plane + o] = nn * gx[k1] * gy[k2];
}

template <typename real>
__global__ void k_moments_out(const real *__restrict__ f, double *__restrict__ on, double *__restrict__ oux,
                              double *__restrict__ ouy, double *__restrict__ oT, Geo g, Tab<real> t)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long N = (long long)g.nx * g.ny;
    if (idx >= N) return;
    const int j = (int)(idx / g.nx), i = (int)(idx - (long long)j * g.nx);
    const long long o = (long long)j * g.pitch + i;
    double n, jx, jy, e;
    node_sums<real>(f, g.plane, o, t, n, jx, jy, e);
    const double ux = jx / n, uy = jy / n;
    if (on) on[idx] = n;
    if (oux) oux[idx] = ux;
    if (ouy) ouy[idx] = uy;
    if (oT) oT[idx] = 0.5 * (e / n - fma(ux, ux, uy * uy));
}

template <typename real>
__global__ void k_to_f64(const real *__restrict__ f, double *__restrict__ dst, Geo g)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long N = (long long)g.nx * g.ny;
    if (idx >= N * NK) return;
    const int k = (int)(idx / N);
    const long long q = idx - (long long)k * N;
    const int j = (int)(q / g.nx), i = (int)(q - (long long)j * g.nx);
    dst[idx] = (double)f[k * g.plane + (long long)j * g.pitch + i];
}

template <typename real>
__global__ void k_from_f64(real *__restrict__ f, const double *__restrict__ src, Geo g)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long N = (long long)g.nx * g.ny;
    if (idx >= N * NK) return;
    const int k = (int)(idx / N);
    const long long q = idx - (long long)k * N;
    const int j = (int)(q / g.nx), i = (int)(q - (long long)j * g.nx);
    f[k * g.plane + (long long)j * g.pitch + i] = (real)src[idx];
}

// ---------------------------------------------------------------- launchers
// Initialisation, moment output and FP64 conversion kernels (one instance
// per precision, defined in olb_fp64.cu / olb_fp32.cu).
#define OLB_DEFINE_AUX_LAUNCHERS(real)                                                                       \
    cudaError_t launch_init(real *f, const double *n, const double *ux, const double *uy, const double *T,   \
                            const Geo &g, const Tab<real> &t, cudaStream_t s)                                \
    {                                                                                                        \
        const long long N = (long long)g.nx * g.ny;                                                          \
        k_init<real><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(f, n, ux, uy, T, g, t);                     \
        return cudaGetLastError();                                                                           \
    }                                                                                                        \
    cudaError_t launch_moments_out(const real *f, double *n, double *ux, double *uy, double *T,              \
                                   const Geo &g, const Tab<real> &t, cudaStream_t s)                         \
    {                                                                                                        \
        const long long N = (long long)g.nx * g.ny;                                                          \
        k_moments_out<real><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(f, n, ux, uy, T, g, t);              \
        return cudaGetLastError();                                                                           \
    }                                                                                                        \
    cudaError_t launch_to_f64(const real *f, double *dst, const Geo &g, cudaStream_t s)                      \
    {                                                                                                        \
        const long long M = (long long)g.nx * g.ny * NK;                                                     \
        k_to_f64<real><<<(unsigned)((M + 255) / 256), 256, 0, s>>>(f, dst, g);                               \
        return cudaGetLastError();                                                                           \
    }                                                                                                        \
    cudaError_t launch_from_f64(real *f, const double *src, const Geo &g, cudaStream_t s)                    \
    {                                                                                                        \
        const long long M = (long long)g.nx * g.ny * NK;                                                     \
        k_from_f64<real><<<(unsigned)((M + 255) / 256), 256, 0, s>>>(f, src, g);                             \
        return cudaGetLastError();                                                                           \
    }

}  // namespace olb
