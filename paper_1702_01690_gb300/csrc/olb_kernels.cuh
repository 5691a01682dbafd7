// olb_kernels.cuh -- device building blocks shared by the stage kernel
// (olb_fused.cuh): stencil coefficients, WENO-5, equilibrium factors,
// double-float arithmetic, and the initialisation / moment-output /
// conversion / global-sum kernels, templated on the population precision
// (double, or float stored as hi + lo pairs).
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

// The same with one Newton-Raphson step: measured on a GB300 over 2^20
// random d, the seed is within 2^-19.9 of 1/d and one step within 2^-39.9
// (9.8e-13).  Used for the normalisation of the WENO weights only, where a
// relative error of 1e-12 in the weights moves a face value by 1e-12 of its
// correction (the face value minus its upwind node), far below rounding of
// the state; moments and pressures keep recip_nr.
__device__ __forceinline__ double recip_nr1(double d)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    return fma(r, fma(-d, r, 1.0), r);
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
// A_q = 10 delta_q (prod_{r != q} sigma_r)^2, which needs one reciprocal
// (recip_nr1),
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
    return fma(fma(A1, G1, fma(A2, G2, A3 * G3)), recip_nr1(6.0 * den), v2);
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

// The same factors split by Hermite order parity: ge_k from the even orders
// l = 0, 2, 4 and go_k from the odd ones l = 1, 3 (g_k = ge_k + go_k).  The
// tables give w_k He_l(p_k) exactly even or odd under p_k -> -p_k
// (k -> 4 - k), and ge, go are formed by the same operations on those values,
// so ge_{4-k} = ge_k and go_{4-k} = -go_k hold exactly, after rounding: a sum
// over p of p ge (the momentum of the symmetric part) is exactly zero.
__device__ __forceinline__ void eq_factors_split(const Tab<float> &t, float u, float2 T, float ge[NQ], float go[NQ])
{
    // T - 1 from the pair T = hi + lo (hi - 1 is exact for 1/2 <= hi <= 2)
    const float th = (T.x - 1.0f) + T.y;
    const float u2 = u * u;
    const float c2 = 0.5f * (u2 + th);
    const float c3 = u * fmaf(u2, 1.0f / 6.0f, 0.5f * th);
    const float c4 = fmaf(u2 * u2, 1.0f / 24.0f, fmaf(0.25f * th, u2, 0.125f * th * th));
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        ge[k] = fmaf(t.wHe[k][4], c4, fmaf(t.wHe[k][2], c2, t.wHe[k][0]));
        go[k] = fmaf(t.wHe[k][3], c3, t.wHe[k][1] * u);
    }
}

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

// ---------------------------------------------------------------- compensated FP32 storage
// The FP32 variant stores every population as a pair hi + lo of floats (hi
// the value rounded to FP32, lo the remainder).  A stage increment dt L is far
// below the FP32 resolution of f on fine grids (1e-7 .. 1e-5 of f), so plain
// FP32 storage would round most of it away; the pair keeps it.  The arithmetic
// stays FP32: first differences of neighbouring pairs,
// (h1 - h0) + (l1 - l0), are accurate to FP32 rounding of the difference
// itself (h1 - h0 is exact for neighbouring values of the same sign within a
// factor 2, Sterbenz), so fluxes, whose differences are all that the
// advection sees, keep their relative accuracy; the RK-3 combination is done
// in double-float arithmetic.
__device__ __forceinline__ float pdiff(float h1, float l1, float h0, float l0) { return (h1 - h0) + (l1 - l0); }

// a + x for a pair a and a float x (|x| anything), renormalised.
__device__ __forceinline__ f2 f2_add_f(f2 a, float x)
{
    const f2 s = two_sum(a.hi, x);
    return fast_two_sum(s.hi, s.lo + a.lo);
}

// c a for a double-float constant c and a pair a (both parts of c a formed
// with exact products where it matters): unnormalised hi + lo.
__device__ __forceinline__ f2 f2_cmul(f2 c, float ah, float al)
{
    const float p = c.hi * ah;
    const float e = fmaf(c.hi, ah, -p);
    return {p, fmaf(c.hi, al, fmaf(c.lo, ah, e))};
}

// Sum of a row of five pairs as a double-float value: TwoSum of the hi parts,
// their rounding errors and the lo parts gathered in one float.
__device__ __forceinline__ f2 pair_sum5(const float h[NQ], const float l[NQ])
{
    float s = h[0], e = l[0];
#pragma unroll
    for (int k = 1; k < NQ; ++k) {
        const f2 t = two_sum(s, h[k]);
        s = t.hi;
        e += t.lo + l[k];
    }
    return fast_two_sum(s, e);
}

// Compensated FP32: the face value v2 + c of the upwind-ordered stencil is
// kept as v2 (a stored pair) and the correction c = sum_q wbar_q (Fhat^q - v2)
// of Eq. weno5_flux, which depends on the first differences only; the stage
// kernel stores c and takes v2 from the populations.
__device__ __forceinline__ float weno5_corr(float d01, float d12, float d23, float d34)
{
    const float q12 = d12 * d12, q23 = d23 * d23;
    return weno5_core(d01, d12, d23, d34, q23, 2.5f * q12, 2.5f * q23, 0.0f);
}

// weno5_strip for pairs: the stencil of face j is (ph, pl)[(j + m) step],
// m = 0..4, the corrections go to out[j ostep]; the first differences of the
// pairs are carried from face to face.
template <int S>
__device__ __forceinline__ void weno5_strip_c(const float *ph, const float *pl, int step, float *out, int ostep)
{
    float d01 = pdiff(ph[step], pl[step], ph[0], pl[0]);
    float d12 = pdiff(ph[2 * step], pl[2 * step], ph[step], pl[step]);
    float d23 = pdiff(ph[3 * step], pl[3 * step], ph[2 * step], pl[2 * step]);
    float h12 = 2.5f * (d12 * d12);
#pragma unroll
    for (int j = 0; j < S; ++j) {
        const float d34 = pdiff(ph[(j + 4) * step], pl[(j + 4) * step], ph[(j + 3) * step], pl[(j + 3) * step]);
        const float q23 = d23 * d23, h23 = 2.5f * q23;
        out[j * ostep] = weno5_core(d01, d12, d23, d34, q23, h12, h23, 0.0f);
        d01 = d12;
        d12 = d23;
        d23 = d34;
        h12 = h23;
    }
}

// FP32: the symmetric part s_kappa = Ex[k1] gy[k2] of the equilibrium, as
// the stage kernel rounds it (Ex = n ge(u_x), gy = ge(u_y), eq_factors_split),
// carries the node's mass n and energy e = sum |p|^2 f only to FP32 rounding
// (~1e-7 n); relaxing towards it would create or destroy mass and energy at
// that rate every stage.  eq_correction returns alpha, beta of the correction
// c_kappa = W_k1 W_k2 (alpha + beta |p_kappa|^2 + gamma (p_x^2 - p_y^2)),
// symmetric in p (no momentum), with sum_kappa c = sum s - n,
// sum |p|^2 c = sum |p|^2 s - e and sum (p_x^2 - p_y^2) c equal to the
// defect of that moment, from the Gauss-Hermite moments sum W W = 1,
// sum W W |p|^2 = 2, sum W W |p|^4 = 8: alpha + 2 beta = D_m,
// 2 alpha + 8 beta = D_e.  The sums of the 25 rounded
// products are exact (TwoSum); rows and columns 3, 4 equal rows and columns
// 1, 0 (ge is exactly even), and R^2 of the middle root is 0.
__device__ __forceinline__ f2 exact_sum5(float a0, float a1, float a2, float a3, float a4)
{
    float s = a0, e = 0.0f;
    const float a[4] = {a1, a2, a3, a4};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const f2 t = two_sum(s, a[k]);
        s = t.hi;
        e += t.lo;
    }
    return fast_two_sum(s, e);
}
__device__ __forceinline__ void eq_correction(const Tab<float> &t, const float Ex[NQ], const float gy[NQ], float2 n,
                                              float2 e, float ux, float uy, float &alpha, float &beta, float &gamma)
{
    float P[NQ][NQ];
#pragma unroll
    for (int k1 = 0; k1 < NQ; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < NQ; ++k2) P[k1][k2] = Ex[k1] * gy[k2];
    const f2 r0 = exact_sum5(P[0][0], P[0][1], P[0][2], P[0][3], P[0][4]);
    const f2 r1 = exact_sum5(P[1][0], P[1][1], P[1][2], P[1][3], P[1][4]);
    const f2 r2 = exact_sum5(P[2][0], P[2][1], P[2][2], P[2][3], P[2][4]);
    const f2 c0 = exact_sum5(P[0][0], P[1][0], P[2][0], P[3][0], P[4][0]);
    const f2 c1 = exact_sum5(P[0][1], P[1][1], P[2][1], P[3][1], P[4][1]);
    const f2 mass = f2_add(f2_scale(f2_add(r0, r1), 2.0f), r2);
    const f2 R24{t.R2[4], t.R2lo[4]}, R23{t.R2[3], t.R2lo[3]};
    const f2 s4 = f2_add(r0, c0), s3 = f2_add(r1, c1);
    const f2 ea = f2_cmul(R24, s4.hi, s4.lo), eb = f2_cmul(R23, s3.hi, s3.lo);
    const f2 energy = f2_scale(f2_add(fast_two_sum(ea.hi, ea.lo), fast_two_sum(eb.hi, eb.lo)), 2.0f);
    const f2 dm = f2_add(mass, f2{-n.x, -n.y}), de = f2_add(energy, f2{-e.x, -e.y});
    const float Dm = dm.hi + dm.lo, De = de.hi + de.lo;
    beta = 0.25f * fmaf(-2.0f, Dm, De);
    alpha = fmaf(2.0f, Dm, -0.5f * De);
    // the anisotropic second moment sum (p_x^2 - p_y^2) s, whose target is
    // n (u_x^2 - u_y^2), rounds the same way; gamma (p_x^2 - p_y^2) W W
    // (sum W W (p_x^2 - p_y^2)^2 = 4, orthogonal to the two terms above)
    // removes that defect too, so that relaxation keeps P_xx - P_yy
    const f2 a4 = f2_add(r0, f2{-c0.hi, -c0.lo}), a3 = f2_add(r1, f2{-c1.hi, -c1.lo});
    const f2 xa = f2_cmul(R24, a4.hi, a4.lo), xb = f2_cmul(R23, a3.hi, a3.lo);
    const f2 an = f2_scale(f2_add(fast_two_sum(xa.hi, xa.lo), fast_two_sum(xb.hi, xb.lo)), 2.0f);
    const float Da = (an.hi - n.x * (ux * ux - uy * uy)) + an.lo;
    gamma = 0.25f * Da;
}

// Moments of the 25 populations at one node in FP64: n, jx, jy, e (FP32
// storage: hi + lo of each population, summed in FP64; output kernels only).
template <typename real>
__device__ __forceinline__ void node_sums(const real *__restrict__ f, long long plane, long long o,
                                          const Tab<double> &t, double &n, double &jx, double &jy, double &e)
{
    double sx[NQ], sy[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) sy[k] = 0.0;
#pragma unroll
    for (int k1 = 0; k1 < NQ; ++k1) {
        double r = 0.0;
#pragma unroll
        for (int k2 = 0; k2 < NQ; ++k2) {
            const long long q = (NQ * k1 + k2) * plane + o;
            double v = (double)__ldg(f + q);
            if constexpr (sizeof(real) == 4) v += (double)__ldg(f + NK * plane + q);
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

// Store the FP64 value v of population plane offset q: FP64 as is, FP32 as
// the pair hi + lo.
__device__ __forceinline__ void store_pop(double *f, long long, long long q, double v) { f[q] = v; }
__device__ __forceinline__ void store_pop(float *f, long long plane, long long q, double v)
{
    const float hi = __double2float_rn(v);
    f[q] = hi;
    f[NK * plane + q] = __double2float_rn(v - (double)hi);
}
__device__ __forceinline__ double load_pop(const double *f, long long, long long q) { return f[q]; }
__device__ __forceinline__ double load_pop(const float *f, long long plane, long long q)
{
    return (double)f[q] + (double)f[NK * plane + q];
}

// ---------------------------------------------------------------- init / output
// f = f^eq(n, u, T) (Eq. feq), evaluated in FP64 for both storages.
template <typename real>
__global__ void k_init(real *__restrict__ f, const double *__restrict__ n, const double *__restrict__ ux,
                       const double *__restrict__ uy, const double *__restrict__ T, Geo g, Tab<double> t)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)g.nx * g.ny) return;
    const int j = (int)(idx / g.nx), i = (int)(idx - (long long)j * g.nx);
    const long long o = (long long)j * g.pitch + i;
    double gx[NQ], gy[NQ];
    eq_factors<double>(t, ux[idx], T[idx], gx);
    eq_factors<double>(t, uy[idx], T[idx], gy);
    const double nn = n[idx];
#pragma unroll
    for (int k1 = 0; k1 < NQ; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < NQ; ++k2) store_pop(f, g.plane, (NQ * k1 + k2) * g.plane + o, nn * gx[k1] * gy[k2]);
}

template <typename real>
__global__ void k_moments_out(const real *__restrict__ f, double *__restrict__ on, double *__restrict__ oux,
                              double *__restrict__ ouy, double *__restrict__ oT, Geo g, Tab<double> t)
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
    dst[idx] = load_pop(f, g.plane, k * g.plane + (long long)j * g.pitch + i);
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
    store_pop(f, g.plane, k * g.plane + (long long)j * g.pitch + i, src[idx]);
}

// Global sums in FP64 (olb_totals), pass 1: each of TOTALS_BLOCKS blocks
// takes the nodes idx = block*threads + thread + m*(blocks*threads), sums the
// node moments n, n u_x, n u_y, e = sum |p|^2/2 f in FP64 per thread, then
// over the block in a fixed tree order, and writes 4 partial sums.  Pass 2
// (one block) adds the partials in a fixed order and scales by ds^2.  The
// order depends only on the grid size: results are reproducible bit for bit.
template <typename real>
__global__ void __launch_bounds__(TOTALS_THREADS) k_totals(const real *__restrict__ f, double *__restrict__ partial,
                                                           Geo g, Tab<double> t)
{
    __shared__ double red[4][TOTALS_THREADS];
    const long long N = (long long)g.nx * g.ny;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long idx = (long long)blockIdx.x * TOTALS_THREADS + threadIdx.x; idx < N;
         idx += (long long)TOTALS_BLOCKS * TOTALS_THREADS) {
        const int j = (int)(idx / g.nx), i = (int)(idx - (long long)j * g.nx);
        double n, jx, jy, e;
        node_sums<real>(f, g.plane, (long long)j * g.pitch + i, t, n, jx, jy, e);
        acc[0] += n;
        acc[1] += jx;
        acc[2] += jy;
        acc[3] += 0.5 * e;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = TOTALS_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) partial[(long long)blockIdx.x * 4 + threadIdx.x] = red[threadIdx.x][0];
}

static __global__ void __launch_bounds__(TOTALS_THREADS) k_totals_final(const double *__restrict__ partial,
                                                                 double *__restrict__ out, double area)
{
    __shared__ double red[4][TOTALS_THREADS];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < TOTALS_BLOCKS; b += TOTALS_THREADS)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += partial[4 * b + q];
#pragma unroll
    for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = TOTALS_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[threadIdx.x] = red[threadIdx.x][0] * area;
}

// ---------------------------------------------------------------- launchers
// Initialisation, moment output and FP64 conversion kernels (one instance
// per precision, defined in olb_fp64.cu / olb_fp32.cu).
#define OLB_DEFINE_AUX_LAUNCHERS(real)                                                                       \
    cudaError_t launch_init(real *f, const double *n, const double *ux, const double *uy, const double *T,   \
                            const Geo &g, const Tab<double> &t, cudaStream_t s)                              \
    {                                                                                                        \
        const long long N = (long long)g.nx * g.ny;                                                          \
        k_init<real><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(f, n, ux, uy, T, g, t);                     \
        return cudaGetLastError();                                                                           \
    }                                                                                                        \
    cudaError_t launch_moments_out(const real *f, double *n, double *ux, double *uy, double *T,              \
                                   const Geo &g, const Tab<double> &t, cudaStream_t s)                       \
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
    }                                                                                                        \
    cudaError_t launch_totals(const real *f, double *partial, double *out, const Geo &g,                     \
                              const Tab<double> &t, cudaStream_t s)                                          \
    {                                                                                                        \
        k_totals<real><<<TOTALS_BLOCKS, TOTALS_THREADS, 0, s>>>(f, partial, g, t);                           \
        k_totals_final<<<1, TOTALS_THREADS, 0, s>>>(partial, out, g.ds * g.ds);                              \
        return cudaGetLastError();                                                                           \
    }

}  // namespace olb
