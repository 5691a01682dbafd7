// olb_kernels.cuh -- device code of one RK-3 stage, templated on the
// population precision (double, or float with Kahan-compensated moments).
//
// Per stage two kernels run:
//   k_moments  one thread per node: n, u, T, Delta p from the 25 populations
//              (Sec. 2.2, Eq. vdw); extra warps, one per (wall, row), form the
//              WENO flux of the 10 outgoing velocities at the wall face and
//              reduce it with warp shuffles into n_w (Eq. nw).
//   k_stage    one CTA per TX x TY tile, one thread per node: force from the
//              49-point stencils on a shared-memory tile of Delta p and n with a
//              3-node halo (Eqs. F_def, stencil_grad, stencil_glap), the local
//              part of L (momentum derivative Eq. derf, BGK with Eq. feq),
//              then for each velocity the WENO-5 face fluxes of a shared-memory
//              population tile (Eqs. weno5_*), each face computed once, and
//              the RK-3 combination of Eq. rk3.
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
// v0..v4 = f_{i-2} .. f_{i+2} in the upwind orientation; returns the WENO-5
// interface value sum_q wbar_q Fhat^q (without p/m).
//
// Weights: wbar_q is proportional to delta_q / sigma_q^2.  Multiplying every
// term by sigma_1^2 sigma_2^2 sigma_3^2 gives weights proportional to
// A_q = delta_q prod_{r != q} sigma_r^2, which needs one division, equals the
// table row for a single vanishing indicator, and is 0/0 only when two or
// three vanish; those cases take Table tab:weno (the ideal weights of the
// vanishing set).  If the products underflow without an exact zero the
// min-scaled form delta_q (s/sigma_q)^2 is used instead.
__device__ __forceinline__ double weno5(double v0, double v1, double v2, double v3, double v4)
{
    const double a1 = v0 - 2.0 * v1 + v2, b1 = v0 - 4.0 * v1 + 3.0 * v2;
    const double a2 = v1 - 2.0 * v2 + v3, b2 = v1 - v3;
    const double a3 = v2 - 2.0 * v3 + v4, b3 = 3.0 * v2 - 4.0 * v3 + v4;
    const double s1 = (13.0 / 12.0) * a1 * a1 + 0.25 * b1 * b1;
    const double s2 = (13.0 / 12.0) * a2 * a2 + 0.25 * b2 * b2;
    const double s3 = (13.0 / 12.0) * a3 * a3 + 0.25 * b3 * b3;
    const double F1 = (1.0 / 3.0) * v0 - (7.0 / 6.0) * v1 + (11.0 / 6.0) * v2;
    const double F2 = (-1.0 / 6.0) * v1 + (5.0 / 6.0) * v2 + (1.0 / 3.0) * v3;
    const double F3 = (1.0 / 3.0) * v2 + (5.0 / 6.0) * v3 - (1.0 / 6.0) * v4;
    const double q1 = s1 * s1, q2 = s2 * s2, q3 = s3 * s3;
    const double A1 = 0.1 * (q2 * q3), A2 = 0.6 * (q1 * q3), A3 = 0.3 * (q1 * q2);
    const double den = A1 + A2 + A3;
    if (den > 0.0) return (A1 * F1 + A2 * F2 + A3 * F3) / den;
    double w1, w2, w3;
    if (s1 == 0.0 || s2 == 0.0 || s3 == 0.0) {
        w1 = (s1 == 0.0) ? 0.1 : 0.0;
        w2 = (s2 == 0.0) ? 0.6 : 0.0;
        w3 = (s3 == 0.0) ? 0.3 : 0.0;
    } else {
        const double s = fmin(s1, fmin(s2, s3));
        const double r1 = s / s1, r2 = s / s2, r3 = s / s3;
        w1 = 0.1 * r1 * r1;
        w2 = 0.6 * r2 * r2;
        w3 = 0.3 * r3 * r3;
    }
    return (w1 * F1 + w2 * F2 + w3 * F3) / (w1 + w2 + w3);
}

// FP32 form: the products of four squared indicators underflow in single
// precision, so the weights are always the min-scaled delta_q (s/sigma_q)^2
// (same normalised weights), with Table tab:weno when an indicator vanishes.
__device__ __forceinline__ float weno5(float v0, float v1, float v2, float v3, float v4)
{
    const float a1 = v0 - 2.0f * v1 + v2, b1 = v0 - 4.0f * v1 + 3.0f * v2;
    const float a2 = v1 - 2.0f * v2 + v3, b2 = v1 - v3;
    const float a3 = v2 - 2.0f * v3 + v4, b3 = 3.0f * v2 - 4.0f * v3 + v4;
    const float s1 = (13.0f / 12.0f) * a1 * a1 + 0.25f * b1 * b1;
    const float s2 = (13.0f / 12.0f) * a2 * a2 + 0.25f * b2 * b2;
    const float s3 = (13.0f / 12.0f) * a3 * a3 + 0.25f * b3 * b3;
    const float F1 = (1.0f / 3.0f) * v0 - (7.0f / 6.0f) * v1 + (11.0f / 6.0f) * v2;
    const float F2 = (-1.0f / 6.0f) * v1 + (5.0f / 6.0f) * v2 + (1.0f / 3.0f) * v3;
    const float F3 = (1.0f / 3.0f) * v2 + (5.0f / 6.0f) * v3 - (1.0f / 6.0f) * v4;
    float w1, w2, w3;
    const float s = fminf(s1, fminf(s2, s3));
    if (s > 0.0f) {
        const float r1 = __fdividef(s, s1), r2 = __fdividef(s, s2), r3 = __fdividef(s, s3);
        w1 = 0.1f * r1 * r1;
        w2 = 0.6f * r2 * r2;
        w3 = 0.3f * r3 * r3;
    } else {
        w1 = (s1 == 0.0f) ? 0.1f : 0.0f;
        w2 = (s2 == 0.0f) ? 0.6f : 0.0f;
        w3 = (s3 == 0.0f) ? 0.3f : 0.0f;
    }
    return __fdividef(w1 * F1 + w2 * F2 + w3 * F3, w1 + w2 + w3);
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
    const real c3 = u * (u2 * real(1.0 / 6.0) + real(0.5) * th);
    const real c4 = u2 * u2 * real(1.0 / 24.0) + real(0.25) * th * u2 + real(0.125) * th * th;
#pragma unroll
    for (int k = 0; k < NQ; ++k)
        g[k] = t.wHe[k][0] + t.wHe[k][1] * c1 + t.wHe[k][2] * c2 + t.wHe[k][3] * c3 + t.wHe[k][4] * c4;
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
        jx += t.R[k] * sx[k];
        jy += t.R[k] * sy[k];
        e += t.R2[k] * (sx[k] + sy[k]);
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

// ---------------------------------------------------------------- K1
constexpr int MOM_THREADS = 256;

template <typename real>
__global__ void __launch_bounds__(MOM_THREADS)
k_moments(const real *__restrict__ f, real *__restrict__ fld, real *__restrict__ nw,
          int *__restrict__ status, Geo g, Tab<real> t, int node_blocks)
{
    if ((int)blockIdx.x < node_blocks) {
        const long long idx = (long long)blockIdx.x * MOM_THREADS + threadIdx.x;
        if (idx >= (long long)g.nx * g.ny) return;
        const int j = (int)(idx / g.nx), i = (int)(idx - (long long)j * g.nx);
        const long long o = (long long)j * g.pitch + i;
        double n, jx, jy, e;
        node_sums<real>(f, g.plane, o, t, n, jx, jy, e);
        const double ux = jx / n, uy = jy / n;
        const double T = 0.5 * (e / n - ux * ux - uy * uy);
        // Delta p = n T - p^w, p^w = n T / (1 - b n) - a n^2 (Eq. vdw)
        const double dp = n * T - (n * T / (1.0 - g.b * n) - g.a * n * n);
        fld[0 * g.plane + o] = (real)n;
        fld[1 * g.plane + o] = (real)ux;
        fld[2 * g.plane + o] = (real)uy;
        fld[3 * g.plane + o] = (real)T;
        fld[4 * g.plane + o] = (real)dp;
        const bool ok = (n > 0.0) && (T > 0.0) && (g.b * n < 1.0) && isfinite(n) && isfinite(T) &&
                        isfinite(ux) && isfinite(uy);
        if (!ok) atomicOr(status, 1);
        return;
    }
    // Wall densities: one warp per (wall, row); lanes 0..9 take the outgoing
    // velocities (p_x < 0 at the left wall, p_x > 0 at the right wall).
    const int warp = ((int)blockIdx.x - node_blocks) * (MOM_THREADS / 32) + (int)(threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= 2 * g.ny) return;
    const int side = warp / g.ny, j = warp - side * g.ny;
    real flux = real(0);
    if (lane < 10) {
        const int k1 = side ? 3 + lane / 5 : lane / 5;
        const int k2 = lane % 5;
        const real *fp = f + (NQ * k1 + k2) * g.plane + (long long)j * g.pitch;
        // nearest three fluid nodes, nearest first
        const real a0 = side ? fp[g.nx - 1] : fp[0];
        const real a1 = side ? fp[g.nx - 2] : fp[1];
        const real a2 = side ? fp[g.nx - 3] : fp[2];
        // quadratic extrapolation into the first two ghost layers (Sec. 3.4.2)
        const real g0 = real(3) * a0 - real(3) * a1 + a2;
        const real g1 = real(6) * a0 - real(8) * a1 + real(3) * a2;
        // upwind-ordered stencil of the wall face, mirrored for the left wall
        flux = t.R[k1] * weno5(a2, a1, a0, g0, g1);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) flux += __shfl_xor_sync(0xffffffffu, flux, off);
    if (lane == 0) nw[side * g.ny + j] = -flux * t.inv_den[side];
}

// ---------------------------------------------------------------- K2
template <typename real, int TX, int TY>
struct StageSmem {
    static constexpr int NT = TX * TY, HX = TX + 6, HY = TY + 6;
    real dp[HY][HX];
    real n[HY][HX];
    real f[HY][HX];
    real fx[TY][TX + 1];
    real fy[TY + 1][TX];
    real part[NK][NT];
};

template <typename real, int TX, int TY>
__global__ void __launch_bounds__(TX *TY)
k_stage(const real *__restrict__ fs, const real *fn, real *out, const real *__restrict__ fld,
        const real *__restrict__ nw, Geo g, Tab<real> t, real ca, real cb, real cc)
{
    using S = StageSmem<real, TX, TY>;
    constexpr int NT = S::NT, HX = S::HX, HY = S::HY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S &sm = *reinterpret_cast<S *>(smem_raw);

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int i = x0 + tx, j = y0 + ty;
    const bool active = (i < g.nx) && (j < g.ny);
    const long long o = (long long)j * g.pitch + i;

    // ---- Delta p and n tile with a 3-node halo (field rule of Sec. 3.4.3)
    for (int e = tid; e < HX * HY; e += NT) {
        const int r = e / HX, c = e - r * HX;
        const int gx = g.walls ? reflect(x0 - 3 + c, g.nx) : wrap(x0 - 3 + c, g.nx);
        const int gy = wrap(y0 - 3 + r, g.ny);
        const long long go = (long long)gy * g.pitch + gx;
        sm.n[r][c] = __ldg(fld + 0 * g.plane + go);
        sm.dp[r][c] = __ldg(fld + 4 * g.plane + go);
    }
    __syncthreads();

    // ---- local part of L and the non-advective part of the RK combination
    if (active) {
        real ddx = 0, ddy = 0, ldx = 0, ldy = 0;
#pragma unroll
        for (int l = 1; l <= 3; ++l)
#pragma unroll
            for (int m = -3; m <= 3; ++m) {
                const int am = m < 0 ? -m : m;
                constexpr int cy = 3, cx = 3;
                if (grad_w(l, am) != 0.0) {
                    const real w = real(l * grad_w(l, am));
                    ddx += w * (sm.dp[ty + cy + m][tx + cx + l] - sm.dp[ty + cy + m][tx + cx - l]);
                    ddy += w * (sm.dp[ty + cy + l][tx + cx + m] - sm.dp[ty + cy - l][tx + cx + m]);
                }
                if (glap_c(am, l) != 0.0) {
                    const real w = real(glap_c(am, l));
                    ldx += w * (sm.n[ty + cy + m][tx + cx + l] - sm.n[ty + cy + m][tx + cx - l]);
                    ldy += w * (sm.n[ty + cy + l][tx + cx + m] - sm.n[ty + cy - l][tx + cx + m]);
                }
            }
        const real nn = sm.n[ty + 3][tx + 3];
        const real ux = __ldg(fld + 1 * g.plane + o);
        const real uy = __ldg(fld + 2 * g.plane + o);
        const real T = __ldg(fld + 3 * g.plane + o);
        // force (Eq. F_def): F = grad(Delta p)/n + sigma grad(Laplacian n)
        const real Fx = ddx * real(g.inv_ds) / nn + real(g.sigma) * ldx * real(g.inv_ds3);
        const real Fy = ddy * real(g.inv_ds) / nn + real(g.sigma) * ldy * real(g.inv_ds3);
        real gx[NQ], gy[NQ];
        eq_factors<real>(t, ux, T, gx);
        eq_factors<real>(t, uy, T, gy);
        real fv[NK];
#pragma unroll
        for (int k = 0; k < NK; ++k) fv[k] = __ldg(fs + k * g.plane + o);
        const real itau = real(g.inv_tau);
#pragma unroll
        for (int k1 = 0; k1 < NQ; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < NQ; ++k2) {
                real dx = 0, dy = 0;
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    dx += t.D[k1][q] * fv[NQ * q + k2];
                    dy += t.D[k2][q] * fv[NQ * k1 + q];
                }
                const int k = NQ * k1 + k2;
                const real feq = nn * gx[k1] * gy[k2];
                const real Lloc = -(Fx * dx + Fy * dy) - (fv[k] - feq) * itau;
                real p = cb * fv[k] + cc * Lloc;
                if (ca != real(0)) p += ca * fn[k * g.plane + o];
                sm.part[k][tid] = p;
            }
    }

    // ---- advection, one velocity at a time
    const int nfx = (TX + 1) * TY, nfy = TX * (TY + 1);
    for (int k = 0; k < NK; ++k) {
        const int k1 = k / NQ, k2 = k - NQ * (k / NQ);
        const real px = t.R[k1], py = t.R[k2];
        const real *fk = fs + k * g.plane;
        __syncthreads();  // previous velocity's faces are consumed
        // population tile: rows of the tile with the x halo, columns of the
        // tile with the y halo (corners are never read)
        for (int e = tid; e < TY * HX + 6 * TX; e += NT) {
            int r, c;
            if (e < TY * HX) {
                r = 3 + e / HX;
                c = e - (r - 3) * HX;
            } else {
                const int e2 = e - TY * HX;
                const int rr = e2 / TX;
                r = rr < 3 ? rr : TY + rr;
                c = 3 + (e2 - rr * TX);
            }
            const int gy = wrap(y0 - 3 + r, g.ny);
            int gx = x0 - 3 + c;
            real v;
            if (gx >= 0 && gx < g.nx) {
                v = __ldg(fk + (long long)gy * g.pitch + gx);
            } else if (!g.walls) {
                v = __ldg(fk + (long long)gy * g.pitch + wrap(gx, g.nx));
            } else {
                // diffuse-wall ghosts (Sec. 3.4.2)
                const bool right = gx >= g.nx;
                const int m = right ? gx - g.nx : -1 - gx;
                const bool out_going = right ? (k1 > 2) : (k1 < 2);
                const bool in_coming = right ? (k1 < 2) : (k1 > 2);
                v = real(0);
                if (m <= 1 && out_going) {
                    const real *row = fk + (long long)gy * g.pitch;
                    const real a0 = right ? __ldg(row + g.nx - 1) : __ldg(row + 0);
                    const real a1 = right ? __ldg(row + g.nx - 2) : __ldg(row + 1);
                    const real a2 = right ? __ldg(row + g.nx - 3) : __ldg(row + 2);
                    v = m == 0 ? real(3) * a0 - real(3) * a1 + a2 : real(6) * a0 - real(8) * a1 + real(3) * a2;
                } else if (m <= 2 && in_coming) {
                    v = __ldg(nw + (right ? g.ny : 0) + gy) * t.geqw[right ? 1 : 0][k];
                }
            }
            sm.f[r][c] = v;
        }
        __syncthreads();
        // faces: x faces of the tile rows, then y faces of the tile columns
        const int nx_faces = (k1 == 2) ? 0 : nfx;
        const int ny_faces = (k2 == 2) ? 0 : nfy;
        for (int e = tid; e < nx_faces + ny_faces; e += NT) {
            if (e < nx_faces) {
                const int r = e / (TX + 1), c = e - r * (TX + 1);
                if (y0 + r < g.ny && x0 + c <= g.nx) {
                    const real *row = &sm.f[3 + r][0];
                    sm.fx[r][c] = (k1 > 2) ? weno5(row[c], row[c + 1], row[c + 2], row[c + 3], row[c + 4])
                                           : weno5(row[c + 5], row[c + 4], row[c + 3], row[c + 2], row[c + 1]);
                }
            } else {
                const int e2 = e - nx_faces;
                const int r = e2 / TX, c = e2 - r * TX;
                if (x0 + c < g.nx && y0 + r <= g.ny) {
                    const int cc3 = 3 + c;
                    sm.fy[r][c] = (k2 > 2) ? weno5(sm.f[r][cc3], sm.f[r + 1][cc3], sm.f[r + 2][cc3],
                                                   sm.f[r + 3][cc3], sm.f[r + 4][cc3])
                                           : weno5(sm.f[r + 5][cc3], sm.f[r + 4][cc3], sm.f[r + 3][cc3],
                                                   sm.f[r + 2][cc3], sm.f[r + 1][cc3]);
                }
            }
        }
        __syncthreads();
        if (active) {
            real adv = 0;
            if (k1 != 2) adv += px * (sm.fx[ty][tx + 1] - sm.fx[ty][tx]);
            if (k2 != 2) adv += py * (sm.fy[ty + 1][tx] - sm.fy[ty][tx]);
            out[k * g.plane + o] = sm.part[k][tid] - cc * (adv * real(g.inv_ds));
        }
    }
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
    if (oT) oT[idx] = 0.5 * (e / n - ux * ux - uy * uy);
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
// Instantiated once per precision by olb_fp64.cu / olb_fp32.cu with the
// stage tile TX x TY chosen there.
#define OLB_DEFINE_LAUNCHERS(real, TX, TY)                                                                   \
    cudaError_t prepare(real *)                                                                              \
    {                                                                                                        \
        return cudaFuncSetAttribute(k_stage<real, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                    (int)sizeof(StageSmem<real, TX, TY>));                                   \
    }                                                                                                        \
    cudaError_t launch_moments(const real *f, real *fld, real *nw, int *status, const Geo &g,                \
                               const Tab<real> &t, cudaStream_t s)                                           \
    {                                                                                                        \
        const long long N = (long long)g.nx * g.ny;                                                          \
        const int node_blocks = (int)((N + MOM_THREADS - 1) / MOM_THREADS);                                  \
        const int wall_blocks = g.walls ? (2 * g.ny + MOM_THREADS / 32 - 1) / (MOM_THREADS / 32) : 0;        \
        k_moments<real><<<node_blocks + wall_blocks, MOM_THREADS, 0, s>>>(f, fld, nw, status, g, t,          \
                                                                          node_blocks);                      \
        return cudaGetLastError();                                                                           \
    }                                                                                                        \
    cudaError_t launch_stage(const real *fs, const real *fn, real *out, const real *fld, const real *nw,     \
                             const Geo &g, const Tab<real> &t, StageCoef c, cudaStream_t s)                  \
    {                                                                                                        \
        dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY);                                               \
        k_stage<real, TX, TY><<<grid, TX * TY, sizeof(StageSmem<real, TX, TY>), s>>>(                        \
            fs, fn, out, fld, nw, g, t, (real)c.ca, (real)c.cb, (real)c.cc);                                 \
        return cudaGetLastError();                                                                           \
    }                                                                                                        \
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
