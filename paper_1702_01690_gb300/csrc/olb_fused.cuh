// olb_fused.cuh -- one RK-3 stage of the off-lattice Boltzmann model in a
// single kernel per stage (templated on precision and tile shape).
//
// One CTA owns a TX x TY tile of nodes and stages the populations of the
// tile plus a 3-node halo on every side in shared memory:
//   1. load f_s for the (TX+8) x (TY+6) region (x offset -4 keeps the rows
//      of the region 16-byte aligned; y and periodic x wrap);
//   2. moments n, u, T, Delta p at every fluid node of the region (Sec. 2.2,
//      Eq. vdw), with the even reflection of Delta p and n at walls
//      (Sec. 3.4.3);
//   3. walls (Sec. 3.4.2): extrapolated ghosts for the outgoing velocities,
//      the WENO flux of those velocities at the wall face, summed per tile
//      row into n_w (Eq. nw) by a warp-shuffle reduction over the half-warp
//      that computes the row's ten fluxes, and f^eq_w ghosts for the
//      incoming velocities;
//   4. force F = grad(Delta p)/n + sigma grad(Laplacian n) at the tile nodes
//      from the 49-point stencils (Eqs. F_def, stencil_grad, stencil_glap);
//   5. for KP velocities at a time (one lane of TX*TY threads, rounded up to
//      whole warps, each): every x
//      and y face of the tile once (WENO-5, Eqs. weno5_*), then per node the
//      flux differences, the momentum derivative (Eq. derf), BGK with f^eq
//      (Eqs. feq, g_alpha) and the RK-3 combination of Eq. rk3, written to
//      the output buffer.  KP > 1 gives small tiles enough warps.
//
// FP32 (real = float) keeps every population as a pair hi + lo of floats
// (compensated storage, olb_kernels.cuh): the staged region holds both parts,
// moments are summed in double-float arithmetic, a face stores only its WENO
// correction (the face value minus its upwind node, a function of first
// differences of pairs) so that flux differences are first differences too,
// the collision uses the equilibrium split into its exactly symmetric and
// antisymmetric parts in p (no FP32 rounding of f^eq or of f/tau changes the
// momentum), and the RK-3 combination is done in double-float arithmetic.
#pragma once

#include "olb_mlp.cuh"

namespace olb {

// n and Delta p of the region, kept for the 49-point stencils.  The stencils
// cancel to O(ds^k) of their terms on fine grids, so the FP32 kernel keeps
// each value as an unevaluated sum hi + lo of two floats (hi = the value
// rounded to FP32, lo = the FP64 remainder rounded to FP32): differences of
// neighbouring values then keep ~FP64 accuracy at FP32 cost.
template <typename real>
struct FieldT {
    using type = double;
};
template <>
struct FieldT<float> {
    using type = float2;
};

__device__ __forceinline__ double make_field(double v, double) { return v; }
__device__ __forceinline__ float2 make_field(double v, float)
{
    const float hi = __double2float_rn(v);
    return make_float2(hi, __double2float_rn(v - (double)hi));
}
__device__ __forceinline__ double field_diff(double a, double b) { return a - b; }
__device__ __forceinline__ float field_diff(float2 a, float2 b) { return (a.x - b.x) + (a.y - b.y); }
__device__ __forceinline__ double field_val(double a) { return a; }
__device__ __forceinline__ float field_val(float2 a) { return a.x + a.y; }

// lo parts of the staged populations (FP32 only; FP64 has none)
template <typename real, int HY, int HX>
struct PopLo {
    real lo[NK][HY][HX];
};
template <int HY, int HX>
struct PopLo<double, HY, HX> {
};

template <typename real, int TX, int TY, int KP>
struct FusedSmem {
    // LS: threads per velocity lane, the tile's nodes rounded up to whole
    // warps (so that every lane starts on a warp); NT threads in all
    static constexpr int HX = TX + 8, HY = TY + 6, NN = TX * TY, LS = (NN + 31) / 32 * 32, NT = LS * KP;
    using fld = typename FieldT<real>::type;
    real pop[NK][HY][HX];
    PopLo<real, HY, HX> pl;
    fld n[HY][HX];
    fld dp[HY][HX];
    real ux[TY][TX];
    real uy[TY][TX];
    fld T[TY][TX];  // FP32: hi + lo pair
    // FP32: e = sum |p|^2 f at the tile nodes as a double-float pair (the
    // target energy of the equilibrium's correction); unused in FP64
    fld eng[sizeof(real) == 4 ? TY : 1][sizeof(real) == 4 ? TX : 1];
    // per tile node, shared by the KP velocity lanes (with one lane they stay
    // in registers): the stencil sums of grad(Delta p) and grad(Laplacian n),
    // inv_ds / n, E_q = (c/tau) n g_q(u_x, T) and g_q(u_y, T) (FP32: the
    // even and odd parts n ge_q(u_x, T), n go_q(u_x, T), ge_q(u_y, T),
    // go_q(u_y, T) instead), and, on tiles that keep every face, G_x = c F_x
    // and G_y in L_G, L_G + 1
    static constexpr int NEQ = sizeof(real) == 8 ? 2 : 4;  // equilibrium factor sets
    static constexpr int L_DDX = 0, L_DDY = 1, L_LDX = 2, L_LDY = 3, L_DN = 4, L_E = 5, L_GY = 5 + NQ,
                         L_OX = 5 + 2 * NQ, L_OY = 5 + 3 * NQ, L_G = 5 + NEQ * NQ,
                         L_CA = 7 + NEQ * NQ, L_CB = 8 + NEQ * NQ, L_CC = 9 + NEQ * NQ;  // FP32: the correction
    real loc[KP > 1 ? 7 + NEQ * NQ + (sizeof(real) == 4 ? 3 : 0) : 1][KP > 1 ? NN : 1];
    // WENO-5 face values.  Small tiles (at most 64 nodes) hold the faces of
    // all 25 velocities, so one pass computes them all and the node updates
    // follow without further barriers; larger tiles hold KP velocities'.
    static constexpr bool ALL_FACES = TX * TY <= 64;
    static constexpr int KF = ALL_FACES ? NK : KP;
    union {
        real fx[KF][TY][TX + 1];
        // wall density n_w of each tile row at the left and right diffuse wall
        // (Eq. nw): written and read between the moments and the force,
        // before any face value is stored
        real wnw[2][TY];
    };
    real fy[KF][TY + 1][TX];
    unsigned long long mbar;  // completion barrier of the TMA copy of phase 1
};

template <typename real>
__device__ __forceinline__ real sel5(const real v[NQ], int k)
{
    real r = v[0];
    r = (k == 1) ? v[1] : r;
    r = (k == 2) ? v[2] : r;
    r = (k == 3) ? v[3] : r;
    r = (k == 4) ? v[4] : r;
    return r;
}

// Face value of one upwind-ordered stencil: Jiang-Shu weights, or the
// learned network's (parameters in shared memory) when LEARNED.
template <typename real, bool LEARNED>
__device__ __forceinline__ real face_value(const float *mlp, real v0, real v1, real v2, real v3, real v4)
{
    if constexpr (LEARNED)
        return weno5_learned<real>(mlp, v0, v1, v2, v3, v4);
    else
        return weno5(v0, v1, v2, v3, v4);
}

// FP32 pairs: the correction c (face value minus the upwind node v2) of the
// stencil with first differences d01 .. d34.
template <bool LEARNED>
__device__ __forceinline__ float face_corr(const float *mlp, float d01, float d12, float d23, float d34)
{
    if constexpr (LEARNED)
        return weno5_learned_corr(mlp, d01, d12, d23, d34);
    else
        return weno5_corr(d01, d12, d23, d34);
}

// ---------------------------------------------------------------- moments of a node
// n, u, T and Delta p of one node from its 25 populations (Sec. 2.2; T from
// the trace of Eq. sigmaq_def; Delta p = n T - p^w, Eq. vdw), and whether they
// are admissible (finite, n > 0, T > 0, b n < 1).  get(k) returns population
// k: the value (FP64) or the pair hi + lo (FP32).
template <typename real>
struct NodeMoments;
template <>
struct NodeMoments<double> {
    double n, dp, ux, uy, T;
    bool ok;
};
template <>
struct NodeMoments<float> {
    float2 n, dp, T, E;  // hi + lo pairs (E = sum |p|^2 f)
    float ux, uy;
    bool ok;
};

template <typename real, typename Get>
__device__ __forceinline__ NodeMoments<real> node_moments(Get get, const Geo &g, const Tab<real> &t)
{
    NodeMoments<real> m;
    if constexpr (sizeof(real) == 8) {
        // row and column sums of the 5 x 5 populations; the middle root is 0
        // (R[2] = R2[2] = 0), so its sums drop out of j and e
        double sx[NQ], sy[NQ];
#pragma unroll
        for (int k1 = 0; k1 < NQ; ++k1) {
            double s = get(NQ * k1);
            if (k1 == 0) sy[0] = s;
            else sy[0] += s;
#pragma unroll
            for (int k2 = 1; k2 < NQ; ++k2) {
                const double v = get(NQ * k1 + k2);
                s += v;
                if (k1 == 0) sy[k2] = v;
                else sy[k2] += v;
            }
            sx[k1] = s;
        }
        double n = sx[0];
        double jx = t.R[0] * sx[0];
        double jy = t.R[0] * sy[0];
        double en = t.R2[0] * (sx[0] + sy[0]);
#pragma unroll
        for (int k = 1; k < NQ; ++k) {
            n += sx[k];
            if (k == 2) continue;
            jx = fma(t.R[k], sx[k], jx);
            jy = fma(t.R[k], sy[k], jy);
            en = fma(t.R2[k], sx[k] + sy[k], en);
        }
        const double inv_n = recip_nr(n);
        const double ux = jx * inv_n, uy = jy * inv_n;
        const double T = 0.5 * fma(en, inv_n, -fma(ux, ux, uy * uy));
        // Delta p = n T - p^w, p^w = n T / (1 - b n) - a n^2 (Eq. vdw)
        const double nT = n * T;
        m.n = n;
        m.dp = nT - fma(nT, recip_nr(1.0 - g.b * n), -g.a * n * n);
        m.ux = ux;
        m.uy = uy;
        m.T = T;
        m.ok = (n > 0.0) && (T > 0.0) && (g.b * n < 1.0) && isfinite(n) && isfinite(T) && isfinite(ux) && isfinite(uy);
    } else {
        // FP32, compensated storage: row and column sums of the 5 x 5 pairs
        // as double-float values; n and e = sum |p|^2 f from them in
        // double-float arithmetic.  j needs FP32 accuracy of j itself:
        // R_4 (sx_4 - sx_0) + R_3 (sx_3 - sx_1) with the differences of the
        // double-float sums (R_0 = -R_4, R_1 = -R_3, R_2 = 0).
        f2 sx[NQ], sy[NQ];
        {
            float h[NQ], l[NQ];
#pragma unroll
            for (int k1 = 0; k1 < NQ; ++k1) {
#pragma unroll
                for (int k2 = 0; k2 < NQ; ++k2) {
                    const float2 v = get(NQ * k1 + k2);
                    h[k2] = v.x;
                    l[k2] = v.y;
                }
                sx[k1] = pair_sum5(h, l);
            }
#pragma unroll
            for (int k2 = 0; k2 < NQ; ++k2) {
#pragma unroll
                for (int k1 = 0; k1 < NQ; ++k1) {
                    const float2 v = get(NQ * k1 + k2);
                    h[k1] = v.x;
                    l[k1] = v.y;
                }
                sy[k2] = pair_sum5(h, l);
            }
        }
        const f2 one{1.0f, 0.0f};
        const f2 vdw_a = f2_of(g.a), vdw_b = f2_of(g.b);
        const f2 N = f2_add(f2_add(f2_add(sx[0], sx[4]), f2_add(sx[1], sx[3])), sx[2]);
        const float jx = fmaf(t.R[4], pdiff(sx[4].hi, sx[4].lo, sx[0].hi, sx[0].lo),
                              t.R[3] * pdiff(sx[3].hi, sx[3].lo, sx[1].hi, sx[1].lo));
        const float jy = fmaf(t.R[4], pdiff(sy[4].hi, sy[4].lo, sy[0].hi, sy[0].lo),
                              t.R[3] * pdiff(sy[3].hi, sy[3].lo, sy[1].hi, sy[1].lo));
        const f2 S4 = f2_add(f2_add(sx[0], sx[4]), f2_add(sy[0], sy[4]));
        const f2 S3 = f2_add(f2_add(sx[1], sx[3]), f2_add(sy[1], sy[3]));
        const f2 R24{t.R2[4], t.R2lo[4]}, R23{t.R2[3], t.R2lo[3]};
        const f2 Ea = f2_cmul(R24, S4.hi, S4.lo), Eb = f2_cmul(R23, S3.hi, S3.lo);
        const f2 E = f2_add(fast_two_sum(Ea.hi, Ea.lo), fast_two_sum(Eb.hi, Eb.lo));
        // u, T and Delta p = n T - p^w = n^2 (a - b T / (1 - b n)) (Eq. vdw):
        // T and Delta p in double-float arithmetic, so that the stencils of n
        // and Delta p see ~44-bit values without the FP64 pipe
        const f2 IN = f2_div(one, N);
        const float UX = jx * IN.hi, UY = jy * IN.hi;
        const f2 T = f2_scale(f2_add_f(f2_mul(E, IN), -fmaf(UX, UX, UY * UY)), 0.5f);
        const f2 BN = f2_mul(vdw_b, N);
        const f2 Q = f2_div(f2_mul(vdw_b, T), f2_add(one, f2_neg(BN)));
        const f2 DP = f2_mul(f2_mul(N, N), f2_add(vdw_a, f2_neg(Q)));
        m.n = make_float2(N.hi, N.lo);
        m.dp = make_float2(DP.hi, DP.lo);
        m.T = make_float2(T.hi, T.lo);
        m.E = make_float2(E.hi, E.lo);
        m.ux = UX;
        m.uy = UY;
        m.ok = (N.hi > 0.0f) && (T.hi > 0.0f) && (BN.hi < 1.0f) && isfinite(N.hi) && isfinite(T.hi) && isfinite(UX) &&
               isfinite(UY);
    }
    return m;
}

// Fields of the per-node pre-pass (k_fields), [ny][pitch] each: n and
// Delta p (FP32: hi + lo pairs), u_x, u_y, T (FP32: T a pair, and e = sum
// |p|^2 f as a pair for the equilibrium's correction).
template <typename real>
struct StageFields {
    using fld = typename FieldT<real>::type;
    fld *n, *dp, *T, *E;
    real *ux, *uy;
};

// Pointers of the fields in a buffer of 5 planes of pitch * ny 8-byte
// elements (fields_bytes): FP64 n, Delta p, T, u_x, u_y; FP32 n, Delta p,
// T, e (float2 each), then u_x and u_y (float) sharing the last plane.
template <typename real>
__host__ __device__ inline StageFields<real> fields_of(void *base, const Geo &g)
{
    StageFields<real> f{};
    char *b = static_cast<char *>(base);
    const size_t plane = (size_t)g.plane * 8;
    f.n = reinterpret_cast<typename FieldT<real>::type *>(b);
    f.dp = reinterpret_cast<typename FieldT<real>::type *>(b + plane);
    f.T = reinterpret_cast<typename FieldT<real>::type *>(b + 2 * plane);
    if constexpr (sizeof(real) == 8) {
        f.E = nullptr;
        f.ux = reinterpret_cast<real *>(b + 3 * plane);
        f.uy = reinterpret_cast<real *>(b + 4 * plane);
    } else {
        f.E = reinterpret_cast<typename FieldT<real>::type *>(b + 3 * plane);
        f.ux = reinterpret_cast<real *>(b + 4 * plane);
        f.uy = reinterpret_cast<real *>(b + 4 * plane + plane / 2);
    }
    return f;
}

// One thread per node: the moments of f_s, stored for the stage kernel,
// which then reads them on its tile and halo instead of recomputing them
// at every halo position; inadmissible moments set bit 0 of the status.
template <typename real>
__global__ void __launch_bounds__(256) k_fields(const real *__restrict__ fs, StageFields<real> out, int *status,
                                                const __grid_constant__ Geo g, const __grid_constant__ Tab<real> t)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)g.nx * g.ny) return;
    const int j = (int)(idx / g.nx), i = (int)(idx - (long long)j * g.nx);
    const long long o = (long long)j * g.pitch + i;
    NodeMoments<real> m;
    if constexpr (sizeof(real) == 8)
        m = node_moments<real>([&](int k) { return __ldg(fs + k * g.plane + o); }, g, t);
    else
        m = node_moments<real>(
            [&](int k) { return make_float2(__ldg(fs + k * g.plane + o), __ldg(fs + (NK + k) * g.plane + o)); }, g, t);
    out.n[o] = m.n;
    out.dp[o] = m.dp;
    out.ux[o] = m.ux;
    out.uy[o] = m.uy;
    out.T[o] = m.T;
    if constexpr (sizeof(real) == 4) out.E[o] = m.E;
    if (!m.ok) atomicOr(status, 1);
}

// ---------------------------------------------------------------- TMA staging
// Iterations of the bounded wait for the copy (each try_wait suspends for at
// most a short, hardware-defined time): far above the microseconds a copy of
// a tile's region takes, far below a hang.
constexpr int TMA_WAIT_LIMIT = 1 << 16;

__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity)
{
    for (int i = 0; i < TMA_WAIT_LIMIT; ++i) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Phase 1 for a tile whose staged region lies inside the grid: one TMA copy
// of the box (HX, HY, planes) at (gx0, gy0, 0) of the tensor map into the
// staging arrays (pop, then the lo planes in FP32, contiguous in FusedSmem in
// the box's order), completion tracked by an mbarrier.  tma_issue starts the
// copy (all threads call it; it synchronises); tma_finish waits for it with
// the bounded wait.  If the wait runs out, bit 1 of the status word is set,
// the copy is waited for once more (bounded) and false is returned: the
// caller leaves the tile untouched and the CTA stops.  After a completed copy
// the barrier is invalidated, so that a CTA that stages several tiles
// initialises it afresh for each.
template <typename real, int TX, int TY, int KP>
__device__ __forceinline__ void tma_issue(FusedSmem<real, TX, TY, KP> &sm, const TmaMap *tmap, int gx0, int gy0)
{
    constexpr unsigned bytes = sizeof(sm.pop) + (sizeof(real) == 4 ? sizeof(sm.pop) : 0);
    const unsigned mbar = (unsigned)__cvta_generic_to_shared(&sm.mbar);
    const unsigned dst = (unsigned)__cvta_generic_to_shared(&sm.pop[0][0][0]);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];" ::"r"(dst),
            "l"(reinterpret_cast<unsigned long long>(tmap)), "r"(gx0), "r"(gy0), "r"(0), "r"(mbar)
            : "memory");
    }
    __syncthreads();  // the barrier is initialised before anyone waits on it
}
template <typename real, int TX, int TY, int KP>
__device__ __forceinline__ bool tma_finish(FusedSmem<real, TX, TY, KP> &sm, int *status)
{
    const unsigned mbar = (unsigned)__cvta_generic_to_shared(&sm.mbar);
    const bool ok = mbar_wait(mbar, 0);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) atomicOr(status, 2);
        mbar_wait(mbar, 0);
        return false;
    }
    // every thread has passed its wait (the barrier above)
    if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(mbar) : "memory");
    return true;
}

// One stage for the tile whose lower-left node is (x0, y0); all threads of
// the CTA call it (it synchronises).  ca, cb, cc: the stage's coefficients of
// f^n, f_s and dt L (Eq. rk3), in the population precision; ca_lo, cb_lo:
// their remainders (FP32: 1/3 and 2/3 as double-float constants; 0 in FP64).
// g and t may live in parameter space (single grid) or shared memory
// (batch); tw: the table of the wall entries (geqw, inv_den), t itself for
// a single grid, the run's own in a batch, whose velocity tables t are common
// to all runs and passed as a kernel parameter; mlp: the learned network's
// parameters in shared memory (LEARNED
// only); tmap: TMA map of fs (of this run, in a batch) for this tile shape,
// or nullptr; fields: the moments of fs from k_fields, or nullptr to compute
// them here.  Returns false when the TMA copy timed out (the CTA must stop).
template <typename real, int TX, int TY, int KP, bool LEARNED = false>
__device__ __forceinline__ bool stage_tile(FusedSmem<real, TX, TY, KP> &sm, const real *__restrict__ fs,
                                           const real *fn, real *out, int *__restrict__ status, const Geo &g,
                                           const Tab<real> &t, const Tab<real> &tw, const int x0, const int y0,
                                           const real ca,
                                           const real cb, const real cc, const real ca_lo, const real cb_lo,
                                           const float *mlp = nullptr, const TmaMap *tmap = nullptr,
                                           const StageFields<real> *fields = nullptr)
{
    using S = FusedSmem<real, TX, TY, KP>;
    constexpr int NT = S::NT, NN = S::NN, HX = S::HX, HY = S::HY;

    // thread = (tile node, velocity lane): KP velocities are advanced at once
    const int tid = threadIdx.x;
    const int node = tid % S::LS, lane_k = tid / S::LS;
    const int tx = node % TX, ty = node / TX;
    const int i = x0 + tx, j = y0 + ty;
    const bool active = (node < NN) && (i < g.nx) && (j < g.ny);

    // ---- 1. populations of the region (c <-> x = x0 - 4 + c, r <-> y = y0 - 3 + r)
    //    A region inside the grid comes in one TMA copy.  Otherwise:
    //    periodic sides wrap.  Ghost layers 0..2 of a specular side hold the
    //    populations of the first three nodes inside with the normal
    //    velocity component reversed (Sec. 3.4.1); diffuse-wall ghosts are
    //    set in phase 3; anything further out is never read and holds 0.
    const bool inside = tmap != nullptr && x0 >= 4 && x0 + TX + 4 <= g.nx && y0 >= 3 && y0 + TY + 3 <= g.ny;
    // the pre-pass fields of this thread's first moment position (phase 2's
    // item e = tid) are fetched into registers now, so that their latency
    // overlaps the staging of the populations
    using fld = typename S::fld;
    fld pf_n{}, pf_dp{}, pf_T{}, pf_E{};
    real pf_ux = 0, pf_uy = 0;
    bool pf_ok = false, pf_node = false;
    int pf_r = 0, pf_c = 0;
    if (fields != nullptr && tid < HY * (HX - 2)) {
        pf_r = tid / (HX - 2);
        pf_c = tid - pf_r * (HX - 2) + 1;
        const int gx = x0 - 4 + pf_c, gyr = y0 - 3 + pf_r;
        pf_ok = !(g.walls && (gx < 0 || gx >= g.nx)) && !(g.spec_y && (gyr < 0 || gyr >= g.ny));
        if (pf_ok) {
            const long long o = (long long)wrap(gyr, g.ny) * g.pitch + wrap(gx, g.nx);
            pf_n = fields->n[o];
            pf_dp = fields->dp[o];
            const int tr = pf_r - 3, tc = pf_c - 4;
            pf_node = tr >= 0 && tr < TY && tc >= 0 && tc < TX;
            if (pf_node) {
                pf_ux = fields->ux[o];
                pf_uy = fields->uy[o];
                pf_T = fields->T[o];
                if constexpr (sizeof(real) == 4) pf_E = fields->E[o];
            }
        }
    }
    // With the moments from the pre-pass, a tile inside the grid touches its
    // staged populations first in the face pass (no walls, no sides, no
    // moments to compute), so phases 2-4 run while the copy is in flight
    const bool defer = inside && fields != nullptr;
    if (inside) {
        tma_issue(sm, tmap, x0 - 4, y0 - 3);
        if (!defer && !tma_finish(sm, status)) return false;
    } else {
        for (int e = tid; e < HY * HX; e += NT) {
            const int r = e / HX, c = e - r * HX;
            int gy = y0 - 3 + r, gx = x0 - 4 + c;
            bool flip_x = false, flip_y = false, zero = false;
            if (gy < 0 || gy >= g.ny) {
                if (!g.spec_y) {
                    gy = wrap(gy, g.ny);
                } else if ((gy < 0 ? -1 - gy : gy - g.ny) <= 2) {
                    gy = gy < 0 ? -1 - gy : 2 * g.ny - 1 - gy;
                    flip_y = true;
                } else {
                    zero = true;
                }
            }
            if (gx < 0 || gx >= g.nx) {
                const bool lo = gx < 0;
                if (!g.walls) {
                    gx = wrap(gx, g.nx);
                } else if ((lo ? g.spec_lo : g.spec_hi) && (lo ? -1 - gx : gx - g.nx) <= 2) {
                    gx = lo ? -1 - gx : 2 * g.nx - 1 - gx;
                    flip_x = true;
                } else {
                    zero = true;
                }
            }
            if (zero) {
#pragma unroll 5
                for (int k = 0; k < NK; ++k) {
                    sm.pop[k][r][c] = real(0);
                    if constexpr (sizeof(real) == 4) sm.pl.lo[k][r][c] = 0.0f;
                }
                continue;
            }
            const real *src = fs + (long long)gy * g.pitch + gx;
            if (!flip_x && !flip_y) {
#pragma unroll 5
                for (int k = 0; k < NK; ++k) {
                    sm.pop[k][r][c] = __ldg(src + k * g.plane);
                    if constexpr (sizeof(real) == 4) sm.pl.lo[k][r][c] = __ldg(src + (NK + k) * g.plane);
                }
            } else {
#pragma unroll
                for (int k1 = 0; k1 < NQ; ++k1)
#pragma unroll
                    for (int k2 = 0; k2 < NQ; ++k2) {
                        const int kk = NQ * (flip_x ? NQ - 1 - k1 : k1) + (flip_y ? NQ - 1 - k2 : k2);
                        sm.pop[NQ * k1 + k2][r][c] = __ldg(src + kk * g.plane);
                        if constexpr (sizeof(real) == 4) sm.pl.lo[NQ * k1 + k2][r][c] = __ldg(src + (NK + kk) * g.plane);
                    }
            }
        }
    }
    __syncthreads();

    // ---- 2. moments at every fluid position of the region that the 7 x 7
    // force stencils reach (columns 1 .. HX-2; ghost positions of walls and
    // specular sides take the reflected fields in phase 3).  A tile at a
    // diffuse wall also computes here, on warps of their own, the wall-face
    // flux of every outgoing velocity in every tile row (Sec. 3.4.2: the
    // WENO-5 face value at the wall from the three nearest fluid nodes and the
    // two ghosts extrapolated from them) and stores those two ghosts; both
    // need the phase-1 populations only, and the FP64 units of the
    // sub-partitions with fewer moment warps have room.
    const bool x_lo = g.walls && x0 == 0;                // ghost columns at x = 0
    const bool x_hi = g.walls && (x0 + TX + 3 >= g.nx);  // ghost columns at x = nx ds
    const bool left_wall = x_lo && g.wall_lo;
    const bool right_wall = x_hi && g.wall_hi;
    // wall-flux items start on the first warp after the moment positions
    constexpr int e_flux = (HY * (HX - 2) + 31) / 32 * 32;
    const int nflux = ((int)left_wall + (int)right_wall) * TY * 16;
    if (fields != nullptr) {
        // moments from the per-node pre-pass (k_fields): n and Delta p on the
        // region, u, T (FP32: and e) at the tile nodes; item tid was fetched
        // before phase 1
        if (pf_ok) {
            sm.n[pf_r][pf_c] = pf_n;
            sm.dp[pf_r][pf_c] = pf_dp;
            if (pf_node) {
                sm.ux[pf_r - 3][pf_c - 4] = pf_ux;
                sm.uy[pf_r - 3][pf_c - 4] = pf_uy;
                sm.T[pf_r - 3][pf_c - 4] = pf_T;
                if constexpr (sizeof(real) == 4) sm.eng[pf_r - 3][pf_c - 4] = pf_E;
            }
        }
        for (int e = tid + NT; e < HY * (HX - 2); e += NT) {
            const int r = e / (HX - 2), c = e - r * (HX - 2) + 1;
            const int gx = x0 - 4 + c, gyr = y0 - 3 + r;
            if (g.walls && (gx < 0 || gx >= g.nx)) continue;
            if (g.spec_y && (gyr < 0 || gyr >= g.ny)) continue;
            const long long o = (long long)wrap(gyr, g.ny) * g.pitch + wrap(gx, g.nx);
            sm.n[r][c] = fields->n[o];
            sm.dp[r][c] = fields->dp[o];
            const int tr = r - 3, tc = c - 4;
            if (tr >= 0 && tr < TY && tc >= 0 && tc < TX) {
                sm.ux[tr][tc] = fields->ux[o];
                sm.uy[tr][tc] = fields->uy[o];
                sm.T[tr][tc] = fields->T[o];
                if constexpr (sizeof(real) == 4) sm.eng[tr][tc] = fields->E[o];
            }
        }
    } else {
        for (int e = tid; e < HY * (HX - 2); e += NT) {
            const int r = e / (HX - 2), c = e - r * (HX - 2) + 1;
            const int gx = x0 - 4 + c, gyr = y0 - 3 + r;
            if (g.walls && (gx < 0 || gx >= g.nx)) continue;
            if (g.spec_y && (gyr < 0 || gyr >= g.ny)) continue;
            const int tr = r - 3, tc = c - 4;
            const bool tile_node = tr >= 0 && tr < TY && tc >= 0 && tc < TX;
            const bool own = tile_node && x0 + tc < g.nx && y0 + tr < g.ny;
            NodeMoments<real> m;
            if constexpr (sizeof(real) == 8)
                m = node_moments<real>([&](int k) { return sm.pop[k][r][c]; }, g, t);
            else
                m = node_moments<real>([&](int k) { return make_float2(sm.pop[k][r][c], sm.pl.lo[k][r][c]); }, g,
                                       t);
            sm.n[r][c] = m.n;
            sm.dp[r][c] = m.dp;
            if (tile_node) {
                sm.ux[tr][tc] = m.ux;
                sm.uy[tr][tc] = m.uy;
                sm.T[tr][tc] = m.T;
                if constexpr (sizeof(real) == 4) sm.eng[tr][tc] = m.E;
                if (own && !m.ok) atomicOr(status, 1);
            }
        }
    }
    // wall flux item f runs on thread (e_flux + f) mod NT: on the warps after
    // those with moment positions.  Each tile row of a wall takes a
    // half-warp: lanes v = 0..9 compute the flux of outgoing velocity v (the
    // half-range p_x < 0 at x = 0, p_x > 0 at x = nx ds), lanes 10..15 add 0,
    // and a shuffle reduction over the half-warp gives the row's sum.  (e_flux
    // and NT are multiples of 32, so f runs over whole half-warps.)
    for (int f = (tid - e_flux % NT + NT) % NT; f < nflux; f += NT) {
        // (wall, tile row tr, outgoing velocity v); the left wall's items first
        const int side = (f >= TY * 16 || !left_wall) ? 1 : 0;
        const int fr = f >= TY * 16 ? f - TY * 16 : f;
        const int tr = fr >> 4, v = fr & 15;
        const int k1 = side ? 3 + v / 5 : v / 5;
        const int k = NQ * k1 + v % 5;
        // nearest three fluid nodes, nearest first; ghost layers 0 and 1
        // are the next two columns outwards
        const int c0 = side ? g.nx - 1 - (x0 - 4) : 0 - (x0 - 4);
        const int dc = side ? -1 : 1;
        real wf = 0;
        if (v >= 10) {
            // idle lane of the row's half-warp
        } else if constexpr (sizeof(real) == 8) {
            const real a0 = sm.pop[k][tr + 3][c0], a1 = sm.pop[k][tr + 3][c0 + dc];
            const real a2 = sm.pop[k][tr + 3][c0 + 2 * dc];
            const real g0 = fma(real(3), a0 - a1, a2);
            const real g1 = fma(real(6), a0, fma(real(-8), a1, real(3) * a2));
            if (c0 - dc >= 0 && c0 - dc < HX) sm.pop[k][tr + 3][c0 - dc] = g0;
            if (c0 - 2 * dc >= 0 && c0 - 2 * dc < HX) sm.pop[k][tr + 3][c0 - 2 * dc] = g1;
            wf = t.R[k1] * face_value<real, LEARNED>(mlp, a2, a1, a0, g0, g1);
        } else {
            // pairs: the ghosts 3a0 - 3a1 + a2 and 6a0 - 8a1 + 3a2 as a0 plus
            // combinations of the differences D1 = a0 - a1, D2 = a1 - a2, and
            // the stencil (a2, a1, a0, g0, g1) by its first differences
            // (D2, D1, 2 D1 - D2, 3 D1 - 2 D2)
            const int row = tr + 3;
            const float h0 = sm.pop[k][row][c0], l0 = sm.pl.lo[k][row][c0];
            const float h1 = sm.pop[k][row][c0 + dc], l1 = sm.pl.lo[k][row][c0 + dc];
            const float h2 = sm.pop[k][row][c0 + 2 * dc], l2 = sm.pl.lo[k][row][c0 + 2 * dc];
            const float D1 = pdiff(h0, l0, h1, l1), D2 = pdiff(h1, l1, h2, l2);
            const float e0 = fmaf(2.0f, D1, -D2), e1 = fmaf(5.0f, D1, -3.0f * D2);
            const f2 G0 = f2_add_f(f2{h0, l0}, e0), G1 = f2_add_f(f2{h0, l0}, e1);
            if (c0 - dc >= 0 && c0 - dc < HX) {
                sm.pop[k][row][c0 - dc] = G0.hi;
                sm.pl.lo[k][row][c0 - dc] = G0.lo;
            }
            if (c0 - 2 * dc >= 0 && c0 - 2 * dc < HX) {
                sm.pop[k][row][c0 - 2 * dc] = G1.hi;
                sm.pl.lo[k][row][c0 - 2 * dc] = G1.lo;
            }
            const float corr = face_corr<LEARNED>(mlp, D2, D1, e0, fmaf(3.0f, D1, -2.0f * D2));
            wf = t.R[k1] * (h0 + (l0 + corr));
        }
        const unsigned half = (tid & 16) ? 0xffff0000u : 0x0000ffffu;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) wf += __shfl_xor_sync(half, wf, o);
        if (v == 0) sm.wnw[side][tr] = -wf * tw.inv_den[side];
    }

    // ---- 3. sides: n and Delta p reflected evenly into the ghost layers of
    // walls and specular planes (Sec. 3.4.3; y first, then x over every row,
    // which makes the corners a double reflection); at diffuse walls the
    // incoming ghosts of the tile rows, f^eq_w = n_w g g (Sec. 3.4.2, Eq.
    // diffuse_flux), with the wall density n_w of Eq. nw from the sum of the
    // row's outgoing fluxes
    if (g.spec_y && (y0 == 0 || y0 + TY + 2 >= g.ny)) {
        __syncthreads();
        for (int e = tid; e < HY * HX; e += NT) {
            const int r = e / HX, c = e - r * HX;
            const int gyr = y0 - 3 + r;
            if (gyr >= 0 && gyr < g.ny) continue;
            if ((gyr < 0 ? -1 - gyr : gyr - g.ny) > 2) continue;
            const int rm = (gyr < 0 ? -1 - gyr : 2 * g.ny - 1 - gyr) - (y0 - 3);
            sm.n[r][c] = sm.n[rm][c];
            sm.dp[r][c] = sm.dp[rm][c];
        }
    }
    if (x_lo || x_hi) {
        __syncthreads();
        constexpr int e_in = (HY * HX + 31) / 32 * 32;  // first incoming-ghost item, on a warp boundary
        const int nin = ((int)left_wall + (int)right_wall) * TY * 30;
        for (int e = tid; e < e_in + nin; e += NT) {
            if (e < HY * HX) {
                const int r = e / HX, c = e - r * HX;
                const int gx = x0 - 4 + c;
                if (gx >= 0 && gx < g.nx) continue;
                const bool right = gx >= g.nx;
                if ((right ? gx - g.nx : -1 - gx) > 2) continue;  // beyond ghost layer 2
                const int cm = (right ? 2 * g.nx - 1 - gx : -1 - gx) - (x0 - 4);
                sm.n[r][c] = sm.n[r][cm];
                sm.dp[r][c] = sm.dp[r][cm];
            } else if (e >= e_in) {
                // (wall, tile row tr, ghost layer m, incoming velocity v)
                const int f = e - e_in;
                const int side = (f >= TY * 30 || !left_wall) ? 1 : 0;
                const int fr = f >= TY * 30 ? f - TY * 30 : f;
                const int tr = fr / 30, m = (fr - 30 * tr) / 10, v = fr - 30 * tr - 10 * m;
                const int c = side ? g.nx + m - (x0 - 4) : -1 - m - (x0 - 4);
                if (c < 0 || c >= HX) continue;
                const int k = NQ * (side ? v / 5 : 3 + v / 5) + v % 5;
                sm.pop[k][tr + 3][c] = sm.wnw[side][tr] * tw.geqw[side][k];
                if constexpr (sizeof(real) == 4) sm.pl.lo[k][tr + 3][c] = 0.0f;
            }
        }
    }
    __syncthreads();

    // ---- 4. force and equilibrium factors at the tile nodes.  The four
    // stencil sums and the two factor sets are split over the velocity lanes
    // (KP = 4: ddx | ddy | ldx, g(u_x) | ldy, g(u_y); KP = 2: x | y parts).
    constexpr int cy = 3, cx = 4;
    auto grad_sum = [&](bool along_x) {
        real acc = 0;
#pragma unroll
        for (int l = 1; l <= 3; ++l)
#pragma unroll
            for (int m = -3; m <= 3; ++m) {
                const int am = m < 0 ? -m : m;
                if (grad_w(l, am) != 0.0) {
                    const real w = real(l * grad_w(l, am));
                    acc = along_x ? fma(w, field_diff(sm.dp[ty + cy + m][tx + cx + l], sm.dp[ty + cy + m][tx + cx - l]), acc)
                                  : fma(w, field_diff(sm.dp[ty + cy + l][tx + cx + m], sm.dp[ty + cy - l][tx + cx + m]), acc);
                }
            }
        return acc;
    };
    auto glap_sum = [&](bool along_x) {
        real acc = 0;
        if constexpr (sizeof(real) == 4) {
            // FP32: the stencil cancels its O(ds) terms down to O(ds^3) (a
            // factor ~1/(ds k)^2 on fine grids), so the weighted differences
            // are summed in double-float arithmetic with double-float weights
            // (exact products of the hi parts, TwoSum accumulation): the sum
            // keeps FP32 accuracy of itself, not of its terms
            f2 sum{0.0f, 0.0f};
#pragma unroll
            for (int l = 1; l <= 3; ++l)
#pragma unroll
                for (int m = -3; m <= 3; ++m) {
                    const int am = m < 0 ? -m : m;
                    if (glap_c(am, l) != 0.0) {
                        const float wh = (float)glap_c(am, l);
                        const float wl = (float)(glap_c(am, l) - (double)(float)glap_c(am, l));
                        const float2 a = along_x ? sm.n[ty + cy + m][tx + cx + l] : sm.n[ty + cy + l][tx + cx + m];
                        const float2 b = along_x ? sm.n[ty + cy + m][tx + cx - l] : sm.n[ty + cy - l][tx + cx + m];
                        const f2 dh = two_sum(a.x, -b.x);
                        const float dl = dh.lo + (a.y - b.y);
                        const float p = wh * dh.hi;
                        const float e = fmaf(wh, dh.hi, -p);
                        const float tl = fmaf(wh, dl, fmaf(wl, dh.hi, e));
                        const f2 t2 = two_sum(sum.hi, p);
                        sum = f2{t2.hi, t2.lo + (sum.lo + tl)};
                    }
                }
            acc = sum.hi + sum.lo;
        } else {
#pragma unroll
            for (int l = 1; l <= 3; ++l)
#pragma unroll
                for (int m = -3; m <= 3; ++m) {
                    const int am = m < 0 ? -m : m;
                    if (glap_c(am, l) != 0.0) {
                        const real w = real(glap_c(am, l));
                        acc = along_x ? fma(w, field_diff(sm.n[ty + cy + m][tx + cx + l], sm.n[ty + cy + m][tx + cx - l]), acc)
                                      : fma(w, field_diff(sm.n[ty + cy + l][tx + cx + m], sm.n[ty + cy - l][tx + cx + m]), acc);
                    }
                }
        }
        return acc;
    };
    // With c the stage's coefficient of dt L (Eq. rk3), the node update below
    // needs per node G = c F, E_q = (c/tau) n g_q(u_x, T) and g_q(u_y, T)
    // (FP32: n ge_q(u_x, T), n go_q(u_x, T), ge_q(u_y, T), go_q(u_y, T), the
    // even and odd parts of the factors, in E, Ox, gy, Oy).
    const real sg3 = real(g.sigma) * real(g.inv_ds3);
    const real cit = cc * real(g.inv_tau);
    constexpr bool F32 = sizeof(real) == 4;
    real Gx = 0, Gy = 0, E[NQ], gy[NQ], Ox[NQ], Oy[NQ];
    real qa = 0, qb = 0, qc = 0;  // FP32: alpha, beta, gamma of the equilibrium's correction (eq_correction)
    // equilibrium factor sets of the node at (tx_, ty_): x (scaled by n, and
    // for FP64 by c/tau) into ex, ox and y into ey, oy
    auto eq_sets = [&](bool x_set, real *a, real *b) {
        if constexpr (F32) {
            if (x_set) {
                eq_factors_split(t, sm.ux[ty][tx], sm.T[ty][tx], a, b);
                const real nn = sm.n[ty + 3][tx + 4].x;
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    a[q] = nn * a[q];
                    b[q] = nn * b[q];
                }
            } else {
                eq_factors_split(t, sm.uy[ty][tx], sm.T[ty][tx], a, b);
            }
        } else {
            if (x_set) {
                eq_factors<real>(t, sm.ux[ty][tx], sm.T[ty][tx], a);
                const real cn = cit * field_val(sm.n[ty + 3][tx + 4]);
#pragma unroll
                for (int q = 0; q < NQ; ++q) a[q] = cn * a[q];
            } else {
                eq_factors<real>(t, sm.uy[ty][tx], sm.T[ty][tx], a);
            }
        }
    };
    if constexpr (KP == 1) {
        if (active) {
            const real ddx = grad_sum(true), ddy = grad_sum(false);
            const real ldx = glap_sum(true), ldy = glap_sum(false);
            const real nn = field_val(sm.n[ty + cy][tx + cx]);
            const real dn = real(g.inv_ds) / nn;
            Gx = cc * fma(ddx, dn, sg3 * ldx);
            Gy = cc * fma(ddy, dn, sg3 * ldy);
            eq_sets(true, E, Ox);
            eq_sets(false, gy, Oy);
            if constexpr (F32)
                eq_correction(t, E, gy, sm.n[ty + 3][tx + 4], sm.eng[ty][tx], sm.ux[ty][tx], sm.uy[ty][tx], qa, qb, qc);
        }
    } else {
        static_assert(KP == 2 || KP == 4 || KP == 5 || KP == 8, "velocity lanes: 1, 2, 4, 5 or 8");
        using Sm = FusedSmem<real, TX, TY, KP>;
        if (active) {
            // KP = 8: lanes 0..5 take ddx, ddy, ldx, ldy, E, g(u_y);
            // KP = 5: lanes 0..3 ddx, ddy, ldx, ldy, lane 4 E and g(u_y);
            // KP = 4: lane 0 ddx, lane 1 ddy, lane 2 ldx + E, lane 3 ldy + g(u_y);
            // KP = 2: lane 0 the x parts, lane 1 the y parts
            const bool lane_ldx = KP == 2 ? lane_k == 0 : lane_k == 2;
            const bool lane_ldy = KP == 2 ? lane_k == 1 : lane_k == 3;
            const bool lane_gx = KP == 2 ? lane_k == 0 : (KP == 4 ? lane_k == 2 : lane_k == 4);
            const bool lane_gy = KP == 2 ? lane_k == 1 : (KP == 4 ? lane_k == 3 : (KP == 5 ? lane_k == 4 : lane_k == 5));
            if (lane_k == 0) {
                sm.loc[Sm::L_DDX][node] = grad_sum(true);
                sm.loc[Sm::L_DN][node] = real(g.inv_ds) / field_val(sm.n[ty + cy][tx + cx]);
            }
            if (lane_k == 1) sm.loc[Sm::L_DDY][node] = grad_sum(false);
            if (lane_ldx) sm.loc[Sm::L_LDX][node] = glap_sum(true);
            if (lane_ldy) sm.loc[Sm::L_LDY][node] = glap_sum(false);
            if (lane_gx) {
                eq_sets(true, E, Ox);
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    sm.loc[Sm::L_E + q][node] = E[q];
                    if constexpr (F32) sm.loc[Sm::L_OX + q][node] = Ox[q];
                }
            }
            if (lane_gy) {
                eq_sets(false, gy, Oy);
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    sm.loc[Sm::L_GY + q][node] = gy[q];
                    if constexpr (F32) sm.loc[Sm::L_OY + q][node] = Oy[q];
                }
            }
            if constexpr (F32) {
                // the equilibrium's mass and energy correction, on a lane with
                // little else to do (KP = 8: lane 6; KP = 5, 4, 2: lane 1), from
                // the same factors the other lanes store (same operations)
                if (lane_k == (KP == 8 ? 6 : 1)) {
                    real ex[NQ], ox[NQ], ey[NQ], oy[NQ];
                    eq_sets(true, ex, ox);
                    eq_sets(false, ey, oy);
                    eq_correction(t, ex, ey, sm.n[ty + 3][tx + 4], sm.eng[ty][tx], sm.ux[ty][tx], sm.uy[ty][tx], qa,
                                  qb, qc);
                    sm.loc[Sm::L_CA][node] = qa;
                    sm.loc[Sm::L_CB][node] = qb;
                    sm.loc[Sm::L_CC][node] = qc;
                }
            }
        }
        __syncthreads();
        // G = c F at the node: in registers of each lane, or, on tiles that
        // keep every face, once per node in shared memory (read after the
        // barrier that ends the face pass)
        if (active && (!Sm::ALL_FACES || lane_k == 0)) {
            const real dn = sm.loc[Sm::L_DN][node];
            Gx = cc * fma(sm.loc[Sm::L_DDX][node], dn, sg3 * sm.loc[Sm::L_LDX][node]);
            Gy = cc * fma(sm.loc[Sm::L_DDY][node], dn, sg3 * sm.loc[Sm::L_LDY][node]);
            if constexpr (Sm::ALL_FACES) {
                sm.loc[Sm::L_G][node] = Gx;
                sm.loc[Sm::L_G + 1][node] = Gy;
            }
        }
    }

    // ---- 5. advection, collision and RK combination, KP velocities at a time
    const int nfx = (TX + 1) * TY, nfy = TX * (TY + 1);
    const real cf = cb - cit;
    const real cadv = cc * real(g.inv_ds);
    using Sf = FusedSmem<real, TX, TY, KP>;
    constexpr int KF = Sf::KF;
    // one face value: x face (r, c) or y face (r, c) of velocity k, stored in
    // slot (FP32: its WENO correction, from first differences of the pairs)
    auto face = [&](int k, int slot, bool along_x, int r, int c) {
        const int k1 = k / NQ, k2 = k - NQ * (k / NQ);
        if (along_x) {
            if (y0 + r < g.ny && x0 + c <= g.nx) {
                // face at x = x0 + c: nodes x0+c-3 .. x0+c+2 are columns c+1 .. c+6
                const real *row = &sm.pop[k][3 + r][0];
                if constexpr (F32) {
                    const float *lo = &sm.pl.lo[k][3 + r][0];
                    auto pd = [&](int a_, int b_) { return pdiff(row[a_], lo[a_], row[b_], lo[b_]); };
                    sm.fx[slot][r][c] =
                        (k1 > 2) ? face_corr<LEARNED>(mlp, pd(c + 2, c + 1), pd(c + 3, c + 2), pd(c + 4, c + 3), pd(c + 5, c + 4))
                                 : face_corr<LEARNED>(mlp, pd(c + 5, c + 6), pd(c + 4, c + 5), pd(c + 3, c + 4), pd(c + 2, c + 3));
                } else {
                    sm.fx[slot][r][c] =
                        (k1 > 2) ? face_value<real, LEARNED>(mlp, row[c + 1], row[c + 2], row[c + 3], row[c + 4], row[c + 5])
                                 : face_value<real, LEARNED>(mlp, row[c + 6], row[c + 5], row[c + 4], row[c + 3], row[c + 2]);
                }
            }
        } else if (x0 + c < g.nx && y0 + r <= g.ny) {
            // face at y = y0 + r: rows y0+r-3 .. y0+r+2 are rows r .. r+5
            const int cc4 = 4 + c;
            const real(*P)[HX] = sm.pop[k];
            if constexpr (F32) {
                const float(*Lo)[HX] = sm.pl.lo[k];
                auto pd = [&](int a_, int b_) { return pdiff(P[a_][cc4], Lo[a_][cc4], P[b_][cc4], Lo[b_][cc4]); };
                sm.fy[slot][r][c] = (k2 > 2) ? face_corr<LEARNED>(mlp, pd(r + 1, r), pd(r + 2, r + 1), pd(r + 3, r + 2), pd(r + 4, r + 3))
                                             : face_corr<LEARNED>(mlp, pd(r + 4, r + 5), pd(r + 3, r + 4), pd(r + 2, r + 3), pd(r + 1, r + 2));
            } else {
                sm.fy[slot][r][c] = (k2 > 2) ? face_value<real, LEARNED>(mlp, P[r][cc4], P[r + 1][cc4], P[r + 2][cc4],
                                                                        P[r + 3][cc4], P[r + 4][cc4])
                                            : face_value<real, LEARNED>(mlp, P[r + 5][cc4], P[r + 4][cc4], P[r + 3][cc4],
                                                                        P[r + 2][cc4], P[r + 1][cc4]);
            }
        }
    };
    // learned weights (FP32 instances): the face of item (k, slot, along_x,
    // r, c), or none (valid false); every lane of the warp calls it together,
    // from a single call site, since the warp evaluates the network of its 32
    // stencils on the tensor pipe
    float *const mlp_sc = (LEARNED && F32) ? const_cast<float *>(mlp) + MLP_SCRATCH_OFF + (tid >> 5) * MLP_WARP_SCRATCH : nullptr;
    auto learned_face = [&](int k, int slot, bool along_x, int r, int c, bool valid) {
        const int k1 = k / NQ, k2 = k - NQ * (k / NQ);
        valid = valid && (along_x ? (y0 + r < g.ny && x0 + c <= g.nx) : (x0 + c < g.nx && y0 + r <= g.ny));
        // the stencil v0 .. v4 in the upwind orientation, as positions of the
        // staged region: x faces along row 3 + r, y faces along column 4 + c
        int p0 = 0, step = 1;
        if (along_x) {
            p0 = (k1 > 2) ? c + 1 : c + 6;
            step = (k1 > 2) ? 1 : -1;
        } else {
            p0 = (k2 > 2) ? r : r + 5;
            step = (k2 > 2) ? 1 : -1;
        }
        real d[4] = {0, 0, 0, 0}, v2 = 0;
        if (valid) {
            const real *P = &sm.pop[k][0][0];
            auto at = [&](int m) { return along_x ? (3 + r) * HX + p0 + m * step : (p0 + m * step) * HX + 4 + c; };
            if constexpr (F32) {
                const float *Lo = &sm.pl.lo[k][0][0];
#pragma unroll
                for (int m = 0; m < 4; ++m) d[m] = pdiff(P[at(m + 1)], Lo[at(m + 1)], P[at(m)], Lo[at(m)]);
            } else {
#pragma unroll
                for (int m = 0; m < 4; ++m) d[m] = P[at(m + 1)] - P[at(m)];
                v2 = P[at(2)];
            }
        }
        // the guard in the population precision, the network's input and
        // correction in FP32 from the rounded differences
        const bool acts = learned_guard<real>(d[0], d[1], d[2], d[3]);
        const float e[4] = {(float)d[0], (float)d[1], (float)d[2], (float)d[3]};
        float x[MLP_IN], w[MLP_OUT] = {0.0f, 0.0f, 0.0f};
        learned_input_x(e, acts, x);
        // the whole warp skips the network when none of its stencils needs it
        if (__any_sync(0xffffffffu, acts)) mlp_weights_warp(mlp, x, w, mlp_sc);
        if (valid) {
            real res;
            if (acts) {
                res = v2 + (real)learned_corr_from(w, e);
            } else {
                const real q12 = d[1] * d[1], q23 = d[2] * d[2];
                res = weno5_core(d[0], d[1], d[2], d[3], q23, real(2.5) * q12, real(2.5) * q23, v2);
            }
            if (along_x) sm.fx[slot][r][c] = res;
            else sm.fy[slot][r][c] = res;
        }
    };
    // node update of velocity k (faces in slot) at tile node (tx_, ty_):
    // FP64 with Ek = E_q(k1), gyk = g_q(k2); FP32 with Ek = n ge(k1),
    // oxk = n go(k1), gyk = ge(k2), oyk = go(k2)
    auto update = [&](int k1, int k2, int slot, int tx_, int ty_, real Gx_, real Gy_, real Ek, real gyk, real oxk,
                      real oyk, real qa_, real qb_, real qc_) {
        const int k = NQ * k1 + k2;
        const int r = ty_ + 3, c = tx_ + 4;
        real dx = 0, dy = 0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            dx = fma(t.D[k1][q], sm.pop[NQ * q + k2][r][c], dx);
            dy = fma(t.D[k2][q], sm.pop[NQ * k1 + q][r][c], dy);
        }
        const real f = sm.pop[k][r][c];
        const long long o = (long long)(y0 + ty_) * g.pitch + (x0 + tx_);
        if constexpr (F32) {
            // flux difference = difference of the upwind nodes of the two
            // faces (a first difference of pairs) + difference of corrections
            const float(*P)[HX] = sm.pop[k];
            const float(*Lo)[HX] = sm.pl.lo[k];
            float adv = 0.0f;
            if (k1 != 2) {
                const int cu = k1 > 2 ? c : c + 1;
                adv = t.R[k1] * (pdiff(P[r][cu], Lo[r][cu], P[r][cu - 1], Lo[r][cu - 1]) +
                                 (sm.fx[slot][ty_][tx_ + 1] - sm.fx[slot][ty_][tx_]));
            }
            if (k2 != 2) {
                const int ru = k2 > 2 ? r : r + 1;
                adv = fmaf(t.R[k2], pdiff(P[ru][c], Lo[ru][c], P[ru - 1][c], Lo[ru - 1][c]) +
                                        (sm.fy[slot][ty_ + 1][tx_] - sm.fy[slot][ty_][tx_]), adv);
            }
            // f - f^eq with f^eq = n (ge ge + ge go + go (ge + go)) - c: the
            // exactly symmetric part first, then the parts odd in p_y and in
            // p_x (each exactly odd after rounding), so that FP32 rounding of
            // the equilibrium carries no momentum; c (eq_correction) restores
            // its mass and energy
            const float fl = Lo[r][c];
            const float corr =
                (t.wHe[k1][0] * t.wHe[k2][0]) * fmaf(qc_, t.R2[k1] - t.R2[k2], fmaf(qb_, t.R2[k1] + t.R2[k2], qa_));
            const float neq = ((((f - Ek * gyk) + fl) - Ek * oyk) - oxk * (gyk + oyk)) + corr;
            // c L = -c xi.grad f - c F.grad_p f - (c/tau)(f - f^eq), then
            // out = ca f_n + cb f_s + c L (Eq. rk3) in double-float arithmetic
            const float inc = -fmaf(cit, neq, fmaf(Gx_, dx, fmaf(Gy_, dy, cadv * adv)));
            f2 acc = f2_cmul(f2{cb, cb_lo}, f, fl);
            if (ca != 0.0f) {
                const f2 an = f2_cmul(f2{ca, ca_lo}, fn[k * g.plane + o], fn[(NK + k) * g.plane + o]);
                const f2 sh = two_sum(acc.hi, an.hi);
                acc = f2{sh.hi, sh.lo + (acc.lo + an.lo)};
            }
            const f2 si = two_sum(acc.hi, inc);
            const f2 v = fast_two_sum(si.hi, si.lo + acc.lo);
            out[k * g.plane + o] = v.hi;
            out[(NK + k) * g.plane + o] = v.lo;
        } else {
            real adv = 0;
            if (k1 != 2) adv = t.R[k1] * (sm.fx[slot][ty_][tx_ + 1] - sm.fx[slot][ty_][tx_]);
            if (k2 != 2) adv = fma(t.R[k2], sm.fy[slot][ty_ + 1][tx_] - sm.fy[slot][ty_][tx_], adv);
            // c L = -c xi.grad f - c F.grad_p f - (c/tau)(f - f^eq) with f^eq = n g g
            // (Eqs. feq, g_alpha), combined with b f (and a f_n) as in Eq. rk3
            real v = fma(cf, f, fma(Ek, gyk, -fma(Gx_, dx, fma(Gy_, dy, cadv * adv))));
            if (ca != real(0)) v = fma(ca, fn[k * g.plane + o], v);
            out[k * g.plane + o] = v;
        }
    };
    if (defer && !tma_finish(sm, status)) return false;  // the populations of phase 1
    for (int kb = 0; kb < NK; kb += KF) {
        __syncthreads();  // loc ready / the previous velocities' faces are consumed
        if constexpr (LEARNED && sizeof(real) == 4) {
            // FP32 with learned weights: the network on the tensor pipe, one
            // warp per 32 stencils (FP64 instances, bound by the FP64 pipe,
            // evaluate it per thread in the loop further down: the warp
            // network measured no faster there, and its scratch does not fit
            // the largest FP64 tile).  The faces of this pass (all 25 velocities' on small tiles, else
            // those of velocities kb .. kb+KP-1), enumerated as below, on
            // whole warps: items past the end take part in the network only.
            // Small tiles: the x faces of the 20 velocities with xi_x != 0,
            // then the y faces of the 20 with xi_y != 0, located by division
            // (as in the dense pass below); otherwise the KP velocities'
            // faces, located in their prefix table
            int end[KF], total = 0;
            if constexpr (Sf::ALL_FACES) {
                total = 20 * (nfx + nfy);
            } else {
#pragma unroll
                for (int sub = 0; sub < KF; ++sub) {
                    const int k = kb + sub;
                    if (k < NK) total += (k / NQ != 2 ? nfx : 0) + (k % NQ != 2 ? nfy : 0);
                    end[sub] = total;
                }
            }
            const int padded = (total + 31) & ~31;
            for (int e = tid; e < padded; e += NT) {
                int k, sub, f;
                bool valid = e < total;
                if constexpr (Sf::ALL_FACES) {
                    const int ee = valid ? e : 0;
                    if (ee < 20 * nfx) {
                        const int kx = ee / nfx;
                        k = kx < 2 * NQ ? kx : kx + NQ;
                        f = ee - kx * nfx;
                    } else {
                        const int e2 = ee - 20 * nfx, ky = e2 / nfy, q = ky & 3;
                        k = (ky >> 2) * NQ + (q < 2 ? q : q + 1);
                        f = nfx + e2 - ky * nfy;
                    }
                    sub = k;
                } else {
                    int start = 0;
                    sub = 0;
#pragma unroll
                    for (int q = 0; q + 1 < KF; ++q)
                        if (e >= end[q]) {
                            sub = q + 1;
                            start = end[q];
                        }
                    k = kb + sub;
                    f = e - start;
                    if (k / NQ == 2) f += nfx;
                    valid = valid && k < NK;
                }
                const bool along_x = f < nfx;
                const int r = along_x ? f / (TX + 1) : (f - nfx) / TX;
                const int c = along_x ? f - r * (TX + 1) : f - nfx - r * TX;
                // one call site: the warp's network must run as one instruction
                // stream (mma.sync needs every lane at the same instruction)
                learned_face(k, sub, along_x, valid ? r : 0, valid ? c : 0, valid);
            }
        } else if constexpr (Sf::ALL_FACES && sizeof(real) == 4) {
            // FP32 (issue-bound): every face of every velocity once, in strips
            // of SX (SY) consecutive faces along a tile row (column), each
            // strip in the upwind direction of its velocity: the x strips of
            // the 20 velocities with xi_x != 0 (k1 != 2), then the y strips of
            // the 20 with xi_y != 0 (k2 != 2).  (In FP64 the FP64 unit paces
            // each warp, and the fewer, longer strip items leave too few warps
            // per sub-partition at the end of the pass: single faces are faster.)
            constexpr int SX = (TX + 1) % 4 == 0 ? 4 : ((TX + 1) % 3 == 0 ? 3 : 1);
            constexpr int SY = (TY + 1) % 4 == 0 ? 4 : ((TY + 1) % 3 == 0 ? 3 : 1);
            constexpr int NSX = (TX + 1) / SX, NSY = (TY + 1) / SY;    // strips per row, per column
            constexpr int nsx = NSX * TY, nsy = NSY * TX;              // strips per velocity
            for (int e = tid; e < 20 * (nsx + nsy); e += NT) {
                if (e < 20 * nsx) {
                    const int kx = e / nsx, f = e - kx * nsx;
                    const int k = kx < 2 * NQ ? kx : kx + NQ;
                    const int r = f / NSX, cs = (f - r * NSX) * SX;
                    // face at x = x0 + c reads columns c+1 .. c+5 (xi_x > 0) or c+6 .. c+2
                    const real *row = &sm.pop[k][3 + r][0];
                    const real *rlo = &sm.pl.lo[k][3 + r][0];
                    if (k / NQ > 2) weno5_strip_c<SX>(row + cs + 1, rlo + cs + 1, 1, &sm.fx[k][r][cs], 1);
                    else weno5_strip_c<SX>(row + cs + SX + 5, rlo + cs + SX + 5, -1, &sm.fx[k][r][cs + SX - 1], -1);
                } else {
                    const int e2 = e - 20 * nsx, ky = e2 / nsy, f = e2 - ky * nsy, q = ky & 3;
                    const int k = (ky >> 2) * NQ + (q < 2 ? q : q + 1);
                    const int rs = (f / TX) * SY, c = f - (f / TX) * TX;
                    // face at y = y0 + r reads rows r .. r+4 (xi_y > 0) or r+5 .. r+1
                    if (k % NQ > 2)
                        weno5_strip_c<SY>(&sm.pop[k][rs][4 + c], &sm.pl.lo[k][rs][4 + c], HX, &sm.fy[k][rs][c], TX);
                    else
                        weno5_strip_c<SY>(&sm.pop[k][rs + SY + 4][4 + c], &sm.pl.lo[k][rs + SY + 4][4 + c], -HX,
                                          &sm.fy[k][rs + SY - 1][c], -TX);
                }
            }
            // (faces outside the grid are computed from staged values and never read)
        } else if constexpr (Sf::ALL_FACES) {
            // every face of every velocity once, enumerated densely: the x faces
            // of the 20 velocities with xi_x != 0 (k1 != 2), then the y faces of
            // the 20 with xi_y != 0 (k2 != 2)
            for (int e = tid; e < 20 * (nfx + nfy); e += NT) {
                if (e < 20 * nfx) {
                    const int kx = e / nfx, f = e - kx * nfx;
                    const int k = kx < 2 * NQ ? kx : kx + NQ;
                    const int r = f / (TX + 1);
                    face(k, k, true, r, f - r * (TX + 1));
                } else {
                    const int e2 = e - 20 * nfx, ky = e2 / nfy, f = e2 - ky * nfy, q = ky & 3;
                    const int k = (ky >> 2) * NQ + (q < 2 ? q : q + 1);
                    const int r = f / TX;
                    face(k, k, false, r, f - r * TX);
                }
            }
        } else {
            // faces of the KP velocities kb .. kb+KP-1, each computed once and
            // enumerated densely: x faces of the tile rows unless xi_x = 0
            // (k1 = 2), then y faces of the tile columns unless xi_y = 0 (k2 = 2)
            int end[KP], total = 0;
#pragma unroll
            for (int sub = 0; sub < KP; ++sub) {
                const int k = kb + sub;
                if (k < NK) total += (k / NQ != 2 ? nfx : 0) + (k % NQ != 2 ? nfy : 0);
                end[sub] = total;
            }
            for (int e = tid; e < total; e += NT) {
                int sub = 0, start = 0;
#pragma unroll
                for (int q = 0; q + 1 < KP; ++q)
                    if (e >= end[q]) {
                        sub = q + 1;
                        start = end[q];
                    }
                const int k = kb + sub;
                int f = e - start;
                if (k / NQ == 2) f += nfx;
                if (f < nfx) {
                    const int r = f / (TX + 1);
                    face(k, sub, true, r, f - r * (TX + 1));
                } else {
                    const int r = (f - nfx) / TX;
                    face(k, sub, false, r, f - nfx - r * TX);
                }
            }
        }
        __syncthreads();
        if constexpr (Sf::ALL_FACES && F32 && KP == NQ) {
            // FP32 (issue-bound) node updates with five lanes: thread (node,
            // lane k2) advances the five velocities 5 k1 + k2, k1 unrolled,
            // so that the k1 tables are immediate operands and the node's
            // factors are read once
            if (active) {
                const int k2 = lane_k;
                const real Gx_ = sm.loc[Sf::L_G][node], Gy_ = sm.loc[Sf::L_G + 1][node];
                const real qa_ = sm.loc[Sf::L_CA][node], qb_ = sm.loc[Sf::L_CB][node], qc_ = sm.loc[Sf::L_CC][node];
                const real gyk = sm.loc[Sf::L_GY + k2][node], oyk = sm.loc[Sf::L_OY + k2][node];
#pragma unroll
                for (int k1 = 0; k1 < NQ; ++k1)
                    update(k1, k2, NQ * k1 + k2, tx, ty, Gx_, Gy_, sm.loc[Sf::L_E + k1][node], gyk,
                           sm.loc[Sf::L_OX + k1][node], oyk, qa_, qb_, qc_);
            }
        } else if constexpr (Sf::ALL_FACES) {
            // node updates, enumerated densely over (velocity, tile node)
            for (int e = tid; e < NK * NN; e += NT) {
                const int k = e / NN, nd = e - k * NN;
                const int tx_ = nd % TX, ty_ = nd / TX;
                if (x0 + tx_ >= g.nx || y0 + ty_ >= g.ny) continue;
                const int k1 = k / NQ, k2 = k - NQ * (k / NQ);
                real oxk = 0, oyk = 0, qa_ = 0, qb_ = 0, qc_ = 0;
                if constexpr (F32) {
                    oxk = sm.loc[Sf::L_OX + k1][nd];
                    oyk = sm.loc[Sf::L_OY + k2][nd];
                    qa_ = sm.loc[Sf::L_CA][nd];
                    qb_ = sm.loc[Sf::L_CB][nd];
                    qc_ = sm.loc[Sf::L_CC][nd];
                }
                update(k1, k2, k, tx_, ty_, sm.loc[Sf::L_G][nd], sm.loc[Sf::L_G + 1][nd], sm.loc[Sf::L_E + k1][nd],
                       sm.loc[Sf::L_GY + k2][nd], oxk, oyk, qa_, qb_, qc_);
            }
        } else {
            const int k = kb + lane_k;
            if (active && k < NK) {
                const int k1 = k / NQ, k2 = k - NQ * (k / NQ);
                real Ek, gyk, oxk = 0, oyk = 0, qa_ = qa, qb_ = qb, qc_ = qc;
                if constexpr (KP > 1) {
                    Ek = sm.loc[Sf::L_E + k1][node];
                    gyk = sm.loc[Sf::L_GY + k2][node];
                    if constexpr (F32) {
                        oxk = sm.loc[Sf::L_OX + k1][node];
                        oyk = sm.loc[Sf::L_OY + k2][node];
                        qa_ = sm.loc[Sf::L_CA][node];
                        qb_ = sm.loc[Sf::L_CB][node];
                        qc_ = sm.loc[Sf::L_CC][node];
                    }
                } else {
                    Ek = sel5(E, k1);
                    gyk = sel5(gy, k2);
                    if constexpr (F32) {
                        oxk = sel5(Ox, k1);
                        oyk = sel5(Oy, k2);
                    }
                }
                update(k1, k2, lane_k, tx, ty, Gx, Gy, Ek, gyk, oxk, oyk, qa_, qb_, qc_);
            }
        }
    }
    return true;
}

// Shared memory of the single-grid kernel: the tile staging, then (learned
// weights only) the network's parameters at a 16-byte aligned offset and the
// warps' scratch for the network's tensor-pipe layer.
template <typename real, int TX, int TY, int KP>
constexpr size_t mlp_offset()
{
    return (sizeof(FusedSmem<real, TX, TY, KP>) + 15) / 16 * 16;
}
template <typename real, int TX, int TY, int KP, bool LEARNED>
constexpr size_t fused_smem_bytes()
{
    // learned: the parameters; FP32 also the split W2 and MLP_WARP_SCRATCH
    // floats per warp
    constexpr size_t mlp_floats = sizeof(real) == 4
                                      ? MLP_SCRATCH_OFF + FusedSmem<real, TX, TY, KP>::NT / 32 * MLP_WARP_SCRATCH
                                      : MLP_P + 1;
    return LEARNED ? mlp_offset<real, TX, TY, KP>() + mlp_floats * sizeof(float) : sizeof(FusedSmem<real, TX, TY, KP>);
}

// CTAs per SM that the register allocation must leave room for: as many as
// the shared memory (228 KB per SM, 1 KB of it reserved per CTA) and the
// 2048 threads of an SM allow.  Without this bound the compiler may take
// more registers than that occupancy leaves (e.g. 80 for a 512-thread CTA
// that could otherwise share its SM), capped at cap when cap > 0.
constexpr int fused_min_ctas(size_t smem_bytes, int threads, int cap = 0)
{
    const int by_smem = (int)((228 * 1024) / (smem_bytes + 1024)), by_threads = 2048 / threads;
    const int n = by_smem < by_threads ? by_smem : by_threads;
    return n < 1 ? 1 : (cap > 0 && n > cap ? cap : n);
}

// Single grid: one CTA per tile.  Learned-weight instances leave their
// network the registers it needs: FP32 (tensor-pipe network) at most two CTAs
// per SM, FP64 (per-thread network) one.
template <typename real, int TX, int TY, int KP, bool LEARNED>
__global__ void __launch_bounds__(FusedSmem<real, TX, TY, KP>::NT,
                                  fused_min_ctas(fused_smem_bytes<real, TX, TY, KP, LEARNED>(),
                                                 FusedSmem<real, TX, TY, KP>::NT,
                                                 LEARNED ? (sizeof(real) == 4 ? 2 : 1) : 0))
k_fused(const real *__restrict__ fs, const real *fn, real *out, int *__restrict__ status,
        const __grid_constant__ Geo g, const __grid_constant__ Tab<real> t, real ca, real cb, real cc, real ca_lo,
        real cb_lo, const float *__restrict__ mlp, const __grid_constant__ TmaArg tma,
        const __grid_constant__ StageFields<real> fields)
{
    // 128-byte aligned: the TMA copy of phase 1 lands at offset 0
    extern __shared__ __align__(128) unsigned char smem_raw[];
    auto &sm = *reinterpret_cast<FusedSmem<real, TX, TY, KP> *>(smem_raw);
    float *mlp_sm = nullptr;
    if constexpr (LEARNED) {
        mlp_sm = reinterpret_cast<float *>(smem_raw + mlp_offset<real, TX, TY, KP>());
        for (int p = threadIdx.x; p < MLP_P; p += blockDim.x) mlp_sm[p] = __ldg(mlp + p);
        if constexpr (sizeof(real) == 4) {
            __syncthreads();
            mlp_split_w2(mlp_sm);
        }
        // made visible by the first barrier inside stage_tile
    }
    stage_tile<real, TX, TY, KP, LEARNED>(sm, fs, fn, out, status, g, t, t, blockIdx.x * TX, blockIdx.y * TY, ca, cb,
                                          cc, ca_lo, cb_lo, mlp_sm, tma.on ? &tma.map : nullptr,
                                          fields.n ? &fields : nullptr);
}

// Batch of independent runs (uneven grid sizes, own parameters): one CTA per
// (run, tile) work item, in the order of the items, so that the hardware
// dispatches neighbouring tiles together and their halos stay in L2 (a
// persistent grid-stride loop let the CTAs drift apart and measured slower);
// tile_start[r] is the first item of run r (prefix sum, tile_start[nruns] =
// total).  Each run has its populations at offset `off` of the three shared
// buffers and its own status word.
// 16-byte aligned and sized: the kernel copies one descriptor into shared
// memory with 16-byte loads, so consecutive array elements must stay aligned
// and the whole struct must be covered by whole int4 words.
template <typename real>
struct __align__(16) BatchRun {
    Geo g;
    Tab<real> t;
    long long off;   // populations: element offset in the three buffers
    long long foff;  // stage fields: byte offset in the fields buffer
    int ntx, pad;
};
static_assert(sizeof(BatchRun<double>) % 16 == 0, "BatchRun<double> must be a whole number of int4 words");
static_assert(sizeof(BatchRun<float>) % 16 == 0, "BatchRun<float> must be a whole number of int4 words");

template <typename real, int TX, int TY, int KP>
__global__ void __launch_bounds__(FusedSmem<real, TX, TY, KP>::NT,
                                  // FP64: at most two (more would spill the per-item
                                  // state); FP32: as many as fit, like the single grid
                                  sizeof(real) == 4
                                      ? fused_min_ctas(sizeof(FusedSmem<real, TX, TY, KP>) + sizeof(BatchRun<real>),
                                                       FusedSmem<real, TX, TY, KP>::NT)
                                      : (fused_min_ctas(sizeof(FusedSmem<real, TX, TY, KP>) + sizeof(BatchRun<real>),
                                                        FusedSmem<real, TX, TY, KP>::NT) > 1 ? 2 : 1))
k_fused_batch(const real *__restrict__ fs, const real *fn, real *out, int *__restrict__ status,
              const BatchRun<real> *__restrict__ runs, const int *__restrict__ tile_start, int nruns,
              const __grid_constant__ Tab<real> tv, real ca, real cb, real ccoef, real ca_lo, real cb_lo,
              char *fields, const TmaMap *__restrict__ tmaps)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    auto &sm = *reinterpret_cast<FusedSmem<real, TX, TY, KP> *>(smem_raw);
    __shared__ __align__(16) BatchRun<real> run;
    const int item = blockIdx.x;
    int lo = 0, hi = nruns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(tile_start + mid) <= item) lo = mid;
        else hi = mid - 1;
    }
    {
        const int4 *src = reinterpret_cast<const int4 *>(runs + lo);
        int4 *dst = reinterpret_cast<int4 *>(&run);
        for (int w = threadIdx.x; w < (int)(sizeof(BatchRun<real>) / sizeof(int4)); w += blockDim.x)
            dst[w] = __ldg(src + w);
    }
    __syncthreads();
    const int lt = item - __ldg(tile_start + lo);
    const int x0 = (lt % run.ntx) * TX, y0 = (lt / run.ntx) * TY;
    const StageFields<real> fl = fields ? fields_of<real>(fields + run.foff, run.g) : StageFields<real>{};
    // the run's tensor map of fs lives in global memory, written by the host
    // before the launch: acquire it for the tensormap proxy before the thread
    // that issues the copy uses it
    const TmaMap *tm = tmaps ? tmaps + lo : nullptr;
    if (tm && threadIdx.x == 0)
        asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(tm) : "memory");
    stage_tile<real, TX, TY, KP>(sm, fs + run.off, fn + run.off, out + run.off, status + lo, run.g, tv, run.t, x0, y0,
                                 ca, cb, ccoef * (real)run.g.dt, ca_lo, cb_lo, nullptr, tm, fields ? &fl : nullptr);
}

// The moments pre-pass for a batch: one thread per node of every run (a
// grid-stride loop over the prefix sum node_start of the runs' node counts),
// writing each run's fields at its offset of the fields buffer.
template <typename real>
__global__ void __launch_bounds__(256) k_fields_batch(const real *__restrict__ fs, char *fields,
                                                      const BatchRun<real> *__restrict__ runs,
                                                      const long long *__restrict__ node_start, int nruns,
                                                      long long total, int *status)
{
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = nruns - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(node_start + mid) <= idx) lo = mid;
            else hi = mid - 1;
        }
        const BatchRun<real> &run = runs[lo];
        const Geo &g = run.g;
        const long long q = idx - __ldg(node_start + lo);
        const int j = (int)(q / g.nx), i = (int)(q - (long long)j * g.nx);
        const long long o = (long long)j * g.pitch + i;
        const real *f = fs + run.off;
        NodeMoments<real> m;
        if constexpr (sizeof(real) == 8)
            m = node_moments<real>([&](int k) { return __ldg(f + k * g.plane + o); }, g, run.t);
        else
            m = node_moments<real>(
                [&](int k) { return make_float2(__ldg(f + k * g.plane + o), __ldg(f + (NK + k) * g.plane + o)); }, g,
                run.t);
        const StageFields<real> out = fields_of<real>(fields + run.foff, g);
        out.n[o] = m.n;
        out.dp[o] = m.dp;
        out.ux[o] = m.ux;
        out.uy[o] = m.uy;
        out.T[o] = m.T;
        if constexpr (sizeof(real) == 4) out.E[o] = m.E;
        if (!m.ok) atomicOr(status + lo, 1);
    }
}

template <typename real, int TX, int TY, int KP, bool LEARNED = false>
cudaError_t fused_prepare_one()
{
    cudaError_t e = cudaFuncSetAttribute(k_fused<real, TX, TY, KP, LEARNED>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fused_smem_bytes<real, TX, TY, KP, LEARNED>());
    if (e != cudaSuccess || LEARNED) return e;
    return cudaFuncSetAttribute(k_fused_batch<real, TX, TY, KP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(FusedSmem<real, TX, TY, KP>));
}

template <typename real, int TX, int TY, int KP, bool LEARNED = false>
cudaError_t fused_launch_one(const real *fs, const real *fn, real *out, int *status, const Geo &g,
                             const Tab<real> &t, StageCoef c, const float *mlp, const TmaMap *tmap, void *fields,
                             cudaStream_t s)
{
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY);
    TmaArg tma{};
    if (tmap) {
        tma.map = *tmap;
        tma.on = 1;
    }
    StageFields<real> fl{};
    if (fields) {
        // the moments of fs first (one thread per node), then the stage
        fl = fields_of<real>(fields, g);
        const long long N = (long long)g.nx * g.ny;
        k_fields<real><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(fs, fl, status, g, t);
    }
    k_fused<real, TX, TY, KP, LEARNED><<<grid, FusedSmem<real, TX, TY, KP>::NT, fused_smem_bytes<real, TX, TY, KP, LEARNED>(), s>>>(
        fs, fn, out, status, g, t, (real)c.ca, (real)c.cb, (real)c.cc, (real)(c.ca - (double)(real)c.ca),
        (real)(c.cb - (double)(real)c.cb), mlp, tma, fl);
    return cudaGetLastError();
}

template <typename real, int TX, int TY, int KP>
cudaError_t fused_batch_launch_one(const real *fs, const real *fn, real *out, int *status, const void *runs,
                                   const int *tile_start, int nruns, int total, const Tab<real> &t, StageCoef c,
                                   void *fields, const long long *node_start, long long total_nodes,
                                   const TmaMap *tmaps, cudaStream_t s)
{
    if (total < 1) return cudaSuccess;
    if (fields && total_nodes > 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long long want = (total_nodes + 255) / 256, cap = 8LL * sms * 8;
        k_fields_batch<real><<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(
            fs, static_cast<char *>(fields), static_cast<const BatchRun<real> *>(runs), node_start, nruns, total_nodes,
            status);
    }
    k_fused_batch<real, TX, TY, KP><<<total, FusedSmem<real, TX, TY, KP>::NT, sizeof(FusedSmem<real, TX, TY, KP>), s>>>(
        fs, fn, out, status, static_cast<const BatchRun<real> *>(runs), tile_start, nruns, t, (real)c.ca, (real)c.cb,
        (real)c.cc, (real)(c.ca - (double)(real)c.ca), (real)(c.cb - (double)(real)c.cb), static_cast<char *>(fields),
        tmaps);
    return cudaGetLastError();
}

// Shapes compiled for each precision: TX x TY nodes per CTA, KP velocities
// advanced at once (KP lanes of TX*TY threads rounded up to whole warps).  Must match TILE_X/TILE_Y/TILE_K in
// olb_internal.cuh.
#define OLB_FUSED_SHAPE_CASES(real, DO) \
    DO(real, 8, 8, 4) DO(real, 16, 8, 2) DO(real, 16, 8, 1) DO(real, 32, 8, 1) DO(real, 32, 16, 1) DO(real, 8, 8, 8) \
    DO(real, 7, 8, 8) DO(real, 8, 8, 5)
// Shapes with a learned-weights instance (the default shapes of both precisions).
#define OLB_FUSED_LEARNED_CASES(real, DO) DO(real, 8, 8, 4) DO(real, 16, 8, 2) DO(real, 32, 16, 1)
#define OLB_FUSED_PREP_CASE(real, A, B, C) \
    if (!learned && tx == A && ty == B && kp == C) return fused_prepare_one<real, A, B, C>();
#define OLB_FUSED_PREP_LEARNED(real, A, B, C) \
    if (learned && tx == A && ty == B && kp == C) return fused_prepare_one<real, A, B, C, true>();
#define OLB_FUSED_LAUNCH_CASE(real, A, B, C)           \
    if (!mlp && tx == A && ty == B && kp == C)          \
        return fused_launch_one<real, A, B, C>(fs, fn, out, status, g, t, c, mlp, tma, fields, s);
#define OLB_FUSED_LAUNCH_LEARNED(real, A, B, C)                 \
    if (mlp && tx == A && ty == B && kp == C)                   \
        return fused_launch_one<real, A, B, C, true>(fs, fn, out, status, g, t, c, mlp, tma, fields, s);
#define OLB_FUSED_BATCH_CASE(real, A, B, C)                                                                  \
    if (tx == A && ty == B && kp == C)                                                                       \
        return fused_batch_launch_one<real, A, B, C>(fs, fn, out, status, runs, tile_start, nruns, total, t,     \
                                                     c, fields, node_start, total_nodes, tmaps, s);
#define OLB_DEFINE_FUSED(real)                                                                                \
    cudaError_t prepare_fused(real *, int tx, int ty, int kp, bool learned)                                   \
    {                                                                                                         \
        OLB_FUSED_SHAPE_CASES(real, OLB_FUSED_PREP_CASE)                                                      \
        OLB_FUSED_LEARNED_CASES(real, OLB_FUSED_PREP_LEARNED)                                                 \
        return cudaErrorInvalidValue;                                                                         \
    }                                                                                                         \
    cudaError_t launch_fused(const real *fs, const real *fn, real *out, int *status, const Geo &g,            \
                             const Tab<real> &t, StageCoef c, int tx, int ty, int kp, const float *mlp,       \
                             const TmaMap *tma, void *fields, cudaStream_t s)                                 \
    {                                                                                                         \
        OLB_FUSED_SHAPE_CASES(real, OLB_FUSED_LAUNCH_CASE)                                                    \
        OLB_FUSED_LEARNED_CASES(real, OLB_FUSED_LAUNCH_LEARNED)                                               \
        return cudaErrorInvalidValue;                                                                         \
    }                                                                                                         \
    cudaError_t launch_fused_batch(const real *fs, const real *fn, real *out, int *status, const void *runs,  \
                                   const int *tile_start, int nruns, int total, const Tab<real> &t,         \
                                   StageCoef c, int tx, int ty, int kp, void *fields,                         \
                                   const long long *node_start, long long total_nodes, const TmaMap *tmaps,   \
                                   cudaStream_t s)                                                            \
    {                                                                                                         \
        OLB_FUSED_SHAPE_CASES(real, OLB_FUSED_BATCH_CASE)                                                     \
        return cudaErrorInvalidValue;                                                                         \
    }                                                                                                         \
    size_t batch_run_bytes(real *) { return sizeof(BatchRun<real>); }                                         \
    void batch_run_fill(real *, void *dst, const Geo &g, const Tab<real> &t, long long off, long long foff,   \
                        int ntx)                                                                              \
    {                                                                                                         \
        BatchRun<real> r{};                                                                                   \
        r.g = g;                                                                                              \
        r.t = t;                                                                                              \
        r.off = off;                                                                                          \
        r.foff = foff;                                                                                        \
        r.ntx = ntx;                                                                                          \
        *static_cast<BatchRun<real> *>(dst) = r;                                                              \
    }

}  // namespace olb
