// olb_internal.cuh -- types shared by the library's translation units.
//
// Device data layout (all arrays owned by the context):
//   populations  FP64: double f[25][ny][pitch]   kappa = 5*k1 + k2 (x-major
//                velocity index), pitch = nx rounded up to 32 elements so
//                every row starts on a 128/256-byte boundary
//                FP32: float f[2][25][ny][pitch], the value of population
//                kappa held as the unevaluated sum hi + lo of plane kappa
//                (hi, the value rounded to FP32) and plane 25 + kappa (lo,
//                the remainder rounded to FP32): compensated storage, so that
//                an RK increment far below FP32 resolution of f survives
//   status       int                     bit 0: invalid moment seen; bit 1: a
//                                        bounded wait for a TMA copy ran out
// The stage kernel keeps moments, force and wall densities of its tile in
// shared memory; no other global scratch is needed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

struct olb_params;

namespace olb {

constexpr int NQ = 5;   // Gauss-Hermite points per axis (Table trots)
constexpr int NK = 25;  // velocities

// Planes of one population buffer: 25 in FP64; 50 in FP32 (hi planes, then
// the lo planes of the compensated storage).
template <typename real>
constexpr int pop_planes()
{
    return sizeof(real) == 8 ? NK : 2 * NK;
}

// Geometry and physical parameters, passed by value to every kernel.
struct Geo {
    int nx, ny, pitch;
    int walls;           // 1: the x sides are not periodic (walls or specular)
    int wall_lo, wall_hi;  // diffuse wall at x = 0 / at x = nx ds (Sec. 3.4.2)
    int spec_lo, spec_hi;  // specular plane at x = 0 / at x = nx ds (Sec. 3.4.1)
    int spec_y;            // specular planes at y = 0 and y = ny ds
    long long plane;     // pitch * ny
    double ds, inv_ds, inv_ds3, dt, inv_tau, sigma, a, b;
};

// Velocity-space tables (Sec. 2.2, 2.3), in the population precision.
template <typename real>
struct Tab {
    real R[NQ];          // roots of He_5, ascending
    real R2[NQ];         // R^2
    real R2lo[NQ];       // R^2 - R2 (the remainder of R^2 in this precision; 0 in FP64)
    real D[NQ][NQ];      // (d_p f)_k = sum_k' D[k][k'] f_k'   (Eq. derf)
    real wHe[NQ][NQ];    // w_k He_l(p_k), l = 0..4            (Eq. g_alpha)
    real geqw[2][NK];    // g_{k1}(0, Tw) g_{k2}(uw, Tw) per wall
    real inv_den[2];     // 1 / sum_incoming g g p per wall    (Eq. nw)
};

// Host-side tables in FP64 (computed once from the closed forms).
struct HostTables {
    double R[NQ], W[NQ], D[NQ][NQ], wHe[NQ][NQ];
};
void host_tables(HostTables *t);
double host_g(const HostTables &t, int k, double u, double T);

template <typename real>
void fill_tab(Tab<real> *tab, const HostTables &h, const double Tw[2], const double uw[2]);

// Parameter validation of olb_create (OLB_OK / OLB_ERR_ARG / OLB_ERR_CFL)
// and the mapping of CUDA errors to status codes (olb_api.cu).
int validate_params(const ::olb_params *p);
// Host fields [N] admissible as an initial state: n > 0, b n < 1, T > 0, all
// finite (olb_api.cu; large arrays are checked by several host threads).
bool fields_admissible(const double *n, const double *ux, const double *uy, const double *T, size_t N, double b);
void set_sides(Geo *g, const ::olb_params *p);
int cuda_status(cudaError_t e);

// A TMA tensor map (CUtensorMap, 128 bytes, 64-byte aligned) over one
// population buffer as a 3-D tensor [planes][ny][nx] with row stride pitch,
// box (TX + 8) x (TY + 6) x planes: the staged region of a tile in one copy.
struct alignas(64) TmaMap {
    unsigned char bytes[128];
};
// Kernel argument: the map and whether to use it (tiles whose staged region
// lies inside the grid are loaded with one TMA copy when on != 0).
struct alignas(64) TmaArg {
    TmaMap map;
    int on;
};
// Encode the map of buffer `base` for tile shape tx x ty (olb_api.cu); false
// if the shape's rows are not a multiple of 16 bytes or the driver refuses.
bool tma_encode(TmaMap *out, const void *base, bool fp64, const Geo &g, int tx, int ty);

// RK-3 stage coefficients: out = ca f^n + cb f_s + cc L[f_s] (Eq. rk3).
struct StageCoef {
    double ca, cb, cc;
};

// Launchers, one set per precision (olb_fp64.cu, olb_fp32.cu).  Output
// pointers of launch_moments_out may be NULL to skip a field.  launch_fused
// with fields != NULL (a buffer of fields_bytes(g)) runs the per-node
// moments pre-pass first and lets the stage kernel read its results.
#define OLB_DECLARE_LAUNCHERS(real)                                                                    \
    cudaError_t prepare_fused(real *, int tx, int ty, int kp, bool learned);                           \
    cudaError_t launch_fused(const real *fs, const real *fn, real *out, int *status, const Geo &g,     \
                             const Tab<real> &t, StageCoef c, int tx, int ty, int kp,                  \
                             const float *mlp, const TmaMap *tma, void *fields, cudaStream_t s);       \
    cudaError_t launch_fused_batch(const real *fs, const real *fn, real *out, int *status,             \
                                   const void *runs, const int *tile_start, int nruns, int total,      \
                                   const Tab<real> &t, StageCoef c, int tx, int ty, int kp,            \
                                   void *fields,                                                       \
                                   const long long *node_start, long long total_nodes,                 \
                                   const TmaMap *tmaps, cudaStream_t s);                               \
    size_t batch_run_bytes(real *);                                                                    \
    void batch_run_fill(real *, void *dst, const Geo &g, const Tab<real> &t, long long off,            \
                        long long foff, int ntx);                                                      \
    cudaError_t launch_init(real *f, const double *n, const double *ux, const double *uy,              \
                            const double *T, const Geo &g, const Tab<double> &t, cudaStream_t s);       \
    cudaError_t launch_moments_out(const real *f, double *n, double *ux, double *uy, double *T,        \
                                   const Geo &g, const Tab<double> &t, cudaStream_t s);                 \
    cudaError_t launch_to_f64(const real *f, double *dst, const Geo &g, cudaStream_t s);               \
    cudaError_t launch_from_f64(real *f, const double *src, const Geo &g, cudaStream_t s);             \
    cudaError_t launch_totals(const real *f, double *partial, double *out, const Geo &g,               \
                              const Tab<double> &t, cudaStream_t s);

OLB_DECLARE_LAUNCHERS(double)
OLB_DECLARE_LAUNCHERS(float)

// Bytes of the per-node moment fields of the stage pre-pass: 5 planes of
// pitch * ny 8-byte elements.
inline size_t fields_bytes(const Geo &g) { return (size_t)5 * g.plane * 8; }

// Global sums (olb_totals): fixed grid of the first reduction pass, whose
// per-block partial sums (4 each) the second pass adds in a fixed order.
constexpr int TOTALS_BLOCKS = 1024, TOTALS_THREADS = 256;

// Stage-kernel shapes compiled for both precisions: TX x TY nodes per CTA
// and KP velocities advanced at once.
constexpr int NUM_TILES = 8;
constexpr int TILE_X[NUM_TILES] = {8, 16, 16, 32, 32, 8, 7, 8};
constexpr int TILE_Y[NUM_TILES] = {8, 8, 8, 8, 16, 8, 8, 8};
constexpr int TILE_K[NUM_TILES] = {4, 2, 1, 1, 1, 8, 8, 5};

}  // namespace olb
