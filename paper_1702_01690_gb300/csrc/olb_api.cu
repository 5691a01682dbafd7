// olb_api.cu -- the C ABI declared in include/olb.h: parameter validation,
// device memory, velocity-space tables, CUDA-graph replay of RK-3 steps.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include <cuda.h>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/olb.h"
#include "olb_internal.cuh"

using namespace olb;

// ---------------------------------------------------------------- TMA maps

namespace {
// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (the library links only the CUDA runtime).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    });
    return fn;
}
}  // namespace

bool olb::tma_encode(TmaMap *out, const void *base, bool fp64, const Geo &g, int tx, int ty)
{
    static_assert(sizeof(TmaMap) == sizeof(CUtensorMap), "TmaMap must hold a CUtensorMap");
    const size_t elt = fp64 ? 8 : 4;
    const unsigned hx = (unsigned)tx + 8, hy = (unsigned)ty + 6;
    // the box's rows must be whole 16-byte units, and its x start x0 - 4
    // (x0 a multiple of tx) must sit on a 16-byte boundary for every tile
    if ((hx * elt) % 16 != 0 || ((size_t)tx * elt) % 16 != 0 || (4 * elt) % 16 != 0) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint32_t planes = fp64 ? (cuuint32_t)pop_planes<double>() : (cuuint32_t)pop_planes<float>();
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, planes};
    const cuuint64_t strides[2] = {(cuuint64_t)g.pitch * elt, (cuuint64_t)g.plane * elt};
    const cuuint32_t box[3] = {hx, hy, planes};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap m;
    const CUresult r = fn(&m, fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                          const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    std::memcpy(out->bytes, &m, sizeof(m));
    return true;
}

// ---------------------------------------------------------------- tables

namespace olb {

// Probabilists' Hermite polynomial He_l(x) (orthogonal under the weight
// exp(-x^2/2)/sqrt(2 pi), Eq. eweight).
static double he(int l, double x)
{
    double a = 1.0, b = x;
    if (l == 0) return a;
    for (int k = 1; k < l; ++k) {
        const double c = x * b - k * a;
        a = b;
        b = c;
    }
    return b;
}

void host_tables(HostTables *t)
{
    // Table trots: roots of He_5 and W_q = 5!/He_6(R_q)^2 in closed form.
    const double r10 = std::sqrt(10.0);
    const double big = std::sqrt(5.0 + r10), small = std::sqrt(5.0 - r10);
    const double R[NQ] = {-big, -small, 0.0, small, big};
    const double W[NQ] = {(7.0 - 2.0 * r10) / 60.0, (7.0 + 2.0 * r10) / 60.0, 8.0 / 15.0,
                          (7.0 + 2.0 * r10) / 60.0, (7.0 - 2.0 * r10) / 60.0};
    for (int k = 0; k < NQ; ++k) {
        t->R[k] = R[k];
        t->W[k] = W[k];
        for (int l = 0; l < NQ; ++l) t->wHe[k][l] = W[k] * he(l, R[k]);
    }
    // Eq. derf: (d_p f)_k = -w_k sum_{l<N} He_{l+1}(p_k)/l! sum_k' f_k' He_l(p_k')
    //         = sum_k' D[k][k'] f_k'
    const double fact[4] = {1.0, 1.0, 2.0, 6.0};
    for (int k = 0; k < NQ; ++k)
        for (int kp = 0; kp < NQ; ++kp) {
            double s = 0.0;
            for (int l = 0; l < 4; ++l) s += he(l + 1, R[k]) * he(l, R[kp]) / fact[l];
            t->D[k][kp] = -W[k] * s;
        }
}

// g_k(u, T) of Eq. g_alpha (N = 4, m = 1).
double host_g(const HostTables &t, int k, double u, double T)
{
    const double th = T - 1.0;
    const double c[5] = {1.0, u, 0.5 * (u * u + th), u * u * u / 6.0 + 0.5 * th * u,
                         u * u * u * u / 24.0 + 0.25 * th * u * u + 0.125 * th * th};
    double s = 0.0;
    for (int l = 0; l < 5; ++l) s += t.wHe[k][l] * c[l];
    return s;
}

template <typename real>
void fill_tab(Tab<real> *tab, const HostTables &h, const double Tw[2], const double uw[2])
{
    for (int k = 0; k < NQ; ++k) {
        tab->R[k] = (real)h.R[k];
        tab->R2[k] = (real)(h.R[k] * h.R[k]);
        tab->R2lo[k] = (real)(h.R[k] * h.R[k] - (double)tab->R2[k]);
        for (int q = 0; q < NQ; ++q) {
            tab->D[k][q] = (real)h.D[k][q];
            tab->wHe[k][q] = (real)h.wHe[k][q];
        }
    }
    for (int s = 0; s < 2; ++s) {
        double den = 0.0;
        for (int k1 = 0; k1 < NQ; ++k1)
            for (int k2 = 0; k2 < NQ; ++k2) {
                const double gg = host_g(h, k1, 0.0, Tw[s]) * host_g(h, k2, uw[s], Tw[s]);
                tab->geqw[s][NQ * k1 + k2] = (real)gg;
                // incoming: p_x > 0 at the wall x = 0, p_x < 0 at x = nx ds
                const bool incoming = s == 0 ? (k1 > 2) : (k1 < 2);
                if (incoming) den += gg * h.R[k1];
            }
        tab->inv_den[s] = (real)(den != 0.0 ? 1.0 / den : 0.0);
    }
}
template void fill_tab<double>(Tab<double> *, const HostTables &, const double *, const double *);
template void fill_tab<float>(Tab<float> *, const HostTables &, const double *, const double *);

}  // namespace olb

// ---------------------------------------------------------------- allocator

static olb_alloc_fn g_alloc = nullptr;
static olb_free_fn g_free = nullptr;
static void *g_alloc_user = nullptr;

extern "C" int olb_set_allocator(olb_alloc_fn alloc, olb_free_fn release, void *user)
{
    if ((alloc == nullptr) != (release == nullptr)) return OLB_ERR_ARG;
    g_alloc = alloc;
    g_free = release;
    g_alloc_user = user;
    return OLB_OK;
}

// ---------------------------------------------------------------- context

constexpr int GRAPH_STEPS = 16;  // RK-3 steps per replay of the long graph

struct olb_ctx {
    olb_params p;
    int device;
    cudaStream_t stream;
    Geo geo;
    Tab<double> tab64;
    Tab<float> tab32;
    size_t elt;                 // bytes per population value
    void *f[3];                 // f^n, f^(1), f^(2)
    int *status;
    int tx, ty, kp;             // stage-kernel tile shape and velocity lanes
    float *mlp;                 // learned WENO weights: network parameters
    bool mlp_set;
    double *stage4;             // FP64 [4][ny][nx] staging for host transfers
    double *totals;             // olb_totals: partial sums, then the sums
    void *fields;               // moments of the stage's input (fields_bytes), read by the stage kernel
    struct Alloc {
        void *ptr;
        size_t bytes;
    } allocs[12];
    int nallocs;
    olb_alloc_fn afn;
    olb_free_fn ffn;
    void *auser;
    cudaStream_t cap;
    cudaGraphExec_t exec1, execG;
    bool initialized;
    TmaMap tma[3];              // TMA maps of f^n, f^(1), f^(2) for the current shape
    bool tma_ok;                // the shape's staged rows suit TMA and the maps exist
};

static void *ctx_alloc(olb_ctx *c, size_t bytes)
{
    void *p = nullptr;
    if (c->afn) {
        p = c->afn(bytes, (void *)c->stream, c->auser);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->allocs[c->nallocs++] = {p, bytes};
    return p;
}

static void ctx_free_all(olb_ctx *c)
{
    for (int k = 0; k < c->nallocs; ++k) {
        if (c->ffn)
            c->ffn(c->allocs[k].ptr, c->allocs[k].bytes, (void *)c->stream, c->auser);
        else
            cudaFree(c->allocs[k].ptr);
    }
    c->nallocs = 0;
}

static bool is_fp64(const olb_ctx *c) { return c->p.precision == OLB_FP64; }

// One RK-3 step (Eq. rk3) as 3 launches of the fused stage kernel:
//   f1 = f + dt L[f];  f2 = 3/4 f + 1/4 f1 + 1/4 dt L[f1];
//   f  = 1/3 f + 2/3 f2 + 2/3 dt L[f2]  (written in place: f is read only at
//   the node being written).
static StageCoef stage_coef(double dt, int st)
{
    const StageCoef coef[3] = {{0.0, 1.0, dt}, {0.75, 0.25, 0.25 * dt}, {1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0 * dt}};
    return coef[st];
}

template <typename real>
static const Tab<real> &ctx_tab(const olb_ctx *c);
template <>
const Tab<double> &ctx_tab<double>(const olb_ctx *c) { return c->tab64; }
template <>
const Tab<float> &ctx_tab<float>(const olb_ctx *c) { return c->tab32; }

template <typename real>
static cudaError_t enqueue_stage(olb_ctx *c, int st, cudaStream_t s)
{
    real *f0 = (real *)c->f[0], *f1 = (real *)c->f[1], *f2 = (real *)c->f[2];
    const real *src[3] = {f0, f1, f2};
    real *dst[3] = {f1, f2, f0};
    const StageCoef coef = stage_coef(c->p.dt, st);
    const int src_buf[3] = {0, 1, 2};
    return launch_fused(src[st], f0, dst[st], c->status, c->geo, ctx_tab<real>(c), coef, c->tx, c->ty, c->kp,
                        c->p.weno_mode == OLB_WENO_LEARNED ? c->mlp : nullptr,
                        c->tma_ok ? &c->tma[src_buf[st]] : nullptr, c->fields, s);
}

template <typename real>
static cudaError_t enqueue_step(olb_ctx *c, cudaStream_t s)
{
    for (int st = 0; st < 3; ++st) {
        cudaError_t e = enqueue_stage<real>(c, st, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t enqueue_steps(olb_ctx *c, int n, cudaStream_t s)
{
    for (int k = 0; k < n; ++k) {
        cudaError_t e = is_fp64(c) ? enqueue_step<double>(c, s) : enqueue_step<float>(c, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t build_graph(olb_ctx *c, int nsteps, cudaGraphExec_t *exec)
{
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t e2 = enqueue_steps(c, nsteps, c->cap);
    e = cudaStreamEndCapture(c->cap, &graph);
    if (e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return e2;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    return e;
}

int olb::cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return OLB_OK;
    if (e == cudaErrorMemoryAllocation) return OLB_ERR_NOMEM;
    return OLB_ERR_CUDA;
}

extern "C" const char *olb_status_string(int status)
{
    switch (status) {
    case OLB_OK: return "OLB_OK";
    case OLB_ERR_ARG: return "OLB_ERR_ARG: invalid argument";
    case OLB_ERR_CFL: return "OLB_ERR_CFL: p_max dt/ds >= 1 or dt > 2.5 tau";
    case OLB_ERR_CUDA: return "OLB_ERR_CUDA: a CUDA runtime call failed";
    case OLB_ERR_DIVERGED: return "OLB_ERR_DIVERGED: invalid moment (non-finite, n <= 0, b n >= 1 or T <= 0)";
    case OLB_ERR_TIMEOUT: return "OLB_ERR_TIMEOUT: a bounded device wait ran out";
    case OLB_ERR_STATE: return "OLB_ERR_STATE: call out of order";
    case OLB_ERR_NOMEM: return "OLB_ERR_NOMEM: device allocation failed";
    default: return "unknown olb status";
    }
}

void olb::set_sides(Geo *g, const olb_params *p)
{
    g->walls = p->side_x != OLB_SIDE_PERIODIC;
    g->wall_lo = p->side_x == OLB_SIDE_DIFFUSE;
    g->wall_hi = p->side_x == OLB_SIDE_DIFFUSE || p->side_x == OLB_SIDE_SPECULAR_DIFFUSE;
    g->spec_lo = p->side_x == OLB_SIDE_SPECULAR || p->side_x == OLB_SIDE_SPECULAR_DIFFUSE;
    g->spec_hi = p->side_x == OLB_SIDE_SPECULAR;
    g->spec_y = p->side_y == OLB_SIDE_SPECULAR;
}

int olb::validate_params(const olb_params *p)
{
    if (!p) return OLB_ERR_ARG;
    if (p->nx < 1 || p->ny < 1) return OLB_ERR_ARG;
    if (p->side_x < OLB_SIDE_PERIODIC || p->side_x > OLB_SIDE_SPECULAR_DIFFUSE) return OLB_ERR_ARG;
    if (p->side_y != OLB_SIDE_PERIODIC && p->side_y != OLB_SIDE_SPECULAR) return OLB_ERR_ARG;
    if (p->side_x != OLB_SIDE_PERIODIC && p->nx < 3) return OLB_ERR_ARG;
    if (p->side_y != OLB_SIDE_PERIODIC && p->ny < 3) return OLB_ERR_ARG;
    if (p->precision != OLB_FP64 && p->precision != OLB_FP32_KAHAN) return OLB_ERR_ARG;
    if (p->weno_mode != OLB_WENO_JS && p->weno_mode != OLB_WENO_LEARNED) return OLB_ERR_ARG;
    if (!(p->ds > 0.0) || !(p->dt > 0.0) || !(p->tau > 0.0)) return OLB_ERR_ARG;
    if (!std::isfinite(p->ds) || !std::isfinite(p->dt) || !std::isfinite(p->tau)) return OLB_ERR_ARG;
    if (!(p->sigma >= 0.0) || !(p->b >= 0.0) || !std::isfinite(p->a) || !std::isfinite(p->sigma) ||
        !std::isfinite(p->b))
        return OLB_ERR_ARG;
    for (int s = 0; s < 2; ++s) {
        const bool wall = p->side_x == OLB_SIDE_DIFFUSE || (s == 1 && p->side_x == OLB_SIDE_SPECULAR_DIFFUSE);
        if (wall && (!(p->Tw[s] > 0.0) || !std::isfinite(p->Tw[s]) || !std::isfinite(p->uw[s]))) return OLB_ERR_ARG;
    }
    if ((long long)p->nx * p->ny > (1LL << 31) / 32) return OLB_ERR_ARG;
    const double pmax = std::sqrt(5.0 + std::sqrt(10.0));
    if (!(pmax * p->dt / p->ds < 1.0)) return OLB_ERR_CFL;
    if (p->dt > 2.5 * p->tau) return OLB_ERR_CFL;
    return OLB_OK;
}

static cudaError_t prepare_tile(olb_ctx *c)
{
    const bool learned = c->p.weno_mode == OLB_WENO_LEARNED;
    cudaError_t e = is_fp64(c) ? prepare_fused((double *)nullptr, c->tx, c->ty, c->kp, learned)
                               : prepare_fused((float *)nullptr, c->tx, c->ty, c->kp, learned);
    if (e != cudaSuccess) return e;
    // TMA maps of the three buffers for this shape (tiles whose region lies
    // inside the grid then load it with one copy); without them every tile
    // takes the per-element loads
    c->tma_ok = true;
    for (int k = 0; k < 3 && c->tma_ok; ++k)
        c->tma_ok = tma_encode(&c->tma[k], c->f[k], is_fp64(c), c->geo, c->tx, c->ty);
    return cudaSuccess;
}

// Default shape, the fastest measured on a GB300 for each precision.  FP64:
// 8 x 8 nodes with 4 velocity lanes (its faces of all 25 velocities fit in
// shared memory, so a stage has one face pass and one barrier), except that
// small grids take 7 x 8 tiles with 8 lanes when that lowers the most nodes
// any SM has to advance (1024 x 8: 147 tiles of 56 nodes rather than 128 of
// 64 on 152 SMs).  FP32 (compensated pairs, twice the staged bytes of plain
// FP32): 8 x 8 nodes with 8 lanes on every grid (4096^2: 10.2 ms per stage
// against 11.0 for 8 x 8 x 4, 14.0 for 16 x 8 x 2 and 14.2 for 32 x 16 x 1),
// 4 lanes with learned weights.  olb_set_tile overrides.
static void default_tile(olb_ctx *c)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
    const bool learned = c->p.weno_mode == OLB_WENO_LEARNED;
    const bool fp64 = is_fp64(c);
    const int narrow = 6;
    auto tiles = [&](int k) {
        return (long long)((c->geo.nx + TILE_X[k] - 1) / TILE_X[k]) * ((c->geo.ny + TILE_Y[k] - 1) / TILE_Y[k]);
    };
    auto most_nodes = [&](int k) { return (tiles(k) + sms - 1) / sms * TILE_X[k] * TILE_Y[k]; };
    int k = fp64 || learned ? 0 : 7;
    if (fp64 && !learned && most_nodes(narrow) < most_nodes(0)) k = narrow;
    c->tx = TILE_X[k];
    c->ty = TILE_Y[k];
    c->kp = TILE_K[k];
}

extern "C" int olb_create(const olb_params *p, void *stream, olb_ctx **out)
{
    if (!out) return OLB_ERR_ARG;
    *out = nullptr;
    int v = validate_params(p);
    if (v != OLB_OK) return v;
    olb_ctx *c = new (std::nothrow) olb_ctx();
    if (!c) return OLB_ERR_NOMEM;
    c->p = *p;
    c->stream = (cudaStream_t)stream;
    c->afn = g_alloc;
    c->ffn = g_free;
    c->auser = g_alloc_user;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return OLB_ERR_CUDA;
    }
    Geo &g = c->geo;
    g.nx = p->nx;
    g.ny = p->ny;
    g.pitch = (p->nx + 31) / 32 * 32;
    g.plane = (long long)g.pitch * g.ny;
    set_sides(&g, p);
    g.ds = p->ds;
    g.inv_ds = 1.0 / p->ds;
    g.inv_ds3 = 1.0 / (p->ds * p->ds * p->ds);
    g.dt = p->dt;
    g.inv_tau = 1.0 / p->tau;
    g.sigma = p->sigma;
    g.a = p->a;
    g.b = p->b;
    HostTables h;
    host_tables(&h);
    fill_tab<double>(&c->tab64, h, p->Tw, p->uw);
    fill_tab<float>(&c->tab32, h, p->Tw, p->uw);
    c->elt = is_fp64(c) ? sizeof(double) : sizeof(float);
    const size_t pop = (size_t)(is_fp64(c) ? pop_planes<double>() : pop_planes<float>()) * g.plane * c->elt;
    const size_t N = (size_t)g.nx * g.ny;
    for (int k = 0; k < 3; ++k) c->f[k] = ctx_alloc(c, pop);
    c->status = (int *)ctx_alloc(c, 256);
    c->stage4 = (double *)ctx_alloc(c, 4 * N * sizeof(double));
    c->mlp = p->weno_mode == OLB_WENO_LEARNED ? (float *)ctx_alloc(c, 1348 * sizeof(float)) : nullptr;
    // olb_totals: TOTALS_BLOCKS x 4 partial sums, then the 4 sums
    c->totals = (double *)ctx_alloc(c, (size_t)(4 * TOTALS_BLOCKS + 4) * sizeof(double));
    c->fields = ctx_alloc(c, fields_bytes(g));
    default_tile(c);
    bool ok = c->f[0] && c->f[1] && c->f[2] && c->status && c->stage4 && c->totals && c->fields &&
              (p->weno_mode != OLB_WENO_LEARNED || c->mlp);
    cudaError_t e = cudaSuccess;
    if (ok) {
        // zero everything once so padding lanes never hold garbage
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaMemsetAsync(c->f[k], 0, pop, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
        if (e == cudaSuccess) e = prepare_tile(c);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (!ok || e != cudaSuccess) {
        cudaGetLastError();
        ctx_free_all(c);
        delete c;
        return ok ? cuda_status(e) : OLB_ERR_NOMEM;
    }
    *out = c;
    return OLB_OK;
}

extern "C" void olb_destroy(olb_ctx *c)
{
    if (!c) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->exec1) cudaGraphExecDestroy(c->exec1);
    if (c->execG) cudaGraphExecDestroy(c->execG);
    if (c->cap) cudaStreamDestroy(c->cap);
    ctx_free_all(c);
    cudaGetLastError();
    cudaSetDevice(prev);
    delete c;
}

static void drop_graphs(olb_ctx *c);

// Scoped switch to the context's device.
struct DeviceGuard {
    int prev;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() { cudaSetDevice(prev); }
};

static int init_from_device(olb_ctx *c, const double *n, const double *ux, const double *uy, const double *T)
{
    cudaError_t e = is_fp64(c) ? launch_init((double *)c->f[0], n, ux, uy, T, c->geo, c->tab64, c->stream)
                               : launch_init((float *)c->f[0], n, ux, uy, T, c->geo, c->tab64, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    c->initialized = true;
    return OLB_OK;
}

// Host fields admissible as an initial state: n > 0, b n < 1, T > 0, all
// finite (NaN fails every comparison).  One pass without early exits over
// [q0, q1).
static bool admissible_range(const double *n, const double *ux, const double *uy, const double *T, size_t q0,
                             size_t q1, double b)
{
    const double inf = HUGE_VAL;
    int ok = 1;
    for (size_t q = q0; q < q1; ++q)
        ok &= (n[q] > 0.0) & (n[q] < inf) & (b * n[q] < 1.0) & (T[q] > 0.0) & (T[q] < inf) & (ux[q] > -inf) &
              (ux[q] < inf) & (uy[q] > -inf) & (uy[q] < inf);
    return ok != 0;
}

// The check is bound by host memory bandwidth (32 B per node): grids of more
// than 2^19 nodes are split over up to 16 host threads, at least 2^18 nodes
// each (a 4096^2 grid reads 537 MB).
bool olb::fields_admissible(const double *n, const double *ux, const double *uy, const double *T, size_t N,
                            double b)
{
    constexpr size_t CHUNK = size_t(1) << 18;
    const unsigned hw = std::thread::hardware_concurrency();
    size_t nt = (N + CHUNK - 1) / CHUNK;
    if (nt > 16) nt = 16;
    if (hw > 0 && nt > hw) nt = hw;
    if (N <= 2 * CHUNK || nt < 2) return admissible_range(n, ux, uy, T, 0, N, b);
    std::vector<char> ok(nt, 0);
    std::vector<std::thread> th;
    th.reserve(nt - 1);
    const size_t per = (N + nt - 1) / nt;
    try {
        for (size_t k = 1; k < nt; ++k) {
            const size_t q0 = k * per, q1 = q0 + per < N ? q0 + per : N;
            th.emplace_back([=, &ok] { ok[k] = admissible_range(n, ux, uy, T, q0, q1, b); });
        }
    } catch (...) {
        // no thread could be started: check the rest here
        for (auto &t : th) t.join();
        bool all = admissible_range(n, ux, uy, T, 0, per, b);
        for (size_t k = 1; k < nt; ++k) {
            const size_t q0 = k * per, q1 = q0 + per < N ? q0 + per : N;
            all = all && (k <= th.size() ? ok[k] != 0 : admissible_range(n, ux, uy, T, q0, q1, b));
        }
        return all;
    }
    ok[0] = admissible_range(n, ux, uy, T, 0, per, b);
    for (auto &t : th) t.join();
    for (size_t k = 0; k < nt; ++k)
        if (!ok[k]) return false;
    return true;
}

// Device address of page-locked (pinned, mapped) host memory, which kernels
// read and write directly; nullptr for anything else (pageable memory takes
// a staging copy).
static void *mapped_view(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

extern "C" int olb_init_fields(olb_ctx *c, const double *n, const double *ux, const double *uy, const double *T)
{
    if (!c || !n || !ux || !uy || !T) return OLB_ERR_ARG;
    const size_t N = (size_t)c->geo.nx * c->geo.ny;
    if (!fields_admissible(n, ux, uy, T, N, c->p.b)) return OLB_ERR_ARG;
    DeviceGuard dg(c->device);
    const double *src[4] = {n, ux, uy, T};
    const double *dev[4];
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
        dev[k] = static_cast<const double *>(mapped_view(src[k]));
        if (!dev[k]) {
            e = cudaMemcpyAsync(c->stage4 + k * N, src[k], N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
            dev[k] = c->stage4 + k * N;
        }
    }
    if (e != cudaSuccess) return cuda_status(e);
    int r = init_from_device(c, dev[0], dev[1], dev[2], dev[3]);
    if (r != OLB_OK) return r;
    return cuda_status(cudaStreamSynchronize(c->stream));
}

extern "C" int olb_init_fields_device(olb_ctx *c, const double *n, const double *ux, const double *uy,
                                      const double *T)
{
    if (!c || !n || !ux || !uy || !T) return OLB_ERR_ARG;
    DeviceGuard dg(c->device);
    return init_from_device(c, n, ux, uy, T);
}

extern "C" int olb_step_async(olb_ctx *c, int nsteps)
{
    if (!c || nsteps < 0) return OLB_ERR_ARG;
    if (!c->initialized) return OLB_ERR_STATE;
    if (c->p.weno_mode == OLB_WENO_LEARNED && !c->mlp_set) return OLB_ERR_STATE;
    if (nsteps == 0) return OLB_OK;
    DeviceGuard dg(c->device);
    cudaError_t e = cudaSuccess;
    if (!c->cap) {
        e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = build_graph(c, 1, &c->exec1);
        if (e == cudaSuccess) e = build_graph(c, GRAPH_STEPS, &c->execG);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_status(e);
        }
    }
    int k = 0;
    for (; k + GRAPH_STEPS <= nsteps && e == cudaSuccess; k += GRAPH_STEPS) e = cudaGraphLaunch(c->execG, c->stream);
    for (; k < nsteps && e == cudaSuccess; ++k) e = cudaGraphLaunch(c->exec1, c->stream);
    return cuda_status(e);
}

extern "C" int olb_get_status(olb_ctx *c)
{
    if (!c) return OLB_ERR_ARG;
    DeviceGuard dg(c->device);
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return (h & 2) ? OLB_ERR_TIMEOUT : (h ? OLB_ERR_DIVERGED : OLB_OK);
}

extern "C" int olb_step(olb_ctx *c, int nsteps)
{
    int r = olb_step_async(c, nsteps);
    if (r != OLB_OK) return r;
    return olb_get_status(c);
}

static int moments_device(olb_ctx *c, double *n, double *ux, double *uy, double *T)
{
    cudaError_t e = is_fp64(c) ? launch_moments_out((const double *)c->f[0], n, ux, uy, T, c->geo, c->tab64, c->stream)
                               : launch_moments_out((const float *)c->f[0], n, ux, uy, T, c->geo, c->tab64, c->stream);
    return cuda_status(e);
}

extern "C" int olb_moments_device(olb_ctx *c, double *n, double *ux, double *uy, double *T)
{
    if (!c) return OLB_ERR_ARG;
    if (!c->initialized) return OLB_ERR_STATE;
    DeviceGuard dg(c->device);
    return moments_device(c, n, ux, uy, T);
}

extern "C" int olb_moments(olb_ctx *c, double *n, double *ux, double *uy, double *T)
{
    if (!c) return OLB_ERR_ARG;
    if (!c->initialized) return OLB_ERR_STATE;
    DeviceGuard dg(c->device);
    const size_t N = (size_t)c->geo.nx * c->geo.ny;
    double *host[4] = {n, ux, uy, T};
    double *dev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool staged[4] = {false, false, false, false};
    for (int k = 0; k < 4; ++k) {
        if (!host[k]) continue;
        dev[k] = static_cast<double *>(mapped_view(host[k]));
        if (!dev[k]) {
            dev[k] = c->stage4 + k * N;
            staged[k] = true;
        }
    }
    int r = moments_device(c, dev[0], dev[1], dev[2], dev[3]);
    if (r != OLB_OK) return r;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        if (staged[k]) e = cudaMemcpyAsync(host[k], dev[k], N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_status(e);
}

// Global sums of the current populations (FP64, fixed order) into device
// out[4] on the context's stream.
static cudaError_t enqueue_totals(olb_ctx *c, double *out)
{
    double *partial = c->totals;
    return is_fp64(c) ? launch_totals((const double *)c->f[0], partial, out, c->geo, c->tab64, c->stream)
                      : launch_totals((const float *)c->f[0], partial, out, c->geo, c->tab64, c->stream);
}

extern "C" int olb_totals(olb_ctx *c, double *out)
{
    if (!c || !out) return OLB_ERR_ARG;
    if (!c->initialized) return OLB_ERR_STATE;
    DeviceGuard dg(c->device);
    double *dev = c->totals + 4 * TOTALS_BLOCKS;
    cudaError_t e = enqueue_totals(c, dev);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dev, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_status(e);
}

extern "C" int olb_step_totals(olb_ctx *c, int nsteps, int every, double *out)
{
    if (!c || !out || nsteps < 0 || every < 1) return OLB_ERR_ARG;
    if (!c->initialized) return OLB_ERR_STATE;
    if (c->p.weno_mode == OLB_WENO_LEARNED && !c->mlp_set) return OLB_ERR_STATE;
    const long long nrec = nsteps / every;
    if (4 * nrec > 4LL * c->geo.nx * c->geo.ny) return OLB_ERR_ARG;
    DeviceGuard dg(c->device);
    // the records go to the staging buffer (4 per record), read back at the end
    for (long long r = 0; r < nrec; ++r) {
        int rc = olb_step_async(c, every);
        if (rc != OLB_OK) return rc;
        cudaError_t e = enqueue_totals(c, c->stage4 + 4 * r);
        if (e != cudaSuccess) return cuda_status(e);
    }
    int rc = olb_step_async(c, nsteps - (int)(nrec * every));
    if (rc != OLB_OK) return rc;
    cudaError_t e = cudaSuccess;
    if (nrec > 0)
        e = cudaMemcpyAsync(out, c->stage4, (size_t)(4 * nrec) * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    return olb_get_status(c);
}

extern "C" int olb_get_populations(olb_ctx *c, double *f)
{
    if (!c || !f) return OLB_ERR_ARG;
    if (!c->initialized) return OLB_ERR_STATE;
    DeviceGuard dg(c->device);
    const Geo &g = c->geo;
    cudaError_t e;
    if (is_fp64(c)) {
        e = cudaMemcpy2DAsync(f, (size_t)g.nx * sizeof(double), c->f[0], (size_t)g.pitch * sizeof(double),
                              (size_t)g.nx * sizeof(double), (size_t)NK * g.ny, cudaMemcpyDeviceToHost, c->stream);
    } else {
        const size_t bytes = (size_t)NK * g.nx * g.ny * sizeof(double);
        double *tmp = nullptr;
        e = cudaMallocAsync((void **)&tmp, bytes, c->stream);
        if (e == cudaSuccess) e = launch_to_f64((const float *)c->f[0], tmp, g, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(f, tmp, bytes, cudaMemcpyDeviceToHost, c->stream);
        if (tmp) cudaFreeAsync(tmp, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_status(e);
}

extern "C" int olb_set_populations(olb_ctx *c, const double *f)
{
    if (!c || !f) return OLB_ERR_ARG;
    DeviceGuard dg(c->device);
    const Geo &g = c->geo;
    cudaError_t e;
    if (is_fp64(c)) {
        e = cudaMemcpy2DAsync(c->f[0], (size_t)g.pitch * sizeof(double), f, (size_t)g.nx * sizeof(double),
                              (size_t)g.nx * sizeof(double), (size_t)NK * g.ny, cudaMemcpyHostToDevice, c->stream);
    } else {
        const size_t bytes = (size_t)NK * g.nx * g.ny * sizeof(double);
        double *tmp = nullptr;
        e = cudaMallocAsync((void **)&tmp, bytes, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, f, bytes, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = launch_from_f64((float *)c->f[0], tmp, g, c->stream);
        if (tmp) cudaFreeAsync(tmp, c->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) c->initialized = true;
    return cuda_status(e);
}

template <typename real>
static int profile_impl(olb_ctx *c, int nsteps, double *ms, int *launches)
{
    const int nev = 3 * nsteps;
    cudaEvent_t *ev = new cudaEvent_t[2 * nev];
    int made = 0;
    cudaError_t e = cudaSuccess;
    for (; made < 2 * nev && e == cudaSuccess; ++made) e = cudaEventCreate(&ev[made]);
    int q = 0;
    for (int s = 0; s < nsteps && e == cudaSuccess; ++s)
        for (int st = 0; st < 3 && e == cudaSuccess; ++st, ++q) {
            e = cudaEventRecord(ev[2 * q], c->stream);
            if (e == cudaSuccess) e = enqueue_stage<real>(c, st, c->stream);
            if (e == cudaSuccess) e = cudaEventRecord(ev[2 * q + 1], c->stream);
        }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    double acc = 0.0;
    for (int k = 0; k < q && e == cudaSuccess; ++k) {
        float m = 0.f;
        e = cudaEventElapsedTime(&m, ev[2 * k], ev[2 * k + 1]);
        acc += m;
    }
    for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
    delete[] ev;
    if (e != cudaSuccess) return cuda_status(e);
    if (ms) ms[0] = q ? acc / q : 0.0;
    if (launches) launches[0] = q;
    return OLB_OK;
}

extern "C" int olb_profile(olb_ctx *c, int nsteps, double *ms, int *launches)
{
    if (!c || nsteps < 1) return OLB_ERR_ARG;
    if (!c->initialized) return OLB_ERR_STATE;
    DeviceGuard dg(c->device);
    return is_fp64(c) ? profile_impl<double>(c, nsteps, ms, launches) : profile_impl<float>(c, nsteps, ms, launches);
}

static void drop_graphs(olb_ctx *c)
{
    if (c->exec1) cudaGraphExecDestroy(c->exec1);
    if (c->execG) cudaGraphExecDestroy(c->execG);
    c->exec1 = c->execG = nullptr;
    if (c->cap) cudaStreamDestroy(c->cap);
    c->cap = nullptr;
}

extern "C" int olb_set_tile(olb_ctx *c, int tx, int ty, int kp)
{
    if (!c) return OLB_ERR_ARG;
    int k = 0;
    while (k < NUM_TILES && !(TILE_X[k] == tx && TILE_Y[k] == ty && TILE_K[k] == kp)) ++k;
    if (k == NUM_TILES) return OLB_ERR_ARG;
    DeviceGuard dg(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    const int otx = c->tx, oty = c->ty, okp = c->kp;
    c->tx = tx;
    c->ty = ty;
    c->kp = kp;
    e = prepare_tile(c);
    if (e != cudaSuccess) {
        // a shape whose shared memory exceeds the per-CTA limit is refused
        c->tx = otx;
        c->ty = oty;
        c->kp = okp;
        cudaGetLastError();
        return e == cudaErrorInvalidValue ? OLB_ERR_ARG : cuda_status(e);
    }
    drop_graphs(c);
    return OLB_OK;
}

extern "C" int olb_get_tile(olb_ctx *c, int *tx, int *ty, int *kp)
{
    if (!c || !tx || !ty || !kp) return OLB_ERR_ARG;
    *tx = c->tx;
    *ty = c->ty;
    *kp = c->kp;
    return OLB_OK;
}

extern "C" int olb_set_weno_mlp(olb_ctx *c, const float *theta)
{
    if (!c || !theta) return OLB_ERR_ARG;
    if (c->p.weno_mode != OLB_WENO_LEARNED) return OLB_ERR_STATE;
    for (int k = 0; k < 1347; ++k)
        if (!std::isfinite(theta[k])) return OLB_ERR_ARG;
    DeviceGuard dg(c->device);
    cudaError_t e = cudaMemcpyAsync(c->mlp, theta, 1347 * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    c->mlp_set = true;
    return OLB_OK;
}
