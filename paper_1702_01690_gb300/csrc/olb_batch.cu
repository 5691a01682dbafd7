// olb_batch.cu -- many independent runs (uneven grids, own parameters) in one
// launch per RK-3 stage (one CTA per tile of every run), replayed from CUDA
// graphs, with an autotuner that times the compiled stage shapes.
//
// Device layout: the populations of all runs share three buffers (f^n, f^(1),
// f^(2)); run r occupies 25 x ny_r x pitch_r values at offset off_r of each.
// A descriptor per run (geometry, velocity and wall tables, offset, tiles per
// row) and the prefix sum of tiles per run drive the stage kernel
// (k_fused_batch in olb_fused.cuh); each run has its own status word.  Where
// the tile shape suits TMA, each run also has a tensor map per buffer
// ([3][count], in device memory): tiles inside a run are staged by one copy.
#include <cmath>
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/olb.h"
#include "olb_internal.cuh"

using namespace olb;

namespace {
constexpr int BATCH_GRAPH_STEPS = 16;

// Process-wide autotune results: batch signature -> shape index.
std::mutex g_tune_lock;
std::map<std::string, int> g_tune_cache;
}  // namespace

struct olb_batch {
    int count = 0;
    int precision = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<olb_params> p;
    std::vector<Geo> geo;
    std::vector<long long> off;          // element offset of each run
    std::vector<Tab<double>> tab64;
    std::vector<Tab<float>> tab32;
    size_t elt = 8;
    long long total_elems = 0;           // per population buffer
    void *f[3] = {nullptr, nullptr, nullptr};
    int *status = nullptr;               // [count]
    void *runs = nullptr;                // BatchRun<real>[count]
    int *tile_start = nullptr;           // [count + 1]
    double *stage4 = nullptr;            // FP64 [4][max nodes] staging
    void *fields = nullptr;              // stage fields of every run (moments pre-pass)
    std::vector<long long> foff;         // byte offset of each run's fields
    long long *node_start = nullptr;     // [count + 1] prefix sum of the runs' node counts
    long long total_nodes = 0;
    long long max_nodes = 0;
    TmaMap *tmaps = nullptr;             // [3][count] tensor maps (runs x buffers) for the current shape
    bool tma_ok = false;                 // every map encoded
    int tx = 16, ty = 8, kp = 2, total_tiles = 0;
    std::vector<char> init;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec1 = nullptr, execG = nullptr;
};

static bool b_fp64(const olb_batch *b) { return b->precision == OLB_FP64; }

struct BDevice {
    int prev;
    explicit BDevice(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~BDevice() { cudaSetDevice(prev); }
};

static void batch_drop_graphs(olb_batch *b)
{
    if (b->exec1) cudaGraphExecDestroy(b->exec1);
    if (b->execG) cudaGraphExecDestroy(b->execG);
    b->exec1 = b->execG = nullptr;
    if (b->cap) cudaStreamDestroy(b->cap);
    b->cap = nullptr;
}

// Descriptors and tile prefix for the current shape (synchronous upload).
static cudaError_t batch_upload(olb_batch *b)
{
    const size_t rb = b_fp64(b) ? batch_run_bytes((double *)nullptr) : batch_run_bytes((float *)nullptr);
    std::vector<char> host(rb * b->count);
    std::vector<int> start(b->count + 1);
    int acc = 0;
    for (int r = 0; r < b->count; ++r) {
        const Geo &g = b->geo[r];
        const int ntx = (g.nx + b->tx - 1) / b->tx, nty = (g.ny + b->ty - 1) / b->ty;
        start[r] = acc;
        acc += ntx * nty;
        if (b_fp64(b))
            batch_run_fill((double *)nullptr, host.data() + rb * r, g, b->tab64[r], b->off[r], b->foff[r], ntx);
        else
            batch_run_fill((float *)nullptr, host.data() + rb * r, g, b->tab32[r], b->off[r], b->foff[r], ntx);
    }
    start[b->count] = acc;
    b->total_tiles = acc;
    // tensor maps of every run in every buffer; if one cannot be encoded
    // (shape unsuited to TMA, or no driver entry point) no run uses TMA
    std::vector<TmaMap> maps((size_t)3 * b->count);
    b->tma_ok = true;
    for (int k = 0; k < 3 && b->tma_ok; ++k)
        for (int r = 0; r < b->count && b->tma_ok; ++r)
            b->tma_ok = tma_encode(&maps[(size_t)k * b->count + r], (const char *)b->f[k] + b->off[r] * b->elt,
                                   b_fp64(b), b->geo[r], b->tx, b->ty);
    cudaError_t e = cudaMemcpyAsync(b->runs, host.data(), host.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->tile_start, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && b->tma_ok)
        e = cudaMemcpyAsync(b->tmaps, maps.data(), maps.size() * sizeof(TmaMap), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e;
}

static cudaError_t batch_prepare(olb_batch *b)
{
    return b_fp64(b) ? prepare_fused((double *)nullptr, b->tx, b->ty, b->kp, false)
                     : prepare_fused((float *)nullptr, b->tx, b->ty, b->kp, false);
}

// The velocity tables (identical in every run's Tab; only the wall entries
// differ, and the kernel reads those from each run's descriptor).
static const Tab<double> &batch_tab(const olb_batch *b, double *) { return b->tab64[0]; }
static const Tab<float> &batch_tab(const olb_batch *b, float *) { return b->tab32[0]; }

template <typename real>
static cudaError_t batch_stage(olb_batch *b, int st, cudaStream_t s)
{
    real *f0 = (real *)b->f[0], *f1 = (real *)b->f[1], *f2 = (real *)b->f[2];
    const real *src[3] = {f0, f1, f2};
    real *dst[3] = {f1, f2, f0};
    // the dt-proportional coefficient is multiplied by each run's own dt
    const StageCoef coef[3] = {{0.0, 1.0, 1.0}, {0.75, 0.25, 0.25}, {1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0}};
    // src[st] is buffer st: its maps are row st of tmaps
    const TmaMap *maps = b->tma_ok ? b->tmaps + (size_t)st * b->count : nullptr;
    return launch_fused_batch(src[st], f0, dst[st], b->status, b->runs, b->tile_start, b->count, b->total_tiles,
                              batch_tab(b, (real *)nullptr), coef[st], b->tx, b->ty, b->kp, b->fields, b->node_start,
                              b->total_nodes, maps, s);
}

static cudaError_t batch_enqueue_steps(olb_batch *b, int n, cudaStream_t s)
{
    for (int k = 0; k < n; ++k)
        for (int st = 0; st < 3; ++st) {
            cudaError_t e = b_fp64(b) ? batch_stage<double>(b, st, s) : batch_stage<float>(b, st, s);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

static cudaError_t batch_graph(olb_batch *b, int nsteps, cudaGraphExec_t *exec)
{
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t e2 = batch_enqueue_steps(b, nsteps, b->cap);
    e = cudaStreamEndCapture(b->cap, &graph);
    if (e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return e2;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    return e;
}

static void batch_free(olb_batch *b)
{
    for (int k = 0; k < 3; ++k) cudaFree(b->f[k]);
    cudaFree(b->status);
    cudaFree(b->runs);
    cudaFree(b->tile_start);
    cudaFree(b->stage4);
    cudaFree(b->fields);
    cudaFree(b->node_start);
    cudaFree(b->tmaps);
}

static bool batch_shape_index(int tx, int ty, int kp, int *k)
{
    for (int q = 0; q < NUM_TILES; ++q)
        if (TILE_X[q] == tx && TILE_Y[q] == ty && TILE_K[q] == kp) {
            *k = q;
            return true;
        }
    return false;
}

extern "C" int olb_batch_create(const olb_params *runs, int count, void *stream, olb_batch **out)
{
    if (!out) return OLB_ERR_ARG;
    *out = nullptr;
    if (!runs || count < 1) return OLB_ERR_ARG;
    for (int r = 0; r < count; ++r) {
        const int v = validate_params(&runs[r]);
        if (v != OLB_OK) return v;
        if (runs[r].precision != runs[0].precision) return OLB_ERR_ARG;
        if (runs[r].weno_mode != OLB_WENO_JS) return OLB_ERR_ARG;
    }
    olb_batch *b = new (std::nothrow) olb_batch();
    if (!b) return OLB_ERR_NOMEM;
    b->count = count;
    b->precision = runs[0].precision;
    b->stream = (cudaStream_t)stream;
    b->elt = b_fp64(b) ? sizeof(double) : sizeof(float);
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return OLB_ERR_CUDA;
    }
    HostTables h;
    host_tables(&h);
    b->p.assign(runs, runs + count);
    b->geo.resize(count);
    b->off.resize(count);
    b->tab64.resize(count);
    b->tab32.resize(count);
    b->init.assign(count, 0);
    b->foff.resize(count);
    long long acc = 0, facc = 0;
    std::vector<long long> nstart(count + 1, 0);
    for (int r = 0; r < count; ++r) {
        const olb_params *p = &runs[r];
        Geo &g = b->geo[r];
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
        fill_tab<double>(&b->tab64[r], h, p->Tw, p->uw);
        fill_tab<float>(&b->tab32[r], h, p->Tw, p->uw);
        b->off[r] = acc;
        acc += ((long long)(b_fp64(b) ? pop_planes<double>() : pop_planes<float>()) * g.plane + 63) / 64 * 64;
        b->foff[r] = facc;
        facc += ((long long)fields_bytes(g) + 255) / 256 * 256;
        nstart[r + 1] = nstart[r] + (long long)g.nx * g.ny;
        b->max_nodes = std::max(b->max_nodes, (long long)g.nx * g.ny);
    }
    b->total_elems = acc;
    // default shape: as for a single grid of the batch's total size
    const bool fp64 = b_fp64(b);
    b->tx = 16;
    b->ty = 8;
    b->kp = fp64 ? 2 : 1;
    if (!fp64) {
        b->tx = 32;
        b->ty = 16;
    }
    const size_t rb = fp64 ? batch_run_bytes((double *)nullptr) : batch_run_bytes((float *)nullptr);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaMalloc(&b->f[k], (size_t)acc * b->elt);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->status, (size_t)count * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->runs, rb * count);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->tile_start, (size_t)(count + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->stage4, (size_t)4 * b->max_nodes * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b->fields, (size_t)facc);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->node_start, (size_t)(count + 1) * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->tmaps, (size_t)3 * count * sizeof(TmaMap));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->node_start, nstart.data(), (size_t)(count + 1) * sizeof(long long),
                            cudaMemcpyHostToDevice, b->stream);
    b->total_nodes = nstart[count];
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaMemsetAsync(b->f[k], 0, (size_t)acc * b->elt, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->status, 0, (size_t)count * sizeof(int), b->stream);
    if (e == cudaSuccess) e = batch_prepare(b);
    if (e == cudaSuccess) e = batch_upload(b);
    if (e != cudaSuccess) {
        const int code = cuda_status(e);
        cudaGetLastError();
        batch_free(b);
        delete b;
        return code;
    }
    *out = b;
    return OLB_OK;
}

extern "C" void olb_batch_destroy(olb_batch *b)
{
    if (!b) return;
    BDevice dg(b->device);
    cudaStreamSynchronize(b->stream);
    batch_drop_graphs(b);
    batch_free(b);
    cudaGetLastError();
    delete b;
}

static Geo run_geo_at(const olb_batch *b, int r) { return b->geo[r]; }

extern "C" int olb_batch_init_fields(olb_batch *b, int run, const double *n, const double *ux, const double *uy,
                                     const double *T)
{
    if (!b || run < 0 || run >= b->count || !n || !ux || !uy || !T) return OLB_ERR_ARG;
    const Geo g = run_geo_at(b, run);
    const size_t N = (size_t)g.nx * g.ny;
    if (!fields_admissible(n, ux, uy, T, N, b->p[run].b)) return OLB_ERR_ARG;
    BDevice dg(b->device);
    const double *src[4] = {n, ux, uy, T};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(b->stage4 + k * N, src[k], N * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = b_fp64(b) ? launch_init((double *)b->f[0] + b->off[run], b->stage4, b->stage4 + N, b->stage4 + 2 * N,
                                    b->stage4 + 3 * N, g, b->tab64[run], b->stream)
                      : launch_init((float *)b->f[0] + b->off[run], b->stage4, b->stage4 + N, b->stage4 + 2 * N,
                                    b->stage4 + 3 * N, g, b->tab64[run], b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->status + run, 0, sizeof(int), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_status(e);
    b->init[run] = 1;
    return OLB_OK;
}

extern "C" int olb_batch_step_async(olb_batch *b, int nsteps)
{
    if (!b || nsteps < 0) return OLB_ERR_ARG;
    for (int r = 0; r < b->count; ++r)
        if (!b->init[r]) return OLB_ERR_STATE;
    if (nsteps == 0) return OLB_OK;
    BDevice dg(b->device);
    cudaError_t e = cudaSuccess;
    if (!b->cap) {
        e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = batch_graph(b, 1, &b->exec1);
        if (e == cudaSuccess) e = batch_graph(b, BATCH_GRAPH_STEPS, &b->execG);
        if (e != cudaSuccess) {
            cudaGetLastError();
            batch_drop_graphs(b);
            return cuda_status(e);
        }
    }
    int k = 0;
    for (; k + BATCH_GRAPH_STEPS <= nsteps && e == cudaSuccess; k += BATCH_GRAPH_STEPS)
        e = cudaGraphLaunch(b->execG, b->stream);
    for (; k < nsteps && e == cudaSuccess; ++k) e = cudaGraphLaunch(b->exec1, b->stream);
    return cuda_status(e);
}

extern "C" int olb_batch_get_status(olb_batch *b, int *per_run)
{
    if (!b) return OLB_ERR_ARG;
    BDevice dg(b->device);
    std::vector<int> h(b->count, 0);
    cudaError_t e = cudaMemcpyAsync(h.data(), b->status, h.size() * sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_status(e);
    int any = OLB_OK;
    for (int r = 0; r < b->count; ++r) {
        const int code = h[r] ? OLB_ERR_DIVERGED : OLB_OK;
        if (per_run) per_run[r] = code;
        if (code != OLB_OK) any = code;
    }
    return any;
}

extern "C" int olb_batch_step(olb_batch *b, int nsteps)
{
    const int r = olb_batch_step_async(b, nsteps);
    if (r != OLB_OK) return r;
    return olb_batch_get_status(b, nullptr);
}

extern "C" int olb_batch_moments(olb_batch *b, int run, double *n, double *ux, double *uy, double *T)
{
    if (!b || run < 0 || run >= b->count) return OLB_ERR_ARG;
    if (!b->init[run]) return OLB_ERR_STATE;
    BDevice dg(b->device);
    const Geo g = run_geo_at(b, run);
    const size_t N = (size_t)g.nx * g.ny;
    double *dev[4] = {b->stage4, b->stage4 + N, b->stage4 + 2 * N, b->stage4 + 3 * N};
    double *host[4] = {n, ux, uy, T};
    cudaError_t e = b_fp64(b) ? launch_moments_out((const double *)b->f[0] + b->off[run], host[0] ? dev[0] : nullptr,
                                                   host[1] ? dev[1] : nullptr, host[2] ? dev[2] : nullptr,
                                                   host[3] ? dev[3] : nullptr, g, b->tab64[run], b->stream)
                              : launch_moments_out((const float *)b->f[0] + b->off[run], host[0] ? dev[0] : nullptr,
                                                   host[1] ? dev[1] : nullptr, host[2] ? dev[2] : nullptr,
                                                   host[3] ? dev[3] : nullptr, g, b->tab64[run], b->stream);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        if (host[k]) e = cudaMemcpyAsync(host[k], dev[k], N * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return cuda_status(e);
}

extern "C" int olb_batch_get_populations(olb_batch *b, int run, double *f)
{
    if (!b || run < 0 || run >= b->count || !f) return OLB_ERR_ARG;
    if (!b->init[run]) return OLB_ERR_STATE;
    BDevice dg(b->device);
    const Geo g = run_geo_at(b, run);
    cudaError_t e;
    if (b_fp64(b)) {
        e = cudaMemcpy2DAsync(f, (size_t)g.nx * sizeof(double), (const double *)b->f[0] + b->off[run],
                              (size_t)g.pitch * sizeof(double), (size_t)g.nx * sizeof(double), (size_t)NK * g.ny,
                              cudaMemcpyDeviceToHost, b->stream);
    } else {
        const size_t bytes = (size_t)NK * g.nx * g.ny * sizeof(double);
        double *tmp = nullptr;
        e = cudaMallocAsync((void **)&tmp, bytes, b->stream);
        if (e == cudaSuccess) e = launch_to_f64((const float *)b->f[0] + b->off[run], tmp, g, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(f, tmp, bytes, cudaMemcpyDeviceToHost, b->stream);
        if (tmp) cudaFreeAsync(tmp, b->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return cuda_status(e);
}

extern "C" int olb_batch_set_tile(olb_batch *b, int tx, int ty, int kp)
{
    if (!b) return OLB_ERR_ARG;
    int k = 0;
    if (!batch_shape_index(tx, ty, kp, &k)) return OLB_ERR_ARG;
    BDevice dg(b->device);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_status(e);
    const int otx = b->tx, oty = b->ty, okp = b->kp;
    b->tx = tx;
    b->ty = ty;
    b->kp = kp;
    e = batch_prepare(b);
    if (e == cudaSuccess) e = batch_upload(b);
    if (e != cudaSuccess) {
        b->tx = otx;
        b->ty = oty;
        b->kp = okp;
        cudaGetLastError();
        batch_upload(b);
        return e == cudaErrorInvalidValue ? OLB_ERR_ARG : cuda_status(e);
    }
    batch_drop_graphs(b);
    return OLB_OK;
}

extern "C" int olb_batch_get_tile(olb_batch *b, int *tx, int *ty, int *kp)
{
    if (!b || !tx || !ty || !kp) return OLB_ERR_ARG;
    *tx = b->tx;
    *ty = b->ty;
    *kp = b->kp;
    return OLB_OK;
}

// Mean device ms per stage launch over nsteps steps, launched individually
// between events (the populations advance).
static int batch_time(olb_batch *b, int nsteps, double *ms)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
    if (e == cudaSuccess) e = batch_enqueue_steps(b, nsteps, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_status(e);
    *ms = t / (3.0 * nsteps);
    return OLB_OK;
}

extern "C" int olb_batch_profile(olb_batch *b, int nsteps, double *ms)
{
    if (!b || nsteps < 1 || !ms) return OLB_ERR_ARG;
    for (int r = 0; r < b->count; ++r)
        if (!b->init[r]) return OLB_ERR_STATE;
    BDevice dg(b->device);
    return batch_time(b, nsteps, ms);
}

extern "C" int olb_batch_autotune(olb_batch *b, int nsteps, int *tx, int *ty, int *kp)
{
    if (!b || nsteps < 1) return OLB_ERR_ARG;
    for (int r = 0; r < b->count; ++r)
        if (!b->init[r]) return OLB_ERR_STATE;
    BDevice dg(b->device);
    std::string sig = std::to_string(b->precision) + ":" + std::to_string(b->device);
    for (int r = 0; r < b->count; ++r)
        sig += ";" + std::to_string(b->geo[r].nx) + "x" + std::to_string(b->geo[r].ny) + (b->geo[r].walls ? "w" : "p") +
               std::to_string(b->geo[r].wall_lo * 8 + b->geo[r].wall_hi * 4 + b->geo[r].spec_lo * 2 + b->geo[r].spec_hi) +
               (b->geo[r].spec_y ? "s" : "");
    int best = -1;
    {
        std::lock_guard<std::mutex> guard(g_tune_lock);
        auto it = g_tune_cache.find(sig);
        if (it != g_tune_cache.end()) best = it->second;
    }
    if (best < 0) {
        // time every shape on a copy of the state, then put the state back
        const size_t bytes = (size_t)b->total_elems * b->elt;
        void *backup = nullptr;
        cudaError_t e = cudaMallocAsync(&backup, bytes, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(backup, b->f[0], bytes, cudaMemcpyDeviceToDevice, b->stream);
        if (e != cudaSuccess) return cuda_status(e);
        double best_ms = 1e300;
        const int otx = b->tx, oty = b->ty, okp = b->kp;
        for (int q = 0; q < NUM_TILES; ++q) {
            b->tx = TILE_X[q];
            b->ty = TILE_Y[q];
            b->kp = TILE_K[q];
            if (batch_prepare(b) != cudaSuccess) {
                cudaGetLastError();
                continue;  // shape does not fit this precision
            }
            double ms = 0.0;
            int rc = batch_upload(b) == cudaSuccess ? OLB_OK : OLB_ERR_CUDA;
            if (rc == OLB_OK) rc = batch_time(b, 1, &ms);  // warm-up
            if (rc == OLB_OK) rc = batch_time(b, nsteps, &ms);
            cudaMemcpyAsync(b->f[0], backup, bytes, cudaMemcpyDeviceToDevice, b->stream);
            if (rc == OLB_OK && ms < best_ms) {
                best_ms = ms;
                best = q;
            }
        }
        cudaMemsetAsync(b->status, 0, (size_t)b->count * sizeof(int), b->stream);
        cudaFreeAsync(backup, b->stream);
        cudaStreamSynchronize(b->stream);
        b->tx = otx;
        b->ty = oty;
        b->kp = okp;
        if (best < 0) return OLB_ERR_CUDA;
        std::lock_guard<std::mutex> guard(g_tune_lock);
        g_tune_cache[sig] = best;
    }
    const int rc = olb_batch_set_tile(b, TILE_X[best], TILE_Y[best], TILE_K[best]);
    if (rc != OLB_OK) return rc;
    if (tx) *tx = b->tx;
    if (ty) *ty = b->ty;
    if (kp) *kp = b->kp;
    return OLB_OK;
}
