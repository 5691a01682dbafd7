// olb_static.cu -- olb_step_static: whole RK-3 steps of a small FP64 grid
// without allocating any device memory.
//
// Who needs it: a caller that must not call cudaMalloc / cudaFree when it
// steps the model -- cudaMalloc and cudaFree synchronise the whole device and
// stall every other stream (fatal inside a latency-bound loop shared with
// other work), and some host applications hand all device memory to their
// own pool up front or run the library as a plug-in that may not touch the
// allocator at all.  Such a caller owns the populations; the two
// intermediate RK-3 buffers and the status word live in one file-scope
// device array instead, sized for grids of at most OLB_STATIC_MAX_NODES
// nodes, which every GPU that loads the library holds until the process ends.
//
// The array's name is only a host-side stand-in in host code; its device
// address comes from cudaGetSymbolAddress, taken once per device (under a
// lock, with that device current) on the first call made on that device.
#include <cmath>
#include <mutex>

#include "../../include/olb.h"
#include "olb_internal.cuh"

using namespace olb;

namespace {

constexpr long long kMaxNodes = OLB_STATIC_MAX_NODES;
// f^(1), f^(2) as [25][ny][nx] each, then 256 bytes for the status word.
constexpr long long kScratchDoubles = 2LL * NK * kMaxNodes + 32;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
double *g_scratch_ptr[kMaxDevices] = {};

int scratch_address(int device, double **out)
{
    if (device < 0 || device >= kMaxDevices) return OLB_ERR_CUDA;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return OLB_ERR_CUDA;
        }
        g_scratch_ptr[device] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[device];
    return OLB_OK;
}

int check_params(const olb_params *p)
{
    if (!p) return OLB_ERR_ARG;
    if (p->precision != OLB_FP64 || p->weno_mode != OLB_WENO_JS) return OLB_ERR_ARG;
    if (p->nx < 1 || p->ny < 1 || (long long)p->nx * p->ny > kMaxNodes) return OLB_ERR_ARG;
    if (p->side_y != OLB_SIDE_PERIODIC) return OLB_ERR_ARG;
    if (p->side_x != OLB_SIDE_PERIODIC && p->side_x != OLB_SIDE_DIFFUSE) return OLB_ERR_ARG;
    if (p->side_x == OLB_SIDE_DIFFUSE) {
        if (p->nx < 3) return OLB_ERR_ARG;
        for (int s = 0; s < 2; ++s)
            if (!(p->Tw[s] > 0.0) || !std::isfinite(p->Tw[s]) || !std::isfinite(p->uw[s])) return OLB_ERR_ARG;
    }
    if (!(p->ds > 0.0) || !(p->dt > 0.0) || !(p->tau > 0.0) || !std::isfinite(p->ds) || !std::isfinite(p->dt) ||
        !std::isfinite(p->tau))
        return OLB_ERR_ARG;
    if (!(p->sigma >= 0.0) || !(p->b >= 0.0) || !std::isfinite(p->a) || !std::isfinite(p->b) ||
        !std::isfinite(p->sigma))
        return OLB_ERR_ARG;
    const double pmax = std::sqrt(5.0 + std::sqrt(10.0));
    if (!(pmax * p->dt / p->ds < 1.0) || p->dt > 2.5 * p->tau) return OLB_ERR_CFL;
    return OLB_OK;
}

}  // namespace

extern "C" int olb_step_static(const olb_params *p, void *stream, double *f, int nsteps)
{
    int v = check_params(p);
    if (v != OLB_OK) return v;
    if (!f || nsteps < 0) return OLB_ERR_ARG;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return OLB_ERR_CUDA;
    }
    double *scratch = nullptr;
    v = scratch_address(device, &scratch);
    if (v != OLB_OK) return v;

    Geo g{};
    g.nx = p->nx;
    g.ny = p->ny;
    g.pitch = p->nx;  // the caller's [25][ny][nx] layout, no padding
    g.plane = (long long)g.nx * g.ny;
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
    Tab<double> tab;
    fill_tab<double>(&tab, h, p->Tw, p->uw);

    double *f1 = scratch;
    double *f2 = scratch + (long long)NK * g.plane;
    int *status = reinterpret_cast<int *>(scratch + 2LL * NK * kMaxNodes);
    cudaStream_t s = (cudaStream_t)stream;

    // shape, as olb_create picks it for FP64: 8 x 8 nodes with 4 velocity
    // lanes, or 7 x 8 nodes with 8 lanes when that lowers the most nodes one
    // SM advances (grids here have at most 256 tiles, a wave or two)
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        return OLB_ERR_CUDA;
    }
    auto most_nodes = [&](int tx_, int ty_) {
        const long long tiles = (long long)((g.nx + tx_ - 1) / tx_) * ((g.ny + ty_ - 1) / ty_);
        return (tiles + sms - 1) / sms * tx_ * ty_;
    };
    const bool narrow = most_nodes(7, 8) < most_nodes(8, 8);
    const int tx = narrow ? 7 : 8, ty = 8, kp = narrow ? 8 : 4;
    cudaError_t e = prepare_fused((double *)nullptr, tx, ty, kp, false);
    // the scratch keeps the previous call's contents: the status word must start at zero
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), s);
    const double dt = p->dt;
    const StageCoef coef[3] = {{0.0, 1.0, dt}, {0.75, 0.25, 0.25 * dt}, {1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0 * dt}};
    const double *src[3] = {f, f1, f2};
    double *dst[3] = {f1, f2, f};
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k)
        for (int st = 0; st < 3 && e == cudaSuccess; ++st)
            e = launch_fused(src[st], f, dst[st], status, g, tab, coef[st], tx, ty, kp, nullptr, nullptr, nullptr, s);
    int hstatus = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return OLB_ERR_CUDA;
    }
    return hstatus ? OLB_ERR_DIVERGED : OLB_OK;
}
