// pm_mse_loss_noalloc: the density-MSE loss and its adjoint seed (the work
// of pm_mse_loss with cloud-in-cell assignment) for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code whose device memory is all
// reserved up front by another allocator (a framework's caching pool, a
// serving process's fixed arena), and latency-critical loops that cannot
// take the implicit device-wide synchronisation of cudaMalloc / cudaFree.
// For them this entry point needs no context and allocates nothing: its one
// piece of scratch (the painted density mesh and the per-run loss sums)
// lives in a file-scope __device__ array of fixed size, which every GPU that
// loads the library keeps until the process exits.

#include <mutex>

#include "../../include/pmgb.h"
#include "pm_internal.h"

namespace {

// Largest mesh the scratch holds: n_batch * n_m^3 cells in total (128^3 for
// one run), plus room for up to kMaxRuns double-precision loss sums.
constexpr int64_t kMaxCells = int64_t(1) << 21;
constexpr int kMaxRuns = 64;
constexpr int64_t kScratchFloats = kMaxCells + 2 * kMaxRuns;

static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, never a device address).
// The cached address belongs to the device's current context: after a
// cudaDeviceReset in this process it is stale, so callers must not reset a
// device and then call this entry point again.
cudaError_t scratch_address(float **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<float *>(ptr);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

__global__ void k_loss_out(const double *acc, double *loss, int nb, double inv_cells) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) loss[b] = acc[b] * inv_cells;
}

}  // namespace

extern "C" int pm_mse_loss_noalloc(int32_t n_p, int32_t n_m, int32_t n_batch, double box, const float *s,
                                   const float *target, double *loss, float *dlds, void *stream) {
    using namespace pmgb;
    // the same size rules as pm_create (n_p, n_m even and at most 4096), checked
    // before n_p^3 is formed so that it cannot overflow
    if (n_p < 2 || n_p % 2 || n_p > 4096 || n_m < 4 || n_m % 2 || n_m > 4096 || n_batch < 1 || !(box > 0))
        return PM_EINVAL;
    if (!s || !target || !loss) return PM_EINVAL;
    if ((uintptr_t)s % 4 || (uintptr_t)target % 4 || (uintptr_t)loss % 8 || (dlds && (uintptr_t)dlds % 4))
        return PM_EINVAL;
    const int64_t cells = (int64_t)n_m * n_m * n_m;
    if (n_batch > kMaxRuns || cells * n_batch > kMaxCells) return PM_ERANGE;
    if ((int64_t)n_p * n_p * n_p > (int64_t(1) << 31)) return PM_ERANGE;

    float *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return PM_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *mesh = scratch;
    double *acc = reinterpret_cast<double *>(scratch + kMaxCells);

    // Everything the previous call left behind is cleared here.
    if (cudaMemsetAsync(mesh, 0, sizeof(float) * cells * n_batch, st) != cudaSuccess) return PM_ECUDA;
    if (cudaMemsetAsync(acc, 0, sizeof(double) * n_batch, st) != cudaSuccess) return PM_ECUDA;

    Geom g{};
    g.np = n_p;
    g.nm = n_m;
    g.nb = n_batch;
    g.npart = (int64_t)n_p * n_p * n_p;
    g.ratio = (n_m % n_p == 0) ? n_m / n_p : 0;
    g.inv_np = 1.0f / n_p;
    g.inv_h = (float)(n_m / box);
    g.alpha = (float)((double)n_m * n_m * n_m / ((double)n_p * n_p * n_p));
    const MeshRef ref{mesh, 0, cells, n_m};

    PaintArgs pa{};
    pa.g = g;
    pa.s = const_cast<float *>(s);
    pa.mesh = ref;
    if (launch_paint(PAINT_DENSITY, pa, st) != cudaSuccess) return PM_ECUDA;
    if (launch_mse(ref, target, n_m, n_batch, acc, st) != cudaSuccess) return PM_ECUDA;
    if (dlds) {
        ReadArgs ra{};
        ra.g = g;
        ra.s = const_cast<float *>(s);
        ra.mesh = ref;
        ra.f = dlds;
        if (launch_read(READ_GRAD, ra, st) != cudaSuccess) return PM_ECUDA;
    }
    k_loss_out<<<1, kMaxRuns, 0, st>>>(acc, loss, n_batch, 1.0 / (double)cells);
    if (cudaGetLastError() != cudaSuccess) return PM_ECUDA;
    return PM_OK;
}
