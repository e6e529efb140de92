// cbct_residual_static: the data-term residual and its sum of squares with
// the per-block partial sums kept in a fixed, library-owned device array
// instead of a caller-provided workspace, for callers that may not allocate
// device memory at all (see include/cbct.h).
#include "cbct_internal.cuh"

#include <mutex>

namespace cbct {

// Partial sums of the residual projector, one double per block. Every GPU
// that loads the library holds this array until the process exits.
constexpr int kStaticPartials = CBCT_STATIC_MAX_PARTIALS;
static __device__ __align__(256) double g_static_partials[kStaticPartials];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_partials_addr[kMaxDevices] = {};
} // namespace

// Device address of g_static_partials on the current device. The name of the
// array in host code only stands in for the symbol, so the address is looked
// up once per device with that device current.
static cudaError_t static_partials(int dev, double **out)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_partials_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_partials);
        if (e != cudaSuccess) return e;
        g_partials_addr[dev] = static_cast<double *>(p);
    }
    *out = g_partials_addr[dev];
    return cudaSuccess;
}

} // namespace cbct

using namespace cbct;

extern "C" cbct_status cbct_residual_static(const cbct_geometry *geom, const float *d_vol, const float *d_y,
                                            float *d_r, double *d_sumsq, void *stream)
{
    if (!geom) return report_error(CBCT_ERR_INVALID_ARG, "geometry is NULL");
    if (!d_vol || !d_y || !d_r || !d_sumsq) return report_error(CBCT_ERR_INVALID_ARG, "NULL device pointer");
    if ((((uintptr_t)d_vol) | ((uintptr_t)d_y) | ((uintptr_t)d_r)) & 15u)
        return report_error(CBCT_ERR_INVALID_ARG, "arrays must be 16-byte aligned");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return report_error(CBCT_ERR_CUDA, "no CUDA device");
    if (dev != geometry_device(geom))
        return report_error(CBCT_ERR_INVALID_ARG, "geometry belongs to another device");
    if (dev < 0 || dev >= kMaxDevices) return report_error(CBCT_ERR_UNSUPPORTED, "device index above 63");
    const VolGeom *v = geometry_level(geom, 0);
    const DetGeom *d = geometry_detector(geom);
    const int n = fp_partials_count(*v, *d);
    if (n > kStaticPartials)
        return report_error(CBCT_ERR_UNSUPPORTED,
                            "geometry needs more partial sums than the fixed array holds (the forward "
                            "launch's block count must not exceed CBCT_STATIC_MAX_PARTIALS); use cbct_residual");
    double *partials = nullptr;
    cudaError_t e = static_partials(dev, &partials);
    if (e != cudaSuccess) return report_error(CBCT_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    // every block overwrites its own slot, so nothing needs clearing first
    e = launch_forward(*v, *d, d_vol, d_y, d_r, nullptr, partials, 1, s);
    if (e == cudaSuccess) e = launch_sum_partials(partials, n, 1, 1, d_sumsq, s);
    if (e != cudaSuccess) return report_error(CBCT_ERR_CUDA, cudaGetErrorString(e));
    return report_error(CBCT_OK, "");
}
