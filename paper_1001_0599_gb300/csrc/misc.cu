// Small kernels of the reconstruction driver: FP64 finalisation of block
// partials, the power-iteration update, multigrid prolongation (Sec. II.C.3)
// and fills.
#include "cbct_internal.cuh"

namespace cbct {

// out[i] = sum over b of partials[b*stride + i], i < k, in a fixed order, FP64.
// If scale_out is set, out[i] *= scale.
__global__ void sum_partials_kernel(const double *__restrict__ partials, int n, int stride, int k,
                                    double *__restrict__ out, double scale)
{
    __shared__ double red[32];
    for (int i = 0; i < k; i++) {
        double acc = 0.0;
        for (int b = threadIdx.x; b < n; b += blockDim.x) acc += partials[(size_t)b * stride + i];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
            out[i] = s * scale;
        }
        __syncthreads();
    }
}

cudaError_t launch_sum_partials(const double *partials, int n, int stride, int k, double *out,
                                cudaStream_t s)
{
    launch_begin(K_REDUCE, s);
    sum_partials_kernel<<<1, 1024, 0, s>>>(partials, n, stride, k, out, 1.0);
    launch_end(K_REDUCE, s);
    return cudaGetLastError();
}

// data term E2 = sum r^2 / m into st->e2
__global__ void e2_kernel(const double *__restrict__ partials, int n, double inv_m, DevState *st)
{
    __shared__ double red[32];
    double acc = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) acc += partials[b];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
        st->e2 = s * inv_m;
    }
}

cudaError_t launch_e2(const double *partials, int n, double inv_m, DevState *st, cudaStream_t s)
{
    launch_begin(K_REDUCE, s);
    e2_kernel<<<1, 1024, 0, s>>>(partials, n, inv_m, st);
    launch_end(K_REDUCE, s);
    return cudaGetLastError();
}

// Power iteration on kappa P^T P (v = w / |w| kept implicit): from the
// partials of |w|^2, L = |w| / |v|; the next forward projection reads
// 1/|w| as its input scale.
__global__ void power_update_kernel(DevState *st, const double *__restrict__ partials, int n, int last,
                                    double *d_L_out)
{
    __shared__ double red[32];
    double acc = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) acc += partials[b];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double w2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) w2 += red[w];
        const double L = sqrt(w2 / st->vnorm2);
        st->lipschitz = L;
        st->inv_wnorm = w2 > 0.0 ? 1.0 / sqrt(w2) : 0.0;
        st->vnorm2 = 1.0;
        if (last) {
            st->tau = L > 0.0 ? 1.0 / L : 0.0;
            if (d_L_out) *d_L_out = L;
        }
    }
}

cudaError_t launch_power_update(DevState *st, const double *partials, int n, double, int, int last,
                                double *d_L_out, cudaStream_t s)
{
    launch_begin(K_REDUCE, s);
    power_update_kernel<<<1, 1024, 0, s>>>(st, partials, n, last, d_L_out);
    launch_end(K_REDUCE, s);
    return cudaGetLastError();
}

__global__ void power_init_kernel(DevState *st, double nvox)
{
    if (threadIdx.x == 0) {
        if (nvox > 0.0) st->vnorm2 = nvox;   // start from ones; otherwise vnorm2 was set by a norm pass
        st->inv_wnorm = 1.0;
    }
}

// per-block sums of x^2 (compensated FP32 in the block, FP64 out)
__global__ void __launch_bounds__(256) sumsq_kernel(const float *__restrict__ x, size_t n,
                                                    double *__restrict__ partials)
{
    __shared__ double red[32];
    float acc = 0.f;
    DF v[1] = {df_zero()};
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    int k = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float t = __ldg(x + i);
        acc += t * t;
        if (++k == 16) {
            v[0] = df_add(v[0], acc);
            acc = 0.f;
            k = 0;
        }
    }
    v[0] = df_add(v[0], acc);
    double tot[1];
    block_sum_df<1>(v, red, tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot[0];
}

cudaError_t launch_sumsq(const float *x, size_t n, double *partials, int blocks, double *out, cudaStream_t s)
{
    launch_begin(K_REDUCE, s);
    sumsq_kernel<<<blocks, 256, 0, s>>>(x, n, partials);
    note_extra_launch();
    sum_partials_kernel<<<1, 1024, 0, s>>>(partials, blocks, 1, 1, out, 1.0);
    launch_end(K_REDUCE, s);
    return cudaGetLastError();
}

cudaError_t launch_power_init(DevState *st, double nvox, cudaStream_t s)
{
    launch_begin(K_MISC, s);
    power_init_kernel<<<1, 32, 0, s>>>(st, nvox);
    launch_end(K_MISC, s);
    return cudaGetLastError();
}

// st->tau = given (> 0) or the power-iteration result; st->scale = tau kappa;
// record the level's step into the stats.
__global__ void set_tau_kernel(DevState *st, double tau_given, double kappa, cbct_recon_stats *rs,
                               int level)
{
    if (threadIdx.x == 0) {
        const bool given = tau_given > 0.0;
        if (given) {
            st->tau = tau_given;
            st->lipschitz = 0.0;
        }
        st->scale = st->tau * kappa;
        if (rs && level >= 0 && level < CBCT_MAX_LEVELS) {
            rs->tau[level] = st->tau;
            rs->lipschitz[level] = given ? 0.0 : st->lipschitz;
        }
    }
}

cudaError_t launch_set_tau(DevState *st, double tau_given, double kappa, cbct_recon_stats *rs, int level,
                           cudaStream_t s)
{
    launch_begin(K_MISC, s);
    set_tau_kernel<<<1, 32, 0, s>>>(st, tau_given, kappa, rs, level);
    launch_end(K_MISC, s);
    return cudaGetLastError();
}

__global__ void fill_kernel(float *__restrict__ p, size_t n, float value)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = value;
}

cudaError_t launch_fill(float *p, size_t n, float value, cudaStream_t s)
{
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    launch_begin(K_FILL, s);
    fill_kernel<<<blocks, 256, 0, s>>>(p, n, value);
    launch_end(K_FILL, s);
    return cudaGetLastError();
}

// Cell-centred trilinear prolongation, clamp to edge: fine index i sits at
// coarse continuous index (i + 0.5)/2 - 0.5.
__device__ __forceinline__ void lin_coord(int nc, int i, int &i0, int &i1, float &w)
{
    float I = 0.5f * ((float)i + 0.5f) - 0.5f;
    I = fminf(fmaxf(I, 0.f), (float)(nc - 1));
    int k = (int)floorf(I);
    if (k > nc - 2) k = nc - 2;
    if (k < 0) k = 0;
    i0 = k;
    i1 = min(k + 1, nc - 1);
    w = (nc == 1) ? 0.f : I - (float)k;
}

__global__ void prolong_kernel(int ncx, int ncy, int ncz, const float *__restrict__ c, float *__restrict__ f)
{
    const int nz = 2 * ncz, ny = 2 * ncy, nx = 2 * ncx;
    const size_t n = (size_t)nx * ny * nz;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int z = (int)(i % nz);
        const size_t t = i / nz;
        const int y = (int)(t % ny), x = (int)(t / ny);
        int x0, x1, y0, y1, z0, z1;
        float wx, wy, wz;
        lin_coord(ncx, x, x0, x1, wx);
        lin_coord(ncy, y, y0, y1, wy);
        lin_coord(ncz, z, z0, z1, wz);
        auto C = [&](int a, int b, int cc) { return __ldg(c + ((size_t)a * ncy + b) * ncz + cc); };
        const float v00 = (1.f - wz) * C(x0, y0, z0) + wz * C(x0, y0, z1);
        const float v01 = (1.f - wz) * C(x0, y1, z0) + wz * C(x0, y1, z1);
        const float v10 = (1.f - wz) * C(x1, y0, z0) + wz * C(x1, y0, z1);
        const float v11 = (1.f - wz) * C(x1, y1, z0) + wz * C(x1, y1, z1);
        f[i] = (1.f - wx) * ((1.f - wy) * v00 + wy * v01) + wx * ((1.f - wy) * v10 + wy * v11);
    }
}

cudaError_t launch_prolong(int ncx, int ncy, int ncz, const float *c, float *f, cudaStream_t s)
{
    const size_t n = (size_t)8 * ncx * ncy * ncz;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    launch_begin(K_PROLONG, s);
    prolong_kernel<<<blocks, 256, 0, s>>>(ncx, ncy, ncz, c, f);
    launch_end(K_PROLONG, s);
    return cudaGetLastError();
}

__global__ void state_init_kernel(DevState *st, cbct_recon_stats *rs)
{
    if (threadIdx.x == 0) {
        DevState z = {};
        *st = z;
        if (rs) {
            rs->n_iters = 0;
            rs->flags = 0;
            rs->status = CBCT_OK;
            rs->n_steps = 0;
            for (int l = 0; l < CBCT_MAX_LEVELS; l++) {
                rs->tau[l] = 0.0;
                rs->lipschitz[l] = 0.0;
            }
        }
    }
}

cudaError_t launch_state_init(DevState *st, cbct_recon_stats *rs, cudaStream_t s)
{
    launch_begin(K_MISC, s);
    state_init_kernel<<<1, 32, 0, s>>>(st, rs);
    launch_end(K_MISC, s);
    return cudaGetLastError();
}

} // namespace cbct
