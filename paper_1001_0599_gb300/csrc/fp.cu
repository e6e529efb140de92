// Cone-beam forward projector P (Eq. 1) for sm_103a, ray-driven.
//
// Discretisation: every source-to-pixel ray is sampled at in-plane distances
// rho_k = k drho from the source; the sample value is the trilinear
// interpolant of the voxel grid (zero outside) and each sample carries the
// length ds = drho |n| / |n_xy|. Because the in-plane position of sample k
// depends only on (view, iu), one warp takes one detector column iu and 32
// consecutive rows iv: the xy corners and weights of a sample are
// warp-uniform, and the 32 lanes read neighbouring z values of the same four
// voxel columns (z-fastest volume), so the gathers coalesce in L1. The tile
// of 8 columns x 32 rows is transposed through shared memory and written as
// 32-byte row segments of the u-fastest sinogram. Residual modes fuse
// T = P f - y (Sec. II.C.2) and the FP64-grade sum of T^2 into the epilogue.
#include "cbct_internal.cuh"

#include <climits>

namespace cbct {

constexpr int FP_WARPS = 8;   // detector columns per block
constexpr int FP_ROWS = 32;   // detector rows per block (one per lane)

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

template <int MODE>
__global__ void __launch_bounds__(FP_WARPS * 32)
fp_kernel(VolGeom g, DetGeom d, const float *__restrict__ vol, const float *__restrict__ y,
          float *__restrict__ out, const double *__restrict__ d_scale, double *__restrict__ partials)
{
    __shared__ float tile[FP_ROWS][FP_WARPS + 1];
    __shared__ float tile_ds[FP_ROWS][FP_WARPS + 1];
    __shared__ double red[32];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int view = blockIdx.z;
    const int iu = blockIdx.x * FP_WARPS + warp;
    const int iv = blockIdx.y * FP_ROWS + lane;

    float acc = 0.f, ds = 0.f;
    if (iu < d.nu) {  // warp-uniform
        const RayCol rc = g.cols[(size_t)view * d.nu + iu];
        const float v = ((float)iv - d.cv) * d.dv;
        const float vl = v * rc.inv_lxy;       // v / L_xy
        const float tz = vl * g.inv_dz;        // z voxel units per unit rho
        ds = g.drho * sqrtf(1.f + vl * vl);

        // samples whose z lies in (-1, nz) in voxel units; the rest weigh zero
        int jlo = rc.jlo, jhi = rc.jhi;
        if (iv >= d.nv) {
            jlo = INT_MAX;
            jhi = INT_MIN;
        } else if (tz != 0.f) {
            float r1 = (-1.f - g.cz) / tz, r2 = ((float)g.nz - g.cz) / tz;
            float rlo = fminf(r1, r2), rhi = fmaxf(r1, r2);
            rlo = fmaxf(rlo, -1.f);
            rhi = fminf(rhi, 1.0e7f);
            int klo = (int)floorf(rlo / g.drho) - 1, khi = (int)ceilf(rhi / g.drho) + 1;
            jlo = max(jlo, klo - rc.kc);
            jhi = min(jhi, khi - rc.kc);
        }
        const int wlo = __reduce_min_sync(0xffffffffu, jlo);
        const int whi = __reduce_max_sync(0xffffffffu, jhi);

        const int nx = g.nx, ny = g.ny, nz = g.nz;
        for (int j = wlo; j <= whi; ++j) {
            float fx, fy;
            sample_xy(g, rc, j, fx, fy);
            const float a0f = floorf(fx), b0f = floorf(fy);
            const int a0 = (int)a0f, b0 = (int)b0f;
            if (a0 < -1 || a0 >= nx || b0 < -1 || b0 >= ny) continue;  // uniform
            const float wx1 = fx - a0f, wy1 = fy - b0f;
            float wx0 = 1.f - wx1, wy0 = 1.f - wy1, wx1m = wx1, wy1m = wy1;
            if (a0 < 0) wx0 = 0.f;
            if (a0 + 1 >= nx) wx1m = 0.f;
            if (b0 < 0) wy0 = 0.f;
            if (b0 + 1 >= ny) wy1m = 0.f;
            const int ia0 = clampi(a0, 0, nx - 1), ia1 = clampi(a0 + 1, 0, nx - 1);
            const int ib0 = clampi(b0, 0, ny - 1), ib1 = clampi(b0 + 1, 0, ny - 1);
            const float w00 = wx0 * wy0, w01 = wx0 * wy1m, w10 = wx1m * wy0, w11 = wx1m * wy1m;
            const float *p00 = vol + ((size_t)ia0 * ny + ib0) * nz;
            const float *p01 = vol + ((size_t)ia0 * ny + ib1) * nz;
            const float *p10 = vol + ((size_t)ia1 * ny + ib0) * nz;
            const float *p11 = vol + ((size_t)ia1 * ny + ib1) * nz;

            const float rho = sample_rho(g, rc, j);
            const float zeta = __fmaf_rn(rho, tz, g.cz);
            const float c0f = floorf(zeta);
            const int c0 = (int)c0f;
            const float wz1 = zeta - c0f;
            float wz0 = 1.f - wz1, wz1m = wz1;
            if (c0 < 0 || c0 >= nz) wz0 = 0.f;
            if (c0 + 1 < 0 || c0 + 1 >= nz) wz1m = 0.f;
            const int ic0 = clampi(c0, 0, nz - 1), ic1 = clampi(c0 + 1, 0, nz - 1);

            const float col0 = w00 * __ldg(p00 + ic0) + w01 * __ldg(p01 + ic0) +
                               w10 * __ldg(p10 + ic0) + w11 * __ldg(p11 + ic0);
            const float col1 = w00 * __ldg(p00 + ic1) + w01 * __ldg(p01 + ic1) +
                               w10 * __ldg(p10 + ic1) + w11 * __ldg(p11 + ic1);
            acc += wz0 * col0 + wz1m * col1;
        }
    }

    tile[lane][warp] = acc * ds;
    tile_ds[lane][warp] = ds;
    __syncthreads();

    // transposed write-back: 32 rows x 8 consecutive columns
    const int row = threadIdx.x >> 3, col = threadIdx.x & 7;
    const int oiv = blockIdx.y * FP_ROWS + row, oiu = blockIdx.x * FP_WARPS + col;
    float r2 = 0.f;
    if (oiv < d.nv && oiu < d.nu) {
        const size_t o = ((size_t)view * d.nv + oiv) * d.nu + oiu;
        const float p = tile[row][col];
        if (MODE == 0) {
            const float scale = d_scale ? (float)(*d_scale) : 1.f;
            out[o] = p * scale;
        } else {
            const float r = p - __ldg(y + o);
            r2 = r * r;
            out[o] = (MODE == 1) ? r : r * tile_ds[row][col];
        }
    }
    if (MODE != 0) {
        DF v[1] = {DF{r2, 0.f}};
        double tot[1];
        block_sum_df<1>(v, red, tot);
        if (threadIdx.x == 0)
            partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = tot[0];
    }
}

int fp_grid_blocks(const DetGeom &d)
{
    return ((d.nu + FP_WARPS - 1) / FP_WARPS) * ((d.nv + FP_ROWS - 1) / FP_ROWS) * d.n_views;
}

cudaError_t launch_forward(const VolGeom &v, const DetGeom &d, const float *vol, const float *y,
                           float *out, const double *d_scale, double *partials, int mode,
                           cudaStream_t s)
{
    dim3 grid((d.nu + FP_WARPS - 1) / FP_WARPS, (d.nv + FP_ROWS - 1) / FP_ROWS, d.n_views);
    dim3 block(FP_WARPS * 32);
    const int kid = mode == 0 ? K_FP : K_FP_RESID;
    launch_begin(kid, s);
    if (mode == 0)
        fp_kernel<0><<<grid, block, 0, s>>>(v, d, vol, y, out, d_scale, partials);
    else if (mode == 1)
        fp_kernel<1><<<grid, block, 0, s>>>(v, d, vol, y, out, d_scale, partials);
    else
        fp_kernel<2><<<grid, block, 0, s>>>(v, d, vol, y, out, d_scale, partials);
    launch_end(kid, s);
    return cudaGetLastError();
}

} // namespace cbct
