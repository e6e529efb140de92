// Matched backprojector P^T for sm_103a: a voxel-driven gather that is the
// exact transpose of the ray-driven projector in fp.cu (the matrix view of
// Sec. II.C.2), with no atomics -- every voxel is written once.
//
// For voxel (a, b, c) and view theta, the non-zero entries of column
// (a, b, c) of P come from the samples j of the in-plane ray lines iu whose
// xy position falls inside the voxel column's 2dx x 2dy tent support, and,
// for each such sample, from the detector rows iv whose sample height lies
// within one dz of z_c. The xy weight of a (iu, j) pair is shared by a whole
// voxel column, so one warp owns one column and its 32 lanes own 32
// consecutive z voxels: the (iu, j) loop and the xy weights are warp-uniform
// and each lane only resolves its rows. Per view, the block stages the
// detector patch its voxel tile can see into shared memory (odd pitch, so the
// ~2-rows-per-lane access spreads over the banks); the patch holds ds * r,
// i.e. the per-ray sample length is folded in once per pixel.
#include "cbct_internal.cuh"

#include <algorithm>
#include <cmath>

namespace cbct {

constexpr int BP_TX = 4, BP_TY = 4;   // voxel columns per block
constexpr int BP_ZC = 2;              // z chunks of 32 per lane
constexpr int BP_TZ = 32 * BP_ZC;
constexpr int BP_WARPS = 8;
constexpr int BP_COLS_PER_WARP = BP_TX * BP_TY / BP_WARPS;

struct Box {
    float xlo, xhi, ylo, yhi;
};

// detector column range [*iu0, *iu1] that can see the xy box in view (c, s)
__device__ __forceinline__ void box_u_range(const DetGeom &d, float c, float s, const Box &bx,
                                            int &iu0, int &iu1, float &xr_lo, float &xr_hi)
{
    float umin = 3.0e38f, umax = -3.0e38f;
    xr_lo = 3.0e38f;
    xr_hi = -3.0e38f;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const float x = (k & 1) ? bx.xhi : bx.xlo;
        const float y = (k & 2) ? bx.yhi : bx.ylo;
        const float xr = x * c + y * s;          // depth along the central ray
        const float yr = -x * s + y * c;
        const float u = -yr * d.sdd / (xr + d.sad);
        umin = fminf(umin, u);
        umax = fmaxf(umax, u);
        xr_lo = fminf(xr_lo, xr);
        xr_hi = fmaxf(xr_hi, xr);
    }
    iu0 = max((int)floorf(umin * d.inv_du + d.cu) - 1, 0);
    iu1 = min((int)ceilf(umax * d.inv_du + d.cu) + 1, d.nu - 1);
}

template <int MODE, bool PRESCALED>
__global__ void __launch_bounds__(BP_WARPS * 32)
bp_kernel(VolGeom g, DetGeom d, const float *__restrict__ sino, const float *__restrict__ f,
          float *__restrict__ out, const double *__restrict__ d_scale, float scale_val, float kappa,
          double *__restrict__ partials, int patch_cap)
{
    extern __shared__ float patch[];
    __shared__ int s_box[5];
    __shared__ double red[32];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int a_base = blockIdx.x * BP_TX, b_base = blockIdx.y * BP_TY, c_base = blockIdx.z * BP_TZ;
    const int nx = g.nx, ny = g.ny, nz = g.nz, nu = d.nu, nv = d.nv;

    // tile support box (voxel centres +- one pitch)
    const float x_first = ((float)a_base - g.cx) * g.dx;
    const float y_first = ((float)b_base - g.cy) * g.dy;
    const Box tile_box{x_first - g.dx, x_first + (float)BP_TX * g.dx,
                       y_first - g.dy, y_first + (float)BP_TY * g.dy};
    const float z_lo = ((float)c_base - g.cz - 1.f) * g.dz;
    const float z_hi = ((float)(c_base + BP_TZ) - g.cz) * g.dz;

    float acc[BP_COLS_PER_WARP][BP_ZC];
#pragma unroll
    for (int i = 0; i < BP_COLS_PER_WARP; i++)
#pragma unroll
        for (int k = 0; k < BP_ZC; k++) acc[i][k] = 0.f;

    for (int view = 0; view < d.n_views; ++view) {
        const float2 cs = d.views[view];
        if (threadIdx.x == 0) {
            int iu0, iu1;
            float xr_lo, xr_hi;
            box_u_range(d, cs.x, cs.y, tile_box, iu0, iu1, xr_lo, xr_hi);
            // rows: v = z sdd / (depth + sad) over the tile's z and depth ranges
            const float m_near = d.sdd / (xr_lo + d.sad), m_far = d.sdd / (xr_hi + d.sad);
            const float v1 = z_lo * m_near, v2 = z_lo * m_far, v3 = z_hi * m_near, v4 = z_hi * m_far;
            const float vmin = fminf(fminf(v1, v2), fminf(v3, v4));
            const float vmax = fmaxf(fmaxf(v1, v2), fmaxf(v3, v4));
            const int iv0 = max((int)floorf(vmin * d.inv_dv + d.cv) - 1, 0);
            const int iv1 = min((int)ceilf(vmax * d.inv_dv + d.cv) + 1, nv - 1);
            const int w = iu1 - iu0 + 1, h = iv1 - iv0 + 1;
            const int pitch = w | 1;
            s_box[0] = iu0;
            s_box[1] = iu1;
            s_box[2] = iv0;
            s_box[3] = iv1;
            s_box[4] = (w > 0 && h > 0 && h * pitch <= patch_cap) ? pitch : 0;
        }
        __syncthreads();
        const int iu0 = s_box[0], iu1 = s_box[1], iv0 = s_box[2], iv1 = s_box[3];
        const int pitch = s_box[4];
        const bool staged = pitch > 0;
        if (iu1 < iu0 || iv1 < iv0) {
            __syncthreads();
            continue;
        }
        if (staged) {
            const int w = iu1 - iu0 + 1, h = iv1 - iv0 + 1;
            const float *src = sino + (size_t)view * nv * nu;
            for (int r = warp; r < h; r += BP_WARPS) {
                const int iv = iv0 + r;
                for (int cc = lane; cc < w; cc += 32) {
                    const int iu = iu0 + cc;
                    float val = __ldg(src + (size_t)iv * nu + iu);
                    if (!PRESCALED) {
                        const float vl = (((float)iv - d.cv) * d.dv) * g.cols[(size_t)view * nu + iu].inv_lxy;
                        val *= g.drho * sqrtf(1.f + vl * vl);
                    }
                    patch[r * pitch + cc] = val;
                }
            }
        }
        __syncthreads();

#pragma unroll
        for (int ci = 0; ci < BP_COLS_PER_WARP; ++ci) {
            const int tcol = warp + ci * BP_WARPS;
            const int a = a_base + (tcol % BP_TX), b = b_base + (tcol / BP_TX);
            if (a >= nx || b >= ny) continue;  // warp-uniform
            const float xa = ((float)a - g.cx) * g.dx, yb = ((float)b - g.cy) * g.dy;
            const Box cbox{xa - g.dx, xa + g.dx, yb - g.dy, yb + g.dy};
            int ju0, ju1;
            float dlo, dhi;
            box_u_range(d, cs.x, cs.y, cbox, ju0, ju1, dlo, dhi);
            ju0 = max(ju0, iu0);
            ju1 = min(ju1, iu1);
            for (int iu = ju0; iu <= ju1; ++iu) {
                const RayCol rc = g.cols[(size_t)view * nu + iu];
                // samples of this line inside the column's tent support
                float tlo = -3.0e38f, thi = 3.0e38f;
                if (fabsf(rc.ex) > 1e-20f) {
                    const float inv = 1.f / rc.ex;
                    const float t1 = (xa - g.dx - rc.mx) * inv, t2 = (xa + g.dx - rc.mx) * inv;
                    tlo = fmaxf(tlo, fminf(t1, t2));
                    thi = fminf(thi, fmaxf(t1, t2));
                } else if (fabsf(rc.mx - xa) >= g.dx) {
                    continue;
                }
                if (fabsf(rc.ey) > 1e-20f) {
                    const float inv = 1.f / rc.ey;
                    const float t1 = (yb - g.dy - rc.my) * inv, t2 = (yb + g.dy - rc.my) * inv;
                    tlo = fmaxf(tlo, fminf(t1, t2));
                    thi = fminf(thi, fmaxf(t1, t2));
                } else if (fabsf(rc.my - yb) >= g.dy) {
                    continue;
                }
                if (!(tlo < thi)) continue;
                const float inv_drho = 1.f / g.drho;
                int jl = (int)ceilf((tlo + rc.delta) * inv_drho) - 1;
                int jh = (int)floorf((thi + rc.delta) * inv_drho) + 1;
                jl = max(jl, (int)rc.jlo);
                jh = min(jh, (int)rc.jhi);
                const float sc_base = d.dv * rc.inv_lxy * g.inv_dz;
                for (int j = jl; j <= jh; ++j) {
                    float fx, fy;
                    sample_xy(g, rc, j, fx, fy);
                    const float a0f = floorf(fx), b0f = floorf(fy);
                    const int a0 = (int)a0f, b0 = (int)b0f;
                    const float wx1 = fx - a0f, wy1 = fy - b0f;
                    const float wx = (a == a0) ? 1.f - wx1 : ((a == a0 + 1) ? wx1 : 0.f);
                    const float wy = (b == b0) ? 1.f - wy1 : ((b == b0 + 1) ? wy1 : 0.f);
                    const float wxy = wx * wy;
                    if (wxy == 0.f) continue;  // uniform
                    const float rho = sample_rho(g, rc, j);
                    const float sc = rho * sc_base;    // z (voxel units) per detector row
                    const float inv_sc = 1.f / sc;
#pragma unroll
                    for (int zc = 0; zc < BP_ZC; ++zc) {
                        const int c = c_base + zc * 32 + lane;
                        const float q = d.cv + ((float)c - g.cz) * inv_sc;  // row whose sample hits z_c
                        int r_lo = max((int)ceilf(q - inv_sc), 0);
                        int r_hi = min((int)floorf(q + inv_sc), nv - 1);
                        float s = 0.f;
                        if (staged) {
                            r_lo = max(r_lo, iv0);
                            r_hi = min(r_hi, iv1);
                            const float *pp = patch + (iu - iu0);
                            for (int r = r_lo; r <= r_hi; ++r) {
                                const float w = fmaxf(1.f - sc * fabsf((float)r - q), 0.f);
                                s += w * pp[(r - iv0) * pitch];
                            }
                        } else {
                            const float *src = sino + (size_t)view * nv * nu + iu;
                            for (int r = r_lo; r <= r_hi; ++r) {
                                const float w = fmaxf(1.f - sc * fabsf((float)r - q), 0.f);
                                float val = __ldg(src + (size_t)r * nu);
                                if (!PRESCALED) {
                                    const float vl = (((float)r - d.cv) * d.dv) * rc.inv_lxy;
                                    val *= g.drho * sqrtf(1.f + vl * vl);
                                }
                                s += w * val;
                            }
                        }
                        acc[ci][zc] += wxy * s;
                    }
                }
            }
        }
        __syncthreads();
    }

    // epilogue: one write per voxel
    const float scale = (MODE == 1) ? (d_scale ? (float)(*d_scale) : scale_val) : 0.f;
    float sq = 0.f;
#pragma unroll
    for (int ci = 0; ci < BP_COLS_PER_WARP; ++ci) {
        const int tcol = warp + ci * BP_WARPS;
        const int a = a_base + (tcol % BP_TX), b = b_base + (tcol / BP_TX);
        if (a >= nx || b >= ny) continue;
#pragma unroll
        for (int zc = 0; zc < BP_ZC; ++zc) {
            const int c = c_base + zc * 32 + lane;
            if (c >= nz) continue;
            const size_t idx = ((size_t)a * ny + b) * nz + c;
            if (MODE == 0) {
                out[idx] = acc[ci][zc];
            } else if (MODE == 1) {
                out[idx] = __fmaf_rn(-scale, acc[ci][zc], __ldg(f + idx));
            } else {
                const float w = kappa * acc[ci][zc];
                out[idx] = w;
                sq += w * w;
            }
        }
    }
    if (MODE == 2) {
        DF v[1] = {DF{sq, 0.f}};
        double tot[1];
        block_sum_df<1>(v, red, tot);
        if (threadIdx.x == 0)
            partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = tot[0];
    }
}

int bp_grid_blocks(const VolGeom &v)
{
    return ((v.nx + BP_TX - 1) / BP_TX) * ((v.ny + BP_TY - 1) / BP_TY) * ((v.nz + BP_TZ - 1) / BP_TZ);
}

// Upper bound of the staged patch (host side, FP64, mirrors the device box
// computation with two pixels of slack); tiles that still do not fit fall
// back to reading the sinogram from global memory.
size_t bp_smem_bytes(const VolGeom &v, const DetGeom &d)
{
    const double R = sqrt(pow(0.5 * (v.nx + 1) * v.dx, 2) + pow(0.5 * (v.ny + 1) * v.dy, 2));
    const double m_max = d.sdd / (d.sad - R), m_min = d.sdd / (d.sad + R);
    const double diag = sqrt(pow((BP_TX + 1) * (double)v.dx, 2) + pow((BP_TY + 1) * (double)v.dy, 2));
    const double w = std::min(diag * m_max / d.du + 6.0, (double)d.nu);
    const double zext = (BP_TZ + 1) * (double)v.dz;
    const double zabs = 0.5 * (v.nz + 1) * v.dz;
    const double h = std::min((zext * m_max + zabs * (m_max - m_min)) / d.dv + 6.0, (double)d.nv);
    double cap = (double)((int)ceil(w) | 1) * ceil(h);
    const double cap_max = 48.0 * 1024.0;   // floats: 192 KB
    if (cap > cap_max) cap = cap_max;
    return (size_t)cap * sizeof(float);
}

cudaError_t launch_back(const VolGeom &v, const DetGeom &d, const float *sino, const float *f,
                        float *out, const double *d_scale, double scale_val, double kappa,
                        double *partials, int mode, int prescaled, cudaStream_t s)
{
    dim3 grid((v.nx + BP_TX - 1) / BP_TX, (v.ny + BP_TY - 1) / BP_TY, (v.nz + BP_TZ - 1) / BP_TZ);
    dim3 block(BP_WARPS * 32);
    const size_t smem = bp_smem_bytes(v, d);
    const int cap = (int)(smem / sizeof(float));
    const int kid = mode == 1 ? K_BP_STEP : K_BP;
    cudaError_t e = cudaSuccess;
#define CBCT_BP_LAUNCH(M, P)                                                                        \
    do {                                                                                            \
        e = cudaFuncSetAttribute(bp_kernel<M, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                 (int)smem);                                                        \
        if (e != cudaSuccess) return e;                                                             \
        launch_begin(kid, s);                                                                       \
        bp_kernel<M, P><<<grid, block, smem, s>>>(v, d, sino, f, out, d_scale, (float)scale_val,    \
                                                  (float)kappa, partials, cap);                     \
        launch_end(kid, s);                                                                         \
    } while (0)
    if (mode == 0) {
        if (prescaled) CBCT_BP_LAUNCH(0, true);
        else CBCT_BP_LAUNCH(0, false);
    } else if (mode == 1) {
        if (prescaled) CBCT_BP_LAUNCH(1, true);
        else CBCT_BP_LAUNCH(1, false);
    } else {
        if (prescaled) CBCT_BP_LAUNCH(2, true);
        else CBCT_BP_LAUNCH(2, false);
    }
#undef CBCT_BP_LAUNCH
    return cudaGetLastError();
}

} // namespace cbct
