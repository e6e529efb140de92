// Matched backprojector P^T for sm_103a: a voxel-driven gather that is the
// exact transpose of the ray-driven projector in fp.cu (the matrix view of
// Sec. II.C.2), with no atomics -- every voxel is written once.
//
// For voxel (a, b, c) and view theta, the non-zero entries of column
// (a, b, c) of P come from the samples j of the in-plane ray lines iu whose
// xy position falls inside the voxel column's 2dx x 2dy tent support, and,
// for each such sample, from the detector rows iv whose sample height lies
// within one dz of z_c. The xy weights of a (iu, j) sample are shared by
// whole voxel columns and every sample touches at most four columns, so one
// warp owns a 4 x 4 group of columns (its 32 lanes own consecutive z voxels):
// the warp visits every sample in the group's footprint once, each lane forms
// the sample's z tent sum for its voxels once, and the sum is added to the
// (up to four) columns the sample touches, held in registers and selected by
// a warp-uniform switch on the sample's xy cell.
//
// Per view the block stages the detector patch its voxel tile can see into
// shared memory column-major ([iu][iv], odd column pitch), padded by NR zero
// rows, and pre-weighted by the ray's sample length ds. A lane's rows for one
// sample are then NR consecutive words read with immediate offsets; the
// z tent weight max(0, 1 - sc |r - q|) zeroes the rows outside the tent, and
// NR (>= the largest number of rows a voxel's tent can span on this grid) is
// a template parameter, so the row loop is fully unrolled.
#include "cbct_internal.cuh"

#include <algorithm>
#include <cmath>

namespace cbct {

constexpr int BP_G = 4;               // a warp owns a BP_G x BP_G group of voxel columns
constexpr int BP_GX = 2, BP_GY = 2;   // groups per block along x, y
constexpr int BP_TX = BP_G * BP_GX, BP_TY = BP_G * BP_GY;   // voxel columns per block
constexpr int BP_ZC = 2;              // z chunks of 32 per lane
constexpr int BP_TZ = 32 * BP_ZC;
constexpr int BP_WARPS = BP_GX * BP_GY;
constexpr int BP_MAX_ROWS = 64;       // runtime row-loop bound (generic variant)

struct Box {
    float xlo, xhi, ylo, yhi;
};

__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.f, x); }

// detector columns [iu0, iu1] that can see the xy box in view (c, s), and the
// box's depth range along the central ray
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
        const float xr = x * c + y * s;
        const float yr = -x * s + y * c;
        const float u = -yr * d.sdd * fast_rcp(xr + d.sad);
        umin = fminf(umin, u);
        umax = fmaxf(umax, u);
        xr_lo = fminf(xr_lo, xr);
        xr_hi = fmaxf(xr_hi, xr);
    }
    iu0 = max((int)floorf(umin * d.inv_du + d.cu) - 1, 0);
    iu1 = min((int)ceilf(umax * d.inv_du + d.cu) + 1, d.nu - 1);
}

// The z tent sum of one sample for one lane's voxel c: sum over the rows r
// whose sample height is within one dz of z_c of (1 - sc |r - q|) * row value.
template <int NR, bool PRESCALED>
__device__ __forceinline__ float tent_rows(const DetGeom &d, const VolGeom &g, const float *pcol,
                                           const float *gcol, const RayCol &rc, bool staged, int s0,
                                           int s1, float q, float m, float sc)
{
    float s = 0.f;
    if (NR > 0 && staged) {
        int r0 = (int)ceilf(q - m);
        r0 = min(max(r0, s0), s1 - NR + 1);
        const float dq = (float)r0 - q;
        const float *p = pcol + r0;
#pragma unroll
        for (int t = 0; t < (NR > 0 ? NR : 1); ++t) {
            const float w = fmaxf(__fmaf_rn(-sc, fabsf(dq + (float)t), 1.f), 0.f);
            s = __fmaf_rn(w, p[t], s);
        }
    } else {
        const int r_lo = max((int)ceilf(q - m), 0);
        const int r_hi = min(min((int)floorf(q + m), d.nv - 1), r_lo + BP_MAX_ROWS);
        for (int r = r_lo; r <= r_hi; ++r) {
            const float w = fmaxf(__fmaf_rn(-sc, fabsf((float)r - q), 1.f), 0.f);
            float val;
            if (staged && r >= s0 && r <= s1) {
                val = pcol[r];
            } else {
                val = __ldg(gcol + (size_t)r * d.nu);
                if (!PRESCALED) {
                    const float vl = (((float)r - d.cv) * d.dv) * rc.inv_lxy;
                    val *= g.drho * sqrtf(1.f + vl * vl);
                }
            }
            s = __fmaf_rn(w, val, s);
        }
    }
    return s;
}

// Add a sample's z sums into the (up to four) columns of the warp's G x G
// group that its xy cell (RA, RB) (relative to the group) touches; corners
// outside the group belong to a neighbouring group's warp.
template <int IA, int IB>
__device__ __forceinline__ void add_one(float (&acc)[BP_G][BP_G][BP_ZC], float w, const float (&s)[BP_ZC])
{
    if constexpr (IA >= 0 && IA < BP_G && IB >= 0 && IB < BP_G) {
#pragma unroll
        for (int zc = 0; zc < BP_ZC; ++zc) acc[IA][IB][zc] = __fmaf_rn(w, s[zc], acc[IA][IB][zc]);
    }
}

template <int RA, int RB>
__device__ __forceinline__ void add_corners(float (&acc)[BP_G][BP_G][BP_ZC], float w00, float w01, float w10,
                                            float w11, const float (&s)[BP_ZC])
{
    add_one<RA, RB>(acc, w00, s);
    add_one<RA, RB + 1>(acc, w01, s);
    add_one<RA + 1, RB>(acc, w10, s);
    add_one<RA + 1, RB + 1>(acc, w11, s);
}

// NR > 0: rows per (lane, sample) fully unrolled; NR == 0: runtime loop.
// Block: BP_WARPS warps, each owning a BP_G x BP_G group of voxel columns and
// the block's 32*BP_ZC z values (one per lane and chunk).
template <int MODE, bool PRESCALED, int NR>
__global__ void __launch_bounds__(BP_WARPS * 32)
bp_kernel(VolGeom g, DetGeom d, const float *__restrict__ sino, const float *__restrict__ f,
          float *__restrict__ out, const double *__restrict__ d_scale, float scale_val, float kappa,
          double *__restrict__ partials, int patch_cap, int pad)
{
    extern __shared__ float patch[];
    __shared__ int s_box[6];
    __shared__ double red[32];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int a_base = blockIdx.x * BP_TX, b_base = blockIdx.y * BP_TY, c_base = blockIdx.z * BP_TZ;
    const int nx = g.nx, ny = g.ny, nz = g.nz, nu = d.nu, nv = d.nv;
    const int A = a_base + (warp % BP_GX) * BP_G, B = b_base + (warp / BP_GX) * BP_G;

    const float x_first = ((float)a_base - g.cx) * g.dx;
    const float y_first = ((float)b_base - g.cy) * g.dy;
    const Box tile_box{x_first - g.dx, x_first + (float)BP_TX * g.dx,
                       y_first - g.dy, y_first + (float)BP_TY * g.dy};
    const float z_lo = ((float)c_base - g.cz - 1.f) * g.dz;
    const float z_hi = ((float)(c_base + BP_TZ) - g.cz) * g.dz;
    const float xA = ((float)A - g.cx) * g.dx, yB = ((float)B - g.cy) * g.dy;
    const Box gbox{xA - g.dx, xA + (float)BP_G * g.dx, yB - g.dy, yB + (float)BP_G * g.dy};
    const bool group_live = A < nx && B < ny;

    float acc[BP_G][BP_G][BP_ZC];
#pragma unroll
    for (int i = 0; i < BP_G; i++)
#pragma unroll
        for (int k = 0; k < BP_G; k++)
#pragma unroll
            for (int z = 0; z < BP_ZC; z++) acc[i][k][z] = 0.f;

    for (int view = 0; view < d.n_views; ++view) {
        const float2 cs = d.views[view];
        if (threadIdx.x == 0) {
            int iu0, iu1;
            float xr_lo, xr_hi;
            box_u_range(d, cs.x, cs.y, tile_box, iu0, iu1, xr_lo, xr_hi);
            const float m_near = d.sdd / (xr_lo + d.sad), m_far = d.sdd / (xr_hi + d.sad);
            const float v1 = z_lo * m_near, v2 = z_lo * m_far, v3 = z_hi * m_near, v4 = z_hi * m_far;
            const float vmin = fminf(fminf(v1, v2), fminf(v3, v4));
            const float vmax = fmaxf(fmaxf(v1, v2), fmaxf(v3, v4));
            const int iv0 = max((int)floorf(vmin * d.inv_dv + d.cv) - 1, 0);
            const int iv1 = min((int)ceilf(vmax * d.inv_dv + d.cv) + 1, nv - 1);
            const int s0 = iv0 - pad, s1 = iv1 + pad;       // staged rows, zero outside the detector
            const int w = iu1 - iu0 + 1, h = s1 - s0 + 1;
            const int hp = h | 1;                           // odd column pitch
            s_box[0] = iu0;
            s_box[1] = iu1;
            s_box[2] = s0;
            s_box[3] = s1;
            s_box[4] = (iu1 >= iu0 && iv1 >= iv0 && w * hp <= patch_cap) ? hp : 0;
            s_box[5] = (iu1 >= iu0 && iv1 >= iv0) ? 1 : 0;
        }
        __syncthreads();
        const int iu0 = s_box[0], iu1 = s_box[1], s0 = s_box[2], s1 = s_box[3];
        const int hp = s_box[4];
        if (!s_box[5]) {
            __syncthreads();
            continue;
        }
        const bool staged = hp > 0;
        if (staged) {
            const int w = iu1 - iu0 + 1, h = s1 - s0 + 1;
            const float *src = sino + (size_t)view * nv * nu;
            for (int r = warp; r < h; r += BP_WARPS) {
                const int iv = s0 + r;
                const bool in = iv >= 0 && iv < nv;
                for (int cc = lane; cc < w; cc += 32) {
                    const int iu = iu0 + cc;
                    float val = 0.f;
                    if (in) {
                        val = __ldg(src + (size_t)iv * nu + iu);
                        if (!PRESCALED) {
                            const float vl = (((float)iv - d.cv) * d.dv) * g.cols[(size_t)view * nu + iu].inv_lxy;
                            val *= g.drho * sqrtf(1.f + vl * vl);
                        }
                    }
                    patch[cc * hp + r] = val;
                }
            }
        }
        __syncthreads();

        if (group_live) {  // warp-uniform
            int ju0, ju1;
            float dlo, dhi;
            box_u_range(d, cs.x, cs.y, gbox, ju0, ju1, dlo, dhi);
            ju0 = max(ju0, iu0);
            ju1 = min(ju1, iu1);
            const float inv_drho = fast_rcp(g.drho);
            for (int iu = ju0; iu <= ju1; ++iu) {
                const RayCol rc = g.cols[(size_t)view * nu + iu];
                // samples of this line inside the group's support box
                float tlo = -3.0e38f, thi = 3.0e38f;
                if (fabsf(rc.ex) > 1e-20f) {
                    const float inv = fast_rcp(rc.ex);
                    const float t1 = (gbox.xlo - rc.mx) * inv, t2 = (gbox.xhi - rc.mx) * inv;
                    tlo = fmaxf(tlo, fminf(t1, t2));
                    thi = fminf(thi, fmaxf(t1, t2));
                } else if (!(rc.mx > gbox.xlo && rc.mx < gbox.xhi)) {
                    continue;
                }
                if (fabsf(rc.ey) > 1e-20f) {
                    const float inv = fast_rcp(rc.ey);
                    const float t1 = (gbox.ylo - rc.my) * inv, t2 = (gbox.yhi - rc.my) * inv;
                    tlo = fmaxf(tlo, fminf(t1, t2));
                    thi = fminf(thi, fmaxf(t1, t2));
                } else if (!(rc.my > gbox.ylo && rc.my < gbox.yhi)) {
                    continue;
                }
                if (!(tlo < thi)) continue;
                const int jl = max((int)ceilf((tlo + rc.delta) * inv_drho) - 1, (int)rc.jlo);
                const int jh = min((int)floorf((thi + rc.delta) * inv_drho) + 1, (int)rc.jhi);
                const float sc_base = d.dv * rc.inv_lxy * g.inv_dz;
                const float *pcol = patch + (iu - iu0) * hp - s0;   // pcol[r] = row r of column iu
                const float *gcol = sino + (size_t)view * nv * nu + iu;
                for (int j = jl; j <= jh; ++j) {
                    float fx, fy;
                    sample_xy(g, rc, j, fx, fy);
                    const float a0f = floorf(fx), b0f = floorf(fy);
                    const int ra = (int)a0f - A, rb = (int)b0f - B;
                    if (ra < -1 || ra >= BP_G || rb < -1 || rb >= BP_G) continue;  // uniform
                    const float wx1 = fx - a0f, wy1 = fy - b0f;
                    const float wx0 = 1.f - wx1, wy0 = 1.f - wy1;
                    const float rho = sample_rho(g, rc, j);
                    const float sc = rho * sc_base;        // z (voxel units) per detector row
                    const float m = fast_rcp(sc);          // tent half-width in rows
                    float s[BP_ZC];
#pragma unroll
                    for (int zc = 0; zc < BP_ZC; ++zc) {
                        const int c = c_base + zc * 32 + lane;
                        const float q = d.cv + ((float)c - g.cz) * m;   // row whose sample hits z_c
                        s[zc] = tent_rows<NR, PRESCALED>(d, g, pcol, gcol, rc, staged, s0, s1, q, m, sc);
                    }
                    const float w00 = wx0 * wy0, w01 = wx0 * wy1, w10 = wx1 * wy0, w11 = wx1 * wy1;
                    switch ((ra + 1) * (BP_G + 1) + (rb + 1)) {
#define CBCT_CORNER(RA, RB)                                                                         \
    case ((RA) + 1) * (BP_G + 1) + ((RB) + 1):                                                      \
        add_corners<RA, RB>(acc, w00, w01, w10, w11, s);                                            \
        break;
#define CBCT_CORNER_ROW(RA)                                                                         \
    CBCT_CORNER(RA, -1) CBCT_CORNER(RA, 0) CBCT_CORNER(RA, 1) CBCT_CORNER(RA, 2) CBCT_CORNER(RA, 3)
                        CBCT_CORNER_ROW(-1)
                        CBCT_CORNER_ROW(0)
                        CBCT_CORNER_ROW(1)
                        CBCT_CORNER_ROW(2)
                        CBCT_CORNER_ROW(3)
#undef CBCT_CORNER_ROW
#undef CBCT_CORNER
                    default:
                        break;
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
    for (int ia = 0; ia < BP_G; ++ia)
#pragma unroll
        for (int ib = 0; ib < BP_G; ++ib) {
            const int a = A + ia, b = B + ib;
            if (a >= nx || b >= ny) continue;
#pragma unroll
            for (int zc = 0; zc < BP_ZC; ++zc) {
                const int c = c_base + zc * 32 + lane;
                if (c >= nz) continue;
                const size_t idx = ((size_t)a * ny + b) * nz + c;
                if (MODE == 0) {
                    out[idx] = acc[ia][ib][zc];
                } else if (MODE == 1) {
                    out[idx] = __fmaf_rn(-scale, acc[ia][ib][zc], __ldg(f + idx));
                } else {
                    const float w = kappa * acc[ia][ib][zc];
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

static double support_r(const VolGeom &v)
{
    return sqrt(pow(0.5 * (v.nx + 1) * v.dx, 2) + pow(0.5 * (v.ny + 1) * v.dy, 2));
}

// Largest number of detector rows one voxel's z tent can cover on this grid:
// floor(2 m) + 1 with m = 1/sc at the smallest sc = rho dv / (L_xy dz).
static int bp_rows_needed(const VolGeom &v, const DetGeom &d)
{
    const double R = support_r(v);
    const double umax = 0.5 * (d.nu - 1) * d.du;
    const double lxy_max = sqrt((double)d.sdd * d.sdd + umax * umax);
    const double sc_min = (d.sad - R) * d.dv / (lxy_max * v.dz);
    return (int)floor(2.0 / sc_min) + 2;
}

static int bp_nr_variant(const VolGeom &v, const DetGeom &d)
{
    const int need = bp_rows_needed(v, d);
    for (int nr : {6, 12, 24})
        if (need <= nr) return nr;
    return 0;
}

// Upper bound of the staged patch (host side, FP64, mirrors the device box
// computation with slack); tiles that still do not fit fall back to reading
// the sinogram from global memory.
size_t bp_smem_bytes(const VolGeom &v, const DetGeom &d)
{
    const double R = support_r(v);
    const double m_max = d.sdd / (d.sad - R), m_min = d.sdd / (d.sad + R);
    const double diag = sqrt(pow((BP_TX + 1) * (double)v.dx, 2) + pow((BP_TY + 1) * (double)v.dy, 2));
    const double w = std::min(diag * m_max / d.du + 6.0, (double)d.nu);
    const double zext = (BP_TZ + 1) * (double)v.dz;
    const double zabs = 0.5 * (v.nz + 1) * v.dz;
    const int nr = bp_nr_variant(v, d);
    const double h = std::min((zext * m_max + zabs * (m_max - m_min)) / d.dv + 6.0, (double)d.nv) + 2.0 * nr + 1;
    double cap = ceil(w) * (double)((int)ceil(h) | 1);
    const double cap_max = 48.0 * 1024.0;   // floats: 192 KB
    if (cap > cap_max) cap = cap_max;
    return (size_t)cap * sizeof(float);
}

template <int MODE, bool P, int NR>
static cudaError_t launch_one(dim3 grid, dim3 block, size_t smem, cudaStream_t s, const VolGeom &v,
                              const DetGeom &d, const float *sino, const float *f, float *out,
                              const double *d_scale, double scale_val, double kappa, double *partials, int cap,
                              int pad)
{
    cudaError_t e = cudaFuncSetAttribute(bp_kernel<MODE, P, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    bp_kernel<MODE, P, NR><<<grid, block, smem, s>>>(v, d, sino, f, out, d_scale, (float)scale_val, (float)kappa,
                                                     partials, cap, pad);
    return cudaGetLastError();
}

template <int MODE, bool P>
static cudaError_t launch_nr(int nr, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const VolGeom &v,
                             const DetGeom &d, const float *sino, const float *f, float *out,
                             const double *d_scale, double scale_val, double kappa, double *partials, int cap)
{
    switch (nr) {
    case 6:
        return launch_one<MODE, P, 6>(grid, block, smem, s, v, d, sino, f, out, d_scale, scale_val, kappa,
                                      partials, cap, 6);
    case 12:
        return launch_one<MODE, P, 12>(grid, block, smem, s, v, d, sino, f, out, d_scale, scale_val, kappa,
                                       partials, cap, 12);
    case 24:
        return launch_one<MODE, P, 24>(grid, block, smem, s, v, d, sino, f, out, d_scale, scale_val, kappa,
                                       partials, cap, 24);
    default:
        return launch_one<MODE, P, 0>(grid, block, smem, s, v, d, sino, f, out, d_scale, scale_val, kappa,
                                      partials, cap, 0);
    }
}

cudaError_t launch_back(const VolGeom &v, const DetGeom &d, const float *sino, const float *f,
                        float *out, const double *d_scale, double scale_val, double kappa,
                        double *partials, int mode, int prescaled, cudaStream_t s)
{
    dim3 grid((v.nx + BP_TX - 1) / BP_TX, (v.ny + BP_TY - 1) / BP_TY, (v.nz + BP_TZ - 1) / BP_TZ);
    dim3 block(BP_WARPS * 32);
    const size_t smem = bp_smem_bytes(v, d);
    const int cap = (int)(smem / sizeof(float));
    const int nr = bp_nr_variant(v, d);
    const int kid = mode == 1 ? K_BP_STEP : K_BP;
    cudaError_t e;
    launch_begin(kid, s);
    if (mode == 0)
        e = launch_nr<0, false>(nr, grid, block, smem, s, v, d, sino, f, out, d_scale, scale_val, kappa, partials,
                                cap);
    else if (mode == 1 && prescaled)
        e = launch_nr<1, true>(nr, grid, block, smem, s, v, d, sino, f, out, d_scale, scale_val, kappa, partials,
                               cap);
    else if (mode == 1)
        e = launch_nr<1, false>(nr, grid, block, smem, s, v, d, sino, f, out, d_scale, scale_val, kappa, partials,
                                cap);
    else
        e = launch_nr<2, false>(nr, grid, block, smem, s, v, d, sino, f, out, d_scale, scale_val, kappa, partials,
                                cap);
    launch_end(kid, s);
    return e;
}

} // namespace cbct
