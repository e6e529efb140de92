// Cone-beam forward projector P (Eq. 1) for sm_103a, ray-driven.
//
// Discretisation: every source-to-pixel ray is sampled at in-plane distances
// rho_k = k drho from the source; the sample value is the trilinear
// interpolant of the voxel grid (zero outside) and each sample carries the
// length ds = drho |n| / |n_xy|. Because the in-plane position of sample k
// depends only on (view, iu), one warp takes one detector column iu and
// 32*RPL consecutive rows iv. Per sample the four xy corners and weights are
// warp-uniform; the warp first blends the four voxel columns over the z range
// its rows touch (one coalesced z segment per lane, h(c) = sum of the four
// corner values weighted bilinearly), parks that segment in shared memory,
// and then every row only interpolates h linearly at its own height. The
// block's tile of 8 columns x 32*RPL rows is transposed through shared memory
// and written as 32-byte row segments of the u-fastest sinogram. Residual
// modes fuse T = P f - y (Sec. II.C.2) and the FP64-grade sum of T^2.
#include "cbct_internal.cuh"

#include <algorithm>
#include <climits>

namespace cbct {

constexpr int FP_WARPS = 8;   // detector columns per block
constexpr int FP_HMAX = 64;   // z values of one blended segment

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

template <int MODE, int RPL>
__global__ void __launch_bounds__(FP_WARPS * 32)
fp_kernel(VolGeom g, DetGeom d, const float *__restrict__ vol, const float *__restrict__ y,
          float *__restrict__ out, const double *__restrict__ d_scale, double *__restrict__ partials)
{
    constexpr int ROWS = 32 * RPL;
    __shared__ float tile[ROWS][FP_WARPS + 1];
    __shared__ float tile_ds[(MODE == 2 || MODE == 3) ? ROWS : 1][FP_WARPS + 1];
    __shared__ float hbuf[FP_WARPS][FP_HMAX + 2];
    __shared__ double red[32];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int view = blockIdx.z;
    const int iu = blockIdx.x * FP_WARPS + warp;
    const int row0 = blockIdx.y * ROWS;
    const int nz = g.nz;

    float acc[RPL], tz[RPL], ds[RPL];
#pragma unroll
    for (int k = 0; k < RPL; k++) acc[k] = 0.f;

    if (iu < d.nu) {  // warp-uniform
        const RayCol rc = g.cols[(size_t)view * d.nu + iu];
        const float kz = d.dv * rc.inv_lxy;        // v / L_xy per detector row
#pragma unroll
        for (int k = 0; k < RPL; k++) {
            const float vrow = ((float)(row0 + lane + 32 * k) - d.cv);
            const float vl = vrow * kz;
            tz[k] = vl * g.inv_dz;
            ds[k] = g.drho * sqrtf(1.f + vl * vl);
        }
        const int last = min(row0 + ROWS - 1, d.nv - 1);
        const float tz_a = (((float)row0 - d.cv) * kz) * g.inv_dz;
        const float tz_b = (((float)last - d.cv) * kz) * g.inv_dz;

        // rows leave the volume through its top or bottom once rho is large
        int jhi = rc.jhi;
        float rho_max = 3.0e38f;
        if (tz_b < 0.f) rho_max = fminf(rho_max, (1.f + g.cz) / (-tz_b));
        if (tz_a > 0.f) rho_max = fminf(rho_max, ((float)nz - g.cz) / tz_a);
        if (rho_max < 1.0e7f) jhi = min(jhi, (int)ceilf(rho_max / g.drho) + 1 - rc.kc);
        const int jlo = rc.jlo;

        const int nx = g.nx, ny = g.ny;
        float *hb = hbuf[warp];
        for (int j = jlo; j <= jhi; ++j) {
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
            const int o00 = (ia0 * ny + ib0) * nz, o01 = (ia0 * ny + ib1) * nz;
            const int o10 = (ia1 * ny + ib0) * nz, o11 = (ia1 * ny + ib1) * nz;

            const float rho = sample_rho(g, rc, j);
            const float za = __fmaf_rn(rho, tz_a, g.cz), zb = __fmaf_rn(rho, tz_b, g.cz);
            const int clo = max((int)floorf(za), -1);
            const int chi = min((int)floorf(zb) + 1, nz);
            const int span = chi - clo + 1;
            if (span <= FP_HMAX) {
                for (int t = lane; t < span; t += 32) {
                    const int c = clo + t;
                    float h = 0.f;
                    if (c >= 0 && c < nz)
                        h = w00 * __ldg(vol + o00 + c) + w01 * __ldg(vol + o01 + c) +
                            w10 * __ldg(vol + o10 + c) + w11 * __ldg(vol + o11 + c);
                    hb[t] = h;
                }
                __syncwarp();
#pragma unroll
                for (int k = 0; k < RPL; k++) {
                    const float zeta = __fmaf_rn(rho, tz[k], g.cz);
                    const float c0f = floorf(zeta);
                    const int idx = (int)c0f - clo;
                    if (idx >= 0 && idx <= span - 2) {
                        const float wz1 = zeta - c0f;
                        const float h0 = hb[idx], h1 = hb[idx + 1];
                        acc[k] += h0 + wz1 * (h1 - h0);
                    }
                }
                __syncwarp();
            } else {
                // steep rows: direct trilinear gathers per lane
#pragma unroll
                for (int k = 0; k < RPL; k++) {
                    const float zeta = __fmaf_rn(rho, tz[k], g.cz);
                    const float c0f = floorf(zeta);
                    const int c0 = (int)c0f;
                    if (c0 < -1 || c0 >= nz) continue;
                    const float wz1 = zeta - c0f;
                    const float wz0 = c0 >= 0 ? 1.f - wz1 : 0.f;
                    const float wz1m = c0 + 1 < nz ? wz1 : 0.f;
                    const int ic0 = clampi(c0, 0, nz - 1), ic1 = clampi(c0 + 1, 0, nz - 1);
                    const float h0 = w00 * __ldg(vol + o00 + ic0) + w01 * __ldg(vol + o01 + ic0) +
                                     w10 * __ldg(vol + o10 + ic0) + w11 * __ldg(vol + o11 + ic0);
                    const float h1 = w00 * __ldg(vol + o00 + ic1) + w01 * __ldg(vol + o01 + ic1) +
                                     w10 * __ldg(vol + o10 + ic1) + w11 * __ldg(vol + o11 + ic1);
                    acc[k] += wz0 * h0 + wz1m * h1;
                }
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < RPL; k++) ds[k] = 0.f;
    }

#pragma unroll
    for (int k = 0; k < RPL; k++) {
        tile[lane + 32 * k][warp] = acc[k] * ds[k];
        if (MODE == 2 || MODE == 3) tile_ds[lane + 32 * k][warp] = ds[k];
    }
    __syncthreads();

    // transposed write-back: ROWS rows x 8 consecutive columns
    float r2 = 0.f;
    const float scale = ((MODE == 0 || MODE == 3) && d_scale) ? (float)(*d_scale) : 1.f;
    for (int e = threadIdx.x; e < ROWS * FP_WARPS; e += FP_WARPS * 32) {
        const int row = e >> 3, col = e & 7;
        const int oiv = row0 + row, oiu = blockIdx.x * FP_WARPS + col;
        if (oiv < d.nv && oiu < d.nu) {
            const size_t o = ((size_t)view * d.nv + oiv) * d.nu + oiu;
            const float p = tile[row][col];
            if (MODE == 0) {
                out[o] = p * scale;
            } else if (MODE == 3) {
                out[o] = p * scale * tile_ds[row][col];
            } else {
                const float r = p - __ldg(y + o);
                r2 += r * r;
                out[o] = (MODE == 1) ? r : r * tile_ds[MODE == 2 ? row : 0][col];
            }
        }
    }
    if (MODE == 1 || MODE == 2) {
        DF v[1] = {DF{r2, 0.f}};
        double tot[1];
        block_sum_df<1>(v, red, tot);
        if (threadIdx.x == 0)
            partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = tot[0];
    }
}

// ---------------------------------------------------------------------------
// Sheet variant: one block per ray line (view, iu) and all its detector rows.
// The samples j of the line are processed in chunks of FS_J: (1) one lane per
// sample computes its xy corners and bilinear weights, (2) the block blends
// the four voxel columns of every sample over the z range the rows can see,
// giving the in-plane "sheet" H(j, c), and (3) every thread walks its rows
// through the chunk, interpolating H linearly at the row's height. No work is
// repeated across warps; H is padded with two zero entries on each side of z
// so rows outside the volume need no branches.
// ---------------------------------------------------------------------------
constexpr int FS_THREADS = 128;
constexpr int FS_J = 32;

// Four consecutive stored values widened to FP32 (16-byte or 8-byte load;
// the caller guarantees the alignment).
__device__ __forceinline__ float4 ld4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ float4 ld4(const __nv_bfloat16 *p)
{
    const uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u), __uint_as_float(u.y << 16),
                       __uint_as_float(u.y & 0xffff0000u));
}
__device__ __forceinline__ float4 ld4(const __half *p)
{
    const uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

// Zero entries on each z side of a sheet row (the rows' interpolation reads
// c0 in [-2, nz] and c0 + 1); four keep 16-byte alignment of the row body.
constexpr int FS_PAD = 4;

// One chunk of xy-blended sheet rows: H[jj][c] = sum of the four xy corner
// columns weighted, for the z range [clo, chi]. With nz a multiple of 4 each
// lane blends four consecutive z values per step (vector loads and store);
// the range is widened to whole quads, which stay inside the volume.
template <typename T>
__device__ __forceinline__ void build_sheet(float *H, int hs, int nz, const T *__restrict__ vol,
                                            const int (*s_o)[FS_J], const float (*s_w)[FS_J], int nj, int clo,
                                            int chi, int warp, int lane)
{
    const bool quads = (nz & 3) == 0;
    for (int jj = warp; jj < nj; jj += FS_THREADS / 32) {
        const int o0 = s_o[0][jj], o1 = s_o[1][jj], o2 = s_o[2][jj], o3 = s_o[3][jj];
        const float w0 = s_w[0][jj], w1 = s_w[1][jj], w2 = s_w[2][jj], w3 = s_w[3][jj];
        float *Hr = H + jj * hs + FS_PAD;
        if (quads) {
            for (int c = (clo & ~3) + 4 * lane; c <= chi; c += 128) {
                const float4 v0 = ld4(vol + o0 + c), v1 = ld4(vol + o1 + c);
                const float4 v2 = ld4(vol + o2 + c), v3 = ld4(vol + o3 + c);
                float4 h;
                h.x = w0 * v0.x + w1 * v1.x + w2 * v2.x + w3 * v3.x;
                h.y = w0 * v0.y + w1 * v1.y + w2 * v2.y + w3 * v3.y;
                h.z = w0 * v0.z + w1 * v1.z + w2 * v2.z + w3 * v3.z;
                h.w = w0 * v0.w + w1 * v1.w + w2 * v2.w + w3 * v3.w;
                *reinterpret_cast<float4 *>(Hr + c) = h;
            }
        } else {
            for (int c = clo + lane; c <= chi; c += 32)
                Hr[c] = w0 * ldt(vol + o0 + c) + w1 * ldt(vol + o1 + c) + w2 * ldt(vol + o2 + c) +
                        w3 * ldt(vol + o3 + c);
        }
    }
}

__device__ __forceinline__ void store_t(float *p, float v) { *p = v; }
__device__ __forceinline__ void store_t(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void store_t(__half *p, float v) { *p = __float2half_rn(v); }

// Rows of one ray line: projection (modes 0, 3) or residual (modes 1, 2) out,
// returns the thread's sum of squared residuals
template <int MODE, int RT, typename T>
__device__ __forceinline__ float sheet_epilogue(const T *__restrict__ y, T *__restrict__ out, const float (&acc)[RT],
                                                const float (&ds)[RT], float scale, size_t o_base, int tid, int nv,
                                                int nu)
{
    float r2 = 0.f;
#pragma unroll
    for (int k = 0; k < RT; k++) {
        const int iv = tid + FS_THREADS * k;
        if (iv < nv) {
            const size_t o = o_base + (size_t)iv * nu;
            const float p = acc[k] * ds[k];
            if (MODE == 0) {
                store_t(out + o, p * scale);
            } else if (MODE == 3) {
                store_t(out + o, p * scale * ds[k]);
            } else {
                const float r = p - ldt(y + o);
                r2 += r * r;
                store_t(out + o, (MODE == 1) ? r : r * ds[k]);
            }
        }
    }
    return r2;
}

constexpr float FS_ROUND = 12582912.f;     // 1.5 * 2^23: x + FS_ROUND rounds x to an integer
constexpr int FS_ROUND_BITS = 0x4B400000;  // bit pattern of FS_ROUND

// Every row k in LIVE walks the chunk's samples: the row's height at sample jj
// in voxel units, zeta = cz + rho_jj tz_k, splits into the voxel c0 = floor
// (a round-down add against 1.5 * 2^23, on the FMA and integer pipes) and the
// weight of c0 + 1; the sheet row is read at c0 and c0 + 1 (clamped into its
// zero pads).
template <int RT, unsigned LIVE>
__device__ __forceinline__ void sheet_walk(const float *H, int hs, const float *s_rho, int nj, const float (&tz)[RT],
                                           float cz, int nz, float (&acc)[RT])
{
#pragma unroll 4
    for (int jj = 0; jj < nj; ++jj) {
        const float rho = s_rho[jj];
        const int row = jj * hs + FS_PAD;
#pragma unroll
        for (int k = 0; k < RT; k++) {
            if (!((LIVE >> k) & 1u)) continue;
            const float zeta = __fmaf_rn(rho, tz[k], cz);
            const float tb = __fadd_rd(zeta, FS_ROUND);   // FS_ROUND + floor(zeta)
            const float c0f = tb - FS_ROUND;
            const int c0 = clampi(__float_as_int(tb) - FS_ROUND_BITS, -2, nz);
            const float wz1 = zeta - c0f;
            const float h0 = H[row + c0], h1 = H[row + c0 + 1];
            acc[k] += h0 + wz1 * (h1 - h0);
        }
    }
}

// the row walk specialised for the live set of bands (all 2^RT sets for up
// to three rows per thread; a runtime test per band beyond that)
template <int RT>
__device__ __forceinline__ void sheet_walk_bands(unsigned live, const float *H, int hs, const float *s_rho, int nj,
                                                 const float (&tz)[RT], float cz, int nz, float (&acc)[RT])
{
    if constexpr (RT <= 3) {
        switch (live) {
        case 1: sheet_walk<RT, 1>(H, hs, s_rho, nj, tz, cz, nz, acc); break;
        case 2: sheet_walk<RT, 2>(H, hs, s_rho, nj, tz, cz, nz, acc); break;
        case 3: sheet_walk<RT, 3>(H, hs, s_rho, nj, tz, cz, nz, acc); break;
        case 4: sheet_walk<RT, 4>(H, hs, s_rho, nj, tz, cz, nz, acc); break;
        case 5: sheet_walk<RT, 5>(H, hs, s_rho, nj, tz, cz, nz, acc); break;
        case 6: sheet_walk<RT, 6>(H, hs, s_rho, nj, tz, cz, nz, acc); break;
        case 7: sheet_walk<RT, 7>(H, hs, s_rho, nj, tz, cz, nz, acc); break;
        default: break;
        }
    } else {
        // tall detectors: one specialisation per band would multiply the code; walk
        // every band, testing liveness per sample
#pragma unroll 2
        for (int jj = 0; jj < nj; ++jj) {
            const float rho = s_rho[jj];
            const int row = jj * hs + FS_PAD;
#pragma unroll
            for (int k = 0; k < RT; k++) {
                if (!((live >> k) & 1u)) continue;
                const float zeta = __fmaf_rn(rho, tz[k], cz);
                const float tb = __fadd_rd(zeta, FS_ROUND);
                const float c0f = tb - FS_ROUND;
                const int c0 = clampi(__float_as_int(tb) - FS_ROUND_BITS, -2, nz);
                const float wz1 = zeta - c0f;
                const float h0 = H[row + c0], h1 = H[row + c0 + 1];
                acc[k] += h0 + wz1 * (h1 - h0);
            }
        }
    }
}

// register budgets: 64 for up to 3 rows per thread (8 blocks of 128 threads
// per SM; deep volumes are limited by the sheet's shared memory first), and
// enough for 4 or 8 rows to avoid local-memory spills
template <int MODE, int RT>
__global__ void __launch_bounds__(FS_THREADS, RT <= 3 ? 8 : (RT == 4 ? 7 : 6))
fp_sheet_kernel(VolGeom g, DetGeom d, const void *__restrict__ vol, const void *__restrict__ y,
                void *__restrict__ out, int st, const double *__restrict__ d_scale, double *__restrict__ partials)
{
    extern __shared__ float H[];               // [FS_J][nz + 2 FS_PAD]
    __shared__ int s_o[4][FS_J];
    __shared__ float s_w[4][FS_J];
    __shared__ float s_rho[FS_J];
    __shared__ int s_range[2];
    __shared__ double red[32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int iu = blockIdx.x, view = blockIdx.y;
    const int nx = g.nx, ny = g.ny, nz = g.nz, nv = d.nv;
    const int hs = nz + 2 * FS_PAD;
    const RayCol rc = g.cols[(size_t)view * d.nu + iu];
    const float kz = d.dv * rc.inv_lxy;

    float acc[RT], tz[RT], ds[RT];
#pragma unroll
    for (int k = 0; k < RT; k++) {
        const float vl = ((float)(tid + FS_THREADS * k) - d.cv) * kz;
        tz[k] = vl * g.inv_dz;
        ds[k] = g.drho * sqrtf(1.f + vl * vl);
        acc[k] = 0.f;
    }
    const float tz_min = ((0.f - d.cv) * kz) * g.inv_dz;
    const float tz_max = (((float)(nv - 1) - d.cv) * kz) * g.inv_dz;
    for (int j = tid; j < FS_J; j += FS_THREADS) {
        float *Hr = H + j * hs;
#pragma unroll
        for (int t = 0; t < FS_PAD; ++t) Hr[t] = Hr[nz + FS_PAD + t] = 0.f;
    }
    // rows leave the volume through its top or bottom once rho is large
    int jhi = rc.jhi;
    {
        float rho_max = 3.0e38f;
        if (tz_max < 0.f) rho_max = fminf(rho_max, (1.f + g.cz) / (-tz_max));
        if (tz_min > 0.f) rho_max = fminf(rho_max, ((float)nz - g.cz) / tz_min);
        if (rho_max < 1.0e7f) jhi = min(jhi, (int)ceilf(rho_max / g.drho) + 1 - rc.kc);
    }

    for (int j0 = rc.jlo; j0 <= jhi; j0 += FS_J) {
        const int nj = min(FS_J, jhi - j0 + 1);
        if (warp == 0) {
            if (lane < nj) {
                float fx, fy;
                sample_xy(g, rc, j0 + lane, fx, fy);
                const float a0f = floorf(fx), b0f = floorf(fy);
                const int a0 = (int)a0f, b0 = (int)b0f;
                const float wx1 = fx - a0f, wy1 = fy - b0f;
                float wx0 = 1.f - wx1, wy0 = 1.f - wy1, wx1m = wx1, wy1m = wy1;
                if (a0 < 0 || a0 >= nx) wx0 = 0.f;
                if (a0 + 1 < 0 || a0 + 1 >= nx) wx1m = 0.f;
                if (b0 < 0 || b0 >= ny) wy0 = 0.f;
                if (b0 + 1 < 0 || b0 + 1 >= ny) wy1m = 0.f;
                const int ia0 = clampi(a0, 0, nx - 1), ia1 = clampi(a0 + 1, 0, nx - 1);
                const int ib0 = clampi(b0, 0, ny - 1), ib1 = clampi(b0 + 1, 0, ny - 1);
                s_o[0][lane] = (ia0 * ny + ib0) * nz;
                s_o[1][lane] = (ia0 * ny + ib1) * nz;
                s_o[2][lane] = (ia1 * ny + ib0) * nz;
                s_o[3][lane] = (ia1 * ny + ib1) * nz;
                s_w[0][lane] = wx0 * wy0;
                s_w[1][lane] = wx0 * wy1m;
                s_w[2][lane] = wx1m * wy0;
                s_w[3][lane] = wx1m * wy1m;
                s_rho[lane] = sample_rho(g, rc, j0 + lane);
            }
            if (lane == 0) {
                // z range the rows can reach over this chunk (rho grows with j)
                const float ra = sample_rho(g, rc, j0), rb = sample_rho(g, rc, j0 + nj - 1);
                const float zmin = fminf(fminf(__fmaf_rn(ra, tz_min, g.cz), __fmaf_rn(rb, tz_min, g.cz)),
                                         fminf(__fmaf_rn(ra, tz_max, g.cz), __fmaf_rn(rb, tz_max, g.cz)));
                const float zmax = fmaxf(fmaxf(__fmaf_rn(ra, tz_min, g.cz), __fmaf_rn(rb, tz_min, g.cz)),
                                         fmaxf(__fmaf_rn(ra, tz_max, g.cz), __fmaf_rn(rb, tz_max, g.cz)));
                s_range[0] = max((int)floorf(zmin) - 1, 0);
                s_range[1] = min((int)floorf(zmax) + 2, nz - 1);
            }
        }
        __syncthreads();
        const int clo = s_range[0], chi = s_range[1];
        if (st == CBCT_STORAGE_BF16)
            build_sheet(H, hs, nz, static_cast<const __nv_bfloat16 *>(vol), s_o, s_w, nj, clo, chi, warp, lane);
        else if (st == CBCT_STORAGE_F16)
            build_sheet(H, hs, nz, static_cast<const __half *>(vol), s_o, s_w, nj, clo, chi, warp, lane);
        else
            build_sheet(H, hs, nz, static_cast<const float *>(vol), s_o, s_w, nj, clo, chi, warp, lane);
        __syncthreads();
        // 32-row bands whose rows stay outside the volume over the whole chunk
        // (rows above the top or below the bottom for every sample) are skipped;
        // the set of live bands is warp-uniform, so the row walk is specialised
        // for it once per chunk instead of testing every band at every sample
        unsigned live = 0;
        {
            const float ra = s_rho[0], rb = s_rho[nj - 1];
#pragma unroll
            for (int k = 0; k < RT; k++) {
                const float t_lo = __shfl_sync(0xffffffffu, tz[k], 0), t_hi = __shfl_sync(0xffffffffu, tz[k], 31);
                const float z1 = __fmaf_rn(ra, t_lo, g.cz), z2 = __fmaf_rn(rb, t_lo, g.cz);
                const float z3 = __fmaf_rn(ra, t_hi, g.cz), z4 = __fmaf_rn(rb, t_hi, g.cz);
                const float zlo = fminf(fminf(z1, z2), fminf(z3, z4)), zhi = fmaxf(fmaxf(z1, z2), fmaxf(z3, z4));
                if (!(zhi < -1.f || zlo >= (float)nz)) live |= 1u << k;
            }
        }
        sheet_walk_bands<RT>(live, H, hs, s_rho, nj, tz, g.cz, nz, acc);
        __syncthreads();
    }

    const float scale = ((MODE == 0 || MODE == 3) && d_scale) ? (float)(*d_scale) : 1.f;
    const size_t o_base = (size_t)view * nv * d.nu + iu;
    float r2;
    if (st == CBCT_STORAGE_BF16)
        r2 = sheet_epilogue<MODE, RT>(static_cast<const __nv_bfloat16 *>(y), static_cast<__nv_bfloat16 *>(out),
                                      acc, ds, scale, o_base, tid, nv, d.nu);
    else if (st == CBCT_STORAGE_F16)
        r2 = sheet_epilogue<MODE, RT>(static_cast<const __half *>(y), static_cast<__half *>(out), acc, ds, scale,
                                      o_base, tid, nv, d.nu);
    else
        r2 = sheet_epilogue<MODE, RT>(static_cast<const float *>(y), static_cast<float *>(out), acc, ds, scale,
                                      o_base, tid, nv, d.nu);
    if (MODE == 1 || MODE == 2) {
        DF v[1] = {DF{r2, 0.f}};
        double tot[1];
        block_sum_df<1>(v, red, tot);
        if (tid == 0) partials[(size_t)view * d.nu + iu] = tot[0];
    }
}

// rows per thread of the sheet variant (0: use the warp variant)
static int fp_sheet_rows(const VolGeom &v, const DetGeom &d)
{
    if ((size_t)FS_J * (v.nz + 2 * FS_PAD) * sizeof(float) > 96 * 1024) return 0;
    for (int rt : {1, 2, 3, 4, 8})
        if (d.nv <= FS_THREADS * rt) return rt;
    return 0;
}

// rows per lane for a level: the largest of 1, 2, 4 whose warp z span stays
// within one blended segment at the steepest rows
int fp_rows_per_lane(const VolGeom &v, const DetGeom &d)
{
    const double R = sqrt(pow(0.5 * (v.nx + 1) * v.dx, 2) + pow(0.5 * (v.ny + 1) * v.dy, 2));
    const double sc_max = (d.sad + R) * d.dv / ((double)d.sdd * v.dz);  // z voxels per detector row
    int rpl = 1;
    for (int cand : {2, 4})
        if (32.0 * cand * sc_max + 3.0 <= FP_HMAX) rpl = cand;
    return rpl;
}

static dim3 fp_grid(const DetGeom &d, int rpl)
{
    return dim3((d.nu + FP_WARPS - 1) / FP_WARPS, (d.nv + 32 * rpl - 1) / (32 * rpl), d.n_views);
}

int fp_grid_blocks(const DetGeom &d)
{
    const dim3 gr = fp_grid(d, 1);  // the largest grid of either variant
    return (int)std::max<size_t>((size_t)gr.x * gr.y * gr.z, (size_t)d.nu * d.n_views);
}

template <int MODE>
static void launch_mode(const VolGeom &v, const DetGeom &d, const float *vol, const float *y, float *out,
                        const double *d_scale, double *partials, int rpl, cudaStream_t s)
{
    const dim3 block(FP_WARPS * 32);
    if (rpl == 4)
        fp_kernel<MODE, 4><<<fp_grid(d, 4), block, 0, s>>>(v, d, vol, y, out, d_scale, partials);
    else if (rpl == 2)
        fp_kernel<MODE, 2><<<fp_grid(d, 2), block, 0, s>>>(v, d, vol, y, out, d_scale, partials);
    else
        fp_kernel<MODE, 1><<<fp_grid(d, 1), block, 0, s>>>(v, d, vol, y, out, d_scale, partials);
}

int fp_partials_count(const VolGeom &v, const DetGeom &d)
{
    if (fp_sheet_rows(v, d) > 0) return d.nu * d.n_views;
    const dim3 gr = fp_grid(d, fp_rows_per_lane(v, d));
    return (int)(gr.x * gr.y * gr.z);
}

template <int MODE, int RT>
static cudaError_t launch_sheet_rt(const VolGeom &v, const DetGeom &d, const void *vol, const void *y,
                                   void *out, int st, const double *d_scale, double *partials, cudaStream_t s)
{
    const size_t smem = (size_t)FS_J * (v.nz + 2 * FS_PAD) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(fp_sheet_kernel<MODE, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    fp_sheet_kernel<MODE, RT><<<dim3(d.nu, d.n_views), FS_THREADS, smem, s>>>(v, d, vol, y, out, st, d_scale,
                                                                             partials);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_sheet(int rt, const VolGeom &v, const DetGeom &d, const void *vol, const void *y,
                                void *out, int st, const double *d_scale, double *partials, cudaStream_t s)
{
    switch (rt) {
    case 1: return launch_sheet_rt<MODE, 1>(v, d, vol, y, out, st, d_scale, partials, s);
    case 2: return launch_sheet_rt<MODE, 2>(v, d, vol, y, out, st, d_scale, partials, s);
    case 3: return launch_sheet_rt<MODE, 3>(v, d, vol, y, out, st, d_scale, partials, s);
    case 4: return launch_sheet_rt<MODE, 4>(v, d, vol, y, out, st, d_scale, partials, s);
    default: return launch_sheet_rt<MODE, 8>(v, d, vol, y, out, st, d_scale, partials, s);
    }
}

bool fp_supports_storage(const VolGeom &v, const DetGeom &d, int st)
{
    return st == CBCT_STORAGE_F32 || fp_sheet_rows(v, d) > 0;
}

cudaError_t launch_forward_st(const VolGeom &v, const DetGeom &d, const void *vol, const void *y, void *out,
                              int st, const double *d_scale, double *partials, int mode, cudaStream_t s)
{
    const int kid = (mode == 0 || mode == 3) ? K_FP : K_FP_RESID;
    const int rt = fp_sheet_rows(v, d);
    if (rt > 0) {
        launch_begin(kid, s);
        cudaError_t e;
        if (mode == 0)
            e = launch_sheet<0>(rt, v, d, vol, y, out, st, d_scale, partials, s);
        else if (mode == 3)
            e = launch_sheet<3>(rt, v, d, vol, y, out, st, d_scale, partials, s);
        else if (mode == 1)
            e = launch_sheet<1>(rt, v, d, vol, y, out, st, d_scale, partials, s);
        else
            e = launch_sheet<2>(rt, v, d, vol, y, out, st, d_scale, partials, s);
        launch_end(kid, s);
        return e;
    }
    if (st != CBCT_STORAGE_F32) return cudaErrorNotSupported;
    const float *fv = static_cast<const float *>(vol);
    const float *fy = static_cast<const float *>(y);
    float *fo = static_cast<float *>(out);
    const int rpl = fp_rows_per_lane(v, d);
    launch_begin(kid, s);
    if (mode == 0)
        launch_mode<0>(v, d, fv, fy, fo, d_scale, partials, rpl, s);
    else if (mode == 3)
        launch_mode<3>(v, d, fv, fy, fo, d_scale, partials, rpl, s);
    else if (mode == 1)
        launch_mode<1>(v, d, fv, fy, fo, d_scale, partials, rpl, s);
    else
        launch_mode<2>(v, d, fv, fy, fo, d_scale, partials, rpl, s);
    launch_end(kid, s);
    return cudaGetLastError();
}

cudaError_t launch_forward(const VolGeom &v, const DetGeom &d, const float *vol, const float *y,
                           float *out, const double *d_scale, double *partials, int mode,
                           cudaStream_t s)
{
    return launch_forward_st(v, d, vol, y, out, CBCT_STORAGE_F32, d_scale, partials, mode, s);
}

// ---------------------------------------------------------------------------
// storage conversion (grid-stride, one element per thread per step)
// ---------------------------------------------------------------------------
__global__ void convert_kernel(const void *__restrict__ src, int src_st, void *__restrict__ dst, int dst_st,
                               size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        st_st(dst, i, ld_st(src, i, src_st), dst_st);
}

cudaError_t launch_convert(const void *src, int src_st, void *dst, int dst_st, size_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, (size_t)152 * 16);
    launch_begin(K_MISC, s);
    convert_kernel<<<blocks, 256, 0, s>>>(src, src_st, dst, dst_st, n);
    launch_end(K_MISC, s);
    return cudaGetLastError();
}

} // namespace cbct
