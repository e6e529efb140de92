// Device helpers shared by the two matched-transpose kernels (bp.cu, bps.cu):
// the xy footprint of a voxel box on the detector, the staging of a detector
// patch into shared memory, and the warp-uniform dispatch that adds a
// sample's z sums to the voxel columns its bilinear cell touches.
#pragma once

#include "cbct_internal.cuh"

#include <utility>

namespace cbct {

constexpr int BP_G = 4;   // a warp owns a BP_G x BP_G group of voxel columns

struct Box {
    float xlo, xhi, ylo, yhi;
};

__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.f, x); }

// One row T of a z tent window starting at shared address pa: the weight
// 1 - sc |dq + T|, clamped at zero from row CLAMP_FROM on (the rows where it
// can be negative), times the row, into one of two interleaved sums.
template <int CLAMP_FROM, int T>
__device__ __forceinline__ void tent_row(uint32_t pa, float dq, float sc, float &s, float &s2)
{
    float w = __fmaf_rn(-sc, fabsf(dq + (float)T), 1.f);
    if (T >= CLAMP_FROM) w = fmaxf(w, 0.f);
    const float v = lds_off<4 * T>(pa);
    if (T & 1)
        s2 = __fmaf_rn(w, v, s2);
    else
        s = __fmaf_rn(w, v, s);
}

// rows 0 .. W-1; the weight is clamped at zero from row CLAMP_FROM on
template <int CLAMP_FROM, int... T>
__device__ __forceinline__ void tent_rows_imm(uint32_t pa, float dq, float sc, float &s, float &s2,
                                              std::integer_sequence<int, T...>)
{
    (tent_row<CLAMP_FROM, T>(pa, dq, sc, s, s2), ...);
}

// Does sample j of the line touch the BP_G x BP_G group of columns at (A, B)?
// Its cell (floor of the sample's voxel coordinates) must lie in
// [A-1, A+BP_G-1] x [B-1, B+BP_G-1].
__device__ __forceinline__ bool sample_in_group(const VolGeom &g, const RayCol &rc, int j, int A, int B)
{
    float fx, fy;
    sample_xy(g, rc, j, fx, fy);
    const int ra = (int)floorf(fx) - A, rb = (int)floorf(fy) - B;
    return ra >= -1 && ra < BP_G && rb >= -1 && rb < BP_G;
}

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

// Stage rows [s0, s0 + h) x columns [iu0, iu0 + w) of one view's sinogram
// into the column-major patch (pitch hp), zero outside the detector, weighted
// by ds unless the sinogram is pre-weighted.
template <bool PRESCALED, int NWARPS, typename T>
__device__ __forceinline__ void stage_patch(float *patch, const T *__restrict__ src, const VolGeom &g, const DetGeom &d,
                                            int view, int iu0, int s0, int w, int h, int hp, int wid, int lane)
{
    const int nu = d.nu, nv = d.nv;
    for (int r = wid; r < h; r += NWARPS) {
        const int iv = s0 + r;
        const bool in = iv >= 0 && iv < nv;
        for (int cc = lane; cc < w; cc += 32) {
            const int iu = iu0 + cc;
            float val = 0.f;
            if (in) {
                val = ldt(src + (size_t)iv * nu + iu);
                if (!PRESCALED) {
                    const float vl = (((float)iv - d.cv) * d.dv) * g.cols[(size_t)view * nu + iu].inv_lxy;
                    val *= g.drho * sqrtf(1.f + vl * vl);
                }
            }
            patch[cc * hp + r] = val;
        }
    }
}

// The same for a sinogram already weighted by ds and stored FP32, with
// asynchronous 4-byte copies (cp.async): the copies hold no registers and are
// all in flight at once, and rows outside the detector are zero-filled by the
// copy itself (source size 0). Complete with stage_async_wait() and a block
// barrier.
template <int NWARPS>
__device__ __forceinline__ void stage_patch_async(float *patch, const float *__restrict__ src, int nu, int nv, int iu0,
                                                  int s0, int w, int h, int hp, int wid, int lane)
{
    for (int r = wid; r < h; r += NWARPS) {
        const int iv = s0 + r;
        const bool in = iv >= 0 && iv < nv;
        const float *row = src + (size_t)(in ? iv : 0) * nu + iu0;
        for (int cc = lane; cc < w; cc += 32) {
            const unsigned dst = (unsigned)__cvta_generic_to_shared(patch + cc * hp + r);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(row + cc),
                         "r"(in ? 4 : 0)
                         : "memory");
        }
    }
}

__device__ __forceinline__ void stage_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Add a sample's z sums into the (up to four) columns of the warp's G x G
// group that its xy cell (RA, RB) (relative to the group) touches; corners
// outside the group belong to a neighbouring group's warp.
template <int IA, int IB, int ZC>
__device__ __forceinline__ void add_one(float (&acc)[BP_G][BP_G][ZC], float w, const float (&s)[ZC])
{
    if constexpr (IA >= 0 && IA < BP_G && IB >= 0 && IB < BP_G) {
#pragma unroll
        for (int zc = 0; zc < ZC; ++zc) acc[IA][IB][zc] = __fmaf_rn(w, s[zc], acc[IA][IB][zc]);
    }
}

template <int RA, int RB, int ZC>
__device__ __forceinline__ void add_corners(float (&acc)[BP_G][BP_G][ZC], float w00, float w01, float w10,
                                            float w11, const float (&s)[ZC])
{
    add_one<RA, RB, ZC>(acc, w00, s);
    add_one<RA, RB + 1, ZC>(acc, w01, s);
    add_one<RA + 1, RB, ZC>(acc, w10, s);
    add_one<RA + 1, RB + 1, ZC>(acc, w11, s);
}

// Add one sample's z sums to the group's columns its cell touches: a
// warp-uniform switch over the 25 cells of the group and its one-voxel rim
// (cell = (ra + 1) * 5 + (rb + 1), ra and rb relative to the group).
template <int ZC>
__device__ __forceinline__ void add_entry_cell(float (&acc)[BP_G][BP_G][ZC], int cell, float w00, float w01,
                                               float w10, float w11, const float (&sv)[ZC])
{
    switch (cell) {
#define CBCT_CORNER(RA, RB)                                                                         \
    case ((RA) + 1) * (BP_G + 1) + ((RB) + 1):                                                      \
        add_corners<RA, RB, ZC>(acc, w00, w01, w10, w11, sv);                                       \
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

} // namespace cbct
