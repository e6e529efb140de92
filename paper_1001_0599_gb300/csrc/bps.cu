// Matched transpose P^T for grids whose voxel z tents span few detector rows
// (NR <= 8: the finest multigrid levels), sm_103a. It computes the same gather
// as bp.cu -- the exact transpose of the ray-driven projector of fp.cu (the
// matrix view of Sec. II.C.2), every voxel written once, no atomics on data --
// with three changes that cut the work per non-zero weight:
//
// * Exact sample lists. A warp owns a 4 x 4 group of voxel columns; per view
//   its list holds exactly the samples whose bilinear cell touches the group
//   (each line's candidate range is trimmed at both ends by the sample's own
//   cell), so no tent is computed for a sample that adds nothing.
// * Long z columns per lane. Each lane owns ZC z voxels 32 apart (up to 128 z
//   per warp), so the per-sample costs -- the list entry and the dispatch to
//   the touched columns -- are shared by ZC tent sums. The tent window start
//   ceil(q - m) is taken with a round-up add against 1.5 * 2^23, which keeps
//   the float-to-int work on the FMA and integer pipes. Samples whose tent
//   spans fewer rows take a window one row shorter.
// * Stream-K schedule. The (column tile, view) units are cut into equal
//   contiguous ranges, one per resident block, so every SM gets the same
//   number of tile-views. A tile whose views are split between blocks is
//   combined in the kernel: each part writes its sums to scratch, and the
//   last part to arrive (per-tile arrival counter) adds all parts in view
//   order and applies the epilogue. The order is fixed by the schedule, so
//   results are deterministic, and no view-group volume ever reaches DRAM
//   except through the short-lived scratch.
#include "bp_common.cuh"

#ifndef BS_UNIT
#define BS_UNIT 0   // which launch mode this translation unit instantiates (host code in unit 0)
#endif

#include <algorithm>
#include <array>
#include <cmath>
#include <mutex>
#include <utility>
#include <vector>

namespace cbct {

constexpr int BS_TX = 8, BS_TY = 8;        // voxel columns per tile (2 x 2 warp groups)
constexpr int BS_WARPS = 4;
constexpr int BS_THREADS = 32 * BS_WARPS;
#ifndef CBCT_BS_NENT
#define CBCT_BS_NENT 64                   // list entries per warp and batch (build-time tuning)
#endif
constexpr int BS_NENT = CBCT_BS_NENT;
#ifndef CBCT_BS_NENT_BIG
#define CBCT_BS_NENT_BIG 128              // larger batch of the 4-chunk variants, taken where it costs no occupancy (0: never)
#endif
constexpr int BS_NENT_BIG = CBCT_BS_NENT_BIG > 0 ? CBCT_BS_NENT_BIG : CBCT_BS_NENT;
constexpr float BS_ROUND = 12582912.f;     // 1.5 * 2^23: x + BS_ROUND rounds x to an integer
constexpr int BS_ROUND_BITS = 0x4B400000;  // bit pattern of BS_ROUND
constexpr int BS_SHORT = 256;              // entry flag: the tent fits the shorter window
#ifndef CBCT_BS_ZC4_BLOCKS
#define CBCT_BS_ZC4_BLOCKS 4               // resident blocks per SM of the 4-chunk variants (registers)
#endif

struct __align__(16) BsEntry {
    int col;      // patch column offset of the sample's line, minus the first staged row
    int cell;     // (ra + 1) * 5 + (rb + 1), ra, rb in [-1, 3] relative to the group; | BS_SHORT
    float sc, m;  // z voxels per detector row at the sample, and its reciprocal
    float w00, w01, w10, w11;
};

struct BsArgs {
    VolGeom g;
    DetGeom d;
    const void *sino;
    int st;                   // cbct_storage of sino
    int prescaled;            // sino already weighted by ds
    const float *f;
    float *out;
    const double *d_scale;
    float scale_val, kappa;
    double *partials;         // mode 2: one sum of squares per tile
    float *scratch;           // [grid][2][tile voxels]; null: every block takes whole tiles
    unsigned int *counters;   // [tiles], zero at launch (with scratch)
    int cap;                  // staged patch capacity, floats
    int pad;                  // zero rows staged above and below
    int ntx, nty, nzb;        // tiles along x, y and z blocks
};

// One ray-table entry through two 16-byte loads that the compiler may not
// move (a reload is cheaper than keeping the line in registers).
__device__ __forceinline__ RayCol ld_raycol(const RayCol *p)
{
    uint32_t w[8];
    asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
                 : "l"(p));
    asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4 + 16];"
                 : "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
                 : "l"(p));
    RayCol r;
    r.mx = __uint_as_float(w[0]);
    r.my = __uint_as_float(w[1]);
    r.ex = __uint_as_float(w[2]);
    r.ey = __uint_as_float(w[3]);
    r.delta = __uint_as_float(w[4]);
    r.inv_lxy = __uint_as_float(w[5]);
    r.kc = (int)w[6];
    r.jlo = (int16_t)(w[7] & 0xffffu);
    r.jhi = (int16_t)(w[7] >> 16);
    return r;
}

// the block whose unit range [b U / B, (b+1) U / B) holds unit x
__device__ __forceinline__ long long bs_owner(long long x, long long U, long long B) { return ((x + 1) * B - 1) / U; }
__device__ __forceinline__ long long bs_start(long long b, long long U, long long B) { return b * U / B; }

// z tent sum of one sample for one voxel: the sum over the W rows from
// r0 = ceil(q - m) of max(0, 1 - sc |r - q|) R_r, q the row whose sample
// height is the voxel's centre and R the patch column starting at index col.
// Row t of the window lies at r0 + t - q in [t - m, t - m + 1), so its weight
// is non-negative for t <= 2m - 1: a window of W = floor(2m) + 1 rows needs
// the clamp at zero only on its last two rows. The window start is clamped
// into the staged rows [qlo, qhi] (inactive on a correctly staged patch:
// a bounds guard; rows beyond the detector hold zeros).
template <int W, bool CLAMP>
__device__ __forceinline__ float bs_tent(const float *patch, uint32_t pbase, int col, float q, float m, float sc,
                                         float qlo, float qhi)
{
    const float qm = CLAMP ? fminf(fmaxf(q - m, qlo), qhi) : q - m;
    const float tb = __fadd_ru(qm, BS_ROUND);   // BS_ROUND + ceil(qm), exact for |qm| < 2^22
    const int base = col + (__float_as_int(tb) - BS_ROUND_BITS);
    const float dq = (tb - BS_ROUND) - q;
    float s = 0.f, s2 = 0.f;
#if CBCT_LDS_IMM
    tent_rows_imm<W - 2>(pbase + 4u * (uint32_t)base, dq, sc, s, s2, std::make_integer_sequence<int, W>{});
#else
#pragma unroll
    for (int t = 0; t < W; ++t) {
        float w = __fmaf_rn(-sc, fabsf(dq + (float)t), 1.f);
        if (t >= W - 2) w = fmaxf(w, 0.f);
        if (t & 1)
            s2 = __fmaf_rn(w, patch[base + t], s2);
        else
            s = __fmaf_rn(w, patch[base + t], s);
    }
#endif
    return s + s2;
}

template <int MODE, int ZC>
__device__ __forceinline__ void bs_store(const BsArgs &a, const float (&v)[BP_G][BP_G][ZC], int A, int B, int c_base,
                                         int lane, float scale, float &sq)
{
    const VolGeom &g = a.g;
#pragma unroll
    for (int ia = 0; ia < BP_G; ++ia)
#pragma unroll
        for (int ib = 0; ib < BP_G; ++ib) {
            const int x = A + ia, y = B + ib;
            if (x >= g.nx || y >= g.ny) continue;
#pragma unroll
            for (int zc = 0; zc < ZC; ++zc) {
                const int c = c_base + zc * 32 + lane;
                if (c >= g.nz) continue;
                const size_t idx = ((size_t)x * g.ny + y) * g.nz + c;
                if (MODE == 0) {
                    a.out[idx] = v[ia][ib][zc];
                } else if (MODE == 1) {
                    a.out[idx] = __fmaf_rn(-scale, v[ia][ib][zc], __ldg(a.f + idx));
                } else {
                    const float w = a.kappa * v[ia][ib][zc];
                    a.out[idx] = w;
                    sq += w * w;
                }
            }
            __syncwarp();   // keeps the loads of f from being hoisted all at once (registers)
        }
}

// position of a lane's voxel in a tile's scratch partial: [tile x][tile y][z]
__device__ __forceinline__ int bs_local(int warp, int ia, int ib, int zlocal, int tz)
{
    return (((warp & 1) * BP_G + ia) * BS_TY + (warp >> 1) * BP_G + ib) * tz + zlocal;
}

// MODE 0: out = P^T sino; MODE 1: out = f - scale P^T sino; MODE 2: out =
// kappa P^T sino with the tile's sum of squares in partials[tile]. NENT: list
// entries per warp and batch.
template <int MODE, int NR, int ZC, int NENT>
__global__ void __launch_bounds__(BS_THREADS, ZC >= 4 ? CBCT_BS_ZC4_BLOCKS : 5)
bs_kernel(const BsArgs a)
{
    constexpr int TZ = 32 * ZC;
    constexpr int TVOX = BS_TX * BS_TY * TZ;
    extern __shared__ float patch[];
    __shared__ BsEntry s_ent[BS_WARPS][NENT];
    const uint32_t pbase = (uint32_t)__cvta_generic_to_shared(patch);
    __shared__ int s_box[6];
    __shared__ double red[32];
    __shared__ int s_last;

    const VolGeom &g = a.g;
    const DetGeom &d = a.d;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int V = d.n_views;
    const long long T = (long long)a.ntx * a.nty * a.nzb;
    const long long U = T * V;
    const long long NB = gridDim.x;
    const long long u_begin = bs_start(blockIdx.x, U, NB), u_end = bs_start((long long)blockIdx.x + 1, U, NB);
    const float scale = (MODE == 1) ? (a.d_scale ? (float)(*a.d_scale) : a.scale_val) : 0.f;
    const float inv_drho = fast_rcp(g.drho);

    bool first_segment = true;
    for (long long u = u_begin; u < u_end; first_segment = false) {
        const int t = (int)(u / V);
        const int v0 = (int)(u - (long long)t * V);
        const int v1 = (int)min((long long)V, (long long)v0 + (u_end - u));
        const int zb = t % a.nzb, rest = t / a.nzb;
        const int ty = rest % a.nty, tx = rest / a.nty;
        const int a_base = tx * BS_TX, b_base = ty * BS_TY, c_base = zb * TZ;
        const int A = a_base + (warp & 1) * BP_G, B = b_base + (warp >> 1) * BP_G;

        const bool group_live = A < g.nx && B < g.ny;
        float ccz[ZC];   // voxel z index relative to the volume centre, per chunk
#pragma unroll
        for (int zc = 0; zc < ZC; ++zc) ccz[zc] = (float)(c_base + zc * 32 + lane) - g.cz;

        float acc[BP_G][BP_G][ZC];
#pragma unroll
        for (int i = 0; i < BP_G; i++)
#pragma unroll
            for (int k = 0; k < BP_G; k++)
#pragma unroll
                for (int z = 0; z < ZC; z++) acc[i][k][z] = 0.f;

        for (int view = v0; view < v1; ++view) {
            const float2 cs = d.views[view];
            if (threadIdx.x == 0) {
                const float x_first = ((float)a_base - g.cx) * g.dx;
                const float y_first = ((float)b_base - g.cy) * g.dy;
                const Box tile_box{x_first - g.dx, x_first + (float)BS_TX * g.dx, y_first - g.dy,
                                   y_first + (float)BS_TY * g.dy};
                const float z_lo = ((float)c_base - g.cz - 1.f) * g.dz;
                const float z_hi = ((float)(c_base + TZ) - g.cz) * g.dz;
                int iu0, iu1;
                float xr_lo, xr_hi;
                box_u_range(d, cs.x, cs.y, tile_box, iu0, iu1, xr_lo, xr_hi);
                const float m_near = d.sdd / (xr_lo + d.sad), m_far = d.sdd / (xr_hi + d.sad);
                const float q1 = z_lo * m_near, q2 = z_lo * m_far, q3 = z_hi * m_near, q4 = z_hi * m_far;
                const float vmin = fminf(fminf(q1, q2), fminf(q3, q4));
                const float vmax = fmaxf(fmaxf(q1, q2), fmaxf(q3, q4));
                const int iv0 = max((int)floorf(vmin * d.inv_dv + d.cv) - 1, 0);
                const int iv1 = min((int)ceilf(vmax * d.inv_dv + d.cv) + 1, d.nv - 1);
                const int s0 = iv0 - a.pad, s1 = iv1 + a.pad;
                const int w = iu1 - iu0 + 1, hp = (s1 - s0 + 1) | 1;
                s_box[0] = iu0;
                s_box[1] = iu1;
                s_box[2] = s0;
                s_box[3] = s1;
                s_box[4] = hp;
                // the host sized the patch for every tile and view with two pixels of
                // slack; the size test only keeps shared memory in bounds
                s_box[5] = (iu1 >= iu0 && iv1 >= iv0 && w * hp <= a.cap) ? 1 : 0;
            }
            __syncthreads();
            const int iu0 = s_box[0], iu1 = s_box[1], s0 = s_box[2], s1 = s_box[3], hp = s_box[4];
            if (!s_box[5]) {
                __syncthreads();
                continue;
            }
            {
                const int w = iu1 - iu0 + 1, h = s1 - s0 + 1;
                const size_t src = (size_t)view * d.nv * d.nu;
                if (a.prescaled && a.st == CBCT_STORAGE_F32) {
                    stage_patch_async<BS_WARPS>(patch, static_cast<const float *>(a.sino) + src, d.nu, d.nv, iu0, s0,
                                                w, h, hp, warp, lane);
                    stage_async_wait();
                } else if (a.prescaled) {
                    if (a.st == CBCT_STORAGE_BF16)
                        stage_patch<true, BS_WARPS>(patch, static_cast<const __nv_bfloat16 *>(a.sino) + src, g, d,
                                                    view, iu0, s0, w, h, hp, warp, lane);
                    else if (a.st == CBCT_STORAGE_F16)
                        stage_patch<true, BS_WARPS>(patch, static_cast<const __half *>(a.sino) + src, g, d, view,
                                                    iu0, s0, w, h, hp, warp, lane);
                    else
                        stage_patch<true, BS_WARPS>(patch, static_cast<const float *>(a.sino) + src, g, d, view,
                                                    iu0, s0, w, h, hp, warp, lane);
                } else {
                    if (a.st == CBCT_STORAGE_BF16)
                        stage_patch<false, BS_WARPS>(patch, static_cast<const __nv_bfloat16 *>(a.sino) + src, g, d,
                                                     view, iu0, s0, w, h, hp, warp, lane);
                    else if (a.st == CBCT_STORAGE_F16)
                        stage_patch<false, BS_WARPS>(patch, static_cast<const __half *>(a.sino) + src, g, d, view,
                                                     iu0, s0, w, h, hp, warp, lane);
                    else
                        stage_patch<false, BS_WARPS>(patch, static_cast<const float *>(a.sino) + src, g, d, view,
                                                     iu0, s0, w, h, hp, warp, lane);
                }
            }
            __syncthreads();

            if (group_live) {   // warp-uniform
                const float xA = ((float)A - g.cx) * g.dx, yB = ((float)B - g.cy) * g.dy;
                const Box gbox{xA - g.dx, xA + (float)BP_G * g.dx, yB - g.dy, yB + (float)BP_G * g.dy};
                int ju0, ju1;
                float dlo, dhi;
                box_u_range(d, cs.x, cs.y, gbox, ju0, ju1, dlo, dhi);
                ju0 = max(ju0, iu0);
                ju1 = min(ju1, iu1);
                const float qlo = (float)s0;
                const float qhi_long = (float)(s1 - NR + 1), qhi_short = (float)(s1 - NR + 2);
                for (int iub = ju0; iub <= ju1; iub += 32) {
                    const int iu = iub + lane;
                    int jl = 0, jh = -1;
                    RayCol rc{};
                    if (iu <= ju1) {
                        rc = g.cols[(size_t)view * d.nu + iu];
                        float tlo = -3.0e38f, thi = 3.0e38f;
                        bool hit = true;
                        if (fabsf(rc.ex) > 1e-20f) {
                            const float inv = fast_rcp(rc.ex);
                            const float t1 = (gbox.xlo - rc.mx) * inv, t2 = (gbox.xhi - rc.mx) * inv;
                            tlo = fmaxf(tlo, fminf(t1, t2));
                            thi = fminf(thi, fmaxf(t1, t2));
                        } else if (!(rc.mx > gbox.xlo && rc.mx < gbox.xhi)) {
                            hit = false;
                        }
                        if (fabsf(rc.ey) > 1e-20f) {
                            const float inv = fast_rcp(rc.ey);
                            const float t1 = (gbox.ylo - rc.my) * inv, t2 = (gbox.yhi - rc.my) * inv;
                            tlo = fmaxf(tlo, fminf(t1, t2));
                            thi = fminf(thi, fmaxf(t1, t2));
                        } else if (!(rc.my > gbox.ylo && rc.my < gbox.yhi)) {
                            hit = false;
                        }
                        if (hit && tlo < thi) {
                            jl = max((int)ceilf((tlo + rc.delta) * inv_drho) - 1, (int)rc.jlo);
                            jh = min((int)floorf((thi + rc.delta) * inv_drho) + 1, (int)rc.jhi);
                            // the samples touching the group are contiguous along the line:
                            // trim the candidate range to them
                            while (jl <= jh && !sample_in_group(g, rc, jl, A, B)) ++jl;
                            while (jh >= jl && !sample_in_group(g, rc, jh, A, B)) --jh;
                        }
                    }
                    const int cnt = max(jh - jl + 1, 0);
                    int incl = cnt;   // inclusive warp scan of the counts
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int v2 = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += v2;
                    }
                    const int total = __shfl_sync(0xffffffffu, incl, 31);
                    const int first = incl - cnt;
                    const int col_off = (iu - iu0) * hp - s0;
                    for (int b0 = 0; b0 < total; b0 += NENT) {
                        const int lo = max(first, b0), hi = min(first + cnt, b0 + NENT);
                        // the line is read again per batch so that it holds no registers
                        // while the batch is processed
                        const RayCol rc2 = lo < hi ? ld_raycol(g.cols + (size_t)view * d.nu + iu) : RayCol{};
                        const float sc_base = d.dv * rc2.inv_lxy * g.inv_dz;
                        for (int e = lo; e < hi; ++e) {
                            const int j = jl + (e - first);
                            float fx, fy;
                            sample_xy(g, rc2, j, fx, fy);
                            const float a0f = floorf(fx), b0f = floorf(fy);
                            const int ra = (int)a0f - A, rb = (int)b0f - B;
                            const float wx1 = fx - a0f, wy1 = fy - b0f;
                            const float wx0 = 1.f - wx1, wy0 = 1.f - wy1;
                            const float sc = sample_rho(g, rc2, j) * sc_base;
                            const float m = __frcp_rn(sc);
                            BsEntry en;
                            // rows strictly inside the tent: at most floor(2m) + 1
                            en.cell = ((ra + 1) * (BP_G + 1) + (rb + 1)) |
                                      ((2.0002f * m < (float)(NR - 1)) ? BS_SHORT : 0);
                            en.col = col_off;
                            en.sc = sc;
                            en.m = m;
                            en.w00 = wx0 * wy0;
                            en.w01 = wx0 * wy1;
                            en.w10 = wx1 * wy0;
                            en.w11 = wx1 * wy1;
                            s_ent[warp][e - b0] = en;
                        }
                        __syncwarp();
                        const int nb = min(NENT, total - b0);
                        for (int e = 0; e < nb; ++e) {
                            // the entry's geometry first; its weights only once the tents are done
                            const float4 h = *reinterpret_cast<const float4 *>(&s_ent[warp][e]);
                            const int col = __float_as_int(h.x), cell = __float_as_int(h.y);
                            const float sc = h.z, m = h.w;
                            float sv[ZC];
                            if (cell & BS_SHORT) {
#pragma unroll
                                for (int zc = 0; zc < ZC; ++zc)
                                    sv[zc] = bs_tent<NR - 1, true>(patch, pbase, col, __fmaf_rn(ccz[zc], m, d.cv), m, sc, qlo,
                                                                   qhi_short);
                            } else {
#pragma unroll
                                for (int zc = 0; zc < ZC; ++zc)
                                    sv[zc] = bs_tent<NR, true>(patch, pbase, col, __fmaf_rn(ccz[zc], m, d.cv), m, sc, qlo,
                                                               qhi_long);
                            }
                            const float4 wq = *reinterpret_cast<const float4 *>(&s_ent[warp][e].w00);
                            add_entry_cell<ZC>(acc, cell & 255, wq.x, wq.y, wq.z, wq.w, sv);
                        }
                        __syncwarp();
                    }
                }
            }
            __syncthreads();
        }

        // epilogue of the tile segment [v0, v1): a whole tile is stored at once; a
        // part goes to scratch, and the last part to arrive sums all parts
        bool store = (v0 == 0 && v1 == V) || a.scratch == nullptr;
        if (!store) {
            const long long tv0 = (long long)t * V;
            const long long bf = bs_owner(tv0, U, NB);
            const int nparts = (int)(bs_owner(tv0 + V - 1, U, NB) - bf + 1);
            float *mine = a.scratch + ((size_t)blockIdx.x * 2 + (first_segment ? 0 : 1)) * TVOX;
#pragma unroll
            for (int ia = 0; ia < BP_G; ++ia)
#pragma unroll
                for (int ib = 0; ib < BP_G; ++ib)
#pragma unroll
                    for (int zc = 0; zc < ZC; ++zc)
                        __stcg(mine + bs_local(warp, ia, ib, zc * 32 + lane, TZ), acc[ia][ib][zc]);
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) s_last = (atomicAdd(a.counters + t, 1u) == (unsigned)(nparts - 1));
            __syncthreads();
            store = s_last != 0;
            if (store) {   // block-uniform: add all parts in view order
                __threadfence();
                // blocks after the first start inside the tile (their first segment);
                // the first block's segment is its first only if it starts at the tile
                const int w0 = (bs_start(bf, U, NB) == tv0) ? 0 : 1;
                const float *part0 = a.scratch + ((size_t)bf * 2 + w0) * TVOX;
                const float *part1 = a.scratch + ((size_t)bf + 1) * 2 * TVOX;   // parts p >= 1: 2 TVOX apart
#pragma unroll
                for (int ia = 0; ia < BP_G; ++ia)
#pragma unroll
                    for (int ib = 0; ib < BP_G; ++ib)
#pragma unroll
                        for (int zc = 0; zc < ZC; ++zc) {
                            const int loc = bs_local(warp, ia, ib, zc * 32 + lane, TZ);
                            float s = __ldcg(part0 + loc);
                            for (int p = 1; p < nparts; ++p) s += __ldcg(part1 + (size_t)(p - 1) * 2 * TVOX + loc);
                            acc[ia][ib][zc] = s;
                        }
                if (threadIdx.x == 0) a.counters[t] = 0u;   // ready for the next launch
            }
        }
        if (store) {   // block-uniform
            float sq = 0.f;
            bs_store<MODE, ZC>(a, acc, A, B, c_base, lane, scale, sq);
            if (MODE == 2) {
                DF v[1] = {DF{sq, 0.f}};
                double tot[1];
                block_sum_df<1>(v, red, tot);
                if (threadIdx.x == 0) a.partials[t] = tot[0];
            }
        }
        __syncthreads();
        u += v1 - v0;
    }
}

template <int MODE, int NR, int ZC, int NENT>
static cudaError_t bs_prepare(size_t smem, int *occ)
{
    cudaError_t e = cudaFuncSetAttribute(bs_kernel<MODE, NR, ZC, NENT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(bs_kernel<MODE, NR, ZC, NENT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    if (occ)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, bs_kernel<MODE, NR, ZC, NENT>, BS_THREADS, smem);
    return cudaSuccess;
}

template <int MODE, int NR, int ZC, int NENT>
static cudaError_t bs_go(int grid, size_t smem, cudaStream_t s, const BsArgs &a, int *occ)
{
    cudaError_t e = bs_prepare<MODE, NR, ZC, NENT>(smem, occ);
    if (e != cudaSuccess || occ) return e;
    bs_kernel<MODE, NR, ZC, NENT><<<grid, BS_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

// nent: list batch (BS_NENT, or BS_NENT_BIG for the 4-chunk variants)
template <int MODE>
cudaError_t bs_dispatch(int nr, int zc, int nent, int grid, size_t smem, cudaStream_t s, const BsArgs &a, int *occ)
{
#define CBCT_BS_CASE(NRV)                                                                           \
    case NRV:                                                                                       \
        if (zc == 1) return bs_go<MODE, NRV, 1, BS_NENT>(grid, smem, s, a, occ);                    \
        if (zc == 2) return bs_go<MODE, NRV, 2, BS_NENT>(grid, smem, s, a, occ);                    \
        if (nent == BS_NENT_BIG) return bs_go<MODE, NRV, 4, BS_NENT_BIG>(grid, smem, s, a, occ);    \
        return bs_go<MODE, NRV, 4, BS_NENT>(grid, smem, s, a, occ);
    switch (nr) {
        CBCT_BS_CASE(4)
        CBCT_BS_CASE(5)
        CBCT_BS_CASE(6)
        CBCT_BS_CASE(8)
    default:
        return cudaErrorInvalidValue;
    }
#undef CBCT_BS_CASE
}

#define CBCT_BS_SIG(MODE) \
    cudaError_t bs_dispatch<MODE>(int, int, int, int, size_t, cudaStream_t, const BsArgs &, int *)
#if BS_UNIT == 0
extern template CBCT_BS_SIG(1);
extern template CBCT_BS_SIG(2);
template CBCT_BS_SIG(0);
#elif BS_UNIT == 1
template CBCT_BS_SIG(1);
#else
template CBCT_BS_SIG(2);
#endif
#undef CBCT_BS_SIG

#if BS_UNIT == 0
// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// Tent window for the grid (0: the grid needs bp.cu's kernel). The shorter
// window (nr - 1 rows) leaves its first nr - 4 rows unclamped, which needs
// every sample's m = 1/sc >= (nr - 3) / 2; the smallest m on the grid belongs
// to the sample farthest from the source on the central detector column,
// sc = (sad + R) dv / (sdd dz), R the radius of the volume's support.
static int bs_nr(const VolGeom &v, const DetGeom &d)
{
    const int need = bp_rows_needed(v, d);
    const double R = std::sqrt(std::pow(0.5 * (v.nx + 1) * v.dx, 2) + std::pow(0.5 * (v.ny + 1) * v.dy, 2));
    const double m_min = ((double)d.sdd * v.dz) / ((d.sad + R + 2.0 * v.drho) * d.dv) * (1.0 - 1e-4);
    for (int nr : {4, 5, 6, 8})
        if (need <= nr) return m_min >= 0.5 * (nr - 3) ? nr : 0;
    return 0;
}

#ifndef CBCT_BS_ZC_MAX
#define CBCT_BS_ZC_MAX 4   // most z chunks per lane (build-time tuning: 1, 2 or 4)
#endif

int bs_zc(const VolGeom &v) { return v.nz <= 32 || CBCT_BS_ZC_MAX == 1 ? 1 : (v.nz <= 64 || CBCT_BS_ZC_MAX == 2 ? 2 : 4); }

static constexpr long BS_CAP_MAX = 40L * 1024L;   // floats of staged patch (160 KB)

int bs_patch_floats(const VolGeom &v, const DetGeom &d, const double *angles)
{
    const int nr = bs_nr(v, d);
    if (nr == 0) return 0;
    const long need = bp_patch_floats_tile(v, d, angles, 32 * bs_zc(v), nr);
    return need <= BS_CAP_MAX ? (int)need : 0;
}

bool bs_usable(const VolGeom &v, const DetGeom &d) { return v.bs_cap > 0 && bs_nr(v, d) > 0; }

static int bs_tiles(const VolGeom &v)
{
    const int tz = 32 * bs_zc(v);
    return ((v.nx + BS_TX - 1) / BS_TX) * ((v.ny + BS_TY - 1) / BS_TY) * ((v.nz + tz - 1) / tz);
}

int bs_partials_count(const VolGeom &v) { return bs_tiles(v); }

static int bs_sm_count(int dev)
{
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

static int bs_occupancy(const VolGeom &v, const DetGeom &d, int mode, int nent)
{
    int occ = 0;
    BsArgs a{};
    const size_t smem = (size_t)v.bs_cap * sizeof(float);
    cudaError_t e;
    if (mode == 0)
        e = bs_dispatch<0>(bs_nr(v, d), bs_zc(v), nent, 1, smem, 0, a, &occ);
    else if (mode == 1)
        e = bs_dispatch<1>(bs_nr(v, d), bs_zc(v), nent, 1, smem, 0, a, &occ);
    else
        e = bs_dispatch<2>(bs_nr(v, d), bs_zc(v), nent, 1, smem, 0, a, &occ);
    if (e != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 0;
    }
    return occ;
}

// Launch plan of the grid's variant (per device, geometry shape and mode):
// the list batch -- the larger one where it leaves as many resident blocks
// per SM as the smaller one (measured: cubic finest grid 7.39 -> 7.15 ms with
// both at 4 blocks per SM; where the larger batch costs a block per SM, the
// paper finest grid ran 3.89 -> 4.28 ms) -- and the stream-K grid, its
// resident blocks.
struct BsPlan {
    int blocks, nent;
};

static BsPlan bs_plan(const VolGeom &v, const DetGeom &d, int mode)
{
    static std::mutex mu;
    static std::vector<std::pair<std::array<int, 8>, BsPlan>> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const std::array<int, 8> key{dev, v.nx, v.ny, v.nz, d.nu, d.nv, v.bs_cap, mode};
    {
        std::lock_guard<std::mutex> lk(mu);
        for (const auto &kv : cache)
            if (kv.first == key) return kv.second;
    }
    int nent = BS_NENT, occ = bs_occupancy(v, d, mode, BS_NENT);
    if (BS_NENT_BIG != BS_NENT && bs_zc(v) == 4) {
        const int occ_big = bs_occupancy(v, d, mode, BS_NENT_BIG);
        if (occ_big >= occ && occ_big > 0) {
            nent = BS_NENT_BIG;
            occ = occ_big;
        }
    }
    const BsPlan plan{std::max(occ, 1) * bs_sm_count(dev), nent};
    std::lock_guard<std::mutex> lk(mu);
    cache.emplace_back(key, plan);
    return plan;
}

static int bs_grid(const VolGeom &v, const DetGeom &d, int mode)
{
    const long long units = (long long)bs_tiles(v) * d.n_views;
    return (int)std::min<long long>(bs_plan(v, d, mode).blocks, units);
}

// scratch floats of a stream-K launch: two tile partials per block
size_t bs_scratch_floats(const VolGeom &v, const DetGeom &d)
{
    if (!bs_usable(v, d)) return 0;
    int g = 0;
    for (int mode = 0; mode < 3; ++mode) g = std::max(g, bs_grid(v, d, mode));
    return (size_t)g * 2 * BS_TX * BS_TY * 32 * bs_zc(v);
}

size_t bs_counter_count(const VolGeom &v, const DetGeom &d) { return bs_usable(v, d) ? (size_t)bs_tiles(v) : 0; }

cudaError_t launch_bs(const VolGeom &v, const DetGeom &d, const void *sino, int st, const float *f, float *out,
                      const double *d_scale, double scale_val, double kappa, double *partials, int mode,
                      int prescaled, float *scratch, unsigned int *counters, cudaStream_t s)
{
    BsArgs a{};
    a.g = v;
    a.d = d;
    a.sino = sino;
    a.st = st;
    a.prescaled = prescaled;
    a.f = f;
    a.out = out;
    a.d_scale = d_scale;
    a.scale_val = (float)scale_val;
    a.kappa = (float)kappa;
    a.partials = partials;
    a.cap = v.bs_cap;
    a.pad = bs_nr(v, d);
    const int zc = bs_zc(v), tz = 32 * zc;
    a.ntx = (v.nx + BS_TX - 1) / BS_TX;
    a.nty = (v.ny + BS_TY - 1) / BS_TY;
    a.nzb = (v.nz + tz - 1) / tz;
    int grid = bs_tiles(v);
    if (scratch && counters) {
        grid = bs_grid(v, d, mode);
        a.scratch = scratch;
        a.counters = counters;
        cudaError_t e = cudaMemsetAsync(counters, 0, sizeof(unsigned int) * (size_t)bs_tiles(v), s);
        if (e != cudaSuccess) return e;
    }
    const size_t smem = (size_t)v.bs_cap * sizeof(float);
    const int nent = bs_plan(v, d, mode).nent;
    if (mode == 0) return bs_dispatch<0>(a.pad, zc, nent, grid, smem, s, a, nullptr);
    if (mode == 1) return bs_dispatch<1>(a.pad, zc, nent, grid, smem, s, a, nullptr);
    return bs_dispatch<2>(a.pad, zc, nent, grid, smem, s, a, nullptr);
}

#endif // BS_UNIT == 0

} // namespace cbct
