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
#include "bp_common.cuh"

#ifndef BP_MODE_UNIT
#define BP_MODE_UNIT 0
#endif

#include <algorithm>
#include <array>
#include <cmath>
#include <mutex>
#include <utility>
#include <vector>

namespace cbct {

constexpr int BP_GX = 2, BP_GY = 2;   // groups per block along x, y
constexpr int BP_TX = BP_G * BP_GX, BP_TY = BP_G * BP_GY;   // voxel columns per block
constexpr int BP_WARPS = BP_GX * BP_GY;
constexpr int BP_MAX_ROWS = 64;       // runtime row-loop bound (generic variant)

// One sample of a warp's footprint list: xy cell relative to the group in the
// low 8 bits and the detector column above them (-1: outside the group),
// patch column offset, bilinear corner weights, z voxels per detector row
// (sc) and its reciprocal.
struct __align__(16) SampleEntry {
    int cell, col;
    float w00, w01, w10, w11, sc, m;
};
constexpr int BP_ENTRIES = 96;    // entries per warp and batch

template <int ZC>
__device__ __forceinline__ void add_entry(float (&acc)[BP_G][BP_G][ZC], const SampleEntry &en, const float (&sv)[ZC])
{
    add_entry_cell<ZC>(acc, en.cell & 255, en.w00, en.w01, en.w10, en.w11, sv);
}

// Warps per column group for a row count NR: voxels whose z tent spans many
// detector rows come with tall staged patches and so with few blocks per SM;
// more warps per group then keep the SM busy.
__host__ __device__ constexpr int bp_split_for(int nr) { return (nr == 0 || nr > 16) ? 4 : (nr > 8 ? 2 : 1); }

struct BpLaunch {
    VolGeom v;
    DetGeom d;
    const void *sino;
    int st;      // cbct_storage of sino
    const float *f;
    float *out;
    const double *d_scale;
    float scale_val, kappa;
    double *partials;
    int cap, zblocks, vpg;
    int split;   // warps per column group
    int *occ;    // non-null: report resident blocks per SM of the selected variant instead of launching
};

template <int MODE, bool P>
cudaError_t bp_dispatch(int zc, int nr, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const BpLaunch &L);

// The z tent sum of one sample for one lane's voxel c: sum over the rows r
// whose sample height is within one dz of z_c of (1 - sc |r - q|) * row value,
// rows inside the staged patch from shared memory and the others from the
// sinogram in global memory (blocks whose patch did not fit, or rows beyond
// it); the values are weighted by ds unless the sinogram is pre-weighted.
template <bool PRESCALED>
__device__ __forceinline__ float tent_rows_global(const DetGeom &d, const VolGeom &g, const float *pcol,
                                                  const void *gsino, size_t gbase, int st, const RayCol &rc,
                                                  bool staged, int s0, int s1, float q, float m, float sc)
{
    float s = 0.f;
    const int r_lo = max((int)ceilf(q - m), 0);
    const int r_hi = min(min((int)floorf(q + m), d.nv - 1), r_lo + BP_MAX_ROWS);
    for (int r = r_lo; r <= r_hi; ++r) {
        const float w = fmaxf(__fmaf_rn(-sc, fabsf((float)r - q), 1.f), 0.f);
        float val;
        if (staged && r >= s0 && r <= s1) {
            val = pcol[r];
        } else {
            val = ld_st(gsino, gbase + (size_t)r * d.nu, st);
            if (!PRESCALED) {
                const float vl = (((float)r - d.cv) * d.dv) * rc.inv_lxy;
                val *= g.drho * sqrtf(1.f + vl * vl);
            }
        }
        s = __fmaf_rn(w, val, s);
    }
    return s;
}

// Staged variant only (no global fallback): NR rows from the padded patch.
template <int NR>
__device__ __forceinline__ float tent_rows_staged(const float *pcol, uint32_t pa_col, bool staged, int s0, int s1,
                                                  float q, float m, float sc)
{
    float s = 0.f, s2 = 0.f;
    if (NR > 0 && staged) {
        int r0 = (int)ceilf(q - m);
        r0 = min(max(r0, s0), s1 - NR + 1);
        const float dq = (float)r0 - q;
#if CBCT_LDS_IMM
        tent_rows_imm<0>(pa_col + 4u * (uint32_t)r0, dq, sc, s, s2, std::make_integer_sequence<int, (NR > 0 ? NR : 1)>{});
        return s + s2;
    }
    return s + s2;
#else
        const float *p = pcol + r0;
#pragma unroll
        for (int t = 0; t < (NR > 0 ? NR : 1); ++t) {
            const float w = fmaxf(__fmaf_rn(-sc, fabsf(dq + (float)t), 1.f), 0.f);
            if (t & 1)
                s2 = __fmaf_rn(w, p[t], s2);
            else
                s = __fmaf_rn(w, p[t], s);
        }
    }
    return s + s2;
#endif
}

// NR > 0: rows per (lane, sample) fully unrolled; NR == 0: runtime loop.
// Block: BP_WARPS x SPLIT warps. Warp w owns the BP_G x BP_G group of voxel
// columns w % BP_WARPS and the block's 32*ZC z values (one per lane and
// chunk); the SPLIT warps of a group take every SPLIT-th sample of its
// footprint and add their sums at the end (coarse grids, whose large detector
// patches leave room for few blocks per SM). With a view split (MODE 3) block z
// index = z block + zblocks * view group, and the block adds only its group's
// views and writes the raw sums to out + group * N_vox.
// Interval sums for long tents. Rows whose sample height lies between voxel
// centres k and k+1 (rows ceil(q_k) <= r < ceil(q_k1), q_k the row at height k
// and q_k1 the one at height k+1, evaluated exactly as the neighbouring lane
// evaluates its own, so that the intervals partition the rows) give
// A_k = sum R_r and B_k = sum (r - q_k) sc R_r, and the tent sum of voxel c is
// B_{c-1} + A_c - B_c: each row is read once per voxel pair instead of twice.
// The window of NI rows starts at ceil(q_k), clamped into the staged range;
// rows it then covers below the interval are zero padding.
template <int NI>
__device__ __forceinline__ void interval_sums(const float *pcol, int s0, int s1, float q, float qn, float sc,
                                              float &A, float &B)
{
    const int lo = (int)ceilf(q), hi = (int)ceilf(qn);
    const int w0 = min(max(lo, s0), s1 - NI + 1);
    const int n = hi - w0;   // window rows inside the interval: t < n
    const float x0 = ((float)w0 - q) * sc;
    float a = 0.f, b = 0.f, a2 = 0.f, b2 = 0.f;
    // (rows read only inside the interval: unconditional immediate-offset
    // reads with a select measured 5 % slower on the coarsest cubic grid)
    const float *p = pcol + w0;
#pragma unroll
    for (int t = 0; t < NI; ++t) {
        const float x = __fmaf_rn((float)t, sc, x0);
        const float v = t < n ? p[t] : 0.f;
        if (t & 1) {
            a2 += v;
            b2 = __fmaf_rn(x, v, b2);
        } else {
            a += v;
            b = __fmaf_rn(x, v, b);
        }
    }
    A = a + a2;
    B = b + b2;
}

// samples taken together in the transpose's main loop (short tents)
#ifndef CBCT_BP_STEP
#define CBCT_BP_STEP 2
#endif
constexpr int BP_STEP = CBCT_BP_STEP;

template <int MODE, bool PRESCALED, int NR, int ZC, int SPLIT>
__global__ void __launch_bounds__(BP_WARPS * 32 * SPLIT, SPLIT == 1 ? 5 : (SPLIT == 2 ? 2 : 1))
bp_kernel(VolGeom g, DetGeom d, const void *__restrict__ sino, int st, const float *__restrict__ f,
          float *__restrict__ out, const double *__restrict__ d_scale, float scale_val, float kappa,
          double *__restrict__ partials, int patch_cap, int pad, int zblocks, int views_per_group)
{
    constexpr int BP_ZC = ZC;
    constexpr int BP_TZ = 32 * ZC;
    constexpr int NWARPS = BP_WARPS * SPLIT;
    constexpr int NENT = BP_ENTRIES / SPLIT;   // list slots per warp and batch
    extern __shared__ float patch[];
    const uint32_t pbase = (uint32_t)__cvta_generic_to_shared(patch);
    __shared__ int s_box[6];
    __shared__ double red[32];
    __shared__ SampleEntry s_ent[BP_WARPS * BP_ENTRIES];

    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int warp = wid % BP_WARPS, part = wid / BP_WARPS;
    const int zb = (int)blockIdx.z % zblocks, vg = (int)blockIdx.z / zblocks;
    const int a_base = blockIdx.x * BP_TX, b_base = blockIdx.y * BP_TY, c_base = zb * BP_TZ;
    const int nx = g.nx, ny = g.ny, nz = g.nz, nu = d.nu, nv = d.nv;
    const int view_begin = vg * views_per_group;
    const int view_end = min(d.n_views, view_begin + views_per_group);
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

    for (int view = view_begin; view < view_end; ++view) {
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
            const size_t src = (size_t)view * nv * nu;
            if (PRESCALED && st == CBCT_STORAGE_F32) {
                stage_patch_async<NWARPS>(patch, static_cast<const float *>(sino) + src, nu, nv, iu0, s0, w, h, hp,
                                          wid, lane);
                stage_async_wait();
            } else if (st == CBCT_STORAGE_BF16)
                stage_patch<PRESCALED, NWARPS>(patch, static_cast<const __nv_bfloat16 *>(sino) + src, g, d, view,
                                              iu0, s0, w, h, hp, wid, lane);
            else if (st == CBCT_STORAGE_F16)
                stage_patch<PRESCALED, NWARPS>(patch, static_cast<const __half *>(sino) + src, g, d, view, iu0, s0,
                                              w, h, hp, wid, lane);
            else
                stage_patch<PRESCALED, NWARPS>(patch, static_cast<const float *>(sino) + src, g, d, view, iu0, s0,
                                              w, h, hp, wid, lane);
        }
        __syncthreads();

        if (group_live) {  // warp-uniform
            int ju0, ju1;
            float dlo, dhi;
            box_u_range(d, cs.x, cs.y, gbox, ju0, ju1, dlo, dhi);
            ju0 = max(ju0, iu0);
            ju1 = min(ju1, iu1);
            SampleEntry *ent = s_ent + wid * NENT;
            const float inv_drho = fast_rcp(g.drho);
            // lanes take detector columns; each enumerates its line's samples in
            // the group's footprint (entries ordered by column, then sample)
            for (int iub = ju0; iub <= ju1; iub += 32) {
                const int iu = iub + lane;
                int jl = 0, jh = -1;
                RayCol rc{};
                if (iu <= ju1) {
                    rc = g.cols[(size_t)view * nu + iu];
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
                        // the samples touching the group are contiguous along the line: trim
                        // the candidate range to them
                        while (jl <= jh && !sample_in_group(g, rc, jl, A, B)) ++jl;
                        while (jh >= jl && !sample_in_group(g, rc, jh, A, B)) --jh;
                    }
                }
                const int cnt = max(jh - jl + 1, 0);
                int incl = cnt;  // inclusive warp scan of the counts
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v2 = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v2;
                }
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                const int first = incl - cnt;
                const float sc_base = d.dv * rc.inv_lxy * g.inv_dz;
                const int col_off = (iu - iu0) * hp - s0;
                for (int b0 = 0; b0 < total; b0 += NENT * SPLIT) {
                    // fill this warp's entries of the batch window (every SPLIT-th one)
                    const int lo = max(first, b0), hi = min(first + cnt, b0 + NENT * SPLIT);
                    for (int e = lo; e < hi; ++e) {
                        if (SPLIT > 1 && (e - b0) % SPLIT != part) continue;
                        const int j = jl + (e - first);
                        float fx, fy;
                        sample_xy(g, rc, j, fx, fy);
                        const float a0f = floorf(fx), b0f = floorf(fy);
                        const int ra = (int)a0f - A, rb = (int)b0f - B;
                        const float wx1 = fx - a0f, wy1 = fy - b0f;
                        const float wx0 = 1.f - wx1, wy0 = 1.f - wy1;
                        const float sc = sample_rho(g, rc, j) * sc_base;
                        SampleEntry en;
                        en.cell = (ra < -1 || ra >= BP_G || rb < -1 || rb >= BP_G)
                                      ? -1
                                      : ((ra + 1) * (BP_G + 1) + (rb + 1)) | (iu << 8);
                        en.col = col_off;
                        en.w00 = wx0 * wy0;
                        en.w01 = wx0 * wy1;
                        en.w10 = wx1 * wy0;
                        en.w11 = wx1 * wy1;
                        en.sc = sc;
                        en.m = fast_rcp(sc);
                        ent[(e - b0) / SPLIT] = en;
                    }
                    __syncwarp();
                    const int nwin = min(NENT * SPLIT, total - b0);
                    const int nb = (nwin - part + SPLIT - 1) / SPLIT;
                    int e = 0;
                    if (BP_STEP > 1 && SPLIT == 1 && NR > 0 && staged) {
                        // BP_STEP samples per step: their tents are independent, which
                        // multiplies the arithmetic chains in flight (entries outside
                        // the group still read inside the patch and are dropped).
                        // Short tents only: the long-tent variants (several warps per
                        // group) measured slower this way.
                        for (; e + BP_STEP - 1 < nb; e += BP_STEP) {
                            SampleEntry es[BP_STEP];
                            float sv[BP_STEP][BP_ZC];
#pragma unroll
                            for (int u = 0; u < BP_STEP; ++u) es[u] = ent[e + u];
#pragma unroll
                            for (int zc = 0; zc < BP_ZC; ++zc) {
                                const float cz = (float)(c_base + zc * 32 + lane) - g.cz;
#pragma unroll
                                for (int u = 0; u < BP_STEP; ++u)
                                    sv[u][zc] = tent_rows_staged<NR>(patch + es[u].col, pbase + 4u * (uint32_t)es[u].col,
                                                                     staged, s0, s1,
                                                                     d.cv + cz * es[u].m, es[u].m, es[u].sc);
                            }
#pragma unroll
                            for (int u = 0; u < BP_STEP; ++u)
                                if (es[u].cell >= 0) add_entry<ZC>(acc, es[u], sv[u]);
                        }
                    }
                    for (; e < nb; ++e) {
                        const SampleEntry en = ent[e];
                        if (en.cell < 0) continue;  // uniform
                        const float *pcol = patch + en.col;
                        const uint32_t pa_col = pbase + 4u * (uint32_t)en.col;
                        float sv[BP_ZC];
                        if (SPLIT > 1 && NR >= 16 && staged) {
                            // long tents (NR even, >= 16; measured: coarsest paper grid
                            // 1.28 -> 1.15 ms, while NR = 10 ran 2 % slower): interval
                            // sums, the interval below the warp's first voxel summed
                            // across the lanes
                            constexpr int NI = NR / 2;
                            float A[BP_ZC], B[BP_ZC];
#pragma unroll
                            for (int zc = 0; zc < BP_ZC; ++zc) {
                                const int c = c_base + zc * 32 + lane;
                                interval_sums<NI>(pcol, s0, s1, d.cv + ((float)c - g.cz) * en.m,
                                                  d.cv + ((float)(c + 1) - g.cz) * en.m, en.sc, A[zc], B[zc]);
                            }
                            float be = 0.f;
                            {
                                const float qe = d.cv + ((float)(c_base - 1) - g.cz) * en.m;
                                const float qn = d.cv + ((float)c_base - g.cz) * en.m;
                                const int lo = (int)ceilf(qe), hi = (int)ceilf(qn);
                                const int w0 = min(max(lo, s0), s1 - NI + 1);
                                if (lane < NI && lane < hi - w0) {
                                    const float x = __fmaf_rn((float)lane, en.sc, ((float)w0 - qe) * en.sc);
                                    be = x * pcol[w0 + lane];
                                }
#pragma unroll
                                for (int o = 16; o > 0; o >>= 1) be += __shfl_xor_sync(0xffffffffu, be, o);
                            }
#pragma unroll
                            for (int zc = 0; zc < BP_ZC; ++zc) {
                                float bprev = __shfl_up_sync(0xffffffffu, B[zc], 1);
                                const float b31 = __shfl_sync(0xffffffffu, B[zc > 0 ? zc - 1 : 0], 31);
                                if (lane == 0) bprev = zc == 0 ? be : b31;
                                sv[zc] = bprev + A[zc] - B[zc];
                            }
                            add_entry<ZC>(acc, en, sv);
                            continue;
                        }
#pragma unroll
                        for (int zc = 0; zc < BP_ZC; ++zc) {
                            const int c = c_base + zc * 32 + lane;
                            const float q = d.cv + ((float)c - g.cz) * en.m;   // row whose sample hits z_c
                            sv[zc] = tent_rows_staged<NR>(pcol, pa_col, staged, s0, s1, q, en.m, en.sc);
                        }
                        if (!(NR > 0 && staged)) {
                            // generic path: rows outside the staged patch come from global memory
                            const int iu_e = en.cell >> 8;
                            const RayCol rce = g.cols[(size_t)view * nu + iu_e];
                            const size_t gbase = (size_t)view * nv * nu + iu_e;
#pragma unroll
                            for (int zc = 0; zc < BP_ZC; ++zc) {
                                const int c = c_base + zc * 32 + lane;
                                const float q = d.cv + ((float)c - g.cz) * en.m;
                                sv[zc] = tent_rows_global<PRESCALED>(d, g, pcol, sino, gbase, st, rce, staged,
                                                                     s0, s1, q, en.m, en.sc);
                            }
                        }
                        add_entry<ZC>(acc, en, sv);
                    }
                    __syncwarp();
                }
            }
        }
        __syncthreads();
    }

    if (SPLIT > 1) {
        // add the other parts' sums into part 0 (the patch is free now)
        float *xch = patch;   // [SPLIT-1][BP_WARPS][BP_G*BP_G*ZC][32]
        constexpr int PER = BP_G * BP_G * ZC;
        if (part > 0) {
            float *dst = xch + ((size_t)(part - 1) * BP_WARPS + warp) * PER * 32;
#pragma unroll
            for (int ia = 0; ia < BP_G; ++ia)
#pragma unroll
                for (int ib = 0; ib < BP_G; ++ib)
#pragma unroll
                    for (int zc = 0; zc < ZC; ++zc) dst[((ia * BP_G + ib) * ZC + zc) * 32 + lane] = acc[ia][ib][zc];
        }
        __syncthreads();
        if (part == 0) {
            for (int pp = 1; pp < SPLIT; ++pp) {
                const float *src = xch + ((size_t)(pp - 1) * BP_WARPS + warp) * PER * 32;
#pragma unroll
                for (int ia = 0; ia < BP_G; ++ia)
#pragma unroll
                    for (int ib = 0; ib < BP_G; ++ib)
#pragma unroll
                        for (int zc = 0; zc < ZC; ++zc) acc[ia][ib][zc] += src[((ia * BP_G + ib) * ZC + zc) * 32 + lane];
            }
        }
    }

    // epilogue: one write per voxel (part-0 warps)
    const float scale = (MODE == 1) ? (d_scale ? (float)(*d_scale) : scale_val) : 0.f;
    float sq = 0.f;
#pragma unroll
    for (int ia = 0; ia < BP_G; ++ia)
#pragma unroll
        for (int ib = 0; ib < BP_G; ++ib) {
            const int a = A + ia, b = B + ib;
            if (part != 0) continue;
            if (a >= nx || b >= ny) continue;
#pragma unroll
            for (int zc = 0; zc < BP_ZC; ++zc) {
                const int c = c_base + zc * 32 + lane;
                if (c >= nz) continue;
                const size_t idx = ((size_t)a * ny + b) * nz + c;
                if (MODE == 0) {
                    out[idx] = acc[ia][ib][zc];
                } else if (MODE == 3) {
                    out[(size_t)vg * ((size_t)nx * ny * nz) + idx] = acc[ia][ib][zc];
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

#if BP_MODE_UNIT == 0
static int bp_zc(const VolGeom &v) { return v.bp_zc > 0 ? v.bp_zc : (v.nz <= 32 ? 1 : 2); }

static int bp_zblocks(const VolGeom &v) { return (v.nz + 32 * bp_zc(v) - 1) / (32 * bp_zc(v)); }

static int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n < 1) n = 1;
    }
    return n;
}

size_t bp_split_floats(const VolGeom &v, const DetGeom &d)
{
    // the stream-K transpose keeps its tile partials and arrival counters here
    if (bs_usable(v, d)) return bs_scratch_floats(v, d) + bs_counter_count(v, d);
    const int gcount = bp_view_groups(v, d);
    return gcount > 1 ? (size_t)gcount * v.nx * v.ny * v.nz : 0;
}

constexpr int BPC_THREADS = 256;
constexpr int BPC_BLOCKS = 1024;

int bp_grid_blocks(const VolGeom &v)
{
    const int direct = ((v.nx + BP_TX - 1) / BP_TX) * ((v.ny + BP_TY - 1) / BP_TY) * bp_zblocks(v);
    return std::max(direct, BPC_BLOCKS);
}

static double support_r(const VolGeom &v)
{
    return sqrt(pow(0.5 * (v.nx + 1) * v.dx, 2) + pow(0.5 * (v.ny + 1) * v.dy, 2));
}

// Largest number of detector rows one voxel's z tent can cover on this grid:
// floor(2 m) + 1 with m = 1/sc at the smallest sc = rho dv / (L_xy dz).
int bp_rows_needed(const VolGeom &v, const DetGeom &d)
{
    const double R = support_r(v);
    const double umax = 0.5 * (d.nu - 1) * d.du;
    const double lxy_max = sqrt((double)d.sdd * d.sdd + umax * umax);
    const double sc_min = (d.sad - R) * d.dv / (lxy_max * v.dz);
    // rows strictly inside (q - m, q + m): at most floor(2m) + 1; the 1e-4
    // slack covers the FP32 evaluation of m on the device
    return (int)floor(2.0 / sc_min * (1.0 + 1e-4)) + 1;
}

static int bp_nr_variant(const VolGeom &v, const DetGeom &d)
{
    const int need = bp_rows_needed(v, d);
    for (int nr : {4, 5, 6, 8, 10, 12, 16, 20, 24})
        if (need <= nr) return nr;
    return 0;
}

// Largest staged patch (floats) of any block and view on this grid: a host
// mirror (FP64) of the device's box computation, with two pixels of slack on
// each side. Blocks whose patch still does not fit read the sinogram from
// global memory instead.
int bp_patch_floats(const VolGeom &v, const DetGeom &d, const double *angles)
{
    const long cap_max = 48L * 1024L;   // floats: 192 KB
    return (int)std::min<long>(bp_patch_floats_tile(v, d, angles, 32 * bp_zc(v), bp_nr_variant(v, d)), cap_max);
}

// z chunks per lane: two (64 z voxels per block) unless the grid is 32 deep
// or less, or the taller patch of 64 z voxels would not fit shared memory for
// every tile and view (the blocks that do not fit read rows from global
// memory at a fraction of the speed and run far longer than the rest).
int bp_choose_zc(const VolGeom &v, const DetGeom &d, const double *angles)
{
    if (v.nz <= 32) return 1;
    const long cap_max = 48L * 1024L;
    return bp_patch_floats_tile(v, d, angles, 64, bp_nr_variant(v, d)) <= cap_max ? 2 : 1;
}

// The same for tiles of BP_TX x BP_TY columns and tz z values with nr zero
// rows of padding on each side.
int bp_patch_floats_tile(const VolGeom &v, const DetGeom &d, const double *angles, int tz, int nr)
{
    const int nbx = (v.nx + BP_TX - 1) / BP_TX, nby = (v.ny + BP_TY - 1) / BP_TY, nbz = (v.nz + tz - 1) / tz;
    const double cx = 0.5 * (v.nx - 1), cy = 0.5 * (v.ny - 1), cz = 0.5 * (v.nz - 1);
    const double cu = 0.5 * (d.nu - 1), cv = 0.5 * (d.nv - 1);
    long best = 0;
    for (int k = 0; k < d.n_views; k++) {
        const double c = cos(angles[k]), sn = sin(angles[k]);
        for (int bx = 0; bx < nbx; bx++)
            for (int by = 0; by < nby; by++) {
                const double x0 = (bx * BP_TX - cx) * v.dx - v.dx, x1 = (bx * BP_TX - cx) * v.dx + BP_TX * v.dx;
                const double y0 = (by * BP_TY - cy) * v.dy - v.dy, y1 = (by * BP_TY - cy) * v.dy + BP_TY * v.dy;
                double umin = 1e300, umax = -1e300, xrlo = 1e300, xrhi = -1e300;
                for (int q = 0; q < 4; q++) {
                    const double x = (q & 1) ? x1 : x0, y = (q & 2) ? y1 : y0;
                    const double xr = x * c + y * sn, yr = -x * sn + y * c;
                    const double u = -yr * d.sdd / (xr + d.sad);
                    umin = std::min(umin, u);
                    umax = std::max(umax, u);
                    xrlo = std::min(xrlo, xr);
                    xrhi = std::max(xrhi, xr);
                }
                const int iu0 = std::max((int)floor(umin / d.du + cu) - 3, 0);
                const int iu1 = std::min((int)ceil(umax / d.du + cu) + 3, d.nu - 1);
                const double mn = d.sdd / (xrlo + d.sad), mf = d.sdd / (xrhi + d.sad);
                for (int bz = 0; bz < nbz; bz++) {
                    const double zlo = (bz * tz - cz - 1.0) * v.dz, zhi = (bz * tz + tz - cz) * v.dz;
                    const double vmin = std::min(std::min(zlo * mn, zlo * mf), std::min(zhi * mn, zhi * mf));
                    const double vmax = std::max(std::max(zlo * mn, zlo * mf), std::max(zhi * mn, zhi * mf));
                    const int iv0 = std::max((int)floor(vmin / d.dv + cv) - 3, 0);
                    const int iv1 = std::min((int)ceil(vmax / d.dv + cv) + 3, d.nv - 1);
                    if (iu1 < iu0 || iv1 < iv0) continue;
                    const long w = iu1 - iu0 + 1, h = (iv1 - iv0 + 1) + 2L * nr;
                    best = std::max(best, w * (h | 1));
                }
            }
    }
    return (int)std::min<long>(best, (long)INT32_MAX);
}

// Dynamic shared memory of a transpose launch on this grid.
size_t bp_smem_bytes(const VolGeom &v, const DetGeom &d)
{
    if (v.bp_cap > 0) return (size_t)v.bp_cap * sizeof(float);
    return bp_smem_bound(v, d);
}

// Analytic upper bound of the staged patch (used when no exact size is known).
size_t bp_smem_bound(const VolGeom &v, const DetGeom &d)
{
    const double R = support_r(v);
    const double m_max = d.sdd / (d.sad - R), m_min = d.sdd / (d.sad + R);
    const double diag = sqrt(pow((BP_TX + 1) * (double)v.dx, 2) + pow((BP_TY + 1) * (double)v.dy, 2));
    const double w = std::min(diag * m_max / d.du + 6.0, (double)d.nu);
    const double zext = (32 * bp_zc(v) + 1) * (double)v.dz;
    const double zabs = 0.5 * (v.nz + 1) * v.dz;
    const int nr = bp_nr_variant(v, d);
    const double h = std::min((zext * m_max + zabs * (m_max - m_min)) / d.dv + 6.0, (double)d.nv) + 2.0 * nr + 1;
    double cap = ceil(w) * (double)((int)ceil(h) | 1);
    const double cap_max = 48.0 * 1024.0;   // floats: 192 KB
    if (cap > cap_max) cap = cap_max;
    return (size_t)cap * sizeof(float);
}

// out = epilogue(sum over view groups g of part[g]) in a fixed order
template <int MODE>
__global__ void __launch_bounds__(BPC_THREADS)
bp_combine_kernel(const float *__restrict__ part, int groups, size_t n, const float *__restrict__ f,
                  float *__restrict__ out, const double *__restrict__ d_scale, float scale_val, float kappa,
                  double *__restrict__ partials)
{
    __shared__ double red[32];
    const float scale = (MODE == 1) ? (d_scale ? (float)(*d_scale) : scale_val) : 0.f;
    float sq = 0.f;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float s = 0.f;
        for (int gi = 0; gi < groups; ++gi) s += __ldg(part + (size_t)gi * n + i);
        if (MODE == 0) {
            out[i] = s;
        } else if (MODE == 1) {
            out[i] = __fmaf_rn(-scale, s, __ldg(f + i));
        } else {
            const float w = kappa * s;
            out[i] = w;
            sq += w * w;
        }
    }
    if (MODE == 2) {
        DF v[1] = {DF{sq, 0.f}};
        double tot[1];
        block_sum_df<1>(v, red, tot);
        if (threadIdx.x == 0) partials[blockIdx.x] = tot[0];
    }
}

// View groups. A grid's column tiles give `base` blocks, of which the GPU
// holds `slots` at once (SMs x resident blocks of the selected variant); a
// launch takes ceil(blocks / slots) waves. Splitting the views into groups
// multiplies the blocks and divides each block's views, and a combine pass
// adds the groups' raw sums in a fixed order. The group count minimises
// waves x (views per block + per-block overhead) + the combine's cost, both
// overheads in units of one view of one block (0.3 and 0.15, measured on the
// paper-scale levels); one group when the tiles alone fill many waves.
static int bp_blocks_per_sm(const VolGeom &v, const DetGeom &d)
{
    static std::mutex mu;
    static std::vector<std::pair<std::array<int, 6>, int>> cache;
    const std::array<int, 6> key{v.nx, v.ny, v.nz, d.nu, d.nv, v.bp_cap};
    {
        std::lock_guard<std::mutex> lk(mu);
        for (const auto &kv : cache)
            if (kv.first == key) return kv.second;
    }
    int occ = 0;
    BpLaunch L{};
    L.v = v;
    L.d = d;
    L.occ = &occ;
    L.split = bp_split_for(bp_nr_variant(v, d));
    if (bp_dispatch<3, true>(bp_zc(v), bp_nr_variant(v, d), dim3(1), dim3(1), bp_smem_bytes(v, d), 0, L) !=
            cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    std::lock_guard<std::mutex> lk(mu);
    cache.emplace_back(key, occ);
    return occ;
}

int bp_view_groups(const VolGeom &v, const DetGeom &d)
{
    const long base = (long)((v.nx + BP_TX - 1) / BP_TX) * ((v.ny + BP_TY - 1) / BP_TY) * bp_zblocks(v);
    const long slots = (long)sm_count() * bp_blocks_per_sm(v, d);
    if (base >= 16 * slots) return 1;
    double best = 1e300;
    int best_g = 1;
    for (int g = 1; g <= d.n_views; ++g) {
        const int per = (d.n_views + g - 1) / g;            // views per block, as the launch splits them
        if ((d.n_views + per - 1) / per != g) continue;     // the same split as a smaller g
        const double waves = (double)((base * g + slots - 1) / slots);
        const double cost = waves * (per + 0.3) + (g > 1 ? 0.15 * g : 0.0);
        if (cost < best - 1e-9) {
            best = cost;
            best_g = g;
        }
    }
    return best_g;
}

int bp_partials_count(const VolGeom &v, const DetGeom &d, bool split)
{
    if (bs_usable(v, d)) return bs_partials_count(v);
    if (split && bp_view_groups(v, d) > 1) return BPC_BLOCKS;
    return ((v.nx + BP_TX - 1) / BP_TX) * ((v.ny + BP_TY - 1) / BP_TY) * bp_zblocks(v);
}

#endif // BP_MODE_UNIT == 0

template <int MODE, bool P, int NR, int ZC, int SPLIT>
static cudaError_t launch_split(dim3 grid, size_t smem, cudaStream_t s, const BpLaunch &L)
{
    // the parts' exchange at the end reuses the patch buffer
    const size_t xch = (size_t)(SPLIT - 1) * BP_WARPS * BP_G * BP_G * ZC * 32 * sizeof(float);
    if (xch > smem) smem = xch;
    cudaError_t e = cudaFuncSetAttribute(bp_kernel<MODE, P, NR, ZC, SPLIT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // the staged patches, not L1, hold the reused data: ask for the largest carveout
    e = cudaFuncSetAttribute(bp_kernel<MODE, P, NR, ZC, SPLIT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    if (L.occ)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(L.occ, bp_kernel<MODE, P, NR, ZC, SPLIT>,
                                                             BP_WARPS * 32 * SPLIT, smem);
    bp_kernel<MODE, P, NR, ZC, SPLIT><<<grid, BP_WARPS * 32 * SPLIT, smem, s>>>(
        L.v, L.d, L.sino, L.st, L.f, L.out, L.d_scale, L.scale_val, L.kappa, L.partials, L.cap, NR, L.zblocks,
        L.vpg);
    return cudaGetLastError();
}

template <int MODE, bool P, int NR, int ZC>
static cudaError_t launch_one(dim3 grid, dim3 block, size_t smem, cudaStream_t s, const BpLaunch &L)
{
    (void)block;
    return launch_split<MODE, P, NR, ZC, bp_split_for(NR)>(grid, smem, s, L);
}

template <int MODE, bool P, int ZC>
static cudaError_t launch_nr(int nr, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const BpLaunch &L)
{
    switch (nr) {
    case 4: return launch_one<MODE, P, 4, ZC>(grid, block, smem, s, L);
    case 5: return launch_one<MODE, P, 5, ZC>(grid, block, smem, s, L);
    case 6: return launch_one<MODE, P, 6, ZC>(grid, block, smem, s, L);
    case 8: return launch_one<MODE, P, 8, ZC>(grid, block, smem, s, L);
    case 10: return launch_one<MODE, P, 10, ZC>(grid, block, smem, s, L);
    case 12: return launch_one<MODE, P, 12, ZC>(grid, block, smem, s, L);
    case 16: return launch_one<MODE, P, 16, ZC>(grid, block, smem, s, L);
    case 20: return launch_one<MODE, P, 20, ZC>(grid, block, smem, s, L);
    case 24: return launch_one<MODE, P, 24, ZC>(grid, block, smem, s, L);
    default: return launch_one<MODE, P, 0, ZC>(grid, block, smem, s, L);
    }
}

// One dispatcher per (mode, prescaled) pair; BP_MODE_UNIT selects which pairs
// this translation unit instantiates so the variants compile in parallel.
template <int MODE, bool P>
cudaError_t bp_dispatch(int zc, int nr, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const BpLaunch &L)
{
    if (zc == 1) return launch_nr<MODE, P, 1>(nr, grid, block, smem, s, L);
    return launch_nr<MODE, P, 2>(nr, grid, block, smem, s, L);
}

#if BP_MODE_UNIT == 0
template cudaError_t bp_dispatch<0, false>(int, int, dim3, dim3, size_t, cudaStream_t, const BpLaunch &);
#elif BP_MODE_UNIT == 1
template cudaError_t bp_dispatch<1, true>(int, int, dim3, dim3, size_t, cudaStream_t, const BpLaunch &);
#elif BP_MODE_UNIT == 2
template cudaError_t bp_dispatch<1, false>(int, int, dim3, dim3, size_t, cudaStream_t, const BpLaunch &);
#elif BP_MODE_UNIT == 3
template cudaError_t bp_dispatch<2, true>(int, int, dim3, dim3, size_t, cudaStream_t, const BpLaunch &);
#elif BP_MODE_UNIT == 4
template cudaError_t bp_dispatch<3, true>(int, int, dim3, dim3, size_t, cudaStream_t, const BpLaunch &);
#elif BP_MODE_UNIT == 5
template cudaError_t bp_dispatch<3, false>(int, int, dim3, dim3, size_t, cudaStream_t, const BpLaunch &);
#endif

#if BP_MODE_UNIT == 0
cudaError_t launch_back(const VolGeom &v, const DetGeom &d, const float *sino, const float *f,
                        float *out, const double *d_scale, double scale_val, double kappa,
                        double *partials, int mode, int prescaled, float *split_ws, cudaStream_t s)
{
    return launch_back_st(v, d, sino, CBCT_STORAGE_F32, f, out, d_scale, scale_val, kappa, partials, mode,
                          prescaled, split_ws, s);
}

cudaError_t launch_back_st(const VolGeom &v, const DetGeom &d, const void *sino, int st, const float *f,
                           float *out, const double *d_scale, double scale_val, double kappa,
                           double *partials, int mode, int prescaled, float *split_ws, cudaStream_t s)
{
    if (bs_usable(v, d) && (mode != 2 || prescaled)) {
        const int kid = mode == 1 ? K_BP_STEP : K_BP;
        unsigned int *counters =
            split_ws ? reinterpret_cast<unsigned int *>(split_ws + bs_scratch_floats(v, d)) : nullptr;
        launch_begin(kid, s);
        const cudaError_t e = launch_bs(v, d, sino, st, f, out, d_scale, scale_val, kappa, partials, mode, prescaled,
                                        split_ws, counters, s);
        launch_end(kid, s);
        return e;
    }
    const int zc = bp_zc(v), zblocks = bp_zblocks(v);
    const int groups = split_ws ? bp_view_groups(v, d) : 1;
    const int vpg = (d.n_views + groups - 1) / groups;
    dim3 grid((v.nx + BP_TX - 1) / BP_TX, (v.ny + BP_TY - 1) / BP_TY, zblocks * groups);
    dim3 block(BP_WARPS * 32);
    const size_t smem = bp_smem_bytes(v, d);
    const int cap = (int)(smem / sizeof(float));
    const int nr = bp_nr_variant(v, d);
    const int kid = mode == 1 ? K_BP_STEP : K_BP;
    cudaError_t e;
    const int split = bp_split_for(nr);
    BpLaunch L{v, d, sino, st, f, out, d_scale, (float)scale_val, (float)kappa, partials, cap, zblocks, vpg, split};
    launch_begin(kid, s);
    if (groups > 1) {
        BpLaunch Ls = L;
        Ls.out = split_ws;
        if (prescaled)
            e = bp_dispatch<3, true>(zc, nr, grid, block, smem, s, Ls);
        else
            e = bp_dispatch<3, false>(zc, nr, grid, block, smem, s, Ls);
        if (e == cudaSuccess) {
            note_extra_launch();
            const size_t n = (size_t)v.nx * v.ny * v.nz;
            if (mode == 0)
                bp_combine_kernel<0><<<BPC_BLOCKS, BPC_THREADS, 0, s>>>(split_ws, groups, n, f, out, d_scale,
                                                                       (float)scale_val, (float)kappa, partials);
            else if (mode == 1)
                bp_combine_kernel<1><<<BPC_BLOCKS, BPC_THREADS, 0, s>>>(split_ws, groups, n, f, out, d_scale,
                                                                       (float)scale_val, (float)kappa, partials);
            else
                bp_combine_kernel<2><<<BPC_BLOCKS, BPC_THREADS, 0, s>>>(split_ws, groups, n, f, out, d_scale,
                                                                       (float)scale_val, (float)kappa, partials);
            e = cudaGetLastError();
        }
    } else if (mode == 0) {
        e = bp_dispatch<0, false>(zc, nr, grid, block, smem, s, L);
    } else if (mode == 1 && prescaled) {
        e = bp_dispatch<1, true>(zc, nr, grid, block, smem, s, L);
    } else if (mode == 1) {
        e = bp_dispatch<1, false>(zc, nr, grid, block, smem, s, L);
    } else if (prescaled) {
        e = bp_dispatch<2, true>(zc, nr, grid, block, smem, s, L);   // power iteration: ds-weighted input
    } else {
        e = cudaErrorInvalidValue;   // the power-iteration transpose takes a ds-weighted sinogram
    }
    launch_end(kid, s);
    return e;
}
#endif // BP_MODE_UNIT == 0

} // namespace cbct
