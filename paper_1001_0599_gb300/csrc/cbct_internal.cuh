// Internal definitions shared by the libcbct translation units (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cbct.h"

namespace cbct {

// ---------------------------------------------------------------------------
// Geometry as the kernels see it
// ---------------------------------------------------------------------------

// One in-plane ray line (view, iu), derived in FP64 on the host. Sample j of
// the line (k = kc + j in the paper's discretisation of Eq. 1, in-plane
// distance rho_k = k drho from the source) sits at
//     t = j drho - delta,   (x, y) = (mx, my) + t (ex, ey),
//     z(iv) = rho_k v(iv) / L_xy.
// (mx, my) is the point of the line closest to the rotation axis, so x, y
// stay small and keep FP32 precision.
struct RayCol {
    float mx, my;     // closest point of the line to the axis, mm
    float ex, ey;     // unit in-plane direction
    float delta;      // rho_c - kc drho, rho_c = in-plane distance source -> (mx, my)
    float inv_lxy;    // 1 / L_xy(u), L_xy = in-plane source-pixel distance
    int kc;           // sample index nearest (mx, my)
    int16_t jlo, jhi; // samples kc+jlo .. kc+jhi cover the volume's support (empty if jlo > jhi)
};
static_assert(sizeof(RayCol) == 32, "RayCol must stay 32 bytes");

struct VolGeom {
    int nx, ny, nz;
    float dx, dy, dz;
    float inv_dx, inv_dy, inv_dz;
    float cx, cy, cz;          // (n - 1) / 2
    float drho;                // in-plane sample spacing
    const RayCol *cols;        // [n_views][nu]
    int bp_cap;                // largest staged detector patch of the transpose, floats (0: bound)
    int bs_cap;                // staged patch of the stream-K transpose (bps.cu), floats (0: not used)
    int bp_zc;                 // z chunks per lane of bp.cu's transpose (0: by nz alone)
};

struct DetGeom {
    int nu, nv, n_views;
    float du, dv, inv_du, inv_dv, cu, cv;
    float sad, sdd;
    const float2 *views;       // (cos, sin) per view
};

// Continuous voxel coordinates of sample j of a ray line (shared by the
// projector and its transpose so both see identical sample positions).
#ifndef CBCT_LDS_IMM
#define CBCT_LDS_IMM 1   // transpose tent rows read with immediate offsets (build-time tuning: 0 or 1)
#endif

// Shared-memory load at a 32-bit shared-window address plus a compile-time
// byte offset carried in the load's immediate field: a run of consecutive
// rows then costs one address computation, not one per row.
template <int OFF>
__device__ __forceinline__ float lds_off(uint32_t addr)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(addr), "n"(OFF));
    return v;
}

__device__ __forceinline__ void sample_xy(const VolGeom &g, const RayCol &rc, int j, float &fx,
                                          float &fy)
{
    float t = __fmaf_rn((float)j, g.drho, -rc.delta);
    float x = __fmaf_rn(t, rc.ex, rc.mx);
    float y = __fmaf_rn(t, rc.ey, rc.my);
    fx = __fmaf_rn(x, g.inv_dx, g.cx);
    fy = __fmaf_rn(y, g.inv_dy, g.cy);
}

__device__ __forceinline__ float sample_rho(const VolGeom &g, const RayCol &rc, int j)
{
    return __fmul_rn((float)(rc.kc + j), g.drho);
}

// ---------------------------------------------------------------------------
// Compensated FP32 ("double-float") accumulation for the reduction trees:
// GB300's FP64 rate is a small fraction of FP32, so per-thread and per-warp
// partial sums are carried as exact (hi, lo) float pairs and converted to
// FP64 only where blocks are combined.
// ---------------------------------------------------------------------------
struct DF {
    float hi, lo;
};

// Geometry of the Eq. 6 kernel (eq6.cu) for one grid, derived in FP64 on
// the host and handed over as double-float pairs where the detector
// coordinate needs more than FP32.
struct Eq6Geom {
    DF dx, dy, dz;             // voxel pitch
    float cx, cy, cz;          // (n - 1) / 2
    DF sad;                    // source-to-axis distance
    DF ku, kv;                 // L0 / du, L0 / dv (L0 = source-to-detector distance)
    float cu, cv;              // (nu - 1) / 2, (nv - 1) / 2
    float two_l0sq;            // 2 L0^2
    const float4 *views;       // (cos hi, cos lo, sin hi, sin lo) per view
};

__device__ __forceinline__ DF df_zero() { return DF{0.f, 0.f}; }

__device__ __forceinline__ DF df_add(DF a, float b)
{
    float s = __fadd_rn(a.hi, b);
    float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    e = __fadd_rn(e, a.lo);
    float hi = __fadd_rn(s, e);
    float lo = __fsub_rn(e, __fsub_rn(hi, s));
    return DF{hi, lo};
}

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    float s = __fadd_rn(a.hi, b.hi);
    float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    float hi = __fadd_rn(s, e);
    float lo = __fsub_rn(e, __fsub_rn(hi, s));
    return DF{hi, lo};
}

__device__ __forceinline__ DF df_warp_sum(DF v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        DF w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = df_add(v, w);
    }
    return v;
}

// Block-wide sum of K double-float values per thread; thread 0 receives the
// FP64 totals in out[]. Deterministic order. scratch: >= 32*K doubles smem.
template <int K>
__device__ __forceinline__ void block_sum_df(DF (&v)[K], double *scratch, double (&out)[K])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = df_warp_sum(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) scratch[warp * K + k] = (double)v[k].hi + (double)v[k].lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            double s = 0.0;
            for (int w = 0; w < nwarp; w++) s += scratch[w * K + k];
            out[k] = s;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Device state shared by the kernels of one call (lives in the workspace)
// ---------------------------------------------------------------------------
struct GridBarrier {
    unsigned int count;
    unsigned int gen;
    int error;        // set when a bounded wait gave up
    int pad;
};

struct DevState {
    GridBarrier bar;
    double tau;          // current level's step
    double scale;        // tau * kappa
    double lipschitz;
    double vnorm2;       // power iteration: |v|^2 of the current iterate
    double inv_wnorm;    // power iteration: 1/|w|
    double e2;           // last data term
    double red[8];       // results of the last grid-wide reduction
    int rof_inner;
    int rof_bt;
    int rof_flags;
    int rof_done;
    int step_log_pos;    // next free entry of the recon step log
    int iter_pos;        // next iteration record
    int pad[2];
};

// ---------------------------------------------------------------------------
// Launch bookkeeping (profiling + launch count), defined in api.cu
// ---------------------------------------------------------------------------
enum KernelId {
    K_FP = 0,
    K_FP_RESID,
    K_BP,
    K_BP_STEP,
    K_ROF,
    K_REDUCE,
    K_PROLONG,
    K_FILL,
    K_MISC,
    K_EQ6,
    K_COUNT
};

void launch_begin(int kernel, cudaStream_t s);
void launch_end(int kernel, cudaStream_t s);
void note_extra_launch();   // a second kernel inside one timed launch_begin/launch_end bracket

// ---------------------------------------------------------------------------
// Kernel launchers (one per translation unit)
// ---------------------------------------------------------------------------

// forward projector. mode 0: out = scale * P vol (scale from d_scale if given)
// mode 1: out = P vol - y (unscaled residual), partials <- sum r^2
// mode 2: out = ds * (P vol - y) (residual pre-weighted for the transpose), partials <- sum r^2
// mode 3: out = scale * ds * P vol (projection pre-weighted for the transpose)
// Storage type of a volume or sinogram array (cbct_storage): values are
// widened to FP32 on load and rounded to nearest on store; all arithmetic is
// FP32 and reductions FP64.
__device__ __forceinline__ float ld_st(const void *p, size_t i, int st)
{
    if (st == CBCT_STORAGE_BF16) return __bfloat162float(__ldg(static_cast<const __nv_bfloat16 *>(p) + i));
    if (st == CBCT_STORAGE_F16) return __half2float(__ldg(static_cast<const __half *>(p) + i));
    return __ldg(static_cast<const float *>(p) + i);
}
__device__ __forceinline__ void st_st(void *p, size_t i, float v, int st)
{
    if (st == CBCT_STORAGE_BF16)
        static_cast<__nv_bfloat16 *>(p)[i] = __float2bfloat16_rn(v);
    else if (st == CBCT_STORAGE_F16)
        static_cast<__half *>(p)[i] = __float2half_rn(v);
    else
        static_cast<float *>(p)[i] = v;
}
template <typename T> __device__ __forceinline__ float ldt(const T *p);
template <> __device__ __forceinline__ float ldt<float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float ldt<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(__ldg(p));
}
template <> __device__ __forceinline__ float ldt<__half>(const __half *p) { return __half2float(__ldg(p)); }
inline size_t storage_bytes(int st) { return st == CBCT_STORAGE_F32 ? 4 : 2; }

int fp_grid_blocks(const DetGeom &d);                          // largest grid (workspace sizing)
int fp_partials_count(const VolGeom &v, const DetGeom &d);      // blocks of the launch for this level
cudaError_t launch_forward(const VolGeom &v, const DetGeom &d, const float *vol, const float *y,
                           float *out, const double *d_scale, double *partials, int mode,
                           cudaStream_t s);
// the same with vol, y and out stored as `st` (cbct_storage); reduced storage
// needs the sheet variant (cudaErrorNotSupported otherwise)
cudaError_t launch_forward_st(const VolGeom &v, const DetGeom &d, const void *vol, const void *y, void *out,
                              int st, const double *d_scale, double *partials, int mode, cudaStream_t s);
bool fp_supports_storage(const VolGeom &v, const DetGeom &d, int st);
// element-wise conversion between storage types (n elements)
cudaError_t launch_convert(const void *src, int src_st, void *dst, int dst_st, size_t n, cudaStream_t s);

// transpose. mode 0: out = P^T sino; mode 1: out = f - scale P^T sino with
// scale = *d_scale if given, else scale_val (sino pre-weighted by ds when
// prescaled != 0); mode 2: out = kappa P^T sino with partials <- sum out^2
// (power iteration)
// (mode 3 internal: raw per-view-group sums). split_ws (may be null) holds
// bp_split_floats() floats; with it, grids too small for the GPU split their
// views over blocks and a combine pass adds the groups in a fixed order.
int bp_grid_blocks(const VolGeom &v);                                    // partial slots to reserve
int bp_partials_count(const VolGeom &v, const DetGeom &d, bool split);   // partials of a mode-2 launch
int bp_view_groups(const VolGeom &v, const DetGeom &d);
size_t bp_split_floats(const VolGeom &v, const DetGeom &d);
size_t bp_smem_bytes(const VolGeom &v, const DetGeom &d);
int bp_patch_floats(const VolGeom &v, const DetGeom &d, const double *angles);
int bp_choose_zc(const VolGeom &v, const DetGeom &d, const double *angles);
int bp_patch_floats_tile(const VolGeom &v, const DetGeom &d, const double *angles, int tz, int nr);
int bp_rows_needed(const VolGeom &v, const DetGeom &d);   // most detector rows one voxel's z tent spans
size_t bp_smem_bound(const VolGeom &v, const DetGeom &d);
cudaError_t launch_back(const VolGeom &v, const DetGeom &d, const float *sino, const float *f,
                        float *out, const double *d_scale, double scale_val, double kappa,
                        double *partials, int mode, int prescaled, float *split_ws, cudaStream_t s);
// the same with the sinogram stored as `st` (cbct_storage)
cudaError_t launch_back_st(const VolGeom &v, const DetGeom &d, const void *sino, int st, const float *f,
                           float *out, const double *d_scale, double scale_val, double kappa,
                           double *partials, int mode, int prescaled, float *split_ws, cudaStream_t s);

// Stream-K transpose for short z tents (bps.cu): the same modes 0-2 as
// launch_back. Grids it serves (bs_usable) give one mode-2 partial per column
// tile (bs_partials_count). scratch (bs_scratch_floats floats) and counters
// (bs_counter_count) may be null: every block then takes whole tiles.
int bs_patch_floats(const VolGeom &v, const DetGeom &d, const double *angles);
bool bs_usable(const VolGeom &v, const DetGeom &d);
int bs_partials_count(const VolGeom &v);
size_t bs_scratch_floats(const VolGeom &v, const DetGeom &d);
size_t bs_counter_count(const VolGeom &v, const DetGeom &d);
cudaError_t launch_bs(const VolGeom &v, const DetGeom &d, const void *sino, int st, const float *f, float *out,
                      const double *d_scale, double scale_val, double kappa, double *partials, int mode,
                      int prescaled, float *scratch, unsigned int *counters, cudaStream_t s);

// Eq. 6 voxel-driven gradient (eq6.cu). mode 0: out = G(T); mode 1:
// out = f - scale G(T) with scale = scale_val (* *d_scale when given)
// trilinear gather microbenchmark (gather.cu)
cudaError_t launch_gather(const float *vol, int nx, int ny, int nz, int n_lines, int n_samples, float *out,
                          cudaStream_t s);

cudaError_t launch_eq6(const VolGeom &v, const DetGeom &d, const Eq6Geom &e, const float *T, const float *f,
                       float *out, const double *d_scale, double scale_val, int mode, cudaStream_t s);

// small kernels (misc.cu)
cudaError_t launch_sum_partials(const double *partials, int n, int stride, int k, double *out,
                                cudaStream_t s);
cudaError_t launch_e2(const double *partials, int n, double inv_m, DevState *st, cudaStream_t s);
cudaError_t launch_power_init(DevState *st, double nvox, cudaStream_t s);   // nvox <= 0: keep vnorm2
cudaError_t launch_sumsq(const float *x, size_t n, double *partials, int blocks, double *out, cudaStream_t s);
cudaError_t launch_power_update(DevState *st, const double *partials, int n, double kappa_unused,
                                int first, int last, double *d_L_out, cudaStream_t s);
cudaError_t launch_set_tau(DevState *st, double tau_given, double kappa, cbct_recon_stats *rs,
                           int level, cudaStream_t s);
cudaError_t launch_state_init(DevState *st, cbct_recon_stats *rs, cudaStream_t s);
cudaError_t launch_fill(float *p, size_t n, float value, cudaStream_t s);
cudaError_t launch_prolong(int ncx, int ncy, int ncz, const float *c, float *f, cudaStream_t s);

// ROF persistent kernel (tv.cu)
struct RofArgs {
    const float *g;       // auxiliary image g (read only)
    float *f;             // iterate (in/out)
    float *d;             // gradient workspace
    double *partials;     // [grid][4]
    DevState *st;
    cbct_tv_stats *tv_stats;           // optional
    cbct_recon_stats *recon_stats;     // optional: append steps + iteration record
    const int32_t *replay;             // optional: n, m_1..m_n
    int nx, ny, nz;
    float inv_dx, inv_dy, inv_dz;
    double lambda, tau, eps;
    const double *tau_dev;  // when set, tau is read from device memory at launch
    double c, alpha, rel_tol, s0;
    int max_inner, max_bt;
    int start_at_g;       // iterate starts at g (f is written by the first update)
    int clamp;            // clamp f >= 0 at the end (Step 3 of Algorithm A1)
    int mode;             // 0 full solve, 1 energy+grad only, 2 trial only
    double trial_s;       // mode 2
    double *out;          // modes 1, 2: results (E, mean d^2)
    const float *dir;     // mode 2: direction
    const float *cur;     // modes 1, 2: iterate
    int level;
    void *f_store;        // optional: the solve's result also written here in storage type store_type
    int store_type;       // cbct_storage of f_store
    int withhold_arrival; // failure-detection check: no block ever completes the barrier, so
                          // every bounded wait expires and the kernel reports a timeout
};
int rof_grid_blocks();
int rof_bricks(int nx, int ny, int nz);    // partial sums of a solve: 4 per brick
void set_rof_grid_share(int k);            // this thread's solves use 1/k of the GPU
cudaError_t launch_rof(const RofArgs &a, cudaStream_t s);

// Read-only views of a geometry handle and error reporting (api.cu), for
// entry points that live in other translation units.
const VolGeom *geometry_level(const cbct_geometry *g, int level);
const DetGeom *geometry_detector(const cbct_geometry *g);
int geometry_device(const cbct_geometry *g);
uint64_t geometry_serial(const cbct_geometry *g);  // unique per created geometry
cbct_status report_error(cbct_status st, const char *msg);

} // namespace cbct
