/*
 * libcbct -- GB300 (sm_103a) CUDA library for TV-regularised cone-beam CT
 * reconstruction by forward-backward splitting (Jia et al., "GPU-based Fast
 * Low-dose Cone Beam CT Reconstruction via Total Variation", arXiv:1001.0599).
 *
 * Plain C ABI: host or device pointers and sizes only. Every compute call is
 * asynchronous on the caller's CUDA stream (passed as `void *`, a
 * cudaStream_t; NULL = the legacy default stream) and returns after argument
 * checks; argument errors are reported synchronously and nothing is launched.
 * The library never allocates device memory inside a compute call: device
 * memory is allocated only by cbct_geometry_create (its ray tables) and by
 * cbct_server_create (the serving arena), and every other buffer is
 * caller-owned. No C++ exception crosses this boundary.
 *
 * Layouts (caller-owned device arrays, 16-byte aligned, contiguous, FP32):
 *   volume   f[a][b][c], a < nx, b < ny, c < nz (z fastest). Voxel centres
 *            x_a = (a - (nx-1)/2) dx, y_b = (b - (ny-1)/2) dy,
 *            z_c = (c - (nz-1)/2) dz; z is the rotation axis.
 *   sinogram s[k][iv][iu], k < n_views, iv < nv, iu < nu (u fastest). Pixel
 *            centres u = (iu - (nu-1)/2) du, v = (iv - (nv-1)/2) dv.
 * Geometry (Fig. 1, Eq. A2 at angle 0): source Rz(theta)(-sad, 0, 0),
 * detector centre Rz(theta)(sdd - sad, 0, 0), detector axes
 * e_u = Rz(theta)(0, -1, 0) and e_v = (0, 0, 1).
 */
#ifndef CBCT_H
#define CBCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CBCT_OK = 0,
    CBCT_ERR_INVALID_ARG = 1,          /* bad pointer, size, alignment or geometry */
    CBCT_ERR_CUDA = 2,                 /* a CUDA runtime call failed; see cbct_last_error */
    CBCT_ERR_OUT_OF_MEMORY = 3,        /* cbct_geometry_create could not allocate */
    CBCT_ERR_WORKSPACE_TOO_SMALL = 4,  /* ws_bytes below cbct_workspace_size */
    CBCT_ERR_NOT_CONVERGED = 5,        /* reported through stats.flags after the stream syncs */
    CBCT_ERR_UNSUPPORTED = 6,          /* e.g. multigrid on a grid not divisible by 2^(levels-1) */
    CBCT_ERR_TIMEOUT = 7               /* a bounded device-side wait gave up (stats.status) */
} cbct_status;

/* Storage type of a volume or sinogram array for the reduced-precision
 * entry points and cbct_recon_params.storage (no counterpart in the paper,
 * which stores FP32): values widen to FP32 on every load and round to
 * nearest on every store; interpolation and accumulation stay FP32 and
 * reductions FP64. */
typedef enum {
    CBCT_STORAGE_F32 = 0,
    CBCT_STORAGE_BF16 = 1,   /* bfloat16: 8-bit significand, FP32 range */
    CBCT_STORAGE_F16 = 2     /* IEEE binary16: 11-bit significand, max 65504 */
} cbct_storage;

/* Opaque geometry handle: validated copy of the description plus per-level
 * ray tables (FP64-derived, stored FP32) on the device that was current at
 * creation. Only that device may use it. */
typedef struct cbct_geometry cbct_geometry;

typedef struct {
    int nx, ny, nz;          /* voxels */
    double dx, dy, dz;       /* voxel pitch, mm */
    int nu, nv;              /* detector pixels */
    double du, dv;           /* pixel pitch, mm */
    double sad, sdd;         /* source-axis and source-detector distance, mm; the
                                volume's support must lie strictly between source
                                and detector */
    int n_views;
    const double *angles;    /* n_views angles in radians (host, copied); any set,
                                e.g. 200-degree short scans */
    double step_ratio;       /* in-plane sample spacing drho / min(dx, dy); 0 -> 0.5 */
} cbct_geometry_desc;

/* ROF sub-problem controls (Sec. II.B, Eq. 5). */
typedef struct {
    double eps_tv;           /* smoothing inside |grad f|: phi = sqrt(eps^2 + |Df|^2), 1/mm^2 */
    double c;                /* Armijo constant, paper: 0.01 */
    double alpha;            /* step reduction factor, paper: 0.6 */
    double rel_tol;          /* stop when |E_new - E_0| / E_0 < rel_tol, paper: 0.1 % */
    int max_inner;           /* cap on accepted gradient steps (>= 1) */
    int max_backtracks;      /* cap on step reductions per step (>= 0) */
    double s0;               /* initial trial step; <= 0 means tau */
} cbct_tv_params;

/* Written to device memory by cbct_tv_denoise. flags: bit 0 = a step found no
 * acceptable size (solve ended there), bit 1 = max_inner reached; status:
 * CBCT_OK or CBCT_ERR_TIMEOUT. */
typedef struct {
    int n_inner;
    int backtracks;          /* total step reductions over accepted steps */
    int flags;
    int status;
    double e_first;          /* E_ROF at the start */
    double e_last;           /* E_ROF at the end */
} cbct_tv_stats;

#define CBCT_MAX_LEVELS 4
#define CBCT_MAX_ITERS 512
#define CBCT_MAX_STEP_LOG 8192

typedef struct {
    double lambda;                   /* weight of E1 (TV) against E2 (data), = 1/mu of Eq. 2 */
    int n_levels;                    /* multigrid levels, 1..CBCT_MAX_LEVELS (Sec. II.C.3) */
    int iters[CBCT_MAX_LEVELS];      /* FBS iterations per level, coarsest first */
    double tau[CBCT_MAX_LEVELS];     /* step per level (mean metric); <= 0: 1/L by power iteration */
    int power_iters;                 /* power iterations for L (0 -> 20), started from ones */
    int clamp;                       /* apply Step 3 of Algorithm A1 (f >= 0) */
    int power_iters_fine;            /* > 0: every level after the first runs this many power
                                        iterations started from the prolongation of the previous
                                        level's last iterate instead of power_iters from ones */
    int gradient_mode;               /* Step 1 gradient: 0 = matched P^T (exact gradient of E2),
                                        1 = the paper's closed form, Eq. 6 (unmatched, cheaper) */
    cbct_tv_params tv;
    /* Optional replay of a recorded step schedule (testing): host array of
     * records, one per FBS iteration in order: n, then n step-reduction
     * counts. When given, the ROF solves take these steps instead of
     * searching. NULL for normal operation. */
    const int32_t *replay;
    int replay_len;
    int storage;                     /* cbct_storage of the measured sinogram, the residual and
                                        the volume copy the projector gathers from (the iterate
                                        itself, its ROF state and all sums stay FP32/FP64) */
} cbct_recon_params;

typedef struct {
    double e2;               /* data term E2 = sum r^2 / (N_theta N_pix) at the iterate entering */
    double e_rof_first;
    double e_rof_last;
    int level;
    int n_inner;
    int backtracks;
    int flags;               /* cbct_tv_stats.flags of this iteration's ROF solve */
} cbct_iter_stats;

typedef struct {
    double tau[CBCT_MAX_LEVELS];         /* step used per level */
    double lipschitz[CBCT_MAX_LEVELS];   /* power-iteration L per level (0 if tau given) */
    int n_iters;
    int flags;                           /* OR of every iteration's flags */
    int status;                          /* CBCT_OK or CBCT_ERR_TIMEOUT */
    int n_steps;                         /* entries used in steps[] */
    cbct_iter_stats iters[CBCT_MAX_ITERS];
    int32_t steps[CBCT_MAX_STEP_LOG];    /* every accepted step's reduction count, in order */
} cbct_recon_stats;

/* ---- geometry ---------------------------------------------------------- */

/* Validate desc and build the handle (Eq. 1's geometry, Fig. 1). Allocates
 * the device ray tables on the current device (with the serving arena of
 * cbct_server_create, the library's only device allocations). Returns
 * INVALID_ARG for a bad description, OUT_OF_MEMORY
 * or CUDA for allocation/copy failures; *out is NULL on failure. */
cbct_status cbct_geometry_create(const cbct_geometry_desc *desc, cbct_geometry **out);
void cbct_geometry_destroy(cbct_geometry *geom);
/* Grid of multigrid level `level` (0 = finest; each level halves nx, ny, nz
 * and doubles the pitch). UNSUPPORTED if the grid does not divide. */
cbct_status cbct_geometry_level_dims(const cbct_geometry *geom, int level, int *nx, int *ny, int *nz);

/* ---- projector (Eq. 1) ------------------------------------------------- */

/* d_sino = P d_vol: for every ray (view, iv, iu), the sum over integer k of
 * ds * f(S + k drho n / |n_xy|), f the trilinear interpolant of the voxel
 * values (zero outside the grid), n = pixel - source, ds = drho |n| / |n_xy|.
 * Overwrites d_sino (n_views*nv*nu floats) from d_vol (nx*ny*nz floats). */
cbct_status cbct_forward_project(const cbct_geometry *geom, const float *d_vol, float *d_sino,
                                 void *stream);

/* Residual of the data term (T^theta of Sec. II.C.2): d_r = P d_vol - d_y,
 * and *d_sumsq (one double, device) = sum of d_r^2 accumulated in FP64.
 * Needs a workspace of cbct_workspace_size bytes. */
cbct_status cbct_residual(const cbct_geometry *geom, const float *d_vol, const float *d_y,
                          float *d_r, double *d_sumsq, void *d_ws, size_t ws_bytes, void *stream);

/* cbct_residual without a workspace, for callers that are not allowed to
 * allocate device memory (the paper has no counterpart of this call). Some
 * hosts own every device allocation themselves -- a framework memory pool,
 * an embedded or safety-certified pipeline with a fixed memory budget, code
 * running where cudaMalloc is forbidden -- and cannot hand out scratch
 * buffers. Here the FP64 partial sums live in a fixed array inside the
 * library (CBCT_STATIC_MAX_PARTIALS doubles, 2 MiB, held by every GPU that
 * loads the library until the process exits), so the call allocates
 * nothing. The first call on each device looks up that array's device
 * address; make that first call before any stream capture. All calls share
 * the one array: calls that may overlap on the GPU (different streams, or
 * several threads) race and give wrong sums; serialise them. The array
 * holds one partial sum per block of the forward launch, and a geometry
 * whose launch has more blocks than CBCT_STATIC_MAX_PARTIALS is rejected
 * with CBCT_ERR_UNSUPPORTED. That count is n_views * nu on the sheet
 * projector (detectors of at most 1024 rows and volumes of at most 760
 * slices), and n_views * ceil(nu / 8) * ceil(nv / (32 r)) on the
 * warp-per-column projector that serves every other geometry, where r is
 * 1, 2 or 4 detector rows per lane, the largest whose rows' z span fits the
 * kernel's 64-slice segment. The array's device address is looked up once
 * per device and kept; a device reset (cudaDeviceReset) or any other
 * teardown of the device's primary context invalidates it, so this call
 * must not be used on that device afterwards in the same process.
 * Results equal cbct_residual's. */
#define CBCT_STATIC_MAX_PARTIALS 262144
cbct_status cbct_residual_static(const cbct_geometry *geom, const float *d_vol, const float *d_y,
                                 float *d_r, double *d_sumsq, void *stream);

/* d_vol = P^T d_sino, the exact transpose of cbct_forward_project (the matrix
 * view of Sec. II.C.2), evaluated per voxel as a gather: no atomics, every
 * voxel written once. Overwrites d_vol. */
cbct_status cbct_back_project(const cbct_geometry *geom, const float *d_sino, float *d_vol,
                              void *stream);

/* The paper's closed-form gradient of the data term (Eq. 6 with Eq. A6, A7),
 * voxel-driven: d_vol(x) = sum over views of 2 L^3(u*,v*) / (L0 l^2(x)) *
 * T(u*, v*), T = d_T bilinearly interpolated on the detector (zero outside),
 * without Eq. 6's 1/(N_theta A) prefactor. Not the transpose of P: it tends
 * to 2 du dv / (voxel volume) * P^T T as the grids refine. Overwrites d_vol. */
cbct_status cbct_eq6_gradient(const cbct_geometry *geom, const float *d_T, float *d_vol, void *stream);

/* Step 1 of Algorithm A1: d_g = d_f - scale * P^T d_r, with scale = tau*kappa,
 * kappa = 2 N_vox / (N_theta N_pix) for the mean-normalised E2 of Eq. 2.
 * d_g may alias neither d_f nor d_r. */
cbct_status cbct_gradient_step(const cbct_geometry *geom, const float *d_r, const float *d_f,
                               float *d_g, double scale, void *stream);

/* ---- reduced-precision storage ----------------------------------------- */

/* P (Eq. 1) of a volume stored as `storage` into a sinogram stored the same
 * way (FP32 arithmetic in between; each stored value rounded to nearest).
 * Both arrays 16-byte aligned, in the layouts above. Reduced storage needs
 * the shared-memory sheet projector (nv <= 1024 and nz <= 760); otherwise
 * CBCT_ERR_UNSUPPORTED. An unknown storage value is CBCT_ERR_INVALID_ARG. */
cbct_status cbct_forward_project_ex(const cbct_geometry *geom, const void *d_vol, void *d_sino, int storage,
                                    void *stream);
/* The matched transpose of a sinogram stored as `storage`, into an FP32
 * volume (overwritten); the same argument rules as cbct_forward_project_ex. */
cbct_status cbct_back_project_ex(const cbct_geometry *geom, const void *d_sino, int storage, float *d_vol,
                                 void *stream);
/* n elements from src_storage to dst_storage (round to nearest). */
cbct_status cbct_convert(const void *d_src, int src_storage, void *d_dst, int dst_storage, size_t n,
                         void *stream);

/* ---- TV / ROF (Sec. II.B) ---------------------------------------------- */

/* E_ROF[f] = lambda E1[f] + (1/(2 tau)) mean((f - g)^2), E1 = mean of
 * sqrt(eps^2 + |Df|^2) with forward differences; zero boundary on x and y,
 * reflective on z. Writes d_d = N_vox dE_ROF/df (volume) and
 * d_out[0] = E_ROF[f], d_out[1] = mean(d^2) (two doubles, device). */
cbct_status cbct_tv_energy_grad(const cbct_geometry *geom, const float *d_f, const float *d_g,
                                double lambda, double tau, double eps_tv, float *d_d,
                                double *d_out, void *d_ws, size_t ws_bytes, void *stream);

/* Armijo trial of Eq. 5: d_out[0] = E_ROF[f - s d] (one double, device). */
cbct_status cbct_tv_trial(const cbct_geometry *geom, const float *d_f, const float *d_d,
                          const float *d_g, double s, double lambda, double tau, double eps_tv,
                          double *d_out, void *d_ws, size_t ws_bytes, void *stream);

/* Step 2 of Algorithm A1: minimise E_ROF by gradient descent with Armijo
 * backtracking (Eq. 5), entirely on the device (one persistent kernel, no
 * host round trip). d_f holds the start on entry (normally a copy of d_g)
 * and the result on exit. d_stats (device, optional) receives the solve's
 * statistics. */
cbct_status cbct_tv_denoise(const cbct_geometry *geom, const float *d_g, float *d_f,
                            double lambda, double tau, const cbct_tv_params *params,
                            void *d_ws, size_t ws_bytes, cbct_tv_stats *d_stats, void *stream);

/* Failure-detection check (no counterpart in the paper): runs the ROF
 * kernel's first grid barrier with no block ever completing it, so every
 * block's bounded wait expires (after 2 s) and the kernel returns. Once the
 * stream has synchronised, d_stats->status (device) reads CBCT_ERR_TIMEOUT,
 * and the context is still usable. Uses the workspace's g and d volumes. */
cbct_status cbct_check_barrier_timeout(const cbct_geometry *geom, void *d_ws, size_t ws_bytes,
                                       cbct_tv_stats *d_stats, void *stream);

/* ---- multigrid and step size ------------------------------------------ */

/* Cell-centred trilinear prolongation (clamp to edge) from a
 * (ncx, ncy, ncz) grid to (2ncx, 2ncy, 2ncz): the "smooth extension" of
 * Sec. II.C.3. */
cbct_status cbct_prolongate(int ncx, int ncy, int ncz, const float *d_coarse, float *d_fine,
                            void *stream);

/* Lipschitz constant of kappa P^T P on multigrid level `level` by n_iter
 * power iterations from the all-ones volume; *d_L (one double, device). */
cbct_status cbct_power_lipschitz(const cbct_geometry *geom, int level, int n_iter, double *d_L,
                                 void *d_ws, size_t ws_bytes, void *stream);

/* ---- full reconstruction (Algorithm A1 + multigrid) --------------------- */

/* Bytes of workspace every call above needs for this geometry and params
 * (params may be NULL: single level). */
cbct_status cbct_workspace_size(const cbct_geometry *geom, const cbct_recon_params *params,
                                size_t *bytes);

/* Minimise E2 + lambda E1 s.t. f >= 0 (Eq. 2) by Algorithm A1 under the
 * coarse-to-fine schedule of Sec. II.C.3. d_sino: measured line integrals.
 * d_vol: on entry the start on the coarsest grid is zero (d_vol is ignored
 * on entry when n_levels > 1, used as the start when n_levels == 1); on exit
 * the finest-grid result. d_stats (device, optional). All work is enqueued
 * on the stream; nothing waits on the host. */
cbct_status cbct_reconstruct(const cbct_geometry *geom, const float *d_sino, float *d_vol,
                             const cbct_recon_params *params, void *d_ws, size_t ws_bytes,
                             cbct_recon_stats *d_stats, void *stream);

/* Same with HOST buffers: copies h_sino in, reconstructs, copies the result
 * to h_vol and the statistics to h_stats (optional), and waits for the
 * stream. The workspace must hold cbct_workspace_size_host bytes. */
cbct_status cbct_workspace_size_host(const cbct_geometry *geom, const cbct_recon_params *params,
                                     size_t *bytes);
cbct_status cbct_reconstruct_host(const cbct_geometry *geom, const float *h_sino, float *h_vol,
                                  const cbct_recon_params *params, void *d_ws, size_t ws_bytes,
                                  cbct_recon_stats *h_stats, void *stream);

/* ---- serving: a native scheduler for streams of scans -------------------
 *
 * The paper reconstructs one scan at a time; this runtime (no counterpart in
 * the paper) serves a stream of independent scans on one GPU. It owns one
 * device arena, allocated once at creation, from which each admitted scan
 * receives a resident slot (sinogram, volume, workspace, statistics). A scan
 * is admitted, in arrival order, when its slot fits in the arena (an idle
 * slot of the same geometry and parameters is reused; idle slots of other
 * shapes are evicted, least recently used first, to make room). Admitted
 * scans are copied in on a host-to-device stream, reconstructed on one of
 * `concurrency` compute streams (the one with the least work queued), and
 * copied out on that stream's device-to-host stream, so copies overlap
 * computation and small scans share the GPU. The TV step is a grid-wide
 * cooperative kernel; with concurrency k each solve's grid takes 1/k of the
 * GPU's resident capacity, so k solves fit at once, and its sums do not
 * depend on the grid size, so a served scan equals the same scan
 * reconstructed directly, bit for bit. With use_graphs, the
 * first reconstruction in a slot is captured as a CUDA graph and every later
 * scan in that slot replays it (one launch per scan). With reuse_steps, the
 * per-level step sizes that a scan's power iterations find (they depend on
 * the geometry and the parameters only, not on the data) are kept per
 * (geometry, parameters) pair, and later scans of the pair run with those
 * taus given instead of repeating the power iterations; the kernels are
 * deterministic, so such a scan still equals the direct reconstruction bit
 * for bit, and its statistics report the same tau and L.
 *
 * Host buffers must be page-locked (cudaHostAlloc / cudaHostRegister) and stay
 * valid, like the geometry, until the scan's cbct_server_wait returns. Slots
 * are matched to geometries by a serial number given at creation, so a slot
 * is never reused for a new geometry that happens to share an address. All
 * entry points are thread-safe. While a server exists its worker threads
 * launch kernels; kernel profiling (cbct_profile_*) does not see them. */
typedef struct cbct_server cbct_server;

typedef struct {
    size_t arena_bytes;   /* device bytes for resident scans; 0: half the free memory, at most 64 GiB */
    int max_resident;     /* resident slots at most (0: no limit) */
    int use_graphs;       /* 1: capture each slot's reconstruction once and replay it */
    int concurrency;      /* reconstructions in flight at once, each on its own compute stream
                             with its TV solves on 1/concurrency of the GPU (0 or 1: one at a time) */
    int reuse_steps;      /* 1: reuse each (geometry, parameters) pair's power-iteration taus */
} cbct_server_config;

typedef struct {
    uint64_t ticket;
    int32_t status;         /* cbct_status of the scan */
    int32_t graph_replay;   /* 1: ran as a replay of the slot's captured graph */
    uint32_t recon_flags;   /* cbct_recon_stats.flags */
    int32_t slot;           /* slot index it ran in */
    double t_submit, t_admit, t_done;  /* host seconds since server creation */
    double gpu_ms;          /* device time of the reconstruction (CUDA events) */
    int32_t steps_reused;   /* 1: ran with the taus of an earlier scan of its geometry */
} cbct_scan_result;

typedef struct {
    size_t arena_bytes, bytes_in_use, peak_bytes_in_use;
    int32_t slots, busy_slots, graphs_captured, graph_failures;
    int64_t submitted, completed, evictions;
    int64_t step_reuses;    /* scans that ran with reused taus */
} cbct_server_info;

cbct_status cbct_server_create(const cbct_server_config *cfg, cbct_server **out);
/* Waits for every submitted scan, then frees the arena, graphs and threads. */
void cbct_server_destroy(cbct_server *server);
/* Queue one scan: reconstruct h_sino (page-locked, n_views*nv*nu floats)
 * with params (no replay schedule) into h_vol (page-locked, nx*ny*nz floats);
 * h_stats (page-locked, optional). Rejects a scan whose slot cannot fit in
 * the arena even when it is empty (CBCT_ERR_OUT_OF_MEMORY). */
cbct_status cbct_server_submit(cbct_server *server, const cbct_geometry *geom, const cbct_recon_params *params,
                               const float *h_sino, float *h_vol, cbct_recon_stats *h_stats, uint64_t *ticket);
/* Block until the scan is done and its result is in h_vol; fills *result.
 * Each ticket can be waited for once. */
cbct_status cbct_server_wait(cbct_server *server, uint64_t ticket, cbct_scan_result *result);
cbct_status cbct_server_query(cbct_server *server, cbct_server_info *info);

/* ---- diagnostics -------------------------------------------------------- */

/* Message of the last failing call on this thread ("" if none). */
const char *cbct_last_error(void);
/* Library kernel launches since load (all threads). */
int64_t cbct_launch_count(void);
/* Gather microbenchmark for the measurement of the projector pair (no
 * counterpart in the paper): n_lines warps each walk an in-plane line of
 * n_samples samples through d_vol (nx*ny*nz floats, z fastest, device,
 * every size >= 2), their 32 lanes taking 32 neighbouring detector rows, and
 * every lane gathers one trilinear footprint (8 values, 32 bytes) per
 * sample with plain read-only loads. Writes one sum per lane to d_out
 * (n_lines*32 floats, device). Time it on the stream to get the gather rate,
 * n_lines * 32 * n_samples footprints per launch. */
cbct_status cbct_gather_bench(const float *d_vol, int nx, int ny, int nz, int n_lines, int n_samples,
                              float *d_out, void *stream);
/* Per-kernel timing with CUDA events on the launch stream: while enabled,
 * every launch is bracketed by two events; cbct_profile_collect waits for
 * them and adds their durations to per-kernel totals. Kernel ids
 * 0 .. cbct_profile_kernels()-1. Launches from several host threads are
 * recorded safely (each thread pairs its own events); collect, query and
 * reset while no launch is being issued. */
cbct_status cbct_profile_enable(int on);
cbct_status cbct_profile_collect(void);
int cbct_profile_kernels(void);
const char *cbct_profile_name(int kernel);
cbct_status cbct_profile_query(int kernel, int64_t *launches, double *total_ms);
/* The same restricted to launches made by a reconstruction on multigrid
 * level `level` (0 = finest), or outside any reconstruction (level -1). */
cbct_status cbct_profile_query_level(int kernel, int level, int64_t *launches, double *total_ms);
void cbct_profile_reset(void);

#ifdef __cplusplus
}
#endif
#endif /* CBCT_H */
