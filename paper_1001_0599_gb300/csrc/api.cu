// C ABI of libcbct: argument checks, the geometry handle, workspace layout
// and the host-side drivers (Algorithm A1 under the multigrid schedule of
// Sec. II.C.3; power iteration for the step size). All device work is
// enqueued on the caller's stream; nothing waits on the host except
// cbct_reconstruct_host and the profiling collector.
#include "cbct_internal.cuh"

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <vector>

using namespace cbct;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static cbct_status fail(cbct_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

static cbct_status ok()
{
    g_err.clear();
    return CBCT_OK;
}

#define CUDA_TRY(call)                                                                              \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail(CBCT_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,     \
                        __LINE__);                                                                  \
    } while (0)

// ---------------------------------------------------------------------------
// launch bookkeeping and profiling
// ---------------------------------------------------------------------------
namespace {
std::atomic<int64_t> g_launches{0};
struct ProfSlot {
    int kernel;
    int level;     // multigrid level of the launch (0 = finest), -1 outside a reconstruction
    bool done;     // both events recorded
    cudaEvent_t start, stop;
};
std::atomic<bool> g_prof_on{false};
thread_local bool t_quiet = false;   // threads whose launches the profiler skips
// Event pairs, reused across collections. A deque keeps references stable
// while other threads append; g_prof_mutex guards the pool, the counters
// and the totals, and each thread remembers the slot its open launch took,
// so launches from several host threads pair their own events.
std::mutex g_prof_mutex;
std::deque<ProfSlot> g_pool;
size_t g_pool_used = 0;
thread_local long t_slot = -1;
// per kernel and level slot (slot 0: outside a reconstruction, slot l + 1: level l)
int64_t g_prof_count[K_COUNT][CBCT_MAX_LEVELS + 1] = {};
double g_prof_ms[K_COUNT][CBCT_MAX_LEVELS + 1] = {};
thread_local int t_level = -1;   // level the calling thread's reconstruction is on
const char *g_names[K_COUNT] = {"forward_project", "forward_residual", "back_project",
                                "back_project_step", "rof_persistent", "reduce",
                                "prolongate", "fill", "misc", "eq6_gradient"};
} // namespace

namespace cbct {
void launch_begin(int kernel, cudaStream_t s)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_prof_on.load(std::memory_order_relaxed) || t_quiet) return;
    ProfSlot *p = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_prof_mutex);
        if (g_pool_used == g_pool.size()) {
            ProfSlot q{};
            if (cudaEventCreate(&q.start) != cudaSuccess || cudaEventCreate(&q.stop) != cudaSuccess) return;
            g_pool.push_back(q);
        }
        t_slot = (long)g_pool_used++;
        p = &g_pool[(size_t)t_slot];
        p->kernel = kernel;
        p->level = t_level;
        p->done = false;
    }
    cudaEventRecord(p->start, s);
}

void note_extra_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_thread_quiet(bool quiet) { t_quiet = quiet; }

void launch_end(int kernel, cudaStream_t s)
{
    if (t_slot < 0) return;
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    if ((size_t)t_slot < g_pool_used && g_pool[(size_t)t_slot].kernel == kernel) {
        ProfSlot &p = g_pool[(size_t)t_slot];
        cudaEventRecord(p.stop, s);
        p.done = true;
    }
    t_slot = -1;
}
} // namespace cbct

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
struct LevelData {
    bool ok;
    VolGeom vg;
    RayCol *d_cols;
    double drho;
    double dx, dy, dz;
    Eq6Geom eq6;
};

struct cbct_geometry {
    uint64_t serial;           // unique per created geometry
    cbct_geometry_desc desc;
    std::vector<double> angles;
    int device;
    DetGeom det;
    float2 *d_views;
    float4 *d_views_df;        // (cos, sin) as double-float pairs (Eq. 6 kernel)
    int n_levels;
    LevelData lev[CBCT_MAX_LEVELS];
};

// a double as a double-float pair (hi = nearest float, lo = the remainder)
static DF df_of(double x)
{
    const float h = (float)x;
    return DF{h, (float)(x - (double)h)};
}

static double support_radius(int nx, int ny, double dx, double dy)
{
    return std::sqrt(std::pow(0.5 * (nx + 1) * dx, 2) + std::pow(0.5 * (ny + 1) * dy, 2));
}

static bool build_level_table(const cbct_geometry_desc &d, const double *angles, int nx, int ny,
                              double dx, double dy, double drho, std::vector<RayCol> &out)
{
    out.resize((size_t)d.n_views * d.nu);
    const double X = 0.5 * (nx + 1) * dx, Y = 0.5 * (ny + 1) * dy;
    for (int k = 0; k < d.n_views; k++) {
        const double c = std::cos(angles[k]), s = std::sin(angles[k]);
        const double Sx = -d.sad * c, Sy = -d.sad * s;
        for (int iu = 0; iu < d.nu; iu++) {
            const double u = (iu - 0.5 * (d.nu - 1)) * d.du;
            const double Px = (d.sdd - d.sad) * c + u * s, Py = (d.sdd - d.sad) * s - u * c;
            const double nxr = Px - Sx, nyr = Py - Sy;
            const double lxy = std::hypot(nxr, nyr);
            const double ex = nxr / lxy, ey = nyr / lxy;
            const double rho_c = -(Sx * ex + Sy * ey);
            const double mx = Sx + rho_c * ex, my = Sy + rho_c * ey;
            const long long kc = std::llround(rho_c / drho);
            const double delta = rho_c - (double)kc * drho;
            double lo = -1e300, hi = 1e300;
            bool empty = false;
            if (std::fabs(ex) > 1e-15) {
                double t1 = (-X - Sx) / ex, t2 = (X - Sx) / ex;
                lo = std::max(lo, std::min(t1, t2));
                hi = std::min(hi, std::max(t1, t2));
            } else if (!(Sx > -X && Sx < X)) {
                empty = true;
            }
            if (std::fabs(ey) > 1e-15) {
                double t1 = (-Y - Sy) / ey, t2 = (Y - Sy) / ey;
                lo = std::max(lo, std::min(t1, t2));
                hi = std::min(hi, std::max(t1, t2));
            } else if (!(Sy > -Y && Sy < Y)) {
                empty = true;
            }
            RayCol rc{};
            rc.mx = (float)mx;
            rc.my = (float)my;
            rc.ex = (float)ex;
            rc.ey = (float)ey;
            rc.delta = (float)delta;
            rc.inv_lxy = (float)(1.0 / lxy);
            rc.kc = (int)kc;
            if (empty || !(lo < hi)) {
                rc.jlo = 1;
                rc.jhi = 0;
            } else {
                const long long jl = (long long)std::floor(lo / drho) - 1 - kc;
                const long long jh = (long long)std::ceil(hi / drho) + 1 - kc;
                if (jl < -32767 || jh > 32767) return false;
                rc.jlo = (int16_t)jl;
                rc.jhi = (int16_t)jh;
            }
            out[(size_t)k * d.nu + iu] = rc;
        }
    }
    return true;
}

static cbct_status check_desc(const cbct_geometry_desc *d)
{
    if (!d) return fail(CBCT_ERR_INVALID_ARG, "desc is NULL");
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || d->nu < 1 || d->nv < 1 || d->n_views < 1)
        return fail(CBCT_ERR_INVALID_ARG, "sizes must be >= 1");
    if ((double)d->nx * d->ny * d->nz >= 2147483648.0 || (double)d->n_views * d->nu * d->nv > 4.0e9)
        return fail(CBCT_ERR_INVALID_ARG, "volume must stay below 2^31 voxels, sinogram below 4e9 pixels");
    if (d->n_views > 65535) return fail(CBCT_ERR_INVALID_ARG, "n_views above 65535");
    if (!(d->dx > 0 && d->dy > 0 && d->dz > 0 && d->du > 0 && d->dv > 0))
        return fail(CBCT_ERR_INVALID_ARG, "pitches must be > 0");
    if (!(d->step_ratio >= 0) || d->step_ratio > 16)
        return fail(CBCT_ERR_INVALID_ARG, "step_ratio must be in [0, 16]");
    if (!d->angles) return fail(CBCT_ERR_INVALID_ARG, "angles is NULL");
    for (int k = 0; k < d->n_views; k++)
        if (!std::isfinite(d->angles[k])) return fail(CBCT_ERR_INVALID_ARG, "angle %d not finite", k);
    if (!(std::isfinite(d->sad) && std::isfinite(d->sdd)))
        return fail(CBCT_ERR_INVALID_ARG, "sad/sdd not finite");
    const double R = support_radius(d->nx, d->ny, d->dx, d->dy);
    if (!(d->sad - R > 0 && d->sdd > d->sad + R))
        return fail(CBCT_ERR_INVALID_ARG,
                    "volume support (radius %.3f mm) must lie strictly between source and detector", R);
    return CBCT_OK;
}

extern "C" cbct_status cbct_geometry_create(const cbct_geometry_desc *desc, cbct_geometry **out)
{
    if (!out) return fail(CBCT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    cbct_status st = check_desc(desc);
    if (st != CBCT_OK) return st;
    cbct_geometry *G = new (std::nothrow) cbct_geometry();
    if (!G) return fail(CBCT_ERR_OUT_OF_MEMORY, "host allocation failed");
    static std::atomic<uint64_t> next_serial{1};
    G->serial = next_serial.fetch_add(1);
    G->desc = *desc;
    if (G->desc.step_ratio == 0) G->desc.step_ratio = 0.5;
    G->angles.assign(desc->angles, desc->angles + desc->n_views);
    G->desc.angles = G->angles.data();
    const cbct_geometry_desc &d = G->desc;
    if (cudaGetDevice(&G->device) != cudaSuccess) {
        delete G;
        return fail(CBCT_ERR_CUDA, "no CUDA device");
    }
    auto cleanup = [&]() {
        for (auto &L : G->lev)
            if (L.d_cols) cudaFree(L.d_cols);
        if (G->d_views) cudaFree(G->d_views);
        if (G->d_views_df) cudaFree(G->d_views_df);
        delete G;
    };
    std::vector<float2> views(d.n_views);
    for (int k = 0; k < d.n_views; k++) views[k] = make_float2((float)std::cos(d.angles[k]), (float)std::sin(d.angles[k]));
    if (cudaMalloc(&G->d_views, sizeof(float2) * d.n_views) != cudaSuccess) {
        cleanup();
        return fail(CBCT_ERR_OUT_OF_MEMORY, "cudaMalloc of the view table failed");
    }
    if (cudaMemcpy(G->d_views, views.data(), sizeof(float2) * d.n_views, cudaMemcpyHostToDevice) != cudaSuccess) {
        cleanup();
        return fail(CBCT_ERR_CUDA, "copy of the view table failed");
    }
    std::vector<float4> views_df(d.n_views);
    for (int k = 0; k < d.n_views; k++) {
        const DF c = df_of(std::cos(d.angles[k])), sn = df_of(std::sin(d.angles[k]));
        views_df[k] = make_float4(c.hi, c.lo, sn.hi, sn.lo);
    }
    if (cudaMalloc(&G->d_views_df, sizeof(float4) * d.n_views) != cudaSuccess) {
        cleanup();
        return fail(CBCT_ERR_OUT_OF_MEMORY, "cudaMalloc of the view table failed");
    }
    if (cudaMemcpy(G->d_views_df, views_df.data(), sizeof(float4) * d.n_views, cudaMemcpyHostToDevice) !=
        cudaSuccess) {
        cleanup();
        return fail(CBCT_ERR_CUDA, "copy of the view table failed");
    }
    DetGeom &det = G->det;
    det.nu = d.nu;
    det.nv = d.nv;
    det.n_views = d.n_views;
    det.du = (float)d.du;
    det.dv = (float)d.dv;
    det.inv_du = (float)(1.0 / d.du);
    det.inv_dv = (float)(1.0 / d.dv);
    det.cu = (float)(0.5 * (d.nu - 1));
    det.cv = (float)(0.5 * (d.nv - 1));
    det.sad = (float)d.sad;
    det.sdd = (float)d.sdd;
    det.views = G->d_views;

    G->n_levels = 0;
    std::vector<RayCol> table;
    for (int l = 0; l < CBCT_MAX_LEVELS; l++) {
        LevelData &L = G->lev[l];
        L.ok = false;
        const int f = 1 << l;
        if (l > 0 && (d.nx % f || d.ny % f || d.nz % f)) break;
        const int nx = d.nx / f, ny = d.ny / f, nz = d.nz / f;
        const double dx = d.dx * f, dy = d.dy * f, dz = d.dz * f;
        if (l > 0) {
            const double R = support_radius(nx, ny, dx, dy);
            if (!(d.sad - R > 0 && d.sdd > d.sad + R)) break;
        }
        const double drho = d.step_ratio * std::min(dx, dy);
        if (!build_level_table(d, d.angles, nx, ny, dx, dy, drho, table)) {
            if (l == 0) {
                cleanup();
                return fail(CBCT_ERR_UNSUPPORTED, "more than 32767 samples per ray; raise step_ratio");
            }
            break;
        }
        if (cudaMalloc(&L.d_cols, sizeof(RayCol) * table.size()) != cudaSuccess) {
            cleanup();
            return fail(CBCT_ERR_OUT_OF_MEMORY, "cudaMalloc of the ray table failed");
        }
        if (cudaMemcpy(L.d_cols, table.data(), sizeof(RayCol) * table.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            cleanup();
            return fail(CBCT_ERR_CUDA, "copy of the ray table failed");
        }
        VolGeom &v = L.vg;
        v.nx = nx;
        v.ny = ny;
        v.nz = nz;
        v.dx = (float)dx;
        v.dy = (float)dy;
        v.dz = (float)dz;
        v.inv_dx = (float)(1.0 / dx);
        v.inv_dy = (float)(1.0 / dy);
        v.inv_dz = (float)(1.0 / dz);
        v.cx = (float)(0.5 * (nx - 1));
        v.cy = (float)(0.5 * (ny - 1));
        v.cz = (float)(0.5 * (nz - 1));
        v.drho = (float)drho;
        v.cols = L.d_cols;
        v.bp_cap = 0;
        v.bs_cap = 0;
        v.bp_zc = 0;
        v.bp_zc = bp_choose_zc(v, det, d.angles);
        v.bp_cap = bp_patch_floats(v, det, d.angles);
        v.bs_cap = bs_patch_floats(v, det, d.angles);
        L.drho = drho;
        L.dx = dx;
        L.dy = dy;
        L.dz = dz;
        Eq6Geom &e = L.eq6;
        e.dx = df_of(dx);
        e.dy = df_of(dy);
        e.dz = df_of(dz);
        e.cx = v.cx;
        e.cy = v.cy;
        e.cz = v.cz;
        e.sad = df_of(d.sad);
        e.ku = df_of(d.sdd / d.du);
        e.kv = df_of(d.sdd / d.dv);
        e.cu = det.cu;
        e.cv = det.cv;
        e.two_l0sq = (float)(2.0 * d.sdd * d.sdd);
        e.views = G->d_views_df;
        L.ok = true;
        G->n_levels = l + 1;
    }
    *out = G;
    return ok();
}

extern "C" void cbct_geometry_destroy(cbct_geometry *G)
{
    if (!G) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != G->device) cudaSetDevice(G->device);
    for (auto &L : G->lev)
        if (L.d_cols) cudaFree(L.d_cols);
    if (G->d_views) cudaFree(G->d_views);
    if (G->d_views_df) cudaFree(G->d_views_df);
    if (prev >= 0 && prev != G->device) cudaSetDevice(prev);
    delete G;
}

extern "C" cbct_status cbct_geometry_level_dims(const cbct_geometry *G, int level, int *nx, int *ny, int *nz)
{
    if (!G || !nx || !ny || !nz) return fail(CBCT_ERR_INVALID_ARG, "NULL argument");
    if (level < 0 || level >= G->n_levels)
        return fail(CBCT_ERR_UNSUPPORTED, "level %d not available (grid has %d levels)", level, G->n_levels);
    *nx = G->lev[level].vg.nx;
    *ny = G->lev[level].vg.ny;
    *nz = G->lev[level].vg.nz;
    return ok();
}

// ---------------------------------------------------------------------------
// argument checks
// ---------------------------------------------------------------------------
static cbct_status check_geom(const cbct_geometry *G)
{
    if (!G) return fail(CBCT_ERR_INVALID_ARG, "geometry is NULL");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(CBCT_ERR_CUDA, "no CUDA device");
    if (dev != G->device)
        return fail(CBCT_ERR_INVALID_ARG, "geometry belongs to device %d, current device is %d", G->device, dev);
    return CBCT_OK;
}

static cbct_status check_ptr(const void *p, const char *name)
{
    if (!p) return fail(CBCT_ERR_INVALID_ARG, "%s is NULL", name);
    if (((uintptr_t)p) & 15u) return fail(CBCT_ERR_INVALID_ARG, "%s is not 16-byte aligned", name);
    return CBCT_OK;
}

#define CHECK(x)                                                                                    \
    do {                                                                                            \
        cbct_status s_ = (x);                                                                       \
        if (s_ != CBCT_OK) return s_;                                                               \
    } while (0)

static size_t nvox(const VolGeom &v) { return (size_t)v.nx * v.ny * v.nz; }
static size_t nray(const DetGeom &d) { return (size_t)d.n_views * d.nv * d.nu; }
static double kappa_of(const VolGeom &v, const DetGeom &d) { return 2.0 * (double)nvox(v) / (double)nray(d); }

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
struct Layout {
    size_t state, partials, r, g, d, split, eig, coarse[CBCT_MAX_LEVELS], replay, stats, hsino, hvol, ysto, fsto,
        total;
    int n_partials;
};

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

static Layout layout(const cbct_geometry *G, const cbct_recon_params *p, bool host_variant)
{
    Layout L{};
    size_t off = 0;
    const VolGeom &v0 = G->lev[0].vg;
    L.state = off;
    off = align_up(off + sizeof(DevState));
    int np = fp_grid_blocks(G->det);
    for (int l = 0; l < G->n_levels; l++) np = std::max(np, bp_grid_blocks(G->lev[l].vg));
    np = std::max(np, 4 * rof_bricks(v0.nx, v0.ny, v0.nz));
    L.n_partials = np;
    L.partials = off;
    off = align_up(off + sizeof(double) * (size_t)np);
    L.r = off;
    off = align_up(off + sizeof(float) * nray(G->det));
    L.g = off;
    off = align_up(off + sizeof(float) * nvox(v0));
    L.d = off;
    off = align_up(off + sizeof(float) * nvox(v0));
    size_t split = 0;
    for (int l = 0; l < G->n_levels; l++) split = std::max(split, bp_split_floats(G->lev[l].vg, G->det));
    L.split = off;
    off = align_up(off + sizeof(float) * split);
    // last power iterate of a coarse level, kept for the next level's warm start
    L.eig = off;
    if (G->n_levels > 1) off = align_up(off + sizeof(float) * nvox(G->lev[1].vg));
    const int levels = p ? std::max(1, std::min(p->n_levels, CBCT_MAX_LEVELS)) : 1;
    for (int l = 1; l < levels && l < G->n_levels; l++) {
        L.coarse[l] = off;
        off = align_up(off + sizeof(float) * nvox(G->lev[l].vg));
    }
    L.replay = off;
    if (p && p->replay && p->replay_len > 0) off = align_up(off + sizeof(int32_t) * (size_t)p->replay_len);
    // reduced storage: the measured sinogram and the projector's volume copy
    L.ysto = L.fsto = off;
    if (p && p->storage != CBCT_STORAGE_F32) {
        L.ysto = off;
        off = align_up(off + 2 * nray(G->det));
        L.fsto = off;
        off = align_up(off + 2 * nvox(v0));
    }
    if (host_variant) {
        L.stats = off;
        off = align_up(off + sizeof(cbct_recon_stats));
        L.hsino = off;
        off = align_up(off + sizeof(float) * nray(G->det));
        L.hvol = off;
        off = align_up(off + sizeof(float) * nvox(v0));
    }
    L.total = off;
    return L;
}

template <typename T>
static T *at(void *ws, size_t off)
{
    return reinterpret_cast<T *>(static_cast<char *>(ws) + off);
}

static cbct_status check_ws(const cbct_geometry *G, const cbct_recon_params *p, void *ws, size_t bytes,
                            bool host_variant)
{
    CHECK(check_ptr(ws, "workspace"));
    if (((uintptr_t)ws) & 255u) return fail(CBCT_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    const Layout L = layout(G, p, host_variant);
    if (bytes < L.total)
        return fail(CBCT_ERR_WORKSPACE_TOO_SMALL, "workspace has %zu bytes, needs %zu", bytes, L.total);
    return CBCT_OK;
}

extern "C" cbct_status cbct_workspace_size(const cbct_geometry *G, const cbct_recon_params *p, size_t *bytes)
{
    CHECK(check_geom(G));
    if (!bytes) return fail(CBCT_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = layout(G, p, false).total;
    return ok();
}

extern "C" cbct_status cbct_workspace_size_host(const cbct_geometry *G, const cbct_recon_params *p, size_t *bytes)
{
    CHECK(check_geom(G));
    if (!bytes) return fail(CBCT_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = layout(G, p, true).total;
    return ok();
}

// ---------------------------------------------------------------------------
// projector entry points
// ---------------------------------------------------------------------------
extern "C" cbct_status cbct_forward_project(const cbct_geometry *G, const float *d_vol, float *d_sino, void *stream)
{
    CHECK(check_geom(G));
    CHECK(check_ptr(d_vol, "d_vol"));
    CHECK(check_ptr(d_sino, "d_sino"));
    CUDA_TRY(launch_forward(G->lev[0].vg, G->det, d_vol, nullptr, d_sino, nullptr, nullptr, 0,
                            (cudaStream_t)stream));
    return ok();
}

extern "C" cbct_status cbct_residual(const cbct_geometry *G, const float *d_vol, const float *d_y, float *d_r,
                                     double *d_sumsq, void *ws, size_t ws_bytes, void *stream)
{
    CHECK(check_geom(G));
    CHECK(check_ptr(d_vol, "d_vol"));
    CHECK(check_ptr(d_y, "d_y"));
    CHECK(check_ptr(d_r, "d_r"));
    if (!d_sumsq) return fail(CBCT_ERR_INVALID_ARG, "d_sumsq is NULL");
    CHECK(check_ws(G, nullptr, ws, ws_bytes, false));
    const Layout L = layout(G, nullptr, false);
    cudaStream_t s = (cudaStream_t)stream;
    double *partials = at<double>(ws, L.partials);
    CUDA_TRY(launch_forward(G->lev[0].vg, G->det, d_vol, d_y, d_r, nullptr, partials, 1, s));
    CUDA_TRY(launch_sum_partials(partials, fp_partials_count(G->lev[0].vg, G->det), 1, 1, d_sumsq, s));
    return ok();
}

extern "C" cbct_status cbct_back_project(const cbct_geometry *G, const float *d_sino, float *d_vol, void *stream)
{
    CHECK(check_geom(G));
    CHECK(check_ptr(d_sino, "d_sino"));
    CHECK(check_ptr(d_vol, "d_vol"));
    CUDA_TRY(launch_back(G->lev[0].vg, G->det, d_sino, nullptr, d_vol, nullptr, 0.0, 0.0, nullptr, 0, 0, nullptr,
                         (cudaStream_t)stream));
    return ok();
}

static cbct_status check_storage(int st)
{
    if (st < CBCT_STORAGE_F32 || st > CBCT_STORAGE_F16)
        return fail(CBCT_ERR_INVALID_ARG, "storage must be a cbct_storage value");
    return CBCT_OK;
}

extern "C" cbct_status cbct_forward_project_ex(const cbct_geometry *G, const void *d_vol, void *d_sino, int storage,
                                               void *stream)
{
    CHECK(check_geom(G));
    CHECK(check_ptr(d_vol, "d_vol"));
    CHECK(check_ptr(d_sino, "d_sino"));
    CHECK(check_storage(storage));
    if (!fp_supports_storage(G->lev[0].vg, G->det, storage))
        return fail(CBCT_ERR_UNSUPPORTED, "reduced storage needs nv <= 1024 and nz <= 760");
    CUDA_TRY(launch_forward_st(G->lev[0].vg, G->det, d_vol, nullptr, d_sino, storage, nullptr, nullptr, 0,
                               (cudaStream_t)stream));
    return ok();
}

extern "C" cbct_status cbct_back_project_ex(const cbct_geometry *G, const void *d_sino, int storage, float *d_vol,
                                            void *stream)
{
    CHECK(check_geom(G));
    CHECK(check_ptr(d_sino, "d_sino"));
    CHECK(check_ptr(d_vol, "d_vol"));
    CHECK(check_storage(storage));
    CUDA_TRY(launch_back_st(G->lev[0].vg, G->det, d_sino, storage, nullptr, d_vol, nullptr, 0.0, 0.0, nullptr, 0, 0,
                            nullptr, (cudaStream_t)stream));
    return ok();
}

extern "C" cbct_status cbct_convert(const void *d_src, int src_storage, void *d_dst, int dst_storage, size_t n,
                                    void *stream)
{
    CHECK(check_storage(src_storage));
    CHECK(check_storage(dst_storage));
    if (n > 0 && (!d_src || !d_dst)) return fail(CBCT_ERR_INVALID_ARG, "NULL device pointer");
    CUDA_TRY(launch_convert(d_src, src_storage, d_dst, dst_storage, n, (cudaStream_t)stream));
    return ok();
}

extern "C" cbct_status cbct_eq6_gradient(const cbct_geometry *G, const float *d_T, float *d_vol, void *stream)
{
    CHECK(check_geom(G));
    CHECK(check_ptr(d_T, "d_T"));
    CHECK(check_ptr(d_vol, "d_vol"));
    CUDA_TRY(launch_eq6(G->lev[0].vg, G->det, G->lev[0].eq6, d_T, nullptr, d_vol, nullptr, 0.0, 0, (cudaStream_t)stream));
    return ok();
}

extern "C" cbct_status cbct_gradient_step(const cbct_geometry *G, const float *d_r, const float *d_f, float *d_g,
                                          double scale, void *stream)
{
    CHECK(check_geom(G));
    CHECK(check_ptr(d_r, "d_r"));
    CHECK(check_ptr(d_f, "d_f"));
    CHECK(check_ptr(d_g, "d_g"));
    if (d_g == d_f) return fail(CBCT_ERR_INVALID_ARG, "d_g must not alias d_f");
    if (!std::isfinite(scale)) return fail(CBCT_ERR_INVALID_ARG, "scale not finite");
    CUDA_TRY(launch_back(G->lev[0].vg, G->det, d_r, d_f, d_g, nullptr, scale, 0.0, nullptr, 1, 0, nullptr,
                         (cudaStream_t)stream));
    return ok();
}

// ---------------------------------------------------------------------------
// TV / ROF entry points
// ---------------------------------------------------------------------------
static RofArgs rof_base(const cbct_geometry *G, int level, void *ws, const Layout &L)
{
    const VolGeom &v = G->lev[level].vg;
    RofArgs a{};
    a.partials = at<double>(ws, L.partials);
    a.st = at<DevState>(ws, L.state);
    a.nx = v.nx;
    a.ny = v.ny;
    a.nz = v.nz;
    a.inv_dx = v.inv_dx;
    a.inv_dy = v.inv_dy;
    a.inv_dz = v.inv_dz;
    a.level = level;
    return a;
}

static cbct_status check_tv_scalars(double lambda, double tau, double eps)
{
    if (!(std::isfinite(lambda) && lambda >= 0)) return fail(CBCT_ERR_INVALID_ARG, "lambda must be finite, >= 0");
    if (!(std::isfinite(tau) && tau > 0)) return fail(CBCT_ERR_INVALID_ARG, "tau must be finite, > 0");
    if (!(std::isfinite(eps) && eps >= 0)) return fail(CBCT_ERR_INVALID_ARG, "eps_tv must be finite, >= 0");
    return CBCT_OK;
}

static cbct_status check_tv_params(const cbct_tv_params *p)
{
    if (!p) return fail(CBCT_ERR_INVALID_ARG, "tv params NULL");
    if (!(p->c > 0 && p->c < 1)) return fail(CBCT_ERR_INVALID_ARG, "Armijo c must be in (0, 1)");
    if (!(p->alpha > 0 && p->alpha < 1)) return fail(CBCT_ERR_INVALID_ARG, "alpha must be in (0, 1)");
    if (!(p->rel_tol >= 0 && std::isfinite(p->rel_tol))) return fail(CBCT_ERR_INVALID_ARG, "rel_tol must be >= 0");
    if (p->max_inner < 1 || p->max_inner > 100000) return fail(CBCT_ERR_INVALID_ARG, "max_inner out of range");
    if (p->max_backtracks < 0 || p->max_backtracks > 1000)
        return fail(CBCT_ERR_INVALID_ARG, "max_backtracks out of range");
    if (!std::isfinite(p->s0)) return fail(CBCT_ERR_INVALID_ARG, "s0 not finite");
    if (!(std::isfinite(p->eps_tv) && p->eps_tv >= 0)) return fail(CBCT_ERR_INVALID_ARG, "eps_tv must be >= 0");
    return CBCT_OK;
}

extern "C" cbct_status cbct_tv_energy_grad(const cbct_geometry *G, const float *d_f, const float *d_g, double lambda,
                                           double tau, double eps_tv, float *d_d, double *d_out, void *ws,
                                           size_t ws_bytes, void *stream)
{
    CHECK(check_geom(G));
    CHECK(check_ptr(d_f, "d_f"));
    CHECK(check_ptr(d_g, "d_g"));
    CHECK(check_ptr(d_d, "d_d"));
    if (!d_out) return fail(CBCT_ERR_INVALID_ARG, "d_out is NULL");
    CHECK(check_tv_scalars(lambda, tau, eps_tv));
    CHECK(check_ws(G, nullptr, ws, ws_bytes, false));
    const Layout L = layout(G, nullptr, false);
    RofArgs a = rof_base(G, 0, ws, L);
    a.g = d_g;
    a.cur = d_f;
    a.d = d_d;
    a.lambda = lambda;
    a.tau = tau;
    a.eps = eps_tv;
    a.mode = 1;
    a.out = d_out;
    CUDA_TRY(launch_rof(a, (cudaStream_t)stream));
    return ok();
}

extern "C" cbct_status cbct_check_barrier_timeout(const cbct_geometry *G, void *ws, size_t ws_bytes,
                                                  cbct_tv_stats *d_stats, void *stream)
{
    CHECK(check_geom(G));
    if (!d_stats) return fail(CBCT_ERR_INVALID_ARG, "d_stats is NULL");
    CHECK(check_ws(G, nullptr, ws, ws_bytes, false));
    const Layout L = layout(G, nullptr, false);
    cudaStream_t s = (cudaStream_t)stream;
    const VolGeom &v = G->lev[0].vg;
    float *g = at<float>(ws, L.g), *d = at<float>(ws, L.d);
    CUDA_TRY(launch_fill(g, nvox(v), 0.f, s));
    RofArgs a = rof_base(G, 0, ws, L);
    a.g = g;
    a.cur = g;
    a.d = d;
    a.lambda = 1.0;
    a.tau = 1.0;
    a.eps = 1e-3;
    a.mode = 1;
    a.out = at<double>(ws, L.partials);   // the energies never arrive; any scratch will do
    a.tv_stats = d_stats;
    a.withhold_arrival = 1;
    CUDA_TRY(launch_rof(a, s));
    return ok();
}

extern "C" cbct_status cbct_tv_trial(const cbct_geometry *G, const float *d_f, const float *d_d, const float *d_g,
                                     double s, double lambda, double tau, double eps_tv, double *d_out, void *ws,
                                     size_t ws_bytes, void *stream)
{
    CHECK(check_geom(G));
    CHECK(check_ptr(d_f, "d_f"));
    CHECK(check_ptr(d_d, "d_d"));
    CHECK(check_ptr(d_g, "d_g"));
    if (!d_out) return fail(CBCT_ERR_INVALID_ARG, "d_out is NULL");
    if (!std::isfinite(s)) return fail(CBCT_ERR_INVALID_ARG, "s not finite");
    CHECK(check_tv_scalars(lambda, tau, eps_tv));
    CHECK(check_ws(G, nullptr, ws, ws_bytes, false));
    const Layout L = layout(G, nullptr, false);
    RofArgs a = rof_base(G, 0, ws, L);
    a.g = d_g;
    a.cur = d_f;
    a.dir = d_d;
    a.trial_s = s;
    a.lambda = lambda;
    a.tau = tau;
    a.eps = eps_tv;
    a.mode = 2;
    a.out = d_out;
    CUDA_TRY(launch_rof(a, (cudaStream_t)stream));
    return ok();
}

static void fill_tv(RofArgs &a, const cbct_tv_params *p)
{
    a.eps = p->eps_tv;
    a.c = p->c;
    a.alpha = p->alpha;
    a.rel_tol = p->rel_tol;
    a.max_inner = p->max_inner;
    a.max_bt = p->max_backtracks;
    a.s0 = p->s0;
}

extern "C" cbct_status cbct_tv_denoise(const cbct_geometry *G, const float *d_g, float *d_f, double lambda,
                                       double tau, const cbct_tv_params *p, void *ws, size_t ws_bytes,
                                       cbct_tv_stats *d_stats, void *stream)
{
    CHECK(check_geom(G));
    CHECK(check_ptr(d_g, "d_g"));
    CHECK(check_ptr(d_f, "d_f"));
    if (d_f == d_g) return fail(CBCT_ERR_INVALID_ARG, "d_f must not alias d_g");
    CHECK(check_tv_params(p));
    CHECK(check_tv_scalars(lambda, tau, p->eps_tv));
    CHECK(check_ws(G, nullptr, ws, ws_bytes, false));
    const Layout L = layout(G, nullptr, false);
    RofArgs a = rof_base(G, 0, ws, L);
    a.g = d_g;
    a.f = d_f;
    a.d = at<float>(ws, L.d);
    a.lambda = lambda;
    a.tau = tau;
    fill_tv(a, p);
    a.start_at_g = 0;
    a.clamp = 0;
    a.mode = 0;
    a.tv_stats = d_stats;
    CUDA_TRY(launch_rof(a, (cudaStream_t)stream));
    return ok();
}

// ---------------------------------------------------------------------------
// multigrid and step size
// ---------------------------------------------------------------------------
extern "C" cbct_status cbct_prolongate(int ncx, int ncy, int ncz, const float *d_coarse, float *d_fine, void *stream)
{
    if (ncx < 1 || ncy < 1 || ncz < 1) return fail(CBCT_ERR_INVALID_ARG, "sizes must be >= 1");
    CHECK(check_ptr(d_coarse, "d_coarse"));
    CHECK(check_ptr(d_fine, "d_fine"));
    CUDA_TRY(launch_prolong(ncx, ncy, ncz, d_coarse, d_fine, (cudaStream_t)stream));
    return ok();
}

// power iteration on level `level`; w and s live in the workspace (g and r).
// warm: start from the prolongation of the previous (coarser) level's last
// iterate held in the eig buffer instead of from ones.
static cbct_status run_power(const cbct_geometry *G, int level, int n_iter, void *ws, const Layout &L,
                             double *d_L_out, cudaStream_t s, bool warm = false)
{
    const VolGeom &v = G->lev[level].vg;
    DevState *st = at<DevState>(ws, L.state);
    float *w = at<float>(ws, L.g);
    float *sino = at<float>(ws, L.r);
    double *partials = at<double>(ws, L.partials);
    const double kappa = kappa_of(v, G->det);
    if (warm) {
        const VolGeom &vc = G->lev[level + 1].vg;
        CUDA_TRY(launch_prolong(vc.nx, vc.ny, vc.nz, at<float>(ws, L.eig), w, s));
        CUDA_TRY(launch_sumsq(w, nvox(v), partials, 1024, &st->vnorm2, s));
        CUDA_TRY(launch_power_init(st, 0.0, s));
    } else {
        CUDA_TRY(launch_power_init(st, (double)nvox(v), s));
        CUDA_TRY(launch_fill(w, nvox(v), 1.f, s));
    }
    for (int it = 0; it < n_iter; it++) {
        // projection pre-weighted by ds (mode 3) feeds the transpose's staged patch directly
        CUDA_TRY(launch_forward(v, G->det, w, nullptr, sino, &st->inv_wnorm, nullptr, 3, s));
        CUDA_TRY(launch_back(v, G->det, sino, nullptr, w, nullptr, 0.0, kappa, partials, 2, 1,
                             at<float>(ws, L.split), s));
        CUDA_TRY(launch_power_update(st, partials, bp_partials_count(v, G->det, true), kappa, it == 0,
                                     it == n_iter - 1, d_L_out, s));
    }
    return CBCT_OK;
}

extern "C" cbct_status cbct_power_lipschitz(const cbct_geometry *G, int level, int n_iter, double *d_L, void *ws,
                                            size_t ws_bytes, void *stream)
{
    CHECK(check_geom(G));
    if (level < 0 || level >= G->n_levels) return fail(CBCT_ERR_UNSUPPORTED, "level %d not available", level);
    if (n_iter < 1 || n_iter > 10000) return fail(CBCT_ERR_INVALID_ARG, "n_iter out of range");
    if (!d_L) return fail(CBCT_ERR_INVALID_ARG, "d_L is NULL");
    CHECK(check_ws(G, nullptr, ws, ws_bytes, false));
    const Layout L = layout(G, nullptr, false);
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(launch_state_init(at<DevState>(ws, L.state), nullptr, s));
    CHECK(run_power(G, level, n_iter, ws, L, d_L, s));
    return ok();
}

// ---------------------------------------------------------------------------
// reconstruction driver
// ---------------------------------------------------------------------------
static cbct_status check_recon_params(const cbct_geometry *G, const cbct_recon_params *p,
                                      std::vector<int> &replay_off)
{
    if (!p) return fail(CBCT_ERR_INVALID_ARG, "params NULL");
    if (p->n_levels < 1 || p->n_levels > CBCT_MAX_LEVELS)
        return fail(CBCT_ERR_INVALID_ARG, "n_levels must be in 1..%d", CBCT_MAX_LEVELS);
    if (p->n_levels > G->n_levels)
        return fail(CBCT_ERR_UNSUPPORTED, "grid supports %d multigrid levels, %d requested", G->n_levels, p->n_levels);
    if (!(std::isfinite(p->lambda) && p->lambda >= 0)) return fail(CBCT_ERR_INVALID_ARG, "lambda must be >= 0");
    int total = 0;
    for (int l = 0; l < p->n_levels; l++) {
        if (p->iters[l] < 0 || p->iters[l] > CBCT_MAX_ITERS)
            return fail(CBCT_ERR_INVALID_ARG, "iters[%d] out of range", l);
        if (!std::isfinite(p->tau[l])) return fail(CBCT_ERR_INVALID_ARG, "tau[%d] not finite", l);
        total += p->iters[l];
    }
    if (total > CBCT_MAX_ITERS) return fail(CBCT_ERR_INVALID_ARG, "more than %d iterations", CBCT_MAX_ITERS);
    if (p->power_iters < 0 || p->power_iters > 10000) return fail(CBCT_ERR_INVALID_ARG, "power_iters out of range");
    if (p->power_iters_fine < 0 || p->power_iters_fine > 10000)
        return fail(CBCT_ERR_INVALID_ARG, "power_iters_fine out of range");
    if (p->gradient_mode != 0 && p->gradient_mode != 1)
        return fail(CBCT_ERR_INVALID_ARG, "gradient_mode must be 0 (matched P^T) or 1 (Eq. 6)");
    if (p->storage < CBCT_STORAGE_F32 || p->storage > CBCT_STORAGE_F16)
        return fail(CBCT_ERR_INVALID_ARG, "storage must be a cbct_storage value");
    if (p->storage != CBCT_STORAGE_F32) {
        if (p->gradient_mode != 0) return fail(CBCT_ERR_UNSUPPORTED, "reduced storage takes the matched gradient");
        for (int l = 0; l < p->n_levels; l++)
            if (!fp_supports_storage(G->lev[l].vg, G->det, p->storage))
                return fail(CBCT_ERR_UNSUPPORTED, "reduced storage needs nv <= 1024 and nz <= 760");
    }
    CHECK(check_tv_params(&p->tv));
    replay_off.clear();
    if (p->replay) {
        if (p->replay_len < total) return fail(CBCT_ERR_INVALID_ARG, "replay too short");
        int pos = 0;
        for (int k = 0; k < total; k++) {
            if (pos >= p->replay_len) return fail(CBCT_ERR_INVALID_ARG, "replay too short at iteration %d", k);
            const int n = p->replay[pos];
            if (n < 0 || pos + 1 + n > p->replay_len || n > 100000)
                return fail(CBCT_ERR_INVALID_ARG, "bad replay record at iteration %d", k);
            for (int i = 0; i < n; i++)
                if (p->replay[pos + 1 + i] < 0 || p->replay[pos + 1 + i] > 1000)
                    return fail(CBCT_ERR_INVALID_ARG, "bad replay step count");
            replay_off.push_back(pos);
            pos += 1 + n;
        }
    }
    return CBCT_OK;
}

static cbct_status recon_core(const cbct_geometry *G, const float *d_sino, float *d_vol, const cbct_recon_params *p,
                              void *ws, const Layout &L, cbct_recon_stats *d_stats,
                              const std::vector<int> &replay_off, bool zero_start, cudaStream_t s)
{
    struct LevelTag {   // profiler level tag, cleared on every exit
        ~LevelTag() { t_level = -1; }
    } level_tag;
    DevState *st = at<DevState>(ws, L.state);
    double *partials = at<double>(ws, L.partials);
    float *r = at<float>(ws, L.r);
    float *g = at<float>(ws, L.g);
    float *d = at<float>(ws, L.d);
    const int32_t *d_replay = nullptr;
    if (p->replay) {
        int32_t *dr = at<int32_t>(ws, L.replay);
        CUDA_TRY(cudaMemcpyAsync(dr, p->replay, sizeof(int32_t) * (size_t)p->replay_len, cudaMemcpyHostToDevice, s));
        d_replay = dr;
    }
    CUDA_TRY(launch_state_init(st, d_stats, s));
    const int sto = p->storage;
    void *ysto = at<void>(ws, L.ysto), *fsto = at<void>(ws, L.fsto);
    if (sto != CBCT_STORAGE_F32) CUDA_TRY(launch_convert(d_sino, CBCT_STORAGE_F32, ysto, sto, nray(G->det), s));
    const int Lv = p->n_levels;
    const int power_iters = p->power_iters > 0 ? p->power_iters : 20;
    float *prev = nullptr;
    int k = 0;
    int eig_level = -1;   // geometry level whose last power iterate sits in the eig buffer
    for (int lev = 0; lev < Lv; lev++) {
        const int gl = Lv - 1 - lev;  // geometry level: 0 = finest
        const VolGeom &v = G->lev[gl].vg;
        t_level = gl;
        float *f = gl == 0 ? d_vol : at<float>(ws, L.coarse[gl]);
        if (lev == 0) {
            if (Lv > 1 || zero_start) CUDA_TRY(launch_fill(f, nvox(v), 0.f, s));
        } else {
            const VolGeom &vc = G->lev[gl + 1].vg;
            CUDA_TRY(launch_prolong(vc.nx, vc.ny, vc.nz, prev, f, s));
        }
        const double kappa = kappa_of(v, G->det);
        if (!(p->tau[lev] > 0)) {
            const bool warm = p->power_iters_fine > 0 && eig_level == gl + 1;
            CHECK(run_power(G, gl, warm ? p->power_iters_fine : power_iters, ws, L, nullptr, s, warm));
            if (p->power_iters_fine > 0 && gl > 0) {
                CUDA_TRY(cudaMemcpyAsync(at<float>(ws, L.eig), at<float>(ws, L.g), sizeof(float) * nvox(v),
                                         cudaMemcpyDeviceToDevice, s));
                eig_level = gl;
            }
        }
        CUDA_TRY(launch_set_tau(st, p->tau[lev] > 0 ? p->tau[lev] : 0.0, kappa, d_stats, lev, s));
        const double inv_m = 1.0 / (double)nray(G->det);
        for (int it = 0; it < p->iters[lev]; it++, k++) {
            if (p->gradient_mode == 1) {
                // Step 1 with the paper's closed-form gradient (Eq. 6) in place of P^T:
                // P^T T tends to (voxel volume / (2 du dv)) G(T) (Eq. 6 carries a factor 2)
                CUDA_TRY(launch_forward(v, G->det, f, d_sino, r, nullptr, partials, 1, s));
                CUDA_TRY(launch_e2(partials, fp_partials_count(v, G->det), inv_m, st, s));
                const double eq6_factor = G->lev[gl].dx * G->lev[gl].dy * G->lev[gl].dz / (2.0 * G->desc.du * G->desc.dv);
                CUDA_TRY(launch_eq6(v, G->det, G->lev[gl].eq6, r, f, g, &st->scale, eq6_factor, 1, s));
            } else if (sto != CBCT_STORAGE_F32) {
                // Step 1 with y, r and the projector's copy of f stored as `sto`; after
                // the level's first iteration the ROF solve wrote that copy with f
                if (it == 0) CUDA_TRY(launch_convert(f, CBCT_STORAGE_F32, fsto, sto, nvox(v), s));
                CUDA_TRY(launch_forward_st(v, G->det, fsto, ysto, r, sto, nullptr, partials, 2, s));
                CUDA_TRY(launch_e2(partials, fp_partials_count(v, G->det), inv_m, st, s));
                CUDA_TRY(launch_back_st(v, G->det, r, sto, f, g, &st->scale, 0.0, 0.0, nullptr, 1, 1,
                                        at<float>(ws, L.split), s));
            } else {
                // Step 1: r = ds (P f - y), E2; g = f - tau kappa P^T r
                CUDA_TRY(launch_forward(v, G->det, f, d_sino, r, nullptr, partials, 2, s));
                CUDA_TRY(launch_e2(partials, fp_partials_count(v, G->det), inv_m, st, s));
                CUDA_TRY(launch_back(v, G->det, r, f, g, &st->scale, 0.0, 0.0, nullptr, 1, 1, at<float>(ws, L.split),
                                     s));
            }
            // Steps 2-3: ROF from g, clamp fused into its last update
            RofArgs a = rof_base(G, gl, ws, L);
            a.g = g;
            a.f = f;
            a.d = d;
            a.lambda = p->lambda;
            a.tau = 0.0;  // the level's step lives on the device (power iteration)
            fill_tv(a, &p->tv);
            a.start_at_g = 1;
            a.clamp = p->clamp ? 1 : 0;
            a.mode = 0;
            a.recon_stats = d_stats;
            a.replay = d_replay ? d_replay + replay_off[k] : nullptr;
            a.level = lev;
            a.tau_dev = &st->tau;
            if (sto != CBCT_STORAGE_F32 && p->gradient_mode != 1) {
                a.f_store = fsto;
                a.store_type = sto;
            }
            CUDA_TRY(launch_rof(a, s));
        }
        prev = f;
    }
    return CBCT_OK;
}

extern "C" cbct_status cbct_reconstruct(const cbct_geometry *G, const float *d_sino, float *d_vol,
                                        const cbct_recon_params *p, void *ws, size_t ws_bytes,
                                        cbct_recon_stats *d_stats, void *stream)
{
    CHECK(check_geom(G));
    CHECK(check_ptr(d_sino, "d_sino"));
    CHECK(check_ptr(d_vol, "d_vol"));
    std::vector<int> replay_off;
    CHECK(check_recon_params(G, p, replay_off));
    CHECK(check_ws(G, p, ws, ws_bytes, false));
    const Layout L = layout(G, p, false);
    CHECK(recon_core(G, d_sino, d_vol, p, ws, L, d_stats, replay_off, false, (cudaStream_t)stream));
    return ok();
}

extern "C" cbct_status cbct_reconstruct_host(const cbct_geometry *G, const float *h_sino, float *h_vol,
                                             const cbct_recon_params *p, void *ws, size_t ws_bytes,
                                             cbct_recon_stats *h_stats, void *stream)
{
    CHECK(check_geom(G));
    if (!h_sino || !h_vol) return fail(CBCT_ERR_INVALID_ARG, "host buffers must not be NULL");
    std::vector<int> replay_off;
    CHECK(check_recon_params(G, p, replay_off));
    CHECK(check_ws(G, p, ws, ws_bytes, true));
    const Layout L = layout(G, p, true);
    cudaStream_t s = (cudaStream_t)stream;
    float *dsino = at<float>(ws, L.hsino);
    float *dvol = at<float>(ws, L.hvol);
    cbct_recon_stats *dstats = at<cbct_recon_stats>(ws, L.stats);
    CUDA_TRY(cudaMemcpyAsync(dsino, h_sino, sizeof(float) * nray(G->det), cudaMemcpyHostToDevice, s));
    CHECK(recon_core(G, dsino, dvol, p, ws, L, dstats, replay_off, true, s));
    CUDA_TRY(cudaMemcpyAsync(h_vol, dvol, sizeof(float) * nvox(G->lev[0].vg), cudaMemcpyDeviceToHost, s));
    if (h_stats) CUDA_TRY(cudaMemcpyAsync(h_stats, dstats, sizeof(cbct_recon_stats), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return ok();
}

// ---------------------------------------------------------------------------
// diagnostics
// ---------------------------------------------------------------------------
extern "C" const char *cbct_last_error(void) { return g_err.c_str(); }

extern "C" int64_t cbct_launch_count(void) { return g_launches.load(); }

extern "C" cbct_status cbct_gather_bench(const float *d_vol, int nx, int ny, int nz, int n_lines, int n_samples,
                                         float *d_out, void *stream)
{
    if (!d_vol || !d_out) return fail(CBCT_ERR_INVALID_ARG, "NULL device pointer");
    if (nx < 2 || ny < 2 || nz < 2 || n_lines < 1 || n_samples < 1)
        return fail(CBCT_ERR_INVALID_ARG, "volume must be at least 2 voxels along each axis, lines and samples >= 1");
    CUDA_TRY(launch_gather(d_vol, nx, ny, nz, n_lines, n_samples, d_out, (cudaStream_t)stream));
    return ok();
}

extern "C" cbct_status cbct_profile_enable(int on)
{
    g_prof_on = on != 0;
    return ok();
}

extern "C" cbct_status cbct_profile_collect(void)
{
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    for (size_t i = 0; i < g_pool_used; i++) {
        ProfSlot &p = g_pool[i];
        if (!p.done) continue;   // a launch that failed before its end event
        CUDA_TRY(cudaEventSynchronize(p.stop));
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, p.start, p.stop));
        const int slot = (p.level >= 0 && p.level < CBCT_MAX_LEVELS) ? p.level + 1 : 0;
        g_prof_ms[p.kernel][slot] += ms;
        g_prof_count[p.kernel][slot] += 1;
    }
    g_pool_used = 0;
    return ok();
}

extern "C" int cbct_profile_kernels(void) { return K_COUNT; }

extern "C" const char *cbct_profile_name(int k) { return (k >= 0 && k < K_COUNT) ? g_names[k] : ""; }

extern "C" cbct_status cbct_profile_query(int k, int64_t *launches, double *total_ms)
{
    if (k < 0 || k >= K_COUNT || !launches || !total_ms) return fail(CBCT_ERR_INVALID_ARG, "bad kernel id");
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    *launches = 0;
    *total_ms = 0.0;
    for (int l = 0; l <= CBCT_MAX_LEVELS; l++) {
        *launches += g_prof_count[k][l];
        *total_ms += g_prof_ms[k][l];
    }
    return ok();
}

extern "C" cbct_status cbct_profile_query_level(int k, int level, int64_t *launches, double *total_ms)
{
    if (k < 0 || k >= K_COUNT || !launches || !total_ms || level < -1 || level >= CBCT_MAX_LEVELS)
        return fail(CBCT_ERR_INVALID_ARG, "bad kernel id or level");
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    *launches = g_prof_count[k][level + 1];
    *total_ms = g_prof_ms[k][level + 1];
    return ok();
}

extern "C" void cbct_profile_reset(void)
{
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    for (int k = 0; k < K_COUNT; k++) {
        for (int l = 0; l <= CBCT_MAX_LEVELS; l++) {
            g_prof_count[k][l] = 0;
            g_prof_ms[k][l] = 0.0;
        }
    }
    g_pool_used = 0;
}

// ---------------------------------------------------------------------------
// accessors for other translation units
// ---------------------------------------------------------------------------
namespace cbct {
const VolGeom *geometry_level(const cbct_geometry *g, int level)
{
    return (g && level >= 0 && level < g->n_levels) ? &g->lev[level].vg : nullptr;
}
const DetGeom *geometry_detector(const cbct_geometry *g) { return g ? &g->det : nullptr; }
int geometry_device(const cbct_geometry *g) { return g ? g->device : -1; }
uint64_t geometry_serial(const cbct_geometry *g) { return g ? g->serial : 0; }
cbct_status report_error(cbct_status st, const char *msg)
{
    if (st == CBCT_OK) return ok();
    return fail(st, "%s", msg);
}
} // namespace cbct
