// ROF sub-problem of Algorithm A1 (Step 2, Sec. II.B) as one persistent,
// cooperatively launched kernel for sm_103a.
//
// E_ROF[f] = lambda mean(phi) + (1/(2 tau)) mean((f - g)^2),
// phi_k = sqrt(eps^2 + |D f_k|^2), forward differences with zero ghosts on
// the + side of x and y and a reflective ghost on z (Sec. II.B).
// d = N_vox dE_ROF/df = lambda (div_backward q) + (f - g)/tau, q = D f / phi.
//
// Gradient descent with Armijo backtracking (Eq. 5) needs a global sum
// between every sweep and a data-dependent decision after it. Instead of a
// host round trip per trial, every block of a co-resident grid runs the same
// loop; a bounded grid barrier lets the last-arriving block add the
// per-block FP64 partials in a fixed order and publish the totals, which
// all blocks then read, so all take the same decision. Each sweep works on
// 8 x 8 x 32 voxel bricks staged with a one-voxel halo in shared memory.
#include "cbct_internal.cuh"

#include <mutex>

#include <cooperative_groups.h>

namespace cbct {

constexpr int BX = 8, BY = 8, BZ = 32;
constexpr int HX = BX + 2, HY = BY + 2, HZ = BZ + 2;
constexpr int TV_THREADS = 256;
constexpr int TV_WARPS = TV_THREADS / 32;
constexpr int PER_THREAD = BX * BY / TV_WARPS;       // (x, y) positions per lane
constexpr unsigned long long BARRIER_LIMIT_NS = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_volatile_u32(const unsigned int *p)
{
    return *(const volatile unsigned int *)p;
}

struct TvShared {
    float F[HX * HY * HZ];
    double red[32 * 4];
    double res[8];
    int flag_last;
    unsigned int gen;
    int err;
};

// Grid barrier; when K > 0 the last block to arrive sums K partials per block
// (fixed order, FP64) into st->red before releasing the others. Every wait is
// bounded; on timeout the error flag is raised and the caller leaves.
template <int K>
__device__ bool grid_sync(DevState *st, const double *partials, TvShared &sh)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        sh.gen = ld_volatile_u32(&st->bar.gen);
        __threadfence();
        const unsigned int arrived = atomicAdd(&st->bar.count, 1u);
        sh.flag_last = (arrived == gridDim.x - 1);
    }
    __syncthreads();
    if (sh.flag_last) {
        __threadfence();
        if (K > 0) {
            double acc[K > 0 ? K : 1];
#pragma unroll
            for (int k = 0; k < K; k++) acc[k] = 0.0;
            for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
                for (int k = 0; k < K; k++) acc[k] += __ldcg(partials + (size_t)b * 4 + k);
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
            for (int k = 0; k < K; k++) {
                double v = acc[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) sh.red[warp * 4 + k] = v;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
#pragma unroll
                for (int k = 0; k < K; k++) {
                    double s = 0.0;
                    for (int w = 0; w < TV_WARPS; w++) s += sh.red[w * 4 + k];
                    st->red[k] = s;
                }
            }
        }
        if (threadIdx.x == 0) {
            __threadfence();
            atomicExch(&st->bar.count, 0u);
            __threadfence();
            atomicAdd(&st->bar.gen, 1u);
        }
    } else if (threadIdx.x == 0) {
        const unsigned long long t0 = globaltimer_ns();
        unsigned int spins = 0;
        while (ld_volatile_u32(&st->bar.gen) == sh.gen) {
            if ((++spins & 63u) == 0 && globaltimer_ns() - t0 > BARRIER_LIMIT_NS) {
                atomicExch(&st->bar.error, 1);
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sh.err = *(volatile int *)&st->bar.error;
#pragma unroll
        for (int k = 0; k < K; k++) sh.res[k] = *(volatile double *)&st->red[k];
    }
    __syncthreads();
    return sh.err == 0;
}

struct BrickIdx {
    int nbx, nby, nbz, total;
};

__device__ __forceinline__ BrickIdx brick_count(const RofArgs &a)
{
    BrickIdx b;
    b.nbx = (a.nx + BX - 1) / BX;
    b.nby = (a.ny + BY - 1) / BY;
    b.nbz = (a.nz + BZ - 1) / BZ;
    b.total = b.nbx * b.nby * b.nbz;
    return b;
}

// Stage cur - s*dir (dir may be null) on the brick plus a one-voxel halo;
// points outside the grid hold 0 (they are never used as values: the
// boundary rules are applied explicitly).
__device__ __forceinline__ void stage(const RofArgs &a, TvShared &sh, const float *cur,
                                      const float *dir, float s, int x0, int y0, int z0)
{
    for (int i = threadIdx.x; i < HX * HY * HZ; i += blockDim.x) {
        const int hz = i % HZ;
        const int rest = i / HZ;
        const int hy = rest % HY, hx = rest / HY;
        const int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = z0 - 1 + hz;
        float v = 0.f;
        if (gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz) {
            const size_t idx = ((size_t)gx * a.ny + gy) * a.nz + gz;
            v = __ldcg(cur + idx);
            if (dir) v = __fmaf_rn(-s, __ldcg(dir + idx), v);
        }
        sh.F[i] = v;
    }
}

__device__ __forceinline__ int hidx(int hx, int hy, int hz) { return (hx * HY + hy) * HZ + hz; }

// D f at grid point (gx, gy, gz) held at halo position (hx, hy, hz)
__device__ __forceinline__ void fdiff(const RofArgs &a, const float *F, int hx, int hy, int hz, int gx,
                                      int gy, int gz, float &Dx, float &Dy, float &Dz)
{
    const float fk = F[hidx(hx, hy, hz)];
    const float fxp = (gx + 1 < a.nx) ? F[hidx(hx + 1, hy, hz)] : 0.f;
    const float fyp = (gy + 1 < a.ny) ? F[hidx(hx, hy + 1, hz)] : 0.f;
    const float fzp = (gz + 1 < a.nz) ? F[hidx(hx, hy, hz + 1)] : fk;
    Dx = (fxp - fk) * a.inv_dx;
    Dy = (fyp - fk) * a.inv_dy;
    Dz = (fzp - fk) * a.inv_dz;
}

// Sweep computing d, the energy and mean(d^2) partials (returns the block's
// contributions in v[0], v[1]).
__device__ void sweep_grad(const RofArgs &a, TvShared &sh, const float *cur, float *dout, DF (&v)[2])
{
    const BrickIdx bi = brick_count(a);
    const float lam = (float)a.lambda, inv_tau = (float)(1.0 / a.tau);
    const float inv_2tau = (float)(0.5 / a.tau), eps2 = (float)(a.eps * a.eps);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int br = blockIdx.x; br < bi.total; br += gridDim.x) {
        const int bz = br % bi.nbz, t = br / bi.nbz;
        const int by = t % bi.nby, bx = t / bi.nby;
        const int x0 = bx * BX, y0 = by * BY, z0 = bz * BZ;
        stage(a, sh, cur, nullptr, 0.f, x0, y0, z0);
        __syncthreads();
        float e_part = 0.f, d2_part = 0.f;
#pragma unroll 2
        for (int i = 0; i < PER_THREAD; i++) {
            const int p = warp + i * TV_WARPS;
            const int lx = p % BX, ly = p / BX;
            const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lane;
            if (gx >= a.nx || gy >= a.ny || gz >= a.nz) continue;
            const int hx = lx + 1, hy = ly + 1, hz = lane + 1;
            float Dx, Dy, Dz;
            fdiff(a, sh.F, hx, hy, hz, gx, gy, gz, Dx, Dy, Dz);
            const float phi = sqrtf(eps2 + Dx * Dx + Dy * Dy + Dz * Dz);
            const float inv_phi = 1.f / phi;
            float div = -(Dx * inv_phi) * a.inv_dx - (Dy * inv_phi) * a.inv_dy - (Dz * inv_phi) * a.inv_dz;
            if (gx > 0) {
                float ex, ey, ez;
                fdiff(a, sh.F, hx - 1, hy, hz, gx - 1, gy, gz, ex, ey, ez);
                div += ex / sqrtf(eps2 + ex * ex + ey * ey + ez * ez) * a.inv_dx;
            }
            if (gy > 0) {
                float ex, ey, ez;
                fdiff(a, sh.F, hx, hy - 1, hz, gx, gy - 1, gz, ex, ey, ez);
                div += ey / sqrtf(eps2 + ex * ex + ey * ey + ez * ez) * a.inv_dy;
            }
            if (gz > 0) {
                float ex, ey, ez;
                fdiff(a, sh.F, hx, hy, hz - 1, gx, gy, gz - 1, ex, ey, ez);
                div += ez / sqrtf(eps2 + ex * ex + ey * ey + ez * ez) * a.inv_dz;
            }
            const size_t idx = ((size_t)gx * a.ny + gy) * a.nz + gz;
            const float fj = sh.F[hidx(hx, hy, hz)];
            const float diff = fj - __ldg(a.g + idx);
            const float dj = lam * div + diff * inv_tau;
            dout[idx] = dj;
            e_part += lam * phi + diff * diff * inv_2tau;
            d2_part += dj * dj;
        }
        v[0] = df_add(v[0], e_part);
        v[1] = df_add(v[1], d2_part);
        __syncthreads();
    }
}

// Sweep computing the partial energy of cur - s*dir.
__device__ void sweep_trial(const RofArgs &a, TvShared &sh, const float *cur, const float *dir, float s,
                            DF &v)
{
    const BrickIdx bi = brick_count(a);
    const float lam = (float)a.lambda, inv_2tau = (float)(0.5 / a.tau);
    const float eps2 = (float)(a.eps * a.eps);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int br = blockIdx.x; br < bi.total; br += gridDim.x) {
        const int bz = br % bi.nbz, t = br / bi.nbz;
        const int by = t % bi.nby, bx = t / bi.nby;
        const int x0 = bx * BX, y0 = by * BY, z0 = bz * BZ;
        stage(a, sh, cur, dir, s, x0, y0, z0);
        __syncthreads();
        float e_part = 0.f;
#pragma unroll 2
        for (int i = 0; i < PER_THREAD; i++) {
            const int p = warp + i * TV_WARPS;
            const int lx = p % BX, ly = p / BX;
            const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lane;
            if (gx >= a.nx || gy >= a.ny || gz >= a.nz) continue;
            float Dx, Dy, Dz;
            fdiff(a, sh.F, lx + 1, ly + 1, lane + 1, gx, gy, gz, Dx, Dy, Dz);
            const float phi = sqrtf(eps2 + Dx * Dx + Dy * Dy + Dz * Dz);
            const size_t idx = ((size_t)gx * a.ny + gy) * a.nz + gz;
            const float diff = sh.F[hidx(lx + 1, ly + 1, lane + 1)] - __ldg(a.g + idx);
            e_part += lam * phi + diff * diff * inv_2tau;
        }
        v = df_add(v, e_part);
        __syncthreads();
    }
}

// f = cur - s*dir (dir may be null: copy), optionally clamped at 0.
__device__ void sweep_update(const RofArgs &a, const float *cur, const float *dir, float s, float *f,
                             bool clamp)
{
    const size_t n = (size_t)a.nx * a.ny * a.nz;
    const size_t n4 = n / 4;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const float4 *c4 = reinterpret_cast<const float4 *>(cur);
    const float4 *d4 = reinterpret_cast<const float4 *>(dir);
    float4 *f4 = reinterpret_cast<float4 *>(f);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        float4 c = __ldcg(c4 + i);
        if (dir) {
            const float4 dd = __ldcg(d4 + i);
            c.x = __fmaf_rn(-s, dd.x, c.x);
            c.y = __fmaf_rn(-s, dd.y, c.y);
            c.z = __fmaf_rn(-s, dd.z, c.z);
            c.w = __fmaf_rn(-s, dd.w, c.w);
        }
        if (clamp) {
            c.x = fmaxf(c.x, 0.f);
            c.y = fmaxf(c.y, 0.f);
            c.z = fmaxf(c.z, 0.f);
            c.w = fmaxf(c.w, 0.f);
        }
        __stcg(f4 + i, c);
    }
    for (size_t i = n4 * 4 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float c = __ldcg(cur + i);
        if (dir) c = __fmaf_rn(-s, __ldcg(dir + i), c);
        if (clamp) c = fmaxf(c, 0.f);
        __stcg(f + i, c);
    }
}

__device__ __forceinline__ void write_partials(const RofArgs &a, TvShared &sh, DF *v, int k)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < k; q++) {
        DF w = df_warp_sum(v[q]);
        if (lane == 0) sh.red[warp * 4 + q] = (double)w.hi + (double)w.lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < k; q++) {
            double s = 0.0;
            for (int w = 0; w < TV_WARPS; w++) s += sh.red[w * 4 + q];
            a.partials[(size_t)blockIdx.x * 4 + q] = s;
        }
    }
    __syncthreads();
}

// 4 resident blocks per SM (64 registers): the brick sweeps are latency-bound,
// and the extra block per SM took a finest-level paper solve 0.52 -> 0.45 ms
__global__ void __launch_bounds__(TV_THREADS, 4)
rof_kernel(RofArgs args)
{
    __shared__ TvShared sh;
    RofArgs a = args;
    if (a.tau_dev) a.tau = *a.tau_dev;
    const double nvox = (double)a.nx * a.ny * a.nz;

    if (a.mode == 1) {  // energy + gradient at a.cur
        DF v[2] = {df_zero(), df_zero()};
        sweep_grad(a, sh, a.cur, a.d, v);
        write_partials(a, sh, v, 2);
        if (!grid_sync<2>(a.st, a.partials, sh)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.out[0] = sh.res[0] / nvox;
            a.out[1] = sh.res[1] / nvox;
        }
        return;
    }
    if (a.mode == 2) {  // trial energy at a.cur - s a.dir
        DF v[1] = {df_zero()};
        sweep_trial(a, sh, a.cur, a.dir, (float)a.trial_s, v[0]);
        write_partials(a, sh, v, 1);
        if (!grid_sync<1>(a.st, a.partials, sh)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) a.out[0] = sh.res[0] / nvox;
        return;
    }

    // full solve
    const bool replay = a.replay != nullptr;
    const int n_steps = replay ? a.replay[0] : a.max_inner;
    const float *cur = a.start_at_g ? a.g : a.f;
    bool wrote_f = !a.start_at_g;
    bool clamped = false;
    int n_inner = 0, bt_total = 0, flags = 0;
    double e_first = 0.0, e_last = 0.0;
    const double s0 = a.s0 > 0.0 ? a.s0 : a.tau;

    for (int it = 0; it < n_steps; ++it) {
        DF v[2] = {df_zero(), df_zero()};
        sweep_grad(a, sh, cur, a.d, v);
        write_partials(a, sh, v, 2);
        if (!grid_sync<2>(a.st, a.partials, sh)) return;
        const double E0 = sh.res[0] / nvox, D2 = sh.res[1] / nvox;
        if (it == 0) e_first = E0;
        e_last = E0;
        if (!replay && (D2 == 0.0 || E0 == 0.0)) break;

        double step = s0, Enew = E0;
        int bt = 0;
        bool accepted = false;
        if (replay) {
            const int m = a.replay[1 + it];
            for (bt = 0; bt < m; bt++) step *= a.alpha;
            accepted = true;
        } else {
            for (bt = 0; bt <= a.max_bt; ++bt) {
                DF e[1] = {df_zero()};
                sweep_trial(a, sh, cur, a.d, (float)step, e[0]);
                write_partials(a, sh, e, 1);
                if (!grid_sync<1>(a.st, a.partials, sh)) return;
                Enew = sh.res[0] / nvox;
                if (Enew <= E0 - a.c * step * D2) {  // Armijo, Eq. 5
                    accepted = true;
                    break;
                }
                step *= a.alpha;
            }
        }
        if (!accepted) {
            flags |= 1;
            break;
        }
        const double rel = replay ? 1.0 : fabs(Enew - E0) / E0;
        const bool stop = replay ? (it == n_steps - 1) : (rel < a.rel_tol || it == n_steps - 1);
        const bool do_clamp = a.clamp && stop;
        sweep_update(a, cur, a.d, (float)step, a.f, do_clamp);
        cur = a.f;
        wrote_f = true;
        clamped = do_clamp;
        if (blockIdx.x == 0 && threadIdx.x == 0 && a.recon_stats) {
            const int pos = a.st->step_log_pos;
            if (pos < CBCT_MAX_STEP_LOG) a.recon_stats->steps[pos] = bt;
            a.st->step_log_pos = pos + 1;
        }
        n_inner++;
        bt_total += bt;
        if (!replay) e_last = Enew;
        if (stop) {
            if (!replay && !(rel < a.rel_tol)) flags |= 2;
            break;
        }
        if (!grid_sync<0>(a.st, a.partials, sh)) return;
    }
    if (!wrote_f || (a.clamp && !clamped)) {
        // the loop ended without writing the final iterate: f = clamp(cur)
        if (!grid_sync<0>(a.st, a.partials, sh)) return;
        sweep_update(a, cur, nullptr, 0.f, a.f, a.clamp != 0);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (a.tv_stats) {
            a.tv_stats->n_inner = n_inner;
            a.tv_stats->backtracks = bt_total;
            a.tv_stats->flags = flags;
            a.tv_stats->status = CBCT_OK;
            a.tv_stats->e_first = e_first;
            a.tv_stats->e_last = e_last;
        }
        if (a.recon_stats) {
            const int k = a.st->iter_pos;
            if (k < CBCT_MAX_ITERS) {
                cbct_iter_stats &r = a.recon_stats->iters[k];
                r.e2 = a.st->e2;
                r.e_rof_first = e_first;
                r.e_rof_last = e_last;
                r.level = a.level;
                r.n_inner = n_inner;
                r.backtracks = bt_total;
                r.flags = flags;
            }
            a.st->iter_pos = k + 1;
            a.recon_stats->n_iters = k + 1;
            a.recon_stats->flags |= flags;
            a.recon_stats->n_steps = a.st->step_log_pos < CBCT_MAX_STEP_LOG ? a.st->step_log_pos
                                                                             : CBCT_MAX_STEP_LOG;
        }
    }
}

// status kernel: report a barrier timeout into the stats (runs after rof_kernel)
__global__ void rof_status_kernel(DevState *st, cbct_tv_stats *tv, cbct_recon_stats *rs)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int err = st->bar.error;
        if (err) {
            if (tv) tv->status = CBCT_ERR_TIMEOUT;
            if (rs) rs->status = CBCT_ERR_TIMEOUT;
        }
    }
}

// cooperative grid size of rof_kernel (SMs x resident blocks), per device
static std::mutex g_rof_mutex;
static int g_rof_blocks[64] = {};

int rof_grid_blocks()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 0;
    std::lock_guard<std::mutex> lock(g_rof_mutex);
    int *cached = dev < 64 ? &g_rof_blocks[dev] : nullptr;
    if (cached && *cached) return *cached;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rof_kernel, TV_THREADS, 0);
    if (per_sm < 1) per_sm = 1;
    const int n = sms * per_sm;
    if (cached) *cached = n;
    return n;
}

cudaError_t launch_rof(const RofArgs &a, cudaStream_t s)
{
    const int nbricks = ((a.nx + BX - 1) / BX) * ((a.ny + BY - 1) / BY) * ((a.nz + BZ - 1) / BZ);
    int blocks = rof_grid_blocks();
    if (blocks > nbricks) blocks = nbricks;
    if (blocks < 1) blocks = 1;
    cudaError_t e = cudaMemsetAsync(&a.st->bar, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
    if (a.withhold_arrival) {
        // arrivals start far above the grid size, so none is ever the last
        e = cudaMemsetAsync(&a.st->bar.count, 0x7f, sizeof(unsigned int), s);
        if (e != cudaSuccess) return e;
    }
    RofArgs args = a;
    void *params[] = {&args};
    launch_begin(K_ROF, s);
    e = cudaLaunchCooperativeKernel((const void *)rof_kernel, dim3(blocks), dim3(TV_THREADS), params, 0, s);
    launch_end(K_ROF, s);
    if (e != cudaSuccess) return e;
    if (a.tv_stats || a.recon_stats) {
        launch_begin(K_MISC, s);
        rof_status_kernel<<<1, 32, 0, s>>>(a.st, a.tv_stats, a.recon_stats);
        launch_end(K_MISC, s);
    }
    return cudaGetLastError();
}

} // namespace cbct
