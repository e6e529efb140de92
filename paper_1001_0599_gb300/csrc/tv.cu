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
// loop; a bounded grid barrier lets the last-arriving block add the FP64
// partial sums in a fixed order and publish the totals, which all blocks
// then read, so all take the same decision.
//
// Each sweep works on 8 x 8 x 32 voxel bricks staged with a one-voxel halo
// in shared memory. Bricks are moved by the Tensor Memory Accelerator: a
// 3-D tiled copy (cp.async.bulk.tensor) of a 40 x 10 x 10 box per operand,
// completing on an mbarrier, double-buffered so that the next brick's copy
// is in flight while the current one is computed (the box starts 4 slices
// below the brick, since a tiled copy must start on a 16-byte boundary in
// its innermost dimension; coordinates outside the volume read as zero,
// which is the staging the boundary rules expect). Grids whose z extent or
// buffers do not meet the copy engine's alignment rules stage with plain
// loads instead.
//
// Partial sums are kept per brick, not per block, and the last block adds
// them in brick order, so every result is independent of the grid size:
// a solve launched on part of the GPU (several scans at once) gives the
// same bits as one launched on all of it.
#include "cbct_internal.cuh"

#include <cuda.h>   // CUtensorMap and its enums (types only; the encoder is fetched at run time)

#include <cstring>
#include <mutex>

namespace cbct {

constexpr int BX = 8, BY = 8, BZ = 32;
constexpr int SX = BX + 2, SY = BY + 2;   // staged box: one-voxel halo in x and y
constexpr int SZ0 = 4;                     // slices staged below the brick (16-byte start rule)
constexpr int SZ = BZ + 2 * SZ0;           // 40 staged slices: z0 - 4 .. z0 + 35
constexpr int SBOX = SX * SY * SZ;         // floats per staged operand
constexpr int TV_THREADS = 256;
constexpr int TV_WARPS = TV_THREADS / 32;
constexpr int PER_THREAD = BX * BY / TV_WARPS;       // (x, y) positions per lane
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;   // 2 s
constexpr size_t TV_DYN_SMEM = sizeof(float) * 2 * 2 * SBOX + 1024;  // [stage][cur, dir] + alignment slack
static_assert(SBOX * sizeof(float) % 128 == 0, "staging buffers must stay 128-byte aligned");

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

// Tensor maps of the solve's volumes (built on the host per launch).
enum { MAP_G = 0, MAP_F, MAP_D, MAP_CUR, MAP_DIR, MAP_COUNT };
struct RofMaps {
    CUtensorMap m[MAP_COUNT];
};

struct TvShared {
    unsigned long long mbar[2];   // one per staging buffer
    double red[32 * 4];
    double wsum[2][TV_WARPS][2];   // per-brick warp sums, by brick parity
    double res[8];
    int flag_last;
    unsigned int gen;
    int err;
    int any_fail;
};

__device__ __forceinline__ int sidx(int hx, int hy, int hz) { return (hx * SY + hy) * SZ + hz; }

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---- mbarrier and tensor copies (single-CTA, this GPU's memory only) ----
__device__ __forceinline__ void mbar_init(unsigned long long *b)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ void mbar_expect(unsigned long long *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long *b, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(smem_u32(b)), "r"(parity)
                 : "memory");
    return done != 0;
}

// Bounded wait for the phase with the given parity; false after 2 s.
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, uint32_t parity)
{
    if (mbar_test(b, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned int spin = 1;; ++spin) {
        if (mbar_test(b, parity)) return true;
        if ((spin & 255u) == 0 && globaltimer_ns() - t0 > WAIT_LIMIT_NS) return false;
    }
}

__device__ __forceinline__ void tma_box(float *dst, const CUtensorMap *map, int z, int y, int x,
                                        unsigned long long *b)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(map)), "r"(z), "r"(y), "r"(x), "r"(smem_u32(b))
                 : "memory");
}

// generic-proxy accesses before this point are ordered before later tensor copies
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

// Grid barrier; when K > 0 the last block to arrive sums K partials per item
// over n items (fixed order, FP64) into st->red before releasing the others.
// Every wait is bounded; on timeout the error flag is raised and the caller
// leaves.
template <int K>
__device__ bool grid_sync(DevState *st, const double *partials, int n, TvShared &sh)
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
            for (int b = threadIdx.x; b < n; b += blockDim.x)
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
            if ((++spins & 63u) == 0 && globaltimer_ns() - t0 > WAIT_LIMIT_NS) {
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

__device__ __forceinline__ void brick_origin(const BrickIdx &bi, int br, int &x0, int &y0, int &z0)
{
    const int bz = br % bi.nbz, t = br / bi.nbz;
    const int by = t % bi.nby, bx = t / bi.nby;
    x0 = bx * BX;
    y0 = by * BY;
    z0 = bz * BZ;
}

// ---------------------------------------------------------------------------
// brick staging: buffer b of the double buffer holds cur (or cur - s dir)
// over the 40 x 10 x 10 box of one brick
// ---------------------------------------------------------------------------
struct Pipe {
    int stage;        // buffer that receives the next brick
    uint32_t phase;   // bit b: parity of buffer b's next completion
};

__device__ __forceinline__ float *stage_buf(float *dyn, int b) { return dyn + (size_t)b * 2 * SBOX; }

// Start the copy of brick (x0, y0, z0) into buffer b (tensor path; thread 0).
template <bool DIR>
__device__ __forceinline__ void stage_issue(const RofMaps *mp, int cur_map, int dir_map, float *buf,
                                            unsigned long long *mb, int x0, int y0, int z0)
{
    if (threadIdx.x != 0) return;
    fence_proxy_async();
    mbar_expect(mb, (uint32_t)((DIR ? 2 : 1) * SBOX * sizeof(float)));
    tma_box(buf, &mp->m[cur_map], z0 - SZ0, y0 - 1, x0 - 1, mb);
    if (DIR) tma_box(buf + SBOX, &mp->m[dir_map], z0 - SZ0, y0 - 1, x0 - 1, mb);
}

// Plain loads of the same box (grids the copy engine cannot serve).
template <bool DIR>
__device__ __forceinline__ void stage_plain(const RofArgs &a, float *buf, const float *cur, const float *dir,
                                            float s, int x0, int y0, int z0)
{
    for (int i = threadIdx.x; i < SBOX; i += blockDim.x) {
        const int hz = i % SZ, rest = i / SZ;
        const int hy = rest % SY, hx = rest / SY;
        const int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = z0 - SZ0 + hz;
        float v = 0.f;
        if (gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz) {
            const size_t idx = ((size_t)gx * a.ny + gy) * a.nz + gz;
            v = __ldcg(cur + idx);
            if (DIR) v = __fmaf_rn(-s, __ldcg(dir + idx), v);
        }
        buf[i] = v;
    }
}

// Brick data ready in buffer b (combined to cur - s dir when DIR). Returns
// false, for the whole block, when the copy did not arrive within the limit.
template <bool TMA, bool DIR>
__device__ __forceinline__ bool stage_ready(const RofArgs &a, float *buf, unsigned long long *mb, uint32_t parity,
                                            const float *cur, const float *dir, float s, int x0, int y0, int z0)
{
    if (TMA) {
        const bool ok = mbar_wait(mb, parity);
        if (__syncthreads_or(!ok)) return false;
        if (DIR) {
            for (int i = threadIdx.x; i < SBOX; i += blockDim.x) buf[i] = __fmaf_rn(-s, buf[SBOX + i], buf[i]);
            __syncthreads();
        }
    } else {
        stage_plain<DIR>(a, buf, cur, dir, s, x0, y0, z0);
        __syncthreads();
    }
    return true;
}

// After a copy timed out: raise the error flag and give the other buffer's
// copy in flight (if any) a bounded time to land before the block leaves.
__device__ __forceinline__ void stage_abort(const RofArgs &a, unsigned long long *mb_other, bool other_pending,
                                            uint32_t other_parity)
{
    if (threadIdx.x == 0) {
        atomicExch(&a.st->bar.error, 1);
        if (other_pending) mbar_wait(mb_other, other_parity);
    }
    __syncthreads();
}

// One partial sum per brick and quantity. Each warp's sum (double-float
// over its lanes) goes to shared memory; after the brick's closing barrier
// thread 0 adds the warps in order and writes the brick's partial
// (out = partials + 4 brick), so the block pays no extra barrier for it.
template <int K>
__device__ __forceinline__ void brick_warp_sums(const float (&p)[K], TvShared &sh, int parity)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < K; q++) {
        const DF w = df_warp_sum(DF{p[q], 0.f});
        if (lane == 0) sh.wsum[parity][warp][q] = (double)w.hi + (double)w.lo;
    }
}

template <int K>
__device__ __forceinline__ void brick_flush(const TvShared &sh, int parity, double *out)
{
    if (threadIdx.x != 0) return;
#pragma unroll
    for (int q = 0; q < K; q++) {
        double s = 0.0;
        for (int w = 0; w < TV_WARPS; w++) s += sh.wsum[parity][w][q];
        out[q] = s;
    }
}

// D f at grid point (gx, gy, gz) held at staged position (hx, hy, hz)
__device__ __forceinline__ void fdiff(const RofArgs &a, const float *F, int hx, int hy, int hz, int gx,
                                      int gy, int gz, float &Dx, float &Dy, float &Dz)
{
    const float fk = F[sidx(hx, hy, hz)];
    const float fxp = (gx + 1 < a.nx) ? F[sidx(hx + 1, hy, hz)] : 0.f;
    const float fyp = (gy + 1 < a.ny) ? F[sidx(hx, hy + 1, hz)] : 0.f;
    const float fzp = (gz + 1 < a.nz) ? F[sidx(hx, hy, hz + 1)] : fk;
    Dx = (fxp - fk) * a.inv_dx;
    Dy = (fyp - fk) * a.inv_dy;
    Dz = (fzp - fk) * a.inv_dz;
}

// ---------------------------------------------------------------------------
// sweeps over the bricks, each brick's copy overlapped with the previous
// brick's arithmetic
// ---------------------------------------------------------------------------
struct SweepOps {
    int cur_map, dir_map;       // tensor maps of cur and dir (tensor path)
    const float *cur, *dir;     // the same buffers (plain path)
    float s;                    // the staged volume is cur - s dir when a direction is given
};

// KIND 0: d = N dE_ROF/df at cur, with the energy and mean(d^2) partials;
// KIND 1: the energy partial of cur - s dir.
template <bool TMA, int KIND>
__device__ bool sweep(const RofArgs &a, const RofMaps *mp, TvShared &sh, float *dyn, Pipe &pp, const SweepOps &op,
                      float *dout)
{
    constexpr bool DIR = KIND == 1;
    constexpr int K = KIND == 0 ? 2 : 1;
    const BrickIdx bi = brick_count(a);
    const float lam = (float)a.lambda, inv_tau = (float)(1.0 / a.tau);
    const float inv_2tau = (float)(0.5 / a.tau), eps2 = (float)(a.eps * a.eps);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int br = blockIdx.x;
    if (TMA && br < bi.total) {
        int x0, y0, z0;
        brick_origin(bi, br, x0, y0, z0);
        stage_issue<DIR>(mp, op.cur_map, op.dir_map, stage_buf(dyn, pp.stage), &sh.mbar[pp.stage], x0, y0, z0);
    }
    int prev = -1, it = 0;   // previous brick of this block, and the brick count
    for (; br < bi.total; br += gridDim.x, ++it) {
        const int b = pp.stage;
        const uint32_t par = (pp.phase >> b) & 1u;
        const int nxt = br + gridDim.x;
        if (TMA && nxt < bi.total) {
            int nx0, ny0, nz0;
            brick_origin(bi, nxt, nx0, ny0, nz0);
            stage_issue<DIR>(mp, op.cur_map, op.dir_map, stage_buf(dyn, b ^ 1), &sh.mbar[b ^ 1], nx0, ny0, nz0);
        }
        if (prev >= 0) brick_flush<K>(sh, (it - 1) & 1, a.partials + (size_t)prev * 4);
        int x0, y0, z0;
        brick_origin(bi, br, x0, y0, z0);
        // g of this thread's voxels, loaded before the staged data is awaited
        float gv[PER_THREAD];
#pragma unroll
        for (int i = 0; i < PER_THREAD; i++) {
            const int p = warp + i * TV_WARPS;
            const int gx = x0 + p % BX, gy = y0 + p / BX, gz = z0 + lane;
            gv[i] = (gx < a.nx && gy < a.ny && gz < a.nz) ? __ldg(a.g + ((size_t)gx * a.ny + gy) * a.nz + gz) : 0.f;
        }
        float *F = stage_buf(dyn, b);
        const bool ready = stage_ready<TMA, DIR>(a, F, &sh.mbar[b], par, op.cur, op.dir, op.s, x0, y0, z0);
        if (TMA) {
            pp.phase ^= 1u << b;
            pp.stage ^= 1;
        }
        if (!ready) {
            stage_abort(a, &sh.mbar[b ^ 1], TMA && nxt < bi.total, (pp.phase >> (b ^ 1)) & 1u);
            return false;
        }
        float part[K];
#pragma unroll
        for (int q = 0; q < K; q++) part[q] = 0.f;
        // warp w owns the voxel column lx = w of the brick, lane the slice
        // z0 + lane, and steps through ly = 0..7
        const int lx = warp, gx = x0 + lx, gz = z0 + lane;
        const int hx = lx + 1, hz = lane + SZ0;
        if (gx < a.nx) {   // warp-uniform
            float qy_prev = 0.f;   // q_y of the voxel below in y (KIND 0)
#pragma unroll 2
            for (int i = 0; i < PER_THREAD; i++) {
                const int ly = i, gy = y0 + ly, hy = ly + 1;
                if (gy >= a.ny) break;   // warp-uniform
                float Dx, Dy, Dz;
                fdiff(a, F, hx, hy, hz, gx, gy, gz, Dx, Dy, Dz);
                // phi = sqrt(eps^2 + |D f|^2) and 1/phi from one reciprocal square root
                const float s2 = eps2 + Dx * Dx + Dy * Dy + Dz * Dz;
                const float inv_phi = rsqrtf(s2);
                const float phi = s2 * inv_phi;
                const float diff = F[sidx(hx, hy, hz)] - gv[i];
                const bool live = gz < a.nz;
                if (KIND == 0) {
                    // q = D f / phi here; the backward divergence needs q_x, q_y, q_z of
                    // the neighbours below: q_z from the lane below (lane 0 evaluates
                    // its own), q_y from this thread's previous step, q_x evaluated
                    const float qx = Dx * inv_phi, qy = Dy * inv_phi, qz = Dz * inv_phi;
                    float div = -qx * a.inv_dx - qy * a.inv_dy - qz * a.inv_dz;
                    float qz_below = __shfl_up_sync(0xffffffffu, qz, 1);
                    if (lane == 0 && gz > 0) {
                        float ex, ey, ez;
                        fdiff(a, F, hx, hy, hz - 1, gx, gy, gz - 1, ex, ey, ez);
                        qz_below = ez * rsqrtf(eps2 + ex * ex + ey * ey + ez * ez);
                    }
                    if (gz > 0) div += qz_below * a.inv_dz;
                    if (gy > 0) {
                        if (i == 0) {
                            float ex, ey, ez;
                            fdiff(a, F, hx, hy - 1, hz, gx, gy - 1, gz, ex, ey, ez);
                            qy_prev = ey * rsqrtf(eps2 + ex * ex + ey * ey + ez * ez);
                        }
                        div += qy_prev * a.inv_dy;
                    }
                    if (gx > 0) {
                        float ex, ey, ez;
                        fdiff(a, F, hx - 1, hy, hz, gx - 1, gy, gz, ex, ey, ez);
                        div += ex * rsqrtf(eps2 + ex * ex + ey * ey + ez * ez) * a.inv_dx;
                    }
                    qy_prev = qy;
                    if (live) {
                        const float dj = lam * div + diff * inv_tau;
                        dout[((size_t)gx * a.ny + gy) * a.nz + gz] = dj;
                        part[0] += lam * phi + diff * diff * inv_2tau;
                        part[K - 1] += dj * dj;
                    }
                } else if (live) {
                    part[0] += lam * phi + diff * diff * inv_2tau;
                }
            }
        }
        brick_warp_sums<K>(part, sh, it & 1);
        __syncthreads();
        prev = br;
    }
    if (prev >= 0) brick_flush<K>(sh, (it - 1) & 1, a.partials + (size_t)prev * 4);
    return true;
}

// f = cur - s*dir (dir may be null: copy), optionally clamped at 0; with
// `store`, the value is also written to a.f_store rounded to a.store_type
// (the copy the reduced-storage projector gathers from).
__device__ void sweep_update(const RofArgs &a, const float *cur, const float *dir, float s, float *f,
                             bool clamp, bool store = false)
{
    if (store) {
        const size_t n = (size_t)a.nx * a.ny * a.nz;
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
            float c = __ldcg(cur + i);
            if (dir) c = __fmaf_rn(-s, __ldcg(dir + i), c);
            if (clamp) c = fmaxf(c, 0.f);
            __stcg(f + i, c);
            st_st(a.f_store, i, c, a.store_type);
        }
        return;
    }
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

// ---------------------------------------------------------------------------
// the solve
// ---------------------------------------------------------------------------
template <bool TMA>
__global__ void __launch_bounds__(TV_THREADS, 3)
rof_kernel(const RofArgs args, const __grid_constant__ RofMaps maps)
{
    __shared__ TvShared sh;
    extern __shared__ float dyn_raw[];
    // staging buffers from the next 1024-byte boundary of the shared window
    // (tensor copies land on 128-byte aligned addresses; every buffer offset
    // below is a multiple of 128 bytes)
    float *dyn = dyn_raw + ((1024u - (smem_u32(dyn_raw) & 1023u)) & 1023u) / sizeof(float);
    RofArgs a = args;
    if (a.tau_dev) a.tau = *a.tau_dev;
    const double nvox = (double)a.nx * a.ny * a.nz;
    const int nb = brick_count(a).total;
    const RofMaps *mp = &maps;
    if (TMA && threadIdx.x == 0) {
        mbar_init(&sh.mbar[0]);
        mbar_init(&sh.mbar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    Pipe pp{0, 0u};

    if (a.mode == 1) {  // energy + gradient at a.cur
        const SweepOps op{MAP_CUR, MAP_CUR, a.cur, nullptr, 0.f};
        if (!sweep<TMA, 0>(a, mp, sh, dyn, pp, op, a.d)) return;
        if (!grid_sync<2>(a.st, a.partials, nb, sh)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.out[0] = sh.res[0] / nvox;
            a.out[1] = sh.res[1] / nvox;
        }
        return;
    }
    if (a.mode == 2) {  // trial energy at a.cur - s a.dir
        const SweepOps op{MAP_CUR, MAP_DIR, a.cur, a.dir, (float)a.trial_s};
        if (!sweep<TMA, 1>(a, mp, sh, dyn, pp, op, nullptr)) return;
        if (!grid_sync<1>(a.st, a.partials, nb, sh)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) a.out[0] = sh.res[0] / nvox;
        return;
    }

    // full solve
    const bool replay = a.replay != nullptr;
    const int n_steps = replay ? a.replay[0] : a.max_inner;
    const float *cur = a.start_at_g ? a.g : a.f;
    int cur_map = a.start_at_g ? MAP_G : MAP_F;
    bool wrote_f = !a.start_at_g;
    bool clamped = false, stored = false;
    int n_inner = 0, bt_total = 0, flags = 0;
    double e_first = 0.0, e_last = 0.0;
    const double s0 = a.s0 > 0.0 ? a.s0 : a.tau;

    for (int it = 0; it < n_steps; ++it) {
        const SweepOps og{cur_map, cur_map, cur, nullptr, 0.f};
        if (!sweep<TMA, 0>(a, mp, sh, dyn, pp, og, a.d)) return;
        if (!grid_sync<2>(a.st, a.partials, nb, sh)) return;
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
                const SweepOps ot{cur_map, MAP_D, cur, a.d, (float)step};
                if (!sweep<TMA, 1>(a, mp, sh, dyn, pp, ot, nullptr)) return;
                if (!grid_sync<1>(a.st, a.partials, nb, sh)) return;
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
        const bool do_store = a.f_store != nullptr && stop;
        sweep_update(a, cur, a.d, (float)step, a.f, do_clamp, do_store);
        stored = do_store;
        cur = a.f;
        cur_map = MAP_F;
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
        if (!grid_sync<0>(a.st, a.partials, nb, sh)) return;
    }
    if (!wrote_f || (a.clamp && !clamped) || (a.f_store && !stored)) {
        // the loop ended without writing the final iterate: f = clamp(cur)
        // (and its stored copy)
        if (!grid_sync<0>(a.st, a.partials, nb, sh)) return;
        sweep_update(a, cur, nullptr, 0.f, a.f, a.clamp != 0, a.f_store != nullptr);
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

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int rof_bricks(int nx, int ny, int nz)
{
    return ((nx + BX - 1) / BX) * ((ny + BY - 1) / BY) * ((nz + BZ - 1) / BZ);
}

// The tensor-map encoder of the driver, fetched once through the runtime (no
// link-time dependency on the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn tensor_map_encoder()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Tiled map of an nx x ny x nz FP32 volume (z fastest) with the staging box;
// false when the copy engine's rules are not met (16-byte aligned base, rows
// of a multiple of 16 bytes, box no larger than the volume).
static bool encode_volume(CUtensorMap *m, const float *base, int nx, int ny, int nz)
{
    EncodeTiledFn fn = tensor_map_encoder();
    if (!fn || !base || ((uintptr_t)base & 15u) || nz % 4 != 0 || nz < SZ || ny < SY || nx < SX) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nz, (cuuint64_t)ny, (cuuint64_t)nx};
    const cuuint64_t strides[2] = {(cuuint64_t)nz * sizeof(float), (cuuint64_t)ny * nz * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)SZ, (cuuint32_t)SY, (cuuint32_t)SX};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Maps of every volume the launch stages from; false: stage with plain loads.
static bool build_maps(const RofArgs &a, RofMaps &m)
{
    std::memset(&m, 0, sizeof(m));
    if (a.mode == 0)
        return encode_volume(&m.m[MAP_G], a.g, a.nx, a.ny, a.nz) && encode_volume(&m.m[MAP_F], a.f, a.nx, a.ny, a.nz) &&
               encode_volume(&m.m[MAP_D], a.d, a.nx, a.ny, a.nz);
    if (!encode_volume(&m.m[MAP_CUR], a.cur, a.nx, a.ny, a.nz)) return false;
    return a.mode != 2 || encode_volume(&m.m[MAP_DIR], a.dir, a.nx, a.ny, a.nz);
}

static cudaError_t rof_prepare()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(rof_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TV_DYN_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(rof_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TV_DYN_SMEM);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

// cooperative grid size of rof_kernel (SMs x resident blocks), per device
static std::mutex g_rof_mutex;
static int g_rof_blocks[64] = {};
static thread_local int t_rof_share = 1;   // solves this thread launches share the GPU with this many others

void set_rof_grid_share(int k) { t_rof_share = k > 1 ? k : 1; }

int rof_grid_blocks()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 0;
    if (rof_prepare() != cudaSuccess) return 0;
    int n = 0;
    {
        std::lock_guard<std::mutex> lock(g_rof_mutex);
        int *cached = dev < 64 ? &g_rof_blocks[dev] : nullptr;
        if (cached && *cached) {
            n = *cached;
        } else {
            int sms = 0, per_sm = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rof_kernel<true>, TV_THREADS, TV_DYN_SMEM);
            if (per_sm < 1) per_sm = 1;
            n = sms * per_sm;
            if (cached) *cached = n;
        }
    }
    return n / t_rof_share > 0 ? n / t_rof_share : 1;
}

cudaError_t launch_rof(const RofArgs &a, cudaStream_t s)
{
    const int nbricks = rof_bricks(a.nx, a.ny, a.nz);
    int blocks = rof_grid_blocks();
    if (blocks > nbricks) blocks = nbricks;
    if (blocks < 1) blocks = 1;
    cudaError_t e = rof_prepare();
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(&a.st->bar, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
    if (a.withhold_arrival) {
        // arrivals start far above the grid size, so none is ever the last
        e = cudaMemsetAsync(&a.st->bar.count, 0x7f, sizeof(unsigned int), s);
        if (e != cudaSuccess) return e;
    }
    RofArgs args = a;
    RofMaps maps;
    const bool tma = build_maps(a, maps);
    void *params[] = {&args, &maps};
    launch_begin(K_ROF, s);
    e = cudaLaunchCooperativeKernel(tma ? (const void *)rof_kernel<true> : (const void *)rof_kernel<false>,
                                    dim3(blocks), dim3(TV_THREADS), params, TV_DYN_SMEM, s);
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
