// Gather microbenchmark (measurement only; no counterpart in the paper): the
// rate at which an SM can gather trilinear footprints -- 8 voxel values,
// 32 bytes -- from an L2-resident FP32 volume with the lane-to-address
// pattern of a ray-driven projector: a warp walks one in-plane ray line and
// its 32 lanes take 32 consecutive detector rows, so at every sample the
// lanes read the same four voxel columns at nearby heights. Each lane does
// the textbook per-sample gather (8 read-only loads, 7 interpolations). The
// samples per second of this kernel are the denominator against which the
// projector's and transpose's "gathered bytes" (32 B per trilinear sample
// they account for) are reported.
#include "cbct_internal.cuh"

namespace cbct {

constexpr int GB_WARPS = 8;

__global__ void __launch_bounds__(GB_WARPS * 32)
gather_kernel(const float *__restrict__ vol, int nx, int ny, int nz, int n_lines, int n_samples,
              float *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * GB_WARPS;
    const float hx = 0.5f * (float)(nx - 2), hy = 0.5f * (float)(ny - 2), hz = 0.5f * (float)(nz - 2);
    for (int l = blockIdx.x * GB_WARPS + (threadIdx.x >> 5); l < n_lines; l += nwarps) {
        // line l: through the volume centre region at angle l * golden angle,
        // offset across the line; rows diverge along the line like a cone
        const float th = 2.39996323f * (float)l;
        float s, c;
        __sincosf(th, &s, &c);
        const float off = 0.4f * hx * (float)((l * 7919) % 101 - 50) / 50.f;
        const float x0 = hx - c * hx * 0.95f - s * off, y0 = hy - s * hy * 0.95f + c * off;
        const float step_x = c * 1.9f * hx / (float)n_samples, step_y = s * 1.9f * hy / (float)n_samples;
        const float zrow = (float)(lane - 16) * 0.55f;
        float acc = 0.f;
        for (int j = 0; j < n_samples; ++j) {
            const float fx = fminf(fmaxf(__fmaf_rn((float)j, step_x, x0), 0.f), (float)(nx - 2));
            const float fy = fminf(fmaxf(__fmaf_rn((float)j, step_y, y0), 0.f), (float)(ny - 2));
            const float fz = fminf(fmaxf(hz + zrow * (0.8f + 0.4f * (float)j / (float)n_samples), 0.f),
                                   (float)(nz - 2));
            const float ax = floorf(fx), ay = floorf(fy), az = floorf(fz);
            const float wx = fx - ax, wy = fy - ay, wz = fz - az;
            const size_t i000 = (((size_t)ax * ny) + (size_t)ay) * nz + (size_t)az;
            const size_t sx = (size_t)ny * nz, sy = (size_t)nz;
            const float v000 = __ldg(vol + i000), v001 = __ldg(vol + i000 + 1);
            const float v010 = __ldg(vol + i000 + sy), v011 = __ldg(vol + i000 + sy + 1);
            const float v100 = __ldg(vol + i000 + sx), v101 = __ldg(vol + i000 + sx + 1);
            const float v110 = __ldg(vol + i000 + sx + sy), v111 = __ldg(vol + i000 + sx + sy + 1);
            const float a00 = __fmaf_rn(wz, v001 - v000, v000), a01 = __fmaf_rn(wz, v011 - v010, v010);
            const float a10 = __fmaf_rn(wz, v101 - v100, v100), a11 = __fmaf_rn(wz, v111 - v110, v110);
            const float b0 = __fmaf_rn(wy, a01 - a00, a00), b1 = __fmaf_rn(wy, a11 - a10, a10);
            acc += __fmaf_rn(wx, b1 - b0, b0);
        }
        out[(size_t)l * 32 + lane] = acc;
    }
}

cudaError_t launch_gather(const float *vol, int nx, int ny, int nz, int n_lines, int n_samples, float *out,
                          cudaStream_t s)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather_kernel, GB_WARPS * 32, 0);
    if (per_sm < 1) per_sm = 1;
    const int need = (n_lines + GB_WARPS - 1) / GB_WARPS;
    const int blocks = need < sms * per_sm ? need : sms * per_sm;
    launch_begin(K_MISC, s);
    gather_kernel<<<blocks > 0 ? blocks : 1, GB_WARPS * 32, 0, s>>>(vol, nx, ny, nz, n_lines, n_samples, out);
    launch_end(K_MISC, s);
    return cudaGetLastError();
}

} // namespace cbct
