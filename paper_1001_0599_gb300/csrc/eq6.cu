// The paper's closed-form, voxel-driven gradient of the data term (Eq. 6,
// with the projection coordinates of Eq. A6 and the Jacobian of Eq. A7):
//
//   G(x) = sum_theta 2 L^3(u*, v*) / (L0 l^2(x)) * T^theta(u*, v*),
//
// u* = -(y' - y_s) L0 / (x' - x_s), v* = (z - z_s) L0 / (x' - x_s) in the
// frame rotated so the projection runs along +x', l = |x - S|,
// L = sqrt(L0^2 + u*^2 + v*^2), and T (the residual sinogram) bilinearly
// interpolated on the detector (zero outside). Without the 1/(N_theta A)
// prefactor of Eq. 6. This is the paper's unmatched backprojector: about as
// much work per voxel and view as one bilinear sample, an order of magnitude
// less than the matched transpose.
//
// Thread mapping: a warp covers an 8 x 4 tile of voxel columns at one z, so
// its 32 detector samples of a view fall on one or two detector rows within
// a few sectors (a z-fastest mapping would put every lane on its own row and
// cost a sector per lane per read); the 8 warps of a block take 8 consecutive
// z, and the results leave through shared memory as 32-byte runs along z.
#include "cbct_internal.cuh"

namespace cbct {

constexpr int EQ6_TX = 8, EQ6_TY = 4, EQ6_TZ = 8;
constexpr int EQ6_THREADS = EQ6_TX * EQ6_TY * EQ6_TZ;

template <int MODE>
__global__ void __launch_bounds__(EQ6_THREADS)
eq6_kernel(VolGeom g, DetGeom d, const float *__restrict__ T, const float *__restrict__ f,
           float *__restrict__ out, const double *__restrict__ d_scale, float scale_val)
{
    __shared__ float tile[EQ6_TX * EQ6_TY][EQ6_TZ + 1];
    const int lane = threadIdx.x & 31, wz = threadIdx.x >> 5;
    const int a = blockIdx.x * EQ6_TX + (lane & (EQ6_TX - 1));
    const int b = blockIdx.y * EQ6_TY + (lane / EQ6_TX);
    const int c0 = blockIdx.z * EQ6_TZ;
    const int c = c0 + wz;
    float acc = 0.f;
    if (a < g.nx && b < g.ny && c < g.nz) {
        const float x = ((float)a - g.cx) * g.dx, y = ((float)b - g.cy) * g.dy, z = ((float)c - g.cz) * g.dz;
        const float L0 = d.sdd;
        for (int k = 0; k < d.n_views; ++k) {
            const float2 cs = d.views[k];
            const float xr = x * cs.x + y * cs.y;       // depth along the central ray
            const float yr = -x * cs.y + y * cs.x;
            const float depth = xr + d.sad;             // x' - x_s
            const float inv_depth = __frcp_rn(depth);     // correctly rounded, as 1 / depth
            const float us = -yr * L0 * inv_depth;      // Eq. A6
            const float vs = z * L0 * inv_depth;
            const float l2 = depth * depth + yr * yr + z * z;
            const float Lsq = L0 * L0 + us * us + vs * vs;
            // 2 L^3 / (L0 l^2): L = Lsq rsqrt(Lsq) and one reciprocal (a few ulp of
            // FP32, far inside the detector-coordinate rounding of the sample)
            const float w = 2.f * Lsq * (Lsq * rsqrtf(Lsq)) * __frcp_rn(L0 * l2);
            // bilinear detector interpolation, zero outside
            const float fu = __fmaf_rn(us, d.inv_du, d.cu), fv = __fmaf_rn(vs, d.inv_dv, d.cv);
            const float u0f = floorf(fu), v0f = floorf(fv);
            const int u0 = (int)u0f, v0 = (int)v0f;
            if (u0 < -1 || u0 >= d.nu || v0 < -1 || v0 >= d.nv) continue;
            const float wu = fu - u0f, wv = fv - v0f;
            const float *img = T + (size_t)k * d.nv * d.nu;
            float s = 0.f;
            if (v0 >= 0) {
                const float *row = img + (size_t)v0 * d.nu;
                if (u0 >= 0) s += (1.f - wu) * (1.f - wv) * __ldg(row + u0);
                if (u0 + 1 < d.nu) s += wu * (1.f - wv) * __ldg(row + u0 + 1);
            }
            if (v0 + 1 < d.nv) {
                const float *row = img + (size_t)(v0 + 1) * d.nu;
                if (u0 >= 0) s += (1.f - wu) * wv * __ldg(row + u0);
                if (u0 + 1 < d.nu) s += wu * wv * __ldg(row + u0 + 1);
            }
            acc = __fmaf_rn(w, s, acc);
        }
    }
    tile[lane][wz] = acc;
    __syncthreads();
    // write-out: 8 threads per voxel column, one z each (32-byte runs)
    const int col = threadIdx.x / EQ6_TZ, zz = threadIdx.x % EQ6_TZ;
    const int oa = blockIdx.x * EQ6_TX + (col & (EQ6_TX - 1));
    const int ob = blockIdx.y * EQ6_TY + (col / EQ6_TX);
    const int oc = c0 + zz;
    if (oa >= g.nx || ob >= g.ny || oc >= g.nz) return;
    const size_t i = ((size_t)oa * g.ny + ob) * g.nz + oc;
    const float v = tile[col][zz];
    if (MODE == 0) {
        out[i] = v;
    } else {
        const float scale = d_scale ? (float)(*d_scale) * scale_val : scale_val;
        out[i] = __fmaf_rn(-scale, v, __ldg(f + i));
    }
}

// mode 0: out = G(T); mode 1: out = f - scale G(T), scale = scale_val, times
// *d_scale when given
cudaError_t launch_eq6(const VolGeom &v, const DetGeom &d, const float *T, const float *f, float *out,
                       const double *d_scale, double scale_val, int mode, cudaStream_t s)
{
    const dim3 grid((unsigned)((v.nx + EQ6_TX - 1) / EQ6_TX), (unsigned)((v.ny + EQ6_TY - 1) / EQ6_TY),
                    (unsigned)((v.nz + EQ6_TZ - 1) / EQ6_TZ));
    launch_begin(K_EQ6, s);
    if (mode == 0)
        eq6_kernel<0><<<grid, EQ6_THREADS, 0, s>>>(v, d, T, f, out, d_scale, (float)scale_val);
    else
        eq6_kernel<1><<<grid, EQ6_THREADS, 0, s>>>(v, d, T, f, out, d_scale, (float)scale_val);
    launch_end(K_EQ6, s);
    return cudaGetLastError();
}

} // namespace cbct
