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
// Precision. The result is a bilinear sample of the residual, so an error
// of e pixels in the detector coordinate moves it by about e relative on a
// rough residual. An FP32 coordinate of several hundred pixels carries
// 2^-24 * 512 ~ 3e-5 pixels of rounding, too much for 1e-5 parity against
// an FP64 evaluation. The coordinate chain is therefore carried in
// double-float (hi + lo FP32 pairs, about 44 bits): voxel position, the
// rotation by (cos, sin) given in double-float from the host, depth,
// 1/depth (one Newton step), the Eq. A6 quotients and the pixel offset; the
// integer pixel is split off before the fraction is rounded to FP32, so
// the interpolation weights are exact to about 1e-7 pixel. The weight
// 2 L^3 / (L0 l^2) equals 2 L0^2 l / depth^3 (similar triangles:
// L / l = L0 / depth) and stays FP32 (a relative error of a few 1e-7).
//
// Thread mapping: a warp covers an 8 x 4 tile of voxel columns; each lane
// walks EQ6_ZPT consecutive z of its column, so the per-(column, view) part
// of the chain is shared by EQ6_ZPT voxels, and at every step the warp's 32
// samples of a view fall on one or two detector rows within a few sectors.
// The 8 warps of a block take 8 consecutive z runs of the same columns.
// Results leave as 32-byte runs along z.
#include "cbct_internal.cuh"

namespace cbct {

constexpr int EQ6_TX = 8, EQ6_TY = 4, EQ6_WARPS = 8, EQ6_ZPT = 8;
constexpr int EQ6_THREADS = 32 * EQ6_WARPS;
constexpr int EQ6_TZ = EQ6_WARPS * EQ6_ZPT;   // z voxels per block

// ---- double-float helpers (error-free transformations with FMA) ----
__device__ __forceinline__ DF e6_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return DF{s, e};
}

__device__ __forceinline__ DF e6_fast_two_sum(float a, float b)   // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF e6_add(DF a, DF b)
{
    DF s = e6_two_sum(a.hi, b.hi);
    return e6_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ DF e6_mul(DF a, DF b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return e6_fast_two_sum(p, e);
}

__device__ __forceinline__ DF e6_mul(DF a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    const float e = __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p));
    return e6_fast_two_sum(p, e);
}

__device__ __forceinline__ DF e6_neg(DF a) { return DF{-a.hi, -a.lo}; }

// 1 / a: an FP32 reciprocal refined by one Newton step in double-float
__device__ __forceinline__ DF e6_recip(DF a)
{
    const float r = __frcp_rn(a.hi);
    // residual 1 - a r, with the hi product's rounding recovered by FMA
    const float e = __fmaf_rn(-a.lo, r, __fmaf_rn(-a.hi, r, 1.f));
    return e6_fast_two_sum(r, __fmul_rn(r, e));
}

// integer part and fraction in [0, 1) of a double-float coordinate
__device__ __forceinline__ void e6_split(DF x, int &i, float &frac)
{
    float fi = floorf(x.hi);
    float fr = __fadd_rn(__fsub_rn(x.hi, fi), x.lo);   // x.hi - fi is exact
    if (fr < 0.f) {
        fi -= 1.f;
        fr = __fadd_rn(fr, 1.f);
    }
    if (fr >= 1.f) {
        fi += 1.f;
        fr = __fsub_rn(fr, 1.f);
    }
    i = (int)fi;
    frac = fr;
}

// bilinear detector sample, zero outside (the oracle's detector_bilinear)
__device__ __forceinline__ float e6_sample(const float *__restrict__ img, int nu, int nv, int u0, float wu, int v0,
                                           float wv)
{
    if (u0 < -1 || u0 >= nu || v0 < -1 || v0 >= nv) return 0.f;
    float s0 = 0.f, s1 = 0.f;
    if (v0 >= 0) {
        const float *row = img + (size_t)v0 * nu;
        if (u0 >= 0) s0 = __fmaf_rn(1.f - wu, __ldg(row + u0), s0);
        if (u0 + 1 < nu) s0 = __fmaf_rn(wu, __ldg(row + u0 + 1), s0);
    }
    if (v0 + 1 < nv) {
        const float *row = img + (size_t)(v0 + 1) * nu;
        if (u0 >= 0) s1 = __fmaf_rn(1.f - wu, __ldg(row + u0), s1);
        if (u0 + 1 < nu) s1 = __fmaf_rn(wu, __ldg(row + u0 + 1), s1);
    }
    return __fmaf_rn(1.f - wv, s0, wv * s1);
}

template <int MODE>
__global__ void __launch_bounds__(EQ6_THREADS)
eq6_kernel(VolGeom g, DetGeom d, Eq6Geom e, const float *__restrict__ T, const float *__restrict__ f,
           float *__restrict__ out, const double *__restrict__ d_scale, float scale_val)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int a = blockIdx.x * EQ6_TX + (lane & (EQ6_TX - 1));
    const int b = blockIdx.y * EQ6_TY + (lane / EQ6_TX);
    const int c0 = blockIdx.z * EQ6_TZ + warp * EQ6_ZPT;   // warp-uniform
    if (c0 >= g.nz) return;
    const bool live = a < g.nx && b < g.ny;
    const int nzr = min(EQ6_ZPT, g.nz - c0);

    float acc[EQ6_ZPT];
#pragma unroll
    for (int i = 0; i < EQ6_ZPT; i++) acc[i] = 0.f;

    if (live) {
        // voxel centre in double-float: (index - centre) * pitch, the first factor exact
        const DF x = e6_mul(e.dx, (float)a - e.cx), y = e6_mul(e.dy, (float)b - e.cy);
        DF z[EQ6_ZPT];
#pragma unroll
        for (int i = 0; i < EQ6_ZPT; i++) z[i] = e6_mul(e.dz, (float)(c0 + i) - e.cz);
        for (int k = 0; k < d.n_views; ++k) {
            const float4 cs4 = __ldg(e.views + k);
            const DF ct{cs4.x, cs4.y}, st{cs4.z, cs4.w};
            // coordinates in the frame where the projection runs along +x'
            const DF xr = e6_add(e6_mul(x, ct), e6_mul(y, st));
            const DF yr = e6_add(e6_mul(y, ct), e6_neg(e6_mul(x, st)));
            const DF depth = e6_add(xr, e.sad);                    // x' - x_s
            const DF inv = e6_recip(depth);
            // Eq. A6 in pixel units, offset by the detector centre
            const DF fu = e6_add(e6_neg(e6_mul(e6_mul(yr, e.ku), inv)), DF{e.cu, 0.f});
            const DF kvi = e6_mul(e.kv, inv);
            int u0;
            float wu;
            e6_split(fu, u0, wu);
            // 2 L^3 / (L0 l^2) = 2 L0^2 l / depth^3, l^2 = depth^2 + y'^2 + z^2
            const float ih = inv.hi;
            const float wc = e.two_l0sq * ih * ih * ih;
            const float rho2 = __fmaf_rn(depth.hi, depth.hi, yr.hi * yr.hi);
            const float *img = T + (size_t)k * d.nv * d.nu;
            const bool u_in = u0 >= -1 && u0 < d.nu;
#pragma unroll
            for (int i = 0; i < EQ6_ZPT; i++) {
                if (i >= nzr || !u_in) continue;
                const DF fv = e6_add(e6_mul(z[i], kvi), DF{e.cv, 0.f});
                int v0;
                float wv;
                e6_split(fv, v0, wv);
                const float l2 = __fmaf_rn(z[i].hi, z[i].hi, rho2);
                const float l = l2 * rsqrtf(l2);
                acc[i] = __fmaf_rn(wc * l, e6_sample(img, d.nu, d.nv, u0, wu, v0, wv), acc[i]);
            }
        }
    }
    if (!live) return;
    const size_t base = ((size_t)a * g.ny + b) * g.nz + c0;
    const float scale = (MODE == 1) ? (d_scale ? (float)(*d_scale) * scale_val : scale_val) : 0.f;
    if (nzr == EQ6_ZPT && (base & 3) == 0) {
        float4 *o = reinterpret_cast<float4 *>(out + base);
        if (MODE == 0) {
            o[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
            o[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
        } else {
            const float4 *fi = reinterpret_cast<const float4 *>(f + base);
            const float4 f0 = __ldg(fi), f1 = __ldg(fi + 1);
            o[0] = make_float4(__fmaf_rn(-scale, acc[0], f0.x), __fmaf_rn(-scale, acc[1], f0.y),
                               __fmaf_rn(-scale, acc[2], f0.z), __fmaf_rn(-scale, acc[3], f0.w));
            o[1] = make_float4(__fmaf_rn(-scale, acc[4], f1.x), __fmaf_rn(-scale, acc[5], f1.y),
                               __fmaf_rn(-scale, acc[6], f1.z), __fmaf_rn(-scale, acc[7], f1.w));
        }
    } else {
#pragma unroll
        for (int i = 0; i < EQ6_ZPT; i++) {
            if (i >= nzr) break;
            out[base + i] = (MODE == 0) ? acc[i] : __fmaf_rn(-scale, acc[i], __ldg(f + base + i));
        }
    }
}

static_assert(EQ6_ZPT == 8, "the vector store writes 8 z values");

// mode 0: out = G(T); mode 1: out = f - scale G(T), scale = scale_val, times
// *d_scale when given
cudaError_t launch_eq6(const VolGeom &v, const DetGeom &d, const Eq6Geom &e, const float *T, const float *f,
                       float *out, const double *d_scale, double scale_val, int mode, cudaStream_t s)
{
    const dim3 grid((unsigned)((v.nx + EQ6_TX - 1) / EQ6_TX), (unsigned)((v.ny + EQ6_TY - 1) / EQ6_TY),
                    (unsigned)((v.nz + EQ6_TZ - 1) / EQ6_TZ));
    launch_begin(K_EQ6, s);
    if (mode == 0)
        eq6_kernel<0><<<grid, EQ6_THREADS, 0, s>>>(v, d, e, T, f, out, d_scale, (float)scale_val);
    else
        eq6_kernel<1><<<grid, EQ6_THREADS, 0, s>>>(v, d, e, T, f, out, d_scale, (float)scale_val);
    launch_end(K_EQ6, s);
    return cudaGetLastError();
}

} // namespace cbct
