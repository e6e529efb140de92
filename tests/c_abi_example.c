/* Plain-C use of libcbct through include/cbct.h only (no Python): build a
 * geometry, project a volume, apply the matched transpose, and check the
 * adjoint identity <P f, s> = <f, P^T s> (Eq. 1 and its transpose) on
 * seeded data. Exit status 0 on success. Test infrastructure. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "cbct.h"

#define CHECK(call)                                                                                 \
    do {                                                                                            \
        cbct_status s_ = (call);                                                                    \
        if (s_ != CBCT_OK) {                                                                        \
            fprintf(stderr, "%s failed: %d %s\n", #call, (int)s_, cbct_last_error());               \
            return 1;                                                                               \
        }                                                                                           \
    } while (0)

static unsigned long long lcg = 12345;
static float next_uniform(void)
{
    lcg = lcg * 6364136223846793005ull + 1442695040888963407ull;
    return (float)((lcg >> 40) & 0xffffff) / 16777216.0f;
}

int main(void)
{
    enum { NX = 24, NY = 20, NZ = 16, NU = 40, NV = 28, NVIEW = 8 };
    double angles[NVIEW];
    for (int k = 0; k < NVIEW; k++) angles[k] = 2.0 * 3.14159265358979323846 * k / NVIEW;
    cbct_geometry_desc d = {NX, NY, NZ, 2.0, 2.0, 2.0, NU, NV, 1.6, 1.6, 300.0, 480.0, NVIEW, angles, 0.5};
    cbct_geometry *g = NULL;
    CHECK(cbct_geometry_create(&d, &g));

    const size_t nvox = (size_t)NX * NY * NZ, nray = (size_t)NVIEW * NV * NU;
    float *hf = (float *)malloc(nvox * sizeof(float)), *hs = (float *)malloc(nray * sizeof(float));
    float *hp = (float *)malloc(nray * sizeof(float)), *hb = (float *)malloc(nvox * sizeof(float));
    for (size_t i = 0; i < nvox; i++) hf[i] = next_uniform();
    for (size_t i = 0; i < nray; i++) hs[i] = next_uniform();

    float *df = NULL, *ds = NULL, *dp = NULL, *db = NULL;
    if (cudaMalloc((void **)&df, nvox * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&ds, nray * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&dp, nray * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&db, nvox * sizeof(float)) != cudaSuccess) {
        fprintf(stderr, "cudaMalloc failed\n");
        return 1;
    }
    cudaMemcpy(df, hf, nvox * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(ds, hs, nray * sizeof(float), cudaMemcpyHostToDevice);
    CHECK(cbct_forward_project(g, df, dp, NULL));
    CHECK(cbct_back_project(g, ds, db, NULL));
    if (cudaDeviceSynchronize() != cudaSuccess) {
        fprintf(stderr, "kernel failure\n");
        return 1;
    }
    cudaMemcpy(hp, dp, nray * sizeof(float), cudaMemcpyDeviceToHost);
    cudaMemcpy(hb, db, nvox * sizeof(float), cudaMemcpyDeviceToHost);

    double a = 0.0, b = 0.0;
    for (size_t i = 0; i < nray; i++) a += (double)hp[i] * hs[i];
    for (size_t i = 0; i < nvox; i++) b += (double)hf[i] * hb[i];
    const double rel = fabs(a - b) / fmax(fabs(a), fabs(b));
    printf("<Pf,s> = %.9g  <f,P^T s> = %.9g  relative difference %.3g\n", a, b, rel);

    cudaFree(df);
    cudaFree(ds);
    cudaFree(dp);
    cudaFree(db);
    free(hf);
    free(hs);
    free(hp);
    free(hb);
    cbct_geometry_destroy(g);
    return (a > 0.0 && rel < 1e-5) ? 0 : 2;
}
