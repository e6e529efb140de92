/*
 * FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see cbct_oracle.h).
 *
 * Plain restatement of Jia et al. (arXiv:1001.0599):
 *   Eq. 1   cone-beam line integral, discretised as uniform samples in the
 *           in-plane distance from the source with trilinear interpolation;
 *   Eq. 2   energies E1 (TV) and E2 (data), mean-normalised;
 *   Alg. A1 forward-backward splitting: gradient step, ROF, clamp;
 *   Eq. 5   Armijo rule for the ROF gradient descent (Sec. II.B);
 *   Sec. II.B boundary conditions: zero on x, y; reflective on z;
 *   Eq. 6 / A6 / A7  the paper's closed-form voxel-driven gradient;
 *   Sec. II.C.3 multigrid prolongation.
 * No blocking, fusion or reordering: each quantity is computed from its
 * definition. OpenMP only splits independent rays / voxels across threads.
 */
#include "cbct_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(a, b, c) (((size_t)(a) * (size_t)ny + (size_t)(b)) * (size_t)nz + (size_t)(c))

/* ------------------------------------------------------------------------ */
/* Geometry (Fig. 1, Eq. A2)                                                 */
/* ------------------------------------------------------------------------ */

double orc_drho(const orc_geom *g)
{
    double h = g->dx < g->dy ? g->dx : g->dy;
    return g->step_ratio * h;
}

/* radius (in the xy plane) of the support of the trilinear interpolant */
static double support_radius_xy(const orc_geom *g)
{
    double hx = 0.5 * (g->nx + 1) * g->dx, hy = 0.5 * (g->ny + 1) * g->dy;
    return sqrt(hx * hx + hy * hy);
}

int orc_check_geometry(const orc_geom *g)
{
    if (g->nx < 1 || g->ny < 1 || g->nz < 1 || g->nu < 1 || g->nv < 1 || g->n_views < 1)
        return -1;
    if (!(g->dx > 0 && g->dy > 0 && g->dz > 0 && g->du > 0 && g->dv > 0 && g->step_ratio > 0))
        return -1;
    double R = support_radius_xy(g);
    if (!(g->sad - R > 0 && g->sdd > g->sad + R)) return -1;
    return 0;
}

typedef struct {
    double s[3];      /* source */
    double e[3];      /* direction scaled to unit in-plane length */
    double ds;        /* integration weight of one sample: drho * L / L_xy */
    double rho_end;   /* in-plane distance from the source to the pixel */
} ray_t;

static void ray_setup(const orc_geom *g, int view, int iv, int iu, ray_t *r)
{
    double th = g->angles[view];
    double c = cos(th), s = sin(th);
    double u = (iu - 0.5 * (g->nu - 1)) * g->du;
    double v = (iv - 0.5 * (g->nv - 1)) * g->dv;
    double S[3] = {-g->sad * c, -g->sad * s, 0.0};
    /* pixel centre P = D + u e_u + v e_v, e_u = Rz(theta)(0,-1,0) = (s,-c,0) */
    double P[3] = {(g->sdd - g->sad) * c + u * s, (g->sdd - g->sad) * s - u * c, v};
    double n[3] = {P[0] - S[0], P[1] - S[1], P[2] - S[2]};
    double L = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double Lxy = sqrt(n[0] * n[0] + n[1] * n[1]);
    for (int i = 0; i < 3; i++) {
        r->s[i] = S[i];
        r->e[i] = n[i] / Lxy;
    }
    r->ds = orc_drho(g) * L / Lxy;
    r->rho_end = Lxy;
}

/* Walk the samples of one ray. mode 0: return sum_k ds * f(X_k) (Eq. 1).
 * mode 1: add val * ds * w into every voxel the samples touch (the exact
 * transpose of mode 0). Counts non-zero terms into *nnz when given. */
static double ray_apply(const orc_geom *g, const ray_t *r, double *vol, double val,
                        int mode, int64_t *nnz)
{
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const double drho = orc_drho(g);
    const double R = support_radius_xy(g);
    long k0 = (long)floor((g->sad - R) / drho) - 1;
    long k1 = (long)ceil((g->sad + R) / drho) + 1;
    if (k0 < 0) k0 = 0;
    double acc = 0.0;
    for (long k = k0; k <= k1; k++) {
        double rho = (double)k * drho;
        if (rho > r->rho_end) break;
        double X = r->s[0] + rho * r->e[0];
        double Y = r->s[1] + rho * r->e[1];
        double Z = r->s[2] + rho * r->e[2];
        /* continuous voxel coordinates of the sample */
        double fx = X / g->dx + 0.5 * (nx - 1);
        double fy = Y / g->dy + 0.5 * (ny - 1);
        double fz = Z / g->dz + 0.5 * (nz - 1);
        double a0 = floor(fx), b0 = floor(fy), c0 = floor(fz);
        double wx1 = fx - a0, wy1 = fy - b0, wz1 = fz - c0;
        double wxs[2] = {1.0 - wx1, wx1}, wys[2] = {1.0 - wy1, wy1}, wzs[2] = {1.0 - wz1, wz1};
        for (int i = 0; i < 2; i++) {
            long a = (long)a0 + i;
            if (a < 0 || a >= nx) continue;
            for (int j = 0; j < 2; j++) {
                long b = (long)b0 + j;
                if (b < 0 || b >= ny) continue;
                for (int l = 0; l < 2; l++) {
                    long cz = (long)c0 + l;
                    if (cz < 0 || cz >= nz) continue;
                    double w = wxs[i] * wys[j] * wzs[l];
                    if (w == 0.0) continue;
                    size_t id = IDX(a, b, cz);
                    if (mode == 0)
                        acc += r->ds * w * vol[id];
                    else
                        vol[id] += val * r->ds * w;
                    if (nnz) (*nnz)++;
                }
            }
        }
    }
    return acc;
}

int orc_forward_project(const orc_geom *g, const double *vol, double *sino)
{
    if (orc_check_geometry(g)) return -1;
    const long nrays = (long)g->n_views * g->nv * g->nu;
#pragma omp parallel for schedule(dynamic, 64)
    for (long i = 0; i < nrays; i++) {
        int iu = (int)(i % g->nu);
        int iv = (int)((i / g->nu) % g->nv);
        int view = (int)(i / ((long)g->nu * g->nv));
        ray_t r;
        ray_setup(g, view, iv, iu, &r);
        sino[i] = ray_apply(g, &r, (double *)vol, 0.0, 0, NULL);
    }
    return 0;
}

int orc_forward_rays(const orc_geom *g, const double *vol, int n, const int *view,
                     const int *iv, const int *iu, double *out)
{
    if (orc_check_geometry(g)) return -1;
#pragma omp parallel for schedule(dynamic, 8)
    for (int i = 0; i < n; i++) {
        ray_t r;
        ray_setup(g, view[i], iv[i], iu[i], &r);
        out[i] = ray_apply(g, &r, (double *)vol, 0.0, 0, NULL);
    }
    return 0;
}

int orc_back_project(const orc_geom *g, const double *sino, double *vol)
{
    if (orc_check_geometry(g)) return -1;
    const size_t nvox = (size_t)g->nx * g->ny * g->nz;
    const long nrows = (long)g->n_views * g->nv;
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    double *priv = (double *)calloc((size_t)nt * nvox, sizeof(double));
    if (!priv) return -2;
#pragma omp parallel num_threads(nt)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double *mine = priv + (size_t)t * nvox;
#pragma omp for schedule(static)
        for (long row = 0; row < nrows; row++) {
            int iv = (int)(row % g->nv);
            int view = (int)(row / g->nv);
            for (int iu = 0; iu < g->nu; iu++) {
                double val = sino[(size_t)row * g->nu + iu];
                if (val == 0.0) continue;
                ray_t r;
                ray_setup(g, view, iv, iu, &r);
                ray_apply(g, &r, mine, val, 1, NULL);
            }
        }
    }
    /* fixed-order sum of the per-thread volumes */
#pragma omp parallel for schedule(static)
    for (size_t j = 0; j < nvox; j++) {
        double s = 0.0;
        for (int t = 0; t < nt; t++) s += priv[(size_t)t * nvox + j];
        vol[j] = s;
    }
    free(priv);
    return 0;
}

int64_t orc_count_terms(const orc_geom *g)
{
    if (orc_check_geometry(g)) return -1;
    const long nrays = (long)g->n_views * g->nv * g->nu;
    int64_t total = 0;
    double *dummy = (double *)calloc((size_t)g->nx * g->ny * g->nz, sizeof(double));
    if (!dummy) return -2;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : total)
    for (long i = 0; i < nrays; i++) {
        int iu = (int)(i % g->nu);
        int iv = (int)((i / g->nu) % g->nv);
        int view = (int)(i / ((long)g->nu * g->nv));
        ray_t r;
        int64_t n = 0;
        ray_setup(g, view, iv, iu, &r);
        ray_apply(g, &r, dummy, 0.0, 0, &n);
        total += n;
    }
    free(dummy);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Eq. 6 (with A6, A7): voxel-driven closed-form functional gradient         */
/* ------------------------------------------------------------------------ */

static double detector_bilinear(const orc_geom *g, const double *img, double u, double v)
{
    double fu = u / g->du + 0.5 * (g->nu - 1);
    double fv = v / g->dv + 0.5 * (g->nv - 1);
    double iu0 = floor(fu), iv0 = floor(fv);
    double wu = fu - iu0, wv = fv - iv0;
    double acc = 0.0;
    for (int j = 0; j < 2; j++) {
        long iv = (long)iv0 + j;
        if (iv < 0 || iv >= g->nv) continue;
        for (int i = 0; i < 2; i++) {
            long iu = (long)iu0 + i;
            if (iu < 0 || iu >= g->nu) continue;
            double w = (i ? wu : 1.0 - wu) * (j ? wv : 1.0 - wv);
            acc += w * img[(size_t)iv * g->nu + iu];
        }
    }
    return acc;
}

int orc_eq6_backproject(const orc_geom *g, const double *sino, double *vol)
{
    if (orc_check_geometry(g)) return -1;
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const double L0 = g->sdd;
#pragma omp parallel for collapse(2) schedule(static)
    for (int a = 0; a < nx; a++)
        for (int b = 0; b < ny; b++)
            for (int c = 0; c < nz; c++) {
                double x = (a - 0.5 * (nx - 1)) * g->dx;
                double y = (b - 0.5 * (ny - 1)) * g->dy;
                double z = (c - 0.5 * (nz - 1)) * g->dz;
                double acc = 0.0;
                for (int k = 0; k < g->n_views; k++) {
                    double th = g->angles[k], ct = cos(th), st = sin(th);
                    /* coordinates in the frame where the projection runs along +x */
                    double xr = x * ct + y * st, yr = -x * st + y * ct;
                    double xs = -g->sad, ys = 0.0, zs = 0.0;
                    double us = -(yr - ys) * L0 / (xr - xs);                 /* A6 */
                    double vs = (z - zs) * L0 / (xr - xs);
                    double Ls = sqrt(L0 * L0 + us * us + vs * vs);
                    double l2 = (xr - xs) * (xr - xs) + (yr - ys) * (yr - ys) + (z - zs) * (z - zs);
                    double T = detector_bilinear(g, sino + (size_t)k * g->nu * g->nv, us, vs);
                    acc += 2.0 * Ls * Ls * Ls / (L0 * l2) * T;                /* Eq. 6 */
                }
                vol[IDX(a, b, c)] = acc;
            }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* TV energy (Eq. 2) and the ROF sub-problem (Sec. II.B, Eq. 5)              */
/* ------------------------------------------------------------------------ */

/* Forward differences at voxel (a,b,c). Ghost values on the + side: zero
 * along x and y (zero boundary condition), the voxel itself along z
 * (reflective), so the z difference vanishes at the last slice. */
static void fwd_diff(int nx, int ny, int nz, double dx, double dy, double dz,
                     const double *f, int a, int b, int c, double D[3])
{
    double f0 = f[IDX(a, b, c)];
    double fxp = (a + 1 < nx) ? f[IDX(a + 1, b, c)] : 0.0;
    double fyp = (b + 1 < ny) ? f[IDX(a, b + 1, c)] : 0.0;
    double fzp = (c + 1 < nz) ? f[IDX(a, b, c + 1)] : f0;
    D[0] = (fxp - f0) / dx;
    D[1] = (fyp - f0) / dy;
    D[2] = (fzp - f0) / dz;
}

double orc_tv_e1(int nx, int ny, int nz, double dx, double dy, double dz,
                 const double *f, double eps)
{
    double sum = 0.0;
#pragma omp parallel for collapse(2) reduction(+ : sum) schedule(static)
    for (int a = 0; a < nx; a++)
        for (int b = 0; b < ny; b++)
            for (int c = 0; c < nz; c++) {
                double D[3];
                fwd_diff(nx, ny, nz, dx, dy, dz, f, a, b, c, D);
                sum += sqrt(eps * eps + D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
            }
    return sum / ((double)nx * ny * nz);
}

/* E_ROF[f] = lambda E1[f] + (1/(2 tau)) mean((f - g)^2): Step 2 of Alg. A1
 * divided by mu (lambda = 1/mu, tau = mu/beta in the mean metric). */
double orc_rof_energy(int nx, int ny, int nz, double dx, double dy, double dz,
                      const double *f, const double *g, double lambda, double tau, double eps)
{
    const size_t n = (size_t)nx * ny * nz;
    double fid = 0.0;
#pragma omp parallel for reduction(+ : fid) schedule(static)
    for (size_t j = 0; j < n; j++) fid += (f[j] - g[j]) * (f[j] - g[j]);
    return lambda * orc_tv_e1(nx, ny, nz, dx, dy, dz, f, eps) + fid / (2.0 * tau * (double)n);
}

/* d = N_vox * dE_ROF/df (the functional derivative of Sec. II.C.1 on a grid
 * of unit cell volume), built by differentiating every phi_k with the chain
 * rule and adding the result into the voxels phi_k depends on. */
void orc_rof_gradient(int nx, int ny, int nz, double dx, double dy, double dz,
                      const double *f, const double *g, double lambda, double tau,
                      double eps, double *d)
{
    const size_t n = (size_t)nx * ny * nz;
    for (size_t j = 0; j < n; j++) d[j] = (f[j] - g[j]) / tau;
    /* serial scatter: plain and order-fixed */
    for (int a = 0; a < nx; a++)
        for (int b = 0; b < ny; b++)
            for (int c = 0; c < nz; c++) {
                double D[3];
                fwd_diff(nx, ny, nz, dx, dy, dz, f, a, b, c, D);
                double phi = sqrt(eps * eps + D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
                double qx = lambda * D[0] / (phi * dx);
                double qy = lambda * D[1] / (phi * dy);
                double qz = lambda * D[2] / (phi * dz);
                /* d phi / d f(a,b,c) collects -D_i/(phi h_i) from every axis */
                d[IDX(a, b, c)] -= qx + qy;
                if (a + 1 < nx) d[IDX(a + 1, b, c)] += qx;
                if (b + 1 < ny) d[IDX(a, b + 1, c)] += qy;
                if (c + 1 < nz) {
                    d[IDX(a, b, c)] -= qz;
                    d[IDX(a, b, c + 1)] += qz;
                }
            }
}

int orc_rof_solve(int nx, int ny, int nz, double dx, double dy, double dz,
                  const double *g, double *f, double lambda, double tau,
                  const orc_tv_params *p, const int *replay, int n_replay,
                  int *log, int log_cap, orc_rof_stats *st)
{
    const size_t n = (size_t)nx * ny * nz;
    double *d = (double *)malloc(n * sizeof(double));
    double *ft = (double *)malloc(n * sizeof(double));
    if (!d || !ft) {
        free(d);
        free(ft);
        return -2;
    }
    const double s0 = p->s0 > 0 ? p->s0 : tau;
    orc_rof_stats s = {0, 0, 0.0, 0.0};
    double E0 = orc_rof_energy(nx, ny, nz, dx, dy, dz, f, g, lambda, tau, p->eps_tv);
    s.e_first = E0;
    int steps = replay ? n_replay : p->max_inner;
    for (int it = 0; it < steps; it++) {
        orc_rof_gradient(nx, ny, nz, dx, dy, dz, f, g, lambda, tau, p->eps_tv, d);
        double d2 = 0.0;
        for (size_t j = 0; j < n; j++) d2 += d[j] * d[j];
        d2 /= (double)n;                       /* (1/V) integral of d^2, Eq. 5 */
        if (!replay && (d2 == 0.0 || E0 == 0.0)) break;
        double step = s0, Enew = 0.0;
        int bt, accepted = 0;
        if (replay) {
            for (bt = 0; bt < replay[it]; bt++) step *= p->alpha;
            for (size_t j = 0; j < n; j++) ft[j] = f[j] - step * d[j];
            Enew = orc_rof_energy(nx, ny, nz, dx, dy, dz, ft, g, lambda, tau, p->eps_tv);
            accepted = 1;
        } else {
            for (bt = 0; bt <= p->max_backtracks; bt++) {
                for (size_t j = 0; j < n; j++) ft[j] = f[j] - step * d[j];
                Enew = orc_rof_energy(nx, ny, nz, dx, dy, dz, ft, g, lambda, tau, p->eps_tv);
                if (Enew <= E0 - p->c * step * d2) {   /* Armijo, Eq. 5 */
                    accepted = 1;
                    break;
                }
                step *= p->alpha;
            }
        }
        if (!accepted) {
            s.flags |= 1;
            break;
        }
        memcpy(f, ft, n * sizeof(double));
        if (log && s.n_inner < log_cap) log[s.n_inner] = bt;
        s.n_inner++;
        double rel = fabs(Enew - E0) / E0;
        E0 = Enew;
        if (!replay && rel < p->rel_tol) break;
        if (!replay && it == steps - 1) s.flags |= 2;
    }
    s.e_last = E0;
    if (st) *st = s;
    free(d);
    free(ft);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm A1                                                              */
/* ------------------------------------------------------------------------ */

double orc_data_term(const orc_geom *g, const double *f, const double *y, double *r_out)
{
    const size_t m = (size_t)g->n_views * g->nv * g->nu;
    double *r = r_out ? r_out : (double *)malloc(m * sizeof(double));
    orc_forward_project(g, f, r);
    double e2 = 0.0;
    for (size_t i = 0; i < m; i++) {
        r[i] -= y[i];
        e2 += r[i] * r[i];
    }
    if (!r_out) free(r);
    return e2 / (double)m;
}

int orc_fbs_iteration(const orc_geom *g, const double *y, double *f, double lambda,
                      double tau, const orc_tv_params *p, int clamp,
                      const int *replay, int n_replay, int *log, int log_cap,
                      orc_rof_stats *st, double *e2_out)
{
    const size_t n = (size_t)g->nx * g->ny * g->nz;
    const size_t m = (size_t)g->n_views * g->nv * g->nu;
    double *r = (double *)malloc(m * sizeof(double));
    double *bp = (double *)malloc(n * sizeof(double));
    double *gaux = (double *)malloc(n * sizeof(double));
    if (!r || !bp || !gaux) {
        free(r);
        free(bp);
        free(gaux);
        return -2;
    }
    double e2 = orc_data_term(g, f, y, r);
    orc_back_project(g, r, bp);
    const double kappa = 2.0 * (double)n / (double)m;
    /* Step 1: gradient update of the data term */
    for (size_t j = 0; j < n; j++) gaux[j] = f[j] - tau * kappa * bp[j];
    /* Step 2: ROF, starting from g */
    memcpy(f, gaux, n * sizeof(double));
    int rc = orc_rof_solve(g->nx, g->ny, g->nz, g->dx, g->dy, g->dz, gaux, f, lambda, tau, p,
                           replay, n_replay, log, log_cap, st);
    /* Step 3: non-negativity */
    if (clamp)
        for (size_t j = 0; j < n; j++)
            if (f[j] < 0.0) f[j] = 0.0;
    if (e2_out) *e2_out = e2;
    free(r);
    free(bp);
    free(gaux);
    return rc;
}

double orc_power_lipschitz_from(const orc_geom *g, double *v, int n_iter)
{
    const size_t n = (size_t)g->nx * g->ny * g->nz;
    const size_t m = (size_t)g->n_views * g->nv * g->nu;
    const double kappa = 2.0 * (double)n / (double)m;
    double *w = (double *)malloc(n * sizeof(double));
    double *s = (double *)malloc(m * sizeof(double));
    double L = 0.0;
    for (int it = 0; it < n_iter; it++) {
        orc_forward_project(g, v, s);
        orc_back_project(g, s, w);
        double nv2 = 0.0, nw2 = 0.0;
        for (size_t j = 0; j < n; j++) {
            w[j] *= kappa;
            nv2 += v[j] * v[j];
            nw2 += w[j] * w[j];
        }
        L = sqrt(nw2) / sqrt(nv2);
        double inv = 1.0 / sqrt(nw2);
        for (size_t j = 0; j < n; j++) v[j] = w[j] * inv;
    }
    free(w);
    free(s);
    return L;
}

double orc_power_lipschitz(const orc_geom *g, int n_iter)
{
    const size_t n = (size_t)g->nx * g->ny * g->nz;
    double *v = (double *)malloc(n * sizeof(double));
    for (size_t j = 0; j < n; j++) v[j] = 1.0;
    const double L = orc_power_lipschitz_from(g, v, n_iter);
    free(v);
    return L;
}

/* ------------------------------------------------------------------------ */
/* Multigrid prolongation (Sec. II.C.3)                                      */
/* ------------------------------------------------------------------------ */

static void lin_coord(int nc, int i, int *i0, double *w)
{
    /* fine cell i has centre at coarse continuous index (i + 0.5)/2 - 0.5 */
    double I = 0.5 * (i + 0.5) - 0.5;
    if (I < 0.0) I = 0.0;
    if (I > nc - 1) I = nc - 1;
    int k = (int)floor(I);
    if (k > nc - 2) k = nc - 2;
    if (k < 0) k = 0;
    *i0 = k;
    *w = (nc == 1) ? 0.0 : I - k;
}

void orc_prolong(int ncx, int ncy, int ncz, const double *coarse, double *fine)
{
    const int nx = 2 * ncx, ny = 2 * ncy, nz = 2 * ncz;
    for (int a = 0; a < nx; a++)
        for (int b = 0; b < ny; b++)
            for (int c = 0; c < nz; c++) {
                int a0, b0, c0;
                double wa, wb, wc;
                lin_coord(ncx, a, &a0, &wa);
                lin_coord(ncy, b, &b0, &wb);
                lin_coord(ncz, c, &c0, &wc);
                double acc = 0.0;
                for (int i = 0; i < 2; i++)
                    for (int j = 0; j < 2; j++)
                        for (int l = 0; l < 2; l++) {
                            double w = (i ? wa : 1 - wa) * (j ? wb : 1 - wb) * (l ? wc : 1 - wc);
                            if (w == 0.0) continue;
                            int ai = a0 + i < ncx ? a0 + i : ncx - 1;
                            int bj = b0 + j < ncy ? b0 + j : ncy - 1;
                            int cl = c0 + l < ncz ? c0 + l : ncz - 1;
                            acc += w * coarse[((size_t)ai * ncy + bj) * ncz + cl];
                        }
                fine[((size_t)a * ny + b) * nz + c] = acc;
            }
}
