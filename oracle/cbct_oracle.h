/*
 * FP64 CPU oracle for TV-regularised cone-beam CT reconstruction
 * (Jia et al., "GPU-based Fast Low-dose Cone Beam CT Reconstruction via
 * Total Variation", arXiv:1001.0599).
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, deliberately unoptimised
 * restatement of the method used to check the CUDA library. Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * it. It shares no code, header, table or constant with the CUDA path.
 *
 * Conventions (the paper leaves them to Fig. 1, whose image is missing; the
 * signs follow Eq. A2 at angle 0):
 *   - volume f[a][b][c] (c = z fastest), voxel centres x_a = (a-(nx-1)/2)dx,
 *     likewise y, z; z is the rotation (superior-inferior) axis;
 *   - sinogram s[view][iv][iu] (u fastest); pixel centres
 *     u = (iu-(nu-1)/2)du, v = (iv-(nv-1)/2)dv;
 *   - source S = Rz(theta)(-sad,0,0); detector centre Rz(theta)(sdd-sad,0,0);
 *     detector axes e_u = Rz(theta)(0,-1,0), e_v = (0,0,1).
 *
 * Parity pins: every function here is pinned by a test in tests/ against a
 * closed form, a library routine or a brute-force evaluation, except the
 * image-quality metrics of Sec. III (parity unpinned: no paper number exists
 * for synthetic phantoms).
 */
#ifndef CBCT_ORACLE_H
#define CBCT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    int nu, nv;
    double du, dv;
    double sad, sdd;
    int n_views;
    const double *angles;   /* radians, n_views entries */
    double step_ratio;      /* in-plane sample spacing / min(dx, dy) */
} orc_geom;

typedef struct {
    double eps_tv;          /* smoothing of |grad f| inside the square root */
    double c;               /* Armijo constant (Eq. 5): 0.01 */
    double alpha;           /* step reduction factor: 0.6 */
    double rel_tol;         /* stop when |E_new - E_0| / E_0 < rel_tol: 1e-3 */
    int max_inner;          /* cap on gradient-descent steps */
    int max_backtracks;     /* cap on step reductions per step */
    double s0;              /* initial trial step; <= 0 means tau */
} orc_tv_params;

/* Per ROF solve: log[i] = number of step reductions before step i was
 * accepted; n_inner = accepted steps; flags bit 0 = a step found no
 * acceptable size (the solve ends there), bit 1 = max_inner reached. */
typedef struct {
    int n_inner;
    int flags;
    double e_first;         /* E_ROF at the start */
    double e_last;          /* E_ROF at the end */
} orc_rof_stats;

int  orc_check_geometry(const orc_geom *g);
double orc_drho(const orc_geom *g);

/* Eq. 1, discretised: p = sum_k ds * f(S + k*drho * n / |n_xy|). */
int  orc_forward_project(const orc_geom *g, const double *vol, double *sino);
/* same for a list of rays (view, iv, iu triples) */
int  orc_forward_rays(const orc_geom *g, const double *vol, int n,
                      const int *view, const int *iv, const int *iu, double *out);
/* exact transpose of orc_forward_project (scatter form) */
int  orc_back_project(const orc_geom *g, const double *sino, double *vol);
/* number of (ray, sample, voxel) terms with non-zero weight */
int64_t orc_count_terms(const orc_geom *g);

/* Eq. 6: the paper's voxel-driven closed-form gradient (unmatched); returns
 * sum_theta 2 L^3 / (L0 l^2) T(u*, v*) with T bilinearly interpolated on the
 * detector (zero outside), WITHOUT the 1/(N_theta A) prefactor. */
int  orc_eq6_backproject(const orc_geom *g, const double *sino, double *vol);

/* Eq. 2 energies with mean normalisation. */
double orc_tv_e1(int nx, int ny, int nz, double dx, double dy, double dz,
                 const double *f, double eps);
double orc_rof_energy(int nx, int ny, int nz, double dx, double dy, double dz,
                      const double *f, const double *g, double lambda, double tau, double eps);
void orc_rof_gradient(int nx, int ny, int nz, double dx, double dy, double dz,
                      const double *f, const double *g, double lambda, double tau,
                      double eps, double *d);
/* Sec. II.B sub-problem: gradient descent with Armijo backtracking (Eq. 5).
 * f holds the start on entry (normally f = g) and the result on exit.
 * If replay != NULL the step sizes are taken from replay[0..n_replay-1]
 * (reduction counts) instead of being searched. log may be NULL. */
int orc_rof_solve(int nx, int ny, int nz, double dx, double dy, double dz,
                  const double *g, double *f, double lambda, double tau,
                  const orc_tv_params *p, const int *replay, int n_replay,
                  int *log, int log_cap, orc_rof_stats *st);

/* data term E2 = sum r^2 / (N_theta N_pix) of r = P f - y */
double orc_data_term(const orc_geom *g, const double *f, const double *y, double *r_out);

/* One Algorithm A1 iteration: g = f - tau*kappa*P^T(P f - y); f = ROF(g);
 * f = max(f, 0) when clamp != 0.  kappa = 2 N_vox / (N_theta N_pix). */
int orc_fbs_iteration(const orc_geom *g, const double *y, double *f, double lambda,
                      double tau, const orc_tv_params *p, int clamp,
                      const int *replay, int n_replay, int *log, int log_cap,
                      orc_rof_stats *st, double *e2_out);

/* Lipschitz constant of kappa P^T P by power iteration from v = 1. */
double orc_power_lipschitz(const orc_geom *g, int n_iter);
/* Same from the start vector v (any scale); on return v holds the last
 * normalised iterate. */
double orc_power_lipschitz_from(const orc_geom *g, double *v, int n_iter);

/* Cell-centred trilinear prolongation from (nx/2, ny/2, nz/2) to (nx, ny, nz),
 * clamp to edge (Sec. II.C.3). */
void orc_prolong(int ncx, int ncy, int ncz, const double *coarse, double *fine);

#ifdef __cplusplus
}
#endif
#endif
