/*
 * recon_oracle.h -- plain CPU FP64 oracle of the nonlinear-reconstruction
 * displacement-potential solve (Zhu, Yu, Pen, Chen & Yu 2016, "Nonlinear
 * reconstruction", arXiv:1611.09638, Sec. II and Appendix A).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and recon_oracle.c are the slow,
 * obviously-correct reference that the CUDA library is checked against.  Only
 * the tests, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Conventions (the same on both sides, stated independently):
 *   - Periodic vertex grid, n[0] x n[1] x n[2] nodes, spacing 1 (grid units),
 *     C order with the last axis fastest: idx = (i*n1 + j)*n2 + k.
 *   - Densities and masses in units of the mean density rho_bar, so the target
 *     mass per curvilinear cell is exactly 1.
 *   - Tracer / particle coordinates are stored as np x 3 row-major doubles.
 *
 * Every function returns 0 on success and a negative value on invalid input.
 */
#ifndef RECON_ORACLE_H
#define RECON_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Compression-limiter readings of the printed App. A formula for C. */
#define ORC_CLIM_SOFT 0     /* C = 4 max(0, xi_m/lambda0 - 1)^2                */
#define ORC_CLIM_LITERAL 1  /* C = 4 [xi_m/lambda0 - H(xi_m/lambda0 - 1)]^2     */
#define ORC_CLIM_STEP 2     /* C = 4 [(xi_m/lambda0) H(xi_m/lambda0 - 1)]^2     */

typedef struct {
    int n[3];               /* grid nodes per axis: powers of two, >= 8          */
    double xi_m;            /* maximal compression factor (App. A), 0.1          */
    double v_m;             /* expansion volume limit (App. A), 10               */
    double a_min;           /* coefficient floor in voids, 0.01                  */
    int climiter;           /* ORC_CLIM_*                                        */
    double s_side;          /* smoothing S: per-axis side weight, 1/4            */
    int nu1, nu2;           /* pre / post RB-GS sweeps per V-cycle level          */
    double tol_in;          /* multigrid: stop at ||s - L phidot|| <= tol_in ||s|| */
    int max_vcycles;        /* multigrid: V-cycle cap per outer step             */
    double tol_out;         /* outer: stop when rms(s) <= tol_out                */
    int k_max;              /* outer: step cap                                   */
    double d_max;           /* step limiter: max |alpha grad dphi| in cells      */
    double alpha_min;       /* step limiter: smallest admissible alpha           */
    double lambda_floor;    /* step limiter: required lambda_min(I + Hess phi)   */
    int density_update;     /* 0: CIC re-deposit of tracers each step; 1: the
                               linear update m += alpha D(dphi) of App. A      */
    int warm_start;         /* initial guess of each step's linear solve (the
                               paper does not state it): 0: phidot = 0; 1: the
                               last step's phidot; 2: extrapolated from the
                               last two, phidot_{k-1} + (alpha_{k-1} /
                               alpha_{k-2}) (phidot_{k-1} - phidot_{k-2}) (step
                               1 takes phidot_0)                               */
} orc_params;

/* Per-step record of orc_solve (arrays of length k_max, caller-owned; any may
 * be NULL). */
typedef struct {
    double* alpha;      /* accepted step length alpha_k                          */
    double* R;          /* rms(s) at the start of step k                         */
    int* ncycles;       /* V-cycles used by the step's linear solve              */
    double* relres;     /* final ||s - L phidot|| / ||s|| of the step            */
    double* min_det;    /* min over nodes of det(I + Hess phi) at step start     */
    double* min_lam;    /* min over nodes of lambda0 at step start               */
    double* mass;       /* sum of the deposited mass m at step start             */
} orc_trace;

/* Threads for the loops that split over planes (OpenMP builds; results do
 * not depend on the count).  nthreads > 0 sets the count; returns the count
 * in use (1 in a build without OpenMP). */
int orc_set_threads(int nthreads);

/* CIC deposit (Sec. III density gridding; Sec. IV "assign particles to a
 * uniform grid"): out[j] = sum_p w_p prod_a max(0, 1 - |d_a|), d = x_p - j wrapped
 * periodically.  x in grid units, w == NULL means unit masses. */
int orc_cic_deposit(const int n[3], const double* x, const double* w, int64_t np,
                    double* out);

/* L u = sum_a h_a^-2 [A+ (u+ - u) - A- (u - u-)], A+- = (a + a+-)/2 at level
 * dims n with spacing h (App. A, Eq. elliptic with x ~ xi). */
int orc_apply_L(const int n[3], const double h[3], const double* a, const double* u,
                double* out);
/* One red-black Gauss-Seidel sweep (red = (i+j+k) even first) of L u = f. */
int orc_rbgs_sweep(const int n[3], const double h[3], const double* a, const double* f,
                   double* u);
/* Full-weighting restriction fine n -> coarse; axis a is coarsened iff n[a] > 4. */
int orc_restrict(const int n[3], const double* fine, double* coarse);
/* Trilinear prolongation of a coarse field onto fine dims n, added to fine. */
int orc_prolong_add(const int n[3], const double* coarse, double* fine);
/* Smoothing operator S (App. A, "nearest neighbours"): the weighted mean over
 * the 3x3x3 neighbourhood with weights (s_side, 1 - 2 s_side, s_side) per
 * axis.  With s_side = 1/4 it removes every mode with some k_a = pi. */
int orc_apply_S(const int n[3], double s_side, const double* u, double* out);
/* One V(nu1,nu2) cycle on L(a) u = f, updating u in place. */
int orc_vcycle(const orc_params* p, const double* a, const double* f, double* u);
/* Multigrid solve of L(a) u = s from u = 0 (App. A: "multigrid algorithm").
 * u is determined up to a constant (periodic operator); its mean is not
 * removed here.  Returns the cycle count in *ncycles and ||s-Lu||/||s|| in
 * *relres. */
int orc_mg_solve(const orc_params* p, const double* a, const double* s, double* u,
                 int* ncycles, double* relres);
/* The same solve from the initial guess held in u (a V-cycle is affine in u,
 * so this equals u0 plus the solve of L e = s - L u0 from e = 0, stopped at
 * the same absolute residual tol_in ||s||).  At least one cycle runs. */
int orc_mg_solve_from(const orc_params* p, const double* a, const double* s, double* u,
                      int* ncycles, double* relres);

/* Geometry of the map x = xi + grad phi (Eq. mapping): per node the volume
 * element sqrt_g = det(I + Hess phi) and the minimum eigenvalue lambda0 of the
 * triad (App. A).  Either output may be NULL. */
int orc_geometry(const int n[3], const double* phi, double* sqrt_g, double* lambda0);
/* Source of App. A Eq. (elliptic): t = Sigma + C + E with Sigma = 1 - m,
 * s = S t - mean(S t).  t_out may be NULL. */
int orc_source(const orc_params* p, const double* phi, const double* m, double* s,
               double* t_out);
/* Step limiter: largest alpha in {1, 1/2, 1/4, ...} >= alpha_min with
 * lambda_min(I + Hess(phi) + alpha Hess(dphi)) > lambda_floor at every node and
 * alpha max|grad dphi| <= d_max.  Returns 0 and *alpha, or -5 if none. */
int orc_step_limiter(const orc_params* p, const double* phi, const double* dphi,
                     double* alpha);
/* Mesh advance: every tracer xi_c -= alpha V(xi_c), V = (I + Hess phi)^-1 G at
 * the nodes (phi before the update), G the central-difference gradient of
 * dphi, interpolated with CIC weights; then phi += alpha dphi. */
int orc_advance(const int n[3], double alpha, const double* dphi, double* phi,
                double* xi, int64_t np);

/* Exact change of the mass per curvilinear cell under a mesh motion grad v
 * (App. A, Eq. elliptic_diff): out = d_mu (m (e^-1)^{mu nu} d_nu v), e = I +
 * Hess phi, in flux form: each axis' second difference with face coefficients
 * (K_c + K_n)/2 of K = m e^-1, and each cross term as the difference of
 * centred differences, so that sum(out) = 0. */
int orc_mass_change(const int n[3], const double* phi, const double* m, const double* v,
                    double* out);

/* Whole solve (Sec. II moving-mesh iteration, App. A).  rho: density on the
 * grid (any positive units).  phi: output, n cells.  xi: optional np = ncells
 * x 3 output of final tracer coordinates.  m_out: optional final deposit.
 * replay_alpha: optional length-k_max array forcing alpha_k instead of the
 * limiter search.  Returns 0 converged, 1 k_max reached, 2 stopped because
 * the step limiter found no alpha >= alpha_min (outputs are the last valid
 * map), <0 error.
 * *steps receives the number of completed advances. */
int orc_solve(const orc_params* p, const double* rho, const double* replay_alpha,
              double* phi, double* xi, double* m_out, int* steps, orc_trace* tr);

/* Outputs (Sec. II Eq. rec, Sec. III): delta_r = -Laplacian_7 phi, and the
 * Eulerian node positions x_j = j + central-difference grad phi (ncells x 3). */
int orc_delta_r(const int n[3], const double* phi, double* out);
int orc_mesh_x(const int n[3], const double* phi, double* out);

/* Minimum eigenvalue of a symmetric 3x3 matrix by cyclic Jacobi rotations. */
double orc_min_eig_sym3(const double A[3][3]);

/* Vector-Jacobian product of the map rho -> delta_r of a solve (Sec. II,
 * App. A; tracer re-deposit form) over its K advances with the step lengths
 * alpha[0..K-1] held fixed (the limiter's choice is piecewise constant in
 * rho).  gbar: dL/d delta_r (ncells, grid units); grad: dL/d rho (ncells).
 * The reverse sweep goes through the steps in the opposite order: the phi
 * update, the tracer advance xi -= alpha e^-1 grad dphi (CIC interpolation),
 * dphi = S phidot - mean, the linear solve L(a) phidot = s (its adjoint is a
 * solve with the same symmetric operator, and the coefficient sensitivity
 * is (1/2) sum over a node's faces of the face differences of the two
 * solutions), a = max(m, a_min), s = S t - mean, the source
 * t = Sigma + C(lambda0) + E (d lambda0 = v^T de v with v the eigenvector of
 * lambda0; the Heaviside factors have zero derivative almost everywhere),
 * the geometry e = I + Hess phi, and the CIC deposit of the tracers' masses;
 * finally w = rho / mean(rho).  Both linear solves run to p->tol_in.
 * Requires density_update = 0.  Returns 0 or <0 (invalid input, no memory). */
int orc_adjoint(const orc_params* p, const double* rho, const double* alpha, int K,
                const double* gbar, double* grad);

#ifdef __cplusplus
}
#endif
#endif
