/*
 * recon.h -- C ABI of the GB300 (sm_103a) nonlinear-reconstruction solver.
 *
 * The library solves for the displacement potential phi(xi) of "Nonlinear
 * reconstruction" (Zhu, Yu, Pen, Chen & Yu 2016, arXiv:1611.09638): the
 * pure-gradient coordinate map x = xi + grad phi (Sec. II, Eq. mapping) that
 * stays positive definite and carries an observed density to constant mass per
 * curvilinear cell.  It is found by the moving-mesh iteration of Sec. II and
 * App. A: each step deposits the density on the deformed mesh by CIC, builds
 * the limited, smoothed source S(Sigma + C + E) of App. A Eq. (elliptic),
 * solves the linearised elliptic equation with variable-coefficient multigrid
 * V-cycles, limits the step so the map stays positive definite, and advances
 * the mesh.  The output is the reconstructed density delta_r = -lap phi
 * (Sec. II, Eq. rec).
 *
 * Conventions
 *   - Periodic vertex grid of n[0] x n[1] x n[2] nodes (each a power of two,
 *     >= 8), C order with the last axis fastest: idx = (i*n1 + j)*n2 + k.
 *   - Cells are cubes of side h = box[a] / n[a] (all three equal).  With
 *     box = {0,0,0} the grid unit is used (h = 1).
 *   - Every array argument of the handle calls is a plain pointer to host OR
 *     device memory (the library tells them apart through unified
 *     addressing); host memory and another device's memory are copied to the
 *     handle's device (the device current at recon_create) before a kernel
 *     reads them.  Inputs are borrowed for the duration of the call only; the
 *     handle owns all of its device state.
 *   - Every call returns a status (RECON_OK = 0, errors < 0, RECON_NOT_CONVERGED
 *     = 1 is a warning with valid results) and never traps or aborts; the
 *     thread-local text of the last error is returned by recon_last_error().
 *   - All work runs on the CUDA stream given at create.  recon_solve and
 *     recon_field return after the stream has finished their work.
 */
#ifndef RECON_H
#define RECON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RECON_OK 0
#define RECON_NOT_CONVERGED 1 /* k_max steps done before rms(s) <= tol_out */
#define RECON_STALLED 2       /* the step limiter found no alpha >= alpha_min;
                                 the iteration stopped, results are the last
                                 (positive definite) map                    */
#define RECON_E_INVALID (-1)  /* bad argument / parameter                  */
#define RECON_E_OOM (-2)      /* device allocation failed                 */
#define RECON_E_CUDA (-3)     /* a CUDA runtime call failed               */
#define RECON_E_NONFINITE (-4) /* NaN/Inf or negative input               */
#define RECON_E_LIMITER (-5)  /* reserved (a limiter stall is RECON_STALLED) */
#define RECON_E_TIMEOUT (-6)  /* a bounded wait on the device ran out (the
                                 bulk-copy waits of the streaming sweep); no
                                 call waits on the device without a bound  */
#define RECON_E_STATE (-7)    /* call out of order (e.g. solve before deposit) */
#define RECON_E_UNSUPPORTED (-8) /* reserved: every declared call is built  */

/* arithmetic of the solve */
#define RECON_FP64 0  /* every step in FP64                                   */
#define RECON_MIXED 1 /* FP32 smoothing / restriction / prolongation inside an
                         FP64 defect correction; residual, phi, mesh, limiter FP64
                         (the multigrid stopping test's norm of the FP64 residual
                         is summed from its FP32 copy)                           */

/* readings of the printed compression limiter C(phi) of App. A */
#define RECON_CLIM_SOFT 0    /* C = 4 max(0, xi_m/lambda0 - 1)^2            */
#define RECON_CLIM_LITERAL 1 /* C = 4 [xi_m/lambda0 - H(xi_m/lambda0 - 1)]^2 */
#define RECON_CLIM_STEP 2    /* C = 4 [(xi_m/lambda0) H(xi_m/lambda0 - 1)]^2 */

/* recon_deposit modes */
#define RECON_PARTICLES 0 /* data: np x 3 positions (box units), mass: np or NULL */
#define RECON_GRID 1      /* data: n[0]*n[1]*n[2] density values, mass: NULL      */

/* recon_field selectors (all FP64) */
#define RECON_FIELD_PHI 0      /* phi, in box units squared (h^2 x grid units)   */
#define RECON_FIELD_DELTA_R 1  /* delta_r = -7-point Laplacian of phi (Eq. rec)   */
#define RECON_FIELD_MESH_X 2   /* ncells x 3: x = xi + central grad phi, box units */
#define RECON_FIELD_MASS 3     /* m: mass per curvilinear cell / mean, last deposit */
#define RECON_FIELD_DET 4      /* sqrt(g) = det(I + Hess phi)                      */
#define RECON_FIELD_LAMBDA0 5  /* minimum eigenvalue of I + Hess phi               */
#define RECON_FIELD_DENSITY 6  /* the deposited input density rho (as given/gridded) */

typedef struct {
    int n[3];            /* grid nodes per axis                                */
    double box[3];       /* box side per axis in physical units, or all 0      */
    int precision;       /* RECON_FP64 or RECON_MIXED                          */
    double xi_m;         /* maximal compression factor, 1/10 (App. A)          */
    double v_m;          /* expansion volume limit, 10 (App. A)                */
    double a_min;        /* floor of the operator coefficient in voids, 0.01   */
    int climiter;        /* RECON_CLIM_*                                       */
    double s_side;       /* smoothing S: per-axis side weight of the 3x3x3 mean, 1/4 */
    int nu1, nu2;        /* pre / post red-black Gauss-Seidel sweeps per level;
                            -1 (default): 2 / 2 in RECON_FP64, 1 / 1 in
                            RECON_MIXED (see recon_resolve_params)            */
    double tol_in;       /* stop the linear solve at ||s - L phidot|| <= tol_in ||s|| */
    int max_vcycles;     /* V-cycle cap per step; -1 (default): 50 in
                            RECON_FP64, 100 in RECON_MIXED                      */
    double tol_out;      /* stop the iteration when rms(s) <= tol_out          */
    int k_max;           /* step cap, 200: the iteration runs to its own end
                            (rms(s) <= tol_out, or no admissible step)         */
    double d_max;        /* step limiter: max |alpha grad dphi| in cells       */
    double alpha_min;    /* step limiter: smallest admissible alpha            */
    double lambda_floor; /* step limiter: lambda_min(I + Hess phi) must exceed it */
    const double* replay_alpha; /* optional host array[k_max]: force alpha_k   */
    int profile;         /* nonzero: time the finest-level smoothing sweeps with
                            CUDA events (reported in recon_stats.smooth_ms)    */
    int inner_vcycles;   /* RECON_MIXED: FP32 V-cycles per FP64 defect
                            correction (1..16; -1, the default: 5 with per-face
                            coarse coefficients, else 6); the FP64 residual is
                            formed once per group, so the stopping test sees
                            multiples of it                                     */
    int density_update;  /* 0: CIC re-deposit of the tracers on the deformed mesh
                            every step (default); 1: App. A's linear update
                            m += alpha d_mu(m e^-1 d dphi) of the mass per cell  */
    int device_loop;     /* 1 (default): the whole iteration runs as one CUDA graph
                            whose conditional nodes the device sets (step loop,
                            multigrid loop, step acceptance), with no host round
                            trip until the solve ends; 0: host-driven loop that
                            reads each decision back.  profile forces 0.        */
    int checkpoint;      /* 1: every step keeps phi_k, the tracer offsets and
                            phidot_k on the device for recon_adjoint
                            (5 x 8 bytes x cells x k_max, allocated at create);
                            needs density_update = 0.  Default 0.               */
    int stream_planes;   /* RECON_MIXED: i-planes per block of the streaming FP32
                            red-black sweep on every level it runs on.  0 (the
                            default): the fastest of 4, 8 and 16, timed per level
                            at create; 4, 8 or 16: that value wherever the level's
                            first dimension is a multiple of it.  Every choice
                            computes the same bits.                            */
    int restrict_planes; /* RECON_MIXED: coarse i-planes per block of the
                            streaming residual + full-weighting restriction.  0
                            (the default): timed per level at create; 1, 2, 4, 8
                            or 16: that value wherever it divides the coarse
                            level.  Every choice computes the same bits.         */
    int coarse_faces;    /* RECON_MIXED, cubic grids: how the FP32 V-cycle's
                            coarse levels carry the coefficient.  0: a nodal
                            coefficient restricted by full weighting, faces its
                            two-node means (the re-discretised operator of
                            RECON_FP64); 1: per-face coefficients, each the
                            full-weighted mean over the fine lines beneath it of
                            the series (harmonic) combination of the two fine
                            faces it spans.  Either way the solve stops at the
                            same FP64 residual; 1 takes fewer V-cycles where the
                            coefficient jumps.  1 needs RECON_MIXED and a cubic
                            grid of at least 64^3.  -1 (default): 1 where that
                            holds, else 0.                                     */
    int tune_inner;      /* RECON_MIXED: 1: the first recon_solve on the handle
                            times the first step's linear solve with 3, 4, 5, 6
                            and 8 FP32 V-cycles per FP64 defect correction and
                            keeps the fastest for this and later solves (the
                            solution is the same to the stopping residual; the
                            choice follows the timing); 2: the same over every
                            smoothing schedule (nu1, nu2) in (1,1), (1,2),
                            (2,1), (2,2) as well.  Ignored with profile.
                            0 (default): keep inner_vcycles, nu1 and nu2.       */
    int group_max;       /* RECON_MIXED: the most FP32 V-cycles one FP64 defect
                            correction may run (inner_vcycles .. 64).  Above
                            inner_vcycles the V-cycles run in blocks of
                            inner_vcycles, and after each block the device
                            decides, from the contraction per V-cycle the last
                            FP64 residual showed, whether to form the next FP64
                            residual now or to run another block first (fewer
                            FP64 residuals per step).  -1 (default):
                            inner_vcycles, one FP64 residual per group.         */
    int tma;             /* RECON_MIXED: 1 (default): the streaming FP32 sweep
                            stages the u, a and f planes of tiles clear of the
                            periodic seams with bulk tensor copies (TMA) into
                            shared memory; 0: every tile uses per-thread 16-byte
                            copies.  Both compute the same bits.  A sweep whose
                            wait for a copy runs out (~1 s) makes recon_solve
                            return RECON_E_TIMEOUT.                            */
    int warm_start;      /* initial guess of each step's linear solve (the paper
                            leaves it open; every choice stops at the same
                            residual tol_in ||s||).  2 (default): extrapolated
                            from the last two steps' phidot,
                            phidot_{k-1} + (alpha_{k-1} / alpha_{k-2})
                            (phidot_{k-1} - phidot_{k-2}) (one more FP64 array);
                            1: the last step's phidot; 0: phidot = 0.  Before
                            the first step phidot = 0, and step 1 takes
                            phidot_0 under 2.                                  */
} recon_params;

/* Per-solve record.  The per-step arrays are optional caller-owned host
 * buffers of length k_max (NULL to skip). */
typedef struct {
    int status;          /* same value recon_solve returned                    */
    int steps;           /* mesh advances done                                 */
    int vcycles;         /* V-cycles over all steps                            */
    double R0, R;        /* rms(s) at the first and at the last step start     */
    double min_det;      /* min det(I + Hess phi) at the end                   */
    double min_lambda0;  /* min lambda0 at the end                             */
    double max_delta_r;  /* max delta_r at the end                             */
    double mass_error;   /* |sum m - ncells| / ncells at the last deposit      */
    double ms;           /* wall time of the solve (CUDA events), milliseconds */
    double* alpha;       /* [k_max] accepted alpha per step                    */
    double* Rk;          /* [k_max] rms(s) at step start                       */
    int* ncycles;        /* [k_max] V-cycles per step                          */
    double* relres;      /* [k_max] final relative residual per step           */
    long long launches;  /* kernels this solve launched                        */
    double smooth_ms;    /* with params.profile: time in finest-level sweeps   */
    int smooth_sweeps;   /* with params.profile: number of those sweeps        */
    double smooth_bytes; /* algorithmic bytes of one such sweep (read u, a, f;
                            write u), for the roofline                          */
    int inner_vcycles;   /* RECON_MIXED: FP32 V-cycles per FP64 defect correction
                            the solve used (params.tune_inner may have chosen it) */
    int nu1, nu2;        /* pre / post sweeps per level the solve used           */
} recon_stats;

/* Fill *p with the defaults above for an n0 x n1 x n2 grid (grid units,
 * FP64).  The multigrid settings nu1, nu2, inner_vcycles and max_vcycles are
 * left at -1, which recon_create resolves by p->precision.  Always succeeds
 * for a non-NULL p. */
int recon_default_params(recon_params* p, int n0, int n1, int n2);

/* Replace, in place, every multigrid setting of *p left at -1 by the value
 * recon_create uses for p->precision and p->n (nu1 = nu2 = 2, max_vcycles =
 * 50 and coarse_faces = 0 in RECON_FP64; in RECON_MIXED nu1 = nu2 = 1,
 * max_vcycles = 100, coarse_faces = 1 on cubic grids of at least 64^3 (else
 * 0), and inner_vcycles = 5 with coarse_faces = 1, else 6; group_max =
 * inner_vcycles).  The paper leaves the cycle shape open; these are the
 * settings that reach the stopping residual in the least time on the 256^3
 * workload.  Other fields are not touched or checked.  RECON_E_INVALID for
 * a NULL p. */
int recon_resolve_params(recon_params* p);

/* Create a solver (Sec. II, App. A): validates p (dims powers of two >= 8,
 * cubic cells, 0 < xi_m < 1, v_m > 1, ...), allocates every device buffer of
 * the grid and its multigrid hierarchy on the current device, and binds the
 * handle to cuda_stream (a cudaStream_t; NULL = the legacy default stream).
 * On error *out is NULL. */
int recon_create(void** out, const recon_params* p, void* cuda_stream);

/* Grid the observed density (Sec. III, "generate the density field on a
 * grid").  RECON_PARTICLES: data holds np x 3 positions in box units (any real
 * value; wrapped periodically), mass holds np masses or is NULL for unit mass;
 * the CIC deposit accumulates in 64-bit fixed point, so the result does not
 * depend on the order of the particles.  RECON_GRID: data holds the density on
 * the grid (np must equal the cell count), mass must be NULL.  Rejects
 * NaN/Inf, negative masses or densities, and zero total mass.  Particle
 * arrays in host memory (or on another device) are copied into a device
 * staging buffer that the handle keeps, sized to the largest such input,
 * until recon_destroy. */
int recon_deposit(void* h, int mode, const double* data, const double* mass, int64_t np);

/* Run the whole moving-mesh solve from phi = 0 on the deposited density
 * (Sec. II; App. A).  Returns RECON_OK when rms(s) <= tol_out,
 * RECON_NOT_CONVERGED after k_max steps, RECON_STALLED when the step limiter
 * admits no alpha >= alpha_min (results valid in all three), or an error.
 * stats may be NULL; with stats, the end-of-solve minima of det and lambda0
 * and the maximum of delta_r are computed as well.  With device_loop = 1 the
 * first call on a handle records the iteration as a CUDA graph (on private
 * streams) and every call launches it on the handle's stream; later deposits
 * on the handle reuse it.  The call returns when the stream has finished. */
int recon_solve(void* h, recon_stats* stats);

/* recon_solve_batch: solves count independent problems (for example many
 * mock catalogues of different sizes), one per handle, each as recon_solve
 * would.  Every handle created with device_loop = 1 has its whole solve
 * launched (as one CUDA graph on the handle's own stream) before the call
 * waits for any of them, so handles created on distinct streams run their
 * solves concurrently on the device; handles with device_loop = 0 are solved
 * one after another while the others run.  Each handle must have a deposited
 * density and may appear once.  stats: NULL, or an array of count records
 * filled as by recon_solve.  Returns RECON_OK when every solve returned a
 * non-negative status (RECON_NOT_CONVERGED / RECON_STALLED are reported per
 * handle in stats), else the first negative status; the handles whose solve
 * failed are left without a result.  Not a method of the paper: it batches
 * the iteration of Sec. II / App. A over independent inputs. */
int recon_solve_batch(void* const* handles, int count, recon_stats* stats);

/* Copy one output field (RECON_FIELD_*) of the last solve to dst (host or
 * device), dst_bytes >= its size (ncells x 8, MESH_X ncells x 24). */
int recon_field(void* h, int which, void* dst, size_t dst_bytes);

/* recon_adjoint: vector-Jacobian product of the last solve (Sec. II, App. A)
 * from grad_delta_r = dL/d(delta_r) to grad_rho = dL/d(rho), with the step
 * lengths alpha_k held at the values that solve chose (the limiter's choice
 * is piecewise constant in rho; the Heaviside switches of the limiters have
 * zero derivative almost everywhere).  rho is the density grid of the last
 * recon_deposit (for RECON_PARTICLES: the particles' CIC grid).  Both buffers
 * hold ncells doubles in C order (z fastest), host or device, caller-owned;
 * delta_r is in the units recon_field returns it.  The sweep goes back
 * through the steps with the states the solve kept (params.checkpoint = 1)
 * and runs one adjoint linear solve per step with the forward's multigrid
 * and tolerance.  One step of the sweep (the transpose of the tracers' CIC
 * interpolation) accumulates with FP64 atomics, so results agree between runs
 * to rounding, not bit for bit.  Afterwards recon_field returns the solve's
 * outputs as before.  Returns RECON_E_INVALID for NULL arguments and
 * RECON_E_STATE without checkpoints or a completed solve. */
int recon_adjoint(void* h, const double* grad_delta_r, double* grad_rho);

/* Release every device buffer of the handle (after finishing its stream). */
void recon_destroy(void* h);

/* Text of the last error on this thread ("" if none). */
const char* recon_last_error(void);

/* CIC deposit of particles without any device allocation.  The paper has no
 * counterpart: this is the deposit of recon_deposit(RECON_PARTICLES) for
 * callers that cannot call cudaMalloc where they need it -- e.g. code whose
 * device memory is owned by another allocator that must account for every
 * byte, or a loop where an allocation would synchronise the device.
 *   n0, n1, n2  grid dims, powers of two; n0*n1*n2 <= 2^21 (128^3) cells
 *   cell        cell side in the units of pos (positions wrap periodically)
 *   pos         device array of np x 3 doubles; mass: device array of np
 *               doubles, or NULL for unit masses
 *   rho         device array of n0*n1*n2 doubles, receives the mass per cell
 *   cuda_stream stream for the work (cudaStream_t, NULL = legacy stream)
 * pos, mass and rho must be memory of the current device (or managed).  The
 * accumulators live in one fixed 16 MiB device array of the library (resident
 * on every GPU that loads the library, until exit).  The first call on a
 * device looks up that array's device address; after a cudaDeviceReset of the
 * device the call must not be used there again in the same process.  Every
 * call reuses the same array, so calls that overlap on the GPU (other streams
 * or threads) race.  The call synchronises its stream once to check the
 * inputs on the host, so it cannot be used while the stream is being captured
 * into a CUDA graph.  Larger grids, host or other-device pointers, NaN/Inf or
 * negative inputs and zero total mass are rejected with a status
 * (RECON_E_INVALID / RECON_E_NONFINITE); nothing is allocated or freed. */
int recon_deposit_cic_noalloc(int n0, int n1, int n2, double cell, const double* pos,
                              const double* mass, int64_t np, double* rho, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
