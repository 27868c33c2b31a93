// recon_internal.cuh -- shared declarations of the CUDA kernels' launch
// wrappers and the grid helpers (internal to librecon.so).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <set>
#include <utility>

namespace recon {

// Kernels launched by this library (for the launch count a solve reports).
inline std::atomic<long long>& launch_counter() {
    static std::atomic<long long> c{0};
    return c;
}

// Allows kernel fn up to `bytes` of dynamic shared memory on the current
// device; the attribute is set once per kernel and device.
inline void allow_smem(const void* fn, int bytes) {
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    if (done.insert(std::make_pair(fn, dev)).second)
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Periodic power-of-two grid: n0 x n1 x n2 nodes, last axis fastest.
struct Dims {
    int n0, n1, n2;
    int s1, s2;      // log2(n1), log2(n2)
    int cells;       // n0 * n1 * n2 (<= 2^30)
};

inline Dims make_dims(int n0, int n1, int n2) {
    Dims d;
    d.n0 = n0, d.n1 = n1, d.n2 = n2;
    d.s1 = 0;
    while ((1 << d.s1) < n1) ++d.s1;
    d.s2 = 0;
    while ((1 << d.s2) < n2) ++d.s2;
    d.cells = n0 * n1 * n2;
    return d;
}

__host__ __device__ inline int cell_index(const Dims& d, int i, int j, int k) {
    return ((((i & (d.n0 - 1)) << d.s1) | (j & (d.n1 - 1))) << d.s2) | (k & (d.n2 - 1));
}

__host__ __device__ inline void cell_coords(const Dims& d, int c, int& i, int& j, int& k) {
    k = c & (d.n2 - 1);
    j = (c >> d.s2) & (d.n1 - 1);
    i = c >> (d.s1 + d.s2);
}

// Number of blocks of the fixed-size reduction launches (2 x 608 = 8 per SM
// on a 152-SM part) and their block size.  Reductions write one partial per
// block and are finished by a single block in a fixed order, so every sum is
// deterministic.
constexpr int kRedBlocks = 1216;
constexpr int kRedThreads = 256;

// Scalars produced on the device and read back by the host.
enum Scalar {
    SC_SUM_RHO = 0,   // sum of the deposited density
    SC_BAD,           // nonzero if an input was NaN/Inf/negative (as double)
    SC_SUM_T,         // sum of t = Sigma + C + E
    SC_MIN_DET,       // min det(I + Hess phi)
    SC_SUM_S2,        // sum of s^2
    SC_SUM_M,         // sum of m
    SC_RES2,          // sum of residual^2
    SC_SUM_DPHI,      // sum of S(phidot)
    SC_MAX_K,         // max over nodes of the per-node limiter exponent
    SC_MAX_G,         // max |grad dphi|
    SC_MIN_LAM,       // min lambda0
    SC_MAX_DR,        // max delta_r
    SC_ALPHA,         // step length of the current step
    SC_ADJ_A,         // adjoint sweep: sums used for mean projections
    SC_ADJ_B,
    SC_COUNT
};

// Operator of one multigrid level: 1/h_a^2 per axis.
struct Level {
    Dims d;
    double h2i[3];
    int coarsen[3];  // axis halved on the way to the next level
    // planes per block measured fastest at create (tune_streaming_level) for
    // the plain sweep, the sweep with the prolongation folded in and the
    // residual restriction; 0: the occupancy cost model decides
    int tune[3];
    // 0: the operator's coefficient is nodal (a, faces (a_c + a_n) / 2);
    // 1: it is given per face, as one array of 3 x cells face sums
    // G = 2 x the face coefficient (x faces, then y, then z; entry c is the
    // face between node c and its +1 neighbour), built from the level above
    // by launch_faces_line
    int face;
    // 1: the streaming sweep stages the planes of tiles clear of the periodic
    // seams with bulk tensor copies (same values as the per-thread copies)
    int tma;
};

// Mean device time (ms) of `reps` launches issued by launch() on st, after
// one untimed launch.
template <typename F>
float time_launches(cudaStream_t st, int reps, F&& launch) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch();
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms / reps;
}

struct SourceParams {
    double xi_m, v_m;
    int climiter;
};

struct LimiterParams {
    double lambda_floor;
    int kmax;  // largest exponent k with 2^-k >= alpha_min
};

// The coarse levels handled by one block in shared memory (launch_coarse_vcycle).
constexpr int kCoarseMaxLevels = 8;
constexpr size_t kCoarseMaxSmem = 200 * 1024;
struct CoarseSet {
    int nlev;                              // levels l0 .. last (last is 4^3)
    int nu1, nu2;
    Level lv[kCoarseMaxLevels];
    const void* a[kCoarseMaxLevels];       // coefficient of each level (T*)
};

// The coarse end from a 32^3 level (32^3, 16^3, 8^3, 4^3, every axis halved)
// in one launch of one thread-block cluster (coarse_cluster.cu); false with
// nothing launched when cs is not that set.
bool coarse_cluster_fits(const CoarseSet& cs);
template <typename T>
bool launch_coarse_cluster(const CoarseSet& cs, const T* f, T* u, const double* minv, bool zero_u,
                           cudaStream_t st);

// ---- reductions -----------------------------------------------------------
// op: 0 = sum, 1 = min, 2 = max.  Finishes kRedBlocks partials into slot.
void finish_reduce(const double* partials, int op, double* scalars, int slot, cudaStream_t st);

// ---- multigrid (T = float or double) --------------------------------------
template <typename T>
void launch_rbgs_sweep(const Level& L, T* u, const T* f, const T* a, cudaStream_t st);
// Up to nsweeps full red-black sweeps u_new <- RBGS^k(u_old) in a single
// streaming pass (smoother.cu); u_old == nullptr means u_old = 0.  Returns k,
// the sweeps done; 0 (nothing launched) when the level is not a multiple of
// the kernel's tile or the precision does not use the streaming kernel.
// Residual and full-weighting restriction of an FP32 level in one streaming
// pass; returns 1, or 0 with nothing launched where the level does not fit
// its tiles (then launch_resid_restrict does the work).
// Tuning of an FP32 level at create: every planes-per-block choice of the
// streaming sweep (plain and, with a coarse level, with the prolongation) and
// of the streaming residual restriction is timed on the level's own buffers
// (their contents do not matter: every choice computes the same values) and
// the fastest is stored in L.tune.  No-op where the kernels do not apply.
void tune_sweep_level(Level& L, const Level* coarse, const float* uc, float* u, float* w,
                      const float* f, const float* a, cudaStream_t st);
void tune_resid_restrict_level(Level& fine, const Level& coarse, const float* u, const float* f,
                               const float* a, float* out, cudaStream_t st);
int launch_resid_restrict_stream(const Level& fine, const Level& coarse, const float* u,
                                 const float* f, const float* a, float* out, cudaStream_t st);

// The first post-smoothing sweep of an FP32 level with the V-cycle's
// coarse-grid correction folded in (u_new <- RBGS(u_old + P(uc))) where the
// level fits the streaming sweep and every axis is halved; with u64 also
// u64 += u_new (the defect correction, when this is the level's only
// post-smoothing sweep).  Returns 1, or 0 with nothing launched (then
// prolongate and sweep separately).
bool rbgs_prolong_fits(const Level& fine);
// Whether a streaming sweep gave up waiting for a bulk copy since the last
// call (on the current device); clears the record.
bool sweep_wait_failed();
// RECON_CHECKED build: the id of the first failed index check of each
// instrumented translation unit since the last call (read and cleared;
// always 0 in the normal build).
int bounds_fail_smoother();
int bounds_fail_transfer();
int bounds_fail_cluster();
int bounds_fail_steps();
int launch_rbgs_prolong(const Level& fine, const Level& coarse, const float* uc, const float* u_old,
                        float* u_new, const float* f, const float* a, cudaStream_t st,
                        double* u64 = nullptr);

// A streaming FP32 sweep that also adds its result to an FP64 field
// (u_new <- RBGS(u_old), u64 += u_new); returns 1, or 0 with nothing launched.
int launch_rbgs_correct(const Level& L, const float* u_old, float* u_new, const float* f,
                        const float* a, double* u64, cudaStream_t st);

template <typename T>
int launch_rbgs_fused(const Level& L, const T* u_old, T* u_new, const T* f, const T* a,
                      int nsweeps, cudaStream_t st);
template <>
int launch_rbgs_fused<float>(const Level&, const float*, float*, const float*, const float*,
                             int, cudaStream_t);
template <>
int launch_rbgs_fused<double>(const Level&, const double*, double*, const double*,
                              const double*, int, cudaStream_t);
template <typename T>
void launch_restrict(const Level& fine, const Level& coarse, const T* in, T* out, cudaStream_t st);
// Face sums of a coarse level (every axis halved) from the level above
// (nodal coefficient, or its face sums when fine.face): along each axis the
// two fine faces a coarse face spans act in series (harmonic mean), and the
// fine lines under it are averaged with the full-weighting weights across.
void launch_faces_line(const Level& fine, const Level& coarse, const float* in, float* out,
                       cudaStream_t st);
// y = (float) x, elementwise
void launch_to_f32(int cells, const double* x, float* y, cudaStream_t st);
// full-weighting restriction of the residual f - L u, without storing it
template <typename T>
void launch_resid_restrict(const Level& fine, const Level& coarse, const T* u, const T* f,
                           const T* a, T* out, cudaStream_t st);
template <typename T>
void launch_prolong_add(const Level& fine, const Level& coarse, const T* uc, T* u, cudaStream_t st);
// Coarsest (4x4x4) level: invert the bordered 65 x 65 system [L 1; 1^T 0]
// once per coefficient (FP64), then solve by one matrix-vector product.
template <typename T>
void launch_coarse_invert(const Level& L, const T* a, double* minv, cudaStream_t st);
template <typename T>
void launch_coarse_solve(const double* minv, const T* f, T* u, cudaStream_t st);
// V-cycle of the levels in cs in one block: L u = f on the first of them,
// u updated in place (zero_u: u = 0 on entry, not read); returns false,
// launching nothing, if they do not fit.
template <typename T>
bool launch_coarse_vcycle(const CoarseSet& cs, const T* f_top, T* u_top, const double* minv,
                          bool zero_u, cudaStream_t st);
// Finest FP64 level (unit spacing): face coefficients F (3 x cells:
// A = (a_c + a_{c+e}) / 2 for the +x, +y, +z face of each node), the node
// diagonal D = sum of its six A, and optionally inv_d = 1 / D.
void launch_faces64(const Level& L, const double* a, double* F, double* D, double* inv_d,
                    cudaStream_t st);
// FP64 residual of level 0 in mixed mode: r32 = f - L u (FP64), plus sum r^2
void launch_residual64_to32(const Level& L, const double* u, const double* f, const double* F,
                            const double* D, float* r32, double* partials, cudaStream_t st);
// FP64 residual norm only: partials of (f - L u)^2
void launch_residual_norm64(const Level& L, const double* u, const double* f, const double* F,
                            const double* D, double* partials, cudaStream_t st);
// FP64 red-black sweep of the finest level: u_c = (sum_n A_n u_n - f_c) / D_c
void launch_rbgs_sweep64_unit(const Level& L, double* u, const double* f, const double* F,
                              const double* inv_d, cudaStream_t st);
// u64 += e32
void launch_correct(int cells, double* u, const float* e, cudaStream_t st);

// ---- steps of the outer iteration -----------------------------------------
void launch_validate_grid(int cells, const double* rho, double* partials_sum, double* partials_bad,
                          cudaStream_t st);
void launch_validate_particles(int64_t np, const double* pos, const double* mass,
                               double* partials_sum, double* partials_bad, cudaStream_t st);
void launch_deposit_particles(const Dims& d, int64_t np, const double* pos, const double* mass,
                              double inv_h, double scale, unsigned long long* mfix, cudaStream_t st);
void launch_fix_to_double(int cells, unsigned long long* mfix, double inv_scale, double* out,
                          cudaStream_t st);
void launch_init_tracers(int cells, const double* rho, const double* sum_rho, double* w,
                         double* ox, double* oy, double* oz, double* phi, float* phi32,
                         cudaStream_t st);
void launch_deposit_tracers(const Dims& d, const double* ox, const double* oy, const double* oz,
                            const double* w, double scale, unsigned long long* mfix,
                            cudaStream_t st);
void launch_mass_coef(int cells, unsigned long long* mfix, double inv_scale, double a_min,
                      double* m, double* a64, float* a32, double* partials, cudaStream_t st);
// e6 (6 x cells): the triad e = I + Hess phi (xx, yy, zz, xy, xz, yz) of the
// step, written by the geometry pass and read by the limiter and the advance.
void launch_geometry_source(const Dims& d, const SourceParams& sp, const double* phi,
                            const double* m, double* t, double* e6, double* part_sum,
                            double* part_min, cudaStream_t st);
// S in three axis passes through tmp2 (2 x cells scratch); out32 (optional)
// receives an FP32 copy of the result.
void launch_smooth_S(const Dims& d, double s_side, const double* in, const double* shift_scalar,
                     double* out, float* out32, double* tmp2, double* part_sum, double* part_sq,
                     cudaStream_t st);
// phi32, dphi32: FP32 copies of phi and dphi used to screen nodes that clear
// the limiter's floor by a wide margin.
void launch_limiter(const Dims& d, const LimiterParams& lp, const double* e6, const double* dphi,
                    const float* phi32, const float* dphi32, double* part_k, double* part_g,
                    cudaStream_t st);
void launch_node_velocity(const Dims& d, const double* e6, const double* dphi, double* vx,
                          double* vy, double* vz, cudaStream_t st);
// The step's node displacements alpha V in fixed point (2^-51 cells), for
// launch_advance.
void launch_node_displacement(const Dims& d, const double* e6, const double* dphi, const double* alpha,
                              long long* dx, long long* dy, long long* dz, cudaStream_t st);
// Tracers move by -alpha V(xi) (the fixed-point displacements CIC-interpolated
// in integer arithmetic); phi += alpha (dphi - mean), mean = *sum_dphi / cells.
void launch_advance(const Dims& d, const long long* dx, const long long* dy, const long long* dz,
                    const double* alpha, const double* dphi, const double* sum_dphi, double* ox,
                    double* oy, double* oz, double* phi, float* phi32, cudaStream_t st);
// App. A's linear density update: m += alpha d_mu(m (e^-1)^{mu nu} d_nu dphi)
// (K6: 6 x cells scratch), the coefficient from a carried m, and phi's update
// without tracers.
void launch_mass_literal(const Dims& d, const double* e6, const double* dphi,
                         const double* alpha, double* m, double* K6, cudaStream_t st);
void launch_coef_from_m(int cells, const double* m, double a_min, double* a64, float* a32,
                        double* partials, cudaStream_t st);
void launch_phi_advance(int cells, const double* alpha, const double* dphi,
                        const double* sum_dphi, double* phi, float* phi32, cudaStream_t st);
// outputs
void launch_delta_r(const Dims& d, const double* phi, double* out, double* part_max,
                    cudaStream_t st);
void launch_mesh_x(const Dims& d, const double* phi, double h, double* out, cudaStream_t st);
void launch_geometry_out(const Dims& d, const double* phi, double* det, double* lam,
                         double* part_min_det, double* part_min_lam, cudaStream_t st);
void launch_scale(int cells, const double* in, double s, double* out, cudaStream_t st);

// ---- device-side control of the iteration (control.cu) -----------------
// The control block of one solve: every decision of the iteration is taken by
// a one-thread kernel and recorded here (the host-driven loop reads it back;
// inside the solve graph the same kernels also set the conditional nodes).
struct Ctl {
    int k;              // steps advanced so far
    int status;         // RECON_OK / RECON_NOT_CONVERGED / RECON_STALLED
    int vtot, ncyc;     // V-cycles in total and in the current step's solve
    int final_deposit;  // the last map still needs its deposit
    int n_step, n_cont, n_mg, n_adv, n_fin;  // executions of each graph body
    int go_cont, go_mg, go_adv, go_step, go_fin;
    // grouped FP64 checks (params.group_max): V-cycles in the current defect
    // correction, the count at which it forms its FP64 residual, whether the
    // next block starts a new correction, whether this block ends one, and
    // executions of the check body
    int gcyc, gtarget, fresh, chk, n_chk;
    int pad;
    double R0, R, s2, rel, alpha, last_mass;
    double rel0;        // relative residual when the current correction began
};

// Per-step records on the device (k_max entries each).
struct CtlArrays {
    double* Rk;
    double* alpha;
    double* relres;
    int* ncycles;
};

// Conditional nodes of the solve graph; active = 0 outside a graph.
struct CtlHandles {
    int active;
    cudaGraphConditionalHandle step, cont, mg, adv, fin, chk;
};

void launch_ctl_init(Ctl* c, cudaStream_t st);
void launch_ctl_step_begin(Ctl* c, const double* scal, const CtlArrays& a, double ncells,
                           double tol_out, const CtlHandles& h, cudaStream_t st);
void launch_ctl_mg_begin(Ctl* c, const CtlArrays& a, int mixed, double tol_in,
                         int max_vcycles, const CtlHandles& h, cudaStream_t st);
// Grouped FP64 checks: after a block of `block` FP32 V-cycles, whether the
// defect correction ends here (its FP64 residual is formed next); and after
// that residual, the stopping test and the length of the next correction.
void launch_ctl_block(Ctl* c, const CtlArrays& a, int block, int max_vcycles, const CtlHandles& h,
                      cudaStream_t st);
void launch_ctl_group_check(Ctl* c, const double* scal, const CtlArrays& a, int block, int group_max,
                            double tol_in, int max_vcycles, const CtlHandles& h, cudaStream_t st);
// u = 0 where the control block says a new defect correction starts
void launch_zero_if_fresh(const Ctl* c, float* u, int cells, cudaStream_t st);
// The extrapolated initial guess of the step's linear solve (warm_start = 2):
// u += (alpha_{k-1} / alpha_{k-2}) (u - prev) for k >= 2, prev = old u for k >= 1.
void launch_warm_extrapolate(const Ctl* c, const double* alpha, double* u, double* prev, int cells,
                             cudaStream_t st);
void launch_ctl_mg_check(Ctl* c, const double* scal, const CtlArrays& a, int per_launch,
                         double tol_in, int max_vcycles, const CtlHandles& h, cudaStream_t st);
void launch_ctl_select_alpha(Ctl* c, double* scal, const CtlArrays& a, const double* replay,
                             int kmax_exp, double d_max, double alpha_min, const CtlHandles& h,
                             cudaStream_t st);
void launch_ctl_step_end(Ctl* c, int k_max, const CtlHandles& h, cudaStream_t st);
void launch_ctl_final(Ctl* c, int want, const CtlHandles& h, cudaStream_t st);
void launch_ctl_final_mass(Ctl* c, const double* scal, cudaStream_t st);

// ---- per-step checkpoints and the adjoint sweep (adjoint.cu) --------------
// Slot k (= ctl->k) of base holds phi_k, the tracer offsets ox, oy, oz and
// phidot_k of step k, 5 x cells doubles.
void launch_ckpt_state(const Ctl* ctl, int cells, const double* phi, const double* ox,
                       const double* oy, const double* oz, double* base, cudaStream_t st);
void launch_ckpt_phidot(const Ctl* ctl, int cells, const double* phidot, double* base,
                        cudaStream_t st);
void launch_adj_lap(const Dims& d, const double* gbar, double* phibar, cudaStream_t st);
void launch_adj_tracers(const Dims& d, const double* ox, const double* oy, const double* oz,
                        const double* v3, const double* alpha, double* xb3, double* vb3,
                        cudaStream_t st);
void launch_adj_velocity(const Dims& d, const double* e6, const double* v3, const double* vb3,
                         double* gb3, double* eb6, cudaStream_t st);
void launch_adj_dbar(const Dims& d, const double* alpha, const double* phibar, const double* gb3,
                     double* dbar, double* psum, cudaStream_t st);
void launch_adj_coef(const Dims& d, const double* lam, const double* pd, const double* m,
                     double a_min, double* mbar, double* psum, cudaStream_t st);
void launch_adj_source(const Dims& d, const SourceParams& sp, const double* e6, const double* m,
                       const double* tbar, double* mbar, double* eb6, cudaStream_t st);
void launch_adj_hess(const Dims& d, const double* eb6, double* phibar, cudaStream_t st);
void launch_adj_deposit(const Dims& d, const double* ox, const double* oy, const double* oz,
                        const double* w, const double* mbar, double* wbar, double* xb3,
                        cudaStream_t st);
void launch_adj_dot(int cells, const double* a, const double* b, double* psum, cudaStream_t st);
void launch_adj_final(int cells, const double* wbar, const double* sum_wbw, const double* sum_rho,
                      double* grad, cudaStream_t st);

}  // namespace recon
