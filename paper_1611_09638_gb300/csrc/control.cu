// control.cu -- the decisions of the moving-mesh iteration (Sec. II, App. A)
// taken on the device: the stopping test on R_k = rms(s) at each step start,
// the stopping test of the multigrid solve on ||s - L phidot|| / ||s||, and
// the choice of the step length alpha by the limiter's halving rule (or its
// replay).  One thread of one block runs each of them; every decision is
// written to the control block (read back by the host-driven loop) and, when
// the kernel runs inside the solve graph, also to the graph's conditional
// nodes, so that the whole iteration runs without a host round trip.
#include "../../include/recon.h"
#include "recon_internal.cuh"

namespace recon {

namespace {

__device__ inline void set_cond(const CtlHandles& h, cudaGraphConditionalHandle c, int v) {
    if (h.active) cudaGraphSetConditional(c, v ? 1u : 0u);
}

__global__ void k_ctl_init(Ctl* c) {
    c->k = 0, c->status = RECON_NOT_CONVERGED, c->vtot = 0, c->ncyc = 0;
    c->final_deposit = 1;
    c->n_step = c->n_cont = c->n_mg = c->n_adv = c->n_fin = 0;
    c->go_cont = c->go_mg = c->go_adv = c->go_step = 0;
    c->gcyc = c->gtarget = c->chk = c->n_chk = 0;
    c->fresh = 1;
    c->R0 = c->R = c->s2 = c->rel = c->alpha = c->last_mass = 0.0;
    c->rel0 = 1.0;
}

// Step start: R_k from the sum of s^2; stop when R_k <= tol_out.
__global__ void k_ctl_step_begin(Ctl* c, const double* scal, CtlArrays a, double ncells,
                                 double tol_out, CtlHandles h) {
    const int k = c->k;
    const double s2 = scal[SC_SUM_S2];
    const double R = sqrt(s2 / ncells);
    c->s2 = s2, c->R = R;
    if (k == 0) c->R0 = R;
    c->last_mass = scal[SC_SUM_M];
    a.Rk[k] = R;
    c->n_step += 1;
    const int go = !(R <= tol_out);
    if (!go) c->status = RECON_OK, c->final_deposit = 0;
    c->go_cont = go;
    set_cond(h, h.cont, go);
    if (!go) {
        c->go_step = 0;
        set_cond(h, h.step, 0);
    }
}

// Multigrid start: phidot = 0, so the defect is s and its relative size 1.
__global__ void k_ctl_mg_begin(Ctl* c, CtlArrays a, int mixed, double tol_in,
                               int max_vcycles, CtlHandles h) {
    const int k = c->k;
    c->n_cont += 1;
    c->ncyc = 0;
    const double rel = 1.0;
    c->rel = rel;
    c->gcyc = 0, c->fresh = 1, c->rel0 = rel;
    c->gtarget = 0;  // the first correction forms its residual after one block
    a.ncycles[k] = 0, a.relres[k] = rel;
    const int go = c->s2 > 0.0 && max_vcycles > 0 && !(mixed && rel <= tol_in);
    c->go_mg = go;
    set_cond(h, h.mg, go);
}

// After one multigrid iteration (per_launch V-cycles and the FP64 residual).
__global__ void k_ctl_mg_check(Ctl* c, const double* scal, CtlArrays a, int per_launch,
                               double tol_in, int max_vcycles, CtlHandles h) {
    const int k = c->k;
    c->n_mg += 1;
    c->ncyc += per_launch;
    c->vtot += per_launch;
    const double rel = sqrt(scal[SC_RES2] / c->s2);
    c->rel = rel;
    a.ncycles[k] = c->ncyc, a.relres[k] = rel;
    const int go = !(rel <= tol_in) && c->ncyc < max_vcycles;
    c->go_mg = go;
    set_cond(h, h.mg, go);
}

// After a block of FP32 V-cycles: the correction forms its FP64 residual when
// it has run the cycles the last check asked for (or the step's cap is near).
__global__ void k_ctl_block(Ctl* c, CtlArrays a, int block, int max_vcycles, CtlHandles h) {
    const int k = c->k;
    c->n_mg += 1;
    c->gcyc += block;
    c->ncyc += block;
    c->vtot += block;
    a.ncycles[k] = c->ncyc;
    const int chk = c->gcyc >= c->gtarget || c->ncyc >= max_vcycles;
    c->chk = chk;
    c->fresh = 0;
    set_cond(h, h.chk, chk);
    if (!chk) {
        c->go_mg = 1;
        set_cond(h, h.mg, 1);
    }
}

// After the FP64 residual that ends a defect correction: the stopping test,
// then the length of the next correction, from the contraction per V-cycle
// this one achieved, rho = (rel / rel0)^(1 / cycles): the cycles that take
// rel below tol_in, in whole blocks, between one block and group_max.
__global__ void k_ctl_group_check(Ctl* c, const double* scal, CtlArrays a, int block, int group_max,
                                  double tol_in, int max_vcycles, CtlHandles h) {
    const int k = c->k;
    c->n_chk += 1;
    const double rel = sqrt(scal[SC_RES2] / c->s2);
    c->rel = rel;
    a.relres[k] = rel;
    const int go = !(rel <= tol_in) && c->ncyc < max_vcycles;
    int need = block;
    if (go && c->gcyc > 0 && rel > 0.0 && rel < c->rel0) {
        const double rho = pow(rel / c->rel0, 1.0 / (double)c->gcyc);
        if (rho > 0.0 && rho < 1.0) {
            const double cyc = log(tol_in / rel) / log(rho);
            need = cyc < (double)group_max ? (int)ceil(cyc) : group_max;
            need = ((need + block - 1) / block) * block;
            if (need > group_max) need = (group_max / block) * block;
            if (need < block) need = block;
        }
    }
    c->gtarget = need;
    c->gcyc = 0;
    c->fresh = 1;
    c->rel0 = rel;
    c->go_mg = go;
    set_cond(h, h.mg, go);
}

__global__ void k_zero_if_fresh(const Ctl* __restrict__ c, float* __restrict__ u, int cells) {
    if (!c->fresh) return;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cells; e += gridDim.x * blockDim.x) u[e] = 0.f;
}

// Initial guess of step k's linear solve from the last two solutions (u holds
// phidot_{k-1}, prev phidot_{k-2}): u += r (u - prev) with r = alpha_{k-1} /
// alpha_{k-2}, the step lengths that moved the mesh between them; prev takes
// phidot_{k-1}.  At k = 1 prev only takes phidot_0; at k = 0 nothing happens.
__global__ void k_warm_extrapolate(const Ctl* __restrict__ c, const double* __restrict__ alpha,
                                   double* __restrict__ u, double* __restrict__ prev, int cells) {
    const int k = c->k;
    if (k < 1) return;
    const double r = k >= 2 ? alpha[k - 1] / alpha[k - 2] : 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cells; e += gridDim.x * blockDim.x) {
        const double cur = u[e];
        if (k >= 2) u[e] = cur + r * (cur - prev[e]);
        prev[e] = cur;
    }
}

// Step length: the largest 2^-j the limiter certified, halved further while
// max |alpha grad dphi| > d_max; below alpha_min the iteration stops with the
// current map (RECON_STALLED).  With a replay array alpha_k is taken from it.
__global__ void k_ctl_select_alpha(Ctl* c, double* scal, CtlArrays a, const double* replay,
                                   int kmax_exp, double d_max, double alpha_min, CtlHandles h) {
    const int k = c->k;
    double alpha;
    if (replay) {
        alpha = replay[k];
    } else {
        const int kpd = (int)scal[SC_MAX_K];
        const double gmax = scal[SC_MAX_G];
        alpha = kpd > kmax_exp ? 0.0 : ldexp(1.0, -kpd);
        while (alpha * gmax > d_max && alpha >= alpha_min) alpha *= 0.5;
        if (alpha < alpha_min) {
            c->status = RECON_STALLED;
            c->go_adv = 0, c->go_step = 0;
            set_cond(h, h.adv, 0);
            set_cond(h, h.step, 0);
            return;
        }
    }
    c->alpha = alpha;
    scal[SC_ALPHA] = alpha;
    a.alpha[k] = alpha;
    c->go_adv = 1;
    set_cond(h, h.adv, 1);
}

// After the advance: next step, or stop at k_max.
__global__ void k_ctl_step_end(Ctl* c, int k_max, CtlHandles h) {
    c->n_adv += 1;
    c->k += 1;
    const int go = c->k < k_max;
    c->go_step = go;
    set_cond(h, h.step, go);
}

// After the step loop: the last map's tracers are deposited once more for
// the mass statistics unless the loop stopped on R_k (then m is current).
__global__ void k_ctl_final(Ctl* c, int want, CtlHandles h) {
    const int go = want && c->final_deposit;
    c->go_fin = go;
    set_cond(h, h.fin, go);
}

__global__ void k_ctl_final_mass(Ctl* c, const double* scal) {
    c->n_fin += 1;
    c->last_mass = scal[SC_SUM_M];
}

}  // namespace

void launch_ctl_init(Ctl* c, cudaStream_t st) {
    launch_counter()++;
    k_ctl_init<<<1, 1, 0, st>>>(c);
}
void launch_ctl_step_begin(Ctl* c, const double* scal, const CtlArrays& a, double ncells,
                           double tol_out, const CtlHandles& h, cudaStream_t st) {
    launch_counter()++;
    k_ctl_step_begin<<<1, 1, 0, st>>>(c, scal, a, ncells, tol_out, h);
}
void launch_ctl_mg_begin(Ctl* c, const CtlArrays& a, int mixed, double tol_in,
                         int max_vcycles, const CtlHandles& h, cudaStream_t st) {
    launch_counter()++;
    k_ctl_mg_begin<<<1, 1, 0, st>>>(c, a, mixed, tol_in, max_vcycles, h);
}
void launch_ctl_mg_check(Ctl* c, const double* scal, const CtlArrays& a, int per_launch,
                         double tol_in, int max_vcycles, const CtlHandles& h, cudaStream_t st) {
    launch_counter()++;
    k_ctl_mg_check<<<1, 1, 0, st>>>(c, scal, a, per_launch, tol_in, max_vcycles, h);
}
void launch_ctl_block(Ctl* c, const CtlArrays& a, int block, int max_vcycles, const CtlHandles& h,
                      cudaStream_t st) {
    launch_counter()++;
    k_ctl_block<<<1, 1, 0, st>>>(c, a, block, max_vcycles, h);
}

void launch_ctl_group_check(Ctl* c, const double* scal, const CtlArrays& a, int block, int group_max,
                            double tol_in, int max_vcycles, const CtlHandles& h, cudaStream_t st) {
    launch_counter()++;
    k_ctl_group_check<<<1, 1, 0, st>>>(c, scal, a, block, group_max, tol_in, max_vcycles, h);
}

void launch_warm_extrapolate(const Ctl* c, const double* alpha, double* u, double* prev, int cells,
                             cudaStream_t st) {
    launch_counter()++;
    k_warm_extrapolate<<<kRedBlocks, kRedThreads, 0, st>>>(c, alpha, u, prev, cells);
}

void launch_zero_if_fresh(const Ctl* c, float* u, int cells, cudaStream_t st) {
    launch_counter()++;
    k_zero_if_fresh<<<kRedBlocks, kRedThreads, 0, st>>>(c, u, cells);
}

void launch_ctl_select_alpha(Ctl* c, double* scal, const CtlArrays& a, const double* replay,
                             int kmax_exp, double d_max, double alpha_min, const CtlHandles& h,
                             cudaStream_t st) {
    launch_counter()++;
    k_ctl_select_alpha<<<1, 1, 0, st>>>(c, scal, a, replay, kmax_exp, d_max, alpha_min, h);
}
void launch_ctl_step_end(Ctl* c, int k_max, const CtlHandles& h, cudaStream_t st) {
    launch_counter()++;
    k_ctl_step_end<<<1, 1, 0, st>>>(c, k_max, h);
}
void launch_ctl_final(Ctl* c, int want, const CtlHandles& h, cudaStream_t st) {
    launch_counter()++;
    k_ctl_final<<<1, 1, 0, st>>>(c, want, h);
}
void launch_ctl_final_mass(Ctl* c, const double* scal, cudaStream_t st) {
    launch_counter()++;
    k_ctl_final_mass<<<1, 1, 0, st>>>(c, scal);
}

}  // namespace recon
