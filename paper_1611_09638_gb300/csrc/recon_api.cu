// recon_api.cu -- the C ABI (include/recon.h) and the host orchestration of
// the moving-mesh solve (Sec. II, App. A of Zhu et al. 2016): per step the
// deposit on the deformed mesh, the limited smoothed source, the multigrid
// solve of the linearised equation (FP64, or FP32 V-cycles inside an FP64
// defect correction), the smoothed increment, the step limiter and the advance.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/recon.h"
#include "recon_internal.cuh"

using namespace recon;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(RECON_E_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                                  \
    } while (0)

// Kernels recorded in each body of the solve graph.
// NVTX range for profiler timelines (no cost without a tool attached).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

struct GraphCounts {
    long long init = 0, step = 0, cont = 0, mg = 0, adv = 0, fin = 0, chk = 0;
};

struct Handle {
    recon_params p{};
    std::vector<double> replay;
    cudaStream_t st = nullptr;
    int device = 0;
    Dims d{};
    int cells = 0;
    double h = 1.0;
    std::vector<Level> lv;
    bool mixed = false;

    // FP64 state (device)
    double *rho = nullptr, *w = nullptr, *ox = nullptr, *oy = nullptr, *oz = nullptr;
    double *phi = nullptr, *m = nullptr, *a64 = nullptr, *t = nullptr, *s = nullptr;
    double *phidot = nullptr, *dphi = nullptr, *v3 = nullptr;  // v3: 3 x cells
    double* phidot_prev = nullptr;  // warm_start = 2: phidot of the step before the last
    // staging of host particle inputs (grown to the largest, kept until destroy)
    void* stage = nullptr;
    size_t stage_bytes = 0;
    double* e6 = nullptr;  // triad I + Hess phi of the current step, 6 x cells
    double* inv64 = nullptr;  // FP64 mode: 1 / diagonal of the finest level
    double* F64 = nullptr;    // face coefficients (a_c + a_{c+e}) / 2 of the finest level, 3 x cells
    double* D64 = nullptr;    // node diagonal: sum of the node's six face coefficients
    float *phi32 = nullptr, *dphi32 = nullptr;  // FP32 copies for the limiter's screen
    double* v3m = nullptr;  // density_update = 1: K = m e^-1 (6 x cells)
    unsigned long long* mfix = nullptr;
    // multigrid per level: FP64 (FP64 mode) or FP32 (mixed mode)
    std::vector<double*> u64, f64, c64, r64;
    std::vector<float*> u32, f32, c32, r32;
    double* minv = nullptr;
    int l0 = -1;        // first level of the single-block coarse V-cycle
    CoarseSet cs{};     // those levels and their coefficients
    int lc = -1;        // the 32^3 level whose V-cycle runs as one cluster launch
    CoarseSet cc{};     // the levels from it down
    double* part[4] = {nullptr, nullptr, nullptr, nullptr};
    double* scal = nullptr;   // device scalars
    double* hscal = nullptr;  // pinned host copy
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<void*> allocs;
    // params.profile: event pairs around the finest-level smoothing sweeps
    std::vector<cudaEvent_t> prof_ev;
    size_t prof_used = 0;
    int prof_sweeps = 0;
    double prof_ms = 0.0;  // sweep time accumulated over graph launches

    // One multigrid iteration (V-cycle, residual, norm readback) recorded once
    // as a CUDA graph on a private stream and replayed on the handle's stream.
    cudaStream_t cap = nullptr;
    bool capturing = false;
    cudaGraphExec_t cyc_exec = nullptr;
    cudaGraphExec_t chk_exec = nullptr;  // grouped checks: the check body, host-driven loop
    long long chk_kernels = 0;
    bool adaptive = false;     // mixed precision with group_max > inner_vcycles
    bool inner_tuned = false;  // params.tune_inner: the first solve has chosen inner_vcycles
    long long cyc_kernels = 0;
    int cyc_sweeps = 0;
    std::vector<cudaEvent_t> cyc_ev;
    size_t cyc_ev_used = 0;

    // control of the iteration (control.cu): device block, pinned copy, and
    // the per-step records (Rk, alpha, relres, ncycles; harr: pinned copy)
    Ctl* ctl = nullptr;
    Ctl* hctl = nullptr;
    CtlArrays arr{};
    double* harr = nullptr;
    double* replay_d = nullptr;  // replay_alpha on the device (or null)
    LimiterParams lp{};

    // params.checkpoint: phi_k, tracer offsets and phidot_k of every step
    // (5 x cells doubles per step) and the adjoint sweep's buffers
    double* ckpt = nullptr;
    struct {
        double *phibar = nullptr, *xib = nullptr, *wbar = nullptr, *vb = nullptr, *gb = nullptr;
        double *eb = nullptr, *dbar = nullptr, *mbar = nullptr;
    } adj;
    Ctl* actl = nullptr;   // control block of the adjoint's linear solves
    CtlArrays aarr{};

    // params.device_loop: the whole solve as one graph with conditional nodes
    cudaStream_t gst[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // capture streams
    cudaGraphExec_t solve_exec = nullptr;
    GraphCounts gn{};

    bool have_density = false, solved = false;
    double rho_sum = 0.0;
};

template <typename T>
int dalloc(Handle* H, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(RECON_E_OOM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                    cudaGetErrorString(e));
    }
    H->allocs.push_back(q);
    *p = (T*)q;
    return RECON_OK;
}

void free_all(Handle* H) {
    for (void* q : H->allocs) cudaFree(q);
    H->allocs.clear();
    if (H->stage) cudaFree(H->stage);
    H->stage = nullptr, H->stage_bytes = 0;
    if (H->hscal) cudaFreeHost(H->hscal);
    if (H->ev0) cudaEventDestroy(H->ev0);
    if (H->ev1) cudaEventDestroy(H->ev1);
    H->hscal = nullptr, H->ev0 = H->ev1 = nullptr;
    for (cudaEvent_t e : H->prof_ev) cudaEventDestroy(e);
    H->prof_ev.clear();
    if (H->cyc_exec) cudaGraphExecDestroy(H->cyc_exec);
    H->cyc_exec = nullptr;
    if (H->chk_exec) cudaGraphExecDestroy(H->chk_exec);
    H->chk_exec = nullptr;
    for (cudaEvent_t e : H->cyc_ev) cudaEventDestroy(e);
    H->cyc_ev.clear();
    if (H->cap) cudaStreamDestroy(H->cap);
    H->cap = nullptr;
    if (H->solve_exec) cudaGraphExecDestroy(H->solve_exec);
    H->solve_exec = nullptr;
    for (int q = 0; q < 5; ++q) {
        if (H->gst[q]) cudaStreamDestroy(H->gst[q]);
        H->gst[q] = nullptr;
    }
    if (H->hctl) cudaFreeHost(H->hctl);
    if (H->harr) cudaFreeHost(H->harr);
    H->hctl = nullptr, H->harr = nullptr;
}

// Record one profiling event on the handle's stream (events are pooled; the
// ones recorded into the multigrid graph belong to it).
void prof_mark(Handle* H) {
    std::vector<cudaEvent_t>& pool = H->capturing ? H->cyc_ev : H->prof_ev;
    size_t& used = H->capturing ? H->cyc_ev_used : H->prof_used;
    if (used == pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        pool.push_back(e);
    }
    cudaEvent_t e = pool[used++];
    if (H->capturing) cudaEventRecordWithFlags(e, H->st, cudaEventRecordExternal);
    else cudaEventRecord(e, H->st);
}

template <typename T>
void sweeps_unprofiled(Handle* H, int l, int nu, T** cur, T** oth, const T* f, const T* c,
                       bool zero_first) {
    bool zero = zero_first;
    for (int s = 0; s < nu;) {
        const int k = launch_rbgs_fused<T>(H->lv[l], zero ? nullptr : *cur, *oth, f, c, nu - s, H->st);
        if (k > 0) {
            T* t = *cur;
            *cur = *oth, *oth = t;
            s += k;
        } else {
            if (zero) cudaMemsetAsync(*cur, 0, sizeof(T) * H->lv[l].d.cells, H->st);
            if constexpr (sizeof(T) == sizeof(double)) {
                if (l == 0 && H->inv64)
                    launch_rbgs_sweep64_unit(H->lv[0], *cur, f, H->F64, H->inv64, H->st);
                else
                    launch_rbgs_sweep<T>(H->lv[l], *cur, f, c, H->st);
            } else {
                launch_rbgs_sweep<T>(H->lv[l], *cur, f, c, H->st);
            }
            s += 1;
        }
        zero = false;
    }
    if (zero) cudaMemsetAsync(*cur, 0, sizeof(T) * H->lv[l].d.cells, H->st);  // nu == 0
}

// nu red-black sweeps of level l on the field held in *cur (zero_first: it is
// 0 on entry and need not be read or cleared).  Where the level fits the
// streaming kernel (FP32 levels) the sweeps run out of place, ping-ponging
// between *cur and *oth, and the two pointers are swapped so that *cur holds
// the result; elsewhere the two colour passes run in place.  With
// params.profile the finest level's full sweeps (read u, a, f; write u) are
// bracketed with events; a sweep from u = 0 reads no u and is left out.
template <typename T>
void smooth_sweeps(Handle* H, int l, int nu, T** cur, T** oth, const T* f, const T* c,
                   bool zero_first) {
    if (!(H->p.profile && l == 0)) {
        sweeps_unprofiled<T>(H, l, nu, cur, oth, f, c, zero_first);
        return;
    }
    if (zero_first) {
        const int first = nu > 0 ? 1 : 0;
        sweeps_unprofiled<T>(H, l, first, cur, oth, f, c, true);
        nu -= first;
    }
    if (nu <= 0) return;
    prof_mark(H);
    sweeps_unprofiled<T>(H, l, nu, cur, oth, f, c, false);
    prof_mark(H);
    H->prof_sweeps += nu;
}

bool pow2_ge(int v, int lo) { return v >= lo && (v & (v - 1)) == 0; }

// Per-face coarse coefficients: cubic grids of at least 64^3 (every level
// halves every axis, and the levels from 32^3 down form one cluster launch).
bool faces_apply(const recon_params* p) {
    return p->n[0] == p->n[1] && p->n[1] == p->n[2] && p->n[0] >= 64;
}

// The multigrid settings left at -1 take the precision's defaults: V(2, 2)
// cycles and at most 50 per step in FP64; in mixed precision V(1, 1) FP32
// cycles, 6 per FP64 defect correction and at most 100 per step (the FP64
// residual of a correction costs as much as several FP32 sweeps, so cheaper
// cycles in longer groups reach the same residual sooner).
void resolve_params(recon_params* p) {
    const bool mixed = p->precision == RECON_MIXED;
    if (p->coarse_faces == -1) p->coarse_faces = mixed && faces_apply(p) ? 1 : 0;
    if (p->nu1 == -1) p->nu1 = mixed ? 1 : 2;
    if (p->nu2 == -1) p->nu2 = mixed ? 1 : 2;
    // with per-face coarse coefficients a V-cycle contracts more, so the FP64
    // residual is worth forming after fewer of them
    if (p->inner_vcycles == -1) p->inner_vcycles = p->coarse_faces == 1 ? 5 : 6;
    if (p->max_vcycles == -1) p->max_vcycles = mixed ? 100 : 50;
    if (p->group_max == -1) p->group_max = p->inner_vcycles;
}

int check_params(const recon_params* p) {
    if (!p) return fail(RECON_E_INVALID, "params is NULL");
    for (int a = 0; a < 3; ++a)
        if (!pow2_ge(p->n[a], 8) || p->n[a] > 4096)
            return fail(RECON_E_INVALID, "n[%d] = %d must be a power of two in [8, 4096]", a, p->n[a]);
    if ((long long)p->n[0] * p->n[1] * p->n[2] > (1ll << 30))
        return fail(RECON_E_INVALID, "grid larger than 2^30 cells");
    bool zero_box = p->box[0] == 0.0 && p->box[1] == 0.0 && p->box[2] == 0.0;
    if (!zero_box) {
        for (int a = 0; a < 3; ++a)
            if (!(p->box[a] > 0.0) || !std::isfinite(p->box[a]))
                return fail(RECON_E_INVALID, "box[%d] must be positive", a);
        double h0 = p->box[0] / p->n[0];
        for (int a = 1; a < 3; ++a)
            if (std::fabs(p->box[a] / p->n[a] - h0) > 1e-12 * h0)
                return fail(RECON_E_INVALID, "cells must be cubic (box[a]/n[a] equal)");
    }
    if (p->precision != RECON_FP64 && p->precision != RECON_MIXED)
        return fail(RECON_E_INVALID, "precision must be RECON_FP64 or RECON_MIXED");
    if (!(p->xi_m > 0.0 && p->xi_m < 1.0)) return fail(RECON_E_INVALID, "need 0 < xi_m < 1");
    if (!(p->v_m > 1.0)) return fail(RECON_E_INVALID, "need v_m > 1");
    if (!(p->a_min > 0.0)) return fail(RECON_E_INVALID, "need a_min > 0");
    if (p->climiter < 0 || p->climiter > 2) return fail(RECON_E_INVALID, "bad climiter");
    if (!(p->s_side >= 0.0 && p->s_side <= 0.25)) return fail(RECON_E_INVALID, "need 0 <= s_side <= 1/4");
    if (p->nu1 < 0 || p->nu2 < 0 || p->nu1 + p->nu2 == 0 || p->nu1 > 16 || p->nu2 > 16)
        return fail(RECON_E_INVALID, "bad nu1/nu2");
    if (!(p->tol_in > 0.0) || p->max_vcycles < 1) return fail(RECON_E_INVALID, "bad tol_in/max_vcycles");
    if (!(p->tol_out >= 0.0) || p->k_max < 0) return fail(RECON_E_INVALID, "bad tol_out/k_max");
    if (!(p->d_max > 0.0)) return fail(RECON_E_INVALID, "need d_max > 0");
    if (!(p->alpha_min > 0.0 && p->alpha_min <= 1.0)) return fail(RECON_E_INVALID, "need 0 < alpha_min <= 1");
    if (!(p->lambda_floor >= 0.0 && p->lambda_floor < 1.0)) return fail(RECON_E_INVALID, "need 0 <= lambda_floor < 1");
    if (p->inner_vcycles < 1 || p->inner_vcycles > 16) return fail(RECON_E_INVALID, "need 1 <= inner_vcycles <= 16");
    if (p->density_update != 0 && p->density_update != 1) return fail(RECON_E_INVALID, "density_update must be 0 or 1");
    if (p->device_loop != 0 && p->device_loop != 1) return fail(RECON_E_INVALID, "device_loop must be 0 or 1");
    if (p->checkpoint != 0 && p->checkpoint != 1) return fail(RECON_E_INVALID, "checkpoint must be 0 or 1");
    if (p->checkpoint && p->density_update != 0)
        return fail(RECON_E_INVALID, "checkpoint (the adjoint) needs density_update = 0");
    if (p->stream_planes != 0 && p->stream_planes != 4 && p->stream_planes != 8 && p->stream_planes != 16)
        return fail(RECON_E_INVALID, "stream_planes must be 0, 4, 8 or 16");
    if (p->restrict_planes < 0 || p->restrict_planes > 16 || (p->restrict_planes & (p->restrict_planes - 1)))
        return fail(RECON_E_INVALID, "restrict_planes must be 0, 1, 2, 4, 8 or 16");
    if (p->coarse_faces != 0 && p->coarse_faces != 1) return fail(RECON_E_INVALID, "coarse_faces must be 0 or 1");
    if (p->coarse_faces == 1 && (p->precision != RECON_MIXED || !faces_apply(p)))
        return fail(RECON_E_INVALID, "coarse_faces = 1 needs RECON_MIXED on a cubic grid of at least 64^3");
    if (p->tune_inner < 0 || p->tune_inner > 2) return fail(RECON_E_INVALID, "tune_inner must be 0, 1 or 2");
    if (p->tma != 0 && p->tma != 1) return fail(RECON_E_INVALID, "tma must be 0 or 1");
    if (p->warm_start < 0 || p->warm_start > 2) return fail(RECON_E_INVALID, "warm_start must be 0, 1 or 2");
    if (p->group_max < p->inner_vcycles || p->group_max > 64)
        return fail(RECON_E_INVALID, "need inner_vcycles <= group_max <= 64");
    return RECON_OK;
}

// 2^F with F chosen so that any partial sum of terms totalling <= total stays
// below 2^61 in the signed 64-bit accumulator.
double fixed_scale(double total) {
    int e = 0;
    std::frexp(total > 1.0 ? total : 1.0, &e);  // total < 2^e
    return std::ldexp(1.0, 61 - e);
}

int sync_scalars(Handle* H) {
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(H->hscal, H->scal, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, H->st));
    CK(cudaStreamSynchronize(H->st));
    return RECON_OK;
}

// ------------------------------------------------------------ V-cycles

template <typename T>
struct MG {
    std::vector<T*>& u;
    std::vector<T*>& f;
    std::vector<T*>& c;
    std::vector<T*>& r;
};

// One V(nu1, nu2) cycle of level l on L u = f; zero_u: u = 0 on entry.  The
// level's residual buffer doubles as the ping-pong partner of the streaming
// smoother; with even sweep counts the result is back in u, otherwise it is
// copied there.
// correct_into (mixed mode, finest level): if not null, the V-cycle's
// result is also added to this FP64 field, by the last sweep where it can be;
// returns whether it was.
template <typename T>
bool vcycle(Handle* H, MG<T>& g, int l, T* u, const T* f, bool zero_u,
            double* correct_into = nullptr) {
    const int last = (int)H->lv.size() - 1;
    const Level& L = H->lv[l];
    if (l == H->lc && launch_coarse_cluster<T>(H->cc, f, u, H->minv, zero_u, H->st)) return false;
    if (l == H->l0 && launch_coarse_vcycle<T>(H->cs, f, u, H->minv, zero_u, H->st)) return false;
    if (l == last) {
        launch_coarse_solve<T>(H->minv, f, u, H->st);
        return false;
    }
    T* cur = u;
    T* oth = g.r[l];
    smooth_sweeps<T>(H, l, H->p.nu1, &cur, &oth, f, g.c[l], zero_u);
    bool streamed = false;
    if constexpr (sizeof(T) == sizeof(float))
        streamed = launch_resid_restrict_stream(L, H->lv[l + 1], cur, f, g.c[l], g.f[l + 1], H->st);
    if (!streamed) launch_resid_restrict<T>(L, H->lv[l + 1], cur, f, g.c[l], g.f[l + 1], H->st);
    vcycle<T>(H, g, l + 1, g.u[l + 1], g.f[l + 1], true);
    int nu2 = H->p.nu2;
    bool folded = false, corrected = false;
    if constexpr (sizeof(T) == sizeof(float)) {
        // the coarse correction folded into the first post-smoothing sweep,
        // and the defect correction too where that sweep is the last
        double* c64 = nu2 == 1 ? correct_into : nullptr;
        if (nu2 >= 1 &&
            launch_rbgs_prolong(L, H->lv[l + 1], g.u[l + 1], cur, oth, f, g.c[l], H->st, c64)) {
            std::swap(cur, oth);
            nu2 -= 1;
            folded = true;
            corrected = c64 != nullptr;
        }
    }
    if (!folded) launch_prolong_add<T>(L, H->lv[l + 1], g.u[l + 1], cur, H->st);
    if constexpr (sizeof(T) == sizeof(float)) {
        // the defect correction folded into the last sweep
        if (correct_into && !corrected && nu2 >= 1) {
            smooth_sweeps<T>(H, l, nu2 - 1, &cur, &oth, f, g.c[l], false);
            if (launch_rbgs_correct(L, cur, oth, f, g.c[l], correct_into, H->st)) {
                std::swap(cur, oth);
                corrected = true;
            } else {
                smooth_sweeps<T>(H, l, 1, &cur, &oth, f, g.c[l], false);
            }
            nu2 = 0;
        }
    }
    smooth_sweeps<T>(H, l, nu2, &cur, &oth, f, g.c[l], false);
    if (cur != u)
        cudaMemcpyAsync(u, cur, sizeof(T) * L.d.cells, cudaMemcpyDeviceToDevice, H->st);
    return corrected;
}

template <typename T>
void build_hierarchy(Handle* H, std::vector<T*>& c) {
    launch_faces64(H->lv[0], H->a64, H->F64, H->D64, H->inv64, H->st);
    for (size_t l = 0; l + 1 < H->lv.size(); ++l) {
        if constexpr (sizeof(T) == sizeof(float)) {
            if (H->lv[l + 1].face) {
                launch_faces_line(H->lv[l], H->lv[l + 1], c[l], c[l + 1], H->st);
                continue;
            }
        }
        launch_restrict<T>(H->lv[l], H->lv[l + 1], c[l], c[l + 1], H->st);
    }
    launch_coarse_invert<T>(H->lv.back(), c.back(), H->minv, H->st);
}

// Mass per current curvilinear cell (tracer CIC deposit, or the carried m
// of App. A's variant), the operator coefficient a = max(m, a_min) and sum m.
int deposit_step(Handle* H) {
    if (H->p.density_update == 1) {
        // the carried mass per cell: only the coefficient and the mass sum
        launch_coef_from_m(H->cells, H->m, H->p.a_min, H->a64, H->mixed ? H->c32[0] : nullptr,
                           H->part[0], H->st);
        finish_reduce(H->part[0], 0, H->scal, SC_SUM_M, H->st);
        return RECON_OK;
    }
    const double scale = fixed_scale((double)H->cells);
    launch_deposit_tracers(H->d, H->ox, H->oy, H->oz, H->w, scale, H->mfix, H->st);
    launch_mass_coef(H->cells, H->mfix, 1.0 / scale, H->p.a_min, H->m, H->a64,
                     H->mixed ? H->c32[0] : nullptr, H->part[0], H->st);
    finish_reduce(H->part[0], 0, H->scal, SC_SUM_M, H->st);
    return RECON_OK;
}

// ------------------------------------------------------------ the iteration
//
// One solve is a sequence of segments, each a fixed list of kernel launches
// ending in a control kernel (control.cu) that takes the segment's decision:
//   init;  while (go_step) { step head [R_k test];  if (go_cont) {
//       multigrid head;  while (go_mg) multigrid iteration;
//       step tail [alpha];  if (go_adv) advance [k += 1] } }
//   if (go_fin) final deposit.
// The host-driven loop launches the segments and reads the control block
// back after each decision; with device_loop the same segments are recorded
// once into a CUDA graph whose conditional nodes the control kernels set.

// Step head: deposit on the deformed mesh, geometry and limited source
// t = Sigma + C + E, s = S t - mean (Eq. elliptic of App. A), R_k test.
void step_head(Handle* H, const CtlHandles& h) {
    const recon_params& p = H->p;
    if (H->ckpt) launch_ckpt_state(H->ctl, H->cells, H->phi, H->ox, H->oy, H->oz, H->ckpt, H->st);
    deposit_step(H);
    SourceParams sp{p.xi_m, p.v_m, p.climiter};
    launch_geometry_source(H->d, sp, H->phi, H->m, H->t, H->e6, H->part[0], H->part[1], H->st);
    finish_reduce(H->part[0], 0, H->scal, SC_SUM_T, H->st);
    finish_reduce(H->part[1], 1, H->scal, SC_MIN_DET, H->st);
    launch_smooth_S(H->d, p.s_side, H->t, H->scal + SC_SUM_T, H->s, nullptr, H->v3, nullptr,
                    H->part[2], H->st);
    finish_reduce(H->part[2], 0, H->scal, SC_SUM_S2, H->st);
    launch_ctl_step_begin(H->ctl, H->scal, H->arr, (double)H->cells, p.tol_out, h, H->st);
}

// Multigrid head: coefficient hierarchy, the initial guess of phidot and
// (mixed) the first FP64 defect handed to the FP32 V-cycle.  warm: phidot
// keeps the last step's solution (0 before the first step, from solve_init),
// with warm_start = 2 extrapolated from the last two (k_warm_extrapolate),
// and the first defect is the FP64 residual s - L phidot; otherwise
// phidot = 0 and the defect is s itself (its FP32 copy).
void mg_head(Handle* H, const CtlHandles& h, bool warm) {
    if (H->mixed) build_hierarchy<float>(H, H->c32);
    else build_hierarchy<double>(H, H->c64);
    if (warm && H->p.warm_start == 2)
        launch_warm_extrapolate(H->ctl, H->arr.alpha, H->phidot, H->phidot_prev, H->cells, H->st);
    if (warm) {
        if (H->mixed)
            launch_residual64_to32(H->lv[0], H->phidot, H->s, H->F64, H->D64, H->f32[0], H->part[0], H->st);
    } else {
        cudaMemsetAsync(H->phidot, 0, sizeof(double) * H->cells, H->st);
        if (H->mixed) launch_to_f32(H->cells, H->s, H->f32[0], H->st);
    }
    launch_ctl_mg_begin(H->ctl, H->arr, H->mixed ? 1 : 0, H->p.tol_in, H->p.max_vcycles,
                        h, H->st);
}

// Grouped FP64 checks (params.group_max > inner_vcycles): one block of
// inner_vcycles FP32 V-cycles on the correction e (zeroed where a new defect
// correction starts), then the control's decision whether the correction
// ends after this block.
void mg_block(Handle* H, const CtlHandles& h) {
    MG<float> g{H->u32, H->f32, H->c32, H->r32};
    launch_zero_if_fresh(H->ctl, H->u32[0], H->cells, H->st);
    for (int v = 0; v < H->p.inner_vcycles; ++v)
        vcycle<float>(H, g, 0, H->u32[0], H->f32[0], false, nullptr);
    launch_ctl_block(H->ctl, H->arr, H->p.inner_vcycles, H->p.max_vcycles, h, H->st);
}

// The end of a defect correction under grouped checks: phidot += e, the FP64
// residual (and its FP32 copy, the next right-hand side), the stopping test
// and the length of the next correction.
void mg_check_body(Handle* H, const CtlHandles& h) {
    launch_correct(H->cells, H->phidot, H->u32[0], H->st);
    launch_residual64_to32(H->lv[0], H->phidot, H->s, H->F64, H->D64, H->f32[0], H->part[0], H->st);
    finish_reduce(H->part[0], 0, H->scal, SC_RES2, H->st);
    launch_ctl_group_check(H->ctl, H->scal, H->arr, H->p.inner_vcycles, H->p.group_max, H->p.tol_in,
                           H->p.max_vcycles, h, H->st);
}

// One multigrid iteration: the V-cycle (FP64 on phidot, or inner_vcycles FP32
// V-cycles on the correction e followed by phidot += e), then the FP64
// residual of L phidot = s (in mixed mode also the next FP32 right-hand side)
// and its squared norm, and the stopping test.  Under grouped checks only the
// block (mg_block): the caller runs mg_check_body where the control asks.
void mg_iter(Handle* H, const CtlHandles& h) {
    const Level& L0 = H->lv[0];
    if (H->adaptive) {
        mg_block(H, h);
        return;
    }
    if (!H->mixed) {
        MG<double> g{H->u64, H->f64, H->c64, H->r64};
        vcycle<double>(H, g, 0, H->phidot, H->s, false);
        launch_residual_norm64(L0, H->phidot, H->s, H->F64, H->D64, H->part[0], H->st);
    } else {
        MG<float> g{H->u32, H->f32, H->c32, H->r32};
        bool corrected = false;
        for (int v = 0; v < H->p.inner_vcycles; ++v) {
            const bool last = v + 1 == H->p.inner_vcycles;
            corrected = vcycle<float>(H, g, 0, H->u32[0], H->f32[0], v == 0, last ? H->phidot : nullptr);
        }
        if (!corrected) launch_correct(H->cells, H->phidot, H->u32[0], H->st);
        launch_residual64_to32(L0, H->phidot, H->s, H->F64, H->D64, H->f32[0], H->part[0], H->st);
    }
    finish_reduce(H->part[0], 0, H->scal, SC_RES2, H->st);
    launch_ctl_mg_check(H->ctl, H->scal, H->arr, H->mixed ? H->p.inner_vcycles : 1, H->p.tol_in,
                        H->p.max_vcycles, h, H->st);
}

// Step tail: dphi = S phidot (mean removed in the advance), the limiter and
// the choice of alpha.
void step_tail(Handle* H, const CtlHandles& h) {
    const recon_params& p = H->p;
    if (H->ckpt) launch_ckpt_phidot(H->ctl, H->cells, H->phidot, H->ckpt, H->st);
    launch_smooth_S(H->d, p.s_side, H->phidot, nullptr, H->dphi, H->dphi32, H->v3, H->part[0],
                    nullptr, H->st);
    finish_reduce(H->part[0], 0, H->scal, SC_SUM_DPHI, H->st);
    if (!H->replay_d) {
        launch_limiter(H->d, H->lp, H->e6, H->dphi, H->phi32, H->dphi32, H->part[1], H->part[2],
                       H->st);
        finish_reduce(H->part[1], 2, H->scal, SC_MAX_K, H->st);
        finish_reduce(H->part[2], 2, H->scal, SC_MAX_G, H->st);
    }
    launch_ctl_select_alpha(H->ctl, H->scal, H->arr, H->replay_d, H->lp.kmax, p.d_max, p.alpha_min,
                            h, H->st);
}

// Advance by the chosen alpha: tracers and phi (or, App. A's variant, the
// mass per cell and phi), then k += 1.
void advance(Handle* H, const CtlHandles& h) {
    const int n = H->cells;
    const double* alpha = H->scal + SC_ALPHA;
    if (H->p.density_update == 1) {
        launch_mass_literal(H->d, H->e6, H->dphi, alpha, H->m, H->v3m, H->st);
        launch_phi_advance(n, alpha, H->dphi, H->scal + SC_SUM_DPHI, H->phi, H->phi32, H->st);
    } else {
        // the node displacements alpha V in fixed point, in the v3 buffer
        long long* d3 = reinterpret_cast<long long*>(H->v3);
        launch_node_displacement(H->d, H->e6, H->dphi, alpha, d3, d3 + n, d3 + 2 * (size_t)n, H->st);
        launch_advance(H->d, d3, d3 + n, d3 + 2 * (size_t)n, alpha, H->dphi, H->scal + SC_SUM_DPHI,
                       H->ox, H->oy, H->oz, H->phi, H->phi32, H->st);
    }
    launch_ctl_step_end(H->ctl, H->p.k_max, h, H->st);
}

// init: tracer c = node c with mass rho_c / rho_bar, phi = 0
void solve_init(Handle* H) {
    launch_ctl_init(H->ctl, H->st);
    cudaMemsetAsync(H->phidot, 0, sizeof(double) * H->cells, H->st);  // the first step's initial guess
    launch_init_tracers(H->cells, H->rho, H->scal + SC_SUM_RHO, H->w, H->ox, H->oy, H->oz, H->phi,
                        H->phi32, H->st);
    if (H->p.density_update == 1)  // App. A: the mass per cell starts as rho / rho_bar
        cudaMemcpyAsync(H->m, H->w, sizeof(double) * H->cells, cudaMemcpyDeviceToDevice, H->st);
}

void final_body(Handle* H) {
    deposit_step(H);
    launch_ctl_final_mass(H->ctl, H->scal, H->st);
}

int read_ctl(Handle* H) {
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(H->hctl, H->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, H->st));
    CK(cudaStreamSynchronize(H->st));
    return RECON_OK;
}

// The multigrid iteration (or, under grouped checks, the check body) with the
// control block's readback, recorded once as a CUDA graph on a private stream
// and replayed on the handle's stream.
template <typename F>
int record_cycle_graph(Handle* H, cudaGraphExec_t* exec, long long* kernels, int* sweeps, F&& segment) {
    if (!H->cap) CK(cudaStreamCreateWithFlags(&H->cap, cudaStreamNonBlocking));
    cudaStream_t user = H->st;
    const long long c0 = launch_counter().load();
    const int s0 = H->prof_sweeps;
    CK(cudaStreamBeginCapture(H->cap, cudaStreamCaptureModeRelaxed));
    H->st = H->cap;
    H->capturing = true;
    segment();
    cudaMemcpyAsync(H->hctl, H->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, H->st);
    H->capturing = false;
    H->st = user;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(H->cap, &g);
    *kernels = launch_counter().load() - c0;
    launch_counter() -= *kernels;
    *sweeps = H->prof_sweeps - s0;
    H->prof_sweeps = s0;
    if (e != cudaSuccess) return fail(RECON_E_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *exec = nullptr;
        return fail(RECON_E_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    return RECON_OK;
}

// The check body of grouped checks, when the block just run asked for it.
int run_check(Handle* H) {
    if (!H->chk_exec) {
        int no_sweeps = 0;
        int rc = record_cycle_graph(H, &H->chk_exec, &H->chk_kernels, &no_sweeps,
                                    [&] { mg_check_body(H, CtlHandles{}); });
        if (rc) return rc;
    }
    CK(cudaGraphLaunch(H->chk_exec, H->st));
    CK(cudaStreamSynchronize(H->st));
    launch_counter() += H->chk_kernels;
    return RECON_OK;
}

int run_cycle(Handle* H) {
    if (!H->cyc_exec) {
        int rc = record_cycle_graph(H, &H->cyc_exec, &H->cyc_kernels, &H->cyc_sweeps,
                                    [&] { mg_iter(H, CtlHandles{}); });
        if (rc) return rc;
    }
    CK(cudaGraphLaunch(H->cyc_exec, H->st));
    CK(cudaStreamSynchronize(H->st));
    launch_counter() += H->cyc_kernels;
    if (H->p.profile) {
        for (size_t q = 0; q + 1 < H->cyc_ev_used; q += 2) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, H->cyc_ev[q], H->cyc_ev[q + 1]) == cudaSuccess) H->prof_ms += ms;
        }
        cudaGetLastError();
        H->prof_sweeps += H->cyc_sweeps;
    }
    if (H->adaptive && H->hctl->chk) return run_check(H);
    return RECON_OK;
}

// params.tune_inner, on the first solve of a mixed-precision handle: the
// first step's linear solve (from phidot = 0 on the step's own source and
// coefficient) is run with 3, 4, 5, 6 and 8 FP32 V-cycles per FP64 defect
// correction, twice over (the first round only brings the clocks up), timed
// with CUDA events, and the fastest count is kept.  Every count stops at the
// same FP64 residual; the solve that follows starts again from phi = 0.
int tune_inner_vcycles(Handle* H) {
    H->inner_tuned = true;
    // (not with profile: the sweep timing events belong to the timed solve)
    if (!H->mixed || !H->p.tune_inner || H->p.profile) return RECON_OK;
    Range range("recon_tune_inner");
    const CtlHandles none{};
    solve_init(H);
    step_head(H, none);
    int rc = read_ctl(H);
    if (rc) return rc;
    if (!H->hctl->go_cont) return RECON_OK;  // nothing to solve at step 0
    const int cand[5] = {3, 4, 5, 6, 8};
    // tune_inner = 2 also tries every smoothing schedule (nu1, nu2) of the
    // FP32 V-cycle (the same in the per-level, single-block and cluster parts)
    const int sched2[4][2] = {{1, 1}, {1, 2}, {2, 1}, {2, 2}};
    const int own[1][2] = {{H->p.nu1, H->p.nu2}};
    const int (*sched)[2] = H->p.tune_inner == 2 ? sched2 : own;
    const int nsched = H->p.tune_inner == 2 ? 4 : 1;
    auto set_schedule = [&](int nu1, int nu2) {
        H->p.nu1 = H->cc.nu1 = H->cs.nu1 = nu1;
        H->p.nu2 = H->cc.nu2 = H->cs.nu2 = nu2;
    };
    int best = H->p.inner_vcycles, best_s = 0;
    float best_ms = 0.f;
    for (int round = 0; round < 2; ++round)
        for (int si = 0; si < nsched; ++si)
        for (int n : cand) {
            if (H->adaptive && n > H->p.group_max) continue;
            set_schedule(sched[si][0], sched[si][1]);
            H->p.inner_vcycles = n;
            if (H->cyc_exec) cudaGraphExecDestroy(H->cyc_exec);
            H->cyc_exec = nullptr;
            if (H->chk_exec) cudaGraphExecDestroy(H->chk_exec);
            H->chk_exec = nullptr;
            CK(cudaEventRecord(H->ev0, H->st));
            mg_head(H, none, false);  // step 0 starts from phidot = 0 either way
            if ((rc = read_ctl(H))) return rc;
            while (H->hctl->go_mg)
                if ((rc = run_cycle(H))) return rc;
            CK(cudaEventRecord(H->ev1, H->st));
            CK(cudaEventSynchronize(H->ev1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, H->ev0, H->ev1));
            if (round == 1 && (best_ms == 0.f || ms < best_ms)) best = n, best_s = si, best_ms = ms;
        }
    set_schedule(sched[best_s][0], sched[best_s][1]);
    H->p.inner_vcycles = best;
    if (H->cyc_exec) cudaGraphExecDestroy(H->cyc_exec);
    H->cyc_exec = nullptr;
    if (H->chk_exec) cudaGraphExecDestroy(H->chk_exec);
    H->chk_exec = nullptr;
    H->adaptive = H->p.group_max > H->p.inner_vcycles;
    return RECON_OK;
}

// The host-driven loop: each decision is read back from the control block.
int solve_host(Handle* H) {
    const CtlHandles none{};
    solve_init(H);
    for (int k = 0; k < H->p.k_max; ++k) {
        Range step_range("recon step");
        step_head(H, none);
        int rc = read_ctl(H);
        if (rc) return rc;
        if (!H->hctl->go_cont) break;
        {
            Range mg_range("recon multigrid");
            mg_head(H, none, H->p.warm_start != 0);
            if ((rc = read_ctl(H))) return rc;
            while (H->hctl->go_mg)
                if ((rc = run_cycle(H))) return rc;
        }
        step_tail(H, none);
        if ((rc = read_ctl(H))) return rc;
        if (!H->hctl->go_adv) break;
        advance(H, none);
    }
    if (H->p.density_update == 0) {  // the carried m of App. A's variant is current
        launch_ctl_final(H->ctl, 1, none, H->st);
        int rc = read_ctl(H);
        if (rc) return rc;
        if (H->hctl->go_fin) final_body(H);
    }
    return RECON_OK;
}

// ---- the solve as one CUDA graph with conditional nodes

// Adds a conditional node of the given type after everything captured so far
// on stream s (which is capturing into some graph) and returns its body.
int add_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                    cudaGraph_t* body) {
    cudaStreamCaptureStatus cs;
    unsigned long long id = 0;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(s, &cs, &id, &g, &deps, &edges, &nd));
    if (cs != cudaStreamCaptureStatusActive) return fail(RECON_E_CUDA, "stream is not capturing");
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = h;
    np.conditional.type = type;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    CK(cudaGraphAddNode(&node, g, deps, edges, nd, &np));
    CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    *body = np.conditional.phGraph_out[0];
    return RECON_OK;
}

// A conditional handle on the graph stream s is capturing into, reset to
// def at every launch of the graph.
int new_handle(cudaStream_t s, unsigned def, cudaGraphConditionalHandle* h) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    CK(cudaGraphConditionalHandleCreate(h, g, def, cudaGraphCondAssignDefault));
    return RECON_OK;
}

// Records the segments into body graph g on stream s; returns the kernels
// recorded (the launch counter is restored).
template <typename F>
int capture_into(Handle* H, cudaStream_t s, cudaGraph_t g, long long* kernels, F&& segment) {
    CK(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    cudaStream_t prev = H->st;
    H->st = s;
    const long long c0 = launch_counter().load();
    int rc = segment();
    const long long kk = launch_counter().load() - c0;
    launch_counter() -= kk;
    if (kernels) *kernels += kk;
    H->st = prev;
    cudaGraph_t out = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &out);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(RECON_E_CUDA, "solve graph capture failed: %s", cudaGetErrorString(e));
    return RECON_OK;
}

int build_solve_graph(Handle* H) {
    for (int q = 0; q < 5; ++q)
        if (!H->gst[q]) CK(cudaStreamCreateWithFlags(&H->gst[q], cudaStreamNonBlocking));
    cudaGraph_t top = nullptr;
    CK(cudaGraphCreate(&top, 0));
    GraphCounts& n = H->gn;
    n = GraphCounts{};
    CtlHandles h{};
    h.active = 1;
    H->capturing = true;
    int rc = capture_into(H, H->gst[0], top, &n.init, [&]() -> int {
        solve_init(H);
        if (H->p.k_max > 0) {
            int r = new_handle(H->gst[0], 1, &h.step);
            if (r) return r;
            cudaGraph_t b_step = nullptr;
            if ((r = add_conditional(H->gst[0], h.step, cudaGraphCondTypeWhile, &b_step))) return r;
            r = capture_into(H, H->gst[1], b_step, &n.step, [&]() -> int {
                int r1 = new_handle(H->gst[1], 0, &h.cont);
                if (r1) return r1;
                step_head(H, h);
                cudaGraph_t b_cont = nullptr;
                if ((r1 = add_conditional(H->gst[1], h.cont, cudaGraphCondTypeIf, &b_cont))) return r1;
                return capture_into(H, H->gst[2], b_cont, &n.cont, [&]() -> int {
                    int r2 = new_handle(H->gst[2], 0, &h.mg);
                    if (!r2) r2 = new_handle(H->gst[2], 0, &h.adv);
                    if (r2) return r2;
                    mg_head(H, h, H->p.warm_start != 0);
                    cudaGraph_t b_mg = nullptr, b_adv = nullptr;
                    if ((r2 = add_conditional(H->gst[2], h.mg, cudaGraphCondTypeWhile, &b_mg))) return r2;
                    r2 = capture_into(H, H->gst[3], b_mg, &n.mg, [&]() -> int {
                        if (!H->adaptive) {
                            mg_iter(H, h);
                            return RECON_OK;
                        }
                        // grouped checks: the block, then the check body where
                        // the block's control kernel asks for it
                        int r3 = new_handle(H->gst[3], 0, &h.chk);
                        if (r3) return r3;
                        mg_block(H, h);
                        cudaGraph_t b_chk = nullptr;
                        if ((r3 = add_conditional(H->gst[3], h.chk, cudaGraphCondTypeIf, &b_chk))) return r3;
                        return capture_into(H, H->gst[4], b_chk, &n.chk, [&]() -> int {
                            mg_check_body(H, h);
                            return RECON_OK;
                        });
                    });
                    if (r2) return r2;
                    step_tail(H, h);
                    if ((r2 = add_conditional(H->gst[2], h.adv, cudaGraphCondTypeIf, &b_adv))) return r2;
                    return capture_into(H, H->gst[3], b_adv, &n.adv, [&]() -> int {
                        advance(H, h);
                        return RECON_OK;
                    });
                });
            });
            if (r) return r;
        }
        if (H->p.density_update == 0) {
            int r = new_handle(H->gst[0], 0, &h.fin);
            if (r) return r;
            launch_ctl_final(H->ctl, 1, h, H->st);
            cudaGraph_t b_fin = nullptr;
            if ((r = add_conditional(H->gst[0], h.fin, cudaGraphCondTypeIf, &b_fin))) return r;
            return capture_into(H, H->gst[1], b_fin, &n.fin, [&]() -> int {
                final_body(H);
                return RECON_OK;
            });
        }
        return RECON_OK;
    });
    H->capturing = false;
    if (rc) {
        cudaGraphDestroy(top);
        cudaGetLastError();
        return rc;
    }
    cudaError_t e = cudaGraphInstantiate(&H->solve_exec, top, 0);
    cudaGraphDestroy(top);
    if (e != cudaSuccess) {
        H->solve_exec = nullptr;
        cudaGetLastError();
        return fail(RECON_E_CUDA, "solve graph instantiation failed: %s", cudaGetErrorString(e));
    }
    return RECON_OK;
}

// Kernels of the end-of-solve statistics (geometry, delta_r, 3 reductions).
constexpr int kStatsKernels = 5;

// Launches the whole solve (graph mode) and, with stats, the end-of-solve
// statistics and the readback of the control block and the per-step
// records; nothing waits for the device.
int solve_launch(Handle* H, bool want_stats) {
    if (!H->solve_exec) {
        int rc = build_solve_graph(H);
        if (rc) return rc;
    }
    CK(cudaEventRecord(H->ev0, H->st));
    CK(cudaGraphLaunch(H->solve_exec, H->st));
    CK(cudaEventRecord(H->ev1, H->st));
    if (want_stats) {
        launch_geometry_out(H->d, H->phi, nullptr, nullptr, H->part[0], H->part[1], H->st);
        finish_reduce(H->part[0], 1, H->scal, SC_MIN_DET, H->st);
        finish_reduce(H->part[1], 1, H->scal, SC_MIN_LAM, H->st);
        launch_delta_r(H->d, H->phi, H->t, H->part[2], H->st);
        finish_reduce(H->part[2], 2, H->scal, SC_MAX_DR, H->st);
        CK(cudaMemcpyAsync(H->hscal, H->scal, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, H->st));
    }
    CK(cudaMemcpyAsync(H->hctl, H->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, H->st));
    const size_t km = (size_t)std::max(H->p.k_max, 1);
    CK(cudaMemcpyAsync(H->harr, H->arr.Rk, 4 * km * sizeof(double), cudaMemcpyDeviceToHost, H->st));
    return RECON_OK;
}

// Fills the record from the control block (after the solve has finished).
void fill_stats(Handle* H, recon_stats* stats, float ms, long long launches, bool stats_kernels) {
    const Ctl& c = *H->hctl;
    stats->status = c.status;
    stats->steps = c.k;
    stats->vcycles = c.vtot;
    stats->R0 = c.R0;
    stats->R = c.R;
    stats->ms = ms;
    stats->mass_error = std::fabs(c.last_mass - (double)H->cells) / (double)H->cells;
    stats->launches = launches;
    stats->inner_vcycles = H->mixed ? H->p.inner_vcycles : 0;
    stats->nu1 = H->p.nu1, stats->nu2 = H->p.nu2;
    const size_t km = (size_t)std::max(H->p.k_max, 1);
    const double* Rk = H->harr;
    const double* al = H->harr + km;
    const double* rr = H->harr + 2 * km;
    const int* nc = (const int*)(H->harr + 3 * km);
    for (int q = 0; q < c.n_step; ++q)
        if (stats->Rk) stats->Rk[q] = Rk[q];
    for (int q = 0; q < c.n_adv; ++q) {
        if (stats->alpha) stats->alpha[q] = al[q];
        if (stats->ncycles) stats->ncycles[q] = nc[q];
        if (stats->relres) stats->relres[q] = rr[q];
    }
    if (stats_kernels) {
        stats->min_det = H->hscal[SC_MIN_DET];
        stats->min_lambda0 = H->hscal[SC_MIN_LAM];
        stats->max_delta_r = H->hscal[SC_MAX_DR];
    }
}

// Kernels one graph-mode solve launched, from the body counts of the graph
// and the control block's execution counters.
long long graph_launches(const Handle* H) {
    const Ctl& c = *H->hctl;
    const GraphCounts& n = H->gn;
    return n.init + c.n_step * n.step + c.n_cont * n.cont + (long long)c.n_mg * n.mg +
           c.n_adv * n.adv + c.n_fin * n.fin + (long long)c.n_chk * n.chk;
}

int solve_finish(Handle* H, recon_stats* stats) {
    CK(cudaStreamSynchronize(H->st));
    // the statistics kernels after the graph were counted at their launch
    const long long kk = graph_launches(H);
    launch_counter() += kk;
    H->solved = true;
    if (stats) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, H->ev0, H->ev1);
        fill_stats(H, stats, ms, kk + kStatsKernels, true);
        stats->smooth_ms = 0.0;
        stats->smooth_sweeps = 0;
        stats->smooth_bytes = 4.0 * (H->mixed ? sizeof(float) : sizeof(double)) * (double)H->cells;
    }
    return H->hctl->status;
}

bool use_graph(const Handle* H) { return H->p.device_loop && !H->p.profile; }

int solve(Handle* H, recon_stats* stats) {
    Range range(use_graph(H) ? "recon_solve (graph)" : "recon_solve (host loop)");
    if (use_graph(H)) {
        int rc = solve_launch(H, stats != nullptr);
        if (rc) return rc;
        return solve_finish(H, stats);
    }
    const long long launches0 = launch_counter().load();
    H->prof_used = 0;
    H->prof_sweeps = 0;
    H->prof_ms = 0.0;
    CK(cudaEventRecord(H->ev0, H->st));
    int rc = solve_host(H);
    if (rc) return rc;
    CK(cudaEventRecord(H->ev1, H->st));
    CK(cudaEventSynchronize(H->ev1));
    H->solved = true;
    if (stats) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, H->ev0, H->ev1);
        launch_geometry_out(H->d, H->phi, nullptr, nullptr, H->part[0], H->part[1], H->st);
        finish_reduce(H->part[0], 1, H->scal, SC_MIN_DET, H->st);
        finish_reduce(H->part[1], 1, H->scal, SC_MIN_LAM, H->st);
        launch_delta_r(H->d, H->phi, H->t, H->part[2], H->st);
        finish_reduce(H->part[2], 2, H->scal, SC_MAX_DR, H->st);
        CK(cudaMemcpyAsync(H->hscal, H->scal, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, H->st));
        CK(cudaMemcpyAsync(H->hctl, H->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, H->st));
        const size_t km = (size_t)std::max(H->p.k_max, 1);
        CK(cudaMemcpyAsync(H->harr, H->arr.Rk, 4 * km * sizeof(double), cudaMemcpyDeviceToHost, H->st));
        CK(cudaStreamSynchronize(H->st));
        fill_stats(H, stats, ms, launch_counter().load() - launches0, true);
        double sm = H->prof_ms;
        for (size_t q = 0; q + 1 < H->prof_used; q += 2) {
            float e = 0.f;
            if (cudaEventElapsedTime(&e, H->prof_ev[q], H->prof_ev[q + 1]) == cudaSuccess) sm += e;
        }
        cudaGetLastError();
        stats->smooth_ms = sm;
        stats->smooth_sweeps = H->prof_sweeps;
        // one sweep reads u, a, f and writes u at the finest level
        stats->smooth_bytes = 4.0 * (H->mixed ? sizeof(float) : sizeof(double)) * (double)H->cells;
    }
    return H->hctl->status;
}

// ---- the adjoint sweep (adjoint.cu has the kernels)

// Runs the linear solve L(a) u = rhs (rhs already in H->s, its sum of
// squares in scal[SC_SUM_S2]) with the forward solve's multigrid, on the
// adjoint's own control block; u is left in H->phidot.
int adjoint_mg(Handle* H) {
    const CtlHandles none{};
    launch_ctl_init(H->ctl, H->st);
    launch_ctl_step_begin(H->ctl, H->scal, H->arr, (double)H->cells, -1.0, none, H->st);
    mg_head(H, none, false);  // each adjoint solve starts from 0
    int rc = read_ctl(H);
    while (!rc && H->hctl->go_mg) {
        mg_iter(H, none);
        rc = read_ctl(H);
        if (!rc && H->adaptive && H->hctl->chk) {
            mg_check_body(H, none);
            rc = read_ctl(H);
        }
    }
    return rc;
}

int adjoint(Handle* H, const double* gbar, double* grad) {
    Range range("recon_adjoint");
    const Dims& d = H->d;
    const int cells = H->cells;
    const size_t n = (size_t)cells;
    const recon_params& p = H->p;
    cudaStream_t st = H->st;
    const int K = H->hctl->k;  // advances of the last solve
    const Ctl saved = *H->hctl;
    const double* alpha_dev = H->arr.alpha;  // the forward's step lengths
    auto& A = H->adj;
    CK(cudaMemcpyAsync(A.dbar, gbar, n * sizeof(double), cudaMemcpyDefault, st));
    launch_adj_lap(d, A.dbar, A.phibar, st);
    CK(cudaMemsetAsync(A.xib, 0, 3 * n * sizeof(double), st));
    CK(cudaMemsetAsync(A.wbar, 0, n * sizeof(double), st));
    std::swap(H->ctl, H->actl);
    std::swap(H->arr, H->aarr);
    SourceParams sp{p.xi_m, p.v_m, p.climiter};
    const double scale = fixed_scale((double)cells);
    int rc = RECON_OK;
    for (int k = K - 1; k >= 0 && !rc; --k) {
        const double* base = H->ckpt + (size_t)k * 5 * n;
        const double *phi_k = base, *ox = base + n, *oy = base + 2 * n, *oz = base + 3 * n;
        const double* pd = base + 4 * n;
        const double* alpha = alpha_dev + k;
        // step k's forward quantities: m_k (and a_k), e_k, dphi_k, V_k
        launch_deposit_tracers(d, ox, oy, oz, H->w, scale, H->mfix, st);
        launch_mass_coef(cells, H->mfix, 1.0 / scale, p.a_min, H->m, H->a64,
                         H->mixed ? H->c32[0] : nullptr, H->part[0], st);
        launch_geometry_source(d, sp, phi_k, H->m, H->t, H->e6, H->part[0], H->part[1], st);
        launch_smooth_S(d, p.s_side, pd, nullptr, H->dphi, nullptr, H->v3, nullptr, nullptr, st);
        launch_node_velocity(d, H->e6, H->dphi, H->v3, H->v3 + n, H->v3 + 2 * n, st);
        // back through the advance, V = e^-1 G and dphi = S phidot - mean
        CK(cudaMemsetAsync(A.vb, 0, 3 * n * sizeof(double), st));
        launch_adj_tracers(d, ox, oy, oz, H->v3, alpha, A.xib, A.vb, st);
        launch_adj_velocity(d, H->e6, H->v3, A.vb, A.gb, A.eb, st);
        launch_adj_dbar(d, alpha, A.phibar, A.gb, A.dbar, H->part[0], st);
        finish_reduce(H->part[0], 0, H->scal, SC_ADJ_A, st);
        launch_smooth_S(d, p.s_side, A.dbar, H->scal + SC_ADJ_A, H->s, nullptr, H->v3, nullptr,
                        H->part[2], st);
        finish_reduce(H->part[2], 0, H->scal, SC_SUM_S2, st);
        // the linear solve: the adjoint solve with the same operator
        rc = adjoint_mg(H);
        if (rc) break;
        // back through a = max(m, a_min), s = S t - mean, the source, the
        // Hessian and the deposit
        launch_adj_coef(d, H->phidot, pd, H->m, p.a_min, A.mbar, H->part[0], st);
        finish_reduce(H->part[0], 0, H->scal, SC_ADJ_B, st);
        launch_smooth_S(d, p.s_side, H->phidot, H->scal + SC_ADJ_B, H->t, nullptr, H->v3, nullptr,
                        nullptr, st);
        launch_adj_source(d, sp, H->e6, H->m, H->t, A.mbar, A.eb, st);
        launch_adj_hess(d, A.eb, A.phibar, st);
        launch_adj_deposit(d, ox, oy, oz, H->w, A.mbar, A.wbar, A.xib, st);
    }
    std::swap(H->ctl, H->actl);
    std::swap(H->arr, H->aarr);
    *H->hctl = saved;
    if (rc) return rc;
    // w = rho / mean(rho)
    launch_adj_dot(cells, A.wbar, H->w, H->part[0], st);
    finish_reduce(H->part[0], 0, H->scal, SC_ADJ_A, st);
    launch_adj_final(cells, A.wbar, H->scal + SC_ADJ_A, H->scal + SC_SUM_RHO, A.dbar, st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(grad, A.dbar, n * sizeof(double), cudaMemcpyDefault, st));
    // the mass and coefficient of the final map again (recon_field)
    deposit_step(H);
    CK(cudaStreamSynchronize(st));
    return RECON_OK;
}

// Memory a kernel on `device` may read directly: device memory of that device,
// or managed memory.  Host memory and other devices' memory are staged.
bool is_local_device_ptr(const void* p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace

namespace recon {
// Set the thread-local error text read by recon_last_error (used by entry
// points defined in other translation units); returns code.
int set_last_error(int code, const char* msg) {
    snprintf(g_err, sizeof(g_err), "%s", msg ? msg : "");
    return code;
}
}  // namespace recon

// RECON_CHECKED build: the first failed index check (its id) of any
// instrumented kernel since the last call, as a status; RECON_OK otherwise
// (always in the normal build).  The device has finished the work by then.
static int bounds_status() {
    int id = bounds_fail_smoother();
    if (!id) id = bounds_fail_transfer();
    if (!id) id = bounds_fail_cluster();
    if (!id) id = bounds_fail_steps();
    if (id) return fail(RECON_E_CUDA, "index bounds check %d failed (RECON_CHECKED build)", id);
    return RECON_OK;
}

extern "C" {

int recon_default_params(recon_params* p, int n0, int n1, int n2) {
    if (!p) return fail(RECON_E_INVALID, "params is NULL");
    std::memset(p, 0, sizeof(*p));
    p->n[0] = n0, p->n[1] = n1, p->n[2] = n2;
    p->precision = RECON_FP64;
    p->xi_m = 0.1;
    p->v_m = 10.0;
    p->a_min = 0.01;
    p->climiter = RECON_CLIM_SOFT;
    p->s_side = 0.25;
    p->nu1 = -1, p->nu2 = -1;  // by precision (resolve_params)
    p->tol_in = 1e-8;
    p->max_vcycles = -1;
    p->tol_out = 1e-3;
    p->k_max = 200;
    p->d_max = 0.5;
    p->alpha_min = std::ldexp(1.0, -20);
    p->lambda_floor = 0.01;
    p->replay_alpha = nullptr;
    p->profile = 0;
    p->inner_vcycles = -1;
    p->density_update = 0;
    p->device_loop = 1;
    p->checkpoint = 0;
    p->stream_planes = 0;
    p->restrict_planes = 0;
    p->coarse_faces = -1;
    p->tune_inner = 0;
    p->group_max = -1;
    p->tma = 1;
    p->warm_start = 2;
    return RECON_OK;
}

int recon_resolve_params(recon_params* p) {
    g_err[0] = 0;
    if (!p) return fail(RECON_E_INVALID, "params is NULL");
    resolve_params(p);
    return RECON_OK;
}

int recon_create(void** out, const recon_params* p_in, void* cuda_stream) {
    g_err[0] = 0;
    if (!out) return fail(RECON_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!p_in) return fail(RECON_E_INVALID, "params is NULL");
    recon_params resolved = *p_in;
    resolve_params(&resolved);
    const recon_params* p = &resolved;
    int rc = check_params(p);
    if (rc) return rc;
    Handle* H = new Handle();
    H->p = *p;
    if (p->replay_alpha) H->replay.assign(p->replay_alpha, p->replay_alpha + p->k_max);
    H->p.replay_alpha = nullptr;
    H->st = (cudaStream_t)cuda_stream;
    H->mixed = p->precision == RECON_MIXED;
    H->adaptive = H->mixed && p->group_max > p->inner_vcycles;
    cudaGetDevice(&H->device);
    H->d = make_dims(p->n[0], p->n[1], p->n[2]);
    H->cells = H->d.cells;
    H->h = (p->box[0] > 0.0) ? p->box[0] / p->n[0] : 1.0;
    // levels: halve every axis longer than 4 until all are 4
    {
        Level L{};
        L.d = H->d;
        for (int a = 0; a < 3; ++a) L.h2i[a] = 1.0;
        while (true) {
            int nn[3] = {L.d.n0, L.d.n1, L.d.n2};
            for (int a = 0; a < 3; ++a) L.coarsen[a] = nn[a] > 4;
            H->lv.push_back(L);
            if (!L.coarsen[0] && !L.coarsen[1] && !L.coarsen[2]) break;
            Level C{};
            int cn[3];
            for (int a = 0; a < 3; ++a) {
                cn[a] = L.coarsen[a] ? nn[a] / 2 : nn[a];
                C.h2i[a] = L.coarsen[a] ? L.h2i[a] * 0.25 : L.h2i[a];
            }
            C.d = make_dims(cn[0], cn[1], cn[2]);
            L = C;
        }
    }
    const size_t n = H->cells;
    const int nl = (int)H->lv.size();
#define AL(ptr, cnt)                          \
    do {                                      \
        if ((rc = dalloc(H, &(ptr), (cnt)))) { \
            free_all(H);                      \
            delete H;                         \
            return rc;                        \
        }                                     \
    } while (0)
    AL(H->rho, n); AL(H->w, n); AL(H->ox, n); AL(H->oy, n); AL(H->oz, n);
    AL(H->phi, n); AL(H->m, n); AL(H->a64, n); AL(H->t, n); AL(H->s, n);
    AL(H->phidot, n); AL(H->dphi, n); AL(H->v3, 3 * n); AL(H->mfix, n); AL(H->e6, 6 * n);
    AL(H->F64, 3 * n); AL(H->D64, n); AL(H->phi32, n); AL(H->dphi32, n);
    if (p->warm_start == 2) AL(H->phidot_prev, n);
    if (p->density_update == 1) AL(H->v3m, 6 * n);
    AL(H->minv, 65 * 130); AL(H->scal, SC_COUNT);
    const size_t km = (size_t)std::max(p->k_max, 1);
    // the per-step records share one block (Rk | alpha | relres | ncycles) so
    // that one copy brings them back
    AL(H->ctl, 1); AL(H->arr.Rk, 4 * km);
    H->arr.alpha = H->arr.Rk + km, H->arr.relres = H->arr.Rk + 2 * km;
    H->arr.ncycles = (int*)(H->arr.Rk + 3 * km);
    if (!H->replay.empty()) AL(H->replay_d, km);
    if (p->checkpoint) {
        AL(H->ckpt, 5 * n * km);
        AL(H->adj.phibar, n); AL(H->adj.xib, 3 * n); AL(H->adj.wbar, n); AL(H->adj.vb, 3 * n);
        AL(H->adj.gb, 3 * n); AL(H->adj.eb, 6 * n); AL(H->adj.dbar, n); AL(H->adj.mbar, n);
        AL(H->actl, 1); AL(H->aarr.Rk, 4);
        H->aarr.alpha = H->aarr.Rk + 1, H->aarr.relres = H->aarr.Rk + 2;
        H->aarr.ncycles = (int*)(H->aarr.Rk + 3);
    }
    for (int q = 0; q < 4; ++q) AL(H->part[q], kRedBlocks);
    if (!H->mixed) {
        H->u64.assign(nl, nullptr), H->f64.assign(nl, nullptr), H->c64.assign(nl, nullptr),
            H->r64.assign(nl, nullptr);
        H->u64[0] = H->phidot, H->f64[0] = H->s, H->c64[0] = H->a64;
        AL(H->r64[0], n);
        AL(H->inv64, n);
        for (int l = 1; l < nl; ++l) {
            size_t cl = H->lv[l].d.cells;
            AL(H->u64[l], cl); AL(H->f64[l], cl); AL(H->c64[l], cl); AL(H->r64[l], cl);
        }
    } else {
        H->u32.assign(nl, nullptr), H->f32.assign(nl, nullptr), H->c32.assign(nl, nullptr),
            H->r32.assign(nl, nullptr);
        // per-face coefficients on the coarse levels of a cubic grid
        const bool faces = p->coarse_faces == 1;
        for (int l = 1; l < nl; ++l) H->lv[l].face = faces ? 1 : 0;
        for (int l = 0; l < nl; ++l) H->lv[l].tma = p->tma;
        for (int l = 0; l < nl; ++l) {
            size_t cl = H->lv[l].d.cells;
            AL(H->u32[l], cl); AL(H->f32[l], cl); AL(H->c32[l], H->lv[l].face ? 3 * cl : cl);
            AL(H->r32[l], cl);
        }
    }
#undef AL
    // planes per block of the streaming FP32 kernels, measured per level on
    // the level's own buffers unless the parameters fix them (every choice
    // computes the same values; a fixed choice the level does not divide
    // falls back to the occupancy cost model at launch)
    if (H->mixed) {
        for (int l = 0; l + 1 < nl; ++l) {
            if (p->stream_planes)
                H->lv[l].tune[0] = H->lv[l].tune[1] = p->stream_planes;
            else
                tune_sweep_level(H->lv[l], &H->lv[l + 1], H->u32[l + 1], H->u32[l], H->r32[l],
                                 H->f32[l], H->c32[l], H->st);
            if (p->restrict_planes)
                H->lv[l].tune[2] = p->restrict_planes;
            else
                tune_resid_restrict_level(H->lv[l], H->lv[l + 1], H->u32[l], H->f32[l], H->c32[l],
                                          H->f32[l + 1], H->st);
        }
        if (cudaGetLastError() != cudaSuccess) {
            free_all(H);
            delete H;
            return fail(RECON_E_CUDA, "tuning the streaming kernels failed");
        }
    }
    // the levels from the first one of at most 16^3 nodes down run in one block
    for (int l = 0; l < nl; ++l)
        if (H->lv[l].d.cells <= 4096 && nl - l <= kCoarseMaxLevels && !H->lv[l].face) {
            H->l0 = l;
            break;
        }
    // a 32^3 level with 16^3, 8^3 and 4^3 below it runs in one cluster launch
    if (nl >= 4) {
        CoarseSet& cc = H->cc;
        cc.nlev = 4;
        cc.nu1 = p->nu1, cc.nu2 = p->nu2;
        for (int l = 0; l < 4; ++l) {
            cc.lv[l] = H->lv[nl - 4 + l];
            cc.a[l] = H->mixed ? (const void*)H->c32[nl - 4 + l] : (const void*)H->c64[nl - 4 + l];
        }
        // (not the finest FP64 level, which sweeps with its stored faces)
        if (coarse_cluster_fits(cc) && (H->mixed || nl > 4)) H->lc = nl - 4;
    }
    if (H->l0 >= 0) {
        H->cs.nlev = nl - H->l0;
        H->cs.nu1 = p->nu1, H->cs.nu2 = p->nu2;
        for (int l = H->l0; l < nl; ++l) {
            H->cs.lv[l - H->l0] = H->lv[l];
            H->cs.a[l - H->l0] = H->mixed ? (const void*)H->c32[l] : (const void*)H->c64[l];
        }
    }
    if (cudaMallocHost((void**)&H->hscal, SC_COUNT * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&H->hctl, sizeof(Ctl)) != cudaSuccess ||
        cudaMallocHost((void**)&H->harr, 4 * km * sizeof(double)) != cudaSuccess ||
        cudaEventCreate(&H->ev0) != cudaSuccess || cudaEventCreate(&H->ev1) != cudaSuccess) {
        cudaGetLastError();
        free_all(H);
        delete H;
        return fail(RECON_E_OOM, "pinned host buffer or event creation failed");
    }
    {
        int kmax = 0;
        while (kmax < 1100 && std::ldexp(1.0, -(kmax + 1)) >= p->alpha_min) ++kmax;
        H->lp = LimiterParams{p->lambda_floor, kmax};
    }
    std::memset(H->hctl, 0, sizeof(Ctl));
    cudaError_t e = cudaMemsetAsync(H->mfix, 0, n * sizeof(unsigned long long), H->st);
    if (e == cudaSuccess && H->replay_d)
        e = cudaMemcpyAsync(H->replay_d, H->replay.data(), H->replay.size() * sizeof(double),
                            cudaMemcpyHostToDevice, H->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(H->st);
    if (e != cudaSuccess) {
        free_all(H);
        delete H;
        return fail(RECON_E_CUDA, "initialisation failed: %s", cudaGetErrorString(e));
    }
    *out = H;
    return RECON_OK;
}

int recon_deposit(void* hp, int mode, const double* data, const double* mass, int64_t np) {
    g_err[0] = 0;
    Handle* H = (Handle*)hp;
    if (!H || !data) return fail(RECON_E_INVALID, "handle or data is NULL");
    const int n = H->cells;
    H->have_density = false;
    H->solved = false;
    if (mode == RECON_GRID) {
        if (mass) return fail(RECON_E_INVALID, "RECON_GRID takes no mass array");
        if (np != n) return fail(RECON_E_INVALID, "RECON_GRID needs np == cell count (%d)", n);
        CK(cudaMemcpyAsync(H->rho, data, sizeof(double) * n, cudaMemcpyDefault, H->st));
        launch_validate_grid(n, H->rho, H->part[0], H->part[1], H->st);
    } else if (mode == RECON_PARTICLES) {
        if (np <= 0) return fail(RECON_E_INVALID, "no particles");
        // host inputs (and another device's) are staged through a device
        // buffer the handle keeps (grown here when an input is larger; the
        // old one is released once the stream has finished with it)
        const double* dpos = data;
        const double* dmass = mass;
        bool host_pos = !is_local_device_ptr(data, H->device),
             host_mass = mass && !is_local_device_ptr(mass, H->device);
        size_t bytes = (host_pos ? 3 * sizeof(double) * np : 0) + (host_mass ? sizeof(double) * np : 0);
        if (bytes) {
            if (bytes > H->stage_bytes) {
                if (H->stage) {
                    CK(cudaStreamSynchronize(H->st));
                    cudaFree(H->stage);
                    H->stage = nullptr, H->stage_bytes = 0;
                }
                if (cudaMalloc(&H->stage, bytes) != cudaSuccess) {
                    cudaGetLastError();
                    H->stage = nullptr;
                    return fail(RECON_E_OOM, "staging buffer of %zu bytes failed", bytes);
                }
                H->stage_bytes = bytes;
            }
            char* q = (char*)H->stage;
            if (host_pos) {
                CK(cudaMemcpyAsync(q, data, 3 * sizeof(double) * np, cudaMemcpyDefault, H->st));
                dpos = (const double*)q;
                q += 3 * sizeof(double) * np;
            }
            if (host_mass) {
                CK(cudaMemcpyAsync(q, mass, sizeof(double) * np, cudaMemcpyDefault, H->st));
                dmass = (const double*)q;
            }
        }
        launch_validate_particles(np, dpos, dmass, H->part[0], H->part[1], H->st);
        finish_reduce(H->part[0], 0, H->scal, SC_SUM_RHO, H->st);
        finish_reduce(H->part[1], 2, H->scal, SC_BAD, H->st);
        int rc = sync_scalars(H);
        if (rc == RECON_OK && H->hscal[SC_BAD] != 0.0)
            rc = fail(RECON_E_NONFINITE, "particle positions or masses are not finite / negative");
        if (rc == RECON_OK && !(H->hscal[SC_SUM_RHO] > 0.0))
            rc = fail(RECON_E_INVALID, "total particle mass is zero");
        if (rc == RECON_OK) {
            const double scale = fixed_scale(H->hscal[SC_SUM_RHO]);
            launch_deposit_particles(H->d, np, dpos, dmass, 1.0 / H->h, scale, H->mfix, H->st);
            launch_fix_to_double(n, H->mfix, 1.0 / scale, H->rho, H->st);
            launch_validate_grid(n, H->rho, H->part[0], H->part[1], H->st);
        }
        if (rc) {
            cudaStreamSynchronize(H->st);
            return rc;
        }
    } else {
        return fail(RECON_E_INVALID, "unknown deposit mode %d", mode);
    }
    finish_reduce(H->part[0], 0, H->scal, SC_SUM_RHO, H->st);
    finish_reduce(H->part[1], 2, H->scal, SC_BAD, H->st);
    int rc = sync_scalars(H);
    if (rc) return rc;
    if (H->hscal[SC_BAD] != 0.0) return fail(RECON_E_NONFINITE, "density has NaN/Inf or negative values");
    if (!(H->hscal[SC_SUM_RHO] > 0.0)) return fail(RECON_E_INVALID, "total density is zero");
    H->rho_sum = H->hscal[SC_SUM_RHO];
    H->have_density = true;
    return RECON_OK;
}

int recon_solve(void* hp, recon_stats* stats) {
    g_err[0] = 0;
    Handle* H = (Handle*)hp;
    if (!H) return fail(RECON_E_INVALID, "handle is NULL");
    if (!H->have_density) return fail(RECON_E_STATE, "recon_deposit must succeed before recon_solve");
    int rc = H->inner_tuned ? RECON_OK : tune_inner_vcycles(H);
    if (rc == RECON_OK) rc = solve(H, stats);
    if (rc >= 0 && H->mixed && sweep_wait_failed())
        rc = fail(RECON_E_TIMEOUT, "a streaming sweep gave up waiting for a bulk copy");
    if (rc >= 0) {
        const int b = bounds_status();
        if (b) rc = b;
    }
    if (rc < 0) {
        cudaStreamSynchronize(H->st);
        H->solved = false;
        if (stats) stats->status = rc;
    }
    return rc;
}

int recon_solve_batch(void* const* handles, int count, recon_stats* stats) {
    g_err[0] = 0;
    Range range("recon_solve_batch");
    if (count < 0 || (count > 0 && !handles)) return fail(RECON_E_INVALID, "bad handle array");
    for (int b = 0; b < count; ++b) {
        Handle* H = (Handle*)handles[b];
        if (!H) return fail(RECON_E_INVALID, "handle %d is NULL", b);
        if (!H->have_density)
            return fail(RECON_E_STATE, "handle %d: recon_deposit must succeed before recon_solve", b);
        for (int c = 0; c < b; ++c)
            if (handles[c] == handles[b]) return fail(RECON_E_INVALID, "handle %d appears twice", b);
    }
    // every graph-mode solve is launched before any is waited for; solves on
    // distinct streams then run concurrently on the device
    std::vector<int> rc(count, RECON_OK);
    for (int b = 0; b < count; ++b) {
        Handle* H = (Handle*)handles[b];
        H->solved = false;
        if (!H->inner_tuned) rc[b] = tune_inner_vcycles(H);
    }
    for (int b = 0; b < count; ++b) {
        Handle* H = (Handle*)handles[b];
        if (rc[b] == RECON_OK && use_graph(H)) rc[b] = solve_launch(H, stats != nullptr);
    }
    int worst = RECON_OK;
    for (int b = 0; b < count; ++b) {
        Handle* H = (Handle*)handles[b];
        recon_stats* st = stats ? stats + b : nullptr;
        int r = rc[b];
        if (r == RECON_OK) r = use_graph(H) ? solve_finish(H, st) : solve(H, st);
        if (r < 0) {
            cudaStreamSynchronize(H->st);
            H->solved = false;
            if (st) st->status = r;
            if (worst >= 0) worst = r;
        }
    }
    if (worst >= 0 && sweep_wait_failed())
        worst = fail(RECON_E_TIMEOUT, "a streaming sweep gave up waiting for a bulk copy");
    if (worst >= 0) {
        const int b = bounds_status();
        if (b) worst = b;
    }
    return worst;
}

int recon_field(void* hp, int which, void* dst, size_t dst_bytes) {
    g_err[0] = 0;
    Handle* H = (Handle*)hp;
    if (!H || !dst) return fail(RECON_E_INVALID, "handle or dst is NULL");
    const size_t n = H->cells;
    const size_t need = (which == RECON_FIELD_MESH_X ? 3 : 1) * n * sizeof(double);
    if (dst_bytes < need) return fail(RECON_E_INVALID, "dst holds %zu bytes, need %zu", dst_bytes, need);
    if (which == RECON_FIELD_DENSITY) {
        if (!H->have_density) return fail(RECON_E_STATE, "no density deposited");
        CK(cudaMemcpyAsync(dst, H->rho, need, cudaMemcpyDefault, H->st));
        CK(cudaStreamSynchronize(H->st));
        return RECON_OK;
    }
    if (!H->solved) return fail(RECON_E_STATE, "no completed solve");
    const double* src = nullptr;
    switch (which) {
        case RECON_FIELD_PHI:
            launch_scale(H->cells, H->phi, H->h * H->h, H->t, H->st);
            src = H->t;
            break;
        case RECON_FIELD_DELTA_R:
            launch_delta_r(H->d, H->phi, H->t, H->part[0], H->st);
            src = H->t;
            break;
        case RECON_FIELD_MESH_X:
            launch_mesh_x(H->d, H->phi, H->h, H->v3, H->st);
            src = H->v3;
            break;
        case RECON_FIELD_MASS:
            src = H->m;
            break;
        case RECON_FIELD_DET:
            launch_geometry_out(H->d, H->phi, H->t, nullptr, H->part[0], H->part[1], H->st);
            src = H->t;
            break;
        case RECON_FIELD_LAMBDA0:
            launch_geometry_out(H->d, H->phi, nullptr, H->t, H->part[0], H->part[1], H->st);
            src = H->t;
            break;
        default:
            return fail(RECON_E_INVALID, "unknown field %d", which);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(dst, src, need, cudaMemcpyDefault, H->st));
    CK(cudaStreamSynchronize(H->st));
    return RECON_OK;
}

int recon_adjoint(void* hp, const double* grad_delta_r, double* grad_rho) {
    g_err[0] = 0;
    Handle* H = (Handle*)hp;
    if (!H || !grad_delta_r || !grad_rho) return fail(RECON_E_INVALID, "handle or buffer is NULL");
    if (!H->ckpt) return fail(RECON_E_STATE, "recon_adjoint needs params.checkpoint = 1 at create");
    if (!H->solved) return fail(RECON_E_STATE, "recon_adjoint needs a completed recon_solve");
    int rc = adjoint(H, grad_delta_r, grad_rho);
    if (rc) cudaStreamSynchronize(H->st);
    if (!rc) rc = bounds_status();
    return rc;
}

void recon_destroy(void* hp) {
    Handle* H = (Handle*)hp;
    if (!H) return;
    cudaStreamSynchronize(H->st);
    free_all(H);
    delete H;
}

const char* recon_last_error(void) { return g_err; }

}  // extern "C"
