/*
 * recon_oracle.c -- plain CPU FP64 oracle of the displacement-potential solve
 * of "Nonlinear reconstruction" (Zhu et al. 2016, arXiv:1611.09638).
 *
 * TEST INFRASTRUCTURE ONLY: the slow, obviously-correct reference the CUDA
 * library is checked against.  FP64, plain loops in ascending index order, no
 * blocking, no fusion.  Only tests, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code with the CUDA library.
 *
 * Threads: built with OpenMP, the loops whose iterations write disjoint
 * outputs and read nothing another iteration writes (stencils, one colour of
 * a red-black sweep, transfers, per-node geometry, per-tracer moves) are split
 * over threads by their outermost index (ORC_FOR_PLANES).  Every sum, and the
 * CIC scatter, stays one serial loop in ascending order, so the results are
 * bit for bit those of the single-threaded build for any thread count.
 *
 * The method, step by step (Sec. II moving-mesh iteration; App. A):
 *   init  rho_bar = mean(rho); tracer c has mass w_c = rho_c / rho_bar at
 *         curvilinear coordinate xi_c = c (its grid node); phi = 0.
 *   step  1. m = CIC deposit of the tracers (mass per curvilinear cell, the
 *            paper's rho sqrt(g); Sec. IV "displace ... then assign to a
 *            uniform grid").
 *         2. triad e = I + Hess(phi), sqrt_g = det e, lambda0 = min eig e
 *            (Eq. mapping; App. A).
 *         3. Sigma = 1 - m, limiters C(lambda0) and E(sqrt_g, Sigma), source
 *            s = S(Sigma + C + E) - mean (App. A, Eq. elliptic).
 *         4. R = rms(s); stop if R <= tol_out ("until the mass per volume
 *            element is approximately constant").
 *         5. with x ~ xi the operator is div(m grad .); a = max(m, a_min);
 *            solve L(a) phidot = s by multigrid V-cycles (App. A), starting
 *            from the last step's phidot (warm_start; the paper leaves the
 *            initial guess open) or from 0.
 *         6. dphi = S phidot (App. A, Delta phi = S phidot), mean removed.
 *         7. step limiter: largest alpha = 2^-k >= alpha_min keeping the
 *            smallest eigenvalue of I + Hess(phi + alpha dphi) above
 *            lambda_floor and the move below d_max cells (Sec. II: positive
 *            definiteness via smoothing and grid limiters); if there is none
 *            the iteration stops with the current map (stalled).
 *         8. phi += alpha dphi (phi = sum of the increments, Sec. II / App. A);
 *            the mesh moves by grad dphi in Eulerian space, so every tracer
 *            moves in xi by -alpha e^-1 grad dphi (Sec. IV "displace the
 *            particles by the negative displacement", with the triad e of
 *            the current map so that tracers stay on the mesh phi defines).
 *   out   delta_r = -Laplacian phi (Sec. II, Eq. rec); x = xi + grad phi.
 */
#include "recon_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#define ORC_FOR_PLANES _Pragma("omp parallel for schedule(static)")
#else
#define ORC_FOR_PLANES
#endif

#define ORC_E_INVALID (-1)
#define ORC_E_NOMEM (-2)
#define ORC_E_LIMITER (-5)

/* ------------------------------------------------------------------ grid */

static long wrapi(long i, long n) {
    long r = i % n;
    return r < 0 ? r + n : r;
}

static size_t at(const int n[3], long i, long j, long k) {
    return ((size_t)wrapi(i, n[0]) * (size_t)n[1] + (size_t)wrapi(j, n[1])) * (size_t)n[2] +
           (size_t)wrapi(k, n[2]);
}

static size_t ncells(const int n[3]) { return (size_t)n[0] * (size_t)n[1] * (size_t)n[2]; }

static int is_pow2_ge(int v, int lo) { return v >= lo && (v & (v - 1)) == 0; }

static int dims_ok(const int n[3], int lo) {
    return is_pow2_ge(n[0], lo) && is_pow2_ge(n[1], lo) && is_pow2_ge(n[2], lo);
}

/* ---------------------------------------------------------------- threads */

int orc_set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* ------------------------------------------------------------ CIC deposit */

/* Cloud-in-cell weights of a coordinate along one axis: node index i0 with
 * weight 1-f and node i0+1 with weight f, after periodic wrapping. */
static void cic_axis(double x, int n, long* i0, double* f) {
    double u = x - (double)n * floor(x / (double)n); /* into [0, n] */
    double fl = floor(u);
    *f = u - fl;
    long i = (long)fl;
    if (i >= n) i -= n;
    *i0 = i;
}

int orc_cic_deposit(const int n[3], const double* x, const double* w, int64_t np,
                    double* out) {
    if (!n || !dims_ok(n, 1) || (!x && np > 0) || !out || np < 0) return ORC_E_INVALID;
    memset(out, 0, ncells(n) * sizeof(double));
    for (int64_t p = 0; p < np; ++p) {
        long i0[3];
        double f[3];
        for (int a = 0; a < 3; ++a) cic_axis(x[3 * p + a], n[a], &i0[a], &f[a]);
        double wp = w ? w[p] : 1.0;
        for (int di = 0; di < 2; ++di)
            for (int dj = 0; dj < 2; ++dj)
                for (int dk = 0; dk < 2; ++dk) {
                    double wx = di ? f[0] : 1.0 - f[0];
                    double wy = dj ? f[1] : 1.0 - f[1];
                    double wz = dk ? f[2] : 1.0 - f[2];
                    out[at(n, i0[0] + di, i0[1] + dj, i0[2] + dk)] += wp * (wx * wy * wz);
                }
    }
    return 0;
}

/* ------------------------------------------------------------ operators */

int orc_apply_L(const int n[3], const double h[3], const double* a, const double* u,
                double* out) {
    if (!n || !h || !a || !u || !out) return ORC_E_INVALID;
    ORC_FOR_PLANES
    for (long i = 0; i < n[0]; ++i)
        for (long j = 0; j < n[1]; ++j)
            for (long k = 0; k < n[2]; ++k) {
                size_t c = at(n, i, j, k);
                double acc = 0.0;
                for (int ax = 0; ax < 3; ++ax) {
                    long di = ax == 0, dj = ax == 1, dk = ax == 2;
                    size_t pl = at(n, i + di, j + dj, k + dk);
                    size_t mi = at(n, i - di, j - dj, k - dk);
                    double ap = 0.5 * (a[c] + a[pl]);
                    double am = 0.5 * (a[c] + a[mi]);
                    acc += (ap * (u[pl] - u[c]) - am * (u[c] - u[mi])) / (h[ax] * h[ax]);
                }
                out[c] = acc;
            }
    return 0;
}

int orc_rbgs_sweep(const int n[3], const double h[3], const double* a, const double* f,
                   double* u) {
    if (!n || !h || !a || !f || !u) return ORC_E_INVALID;
    /* nodes of one colour read only nodes of the other colour (even dims,
     * periodic), so each colour's updates are independent of each other */
    for (int colour = 0; colour < 2; ++colour) {
        ORC_FOR_PLANES
        for (long i = 0; i < n[0]; ++i)
            for (long j = 0; j < n[1]; ++j)
                for (long k = 0; k < n[2]; ++k) {
                    if ((i + j + k) % 2 != colour) continue;
                    size_t c = at(n, i, j, k);
                    double diag = 0.0, off = 0.0;
                    for (int ax = 0; ax < 3; ++ax) {
                        long di = ax == 0, dj = ax == 1, dk = ax == 2;
                        size_t pl = at(n, i + di, j + dj, k + dk);
                        size_t mi = at(n, i - di, j - dj, k - dk);
                        double ap = 0.5 * (a[c] + a[pl]) / (h[ax] * h[ax]);
                        double am = 0.5 * (a[c] + a[mi]) / (h[ax] * h[ax]);
                        diag += ap + am;
                        off += ap * u[pl] + am * u[mi];
                    }
                    /* L u = off - diag u = f at this node */
                    u[c] = (off - f[c]) / diag;
                }
    }
    return 0;
}

static void coarse_dims(const int n[3], int nc[3]) {
    for (int a = 0; a < 3; ++a) nc[a] = n[a] > 4 ? n[a] / 2 : n[a];
}

int orc_restrict(const int n[3], const double* fine, double* coarse) {
    if (!n || !fine || !coarse) return ORC_E_INVALID;
    int nc[3];
    coarse_dims(n, nc);
    int cz[3] = {n[0] > 4, n[1] > 4, n[2] > 4};
    ORC_FOR_PLANES
    for (long I = 0; I < nc[0]; ++I)
        for (long J = 0; J < nc[1]; ++J)
            for (long K = 0; K < nc[2]; ++K) {
                double acc = 0.0;
                for (int oi = -cz[0]; oi <= cz[0]; ++oi)
                    for (int oj = -cz[1]; oj <= cz[1]; ++oj)
                        for (int ok = -cz[2]; ok <= cz[2]; ++ok) {
                            /* weights 1/4, 1/2, 1/4 along coarsened axes, 1 otherwise */
                            double wi = cz[0] ? (oi == 0 ? 0.5 : 0.25) : 1.0;
                            double wj = cz[1] ? (oj == 0 ? 0.5 : 0.25) : 1.0;
                            double wk = cz[2] ? (ok == 0 ? 0.5 : 0.25) : 1.0;
                            long fi = (cz[0] ? 2 * I : I) + oi;
                            long fj = (cz[1] ? 2 * J : J) + oj;
                            long fk = (cz[2] ? 2 * K : K) + ok;
                            acc += wi * wj * wk * fine[at(n, fi, fj, fk)];
                        }
                coarse[at(nc, I, J, K)] = acc;
            }
    return 0;
}

/* Linear interpolation stencil of fine index i along one axis: up to two
 * coarse indices with weights. */
static int prolong_axis(long i, int coarsened, long idx[2], double wt[2]) {
    if (!coarsened) {
        idx[0] = i;
        wt[0] = 1.0;
        return 1;
    }
    if (i % 2 == 0) {
        idx[0] = i / 2;
        wt[0] = 1.0;
        return 1;
    }
    idx[0] = (i - 1) / 2;
    idx[1] = (i + 1) / 2;
    wt[0] = wt[1] = 0.5;
    return 2;
}

int orc_prolong_add(const int n[3], const double* coarse, double* fine) {
    if (!n || !coarse || !fine) return ORC_E_INVALID;
    int nc[3];
    coarse_dims(n, nc);
    ORC_FOR_PLANES
    for (long i = 0; i < n[0]; ++i)
        for (long j = 0; j < n[1]; ++j)
            for (long k = 0; k < n[2]; ++k) {
                long ii[2], jj[2], kk[2];
                double wi[2], wj[2], wk[2];
                int ni = prolong_axis(i, n[0] > 4, ii, wi);
                int nj = prolong_axis(j, n[1] > 4, jj, wj);
                int nk = prolong_axis(k, n[2] > 4, kk, wk);
                double acc = 0.0;
                for (int p = 0; p < ni; ++p)
                    for (int q = 0; q < nj; ++q)
                        for (int r = 0; r < nk; ++r)
                            acc += wi[p] * wj[q] * wk[r] * coarse[at(nc, ii[p], jj[q], kk[r])];
                fine[at(n, i, j, k)] += acc;
            }
    return 0;
}

int orc_apply_S(const int n[3], double s_side, const double* u, double* out) {
    if (!n || !u || !out || u == out) return ORC_E_INVALID;
    /* weights (s_side, 1 - 2 s_side, s_side) along every axis: a weighted mean
     * over the 3x3x3 block of nearest neighbours */
    double w[3] = {s_side, 1.0 - 2.0 * s_side, s_side};
    ORC_FOR_PLANES
    for (long i = 0; i < n[0]; ++i)
        for (long j = 0; j < n[1]; ++j)
            for (long k = 0; k < n[2]; ++k) {
                double acc = 0.0;
                for (int oi = -1; oi <= 1; ++oi)
                    for (int oj = -1; oj <= 1; ++oj)
                        for (int ok = -1; ok <= 1; ++ok)
                            acc += w[oi + 1] * w[oj + 1] * w[ok + 1] * u[at(n, i + oi, j + oj, k + ok)];
                out[at(n, i, j, k)] = acc;
            }
    return 0;
}

/* -------------------------------------------------------------- multigrid */

#define ORC_MAX_LEVELS 32

typedef struct {
    int nlev;
    int n[ORC_MAX_LEVELS][3];
    double h[ORC_MAX_LEVELS][3];
    double* a[ORC_MAX_LEVELS]; /* coefficient per level, a[0] borrowed */
} orc_hier;

static double norm2(const double* v, size_t len) {
    double s = 0.0;
    for (size_t i = 0; i < len; ++i) s += v[i] * v[i];
    return sqrt(s);
}

static double mean(const double* v, size_t len) {
    double s = 0.0;
    for (size_t i = 0; i < len; ++i) s += v[i];
    return s / (double)len;
}

/* Levels: each axis longer than 4 is halved (spacing doubled) until every
 * axis is 4; the coefficient is carried down by full weighting. */
static int hier_build(const int n[3], const double* a0, orc_hier* H) {
    memset(H, 0, sizeof(*H));
    int l = 0;
    for (int ax = 0; ax < 3; ++ax) {
        H->n[0][ax] = n[ax];
        H->h[0][ax] = 1.0;
    }
    H->a[0] = (double*)a0;
    while (H->n[l][0] > 4 || H->n[l][1] > 4 || H->n[l][2] > 4) {
        if (l + 1 >= ORC_MAX_LEVELS) return ORC_E_INVALID;
        for (int ax = 0; ax < 3; ++ax) {
            int c = H->n[l][ax] > 4;
            H->n[l + 1][ax] = c ? H->n[l][ax] / 2 : H->n[l][ax];
            H->h[l + 1][ax] = c ? 2.0 * H->h[l][ax] : H->h[l][ax];
        }
        H->a[l + 1] = (double*)malloc(ncells(H->n[l + 1]) * sizeof(double));
        if (!H->a[l + 1]) return ORC_E_NOMEM;
        orc_restrict(H->n[l], H->a[l], H->a[l + 1]);
        ++l;
    }
    H->nlev = l + 1;
    return 0;
}

static void hier_free(orc_hier* H) {
    for (int l = 1; l < H->nlev; ++l) free(H->a[l]);
    /* partially built levels */
    for (int l = H->nlev > 0 ? H->nlev : 1; l < ORC_MAX_LEVELS; ++l)
        if (H->a[l]) free(H->a[l]);
}

/* Coarsest level: dense solve of [L 1; 1^T 0][u; mu] = [f; 0] by Gaussian
 * elimination with partial pivoting (u has mean zero, L u = f - mean f). */
static int coarse_solve(const int n[3], const double h[3], const double* a, const double* f,
                        double* u) {
    size_t nc = ncells(n), m = nc + 1;
    double* M = (double*)calloc(m * m, sizeof(double));
    double* rhs = (double*)calloc(m, sizeof(double));
    double* e = (double*)calloc(nc, sizeof(double));
    double* col = (double*)calloc(nc, sizeof(double));
    if (!M || !rhs || !e || !col) {
        free(M), free(rhs), free(e), free(col);
        return ORC_E_NOMEM;
    }
    for (size_t c = 0; c < nc; ++c) {
        memset(e, 0, nc * sizeof(double));
        e[c] = 1.0;
        orc_apply_L(n, h, a, e, col);
        for (size_t r = 0; r < nc; ++r) M[r * m + c] = col[r];
    }
    for (size_t r = 0; r < nc; ++r) {
        M[r * m + nc] = 1.0;
        M[nc * m + r] = 1.0;
        rhs[r] = f[r];
    }
    for (size_t p = 0; p < m; ++p) {
        size_t piv = p;
        for (size_t r = p + 1; r < m; ++r)
            if (fabs(M[r * m + p]) > fabs(M[piv * m + p])) piv = r;
        if (piv != p) {
            for (size_t c = 0; c < m; ++c) {
                double t = M[p * m + c];
                M[p * m + c] = M[piv * m + c];
                M[piv * m + c] = t;
            }
            double t = rhs[p];
            rhs[p] = rhs[piv];
            rhs[piv] = t;
        }
        for (size_t r = p + 1; r < m; ++r) {
            double fct = M[r * m + p] / M[p * m + p];
            if (fct == 0.0) continue;
            for (size_t c = p; c < m; ++c) M[r * m + c] -= fct * M[p * m + c];
            rhs[r] -= fct * rhs[p];
        }
    }
    for (size_t p = m; p-- > 0;) {
        double s = rhs[p];
        for (size_t c = p + 1; c < m; ++c) s -= M[p * m + c] * rhs[c];
        rhs[p] = s / M[p * m + p];
    }
    for (size_t r = 0; r < nc; ++r) u[r] = rhs[r];
    free(M), free(rhs), free(e), free(col);
    return 0;
}

static int vcycle_level(const orc_params* p, const orc_hier* H, int l, const double* f,
                        double* u) {
    const int* n = H->n[l];
    const double* h = H->h[l];
    if (l == H->nlev - 1) return coarse_solve(n, h, H->a[l], f, u);
    size_t len = ncells(n);
    for (int s = 0; s < p->nu1; ++s) orc_rbgs_sweep(n, h, H->a[l], f, u);
    double* r = (double*)malloc(len * sizeof(double));
    size_t clen = ncells(H->n[l + 1]);
    double* fc = (double*)malloc(clen * sizeof(double));
    double* uc = (double*)calloc(clen, sizeof(double));
    if (!r || !fc || !uc) {
        free(r), free(fc), free(uc);
        return ORC_E_NOMEM;
    }
    orc_apply_L(n, h, H->a[l], u, r);
    for (size_t i = 0; i < len; ++i) r[i] = f[i] - r[i];
    orc_restrict(n, r, fc);
    int rc = vcycle_level(p, H, l + 1, fc, uc);
    if (rc == 0) {
        orc_prolong_add(n, uc, u);
        for (int s = 0; s < p->nu2; ++s) orc_rbgs_sweep(n, h, H->a[l], f, u);
    }
    free(r), free(fc), free(uc);
    return rc;
}

int orc_vcycle(const orc_params* p, const double* a, const double* f, double* u) {
    if (!p || !a || !f || !u || !dims_ok(p->n, 4)) return ORC_E_INVALID;
    orc_hier H;
    int rc = hier_build(p->n, a, &H);
    if (rc == 0) rc = vcycle_level(p, &H, 0, f, u);
    hier_free(&H);
    return rc;
}

int orc_mg_solve(const orc_params* p, const double* a, const double* s, double* u,
                 int* ncycles, double* relres) {
    if (!p || !a || !s || !u || !dims_ok(p->n, 4)) return ORC_E_INVALID;
    memset(u, 0, ncells(p->n) * sizeof(double));
    return orc_mg_solve_from(p, a, s, u, ncycles, relres);
}

int orc_mg_solve_from(const orc_params* p, const double* a, const double* s, double* u,
                      int* ncycles, double* relres) {
    if (!p || !a || !s || !u || !dims_ok(p->n, 4)) return ORC_E_INVALID;
    size_t len = ncells(p->n);
    double snorm = norm2(s, len);
    int cyc = 0;
    double rel = 0.0;
    if (snorm > 0.0) {
        orc_hier H;
        int rc = hier_build(p->n, a, &H);
        double* r = (double*)malloc(len * sizeof(double));
        if (rc != 0 || !r) {
            hier_free(&H);
            free(r);
            return rc ? rc : ORC_E_NOMEM;
        }
        const double h1[3] = {1.0, 1.0, 1.0};
        rel = 1.0;
        while (cyc < p->max_vcycles) {
            rc = vcycle_level(p, &H, 0, s, u);
            if (rc) break;
            ++cyc;
            orc_apply_L(p->n, h1, a, u, r);
            for (size_t i = 0; i < len; ++i) r[i] = s[i] - r[i];
            rel = norm2(r, len) / snorm;
            if (rel <= p->tol_in) break;
        }
        hier_free(&H);
        free(r);
        if (rc) return rc;
    }
    if (ncycles) *ncycles = cyc;
    if (relres) *relres = rel;
    return 0;
}

/* --------------------------------------------------------------- geometry */

/* Hessian of phi at node (i,j,k): 3-point second differences on the
 * diagonal, 4-point centred cross differences off it. */
static void hessian(const int n[3], const double* f, long i, long j, long k, double H[3][3]) {
    long o[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    double c = f[at(n, i, j, k)];
    for (int a = 0; a < 3; ++a) {
        H[a][a] = f[at(n, i + o[a][0], j + o[a][1], k + o[a][2])] - 2.0 * c +
                  f[at(n, i - o[a][0], j - o[a][1], k - o[a][2])];
        for (int b = a + 1; b < 3; ++b) {
            long pi = o[a][0] + o[b][0], pj = o[a][1] + o[b][1], pk = o[a][2] + o[b][2];
            long qi = o[a][0] - o[b][0], qj = o[a][1] - o[b][1], qk = o[a][2] - o[b][2];
            double v = f[at(n, i + pi, j + pj, k + pk)] - f[at(n, i + qi, j + qj, k + qk)] -
                       f[at(n, i - qi, j - qj, k - qk)] + f[at(n, i - pi, j - pj, k - pk)];
            H[a][b] = H[b][a] = 0.25 * v;
        }
    }
}

static double det3(const double e[3][3]) {
    return e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
           e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
           e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
}

double orc_min_eig_sym3(const double A[3][3]) {
    double m[3][3];
    memcpy(m, A, sizeof(m));
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = m[0][1] * m[0][1] + m[0][2] * m[0][2] + m[1][2] * m[1][2];
        if (off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (m[p][q] == 0.0) continue;
                /* rotation angle zeroing m[p][q] */
                double theta = (m[q][q] - m[p][p]) / (2.0 * m[p][q]);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < 3; ++r) { /* columns p, q */
                    double mrp = m[r][p], mrq = m[r][q];
                    m[r][p] = c * mrp - s * mrq;
                    m[r][q] = s * mrp + c * mrq;
                }
                for (int r = 0; r < 3; ++r) { /* rows p, q */
                    double mpr = m[p][r], mqr = m[q][r];
                    m[p][r] = c * mpr - s * mqr;
                    m[q][r] = s * mpr + c * mqr;
                }
                m[p][q] = m[q][p] = 0.0;
            }
    }
    double l = m[0][0];
    if (m[1][1] < l) l = m[1][1];
    if (m[2][2] < l) l = m[2][2];
    return l;
}

int orc_geometry(const int n[3], const double* phi, double* sqrt_g, double* lambda0) {
    if (!n || !phi || !dims_ok(n, 1)) return ORC_E_INVALID;
    ORC_FOR_PLANES
    for (long i = 0; i < n[0]; ++i)
        for (long j = 0; j < n[1]; ++j)
            for (long k = 0; k < n[2]; ++k) {
                double H[3][3], e[3][3];
                hessian(n, phi, i, j, k, H);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) e[a][b] = (a == b ? 1.0 : 0.0) + H[a][b];
                size_t c = at(n, i, j, k);
                if (sqrt_g) sqrt_g[c] = det3(e);
                if (lambda0) lambda0[c] = orc_min_eig_sym3(e);
            }
    return 0;
}

static double heaviside(double x) { return x > 0.0 ? 1.0 : 0.0; }

/* Compression limiter C(lambda0) of App. A under the chosen reading. */
static double climit(int reading, double xi_m, double lambda0) {
    double lam = lambda0 > 1e-12 ? lambda0 : 1e-12;
    double q = xi_m / lam;
    double v;
    switch (reading) {
        case ORC_CLIM_LITERAL: v = q - heaviside(q - 1.0); break;
        case ORC_CLIM_STEP: v = q * heaviside(q - 1.0); break;
        default: v = q - 1.0 > 0.0 ? q - 1.0 : 0.0; break;
    }
    return 4.0 * v * v;
}

int orc_source(const orc_params* p, const double* phi, const double* m, double* s,
               double* t_out) {
    if (!p || !phi || !m || !s || !dims_ok(p->n, 1)) return ORC_E_INVALID;
    const int* n = p->n;
    size_t len = ncells(n);
    double* g = (double*)malloc(len * sizeof(double));
    double* lam = (double*)malloc(len * sizeof(double));
    double* t = (double*)malloc(len * sizeof(double));
    if (!g || !lam || !t) {
        free(g), free(lam), free(t);
        return ORC_E_NOMEM;
    }
    orc_geometry(n, phi, g, lam);
    ORC_FOR_PLANES
    for (size_t c = 0; c < len; ++c) {
        double Sigma = 1.0 - m[c];                          /* deviation density */
        double C = climit(p->climiter, p->xi_m, lam[c]);    /* compression limiter */
        double E = -2.0 * heaviside(g[c] - p->v_m) * fabs(Sigma); /* expansion limiter */
        t[c] = Sigma + C + E;
    }
    orc_apply_S(n, p->s_side, t, s);
    double mu = mean(s, len);
    for (size_t c = 0; c < len; ++c) s[c] -= mu;
    if (t_out) memcpy(t_out, t, len * sizeof(double));
    free(g), free(lam), free(t);
    return 0;
}

/* ------------------------------------------------------------ limiter */

/* lambda_min(M) > floor  <=>  M - floor I positive definite (Sylvester's
 * criterion: all leading principal minors positive). */
static int pd_sylvester(const double M0[3][3], double floor) {
    double M[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) M[a][b] = M0[a][b] - (a == b ? floor : 0.0);
    double m1 = M[0][0];
    double m2 = M[0][0] * M[1][1] - M[0][1] * M[1][0];
    double m3 = det3(M);
    return m1 > 0.0 && m2 > 0.0 && m3 > 0.0;
}

/* central-difference gradient component ax of f at a node */
static double cgrad(const int n[3], const double* f, long i, long j, long k, int ax) {
    long di = ax == 0, dj = ax == 1, dk = ax == 2;
    return 0.5 * (f[at(n, i + di, j + dj, k + dk)] - f[at(n, i - di, j - dj, k - dk)]);
}

int orc_step_limiter(const orc_params* p, const double* phi, const double* dphi,
                     double* alpha) {
    if (!p || !phi || !dphi || !alpha || !dims_ok(p->n, 1)) return ORC_E_INVALID;
    const int* n = p->n;
    /* per-plane results (max |grad dphi|, "every node admissible"), combined
     * after the plane loop: a max and an AND do not depend on the order */
    double* gplane = (double*)malloc((size_t)n[0] * sizeof(double));
    int* okplane = (int*)malloc((size_t)n[0] * sizeof(int));
    if (!gplane || !okplane) {
        free(gplane), free(okplane);
        return ORC_E_NOMEM;
    }
    ORC_FOR_PLANES
    for (long i = 0; i < n[0]; ++i) {
        double gm = 0.0;
        for (long j = 0; j < n[1]; ++j)
            for (long k = 0; k < n[2]; ++k)
                for (int ax = 0; ax < 3; ++ax) {
                    double g = fabs(cgrad(n, dphi, i, j, k, ax));
                    if (g > gm) gm = g;
                }
        gplane[i] = gm;
    }
    double gmax = 0.0;
    for (long i = 0; i < n[0]; ++i)
        if (gplane[i] > gmax) gmax = gplane[i];
    int rc = ORC_E_LIMITER;
    for (double al = 1.0; al >= p->alpha_min; al *= 0.5) {
        if (!(al * gmax <= p->d_max)) continue;
        ORC_FOR_PLANES
        for (long i = 0; i < n[0]; ++i) {
            int ok = 1;
            for (long j = 0; ok && j < n[1]; ++j)
                for (long k = 0; ok && k < n[2]; ++k) {
                    double H0[3][3], H1[3][3], M[3][3];
                    hessian(n, phi, i, j, k, H0);
                    hessian(n, dphi, i, j, k, H1);
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b)
                            M[a][b] = (a == b ? 1.0 : 0.0) + H0[a][b] + al * H1[a][b];
                    ok = pd_sylvester(M, p->lambda_floor);
                }
            okplane[i] = ok;
        }
        int ok = 1;
        for (long i = 0; i < n[0]; ++i) ok = ok && okplane[i];
        if (ok) {
            *alpha = al;
            rc = 0;
            break;
        }
    }
    free(gplane), free(okplane);
    return rc;
}

/* -------------------------------------------------------------- advance */

int orc_advance(const int n[3], double alpha, const double* dphi, double* phi, double* xi,
                int64_t np) {
    if (!n || !dphi || !phi || (!xi && np > 0) || !dims_ok(n, 1)) return ORC_E_INVALID;
    size_t len = ncells(n);
    /* Node velocity of a tracer's curvilinear coordinate: the mesh point xi
     * moves by grad dphi in Eulerian space (Eq. mapping), so a tracer at rest
     * in x moves in xi by -e^-1 grad dphi, e = I + Hess(phi) the current
     * triad (App. A).  V = e^-1 G at every node, G the central-difference
     * gradient of dphi; phi is read before its own update. */
    double* V = (double*)malloc(3 * len * sizeof(double));
    if (!V) return ORC_E_NOMEM;
    ORC_FOR_PLANES
    for (long i = 0; i < n[0]; ++i)
        for (long j = 0; j < n[1]; ++j)
            for (long k = 0; k < n[2]; ++k) {
                double H[3][3], e[3][3], G[3];
                hessian(n, phi, i, j, k, H);
                for (int a = 0; a < 3; ++a) {
                    for (int b = 0; b < 3; ++b) e[a][b] = (a == b ? 1.0 : 0.0) + H[a][b];
                    G[a] = cgrad(n, dphi, i, j, k, a);
                }
                /* e^-1 G by Cramer's rule (e symmetric positive definite) */
                double d = det3(e);
                size_t c = at(n, i, j, k);
                for (int a = 0; a < 3; ++a) {
                    double ea[3][3];
                    memcpy(ea, e, sizeof(ea));
                    for (int r = 0; r < 3; ++r) ea[r][a] = G[r];
                    V[3 * c + a] = det3(ea) / d;
                }
            }
    for (size_t c = 0; c < len; ++c) phi[c] += alpha * dphi[c];
    ORC_FOR_PLANES
    for (int64_t t = 0; t < np; ++t) {
        long i0[3];
        double f[3], v[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < 3; ++a) cic_axis(xi[3 * t + a], n[a], &i0[a], &f[a]);
        for (int di = 0; di < 2; ++di)
            for (int dj = 0; dj < 2; ++dj)
                for (int dk = 0; dk < 2; ++dk) {
                    double w = (di ? f[0] : 1.0 - f[0]) * (dj ? f[1] : 1.0 - f[1]) *
                               (dk ? f[2] : 1.0 - f[2]);
                    size_t c = at(n, i0[0] + di, i0[1] + dj, i0[2] + dk);
                    for (int a = 0; a < 3; ++a) v[a] += w * V[3 * c + a];
                }
        for (int a = 0; a < 3; ++a) xi[3 * t + a] -= alpha * v[a];
    }
    free(V);
    return 0;
}

/* ------------------------------------------------ paper-literal update */

int orc_mass_change(const int n[3], const double* phi, const double* m, const double* v,
                    double* out) {
    if (!n || !phi || !m || !v || !out || !dims_ok(n, 1)) return ORC_E_INVALID;
    size_t len = ncells(n);
    double* K = (double*)malloc(9 * len * sizeof(double));
    if (!K) return ORC_E_NOMEM;
    /* K = m e^-1 at every node, the inverse by cofactors / det */
    for (long i = 0; i < n[0]; ++i)
        for (long j = 0; j < n[1]; ++j)
            for (long k = 0; k < n[2]; ++k) {
                double H[3][3], e[3][3];
                hessian(n, phi, i, j, k, H);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) e[a][b] = (a == b ? 1.0 : 0.0) + H[a][b];
                double det = det3(e);
                size_t c = at(n, i, j, k);
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        /* cofactor of e[b][a] (adjugate = transpose of cofactors) */
                        int r0 = b == 0 ? 1 : 0, r1 = b == 2 ? 1 : 2;
                        int c0 = a == 0 ? 1 : 0, c1 = a == 2 ? 1 : 2;
                        double cof = e[r0][c0] * e[r1][c1] - e[r0][c1] * e[r1][c0];
                        if ((a + b) % 2) cof = -cof;
                        K[9 * c + 3 * a + b] = m[c] * cof / det;
                    }
            }
    for (long i = 0; i < n[0]; ++i)
        for (long j = 0; j < n[1]; ++j)
            for (long k = 0; k < n[2]; ++k) {
                long o[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
                size_t c = at(n, i, j, k);
                double acc = 0.0;
                for (int a = 0; a < 3; ++a) {
                    size_t pl = at(n, i + o[a][0], j + o[a][1], k + o[a][2]);
                    size_t mi = at(n, i - o[a][0], j - o[a][1], k - o[a][2]);
                    double kp = 0.5 * (K[9 * c + 4 * a] + K[9 * pl + 4 * a]);
                    double km = 0.5 * (K[9 * c + 4 * a] + K[9 * mi + 4 * a]);
                    acc += kp * (v[pl] - v[c]) - km * (v[c] - v[mi]);
                    for (int b = 0; b < 3; ++b) {
                        if (b == a) continue;
                        long pi = i + o[a][0], pj = j + o[a][1], pk = k + o[a][2];
                        long qi = i - o[a][0], qj = j - o[a][1], qk = k - o[a][2];
                        double dp = v[at(n, pi + o[b][0], pj + o[b][1], pk + o[b][2])] -
                                    v[at(n, pi - o[b][0], pj - o[b][1], pk - o[b][2])];
                        double dm = v[at(n, qi + o[b][0], qj + o[b][1], qk + o[b][2])] -
                                    v[at(n, qi - o[b][0], qj - o[b][1], qk - o[b][2])];
                        acc += 0.25 * (K[9 * pl + 3 * a + b] * dp - K[9 * mi + 3 * a + b] * dm);
                    }
                }
                out[c] = acc;
            }
    free(K);
    return 0;
}

/* ---------------------------------------------------------------- outputs */

int orc_delta_r(const int n[3], const double* phi, double* out) {
    if (!n || !phi || !out || !dims_ok(n, 1)) return ORC_E_INVALID;
    ORC_FOR_PLANES
    for (long i = 0; i < n[0]; ++i)
        for (long j = 0; j < n[1]; ++j)
            for (long k = 0; k < n[2]; ++k) {
                double H[3][3];
                hessian(n, phi, i, j, k, H);
                out[at(n, i, j, k)] = -(H[0][0] + H[1][1] + H[2][2]);
            }
    return 0;
}

int orc_mesh_x(const int n[3], const double* phi, double* out) {
    if (!n || !phi || !out || !dims_ok(n, 1)) return ORC_E_INVALID;
    ORC_FOR_PLANES
    for (long i = 0; i < n[0]; ++i)
        for (long j = 0; j < n[1]; ++j)
            for (long k = 0; k < n[2]; ++k) {
                size_t c = at(n, i, j, k);
                out[3 * c + 0] = (double)i + cgrad(n, phi, i, j, k, 0);
                out[3 * c + 1] = (double)j + cgrad(n, phi, i, j, k, 1);
                out[3 * c + 2] = (double)k + cgrad(n, phi, i, j, k, 2);
            }
    return 0;
}

/* ------------------------------------------------------------ whole solve */

static int params_ok(const orc_params* p) {
    return p && dims_ok(p->n, 8) && p->xi_m > 0.0 && p->xi_m < 1.0 && p->v_m > 1.0 &&
           p->a_min > 0.0 && p->s_side >= 0.0 && p->s_side <= 0.25 && p->nu1 >= 0 && p->nu2 >= 0 && p->nu1 + p->nu2 > 0 &&
           p->tol_in > 0.0 && p->max_vcycles > 0 && p->tol_out >= 0.0 && p->k_max >= 0 &&
           p->d_max > 0.0 && p->alpha_min > 0.0 && p->alpha_min <= 1.0 &&
           p->lambda_floor >= 0.0 && p->lambda_floor < 1.0 &&
           (p->density_update == 0 || p->density_update == 1) &&
           p->warm_start >= 0 && p->warm_start <= 2;
}

/* Initial guess of step k's linear solve under warm_start = 2: u holds
 * phidot_{k-1}, prev phidot_{k-2}; u becomes phidot_{k-1} + (alpha_{k-1} /
 * alpha_{k-2}) (phidot_{k-1} - phidot_{k-2}), a linear extrapolation along
 * the step lengths that moved the mesh, and prev phidot_{k-1}.  Step 1 only
 * keeps phidot_0 in prev. */
static void warm_extrapolate(size_t len, int k, const double* alpha, double* u, double* prev) {
    if (k < 1) return;
    const double r = k >= 2 ? alpha[k - 1] / alpha[k - 2] : 0.0;
    for (size_t c = 0; c < len; ++c) {
        const double cur = u[c];
        if (k >= 2) u[c] = cur + r * (cur - prev[c]);
        prev[c] = cur;
    }
}

int orc_solve(const orc_params* p, const double* rho, const double* replay_alpha,
              double* phi, double* xi_out, double* m_out, int* steps, orc_trace* tr) {
    if (!params_ok(p) || !rho || !phi) return ORC_E_INVALID;
    const int* n = p->n;
    size_t len = ncells(n);
    double rho_sum = 0.0;
    for (size_t c = 0; c < len; ++c) {
        if (!(rho[c] >= 0.0) || !isfinite(rho[c])) return ORC_E_INVALID;
        rho_sum += rho[c];
    }
    if (!(rho_sum > 0.0)) return ORC_E_INVALID;
    double rho_bar = rho_sum / (double)len;

    double* w = (double*)malloc(len * sizeof(double));
    double* xi = (double*)malloc(3 * len * sizeof(double));
    double* m = (double*)malloc(len * sizeof(double));
    double* s = (double*)malloc(len * sizeof(double));
    double* a = (double*)malloc(len * sizeof(double));
    double* phidot = (double*)malloc(len * sizeof(double));
    double* dphi = (double*)malloc(len * sizeof(double));
    double* g = (double*)malloc(len * sizeof(double));
    double* lam = (double*)malloc(len * sizeof(double));
    double* dm = NULL; /* mass change of the App. A update (density_update = 1) */
    double* prev = NULL;   /* warm_start = 2: phidot of the step before the last */
    double* alphas = NULL; /* warm_start = 2: the accepted step lengths */
    int rc = 0, k = 0, done = 0, stalled = 0;
    if (!w || !xi || !m || !s || !a || !phidot || !dphi || !g || !lam) {
        rc = ORC_E_NOMEM;
        goto out;
    }
    memset(phidot, 0, len * sizeof(double));
    if (p->warm_start == 2) {
        prev = (double*)malloc(len * sizeof(double));
        alphas = (double*)malloc((size_t)(p->k_max > 0 ? p->k_max : 1) * sizeof(double));
        if (!prev || !alphas) {
            rc = ORC_E_NOMEM;
            goto out;
        }
    }
    /* init: tracer c = node c with mass rho_c / rho_bar; phi = 0 */
    for (long i = 0; i < n[0]; ++i)
        for (long j = 0; j < n[1]; ++j)
            for (long kk = 0; kk < n[2]; ++kk) {
                size_t c = at(n, i, j, kk);
                w[c] = rho[c] / rho_bar;
                xi[3 * c + 0] = (double)i;
                xi[3 * c + 1] = (double)j;
                xi[3 * c + 2] = (double)kk;
            }
    memset(phi, 0, len * sizeof(double));

    if (p->density_update == 1) {
        /* App. A: the mass per cell starts as the density on the undeformed
         * mesh and is carried by its exact linear change each step */
        dm = (double*)malloc(len * sizeof(double));
        if (!dm) {
            rc = ORC_E_NOMEM;
            goto out;
        }
        memcpy(m, w, len * sizeof(double));
    }
    for (k = 0; k < p->k_max; ++k) {
        if (p->density_update == 0) orc_cic_deposit(n, xi, w, (int64_t)len, m); /* 1 */
        rc = orc_source(p, phi, m, s, NULL);                      /* 2, 3 */
        if (rc) goto out;
        double R = 0.0;
        for (size_t c = 0; c < len; ++c) R += s[c] * s[c];
        R = sqrt(R / (double)len);                                /* 4 */
        if (tr) {
            orc_geometry(n, phi, g, lam);
            double md = g[0], ml = lam[0], ms = 0.0;
            for (size_t c = 0; c < len; ++c) {
                if (g[c] < md) md = g[c];
                if (lam[c] < ml) ml = lam[c];
                ms += m[c];
            }
            if (tr->R) tr->R[k] = R;
            if (tr->min_det) tr->min_det[k] = md;
            if (tr->min_lam) tr->min_lam[k] = ml;
            if (tr->mass) tr->mass[k] = ms;
        }
        if (R <= p->tol_out) {
            done = 1;
            break;
        }
        for (size_t c = 0; c < len; ++c) a[c] = m[c] > p->a_min ? m[c] : p->a_min; /* 5 */
        int ncyc = 0;
        double rel = 0.0;
        /* the linear solve starts from the last step's phidot (warm_start 1;
         * phidot = 0 before the first step), its extrapolation from the last
         * two (2) or from 0 */
        if (p->warm_start == 2) warm_extrapolate(len, k, alphas, phidot, prev);
        rc = p->warm_start ? orc_mg_solve_from(p, a, s, phidot, &ncyc, &rel)
                           : orc_mg_solve(p, a, s, phidot, &ncyc, &rel);
        if (rc) goto out;
        orc_apply_S(n, p->s_side, phidot, dphi);     /* 6 */
        double mu = mean(dphi, len);
        for (size_t c = 0; c < len; ++c) dphi[c] -= mu;
        double alpha;                                             /* 7 */
        if (replay_alpha) {
            alpha = replay_alpha[k];
        } else {
            rc = orc_step_limiter(p, phi, dphi, &alpha);
            if (rc == ORC_E_LIMITER) {
                /* no admissible step: stop with the current (valid) map */
                rc = 0;
                stalled = 1;
                break;
            }
            if (rc) goto out;
        }
        if (p->density_update == 1) {
            /* m' = m + alpha D(dphi) with the triad of the current map */
            rc = orc_mass_change(n, phi, m, dphi, dm);
            if (rc) goto out;
            for (size_t c = 0; c < len; ++c) m[c] += alpha * dm[c];
        }
        rc = orc_advance(n, alpha, dphi, phi, xi, (int64_t)len); /* 8 */
        if (rc) goto out;
        if (alphas) alphas[k] = alpha;
        if (tr) {
            if (tr->alpha) tr->alpha[k] = alpha;
            if (tr->ncycles) tr->ncycles[k] = ncyc;
            if (tr->relres) tr->relres[k] = rel;
        }
    }
    if (m_out) {
        if (p->density_update == 0) orc_cic_deposit(n, xi, w, (int64_t)len, m_out);
        else memcpy(m_out, m, len * sizeof(double));
    }
    if (xi_out) memcpy(xi_out, xi, 3 * len * sizeof(double));
out:
    if (steps) *steps = k;
    free(dm), free(prev), free(alphas);
    free(w), free(xi), free(m), free(s), free(a), free(phidot), free(dphi), free(g), free(lam);
    if (rc) return rc;
    return done ? 0 : (stalled ? 2 : 1);
}

/* ---------------------------------------------------------------- adjoint */

/* Smallest eigenvalue of a symmetric 3x3 matrix with a unit eigenvector, by
 * the same cyclic Jacobi rotations as orc_min_eig_sym3, accumulated into V
 * (columns: eigenvectors, A = V diag V^T). */
static double min_eig_vec_sym3(const double A[3][3], double v[3]) {
    double m[3][3], V[3][3] = {{1.0, 0.0, 0.0}, {0.0, 1.0, 0.0}, {0.0, 0.0, 1.0}};
    memcpy(m, A, sizeof(m));
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = m[0][1] * m[0][1] + m[0][2] * m[0][2] + m[1][2] * m[1][2];
        if (off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (m[p][q] == 0.0) continue;
                double theta = (m[q][q] - m[p][p]) / (2.0 * m[p][q]);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < 3; ++r) {
                    double mrp = m[r][p], mrq = m[r][q];
                    m[r][p] = c * mrp - s * mrq;
                    m[r][q] = s * mrp + c * mrq;
                }
                for (int r = 0; r < 3; ++r) {
                    double mpr = m[p][r], mqr = m[q][r];
                    m[p][r] = c * mpr - s * mqr;
                    m[q][r] = s * mpr + c * mqr;
                }
                m[p][q] = m[q][p] = 0.0;
                for (int r = 0; r < 3; ++r) {
                    double vrp = V[r][p], vrq = V[r][q];
                    V[r][p] = c * vrp - s * vrq;
                    V[r][q] = s * vrp + c * vrq;
                }
            }
    }
    int best = 0;
    if (m[1][1] < m[best][best]) best = 1;
    if (m[2][2] < m[best][best]) best = 2;
    for (int r = 0; r < 3; ++r) v[r] = V[r][best];
    return m[best][best];
}

/* dC/dlambda0 of the compression limiter under the chosen reading (zero
 * where lambda0 is clamped). */
static double climit_deriv(int reading, double xi_m, double lambda0) {
    if (!(lambda0 > 1e-12)) return 0.0;
    double q = xi_m / lambda0, dq = -xi_m / (lambda0 * lambda0);
    double v, dv;
    switch (reading) {
        case ORC_CLIM_LITERAL: v = q - heaviside(q - 1.0); dv = dq; break;
        case ORC_CLIM_STEP: v = q * heaviside(q - 1.0); dv = heaviside(q - 1.0) * dq; break;
        default: v = q - 1.0 > 0.0 ? q - 1.0 : 0.0; dv = q - 1.0 > 0.0 ? dq : 0.0; break;
    }
    return 8.0 * v * dv;
}

/* Transpose of the Hessian stencil: phibar += sum_ab H_ab^T Ebar_ab, Ebar a
 * full 3x3 matrix per node (both off-diagonal entries use the same cross
 * stencil). */
static void hessian_adj(const int n[3], const double* Ebar, double* phibar) {
    long o[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (long i = 0; i < n[0]; ++i)
        for (long j = 0; j < n[1]; ++j)
            for (long k = 0; k < n[2]; ++k) {
                const double* E = Ebar + 9 * at(n, i, j, k);
                for (int a = 0; a < 3; ++a) {
                    double d = E[3 * a + a];
                    phibar[at(n, i + o[a][0], j + o[a][1], k + o[a][2])] += d;
                    phibar[at(n, i, j, k)] -= 2.0 * d;
                    phibar[at(n, i - o[a][0], j - o[a][1], k - o[a][2])] += d;
                    for (int b = a + 1; b < 3; ++b) {
                        double x = 0.25 * (E[3 * a + b] + E[3 * b + a]);
                        long pi = o[a][0] + o[b][0], pj = o[a][1] + o[b][1], pk = o[a][2] + o[b][2];
                        long qi = o[a][0] - o[b][0], qj = o[a][1] - o[b][1], qk = o[a][2] - o[b][2];
                        phibar[at(n, i + pi, j + pj, k + pk)] += x;
                        phibar[at(n, i + qi, j + qj, k + qk)] -= x;
                        phibar[at(n, i - qi, j - qj, k - qk)] -= x;
                        phibar[at(n, i - pi, j - pj, k - pk)] += x;
                    }
                }
            }
}

/* CIC weight of corner (di, dj, dk) of a tracer with fractions f and its
 * derivatives with respect to the three coordinates. */
static double cic_weight(const double f[3], int di, int dj, int dk, double dw[3]) {
    double wx = di ? f[0] : 1.0 - f[0], wy = dj ? f[1] : 1.0 - f[1], wz = dk ? f[2] : 1.0 - f[2];
    double sx = di ? 1.0 : -1.0, sy = dj ? 1.0 : -1.0, sz = dk ? 1.0 : -1.0;
    dw[0] = sx * wy * wz, dw[1] = wx * sy * wz, dw[2] = wx * wy * sz;
    return wx * wy * wz;
}

static void project_mean(double* v, size_t len) {
    double mu = mean(v, len);
    for (size_t c = 0; c < len; ++c) v[c] -= mu;
}

int orc_adjoint(const orc_params* p, const double* rho, const double* alpha, int K,
                const double* gbar, double* grad) {
    if (!params_ok(p) || !rho || !gbar || !grad || K < 0 || (K > 0 && !alpha) ||
        p->density_update != 0)
        return ORC_E_INVALID;
    const int* n = p->n;
    const size_t len = ncells(n);
    double rho_sum = 0.0;
    for (size_t c = 0; c < len; ++c) {
        if (!(rho[c] >= 0.0) || !isfinite(rho[c])) return ORC_E_INVALID;
        rho_sum += rho[c];
    }
    if (!(rho_sum > 0.0)) return ORC_E_INVALID;
    const double rho_bar = rho_sum / (double)len;
    const size_t K1 = (size_t)K + 1;
    double* w = (double*)malloc(len * sizeof(double));
    double* XI = (double*)malloc(K1 * 3 * len * sizeof(double));  /* xi_k, k = 0..K */
    double* PHI = (double*)malloc(K1 * len * sizeof(double));     /* phi_k */
    double* PD = (double*)malloc((K > 0 ? (size_t)K : 1) * len * sizeof(double)); /* phidot_k */
    double* m = (double*)malloc(len * sizeof(double));
    double* s = (double*)malloc(len * sizeof(double));
    double* a = (double*)malloc(len * sizeof(double));
    double* dphi = (double*)malloc(len * sizeof(double));
    double* V = (double*)malloc(3 * len * sizeof(double));
    double* Ein = (double*)malloc(9 * len * sizeof(double));  /* e^-1 per node */
    double* gdet = (double*)malloc(len * sizeof(double));
    double* lam = (double*)malloc(len * sizeof(double));
    double* evec = (double*)malloc(3 * len * sizeof(double));
    double* phibar = (double*)malloc(len * sizeof(double));
    double* xibar = (double*)malloc(3 * len * sizeof(double));
    double* xinew = (double*)malloc(3 * len * sizeof(double));
    double* wbar = (double*)malloc(len * sizeof(double));
    double* dbar = (double*)malloc(len * sizeof(double));
    double* Vbar = (double*)malloc(3 * len * sizeof(double));
    double* Ebar = (double*)malloc(9 * len * sizeof(double));
    double* tmp = (double*)malloc(len * sizeof(double));
    double* lamb = (double*)malloc(len * sizeof(double));
    double* mbar = (double*)malloc(len * sizeof(double));
    int rc = 0;
    if (!w || !XI || !PHI || !PD || !m || !s || !a || !dphi || !V || !Ein || !gdet || !lam ||
        !evec || !phibar || !xibar || !xinew || !wbar || !dbar || !Vbar || !Ebar || !tmp ||
        !lamb || !mbar) {
        rc = ORC_E_NOMEM;
        goto out;
    }

    /* forward: the solve's K advances with the given step lengths, keeping
     * xi_k, phi_k and phidot_k (same steps as orc_solve) */
    for (long i = 0; i < n[0]; ++i)
        for (long j = 0; j < n[1]; ++j)
            for (long kk = 0; kk < n[2]; ++kk) {
                size_t c = at(n, i, j, kk);
                w[c] = rho[c] / rho_bar;
                XI[3 * c + 0] = (double)i, XI[3 * c + 1] = (double)j, XI[3 * c + 2] = (double)kk;
            }
    memset(PHI, 0, len * sizeof(double));
    for (int k = 0; k < K; ++k) {
        double* xi = XI + (size_t)k * 3 * len;
        double* phi = PHI + (size_t)k * len;
        orc_cic_deposit(n, xi, w, (int64_t)len, m);
        if ((rc = orc_source(p, phi, m, s, NULL))) goto out;
        for (size_t c = 0; c < len; ++c) a[c] = m[c] > p->a_min ? m[c] : p->a_min;
        /* the forward solve's initial guess: the last step's phidot with
         * warm_start 1, extrapolated from the last two with 2 (0 before the
         * first step) */
        if (p->warm_start) {
            double* u0 = PD + (size_t)k * len;
            if (k == 0) {
                memset(u0, 0, len * sizeof(double));
            } else if (p->warm_start == 2 && k >= 2) {
                const double r = alpha[k - 1] / alpha[k - 2];
                const double *u1 = u0 - len, *u2 = u0 - 2 * len;
                for (size_t c = 0; c < len; ++c) u0[c] = u1[c] + r * (u1[c] - u2[c]);
            } else {
                memcpy(u0, u0 - len, len * sizeof(double));
            }
            rc = orc_mg_solve_from(p, a, s, u0, NULL, NULL);
        } else {
            rc = orc_mg_solve(p, a, s, PD + (size_t)k * len, NULL, NULL);
        }
        if (rc) goto out;
        orc_apply_S(n, p->s_side, PD + (size_t)k * len, dphi);
        project_mean(dphi, len);
        memcpy(phi + len, phi, len * sizeof(double));
        memcpy(xi + 3 * len, xi, 3 * len * sizeof(double));
        if ((rc = orc_advance(n, alpha[k], dphi, phi + len, xi + 3 * len, (int64_t)len))) goto out;
    }

    /* delta_r = -lap phi_K: phibar_K = -lap^T gbar (the 7-point stencil is
     * symmetric) */
    for (long i = 0; i < n[0]; ++i)
        for (long j = 0; j < n[1]; ++j)
            for (long k = 0; k < n[2]; ++k) {
                size_t c = at(n, i, j, k);
                double acc = 0.0;
                for (int ax = 0; ax < 3; ++ax) {
                    long di = ax == 0, dj = ax == 1, dk = ax == 2;
                    acc += gbar[at(n, i + di, j + dj, k + dk)] + gbar[at(n, i - di, j - dj, k - dk)] -
                           2.0 * gbar[c];
                }
                phibar[c] = -acc;
            }
    memset(xibar, 0, 3 * len * sizeof(double));
    memset(wbar, 0, len * sizeof(double));

    for (int k = K - 1; k >= 0; --k) {
        const double al = alpha[k];
        const double* xi = XI + (size_t)k * 3 * len;
        const double* phi = PHI + (size_t)k * len;
        const double* pd = PD + (size_t)k * len;
        /* step k's forward quantities */
        orc_cic_deposit(n, xi, w, (int64_t)len, m);
        for (size_t c = 0; c < len; ++c) a[c] = m[c] > p->a_min ? m[c] : p->a_min;
        orc_apply_S(n, p->s_side, pd, dphi);
        project_mean(dphi, len);
        for (long i = 0; i < n[0]; ++i)
            for (long j = 0; j < n[1]; ++j)
                for (long kk = 0; kk < n[2]; ++kk) {
                    size_t c = at(n, i, j, kk);
                    double H[3][3], e[3][3], G[3];
                    hessian(n, phi, i, j, kk, H);
                    for (int x = 0; x < 3; ++x) {
                        for (int y = 0; y < 3; ++y) e[x][y] = (x == y ? 1.0 : 0.0) + H[x][y];
                        G[x] = cgrad(n, dphi, i, j, kk, x);
                    }
                    double d = det3(e);
                    gdet[c] = d;
                    lam[c] = min_eig_vec_sym3(e, evec + 3 * c);
                    /* e^-1 by cofactors (e symmetric) */
                    double* Ei = Ein + 9 * c;
                    Ei[0] = (e[1][1] * e[2][2] - e[1][2] * e[2][1]) / d;
                    Ei[1] = (e[0][2] * e[2][1] - e[0][1] * e[2][2]) / d;
                    Ei[2] = (e[0][1] * e[1][2] - e[0][2] * e[1][1]) / d;
                    Ei[3] = (e[1][2] * e[2][0] - e[1][0] * e[2][2]) / d;
                    Ei[4] = (e[0][0] * e[2][2] - e[0][2] * e[2][0]) / d;
                    Ei[5] = (e[0][2] * e[1][0] - e[0][0] * e[1][2]) / d;
                    Ei[6] = (e[1][0] * e[2][1] - e[1][1] * e[2][0]) / d;
                    Ei[7] = (e[0][1] * e[2][0] - e[0][0] * e[2][1]) / d;
                    Ei[8] = (e[0][0] * e[1][1] - e[0][1] * e[1][0]) / d;
                    for (int x = 0; x < 3; ++x)
                        V[3 * c + x] = Ei[3 * x] * G[0] + Ei[3 * x + 1] * G[1] + Ei[3 * x + 2] * G[2];
                }
        /* phi_{k+1} = phi_k + alpha dphi: phibar passes through, dbar = alpha phibar */
        for (size_t c = 0; c < len; ++c) dbar[c] = al * phibar[c];
        /* tracers xi_{k+1} = xi_k - alpha V(xi_k) (CIC interpolation) */
        memset(Vbar, 0, 3 * len * sizeof(double));
        memcpy(xinew, xibar, 3 * len * sizeof(double));
        for (size_t t = 0; t < len; ++t) {
            long i0[3];
            double f[3];
            for (int x = 0; x < 3; ++x) cic_axis(xi[3 * t + x], n[x], &i0[x], &f[x]);
            const double* xb = xibar + 3 * t;
            for (int di = 0; di < 2; ++di)
                for (int dj = 0; dj < 2; ++dj)
                    for (int dk = 0; dk < 2; ++dk) {
                        double dw[3];
                        double wgt = cic_weight(f, di, dj, dk, dw);
                        size_t c = at(n, i0[0] + di, i0[1] + dj, i0[2] + dk);
                        double vdot = V[3 * c] * xb[0] + V[3 * c + 1] * xb[1] + V[3 * c + 2] * xb[2];
                        for (int x = 0; x < 3; ++x) {
                            Vbar[3 * c + x] -= al * wgt * xb[x];
                            xinew[3 * t + x] -= al * dw[x] * vdot;
                        }
                    }
        }
        memcpy(xibar, xinew, 3 * len * sizeof(double));
        /* V = e^-1 G: Gbar = e^-1 Vbar, Ebar = -Gbar V^T */
        memset(tmp, 0, len * sizeof(double));
        for (long i = 0; i < n[0]; ++i)
            for (long j = 0; j < n[1]; ++j)
                for (long kk = 0; kk < n[2]; ++kk) {
                    size_t c = at(n, i, j, kk);
                    const double* Ei = Ein + 9 * c;
                    const double* vb = Vbar + 3 * c;
                    double Gb[3];
                    for (int x = 0; x < 3; ++x)
                        Gb[x] = Ei[3 * x] * vb[0] + Ei[3 * x + 1] * vb[1] + Ei[3 * x + 2] * vb[2];
                    for (int x = 0; x < 3; ++x)
                        for (int y = 0; y < 3; ++y) Ebar[9 * c + 3 * x + y] = -Gb[x] * V[3 * c + y];
                    /* G = central difference of dphi */
                    for (int ax = 0; ax < 3; ++ax) {
                        long di = ax == 0, dj = ax == 1, dk = ax == 2;
                        tmp[at(n, i + di, j + dj, kk + dk)] += 0.5 * Gb[ax];
                        tmp[at(n, i - di, j - dj, kk - dk)] -= 0.5 * Gb[ax];
                    }
                }
        for (size_t c = 0; c < len; ++c) dbar[c] += tmp[c];
        /* dphi = S phidot - mean: phidotbar = S P dbar */
        project_mean(dbar, len);
        orc_apply_S(n, p->s_side, dbar, tmp);
        /* phidot = P L(a)^+ P s: sbar = P L(a)^+ P phidotbar (L symmetric) */
        if ((rc = orc_mg_solve(p, a, tmp, lamb, NULL, NULL))) goto out;
        project_mean(lamb, len);
        /* coefficient: abar_j = sum over the faces f of node j of
         * (1/2) (lamb_n - lamb_j)(phidot_n - phidot_j); a = max(m, a_min) */
        memset(mbar, 0, len * sizeof(double));
        for (long i = 0; i < n[0]; ++i)
            for (long j = 0; j < n[1]; ++j)
                for (long kk = 0; kk < n[2]; ++kk) {
                    size_t c = at(n, i, j, kk);
                    for (int ax = 0; ax < 3; ++ax) {
                        long di = ax == 0, dj = ax == 1, dk = ax == 2;
                        size_t q = at(n, i + di, j + dj, kk + dk);
                        double A = 0.5 * (lamb[q] - lamb[c]) * (pd[q] - pd[c]);
                        mbar[c] += A;
                        mbar[q] += A;
                    }
                }
        for (size_t c = 0; c < len; ++c)
            if (!(m[c] > p->a_min)) mbar[c] = 0.0;
        /* s = P S t: tbar = S P sbar */
        orc_apply_S(n, p->s_side, lamb, tmp);
        /* t = Sigma + C(lambda0) + E(sqrt g, Sigma), Sigma = 1 - m */
        for (size_t c = 0; c < len; ++c) {
            double Sig = 1.0 - m[c];
            double sg = Sig > 0.0 ? 1.0 : (Sig < 0.0 ? -1.0 : 0.0);
            mbar[c] += tmp[c] * (-1.0 + 2.0 * heaviside(gdet[c] - p->v_m) * sg);
            double lb = tmp[c] * climit_deriv(p->climiter, p->xi_m, lam[c]);
            const double* v = evec + 3 * c;
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y) Ebar[9 * c + 3 * x + y] += lb * v[x] * v[y];
        }
        hessian_adj(n, Ebar, phibar);
        /* m = CIC deposit of the tracers' masses at xi_k */
        for (size_t t = 0; t < len; ++t) {
            long i0[3];
            double f[3];
            for (int x = 0; x < 3; ++x) cic_axis(xi[3 * t + x], n[x], &i0[x], &f[x]);
            for (int di = 0; di < 2; ++di)
                for (int dj = 0; dj < 2; ++dj)
                    for (int dk = 0; dk < 2; ++dk) {
                        double dw[3];
                        double wgt = cic_weight(f, di, dj, dk, dw);
                        double mb = mbar[at(n, i0[0] + di, i0[1] + dj, i0[2] + dk)];
                        wbar[t] += wgt * mb;
                        for (int x = 0; x < 3; ++x) xibar[3 * t + x] += w[t] * dw[x] * mb;
                    }
        }
    }
    /* w = rho / rho_bar with rho_bar the mean of rho */
    {
        double sw = 0.0;
        for (size_t c = 0; c < len; ++c) sw += wbar[c] * w[c];
        for (size_t c = 0; c < len; ++c) grad[c] = (wbar[c] - sw / (double)len) / rho_bar;
    }
out:
    free(w), free(XI), free(PHI), free(PD), free(m), free(s), free(a), free(dphi), free(V);
    free(Ein), free(gdet), free(lam), free(evec), free(phibar), free(xibar), free(xinew);
    free(wbar), free(dbar), free(Vbar), free(Ebar), free(tmp), free(lamb), free(mbar);
    return rc;
}
