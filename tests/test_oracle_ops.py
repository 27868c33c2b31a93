"""Pins of the oracle's building blocks against mathematics it does not use.

Each test checks one oracle step against an independent construction: brute
force, a matrix built another way, a closed form, a library routine solving the
same mathematical problem by a different method, or an exact identity.
"""
import json
import os

import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(20161130)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ deposit

def _brute_cic(n, x, w):
    """Sum over every (particle, node) pair of the product of 1D hat
    functions of the minimum-image separation."""
    out = np.zeros(n)
    grids = np.meshgrid(*[np.arange(v) for v in n], indexing="ij")
    for p in range(x.shape[0]):
        wt = np.ones(n)
        for a in range(3):
            d = (x[p, a] - grids[a] + n[a] / 2) % n[a] - n[a] / 2
            wt *= np.maximum(0.0, 1.0 - np.abs(d))
        out += w[p] * wt
    return out


def test_cic_deposit_matches_brute_force():
    n = (8, 4 * 2, 16)
    x = RNG.uniform(-20, 40, size=(60, 3))
    w = RNG.uniform(0.1, 3.0, size=60)
    got = O.cic_deposit(n, x, w)
    ref = _brute_cic(n, x, w)
    assert np.max(np.abs(got - ref)) < 1e-13
    assert abs(got.sum() - w.sum()) < 1e-12  # mass conservation


def test_cic_particle_on_node_and_unit_mass():
    n = (8, 8, 8)
    x = np.array([[3.0, 5.0, 7.0], [8.0, -8.0, 16.0]])  # second wraps onto (0,0,0)
    got = O.cic_deposit(n, x)
    assert got[3, 5, 7] == 1.0 and got[0, 0, 0] == 1.0 and got.sum() == 2.0


# ---------------------------------------------------------------- operator L

def _fwd_diff(n, ax):
    """Sparse-free dense forward difference (D u)_j = u_{j+e_ax} - u_j."""
    N = int(np.prod(n))
    idx = np.arange(N).reshape(n)
    D = np.zeros((N, N))
    D[idx.ravel(), idx.ravel()] = -1.0
    D[idx.ravel(), np.roll(idx, -1, axis=ax).ravel()] += 1.0
    return D


def _L_matrix(a, h):
    """L = -sum_a h_a^-2 D_a^T diag(face a) D_a, face a_{j+1/2} = (a_j + a_{j+e})/2:
    the flux form of div(a grad) built from incidence matrices."""
    n = a.shape
    N = a.size
    L = np.zeros((N, N))
    for ax in range(3):
        D = _fwd_diff(n, ax)
        face = 0.5 * (a + np.roll(a, -1, axis=ax)).ravel()
        L -= D.T @ (face[:, None] * D) / h[ax] ** 2
    return L


def test_apply_L_equals_incidence_matrix_form():
    n = (4, 8, 4)
    a = np.exp(RNG.normal(size=n))
    u = RNG.normal(size=n)
    h = (1.0, 2.0, 4.0)
    got = O.apply_L(a, u, h)
    ref = (_L_matrix(a, h) @ u.ravel()).reshape(n)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_apply_L_nullspace_symmetry_sign():
    n = (8, 8, 8)
    a = np.exp(RNG.normal(size=n))
    assert np.max(np.abs(O.apply_L(a, np.full(n, 3.7)))) < 1e-12
    u, v = RNG.normal(size=n), RNG.normal(size=n)
    assert abs(np.vdot(u, O.apply_L(a, v)) - np.vdot(v, O.apply_L(a, u))) < 1e-10
    assert np.vdot(u, O.apply_L(a, u)) < 0


# ------------------------------------------------------------ RB-GS sweep

def test_rbgs_black_nodes_satisfied_after_sweep():
    """Gauss-Seidel with black last: after a sweep every black equation holds
    exactly; and the exact solution is a fixed point of the sweep."""
    n = (8, 4 * 2, 8)
    a = np.exp(RNG.normal(size=n))
    f = RNG.normal(size=n)
    f -= f.mean()
    u = O.rbgs_sweep(a, f, RNG.normal(size=n))
    r = f - O.apply_L(a, u)
    i, j, k = np.indices(n)
    black = (i + j + k) % 2 == 1
    assert np.max(np.abs(r[black])) < 1e-12
    assert np.max(np.abs(r[~black])) > 1e-6
    L = _L_matrix(a, (1, 1, 1))
    M = np.block([[L, np.ones((L.shape[0], 1))], [np.ones((1, L.shape[0])), np.zeros((1, 1))]])
    sol = np.linalg.solve(M, np.r_[f.ravel(), 0.0])[:-1].reshape(n)
    assert np.max(np.abs(O.rbgs_sweep(a, f, sol) - sol)) < 1e-11


# ----------------------------------------------- restriction / prolongation

@pytest.mark.parametrize("n", [(8, 8, 8), (16, 4, 8), (32, 4, 4)])
def test_prolongation_is_scaled_transpose_of_full_weighting(n):
    nc = O.coarse_dims(n)
    ncoarsened = sum(1 for v in n if v > 4)
    f = RNG.normal(size=n)
    c = RNG.normal(size=nc)
    lhs = np.vdot(O.restrict(f), c) * 2 ** ncoarsened
    rhs = np.vdot(f, O.prolong_add(c, np.zeros(n)))
    assert abs(lhs - rhs) < 1e-11 * abs(rhs)


def test_restrict_and_prolong_reproduce_smooth_fields():
    n = (16, 16, 8)
    i = np.arange(16)
    # a constant is reproduced exactly; a coarse-grid-linear field is
    # interpolated exactly away from the periodic seam
    assert np.allclose(O.restrict(np.full(n, 2.5)), 2.5, atol=1e-14)
    assert np.allclose(O.prolong_add(np.full(O.coarse_dims(n), 2.5), np.zeros(n)), 2.5, atol=1e-14)
    c = np.broadcast_to(np.arange(8.0)[:, None, None], O.coarse_dims(n)).copy()
    fine = O.prolong_add(c, np.zeros(n))
    assert np.allclose(fine[:14, 0, 0], i[:14] / 2.0, atol=1e-14)


# ------------------------------------------------------------- smoothing S

def test_S_fourier_symbol_kills_nyquist_planes():
    n = (8, 16, 8)
    grids = np.indices(n)
    for m in [(1, 0, 0), (2, 3, 1), (4, 0, 0), (0, 8, 0), (4, 8, 4), (3, 5, 2)]:
        kv = [2 * np.pi * m[a] / n[a] for a in range(3)]
        wave = np.cos(sum(kv[a] * grids[a] for a in range(3)))
        sym = np.prod([0.5 + 0.5 * np.cos(k) for k in kv])
        assert np.max(np.abs(O.apply_S(wave) - sym * wave)) < 1e-13
    u = RNG.normal(size=n)
    assert abs(O.apply_S(u).sum() - u.sum()) < 1e-10


# --------------------------------------------------------------- multigrid

def _fft_poisson(s):
    """Exact solve of the 7-point periodic Laplacian (a = 1) by FFT."""
    n = s.shape
    ks = [2 * np.pi * np.fft.fftfreq(v) for v in n]
    lam = sum(np.reshape(2 * np.cos(k) - 2, [-1 if a == b else 1 for b in range(3)])
              for a, k in enumerate(ks))
    lam = np.broadcast_to(lam, n).copy()
    sk = np.fft.fftn(s)
    lam[0, 0, 0] = 1.0
    uk = sk / lam
    uk[0, 0, 0] = 0.0
    return np.fft.ifftn(uk).real


@pytest.mark.parametrize("n", [(16, 32, 8), (8, 8, 8), (32, 8, 8)])
def test_mg_solve_constant_coefficient_matches_fft(n):
    s = RNG.normal(size=n)
    s -= s.mean()
    p = O.OracleParams(n=n, tol_in=1e-12, max_vcycles=100)
    u, ncyc, rel = O.mg_solve(p, np.ones(n), s)
    ref = _fft_poisson(s)
    assert rel <= 1e-12 and ncyc < 40
    # the periodic operator fixes u up to a constant
    assert np.linalg.norm((u - u.mean()) - ref) <= 1e-10 * np.linalg.norm(ref)


def test_mg_solve_variable_coefficient_matches_dense_direct():
    n = (8, 8, 8)
    a = np.maximum(np.exp(1.5 * RNG.normal(size=n)), 0.01)
    s = RNG.normal(size=n)
    s -= s.mean()
    p = O.OracleParams(n=n, tol_in=1e-13, max_vcycles=200)
    u, ncyc, rel = O.mg_solve(p, a, s)
    L = _L_matrix(a, (1, 1, 1))
    M = np.block([[L, np.ones((L.shape[0], 1))], [np.ones((1, L.shape[0])), np.zeros((1, 1))]])
    ref = np.linalg.solve(M, np.r_[s.ravel(), 0.0])[:-1].reshape(n)
    assert rel <= 1e-13
    assert np.linalg.norm((u - u.mean()) - ref) <= 1e-10 * np.linalg.norm(ref)


def test_vcycle_contracts():
    n = (16, 16, 16)
    s = RNG.normal(size=n)
    s -= s.mean()
    p = O.OracleParams(n=n)
    u = O.vcycle(p, np.ones(n), s, np.zeros(n))
    r1 = np.linalg.norm(s - O.apply_L(np.ones(n), u)) / np.linalg.norm(s)
    assert r1 < 0.2


# ---------------------------------------------------------------- geometry

def test_min_eig_sym3_matches_lapack():
    mats = [np.diag([3.0, 1.0, 2.0]), np.eye(3), np.diag([1e-9, 1.0, 1.0]),
            np.array([[2.0, 1.0, 0.0], [1.0, 2.0, 0.0], [0.0, 0.0, 1.0 + 1e-12]])]
    for _ in range(200):
        B = RNG.normal(size=(3, 3))
        mats.append(B + B.T)
    for A in mats:
        ref = np.linalg.eigvalsh(A)[0]
        assert abs(O.min_eig_sym3(A) - ref) <= 1e-13 * max(1.0, np.abs(A).max())


def test_geometry_plane_wave_closed_form():
    """phi = A cos(k.x): the 3-point second difference is -4 sin^2(k_a/2) phi
    and the 4-point cross difference -sin k_a sin k_b phi."""
    n = (16, 8, 32)
    m = (3, 1, 5)
    kv = np.array([2 * np.pi * m[a] / n[a] for a in range(3)])
    grids = np.indices(n)
    phi = 0.8 * np.cos(sum(kv[a] * grids[a] for a in range(3)))
    g, lam = O.geometry(phi)
    for idx in [(0, 0, 0), (5, 3, 17), (15, 7, 31), (7, 2, 4)]:
        p = phi[idx]
        H = np.empty((3, 3))
        for a in range(3):
            for b in range(3):
                H[a, b] = -4 * np.sin(kv[a] / 2) ** 2 * p if a == b else -np.sin(kv[a]) * np.sin(kv[b]) * p
        e = np.eye(3) + H
        assert abs(g[idx] - np.linalg.det(e)) < 1e-12
        assert abs(lam[idx] - np.linalg.eigvalsh(e)[0]) < 1e-12


def test_source_limiters_closed_form():
    n = (16, 8, 8)
    i = np.arange(16)[:, None, None] * np.ones(n)
    # uniform mass, undeformed mesh: no source
    s, t = O.source(O.OracleParams(n=n), np.zeros(n), np.ones(n))
    assert np.max(np.abs(s)) == 0.0 and np.max(np.abs(t)) == 0.0
    # phi = B cos(2 pi i / 16): e = diag(1 - 4 sin^2(pi/16) B cos, 1, 1), so
    # e_xx runs over [0.05, 1.95]: compressed below xi_m and expanded above v_m
    p = O.OracleParams(n=n, v_m=1.5)
    c1 = 4 * np.sin(np.pi / 16) ** 2
    phi = (0.95 / c1) * np.cos(2 * np.pi * i / 16)
    m = 1.0 + 0.3 * np.sin(2 * np.pi * i / 16)
    s, t = O.source(p, phi, m)
    exx = 1 - c1 * phi
    lam0 = np.minimum(exx, 1.0)
    sig = 1 - m
    C = 4 * np.maximum(0.0, p.xi_m / lam0 - 1) ** 2
    E = -2.0 * (exx > p.v_m) * np.abs(sig)
    assert C.max() > 1.0 and E.min() < 0.0  # both limiters active
    assert np.max(np.abs(t - (sig + C + E))) < 1e-12 * np.abs(C).max()
    ref = O.apply_S(sig + C + E)
    assert np.max(np.abs(s - (ref - ref.mean()))) < 1e-12 * np.abs(ref).max()


def test_climiter_readings():
    n = (8, 8, 8)
    i = np.arange(8)[:, None, None] * np.ones(n)
    phi = 0.9 * np.cos(2 * np.pi * i / 8) / (4 * np.sin(np.pi / 8) ** 2)  # exx = 1 - 0.9 cos
    lam0 = np.minimum(1 - 0.9 * np.cos(2 * np.pi * i / 8), 1.0)
    q = 0.1 / lam0
    heav = (q - 1 > 0).astype(float)
    expect = {O.CLIM_SOFT: 4 * np.maximum(q - 1, 0) ** 2,
              O.CLIM_LITERAL: 4 * (q - heav) ** 2,
              O.CLIM_STEP: 4 * (q * heav) ** 2}
    for reading, C in expect.items():
        p = O.OracleParams(n=n, climiter=reading)
        _, t = O.source(p, phi, np.ones(n))
        assert np.max(np.abs(t - C)) < 1e-11


# ------------------------------------------------------------ step limiter

def test_step_limiter_closed_form():
    """phi = 0, dphi = A cos(2 pi i/N): lambda_min(I + alpha H) = 1 - alpha c,
    c = 4 A sin^2(pi/N); max |grad dphi| = A sin(2 pi/N)."""
    N = 16
    n = (N, 8, 8)
    i = np.arange(N)[:, None, None] * np.ones(n)
    c1 = 4 * np.sin(np.pi / N) ** 2
    for target in (1.0, 0.5, 0.125):
        # alpha = target passes (1 - 0.735 > 0.02) and 2 * target fails
        A = 0.75 * (1 - 0.02) / (c1 * target)
        dphi = A * np.cos(2 * np.pi * i / N)
        p = O.OracleParams(n=n, d_max=1e9)
        assert O.step_limiter(p, np.zeros(n), dphi) == target
    # the move limit: alpha max|grad dphi| <= d_max
    dphi = 3.0 * np.cos(2 * np.pi * i / N)
    gmax = 3.0 * np.sin(2 * np.pi / N)
    p = O.OracleParams(n=n, d_max=0.3, lambda_floor=0.0)
    al = O.step_limiter(p, np.zeros(n), dphi)
    assert al * gmax <= 0.3 < 2 * al * gmax


def test_step_limiter_closed_form_with_cross_terms():
    """dphi = A cos(2 pi (i + j + k) / N), phi = 0: every Hessian has equal
    diagonal entries D cos(theta) and equal off-diagonal ones O cos(theta)
    (D = -4 A sin^2(pi/N) from the 3-point second difference, O = -A
    sin^2(2 pi/N) from the 4-point cross difference), so the eigenvalues of
    I + alpha H are 1 + alpha cos(theta) (D - O) (twice) and 1 + alpha
    cos(theta) (D + 2 O); the smallest, at theta = 0, is 1 - alpha c with
    c = A (4 sin^2(pi/N) + 2 sin^2(2 pi/N)).  Sylvester's criterion must use
    every off-diagonal entry to find it."""
    N = 16
    n = (N, N, N)
    i, j, k = np.indices(n)
    c1 = 4 * np.sin(np.pi / N) ** 2 + 2 * np.sin(2 * np.pi / N) ** 2
    for target in (1.0, 0.25, 0.0625):
        A = 0.75 * (1 - 0.01) / (c1 * target)
        dphi = A * np.cos(2 * np.pi * (i + j + k) / N)
        p = O.OracleParams(n=n, d_max=1e9)
        assert O.step_limiter(p, np.zeros(n), dphi) == target


# ----------------------------------------------------------------- advance

def test_advance_closed_form():
    N = 16
    n = (N, 8, 8)
    i = np.arange(N)[:, None, None] * np.ones(n)
    A, B, alpha = 0.7, 2.0, 0.5
    dphi = A * np.cos(2 * np.pi * i / N)
    phi = B * np.sin(2 * np.pi * i / N)
    xi = np.array([[3.0, 2.0, 5.0], [10.0, 7.0, 0.0]])
    phi2, xi2 = O.advance(alpha, dphi, phi, xi)
    assert np.max(np.abs(phi2 - (phi + alpha * dphi))) < 1e-14
    for t, node in enumerate([3, 10]):
        G = -A * np.sin(2 * np.pi / N) * np.sin(2 * np.pi * node / N)   # central difference
        exx = 1 - 4 * np.sin(np.pi / N) ** 2 * B * np.sin(2 * np.pi * node / N)
        assert abs(xi2[t, 0] - (node - alpha * G / exx)) < 1e-13
        assert xi2[t, 1] == xi[t, 1] and xi2[t, 2] == xi[t, 2]


def test_advance_off_node_closed_form():
    """Tracers at fractional offsets on all three axes of an anisotropic grid.
    With phi = x'Px/2 and dphi = x'Qx/2 + b'x (x = node - c) the central
    differences are exact, so every node has e = I + P and G = Qx + b, the
    node velocity e^-1 G is affine in position, CIC interpolation of it is
    exact, and each tracer moves to xi - alpha (I + P)^-1 (Q (xi - c) + b).
    A weight taken from the wrong axis, a swapped corner or a wrong column in
    the solve for e^-1 G each move the result by far more than the tolerance."""
    n = (16, 8, 32)
    c = np.array([8.0, 4.0, 16.0])
    P = np.array([[0.30, 0.05, -0.07], [0.05, -0.20, 0.11], [-0.07, 0.11, 0.15]])
    Q = np.array([[0.40, -0.13, 0.09], [-0.13, 0.25, 0.06], [0.09, 0.06, -0.30]])
    b = np.array([0.20, -0.35, 0.50])
    alpha = 0.375
    g = np.stack(np.meshgrid(*[np.arange(m, dtype=float) for m in n], indexing="ij"), axis=-1) - c
    phi = 0.5 * np.einsum("...a,ab,...b->...", g, P, g)
    dphi = 0.5 * np.einsum("...a,ab,...b->...", g, Q, g) + g @ b
    # every stencil around these tracers stays clear of the periodic seam
    xi = np.array([[7.25, 3.625, 15.875], [4.5, 2.125, 22.375], [10.875, 4.25, 9.0625]])
    phi2, xi2 = O.advance(alpha, dphi, phi, xi)
    assert np.max(np.abs(phi2 - (phi + alpha * dphi))) < 1e-13
    want = xi - alpha * np.linalg.solve(np.eye(3) + P, (Q @ (xi - c).T + b[:, None])).T
    assert np.max(np.abs(xi2 - want)) < 1e-12, (xi2, want)


def test_paper_constants_are_the_defaults():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as fh:
        g = json.load(fh)
    p = O.OracleParams()
    assert p.xi_m == g["xi_m"]["value"] and p.v_m == g["v_m"]["value"]
    # delta_r = 3 - tr(e); a triad with every diagonal entry >= 0.1 gives <= 2.7
    assert 3 - 3 * g["min_diag_triad"]["value"] == pytest.approx(g["delta_r_bound"]["value"])
    assert g["delta_r_max_observed"]["value"] <= g["delta_r_bound"]["value"]


# ------------------------------------------------- paper-literal mass update

def test_mass_change_reduces_to_the_solve_operator_and_conserves_mass():
    n = (16, 8, 16)
    m = np.exp(0.3 * RNG.normal(size=n))
    v = RNG.normal(size=n)
    assert np.abs(O.mass_change(np.zeros(n), m, v) - O.apply_L(m, v)).max() < 1e-13
    i = np.indices(n)
    phi = 0.4 * np.cos(2 * np.pi * (i[0] / 16 + i[2] / 16)) + 0.3 * np.sin(2 * np.pi * i[1] / 8)
    d = O.mass_change(phi, m, v)
    assert abs(d.sum()) < 1e-11 * np.abs(d).sum()


def _continuum_mass_change(N):
    """d_mu(m (I + Hess phi)^-1 d_nu v) of smooth periodic fields, with the
    derivatives of phi and v analytic and the outer divergence spectral."""
    x = np.indices((N, N, N)) * (2 * np.pi / N)
    A, B = 0.25 * (N / (2 * np.pi)) ** 2, 0.15 * (N / (2 * np.pi)) ** 2
    m = 1.0 + 0.3 * np.sin(x[0]) * np.cos(x[1]) + 0.2 * np.cos(x[2])
    phi = A * np.cos(x[0] + x[1]) + B * np.sin(x[2] - x[0])
    v = np.sin(x[0] + 2 * x[2]) + 0.5 * np.cos(x[1])
    s = 2 * np.pi / N  # d/d(grid index) of the phase
    H = np.zeros((3, 3) + m.shape)
    c1, c2 = -A * np.cos(x[0] + x[1]) * s * s, -B * np.sin(x[2] - x[0]) * s * s
    for a, b, w in ((0, 0, c1 + c2), (1, 1, c1), (2, 2, c2), (0, 1, c1), (0, 2, -c2)):
        H[a, b] += w
        if a != b:
            H[b, a] += w
    e = np.moveaxis(H, (0, 1), (-2, -1)) + np.eye(3)
    Kt = m[..., None, None] * np.linalg.inv(e)
    gv = np.stack([np.cos(x[0] + 2 * x[2]) * s, -0.5 * np.sin(x[1]) * s,
                   2 * np.cos(x[0] + 2 * x[2]) * s], -1)
    flux = np.einsum("...ab,...b->...a", Kt, gv)
    k = np.fft.fftfreq(N) * 2 * np.pi
    out = np.zeros_like(m)
    for a in range(3):
        shape = [1, 1, 1]
        shape[a] = N
        out += np.fft.ifftn(1j * k.reshape(shape) * np.fft.fftn(flux[..., a])).real
    return m, phi, v, out


def test_mass_change_converges_to_the_continuum_divergence_at_second_order():
    errs = []
    for N in (16, 32):
        m, phi, v, ref = _continuum_mass_change(N)
        got = O.mass_change(phi, m, v)
        errs.append(np.abs(got - ref).max() / np.abs(ref).max())
    assert errs[1] < 0.02 and 3.0 < errs[0] / errs[1] < 5.0, errs
