"""Pins of the oracle's whole moving-mesh iteration (Sec. II, App. A).

The nonlinear trajectory with the limiters active has no closed form; these
tests pin the iteration where the mathematics fixes the answer: the uniform
fixed point, the plane-parallel (1D) problem whose monotone map is given by the
cumulative mass, the small-amplitude (Poisson) limit, Zel'dovich recovery, the
invariants the paper states, and symmetries.
"""
import numpy as np
import pytest

import oracle as O
from paper_1611_09638_gb300.inputs import linear_field, lpt_particles


def _plane_wave_rho(N, A, ny=8, nz=8):
    i = np.arange(N)
    return np.broadcast_to((1 + A * np.sin(2 * np.pi * i / N))[:, None, None], (N, ny, nz)).copy()


def _closed_form_x(N, A, xi):
    """Monotone 1D map with rho dx = rho_bar dxi for rho = 1 + A sin(2 pi x/N):
    xi(x) = x - (A N / 2 pi) cos(2 pi x / N) (zero-mean displacement), inverted
    by Newton iteration."""
    x = np.array(xi, dtype=float)
    for _ in range(60):
        F = x - A * N / (2 * np.pi) * np.cos(2 * np.pi * x / N) - xi
        x -= F / (1 + A * np.sin(2 * np.pi * x / N))
    return x


def test_uniform_density_is_the_fixed_point():
    n = (16, 8, 8)
    r = O.solve(O.OracleParams(n=n), np.full(n, 3.0))
    assert r.status == 0 and r.steps == 0 and r.R[0] == 0.0
    assert np.all(r.phi == 0.0)


def test_1d_plane_wave_converges_to_closed_form_at_first_order():
    """The 3D iteration on an N x 8 x 8 grid with a plane-parallel density is
    the 1D problem; its map must approach the cumulative-mass closed form as
    the grid is refined (first order: the CIC tracer representation), and
    delta_r stays below 1 (Sec. III, 1D remark)."""
    A = 0.05
    errs = []
    for N in (32, 64, 128):
        rho = _plane_wave_rho(N, A)
        r = O.solve(O.OracleParams(n=rho.shape, k_max=40, tol_out=1e-12, tol_in=1e-10), rho)
        i = np.arange(N, dtype=float)
        X = O.mesh_x(r.phi)[:, 0, 0, 0]
        errs.append(np.abs(X - _closed_form_x(N, A, i)).max() / (A * N / (2 * np.pi)))
        # tracers: the tracer of node c sits at the closed-form xi(x = c)
        xi_exact = i - A * N / (2 * np.pi) * np.cos(2 * np.pi * i / N)
        assert np.abs(r.xi[:, 0, 0, 0] - xi_exact).max() < 0.05 * 32 / N * (A * N / (2 * np.pi)) * 4
        assert O.delta_r(r.phi).max() < 1.0
        # the solution is plane-parallel
        assert np.ptp(r.phi, axis=(1, 2)).max() < 1e-8 * np.abs(r.phi).max()
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 0.05
    assert np.all(order > 0.8) and np.all(order < 1.3), (errs, order)


def test_first_step_is_the_poisson_solve_in_the_linear_limit():
    """For rho = 1 + A d the coefficient is 1 + O(A), so the first increment
    equals the exact FFT solve of the 7-point Laplacian to relative O(A)."""
    n = (16, 16, 16)
    d = linear_field(16, 200.0, 5)
    d /= d.std()
    errs = []
    for A in (1e-3, 1e-2):
        m = 1 + A * d
        p = O.OracleParams(n=n, tol_in=1e-12)
        s, _ = O.source(p, np.zeros(n), m)
        u, _, _ = O.mg_solve(p, np.maximum(m, p.a_min), s)
        k = [2 * np.pi * np.fft.fftfreq(16)] * 3
        lam = (2 * np.cos(k[0]) - 2)[:, None, None] + (2 * np.cos(k[1]) - 2)[None, :, None] + \
              (2 * np.cos(k[2]) - 2)[None, None, :]
        lam[0, 0, 0] = 1.0
        uk = np.fft.fftn(s) / lam
        uk[0, 0, 0] = 0.0
        ref = np.fft.ifftn(uk).real
        errs.append(np.linalg.norm((u - u.mean()) - ref) / np.linalg.norm(ref))
    ratio = errs[1] / errs[0]
    assert errs[0] < 1e-3 and 8.0 < ratio < 12.0, errs


def test_small_amplitude_solve_is_linear_and_recovers_delta_on_large_scales():
    n = (16, 16, 16)
    d = linear_field(16, 400.0, 7)
    d /= d.std()
    out = {}
    for A in (1e-4, 1e-3):
        r = O.solve(O.OracleParams(n=n, k_max=12, tol_out=1e-14, tol_in=1e-10), 1 + A * d)
        assert np.all(r.alpha == 1.0)
        out[A] = O.delta_r(r.phi)
    # homogeneous of degree one as A -> 0
    assert np.linalg.norm(out[1e-3] / 10 - out[1e-4]) < 2e-3 * np.linalg.norm(out[1e-4])
    # delta_r = -lap phi reproduces delta on the large scales
    fk = np.fft.fftn(out[1e-3] - 1e-3 * d)
    dk = np.fft.fftn(1e-3 * d)
    kk = np.sqrt(sum(np.reshape(np.fft.fftfreq(16) * 16, [-1 if a == b else 1 for b in range(3)]) ** 2
                     for a in range(3)))
    low = kk <= 2.0
    assert np.linalg.norm(fk[low]) < 0.1 * np.linalg.norm(dk[low])


def test_zeldovich_displacement_recovered_on_large_scales():
    """Before shell crossing the potential isobaric frame is the Lagrangian
    one (Sec. II), so x(xi = q) - q recovers the Zel'dovich displacement."""
    n, box = 16, 400.0
    pos, _ = lpt_particles(n, box, 11, order=1)
    h = box / n
    rho = O.cic_deposit((n, n, n), pos / h)
    q = np.stack(np.meshgrid(*(np.arange(n),) * 3, indexing="ij"), -1).reshape(-1, 3) * h
    psi = ((pos - q + box / 2) % box - box / 2) / h
    r = O.solve(O.OracleParams(n=(n, n, n), k_max=20, tol_out=1e-12), rho)
    rec = O.mesh_x(r.phi).reshape(-1, 3) - q / h
    kk = np.sqrt(sum(np.reshape(np.fft.fftfreq(n) * n, [-1 if a == b else 1 for b in range(3)]) ** 2
                     for a in range(3)))
    low = kk <= 3.0
    for a in range(3):
        pk = np.fft.fftn(psi[:, a].reshape(n, n, n))[low]
        rk = np.fft.fftn(rec[:, a].reshape(n, n, n))[low]
        corr = np.real(np.vdot(pk, rk)) / (np.linalg.norm(pk) * np.linalg.norm(rk))
        assert corr > 0.95, corr


def test_invariants_every_step():
    """Mass conservation, positive-definite map with lambda0 above the floor,
    mean-zero phi, delta_r < 3 - 3 lambda_floor, on a strongly nonlinear input."""
    n, box = 16, 50.0
    pos, _ = lpt_particles(n, box, 3, order=2)
    rho = O.cic_deposit((n, n, n), pos / (box / n))
    assert (rho / rho.mean() - 1).std() > 1.0
    p = O.OracleParams(n=(n, n, n), k_max=12)
    r = O.solve(p, rho)
    assert r.steps == 12
    assert np.all(np.abs(r.mass - n ** 3) < 1e-9)
    assert np.all(r.min_det > 0) and np.all(r.min_lam > p.lambda_floor)
    g, lam = O.geometry(r.phi)
    assert g.min() > 0 and lam.min() > p.lambda_floor
    assert abs(r.phi.mean()) < 1e-12 * np.abs(r.phi).max()
    assert O.delta_r(r.phi).max() < 3 - 3 * p.lambda_floor
    assert np.all(r.relres <= p.tol_in)
    assert abs(r.m.sum() - n ** 3) < 1e-9


def test_limiter_stall_stops_with_a_valid_map():
    """With a floor the map cannot keep above, the iteration stops (status 2)
    on the last accepted map, which still satisfies every invariant."""
    n, box = 16, 50.0
    pos, _ = lpt_particles(n, box, 3, order=2)
    rho = O.cic_deposit((n, n, n), pos / (box / n))
    p = O.OracleParams(n=(n, n, n), k_max=40, lambda_floor=0.6)
    r = O.solve(p, rho)
    assert r.status == 2 and 0 < r.steps < 40
    g, lam = O.geometry(r.phi)
    assert lam.min() > p.lambda_floor and g.min() > 0
    assert abs(r.m.sum() - n ** 3) < 1e-9


def test_shift_and_axis_permutation_equivariance():
    n = 16
    pos, _ = lpt_particles(n, 100.0, 4, order=1)
    rho = O.cic_deposit((n, n, n), pos / (100.0 / n))
    p = O.OracleParams(n=(n, n, n), k_max=4)
    base = O.solve(p, rho)
    sh = O.solve(p, np.roll(rho, (2, 4, 6), axis=(0, 1, 2)))
    assert np.array_equal(sh.alpha, base.alpha)
    ref = np.roll(base.phi, (2, 4, 6), axis=(0, 1, 2))
    assert np.abs(sh.phi - ref).max() < 1e-9 * np.abs(ref).max()
    tr = O.solve(p, np.ascontiguousarray(rho.transpose(2, 0, 1)))
    ref = base.phi.transpose(2, 0, 1)
    assert np.abs(tr.phi - ref).max() < 1e-9 * np.abs(ref).max()


def test_replayed_alpha_reproduces_the_solve():
    n = 16
    pos, _ = lpt_particles(n, 100.0, 4, order=1)
    rho = O.cic_deposit((n, n, n), pos / (100.0 / n))
    p = O.OracleParams(n=(n, n, n), k_max=5)
    a = O.solve(p, rho)
    b = O.solve(p, rho, replay_alpha=np.r_[a.alpha, np.zeros(5 - a.steps)])
    assert np.array_equal(a.phi, b.phi)


def test_warm_start_reaches_the_same_solution_in_fewer_cycles():
    """Each step's linear solve from 0 (warm_start = 0), from the last step's
    phidot (1) or from its extrapolation along the step lengths (2) stops at
    the same residual: converged to rounding (tol_in 1e-12) the solves agree
    to rounding, at the default tolerance they agree to the size of that
    tolerance and the warm starts need fewer V-cycles, the extrapolation
    fewest; the first step, which has no earlier solution, is the same."""
    n = 32
    pos, _ = lpt_particles(n, 50.0, 6, order=2)
    rho = O.cic_deposit((n, n, n), pos / (50.0 / n))
    runs = {}
    for tol in (1e-12, 1e-8):
        for ws in (0, 1, 2):
            runs[tol, ws] = O.solve(O.OracleParams(n=(n, n, n), k_max=8, tol_in=tol, max_vcycles=200,
                                                   warm_start=ws), rho)
    for tol in (1e-12, 1e-8):
        cold = runs[tol, 0]
        for ws in (1, 2):
            warm = runs[tol, ws]
            assert cold.steps == warm.steps == 8 and np.array_equal(cold.alpha, warm.alpha)
            assert cold.ncycles[0] == warm.ncycles[0]
            assert np.all(warm.relres <= tol)
    conv = runs[1e-12, 0].phi
    rel = lambda r: np.linalg.norm(r.phi - conv) / np.linalg.norm(conv)
    assert rel(runs[1e-12, 1]) < 1e-11 and rel(runs[1e-12, 2]) < 1e-11
    for ws in (0, 1, 2):
        assert rel(runs[1e-8, ws]) < 1e-6
    total = {ws: runs[1e-8, ws].ncycles[1:].sum() for ws in (0, 1, 2)}
    assert total[2] <= total[1] < total[0], total


@pytest.mark.parametrize("bad", ["dims", "negative", "zero", "nan"])
def test_invalid_inputs_are_rejected(bad):
    n = (16, 8, 8)
    rho = np.ones(n)
    p = O.OracleParams(n=n)
    if bad == "dims":
        p = O.OracleParams(n=(12, 8, 8))
        rho = np.ones((12, 8, 8))
    elif bad == "negative":
        rho[1, 2, 3] = -1.0
    elif bad == "zero":
        rho[:] = 0.0
    else:
        rho[0, 0, 0] = np.nan
    with pytest.raises(RuntimeError):
        O.solve(p, rho)


def test_paper_literal_density_update():
    """App. A's variant: the mass per cell is carried by its exact linear change
    m += alpha d_mu(m e^-1 d dphi) instead of re-depositing tracers.  Mass is
    conserved to rounding, the map stays positive definite above the floor, and
    the first step coincides with the tracer form (both start from m = rho)."""
    n, box = 16, 100.0
    pos, _ = lpt_particles(n, box, 4, order=1)
    rho = O.cic_deposit((n, n, n), pos / (box / n))
    p = O.OracleParams(n=(n, n, n), k_max=8, density_update=1)
    r = O.solve(p, rho)
    assert r.steps == 8
    assert np.all(np.abs(r.mass - n ** 3) < 1e-9 * n ** 3)
    assert abs(r.m.sum() - n ** 3) < 1e-9 * n ** 3
    assert np.all(r.min_det > 0) and np.all(r.min_lam > p.lambda_floor)
    a = O.solve(O.OracleParams(n=(n, n, n), k_max=1, density_update=1), rho)
    b = O.solve(O.OracleParams(n=(n, n, n), k_max=1), rho)
    assert np.array_equal(a.phi, b.phi)
    u = O.solve(O.OracleParams(n=(16, 8, 8), density_update=1), np.full((16, 8, 8), 2.0))
    assert u.status == 0 and u.steps == 0


def test_thread_count_does_not_change_a_bit():
    """The OpenMP build splits only loops with independent iterations over
    threads and keeps every sum serial, so 1 and 4 threads give the same bits
    (a whole solve with the limiter active, and the operators on their own)."""
    n, box = 16, 50.0
    pos, _ = lpt_particles(n, box, 3, order=2)
    rho = O.cic_deposit((n, n, n), pos / (box / n))
    p = O.OracleParams(n=(n, n, n), k_max=6)
    old = O.set_threads()
    try:
        outs = []
        for t in (1, 4):
            O.set_threads(t)
            r = O.solve(p, rho)
            outs.append((r.phi, r.xi, r.alpha, r.ncycles, O.geometry(r.phi)[1],
                         O.apply_S(r.phi), O.delta_r(r.phi)))
        for a, b in zip(*outs):
            assert np.array_equal(a, b)
    finally:
        O.set_threads(old)
