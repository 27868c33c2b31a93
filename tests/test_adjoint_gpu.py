"""The GPU adjoint (recon_adjoint: dL/d rho from dL/d delta_r, the step
lengths held at the solve's values) against the oracle's adjoint, which is
pinned by finite differences (tests/test_oracle_adjoint.py), and against
central finite differences of the GPU's own solve: on 64 cells of the
32^3 / 100 Mpc/h ZA workload, and on the 128^3 / 200 Mpc/h ZA configuration
with the loss L = sum_k w(k) |delta_r(k) - delta_L(k)|^2, w = 1 for
k < 0.5 h/Mpc, along a random direction and on 64 random cells, in FP64 and
in mixed precision.

Finite differences use FP64 solves to a 1e-13 relative residual with the
base solve's step lengths replayed, so that they resolve the derivative.
"""
import numpy as np
import pytest

import oracle as O
from paper_1611_09638_gb300 import ReconError, Recon, reconstruct
from paper_1611_09638_gb300.inputs import lpt_particles

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _density(n, box, seed):
    pos, dL = lpt_particles(n, box, seed, order=1)
    return O.cic_deposit((n, n, n), pos / (box / n)), dL


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _delta_r(R, rho):
    R.deposit_grid(_dev(rho))
    R.solve(record=False)
    return R.field("delta_r").cpu().numpy()


def c4_loss(delta_r, delta_L, box, kcut=0.5):
    """L = sum_k w(k) |F(k)|^2 over the full FFT of delta_r - delta_L, w = 1
    for |k| < kcut h/Mpc; returns (L, dL/d delta_r)."""
    n = delta_r.shape[0]
    F = np.fft.fftn(delta_r - delta_L)
    k1 = np.fft.fftfreq(n, d=box / n) * 2 * np.pi
    kk = np.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + k1[None, None, :] ** 2)
    W = (kk < kcut).astype(float)
    L = float(np.sum(W * np.abs(F) ** 2))
    g = 2.0 * n ** 3 * np.real(np.fft.ifftn(W * F))
    return L, g


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-5), ("mixed", 1e-4)])
def test_adjoint_matches_the_oracle(precision, tol):
    n, box = 32, 100.0
    rho, _ = _density(n, box, 1000)
    with Recon((n, n, n), box=box, precision=precision, k_max=8, checkpoint=1) as R:
        R.deposit_grid(_dev(rho))
        st = R.solve()
        gbar = np.random.default_rng(4).standard_normal((n, n, n))
        g = R.adjoint(_dev(gbar)).cpu().numpy()
        g2 = R.adjoint(gbar, np.empty((n, n, n)))  # host buffers; atomics: equal to rounding
        assert rel(g2, g) <= 1e-12
        # the solve's outputs are unchanged by the sweep
        phi = R.field("phi").cpu().numpy()
    ref = O.adjoint(O.OracleParams(n=(n, n, n), k_max=8), rho, st.alpha, gbar)
    assert st.steps == 8
    assert rel(g, ref) <= tol, rel(g, ref)
    assert np.isfinite(phi).all()


def test_adjoint_matches_finite_differences_on_64_cells():
    n, box = 32, 100.0
    rho, _ = _density(n, box, 1000)
    kw = dict(box=box, precision="fp64", k_max=6, tol_in=1e-13, max_vcycles=200)
    with Recon((n, n, n), checkpoint=1, **kw) as R:
        R.deposit_grid(_dev(rho))
        st = R.solve()
        gbar = np.random.default_rng(5).standard_normal((n, n, n))
        g = R.adjoint(_dev(gbar)).cpu().numpy().ravel()
    rng = np.random.default_rng(3000)
    cells = rng.choice(np.flatnonzero(rho.ravel() > 1e-3 * rho.mean()), 64, replace=False)
    eps = 1e-5 * rho.mean()
    scale = np.abs(g).max()
    bad = []
    with Recon((n, n, n), replay_alpha=st.alpha, **kw) as F:
        for c in cells:
            e = np.zeros(rho.size)
            e[c] = eps
            e = e.reshape(rho.shape)
            fd = (np.sum(gbar * _delta_r(F, rho + e)) - np.sum(gbar * _delta_r(F, rho - e))) / (2 * eps)
            if abs(g[c] - fd) > 1e-4 * max(abs(fd), 1e-2 * scale):
                bad.append((int(c), g[c], fd))
    assert not bad, bad


def test_adjoint_of_the_band_limited_loss_at_128_cubed():
    """C4: 128^3 / 200 Mpc/h ZA (seed 1004), FP64 and mixed; the directional
    derivative along a random positive direction by central differences."""
    n, box = 128, 200.0
    rho, dL = _density(n, box, 1004)
    kw = dict(box=box, k_max=10, tol_in=1e-13, max_vcycles=200)
    with Recon((n, n, n), precision="fp64", checkpoint=1, **kw) as R:
        R.deposit_grid(_dev(rho))
        st = R.solve()
        L0, gbar = c4_loss(R.field("delta_r").cpu().numpy(), dL, box)
        g = R.adjoint(_dev(gbar)).cpu().numpy()
    d = np.random.default_rng(3000).random((n, n, n)) * rho
    eps = 1e-6
    with Recon((n, n, n), precision="fp64", replay_alpha=st.alpha, **kw) as F:
        Lp, _ = c4_loss(_delta_r(F, rho + eps * d), dL, box)
        Lm, _ = c4_loss(_delta_r(F, rho - eps * d), dL, box)
    fd = (Lp - Lm) / (2 * eps)
    assert abs(np.sum(g * d) - fd) <= 1e-4 * abs(fd), (np.sum(g * d), fd)
    # the mixed-precision adjoint of the same solve: it takes the same step
    # lengths, and its gradient matches the FP64 one
    with Recon((n, n, n), precision="mixed", checkpoint=1, box=box, k_max=10, tol_in=1e-12,
               max_vcycles=300) as R:
        R.deposit_grid(_dev(rho))
        stm = R.solve()
        np.testing.assert_array_equal(stm.alpha, st.alpha)
        gm = R.adjoint(_dev(gbar)).cpu().numpy()
    assert rel(gm, g) <= 1e-4


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c4_gradient_matches_finite_differences_on_64_cells(precision):
    """C4 as configured: 128^3 / 200 Mpc/h ZA (seed 1004), the band-limited
    loss L = sum_k w(k) |delta_r(k) - delta_L(k)|^2 (w = 1 for k < 0.5 h/Mpc),
    its gradient with respect to the deposited density from the checkpointed
    adjoint in FP64 and in mixed precision, against central finite
    differences on 64 random cells (seed 3000) to 1e-4 relative.  The
    differences are taken on FP64 solves to a 1e-13 relative residual with the
    adjoint solve's step lengths replayed (the derivative holds them fixed);
    a cell whose derivative is below 1e-2 of the largest one is compared to
    1e-4 of that floor instead of its own size."""
    n, box, K = 128, 200.0, 10
    rho, dL = _density(n, box, 1004)
    tight = dict(tol_in=1e-13 if precision == "fp64" else 1e-12,
                 max_vcycles=200 if precision == "fp64" else 300)
    with Recon((n, n, n), box=box, precision=precision, k_max=K, checkpoint=1, **tight) as R:
        R.deposit_grid(_dev(rho))
        st = R.solve()
        assert st.steps == K
        _, gbar = c4_loss(R.field("delta_r").cpu().numpy(), dL, box)
        g = R.adjoint(_dev(gbar)).cpu().numpy().ravel()
    rng = np.random.default_rng(3000)
    cells = rng.choice(np.flatnonzero(rho.ravel() > 1e-3 * rho.mean()), 64, replace=False)
    eps = 1e-5 * rho.mean()
    floor = 1e-2 * np.abs(g).max()
    bad = []
    with Recon((n, n, n), box=box, precision="fp64", k_max=K, replay_alpha=st.alpha,
               tol_in=1e-13, max_vcycles=200) as F:
        for c in cells:
            e = np.zeros(rho.size)
            e[c] = eps
            e = e.reshape(rho.shape)
            Lp, _ = c4_loss(_delta_r(F, rho + e), dL, box)
            Lm, _ = c4_loss(_delta_r(F, rho - e), dL, box)
            fd = (Lp - Lm) / (2 * eps)
            if abs(g[c] - fd) > 1e-4 * max(abs(fd), floor):
                bad.append((int(c), g[c], fd))
    assert not bad, bad


def test_autograd_function_and_errors():
    n, box = 16, 50.0
    rho, _ = _density(n, box, 7)
    with Recon((n, n, n), box=box, k_max=4, checkpoint=1) as R:
        with pytest.raises(ReconError):  # no solve yet
            R.adjoint(_dev(np.zeros((n, n, n))))
        r = _dev(rho).requires_grad_(True)
        dr = reconstruct(R, r)
        gbar = torch.from_numpy(np.random.default_rng(1).standard_normal((n, n, n))).cuda()
        (dr * gbar).sum().backward()
        direct = R.adjoint(gbar)
        assert torch.allclose(r.grad, direct, rtol=1e-10, atol=1e-12 * direct.abs().max().item())
    with Recon((n, n, n), box=box, k_max=2) as R:
        R.deposit_grid(_dev(rho))
        R.solve()
        with pytest.raises(ReconError):  # created without checkpoints
            R.adjoint(_dev(np.zeros((n, n, n))))
