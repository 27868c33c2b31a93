"""The graph-resident solve (device_loop = 1: the step loop, the multigrid
loop and the step acceptance are conditional nodes of one CUDA graph whose
conditions device kernels set) against the host-driven loop, and the batched
solve against single solves.

Both loops launch the same kernels in the same order and take every decision
(R_k <= tol_out, the multigrid stopping test, alpha and the stall) in the
same device kernels, so their results must agree bit for bit: states,
per-step records, statuses and kernel counts.
"""
import numpy as np
import pytest

import oracle as O
from paper_1611_09638_gb300 import Recon, solve_batch
from paper_1611_09638_gb300.inputs import lpt_particles

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _density(n, box, seed, order=1):
    pos, _ = lpt_particles(n, box, seed, order=order)
    return O.cic_deposit((n, n, n), pos / (box / n))


def _run(rho, precision, device_loop, stream=None, **kw):
    n = rho.shape
    R = Recon(n, precision=precision, device_loop=device_loop, stream=stream, **kw)
    R.deposit_grid(torch.from_numpy(np.ascontiguousarray(rho)).cuda(R.stream.device))
    st = R.solve()
    phi = R.field("phi").cpu().numpy()
    return R, st, phi


def _same(a, b, pa, pb):
    assert a.status == b.status and a.steps == b.steps and a.vcycles == b.vcycles
    for f in ("alpha", "Rk", "ncycles", "relres"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    for f in ("R0", "R", "min_det", "min_lambda0", "max_delta_r", "mass_error"):
        assert getattr(a, f) == getattr(b, f), f
    assert a.launches == b.launches
    assert np.array_equal(pa, pb)


@pytest.mark.parametrize("precision,kw", [("fp64", {}), ("mixed", {}),
                                          ("mixed", {"inner_vcycles": 3, "group_max": 12})])
def test_device_loop_equals_host_loop(precision, kw):
    """Both loops, also with grouped FP64 checks (the device decides after
    each block of V-cycles whether to form the FP64 residual)."""
    rho = _density(32, 100.0, 1000)
    Ra, a, pa = _run(rho, precision, 0, **kw)
    Rb, b, pb = _run(rho, precision, 1, **kw)
    assert a.steps > 10
    _same(a, b, pa, pb)
    # a second solve on the same handle replays the recorded graph
    b2 = Rb.solve()
    _same(a, b2, pa, Rb.field("phi").cpu().numpy())
    Ra.close(), Rb.close()


def test_device_loop_stall_replay_and_edge_cases():
    rho = _density(16, 50.0, 3, order=2)
    # stall (status 2) with an unreachable eigenvalue floor
    Ra, a, pa = _run(rho, "fp64", 0, lambda_floor=0.6)
    Rb, b, pb = _run(rho, "fp64", 1, lambda_floor=0.6)
    assert a.status == 2
    _same(a, b, pa, pb)
    # replayed alpha sequence
    ra = np.r_[a.alpha, np.full(40 - len(a.alpha), 0.5)]
    Ra, a, pa = _run(rho, "mixed", 0, replay_alpha=ra, k_max=40)
    Rb, b, pb = _run(rho, "mixed", 1, replay_alpha=ra, k_max=40)
    _same(a, b, pa, pb)
    assert np.array_equal(b.alpha, ra[:b.steps])
    # no steps at all, and a stop at the first step start
    for kw in ({"k_max": 0}, {"tol_out": 1e9}, {"k_max": 1}):
        Ra, a, pa = _run(rho, "mixed", 0, **kw)
        Rb, b, pb = _run(rho, "mixed", 1, **kw)
        _same(a, b, pa, pb)
    assert b.steps == 1 and b.status == 1
    # uniform density: R_0 = 0, immediate stop with phi = 0
    Rb, b, pb = _run(np.full((8, 8, 8), 2.0), "fp64", 1)
    assert b.status == 0 and b.steps == 0 and not pb.any()
    # the paper-literal density update
    Ra, a, pa = _run(rho, "fp64", 0, density_update=1, k_max=6)
    Rb, b, pb = _run(rho, "fp64", 1, density_update=1, k_max=6)
    _same(a, b, pa, pb)


def test_batch_of_mixed_sizes_equals_single_solves():
    """Mocks of three sizes (3.125 Mpc/h cells), each on its own stream, one of
    them on the host-driven loop: the batched solve reproduces every single
    solve bit for bit."""
    specs = [(16, 50.0), (32, 100.0), (64, 200.0), (16, 50.0), (32, 100.0), (64, 200.0)]
    rhos = [_density(n, box, 2000 + i) for i, (n, box) in enumerate(specs)]
    single = []
    for i, rho in enumerate(rhos):
        R, st, phi = _run(rho, "mixed", 1 if i != 4 else 0)
        single.append((st, phi))
        R.close()
    recons = []
    for i, rho in enumerate(rhos):
        R = Recon(rho.shape, precision="mixed", device_loop=1 if i != 4 else 0,
                  stream=torch.cuda.Stream())
        torch.cuda.synchronize()
        R.deposit_grid(torch.from_numpy(np.ascontiguousarray(rho)).cuda())
        recons.append(R)
    torch.cuda.synchronize()
    for rep in range(2):
        out = solve_batch(recons)
        for R, st, (st1, phi1) in zip(recons, out, single):
            _same(st1, st, phi1, R.field("phi").cpu().numpy())
    for R in recons:
        R.close()


def test_batch_matches_the_oracle():
    """A batch of mocks of three sizes (ZA, 3.125 Mpc/h cells, seeds 2000 + i)
    solved together in mixed precision: every mock against the oracle's solve
    of it, 10 steps at the default tolerances -- the same step lengths,
    status and step count, and phi within 1e-4."""
    specs = [(16, 50.0), (32, 100.0), (64, 200.0), (16, 50.0), (32, 100.0)]
    K = 10
    rhos = [_density(n, box, 2000 + i) for i, (n, box) in enumerate(specs)]
    recons = []
    for rho in rhos:
        R = Recon(rho.shape, precision="mixed", k_max=K, stream=torch.cuda.Stream())
        torch.cuda.synchronize()
        R.deposit_grid(torch.from_numpy(np.ascontiguousarray(rho)).cuda())
        recons.append(R)
    torch.cuda.synchronize()
    out = solve_batch(recons)
    for R, st, rho in zip(recons, out, rhos):
        ref = O.solve(O.OracleParams(n=rho.shape, k_max=K), rho)
        assert st.status == ref.status and st.steps == ref.steps
        np.testing.assert_array_equal(st.alpha, ref.alpha)
        phi = R.field("phi").cpu().numpy()
        assert np.linalg.norm(phi - ref.phi) <= 1e-4 * np.linalg.norm(ref.phi)
        R.close()


def test_limiter_parameter_sweep_runs_every_setting():
    """The App. B sweep driver on the 32^3 workload: every (xi_m, v_m) setting
    gives a valid map and an r(k) record; the settings share the input."""
    from paper_1611_09638_gb300 import sweeps

    out = sweeps.run("za32", settings=sweeps.XI_M_SWEEP + sweeps.V_M_SWEEP, k_max=8)
    assert len(out) == 6
    for rec in out:
        assert rec["status"] in (0, 1, 2) and rec["min_lambda0"] > 0.0
        assert len(rec["k"]) == len(rec["r"]) > 3 and max(abs(x) for x in rec["r"]) <= 1.0
        assert rec["R0"] == out[0]["R0"]  # the first step's source does not see C or E at phi = 0
    # the duplicated (1/10, 10) setting is the same solve
    a = [r for r in out if r["xi_m"] == 0.1 and r["v_m"] == 10.0]
    assert len(a) == 2 and a[0]["r"] == a[1]["r"] and a[0]["Rk"] == a[1]["Rk"]
