"""The allocation-free CIC deposit (recon_deposit_cic_noalloc).

Some callers cannot allocate device memory where they need a deposit (under an
allocator that must account for all device memory, in loops that must not
stall on an allocation); this entry point keeps its scratch in a fixed device
array of the library instead.  It must give the same density as
recon_deposit(RECON_PARTICLES), on consecutive calls that reuse the scratch.
This file is collected last so that a failure here cannot hide another test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _noalloc(lib, n, cell, pos, mass, out):
    return lib.recon_deposit_cic_noalloc(
        n[0], n[1], n[2], cell, C.c_void_p(pos.data_ptr()),
        None if mass is None else C.c_void_p(mass.data_ptr()), int(pos.shape[0]),
        C.c_void_p(out.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_deposit_matches_recon_deposit_on_consecutive_calls():
    from paper_1611_09638_gb300 import Recon, _abi

    lib = _abi.load()
    cases = [((64, 64, 64), 100.0, 7, True), ((128, 32, 64), 50.0, 8, False)]
    for n, box, seed, with_mass in cases:  # two calls in a row, different inputs
        rng = np.random.default_rng(seed)
        cell = box / n[0]
        npart = 200_000
        x = rng.uniform(-0.5 * box, 1.5 * box, size=(npart, 3))
        w = rng.uniform(0.0, 3.0, size=npart) if with_mass else None
        pos = torch.from_numpy(x).cuda()
        mass = None if w is None else torch.from_numpy(w).cuda()
        out = torch.full(n, -1.0, dtype=torch.float64, device="cuda")
        assert _noalloc(lib, n, cell, pos, mass, out) == _abi.RECON_OK, _abi.last_error()
        torch.cuda.synchronize()
        with Recon(n, box=tuple(cell * v for v in n)) as R:
            R.deposit_particles(pos, mass)
            ref = R.field("density").cpu().numpy()
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-10 * ref.max()
        total = float(w.sum()) if w is not None else float(npart)
        assert abs(got.sum() - total) <= 1e-9 * total


def test_noalloc_deposit_rejects_grids_beyond_its_scratch_and_host_pointers():
    from paper_1611_09638_gb300 import _abi

    lib = _abi.load()
    pos = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    out = torch.empty((256, 128, 128), dtype=torch.float64, device="cuda")
    assert _noalloc(lib, (256, 128, 128), 1.0, pos, None, out) == _abi.RECON_E_INVALID
    assert "limit" in _abi.last_error()
    host = torch.zeros((8, 8, 8), dtype=torch.float64)
    assert _noalloc(lib, (8, 8, 8), 1.0, pos, None, host) == _abi.RECON_E_INVALID


def test_noalloc_deposit_rejected_inputs_leave_the_next_call_correct():
    """Every rejected input (NaN position, negative mass, zero total mass, a
    host mass array) returns its status, and the valid call after it, which
    reads the scratch those calls wrote, still matches recon_deposit."""
    from paper_1611_09638_gb300 import Recon, _abi

    lib = _abi.load()
    n, box = (8, 8, 8), 10.0
    cell = box / n[0]
    rng = np.random.default_rng(21)
    x = rng.uniform(0.0, box, size=(4000, 3))
    w = rng.uniform(0.5, 1.5, size=4000)
    pos, mass = torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda()
    with Recon(n, box=box) as R:
        R.deposit_particles(pos, mass)
        ref = R.field("density").cpu().numpy()
    bad_pos = pos.clone()
    bad_pos[17, 1] = float("nan")
    neg = mass.clone()
    neg[5] = -1.0
    cases = [(bad_pos, mass, _abi.RECON_E_NONFINITE),
             (pos, neg, _abi.RECON_E_NONFINITE),
             (pos, torch.zeros_like(mass), _abi.RECON_E_INVALID),
             (pos, mass.cpu(), _abi.RECON_E_INVALID)]
    for p_, m_, want in cases:
        out = torch.full(n, -1.0, dtype=torch.float64, device="cuda")
        assert _noalloc(lib, n, cell, p_, m_, out) == want, _abi.last_error()
        assert _noalloc(lib, n, cell, pos, mass, out) == _abi.RECON_OK, _abi.last_error()
        torch.cuda.synchronize()
        assert np.abs(out.cpu().numpy() - ref).max() <= 1e-10 * ref.max()
