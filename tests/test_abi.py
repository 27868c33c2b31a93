"""The C ABI loads and exports every function include/recon.h declares; the
host-only entry points behave as documented (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "recon.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(recon_\w+)\s*\(", text, re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1611_09638_gb300 import _abi

    lib = _abi.load()
    declared = _declared()
    assert len(declared) >= 8
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) <= set(_abi.SYMBOLS)


def test_default_params_match_the_paper_and_the_oracle():
    """The FP64 defaults are the oracle's; the multigrid settings are left at
    -1 and resolved by precision (FP64: V(2, 2), 50 cycles per step)."""
    from paper_1611_09638_gb300 import default_params, resolved_params
    import oracle as O

    p = default_params((32, 16, 8))
    assert (p.nu1, p.nu2, p.inner_vcycles, p.max_vcycles) == (-1, -1, -1, -1)
    p = resolved_params((32, 16, 8))
    q = O.OracleParams()
    assert list(p.n) == [32, 16, 8]
    for f in ("xi_m", "v_m", "a_min", "climiter", "s_side", "nu1", "nu2", "tol_in", "max_vcycles",
              "tol_out", "k_max", "d_max", "alpha_min", "lambda_floor", "density_update",
              "warm_start"):
        assert getattr(p, f) == getattr(q, f), f


def test_mixed_precision_defaults_and_explicit_settings_resolve():
    """Mixed precision resolves to V(1, 1) FP32 cycles, 6 per FP64 defect
    correction and 100 per step; explicit values are kept."""
    from paper_1611_09638_gb300 import resolved_params

    p = resolved_params((16, 16, 16), precision="mixed")
    assert (p.nu1, p.nu2, p.inner_vcycles, p.max_vcycles, p.coarse_faces) == (1, 1, 6, 100, 0)
    # per-face coarse coefficients on cubic grids of at least 64^3, with
    # shorter groups of V-cycles; not in FP64, not on other grids
    p = resolved_params((64, 64, 64), precision="mixed")
    assert (p.inner_vcycles, p.coarse_faces) == (5, 1)
    assert resolved_params((64, 64, 64), precision="fp64").coarse_faces == 0
    assert resolved_params((128, 64, 64), precision="mixed").coarse_faces == 0
    p = resolved_params((64, 64, 64), precision="mixed", coarse_faces=0)
    assert (p.inner_vcycles, p.coarse_faces) == (6, 0)
    p = resolved_params((16, 16, 16), precision="mixed", nu1=2, nu2=3, inner_vcycles=4, max_vcycles=7)
    assert (p.nu1, p.nu2, p.inner_vcycles, p.max_vcycles) == (2, 3, 4, 7)
    p = resolved_params((16, 16, 16), precision="fp64", nu1=1)
    assert (p.nu1, p.nu2) == (1, 2)


def test_struct_layout_matches_header(tmp_path):
    """ctypes mirrors of recon_params / recon_stats have the C compiler's
    sizes and field offsets."""
    import subprocess

    from paper_1611_09638_gb300 import _abi

    src = tmp_path / "lay.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "recon.h"', "int main(void){"]
    for st in (_abi.recon_params, _abi.recon_stats):
        lines.append(f'printf("%zu\\n", sizeof({st.__name__}));')
        for f, _ in st._fields_:
            lines.append(f'printf("%zu\\n", offsetof({st.__name__}, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "lay"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    want = []
    for st in (_abi.recon_params, _abi.recon_stats):
        want.append(C.sizeof(st))
        want += [getattr(st, f).offset for f, _ in st._fields_]
    assert got == want


def test_errors_are_reported_as_status_and_text():
    from paper_1611_09638_gb300 import _abi

    lib = _abi.load()
    assert lib.recon_adjoint(None, None, None) == _abi.RECON_E_INVALID
    assert b"NULL" in lib.recon_last_error()
    assert lib.recon_solve(None, None) == _abi.RECON_E_INVALID


def test_create_rejects_bad_params_before_touching_the_device():
    from paper_1611_09638_gb300 import _abi, default_params

    lib = _abi.load()
    h = C.c_void_p()
    for bad in ({"xi_m": 1.5}, {"v_m": 0.5}, {"nu1": 0, "nu2": 0}, {"s_side": 0.3},
                {"device_loop": 2}, {"density_update": 3}, {"inner_vcycles": 0},
                {"inner_vcycles": 17}, {"nu1": -2}, {"max_vcycles": 0},
                {"checkpoint": 2}, {"checkpoint": 1, "density_update": 1}):
        p = default_params((16, 16, 16), **bad)
        assert lib.recon_create(C.byref(h), C.byref(p), None) == _abi.RECON_E_INVALID
        assert h.value is None
    p = default_params((12, 16, 16))
    assert lib.recon_create(C.byref(h), C.byref(p), None) == _abi.RECON_E_INVALID
    p = default_params((16, 16, 32), box=(100.0, 100.0, 100.0))  # non-cubic cells
    assert lib.recon_create(C.byref(h), C.byref(p), None) == _abi.RECON_E_INVALID


def test_solve_runs_on_the_device_loop_by_default():
    """The default solve is the graph-resident one; profile switches it to
    the host-driven loop (documented in recon.h)."""
    from paper_1611_09638_gb300 import default_params

    assert default_params((16, 16, 16)).device_loop == 1
    assert default_params((16, 16, 16)).checkpoint == 0
    assert default_params((16, 16, 16)).tma == 1  # bulk-copy staging on by default
    assert default_params((16, 16, 16), device_loop=0).device_loop == 0


def test_batch_solve_rejects_bad_arguments_without_a_gpu():
    from paper_1611_09638_gb300 import _abi

    lib = _abi.load()
    hs = (C.c_void_p * 2)(None, None)
    assert lib.recon_solve_batch(hs, 2, None) == _abi.RECON_E_INVALID
    assert lib.recon_solve_batch(None, 1, None) == _abi.RECON_E_INVALID
    assert lib.recon_solve_batch(None, -1, None) == _abi.RECON_E_INVALID
    assert lib.recon_solve_batch(None, 0, None) == _abi.RECON_OK


def test_package_has_no_cpu_fallback():
    import paper_1611_09638_gb300 as R
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        R.Recon((16, 16, 16))


def test_resolve_params_touches_only_the_multigrid_settings():
    """recon_resolve_params replaces only the -1 multigrid entries and rejects
    a NULL pointer with a status and a message."""
    from paper_1611_09638_gb300 import _abi, default_params

    lib = _abi.load()
    p = default_params((16, 32, 64), box=(1.0, 2.0, 4.0), precision="mixed", k_max=7, tol_in=1e-6)
    skip = ("nu1", "nu2", "inner_vcycles", "max_vcycles", "coarse_faces", "group_max", "n", "box",
            "replay_alpha")
    before = {f: getattr(p, f) for f, _ in _abi.recon_params._fields_ if f not in skip}
    assert lib.recon_resolve_params(C.byref(p)) == _abi.RECON_OK
    after = {f: getattr(p, f) for f in before}
    assert after == before and list(p.n) == [16, 32, 64] and list(p.box) == [1.0, 2.0, 4.0]
    assert not p.replay_alpha  # still NULL
    assert lib.recon_resolve_params(None) == _abi.RECON_E_INVALID
    assert b"NULL" in lib.recon_last_error()


def test_checked_library_builds_and_exports_the_same_entry_points():
    """librecon_checked.so (the RECON_CHECKED build) compiles for sm_103a and
    exports the entry points of librecon.so."""
    import subprocess

    from paper_1611_09638_gb300 import build as B

    def exported(path):
        out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                             check=True).stdout
        return {ln.split()[-1] for ln in out.splitlines() if ln.split()[-1].startswith("recon_")}

    plain, checked = exported(B.build()), exported(B.build(checked=True))
    assert plain and plain == checked
