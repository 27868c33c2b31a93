"""The bounds-checked build (RECON_CHECKED, librecon_checked.so).

Its kernels check every shared- and global-memory offset they compute (the
streaming sweep and residual restriction, the cluster's plane owners, the
tiled deposit) and report a failed check as a status instead of trapping.
Here a set of solves that reaches every such kernel and launch shape (odd and
anisotropic grids, FP64 and mixed precision, each planes-per-block choice of
the streaming kernels, bulk-copy and per-thread staging, the face-sum coarse
levels, the adjoint) runs once under the checked build in a child process,
which fails on any reported check, and once under the normal build; phi and
the step records must agree bit for bit and the gradient to rounding.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (grid, precision, extra parameters); two steps each
CASES = [
    ((8, 8, 8), "fp64", {}),
    ((8, 8, 8), "mixed", {}),
    ((16, 8, 32), "mixed", {}),
    ((64, 32, 16), "fp64", {}),
    ((64, 32, 16), "mixed", {}),
    ((64, 64, 64), "mixed", {}),
    ((128, 64, 64), "mixed", {"stream_planes": 4, "restrict_planes": 1}),
    ((128, 64, 64), "mixed", {"stream_planes": 16, "restrict_planes": 16, "coarse_faces": 0}),
    ((32, 64, 256), "mixed", {"tma": 1}),
    ((32, 64, 256), "mixed", {"tma": 0, "stream_planes": 8, "restrict_planes": 2}),
    ((128, 128, 128), "mixed", {"stream_planes": 8, "restrict_planes": 4}),
]

RUNNER = r"""
import json, sys
import numpy as np, torch
from paper_1611_09638_gb300 import Recon, _abi
cases, out = json.loads(sys.argv[1]), sys.argv[2]
_abi.load()
print("library", _abi.lib_path())
res = {}
for idx, (n, prec, kw) in enumerate(cases):
    rng = np.random.default_rng(500 + idx)
    rho = np.exp(0.8 * rng.normal(size=tuple(n)))
    with Recon(tuple(n), precision=prec, k_max=2, **kw) as R:
        R.deposit_grid(torch.from_numpy(rho).cuda())
        st = R.solve()
        res["phi%d" % idx] = R.field("phi").cpu().numpy()
        res["rec%d" % idx] = np.r_[st.status, st.steps, st.vcycles, st.alpha, st.ncycles]
n = (16, 16, 16)
rho = np.exp(0.8 * np.random.default_rng(499).normal(size=n))
g = np.random.default_rng(498).normal(size=n)
with Recon(n, precision="mixed", k_max=3, checkpoint=1) as R:
    R.deposit_grid(torch.from_numpy(rho).cuda())
    R.solve()
    res["grad"] = R.adjoint(torch.from_numpy(g).cuda()).cpu().numpy()
np.savez(out, **res)
"""


def _run(tmp_path, checked):
    env = dict(os.environ)
    env.pop("RECON_BUILD", None)
    if checked:
        env["RECON_BUILD"] = "checked"
    out = str(tmp_path / ("checked.npz" if checked else "plain.npz"))
    p = subprocess.run([sys.executable, "-c", RUNNER, json.dumps(CASES), out], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1200)
    assert p.returncode == 0, p.stderr[-3000:]
    lib = [ln for ln in p.stdout.splitlines() if ln.startswith("library ")]
    assert lib and lib[0].endswith("librecon_checked.so" if checked else "librecon.so"), p.stdout
    return np.load(out)


def test_checked_build_reports_no_failed_check_and_gives_the_same_bits(tmp_path):
    from paper_1611_09638_gb300 import build as B

    B.build(checked=True)
    chk = _run(tmp_path, True)
    plain = _run(tmp_path, False)
    assert sorted(chk.files) == sorted(plain.files)
    for key in plain.files:
        if key == "grad":  # the adjoint's scatter sums with atomics: equal to rounding
            rel = np.linalg.norm(chk[key] - plain[key]) / np.linalg.norm(plain[key])
            assert rel <= 1e-10, rel
        else:
            assert np.array_equal(chk[key], plain[key]), key
