"""Limiter parameter sweeps of App. B (Figs. 6 and 7) on synthetic inputs.

The paper studies how the reconstruction depends on the maximal compression
factor xi_m (1/5, 1/10, 1/20 at v_m = 10) and on the expansion volume limit
v_m (5, 10, 20 at xi_m = 1/10) through the cross-correlation r(k) between
the reconstructed density delta_r and the linear field.  This module runs
those settings through the GPU solve (recon_solve_batch, one handle per
setting) on one of the package's synthetic workloads, for which the linear
field delta_L is known, and returns r(k) with each solve's record.  Either
density representation can be used (density_update 0: tracer re-deposit,
1: App. A's linear update).

    python -m paper_1611_09638_gb300.sweeps --workload lpt256 --out sweep.json
"""
import argparse
import json

import numpy as np

from . import Recon, solve_batch
from .diag import cross_correlation
from .inputs import WORKLOADS

XI_M_SWEEP = [(0.2, 10.0), (0.1, 10.0), (0.05, 10.0)]  # (xi_m, v_m), Fig. 6
V_M_SWEEP = [(0.1, 5.0), (0.1, 10.0), (0.1, 20.0)]     # Fig. 7


def run(workload="lpt256", settings=None, precision="mixed", k_max=40, density_update=0,
        kmax_report=1.0):
    """Solve the workload once per (xi_m, v_m) setting and return a list of
    records: the setting, the solve's status / steps / V-cycles / R_k, the
    end-of-solve invariants, and r(k) of delta_r against delta_L for
    k <= kmax_report h/Mpc (shells of width 2 pi / box)."""
    import torch

    W = WORKLOADS[workload]
    n = W.n
    pos, delta_L = W.particles()
    settings = list(settings) if settings is not None else XI_M_SWEEP + V_M_SWEEP[::2]
    pos_dev = torch.from_numpy(pos).cuda()
    torch.cuda.synchronize()
    recons = []
    for xi_m, v_m in settings:
        R = Recon((n, n, n), box=W.box, precision=precision, stream=torch.cuda.Stream(),
                  xi_m=float(xi_m), v_m=float(v_m), k_max=int(k_max),
                  density_update=int(density_update))
        R.deposit_particles(pos_dev)
        recons.append(R)
    stats = solve_batch(recons)
    out = []
    for (xi_m, v_m), R, st in zip(settings, recons, stats):
        dr = R.field("delta_r").cpu().numpy()
        k, r = cross_correlation(dr, delta_L, W.box)
        keep = (k > 0) & (k <= kmax_report)
        out.append({
            "xi_m": float(xi_m), "v_m": float(v_m), "status": int(st.status),
            "steps": int(st.steps), "vcycles": int(st.vcycles), "R0": float(st.R0),
            "R": float(st.R), "Rk": [float(x) for x in st.Rk],
            "min_lambda0": float(st.min_lambda0), "max_delta_r": float(st.max_delta_r),
            "k": [float(x) for x in k[keep]], "r": [float(x) for x in r[keep]],
        })
        R.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="lpt256", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--k-max", type=int, default=40)
    ap.add_argument("--density-update", type=int, default=0, choices=[0, 1])
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res = {"workload": WORKLOADS[a.workload].name, "precision": a.precision,
           "density_update": a.density_update,
           "runs": run(a.workload, None, a.precision, a.k_max, a.density_update)}
    text = json.dumps(res)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(text)
    print(text)


if __name__ == "__main__":
    main()
