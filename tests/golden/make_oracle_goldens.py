"""Write the oracle's stored values for the full-size parity tests.

    python tests/golden/make_oracle_goldens.py lpt256 [--threads 6] [--k-max 200]
    python tests/golden/make_oracle_goldens.py lpt512 --k-max 1 --tag step1

Runs the CPU FP64 oracle (oracle/, and nothing else of this repository but
the seeded input generator) on one workload twice:
  A  the free-running solve with a tight inner tolerance (tol_in = 1e-12), so
     that each step's linear solve is exact to rounding and the trajectory is
     the method's own, not its inner solver's (at most --k-max steps);
  B  the same solve at the default inner tolerance (tol_in = 1e-8) with A's
     step lengths replayed, as the timed solve runs.
It stores, for each: the per-step record, phi on seeded sample nodes, the
Fourier modes of phi with |m| <= 6 (m the integer wave vector), and r(k)
between delta_r = -lap phi and the seed's linear field for k <= 1 h/Mpc; for
A also m, sqrt(g) and lambda0 on the sample nodes.  The relative L2 distance
of B's phi from A's (the whole field) is what the inner tolerance alone moves
the result by.  Output: tests/golden/<workload>[_<tag>]_oracle.npz.
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from oracle.spectra import cross_correlation  # noqa: E402
from paper_1611_09638_gb300.inputs import WORKLOADS  # noqa: E402

NSAMPLE = 4096
SAMPLE_SEED = 77
MLOW = 6
KMAX_R = 1.0  # h/Mpc


def sample_nodes(n):
    """The seeded sample nodes (also drawn by the tests): NSAMPLE x 3 indices."""
    return np.random.default_rng(SAMPLE_SEED).integers(0, n, size=(NSAMPLE, 3))


def low_mode_mask(n):
    """Integer wave vectors with |m| <= MLOW in the full FFT layout."""
    m = np.fft.fftfreq(n, d=1.0 / n)
    mm = m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2
    return mm <= MLOW ** 2


def summarise(tag, res, W, dL, idx, mask, out):
    phi = res.phi
    out[f"{tag}_alpha"] = res.alpha
    out[f"{tag}_R"] = res.R
    out[f"{tag}_ncycles"] = res.ncycles
    out[f"{tag}_relres"] = res.relres
    out[f"{tag}_status"] = np.array(res.status)
    out[f"{tag}_steps"] = np.array(res.steps)
    out[f"{tag}_phi_samples"] = phi[idx[:, 0], idx[:, 1], idx[:, 2]]
    out[f"{tag}_phi_low"] = np.fft.fftn(phi)[mask]
    out[f"{tag}_phi_norm"] = np.array(np.linalg.norm(phi))
    k, r = cross_correlation(O.delta_r(phi), dL, W.box)
    sel = k <= KMAX_R
    out[f"{tag}_rk_k"] = k[sel]
    out[f"{tag}_rk"] = r[sel]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--k-max", type=int, default=200)
    ap.add_argument("--tag", default="")
    a = ap.parse_args()
    W = WORKLOADS[a.workload]
    n = W.n
    th = O.set_threads(a.threads if a.threads > 0 else (os.cpu_count() or 1))
    pos, dL = W.particles()
    rho = O.cic_deposit((n, n, n), pos / W.cell)
    del pos
    idx, mask = sample_nodes(n), low_mode_mask(n)
    out = {"workload": np.array(a.workload), "n": np.array(n), "box": np.array(W.box),
           "seed": np.array(W.seed), "order": np.array(W.order), "sample_seed": np.array(SAMPLE_SEED),
           "mlow": np.array(MLOW), "k_max": np.array(a.k_max), "threads": np.array(th)}
    t0 = time.time()
    # the stored runs start every step's linear solve from phidot = 0
    pA = O.OracleParams(n=(n, n, n), k_max=a.k_max, tol_in=1e-12, max_vcycles=200, warm_start=0)
    A = O.solve(pA, rho)
    out["A_seconds"] = np.array(time.time() - t0)
    print(f"A: status {A.status}, {A.steps} steps, {int(A.ncycles.sum())} V-cycles, "
          f"{time.time() - t0:.0f} s", flush=True)
    summarise("A", A, W, dL, idx, mask, out)
    g, lam = O.geometry(A.phi)
    out["A_m_samples"] = A.m[idx[:, 0], idx[:, 1], idx[:, 2]]
    out["A_det_samples"] = g[idx[:, 0], idx[:, 1], idx[:, 2]]
    out["A_lambda0_samples"] = lam[idx[:, 0], idx[:, 1], idx[:, 2]]
    del g, lam
    t0 = time.time()
    pB = O.OracleParams(n=(n, n, n), k_max=max(A.steps, 1), tol_in=1e-8, warm_start=0)
    B = O.solve(pB, rho, replay_alpha=A.alpha if A.steps else None)
    out["B_seconds"] = np.array(time.time() - t0)
    summarise("B", B, W, dL, idx, mask, out)
    out["B_vs_A_phi_rel"] = np.array(np.linalg.norm(B.phi - A.phi) / np.linalg.norm(A.phi))
    print(f"B: {B.steps} steps, {int(B.ncycles.sum())} V-cycles, {time.time() - t0:.0f} s; "
          f"|phi_B - phi_A| / |phi_A| = {float(out['B_vs_A_phi_rel']):.3e}", flush=True)
    tag = f"_{a.tag}" if a.tag else ""
    path = os.path.join(HERE, f"{a.workload}{tag}_oracle.npz")
    np.savez_compressed(path, **out)
    print("wrote", path)


if __name__ == "__main__":
    main()
