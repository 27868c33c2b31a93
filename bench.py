"""Benchmark of the reconstruction solve on GB300.

One step = one whole recon_solve (every step of the moving-mesh iteration,
Sec. II / App. A of Zhu et al. 2016) on the 512^3 / 800 Mpc/h 2LPT workload
(BBKS, Gamma 0.2, n_s 1, sigma_8 0.8, seed 1002), from phi = 0 on the
density already resident in HBM, in mixed precision, run to the iteration's
own end (rms(s) <= tol_out, or the step limiter admits no step; at most
--k-max steps); the plain FP64 form of the same solve is timed beside it.
Metric: Mcells/s per full reconstruction solve at fixed residual = ncells /
solve time / 1e6 (whole job: summed over ranks, which solve independent
copies of the workload).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload lpt512]
    python bench.py --workload lpt256       # the 256^3 / 400 Mpc/h workload
    python bench.py --workload mocks96      # 96 mocks of 32^3..128^3, batched solve
    python bench.py --impl reference ...   # the CPU FP64 oracle, bounded sample
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mcells/s per full reconstruction solve at fixed residual, mixed vs FP64 GPU"
FALLBACK_HBM_GBS = 6800.0

# Steps and V(2,2) cycles of one FP64 solve of each workload (the oracle's
# cycle and stopping residual), as the plain FP64 GPU form measured them on
# GB300 with the default parameters.  The CPU oracle baseline (cpu_baseline
# and the reference arm) is one model: (deposit + geometry/source + S + limiter
# + advance) x steps + V-cycle x cycles + one deposit, each pass timed on the
# full grid by the oracle, with these counts.
ORACLE_SOLVE_COUNTS = {
    "lpt512": (27, 305),
    "lpt256": (56, 705),
}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="lpt512")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--fp64-warmup", type=int, default=0,
                    help="untimed FP64 solves first (one FP64 solve at 512^3 takes ~30 s)")
    ap.add_argument("--cpu-threads", type=int, default=0,
                    help="oracle threads for the CPU baseline (0: every host core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-mocks", action="store_true",
                    help="skip the brief batched-mocks timing in the headline line")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the brief 256^3 timing in the 512^3 headline line")
    ap.add_argument("--inner-vcycles", type=int, default=None,
                    help="FP32 V-cycles per FP64 defect correction (library default if unset)")
    ap.add_argument("--group-max", type=int, default=None,
                    help="most FP32 V-cycles per FP64 defect correction under grouped checks")
    ap.add_argument("--k-max", type=int, default=None,
                    help="step cap per solve (default: 200, so that a solve of the 2LPT "
                         "workloads runs to its own end; 40 for the mocks)")
    ap.add_argument("--launch-list", action="store_true",
                    help="only one solve on the host-driven loop (every kernel its own launch), "
                         "for a profiler's launch list; prints its record")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="precision of the --launch-list solve")
    ap.add_argument("--coarse-faces", type=int, default=None,
                    help="mixed precision's coarse-level coefficients (library default if unset)")
    ap.add_argument("--warm-start", type=int, default=None,
                    help="1: each step's linear solve starts from the last step's solution; "
                         "0: from zero (library default if unset; both precisions)")
    ap.add_argument("--tma", type=int, default=None,
                    help="1: the streaming sweep stages planes by bulk tensor copies where it can; "
                         "0: per-thread copies only (library default if unset)")
    ap.add_argument("--stream-planes", type=int, default=None,
                    help="--launch-list: fix the planes per block of the streaming sweep and "
                         "residual restriction (no timing launches at create)")
    ap.add_argument("--tune-inner", type=int, default=2,
                    help="1: each mixed-precision handle picks its FP32 V-cycles per FP64 defect "
                         "correction by timing on its first (untimed) solve; 2: and its smoothing "
                         "schedule (nu1, nu2)")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            pk = json.load(fh)
        for key in ("hbm_gbs", "hbm_GBps", "hbm"):
            if key in pk:
                v = pk[key]
                if isinstance(v, dict):
                    v = v.get("value", v.get("burst"))
                return float(v), "measured"
    except Exception:
        pass
    return FALLBACK_HBM_GBS, "fallback"


def _kernel_source_hash(rec):
    """sha256 of what decides the captured kernel's code: its source file up to
    the line that ends the kernel's part (rec["source_end"]), followed by the
    helper headers it includes (rec["headers"]); host-side launch code after
    that line does not change the kernel."""
    csrc = os.path.join(ROOT, "paper_1611_09638_gb300", "csrc")
    with open(os.path.join(csrc, rec["source"])) as fh:
        text = fh.read()
    end = rec.get("source_end")
    if end:
        text = text[:text.index(end)]
    for h in rec.get("headers", []):
        with open(os.path.join(csrc, h)) as fh:
            text += fh.read()
    return hashlib.sha256(text.encode()).hexdigest()


def _traffic(kernel_tag, cells):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source: (bytes, note).
    The sweep moves each node's bytes once, so a capture on another grid is
    scaled by the cell count, and the note says so."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        if rec.get("kernel") == kernel_tag and rec.get("sha256") == _kernel_source_hash(rec):
            got, at = float(rec["bytes_per_sweep_full_size"]), int(rec["cells_captured"])
            if at == cells:
                return got, None
            return got * cells / at, f"scaled by cells from the capture on {at} cells"
    except Exception:
        pass
    return None, None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in (self.out or "").splitlines():
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) >= 7:
                try:
                    rows.append((float(parts[0]), float(parts[1]), parts[3:7]))
                except ValueError:
                    pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, f in enumerate(fl)
                          if f.lower() in ("active", "1", "yes")})
        return {"sm_mhz": float(np.median([r[0] for r in rows])),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def max_over_ranks(v, world, device):
    """Max of a per-rank timing over all ranks (the slowest rank sets the
    whole-job time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mcells(cells_per_rank, world, ms):
    """Whole-job throughput: every rank solves its own copy of the workload."""
    return world * cells_per_rank / (ms * 1e-3) / 1e6


def _workload(name):
    from paper_1611_09638_gb300.inputs import WORKLOADS

    return WORKLOADS[name]


def run_gb300(a):
    import torch

    from paper_1611_09638_gb300 import Recon, resolved_params

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    W = _workload(a.workload)
    n = W.n
    cells = n ** 3
    pos_host, _ = W.particles()
    pos_dev = torch.from_numpy(pos_host).cuda()
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    mg_kw = {} if a.inner_vcycles is None else {"inner_vcycles": a.inner_vcycles}
    if a.coarse_faces is not None:
        mg_kw["coarse_faces"] = a.coarse_faces
    if a.tune_inner and a.inner_vcycles is None:
        mg_kw["tune_inner"] = a.tune_inner
    if a.group_max is not None:
        mg_kw["group_max"] = a.group_max
    if a.tma is not None:
        mg_kw["tma"] = a.tma
    both_kw = {} if a.warm_start is None else {"warm_start": a.warm_start}
    mg_kw.update(both_kw)

    def run_e2e(R):
        """The same solve end to end through the public calls, on the timed
        handle: host pinned particles in, delta_r to host pinned memory out."""
        pin_pos = torch.from_numpy(pos_host).pin_memory()
        out = torch.empty((n, n, n), dtype=torch.float64).pin_memory()
        R.deposit_particles(pin_pos)
        R.solve(record=False)
        R.field("delta_r", out=out)
        barrier()
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        k2 = max(1, min(a.steps, 3))
        for _ in range(k2):
            R.deposit_particles(pin_pos)
            st_e2e = R.solve(record=False)
            R.field("delta_r", out=out)
        e1.record(stream)
        barrier()
        e2e_ms = max_over_ranks(e0.elapsed_time(e1) / k2, world, "cuda")
        wall_ms = (time.perf_counter() - t0) * 1e3 / k2
        return {"value": whole_job_mcells(cells, world, e2e_ms), "unit": "Mcells/s",
                "h2d_bytes_per_step": int(pos_host.nbytes), "d2h_bytes_per_step": int(out.numel() * 8),
                "ms_per_step": e2e_ms, "host_wall_ms_per_step": wall_ms,
                "steps_per_solve": st_e2e.steps, "vcycles_per_solve": st_e2e.vcycles,
                "path": "recon_deposit(host pinned particles) + recon_solve + "
                        "recon_field(delta_r -> host pinned), on the timed handle"}

    def timed(precision, steps, warmup, profile=False, inner=None, then=None):
        kw = dict(mg_kw) if precision == "mixed" else {}
        kw.update(both_kw)
        if inner:  # the schedule the timed solves' handle chose
            kw.pop("tune_inner", None)
            kw.update(inner_vcycles=inner.inner_vcycles, nu1=inner.nu1, nu2=inner.nu2)
        R = Recon((n, n, n), box=W.box, precision=precision, profile=int(profile), k_max=a.k_max, **kw)
        R.deposit_particles(pos_dev)
        for _ in range(warmup):
            R.solve(record=False)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stats = []
        with Clocks(local) as clk:
            e0.record(stream)
            for _ in range(steps):
                stats.append(R.solve(record=True))
            e1.record(stream)
            barrier()
        ms = e0.elapsed_time(e1) / steps
        extra = then(R) if then else None
        R.close()
        if then:
            return ms, stats, clk.summary(), extra
        return ms, stats, clk.summary()

    # the product path: each solve is one CUDA graph (device-side control)
    if a.no_e2e:
        ms_mixed, st_mixed, clocks = timed("mixed", a.steps, a.warmup)
        e2e = None
    else:
        ms_mixed, st_mixed, clocks, e2e = timed("mixed", a.steps, a.warmup, then=run_e2e)
    # one more solve on the host-driven loop with CUDA events around every
    # finest-level sweep, for the roofline of the dominant kernel
    _, st_prof, _ = timed("mixed", 1, 0, profile=True, inner=st_mixed[0])
    ms_fp64, st_fp64 = None, None
    if a.fp64_steps > 0:
        ms_fp64, st_fp64, _ = timed("fp64", a.fp64_steps, a.fp64_warmup)

    ms_mixed = max_over_ranks(ms_mixed, world, "cuda")
    value = whole_job_mcells(cells, world, ms_mixed)
    s0 = st_mixed[0]
    fp64 = None
    if ms_fp64 is not None:
        ms_fp64 = max_over_ranks(ms_fp64, world, "cuda")
        value_fp64 = whole_job_mcells(cells, world, ms_fp64)
        f0 = st_fp64[0]
        # the two forms take their own step lengths, so a solve can end at a
        # different step; per step the comparison holds either way
        per_step = (ms_fp64 / max(f0.steps, 1)) / (ms_mixed / max(s0.steps, 1))
        fp64 = {"value": value_fp64, "unit": "Mcells/s", "ms_per_step": ms_fp64,
                "timed_solves": a.fp64_steps, "warmup_solves": a.fp64_warmup,
                "status": _status_name(f0.status), "steps_per_solve": f0.steps,
                "vcycles_per_solve": f0.vcycles, "R_end": f0.R,
                "multigrid": _mg_settings(resolved_params((n, n, n), precision="fp64", **both_kw)),
                "same_steps_as_mixed": f0.steps == s0.steps,
                "mixed_over_fp64_per_solve": value / value_fp64,
                "mixed_over_fp64_per_step": per_step,
                "mixed_over_fp64": value / value_fp64 if f0.steps == s0.steps else per_step}

    # roofline of the dominant kernel: the finest-level FP32 red-black sweep
    sm_ms = sum(s.smooth_ms for s in st_prof)
    sweeps = sum(s.smooth_sweeps for s in st_prof)
    sweep_bytes = st_prof[0].smooth_bytes
    peak, peak_kind = _peak_hbm()
    traffic, traffic_note = _traffic("rbgs_f32", cells)
    achieved = sweep_bytes / (sm_ms * 1e-3 / sweeps) / 1e9 if sweeps else None
    roof = {"bound": "hbm", "kernel": "rbgs_f32 finest-level sweep (red + black)",
            "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None, "peak_source": peak_kind,
            "traffic": traffic, "algorithmic_bytes_per_sweep": sweep_bytes,
            "sweeps_timed": sweeps, "share_of_solve": sm_ms / st_prof[0].ms,
            "timed_in": "one extra solve with CUDA events around each finest-level sweep"}
    if traffic_note:
        roof["traffic_note"] = traffic_note

    adj = None if a.no_adjoint else adjoint_timing(a, stream, barrier)
    mocks = None if a.no_mocks else mocks_timing(a, stream, barrier)
    second = None
    if a.workload == "lpt512" and not a.no_secondary:
        second = secondary_timing(a, stream, barrier, mg_kw)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(a, W)

    line = {
        "metric": METRIC, "value": value, "unit": "Mcells/s", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_mixed, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": _config(a, W),
        "solve": {"precision": "mixed", "status": _status_name(s0.status),
                  "steps_per_solve": s0.steps, "vcycles_per_solve": s0.vcycles,
                  "inner_vcycles_used": s0.inner_vcycles, "nu_used": [s0.nu1, s0.nu2],
                  "coarse_levels": "per-face coefficients" if resolved_params(
                      (n, n, n), precision="mixed", **{k: v for k, v in mg_kw.items()
                                                        if k != "tune_inner"}).coarse_faces
                  else "nodal (full-weighted a)",
                  "R0": s0.R0, "R_end": s0.R, "min_lambda0": s0.min_lambda0,
                  "max_delta_r": s0.max_delta_r,
                  "multigrid": _mg_settings(resolved_params((n, n, n), precision="mixed", **mg_kw)),
                  "control": "device loop: one CUDA graph per solve (conditional nodes)"},
        "fp64_gpu": fp64,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "adjoint": adj,
        "batched_mocks": mocks,
        "secondary": second,
        "gpu_launches": int(sum(s.launches for s in st_mixed)),
        "clocks": clocks,
    }
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def adjoint_timing(a, stream, barrier, steps=3):
    """recon_adjoint on the 128^3 / 200 Mpc/h ZA configuration (seed 1004) in
    mixed precision with checkpoints: the forward solve and the sweep back
    (dL/d rho from a band-limited dL/d delta_r), each timed with CUDA events."""
    import torch

    from paper_1611_09638_gb300 import Recon
    from paper_1611_09638_gb300.inputs import WORKLOADS

    W = WORKLOADS["za128"]
    n = W.n
    pos, _ = W.particles()
    K = min(a.k_max, 40)
    R = Recon((n, n, n), box=W.box, precision="mixed", checkpoint=1, k_max=K)
    R.deposit_particles(torch.from_numpy(pos).cuda())
    st = R.solve()
    g = torch.from_numpy(np.random.default_rng(1004).standard_normal((n, n, n))).cuda()
    out = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
    R.adjoint(g, out)
    barrier()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fwd = bwd = 0.0
    for _ in range(steps):
        e[0].record(stream)
        R.solve(record=False)
        e[1].record(stream)
        R.adjoint(g, out)
        e[2].record(stream)
        barrier()
        fwd += e[0].elapsed_time(e[1])
        bwd += e[1].elapsed_time(e[2])
    R.close()
    fwd, bwd = fwd / steps, bwd / steps
    return {"workload": W.name, "precision": "mixed", "steps_per_solve": st.steps,
            "forward_ms": fwd, "adjoint_ms": bwd, "adjoint_over_forward": bwd / fwd,
            "adjoint_mcells_s": n ** 3 / (bwd * 1e-3) / 1e6,
            "k_max": K, "checkpoint_bytes": 5 * 8 * n ** 3 * K}


def secondary_timing(a, stream, barrier, mg_kw, steps=3):
    """The 256^3 / 400 Mpc/h 2LPT workload (seed 1001) in brief, beside the
    512^3 headline: mixed precision (the headline's settings) and FP64, each
    solved to its own end, one untimed solve then `steps` timed ones (one for
    FP64)."""
    import torch

    from paper_1611_09638_gb300 import Recon

    W = _workload("lpt256")
    n = W.n
    pos = torch.from_numpy(W.particles()[0]).cuda()
    out = {"workload": W.name}
    for prec, k in (("mixed", steps), ("fp64", 1)):
        kw = mg_kw if prec == "mixed" else {}
        with Recon((n, n, n), box=W.box, precision=prec, k_max=a.k_max, **kw) as R:
            R.deposit_particles(pos)
            R.solve(record=False)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(k):
                st = R.solve(record=False)
            e1.record(stream)
            barrier()
            ms = e0.elapsed_time(e1) / k
        out[prec] = {"value": n ** 3 / (ms * 1e-3) / 1e6, "unit": "Mcells/s", "ms_per_solve": ms,
                     "timed_solves": k, "steps_per_solve": st.steps, "vcycles_per_solve": st.vcycles,
                     "status": _status_name(st.status)}
        if prec == "mixed":
            out[prec]["inner_vcycles_used"] = st.inner_vcycles
    out["mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    return out


def mocks_timing(a, stream, barrier, steps=2, k_max=40):
    """The batched-mocks configuration (96 ZA mocks of 32^3 / 64^3 / 128^3,
    seeds 2000 + i, mixed precision, 40 steps each: the small mocks' solves do
    not end by themselves within 200 steps) in brief: one untimed batch, then
    `steps` batched solves (recon_solve_batch, every mock on its own stream)
    timed with CUDA events, and the same solves one after another."""
    import torch

    from paper_1611_09638_gb300 import Recon, solve_batch
    from paper_1611_09638_gb300.inputs import mock_batch

    mocks = mock_batch()
    cells = sum(W.n ** 3 for W in mocks)
    recons = []
    for W in mocks:
        R = Recon((W.n,) * 3, box=W.box, precision="mixed", stream=torch.cuda.Stream(),
                  k_max=k_max, tune_inner=1 if a.tune_inner else 0)
        torch.cuda.synchronize()
        R.deposit_particles(torch.from_numpy(W.particles()[0]).cuda())
        recons.append(R)
    solve_batch(recons, record=False)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        stats = solve_batch(recons, record=False)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1) / steps
    e0.record(stream)
    for R in recons:
        R.solve(record=False)
    e1.record(stream)
    barrier()
    ms_seq = e0.elapsed_time(e1)
    by_size = {}
    for W, st in zip(mocks, stats):
        d = by_size.setdefault(f"{W.n}^3", {"mocks": 0, "steps": 0, "vcycles": 0})
        d["mocks"] += 1
        d["steps"] += st.steps
        d["vcycles"] += st.vcycles
    for R in recons:
        R.close()
    return {"workload": "96 ZA mocks: 32 x 32^3/100, 32 x 64^3/200, 32 x 128^3/400 Mpc/h",
            "value": cells / (ms * 1e-3) / 1e6, "unit": "Mcells/s", "ms_per_batch": ms,
            "timed_batches": steps, "k_max": k_max,
            "sequential_value": cells / (ms_seq * 1e-3) / 1e6,
            "per_size": by_size, "control": "recon_solve_batch: 96 solve graphs on 96 streams"}


def run_batch(a):
    """The batched-mocks configuration: 32 Zel'dovich mocks each of 32^3 /
    100, 64^3 / 200 and 128^3 / 400 Mpc/h (seeds 2000 + i), every one on its
    own stream and solved in mixed precision by recon_solve_batch, which
    launches all 96 solve graphs before waiting.  One step = one batched solve
    of all mocks; value = all mocks' cells / step time.  The same handles
    solved one after another are timed beside it."""
    import torch

    from paper_1611_09638_gb300 import Recon, solve_batch
    from paper_1611_09638_gb300.inputs import mock_batch

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    mocks = mock_batch()
    cells = sum(W.n ** 3 for W in mocks)
    host_pos = [W.particles()[0] for W in mocks]
    recons = []
    for W, pos in zip(mocks, host_pos):
        R = Recon((W.n,) * 3, box=W.box, precision="mixed", stream=torch.cuda.Stream(),
                  k_max=a.k_max)
        torch.cuda.synchronize()
        R.deposit_particles(torch.from_numpy(pos).cuda())
        recons.append(R)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(a.warmup):
        solve_batch(recons, record=False)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(a.steps):
            stats.append(solve_batch(recons, record=True))
        e1.record(stream)
        barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / a.steps, world, "cuda")
    clocks = clk.summary()
    # the same solves one after another
    e0.record(stream)
    for R in recons:
        R.solve(record=False)
    e1.record(stream)
    barrier()
    ms_seq = e0.elapsed_time(e1)
    # end to end: host particles in, every mock's delta_r back to the host
    pins = [torch.from_numpy(p).pin_memory() for p in host_pos]
    outs = [torch.empty((W.n,) * 3, dtype=torch.float64).pin_memory() for W in mocks]
    barrier()
    e0.record(stream)
    for R, pp in zip(recons, pins):
        R.deposit_particles(pp)
    solve_batch(recons, record=False)
    for R, o in zip(recons, outs):
        R.field("delta_r", out=o)
    e1.record(stream)
    barrier()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    by_size = {}
    for W, st in zip(mocks, stats[0]):
        d = by_size.setdefault(f"{W.n}^3", {"mocks": 0, "steps": 0, "vcycles": 0, "status": []})
        d["mocks"] += 1
        d["steps"] += st.steps
        d["vcycles"] += st.vcycles
        d["status"].append(st.status)
    for d in by_size.values():
        d["status"] = {str(k): d["status"].count(k) for k in sorted(set(d["status"]))}
    value = whole_job_mcells(cells, world, ms)
    line = {
        "metric": METRIC, "value": value, "unit": "Mcells/s", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "96 ZA mocks: 32 x 32^3/100, 32 x 64^3/200, 32 x 128^3/400 Mpc/h",
                   "cells_per_batch": cells, "seeds": "2000 + i", "precision": "mixed",
                   "k_max": a.k_max, "per_size": by_size,
                   "control": "recon_solve_batch: 96 solve graphs on 96 streams",
                   "l2": "working set ~17 GB per batch, larger than L2",
                   "parallelism": f"replicas x{world}"},
        "sequential": {"value": whole_job_mcells(cells, world, ms_seq), "ms_per_step": ms_seq,
                       "what": "the same 96 solves one after another (recon_solve)"},
        "e2e": {"value": whole_job_mcells(cells, world, ms_e2e), "unit": "Mcells/s",
                "h2d_bytes_per_step": int(sum(p.nbytes for p in host_pos)),
                "d2h_bytes_per_step": int(sum(o.numel() * 8 for o in outs)), "ms_per_step": ms_e2e,
                "path": "recon_deposit(host pinned) x96 + recon_solve_batch + recon_field(delta_r) x96"},
        "gpu_launches": int(sum(st.launches for b in stats for st in b)),
        "clocks": clocks,
    }
    for R in recons:
        R.close()
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def _config(a, W):
    """The workload, the same in both arms."""
    n = W.n
    return {"workload": W.name, "grid": [n, n, n], "box_mpc_h": W.box,
            "displacement": "2LPT" if W.order == 2 else "ZA", "seed": W.seed,
            "k_max": a.k_max, "tol_in": 1e-8, "tol_out": 1e-3,
            "l2": f"inputs larger than L2 (working set ~{n ** 3 * 235 / 1e9:.1f} GB per solve)",
            "parallelism": f"replicas x{_dist()[1]}"}


def _mg_settings(p):
    """The multigrid settings a solve resolved to."""
    return {"nu1": p.nu1, "nu2": p.nu2, "inner_vcycles": p.inner_vcycles if p.precision else None,
            "max_vcycles": p.max_vcycles, "warm_start": p.warm_start,
            "tma": p.tma if p.precision else None}


def _status_name(code):
    return {0: "converged (rms(s) <= tol_out)", 1: "k_max reached",
            2: "stalled (step limiter admits no step)"}.get(int(code), str(code))


def _host_cpu():
    """nproc and the host CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() == "Model name":
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as fh:
                for ln in fh:
                    if ln.lower().startswith(("model name", "cpu part")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "model": model}


class OracleModel:
    """The CPU oracle's solve time on a workload, from a bounded sample: each
    pass of one step (deposit, geometry + source, S, limiter, advance) timed
    once on the full grid, and V-cycles timed on the full grid; a solve is
    steps x passes + cycles x V-cycle + one deposit, with the FP64 solve's
    counts (ORACLE_SOLVE_COUNTS)."""

    def __init__(self, W, threads):
        import oracle as O

        self.O, self.W = O, W
        n = W.n
        self.threads = O.set_threads(threads if threads > 0 else (os.cpu_count() or 1))
        pos, _ = W.particles()
        self.x = pos / W.cell
        rho = O.cic_deposit((n, n, n), self.x)
        self.m = rho / rho.mean()
        self.p = O.OracleParams(n=(n, n, n))
        self.s, _ = O.source(self.p, np.zeros((n, n, n)), self.m)
        self.a = np.maximum(self.m, self.p.a_min)
        self.steps, self.cycles = ORACLE_SOLVE_COUNTS[W_key(W)]

    def passes(self):
        O, n = self.O, self.W.n
        t = {}
        t0 = time.perf_counter()
        O.cic_deposit((n, n, n), self.x, self.m.ravel())
        t["deposit"] = time.perf_counter() - t0
        phi = np.zeros((n, n, n))
        t0 = time.perf_counter()
        O.source(self.p, phi, self.m)
        t["source"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        d = O.apply_S(self.s)
        t["smooth"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        O.step_limiter(self.p, phi, d * 1e-3)
        t["limiter"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        O.advance(1.0, d * 1e-3, phi, self.x)
        t["advance"] = time.perf_counter() - t0
        self.t_passes = t
        return t

    def vcycle(self):
        t0 = time.perf_counter()
        self.O.vcycle(self.p, self.a, self.s, np.zeros_like(self.s))
        return time.perf_counter() - t0

    def solve_seconds(self, t_vcycle):
        t = self.t_passes
        per_step = t["deposit"] + t["source"] + t["smooth"] + t["limiter"] + t["advance"]
        return self.steps * per_step + self.cycles * t_vcycle + t["deposit"]

    def sample(self, nv):
        return (f"{self.W.n}^3 grid: each pass of one step once and {nv} V(2,2) cycle(s) on the "
                f"full grid, scaled to the FP64 solve's {self.steps} steps and {self.cycles} "
                f"V-cycles, {self.threads} oracle thread(s)")


def W_key(W):
    from paper_1611_09638_gb300.inputs import WORKLOADS

    return next(k for k, v in WORKLOADS.items() if v == W)


def cpu_baseline(a, W):
    """The CPU oracle as it stands on a bounded sample of the same workload
    (OracleModel), on every host core unless --cpu-threads says otherwise."""
    M = OracleModel(W, a.cpu_threads)
    t0 = time.perf_counter()
    M.passes()
    tv = M.vcycle()
    solve_s = M.solve_seconds(tv)
    return {"value": W.n ** 3 / solve_s / 1e6, "unit": "Mcells/s", "cores": M.threads,
            "kind": "oracle", "sample": M.sample(1), "host": _host_cpu(),
            "sample_seconds": time.perf_counter() - t0, "vcycle_s": tv,
            "passes_s": M.t_passes, "est_solve_seconds": solve_s}


def run_reference(a):
    """The reference arm: the CPU FP64 oracle (OracleModel, every host core);
    each timed step is one oracle V-cycle on the full grid, the per-step passes
    are timed once before the warm-up."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    W = _workload(a.workload)
    n = W.n
    M = OracleModel(W, a.cpu_threads)
    M.passes()
    for _ in range(a.warmup):
        M.vcycle()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        M.vcycle()
    tv = (time.perf_counter() - t0) / a.steps
    solve_s = M.solve_seconds(tv)
    value = n ** 3 / solve_s / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mcells/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": tv * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(a, W),
            "solve": {"precision": "fp64, CPU oracle (V(2,2) cycles)"},
            "cpu_baseline": {"value": value, "unit": "Mcells/s", "cores": M.threads,
                             "kind": "oracle", "sample": M.sample(a.steps), "host": _host_cpu(),
                             "passes_s": M.t_passes, "est_solve_seconds": solve_s},
            "e2e": {"value": value, "unit": "Mcells/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_launch_list(a):
    """One solve of the workload on the host-driven loop, nothing else."""
    import torch

    from paper_1611_09638_gb300 import Recon

    W = _workload(a.workload)
    n = W.n
    pos, _ = W.particles()
    kw = {}
    if a.precision == "mixed" and a.inner_vcycles is not None:
        kw["inner_vcycles"] = a.inner_vcycles
    if a.precision == "mixed" and a.coarse_faces is not None:
        kw["coarse_faces"] = a.coarse_faces
    if a.precision == "mixed" and a.tma is not None:
        kw["tma"] = a.tma
    if a.warm_start is not None:
        kw["warm_start"] = a.warm_start
    if a.precision == "mixed" and a.stream_planes is not None:
        kw["stream_planes"] = a.stream_planes
        kw["restrict_planes"] = min(a.stream_planes, 8)
    with Recon((n, n, n), box=W.box, precision=a.precision, k_max=a.k_max, device_loop=0, **kw) as R:
        R.deposit_particles(torch.from_numpy(pos).cuda())
        st = R.solve()
    print(json.dumps({"workload": W.name, "precision": a.precision, "k_max": a.k_max,
                      "steps": st.steps, "vcycles": st.vcycles, "launches": st.launches,
                      "ms": st.ms, "status": _status_name(st.status)}))


if __name__ == "__main__":
    args = _args()
    if args.k_max is None:
        args.k_max = 40 if args.workload == "mocks96" else 200
    if args.launch_list:
        run_launch_list(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "mocks96":
        run_batch(args)
    else:
        run_gb300(args)
