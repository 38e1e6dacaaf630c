"""Benchmark of the Léja-point log-determinant hot path on GB300.

Workload (default): Q = L_3D + 0.05 I, 7-point Dirichlet Laplacian on a 128^3 grid
(n = 2,097,152, nnz = 14,581,760, int32 CSR), bounds [0.05, 12.05], Léja degree 60, Hutch++ with
99 Rademacher probes (33/33/33) from seed 1. One step = one full estimate (Algorithm 3): probes,
pass 1 (m fused SpMM steps, width 33), CholeskyQR2 + deflation, pass 2 (m fused SpMM+trace steps,
width 66), host combine.

Metric: Léja SpMM-recurrence GB/s = algorithmic bytes of the 2m Léja steps per estimate x steps
/ device time (the QR and probe time is inside the timed region but adds no bytes). Inputs are
resident in HBM and larger than L2 (the 553 MB-1.1 GB probe blocks, 175 MB matrix).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       [--precision df64|f64|f32] [--degree M]
Under torchrun (N > 1) every rank runs an independent replica with seed + rank (weak scaling,
no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Léja SpMM-recurrence GB/s (% HBM peak)"
UNIT = "GB/s"
GRID_N = 128
SHIFT = 0.05
BOUNDS = (0.05, 12.05)
PROBES = 99
SEED = 1

DTYPE_NAME = {"df64": "df64 = 48-bit float-float (FP32 pairs on the FP32 pipes, 8-byte storage; not IEEE f64)",
              "f64": "f64 (IEEE binary64 on the FP64 pipe)",
              "f32": "f32-mixed (FP32 values and W_j; P and the traces in double-float)"}
ELEM = {"df64": (8, 8, 8, 8), "f64": (8, 8, 8, 8), "f32": (4, 4, 8, 4)}   # s_A, s_W, s_P, s_V

# DRAM bytes (read + write) of one pass-2 trace-step launch per matrix row, from one ncu capture of
# each kernel on the 96^3 Laplacian (n = 884,736): DF64 register gathers 1.4777 GB, DF64 TMA
# 1.4945 GB, FP32-mixed TMA with two column pairs per thread 0.7570 GB. Traffic grows in proportion
# to the rows of a stencil matrix, so the full-size value is this figure times n. Only valid for the
# trace steps of the kernels as captured (profiles/k_leja_tma_*_96cubed.md).
TRACE_STEP_DRAM_BYTES_PER_ROW = {("gather", "df64"): 1.477654528e9 / 884736,
                                 ("tma", "df64"): (1.052240128e9 + 0.442266112e9) / 884736,
                                 ("tma", "f32"): (0.542213632e9 + 0.214823424e9) / 884736}


def step_bytes(n: int, nnz: int, b: int, prec: str, mode: str) -> int:
    """Algorithmic (compulsory) bytes of one fused Léja step over an n x b block:
    CSR values + column indices + row pointers, W_j read, W_{j+1} written, and
    P read+written (pass 1) or V read (pass 2)."""
    s_a, s_w, s_p, s_v = ELEM[prec]
    base = nnz * (s_a + 4) + 4 * (n + 1) + n * b * 2 * s_w
    return base + (n * b * 2 * s_p if mode == "accum" else n * b * s_v)


def estimate_bytes(n: int, nnz: int, k: int, m: int, prec: str) -> int:
    return m * (step_bytes(n, nnz, k, prec, "accum") + step_bytes(n, nnz, 2 * k, prec, "dot"))


def load_peaks() -> tuple[dict, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples taken during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, world: int, device: str) -> float:
    """The largest x over the ranks (the slowest replica's time); x itself on one rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


CPU_SAMPLE_M = 8   # Léja steps per sampled probe column


def _oracle_columns(A, budget_s: float, start_at: float = 0.0, col0: int = 0) -> tuple[int, float]:
    """The FP64 oracle as it stands (Algorithm 2 one column at a time, SciPy CSR mat-vec) on
    Rademacher probe columns of seeds SEED + col0, SEED + col0 + 1, ... until budget_s have passed:
    (columns done, seconds). Waits until start_at (time.time()) first when given."""
    from oracle import logdet as O
    from oracle import rng as R
    sigma = O.sigma_of(BOUNDS[0])
    lt, ut = BOUNDS[0] / sigma, BOUNDS[1] / sigma
    xi, c, g, d, _ = O.newton_leja_setup(lt, ut, CPU_SAMPLE_M)
    M = O._scipy(A)
    if start_at > 0.0:
        while time.time() < start_at:
            time.sleep(0.01)
    cols = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        v = R.rademacher(SEED + col0 + cols, 0, A.n, 1)
        O.leja_apply_columns(M, v, xi, d, c, g, sigma)
        cols += 1
    return cols, time.perf_counter() - t0


def _cpu_worker(args):
    """One process of the all-core oracle sample (started by spawn: no CUDA state inherited)."""
    grid, rank, budget_s, start_at = args
    os.environ["OMP_NUM_THREADS"] = "1"
    from synth import laplacian_3d
    A = laplacian_3d(grid, SHIFT)
    return _oracle_columns(A, budget_s, start_at, col0=rank * 1000)


def _host_cpu() -> dict:
    info = {"nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() in ("Architecture", "Model name", "Socket(s)", "Core(s) per socket", "Thread(s) per core"):
                info[k.strip()] = v.strip()
    except Exception:
        pass
    return info


def cpu_baseline(A, prec: str, budget_s: float = 12.0, all_cores: bool = True) -> dict:
    """The FP64 CPU oracle as it stands (one column at a time, SciPy CSR mat-vec), timed on a
    bounded sample of the headline workload: Algorithm 2 steps on single probe columns for about
    budget_s, on one core; then the same on every host core at once (one spawned process per
    core, each on its own columns: the oracle is single-threaded, so columns are its unit of
    parallel work), reported beside it."""
    # per column-step bytes in the oracle's own FP64 layout: CSR + w read + w written + P read/written
    per = A.nnz * 12 + 4 * (A.n + 1) + A.n * (2 * 8 + 2 * 8)
    cols, dt = _oracle_columns(A, budget_s)
    gbs = cols * CPU_SAMPLE_M * per / dt / 1e9
    host = _host_cpu()
    out = {"value": gbs, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host,
           "sample": f"{cols} probe column(s) x {CPU_SAMPLE_M} Léja steps (Algorithm 2, FP64, SciPy CSR mat-vec) "
                     f"on the {int(round(A.n ** (1 / 3)))}^3 Laplacian in {dt:.1f} s, one process"}
    ncpu = os.cpu_count() or 1
    if all_cores and ncpu > 1:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        start_at = time.time() + 10.0          # after every worker has built the matrix
        with ctx.Pool(ncpu) as pool:
            res = pool.map(_cpu_worker, [(int(round(A.n ** (1 / 3))), r, budget_s / 2, start_at) for r in range(ncpu)])
        tot = sum(c for c, _ in res)
        wall = max(t for _, t in res)
        out["all_cores"] = {"value": tot * CPU_SAMPLE_M * per / wall / 1e9, "unit": UNIT, "cores": ncpu,
                            "sample": f"{tot} probe columns x {CPU_SAMPLE_M} Léja steps over {ncpu} processes "
                                      f"in {wall:.1f} s"}
    return out


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    from synth import laplacian_3d
    A = laplacian_3d(GRID_N, SHIFT)
    for _ in range(args.warmup):
        cpu_baseline(A, args.precision, budget_s=2.0, all_cores=False)
    vals = []
    cb = None
    for _ in range(args.steps):
        cb = cpu_baseline(A, args.precision, budget_s=6.0, all_cores=False)
        vals.append(cb["value"])
    v = statistics.median(vals)
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"L3D+{SHIFT}I {GRID_N}^3 (n={A.n}, nnz={A.nnz}), degree {args.degree}, "
                                   f"{PROBES} Rademacher probes, seed {SEED}", "model": None},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def time_calls(fn, reps: int, warmup: int = 1):
    """Device time of `reps` calls of fn() (CUDA events on the current stream), in ms per call.
    Forward calls need two warm-ups to reach the graph replay: the first tunes the step kernels
    and may grow the workspace (which voids that call's capture), the second captures."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = None
    for _ in range(reps):
        out = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def workload_config1(L, h):
    """2-D Laplacian + 0.1 I on 100 x 100, bounds [0.1, 8.1], 40 Léja points, 30 Rademacher
    probes from seed 0: a latency-bound estimate (n = 10,000)."""
    from synth import laplacian_2d
    from tests.pins import logdet_laplacian_2d
    A = laplacian_2d(100, 0.1)
    dA = L.DeviceCSR.from_host(A)
    out = {}
    for prec in ("df64", "f32"):
        opts = L.options(degree=39, probes=30, seed=0, precision=prec)
        ms, est = time_calls(lambda: L.ll_logdet_forward(h, dA, 0.1, 8.1, opts), 20, 3)
        exact = logdet_laplacian_2d(100, 0.1)
        out[prec] = {"ms_per_estimate": ms, "estimate": est, "rel_err_vs_exact": abs(est - exact) / exact,
                     "launches": h.info()["kernel_launches"]}
    return {"workload": "L2D+0.1I 100^2 (n=10000, nnz=49600), degree 39, 30 Rademacher probes, seed 0", **out}


def workload_config3(L, h, grid: int = 1024, degree: int = 80):
    """Matérn GMRF tau (kappa^2 I + L_2D)^2 on grid x grid (13-point stencil), kappa = 0.3,
    tau = 1, degree 80, 60 Gaussian probes: forward estimate, adjoint (value gradients) and the
    chain to (kappa, tau), against the closed forms."""
    import numpy as np
    import torch
    from synth import matern_2d, matern_2d_derivatives
    from tests.pins import dlogdet_matern_2d, logdet_matern_2d
    kappa, tau = 0.3, 1.0
    A = matern_2d(grid, kappa, tau)
    dk, dt = matern_2d_derivatives(grid, kappa, tau)
    dA = L.DeviceCSR.from_host(A)
    lmax = L.ll_gershgorin(h, dA)[1]
    lmin = tau * kappa ** 4
    dv = torch.as_tensor(np.stack([dk, dt])).cuda()
    exact = logdet_matern_2d(grid, kappa, tau)
    ex_k, ex_t = dlogdet_matern_2d(grid, kappa, tau)
    out = {}
    for prec in ("df64", "f32"):
        opts = L.options(degree=degree, probes=60, seed=0, precision=prec, probe_kind="gaussian", keep_for_backward=True)
        ms_f, est = time_calls(lambda: L.ll_logdet_forward(h, dA, lmin, lmax, opts), 2, 2)
        inf = h.info()
        ms_b, g = time_calls(lambda: L.ll_logdet_backward(h, dA, 1.0), 2, 1)
        kept_w = (inf["kept_w_steps"], inf["kept_w_steps_pass1"])
        th = L.ll_param_grad(h, g, dv)
        del g
        # the exact derivative of the estimate (through the sketch's QR)
        ms_bq, gq = time_calls(lambda: L.ll_logdet_backward(h, dA, 1.0, through_qr=True), 1, 1)
        thq = L.ll_param_grad(h, gq, dv)
        del gq
        # the same backward with W_j recomputed from ceil(sqrt(m)) checkpoints instead of kept
        ck = L.options(degree=degree, probes=60, seed=0, precision=prec, probe_kind="gaussian", keep_for_backward=True,
                       ckpt_stride=int(np.ceil(np.sqrt(degree))))
        L.ll_logdet_forward(h, dA, lmin, lmax, ck)
        ms_bc, gc = time_calls(lambda: L.ll_logdet_backward(h, dA, 1.0), 2, 1)
        del gc
        out[prec] = {"ms_forward": ms_f, "ms_backward": ms_b, "ms_forward_plus_gradient": ms_f + ms_b,
                     "ms_backward_through_qr": ms_bq, "backward_kept_w_steps": kept_w,
                     "ms_backward_checkpointed": ms_bc,
                     "estimate": est, "rel_err_vs_exact": abs(est - exact) / abs(exact),
                     "dlogdet_dkappa": th[0], "dlogdet_dtau": th[1],
                     "rel_err_dkappa": abs(th[0] - ex_k) / abs(ex_k), "rel_err_dtau": abs(th[1] - ex_t) / abs(ex_t),
                     "through_qr_rel_err_dkappa": abs(thq[0] - ex_k) / abs(ex_k),
                     "through_qr_rel_err_dtau": abs(thq[1] - ex_t) / abs(ex_t),
                     "forward_phase_ms": {"pass1": inf["ms_pass1"], "qr": inf["ms_qr"], "pass2": inf["ms_pass2"]}}
    return {"workload": f"Matern tau(kappa^2 I + L2D)^2 {grid}^2 (n={A.n}, nnz={A.nnz}), kappa={kappa}, tau={tau}, "
                        f"bounds [{lmin}, {lmax:.4f}], degree {degree}, 60 Gaussian probes, seed 0", **out}


def workload_c3_time_to_tol(L, h, grid: int = 1024, tol: float = 1e-3, degrees=(80, 120, 160),
                            probe_counts=(60, 120, 240)):
    """Time of the log-determinant plus its gradient at `tol` relative error on the Matérn GMRF
    of config 3 (tau (kappa^2 I + L_2D)^2 on grid^2, kappa = 0.3, tau = 1, Gaussian probes, seed 0).
    A degree x probes sweep in FP32-mixed finds the cheapest setting (forward + frozen-basis
    backward time) whose log-determinant and both theta-gradients (d/dkappa, d/dtau through
    ll_param_grad) are within tol of the closed forms; that setting is then timed in IEEE FP64
    (the plain FP64 form), DF64 and FP32-mixed on the same GPU."""
    import numpy as np
    import torch
    from synth import matern_2d, matern_2d_derivatives
    from tests.pins import dlogdet_matern_2d, logdet_matern_2d
    kappa, tau = 0.3, 1.0
    A = matern_2d(grid, kappa, tau)
    dk, dt = matern_2d_derivatives(grid, kappa, tau)
    dv = torch.as_tensor(np.stack([dk, dt])).cuda()
    exact = logdet_matern_2d(grid, kappa, tau)
    ex_k, ex_t = dlogdet_matern_2d(grid, kappa, tau)
    dev = {"f64": L.DeviceCSR.from_host(A, "f64"), "f32": L.DeviceCSR.from_host(A, "f32")}
    dev["df64"] = dev["f64"]
    lmax = L.ll_gershgorin(h, dev["f64"])[1]
    lmin = tau * kappa ** 4

    def run(prec: str, degree: int, probes: int, warm: int = 2):
        dA = dev[prec]
        opts = L.options(degree=degree, probes=probes, seed=0, precision=prec, probe_kind="gaussian",
                         keep_for_backward=True)
        ms_f, est = time_calls(lambda: L.ll_logdet_forward(h, dA, lmin, lmax, opts), 1, warm)
        ms_b, g = time_calls(lambda: L.ll_logdet_backward(h, dA, 1.0), 1, 1)
        th = L.ll_param_grad(h, g, dv)
        del g
        errs = {"logdet": abs(est - exact) / abs(exact), "dkappa": abs(th[0] - ex_k) / abs(ex_k),
                "dtau": abs(th[1] - ex_t) / abs(ex_t)}
        return {"degree": degree, "probes": probes, "ms_forward": ms_f, "ms_backward": ms_b,
                "ms_logdet_plus_gradient": ms_f + ms_b, "rel_err": errs, "max_rel_err": max(errs.values()),
                "kept_w_stride": h.info()["kept_w_stride"]}

    sweep = [run("f32", d, p) for d in degrees for p in probe_counts]
    ok = [x for x in sweep if x["max_rel_err"] <= tol]
    pick = min(ok, key=lambda x: x["ms_logdet_plus_gradient"]) if ok else min(sweep, key=lambda x: x["max_rel_err"])
    timed = {pr: run(pr, pick["degree"], pick["probes"]) for pr in ("f64", "df64", "f32")}
    return {"workload": (f"Matern tau(kappa^2 I + L2D)^2 {grid}^2 (n={A.n}, nnz={A.nnz}), kappa={kappa}, tau={tau}, "
                         f"Gaussian probes, seed 0; logdet + frozen-basis gradient chained to (kappa, tau)"),
            "tol": tol, "reached": bool(ok), "setting": {"degree": pick["degree"], "probes": pick["probes"]},
            "sweep_f32": sweep, "timed": timed,
            "speedup_f32_vs_f64": timed["f64"]["ms_logdet_plus_gradient"] / timed["f32"]["ms_logdet_plus_gradient"],
            "speedup_df64_vs_f64": timed["f64"]["ms_logdet_plus_gradient"] / timed["df64"]["ms_logdet_plus_gradient"]}


def workload_config4(L, h, count: int = 64):
    """64 GMRFs L_2D + tau_i I, sides log-uniform in [64, 512], tau_i ~ U[0.01, 1] (seed 2), degree
    from the bound ratio, 30 probes each: one persistent launch per pass vs one call per matrix."""
    from synth import gmrf_batch_params, laplacian_2d
    from tests.pins import logdet_laplacian_2d
    params = gmrf_batch_params(count=count, seed=2)
    mats = [laplacian_2d(side, t) for side, t in params]
    bounds = [(t, 8.0 + t) for _, t in params]
    out = {"n_total": sum(A.n for A in mats), "nnz_total": sum(A.nnz for A in mats)}
    import math as _m
    degs = []
    for lo, hi in bounds:
        sg = lo if lo < 1 else 1.0
        kap = (hi / sg) / (lo / sg)
        rho = (_m.sqrt(kap) + 1) / (_m.sqrt(kap) - 1)
        degs.append(max(10, min(250, _m.ceil(_m.log(1e6) / _m.log(rho)))))
    for prec in ("df64", "f32"):
        dm = [L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64") for A in mats]
        opts = L.options(probes=30, seed=2, precision=prec)
        ms_b, est = time_calls(lambda: L.ll_logdet_batched(h, dm, bounds, opts), 2, 2)
        inf = h.info()
        # algorithmic bytes of every Léja step of every matrix (pass 1 on k = 10 columns, pass 2 on 20)
        b1 = sum(m * step_bytes(A.n, A.nnz, 10, prec, "accum") for A, m in zip(mats, degs))
        b2 = sum(m * step_bytes(A.n, A.nnz, 20, prec, "dot") for A, m in zip(mats, degs))
        hr = L.Handle()
        opts_r = L.options(probes=30, seed=2, precision=prec, step_kernel="gather")
        ms_r, _ = time_calls(lambda: L.ll_logdet_batched(hr, dm, bounds, opts_r), 2, 2)
        inf_r = hr.info()

        def one_by_one():
            res = []
            for i, A in enumerate(dm):
                lo, hi = bounds[i]
                sg = lo if lo < 1 else 1.0
                kap = (hi / sg) / (lo / sg)
                rho = (_m.sqrt(kap) + 1) / (_m.sqrt(kap) - 1)
                m = max(10, min(250, _m.ceil(_m.log(1e6) / _m.log(rho))))
                res.append(L.ll_logdet_forward(h, A, lo, hi, L.options(degree=m, probes=30, seed=2 + i, precision=prec)))
            return res
        ms_s, est_s = time_calls(one_by_one, 1, 1)
        exact = [logdet_laplacian_2d(side, t) for side, t in params]
        errs = [abs(e - x) / abs(x) for e, x in zip(est, exact)]
        out[prec] = {"ms_batched": ms_b, "ms_one_call_per_matrix": ms_s, "speedup": ms_s / ms_b,
                     "step_kernel": {v: k for k, v in L.STEP_KERNELS.items()}.get(inf["kernel_pass1"], "?"),
                     "autotuned_shape": {"tuned": inf["batch_tuned"], "threads": [inf["threads_pass1"], inf["threads_pass2"]],
                                         "rows_per_tile": [inf["rows_pass1"], inf["rows_pass2"]]},
                     "pass_gbs": {"pass1": b1 / (inf["ms_pass1"] * 1e-3) / 1e9, "pass2": b2 / (inf["ms_pass2"] * 1e-3) / 1e9},
                     "ms_batched_register_kernel": ms_r,
                     "register_kernel_phase_ms": {"pass1": inf_r["ms_pass1"], "qr": inf_r["ms_qr"], "pass2": inf_r["ms_pass2"]},
                     "max_rel_diff_batched_vs_single": max(abs(a - b) / abs(b) for a, b in zip(est, est_s)),
                     "max_rel_err_vs_exact": max(errs), "median_rel_err_vs_exact": sorted(errs)[len(errs) // 2],
                     "phase_ms": {"pass1": inf["ms_pass1"], "qr": inf["ms_qr"], "pass2": inf["ms_pass2"]}}
    return {"workload": f"{count} x (L2D + tau_i I), sides log-uniform [64,512], tau U[0.01,1], seed 2, 30 probes", **out}


def workload_config5(L, h, log2n: int = 22, degree: int = 150, probes: int = 120, reorder: str = "auto"):
    """Weighted graph Laplacian + 1e-2 I of a power-law (Chung-Lu) graph, n = 2^22, mean degree 16,
    exponent 2.3, weights U[0.5, 1.5], seed 3. Bounds from Gershgorin plus 20 power iterations
    (lmax = min(Gershgorin, 1.05 x Rayleigh quotient), lmin = 0.01); degree 150, Hutch++ 120
    probes. FP32-mixed throughput and its difference from the plain FP64 form on the same GPU (no
    closed form exists at this size)."""
    import time as _t
    from synth import powerlaw_laplacian
    t0 = _t.perf_counter()
    A = powerlaw_laplacian(1 << log2n, seed=3, device="cuda")
    t_gen = _t.perf_counter() - t0
    d64 = L.DeviceCSR.from_host(A, "f64")
    d32 = L.DeviceCSR.from_host(A, "f32")
    glo, ghi = L.ll_gershgorin(h, d64)
    lp = L.ll_power_lmax(h, d64, iters=20, seed=3)
    lmin, lmax = 0.01, min(ghi, 1.05 * lp)
    n, nnz, k = A.n, A.nnz, probes // 3
    out = {"n": n, "nnz": nnz, "max_row_nnz": int((A.rowptr[1:] - A.rowptr[:-1]).max()), "generate_s": t_gen,
           "gershgorin": [glo, ghi], "lambda_power": lp, "bounds": [lmin, lmax]}
    for prec, dA, reps in (("f32", d32, 2), ("f64", d64, 1)):
        opts = L.options(degree=degree, probes=probes, seed=3, precision=prec, reorder=reorder)
        ms, est = time_calls(lambda: L.ll_logdet_forward(h, dA, lmin, lmax, opts), reps, 1)
        inf = h.info()
        b2 = step_bytes(n, nnz, 2 * k, prec, "dot")
        b1 = step_bytes(n, nnz, k, prec, "accum")
        out[prec] = {"ms_per_estimate": ms, "estimate": est, "GBps_estimate": estimate_bytes(n, nnz, k, degree, prec) / (ms / 1e3) / 1e9,
                     "pass1_launch_GBps": b1 / (inf["ms_pass1"] / degree / 1e3) / 1e9,
                     "pass2_launch_GBps": b2 / (inf["ms_pass2"] / degree / 1e3) / 1e9,
                     "kernels": [inf["kernel_pass1"], inf["kernel_pass2"]], "reordered": inf["reordered"],
                     "phase_ms": {"pass1": inf["ms_pass1"], "qr": inf["ms_qr"], "pass2": inf["ms_pass2"]}}
    out["rel_diff_f32_vs_f64"] = abs(out["f32"]["estimate"] - out["f64"]["estimate"]) / abs(out["f64"]["estimate"])
    if log2n == 22:
        # DRAM bytes of one FP32 trace-step launch (k_leja_tma<f32,DOT>, width 80) from ncu at this
        # size (profiles/k_leja_tma_f32_powerlaw_config5.md), beside the algorithmic bytes
        out["trace_step_dram_bytes"] = {"algorithmic": step_bytes(n, nnz, 2 * k, "f32", "dot"),
                                        "ncu_degree_order": 23.8397e9 + 1.3285e9,
                                        "ncu_matrix_order": 27.0815e9 + 1.3390e9}
    out["workload"] = (f"power-law Laplacian + 1e-2 I, n=2^{log2n} ({n}), nnz={nnz}, mean degree 16, exponent 2.3, "
                       f"seed 3, degree {degree}, {probes} probes")
    return out


def workload_f3(L, h, n: int = 10_000_000, probes: int = 30):
    """Section 5.1's synthetic pentadiagonal SPD family at the paper's largest size: five
    diagonals U[0,1] (seed 0), Q + Q^T + n I, n = 10^7. Gershgorin bounds (lambda_min >= 1, so
    sigma = 1), degree from the bounds, Hutch++ with 30 Rademacher probes (seed 0). Throughput,
    and the error against the banded-Cholesky log-determinant (the error is Hutch++'s residual
    variance on a spectrum close to n I; the interpolant is exact to rounding)."""
    import math as _m
    import time as _t
    from synth import pentadiagonal
    from tests.pins import logdet_banded
    t0 = _t.perf_counter()
    A = pentadiagonal(n, seed=0)
    t_gen = _t.perf_counter() - t0
    exact = logdet_banded(A)
    nnz, k = A.nnz, probes // 3
    out = {"n": n, "nnz": nnz, "generate_s": t_gen, "exact_logdet": exact}
    for prec in ("df64", "f32"):
        dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
        lo, hi = L.ll_gershgorin(h, dA)
        sg = lo if lo < 1 else 1.0
        kap = (hi / sg) / (lo / sg)
        rho = (_m.sqrt(kap) + 1) / (_m.sqrt(kap) - 1)
        m = max(10, min(250, _m.ceil(_m.log(1e6) / _m.log(rho))))
        opts = L.options(degree=m, probes=probes, seed=0, precision=prec)
        ms, est = time_calls(lambda: L.ll_logdet_forward(h, dA, lo, hi, opts), 3, 2)
        inf = h.info()
        out[prec] = {"ms_per_estimate": ms, "degree": m, "bounds": [lo, hi], "estimate": est,
                     "rel_err_vs_exact": abs(est - exact) / abs(exact),
                     "GBps_estimate": estimate_bytes(n, nnz, k, m, prec) / (ms / 1e3) / 1e9,
                     "pass1_launch_GBps": step_bytes(n, nnz, k, prec, "accum") / (inf["ms_pass1"] / m / 1e3) / 1e9,
                     "pass2_launch_GBps": step_bytes(n, nnz, 2 * k, prec, "dot") / (inf["ms_pass2"] / m / 1e3) / 1e9,
                     "kernels": [inf["kernel_pass1"], inf["kernel_pass2"]],
                     "phase_ms": {"probes": inf["ms_probes"], "pass1": inf["ms_pass1"], "qr": inf["ms_qr"], "pass2": inf["ms_pass2"]}}
        del dA
    out["workload"] = f"pentadiagonal U[0,1] diagonals, Q + Q^T + n I, n={n}, nnz={nnz}, seed 0, {probes} Rademacher probes"
    return out


def workload_f1(L, h, A, grid: int, degree: int, seeds: int = 3):
    """Plain Hutchinson (Eq. Léja8) beside Hutch++ on the headline 3-D Laplacian at the same
    matvec budget (99 probes): Hutchinson runs the 99 probes through the trace step alone (width
    99, no pass 1 and no QR), Hutch++ runs 33 columns in pass 1 and 66 in pass 2. Time, bytes per
    estimate, and the error against the closed form over a few probe seeds."""
    from tests.pins import logdet_laplacian_3d
    exact = logdet_laplacian_3d(grid, SHIFT)
    n, nnz, m = A.n, A.nnz, degree
    out = {"exact_logdet": exact}
    for prec in ("df64", "f32"):
        dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
        row = {}
        for name in ("hutchinson", "hutchpp"):
            ms_l, errs = [], []
            for s in range(seeds):
                opts = L.options(degree=m, probes=PROBES, seed=SEED + s, precision=prec, estimator=name)
                ms, est = time_calls(lambda: L.ll_logdet_forward(h, dA, *BOUNDS, opts), 3, 2)
                ms_l.append(ms)
                errs.append(abs(est - exact) / abs(exact))
            inf = h.info()
            if name == "hutchinson":
                b = m * step_bytes(n, nnz, PROBES, prec, "dot")
                p2 = step_bytes(n, nnz, PROBES, prec, "dot") / (inf["ms_pass2"] / m / 1e3) / 1e9
            else:
                b = estimate_bytes(n, nnz, PROBES // 3, m, prec)
                p2 = step_bytes(n, nnz, 2 * (PROBES // 3), prec, "dot") / (inf["ms_pass2"] / m / 1e3) / 1e9
            ms = statistics.median(ms_l)
            row[name] = {"ms_per_estimate": ms, "GBps_estimate": b / (ms / 1e3) / 1e9, "pass2_launch_GBps": p2,
                         "rel_err_vs_exact": errs, "seeds": list(range(SEED, SEED + seeds)),
                         "phase_ms": {"probes": inf["ms_probes"], "pass1": inf["ms_pass1"], "qr": inf["ms_qr"],
                                      "pass2": inf["ms_pass2"]}}
        # Algorithm 2's stopping rule in both passes of Hutch++ (degree cap 150): every step runs
        # over the whole block until its last column stops, so the bytes are those of the
        # longest-running column of each pass
        for tol in (1e-2, 1e-4):
            opts = L.options(degree=150, probes=PROBES, seed=SEED, precision=prec, tol=tol)
            ms, est = time_calls(lambda: L.ll_logdet_forward(h, dA, *BOUNDS, opts), 3, 2)
            inf = h.info()
            k = PROBES // 3
            b = (inf["deg_max_pass1"] * step_bytes(n, nnz, k, prec, "accum") +
                 inf["deg_max_pass2"] * step_bytes(n, nnz, 2 * k, prec, "dot"))
            row[f"hutchpp_tol_{tol:g}"] = {
                "ms_per_estimate": ms, "GBps_estimate": b / (ms / 1e3) / 1e9,
                "rel_err_vs_exact": abs(est - exact) / abs(exact),
                "deg_max_pass1": inf["deg_max_pass1"], "deg_max_pass2": inf["deg_max_pass2"],
                "deg_mean_pass2": inf["deg_mean_pass2"],
                "phase_ms": {"probes": inf["ms_probes"], "pass1": inf["ms_pass1"], "qr": inf["ms_qr"],
                             "pass2": inf["ms_pass2"]}}
        out[prec] = row
        del dA
    out["workload"] = (f"L3D+{SHIFT}I on {grid}^3 (n={n}), bounds {list(BOUNDS)}, degree {m}, {PROBES} Rademacher "
                       f"probes: plain Hutchinson vs Hutch++ at equal matvecs, seeds {SEED}..{SEED + seeds - 1}; "
                       f"Hutch++ under Algorithm 2's stopping rule (degree cap 150, tol 1e-2 and 1e-4, seed {SEED})")
    return out


def workload_f4(L, h, N: int = 5000, thetas=(-0.24, -0.23, -0.22, -0.21, -0.20), probes: int = 30):
    """Section 5.3's GMRF: Q(theta) = I + theta Adj on the 5000 x 5000 4-neighbour grid (n = 2.5e7,
    nnz = 1.25e8). For each theta of the grid: Gershgorin bounds [1 - 4|theta|, 1 + 4|theta|]
    (sigma = 1 - 4|theta|), degree from the bounds, Hutch++ with 30 Rademacher probes (seed 0),
    log det Q(theta) and its theta-derivative (adjoint + chain, d a_e / d theta = 1 on the
    neighbour entries) against the closed forms. The structure is built once; the values of each
    theta are written on the device."""
    import math as _m
    import time as _t
    import torch
    from synth import gmrf_theta
    from tests.pins import dlogdet_gmrf_theta, logdet_gmrf_theta
    # the earlier workloads' blocks (kept W_j above all) leave the GMRF's blocks too little memory
    h.trim()
    torch.cuda.empty_cache()
    t0 = _t.perf_counter()
    A = gmrf_theta(N, 1.0)
    t_gen = _t.perf_counter() - t0
    dA = L.DeviceCSR.from_host(A)
    n, nnz, k = A.n, A.nnz, probes // 3
    del A
    counts = dA.rowptr[1:] - dA.rowptr[:-1]
    rows = torch.repeat_interleave(torch.arange(n, device="cuda", dtype=torch.int32), counts)
    offd = (dA.colind != rows).to(torch.float64)          # d a_e / d theta
    del rows
    out = {"n": n, "nnz": nnz, "generate_s": t_gen, "thetas": list(thetas), "rows": []}
    # the bounds and degrees of the grid (Gershgorin of Q(theta): [1 - 4|theta|, 1 + 4|theta|])
    grid = []
    for theta in thetas:
        dA.values = torch.where(offd > 0, torch.full_like(offd, theta), torch.ones_like(offd))
        lo, hi = L.ll_gershgorin(h, dA)
        kap = hi / lo
        rho = (_m.sqrt(kap) + 1) / (_m.sqrt(kap) - 1)
        grid.append((lo, hi, max(10, min(250, _m.ceil(_m.log(1e6) / _m.log(rho))))))
    # the whole grid in one sweep (ll_logdet_sweep: O = Adj, D = 1, one pass pair over all thetas,
    # the same probes for each), on a handle of its own that is closed before the per-theta runs
    hs = L.Handle()
    dO = L.DeviceCSR(n=n, rowptr=dA.rowptr, colind=dA.colind, values=offd)
    dD = torch.ones(n, dtype=torch.float64, device="cuda")
    sweep = {}
    for prec in ("df64", "f32"):
        so = L.options(degree=10, probes=probes, seed=0, precision=prec)
        ms_s, est_s = time_calls(lambda: L.ll_logdet_sweep(hs, dO, dD, list(thetas), [g[:2] for g in grid], so,
                                                           degrees=[g[2] for g in grid]), 2, 1)
        inf = hs.info()
        sweep[prec] = {"ms_sweep": ms_s, "estimates": [float(x) for x in est_s],
                       "phase_ms": {"probes": inf["ms_probes"], "pass1": inf["ms_pass1"], "qr": inf["ms_qr"],
                                    "pass2": inf["ms_pass2"]},
                       "shape_pass2": {"threads": inf["threads_pass2"], "pairs_per_thread": inf["pairs_pass2"],
                                       "rows_per_tile": inf["rows_pass2"]},
                       "launches": inf["kernel_launches"]}
    hs.close()
    del hs, dD
    torch.cuda.empty_cache()
    for theta in thetas:
        dA.values = torch.where(offd > 0, torch.full_like(offd, theta), torch.ones_like(offd))
        lo, hi = L.ll_gershgorin(h, dA)
        sg = lo if lo < 1 else 1.0
        kap = hi / lo
        rho = (_m.sqrt(kap) + 1) / (_m.sqrt(kap) - 1)
        m = max(10, min(250, _m.ceil(_m.log(1e6) / _m.log(rho))))
        exact, dexact = logdet_gmrf_theta(N, theta), dlogdet_gmrf_theta(N, theta)
        row = {"theta": theta, "bounds": [lo, hi], "sigma": sg, "degree": m, "exact_logdet": exact,
               "exact_dlogdet_dtheta": dexact}
        for prec in ("df64", "f32"):
            opts = L.options(degree=m, probes=probes, seed=0, precision=prec, keep_for_backward=(prec == "df64"))
            ms_f, est = time_calls(lambda: L.ll_logdet_forward(h, dA, lo, hi, opts), 2, 2)
            inf = h.info()
            r = {"ms_forward": ms_f, "estimate": est, "rel_err_vs_exact": abs(est - exact) / abs(exact),
                 "GBps_estimate": estimate_bytes(n, nnz, k, m, prec) / (ms_f / 1e3) / 1e9,
                 "phase_ms": {"probes": inf["ms_probes"], "pass1": inf["ms_pass1"], "qr": inf["ms_qr"],
                              "pass2": inf["ms_pass2"]}}
            if prec == "df64":
                ms_b, g = time_calls(lambda: L.ll_logdet_backward(h, dA, 1.0), 1, 0)
                th = float(L.ll_param_grad(h, g, offd[None, :])[0])
                del g
                r.update({"ms_backward": ms_b, "dlogdet_dtheta": th,
                          "rel_err_dtheta": abs(th - dexact) / abs(dexact)})
            row[prec] = r
        out["rows"].append(row)
    for prec, sw in sweep.items():
        seq = sum(r[prec]["ms_forward"] for r in out["rows"])
        sw["ms_sequential_forwards"] = seq
        sw["speedup_vs_sequential"] = seq / sw["ms_sweep"]
        sw["max_rel_diff_vs_forward"] = max(abs(e - r[prec]["estimate"]) / abs(r[prec]["estimate"])
                                            for e, r in zip(sw["estimates"], out["rows"]))
        sw["max_rel_err_vs_exact"] = max(abs(e - r["exact_logdet"]) / abs(r["exact_logdet"])
                                         for e, r in zip(sw["estimates"], out["rows"]))
    out["sweep"] = sweep
    out["workload"] = (f"GMRF Q(theta) = I + theta Adj on {N}^2 (n={n}, nnz={nnz}), theta in {list(thetas)}, "
                       f"Gershgorin bounds, degree from the bounds, Hutch++ {probes} Rademacher probes, seed 0; "
                       f"the grid once per theta (forward, backward) and as one sweep (forward)")
    return out


def profile_case(name: str):
    """Small single-call cases for ncu captures (see profiles/)."""
    import torch

    import paper_2603_02207_gb300 as L
    from paper_2603_02207_gb300 import build as _b
    _b.build()
    h = L.Handle()
    if name == "band":
        from synth import pentadiagonal
        A = pentadiagonal(2_000_000, seed=0)
        dA = L.DeviceCSR.from_host(A)
        lo, hi = L.ll_gershgorin(h, dA)
        L.ll_logdet_forward(h, dA, lo, hi, L.options(degree=8, probes=30, seed=0, precision="df64", use_graph=False))
    torch.cuda.synchronize()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="df64", choices=["df64", "f64", "f32"])
    ap.add_argument("--degree", type=int, default=60)
    ap.add_argument("--variants", type=int, default=1, help="also time the other precisions (1 = yes)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid", type=int, default=GRID_N, help="side of the 3-D grid (128 = the benchmark workload; "
                    "smaller sides are for profiler captures)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--c5-reorder", default="auto", choices=["auto", "none", "degree"],
                    help="row order of the config-5 forwards (auto = degree order for this power-law graph)")
    ap.add_argument("--c5-log2n", type=int, default=22,
                    help="log2 of the config-5 graph size (22 = the benchmark workload; smaller for profiler captures)")
    ap.add_argument("--step-kernel", default="auto", choices=["auto", "gather", "tma"],
                    help="step kernel of the headline passes (auto = autotuned; the others are for profiler captures)")
    ap.add_argument("--qr-gram", default="auto", choices=["auto", "tensor", "dfloat"],
                    help="CholeskyQR2 Gram kernel of the headline estimate (auto = timed per shape; the others "
                         "for profiler captures, under which the timed choice is distorted)")
    ap.add_argument("--rpt", type=int, default=0,
                    help="with --step-kernel: rows per thread (gather) or column pairs per thread (tma, 2 = FP32 "
                         "16-byte rows); for profiler captures")
    ap.add_argument("--workloads", default="c1,c3,c3t,c4,c5,f1,f3,f4",
                    help="extra workloads reported beside the headline (comma list of c1,c3,c3t,c4,c5,f1,f3,f4; "
                         "'' for none; c3t = the Matérn time to 1e-3 relative error)")
    ap.add_argument("--profile-case", default="", choices=["", "band"],
                    help="run one small case for a profiler capture and exit (no JSON line): band = one DF64 "
                         "forward on the pentadiagonal family at n = 2e6, degree 8, 30 probes, graphs off")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return profile_case(args.profile_case)

    import numpy as np
    import torch

    import paper_2603_02207_gb300 as L
    from paper_2603_02207_gb300 import build as _b
    from synth import laplacian_3d

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    _b.build()
    A = laplacian_3d(args.grid, SHIFT)
    n, nnz, k, m = A.n, A.nnz, PROBES // 3, args.degree
    h = L.Handle()
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def time_precision(prec: str, steps: int, warmup: int, sampler=None):
        dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
        opts = L.options(degree=m, probes=PROBES, seed=SEED + rank, precision=prec, step_kernel=args.step_kernel,
                         rows_per_thread=args.rpt, qr_gram=args.qr_gram)
        for _ in range(warmup):
            L.ll_logdet_forward(h, dA, *BOUNDS, opts)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if sampler:
            sampler.start()
        p1, p2, launches, est = [], [], 0, None
        e0.record(stream)
        for _ in range(steps):
            est = L.ll_logdet_forward(h, dA, *BOUNDS, opts)
            inf = h.info()
            p1.append(inf["ms_pass1"])
            p2.append(inf["ms_pass2"])
            launches += inf["kernel_launches"]
        e1.record(stream)
        barrier()
        clocks = sampler.stop() if sampler else None
        ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
        return dict(ms=ms, est=est, p1=p1, p2=p2, launches=launches, clocks=clocks, info=h.info(), dA=dA, opts=opts)

    prec = args.precision
    sampler = ClockSampler(local) if rank == 0 else None
    r = time_precision(prec, args.steps, args.warmup, sampler)
    ms_step = r["ms"] / args.steps
    bytes_est = estimate_bytes(n, nnz, k, m, prec)
    value = world * bytes_est * args.steps / (r["ms"] / 1e3) / 1e9

    # roofline of the dominant kernel (the pass-2 fused SpMM + trace step, width 2k)
    peaks, peak_src = load_peaks()

    def roofline_of(pr: str, rr: dict) -> dict:
        p2_launch_ms = statistics.median(rr["p2"]) / m
        p1_launch_ms = statistics.median(rr["p1"]) / m
        b_p2 = step_bytes(n, nnz, 2 * k, pr, "dot")
        b_p1 = step_bytes(n, nnz, k, pr, "accum")
        achieved = b_p2 / (p2_launch_ms / 1e3) / 1e9
        kname = {L.LL_KERNEL_TMA: "tma", L.LL_KERNEL_GATHER: "gather"}.get(rr["info"]["kernel_pass2"], "gather")
        per_row = TRACE_STEP_DRAM_BYTES_PER_ROW.get((kname, pr))
        kfun = "k_leja_tma" if kname == "tma" else "k_leja_step"
        ach1 = b_p1 / (p1_launch_ms / 1e3) / 1e9
        inf = rr["info"]
        return {"kernel": (f"{kfun}<{pr},DOT> (b={2 * k}, {inf['threads_pass2']} threads/CTA, "
                           f"{2 * inf['pairs_pass2']} columns/thread)"), "bound": "hbm",
                "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "traffic": per_row * n if per_row else None,
                "traffic_source": (f"ncu dram__bytes_read+write of one {kfun} launch on a smaller 3-D Laplacian, "
                                   "scaled by rows") if per_row else None,
                "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs, burst copy)",
                "per_launch_bytes": b_p2, "per_launch_ms": p2_launch_ms,
                "pass1_kernel": {"kernel": (f"{kfun}<{pr},ACCUM> (b={k}, {inf['threads_pass1']} threads/CTA, "
                                            f"{2 * inf['pairs_pass1']} columns/thread)"),
                                 "achieved": ach1, "frac": ach1 / peaks["hbm_gbs"], "per_launch_bytes": b_p1,
                                 "per_launch_ms": p1_launch_ms}}

    roof = roofline_of(prec, r)

    # end to end through the C ABI with host buffers (CSR copied host->device every call)
    e2e = None
    if not args.no_e2e:
        opts = r["opts"]
        Ah = A
        for _ in range(1):
            L.ll_logdet_forward_host(h, Ah, *BOUNDS, opts)
        barrier()
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            L.ll_logdet_forward_host(h, Ah, *BOUNDS, opts)
        e1.record(stream)
        barrier()
        wall = max_over_ranks(time.perf_counter() - t0, world, "cuda")
        vs = 4 if prec == "f32" else 8
        h2d = 4 * (n + 1) + 4 * nnz + vs * nnz
        d2h = (m + 1) * (2 * k) * 8 + 2 * 4
        e2e = {"value": world * bytes_est * args.steps / wall / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": wall * 1e3 / args.steps}

    # every precision side by side, each with the roofline of its own trace and P-axpy steps
    from tests.pins import logdet_laplacian_3d  # closed form, for the reported error only
    exact = logdet_laplacian_3d(args.grid, SHIFT)

    def precision_entry(pr: str, rr: dict, steps: int) -> dict:
        bv = estimate_bytes(n, nnz, k, m, pr)
        v = world * bv * steps / (rr["ms"] / 1e3) / 1e9
        inf = rr["info"]
        return {"dtype": DTYPE_NAME[pr], "value": v, "unit": UNIT, "hbm_frac_of_measured": v / peaks["hbm_gbs"],
                "ms_per_step": rr["ms"] / steps, "estimate": rr["est"],
                "rel_err_vs_exact": abs(rr["est"] - exact) / abs(exact),
                "phase_ms": {"probes": inf["ms_probes"], "pass1": inf["ms_pass1"], "qr": inf["ms_qr"],
                             "pass2": inf["ms_pass2"]},
                "roofline": roofline_of(pr, rr)}

    precisions = {prec: precision_entry(prec, r, args.steps)}
    if args.variants:
        for other in ("df64", "f64", "f32"):
            if other == prec:
                continue
            rv = time_precision(other, 3, 2)
            precisions[other] = precision_entry(other, rv, 3)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    extra = {}
    for w in [x for x in args.workloads.split(",") if x]:
        if w == "f1":
            extra[w] = workload_f1(L, h, A, args.grid, m)
            continue
        fn = {"c1": workload_config1, "c3": workload_config3, "c3t": workload_c3_time_to_tol, "c4": workload_config4,
              "c5": workload_config5, "f3": workload_f3, "f4": workload_f4}[w]
        extra[w] = fn(L, h, log2n=args.c5_log2n, reorder=args.c5_reorder) if w == "c5" else fn(L, h)
    c3t = extra.pop("c3t", None)
    cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline(A, prec)
    info = r["info"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE_NAME[prec], "data": "synthetic",
        "config": {"workload": f"L3D+{SHIFT}I on {args.grid}^3 (n={n}, nnz={nnz}), bounds {list(BOUNDS)}, "
                               f"degree {m}, Hutch++ {PROBES} Rademacher probes (k={k}), seed {SEED}",
                   "global_batch": world, "seq_len": None, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (probe blocks 0.5-1.1 GB, matrix 175 MB); no flush"},
        "hbm_frac_of_measured": value / peaks["hbm_gbs"],
        "matvecs_per_s": world * m * 3 * k * args.steps / (r["ms"] / 1e3),
        "estimate": r["est"], "exact_logdet": exact, "rel_err_vs_exact": abs(r["est"] - exact) / abs(exact),
        "phase_ms": {"probes": info["ms_probes"], "pass1": info["ms_pass1"], "qr": info["ms_qr"],
                     "pass2": info["ms_pass2"], "total": info["ms_total"]},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        "c3_time_to_1e-3": c3t,
        "gpu_launches": r["launches"], "clocks": r["clocks"], "precisions": precisions, "workloads": extra,
    }
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
