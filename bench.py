#!/usr/bin/env python3
"""Environment-step throughput of the GPU channel-flow DNS.

Default line (one GPU): the batched mixed-precision form against the plain
FP64 form on the same grid, both on this GPU in this run.

* value: 256 minimal channels (paper Sec. 3.1 first domain: 2.67h x 2h x 0.8h,
  16 x 65 x 16 modes, Re_tau 180, Re_b 2800, dt 0.005) advanced together by
  one handle, mixed precision (FP32 nonlinear term, FP64 tau solves,
  influence-matrix correction and flow-rate update), each environment with its
  own seeded state and a per-step seeded zero-net-mass-flux Gaussian wall
  action (std 0.05 u_tau); every step replays the captured CUDA graph.
  Environment steps per second, CUDA events per step on the library's stream.
* comparison: the plain FP64 single-environment minimal channel timed the same
  way in the same process; `speedup` is the ratio of the two throughputs.
* served: the same 256 channels behind the continuous-batching server, actor
  threads submitting actions (closed loop at saturation, and with exponential
  think times), with the server's p50/p99 submit-to-result latency.
* accuracy: the cpu_baseline leg replays a 10-step window of one sampled
  environment of the timed handle on the FP64 oracle (same state, same
  actions) and reports the relative error of every output.
* larger_fp64: the larger channel (2 pi h x 2h x pi h, 64 x 65 x 64, FP64,
  opposition control, Sec. 4.1) with the FP64 plane kernel's roofline.
* e2e: the batched mixed form through env_step with pinned host buffers
  (H2D of the 256 actions, D2H of the observations, wall shears and rewards).

The seeded initial states are broadband divergence-free perturbations of
laminar Poiseuille flow (the paper's developed-turbulence fields are not
available); the per-step work does not depend on the values.  The working set
of the 256 channels (0.4 GB) exceeds L2, and a 256 MiB L2 flush is written
between timed steps of every handle, outside the timed events.

--workload selects one of the single-handle or served workloads instead.
--impl reference: the FP64 CPU oracle on the host cores, a bounded sample of
the same workload.  Several GPUs: one process per GPU (torchrun),
independent replicas, no collective on the data path.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

LARGER = dict(nx=64, ny=65, nz=64, lx=2 * math.pi, lz=math.pi, re_tau=180.0, re_bulk=2800.0,
              dt=0.005, control=1, alpha=1.0, steps_per_action=1, y_sense_plus=15.0)
MINIMAL = dict(nx=16, ny=65, nz=16, lx=2.67, lz=0.8, re_tau=180.0, re_bulk=2800.0,
               dt=0.005, control=0, alpha=1.0, steps_per_action=1, y_sense_plus=15.0)
# name -> (parameters, batch, precision, description)
WORKLOADS = {
    "minimal_batch256_mixed": (MINIMAL, 256, 1,
                               "256 minimal channels 16x65x16 (Re_tau 180) in one handle, mixed precision "
                               "(FP32 nonlinear term, FP64 tau solves), per-step seeded ZNMF Gaussian actions "
                               "std 0.05 u_tau, captured-graph replay"),
    "minimal_batch256_fp64": (MINIMAL, 256, 0,
                              "256 minimal channels 16x65x16 (Re_tau 180) in one handle, all FP64, per-step "
                              "seeded ZNMF Gaussian actions std 0.05 u_tau, captured-graph replay"),
    "open_minimal_batch256_mixed": (dict(MINIMAL, top_bc=1, lx=2 * 2.67, lz=2 * 0.8), 256, 1,
                                    "256 minimal open channels 16x65x16 (free-slip top, the paper's 2.67h x h x "
                                    "0.8h box with h = 2 in units of y), mixed precision, per-step seeded ZNMF "
                                    "Gaussian actions std 0.05 u_tau, captured-graph replay"),
    "minimal_fp64": (MINIMAL, 1, 0,
                     "plain FP64 minimal channel 16x65x16 (Re_tau 180), one environment, per-step seeded ZNMF "
                     "Gaussian actions std 0.05 u_tau, captured-graph replay"),
    "larger_fp64": (LARGER, 1, 0,
                    "larger channel Re_tau=180, 64x65x64, all FP64, opposition control, 1 RK3 step per env step"),
    "larger_mixed": (LARGER, 1, 1,
                     "larger channel Re_tau=180, 64x65x64, mixed FP32 nonlinear term / FP64 solves, opposition"),
    "minimal_batch256_policy_mixed": (dict(MINIMAL, control=2), 256, 1,
                                      "256 minimal channels 16x65x16, mixed precision, on-device policy closing "
                                      "the loop: 3x3 window of u, v per agent, two ReLU layers of 64, u_tau tanh "
                                      "output, seeded random weights"),
    "large550_mixed": (dict(MINIMAL, nx=256, ny=193, nz=256, lx=2 * math.pi, lz=math.pi, re_tau=550.0,
                            re_bulk=10030.0, dt=0.002), 1, 1,
                       "large channel Re_tau=550, 256x193x256, mixed precision, seeded ZNMF Gaussian actions "
                       "std 0.05 u_tau"),
    "large395_fp64": (dict(MINIMAL, nx=128, ny=129, nz=128, lx=2 * math.pi, lz=math.pi, re_tau=395.0,
                           re_bulk=6875.0, dt=0.0025), 1, 0,
                      "channel Re_tau=395, 128x129x128, all FP64, seeded ZNMF Gaussian actions std 0.05 u_tau"),
    "large395_mixed": (dict(MINIMAL, nx=128, ny=129, nz=128, lx=2 * math.pi, lz=math.pi, re_tau=395.0,
                            re_bulk=6875.0, dt=0.0025), 1, 1,
                       "channel Re_tau=395, 128x129x128, mixed precision, seeded ZNMF Gaussian actions "
                       "std 0.05 u_tau"),
    "large550_fp64": (dict(MINIMAL, nx=256, ny=193, nz=256, lx=2 * math.pi, lz=math.pi, re_tau=550.0,
                           re_bulk=10030.0, dt=0.002), 1, 0,
                      "large channel Re_tau=550, 256x193x256, all FP64, seeded ZNMF Gaussian actions "
                      "std 0.05 u_tau"),
}
# the default line: batched mixed form against the plain FP64 form on the same grid
DEFAULT_WORKLOAD = "target"
TARGET_BATCHED, TARGET_PLAIN, TARGET_SERVED = "minimal_batch256_mixed", "minimal_fp64", "served_minimal256_mixed"
# on-device policy of the control-2 workloads: (wz, wx, hidden widths, u_tau tanh output, weight seed)
POLICIES = {"minimal_batch256_policy_mixed": (3, 3, (64, 64), True, 77)}


def policy_weights(wz: int, wx: int, hidden: tuple, seed: int) -> np.ndarray:
    """Seeded random weights (no trained policy exists): N(0, 1/fan_in) per
    layer, biases N(0, 0.01); layer layout W [out][in] then b [out]."""
    rng = np.random.default_rng(seed)
    sizes = [2 * wz * wx] + list(hidden) + [1]
    parts = []
    for i in range(len(sizes) - 1):
        parts.append(rng.standard_normal(sizes[i + 1] * sizes[i]) / math.sqrt(sizes[i]))
        parts.append(rng.standard_normal(sizes[i + 1]) * 0.1)
    return np.concatenate(parts)


# served workloads: (list of (parameters, count), slots per class, environments per actor thread,
# description)
MID = dict(LARGER, nx=32, nz=32, control=0)
BIG395 = dict(LARGER, nx=128, ny=129, nz=128, re_tau=395.0, re_bulk=6890.0, control=0)
SERVED = {
    "served_minimal256_mixed": ([(dict(MINIMAL, precision=1), 256)], 256, 32,
                                "served: 256 minimal channels 16x65x16, mixed precision, actor threads with "
                                "exponential think time, continuous batching"),
    "served_mixed_sizes": ([(dict(MINIMAL, precision=1), 24), (dict(MID, precision=1), 12),
                            (dict(LARGER, control=0, precision=1), 8), (dict(BIG395, precision=1), 4)], 24, 4,
                           "served: 48 environments 24x16x65x16 + 12x32x65x32 + 8x64x65x64 (Re_tau 180) + "
                           "4x128x129x128 (Re_tau 395), mixed precision, admitted by HBM budget"),
}
METRIC = "env_steps_per_s"
UNIT = "env-steps/s"
KERNEL_CLASSES = ("stage_pre", "nonlinear_plane", "stage_post", "per_step")
L2_FLUSH_BYTES = 256 << 20


def plane_kernel_flops(nx: int, ny: int, nz: int) -> float:
    """Algorithmic FLOPs of one launch of the nonlinear plane kernel.

    Per Gauss-Lobatto plane: 6 inverse and 3 forward complex FFTs along z of
    length mz on nx/2 columns, 6 inverse and 3 forward real FFTs along x of
    length mx on mz rows (5 n log2 n per complex, 2.5 n log2 n per real
    transform), and the cross product (9 FLOPs per padded point)."""
    mx, mz, nxh = 3 * nx // 2, 3 * nz // 2, nx // 2
    z = 9 * nxh * 5.0 * mz * math.log2(mz)
    x = 9 * mz * 2.5 * mx * math.log2(mx)
    return ny * (z + x + 9.0 * mx * mz)


def kernel_bytes(nx: int, ny: int, nz: int, batch: int, node_bytes: int) -> dict:
    """Algorithmic HBM bytes of one launch of each stage kernel.

    Per Fourier mode (complex FP64 = 16 B, nodal complex = node_bytes):
    stage_pre reads v, omega_y and writes the six nodal fields; the plane kernel
    reads those six and writes the three nodal H fields; stage_post reads H, v,
    omega_y and the two previous nonlinear terms and writes the last four back."""
    M = batch * (nx // 2) * ny * nz
    return {"stage_pre": M * (2 * 16 + 6 * node_bytes),
            "nonlinear_plane": M * 9 * node_bytes,
            "stage_post": M * (3 * node_bytes + 8 * 16)}


def implicit_half_fp64_flops(nx: int, ny: int, nz: int, batch: int, mixed: bool = False) -> float:
    """Algorithmic FP64 FLOPs of one launch of the implicit half of a stage
    (right-hand sides, tau solves, influence correction), counting a fused
    multiply-add as 2.  Per Chebyshev coefficient of one class and real
    component: omega_y right-hand side 12, tau solve 13, update 2; v wall sums
    4, derivative walk and right-hand side 21, two tau solves 26, influence
    sum 3, update 4: 85 per coefficient, (N+1) coefficients of both parities
    over the two classes and 2 components: 170 (N+1) per mode, for every mode
    but the Nyquist row.  In the mixed path the nonlinear-term part of the
    right-hand sides (h_g, t, Dt, h_v and dt (gamma h + zeta h')) is FP32:
    8 of the omega_y and 12 of the v FLOPs, leaving 65 FP64 per coefficient,
    130 (N+1) per mode."""
    modes = batch * (nx // 2) * (nz - 1)
    return (130.0 if mixed else 170.0) * ny * modes


def slowest_rank_ms(total_ms: float, dist, device: str = "cuda") -> float:
    """Job time of a replica run: the maximum over ranks of the per-rank timed
    totals (the slowest rank sets it); a single process keeps its own."""
    if dist is None:
        return total_ms
    import torch
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(steps: int, batch: int, world: int, job_ms: float) -> float:
    """Environment steps of all ranks per second of job time (weak scaling:
    every rank advances its own `batch` environments `steps` times)."""
    return steps * batch * world / (job_ms * 1e-3)




def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the roofline kernel, from one ncu capture of the same workload (summaries
# under profiles/); absent where no capture of the current kernel exists
TRAFFIC_BYTES = {
    ("minimal_batch256_mixed", "stage_post"): (152.163072 + 42.973952) * 1e6,
    # the three passes of one FP64 64x64-mode stage (the scratch stays in L2)
    ("larger_fp64", "nonlinear_plane"): (12.597248 + 19.201792 + 9.604352) * 1e6,
    # the three passes of one FP64 256x256-mode stage (z inverse + x pass + z forward)
    ("large550_fp64", "nonlinear_plane"): (604.911872 + 852.392448 + 910.863872 + 413.775360 + 455.520000
                                           + 259.116544) * 1e6,
}

# FP64 FMA rate: 152 SMs x 2 FP64 FMA/clk/SM x 2 FLOP x 2.07 GHz; an FMA-chain probe
# measured 1.19 TFLOP/s at a 1.96 GHz SM clock, the same rate per clock
FP64_PEAK_TFLOPS = 1.2586
FP64_PEAK_SOURCE = ("FP64 FMA pipe: 152 SMs x 2 FMA/clk x 2 FLOP x 2.07 GHz (nominal 1.25 TFLOP/s; "
                    "FMA probe measured 1.19 at 1.96 GHz)")


def measure_fp64_peak() -> dict:
    """FP64 throughput of a plain library GEMM on this GPU, in this run:
    torch.matmul on 4096 x 4096 float64 operands (cuBLAS DGEMM, 2 n^3 FLOP),
    best of 5 after a warm-up, CUDA events.  The denominator of the FP64
    rooflines, as the copy test and the bf16 GEMM are for the others."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = None
    for _ in range(5):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        torch.matmul(a, b)
        e.record()
        torch.cuda.synchronize()
        ms = s.elapsed_time(e)
        best = ms if best is None else min(best, ms)
    del a, b
    return {"tflops": 2.0 * n ** 3 / (best * 1e-3) / 1e12, "ms": best,
            "how": "torch.matmul float64 4096^3 (cuBLAS DGEMM), best of 5, CUDA events, this run"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_model() -> str:
    """Host CPU model for the oracle timing (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def oracle_single_thread(budget_s: float, workload: str) -> dict | None:
    """The oracle sample in a fresh process with one BLAS/OpenMP thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json, bench; t = bench.oracle_sample(%r, 1000, %r); "
            "print(json.dumps({'steps': len(t), 'seconds': sum(t)}))" % (budget_s, workload))
    try:
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                             timeout=budget_s * 4 + 120)
        r = json.loads(out.stdout.strip().splitlines()[-1])
    except (OSError, subprocess.SubprocessError, ValueError, IndexError):
        return None
    return {"value": r["steps"] / r["seconds"], "cores": 1,
            "sample": f"{r['steps']} whole environment steps, one BLAS/OpenMP thread"}




def _oracle_params(prm: dict, control: int | None = None):
    from oracle import channel
    keys = ("nx", "ny", "nz", "lx", "lz", "re_tau", "re_bulk", "dt", "steps_per_action",
            "y_sense_plus", "control", "alpha")
    kw = {k: prm[k] for k in keys}
    if control is not None:
        kw["control"] = control
    return channel.Params(**kw)


def oracle_sample(budget_s: float, max_steps: int, workload: str = TARGET_BATCHED):
    """Time the FP64 oracle on one environment of the workload: whole
    environment steps until the budget is spent."""
    import seeded_inputs as si
    from oracle import channel
    from oracle import policy as opol
    prm = WORKLOADS[workload][0]
    pol = POLICIES.get(workload) if prm["control"] == 2 else None
    op = _oracle_params(prm, 0 if pol else None)   # the oracle's policy supplies the external action
    ops = channel.Operators(op)
    st = channel.new_state(si.perturbed_poiseuille(op.nx, op.ny, op.nz, 0, 0.1, 99), op)
    rng = np.random.default_rng(0)
    if pol:
        wz, wx, hidden, tanh_out, wseed = pol
        w = policy_weights(wz, wx, hidden, wseed)
        obs = channel.observation(st, ops)
    times = []
    t_all = time.perf_counter()
    while len(times) < max_steps and (time.perf_counter() - t_all) < budget_s:
        act = None
        if op.control == 0 and not pol:
            act = rng.standard_normal((op.nz, op.nx)) * 0.05 * op.u_tau
            act -= act.mean()
        t0 = time.perf_counter()
        if pol:
            act = opol.actions(obs[None], w, wz, wx, hidden, tanh_out, op.u_tau)[0]
        obs, _, _ = channel.env_step(st, ops, act)
        times.append(time.perf_counter() - t0)
    return times


def oracle_window(prm: dict, state: dict, actions: list, budget_s: float):
    """cpu_baseline leg with a check: the FP64 oracle replays a window of
    environment steps of one sampled environment from `state` (the library's
    serialised state before the window) with the same `actions`, timed; after
    the window it keeps stepping (zero action) until the budget is spent.
    Returns (per-step seconds, [(obs, tau_w, reward) of the window], final
    window state in the library's layout)."""
    from oracle import channel
    op = _oracle_params(prm)
    ops = channel.Operators(op)
    st = channel.new_state(state, op)
    st["vw"] = np.array(state["vw"], copy=True)   # the ramp starts from the last applied action
    times, outs, final = [], [], None
    t_all = time.perf_counter()
    for a in actions:
        t0 = time.perf_counter()
        outs.append(channel.env_step(st, ops, a))
        times.append(time.perf_counter() - t0)
    final = channel.canonical(st)
    zero = None if op.control != 0 else np.zeros((op.nz, op.nx))
    while time.perf_counter() - t_all < budget_s:
        t0 = time.perf_counter()
        channel.env_step(st, ops, zero)
        times.append(time.perf_counter() - t0)
    return times, outs, final


def _rel(a, b) -> float:
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0))


def window_errors(lib_outs, lib_final, ora_outs, ora_final, u_tau: float) -> dict:
    """Relative error of every output of a window against the oracle (max over
    its steps for the per-step outputs)."""
    err = {k: _rel(lib_final[k], ora_final[k]) for k in ("v", "g", "U")}
    err["W_vs_U"] = float(np.linalg.norm(lib_final["W"] - ora_final["W"]) / np.linalg.norm(ora_final["U"]))
    err["obs"] = max(_rel(a[0], b[0]) for a, b in zip(lib_outs, ora_outs))
    err["wall_shear"] = max(abs(a[1] - b[1]) / abs(b[1]) for a, b in zip(lib_outs, ora_outs))
    err["reward"] = max(abs(a[2] - b[2]) / max(abs(b[2]), abs(b[1]) / u_tau ** 2) for a, b in zip(lib_outs, ora_outs))
    return err


def config_of(workload: str, world: int = 1, info=None) -> dict:
    """The config dict of a line (identical for our arm and the reference arm)."""
    name = workload if workload != DEFAULT_WORKLOAD else TARGET_BATCHED
    prm, B, prec, desc = WORKLOADS[name]
    ctrl = {0: "external seeded ZNMF Gaussian actions std 0.05 u_tau", 1: "opposition alpha=1",
            2: "on-device policy"}[prm["control"]]
    cfg = {"workload": desc, "grid": [prm["nx"], prm["ny"], prm["nz"]], "batch": B,
           "precision": "mixed FP32/FP64" if prec else "FP64", "re_tau": prm["re_tau"], "re_bulk": prm["re_bulk"],
           "dt": prm["dt"], "control": ctrl,
           "l2": "working set above L2 for the 256-channel handle; 256 MiB L2 flush between timed steps of every "
                 "handle, outside the timed events",
           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}
    if workload == DEFAULT_WORKLOAD:
        cfg["compared_with"] = WORKLOADS[TARGET_PLAIN][3]
    return cfg


def run_reference(args, rank: int, world: int):
    """The FP64 CPU oracle on the host cores, a bounded sample of the workload."""
    if rank != 0:
        return
    name = args.workload if args.workload in WORKLOADS else TARGET_BATCHED
    budget = float(os.environ.get("CH_REFERENCE_BUDGET_S", "90"))
    for _ in range(min(args.warmup, 1)):
        oracle_sample(1e9, 1, name)
    times = oracle_sample(budget, max(1, args.steps), name)
    total = sum(times)
    value = len(times) / total
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": len(times), "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(args.workload, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "cpu": cpu_model(), "kind": "oracle",
                         "sample": f"{len(times)} whole environment steps of one environment of the workload "
                                   f"(budget {budget:.0f} s)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU timing of one handle
# ---------------------------------------------------------------------------

class Handle:
    """One library handle of a workload with its seeded actions, on a dedicated
    stream shared with the L2 flush and the timing events (the library's own
    stream is non-blocking and would not order with torch's legacy stream)."""

    N_CYCLE = 32

    def __init__(self, native, workload: str, rank: int, autotune: bool):
        import torch
        self.native, self.name = native, workload
        self.prm, self.B, self.prec, self.desc = WORKLOADS[workload]
        p = native.params(**self.prm, batch=self.B, precision=self.prec, autotune=1 if autotune else 0)
        self.env = native.env_create(p)
        self.info = native.env_info(self.env)
        if self.prm["control"] == 2:
            wz, wx, hidden, tanh_out, wseed = POLICIES[workload]
            native.env_set_policy(self.env, native.policy(wz, wx, hidden, tanh_out),
                                  policy_weights(wz, wx, hidden, wseed))
        native.env_reset(self.env, seed=1000 * rank, amplitude=0.1, kmax=99)
        self.stream = torch.cuda.Stream()
        native.env_set_stream(self.env, self.stream.cuda_stream)
        nx, nz = self.prm["nx"], self.prm["nz"]
        self.out_len = 2 * nz * nx + 2
        self.d_out = torch.zeros(self.B * self.out_len, dtype=torch.float64, device="cuda")
        self.external = self.prm["control"] == 0
        self.u_tau = self.prm["re_tau"] / self.prm["re_bulk"]
        if self.external:
            # seeded zero-net-mass-flux Gaussian wall actions, std 0.05 u_tau, cycled
            rng = np.random.default_rng(1234 + rank)
            acts = rng.standard_normal((self.N_CYCLE, self.B, nz, nx)) * 0.05 * self.u_tau
            acts -= acts.mean(axis=(2, 3), keepdims=True)
            self.h_acts = torch.from_numpy(acts).pin_memory()
            self.d_acts = self.h_acts.to("cuda")

    def act_ptr(self, i: int):
        return self.d_acts[i % self.N_CYCLE].data_ptr() if self.external else None

    def host_act(self, i: int):
        return self.h_acts[i % self.N_CYCLE].numpy() if self.external else None

    def step_device(self, i: int):
        self.native.env_step_device(self.env, self.act_ptr(i), self.d_out.data_ptr())

    def timed(self, K: int, W: int, flush, dist, profile: bool):
        """W untimed steps, then K steps each between CUDA events (barrier and
        synchronize on both sides).  profile=False replays the captured graph;
        profile=True launches the kernels one by one between per-class events.
        Returns (per-step ms, per-class kernel totals or None)."""
        import torch
        with torch.cuda.stream(self.stream):
            for i in range(W):
                self.step_device(i)
            torch.cuda.synchronize()
            starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
            ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            if profile:
                self.native.env_profile(self.env, True)
            for i in range(K):
                flush.zero_()
                starts[i].record(self.stream)
                self.step_device(W + i)
                ends[i].record(self.stream)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
        kern = None
        if profile:
            kern = {}
            for c, name in enumerate(KERNEL_CLASSES):
                ms, n = self.native.env_profile_read(self.env, c)
                kern[name] = {"ms_total": ms, "launches": n}
            self.native.env_profile(self.env, False)
        return [s.elapsed_time(e) for s, e in zip(starts, ends)], kern

    def e2e(self, K: int, flush, dist, world: int):
        """The same metric through env_step with pinned host buffers (H2D of
        the actions, D2H of the outputs inside the timed region)."""
        import torch
        nx, nz, B = self.prm["nx"], self.prm["nz"], self.B
        obs = torch.zeros((B, 2, nz, nx), dtype=torch.float64).pin_memory().numpy()
        tau = torch.zeros(B, dtype=torch.float64).pin_memory().numpy()
        rew = torch.zeros(B, dtype=torch.float64).pin_memory().numpy()
        for i in range(3):
            self.native.env_step(self.env, self.host_act(i), obs, tau, rew)
        ms = []
        for i in range(K):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            self.native.env_step(self.env, self.host_act(i), obs, tau, rew)
            ms.append(1e3 * (time.perf_counter() - t0))
        total = slowest_rank_ms(sum(ms), dist)
        return {"value": job_throughput(K, B, world, total), "unit": UNIT,
                "h2d_bytes_per_step": 8 * B * nz * nx if self.external else 0,
                "d2h_bytes_per_step": 8 * B * self.out_len}

    def window(self, n: int, slot: int = 0):
        """n environment steps through env_step with the first n cycled actions;
        returns (state of `slot` before, its actions, its outputs per step, its
        state after)."""
        nx, ny, nz, B = self.prm["nx"], self.prm["ny"], self.prm["nz"], self.B
        unpack = lambda: self.native.unpack_state(self.native.env_get_state(self.env, slot), nx, ny, nz)
        before = unpack()
        obs, tau, rew = np.zeros((B, 2, nz, nx)), np.zeros(B), np.zeros(B)
        acts, outs = [], []
        for i in range(n):
            a = self.host_act(i)
            rc = self.native.env_step(self.env, a, obs, tau, rew)
            assert rc == self.native.CH_OK, rc
            acts.append(None if a is None else np.array(a[slot], copy=True))
            outs.append((obs[slot].copy(), float(tau[slot]), float(rew[slot])))
        return before, acts, outs, unpack()

    def close(self):
        self.native.env_destroy(self.env)


def roofline_of(workload: str, kern: dict, fp64_peak: dict | None = None) -> dict:
    """Roofline of the FP64 kernel that bounds the workload, against the FP64
    peak, with algorithmic work per launch and the kernel's average launch
    time from the profiled region.  All-FP64 handles: the larger of the plane
    kernel and the implicit half of the stage; mixed handles: the implicit
    half (FP64 tau solves; the plane kernel is FP32)."""
    prm, B, prec, _ = WORKLOADS[workload]
    nx, ny, nz = prm["nx"], prm["ny"], prm["nz"]
    dom = max(kern, key=lambda k: kern[k]["ms_total"])
    kk = "stage_post"
    if prec == 0 and kern["nonlinear_plane"]["ms_total"] >= kern["stage_post"]["ms_total"]:
        kk = "nonlinear_plane"
    avg_s = kern[kk]["ms_total"] * 1e-3 / max(kern[kk]["launches"], 1)
    if kk == "nonlinear_plane":
        flops = B * plane_kernel_flops(nx, ny, nz)
    else:
        flops = implicit_half_fp64_flops(nx, ny, nz, B, mixed=prec == 1)
    achieved = flops / avg_s / 1e12
    if fp64_peak:
        peak, source = fp64_peak["tflops"], "of measured: " + fp64_peak["how"]
    else:
        peak, source = FP64_PEAK_TFLOPS, FP64_PEAK_SOURCE + " (derived)"
    r = {"kernel": kk, "dominant_kernel": dom, "bound": "alu", "unit": "TFLOP/s", "achieved": achieved,
         "peak": peak, "frac": achieved / peak, "peak_source": source,
         "frac_of_derived_fma_peak": achieved / FP64_PEAK_TFLOPS,
         "flops_per_launch": flops, "avg_launch_ms": avg_s * 1e3,
         "traffic": TRAFFIC_BYTES.get((workload, kk))}
    if prec == 1:
        peaks = measured_peaks()
        nbytes = kernel_bytes(nx, ny, nz, B, 8)[kk]
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        r["hbm"] = {"bytes_per_launch": nbytes, "achieved_gbs": nbytes / avg_s / 1e9, "peak_gbs": hbm,
                    "frac": nbytes / avg_s / 1e9 / hbm,
                    "peak_source": "of measured" if "hbm_gbs" in peaks else "of fallback"}
    return r


def percentiles(ms: list) -> dict:
    a = np.sort(np.asarray(ms))
    return {"p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99))}


def measure_handle(native, workload: str, args, rank: int, world: int, flush, dist, e2e: bool = True,
                   fp64_peak: dict | None = None) -> dict:
    """Graph-replay timing (value), a profiled pass (kernel breakdown and
    roofline) and the end-to-end host-buffer timing of one workload."""
    h = Handle(native, workload, rank, autotune=not args.no_autotune)
    try:
        W = max(3, args.warmup)
        K = args.steps
        step_ms, _ = h.timed(K, W, flush, dist, profile=False)
        total = slowest_rank_ms(sum(step_ms), dist)
        prof_ms, kern = h.timed(K, 1, flush, dist, profile=True)
        res = {"value": job_throughput(K, h.B, world, total), "ms_per_step": total / K, "steps": K,
               "warmup": W, **percentiles(step_ms),
               "kernels_ms_per_step": {k: v["ms_total"] / K for k, v in kern.items()},
               "profiled_ms_per_step": sum(prof_ms) / K,
               "roofline": roofline_of(workload, kern, fp64_peak),
               "gpu_launches": K * h.info.launches_per_step,
               "tiles": {"ppc_pre": h.info.ppc_pre, "ppc_post": h.info.ppc_post,
                         "post_batched": h.info.post_batched, "autotuned": bool(h.info.tuned),
                         "tune_ms": h.info.tune_ms, "plane_cluster": h.info.plane_cluster,
                         "plane_team": h.info.plane_team},
               "finite": bool(np.isfinite(h.d_out.cpu().numpy()).all())}
        nx, ny, nz = h.prm["nx"], h.prm["ny"], h.prm["nz"]
        res["mpts_rk3_steps_per_s"] = res["value"] * nx * ny * nz / 1e6
        step_bytes = sum(v * 3 for v in kernel_bytes(nx, ny, nz, h.B, 16 if h.prec == 0 else 8).values())
        res["algorithmic_gbs_per_step"] = step_bytes / (res["ms_per_step"] * 1e-3) / 1e9
        if e2e:
            res["e2e"] = h.e2e(min(K, 300), flush, dist, world)
        res["_handle"] = h
        return res
    except BaseException:
        h.close()
        raise


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------

def served_run(native, workload: str, rate: float, duration: float, warm: float = 3.0,
               linger_us: int | None = None) -> dict:
    """Continuous-batching server driven by actor threads.

    Each actor thread drives a group of CH_SERVE_GROUP environments of one
    class (default per workload): it submits one action for every environment
    of its group in one call (srv_submit_many), waits for the group's results
    in one call (srv_wait_many), thinks for an exponentially
    distributed time of mean 1/rate (0: none, saturation) and repeats until
    the time budget is spent.  Groups larger than one keep the Python threads
    few, so that the host side does not limit the measured server.
    Latencies are the server's own submit-to-completion clock.  linger_us is
    the server's batching window (srv_set_linger; default CH_SERVE_LINGER_US,
    else 300: the actors of a tick answer within a fraction of a step)."""
    import random
    import threading

    groups, slots, group_default, name = SERVED[workload]
    budget = int(float(os.environ.get("CH_SERVE_BUDGET_GB", "64")) * (1 << 30))
    srv = native.srv_create(budget, slots)
    if linger_us is None:
        linger_us = int(os.environ.get("CH_SERVE_LINGER_US", "300"))
    envs = []
    try:
        native.srv_set_linger(srv, linger_us)
        for prm, count in groups:
            p = native.params(**prm)
            for _ in range(count):
                envs.append((native.srv_admit(srv, p, seed=len(envs), amplitude=0.1, kmax=99), prm))
        stop = threading.Event()
        measuring = threading.Event()
        errors = []
        lat = {}   # class label -> submit-to-result latencies (s) seen by the actors while measuring
        group = max(1, int(os.environ.get("CH_SERVE_GROUP", str(group_default))))

        def actor(eids, prm, seed):
            rng = random.Random(seed)
            nrng = np.random.default_rng(seed)
            nx, nz = prm["nx"], prm["nz"]
            u_tau = prm["re_tau"] / prm["re_bulk"]
            obs = np.zeros((len(eids), 2, nz, nx))
            acts = nrng.standard_normal((16, nz, nx)) * 0.05 * u_tau
            acts -= acts.mean(axis=(1, 2), keepdims=True)
            ids = np.asarray(eids, dtype=np.int32)
            mine = lat.setdefault(f"{nx}x{prm['ny']}x{nz}", [])
            i = 0
            try:
                while not stop.is_set():
                    t0 = time.perf_counter()
                    a = acts[(i + np.arange(len(eids))) % 16] if prm["control"] == 0 else None
                    rids = native.srv_submit_many(srv, ids, a)
                    rc, _, _, st = native.srv_wait_many(srv, rids, 120000, obs)
                    if rc != native.CH_OK or (st != native.CH_OK).any():
                        errors.append(rc if rc != native.CH_OK else int(st[st != native.CH_OK][0]))
                        return
                    if measuring.is_set():
                        mine.extend([time.perf_counter() - t0] * len(eids))
                    i += 1
                    if rate > 0:
                        time.sleep(rng.expovariate(rate))
            except Exception as exc:  # noqa: BLE001
                errors.append(repr(exc))

        for _, prm in envs:
            lat.setdefault(f"{prm['nx']}x{prm['ny']}x{prm['nz']}", [])
        work = []   # actors: consecutive environments of one class, `group` at a time
        k = 0
        while k < len(envs):
            prm = envs[k][1]
            j = k
            while j < len(envs) and j - k < group and envs[j][1] is prm:
                j += 1
            work.append(([e for e, _ in envs[k:j]], prm))
            k = j
        threads = [threading.Thread(target=actor, args=(eids, prm, n)) for n, (eids, prm) in enumerate(work)]
        for t in threads:
            t.start()
        time.sleep(warm)
        native.srv_stats(srv, reset=True)
        measuring.set()
        time.sleep(duration)
        st = native.srv_stats(srv)
        measuring.clear()
        stop.set()
        for t in threads:
            t.join()
    finally:
        native.srv_destroy(srv)
    pts = sum(count * prm["nx"] * prm["ny"] * prm["nz"] for prm, count in groups) / len(envs)
    per_class = {}
    for label, xs in lat.items():
        if xs:
            a = np.sort(np.asarray(xs)) * 1e3
            per_class[label] = {"steps_per_s": len(a) / duration, "p50_ms": float(np.percentile(a, 50)),
                                "p99_ms": float(np.percentile(a, 99))}
    return {"value": st.env_steps_per_s, "unit": UNIT, "completed": int(st.completed),
            "p50_ms": st.p50_us / 1e3, "p99_ms": st.p99_us / 1e3, "mean_ms": st.mean_us / 1e3,
            "think_rate_per_s": rate, "linger_us": linger_us, "seconds": duration, "envs": len(envs),
            "classes": st.classes,
            "slots_per_class": slots, "envs_per_actor_thread": group, "actor_threads": len(work),
            "hbm_used_gb": st.hbm_used / (1 << 30), "mpts_rk3_steps_per_s": st.env_steps_per_s * pts / 1e6,
            "per_class_actor_side": per_class, "errors": errors[:5], "workload": name}


def run_served(args):
    """One served workload as its own line."""
    import torch
    from paper_2301_09889_gb300 import native
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    native.load()
    rate = float(os.environ.get("CH_SERVE_RATE", "0"))
    duration = float(os.environ.get("CH_SERVE_SECONDS", "10"))
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    r = served_run(native, args.workload, rate, duration)
    clk = clocks.stop()
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": r["completed"], "warmup": 3,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": r["workload"], "envs": r["envs"], "slots_per_class": r["slots_per_class"],
                   "classes": r["classes"], "think_rate_per_s": rate, "linger_us": r["linger_us"],
                   "envs_per_actor_thread": r["envs_per_actor_thread"],
                   "actor_threads": r["actor_threads"], "seconds": duration, "hbm_used_gb": r["hbm_used_gb"]},
        "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "mean_ms": r["mean_ms"],
        "mpts_rk3_steps_per_s": r["mpts_rk3_steps_per_s"], "per_class_actor_side": r["per_class_actor_side"],
        "e2e": {"value": r["value"], "unit": UNIT, "note": "served requests: host actions in, host observations out"},
        "errors": r["errors"], "clocks": clk,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the lines of our arm
# ---------------------------------------------------------------------------

def _cpu_leg(h, args) -> tuple[dict | None, dict | None]:
    """cpu_baseline leg: the oracle replays a 10-step window of slot 0 of the
    handle (timed, compared), then keeps stepping until its budget is spent;
    plus a single-threaded oracle sample."""
    if args.no_cpu_baseline:
        return None, None
    before, acts, outs, after = h.window(10)
    budget = float(os.environ.get("CH_CPU_BASELINE_S", "20"))
    times, ora_outs, ora_final = oracle_window(h.prm, before, acts, budget)
    err = window_errors(outs, after, ora_outs, ora_final, h.u_tau)
    cpu = {"value": len(times) / sum(times), "unit": UNIT, "cores": os.cpu_count(), "cpu": cpu_model(),
           "kind": "oracle",
           "sample": f"{len(times)} whole environment steps of one environment of the workload (slot 0 of the "
                     f"timed handle: a 10-step window replayed with its actions, then zero actions; "
                     f"about {budget:.0f} s of CPU work)",
           "single_thread": oracle_single_thread(float(os.environ.get("CH_CPU_BASELINE_1T_S", "10")), h.name)}
    acc = {"vs": "FP64 CPU oracle", "window_steps": 10, "slot": 0, "errors": err,
           "note": "relative L2 of the state (v, omega_y, U; W against ||U||) after the window; max over the "
                   "window of the observation, wall shear and reward errors"}
    return cpu, acc


def run_target(args, rank: int, world: int, native, dist, flush):
    """Default line: batched mixed 256 minimal channels vs the plain FP64
    single-environment minimal channel, the served form, the oracle check and
    the larger FP64 channel."""
    fp64 = measure_fp64_peak()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    batched = measure_handle(native, TARGET_BATCHED, args, rank, world, flush, dist, fp64_peak=fp64)
    plain = measure_handle(native, TARGET_PLAIN, args, rank, world, flush, dist, e2e=False, fp64_peak=fp64)
    larger = measure_handle(native, "larger_fp64", args, rank, world, flush, dist, e2e=False, fp64_peak=fp64)
    clk = clocks.stop()
    hb = batched.pop("_handle")
    for r in (plain, larger):
        r.pop("_handle").close()
    served = None
    if rank == 0 and world == 1 and not args.no_served:
        secs = float(os.environ.get("CH_SERVE_SECONDS", "4"))
        served = {"saturation": served_run(native, TARGET_SERVED, 0.0, secs),
                  "exponential_think_200_per_s": served_run(native, TARGET_SERVED, 200.0, secs)}
    cpu, acc = (None, None)
    if rank == 0 and world == 1:
        cpu, acc = _cpu_leg(hb, args)
    hb.close()
    if rank != 0:
        return
    pick = lambda r, keys: {k: r[k] for k in keys if k in r}
    line = {
        "metric": METRIC, "value": batched["value"], "unit": UNIT, "n_gpus": world, "steps": batched["steps"],
        "warmup": batched["warmup"], "ms_per_step": batched["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": config_of(DEFAULT_WORKLOAD, world),
        "p50_ms": batched["p50_ms"], "p99_ms": batched["p99_ms"],
        "latency_note": "p50/p99 of the device time of one batched step (256 environment steps); the served "
                        "form's submit-to-result percentiles are under served",
        "mpts_rk3_steps_per_s": batched["mpts_rk3_steps_per_s"],
        "comparison": {
            "plain_fp64_single_env": {"workload": WORKLOADS[TARGET_PLAIN][3],
                                      **pick(plain, ("value", "ms_per_step", "p50_ms", "p99_ms",
                                                     "kernels_ms_per_step", "gpu_launches", "finite"))},
            "speedup_env_steps_per_s": batched["value"] / plain["value"],
            "same_gpu_same_run": True},
        "served": served,
        "accuracy": acc,
        "kernels_ms_per_step": batched["kernels_ms_per_step"],
        "profiled_ms_per_step": batched["profiled_ms_per_step"],
        "algorithmic_gbs_per_step": batched["algorithmic_gbs_per_step"],
        "roofline": batched["roofline"],
        "fp64_peak_measured": fp64,
        "cpu_baseline": cpu,
        "e2e": batched["e2e"],
        "gpu_launches": batched["gpu_launches"],
        "tiles": batched["tiles"],
        "larger_fp64": {"workload": WORKLOADS["larger_fp64"][3],
                        **pick(larger, ("value", "ms_per_step", "p50_ms", "p99_ms", "kernels_ms_per_step",
                                        "roofline", "tiles", "finite"))},
        "step_launch": "value, comparison and larger_fp64: one captured CUDA graph per step; kernel times and "
                       "roofline: a second, profiled pass of the same steps launching the kernels one by one "
                       "between per-class CUDA events",
        "clocks": clk,
        "finite": batched["finite"],
    }
    print(json.dumps(line), flush=True)


def run_single(args, rank: int, world: int, native, dist, flush):
    """One single-handle workload as its own line."""
    fp64 = measure_fp64_peak()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    r = measure_handle(native, args.workload, args, rank, world, flush, dist, fp64_peak=fp64)
    clk = clocks.stop()
    h = r.pop("_handle")
    cpu = None
    if rank == 0 and world == 1:
        if h.external:
            cpu, acc = _cpu_leg(h, args)
        else:
            acc = None
            if not args.no_cpu_baseline:
                times = oracle_sample(float(os.environ.get("CH_CPU_BASELINE_S", "20")), 1000, args.workload)
                cpu = {"value": len(times) / sum(times), "unit": UNIT, "cores": os.cpu_count(), "cpu": cpu_model(),
                       "kind": "oracle",
                       "sample": f"{len(times)} whole environment steps of one environment of the workload "
                                 "(about 20 s of CPU work)",
                       "single_thread": oracle_single_thread(float(os.environ.get("CH_CPU_BASELINE_1T_S", "10")),
                                                             args.workload)}
        r["accuracy"] = acc
    h.close()
    if rank != 0:
        return
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": r["steps"],
            "warmup": r["warmup"], "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if h.prec == 0 else "f32+f64", "data": "synthetic",
            "config": config_of(args.workload, world), "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"],
            "mpts_rk3_steps_per_s": r["mpts_rk3_steps_per_s"], "kernels_ms_per_step": r["kernels_ms_per_step"],
            "profiled_ms_per_step": r["profiled_ms_per_step"],
            "algorithmic_gbs_per_step": r["algorithmic_gbs_per_step"], "roofline": r["roofline"],
            "fp64_peak_measured": fp64,
            "cpu_baseline": cpu, "accuracy": r.get("accuracy"), "e2e": r["e2e"], "gpu_launches": r["gpu_launches"],
            "tiles": r["tiles"],
            "step_launch": "value: one captured CUDA graph per step; kernel times and roofline: a profiled pass "
                           "launching the kernels one by one between per-class CUDA events",
            "clocks": clk, "finite": r["finite"]}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=(DEFAULT_WORKLOAD,) + tuple(WORKLOADS) + tuple(SERVED))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-served", action="store_true", help="skip the served runs of the default line")
    ap.add_argument("--no-autotune", action="store_true",
                    help="tile shapes from the size rule instead of timing at env_create "
                         "(for profiler runs, whose timings would mislead the autotuner)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload in SERVED:
        if rank == 0:
            run_served(args)
        return

    import torch

    from paper_2301_09889_gb300 import native

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    native.load()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    if args.workload == DEFAULT_WORKLOAD:
        run_target(args, rank, world, native, dist, flush)
    else:
        run_single(args, rank, world, native, dist, flush)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
