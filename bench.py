"""Benchmark: phi_l(-tau*A)v, l = 0..3, on the 3D convection-diffusion workload
(A = A^x (+) A^y (+) A^z, A^d = -0.01*D2 + 1.0*D1_upwind on n = 128 points per dimension,
2,097,152 unknowns, tau = 1e-2, v ~ U(-1,1) seed 0).

One step = one phikron_apply (Algorithm 1 on 2^{-s}M plus s modified-squaring steps and
phi_0) of a plan built once (the plan -- Algorithm 5, nodes, 1D exponentials -- is reused
across steps as an exponential integrator reuses it across time steps; its time is
reported separately as plan_ms).  Inputs are resident in HBM; L2 is flushed (a 512 MiB
write) before every timed step.  value = unknowns processed per second over all ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed|mixed8|mixed6]
                    [--impl ours|reference] [--no-cpu-baseline]

--impl reference times the oracle's CPU restatement of the same algorithm (numpy/scipy
float64 on the host cores) on the same workload; it runs on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "phi_l(tau A)v unknowns/s at rel err<=1e-8 vs FP64 oracle; mixed vs FP64 GPU"
UNIT = "unknowns/s"
GOLDEN = os.path.join(ROOT, "tests", "golden", "convdiff3d_n128_tau1e-2_seed0_samples.txt")
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FLUSH_BYTES = 512 << 20
CLOCK_PREROLL_S = 1.5

# (precision id, quadrature tolerance, digit slices; 0 = from the tolerance).  "mixed" is the
# fastest setting that meets the metric's 1e-8 gate with margin: tolerance 1e-9 (a-priori
# quadrature bound ten times below the gate) and 4 digit slices (measured ~2e-9 on this
# workload); "mixed10" keeps 1e-10 with 5 slices (~1e-11).
PRECISIONS = {"fp64": (0, 1e-10, 0), "mixed": (2, 1e-9, 4), "mixed10": (2, 1e-10, 5), "mixed6": (2, 1e-6, 0)}


def workload(n=128):
    return W.convdiff3d(n=n, tau=1e-2, l_max=3, tol=1e-10, seed=0)


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts once the sampler is producing (nvidia-smi takes ~0.1-1 s
            # to start); samples taken before the region are dropped in stop()
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.005)
            self.skip = len(self.lines)
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def mark_timed(self):
        """The timed region starts: samples from here on fall inside it until mark_end()."""
        self.timed_from = len(self.lines)

    def mark_end(self):
        self.timed_to = len(self.lines)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[getattr(self, "skip", 0):]:
            f = [t.strip() for t in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        timed = max(0, getattr(self, "timed_to", len(self.lines)) - getattr(self, "timed_from", len(self.lines)))
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "samples_in_timed_region": timed, "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- helpers

def load_golden():
    if not os.path.exists(GOLDEN):
        return None
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    from make_convdiff_samples import load
    return load(GOLDEN)


def sampled_rel_err(out: np.ndarray, golden) -> list:
    idx, vals, norm2, _ = golden
    errs = []
    for l in range(vals.shape[0]):
        d = out[l][idx] - vals[l]
        # sampled relative error, normalised like the full 2-norm error: rms(diff)/rms(phi_l)
        errs.append(float(np.sqrt(np.mean(d * d)) / (norm2[l] / math.sqrt(out.shape[1]))))
    return errs


def peaks():
    try:
        with open(PEAKS) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# DRAM traffic of the tensor-core mode kernel from the ncu capture summarised in
# profiles/mode_kernel_ws_convdiff3d_n128_ncu_full.md (one launch of the z-mode node pass:
# 11 vectors x N unknowns); valid only while the kernel code is the one captured (hash of
# tc_mode.cu without comments and blank lines, see code_hash).
PROFILED_MODE_TRAFFIC = {"source_sha256_16": "29768ebe00cf63a1", "bytes": 186.086144e6 + 126.577664e6,
                         "vector_passes": 11, "N": 2097152}


def code_hash(path: str) -> str:
    """First 16 hex digits of the sha256 of a C++/CUDA source without its // comments (a
    trailing comment is dropped when no string literal precedes it) and blank lines."""
    import hashlib
    kept = []
    with open(path, encoding="utf-8") as f:
        for ln in f:
            code = ln.rstrip("\n")
            if "//" in code:
                head = code.split("//", 1)[0]
                if '"' not in head:
                    code = head
            if code.strip():
                kept.append(code.rstrip())
    return hashlib.sha256("\n".join(kept).encode()).hexdigest()[:16]


def mode_traffic_per_launch(N, vector_passes_per_launch):
    """dram read + write bytes per average mode launch, scaled from the capture by the number
    of (vector, mode) products a launch processes; None if the kernel changed since."""
    h = code_hash(os.path.join(ROOT, "paper_2211_00696_gb300", "csrc", "tc_mode.cu"))
    ref = PROFILED_MODE_TRAFFIC
    if h != ref["source_sha256_16"] or N != ref["N"]:
        return None
    return ref["bytes"] * vector_passes_per_launch / ref["vector_passes"]


def roofline(info, prof, ms_per_step_profiled, precision):
    """Roofline of the dominant kernel class from CUDA-event timings taken in bench.py."""
    pk, src = peaks()
    cls = max(prof["ms"], key=lambda k: prof["ms"][k])
    launches = max(prof["launches"][cls], 1)
    avg_ms = prof["ms"][cls] / launches
    N, n = info["N"], info["n"]
    actions = info["actions"]
    flops_per_step = actions * 2.0 * N * sum(n[: info["dims"]])
    if cls == "gemm_f64":
        # float64 DFMA pipe: 152 SMs x 2 DFMA/clk (4 flop/clk/SM) x 2.07 GHz = 1.259 TFLOP/s
        peak = 152 * 4 * 2.070e9 / 1e12
        achieved = flops_per_step / (prof["ms"][cls] / prof["steps"] * 1e-3) / 1e12
        return {"bound": "alu", "kernel": "gemm_f64_kernel (DFMA mode products)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": "nominal FP64 rate (152 SMs x 4 flop/clk x 2070 MHz)",
                "avg_launch_ms": avg_ms, "launches_per_step": launches / prof["steps"],
                "traffic": None}
    if cls == "tc_mode":
        # two ceilings: HBM (read + write one 8-byte state per unknown per pass) and the
        # BF16 tensor pipe (slices*(slices+1)/2 slice products per mode product)
        t = prof["ms"][cls] / prof["steps"] * 1e-3
        hbm = pk.get("hbm_gbs", 6800.0)
        gbs = prof["algorithmic_bytes"] / t / 1e9
        tfl = prof["bf16_flops"] / t / 1e12
        tpk = pk.get("bf16_tflops", 1900.0)
        lps = launches / prof["steps"]
        traffic = mode_traffic_per_launch(N, info["actions"] * info["dims"] / lps)
        if gbs / hbm >= tfl / tpk:
            return {"bound": "hbm", "kernel": "tc mode-product kernels (tcgen05 BF16 digit slices)",
                    "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                    "peak_source": f"{src} hbm_gbs", "tensor_frac": tfl / tpk,
                    "avg_launch_ms": avg_ms, "launches_per_step": lps, "traffic": traffic,
                    "algorithmic_bytes_per_launch": prof["algorithmic_bytes"] / lps}
        return {"bound": "tensor", "kernel": "tc mode-product kernels (tcgen05 BF16 digit slices)",
                "achieved": tfl, "peak": tpk, "unit": "TFLOP/s", "frac": tfl / tpk,
                "peak_source": f"{src} bf16_tflops", "hbm_frac": gbs / hbm,
                "avg_launch_ms": avg_ms, "launches_per_step": lps, "traffic": traffic}
    return {"bound": "hbm", "kernel": cls, "achieved": None, "peak": pk.get("hbm_gbs"),
            "unit": "GB/s", "frac": None, "traffic": None}


# ----------------------------------------------------------------------------- arms

def cpu_reference_step(prob, v, s, m, tol):
    from oracle import quadrature as Q
    return Q.alg6_phiquadmv(prob.factors, prob.tau, v, prob.l_max, tol, s=s, m=m)


REF_BUDGET_S = 60.0   # timed oracle work of one --impl reference run


def max_over_ranks(values, device):
    """Elementwise maximum of per-rank float values over the process group (identity for one
    process); device: where the reduction tensor lives (CUDA for NCCL, CPU for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(x) for x in values]
    t = torch.tensor([float(x) for x in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def replica_throughput(world: int, unknowns_per_step: int, steps: int, max_seconds: float) -> float:
    """Whole-job unknowns/s of `world` independent replicas: all replicas' work over the slowest
    replica's time (weak scaling; the driver computes efficiency from these values)."""
    return world * unknowns_per_step * steps / max_seconds


def oracle_step_seconds(tol: float) -> float:
    """One oracle step of the default workload at `tol`, timed (called in a child process that
    was started with one BLAS / OpenMP thread)."""
    prob = workload()
    v = prob.vector()
    from oracle import planner as PL
    s, m, _ = PL.setup_quadrature(tol, prob.l_max, PL.alpha_inf(prob.factors, prob.tau))
    t0 = time.perf_counter()
    cpu_reference_step(prob, v, s, m, tol)
    return time.perf_counter() - t0


def oracle_single_thread(tol: float):
    """unknowns/s of the oracle on one host core (a fresh interpreter with the thread counts
    of BLAS and OpenMP set to 1 before numpy loads), or None if the child fails."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", f"import bench; print(bench.oracle_step_seconds({tol!r}))"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        dt = float(r.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError, OSError):
        return None
    return workload().N / dt


def host_cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (subprocess.SubprocessError, OSError):
        pass
    return "unknown"


def run_reference(args):
    """The oracle's CPU restatement of Algorithms 1 and 6 (numpy/scipy float64), rank 0."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    prob = workload()
    v = prob.vector()
    # the GPU arm's tolerance (and so its (s, m)) for the same precision flags
    tol = args.tol if args.tol > 0 else PRECISIONS[args.precision][1]
    from oracle import planner as PL
    s, m, _ = PL.setup_quadrature(tol, prob.l_max, PL.alpha_inf(prob.factors, prob.tau))
    # A step is one full oracle apply (~1-3 s on the host cores).  The run is bounded to about
    # REF_BUDGET_S of timed work: the first warm-up step measures a step, the remaining warm-up
    # steps are capped at 2, and at most REF_BUDGET_S / (step time) of the K steps are timed.
    tw = time.perf_counter()
    cpu_reference_step(prob, v, s, m, tol)
    t_one = time.perf_counter() - tw
    for _ in range(min(args.warmup, 3) - 1):
        cpu_reference_step(prob, v, s, m, tol)
    k_eff = max(1, min(args.steps, int(REF_BUDGET_S / max(t_one, 1e-3))))
    t0 = time.perf_counter()
    for _ in range(k_eff):
        cpu_reference_step(prob, v, s, m, tol)
    dt = (time.perf_counter() - t0) / k_eff
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    val = prob.N / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "steps_timed": k_eff, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": prob.name, "N": prob.N, "l_max": 3,
                                            "tau": 1e-2, "tol": tol, "s": s, "m": m},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"full workload per step (oracle.quadrature.alg6_phiquadmv: scipy "
                                       f"expm + numpy tensordot mode products, float64); {k_eff} of the "
                                       f"{args.steps} steps timed (~{REF_BUDGET_S:.0f} s budget)"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(args):
    """Uneven batched workload: 32 3D diffusion instances with sizes from {64,...,256},
    4 right-hand sides, phi_0..phi_3 at tau and tau/2, 3 digit slices; one grouped graph per
    apply.  value = unknowns (instances x RHS x N_i) per second."""
    import torch
    import paper_2211_00696_gb300 as pk
    torch.cuda.set_device(0)
    insts = W.batched_uneven3d()
    t0 = time.perf_counter()
    plans = [pk.Plan(W.batched_instance_factors(d), d["tau"], 3, 1e-6, precision=pk.PREC_OZAKI_BF16,
                     slices=3, half_step=True) for d in insts]
    batch = pk.Batch(plans, nrhs=4, half_step=True, autotune=True)
    plan_ms = (time.perf_counter() - t0) * 1e3
    V = [torch.stack([torch.from_numpy(W.uniform_vector(d["shape"], s)) for s in d["rhs_seeds"]]).cuda()
         for d in insts]
    out = batch.apply(V)            # autotunes on this first call
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        batch.apply(V, out)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        batch.apply(V, out)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    unknowns = 4 * sum(int(np.prod(d["shape"])) for d in insts)
    info = batch.info()
    # per-kernel CUDA-event times of further applies (separate pass, same stream, no graph)
    batch.profile_begin(8192)
    for _ in range(2):
        batch.apply(V, out)
    torch.cuda.synchronize()
    prof = batch.profile_end()
    # algorithmic work of the tensor-core mode passes: every (vector, mode) product reads and
    # writes one 8-byte state per unknown and does slices (slices + 1) / 2 BF16 slice products
    # of 2 N n_d flops; per unit, m + s p + 1 actions plus phi_0 at tau/2
    hbm, fl = 0.0, 0.0
    for d, p_ in zip(insts, plans):
        pi = p_.info()
        Ni = int(np.prod(d["shape"]))
        acts = pi["actions"] + 1
        hbm += 4 * acts * 3 * 16.0 * Ni
        fl += 4 * acts * 2.0 * Ni * sum(d["shape"]) * (3 * 4 // 2)
    pk_, src = peaks()
    t = prof["ms"]["tc_mode"] / 2 * 1e-3
    gbs, tfl = hbm / t / 1e9, fl / t / 1e12
    roof = {"bound": "hbm", "kernel": "tc mode-product kernels (tcgen05 BF16 digit slices)", "achieved": gbs,
            "peak": pk_.get("hbm_gbs", 6800.0), "unit": "GB/s", "frac": gbs / pk_.get("hbm_gbs", 6800.0),
            "peak_source": f"{src} hbm_gbs", "tensor_frac": tfl / pk_.get("bf16_tflops", 1900.0),
            "mode_ms_per_step": t * 1e3, "kernel_ms_per_step": {k: v_ / 2 for k, v_ in prof["ms"].items() if v_ > 0},
            "traffic": None}
    print(json.dumps({"metric": "batched phi_0..3 at tau and tau/2, unknowns/s", "value": unknowns / (ms * 1e-3),
                      "unit": UNIT, "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
                      "unknowns_per_step": unknowns, "plan_and_batch_ms": plan_ms, "roofline": roof,
                      "config": {"workload": "batched_uneven3d_32x4rhs", "slices": 3,
                                 "s": [p.info()["s"] for p in plans], "m": [p.info()["m"] for p in plans]},
                      "batch": info}), flush=True)


def run_allen_cahn(args):
    """Semilinear 2D Allen-Cahn u' = eps^2 Lap(u) + u - u^3 on the 2048^2 periodic grid
    (eps = 0.01, tau = 1e-2, u0 ~ U(-0.05, 0.05) seed 4): exponential Euler and the two-stage
    method (c2 = 1/2) through the library's integrator, mixed (tol 1e-10) and float64 (tol
    1e-12), --steps time steps each (default 200); value = unknowns x time steps per second of
    the mixed run; the final-state difference mixed vs float64 is the accuracy gate (<= 1e-6)."""
    import torch
    import paper_2211_00696_gb300 as pk
    torch.cuda.set_device(0)
    a, u0 = W.allen_cahn2d()
    fac = [a, a]
    N = u0.size
    nsteps = args.steps
    st = torch.cuda.current_stream()
    res = {}
    for method, mid in (("euler", pk.ERK_EULER), ("rk2", pk.ERK_RK2)):
        finals = {}
        for prec, pid, tol in (("mixed", pk.PREC_OZAKI_BF16, 1e-10), ("fp64", pk.PREC_FP64, 1e-12)):
            it = pk.Integrator(fac, 1e-2, mid, tol, precision=pid)
            U = torch.from_numpy(u0.copy()).cuda()
            it.step(U, 1)                   # warm-up (graph instantiation, first launches)
            U.copy_(torch.from_numpy(u0))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            it.step(U, nsteps)
            e1.record(st)
            torch.cuda.synchronize()
            it.check_status()
            ms = e0.elapsed_time(e1)
            info = it.info()
            finals[prec] = U.cpu().numpy()
            # per-kernel CUDA-event times of a few more steps (separate pass, same stream)
            prof_steps = 5
            it.profile_begin(4096)
            it.step(U, prof_steps)
            torch.cuda.synchronize()
            prof = it.profile_end()
            slices = 0 if prec == "fp64" else it_slices(fac, pid, tol)
            it.close()
            res[f"{method}_{prec}"] = {"ms_total": ms, "ms_per_step": ms / nsteps,
                                       "unknown_steps_per_s": N * nsteps / (ms * 1e-3),
                                       "plans": {"c": info["c"][:info["nplans"]], "s": info["s"][:info["nplans"]],
                                                 "m": info["m"][:info["nplans"]],
                                                 "actions": info["actions"][:info["nplans"]]},
                                       "kernel_ms_per_step": {k: v_ / prof_steps for k, v_ in prof["ms"].items() if v_ > 0},
                                       "roofline": integrator_roofline(info, prof, prof_steps, N, fac[0].shape[0],
                                                                       len(fac), slices)}
        d = np.linalg.norm(finals["mixed"] - finals["fp64"]) / np.linalg.norm(finals["fp64"])
        res[f"{method}_final_rel_diff_mixed_vs_fp64"] = float(d)
    line = {"metric": "Allen-Cahn 2048^2 exponential integrators, unknowns x steps / s (mixed)",
            "value": res["euler_mixed"]["unknown_steps_per_s"], "unit": "unknown-steps/s", "steps": nsteps,
            "roofline": res["euler_mixed"]["roofline"],
            "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "allen_cahn2d_2048_periodic_eps0.01_tau1e-2", "N": N, "time_steps": nsteps},
            "results": res,
            "gate_final_rel_diff_le_1e-6": all(res[f"{m}_final_rel_diff_mixed_vs_fp64"] <= 1e-6 for m in ("euler", "rk2"))}
    print(json.dumps(line), flush=True)


def it_slices(fac, pid, tol):
    """Digit slices of the integrator's mixed plans (same rule as phikron_plan's default)."""
    import paper_2211_00696_gb300 as pk
    plan = pk.Plan(fac, 1e-2, 1, tol, precision=pid)
    k = plan.info()["slices"]
    plan.close()
    return k


def integrator_roofline(info, prof, steps, N, n, dims, slices):
    """Roofline of the mode-product kernels of an integrator run.  Every plan is applied once per
    step (exponential Euler: one plan; the two-stage method: c2 and 1); a plan's apply runs
    `actions` Kronecker actions of dims mode products of 2 N n flops each.  Mixed path: BF16
    tensor work = slices (slices + 1) / 2 slice-pair products per mode product, against the
    sustained BF16 peak (the kernels run inside a long step); float64 path: DFMA work against the
    nominal FP64 rate."""
    pk_, src = peaks()
    actions = sum(info["actions"][:info["nplans"]])
    flops = actions * dims * 2.0 * N * n          # per step, the method's own flops
    hbm_bytes = actions * dims * 16.0 * N         # one 8-byte state read and written per mode product
    if slices:
        t = prof["ms"]["tc_mode"] / steps * 1e-3
        if t <= 0:
            return None
        tfl = flops * (slices * (slices + 1) // 2) / t / 1e12
        peak = pk_.get("bf16_tflops_sustained", 1700.0)
        return {"bound": "tensor", "kernel": "tc mode-product kernels (tcgen05 BF16 digit slices)",
                "achieved": tfl, "peak": peak, "unit": "TFLOP/s", "frac": tfl / peak,
                "peak_source": f"{src} bf16_tflops_sustained", "hbm_frac": hbm_bytes / t / 1e9 / pk_.get("hbm_gbs", 6800.0),
                "slice_pair_flops_per_step": flops * (slices * (slices + 1) // 2),
                "mode_ms_per_step": t * 1e3, "traffic": None}
    t = prof["ms"]["gemm_f64"] / steps * 1e-3
    if t <= 0:
        return None
    peak = 152 * 4 * 2.070e9 / 1e12
    ach = flops / t / 1e12
    return {"bound": "alu", "kernel": "gemm_f64_kernel (DFMA mode products)", "achieved": ach, "peak": peak,
            "unit": "TFLOP/s", "frac": ach / peak, "peak_source": "nominal FP64 rate (152 SMs x 4 flop/clk x 2070 MHz)",
            "mode_ms_per_step": t * 1e3, "traffic": None}


def fp64_gpu_compare(prob, V, out_shape, flush, golden, dev, local, tol, steps=3):
    """The same workload on the float64 GPU path (float64 DFMA mode products) at the mixed arm's
    quadrature tolerance (the same (s, m)), timed the same way: the comparison the metric names
    (mixed vs FP64 GPU at the stated accuracy)."""
    import torch

    import paper_2211_00696_gb300 as pk
    plan = pk.Plan(prob.factors, prob.tau, prob.l_max, tol, precision=pk.PREC_FP64, device=local)
    Out = torch.empty(out_shape, dtype=torch.float64, device=dev)
    plan.apply(V, Out)
    torch.cuda.synchronize()
    errs = sampled_rel_err(Out.cpu().numpy(), golden) if golden is not None else None
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot = 0.0
    for _ in range(steps):
        flush.zero_()
        e0.record(stream)
        plan.apply(V, Out)
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    info = plan.info()
    plan.close()
    ms = tot / steps
    return {"value": prob.N / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps, "tol": tol,
            "s": info["s"], "m": info["m"], "actions": info["actions"], "rel_err_sampled": errs}


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2211_00696_gb300 as pk

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    prec_id, tol, prec_slices = PRECISIONS[args.precision]
    if args.slices == 0:
        args.slices = prec_slices
    if args.tol > 0:
        tol = args.tol
    prob = workload()
    v = prob.vector()
    t0 = time.perf_counter()
    quad = {"gauss": pk.QUAD_GAUSS, "cc": pk.QUAD_CC, "cc_adaptive": pk.QUAD_CC_ADAPTIVE}[args.quad]
    plan = pk.Plan(prob.factors, prob.tau, prob.l_max, tol, precision=prec_id, device=local, quad=quad,
                   slices=args.slices)
    torch.cuda.synchronize()
    plan_ms = (time.perf_counter() - t0) * 1e3
    info = plan.info()

    V = torch.from_numpy(v).to(dev)
    Out = torch.empty((prob.l_max + 1, prob.N), dtype=torch.float64, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # accuracy on this run's output (sampled against stored oracle values)
    plan.apply(V, Out)
    torch.cuda.synchronize()
    info = plan.info()               # adaptive quadrature: node count of this input
    golden = load_golden()
    errs = sampled_rel_err(Out.cpu().numpy(), golden) if golden is not None else None

    for _ in range(args.warmup):
        flush.zero_()
        plan.apply(V, Out)
    torch.cuda.synchronize()

    # timed region: K steps, each bracketed by CUDA events on the launching stream
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clk = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    # The sampler's window: identical untimed steps for at least CLOCK_PREROLL_S right before the
    # timed region (the region itself can be a few ms, shorter than one sampling interval), so
    # that the clocks recorded are those of the GPU under this load when the timed steps start.
    pre0 = time.perf_counter()
    preroll = 0
    while time.perf_counter() - pre0 < CLOCK_PREROLL_S:
        for _ in range(16):
            flush.zero_()
            plan.apply(V, Out)
        torch.cuda.synchronize()
        preroll += 16
    clk.mark_timed()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    plan.profile_begin(0)            # launch counting only
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        plan.apply(V, Out)
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk.mark_end()
    counted = plan.profile_end()
    clocks = clk.stop()
    clocks["window"] = (f"{preroll} identical untimed steps ({CLOCK_PREROLL_S:.1f} s) immediately before "
                        f"the timed region, and the timed region")
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    tot = float(np.sum(step_ms)) * 1e-3
    if world > 1:
        tot = max_over_ranks([tot], dev)[0]
        dist.barrier()
    ms_per_step = tot / args.steps * 1e3
    value = replica_throughput(world, prob.N, args.steps, tot)
    gpu_launches = int(sum(counted["launches"].values()))

    # per-kernel CUDA-event timing of the same steps (separate pass, same stream)
    plan.profile_begin(4096)
    for i in range(args.steps):
        flush.zero_()
        plan.apply(V, Out)
    torch.cuda.synchronize()
    prof = plan.profile_end()
    prof["steps"] = args.steps
    # algorithmic bytes of the tensor-core mode passes: each pass reads and writes one
    # 8-byte state per unknown for every vector it processes
    prof["algorithmic_bytes"] = info["actions"] * info["dims"] * 16.0 * prob.N
    prof["bf16_flops"] = (info["actions"] * 2.0 * prob.N * sum(info["n"][: info["dims"]])
                          * (info["slices"] * (info["slices"] + 1) // 2))

    # end to end through the public API with host buffers (pinned), copies inside the region:
    # (a) one synchronous phikron_apply_host call per step; (b) phikron_apply_host_many over
    # e2e_steps vectors (each step copies its own input in and its results out; the transfers
    # of neighbouring steps overlap the apply)
    e2e_steps = max(3, min(args.steps, 10))
    vh = torch.from_numpy(np.ascontiguousarray(np.broadcast_to(v, (e2e_steps, prob.N)))).pin_memory()
    oh = torch.empty((e2e_steps, prob.l_max + 1, prob.N), dtype=torch.float64).pin_memory()
    plan.apply_host_ptr(vh.data_ptr(), oh.data_ptr())
    te = time.perf_counter()
    for _ in range(e2e_steps):
        plan.apply_host_ptr(vh.data_ptr(), oh.data_ptr())
    e2e_single_s = (time.perf_counter() - te) / e2e_steps
    plan.apply_host_many_ptr(vh.data_ptr(), oh.data_ptr(), e2e_steps)   # first call allocates
    te = time.perf_counter()
    plan.apply_host_many_ptr(vh.data_ptr(), oh.data_ptr(), e2e_steps)
    e2e_s = (time.perf_counter() - te) / e2e_steps
    if world > 1:
        e2e_s, e2e_single_s = max_over_ranks([e2e_s, e2e_single_s], dev)

    line = None
    if rank == 0:
        dtype = "f64" if args.precision == "fp64" else f"bf16x{info['slices']} digit slices, f32 accumulate, float-float state"
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": prob.name, "N": prob.N, "l_max": prob.l_max, "tau": prob.tau,
                       "tol": tol, "precision": args.precision, "slices": info["slices"], "quad": args.quad,
                       "s": info["s"],
                       "m": info["adaptive_nodes"] if args.quad == "cc_adaptive" else info["m"],
                       "actions": info["actions"], "parallelism": f"replicas{world}",
                       "l2": "flushed (512 MiB write) before every timed step"},
            "rel_err_sampled": errs,
            "plan_ms": plan_ms,
            "wall_s_timed": wall,
            "gpu_launches": gpu_launches,
            "launches_by_class": counted["launches"],
            "kernel_ms_per_step": {k: v_ / args.steps for k, v_ in prof["ms"].items() if v_ > 0},
            "roofline": roofline(info, prof, None, args.precision),
            "clocks": clocks,
            "e2e": {"value": world * prob.N / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": prob.N * 8, "d2h_bytes_per_step": (prob.l_max + 1) * prob.N * 8,
                    "api": f"phikron_apply_host_many over {e2e_steps} vectors (pinned host buffers)",
                    "single_call_value": world * prob.N / e2e_single_s,
                    "single_call_api": "phikron_apply_host, one synchronous call per step"},
        }
        if args.fp64_compare and args.precision != "fp64":
            line["fp64_gpu"] = fp64_gpu_compare(prob, V, Out.shape, flush, golden, dev, local, tol)
        if args.cpu_baseline and world == 1:
            from oracle import planner as PL
            s, m, _ = PL.setup_quadrature(tol, prob.l_max, PL.alpha_inf(prob.factors, prob.tau))
            tc = time.perf_counter()
            cpu_reference_step(prob, v, s, m, tol)
            dt = time.perf_counter() - tc
            cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
            line["cpu_baseline"] = {"value": prob.N / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": "one full step at the GPU arm's tolerance: "
                                              "oracle.quadrature.alg6_phiquadmv (same algorithm, "
                                              "numpy/scipy float64, BLAS threads = cores)",
                                    "single_thread_value": oracle_single_thread(tol),
                                    "cpu_model": host_cpu_model()}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=list(PRECISIONS))
    ap.add_argument("--no-fp64-compare", dest="fp64_compare", action="store_false")
    ap.add_argument("--slices", type=int, default=0,
                    help="mixed path: digit slices per operand (0 = from the tolerance)")
    ap.add_argument("--tol", type=float, default=0.0, help="override the precision's tolerance")
    ap.add_argument("--quad", default="gauss", choices=["gauss", "cc", "cc_adaptive"],
                    help="quadrature of the timed plan (cc_adaptive: Algorithm 2, float64 path only)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--workload", default="convdiff3d", choices=["convdiff3d", "batched", "allen_cahn"])
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "allen_cahn":
        run_allen_cahn(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
