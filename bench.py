#!/usr/bin/env python3
"""FSI time steps per second on one GB300: the 128 x 128 Q2/P1disc lid-driven
cavity with an immersed elastic disk (7776 P1 triangles), kappa = 1e3,
nu = 0.01, dt = 1e-3, block-triangular preconditioner, 1e-8 relative residual.

One bench step = one time step of the method (assemble C_f(X^n) and the
right-hand side, solve the saddle-point system, advance).  The headline
``value`` is the mixed-precision path (FP32 operators and multigrid inside
FP64 refinement); the FP64 path is reported beside it under ``fp64``.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank runs its own replica of the workload (the
solve of one instance does not shard); ``value`` sums the ranks' steps over
the slowest rank's time.  ``--impl reference`` times the CPU oracle (sparse
direct solve per step) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

# many independent instances run on their own streams: give the device enough
# hardware queues that they are not multiplexed onto a few (set before CUDA starts)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FSI time-steps/s & HBM GB/s: mixed vs FP64 @1e-8 resid; p50/p99 latency"
L2_FLUSH_BYTES = 512 << 20


def workload():
    import fsi_inputs as fi
    return fi.cavity128_case()


def workload_config(case):
    return {"workload": "cavity128_lid_disk7776: N=128 Q2/P1disc fluid, disk R=0.2 m=36 (3997 nodes, 7776 P1 "
                        "triangles), kappa=1e3, nu=0.01, rho=1, dt=1e-3, lid 1, rtol 1e-8",
            "preconditioner": "block upper-triangular; Stokes block by %d Richardson steps of a V-cycle pair "
                              "(Chebyshev degree %d)" % (STOKES_ITS, MG_DEGREE or 2),
            "multigrid": {"fused_fine_levels": MG_FUSED == 0, "cluster": MG_CLUSTER,
                          "coarsest_cells": MG_COARSE or 16},
            "restart": {"mixed": RESTART_MIXED, "fp64": RESTART}, "inner_rtol": INNER_RTOL,
            "N": case.N, "solid_nodes": int(case.ref_xy.shape[0]), "solid_tris": int(case.tris.shape[0]),
            "dofs": None, "l2": "flushed between timed steps (512 MiB write)"}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ our GPU arm
PRECOND = 2      # block upper-triangular [[A11, A12], [0, A22]]
RESTART = 100    # FGMRES restart of the FP64 arm and the size sweep (the library default is the paper's 200)
RESTART_MIXED = 30   # restart inside each refinement cycle of the mixed arm (cheaper Gram-Schmidt, same iterations)
INNER_RTOL = 1e-4    # relative tolerance of each refinement cycle of the mixed arm
STOKES_ITS = 8   # Richardson steps on the Stokes block per preconditioner application
MAX_IT = 6000


def _step_unchecked(prob):
    prob.assemble_step()
    info = prob.solve_step(check=False)
    prob.advance()
    return info


AUTOTUNE = 0     # 0: one fixed SpMV tile shape (faster inside a step); 1: the library's autotuner
MG_FUSED = 0     # 0: fused matrix-free kernels on the finest FP32 multigrid levels; -1: per-level sparse kernels
MG_CLUSTER = 0   # 0: coarse levels in one cluster launch; -1: per-level launches; n > 0: cluster levels <= n cells
MG_DEGREE = 0    # Chebyshev degree of each multigrid smoothing (0: the library's default, 2)
MG_COARSE = 0    # coarsest multigrid grid in cells (0: the library's default, 16)
CS_DEGREE = 0    # Chebyshev steps per solid mass solve (0: the library's default)
MG_COARSE_P = 0  # coarsest pressure grid in cells (0: the library's default)


def arm_settings(precision):
    """FGMRES restart, inner tolerance and tile-shape tuning of one arm."""
    if precision == 1:
        return dict(restart=RESTART_MIXED, inner_rtol=INNER_RTOL, autotune=AUTOTUNE)
    return dict(restart=RESTART, autotune=AUTOTUNE)


def mg_settings():
    """Multigrid kernel choice and smoothing degree of the bench's arms (command-line switches)."""
    return dict(mg_fused=MG_FUSED, mg_cluster=MG_CLUSTER, mg_degree=MG_DEGREE, mg_coarse=MG_COARSE,
                cs_degree=CS_DEGREE, mg_coarse_p=MG_COARSE_P)


def time_arm(fsi, torch, case, precision, steps, warmup, stream, flush, precond=PRECOND, stokes_its=STOKES_ITS,
             max_it=MAX_IT, check=True, settings=None, first_state=None):
    """Time `steps` time steps after `warmup` untimed ones; with a list
    `first_state`, the state after the first (untimed) step is appended to it."""
    prob = fsi.problem_from_case(case, precision=precision, precond=precond, rtol=1e-8, stream=stream.cuda_stream,
                                 max_it=max_it, stokes_its=stokes_its, **(settings or arm_settings(precision)),
                                 **mg_settings())
    step = prob.step if check else (lambda: _step_unchecked(prob))
    infos = []
    for k in range(warmup):
        step()
        if k == 0 and first_state is not None:
            first_state.append(prob.get_state())
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)          # evict L2 between timed steps (outside the events)
        ev[k][0].record(stream)
        infos.append(step())
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    counts = prob.graph_kernel_counts()
    launches = 0
    for inf in infos:
        cycles = inf.refinements + 1 if precision == 1 else inf.restarts + 2
        launches += int(counts[0] + counts[1] + cycles * counts[2] + inf.iterations * counts[3] + counts[4])
    stats = {
        "ms": ms,
        "status": [i.status for i in infos],
        "iterations": [i.iterations for i in infos],
        "refinements": [i.refinements for i in infos],
        "rel_residual_max": max(i.rel_residual for i in infos),
        "launches": launches,
    }
    return prob, stats


def time_e2e(fsi, case, precision, steps, warmup, stream):
    """Through the C ABI with host buffers: set_state (H2D) + step + get_state
    (D2H), over the same time steps as the device-timed arm (after the same
    warm-up steps: the first steps of the trajectory need more iterations)."""
    prob = fsi.problem_from_case(case, precision=precision, precond=PRECOND, rtol=1e-8, stream=stream.cuda_stream,
                                 max_it=MAX_IT, stokes_its=STOKES_ITS, **arm_settings(precision), **mg_settings())
    for _ in range(warmup):
        prob.step()
    u, p, X, lam = prob.get_state()
    t = []
    for _ in range(steps):
        t0 = time.perf_counter()
        prob.set_state(u, X)
        prob.step()
        u, p, X, lam = prob.get_state()
        t.append(time.perf_counter() - t0)
    h2d = (u.size + X.size) * 8
    d2h = (u.size + p.size + X.size + lam.size) * 8
    prob.close()
    return t, h2d, d2h


def slowest_rank(dist, torch, device, seconds):
    """Each entry of `seconds` (this rank's wall times) replaced by its
    maximum over the ranks (the job's time is the slowest replica's); no
    collective without a process group."""
    if not dist:
        return list(seconds)
    t = torch.tensor(list(seconds), device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def replica_value(world: int, steps: int, slowest_s: float) -> float:
    """Whole-job throughput of `world` replicas that each ran `steps` steps,
    over the slowest replica's time (weak scaling: fixed work per rank)."""
    return world * steps / slowest_s


def run_ours(args):
    import torch
    from paper_2301_10041_gb300 import build, fsi

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    fsi.load_library()
    case = workload()

    cpu = None
    oracle_npz = ""
    if rank == 0 and not args.no_cpu_baseline:
        import tempfile
        oracle_npz = os.path.join(tempfile.mkdtemp(prefix="fsi_oracle_"), "step1.npz")
        cpu = start_cpu_baseline(args, oracle_npz)

    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall0 = time.perf_counter()
    first_m, first_d = [], []
    prob_m, mixed = time_arm(fsi, torch, case, 1, args.steps, args.warmup, stream, flush, stokes_its=STOKES_ITS,
                             first_state=first_m)
    t_wall1 = time.perf_counter()
    clk = clocks.stop()
    prob_d, fp64 = time_arm(fsi, torch, case, 0, args.steps, args.warmup, stream, flush, stokes_its=STOKES_ITS,
                            first_state=first_d)
    roof = roofline(prob_m, args)
    if not args.no_large_n:
        roof["large_n"] = large_n_roofline(fsi, stream, local, roof.get("hbm_peak", roof["peak"]), args.large_n)
    e2e_t, h2d, d2h = time_e2e(fsi, case, 1, max(3, min(args.steps, 10)), args.warmup, stream)
    prob_m.close()
    prob_d.close()

    mixed_s, fp64_s, e2e_s = slowest_rank(dist, torch, "cuda",
                                          [sum(mixed["ms"]) / 1000.0, sum(fp64["ms"]) / 1000.0, sum(e2e_t)])
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    ms = mixed["ms"]
    out = {
        "metric": METRIC,
        "value": replica_value(world, args.steps, mixed_s),
        "unit": "time-steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1000.0 * mixed_s / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 operators + f64 refinement",
        "data": "synthetic (analytic disk mesh, fluid at rest, lid 1)",
        "config": workload_config(case),
        "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                       "mean": float(np.mean(ms))},
        "iterations_per_step": float(np.mean(mixed["iterations"])),
        "refinements_per_step": float(np.mean(mixed["refinements"])),
        "rel_residual_max": mixed["rel_residual_max"],
        "fp64": {"value": replica_value(world, args.steps, fp64_s), "unit": "time-steps/s",
                 "ms_per_step": 1000.0 * fp64_s / args.steps,
                 "latency_ms": {"p50": float(np.percentile(fp64["ms"], 50)),
                                "p99": float(np.percentile(fp64["ms"], 99))},
                 "iterations_per_step": float(np.mean(fp64["iterations"])),
                 "rel_residual_max": fp64["rel_residual_max"]},
        "e2e": {"value": replica_value(world, len(e2e_t), e2e_s), "unit": "time-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": mixed["launches"],
        "roofline": roof,
        "clocks": clk,
        "wall_s": t_wall1 - t_wall0,
    }
    out["config"]["dofs"] = int(prob_dofs(case))
    out["config"]["parallelism"] = f"replicas x{world}"
    if cpu is not None:
        out["cpu_baseline"] = finish_cpu_baseline(cpu)
        if os.path.exists(oracle_npz):
            out["error_vs_oracle"] = {
                "what": "relative L2 error per field of time step 1 (from the initial state) against the oracle's "
                        "direct solve of the same step; X as the displacement X - X^0",
                "mixed": field_errors(case, first_m[0], oracle_npz),
                "fp64": field_errors(case, first_d[0], oracle_npz)}
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def prob_dofs(case):
    n_u = 2 * (2 * case.N - 1) ** 2
    return n_u + 3 * case.N ** 2 + 4 * case.ref_xy.shape[0]


def fp32_peak_tflops(peaks):
    """FP32 FMA peak of the GPU: SMs x 128 FP32 lanes x 2 FLOP x the maximum
    SM clock (MEASURED_PEAKS.json sm_max_mhz, else 2070 MHz)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = peaks.get("sm_max_mhz", 2070.0)
    return sms * 128 * 2 * mhz * 1e6 / 1e12, {"sms": sms, "fp32_lanes_per_sm": 128, "sm_max_mhz": mhz}


FUSED = (("velocity_down_fused_f32", 10), ("velocity_up_fused_f32", 11), ("pressure_down_fused_f32", 12),
         ("pressure_up_fused_f32", 13))


def fused_kernels(prob, hbm_peak, alu_peak, reps):
    """Time of each fused finest-level launch (L2 evicted before each), its
    algorithmic bytes and FLOPs, and both roofline fractions."""
    out = {}
    for name, which in FUSED:
        try:
            ms, by = prob.time_kernel(which, reps=reps)
            fl = prob.kernel_flops(which)
        except Exception:
            continue
        out[name] = {"us": ms * 1e3, "bytes": by, "flops": fl, "gbs": by / ms / 1e6, "hbm_frac": by / ms / 1e6 / hbm_peak,
                     "tflops": fl / ms / 1e9, "alu_frac": fl / ms / 1e9 / alu_peak}
    return out


def roofline(prob, args):
    """Roofline of the dominant kernel of the mixed path.  On the 128 x 128
    cavity the largest share of the launch list (profiles/) is the fused
    down launch of the velocity levels (pre-smoothing, residual, restriction;
    k_mfu_down): it reads and writes vectors only, so its roofline is the
    FP32 FMA rate (algorithmic FLOPs without the overlap work of the tiles)
    and its HBM fraction is reported beside it.  Timed live on the library's
    stream with CUDA events, L2 evicted before every launch.  The other fused
    launches, the FP32 full-system operator (sparse, HBM-bound) and the
    per-level sparse smoothing step (the kernel of the FP64 arm and of
    mg_fused = -1) are reported beside it."""
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    alu_peak, alu_how = fp32_peak_tflops(peaks)
    out = {}
    for name, which in (("full_operator_f32", 0), ("sell_velocity_chebyshev_f32", 2)):
        ms, by = prob.time_kernel(which, reps=30)
        out[name] = {"us": ms * 1e3, "bytes": by, "gbs": by / ms / 1e6, "hbm_frac": by / ms / 1e6 / peak}
    out.update(fused_kernels(prob, peak, alu_peak, 30))
    # V-cycles as a whole (L2 warm, as inside a solve): algorithmic bytes
    # (vectors once per level, the dense coarsest inverse once) and FLOPs
    for name, which in (("vcycle_velocity_f32", 4), ("vcycle_pressure_f32", 5)):
        try:
            ms, by = prob.time_kernel(which, reps=30)
            fl = prob.kernel_flops(which)
            out[name] = {"us": ms * 1e3, "bytes": by, "flops": fl, "gbs": by / ms / 1e6,
                         "hbm_frac": by / ms / 1e6 / peak, "tflops": fl / ms / 1e9,
                         "alu_frac": fl / ms / 1e9 / alu_peak}
        except Exception:
            pass
    # C_f assembly (S2-S4) with the located-point rule of this workload, and
    # with the paper's exact rule (mesh intersection) on the same X^n
    try:
        ms, _ = prob.time_kernel(8, reps=20)
        out["cf_assembly_point_rule"] = {"us": ms * 1e3}
        from paper_2301_10041_gb300 import fsi as _f
        import fsi_inputs as _fi
        c = _fi.cavity128_case()
        px = _f.problem_from_case(c, precision=1, precond=PRECOND, stokes_its=STOKES_ITS, coupling=1,
                                  **arm_settings(1))
        px.assemble_step()
        ms, _ = px.time_kernel(9, reps=20)
        out["cf_assembly_exact_rule"] = {"us": ms * 1e3}
        px.close()
    except Exception as e:  # report, do not fail the bench line
        out["cf_assembly_error"] = str(e)
    traffic = None   # DRAM bytes per launch from the committed ncu summary of this kernel
    prof = os.path.join(ROOT, "profiles", "ncu_velocity_down_fused_n128.md")
    if os.path.exists(prof):
        for line in open(prof):
            if line.startswith("dram_bytes_per_launch:"):
                traffic = float(line.split(":")[1])
    dom = out.get("velocity_down_fused_f32")
    if dom is None:   # fused levels off (--no-mg-fused): the per-level sparse smoothing step
        d = out["sell_velocity_chebyshev_f32"]
        return {"bound": "hbm", "kernel": "k_sell<float,2,2,false,4,MODE_CHEB> (finest velocity level)",
                "achieved": d["gbs"], "peak": peak, "unit": "GB/s", "frac": d["hbm_frac"], "traffic": None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6800 GB/s",
                "launch_us": d["us"], "algorithmic_bytes": d["bytes"], "others": out}
    return {"bound": "alu", "kernel": "k_mfu_down<float,8,2,512> (fused down launch, finest velocity level)",
            "achieved": dom["tflops"], "peak": alu_peak, "unit": "TFLOP/s", "frac": dom["alu_frac"],
            "traffic": traffic, "peak_source": "derived: FP32 FMA lanes x 2 x max SM clock",
            "peak_derivation": alu_how, "launch_us": dom["us"], "algorithmic_flops": dom["flops"],
            "algorithmic_bytes": dom["bytes"], "hbm_gbs": dom["gbs"], "hbm_frac": dom["hbm_frac"],
            "hbm_peak": peak, "others": out}


def large_n_roofline(fsi, stream, device_index, peak, N):
    """The same kernels on the largest sweep member (ellipse, N = 1024 by
    default: 13.5 M unknowns, matrices of GBs, far larger than L2), where
    they are bandwidth-bound; clocks sampled over this leg."""
    import fsi_inputs as fi
    case = fi.ellipse_case(N)
    prob = fsi.problem_from_case(case, precision=1, precond=PRECOND, rtol=1e-8, stream=stream.cuda_stream,
                                 max_it=MAX_IT, stokes_its=STOKES_ITS, **arm_settings(1))
    prob64 = None
    prob.assemble_step()
    clocks = ClockSampler(device_index)
    clocks.start()
    out = {"N": N, "dofs": int(prob_dofs(case)), "workload": "ellipse sweep member, m = ceil(0.4 N)"}
    for name, which in (("full_operator_f32", 0), ("sell_velocity_chebyshev_f32", 2), ("full_operator_f64", 1)):
        ms, by = prob.time_kernel(which, reps=30)
        out[name] = {"us": ms * 1e3, "bytes": by, "gbs": by / ms / 1e6, "frac": by / ms / 1e6 / peak}
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    alu_peak = fp32_peak_tflops(peaks)[0]
    out.update(fused_kernels(prob, peak, alu_peak, 20))
    for name, which in (("vcycle_velocity_f32", 4), ("vcycle_pressure_f32", 5)):
        ms, by = prob.time_kernel(which, reps=10)
        fl = prob.kernel_flops(which)
        out[name] = {"us": ms * 1e3, "bytes": by, "flops": fl, "gbs": by / ms / 1e6, "hbm_frac": by / ms / 1e6 / peak,
                     "tflops": fl / ms / 1e9, "alu_frac": fl / ms / 1e9 / alu_peak}
    prob.close()
    prob64 = fsi.problem_from_case(case, precision=0, precond=PRECOND, rtol=1e-8, stream=stream.cuda_stream,
                                   max_it=MAX_IT, stokes_its=STOKES_ITS, **arm_settings(0))
    prob64.assemble_step()
    ms, by = prob64.time_kernel(3, reps=30)
    out["sell_velocity_chebyshev_f64"] = {"us": ms * 1e3, "bytes": by, "gbs": by / ms / 1e6,
                                          "frac": by / ms / 1e6 / peak}
    prob64.close()
    out["clocks"] = clocks.stop()
    out["l2"] = "evicted before every launch (256 MiB write)"
    return out


# ------------------------------------------------------- CPU oracle timing
CPU_SCRIPT = r"""
import json, os, sys, time
sys.path.insert(0, sys.argv[1])
import numpy as np
import fsi_inputs as fi
from oracle import fsi_oracle as fo
steps = int(sys.argv[2]); budget = float(sys.argv[3])
save = sys.argv[4] if len(sys.argv) > 4 else ""
case = fi.cavity128_case()
t0 = time.perf_counter()
prob = fo.OracleProblem(case.N, case.rho_f, case.nu, case.kappa, case.dt, case.lid_u, case.ref_xy, case.tris)
setup = time.perf_counter() - t0
u, X = case.u0, case.X0
times = []
start = time.perf_counter()
for k in range(steps):
    t = time.perf_counter()
    u, p, X, lam = prob.step(u, X)
    times.append(time.perf_counter() - t)
    if k == 0 and save:
        np.savez(save, u=u, p=p, X=X, lam=lam)
    if time.perf_counter() - start > budget:
        break
print(json.dumps({"setup_s": setup, "step_s": times}))
"""


def start_cpu_baseline(args, save_path=""):
    """The oracle on the host cores in a child process, beside the GPU arms;
    with save_path it also writes its first time step's solution there."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    env.pop("CUDA_VISIBLE_DEVICES", None)
    return subprocess.Popen([sys.executable, "-c", CPU_SCRIPT, ROOT, str(args.cpu_steps), str(args.cpu_budget),
                             save_path],
                            stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)


def field_errors(case, gpu_state, oracle_npz):
    """Relative L2 error of each field of the first time step (u with its
    wall values, p, the displacement X - X^0, lambda) against the oracle's
    direct solve of the same step."""
    o = np.load(oracle_npz)
    u, p, X, lam = gpu_state

    def rel(a, b):
        return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))

    return {"u": rel(u, o["u"]), "p": rel(p, o["p"]), "X": rel(X - case.X0, o["X"] - case.X0),
            "lam": rel(lam, o["lam"])}


def finish_cpu_baseline(proc):
    out, err = proc.communicate()
    try:
        r = json.loads(out.strip().splitlines()[-1])
    except Exception:
        return {"value": None, "unit": "time-steps/s", "cores": 1, "kind": "oracle",
                "sample": "failed: " + (err or "")[-300:]}
    st = r["step_s"]
    return {"value": len(st) / sum(st), "unit": "time-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(st)} full time step(s) of the same N=128 workload (C_f by brute-force point "
                      f"location + bordered sparse LU of Eq. (matrix)), single thread, {sum(st):.1f} s; "
                      f"constant-matrix setup {r['setup_s']:.1f} s excluded"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    env_cores = 1
    proc = subprocess.run([sys.executable, "-c", CPU_SCRIPT, ROOT, str(max(1, args.steps)), str(args.cpu_budget)],
                          capture_output=True, text=True,
                          env=dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1"))
    try:
        r = json.loads(proc.stdout.strip().splitlines()[-1])
    except Exception:
        print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " + proc.stderr[-200:]}))
        return
    st = r["step_s"]
    v = len(st) / sum(st)
    sample = (f"{len(st)} of {args.steps} requested time steps of the N=128 workload within a "
              f"{args.cpu_budget:.0f} s budget; constant-matrix setup ({r['setup_s']:.1f} s) is the warm-up")
    case = workload()
    out = {"metric": METRIC, "value": v, "unit": "time-steps/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
           "steps": len(st), "warmup": args.warmup, "ms_per_step": 1000.0 * sum(st) / len(st),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (analytic disk mesh, fluid at rest, lid 1)", "config": workload_config(case),
           "impl": "reference",
           "cpu_baseline": {"value": v, "unit": "time-steps/s", "cores": env_cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": "time-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    out["config"]["dofs"] = int(prob_dofs(case))
    print(json.dumps(out))


def run_profile_step(args):
    """A small run for per-kernel profilers: the mixed-precision problem of the
    bench workload, ``--warmup`` untimed steps, then one step.  Run it with
    FSI_HOST_LOOP=1 so that the Arnoldi loop is host-driven and ncu can see
    every kernel (graphs with conditional nodes hide their kernels from it)."""
    from paper_2301_10041_gb300 import build, fsi
    build.build()
    case = workload()
    prob = fsi.problem_from_case(case, precision=1, precond=PRECOND, rtol=1e-8, max_it=MAX_IT, stokes_its=STOKES_ITS,
                                 coupling=1 if args.coupling == "exact" else 0, **arm_settings(1), **mg_settings())
    for _ in range(args.warmup):
        prob.step()
    info = prob.step()
    print(json.dumps({"profile_step": True, "iterations": info.iterations, "refinements": info.refinements,
                      "rel_residual": info.rel_residual, "kernel_nodes": prob.graph_kernel_counts().tolist()}))
    prob.close()


def batch_arm(fsi, torch, cases, precision, args):
    """One arm of the batched workload: every instance created, then
    ``--warmup`` untimed and ``--steps`` timed ticks of fsi_step_batch."""
    t0 = time.perf_counter()
    probs = [fsi.problem_from_case(c, precision=precision, precond=PRECOND, restart=BATCH_RESTART, max_it=6000,
                                   stokes_its=args.batch_stokes_its, **mg_settings()) for c in cases]
    t_create = time.perf_counter() - t0
    for _ in range(args.warmup):
        fsi.step_batch(probs)
    torch.cuda.synchronize()
    ticks = []
    its = []
    failures = 0
    failed = []   # (tick, instance, N, kappa, nu, status, iterations, refinements, rel_residual)
    for k in range(args.steps):
        t = time.perf_counter()
        st, infos = fsi.step_batch(probs)
        ticks.append(time.perf_counter() - t)
        its.append(sum(i.iterations for i in infos))
        failures += sum(1 for i in infos if i.status != 0)
        for j, i in enumerate(infos):
            if i.status != 0 and len(failed) < 64:
                c = cases[j]
                failed.append([k, j, c.N, c.kappa, c.nu, i.status, i.iterations, i.refinements, i.rel_residual])
    for p in probs:
        p.close()
    n = len(cases)
    return {"value": n * args.steps / sum(ticks), "unit": "time-steps/s",
            "tick_ms": {"p50": float(np.percentile(ticks, 50)) * 1e3, "p99": float(np.percentile(ticks, 99)) * 1e3},
            "krylov_iterations_per_instance_step": float(np.sum(its)) / (n * args.steps),
            "create_s": t_create, "failed_instance_steps": failures,
            "failed": {"columns": ["tick", "instance", "N", "kappa", "nu", "status", "iterations", "refinements",
                                   "rel_residual"], "rows": failed}}


BATCH_RESTART = 60


def run_profile_kernel(args):
    """A small run for a per-kernel profiler: one problem of the size sweep
    (ellipse, --profile-n cells, --profile-precision) and --profile-reps
    launches of the kernel --profile-kernel of fsi_time_kernel (each after an
    L2-evicting write), nothing else."""
    import fsi_inputs as fi
    from paper_2301_10041_gb300 import build, fsi
    build.build()
    case = fi.ellipse_case(args.profile_n)
    prob = fsi.problem_from_case(case, precision=args.profile_precision, precond=PRECOND, rtol=1e-8,
                                 max_it=MAX_IT, stokes_its=STOKES_ITS, **arm_settings(args.profile_precision),
                                 **mg_settings())
    prob.assemble_step()
    ms, by = prob.time_kernel(args.profile_kernel, reps=args.profile_reps)
    print(json.dumps({"profile_kernel": args.profile_kernel, "N": args.profile_n,
                      "precision": args.profile_precision, "us": ms * 1e3, "bytes": by}))
    prob.close()


def run_batch(args):
    """Batched uneven instances (256 cavity instances of uneven size): fsi_step_batch over the
    whole set each tick, every instance on its own stream; the mixed-precision arm and the
    plain FP64 arm, both to the 1e-8 residual."""
    import torch
    import fsi_inputs as fi
    from paper_2301_10041_gb300 import build, fsi
    build.build()
    n = args.batch_instances
    cases = [fi.batch_instance(i) for i in range(n)]
    arms = {}
    for name in args.arms.split(","):
        arms[name] = batch_arm(fsi, torch, cases, 1 if name == "mixed" else 0, args)
        print(json.dumps({"batch_arm": name, **arms[name]}), file=sys.stderr, flush=True)
    head = arms.get("mixed") or next(iter(arms.values()))
    out = {"metric": METRIC, "workload": "batch", "value": head["value"], "unit": "time-steps/s",
           "instances": n, "steps": args.steps, "warmup": args.warmup, "arms": arms,
           "dtype": "f32 operators + f64 refinement (mixed arm); f64 (fp64 arm)", "data": "synthetic",
           "config": {"workload": "256 cavity instances, N~U{16,32,48,64,96}, R~U[0.1,0.3], kappa log-U[1,1e4], "
                                  "nu log-U[1e-3,1], m=ceil(2RN), restart %d, block upper-triangular, %d inner "
                                  "Stokes steps, rtol 1e-8" % (BATCH_RESTART, args.batch_stokes_its),
                      "instances": n, "mg": mg_settings()}}
    print(json.dumps(out))


# ------------------------------------------------------------ size sweep
SWEEP_SIZES = (64, 256, 512, 1024)
# (label, precond, Stokes Richardson steps): the paper's two block
# preconditioners with one V-cycle pair per inner block and with 16 Richardson
# steps of it (a nearly exact Stokes block, as the paper's exact inner
# solves), and the bench default
SWEEP_VARIANTS = (("block-diagonal", 0, 1),
                  ("block-lower-triangular", 1, 1),
                  ("block-diagonal, 16 Stokes Richardson steps", 0, 16),
                  ("block-lower-triangular, 16 Stokes Richardson steps", 1, 16),
                  ("block-upper-triangular + 8 Stokes Richardson steps", PRECOND, STOKES_ITS))
SWEEP_MAX_IT = 2000


def run_sweep(args):
    """Ellipse size sweep (N = 64 .. 1024, m = ceil(0.4 N)): Krylov iterations
    per step of each preconditioner, time per step, and the roofline of the
    finest-level kernels at every size (HBM-bound once the matrices leave L2)."""
    import torch
    import fsi_inputs as fi
    from paper_2301_10041_gb300 import build, fsi
    build.build()
    fsi.load_library()
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("hbm_gbs", 6800.0)
    sizes = [int(v) for v in args.sweep_sizes.split(",")]
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    rows = []
    for N in sizes:
        case = fi.ellipse_case(N)
        for label, pc, sits in SWEEP_VARIANTS:
            t0 = time.perf_counter()
            prob, st = time_arm(fsi, torch, case, 1, args.sweep_steps, 1, stream, flush, precond=pc,
                                stokes_its=sits, max_it=args.sweep_max_it, check=False,
                                settings=dict(restart=RESTART))
            row = {"N": N, "preconditioner": label, "precond": pc, "stokes_its": sits,
                   "dofs": int(prob_dofs(case)), "solid_nodes": int(case.ref_xy.shape[0]),
                   "solid_tris": int(case.tris.shape[0]),
                   "iterations_per_step": st["iterations"], "status": st["status"],
                   "converged_steps": sum(1 for v in st["status"] if v == 0),
                   "ms_per_step": float(np.mean(st["ms"])), "rel_residual_max": st["rel_residual_max"],
                   "wall_s": time.perf_counter() - t0}
            if pc == PRECOND and sits == STOKES_ITS:
                kern = {}
                for name, which in (("full_operator_f32", 0), ("full_operator_f64", 1),
                                    ("velocity_chebyshev_f32", 2), ("velocity_chebyshev_f64", 3)):
                    ms, by = prob.time_kernel(which, reps=20)
                    kern[name] = {"us": ms * 1e3, "bytes": by, "gbs": by / ms / 1e6, "frac": by / ms / 1e6 / peak}
                row["kernels"] = kern
            prob.close()
            rows.append(row)
            print(json.dumps({"sweep_row": row}), file=sys.stderr, flush=True)
    out = {"metric": METRIC, "workload": "sweep", "unit": "time-steps/s",
           "value": None, "rows": rows, "hbm_peak_gbs": peak,
           "config": {"workload": "ellipse 0.2/0.1 rotated 30 deg, m=ceil(0.4N), kappa=1e2, nu=1, rho=1, dt=0.01, "
                                  "walls and fluid at rest, mixed precision, rtol 1e-8, restart %d" % RESTART,
                      "sizes": sizes, "steps_per_case": args.sweep_steps, "max_it": args.sweep_max_it,
                      "l2": "flushed between timed steps (512 MiB write)"}}
    print(json.dumps(out))


# ------------------------------------------------------- nonlinear solid (bar)
BAR_SIZES = (32, 64, 128)


def run_bar(args):
    """The nonlinear bar (Section 6: exponential strain energy, Newton's
    method) at growing fluid grids with the solid mesh refined alongside:
    Newton iterations per step, Krylov iterations per Newton iteration and
    time per step for the block-diagonal and block-triangular preconditioners
    (the quantities of the paper's nonlinear table)."""
    import torch
    import fsi_inputs as fi
    from paper_2301_10041_gb300 import build, fsi
    build.build()
    fsi.load_library()
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    rows = []
    for N in [int(v) for v in args.bar_sizes.split(",")]:
        case = fi.bar_case(N=N, nx=N // 2, ny=max(2, N // 8))
        for label, pc in (("block-diagonal", 0), ("block-lower-triangular", 1)):
            prob = fsi.problem_from_case(case, precision=1, precond=pc, rtol=1e-8, stream=stream.cuda_stream,
                                         max_it=MAX_IT, restart=60, stokes_its=1)
            for _ in range(1):
                prob.step()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.bar_steps)]
            infos = []
            torch.cuda.synchronize()
            for k in range(args.bar_steps):
                with torch.cuda.stream(stream):
                    flush.fill_(k & 0xFF)
                ev[k][0].record(stream)
                infos.append(prob.step())
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            ms = [a.elapsed_time(b) for a, b in ev]
            newton = [i.newton_iterations for i in infos]
            rows.append({"N": N, "preconditioner": label, "dofs": int(prob_dofs(case)),
                         "solid_nodes": int(case.ref_xy.shape[0]), "newton_per_step": newton,
                         "krylov_per_newton": [round(i.iterations / max(1, i.newton_iterations), 1) for i in infos],
                         "ms_per_step": float(np.mean(ms)), "status": [i.status for i in infos]})
            print(json.dumps({"bar_row": rows[-1]}), file=sys.stderr, flush=True)
            prob.close()
    print(json.dumps({"metric": METRIC, "workload": "bar", "unit": "time-steps/s", "value": None, "rows": rows,
                      "config": {"workload": "bar [0,0.4]x[0.45,0.55], W = (gamma/2eta) exp(eta(tr F^T F - 2)), "
                                             "gamma 1.333, eta 9.242, rho 1, nu 0.2, dt 0.002, bent start, mixed "
                                             "precision, rtol 1e-8, Newton 1e-6, one V-cycle pair per Stokes "
                                             "application", "steps": args.bar_steps}}))


# ----------------------------------------------- quarter annulus (Table 1)
ANNULUS_SIZES = (48, 96, 192, 384)


def run_annulus(args):
    """The linear-solid refinement test of Section 6 (the paper's Table 1:
    quarter annulus released from a stretched state, kappa = 10, nu = 0.1,
    dt = 0.01): Krylov iterations per step of the block-diagonal and
    block-lower-triangular preconditioners as the fluid grid and the solid
    mesh are refined together, with one V-cycle pair per Stokes application
    and with 16 Richardson steps of it (nearly exact Stokes block; the solid
    block is exact up to its Chebyshev solves)."""
    import torch
    import fsi_inputs as fi
    from paper_2301_10041_gb300 import build, fsi
    build.build()
    fsi.load_library()
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    rows = []
    for N in [int(v) for v in args.annulus_sizes.split(",")]:
        # --annulus-symmetric: the paper's free-slip walls by symmetry (the
        # full annulus on an N grid, equivalent to the quarter on N/2)
        # --annulus-q1: the paper's Q1 solid (one quadrilateral per (r, t) cell)
        q1 = args.annulus_q1
        case = (fi.symmetric_annulus_case(N // 2, quads=q1) if args.annulus_symmetric
                else fi.annulus_case(N, quads=q1))
        variants = [(lab, pc, int(si)) for si in args.annulus_stokes_its.split(",")
                    for lab, pc in (("block-diagonal", 0), ("block-lower-triangular", 1))]
        for label, pc, sits in variants:
            prob, st = time_arm(fsi, torch, case, 1, args.annulus_steps, 1, stream, flush, precond=pc,
                                stokes_its=sits, max_it=SWEEP_MAX_IT, check=False, settings=dict(restart=RESTART))
            rows.append({"N": N, "preconditioner": label, "stokes_its": sits, "dofs": int(prob_dofs(case)),
                         "solid_nodes": int(case.ref_xy.shape[0]), "iterations_per_step": st["iterations"],
                         "status": st["status"], "ms_per_step": float(np.mean(st["ms"]))})
            print(json.dumps({"annulus_row": rows[-1]}), file=sys.stderr, flush=True)
            prob.close()
    walls = ("free-slip x = 0, y = 0 by symmetry (full annulus, nu/4, kappa/4, grid N = 2 Nq)"
             if args.annulus_symmetric else "no-slip walls")
    print(json.dumps({"metric": METRIC, "workload": "annulus", "unit": "time-steps/s", "value": None, "rows": rows,
                      "config": {"workload": "quarter annulus 0.3<=|s|<=0.5 released from X = (s1/1.4, 1.4 s2), "
                                             "kappa 10, rho 1, nu 0.1, dt 0.01, %s, %s solid, mixed precision, "
                                             "rtol 1e-8, restart %d"
                                             % (walls, "Q1" if args.annulus_q1 else "P1", RESTART),
                                 "steps": args.annulus_steps, "stokes_its": args.annulus_stokes_its}}))


def run_serve(args):
    """Served stream (Poisson arrivals of cavity requests): Poisson arrivals replayed in wall
    time, admission by device footprint, continuous batching."""
    import fsi_inputs as fi
    from paper_2301_10041_gb300 import build
    from paper_2301_10041_gb300.serve import Request, Server, gpu_ops
    build.build()
    trace = fi.serve_trace(args.serve_requests)
    def largest_body(N):   # R <= 0.3, m = ceil(2 R N): the largest ring mesh for this grid
        m = int(np.ceil(2 * 0.3 * N))
        return 1 + 3 * m * (m + 1), 6 * m * m

    arms = {}
    for name in args.arms.split(","):
        ops = gpu_ops(precision=1 if name == "mixed" else 0, restart=60, stokes_its=args.serve_stokes_its,
                      max_solid_nodes=largest_body)
        reqs = [Request(rid=i, arrival=t, case=fi.serve_case(spec), steps=50) for i, (t, spec) in enumerate(trace)]
        srv = Server(ops, budget_bytes=int(args.serve_budget_gb * (1 << 30)), max_resident=args.serve_max_resident,
                     admit_per_tick=2, policy=args.serve_policy)
        wall = srv.run(reqs, realtime=True, max_wall=args.serve_wall)
        rep = srv.report(wall)
        rep["offered_steps_per_s"] = sum(r.steps for r in reqs if r.arrival <= wall) / wall
        rep["failed_requests"] = sum(1 for r in srv.finished if r.error)
        arms[name] = rep
        print(json.dumps({"serve_arm": name, **rep}), file=sys.stderr, flush=True)
    head = arms.get("mixed") or next(iter(arms.values()))
    out = {"metric": METRIC, "workload": "serve", "value": head["steps_per_s"], "unit": "time-steps/s",
           "offered_steps_per_s": head["offered_steps_per_s"], "p50_step_ms": head["step_latency_ms"]["p50"],
           "p99_step_ms": head["step_latency_ms"]["p99"], "arms": arms,
           "config": {"workload": "Poisson 200/s, N in {32,64,128,256} p=.4/.3/.2/.1, disk/ellipse, R~U[0.1,0.3], "
                                  "kappa log-U[1,1e4], 50 steps each", "requests": args.serve_requests,
                      "budget_gb": args.serve_budget_gb, "wall_cap_s": args.serve_wall,
                      "admission": args.serve_policy, "max_resident": args.serve_max_resident}}
    print(json.dumps(out))


def main():
    global AUTOTUNE, MG_FUSED, MG_CLUSTER, MG_DEGREE, MG_COARSE, MG_COARSE_P, CS_DEGREE, STOKES_ITS
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-large-n", action="store_true", help="skip the N = 1024 roofline leg")
    ap.add_argument("--large-n", type=int, default=1024, help="grid of the large-N roofline leg")
    ap.add_argument("--cpu-steps", type=int, default=1)
    ap.add_argument("--cpu-budget", type=float, default=300.0)
    ap.add_argument("--profile-step", action="store_true",
                    help="only build the mixed problem, run --warmup steps and one more (for ncu)")
    ap.add_argument("--profile-kernel", type=int, default=-1,
                    help="only time kernel WHICH of fsi_time_kernel on one ellipse problem (for ncu)")
    ap.add_argument("--profile-n", type=int, default=512)
    ap.add_argument("--profile-precision", type=int, default=0)
    ap.add_argument("--profile-reps", type=int, default=2)
    ap.add_argument("--workload", choices=["cavity128", "batch", "serve", "sweep", "bar", "annulus"],
                    default="cavity128",
                    help="cavity128 (default, the contract line); the others print their own lines")
    ap.add_argument("--batch-instances", type=int, default=256)
    ap.add_argument("--batch-stokes-its", type=int, default=12,
                    help="Richardson steps on the Stokes block per preconditioner application (batch workload; "
                         "12: every instance-step reaches 1e-8, 8 left the stiffest instance stalled)")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    ap.add_argument("--serve-max-resident", type=int, default=16)
    ap.add_argument("--serve-wall", type=float, default=60.0)
    ap.add_argument("--serve-stokes-its", type=int, default=8)
    ap.add_argument("--serve-policy", choices=["sjf", "fifo"], default="sjf",
                    help="admission: shortest predicted work first with an age bound, or first come first served")
    ap.add_argument("--arms", default="mixed,fp64",
                    help="batch and serve workloads: which precisions to run (mixed, fp64)")
    ap.add_argument("--no-mg-fused", action="store_true",
                    help="per-level sparse kernels on every multigrid level instead of the fused matrix-free ones")
    ap.add_argument("--stokes-its", type=int, default=STOKES_ITS,
                    help="Richardson steps on the Stokes block per preconditioner application (bench workload)")
    ap.add_argument("--mg-degree", type=int, default=0, help="Chebyshev degree of each multigrid smoothing")
    ap.add_argument("--mg-coarse-p", type=int, default=0,
                    help="coarsest pressure multigrid grid in cells (0: the library's default)")
    ap.add_argument("--cs-degree", type=int, default=0,
                    help="Chebyshev steps per solid mass solve (0: the library's default)")
    ap.add_argument("--mg-coarse", type=int, default=0,
                    help="coarsest multigrid grid in cells (0: the library's default)")
    ap.add_argument("--mg-cluster", type=int, default=0,
                    help="0: coarse levels in one cluster launch; -1: per-level launches; n > 0: only levels of at "
                         "most n cells a side in the cluster")
    ap.add_argument("--autotune", action="store_true",
                    help="per-level SpMV tile shapes chosen by the library's autotuner instead of one fixed shape")
    ap.add_argument("--coupling", choices=["point", "exact"], default="point",
                    help="C_f rule of --profile-step (the bench line always uses the point rule)")
    ap.add_argument("--sweep-sizes", default=",".join(str(v) for v in SWEEP_SIZES))
    ap.add_argument("--bar-sizes", default=",".join(str(v) for v in BAR_SIZES))
    ap.add_argument("--bar-steps", type=int, default=5)
    ap.add_argument("--annulus-sizes", default=",".join(str(v) for v in ANNULUS_SIZES))
    ap.add_argument("--annulus-steps", type=int, default=2)
    ap.add_argument("--annulus-symmetric", action="store_true",
                    help="free-slip walls x = 0, y = 0 by symmetry (full annulus, nu and kappa scaled)")
    ap.add_argument("--annulus-q1", action="store_true",
                    help="Q1 quadrilateral solid (the paper's element) instead of P1 triangles")
    ap.add_argument("--annulus-stokes-its", default="1,16",
                    help="Richardson steps on the Stokes block: 1 = one V-cycle pair, 16 = nearly exact")
    ap.add_argument("--sweep-steps", type=int, default=2)
    ap.add_argument("--sweep-max-it", type=int, default=SWEEP_MAX_IT)
    args = ap.parse_args()
    MG_CLUSTER = args.mg_cluster
    MG_DEGREE = args.mg_degree
    MG_COARSE = args.mg_coarse
    CS_DEGREE = args.cs_degree
    MG_COARSE_P = args.mg_coarse_p
    STOKES_ITS = args.stokes_its
    if args.autotune:
        AUTOTUNE = 1
    if args.no_mg_fused:
        MG_FUSED = -1
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "bar":
        return run_bar(args)
    if args.workload == "annulus":
        return run_annulus(args)
    if args.profile_step:
        return run_profile_step(args)
    if args.profile_kernel >= 0:
        return run_profile_kernel(args)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
