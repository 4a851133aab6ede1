"""Benchmark of the MPPI solve on GB300 (one JSON line on rank 0).

Workload (one "step"): one batched MPPI solve of 256 independent drones, each
on its own seeded 5-9 gate course, K log-uniform in [1024, 16384], N uniform
in [20, 80], dt = 0.02 s, objectives 1/3 each (gate progress, contouring,
tracking), launched as one CUDA graph (one branch per objective: noise ->
rollout+cost+weights+update, and the nominal rollouts at the end of the gate
branch).  The launch shape (block size, graph form, where the normals are
drawn, samples per thread) is autotuned first, untimed.  Metric:
rollout-steps/s = sum_i K_i N_i / step time.

  value       device-timed (CUDA events on the launch stream) over --steps
              steps after an untimed busy phase, inputs resident in HBM
              (mppi_batch_solve_async on device buffers)
  e2e         the public host call mppi_batch_solve: x0/t0 from host memory,
              u0 back to host memory, inside the timed region
  plain       the same 256 solves through mppi_solve one drone at a time
              (one solve per launch sequence, single-solve launch shape), the
              single-drone K=4096/N=50 solve and the paper's Table I sizes:
              solves/s and p50/p99 latency
  roofline    the rollout kernels (dominant): algorithmic FP32 operations
              per launch / mean launch time, against the FP32 pipe peak
              SMs x 128 lanes x 2 x max SM clock
  cpu_baseline  the FP64 oracle on a bounded sample of the same workload, and
              the error of fresh CUDA solves of the first sampled drones
              against it (parity_vs_oracle)
  also        the rotor-thrust-rate model on the same batch, the closed-loop
              objective comparison, and a served fleet (continuous batching)

With torchrun (N > 1) every rank solves its own 256 drones (weak scaling, no
collective on the data path); value = all ranks' rollout steps / max time.
`--impl reference` times the oracle (the reference arm for this path).
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

# algorithmic FP32 operations per rollout step (FMA = 2, add/mul/min/max/
# compare = 1, rsqrt = 1), counted from the kernel's arithmetic for the gate
# objective without drag: sampling 16, RK4 358, objective 28, feasibility
# penalty 17, cost Kahan step 4; contouring's objective counts 92 and adds a
# 5th input, tracking's stage and terminal terms give 478
FLOPS_PER_STEP = {0: 423.0, 1: 491.0, 2: 478.0}
# the same for the rotor-thrust-rate model: its RK4 step counts 466 against 358
# (saturating compensated thrust ramps, three sets of rotor forces and torques)
FLOPS_PER_STEP_ROTOR = {0: 531.0, 1: 599.0, 2: 586.0}


def _captured_per_step(kind: str):
    """Per-rollout-step figures of one kind ("bytes_per_step" or
    "fp32_ops_per_step") by objective, from the ncu capture recorded under
    profiles/, or None when the kernel source is not the one that was
    captured."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "rollout_kernel_traffic.txt")
    src = os.path.join(ROOT, "paper_2509_14726_gb300", "csrc")
    try:
        with open(path) as f:
            lines = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
        h = hashlib.sha256()
        for name in ("mppi_rollout.cuh", "mppi_device.cuh"):
            with open(os.path.join(src, name), "rb") as f:
                h.update(f.read())
    except OSError:
        return None
    rec = {ln[0]: ln[1:] for ln in lines if ln[0] == "source_sha256"}
    if rec.get("source_sha256", [None])[0] != h.hexdigest():
        return None
    per = {ln[1]: float(ln[2]) for ln in lines if ln[0] == kind}
    names = {0: "gate", 1: "contour", 2: "track"}
    if any(names[o] not in per for o in (0, 1, 2)):
        return None
    return {o: per[names[o]] for o in (0, 1, 2)}


def measured_traffic(steps_by_objective):
    """DRAM bytes of the three rollout launches of one step: the captured
    bytes per rollout step per objective scaled by this workload's K x N."""
    per = _captured_per_step("bytes_per_step")
    if per is None:
        return None
    return sum(per[o] * steps_by_objective[o] for o in (0, 1, 2))


def measured_fp32_ops(steps_by_objective):
    """FP32 operations (FFMA = 2, FADD, FMUL) the three rollout launches of
    one step execute, by ncu's SASS counters per rollout step scaled by this
    workload's K x N; with the per-step figures."""
    per = _captured_per_step("fp32_ops_per_step")
    if per is None:
        return None, None
    return sum(per[o] * steps_by_objective[o] for o in (0, 1, 2)), per


def paper_table1_latency(M, W, reps: int = 300) -> dict:
    """Single-solve latency at the paper's Table I size for each objective
    (the paper reports about 0.4 ms on an RTX 3090 for 8192 samples), for
    three ways of drawing the normals: the separate Philox pass before the
    rollout, the rollout keeping them in shared memory, and the separate pass
    run after each solve for the next one.  Columns (ms):
      p50, p99: host-synchronous mppi_solve through the Python binding, the
                device idle when the call starts (a controller that solves
                once per control period);
      c_p50:    the same call made through ctypes with the arguments built
                once (the C-ABI call itself, without the binding's marshalling);
      device:   device time per solve, solves enqueued back to back
                (mppi_solve_async; for the ahead mode this includes the draw
                for the next solve)."""
    import ctypes as C
    import torch
    out = {}
    names = {0: "gate", 1: "contour", 2: "track"}
    modes = (("noise_pass", M.NOISEGEN_KERNEL), ("noise_in_smem", M.NOISEGEN_SMEM),
             ("noise_ahead", M.NOISEGEN_AHEAD))
    L = M.load()
    for K in (8192, 2048):
        for obj in (0, 1, 2):
            mc, sc, tr, x0 = W.paper_table1(obj, K)
            if obj == 2:
                x0 = tr.ref[0].astype(np.float64)  # on the reference at t = 0
            row = {}
            for mode, gen in modes:
                ctl = M.Controller(mc, sc, tr, noise_gen=gen)
                for _ in range(30):
                    ctl.solve(x0, 0.0)
                lat, lat_c = [], []
                for _ in range(reps):
                    torch.cuda.synchronize()
                    t = time.perf_counter()
                    ctl.solve(x0, 0.0)
                    lat.append(time.perf_counter() - t)
                x = np.ascontiguousarray(np.float32(x0))
                u = np.zeros(5, np.float32)
                xp, up, hh = x.ctypes.data_as(M.PF), u.ctypes.data_as(M.PF), C.c_void_p(ctl.h)
                for _ in range(reps):
                    torch.cuda.synchronize()
                    t = time.perf_counter()
                    rc = L.mppi_solve(hh, xp, 0.0, None, up)
                    lat_c.append(time.perf_counter() - t)
                    assert rc == M.MPPI_OK, rc
                s = torch.cuda.Stream()
                dx = torch.tensor(np.float32(x0), device="cuda")
                du = torch.zeros(5, dtype=torch.float32, device="cuda")
                torch.cuda.synchronize()
                with torch.cuda.stream(s):
                    for _ in range(10):
                        M.mppi_solve_async(ctl.h, dx.data_ptr(), 0.0, s, du.data_ptr())
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(s)
                    for _ in range(reps):
                        M.mppi_solve_async(ctl.h, dx.data_ptr(), 0.0, s, du.data_ptr())
                    e1.record(s)
                s.synchronize()
                row[mode] = [round(float(np.percentile(lat, 50) * 1e3), 4), round(float(np.percentile(lat, 99) * 1e3), 4),
                             round(float(np.percentile(lat_c, 50) * 1e3), 4), round(e0.elapsed_time(e1) / reps, 4)]
                ctl.close()
            out[f"K{K}_N20_{names[obj]}"] = row
    out["columns"] = "p50_ms, p99_ms, c_p50_ms, device_ms_per_solve"
    out["protocol"] = ("p50/p99: mppi_solve via the Python binding with the device idle at each call; c_p50: the "
                       "same C-ABI call via ctypes with prebuilt arguments; device: back-to-back solves, CUDA events")
    out["paper_rtx3090_ms"] = 0.4
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--drones", type=int, default=256)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-closed-loop", action="store_true")
    ap.add_argument("--no-rotor", action="store_true")
    ap.add_argument("--cpu-sample-s", type=float, default=12.0)
    ap.add_argument("--repeats", type=int, default=25,
                    help="batched solves of the fleet per timed step (consecutive control periods)")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="arrival window of the serving run (the configured fleet asks for 60 s)")
    ap.add_argument("--table1-only", action="store_true",
                    help="print only the single-solve latency at the paper's Table I sizes (one JSON line)")
    ap.add_argument("--table1-reps", type=int, default=300, help="timed solves per Table I case and column")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v: float) -> float:
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, v: float) -> float:
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate(world: int, steps_this_rank: float, ms_this_rank: float):
    """Whole-job throughput: all ranks' rollout steps over the slowest rank's
    time per step.  Returns (value, ms_max, total_steps)."""
    ms_max = max_over_ranks(world, ms_this_rank)
    total = sum_over_ranks(world, steps_this_rank)
    return total / (ms_max / 1e3), ms_max, total


def workload(rank: int, n: int):
    from paper_2509_14726_gb300 import workloads as W
    return W.c3_batch(n_drones=n, seed=3 + 1000 * rank)


def make_cfg(it):
    from paper_2509_14726_gb300 import workloads as W
    return W.SolveConfig(objective=it.objective, K=it.K, N=it.N, dt=0.02, lam=1.0, seed=0, drone_id=it.drone_id)


def start_states(items, t0: float):
    X = []
    for it in items:
        x = it.x0.copy()
        if it.objective == 2:
            # start on the reference at t0 (the track's own table row)
            tr = it.track
            i = int(round(t0 / tr.dt_ref)) % tr.ref.shape[0]
            x = tr.ref[i].copy()
        X.append(x)
    return np.array(X)


def host_facts() -> dict:
    """Host CPU: logical cores, nproc, model name (lscpu / /proc/cpuinfo)."""
    facts = {"os_cpu_count": os.cpu_count()}
    try:
        facts["nproc"] = int(subprocess.run(["nproc"], capture_output=True, text=True).stdout.strip())
    except Exception:
        facts["nproc"] = None
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Vendor ID") and ":" in line:
                model = (model + " / " if model else "") + line.split(":", 1)[1].strip()
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    facts["cpu_model"] = model
    facts["machine"] = os.uname().machine
    return facts


def oracle_parity(items, M, n_parity: int = 6) -> dict:
    """Fresh CUDA handles and the single-thread FP64 oracle solve the first
    n_parity drones of the workload from the same binary32-rounded inputs.
    Per drone: the per-sample cost error (relative and absolute), gate
    decisions, and the nominal error against the literal 1e-5 bound; a miss
    carries the solve's binary32 floor (oracle.conditioning)."""
    from oracle import oracle as O
    from oracle.conditioning import binary32_floor
    from paper_2509_14726_gb300 import workloads as W
    O.build()
    t0 = 0.3
    X = start_states(items, t0)
    out = {"bound_nominal": 1e-5, "bound_cost_rel": 1e-4, "per_drone": [], "literal_pass": 0, "literal_miss": 0,
           "max_rel_J": 0.0, "max_abs_J": 0.0, "max_dU": 0.0, "decision_mismatches": 0}
    for i, it in enumerate(items[:n_parity]):
        mc, sc, tr = W.f32_model(W.ModelConfig()), W.f32_solve(make_cfg(it)), it.track.as_f32()
        x = np.float32(X[i]).astype(np.float64)
        r = O.OracleController(mc, sc, tr).solve(x, t0)
        gpu = M.Controller(mc, sc, tr)
        gpu.solve(x, t0)
        J = gpu.costs()
        ok = r["near_flag"] == 0
        denom = np.maximum(np.abs(r["J"]), r["Jabs"])
        dJ = np.abs(J - r["J"])
        rel = dJ / np.where(denom > 0, denom, 1.0)
        nu = 5 if it.objective == 1 else 4
        dU = float(np.max(np.abs(gpu.unew()[:, :nu] - r["Unew"][:, :nu])))
        npass, first = gpu.sample_info()
        mism = int(((npass != r["npass"]) | (first != r["first_pass"]))[ok].sum()) if it.objective == 0 else 0
        row = {"drone": i, "objective": it.objective, "K": it.K, "N": it.N, "max_rel_J": float(rel[ok].max()),
               "max_abs_J": float(dJ[ok].max()), "max_dU": dU, "literal": dU <= 1e-5, "flagged": int((~ok).sum())}
        if dU > 1e-5:
            row["binary32_floor"] = binary32_floor(r, sc.lam, nu)
        out["per_drone"].append(row)
        out["literal_pass" if dU <= 1e-5 else "literal_miss"] += 1
        out["max_rel_J"] = max(out["max_rel_J"], row["max_rel_J"])
        out["max_abs_J"] = max(out["max_abs_J"], row["max_abs_J"])
        out["max_dU"] = max(out["max_dU"], dU)
        out["decision_mismatches"] += mism
        gpu.close()
    return out


def cpu_baseline(items, budget_s: float, omp: bool = True) -> dict:
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    whole solves of the first drones (binary32-rounded inputs, as the CUDA
    path receives them) until the time budget is used.  omp: the build with
    OpenMP over the samples of a solve, on every host core; else one thread."""
    from oracle import oracle as O
    from paper_2509_14726_gb300 import workloads as W
    O.build(omp=omp)
    t0 = 0.3
    X = start_states(items, t0)
    steps, solves, used = 0, 0, 0.0
    for i, it in enumerate(items):
        mc, sc, tr = W.f32_model(W.ModelConfig()), W.f32_solve(make_cfg(it)), it.track.as_f32()
        x = np.float32(X[i]).astype(np.float64)
        ctl = O.OracleController(mc, sc, tr, omp=omp)
        t = time.perf_counter()
        ctl.solve(x, t0, want_Us=False)
        used += time.perf_counter() - t
        steps += it.K * it.N
        solves += 1
        if used >= budget_s:
            break
    cores = O.threads(omp)
    return {"value": steps / used, "unit": "rollout-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{solves} whole solves (drones 0..{solves - 1} of the batch workload, {steps} rollout "
                      f"steps, {used:.1f} s, {'OpenMP over samples, ' if omp else ''}{cores} thread(s))",
            "solves_per_s": solves / used, "seconds": used}


def run_reference(args, world, rank):
    if rank != 0:
        return
    items = workload(0, args.drones)
    per_step = []
    for s in range(args.warmup + args.steps):
        # about two minutes over the whole run, at least one whole solve per step
        cb = cpu_baseline(items, budget_s=max(0.1, 120.0 / max(1, args.warmup + args.steps)), omp=True)
        if s >= args.warmup:
            per_step.append(cb)
    v = float(np.mean([c["value"] for c in per_step]))
    ms = float(np.mean([c["seconds"] for c in per_step]) * 1e3)
    line = {
        "impl": "reference", "metric": "rollout-steps/s", "value": v, "unit": "rollout-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "batched uneven MPPI solves: 256 drones, K logU[1024,16384], N U[20,80], "
                               "dt 0.02, 5-9 gate courses, objectives 1/3 each; a step is the oracle's whole "
                               "solves of the batch's drones in order, up to a time budget",
                   "sample_per_step": per_step[0]["sample"]},
        "cpu_baseline": {"value": v, "unit": "rollout-steps/s", "cores": per_step[0]["cores"], "kind": "oracle",
                         "sample": per_step[0]["sample"], "host": host_facts()},
        "e2e": {"value": v, "unit": "rollout-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    assert torch.cuda.is_available(), "bench needs a CUDA device"
    torch.cuda.set_device(local if world > 1 else 0)
    import __graft_entry__ as g
    g.build()
    from paper_2509_14726_gb300 import mppi as M
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    if args.table1_only:
        from paper_2509_14726_gb300 import workloads as W
        if rank == 0:
            print(json.dumps({"paper_table1_single_solve": paper_table1_latency(M, W, args.table1_reps)}))
        return

    items = workload(rank, args.drones)
    t0 = 0.3
    X0 = start_states(items, t0)
    from paper_2509_14726_gb300 import workloads as W
    # ---- autotuning (untimed): block size and graph form of the batch plan ----
    tuning = {"block": 128, "graph_mode": 1, "noise_gen": M.NOISEGEN_DEFAULT, "spt": 1, "table": None}
    if not args.no_tune:
        from paper_2509_14726_gb300 import autotune as AT

        def make_handles(block, noise_gen=None, spt=1):
            return [M.Controller(W.ModelConfig(), make_cfg(it), it.track, block=block, noise_gen=noise_gen, spt=spt)
                    for it in items]

        tuning = AT.tune_batch(make_handles, X0, t0, blocks=(64, 96, 128), modes=(1, 2), cache=None,
                               noise_gens=(M.NOISEGEN_KERNEL, M.NOISEGEN_FUSED, M.NOISEGEN_REGEN), spts=(1, 2, 4))
    ctls = [M.Controller(W.ModelConfig(), make_cfg(it), it.track, block=tuning["block"], noise_gen=tuning["noise_gen"],
                         spt=tuning["spt"]) for it in items]
    hs = [c.h for c in ctls]
    steps_per_solve = float(sum(it.K * it.N for it in items))
    flops = {o: sum(it.K * it.N * FLOPS_PER_STEP[o] for it in items if it.objective == o) for o in (0, 1, 2)}
    plan = M.mppi_batch_create(hs, use_graph=tuning["graph_mode"])
    stream = torch.cuda.Stream()
    d_x0 = torch.tensor(np.float32(X0), device="cuda")
    d_t0 = torch.full((len(items),), t0, dtype=torch.float64, device="cuda")
    d_u0 = torch.zeros((len(items), 5), dtype=torch.float32, device="cuda")

    # ---- warm-up ----
    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            M.mppi_batch_solve_async(plan, d_x0.data_ptr(), d_t0.data_ptr(), stream, d_u0.data_ptr())
    stream.synchronize()

    # ---- device-timed region (inputs resident) ----
    sampler = ClockSampler(dev)
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    # keep the GPU busy (untimed) while the sampler comes up, so that the
    # timed region starts on a warm GPU and the clock samples fall under load
    t_busy = time.perf_counter() + 0.3
    with torch.cuda.stream(stream):
        while time.perf_counter() < t_busy:
            M.mppi_batch_solve_async(plan, d_x0.data_ptr(), d_t0.data_ptr(), stream, d_u0.data_ptr())
            stream.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    launches0 = M.mppi_kernel_launches()
    R = max(1, args.repeats)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(args.steps):
            for _ in range(R):
                M.mppi_batch_solve_async(plan, d_x0.data_ptr(), d_t0.data_ptr(), stream, d_u0.data_ptr())
        e1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    launches = M.mppi_kernel_launches() - launches0
    ms = e0.elapsed_time(e1) / args.steps
    value, ms_max, total_steps = aggregate(world, R * steps_per_solve, ms)

    # ---- end to end through the host API ----
    x0_host = np.float32(X0)
    t0_host = np.full(len(items), t0)
    lat = []
    barrier(world)
    for _ in range(max(3, args.warmup)):
        M.mppi_batch_solve(plan, len(items), x0_host, t0_host)
    step_s = []
    for _ in range(args.steps):
        ts = time.perf_counter()
        for _ in range(R):
            t = time.perf_counter()
            M.mppi_batch_solve(plan, len(items), x0_host, t0_host)
            lat.append(time.perf_counter() - t)
        step_s.append(time.perf_counter() - ts)
    e2e_s = max_over_ranks(world, float(np.mean(step_s)))
    e2e = {"value": total_steps / e2e_s, "unit": "rollout-steps/s",
           "h2d_bytes_per_step": R * len(items) * (13 * 4 + 8), "d2h_bytes_per_step": R * len(items) * (5 * 4 + 4),
           "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
           "solves_per_s": len(items) / float(np.mean(lat))}

    # ---- per-kernel timing for the roofline (same launches, no graph) ----
    prof = M.mppi_batch_profile(plan, max(3, args.steps // 2), stream)
    roll_ms = float(prof[1] + prof[2] + prof[3])
    roll_flops = flops[0] + flops[1] + flops[2]
    peak = n_sm * 128 * 2 * 2070e6 / 1e12
    achieved = roll_flops / (roll_ms / 1e3) / 1e12
    steps_by_obj = {o: sum(it.K * it.N for it in items if it.objective == o) for o in (0, 1, 2)}
    traffic = measured_traffic(steps_by_obj)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "rollout_kernel (3 launches, one per objective)",
                "traffic_note": "DRAM bytes of the 3 launches: ncu per-step figures of the 64-drone capture "
                                "scaled by this batch's K x N (null if the kernel source changed since)",
                "peak_note": f"FP32 pipe: {n_sm} SMs x 128 lanes x 2 x 2070 MHz (max SM clock)",
                "phase_ms": {"noise": float(prof[0]), "rollout_gate": float(prof[1]),
                             "rollout_contour": float(prof[2]), "rollout_track": float(prof[3]),
                             "nominal": float(prof[4]), "total_no_graph": float(prof[5])}}
    if clocks.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved / (n_sm * 128 * 2 * clocks["sm_mhz"] * 1e6 / 1e12)
    noise_bytes = sum(it.K * it.N * (16 + (4 if it.objective == 1 else 0)) for it in items)
    roofline["noise_kernel_gbs"] = noise_bytes / (float(prof[0]) / 1e3) / 1e9 if prof[0] > 0 else None
    # the same fraction on the FP32 operations the hardware counted (ncu SASS
    # counters of the captured kernel: FFMA = 2, FADD, FMUL; min/max, compares
    # and MUFU not counted), beside the algorithmic count above
    ops, per = measured_fp32_ops(steps_by_obj)
    if ops is not None:
        roofline["ncu_fp32_ops_per_step"] = {n: per[o] for o, n in ((0, "gate"), (1, "contour"), (2, "track"))}
        roofline["frac_ncu_fp32_ops"] = ops / (roll_ms / 1e3) / 1e12 / peak

    # ---- the same batch with the rotor-thrust-rate model (Eq. 2 as printed) ----
    rotor_out = None
    if rank == 0 and not args.no_rotor:
        rctl = [M.Controller(W.rotor_model(), W.rotor_solve(make_cfg(it)), it.track) for it in items]
        rplan = M.mppi_batch_create([c.h for c in rctl], use_graph=1)
        with torch.cuda.stream(stream):
            for _ in range(3):
                M.mppi_batch_solve_async(rplan, d_x0.data_ptr(), d_t0.data_ptr(), stream, d_u0.data_ptr())
            r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            r0.record(stream)
            for _ in range(10):
                M.mppi_batch_solve_async(rplan, d_x0.data_ptr(), d_t0.data_ptr(), stream, d_u0.data_ptr())
            r1.record(stream)
        stream.synchronize()
        rms = r0.elapsed_time(r1) / 10
        M.mppi_batch_solve(rplan, len(items), np.float32(X0), np.full(len(items), t0))  # host inputs of the plan
        rprof = M.mppi_batch_profile(rplan, 5, stream)
        rroll_ms = float(rprof[1] + rprof[2] + rprof[3])
        rflops = sum(it.K * it.N * FLOPS_PER_STEP_ROTOR[it.objective] for it in items)
        rotor_out = {"value": steps_per_solve / (rms / 1e3), "unit": "rollout-steps/s", "ms_per_step": rms,
                     "phase_ms": {"noise": float(rprof[0]), "rollout_gate": float(rprof[1]),
                                  "rollout_contour": float(rprof[2]), "rollout_track": float(rprof[3]),
                                  "nominal": float(rprof[4])},
                     "roofline": {"bound": "alu", "achieved": rflops / (rroll_ms / 1e3) / 1e12, "peak": peak,
                                  "unit": "TFLOP/s", "frac": rflops / (rroll_ms / 1e3) / 1e12 / peak}}
        M.mppi_batch_destroy(rplan)
        for c in rctl:
            c.close()

    # ---- plain path: one solve per launch sequence ----
    plain = None
    if not args.no_plain and rank == 0:
        # the same 256 solves, one mppi_solve call each, on handles with the
        # single-solve launch shape (one sample per thread: the batch's tuned
        # shape can be slower for a solve launched alone)
        pctls = [M.Controller(W.ModelConfig(), make_cfg(it), it.track) for it in items]
        lat_p = []
        for c, x in zip(pctls, X0):
            c.solve(x, t0)
        tt = time.perf_counter()
        for c, x in zip(pctls, X0):
            t = time.perf_counter()
            c.solve(x, t0)
            lat_p.append(time.perf_counter() - t)
        wall = time.perf_counter() - tt
        for c in pctls:
            c.close()
        plain = {"batch_one_solve_per_launch": {
            "value": steps_per_solve / wall, "unit": "rollout-steps/s", "solves_per_s": len(items) / wall,
            "p50_ms": float(np.percentile(lat_p, 50) * 1e3), "p99_ms": float(np.percentile(lat_p, 99) * 1e3)}}
        # single drone, full scale (K=4096, N=50, gate progress)
        from paper_2509_14726_gb300 import workloads as W
        mc, sc, tr, x0 = W.c2_full_scale(0)
        c2 = M.Controller(mc, sc, tr)
        for _ in range(20):
            c2.solve(x0, 0.0)
        lat2 = []
        for _ in range(200):
            t = time.perf_counter()
            c2.solve(x0, 0.0)
            lat2.append(time.perf_counter() - t)
        plain["single_K4096_N50_gate"] = {
            "solves_per_s": 1.0 / float(np.mean(lat2)), "p50_ms": float(np.percentile(lat2, 50) * 1e3),
            "p99_ms": float(np.percentile(lat2, 99) * 1e3),
            "value": 4096 * 50 / float(np.mean(lat2)), "unit": "rollout-steps/s"}
        c2.close()
        e2e["batched_vs_plain_solves_per_s"] = e2e["solves_per_s"] / plain["batch_one_solve_per_launch"]["solves_per_s"]
        # the paper's solve size (Table I: 8192 samples, horizon 20, dt 0.03,
        # lambda 0.01; 2048 samples onboard): host-synchronous mppi_solve
        # latency, and device time per solve back to back
        plain["paper_table1_single_solve"] = paper_table1_latency(M, W, args.table1_reps)

    # ---- closed-loop comparison of the objectives (Sec. V-A protocol) ----
    closed = None
    if not args.no_closed_loop and rank == 0:
        from paper_2509_14726_gb300 import closed_loop as CL
        tracks = {"circle_4_gates_r5": W.circle_track(4, 5.0), "figure8_8_gates": W.figure8_track(),
                  "course_7_gates_seed7": W.random_course(7)}
        closed = {"protocol": "3 laps, 50 Hz, K 4096, N 50; plant = the library's RK4 model; all start 1 m "
                              "before gate 0 (tracking on its 8 m/s reference); 60 s limit",
                  "runs": CL.comparison(tracks, laps=3, models=("ctbr", "rotor"), t_max=60.0)}

    # ---- serving: the configured fleet at its own rates, continuous batching vs plain ----
    serving_out = None
    if not args.no_serving and rank == 0:
        from paper_2509_14726_gb300 import serving as SV
        fleet = W.c5_fleet(2000)
        win = float(args.serve_seconds)
        sched = SV.make_schedule(fleet, duration_s=win, time_scale=1.0, K_choices=[1024, 4096, 16384],
                                 N_choices=[30, 50, 80], seed=0)
        # a request that has not started one control period after its arrival
        # is refused (its drone has moved on): offered = achieved + refused
        served = SV.run_served(fleet, sched, budget_bytes=40 << 30, n_slots=3, max_batch=512, deadline_periods=1.0)
        plain_s = SV.run_plain(fleet, sched, time_limit_s=win + 1.0, deadline_periods=1.0)
        sub = fleet[:200]
        sched_lo = SV.make_schedule(sub, duration_s=2.0, time_scale=0.1, K_choices=[1024, 4096, 16384],
                                    N_choices=[30, 50, 80], seed=0)
        keys = ("offered_per_s", "achieved_per_s", "refused_per_s", "p50_ms", "p99_ms", "rollout_steps_per_s")

        def brief(d, extra=()):
            return {k: (round(d[k], 4) if isinstance(d.get(k), float) else d.get(k)) for k in keys + tuple(extra)}
        lo_s, lo_p = SV.run_served(sub, sched_lo), SV.run_plain(sub, sched_lo, time_limit_s=4.0)
        serving_out = {
            "fleet": "2000 drones at 50/100/200 Hz (Poisson-jittered), K in {1024,4096,16384}, N in {30,50,80}, "
                     "5-9 gate courses, 40 GB scratch pool; deadline 1 control period",
            "window_s": win, "configured_window_s": 60.0,
            "window_note": "the arrival schedule replays in real time, once per path; 60 s per path would "
                           "add two minutes to the bench (--serve-seconds 60 runs it)",
            "served": brief(served, ("batches", "mean_batch")), "plain_one_solve_per_request": brief(plain_s),
            "one_gpu_over_capacity": served["refused_per_s"] > 0.01 * served["offered_per_s"],
            "low_load_200_drones_x0.1": {"served": brief(lo_s), "plain": brief(lo_p)}}

    cpu = None
    parity = None
    if rank == 0:
        parity = oracle_parity(items, M)
        cpu = cpu_baseline(items, args.cpu_sample_s, omp=True)
        single = cpu_baseline(items, max(1.0, args.cpu_sample_s / 3), omp=False)
        cpu["single_core"] = {"value": single["value"], "sample": single["sample"]}
        cpu["host"] = host_facts()

    if rank == 0:
        def r4(v):
            return round(float(v), 4) if isinstance(v, (float, np.floating)) else v

        closed_brief = None
        if closed is not None:
            closed_brief = {"protocol": closed["protocol"],
                            "runs": {k: (f"{r4(f['time_s'])} s, err {r4(f['waypoint_error_m'])} m"
                                         + (f", rmse {r4(f['tracking_rmse_m'])} m" if f["tracking_rmse_m"] else "")
                                         + ("" if f["completed"] else f", not finished ({f['gates_passed']} gates)"))
                                     for k, f in closed["runs"].items()}}
        tuning_brief = {"block": tuning["block"], "graph_mode": tuning["graph_mode"], "noise_gen": tuning["noise_gen"],
                        "spt": tuning["spt"],
                        "table_ms": [[t["block"], t["graph_mode"], t["noise_gen"], t["spt"], r4(t["ms"])]
                                     for t in (tuning["table"] or [])]}
        parity_brief = {k: parity[k] for k in ("bound_nominal", "bound_cost_rel", "literal_pass", "literal_miss",
                                                "max_rel_J", "max_abs_J", "max_dU", "decision_mismatches")}
        parity_brief["per_drone"] = [
            f"{p['drone']}: obj {p['objective']} K {p['K']} N {p['N']}: rel J {p['max_rel_J']:.2g} "
            f"(abs {p['max_abs_J']:.2g}), |dU| "
            f"{p['max_dU']:.3g}" + ("" if p["literal"] else f" > 1e-5, binary32 floor {p.get('binary32_floor') or 0:.3g}")
            for p in parity["per_drone"]]
        line = {
            "metric": "rollout-steps/s", "value": value, "unit": "rollout-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded gate courses, arc-length splines, 8 m/s references)",
            "config": {"workload": f"batched uneven MPPI solves: {len(items)} drones per GPU, K logU[1024,16384], "
                                   f"N U[20,80], dt 0.02, 5-9 gate courses, objectives 1/3 each, one CUDA graph; "
                                   f"a step is {R} consecutive batched solves of the fleet (control periods)",
                       "rollout_steps_per_step": R * steps_per_solve, "solves_per_step": R * len(items),
                       "l2": "working set (noise 16-20 B per rollout step, ~1.3 GB at 256 drones) larger than the 129 MB L2",
                       "parallelism": f"dp{world} (drones sharded, no collective)"},
            "solves_per_s": R * len(items) * world / (ms_max / 1e3),
            "gpu_launches": int(launches),
            "roofline": roofline, "e2e": e2e, "clocks": clocks, "cpu_baseline": cpu,
            "rotor_model_batch": rotor_out, "closed_loop": closed_brief, "tuning": tuning_brief,
            "plain": plain, "serving": serving_out, "parity_vs_oracle": parity_brief,
        }
        print(json.dumps(line), flush=True)
    M.mppi_batch_destroy(plan)
    for c in ctls:
        c.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
