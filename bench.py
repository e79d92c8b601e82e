"""Benchmark of the hybrid symplectic step on the 64k MMSN disk.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: 65536 equal-mass planetesimals (5 Earth masses on 0.5-4 AU,
Sigma ~ a^-1.5, e/i Rayleigh 0.01/0.005) plus Jupiter and Saturn analogues,
N = 65538 bodies, dt = 6 days, synthetic seeded initial conditions. One step
is the whole hot path: B(h/2) C(h/2) A(h) C(h/2) B(h/2) with the O(N^2) kick
and flags, encounter groups, Bulirsch-Stoer and the incremental force update.

Metric: pair interactions per second, N (N - 1) per step (one force
evaluation per step), FP64. The line also carries steps/s, the mixed-precision
kick's throughput, the roofline of the dominant kernel (the kick), the end-to-
end number through the C ABI with host buffers, the oracle on the host cores,
and the SM clocks sampled during the timed region.

Accuracy of the reduced-precision kicks on the same workload (its 1000-step
form): the literal mixed form and double-single run 100 and 1000 steps next to
an FP64 run from the same state and radii, and their state errors against it
are reported, with the error of each against the oracle after 100 steps. The
oracle's 100 steps are the run the CPU-baseline leg times (warm-up and timed
steps, the reference arm's sample), continued in a background thread on the
host cores while the GPU runs the other legs.

Under torchrun (N > 1) the ranks integrate one system together: every rank
holds the whole state and evaluates the O(N^2) kick for its own block of
target rows, and two NCCL all-gathers per step join the blocks (the row-
sharded step, nb_set_shard). The work is fixed as N grows (strong scaling);
the value is the job's pair interactions per second of the slowest rank's
time. At N > 1 the headline step and its end-to-end form are timed.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair interactions/s & steps/s at N=65536 (FP64, % peak); mixed vs FP64"
UNIT = "pair interactions/s"
WORKLOAD = "mmsn_64k_js"
FLOP_PER_PAIR = 20        # direct-summation convention (Nyland, Harris & Prins 2007)
FP64_INSTR_PER_PAIR = 7  # FP64 instructions per pair in the row kick's loop (FP64 mode)
# the unordered-pair kick: 9 FP64 instructions per pair {i, j} (r^-3 = y0^3 p with p
# on the integer pipe, the two mass scales, six FMAs), 4.5 per ordered pair
FP64_INSTR_PER_PAIR_SYM = 4.5
ACC_SHORT, ACC_LONG = 100, 1000  # steps of the accuracy leg (oracle comparison, long run)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--n", type=int, default=None, help="planetesimal count override (small runs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-options", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the 100/1000-step accuracy leg of the reduced-precision kicks")
    ap.add_argument("--batch-shape", default=None,
                    help="threads:chunk:tile_rows:buckets of the batched leg instead of the "
                         "autotuner's (profiling)")
    ap.add_argument("--batch-systems", type=int, default=4096,
                    help="systems of the batched leg (4096 is the workload; fewer for profiling)")
    ap.add_argument("--adjoint-steps", type=int, default=2000,
                    help="steps of the adjoint leg (2000 is the workload; fewer for profiling)")
    ap.add_argument("--adjoint-every", type=int, default=100, help="checkpoint interval")
    ap.add_argument("--resolution", action="store_true",
                    help="resolution study instead of the benchmark line: throughput vs N on the "
                         "16k disk family (N = 2048..65536 + Jupiter and Saturn), GPU and oracle "
                         "on 1 and on all host cores")
    ap.add_argument("--precision", choices=["fp64", "mixed", "ds"], default="fp64",
                    help="kick precision of the timed run (profiling); the line's value is fp64")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, world: int, device) -> float:
    """The largest of every rank's value (the slowest rank's time); the
    value itself on one rank."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_step: float, steps: int, max_ms: float) -> float:
    """Units the whole job processes (all ranks together: one sharded system)
    per second of the slowest rank."""
    return units_per_step * steps / (max_ms * 1e-3)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu),
                                       "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [q.strip() for q in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def read_traffic(path):
    """key: value lines of a profiles/ summary (comments start with #)."""
    out = {}
    if os.path.exists(path):
        for line in open(path):
            line = line.split("#", 1)[0].strip()
            if ":" in line:
                k, v = line.split(":", 1)
                out[k.strip()] = v.strip()
    return out


def pairs_per_step(n):
    return float(n) * float(n - 1)


def flush_l2(buf):
    buf.add_(1)  # 256 MiB read+write, larger than the 126 MB L2


# ------------------------------------------------------------------ oracle arms
def oracle_step_time(disk, steps: int, threads: int):
    """Wall time per step of the CPU oracle on `threads` host cores."""
    os.environ["OMP_NUM_THREADS"] = str(threads)
    from oracle import nbref
    nbref.set_threads(threads)
    p = nbref.params(dt_rcrit=disk.dt)
    s = nbref.RefSystem(p, disk.x, disk.v, disk.m, disk.R)
    t0 = time.perf_counter()
    st = s.step(steps, disk.dt)
    t1 = time.perf_counter()
    if st != 0:
        raise RuntimeError("oracle step failed: %d" % st)
    return (t1 - t0) / steps


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2604_09184_b300 import ics
    disk = ics.workload(args.workload, n=args.n)
    threads = os.cpu_count() or 1
    # each timed step is one full oracle step of the same workload
    os.environ["OMP_NUM_THREADS"] = str(threads)
    from oracle import nbref
    p = nbref.params(dt_rcrit=disk.dt)
    s = nbref.RefSystem(p, disk.x, disk.v, disk.m, disk.R)
    for _ in range(args.warmup):
        s.step(1, disk.dt)
    t0 = time.perf_counter()
    s.step(args.steps, disk.dt)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    v = pairs_per_step(disk.n) / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "n_bodies": disk.n,
                                        "dt_days": disk.dt, "precision": "fp64",
                                        "parallelism": "%d host threads (OpenMP)" % threads,
                                        "l2": "host run"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "%d full oracle steps of %s (N=%d)" % (args.steps,
                                                                           args.workload, disk.n)},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2604_09184_b300 import build, ics
    build.build()
    from paper_2604_09184_b300 import nb

    disk = ics.workload(args.workload, n=args.n)
    n = disk.n
    pps = pairs_per_step(n)

    # CPU baseline first (before any GPU work), rank 0 only: the reference arm's
    # sample (warm-up, then the timed steps) of the same workload
    cpu, oracle_run = None, None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, oracle_run = cpu_baseline_leg(disk, args)

    stream = torch.cuda.current_stream()
    f64_peak, f32_peak = nb.measure_peaks()

    prec = {"fp64": nb.NB_PREC_FP64, "mixed": nb.NB_PREC_MIXED, "ds": nb.NB_PREC_DS}[args.precision]
    p = nb.params(dt_rcrit=disk.dt, precision=prec)
    sysm = nb.NBodySystem(p, disk.x, disk.v, disk.m, disk.R)
    sharding = None
    if world > 1:
        # one system on all ranks: the kick's target rows split across them
        from paper_2604_09184_b300 import shard
        sharding = shard.Shard(sysm, rank, world)
        for k in ("no_cpu", "no_mixed", "no_batch", "no_adjoint", "no_options", "no_accuracy"):
            setattr(args, k, True)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(max(args.warmup, 0)):
        sysm.step(1, disk.dt)
    sysm.set_timing(True)
    launches0 = sysm.timing()["launches"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush_l2(flush)
        ev[k][0].record(stream)
        sysm.step(1, disk.dt)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    tm = sysm.timing()
    gpu_launches = tm["launches"] - launches0
    total_ms = max_over_ranks(total_ms, world, "cuda")
    ms_per_step = total_ms / max(args.steps, 1)
    value = job_rate(pps, args.steps, total_ms)
    kick_ms = tm["kick_ms"] / max(tm["kick_launches"], 1)
    st = sysm.stats()

    # ordered pairs one launch of this rank's kick evaluates: its target rows
    # against all bodies (every row on one GPU)
    kick_pairs = pps if sharding is None else float(sharding.row1 - sharding.row0) * (n - 1)
    achieved = FLOP_PER_PAIR * kick_pairs / (kick_ms * 1e-3)
    sym = bool(st.get("kick_symmetric", 0))
    ipp = FP64_INSTR_PER_PAIR_SYM if sym else FP64_INSTR_PER_PAIR
    roofline = {
        "bound": "alu", "achieved": achieved / 1e12, "peak": f64_peak / 1e12, "unit": "TFLOP/s",
        "frac": achieved / f64_peak, "traffic": None,
        "kernel": "k_kick_sym" if sym else "k_kick<FP64>", "kick_ms": kick_ms,
        "flop_per_pair": FLOP_PER_PAIR,
        "peak_source": "FP64 DFMA loop measured in this run (nb_measure_peaks)",
        "fp64_pipe_frac_by_count": ipp * kick_pairs / (kick_ms * 1e-3) / (f64_peak / 2),
        "fp64_instr_per_pair_design": ipp,
        "fp32_peak_tflops": f32_peak / 1e12,
        "note": "achieved counts 20 flop per ordered pair (the direct-summation convention); "
                "the kick forms dx, dy, dz and r^2 on the integer pipe (exact fixed-point "
                "differences)%s, so its FP64 pipe executes ~%g FP64 instructions per ordered "
                "pair and the conventional rate can exceed the DFMA peak; fp64_pipe_frac is the "
                "FP64 pipe's busy share measured by ncu on one launch of this kernel at this N"
                % (", evaluates each unordered pair once for both bodies and forms r^-3's "
                   "residual and series on the integer pipe too" if sym else "", ipp),
    }
    prof = "kick_sym_mmsn_64k" if sym else "kick_fp64_mmsn_64k"
    tr = read_traffic(os.path.join(ROOT, "profiles", prof + "_dram.txt"))
    # the profiles describe a whole-system launch; a rank's row block is not one
    if tr.get("n") == str(n) and sharding is None:
        roofline["traffic"] = float(tr["bytes_per_launch"])
        roofline["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum, 1 "
                                      "launch, profiles/%s_dram.txt" % prof)
    # pipe shares measured by ncu (one launch of each kick at this N), not asserted
    pf = read_traffic(os.path.join(ROOT, "profiles", prof + "_pipes.txt"))
    if pf.get("n") == str(n) and sharding is None:
        roofline["fp64_pipe_frac"] = float(pf["fp64_pipe_pct"]) / 100
        roofline["alu_pipe_frac"] = float(pf["alu_pipe_pct"]) / 100
        roofline["issue_active_frac"] = float(pf["issue_active_pct"]) / 100
        roofline["fp64_instr_per_pair"] = float(pf["fp64_inst_per_pair"])
        roofline["pipes_source"] = ("ncu sm__pipe_fp64_cycles_active, sm__pipe_alu_cycles_active, "
                                    "sm__issue_active (% of peak sustained active) and "
                                    "sm__inst_executed_pipe_fp64.sum, profiles/"
                                    + prof + "_pipes.txt")
    # the drift's HBM figures (ncu at this N): algorithmic bytes over its time
    dr = read_traffic(os.path.join(ROOT, "profiles", "drift_mmsn_64k.txt"))
    if dr.get("n") == str(n):
        t_us = float(dr["gpu_time_us"])
        hbm = load_peaks().get("hbm_gbs")
        roofline["drift"] = {
            "kernel": dr["kernel"], "bound": "fp64", "gpu_time_us": t_us,
            "algorithmic_bytes": int(dr["algorithmic_bytes"]),
            "achieved_gbs": int(dr["algorithmic_bytes"]) / (t_us * 1e3),
            "hbm_frac": int(dr["algorithmic_bytes"]) / (t_us * 1e3) / hbm if hbm else None,
            "dram_bytes": int(dr["dram_bytes_read"]) + int(dr["dram_bytes_write"]),
            "fp64_pipe_frac": float(dr["fp64_pipe_pct"]) / 100,
            "source": "ncu, 3 launches, profiles/drift_mmsn_64k.txt (HBM peak: "
                      "MEASURED_PEAKS.json hbm_gbs)"}
    if args.precision == "ds":
        ds = ds_pipes(n, "k_kick_ds_sym" if sym else "k_kick_ds")
        if ds:
            roofline["double_single"] = ds
    if args.precision != "fp64":
        # the line's kick is the reduced-precision one: the FP64 kernel's pipe
        # shares and traffic do not describe it
        for k in ("fp64_pipe_frac", "alu_pipe_frac", "issue_active_frac", "fp64_instr_per_pair",
                  "pipes_source", "traffic_source", "fp64_pipe_frac_by_count",
                  "fp64_instr_per_pair_design"):
            roofline.pop(k, None)
        roofline["traffic"] = None
        roofline["kernel"] = (("k_kick_ds_sym" if sym else "k_kick_ds") if args.precision == "ds"
                              else "k_kick<MIXED>")
        roofline["note"] = ("achieved counts 20 flop per pair (the direct-summation convention) "
                            "against the FP64 DFMA peak, for comparison with the FP64 line")
        if args.precision == "ds" and "double_single" in roofline:
            ds = roofline.pop("double_single")
            roofline.update({k: ds[k] for k in ("fp32_pipe_frac", "fp64_pipe_frac",
                                                "issue_active_frac", "inst_per_pair")})
            roofline["pipes_source"] = ds["source"]

    # reduced-precision kicks on the same workload: the literal mixed mode
    # (float seed + one FP64 Newton step) and double-single on the FP32 pipe
    mixed = None
    if not args.no_mixed:
        mixed = {"mixed": run_variant(nb, torch, disk, args, nb.NB_PREC_MIXED, ms_per_step,
                                      kick_ms, pps, flush, stream),
                 "double_single": run_variant(nb, torch, disk, args, nb.NB_PREC_DS, ms_per_step,
                                              kick_ms, pps, flush, stream)}
        ds = ds_pipes(n, mixed["double_single"]["kernel"])
        if ds:
            roofline["double_single"] = ds
        mixed["note"] = (
            "the literal mixed form (FP32 rsqrt seed + one FP64 Newton step, a row kick) gives "
            "%.2fx per kick against the FP64 kick on B300: the FP64 kick already takes r^-3 "
            "from an FP32 seed, forms dx, dy, dz, r^2 and r^-3's residual series on the integer "
            "pipe and (from N = 4096) evaluates each pair once for both bodies, 4.5 FP64 "
            "instructions per ordered pair, while the mixed form removes one of the row kick's "
            "7. Double-single (float-pair arithmetic on the FP32 pipe) is the form that gives "
            "a speed-up: %.2fx per kick, %.2fx per step" % (
                mixed["mixed"]["speedup_kick"], mixed["double_single"]["speedup_kick"],
                mixed["double_single"]["speedup_step"]))

    batched = None
    if not args.no_batch:
        batched = run_batched(nb, torch, args, flush, stream, n_systems=args.batch_systems,
                              f64_peak=f64_peak)

    # the step with the start-of-step options of the non-Newtonian row on:
    # gas drag at both ends of the step and the ejection scan
    options = None
    if not args.no_options:
        options = run_options(nb, torch, disk, args, ms_per_step, flush, stream)

    adjoint = None
    if not args.no_adjoint:
        adjoint = run_adjoint(nb, torch, stream, args.adjoint_steps, args.adjoint_every)

    # end to end through the C ABI with host buffers: per step, load the state
    # from pinned host memory, step, read the state back to pinned host memory
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(nb, torch, sysm, disk, args.steps, pps, world)

    # accuracy of the reduced-precision kicks (untimed; last, so that the oracle
    # thread it starts overlaps no timed leg)
    accuracy = None
    if not args.no_accuracy and world == 1:
        del sysm
        accuracy = run_accuracy(nb, disk, oracle_run)
        if mixed is not None:
            for key in ("mixed", "double_single"):
                mixed[key].update(accuracy.pop(key))

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "steps_per_s": 1e3 / ms_per_step,
        "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n_bodies": n, "dt_days": disk.dt,
                   "precision": args.precision,
                   "parallelism": ("row-sharded kick over %d GPUs (rows %d..%d on rank 0), two "
                                   "NCCL all-gathers per step" % (world, sharding.row0,
                                                                  sharding.row1)
                                   if sharding else "1 GPU"),
                   "l2": "flushed before each timed step (256 MiB write, outside the step events)"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "mixed": mixed,
        "accuracy": accuracy,
        "batched": batched, "adjoint": adjoint, "options": options,
        "clocks": clk, "gpu_launches": gpu_launches,
        "encounters": {"pairs": st["encounter_pairs"], "groups": st["groups"],
                       "bs_substeps": st["bs_substeps"], "merges": st["merges"],
                       "steps_total": st["steps"]},
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def cpu_baseline_leg(disk, args):
    """The oracle on all host cores over the sample the reference arm times
    (args.warmup untimed steps, then args.steps timed full steps of the
    workload, from the same initial state). Returns the cpu_baseline entry and
    the oracle run, whose state and encounter log the accuracy leg continues
    to ACC_SHORT steps."""
    import threading  # noqa: F401  (the continuation runs in a thread)
    from oracle import nbref
    threads = os.cpu_count() or 1
    os.environ["OMP_NUM_THREADS"] = str(threads)
    nbref.set_threads(threads)
    p = nbref.params(dt_rcrit=disk.dt)
    s = nbref.RefSystem(p, disk.x, disk.v, disk.m, disk.R)
    rc0 = s.state()["rc"]
    logs = []
    if args.warmup > 0:
        if s.step(args.warmup, disk.dt) != 0:
            raise RuntimeError("oracle step failed")
        logs.append(s.encounter_list())
    t0 = time.perf_counter()
    if s.step(args.steps, disk.dt) != 0:
        raise RuntimeError("oracle step failed")
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    logs.append(s.encounter_list())
    cpu = {"value": pairs_per_step(disk.n) / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": "%d full oracle steps of %s (N=%d) after %d untimed, %d OpenMP threads, "
                     "%.2f s per step (the reference arm's sample)" % (
                         args.steps, args.workload, disk.n, args.warmup, threads, dt)}
    return cpu, {"sys": s, "logs": logs, "rc": rc0, "threads": threads, "nbref": nbref}


def _state_err(a, b, enc=None):
    """Relative position error of state a against state b over their common
    ids: max, median, bodies above 1e-12, and whether the id sets agree. With
    b's encounter log enc ((step, id_i, id_j) rows) also the same split into
    bodies that entered an encounter and the quiet rest: the 1e-12 bar holds
    for the quiet bodies, while a direct-solver integration through an
    encounter amplifies rounding (the parity tests bound those bodies by the
    oracle's own spread under 1-ulp input changes)."""
    common, ia, ib = np.intersect1d(a["ids"], b["ids"], return_indices=True)
    rel = np.linalg.norm(a["x"][ia] - b["x"][ib], axis=1) / np.linalg.norm(b["x"][ib], axis=1)
    out = {"max": float(rel.max()), "median": float(np.median(rel)),
           "bodies_above_1e-12": int((rel > 1e-12).sum()), "bodies": int(len(rel)),
           "ids_identical": bool(len(a["ids"]) == len(b["ids"]) == len(common))}
    if enc is not None:
        met = np.isin(common, np.asarray(enc)[:, 1:].reshape(-1)) if len(enc) else \
            np.zeros(len(rel), bool)
        out["encounter_bodies"] = int(met.sum())
        out["encounter_bodies_above_1e-12"] = int((rel[met] > 1e-12).sum())
        out["quiet_max"] = float(rel[~met].max()) if (~met).any() else 0.0
    return out


def run_accuracy(nb, disk, oracle_run):
    """The workload in FP64, in the literal mixed form and in double-single
    from the same state and critical radii: ACC_SHORT and ACC_LONG steps each.
    Errors of the reduced-precision runs against the FP64 run at both counts,
    and of all three against the oracle at ACC_SHORT (the oracle run of the
    CPU-baseline leg, continued meanwhile in a background thread)."""
    import threading
    from paper_2604_09184_b300 import nb as nbm
    rc = None
    th = None
    orc = None
    if oracle_run is not None:
        rc = oracle_run["rc"]
        s, nbref = oracle_run["sys"], oracle_run["nbref"]
        done = s.step_index
        if done <= ACC_SHORT:
            def rest():
                # leave cores to the GPU launches meanwhile (results do not
                # depend on the thread count)
                nbref.set_threads(max(oracle_run["threads"] - 2, 1))
                if done < ACC_SHORT:
                    s.step(ACC_SHORT - done, disk.dt)
                    oracle_run["logs"].append(s.encounter_list())
            th = threading.Thread(target=rest)
            th.start()
    runs = {}
    for name, prec in (("fp64", nbm.NB_PREC_FP64), ("mixed", nbm.NB_PREC_MIXED),
                       ("double_single", nbm.NB_PREC_DS)):
        g = nb.NBodySystem(nb.params(dt_rcrit=disk.dt, precision=prec), disk.x, disk.v, disk.m,
                           disk.R, rc=rc)
        g.step(ACC_SHORT, disk.dt)
        s100, e100 = g.state(), g.encounter_list()
        g.step(ACC_LONG - ACC_SHORT, disk.dt)
        runs[name] = (s100, e100, g.state(), g.stats())
        del g
    if th is not None:
        th.join()
        sref = oracle_run["sys"].state()
        eref = np.concatenate([q for q in oracle_run["logs"] if len(q)]) if any(
            len(q) for q in oracle_run["logs"]) else np.zeros((0, 3), np.int32)
        orc = (sref, eref)
    out = {"workload": "%s, %d and %d steps from the initial state" % (disk.name, ACC_SHORT,
                                                                       ACC_LONG)}
    f100, fe100, f1000, fst = runs["fp64"]
    if orc is not None:
        out["fp64"] = {"err_oracle_%d" % ACC_SHORT: _state_err(f100, orc[0], orc[1]),
                       "encounters_identical_oracle_%d" % ACC_SHORT: bool(
                           np.array_equal(fe100, orc[1]))}
    for name in ("mixed", "double_single"):
        s100, e100, s1000, st = runs[name]
        r = {"err_state_%d" % ACC_SHORT: _state_err(s100, f100),
             "err_state_%d" % ACC_LONG: _state_err(s1000, f1000),
             "encounters_identical_fp64_%d" % ACC_SHORT: bool(np.array_equal(e100, fe100)),
             "merges_%d" % ACC_LONG: st["merges"], "merges_fp64_%d" % ACC_LONG: fst["merges"]}
        if orc is not None:
            r["err_oracle_%d" % ACC_SHORT] = _state_err(s100, orc[0], orc[1])
            r["encounters_identical_oracle_%d" % ACC_SHORT] = bool(np.array_equal(e100, orc[1]))
        r["bound"] = ("per-body kick error <= 1e-10 |a_i| against the FP64 kick and the oracle "
                      "(tests); the state errors are set by the encounters' amplification of "
                      "that difference, to be read against the FP64 run's own oracle error")
        out[name] = r
    return out


def ds_pipes(n, kernel):
    """The double-single kick's pipe shares at this N from its ncu capture in
    profiles/ (one launch, each metric 1 pass), or None."""
    name = "kick_ds_sym_mmsn_64k_pipes.txt" if kernel == "k_kick_ds_sym" else \
        "kick_ds_mmsn_64k_pipes.txt"
    pd = read_traffic(os.path.join(ROOT, "profiles", name))
    if pd.get("n") != str(n) or pd.get("kernel") != kernel:
        return None
    return {"kernel": kernel, "bound": "issue",
            "fp32_pipe_frac": float(pd["fma_pipe_pct"]) / 100,
            "fp64_pipe_frac": float(pd["fp64_pipe_pct"]) / 100,
            "issue_active_frac": float(pd["issue_active_pct"]) / 100,
            "inst_per_pair": float(pd["inst_per_pair"]),
            "source": "ncu sm__pipe_fma_cycles_active (the FP32 FMA pipes), "
                      "sm__pipe_fp64_cycles_active, sm__issue_active, smsp__inst_executed.sum, "
                      "one launch, profiles/" + name}


def run_variant(nb, torch, disk, args, precision, ms64, kick64, pps, flush, stream):
    """Same timed loop with another kick precision; accuracy of its kick against
    the FP64 kick on the initial state."""
    pm = nb.params(dt_rcrit=disk.dt, precision=precision)
    sm = nb.NBodySystem(pm, disk.x, disk.v, disk.m, disk.R)
    # the initial force of this system and of an FP64 one: the kernels the steps run
    a_var, p_var = sm.fsal()
    sym = bool(sm.stats()["kick_symmetric"])
    s64 = nb.NBodySystem(nb.params(dt_rcrit=disk.dt), disk.x, disk.v, disk.m, disk.R)
    a64, p64 = s64.fsal()
    del s64
    for _ in range(max(args.warmup, 0)):
        sm.step(1, disk.dt)
    sm.set_timing(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush_l2(flush)
        ev[k][0].record(stream)
        sm.step(1, disk.dt)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / max(args.steps, 1)
    tm = sm.timing()
    kms = tm["kick_ms"] / max(tm["kick_launches"], 1)
    del sm
    rel = np.linalg.norm(a_var - a64, axis=1) / np.linalg.norm(a64, axis=1)
    same_flags = sorted(map(tuple, p64.tolist())) == sorted(map(tuple, p_var.tolist()))
    kernel = {nb.NB_PREC_MIXED: "k_kick<MIXED>",
              nb.NB_PREC_DS: "k_kick_ds_sym" if sym else "k_kick_ds"}[precision]
    return {"value": pps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "kick_ms": kms,
            "kernel": kernel, "speedup_step": ms64 / ms, "speedup_kick": kick64 / kms,
            "max_rel_err_accel_vs_fp64": float(rel.max()),
            "median_rel_err_accel_vs_fp64": float(np.median(rel)), "flags_identical": same_flags,
            "accel_compared": "initial force of the system in this precision against that of "
                              "the FP64 system (the kernels the steps run)"}


def run_batched(nb, torch, args, flush, stream, n_systems=4096, dt=3.0, sample=32, f64_peak=None):
    """The 4096-system ensemble (N log-uniform in [16, 512]): per step an
    opening, a tiled kick and a closing launch over all systems, replayed from
    a captured graph in the autotuned shape; speedup against integrating the
    same systems one at a time through the single-system path, estimated on a
    random sample of systems."""
    from paper_2604_09184_b300 import ics
    disks = ics.ensemble(n_systems=n_systems)
    pairs = float(sum(d.n * (d.n - 1) for d in disks))
    b = nb.NBodyBatch(nb.params(dt_rcrit=dt), disks)
    if args.batch_shape:
        t_, c_, r_, k_ = (int(q) for q in args.batch_shape.split(":"))
        b.set_shape(t_, c_)
        b.set_schedule(r_, k_)
    else:
        b.autotune(dt)
    shape = b.shape()  # threads, steps per graph chunk, kick tile rows, buckets
    threads, chunk = shape["threads"], shape["chunk"]
    for _ in range(max(args.warmup, 0)):
        b.step(1, dt)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush_l2(flush)
        ev[k][0].record(stream)
        b.step(1, dt)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms_call = sum(a.elapsed_time(c) for a, c in ev) / max(args.steps, 1)
    # production use: many steps per call, replayed from the captured graph
    flush_l2(flush)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b.step(chunk, dt)  # capture the chunk's graph outside the timed call
    torch.cuda.synchronize()
    flush_l2(flush)
    e0.record(stream)
    b.step(2 * chunk, dt)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / (2 * chunk)
    bal = b.balance()  # the last close launch
    st = b.stats()
    sym = bool(st.get("kick_symmetric", 0))
    del b
    # single-system path on a random sample of the same systems
    rng = np.random.default_rng(7)
    pick = rng.choice(n_systems, size=min(sample, n_systems), replace=False)
    t_single = []
    for k in pick:
        d = disks[int(k)]
        s1 = nb.NBodySystem(nb.params(dt_rcrit=dt), d.x, d.v, d.m, d.R)
        s1.step(1, dt)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(3):
            s1.step(1, dt)
        e1.record(stream)
        torch.cuda.synchronize()
        t_single.append(e0.elapsed_time(e1) / 3)
        del s1
    single_ms = float(np.mean(t_single)) * n_systems
    return {"workload": "ensemble_4096 (N log-uniform 16..512, dt 3 d)", "systems": n_systems,
            "pairs_per_step": pairs, "value": pairs / (ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms, "steps_per_s": 1e3 / ms,
            "autotuned_shape": {"threads_per_cta": threads, "steps_per_graph": chunk,
                                "kick_tile_rows": None if sym else shape["tile_rows"],
                                "buckets": shape["buckets"],
                                "schedule": "per step and bucket (every k-th system of the "
                                            "largest-first order, its own stream): open (per "
                                            "system), kick (%s), close (per system)" % (
                                                "one warp per 32-body block pair of one "
                                                "system, each pair once for both bodies" if sym
                                                else "tiles of %d rows of one system"
                                                % shape["tile_rows"])},
            "timing": "one call of 2 graph replays of the autotuned chunk, L2 flushed before",
            "ms_per_step_one_call_per_step": ms_call,
            "single_system_path_ms_per_step_est": single_ms, "speedup_vs_single": single_ms / ms,
            "speedup_vs_single_one_call_per_step": single_ms / ms_call,
            "single_sample": int(len(pick)), "bs_substeps": st["bs_substeps"],
            "load_balance": {"efficiency": bal["efficiency"], "ctas": bal["ctas"],
                             "max_cta_ms": bal["max_cta_ms"],
                             "definition": "sum of CTA busy times / (CTAs x longest), the last "
                                           "close launch"},
            "groups": st["groups"], "merges": st["merges"],
            "roofline": batched_roofline(pairs, ms, f64_peak, sym)}


def batched_roofline(pairs, ms, f64_peak, sym):
    """The ensemble step against the FP64 pipe: the kick's FP64 instructions
    per ordered pair (4.5 for the unordered-pair kick, 7 for the row kick; dx,
    dy, dz and r^2 on the integer pipe, as in the single-system kicks) at the
    step's rate, over the DFMA peak measured in the same run; and the kick's
    own FP64 pipe share in one launch (ncu, profiles/)."""
    ipp = FP64_INSTR_PER_PAIR_SYM if sym else FP64_INSTR_PER_PAIR
    kernel = "k_batch_kick_sym" if sym else "k_batch_kick<32, 32>"
    out = {"bound": "alu", "kernel": kernel, "fp64_instr_per_pair_design": ipp}
    if f64_peak:
        out["fp64_pipe_frac_by_count_step"] = ipp * pairs / (ms * 1e-3) / (f64_peak / 2)
        out["peak_source"] = "FP64 DFMA loop measured in this run (nb_measure_peaks)"
    name = "batch_kick_sym_ensemble_4096_pipes.txt" if sym else \
        "batch_kick_ensemble_4096_pipes.txt"
    pb = read_traffic(os.path.join(ROOT, "profiles", name))
    if pb.get("systems") == "4096" and pb.get("kernel") == kernel:
        out["kick_fp64_pipe_frac"] = float(pb["fp64_pipe_pct"]) / 100
        out["kick_fp64_instr_per_lane_pair"] = float(pb["fp64_inst_per_lane_pair"])
        out["kick_ms_one_launch"] = float(pb["gpu_time_ms"])
        out["pipes_source"] = ("ncu sm__pipe_fp64_cycles_active and sm__inst_executed_pipe_fp64.sum, "
                               "one launch of the whole ensemble's kick, profiles/" + name)
    return out


def run_options(nb, torch, disk, args, ms_plain, flush, stream, steps=3):
    """The same step with gas drag (nominal nebula density) and ejection beyond
    100 AU switched on; reports the step time and its overhead."""
    s = nb.NBodySystem(nb.params(dt_rcrit=disk.dt, gas=1, eject_r=100.0), disk.x, disk.v,
                       disk.m, disk.R)
    for _ in range(max(args.warmup, 1)):
        s.step(1, disk.dt)
    ms = []
    for _ in range(steps):
        flush_l2(flush)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(1, disk.dt)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    st = s.stats()
    del s
    t = sum(ms) / len(ms)
    out = {"gas_drag_and_ejection_ms_per_step": t, "plain_ms_per_step": ms_plain,
           "overhead_ms": t - ms_plain, "ejections": st["ejections"],
           "setting": "gas rho0 = 2.36e-3 Msun/AU^3 (1.4e-9 g/cm^3) s^-2.75, eta 2e-3, C_D 1; "
                      "eject_r 100 AU; %d steps after %d warm-up" % (steps, max(args.warmup, 1))}
    # multi-level changeover on the encounter-dominated 2049-body disk
    from paper_2604_09184_b300 import ics
    d2 = ics.workload("adjoint_2k_j")
    ml = []
    for L in (0, 1, 2):
        s = nb.NBodySystem(nb.params(dt_rcrit=d2.dt, ml_levels=L, ml_factor=3, merge=0), d2.x,
                           d2.v, d2.m, d2.R)
        E0 = s.energy_momentum()["E"]
        s.step(2, d2.dt)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(200, d2.dt)
        e1.record(stream)
        torch.cuda.synchronize()
        st = s.stats()
        ml.append({"ml_levels": L, "ml_factor": 3, "ms_per_step": e0.elapsed_time(e1) / 200,
                   "energy_error": abs(s.energy_momentum()["E"] / E0 - 1),
                   "bs_derivs": st["bs_derivs"], "ml_substeps": st["ml_substeps"]})
        del s
    out["multilevel"] = {"workload": "adjoint_2k_j (2049 bodies), 202 steps, mergers off",
                         "runs": ml}
    return out


def run_adjoint(nb, torch, stream, nsteps=2000, every=100, fd_steps=100, fd_coords=32):
    """Gradient of the adjoint workload's loss (the sum of |x|^2 over 16 tagged
    bodies plus the final total energy, Eqs. Ha-Hc) on the 2048-planetesimal
    disk with Jupiter (2000 steps of 6 d) with respect to the initial x, v, m:
    checkpointed forward, then the backward pass (segment replays plus the
    adjoint kernels), both timed with CUDA events on the library's stream,
    state and cotangents on the device. The energy's cotangent comes from
    nb_energy_grad. Its error: the same gradient over fd_steps steps against
    central differences of the forward map (nb_step, bit-identical to the
    adjoint's forward) on fd_coords sampled entries, two step sizes each."""
    from paper_2604_09184_b300 import ics
    disk = ics.workload("adjoint_2k_j")
    rc = nb_rc_initial(nb, disk)
    n = disk.n
    tagged = 16
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")  # noqa: E731
    dev = [cu(q) for q in (disk.x, disk.v, disk.m, disk.R, rc)]

    def cotangent(adj):
        st = adj.state()
        gx, gv, gm = nb.energy_grad(st["x"], st["v"], st["m"], st["alive"])
        gx[:tagged] += 2.0 * st["x"][:tagged]
        return gx, gv, gm

    a = nb.NBodyAdjoint(nb.params(dt_rcrit=disk.dt), *dev, nsteps, every)
    # warm-up on a short run
    a.forward(disk.dt, nsteps=every)
    a.backward(*cotangent(a))
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(stream)
    a.forward(disk.dt)
    e[1].record(stream)
    g = cotangent(a)
    e[2].record(stream)
    dx, dv, dm = a.backward(*g)
    e[3].record(stream)
    torch.cuda.synchronize()
    fwd_ms, bwd_ms = e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])
    ok = bool(torch.isfinite(dx).all() and torch.isfinite(dv).all() and torch.isfinite(dm).all())
    ckpt = (nsteps // every + 2) * (13 * n * 8 + n * 4)
    del a
    fd = adjoint_fd_error(nb, torch, disk, rc, dev, cotangent, fd_steps, fd_coords, tagged)
    return {"workload": "adjoint_2k_j (2048 planetesimals + Jupiter, dt 6 d)", "n_bodies": n,
            "steps": nsteps, "checkpoint_every": every,
            "loss": "sum of |x_T|^2 over the first %d bodies + total energy E_T (Eqs. Ha-Hc); "
                    "gradients w.r.t. all initial x, v, m" % tagged,
            "forward_ms": fwd_ms, "backward_ms": bwd_ms,
            "backward_over_forward": bwd_ms / fwd_ms,
            "forward_ms_per_step": fwd_ms / nsteps, "backward_ms_per_step": bwd_ms / nsteps,
            "gradient_steps_per_s": nsteps / (bwd_ms * 1e-3), "checkpoint_bytes": ckpt,
            "finite": ok, "err_vs_fd": fd,
            "timing": "CUDA events on the library's stream around nb_adjoint_forward and around "
                      "nb_adjoint_backward (device cotangents and gradients, no host copies)"}


def adjoint_fd_error(nb, torch, disk, rc, dev, cotangent, steps, ncoord, tagged):
    """Adjoint gradient of the same loss over `steps` steps against central
    differences of the forward map: per sampled entry the differences at two
    step sizes (1e-6 and 1e-7 relative; 1e-2 and 1e-3 for masses), the error of
    the smaller against the adjoint, over their spread plus 1e-7 of the
    gradient's scale (as in the tests)."""
    a = nb.NBodyAdjoint(nb.params(dt_rcrit=disk.dt), *dev, steps, 25)
    a.forward(disk.dt)
    grads = [t.cpu().numpy() for t in a.backward(*cotangent(a))]
    del a

    def loss(x, v, m):
        s = nb.NBodySystem(nb.params(dt_rcrit=disk.dt), x, v, m, disk.R, rc=rc)
        s.step(steps, disk.dt)
        st = s.state()
        tag = st["ids"] < tagged
        q = s.stats()
        ev = (q["groups"], q["bs_substeps"], q["merges"], q["encounter_pairs"])
        return float((st["x"][tag] ** 2).sum() + s.energy_momentum()["E"]), ev

    arrays = (disk.x, disk.v, disk.m)
    _, ev0 = loss(*arrays)
    rng = np.random.default_rng(17)
    worst, ratios, changed = 0.0, [], []
    for _ in range(ncoord):
        k = int(rng.integers(0, 3))
        idx = tuple(int(rng.integers(0, q)) for q in arrays[k].shape)
        f, same = [], True
        for rel in ((1e-2, 1e-3) if k == 2 else (1e-6, 1e-7)):
            h = rel * abs(arrays[k][idx]) or 1e-9
            plus = [q.copy() for q in arrays]
            minus = [q.copy() for q in arrays]
            plus[k][idx] += h
            minus[k][idx] -= h
            (lp, ep), (lm, em) = loss(*plus), loss(*minus)
            f.append((lp - lm) / (2 * h))
            same = same and ep == ev0 and em == ev0
        scale = float(np.abs(grads[k]).max())
        err = abs(f[1] - grads[k][idx])
        if same:
            worst = max(worst, err / (abs(f[0] - f[1]) + 1e-7 * scale))
            ratios.append(err / scale)
        else:
            changed.append(err / scale)
    return {"steps": steps, "entries": ncoord, "entries_same_events": len(ratios),
            "worst_err_over_bound": worst,
            "median_err_of_scale": float(np.median(ratios)) if ratios else None,
            "max_err_of_scale": float(np.max(ratios)) if ratios else None,
            "entries_other_events": len(changed),
            "max_err_of_scale_other_events": float(np.max(changed)) if changed else None,
            "reference": "central differences of nb_step (the adjoint's forward map, bit for bit); "
                         "bound = spread of the two step sizes + 1e-7 of the gradient's scale; "
                         "entries whose +-h runs took another direct-solver decision (group, "
                         "accepted substeps, merger) are reported apart"}


def nb_rc_initial(nb, disk):
    s = nb.NBodySystem(nb.params(dt_rcrit=disk.dt), disk.x, disk.v, disk.m, disk.R)
    rc = s.state()["rc"]
    del s
    return rc


def run_e2e(nb, torch, sysm, disk, steps, pps, world=1):
    """The headline step end to end through the C ABI with host buffers. On
    a row-sharded system every rank loads the same state and steps it (the
    step's all-gathers join the ranks); the slowest rank's time counts."""
    n = disk.n
    st = sysm.state()
    a, pairs = sysm.fsal()
    pin = lambda arr: torch.from_numpy(np.ascontiguousarray(arr)).pin_memory()  # noqa: E731
    hx, hv, hm, hR, hrc = pin(st["x"]), pin(st["v"]), pin(st["m"]), pin(st["R"]), pin(st["rc"])
    hid = pin(st["ids"].astype(np.int32))
    ha = pin(a[:n])
    hp = pin(pairs.astype(np.int32).reshape(-1, 2))
    ox, ov, om, oR, orc = (torch.empty_like(t).pin_memory() for t in (hx, hv, hm, hR, hrc))
    oid = torch.empty_like(hid).pin_memory()
    import ctypes as C
    L = nb.lib()
    k = C.c_int()
    h2d = sum(t.numel() * t.element_size() for t in (hx, hv, hm, hR, hrc, hid, ha, hp))
    d2h = sum(t.numel() * t.element_size() for t in (ox, ov, om, oR, orc, oid))
    if sysm.n != n:
        return None
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    err = None
    for _ in range(steps):
        rcode = L.nb_set_state(sysm._h, C.c_void_p(hx.data_ptr()), C.c_void_p(hv.data_ptr()),
                               C.c_void_p(hm.data_ptr()), C.c_void_p(hR.data_ptr()),
                               C.c_void_p(hrc.data_ptr()), C.c_void_p(hid.data_ptr()),
                               C.c_void_p(ha.data_ptr()), C.c_void_p(hp.data_ptr()),
                               int(hp.shape[0]), 0)
        if not rcode:
            rcode = L.nb_step(sysm._h, 1, disk.dt)
        if not rcode:
            rcode = L.nb_get_state(sysm._h, C.c_void_p(ox.data_ptr()), C.c_void_p(ov.data_ptr()),
                                   C.c_void_p(om.data_ptr()), C.c_void_p(oR.data_ptr()),
                                   C.c_void_p(orc.data_ptr()), C.c_void_p(oid.data_ptr()),
                                   C.byref(k), 0)
        if rcode:
            err = nb.status_string(rcode)
            break
    torch.cuda.synchronize()
    t = max_over_ranks((time.perf_counter() - t0) / max(steps, 1), world, "cuda")
    if err:
        return {"error": err}
    return {"value": pps / t, "unit": UNIT, "ms_per_step": t * 1e3,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "api": "nb_set_state (pinned host) + nb_step(1) + nb_get_state (pinned host)"}


def run_resolution(args, sizes=(2048, 4096, 8192, 16384, 32768, 65536), max_n_1core=32768):
    """Throughput vs N on the paper's resolution-study disk (0.5-4 AU, 5 Earth
    masses, Jupiter and Saturn; the planetesimal count varies, the disk mass
    does not), with the paper's speed ratios (GPU vs 1 and vs 16 CPU cores,
    GENGA on an RTX 4070 Ti or P100 vs a Ryzen 9 7950X3D) quoted as context.
    The oracle runs first, on all host cores and on one (one full step each;
    one core only up to max_n_1core bodies, larger N would take minutes)."""
    import torch
    from paper_2604_09184_b300 import build, ics
    cores = os.cpu_count() or 1
    rows = []
    for n in sizes:
        d = ics.workload("mmsn_16k_js", n=n)
        row = {"n_bodies": d.n, "pairs_per_step": pairs_per_step(d.n)}
        row["oracle_all_cores_s_per_step"] = oracle_step_time(d, 1, cores)
        row["oracle_1_core_s_per_step"] = (oracle_step_time(d, 1, 1) if n <= max_n_1core
                                           else None)
        rows.append((d, row))
    build.build()
    from paper_2604_09184_b300 import nb
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = []
    for d, row in rows:
        s = nb.NBodySystem(nb.params(dt_rcrit=d.dt), d.x, d.v, d.m, d.R)
        for _ in range(max(args.warmup, 1)):
            s.step(1, d.dt)
        ms = []
        for _ in range(max(args.steps, 1)):
            flush_l2(flush)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(1, d.dt)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        del s
        t = sum(ms) / len(ms) * 1e-3
        row["gpu_s_per_step"] = t
        row["gpu_pairs_per_s"] = row["pairs_per_step"] / t
        row["gpu_steps_per_s"] = 1.0 / t
        row["gpu_over_oracle_all_cores"] = row["oracle_all_cores_s_per_step"] / t
        o1 = row["oracle_1_core_s_per_step"]
        row["gpu_over_oracle_1_core"] = o1 / t if o1 else None
        out.append(row)
    line = {"metric": "pair interactions/s and steps/s vs N (resolution study)", "unit":
            "pair interactions/s", "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "host_cores": cores,
            "config": {"workload": "mmsn_16k_js family: 0.5-4 AU, 5 Earth masses, J + S, dt 6 d",
                       "l2": "flushed before each timed step"},
            "resolution": out,
            "paper_context": {"gpu_over_1_core_large_n": 150, "gpu_over_16_cores_large_n": 20,
                              "cpu_over_gpu_small_n": ">= 10",
                              "hardware": "GENGA on RTX 4070 Ti or Tesla P100 vs Ryzen 9 7950X3D"}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.resolution:
        return run_resolution(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
