"""Benchmark of the Lees-Edwards shear-flow MD step on GB300.

One benchmark step is one MD step of the whole hot path (kick/drift, the
rebuild trigger and, when it fires, resort + LE-aware Verlet list, pair forces
with the peculiar-velocity Langevin thermostat, stress and profile sums) on the
large single LJ box: N = 4,194,304 particles, density 0.8442, rc = 2.5,
skin 0.3, shear rate 0.05, dt 0.005, Langevin xi = 1, FP32 forces with
FP64-class positions.  Inputs are resident in HBM when the timed region starts
(the state touched per step, ~1.9 GB, is far larger than the 129 MB L2).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on bounded samples of the same workload instead.
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

import synth  # noqa: E402

METRIC = "particle-steps/s"
UNIT = "particle-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sub", action="store_true",
                    help="box workload: skip the bounded batched and served sub-records")
    ap.add_argument("--eager", action="store_true",
                    help="launch kernels without CUDA graphs (for profilers that cannot see "
                         "kernels inside conditional graphs)")
    ap.add_argument("--workload", default="box", choices=["box", "batched", "served", "kg"],
                    help="box: the 4,194,304-particle LJ box (the benchmark line); batched: "
                         "256 uneven LJ boxes stepped alone vs in one batch; served: the "
                         "shear-sweep request stream with continuous batching")
    ap.add_argument("--systems", type=int, default=256, help="batched workload: box count")
    ap.add_argument("--angle-k", type=float, default=0.0,
                    help="kg workload: bending constant k_a of Eq. 12 (0: WCA + FENE only)")
    ap.add_argument("--kg-equilibrate", type=int, default=5000,
                    help="kg workload: uncapped steps at rest after the push-off (untimed)")
    ap.add_argument("--no-plain", action="store_true",
                    help="batched workload: time the batch alone (no per-box comparison, "
                         "no tuning), for profiler captures")
    ap.add_argument("--requests", type=int, default=200,
                    help="served workload: requests taken from the seeded trace (of 1000)")
    ap.add_argument("--arrival-rate", type=float, default=50.0,
                    help="served workload: request arrivals per second (the trace's 50/s "
                         "arrival times stretched or compressed)")
    ap.add_argument("--particles", type=int, default=4194304,
                    help="box size (the default is the benchmark workload; smaller boxes "
                         "of the same density are for profiler captures)")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard_systems(specs, rank: int, world: int):
    """The systems of `rank` among `world` ranks (the package's placement:
    independent boxes need no exchange, so each goes to exactly one rank)."""
    from paper_2109_11083_gb300.placement import shard_systems as shard
    return shard(specs, rank, world)


def job_totals(seconds: float, units: float):
    """Whole-job figures over all ranks: the slowest rank's time and the sum
    of the units the ranks processed (the rank's own values without a
    process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(seconds), float(units)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def workload_config(w):
    return {"workload": w.name, "n_particles": w.n, "density": w.rho, "box": round(w.box, 6),
            "rc": w.rc, "skin": w.skin, "shear_rate": w.shear_rate, "dt": w.dt,
            "langevin_xi": w.xi, "kT": w.kT, "thermostat": "peculiar",
            "l2_policy": "inputs larger than L2 (state touched per step ~1.9 GB >> 129 MB)"}


# ------------------------------------------------------------------ oracle arm
def oracle_rate(n_sample: int, target_s: float, max_steps: int | None = None):
    """The CPU oracle, as it stands, on an n_sample-particle sub-box of the
    same LJ workload: (particle-steps/s, steps, seconds)."""
    import oracle
    base = synth.lj_box_4m()
    w = synth.scaled_lj(base, n_sample)
    pos, vel = synth.lj_initial_state(w)
    vel[:, 0] += w.shear_rate * (pos[:, 2] - 0.5 * w.box)
    p = oracle.params(w.box, w.shear_rate, w.rc, dt=w.dt, xi=w.xi, kT=w.kT, seed=w.seed)
    s = oracle.State(p, pos, vel)
    t0 = time.perf_counter()
    s.run(1)
    one = time.perf_counter() - t0
    steps = max(1, min(max_steps or 10 ** 9, int(target_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    s.run(steps)
    dt = time.perf_counter() - t0
    return n_sample * steps / dt, steps, dt


def _oracle_worker(n_sample: int, target_s: float, barrier, out):
    """One host core's share of the all-core oracle rate (spawned process)."""
    import oracle
    base = synth.lj_box_4m()
    w = synth.scaled_lj(base, n_sample)
    pos, vel = synth.lj_initial_state(w)
    vel[:, 0] += w.shear_rate * (pos[:, 2] - 0.5 * w.box)
    p = oracle.params(w.box, w.shear_rate, w.rc, dt=w.dt, xi=w.xi, kT=w.kT, seed=w.seed)
    s = oracle.State(p, pos, vel)
    t0 = time.perf_counter()
    s.run(1)
    steps = max(1, int(target_s / max(time.perf_counter() - t0, 1e-6)))
    barrier.wait()
    t0 = time.perf_counter()
    s.run(steps)
    out.put((n_sample * steps, time.perf_counter() - t0))


def oracle_rate_all_cores(n_sample: int, target_s: float, procs: int):
    """The oracle, as it stands (one thread per process), run concurrently as
    `procs` independent processes, one per host core, each on its own copy of
    an n_sample-particle sub-box: (summed particle-steps/s, seconds)."""
    import multiprocessing as mp
    import oracle
    oracle.build()      # compiled once, before the processes load it
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    q = ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(n_sample, target_s, barrier, q))
          for _ in range(procs)]
    for pr in ps:
        pr.start()
    res = [q.get() for _ in ps]
    for pr in ps:
        pr.join()
    return sum(u / t for u, t in res), max(t for _, t in res)


def cpu_baseline_record():
    """The oracle on the host's cores: one thread, then every core the
    process may run on (os.sched_getaffinity), each on sub-boxes of the
    benchmark's LJ workload (the oracle's cost per particle-step does not
    depend on N: cell list)."""
    cores = len(os.sched_getaffinity(0))
    rate1, steps, secs = oracle_rate(131072, 10.0)
    rate_all, secs_all = oracle_rate_all_cores(32768, 8.0, cores)
    return {"value": rate_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "host_cores": cores,
            "sample": (f"{cores} concurrent processes (one per host core), each stepping its "
                       f"own 32768-particle sub-box of the same LJ workload for ~{secs_all:.0f} s "
                       f"(FP64 oracle, cell list, one thread each)"),
            "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                              "sample": f"131072-particle sub-box, {steps} oracle steps "
                                        f"({secs:.1f} s, one thread)"}}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    base = synth.lj_box_4m()
    # each timed step is one oracle step of a 16,384-particle sub-box (about
    # 0.1 s on one core), so --steps K finishes in roughly K/10 seconds
    n_sample = 16384
    import oracle
    w = synth.scaled_lj(base, n_sample)
    pos, vel = synth.lj_initial_state(w)
    vel[:, 0] += w.shear_rate * (pos[:, 2] - 0.5 * w.box)
    p = oracle.params(w.box, w.shear_rate, w.rc, dt=w.dt, xi=w.xi, kT=w.kT, seed=w.seed)
    s = oracle.State(p, pos, vel)
    s.run(max(args.warmup, 0))
    t0 = time.perf_counter()
    s.run(args.steps)
    dt = time.perf_counter() - t0
    value = n_sample * args.steps / dt
    sample = (f"{n_sample}-particle sub-box of the same LJ workload (fcc, density 0.8442, "
              f"rc 2.5, skin unused, shear 0.05, dt 0.005, xi 1), one oracle step per "
              f"benchmark step, cell-list FP64 oracle")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(base),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="le_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(parts)
            except ValueError:
                continue
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def force_kernel_bytes(n: int, mean_nb: float) -> float:
    """Algorithmic HBM bytes of one pair-force evaluation (the K4 count):
    per particle its own position 16 + list count 4 + 4 per list entry +
    the force written 16.  Neighbour positions are gathered from cache
    (counted once in the own-position read)."""
    return n * (16 + 4 + 4 * mean_nb + 16)


def force_launch_bytes(n: int, mean_nb: float, fused_drift: bool = False) -> float:
    """The same launch's bytes with its fused epilogue (Langevin, second half
    kick, samples): + half-step velocity 16 + particle id 4 read, total force
    16 and velocity 16 written.  Fused with the next step's kick and drift
    (FP32 inside a multi-step call), no force is written and the launch also
    reads p, its low part and the build position (48) and writes p, the low
    part and the next fixed-point copy (48)."""
    if fused_drift:
        return n * (16 + 4 + 4 * mean_nb) + n * (16 + 4 + 16) + n * (48 + 48)
    return force_kernel_bytes(n, mean_nb) + n * (16 + 4 + 16 + 16)


def alu_check(le, n: int, mean_nb: float, launch_s: float):
    """Secondary check of the pair kernel against the CUDA cores' FP32 peak
    (measured by le_fp32_peak, outside the timed region): 21 flops per listed
    pair (r^2 5, reciprocal 1, scaling 1, r^-6 2, LJ factor 4, force and
    virial sums 8; an FMA is 2), every list entry evaluated."""
    try:
        fma, fma2 = le.le_fp32_peak()
    except Exception as e:  # reported, not fatal: the line's roofline is HBM
        return {"error": str(e)}
    flops = 21.0 * n * mean_nb / launch_s * 1e-12
    return {"bound": "alu", "flops_per_pair": 21, "achieved_tflops": flops,
            "peak_tflops_fma": fma, "peak_tflops_fma2": fma2,
            "frac_of_fma2_peak": flops / fma2 if fma2 > 0 else None,
            "what": "k_force FP32 arithmetic (paired fma.rn.f32x2 form) against the measured "
                    "CUDA-core FMA throughput; the kernel is bound by its L1 gathers"}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profiled_traffic(kernel_file: str):
    """Per-particle DRAM bytes of the pair-force kernel from the committed ncu
    summary, if it was taken on the current source."""
    import hashlib
    summary = os.path.join(ROOT, "profiles", "k_force_lj_box_n4194304.md")
    if not os.path.exists(summary):
        return None
    sha = hashlib.sha256(open(kernel_file, "rb").read()).hexdigest()[:16]
    vals = {}
    for line in open(summary):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha256_16") != sha:
        return None
    try:
        return float(vals["dram_bytes_per_particle"])
    except (KeyError, ValueError):
        return None


def fp32_error_statement():
    """The FP32 path's measured error against the FP64 oracle per output, as
    recorded by the GPU parity tests in the committed summary (None when the
    summary is absent)."""
    path = os.path.join(ROOT, "profiles", "fp32_error_lj.json")
    try:
        return json.load(open(path))
    except Exception:
        return None


def run_ours(args):
    import torch
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", rank=rank, world_size=world)
    torch.cuda.set_device(local)
    import paper_2109_11083_gb300 as le

    w = synth.lj_box_4m()
    if args.particles != w.n:
        w = synth.scaled_lj(w, args.particles, f"lj_box_n{args.particles}_fp32")
    pos, vel = synth.lj_initial_state(w)
    vel[:, 0] += w.shear_rate * (pos[:, 2] - 0.5 * w.box)
    stream = torch.cuda.current_stream()
    sim = le.Sim(w.box, w.shear_rate, w.rc, w.skin, stream=stream, dt=w.dt, xi=w.xi, kT=w.kT,
                 seed=w.seed, system_id=rank, precision=le.LE_FP32, sample_every=1,
                 profile_bins=20)
    sim.set_particles(pos, vel)
    if args.eager:
        sim.set_eager(True)
    sim.step(args.warmup)
    # launch shapes from the autotuner (trial steps are rolled back: the
    # state and every later result are the same as without it)
    tuned = None if args.eager else sim.tune(64)
    c0 = sim.counters()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    time.sleep(0.3)   # let the sampler take its first reading under load
    force_ms, drift_ms, total_ms = sim.step_profiled(args.steps)
    barrier()
    clk = clocks.stop()
    c1 = sim.counters()
    max_s, units = job_totals(total_ms * 1e-3, w.n * args.steps)
    max_ms = max_s * 1e3
    value = units / max_s

    rebuilds = c1["rebuilds"] - c0["rebuilds"]
    ncell = c1["cells"][0] * c1["cells"][1] * c1["cells"][2]
    passes = math.ceil(max(1, math.ceil(math.log2(max(2, ncell)))) / 9)
    # per step: decide, force, and a drift launch in the first step only (the
    # force launch of every other step ran its drift: FP32 without DPD); per
    # rebuild: bin, 5 per sort pass (counts, 3 scan kernels, scatter),
    # permute (with the cell ranges), list, finish
    fused = True  # this box runs FP32 with the Langevin thermostat
    launches = (2 * args.steps + 1 if fused else 3 * args.steps) + rebuilds * (1 + 5 * passes + 3)
    mean_nb = c1["list_mean"]
    kbytes = force_kernel_bytes(w.n, mean_nb)
    f_avg_s = force_ms / args.steps * 1e-3
    achieved = kbytes / f_avg_s / 1e9
    achieved_fused = force_launch_bytes(w.n, mean_nb, fused_drift=fused) / f_avg_s / 1e9
    peak, peak_kind = measured_peak()
    traffic_pp = profiled_traffic(os.path.join(ROOT, "paper_2109_11083_gb300", "csrc",
                                               "le_kernels.cu"))

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_baseline_record()
        e2e = None
        if not args.no_e2e:
            import torch as _t
            hp = _t.from_numpy(pos).pin_memory().numpy()
            hv = _t.from_numpy(vel).pin_memory().numpy()
            out_p = _t.empty((w.n, 3), dtype=_t.float64).pin_memory().numpy()
            out_v = _t.empty((w.n, 3), dtype=_t.float64).pin_memory().numpy()
            def e2e_once():
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                sim.set_particles(hp, hv)
                sim.step(args.steps)
                le.le_positions(sim.h, w.n, out_p, out_v)
                sim.stress(instantaneous=False)
                sim.velocity_profile()
                torch.cuda.synchronize()
                return time.perf_counter() - t0
            # one untimed pass first: a call of K steps captures, once per
            # process, the graph of its K mod 16 remaining steps
            e2e_once()
            e_s = e2e_once()
            e2e = {"value": w.n * args.steps / e_s, "unit": UNIT,
                   "h2d_bytes_per_step": 48 * w.n / args.steps,
                   "d2h_bytes_per_step": (48 * w.n + 8 * 3 + 16 * 20) / args.steps,
                   "what": "le_set_particles (host pinned pos/vel, initial list and forces) + "
                           "le_step(K) + le_positions + le_stress + le_velocity_profile; "
                           "the second of two passes (the first captures the step graphs)"}
        sub = {}
        if not args.no_sub and world == 1:
            # the metric's other half, bounded: batched and served forms against
            # the plain one-system-per-launch form on this GPU, equal accuracy
            # checked bitwise (outside the timed region of the line's value)
            specs = synth.batched_systems(count=256)
            rec = measure_batched(le, specs, 64, 3, compare=True, tune_steps=0, n_check=16)
            sub["batched"] = {"config": batched_config(specs, 1), "steps": 64,
                              "value": rec["value"], "unit": UNIT, "plain": rec["plain"],
                              "batched_over_plain": rec["batched_over_plain"],
                              "equal_accuracy": rec["equal_accuracy"]}
            from paper_2109_11083_gb300 import serve
            # the request stream at the configured 50 arrivals/s, and the same
            # requests arriving 20 times faster (a backlog: the capacity of
            # each form), each against the plain one-at-a-time server
            srv = serve.served_record(count=60, steps=400, rate=50.0, n_check=6,
                                      plain_fifo_too=True)
            srv["config"] = {"workload": "served_60_requests_poisson50_lj_kg_fp32"}
            sat = serve.served_record(count=60, steps=400, rate=1000.0, plain_fifo_too=True)
            sat["config"] = {"workload": "served_60_requests_poisson1000_lj_kg_fp32"}
            sub["served"] = srv
            sub["served_backlog"] = sat
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(w), parallelism="replicas" if world > 1 else "single",
                           launch_shapes=({"force_threads": tuned[0], "list_threads": tuned[1],
                                           "chosen_by": "autotuner (le_tune), trials rolled back"}
                                          if tuned else None)),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "kernel": ("k_force (pair force + Langevin + kick + samples"
                                    + (", + the next step's kick and drift in all but the "
                                       "last step)" if fused else ")")),
                         "algorithmic_bytes_per_launch": kbytes,
                         "bytes_count": "pair force alone: (16 + 4 + 4 n_list + 16) B per particle",
                         "achieved_with_fused_epilogue": achieved_fused,
                         "fused_bytes_count": ("(152 + 4 n_list) B per particle: the pair force "
                                               "without the force write, the epilogue and the "
                                               "next drift" if fused else
                                               "(88 + 4 n_list) B per particle: the pair force "
                                               "and the epilogue"),
                         "avg_launch_ms": f_avg_s * 1e3,
                         "traffic": (traffic_pp * w.n if traffic_pp else None)},
            "kernel_ms_per_step": {"k_force": force_ms / args.steps,
                                   "k_drift": drift_ms / args.steps,
                                   "rest": (total_ms - force_ms - drift_ms) / args.steps},
            "rebuilds": rebuilds, "image_rebuilds": c1["image_rebuilds"] - c0["image_rebuilds"],
            "mean_list_length": mean_nb,
            "alu_check": alu_check(le, w.n, mean_nb, f_avg_s),
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": launches,
        }
        line.update(sub)
        fp32 = fp32_error_statement()
        if fp32:
            line["fp32_error"] = fp32
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def make_box_sim(le, spec, stream=None):
    """One LJ box of the batched workload (fcc, MB velocities + shear profile)."""
    pos, box = synth.lj_box(spec["n"], spec["rho"], spec["seed"])
    vel = synth.mb_velocities(spec["n"], 1.0, spec["seed"])
    gd = spec["shear_rate"]
    vel[:, 0] += gd * (pos[:, 2] - 0.5 * box)
    sim = le.Sim(box, gd, 2.5, 0.3, stream=stream, dt=0.005, xi=1.0, kT=1.0, seed=spec["seed"],
                 system_id=spec["seed"], precision=le.LE_FP32, profile_bins=20)
    sim.set_particles(pos, vel)
    return sim


def measure_batched(le, specs, steps: int, warmup: int, compare: bool = True,
                    tune_steps: int = 32, barrier=lambda: None, world: int = 1,
                    n_check: int = 16):
    """Boxes `specs` stepped one handle at a time (plain), as one untuned
    batch, and as a batch with launch shapes from the autotuner; members
    checked bitwise against plain.  Returns the timings and checks."""
    import torch
    plain = [make_box_sim(le, s) for s in specs] if compare else []
    batched = [make_box_sim(le, s) for s in specs] if compare else []
    tuned = [make_box_sim(le, s) for s in specs]
    total = sum(s["n"] for s in specs)
    w = max(warmup, 3)
    for s in plain:
        s.step(w)
    b = le.Batch()
    for s in batched:
        b.add(s)
    if compare:
        b.step(w)
    # the same boxes once more, launch shapes picked by the autotuner on the
    # whole batch (the trials are rolled back, so these members stay on the
    # same trajectories)
    bt = le.Batch()
    for s in tuned:
        bt.add(s)
    bt.step(w)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tf, tl, tms = bt.tune(tune_steps) if (compare and tune_steps) else (None, None, None)
    torch.cuda.synchronize()
    t_tune = time.perf_counter() - t0
    barrier()
    t0 = time.perf_counter()
    for s in plain:
        s.step(steps)
    barrier()
    t_plain = time.perf_counter() - t0
    t0 = time.perf_counter()
    if compare:
        b.step(steps)
    barrier()
    t_untuned = time.perf_counter() - t0
    t0 = time.perf_counter()
    bt.step(steps)
    barrier()
    t_batch = time.perf_counter() - t0
    t_plain, u_plain = job_totals(t_plain, total * steps)
    t_untuned, u_untuned = job_totals(t_untuned, total * steps)
    t_batch, u_batch = job_totals(t_batch, total * steps)
    equal = True
    for k in range(0, len(plain), max(1, len(plain) // n_check)):
        rp, vp = plain[k].positions()
        for other in (batched[k], tuned[k]):
            rb, vb = other.positions()
            equal = equal and bool(np.array_equal(rp, rb) and np.array_equal(vp, vb))
    if world > 1:  # every rank's members must be equal
        flag = torch.tensor([1 if equal else 0], device="cuda", dtype=torch.int32)
        torch.distributed.all_reduce(flag, op=torch.distributed.ReduceOp.MIN)
        equal = bool(flag.item())
    b.close()
    bt.close()
    for s in plain + batched + tuned:
        s.close()
    return {"value": u_batch / t_batch, "unit": UNIT, "t_batch": t_batch, "warmup": w,
            "plain": {"value": u_plain / t_plain, "unit": UNIT,
                      "what": "each box stepped by its own le_step, one after another"}
            if compare else None,
            "batched_over_plain": t_plain / t_batch if compare else None,
            "autotune": {"force_threads": tf, "list_threads": tl, "seconds": t_tune,
                         "trial_ms_per_step": tms,
                         "untuned_value": u_untuned / t_untuned} if compare else None,
            "equal_accuracy": {"bitwise_equal_members": equal,
                               "checked": len(range(0, len(plain), max(1, len(plain) // n_check))),
                               "what": "plain vs batched and vs autotuned batched"}
            if compare else None}


def batched_config(all_specs, world):
    return {"workload": f"batched_{len(all_specs)}_uneven_lj_fp32",
            "systems": len(all_specs), "total_particles": sum(s["n"] for s in all_specs),
            "parallelism": f"systems sharded over {world} ranks" if world > 1 else "single",
            "n_range": [500, 32000], "density_range": [0.7, 0.9], "shear_range": [1e-3, 1.0],
            "rc": 2.5, "skin": 0.3, "dt": 0.005}


def run_batched(args):
    """256 independent LJ boxes of uneven N (500 to 32,000) stepped one handle at a time
    (plain) and all together in one batch, equal accuracy checked bitwise."""
    import torch
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", rank=rank, world_size=world)
    torch.cuda.set_device(local)
    import paper_2109_11083_gb300 as le
    all_specs = synth.batched_systems(count=args.systems)
    # N > 1: the boxes are sharded over the ranks (no exchange); the total work
    # is fixed, so this is strong scaling
    specs = shard_systems(all_specs, rank, world) if world > 1 else all_specs

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
    rec = measure_batched(le, specs, args.steps, args.warmup, compare=not args.no_plain,
                          barrier=barrier, world=world)
    line = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": rec["warmup"],
            "ms_per_step": rec["t_batch"] / args.steps * 1e3, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": batched_config(all_specs, world),
            "plain": rec["plain"], "batched_over_plain": rec["batched_over_plain"],
            "autotune": rec["autotune"], "equal_accuracy": rec["equal_accuracy"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def le_min_image(d, box, dX):
    """Lees-Edwards minimum image of separations d (n x 3) in a cubic box."""
    d = d.copy()
    up, dn = d[:, 2] > 0.5 * box, d[:, 2] < -0.5 * box
    d[up, 2] -= box
    d[up, 0] -= dX
    d[dn, 2] += box
    d[dn, 0] += dX
    d[:, :2] -= box * np.rint(d[:, :2] / box)
    return d


def run_kg(args):
    """A Kremer-Grest melt of 200 chains x 100 beads (WCA + FENE, optional
    Eq. 12 bending with --angle-k), FP32 forces, dt 0.01, shear rate 1e-3,
    Langevin xi 0.5.  The initial condition is the stated one: freely jointed
    random walks of bond length 0.97, a force-capped push-off (FP64; caps 10,
    30, 100, 300, 1000, 400 steps each, dt 0.005, at rest), then an uncapped
    equilibration at rest (--kg-equilibrate steps, FP32) -- none of it timed."""
    import torch
    import paper_2109_11083_gb300 as le
    from paper_2109_11083_gb300 import prepare
    torch.cuda.set_device(0)
    w = synth.kg_melt_200x100()
    pos, box, bonds = synth.random_walk_chains(w.nchains, w.nbeads, w.rho, w.seed)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    pos, vel = prepare.push_off(pos, box, bonds, seed=w.seed, stream=stream.cuda_stream)
    eq = le.Sim(box, 0.0, w.rc, w.skin, stream=stream.cuda_stream, dt=w.dt, xi=w.xi, kT=w.kT,
                fene_k=w.fene_k, fene_R0=w.fene_R0, seed=w.seed + 1, system_id=1,
                precision=le.LE_FP32, sample_every=0, angle_k=args.angle_k)
    eq.set_bonds(bonds)
    eq.set_particles(pos, vel)
    eq.step(args.kg_equilibrate)
    pos, vel = eq.positions()
    eq.close()
    t_prep = time.perf_counter() - t0
    vel[:, 0] += w.shear_rate * (pos[:, 2] - 0.5 * box)
    sim = le.Sim(box, w.shear_rate, w.rc, w.skin, stream=stream.cuda_stream, dt=w.dt, xi=w.xi,
                 kT=w.kT, fene_k=w.fene_k, fene_R0=w.fene_R0, seed=w.seed, system_id=1,
                 precision=le.LE_FP32, sample_every=1, angle_k=args.angle_k)
    sim.set_bonds(bonds)
    sim.set_particles(pos, vel)
    sim.step(max(args.warmup, 3))
    tuned = sim.tune(64)
    sim.reset_samples()
    c0 = sim.counters()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    c1 = sim.counters()
    r, _ = sim.positions()
    d = le_min_image(r[bonds[:, 1]] - r[bonds[:, 0]], box, c1["dX"])
    ree = d.reshape(w.nchains, w.nbeads - 1, 3).sum(axis=1)
    _, xz, nsamp = sim.stress(instantaneous=False)
    line = {"metric": METRIC, "value": w.n * args.steps / (ms * 1e-3), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "n_beads": w.n, "chains": w.nchains,
                       "beads_per_chain": w.nbeads, "density": w.rho, "box": round(box, 6),
                       "rc": w.rc, "skin": w.skin, "fene_k": w.fene_k, "fene_R0": w.fene_R0,
                       "angle_k": args.angle_k, "shear_rate": w.shear_rate, "dt": w.dt,
                       "langevin_xi": w.xi, "kT": w.kT,
                       "start": (f"random walks (bond 0.97), capped push-off "
                                 f"{list(prepare.PUSH_OFF_CAPS)} x {prepare.PUSH_OFF_STEPS} steps "
                                 f"(FP64), {args.kg_equilibrate} steps at rest; "
                                 f"{t_prep:.1f} s, untimed"),
                       "launch_shapes": {"force_threads": tuned[0], "list_threads": tuned[1]}},
            "rebuilds": c1["rebuilds"] - c0["rebuilds"],
            "chains": {"R_ee2_mean": float((ree ** 2).sum(axis=1).mean()),
                       "bond_mean": float(np.linalg.norm(d, axis=1).mean()),
                       "what": "from the LE minimum-image bond vectors after the timed steps"},
            "viscosity_short_run": {"eta": xz / w.shear_rate, "samples": nsamp,
                                    "what": "<sigma_xz>/shear_rate over the timed steps only "
                                            "(far too short for a converged value at 1e-3)"}}
    print(json.dumps(line), flush=True)
    sim.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "kg":
        return run_kg(args)
    if args.workload == "served":
        from paper_2109_11083_gb300 import serve
        return serve.main_bench(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
