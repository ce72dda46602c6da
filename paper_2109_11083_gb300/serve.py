"""Shear-sweep serving with continuous batching.

Requests (an LJ or Kremer-Grest box at one shear rate, a number of steps)
arrive over time.  The server keeps every admitted request's particle state
resident on the device as a handle in one batch (include/le.h, le_batch_*),
admits waiting requests whenever the batch's device-memory budget has room
(le_estimate_device_bytes), advances all resident requests together in
quanta of steps (one graph launch per 16 steps for the whole batch), and
retires each request when its steps are done, returning its time-averaged
vx(z) profile and viscosity (Eq. 14: <sigma_xz> / shear rate) over the last
20% of its steps, the averaging window of the paper's profiles (Sec. 3.1).

Requests that arrive while others run join between quanta, so their work
overlaps on the device; a member's trajectory does not depend on who else is
in the batch (the batch runs every member's own kernels), so each result is
the same as running the request alone.
"""
from __future__ import annotations

import collections
import json
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import LE_FP32, Batch, Sim, le_default_params, le_estimate_device_bytes


@dataclass
class Request:
    id: int
    arrival: float              # seconds after the start of the trace
    kind: str                   # "lj" or "kg"
    n: int
    rho: float
    shear_rate: float
    steps: int
    seed: int
    nchains: int = 0
    nbeads: int = 0


@dataclass
class Result:
    id: int
    latency: float              # completion - arrival, seconds
    wait: float                 # admission - arrival, seconds
    particles: int
    steps: int
    viscosity: float
    profile: np.ndarray
    counts: np.ndarray


@dataclass
class _Live:
    req: Request
    sim: Sim
    done: int = 0
    admitted: float = 0.0
    bytes: int = 0
    sampling: bool = False
    extra: dict = field(default_factory=dict)


def build_request_state(req: Request):
    """Positions, velocities (with the shear profile), box and bonds."""
    import synth
    if req.kind == "lj":
        pos, box = synth.lj_box(req.n, req.rho, req.seed)
        bonds = None
    else:
        pos, box, bonds = synth.lattice_chains(req.nchains, req.nbeads, req.rho, req.seed)
    vel = synth.mb_velocities(pos.shape[0], 1.0, req.seed)
    vel[:, 0] += req.shear_rate * (pos[:, 2] - 0.5 * box)
    return pos, vel, box, bonds


def request_params(req: Request):
    """(rc, skin, keyword parameters) of a request's handle."""
    kw = dict(dt=0.005, xi=1.0, kT=1.0, seed=req.seed, system_id=req.id, precision=LE_FP32,
              profile_bins=20, sample_every=1)
    if req.kind == "lj":
        return 2.5, 0.3, kw
    kw.update(fene_k=30.0, fene_R0=1.5, xi=0.5, dt=0.005)
    return 2 ** (1 / 6), 0.3, kw


def open_request(req: Request, stream=None) -> Sim:
    pos, vel, box, bonds = build_request_state(req)
    rc, skin, kw = request_params(req)
    sim = Sim(box, req.shear_rate, rc, skin, stream=stream, **kw)
    if bonds is not None:
        sim.set_bonds(bonds)
    sim.set_particles(pos, vel)
    return sim


def request_bytes(req: Request) -> int:
    pos_n = req.n
    rc, skin, kw = request_params(req)
    p = le_default_params()
    for k, v in kw.items():
        setattr(p, k, v)
    box = (pos_n / req.rho) ** (1 / 3)
    if req.kind == "kg":
        box = (math.ceil(pos_n ** (1 / 3) - 1e-9) ** 3 / req.rho) ** (1 / 3)
    nb = req.nchains * (req.nbeads - 1) if req.kind == "kg" else 0
    return le_estimate_device_bytes(box, req.shear_rate, rc, skin, p, pos_n, nb)


def sample_start(steps: int) -> int:
    """Samples are averaged over the last 20% of a request's steps."""
    return steps - max(1, steps // 5)


def run_alone(req: Request) -> tuple[float, np.ndarray, np.ndarray]:
    """The request on its own handle: (viscosity, profile, counts)."""
    sim = open_request(req)
    s0 = sample_start(req.steps)
    sim.step(s0)
    sim.reset_samples()
    sim.step(req.steps - s0)
    _, xz, _ = sim.stress(instantaneous=False)
    prof, cnt = sim.velocity_profile()
    sim.close()
    eta = xz / req.shear_rate if req.shear_rate != 0 else float("nan")
    return eta, prof, cnt


class Server:
    """Continuous batching of shear-sweep requests on one GPU."""

    def __init__(self, budget_bytes: int, quantum: int = 100, stream=None, clock=time.perf_counter):
        self.budget = int(budget_bytes)
        self.quantum = int(quantum)
        self.stream = stream
        self.clock = clock
        self.batch = Batch(budget_bytes=self.budget, stream=stream)
        self.live: list[_Live] = []
        self.used = 0
        self.particle_steps = 0
        self.max_queue = 0
        self.time_scale = 1.0

    def _admit(self, req: Request, now: float) -> bool:
        need = request_bytes(req)
        if need > self.budget:
            raise ValueError(f"request {req.id} needs {need} bytes, beyond the whole budget")
        if self.used + need > self.budget:
            return False
        sim = open_request(req, self.stream)
        try:
            self.batch.add(sim)
        except Exception:
            sim.close()
            return False
        self.live.append(_Live(req, sim, admitted=now, bytes=need))
        self.used += need
        return True

    def _retire(self, lv: _Live, now: float) -> Result:
        _, xz, _ = lv.sim.stress(instantaneous=False)
        prof, cnt = lv.sim.velocity_profile()
        self.batch.remove(lv.sim)
        lv.sim.close()
        self.used -= lv.bytes
        r = lv.req
        eta = xz / r.shear_rate if r.shear_rate != 0 else float("nan")
        arrival = r.arrival * self.time_scale  # on the wall clock of this run
        return Result(r.id, now - arrival, lv.admitted - arrival, r.n, r.steps, eta, prof, cnt)

    def run(self, requests: list[Request], time_scale: float = 1.0) -> list[Result]:
        """Serves the requests; arrival times are scaled by time_scale (wall
        clock).  Returns the results in completion order."""
        self.time_scale = float(time_scale)
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting: collections.deque[Request] = collections.deque()
        results: list[Result] = []
        t0 = self.clock()
        while pending or waiting or self.live:
            now = self.clock() - t0
            while pending and pending[0].arrival * time_scale <= now:
                waiting.append(pending.popleft())
            self.max_queue = max(self.max_queue, len(waiting))
            while waiting and self._admit(waiting[0], now):
                waiting.popleft()
            if not self.live:
                if pending:
                    time.sleep(max(0.0, pending[0].arrival * time_scale - now))
                continue
            # the quantum ends at the next member event (sampling start or end)
            q = self.quantum
            for lv in self.live:
                s0 = sample_start(lv.req.steps)
                nxt = s0 if lv.done < s0 else lv.req.steps
                q = min(q, nxt - lv.done)
            q = max(q, 1)
            self.batch.step(q)
            now = self.clock() - t0
            for lv in list(self.live):
                lv.done += q
                self.particle_steps += lv.req.n * q
                if lv.done == sample_start(lv.req.steps) and not lv.sampling:
                    lv.sim.reset_samples()
                    lv.sampling = True
                if lv.done >= lv.req.steps:
                    self.live.remove(lv)
                    results.append(self._retire(lv, now))
        self.elapsed = self.clock() - t0
        return results

    def close(self):
        for lv in self.live:
            lv.sim.close()
        self.live = []
        self.batch.close()


def trace_requests(count: int, steps: int, rate: float = 50.0, max_particles: int = 200000,
                   seed: int | None = None) -> list[Request]:
    """Requests of the served workload (synth.request_trace) with `steps` each."""
    import synth
    kw = {} if seed is None else {"seed": seed}
    out = []
    for r in synth.request_trace(count=count, rate=rate, **kw):
        n = min(r["n"], max_particles)
        if r["kind"] == "kg":
            nb = max(2, r["nbeads"])
            nc = max(1, n // nb)
            out.append(Request(r["id"], r["arrival"], "kg", nc * nb, r["rho"], r["shear_rate"],
                               steps, r["seed"] % (2 ** 31), nc, nb))
        else:
            out.append(Request(r["id"], r["arrival"], "lj", max(n, 500), r["rho"],
                               r["shear_rate"], steps, r["seed"] % (2 ** 31)))
    return out


def plain_fifo(requests: list[Request], time_scale: float = 1.0, clock=time.perf_counter):
    """The plain form of the same stream: one request at a time on its own
    handle, first come first served.  Returns (latencies, particle-steps,
    elapsed seconds)."""
    order = sorted(requests, key=lambda r: r.arrival)
    lat = []
    work = 0
    t0 = clock()
    for r in order:
        now = clock() - t0
        if r.arrival * time_scale > now:
            time.sleep(r.arrival * time_scale - now)
        run_alone(r)
        lat.append(clock() - t0 - r.arrival * time_scale)
        work += r.n * r.steps
    return np.array(lat), work, clock() - t0


def served_record(count: int, steps: int, rate: float = 50.0, n_check: int = 0,
                  budget_bytes: int = 150 * 2 ** 30, quantum: int = 100,
                  plain_fifo_too: bool = False) -> dict:
    """Serves `count` requests of the trace (each `steps` steps, arrivals at
    `rate` per second) and summarises latency and throughput.  With n_check >
    0, the first n_check requests are also run alone, and each served result
    must equal its alone result bitwise.  With plain_fifo_too, the whole
    stream is also served the plain way (one request at a time on its own
    handle, first come first served) for its throughput and latency."""
    reqs = trace_requests(count, steps)
    srv = Server(budget_bytes=budget_bytes, quantum=quantum)
    res = srv.run(reqs, time_scale=50.0 / rate)
    srv.close()
    lat = np.array([r.latency for r in res])
    wait = np.array([r.wait for r in res])
    out = {"value": srv.particle_steps / srv.elapsed, "unit": "particle-steps/s",
           "requests": count, "steps_per_request": steps, "arrival_rate_per_s": rate,
           "particles_per_request": [int(min(r.n for r in reqs)), int(max(r.n for r in reqs))],
           "budget_bytes": budget_bytes, "quantum_steps": quantum,
           "latency_s": {"p50": float(np.percentile(lat, 50)),
                         "p99": float(np.percentile(lat, 99)), "mean": float(lat.mean())},
           "wait_s": {"p50": float(np.percentile(wait, 50)),
                      "p99": float(np.percentile(wait, 99))},
           "max_queue": srv.max_queue, "makespan_s": srv.elapsed,
           "offered_particle_steps_per_s": float(sum(r.n * r.steps for r in reqs) /
                                                 (max(r.arrival for r in reqs) * 50.0 / rate))}
    if plain_fifo_too:
        plat, work, el = plain_fifo(reqs, time_scale=50.0 / rate)
        out["plain_fifo"] = {"value": work / el, "unit": "particle-steps/s",
                             "latency_s": {"p50": float(np.percentile(plat, 50)),
                                           "p99": float(np.percentile(plat, 99))},
                             "makespan_s": el,
                             "what": "the same stream served one request at a time, each on "
                                     "its own handle, first come first served"}
        out["served_over_plain_fifo"] = out["value"] / (work / el)
    if n_check > 0:
        by_id = {r.id: r for r in res}
        equal = True
        for r in sorted(reqs, key=lambda r: r.id)[:n_check]:
            eta, prof, cnt = run_alone(r)
            got = by_id[r.id]
            equal = equal and (np.array_equal(prof, got.profile, equal_nan=True)
                               and np.array_equal(cnt, got.counts)
                               and (eta == got.viscosity or (eta != eta and got.viscosity
                                                            != got.viscosity)))
        out["equal_accuracy"] = {"bitwise_equal_requests": bool(equal), "checked": n_check,
                                 "what": "served result vs the same request run alone"}
    return out


def main_bench(args) -> int:
    """`bench.py --workload served`: a Poisson stream of mixed LJ/KG shear-sweep
    requests served with continuous batching; p50/p99 latency and aggregate
    particle-steps/s."""
    count = max(1, int(getattr(args, "requests", 200)))
    steps = max(args.steps // 4, 50)
    rate = float(getattr(args, "arrival_rate", 50.0))
    rec = served_record(count, steps, rate)
    line = {"metric": "particle-steps/s", "value": rec["value"], "unit": "particle-steps/s",
            "n_gpus": 1, "steps": steps, "warmup": 0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"served_{count}_requests_poisson{rate:g}_lj_kg_fp32",
                       "requests": count, "steps_per_request": steps, "arrival_rate_per_s": rate,
                       "particles_per_request": rec["particles_per_request"],
                       "budget_bytes": rec["budget_bytes"], "quantum_steps": rec["quantum_steps"]},
            "latency_s": rec["latency_s"], "wait_s": rec["wait_s"],
            "max_queue": rec["max_queue"], "makespan_s": rec["makespan_s"],
            "offered_particle_steps_per_s": rec["offered_particle_steps_per_s"]}
    print(json.dumps(line), flush=True)
    return 0
