"""The serving scheduler's host logic on CPU, with the batch, the systems and
the clock replaced by fakes (no GPU, no library calls): admission by the
memory budget, quanta that end at a member's sampling start or end, the
particle-step count, and latency / wait on the clock of a run whose arrival
times are stretched."""
import numpy as np
import pytest

serve = pytest.importorskip("paper_2109_11083_gb300.serve")


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeSim:
    def __init__(self, req):
        self.req = req
        self.resets = 0

    def stress(self, instantaneous=False):
        return None, 0.5, 1

    def velocity_profile(self):
        return np.zeros(4), np.zeros(4, dtype=np.int64)

    def reset_samples(self):
        self.resets += 1

    def close(self):
        pass


def _install(monkeypatch, clock, log, sims=None):
    class FakeBatch:
        def __init__(self, budget_bytes=0, stream=None):
            self.members = []

        def add(self, sim):
            self.members.append(sim)

        def remove(self, sim):
            self.members.remove(sim)

        def step(self, q):
            log.append((q, sorted(m.req.id for m in self.members)))
            clock.t += 1e-3 * q  # 1 ms per step, whatever the members

        def close(self):
            pass

    monkeypatch.setattr(serve, "Batch", FakeBatch)
    def open_request(req, stream=None):
        sim = FakeSim(req)
        if sims is not None:
            sims[req.id] = sim
        return sim

    monkeypatch.setattr(serve, "open_request", open_request)
    monkeypatch.setattr(serve, "request_bytes", lambda req: req.n)
    monkeypatch.setattr(serve.time, "sleep", lambda s: setattr(clock, "t", clock.t + max(s, 0.0)))


def _req(i, arrival, n, steps):
    return serve.Request(i, arrival, "lj", n, 0.8442, 0.1, steps, i)


def test_budget_quanta_and_counts(monkeypatch):
    clock, log, sims = FakeClock(), [], {}
    _install(monkeypatch, clock, log, sims)
    reqs = [_req(0, 0.0, 600, 250), _req(1, 0.0, 500, 100), _req(2, 0.01, 300, 50)]
    srv = serve.Server(budget_bytes=1000, quantum=100, clock=clock)
    res = srv.run(reqs)
    srv.close()
    assert sorted(r.id for r in res) == [0, 1, 2]
    # request 1 (500 bytes) waits until request 0 leaves: never both live
    for q, live in log:
        assert not (0 in live and 1 in live)
        assert sum({0: 600, 1: 500, 2: 300}[k] for k in live) <= 1000
    # quanta never exceed the quantum, and every member's sampling window
    # (the last 20% of its steps) starts exactly once
    assert all(0 < q <= 100 for q, _ in log)
    assert all(sims[k].resets == 1 for k in (0, 1, 2))
    assert srv.particle_steps == sum(r.n * r.steps for r in reqs)
    by_id = {r.id: r for r in res}
    assert by_id[1].wait > 0 and by_id[0].wait == 0
    for r in res:
        assert r.latency >= r.wait >= 0


def test_stretched_arrivals_are_measured_on_the_run_clock(monkeypatch):
    """Arrival times scaled by time_scale: latency and wait are taken from the
    scaled arrival, so an idle server admits on arrival (wait 0) and the
    latency is the request's own stepping time."""
    clock, log = FakeClock(), []
    _install(monkeypatch, clock, log)
    reqs = [_req(0, 0.0, 100, 100), _req(1, 1.0, 100, 100)]
    srv = serve.Server(budget_bytes=10 ** 6, quantum=100, clock=clock)
    res = {r.id: r for r in srv.run(reqs, time_scale=3.0)}
    srv.close()
    assert res[1].wait == pytest.approx(0.0, abs=1e-9)
    assert res[1].latency == pytest.approx(0.1, abs=1e-9)  # 100 steps x 1 ms
    assert res[0].latency == pytest.approx(0.1, abs=1e-9)
