"""Serving with continuous batching: requests that arrive while others run
join the batch, and each result equals the result of the same request run
alone."""
import numpy as np
import pytest

le = pytest.importorskip("paper_2109_11083_gb300")
from paper_2109_11083_gb300 import serve  # noqa: E402

pytestmark = pytest.mark.gpu


def _requests():
    return [
        serve.Request(0, 0.00, "lj", 2000, 0.8442, 0.5, 240, 11),
        serve.Request(1, 0.00, "kg", 20 * 40, 0.85, 0.1, 180, 12, nchains=40, nbeads=20),
        serve.Request(2, 0.05, "lj", 3500, 0.8442, 1e-2, 300, 13),
        serve.Request(3, 0.10, "lj", 1200, 0.8442, 1.0, 120, 14),
    ]


def test_served_results_equal_the_same_requests_alone():
    reqs = _requests()
    srv = serve.Server(budget_bytes=4 * 2 ** 30, quantum=40)
    res = {r.id: r for r in srv.run(reqs)}
    srv.close()
    assert sorted(res) == [0, 1, 2, 3]
    assert srv.max_queue >= 0 and srv.particle_steps == sum(r.n * r.steps for r in reqs)
    for r in reqs:
        eta, prof, cnt = serve.run_alone(r)
        got = res[r.id]
        assert got.viscosity == eta
        assert np.array_equal(got.counts, cnt)
        assert np.array_equal(np.nan_to_num(got.profile), np.nan_to_num(prof))
        assert got.latency >= 0 and got.wait >= 0


def test_budget_holds_requests_back_until_memory_frees():
    reqs = _requests()[:3]
    need = max(serve.request_bytes(r) for r in reqs)
    srv = serve.Server(budget_bytes=int(need * 1.05), quantum=60)   # one request at a time
    res = srv.run(reqs)
    srv.close()
    assert len(res) == 3
    # with room for one request only, later ones waited for earlier ones
    assert max(r.wait for r in res) > 0
