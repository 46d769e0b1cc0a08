"""Host side of the serving driver, with a stand-in server: requests are submitted no earlier than
their arrival times, results come back in request order, and the summary's rates and latency
percentiles are those of the results."""
import threading
import time

import numpy as np
import pytest

from paper_2012_13133_gb300 import serve


class FakeServer:
    """Completes each request a fixed service time after its submission (one at a time)."""

    def __init__(self, service_s):
        self.service_s = service_s
        self.submitted = {}
        self.lock = threading.Lock()
        self.t0 = time.perf_counter()

    def submit(self, kind, mask, y, X, cov, opts, target_cells=None, target_X=None):
        with self.lock:
            t = len(self.submitted)
            self.submitted[t] = (time.perf_counter() - self.t0, y[0])
        return t

    def wait(self, ticket, timeout_s):
        time.sleep(self.service_s)
        with self.lock:
            at, tag = self.submitted[ticket]
        return dict(latency_ms=1e3 * (time.perf_counter() - self.t0 - at), status=0, loglik=float(tag))


def test_replay_respects_arrivals_and_keeps_request_order():
    reqs = [dict(kind=0, mask=None, y=np.array([float(i)]), X=None, cov=None, opts=None) for i in range(6)]
    arrivals = np.array([0.0, 0.01, 0.02, 0.06, 0.06, 0.1])
    srv = FakeServer(0.002)
    results, wall = serve.replay(srv, reqs, arrivals)
    assert [r["loglik"] for r in results] == [float(i) for i in range(6)]
    times = sorted(v[0] for v in srv.submitted.values())
    assert all(t >= a - 1e-3 for t, a in zip(times, arrivals))
    assert wall >= arrivals[-1]


def test_summary_of_results():
    res = [dict(latency_ms=float(v), status=s) for v, s in zip(range(1, 101), [0] * 97 + [4] * 3)]
    s = serve.summarise(res, 2.0)
    assert s["requests"] == 100 and s["requests_per_s"] == 50.0
    assert s["p50_ms"] == pytest.approx(50.5) and s["p99_ms"] == pytest.approx(99.01)
    assert s["status_counts"] == {"0": 97, "4": 3}
