"""Host-side helpers of the serving harness (no GPU): Poisson arrivals, request picks and the
latency report the bench line and the serving study print."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from paper_1712_09407_gb300 import serving  # noqa: E402


def test_poisson_arrivals_rate_and_order():
    a = serving.poisson_arrivals(200.0, 50.0, seed=3)
    assert np.all(np.diff(a) > 0) and a[0] > 0 and a[-1] < 50.0
    # 10000 expected arrivals: the count is within 4 sigma of the mean
    assert abs(len(a) - 10000) < 4 * 100
    # gaps are exponential with mean 1/rate: mean and the fraction above the mean
    g = np.diff(np.concatenate([[0.0], a]))
    assert g.mean() == pytest.approx(1 / 200.0, rel=0.03)
    assert np.mean(g > 1 / 200.0) == pytest.approx(np.exp(-1.0), abs=0.015)
    assert np.array_equal(a, serving.poisson_arrivals(200.0, 50.0, seed=3))


def test_make_requests_draws_from_the_pool_with_replacement():
    pool = [(np.full(n, i, np.float32), np.zeros(n, np.float32), np.zeros(n, np.uint8), np.array([n]), n)
            for i, n in enumerate((3, 5, 7))]
    arr = np.linspace(0.1, 1.0, 50)
    reqs = serving.make_requests(pool, arr, seed=5)
    assert [r.rid for r in reqs] == list(range(50))
    assert [r.arrival for r in reqs] == pytest.approx(list(arr))
    for r in reqs:
        k = int(r.y[0])
        assert r.n == pool[k][4] and r.counts[0] == r.n and r.y is pool[k][0]
    assert len({int(r.y[0]) for r in reqs}) == 3
    again = serving.make_requests(pool, arr, seed=5)
    assert [int(r.y[0]) for r in again] == [int(r.y[0]) for r in reqs]


def test_latency_report_percentiles_and_counts():
    reqs = []
    for i in range(1000):
        r = serving.Request(i, float(i) * 1e-3, None, None, None, np.zeros(1), 10)
        r.status = "done"
        r.t_done = r.arrival + (i + 1) * 1e-5          # latencies 0.01 .. 10 ms
        r.batch_size = 1 + i % 3
        reqs.append(r)
    reqs[0].status = "rejected"
    reqs[1].status = "error 4"
    rep = serving.latency_report(reqs, 2.0)
    lat = np.arange(3, 1001) * 1e-2
    assert rep["n"] == 998 and rep["rejected"] == 1 and rep["errors"] == 1
    assert rep["p50_ms"] == pytest.approx(np.percentile(lat, 50))
    assert rep["p99_ms"] == pytest.approx(np.percentile(lat, 99))
    assert rep["p999_ms"] == pytest.approx(np.percentile(lat, 99.9))
    assert rep["max_ms"] == pytest.approx(10.0)
    assert rep["events_per_s"] == pytest.approx(998 / 2.0) and rep["clusters_per_s"] == pytest.approx(9980 / 2.0)
    assert rep["mean_batch"] == pytest.approx(np.mean([1 + i % 3 for i in range(2, 1000)]))
    assert serving.latency_report([], 1.0) == {"n": 0}
