"""Serving with continuous batching: every request's result is the same as counting it alone."""
import numpy as np
import pytest

from paper_1811_09136_gb300 import batched, serve


def test_poisson_arrivals_rate_and_determinism():
    a = serve.poisson_arrivals(20_000, 200.0, seed=5)
    b = serve.poisson_arrivals(20_000, 200.0, seed=5)
    assert np.array_equal(a, b)
    gaps = np.diff(np.concatenate([[0.0], a]))
    assert (gaps > 0).all()
    assert abs(gaps.mean() - 1 / 200.0) < 0.05 / 200.0        # exponential gaps with mean 1/rate
    assert abs(gaps.std() - 1 / 200.0) < 0.05 / 200.0


def _trace(n=14, rate=400.0):
    specs = batched.mix_specs(6, seed=77, n_min=500, n_max=6000, epn=(4.0, 10.0))
    streams = batched.generate_all(specs, processes=1)
    arr = serve.poisson_arrivals(n, rate, seed=9)
    reqs = []
    for i in range(n):
        sp = specs[i % len(specs)]
        reqs.append(serve.Request(i, float(arr[i]), streams[sp.index], sp.m, sp.m, 100 + i,
                                  chunk=(1 << 10) if i % 2 else (1 << 12)))
    return reqs


@pytest.mark.gpu
@pytest.mark.parametrize("max_live,budget", [(4, None), (16, None), (8, 40 << 20)])
def test_each_result_is_the_same_alone_and_in_the_mix(max_live, budget):
    reqs = _trace()
    rep = serve.serve(reqs, max_live=max_live, budget_bytes=budget, keep_local=True)
    assert len(rep.requests) == len(reqs)
    assert rep.max_live > 1                     # requests really overlapped on the device
    for r in rep.requests:
        g, proc, local = serve.count_alone(r)
        assert np.array_equal(r.proc, proc)
        assert np.array_equal(r.local, local)
        assert abs(r.tau_hat - g) <= 1e-12 * max(abs(g), 1.0)
        assert r.done >= r.admitted >= r.arrival
    s = rep.summary()
    assert s["p99_latency_s"] >= s["p50_latency_s"] > 0


@pytest.mark.gpu
def test_reused_handles_give_the_same_results():
    """Requests of the same shape reuse a finished handle (rept_reset_async with the new seed)."""
    specs = batched.mix_specs(2, seed=55, n_min=500, n_max=3000, epn=(4.0, 8.0))
    streams = batched.generate_all(specs, processes=1)
    arr = serve.poisson_arrivals(10, 50.0, seed=3)
    reqs = [serve.Request(i, float(arr[i]), streams[i % 2], specs[i % 2].m, specs[i % 2].m, 500 + i, chunk=1 << 11)
            for i in range(10)]
    rep = serve.serve(reqs, max_live=2, keep_local=True)
    for r in rep.requests:
        g, proc, local = serve.count_alone(r)
        assert np.array_equal(r.proc, proc) and np.array_equal(r.local, local)
        assert abs(r.tau_hat - g) <= 1e-12 * max(abs(g), 1.0)
