"""Serving with continuous batching: every request's result is the oracle's, and the same as counting
it alone."""
import numpy as np
import pytest

import oracle as O
from paper_1811_09136_gb300 import batched, serve


def _assert_oracle(r):
    """The served request's tau^(i), local counts and tau_hat against the sequential oracle."""
    s = r.stream
    ref = O.rept_stream(s.src, s.dst, s.n_nodes, r.m, r.c, r.seed, pair_counters=False)
    ref_g, _ = O.estimates(r.m, r.c, ref, s.n_nodes)
    assert np.array_equal(r.proc, ref.tau_proc), r.rid
    if r.local is not None:
        assert np.array_equal(r.local, ref.local1), r.rid
    assert abs(r.tau_hat - ref_g) <= 1e-12 * max(abs(ref_g), 1.0), (r.rid, r.tau_hat, ref_g)


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
        _assert_oracle(r)
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
        _assert_oracle(r)
        g, proc, local = serve.count_alone(r)
        assert np.array_equal(r.proc, proc) and np.array_equal(r.local, local)
        assert abs(r.tau_hat - g) <= 1e-12 * max(abs(g), 1.0)


@pytest.mark.gpu
def test_cancelled_requests_leave_the_others_exact():
    """A request given up before admission is dropped; one given up after admission stops being fed
    (its rounds in flight finish) and its handle is reused; every other request still gets exactly
    its counts alone.  A fake clock (1 ms per reading) makes the timing deterministic."""
    reqs = _trace(n=10, rate=400.0)
    longest = max(range(1, 10), key=lambda i: len(reqs[i].stream))
    reqs[longest].chunk = 1 << 8
    reqs[longest].cancel_after = 0.01          # about ten clock readings after its arrival
    reqs[0].cancel_after = 0.0                 # gives up at once, before admission

    class Tick:
        t = 0.0

        def __call__(self):
            self.t += 0.001
            return self.t

    rep = serve.serve(reqs, max_live=8, keep_local=True, clock=Tick())
    cancelled = {r.rid for r in rep.cancelled}
    assert cancelled == {0, longest}, cancelled
    gone = {r.rid: r for r in rep.cancelled}
    assert np.isnan(gone[0].admitted) and not np.isnan(gone[longest].admitted)
    assert all(np.isnan(r.tau_hat) for r in rep.cancelled)
    assert len(rep.requests) == len(reqs) - 2
    for r in rep.requests:
        _assert_oracle(r)
        g, proc, local = serve.count_alone(r)
        assert np.array_equal(r.proc, proc) and np.array_equal(r.local, local)
        assert abs(r.tau_hat - g) <= 1e-12 * max(abs(g), 1.0)
    assert rep.summary()["cancelled"] == 2
