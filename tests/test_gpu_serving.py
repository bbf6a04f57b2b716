"""Request loop: every request served in the mix (continuous batching with
memory-based admission, Poisson arrivals) ends with exactly the loads of the
same request run alone as a plain solve."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_served_results_equal_plain_solves():
    from paper_2107_01370_gb300 import build, lbfsi, serving
    build.build()
    lbfsi.load()
    reqs = serving.viv_requests(n=12, steps=40, seed=3)
    for r in reqs:                      # keep the test small: the two smaller sizes
        r.nr, r.ntheta = serving.SIZES[r.rid % 2]
    serving.poisson_arrivals(reqs, rate=400.0, seed=2)
    cache = serving.CaseCache()
    # a pool that holds only part of the requests at once
    done_b, loads_b, wall_b, peak = serving.run_batched(reqs, pool_bytes=24 << 20, chunk=7, cache=cache)
    done_s, loads_s, wall_s = serving.run_sequential(reqs, cache=cache)
    assert sorted(done_b) == sorted(done_s) == list(range(12))
    assert 1 < peak < 12
    for rid in range(12):
        assert np.array_equal(loads_b[rid], loads_s[rid]), rid
    p50, p99 = serving.latency_stats(done_b)
    assert 0 < p50 <= p99
