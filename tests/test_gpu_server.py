"""Serving engine: continuous batching of requests that arrive at different
times; each result equals the same request priced alone (bit for bit),
admission waits for device memory, work of different requests overlaps."""
import threading
import time

import numpy as np
import pytest

from paper_2309_10477_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nv(cuda_lib):
    from paper_2309_10477_gb300 import native
    return native


def _items(nv, n, seed, paths=(2, 20000), steps=(1, 200)):
    g = np.random.default_rng(seed)
    out = []
    for i, d in enumerate(wl.batched_contracts(n, seed=seed)):
        payoff, K, T, _, _ = d["contract"]
        out.append(nv.make_batch_item(nv.make_params(**d["params"]),
                                      nv.make_contract(payoff, K, T, int(i % 5 == 2), 0),
                                      int(g.integers(*paths)), int(g.integers(*steps)), 77 + i))
    return out


def _alone(nv, it):
    r = nv.heston_mc_price_greeks_ex(it.params, [it.contract], it.n_paths, it.n_steps, it.rng_seed,
                                     nv.make_options(prec=nv.HESTON_FP32))[0]
    return np.array([getattr(r, k) for k in nv.ESTIMATORS] + list(r.se))


def _vec(nv, r):
    return np.array([getattr(r, k) for k in nv.ESTIMATORS] + list(r.se))


def test_server_results_equal_each_request_alone(nv):
    items = _items(nv, 40, 3)
    with nv.HestonServer(256 << 20, tiles_per_round=512) as srv:
        tickets = []
        for i, it in enumerate(items):
            tickets.append(srv.submit(it))
            if i % 7 == 0:
                time.sleep(0.002)              # arrivals while earlier requests run
        got = [srv.wait(t, 60000) for t in tickets]
        st = srv.stats()
    assert all(g is not None for g in got)
    for it, (r, lat) in zip(items, got):
        assert np.array_equal(_vec(nv, r), _alone(nv, it), equal_nan=True)
        assert lat > 0
    assert st.completed == len(items) and st.queued == 0 and st.active == 0
    assert st.rounds > 1


def test_server_admission_waits_for_memory(nv):
    items = _items(nv, 12, 9, paths=(60000, 65536))          # ~1000 tiles each, 96 KB of rows
    with nv.HestonServer(3 * 768 * 130, tiles_per_round=300) as srv:    # room for 3 at a time
        tickets = [srv.submit(it) for it in items]
        got = [srv.wait(t, 120000) for t in tickets]
        st = srv.stats()
    assert st.memory_peak <= 3 * 768 * 130
    assert st.completed == len(items)
    for it, (r, _) in zip(items, got):
        assert np.array_equal(_vec(nv, r), _alone(nv, it), equal_nan=True)


def test_server_overlaps_requests(nv):
    """A long request and short ones submitted after it: the short ones finish
    first, because every round shares the GPU among the active requests."""
    big = nv.make_batch_item(nv.make_params(**wl.BASE_PARAMS), nv.make_contract(1, 100.0, 1.0),
                             1 << 22, 500, 5)
    small = _items(nv, 6, 21, paths=(1000, 4000), steps=(10, 50))
    with nv.HestonServer(1 << 30, tiles_per_round=4096) as srv:
        t0 = time.monotonic()
        tb = srv.submit(big)
        ts = [srv.submit(it) for it in small]
        done_small = [srv.wait(t, 60000) for t in ts]
        t_small = time.monotonic()
        rb = srv.wait(tb, 60000)
        t_big = time.monotonic()
    assert all(d is not None for d in done_small) and rb is not None
    assert t_small - t0 < t_big - t0
    assert max(lat for _, lat in done_small) < rb[1]
    assert np.array_equal(_vec(nv, rb[0]), _alone(nv, big), equal_nan=True)


def test_server_concurrent_submitters_and_rejections(nv):
    items = _items(nv, 30, 4)
    with nv.HestonServer(64 << 20) as srv:
        tickets = [None] * len(items)

        def worker(lo, hi):
            for i in range(lo, hi):
                tickets[i] = srv.submit(items[i])

        th = [threading.Thread(target=worker, args=(0, 15)), threading.Thread(target=worker, args=(15, 30))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert len(set(tickets)) == len(items)
        for it, tk in zip(items, tickets):
            r, _ = srv.wait(tk, 60000)
            assert np.array_equal(_vec(nv, r), _alone(nv, it), equal_nan=True)
        too_big = nv.make_batch_item(items[0].params, items[0].contract, 1 << 30, 10, 1)
        with pytest.raises(nv.HestonError) as e:
            srv.submit(too_big)
        assert e.value.status == nv.HESTON_ERR_NOMEM
        bad = nv.make_batch_item(items[0].params, items[0].contract, 1, 10, 1)
        with pytest.raises(nv.HestonError) as e:
            srv.submit(bad)
        assert e.value.status == nv.HESTON_ERR_INVALID_ARG
        with pytest.raises(nv.HestonError):
            srv.wait(10 ** 9, 1)                  # never issued
