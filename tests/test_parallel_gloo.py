"""Multi-rank path sharding on CPU: two gloo ranks each produce the tile rows
of their path range (with the oracle standing in for the GPU kernel), gather
them with paper_2309_10477_gb300.parallel, and must hold exactly the rows of
the unsharded run, in order; a fixed-order sum over them then equals the
single-process sum bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2309_10477_gb300 import parallel

P = oracle.Params(S0=100.0, v0=0.04, kappa=2.0, theta=0.04, xi=0.3, rho=-0.7, r=0.05)
CS = [oracle.Contract(0, 100.0, 1.0), oracle.Contract(1, 95.0, 1.0)]
N_STEPS, SEED = 12, 5


def _tile_rows(begin, end):
    """Rows (sum_x[6C], sum_x^2[6C]) per 64-path tile of [begin, end), from the oracle."""
    rows = []
    for t0 in range(begin, end, 64):
        idx = np.arange(t0, min(end, t0 + 64))
        _, est = oracle.debug_paths(P, CS, idx, N_STEPS, SEED)
        rows.append(np.concatenate([est.sum(axis=0).ravel(), (est * est).sum(axis=0).ravel()]))
    return np.array(rows).reshape(-1, 12 * len(CS))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n_paths, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b, e = parallel.shard_bounds(n_paths, world, rank)
        local = torch.from_numpy(_tile_rows(b, e)) if e > b else torch.zeros((0, 12 * len(CS)),
                                                                                dtype=torch.float64)
        rows = parallel.gather_tile_rows(local, n_paths, world)
        q.put((rank, rows.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n_paths", [(2, 64 * 9 + 17), (2, 64 * 4), (3, 64 * 5 + 1)])
def test_gloo_ranks_gather_the_unsharded_rows(world, n_paths):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_paths, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = _tile_rows(0, n_paths)
    for r in range(world):
        assert np.array_equal(got[r], ref), r
    # fixed-order reduction of the gathered rows equals the single-process one
    assert np.array_equal(np.cumsum(got[0], axis=0)[-1], np.cumsum(ref, axis=0)[-1])


def test_shard_bounds_cover_exactly_and_align():
    for n in (1, 63, 64, 65, 1000, 1 << 22):
        for world in (1, 2, 3, 8):
            spans = [parallel.shard_bounds(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            for (b0, e0), (b1, _) in zip(spans, spans[1:]):
                assert e0 == b1
            assert all(b % 64 == 0 for b, e in spans if e > b)
            sizes = [-(-(e - b) // 64) for b, e in spans]
            assert max(sizes) - min(sizes) <= 1


# ---------------------------------------------------------------------------
# price_greeks_sharded end to end on gloo ranks: the oracle's tile rows stand
# in for heston_mc_launch_tiles and a fixed-order host sum for
# heston_mc_reduce_tiles; every rank must return the single-process result.
# ---------------------------------------------------------------------------

def _launch_stub(params, contracts, path_begin, n, n_steps, seed, options, rows):
    rows[:] = torch.from_numpy(_tile_rows(path_begin, path_begin + n))


def _reduce_stub(rows, n_tiles, n_contracts, n_paths, device):
    assert rows.shape == (n_tiles, 12 * n_contracts)
    tot = np.zeros(12 * n_contracts)
    for t in range(n_tiles):                 # fixed order: tile rows in path order
        tot += rows[t].numpy()
    E = 6 * n_contracts
    mean = tot[:E] / n_paths
    se = np.sqrt(np.maximum((tot[E:] - n_paths * mean * mean) / (n_paths - 1), 0.0) / n_paths)
    return torch.from_numpy(np.concatenate([mean.reshape(-1, 6), se.reshape(-1, 6)], axis=1).ravel())


def _sharded_worker(rank, world, port, n_paths, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = parallel.price_greeks_sharded(None, CS, n_paths, N_STEPS, SEED, None,
                                            device=torch.device("cpu"), launch_tiles=_launch_stub,
                                            reduce_tiles=_reduce_stub)
        q.put((rank, out.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n_paths", [(2, 64 * 7 + 9), (3, 64 * 3)])
def test_gloo_price_greeks_sharded_equals_one_process(world, n_paths):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, world, port, n_paths, q))
             for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    alone = parallel.price_greeks_sharded(None, CS, n_paths, N_STEPS, SEED, None,
                                          device=torch.device("cpu"), launch_tiles=_launch_stub,
                                          reduce_tiles=_reduce_stub).numpy()
    for r in range(world):
        assert np.array_equal(got[r], alone), r
    om, ose = oracle.mc_price_greeks(P, CS, n_paths, N_STEPS, SEED)
    np.testing.assert_allclose(alone[:, :6], om, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(alone[:, 6:], ose, rtol=1e-9, atol=1e-13)
