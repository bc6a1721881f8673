"""parallel.price_greeks_sharded on the GPU at world size 1 (no process
group): the launch of its path range, the tile rows and the fixed-order
reduction give exactly the bits of heston_mc_price_greeks_ex, estimates and
standard errors; and the same function with its launch replaced by three
heston_mc_launch_tiles calls over uneven path ranges (the ranks of a
three-way split) still gives those bits."""
import numpy as np
import pytest

from paper_2309_10477_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec_name", ["fp32", "fp64"])
def test_sharded_world_one_equals_the_synchronous_estimate(cuda_lib, prec_name):
    import torch
    from paper_2309_10477_gb300 import native as nv, parallel
    prec = nv.HESTON_FP32 if prec_name == "fp32" else nv.HESTON_FP64
    w = wl.multi_strike_fp32(1 << 15)
    n = w.n_paths + 37                         # a ragged last tile
    params = nv.make_params(**w.params)
    cs = [nv.make_contract(*c) for c in w.contracts]
    opts = nv.make_options(prec=prec, stream=torch.cuda.current_stream())
    got = parallel.price_greeks_sharded(params, cs, n, w.n_steps, w.seed, opts).numpy()
    ref = nv.heston_mc_price_greeks_ex(params, cs, n, w.n_steps, w.seed, nv.make_options(prec=prec))
    gm, gse = nv.results_to_arrays(ref)
    assert np.array_equal(got[:, :6], gm, equal_nan=True)
    assert np.array_equal(got[:, 6:], gse, equal_nan=True)

    # three uneven "ranks" launched one after the other into their slices
    bounds = [(0, 64 * 100), (64 * 100, 64 * 101), (64 * 101, n)]

    def launch_split(p, c, begin, count, n_steps, seed, o, rows):
        assert (begin, count) == (0, n)
        for b, e in bounds:
            t0, t1 = b // 64, -(-e // 64)
            nv.heston_mc_launch_tiles(p, c, b, e - b, n_steps, seed, o, rows[t0:t1])

    got3 = parallel.price_greeks_sharded(params, cs, n, w.n_steps, w.seed, opts,
                                         launch_tiles=launch_split).numpy()
    assert np.array_equal(got3, got, equal_nan=True)
