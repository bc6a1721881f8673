"""heston_mc_launch_noalloc: the estimate for callers that must not allocate.

Some callers cannot let a library allocate device memory: an engine whose
device memory belongs to another allocator (a framework's caching allocator
or a fixed arena), or a latency-critical request loop where cudaMalloc can
synchronise the device.  This entry point runs the same kernels as
heston_mc_launch with the workspace in a static device array.  The test calls
it through the C ABI, twice in a row on different problems and then on the
first again (so each call starts from the previous call's leftovers), and
checks every output against heston_mc_launch with the FP64 parity tolerance.
It lives in a file of its own, collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2309_10477_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _launch_ref(nv, torch, params, cs, n, N, seed, prec):
    nc = len(cs)
    ws_bytes = nv.heston_mc_workspace_bytes(nc, n)
    ws = torch.empty(ws_bytes // 8, dtype=torch.float64, device="cuda")
    out = torch.empty(nc * 12, dtype=torch.float64, device="cuda")
    opts = nv.make_options(prec=prec, stream=torch.cuda.current_stream())
    nv.heston_mc_launch(params, cs, n, N, seed, opts, ws, ws_bytes, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _launch_noalloc(nv, torch, params, cs, n, N, seed, prec):
    out = torch.full((len(cs) * 12,), float("nan"), dtype=torch.float64, device="cuda")
    opts = nv.make_options(prec=prec, stream=torch.cuda.current_stream())
    rc = nv.heston_mc_launch_noalloc(params, cs, n, N, seed, opts, out)
    torch.cuda.synchronize()
    assert rc == nv.HESTON_OK
    return out.cpu().numpy()


def test_noalloc_matches_launch_on_consecutive_calls(cuda_lib):
    import torch
    from paper_2309_10477_gb300 import native as nv
    big = wl.multi_strike_fp32(1 << 18)
    cases = [
        (nv.make_params(**wl.BASE_PARAMS), [nv.make_contract(*c) for c in big.contracts],
         big.n_paths, big.n_steps, 42, nv.HESTON_FP32),
        (nv.make_params(**wl.PAPER_PARAMS),
         [nv.make_contract(0, 100.0, 1.0), nv.make_contract(1, 95.0, 1.0, 1, 4)],
         64 * 37 + 5, 32, 7, nv.HESTON_FP64),
    ]
    refs = [_launch_ref(nv, torch, *c) for c in cases]
    for i in (0, 1, 0):
        got = _launch_noalloc(nv, torch, *cases[i])
        np.testing.assert_allclose(got, refs[i], rtol=1e-9, atol=1e-11)


def test_noalloc_rejects_requests_beyond_its_scratch(cuda_lib):
    import torch
    from paper_2309_10477_gb300 import native as nv
    cs = [nv.make_contract(0, 100.0, 1.0)] * 8
    n = 1 << 22            # 8 contracts x 65536 tiles of 96 doubles > 16 MiB
    assert nv.heston_mc_workspace_bytes(len(cs), n) > nv.HESTON_NOALLOC_SCRATCH_BYTES
    out = torch.full((len(cs) * 12,), 7.0, dtype=torch.float64, device="cuda")
    arr = (nv.heston_contract * len(cs))(*cs)
    p = nv.make_params(**wl.BASE_PARAMS)
    opts = nv.make_options(prec=nv.HESTON_FP32, stream=torch.cuda.current_stream())
    rc = nv.load().heston_mc_launch_noalloc(ctypes.byref(p), arr, len(cs), n, 16, 1,
                                            ctypes.byref(opts), out.data_ptr())
    torch.cuda.synchronize()
    assert rc == nv.HESTON_ERR_WORKSPACE
    assert (out.cpu().numpy() == 7.0).all()
