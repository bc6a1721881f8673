"""C-ABI checks that need no GPU: the library loads, exports every function
declared in include/*.h, and rejects invalid arguments before any CUDA call."""
import ctypes
import glob
import math
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nv():
    from paper_2309_10477_gb300 import build, native
    build.build()
    native.load()
    return native


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(\w+)\s*\(", text, flags=re.M):
            if not m.group(0).lstrip().startswith(("typedef", "#", "return")):
                names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("heston_mc_price_greeks", "heston_mc_price_greeks_ex", "heston_mc_launch",
                     "heston_mc_workspace_bytes", "heston_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(nv):
    lib = ctypes.CDLL(nv.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", nv.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(_declared_functions()) <= exported


def test_status_strings(nv):
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7):
        assert nv.heston_status_string(code)
    assert nv.heston_status_string(12345) == "unknown status"


def _call(nv, params=None, contracts=None, n_paths=1024, n_steps=10, options=None):
    p = params or nv.make_params(100.0, 0.04, 2.0, 0.04, 0.3, -0.7, 0.05)
    cs = contracts or [nv.make_contract(0, 100.0, 1.0)]
    arr = (nv.heston_contract * len(cs))(*cs)
    out = (nv.heston_result * max(1, len(cs)))()
    opt = ctypes.byref(options) if options is not None else None
    return nv.load().heston_mc_price_greeks_ex(ctypes.byref(p), arr, len(cs), n_paths, n_steps,
                                               42, opt, out)


@pytest.mark.parametrize("field,value", [("S0", 0.0), ("S0", -1.0), ("v0", -1e-3),
                                         ("kappa", -1.0), ("theta", -0.1), ("xi", -0.2),
                                         ("rho", 1.5), ("rho", -1.0001), ("r", math.nan),
                                         ("S0", math.inf)])
def test_invalid_params_rejected(nv, field, value):
    p = nv.make_params(100.0, 0.04, 2.0, 0.04, 0.3, -0.7, 0.05)
    setattr(p, field, value)
    assert _call(nv, params=p) == nv.HESTON_ERR_INVALID_ARG


def test_invalid_sizes_and_contracts_rejected(nv):
    E = nv.HESTON_ERR_INVALID_ARG
    assert _call(nv, n_steps=0) == E
    assert _call(nv, n_paths=1) == E
    assert _call(nv, n_paths=(1 << 40) + 1) == E
    assert _call(nv, contracts=[nv.make_contract(0, -1.0, 1.0)]) == E
    assert _call(nv, contracts=[nv.make_contract(0, 100.0, 0.0)]) == E
    assert _call(nv, contracts=[nv.make_contract(2, 100.0, 1.0)]) == E
    assert _call(nv, contracts=[nv.make_contract(0, 100.0, 1.0, is_put=2)]) == E
    # N % M != 0, contracts with different T or different Asian M
    assert _call(nv, n_steps=10, contracts=[nv.make_contract(1, 100.0, 1.0, n_monitor=3)]) == E
    assert _call(nv, contracts=[nv.make_contract(0, 100.0, 1.0), nv.make_contract(0, 100.0, 2.0)]) == E
    assert _call(nv, n_steps=12, contracts=[nv.make_contract(1, 100.0, 1.0, n_monitor=3),
                                            nv.make_contract(1, 90.0, 1.0, n_monitor=4)]) == E
    assert _call(nv, contracts=[nv.make_contract(0, 100.0, 1.0)] * 9) == E
    bad = nv.make_options()
    bad.trunc = 7
    assert _call(nv, options=bad) == E
    bad = nv.make_options()
    bad.block_threads = 48
    assert _call(nv, options=bad) == E


def test_null_pointers_rejected(nv):
    lib = nv.load()
    out = nv.heston_result()
    p = nv.make_params(100.0, 0.04, 2.0, 0.04, 0.3, -0.7, 0.05)
    c = nv.make_contract(0, 100.0, 1.0)
    assert lib.heston_mc_price_greeks(None, ctypes.byref(c), 100, 10, 1, ctypes.byref(out)) == -1
    assert lib.heston_mc_price_greeks(ctypes.byref(p), None, 100, 10, 1, ctypes.byref(out)) == -1
    assert lib.heston_mc_price_greeks(ctypes.byref(p), ctypes.byref(c), 100, 10, 1, None) == -1
    b = ctypes.c_size_t()
    assert lib.heston_mc_workspace_bytes(0, 100, ctypes.byref(b)) == -1
    assert lib.heston_mc_workspace_bytes(1, 100, None) == -1


def test_workspace_size_formula(nv):
    # tile rows (12 doubles per contract per 64-path tile) + group rows, 256-byte aligned
    for nc, n in ((1, 2), (6, 1 << 22), (8, 12345)):
        tiles = -(-n // 64)
        groups = -(-tiles // 256)
        w = 12 * nc * 8
        al = lambda x: (x + 255) // 256 * 256
        assert nv.heston_mc_workspace_bytes(nc, n) == al(tiles * w) + al(groups * w)
