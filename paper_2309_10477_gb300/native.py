"""ctypes binding of ``libhestonmc.so`` (C ABI in ``include/heston_mc.h``).

Argument marshalling only: every step of the path runs in the CUDA kernels of
``csrc/heston_mc.cu``.  The functions keep the C names.  Device buffers may be
given as ``torch.Tensor`` (CUDA) or raw integer addresses; streams as
``torch.cuda.Stream`` or raw handles.  If the shared library has not been
built, ``load()`` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhestonmc.so")

HESTON_OK = 0
HESTON_WARN_GAMMA_UNDEFINED = 1
HESTON_WARN_TANGENT_UNSTABLE = 2
HESTON_ERR_INVALID_ARG = -1
HESTON_ERR_CUDA = -2
HESTON_ERR_NOMEM = -3
HESTON_ERR_TIMEOUT = -4
HESTON_ERR_CANCELLED = -5
HESTON_ERR_UNSUPPORTED = -6
HESTON_ERR_WORKSPACE = -7
HESTON_MAX_CONTRACTS = 8
HESTON_TILE_PATHS = 64
HESTON_NOALLOC_SCRATCH_BYTES = 16 << 20

HESTON_EUROPEAN, HESTON_ASIAN_ARITH = 0, 1
HESTON_TRUNC_FULL, HESTON_TRUNC_PAPER_FLOOR = 0, 1
HESTON_RNG_PHILOX, HESTON_RNG_SOBOL_BB = 0, 1
HESTON_FP32, HESTON_FP64 = 0, 1
HESTON_SCHEME_MILSTEIN, HESTON_SCHEME_EULER, HESTON_SCHEME_QE = 0, 1, 2

ESTIMATORS = ("price", "delta", "gamma", "vega", "rho", "theta")
RECORD_FIELDS = ("X", "V", "X_v", "V_v", "X_T", "V_T", "sumS", "sumtS", "sumS_Xv", "sumS_XT",
                 "GE", "QE", "GA", "QA", "minabsV")


class heston_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("S0", "v0", "kappa", "theta", "xi", "rho", "r")]


class heston_contract(ctypes.Structure):
    _fields_ = [("payoff", ctypes.c_int32), ("is_put", ctypes.c_int32), ("K", ctypes.c_double),
                ("T", ctypes.c_double), ("n_monitor", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class heston_options(ctypes.Structure):
    _fields_ = [("trunc", ctypes.c_int32), ("rng", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("n_shifts", ctypes.c_uint32), ("cuda_stream", ctypes.c_void_p),
                ("device", ctypes.c_int32), ("grid_ctas", ctypes.c_uint32),
                ("block_threads", ctypes.c_uint32), ("scheme", ctypes.c_int32),
                ("reserved", ctypes.c_uint32)]


class heston_result(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ESTIMATORS] + [
        ("se", ctypes.c_double * 6), ("n_paths", ctypes.c_uint64), ("status", ctypes.c_int32),
        ("reserved", ctypes.c_int32)]


class heston_batch_item(ctypes.Structure):
    _fields_ = [("params", heston_params), ("contract", heston_contract), ("n_paths", ctypes.c_uint64),
                ("n_steps", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("rng_seed", ctypes.c_uint64)]


class heston_batch_plan(ctypes.Structure):
    _fields_ = [("total_tiles", ctypes.c_uint64), ("total_groups", ctypes.c_uint64),
                ("total_path_steps", ctypes.c_uint64), ("n_items", ctypes.c_uint32),
                ("trunc", ctypes.c_int32), ("descriptor_bytes", ctypes.c_size_t),
                ("workspace_bytes", ctypes.c_size_t)]


class heston_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("trunc", ctypes.c_int32), ("memory_bytes", ctypes.c_size_t),
                ("max_active", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("tiles_per_round", ctypes.c_uint64)]


class heston_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rounds", ctypes.c_uint64), ("tiles_done", ctypes.c_uint64),
                ("queued", ctypes.c_uint32), ("active", ctypes.c_uint32),
                ("memory_in_use", ctypes.c_size_t), ("memory_peak", ctypes.c_size_t)]


class HestonError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None


def load():
    """Load the in-tree CUDA library; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                           "(the CUDA path has no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    u32, u64, i32, vp, sz = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p,
                             ctypes.c_size_t)
    sig = {
        "heston_mc_price_greeks": ([P(heston_params), P(heston_contract), u64, u32, u64,
                                    P(heston_result)], i32),
        "heston_mc_price_greeks_ex": ([P(heston_params), P(heston_contract), u32, u64, u32, u64,
                                       P(heston_options), P(heston_result)], i32),
        "heston_mc_workspace_bytes": ([u32, u64, P(sz)], i32),
        "heston_mc_launch": ([P(heston_params), P(heston_contract), u32, u64, u32, u64,
                              P(heston_options), vp, sz, vp], i32),
        "heston_mc_launch_noalloc": ([P(heston_params), P(heston_contract), u32, u64, u32, u64,
                                      P(heston_options), vp], i32),
        "heston_mc_launch_tiles": ([P(heston_params), P(heston_contract), u32, u64, u64, u32, u64,
                                    P(heston_options), vp], i32),
        "heston_mc_reduce_tiles": ([vp, u64, u32, u64, vp, sz, vp, vp], i32),
        "heston_mc_debug_paths": ([P(heston_params), P(heston_contract), u32, u32, u64,
                                   P(heston_options), P(u64), u32, P(ctypes.c_double),
                                   P(ctypes.c_double)], i32),
        "heston_rng_debug": ([u64, P(u64), P(u32), u32, i32, P(u32), P(ctypes.c_double)], i32),
        "heston_bm64_debug": ([u32, u32, P(ctypes.c_double)], i32),
        "heston_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "heston_batch_plan_make": ([P(heston_batch_item), u32, P(heston_options),
                                    P(heston_batch_plan)], i32),
        "heston_batch_prepare": ([P(heston_batch_item), P(heston_options), P(heston_batch_plan), vp],
                                 i32),
        "heston_mc_launch_batch": ([P(heston_batch_plan), vp, P(heston_options), vp, vp, vp], i32),
        "heston_mc_price_greeks_batch": ([P(heston_batch_item), u32, P(heston_options),
                                          P(heston_result)], i32),
        "heston_adjoint_workspace_bytes": ([u64, u32, P(sz)], i32),
        "heston_mc_adjoint_forward": ([P(heston_params), P(heston_contract), u64, u32, u64,
                                       P(heston_options), vp, sz, vp], i32),
        "heston_mc_adjoint_backward": ([P(heston_params), P(heston_contract), u64, u32, u64,
                                        P(heston_options), vp, sz, vp], i32),
        "heston_mc_adjoint_debug_paths": ([P(heston_params), P(heston_contract), u64, u32, u64,
                                           P(heston_options), vp, sz, vp], i32),
        "heston_release_cached_memory": ([i32], i32),
        "heston_server_create": ([P(heston_server_config), P(vp)], i32),
        "heston_server_submit": ([vp, P(heston_batch_item), P(u64)], i32),
        "heston_server_poll": ([vp, u64, P(heston_result), P(ctypes.c_double)], i32),
        "heston_server_wait": ([vp, u64, u32, P(heston_result), P(ctypes.c_double)], i32),
        "heston_server_stats_get": ([vp, P(heston_server_stats)], i32),
        "heston_server_destroy": ([vp], i32),
        "heston_sobol_directions": ([u32, P(u32)], i32),
        "heston_qmc_tables_bytes": ([u32, P(sz)], i32),
        "heston_qmc_build_tables": ([u32, vp, sz, i32], i32),
        "heston_mc_workspace_bytes_qmc": ([u32, u64, u32, u32, P(sz)], i32),
        "heston_mc_launch_qmc": ([P(heston_params), P(heston_contract), u32, u64, u32, u64,
                                  P(heston_options), vp, vp, sz, vp], i32),
        "heston_qmc_debug_paths": ([P(heston_params), P(heston_contract), u32, u32, u64,
                                    P(heston_options), u32, P(u32), u32, P(ctypes.c_double),
                                    P(ctypes.c_double)], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def heston_status_string(status: int) -> str:
    return load().heston_status_string(status).decode()


def _check(rc: int) -> int:
    if rc < 0:
        raise HestonError(rc, heston_status_string(rc))
    return rc


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "cuda_stream"):
        return x.cuda_stream
    raise TypeError(f"cannot take a device address of {type(x)}")


def make_params(S0, v0, kappa, theta, xi, rho, r) -> heston_params:
    return heston_params(S0, v0, kappa, theta, xi, rho, r)


def make_contract(payoff, K, T, is_put=0, n_monitor=0) -> heston_contract:
    return heston_contract(payoff, is_put, K, T, n_monitor, 0)


def make_options(trunc=HESTON_TRUNC_FULL, prec=HESTON_FP64, stream=None, device=-1, grid_ctas=0,
                 block_threads=0, rng=HESTON_RNG_PHILOX, n_shifts=0,
                 scheme=HESTON_SCHEME_MILSTEIN) -> heston_options:
    return heston_options(trunc, rng, prec, n_shifts, _ptr(stream) or None, device, grid_ctas,
                          block_threads, scheme, 0)


def _contract_array(contracts):
    arr = (heston_contract * len(contracts))()
    for i, c in enumerate(contracts):
        arr[i] = c
    return arr


def heston_mc_price_greeks(params: heston_params, contract: heston_contract, n_paths: int,
                           n_steps: int, rng_seed: int) -> heston_result:
    out = heston_result()
    _check(load().heston_mc_price_greeks(ctypes.byref(params), ctypes.byref(contract), n_paths,
                                         n_steps, rng_seed, ctypes.byref(out)))
    return out


def heston_mc_price_greeks_ex(params, contracts, n_paths, n_steps, rng_seed, options=None):
    """Synchronous multi-contract call; returns a list of heston_result."""
    cs = _contract_array(contracts)
    out = (heston_result * len(contracts))()
    opt = ctypes.byref(options) if options is not None else None
    _check(load().heston_mc_price_greeks_ex(ctypes.byref(params), cs, len(contracts), n_paths,
                                            n_steps, rng_seed, opt, out))
    return list(out)


def heston_mc_workspace_bytes(n_contracts: int, n_paths: int) -> int:
    b = ctypes.c_size_t()
    _check(load().heston_mc_workspace_bytes(n_contracts, n_paths, ctypes.byref(b)))
    return b.value


def heston_mc_launch(params, contracts, n_paths, n_steps, rng_seed, options, workspace,
                     workspace_bytes, out) -> int:
    """Asynchronous launch; ``workspace`` and ``out`` are device buffers."""
    cs = _contract_array(contracts)
    return _check(load().heston_mc_launch(ctypes.byref(params), cs, len(contracts), n_paths,
                                          n_steps, rng_seed, ctypes.byref(options), _ptr(workspace),
                                          workspace_bytes, _ptr(out)))


def heston_mc_launch_noalloc(params, contracts, n_paths, n_steps, rng_seed, options, out) -> int:
    """heston_mc_launch with the library's static device scratch: for callers
    that must not allocate device memory (see include/heston_mc.h).  ``out``
    is a device buffer of 12 doubles per contract."""
    cs = _contract_array(contracts)
    return _check(load().heston_mc_launch_noalloc(ctypes.byref(params), cs, len(contracts),
                                                  n_paths, n_steps, rng_seed,
                                                  ctypes.byref(options), _ptr(out)))


def heston_mc_launch_tiles(params, contracts, path_begin, n_paths, n_steps, rng_seed, options,
                           tile_sums) -> int:
    cs = _contract_array(contracts)
    return _check(load().heston_mc_launch_tiles(ctypes.byref(params), cs, len(contracts),
                                                path_begin, n_paths, n_steps, rng_seed,
                                                ctypes.byref(options), _ptr(tile_sums)))


def heston_mc_reduce_tiles(tile_sums, n_tiles, n_contracts, n_paths_total, workspace,
                           workspace_bytes, out, stream=None) -> int:
    return _check(load().heston_mc_reduce_tiles(_ptr(tile_sums), n_tiles, n_contracts,
                                                n_paths_total, _ptr(workspace), workspace_bytes,
                                                _ptr(out), _ptr(stream) or None))


def heston_mc_debug_paths(params, contracts, n_steps, rng_seed, options, paths):
    """Per-path records (count, 15) and estimators (count, C, 6) as numpy arrays."""
    paths = np.ascontiguousarray(np.asarray(paths, dtype=np.uint64))
    n = len(paths)
    rec = np.zeros((n, len(RECORD_FIELDS)))
    est = np.zeros((n, len(contracts), 6))
    cs = _contract_array(contracts)
    D = ctypes.POINTER(ctypes.c_double)
    _check(load().heston_mc_debug_paths(ctypes.byref(params), cs, len(contracts), n_steps,
                                        rng_seed, ctypes.byref(options),
                                        paths.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), n,
                                        rec.ctypes.data_as(D), est.ctypes.data_as(D)))
    return rec, est


def heston_rng_debug(rng_seed, paths, steps, prec=HESTON_FP64):
    """Philox words (count, 4) and normals (count, 2) computed on the device."""
    paths = np.ascontiguousarray(np.asarray(paths, dtype=np.uint64))
    steps = np.ascontiguousarray(np.asarray(steps, dtype=np.uint32))
    n = len(paths)
    words = np.zeros((n, 4), dtype=np.uint32)
    normals = np.zeros((n, 2))
    _check(load().heston_rng_debug(rng_seed,
                                   paths.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                   steps.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), n, prec,
                                   words.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                   normals.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return words, normals


def heston_bm64_debug(first: int, count: int) -> np.ndarray:
    """(count, 6): ln(n 2^-24) by the FP64 Box-Muller's table method and by
    CUDA's log (n = first + i + 1), then sin and cos of 2 pi g 2^-24 by the
    table method and by CUDA's sincospi (g = first + i)."""
    out = np.zeros((count, 6))
    _check(load().heston_bm64_debug(first, count, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def results_to_arrays(results):
    """(C, 6) means and (C, 6) standard errors from a list of heston_result."""
    m = np.array([[getattr(r, k) for k in ESTIMATORS] for r in results])
    se = np.array([list(r.se) for r in results])
    return m, se


def heston_sobol_directions(n_dims: int) -> np.ndarray:
    """Direction integers built by the library's host code: (n_dims, 32) uint32."""
    out = np.zeros((n_dims, 32), dtype=np.uint32)
    _check(load().heston_sobol_directions(n_dims, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))))
    return out


def heston_qmc_tables_bytes(n_steps: int) -> int:
    b = ctypes.c_size_t()
    _check(load().heston_qmc_tables_bytes(n_steps, ctypes.byref(b)))
    return b.value


def heston_qmc_build_tables(n_steps: int, tables, nbytes: int, device: int = -1) -> int:
    return _check(load().heston_qmc_build_tables(n_steps, _ptr(tables), nbytes, device))


def heston_mc_workspace_bytes_qmc(n_contracts, n_paths, n_steps, n_shifts) -> int:
    b = ctypes.c_size_t()
    _check(load().heston_mc_workspace_bytes_qmc(n_contracts, n_paths, n_steps, n_shifts,
                                                ctypes.byref(b)))
    return b.value


def heston_mc_launch_qmc(params, contracts, n_paths, n_steps, rng_seed, options, tables,
                         workspace, workspace_bytes, out) -> int:
    cs = _contract_array(contracts)
    return _check(load().heston_mc_launch_qmc(ctypes.byref(params), cs, len(contracts), n_paths,
                                              n_steps, rng_seed, ctypes.byref(options),
                                              _ptr(tables), _ptr(workspace), workspace_bytes,
                                              _ptr(out)))


def heston_qmc_debug_paths(params, contracts, n_steps, rng_seed, options, replicate, points):
    points = np.ascontiguousarray(np.asarray(points, dtype=np.uint32))
    n = len(points)
    rec = np.zeros((n, len(RECORD_FIELDS)))
    est = np.zeros((n, len(contracts), 6))
    cs = _contract_array(contracts)
    D = ctypes.POINTER(ctypes.c_double)
    _check(load().heston_qmc_debug_paths(ctypes.byref(params), cs, len(contracts), n_steps,
                                         rng_seed, ctypes.byref(options), replicate,
                                         points.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                         n, rec.ctypes.data_as(D), est.ctypes.data_as(D)))
    return rec, est


def make_batch_item(params: heston_params, contract: heston_contract, n_paths: int, n_steps: int,
                    rng_seed: int) -> heston_batch_item:
    return heston_batch_item(params, contract, n_paths, n_steps, 0, rng_seed)


def _items_array(items):
    arr = (heston_batch_item * len(items))()
    for i, it in enumerate(items):
        arr[i] = it
    return arr


def heston_batch_plan_make(items, options=None) -> heston_batch_plan:
    plan = heston_batch_plan()
    arr = _items_array(items)
    opt = ctypes.byref(options) if options is not None else None
    _check(load().heston_batch_plan_make(arr, len(items), opt, ctypes.byref(plan)))
    return plan


def heston_batch_prepare(items, options, plan, desc) -> int:
    arr = _items_array(items)
    return _check(load().heston_batch_prepare(arr, ctypes.byref(options), ctypes.byref(plan),
                                              _ptr(desc)))


def heston_mc_launch_batch(plan, desc, options, workspace, out, status=None) -> int:
    return _check(load().heston_mc_launch_batch(ctypes.byref(plan), _ptr(desc), ctypes.byref(options),
                                                _ptr(workspace), _ptr(out), _ptr(status) or None))


def heston_mc_price_greeks_batch(items, options=None):
    arr = _items_array(items)
    out = (heston_result * len(items))()
    opt = ctypes.byref(options) if options is not None else None
    _check(load().heston_mc_price_greeks_batch(arr, len(items), opt, out))
    return list(out)


def heston_adjoint_workspace_bytes(n_paths: int, n_steps: int) -> int:
    b = ctypes.c_size_t()
    _check(load().heston_adjoint_workspace_bytes(n_paths, n_steps, ctypes.byref(b)))
    return b.value


def heston_mc_adjoint_forward(params, contract, n_paths, n_steps, rng_seed, options, workspace,
                              workspace_bytes, price) -> int:
    return _check(load().heston_mc_adjoint_forward(ctypes.byref(params), ctypes.byref(contract),
                                                   n_paths, n_steps, rng_seed, ctypes.byref(options),
                                                   _ptr(workspace), workspace_bytes, _ptr(price)))


def heston_mc_adjoint_backward(params, contract, n_paths, n_steps, rng_seed, options, workspace,
                               workspace_bytes, grad) -> int:
    return _check(load().heston_mc_adjoint_backward(ctypes.byref(params), ctypes.byref(contract),
                                                    n_paths, n_steps, rng_seed, ctypes.byref(options),
                                                    _ptr(workspace), workspace_bytes, _ptr(grad)))


def heston_mc_adjoint_debug_paths(params, contract, n_paths, n_steps, rng_seed, options, workspace,
                                  workspace_bytes, per_path) -> int:
    return _check(load().heston_mc_adjoint_debug_paths(ctypes.byref(params), ctypes.byref(contract),
                                                       n_paths, n_steps, rng_seed, ctypes.byref(options),
                                                       _ptr(workspace), workspace_bytes, _ptr(per_path)))


class HestonServer:
    """Handle of a native serving engine (heston_server_* in the C ABI)."""

    def __init__(self, memory_bytes: int, max_active: int = 1024, tiles_per_round: int = 0,
                 trunc: int = HESTON_TRUNC_FULL, device: int = -1):
        cfg = heston_server_config(device, trunc, memory_bytes, max_active, 0, tiles_per_round)
        h = ctypes.c_void_p()
        _check(load().heston_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def submit(self, item: heston_batch_item) -> int:
        t = ctypes.c_uint64()
        _check(load().heston_server_submit(self._h, ctypes.byref(item), ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, timeout_ms: int = 60000):
        """(heston_result, latency seconds), or None on timeout."""
        r = heston_result()
        lat = ctypes.c_double()
        rc = _check(load().heston_server_wait(self._h, ticket, timeout_ms, ctypes.byref(r),
                                              ctypes.byref(lat)))
        return (r, lat.value) if rc == 1 else None

    def poll(self, ticket: int):
        r = heston_result()
        lat = ctypes.c_double()
        rc = _check(load().heston_server_poll(self._h, ticket, ctypes.byref(r), ctypes.byref(lat)))
        return (r, lat.value) if rc == 1 else None

    def stats(self) -> heston_server_stats:
        st = heston_server_stats()
        _check(load().heston_server_stats_get(self._h, ctypes.byref(st)))
        return st

    def close(self):
        if self._h:
            _check(load().heston_server_destroy(self._h))
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def heston_release_cached_memory(device: int = -1) -> None:
    """Return the library's cached stream-ordered scratch to the driver."""
    _check(load().heston_release_cached_memory(device))
