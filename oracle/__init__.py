"""FP64 CPU oracle for Monte Carlo Heston pricing and Greeks (arXiv 2309.10477).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (``paper_2309_10477_gb300``) never imports it and shares no code with it.

Contents:
  * ``heston_oracle.c`` -- Philox4x32-10, Box-Muller, the Milstein scheme of
    Sec. 2.4.2 with full truncation or the paper's floor, the Euler scheme of
    Sec. 2.4.1, Andersen's QE scheme (named in Sec. 5), pathwise tangents,
    per-path estimators and the Monte Carlo driver of Sec. 2.5 (plain C, FP64).
  * ``closed_form`` -- Black-Scholes and the Heston characteristic-function
    price and Greeks (the "real price" the paper quotes in Sec. 3).
  * ``sobol`` -- Sobol points, digital shifts, inverse normal and Brownian
    bridge for the randomised quasi-Monte Carlo variant (Sec. 2.7).
  * ``exact`` -- Broadie-Kaya exact simulation (Sec. 2.2-2.3): noncentral
    chi-square variance step, integrated variance by Fourier inversion of its
    conditional CDF, conditional log-price.

Parity pins live in ``tests/test_oracle_*.py``; functions with no pin say
"parity unpinned" in their docstring.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "heston_oracle.c")
_LIB = os.path.join(_HERE, "liborc_heston.so")
_lock = threading.Lock()
_lib = None

PATH_FIELDS = ("X", "V", "X_v", "V_v", "X_T", "V_T", "sumS", "sumtS", "sumS_Xv",
               "sumS_XT", "GE", "QE", "GA", "QA", "minabsV")
ESTIMATORS = ("price", "delta", "gamma", "vega", "rho", "theta")
TRUNC_FULL, TRUNC_FLOOR = 0, 1
SCHEME_MILSTEIN, SCHEME_EULER, SCHEME_QE = 0, 1, 2
EUROPEAN, ASIAN = 0, 1


def build(force: bool = False) -> str:
    """Compile heston_oracle.c with gcc (-O3, no fast-math, no FMA contraction, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-std=c11", "-O3", "-fno-fast-math", "-ffp-contract=off",
                "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                           capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True)
        os.replace(tmp, _LIB)
        return _LIB


class _Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("S0", "v0", "kappa", "theta", "xi", "rho", "r")]


class _Contract(ctypes.Structure):
    _fields_ = [("payoff", ctypes.c_int32), ("is_put", ctypes.c_int32), ("K", ctypes.c_double),
                ("T", ctypes.c_double), ("n_monitor", ctypes.c_uint32), ("pad_", ctypes.c_uint32)]


def _load():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _configure(lib):
    """Declare the argument and return types of the library's entry points."""
    P = ctypes.POINTER
    d, u32, u64, i32 = ctypes.c_double, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    lib.orc_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
    lib.orc_uniform_pair.argtypes = [u64, u64, u32, u32, P(d), P(d)]
    lib.orc_normal_pair.argtypes = [u64, u64, u32, u32, P(d), P(d)]
    lib.orc_path_normals.argtypes = [u64, u64, u32, u32, P(d), P(d)]
    lib.orc_mc_sums.argtypes = [P(_Params), P(_Contract), u32, u64, u64, u32, u64, i32, i32,
                                i32, P(d), P(d)]
    lib.orc_mc_sums.restype = i32
    lib.orc_mc_sums_perturbed.argtypes = [P(_Params), P(_Contract), u32, u64, u64, u32, u64, i32,
                                          i32, i32, d, d, u64, P(d), P(d)]
    lib.orc_mc_sums_perturbed.restype = i32
    lib.orc_debug_paths.argtypes = [P(_Params), P(_Contract), u32, P(u64), u64, u32, u64, i32,
                                    i32, P(d), P(d)]
    lib.orc_debug_paths.restype = i32
    lib.orc_path_from_normals.argtypes = [P(_Params), P(_Contract), u32, u32, i32, i32, P(d), P(d),
                                          P(d), P(d), P(d), P(d)]
    lib.orc_path_from_normals.restype = i32
    lib.orc_paths_from_normals.argtypes = [P(_Params), P(_Contract), u32, u32, i32, i32, u64,
                                           P(d), P(d), P(d), P(d)]
    lib.orc_paths_from_normals.restype = i32
    lib.orc_mc_gradient.argtypes = [P(_Params), P(_Contract), u64, u32, u64, P(d), P(d)]
    lib.orc_mc_gradient.restype = i32
    lib.orc_debug_gradients.argtypes = [P(_Params), P(_Contract), P(u64), u64, u32, u64, P(d)]
    lib.orc_debug_gradients.restype = i32
    lib.orc_gradients_from_normals.argtypes = [P(_Params), P(_Contract), u32, u64, P(d), P(d), P(d)]
    lib.orc_gradients_from_normals.restype = i32
    lib.orc_max_threads.restype = i32
    lib.orc_set_threads.argtypes = [i32]
    lib.orc_set_threads.restype = None
    return lib


class using_library:
    """Test support: route every oracle call through another build of
    heston_oracle.c (a copy with a mistake planted in it) for the duration of
    a ``with`` block, then restore the library in use before."""

    def __init__(self, path: str):
        self.path = path
        self.saved = None

    def __enter__(self):
        global _lib
        self.saved = _lib
        _lib = _configure(ctypes.CDLL(self.path))
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass(frozen=True)
class Params:
    """Heston parameters of Eq. (heston_eq); ``xi`` is the paper's sigma."""
    S0: float
    v0: float
    kappa: float
    theta: float
    xi: float
    rho: float
    r: float

    def _c(self):
        return _Params(self.S0, self.v0, self.kappa, self.theta, self.xi, self.rho, self.r)

    def replace(self, **kw):
        d = self.__dict__.copy()
        d.update(kw)
        return Params(**d)


@dataclass(frozen=True)
class Contract:
    """payoff: 0 European, 1 arithmetic Asian; n_monitor: M dates (0 = every step)."""
    payoff: int
    K: float
    T: float
    is_put: int = 0
    n_monitor: int = 0


def _contracts(cs):
    arr = (_Contract * len(cs))()
    for i, c in enumerate(cs):
        arr[i] = _Contract(c.payoff, c.is_put, c.K, c.T, c.n_monitor, 0)
    return arr


def philox4x32_10(ctr, key):
    """Raw Philox4x32-10 block: 4 counter words, 2 key words -> 4 words."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def uniform_pair(seed, path, step, stream_tag=0):
    lib = _load()
    a, b = ctypes.c_double(), ctypes.c_double()
    lib.orc_uniform_pair(seed, path, step, stream_tag, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def path_normals(seed, path, n_steps, stream_tag=0):
    """(Za, Zb) arrays of length n_steps for one path under the RNG contract."""
    lib = _load()
    za = np.empty(n_steps)
    zb = np.empty(n_steps)
    lib.orc_path_normals(seed, path, n_steps, stream_tag, _dptr(za), _dptr(zb))
    return za, zb


def _check_rc(rc):
    if rc != 0:
        raise ValueError("oracle rejected the inputs")


def mc_sums(params: Params, contracts, n_paths, n_steps, seed, trunc=TRUNC_FULL,
            path_begin=0, n_threads=0, scheme=SCHEME_MILSTEIN):
    """Sums (sum_x, sum_x^2) per contract and estimator, shape (C, 6) each."""
    lib = _load()
    cs = _contracts(contracts)
    E = 6 * len(contracts)
    s = np.zeros(E)
    s2 = np.zeros(E)
    p = params._c()
    rc = lib.orc_mc_sums(ctypes.byref(p), cs, len(contracts), path_begin, n_paths, n_steps, seed,
                         trunc, scheme, n_threads, _dptr(s), _dptr(s2))
    _check_rc(rc)
    return s.reshape(-1, 6), s2.reshape(-1, 6)


def mc_price_greeks_perturbed(params: Params, contracts, n_paths, n_steps, seed, eps_abs, eps_rel,
                              pert_seed, trunc=TRUNC_FULL, scheme=SCHEME_MILSTEIN, n_threads=0):
    """mc_price_greeks with every normal moved by (eps_abs + eps_rel R) (2U - 1),
    R = sqrt(Za^2 + Zb^2), U from a separate Philox stream keyed by pert_seed:
    a probe of how far the estimates move under perturbations of that size."""
    lib = _load()
    cs = _contracts(contracts)
    E = 6 * len(contracts)
    s = np.zeros(E)
    s2 = np.zeros(E)
    p = params._c()
    rc = lib.orc_mc_sums_perturbed(ctypes.byref(p), cs, len(contracts), 0, n_paths, n_steps, seed,
                                   trunc, scheme, n_threads, eps_abs, eps_rel, pert_seed, _dptr(s),
                                   _dptr(s2))
    _check_rc(rc)
    return mean_se(s.reshape(-1, 6), s2.reshape(-1, 6), n_paths)


def mean_se(s, s2, n):
    """Mean and standard error of the mean from (sum_x, sum_x^2) over n paths."""
    mean = s / n
    var = (s2 - n * mean * mean) / (n - 1)
    return mean, np.sqrt(np.maximum(var, 0.0) / n)


def mc_price_greeks(params: Params, contracts, n_paths, n_steps, seed, trunc=TRUNC_FULL,
                    n_threads=0, scheme=SCHEME_MILSTEIN):
    """Estimates and SEs per contract: two (C, 6) arrays in ESTIMATORS order."""
    s, s2 = mc_sums(params, contracts, n_paths, n_steps, seed, trunc, 0, n_threads, scheme)
    return mean_se(s, s2, n_paths)


def debug_paths(params: Params, contracts, paths, n_steps, seed, trunc=TRUNC_FULL,
                scheme=SCHEME_MILSTEIN):
    """Per-path records (count, 15) in PATH_FIELDS order and estimators (count, C, 6)."""
    lib = _load()
    paths = np.ascontiguousarray(np.asarray(paths, dtype=np.uint64))
    cs = _contracts(contracts)
    rec = np.zeros((len(paths), len(PATH_FIELDS)))
    est = np.zeros((len(paths), len(contracts), 6))
    p = params._c()
    rc = lib.orc_debug_paths(ctypes.byref(p), cs, len(contracts),
                             paths.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), len(paths),
                             n_steps, seed, trunc, scheme, _dptr(rec), _dptr(est))
    _check_rc(rc)
    return rec, est


def path_from_normals(params: Params, contracts, za, zb, trunc=TRUNC_FULL, scheme=SCHEME_MILSTEIN):
    """One path from given normals: (record, estimators (C, 6), X_k, V_k for k=0..N)."""
    lib = _load()
    za = np.ascontiguousarray(za, dtype=np.float64)
    zb = np.ascontiguousarray(zb, dtype=np.float64)
    n = len(za)
    cs = _contracts(contracts)
    rec = np.zeros(len(PATH_FIELDS))
    est = np.zeros((len(contracts), 6))
    tx = np.zeros(n + 1)
    tv = np.zeros(n + 1)
    p = params._c()
    rc = lib.orc_path_from_normals(ctypes.byref(p), cs, len(contracts), n, trunc, scheme, _dptr(za),
                                   _dptr(zb), _dptr(rec), _dptr(est), _dptr(tx), _dptr(tv))
    _check_rc(rc)
    return rec, est, tx, tv


def paths_from_normals(params: Params, contracts, za, zb, trunc=TRUNC_FULL, scheme=SCHEME_MILSTEIN):
    """Many paths from given normals (n_paths, N): records (n, 15) and estimators (n, C, 6)."""
    lib = _load()
    za = np.ascontiguousarray(za, dtype=np.float64)
    zb = np.ascontiguousarray(zb, dtype=np.float64)
    n, N = za.shape
    cs = _contracts(contracts)
    rec = np.zeros((n, len(PATH_FIELDS)))
    est = np.zeros((n, len(contracts), 6))
    p = params._c()
    rc = lib.orc_paths_from_normals(ctypes.byref(p), cs, len(contracts), N, trunc, scheme, n, _dptr(za),
                                    _dptr(zb), _dptr(rec), _dptr(est))
    _check_rc(rc)
    return rec, est


PARAM_NAMES = ("S0", "v0", "kappa", "theta", "xi", "rho", "r")


def mc_gradient(params: Params, contract: Contract, n_paths, n_steps, seed):
    """Price and d price / d (S0, v0, kappa, theta, xi, rho, r) with SEs
    (forward-mode tangents, full truncation): two arrays of 8."""
    lib = _load()
    cs = _contracts([contract])
    mean = np.zeros(8)
    se = np.zeros(8)
    p = params._c()
    _check_rc(lib.orc_mc_gradient(ctypes.byref(p), cs, n_paths, n_steps, seed, _dptr(mean), _dptr(se)))
    return mean, se


def debug_gradients(params: Params, contract: Contract, paths, n_steps, seed):
    """Per-path (payoff, 7 derivatives): (count, 8)."""
    lib = _load()
    paths = np.ascontiguousarray(np.asarray(paths, dtype=np.uint64))
    out = np.zeros((len(paths), 8))
    p = params._c()
    _check_rc(lib.orc_debug_gradients(ctypes.byref(p), _contracts([contract]),
                                      paths.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                      len(paths), n_steps, seed, _dptr(out)))
    return out


def gradients_from_normals(params: Params, contract: Contract, za, zb):
    """Per-path (payoff, 7 derivatives) from given normals (n_paths, N): (n, 8)."""
    lib = _load()
    za = np.ascontiguousarray(za, dtype=np.float64)
    zb = np.ascontiguousarray(zb, dtype=np.float64)
    n, N = za.shape
    out = np.zeros((n, 8))
    p = params._c()
    _check_rc(lib.orc_gradients_from_normals(ctypes.byref(p), _contracts([contract]), N, n, _dptr(za),
                                             _dptr(zb), _dptr(out)))
    return out


def max_threads() -> int:
    return int(_load().orc_max_threads())


def set_threads(n: int) -> None:
    """Threads of later calls that take no count of their own (0: one per core)."""
    _load().orc_set_threads(int(n))
