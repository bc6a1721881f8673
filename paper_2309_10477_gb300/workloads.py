"""Seeded synthetic workloads (parameter sets and contract lists).

Holds none of the method's arithmetic: only the inputs that the CUDA path,
the tests and the benchmark share.  Every workload is parametric; no dataset
is involved.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

EUROPEAN, ASIAN = 0, 1


@dataclass(frozen=True)
class Workload:
    name: str
    params: dict            # S0, v0, kappa, theta, xi, rho, r
    contracts: tuple        # (payoff, K, T, is_put, n_monitor) tuples
    n_paths: int
    n_steps: int
    seed: int
    prec: str               # "fp32" or "fp64"
    trunc: str = "full"
    extra: dict = field(default_factory=dict)


# Heston parameters shared by the single-contract and multi-strike workloads.
BASE_PARAMS = dict(S0=100.0, v0=0.04, kappa=2.0, theta=0.04, xi=0.3, rho=-0.7, r=0.05)

# The paper's Table "Heston model parameters" with rho = -0.7 (the table omits
# rho; -0.7 reproduces the printed analytic values).
PAPER_PARAMS = dict(S0=100.0, v0=0.010201, kappa=6.21, theta=0.019, xi=0.61, rho=-0.7, r=0.0319)


def single_european_fp64() -> Workload:
    """One European call, 100 steps, 2^16 paths, FP64 path."""
    return Workload("european_call_k100_n100_p2^16_fp64", BASE_PARAMS,
                    ((EUROPEAN, 100.0, 1.0, 0, 0),), 1 << 16, 100, 42, "fp64")


def multi_strike_fp32(n_paths: int = 1 << 22) -> Workload:
    """European + arithmetic Asian (252 equal dates) x K in {90, 100, 110},
    252 steps, FP32 path with FP64 sums: 36 estimates on one set of paths."""
    cs = tuple((pay, K, 1.0, 0, 252 if pay == ASIAN else 0)
               for pay in (EUROPEAN, ASIAN) for K in (90.0, 100.0, 110.0))
    return Workload(f"euro+asian252_k90-100-110_n252_p2^{n_paths.bit_length() - 1}_fp32",
                    BASE_PARAMS, cs, n_paths, 252, 42, "fp32")


def paper_asian_4_dates() -> Workload:
    """The paper's Asian experiment: 4 dates [0.25, 0.5, 0.75, 1], 128 steps."""
    return Workload("paper_asian4_n128", PAPER_PARAMS,
                    ((ASIAN, 100.0, 1.0, 0, 4), (EUROPEAN, 100.0, 1.0, 0, 0)), 32000, 128, 7, "fp32")


def batched_contracts(n: int = 1024, seed: int = 42):
    """Uneven contract mix: K~U[70,130], T in {0.25,0.5,1,2}, kappa~U[0.5,5],
    theta, v0~U[0.01,0.09], xi~U[0.1,1], rho~U[-0.9,0], r~U[0,0.06],
    paths 2^U (U~U[14,20]) rounded to 256, steps U{50..500}, European / Asian
    50/50 (Asian M = N).  Returns a list of dicts."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        p = dict(S0=100.0, v0=float(g.uniform(0.01, 0.09)), kappa=float(g.uniform(0.5, 5.0)),
                 theta=float(g.uniform(0.01, 0.09)), xi=float(g.uniform(0.1, 1.0)),
                 rho=float(g.uniform(-0.9, 0.0)), r=float(g.uniform(0.0, 0.06)))
        T = float(g.choice([0.25, 0.5, 1.0, 2.0]))
        K = float(g.uniform(70.0, 130.0))
        n_paths = int(round(2.0 ** g.uniform(14.0, 20.0) / 256.0)) * 256
        n_steps = int(g.integers(50, 501))
        payoff = int(g.integers(0, 2))
        out.append(dict(params=p, contract=(payoff, K, T, 0, 0), n_paths=max(n_paths, 256),
                        n_steps=n_steps))
    return out


def serving_requests(n: int, seed: int = 2309):
    """Serving stream requests: contracts drawn as in batched_contracts (same
    parameter and contract distributions), paths 2^U with U~U[16,22] rounded
    to 256, steps U{50..252}.  Returns a list of dicts like batched_contracts."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for d in batched_contracts(n, seed=seed + 1):
        n_paths = int(round(2.0 ** g.uniform(16.0, 22.0) / 256.0)) * 256
        d = dict(d, n_paths=max(n_paths, 256), n_steps=int(g.integers(50, 253)))
        out.append(d)
    return out
