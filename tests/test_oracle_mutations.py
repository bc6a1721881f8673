"""The oracle's pins catch plausible mistakes: each entry below plants one
mistake in a copy of oracle/heston_oracle.c (a dropped term, a wrong sign,
index or operand, a wrong constant, the paper's printed Asian Rho), builds it,
routes the oracle through that build, and runs the oracle's own pin tests
(brute force by hand, the RNG against cuRAND's host generator, the two-date
Asian integral, the parameter gradient against finite differences and the
closed form, the schemes' closed forms, moments and finite differences)
until one fails.
Every mistake must fail at least one pin; the unchanged copy must pass all
of them."""
import concurrent.futures
import inspect
import itertools
import os
import shutil
import subprocess

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "heston_oracle.c")

# (name, text in heston_oracle.c, replacement): each text occurs exactly once.
MUTATIONS = [
    # Philox4x32-10
    ("philox multiplier", "#define ORC_PHILOX_M0 0xD2511F53u", "#define ORC_PHILOX_M0 0xD2511F55u"),
    ("philox key increment", "#define ORC_PHILOX_W1 0xBB67AE85u", "#define ORC_PHILOX_W1 0xBB67AE86u"),
    ("philox nine rounds", "round < 10", "round < 9"),
    ("philox key schedule late", "if (round > 0) {", "if (round > 1) {"),
    ("philox high and low swapped", "uint32_t y1 = lo1;", "uint32_t y1 = hi1;"),
    ("philox wrong xor word", "uint32_t y2 = hi0 ^ x3 ^ k1;", "uint32_t y2 = hi0 ^ x1 ^ k1;"),
    # counter and uniforms
    ("counter step not halved", "step / 2u, (uint32_t)path", "step, (uint32_t)path"),
    ("odd step takes the wrong word", "uint32_t a = (step & 1u) ? x[2] : x[0];",
     "uint32_t a = (step & 1u) ? x[3] : x[0];"),
    ("u1 without the offset", "ldexp((double)((a >> 8) + 1u), -24)", "ldexp((double)(a >> 8), -24)"),
    ("u2 from 25 bits", "ldexp((double)(b >> 8), -24)", "ldexp((double)(b >> 7), -25)"),
    # Box-Muller
    ("Za from the sine", "*za = rad * cos(ORC_TWO_PI * u2);", "*za = rad * sin(ORC_TWO_PI * u2);"),
    ("radius without the factor 2", "double rad = sqrt(-2.0 * log(u1));", "double rad = sqrt(-log(u1));"),
    # correlation and Gamma's W
    ("correlation operands transposed", "const double Z2 = p->rho * Z1 + sq * Zb[k];",
     "const double Z2 = p->rho * Zb[k] + sq * Z1;"),
    ("W sign", "const double W = sq * Za[k] - p->rho * Zb[k];", "const double W = sq * Za[k] + p->rho * Zb[k];"),
    # log-price step
    ("drift without the half", "Xn = X + (p->r - 0.5 * Vp) * dt + u * Z1;", "Xn = X + (p->r - Vp) * dt + u * Z1;"),
    ("log-price driven by Z2", "Xn = X + (p->r - 0.5 * Vp) * dt + u * Z1;", "Xn = X + (p->r - 0.5 * Vp) * dt + u * Z2;"),
    # variance step, full truncation
    ("Milstein term doubled", "                     + 0.25 * p->xi * p->xi * dt * (Z2 * Z2 - 1.0) * mil;",
     "                     + 0.5 * p->xi * p->xi * dt * (Z2 * Z2 - 1.0) * mil;"),
    ("drift on the raw state", "Vn = V + p->kappa * (p->theta - Vp) * dt", "Vn = V + p->kappa * (p->theta - V) * dt"),
    ("Milstein term not gated at V = 0", "const double mil = pos ? mil_on : 0.0;", "const double mil = mil_on;"),
    # paper's floor
    ("floor not applied", "Vn = keep ? Vt : 0.0;", "Vn = Vt;"),
    # tangents
    ("v0-tangent of V driven by Z1", "Vn_v = V_v - p->kappa * Vp_v * dt + p->xi * u_v * Z2;",
     "Vn_v = V_v - p->kappa * Vp_v * dt + p->xi * u_v * Z1;"),
    ("du/dv0 without the half", "(Vp_v * dt) / (2.0 * u)", "(Vp_v * dt) / u"),
    ("du/dT without d(dt)/dT", "(Vp_T * dt + Vp * ddt) / (2.0 * u)", "(Vp_T * dt) / (2.0 * u)"),
    ("dX/dT without the drift term", "Xn_T = X_T + (p->r - 0.5 * Vp) * ddt - 0.5 * Vp_T * dt + u_T * Z1;",
     "Xn_T = X_T - 0.5 * Vp_T * dt + u_T * Z1;"),
    ("dV/dT without the mean-reversion term",
     "Vn_T = V_T + p->kappa * (p->theta - Vp) * ddt - p->kappa * Vp_T * dt",
     "Vn_T = V_T - p->kappa * Vp_T * dt"),
    # Gamma weights
    ("Gamma weight on Za", "GE += u * W;", "GE += u * Za[k];"),
    ("Gamma window one step long", "if (k < stride) { GA += u * W; QA += Vp * dt; }",
     "if (k <= stride) { GA += u * W; QA += Vp * dt; }"),
    # Asian dates
    ("date time one step early", "const double t = (double)(k + 1) * dt;", "const double t = (double)k * dt;"),
    ("dates shifted", "if ((k + 1) % stride == 0) {", "if (k % stride == 0) {"),
    ("T-tangent sum from the v0-tangent", "sumS_XT += S * X_T;", "sumS_XT += S * X_v;"),
    # estimators
    ("European Delta undiscounted", "est[1] = D * (ST / S0) * ind;", "est[1] = (ST / S0) * ind;"),
    ("European Gamma without the -1", "est[2] = D * ind * (ST / (S0 * S0)) * (lr - 1.0);",
     "est[2] = D * ind * (ST / (S0 * S0)) * lr;"),
    ("Gamma weight without sqrt(1 - rho^2)", "const double lr = w->GE / (sq * w->QE);",
     "const double lr = w->GE / w->QE;"),
    ("European Rho with S_T", "est[4] = D * K * T * ind;", "est[4] = D * ST * T * ind;"),
    ("European Theta sign", "est[5] = r * est[0] - D * ind * ST * w->X_T;",
     "est[5] = r * est[0] + D * ind * ST * w->X_T;"),
    ("European put payoff reversed", "est[0] = D * (ST < K ? K - ST : 0.0);", "est[0] = D * (ST < K ? ST - K : 0.0);"),
    ("the paper's printed Asian Rho", "est[4] = D * ind * (tSbar - T * (Sbar - K));",
     "est[4] = D * K * T * ind * (tSbar - T * (Sbar - K));"),
    ("Asian Gamma over all steps", "const double lr = w->GA / (sq * w->QA);", "const double lr = w->GE / (sq * w->QE);"),
    ("Asian put Delta sign", "est[1] = -D * (Sbar / S0) * ind;", "est[1] = D * (Sbar / S0) * ind;"),
    ("Asian Vega from the T-tangent", "est[3] = D * ind * dSbar_v;", "est[3] = D * ind * dSbar_T;"),
    # Euler and Andersen's QE
    ("Euler with the Milstein term", "const double mil_on = scheme == ORC_SCHEME_MILSTEIN ? 1.0 : 0.0;",
     "const double mil_on = 1.0;"),
    ("QE quadratic root sign", "const double b2 = y - 1.0 + root;", "const double b2 = y - 1.0 - root;"),
    ("QE exponential rate", "const double beta = (1.0 - pr) / m;", "const double beta = (1.0 + pr) / m;"),
    ("QE log-price K2 sign", "const double K2 = 0.5 * dt * (p->kappa * p->rho / p->xi - 0.5) + p->rho / p->xi;",
     "const double K2 = 0.5 * dt * (p->kappa * p->rho / p->xi - 0.5) - p->rho / p->xi;"),
    ("QE Gamma scale without the half", "const double ut = sqrt(0.5 * dt * (V + Vn));",
     "const double ut = sqrt(dt * (V + Vn));"),
    ("QE v0-tangent without the factor 2", "*Vn_v = a_v * (b + Za) * (b + Za) + 2.0 * a * (b + Za) * b_v;",
     "*Vn_v = a_v * (b + Za) * (b + Za) + a * (b + Za) * b_v;"),
    # the forward-mode parameter gradient (the adjoint kernel's reference)
    ("gradient dZ2/drho sign", "const double dZ2 = (i == 5) ? za - (p->rho / sq) * zb : 0.0;",
     "const double dZ2 = (i == 5) ? za + (p->rho / sq) * zb : 0.0;"),
    ("gradient drift without r", "nX[i] = dX[i] + dr * dt - 0.5 * dVp * dt + du * za;",
     "nX[i] = dX[i] - 0.5 * dVp * dt + du * za;"),
    ("gradient Milstein xi-term halved", "+ (0.5 * p->xi * dxi * dt * (Z2 * Z2 - 1.0)",
     "+ (0.25 * p->xi * dxi * dt * (Z2 * Z2 - 1.0)"),
    ("gradient without the discount derivative", "grad[6] += -T * D * phi;", "grad[6] += 0.0 * T * D * phi;"),
    ("gradient S0 scaling missing", "dAval[0] += Aval / p->S0;", "dAval[0] += 0.0;"),
    # Monte Carlo sums
    ("sum of squares without the square", "s[E + c * 6 + e] += est[e] * est[e];", "s[E + c * 6 + e] += est[e];"),
    ("path index without its range start", "orc_path_normals(seed, path_begin + i, N, 0u, Za, Zb);",
     "orc_path_normals(seed, i, N, 0u, Za, Zb);"),
]

# The pin tests run against each mutant, fastest first.
PIN_MODULES = ["test_oracle_brute_force", "test_oracle_rng", "test_oracle_asian_two_dates",
               "test_oracle_gradient", "test_oracle_schemes", "test_oracle_scheme"]


def _cases(fn):
    """Keyword arguments of every parametrized case of a test function."""
    axes = []
    for m in getattr(fn, "pytestmark", []):
        if m.name != "parametrize":
            continue
        names = m.args[0]
        names = [a.strip() for a in names.split(",")] if isinstance(names, str) else list(names)
        cases = []
        for v in m.args[1]:
            if hasattr(v, "values"):                   # pytest.param(...)
                v = v.values if len(names) > 1 else v.values[0]
            cases.append(dict(zip(names, v)) if len(names) > 1 else {names[0]: v})
        axes.append(cases)
    for combo in itertools.product(*axes):
        kw = {}
        for d in combo:
            kw.update(d)
        yield kw


def _pins():
    import importlib
    out = []
    for mod_name in PIN_MODULES:
        mod = importlib.import_module(mod_name)
        for name, fn in inspect.getmembers(mod, inspect.isfunction):
            if not name.startswith("test_") or fn.__module__ != mod_name:
                continue
            params = set(inspect.signature(fn).parameters)
            for kw in _cases(fn):
                if set(kw) == params:
                    out.append((f"{mod_name}::{name}{kw or ''}", fn, kw))
    return out


def _first_failing_pin(pins):
    """The name of the first pin that fails with the library in use, or None."""
    for name, fn, kw in pins:
        try:
            fn(**kw)
        except pytest.skip.Exception:
            continue
        except Exception:                      # an assertion or an error: the pin caught it
            return name
    return None


def _build(src_text, path):
    c = path + ".c"
    with open(c, "w") as f:
        f.write(src_text)
    base = ["gcc", "-std=c11", "-O1", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared", c, "-o", path, "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True)
    if r.returncode != 0:
        subprocess.run(base, check=True, capture_output=True)
    return path


@pytest.fixture(scope="module")
def builds(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc is needed to build the planted copies")
    src = open(SRC).read()
    d = str(tmp_path_factory.mktemp("oracle_mutants"))
    jobs = {"unchanged": src}
    for i, (name, old, new) in enumerate(MUTATIONS):
        assert src.count(old) == 1, name
        jobs[name] = src.replace(old, new)
    with concurrent.futures.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        futs = {name: ex.submit(_build, text, os.path.join(d, f"m{i:02d}.so"))
                for i, (name, text) in enumerate(jobs.items())}
        return {name: f.result() for name, f in futs.items()}


def test_unchanged_copy_passes_every_pin(builds):
    pins = _pins()
    assert len(pins) >= 60
    with oracle.using_library(builds["unchanged"]):
        assert _first_failing_pin(pins) is None


def test_every_planted_mistake_fails_a_pin(builds):
    pins = _pins()
    survivors = []
    for name, _, _ in MUTATIONS:
        with oracle.using_library(builds[name]):
            if _first_failing_pin(pins) is None:
                survivors.append(name)
    assert not survivors, survivors
