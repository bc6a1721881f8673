"""The pins of the oracle's Python modules catch plausible mistakes in them:
each entry plants one mistake in a module's source, runs the mutated source
in place of the module, and runs that module's pins until one fails.  Every
mistake must fail a pin; the unchanged source must pass them all.

* oracle/sobol.py (pins: tests/test_oracle_qmc.py): the direction-number
  recurrence, the Sobol point bits, Property A, the uniform mapping, the
  Brownian bridge's weights and variances, the replicate SE.  The pin that
  compares with the library's own direction table is left out: a pin never
  leans on the CUDA path.  Conventions that mathematics cannot fix (which
  counter tags seed the shifts, which dimension drives which motion) are not
  planted: only the comparison with the GPU decides those.
* oracle/closed_form.py (pins: tests/test_oracle_closed_form.py): the Heston
  characteristic function, the two probabilities and the Greeks assembled
  from them, Black-Scholes with a total variance.
* oracle/exact.py (pins: tests/test_oracle_exact.py): the gamma and
  noncentral chi-square samplers, the integrated variance's characteristic
  function, the log-price given the variance path, the Delta/Rho estimators.
  Two changes that look like mistakes are not: Marsaglia-Tsang with a larger
  c stays an exact rejection sampler (its acceptance ratio stays <= 1), and
  conjugating the characteristic function leaves the CDF inversion, which
  uses its real part only, unchanged."""
import contextlib
import importlib
import inspect
import itertools

import pytest

from oracle import closed_form, exact, sobol

SOBOL_MUTATIONS = [
    ("recurrence without m_(k-s)", "        val = m[k - s] ^ (m[k - s] << s)", "        val = m[k - s] << s"),
    ("recurrence term shifted", "                val ^= m[k - i] << i", "                val ^= m[k - i] << (i + 1)"),
    ("dimension 0 reversed", "    V[0] = [1 << (31 - k) for k in range(32)]",
     "    V[0] = [1 << (31 - k) for k in reversed(range(32))]"),
    ("point bits read two at a time", "sel = ((idx >> np.uint64(b)) & np.uint64(1)).astype(bool)",
     "sel = ((idx >> np.uint64(b)) & np.uint64(3)).astype(bool)"),
    ("Property A not enforced", "        if j < 32:", "        if j < 1:"),
    ("first digit read from the second bit", "row |= ((v[k] >> 31) & 1) << k", "row |= ((v[k] >> 30) & 1) << k"),
    ("primitivity not checked", "    return all(_gf2_powmod(0b10, order // q, poly, deg) != 1 for q in _prime_factors(order))",
     "    return True"),
    ("uniform offset one", "return ((y >> np.uint32(8)).astype(np.float64) + 0.5) * 2.0**-24",
     "return ((y >> np.uint32(8)).astype(np.float64) + 1.0) * 2.0**-24"),
    ("bridge standard deviation", "+ np.sqrt((m - l) * (r - m) / (r - l)) * z[:, j])",
     "+ np.sqrt((m - l) * (r - m)) / (r - l) * z[:, j])"),
    ("bridge weight from the wrong end", "W[:, l] + (m - l) / (r - l) * (W[:, r] - W[:, l])",
     "W[:, l] + (r - m) / (r - l) * (W[:, r] - W[:, l])"),
    ("bridge end point without the square root", "W[:, self.N] = np.sqrt(self.N) * z[:, 0]",
     "W[:, self.N] = self.N * z[:, 0]"),
    ("step normals as levels", "return np.diff(self.build(z), axis=1)", "return self.build(z)[:, 1:]"),
    ("replicate SE over R", "se = reps.std(axis=0, ddof=1) / np.sqrt(n_shifts)",
     "se = reps.std(axis=0, ddof=1) / n_shifts"),
]

CLOSED_FORM_MUTATIONS = [
    ("cf: b sign", "    b = kappa - rho * xi * iw", "    b = kappa + rho * xi * iw"),
    ("cf: d with -w^2", "    d = np.sqrt(b * b + xi * xi * (iw + w * w))", "    d = np.sqrt(b * b + xi * xi * (iw - w * w))"),
    ("cf: log term without the 2", "(b - d) * T - 2.0 * np.log((1.0 - g * e) / (1.0 - g)))",
     "(b - d) * T - np.log((1.0 - g * e) / (1.0 - g)))"),
    ("cf: D with 1 + e", "Dv = ((b - d) / (xi * xi)) * (1.0 - e) / (1.0 - g * e)",
     "Dv = ((b - d) / (xi * xi)) * (1.0 + e) / (1.0 - g * e)"),
    ("P1 normalised by S0", "            phi = phi / fwd", "            phi = phi / S0"),
    ("integrand without the i", "return (np.exp(-1j * u * lnK) * val / (1j * u)).real",
     "return (np.exp(-1j * u * lnK) * val / u).real"),
    ("Heston Rho without T", "rho=K * T * D * P2", "rho=K * D * P2"),
    ("Heston Vega sign", "    vega = S0 * dP1 - K * D * dP2", "    vega = S0 * dP1 + K * D * dP2"),
    ("Richardson weights", "        return (4 * c2 - c1) / 3", "        return (4 * c2 - c1) / 4"),
    ("BS d1 sign of the variance", "    d1 = (math.log(S0 / K) + r * T + 0.5 * w) / sw",
     "    d1 = (math.log(S0 / K) + r * T - 0.5 * w) / sw"),
    ("BS Gamma over S0 squared", "    gamma = _npdf(d1) / (S0 * sw)", "    gamma = _npdf(d1) / (S0 * S0 * sw)"),
    ("BS put Rho on d2", "        rho = -K * T * D * ndtr(-d2)", "        rho = -K * T * D * ndtr(d2)"),
]


EXACT_MUTATIONS = [
    ("gamma: d = a - 1/2", "    d = a - 1.0 / 3.0", "    d = a - 1.0 / 2.0"),
    ("gamma: small-shape boost inverted", "out[small] *= u ** (1.0 / shape[small])", "out[small] *= u ** shape[small]"),
    ("CIR scale over 2 kappa", "    c = xi * xi * (1.0 - e) / (4.0 * kappa)", "    c = xi * xi * (1.0 - e) / (2.0 * kappa)"),
    ("CIR degrees of freedom halved", "    d = 4.0 * kappa * theta / (xi * xi)\n    lam",
     "    d = 2.0 * kappa * theta / (xi * xi)\n    lam"),
    ("CIR noncentral term without the root", "return c * (chi + (z + np.sqrt(lam)) ** 2)", "return c * (chi + (z + lam) ** 2)"),
    ("CIR Poisson mean doubled", "n = rng.poisson(0.5 * lam)", "n = rng.poisson(lam)"),
    ("integrated variance: g without the 2", "g = np.sqrt(kappa * kappa - 2.0 * xi * xi * 1j * a)",
     "g = np.sqrt(kappa * kappa - xi * xi * 1j * a)"),
    ("log-price drift without the half", "lnS = lnS + p.r * dt - 0.5 * Ii + p.rho * w2",
     "lnS = lnS + p.r * dt - Ii + p.rho * w2"),
    ("w2 sign of kappa I", "w2 = (Vt - V - p.kappa * p.theta * dt + p.kappa * Ii) / p.xi",
     "w2 = (Vt - V - p.kappa * p.theta * dt - p.kappa * Ii) / p.xi"),
    ("Rho without the discount term", "    rho = D * ind * dAr - T * price", "    rho = D * ind * dAr"),
    ("Asian Rho weight as T", "        dAr = (S * t[None, :]).mean(axis=1)", "        dAr = T * S.mean(axis=1)"),
]

# module: (its mutations, the pin module, pins left out, fixtures the pins take,
# pins to run first, in this order -- the cheapest; the rest follow in source order)
MODULES = {
    "sobol": (sobol, SOBOL_MUTATIONS, "test_oracle_qmc", {"test_library_direction_table_matches_oracle"},
              {"V": lambda: sobol.direction_numbers(504)}, []),
    "closed_form": (closed_form, CLOSED_FORM_MUTATIONS, "test_oracle_closed_form", set(), {}, []),
    # the martingale pin (13 s) catches none of these that the others miss; it runs in its own file
    "exact": (exact, EXACT_MUTATIONS, "test_oracle_exact", {"test_exact_paths_are_discounted_martingales"}, {},
              ["test_marsaglia_tsang_gamma", "test_cir_transition_moments",
               "test_characteristic_function_and_integrated_variance_mean",
               "test_exact_european_matches_closed_form", "test_exact_asian_matches_paper_exact_simulation"]),
}


def _cases(fn):
    axes = []
    for m in getattr(fn, "pytestmark", []):
        if m.name != "parametrize":
            continue
        names = m.args[0]
        names = [a.strip() for a in names.split(",")] if isinstance(names, str) else list(names)
        axes.append([dict(zip(names, v)) if len(names) > 1 else {names[0]: v} for v in m.args[1]])
    for combo in itertools.product(*axes):
        kw = {}
        for d in combo:
            kw.update(d)
        yield kw


def _pins(pin_module, excluded, fixtures, first=()):
    mod = importlib.import_module(pin_module)
    out = []
    fns = [(n, f) for n, f in inspect.getmembers(mod, inspect.isfunction)
           if n.startswith("test_") and f.__module__ == mod.__name__ and n not in excluded]
    fns.sort(key=lambda nf: (list(first).index(nf[0]) if nf[0] in first else len(first),
                             nf[1].__code__.co_firstlineno))
    for name, fn in fns:
        params = set(inspect.signature(fn).parameters)
        for kw in _cases(fn):
            rest = params - set(kw)
            assert rest <= set(fixtures), (name, rest)
            out.append((f"{name}{kw or ''}", fn, kw, sorted(rest)))
    return out


def _first_failing_pin(pins, fixtures):
    """The first pin that fails with the module's current source, or None.
    Fixtures are made once, from the current source, when a pin first needs one."""
    made = {}
    for name, fn, kw, needs in pins:
        try:
            for f in needs:
                if f not in made:
                    made[f] = fixtures[f]()
            fn(**kw, **{f: made[f] for f in needs})
        except pytest.skip.Exception:
            continue
        except Exception:                      # an assertion or an error: the pin caught it
            return name
    return None


@contextlib.contextmanager
def _module_source(module, text):
    """Run `text` in the module's namespace for the block; restore the original after."""
    original = open(module.__file__).read()
    try:
        exec(compile(text, module.__file__, "exec"), module.__dict__)
        yield
    finally:
        exec(compile(original, module.__file__, "exec"), module.__dict__)


@pytest.mark.parametrize("which", sorted(MODULES))
def test_unchanged_source_passes_every_pin(which):
    module, _, pin_module, excluded, fixtures, first = MODULES[which]
    pins = _pins(pin_module, excluded, fixtures, first)
    assert len(pins) >= 5
    with _module_source(module, open(module.__file__).read()):
        assert _first_failing_pin(pins, fixtures) is None


@pytest.mark.parametrize("which", sorted(MODULES))
def test_every_planted_mistake_fails_a_pin(which):
    module, mutations, pin_module, excluded, fixtures, first = MODULES[which]
    src = open(module.__file__).read()
    pins = _pins(pin_module, excluded, fixtures, first)
    survivors = []
    for name, old, new in mutations:
        assert src.count(old) == 1, name
        with _module_source(module, src.replace(old, new)):
            if _first_failing_pin(pins, fixtures) is None:
                survivors.append(name)
    assert not survivors, survivors
