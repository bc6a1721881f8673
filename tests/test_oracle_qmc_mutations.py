"""The QMC oracle's pins (tests/test_oracle_qmc.py) catch plausible mistakes in
oracle/sobol.py: each entry plants one mistake in its source (the
direction-number recurrence, the Sobol point bits, Property A, the uniform
mapping, the Brownian bridge's weights and variances, the replicate SE), runs
the mutated module in place of the original, and runs the pins until one
fails.  Every mistake must fail a pin; the unchanged source must pass them
all.  The pin that compares with the library's own direction table is left
out: a pin never leans on the CUDA path.  Conventions that mathematics
cannot fix (which counter tags seed the shifts, which dimension drives which
motion) are not planted: only the comparison with the GPU decides those."""
import contextlib
import importlib
import inspect
import itertools

import pytest

from oracle import sobol

MUTATIONS = [
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

EXCLUDED = {"test_library_direction_table_matches_oracle"}


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


def _pins():
    mod = importlib.import_module("test_oracle_qmc")
    out = []
    for name, fn in inspect.getmembers(mod, inspect.isfunction):
        if not name.startswith("test_") or fn.__module__ != mod.__name__ or name in EXCLUDED:
            continue
        params = set(inspect.signature(fn).parameters)
        for kw in _cases(fn):
            rest = params - set(kw)
            assert rest <= {"V"}, (name, rest)
            out.append((f"{name}{kw or ''}", fn, kw, "V" in rest))
    return out


def _first_failing_pin(pins):
    V = None
    for name, fn, kw, needs_v in pins:
        try:
            if needs_v:
                if V is None:
                    V = sobol.direction_numbers(504)      # the pins' module fixture
                fn(V=V, **kw)
            else:
                fn(**kw)
        except pytest.skip.Exception:
            continue
        except Exception:
            return name
    return None


@contextlib.contextmanager
def _module_source(text):
    """Run `text` in sobol's namespace for the block; restore the original after."""
    original = open(sobol.__file__).read()
    try:
        exec(compile(text, sobol.__file__, "exec"), sobol.__dict__)
        yield
    finally:
        exec(compile(original, sobol.__file__, "exec"), sobol.__dict__)


def test_unchanged_source_passes_every_pin():
    pins = _pins()
    assert len(pins) >= 10
    with _module_source(open(sobol.__file__).read()):
        assert _first_failing_pin(pins) is None


def test_every_planted_mistake_fails_a_pin():
    src = open(sobol.__file__).read()
    pins = _pins()
    survivors = []
    for name, old, new in MUTATIONS:
        assert src.count(old) == 1, name
        with _module_source(src.replace(old, new)):
            if _first_failing_pin(pins) is None:
                survivors.append(name)
    assert not survivors, survivors
