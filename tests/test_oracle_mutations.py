"""Planted mistakes in the CPU oracle are caught by its pins.

Each case copies the oracle (its C source and its Python module), plants one
plausible mistake in the copy (a wrong sign or branch of the propagator, a
swapped index or operand of the level-wise dynamic program, a dropped weight,
term or compensation, a wrong bound, interpolation or enumeration step), builds
the copy with the oracle's own compiler flags, and runs every pin of
``test_oracle_pins.py`` against it: at least one pin must fail.  The unchanged
copy must pass them all.  This checks the pins, not the oracle; it runs on the CPU
only and never touches the oracle that the other tests use.
"""
import importlib.util
import inspect
import os

import pytest

import oracle
import test_oracle_mc as mc_pins
import test_oracle_pins as pins

ORACLE_DIR = os.path.dirname(os.path.abspath(oracle.__file__))
SOURCE = os.path.join(ORACLE_DIR, "cos_oracle.c")
MODULE = os.path.join(ORACLE_DIR, "__init__.py")
MC_MODULE = os.path.join(ORACLE_DIR, "metropolis.py")

# (name, text in cos_oracle.c, replacement, which occurrence)
MUTATIONS = [
    ("propagator: tau = 0 takes the tau < 0 branch", "if (tau >= 0.0) {", "if (tau > 0.0) {", 0),
    ("propagator: antiperiodic branch loses its sign", "    return exp(-eps * shifted)", "    return -exp(-eps * shifted)", 0),
    ("propagator: prefactor exponent sign", "return -exp(-eps * tau) / (1.0 + exp(-beta * eps));",
     "return -exp(-eps * tau) / (1.0 + exp(beta * eps));", 0),
    ("propagator: decay exponent sign", "return -exp(-eps * tau) /", "return -exp(eps * tau) /", 0),
    ("propagator: shift by -beta", "double shifted = tau + beta;", "double shifted = tau - beta;", 0),
    ("walk: source and destination swapped", "v[r[1]] += v[r[0]] * w;", "v[r[0]] += v[r[1]] * w;", 0),
    ("walk: edge weight dropped", "v[r[1]] += v[r[0]] * w;", "v[r[1]] += v[r[0]];", 0),
    ("walk: tau = t_j - t_i", "double tau = ts[r[3]] - ts[r[4]];", "double tau = ts[r[4]] - ts[r[3]];", 0),
    ("walk: fermion-loop sign ignored", "if (r[2] & COS_ORACLE_SIGN_BIT) w = -w;   /* closes a fermion loop */",
     "/* sign ignored */", 0),
    ("walk: A sums signed paths", "a[r[1]] += a[r[0]] * fabs(w);", "a[r[1]] += a[r[0]] * w;", 0),
    ("walk: root holds 2", "v[0] = 1.0;", "v[0] = 2.0;", 0),
    ("walk: result read from the node before the sink", "R[s] = v[N - 1];", "R[s] = v[N - 2];", 0),
    ("path sum: weights of the wrong edge", "node_values[r[1]] += node_values[r[0]] * w[e];",
     "node_values[r[1]] += node_values[r[0]] * w[E - 1 - e];", 0),
    ("count: every edge adds one", "wrap[r[1]] += wrap[r[0]];", "wrap[r[1]] += 1;", 0),
    ("count: overflow flagged past 2^32", "exact[N - 1] > (unsigned __int128)INT64_MAX",
     "exact[N - 1] > (unsigned __int128)UINT32_MAX", 0),
    ("Neumaier: one compensation branch dropped", "if (fabs(sum) >= fabs(y)) c += (sum - u) + y;",
     "if (fabs(sum) >= fabs(y)) c += 0.0;", 0),
    ("long double: tau = 0 takes the tau < 0 branch", "if (ti >= tj) return", "if (ti > tj) return", 0),
    ("long double: antiperiodic branch loses its sign", "return expl(-eps * (tau + beta))",
     "return -expl(-eps * (tau + beta))", 0),
    ("long double: source and destination swapped", "v[r[1]] += v[r[0]] * w;", "v[r[0]] += v[r[1]] * w;", 1),
]


# the same for the oracle's Python module: per-edge factors, tabulated propagators,
# their rounding bound, brute-force enumeration
PY_MUTATIONS = [
    ("edge factors: fermion-loop sign ignored", "    out[(e[:, 2] & SIGN_BIT) != 0] *= -1.0\n    return out",
     "    return out", 0),
    ("edge factors: tau = t_j - t_i", "tau = t_sample[e[:, 3]] - t_sample[e[:, 4]]",
     "tau = t_sample[e[:, 4]] - t_sample[e[:, 3]]", 0),
    ("tabulated: tau = 0 read from the tau < 0 half", "    pos = tau >= 0.0\n    x = tau.astype(ld)",
     "    pos = tau > 0.0\n    x = tau.astype(ld)", 0),
    ("tabulated: negative half shifted the wrong way", "x = np.where(pos, x, x + ld(T))",
     "x = np.where(pos, x, x - ld(T))", 0),
    ("tabulated: halves swapped", "    half = np.where(pos[:, None], table[0][None, :], table[1][None, :])\n    rows",
     "    half = np.where(pos[:, None], table[1][None, :], table[0][None, :])\n    rows", 0),
    ("tabulated: no interpolation", "b = half[rows, m + 1].astype(ld)", "b = half[rows, m].astype(ld)", 0),
    ("tabulated: slope sign", "return (a + f * (b - a)).astype(np.float64)",
     "return (a + f * (a - b)).astype(np.float64)", 0),
    ("tabulated: past the grid takes the last node's left neighbour", "f = np.where(below, 0, np.where(past, 1, f))",
     "f = np.where(below, 0, np.where(past, 0, f))", 0),
    ("tabulated factors: fermion-loop sign ignored",
     "    out[(e[:, 2] & SIGN_BIT) != 0] *= -1.0\n    return (out, sc)", "    return (out, sc)", 0),
    ("tabulated: A is R", "        A[s] = F[-1]", "        A[s] = R[s]", 0),
    ("rounding bound: grid-position term dropped", "UNIT_ROUNDOFF * (4.0 * (np.abs(x) + T)",
     "UNIT_ROUNDOFF * (0.0 * (np.abs(x) + T)", 0),
    ("paths to the sink: parent and child swapped", "weights=w[lo:hi] * out[dst]", "weights=w[lo:hi] * out[src]", 0),
    ("brute force: |path| sums signed paths", "a += abs(prod)", "a += prod", 0),
    ("brute force: paths lose their edges", "stack.append((int(e[q, 1]), path + [q]))",
     "stack.append((int(e[q, 1]), path))", 0),
]


# the same for the Metropolis walkers, against the pins of test_oracle_mc.py
MC_MUTATIONS = [
    ("Metropolis: acceptance rule inverted", "acc = lhs < rhs", "acc = lhs > rhs", 0),
    ("Metropolis: weight |R| replaced by R", "lhs, rhs = u * np.abs(R), np.abs(Rp)", "lhs, rhs = u * R, Rp", 0),
    ("Metropolis: every move accepted", "acc = lhs < rhs", "acc = np.ones(S, dtype=bool)", 0),
    ("Metropolis: last coordinate never proposed", "i = ((w0 * np.uint64(num_times)) >> np.uint64(32))",
     "i = ((w0 * np.uint64(max(num_times - 1, 1))) >> np.uint64(32))", 0),
    ("Metropolis: tally of the proposal", "n_pos += int((R > 0).sum())", "n_pos += int((Rp > 0).sum())", 0),
    ("Metropolis: streams share the sample generator's counters", "0x80000000 | ((step >> 32) & 0x7FFFFFFF)",
     "((step >> 32) & 0x7FFFFFFF)", 0),
    ("Metropolis: proposals in [0, 1) instead of [0, beta)", "return i, beta * x, u", "return i, x, u", 0),
    ("Metropolis: accepted moves not kept", "t[acc] = tp[acc]", "pass", 0),
]


def _plant(text, old, new, which):
    at = -1
    for _ in range(which + 1):
        at = text.index(old, at + 1)          # the occurrence to change must exist
    return text[:at] + new + text[at + len(old):]


def _pin_calls():
    """Every pin of test_oracle_pins as (name, zero-argument call), parametrized ones
    once per parameter value, in name order."""
    calls = []
    for name in dir(pins):
        if not name.startswith("test_"):
            continue
        f = getattr(pins, name)
        params = list(inspect.signature(f).parameters)
        sets = [{}]
        for mark in getattr(f, "pytestmark", []):
            if mark.name == "parametrize":
                arg, values = mark.args
                sets = [{arg: v} for v in values]
        if any(p not in sets[0] for p in params):
            continue
        calls.extend((f"{name}{kw or ''}", (lambda f=f, kw=kw: f(**kw))) for kw in sets)
    return calls


def _oracle_from(src_text, tmp_path, tag, py_text=None):
    """A separate instance of the oracle package whose C library is built from src_text
    (and whose Python module is py_text, when given)."""
    d = tmp_path / tag
    d.mkdir()
    src = d / "cos_oracle.c"
    src.write_text(src_text)
    module = MODULE
    if py_text is not None:
        module = str(d / "oracle_module.py")
        with open(module, "w") as f:
            f.write(py_text)
    spec = importlib.util.spec_from_file_location(f"oracle_{tag}", module)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._SRC, mod._BUILD, mod._LIB_PATH, mod._lib = str(src), str(d), str(d / "libcos_oracle.so"), None
    mod.build()
    return mod


def _failing_pins(mod, monkeypatch, stop_at_first=True):
    monkeypatch.setattr(pins, "oracle", mod)
    failed = []
    for name, call in _pin_calls():
        try:
            call()
        except (AssertionError, ValueError, FloatingPointError):
            failed.append(name)
            if stop_at_first:
                break
    return failed


def test_unchanged_copy_passes_every_pin(tmp_path, monkeypatch):
    with open(SOURCE) as f:
        src = f.read()
    with open(MODULE) as f:
        py = f.read()
    assert len(_pin_calls()) >= 30
    for tag, text in (("control", None), ("control_py", py)):   # the package, then a copied module
        mod = _oracle_from(src, tmp_path, tag, py_text=text)
        assert _failing_pins(mod, monkeypatch, stop_at_first=False) == []


def _mc_module(py_text, tmp_path, tag):
    """A copy of oracle.metropolis built from py_text (its relative import of the
    oracle's evaluate still resolves to the unchanged package)."""
    path = tmp_path / f"{tag}.py"
    path.write_text(py_text)
    spec = importlib.util.spec_from_file_location(f"oracle.metropolis_{tag}", str(path))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _failing_mc_pins(mod, monkeypatch):
    monkeypatch.setattr(mc_pins, "mc", mod)
    failed = []
    for name in dir(mc_pins):
        if name.startswith("test_"):
            try:
                getattr(mc_pins, name)()
            except (AssertionError, ValueError, IndexError, FloatingPointError):
                failed.append(name)
    return failed


def test_unchanged_metropolis_copy_passes_every_pin(tmp_path, monkeypatch):
    with open(MC_MODULE) as f:
        assert _failing_mc_pins(_mc_module(f.read(), tmp_path, "control"), monkeypatch) == []


@pytest.mark.parametrize("name,old,new,which", MC_MUTATIONS, ids=[m[0] for m in MC_MUTATIONS])
def test_planted_metropolis_mistake_fails_a_pin(tmp_path, monkeypatch, name, old, new, which):
    with open(MC_MODULE) as f:
        mod = _mc_module(_plant(f.read(), old, new, which), tmp_path, "mutant")
    assert _failing_mc_pins(mod, monkeypatch), f"no pin catches: {name}"


@pytest.mark.parametrize("name,old,new,which", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, monkeypatch, name, old, new, which):
    with open(SOURCE) as f:
        mod = _oracle_from(_plant(f.read(), old, new, which), tmp_path, "mutant")
    assert _failing_pins(mod, monkeypatch), f"no pin catches: {name}"


@pytest.mark.parametrize("name,old,new,which", PY_MUTATIONS, ids=[m[0] for m in PY_MUTATIONS])
def test_planted_python_mistake_fails_a_pin(tmp_path, monkeypatch, name, old, new, which):
    with open(SOURCE) as f:
        src = f.read()
    with open(MODULE) as f:
        py = _plant(f.read(), old, new, which)
    mod = _oracle_from(src, tmp_path, "mutant", py_text=py)
    assert _failing_pins(mod, monkeypatch), f"no pin catches: {name}"
