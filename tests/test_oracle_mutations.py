"""The oracle's pins catch plausible mistakes (mutation tests, CPU only).

Each case copies oracle.c, plants one mistake of the kind a reader could make
when writing Secs. II.B-II.C (a sign flip, a neighbour index swapped, a table
looked up on the wrong abscissa, masses swapped in Eq. 2.8, ...), compiles the
copy with the same flags, routes the oracle module to it and runs the pins of
``test_fluid_pins.py``.  At least one pin must fail for every mutant; the
unmutated source passes them all (the ordinary test run).
"""
import concurrent.futures as cf
import importlib.util
import inspect
import os

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))

# (name, text in oracle.c, replacement): each text occurs exactly once
MUTANTS = [
    ("advection coefficient of j-1, sign", "a[k] = -h * A[j - 1];", "a[k] = h * A[j - 1];"),
    ("advection coefficient of j+1, sign", "c[k] = h * A[j + 1];", "c[k] = -h * A[j + 1];"),
    ("advection ratio A_{j-1} -> A_j", "a[k] = -h * A[j - 1];", "a[k] = -h * A[j];"),
    ("advection ratio A_{j+1} -> A_j", "c[k] = h * A[j + 1];", "c[k] = h * A[j];"),
    ("pressure term sign", "E[j] * dt / s->m_ion -\n", "E[j] * dt / s->m_ion +\n"),
    ("pressure term, T of the other neighbour",
     "ni[j + 1] * T[j + 1] - ni[j - 1] * T[j - 1]", "ni[j + 1] * T[j - 1] - ni[j - 1] * T[j + 1]"),
    ("exchange frequency on the E/N abscissa",
     "return interp_lin(s->tab_u, s->tab_nu, s->p.n_tab, u_abs);",
     "return interp_lin(s->tab_eon, s->tab_nu, s->p.n_tab, u_abs);"),
    ("exchange frequency at the new-level flux", "double nu = exch_freq(s, fabs(A[j]));",
     "double nu = exch_freq(s, fabs(gam[j]));"),
    ("collision term, implicit half dropped", "b[k] = 1.0 + nu * dt / 2.0;", "b[k] = 1.0 + nu * dt;"),
    ("mobility abscissa without the Td scale", "double eon_td = e_abs / s->ngas * 1e21;",
     "double eon_td = e_abs / s->ngas;"),
    ("Eq. 2.8 masses swapped in the factor", "return t + (mi + mn) / (5.0 * mi + 3.0 * mn) * mn",
     "return t + (mi + mn) / (5.0 * mn + 3.0 * mi) * mn"),
    ("Eq. 2.8 ion mass for the neutral one", "(mi + mn) / (5.0 * mi + 3.0 * mn) * mn * ud * ud",
     "(mi + mn) / (5.0 * mi + 3.0 * mn) * mi * ud * ud"),
    ("Eq. 2.7 diffusion without the field-heated temperature",
     "double D = mu * ion_temp(s, mu, fabs(E[j])) / Q_E;", "double D = mu * K_B * s->p.gas_temp_k / Q_E;"),
    ("drift-diffusion gradient over one cell",
     "gnew[j] = mu * ni[j] * E[j] - D * (ni[j + 1] - ni[j - 1]) / (2.0 * dz);",
     "gnew[j] = mu * ni[j] * E[j] - D * (ni[j + 1] - ni[j - 1]) / dz;"),
    ("wall flux with |E|", "return mobility(s, fabs(E)) * n * E;", "return mobility(s, fabs(E)) * n * fabs(E);"),
    ("wall flux alpha switch reversed", "int into = wall == 0 ? (E < 0.0) : (E > 0.0);",
     "int into = wall == 0 ? (E > 0.0) : (E < 0.0);"),
    ("wall row of Eq. 2.4 over a full cell", "nnew[0] = ni[0] - dt / dz * (gnew[1] - gnew[0]) + dt * gsrc[0];",
     "nnew[0] = ni[0] - dt / (2.0 * dz) * (gnew[1] - gnew[0]) + dt * gsrc[0];"),
    ("density floor ignored", "A[j] = ni[j] >= s->n_floor ? gam[j] / ni[j] : 0.0;",
     "A[j] = ni[j] > 0.0 ? gam[j] / ni[j] : 0.0;"),
]


def _pins():
    spec = importlib.util.spec_from_file_location("fluid_pins_for_mutants", os.path.join(HERE, "test_fluid_pins.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    out = []
    for name, fn in inspect.getmembers(mod, inspect.isfunction):
        if not name.startswith("test_"):
            continue
        marks = getattr(fn, "pytestmark", [])
        params = [m for m in marks if m.name == "parametrize"]
        cases = [{}]
        for m in params:
            argnames = [a.strip() for a in m.args[0].split(",")] if isinstance(m.args[0], str) else m.args[0]
            new = []
            for c in cases:
                for v in m.args[1]:
                    vals = v if len(argnames) > 1 else (v,)
                    new.append({**c, **dict(zip(argnames, vals))})
            cases = new
        out.extend((name, fn, c) for c in cases)
    return out


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    src = open(oracle.SRC).read()
    root = tmp_path_factory.mktemp("mutants")
    jobs = {}
    for i, (name, old, new) in enumerate(MUTANTS):
        assert src.count(old) == 1, name
        path = root / f"m{i}.c"
        path.write_text(src.replace(old, new))
        jobs[name] = (str(path), str(root / f"libm{i}.so"))
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futs = {name: ex.submit(oracle.build, True, s, o) for name, (s, o) in jobs.items()}
        return {name: f.result() for name, f in futs.items()}


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_fluid_pins_catch_mutant(name, mutant_libs):
    pins = _pins()
    good = oracle.lib()
    caught = []
    oracle.use_library(oracle.load(mutant_libs[name]))
    try:
        for pname, fn, kw in pins:
            try:
                fn(**kw)
            except AssertionError:
                caught.append(pname)
    finally:
        oracle.use_library(good)
    assert caught, f"no fluid pin fails under the mutant '{name}'"
