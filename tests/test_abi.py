"""The C-ABI library builds, loads and exports every entry point that
include/hybrid1d.h declares (no GPU needed: nothing is computed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "hybrid1d.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(hyb_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("hyb_create_discharge", "hyb_advance", "hyb_read_moments", "hyb_destroy",
                 "hyb_batch_create", "hyb_batch_admit", "hyb_batch_advance", "hyb_batch_poll"):
        assert need in names


def test_library_exports_every_declared_symbol():
    from paper_1508_02892_gb300 import build, hybrid
    build.build()
    L = hybrid.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert set(_declared()) <= set(hybrid.EXPORTS)


def _struct_fields(src, name):
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)      # comments, also over several lines
    fields = []
    for decl in body.split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        decl = re.sub(r"^(const\s+)?\w+\s*", "", decl)     # the type
        for part in decl.split(","):
            m = re.match(r"\s*\*?\s*(\w+)", part)
            if m:
                fields.append(m.group(1))
    return fields


def test_binding_structs_match_header_field_order():
    from paper_1508_02892_gb300 import hybrid
    with open(os.path.join(ROOT, "include", "hybrid1d.h")) as f:
        src = f.read()
    for cname, py in (("hyb_params", hybrid.Params), ("hyb_tuning", hybrid.Tuning), ("hyb_profile", hybrid.Profile),
                      ("hyb_swarm_params", hybrid.SwarmParams), ("hyb_swarm_result", hybrid.SwarmResult),
                      ("hyb_counters", hybrid.Counters)):
        assert _struct_fields(src, cname) == [f for f, _ in py._fields_], cname


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1508_02892_gb300 import hybrid
    monkeypatch.setattr(hybrid, "_lib", None)
    monkeypatch.setattr(hybrid, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="not built"):
        hybrid.lib()


def test_host_validation_rejects_bad_params():
    """Argument checks run on the host before any device work."""
    import numpy as np

    from paper_1508_02892_gb300 import hybrid, workloads
    p = workloads.config1(n_particles=100)
    p["n_cells"] = 1
    with pytest.raises(hybrid.HybError) as e:
        hybrid.footprint(p)
    assert e.value.code == -1
    p = workloads.config1(n_particles=100)
    p["xs_el"] = p["xs_el"].copy()
    p["xs_el"][5] = np.nan
    with pytest.raises(hybrid.HybError) as e:
        hybrid.footprint(p)
    assert e.value.code == -4
    p = workloads.config1(n_particles=100)
    assert hybrid.footprint(p) > 0


def test_workload_dicts_fill_every_parameter():
    """Every scalar field of hyb_params has a value in the workload dicts (so
    no parameter silently takes 0), and the oracle's parameter struct has the
    same physics fields."""
    import oracle
    from paper_1508_02892_gb300 import hybrid, workloads as W
    p = W.config1()
    tables = {"tab_eon_td", "tab_mu", "tab_nu", "xs_ev", "xs_el", "xs_exc", "xs_ion", "xs_rec", "n_tab", "n_xs"}
    for name, _ in hybrid.Params._fields_:
        if name in tables:
            continue
        assert name in p, name
    # the method's parameters are named alike on both sides (the library adds
    # layout-only ones: precision, capacity, sort interval)
    lib_names = {n for n, _ in hybrid.Params._fields_} - {"precision", "capacity_factor", "sort_interval"}
    orc_names = {n for n, _ in oracle.OrcParams._fields_} - {"flags"}
    assert lib_names == orc_names, (lib_names ^ orc_names)
