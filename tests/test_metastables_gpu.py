"""Metastables, Penning and pooling ionization and metastable gamma emission
(Sec. II.D) on the GPU against the FP64 oracle.

FP64: particles by id (the Penning and pooling electrons included), every
counter, the fields, the moments and the metastable density agree with the
oracle to the tolerances of the other FP64 parity tests (1e-12 per particle,
1e-11 on grids).  Both sides draw the same Philox numbers: the per-node counts
with call 3 of a key made of the process and the node, the birth states with
call 2 of the new electron's id.  Inside a batch every discharge gives what it
gives alone; in FP32 split mode the counts follow the oracle's within a few
per cent.
"""
import numpy as np
import pytest

import oracle
from paper_1508_02892_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PART_TOL = 1e-12
GRID_TOL = 1e-11
COUNTERS = ("step", "particles", "births_iz", "births_see0", "births_see1", "losses0", "losses1", "elastic",
            "excitation", "ionization", "null", "clamps", "recombinations", "births_penning", "births_pooling")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _close(a, b, L, tol):
    assert a["id"].size == b["id"].size, (a["id"].size, b["id"].size)
    assert np.array_equal(a["id"], b["id"])
    if a["id"].size == 0:
        return
    assert np.max(np.abs(a["z"] - b["z"])) <= tol * L
    va = np.stack([a["vx"], a["vy"], a["vz"]])
    vb = np.stack([b["vx"], b["vy"], b["vz"]])
    speed = np.maximum(np.linalg.norm(vb, axis=0), 1e-3 * np.abs(vb).max())
    assert (np.linalg.norm(va - vb, axis=0) / speed).max() <= tol


def _grid(a, b, tol, name):
    scale = max(np.abs(b).max(), 1e-300)
    assert np.abs(a - b).max() / scale <= tol, (name, np.abs(a - b).max() / scale)


def _params(**kw):
    met = W.metastable_params(met_n0_m3=3e19, gamma_met=0.1)
    base = dict(precision=W.FP64, n_particles=20000, te0_ev=8.0, ion_model=W.ION_DD_TABLE, weight=2e6,
                v_rf_amp_v=300.0, seed=71, **met)
    base.update(kw)
    return W.config1(**base)


def _check(g, o, p):
    ca, cb = g.counters(), o.counters()
    for k in COUNTERS:
        assert ca[k] == cb[k], (k, ca[k], cb[k])
    assert ca["status"] == 0
    _close(g.particles(), o.particles(), p["gap_m"], PART_TOL)
    fa, fb = g.fields(), o.fields()
    for k in ("ne", "ni", "gamma", "phi", "E", "gsrc"):
        _grid(fa[k], fb[k], GRID_TOL, k)
    ma, mb = g.moments(), o.moments()
    for k in ("ne", "ni", "gamma", "ebar", "eedf"):
        _grid(ma[k], mb[k], GRID_TOL, k)
    sa, sb = g.metastables(), o.metastables()
    _grid(sa["met"], sb["met"], GRID_TOL, "met")
    _grid(sa["avg"], sb["avg"], GRID_TOL, "met avg")
    _grid(sa["flux"], sb["flux"], GRID_TOL, "met flux")


def test_fp64_metastables_match_the_oracle():
    from paper_1508_02892_gb300 import hybrid
    p = _params()
    g, o = hybrid.Discharge(p), oracle.Oracle(p)
    g.advance(100)
    o.step(100)
    c = o.counters()
    assert c["births_penning"] > 500 and c["births_pooling"] > 500 and c["excitation"] > 0
    assert c["births_see0"] + c["births_see1"] > 0
    _check(g, o, p)
    g.close()


def test_fp64_metastables_drift_diffusion_on_eight_ctas():
    """Drift-diffusion ions (no cluster barrier of their own before the
    continuity pass) with the field step on 8 CTAs: the metastables'
    ionization adds to the ion source at neighbouring CTAs' edge nodes, and
    every addition must be in before the continuity pass reads it."""
    from paper_1508_02892_gb300 import hybrid
    p = _params(n_cells=333, seed=79)
    g, o = hybrid.Discharge(p), oracle.Oracle(p)
    g.set_tuning(field_cluster=8)
    g.advance(100)
    o.step(100)
    assert o.counters()["births_penning"] > 500
    _check(g, o, p)
    g.close()


def test_fp64_written_profile_ragged_grid_full_fluid():
    """A metastable profile written through the API on a ragged grid with the
    full ion fluid and a sort every 9 steps."""
    from paper_1508_02892_gb300 import hybrid
    p = _params(n_particles=9999, n_cells=77, ion_model=W.ION_FULL, gamma_see=0.2, sort_interval=9, seed=72,
                met_n0_m3=0.0, capacity_factor=3.0)
    g, o = hybrid.Discharge(p), oracle.Oracle(p)
    G = g.info["n_nodes"]
    z = np.linspace(0.0, 1.0, G)
    prof = 6e19 * np.sin(np.pi * z) ** 2
    prof[0] = prof[-1] = 0.0
    g.set_metastables(prof)
    o.set_metastables(prof)
    g.advance(80)
    o.step(80)
    assert o.counters()["births_pooling"] > 100
    _check(g, o, p)
    g.close()


def test_metastable_discharge_in_a_mixed_batch():
    from paper_1508_02892_gb300 import hybrid
    ps = [_params(n_particles=6000, n_cells=90, seed=73, capacity_factor=3.0),
          W.config1(precision=W.FP64, n_particles=5000, n_cells=80, seed=74, te0_ev=6.0),
          W.config1(precision=W.FP64, n_particles=4000, n_cells=60, seed=75, xs_rec=W.recombination_table(2e-6)),
          _params(n_particles=3000, n_cells=50, seed=76, ion_model=W.ION_FULL, gamma_met=0.0, capacity_factor=5.0)]
    for lanes in (1, 2):
        b = hybrid.Batch(4, hybrid.HYB_FP64)
        b.set_tuning(lanes=lanes, sort_interval=20)
        slots = [b.admit(q) for q in ps]
        b.advance(90)
        for s, q in zip(slots, ps):
            g = hybrid.Discharge(q)
            g.advance(90)
            _close(b.particles(s), g.particles(), q["gap_m"], PART_TOL)
            ca, cb = b.counters(s), g.counters()
            for k in COUNTERS:
                assert ca[k] == cb[k], (lanes, s, k, ca[k], cb[k])
            if q.get("metastables"):
                _grid(b.metastables(s)["met"], g.metastables()["met"], GRID_TOL, "met")
            else:
                with pytest.raises(hybrid.HybError):
                    b.metastables(s)
            ma, mb = b.moments(s), g.moments()
            for k in ("ne", "ni", "gamma", "ebar", "eedf"):
                _grid(ma[k], mb[k], GRID_TOL, k)
            g.close()
        b.close()


def test_split_metastable_counts_track_the_oracle():
    from paper_1508_02892_gb300 import hybrid
    p = _params(precision=W.FP32_SPLIT, n_particles=40000, seed=77)
    g, o = hybrid.Discharge(p), oracle.Oracle(p)
    g.advance(300)
    o.step(300)
    a, b = g.counters(), o.counters()
    assert a["status"] == 0
    for k in ("births_penning", "births_pooling", "excitation"):
        assert b[k] > 1000 and abs(a[k] - b[k]) <= 0.03 * b[k], (k, a[k], b[k])
    ma, mb = g.metastables()["avg"], o.metastables()["avg"]
    assert np.linalg.norm(ma - mb) / np.linalg.norm(mb) < 0.01
    g.close()


def test_metastable_parameters_are_checked():
    from paper_1508_02892_gb300 import hybrid
    with pytest.raises(hybrid.HybError):
        hybrid.Discharge(_params(ion_model=W.ION_KINETIC))
    with pytest.raises(hybrid.HybError):
        hybrid.Discharge(_params(met_diff_m2s=20.0))               # D dt / dz^2 = 0.64
    g = hybrid.Discharge(_params(n_particles=1000, n_cells=40))
    bad = np.full(41, 1e18)
    with pytest.raises(hybrid.HybError):
        g.set_metastables(bad)                                   # electrode nodes must be 0
    g.close()
    f = hybrid.Discharge(W.config1(precision=W.FP64, n_particles=1000, n_cells=40))
    with pytest.raises(hybrid.HybError):
        f.metastables()
    f.close()


def test_electrons_from_metastables_alone():
    """Degenerate start: no electrons at all, only metastables.  Every electron
    then comes from Penning and pooling ionization; the run equals the
    oracle's in FP64."""
    from paper_1508_02892_gb300 import hybrid
    p = _params(n_particles=0, weight=2e6, n_cells=70, met_n0_m3=2e19, seed=78)
    g, o = hybrid.Discharge(p), oracle.Oracle(p)
    g.advance(60)
    o.step(60)
    c = o.counters()
    assert c["births_penning"] + c["births_pooling"] > 100 and c["particles"] > 0
    _check(g, o, p)
    g.close()
