"""Kinetic ions on the GPU (the paper's fully kinetic comparison model with the
ion-neutral collisions of Sec. II.C) against the FP64 oracle.

FP64: the electrons, the ions (by id), every counter, the fields and the
moments agree with the oracle to the tolerances of the other FP64 parity tests
(1e-12 per particle, 1e-11 on grids); both sides draw the same Philox numbers
(ion birth velocity call 4, ion collisions calls 5 and 6).  Inside a batch
with fluid-ion discharges every discharge gives what it gives alone.  Split
mode (electrons and ions as cell + FP32 offset, FP32 velocities): exact ion
bookkeeping, and the ion count, collisions and profiles within a few per cent
of the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_1508_02892_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PART_TOL = 1e-12
GRID_TOL = 1e-11
COUNTERS = ("step", "particles", "births_iz", "births_see0", "births_see1", "losses0", "losses1", "elastic",
            "excitation", "ionization", "null", "clamps", "recombinations")


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


def _kinetic(**kw):
    base = dict(precision=W.FP64, n_particles=20000, ion_model=W.ION_KINETIC, te0_ev=8.0, v_rf_amp_v=300.0,
                gamma_see=0.2, weight=2e6, seed=61)
    base.update(kw)
    return W.config1(**base)


def _check(g, o, p):
    ca, cb = g.counters(), o.counters()
    for k in COUNTERS:
        assert ca[k] == cb[k], (k, ca[k], cb[k])
    assert ca["status"] == 0
    ic = o.ion_counters()
    assert ca["ions"] == ic["ions"]
    assert ca["ion_losses0"] == ic["losses0"] and ca["ion_losses1"] == ic["losses1"]
    assert ca["ion_collisions"] == ic["collisions"]
    _close(g.particles(), o.particles(), p["gap_m"], PART_TOL)
    _close(g.ions(), o.ions(), p["gap_m"], PART_TOL)
    fa, fb = g.fields(), o.fields()
    for k in ("ne", "ni", "gamma", "phi", "E", "gsrc"):
        _grid(fa[k], fb[k], GRID_TOL, k)
    ma, mb = g.moments(), o.moments()
    for k in ("ne", "ni", "gamma", "ebar", "eedf"):
        _grid(ma[k], mb[k], GRID_TOL, k)


def test_fp64_kinetic_ions_match_the_oracle():
    """Births and ion collisions are many here; ion wall losses are not (in
    100 steps of 0.2 ps an ion moves about 20 nm, so the count over a 0.5 mm
    gap is a Poisson count of mean below 1): the ragged case below, on a
    20 um gap, is the one that exercises them."""
    from paper_1508_02892_gb300 import hybrid
    p = _kinetic()
    g, o = hybrid.Discharge(p), oracle.Oracle(p)
    _close(g.ions(), o.ions(), p["gap_m"], 1e-15)          # the initial load
    g.advance(100)
    o.step(100)
    c, ic = o.counters(), o.ion_counters()
    assert c["births_iz"] > 100 and ic["collisions"] > 0
    _check(g, o, p)
    g.close()
    # the ion-step counter: in step 0 every loaded ion and every ion born in it moves
    g1 = hybrid.Discharge(p)
    g1.advance(1)
    c1 = g1.counters()
    assert c1["ion_pushes"] == p["n_particles"] + c1["births_iz"]
    g1.close()


def test_ion_kernels_have_their_own_profile_interval():
    from paper_1508_02892_gb300 import hybrid
    p = _kinetic(n_particles=5000, n_cells=60)
    b = hybrid.Batch(2, hybrid.HYB_FP64)
    s = b.admit(p)
    b.set_tuning(lanes=1)
    b.set_profiling(True)
    b.advance(40)
    prof = b.profile()
    assert prof["n_ion"] == prof["n_electron"] == 40 and prof["ms_ion"] > 0
    c = b.counters(s)
    assert c["ion_pushes"] > 40 * p["n_particles"] // 2
    b.close()


def test_fp64_kinetic_ions_ragged_and_resorted():
    """A ragged size, a sort every 7 steps, and a gap of 20 um, narrow enough
    for ions to reach both walls within the run and release gamma electrons
    (about 20 ion losses a wall with 77,777 ions, and gamma 0.2 of them)."""
    from paper_1508_02892_gb300 import hybrid
    p = _kinetic(n_particles=77777, n_cells=97, gap_m=2e-5, sort_interval=7, te0_ev=20.0, weight=4e5,
                 v_rf_amp_v=500.0, seed=62)
    g, o = hybrid.Discharge(p), oracle.Oracle(p)
    g.advance(90)
    o.step(90)
    ic, c = o.ion_counters(), o.counters()
    assert ic["losses0"] > 0 and ic["losses1"] > 0 and c["births_see0"] + c["births_see1"] > 0
    _check(g, o, p)
    g.close()


def test_kinetic_and_fluid_discharges_share_a_batch():
    from paper_1508_02892_gb300 import hybrid
    ps = [_kinetic(n_particles=6000, n_cells=90, seed=63),
          W.config1(precision=W.FP64, n_particles=5000, n_cells=80, seed=64, te0_ev=6.0),
          W.config1(precision=W.FP64, n_particles=9000, n_cells=120, seed=65, ion_model=W.ION_FULL, gamma_see=0.2,
                    weight=2e6, v_rf_amp_v=300.0),
          _kinetic(n_particles=3000, n_cells=60, seed=66, te0_ev=12.0)]
    for lanes in (1, 2):
        b = hybrid.Batch(4, hybrid.HYB_FP64)
        b.set_tuning(lanes=lanes, sort_interval=20)
        slots = [b.admit(q) for q in ps]
        b.advance(120)
        for s, q in zip(slots, ps):
            g = hybrid.Discharge(q)
            g.advance(120)
            _close(b.particles(s), g.particles(), q["gap_m"], PART_TOL)
            ca, cb = b.counters(s), g.counters()
            for k in COUNTERS + ("ions", "ion_losses0", "ion_losses1", "ion_collisions"):
                assert ca[k] == cb[k], (lanes, s, k, ca[k], cb[k])
            if q["ion_model"] == W.ION_KINETIC:
                _close(b.ions(s), g.ions(), q["gap_m"], PART_TOL)
                assert ca["ions"] > 0
            else:
                assert ca["ions"] == 0
                with pytest.raises(hybrid.HybError):
                    b.ions(s)
            ma, mb = b.moments(s), g.moments()
            for k in ("ne", "ni", "gamma", "ebar", "eedf"):
                _grid(ma[k], mb[k], GRID_TOL, k)
            g.close()
        b.close()


def test_split_electrons_and_ions_track_the_oracle():
    """Split mode: electrons and ions as cell + FP32 offset with FP32
    velocities, the ion collisions in FP32.  The ion count follows births minus
    wall losses exactly and n_i integrates to w N_i (FP32 sums); over 300
    steps the ion count, the ion collisions, the time-averaged n_i profile and
    the mean ion energy stay close to the FP64 oracle's."""
    from paper_1508_02892_gb300 import hybrid
    p = _kinetic(precision=W.FP32_SPLIT, n_particles=40000, seed=67)
    g, o = hybrid.Discharge(p), oracle.Oracle(p)
    g.advance(300)
    o.step(300)
    c = g.counters()
    assert c["status"] == 0
    assert c["ions"] == p["n_particles"] + c["births_iz"] - c["ion_losses0"] - c["ion_losses1"]
    ions = g.ions()
    assert ions["id"].size == c["ions"]
    assert np.all((ions["z"] >= 0) & (ions["z"] < p["gap_m"]))
    ni = g.fields()["ni"]
    G = ni.size
    dz = p["gap_m"] / (G - 1)
    dv = np.full(G, dz)
    dv[0] = dv[-1] = dz / 2
    assert (ni * dv).sum() == pytest.approx(p["weight"] * c["ions"], rel=1e-5, abs=0)
    ic = o.ion_counters()
    assert abs(c["ions"] - ic["ions"]) <= 0.03 * ic["ions"], (c["ions"], ic["ions"])
    assert abs(c["ion_collisions"] - ic["collisions"]) <= 0.03 * ic["collisions"]
    ma, mb = g.moments(), o.moments()
    assert np.linalg.norm(ma["ni"] - mb["ni"]) / np.linalg.norm(mb["ni"]) < 0.02
    oi = o.ions()
    e_g = np.mean(ions["vx"] ** 2 + ions["vy"] ** 2 + ions["vz"] ** 2)
    e_o = np.mean(oi["vx"] ** 2 + oi["vy"] ** 2 + oi["vz"] ** 2)
    assert e_g == pytest.approx(e_o, rel=0.03, abs=0)
    g.close()


def test_split_batch_with_kinetic_and_fluid_discharges():
    """A split batch holding kinetic and fluid discharges: every discharge
    keeps its bookkeeping and matches its single run statistically."""
    from paper_1508_02892_gb300 import hybrid
    ps = [_kinetic(precision=W.FP32_SPLIT, n_particles=20000, n_cells=150, seed=81),
          W.config1(precision=W.FP32_SPLIT, n_particles=20000, n_cells=120, seed=82, te0_ev=6.0),
          _kinetic(precision=W.FP32_SPLIT, n_particles=8000, n_cells=90, seed=83, te0_ev=12.0)]
    b = hybrid.Batch(3, hybrid.HYB_FP32_SPLIT)
    b.set_tuning(lanes=2)
    slots = [b.admit(q) for q in ps]
    b.advance(200)
    for s, q in zip(slots, ps):
        ca = b.counters(s)
        assert ca["status"] == 0 and ca["step"] == 200
        g = hybrid.Discharge(q)
        g.advance(200)
        cb = g.counters()
        if q["ion_model"] == W.ION_KINETIC:
            assert ca["ions"] == q["n_particles"] + ca["births_iz"] - ca["ion_losses0"] - ca["ion_losses1"]
            assert b.ions(s)["id"].size == ca["ions"]
            assert abs(ca["ions"] - cb["ions"]) <= 0.03 * cb["ions"]
        else:
            assert ca["ions"] == 0
        ma, mb = b.moments(s), g.moments()
        for k in ("ne", "ni"):
            assert np.linalg.norm(ma[k] - mb[k]) / np.linalg.norm(mb[k]) < 0.03, (s, k)
        g.close()
    b.close()


def test_ion_density_is_not_writable_for_kinetic_ions():
    from paper_1508_02892_gb300 import hybrid
    p = _kinetic(n_particles=2000, n_cells=40)
    g = hybrid.Discharge(p)
    with pytest.raises(hybrid.HybError):
        g.set_ion_density(np.ones(41) * 1e15)
    g.close()
    q = W.config1(precision=W.FP64, n_particles=2000, n_cells=40)
    f = hybrid.Discharge(q)
    with pytest.raises(hybrid.HybError):
        f.ions()
    f.close()


def test_empty_kinetic_discharge():
    """No electrons and no ions: the kinetic path runs, nothing is born, the
    field is the vacuum field, and the result equals the oracle's."""
    from paper_1508_02892_gb300 import hybrid
    p = _kinetic(n_particles=0, n0_m3=0.0, weight=1e6, n_cells=40)
    g, o = hybrid.Discharge(p), oracle.Oracle(p)
    g.advance(20)
    o.step(20)
    c = g.counters()
    assert c["status"] == 0 and c["ions"] == 0 and c["particles"] == 0 and c["ion_pushes"] == 0
    assert g.ions()["id"].size == 0
    _check(g, o, p)
    g.close()
