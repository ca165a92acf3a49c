"""Kinetic ions in the oracle (the paper's fully kinetic comparison model,
with the ion-neutral collisions of Sec. II.C), pinned by:
* the drift of ions in a uniform field against the paper's Table 2 mobility
  (the collision operator is the one the paper used to make that table);
* stationarity of the gas Maxwellian at zero field (KS test);
* exact bookkeeping: one new ion per ionization, ion wall losses as the wall
  flux, and sum n_i dV = w N_i (CIC partition of unity).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1508_02892_gb300 import workloads as W

QE = 1.602176634e-19
KB = 1.380649e-23
M_HE = 4.002602 * 1.66053906660e-27


def _no_electron_collisions(**kw):
    xs = W.xs_tables(W.GAS_HE)
    return W.config1(ion_model=W.ION_KINETIC, xs_el=0 * xs["xs_el"], xs_exc=0 * xs["xs_exc"],
                     xs_ion=0 * xs["xs_ion"], **kw)


def test_ion_drift_matches_the_paper_mobility():
    """A DC voltage across the gap, charges too light to distort the field:
    after the relaxation window the ions drift at mu(E) E with mu from Table 2."""
    V = 300.0
    p = _no_electron_collisions(n_particles=20000, weight=1e-3, v_rf_amp_v=0.0, v_dc_v=V, seed=12)
    o = oracle.Oracle(p)
    E = V / p["gap_m"]
    o.step(1500)                              # about 25 momentum-relaxation times
    drift = []
    for _ in range(10):
        o.step(60)
        ions = o.ions()
        drift.append(ions["vz"].mean())
    u = np.mean(drift)
    E0 = 1.47e6
    mu = (1.18 - 0.185 * E / E0) * 1e-3
    assert u == pytest.approx(mu * E, rel=0.08, abs=0)
    assert abs(np.mean(drift[:5]) - np.mean(drift[5:])) < 0.03 * u     # stationary


def test_zero_field_keeps_the_gas_maxwellian():
    from scipy import stats
    p = _no_electron_collisions(n_particles=20000, weight=1e-3, v_rf_amp_v=0.0, seed=13)
    o = oracle.Oracle(p)
    o.step(400)
    ions = o.ions()
    vt = math.sqrt(KB * 300.0 / M_HE)
    for k in ("vx", "vy", "vz"):
        assert stats.kstest(ions[k] / vt, "norm").pvalue > 1e-3
    c = o.ion_counters()
    # thermal ions accept about nu / nu_max ~ 5 % (the bound covers 100 eV)
    assert c["collisions"] > 0.02 * c["candidates"] > 0


def test_ion_bookkeeping_is_exact():
    p = W.config1(n_particles=8000, ion_model=W.ION_KINETIC, te0_ev=20.0, v_rf_amp_v=300.0, gamma_see=0.3,
                  n_cells=100, weight=2e5, seed=14)
    o = oracle.Oracle(p)
    G = o.G
    dz = p["gap_m"] / (G - 1)
    dv = np.full(G, dz)
    dv[0] = dv[-1] = dz / 2
    prev, iprev = o.counters(), o.ion_counters()
    births = 0
    for _ in range(80):
        o.step(1)
        c, ic = o.counters(), o.ion_counters()
        d_iz = c["births_iz"] - prev["births_iz"]
        births += d_iz
        l0, l1 = ic["losses0"] - iprev["losses0"], ic["losses1"] - iprev["losses1"]
        assert ic["ions"] == iprev["ions"] + d_iz - l0 - l1
        ni = o.grid(oracle.GRID_NI)
        assert (ni * dv).sum() == pytest.approx(o.weight * ic["ions"], rel=1e-12, abs=0)
        fl = o.flux_in()
        assert fl[0] == pytest.approx(l0 * o.weight / p["dt_s"], rel=1e-12, abs=1e-30)
        assert fl[1] == pytest.approx(l1 * o.weight / p["dt_s"], rel=1e-12, abs=1e-30)
        prev, iprev = c, ic
    assert births > 0


def test_ion_push_closed_form_and_walls():
    """One ion step in a uniform field without a collision (no candidate, or a
    null one) is the leapfrog with the ion's mass: v' = v + (e/M) E dt,
    z' = z + v' dt, exactly; an ion crossing z = 0 or z = L is removed there."""
    p = _no_electron_collisions(n_particles=1, weight=1e-3, v_rf_amp_v=0.0)
    o = oracle.Oracle(p)
    G = o.G
    L, dt = p["gap_m"], p["dt_s"]
    E0 = 3.0e6
    E = np.full(G, E0)
    M = M_HE
    rng = np.random.default_rng(7)
    plain = 0
    for k in range(400):
        z = rng.uniform(0.05, 0.95) * L
        v = rng.normal(0.0, 800.0, 3)
        oc, out = o.ion_step_one(E, 5, [z, v[0], v[1], v[2]], (1 << 61) + k)
        if oc == 2:
            continue
        plain += 1
        vz = v[2] + QE / M * E0 * dt
        assert oc in (0, 1)
        np.testing.assert_allclose(out, [z + vz * dt, v[0], v[1], vz], rtol=1e-15, atol=0)
    assert plain > 300
    # walls: an ion placed just inside z = 0 moving out, and one just inside z = L
    oc, _ = o.ion_step_one(E * 0, 5, [1e-12, 0.0, 0.0, -1e3], 1 << 61)
    assert oc == oracle.OUT_LOST0
    oc, _ = o.ion_step_one(E * 0, 5, [L - 1e-12, 0.0, 0.0, 1e3], 1 << 61)
    assert oc == oracle.OUT_LOST1
