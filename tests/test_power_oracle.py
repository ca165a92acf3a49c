"""Power control of Eq. 2.9 in the oracle, pinned by closed forms.

In a vacuum gap only the displacement current flows, J = eps0 dE/dt with
E = V/L, so the power V J = d/dt (eps0 V^2 / 2L) is reactive: with V taken at
mid-step the discrete sum over a period telescopes to eps0 (V_end^2 -
V_start^2)/(2L) = 0 when the period is a whole number of steps.  The absorbed
power is then zero and Eq. 2.9 raises the amplitude by exactly (1 + alpha) per
period.  With a DC voltage and ions only, the conduction current e Gamma_i(0)
of ions driven into the powered electrode gives V e Gamma_i > 0 on average.
"""
import math

import pytest

import oracle
from paper_1508_02892_gb300 import workloads as W

EPS0 = 8.8541878128e-12


def _vacuum(**kw):
    return W.config1(n_particles=0, n0_m3=0.0, weight=1.0, f_rf_hz=1.0 / (200 * 2e-13), v_rf_amp_v=150.0, **kw)


def test_vacuum_gap_absorbs_no_power():
    p = _vacuum()
    o = oracle.Oracle(p)
    o.step(600)
    pw = o.power()
    assert pw["steps_per_period"] == 200 and pw["periods"] == 3
    reactive = EPS0 * 2 * math.pi * p["f_rf_hz"] * p["v_rf_amp_v"] ** 2 / p["gap_m"]
    assert abs(pw["p_last"]) < 1e-9 * reactive
    assert pw["v_rf"] == p["v_rf_amp_v"]


def test_controller_raises_the_amplitude_by_one_plus_alpha_per_period():
    p = _vacuum(power_w_m2=1000.0, power_alpha=0.1)
    o = oracle.Oracle(p)
    o.step(600)
    pw = o.power()
    assert pw["periods"] == 3
    assert pw["v_rf"] == pytest.approx(150.0 * 1.1 ** 3, rel=1e-9, abs=0)
    o.step(199)                               # mid-period: the amplitude holds
    assert o.power()["v_rf"] == pw["v_rf"]


def test_dc_ion_current_into_the_powered_electrode_absorbs_power():
    """V < 0 at z = 0 drives the ions of a uniform density (no electrons) into
    that electrode; over a period at fixed V the absorbed power is V times the
    period mean of e Gamma_i(0) plus the displacement term eps0 V (E_0(end) -
    E_0(start)) / T, and it is positive."""
    p = W.config1(n_particles=0, weight=1.0, v_rf_amp_v=0.0, v_dc_v=-100.0, f_rf_hz=1.0 / (200 * 2e-13))
    o = oracle.Oracle(p)
    e_start = o.fields()["E"][0]
    gam = []
    for _ in range(200):
        o.step(1)
        gam.append(o.fields()["gamma"][0])
    e_end = o.fields()["E"][0]
    T = 200 * p["dt_s"]
    V = p["v_dc_v"]
    expect = V * 1.602176634e-19 * sum(gam) / 200 + EPS0 * V * (e_end - e_start) / T
    pw = o.power()
    assert max(gam) < 0.0                      # ions flow into z = 0 throughout
    assert pw["p_last"] > 0.0
    assert pw["p_last"] == pytest.approx(expect, rel=1e-9, abs=0)
