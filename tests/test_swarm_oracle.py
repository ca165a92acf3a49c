"""Pins of the oracle's auxiliary ion-swarm Monte Carlo (Sec. II.C) against
what the mathematics and the paper fix, independently of the code itself:

* Maxwell-molecule gas (Q_i only, so N Q g does not depend on g): with
  nu_max equal to that constant rate every candidate collides, and the mean
  velocity obeys the exact recursion m_n = (1 - P m_N/(M+m_N)) (m_{n-1} + a dt)
  of the discrete scheme (isotropic centre-of-mass scattering keeps the
  centre-of-mass velocity on average); its continuum limit is the drift
  e E / (M_r nu).
* At zero field the ions relax to a Maxwellian at the gas temperature (KS).
* Null-collision bookkeeping: candidate fraction P_max, acceptance nu/nu_max.
* Table 2 (mobility fit) and Table 3 (exchange-frequency fit) of the paper,
  which the paper's own run of this Monte Carlo produced, for E < 5 MV/m.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1508_02892_gb300 import workloads as W

QE = 1.602176634e-19
KB = 1.380649e-23
AMU = 1.66053906660e-27
M_HE = 4.002602 * AMU


def _maxwell_rate(pressure=101325.0, temp=300.0):
    n = pressure / (KB * temp)
    m_red = M_HE / 2
    return n * 7.63e-20 * math.sqrt(2 * QE / m_red)


def test_maxwell_gas_rate_is_speed_independent():
    n = 101325.0 / (KB * 300.0)
    m_red = M_HE / 2
    L = oracle.lib()
    vals = [L.orc_swarm_nu(n, m_red, W.SWARM_QI_ONLY, g) for g in (1.0, 300.0, 3e3, 3e4, 3e5)]
    assert max(vals) / min(vals) - 1 < 1e-12
    assert abs(vals[0] / _maxwell_rate() - 1) < 1e-12
    assert abs(L.orc_swarm_nu(n, m_red, W.SWARM_QI_ONLY, 0.0) / _maxwell_rate() - 1) < 1e-12
    # the full model adds 2 Q_b g > 0, which vanishes with g
    assert L.orc_swarm_nu(n, m_red, W.SWARM_QM, 1e-3) / _maxwell_rate() - 1 < 1e-4
    assert L.orc_swarm_nu(n, m_red, W.SWARM_QM, 3e3) > 1.5 * _maxwell_rate()


def test_maxwell_gas_drift_follows_the_exact_recursion():
    nu = _maxwell_rate()
    E, dt, n_steps, n_relax, n_ions = 1e6, 1e-13, 12000, 2000, 1500
    p = W.swarm_params(xs_model=W.SWARM_QI_ONLY, nu_max=nu, n_ions=n_ions, n_steps=n_steps, n_relax=n_relax,
                       dt_s=dt, seed=3)
    r = oracle.swarm_run(p, E)
    P = -math.expm1(-nu * dt)
    assert r["p_max"] == pytest.approx(P, rel=1e-14, abs=0)
    assert r["collisions"] == r["candidates"]          # nu_max = nu: no null collisions
    q = 1.0 - P * 0.5                                   # m_N / (M + m_N) = 1/2
    a = QE * E / M_HE * dt
    m, acc = 0.0, 0.0
    for n in range(n_steps):
        m = q * (m + a)
        if n >= n_relax:
            acc += m
    expect = acc / (n_steps - n_relax)
    assert r["drift"] == pytest.approx(expect, rel=0.02, abs=0)
    # the recursion's fixed point tends to the continuum drift e E / (M_r nu), M_r = M/2
    m_inf = q * a / (1.0 - q)
    assert m_inf == pytest.approx(QE * E / (M_HE / 2 * nu), rel=2e-3, abs=0)
    # candidates: binomial with probability P over n_ions * n_steps trials
    trials = n_ions * n_steps
    assert abs(r["candidates"] - P * trials) < 5 * math.sqrt(trials * P * (1 - P))


def test_acceptance_fraction_is_nu_over_nu_max():
    nu = _maxwell_rate()
    p = W.swarm_params(xs_model=W.SWARM_QI_ONLY, nu_max=2.0 * nu, n_ions=1000, n_steps=4000, n_relax=0, seed=5)
    r = oracle.swarm_run(p, 5e5)
    frac = r["collisions"] / r["candidates"]
    assert abs(frac - 0.5) < 5 * math.sqrt(0.25 / r["candidates"])
    assert r["overruns"] == 0


def test_zero_field_relaxes_to_the_gas_maxwellian():
    from scipy import stats
    p = W.swarm_params(ion_temp0_k=1500.0, n_ions=3000, n_steps=6000, n_relax=3000, seed=9)
    r, v = oracle.swarm_run(p, 0.0, velocities=True)
    assert r["overruns"] == 0
    vt = math.sqrt(KB * 300.0 / M_HE)
    mean_e = 1.5 * KB * 300.0 / QE
    assert r["mean_energy_ev"] == pytest.approx(mean_e, rel=0.03, abs=0)
    assert abs(r["drift"]) < 0.02 * vt
    for k in range(3):
        assert stats.kstest(v[:, k] / vt, "norm").pvalue > 1e-3


def _table2(E):
    """Table 2 of the paper: He+ mobility fit, 1e-3 m^2/(V s)."""
    E0 = 1.47e6
    return (1.18 - 0.185 * E / E0) * 1e-3 if E < E0 else 0.94 * (E0 / E) ** 0.3 * 1e-3


def _table2_ok(E, mu, rel=0.08):
    """Within rel of Table 2; the paper's two-piece fit jumps by 5.5 % at E0 =
    1.47 MV/m, so within 5 % of E0 either branch counts."""
    E0 = 1.47e6
    branches = [(1.18 - 0.185 * E / E0) * 1e-3, 0.94 * (E0 / E) ** 0.3 * 1e-3] if abs(E / E0 - 1) < 0.05 \
        else [_table2(E)]
    return any(abs(mu / b - 1) <= rel for b in branches)


def _table3(u):
    """Table 3 of the paper: He+ momentum-exchange frequency fit, 1e10 s^-1."""
    u0 = 2e3
    return (2.07 + 0.88 * (u / u0) ** 1.89) * 1e10 if u < u0 else (1.54 + 1.36 * u / u0) * 1e10


@pytest.mark.parametrize("E,n_ions", [(2e5, 8000), (1e6, 400), (1.47e6, 400), (3e6, 400), (5e6, 400)])
def test_mobility_reproduces_the_paper_tables(E, n_ions):
    """The paper fitted Tables 2/3 to its run of this Monte Carlo and reports
    good agreement below 5 MV/m; the fit error of the two-piece forms is a
    few per cent (8 % allowed).  A factor in the cross sections, the reduced
    mass or the scattering frame moves the result by tens of per cent.  At
    0.2 MV/m the drift is about a third of the thermal speed and the mean of
    v_z over 400 ions scatters by 6 % from seed to seed, so that field runs
    8000 ions (1.3 % by the square root of the count)."""
    p = W.swarm_params(n_ions=n_ions, n_steps=16000, n_relax=3000, seed=21)
    r = oracle.swarm_run(p, E)
    assert r["overruns"] == 0
    assert _table2_ok(E, r["mobility"])
    assert r["nu_exchange"] == pytest.approx(_table3(r["drift"]), rel=0.08, abs=0)
    # Eq. 2.6 ties the two outputs
    assert r["nu_exchange"] * r["mobility"] * M_HE / QE == pytest.approx(1.0, rel=1e-12, abs=0)
