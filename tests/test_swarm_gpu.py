"""GPU ion-swarm Monte Carlo (Sec. II.C) against the FP64 oracle.

FP64: every ion's final velocity agrees with the oracle's to 1e-12 relative
(both draw the same Philox numbers; only rounding differs), the collision
counts exactly, at small size and on ions sampled from a run of the table
size.  FP32: mobilities within 2 % of the oracle's.  The mobility and
exchange-frequency tables built on the GPU reproduce the paper's Tables 2/3
below 5 MV/m and drive the full ion-fluid model of a discharge.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1508_02892_gb300 import workloads as W

pytestmark = pytest.mark.gpu

QE = 1.602176634e-19
M_HE = 4.002602 * 1.66053906660e-27


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _vel_buffer(n):
    import torch
    return torch.zeros(3 * n, dtype=torch.float64, device="cuda")


def _compare_ions(vg, vo):
    scale = max(np.abs(vo).max(), 1.0)
    err = np.abs(vg - vo).max() / scale
    assert err <= 1e-12, err


@pytest.mark.parametrize("xs_model", [W.SWARM_QM, W.SWARM_QI_ONLY])
def test_fp64_swarm_matches_oracle_ion_by_ion(xs_model):
    from paper_1508_02892_gb300 import hybrid
    fields = [0.0, 7e5, 3e6]
    n = 300
    p = W.swarm_params(n_ions=n, n_steps=3000, n_relax=1000, nu_max=3.5e11, xs_model=xs_model, seed=17)
    v = _vel_buffer(n * len(fields))
    res, rc = hybrid.swarm_run(p, fields, velocities=v)
    assert rc == 0
    vg = v.cpu().numpy().reshape(len(fields), n, 3)
    for f, E in enumerate(fields):
        r, vo = oracle.swarm_run(p, E, id_base=f * n, velocities=True)
        g = res[f]
        for k in ("candidates", "collisions", "overruns"):
            assert g[k] == r[k], (f, k)
        assert g["p_max"] == r["p_max"]
        _compare_ions(vg[f], vo)
        vt = math.sqrt(1.380649e-23 * 300.0 / M_HE)
        assert abs(g["drift"] - r["drift"]) <= 1e-12 * vt
        assert g["mean_energy_ev"] == pytest.approx(r["mean_energy_ev"], rel=1e-12, abs=0)


def test_computed_bound_matches_the_oracle():
    from paper_1508_02892_gb300 import hybrid
    p = W.swarm_params(n_ions=64, n_steps=200, n_relax=100, eps_max_ev=20.0)
    res, _ = hybrid.swarm_run(p, [1e6])
    r = oracle.swarm_run(p, 1e6)
    assert res[0]["nu_max"] == pytest.approx(r["nu_max"], rel=1e-12, abs=0)


def test_fp32_mobility_close_to_the_fp64_oracle():
    from paper_1508_02892_gb300 import hybrid
    fields = [5e5, 2e6, 5e6]
    p = W.swarm_params(n_ions=400, n_steps=16000, n_relax=3000, seed=21)
    res, rc = hybrid.swarm_run(dict(p, precision=W.FP32_SPLIT), fields)
    assert rc == 0
    for f, E in enumerate(fields):
        r = oracle.swarm_run(p, E, id_base=f * p["n_ions"])
        assert res[f]["mobility"] == pytest.approx(r["mobility"], rel=0.02, abs=0)


def test_table_size_run_sampled_against_the_oracle():
    """The size the tables are built at (here 8 fields x 8192 ions x 20000
    steps, FP64): ions picked from two fields are re-run one by one by the
    oracle from their ids and must end with the same velocities."""
    from paper_1508_02892_gb300 import hybrid
    fields = list(W.swarm_fields(8, 5e6))
    n = 8192
    p = W.swarm_params(n_ions=n, n_steps=20000, n_relax=4000, seed=5)
    v = _vel_buffer(n * len(fields))
    res, rc = hybrid.swarm_run(p, fields, velocities=v)
    assert rc == 0
    vg = v.cpu().numpy().reshape(len(fields), n, 3)
    for f in (2, 7):
        base = 4000
        _, vo = oracle.swarm_run(dict(p, n_ions=24), fields[f], id_base=f * n + base, velocities=True)
        _compare_ions(vg[f, base:base + 24], vo)
    from paper_1508_02892_gb300 import hybrid as H
    assert H.debug_checks() == ((0, 0, 0), (0, 0, 0))


def _table2(E):
    E0 = 1.47e6
    return (1.18 - 0.185 * E / E0) * 1e-3 if E < E0 else 0.94 * (E0 / E) ** 0.3 * 1e-3


def _table2_ok(E, mu, rel=0.08):
    """Within rel of Table 2; the paper's two-piece fit jumps by 5.5 % at E0 =
    1.47 MV/m, so within 5 % of E0 either branch counts."""
    E0 = 1.47e6
    branches = [(1.18 - 0.185 * E / E0) * 1e-3, 0.94 * (E0 / E) ** 0.3 * 1e-3] if abs(E / E0 - 1) < 0.05 \
        else [_table2(E)]
    return any(abs(mu / b - 1) <= rel for b in branches)


def test_tables_reproduce_the_paper_and_drive_the_full_fluid_model():
    from paper_1508_02892_gb300 import hybrid
    eon = np.linspace(0.0, 200.0, 21)                  # Td; 200 Td = 4.9 MV/m at 1 atm, 300 K
    p = W.swarm_params(n_ions=4096, n_steps=20000, n_relax=4000, precision=W.FP32_SPLIT, seed=8)
    mu, nu, rc = hybrid.swarm_tables(p, eon)
    assert rc == 0
    ngas = 101325.0 / (1.380649e-23 * 300.0)
    E = eon * 1e-21 * ngas
    for k in range(1, eon.size):
        assert _table2_ok(E[k], mu[k]), (eon[k], mu[k], _table2(E[k]))
    assert mu[0] == mu[1] and nu[0] == nu[1]
    np.testing.assert_allclose(nu * mu * M_HE / QE, 1.0, rtol=1e-12)
    assert np.all(np.diff(mu[1:] * E[1:]) > 0)        # drift speed increases with the field
    q = W.config1(precision=W.FP64, n_particles=20000, ion_model=W.ION_FULL, gamma_see=0.1, weight=2e6,
                  v_rf_amp_v=300.0, tab_eon_td=eon, tab_mu=mu, tab_nu=nu)
    d = hybrid.Discharge(q)
    d.advance(60)
    c = d.counters()
    assert c["status"] == 0 and c["step"] == 60
    o = oracle.Oracle(q)
    o.step(60)
    ni_g, ni_o = d.fields()["ni"], o.fields()["ni"]
    assert np.abs(ni_g - ni_o).max() / np.abs(ni_o).max() <= 1e-11
