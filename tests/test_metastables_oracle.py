"""Metastables and the ionization they cause (Sec. II.D) in the oracle, pinned by:
* diffusion: a sine mode between the absorbing electrodes decays at the exact
  rate of the explicit scheme, close to the continuum rate D pi^2 / L^2;
* Penning and pooling losses against the solutions of dn/dt = -k n and
  dn/dt = -2 R n^2;
* the number of Penning and pooling electrons against the metastables lost
  (one electron per Penning event, one per two pooled metastables), and per
  node exactly floor(m) or floor(m) + 1 of them;
* the birth state: the process's energy exactly, isotropic directions, and
  uniform positions in the node's cell (KS tests);
* exact inventory: the metastables gained from the excitation events minus the
  flux into the walls; gamma emission by metastables at that flux;
* exact electron and ion bookkeeping with every process on.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1508_02892_gb300 import workloads as W

QE = 1.602176634e-19
ME = 9.1093837015e-31


def _quiet(**kw):
    """Electrons that do not collide (zero cross sections): the metastables
    evolve on their own."""
    xs = W.xs_tables(W.GAS_HE)
    base = dict(n_particles=0, weight=1e9, xs_el=0 * xs["xs_el"], xs_exc=0 * xs["xs_exc"], xs_ion=0 * xs["xs_ion"])
    met = W.metastable_params(met_diff_m2s=0.0, penning_rate_m3s=0.0, pooling_rate_m3s=0.0)
    base.update(met)
    base.update(kw)
    return W.config1(**base)


def _geometry(o, p):
    G = o.G
    return G, p["gap_m"] / (G - 1), p["dt_s"]


def test_sine_mode_decays_at_the_rate_of_the_scheme():
    D = 3.125                                   # D dt / dz^2 = 0.1
    p = _quiet(met_diff_m2s=D)
    o = oracle.Oracle(p)
    G, dz, dt = _geometry(o, p)
    j = np.arange(G)
    A = 1e18
    n0 = A * np.sin(np.pi * j / (G - 1))
    n0[0] = n0[-1] = 0.0
    o.set_metastables(n0)
    M = 400
    o.step(M)
    lam = 1.0 - 4.0 * D * dt / dz ** 2 * math.sin(math.pi / (2 * (G - 1))) ** 2
    m = o.metastables()
    assert np.abs(m["met"] - lam ** M * n0).max() <= 1e-12 * A
    # the flux into each wall in the last step: D n_1 / dz at the step's start
    f = D * A * lam ** (M - 1) * math.sin(math.pi / (G - 1)) / dz
    assert m["flux"][0] == pytest.approx(f, rel=1e-12, abs=0)
    assert m["flux"][1] == pytest.approx(f, rel=1e-9, abs=0)
    # and the continuum solution A exp(-D pi^2 t / L^2) sin(pi z / L)
    L = p["gap_m"]
    cont = A * math.exp(-D * math.pi ** 2 * M * dt / L ** 2) * np.sin(np.pi * j / (G - 1))
    assert np.abs(m["met"] - cont).max() <= 1e-4 * A


def test_penning_loss_and_births():
    k_rate, n_N, n0 = 1e-12, 5e21, 1e17         # k dt = 1e-3, 0.25 electrons per node and step
    p = _quiet(met_n0_m3=n0, penning_rate_m3s=k_rate, penning_target_m3=n_N)
    o = oracle.Oracle(p)
    G, dz, dt = _geometry(o, p)
    M = 500
    o.step(M)
    met = o.metastables()["met"]
    assert met[0] == met[-1] == 0.0
    k = k_rate * n_N
    np.testing.assert_allclose(met[1:-1], n0 * math.exp(-k * M * dt), rtol=1e-3)
    # every metastable lost made one electron: expected births (G - 2) dz (n0 - n_M) / w
    c = o.counters()
    expected = (G - 2) * dz * (n0 - met[1]) / p["weight"]
    assert expected > 1000
    assert abs(c["births_penning"] - expected) < 4 * math.sqrt(expected)
    assert c["births_pooling"] == 0 and c["particles"] == c["births_penning"] - c["losses0"] - c["losses1"]


def test_pooling_loss_and_births():
    R, n0 = 2.5e-8, 1e17                        # 2 R n0 dt = 1e-3, 0.125 electrons per node and step
    p = _quiet(met_n0_m3=n0, pooling_rate_m3s=R)
    o = oracle.Oracle(p)
    G, dz, dt = _geometry(o, p)
    M = 500
    o.step(M)
    met = o.metastables()["met"]
    np.testing.assert_allclose(met[1:-1], n0 / (1.0 + 2.0 * R * n0 * M * dt), rtol=1e-3)
    # one electron per two metastables pooled
    expected = (G - 2) * dz * (n0 - met[1]) / (2.0 * p["weight"])
    c = o.counters()
    assert expected > 1000
    assert abs(c["births_pooling"] - expected) < 4 * math.sqrt(expected)
    assert c["births_penning"] == 0


@pytest.mark.parametrize("proc", ["penning", "pooling"])
def test_birth_state_and_counts_per_node(proc):
    from scipy import stats
    if proc == "penning":
        p = _quiet(met_n0_m3=1e18, penning_rate_m3s=1e-12, penning_target_m3=5e21)   # m = 2.5 per node
        tag, energy = 6, p["penning_energy_ev"]
    else:
        p = _quiet(met_n0_m3=1e18, pooling_rate_m3s=5e-9)                             # m = 2.5 per node
        tag, energy = 7, p["pooling_energy_ev"]
    o = oracle.Oracle(p)
    G, dz, dt = _geometry(o, p)
    o.step(1)
    q = o.particles()
    ids = q["id"]
    mine = (ids >> np.uint64(60)) == np.uint64(tag)
    assert mine.all() and ids.size > 0
    assert np.all(((ids >> np.uint64(20)) & np.uint64(0xFFFFFFFF)) == 0)      # born in step 0
    k = np.sort((ids & np.uint64(0xFFFFF)).astype(np.int64))
    assert np.array_equal(k, np.arange(ids.size))                            # running index
    sp = math.sqrt(2.0 * QE * energy / ME)
    speed = np.sqrt(q["vx"] ** 2 + q["vy"] ** 2 + q["vz"] ** 2)
    np.testing.assert_allclose(speed, sp, rtol=1e-13)
    x = q["z"] / dz + 0.5
    node = np.floor(x).astype(int)
    assert node.min() >= 1 and node.max() <= G - 2
    per_node = np.bincount(node, minlength=G)[1:-1]
    assert set(np.unique(per_node)) <= {2, 3}
    n3 = int((per_node == 3).sum())
    assert abs(n3 - 0.5 * (G - 2)) < 4 * math.sqrt(0.25 * (G - 2))
    assert stats.kstest(x - node, "uniform").pvalue > 1e-3
    assert stats.kstest(q["vz"] / sp, "uniform", args=(-1, 2)).pvalue > 1e-3
    phi = np.arctan2(q["vy"], q["vx"])
    assert stats.kstest(phi, "uniform", args=(-np.pi, 2 * np.pi)).pvalue > 1e-3


def test_inventory_from_excitation_minus_wall_flux():
    """With the reactions off, every step: sum over interior nodes of n_m dz
    grows by w x (excitations of the step) and loses dt x (flux into both
    walls), to rounding."""
    p = W.config1(n_particles=4000, te0_ev=25.0, n_cells=60, seed=5,
                  **W.metastable_params(met_diff_m2s=1.0, met_n0_m3=1e18, penning_rate_m3s=0.0,
                                        pooling_rate_m3s=0.0))
    o = oracle.Oracle(p)
    G, dz, dt = _geometry(o, p)
    w = o.weight
    inv = o.metastables()["met"][1:-1].sum() * dz
    exc = 0
    gained = 0
    for _ in range(40):
        o.step(1)
        c = o.counters()
        m = o.metastables()
        now = m["met"][1:-1].sum() * dz
        d_exc = c["excitation"] - exc
        gained += d_exc
        expect = inv + w * d_exc - dt * m["flux"].sum()
        assert now == pytest.approx(expect, rel=1e-12, abs=1e-12 * max(inv, w))
        inv, exc = now, c["excitation"]
    assert gained > 100 and c["clamps"] == 0


def test_metastables_release_gamma_electrons():
    """gamma from metastables alone: per wall and step, floor(ns) or
    floor(ns) + 1 secondaries with ns = gamma_m Gamma_m dt / w."""
    p = _quiet(met_diff_m2s=3.0, met_n0_m3=1e19, gamma_met=0.3)
    o = oracle.Oracle(p)
    G, dz, dt = _geometry(o, p)
    prev = o.counters()
    tot = 0
    for _ in range(20):
        o.step(1)
        c = o.counters()
        f = o.metastables()["flux"]
        for wall in (0, 1):
            ns = 0.3 * f[wall] * dt / p["weight"]
            d = c[f"births_see{wall}"] - prev[f"births_see{wall}"]
            assert d in (math.floor(ns), math.floor(ns) + 1), (ns, d)
            tot += d
        prev = c
    assert tot > 100


def test_bookkeeping_with_every_process():
    p = W.config1(n_particles=6000, te0_ev=25.0, n_cells=80, seed=9, gamma_see=0.2, ion_model=W.ION_DD_TABLE,
                  weight=2e6, **W.metastable_params(met_n0_m3=2e19, penning_rate_m3s=1e-13, pooling_rate_m3s=1e-13,
                                                    gamma_met=0.2, met_diff_m2s=0.5))
    o = oracle.Oracle(p)
    G, dz, dt = _geometry(o, p)
    dv = np.full(G, dz)
    dv[0] = dv[-1] = dz / 2
    prev = o.counters()
    seen = {"births_penning": 0, "births_pooling": 0, "births_iz": 0}
    for _ in range(40):
        o.step(1)
        c = o.counters()
        d = {k: c[k] - prev[k] for k in c}
        assert d["particles"] == (d["births_iz"] + d["births_penning"] + d["births_pooling"] + d["births_see0"] +
                                  d["births_see1"] - d["losses0"] - d["losses1"])
        src = (o.grid(oracle.GRID_GSRC) * dv).sum() * dt
        assert src == pytest.approx(o.weight * (d["births_iz"] + d["births_penning"] + d["births_pooling"]),
                                    rel=1e-12, abs=1e-300)
        for k in seen:
            seen[k] += d[k]
        prev = c
    assert all(v > 0 for v in seen.values()), seen
    assert c["status"] == 0


def test_metastables_need_fluid_ions_and_a_stable_step():
    with pytest.raises(ValueError):
        oracle.Oracle(W.config1(ion_model=W.ION_KINETIC, **W.metastable_params()))
    with pytest.raises(ValueError):
        oracle.Oracle(W.config1(**W.metastable_params(met_diff_m2s=20.0)))      # D dt / dz^2 = 0.64
