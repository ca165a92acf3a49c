"""The widened paths at full size (the 2e6-electron, 1000-cell discharge of the
single-instance production configuration, FP32 split), checked through
properties that hold at any size and, for the kinetic ions, a sample of ions
stepped one by one by the FP64 oracle from the GPU's pre-step state:

* kinetic ions: exact electron and ion bookkeeping, unique ids, n_i
  integrating to w N_i; sampled ions agree with the oracle's step to FP32
  rounding, collision outcomes except draws within rounding of a threshold;
* metastables with Penning and pooling: exact electron bookkeeping with the
  new births, n_m >= 0 and 0 at the electrodes; with the reactions off the
  metastable inventory changes every step by w x the excitations minus the
  wall flux;
* recombination: exact bookkeeping with the removed electrons;
* power control with a 40-step RF period: the amplitude follows Eq. 2.9 from
  the reported period power.
"""
import numpy as np
import pytest

import oracle
from paper_1508_02892_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _dv(G, L):
    dz = L / (G - 1)
    dv = np.full(G, dz)
    dv[0] = dv[-1] = dz / 2
    return dv


def _electrons_balance(c):
    return (c["births_iz"] + c["births_see0"] + c["births_see1"] + c["births_penning"] + c["births_pooling"] -
            c["losses0"] - c["losses1"] - c["recombinations"])


def test_kinetic_ions_full_size_and_sampled_against_oracle():
    from paper_1508_02892_gb300 import hybrid
    p = W.config2(ion_model=W.ION_KINETIC, capacity_factor=1.5)
    g = hybrid.Discharge(p)
    g.advance(40)
    before = g.ions()
    E = g.fields()["E"]
    step = g.counters()["step"]
    g.advance(1)
    after = g.ions()
    c = g.counters()
    assert c["status"] == 0
    assert c["particles"] == p["n_particles"] + _electrons_balance(c)
    assert c["ions"] == p["n_particles"] + c["births_iz"] - c["ion_losses0"] - c["ion_losses1"]
    assert after["id"].size == c["ions"] and np.unique(after["id"]).size == after["id"].size
    assert np.all((after["z"] >= 0) & (after["z"] < p["gap_m"]))
    ni = g.fields()["ni"]
    assert (ni * _dv(ni.size, p["gap_m"])).sum() == pytest.approx(g.info["weight"] * c["ions"], rel=1e-5, abs=0)
    # sampled ions against the oracle's one-ion step
    o = oracle.Oracle(dict(p, n_particles=1))
    rng = np.random.default_rng(5)
    idx = rng.choice(before["id"].size, 8000, replace=False)
    pos = {int(k): i for i, k in enumerate(after["id"])}
    mism = 0
    collided = 0
    for j in idx:
        st = [before["z"][j], before["vx"][j], before["vy"][j], before["vz"][j]]
        iid = int(before["id"][j])
        oc, out = o.ion_step_one(E, step, st, iid)
        if oc in (oracle.OUT_LOST0, oracle.OUT_LOST1):
            mism += iid in pos
            continue
        if iid not in pos:
            mism += 1
            continue
        collided += oc == 2
        k = pos[iid]
        got = np.array([after["z"][k], after["vx"][k], after["vy"][k], after["vz"][k]])
        sp = np.linalg.norm(out[1:])
        ok = abs(got[0] - out[0]) <= 2e-6 * p["gap_m"] and np.linalg.norm(got[1:] - out[1:]) <= 1e-4 * sp + 1.0
        mism += not ok
    assert collided > 20
    assert mism <= 3, mism
    assert hybrid.debug_checks() == ((0, 0, 0), (0, 0, 0))
    g.close()


def test_metastables_full_size_bookkeeping():
    from paper_1508_02892_gb300 import hybrid
    p = W.config2(**W.metastable_params(met_n0_m3=3e19, gamma_met=0.1))
    g = hybrid.Discharge(p)
    g.advance(60)
    c = g.counters()
    assert c["status"] == 0 and c["births_penning"] > 0 and c["births_pooling"] > 0
    assert c["particles"] == p["n_particles"] + _electrons_balance(c)
    s = g.particles()
    assert s["id"].size == c["particles"] and np.unique(s["id"]).size == s["id"].size
    m = g.metastables()
    assert np.all(m["met"] >= 0) and m["met"][0] == 0 and m["met"][-1] == 0
    assert hybrid.debug_checks() == ((0, 0, 0), (0, 0, 0))
    g.close()


def test_metastable_inventory_full_size():
    from paper_1508_02892_gb300 import hybrid
    p = W.config2(te0_ev=10.0, **W.metastable_params(met_n0_m3=1e18, met_diff_m2s=1.0, penning_rate_m3s=0.0,
                                                      pooling_rate_m3s=0.0))
    g = hybrid.Discharge(p)
    g.advance(5)
    G = g.info["n_nodes"]
    dz = p["gap_m"] / (G - 1)
    w, dt = g.info["weight"], p["dt_s"]
    inv = g.metastables()["met"][1:-1].sum() * dz
    exc = g.counters()["excitation"]
    for _ in range(5):
        g.advance(1)
        m, c = g.metastables(), g.counters()
        now = m["met"][1:-1].sum() * dz
        expect = inv + w * (c["excitation"] - exc) - dt * m["flux"].sum()
        assert now == pytest.approx(expect, rel=1e-9, abs=0)
        inv, exc = now, c["excitation"]
    g.close()


def test_recombination_full_size_bookkeeping():
    from paper_1508_02892_gb300 import hybrid
    p = W.config2(xs_rec=W.recombination_table(1e-8))
    g = hybrid.Discharge(p)
    g.advance(60)
    c = g.counters()
    assert c["status"] == 0 and c["recombinations"] > 1000
    assert c["particles"] == p["n_particles"] + _electrons_balance(c)
    g.close()


def test_power_control_full_size_follows_eq_2_9():
    from paper_1508_02892_gb300 import hybrid
    P0, alpha, U0 = 5e5, 0.2, 250.0
    p = W.config2(f_rf_hz=1.0 / (40 * 2e-13), power_w_m2=P0, power_alpha=alpha)
    g = hybrid.Discharge(p)
    g.advance(40)
    c1 = g.counters()
    assert c1["power_periods"] == 1
    assert c1["v_rf"] == pytest.approx(U0 * (1.0 - alpha * (c1["power_last"] - P0) / P0), rel=1e-12, abs=0)
    g.advance(40)
    c2 = g.counters()
    assert c2["power_periods"] == 2
    assert c2["v_rf"] == pytest.approx(c1["v_rf"] * (1.0 - alpha * (c2["power_last"] - P0) / P0), rel=1e-12, abs=0)
    g.close()
