"""The split production path (FP32 particles, FP64 field step) against the FP64
oracle on the kinds of discharge the benchmark runs.

The error against the FP64 oracle is stated for every reported moment.
Three workloads beyond config 1's drift-diffusion:
  * a reduced config 2 (He, 1 mm / 1000 cells, 250 V, gamma 0.1, full ion
    fluid, Eq. 2.3, with the He+ tables), 3e4 electrons, 400 steps;
  * a drift-diffusion discharge with the tabulated mobility and Eq. 2.7-2.8
    diffusion drawn from the batched ranges (gamma 0.1), 3e4 electrons,
    400 steps;
  * a full-fluid discharge driven hard enough for ionization and gamma
    emission to happen in a short run (0.5 mm / 200 cells, 400 V, 15 eV
    electrons, gamma 0.3, light macroparticles), 2e4 electrons, 300 steps.
At the configs' weights a few hundred steps emit almost no secondaries (the
mean count per step is gamma mu E dt N / L, about 1e-6 here), so the third
case carries the emission and ionization paths.
For each, the 16-seed ensemble means of the time-averaged n_e, n_i, <E>,
Gamma_i and the EEDF agree with the oracle's within 2 % (L2), printed beside
the seed-to-seed noise floor (oracle ensemble of the even seeds against that
of the odd ones).  Both sides draw the same random numbers, so the runs track
each other until an FP32 rounding flips a threshold.
"""
import numpy as np
import pytest

import oracle
from paper_1508_02892_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("ne", "ni", "ebar", "gamma", "eedf")
STEPS = {"full_fluid_gamma": 400, "dd_table_gamma": 400, "full_fluid_emitting": 300}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _base(case):
    if case == "full_fluid_gamma":
        return W.config2(n_particles=30000)
    if case == "full_fluid_emitting":
        return W.config1(precision=W.FP32_SPLIT, n_particles=20000, te0_ev=15.0, v_rf_amp_v=400.0, gamma_see=0.3,
                         ion_model=W.ION_FULL, weight=2e5)
    # the first drift-diffusion (tabulated mobility) discharge of the batched mix
    for p in W.config3_instances(64):
        if p["ion_model"] == W.ION_DD_TABLE:
            p = dict(p)
            p["n_particles"] = 30000
            return p
    raise AssertionError("no drift-diffusion discharge in the mix")


def _l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("case", ["full_fluid_gamma", "dd_table_gamma", "full_fluid_emitting"])
def test_split_production_moments_within_2pct(case):
    from paper_1508_02892_gb300 import hybrid
    base = _base(case)
    assert base["precision"] == W.FP32_SPLIT and base["gamma_see"] > 0
    plist = [dict(base, seed=300 + s) for s in range(16)]
    steps = STEPS[case]
    orc = oracle.run_ensemble(plist, steps)
    gpu = []
    for p in plist:
        g = hybrid.Discharge(p)
        g.advance(steps)
        gpu.append(g.moments())
        assert g.counters()["status"] == 0
        g.close()
    see = sum(m["counters"]["births_see0"] + m["counters"]["births_see1"] for m in orc)
    iz = sum(m["counters"]["ionization"] for m in orc)
    print(f"{case}: oracle ensemble has {see} secondaries and {iz} ionizations")
    if case == "full_fluid_emitting":
        assert see > 0 and iz > 0
    for k in KEYS:
        a = np.mean([m[k] for m in gpu], axis=0)
        b = np.mean([m[k] for m in orc], axis=0)
        noise = _l2(np.mean([m[k] for m in orc[0::2]], axis=0), np.mean([m[k] for m in orc[1::2]], axis=0))
        err = _l2(a, b)
        print(f"{case}: split vs oracle, 16 seeds, {k}: L2 {err:.3e} (seed noise floor {noise:.3e})")
        assert err < 0.02, (case, k, err)
