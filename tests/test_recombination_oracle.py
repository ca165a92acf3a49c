"""Electron-ion recombination in the oracle (Sec. II.D): a null-collision
procedure of its own on the non-uniform ion density, nu_rec,max = max_z n_i *
max sigma v, with the actual probability taken at the electron's position.
Pinned by the binomial law of the events in a step, by their spatial
distribution following the ion density, and by exact bookkeeping of the
removed electrons and of the ion sink."""
import math

import numpy as np
import pytest

import oracle
from paper_1508_02892_gb300 import workloads as W

QE = 1.602176634e-19
ME = 9.1093837015e-31


def _beam(n, gap, energy_ev, seed):
    """n electrons uniform in (0.01 L, 0.99 L), one speed, isotropic directions."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.uniform(0.01 * gap, 0.99 * gap, n)
    ct = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2 * math.pi, n)
    st = np.sqrt(1 - ct ** 2)
    v = math.sqrt(2 * QE * energy_ev / ME)
    return z, v * st * np.cos(ph), v * st * np.sin(ph), v * ct, np.arange(n, dtype=np.uint64)


def _setup(n, ni_profile, k, energy_node, seed=3, **kw):
    xs = W.xs_tables(W.GAS_HE)
    # no electron-neutral collisions: the recombination is the only process
    p = W.config1(n_particles=10, n0_m3=1e10, weight=1e2, v_rf_amp_v=0.0, xs_el=0 * xs["xs_el"],
                  xs_exc=0 * xs["xs_exc"], xs_ion=0 * xs["xs_ion"], xs_rec=W.recombination_table(k),
                  capacity_factor=2.0 * n / 10, seed=seed, **kw)
    o = oracle.Oracle(p)
    o.set_grid(oracle.GRID_NI, ni_profile(o.G))
    e = xs["xs_ev"][energy_node]
    o.set_particles(*_beam(n, p["gap_m"], e, seed + 1))
    return p, o, e


def test_events_in_a_step_follow_the_binomial_law():
    """Uniform n_i, sigma = k/v so sigma v = k at the nodes; the beam sits on a
    node.  The bound is max over segments of max(sigma_i, sigma_i+1) v_i+1 =
    k (E_i+1/E_i)^(1/2), so a candidate turns real with probability
    (E_i/E_i+1)^(1/2) and an electron recombines with P_rec times that."""
    n, nival, k = 200000, 1e10, 2.5e1                     # nu = n_i k = 2.5e11 /s, nu dt = 0.05
    p, o, e = _setup(n, lambda G: np.full(G, nival), k, 600)
    o.step(1)
    c = o.counters()
    ratio = 10 ** (math.log10(1000.0 / 0.01) / 999)       # E_i+1 / E_i of the log grid
    numax = nival * k * math.sqrt(ratio)
    prob = -math.expm1(-numax * p["dt_s"]) / math.sqrt(ratio)
    mean = n * prob
    assert abs(c["recombinations"] - mean) < 5 * math.sqrt(mean * (1 - prob))
    assert c["particles"] == n - c["recombinations"] - c["losses0"] - c["losses1"]


def test_positions_follow_the_ion_density():
    n, k = 200000, 2.5e1
    prof = lambda G: 1e10 * np.linspace(0.0, 1.0, G)       # n_i rises linearly from 0 at z = 0
    p, o, e = _setup(n, prof, k, 600, seed=8)
    before = dict(zip(*(lambda s: (s["id"].tolist(), s["z"]))(o.particles())))
    vz = dict(zip(*(lambda s: (s["id"].tolist(), s["vz"]))(o.particles())))
    o.step(1)
    after = set(o.particles()["id"].tolist())
    L = p["gap_m"]
    gone = [i for i in before if i not in after]
    zs = np.array([before[i] + vz[i] * p["dt_s"] for i in gone])
    zs = zs[(zs >= 0) & (zs < L)]                          # drop the few absorbed at a wall
    assert zs.size > 3000
    edges = np.linspace(0.01 * L, 0.99 * L, 11)
    h, _ = np.histogram(zs, edges)
    mid = 0.5 * (edges[1:] + edges[:-1])
    expect = h.sum() * mid / mid.sum()                     # electrons uniform, rate proportional to n_i(z)
    chi2 = ((h - expect) ** 2 / expect).sum()
    from scipy import stats
    assert stats.chi2.sf(chi2, 9) > 1e-3


def test_bookkeeping_with_recombination_is_exact():
    """Every step: N_{n+1} = N_n + births - losses - recombinations, and the
    ion source integral sum_j G_j dV_j dt = w (births - recombinations)."""
    xs = W.xs_tables(W.GAS_HE)
    p = W.config1(n_particles=6000, te0_ev=20.0, v_rf_amp_v=300.0, n_cells=100, weight=2e5,
                  xs_rec=W.recombination_table(5e-8))
    o = oracle.Oracle(p)
    G = o.G
    dz = p["gap_m"] / (G - 1)
    dv = np.full(G, dz)
    dv[0] = dv[-1] = dz / 2
    prev = o.counters()
    total_rec = 0
    for _ in range(60):
        o.step(1)
        c = o.counters()
        d = {k: c[k] - prev[k] for k in c}
        total_rec += d["recombinations"]
        assert c["particles"] == prev["particles"] + d["births_iz"] + d["births_see0"] + d["births_see1"] \
            - d["losses0"] - d["losses1"] - d["recombinations"]
        src = o.grid(oracle.GRID_GSRC)
        assert (src * dv).sum() * p["dt_s"] == pytest.approx((d["births_iz"] - d["recombinations"]) * o.weight,
                                                             rel=1e-12, abs=1e-3)
        prev = c
    assert total_rec > 0
