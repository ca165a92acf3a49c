"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms, exact invariants, or statistics with a
stated confidence interval.  Runs on CPU only.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1508_02892_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
QE, ME, KB, EPS0, AMU = 1.602176634e-19, 9.1093837015e-31, 1.380649e-23, 8.8541878128e-12, 1.66053906660e-27


def _quiet(**kw):
    """A discharge with no charge (weight 0, no ions) and no drive: E == 0."""
    p = W.base_params(n_particles=0, n0_m3=0.0, v_rf_amp_v=0.0, v_dc_v=0.0, f_rf_hz=0.0)
    p.update(kw)
    return p


def _set_xs(p, el=0.0, exc=0.0, ion=0.0, e_exc=None, e_iz=None):
    n = p["xs_ev"].size
    p["xs_el"] = np.full(n, el) if np.isscalar(el) else np.asarray(el, float)
    p["xs_exc"] = np.full(n, exc) if np.isscalar(exc) else np.asarray(exc, float)
    p["xs_ion"] = np.full(n, ion) if np.isscalar(ion) else np.asarray(ion, float)
    if e_exc is not None:
        p["e_exc_ev"] = e_exc
    if e_iz is not None:
        p["e_iz_ev"] = e_iz
    return p


def _speed(ev):
    return math.sqrt(2 * QE * ev / ME)


def _iso_particles(n, ev, gap, seed, zfrac=0.5):
    rng = np.random.default_rng(seed)
    ct = rng.uniform(-1, 1, n)
    ph = rng.uniform(0, 2 * np.pi, n)
    st = np.sqrt(1 - ct ** 2)
    s = _speed(ev)
    return (np.full(n, zfrac * gap), s * st * np.cos(ph), s * st * np.sin(ph), s * ct,
            np.arange(n, dtype=np.uint64))


# ------------------------------------------------------------------ RNG ---

def test_philox_known_answers():
    with open(os.path.join(GOLD, "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])


def test_splitmix64_known_answers():
    with open(os.path.join(GOLD, "splitmix64_seed0.txt")) as f:
        vals = [int(l, 16) for l in f if l.strip() and not l.startswith("#")]
    g = 0x9E3779B97F4A7C15
    for k, v in enumerate(vals, start=1):
        assert oracle.mix64((k * g) & (2 ** 64 - 1)) == v


def test_u01_open_interval_and_exact_in_float():
    for x in (0, 1, 511, 512, 0x7FFFFFFF, 0xFFFFFFFF):
        u = oracle.u01(x)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u           # same value in FP32 and FP64
    assert oracle.u01(0) == 2.0 ** -24
    assert oracle.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24


def test_child_and_secondary_ids_disjoint():
    kids = {oracle.child_id(i, s) for i in range(200) for s in range(50)}
    assert len(kids) == 200 * 50
    assert all(k >> 63 == 1 for k in kids)
    sec = {oracle.see_id(w, s, k) for w in (0, 1) for s in range(100) for k in range(20)}
    assert len(sec) == 2 * 100 * 20
    assert all(k >> 62 == 1 for k in sec)          # bit 62 set, bit 63 clear


# -------------------------------------------------------- cross sections ---

def test_gas_density_ideal_gas():
    o = oracle.Oracle(W.config1(n_particles=10))
    # Loschmidt-type number at 1 atm, 300 K: 2.4463e25 m^-3
    assert o.ngas == pytest.approx(2.44631e25, rel=1e-5, abs=0)


def test_xs_lookup_matches_bruteforce_interpolation():
    p = W.config1(n_particles=10)
    o = oracle.Oracle(p)
    ev = p["xs_ev"]
    rng = np.random.default_rng(3)
    es = np.concatenate([ev[::37], np.exp(rng.uniform(np.log(0.011), np.log(990), 400))])
    for e in es:
        i = int(np.clip(np.searchsorted(ev, e, side="right") - 1, 0, ev.size - 2))
        f = (e - ev[i]) / (ev[i + 1] - ev[i])
        want = [p[k][i] + f * (p[k][i + 1] - p[k][i]) for k in ("xs_el", "xs_exc", "xs_ion")]
        if e < p["e_exc_ev"]:
            want[1] = 0.0
        if e < p["e_iz_ev"]:
            want[2] = 0.0
        got = o.xs(e)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-35)
    # clamping outside the table
    np.testing.assert_allclose(o.xs(1e-5), [p["xs_el"][0], 0, 0], rtol=1e-15)
    np.testing.assert_allclose(o.xs(5e3), [p["xs_el"][-1], p["xs_exc"][-1], p["xs_ion"][-1]], rtol=1e-15)
    # strictly zero just below each threshold, positive just above
    assert o.xs(p["e_exc_ev"] * (1 - 1e-9))[1] == 0.0
    assert o.xs(p["e_iz_ev"] * (1 - 1e-9))[2] == 0.0
    assert o.xs(p["e_exc_ev"] * 1.01)[1] > 0.0


def test_nu_max_bounds_collision_frequency():
    p = W.config1(n_particles=10)
    o = oracle.Oracle(p)
    es = np.exp(np.linspace(np.log(0.01), np.log(1000.0), 20001))
    nu = np.array([o.ngas * o.xs(e).sum() * _speed(e) for e in es])
    assert nu.max() <= o.nu_max * (1 + 1e-12)
    assert nu.max() >= o.nu_max * (1 - 1e-3)
    assert o.p_max == pytest.approx(-math.expm1(-o.nu_max * p["dt_s"]), rel=1e-14, abs=0)


# ---------------------------------------------------------------- pusher ---

def test_free_flight_closed_form():
    """Uniform field, no collisions, no charge: leapfrog is exact for constant
    force, z_n = z0 + n dt v0 + a dt^2 n(n+1)/2 with v^{-1/2} = v0."""
    L, V0, dt, n = 1e-2, 50.0, 1e-13, 300
    p = _set_xs(_quiet(gap_m=L, n_cells=100, v_dc_v=V0, dt_s=dt))
    o = oracle.Oracle(p)
    z0 = np.array([0.3, 0.5, 0.7]) * L
    vz0 = np.array([1e5, -2e5, 0.0])
    vx0 = np.array([3e4, 0.0, -1e4])
    o.set_particles(z0, vx0, np.zeros(3), vz0, np.arange(3, dtype=np.uint64))
    assert o.p_max == 0.0
    o.step(n)
    s = o.particles()
    a = -QE / ME * (V0 / L)
    np.testing.assert_allclose(s["vz"], vz0 + n * a * dt, rtol=1e-10)
    np.testing.assert_allclose(s["z"], z0 + n * dt * vz0 + a * dt * dt * n * (n + 1) / 2, rtol=1e-11)
    np.testing.assert_array_equal(s["vx"], vx0)
    # work-energy: eE0 times displacement equals the kinetic-energy gain of the
    # half-step velocities, to O(dt^2 a^2)
    c = o.counters()
    assert c["elastic"] + c["excitation"] + c["ionization"] + c["null"] == 0


def test_cic_gather_exact_for_linear_field():
    L = 1e-3
    p = _set_xs(_quiet(gap_m=L, n_cells=50))
    o = oracle.Oracle(p)
    zn = np.linspace(0, L, 51)
    a0, b0 = 3e4, -4e7
    E = a0 + b0 * zn
    rng = np.random.default_rng(5)
    dt = p["dt_s"]
    for _ in range(200):
        z = rng.uniform(0.01 * L, 0.99 * L)
        v = rng.normal(0, 3e5, 3)
        oc, out, _, _ = o.particle_step_one(E, 7, [z, *v], 11)
        vz = v[2] - QE / ME * (a0 + b0 * z) * dt
        assert oc == oracle.OUT_NONE
        assert out[3] == pytest.approx(vz, rel=1e-12, abs=1e-9)
        assert out[0] == pytest.approx(z + vz * dt, rel=1e-13, abs=0)
        assert out[1] == v[0] and out[2] == v[1]


def test_wall_absorption():
    L = 1e-3
    p = _set_xs(_quiet(gap_m=L, n_cells=10))
    o = oracle.Oracle(p)
    E = np.zeros(11)
    dt = p["dt_s"]
    oc, *_ = o.particle_step_one(E, 0, [0.5e-9, 0, 0, -1e4], 1)
    assert oc == oracle.OUT_LOST0                   # z = 5e-10 - 2e-9 < 0
    oc, *_ = o.particle_step_one(E, 0, [L - 0.5e-9, 0, 0, 1e4], 1)
    assert oc == oracle.OUT_LOST1
    oc, *_ = o.particle_step_one(E, 0, [0.5e-9, 0, 0, 1e3], 1)
    assert oc == oracle.OUT_NONE


# ------------------------------------------------------------- deposit ---

def test_cic_deposit_partition_and_first_moment():
    L, G = 1e-3, 41
    w = 1e9
    p = _set_xs(_quiet(gap_m=L, n_cells=G - 1, weight=w))
    o = oracle.Oracle(p)
    rng = np.random.default_rng(9)
    z = rng.uniform(0, L, 1000)
    o.set_particles(z, z * 0, z * 0, z * 0, np.arange(1000, dtype=np.uint64))
    ne = o.grid(oracle.GRID_NE)
    dz = L / (G - 1)
    dv = np.full(G, dz)
    dv[0] = dv[-1] = dz / 2
    cnt = ne * dv / w
    assert cnt.sum() == pytest.approx(1000, rel=1e-13, abs=0)                 # partition of unity
    assert (cnt * np.linspace(0, L, G)).sum() == pytest.approx(z.sum(), rel=1e-12, abs=0)  # CIC keeps the centroid
    # one particle: only its two nodes, with weights 1-o and o
    o.set_particles(np.array([0.3 * dz + 7 * dz]), np.zeros(1), np.zeros(1), np.zeros(1), np.zeros(1, np.uint64))
    cnt = o.grid(oracle.GRID_NE) * dv / w
    assert cnt[7] == pytest.approx(0.7, rel=1e-12, abs=0) and cnt[8] == pytest.approx(0.3, rel=1e-12, abs=0)
    assert np.count_nonzero(cnt) == 2


# ------------------------------------------------------------------ MCC ---

def test_null_collision_rate_constant_sigma():
    """Constant sigma, no field, no energy loss: the real-collision fraction per
    step is P_max * N sigma v / nu_max (binomial, 4.5 sigma)."""
    sig, ev, n, steps = 6e-20, 2.0, 20000, 10
    p = _set_xs(_quiet(gap_m=1.0, n_cells=10, gas_mass_amu=1e15), el=sig)
    o = oracle.Oracle(p)
    nu_max_cf = o.ngas * sig * _speed(1000.0)
    assert o.nu_max == pytest.approx(nu_max_cf, rel=1e-12, abs=0)
    o.set_particles(*_iso_particles(n, ev, 1.0, 1))
    o.step(steps)
    c = o.counters()
    prob = o.p_max * o.ngas * sig * _speed(ev) / o.nu_max
    N = n * steps
    assert abs(c["elastic"] - N * prob) < 4.5 * math.sqrt(N * prob * (1 - prob))
    assert c["elastic"] + c["null"] == pytest.approx(N * o.p_max, abs=4.5 * math.sqrt(N * o.p_max * (1 - o.p_max)))
    s = o.particles()
    np.testing.assert_allclose(np.sqrt(s["vx"] ** 2 + s["vy"] ** 2 + s["vz"] ** 2), _speed(ev), rtol=1e-9)


def test_null_collision_rate_small_dt_limit():
    """With nu_max dt << 1 the per-step collision fraction tends to N sigma v dt."""
    sig, ev, n, steps, dt = 6e-20, 5.0, 20000, 20, 2e-16
    p = _set_xs(_quiet(gap_m=1.0, n_cells=10, gas_mass_amu=1e15, dt_s=dt), el=sig)
    o = oracle.Oracle(p)
    assert o.nu_max * dt < 0.02
    o.set_particles(*_iso_particles(n, ev, 1.0, 2))
    o.step(steps)
    N = n * steps
    prob = o.ngas * sig * _speed(ev) * dt
    got = o.counters()["elastic"] / N
    assert abs(got - prob) < 4.5 * math.sqrt(prob / N) + 0.01 * prob


def test_process_selection_energy_losses_and_isotropy():
    """Three constant cross sections at 100 eV: outcome fractions P_max nu_k/nu_max;
    excitation loses exactly E_exc; ionization splits E - E_iz between the two
    electrons; new directions are isotropic."""
    p = _set_xs(_quiet(gap_m=1.0, n_cells=10, gas_mass_amu=1e15), el=3e-20, exc=2e-20, ion=1e-20,
                e_exc=1.0, e_iz=2.0)
    o = oracle.Oracle(p)
    E = np.zeros(11)
    ev = 100.0
    n = 30000
    z, vx, vy, vz, ids = _iso_particles(n, ev, 1.0, 4)
    outs = np.zeros(n, int)
    cts = []
    for i in range(n):
        oc, out, child, cid = o.particle_step_one(E, 3, [z[i], vx[i], vy[i], vz[i]], int(ids[i]))
        outs[i] = oc
        e1 = 0.5 * ME * (out[1:] ** 2).sum() / QE
        if oc == oracle.OUT_EXC:
            assert e1 == pytest.approx(ev - 1.0, rel=1e-12, abs=0)
        elif oc == oracle.OUT_ION:
            e2 = 0.5 * ME * (child[1:] ** 2).sum() / QE
            assert e1 + e2 == pytest.approx(ev - 2.0, rel=1e-12, abs=0)
            assert cid == oracle.child_id(int(ids[i]), 3)
            assert child[0] == out[0]
        elif oc == oracle.OUT_ELASTIC:
            assert e1 == pytest.approx(ev, rel=1e-9, abs=0)
        if oc in (oracle.OUT_ELASTIC, oracle.OUT_EXC, oracle.OUT_ION):
            cts.append(out[3] / np.linalg.norm(out[1:]))
    nu = o.ngas * np.array([3e-20, 2e-20, 1e-20]) * _speed(ev)
    for k, code in enumerate((oracle.OUT_ELASTIC, oracle.OUT_EXC, oracle.OUT_ION)):
        prob = o.p_max * nu[k] / o.nu_max
        got = (outs == code).sum()
        assert abs(got - n * prob) < 4.5 * math.sqrt(n * prob * (1 - prob))
    cts = np.array(cts)
    m = cts.size
    assert abs(cts.mean()) < 4.5 / math.sqrt(3 * m)
    assert abs((cts ** 2).mean() - 1 / 3) < 4.5 * math.sqrt(4 / 45 / m)


def _const_nu_table(p, ngas, nu0):
    ev = p["xs_ev"]
    return nu0 / (ngas * np.sqrt(2 * QE * ev / ME))


def test_elastic_energy_relaxation_cold_gas():
    """Constant nu, elastic only, cold gas: each real collision multiplies the
    energy by 1 - (2m/M)(1 - cos chi) with <1 - cos chi> = 1, so
    <E_n> = E_0 (1 - p 2m/M)^n -> E_0 exp(-(2m/M) nu t)."""
    M_amu = 100 * ME / AMU
    nu0, dt, ev0, n, steps = 1e11, 2e-13, 5.0, 20000, 500
    p = _quiet(gap_m=1.0, n_cells=10, gas_mass_amu=M_amu, dt_s=dt)
    ngas = p["pressure_pa"] / (KB * p["gas_temp_k"])
    p = _set_xs(p, el=_const_nu_table(p, ngas, nu0))
    o = oracle.Oracle(p)
    o.set_particles(*_iso_particles(n, ev0, 1.0, 8))
    o.step(steps)
    s = o.particles()
    e = 0.5 * ME * (s["vx"] ** 2 + s["vy"] ** 2 + s["vz"] ** 2) / QE
    prob = o.p_max * nu0 / o.nu_max
    want = ev0 * (1 - prob * 2 * ME / (M_amu * AMU)) ** steps
    assert abs(e.mean() - want) < 4.5 * e.std() / math.sqrt(n) + 2e-4 * want
    cont = ev0 * math.exp(-2 * ME / (M_amu * AMU) * nu0 * steps * dt)
    assert e.mean() == pytest.approx(cont, rel=0.02, abs=0)


def test_maxwellian_relaxation_thermal_gas():
    """Field-free box, elastic collisions with a Maxwellian target (test-only
    oracle switch): a mono-energetic beam relaxes to a Maxwellian at T_g."""
    kt_ev = 0.5
    tg = kt_ev * QE / KB
    M_amu = 20 * ME / AMU
    nu0, dt, n, steps = 1e11, 2e-13, 4000, 4000
    p = _quiet(gap_m=10.0, n_cells=10, gas_mass_amu=M_amu, dt_s=dt, gas_temp_k=tg,
               flags=oracle.FLAG_THERMAL_GAS)
    ngas = p["pressure_pa"] / (KB * tg)
    p = _set_xs(p, el=_const_nu_table(p, ngas, nu0))
    o = oracle.Oracle(p)
    s = _speed(5.0)
    o.set_particles(np.full(n, 5.0), np.zeros(n), np.zeros(n), np.full(n, s), np.arange(n, dtype=np.uint64))
    o.step(steps)
    st = o.particles()
    sd = math.sqrt(kt_ev * QE / ME)
    for comp in ("vx", "vy", "vz"):
        assert stats.kstest(st[comp] / sd, "norm").pvalue > 1e-4
    e = 0.5 * ME * (st["vx"] ** 2 + st["vy"] ** 2 + st["vz"] ** 2) / QE
    assert e.mean() == pytest.approx(1.5 * kt_ev, rel=4.5 * math.sqrt(2 / 3 / n), abs=0)


# ------------------------------------------------------------- Poisson ---

def test_poisson_uniform_charge_closed_form():
    L, G, V, rho0 = 1e-3, 101, 100.0, 1.6e-3
    z = np.linspace(0, L, G)
    phi, E = oracle.poisson(np.full(G, rho0), L / (G - 1), V, 0.0)
    want = V * (1 - z / L) + rho0 * z * (L - z) / (2 * EPS0)
    np.testing.assert_allclose(phi, want, rtol=0, atol=1e-12 * np.abs(want).max())
    wantE = V / L - rho0 * (L - 2 * z) / (2 * EPS0)
    np.testing.assert_allclose(E, wantE, rtol=0, atol=1e-9 * np.abs(wantE).max())
    assert EPS0 * (E[-1] - E[0]) == pytest.approx(rho0 * L, rel=1e-9, abs=0)


def test_poisson_gauss_law_random_charge():
    rng = np.random.default_rng(1)
    L, G = 2e-3, 301
    dz = L / (G - 1)
    rho = rng.normal(0, 1e-3, G)
    phi, E = oracle.poisson(rho, dz, 37.0, 0.0)
    q = rho * dz
    q[0] *= 0.5
    q[-1] *= 0.5
    assert EPS0 * (E[-1] - E[0]) == pytest.approx(q.sum(), rel=1e-8, abs=1e-12 * np.abs(rho).max() * L)
    # the discrete equation itself
    lap = (phi[:-2] - 2 * phi[1:-1] + phi[2:]) / dz ** 2
    np.testing.assert_allclose(-EPS0 * lap, rho[1:-1], rtol=0, atol=1e-6 * np.abs(rho).max())


# ----------------------------------------------------------- ion fluid ---

def _fluid(model, G=201, L=1e-3, **kw):
    p = _quiet(gap_m=L, n_cells=G - 1, ion_model=model, n0_m3=1e16, **kw)
    p["weight"] = 1.0       # keep the electron weight defined; no electrons exist
    return oracle.Oracle(p)


def test_dd_pure_diffusion_variance_grows_2Dt():
    o = _fluid(W.ION_DD_CONST)
    G, L = 201, 1e-3
    z = np.linspace(0, L, G)
    n = 1e16 * np.exp(-0.5 * ((z - L / 2) / (L / 20)) ** 2)
    gam = np.zeros(G)
    dt = 2e-13
    D = 1e-3 * KB * 300.0 / QE
    E = np.zeros(G)
    m0 = n.sum()
    var0 = (n * z ** 2).sum() / m0 - ((n * z).sum() / m0) ** 2
    steps = 2000
    for _ in range(steps):
        n, gam, flux, cl = o.fluid_update(E, np.zeros(G), n, gam)
        assert cl == 0
    var = (n * z ** 2).sum() / n.sum() - ((n * z).sum() / n.sum()) ** 2
    assert n.sum() == pytest.approx(m0, rel=1e-12, abs=0)
    assert var - var0 == pytest.approx(2 * D * steps * dt, rel=1e-6, abs=0)


def test_dd_pure_drift_centroid_moves_at_mu_E():
    o = _fluid(W.ION_DD_CONST)
    G, L = 201, 1e-3
    z = np.linspace(0, L, G)
    n = 1e16 * np.exp(-0.5 * ((z - L / 2) / (L / 20)) ** 2)
    gam = np.zeros(G)
    dt, E0, mu = 2e-13, 1e5, 1e-3
    E = np.full(G, E0)
    c0 = (n * z).sum() / n.sum()
    steps = 3000
    for _ in range(steps):
        n, gam, flux, cl = o.fluid_update(E, np.zeros(G), n, gam)
    c1 = (n * z).sum() / n.sum()
    assert c1 - c0 == pytest.approx(mu * E0 * steps * dt, rel=1e-6, abs=0)


def _const_tables(p, mu0, nu0):
    p["tab_mu"] = np.full(p["tab_eon_td"].size, mu0)
    p["tab_nu"] = np.full(p["tab_eon_td"].size, nu0)
    return p


def test_full_model_relaxes_to_drift_diffusion_flux():
    """Eq. 2.2 -> Eq. 2.5: with constant nu = e/(M mu) and a steady uniform field
    the full-model flux relaxes to mu n E in the interior."""
    G, L, mu0 = 101, 1e-3, 1.18e-3
    M = 4.002602 * AMU
    nu0 = QE / (M * mu0)
    p = _quiet(gap_m=L, n_cells=G - 1, ion_model=W.ION_FULL, n0_m3=1e16)
    p["weight"] = 1.0
    o = oracle.Oracle(_const_tables(p, mu0, nu0))
    n = np.full(G, 1e16)
    gam = np.zeros(G)
    E = np.full(G, 2e4)
    src = np.zeros(G)
    for _ in range(6000):                  # nu dt = 4.8e-3: e^-29 after 6000 steps
        _, gam, _, _ = o.fluid_update(E, src, n, gam)
    np.testing.assert_allclose(gam[5:-5], mu0 * 1e16 * 2e4, rtol=1e-6)


@pytest.mark.parametrize("model", [W.ION_DD_CONST, W.ION_DD_TABLE, W.ION_FULL])
def test_fluid_discrete_conservation(model):
    """Sum of dV_j (n^{n+1} - n^n) = dt sum dV_j G_j - dt (Gamma_N - Gamma_0)."""
    G, L = 151, 1e-3
    o = _fluid(model, G=G, L=L)
    rng = np.random.default_rng(11)
    z = np.linspace(0, L, G)
    n = 1e16 * (1 + 0.3 * np.sin(3 * np.pi * z / L)) + 1e14
    gam = rng.normal(0, 1e18, G)
    E = 3e5 * np.cos(2 * np.pi * z / L)
    src = np.abs(rng.normal(0, 1e24, G))
    dz = L / (G - 1)
    dv = np.full(G, dz)
    dv[0] = dv[-1] = dz / 2
    dt = 2e-13
    n1, g1, flux, cl = o.fluid_update(E, src, n, gam)
    assert cl == 0
    lhs = (dv * (n1 - n)).sum()
    rhs = dt * (dv * src).sum() - dt * (g1[-1] - g1[0])
    assert lhs == pytest.approx(rhs, rel=1e-9, abs=0)
    assert flux[0] == max(-g1[0], 0.0) and flux[1] == max(g1[-1], 0.0)
    # the wall flux follows the alpha switch: field-driven, only into the wall
    assert (g1[0] == 0.0) == (E[0] >= 0.0)
    assert (g1[-1] == 0.0) == (E[-1] <= 0.0)


def test_table2_table3_consistency_through_eq_2_6():
    with open(os.path.join(GOLD, "table2_table3_consistency.txt")) as f:
        kv = dict(l.split() for l in f if l.strip() and not l.startswith("#"))
    t = W.ion_tables("he", W.ATM, 300.0)
    assert t["tab_mu"][0] == pytest.approx(float(kv["mu0_m2_per_Vs"]), rel=1e-12, abs=0)
    assert t["tab_nu"][0] == pytest.approx(float(kv["nu0_per_s"]), rel=1e-12, abs=0)
    M = 4.002602 * AMU
    assert QE / (M * t["tab_mu"][0]) == pytest.approx(t["tab_nu"][0], rel=float(kv["rel_tol"]), abs=0)


# --------------------------------------------------------- gamma emission ---

def test_secondary_emission_statistics():
    """Mean number per step gamma Gamma S dt / N_p/sp (integer part + Bernoulli);
    born inside the gap within one push of the wall, 1 eV, Lambertian."""
    L = 1e-3
    p = _quiet(gap_m=L, n_cells=10, gamma_see=0.25, weight=1e8, dt_s=2e-13)
    o = oracle.Oracle(p)
    flux = np.array([4.6e21, 1.0e21])
    o.set_flux_in(flux)
    steps = 20000
    counts = np.array([o.emit_only(s) for s in range(steps)])
    mean = 0.25 * flux * 2e-13 / 1e8           # 2.3 and 0.5 per step
    tot = mean.sum()
    frac = mean - np.floor(mean)
    var = (frac * (1 - frac)).sum()
    assert abs(counts.mean() - tot) < 4.5 * math.sqrt(var / steps)
    assert counts.min() >= np.floor(mean).sum()
    s = o.particles()
    sp = _speed(1.0)
    v = np.sqrt(s["vx"] ** 2 + s["vy"] ** 2 + s["vz"] ** 2)
    np.testing.assert_allclose(v, sp, rtol=1e-12)
    w0 = (s["id"] >> np.uint64(60)) & np.uint64(3)
    at0 = w0 == 0
    assert np.all(s["vz"][at0] > 0) and np.all(s["vz"][~at0] < 0)
    assert np.all((s["z"][at0] > 0) & (s["z"][at0] <= s["vz"][at0] * 2e-13))
    assert np.all((s["z"][~at0] < L) & (s["z"][~at0] >= L + s["vz"][~at0] * 2e-13))
    ct = np.abs(s["vz"]) / v
    m = ct.size
    assert abs(ct.mean() - 2 / 3) < 4.5 * math.sqrt(1 / 18 / m)  # Lambertian: <cos> = 2/3, var 1/18


# ------------------------------------------------------ whole-step invariants ---

def test_initial_load_maxwellian_uniform():
    p = W.config1(n_particles=40000, te0_ev=3.0)
    o = oracle.Oracle(p)
    s = o.particles()
    assert np.array_equal(s["id"], np.arange(40000, dtype=np.uint64))
    assert stats.kstest(s["z"] / p["gap_m"], "uniform").pvalue > 1e-4
    sd = math.sqrt(QE * 3.0 / ME)
    for c in ("vx", "vy", "vz"):
        assert stats.kstest(s[c] / sd, "norm").pvalue > 1e-4


def test_step_bookkeeping_exact():
    """Particle count, CIC charge and ion inventory close exactly every step:
    N_{n+1} = N_n + births + secondaries - losses; sum n_e dV = w (N_{n+1} -
    births_n - secondaries_n) (children are deposited one step later and the
    secondaries born at the end of step n enter at step n+1); ion inventory
    changes by births w - dt (Gamma_N - Gamma_0)."""
    p = W.config1(n_particles=4000, te0_ev=25.0, v_rf_amp_v=400.0, gamma_see=0.3, n_cells=100, weight=2e5)
    o = oracle.Oracle(p)
    G = o.G
    dz = p["gap_m"] / (G - 1)
    dv = np.full(G, dz)
    dv[0] = dv[-1] = dz / 2
    prev = o.counters()
    ni_prev = o.grid(oracle.GRID_NI)
    w = o.weight
    seen_births = seen_see = 0
    for _ in range(150):
        o.step(1)
        c = o.counters()
        d = {k: c[k] - prev[k] for k in c}
        births = d["births_iz"]
        see = d["births_see0"] + d["births_see1"]
        seen_births += births
        seen_see += see
        assert c["particles"] == prev["particles"] + births + see - d["losses0"] - d["losses1"]
        ne = o.grid(oracle.GRID_NE)
        assert (ne * dv).sum() == pytest.approx(w * (c["particles"] - births - see), rel=1e-12, abs=0)
        ni = o.grid(oracle.GRID_NI)
        g = o.grid(oracle.GRID_GAMMA)
        src = o.grid(oracle.GRID_GSRC)
        assert (src * dv).sum() * p["dt_s"] == pytest.approx(births * w, rel=1e-12, abs=1e-3)
        assert c["clamps"] == 0
        lhs = (dv * (ni - ni_prev)).sum()
        rhs = births * w - p["dt_s"] * (g[-1] - g[0])
        assert lhs == pytest.approx(rhs, rel=1e-6, abs=1e-9 * (dv * ni).sum())
        prev, ni_prev = c, ni
    assert seen_births > 0 and seen_see > 0


def test_moments_time_average_and_eedf_normalisation():
    p = W.config1(n_particles=3000)
    o = oracle.Oracle(p)
    ne_sum = np.zeros(o.G)
    for _ in range(20):
        o.step(1)
        ne_sum += o.grid(oracle.GRID_NE)
    m = o.moments()
    assert m["n_samples"] == 20
    np.testing.assert_allclose(m["ne"], ne_sum / 20, rtol=1e-13)
    de = p["eedf_max_ev"] / p["eedf_bins"]
    assert m["eedf"][:-1].sum() * de + m["eedf"][-1] == pytest.approx(1.0, rel=1e-12, abs=0)
    # mean energy of a 2 eV Maxwellian, early in the run: 3 eV
    ebar = m["ebar"][m["ebar"] > 0]
    assert 2.0 < np.median(ebar) < 4.0


def test_draw_layout_of_the_mcc():
    """The documented stream layout: draw `call` of particle `id` at step n is
    the Philox4x32-10 block at counter (n, id_lo, call, id_hi) under key
    (seed_lo, seed_hi); the MCC takes words 0 and 1 for R1 < P_max and
    R2 nu_max < nu(E), words 2 and 3 for the new direction (cos chi = 1 - 2u,
    phi = 2 pi u).  Ids with the high word set (children) pin id_hi's place;
    a seed with both words set pins the key's."""
    L = 1e-3
    p = _set_xs(_quiet(gap_m=L, n_cells=10, pressure_pa=1.28e4, seed=0x0123456789ABCDEF), el=6e-20)
    o = oracle.Oracle(p)
    E = np.zeros(11)
    seed = p["seed"]
    key = [seed & 0xFFFFFFFF, seed >> 32]
    assert 0.3 < o.p_max < 0.7
    ev = 300.0
    v = math.sqrt(2 * ev * QE / ME)
    n = 5
    seen = set()
    for k in range(300):
        pid = k if k % 2 == 0 else (1 << 63) | (k * 0x9E3779B97F4A7C15 & ((1 << 63) - 1))
        st = [0.5 * L, 0.0, 0.0, v]
        oc, out, _, _ = o.particle_step_one(E, n, st, pid)
        r = oracle.philox4x32_10([n, pid & 0xFFFFFFFF, 0, pid >> 32], key)
        u = [oracle.u01(x) for x in r]
        if not u[0] < o.p_max:
            want = oracle.OUT_NONE
        elif u[1] * o.nu_max < o.ngas * o.xs(ev)[0] * v:
            want = oracle.OUT_ELASTIC
        else:
            want = oracle.OUT_NULL
        assert oc == want, (k, oc, want)
        seen.add(oc)
        if oc == oracle.OUT_ELASTIC:
            sp = np.linalg.norm(out[1:])
            assert out[3] / sp == pytest.approx(1.0 - 2.0 * u[2], abs=1e-12)
            assert math.atan2(out[2], out[1]) % (2 * math.pi) == pytest.approx(2 * math.pi * u[3], abs=1e-9)
    assert seen == {oracle.OUT_NONE, oracle.OUT_ELASTIC, oracle.OUT_NULL}
