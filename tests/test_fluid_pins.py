"""Pins of the oracle's ion-fluid arithmetic (Secs. II.B-II.C of the paper).

Every expected value here is written from the printed equations and solved
with numpy on the spot; nothing calls the oracle's own formulas:
  * Eq. 2.3 (full model): hand-assembled 3- and 5-node systems with
    non-uniform n, T, E and a flux of both signs, solved densely, and the
    continuity rows of Eq. 2.4 with the half-cell wall rows;
  * the table lookups: mu at E/N (Tables 2/4 as input), nu at the drift speed
    u on the abscissa u_k = mu_k E_k (Tables 3/5), at nodes, midpoints and both
    clamps, against numpy.interp;
  * Eq. 2.8 ion temperature at two fields and two mass ratios;
  * drift-diffusion with the table mobility and the Eq. 2.7 D: the explicit
    scheme's exact moment laws (centroid moves mu E dt per step, variance grows
    2 D dt - (mu E dt)^2 per step);
  * the field-driven wall flux alpha mu n E of Sec. II.C.
Each test also checks that the terms it pins change its answer well beyond
its tolerance, and ``test_oracle_mutations.py`` plants plausible mistakes in a
copy of the oracle and checks that these tests fail.  CPU only.
"""
import numpy as np
import pytest

import oracle
from paper_1508_02892_gb300 import workloads as W

QE, KB, AMU = 1.602176634e-19, 1.380649e-23, 1.66053906660e-27
M_HE = 4.002602 * AMU
NGAS = W.ATM / (KB * 300.0)


def _oracle(model, G, L, dt, **kw):
    p = W.base_params(n_particles=0, n0_m3=1e16, v_rf_amp_v=0.0, v_dc_v=0.0, f_rf_hz=0.0, gap_m=L,
                      n_cells=G - 1, ion_model=model, dt_s=dt, weight=1.0)
    p.update(kw)
    return oracle.Oracle(p), p


def _mu(p, e_abs):
    """Mobility from the input table at E/N in Td (Sec. II.C)."""
    return np.interp(np.abs(e_abs) / NGAS * 1e21, p["tab_eon_td"], p["tab_mu"])


def _u_nodes(p):
    """Abscissa of the exchange-frequency table: drift speed mu_k E_k."""
    return p["tab_mu"] * p["tab_eon_td"] * 1e-21 * NGAS


def _nu(p, u_abs):
    return np.interp(np.abs(u_abs), _u_nodes(p), p["tab_nu"])


def _temp(mu, e_abs, mi=M_HE, mn=M_HE):
    """Eq. 2.8: T_i = T_N + (m_i + m_N)/(5 m_i + 3 m_N) m_N (mu |E|)^2 (J)."""
    return KB * 300.0 + (mi + mn) / (5 * mi + 3 * mn) * mn * (mu * np.abs(e_abs)) ** 2


def _wall(p, n, E, wall):
    into = E < 0 if wall == 0 else E > 0
    return _mu(p, E) * n * E if into else 0.0


def _eq23(p, n, gam_old, E, dt, dz, advection=True, pressure=True, nu_at=None, A=None, own_ratio=False):
    """Solve Eq. 2.3 for Gamma^{n+1/2} at the interior nodes with the wall
    fluxes as Dirichlet values, by a dense solve of the printed equation.
    A (default Gamma^{n-1/2}/n^n) is the ratio in the advection term and the
    drift speed at which nu is looked up.  advection/pressure=False drop a
    term, nu_at looks nu up elsewhere and own_ratio takes the node's own ratio
    A_j in place of A_{j+-1}: the variants that show a term is live."""
    G = n.size
    mu = _mu(p, E)
    T = _temp(mu, E)
    if A is None:
        A = gam_old / n                                # Gamma^{n-1/2} / n^n
    u = A if nu_at is None else nu_at
    nu = _nu(p, u)
    g0, gN = _wall(p, n[0], E[0], 0), _wall(p, n[-1], E[-1], 1)
    m = G - 2
    M = np.zeros((m, m))
    rhs = np.zeros(m)
    h = dt / (2 * dz)
    for k in range(m):
        j = k + 1
        M[k, k] = 1 + nu[j] * dt / 2
        rhs[k] = gam_old[j] * (1 - nu[j] * dt / 2) + QE * n[j] * E[j] * dt / M_HE
        if pressure:
            rhs[k] -= dt / (2 * dz * M_HE) * (n[j + 1] * T[j + 1] - n[j - 1] * T[j - 1])
        if advection:
            # + h (Gamma_{j+1} A_{j+1} - Gamma_{j-1} A_{j-1})
            for jj, sgn in ((j + 1, 1.0), (j - 1, -1.0)):
                coef = sgn * h * (A[j] if own_ratio else A[jj])
                if jj == 0:
                    rhs[k] -= coef * g0
                elif jj == G - 1:
                    rhs[k] -= coef * gN
                else:
                    M[k, jj - 1] += coef
    x = np.linalg.solve(M, rhs)
    return np.concatenate([[g0], x, [gN]])


def _continuity(n, g, src, dt, dz):
    """Eq. 2.4 at the interior nodes; the wall rows integrate the continuity
    equation over the half cell [z_0, z_1/2] with Gamma_1/2 = (Gamma_0 + Gamma_1)/2."""
    out = n.copy()
    out[1:-1] = n[1:-1] - dt / (2 * dz) * (g[2:] - g[:-2]) + dt * src[1:-1]
    g_half0 = 0.5 * (g[0] + g[1])
    g_halfN = 0.5 * (g[-1] + g[-2])
    out[0] = n[0] - 2 * dt / dz * (g_half0 - g[0]) + dt * src[0]
    out[-1] = n[-1] - 2 * dt / dz * (g[-1] - g_halfN) + dt * src[-1]
    return out


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


# five-node case: n, T (through E), Gamma^{n-1/2} of both signs, both walls
# receiving ions (E < 0 at z = 0, E > 0 at z = L)
N5 = np.array([2.0e16, 1.0e16, 3.0e16, 1.5e16, 0.8e16])
E5 = np.array([-3.0e6, 1.0e6, -2.0e6, 5.0e5, 4.0e6])
G5 = np.array([-5.0e19, 1.0e20, -2.0e20, 1.0e20, 4.0e19])
SRC5 = np.array([3.0e27, 1.0e27, 0.0, 2.0e27, 5.0e26])


@pytest.mark.parametrize("case", ["3-node", "5-node"])
def test_eq_2_3_hand_solved_system(case):
    if case == "3-node":
        n, E, g, src = N5[1:4].copy(), E5[[0, 1, 4]].copy(), G5[1:4].copy(), SRC5[1:4].copy()
        L = 5.0e-5
    else:
        n, E, g, src = N5, E5, G5, SRC5
        L = 1.0e-4
    G = n.size
    dt, dz = 1.0e-11, L / (G - 1)
    o, p = _oracle(W.ION_FULL, G, L, dt)
    n1, g1, flux, cl = o.fluid_update(E, src, n, g)
    want_g = _eq23(p, n, g, E, dt, dz)
    assert cl == 0
    np.testing.assert_allclose(g1, want_g, rtol=1e-12, atol=1e-12 * np.abs(want_g).max())
    np.testing.assert_allclose(n1, _continuity(n, want_g, src, dt, dz), rtol=1e-12)
    assert flux[0] == -want_g[0] and flux[1] == want_g[-1]
    assert want_g[0] < 0 < want_g[-1]
    # every term pinned here moves the answer far beyond the tolerance
    for kw in (dict(advection=False), dict(pressure=False), dict(nu_at=E / NGAS * 1e21), dict(own_ratio=True)):
        assert _rel(_eq23(p, n, g, E, dt, dz, **kw)[1:-1], want_g[1:-1]) > 1e-6, kw


def test_eq_2_3_three_nodes_by_hand():
    """The single interior row of a 3-node system, solved by hand."""
    n = np.array([1.0e16, 3.0e16, 2.0e16])
    E = np.array([-1.0e6, 2.0e6, 3.0e6])
    g = np.array([-2.0e19, 6.0e19, 1.0e20])
    dt, L = 1.0e-11, 5.0e-5
    dz = L / 2
    o, p = _oracle(W.ION_FULL, 3, L, dt)
    _, g1, _, _ = o.fluid_update(E, np.zeros(3), n, g)
    mu = _mu(p, E)
    T = _temp(mu, E)
    g0 = mu[0] * n[0] * E[0]                # into the wall at z = 0
    g2 = mu[2] * n[2] * E[2]                # into the wall at z = L
    nu1 = _nu(p, g[1] / n[1])
    h = dt / (2 * dz)
    rhs = (g[1] * (1 - nu1 * dt / 2) + QE * n[1] * E[1] * dt / M_HE
           - h / M_HE * (n[2] * T[2] - n[0] * T[0])
           - h * (g2 * g[2] / n[2] - g0 * g[0] / n[0]))
    want = rhs / (1 + nu1 * dt / 2)
    assert g1[0] == pytest.approx(g0, rel=1e-14, abs=0)
    assert g1[2] == pytest.approx(g2, rel=1e-14, abs=0)
    assert g1[1] == pytest.approx(want, rel=1e-13, abs=0)


def test_eq_2_3_density_floor_drops_advection_ratio():
    """Below the floor (1e-6 n0) the ratio Gamma/n is taken as 0: the node's
    advection coefficient and the drift speed of its nu vanish, while its own
    Gamma^{n-1/2} still enters its right-hand side."""
    n = N5.copy()
    n[2] = 1e9                               # below 1e-6 * 1e16
    dt, L = 1.0e-11, 1.0e-4
    dz = L / 4
    o, p = _oracle(W.ION_FULL, 5, L, dt)
    _, g1, _, _ = o.fluid_update(E5, np.zeros(5), n, G5)
    A = G5 / n
    A[2] = 0.0
    want = _eq23(p, n, G5, E5, dt, dz, A=A)
    np.testing.assert_allclose(g1, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    assert _rel(_eq23(p, n, G5, E5, dt, dz)[1:-1], want[1:-1]) > 1e-6


@pytest.mark.parametrize("kind", ["he", "heavy"])
def test_mobility_lookup_nodes_midpoints_clamps(kind):
    gas = W.GAS_HE if kind == "he" else W.GAS_AR
    o, p = _oracle(W.ION_DD_TABLE, 11, 1e-4, 2e-13, gas=gas)
    eon, mu = p["tab_eon_td"], p["tab_mu"]
    e_of = lambda td: td * 1e-21 * NGAS
    for k in (1, 7, 30, 62):
        assert o.transport(e_of(eon[k]))[0] == pytest.approx(mu[k], rel=1e-12, abs=0)
        mid = 0.5 * (eon[k] + eon[k + 1])
        assert o.transport(e_of(mid))[0] == pytest.approx(0.5 * (mu[k] + mu[k + 1]), rel=1e-12, abs=0)
    assert o.transport(0.0)[0] == mu[0]
    assert o.transport(e_of(2.5 * eon[-1]))[0] == mu[-1]
    # a sample of fields against numpy's interpolation
    for e in np.linspace(0, 1.1 * e_of(eon[-1]), 37):
        assert o.transport(e)[0] == pytest.approx(float(_mu(p, e)), rel=1e-12, abs=0)


@pytest.mark.parametrize("kind", ["he", "heavy"])
def test_exchange_frequency_lookup_on_drift_speed(kind):
    gas = W.GAS_HE if kind == "he" else W.GAS_AR
    o, p = _oracle(W.ION_FULL, 11, 1e-4, 2e-13, gas=gas)
    uk, nu = _u_nodes(p), p["tab_nu"]
    assert np.all(np.diff(uk) > 0)           # monotone abscissa
    for k in (0, 5, 20, 62):
        assert o.transport(0.0, uk[k])[3] == pytest.approx(nu[k], rel=1e-12, abs=0)
        assert o.transport(0.0, 0.5 * (uk[k] + uk[k + 1]))[3] == pytest.approx(0.5 * (nu[k] + nu[k + 1]),
                                                                               rel=1e-12, abs=0)
    assert o.transport(0.0, 0.0)[3] == nu[0]
    assert o.transport(0.0, 3 * uk[-1])[3] == nu[-1]
    for u in np.linspace(0, 1.2 * uk[-1], 41):
        assert o.transport(0.0, u)[3] == pytest.approx(float(_nu(p, u)), rel=1e-12, abs=0)
    # the abscissa is the drift speed, not E/N: the two lookups differ
    assert abs(o.transport(0.0, 500.0)[3] - float(np.interp(500.0, p["tab_eon_td"], nu))) > 1e-3 * nu[0]


@pytest.mark.parametrize("mass_ratio", [1.0, 10.0])
@pytest.mark.parametrize("e_field", [5.0e5, 8.0e6])
def test_ion_temperature_eq_2_8(mass_ratio, e_field):
    o, p = _oracle(W.ION_DD_TABLE, 11, 1e-4, 2e-13, ion_mass_amu=4.002602 * mass_ratio)
    mu, T, D, _ = o.transport(e_field)
    mi, mn = M_HE * mass_ratio, M_HE
    ud = float(_mu(p, e_field)) * e_field
    # the mass factor in closed form: 1/4 for equal masses, 11/53 for m_i = 10 m_N
    frac = {1.0: 0.25, 10.0: 11.0 / 53.0}[mass_ratio]
    want = KB * 300.0 + frac * mn * ud * ud
    assert T == pytest.approx(want, rel=1e-13, abs=0)
    assert D == pytest.approx(mu * want / QE, rel=1e-13, abs=0)        # Eq. 2.7
    assert (T - KB * 300.0) / (KB * 300.0) > 1e-3                # the field term is live
    # constant-mobility drift-diffusion keeps the gas temperature
    oc, _ = _oracle(W.ION_DD_CONST, 11, 1e-4, 2e-13, ion_mass_amu=4.002602 * mass_ratio)
    assert oc.transport(e_field)[1] == KB * 300.0
    del mi


def test_dd_table_moment_laws_with_eq_2_7_diffusion():
    """Explicit drift-diffusion (Eq. 2.5 at level n into Eq. 2.4) in a uniform
    field: the centroid moves mu E dt and the variance grows by exactly
    2 D dt - (mu E dt)^2 per step, with mu from the table at E/N and D from
    Eqs. 2.7-2.8."""
    G, L, dt = 201, 1e-3, 2e-13
    o, p = _oracle(W.ION_DD_TABLE, G, L, dt)
    z = np.linspace(0, L, G)
    n = 1e16 * np.exp(-0.5 * ((z - L / 2) / (L / 20)) ** 2)
    gam = np.zeros(G)
    E0 = 2.0e6
    E = np.full(G, E0)
    mu = float(_mu(p, E0))
    D = mu * _temp(mu, E0) / QE
    u = mu * E0
    steps = 1500
    m0 = n.sum()
    c0 = (n * z).sum() / m0
    v0 = (n * z * z).sum() / m0 - c0 ** 2
    for _ in range(steps):
        n, gam, _, cl = o.fluid_update(E, np.zeros(G), n, gam)
        assert cl == 0
    c1 = (n * z).sum() / n.sum()
    v1 = (n * z * z).sum() / n.sum() - c1 ** 2
    assert n.sum() == pytest.approx(m0, rel=1e-12, abs=0)
    assert c1 - c0 == pytest.approx(u * dt * steps, rel=1e-7, abs=0)
    want = (2 * D * dt - (u * dt) ** 2) * steps
    assert v1 - v0 == pytest.approx(want, rel=1e-6, abs=0)
    # both the field-heated D and the FTCS term are well above the tolerance
    d_gas = mu * KB * 300.0 / QE
    assert abs(2 * (D - d_gas) * dt * steps) > 1e-2 * want
    assert (u * dt) ** 2 * steps > 1e-4 * want


@pytest.mark.parametrize("model", [W.ION_DD_CONST, W.ION_DD_TABLE, W.ION_FULL])
def test_wall_flux_is_mu_n_E_into_the_electrode(model):
    G, L, dt = 11, 1e-4, 2e-13
    o, p = _oracle(model, G, L, dt)
    n = np.linspace(1e16, 3e16, G)
    gam = np.zeros(G)
    mu = (lambda e: p["mu_const"]) if model == W.ION_DD_CONST else (lambda e: float(_mu(p, e)))
    E = np.full(G, 1e5)
    E[0], E[-1] = -2.5e6, 7.0e6              # both point into their electrode
    _, g1, flux, _ = o.fluid_update(E, np.zeros(G), n, gam)
    assert g1[0] == pytest.approx(mu(E[0]) * n[0] * E[0], rel=1e-14, abs=0)
    assert g1[-1] == pytest.approx(mu(E[-1]) * n[-1] * E[-1], rel=1e-14, abs=0)
    assert flux[0] == pytest.approx(-g1[0], rel=0, abs=0) and flux[1] == pytest.approx(g1[-1], rel=0, abs=0)
    E[0], E[-1] = 2.5e6, -7.0e6              # both point out of their electrode: alpha = 0
    _, g1, flux, _ = o.fluid_update(E, np.zeros(G), n, gam)
    assert g1[0] == 0.0 and g1[-1] == 0.0 and flux[0] == 0.0 and flux[1] == 0.0
