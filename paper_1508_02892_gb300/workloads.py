"""Seeded synthetic inputs for the electron PIC/MCC step of arXiv 1508.02892.

This module is the one place both the CUDA library's tests/benchmark and the
FP64 oracle take their inputs from.  It holds no step of the method: it only
writes parameter dictionaries and input tables (cross sections, ion transport
tables) and seeded particle sets.  Every derived quantity of the method (gas
density, weights, nu_max, table lookups, ...) is computed separately on each
side.

Stand-ins (the paper's tabulated data are not available):
  * electron-neutral cross sections: 1000 points log-spaced over 0.01-1000 eV;
    elastic flat; an inelastic process with threshold E_th and peak sigma_pk has
    sigma = sigma_pk * e * ln(x) / x, x = E/E_th >= 1 (peaks at x = e), and zero
    below threshold (Table 1 lists the processes; the XPDP1 data is replaced);
  * ion mobility and momentum-exchange frequency: 64 points over E/N in
    0..2000 Td, from the fits of Tables 2/3 (He+ in He) or Tables 4/5 (heavy
    ions, used for the Ar+ stand-in), the frequency evaluated at u_k = mu_k E_k.
"""
from __future__ import annotations

import math

import numpy as np

ATM = 101325.0
KB_INPUT = 1.380649e-23   # only to turn E/N into E when sampling the printed fits

GAS_HE, GAS_AR = 0, 1
ION_DD_CONST, ION_DD_TABLE, ION_FULL, ION_KINETIC = 0, 1, 2, 3
FP64, FP32_SPLIT = 0, 1

HE_EXC_EV, HE_IZ_EV = 19.8, 24.6
AR_EXC_EV, AR_IZ_EV = 11.5, 15.8


def xs_tables(gas: int = GAS_HE, n: int = 1000, e_lo: float = 0.01, e_hi: float = 1000.0):
    """Cross-section tables (energies in eV, sigma in m^2)."""
    ev = e_lo * 10.0 ** (np.arange(n) * (math.log10(e_hi / e_lo) / (n - 1)))
    ev[0], ev[-1] = e_lo, e_hi
    if gas == GAS_HE:
        s_el, (e_x, s_x), (e_i, s_i) = 6e-20, (HE_EXC_EV, 5e-21), (HE_IZ_EV, 3.5e-21)
    else:
        # Ar: elastic 1e-19 m^2; inelastic peaks are placeholders (not given)
        s_el, (e_x, s_x), (e_i, s_i) = 1e-19, (AR_EXC_EV, 1e-20), (AR_IZ_EV, 3e-20)

    def shape(e_th, s_pk):
        x = ev / e_th
        out = np.zeros_like(ev)
        m = x >= 1.0
        out[m] = s_pk * math.e * np.log(x[m]) / x[m]
        return out

    return {"xs_ev": ev, "xs_el": np.full(n, s_el), "xs_exc": shape(e_x, s_x),
            "xs_ion": shape(e_i, s_i), "e_exc_ev": e_x, "e_iz_ev": e_i}


def _mu_he(e):      # Table 2, m^2/(V s)
    e0 = 1.47e6
    e = np.abs(e)
    return np.where(e < e0, 1.18 - 0.185 * e / e0, 0.94 * (e0 / np.maximum(e, 1e-30)) ** 0.3) * 1e-3


def _nu_he(u):      # Table 3, 1/s
    u0 = 2e3
    u = np.abs(u)
    return np.where(u < u0, 2.07 + 0.88 * (u / u0) ** 1.89, 1.54 + 1.36 * u / u0) * 1e10


def _mu_heavy(e):   # Table 4, m^2/(V s)
    e0 = 2e6
    e = np.abs(e)
    return np.where(e < e0, 3.05 - 0.75 * e / e0, 2.3 * (e0 / np.maximum(e, 1e-30)) ** 0.37) * 1e-4


def _nu_heavy(u):   # Table 5 as printed, 1/s
    u0 = 4e2
    u = np.abs(u)
    return np.where(u < u0, 6.0 + 7e-6 * u ** 2.04, 4.5 + 27.0 * u / u0) * 1e9


def ion_tables(kind: str, pressure_pa: float, gas_temp_k: float, n: int = 64, eon_max_td: float = 2000.0):
    """Mobility and exchange-frequency tables over E/N (Td)."""
    ngas = pressure_pa / (KB_INPUT * gas_temp_k)
    eon = np.linspace(0.0, eon_max_td, n)
    e = eon * 1e-21 * ngas
    mu_f, nu_f = (_mu_he, _nu_he) if kind == "he" else (_mu_heavy, _nu_heavy)
    mu = mu_f(e)
    nu = nu_f(mu * e)
    return {"tab_eon_td": eon, "tab_mu": mu, "tab_nu": nu}


def base_params(**kw) -> dict:
    p = dict(gap_m=0.5e-3, n_cells=200, gas=GAS_HE, pressure_pa=ATM, gas_temp_k=300.0,
             v_rf_amp_v=150.0, f_rf_hz=13.56e6, v_dc_v=0.0, dt_s=2e-13, n_particles=20000,
             n0_m3=1e16, te0_ev=2.0, weight=0.0, gamma_see=0.0, see_energy_ev=1.0,
             ion_model=ION_DD_CONST, ion_mass_amu=0.0, gas_mass_amu=0.0, mu_const=1.0e-3,
             seed=1, eedf_bins=256, eedf_max_ev=64.0, flags=0, precision=FP64,
             capacity_factor=2.0, sort_interval=0, power_w_m2=0.0, power_alpha=0.0, metastables=0,
             met_diff_m2s=0.0, met_n0_m3=0.0, penning_rate_m3s=0.0, penning_target_m3=0.0, penning_energy_ev=0.0,
             pooling_rate_m3s=0.0, pooling_energy_ev=0.0, gamma_met=0.0)
    p.update(kw)
    gas = p["gas"]
    kind = "he" if gas == GAS_HE else "heavy"
    # the stand-in tables, unless the caller gave tables of its own
    for k, v in {**xs_tables(gas), **ion_tables(kind, p["pressure_pa"], p["gas_temp_k"])}.items():
        p.setdefault(k, v)
    return p


def metastable_params(**kw) -> dict:
    """He metastables with a N2 admixture (Sec. II.D reactions), stand-in values
    of the usual order of magnitude: D p = 470 cm^2 Torr/s at 1 atm, Penning
    ionization of N2 at 7e-17 m^3/s by a 10 ppm admixture, pooling at 1.5e-15
    m^3/s; electron energies E_exc - E_I(N2) and 2 E_exc - E_iz with Table 1's
    19.8 and 24.6 eV."""
    p = dict(metastables=1, met_diff_m2s=6.2e-5, met_n0_m3=0.0, penning_rate_m3s=7e-17,
             penning_target_m3=1e-5 * ATM / (1.380649e-23 * 300.0), penning_energy_ev=19.8 - 15.58,
             pooling_rate_m3s=1.5e-15, pooling_energy_ev=2 * 19.8 - 24.6, gamma_met=0.0)
    p.update(kw)
    return p


def config1(**kw) -> dict:
    """Plain method, FP64, one instance: He 1 atm 300 K, 0.5 mm / 200 cells,
    150 V 13.56 MHz, gamma 0, 2e4 electrons at 2 eV, DD with mu = 1e-3."""
    p = base_params(precision=FP64)
    p.update(kw)
    return p


def config2(**kw) -> dict:
    """Single-instance production run: He 1 atm, 1 mm / 1000 cells, 250 V,
    2e6 electrons, gamma 0.1, full ion fluid with He+ tables, FP32 split."""
    p = base_params(gap_m=1e-3, n_cells=1000, v_rf_amp_v=250.0, n_particles=2_000_000,
                    gamma_see=0.1, ion_model=ION_FULL, precision=FP32_SPLIT, seed=2)
    p.update(kw)
    return p


def config5(**kw) -> dict:
    """Heavy ions in gamma mode: Ar 1 atm, 1 mm / 4000 cells, 400 V, gamma 0.15,
    5e7 electrons, full fluid with the heavy-ion stand-in tables, dt 1e-13."""
    p = base_params(gas=GAS_AR, gap_m=1e-3, n_cells=4000, v_rf_amp_v=400.0, n_particles=50_000_000,
                    gamma_see=0.15, ion_model=ION_FULL, precision=FP32_SPLIT, dt_s=1e-13, seed=5,
                    capacity_factor=1.5)
    p.update(kw)
    return p


def config3_instances(n: int = 64, seed: int = 2026, n_max: float = 2e6, scale: float = 1.0):
    """Batched helium discharges: gap U(0.3, 2) mm, cells 150..2000 monotone in
    the gap, electrons log-uniform 1e4..n_max, voltage U(100, 400) V, drift-
    diffusion (tabulated mobility) or full fluid with probability 1/2 each,
    instance i seeded 1000 + i.  `scale` multiplies the particle counts."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        gap = rng.uniform(0.3e-3, 2e-3)
        cells = int(round(150 + (gap - 0.3e-3) / 1.7e-3 * 1850))
        npart = int(math.exp(rng.uniform(math.log(1e4), math.log(n_max))) * scale)
        volt = rng.uniform(100.0, 400.0)
        model = ION_FULL if rng.uniform() < 0.5 else ION_DD_TABLE
        out.append(base_params(gap_m=gap, n_cells=cells, n_particles=max(npart, 64), v_rf_amp_v=volt,
                               gamma_see=0.1, ion_model=model, precision=FP32_SPLIT, seed=1000 + i))
    return out


def config4_requests(n_requests: int = 200, rate_hz: float = 20.0, seed: int = 4242, n_max: float = 4e6,
                     steps: int = 5000, scale: float = 1.0):
    """Serving load: Poisson arrivals (exponential gaps, mean 1/rate), each a
    discharge drawn from the batched ranges advanced by `steps` steps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    reqs = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        gap = rng.uniform(0.3e-3, 2e-3)
        cells = int(round(150 + (gap - 0.3e-3) / 1.7e-3 * 1850))
        npart = int(math.exp(rng.uniform(math.log(1e4), math.log(n_max))) * scale)
        volt = rng.uniform(100.0, 400.0)
        model = ION_FULL if rng.uniform() < 0.5 else ION_DD_TABLE
        p = base_params(gap_m=gap, n_cells=cells, n_particles=max(npart, 64), v_rf_amp_v=volt,
                        gamma_see=0.1, ion_model=model, precision=FP32_SPLIT, seed=5000 + i)
        reqs.append({"arrival_s": t, "steps": steps, "params": p})
    return reqs


def random_particles(n: int, gap_m: float, te_ev: float, seed: int, id_base: int = 0):
    """Seeded particle set: uniform positions in [0, gap), Maxwellian velocities
    (numpy normal), ids id_base..id_base+n-1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    vth = math.sqrt(1.602176634e-19 * te_ev / 9.1093837015e-31)
    z = rng.uniform(0.0, gap_m, n)
    v = rng.normal(0.0, vth, (3, n))
    return {"z": z, "vx": v[0].copy(), "vy": v[1].copy(), "vz": v[2].copy(),
            "id": np.arange(id_base, id_base + n, dtype=np.uint64)}


SWARM_QM, SWARM_QI_ONLY = 0, 1


def swarm_params(**kw) -> dict:
    """Auxiliary ion swarm (Sec. II.C): He+ in He at 1 atm and 300 K, ions
    starting from a 300 K Maxwellian, dt 1e-13 s, 20000 steps of which the
    first 4000 relax, Q_m = Q_i + 2 Q_b, FP64, collision bound over relative
    energies up to 10 eV."""
    p = dict(gas_mass_amu=0.0, ion_mass_amu=0.0, pressure_pa=101325.0, gas_temp_k=300.0, ion_temp0_k=300.0,
             dt_s=1e-13, nu_max=0.0, eps_max_ev=10.0, n_ions=4096, n_steps=20000, n_relax=4000,
             xs_model=SWARM_QM, precision=FP64, seed=11)
    p.update(kw)
    return p


def swarm_fields(n: int = 64, e_max: float = 5e6) -> np.ndarray:
    """Field values for a mobility table: n points evenly spaced in (0, e_max]."""
    return np.linspace(e_max / n, e_max, n)


def recombination_table(k_m3_s: float, gas: int = GAS_HE) -> np.ndarray:
    """Stand-in electron-ion recombination cross section on the electron
    cross-section grid: sigma(E) = k / v(E), i.e. a rate coefficient sigma v = k
    (m^3/s) independent of energy at the table nodes.  The paper names the
    process (Sec. II.D) but gives no data for it."""
    ev = xs_tables(gas)["xs_ev"]
    v = np.sqrt(2.0 * 1.602176634e-19 * ev / 9.1093837015e-31)
    return k_m3_s / v

