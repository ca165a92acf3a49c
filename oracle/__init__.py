"""FP64 CPU oracle of the kinetic-electron PIC/MCC step (arXiv 1508.02892, Sec. II).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package.  It shares
no code with the CUDA library in ``paper_1508_02892_gb300``; the one thing both
sides take from a common place is the seeded input generator
``paper_1508_02892_gb300.workloads`` (parameters and tables, no method
arithmetic).

The arithmetic lives in ``oracle.c`` (plain C, FP64, single thread); this module
compiles it with gcc and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

GRID_NE, GRID_NI, GRID_GAMMA, GRID_PHI, GRID_E, GRID_GSRC = range(6)
ION_KINETIC = 3
OUT_NONE, OUT_ELASTIC, OUT_EXC, OUT_ION, OUT_NULL, OUT_LOST0, OUT_LOST1 = range(7)
FLAG_THERMAL_GAS = 2

COUNTER_NAMES = ("step", "particles", "births_iz", "births_see0", "births_see1", "losses0",
                 "losses1", "elastic", "excitation", "ionization", "null", "clamps", "status", "recombinations",
                 "births_penning", "births_pooling")


SRC = _SRC


def build(force: bool = False, src: str | None = None, out: str | None = None) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, -O2, no FP contraction so
    that x86 and Arm give the same bits).  `src`/`out` build another copy of
    the source (the mutation tests plant mistakes in such a copy)."""
    src = src or _SRC
    out = out or _LIB_PATH
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class OrcParams(C.Structure):
    _fields_ = [
        ("gap_m", C.c_double), ("n_cells", C.c_int32), ("gas", C.c_int32),
        ("pressure_pa", C.c_double), ("gas_temp_k", C.c_double),
        ("v_rf_amp_v", C.c_double), ("f_rf_hz", C.c_double), ("v_dc_v", C.c_double),
        ("dt_s", C.c_double), ("n_particles", C.c_int64), ("n0_m3", C.c_double),
        ("te0_ev", C.c_double), ("weight", C.c_double), ("gamma_see", C.c_double),
        ("see_energy_ev", C.c_double), ("ion_model", C.c_int32),
        ("ion_mass_amu", C.c_double), ("gas_mass_amu", C.c_double), ("mu_const", C.c_double),
        ("tab_eon_td", C.POINTER(C.c_double)), ("tab_mu", C.POINTER(C.c_double)),
        ("tab_nu", C.POINTER(C.c_double)), ("n_tab", C.c_int32),
        ("xs_ev", C.POINTER(C.c_double)), ("xs_el", C.POINTER(C.c_double)),
        ("xs_exc", C.POINTER(C.c_double)), ("xs_ion", C.POINTER(C.c_double)),
        ("n_xs", C.c_int32), ("e_exc_ev", C.c_double), ("e_iz_ev", C.c_double),
        ("seed", C.c_uint64), ("eedf_bins", C.c_int32), ("eedf_max_ev", C.c_double),
        ("flags", C.c_int32), ("power_w_m2", C.c_double), ("power_alpha", C.c_double),
        ("xs_rec", C.POINTER(C.c_double)), ("metastables", C.c_int32), ("met_diff_m2s", C.c_double),
        ("met_n0_m3", C.c_double), ("penning_rate_m3s", C.c_double), ("penning_target_m3", C.c_double),
        ("penning_energy_ev", C.c_double), ("pooling_rate_m3s", C.c_double), ("pooling_energy_ev", C.c_double),
        ("gamma_met", C.c_double),
    ]


class OrcSwarmParams(C.Structure):
    _fields_ = [("gas_mass_amu", C.c_double), ("ion_mass_amu", C.c_double), ("pressure_pa", C.c_double),
                ("gas_temp_k", C.c_double), ("ion_temp0_k", C.c_double), ("dt_s", C.c_double),
                ("e_field", C.c_double), ("nu_max", C.c_double), ("eps_max_ev", C.c_double),
                ("n_ions", C.c_int64), ("n_steps", C.c_int64), ("n_relax", C.c_int64), ("id_base", C.c_int64),
                ("xs_model", C.c_int32), ("seed", C.c_uint64)]


class OrcSwarmResult(C.Structure):
    _fields_ = [("drift", C.c_double), ("mean_energy_ev", C.c_double), ("mobility", C.c_double),
                ("nu_exchange", C.c_double), ("nu_max", C.c_double), ("p_max", C.c_double),
                ("candidates", C.c_int64), ("collisions", C.c_int64), ("overruns", C.c_int64)]


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib


def use_library(L) -> None:
    """Route every later call of this module to the library L (from load());
    the mutation tests swap a planted-mistake copy in and back out."""
    global _lib
    with _lock:
        _lib = L


def load(path: str):
    """Load a compiled copy of oracle.c and declare its signatures."""
    L = C.CDLL(path)
    vp, i64, u64, u32, i32, dbl = C.c_void_p, C.c_int64, C.c_uint64, C.c_uint32, C.c_int32, C.c_double
    pd = C.POINTER(C.c_double)
    pu64 = C.POINTER(C.c_uint64)
    pi64 = C.POINTER(C.c_int64)
    pu32 = C.POINTER(C.c_uint32)
    sig = {
        "orc_create": (vp, [C.POINTER(OrcParams)]),
        "orc_destroy": (None, [vp]),
        "orc_step": (C.c_int, [vp, i64]),
        "orc_num_particles": (i64, [vp]),
        "orc_num_nodes": (C.c_int, [vp]),
        "orc_get_particles": (None, [vp, pd, pd, pd, pd, pu64]),
        "orc_set_particles": (None, [vp, i64, pd, pd, pd, pd, pu64]),
        "orc_get_grid": (None, [vp, C.c_int, pd]),
        "orc_set_grid": (None, [vp, C.c_int, pd]),
        "orc_get_moments": (i64, [vp, pd, pd, pd, pd, pd]),
        "orc_get_eedf_counts": (None, [vp, pd]),
        "orc_get_counters": (None, [vp, pi64]),
        "orc_get_flux_in": (None, [vp, pd]),
        "orc_set_flux_in": (None, [vp, pd]),
        "orc_emit_only": (i64, [vp, u32]),
        "orc_init_field": (None, [vp]),
        "orc_xs_eval": (None, [vp, dbl, pd]),
        "orc_nu_max": (dbl, [vp]),
        "orc_p_max": (dbl, [vp]),
        "orc_weight": (dbl, [vp]),
        "orc_ngas": (dbl, [vp]),
        "orc_philox4x32_10": (None, [pu32, pu32, pu32]),
        "orc_u01": (dbl, [u32]),
        "orc_mix64": (u64, [u64]),
        "orc_child_id": (u64, [u64, u32]),
        "orc_see_id": (u64, [C.c_int, u32, u32]),
        "orc_poisson": (None, [C.c_int, dbl, pd, dbl, dbl, pd, pd]),
        "orc_fluid_update": (i64, [vp, pd, pd, pd, pd, pd]),
        "orc_particle_step_one": (C.c_int, [vp, pd, u32, pd, u64, pd, pd, pu64]),
        "orc_ion_step_one": (C.c_int, [vp, pd, u32, pd, u64, pd]),
        "orc_swarm_run": (None, [C.POINTER(OrcSwarmParams), C.POINTER(OrcSwarmResult), pd]),
        "orc_get_power": (None, [vp, pd, pi64]),
        "orc_get_ion_counters": (None, [vp, pi64]),
        "orc_get_metastables": (None, [vp, pd, pd, pd]),
        "orc_set_metastables": (None, [vp, pd]),
        "orc_get_ions": (None, [vp, pd, pd, pd, pd, pu64]),
        "orc_swarm_nu": (dbl, [dbl, dbl, C.c_int, dbl]),
        "orc_swarm_nu_bound": (dbl, [dbl, dbl, C.c_int, dbl]),
        "orc_swarm_qi": (dbl, [dbl]),
        "orc_swarm_qb": (dbl, [dbl]),
        "orc_ion_transport": (None, [vp, dbl, dbl, pd]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


# ----------------------------------------------------------------- helpers ---

def swarm_run(params: dict, e_field: float, id_base: int = 0, velocities: bool = False):
    """The ion-swarm Monte Carlo of Sec. II.C at one field value (ions
    id_base .. id_base + n_ions - 1); returns the result dict and, if asked,
    the final velocities (n_ions x 3)."""
    p = OrcSwarmParams()
    for name, _ in OrcSwarmParams._fields_:
        if name in params:
            setattr(p, name, params[name])
    p.e_field = float(e_field)
    p.id_base = int(id_base)
    r = OrcSwarmResult()
    v = np.zeros(3 * int(p.n_ions)) if velocities else None
    lib().orc_swarm_run(C.byref(p), C.byref(r), _dp(v) if v is not None else None)
    out = {f: getattr(r, f) for f, _ in OrcSwarmResult._fields_}
    return (out, v.reshape(-1, 3)) if velocities else out


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return tuple(int(x) for x in o)


def u01(x):
    return lib().orc_u01(int(x) & 0xFFFFFFFF)


def mix64(x):
    return lib().orc_mix64(int(x) & 0xFFFFFFFFFFFFFFFF)


def child_id(parent, step):
    return lib().orc_child_id(int(parent), int(step))


def see_id(wall, step, k):
    return lib().orc_see_id(int(wall), int(step), int(k))


def poisson(rho, dz, phi0, phiN):
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    G = rho.size
    phi = np.zeros(G)
    E = np.zeros(G)
    lib().orc_poisson(G, float(dz), _dp(rho), float(phi0), float(phiN), _dp(phi), _dp(E))
    return phi, E


class Oracle:
    """One discharge advanced by the FP64 oracle.  `params` is the dict made by
    ``paper_1508_02892_gb300.workloads`` (scalars plus numpy tables)."""

    def __init__(self, params: dict):
        self._keep = {}
        p = OrcParams()
        for name, ctype in OrcParams._fields_:
            if name in ("tab_eon_td", "tab_mu", "tab_nu", "xs_ev", "xs_el", "xs_exc", "xs_ion"):
                arr = np.ascontiguousarray(params.get(name, np.zeros(1)), dtype=np.float64)
                self._keep[name] = arr
                setattr(p, name, _dp(arr))
            elif name == "xs_rec":
                if params.get("xs_rec") is not None:
                    arr = np.ascontiguousarray(params["xs_rec"], dtype=np.float64)
                    self._keep[name] = arr
                    setattr(p, name, _dp(arr))
            elif name in ("n_tab", "n_xs"):
                continue
            elif name in params:
                setattr(p, name, params[name])
        p.n_tab = self._keep["tab_eon_td"].size if "tab_eon_td" in params else 0
        p.n_xs = self._keep["xs_ev"].size
        self._p = p
        self.h = lib().orc_create(C.byref(p))
        if not self.h:
            raise ValueError("oracle rejected the parameters")
        self.G = lib().orc_num_nodes(self.h)
        self.eedf_bins = int(params.get("eedf_bins", 256) or 256)

    def close(self):
        if self.h:
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- driving
    def step(self, n=1):
        return lib().orc_step(self.h, int(n))

    def init_field(self):
        lib().orc_init_field(self.h)

    # --- state
    @property
    def n_particles(self):
        return lib().orc_num_particles(self.h)

    def particles(self):
        n = self.n_particles
        z, vx, vy, vz = (np.zeros(n) for _ in range(4))
        ids = np.zeros(n, dtype=np.uint64)
        lib().orc_get_particles(self.h, _dp(z), _dp(vx), _dp(vy), _dp(vz),
                                ids.ctypes.data_as(C.POINTER(C.c_uint64)))
        return {"z": z, "vx": vx, "vy": vy, "vz": vz, "id": ids}

    def set_particles(self, z, vx, vy, vz, ids):
        z, vx, vy, vz = (np.ascontiguousarray(a, dtype=np.float64) for a in (z, vx, vy, vz))
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        lib().orc_set_particles(self.h, z.size, _dp(z), _dp(vx), _dp(vy), _dp(vz),
                                ids.ctypes.data_as(C.POINTER(C.c_uint64)))

    def grid(self, which):
        out = np.zeros(self.G)
        lib().orc_get_grid(self.h, int(which), _dp(out))
        return out

    def set_grid(self, which, values):
        v = np.ascontiguousarray(values, dtype=np.float64)
        assert v.size == self.G
        lib().orc_set_grid(self.h, int(which), _dp(v))

    def fields(self):
        return {"ne": self.grid(GRID_NE), "ni": self.grid(GRID_NI), "gamma": self.grid(GRID_GAMMA),
                "phi": self.grid(GRID_PHI), "E": self.grid(GRID_E), "gsrc": self.grid(GRID_GSRC)}

    def moments(self):
        G = self.G
        ne, ni, gi, eb = (np.zeros(G) for _ in range(4))
        eedf = np.zeros(self.eedf_bins + 1)
        ns = lib().orc_get_moments(self.h, _dp(ne), _dp(ni), _dp(gi), _dp(eb), _dp(eedf))
        return {"ne": ne, "ni": ni, "gamma": gi, "ebar": eb, "eedf": eedf, "n_samples": int(ns)}

    def eedf_counts(self):
        out = np.zeros(self.eedf_bins + 1)
        lib().orc_get_eedf_counts(self.h, _dp(out))
        return out

    def counters(self):
        out = (C.c_int64 * len(COUNTER_NAMES))()
        lib().orc_get_counters(self.h, out)
        return dict(zip(COUNTER_NAMES, (int(x) for x in out)))

    def flux_in(self):
        out = np.zeros(2)
        lib().orc_get_flux_in(self.h, _dp(out))
        return out

    def set_flux_in(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        lib().orc_set_flux_in(self.h, _dp(f))

    def emit_only(self, step):
        return lib().orc_emit_only(self.h, int(step))

    # --- pieces
    def xs(self, energy_ev):
        out = np.zeros(3)
        lib().orc_xs_eval(self.h, float(energy_ev), _dp(out))
        return out

    @property
    def nu_max(self):
        return lib().orc_nu_max(self.h)

    @property
    def p_max(self):
        return lib().orc_p_max(self.h)

    @property
    def weight(self):
        return lib().orc_weight(self.h)

    @property
    def ngas(self):
        return lib().orc_ngas(self.h)

    def transport(self, e_abs, u_abs=0.0):
        """(mu, T_i in J, D, nu) the fluid update takes at field |E| and drift
        speed |u| (Sec. II.B-II.C, Eqs. 2.7-2.8)."""
        out = np.zeros(4)
        lib().orc_ion_transport(self.h, float(e_abs), float(u_abs), _dp(out))
        return tuple(float(x) for x in out)

    def fluid_update(self, E, gsrc, ni, gam):
        E, gsrc = (np.ascontiguousarray(a, dtype=np.float64) for a in (E, gsrc))
        ni = np.array(ni, dtype=np.float64)
        gam = np.array(gam, dtype=np.float64)
        flux = np.zeros(2)
        clamps = lib().orc_fluid_update(self.h, _dp(E), _dp(gsrc), _dp(ni), _dp(gam), _dp(flux))
        return ni, gam, flux, int(clamps)

    def metastables(self):
        """Metastable density now, its time average, and the flux into each
        wall in the last step."""
        met, avg, flux = np.zeros(self.G), np.zeros(self.G), np.zeros(2)
        lib().orc_get_metastables(self.h, _dp(met), _dp(avg), _dp(flux))
        return {"met": met, "avg": avg, "flux": flux}

    def set_metastables(self, met):
        v = np.ascontiguousarray(met, dtype=np.float64)
        assert v.size == self.G
        lib().orc_set_metastables(self.h, _dp(v))

    def ion_counters(self):
        """Kinetic ions: number, losses at z = 0 and z = L, collision candidates,
        real collisions."""
        out = (C.c_int64 * 5)()
        lib().orc_get_ion_counters(self.h, out)
        return dict(zip(("ions", "losses0", "losses1", "candidates", "collisions"), (int(x) for x in out)))

    def ions(self):
        n = self.ion_counters()["ions"]
        z, vx, vy, vz = (np.zeros(max(n, 1)) for _ in range(4))
        ids = np.zeros(max(n, 1), dtype=np.uint64)
        lib().orc_get_ions(self.h, _dp(z), _dp(vx), _dp(vy), _dp(vz), ids.ctypes.data_as(C.POINTER(C.c_uint64)))
        return {"z": z[:n], "vx": vx[:n], "vy": vy[:n], "vz": vz[:n], "id": ids[:n]}

    def power(self):
        """(current RF amplitude, last period's absorbed power per m^2, finished
        periods, steps per period) of the Eq. 2.9 control."""
        d = np.zeros(2)
        i = np.zeros(2, dtype=np.int64)
        lib().orc_get_power(self.h, _dp(d), i.ctypes.data_as(C.POINTER(C.c_int64)))
        return {"v_rf": d[0], "p_last": d[1], "periods": int(i[0]), "steps_per_period": int(i[1])}

    def ion_step_one(self, E, step, state4, iid):
        """One kinetic ion's push, wall test and gas collision of step `step` in
        the field E: (outcome, new state); outcome OUT_LOST0/1, or 0 (no
        candidate), 1 (null collision), 2 (collided)."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        inp = np.ascontiguousarray(state4, dtype=np.float64)
        out = np.zeros(4)
        oc = lib().orc_ion_step_one(self.h, _dp(E), int(step), _dp(inp), int(iid), _dp(out))
        return int(oc), out

    def particle_step_one(self, E, step, state4, pid):
        E = np.ascontiguousarray(E, dtype=np.float64)
        inp = np.ascontiguousarray(state4, dtype=np.float64)
        out = np.zeros(4)
        child = np.zeros(4)
        cid = C.c_uint64(0)
        oc = lib().orc_particle_step_one(self.h, _dp(E), int(step), _dp(inp), int(pid), _dp(out),
                                         _dp(child), C.byref(cid))
        return oc, out, child, int(cid.value)


# ------------------------------------------------------------- ensembles ---

def _moments_after(job):
    params, steps = job
    o = Oracle(params)
    o.step(steps)
    out = o.moments()
    out["counters"] = o.counters()
    o.close()
    return out


def run_ensemble(params_list, steps, processes=None):
    """Time-averaged moments (and counters) of each discharge after `steps`
    steps, the discharges spread over `processes` spawned processes (never
    forked: the caller may hold a GPU context)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    jobs = [(p, int(steps)) for p in params_list]
    n = max(1, min(len(jobs), processes or os.cpu_count() or 1))
    if n == 1:
        return [_moments_after(j) for j in jobs]
    with ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_moments_after, jobs))
