"""ctypes binding of libhybrid1d.so (include/hybrid1d.h).

Argument marshalling only: every step of the method runs in the CUDA library.
The library must have been built (``paper_1508_02892_gb300.build.build()``);
loading fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhybrid1d.so")

HYB_OK, HYB_WARN_DT_NULLCOLL = 0, 1
ERRORS = {-1: "HYB_ERR_ARG", -2: "HYB_ERR_OOM", -3: "HYB_ERR_CAPACITY", -4: "HYB_ERR_NONFINITE",
          -5: "HYB_ERR_TIMEOUT", -6: "HYB_ERR_CUDA", -7: "HYB_ERR_UNSTABLE", -8: "HYB_ERR_STATE"}
HYB_FP64, HYB_FP32_SPLIT = 0, 1
STATUS_CAPACITY, STATUS_NONFINITE, STATUS_UNSTABLE, STATUS_EMIT_CAP = 1, 2, 4, 8

_pd = C.POINTER(C.c_double)


class HybError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [
        ("gap_m", C.c_double), ("n_cells", C.c_int32), ("gas", C.c_int32),
        ("pressure_pa", C.c_double), ("gas_temp_k", C.c_double),
        ("v_rf_amp_v", C.c_double), ("f_rf_hz", C.c_double), ("v_dc_v", C.c_double),
        ("dt_s", C.c_double), ("n_particles", C.c_int64), ("n0_m3", C.c_double),
        ("te0_ev", C.c_double), ("weight", C.c_double), ("gamma_see", C.c_double),
        ("see_energy_ev", C.c_double), ("ion_model", C.c_int32), ("ion_mass_amu", C.c_double),
        ("gas_mass_amu", C.c_double), ("mu_const", C.c_double),
        ("tab_eon_td", _pd), ("tab_mu", _pd), ("tab_nu", _pd), ("n_tab", C.c_int32),
        ("xs_ev", _pd), ("xs_el", _pd), ("xs_exc", _pd), ("xs_ion", _pd), ("n_xs", C.c_int32),
        ("e_exc_ev", C.c_double), ("e_iz_ev", C.c_double), ("seed", C.c_uint64),
        ("eedf_bins", C.c_int32), ("eedf_max_ev", C.c_double), ("precision", C.c_int32),
        ("capacity_factor", C.c_double), ("sort_interval", C.c_int32), ("power_w_m2", C.c_double),
        ("power_alpha", C.c_double), ("xs_rec", _pd), ("metastables", C.c_int32), ("met_diff_m2s", C.c_double),
        ("met_n0_m3", C.c_double), ("penning_rate_m3s", C.c_double), ("penning_target_m3", C.c_double),
        ("penning_energy_ev", C.c_double), ("pooling_rate_m3s", C.c_double), ("pooling_energy_ev", C.c_double),
        ("gamma_met", C.c_double),
    ]


class Moments(C.Structure):
    _fields_ = [("ne", _pd), ("ni", _pd), ("gamma_i", _pd), ("mean_energy_ev", _pd), ("eedf", _pd),
                ("n_samples", C.c_int64)]


class Fields(C.Structure):
    _fields_ = [("ne", _pd), ("ni", _pd), ("gamma_i", _pd), ("phi", _pd), ("efield", _pd), ("ion_source", _pd)]


class Counters(C.Structure):
    _fields_ = [("step", C.c_int64), ("particles", C.c_int64), ("births_ionization", C.c_int64),
                ("births_see", C.c_int64 * 2), ("losses", C.c_int64 * 2), ("collisions", C.c_int64 * 4),
                ("clamps", C.c_int64), ("pushes", C.c_int64), ("status", C.c_uint32), ("v_rf_amp_v", C.c_double),
                ("power_last_w_m2", C.c_double), ("power_periods", C.c_int64), ("recombinations", C.c_int64),
                ("ions", C.c_int64), ("ion_losses", C.c_int64 * 2), ("ion_collisions", C.c_int64),
                ("births_penning", C.c_int64), ("births_pooling", C.c_int64), ("ion_pushes", C.c_int64)]


class Info(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("eedf_bins", C.c_int32), ("weight", C.c_double),
                ("gas_density", C.c_double), ("nu_max", C.c_double), ("p_max", C.c_double), ("dz", C.c_double),
                ("capacity", C.c_int64), ("device_bytes", C.c_int64)]


class Profile(C.Structure):
    _fields_ = [("kernel_launches", C.c_int64), ("steps", C.c_int64), ("ms_electron", C.c_double),
                ("ms_field", C.c_double), ("ms_sort", C.c_double), ("n_electron", C.c_int64),
                ("n_field", C.c_int64), ("n_sort", C.c_int64), ("ms_ion", C.c_double), ("n_ion", C.c_int64)]


_lib = None

class SwarmParams(C.Structure):
    _fields_ = [("gas_mass_amu", C.c_double), ("ion_mass_amu", C.c_double), ("pressure_pa", C.c_double),
                ("gas_temp_k", C.c_double), ("ion_temp0_k", C.c_double), ("dt_s", C.c_double),
                ("nu_max", C.c_double), ("eps_max_ev", C.c_double), ("n_ions", C.c_int64), ("n_steps", C.c_int64),
                ("n_relax", C.c_int64), ("xs_model", C.c_int32), ("precision", C.c_int32), ("seed", C.c_uint64)]


class SwarmResult(C.Structure):
    _fields_ = [("e_field", C.c_double), ("drift", C.c_double), ("mean_energy_ev", C.c_double),
                ("mobility", C.c_double), ("nu_exchange", C.c_double), ("nu_max", C.c_double),
                ("p_max", C.c_double), ("candidates", C.c_int64), ("collisions", C.c_int64),
                ("overruns", C.c_int64)]


class Tuning(C.Structure):
    _fields_ = [("lanes", C.c_int32), ("sort_interval", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("field_threads", C.c_int32), ("field_cluster", C.c_int32), ("electron_threads", C.c_int32),
                ("particles_per_thread", C.c_int32), ("rate", C.c_double)]


EXPORTS = {
    "hyb_create_discharge": (C.c_int, [C.POINTER(Params), C.c_void_p, C.POINTER(C.c_void_p)]),
    "hyb_advance": (C.c_int, [C.c_void_p, C.c_int64]),
    "hyb_sync": (C.c_int, [C.c_void_p]),
    "hyb_read_moments": (C.c_int, [C.c_void_p, C.POINTER(Moments)]),
    "hyb_read_fields": (C.c_int, [C.c_void_p, C.POINTER(Fields)]),
    "hyb_read_counters": (C.c_int, [C.c_void_p, C.POINTER(Counters)]),
    "hyb_get_info": (C.c_int, [C.c_void_p, C.POINTER(Info)]),
    "hyb_reset_moments": (C.c_int, [C.c_void_p]),
    "hyb_read_particles": (C.c_int, [C.c_void_p, _pd, _pd, _pd, _pd, C.POINTER(C.c_uint64), C.c_int64,
                                     C.POINTER(C.c_int64)]),
    "hyb_write_particles": (C.c_int, [C.c_void_p, C.c_int64, _pd, _pd, _pd, _pd, C.POINTER(C.c_uint64)]),
    "hyb_write_ion_density": (C.c_int, [C.c_void_p, _pd]),
    "hyb_read_metastables": (C.c_int, [C.c_void_p, _pd, _pd, _pd]),
    "hyb_write_metastables": (C.c_int, [C.c_void_p, _pd]),
    "hyb_batch_read_metastables": (C.c_int, [C.c_void_p, C.c_int32, _pd, _pd, _pd]),
    "hyb_read_ions": (C.c_int, [C.c_void_p, _pd, _pd, _pd, _pd, C.POINTER(C.c_uint64), C.c_int64,
                                C.POINTER(C.c_int64)]),
    "hyb_batch_read_ions": (C.c_int, [C.c_void_p, C.c_int32, _pd, _pd, _pd, _pd, C.POINTER(C.c_uint64), C.c_int64,
                                      C.POINTER(C.c_int64)]),
    "hyb_destroy": (C.c_int, [C.c_void_p]),
    "hyb_batch_create": (C.c_int, [C.c_int32, C.c_int32, C.c_int64, C.c_void_p, C.POINTER(C.c_void_p)]),
    "hyb_footprint": (C.c_int, [C.POINTER(Params), C.POINTER(C.c_int64)]),
    "hyb_batch_admit": (C.c_int, [C.c_void_p, C.POINTER(Params), C.c_int64, C.POINTER(C.c_int32)]),
    "hyb_batch_advance": (C.c_int, [C.c_void_p, C.c_int64]),
    "hyb_batch_poll": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_int32)]),
    "hyb_batch_snapshot": (C.c_int, [C.c_void_p]),
    "hyb_batch_wait": (C.c_int, [C.c_void_p, C.c_double]),
    "hyb_batch_poll_snapshot": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_int32)]),
    "hyb_batch_read_finished": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "hyb_batch_read_moments": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Moments)]),
    "hyb_batch_read_counters": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Counters)]),
    "hyb_batch_read_particles": (C.c_int, [C.c_void_p, C.c_int32, _pd, _pd, _pd, _pd, C.POINTER(C.c_uint64),
                                           C.c_int64, C.POINTER(C.c_int64)]),
    "hyb_batch_evict": (C.c_int, [C.c_void_p, C.c_int32]),
    "hyb_batch_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "hyb_batch_destroy": (C.c_int, [C.c_void_p]),
    "hyb_batch_set_profiling": (C.c_int, [C.c_void_p, C.c_int32]),
    "hyb_batch_profile": (C.c_int, [C.c_void_p, C.POINTER(Profile), C.c_int32]),
    "hyb_batch_get_tuning": (C.c_int, [C.c_void_p, C.POINTER(Tuning)]),
    "hyb_batch_set_tuning": (C.c_int, [C.c_void_p, C.POINTER(Tuning)]),
    "hyb_batch_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Tuning)]),
    "hyb_discharge_batch": (C.c_void_p, [C.c_void_p]),
    "hyb_batch_set_field_arith": (C.c_int, [C.c_void_p, C.c_int32]),
    "hyb_batch_snapshot_moments": (C.c_int, [C.c_void_p]),
    "hyb_batch_read_snapshot_moments": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Moments)]),
    "hyb_swarm_run": (C.c_int, [C.POINTER(SwarmParams), C.c_int32, _pd, C.POINTER(SwarmResult), C.c_void_p,
                                C.c_void_p]),
    "hyb_swarm_tables": (C.c_int, [C.POINTER(SwarmParams), C.c_int32, _pd, _pd, _pd, C.c_void_p]),
    "hyb_debug_checks": (C.c_int, [C.POINTER(C.c_uint64)]),
    "hyb_field_from_particles_noalloc": (C.c_int, [C.POINTER(Params), C.c_int64, C.c_void_p, C.c_void_p,
                                                   C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hyb_last_error": (C.c_char_p, []),
}


def debug_checks():
    """First failed device index guard: (site, index, bound) for the particle
    kernels and for the field kernel; zeros when none failed."""
    out = (C.c_uint64 * 6)()
    _check(lib().hyb_debug_checks(out))
    return tuple(out[:3]), tuple(out[3:])


def _profile(bh, reset):
    p = Profile()
    _check(lib().hyb_batch_profile(bh, C.byref(p), int(reset)))
    return {f: getattr(p, f) for f, _ in Profile._fields_}


def lib():
    """Load libhybrid1d.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} missing (run paper_1508_02892_gb300.build)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc, allow_warn=True):
    if rc < 0 or (rc > 0 and not allow_warn):
        raise HybError(rc, lib().hyb_last_error().decode())
    return rc


def _arr(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def make_params(d: dict):
    """hyb_params from a workload dict; returns (struct, arrays kept alive)."""
    keep = {}
    p = Params()
    for name, ctype in Params._fields_:
        if name in ("tab_eon_td", "tab_mu", "tab_nu", "xs_ev", "xs_el", "xs_exc", "xs_ion", "xs_rec"):
            if name in d and d[name] is not None:
                a = _arr(d[name])
                keep[name] = a
                setattr(p, name, a.ctypes.data_as(_pd))
        elif name in ("n_tab", "n_xs"):
            continue
        elif name in d:
            setattr(p, name, d[name])
    p.n_tab = keep["tab_eon_td"].size if "tab_eon_td" in keep else 0
    p.n_xs = keep["xs_ev"].size if "xs_ev" in keep else 0
    return p, keep


def _default_stream(stream):
    if stream is not None:
        return int(stream)
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return None


def _moments(call, G, nb):
    out = {k: np.zeros(G) for k in ("ne", "ni", "gamma", "ebar")}
    out["eedf"] = np.zeros(nb + 1)
    m = Moments(out["ne"].ctypes.data_as(_pd), out["ni"].ctypes.data_as(_pd), out["gamma"].ctypes.data_as(_pd),
                out["ebar"].ctypes.data_as(_pd), out["eedf"].ctypes.data_as(_pd), 0)
    _check(call(C.byref(m)))
    out["n_samples"] = int(m.n_samples)
    return out


def _counters(call):
    c = Counters()
    _check(call(C.byref(c)))
    return _counters_dict(c)


def _counters_dict(c):
    return {"step": c.step, "particles": c.particles, "births_iz": c.births_ionization,
            "births_see0": c.births_see[0], "births_see1": c.births_see[1], "losses0": c.losses[0],
            "losses1": c.losses[1], "elastic": c.collisions[0], "excitation": c.collisions[1],
            "ionization": c.collisions[2], "null": c.collisions[3], "clamps": c.clamps, "pushes": c.pushes,
            "status": c.status, "v_rf": c.v_rf_amp_v, "power_last": c.power_last_w_m2,
            "power_periods": c.power_periods, "recombinations": c.recombinations, "ions": c.ions,
            "ion_losses0": c.ion_losses[0], "ion_losses1": c.ion_losses[1], "ion_collisions": c.ion_collisions,
            "births_penning": c.births_penning, "births_pooling": c.births_pooling, "ion_pushes": c.ion_pushes}


def _particles(call, cap):
    n = C.c_int64(0)
    z, vx, vy, vz = (np.zeros(cap) for _ in range(4))
    ids = np.zeros(cap, dtype=np.uint64)
    _check(call(z.ctypes.data_as(_pd), vx.ctypes.data_as(_pd), vy.ctypes.data_as(_pd), vz.ctypes.data_as(_pd),
                ids.ctypes.data_as(C.POINTER(C.c_uint64)), cap, C.byref(n)))
    k = n.value
    return {"z": z[:k], "vx": vx[:k], "vy": vy[:k], "vz": vz[:k], "id": ids[:k]}


class Discharge:
    """One discharge advanced on the GPU (hyb_create_discharge ... hyb_destroy)."""

    def __init__(self, params: dict, stream=None):
        self._p, self._keep = make_params(params)
        h = C.c_void_p()
        self.warning = _check(lib().hyb_create_discharge(C.byref(self._p), _default_stream(stream), C.byref(h)))
        self.h = h
        info = Info()
        _check(lib().hyb_get_info(self.h, C.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in Info._fields_}
        self.G = info.n_nodes
        self.eedf_bins = info.eedf_bins

    def close(self):
        if getattr(self, "h", None):
            lib().hyb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def advance(self, n):
        _check(lib().hyb_advance(self.h, int(n)))

    def sync(self):
        return _check(lib().hyb_sync(self.h))

    def moments(self):
        return _moments(lambda m: lib().hyb_read_moments(self.h, m), self.G, self.eedf_bins)

    def fields(self):
        out = {k: np.zeros(self.G) for k in ("ne", "ni", "gamma", "phi", "E", "gsrc")}
        f = Fields(*(out[k].ctypes.data_as(_pd) for k in ("ne", "ni", "gamma", "phi", "E", "gsrc")))
        _check(lib().hyb_read_fields(self.h, C.byref(f)))
        return out

    def counters(self):
        return _counters(lambda c: lib().hyb_read_counters(self.h, c))

    def reset_moments(self):
        _check(lib().hyb_reset_moments(self.h))

    def set_tuning(self, **kw):
        """Launch layout of the batch behind this discharge (fields of
        hyb_tuning: lanes, sort_interval, blocks_per_sm, field_threads,
        field_cluster, electron_threads, particles_per_thread)."""
        bh = lib().hyb_discharge_batch(self.h)
        t = Tuning()
        _check(lib().hyb_batch_get_tuning(bh, C.byref(t)))
        for k, v in kw.items():
            setattr(t, k, int(v))
        _check(lib().hyb_batch_set_tuning(bh, C.byref(t)))

    def set_field_arith(self, split):
        """Test hook: the field step takes the split mode's arithmetic (1) or
        the batch's own (0)."""
        _check(lib().hyb_batch_set_field_arith(lib().hyb_discharge_batch(self.h), int(split)))

    def particles(self, cap=None):
        cap = int(cap or self.info["capacity"])
        return _particles(lambda *a: lib().hyb_read_particles(self.h, *a), cap)

    def ions(self, cap=None):
        """Kinetic ions (sorted by id)."""
        cap = int(cap or self.info["capacity"])
        return _particles(lambda *a: lib().hyb_read_ions(self.h, *a), cap)

    def set_particles(self, z, vx, vy, vz, ids):
        z, vx, vy, vz = (_arr(a) for a in (z, vx, vy, vz))
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        _check(lib().hyb_write_particles(self.h, z.size, z.ctypes.data_as(_pd), vx.ctypes.data_as(_pd),
                                         vy.ctypes.data_as(_pd), vz.ctypes.data_as(_pd),
                                         ids.ctypes.data_as(C.POINTER(C.c_uint64))))

    def set_profiling(self, on=True):
        _check(lib().hyb_batch_set_profiling(lib().hyb_discharge_batch(self.h), int(bool(on))))

    def profile(self, reset=False):
        return _profile(lib().hyb_discharge_batch(self.h), reset)

    def set_ion_density(self, ni):
        ni = _arr(ni)
        _check(lib().hyb_write_ion_density(self.h, ni.ctypes.data_as(_pd)))

    def metastables(self):
        """Metastable density, its time average, and the flux into each wall in
        the last step."""
        return _metastables(lambda *a: lib().hyb_read_metastables(self.h, *a), self.info["n_nodes"])

    def set_metastables(self, met):
        met = _arr(met)
        _check(lib().hyb_write_metastables(self.h, met.ctypes.data_as(_pd)))


def _metastables(call, G):
    met, avg, flux = np.zeros(G), np.zeros(G), np.zeros(2)
    _check(call(met.ctypes.data_as(_pd), avg.ctypes.data_as(_pd), flux.ctypes.data_as(_pd)))
    return {"met": met, "avg": avg, "flux": flux}


def footprint(params: dict) -> int:
    p, keep = make_params(params)
    b = C.c_int64(0)
    _check(lib().hyb_footprint(C.byref(p), C.byref(b)))
    return int(b.value)


class Batch:
    """Many discharges of one precision advanced in lockstep launches
    (hyb_batch_*): admission under an HBM cap, completion polling, eviction."""

    def __init__(self, max_instances, precision=HYB_FP32_SPLIT, hbm_cap_bytes=0, stream=None):
        h = C.c_void_p()
        _check(lib().hyb_batch_create(int(max_instances), int(precision), int(hbm_cap_bytes),
                                      _default_stream(stream), C.byref(h)))
        self.h = h
        self.max_instances = int(max_instances)
        self._shape = {}

    def close(self):
        if getattr(self, "h", None):
            lib().hyb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def admit(self, params: dict, n_steps: int = 0):
        p, keep = make_params(params)
        slot = C.c_int32(-1)
        rc = lib().hyb_batch_admit(self.h, C.byref(p), int(n_steps), C.byref(slot))
        _check(rc)
        bins = int(params.get("eedf_bins", 0) or 256)
        cap = max(4096, int(np.ceil((params.get("capacity_factor") or 2.0) * params["n_particles"])))
        self._shape[slot.value] = (int(params["n_cells"]) + 1, bins, cap)
        return slot.value

    def advance(self, n):
        _check(lib().hyb_batch_advance(self.h, int(n)))

    def poll(self):
        done, rc = self.poll_status()
        _check(rc)
        return done

    def wait(self, timeout_s):
        """Wait at most timeout_s for the queued work: True when done, False
        when the limit passed first (HYB_ERR_TIMEOUT)."""
        rc = lib().hyb_batch_wait(self.h, float(timeout_s))
        if rc == -5:
            return False
        _check(rc)
        return True

    def snapshot(self):
        """Queue a status snapshot after the work queued so far."""
        _check(lib().hyb_batch_snapshot(self.h))

    def poll_snapshot(self):
        """(slots finished or failed as of the oldest queued snapshot, return
        code); waits for that snapshot only."""
        done = (C.c_int32 * self.max_instances)()
        n = C.c_int32(0)
        rc = lib().hyb_batch_poll_snapshot(self.h, done, self.max_instances, C.byref(n))
        if rc < 0 and rc not in (-3, -4, -7):   # a slot's own failure is reported with it
            _check(rc)
        return [done[i] for i in range(n.value)], int(rc)

    def read_finished(self, slot, moments=True):
        """Counters (from the snapshot) and, if asked, moments (side stream)
        of a slot that poll_snapshot reported: (counters, moments or None,
        return code)."""
        G, nb = self._shape[slot][0], self._shape[slot][1]
        c = Counters()
        m = None
        mc = None
        if moments:
            m = {k: np.zeros(G) for k in ("ne", "ni", "gamma", "ebar")}
            m["eedf"] = np.zeros(nb + 1)
            mc = Moments(m["ne"].ctypes.data_as(_pd), m["ni"].ctypes.data_as(_pd), m["gamma"].ctypes.data_as(_pd),
                         m["ebar"].ctypes.data_as(_pd), m["eedf"].ctypes.data_as(_pd), 0)
        rc = lib().hyb_batch_read_finished(self.h, int(slot), C.byref(c), C.byref(mc) if mc is not None else None)
        if rc < 0 and rc not in (-3, -4, -7):
            _check(rc)
        if m is not None:
            m["n_samples"] = int(mc.n_samples)
        return _counters_dict(c), m, int(rc)

    def poll_status(self):
        """(slots finished or failed since the last poll, return code): a
        failed slot is listed with the others and its error is the code."""
        done = (C.c_int32 * self.max_instances)()
        n = C.c_int32(0)
        rc = lib().hyb_batch_poll(self.h, done, self.max_instances, C.byref(n))
        return [done[i] for i in range(n.value)], int(rc)

    def moments(self, slot):
        G, nb, _ = self._shape[slot]
        return _moments(lambda m: lib().hyb_batch_read_moments(self.h, int(slot), m), G, nb)

    def snapshot_moments(self):
        """Queue a copy of every taken slot's time sums after the work queued
        so far (no host wait)."""
        _check(lib().hyb_batch_snapshot_moments(self.h))

    def snapshot_read_moments(self, slot):
        """Moments of `slot` as of the snapshot queued last (waits for that
        snapshot's copy only)."""
        G, nb, _ = self._shape[slot]
        return _moments(lambda m: lib().hyb_batch_read_snapshot_moments(self.h, int(slot), m), G, nb)

    def counters(self, slot):
        return _counters(lambda c: lib().hyb_batch_read_counters(self.h, int(slot), c))

    def particles(self, slot, cap=None):
        cap = int(cap or self._shape[slot][2])
        return _particles(lambda *a: lib().hyb_batch_read_particles(self.h, int(slot), *a), cap)

    def metastables(self, slot):
        return _metastables(lambda *a: lib().hyb_batch_read_metastables(self.h, int(slot), *a), self._shape[slot][0])

    def ions(self, slot, cap=None):
        cap = int(cap or self._shape[slot][2])
        return _particles(lambda *a: lib().hyb_batch_read_ions(self.h, int(slot), *a), cap)

    def evict(self, slot):
        _check(lib().hyb_batch_evict(self.h, int(slot)))
        self._shape.pop(slot, None)

    def set_profiling(self, on=True):
        _check(lib().hyb_batch_set_profiling(self.h, int(bool(on))))

    def profile(self, reset=False):
        return _profile(self.h, reset)

    def tuning(self):
        t = Tuning()
        _check(lib().hyb_batch_get_tuning(self.h, C.byref(t)))
        return {f: getattr(t, f) for f, _ in Tuning._fields_}

    def set_tuning(self, lanes=None, sort_interval=None, blocks_per_sm=None, field_threads=None,
                   field_cluster=None, electron_threads=None, particles_per_thread=None):
        cur = self.tuning()
        t = Tuning(int(lanes if lanes is not None else cur["lanes"]),
                   int(sort_interval if sort_interval is not None else cur["sort_interval"]),
                   int(blocks_per_sm if blocks_per_sm is not None else cur["blocks_per_sm"]),
                   int(field_threads if field_threads is not None else cur["field_threads"]),
                   int(field_cluster if field_cluster is not None else cur["field_cluster"]),
                   int(electron_threads if electron_threads is not None else cur["electron_threads"]),
                   int(particles_per_thread if particles_per_thread is not None else cur["particles_per_thread"]),
                   0.0)
        _check(lib().hyb_batch_set_tuning(self.h, C.byref(t)))
        return self.tuning()

    def autotune(self, trial_steps=200):
        t = Tuning()
        _check(lib().hyb_batch_autotune(self.h, int(trial_steps), C.byref(t)))
        return {f: getattr(t, f) for f, _ in Tuning._fields_}

    def stats(self):
        r, n, b = C.c_int32(0), C.c_int64(0), C.c_int64(0)
        _check(lib().hyb_batch_stats(self.h, C.byref(r), C.byref(n), C.byref(b)))
        return {"running": r.value, "particles": n.value, "bytes": b.value}


def _swarm_struct(params: dict):
    p = SwarmParams()
    for name, _ in SwarmParams._fields_:
        if name in params:
            setattr(p, name, params[name])
    return p


def swarm_run(params: dict, fields, velocities=None, stream=None):
    """hyb_swarm_run at the given field values (V/m).  velocities: None, or a
    device buffer (an object with data_ptr(), 3 * n_ions * len(fields)
    doubles) that receives the final ion velocities.  Returns one dict per
    field and the return code (HYB_WARN_NU_MAX when the bound was exceeded)."""
    p = _swarm_struct(params)
    f = _arr(fields)
    out = (SwarmResult * f.size)()
    rc = _check(lib().hyb_swarm_run(C.byref(p), f.size, f.ctypes.data_as(_pd), out,
                                    velocities.data_ptr() if velocities is not None else None,
                                    _default_stream(stream)))
    return [{k: getattr(r, k) for k, _ in SwarmResult._fields_} for r in out], rc


def swarm_tables(params: dict, eon_td, stream=None):
    """hyb_swarm_tables: mobility and exchange-frequency tables over E/N (Td)."""
    p = _swarm_struct(params)
    x = _arr(eon_td)
    mu, nu = np.zeros(x.size), np.zeros(x.size)
    rc = _check(lib().hyb_swarm_tables(C.byref(p), x.size, x.ctypes.data_as(_pd), mu.ctypes.data_as(_pd),
                                       nu.ctypes.data_as(_pd), _default_stream(stream)))
    return mu, nu, rc

