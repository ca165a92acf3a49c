"""The allocation-free field entry point against the regular path.

hyb_field_from_particles_noalloc is for callers that cannot allocate device
memory, for example an application that reserved all device memory up front
and hands out fixed buffers; it keeps its node sums in a fixed file-scope
device array instead.  Given the same particles,
ion density and time, its electron density, potential and field must equal
what hyb_write_particles followed by hyb_read_fields gives for a discharge
with the same parameters, to the FP64 grid tolerance of the other parity
tests.  Two calls in a row check that each call starts from cleared sums.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1508_02892_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GRID_TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _close(a, b, name):
    scale = max(np.abs(b).max(), 1e-300)
    err = np.abs(a - b).max() / scale
    assert err <= GRID_TOL, (name, err)


def test_noalloc_field_matches_regular_path_on_two_calls():
    import torch

    from paper_1508_02892_gb300 import hybrid
    lib = hybrid.lib()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    cases = [
        (W.config1(precision=W.FP64, n_particles=20000, n_cells=200, weight=3e8, v_dc_v=40.0), 11, 12000, 5),
        (W.config1(precision=W.FP64, n_particles=20000, n_cells=777, weight=1e9, v_rf_amp_v=300.0), 12, 17000, 9),
    ]
    for p, seed, n, steps in cases:
        d = hybrid.Discharge(p)
        d.advance(steps)
        step = d.counters()["step"]
        G = d.G
        ni = p["n0_m3"] * (1.0 + 0.2 * np.sin(np.linspace(0.0, 3.0, G)))
        s = W.random_particles(n, p["gap_m"], 3.0, seed=seed)
        d.set_ion_density(ni)
        d.set_particles(s["z"], s["vx"], s["vy"], s["vz"], s["id"])
        ref = d.fields()
        d.close()

        z = torch.tensor(s["z"], dtype=torch.float64, device="cuda")
        ni_d = torch.tensor(ni, dtype=torch.float64, device="cuda")
        ne = torch.empty(G, dtype=torch.float64, device="cuda")
        phi = torch.empty(G, dtype=torch.float64, device="cuda")
        E = torch.empty(G, dtype=torch.float64, device="cuda")
        P, keep = hybrid.make_params(p)
        rc = lib.hyb_field_from_particles_noalloc(C.byref(P), n, z.data_ptr(), ni_d.data_ptr(), step * p["dt_s"],
                                                  ne.data_ptr(), phi.data_ptr(), E.data_ptr(), stream.cuda_stream)
        assert rc == 0, lib.hyb_last_error()
        torch.cuda.synchronize()
        _close(ne.cpu().numpy(), ref["ne"], "ne")
        _close(phi.cpu().numpy(), ref["phi"], "phi")
        _close(E.cpu().numpy(), ref["E"], "E")


def test_noalloc_edge_positions_against_a_host_cic_sum():
    """Positions below 0, at L and NaN add no charge; a position within
    rounding below L lands on the last node; the rest follow the CIC sum."""
    import torch

    from paper_1508_02892_gb300 import hybrid
    lib = hybrid.lib()
    p = W.config1(precision=W.FP64, n_cells=97, weight=2e8)
    G, L = p["n_cells"] + 1, p["gap_m"]
    dz = L / p["n_cells"]
    s = W.random_particles(5000, L, 2.0, seed=41)
    z = np.concatenate([s["z"], [-dz, L, np.nan, np.nextafter(L, 0.0), 0.0]])
    host = np.zeros(G)
    for zi in z:
        if not (0.0 <= zi < L):
            continue
        x = zi / dz
        c = int(np.floor(x))
        o = x - c
        if c >= p["n_cells"]:
            c, o = p["n_cells"] - 1, 1.0
        host[c] += 1.0 - o
        host[c + 1] += o
    dv = np.full(G, dz)
    dv[0] = dv[-1] = dz / 2
    want = p["weight"] * host / dv
    assert host[-1] > 0.99                       # the particle just below L sits on the last node
    zt = torch.tensor(z, dtype=torch.float64, device="cuda")
    ni = torch.zeros(G, dtype=torch.float64, device="cuda")
    ne = torch.empty(G, dtype=torch.float64, device="cuda")
    phi = torch.empty(G, dtype=torch.float64, device="cuda")
    E = torch.empty(G, dtype=torch.float64, device="cuda")
    P, keep = hybrid.make_params(p)
    for _ in range(2):
        rc = lib.hyb_field_from_particles_noalloc(C.byref(P), z.size, zt.data_ptr(), ni.data_ptr(), 0.0,
                                                  ne.data_ptr(), phi.data_ptr(), E.data_ptr(), None)
        assert rc == 0, lib.hyb_last_error()
        torch.cuda.synchronize()
        _close(ne.cpu().numpy(), want, "ne")


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch

    from paper_1508_02892_gb300 import hybrid
    lib = hybrid.lib()
    p = W.config1(precision=W.FP64, n_cells=4001)
    P, keep = hybrid.make_params(p)
    buf = torch.zeros(4002, dtype=torch.float64, device="cuda")
    rc = lib.hyb_field_from_particles_noalloc(C.byref(P), 0, 0, buf.data_ptr(), 0.0, buf.data_ptr(),
                                              buf.data_ptr(), buf.data_ptr(), None)
    assert rc == -1
    assert b"4000" in lib.hyb_last_error()
