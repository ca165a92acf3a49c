"""Continuous batching on the GPU: runs of different sizes arrive while others
are on the device, share lockstep launches with them, and end at their own
step counts.  Each result must be the one the same run gives alone: in FP64
the particle states to 1e-12 and the moments to 1e-11 (the tolerances of the
other FP64 parity tests; only summation order differs), in the FP32 split
mode the time-averaged profiles and the EEDF to 2 % (L2).
"""
import numpy as np
import pytest

from paper_1508_02892_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _fp64_requests():
    base = dict(precision=W.FP64)
    spec = [  # arrival (s of chunk time), params, steps
        (0.00, dict(n_particles=4000, n_cells=80, seed=41, te0_ev=6.0, ion_model=W.ION_DD_TABLE), 150),
        (0.02, dict(n_particles=12000, n_cells=150, seed=42, ion_model=W.ION_FULL, gamma_see=0.2, weight=2e6,
                    v_rf_amp_v=300.0), 250),
        (0.06, dict(n_particles=2500, n_cells=60, seed=43), 120),
        (0.11, dict(n_particles=8000, n_cells=200, seed=44, ion_model=W.ION_FULL, te0_ev=8.0), 300),
        (0.12, dict(n_particles=700, n_cells=33, seed=45, ion_model=W.ION_DD_TABLE), 100),
        (0.40, dict(n_particles=5000, n_cells=120, seed=46, te0_ev=4.0), 200),
    ]
    return [{"arrival_s": a, "steps": n, "tag": k, "params": W.config1(**base, **kw)}
            for k, (a, kw, n) in enumerate(spec)]


def _serve(reqs, precision, max_slots, keep):
    from paper_1508_02892_gb300 import hybrid
    from paper_1508_02892_gb300.serve import ChunkClock, Server
    clk = ChunkClock(0.05)
    caps = sorted(hybrid.footprint(r["params"]) for r in reqs)
    cap = caps[-1] + caps[-2] + caps[0]          # not all of them fit at once
    srv = Server(max_slots=max_slots, hbm_cap_bytes=cap, precision=precision, clock=clk)
    clk.server = srv
    out = srv.run(reqs, keep=keep)
    srv.close()
    assert srv.max_bytes <= cap
    return out


def test_fp64_results_same_alone_and_in_the_mix():
    from paper_1508_02892_gb300 import hybrid
    reqs = _fp64_requests()
    out = _serve(reqs, hybrid.HYB_FP64, 3, ("counters", "moments", "particles"))
    # the mix really overlapped: some run was admitted while another was running
    spans = sorted((r["admitted_s"], r["done_s"]) for r in out)
    assert any(spans[k + 1][0] < spans[k][1] for k in range(len(spans) - 1))
    for r, q in zip(out, reqs):
        assert r["status"] == 0
        g = hybrid.Discharge(q["params"])
        g.advance(q["steps"])
        a, b = r["particles"], g.particles()
        assert r["counters"]["step"] == q["steps"]
        assert np.array_equal(a["id"], b["id"])
        L = q["params"]["gap_m"]
        assert np.max(np.abs(a["z"] - b["z"]), initial=0.0) <= 1e-12 * L
        va = np.stack([a["vx"], a["vy"], a["vz"]])
        vb = np.stack([b["vx"], b["vy"], b["vz"]])
        if vb.size:
            sp = np.maximum(np.linalg.norm(vb, axis=0), 1e-3 * np.abs(vb).max())
            assert (np.linalg.norm(va - vb, axis=0) / sp).max() <= 1e-12
        cb = g.counters()
        for k in ("step", "particles", "births_iz", "losses0", "losses1", "elastic", "excitation", "ionization",
                  "null", "pushes"):
            assert r["counters"][k] == cb[k], (r["tag"], k)
        mb = g.moments()
        for k in ("ne", "ni", "gamma", "ebar", "eedf"):
            scale = max(np.abs(mb[k]).max(), 1e-300)
            assert np.abs(r["moments"][k] - mb[k]).max() / scale <= 1e-11, (r["tag"], k)
        g.close()


def test_split_results_same_alone_and_in_the_mix():
    from paper_1508_02892_gb300 import hybrid
    reqs = []
    for k, (a, n, c, steps) in enumerate([(0.0, 20000, 200, 400), (0.03, 6000, 100, 300), (0.08, 30000, 300, 500),
                                          (0.1, 3000, 70, 200)]):
        reqs.append({"arrival_s": a, "steps": steps, "tag": k,
                     "params": W.config1(precision=W.FP32_SPLIT, n_particles=n, n_cells=c, seed=60 + k)})
    out = _serve(reqs, hybrid.HYB_FP32_SPLIT, 2, ("counters", "moments"))
    for r, q in zip(out, reqs):
        assert r["status"] == 0 and r["counters"]["step"] == q["steps"]
        g = hybrid.Discharge(q["params"])
        g.advance(q["steps"])
        mb = g.moments()
        for k in ("ne", "ebar", "gamma", "eedf"):
            err = np.linalg.norm(r["moments"][k] - mb[k]) / np.linalg.norm(mb[k])
            assert err < 0.02, (r["tag"], k, err)
        g.close()


def test_moments_snapshot_reads_while_the_next_chunk_runs():
    """hyb_batch_snapshot_moments copies every slot's time sums in stream
    order: read after the next chunk was queued, a snapshot gives exactly the
    moments a synchronous read gave at the same point, and the next snapshot
    the later ones; an empty slot and a batch without a snapshot are refused."""
    from paper_1508_02892_gb300 import hybrid
    b = hybrid.Batch(4, hybrid.HYB_FP32_SPLIT)
    ps = [W.config1(precision=W.FP32_SPLIT, n_particles=n, n_cells=c, seed=s)
          for n, c, s in ((20000, 200, 61), (9000, 97, 62), (15000, 333, 63))]
    slots = [b.admit(p) for p in ps]
    with pytest.raises(hybrid.HybError):
        b.snapshot_read_moments(slots[0])
    b.advance(100)
    direct = [b.moments(s) for s in slots]
    b.snapshot_moments()
    b.advance(100)                       # queued behind the snapshot
    for s, d in zip(slots, direct):
        m = b.snapshot_read_moments(s)
        assert m["n_samples"] == d["n_samples"]
        for k in ("ne", "ni", "gamma", "ebar", "eedf"):
            assert np.array_equal(m[k], d[k]), k
    b.snapshot_moments()
    for s in slots:
        m, d = b.snapshot_read_moments(s), b.moments(s)
        assert m["n_samples"] == d["n_samples"] == 200
        for k in ("ne", "ni", "gamma", "ebar", "eedf"):
            assert np.array_equal(m[k], d[k]), k
    free = [k for k in range(4) if k not in slots][0]
    rc = hybrid.lib().hyb_batch_read_snapshot_moments(b.h, free, hybrid.Moments())
    assert rc == -8, rc  # HYB_ERR_STATE
    # the same grid re-admitted into a slot after the snapshot: refused too
    b.evict(slots[0])
    again = b.admit(ps[0])
    rc = hybrid.lib().hyb_batch_read_snapshot_moments(b.h, again, hybrid.Moments())
    assert rc == -8, rc
    b.close()
