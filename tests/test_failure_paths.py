"""Failure detection on the host side and through the device status words.

CPU: the drift-diffusion stability limits of the explicit scheme (Eq. 2.5 at
level n into Eq. 2.4; u^2 dt <= 2 D and D dt / dz^2 <= 1/2) are checked when a
discharge is created, before any GPU work: the library returns
HYB_ERR_UNSTABLE and the oracle refuses the same parameters.
GPU: a finite ion density so large that the next drift flux overflows
surfaces as HYB_ERR_NONFINITE at the next synchronisation, and a discharge of a batch
that outgrows its particle capacity is reported by hyb_batch_poll with its
slot, evicted, and the other discharges finish with the results of their solo
runs.  No test faults or hangs a GPU: every failure is an ordinary value.
"""
import numpy as np
import pytest

import oracle
from paper_1508_02892_gb300 import workloads as W

UNSTABLE = {
    # drift: u = mu E = 1e-3 * 4e7 m/s, u^2 dt = 3.2e-4 > 2 D = 5.2e-5
    "dd_const_drift": dict(ion_model=W.ION_DD_CONST, v_rf_amp_v=20000.0),
    # diffusion: D dt = 2.6e-14 > dz^2 / 2 = 7.8e-15 (dz = 0.125 um, dt = 1 ns)
    "dd_const_diffusion": dict(ion_model=W.ION_DD_CONST, n_cells=4000, dt_s=1e-9, v_rf_amp_v=0.0),
    # tabulated mobility with the field-heated Eq. 2.7-2.8 diffusion at a
    # 60 MV/m drive field: u^2 dt / 2 D tends to e dt / (2 (1/4) m mu) at high
    # field, above 1 for dt = 1 ns
    "dd_table_drift": dict(ion_model=W.ION_DD_TABLE, v_rf_amp_v=30000.0, dt_s=1e-9),
}


@pytest.mark.parametrize("case", sorted(UNSTABLE))
def test_unstable_drift_diffusion_is_refused_at_create(case):
    from paper_1508_02892_gb300 import build, hybrid
    build.build()
    p = W.config1(precision=W.FP64, n_particles=100, **UNSTABLE[case])
    with pytest.raises(hybrid.HybError) as e:
        hybrid.Discharge(p)
    assert e.value.code == -7                      # HYB_ERR_UNSTABLE
    with pytest.raises(ValueError):
        oracle.Oracle(p)


def test_split_mode_cross_section_table_limit():
    """The split-mode particle step stages the cross-section table in shared
    memory: a table of more than 4096 entries is refused at create, before any
    GPU work; the FP64 mode takes it."""
    from paper_1508_02892_gb300 import build, hybrid
    build.build()
    n = 4097
    ev = np.logspace(-2, 3, n)
    p = W.config1(precision=W.FP32_SPLIT, n_particles=100, xs_ev=ev, xs_el=np.full(n, 6e-20),
                  xs_exc=np.zeros(n), xs_ion=np.zeros(n))
    with pytest.raises(hybrid.HybError) as e:
        hybrid.Discharge(p)
    assert e.value.code == -1 and "4096" in str(e.value)  # HYB_ERR_ARG


def test_stable_drift_diffusion_is_accepted_by_the_oracle():
    for case in UNSTABLE:
        p = W.config1(precision=W.FP64, n_particles=100, ion_model=UNSTABLE[case]["ion_model"])
        oracle.Oracle(p).close()


@pytest.mark.gpu
def test_overflowing_ion_density_reports_nonfinite():
    from paper_1508_02892_gb300 import build, hybrid
    build.build()
    p = W.config1(precision=W.FP64, n_particles=2000)
    g = hybrid.Discharge(p)
    assert g.sync() == 0
    # finite values: the Poisson solve still holds (E ~ 1e289 V/m), but the
    # drift flux mu n E of the next step's fluid update overflows, and the
    # field kernel's finiteness check flags the ion density it produces
    g.set_ion_density(np.full(g.G, 1e300))
    assert g.sync() == 0
    with pytest.raises(hybrid.HybError) as e:
        g.advance(1)
        g.sync()
    assert e.value.code == -4                      # HYB_ERR_NONFINITE
    with pytest.raises(hybrid.HybError) as e:      # the status stays: later reads report it too
        g.counters()
    assert e.value.code == -4
    g.close()
    # a fresh discharge on the same GPU is unaffected
    h = hybrid.Discharge(p)
    h.advance(5)
    assert h.sync() == 0
    h.close()


@pytest.mark.gpu
def test_failed_slot_is_reported_evicted_and_others_finish():
    from paper_1508_02892_gb300 import build, hybrid
    build.build()
    good = [W.config1(precision=W.FP64, n_particles=3000, seed=61),
            W.config1(precision=W.FP64, n_particles=2500, n_cells=120, ion_model=W.ION_FULL, seed=62)]
    # hot electrons and no room for their children: the capacity overflows
    bad = W.config1(precision=W.FP64, n_particles=4000, capacity_factor=1.0, te0_ev=60.0, n_cells=50, seed=63)
    steps = 60
    solo = []
    for p in good:
        g = hybrid.Discharge(p)
        g.advance(steps)
        solo.append((g.particles(), g.counters()))
        g.close()
    b = hybrid.Batch(4, hybrid.HYB_FP64)
    s_good = [b.admit(p, steps) for p in good]
    s_bad = b.admit(bad, 400)
    failed = []
    for _ in range(4):
        b.advance(100)
        done, rc = b.poll_status()
        if s_bad in done:
            assert rc == -3                        # HYB_ERR_CAPACITY
            with pytest.raises(hybrid.HybError) as e:  # reads of the failed slot report it too
                b.counters(s_bad)
            assert e.value.code == -3
            b.evict(s_bad)
            failed.append(s_bad)
        if failed:
            break
    assert failed == [s_bad]
    b.advance(100)
    for s, (parts, ctr) in zip(s_good, solo):
        c = b.counters(s)
        assert c["status"] == 0 and c["step"] == steps
        for k in ("particles", "births_iz", "losses0", "losses1", "elastic", "excitation", "ionization", "null"):
            assert c[k] == ctr[k], k
        q = b.particles(s)
        assert np.array_equal(q["id"], parts["id"])
        np.testing.assert_allclose(q["z"], parts["z"], rtol=0, atol=1e-15 * good[0]["gap_m"])
        np.testing.assert_allclose(q["vz"], parts["vz"], rtol=1e-13, atol=1e-6)
    b.close()


@pytest.mark.gpu
def test_bounded_wait_reports_timeout_and_the_work_goes_on():
    """hyb_batch_wait returns HYB_ERR_TIMEOUT when the queued work outlasts its
    limit (a host-side poll of the stream: nothing on the GPU waits), and the
    work completes when waited for again."""
    from paper_1508_02892_gb300 import build, hybrid
    build.build()
    b = hybrid.Batch(2, hybrid.HYB_FP32_SPLIT)
    s = b.admit(W.config2(n_particles=2_000_000), 1000)
    assert b.wait(60.0)
    b.advance(1000)                                # about 50 ms of queued work
    assert b.wait(1e-4) is False
    assert b.wait(120.0) is True
    c = b.counters(s)
    assert c["step"] == 1000 and c["status"] == 0
    b.close()
