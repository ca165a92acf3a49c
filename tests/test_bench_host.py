"""Host logic of the benchmark's CPU arms: the oracle spread over host cores
(one spawned process per core, discharges dealt largest first) steps every
discharge once per pool step, so its particle-step counts equal those of the
same oracles stepped one after the other."""
import numpy as np

import oracle
from paper_1508_02892_gb300 import workloads as W


def test_oracle_pool_counts_equal_sequential_runs():
    import bench
    params = [W.config1(n_particles=n, n_cells=c, seed=s, te0_ev=8.0)
              for n, c, s in ((3000, 40, 1), (1200, 30, 2), (5000, 50, 3))]
    pool = bench.OraclePool(params, 2)
    assert pool.cores == 2
    got = [pool.step()[0] for _ in range(3)]
    pool.close()
    sims = [oracle.Oracle(p) for p in params]
    want = []
    for _ in range(3):
        want.append(sum(o.n_particles for o in sims))
        for o in sims:
            o.step(1)
    assert got == want


def test_oracle_pool_deals_largest_first():
    import bench
    params = [W.config1(n_particles=n, n_cells=20, seed=k) for k, n in enumerate((100, 9000, 3000, 2500, 400))]
    pool = bench.OraclePool(params, 8)
    assert pool.cores == len(params)        # never more processes than discharges
    n, t = pool.step()
    pool.close()
    assert n == sum(p["n_particles"] for p in params) and t > 0
    assert np.isfinite(t)


def test_source_hash_ignores_comments_but_not_code():
    """The profile-to-source check of the bench survives comment edits only."""
    import bench
    a = "int f(int x) {  // one\n    return x + 1; /* two\n lines */\n}\n"
    b = "int f(int x) {\n  return x + 1;  // other words\n}\n"
    c = "int f(int x) {\n    return x + 2;\n}\n"
    assert bench.source_hash(a) == bench.source_hash(b)
    assert bench.source_hash(a) != bench.source_hash(c)


def test_kernel_hash_covers_the_nvcc_flags_but_not_paths(monkeypatch):
    """A profile taken under other compiler flags (say without -ftz) does not
    match the kernel; the include paths, which differ between machines, do
    not enter the hash."""
    import bench
    from paper_1508_02892_gb300 import build
    flags = build._flags()
    base = bench.kernel_hash()
    monkeypatch.setattr(build, "_flags", lambda: [f for f in flags if f != "-ftz=true"])
    assert bench.kernel_hash() != base
    monkeypatch.setattr(build, "_flags", lambda: [f if not f.startswith("/") else "/elsewhere" + f for f in flags])
    assert bench.kernel_hash() == base
