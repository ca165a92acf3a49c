"""Scheduling logic of the request loop, on the CPU with a stand-in batch:
first-come-first-served admission under the slot and HBM limits, requests
joining while others run, completion at their own step counts, latency from
arrival to the end of the finishing chunk."""
from paper_1508_02892_gb300.serve import ChunkClock, Server, summarize


class FakeBatch:
    def __init__(self, slots):
        self.free = list(range(slots))
        self.run = {}        # slot -> [steps done, target, particles]
        self.log = []

    def admit(self, params, n_steps=0):
        slot = self.free.pop(0)
        self.run[slot] = [0, n_steps, params["n_particles"]]
        self.log.append(("admit", params["tag"], slot))
        return slot

    def advance(self, n):
        for r in self.run.values():
            r[0] = min(r[1], r[0] + n)

    def poll(self):
        return [s for s, r in sorted(self.run.items()) if r[0] >= r[1] and not r[3:]]

    def counters(self, slot):
        r = self.run[slot]
        r.append("reported")
        return {"pushes": r[0] * r[2], "status": 0, "step": r[0]}

    def moments(self, slot):
        return {}

    def evict(self, slot):
        del self.run[slot]
        self.free.append(slot)
        self.free.sort()

    def close(self):
        pass


def _reqs():
    # (arrival, steps, bytes)
    spec = [(0.0, 250, 40), (0.01, 100, 40), (0.02, 300, 50), (0.03, 100, 10), (0.5, 100, 30)]
    return [{"arrival_s": a, "steps": n, "tag": k, "params": {"n_particles": 1000 * (k + 1), "bytes": b, "tag": k}}
            for k, (a, n, b) in enumerate(spec)]


def test_fifo_admission_under_slot_and_memory_limits():
    fb = FakeBatch(2)
    clk = ChunkClock(0.05)
    srv = Server(max_slots=2, hbm_cap_bytes=90, chunk=100, clock=clk, batch=fb,
                 footprint=lambda p: p["bytes"])
    clk.server = srv
    out = srv.run(_reqs(), keep=())
    assert srv.max_bytes <= 90
    order = [t for ev, t, _ in fb.log if ev == "admit"]
    assert order == [0, 1, 2, 3, 4]                    # nobody overtakes
    by = {r["tag"]: r for r in out}
    # request 2 (50 bytes) waits for request 1 to free memory, request 3 for a slot
    assert by[2]["admitted_s"] >= by[1]["done_s"]
    assert by[3]["admitted_s"] >= min(by[0]["done_s"], by[2]["done_s"])
    for r in out:
        assert r["done_s"] >= r["admitted_s"] >= r["arrival_s"]
        assert abs(r["latency_s"] - (r["done_s"] - r["arrival_s"])) < 1e-12
    # whole chunks of 100 steps: 250 steps need 3 chunks after admission
    assert abs(by[0]["done_s"] - by[0]["admitted_s"] - 3 * 0.05) < 1e-9
    assert by[4]["admitted_s"] >= 0.5                  # idle server jumps to the arrival
    s = summarize(out, wall_s=1.0)
    assert s["requests"] == 5 and s["particle_steps"] == sum(
        r["steps"] * r["params"]["n_particles"] for r in _reqs())


class FakeSnapshotBatch(FakeBatch):
    """The same stand-in with the snapshot calls: work is applied in call
    order (the order of a stream), a snapshot copies the state at its place in
    that order, and polls consume snapshots oldest first."""

    def __init__(self, slots):
        super().__init__(slots)
        self.snaps = []
        self.last = None
        self.reads = []
        self.issued = 0
        self.admitted_after = {}

    def admit(self, params, n_steps=0):
        slot = super().admit(params, n_steps)
        self.admitted_after[slot] = self.issued      # earlier snapshots do not show this run
        return slot

    def snapshot(self):
        self.snaps.append((self.issued, {s: list(r[:3]) for s, r in self.run.items()}))
        self.issued += 1

    def poll_snapshot(self):
        seq, snap = self.snaps.pop(0)
        self.last = snap
        done = [s for s, r in sorted(snap.items())
                if r[0] >= r[1] and s in self.run and not self.run[s][3:] and seq >= self.admitted_after[s]]
        for s in done:
            self.run[s].append("reported")
        return done, 0

    def read_finished(self, slot, moments=True):
        r = self.last[slot]
        self.reads.append(slot)
        return {"pushes": r[0] * r[2], "status": 0, "step": r[0]}, {}, 0

    def evict(self, slot):
        assert slot in self.reads                       # results are read before the slot goes
        super().evict(slot)


def test_pipelined_loop_keeps_fifo_limits_and_step_counts():
    fb = FakeSnapshotBatch(2)
    clk = ChunkClock(0.05)
    srv = Server(max_slots=2, hbm_cap_bytes=90, chunk=100, clock=clk, batch=fb, footprint=lambda p: p["bytes"])
    assert srv.pipelined
    clk.server = srv
    out = srv.run(_reqs(), keep=("counters",))
    assert srv.max_bytes <= 90
    order = [t for ev, t, _ in fb.log if ev == "admit"]
    assert order == [0, 1, 2, 3, 4]                    # nobody overtakes
    by = {r["tag"]: r for r in out}
    for r, q in zip(out, _reqs()):
        assert r["counters"]["step"] == q["steps"]       # each run ends at its own step count
        assert r["done_s"] >= r["admitted_s"] >= r["arrival_s"]
    # whole chunks of 100 steps: 250 steps need 3 chunks after admission
    assert abs(by[0]["done_s"] - by[0]["admitted_s"] - 3 * 0.05) < 1e-9
    assert by[2]["admitted_s"] >= by[1]["done_s"]
    assert not fb.run and not fb.snaps                  # everything evicted, every snapshot polled
