"""Continuous-batching request loop over the batch API.

Requests (a discharge's parameters plus a step count) arrive over time.  Each
is admitted into a free slot of one resident batch as soon as a slot and its
device footprint fit under the HBM cap, so runs that arrive while others are
on the GPU join the next chunk of lockstep launches; every discharge keeps its
particles and fields on the device between chunks.  After each chunk the loop
polls for runs that reached their step count, reads their results and evicts
them, which frees the slot and the memory for the queue.

Admission is first come, first served (no request overtakes an earlier one
that does not fit yet).  Latency is counted from a request's arrival to the
end of the chunk in which it finished.

With a batch that takes status snapshots (the default), the loop keeps one
chunk queued ahead: chunk n+1 runs on the GPU while the host reads the runs
that finished in chunk n (counters from the snapshot, moments on a side
stream), evicts them and admits newcomers, whose copies and kernels queue
behind chunk n+1 without the host waiting for it.  A newcomer then starts one
chunk later than in the plain loop, and the GPU does not idle between chunks.
"""
import time
from collections import deque

import numpy as np

from . import hybrid


class Server:
    def __init__(self, max_slots=64, hbm_cap_bytes=120e9, precision=hybrid.HYB_FP32_SPLIT, stream=None,
                 chunk=100, tuning=None, clock=None, batch=None, footprint=None, pipelined=None):
        # batch / footprint: stand-ins with the same methods, for testing the
        # scheduling without a GPU
        self.batch = batch if batch is not None else hybrid.Batch(max_slots, precision, int(hbm_cap_bytes),
                                                                   stream=stream)
        self.footprint = footprint or hybrid.footprint
        if tuning:
            self.batch.set_tuning(**tuning)
        self.max_slots = int(max_slots)
        self.cap = int(hbm_cap_bytes)
        self.chunk = int(chunk)
        self.chunks = 0
        self.clock = clock
        self._t0 = None
        self.pipelined = hasattr(self.batch, "snapshot") if pipelined is None else bool(pipelined)

    def close(self):
        self.batch.close()

    def now(self):
        if self.clock is not None:
            return float(self.clock())
        return time.perf_counter() - self._t0

    def run(self, requests, keep=("counters", "moments")):
        """Serve `requests` (dicts with arrival_s, steps, params and an
        optional tag) to completion; returns one record per request with its
        arrival, admission and completion times, the particle-steps it ran and
        the results named in `keep` ("counters", "moments", "particles")."""
        if self.pipelined:
            return self._run_pipelined(requests, keep)
        self._t0 = time.perf_counter()
        self.max_bytes = 0
        order = sorted(range(len(requests)), key=lambda i: requests[i]["arrival_s"])
        pending = deque(order)
        queue = deque()
        running = {}
        out = [None] * len(requests)
        used = 0
        fp = {}
        while pending or queue or running:
            now = self.now()
            while pending and requests[pending[0]]["arrival_s"] <= now:
                queue.append(pending.popleft())
            while queue and len(running) < self.max_slots:
                i = queue[0]
                r = requests[i]
                if i not in fp:
                    fp[i] = self.footprint(r["params"])
                if self.cap > 0 and used + fp[i] > self.cap:
                    break
                slot = self.batch.admit(r["params"], n_steps=int(r["steps"]))
                queue.popleft()
                used += fp[i]
                self.max_bytes = max(self.max_bytes, used)
                running[slot] = i
                out[i] = {"tag": r.get("tag", i), "arrival_s": r["arrival_s"], "admitted_s": self.now(),
                          "slot": slot}
            if not running:
                if pending and self.clock is None:
                    time.sleep(max(0.0, requests[pending[0]]["arrival_s"] - self.now()))
                elif pending:
                    # a virtual clock only moves with chunks: jump to the arrival
                    self._skip_to(requests[pending[0]]["arrival_s"])
                continue
            self.batch.advance(self.chunk)
            self.chunks += 1
            done = self.batch.poll()
            t_done = self.now()
            for slot in done:
                i = running.pop(slot)
                rec = out[i]
                c = self.batch.counters(slot)
                rec["done_s"] = t_done
                rec["latency_s"] = t_done - rec["arrival_s"]
                rec["particle_steps"] = int(c["pushes"])
                rec["status"] = int(c["status"])
                if "counters" in keep:
                    rec["counters"] = c
                if "moments" in keep:
                    rec["moments"] = self.batch.moments(slot)
                if "particles" in keep:
                    rec["particles"] = self.batch.particles(slot)
                self.batch.evict(slot)
                used -= fp[i]
        return out

    def _run_pipelined(self, requests, keep):
        self._t0 = time.perf_counter()
        self.max_bytes = 0
        order = sorted(range(len(requests)), key=lambda i: requests[i]["arrival_s"])
        pending = deque(order)
        queue = deque()
        running = {}
        out = [None] * len(requests)
        used = 0
        fp = {}
        in_flight = 0      # chunks queued whose snapshot has not been polled
        while pending or queue or running or in_flight:
            now = self.now()
            while pending and requests[pending[0]]["arrival_s"] <= now:
                queue.append(pending.popleft())
            while queue and len(running) < self.max_slots:
                i = queue[0]
                r = requests[i]
                if i not in fp:
                    fp[i] = self.footprint(r["params"])
                if self.cap > 0 and used + fp[i] > self.cap:
                    break
                slot = self.batch.admit(r["params"], n_steps=int(r["steps"]))
                queue.popleft()
                used += fp[i]
                self.max_bytes = max(self.max_bytes, used)
                running[slot] = i
                out[i] = {"tag": r.get("tag", i), "arrival_s": r["arrival_s"], "admitted_s": self.now(),
                          "slot": slot}
            if running and in_flight < 2:
                # queue the next chunk (and its snapshot) before reading the last one
                self.batch.advance(self.chunk)
                self.batch.snapshot()
                in_flight += 1
                if in_flight < 2:
                    continue
            if in_flight == 0:
                if pending and self.clock is None:
                    time.sleep(max(0.0, requests[pending[0]]["arrival_s"] - self.now()))
                elif pending:
                    self._skip_to(requests[pending[0]]["arrival_s"])
                continue
            done, _ = self.batch.poll_snapshot()
            in_flight -= 1
            self.chunks += 1
            t_done = self.now()
            for slot in done:
                i = running.pop(slot)
                rec = out[i]
                c, m, _ = self.batch.read_finished(slot, moments="moments" in keep)
                rec["done_s"] = t_done
                rec["latency_s"] = t_done - rec["arrival_s"]
                rec["particle_steps"] = int(c["pushes"])
                rec["status"] = int(c["status"])
                if "counters" in keep:
                    rec["counters"] = c
                if "moments" in keep:
                    rec["moments"] = m
                if "particles" in keep:
                    rec["particles"] = self.batch.particles(slot)
                self.batch.evict(slot)
                used -= fp[i]
        return out

    def _skip_to(self, t):
        skip = getattr(self.clock, "skip_to", None)
        if skip is None:
            raise RuntimeError("a virtual clock must provide skip_to(t)")
        skip(t)


class ChunkClock:
    """Virtual time that advances by `dt` per chunk the server runs (or jumps
    to the next arrival when the server is idle): a reproducible mix."""

    def __init__(self, dt=0.05):
        self.dt = dt
        self.server = None
        self.offset = 0.0

    def __call__(self):
        return self.offset + (self.server.chunks if self.server else 0) * self.dt

    def skip_to(self, t):
        self.offset = max(self.offset, t - (self.server.chunks if self.server else 0) * self.dt)


def summarize(records, wall_s):
    lat = np.array([r["latency_s"] for r in records if r and "latency_s" in r])
    steps = sum(r["particle_steps"] for r in records if r and "particle_steps" in r)
    return {"requests": int(lat.size), "p50_latency_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_latency_s": float(lat.mean()) if lat.size else None,
            "particle_steps": int(steps), "wall_s": wall_s,
            "throughput": steps / wall_s if wall_s > 0 else None}
