"""Continuous-batching policy of the serving loop, on the CPU with a fake
executor and a fake clock (no GPU): batches hold one scene, FIFO within a
scene, never exceed the memory budget or the batch cap, requests that arrive
while slots are busy are batched into the next free slot, and every request
completes."""
from dataclasses import dataclass

from paper_2412_00578_gb300 import serve


@dataclass
class Cam:
    width: int
    height: int


class FakeClock:
    def __init__(self, dt=1e-4):
        self.t = 0.0
        self.dt = dt

    def __call__(self):
        self.t += self.dt
        return self.t


class FakeExecutor:
    def __init__(self, clock, slots=2, batch_time=5e-3):
        self.clock = clock
        self.busy = [None] * slots
        self.batch_time = batch_time
        self.launched = []

    def free_slots(self):
        return [k for k, b in enumerate(self.busy) if b is None]

    def launch(self, slot, reqs, nbytes, bid):
        self.busy[slot] = (reqs, nbytes, self.clock.t + self.batch_time, bid)
        self.launched.append((slot, [r.rid for r in reqs], nbytes, self.clock.t))

    def poll(self):
        out = []
        for k, b in enumerate(self.busy):
            if b is not None and self.clock.t >= b[2]:
                out.append((k, b[0], b[1], b[3]))
                self.busy[k] = None
        return out


def make_requests(n=300, rate=2000.0):
    import torch

    gen = torch.Generator().manual_seed(1)
    reqs, t = [], 0.0
    for i in range(n):
        t += float(torch.empty(1).exponential_(rate, generator=gen))
        scene = ["small", "big"][int(torch.randint(2, (1,), generator=gen))]
        w, h = [(64, 48), (128, 96), (256, 128)][int(torch.randint(3, (1,), generator=gen))]
        reqs.append(serve.Request(i, scene, Cam(w, h), t))
    return reqs


def test_policy_invariants():
    clock = FakeClock()
    sizes = {"small": 1000, "big": 5000}
    budget = serve.batch_bytes(5000, [Cam(256, 128)] * 6)
    sch = serve.Scheduler(sizes, max_batch=8, memory_budget=budget)
    ex = FakeExecutor(clock, slots=2)
    reqs = make_requests()
    by_id = {r.rid: r for r in reqs}
    done, stats = serve.serve(reqs, sch, ex, clock=clock, idle_sleep=0)
    assert stats["requests"] == len(reqs) and sorted(r.rid for r in done) == list(range(len(reqs)))
    inflight = {}
    for slot, ids, nbytes, t in ex.launched:
        scenes = {by_id[i].scene for i in ids}
        assert len(scenes) == 1 and 1 <= len(ids) <= 8
        assert ids == sorted(ids)  # FIFO within the scene
        assert nbytes <= budget
        assert all(by_id[i].arrival <= t for i in ids)
    assert stats["mean_batch"] > 1.5  # arrivals during busy slots were batched
    assert stats["max_inflight_batches"] == 2
    assert sch.in_use == 0
    for r in done:
        assert r.start >= r.arrival and r.done > r.start


def test_oldest_scene_goes_first():
    sch = serve.Scheduler({"a": 10, "b": 10}, max_batch=4)
    for i, s in enumerate(["b", "a", "b", "a", "b"]):
        sch.submit(serve.Request(i, s, Cam(8, 8), 0.0))
    reqs, _ = sch.next_batch()
    assert [r.rid for r in reqs] == [0, 2, 4]
    reqs, _ = sch.next_batch()
    assert [r.rid for r in reqs] == [1, 3]


def test_expiry_and_cancellation():
    """A request that waits past its deadline is dropped, never launched; a
    cancel withdraws a request that is still waiting and is ignored once the
    request is on the GPU; everything else completes."""
    clock = FakeClock()
    sch = serve.Scheduler({"small": 1000, "big": 5000}, max_batch=2)
    ex = FakeExecutor(clock, slots=1, batch_time=2e-2)  # slow: a queue builds up
    reqs = make_requests(n=120, rate=4000.0)
    for r in reqs:
        r.deadline = 0.05
    cancels = [(reqs[5].arrival + 1e-4, 5), (reqs[0].arrival + 0.5, 0)]
    done, stats = serve.serve(reqs, sch, ex, clock=clock, idle_sleep=0, cancels=cancels)
    launched = {i for _, ids, _, _ in ex.launched for i in ids}
    by_status = {}
    for r in reqs:
        by_status.setdefault(r.status, []).append(r)
    assert stats["expired"] == len(by_status.get("expired", [])) > 0
    assert stats["cancelled"] == 1 and reqs[5].status == "cancelled" and 5 not in launched
    assert reqs[0].status == "done"  # its cancel came after it had started
    for r in by_status["expired"]:
        assert r.rid not in launched and r.start is None
    for r in done:
        assert r.status == "done" and r.start - r.arrival <= r.deadline + 1e-3
    assert len(done) + stats["expired"] + stats["cancelled"] == len(reqs)
