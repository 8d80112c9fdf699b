"""Host logic of the serving loop on CPU, with a stand-in for the device
batch: requests are admitted only after they arrive, a request too large for
the free memory does not hold back smaller ones, every request completes at
its own step count, and the latency summary is consistent."""
import pytest

from paper_2604_17463_gb300 import iblb, serve
from paper_2604_17463_gb300 import workloads as W


class FakeBatch:
    """Admission by a cell budget; each run advances every slot by `chunk`
    (never past its own step count)."""
    log = []

    def __init__(self, lattice, storage, budget, max_slots=64, stream=None):
        self.lattice, self.budget, self.used = lattice, budget, 0
        self.slots = {}
        self.next = 0
        self.launches = 0

    def admit_workload(self, wl):
        if self.used + wl.cells > self.budget:
            return None
        s = self.next
        self.next += 1
        self.slots[s] = [wl, wl.steps]
        self.used += wl.cells
        FakeBatch.log.append(("admit", wl.name))
        return s

    def run(self, chunk):
        for v in self.slots.values():
            v[1] -= min(chunk, v[1])
        self.launches += 1
        FakeBatch.log.append(("run", chunk))

    def sync(self):
        pass

    def steps_to_next_completion(self):
        left = [v[1] for v in self.slots.values() if v[1] > 0]
        return min(left) if left else -1

    def poll(self):
        return [s for s, v in self.slots.items() if v[1] == 0]

    def observables(self, s):
        return {"theta_deg": 90.0, "volume": 1.0, "height": 2.0}

    def release(self, s):
        wl, _ = self.slots.pop(s)
        self.used -= wl.cells

    def info(self):
        return {"kernel_launches": self.launches}

    def close(self):
        pass


def req(name, t, cells_w, steps, lattice=9):
    wl = W.Workload(name, lattice, cells_w, 10, 1, 1.0, 1e-3, 1.0, 90.0, 9, 3, steps,
                    W.circle(8, 2.0, (cells_w / 2.0, 5.0)), None)
    return W.Request(t, wl)


@pytest.fixture
def fake(monkeypatch):
    FakeBatch.log = []
    monkeypatch.setattr(iblb, "Batch", FakeBatch)
    return FakeBatch


def test_every_request_completes_and_summary_is_consistent(fake):
    reqs = [req(f"r{i}", 0.002 * i, 20 + i, 100 * (1 + i % 3)) for i in range(12)]
    out = serve.serve(reqs, iblb.FP16_DEV, budget_2d=10_000, budget_3d=10_000, chunk=100,
                      streams=(0, 0))
    assert out["completed"] == 12
    for r, res in zip(reqs, out["results"]):
        assert res["admitted_s"] >= r.arrival_s - 1e-9       # never before arrival
        assert res["done_s"] >= res["admitted_s"]
        assert res["latency_s"] == pytest.approx(res["done_s"] - r.arrival_s)
        assert res["steps"] == r.work.steps
    assert out["p50_s"] <= out["p99_s"]
    assert out["mlups"] > 0


def test_large_request_does_not_block_smaller_ones(fake):
    # budget 1000 cells (rows of 10): one 600-cell job runs; a 900-cell job
    # must wait for it, while the 200-cell jobs behind it go in at once
    reqs = [req("a600", 0.0, 60, 300), req("b900", 0.0, 90, 100),
            req("c200", 0.0, 20, 100), req("d200", 0.0, 20, 100)]
    out = serve.serve(reqs, iblb.FP32_DEV, budget_2d=1000, budget_3d=1000, chunk=100,
                      streams=(0, 0))
    assert out["completed"] == 4
    order = [n for ev, n in fake.log if ev == "admit"]
    assert order.index("c200") < order.index("b900")
    assert order.index("d200") < order.index("b900")
    assert out["max_queue"] >= 1


def test_rounds_stop_at_the_next_completion(fake):
    # with chunk = 500, a 120-step request completes after a round of 120
    # steps (not 500), and the 1000-step one keeps running in later rounds
    reqs = [req("short", 0.0, 20, 120), req("long", 0.0, 20, 1000)]
    out = serve.serve(reqs, iblb.FP32_DEV, budget_2d=10_000, budget_3d=10_000, chunk=500,
                      streams=(0, 0))
    assert out["completed"] == 2
    runs = [c for ev, c in fake.log if ev == "run"]
    assert runs[0] == 120
    assert runs[1:] == [500, 380]
    assert all(r["steps"] == q.work.steps for r, q in zip(out["results"], reqs))
