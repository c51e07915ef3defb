"""Host logic of the continuous-batching request loop, on CPU with a fake backend."""
from types import SimpleNamespace

import pytest

from paper_1902_08112_gb300 import serve, workloads as W


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeBackend:
    """Each instance converges its load step after (rid % 3) + 2 Newton steps; each Newton step
    costs 1 ms of fake time."""

    def __init__(self, clock):
        self.clock = clock
        self.live = set()
        self.batches = []
        self.peak_bytes = 0

    def bytes_for(self, w):
        return w.n_dofs * 100

    def create(self, w, pressure):
        inst = {"w": w, "k": 0, "rid": None}
        self.live.add(id(inst))
        return inst

    def start_load_step(self, inst, pressure, frac=1.0):
        inst["k"] = 0
        inst["p"] = pressure

    def newton(self, insts):
        self.batches.append(len(insts))
        self.clock.t += 1e-3
        out = []
        for inst in insts:
            inst["k"] += 1
            need = (inst["w"].seed % 3) + 2
            out.append(SimpleNamespace(converged=int(inst["k"] >= need), solve=SimpleNamespace(iterations=5)))
        return out

    def fetch(self, inst):
        return None

    def destroy(self, inst):
        self.live.discard(id(inst))


def reqs(n, sizes=(16,), load_steps=2, gap=0.0):
    ws = W.batch_instances(n, sizes=sizes, seed=3)
    return [serve.Request(i, w, load_steps=load_steps, arrival=i * gap) for i, w in enumerate(ws)]


def test_budget_fifo_and_retirement():
    clk = FakeClock()
    be = FakeBackend(clk)
    rs = reqs(6)
    per = be.bytes_for(rs[0].workload)
    srv = serve.Server(be, hbm_budget=2 * per + per // 2, clock=clk)
    for r in rs:
        srv.submit(r)
    admitted_order = []
    while srv.waiting or srv.active:
        before = {s["req"].rid for s in srv.active}
        srv.tick()
        assert srv.used <= srv.budget
        assert len(srv.active) <= 2
        admitted_order += [rid for rid in sorted(srv.results) if srv.results[rid].admitted and rid not in before
                           and rid not in admitted_order]
    assert admitted_order == sorted(admitted_order)            # FIFO
    assert srv.used == 0 and not be.live                       # everything retired and freed
    for r in srv.results.values():
        assert len(r.load_step_latency) == 2 and r.finished >= r.admitted >= 0.0
        assert all(c for c in r.converged)


def test_requests_join_while_others_run():
    clk = FakeClock()
    be = FakeBackend(clk)
    rs = reqs(4, gap=2.5e-3)        # arrive every 2.5 fake ms, each needs >= 4 Newton steps
    srv = serve.Server(be, hbm_budget=10 ** 12, clock=clk)
    srv.run(rs, realtime=True, idle_sleep=0.0)
    # continuous batching: some tick ran more than one instance, and a later request was admitted
    # before an earlier one finished
    assert max(be.batches) > 1
    res = srv.results
    assert any(res[j].admitted < res[i].finished for i in res for j in res if j > i)


def test_oversize_request_rejected():
    clk = FakeClock()
    be = FakeBackend(clk)
    r = reqs(1)[0]
    srv = serve.Server(be, hbm_budget=10, clock=clk)
    srv.submit(r)
    with pytest.raises(ValueError):
        srv.tick()


def test_summary_percentiles():
    res = {0: serve.Result(0, 0.0, 0.0, 0.01, solve_latency=[0.001, 0.002], load_step_latency=[0.003]),
           1: serve.Result(1, 0.0, 0.0, 0.02, solve_latency=[0.004], load_step_latency=[0.005])}
    s = serve.summarize(res, wall=0.5)
    assert s["linear_solves"] == 3 and s["solves_per_s"] == pytest.approx(6.0)
    assert s["solve_ms_p50"] == pytest.approx(2.0)
    assert s["request_ms_p99"] == pytest.approx(19.9, rel=1e-3)


def test_cancel_releases_bytes():
    """A request cancelled while admitted gives its device bytes back and lets a waiting one in;
    a cancelled waiting request never runs."""
    clk = FakeClock()
    be = FakeBackend(clk)
    rs = reqs(4)
    per = be.bytes_for(rs[0].workload)
    srv = serve.Server(be, hbm_budget=2 * per, clock=clk)
    for r in rs:
        srv.submit(r)
    srv.tick()
    assert {s["req"].rid for s in srv.active} == {0, 1} and srv.used == 2 * per
    assert srv.cancel(0)
    assert srv.used == per and len(be.live) == 1
    assert srv.cancel(3)                       # still waiting
    assert not srv.cancel(99)
    while srv.waiting or srv.active:
        srv.tick()
        assert srv.used <= srv.budget
    assert srv.used == 0 and not be.live
    assert srv.results[0].cancelled and srv.results[3].cancelled
    assert srv.results[3].admitted == 0.0 and srv.results[3].U is None
    assert srv.results[2].admitted > 0.0 and not srv.results[2].cancelled
    assert serve.summarize(srv.results, 1.0)["requests"] == 4
