"""Serving on the GPU: a request's result is the same alone and in a mix of concurrently served
requests (1e-6 relative: both converge every linear solve to 1e-8 and FP32 accumulation order on
tile borders varies), and every request finishes its load steps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1902_08112_gb300 import serve, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def _requests():
    ws = W.batch_instances(5, sizes=(16, 24), seed=7)
    ws.append(W.config_3d_lshape(16, n_levels=3))          # an L-shaped panel in the mix
    return [serve.Request(i, w, load_steps=2, arrival=0.0) for i, w in enumerate(ws)]


def test_alone_vs_mix():
    rs = _requests()
    target = rs[2]
    alone = serve.Server(serve.PffBackend(), hbm_budget=8 << 30)
    alone.run([serve.Request(target.rid, target.workload, load_steps=2)], realtime=False)
    Ua = alone.results[target.rid].U
    mix = serve.Server(serve.PffBackend(), hbm_budget=8 << 30, max_active=3)   # some requests wait and join later
    t0 = mix.now()
    mix.run(rs, realtime=False)
    wall = mix.now() - t0
    Um = mix.results[target.rid].U
    assert np.linalg.norm(Um - Ua) <= 1e-6 * np.linalg.norm(Ua)
    for r in mix.results.values():
        assert r.U is not None and len(r.load_step_latency) == 2
    s = serve.summarize(mix.results, wall)
    assert s["solves_per_s"] > 0 and s["solve_ms_p99"] >= s["solve_ms_p50"]


def test_lshape_alone_vs_mix():
    """The L-shaped panel (cell-masked domain, one clamped face) served alone and in the mix."""
    rs = _requests()
    target = rs[-1]
    alone = serve.Server(serve.PffBackend(), hbm_budget=8 << 30)
    alone.run([serve.Request(target.rid, target.workload, load_steps=2)], realtime=False)
    Ua = alone.results[target.rid].U
    mix = serve.Server(serve.PffBackend(), hbm_budget=8 << 30, max_active=4)
    mix.run(rs, realtime=False)
    Um = mix.results[target.rid].U
    assert np.linalg.norm(Um) > 0
    assert np.linalg.norm(Um - Ua) <= 1e-6 * np.linalg.norm(Ua)
