"""Failure statuses of the C ABI, raised by host-side injections only (no device fault, trap or
hang is provoked): a NaN written into the state from the host gives PFF_ENONFINITE, an iteration
cap too small for the tolerance gives PFF_ENOCONV with the info filled in, calls out of order
give PFF_ESTATE, and a request cancelled while it is served returns its device memory.  After
each failure the hierarchy stays usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1902_08112_gb300 import pff, serve, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _make(w, mgp=64):
    prm = pff.default_params(eps=w.eps, pressure=w.pressure, kappa=w.kappa, mg_precision=mgp)
    return pff.create_hierarchy(pff.make_mesh(w.dim, w.deg, w.n_cells, w.n_levels, w.lo, w.hi), prm)


def test_nan_state_gives_nonfinite_and_recovers():
    w = W.small(W.config_3d_penny(), 16, 2)
    U, po, pt = W.initial_state(w, displacement="smooth")
    h = _make(w)
    try:
        bad = U.copy()
        bad[w.n_nodes // 2] = np.nan                   # one displacement DoF, written on the host
        Ud = t(bad)
        pff.set_state(h, Ud, t(po), t(pt))
        with pytest.raises(pff.PffError) as e:
            pff.newton_step(h, Ud)
        assert e.value.status == pff.ENONFINITE
        assert "non-finite" in pff.last_error(h)
        # the same hierarchy solves once the state is finite again
        Ud = t(U)
        pff.set_state(h, Ud, t(po), t(pt))
        info = pff.newton_step(h, Ud)
        assert info.solve.converged and np.isfinite(Ud.cpu().numpy()).all()
    finally:
        pff.destroy_hierarchy(h)


def test_iteration_cap_gives_noconv_with_info():
    w = W.small(W.config_3d_penny(), 16, 3)
    U, po, pt = W.initial_state(w, displacement="smooth")
    h = _make(w)
    try:
        pff.set_state(h, t(U), t(po), t(pt))
        pff.update_active_set(h)
        b = t(W.random_vector(w.n_dofs, 4))
        x = torch.zeros_like(b)
        with pytest.raises(pff.PffError) as e:
            pff.gmres_solve(h, b, x, rtol=1e-8, restart=30, maxit=1)
        assert e.value.status == pff.ENOCONV
        info = pff.gmres_solve(h, b, torch.zeros_like(b), rtol=1e-8, restart=30, maxit=1, allow_noconv=True)
        assert info.iterations == 1 and not info.converged
        assert 0 < info.res_final < info.res0
        info = pff.gmres_solve(h, b, x, rtol=1e-8, restart=30, maxit=200)
        assert info.converged
    finally:
        pff.destroy_hierarchy(h)


def test_calls_out_of_order_give_estate():
    w = W.small(W.config_2d_single_crack(), 16, 2)
    h = _make(w)
    try:
        x = t(W.random_vector(w.n_dofs, 1))
        y = torch.empty_like(x)
        for call in (lambda: pff.apply_jacobian(h, -1, x, y),
                     lambda: pff.residual(h, y),
                     lambda: pff.vcycle(h, x, y),
                     lambda: pff.update_active_set(h),
                     lambda: pff.setup(h),
                     lambda: pff.newton_step(h, y)):
            with pytest.raises(pff.PffError) as e:
                call()
            assert e.value.status == pff.ESTATE
        U, po, pt = W.initial_state(w)
        pff.set_state(h, t(U), t(po), t(pt))
        pff.apply_jacobian(h, -1, x, y)               # in order now
        torch.cuda.synchronize()
        assert torch.isfinite(y).all()
    finally:
        pff.destroy_hierarchy(h)


def test_batch_reports_the_nonfinite_instance():
    ws = [W.small(W.config_3d_penny(), 8, 2), W.small(W.config_3d_penny(), 16, 2)]
    hs, Us = [], []
    try:
        for k, w in enumerate(ws):
            U, po, pt = W.initial_state(w, displacement="smooth")
            if k == 1:
                U[3] = np.inf
            h = _make(w, mgp=32)
            Ud = t(U)
            pff.set_state(h, Ud, t(po), t(pt))
            hs.append(h)
            Us.append(Ud)
        b = pff.batch_create(hs)
        try:
            with pytest.raises(pff.PffError) as e:
                pff.batch_newton_step(b, Us)
            assert e.value.status == pff.ENONFINITE
            assert "instance 1" in pff.batch_last_error(b)
        finally:
            pff.batch_destroy(b)
    finally:
        for h in hs:
            pff.destroy_hierarchy(h)


def test_cancel_mid_serve_releases_device_memory():
    rs = [serve.Request(i, w, load_steps=3) for i, w in enumerate(W.batch_instances(3, sizes=(16, 24), seed=5))]
    be = serve.PffBackend()
    srv = serve.Server(be, hbm_budget=8 << 30)
    for r in rs:
        srv.submit(r)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    srv.tick()                                         # all three admitted, one Newton step each
    assert len(srv.active) == 3
    used = srv.used
    free1 = torch.cuda.mem_get_info()[0]
    assert srv.cancel(1)
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    assert srv.used == used - be.bytes_for(rs[1].workload)
    assert free2 - free1 >= 0.9 * pff.hierarchy_bytes(be.mesh(rs[1].workload), 0)
    srv.run([], realtime=False)                       # the other two finish
    assert srv.used == 0
    assert srv.results[0].U is not None and srv.results[2].U is not None and srv.results[1].U is None
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)
