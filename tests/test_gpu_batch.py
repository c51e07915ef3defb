"""Batches of independent instances (one launch per level and operation across instances).

Checks, through the C ABI: a batched V-cycle and FGMRES give every instance the same result as
the single-instance calls (FP32 V-cycle: 1e-5; FGMRES: same iteration count +-1, both reach 1e-8
and agree to 1e-6), results are the same alone (a batch of one) and in a mixed batch (1e-6:
FP32 atomic accumulation order on tile borders varies run to run at the 1e-7 level),
and a batched Newton step matches the single-instance Newton step (active set exact)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1902_08112_gb300 import pff, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel(a, b):
    a = a.cpu().numpy()
    b = b.cpu().numpy()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


SIZES = [(8, 2), (16, 3), (12, 2), (24, 3), (16, 2)]   # (cells per edge, levels): uneven mix


def make_instances(sizes=SIZES, seed=0, mgp=32):
    out = []
    rng = np.random.default_rng(seed)
    for k, (n, L) in enumerate(sizes):
        w = W.small(W.config_3d_penny(), n, L)
        w.pressure = float(rng.uniform(5e-4, 2e-3))
        w.cracks = [W.Crack(tuple(rng.uniform(-4, 4, 3)), (0.0, 0.0, 1.0), float(rng.uniform(1.0, 3.0)))]
        U, po, pt = W.initial_state(w, displacement="smooth")
        prm = pff.default_params(eps=w.eps, pressure=w.pressure, kappa=w.kappa, seed=100 + k, mg_precision=mgp)
        h = pff.create_hierarchy(pff.make_mesh(3, 1, w.n_cells, w.n_levels, w.lo, w.hi), prm)
        Ud, pod, ptd = t(U), t(po), t(pt)
        pff.set_state(h, Ud, pod, ptd)
        pff.update_active_set(h)
        out.append({"w": w, "h": h, "U": Ud, "po": pod, "pt": ptd})
    return out


@pytest.fixture(scope="module")
def inst():
    xs = make_instances()
    yield xs
    for x in xs:
        pff.destroy_hierarchy(x["h"])


def test_batch_vcycle_matches_single(inst):
    rs = [t(W.random_vector(x["w"].n_dofs, 10 + i)) for i, x in enumerate(inst)]
    zs_single = []
    for x, r in zip(inst, rs):
        pff.setup(x["h"])
        z = torch.zeros_like(r)
        pff.vcycle(x["h"], r, z)
        zs_single.append(z)
    b = pff.batch_create([x["h"] for x in inst])
    try:
        pff.batch_setup(b)
        zs = [torch.zeros_like(r) for r in rs]
        pff.batch_vcycle(b, rs, zs)
        torch.cuda.synchronize()
        for z, zr in zip(zs, zs_single):
            assert rel(z, zr) <= 1e-5
    finally:
        pff.batch_destroy(b)


def test_batch_gmres_alone_vs_mix_and_single(inst):
    rs = [t(W.random_vector(x["w"].n_dofs, 20 + i)) for i, x in enumerate(inst)]
    # single-instance solves
    single = []
    for x, r in zip(inst, rs):
        xs = torch.zeros_like(r)
        info = pff.gmres_solve(x["h"], r, xs, rtol=1e-8, restart=30, maxit=200)
        single.append((xs, info))
    # the whole mix
    b = pff.batch_create([x["h"] for x in inst])
    try:
        xm = [torch.zeros_like(r) for r in rs]
        infos = pff.batch_gmres_solve(b, rs, xm, rtol=1e-8, maxit=200)
    finally:
        pff.batch_destroy(b)
    # each instance alone (a batch of one)
    for i, (x, r) in enumerate(zip(inst, rs)):
        b1 = pff.batch_create([x["h"]])
        try:
            xa = torch.zeros_like(r)
            ia = pff.batch_gmres_solve(b1, [r], [xa], rtol=1e-8, maxit=200)[0]
        finally:
            pff.batch_destroy(b1)
        assert infos[i].converged and ia.converged
        assert infos[i].res_final <= 1e-8 * infos[i].res0 * 1.0001
        assert ia.iterations == infos[i].iterations
        assert rel(xm[i], xa) <= 1e-6
        xs, si = single[i]
        assert abs(si.iterations - infos[i].iterations) <= 1
        assert rel(xm[i], xs) <= 1e-6


def test_batch_newton_step_matches_single():
    a = make_instances(SIZES[:3], seed=1)
    c = make_instances(SIZES[:3], seed=1)
    try:
        single = []
        for x in a:
            U = x["U"].clone()
            info = pff.newton_step(x["h"], U)
            single.append((U, info))
        b = pff.batch_create([x["h"] for x in c])
        try:
            Us = [x["U"].clone() for x in c]
            infos = pff.batch_newton_step(b, Us)
        finally:
            pff.batch_destroy(b)
        for (Ur, ir), U, ib in zip(single, Us, infos):
            assert ib.n_active == ir.n_active and ib.n_changed == ir.n_changed
            assert ib.res_norm == pytest.approx(ir.res_norm, rel=1e-12)
            assert abs(ib.solve.iterations - ir.solve.iterations) <= 1
            assert rel(U, Ur) <= 1e-6
    finally:
        for x in a + c:
            pff.destroy_hierarchy(x["h"])


def test_batch_rejects_mixed_precision():
    w = W.small(W.config_3d_penny(), 8, 2)
    h1 = pff.create_hierarchy(pff.make_mesh(3, 1, w.n_cells, 2, w.lo, w.hi), pff.default_params(mg_precision=32))
    h2 = pff.create_hierarchy(pff.make_mesh(3, 1, w.n_cells, 2, w.lo, w.hi), pff.default_params(mg_precision=64))
    try:
        with pytest.raises(pff.PffError) as e:
            pff.batch_create([h1, h2])
        assert e.value.status == pff.EINVAL
    finally:
        pff.destroy_hierarchy(h1)
        pff.destroy_hierarchy(h2)


def test_batch_fp64_vcycle_and_solve_match_single():
    """mg_precision 64 in every instance: the batched FP64 V-cycle equals the single-instance one
    (1e-9: atomic accumulation order only) and the batched FGMRES needs the same iterations."""
    xs = make_instances(mgp=64)
    try:
        rs = [t(W.random_vector(x["w"].n_dofs, 40 + i)) for i, x in enumerate(xs)]
        zs_single, its_single = [], []
        for x, r in zip(xs, rs):
            pff.setup(x["h"])
            z = torch.zeros_like(r)
            pff.vcycle(x["h"], r, z)
            zs_single.append(z)
            xx = torch.zeros_like(r)
            its_single.append(pff.gmres_solve(x["h"], r, xx, rtol=1e-8, restart=30, maxit=200).iterations)
        b = pff.batch_create([x["h"] for x in xs])
        try:
            pff.batch_setup(b)
            zs = [torch.zeros_like(r) for r in rs]
            pff.batch_vcycle(b, rs, zs)
            torch.cuda.synchronize()
            for z, zr in zip(zs, zs_single):
                assert rel(z, zr) <= 1e-9
            xb = [torch.zeros_like(r) for r in rs]
            infos = pff.batch_gmres_solve(b, rs, xb, rtol=1e-8, maxit=200)
            assert [i.iterations for i in infos] == its_single
            assert all(i.converged for i in infos)
        finally:
            pff.batch_destroy(b)
    finally:
        for x in xs:
            pff.destroy_hierarchy(x["h"])


def test_batch_submit_retire_poll():
    """Continuous batching through the ABI: an empty batch, instances submitted and retired between
    Newton steps; each instance's step equals the single-instance step (active set exact, same
    iterations +-1, 1e-6), poll returns the last infos, and misuse is rejected."""
    xs = make_instances(SIZES[:4], seed=3)
    ref = make_instances(SIZES[:4], seed=3)
    try:
        b = pff.batch_create([])
        try:
            with pytest.raises(pff.PffError) as e:
                pff.batch_newton_step(b, [])
            assert e.value.status == pff.ESTATE
            for x in xs[:3]:
                pff.batch_submit(b, x["h"])
            assert pff.batch_size(b) == 3
            with pytest.raises(pff.PffError) as e:
                pff.batch_submit(b, xs[0]["h"])            # already in the batch
            assert e.value.status == pff.EINVAL
            pff.batch_retire(b, 1)                         # xs[1] leaves before any step
            pff.batch_submit(b, xs[3]["h"])                # xs[3] joins: order is xs[0], xs[2], xs[3]
            members = [0, 2, 3]
            Us = [xs[k]["U"].clone() for k in members]
            infos = pff.batch_newton_step(b, Us)
            for j, k in enumerate(members):
                Ur = ref[k]["U"].clone()
                ir = pff.newton_step(ref[k]["h"], Ur)
                assert infos[j].n_active == ir.n_active and abs(infos[j].solve.iterations - ir.solve.iterations) <= 1
                assert rel(Us[j], Ur) <= 1e-6
                p = pff.batch_poll(b, j)
                assert p.n_active == infos[j].n_active and p.solve.iterations == infos[j].solve.iterations
            pff.batch_retire(b, 0)
            assert pff.batch_size(b) == 2
            with pytest.raises(pff.PffError) as e:
                pff.batch_retire(b, 5)
            assert e.value.status == pff.EINVAL
            infos2 = pff.batch_newton_step(b, [Us[1], Us[2]])
            assert all(i.solve.converged for i in infos2)
        finally:
            pff.batch_destroy(b)
        w = W.small(W.config_3d_penny(), 8, 2)
        h64 = pff.create_hierarchy(pff.make_mesh(3, 1, w.n_cells, 2, w.lo, w.hi), pff.default_params(mg_precision=64))
        b = pff.batch_create([xs[0]["h"]])
        try:
            with pytest.raises(pff.PffError) as e:
                pff.batch_submit(b, h64)                   # another V-cycle precision
            assert e.value.status == pff.EINVAL
        finally:
            pff.batch_destroy(b)
            pff.destroy_hierarchy(h64)
    finally:
        for x in xs + ref:
            pff.destroy_hierarchy(x["h"])
