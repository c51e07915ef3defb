"""Batched and served paths against the oracle (not against the single-instance GPU path).

An uneven mix of six 3D instances (8^3 .. 24^3 cells and one of 16 x 8 x 12 cells with three
different edge lengths, 1 to 3 levels, eps = 2h or 4h, seeded pressures and crack layouts) runs through the batch ABI; per instance:
  - the batched level operators on every level, in both kernel families (small-level kernels and
    per-cell kernels), against the oracle's assembled G_l x: FP64-accurate to 1e-12 and FP32 to 2e-5
    per block (displacement, phase field), elementwise against the block's largest entry too;
  - the batched FP64 V-cycle against the oracle's V-cycle (1e-9);
  - two batched active-set Newton steps (Algorithm 1): the active set exactly, the residual norm,
    FGMRES iterations within 10 % (FP32 V-cycle: +-1), and the update solving the oracle's
    eliminated system to the 1e-8 tolerance.
And two served requests (a crack instance and the displacement-driven L-shaped panel), two load steps
each in one mix, against the oracle's load steps (Algorithm 1 to its stop test) to 1e-6."""
import math
from dataclasses import replace

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem, krylov, multigrid as mg, pdas  # noqa: E402
from paper_1902_08112_gb300 import pff, serve, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

# (cells per edge, levels, eps factor); the last instance has cells of three edge lengths on a
# non-cubic box
MIX = [(8, 1, 2.0), (12, 2, 4.0), (16, 3, 2.0), (20, 2, 4.0), (24, 3, 2.0), ((16, 8, 12), 2, 2.0)]
ANISO_BOX = ((-10.0, -6.0, -8.0), (10.0, 6.0, 4.0))


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def block_errors(a, b, dim):
    a = a.detach().cpu().numpy().astype(np.float64)
    nn = b.size // (dim + 1)
    out = []
    for blk in (slice(0, dim * nn), slice(dim * nn, None)):
        d, r = a[blk] - b[blk], b[blk]
        out.append((np.linalg.norm(d) / max(np.linalg.norm(r), 1e-300), np.abs(d).max() / max(np.abs(r).max(), 1e-300)))
    return out


def mix_workloads(seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for n, L, ef in MIX:
        base = W.config_3d_penny()
        base.eps_factor = ef
        w = W.small(base, n, L)
        if not isinstance(n, int):
            w = replace(w, lo=ANISO_BOX[0], hi=ANISO_BOX[1], eps=0.0).finalize()
        w.pressure = float(rng.uniform(5e-3, 2e-2))
        w.cracks = [W.Crack(tuple(rng.uniform(-4, 4, 3)), (0.0, 0.0, 1.0), float(rng.uniform(1.5, 3.5)))]
        out.append(w)
    return out


class Inst:
    def __init__(self, w, k, mgp, stream=None):
        self.w = w
        self.seed = 100 + k
        self.U, self.po, self.pt = W.initial_state(w, displacement="smooth")
        self.prm = pff.default_params(eps=w.eps, pressure=w.pressure, kappa=w.kappa, seed=self.seed, mg_precision=mgp)
        self.h = pff.create_hierarchy(pff.make_mesh(3, 1, w.n_cells, w.n_levels, w.lo, w.hi), self.prm, stream)
        self.Ud = t(self.U)
        pff.set_state(self.h, self.Ud, t(self.po), t(self.pt))
        self.mesh = fem.Mesh(3, 1, w.n_cells, w.lo, w.hi)
        self.phys = fem.Phys(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=w.pressure)
        self.dmask = fem.dirichlet_face_mask(self.mesh, 0x3F)

    def oracle_system(self, U):
        R = -fem.residual_A(self.mesh, self.phys, U, self.pt)
        act = pdas.active_set(self.mesh, R, fem.lumped_mass(self.mesh), U, self.po, 100.0, 1e-10,
                              fixed=(self.dmask & fem.BIT_PHI_DIR) != 0)
        Rt, mask = pdas.eliminated_rhs(self.mesh, self.phys, U, self.pt, self.po, self.dmask, act, R)
        lv = mg.build_levels(self.mesh, self.w.n_levels, self.phys, U, self.pt, mask)
        mg.estimate_levels(lv, self.seed, 10)
        return act, Rt, lv


def make_mix(mgp, stream=None):
    return [Inst(w, k, mgp, stream) for k, w in enumerate(mix_workloads())]


def close(xs):
    for x in xs:
        pff.destroy_hierarchy(x.h)


@pytest.fixture(scope="module")
def mix64():
    xs = make_mix(64)
    for x in xs:
        pff.update_active_set(x.h)
    yield xs
    close(xs)


@pytest.mark.parametrize("style", [1, 2], ids=["small_level_kernels", "per_cell_kernels"])
def test_batched_applies_match_oracle(mix64, style):
    xs = mix64
    b = pff.batch_create([x.h for x in xs])
    try:
        pff.batch_set_kernel_style(b, style)
        oracle = [x.oracle_system(x.U) for x in xs]
        Lmax = max(x.w.n_levels for x in xs)
        for level in range(Lmax):
            idx = [i for i, x in enumerate(xs) if x.w.n_levels > level]
            dofs = {i: oracle[i][2][level].mesh.n_dofs for i in idx}
            for prec, dt, tol_n, tol_e in ((64, torch.float64, 1e-12, 1e-12), (32, torch.float32, 2e-5, 1e-4)):
                xin = {i: W.random_vector(dofs[i], 31 * level + i) for i in idx}
                xt = [t(xin[i].astype(np.float32 if prec == 32 else np.float64)) if i in xin
                      else torch.zeros(1, dtype=dt, device=DEV) for i in range(len(xs))]
                yt = [torch.full((dofs[i],) if i in dofs else (1,), 7.0, dtype=dt, device=DEV) for i in range(len(xs))]
                pff.batch_apply_jacobian(b, level, prec, xt, yt)
                torch.cuda.synchronize()
                for i in range(len(xs)):
                    if i not in idx:
                        assert float(yt[i][0]) == 7.0          # instances without this level are untouched
                        continue
                    xv = xin[i].astype(np.float32).astype(np.float64) if prec == 32 else xin[i]
                    ref = oracle[i][2][level].G @ xv
                    for k, (en, ee) in enumerate(block_errors(yt[i], ref, 3)):
                        assert en <= tol_n and ee <= tol_e, (style, level, prec, i, k, en, ee)
    finally:
        pff.batch_destroy(b)


def test_batched_fp64_vcycle_matches_oracle(mix64):
    xs = mix64
    b = pff.batch_create([x.h for x in xs])
    try:
        pff.batch_setup(b)
        rs = [W.random_vector(x.w.n_dofs, 50 + i) for i, x in enumerate(xs)]
        zs = [torch.zeros(x.w.n_dofs, dtype=torch.float64, device=DEV) for x in xs]
        pff.batch_vcycle(b, [t(r) for r in rs], zs)
        torch.cuda.synchronize()
        for x, r, z in zip(xs, rs, zs):
            act, _, lv = x.oracle_system(x.U)
            ga = torch.empty(x.w.n_nodes, dtype=torch.uint8, device=DEV)
            pff.get_active_set(x.h, ga)
            np.testing.assert_array_equal(ga.cpu().numpy().astype(bool), act)
            ref = mg.precondition(lv, r, mg.MGParams())
            zz = z.cpu().numpy()
            assert np.linalg.norm(zz - ref) <= 1e-9 * np.linalg.norm(ref)
    finally:
        pff.batch_destroy(b)


@pytest.mark.parametrize("mgp,graphs,switch", [(64, False, 10), (32, False, 10), (32, True, 10), (32, True, 2)],
                         ids=["fp64mg", "fp32mg", "fp32mg_graph_autotuned", "fp32mg_graph_switch_to_fp64"])
def test_batched_newton_steps_match_oracle(mgp, graphs, switch):
    """graphs: the hierarchies live on a non-default stream, so the batched FGMRES replays its captured
    Arnoldi step, and the level operators run the autotuner's choices.  switch: FGMRES iterations after
    which an FP32-MG instance continues with the FP64 V-cycle (2: most instances switch mid-solve, so the
    replayed step splits its V-cycle by precision)."""
    stream = torch.cuda.Stream() if graphs else None
    xs = make_mix(mgp, stream)
    torch.cuda.synchronize()
    try:
        b = pff.batch_create([x.h for x in xs])
        try:
            if not graphs:
                pff.batch_set_kernel_style(b, 1)
            pff.batch_set_precision_switch(b, switch)
            Uo = [x.U.copy() for x in xs]
            prev = [None] * len(xs)
            for step in range(2):
                Ud = [t(u) for u in Uo]
                torch.cuda.synchronize()
                infos = pff.batch_newton_step(b, Ud)
                if graphs:
                    for level in (-1, 0):
                        style, cps, ms = pff.batch_tuning(b, level, 64)
                        assert style in (1, 2) and cps >= 0 and ms > 0
                precs = pff.batch_mg_precisions(b, len(xs))
                for info, pr in zip(infos, precs):
                    want = 64 if (mgp == 64 or info.solve.iterations > switch) else 32
                    assert pr == want, (precs, [i.solve.iterations for i in infos])
                if switch == 2:
                    assert 64 in precs
                for i, (x, info) in enumerate(zip(xs, infos)):
                    act, Rt, lv = x.oracle_system(Uo[i])
                    ga = torch.empty(x.w.n_nodes, dtype=torch.uint8, device=DEV)
                    torch.cuda.synchronize()
                    pff.get_active_set(x.h, ga)
                    torch.cuda.synchronize()
                    np.testing.assert_array_equal(ga.cpu().numpy().astype(bool), act)
                    assert info.n_active == int(act.sum())
                    assert info.n_changed == (int(act.sum()) if prev[i] is None else int(np.sum(act != prev[i])))
                    assert info.res_norm == pytest.approx(np.linalg.norm(Rt), rel=1e-9)
                    G = lv[-1].G
                    _, its_o, _, _, _ = krylov.fgmres(lambda v: G @ v, Rt, lambda v: mg.precondition(lv, v, mg.MGParams()),
                                                      rtol=1e-8, restart=30, maxit=200)
                    slack = max(1, math.floor(0.1 * its_o)) if mgp == 32 else math.floor(0.1 * its_o)
                    assert abs(info.solve.iterations - its_o) <= slack, (i, info.solve.iterations, its_o)
                    torch.cuda.synchronize()
                    dU = Ud[i].cpu().numpy() - Uo[i]
                    assert np.linalg.norm(Rt - G @ dU) <= 1.01e-8 * np.linalg.norm(Rt)
                    prev[i] = act
                # both sides continue from the GPU iterate (the oracle's own iterate differs by 1e-8)
                Uo = [u.cpu().numpy() for u in Ud]
        finally:
            pff.batch_destroy(b)
    finally:
        close(xs)


def _oracle_serve(w, load_steps, max_newton=12):
    """The oracle's load steps of one served request: p_n = n/N p, phi_old = phi^{n-1},
    phi~ = phi_old (the serving loop does not extrapolate), the previous load step's final active
    set as A_{k-1}, the request's CG seed."""
    m = fem.Mesh(w.dim, w.deg, w.n_cells, w.lo, w.hi, w.cell_mask())
    dmask = fem.dirichlet_face_mask(m, w.dirichlet_faces)
    if w.dirichlet_mask() is not None:
        dmask = dmask | w.dirichlet_mask()
    U, _, _ = W.initial_state(w)
    prev = None
    for n in range(1, load_steps + 1):
        ph = fem.Phys(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=w.pressure * n / load_steps)
        U, infos = pdas.load_step(m, ph, w.n_levels, U, None, dmask, prev, max_newton=max_newton, seed=w.seed,
                                  maxit=200, u_dirichlet=w.u_dirichlet(n / load_steps))
        prev = infos[-1].active
    return U


def test_served_requests_match_oracle():
    crack = W.batch_instances(3, sizes=(16,), seed=11)[1]
    crack.pressure = 2e-2
    lshape = W.config_3d_lshape(16, n_levels=3)              # displacement ramp on the strip, p = 0
    rs = [serve.Request(0, crack, load_steps=2), serve.Request(1, lshape, load_steps=2)]
    srv = serve.Server(serve.PffBackend(), hbm_budget=8 << 30)
    srv.run(rs, realtime=False)
    for r in rs:
        Ug = srv.results[r.rid].U
        Uo = _oracle_serve(r.workload, r.load_steps)
        assert np.linalg.norm(Ug - Uo) <= 1e-6 * np.linalg.norm(Uo), r.rid
