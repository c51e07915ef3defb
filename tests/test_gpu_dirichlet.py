"""Prescribed boundary displacements (pff_set_state / pff_set_dirichlet_values) through the C ABI.

1. Affine patch test on the GPU: phase field clamped to 1 on every node, the displacement prescribed
   as an affine field on the whole boundary, zero inside; two active-set Newton steps must return the
   affine field (the exact discrete solution) to 1e-10 of its size and leave phi untouched.
2. The displacement-driven 3D L-shaped panel (clamped on y = 0, u_y prescribed on a strip of the top
   of the lower arm next to the re-entrant corner, p = 0): the first three steps of its 20-step ramp,
   each solved by Algorithm 1 to its stop test, against the oracle's load steps with the same
   prescribed values (1e-6)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem, pdas  # noqa: E402
from paper_1902_08112_gb300 import pff, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("dim,n,levels,mgp", [(3, 12, 2, 64), (3, 16, 3, 32), (2, 32, 3, 64)])
def test_affine_boundary_values_are_reproduced(dim, n, levels, mgp):
    lo, hi = (0.0,) * dim, tuple(1.0 + 0.25 * a for a in range(dim))
    m = fem.Mesh(dim, 1, (n,) * dim, lo, hi)
    nn = m.n_nodes
    rng = np.random.default_rng(6)
    A, c = 1e-2 * rng.normal(size=(dim, dim)), 1e-2 * rng.normal(size=dim)
    X = m.node_coords()
    ua = np.concatenate([X @ A[k] + c[k] for k in range(dim)])
    faces = (1 << (2 * dim)) - 1
    dmask = np.full(nn, pff.MASK_PHI_DIR, np.uint8)
    prm = pff.default_params(E=2.0, nu=0.25, eps=0.2, pressure=0.3, mg_precision=mgp)
    h = pff.create_hierarchy(pff.make_mesh(dim, 1, (n,) * dim, levels, lo, hi, dirichlet_faces=faces,
                                           dirichlet_mask=dmask), prm)
    try:
        U = t(np.concatenate([np.zeros(dim * nn), np.ones(nn)]))
        ones = t(np.ones(nn))
        pff.set_state(h, U, ones, ones, t(ua))
        info = pff.newton_step(h, U)
        assert info.n_active == 0
        pff.newton_step(h, U)
        torch.cuda.synchronize()
        Ug = U.cpu().numpy()
        assert np.abs(Ug[:dim * nn] - ua).max() <= 1e-10 * np.abs(ua).max()
        np.testing.assert_array_equal(Ug[dim * nn:], np.ones(nn))
    finally:
        pff.destroy_hierarchy(h)


def test_lshape_displacement_ramp_matches_oracle():
    w = W.config_3d_lshape(16, n_levels=3)
    steps, ramp = 3, 20
    cm, dm = w.cell_mask(), w.dirichlet_mask()
    prm = pff.default_params(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, pressure=0.0, mg_precision=64)
    h = pff.create_hierarchy(pff.make_mesh(3, 1, w.n_cells, w.n_levels, w.lo, w.hi,
                                           dirichlet_faces=w.dirichlet_faces, cell_mask=cm, dirichlet_mask=dm), prm)
    m = fem.Mesh(3, 1, w.n_cells, w.lo, w.hi, cm)
    dmask = fem.dirichlet_face_mask(m, w.dirichlet_faces) | dm
    ph = fem.Phys(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=0.0)
    try:
        U0, po, pt = W.initial_state(w)
        U = t(U0)
        pff.set_state(h, U, t(po), t(pt), t(w.u_dirichlet(1 / ramp)))
        Uo, prev = U0.copy(), None
        for step in range(1, steps + 1):
            ud = w.u_dirichlet(step / ramp)
            pff.set_dirichlet_values(h, t(ud))
            li = pff.load_step(h, U, None, 0.0, max_newton=12)
            Uo, infos = pdas.load_step(m, ph, w.n_levels, Uo, None, dmask, prev, max_newton=12, maxit=200,
                                       u_dirichlet=ud)
            prev = infos[-1].active
            torch.cuda.synchronize()
            Ug = U.cpu().numpy()
            assert li.newton_steps == len(infos) and bool(li.converged) == infos[-1].converged
            strip = dm != 0
            np.testing.assert_array_equal(Ug[w.n_nodes:2 * w.n_nodes][strip], ud[w.n_nodes:2 * w.n_nodes][strip])
            assert np.linalg.norm(Ug - Uo) <= 1e-6 * np.linalg.norm(Uo), step
            Uo = Ug.copy()          # both sides continue from the GPU iterate
    finally:
        pff.destroy_hierarchy(h)
