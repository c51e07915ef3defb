"""Prescribed (inhomogeneous) boundary displacements in the oracle's Algorithm 1.

Pin against a closed form: with the phase field clamped to 1 everywhere (g(1) = 1, no degradation)
and the displacement prescribed as an affine field on the whole boundary, the discrete solution is
that affine field (Q1 and Q2 reproduce affine fields; the pressure term, constant over the domain,
only acts on boundary rows).  Starting from zero in the interior, one active-set Newton step reaches it
to the linear solver's tolerance and a second one to rounding; phi never moves.  A dropped lift, a lift
of the wrong component or an increment that is not zero on the Dirichlet rows fails these checks."""
import numpy as np
import pytest

from oracle import fem, pdas


def _affine(m, A, c):
    X = m.node_coords()
    return np.concatenate([X @ A[k] + c[k] for k in range(m.dim)])


@pytest.mark.parametrize("dim,deg,n", [(2, 1, 8), (2, 2, 4), (3, 1, 6)])
def test_affine_boundary_values_are_reproduced(dim, deg, n):
    m = fem.Mesh(dim, deg, (n,) * dim, (0.0,) * dim, tuple(1.0 + 0.25 * a for a in range(dim)))
    rng = np.random.default_rng(4)
    A, c = 1e-2 * rng.normal(size=(dim, dim)), 1e-2 * rng.normal(size=dim)
    ua = _affine(m, A, c)
    nn = m.n_nodes
    faces = (1 << (2 * dim)) - 1
    dmask = fem.dirichlet_face_mask(m, faces) | np.uint8(fem.BIT_PHI_DIR)
    ph = fem.Phys(E=2.0, nu=0.25, Gc=1.0, kappa=1e-10, eps=0.2, p=0.3)
    U0 = np.concatenate([np.zeros(dim * nn), np.ones(nn)])
    ones = np.ones(nn)
    U1, info1 = pdas.newton_step(m, ph, 2, U0, ones, ones, dmask, None, u_dirichlet=ua)
    assert info1.active.sum() == 0
    err1 = np.abs(U1[:dim * nn] - ua).max() / np.abs(ua).max()
    assert err1 <= 1e-7
    U2, _ = pdas.newton_step(m, ph, 2, U1, ones, ones, dmask, info1.active, u_dirichlet=ua)
    assert np.abs(U2[:dim * nn] - ua).max() <= 1e-12 * np.abs(ua).max()
    np.testing.assert_array_equal(U2[dim * nn:], ones)
    # without the prescribed values the iterate stays at zero on the boundary and the affine field is
    # not reached
    U1h, _ = pdas.newton_step(m, ph, 2, U0, ones, ones, dmask, None)
    assert np.abs(U1h[:dim * nn] - ua).max() > 1e-3 * np.abs(ua).max()


def test_lift_touches_only_dirichlet_displacements():
    m = fem.Mesh(2, 1, (4, 4), (0.0, 0.0), (1.0, 1.0))
    nn = m.n_nodes
    dmask = np.zeros(nn, np.uint8)
    dmask[[0, 5]] = fem.BIT_U[0]
    dmask[[7]] = fem.BIT_U[1] | fem.BIT_PHI_DIR
    U = np.arange(3 * nn, dtype=np.float64)
    g = -np.ones(3 * nn)
    L = pdas.lift_dirichlet(m, U, dmask, g)
    changed = np.flatnonzero(L != U)
    np.testing.assert_array_equal(changed, [0, 5, nn + 7])
    assert (L[changed] == -1).all()
