"""Pins of the oracle's FE layer against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms (patch test,
tractions of affine fields, energies of constant states), finite differences of an
independently written energy, the paper's Lame table, and structural facts of the method
(G_uphi = 0, symmetry of G_uu, elimination pattern).
"""
import math
import os

import numpy as np
import pytest

from oracle import fem
from paper_1902_08112_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _mesh(dim, deg, n, lo=-1.0, hi=1.0):
    return fem.Mesh(dim, deg, (n,) * dim, (lo,) * dim, (hi,) * dim)


def _affine_u(mesh, A, b=None):
    X = mesh.node_coords()
    u = X @ np.asarray(A).T
    if b is not None:
        u = u + np.asarray(b)[None, :]
    return np.concatenate([u[:, c] for c in range(mesh.dim)])


def test_lame_matches_paper_table():
    """Sec. 5.1 parameter table: mu, lambda derived from E and nu (3D formulas)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "lame_table.txt")) if not l.startswith("#")]
    for E, nu, mu_t, lam_t in (map(float, r) for r in rows):
        mu, lam = fem.lame(E, nu)
        assert math.floor(mu * 10) / 10 == pytest.approx(mu_t)
        assert math.floor(lam * 10) / 10 == pytest.approx(lam_t)


@pytest.mark.parametrize("dim,deg", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_lumped_mass_sums_to_volume(dim, deg):
    m = fem.Mesh(dim, deg, (3,) * dim, (0.0,) * dim, tuple(1.0 + 0.5 * a for a in range(dim)))
    M = fem.lumped_mass(m)
    vol = np.prod([1.0 + 0.5 * a for a in range(dim)])
    assert M.sum() == pytest.approx(vol, rel=1e-14)
    assert (M > 0).all()


@pytest.mark.parametrize("dim,deg", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_patch_test_affine_displacement(dim, deg):
    """phi = phi~ = 1 and an affine u: sigma is constant, so the u-rows of A vanish at every
    interior node (Q1 and Q2 reproduce affine fields exactly)."""
    m = _mesh(dim, deg, 3)
    rng = np.random.default_rng(1)
    u = _affine_u(m, rng.normal(size=(dim, dim)), rng.normal(size=dim))
    U = np.concatenate([u, np.ones(m.n_nodes)])
    ph = fem.Phys(E=3.0, nu=0.3, p=0.7, eps=0.5)
    A = fem.residual_A(m, ph, U, np.ones(m.n_nodes))
    interior = fem.dirichlet_face_mask(m, 0x3F) == 0
    for c in range(dim):
        Ac = A[c * m.n_nodes:(c + 1) * m.n_nodes]
        assert np.abs(Ac[interior]).max() < 1e-12


@pytest.mark.parametrize("dim,deg", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_face_tractions_of_affine_fields(dim, deg):
    """Sum of the u-residual over the nodes of a face equals the traction sigma.n integrated over
    the face (sigma constant): uniaxial u=(g x,0,..) gives sigma_xx=(lambda+2mu) g,
    sigma_yy = lambda g; shear u=(g y,0,..) gives sigma_xy = mu g."""
    m = fem.Mesh(dim, deg, (2,) * dim, (0.0,) * dim, tuple(1.0 + 0.25 * a for a in range(dim)))
    E, nu, g = 2.0, 0.25, 1e-2
    ph = fem.Phys(E=E, nu=nu, p=0.0, eps=1.0)
    mu, lam = fem.lame(E, nu)
    L = [1.0 + 0.25 * a for a in range(dim)]
    X = m.node_coords()
    nn = m.n_nodes

    def face_area(axis):
        return np.prod([L[a] for a in range(dim) if a != axis])

    def face_nodes(axis):
        return np.isclose(X[:, axis], L[axis])

    ones = np.ones(nn)
    A1 = np.zeros((dim, dim)); A1[0, 0] = g
    U = np.concatenate([_affine_u(m, A1), ones])
    R = fem.residual_A(m, ph, U, ones)
    assert R[0 * nn:1 * nn][face_nodes(0)].sum() == pytest.approx((lam + 2 * mu) * g * face_area(0), rel=1e-12)
    assert R[1 * nn:2 * nn][face_nodes(1)].sum() == pytest.approx(lam * g * face_area(1), rel=1e-12)
    A2 = np.zeros((dim, dim)); A2[0, 1] = g
    U = np.concatenate([_affine_u(m, A2), ones])
    R = fem.residual_A(m, ph, U, ones)
    assert R[0 * nn:1 * nn][face_nodes(1)].sum() == pytest.approx(mu * g * face_area(1), rel=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_energy_of_constant_states(dim):
    """Energy closed forms: affine u with phi=1 gives (E_s + p tr e)|D|; u=0 with constant phi=c
    gives (g(c)*0 + Gc/2 (1-c)^2/eps)|D|."""
    m = _mesh(dim, 1, 2, 0.0, 2.0)
    vol = 2.0 ** dim
    ph = fem.Phys(E=1.5, nu=0.2, p=0.3, eps=0.4, Gc=2.0)
    mu, lam = fem.lame(1.5, 0.2)
    A = np.zeros((dim, dim)); A[0, 0] = 0.01; A[0, 1] = 0.02
    U = np.concatenate([_affine_u(m, A), np.ones(m.n_nodes)])
    e = 0.5 * (A + A.T)
    Es = 0.5 * lam * np.trace(e) ** 2 + mu * np.sum(e * e)
    assert fem.energy(m, ph, U) == pytest.approx((Es + ph.p * np.trace(A)) * vol, rel=1e-13)
    c = 0.3
    U = np.concatenate([np.zeros(dim * m.n_nodes), np.full(m.n_nodes, c)])
    assert fem.energy(m, ph, U) == pytest.approx(0.5 * ph.Gc * (1 - c) ** 2 / ph.eps * vol, rel=1e-13)


def _rand_state(m, seed):
    rng = np.random.default_rng(seed)
    u = 0.05 * rng.standard_normal(m.dim * m.n_nodes)
    phi = rng.uniform(0.1, 1.0, m.n_nodes)
    return np.concatenate([u, phi])


@pytest.mark.parametrize("dim,deg", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_residual_is_energy_gradient(dim, deg):
    """A(U) = dE/dU when phi~ = phi and f = 1 (central differences of the energy, O(delta^2))."""
    m = _mesh(dim, deg, 2)
    ph = fem.Phys(E=1.0, nu=0.2, p=0.05, eps=0.3, Gc=1.0, kappa=1e-3)
    U = _rand_state(m, 3)
    phi = U[dim * m.n_nodes:]
    A = fem.residual_A(m, ph, U, phi)
    rng = np.random.default_rng(4)
    for _ in range(3):
        v = rng.standard_normal(U.size)
        dlt = 1e-5
        fd = (fem.energy(m, ph, U + dlt * v) - fem.energy(m, ph, U - dlt * v)) / (2 * dlt)
        assert fd == pytest.approx(A @ v, rel=1e-7)


@pytest.mark.parametrize("dim,deg", [(2, 1), (2, 2), (3, 1), (3, 2)])
@pytest.mark.parametrize("f", [1.0, 0.5])
def test_jacobian_is_residual_derivative(dim, deg, f):
    """G v = d/dt A(U + t v) at t=0 with phi~ frozen (central differences), all blocks."""
    m = _mesh(dim, deg, 2)
    ph = fem.Phys(E=1.0, nu=0.2, p=0.05, eps=0.3, Gc=1.0, kappa=1e-3, f=f)
    U = _rand_state(m, 5)
    ptil = np.random.default_rng(6).uniform(0, 1, m.n_nodes)
    G = fem.assemble(m, ph, U, ptil, np.zeros(m.n_nodes, np.uint8))
    rng = np.random.default_rng(7)
    for _ in range(3):
        v = rng.standard_normal(U.size)
        dlt = 1e-6
        fd = (fem.residual_A(m, ph, U + dlt * v, ptil) - fem.residual_A(m, ph, U - dlt * v, ptil)) / (2 * dlt)
        Gv = G @ v
        assert np.linalg.norm(fd - Gv) <= 1e-7 * np.linalg.norm(Gv)


def _aniso_mesh(dim, deg):
    """Cells of three different edge lengths (0.6, 2/3, 0.35) on an off-centre box."""
    return fem.Mesh(dim, deg, (2, 3, 2)[:dim], (-0.5, 0.0, 0.2)[:dim], (0.7, 2.0, 0.9)[:dim])


@pytest.mark.parametrize("dim,deg", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_anisotropic_cells(dim, deg):
    """On cells with a different edge length per axis: the energy of an affine u with phi = 1 is
    (E_s + p tr e)|D|, the residual is the energy's gradient and the Jacobian the residual's derivative
    (central differences), and the u-rows of an affine field vanish at interior nodes.  A per-axis
    length taken from the wrong axis (in a derivative, a Gauss weight or a lumped mass) breaks one of
    them."""
    m = _aniso_mesh(dim, deg)
    vol = np.prod([(0.7, 2.0, 0.9)[a] - (-0.5, 0.0, 0.2)[a] for a in range(dim)])
    ph = fem.Phys(E=1.5, nu=0.2, p=0.3, eps=0.4, Gc=2.0, kappa=1e-3)
    mu, lam = fem.lame(1.5, 0.2)
    rng = np.random.default_rng(21)
    A = 0.01 * rng.normal(size=(dim, dim))
    U = np.concatenate([_affine_u(m, A, rng.normal(size=dim)), np.ones(m.n_nodes)])
    e = 0.5 * (A + A.T)
    Es = 0.5 * lam * np.trace(e) ** 2 + mu * np.sum(e * e)
    assert fem.energy(m, ph, U) == pytest.approx((Es + ph.p * np.trace(A)) * vol, rel=1e-12)
    Ares = fem.residual_A(m, ph, U, np.ones(m.n_nodes))
    interior = fem.dirichlet_face_mask(m, 0x3F) == 0
    if interior.any():
        for c in range(dim):
            assert np.abs(Ares[c * m.n_nodes:(c + 1) * m.n_nodes][interior]).max() < 1e-12
    assert fem.lumped_mass(m).sum() == pytest.approx(vol, rel=1e-14)
    U = _rand_state(m, 22)
    phi = U[dim * m.n_nodes:]
    R = fem.residual_A(m, ph, U, phi)
    for _ in range(2):
        v = rng.standard_normal(U.size)
        fd = (fem.energy(m, ph, U + 1e-5 * v) - fem.energy(m, ph, U - 1e-5 * v)) / 2e-5
        assert fd == pytest.approx(R @ v, rel=1e-7)
    ptil = rng.uniform(0, 1, m.n_nodes)
    G = fem.assemble(m, ph, U, ptil, np.zeros(m.n_nodes, np.uint8))
    for _ in range(2):
        v = rng.standard_normal(U.size)
        fd = (fem.residual_A(m, ph, U + 1e-6 * v, ptil) - fem.residual_A(m, ph, U - 1e-6 * v, ptil)) / 2e-6
        Gv = G @ v
        assert np.linalg.norm(fd - Gv) <= 1e-7 * np.linalg.norm(Gv)


@pytest.mark.parametrize("dim,deg", [(2, 1), (3, 1), (3, 2)])
def test_block_structure(dim, deg):
    """G_uphi = 0 exactly (phi~ frozen in the u-equation, Sec. 3.3) and G_uu symmetric."""
    m = _mesh(dim, deg, 2)
    ph = fem.Phys(E=1.0, nu=0.3, p=0.1, eps=0.3, kappa=1e-4)
    U = _rand_state(m, 8)
    ptil = np.random.default_rng(9).uniform(0, 1, m.n_nodes)
    mask = fem.dirichlet_face_mask(m, 0x3F)
    G = fem.assemble(m, ph, U, ptil, mask).toarray()
    nu_ = dim * m.n_nodes
    assert np.count_nonzero(G[:nu_, nu_:]) == 0
    Guu = G[:nu_, :nu_]
    assert np.abs(Guu - Guu.T).max() <= 1e-14 * np.abs(Guu).max()


def test_elimination_pattern():
    """Constrained rows are identity rows, constrained columns are zero (Algorithm 1, step 4)."""
    w = W.small(W.config_2d_single_crack(), 4, 1)
    m = fem.Mesh(w.dim, w.deg, w.n_cells, w.lo, w.hi)
    ph = fem.Phys(eps=w.eps, p=w.pressure)
    U, _, pt = W.random_state(w)
    mask = fem.dirichlet_face_mask(m, 0x3F) | (W.random_active(w, 0.3) * fem.BIT_ACTIVE).astype(np.uint8)
    G = fem.assemble(m, ph, U, pt, mask).toarray()
    Gfull = fem.assemble(m, ph, U, pt, np.zeros_like(mask)).toarray()
    cons = fem.constrained_dofs(m, mask)
    assert cons.sum() > 0
    np.testing.assert_array_equal(G[cons], np.eye(G.shape[0])[cons])
    assert np.count_nonzero(G[np.ix_(~cons, cons)]) == 0
    np.testing.assert_array_equal(G[np.ix_(~cons, ~cons)], Gfull[np.ix_(~cons, ~cons)])


@pytest.mark.parametrize("dim,deg", [(2, 2), (3, 1)])
def test_row_sampler_matches_assembly(dim, deg):
    m = _mesh(dim, deg, 3)
    ph = fem.Phys(E=1.0, nu=0.2, p=0.02, eps=0.5, kappa=1e-6)
    U = _rand_state(m, 10)
    ptil = U[dim * m.n_nodes:]
    mask = fem.dirichlet_face_mask(m, 0x3F)
    mask[::7] |= fem.BIT_ACTIVE
    G = fem.assemble(m, ph, U, ptil, mask)
    x = np.random.default_rng(11).standard_normal(m.n_dofs)
    rows = np.arange(0, m.n_dofs, 5)
    np.testing.assert_allclose(fem.apply_rows(m, ph, U, ptil, mask, x, rows), (G @ x)[rows],
                               rtol=1e-13, atol=1e-13 * np.abs(G @ x).max())


@pytest.mark.parametrize("dim,deg", [(2, 1), (3, 1), (3, 2)])
def test_energy_parts_add_up_and_match_closed_forms(dim, deg):
    """Bulk + crack = total energy; crack energy of a constant phase field c is
    Gc/2 (1-c)^2/eps |D| and its bulk energy is 0 for u = 0 (Sec. 5 energies)."""
    m = _mesh(dim, deg, 2)
    ph = fem.Phys(E=1.3, nu=0.25, p=0.2, eps=0.4, Gc=1.7, kappa=1e-3)
    U = _rand_state(m, 12)
    b, c = fem.energy_parts(m, ph, U)
    assert b + c == pytest.approx(fem.energy(m, ph, U), rel=1e-13)
    cval = 0.4
    U0 = np.concatenate([np.zeros(dim * m.n_nodes), np.full(m.n_nodes, cval)])
    b0, c0 = fem.energy_parts(m, ph, U0)
    assert b0 == 0.0
    assert c0 == pytest.approx(0.5 * ph.Gc * (1 - cval) ** 2 / ph.eps * 2.0 ** dim, rel=1e-13)


@pytest.mark.parametrize("dim,deg", [(2, 1), (3, 1), (3, 2)])
def test_boundary_load_of_affine_field(dim, deg):
    """L_c of Sec. 5 for u = diag(a) x (no shear) with constant phi~ = c: the effective stress on a
    face is g(c) sigma + c^2 p I, so the upper face of axis y carries (g(c) sigma_yy + c^2 p) |face|
    and the lower face the negative of it; sigma_yy = 2 mu a_y + lambda tr(a)."""
    L = [1.0 + 0.25 * a for a in range(dim)]
    m = fem.Mesh(dim, deg, (2,) * dim, (0.0,) * dim, tuple(L))
    E, nu, p, kap, c = 2.0, 0.25, 3e-3, 1e-3, 0.5
    ph = fem.Phys(E=E, nu=nu, p=p, eps=1.0, kappa=kap)
    mu, lam = fem.lame(E, nu)
    a = np.array([1e-2, -2e-2, 5e-3][:dim])
    U = np.concatenate([_affine_u(m, np.diag(a)), np.ones(m.n_nodes)])
    ptil = np.full(m.n_nodes, c)
    area = np.prod([L[k] for k in range(dim) if k != 1])
    syy = 2 * mu * a[1] + lam * a.sum()
    want = ((1 - kap) * c * c + kap) * syy + c * c * p
    assert fem.boundary_load(m, ph, U, ptil, 3, 1) == pytest.approx(want * area, rel=1e-12)
    assert fem.boundary_load(m, ph, U, ptil, 2, 1) == pytest.approx(-want * area, rel=1e-12)
    # no shear: the x-component of the load on a y-face vanishes
    assert abs(fem.boundary_load(m, ph, U, ptil, 3, 0)) < 1e-14


@pytest.mark.parametrize("dim,deg", [(2, 1), (3, 1), (2, 2)])
def test_varying_modulus(dim, deg):
    """Per-cell modulus E_K = s_K E: (a) a constant factor s is the same as the modulus s E
    (residual, Jacobian, energy); (b) with a varying factor the residual is still the gradient of
    the energy and the Jacobian the derivative of the residual (central differences); (c) a cell
    whose factor changes alters only the rows of its own nodes."""
    m = _mesh(dim, deg, 2)
    rng = np.random.default_rng(11)
    U = _rand_state(m, 12)
    ptil = rng.uniform(0, 1, m.n_nodes)
    zero = np.zeros(m.n_nodes, np.uint8)
    s = 0.37
    ph_s = fem.Phys(E=1.0, nu=0.2, p=0.05, eps=0.3, kappa=1e-3, escale=np.full(m.n_cells, s))
    ph_e = fem.Phys(E=s, nu=0.2, p=0.05, eps=0.3, kappa=1e-3)
    np.testing.assert_allclose(fem.residual_A(m, ph_s, U, ptil), fem.residual_A(m, ph_e, U, ptil), rtol=1e-13,
                               atol=1e-15)
    Gs = fem.assemble(m, ph_s, U, ptil, zero).toarray()
    Ge = fem.assemble(m, ph_e, U, ptil, zero).toarray()
    assert np.abs(Gs - Ge).max() <= 1e-13 * np.abs(Ge).max()
    assert fem.energy(m, ph_s, U) == pytest.approx(fem.energy(m, ph_e, U), rel=1e-13)

    es = rng.uniform(0.1, 1.0, m.n_cells)
    ph = fem.Phys(E=1.0, nu=0.2, p=0.05, eps=0.3, kappa=1e-3, escale=es)
    phi = U[dim * m.n_nodes:]
    A = fem.residual_A(m, ph, U, phi)
    G = fem.assemble(m, ph, U, ptil, zero)
    for _ in range(2):
        v = rng.standard_normal(U.size)
        fd = (fem.energy(m, ph, U + 1e-5 * v) - fem.energy(m, ph, U - 1e-5 * v)) / 2e-5
        assert fd == pytest.approx(A @ v, rel=1e-7)
        fdj = (fem.residual_A(m, ph, U + 1e-6 * v, ptil) - fem.residual_A(m, ph, U - 1e-6 * v, ptil)) / 2e-6
        assert np.linalg.norm(fdj - G @ v) <= 1e-7 * np.linalg.norm(G @ v)

    es2 = es.copy()
    es2[0] *= 3.0
    dA = fem.residual_A(m, fem.Phys(E=1.0, nu=0.2, p=0.05, eps=0.3, kappa=1e-3, escale=es2), U, ptil) - \
        fem.residual_A(m, fem.Phys(E=1.0, nu=0.2, p=0.05, eps=0.3, kappa=1e-3, escale=es), U, ptil)
    npa = m.nodes_per_axis()
    idx = np.indices(npa[::-1]).reshape(dim, -1)[::-1]
    in_cell0 = np.all(idx <= deg, axis=0)
    touched = np.abs(dA.reshape(dim + 1, -1)).max(axis=0) > 0
    assert touched.any() and not np.any(touched & ~in_cell0)


def test_coarsened_modulus_is_child_mean():
    """The coarse-level factor is the mean of the 2^d children: constants are kept and the
    integral of the factor is preserved."""
    from oracle import multigrid as mg
    m = fem.Mesh(3, 1, (4, 6, 2), (0.0,) * 3, (1.0, 1.5, 0.5))
    es = np.random.default_rng(13).uniform(0.1, 1.0, m.n_cells)
    c = mg.coarsen_cell_field(m, es)
    assert c.size == m.n_cells // 8
    assert c.sum() * 8 == pytest.approx(es.sum(), rel=1e-14)
    assert np.allclose(mg.coarsen_cell_field(m, np.full(m.n_cells, 0.3)), 0.3, rtol=0, atol=1e-16)
    # first coarse cell: children (0..1, 0..1, 0..1)
    e3 = es.reshape(2, 6, 4)
    assert c[0] == pytest.approx(e3[0:2, 0:2, 0:2].mean(), rel=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_miehe_split_closed_forms(dim):
    """Miehe split (Sec. 2.1) on uniform strains with constant phi = c, p = 0: the bulk energy is
    (g(c) E_s^+ + E_s - E_s^+)|D|, with E_s^+ = E_s for volumetric expansion and uniaxial tension,
    E_s^+ = 0 for volumetric compression, and E_s^+ = E_s / 2 for pure shear (eigenvalues +-gamma,
    tr e = 0); a rotated strain has the same E_s^+."""
    m = _mesh(dim, 1, 2, 0.0, 2.0)
    vol = 2.0 ** dim
    kap, c = 1e-3, 0.4
    ph = fem.Phys(E=1.5, nu=0.2, p=0.0, eps=0.4, Gc=0.0, kappa=kap, split=1)
    mu, lam = fem.lame(1.5, 0.2)
    g = (1 - kap) * c * c + kap

    def bulk(A):
        U = np.concatenate([_affine_u(m, A), np.full(m.n_nodes, c)])
        return fem.energy(m, ph, U)

    def Es_of(A):
        e = 0.5 * (A + A.T)
        return 0.5 * lam * np.trace(e) ** 2 + mu * np.sum(e * e)

    eps_ = 0.01
    cases = [(eps_ * np.eye(dim), 1.0), (-eps_ * np.eye(dim), 0.0)]
    A = np.zeros((dim, dim)); A[0, 0] = eps_
    cases.append((A, 1.0))
    A = np.zeros((dim, dim)); A[0, 1] = A[1, 0] = eps_
    cases.append((A, 0.5))
    for A, frac in cases:
        Es = Es_of(A)
        Esp = frac * Es
        assert bulk(A) == pytest.approx((g * Esp + Es - Esp) * vol, rel=1e-12, abs=1e-18)
    # rotation invariance of E_s^+ (and of E_s) for a generic strain
    rng = np.random.default_rng(3)
    S = rng.standard_normal((dim, dim)) * 0.01
    S = 0.5 * (S + S.T)
    Q, _ = np.linalg.qr(rng.standard_normal((dim, dim)))
    assert bulk(Q @ S @ Q.T) == pytest.approx(bulk(S), rel=1e-11)


@pytest.mark.parametrize("dim,deg", [(2, 1), (3, 1), (3, 2)])
def test_miehe_split_derivatives(dim, deg):
    """With the Miehe split the residual is still the energy gradient (phi~ = phi, f = 1) and the
    Jacobian the derivative of the residual (phi~ frozen), by central differences on random states
    with tension and compression at the quadrature points."""
    m = _mesh(dim, deg, 2)
    ph = fem.Phys(E=1.0, nu=0.2, p=0.05, eps=0.3, Gc=1.0, kappa=1e-3, split=1)
    U = _rand_state(m, 31)
    phi = U[dim * m.n_nodes:]
    A = fem.residual_A(m, ph, U, phi)
    rng = np.random.default_rng(32)
    for _ in range(3):
        v = rng.standard_normal(U.size)
        dlt = 1e-6
        fd = (fem.energy(m, ph, U + dlt * v) - fem.energy(m, ph, U - dlt * v)) / (2 * dlt)
        assert fd == pytest.approx(A @ v, rel=1e-6)
    ptil = rng.uniform(0, 1, m.n_nodes)
    G = fem.assemble(m, ph, U, ptil, np.zeros(m.n_nodes, np.uint8))
    for _ in range(3):
        v = rng.standard_normal(U.size)
        dlt = 1e-7
        fd = (fem.residual_A(m, ph, U + dlt * v, ptil) - fem.residual_A(m, ph, U - dlt * v, ptil)) / (2 * dlt)
        Gv = G @ v
        assert np.linalg.norm(fd - Gv) <= 1e-6 * np.linalg.norm(Gv)
    # the split changes the operator: it differs from the unsplit Jacobian
    G0 = fem.assemble(m, fem.Phys(E=1.0, nu=0.2, p=0.05, eps=0.3, Gc=1.0, kappa=1e-3), U, ptil,
                      np.zeros(m.n_nodes, np.uint8))
    assert abs(G - G0).max() > 1e-3 * abs(G0).max()
    # symmetric displacement block
    Guu = G.toarray()[:dim * m.n_nodes, :dim * m.n_nodes]
    assert np.abs(Guu - Guu.T).max() <= 1e-13 * np.abs(Guu).max()


def _lshape_mask(n):
    """cells of [0,2]^2 minus [1,2]^2 on an n x n grid (x fastest)."""
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    return (~((i >= n // 2) & (j >= n // 2))).ravel().astype(np.uint8)


@pytest.mark.parametrize("deg", [1, 2])
def test_cell_mask_matches_union_of_boxes(deg):
    """A cell-masked box (the L-shaped panel [0,2]^2 minus [1,2]^2) gives the residual, Jacobian and
    lumped mass of assembling the two boxes [0,1]x[0,2] and [1,2]x[0,1] separately and adding them
    on the shared nodes; nodes outside the domain get nothing; the lumped mass sums to |L| = 3."""
    n = 4
    m = fem.Mesh(2, deg, (n, n), (0.0, 0.0), (2.0, 2.0), _lshape_mask(n))
    ph = fem.Phys(E=1.3, nu=0.25, p=0.02, eps=0.5, Gc=0.8, kappa=1e-3)
    rng = np.random.default_rng(41)
    U = np.concatenate([0.01 * rng.standard_normal(2 * m.n_nodes), rng.uniform(0.2, 1.0, m.n_nodes)])
    pt = rng.uniform(0.0, 1.0, m.n_nodes)
    A = fem.residual_A(m, ph, U, pt)
    M = fem.lumped_mass(m)
    X = m.node_coords()
    parts = [fem.Mesh(2, deg, (n // 2, n), (0.0, 0.0), (1.0, 2.0)), fem.Mesh(2, deg, (n // 2, n // 2), (1.0, 0.0), (2.0, 1.0))]
    A_ref = np.zeros_like(A)
    M_ref = np.zeros_like(M)
    for b in parts:
        Xb = b.node_coords()
        # global node index of every node of the part
        key = {tuple(np.round(x, 9)): k for k, x in enumerate(X)}
        gidx = np.array([key[tuple(np.round(x, 9))] for x in Xb])
        Ub = np.concatenate([U[c * m.n_nodes + gidx] for c in range(3)])
        Ab = fem.residual_A(b, ph, Ub, pt[gidx])
        for c in range(3):
            np.add.at(A_ref, c * m.n_nodes + gidx, Ab[c * b.n_nodes:(c + 1) * b.n_nodes])
        np.add.at(M_ref, gidx, fem.lumped_mass(b))
    np.testing.assert_allclose(A, A_ref, rtol=0, atol=1e-13 * np.abs(A_ref).max())
    np.testing.assert_allclose(M, M_ref, rtol=0, atol=1e-15)
    assert M.sum() == pytest.approx(3.0, rel=1e-14)
    outside = ~m.node_touches_domain()
    assert outside.sum() > 0 and np.all(M[outside] == 0.0)
    dm = fem.dirichlet_face_mask(m, 0)
    assert np.all(dm[outside] == (fem.BIT_U[0] | fem.BIT_U[1] | fem.BIT_PHI_DIR))
    G = fem.assemble(m, ph, U, pt, dm)
    cons = fem.constrained_dofs(m, dm)
    Gd = G.toarray()
    assert np.array_equal(np.diag(Gd)[cons], np.ones(cons.sum()))


def test_cell_mask_coarsening_and_energy():
    """Coarse cell masks keep a cell whose children are in the domain; the energy of an affine
    field on the L-shape is E_s |L| (phi = 1, p = 0)."""
    n = 8
    m = fem.Mesh(2, 1, (n, n), (0.0, 0.0), (2.0, 2.0), _lshape_mask(n))
    c = m.coarsen()
    np.testing.assert_array_equal(c.cell_mask, _lshape_mask(n // 2))
    ph = fem.Phys(E=2.0, nu=0.3, p=0.0, eps=0.5, Gc=1.0)
    mu, lam = fem.lame(2.0, 0.3)
    Aff = np.array([[0.01, 0.004], [-0.002, 0.006]])
    U = np.concatenate([_affine_u(m, Aff), np.ones(m.n_nodes)])
    e = 0.5 * (Aff + Aff.T)
    Es = 0.5 * lam * np.trace(e) ** 2 + mu * np.sum(e * e)
    assert fem.energy(m, ph, U) == pytest.approx(Es * 3.0, rel=1e-12)
