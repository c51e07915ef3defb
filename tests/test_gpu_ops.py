"""GPU parity of the level operators, transfers and preconditioner pieces against the oracle.

All calls go through the C ABI (paper_1902_08112_gb300.pff).  Inputs come from the seeded
generators of paper_1902_08112_gb300.workloads; expected values from oracle/ only.

Tolerances: FP64 operators 1e-12 relative (normwise, the required parity); FP32 operators 2e-5
(FP32 unit roundoff 6e-8 times the ~100-term sums of a cell evaluation, with margin); solver
pieces built on the FP64 operators 1e-9 (eigenvalue estimates enter through Chebyshev
coefficients; 10 CG steps amplify rounding).
"""
from dataclasses import replace

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem, multigrid as mg  # noqa: E402
from paper_1902_08112_gb300 import pff, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def t(a, dtype=None):
    x = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        x = x.to(dtype)
    return x.to(DEV)


def rel(a, b):
    a = a.detach().cpu().numpy().astype(np.float64) if hasattr(a, "cpu") else np.asarray(a, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def block_errors(a, b, dim):
    """Per block (displacement, phase field) of a component-blocked vector: the normwise relative
    error and the largest entry error relative to the block's largest reference entry, so that an
    error confined to the smaller block is not hidden by the larger one."""
    a = a.detach().cpu().numpy().astype(np.float64) if hasattr(a, "cpu") else np.asarray(a, np.float64)
    nn = b.size // (dim + 1)
    out = []
    for blk in (slice(0, dim * nn), slice(dim * nn, None)):
        d, r = a[blk] - b[blk], b[blk]
        sc = np.abs(r).max()
        nr = np.linalg.norm(r)
        out.append((np.linalg.norm(d) / (nr if nr > 0 else 1.0), np.abs(d).max() / (sc if sc > 0 else 1.0)))
    return out


def assert_blocks(a, b, dim, tol_norm, tol_elem, what=""):
    for k, (en, ee) in enumerate(block_errors(a, b, dim)):
        assert en <= tol_norm and ee <= tol_elem, (what, "u" if k == 0 else "phi", en, ee)


class Case:
    """A hierarchy on the GPU and the oracle's levels for the same inputs."""

    def __init__(self, w, active_fraction=0.1, mg_precision=64, state="random", f=1.0, variant=0, modulus=False,
                 split=0, coarse_phi_max=0):
        self.w = w
        if state == "random":
            U, po, pt = W.random_state(w)
        else:
            U, po, pt = W.initial_state(w, displacement="smooth")
        self.U, self.po, self.pt = U, po, pt
        self.prm = pff.default_params(eps=w.eps, pressure=w.pressure, kappa=w.kappa, E=w.E, nu=w.nu,
                                      Gc=w.Gc, mg_precision=mg_precision, phi_elastic_factor=f, split=split,
                                      coarse_phi_max=coarse_phi_max)
        cm = w.cell_mask()
        self.h = pff.create_hierarchy(pff.make_mesh(w.dim, w.deg, w.n_cells, w.n_levels, w.lo, w.hi,
                                                    dirichlet_faces=w.dirichlet_faces, cell_mask=cm), self.prm)
        pff.set_kernel_variant(self.h, variant)
        es = W.modulus_field(w) if modulus else None
        if modulus:
            pff.set_modulus(self.h, t(es))
        pff.set_state(self.h, t(U), t(po), t(pt))
        act = W.random_active(w, active_fraction) if active_fraction > 0 else np.zeros(w.n_nodes, np.uint8)
        pff.set_active_set(self.h, t(act))
        self.mesh = fem.Mesh(w.dim, w.deg, w.n_cells, w.lo, w.hi, cm)
        self.phys = fem.Phys(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=w.pressure, f=f, escale=es,
                             split=split)
        self.mask = fem.dirichlet_face_mask(self.mesh, w.dirichlet_faces) | (act * fem.BIT_ACTIVE).astype(np.uint8)
        self.levels = mg.build_levels(self.mesh, w.n_levels, self.phys, U, pt, self.mask,
                                      coarse_phi_max=bool(coarse_phi_max))

    def close(self):
        pff.destroy_hierarchy(self.h)


def _aniso(dim, deg, cells, levels):
    """Cells with a different edge length per axis (0.25, 1/6, 0.3125 at the finest level), an
    off-centre box and a crack inside it."""
    w = W.Workload("aniso", dim, deg, tuple(cells[:dim]), levels, (-2.0, -1.0, -0.5)[:dim], (3.0, 1.0, 2.0)[:dim])
    w.cracks = [W.Crack((0.5, 0.0, 0.5)[:dim], (0.0, 0.0, 1.0)[:dim] if dim == 3 else (0.0, 1.0), 0.8)]
    return w.finalize()


# (workload, kernel variant): 0 = Q1 fast path (df64 / FP32 with stored linearisation data),
# 1 = generic kernels, 2 = one thread per Gauss point, 3 = one thread per cell, 5 = Gauss-point
# lanes adding to y with global atomics, 6 = FP64 per cell with shared-memory derivatives, 7 = the
# same per-cell form for the FP32 operators.  Sizes span several tiles with ragged edges.
CASES = {
    "2d_q1": (lambda: W.small(W.config_2d_single_crack(), 40, 3), 0),
    "2d_q1_generic": (lambda: W.small(W.config_2d_single_crack(), 24, 3), 1),
    "2d_q2": (lambda: W.small(W.config_2d_single_crack(deg=2), 12, 2), 1),
    "3d_q1": (lambda: W.small(W.config_3d_penny(), 20, 3), 0),
    "3d_q1_generic": (lambda: W.small(W.config_3d_penny(), 12, 2), 1),
    "3d_q1_lanes": (lambda: W.small(W.config_3d_penny(), 12, 2), 2),
    "3d_q1_percell": (lambda: W.small(W.config_3d_penny(), 12, 2), 3),
    "2d_q1_lanes": (lambda: W.small(W.config_2d_single_crack(), 24, 2), 2),
    "2d_q1_percell": (lambda: W.small(W.config_2d_single_crack(), 24, 2), 3),
    "3d_q2": (lambda: W.small(W.config_3d_penny(deg=2), 6, 2), 1),
    "3d_q1_direct": (lambda: W.small(W.config_3d_penny(), 12, 2), 5),
    "3d_q1_cell64": (lambda: W.small(W.config_3d_penny(), 20, 3), 6),
    "3d_q1_cell64_modulus": (lambda: W.small(W.config_3d_penny(), 12, 2), 6, True),
    "3d_q1_cell64_lshape": (lambda: W.small(W.config_3d_lshape(), (20, 20, 6), 2), 6),
    "3d_q1_cell32": (lambda: W.small(W.config_3d_penny(), 20, 3), 7),
    "2d_q1_direct": (lambda: W.small(W.config_2d_single_crack(), 24, 2), 5),
    # spatially varying modulus (per-cell factor from a smooth seeded field)
    "3d_q1_modulus": (lambda: W.small(W.config_3d_penny(), 20, 3), 0, True),
    "3d_q1_lanes_modulus": (lambda: W.small(W.config_3d_penny(), 12, 2), 2, True),
    "2d_q2_modulus": (lambda: W.small(W.config_2d_single_crack(deg=2), 12, 2), 1, True),
    # Miehe split (Q1: Gauss-point tangent data; variant 1 and Q2: generic kernels); random states
    # mix tension and compression
    "3d_q1_split": (lambda: W.small(W.config_3d_penny(), 12, 2), 0, False, 1),
    "3d_q1_split_generic": (lambda: W.small(W.config_3d_penny(), 12, 2), 1, False, 1),
    "2d_q1_split": (lambda: W.small(W.config_2d_single_crack(), 24, 2), 0, False, 1),
    "3d_q2_split": (lambda: W.small(W.config_3d_penny(deg=2), 6, 2), 1, False, 1),
    # L-shaped domains (cell masks): fast path, lanes, generic Q2
    "3d_q1_lshape": (lambda: W.small(W.config_3d_lshape(), (16, 16, 4), 2), 0),
    "2d_q1_lshape": (lambda: W.small(W.config_2d_lshape(), 24, 3), 0),
    "3d_q1_lshape_lanes": (lambda: W.small(W.config_3d_lshape(), (16, 16, 4), 2), 2),
    "2d_q2_lshape": (lambda: W.small(W.config_2d_lshape(deg=2), 12, 2), 1),
    # 3D Q2 fast path (warp per cell, sum-factorised stages by shuffles, stored Gauss-point data)
    "3d_q2_fast": (lambda: W.small(W.config_3d_penny(deg=2), 12, 3), 0),
    "3d_q2_fast_modulus": (lambda: W.small(W.config_3d_penny(deg=2), 8, 2), 0, True),
    "3d_q2_fast_lshape": (lambda: W.small(W.config_3d_lshape(deg=2), (8, 8, 4), 2), 0),
    # anisotropic cells (a per-axis length taken from the wrong axis fails these)
    "3d_q1_aniso": (lambda: _aniso(3, 1, (20, 12, 8), 2), 0),
    "3d_q1_cell64_aniso": (lambda: _aniso(3, 1, (20, 12, 8), 2), 6),
    "3d_q1_cell32_aniso": (lambda: _aniso(3, 1, (20, 12, 8), 2), 7),
    "3d_q1_generic_aniso": (lambda: _aniso(3, 1, (8, 4, 4), 2), 1),
    "3d_q1_lanes_aniso": (lambda: _aniso(3, 1, (8, 4, 4), 2), 2),
    "3d_q2_aniso": (lambda: _aniso(3, 2, (8, 4, 4), 2), 0),
    "2d_q1_aniso": (lambda: _aniso(2, 1, (20, 12), 2), 0),
    "2d_q2_aniso": (lambda: _aniso(2, 2, (8, 4), 2), 1),
    # degenerate cases: one level with odd cell counts, no Dirichlet face, every phi DoF active, none
    "3d_q1_one_level": (lambda: W.small(W.config_3d_penny(), (5, 3, 7), 1), 0),
    "3d_q1_cell64_one_level": (lambda: W.small(W.config_3d_penny(), (17, 5, 3), 1), 6),
    "3d_q1_no_dirichlet": (lambda: replace(W.small(W.config_3d_penny(), 8, 2), dirichlet_faces=0), 0),
    "3d_q1_all_active": (lambda: W.small(W.config_3d_penny(), 8, 2), 0, False, 0, 1.0),
    "3d_q1_none_active": (lambda: W.small(W.config_3d_penny(), 8, 2), 6, False, 0, 0.0),
    "3d_q2_all_active": (lambda: W.small(W.config_3d_penny(deg=2), 4, 2), 0, False, 0, 1.0),
    # phi~ on the coarse Q1 levels as the neighbourhood maximum (option coarse_phi_max)
    "3d_q1_phi_max": (lambda: W.small(W.config_3d_penny(), 12, 3), 0, False, 0, 0.1, 1),
    "2d_q1_phi_max": (lambda: W.small(W.config_2d_single_crack(), 24, 3), 0, False, 0, 0.1, 1),
    # SI units (steel in a 1 cm box): coefficients over ~30 decades, inside the float exponent range
    # that the double-float operators inherit
    "3d_q1_si_units": (lambda: W.config_3d_penny_si(12, 1, 2), 0),
    "3d_q1_cell64_si_units": (lambda: W.config_3d_penny_si(12, 1, 2), 6),
    "3d_q1_generic_si_units": (lambda: W.config_3d_penny_si(8, 1, 2), 1),
    "3d_q2_si_units": (lambda: W.config_3d_penny_si(6, 2, 2), 0),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    make_w, variant, *rest = CASES[request.param]
    c = Case(make_w(), variant=variant, modulus=bool(rest and rest[0]), split=rest[1] if len(rest) > 1 else 0,
             active_fraction=rest[2] if len(rest) > 2 else 0.1, coarse_phi_max=rest[3] if len(rest) > 3 else 0)
    yield c
    c.close()


def test_level_state_restriction_exact(case):
    for l, lev in enumerate(case.levels):
        n = lev.mesh.n_nodes
        U = torch.empty(lev.mesh.n_dofs, dtype=torch.float64, device=DEV)
        pt = torch.empty(n, dtype=torch.float64, device=DEV)
        m = torch.empty(n, dtype=torch.uint8, device=DEV)
        pff.level_state(case.h, l, U, pt, m)
        np.testing.assert_array_equal(U.cpu().numpy(), lev.U)
        np.testing.assert_array_equal(pt.cpu().numpy(), lev.ptil)
        np.testing.assert_array_equal(m.cpu().numpy(), lev.mask)


def test_apply_fp64_matches_assembled_product(case):
    for l, lev in enumerate(case.levels):
        x = W.random_vector(lev.mesh.n_dofs, 100 + l)
        y = torch.empty(lev.mesh.n_dofs, dtype=torch.float64, device=DEV)
        pff.apply_jacobian(case.h, l, t(x), y)
        ref = lev.G @ x
        assert rel(y, ref) <= 1e-12, (l, rel(y, ref))
        assert_blocks(y, ref, case.w.dim, 1e-12, 1e-12, l)


def test_apply_fp32_matches_assembled_product(case):
    for l, lev in enumerate(case.levels):
        x = W.random_vector(lev.mesh.n_dofs, 200 + l).astype(np.float32)
        y = torch.empty(lev.mesh.n_dofs, dtype=torch.float32, device=DEV)
        pff.apply_jacobian_f32(case.h, l, t(x), y)
        ref = lev.G @ x.astype(np.float64)
        assert rel(y, ref) <= 2e-5, (l, rel(y, ref))
        assert_blocks(y, ref, case.w.dim, 2e-5, 1e-4, l)


def test_eliminated_rows_are_identity(case):
    lev = case.levels[-1]
    x = W.random_vector(lev.mesh.n_dofs, 300)
    y = torch.empty(lev.mesh.n_dofs, dtype=torch.float64, device=DEV)
    pff.apply_jacobian(case.h, -1, t(x), y)
    cons = ~lev.free
    np.testing.assert_array_equal(y.cpu().numpy()[cons], x[cons])


def test_residual_matches_oracle(case):
    R = torch.empty(case.mesh.n_dofs, dtype=torch.float64, device=DEV)
    pff.residual(case.h, R)
    ref = -fem.residual_A(case.mesh, case.phys, case.U, case.pt)
    assert rel(R, ref) <= 1e-12
    assert_blocks(R, ref, case.w.dim, 1e-12, 1e-12)


def test_diagonal_matches_oracle(case):
    for l, lev in enumerate(case.levels):
        d = torch.empty(lev.mesh.n_dofs, dtype=torch.float64, device=DEV)
        pff.diagonal(case.h, l, 64, d)
        assert rel(d, lev.G.diagonal()) <= 1e-12
        assert_blocks(d, lev.G.diagonal(), case.w.dim, 1e-12, 1e-12, l)


def test_transfers_match_oracle(case):
    for l in range(1, len(case.levels)):
        f, c = case.levels[l], case.levels[l - 1]
        r = W.random_vector(f.mesh.n_dofs, 400 + l)
        rc = torch.empty(c.mesh.n_dofs, dtype=torch.float64, device=DEV)
        pff.restrict(case.h, l, 64, t(r), rc)
        ref = f.P.T @ r
        ref[~c.free] = 0.0
        assert rel(rc, ref) <= 1e-14
        e = W.random_vector(c.mesh.n_dofs, 500 + l)
        x0 = W.random_vector(f.mesh.n_dofs, 600 + l)
        xf = t(x0.copy())
        pff.prolongate_add(case.h, l, 64, t(e), xf)
        corr = f.P @ e
        corr[~f.free] = 0.0
        assert rel(xf, x0 + corr) <= 1e-14


# (kernel variant, split): the Q1 fast path, the generic kernels, the Miehe split, the per-cell
# FP64-accurate apply
@pytest.fixture(scope="module", params=[(0, 0), (1, 0), (0, 1), (6, 0)], ids=["fast", "generic", "split", "cell64"])
def solver_case(request):
    variant, split = request.param
    c = Case(W.small(W.config_3d_penny(), 8, 2), active_fraction=0.05, state="initial", variant=variant,
             split=split)
    mg.estimate_levels(c.levels, 12345, 10)
    yield c
    c.close()


def test_eigen_estimates_match_oracle(solver_case):
    c = solver_case
    for l, lev in enumerate(c.levels):
        lm = pff.eigen_estimates(c.h, l)
        np.testing.assert_allclose(lm, [lev.lam_min[0], lev.lam_max[0], lev.lam_min[1], lev.lam_max[1]], rtol=1e-9)


def test_smoother_matches_oracle(solver_case):
    c = solver_case
    prm = mg.MGParams()
    for l, lev in enumerate(c.levels):
        b = np.where(lev.free, W.random_vector(lev.mesh.n_dofs, 700 + l), 0.0)
        x = torch.zeros(lev.mesh.n_dofs, dtype=torch.float64, device=DEV)
        pff.smooth(c.h, l, 64, t(b), x, True)
        ref = mg.smooth_zero(lev, b, prm)
        assert rel(x, ref) <= 1e-9
        # with an initial guess: x0 + S(b - G x0)
        x0 = np.where(lev.free, W.random_vector(lev.mesh.n_dofs, 800 + l), 0.0)
        xg = t(x0.copy())
        pff.smooth(c.h, l, 64, t(b), xg, False)
        ref = x0 + mg.smooth_zero(lev, b - lev.G @ x0, prm)
        assert rel(xg, ref) <= 1e-9


def test_coarse_solve_matches_oracle(solver_case):
    c = solver_case
    lev = c.levels[0]
    b = np.where(lev.free, W.random_vector(lev.mesh.n_dofs, 900), 0.0)
    x = torch.zeros(lev.mesh.n_dofs, dtype=torch.float64, device=DEV)
    pff.coarse_solve(c.h, t(b), x)
    ref = mg.coarse_solve(lev, b, mg.MGParams())
    assert rel(x, ref) <= 1e-9


def test_vcycle_fp64_matches_oracle(solver_case):
    c = solver_case
    v = W.random_vector(c.mesh.n_dofs, 1000)
    z = torch.zeros(c.mesh.n_dofs, dtype=torch.float64, device=DEV)
    pff.vcycle(c.h, t(v), z)
    ref = mg.precondition(c.levels, v, mg.MGParams())
    assert rel(z, ref) <= 1e-9


def test_block_diagonal_vcycle_matches_oracle(solver_case):
    """P_diag (Sec. 3.3): FP64 V-cycle and coarse solve without the coupling block."""
    c = solver_case
    prm = mg.MGParams(block_diagonal=True)
    pd = pff.default_params(eps=c.w.eps, pressure=c.w.pressure, kappa=c.w.kappa, E=c.w.E, nu=c.w.nu,
                            Gc=c.w.Gc, mg_precision=64, preconditioner=pff.PRECOND_DIAG, split=c.prm.split)
    pff.set_params(c.h, pd)
    try:
        lev = c.levels[0]
        b = np.where(lev.free, W.random_vector(lev.mesh.n_dofs, 901), 0.0)
        x = torch.zeros(lev.mesh.n_dofs, dtype=torch.float64, device=DEV)
        pff.coarse_solve(c.h, t(b), x)
        assert rel(x, mg.coarse_solve(lev, b, prm)) <= 1e-9
        v = W.random_vector(c.mesh.n_dofs, 1001)
        z = torch.zeros(c.mesh.n_dofs, dtype=torch.float64, device=DEV)
        pff.vcycle(c.h, t(v), z)
        assert rel(z, mg.precondition(c.levels, v, prm)) <= 1e-9
    finally:
        pff.set_params(c.h, c.prm)


@pytest.mark.parametrize("n,levels", [(16, 3), (24, 3)])
def test_vcycle_fp32_against_fp64_oracle(n, levels):
    """The FP32 V-cycle (levels, smoother and transfers in FP32 with FP32 accumulation, FP64 coarse
    solve) against the oracle's all-FP64 V-cycle: the error it makes as a preconditioner, per block.
    Measured on GB300: below 1e-6 relative; the bound 1e-5 allows FP32 rounding (6e-8) amplified by
    the smoother's Chebyshev polynomials on every level."""
    c = Case(W.small(W.config_3d_penny(), n, levels), active_fraction=0.05, state="initial", mg_precision=32)
    try:
        mg.estimate_levels(c.levels, 12345, 10)
        v = W.random_vector(c.mesh.n_dofs, 1002)
        z = torch.zeros(c.mesh.n_dofs, dtype=torch.float64, device=DEV)
        pff.vcycle(c.h, t(v), z)
        ref = mg.precondition(c.levels, v, mg.MGParams())
        errs = block_errors(z, ref, 3)
        print(f"FP32 V-cycle vs FP64 oracle ({n}^3, {levels} levels): u {errs[0][0]:.2e}, phi {errs[1][0]:.2e}")
        assert rel(z, ref) <= 1e-5
        for en, _ in errs:
            assert en <= 1e-5
    finally:
        c.close()
