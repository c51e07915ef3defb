"""pff_apply_jacobian_host: the Jacobian apply with x and y in host memory (copies inside the call,
slab-pipelined on 3D levels served by the per-cell kernel) against the device-buffer apply on the
same state, and at the full 128^3 size against sampled rows of the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem  # noqa: E402
from paper_1902_08112_gb300 import pff, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def level_dofs(w, level):
    f = 1 << (w.n_levels - 1 - (level if level >= 0 else w.n_levels - 1))
    return (w.dim + 1) * int(np.prod([c // f + 1 for c in w.n_cells]))


def make(w):
    U, po, pt = W.initial_state(w, displacement="smooth")
    prm = pff.default_params(eps=w.eps, pressure=w.pressure, kappa=w.kappa, E=w.E, nu=w.nu, Gc=w.Gc)
    h = pff.create_hierarchy(pff.make_mesh(w.dim, w.deg, w.n_cells, w.n_levels, w.lo, w.hi,
                                           dirichlet_faces=w.dirichlet_faces, cell_mask=w.cell_mask()), prm)
    pff.set_state(h, t(U), t(po), t(pt))
    pff.update_active_set(h)
    return h, U, po, pt


# (workload, level): 50^3 (7 slabs, the last one ragged), 48^3 (8 slabs), an L-shaped 3D panel
# (cell mask), a small level and a 2D level (one pass, no slabs)
CASES = {
    "3d_50_slabs": (lambda: W.small(W.config_3d_penny(), 50, 2), -1),
    "3d_48_slabs": (lambda: W.small(W.config_3d_penny(), 48, 3), -1),
    "3d_lshape_slabs": (lambda: W.small(W.config_3d_lshape(), (96, 96, 24), 2), -1),
    "3d_small_level": (lambda: W.small(W.config_3d_penny(), 20, 3), 0),
    "2d": (lambda: W.small(W.config_2d_single_crack(), 40, 3), -1),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_host_apply_matches_device_apply(name):
    make_w, level = CASES[name]
    w = make_w()
    h, *_ = make(w)
    try:
        nd = level_dofs(w, level)
        x = W.random_vector(nd, 7)
        yd = torch.empty(nd, dtype=torch.float64, device=DEV)
        pff.apply_jacobian(h, level, t(x), yd)
        xh = torch.from_numpy(x).pin_memory()
        yh = torch.full((nd,), np.nan, dtype=torch.float64).pin_memory()
        pff.apply_jacobian_host(h, level, xh, yh)
        ref = yd.cpu().numpy()
        got = yh.numpy()
        assert np.all(np.isfinite(got))
        # the same contributions summed in another atomic order
        assert np.linalg.norm(got - ref) <= 1e-14 * np.linalg.norm(ref)
        # a second call reuses the buffers and streams
        x2 = W.random_vector(nd, 8)
        pff.apply_jacobian_host(h, level, torch.from_numpy(x2).pin_memory(), yh)
        pff.apply_jacobian(h, level, t(x2), yd)
        assert np.linalg.norm(yh.numpy() - yd.cpu().numpy()) <= 1e-14 * np.linalg.norm(yd.cpu().numpy())
    finally:
        pff.destroy_hierarchy(h)


def test_host_apply_full_size_sampled_rows():
    """128^3 penny, the configuration the bench's end-to-end number uses: sampled rows of the
    host-buffer apply against the oracle's row-by-row element computation."""
    w = W.config_3d_penny()
    h, U, po, pt = make(w)
    try:
        active = torch.empty(w.n_nodes, dtype=torch.uint8, device=DEV)
        pff.get_active_set(h, active)
        act = active.cpu().numpy()
        m = fem.Mesh(3, 1, w.n_cells, w.lo, w.hi)
        ph = fem.Phys(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=w.pressure)
        mask = fem.dirichlet_face_mask(m, 0x3F) | (act * fem.BIT_ACTIVE).astype(np.uint8)
        x = W.random_vector(w.n_dofs, 13)
        yh = torch.empty(w.n_dofs, dtype=torch.float64).pin_memory()
        pff.apply_jacobian_host(h, -1, torch.from_numpy(x).pin_memory(), yh)
        rng = np.random.default_rng(6)
        rows = rng.choice(w.n_dofs, 3000, replace=False)
        nz = w.n_cells[2] + 1
        layer = (w.n_cells[0] + 1) * (w.n_cells[1] + 1)
        # rows on the node layers where two slabs meet
        seams = np.concatenate([np.arange(k * layer, k * layer + 40) for k in range(16, nz, 16)])
        rows = np.concatenate([rows, seams, seams + 3 * w.n_nodes])
        ref = fem.apply_rows(m, ph, U, pt, mask, x, rows)
        got = yh.numpy()[rows]
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    finally:
        pff.destroy_hierarchy(h)
