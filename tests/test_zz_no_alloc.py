"""The allocation-free active-set entry point (pff_active_set_noalloc) gives the same decision
as pff_update_active_set on two calls in a row.

It serves callers that cannot allocate device memory (no hierarchy of their own); its scratch is
a static device array inside the library.  Cases: box meshes (3D Q1, 2D Q2), a 3D L-shaped
domain whose cell mask is passed in device memory (the lumped mass sums over domain cells only,
nodes on no domain cell are never active), and a box whose host Dirichlet mask clamps phi on
seeded random nodes (PFF_MASK_PHI_DIR nodes are never active).  This file is collected last on
purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1902_08112_gb300 import pff, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _case(kind):
    if kind == "3d_q1_box":
        w = W.small(W.config_3d_penny(), 16, 2)
    elif kind == "2d_q2_box":
        w = W.small(W.config_2d_single_crack(deg=2), 24, 2)
    elif kind == "3d_q1_lshape":
        w = W.config_3d_lshape(16, 2)
    else:   # 3d_q1_phidir
        w = W.small(W.config_3d_penny(), 16, 2)
    w.pressure = 0.05
    if kind == "3d_q1_lshape":
        U, po, pt = W.random_state(w, seed=3)
        po = np.maximum(po, U[w.dim * w.n_nodes:])
    else:
        U, po, pt = W.initial_state(w, displacement="smooth")
    dmask = None
    if kind == "3d_q1_phidir":
        dmask = np.where(np.random.default_rng(9).uniform(size=w.n_nodes) < 0.3, pff.MASK_PHI_DIR, 0).astype(np.uint8)
    return w, U, po, pt, dmask


@pytest.mark.parametrize("kind", ["3d_q1_box", "2d_q2_box", "3d_q1_lshape", "3d_q1_phidir"])
def test_noalloc_active_set_matches_hierarchy(kind):
    w, U, po, pt, dmask = _case(kind)
    prm = pff.default_params(eps=w.eps, pressure=w.pressure, kappa=w.kappa, Gc=w.Gc)
    cm = w.cell_mask()
    mesh = pff.make_mesh(w.dim, w.deg, w.n_cells, w.n_levels, w.lo, w.hi, dirichlet_faces=w.dirichlet_faces,
                         cell_mask=cm, dirichlet_mask=dmask)
    h = pff.create_hierarchy(mesh, prm)
    try:
        Ud, pod, ptd = t(U), t(po), t(pt)
        cmd = t(cm) if cm is not None else None
        pff.set_state(h, Ud, pod, ptd)
        mask = torch.empty(w.n_nodes, dtype=torch.uint8, device=DEV)
        pff.level_state(h, -1, None, None, mask)          # Dirichlet bits, no active set yet
        mk = mask.cpu().numpy()
        fixed = (mk & pff.MASK_PHI_DIR) != 0
        if kind in ("3d_q1_lshape", "3d_q1_phidir"):
            assert fixed.any()
        R = torch.empty(w.n_dofs, dtype=torch.float64, device=DEV)
        act = torch.empty(w.n_nodes, dtype=torch.uint8, device=DEV)
        for call in range(2):
            pff.residual(h, R)
            na_ref, nc_ref = pff.update_active_set(h)
            pff.get_active_set(h, act)
            na, nc = pff.active_set_noalloc(mesh, prm, R, Ud, pod, mask, cell_mask=cmd)
            torch.cuda.synchronize()
            got = (mask.cpu().numpy() & pff.MASK_ACTIVE) != 0
            ref = act.cpu().numpy() != 0
            np.testing.assert_array_equal(got, ref)
            assert not got[fixed].any()
            assert na == na_ref > 0
            if call == 0:
                assert nc == na          # from an empty set every active node changed
            else:
                assert nc == nc_ref == 0
    finally:
        pff.destroy_hierarchy(h)


def test_noalloc_rejects_bad_arguments():
    prm = pff.default_params()
    big = pff.make_mesh(3, 1, (1024, 1024, 1024), 1, (0,) * 3, (1,) * 3)   # > 65536 * 1024 nodes
    x = torch.zeros(8, dtype=torch.float64, device=DEV)
    m = torch.zeros(8, dtype=torch.uint8, device=DEV)
    with pytest.raises(pff.PffError) as e:
        pff.active_set_noalloc(big, prm, x, x, x, m)
    assert e.value.status == pff.EINVAL
    # a cut domain whose cell mask exists only on the host cannot be decided without a copy
    w = W.config_3d_lshape(16, 2)
    cut = pff.make_mesh(3, 1, w.n_cells, 1, w.lo, w.hi, cell_mask=w.cell_mask())
    with pytest.raises(pff.PffError) as e:
        pff.active_set_noalloc(cut, prm, x, x, x, m)
    assert e.value.status == pff.EINVAL
