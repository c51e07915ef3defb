"""The allocation-free active-set entry point (pff_active_set_noalloc) gives the same decision
as pff_update_active_set on two calls in a row.

It serves callers that cannot allocate device memory (no hierarchy of their own); its scratch is
a static device array inside the library.  This file is collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1902_08112_gb300 import pff, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("dim,deg,n", [(3, 1, 16), (2, 2, 24)])
def test_noalloc_active_set_matches_hierarchy(dim, deg, n):
    base = W.config_3d_penny(deg=deg) if dim == 3 else W.config_2d_single_crack(deg=deg)
    w = W.small(base, n, 2)
    w.pressure = 0.05
    U, po, pt = W.initial_state(w, displacement="smooth")
    prm = pff.default_params(eps=w.eps, pressure=w.pressure, kappa=w.kappa)
    mesh = pff.make_mesh(w.dim, w.deg, w.n_cells, w.n_levels, w.lo, w.hi)
    h = pff.create_hierarchy(mesh, prm)
    try:
        Ud, pod, ptd = t(U), t(po), t(pt)
        pff.set_state(h, Ud, pod, ptd)
        mask = torch.empty(w.n_nodes, dtype=torch.uint8, device=DEV)
        pff.level_state(h, -1, None, None, mask)          # Dirichlet bits, no active set yet
        R = torch.empty(w.n_dofs, dtype=torch.float64, device=DEV)
        act = torch.empty(w.n_nodes, dtype=torch.uint8, device=DEV)
        for call in range(2):
            pff.residual(h, R)
            na_ref, nc_ref = pff.update_active_set(h)
            pff.get_active_set(h, act)
            na, nc = pff.active_set_noalloc(mesh, prm, R, Ud, pod, mask)
            torch.cuda.synchronize()
            got = (mask.cpu().numpy() & pff.MASK_ACTIVE) != 0
            np.testing.assert_array_equal(got, act.cpu().numpy() != 0)
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
