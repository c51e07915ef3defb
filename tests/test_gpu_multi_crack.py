"""The 3D multi-crack configuration at full size (256^3 Q1, 67.9M DoFs, 6 levels, 8 penny cracks):
sampled apply parity against the oracle's row-by-row element computation, and FGMRES with the
FP32 and the FP64 V-cycle solving a seeded right-hand side to 1e-8, the solution checked on
sampled rows of the oracle's operator (|b_i - (G~x)_i| <= 1e-8 ||b||_2 holds for every row when
the true residual meets the tolerance)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem  # noqa: E402
from paper_1902_08112_gb300 import pff, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_multi_crack_256_fp32_and_fp64_mg():
    w = W.config_3d_multi()
    U, po, pt = W.initial_state(w, displacement="smooth")
    act = W.random_active(w, 0.05)
    m = fem.Mesh(3, 1, w.n_cells, w.lo, w.hi)
    ph = fem.Phys(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=w.pressure)
    mask = fem.dirichlet_face_mask(m, 0x3F) | (act * fem.BIT_ACTIVE).astype(np.uint8)
    cons = fem.constrained_dofs(m, mask)
    b = np.where(cons, 0.0, W.random_vector(w.n_dofs, 21))
    rng = np.random.default_rng(22)
    crack_nodes = np.flatnonzero(po == 0.0)
    rows = np.concatenate([rng.choice(w.n_dofs, 1500, replace=False), crack_nodes[:150] + 3 * w.n_nodes,
                           crack_nodes[:150], np.arange(30)])
    x_probe = W.random_vector(w.n_dofs, 23)
    its = {}
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    for mgp in (32, 64):
        prm = pff.default_params(eps=w.eps, pressure=w.pressure, kappa=w.kappa, E=w.E, nu=w.nu, Gc=w.Gc,
                                 mg_precision=mgp)
        h = pff.create_hierarchy(pff.make_mesh(3, 1, w.n_cells, w.n_levels, w.lo, w.hi), prm)
        try:
            pff.set_state(h, t(U), t(po), t(pt))
            pff.set_active_set(h, t(act))
            if mgp == 32:
                y = torch.empty(w.n_dofs, dtype=torch.float64, device=DEV)
                pff.apply_jacobian(h, -1, t(x_probe), y)
                ref = fem.apply_rows(m, ph, U, pt, mask, x_probe, rows)
                got = y.cpu().numpy()[rows]
                assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
                del y
            x = torch.zeros(w.n_dofs, dtype=torch.float64, device=DEV)
            info = pff.gmres_solve(h, t(b), x, rtol=1e-8, restart=30, maxit=300)
            assert info.converged and info.res_final <= 1e-8 * info.res0
            its[mgp] = info.iterations
            xs = x.cpu().numpy()
            Gx = fem.apply_rows(m, ph, U, pt, mask, xs, rows)
            assert np.abs(b[rows] - Gx).max() <= 1.05e-8 * np.linalg.norm(b)
        finally:
            pff.destroy_hierarchy(h)
    # the FP32 V-cycle inside FP64 FGMRES costs at most a few extra iterations here
    assert its[32] <= its[64] + max(2, its[64] // 2), its
