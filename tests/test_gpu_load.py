"""GPU parity of load stepping (Sec. 2.1, 2.3 with Algorithm 1 per step) against the oracle:
three steps p_n = n p / 3, same Newton step counts, same final active set, and the final state
within the accumulated solver tolerance (each linear solve stops at 1e-8 relative residual)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem, pdas  # noqa: E402
from paper_1902_08112_gb300 import pff, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

# workload, final pressure of the three steps
CASES = {
    "2d_q1_64": (lambda: W.config_2d_single_crack(), 0.05),
    "3d_q1_16": (lambda: W.small(W.config_3d_penny(), 16, 3), 0.05),
    "2d_two_cracks_32": (lambda: W.config_2d_two_cracks(32, 3), 30.0),   # p_n = 10 n (Sec. 5.1)
}


@pytest.mark.parametrize("mgp", [32, 64])
@pytest.mark.parametrize("name", sorted(CASES))
def test_load_steps_match_oracle(name, mgp):
    mk, p_max = CASES[name]
    w = mk()
    U0, po, pt = W.initial_state(w)
    prm = pff.default_params(eps=w.eps, pressure=p_max / 3, kappa=w.kappa, E=w.E, nu=w.nu, Gc=w.Gc,
                             mg_precision=mgp)
    h = pff.create_hierarchy(pff.make_mesh(w.dim, w.deg, w.n_cells, w.n_levels, w.lo, w.hi), prm)
    nn = w.n_nodes
    gpu_steps, gpu_act = [], []
    try:
        U = torch.from_numpy(U0.copy()).to(DEV)
        pff.set_state(h, U, torch.from_numpy(po).to(DEV), torch.from_numpy(pt).to(DEV))
        prev = None
        for n in (1, 2, 3):
            phi_nm1 = U[w.dim * nn:].clone()
            info = pff.load_step(h, U, prev, p_max * n / 3, max_newton=20)
            gpu_steps.append((info.newton_steps, info.converged))
            a = torch.empty(nn, dtype=torch.uint8, device=DEV)
            pff.get_active_set(h, a)
            gpu_act.append(a.cpu().numpy().astype(bool))
            prev = phi_nm1
        Ug = U.cpu().numpy()
        qoi = (pff.energies(h), pff.boundary_load(h, 3, 1))
    finally:
        pff.destroy_hierarchy(h)

    m = fem.Mesh(w.dim, w.deg, w.n_cells, w.lo, w.hi)
    dmask = fem.dirichlet_face_mask(m, 0x3F)
    Uo, prev_phi, prev_act = U0.copy(), None, None
    for n in (1, 2, 3):
        ph = fem.Phys(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=p_max * n / 3)
        phi_nm1 = Uo[w.dim * nn:].copy()
        Uo, infos = pdas.load_step(m, ph, w.n_levels, Uo, prev_phi, dmask, prev_act)
        prev_phi, prev_act = phi_nm1, infos[-1].active
        assert gpu_steps[n - 1][1] == 1 and infos[-1].converged
        assert abs(gpu_steps[n - 1][0] - len(infos)) <= 1
        assert np.array_equal(gpu_act[n - 1], infos[-1].active)
    scale = np.abs(Uo).max()
    assert np.abs(Ug - Uo).max() <= 1e-6 * scale
    ph = fem.Phys(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=p_max)
    ob, oc = fem.energy_parts(m, ph, Uo)
    assert qoi[0][0] == pytest.approx(ob, rel=1e-5)
    assert qoi[0][1] == pytest.approx(oc, rel=1e-5)
