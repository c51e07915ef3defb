"""GPU parity of the Sec. 5 quantities of interest (bulk and crack energies, boundary loads)
against the oracle's FP64 values."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem  # noqa: E402
from paper_1902_08112_gb300 import pff, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

CASES = {
    "2d_q1_64_initial": (lambda: W.config_2d_single_crack(), "initial"),
    "2d_q1_33x17_random": (lambda: W.small(W.config_2d_single_crack(), (34, 18), 2), "random"),
    "3d_q1_16_initial": (lambda: W.small(W.config_3d_penny(), 16, 3), "initial"),
    "3d_q1_12x10x6_random": (lambda: W.small(W.config_3d_penny(), (12, 10, 6), 2), "random"),
    "3d_q1_16_modulus": (lambda: W.small(W.config_3d_penny(), 16, 3), "modulus"),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_energies_match_oracle(name):
    mk, state = CASES[name]
    w = mk()
    U, po, pt = W.random_state(w) if state == "random" else W.initial_state(w, displacement="smooth")
    es = W.modulus_field(w) if state == "modulus" else None
    prm = pff.default_params(eps=w.eps, pressure=w.pressure, kappa=w.kappa, E=w.E, nu=w.nu, Gc=w.Gc)
    h = pff.create_hierarchy(pff.make_mesh(w.dim, w.deg, w.n_cells, w.n_levels, w.lo, w.hi), prm)
    try:
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
        if es is not None:
            pff.set_modulus(h, t(es))
        pff.set_state(h, t(U), t(po), t(pt))
        bulk, crack = pff.energies(h)
        loads = {(f, c): pff.boundary_load(h, f, c) for f in range(2 * w.dim) for c in range(w.dim)}
    finally:
        pff.destroy_hierarchy(h)
    m = fem.Mesh(w.dim, w.deg, w.n_cells, w.lo, w.hi)
    ph = fem.Phys(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=w.pressure, escale=es)
    ob, oc = fem.energy_parts(m, ph, U)
    assert abs(bulk - ob) <= 1e-11 * max(abs(ob), 1e-300) + 1e-14 * abs(oc)
    assert abs(crack - oc) <= 1e-11 * abs(oc)
    ol = {(f, c): fem.boundary_load(m, ph, U, pt, f, c) for f in range(2 * w.dim) for c in range(w.dim)}
    scale = max(abs(v) for v in ol.values())
    for k, v in ol.items():
        assert abs(loads[k] - v) <= 1e-11 * scale, k
