"""Oracle pin by dimensional analysis: the penny crack in SI units (m, Pa, J/m^2) and the same
problem in mm, MPa and N/mm give the same Newton iterates of Algorithm 1 (Sec. 3.1), displacements
scaled by 1e3 and phase field unchanged.  Every term of the energy (Sec. 2.1) has to carry its own
powers of E, Gc, eps, p and the mesh size for this to hold: a dropped or inverted factor, a wrong
power of h in a weight or a derivative, a Gauss weight taken in the wrong dimension moves the balance
of elastic and fracture terms by powers of 1e3 and changes the active sets and the iterates.

With the tie band on the residual scale (tie_scale 1) the default eps_as = 1e-10 lies between the
rounding noise (~1e-20 J in SI, ~1e-17 N mm) and the genuine residual entries (~1e-4 J, ~1e-1 N mm),
so both unit systems classify every node the same way.  c of the active-set test has the units of
the multiplier (stress) and is converted with it."""
from dataclasses import replace

import numpy as np

from oracle import fem, pdas
from paper_1902_08112_gb300 import workloads as W

L = 1e3        # m -> mm
S = 1e-6       # Pa -> MPa = N/mm^2
G = 1e-3       # J/m^2 = N/m -> N/mm


def _run(w, c, steps):
    U, po, pt = W.initial_state(w)
    m = fem.Mesh(3, 1, w.n_cells, w.lo, w.hi)
    ph = fem.Phys(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=w.pressure)
    dm = fem.dirichlet_face_mask(m, 0x3F)
    prev, out = None, []
    for _ in range(steps):
        U, oi = pdas.newton_step(m, ph, w.n_levels, U, po, pt, dm, prev, c_as=c, tie_scale=1)
        out.append((oi.active.copy(), U.copy(), oi.n_changed))
        prev = oi.active
    return out


def test_newton_iterates_are_independent_of_the_unit_system():
    w = W.config_3d_penny_si(12, 1, 2, pressure=1e9)
    wm = replace(w, lo=tuple(L * a for a in w.lo), hi=tuple(L * a for a in w.hi), E=w.E * S, Gc=w.Gc * G,
                 pressure=w.pressure * S, eps=w.eps * L,
                 cracks=[replace(cr, radius=cr.radius * L) for cr in w.cracks])
    si = _run(w, 100.0, 2)
    mm = _run(wm, 100.0 * S, 2)
    nn = w.n_nodes
    for k, ((a_si, U_si, ch_si), (a_mm, U_mm, ch_mm)) in enumerate(zip(si, mm)):
        assert 0 < a_si.sum() < nn, k
        np.testing.assert_array_equal(a_si, a_mm)
        assert ch_si == ch_mm
        u_si, u_mm = U_si[:3 * nn] * L, U_mm[:3 * nn]
        # the two linear solves stop at the relative tolerance 1e-8 of their own unit systems
        assert np.linalg.norm(u_si - u_mm) <= 1e-6 * np.linalg.norm(u_mm), k
        assert np.linalg.norm(U_si[3 * nn:] - U_mm[3 * nn:]) <= 1e-6 * np.linalg.norm(U_mm[3 * nn:]), k
    # the second step moves the active set (the pin covers the Jacobian, not only the residual)
    assert si[1][2] > 0


def test_si_rounding_noise_and_genuine_residuals_are_split_by_the_tie_band():
    """Where phi = phi_old = 1 and u = 0 the exact residual is 0; in SI units its rounding noise is far
    below eps_as on the residual scale, while the multiplier lambda = R/M (M ~ h^3 ~ 1e-10 m^3) lifts the
    same noise to ~1e-9 Pa, above eps_as: the reason for tie_scale 1 in SI units."""
    w = W.config_3d_penny_si(12, 1, 2, pressure=1e7)
    U, po, pt = W.initial_state(w)
    m = fem.Mesh(3, 1, w.n_cells, w.lo, w.hi)
    ph = fem.Phys(E=w.E, nu=w.nu, Gc=w.Gc, kappa=w.kappa, eps=w.eps, p=w.pressure)
    R = -fem.residual_A(m, ph, U, pt)
    M = fem.lumped_mass(m)
    nn = m.n_nodes
    r = np.abs(R[3 * nn:])
    noise = (r > 0) & (r < 1e-15)
    genuine = r >= 1e-15
    assert noise.sum() > 0 and genuine.sum() > 0
    assert r[noise].max() < 1e-16 and r[genuine].min() > 1e-6
    assert (r[noise] / M[noise]).max() > 1e-10        # lambda's noise crosses the default band
    a1 = pdas.active_set(m, R, M, U, po, 100.0, 1e-10, tie_scale=1)
    assert not (a1 & noise).any()
