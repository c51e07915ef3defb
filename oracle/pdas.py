"""One primal-dual active-set step (Algorithm 1, Sec. 3.1) of the oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Step k, with the lumped Gauss-Lobatto mass M of the remark after Algorithm 1:
  1. R_k = -A(U_k)
  2. G_k = A'(U_k)
  3. active set: phi-DoFs i with (M^-1 R_k)_i + c (phi_k - phi_old)_i > 0 (strict).  Values
     within the paper's active-set tolerance eps_as of zero are rounding noise (e.g. where
     phi = phi_old = 1 and u = 0 the exact value is 0) and count as ties, i.e. inactive: the
     test is taken as  > threshold  with threshold = eps_as.
  4. eliminate Dirichlet and active rows/columns: identity rows, zero columns.  Active rows
     carry the increment phi_old - phi (so phi = phi_old on the active set after the update),
     and its column contribution is moved to the right-hand side of the free rows.
  5. solve G~ dU = R~ with FGMRES preconditioned by the monolithic V-cycle (Sec. 3.3)
  6. U_{k+1} = U_k + dU
Stop when the active set repeats and ||R~_k||_2 <= eps_as.

Load stepping (Sec. 2.1, 2.3): at incremental step n, phi_old = phi^{n-1} and the time-lagged
extrapolation phi~ = clamp(2 phi^{n-1} - phi^{n-2}, 0, 1) (phi^{n-1} at the first step) enters
g(phi~) and phi~^2 of the u-equation; Algorithm 1 runs until its stop test, the previous load
step's active set serving as A_{k-1} of the first Newton step.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import fem, multigrid, krylov


@dataclass
class StepInfo:
    active: np.ndarray
    n_changed: int
    res_norm: float
    gmres_its: int
    lin_res: float
    lin_res0: float
    converged: bool


def active_set(mesh: fem.Mesh, R: np.ndarray, M: np.ndarray, U: np.ndarray, phi_old: np.ndarray,
               c: float, threshold: float = 1e-10, fixed: np.ndarray | None = None, tie_scale: int = 0) -> np.ndarray:
    """fixed: bool per node whose phi is prescribed (phi Dirichlet, outside the domain): never active.
    tie_scale 0: the tie band |lambda + c (phi - phi_old)| <= threshold; 1: the band on the scale of the
    residual entry, |M (lambda + c (phi - phi_old))| <= threshold."""
    nn = mesh.n_nodes
    phi = U[mesh.dim * nn:]
    free = M > 0 if fixed is None else (M > 0) & ~fixed
    lam = np.divide(R[mesh.dim * nn:], M, out=np.zeros(nn), where=free)
    v = lam + c * (phi - phi_old)
    return free & ((v * M if tie_scale else v) > threshold)


def eliminated_rhs(mesh, phys, U, ptil, phi_old, dir_mask, active, R):
    """R~ of step 4 and the full eliminated mask."""
    nn = mesh.n_nodes
    d = mesh.dim
    mask = dir_mask | np.where(active, fem.BIT_ACTIVE, 0).astype(np.uint8)
    delta = np.zeros(mesh.n_dofs)
    delta[d * nn:] = np.where(active, phi_old - U[d * nn:], 0.0)
    Gdir = fem.assemble(mesh, phys, U, ptil, dir_mask, phi_bits=fem.BIT_PHI_DIR)
    t = Gdir @ delta
    cons = fem.constrained_dofs(mesh, mask)
    Rt = R - t
    Rt[cons] = 0.0
    Rt[d * nn:][active] = delta[d * nn:][active]
    return Rt, mask


def lift_dirichlet(mesh, U, dir_mask, u_dirichlet):
    """The iterate with prescribed displacements on the Dirichlet DoFs (u-components whose mask bit is
    set); other entries of u_dirichlet are not read."""
    U = np.array(U, dtype=np.float64)
    nn = mesh.n_nodes
    for c in range(mesh.dim):
        on = (np.asarray(dir_mask) & fem.BIT_U[c]) != 0
        U[c * nn:(c + 1) * nn][on] = np.asarray(u_dirichlet)[c * nn:(c + 1) * nn][on]
    return U


def newton_step(mesh, phys, n_levels, U, phi_old, ptil, dir_mask, prev_active, c_as=100.0,
                tol_as=1e-10, rtol=1e-8, restart=30, maxit=500, seed=12345, cg_steps=10,
                prm: multigrid.MGParams | None = None, u_dirichlet=None, tie_scale: int = 0):
    """u_dirichlet: prescribed displacement values (displacement-driven loading, Sec. 5.2/5.3).  The
    iterate takes them on the Dirichlet DoFs before step 1, so R, G and the active set are evaluated at
    a state that satisfies the boundary condition and the increment of step 5 vanishes there (those rows
    are eliminated with a zero right-hand side, step 4)."""
    prm = prm or multigrid.MGParams()
    U = np.asarray(U, dtype=np.float64)
    if u_dirichlet is not None:
        U = lift_dirichlet(mesh, U, dir_mask, u_dirichlet)
    R = -fem.residual_A(mesh, phys, U, ptil)
    M = fem.lumped_mass(mesh)
    act = active_set(mesh, R, M, U, phi_old, c_as, tol_as, fixed=(dir_mask & fem.BIT_PHI_DIR) != 0,
                     tie_scale=tie_scale)
    Rt, mask = eliminated_rhs(mesh, phys, U, ptil, phi_old, dir_mask, act, R)
    levels = multigrid.build_levels(mesh, n_levels, phys, U, ptil, mask, coarse_phi_max=prm.coarse_phi_max)
    multigrid.estimate_levels(levels, seed, cg_steps)
    G = levels[-1].G
    dU, its, lin_res, lin_res0, _ = krylov.fgmres(lambda v: G @ v, Rt,
                                                   lambda v: multigrid.precondition(levels, v, prm),
                                                   rtol=rtol, restart=restart, maxit=maxit)
    n_changed = int(np.sum(act != prev_active)) if prev_active is not None else int(act.sum())
    res = float(np.linalg.norm(Rt))
    conv = prev_active is not None and n_changed == 0 and res <= tol_as
    return U + dU, StepInfo(act, n_changed, res, its, lin_res, lin_res0, conv)


def extrapolate(phi_nm1, phi_nm2=None):
    """phi~ of Sec. 2.3 (linear in time, clamped to [0, 1])."""
    phi_nm1 = np.asarray(phi_nm1, dtype=np.float64)
    if phi_nm2 is None:
        return phi_nm1.copy()
    return np.clip(2.0 * phi_nm1 - np.asarray(phi_nm2, dtype=np.float64), 0.0, 1.0)


def load_step(mesh, phys, n_levels, U, phi_prev, dir_mask, prev_active, max_newton=20, **kw):
    """One incremental step at phys.p; returns (U^n, list of StepInfo)."""
    nn = mesh.n_nodes
    phi_old = np.array(U[mesh.dim * nn:], dtype=np.float64)
    ptil = extrapolate(phi_old, phi_prev)
    infos = []
    for _ in range(max_newton):
        U, info = newton_step(mesh, phys, n_levels, U, phi_old, ptil, dir_mask, prev_active, **kw)
        infos.append(info)
        prev_active = info.active
        if info.converged:
            break
    return U, infos
