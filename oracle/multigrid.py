"""Geometric multigrid of the oracle (Sec. 3.2, 3.3 and 4.2), plain numpy/scipy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

 - Transfers: nested Q1/Q2 grids, prolongation P = nodal interpolation of the coarse FE
   function (the canonical prolongation of Sec. 3.2), restriction of residuals R = P^T.
 - Level state, extrapolation and active set carried to the coarse levels by restriction
   onto coincident nodes (Sec. 4.2): every coarse node is also a fine node, so the active
   indicator stays in {0,1}.  Q2 levels (an extension; the paper uses Q1) take the extrapolated
   phase field phi~ of a coarse node as the maximum of the fine phi~ over the fine nodes at most one
   fine node spacing away from it (the 3^d block around the coincident node, cut at the boundary):
   a Q2 field carries values at edge, face and cell-centre nodes that injection drops, and a coarse
   cell that loses them becomes kappa-weak where the fine cells are stiff.
 - Level operators G_l(U_l) at the restricted state (Sec. 4.2), assembled by the C oracle.
 - Chebyshev-Jacobi smoother on each diagonal block (Sec. 3.2.1, block-diagonal S_full of
   Sec. 3.3), range [1.2 l/5, 1.2 l] with l from 10 Jacobi-preconditioned CG steps.  The
   recurrence is the Chebyshev acceleration of Saad, Iterative Methods for Sparse Linear
   Systems (2nd ed.), Algorithm 12.1, applied to D^-1 A.
 - Coarsest level: Chebyshev as a solver on [0.9 l_min, 1.2 l_max] (Sec. 3.2.2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np
import scipy.sparse as sp

from . import fem
from .rng import uniform_pm1


# ------------------------------------------------------------------ transfers

def _lagrange(deg: int, a: int, t: float) -> float:
    v = 1.0
    for b in range(deg + 1):
        if b != a:
            v *= (t - b / deg) / (a / deg - b / deg)
    return v


def prolongation_1d(deg: int, n_coarse_cells: int) -> np.ndarray:
    """Dense 1D interpolation matrix (fine nodes x coarse nodes): fine node i at position
    i/(2 deg) (coarse cell units) takes the coarse Lagrange interpolant's value there."""
    nc = deg * n_coarse_cells + 1
    nf = 2 * deg * n_coarse_cells + 1
    P = np.zeros((nf, nc))
    for i in range(nf):
        x = i / (2.0 * deg)                   # position in coarse-cell units
        cell = min(int(math.floor(x)), n_coarse_cells - 1)
        t = x - cell
        for a in range(deg + 1):
            P[i, deg * cell + a] = _lagrange(deg, a, t)
    P[np.abs(P) < 1e-15] = 0.0
    return P


def prolongation(mesh_c: fem.Mesh, mesh_f: fem.Mesh) -> sp.csr_matrix:
    """Scalar prolongation (n_nodes_f x n_nodes_c) as the Kronecker product of the 1D ones
    (x fastest, so the x factor is the rightmost)."""
    P = None
    for a in range(mesh_c.dim):
        Pa = sp.csr_matrix(prolongation_1d(mesh_c.deg, mesh_c.n[a]))
        P = Pa if P is None else sp.kron(Pa, P, format="csr")
    return P


def prolongation_full(mesh_c: fem.Mesh, mesh_f: fem.Mesh) -> sp.csr_matrix:
    P = prolongation(mesh_c, mesh_f)
    return sp.block_diag([P] * mesh_c.ncomp, format="csr")


def injection_index(mesh_c: fem.Mesh, mesh_f: fem.Mesh) -> np.ndarray:
    """Fine node index coinciding with each coarse node: coarse (I,J,K) = fine (2I,2J,2K)."""
    npc = mesh_c.nodes_per_axis()
    npf = mesh_f.nodes_per_axis()
    idx = np.indices(npc[::-1]).reshape(mesh_c.dim, -1)[::-1]
    fine = np.zeros(idx.shape[1], dtype=np.int64)
    stride = 1
    for a in range(mesh_c.dim):
        fine += 2 * idx[a] * stride
        stride *= npf[a]
    return fine


# ------------------------------------------------------------------ levels

@dataclass
class Level:
    mesh: fem.Mesh
    mask: np.ndarray          # uint8 per node
    U: np.ndarray
    ptil: np.ndarray
    G: sp.csr_matrix          # eliminated level operator G~_l(U_l)
    free: np.ndarray          # bool per DoF
    dinv: np.ndarray          # inverse diagonal
    ublock: np.ndarray        # DoF indices of the displacement block
    pblock: np.ndarray        # DoF indices of the phase-field block
    lam_max: tuple = (1.0, 1.0)
    lam_min: tuple = (1.0, 1.0)
    P: sp.csr_matrix | None = None   # prolongation from the next coarser level


def neighbourhood_max(mesh_c: fem.Mesh, mesh_f: fem.Mesh, pf: np.ndarray) -> np.ndarray:
    """For every coarse node, the maximum of the fine nodal field pf over the fine nodes whose lattice
    index differs from the coincident node's by at most 1 along every axis (cut at the boundary)."""
    npf = mesh_f.nodes_per_axis()
    a = np.asarray(pf, dtype=np.float64).reshape(tuple(npf[::-1]))
    out = a.copy()
    for ax in range(mesh_f.dim):
        axis = mesh_f.dim - 1 - ax              # array axis of mesh axis 'ax' (x is the last)
        cur = out.copy()
        lo = [slice(None)] * mesh_f.dim
        hi = [slice(None)] * mesh_f.dim
        lo[axis], hi[axis] = slice(0, -1), slice(1, None)
        np.maximum(cur[tuple(lo)], out[tuple(hi)], out=cur[tuple(lo)])      # neighbour at +1
        np.maximum(cur[tuple(hi)], out[tuple(lo)], out=cur[tuple(hi)])      # neighbour at -1
        out = cur
    return out.ravel()[injection_index(mesh_c, mesh_f)]


def coarsen_cell_field(mesh: fem.Mesh, s: np.ndarray) -> np.ndarray:
    """Per-cell field on the next coarser mesh: the mean over the 2^d fine cells of each coarse
    cell (how a varying modulus enters the rediscretised coarse operators of Sec. 4.2)."""
    n = mesh.n
    a = np.asarray(s, dtype=np.float64).reshape(tuple(n[::-1]))
    for ax in range(mesh.dim):
        sl0 = [slice(None)] * mesh.dim
        sl1 = [slice(None)] * mesh.dim
        sl0[ax] = slice(0, None, 2)
        sl1[ax] = slice(1, None, 2)
        a = 0.5 * (a[tuple(sl0)] + a[tuple(sl1)])
    return a.ravel()


def build_levels(mesh: fem.Mesh, n_levels: int, phys: fem.Phys, U, ptil, mask, coarse_phi_max: bool = False) -> list:
    """Level 0 = coarsest, n_levels-1 = finest (the given state and mask).  coarse_phi_max: Q1 levels
    take phi~ as the neighbourhood maximum too (an option beyond the paper; Q2 levels always do)."""
    meshes = [mesh]
    for _ in range(n_levels - 1):
        meshes.append(meshes[-1].coarsen())
    phys_l = [phys]
    for l in range(n_levels - 1):
        es = phys_l[-1].escale
        phys_l.append(replace(phys_l[-1], escale=None if es is None else coarsen_cell_field(meshes[l], es)))
    meshes = meshes[::-1]
    phys_l = phys_l[::-1]
    states = [None] * n_levels
    states[-1] = (np.asarray(U, dtype=np.float64), np.asarray(ptil, dtype=np.float64),
                  np.asarray(mask, dtype=np.uint8))
    for l in range(n_levels - 2, -1, -1):
        inj = injection_index(meshes[l], meshes[l + 1])
        Uf, pf, mf = states[l + 1]
        nnf = meshes[l + 1].n_nodes
        Uc = np.concatenate([Uf[c * nnf + inj] for c in range(mesh.ncomp)])
        pc = neighbourhood_max(meshes[l], meshes[l + 1], pf) if (mesh.deg == 2 or coarse_phi_max) else pf[inj]
        states[l] = (Uc, pc, mf[inj])
    levels = []
    for l in range(n_levels):
        m = meshes[l]
        Ul, pl, ml = states[l]
        G = fem.assemble(m, phys_l[l], Ul, pl, ml)
        free = ~fem.constrained_dofs(m, ml)
        dinv = 1.0 / G.diagonal()
        nn = m.n_nodes
        lev = Level(m, ml, Ul, pl, G, free, dinv,
                    np.arange(0, m.dim * nn), np.arange(m.dim * nn, (m.dim + 1) * nn))
        if l > 0:
            lev.P = prolongation_full(meshes[l - 1], m)
        levels.append(lev)
    return levels


# ------------------------------------------------------------------ eigenvalue estimates

def start_vector(seed: int, level: int, n_dofs: int, free: np.ndarray) -> np.ndarray:
    v = uniform_pm1(seed, level, n_dofs)
    v[~free] = 0.0
    return v


def cg_lanczos_bounds(A, dinv, v0, steps: int):
    """Extreme Ritz values of D^-1 A from 'steps' Jacobi-preconditioned CG iterations started
    at b = v0, x = 0 (Sec. 3.2.1).  The Lanczos tridiagonal is built from the CG step lengths
    alpha_j and ratios beta_j: T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},
    T_j,j+1 = sqrt(beta_j)/alpha_j."""
    r = v0.copy()
    z = dinv * r
    p = z.copy()
    rz = float(r @ z)
    alphas, betas = [], []
    for _ in range(steps):
        if not rz > 0.0:
            break
        q = A @ p
        pq = float(p @ q)
        if not pq > 0.0:
            break
        alpha = rz / pq
        r = r - alpha * q
        z = dinv * r
        rz_new = float(r @ z)
        beta = rz_new / rz
        alphas.append(alpha)
        betas.append(beta)
        p = z + beta * p
        rz = rz_new
    k = len(alphas)
    if k == 0:
        return 1.0, 1.0
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = math.sqrt(betas[j]) / alphas[j]
    ev = np.linalg.eigvalsh(T)
    return float(ev[0]), float(ev[-1])


def estimate_levels(levels: list, seed: int, steps: int = 10) -> None:
    for l, lev in enumerate(levels):
        v = start_vector(seed, l, lev.mesh.n_dofs, lev.free)
        lo, hi = [], []
        for blk in (lev.ublock, lev.pblock):
            A = lev.G[blk][:, blk]
            a, b = cg_lanczos_bounds(A, lev.dinv[blk], v[blk], steps)
            lo.append(a)
            hi.append(b)
        lev.lam_min = tuple(lo)
        lev.lam_max = tuple(hi)


# ------------------------------------------------------------------ Chebyshev

def chebyshev_zero(A, dinv, b, alpha: float, beta: float, k: int) -> np.ndarray:
    """k steps of Chebyshev acceleration (Saad, Algorithm 12.1) for D^-1 A x = D^-1 b on the
    eigenvalue interval [alpha, beta], starting from x = 0; returns x_k."""
    theta = 0.5 * (beta + alpha)
    delta = 0.5 * (beta - alpha)
    sigma1 = theta / delta
    rho = 1.0 / sigma1
    r = b.copy()
    d = (dinv * r) / theta
    x = np.zeros_like(b)
    for s in range(1, k + 1):
        x = x + d
        if s == k:
            break
        r = r - A @ d
        rho_new = 1.0 / (2.0 * sigma1 - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (dinv * r)
        rho = rho_new
    return x


def smoother_range(lam_max: float, safety: float = 1.2, ratio: float = 0.2):
    return ratio * safety * lam_max, safety * lam_max


def coarse_range(lam_min: float, lam_max: float):
    return 0.9 * lam_min, 1.2 * lam_max


def coarse_steps(alpha: float, beta: float, rtol: float, maxit: int) -> int:
    """Smallest k with 1/T_k(sigma1) <= rtol (Chebyshev error bound), capped at maxit."""
    sigma1 = (beta + alpha) / (beta - alpha)
    k = math.ceil(math.acosh(1.0 / rtol) / math.acosh(sigma1))
    return max(1, min(maxit, k))


@dataclass
class MGParams:
    cheb_degree: int = 4
    safety: float = 1.2
    ratio: float = 0.2
    coarse_rtol: float = 1e-6
    coarse_maxit: int = 200
    block_diagonal: bool = False   # P_diag = blockdiag(MG(U~), MG(P~)) of Sec. 3.3 instead of P_full
    coarse_phi_max: bool = False   # phi~ on coarse Q1 levels: neighbourhood maximum (else injection)


def level_operator(lev: Level, prm: MGParams):
    """Operator of the V-cycle on a level: G~ for P_full; for P_diag its two diagonal blocks
    (the coupling block G_phiu, rows of phi and columns of u, is left out)."""
    if not prm.block_diagonal:
        return lev.G
    if getattr(lev, "_Gbd", None) is None:
        G = lev.G.tocoo()
        is_phi_row = np.isin(G.row, lev.pblock)
        is_u_col = np.isin(G.col, lev.ublock)
        keep = ~(is_phi_row & is_u_col)
        lev._Gbd = sp.csr_matrix((G.data[keep], (G.row[keep], G.col[keep])), shape=G.shape)
    return lev._Gbd


def smooth_zero(lev: Level, b: np.ndarray, prm: MGParams) -> np.ndarray:
    """Block-diagonal smoother S_full = blockdiag(S(U), S(P)) (Sec. 3.3) from a zero guess:
    each block runs Chebyshev-Jacobi on its own diagonal block with its own range."""
    x = np.zeros_like(b)
    for bi, blk in enumerate((lev.ublock, lev.pblock)):
        A = lev.G[blk][:, blk]
        a, c = smoother_range(lev.lam_max[bi], prm.safety, prm.ratio)
        x[blk] = chebyshev_zero(A, lev.dinv[blk], b[blk], a, c, prm.cheb_degree)
    return x


def coarse_solve(lev: Level, b: np.ndarray, prm: MGParams) -> np.ndarray:
    """Chebyshev as solver on the coarsest level (Sec. 3.2.2) on [0.9 l_min, 1.2 l_max] of each
    block, in block forward-substitution order (G~ is block lower triangular, Sec. 3.3)."""
    x = np.zeros_like(b)
    ub, pb = lev.ublock, lev.pblock
    a, c = coarse_range(lev.lam_min[0], lev.lam_max[0])
    k = coarse_steps(a, c, prm.coarse_rtol, prm.coarse_maxit)
    x[ub] = chebyshev_zero(lev.G[ub][:, ub], lev.dinv[ub], b[ub], a, c, k)
    rphi = b[pb] if prm.block_diagonal else b[pb] - lev.G[pb][:, ub] @ x[ub]
    a, c = coarse_range(lev.lam_min[1], lev.lam_max[1])
    k = coarse_steps(a, c, prm.coarse_rtol, prm.coarse_maxit)
    x[pb] = chebyshev_zero(lev.G[pb][:, pb], lev.dinv[pb], rphi, a, c, k)
    return x


def vcycle(levels: list, l: int, b: np.ndarray, prm: MGParams) -> np.ndarray:
    """One V-cycle on level l for a right-hand side that is zero on constrained DoFs."""
    lev = levels[l]
    if l == 0:
        return coarse_solve(lev, b, prm)
    G = level_operator(lev, prm)
    x = smooth_zero(lev, b, prm)
    r = b - G @ x
    coarse = levels[l - 1]
    rc = lev.P.T @ r
    rc[~coarse.free] = 0.0
    ec = vcycle(levels, l - 1, rc, prm)
    corr = lev.P @ ec
    corr[~lev.free] = 0.0
    x = x + corr
    x = x + smooth_zero(lev, b - G @ x, prm)
    return x


def precondition(levels: list, v: np.ndarray, prm: MGParams) -> np.ndarray:
    """P_full^-1 = MG(G~), or P_diag^-1 with prm.block_diagonal (Sec. 3.3): V-cycle on the free
    DoFs, identity on eliminated ones."""
    fine = levels[-1]
    b = np.where(fine.free, v, 0.0)
    z = vcycle(levels, len(levels) - 1, b, prm)
    z[~fine.free] = v[~fine.free]
    return z
