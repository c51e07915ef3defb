"""FE layer of the oracle: ctypes binding to pff_oracle.c plus mesh bookkeeping.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Discretisation (Sec. 2.4, Problem 2.2): Q1/Q2 Lagrange elements on a uniform Cartesian box,
component-blocked DoFs [u_x | u_y | (u_z) | phi], nodes lexicographic with x fastest.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pff_oracle.c")
_SO = os.path.join(_HERE, "_pff_oracle.so")

# mask bits per node
BIT_U = (1, 2, 4)      # u_x, u_y, u_z Dirichlet
BIT_ACTIVE = 8         # phi in the active set (Algorithm 1, step 3)
BIT_PHI_DIR = 16       # phi Dirichlet
PHI_ALL = BIT_ACTIVE | BIT_PHI_DIR


def build_oracle(force: bool = False) -> str:
    """Compile the C oracle with plain gcc (no OpenMP, no vector intrinsics)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("deg", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("cell_mask", ctypes.POINTER(ctypes.c_uint8))]


class _Phys(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("lam", ctypes.c_double), ("Gc", ctypes.c_double),
                ("kappa", ctypes.c_double), ("eps", ctypes.c_double), ("p", ctypes.c_double),
                ("f", ctypes.c_double), ("escale", ctypes.POINTER(ctypes.c_double)), ("split", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build_oracle())
        P = ctypes.POINTER
        d = P(ctypes.c_double)
        i64 = P(ctypes.c_int64)
        u8 = P(ctypes.c_uint8)
        L.om_n_nodes.restype = ctypes.c_int64
        L.om_n_nodes.argtypes = [P(_Mesh)]
        L.om_residual.argtypes = [P(_Mesh), P(_Phys), d, d, d]
        L.om_energy.restype = ctypes.c_double
        L.om_energy.argtypes = [P(_Mesh), P(_Phys), d]
        L.om_lumped_mass.argtypes = [P(_Mesh), d]
        L.om_energy_parts.argtypes = [P(_Mesh), P(_Phys), d, d]
        L.om_csr_structure.restype = ctypes.c_int64
        L.om_csr_structure.argtypes = [P(_Mesh), i64]
        L.om_assemble.argtypes = [P(_Mesh), P(_Phys), d, d, u8, ctypes.c_int, i64, i64, d]
        L.om_apply_rows.argtypes = [P(_Mesh), P(_Phys), d, d, u8, ctypes.c_int, d,
                                    ctypes.c_int64, i64, d]
        _lib = L
    return _lib


def lame(E: float, nu: float) -> tuple[float, float]:
    """Lame coefficients from Young's modulus and Poisson ratio, 3D formulas (Sec. 5.1 table:
    E=1e4, nu=0.2 give mu=4166.6, lambda=2777.7); 2D is plane strain."""
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


@dataclass
class Mesh:
    dim: int
    deg: int
    n: tuple            # cells per axis (len dim)
    lo: tuple
    hi: tuple
    cell_mask: np.ndarray | None = None   # uint8 per cell (x fastest), 1 = in the domain; None = box

    def nodes_per_axis(self):
        return tuple(self.deg * self.n[a] + 1 for a in range(self.dim))

    @property
    def n_nodes(self) -> int:
        return int(np.prod(self.nodes_per_axis()))

    @property
    def n_cells(self) -> int:
        return int(np.prod(self.n))

    @property
    def ncomp(self) -> int:
        return self.dim + 1

    @property
    def n_dofs(self) -> int:
        return self.ncomp * self.n_nodes

    def h(self):
        return tuple((self.hi[a] - self.lo[a]) / self.n[a] for a in range(self.dim))

    def coarsen(self) -> "Mesh":
        """Next coarser nested mesh; a coarse cell is in the domain if any of its children is."""
        assert all(c % 2 == 0 for c in self.n)
        cm = None
        if self.cell_mask is not None:
            a = (np.asarray(self.cell_mask).reshape(tuple(self.n[::-1])) != 0)
            for ax in range(self.dim):
                sl0 = [slice(None)] * self.dim
                sl1 = [slice(None)] * self.dim
                sl0[ax] = slice(0, None, 2)
                sl1[ax] = slice(1, None, 2)
                a = a[tuple(sl0)] | a[tuple(sl1)]
            cm = a.ravel().astype(np.uint8)
        return Mesh(self.dim, self.deg, tuple(c // 2 for c in self.n), self.lo, self.hi, cm)

    def node_touches_domain(self) -> np.ndarray:
        """bool per node: the node belongs to at least one cell of the domain."""
        npa = self.nodes_per_axis()
        if self.cell_mask is None:
            return np.ones(self.n_nodes, dtype=bool)
        cm = (np.asarray(self.cell_mask).reshape(tuple(self.n[::-1])) != 0)
        out = np.zeros(tuple(npa[::-1]), dtype=bool)
        for off in np.ndindex(*([self.deg + 1] * self.dim)):
            sl = tuple(slice(o, o + self.deg * nc, self.deg) for o, nc in zip(off[::-1], self.n[::-1]))
            out[sl] |= cm
        return out.ravel()

    def node_coords(self):
        """(n_nodes, dim) coordinates, x fastest."""
        axes = [np.linspace(self.lo[a], self.hi[a], self.nodes_per_axis()[a]) for a in range(self.dim)]
        grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
        return np.stack([g.ravel() for g in grids], axis=1)

    def c(self) -> _Mesh:
        m = _Mesh()
        m.dim, m.deg = self.dim, self.deg
        for a in range(3):
            m.n[a] = self.n[a] if a < self.dim else 1
            m.lo[a] = self.lo[a] if a < self.dim else 0.0
            m.hi[a] = self.hi[a] if a < self.dim else 1.0
        if self.cell_mask is not None:
            arr = np.ascontiguousarray(self.cell_mask, dtype=np.uint8)
            m.cell_mask = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
            m._keep = arr           # the C side reads the array during the call
        return m


@dataclass
class Phys:
    E: float = 1.0
    nu: float = 0.2
    Gc: float = 1.0
    kappa: float = 1e-10
    eps: float = 1.0
    p: float = 1e-3
    f: float = 1.0            # factor on the phi-equation elastic term (1 = energy consistent)
    escale: np.ndarray | None = None   # per cell factor on E (n_cells, x fastest), None = uniform
    split: int = 0            # 0: E_s^+ = E_s (no split); 1: Miehe split (Sec. 2.1)
    extra: dict = field(default_factory=dict)

    def c(self) -> _Phys:
        mu, lam = lame(self.E, self.nu)
        ph = _Phys(mu, lam, self.Gc, self.kappa, self.eps, self.p, self.f, None, int(self.split))
        if self.escale is not None:
            arr = np.ascontiguousarray(self.escale, dtype=np.float64)
            ph.escale = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            ph._keep = arr          # the C side reads the array during the call
        return ph


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _up(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def residual_A(mesh: Mesh, phys: Phys, U, ptil) -> np.ndarray:
    """A(U)(Phi_i) for all i, Eq. (semilinear), no elimination."""
    U, ptil = _f64(U), _f64(ptil)
    out = np.zeros(mesh.n_dofs)
    m, ph = mesh.c(), phys.c()
    lib().om_residual(ctypes.byref(m), ctypes.byref(ph), _dp(U), _dp(ptil), _dp(out))
    return out


def energy(mesh: Mesh, phys: Phys, U) -> float:
    U = _f64(U)
    m, ph = mesh.c(), phys.c()
    return lib().om_energy(ctypes.byref(m), ctypes.byref(ph), _dp(U))


def energy_parts(mesh: Mesh, phys: Phys, U) -> tuple:
    """(bulk, crack) energies of Sec. 5 (no stress split)."""
    U = _f64(U)
    out = np.zeros(2)
    m, ph = mesh.c(), phys.c()
    lib().om_energy_parts(ctypes.byref(m), ctypes.byref(ph), _dp(U), _dp(out))
    return float(out[0]), float(out[1])


def face_nodes(mesh: Mesh, face: int) -> np.ndarray:
    """Indices of the nodes on one face of the box (face 2a: lower, 2a+1: upper face of axis a)."""
    npa = mesh.nodes_per_axis()
    idx = np.indices(npa[::-1]).reshape(mesh.dim, -1)[::-1]
    a, side = divmod(face, 2)
    return np.nonzero(idx[a] == (npa[a] - 1 if side else 0))[0]


def boundary_load(mesh: Mesh, phys: Phys, U, ptil, face: int, comp: int) -> float:
    """L_c of Sec. 5 (traction (sigma n)_c integrated over a face), taken as the reaction: the sum of
    A(U)(phi_i e_c) over the face's nodes."""
    A = residual_A(mesh, phys, U, ptil)
    return float(np.sum(A[comp * mesh.n_nodes + face_nodes(mesh, face)]))


def lumped_mass(mesh: Mesh) -> np.ndarray:
    out = np.zeros(mesh.n_nodes)
    m = mesh.c()
    lib().om_lumped_mass(ctypes.byref(m), _dp(out))
    return out


def assemble(mesh: Mesh, phys: Phys, U, ptil, mask, phi_bits: int = PHI_ALL) -> sp.csr_matrix:
    """Eliminated Jacobian G~ (Algorithm 1, steps 2 and 4) as CSR."""
    U, ptil = _f64(U), _f64(ptil)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    m, ph = mesh.c(), phys.c()
    nd = mesh.n_dofs
    indptr = np.zeros(nd + 1, dtype=np.int64)
    nnz = lib().om_csr_structure(ctypes.byref(m), _ip(indptr))
    indices = np.zeros(nnz, dtype=np.int64)
    data = np.zeros(nnz)
    lib().om_assemble(ctypes.byref(m), ctypes.byref(ph), _dp(U), _dp(ptil), _up(mask), int(phi_bits),
                      _ip(indptr), _ip(indices), _dp(data))
    return sp.csr_matrix((data, indices, indptr), shape=(nd, nd))


def apply_rows(mesh: Mesh, phys: Phys, U, ptil, mask, x, rows, phi_bits: int = PHI_ALL) -> np.ndarray:
    """(G~ x)_r for selected rows r, from element matrices (no global assembly)."""
    U, ptil, x = _f64(U), _f64(ptil), _f64(x)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros(len(rows))
    m, ph = mesh.c(), phys.c()
    lib().om_apply_rows(ctypes.byref(m), ctypes.byref(ph), _dp(U), _dp(ptil), _up(mask), int(phi_bits),
                        _dp(x), len(rows), _ip(rows), _dp(out))
    return out


def constrained_dofs(mesh: Mesh, mask, phi_bits: int = PHI_ALL) -> np.ndarray:
    """Boolean per DoF: True where the row/column is eliminated."""
    mask = np.asarray(mask, dtype=np.uint8)
    parts = [(mask & BIT_U[c]) != 0 for c in range(mesh.dim)]
    parts.append((mask & phi_bits) != 0)
    return np.concatenate(parts)


def dirichlet_face_mask(mesh: Mesh, faces: int) -> np.ndarray:
    """uint8 per node: all u components clamped on the faces in 'faces'
    (bit 2a = lower face of axis a, bit 2a+1 = upper face).  Nodes that belong to no cell of the
    domain (mesh.cell_mask) are fixed in every component (identity rows)."""
    npa = mesh.nodes_per_axis()
    idx = np.indices(npa[::-1]).reshape(mesh.dim, -1)[::-1]   # idx[a] = index along axis a
    on = np.zeros(mesh.n_nodes, dtype=bool)
    for a in range(mesh.dim):
        if faces >> (2 * a) & 1:
            on |= idx[a] == 0
        if faces >> (2 * a + 1) & 1:
            on |= idx[a] == npa[a] - 1
    ubits = sum(BIT_U[c] for c in range(mesh.dim))
    out = np.where(on, ubits, 0).astype(np.uint8)
    outside = ~mesh.node_touches_domain()
    out[outside] = ubits | BIT_PHI_DIR
    return out
