"""Seeded synthetic workloads shaped like the paper's pressurised-crack examples.

This module holds only input generation: mesh sizes, material constants, crack layouts and
the initial phase field they imply, random vectors.  It contains none of the solver's
arithmetic, so both the CUDA library's tests and the oracle's tests may use it.

Recipes (seed 12345 unless stated):
  * 2D single crack: [-10,10]^2, 64^2 Q1, E=1, nu=0.2, Gc=1, kappa=1e-10, eps=2h, p=1e-3,
    phi=0 on every cell meeting |x|<=1, |y|<=h, else 1; phi_old=phi, u=0.
  * 3D penny crack: [-10,10]^3, 128^3 Q1 or 64^3 Q2, same material, crack disk of radius 1 in
    the plane z=0 (cells meeting |z|<=h, x^2+y^2<=1 get phi=0).
  * 3D multi-crack: 8 penny cracks, centres U[-6,6]^3, normals N(0,I) normalised, radii U[1,2].
  * batch instances: N^3 Q1 with N in {16,24,32,48,64}, 1-6 cracks of radius U[0.5,2],
    p ~ U[5e-4, 2e-3].
  * 3D penny crack in SI units: a 1 cm box [-5e-3,5e-3]^3 m, E=2.1e11 Pa, nu=0.3, Gc=2.7e3 J/m^2,
    p=1e7 Pa, crack disk of radius 1 mm; kappa=1e-10, eps=2h.
h is the cell diameter (sqrt(dim) times the edge length); the paper calls h the element
diameter in its first example.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

SEED = 12345
ALL_FACES = 0x3F


@dataclass
class Crack:
    center: tuple
    normal: tuple
    radius: float          # half length in 2D, disk radius in 3D
    half_width: float = 1.0    # half thickness of the crack region in units of h


@dataclass
class Workload:
    name: str
    dim: int
    deg: int
    n_cells: tuple
    n_levels: int
    lo: tuple
    hi: tuple
    E: float = 1.0
    nu: float = 0.2
    Gc: float = 1.0
    kappa: float = 1e-10
    eps: float = 0.0
    pressure: float = 1e-3
    eps_factor: float = 2.0
    dirichlet_faces: int = ALL_FACES
    cracks: list = field(default_factory=list)
    seed: int = SEED
    domain: str = "box"            # "box" or "lshape" (the box minus its x >= mid, y >= mid quarter)
    # displacement-driven loading: the vertical displacement is prescribed on the nodes of the strip
    # {x0 <= x <= x1, y = y_s} (all z), growing linearly to u_ramp over the load steps
    load_strip: tuple | None = None    # ((x0, x1), y_s)
    u_ramp: float = 0.0

    def cell_mask(self):
        """uint8 per cell (x fastest), 1 = in the domain; None for the whole box."""
        if self.domain == "box":
            return None
        nx, ny = self.n_cells[0], self.n_cells[1]
        i = np.arange(nx)[None, :]
        j = np.arange(ny)[:, None]
        plane = ~((i >= nx // 2) & (j >= ny // 2))
        nz = self.n_cells[2] if self.dim == 3 else 1
        return np.broadcast_to(plane, (nz, ny, nx)).ravel().astype(np.uint8)

    def _strip_nodes(self):
        (x0, x1), ys = self.load_strip
        npa = self.nodes_per_axis()
        idx = np.indices(npa[::-1]).reshape(self.dim, -1)[::-1]     # idx[a] = index along axis a
        hx = (self.hi[0] - self.lo[0]) / (npa[0] - 1)
        hy = (self.hi[1] - self.lo[1]) / (npa[1] - 1)
        x = self.lo[0] + idx[0] * hx
        y = self.lo[1] + idx[1] * hy
        tol = 1e-9 * (self.hi[0] - self.lo[0])
        return (np.abs(y - ys) <= tol) & (x >= x0 - tol) & (x <= x1 + tol)

    def dirichlet_mask(self):
        """uint8 per node with the u_y Dirichlet bit on the loading strip (None without one), OR-ed by the
        library into the face mask."""
        if self.load_strip is None:
            return None
        return np.where(self._strip_nodes(), 2, 0).astype(np.uint8)

    def u_dirichlet(self, frac: float):
        """Prescribed displacements (dim * n_nodes, component-blocked) at the fraction 'frac' of the load
        ramp: u_y = frac * u_ramp on the strip, 0 elsewhere (the clamped faces); None without a strip."""
        if self.load_strip is None:
            return None
        u = np.zeros(self.dim * self.n_nodes)
        u[self.n_nodes:2 * self.n_nodes][self._strip_nodes()] = frac * self.u_ramp
        return u

    @property
    def edge(self) -> float:
        return (self.hi[0] - self.lo[0]) / self.n_cells[0]

    @property
    def h(self) -> float:
        """Cell diameter."""
        return math.sqrt(sum(((self.hi[a] - self.lo[a]) / self.n_cells[a]) ** 2 for a in range(self.dim)))

    def nodes_per_axis(self):
        return tuple(self.deg * self.n_cells[a] + 1 for a in range(self.dim))

    @property
    def n_nodes(self) -> int:
        return int(np.prod(self.nodes_per_axis()))

    @property
    def n_dofs(self) -> int:
        return (self.dim + 1) * self.n_nodes

    @property
    def n_cells_total(self) -> int:
        return int(np.prod(self.n_cells))

    def finalize(self) -> "Workload":
        if self.eps == 0.0:
            self.eps = self.eps_factor * self.h
        return self


def config_2d_single_crack(n: int = 64, n_levels: int = 3, deg: int = 1) -> Workload:
    w = Workload("2d_single_crack", 2, deg, (n, n), n_levels, (-10.0, -10.0), (10.0, 10.0))
    w.cracks = [Crack((0.0, 0.0), (0.0, 1.0), 1.0)]
    return w.finalize()


def config_2d_two_cracks(n: int = 128, n_levels: int = 4, deg: int = 1) -> Workload:
    """Sec. 5.1 (multiple fractures): (0,4)^2, a vertical crack {|x-2.5| <= h/2, 0.8 <= y <= 1.5}
    and a horizontal one {0.5 <= x <= 1.5, |y-3| <= h/2}, E=1e4, nu=0.2, Gc=1, kappa=1e-10,
    eps=h, pressure p(t) = 1e3 t with dt = 1e-2 (p_n = 10 n).  128^2 cells give h = 0.044,
    the eps of the paper's parameter table."""
    w = Workload("2d_two_cracks", 2, deg, (n, n), n_levels, (0.0, 0.0), (4.0, 4.0), E=1e4, nu=0.2, Gc=1.0,
                 kappa=1e-10, pressure=10.0, eps_factor=1.0)
    w.cracks = [Crack((2.5, 1.15), (1.0, 0.0), 0.35, half_width=0.5),
                Crack((1.0, 3.0), (0.0, 1.0), 0.5, half_width=0.5)]
    return w.finalize()


def config_3d_lshape(n: int = 32, n_levels: int = 4, deg: int = 1, loading: str = "displacement") -> Workload:
    """L-shaped panel of Sec. 5.3 as a serving instance: [0,2]^2 minus [1,2]^2 extruded to a depth of 0.5
    (n x n x n/4 cells of edge 2/n), clamped on the face y = 0, no initial crack, E = 1, nu = 0.2,
    Gc = 1e-3.  loading 'displacement' (default): no pressure (p = 0, as in Sec. 5.2/5.3) and a
    vertical displacement prescribed on the strip 1 <= x <= 1.25 of the face y = 1 (the top of the
    lower arm, next to the re-entrant corner), growing to 1e-2 over the load steps; 'pressure': the
    pressure term (phi~^2 p, div w) with p = 1e-3, which with phi = 1 is a normal traction on the free
    faces."""
    disp = loading == "displacement"
    w = Workload("3d_lshape", 3, deg, (n, n, n // 4), n_levels, (0.0, 0.0, 0.0), (2.0, 2.0, 0.5), Gc=1e-3,
                 pressure=0.0 if disp else 1e-3, dirichlet_faces=1 << 2, domain="lshape",
                 load_strip=((1.0, 1.25), 1.0) if disp else None, u_ramp=1e-2 if disp else 0.0)
    return w.finalize()


def config_2d_lshape(n: int = 32, n_levels: int = 4, deg: int = 1, loading: str = "displacement") -> Workload:
    """2D L-shaped panel [0,2]^2 minus [1,2]^2, clamped on y = 0, loaded like config_3d_lshape."""
    disp = loading == "displacement"
    w = Workload("2d_lshape", 2, deg, (n, n), n_levels, (0.0, 0.0), (2.0, 2.0), Gc=1e-3,
                 pressure=0.0 if disp else 1e-3, dirichlet_faces=1 << 2, domain="lshape",
                 load_strip=((1.0, 1.25), 1.0) if disp else None, u_ramp=1e-2 if disp else 0.0)
    return w.finalize()


def config_3d_penny(n: int = 128, deg: int = 1, n_levels: int = 5) -> Workload:
    w = Workload("3d_penny", 3, deg, (n, n, n), n_levels, (-10.0,) * 3, (10.0,) * 3)
    w.cracks = [Crack((0.0, 0.0, 0.0), (0.0, 0.0, 1.0), 1.0)]
    return w.finalize()


def config_3d_penny_si(n: int = 16, deg: int = 1, n_levels: int = 3, pressure: float = 1e7) -> Workload:
    """The penny-crack geometry in SI units (steel-like material in a 1 cm box): coefficients spanning
    about 30 decades, residual entries of order 1e-4 N beside rounding noise of order 1e-20."""
    w = Workload("3d_penny_si", 3, deg, (n, n, n), n_levels, (-5e-3,) * 3, (5e-3,) * 3, E=2.1e11, nu=0.3,
                 Gc=2.7e3, pressure=pressure)
    w.cracks = [Crack((0.0, 0.0, 0.0), (0.0, 0.0, 1.0), 1e-3)]
    return w.finalize()


def config_3d_multi(n: int = 256, deg: int = 1, n_levels: int = 6, eps_factor: float = 2.0,
                    seed: int = SEED) -> Workload:
    rng = np.random.default_rng(seed)
    cracks = []
    for _ in range(8):
        c = rng.uniform(-6.0, 6.0, 3)
        nv = rng.normal(size=3)
        nv /= np.linalg.norm(nv)
        cracks.append(Crack(tuple(c), tuple(nv), float(rng.uniform(1.0, 2.0))))
    w = Workload("3d_multi", 3, deg, (n, n, n), n_levels, (-10.0,) * 3, (10.0,) * 3,
                 eps_factor=eps_factor, cracks=cracks, seed=seed)
    return w.finalize()


def batch_instances(count: int = 256, sizes=(16, 24, 32, 48, 64), seed: int = SEED,
                    coarsest: int = 4) -> list:
    """Independent 3D instances for the batching pattern; levels go down to a coarsest grid of
    at most 'coarsest' cells per edge (N=24 and N=48 stop at 3^3... 6^3 accordingly)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        levels = 1
        m = n
        while m % 2 == 0 and m // 2 >= 2 and m > coarsest:
            m //= 2
            levels += 1
        ncr = int(rng.integers(1, 7))
        cracks = []
        for _ in range(ncr):
            c = rng.uniform(-6.0, 6.0, 3)
            nv = rng.normal(size=3)
            nv /= np.linalg.norm(nv)
            cracks.append(Crack(tuple(c), tuple(nv), float(rng.uniform(0.5, 2.0))))
        w = Workload(f"batch_{i}", 3, 1, (n, n, n), levels, (-10.0,) * 3, (10.0,) * 3,
                     pressure=float(rng.uniform(5e-4, 2e-3)), cracks=cracks, seed=seed + i)
        out.append(w.finalize())
    return out


def small(w: Workload, n, n_levels: int | None = None) -> Workload:
    """Same recipe on an n^dim mesh, or n = cells per axis (eps follows the new h)."""
    cells = (n,) * w.dim if isinstance(n, int) else tuple(int(c) for c in n)
    v = replace(w, n_cells=cells, n_levels=n_levels or w.n_levels, eps=0.0)
    return v.finalize()


# ---------------------------------------------------------------- crack -> initial phase field

def _cell_meets_crack(lo: np.ndarray, hi: np.ndarray, crack: Crack, h: float, dim: int) -> np.ndarray:
    """Vectorised test whether axis-aligned cells [lo, hi] meet the closed crack region
    {|n.(x-c)| <= b h, |x - c - (n.(x-c)) n| <= r} (b = crack.half_width).  Exact for axis-aligned
    normals (interval overlap plus nearest-point distance); otherwise sampled on a 5^dim lattice
    per cell."""
    h = crack.half_width * h
    c = np.asarray(crack.center[:dim], dtype=np.float64)
    nv = np.asarray(crack.normal[:dim], dtype=np.float64)
    nv = nv / np.linalg.norm(nv)
    axis = int(np.argmax(np.abs(nv)))
    if abs(abs(nv[axis]) - 1.0) < 1e-14:
        ok = (lo[:, axis] <= c[axis] + h) & (hi[:, axis] >= c[axis] - h)
        dist2 = np.zeros(lo.shape[0])
        for a in range(dim):
            if a == axis:
                continue
            nearest = np.clip(c[a], lo[:, a], hi[:, a])
            dist2 += (nearest - c[a]) ** 2
        return ok & (dist2 <= crack.radius ** 2 * (1 + 1e-12))
    t = np.linspace(0.0, 1.0, 5)
    grids = np.meshgrid(*([t] * dim), indexing="ij")
    offs = np.stack([g.ravel() for g in grids], axis=1)
    hit = np.zeros(lo.shape[0], dtype=bool)
    for o in offs:
        x = lo + (hi - lo) * o
        s = (x - c) @ nv
        tang = x - c - s[:, None] * nv
        hit |= (np.abs(s) <= h) & (np.einsum("ij,ij->i", tang, tang) <= crack.radius ** 2)
    return hit


def initial_phase_field(w: Workload) -> np.ndarray:
    """phi per node: 0 on all nodes of cells meeting a crack region, 1 elsewhere."""
    dim = w.dim
    n = np.array(w.n_cells)
    edge = (np.array(w.hi) - np.array(w.lo)) / n
    hits = []
    for cr in w.cracks:
        # only cells inside the crack region's bounding box (centre +- (radius + half-thickness))
        reach = cr.radius + cr.half_width * w.h
        c = np.asarray(cr.center[:dim], dtype=np.float64)
        i0 = np.clip(np.floor((c - reach - np.array(w.lo)) / edge).astype(int) - 1, 0, n - 1)
        i1 = np.clip(np.floor((c + reach - np.array(w.lo)) / edge).astype(int) + 1, 0, n - 1)
        axes = [np.arange(i0[a], i1[a] + 1) for a in range(dim)]
        grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
        cidx = np.stack([g.ravel() for g in grids], axis=1)
        lo = np.array(w.lo)[None, :] + cidx * edge[None, :]
        hi = lo + edge[None, :]
        hits.append(cidx[_cell_meets_crack(lo, hi, cr, w.h, dim)])
    phi = np.ones(w.n_nodes)
    npa = np.array(w.nodes_per_axis())
    hc = np.concatenate(hits, axis=0) if hits else np.zeros((0, dim), dtype=int)
    strides = np.cumprod(np.concatenate([[1], npa[:-1]]))
    for off in np.ndindex(*([w.deg + 1] * dim)):
        node = ((hc * w.deg + np.array(off)[None, :]) * strides[None, :]).sum(axis=1)
        phi[node] = 0.0
    return phi


def smooth_displacement(w: Workload, amplitude: float = 1e-3, modes: int = 3,
                        seed: int | None = None) -> np.ndarray:
    """A smooth seeded displacement field (a few low Fourier modes per component), zero on
    the box boundary, used as a synthetic linearisation point."""
    rng = np.random.default_rng(w.seed if seed is None else seed)
    npa = w.nodes_per_axis()
    axes = [np.linspace(0.0, 1.0, npa[a]) for a in range(w.dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
    X = [g.ravel() for g in grids]
    out = []
    for _ in range(w.dim):
        f = np.zeros(w.n_nodes)
        for _m in range(modes):
            k = rng.integers(1, 4, size=w.dim)
            a = rng.normal()
            term = np.full(w.n_nodes, a)
            for ax in range(w.dim):
                term = term * np.sin(math.pi * k[ax] * X[ax])
            f += term
        out.append(amplitude * f)
    return np.concatenate(out)


def initial_state(w: Workload, displacement: str = "zero"):
    """(U, phi_old, phi_tilde) with U = [u | phi]; displacement 'zero' or 'smooth'."""
    phi = initial_phase_field(w)
    if displacement == "smooth":
        u = smooth_displacement(w)
    else:
        u = np.zeros(w.dim * w.n_nodes)
    U = np.concatenate([u, phi])
    return U, phi.copy(), phi.copy()


def random_state(w: Workload, seed: int | None = None):
    """Random smooth-ish state with phi in (0,1) everywhere, for operator parity tests."""
    rng = np.random.default_rng(w.seed if seed is None else seed)
    u = smooth_displacement(w, amplitude=1e-2, seed=int(rng.integers(1 << 30)))
    u = u + 1e-3 * rng.standard_normal(u.shape)
    phi = rng.uniform(0.05, 1.0, w.n_nodes)
    ptil = np.clip(phi + 0.05 * rng.standard_normal(w.n_nodes), 0.0, 1.0)
    return np.concatenate([u, phi]), phi.copy(), ptil


def modulus_field(w: Workload, lattice: int = 6, lo: float = 0.1, hi: float = 1.0,
                  seed: int | None = None) -> np.ndarray:
    """Smooth deterministic per-cell factor on E in [lo, hi] (value noise): seeded uniform values
    on a (lattice+1)^dim grid spanning the box, blended with the smoothstep 3t^2 - 2t^3 and
    sampled at the cell centres.  Returns n_cells values, cells lexicographic (x fastest)."""
    rng = np.random.default_rng(w.seed + 77 if seed is None else seed)
    vals = rng.uniform(lo, hi, size=(lattice + 1,) * w.dim)
    centres = []
    for a in range(w.dim):
        t = (np.arange(w.n_cells[a]) + 0.5) / w.n_cells[a] * lattice
        i0 = np.minimum(np.floor(t).astype(int), lattice - 1)
        f = t - i0
        centres.append((i0, f * f * (3.0 - 2.0 * f)))
    grids = np.meshgrid(*[np.arange(w.n_cells[a]) for a in range(w.dim)][::-1], indexing="ij")[::-1]
    out = np.zeros(grids[0].shape)
    for corner in np.ndindex(*([2] * w.dim)):
        wgt = np.ones(grids[0].shape)
        idx = []
        for a in range(w.dim):
            i0, s_ = centres[a]
            ia = i0[grids[a]]
            sa = s_[grids[a]]
            wgt = wgt * (sa if corner[a] else 1.0 - sa)
            idx.append(ia + corner[a])
        out += wgt * vals[tuple(idx)]
    return out.ravel()


def random_vector(n: int, seed: int = SEED) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(n)


def random_active(w: Workload, fraction: float = 0.1, seed: int = SEED) -> np.ndarray:
    """Random 0/1 indicator per node (a synthetic active set for masking tests)."""
    return (np.random.default_rng(seed).uniform(size=w.n_nodes) < fraction).astype(np.uint8)
