"""Thin ctypes binding of the pff C ABI (include/pff.h), same call names without the prefix.

Argument marshalling only: vectors are torch CUDA tensors (contiguous, on the hierarchy's
device) whose data pointers are passed through; every computation runs in libpff.so.  There is
no CPU fallback: loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpff.so")

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, ENONFINITE, ETIMEOUT, ESTATE = range(8)
STATUS_NAMES = ["PFF_OK", "PFF_EINVAL", "PFF_ENOMEM", "PFF_ECUDA", "PFF_ENOCONV", "PFF_ENONFINITE",
                "PFF_ETIMEOUT", "PFF_ESTATE"]
MASK_UX, MASK_UY, MASK_UZ, MASK_ACTIVE, MASK_PHI_DIR = 1, 2, 4, 8, 16


class Mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("degree", ctypes.c_int), ("n_cells", ctypes.c_int * 3),
                ("n_levels", ctypes.c_int), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("dirichlet_faces", ctypes.c_uint), ("dirichlet_mask", ctypes.c_void_p),
                ("cell_mask", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("nu", ctypes.c_double), ("Gc", ctypes.c_double),
                ("kappa", ctypes.c_double), ("eps", ctypes.c_double), ("pressure", ctypes.c_double),
                ("c_as", ctypes.c_double), ("tol_as", ctypes.c_double),
                ("phi_elastic_factor", ctypes.c_double), ("mg_precision", ctypes.c_int),
                ("cheb_degree", ctypes.c_int), ("cg_steps", ctypes.c_int), ("cheb_safety", ctypes.c_double),
                ("cheb_ratio", ctypes.c_double), ("coarse_rtol", ctypes.c_double),
                ("coarse_maxit", ctypes.c_int), ("seed", ctypes.c_uint64), ("preconditioner", ctypes.c_int),
                ("split", ctypes.c_int), ("tie_scale", ctypes.c_int), ("newton_rtol", ctypes.c_double),
                ("coarse_phi_max", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("res0", ctypes.c_double),
                ("res_final", ctypes.c_double)]


class NewtonInfo(ctypes.Structure):
    _fields_ = [("n_active", ctypes.c_int), ("n_changed", ctypes.c_int), ("res_norm", ctypes.c_double),
                ("converged", ctypes.c_int), ("solve", SolveInfo)]


class LoadInfo(ctypes.Structure):
    _fields_ = [("newton_steps", ctypes.c_int), ("converged", ctypes.c_int), ("gmres_iterations", ctypes.c_int),
                ("last", NewtonInfo)]


PRECOND_FULL, PRECOND_DIAG = 0, 1

# C signatures: name -> (restype, argtypes)
_VP, _I, _D, _I64P = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int64)
SIGNATURES = {
    "pff_default_params": (None, [ctypes.POINTER(Params)]),
    "pff_create_hierarchy": (_I, [ctypes.POINTER(Mesh), ctypes.POINTER(Params), _VP, ctypes.POINTER(_VP)]),
    "pff_destroy_hierarchy": (_I, [_VP]),
    "pff_hierarchy_bytes": (ctypes.c_int64, [ctypes.POINTER(Mesh), _I]),
    "pff_level_info": (_I, [_VP, _I, _I64P, _I64P, ctypes.POINTER(ctypes.c_int)]),
    "pff_set_params": (_I, [_VP, ctypes.POINTER(Params)]),
    "pff_set_modulus": (_I, [_VP, _VP]),
    "pff_set_kernel_variant": (_I, [_VP, _I]),
    "pff_set_state": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "pff_set_dirichlet_values": (_I, [_VP, _VP]),
    "pff_set_active_set": (_I, [_VP, _VP]),
    "pff_get_active_set": (_I, [_VP, _VP]),
    "pff_update_active_set": (_I, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "pff_residual": (_I, [_VP, _VP]),
    "pff_energies": (_I, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "pff_boundary_load": (_I, [_VP, _I, _I, ctypes.POINTER(ctypes.c_double)]),
    "pff_apply_jacobian": (_I, [_VP, _I, _VP, _VP]),
    "pff_apply_jacobian_f32": (_I, [_VP, _I, _VP, _VP]),
    "pff_apply_jacobian_host": (_I, [_VP, _I, _VP, _VP]),
    "pff_diagonal": (_I, [_VP, _I, _I, _VP]),
    "pff_level_state": (_I, [_VP, _I, _VP, _VP, _VP]),
    "pff_restrict": (_I, [_VP, _I, _I, _VP, _VP]),
    "pff_prolongate_add": (_I, [_VP, _I, _I, _VP, _VP]),
    "pff_setup": (_I, [_VP]),
    "pff_eigen_estimates": (_I, [_VP, _I, ctypes.POINTER(ctypes.c_double)]),
    "pff_smooth": (_I, [_VP, _I, _I, _VP, _VP, _I]),
    "pff_coarse_solve": (_I, [_VP, _VP, _VP]),
    "pff_vcycle": (_I, [_VP, _VP, _VP]),
    "pff_gmres_solve": (_I, [_VP, _VP, _VP, _D, _I, _I, ctypes.POINTER(SolveInfo)]),
    "pff_newton_step": (_I, [_VP, _VP, ctypes.POINTER(NewtonInfo)]),
    "pff_load_step": (_I, [_VP, _VP, _VP, _D, _I, ctypes.POINTER(LoadInfo)]),
    "pff_profile": (_I, [_VP, _I]),
    "pff_profile_read": (_I, [_VP, _I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "pff_active_set_noalloc": (_I, [ctypes.POINTER(Mesh), ctypes.POINTER(Params), _VP, _VP, _VP, _VP, _VP,
                                   ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _VP]),
    "pff_batch_create": (_I, [_I, ctypes.POINTER(_VP), _I, ctypes.POINTER(_VP)]),
    "pff_batch_destroy": (_I, [_VP]),
    "pff_batch_submit": (_I, [_VP, _VP, ctypes.POINTER(ctypes.c_int)]),
    "pff_batch_retire": (_I, [_VP, _I]),
    "pff_batch_size": (_I, [_VP]),
    "pff_batch_poll": (_I, [_VP, _I, ctypes.POINTER(NewtonInfo)]),
    "pff_batch_setup": (_I, [_VP]),
    "pff_batch_vcycle": (_I, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
    "pff_batch_gmres_solve": (_I, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _D, _I, ctypes.POINTER(SolveInfo)]),
    "pff_batch_newton_step": (_I, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(NewtonInfo)]),
    "pff_batch_apply_jacobian": (_I, [_VP, _I, _I, ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
    "pff_batch_set_kernel_style": (_I, [_VP, _I]),
    "pff_batch_set_precision_switch": (_I, [_VP, _I]),
    "pff_batch_mg_precisions": (_I, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "pff_batch_tuning": (_I, [_VP, _I, _I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_double)]),
    "pff_batch_last_error": (ctypes.c_char_p, [_VP]),
    "pff_fp32_fma_tflops": (_I, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "pff_launch_count": (ctypes.c_longlong, []),
    "pff_last_error": (ctypes.c_char_p, [_VP]),
}

PROF_APPLY64_FINE, PROF_APPLY64_COARSE, PROF_APPLY32, PROF_VCYCLE = 0, 1, 2, 3

_lib = None


def load(path: str = LIB_PATH):
    """Load libpff.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"pff CUDA library not built ({path}); run __graft_entry__.build()")
        try:
            import torch  # noqa: F401  (loads the CUDA runtime the library links against)
        except ImportError:
            pass
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class PffError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensors passed to pff must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(int(t))


def _check(h, st, where, allow=()):
    if st != OK and st not in allow:
        msg = load().pff_last_error(h).decode() if h else ""
        raise PffError(st, where, msg)
    return st


def default_params(**kw) -> Params:
    p = Params()
    load().pff_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def make_mesh(dim, degree, n_cells, n_levels, lo, hi, dirichlet_faces=0x3F, cell_mask=None,
              dirichlet_mask=None) -> Mesh:
    """cell_mask: optional host uint8 array of the finest level's cells (x fastest), 1 = in the domain.
    dirichlet_mask: optional host uint8 array of the finest level's nodes (MASK_U* / MASK_PHI_DIR bits)."""
    m = Mesh()
    m.dim, m.degree, m.n_levels = dim, degree, n_levels
    for a in range(3):
        m.n_cells[a] = int(n_cells[a]) if a < dim else 1
        m.lo[a] = float(lo[a]) if a < dim else 0.0
        m.hi[a] = float(hi[a]) if a < dim else 1.0
    m.dirichlet_faces = dirichlet_faces
    m.dirichlet_mask = None
    m.cell_mask = None
    if cell_mask is not None:
        import numpy as np
        arr = np.ascontiguousarray(cell_mask, dtype=np.uint8)
        m._cell_mask_keep = arr          # the library copies it during pff_create_hierarchy
        m.cell_mask = arr.ctypes.data
    if dirichlet_mask is not None:
        import numpy as np
        arr = np.ascontiguousarray(dirichlet_mask, dtype=np.uint8)
        m._dirichlet_mask_keep = arr     # copied during pff_create_hierarchy
        m.dirichlet_mask = arr.ctypes.data
    return m


def create_hierarchy(mesh: Mesh, params: Params, stream=None):
    h = ctypes.c_void_p()
    s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0))
    st = load().pff_create_hierarchy(ctypes.byref(mesh), ctypes.byref(params), s, ctypes.byref(h))
    _check(None, st, "pff_create_hierarchy")
    return h


def hierarchy_bytes(mesh: Mesh, restart: int = 30) -> int:
    return int(load().pff_hierarchy_bytes(ctypes.byref(mesh), restart))


def destroy_hierarchy(h):
    return _check(h, load().pff_destroy_hierarchy(h), "pff_destroy_hierarchy")


def level_info(h, level=-1):
    nn, nc = ctypes.c_int64(), ctypes.c_int64()
    npa = (ctypes.c_int * 3)()
    _check(h, load().pff_level_info(h, level, ctypes.byref(nn), ctypes.byref(nc), npa), "pff_level_info")
    return nn.value, nc.value, tuple(npa)


def set_params(h, params: Params):
    return _check(h, load().pff_set_params(h, ctypes.byref(params)), "pff_set_params")


def set_kernel_variant(h, variant: int):
    return _check(h, load().pff_set_kernel_variant(h, variant), "pff_set_kernel_variant")


def set_state(h, U, phi_old, phi_tilde, u_dirichlet=None):
    """u_dirichlet: optional device tensor of prescribed displacements (dim * n_nodes or n_dofs entries,
    the layout of U), read on the Dirichlet displacement DoFs only."""
    return _check(h, load().pff_set_state(h, _ptr(U), _ptr(phi_old), _ptr(phi_tilde), _ptr(u_dirichlet)),
                  "pff_set_state")


def set_dirichlet_values(h, u_dirichlet):
    return _check(h, load().pff_set_dirichlet_values(h, _ptr(u_dirichlet)), "pff_set_dirichlet_values")


def set_active_set(h, active):
    return _check(h, load().pff_set_active_set(h, _ptr(active)), "pff_set_active_set")


def get_active_set(h, active):
    return _check(h, load().pff_get_active_set(h, _ptr(active)), "pff_get_active_set")


def update_active_set(h):
    na, nc = ctypes.c_int(), ctypes.c_int()
    _check(h, load().pff_update_active_set(h, ctypes.byref(na), ctypes.byref(nc)), "pff_update_active_set")
    return na.value, nc.value


def energies(h):
    out = (ctypes.c_double * 2)()
    _check(h, load().pff_energies(h, out), "pff_energies")
    return out[0], out[1]


def boundary_load(h, face: int, component: int) -> float:
    out = ctypes.c_double()
    _check(h, load().pff_boundary_load(h, int(face), int(component), ctypes.byref(out)), "pff_boundary_load")
    return out.value


def set_modulus(h, escale):
    return _check(h, load().pff_set_modulus(h, _ptr(escale)), "pff_set_modulus")


def residual(h, R):
    return _check(h, load().pff_residual(h, _ptr(R)), "pff_residual")


def apply_jacobian(h, level, x, y):
    return _check(h, load().pff_apply_jacobian(h, level, _ptr(x), _ptr(y)), "pff_apply_jacobian")


def apply_jacobian_host(h, level, x, y):
    """x, y: CPU tensors (pinned for overlap) of the level's n_dofs doubles."""
    if hasattr(x, "device") and (x.device.type != "cpu" or y.device.type != "cpu"):
        raise ValueError("apply_jacobian_host takes host (CPU) tensors")
    return _check(h, load().pff_apply_jacobian_host(h, level, _ptr(x), _ptr(y)), "pff_apply_jacobian_host")


def apply_jacobian_f32(h, level, x, y):
    return _check(h, load().pff_apply_jacobian_f32(h, level, _ptr(x), _ptr(y)), "pff_apply_jacobian_f32")


def diagonal(h, level, precision, d):
    return _check(h, load().pff_diagonal(h, level, precision, _ptr(d)), "pff_diagonal")


def level_state(h, level, U=None, phi_tilde=None, mask=None):
    return _check(h, load().pff_level_state(h, level, _ptr(U), _ptr(phi_tilde), _ptr(mask)), "pff_level_state")


def restrict(h, fine_level, precision, r_fine, r_coarse):
    return _check(h, load().pff_restrict(h, fine_level, precision, _ptr(r_fine), _ptr(r_coarse)), "pff_restrict")


def prolongate_add(h, fine_level, precision, e_coarse, x_fine):
    return _check(h, load().pff_prolongate_add(h, fine_level, precision, _ptr(e_coarse), _ptr(x_fine)),
                  "pff_prolongate_add")


def setup(h):
    return _check(h, load().pff_setup(h), "pff_setup")


def eigen_estimates(h, level):
    out = (ctypes.c_double * 4)()
    _check(h, load().pff_eigen_estimates(h, level, out), "pff_eigen_estimates")
    return tuple(out)


def smooth(h, level, precision, b, x, zero_guess=True):
    return _check(h, load().pff_smooth(h, level, precision, _ptr(b), _ptr(x), int(bool(zero_guess))), "pff_smooth")


def coarse_solve(h, b, x):
    return _check(h, load().pff_coarse_solve(h, _ptr(b), _ptr(x)), "pff_coarse_solve")


def vcycle(h, r, z):
    return _check(h, load().pff_vcycle(h, _ptr(r), _ptr(z)), "pff_vcycle")


def gmres_solve(h, b, x, rtol=1e-8, restart=30, maxit=200, allow_noconv=False):
    info = SolveInfo()
    allow = (ENOCONV,) if allow_noconv else ()
    st = load().pff_gmres_solve(h, _ptr(b), _ptr(x), rtol, restart, maxit, ctypes.byref(info))
    _check(h, st, "pff_gmres_solve", allow)
    return info


def newton_step(h, U, allow_noconv=False):
    info = NewtonInfo()
    allow = (ENOCONV,) if allow_noconv else ()
    _check(h, load().pff_newton_step(h, _ptr(U), ctypes.byref(info)), "pff_newton_step", allow)
    return info


def load_step(h, U, phi_prev, pressure: float, max_newton: int = 20, allow_noconv=False):
    info = LoadInfo()
    allow = (ENOCONV,) if allow_noconv else ()
    st = load().pff_load_step(h, _ptr(U), _ptr(phi_prev), float(pressure), int(max_newton), ctypes.byref(info))
    _check(h, st, "pff_load_step", allow)
    return info


def profile(h, enable: bool):
    return _check(h, load().pff_profile(h, int(bool(enable))), "pff_profile")


def profile_read(h, cls: int):
    n, ms = ctypes.c_int(), ctypes.c_double()
    _check(h, load().pff_profile_read(h, cls, ctypes.byref(n), ctypes.byref(ms)), "pff_profile_read")
    return n.value, ms.value


def active_set_noalloc(mesh: Mesh, params: Params, R, U, phi_old, mask, stream=None, cell_mask=None):
    """Allocation-free active-set decision on caller buffers (no hierarchy); returns
    (n_active, n_changed).  cell_mask: device uint8 tensor of the fine cells for a cut domain."""
    na, nc = ctypes.c_int(), ctypes.c_int()
    s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0))
    st = load().pff_active_set_noalloc(ctypes.byref(mesh), ctypes.byref(params), _ptr(cell_mask), _ptr(R), _ptr(U),
                                       _ptr(phi_old), _ptr(mask), ctypes.byref(na), ctypes.byref(nc), s)
    _check(None, st, "pff_active_set_noalloc")
    return na.value, nc.value


def _ptr_array(ts):
    arr = (ctypes.c_void_p * len(ts))()
    for i, t_ in enumerate(ts):
        arr[i] = _ptr(t_).value
    return arr


def _bcheck(b, st, where, allow=()):
    if st != OK and st not in allow:
        msg = load().pff_batch_last_error(b).decode() if b else ""
        raise PffError(st, where, msg)
    return st


def batch_create(hierarchies=(), restart=30):
    arr = (ctypes.c_void_p * max(1, len(hierarchies)))(*[h.value for h in hierarchies])
    b = ctypes.c_void_p()
    st = load().pff_batch_create(len(hierarchies), arr if hierarchies else None, restart, ctypes.byref(b))
    _check(None, st, "pff_batch_create")
    return b


def batch_submit(b, h) -> int:
    """Append a hierarchy to a live batch; returns its index."""
    idx = ctypes.c_int()
    _bcheck(b, load().pff_batch_submit(b, h, ctypes.byref(idx)), "pff_batch_submit")
    return idx.value


def batch_retire(b, index: int):
    return _bcheck(b, load().pff_batch_retire(b, int(index)), "pff_batch_retire")


def batch_size(b) -> int:
    return int(load().pff_batch_size(b))


def batch_poll(b, index: int) -> NewtonInfo:
    info = NewtonInfo()
    _bcheck(b, load().pff_batch_poll(b, int(index), ctypes.byref(info)), "pff_batch_poll")
    return info


def batch_destroy(b):
    return _bcheck(b, load().pff_batch_destroy(b), "pff_batch_destroy")


def batch_setup(b):
    return _bcheck(b, load().pff_batch_setup(b), "pff_batch_setup")


def batch_vcycle(b, rs, zs):
    return _bcheck(b, load().pff_batch_vcycle(b, _ptr_array(rs), _ptr_array(zs)), "pff_batch_vcycle")


def batch_gmres_solve(b, rhs, xs, rtol=1e-8, maxit=200, allow_noconv=False):
    infos = (SolveInfo * len(rhs))()
    allow = (ENOCONV,) if allow_noconv else ()
    st = load().pff_batch_gmres_solve(b, _ptr_array(rhs), _ptr_array(xs), rtol, maxit, infos)
    _bcheck(b, st, "pff_batch_gmres_solve", allow)
    return list(infos)


def batch_newton_step(b, Us, allow_noconv=False):
    infos = (NewtonInfo * len(Us))()
    allow = (ENOCONV,) if allow_noconv else ()
    _bcheck(b, load().pff_batch_newton_step(b, _ptr_array(Us), infos), "pff_batch_newton_step", allow)
    return list(infos)


def batch_apply_jacobian(b, level, precision, xs, ys):
    """y_i = G~_i x_i on 'level' (-1: each instance's finest) of every instance; precision 64 or 32."""
    return _bcheck(b, load().pff_batch_apply_jacobian(b, level, precision, _ptr_array(xs), _ptr_array(ys)),
                   "pff_batch_apply_jacobian")


def batch_set_kernel_style(b, style: int):
    return _bcheck(b, load().pff_batch_set_kernel_style(b, style), "pff_batch_set_kernel_style")


def batch_set_precision_switch(b, iterations: int):
    return _bcheck(b, load().pff_batch_set_precision_switch(b, int(iterations)), "pff_batch_set_precision_switch")


def batch_mg_precisions(b, n: int):
    out = (ctypes.c_int * n)()
    _bcheck(b, load().pff_batch_mg_precisions(b, out), "pff_batch_mg_precisions")
    return list(out)


def batch_tuning(b, level: int, precision: int):
    """(style, ctas_per_sm, ms) chosen by the batch's autotuner for a level (-1: finest) and precision."""
    st, c, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _bcheck(b, load().pff_batch_tuning(b, level, precision, ctypes.byref(st), ctypes.byref(c), ctypes.byref(ms)),
            "pff_batch_tuning")
    return st.value, c.value, ms.value


def batch_last_error(b) -> str:
    return load().pff_batch_last_error(b).decode()


def fp32_fma_tflops(stream=None) -> float:
    """Measured FP32 FMA rate of the GPU (TFLOP/s), the arithmetic roofline of the df64 operators."""
    out = ctypes.c_double()
    s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0))
    _check(None, load().pff_fp32_fma_tflops(s, ctypes.byref(out)), "pff_fp32_fma_tflops")
    return out.value


def launch_count() -> int:
    return int(load().pff_launch_count())


def last_error(h) -> str:
    return load().pff_last_error(h).decode()
