"""ctypes binding of libhx (include/hx.h, include/hx_loads.h): same names,
argument marshalling only.

Device vectors are torch CUDA tensors (contiguous, float64 for HX_FP64 or
float32 for HX_FP32); their data pointers and the current torch stream are
handed to the C ABI. Every operation runs in libhx's CUDA kernels: there is no
CPU or PyTorch fallback, and importing a function whose library is missing
raises immediately.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import inputs as _inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhx.so")

HX_OK, HX_ERR_ARG, HX_ERR_CUDA, HX_ERR_NONINVERTIBLE, HX_ERR_NOT_READY = 0, 1, 2, 3, 4
HX_ERR_TIMEOUT, HX_ERR_NOT_CONVERGED, HX_ERR_NAN, HX_ERR_UNSUPPORTED = 5, 6, 7, 8
HX_CNH, HX_INH, HX_FIBER = 0, 1, 2
HX_FP64, HX_FP32 = 0, 1
HX_RECOMPUTE, HX_CACHE_F, HX_CACHE_TENSORS, HX_SPATIAL_TENSORS = 0, 1, 2, 3
STATUS_NAMES = {0: "HX_OK", 1: "HX_ERR_ARG", 2: "HX_ERR_CUDA", 3: "HX_ERR_NONINVERTIBLE", 4: "HX_ERR_NOT_READY",
                5: "HX_ERR_TIMEOUT", 6: "HX_ERR_NOT_CONVERGED", 7: "HX_ERR_NAN", 8: "HX_ERR_UNSUPPORTED"}
STORAGE_NAMES = {HX_RECOMPUTE: "recompute", HX_CACHE_F: "cache_F", HX_CACHE_TENSORS: "cache_tensors",
                 HX_SPATIAL_TENSORS: "spatial_tensors"}

# every symbol the header declares
EXPORTS = ["hx_create", "hx_destroy", "hx_set_stream", "hx_last_error", "hx_sync", "hx_setup_mesh",
           "hx_destroy_mesh", "hx_mesh_info", "hx_node_coords", "hx_apply_bytes", "hx_precompute_qp",
           "hx_residual", "hx_tangent_apply", "hx_tangent_apply_host", "hx_diagonal", "hx_chebyshev_smooth",
           "hx_estimate_lambda_max", "hx_cg_solve", "hx_body_force", "hx_newton_solve", "hx_material_eval", "hx_mg_create",
           "hx_mg_destroy", "hx_mg_info", "hx_mg_setup", "hx_mg_vcycle", "hx_mg_transfer", "hx_mg_cg_solve", "hx_fibre_dispersion", "hx_batch_create",
           "hx_batch_destroy", "hx_batch_tangent_apply", "hx_measure_fma_peak", "hx_launch_count",
           "hx_autotune", "hx_set_apply_variant", "hx_chebyshev_smooth_noalloc", "hx_traction_load",
           "hx_set_wait_test", "hx_set_scatter_mode", "hx_set_host_apply_slabs", "hx_mg_level", "hx_mg_coarse_iters", "hx_batch_cg_solve"]


class HxError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")


class hx_material(C.Structure):
    _fields_ = [("law", C.c_int32), ("mu", C.c_double), ("lambda_", C.c_double), ("kappa", C.c_double),
                ("k1", C.c_double), ("k2", C.c_double), ("a", C.c_double), ("b", C.c_double), ("phi", C.c_double)]


class hx_mesh_desc(C.Structure):
    _fields_ = [("n_elem", C.c_int32), ("p", C.c_int32), ("geo_degree", C.c_int32), ("n_nodes", C.c_int64),
                ("geo_nodes", C.c_void_p), ("n_geo_nodes", C.c_int64), ("geo_conn", C.c_void_p),
                ("dof_conn", C.c_void_p), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dirichlet", C.c_void_p), ("fibre_frames", C.c_void_p)]


class hx_cg_options(C.Structure):
    _fields_ = [("degree", C.c_int32), ("lambda_max", C.c_double), ("smoothing_range", C.c_double),
                ("precond_prec", C.c_int32), ("use_graph", C.c_int32)]


class hx_newton_options(C.Structure):
    _fields_ = [("eps_abs", C.c_double), ("eps_rel", C.c_double), ("max_newton", C.c_int32),
                ("storage", C.c_int32), ("cg_degree", C.c_int32), ("smoothing_range", C.c_double),
                ("precond_prec", C.c_int32), ("cg_tol", C.c_double), ("cg_max_iter", C.c_int32),
                ("lambda_iters", C.c_int32), ("mg", C.c_void_p)]


class hx_mg_options(C.Structure):
    _fields_ = [("smoother_degree", C.c_int32), ("smoothing_range", C.c_double), ("coarse_degree", C.c_int32),
                ("coarse_range", C.c_double), ("precond_prec", C.c_int32), ("storage", C.c_int32),
                ("lambda_iters", C.c_int32), ("min_degree", C.c_int32), ("coarse_weight", C.c_double),
                ("h_levels", C.c_int32), ("coarse_cg_iters", C.c_int32), ("coarse_cg_tol", C.c_double)]


class hx_newton_report(C.Structure):
    _fields_ = [("newton_iters", C.c_int32), ("cg_iters", C.c_int32), ("res0", C.c_double), ("res", C.c_double),
                ("converged", C.c_int32)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libhx.so (built by __graft_entry__.build() or build.py)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libhx.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        P, I32, I64, D, U64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_uint64
        sig = {
            "hx_create": (I32, [C.POINTER(P), C.c_int, P]),
            "hx_destroy": (None, [P]),
            "hx_set_stream": (I32, [P, P]),
            "hx_last_error": (C.c_char_p, [P]),
            "hx_sync": (I32, [P, C.c_int]),
            "hx_setup_mesh": (I32, [P, C.POINTER(hx_mesh_desc), C.POINTER(hx_material), C.POINTER(P)]),
            "hx_destroy_mesh": (None, [P]),
            "hx_mesh_info": (I32, [P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64)]),
            "hx_node_coords": (I32, [P, P]),
            "hx_apply_bytes": (I32, [P, I32, I32, C.POINTER(D)]),
            "hx_precompute_qp": (I32, [P, P, I32, I32]),
            "hx_residual": (I32, [P, P, P, I32]),
            "hx_tangent_apply": (I32, [P, P, P, I32]),
            "hx_tangent_apply_host": (I32, [P, P, P, I32]),
            "hx_diagonal": (I32, [P, P, I32]),
            "hx_chebyshev_smooth": (I32, [P, P, P, P, I32, D, D, I32, I32]),
            "hx_estimate_lambda_max": (I32, [P, P, I32, U64, C.POINTER(D)]),
            "hx_cg_solve": (I32, [P, P, P, D, I32, C.POINTER(hx_cg_options), C.POINTER(I32), C.POINTER(D)]),
            "hx_body_force": (I32, [P, C.POINTER(D), P]),
            "hx_material_eval": (I32, [P, I32, I32, I32, C.c_int64, P, P, P, P, P]),
            "hx_mg_create": (I32, [P, C.POINTER(hx_mg_options), C.POINTER(P)]),
            "hx_mg_destroy": (None, [P]),
            "hx_mg_info": (I32, [P, C.POINTER(I32), C.POINTER(I32)]),
            "hx_mg_setup": (I32, [P, P]),
            "hx_mg_vcycle": (I32, [P, P, P]),
            "hx_mg_transfer": (I32, [P, I32, I32, P, P, I32]),
            "hx_mg_cg_solve": (I32, [P, P, P, D, I32, I32, C.POINTER(I32), C.POINTER(D)]),
            "hx_newton_solve": (I32, [P, P, P, C.POINTER(hx_newton_options), C.POINTER(hx_newton_report)]),
            "hx_fibre_dispersion": (I32, [D, D, C.POINTER(D)]),
            "hx_batch_create": (I32, [P, C.POINTER(P), I32, C.POINTER(P)]),
            "hx_batch_destroy": (None, [P]),
            "hx_batch_tangent_apply": (I32, [P, C.POINTER(P), C.POINTER(P), I32]),
            "hx_measure_fma_peak": (I32, [P, I32, C.POINTER(D)]),
            "hx_launch_count": (U64, [P, I32]),
            "hx_autotune": (I32, [P, I32, P, P, I32, C.POINTER(I32), C.POINTER(D)]),
            "hx_set_apply_variant": (I32, [P, I32, I32, I32]),
            "hx_chebyshev_smooth_noalloc": (I32, [P, P, P, P, I32, D, D, I32, I32]),
            "hx_traction_load": (I32, [C.POINTER(hx_mesh_desc), I32, P, I32, C.POINTER(D), P]),
            "hx_set_wait_test": (I32, [P, I32, C.c_int64]),
            "hx_set_scatter_mode": (I32, [P, I32]),
            "hx_set_host_apply_slabs": (I32, [P, I32]),
            "hx_mg_level": (I32, [P, I32, C.POINTER(I32), C.POINTER(I32), C.POINTER(I32), C.POINTER(I32)]),
            "hx_mg_coarse_iters": (I32, [P, C.POINTER(I32)]),
            "hx_batch_cg_solve": (I32, [P, C.POINTER(P), C.POINTER(P), D, I32, I32, D, I32, I32, C.POINTER(I32),
                                        C.POINTER(D)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return _lib


def _check(st, ctx=None, what=""):
    if st != HX_OK:
        msg = lib().hx_last_error(ctx).decode() if ctx else what
        raise HxError(st, msg or what)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


# ---------------------------------------------------------------------------
# thin wrappers with the C names (torch tensors in, statuses raised)
# ---------------------------------------------------------------------------

def hx_create(device: int = 0, stream=None):
    ctx = C.c_void_p()
    st = lib().hx_create(C.byref(ctx), int(device), stream if stream is not None else _stream())
    _check(st, None, "hx_create")
    return ctx


def hx_destroy(ctx):
    lib().hx_destroy(ctx)


def hx_sync(ctx, timeout_ms: int = -1):
    _check(lib().hx_sync(ctx, int(timeout_ms)), ctx)


def hx_fibre_dispersion(a: float, b: float):
    H = (C.c_double * 3)()
    _check(lib().hx_fibre_dispersion(a, b, H), None, "hx_fibre_dispersion")
    return tuple(H)


def material_struct(mat: dict) -> hx_material:
    return hx_material(int(mat["law"]), mat.get("mu", 1.0), mat.get("lam", 0.0), mat.get("kappa", 0.0),
                       mat.get("k1", 0.0), mat.get("k2", 0.0), mat.get("a", 0.0), mat.get("b", 1.0),
                       mat.get("phi", 0.0))


def _mesh_desc(m: "_inputs.MeshInput", structured: bool = True):
    """hx_mesh_desc of a MeshInput and the arrays it points into (keep them
    alive while the descriptor is used). For boxes the structured numbering
    is used (no connectivity array) unless structured=False."""
    keep = {}
    geo = np.ascontiguousarray(m.geo_nodes, dtype=np.float64)
    gconn = np.ascontiguousarray(m.geo_conn, dtype=np.int32)
    keep["geo"], keep["gconn"] = geo, gconn
    d = hx_mesh_desc()
    d.n_elem = m.n_elem
    d.p = m.p
    d.geo_degree = m.geo_degree
    d.n_nodes = m.n_nodes
    d.geo_nodes = geo.ctypes.data
    d.n_geo_nodes = geo.shape[0]
    d.geo_conn = gconn.ctypes.data
    if m.box is not None and structured:
        d.dof_conn = None
        d.nx, d.ny, d.nz = m.box
    else:
        dconn = np.ascontiguousarray(m.dof_conn, dtype=np.int32)
        keep["dconn"] = dconn
        d.dof_conn = dconn.ctypes.data
    if m.dirichlet is not None and np.any(m.dirichlet):
        dm = np.ascontiguousarray(m.dirichlet, dtype=np.uint8)
        keep["dm"] = dm
        d.dirichlet = dm.ctypes.data
    if m.frames is not None:
        fr = np.ascontiguousarray(m.frames, dtype=np.float64)
        keep["fr"] = fr
        d.fibre_frames = fr.ctypes.data
    return d, keep


def hx_setup_mesh(ctx, mesh_input: "_inputs.MeshInput", mat: dict, structured: bool = True):
    """Upload a MeshInput. For boxes the structured numbering is used (no
    connectivity array) unless structured=False."""
    d, keep = _mesh_desc(mesh_input, structured)
    ms = material_struct(mat)
    out = C.c_void_p()
    st = lib().hx_setup_mesh(ctx, C.byref(d), C.byref(ms), C.byref(out))
    _check(st, ctx)
    return out


def hx_traction_load(mesh_input: "_inputs.MeshInput", faces, traction=None, pressure=None, out=None,
                     structured: bool = True):
    """Neumann load vector of a dead traction on boundary faces (host; see
    include/hx_loads.h): faces [n, 2] (element, local face); either a constant
    traction vector or a pressure along the inward reference normal. Returns
    the [3 n_nodes] FP64 numpy vector `out` (new zeros if None) with the load
    added."""
    if (traction is None) == (pressure is None):
        raise ValueError("give exactly one of traction and pressure")
    d, keep = _mesh_desc(mesh_input, structured)
    fc = np.ascontiguousarray(np.asarray(faces, dtype=np.int32).reshape(-1, 2))
    mode = 0 if traction is not None else 1
    val = np.ascontiguousarray(np.asarray(traction if mode == 0 else [pressure, 0.0, 0.0],
                                          dtype=np.float64).reshape(3))
    f = np.zeros(3 * mesh_input.n_nodes) if out is None else out
    if f.dtype != np.float64 or not f.flags.c_contiguous or f.size != 3 * mesh_input.n_nodes:
        raise ValueError("out must be a contiguous float64 array of 3*n_nodes entries")
    _check(lib().hx_traction_load(C.byref(d), int(fc.shape[0]), fc.ctypes.data, mode,
                                  val.ctypes.data_as(C.POINTER(C.c_double)), f.ctypes.data),
           None, "hx_traction_load")
    return f


def hx_destroy_mesh(mesh):
    lib().hx_destroy_mesh(mesh)


def hx_mesh_info(mesh):
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().hx_mesh_info(mesh, C.byref(a), C.byref(b), C.byref(c)), None, "hx_mesh_info")
    return a.value, b.value, c.value


def hx_node_coords(ctx, mesh, X):
    _check(lib().hx_node_coords(mesh, _ptr(X)), ctx)


def hx_apply_bytes(mesh, storage, prec):
    b = C.c_double()
    _check(lib().hx_apply_bytes(mesh, storage, prec, C.byref(b)), None, "hx_apply_bytes")
    return b.value


def _prec_of(t):
    import torch
    if t.dtype == torch.float64:
        return HX_FP64
    if t.dtype == torch.float32:
        return HX_FP32
    raise TypeError(f"unsupported dtype {t.dtype}")


def _vec_ok(t, n):
    if not t.is_cuda or not t.is_contiguous() or t.numel() != n:
        raise ValueError("expected a contiguous CUDA tensor with %d entries" % n)


def hx_precompute_qp(ctx, mesh, u, store_prec, storage):
    _check(lib().hx_precompute_qp(mesh, _ptr(u), int(store_prec), int(storage)), ctx)


def hx_residual(ctx, mesh, u, r):
    _check(lib().hx_residual(mesh, _ptr(u), _ptr(r), _prec_of(u)), ctx)


def hx_tangent_apply(ctx, mesh, du, out):
    _check(lib().hx_tangent_apply(mesh, _ptr(du), _ptr(out), _prec_of(du)), ctx)


def hx_tangent_apply_host(ctx, mesh, du_host, out_host, prec):
    """du_host/out_host: pinned (or pageable) CPU torch tensors or numpy arrays."""
    def addr(a):
        return C.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data)
    _check(lib().hx_tangent_apply_host(mesh, addr(du_host), addr(out_host), int(prec)), ctx)


def hx_diagonal(ctx, mesh, diag):
    _check(lib().hx_diagonal(mesh, _ptr(diag), _prec_of(diag)), ctx)


def hx_chebyshev_smooth(ctx, mesh, rhs, x, inv_diag, degree, lambda_max, smoothing_range, zero_initial=False):
    _check(lib().hx_chebyshev_smooth(mesh, _ptr(rhs), _ptr(x), _ptr(inv_diag), int(degree), float(lambda_max),
                                     float(smoothing_range), int(bool(zero_initial)), _prec_of(x)), ctx)


def hx_chebyshev_smooth_noalloc(ctx, mesh, rhs, x, inv_diag, degree, lambda_max, smoothing_range,
                                zero_initial=False):
    """hx_chebyshev_smooth for callers that cannot allocate device memory: the
    scratch vectors live in the library's static device array (meshes up to
    1,048,576 DoFs)."""
    _check(lib().hx_chebyshev_smooth_noalloc(mesh, _ptr(rhs), _ptr(x), _ptr(inv_diag), int(degree),
                                             float(lambda_max), float(smoothing_range), int(bool(zero_initial)),
                                             _prec_of(x)), ctx)


def hx_estimate_lambda_max(ctx, mesh, inv_diag, iters=50, seed=1):
    out = C.c_double()
    _check(lib().hx_estimate_lambda_max(mesh, _ptr(inv_diag), int(iters), int(seed), C.byref(out)), ctx)
    return out.value


def hx_cg_solve(ctx, mesh, rhs, x, tol, max_iter, degree, lambda_max, smoothing_range, precond_prec,
                use_graph=True):
    opt = hx_cg_options(int(degree), float(lambda_max), float(smoothing_range), int(precond_prec), int(use_graph))
    it = C.c_int32()
    rel = C.c_double()
    st = lib().hx_cg_solve(mesh, _ptr(rhs), _ptr(x), float(tol), int(max_iter), C.byref(opt), C.byref(it),
                           C.byref(rel))
    if st not in (HX_OK, HX_ERR_NOT_CONVERGED):
        _check(st, ctx)
    return it.value, rel.value, st


def hx_material_eval(ctx, mesh, G, H, prec, form=0, elem=0):
    """S, P, dP ([n, 3, 3] FP64 tensors on the device) of the mesh's law at
    gradients G and directions H ([n, 3, 3] FP64 device tensors)."""
    import torch
    n = G.shape[0]
    G = G.reshape(n, 9).contiguous()
    H = H.reshape(n, 9).contiguous()
    S, P, dP = (torch.empty_like(G) for _ in range(3))
    _check(lib().hx_material_eval(mesh, int(elem), int(form), int(prec), int(n), _ptr(G), _ptr(H), _ptr(S), _ptr(P),
                                  _ptr(dP)), ctx)
    return S.reshape(n, 3, 3), P.reshape(n, 3, 3), dP.reshape(n, 3, 3)


class Multigrid:
    """hp-multigrid preconditioner on a structured-box Mesh (hx_mg_*): p-levels
    down to degree 1, then up to h_levels h-coarsenings; the coarsest level
    runs FP64 Jacobi-CG (coarse_cg_iters > 0) or Chebyshev-Jacobi."""

    def __init__(self, mesh, smoother_degree=3, smoothing_range=15.0, coarse_degree=20, coarse_range=200.0,
                 precond_prec=HX_FP32, storage=HX_CACHE_TENSORS, lambda_iters=20, min_degree=1, coarse_weight=1.0,
                 h_levels=0, coarse_cg_iters=0, coarse_cg_tol=1e-3):
        self.mesh = mesh
        opt = hx_mg_options(int(smoother_degree), float(smoothing_range), int(coarse_degree), float(coarse_range),
                            int(precond_prec), int(storage), int(lambda_iters), int(min_degree),
                            float(coarse_weight), int(h_levels), int(coarse_cg_iters), float(coarse_cg_tol))
        h = C.c_void_p()
        _check(lib().hx_mg_create(mesh.handle, C.byref(opt), C.byref(h)), mesh.ctx)
        self.handle = h
        self.prec = precond_prec

    def levels(self):
        n = C.c_int32()
        d = (C.c_int32 * 16)()
        _check(lib().hx_mg_info(self.handle, C.byref(n), d), self.mesh.ctx)
        return [d[i] for i in range(n.value)]

    def level(self, l):
        """(degree, nx, ny, nz) of level l."""
        v = [C.c_int32() for _ in range(4)]
        _check(lib().hx_mg_level(self.handle, int(l), *[C.byref(x) for x in v]), self.mesh.ctx)
        return tuple(x.value for x in v)

    def coarse_iters(self):
        it = C.c_int32()
        _check(lib().hx_mg_coarse_iters(self.handle, C.byref(it)), self.mesh.ctx)
        return it.value

    def setup(self, u):
        _check(lib().hx_mg_setup(self.handle, _ptr(u)), self.mesh.ctx)

    def vcycle(self, b, x):
        _check(lib().hx_mg_vcycle(self.handle, _ptr(b), _ptr(x)), self.mesh.ctx)

    def transfer(self, level, direction, src, dst):
        _check(lib().hx_mg_transfer(self.handle, int(level), int(direction), _ptr(src), _ptr(dst), _prec_of(src)),
               self.mesh.ctx)

    def cg_solve(self, rhs, x, tol, max_iter, use_graph=True):
        it = C.c_int32()
        rel = C.c_double()
        st = lib().hx_mg_cg_solve(self.handle, _ptr(rhs), _ptr(x), float(tol), int(max_iter), int(use_graph),
                                  C.byref(it), C.byref(rel))
        if st not in (HX_OK, HX_ERR_NOT_CONVERGED):
            _check(st, self.mesh.ctx)
        return it.value, rel.value, st

    def close(self):
        if self.handle:
            lib().hx_mg_destroy(self.handle)
            self.handle = None


def hx_body_force(ctx, mesh, b, f):
    bb = (C.c_double * 3)(*[float(x) for x in b])
    _check(lib().hx_body_force(mesh, bb, _ptr(f)), ctx)


def hx_newton_solve(ctx, mesh, u, f_ext=None, eps_abs=1e-10, eps_rel=1e-8, max_newton=20, storage=HX_CACHE_TENSORS,
                    cg_degree=5, smoothing_range=15.0, precond_prec=HX_FP32, cg_tol=1e-6, cg_max_iter=5000,
                    lambda_iters=30, mg=None):
    """Newton's method (Alg. 1); returns (report dict, status). u is updated in
    place; HX_ERR_NOT_CONVERGED is returned, not raised. mg: a Multigrid on the
    same mesh to precondition the linear solves."""
    opt = hx_newton_options(float(eps_abs), float(eps_rel), int(max_newton), int(storage), int(cg_degree),
                            float(smoothing_range), int(precond_prec), float(cg_tol), int(cg_max_iter),
                            int(lambda_iters), mg.handle if mg is not None else None)
    rep = hx_newton_report()
    st = lib().hx_newton_solve(mesh, _ptr(u), _ptr(f_ext) if f_ext is not None else None, C.byref(opt),
                               C.byref(rep))
    if st not in (HX_OK, HX_ERR_NOT_CONVERGED):
        _check(st, ctx)
    return {"newton_iters": rep.newton_iters, "cg_iters": rep.cg_iters, "res0": rep.res0, "res": rep.res,
            "converged": bool(rep.converged)}, st


def hx_set_apply_variant(ctx, mesh, prec, storage, variant):
    _check(lib().hx_set_apply_variant(mesh, int(prec), int(storage), int(variant)), ctx)


HX_SCATTER_ATOMIC, HX_SCATTER_ORDERED = 0, 1


def hx_set_host_apply_slabs(ctx, mesh, slabs):
    """0: hx_tangent_apply_host copies whole vectors; 1 (default): z-slabs
    with overlapped copies where they apply; 2..8: at most that many slabs."""
    _check(lib().hx_set_host_apply_slabs(mesh, int(slabs)), ctx)


def hx_set_scatter_mode(ctx, mesh, mode):
    """HX_SCATTER_ATOMIC (default) or HX_SCATTER_ORDERED (bitwise repeatable
    assembly through an element buffer and an ordered node gather)."""
    _check(lib().hx_set_scatter_mode(mesh, int(mode)), ctx)


def hx_set_wait_test(ctx, mesh, skip_stage_copies, wait_limit_cycles=0):
    """Test hook: staged applies issue no bulk copy, so their bounded wait
    runs out after wait_limit_cycles (0 = default) and hx_sync reports
    HX_ERR_TIMEOUT."""
    _check(lib().hx_set_wait_test(mesh, int(bool(skip_stage_copies)), int(wait_limit_cycles)), ctx)


def hx_autotune(ctx, mesh, du, out, reps=10):
    """Pick the fastest tile shape of the apply for the mesh's current cache."""
    best = C.c_int32()
    t = (C.c_double * 6)()
    _check(lib().hx_autotune(mesh, _prec_of(du), _ptr(du), _ptr(out), int(reps), C.byref(best), t), ctx)
    return best.value, list(t)


def hx_batch_create(ctx, meshes):
    """Group Mesh objects (same context and law) for one-launch applies."""
    arr = (C.c_void_p * len(meshes))(*[m.handle.value for m in meshes])
    out = C.c_void_p()
    _check(lib().hx_batch_create(ctx, arr, len(meshes), C.byref(out)), ctx)
    return out


def hx_batch_destroy(batch):
    lib().hx_batch_destroy(batch)


def hx_batch_tangent_apply(ctx, batch, dus, outs):
    """out_i = K_i du_i for every mesh of the batch in one persistent launch."""
    a = (C.c_void_p * len(dus))(*[d.data_ptr() for d in dus])
    b = (C.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
    _check(lib().hx_batch_tangent_apply(batch, a, b, _prec_of(dus[0])), ctx)


def hx_batch_cg_solve(ctx, batch, rhss, xs, tol, max_iter, degree, smoothing_range, precond_prec, use_graph=True):
    """Batched FP64 CG with a per-mesh Chebyshev-Jacobi preconditioner, all
    meshes in lockstep (one CUDA graph per iteration). Returns (iters list,
    relative residual list, status); HX_ERR_NOT_CONVERGED and HX_ERR_NAN (a
    mesh's breakdown: its relative residual is NaN) are returned, not
    raised."""
    n = len(xs)
    a = (C.c_void_p * n)(*[t.data_ptr() for t in rhss])
    b = (C.c_void_p * n)(*[t.data_ptr() for t in xs])
    it = (C.c_int32 * n)()
    rel = (C.c_double * n)()
    st = lib().hx_batch_cg_solve(batch, a, b, float(tol), int(max_iter), int(degree), float(smoothing_range),
                                 int(precond_prec), int(bool(use_graph)), it, rel)
    if st not in (HX_OK, HX_ERR_NOT_CONVERGED, HX_ERR_NAN):
        _check(st, ctx)
    return list(it), list(rel), st


def hx_measure_fma_peak(ctx, prec):
    f = C.c_double()
    _check(lib().hx_measure_fma_peak(ctx, int(prec), C.byref(f)), ctx)
    return f.value


def hx_launch_count(ctx, reset=False):
    return int(lib().hx_launch_count(ctx, int(bool(reset))))


# ---------------------------------------------------------------------------
# convenience object used by tests and the benchmark
# ---------------------------------------------------------------------------

class Mesh:
    """A mesh on the device with its context; holds the C handles."""

    def __init__(self, mesh_input, mat: dict, device: int = 0, structured: bool = True, ctx=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.own_ctx = ctx is None
        self.ctx = ctx if ctx is not None else hx_create(device)
        self.input = mesh_input
        self.mat = mat
        self.handle = hx_setup_mesh(self.ctx, mesh_input, mat, structured=structured)
        self.n_nodes, self.n_elem, self.n_qp = hx_mesh_info(self.handle)
        self.n_dofs = 3 * self.n_nodes

    def zeros(self, prec=HX_FP64):
        dt = self.torch.float64 if prec == HX_FP64 else self.torch.float32
        return self.torch.zeros(self.n_dofs, dtype=dt, device=self.device)

    def node_coords(self):
        X = self.torch.zeros(self.n_nodes * 3, dtype=self.torch.float64, device=self.device)
        hx_node_coords(self.ctx, self.handle, X)
        return X.view(-1, 3)

    def precompute(self, u, store_prec=HX_FP64, storage=HX_CACHE_TENSORS):
        hx_precompute_qp(self.ctx, self.handle, u, store_prec, storage)

    def residual(self, u, out=None):
        out = self.torch.empty_like(u) if out is None else out
        hx_residual(self.ctx, self.handle, u, out)
        return out

    def apply(self, du, out=None):
        out = self.torch.empty_like(du) if out is None else out
        hx_tangent_apply(self.ctx, self.handle, du, out)
        return out

    def diagonal(self, prec=HX_FP64):
        d = self.zeros(prec)
        hx_diagonal(self.ctx, self.handle, d)
        return d

    def apply_bytes(self, storage, prec):
        return hx_apply_bytes(self.handle, storage, prec)

    def sync(self, timeout_ms=-1):
        hx_sync(self.ctx, timeout_ms)

    def close(self):
        if self.handle:
            hx_destroy_mesh(self.handle)
            self.handle = None
        if self.own_ctx and self.ctx:
            hx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# autograd: R(u) with the hand-written tangent as its backward
# ---------------------------------------------------------------------------

def _residual_function():
    import torch

    class HxResidual(torch.autograd.Function):
        """r = R(u) (forward: hx_precompute_qp at u, then hx_residual); the
        backward applies K(u)^T g = K(u) g with hx_tangent_apply (the tangent
        of a hyperelastic residual is symmetric)."""

        @staticmethod
        def forward(ctx, u, mesh, storage):
            prec = _prec_of(u)
            u64 = u if u.dtype == torch.float64 else u.double()
            mesh.precompute(u64.contiguous(), prec, storage)
            r = torch.empty_like(u)
            hx_residual(mesh.ctx, mesh.handle, u.contiguous(), r)
            ctx.mesh = mesh
            return r

        @staticmethod
        def backward(ctx, g):
            out = torch.empty_like(g)
            hx_tangent_apply(ctx.mesh.ctx, ctx.mesh.handle, g.contiguous(), out)
            return out, None, None

    return HxResidual


_HxResidual = None


def residual_autograd(mesh: Mesh, u, storage=HX_CACHE_TENSORS):
    """Differentiable R(u) on a Mesh; u is a CUDA tensor (float64 or float32)."""
    global _HxResidual
    if _HxResidual is None:
        _HxResidual = _residual_function()
    return _HxResidual.apply(u, mesh, storage)
