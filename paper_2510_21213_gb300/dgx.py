"""Thin Python binding of the C ABI in include/dg_poisson.h.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libdgx.so. Device arrays are torch CUDA tensors (contiguous,
float64 unless stated); the binding passes their data pointers and the
current torch stream. There is no CPU fallback: importing this module fails
loudly if the library has not been built.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libdgx.so")

DG_OK = 0
DG_ERR_INVALID_ARG = -1
DG_ERR_CUDA = -2
DG_ERR_NOT_CONVERGED = -3
DG_ERR_BREAKDOWN = -4
DG_ERR_NONFINITE = -5
DG_ERR_TIMEOUT = -6
DG_ERR_NO_MEMORY = -7
DG_ERR_UNSUPPORTED = -8

DG_PREC_FP64 = 0
DG_PREC_MIXED = 1
DG_PREC_MIXED_LEARNED = 2
DG_BC_DIRECT = 0
DG_BC_GAUSSSUM = 1
DG_SMOOTH_JACOBI = 0
DG_SMOOTH_SCHWARZ = 1


class dg_mesh_desc(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("n", C.c_int32 * 3), ("p", C.c_int32)]


class dg_solver_opts(C.Structure):
    _fields_ = [
        ("precision", C.c_int32),
        ("rtol", C.c_double),
        ("max_iter", C.c_int32),
        ("penalty_eps", C.c_double),
        ("penalty_form", C.c_int32),
        ("bc_route", C.c_int32),
        ("bc_tol", C.c_double),
        ("batch", C.c_int32),
        ("smoother", C.c_int32),
        ("smoother_degree", C.c_int32),
        ("cheb_range", C.c_double),
        ("inner_rtol", C.c_double),
        ("nn_weights_path", C.c_char_p),
        ("verbose", C.c_int32),
        ("coarse_penalty", C.c_int32),
        ("coarse_smoother_degree", C.c_int32),
        ("p1_smoother", C.c_int32),
        ("gauss_construction", C.c_int32),
        ("tc_smoother", C.c_int32),
        ("nn_use_net", C.c_int32),
        ("device_loop", C.c_int32),
    ]


class dg_solve_stats(C.Structure):
    _fields_ = [
        ("iters", C.c_int32),
        ("outer_refinements", C.c_int32),
        ("status", C.c_int32),
        ("used_fallback", C.c_int32),
        ("rel_residual", C.c_double),
        ("guess_rel_residual", C.c_double),
        ("self_energy", C.c_double),
    ]


class dg_info(C.Structure):
    _fields_ = [
        ("Nq", C.c_int64),
        ("levels", C.c_int32),
        ("level_n", C.c_int32 * 16),
        ("level_p", C.c_int32 * 16),
        ("coarse_dofs", C.c_int32),
        ("n_gauss", C.c_int32),
        ("gauss_rmin", C.c_double),
        ("gauss_rmax", C.c_double),
        ("gauss_relerr", C.c_double),
        ("sigma", C.c_double * 3),
        ("workspace_bytes", C.c_int64),
        ("n_gauss_fp32", C.c_int32),
        ("gauss_relerr_fp32", C.c_double),
        ("batch", C.c_int32),
    ]


_lib = None


def load():
    """Load libdgx.so (built by paper_2510_21213_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2510_21213_gb300.build.build() first")
    lib = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    lib.dg_default_opts.argtypes = [C.POINTER(dg_solver_opts)]
    lib.dg_default_opts.restype = None
    lib.dg_poisson_setup.argtypes = [C.POINTER(dg_mesh_desc), C.POINTER(dg_solver_opts), C.POINTER(vp)]
    lib.dg_get_info.argtypes = [vp, C.POINTER(dg_info)]
    lib.dg_node_coords.argtypes = [vp, vp, vp]
    lib.dg_mesh_node_coords.argtypes = [C.POINTER(dg_mesh_desc), vp, vp]
    lib.dg_mesh_node_coords.restype = C.c_int
    lib.dg_pair_solve_batch.argtypes = [vp, vp, C.c_int64, vp, vp, vp]
    lib.dg_exchange_build.argtypes = [vp, vp, C.c_int32, vp, vp, vp, vp, vp]
    lib.dg_exchange_build_range.argtypes = [vp, vp, C.c_int32, C.c_int64, C.c_int64, vp, vp, vp, vp]
    lib.dg_exchange_build_range.restype = C.c_int
    lib.dg_ace_apply.argtypes = [vp, vp, C.c_int64, vp, vp]
    lib.dg_ace_apply.restype = C.c_int
    lib.dg_jk_apply.argtypes = [vp, vp, C.c_int32, vp, C.c_int64, vp, vp, vp, vp]
    lib.dg_jk_apply.restype = C.c_int
    lib.dg_apply_transfer.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, vp, vp, C.c_int64, vp]
    lib.dg_apply_transfer.restype = C.c_int
    lib.dg_form_rhs.argtypes = [vp, vp, C.c_int64, vp, vp]
    lib.dg_form_rhs.restype = C.c_int
    lib.dg_gauss_sum.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int32, C.c_int32, vp, vp, vp, vp]
    lib.dg_gauss_sum.restype = C.c_int
    lib.dg_octree_refine.argtypes = [vp, C.c_double, C.c_int32, DENSITY_FN, vp, C.c_int32, vp, vp]
    lib.dg_octree_refine.restype = C.c_int
    lib.dg_octree_faces.argtypes = [vp, vp, C.c_int32, vp, vp, vp]
    lib.dg_octree_faces.restype = C.c_int
    lib.dg_octree_apply.argtypes = [vp, vp, C.c_int32, C.c_int32, C.c_double, vp, vp, C.c_int64, vp]
    lib.dg_octree_apply.restype = C.c_int
    lib.dg_octree_setup.argtypes = [vp, vp, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_int32, C.c_int32,
                                    C.c_int32, C.POINTER(vp)]
    lib.dg_octree_setup.restype = C.c_int
    lib.dg_octree_destroy.argtypes = [vp]
    lib.dg_octree_destroy.restype = None
    lib.dg_octree_error_detail.argtypes = [vp]
    lib.dg_octree_error_detail.restype = C.c_char_p
    lib.dg_octree_node_coords.argtypes = [vp, vp, vp, vp]
    lib.dg_octree_node_coords.restype = C.c_int
    lib.dg_octree_operator.argtypes = [vp, vp, vp, C.c_int64, vp]
    lib.dg_octree_operator.restype = C.c_int
    lib.dg_octree_precond.argtypes = [vp, vp, vp, C.c_int64, vp]
    lib.dg_octree_precond.restype = C.c_int
    lib.dg_octree_solve.argtypes = [vp, vp, C.c_int64, vp, vp, vp]
    lib.dg_octree_solve.restype = C.c_int
    lib.dg_octree_exchange_build.argtypes = [vp, vp, C.c_int32, vp, vp, vp, vp, vp]
    lib.dg_octree_exchange_build.restype = C.c_int
    lib.dg_apply_operator.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, C.c_int64, vp]
    lib.dg_boundary_data.argtypes = [vp, C.c_int32, vp, C.c_int64, vp, C.POINTER(C.c_int64), vp]
    lib.dg_apply_smoother.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, C.c_int64, vp]
    lib.dg_apply_patch_solves.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, C.c_int64, vp]
    lib.dg_exchange_build_multi.argtypes = [vp, vp, vp, C.c_int32, vp, vp, vp, vp, vp, C.c_int32, vp]
    lib.dg_exchange_build_multi.restype = C.c_int
    lib.dg_release_cached_handles.argtypes = []
    lib.dg_release_cached_handles.restype = None
    lib.dg_autotune_batch.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32)]
    lib.dg_autotune_batch.restype = C.c_int
    lib.dg_kernel_launch_count.argtypes = []
    lib.dg_kernel_launch_count.restype = C.c_int64
    lib.dg_destroy.argtypes = [vp]
    lib.dg_destroy.restype = None
    lib.dg_error_string.argtypes = [C.c_int]
    lib.dg_error_string.restype = C.c_char_p
    lib.dg_last_error_detail.argtypes = [vp]
    lib.dg_last_error_detail.restype = C.c_char_p
    lib.dg_nn_set_params.argtypes = [vp, vp]
    lib.dg_nn_get_params.argtypes = [vp, vp]
    lib.dg_nn_forward.argtypes = [vp, vp, vp, C.c_int64, C.c_int32, vp]
    lib.dg_nn_backward.argtypes = [vp, vp, vp, vp, C.c_int64, vp]
    lib.dg_nn_adam.argtypes = [vp, vp, C.c_float, C.c_float, C.c_float, C.c_float, vp]
    lib.dg_nn_train_step.argtypes = [vp, vp, vp, C.c_int64, C.c_float, vp, vp]
    lib.dg_nn_guess.argtypes = [vp, vp, C.c_int64, C.c_int32, vp, vp, vp]
    for name in ("dg_poisson_setup", "dg_get_info", "dg_node_coords", "dg_pair_solve_batch", "dg_exchange_build",
                 "dg_apply_operator", "dg_boundary_data", "dg_apply_smoother", "dg_nn_set_params", "dg_nn_get_params",
                 "dg_nn_forward", "dg_nn_backward", "dg_nn_adam", "dg_nn_train_step", "dg_nn_guess"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


class DGError(RuntimeError):
    def __init__(self, code, where, detail=""):
        self.code = code
        msg = load().dg_error_string(code).decode()
        super().__init__(f"{where}: {msg} ({code}) {detail}".strip())


def _check(code, where, handle=None, allow=()):
    if code != DG_OK and code not in allow:
        detail = load().dg_last_error_detail(handle).decode() if handle else ""
        raise DGError(code, where, detail)
    return code


def _stream_ptr(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dev_ptr(t, dtype=None):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def dg_default_opts(**overrides):
    o = dg_solver_opts()
    load().dg_default_opts(C.byref(o))
    for k, v in overrides.items():
        if k == "nn_weights_path" and v is not None:
            v = str(v).encode()
        setattr(o, k, v)
    return o


def dg_poisson_setup(lo, hi, n, p, opts=None):
    """Returns a handle (c_void_p). lo, hi: 3 floats; n: int or 3 ints; p: degree."""
    if np.isscalar(n):
        n = (n, n, n)
    m = dg_mesh_desc((C.c_double * 3)(*lo), (C.c_double * 3)(*hi), (C.c_int32 * 3)(*n), int(p))
    if opts is None:
        opts = dg_default_opts()
    h = C.c_void_p()
    _check(load().dg_poisson_setup(C.byref(m), C.byref(opts), C.byref(h)), "dg_poisson_setup")
    return h


def dg_get_info(h):
    info = dg_info()
    _check(load().dg_get_info(h, C.byref(info)), "dg_get_info", h)
    return info


def dg_node_coords(h):
    """(xyz [Nq, 3], W [Nq]) numpy arrays, element-blocked order."""
    Nq = dg_get_info(h).Nq
    xyz = np.empty((Nq, 3), dtype=np.float64)
    w = np.empty(Nq, dtype=np.float64)
    _check(load().dg_node_coords(h, xyz.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p)), "dg_node_coords", h)
    return xyz, w


def dg_mesh_node_coords(lo, hi, n, p):
    """(xyz [Nq, 3], W [Nq]) of a mesh without a handle (host computation)."""
    if np.isscalar(n):
        n = (n, n, n)
    m = dg_mesh_desc((C.c_double * 3)(*lo), (C.c_double * 3)(*hi), (C.c_int32 * 3)(*n), int(p))
    Nq = int(n[0] * n[1] * n[2] * (p + 1) ** 3)
    xyz = np.empty((Nq, 3), dtype=np.float64)
    w = np.empty(Nq, dtype=np.float64)
    _check(load().dg_mesh_node_coords(C.byref(m), xyz.ctypes.data_as(C.c_void_p), w.ctypes.data_as(C.c_void_p)),
           "dg_mesh_node_coords")
    return xyz, w


def _stats_list(arr):
    return [{"iters": s.iters, "outer_refinements": s.outer_refinements, "status": s.status,
             "used_fallback": s.used_fallback, "rel_residual": s.rel_residual,
             "guess_rel_residual": s.guess_rel_residual, "self_energy": s.self_energy} for s in arr]


def dg_pair_solve_batch(h, f, v=None, stream=None, allow_unconverged=False):
    """f: CUDA float64 [B, Nq]. Returns (v, stats)."""
    import torch

    B = f.shape[0]
    if v is None:
        v = torch.empty_like(f)
    st = (dg_solve_stats * max(B, 1))()
    allow = (DG_ERR_NOT_CONVERGED, DG_ERR_BREAKDOWN, DG_ERR_NONFINITE) if allow_unconverged else ()
    code = load().dg_pair_solve_batch(h, _dev_ptr(f, torch.float64), B, _dev_ptr(v, torch.float64),
                                      C.cast(st, C.c_void_p), _stream_ptr(stream))
    _check(code, "dg_pair_solve_batch", h, allow)
    return v, _stats_list(st[:B])


def dg_exchange_build(h, psi, stream=None, allow_unconverged=False):
    """psi: CUDA float64 [N, Nq]. Returns (K [N, N] numpy, E_H, E_X, stats)."""
    import torch

    N = psi.shape[0]
    K = np.empty((N, N), dtype=np.float64)
    eh = C.c_double()
    ex = C.c_double()
    P = N * (N + 1) // 2 + 1
    st = (dg_solve_stats * P)()
    allow = (DG_ERR_NOT_CONVERGED, DG_ERR_BREAKDOWN, DG_ERR_NONFINITE) if allow_unconverged else ()
    code = load().dg_exchange_build(h, _dev_ptr(psi, torch.float64), N, K.ctypes.data_as(C.c_void_p), C.byref(eh),
                                    C.byref(ex), C.cast(st, C.c_void_p), _stream_ptr(stream))
    _check(code, "dg_exchange_build", h, allow)
    return K, eh.value, ex.value, _stats_list(st[:P])


def dg_exchange_build_range(h, psi, src_begin, src_end, stream=None, allow_unconverged=False):
    """Sources [src_begin, src_end) of an exchange build (0 = Hartree, then the
    pairs): (partial K [N, N] numpy, E_H or 0, stats)."""
    import torch

    N = psi.shape[0]
    K = np.empty((N, N), dtype=np.float64)
    eh = C.c_double()
    n = max(int(src_end) - int(src_begin), 1)
    st = (dg_solve_stats * n)()
    allow = (DG_ERR_NOT_CONVERGED, DG_ERR_BREAKDOWN, DG_ERR_NONFINITE) if allow_unconverged else ()
    code = load().dg_exchange_build_range(h, _dev_ptr(psi, torch.float64), N, int(src_begin), int(src_end),
                                          K.ctypes.data_as(C.c_void_p), C.byref(eh), C.cast(st, C.c_void_p),
                                          _stream_ptr(stream))
    _check(code, "dg_exchange_build_range", h, allow)
    return K, eh.value, _stats_list(st[:int(src_end) - int(src_begin)])


def dg_ace_apply(h, U, stream=None):
    """Compressed exchange operator of the last whole exchange build applied to
    U (CUDA float64 [m, Nq]); returns V_X^ACE U, same shape."""
    import torch

    Y = torch.empty_like(U)
    _check(load().dg_ace_apply(h, _dev_ptr(U, torch.float64), U.shape[0], _dev_ptr(Y, torch.float64),
                               _stream_ptr(stream)), "dg_ace_apply", h)
    return Y


def dg_jk_apply(h, psi, U, hartree=True, exchange=True, stream=None, allow_unconverged=False):
    """Hartree and exchange actions on trial functions U (CUDA float64 [m, Nq])
    for orbitals psi (CUDA float64 [N, Nq]): (J U or None, X U or None, stats),
    J u = v_H u and X u = -sum_j psi_j v_(psi_j u)."""
    import torch

    N, m = psi.shape[0], U.shape[0]
    JU = torch.empty_like(U) if hartree else None
    XU = torch.empty_like(U) if exchange else None
    n = (1 if hartree else 0) + (N * m if exchange else 0)
    st = (dg_solve_stats * max(n, 1))()
    allow = (DG_ERR_NOT_CONVERGED, DG_ERR_BREAKDOWN, DG_ERR_NONFINITE) if allow_unconverged else ()
    code = load().dg_jk_apply(h, _dev_ptr(psi, torch.float64), N, _dev_ptr(U, torch.float64), m,
                              _dev_ptr(JU, torch.float64) if hartree else None,
                              _dev_ptr(XU, torch.float64) if exchange else None, C.cast(st, C.c_void_p),
                              _stream_ptr(stream))
    _check(code, "dg_jk_apply", h, allow)
    return JU, XU, _stats_list(st[:n])


def dg_apply_operator(h, u, level=0, out=None, stream=None):
    """u: CUDA [B, Nq_level] float64 or float32; returns A u."""
    import torch

    if out is None:
        out = torch.empty_like(u)
    fp32 = 1 if u.dtype == torch.float32 else 0
    code = load().dg_apply_operator(h, level, fp32, _dev_ptr(u), _dev_ptr(out, u.dtype), u.shape[0],
                                    _stream_ptr(stream))
    _check(code, "dg_apply_operator", h)
    return out


DENSITY_FN = C.CFUNCTYPE(None, C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_double), C.c_void_p)


def dg_octree_refine(lo, hi, n, p, rho, delta, max_level):
    """Leaves (level, ix, iy, iz) [E, 4] of the octree that refines the root
    grid by the density indicator; rho maps points [k, 3] to values [k]
    (host only)."""
    if np.isscalar(n):
        n = (n, n, n)
    desc = dg_mesh_desc((C.c_double * 3)(*lo), (C.c_double * 3)(*hi), (C.c_int32 * 3)(*n), int(p))

    def cb(xyz, k, out, _user):
        pts = np.ctypeslib.as_array(xyz, shape=(int(k), 3))
        np.ctypeslib.as_array(out, shape=(int(k),))[:] = np.asarray(rho(pts), dtype=np.float64)

    fn = DENSITY_FN(cb)
    cnt = C.c_int32()
    _check(load().dg_octree_refine(C.byref(desc), delta, max_level, fn, None, 0, None, C.byref(cnt)),
           "dg_octree_refine")
    leaves = np.empty((cnt.value, 4), dtype=np.int32)
    _check(load().dg_octree_refine(C.byref(desc), delta, max_level, fn, None, cnt.value,
                                   leaves.ctypes.data_as(C.c_void_p), C.byref(cnt)), "dg_octree_refine")
    return leaves


def dg_octree_faces(lo, hi, n, p, leaves):
    """Face connectivity of octree leaves [E, 4]: (kind [E, 6], nb [E, 6, 4],
    pos [E, 6]) as documented for dg_octree_faces (host only)."""
    if np.isscalar(n):
        n = (n, n, n)
    desc = dg_mesh_desc((C.c_double * 3)(*lo), (C.c_double * 3)(*hi), (C.c_int32 * 3)(*n), int(p))
    leaves = np.ascontiguousarray(leaves, dtype=np.int32)
    E = leaves.shape[0]
    kind = np.empty((E, 6), dtype=np.int32)
    nb = np.empty((E, 6, 4), dtype=np.int32)
    pos = np.empty((E, 6), dtype=np.int32)
    _check(load().dg_octree_faces(C.byref(desc), leaves.ctypes.data_as(C.c_void_p), E,
                                  kind.ctypes.data_as(C.c_void_p), nb.ctypes.data_as(C.c_void_p),
                                  pos.ctypes.data_as(C.c_void_p)), "dg_octree_faces")
    return kind, nb, pos


def dg_octree_apply(lo, hi, n, p, leaves, u, penalty_form=0, penalty_eps=0.125, stream=None):
    """A u on octree leaves [E, 4] for u (CUDA float64 [B, E (p+1)^3])."""
    import torch

    if np.isscalar(n):
        n = (n, n, n)
    leaves = np.ascontiguousarray(leaves, dtype=np.int32)
    # the C entry takes no lengths: u must be [B, n_leaves * (p+1)^3] for this leaf set
    if leaves.ndim != 2 or leaves.shape[1] != 4:
        raise ValueError(f"leaves must be [n_leaves, 4], got {tuple(leaves.shape)}")
    width = leaves.shape[0] * (int(p) + 1) ** 3
    if u.ndim != 2 or u.shape[1] != width:
        raise ValueError(f"u must be [B, {width}] (n_leaves * (p+1)^3), got {tuple(u.shape)}")
    desc = dg_mesh_desc((C.c_double * 3)(*lo), (C.c_double * 3)(*hi), (C.c_int32 * 3)(*n), int(p))
    out = torch.empty_like(u)
    _check(load().dg_octree_apply(C.byref(desc), leaves.ctypes.data_as(C.c_void_p), leaves.shape[0], penalty_form,
                                  penalty_eps, _dev_ptr(u, torch.float64), _dev_ptr(out, torch.float64), u.shape[0],
                                  _stream_ptr(stream)), "dg_octree_apply")
    return out


def dg_gauss_sum(rmin, rmax, tol, construction=0):
    """The Gaussian sum 1/r ~ sum_k c_k exp(-alpha_k r^2) the setup builds for
    [rmin, rmax] at relative tolerance tol (host only): (c, alpha, relerr)."""
    n = C.c_int32()
    err = C.c_double()
    _check(load().dg_gauss_sum(rmin, rmax, tol, construction, 0, C.byref(n), C.byref(err), None, None),
           "dg_gauss_sum")
    c = np.empty(n.value)
    a = np.empty(n.value)
    _check(load().dg_gauss_sum(rmin, rmax, tol, construction, n.value, C.byref(n), C.byref(err),
                               c.ctypes.data_as(C.c_void_p), a.ctypes.data_as(C.c_void_p)), "dg_gauss_sum")
    return c, a, err.value


def dg_form_rhs(h, f, stream=None):
    """Right-hand sides b = 4 pi W f + Nitsche load of g(f) of the solves for
    sources f (CUDA float64 [B, Nq]); returns b, same shape."""
    import torch

    b = torch.empty_like(f)
    _check(load().dg_form_rhs(h, _dev_ptr(f, torch.float64), f.shape[0], _dev_ptr(b, torch.float64),
                              _stream_ptr(stream)), "dg_form_rhs", h)
    return b


def dg_apply_transfer(h, x, level, direction, nq_out, stream=None):
    """Grid transfer between levels `level` and `level` + 1: direction 0
    prolongs x [B, Nq_(level+1)] to [B, Nq_level], direction 1 restricts x
    [B, Nq_level] to [B, Nq_(level+1)] (CUDA float64 or float32); nq_out is
    the output level's node count."""
    import torch

    out = torch.empty((x.shape[0], int(nq_out)), dtype=x.dtype, device=x.device)
    fp32 = 1 if x.dtype == torch.float32 else 0
    code = load().dg_apply_transfer(h, level, direction, fp32, _dev_ptr(x), _dev_ptr(out, x.dtype), x.shape[0],
                                    _stream_ptr(stream))
    _check(code, "dg_apply_transfer", h)
    return out


def dg_apply_smoother(h, r, level=0, out=None, stream=None):
    """r: CUDA [B, Nq_level] float64 or float32; returns M r (smoother preconditioner)."""
    import torch

    if out is None:
        out = torch.empty_like(r)
    fp32 = 1 if r.dtype == torch.float32 else 0
    code = load().dg_apply_smoother(h, level, fp32, _dev_ptr(r), _dev_ptr(out, r.dtype), r.shape[0],
                                    _stream_ptr(stream))
    _check(code, "dg_apply_smoother", h)
    return out


def dg_apply_patch_solves(h, r, level=0, n_elem=None, p_level=None, stream=None):
    """r: CUDA [B, Nq_level] float64 or float32; returns the Schwarz patch
    solutions zp [B, E_level, (p_level+3)^3] (no gather)."""
    import torch

    mp3 = (p_level + 3) ** 3
    zp = torch.empty((r.shape[0], n_elem, mp3), dtype=r.dtype, device=r.device)
    fp32 = 1 if r.dtype == torch.float32 else 0
    code = load().dg_apply_patch_solves(h, level, fp32, _dev_ptr(r), _dev_ptr(zp, r.dtype), r.shape[0],
                                        _stream_ptr(stream))
    _check(code, "dg_apply_patch_solves", h)
    return zp


def dg_boundary_data(h, f, route=DG_BC_GAUSSSUM, stream=None):
    """f: CUDA float64 [B, Nq]. Returns g [B, n_face_nodes] (faces -x,+x,-y,+y,-z,+z)."""
    import torch

    nf = C.c_int64()
    lib = load()
    _check(lib.dg_boundary_data(h, route, None, 0, None, C.byref(nf), None), "dg_boundary_data", h)
    g = torch.empty((f.shape[0], nf.value), dtype=torch.float64, device=f.device)
    _check(lib.dg_boundary_data(h, route, _dev_ptr(f, torch.float64), f.shape[0], _dev_ptr(g), C.byref(nf),
                                _stream_ptr(stream)), "dg_boundary_data", h)
    return g


def dg_exchange_build_multi(systems, opts=None, lanes=4, stream=None, allow_unconverged=False):
    """systems: list of (lo, hi, n, p, psi) with psi a CUDA float64 [N, Nq] tensor.
    Returns lists (K, E_H, E_X, stats) per system."""
    import torch

    nsys = len(systems)
    meshes = (dg_mesh_desc * nsys)()
    psis = (C.c_void_p * nsys)()
    Ns = (C.c_int32 * nsys)()
    Ks, Kp, sts, stp = [], (C.c_void_p * nsys)(), [], (C.c_void_p * nsys)()
    for i, (lo, hi, n, p, psi) in enumerate(systems):
        if np.isscalar(n):
            n = (n, n, n)
        meshes[i] = dg_mesh_desc((C.c_double * 3)(*lo), (C.c_double * 3)(*hi), (C.c_int32 * 3)(*n), int(p))
        psis[i] = _dev_ptr(psi, torch.float64)
        N = psi.shape[0]
        Ns[i] = N
        K = np.empty((N, N), dtype=np.float64)
        Ks.append(K)
        Kp[i] = K.ctypes.data_as(C.c_void_p)
        st = (dg_solve_stats * (N * (N + 1) // 2 + 1))()
        sts.append(st)
        stp[i] = C.cast(st, C.c_void_p)
    eh = (C.c_double * nsys)()
    ex = (C.c_double * nsys)()
    if opts is None:
        opts = dg_default_opts()
    allow = (DG_ERR_NOT_CONVERGED, DG_ERR_BREAKDOWN, DG_ERR_NONFINITE) if allow_unconverged else ()
    code = load().dg_exchange_build_multi(C.cast(meshes, C.c_void_p), C.cast(psis, C.c_void_p), C.cast(Ns, C.c_void_p),
                                          nsys, C.byref(opts), C.cast(Kp, C.c_void_p), C.cast(eh, C.c_void_p),
                                          C.cast(ex, C.c_void_p), C.cast(stp, C.c_void_p), lanes, _stream_ptr(stream))
    _check(code, "dg_exchange_build_multi", None, allow)
    return Ks, list(eh), list(ex), [_stats_list(st) for st in sts]


def dg_release_cached_handles():
    load().dg_release_cached_handles()


def dg_autotune_batch(h, max_sources=0):
    b = C.c_int32()
    _check(load().dg_autotune_batch(h, max_sources, C.byref(b)), "dg_autotune_batch", h)
    return b.value


# ---------------------------------------------------------------------------
# learned initial guess (include/dg_nn.h)
# ---------------------------------------------------------------------------
DG_NN_NPARAM = 31170
DG_NN_HIDDEN = 32
# parameter layout: (name, shape) in order; W[t][ci][co] with t = 9 (dz+1) + 3 (dy+1) + (dx+1)
NN_LAYOUT = (("W1", (3, 3, 3, 2, 32)), ("b1", (32,)), ("W2", (3, 3, 3, 32, 32)), ("b2", (32,)),
             ("W3", (3, 3, 3, 32, 2)), ("b3", (2,)))
WEIGHTS_DIR = os.path.join(_PKG, "weights")


def nn_pack(params):
    """dict of arrays (shapes of NN_LAYOUT) -> flat float32 [DG_NN_NPARAM]."""
    flat = np.concatenate([np.asarray(params[k], dtype=np.float64).reshape(-1) for k, _ in NN_LAYOUT])
    assert flat.size == DG_NN_NPARAM
    return flat.astype(np.float32)


def nn_unpack(flat):
    """flat [DG_NN_NPARAM] -> dict of float64 arrays with the shapes of NN_LAYOUT."""
    flat = np.asarray(flat, dtype=np.float64).reshape(-1)
    out, o = {}, 0
    for k, shp in NN_LAYOUT:
        n = int(np.prod(shp))
        out[k] = flat[o:o + n].reshape(shp)
        o += n
    return out


def save_nn_weights(path, flat, p):
    """Writes the weights file read by dg_poisson_setup (header "DGNN", 1, nparam, p)."""
    flat = np.asarray(flat, dtype="<f4").reshape(-1)
    if flat.size != DG_NN_NPARAM:
        raise ValueError("wrong parameter count")
    with open(path, "wb") as fh:
        fh.write(b"DGNN")
        fh.write(np.array([1, DG_NN_NPARAM, int(p)], dtype="<i4").tobytes())
        fh.write(flat.tobytes())


def load_nn_weights(path):
    """(flat float32 params, p) of a weights file."""
    with open(path, "rb") as fh:
        raw = fh.read()
    if raw[:4] != b"DGNN":
        raise ValueError("not a DGNN weights file")
    ver, n, p = np.frombuffer(raw[4:16], dtype="<i4")
    if ver != 1 or n != DG_NN_NPARAM:
        raise ValueError("unsupported weights file")
    return np.frombuffer(raw[16:16 + 4 * n], dtype="<f4").copy(), int(p)


def default_nn_weights(p):
    """Path of the packaged weights for degree p, or None."""
    path = os.path.join(WEIGHTS_DIR, f"dgnn_p{int(p)}.bin")
    return path if os.path.exists(path) else None


def dg_nn_set_params(h, flat):
    flat = np.ascontiguousarray(np.asarray(flat, dtype=np.float32).reshape(-1))
    if flat.size != DG_NN_NPARAM:
        raise ValueError("wrong parameter count")
    _check(load().dg_nn_set_params(h, flat.ctypes.data_as(C.c_void_p)), "dg_nn_set_params", h)


def dg_nn_get_params(h):
    flat = np.empty(DG_NN_NPARAM, dtype=np.float32)
    _check(load().dg_nn_get_params(h, flat.ctypes.data_as(C.c_void_p)), "dg_nn_get_params", h)
    return flat


def dg_nn_forward(h, x, save_act=False, stream=None):
    """x: CUDA float32 [n_elem, (p+1)^3, 2]. Returns the network output, same shape."""
    import torch

    out = torch.empty_like(x)
    _check(load().dg_nn_forward(h, _dev_ptr(x, torch.float32), _dev_ptr(out, torch.float32), x.shape[0],
                                int(bool(save_act)), _stream_ptr(stream)), "dg_nn_forward", h)
    return out


def dg_nn_backward(h, x, gout, stream=None):
    """Gradient [DG_NN_NPARAM] (CUDA float32) of sum(gout * net(x)); needs dg_nn_forward(x, save_act=True)."""
    import torch

    grad = torch.empty(DG_NN_NPARAM, dtype=torch.float32, device=x.device)
    _check(load().dg_nn_backward(h, _dev_ptr(x, torch.float32), _dev_ptr(gout, torch.float32),
                                 _dev_ptr(grad, torch.float32), x.shape[0], _stream_ptr(stream)), "dg_nn_backward", h)
    return grad


def dg_nn_adam(h, grad, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    import torch

    _check(load().dg_nn_adam(h, _dev_ptr(grad, torch.float32), lr, beta1, beta2, eps, _stream_ptr(stream)),
           "dg_nn_adam", h)


def dg_nn_train_step(h, f, v, lr, stream=None):
    """One training step on sources f with target potentials v (CUDA float64 [B, Nq]).
    Returns (loss, per-source losses)."""
    import torch

    B = f.shape[0]
    if v.shape != f.shape:
        raise ValueError("f and v must have the same shape")
    loss = np.zeros(B + 1, dtype=np.float64)
    _check(load().dg_nn_train_step(h, _dev_ptr(f, torch.float64), _dev_ptr(v, torch.float64), B, lr,
                                   loss.ctypes.data_as(C.c_void_p), _stream_ptr(stream)), "dg_nn_train_step", h)
    return float(loss[0]), loss[1:].copy()


def dg_nn_guess(h, f, use_net=True, stream=None):
    """Initial guess of the solver for sources f (CUDA float64 [B, Nq]): (x0 [B, Nq], rel residuals [B])."""
    import torch

    B = f.shape[0]
    x0 = torch.empty_like(f)
    rel = np.zeros(max(B, 1), dtype=np.float64)
    _check(load().dg_nn_guess(h, _dev_ptr(f, torch.float64), B, int(bool(use_net)), _dev_ptr(x0, torch.float64),
                              rel.ctypes.data_as(C.c_void_p), _stream_ptr(stream)), "dg_nn_guess", h)
    return x0, rel[:B].copy()


def dg_kernel_launch_count():
    return int(load().dg_kernel_launch_count())


def dg_destroy(h):
    if h:
        load().dg_destroy(h)


class PoissonSolver:
    """Owns one handle: a uniform box mesh and its solver settings."""

    def __init__(self, lo, hi, n, p, **opts):
        self.opts = dg_default_opts(**opts)
        self.h = dg_poisson_setup(lo, hi, n, p, self.opts)
        self.info = dg_get_info(self.h)

    @property
    def Nq(self):
        return self.info.Nq

    def node_coords(self):
        return dg_node_coords(self.h)

    def solve(self, f, **kw):
        return dg_pair_solve_batch(self.h, f, **kw)

    def exchange_build(self, psi, **kw):
        return dg_exchange_build(self.h, psi, **kw)

    def exchange_build_range(self, psi, src_begin, src_end, **kw):
        return dg_exchange_build_range(self.h, psi, src_begin, src_end, **kw)

    def jk_apply(self, psi, U, **kw):
        return dg_jk_apply(self.h, psi, U, **kw)

    def apply(self, u, level=0):
        return dg_apply_operator(self.h, u, level)

    def smoother(self, r, level=0):
        return dg_apply_smoother(self.h, r, level)

    def patch_solves(self, r, level=0):
        n1 = self.info.level_p[level] + 1
        return dg_apply_patch_solves(self.h, r, level, r.shape[1] // n1 ** 3, n1 - 1)

    def boundary_data(self, f, route=DG_BC_GAUSSSUM):
        return dg_boundary_data(self.h, f, route)

    def close(self):
        if self.h:
            dg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class OctreeSolver:
    """Owns one octree solver handle (dg_octree_setup): the leaves [E, 4] of an
    octree over the root grid (lo, hi, n, p), FP64 fields [B, E (p+1)^3]."""

    def __init__(self, lo, hi, n, p, leaves, penalty_form=0, penalty_eps=0.125, rtol=1e-10, max_iter=5000,
                 precond=1, precision=DG_PREC_FP64):
        if np.isscalar(n):
            n = (n, n, n)
        self.leaves = np.ascontiguousarray(leaves, dtype=np.int32)
        if self.leaves.ndim != 2 or self.leaves.shape[1] != 4:
            raise ValueError(f"leaves must be [n_leaves, 4], got {tuple(self.leaves.shape)}")
        self.p = int(p)
        self.Nq = self.leaves.shape[0] * (self.p + 1) ** 3
        desc = dg_mesh_desc((C.c_double * 3)(*lo), (C.c_double * 3)(*hi), (C.c_int32 * 3)(*n), self.p)
        h = C.c_void_p()
        _check(load().dg_octree_setup(C.byref(desc), self.leaves.ctypes.data_as(C.c_void_p), self.leaves.shape[0],
                                      penalty_form, penalty_eps, rtol, max_iter, precond, precision, C.byref(h)),
               "dg_octree_setup")
        self.h = h

    def _ck(self, code, where, allow=()):
        if code != DG_OK and code not in allow:
            raise DGError(code, where, load().dg_octree_error_detail(self.h).decode())
        return code

    def _field(self, t, name):
        import torch

        if t.ndim != 2 or t.shape[1] != self.Nq:
            raise ValueError(f"{name} must be [B, {self.Nq}], got {tuple(t.shape)}")
        return _dev_ptr(t, torch.float64)

    def node_coords(self):
        import torch

        xyz = torch.empty((self.Nq, 3), dtype=torch.float64, device="cuda")
        w = torch.empty((self.Nq,), dtype=torch.float64, device="cuda")
        self._ck(load().dg_octree_node_coords(self.h, _dev_ptr(xyz), _dev_ptr(w), _stream_ptr(None)),
                 "dg_octree_node_coords")
        return xyz, w

    def apply(self, u, out=None, stream=None):
        import torch

        if out is None:
            out = torch.empty_like(u)
        self._ck(load().dg_octree_operator(self.h, self._field(u, "u"), self._field(out, "out"), u.shape[0],
                                           _stream_ptr(stream)), "dg_octree_operator")
        return out

    def precond(self, r, stream=None):
        import torch

        z = torch.empty_like(r)
        self._ck(load().dg_octree_precond(self.h, self._field(r, "r"), self._field(z, "z"), r.shape[0],
                                          _stream_ptr(stream)), "dg_octree_precond")
        return z

    def solve(self, f, stream=None, allow_unconverged=False):
        import torch

        B = f.shape[0]
        v = torch.empty_like(f)
        st = (dg_solve_stats * max(B, 1))()
        allow = (DG_ERR_NOT_CONVERGED, DG_ERR_BREAKDOWN, DG_ERR_NONFINITE) if allow_unconverged else ()
        self._ck(load().dg_octree_solve(self.h, self._field(f, "f"), B, self._field(v, "v"), C.cast(st, C.c_void_p),
                                        _stream_ptr(stream)), "dg_octree_solve", allow)
        return v, _stats_list(st[:B])

    def exchange_build(self, psi, stream=None, allow_unconverged=False):
        N = psi.shape[0]
        P = N * (N + 1) // 2 + 1
        K = np.zeros((N, N))
        eh, ex = C.c_double(), C.c_double()
        st = (dg_solve_stats * P)()
        allow = (DG_ERR_NOT_CONVERGED, DG_ERR_BREAKDOWN, DG_ERR_NONFINITE) if allow_unconverged else ()
        self._ck(load().dg_octree_exchange_build(self.h, self._field(psi, "psi"), N, K.ctypes.data_as(C.c_void_p),
                                                 C.byref(eh), C.byref(ex), C.cast(st, C.c_void_p),
                                                 _stream_ptr(stream)), "dg_octree_exchange_build", allow)
        return K, eh.value, ex.value, _stats_list(st[:P])

    def close(self):
        if self.h:
            load().dg_octree_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
