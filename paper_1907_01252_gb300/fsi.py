"""Thin ctypes binding of the C ABI in include/fsi.h (argument marshalling only).

Every computation runs in the CUDA library libfsi.so; PyTorch only provides
device memory and the current stream. Importing this module does not need a
GPU; loading the library needs the compiled libfsi.so and raises if it is
missing (there is no fallback path).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads as wl

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libfsi.so")

FSI_OK, FSI_EINVAL, FSI_ENOMEM, FSI_ECUDA, FSI_ENEWTON, FSI_EGMRES, FSI_EJAC, FSI_ENAN, FSI_EDIVERGE = \
    0, -1, -2, -3, -4, -5, -6, -7, -8


class fsi_mesh(C.Structure):
    _fields_ = [("n_xseg", C.c_int), ("x_breaks", C.POINTER(C.c_double)), ("nx_seg", C.POINTER(C.c_int)),
                ("n_yseg", C.c_int), ("y_breaks", C.POINTER(C.c_double)), ("ny_seg", C.POINTER(C.c_int)),
                ("has_solid", C.c_int), ("solid_x0", C.c_double), ("solid_x1", C.c_double),
                ("solid_y0", C.c_double), ("solid_y1", C.c_double)]


class fsi_params(C.Structure):
    _fields_ = [("rho_f", C.c_double), ("nu_f", C.c_double), ("rho_s", C.c_double), ("mu_s", C.c_double),
                ("lambda_s", C.c_double), ("vbar", C.c_double), ("ramp_t", C.c_double), ("theta0", C.c_double),
                ("alpha0", C.c_double), ("T", C.c_double), ("n_slices", C.c_int), ("m_fine", C.c_int),
                ("m_coarse", C.c_int), ("newton_tol", C.c_double), ("newton_maxit", C.c_int),
                ("gmres_restart", C.c_int), ("gmres_maxit", C.c_int), ("gmres_rtol", C.c_double),
                ("gmres_rtol_first", C.c_double), ("newton_eta", C.c_double),
                ("mg_coarsest_max_dofs", C.c_int), ("mg_smooth", C.c_int), ("mg_omega", C.c_double),
                ("mg_smoother", C.c_int),
                ("mg_coarse_lps", C.c_double), ("mg_reuse", C.c_int), ("mg_rebuild_every", C.c_int),
                ("graph_max_batch", C.c_int), ("precision", C.c_int), ("pipeline_chunk", C.c_int),
                ("max_batch", C.c_int), ("mg_coarse_sweeps", C.c_int), ("tc_contraction", C.c_int),
                ("ff_operator", C.c_int)]


class fsi_stats(C.Structure):
    _fields_ = [("newton_iters", C.c_longlong), ("gmres_iters", C.c_longlong), ("max_newton", C.c_int),
                ("max_gmres", C.c_int), ("status", C.c_int), ("slice_status", C.POINTER(C.c_int)),
                ("slice_status_len", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if not f.startswith("slice_status")}


class fsi_parareal_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("increment_v", C.c_double), ("increment_u", C.c_double),
                ("increment_p", C.c_double), ("fine_steps", C.c_longlong), ("coarse_steps", C.c_longlong),
                ("fine", fsi_stats), ("coarse", fsi_stats), ("history", C.POINTER(C.c_double)),
                ("history_len", C.c_int)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("fine", "coarse", "history", "history_len")}
        d["fine"] = self.fine.as_dict()
        d["coarse"] = self.coarse.as_dict()
        return d


class fsi_mesh3d(C.Structure):
    _fields_ = [("n_xseg", C.c_int), ("x_breaks", C.POINTER(C.c_double)), ("nx_seg", C.POINTER(C.c_int)),
                ("n_yseg", C.c_int), ("y_breaks", C.POINTER(C.c_double)), ("ny_seg", C.POINTER(C.c_int)),
                ("n_zseg", C.c_int), ("z_breaks", C.POINTER(C.c_double)), ("nz_seg", C.POINTER(C.c_int)),
                ("has_solid", C.c_int), ("solid_box", C.c_double * 6)]


class fsi_instance(C.Structure):
    _fields_ = [("mesh", fsi_mesh), ("params", fsi_params), ("U", C.c_void_p), ("max_iter", C.c_int),
                ("tol", C.c_double), ("stats", fsi_parareal_stats), ("status", C.c_int), ("worker", C.c_int),
                ("seconds", C.c_double)]


# name -> (restype, argtypes); the exported symbols of include/fsi.h
_VP, _I, _D = C.c_void_p, C.c_int, C.c_double
SIGNATURES = {
    "fsi_setup": (_I, [C.POINTER(fsi_mesh), C.POINTER(fsi_params), C.POINTER(_VP)]),
    "fsi_destroy": (None, [_VP]),
    "fsi_last_error": (C.c_char_p, []),
    "fsi_n_nodes": (_I, [_VP]),
    "fsi_n_dofs": (_I, [_VP]),
    "fsi_n_levels": (_I, [_VP]),
    "fsi_nnzb": (_I, [_VP]),
    "fsi_bsr_pattern": (_I, [_VP, C.POINTER(_I), C.POINTER(_I)]),
    "fsi_residual": (_I, [_VP, _I, _VP, _VP, C.POINTER(_D), _D, _D, _VP, _VP]),
    "fsi_residual_noalloc": (_I, [_VP, _I, _VP, _VP, C.POINTER(_D), _D, _D, _VP, _VP]),
    "fsi_jacobian": (_I, [_VP, _I, _VP, _VP, _D, _D, _VP, _VP]),
    "fsi_jacobian_old": (_I, [_VP, _I, _VP, _VP, _D, _D, _VP, _VP]),
    "fsi_jacobian_f32": (_I, [_VP, _I, _VP, _VP, _D, _D, _VP, _VP]),
    "fsi_set_material": (_I, [_VP, _D, _D, _D]),
    "fsi_adjoint": (_I, [_VP, _VP, _D, _I, C.POINTER(_D), C.POINTER(_D), C.POINTER(fsi_stats), _VP]),
    "fsi_bsr_spmv": (_I, [_VP, _I, _VP, _VP, _VP, _VP]),
    "fsi_bsr_spmv_f32": (_I, [_VP, _I, _VP, _VP, _VP, _VP]),
    "fsi_bsr_spmv_ff": (_I, [_VP, _I, _VP, _VP, _VP, _VP]),
    "fsi_bsr_spmv_variant": (_I, [_VP, _I, _I, _I, _VP, _VP, _VP, _VP]),
    "fsi_theta_step": (_I, [_VP, _I, _VP, C.POINTER(_D), _D, _D, _VP, C.POINTER(fsi_stats), _VP]),
    "fsi_fine": (_I, [_VP, _I, _VP, C.POINTER(_D), _VP, C.POINTER(fsi_stats), _VP]),
    "fsi_coarse": (_I, [_VP, _I, _VP, C.POINTER(_D), _VP, C.POINTER(fsi_stats), _VP]),
    "parareal_iterate": (_I, [_VP, _VP, _I, _D, C.POINTER(fsi_parareal_stats), _VP]),
    "parareal_continue": (_I, [_VP, _VP, _I, _D, C.POINTER(fsi_parareal_stats), _VP]),
    "fsi_dense_invert": (_I, [_I, _I, _VP, _VP, _I, _VP]),
    "fsi_mesh_size": (_I, [C.POINTER(fsi_mesh), C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    "fsi3d_mesh_size": (_I, [C.POINTER(fsi_mesh3d), C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    "fsi_batch_plan": (_I, [C.POINTER(fsi_instance), _I, _I, C.POINTER(_I), C.POINTER(_I), C.POINTER(_D),
                            C.POINTER(_D)]),
    "fsi_batch_parareal": (_I, [C.POINTER(fsi_instance), _I, _I, _VP]),
    "fsi_batch_autotune": (_I, [C.POINTER(fsi_instance), _I, C.POINTER(_I), _I, C.POINTER(_D), C.POINTER(_I),
                                _VP]),
    "fsi3_setup": (_I, [C.POINTER(fsi_mesh3d), C.POINTER(fsi_params), C.POINTER(_VP)]),
    "fsi3_destroy": (None, [_VP]),
    "fsi3_n_nodes": (_I, [_VP]),
    "fsi3_n_dofs": (_I, [_VP]),
    "fsi3_n_levels": (_I, [_VP]),
    "fsi3_nnzb": (_I, [_VP]),
    "fsi3_bsr_pattern": (_I, [_VP, C.POINTER(_I), C.POINTER(_I)]),
    "fsi3_residual": (_I, [_VP, _I, _VP, _VP, C.POINTER(_D), _D, _D, _VP, _VP]),
    "fsi3_jacobian": (_I, [_VP, _I, _VP, _VP, _D, _D, _VP, _VP]),
    "fsi3_theta_step": (_I, [_VP, _I, _VP, C.POINTER(_D), _D, _D, _VP, C.POINTER(fsi_stats), _VP]),
    "fsi3_fine": (_I, [_VP, _I, _VP, C.POINTER(_D), _VP, C.POINTER(fsi_stats), _VP]),
    "fsi3_coarse": (_I, [_VP, _I, _VP, C.POINTER(_D), _VP, C.POINTER(fsi_stats), _VP]),
    "fsi3_parareal": (_I, [_VP, _VP, _I, _D, C.POINTER(fsi_parareal_stats), _VP]),
    "fsi3_kernel_count": (_I, []),
    "fsi3_kernel_name": (C.c_char_p, [_I]),
    "fsi3_launch_count": (C.c_longlong, [_I]),
    "fsi3_profile_enable": (_I, [_I]),
    "fsi3_profile_read": (_I, [_I, C.POINTER(_D), C.POINTER(C.c_longlong)]),
    "fsi_profile_enable": (_I, [C.c_ulonglong]),
    "fsi_profile_read": (_I, [_I, C.POINTER(_D), C.POINTER(C.c_longlong), C.POINTER(_D)]),
    "fsi_profile_read_bytes": (_I, [_I, C.POINTER(_D)]),
    "fsi_fp64_probe": (_I, [_I, _I, _D, _VP, _VP]),
    "fsi_tc_tile_product": (_I, [_I, _VP, _VP, _VP, _VP]),
    "fsi_launch_count": (C.c_longlong, [_I]),
    "fsi_kernel_count": (_I, []),
    "fsi_kernel_name": (C.c_char_p, [_I]),
}


def kernel_names():
    lib = load_library()
    return [lib.fsi_kernel_name(i).decode() for i in range(lib.fsi_kernel_count())]


def profile_enable(names=()):
    """Time every later launch of the named kernels with CUDA events."""
    lib = load_library()
    ids = kernel_names()
    mask = 0
    for n in names:
        mask |= 1 << ids.index(n)
    _check(lib.fsi_profile_enable(mask))


def profile_read(name):
    """(total milliseconds, timed launches, algorithmic flops) of a kernel since profile_enable."""
    lib = load_library()
    ms, cnt, fl = C.c_double(), C.c_longlong(), C.c_double()
    _check(lib.fsi_profile_read(kernel_names().index(name), C.byref(ms), C.byref(cnt), C.byref(fl)))
    return ms.value, cnt.value, fl.value


def profile_read_bytes(name):
    """Algorithmic DRAM bytes of a kernel's timed launches since profile_enable."""
    lib = load_library()
    b = C.c_double()
    _check(lib.fsi_profile_read_bytes(kernel_names().index(name), C.byref(b)))
    return b.value


def fp64_probe(blocks, iters, sink, seed=1.0):
    """Launch the FP64 FMA probe on the current stream (blocks * 256 * iters * 16 flops)."""
    _check(load_library().fsi_fp64_probe(blocks, iters, seed, _ptr(sink), _stream()))
    return blocks * 256 * iters * 16


def tc_tile_product(A, B, nsplit=3):
    """D = A B^T on the tensor cores (A [128, 32], B [16, 32] FP32 device tensors)."""
    import torch
    D = torch.empty((128, 16), dtype=torch.float32, device=A.device)
    _check(load_library().fsi_tc_tile_product(nsplit, _ptr(A), _ptr(B), _ptr(D), _stream()))
    return D


def launch_count(name=None):
    lib = load_library()
    return lib.fsi_launch_count(-1 if name is None else kernel_names().index(name))

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libfsi.so and declare its signatures; raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class FsiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fsi error {code}: {msg}")
        self.code = code


def _check(rc):
    if rc != FSI_OK:
        raise FsiError(rc, load_library().fsi_last_error().decode())
    return rc


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dbl(arr):
    a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64))
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _mesh_struct(w: wl.Workload):
    """(fsi_mesh, arrays it points into) for a workload's interface-fitted mesh."""
    xb = (C.c_double * len(wl.X_BREAKS))(*wl.X_BREAKS)
    yb = (C.c_double * len(wl.Y_BREAKS))(*wl.Y_BREAKS)
    nxs = (C.c_int * len(w.nx_seg))(*w.nx_seg)
    nys = (C.c_int * len(w.ny_seg))(*w.ny_seg)
    (sx0, sx1), (sy0, sy1) = wl.SOLID_BOX
    mesh = fsi_mesh(len(w.nx_seg), xb, nxs, len(w.ny_seg), yb, nys, int(w.with_solid), sx0, sx1, sy0, sy1)
    return mesh, (xb, yb, nxs, nys)


def _params(w: wl.Workload, max_batch: int, overrides):
    m = w.material
    p = dict(rho_f=m.rho_f, nu_f=m.nu_f, rho_s=m.rho_s, mu_s=m.mu_s, lambda_s=m.lambda_s, vbar=m.vbar,
             ramp_t=m.ramp_t, theta0=m.theta0, alpha0=m.alpha0, T=w.T, n_slices=w.n_slices, m_fine=w.m_fine,
             m_coarse=w.m_coarse, newton_tol=w.newton_tol, newton_maxit=w.newton_maxit,
             gmres_restart=w.gmres_restart, gmres_maxit=w.gmres_maxit, gmres_rtol=w.gmres_rtol,
             gmres_rtol_first=w.gmres_rtol_first, newton_eta=w.newton_eta,
             mg_coarsest_max_dofs=400, mg_smooth=2, mg_omega=0.6, mg_smoother=0, mg_coarse_lps=0.5, mg_reuse=2,
             mg_rebuild_every=4, graph_max_batch=4, precision=0, pipeline_chunk=0, max_batch=max_batch,
             mg_coarse_sweeps=0, tc_contraction=1, ff_operator=0)
    p.update(overrides)
    return p


def dense_invert(A, method=0):
    """Inverse of a device batch [S, n, n] of float64 matrices by the library's
    coarsest-level solver (method 0: cluster kernel when it fits, 1: one CTA per matrix)."""
    import torch
    inv = torch.empty_like(A)
    _check(load_library().fsi_dense_invert(A.shape[0], A.shape[1], _ptr(A), _ptr(inv), method, _stream()))
    return inv


def mesh_size(w: wl.Workload):
    """(n_nodes, n_dofs, nnzb) of a workload's finest mesh, computed on the host (no GPU)."""
    lib = load_library()
    mesh, keep = _mesh_struct(w)
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    _check(lib.fsi_mesh_size(C.byref(mesh), C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def mesh3d_size(breaks, counts, solid_box=None):
    """(n_nodes, n_dofs, nnzb) of a 3D mesh (break points and cells per segment per axis), on the host."""
    lib = load_library()
    keep, vals = [], []
    for br, cn in zip(breaks, counts):
        b = (C.c_double * len(br))(*br)
        c = (C.c_int * len(cn))(*cn)
        keep += [b, c]
        vals += [len(cn), b, c]
    box = (C.c_double * 6)(*(np.ravel(solid_box) if solid_box is not None else np.zeros(6)))
    mesh = fsi_mesh3d(*vals, int(solid_box is not None), box)
    a, b2, c2 = C.c_int(), C.c_int(), C.c_int()
    _check(lib.fsi3d_mesh_size(C.byref(mesh), C.byref(a), C.byref(b2), C.byref(c2)))
    return a.value, b2.value, c2.value


class Context:
    """An fsi_ctx built for a workload (mesh from the break points, materials, solver parameters)."""

    def __init__(self, workload: wl.Workload, max_batch: int = 1, **overrides):
        lib = load_library()
        w = workload
        self._mesh, self._keep = _mesh_struct(w)
        p = _params(w, max_batch, overrides)
        self.params = p
        self._params = fsi_params(**p)
        h = C.c_void_p()
        _check(lib.fsi_setup(C.byref(self._mesh), C.byref(self._params), C.byref(h)))
        self.handle = h
        self.lib = lib
        self.workload = w
        self.max_batch = max_batch
        self.n_nodes = lib.fsi_n_nodes(h)
        self.n_dofs = lib.fsi_n_dofs(h)
        self.nnzb = lib.fsi_nnzb(h)
        self.n_levels = lib.fsi_n_levels(h)

    def close(self):
        if self.handle:
            self.lib.fsi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- step-level entry points ------------------------------------------
    def fsi_residual(self, U, U_old, t_new, k, theta, R=None):
        import torch
        S = U.shape[0]
        R = torch.empty_like(U) if R is None else R
        t, tp = _dbl(t_new)
        _check(self.lib.fsi_residual(self.handle, S, _ptr(U), _ptr(U_old), tp, k, theta, _ptr(R), _stream()))
        return R

    def fsi_residual_noalloc(self, U, U_old, t_new, k, theta, R):
        """Same as fsi_residual with the scratch in a static device array; R must be given
        (preallocated by the caller): this call allocates no device memory."""
        t, tp = _dbl(t_new)
        _check(self.lib.fsi_residual_noalloc(self.handle, U.shape[0], _ptr(U), _ptr(U_old), tp, k, theta, _ptr(R),
                                             _stream()))
        return R

    def fsi_jacobian(self, U, U_old, k, theta, vals=None):
        import torch
        S = U.shape[0]
        vals = torch.empty((S, self.nnzb, 5, 5), dtype=torch.float64, device=U.device) if vals is None else vals
        _check(self.lib.fsi_jacobian(self.handle, S, _ptr(U), _ptr(U_old), k, theta, _ptr(vals), _stream()))
        return vals

    def fsi_jacobian_f32(self, U, U_old, k, theta, vals=None):
        """FP32 Jacobian blocks [S, nnzb, 5, 5] (element contraction as tc_contraction says)."""
        import torch
        S = U.shape[0]
        vals = torch.empty((S, self.nnzb, 5, 5), dtype=torch.float32, device=U.device) if vals is None else vals
        _check(self.lib.fsi_jacobian_f32(self.handle, S, _ptr(U), _ptr(U_old), k, theta, _ptr(vals), _stream()))
        return vals

    def fsi_jacobian_old(self, U, U_old, k, theta, vals=None):
        import torch
        S = U.shape[0]
        vals = torch.empty((S, self.nnzb, 5, 5), dtype=torch.float64, device=U.device) if vals is None else vals
        _check(self.lib.fsi_jacobian_old(self.handle, S, _ptr(U), _ptr(U_old), k, theta, _ptr(vals), _stream()))
        return vals

    def fsi_set_material(self, mu_s, lambda_s, vbar):
        _check(self.lib.fsi_set_material(self.handle, mu_s, lambda_s, vbar))

    def fsi_adjoint(self, U0, t0, n_steps):
        """(J, [dJ/dmu_s, dJ/dlambda_s, dJ/dvbar], stats) of the n_steps fine trajectory from U0 [n_dofs]."""
        J = C.c_double()
        grad = (C.c_double * 3)()
        st = fsi_stats()
        _check(self.lib.fsi_adjoint(self.handle, _ptr(U0), t0, n_steps, C.byref(J), grad, C.byref(st), _stream()))
        return J.value, [grad[0], grad[1], grad[2]], st.as_dict()

    def fsi_bsr_pattern(self):
        rowptr = np.zeros(self.n_nodes + 1, dtype=np.int32)
        colidx = np.zeros(self.nnzb, dtype=np.int32)
        _check(self.lib.fsi_bsr_pattern(self.handle, rowptr.ctypes.data_as(C.POINTER(C.c_int)),
                                        colidx.ctypes.data_as(C.POINTER(C.c_int))))
        return rowptr, colidx

    def fsi_bsr_spmv(self, vals, x, y=None):
        import torch
        y = torch.empty_like(x) if y is None else y
        _check(self.lib.fsi_bsr_spmv(self.handle, x.shape[0], _ptr(vals), _ptr(x), _ptr(y), _stream()))
        return y

    def fsi_bsr_spmv_f32(self, vals, x, y=None):
        """y = A x with FP32 values and vectors (the FP32 operator's product)."""
        import torch
        y = torch.empty_like(x) if y is None else y
        _check(self.lib.fsi_bsr_spmv_f32(self.handle, x.shape[0], _ptr(vals), _ptr(x), _ptr(y), _stream()))
        return y

    def fsi_bsr_spmv_ff(self, vals, x, y=None):
        """y = A x for FP64 vals and x through the float-pair product (ff_operator contexts)."""
        import torch
        y = torch.empty_like(x) if y is None else y
        _check(self.lib.fsi_bsr_spmv_ff(self.handle, x.shape[0], _ptr(vals), _ptr(x), _ptr(y), _stream()))
        return y

    def fsi_bsr_spmv_variant(self, value_type, tile_rows, vals, x, y=None):
        """y = A x in one kernel variant (value_type 0 FP64, 1 FP32, 2 float pairs;
        tile_rows 0 for the row-list kernel, else 8, 16, 32 or 64)."""
        import torch
        y = torch.empty_like(x) if y is None else y
        _check(self.lib.fsi_bsr_spmv_variant(self.handle, x.shape[0], value_type, tile_rows, _ptr(vals), _ptr(x),
                                             _ptr(y), _stream()))
        return y

    def _propagator_call(self, fn, S, *args):
        """Call a propagator entry point with a per-slice status array; the statuses
        are in the returned dict (and on the FsiError raised on failure)."""
        ss = np.zeros(S, dtype=np.int32)
        st = fsi_stats()
        st.slice_status = ss.ctypes.data_as(C.POINTER(C.c_int))
        st.slice_status_len = S
        rc = fn(self.handle, S, *args, C.byref(st), _stream())
        if rc != FSI_OK:
            err = FsiError(rc, self.lib.fsi_last_error().decode())
            err.slice_status = ss.tolist()
            err.stats = st.as_dict()
            raise err
        d = st.as_dict()
        d["slice_status"] = ss.tolist()
        return d

    def fsi_theta_step(self, U_old, t_old, k, theta, U_new=None):
        import torch
        U_new = torch.empty_like(U_old) if U_new is None else U_new
        t, tp = _dbl(t_old)
        d = self._propagator_call(self.lib.fsi_theta_step, U_old.shape[0], _ptr(U_old), tp, k, theta, _ptr(U_new))
        return U_new, d

    def fsi_fine(self, U0, t0, U1=None):
        import torch
        U1 = torch.empty_like(U0) if U1 is None else U1
        t, tp = _dbl(t0)
        return U1, self._propagator_call(self.lib.fsi_fine, U0.shape[0], _ptr(U0), tp, _ptr(U1))

    def fsi_coarse(self, U0, t0, U1=None):
        import torch
        U1 = torch.empty_like(U0) if U1 is None else U1
        t, tp = _dbl(t0)
        return U1, self._propagator_call(self.lib.fsi_coarse, U0.shape[0], _ptr(U0), tp, _ptr(U1))

    def parareal_iterate(self, U, max_iter, tol, history=False):
        """U: device [n_slices + 1, n_dofs]; U[0] is the initial state. In place.
        With history=True the stats hold the (v, u, p) increments of every iteration."""
        st = fsi_parareal_stats()
        hist = np.zeros((max(max_iter, 1), 3)) if history else None
        if history:
            st.history = hist.ctypes.data_as(C.POINTER(C.c_double))
            st.history_len = max_iter
        _check(self.lib.parareal_iterate(self.handle, _ptr(U), max_iter, tol, C.byref(st), _stream()))
        d = st.as_dict()
        if history:
            d["history"] = hist[:d["iterations"]].tolist()
        return U, d

    def parareal_continue(self, U, n_iter, tol, history=False):
        """Up to n_iter more iterations of the context's run on U (in place); the
        stats' iteration count is the run's, the other counts this call's."""
        st = fsi_parareal_stats()
        hist = np.zeros((max(n_iter, 1), 3)) if history else None
        if history:
            st.history = hist.ctypes.data_as(C.POINTER(C.c_double))
            st.history_len = n_iter
        _check(self.lib.parareal_continue(self.handle, _ptr(U), n_iter, tol, C.byref(st), _stream()))
        d = st.as_dict()
        if history:
            d["history"] = hist[:max(0, min(n_iter, d["iterations"]))].tolist()
        return U, d


def kernel_names3():
    lib = load_library()
    return [lib.fsi3_kernel_name(i).decode() for i in range(lib.fsi3_kernel_count())]


def profile3(on=True):
    """Start (clearing earlier records) or stop CUDA-event timing of the 3D kernels."""
    _check(load_library().fsi3_profile_enable(1 if on else 0))


def profile3_read():
    """{kernel name: (summed device ms, timed launches)} of the 3D kernels recorded so far."""
    lib = load_library()
    out = {}
    for i, name in enumerate(kernel_names3()):
        ms, n = C.c_double(), C.c_longlong()
        _check(lib.fsi3_profile_read(i, C.byref(ms), C.byref(n)))
        out[name] = (ms.value, n.value)
    return out


def launch_count3():
    return load_library().fsi3_launch_count(-1)


def fsi_setup(workload, max_batch=1, **overrides):
    return Context(workload, max_batch, **overrides)


def _mesh3d_struct(w: wl.Workload3D):
    """(fsi_mesh3d, arrays it points into) for a 3D workload's interface-fitted mesh."""
    keep, vals = [], []
    for br, cn in zip(w.breaks, w.segments):
        b = (C.c_double * len(br))(*br)
        c = (C.c_int * len(cn))(*cn)
        keep += [b, c]
        vals += [len(cn), b, c]
    box = (C.c_double * 6)(*np.ravel(wl.SOLID_BOX_3D))
    keep.append(box)
    return fsi_mesh3d(*vals, int(w.with_solid), box), keep


class Context3D:
    """An fsi3_ctx (the 3D path) built for a Workload3D. Arrays are device float64
    tensors [S, n_dofs] (7 per node: v, u, p); Jacobian blocks [S, nnzb, 7, 7]."""

    def __init__(self, workload: wl.Workload3D, max_batch: int = 1, **overrides):
        lib = load_library()
        w = workload
        self._mesh, self._keep = _mesh3d_struct(w)
        base = wl.Workload("3d", nx=1, ny=1, T=w.T, n_slices=w.n_slices, m_fine=w.m_fine, m_coarse=w.m_coarse,
                           newton_tol=w.newton_tol, newton_maxit=w.newton_maxit, gmres_restart=w.gmres_restart,
                           gmres_maxit=w.gmres_maxit, gmres_rtol=w.gmres_rtol, gmres_rtol_first=w.gmres_rtol_first,
                           newton_eta=w.newton_eta, material=w.material)
        # 3D defaults: FP32 multigrid, the coloured multiplicative Vanka sweep, smoother sweeps on the
        # coarsest level instead of its dense inverse, a quarter of the stabilisation weight per coarser
        # level, and the hierarchy rebuilt at every Newton iterate (chosen by FGMRES counts of the host solver)
        p = _params(base, max_batch, dict(dict(mg_coarsest_max_dofs=2000, precision=2, graph_max_batch=0,
                                               mg_smoother=1, mg_omega=1.0, mg_smooth=1, mg_coarse_sweeps=8,
                                               mg_coarse_lps=0.25, mg_reuse=0),
                                          **overrides))
        self.params = p
        self._params = fsi_params(**p)
        h = C.c_void_p()
        _check(lib.fsi3_setup(C.byref(self._mesh), C.byref(self._params), C.byref(h)))
        self.handle, self.lib, self.workload, self.max_batch = h, lib, w, max_batch
        self.n_nodes = lib.fsi3_n_nodes(h)
        self.n_dofs = lib.fsi3_n_dofs(h)
        self.nnzb = lib.fsi3_nnzb(h)
        self.n_levels = lib.fsi3_n_levels(h)

    def close(self):
        if self.handle:
            self.lib.fsi3_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def fsi3_residual(self, U, U_old, t_new, k, theta, R=None):
        import torch
        R = torch.empty_like(U) if R is None else R
        t, tp = _dbl(t_new)
        _check(self.lib.fsi3_residual(self.handle, U.shape[0], _ptr(U), _ptr(U_old), tp, k, theta, _ptr(R),
                                      _stream()))
        return R

    def fsi3_jacobian(self, U, U_old, k, theta, vals=None):
        import torch
        S = U.shape[0]
        vals = torch.empty((S, self.nnzb, 7, 7), dtype=torch.float64, device=U.device) if vals is None else vals
        _check(self.lib.fsi3_jacobian(self.handle, S, _ptr(U), _ptr(U_old), k, theta, _ptr(vals), _stream()))
        return vals

    def fsi3_bsr_pattern(self):
        rowptr = np.zeros(self.n_nodes + 1, dtype=np.int32)
        colidx = np.zeros(self.nnzb, dtype=np.int32)
        _check(self.lib.fsi3_bsr_pattern(self.handle, rowptr.ctypes.data_as(C.POINTER(C.c_int)),
                                         colidx.ctypes.data_as(C.POINTER(C.c_int))))
        return rowptr, colidx

    _propagator_call = Context._propagator_call

    def fsi3_theta_step(self, U_old, t_old, k, theta, U_new=None):
        import torch
        U_new = torch.empty_like(U_old) if U_new is None else U_new
        t, tp = _dbl(t_old)
        d = self._propagator_call(self.lib.fsi3_theta_step, U_old.shape[0], _ptr(U_old), tp, k, theta,
                                  _ptr(U_new))
        return U_new, d

    def fsi3_fine(self, U0, t0, U1=None):
        import torch
        U1 = torch.empty_like(U0) if U1 is None else U1
        t, tp = _dbl(t0)
        return U1, self._propagator_call(self.lib.fsi3_fine, U0.shape[0], _ptr(U0), tp, _ptr(U1))

    def fsi3_coarse(self, U0, t0, U1=None):
        import torch
        U1 = torch.empty_like(U0) if U1 is None else U1
        t, tp = _dbl(t0)
        return U1, self._propagator_call(self.lib.fsi3_coarse, U0.shape[0], _ptr(U0), tp, _ptr(U1))

    def fsi3_parareal(self, U, max_iter, tol, history=False):
        """U: device [n_slices + 1, n_dofs]; U[0] is the initial state. In place."""
        st = fsi_parareal_stats()
        hist = np.zeros((max(max_iter, 1), 3)) if history else None
        if history:
            st.history = hist.ctypes.data_as(C.POINTER(C.c_double))
            st.history_len = max_iter
        _check(self.lib.fsi3_parareal(self.handle, _ptr(U), max_iter, tol, C.byref(st), _stream()))
        d = st.as_dict()
        if history:
            d["history"] = hist[:d["iterations"]].tolist()
        return U, d


def tip_functional(ctx: Context, U0, t0, n_steps):
    """torch.autograd.Function for the bar-tip functional of the fine trajectory.

    tip_functional(ctx, U0, t0, n)(params) with params = tensor([mu_s, lambda_s,
    vbar]) returns J; its backward uses the discrete adjoint (fsi_adjoint)."""
    import torch

    class _TipFunctional(torch.autograd.Function):
        @staticmethod
        def forward(fctx, params):
            p = params.detach().cpu().double().tolist()
            ctx.fsi_set_material(*p)
            J, grad, _ = ctx.fsi_adjoint(U0, t0, n_steps)
            fctx.save_for_backward(torch.tensor(grad, dtype=params.dtype, device=params.device))
            return torch.tensor(J, dtype=params.dtype, device=params.device)

        @staticmethod
        def backward(fctx, gout):
            (grad,) = fctx.saved_tensors
            return gout * grad

    return _TipFunctional.apply


class Batch:
    """Independent problems (each a workload with its own mesh, material and
    slice count) advanced by the library's batch runner (fsi_batch_parareal).

    states: one device tensor [n_slices + 1][n_dofs] per problem (U[0] is the
    initial state; zeros from rest when omitted). Each run overwrites
    U[1:] from U[0], as parareal_iterate does. With device_states=False no
    device memory is touched and only plan() may be called (host only)."""

    def __init__(self, workloads, states=None, max_iter=1, tol=0.0, history=False, device_states=True,
                 **overrides):
        self.lib = load_library()
        self.workloads = list(workloads)
        n = len(self.workloads)
        self._inst = (fsi_instance * max(n, 1))()
        self._keep = []
        self.states = []
        self._hist = []
        for i, w in enumerate(self.workloads):
            mesh, keep = _mesh_struct(w)
            self._keep.append(keep)
            nd = mesh_size(w)[1]
            if not device_states:
                U = None
            elif states is None:
                import torch
                U = torch.zeros((w.n_slices + 1, nd), dtype=torch.float64, device="cuda")
            else:
                import torch
                U = states[i]
                if tuple(U.shape) != (w.n_slices + 1, nd) or U.dtype != torch.float64 or not U.is_contiguous():
                    raise ValueError("state %d must be a contiguous float64 [%d, %d] tensor" % (i, w.n_slices + 1, nd))
            self.states.append(U)
            I = self._inst[i]
            I.mesh = mesh
            I.params = fsi_params(**_params(w, w.n_slices, overrides))
            I.U = U.data_ptr() if U is not None else None
            I.max_iter = max_iter
            I.tol = tol
            if history:
                h = np.zeros((max(max_iter, 1), 3))
                self._hist.append(h)
                I.stats.history = h.ctypes.data_as(C.POINTER(C.c_double))
                I.stats.history_len = h.shape[0]

    def __len__(self):
        return len(self.workloads)

    def plan(self, workers):
        """The runner's longest-first schedule: order, planned worker, estimated cost, makespan."""
        n = len(self)
        order, worker = (C.c_int * max(n, 1))(), (C.c_int * max(n, 1))()
        cost, mk = (C.c_double * max(n, 1))(), C.c_double()
        _check(self.lib.fsi_batch_plan(self._inst, n, workers, order, worker, cost, C.byref(mk)))
        return {"order": list(order)[:n], "worker": list(worker)[:n], "cost": list(cost)[:n],
                "makespan": mk.value}

    def run(self, workers):
        """Run every problem; raises FsiError if any failed (per-problem results in results())."""
        _check(self.lib.fsi_batch_parareal(self._inst, len(self), workers, _stream()))
        return self.results()

    def autotune(self, candidates):
        """(best worker count, seconds per candidate) from the library's autotuner."""
        cand = (C.c_int * len(candidates))(*candidates)
        secs = (C.c_double * len(candidates))()
        best = C.c_int()
        _check(self.lib.fsi_batch_autotune(self._inst, len(self), cand, len(candidates), secs, C.byref(best),
                                           _stream()))
        return best.value, list(secs)

    def results(self):
        out = []
        for i in range(len(self)):
            I = self._inst[i]
            d = {"status": I.status, "worker": I.worker, "seconds": I.seconds, "stats": I.stats.as_dict()}
            if self._hist:
                d["history"] = self._hist[i][:max(I.stats.iterations, 0)].tolist()
            out.append(d)
        return out
