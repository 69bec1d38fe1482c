"""Thin Python binding of the C ABI in include/phfem.h (argument marshalling only).

Every function carries the name of the C entry point it calls, takes CUDA
tensors (device pointers) and ints, and raises :class:`PhfemError` on a
non-zero status.  All computation happens in the CUDA library; if the library
has not been built this module raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

PHFEM_FP64, PHFEM_FP32_IR = 0, 1
PHFEM_FORM_TRACE, PHFEM_FORM_FLUX = 0, 1
EDGE_INTERIOR, EDGE_DIRICHLET, EDGE_NEUMANN = 0, 1, 2
PHFEM_OK, PHFEM_EINVAL, PHFEM_EMESH, PHFEM_ENOMEM = 0, -1, -2, -3
PHFEM_ENOCONV, PHFEM_EBREAKDOWN, PHFEM_ENAN, PHFEM_ECUDA = -4, -5, -6, -7
MAX_TERMS = 4


class PhfemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


class MeshInfo(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("nV", "nT", "nE", "nF", "nL", "nD", "nN", "nnz")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class Coeffs(C.Structure):
    _fields_ = [("a_T", C.c_void_p), ("a", C.c_double), ("delta", C.c_double), ("dt", C.c_double),
                ("precision", C.c_int32), ("form", C.c_int32), ("A", C.c_double * 3), ("p", C.c_double * 2)]


class SolveOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("inner_rtol", C.c_double), ("max_iter", C.c_int32),
                ("max_refine", C.c_int32), ("check_every", C.c_int32), ("order", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("refinements", C.c_int32), ("converged", C.c_int32),
                ("steps", C.c_int32), ("rel_residual", C.c_double), ("seconds", C.c_double),
                ("fp64_floor", C.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class Source(C.Structure):
    _fields_ = [("nterms", C.c_int32), ("nt", C.c_int32), ("f_mid", C.c_void_p), ("bc_mid", C.c_void_p),
                ("phi", C.c_void_p)]


class Request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nV", C.c_int32), ("nT", C.c_int32), ("nD", C.c_int32), ("nN", C.c_int32),
                ("xy", C.c_void_p), ("tri", C.c_void_p), ("dirichlet", C.c_void_p), ("neumann", C.c_void_p),
                ("a_T", C.c_void_p), ("delta", C.c_double), ("f", C.c_double), ("uD", C.c_double),
                ("g", C.c_double), ("dt", C.c_double), ("u0", C.c_double), ("steps", C.c_int32),
                ("precision", C.c_int32), ("U_out", C.c_void_p), ("Lambda_out", C.c_void_p),
                ("levels", C.c_int32), ("reserved", C.c_int32), ("f_mid", C.c_void_p), ("bc_mid", C.c_void_p),
                ("u0_mid", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int32), ("done", C.c_int32), ("iterations", C.c_int32),
                ("slot", C.c_int32), ("nE", C.c_int32), ("nL", C.c_int32), ("rel_residual", C.c_double),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_finish", C.c_double),
                ("bytes_reserved", C.c_double), ("bytes_peak", C.c_int64), ("t_dev_start", C.c_double),
                ("t_dev_end", C.c_double), ("priority_class", C.c_int32), ("pad", C.c_int32)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class MgOpts(C.Structure):
    _fields_ = [("nu", C.c_int32), ("smooth_ratio", C.c_double), ("coarse_eps", C.c_double),
                ("coarse_degree", C.c_int32), ("flags", C.c_int32)]


class MgInfo(C.Structure):
    _fields_ = [("levels", C.c_int32), ("nu", C.c_int32), ("coarse_degree", C.c_int32), ("reserved", C.c_int32),
                ("coarse_a", C.c_double), ("coarse_b", C.c_double), ("smooth_ratio", C.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_ if n != "reserved"}


class Errors(C.Structure):
    _fields_ = [("L2", C.c_double), ("H1semi", C.c_double), ("H1", C.c_double), ("M", C.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib = None
_H = C.c_void_p
_P = C.c_void_p
_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)
_allocators = {}  # context handle -> the callback objects (kept alive while the context exists)


def lib() -> C.CDLL:
    """The loaded library (``_build/libphfem.so``); raises if it is missing."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = C.CDLL(path)
        sig = {
            "phfem_ctx_create": (C.c_int, [_P, C.POINTER(_H)]),
            "phfem_ctx_set_l2_window": (C.c_int, [_H, C.c_int]),
            "phfem_ctx_set_cg_kernel": (C.c_int, [_H, C.c_int]),
            "phfem_ctx_create_with_allocator": (C.c_int, [_P, _ALLOC_FN, _FREE_FN, _P, C.POINTER(_H)]),
            "phfem_ctx_destroy": (C.c_int, [_H]),
            "phfem_status_str": (C.c_char_p, [C.c_int]),
            "phfem_last_error": (C.c_char_p, []),
            "phfem_ctx_launches": (C.c_int64, [_H]),
            "phfem_ctx_memory": (C.c_int, [_H, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_int32]),
            "phfem_ctx_profile": (C.c_int, [_H, C.c_int]),
            "phfem_ctx_kernel_time": (C.c_int, [_H, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                                C.c_int]),
            "phfem_mesh_build": (C.c_int, [_H, C.c_int32, _P, C.c_int32, _P, C.c_int32, _P, C.c_int32, _P,
                                           C.POINTER(_H)]),
            "phfem_mesh_info_get": (C.c_int, [_H, C.POINTER(MeshInfo)]),
            "phfem_mesh_tables": (C.c_int, [_H, _P, _P, _P, _P, _P, _P, _P, _P]),
            "phfem_mesh_destroy": (C.c_int, [_H]),
            "phfem_mesh_refine": (C.c_int, [_H, _P, _P, _P, _P, C.POINTER(_H)]),
            "phfem_assemble": (C.c_int, [_H, C.POINTER(Coeffs), _P, _P, C.POINTER(_H)]),
            "phfem_sys_csr": (C.c_int, [_H, _P, _P]),
            "phfem_sys_destroy": (C.c_int, [_H]),
            "phfem_solve": (C.c_int, [_H, C.POINTER(SolveOpts), _P, _P, _P, _P, C.POINTER(Stats)]),
            "phfem_cn_create": (C.c_int, [_H, C.POINTER(Source), _P, _P, C.POINTER(_H)]),
            "phfem_cn_step": (C.c_int, [_H, C.c_int32, C.POINTER(SolveOpts), C.POINTER(Stats)]),
            "phfem_cn_create_data": (C.c_int, [_H, _P, _P, _P, _P, C.c_int32, C.POINTER(_H)]),
            "phfem_cn_step_data": (C.c_int, [_H, _P, _P, C.POINTER(SolveOpts), C.POINTER(Stats)]),
            "phfem_cn_step_graph": (C.c_int, [_H, C.c_int32, C.POINTER(SolveOpts), C.POINTER(Stats)]),
            "phfem_cn_read": (C.c_int, [_H, _P, _P, _P, _P, C.POINTER(C.c_int32)]),
            "phfem_cn_destroy": (C.c_int, [_H]),
            "phfem_batch_create": (C.c_int, [_H, C.c_int32, C.POINTER(_H), C.POINTER(_H)]),
            "phfem_batch_offsets": (C.c_int, [_H, _P, _P, _P]),
            "phfem_batch_solve": (C.c_int, [_H, _P, _P, _P, _P, C.c_int32, C.POINTER(SolveOpts), _P, _P, _P,
                                            C.c_int32, C.c_int32, _P, _P, _P]),
            "phfem_batch_tune": (C.c_int, [_H, _P, _P, _P, _P, C.c_int32, C.POINTER(SolveOpts), C.POINTER(C.c_int32),
                                           C.POINTER(C.c_int32), _P]),
            "phfem_batch_destroy": (C.c_int, [_H]),
            "phfem_server_create": (C.c_int, [C.c_int32, C.c_double, C.POINTER(SolveOpts), C.POINTER(_H)]),
            "phfem_server_submit": (C.c_int, [_H, C.POINTER(Request), C.POINTER(C.c_int64)]),
            "phfem_server_poll": (C.c_int, [_H, C.c_int64, C.c_int32, C.POINTER(Result)]),
            "phfem_server_drain": (C.c_int, [_H]),
            "phfem_server_destroy": (C.c_int, [_H]),
            "phfem_mg_create": (C.c_int, [_H, C.c_int32, C.POINTER(_H), _P, C.POINTER(MgOpts), C.POINTER(_H)]),
            "phfem_mg_info": (C.c_int, [_H, C.POINTER(MgInfo)]),
            "phfem_sys_set_mg": (C.c_int, [_H, _H]),
            "phfem_mg_transfer": (C.c_int, [_H, C.c_int32, C.c_int32, _P, _P]),
            "phfem_mg_destroy": (C.c_int, [_H]),
            "phfem_error_points": (C.c_int, [_H, C.c_int32, _P, _P, _P]),
            "phfem_error_norms": (C.c_int, [_H, C.c_int32, _P, _P, _P, _P, _P, C.POINTER(Errors)]),
            "phfem_mesh_order": (C.c_int, [_H, _P, C.POINTER(C.c_int32)]),
            "phfem_csr_pcg_noalloc": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, _P, C.c_double, C.c_int32,
                                                C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int, what: str):
    if status != 0:
        L = lib()
        raise PhfemError(status, f"{what}: {L.phfem_status_str(status).decode()}: "
                                 f"{L.phfem_last_error().decode()}")


def _ptr(t, dtype=None, n=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if n is not None and t.numel() < n:
        raise ValueError(f"expected at least {n} elements, got {t.numel()}")
    return t.data_ptr()


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


# --- context -----------------------------------------------------------------

def phfem_ctx_create(stream=None, torch_allocator=False):
    """A context on `stream`; with torch_allocator=True the library's device
    memory comes from PyTorch's caching allocator (phfem_ctx_create_with_allocator)."""
    h = _H()
    if not torch_allocator:
        _check(lib().phfem_ctx_create(_stream_ptr(stream), C.byref(h)), "phfem_ctx_create")
        return h
    device = torch.cuda.current_device()

    def alloc(nbytes, strm, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device=device, stream=int(strm or 0))
        except Exception:  # reported to the library as an allocation failure
            return None

    def free(ptr, strm, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    fa, ff = _ALLOC_FN(alloc), _FREE_FN(free)
    _check(lib().phfem_ctx_create_with_allocator(_stream_ptr(stream), fa, ff, None, C.byref(h)),
           "phfem_ctx_create_with_allocator")
    _allocators[h.value] = (fa, ff)
    return h


def phfem_ctx_create_with_allocator(stream=None):
    """The context of phfem_ctx_create(stream, torch_allocator=True)."""
    return phfem_ctx_create(stream, torch_allocator=True)


def phfem_ctx_set_cg_kernel(ctx, variant=0):
    """FP32 Jacobi iteration in the locality order: 0 direction update fused into the product, the rows'
    own data staged in shared memory (default); 1 separate direction kernel; 2 fused, rows through L1/L2."""
    _check(lib().phfem_ctx_set_cg_kernel(ctx, int(variant)), "phfem_ctx_set_cg_kernel")


def phfem_ctx_memory(ctx, reset_peak=False):
    """(bytes now, peak bytes) of the context's own device allocations."""
    now, peak = C.c_int64(), C.c_int64()
    _check(lib().phfem_ctx_memory(ctx, C.byref(now), C.byref(peak), int(bool(reset_peak))), "phfem_ctx_memory")
    return now.value, peak.value


def phfem_ctx_set_l2_window(ctx, enable=True):
    _check(lib().phfem_ctx_set_l2_window(ctx, int(bool(enable))), "phfem_ctx_set_l2_window")


def phfem_ctx_destroy(ctx):
    _check(lib().phfem_ctx_destroy(ctx), "phfem_ctx_destroy")
    _allocators.pop(ctx.value if isinstance(ctx, _H) else ctx, None)


def phfem_ctx_launches(ctx) -> int:
    return int(lib().phfem_ctx_launches(ctx))


def phfem_ctx_profile(ctx, enable):
    """enable: False/True, or n > 1 to time every n-th launch of each kernel."""
    n = int(enable) if not isinstance(enable, bool) else int(enable)
    _check(lib().phfem_ctx_profile(ctx, n), "phfem_ctx_profile")


def phfem_ctx_kernel_time(ctx, kernel: str, reset: bool = True):
    """(total device ms, number of timed launches) of one instrumented kernel."""
    ms, n = C.c_double(), C.c_int64()
    _check(lib().phfem_ctx_kernel_time(ctx, kernel.encode(), C.byref(ms), C.byref(n), int(reset)),
           "phfem_ctx_kernel_time")
    return float(ms.value), int(n.value)


# --- mesh --------------------------------------------------------------------

def phfem_mesh_build(ctx, xy, tri, dirichlet, neumann):
    nV, nT = xy.shape[0], tri.shape[0]
    nD = dirichlet.shape[0] if dirichlet is not None else 0
    nN = neumann.shape[0] if neumann is not None else 0
    h = _H()
    _check(lib().phfem_mesh_build(ctx, nV, _ptr(xy, torch.float64, 2 * nV), nT, _ptr(tri, torch.int32, 3 * nT),
                                  nD, _ptr(dirichlet, torch.int32) if nD else None,
                                  nN, _ptr(neumann, torch.int32) if nN else None, C.byref(h)),
           "phfem_mesh_build")
    return h


def phfem_mesh_refine(mesh, build=True, arrays=False):
    """Red refinement on the device.  Returns the refined mesh handle (build),
    and with arrays=True also the refined xy, tri, dirichlet, neumann tensors."""
    I = phfem_mesh_info_get(mesh)
    dev = torch.device("cuda", torch.cuda.current_device())
    out = None
    if arrays:
        out = dict(xy=torch.empty((I["nV"] + I["nE"], 2), dtype=torch.float64, device=dev),
                   tri=torch.empty((4 * I["nT"], 3), dtype=torch.int32, device=dev),
                   dirichlet=torch.empty((2 * I["nD"], 2), dtype=torch.int32, device=dev),
                   neumann=torch.empty((2 * I["nN"], 2), dtype=torch.int32, device=dev))
    h = _H()
    _check(lib().phfem_mesh_refine(mesh, _ptr(out["xy"]) if out else None, _ptr(out["tri"]) if out else None,
                                   _ptr(out["dirichlet"]) if out and I["nD"] else None,
                                   _ptr(out["neumann"]) if out and I["nN"] else None,
                                   C.byref(h) if build else None), "phfem_mesh_refine")
    if build and arrays:
        return h, out
    return h if build else out


def phfem_mesh_info_get(mesh) -> dict:
    info = MeshInfo()
    _check(lib().phfem_mesh_info_get(mesh, C.byref(info)), "phfem_mesh_info_get")
    return info.as_dict()


def phfem_mesh_tables(mesh, device=None) -> dict:
    """All tables of the mesh as new device tensors."""
    I = phfem_mesh_info_get(mesh)
    dev = device or torch.device("cuda", torch.cuda.current_device())
    i32 = dict(dtype=torch.int32, device=dev)
    out = dict(
        ed2el=torch.empty((I["nE"], 4), **i32), t2e=torch.empty((I["nT"], 3), **i32),
        sigma=torch.empty((I["nT"], 3), dtype=torch.int8, device=dev),
        eclass=torch.empty(I["nE"], dtype=torch.uint8, device=dev),
        free_id=torch.empty(I["nE"], **i32), lam_id=torch.empty(I["nE"], **i32),
        row_ptr=torch.empty(I["nF"] + 1, **i32), col=torch.empty(max(I["nnz"], 1), **i32))
    _check(lib().phfem_mesh_tables(mesh, *(out[k].data_ptr() for k in
                                           ("ed2el", "t2e", "sigma", "eclass", "free_id", "lam_id",
                                            "row_ptr", "col"))), "phfem_mesh_tables")
    out["col"] = out["col"][:I["nnz"]]
    return out


def phfem_mesh_destroy(mesh):
    _check(lib().phfem_mesh_destroy(mesh), "phfem_mesh_destroy")


# --- assembly ----------------------------------------------------------------

def phfem_assemble(mesh, f_mid=None, bc_mid=None, a_T=None, a=1.0, delta=0.0, dt=0.0, precision=PHFEM_FP64,
                   form=PHFEM_FORM_TRACE, A=None, p=None):
    """A: constant SPD tensor as (A11, A12, A22) or a 2x2 array (None: identity);
    p: constant convection velocity (px, py) (None: no convection)."""
    I = phfem_mesh_info_get(mesh)
    c = Coeffs(_ptr(a_T, torch.float64, I["nT"]), float(a), float(delta), float(dt), int(precision), int(form))
    if A is not None:
        import numpy as np
        Aa = np.asarray(A, dtype=np.float64)
        vals = (Aa[0, 0], Aa[0, 1], Aa[1, 1]) if Aa.shape == (2, 2) else tuple(Aa.ravel())
        c.A = (C.c_double * 3)(*[float(v) for v in vals])
    if p is not None:
        c.p = (C.c_double * 2)(float(p[0]), float(p[1]))
    h = _H()
    _check(lib().phfem_assemble(mesh, C.byref(c), _ptr(f_mid, torch.float64, I["nE"]),
                                _ptr(bc_mid, torch.float64, I["nE"]), C.byref(h)), "phfem_assemble")
    return h


def phfem_sys_csr(sys, val, rhs):
    _check(lib().phfem_sys_csr(sys, _ptr(val, torch.float64), _ptr(rhs, torch.float64)), "phfem_sys_csr")


def phfem_sys_destroy(sys):
    _check(lib().phfem_sys_destroy(sys), "phfem_sys_destroy")


def solve_opts(rtol=1e-10, inner_rtol=0.0, max_iter=0, max_refine=0, check_every=0, order=0) -> SolveOpts:
    """order: 0 = the Jacobi iteration in the locality order of the edges, 1 = in the paper's edge order."""
    return SolveOpts(float(rtol), float(inner_rtol), int(max_iter), int(max_refine), int(check_every), int(order))


def phfem_solve(sys, opts=None, w0=None, w=None, U=None, Lambda=None, raise_on_noconv=True) -> dict:
    st = Stats()
    o = opts if opts is not None else solve_opts()
    status = lib().phfem_solve(sys, C.byref(o), _ptr(w0, torch.float64), _ptr(w, torch.float64),
                               _ptr(U, torch.float64), _ptr(Lambda, torch.float64), C.byref(st))
    if status != 0 and (raise_on_noconv or status != -4):
        _check(status, "phfem_solve")
    d = st.as_dict()
    d["status"] = status
    return d


# --- Crank-Nicolson ------------------------------------------------------------

def phfem_cn_create(sys, f_mid, bc_mid, phi, w0, Lambda0=None):
    """f_mid, bc_mid: [Q, nE] CUDA float64; phi: [Q, nt] host float64 (numpy or tensor)."""
    import numpy as np
    phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float64))
    if phi.ndim == 1:
        phi = phi[None, :]
    Q, nt = phi.shape
    src = Source(Q, nt, _ptr(f_mid, torch.float64), _ptr(bc_mid, torch.float64),
                 phi.ctypes.data_as(C.c_void_p).value)
    h = _H()
    _check(lib().phfem_cn_create(sys, C.byref(src), _ptr(w0, torch.float64), _ptr(Lambda0, torch.float64),
                                 C.byref(h)), "phfem_cn_create")
    return h


def phfem_cn_create_data(sys, f0_mid, bc0_mid, w0, max_steps, Lambda0=None):
    """Crank-Nicolson with per-step data (general sources); the data at t_0 here."""
    h = _H()
    _check(lib().phfem_cn_create_data(sys, _ptr(f0_mid, torch.float64), _ptr(bc0_mid, torch.float64),
                                      _ptr(w0, torch.float64), _ptr(Lambda0, torch.float64), int(max_steps),
                                      C.byref(h)), "phfem_cn_create_data")
    return h


def phfem_cn_step_data(cn, f_mid, bc_mid, opts=None) -> dict:
    """One step with the data at the new time level (f and g / u_D at the midpoints)."""
    st = Stats()
    o = opts if opts is not None else solve_opts()
    _check(lib().phfem_cn_step_data(cn, _ptr(f_mid, torch.float64), _ptr(bc_mid, torch.float64), C.byref(o),
                                    C.byref(st)), "phfem_cn_step_data")
    return st.as_dict()


def phfem_cn_step(cn, nsteps, opts=None) -> dict:
    st = Stats()
    o = opts if opts is not None else solve_opts()
    _check(lib().phfem_cn_step(cn, int(nsteps), C.byref(o), C.byref(st)), "phfem_cn_step")
    return st.as_dict()


def phfem_cn_step_graph(cn, nsteps, opts=None) -> dict:
    st = Stats()
    o = opts if opts is not None else solve_opts()
    _check(lib().phfem_cn_step_graph(cn, int(nsteps), C.byref(o), C.byref(st)), "phfem_cn_step_graph")
    return st.as_dict()


def phfem_cn_read(cn, w=None, U=None, Lambda_n=None, Lambda_half=None) -> int:
    step = C.c_int32()
    _check(lib().phfem_cn_read(cn, _ptr(w, torch.float64), _ptr(U, torch.float64), _ptr(Lambda_n, torch.float64),
                               _ptr(Lambda_half, torch.float64), C.byref(step)), "phfem_cn_read")
    return int(step.value)


def phfem_cn_destroy(cn):
    _check(lib().phfem_cn_destroy(cn), "phfem_cn_destroy")


def phfem_status_str(status: int) -> str:
    return lib().phfem_status_str(int(status)).decode()


def phfem_last_error() -> str:
    return lib().phfem_last_error().decode()


# --- batched assembly and solve --------------------------------------------------

def phfem_batch_create(ctx, meshes):
    arr = (_H * len(meshes))(*meshes)
    h = _H()
    _check(lib().phfem_batch_create(ctx, len(meshes), arr, C.byref(h)), "phfem_batch_create")
    return h


def phfem_batch_offsets(batch, count):
    import numpy as np
    t = np.zeros(count + 1, dtype=np.int64)
    e = np.zeros(count + 1, dtype=np.int64)
    l = np.zeros(count + 1, dtype=np.int64)
    _check(lib().phfem_batch_offsets(batch, t.ctypes.data, e.ctypes.data, l.ctypes.data), "phfem_batch_offsets")
    return t, e, l


def phfem_batch_solve(batch, count, delta, a_T=None, f_mid=None, bc_mid=None, precision=PHFEM_FP32_IR,
                      opts=None, w=None, U=None, Lambda=None, block=0, cluster=None):
    import numpy as np
    it = np.zeros(count, dtype=np.int32)
    cv = np.zeros(count, dtype=np.int32)
    rel = np.zeros(count, dtype=np.float64)
    o = opts if opts is not None else solve_opts()
    _check(lib().phfem_batch_solve(batch, _ptr(a_T, torch.float64), _ptr(delta, torch.float64, count),
                                   _ptr(f_mid, torch.float64), _ptr(bc_mid, torch.float64), int(precision),
                                   C.byref(o), _ptr(w, torch.float64), _ptr(U, torch.float64),
                                   _ptr(Lambda, torch.float64), int(block),
                                   int((1 if block else 0) if cluster is None else cluster), it.ctypes.data, cv.ctypes.data,
                                   rel.ctypes.data), "phfem_batch_solve")
    return {"iterations": it, "converged": cv, "rel_residual": rel}


BATCH_SHAPES = [(128, 1), (256, 1), (512, 1), (1024, 1), (256, 4), (512, 4), (1024, 4), (256, 8), (512, 8), (1024, 8)]


def phfem_batch_tune(batch, delta, a_T=None, f_mid=None, bc_mid=None, precision=PHFEM_FP32_IR, opts=None):
    """Times every launch shape (threads per block, CTAs per mesh); returns the
    chosen shape and {shape: host ms}."""
    import numpy as np
    ms = np.zeros(len(BATCH_SHAPES), dtype=np.float64)
    cb, cc = C.c_int32(), C.c_int32()
    o = opts if opts is not None else solve_opts()
    _check(lib().phfem_batch_tune(batch, _ptr(a_T, torch.float64), _ptr(delta, torch.float64),
                                  _ptr(f_mid, torch.float64), _ptr(bc_mid, torch.float64), int(precision),
                                  C.byref(o), C.byref(cb), C.byref(cc), ms.ctypes.data), "phfem_batch_tune")
    return (int(cb.value), int(cc.value)), {f"{b}x{c}": float(t) for (b, c), t in zip(BATCH_SHAPES, ms.tolist())}


def phfem_batch_destroy(batch):
    _check(lib().phfem_batch_destroy(batch), "phfem_batch_destroy")


# --- request server --------------------------------------------------------------

def phfem_server_create(slots, hbm_budget_bytes, opts=None):
    h = _H()
    o = opts if opts is not None else solve_opts()
    _check(lib().phfem_server_create(int(slots), float(hbm_budget_bytes), C.byref(o), C.byref(h)),
           "phfem_server_create")
    return h


def make_request(xy, tri, dirichlet, neumann, kind=0, a_T=None, delta=0.0, f=1.0, uD=0.0, g=0.0, dt=0.0, u0=0.0,
                 steps=0, precision=PHFEM_FP32_IR, U_out=None, Lambda_out=None, levels=0, f_mid=None, bc_mid=None,
                 u0_mid=None) -> Request:
    """f_mid, bc_mid, u0_mid: optional midpoint arrays on the finest mesh's edges; the constants otherwise."""
    return Request(int(kind), xy.shape[0], tri.shape[0], dirichlet.shape[0] if dirichlet is not None else 0,
                   neumann.shape[0] if neumann is not None else 0, _ptr(xy, torch.float64), _ptr(tri, torch.int32),
                   _ptr(dirichlet, torch.int32) if dirichlet is not None and dirichlet.numel() else None,
                   _ptr(neumann, torch.int32) if neumann is not None and neumann.numel() else None,
                   _ptr(a_T, torch.float64), float(delta), float(f), float(uD), float(g), float(dt), float(u0),
                   int(steps), int(precision), _ptr(U_out, torch.float64), _ptr(Lambda_out, torch.float64),
                   int(levels), 0, _ptr(f_mid, torch.float64), _ptr(bc_mid, torch.float64),
                   _ptr(u0_mid, torch.float64))


def phfem_server_submit(server, req: Request) -> int:
    rid = C.c_int64()
    _check(lib().phfem_server_submit(server, C.byref(req), C.byref(rid)), "phfem_server_submit")
    return int(rid.value)


def phfem_server_poll(server, rid, wait=True) -> dict:
    r = Result()
    _check(lib().phfem_server_poll(server, int(rid), int(bool(wait)), C.byref(r)), "phfem_server_poll")
    return r.as_dict()


def phfem_server_drain(server):
    _check(lib().phfem_server_drain(server), "phfem_server_drain")


def phfem_server_destroy(server):
    _check(lib().phfem_server_destroy(server), "phfem_server_destroy")


# --- multigrid preconditioner --------------------------------------------------------

PHFEM_MG_COARSE_STEPWISE = 1


def phfem_mg_create(sys, meshes, a_T=None, nu=0, smooth_ratio=0.0, coarse_eps=0.0, coarse_degree=0, flags=0):
    """Multigrid over meshes (coarsest first, each the refinement of the one
    before, the last the system's mesh).  flags: PHFEM_MG_COARSE_STEPWISE runs
    the coarsest iteration one launch per step."""
    arr = (_H * len(meshes))(*[m.value if isinstance(m, _H) else m for m in meshes])
    I = phfem_mesh_info_get(meshes[-1])
    o = MgOpts(int(nu), float(smooth_ratio), float(coarse_eps), int(coarse_degree), int(flags))
    h = _H()
    _check(lib().phfem_mg_create(sys, len(meshes), arr, _ptr(a_T, torch.float64, I["nT"]), C.byref(o), C.byref(h)),
           "phfem_mg_create")
    return h


def phfem_mg_info(mg) -> dict:
    out = MgInfo()
    _check(lib().phfem_mg_info(mg, C.byref(out)), "phfem_mg_info")
    return out.as_dict()


def phfem_sys_set_mg(sys, mg):
    _check(lib().phfem_sys_set_mg(sys, mg), "phfem_sys_set_mg")


def phfem_mg_transfer(mg, level, direction, inp, out):
    _check(lib().phfem_mg_transfer(mg, int(level), int(direction), _ptr(inp, torch.float64),
                                   _ptr(out, torch.float64)), "phfem_mg_transfer")


def phfem_mg_destroy(mg):
    _check(lib().phfem_mg_destroy(mg), "phfem_mg_destroy")


# --- error report -----------------------------------------------------------------

def phfem_error_points(mesh, nq, tri_xy=None, edge_xy=None, edge_nu=None):
    """Quadrature points of the error report: tri_xy (nT, nq*nq, 2), edge_xy
    (nL, nq, 2) and edge_nu (nL, 2), float64 CUDA tensors (each optional)."""
    I = phfem_mesh_info_get(mesh)
    Q = nq * nq
    _check(lib().phfem_error_points(mesh, int(nq), _ptr(tri_xy, torch.float64, 2 * Q * I["nT"]),
                                    _ptr(edge_xy, torch.float64, 2 * nq * I["nL"]),
                                    _ptr(edge_nu, torch.float64, 2 * I["nL"])), "phfem_error_points")


def phfem_error_norms(mesh, nq, U=None, u_q=None, grad_q=None, Lambda=None, kappa_q=None) -> dict:
    """L2, broken H1 and multiplier mesh-norm errors (host floats)."""
    I = phfem_mesh_info_get(mesh)
    Q = nq * nq
    out = Errors()
    _check(lib().phfem_error_norms(mesh, int(nq), _ptr(U, torch.float64, 3 * I["nT"]),
                                   _ptr(u_q, torch.float64, Q * I["nT"]), _ptr(grad_q, torch.float64, 2 * Q * I["nT"]),
                                   _ptr(Lambda, torch.float64, I["nL"]), _ptr(kappa_q, torch.float64, nq * I["nL"]),
                                   C.byref(out)), "phfem_error_norms")
    return out.as_dict()


def phfem_mesh_order(mesh, perm=None) -> dict:
    """The locality order of the iteration kernels: perm[i] = the edge held by
    internal row i (a CUDA int32 tensor of nE), and the number of rows whose
    neighbours are stored as full indices."""
    n = phfem_mesh_info_get(mesh)["nE"]
    if perm is None:
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
    novf = C.c_int32()
    _check(lib().phfem_mesh_order(mesh, _ptr(perm, torch.int32, n), C.byref(novf)), "phfem_mesh_order")
    return {"perm": perm, "overflow_rows": int(novf.value)}


# --- solve without device allocation -------------------------------------------

NOALLOC_MAX_ROWS = 262144


def phfem_csr_pcg_noalloc(row_ptr, col, val, rhs, x, rtol=1e-10, max_iter=0, stream=None) -> dict:
    """Jacobi-PCG on a CSR system using only the library's fixed device scratch
    (for callers that cannot allocate device memory during the call); x holds
    the initial guess and receives the solution.  rel_residual is that of the
    iteration's recursive residual.  All tensors must be on one device; the
    call runs with that device current, whose scratch array it uses."""
    n = rhs.numel()
    devs = {t.device for t in (row_ptr, col, val, rhs, x) if isinstance(t, torch.Tensor)}
    if len(devs) != 1:
        raise ValueError(f"phfem_csr_pcg_noalloc: tensors on several devices: {sorted(map(str, devs))}")
    it, rel = C.c_int32(), C.c_double()
    with torch.cuda.device(rhs.device):
        _check(lib().phfem_csr_pcg_noalloc(_stream_ptr(stream), n, _ptr(row_ptr, torch.int32, n + 1),
                                           _ptr(col, torch.int32), _ptr(val, torch.float64),
                                           _ptr(rhs, torch.float64, n), _ptr(x, torch.float64, n), float(rtol),
                                           int(max_iter), C.byref(it), C.byref(rel)), "phfem_csr_pcg_noalloc")
    return {"iterations": int(it.value), "rel_residual": float(rel.value)}
