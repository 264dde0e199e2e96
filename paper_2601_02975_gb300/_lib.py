"""ctypes binding of libccmg.so (include/ccmg.h).

Argument marshalling only: every step of the method runs in the library.
Device arrays are torch CUDA tensors (float64, contiguous); host arrays are
numpy arrays.  Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libccmg.so")

CC_OK, CC_ERR_ARG, CC_ERR_GEOMETRY, CC_ERR_SINGULAR, CC_ERR_NO_MEMORY = 0, 1, 2, 3, 4
CC_ERR_NOT_CONVERGED, CC_ERR_DIVERGED, CC_ERR_TIMEOUT, CC_ERR_CUDA, CC_ERR_BUSY = 5, 6, 7, 8, 9
CYCLE_V, CYCLE_W, CYCLE_FMG = 1, 2, 3
PREC_FP64, PREC_MIXED = 0, 1
SMOOTHER_JACOBI, SMOOTHER_MCGS = 0, 1


class cc_hole(C.Structure):
    _fields_ = [("kind", C.c_int), ("cx", C.c_double), ("cy", C.c_double), ("r1", C.c_double),
                ("r2", C.c_double), ("theta", C.c_double)]


class cc_domain(C.Structure):
    _fields_ = [("x0", C.c_double), ("y0", C.c_double), ("x1", C.c_double), ("y1", C.c_double),
                ("n_holes", C.c_int), ("holes", C.POINTER(cc_hole))]


class cc_bc(C.Structure):
    _fields_ = [("type", C.c_int), ("alpha1", C.c_double), ("alpha2", C.c_double)]


class cc_options(C.Structure):
    _fields_ = [("eps", C.c_double), ("nu1", C.c_int), ("nu2", C.c_int), ("omega", C.c_double),
                ("cycle", C.c_int), ("min_coarse_n", C.c_int), ("precision", C.c_int),
                ("max_cycles", C.c_int), ("use_graphs", C.c_int), ("host_only", C.c_int),
                ("fmg_cycle", C.c_int), ("w_depth", C.c_int), ("serve_slots", C.c_int),
                ("cache", C.c_int), ("hole_cells", C.c_double), ("krylov", C.c_int),
                ("smoother", C.c_int), ("device_setup", C.c_int), ("device_loop", C.c_int),
                ("autotune", C.c_int)]


class cc_info(C.Structure):
    _fields_ = [("n", C.c_int), ("n_levels", C.c_int), ("n_dof", C.c_int64), ("n_bd", C.c_int),
                ("n_g", C.c_int), ("n_plg", C.c_int), ("n_block", C.c_int),
                ("device_bytes", C.c_int64), ("level_n", C.c_int * 32),
                ("block_error", C.c_double), ("bottom_error", C.c_double),
                ("block_m", C.c_int * 32), ("block_chunks", C.c_int * 32),
                ("setup_seconds", C.c_double), ("setup_tables_seconds", C.c_double),
                ("setup_kernel_ms", C.c_double), ("sweep_ctas", C.c_int * 32),
                ("block_chunk_rows", C.c_int * 32)]


class cc_result(C.Structure):
    _fields_ = [("status", C.c_int), ("cycles", C.c_int), ("rel_res", C.c_double),
                ("t_submit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double),
                ("kernels", C.c_int64)]


class CCError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


_lib = None
_P = C.c_void_p

# name -> (restype, argtypes); every entry point declared in include/ccmg.h
_SIGS = {
    "cc_default_options": (None, [C.POINTER(cc_options)]),
    "cc_status_string": (C.c_char_p, [C.c_int]),
    "cc_last_error_string": (C.c_char_p, []),
    "cc_setup": (C.c_int, [C.POINTER(cc_domain), C.c_double, C.c_double, C.c_double,
                           C.POINTER(cc_bc), C.c_int, C.c_int, C.POINTER(cc_options), _P,
                           C.POINTER(_P)]),
    "cc_query": (C.c_int, [_P, C.POINTER(cc_info)]),
    "cc_destroy": (C.c_int, [_P]),
    "cc_cell_types": (C.c_int, [_P, _P, _P, _P]),
    "cc_quadrature_nodes": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int64),
                                      C.POINTER(C.c_int64), _P, _P, _P, _P, _P, _P]),
    "cc_solve": (C.c_int, [_P, _P, _P, _P, C.c_double, _P, C.POINTER(cc_result)]),
    "cc_clone": (C.c_int, [_P, _P, C.POINTER(_P)]),
    "cc_serve_budget": (C.c_int, [C.c_int64]),
    "cc_cache_clear": (C.c_int, []),
    "cc_solve_batch": (C.c_int, [C.c_int, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P),
                                 C.POINTER(_P), C.POINTER(C.c_double), C.POINTER(_P),
                                 C.POINTER(cc_result)]),
    "cc_solve_host": (C.c_int, [_P, _P, _P, _P, C.c_double, _P, C.POINTER(cc_result)]),
    "cc_submit": (C.c_int, [_P, _P, _P, _P, C.c_double, C.POINTER(C.c_uint64)]),
    "cc_poll": (C.c_int, [C.c_uint64, C.POINTER(cc_result)]),
    "cc_assemble_rhs": (C.c_int, [_P, _P, _P, _P, _P]),
    "cc_residual": (C.c_int, [_P, C.c_int, _P, _P, _P, _P]),
    "cc_smooth": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "cc_smooth_noalloc": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "cc_restrict_residual": (C.c_int, [_P, C.c_int, _P, _P, _P, _P]),
    "cc_prolong_add": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "cc_cycle": (C.c_int, [_P, _P, _P, _P]),
    "cc_level_tables": (C.c_int, [_P, C.c_int, _P, _P, _P, C.POINTER(C.c_int)]),
    "cc_level_block": (C.c_int, [_P, C.c_int, _P, C.POINTER(C.c_int)]),
    "cc_kernel_timing": (C.c_int, [_P, C.c_int]),
    "cc_kernel_timing_read": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), C.POINTER(C.c_double)]),
}


def lib():
    """Load libccmg.so (built by __graft_entry__.build()); raise if missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().cc_status_string(int(s)).decode()


def _check(st: int, what: str):
    if st != CC_OK:
        msg = lib().cc_last_error_string().decode()
        if msg:
            what = what + " [" + msg + "]"
        raise CCError(st, what)


def default_options(**kw) -> cc_options:
    o = cc_options()
    lib().cc_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(t) -> int:
    """Device pointer of a contiguous float64 CUDA tensor."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _hptr(a: np.ndarray) -> int:
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous numpy array")
    return a.ctypes.data


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Hierarchy:
    """A cc_handle: the multigrid hierarchy of one domain and operator."""

    def __init__(self, dom, a: float, b: float, c: float, bcs: Sequence, n: int,
                 options: Optional[cc_options] = None, stream=None):
        holes = (cc_hole * max(1, len(dom.holes)))()
        for k, e in enumerate(dom.holes):
            if hasattr(e, "amp"):                             # a flower (workloads.Flower)
                holes[k] = cc_hole(1, e.cx, e.cy, e.r0, e.amp, float(e.k))
            elif hasattr(e, "hgt"):                           # workloads.OutsideRect
                holes[k] = cc_hole(2, e.cx, e.cy, e.w, e.hgt, e.theta)
            else:
                holes[k] = cc_hole(0, e.cx, e.cy, e.r1, e.r2, e.theta)
        d = cc_domain(dom.x0, dom.y0, dom.x1, dom.y1, len(dom.holes), holes)
        arr = (cc_bc * len(bcs))()
        for k, bc in enumerate(bcs):
            arr[k] = cc_bc(bc.kind, bc.alpha1, bc.alpha2)
        h = C.c_void_p()
        opt = options if options is not None else default_options()
        strm = None if opt.host_only else _stream(stream)
        st = lib().cc_setup(C.byref(d), a, b, c, arr, len(bcs), n, C.byref(opt),
                            strm, C.byref(h))
        _check(st, "cc_setup")
        self.h = h
        self.options = opt
        self.info = self.query()

    @classmethod
    def from_domain(cls, dom, a, b, c, n, options=None, stream=None):
        """Conditions from a workloads.Domain (box sides then holes)."""
        return cls(dom, a, b, c, list(dom.box_bc) + list(dom.hole_bc), n, options, stream)

    def clone(self, stream=None) -> "Hierarchy":
        """cc_clone: a handle sharing this hierarchy's tables, with its own
        work arrays, so that solves on both can run at the same time."""
        h = C.c_void_p()
        _check(lib().cc_clone(self.h, _stream(stream), C.byref(h)), "cc_clone")
        c = object.__new__(Hierarchy)
        c.h = h
        c.options = self.options
        c.info = c.query()
        return c

    def close(self):
        if getattr(self, "h", None):
            lib().cc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- queries ---------------------------------------------------------
    def query(self) -> cc_info:
        info = cc_info()
        _check(lib().cc_query(self.h, C.byref(info)), "cc_query")
        return info

    def cell_types(self):
        n = self.info.n
        t = np.zeros(n * n, np.uint8)
        k = np.zeros(n * n, np.uint8)
        v = np.zeros(n * n, np.float64)
        _check(lib().cc_cell_types(self.h, _hptr(t), _hptr(k), _hptr(v)), "cc_cell_types")
        return t.reshape(n, n), k.reshape(n, n), v.reshape(n, n)

    def quadrature_nodes(self):
        nc, nv, nb = C.c_int(), C.c_int64(), C.c_int64()
        L = lib()
        _check(L.cc_quadrature_nodes(self.h, C.byref(nc), C.byref(nv), C.byref(nb), None, None,
                                     None, None, None, None), "cc_quadrature_nodes")
        cell = np.zeros(nc.value, np.int32)
        vptr = np.zeros(nc.value + 1, np.int64)
        vnode = np.zeros((nv.value, 3))
        nbd = self.info.n_bd
        bptr = np.zeros(nbd + 1, np.int64)
        bnode = np.zeros((nb.value, 5))
        bbc = np.zeros(nb.value, np.int32)
        _check(L.cc_quadrature_nodes(self.h, C.byref(nc), C.byref(nv), C.byref(nb), _hptr(cell),
                                     _hptr(vptr), _hptr(vnode), _hptr(bptr), _hptr(bnode),
                                     _hptr(bbc)), "cc_quadrature_nodes")
        return dict(cell=cell, vptr=vptr, vnode=vnode, bptr=bptr, bnode=bnode, bbc=bbc)

    def level_tables(self, level: int):
        n = self.info.level_n[level]
        m = C.c_int()
        _check(lib().cc_level_tables(self.h, level, None, None, None, C.byref(m)), "cc_level_tables")
        kind = np.zeros(n * n, np.uint8)
        lat = np.zeros((max(1, m.value), 15), np.int32)
        beta = np.zeros((max(1, m.value), 16))
        _check(lib().cc_level_tables(self.h, level, _hptr(kind), _hptr(lat), _hptr(beta),
                                     C.byref(m)), "cc_level_tables")
        return kind.reshape(n, n), lat[:m.value], beta[:m.value]

    def level_block(self, level: int) -> np.ndarray:
        """Cells of the level's exactly solved block, in solve order."""
        m = C.c_int()
        _check(lib().cc_level_block(self.h, level, None, C.byref(m)), "cc_level_block")
        out = np.zeros(max(1, m.value), np.int32)
        _check(lib().cc_level_block(self.h, level, _hptr(out), C.byref(m)), "cc_level_block")
        return out[:m.value]

    # --- solves ------------------------------------------------------------
    def solve(self, f, g, u, tol: float, stream=None) -> cc_result:
        r = cc_result()
        st = lib().cc_solve(self.h, _ptr(f), _ptr(g), _ptr(u), tol, _stream(stream), C.byref(r))
        if st not in (CC_OK, CC_ERR_NOT_CONVERGED):
            _check(st, "cc_solve")
        return r

    def solve_host(self, f: np.ndarray, g: np.ndarray, u: np.ndarray, tol: float,
                   stream=None) -> cc_result:
        r = cc_result()
        st = lib().cc_solve_host(self.h, _hptr(f), _hptr(g), _hptr(u), tol, _stream(stream),
                                 C.byref(r))
        if st not in (CC_OK, CC_ERR_NOT_CONVERGED):
            _check(st, "cc_solve_host")
        return r

    def submit(self, f, g, u, tol: float) -> int:
        rid = C.c_uint64()
        _check(lib().cc_submit(self.h, _ptr(f), _ptr(g), _ptr(u), tol, C.byref(rid)), "cc_submit")
        return rid.value

    @staticmethod
    def poll(req_id: int):
        r = cc_result()
        st = lib().cc_poll(req_id, C.byref(r))
        return st, r

    # --- operator-level steps ----------------------------------------------
    def assemble_rhs(self, f, g, b, stream=None):
        _check(lib().cc_assemble_rhs(self.h, _ptr(f), _ptr(g), _ptr(b), _stream(stream)),
               "cc_assemble_rhs")

    def residual(self, level, u, b, r, stream=None):
        _check(lib().cc_residual(self.h, level, _ptr(u), _ptr(b), _ptr(r), _stream(stream)),
               "cc_residual")

    def smooth(self, level, u, b, stream=None):
        _check(lib().cc_smooth(self.h, level, _ptr(u), _ptr(b), _stream(stream)), "cc_smooth")

    def smooth_noalloc(self, level, u, b, stream=None):
        """cc_smooth_noalloc: the sweep of `smooth` with no device allocation;
        its temporaries live in one library-wide device array (see ccmg.h)."""
        _check(lib().cc_smooth_noalloc(self.h, level, _ptr(u), _ptr(b), _stream(stream)),
               "cc_smooth_noalloc")

    def restrict_residual(self, level, u, b, rc, stream=None):
        _check(lib().cc_restrict_residual(self.h, level, _ptr(u), _ptr(b), _ptr(rc),
                                          _stream(stream)), "cc_restrict_residual")

    def prolong_add(self, level, ec, u, stream=None):
        _check(lib().cc_prolong_add(self.h, level, _ptr(ec), _ptr(u), _stream(stream)),
               "cc_prolong_add")

    def cycle(self, u, b, stream=None):
        _check(lib().cc_cycle(self.h, _ptr(u), _ptr(b), _stream(stream)), "cc_cycle")

    def kernel_timing(self, which: int):
        """0 off, 1 finest-level sweeps, 2 one-launch dense block solves."""
        _check(lib().cc_kernel_timing(self.h, int(which)), "cc_kernel_timing")

    def kernel_timing_read(self):
        """(timed intervals, total ms, algorithmic bytes per interval, bytes the
        kernels move per interval)"""
        n, ms, by, mv = C.c_int64(), C.c_double(), C.c_double(), C.c_double()
        _check(lib().cc_kernel_timing_read(self.h, C.byref(n), C.byref(ms), C.byref(by),
                                           C.byref(mv)), "cc_kernel_timing_read")
        return n.value, ms.value, by.value, mv.value


def solve_batch(hs, fs, gs, us, tols, streams=None):
    """cc_solve_batch: solve i on handle hs[i] (distinct handles), all at once.
    Returns the list of cc_result; raises on CC_ERR_ARG / CC_ERR_CUDA."""
    n = len(hs)
    P = _P * max(1, n)
    h = P(*[x.h for x in hs])
    f = P(*[_ptr(x) for x in fs])
    g = P(*[_ptr(x) for x in gs])
    u = P(*[_ptr(x) for x in us])
    t = (C.c_double * max(1, n))(*[float(x) for x in tols])
    st_arr = P(*[_stream(x) for x in streams]) if streams is not None else None
    out = (cc_result * max(1, n))()
    st = lib().cc_solve_batch(n, h, f, g, u, t, st_arr, out)
    if st not in (CC_OK, CC_ERR_NOT_CONVERGED, CC_ERR_DIVERGED):
        _check(st, "cc_solve_batch")
    return [out[i] for i in range(n)]


def serve_budget(nbytes: int):
    """cc_serve_budget: cap on the device memory of all serving clones (0: none)."""
    _check(lib().cc_serve_budget(int(nbytes)), "cc_serve_budget")


def cache_clear():
    """cc_cache_clear: drop the setup cache (handles made from it stay valid)."""
    _check(lib().cc_cache_clear(), "cc_cache_clear")
