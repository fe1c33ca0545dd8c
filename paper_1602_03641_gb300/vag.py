"""ctypes binding of libvag (include/vag.h): argument marshalling only.

Every function of the C ABI is exposed under its own name on the loaded
library object (``lib()``), plus thin helpers (``Context``, ``System``) that
turn numpy arrays (host) or torch CUDA tensors (device) into the plain
pointers and sizes the ABI takes.  All arithmetic runs in the CUDA library;
if ``libvag.so`` is missing or cannot be loaded, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import sys as _sys
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvag.so")

VAG_OK, VAG_EINVAL, VAG_ENOMEM, VAG_EBUDGET, VAG_ENOTCONVERGED = 0, 1, 2, 3, 4
VAG_EBREAKDOWN, VAG_ETIMEOUT, VAG_ECUDA, VAG_EMESH = 5, 6, 7, 8
VAG_MEM_HOST, VAG_MEM_DEVICE = 0, 1
VAG_FP64, VAG_MIXED, VAG_MIXED_F16, VAG_FP64_PC32 = 0, 1, 2, 3
VAG_PC_JACOBI, VAG_PC_CHEBYSHEV, VAG_PC_AMG, VAG_PC_AMG_RS = 0, 1, 2, 3
VAG_KRYLOV_CG, VAG_KRYLOV_BICGSTAB, VAG_KRYLOV_GMRES = 0, 1, 2
VAG_KERNEL_SPMV, VAG_KERNEL_SMOOTH, VAG_KERNEL_TRANSPORT_STEP, VAG_KERNEL_SPMV32 = 0, 1, 2, 3
VAG_KERNEL_CELL_LOCAL = 4
VAG_SHAPE_HEX, VAG_SHAPE_TET, VAG_SHAPE_PRISM, VAG_SHAPE_PYRAMID = 0, 1, 2, 3
# local faces of each shape, each cyclic (the library's tables, include/vag.h)
SHAPE_FACES = {
    0: [(0, 2, 6, 4), (1, 3, 7, 5), (0, 1, 5, 4), (2, 3, 7, 6), (0, 1, 3, 2), (4, 5, 7, 6)],
    1: [(1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1)],
    2: [(0, 1, 2), (3, 4, 5), (0, 1, 4, 3), (1, 2, 5, 4), (2, 0, 3, 5)],
    3: [(0, 1, 2, 3), (0, 1, 4), (1, 2, 4), (2, 3, 4), (3, 0, 4)],
}

STATUS_NAMES = {0: "VAG_OK", 1: "VAG_EINVAL", 2: "VAG_ENOMEM", 3: "VAG_EBUDGET", 4: "VAG_ENOTCONVERGED",
                5: "VAG_EBREAKDOWN", 6: "VAG_ETIMEOUT", 7: "VAG_ECUDA", 8: "VAG_EMESH"}


class vag_mesh(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("xyz", C.c_void_p), ("n_cells", C.c_int32),
                ("cell_nodes", C.c_void_p), ("n_ff", C.c_int32), ("ff_nodes", C.c_void_p),
                ("n_faces", C.c_int32), ("face_node_ptr", C.c_void_p), ("face_node_idx", C.c_void_p),
                ("cell_face_ptr", C.c_void_p), ("cell_face_idx", C.c_void_p), ("ff_face_ids", C.c_void_p)]


class vag_props(C.Structure):
    _fields_ = [("lambda_m", C.c_void_p), ("lambda_f", C.c_void_p), ("d_f", C.c_void_p), ("mu", C.c_double),
                ("n_perf", C.c_int32), ("well_ff", C.c_void_p), ("well_wi", C.c_void_p), ("well_pw", C.c_void_p),
                ("well_q", C.c_void_p), ("well_cin", C.c_void_p)]


class vag_dirichlet(C.Structure):
    _fields_ = [("n_dir", C.c_int32), ("nodes", C.c_void_p), ("values", C.c_void_p)]


class vag_system_info(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_cells", C.c_int32), ("n_ff", C.c_int32), ("n_dir", C.c_int32),
                ("n_rows", C.c_int32), ("nnz", C.c_int64), ("n_frac_cells", C.c_int32), ("n_cv", C.c_int32),
                ("nnz_transport", C.c_int64), ("device_bytes", C.c_size_t)]


class vag_solve_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("precond", C.c_int), ("rtol", C.c_double), ("maxit", C.c_int32),
                ("mem", C.c_int), ("krylov", C.c_int32), ("inner_rtol", C.c_double)]


class vag_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("outer", C.c_int32), ("rel_residual", C.c_double),
                ("ms_setup", C.c_double), ("ms_solve", C.c_double), ("status", C.c_int)]


class vag_transport_opts(C.Structure):
    _fields_ = [("phi_m", C.c_void_p), ("phi_f", C.c_void_p), ("cbar", C.c_void_p), ("omega", C.c_double),
                ("cfl", C.c_double), ("dt", C.c_double), ("n_steps", C.c_int32), ("mem", C.c_int)]


class vag_transport_info(C.Structure):
    _fields_ = [("dt_max", C.c_double), ("dt", C.c_double), ("steps", C.c_int32), ("ms", C.c_double)]


class vag_server_opts(C.Structure):
    _fields_ = [("device", C.c_int), ("mem_budget_bytes", C.c_size_t), ("slots", C.c_int32),
                ("max_batch", C.c_int32)]


class vag_request(C.Structure):
    _fields_ = [("mesh", vag_mesh), ("props", vag_props), ("bc", vag_dirichlet),
                ("phi_m", C.c_void_p), ("phi_f", C.c_void_p), ("cbar", C.c_void_p), ("c0", C.c_void_p),
                ("omega", C.c_double), ("cfl", C.c_double), ("n_steps", C.c_int32),
                ("precision", C.c_int), ("precond", C.c_int), ("rtol", C.c_double), ("maxit", C.c_int32),
                ("u_out", C.c_void_p), ("c_out", C.c_void_p)]


class vag_result(C.Structure):
    _fields_ = [("status", C.c_int), ("solve", vag_solve_info), ("transport", vag_transport_info),
                ("latency_ms", C.c_double), ("queue_ms", C.c_double), ("batch_size", C.c_int32)]


class vag_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("rejected", C.c_uint64),
                ("in_queue", C.c_uint64), ("in_flight", C.c_uint64), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("solves_per_s", C.c_double), ("bytes_reserved", C.c_size_t), ("peak_bytes", C.c_size_t)]


P = C.c_void_p
_SIGS = {
    "vag_ctx_create": (C.c_int, [C.c_int, C.c_size_t, C.POINTER(P)]),
    "vag_ctx_destroy": (None, [P]),
    "vag_ctx_set_stream": (C.c_int, [P, P]),
    "vag_last_error": (C.c_char_p, [P]),
    "vag_ctx_bytes_in_use": (C.c_size_t, [P]),
    "vag_launch_count": (C.c_ulonglong, []),
    "vag_assemble": (C.c_int, [P, C.POINTER(vag_mesh), C.POINTER(vag_props), C.POINTER(vag_dirichlet),
                               C.c_int, C.POINTER(P)]),
    "vag_update_props": (C.c_int, [P, C.POINTER(vag_props), C.c_int]),
    "vag_assemble_batch": (C.c_int, [P, C.c_int32, C.POINTER(vag_mesh), C.POINTER(vag_props),
                                     C.POINTER(vag_dirichlet), C.c_int, C.POINTER(P)]),
    "vag_system_get_batch": (C.c_int, [P, C.POINTER(C.c_int32), P, P, P, P]),
    "vag_solve_get_infos": (C.c_int, [P, C.POINTER(vag_solve_info)]),
    "vag_transport_get_dts": (C.c_int, [P, P, P]),
    "vag_spmv_dot_noalloc": (C.c_int, [C.c_int32, P, P, P, P, P, P, P]),
    "vag_server_create": (C.c_int, [C.POINTER(vag_server_opts), C.POINTER(P)]),
    "vag_server_submit": (C.c_int, [P, C.POINTER(vag_request), C.POINTER(C.c_uint64)]),
    "vag_server_wait": (C.c_int, [P, C.c_uint64, C.c_int32, C.POINTER(vag_result)]),
    "vag_server_get_stats": (C.c_int, [P, C.POINTER(vag_server_stats)]),
    "vag_server_last_error": (C.c_char_p, [P]),
    "vag_server_destroy": (None, [P]),
    "vag_system_destroy": (None, [P]),
    "vag_system_get_info": (C.c_int, [P, C.POINTER(vag_system_info)]),
    "vag_solve": (C.c_int, [P, C.POINTER(vag_solve_opts), P, C.POINTER(vag_solve_info)]),
    "vag_spmv": (C.c_int, [P, P, P, C.c_int]),
    "vag_kernel_time": (C.c_int, [P, C.c_int, C.c_int32, C.POINTER(C.c_double)]),
    "vag_transport": (C.c_int, [P, C.POINTER(vag_transport_opts), P, C.POINTER(vag_transport_info)]),
    "vag_transport_step": (C.c_int, [P, C.POINTER(vag_transport_opts), P, C.POINTER(C.c_double),
                                     C.POINTER(vag_transport_info)]),
    "vag_export_system": (C.c_int, [P, P, P, P, P, P, C.c_int]),
    "vag_export_fluxes": (C.c_int, [P, P, P, P, C.c_int]),
    "vag_set_fluxes": (C.c_int, [P, P, P, P, C.c_int]),
    "vag_export_porous_volumes": (C.c_int, [P, P, C.c_int]),
    "vag_export_well_rates": (C.c_int, [P, P, C.c_int]),
    "vag_export_cells": (C.c_int, [P, P, P, P, C.c_int]),
    "vag_peaceman_wi": (C.c_int, [C.c_int32, P, P, P, P, P, C.c_double, P]),
}

_LIB = None


def lib():
    """Load libvag.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1602_03641_gb300.build.build() first")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            if hasattr(L, name):
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
        _LIB = L
    return _LIB


def declared_symbols():
    return list(_SIGS)


def launch_count() -> int:
    """Kernels launched by libvag in this process so far."""
    return int(lib().vag_launch_count())


class VagError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


# ----------------------------------------------------------------- marshal --

def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype=None):
    """Data pointer of a numpy array (host) or torch tensor (device)."""
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    a = x
    if not (a.flags["C_CONTIGUOUS"]):
        raise ValueError("array must be C-contiguous")
    if dtype is not None and a.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {a.dtype}")
    return a.ctypes.data


def _size(a):
    return int(a.numel() if _is_torch(a) else a.size)


def _general_mesh(xyz, face_node_ptr, face_node_idx, cell_face_ptr, cell_face_idx, ff_face_ids):
    """vag_mesh in the general polyhedral form (cell_nodes = NULL)."""
    return vag_mesh(_size(xyz) // 3, _ptr(xyz, np.float64), _size(cell_face_ptr) - 1, None, _size(ff_face_ids), None,
                    _size(face_node_ptr) - 1, _ptr(face_node_ptr, np.int32), _ptr(face_node_idx, np.int32),
                    _ptr(cell_face_ptr, np.int32), _ptr(cell_face_idx, np.int32), _ptr(ff_face_ids, np.int32))


WELL_KEYS = ("ff", "wi", "pw", "q", "cin")


def _wells_arrays(wells):
    """wells: None or a dict with per-perforation arrays ff (fracture-face
    index), wi, pw, q, cin (see vag_props); numpy host or CUDA tensors."""
    if wells is None:
        return []
    return [wells[k] for k in WELL_KEYS]


def _props(lambda_m, lambda_f, d_f, mu, wells=None):
    w = _wells_arrays(wells)
    if not w:
        return vag_props(_ptr(lambda_m, np.float64), _ptr(lambda_f, np.float64), _ptr(d_f, np.float64), float(mu))
    return vag_props(_ptr(lambda_m, np.float64), _ptr(lambda_f, np.float64), _ptr(d_f, np.float64), float(mu),
                     _size(w[0]), _ptr(w[0], np.int32), _ptr(w[1], np.float64), _ptr(w[2], np.float64),
                     _ptr(w[3], np.float64), _ptr(w[4], np.float64))


def peaceman_wi(dx, dz, d_f, lambda_f, r_w, mu=1.0):
    """vag_peaceman_wi: Peaceman well indices (host arrays, broadcast)."""
    dx, dz, d_f, lambda_f, r_w = [np.ascontiguousarray(a, np.float64) for a in
                                  np.broadcast_arrays(dx, dz, d_f, lambda_f, r_w)]
    out = np.empty(dx.size)
    st = lib().vag_peaceman_wi(dx.size, _ptr(dx), _ptr(dz), _ptr(d_f), _ptr(lambda_f), _ptr(r_w), float(mu),
                               _ptr(out))
    if st != VAG_OK:
        raise VagError(st, "vag_peaceman_wi: an input is not positive or r_0 <= r_w")
    return out


def _mem_of(*xs):
    kinds = set()
    for x in xs:
        if x is None:
            continue
        kinds.add(VAG_MEM_DEVICE if (_is_torch(x) and x.is_cuda) else VAG_MEM_HOST)
    if len(kinds) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return kinds.pop() if kinds else VAG_MEM_HOST


class Context:
    def __init__(self, device: int = 0, budget_bytes: int = 0):
        self._L = lib()
        h = P()
        st = self._L.vag_ctx_create(device, budget_bytes, C.byref(h))
        if st != VAG_OK:
            raise VagError(st, "vag_ctx_create failed")
        self.h = h

    def check(self, st):
        if st != VAG_OK:
            raise VagError(st, self._L.vag_last_error(self.h).decode())

    def set_stream(self, stream_ptr: Optional[int]):
        self.check(self._L.vag_ctx_set_stream(self.h, P(stream_ptr) if stream_ptr else None))

    def bytes_in_use(self):
        return int(self._L.vag_ctx_bytes_in_use(self.h))

    def close(self):
        if getattr(self, "h", None):
            self._L.vag_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        if _sys.is_finalizing():      # the CUDA runtime may already be gone
            return
        try:
            self.close()
        except Exception:
            pass

    def assemble(self, xyz, cell_nodes, ff_nodes, lambda_m, lambda_f, d_f, mu, dir_nodes, dir_values, wells=None):
        """Arrays: numpy (host) or CUDA tensors (device), float64 / int32."""
        mem = _mem_of(xyz, cell_nodes, ff_nodes, lambda_m, lambda_f, d_f, dir_nodes, dir_values,
                      *_wells_arrays(wells))
        m = vag_mesh(int(len(xyz) // 3 if xyz.ndim == 1 else xyz.shape[0]), _ptr(xyz, np.float64),
                     int(cell_nodes.numel() // 8 if _is_torch(cell_nodes) else cell_nodes.size // 8),
                     _ptr(cell_nodes, np.int32),
                     int(ff_nodes.numel() // 4 if _is_torch(ff_nodes) else ff_nodes.size // 4),
                     _ptr(ff_nodes, np.int32))
        p = _props(lambda_m, lambda_f, d_f, mu, wells)
        nd = int(dir_nodes.numel() if _is_torch(dir_nodes) else dir_nodes.size)
        b = vag_dirichlet(nd, _ptr(dir_nodes, np.int32), _ptr(dir_values, np.float64))
        h = P()
        self.check(self._L.vag_assemble(self.h, C.byref(m), C.byref(p), C.byref(b), mem, C.byref(h)))
        return System(self, h)

    def assemble_general(self, xyz, face_node_ptr, face_node_idx, cell_face_ptr, cell_face_idx, ff_face_ids,
                         lambda_m, lambda_f, d_f, mu, dir_nodes, dir_values, wells=None):
        """The general polyhedral descriptor (faces as cyclic node lists,
        cells as face lists, fracture faces as face ids); numpy (host) or CUDA
        tensors (device), float64 / int32."""
        mem = _mem_of(xyz, face_node_ptr, face_node_idx, cell_face_ptr, cell_face_idx, ff_face_ids, lambda_m,
                      lambda_f, d_f, dir_nodes, dir_values, *_wells_arrays(wells))
        m = _general_mesh(xyz, face_node_ptr, face_node_idx, cell_face_ptr, cell_face_idx, ff_face_ids)
        p = _props(lambda_m, lambda_f, d_f, mu, wells)
        nd = _size(dir_nodes)
        b = vag_dirichlet(nd, _ptr(dir_nodes, np.int32), _ptr(dir_values, np.float64))
        h = P()
        self.check(self._L.vag_assemble(self.h, C.byref(m), C.byref(p), C.byref(b), mem, C.byref(h)))
        return System(self, h)

    def assemble_batch(self, problems):
        """problems: list of dicts with keys xyz, cell_nodes, ff_nodes,
        lambda_m, lambda_f, d_f, mu, dir_nodes, dir_values (numpy host or
        CUDA tensors, all of one kind)."""
        n = len(problems)
        ms, ps, bs = (vag_mesh * n)(), (vag_props * n)(), (vag_dirichlet * n)()
        keep = []
        mem = None
        for i, q in enumerate(problems):
            general = "face_node_ptr" in q
            topo = ([q[k] for k in ("face_node_ptr", "face_node_idx", "cell_face_ptr", "cell_face_idx",
                                    "ff_face_ids")] if general else [q["cell_nodes"], q["ff_nodes"]])
            arrs = [q["xyz"], *topo, q["lambda_m"], q["lambda_f"], q["d_f"], q["dir_nodes"], q["dir_values"],
                    *_wells_arrays(q.get("wells"))]
            keep.append(arrs)
            mm = _mem_of(*arrs)
            if mem is None:
                mem = mm
            elif mm != mem:
                raise ValueError("mix of host and device arrays in one batch")
            size = _size
            if general:
                ms[i] = _general_mesh(q["xyz"], *topo)
            else:
                ms[i] = vag_mesh(size(q["xyz"]) // 3, _ptr(q["xyz"], np.float64), size(q["cell_nodes"]) // 8,
                                 _ptr(q["cell_nodes"], np.int32), size(q["ff_nodes"]) // 4,
                                 _ptr(q["ff_nodes"], np.int32))
            ps[i] = _props(q["lambda_m"], q["lambda_f"], q["d_f"], q["mu"], q.get("wells"))
            bs[i] = vag_dirichlet(size(q["dir_nodes"]), _ptr(q["dir_nodes"], np.int32),
                                  _ptr(q["dir_values"], np.float64))
        h = P()
        self.check(self._L.vag_assemble_batch(self.h, n, ms, ps, bs, mem, C.byref(h)))
        return System(self, h)


class System:
    def __init__(self, ctx: Context, h):
        self.ctx = ctx
        self.h = h
        self._L = ctx._L

    def close(self):
        if getattr(self, "h", None):
            self._L.vag_system_destroy(self.h)
            self.h = None

    def __del__(self):
        if _sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> vag_system_info:
        i = vag_system_info()
        self.ctx.check(self._L.vag_system_get_info(self.h, C.byref(i)))
        return i

    def batch_layout(self):
        """dict of numpy arrays (n_sys+1): node_start, ff_start, cell_start, row_start."""
        n = C.c_int32()
        self.ctx.check(self._L.vag_system_get_batch(self.h, C.byref(n), None, None, None, None))
        out = {k: np.empty(n.value + 1, np.int32) for k in ("node_start", "ff_start", "cell_start", "row_start")}
        self.ctx.check(self._L.vag_system_get_batch(self.h, C.byref(n), _ptr(out["node_start"]), _ptr(out["ff_start"]),
                                                    _ptr(out["cell_start"]), _ptr(out["row_start"])))
        out["n_sys"] = n.value
        return out

    def solve_infos(self):
        n = self.batch_layout()["n_sys"]
        arr = (vag_solve_info * n)()
        self.ctx.check(self._L.vag_solve_get_infos(self.h, arr))
        return list(arr)

    def transport_dts(self):
        n = self.batch_layout()["n_sys"]
        dmax = np.empty(n); dt = np.empty(n)
        self.ctx.check(self._L.vag_transport_get_dts(self.h, _ptr(dmax), _ptr(dt)))
        return dmax, dt

    def update_props(self, lambda_m, lambda_f, d_f, mu, wells=None):
        mem = _mem_of(lambda_m, lambda_f, d_f, *_wells_arrays(wells))
        p = _props(lambda_m, lambda_f, d_f, mu, wells)
        self.ctx.check(self._L.vag_update_props(self.h, C.byref(p), mem))

    def well_rates(self, n_perf):
        """Rates leaving each perforated face into its well (last solve)."""
        out = np.empty(max(int(n_perf), 1))
        self.ctx.check(self._L.vag_export_well_rates(self.h, _ptr(out), VAG_MEM_HOST))
        return out[:n_perf]

    def solve(self, out=None, precision=VAG_FP64, precond=VAG_PC_JACOBI, rtol=1e-12, maxit=20000,
              raise_on_error=True, krylov=VAG_KRYLOV_CG, inner_rtol=0.0):
        """Returns (u, info); u over [nodes | ffaces | cells]."""
        n = self.info().n_cv
        if out is None:
            out = np.empty(n)
        mem = _mem_of(out)
        o = vag_solve_opts(precision, precond, float(rtol), int(maxit), mem, int(krylov), float(inner_rtol))
        inf = vag_solve_info()
        st = self._L.vag_solve(self.h, C.byref(o), _ptr(out, np.float64), C.byref(inf))
        if raise_on_error:
            self.ctx.check(st)
        inf.ret = st
        return out, inf

    def spmv(self, x, y=None):
        if y is None:
            y = np.empty_like(x)
        mem = _mem_of(x, y)
        self.ctx.check(self._L.vag_spmv(self.h, _ptr(x, np.float64), _ptr(y, np.float64), mem))
        return y

    def kernel_time(self, kernel, reps=100):
        """Mean ms of one launch of a hot kernel on this system's data
        (VAG_KERNEL_SPMV, VAG_KERNEL_SMOOTH, VAG_KERNEL_TRANSPORT_STEP, VAG_KERNEL_SPMV32,
        VAG_KERNEL_CELL_LOCAL)."""
        ms = C.c_double()
        self.ctx.check(self._L.vag_kernel_time(self.h, int(kernel), int(reps), C.byref(ms)))
        return ms.value

    def transport(self, c, phi_m, phi_f, cbar, n_steps, cfl=0.9, dt=0.0, omega=0.5):
        """c is updated in place (numpy or CUDA tensor, [n_cv])."""
        mem = _mem_of(c, phi_m, phi_f, cbar)
        o = vag_transport_opts(_ptr(phi_m, np.float64), _ptr(phi_f, np.float64), _ptr(cbar, np.float64),
                               float(omega), float(cfl), float(dt), int(n_steps), mem)
        inf = vag_transport_info()
        self.ctx.check(self._L.vag_transport(self.h, C.byref(o), _ptr(c, np.float64), C.byref(inf)))
        return inf

    def transport_step(self, c, phi_m, phi_f, cbar, n_steps, cfl=0.9, dt=0.0, omega=0.5):
        """vag_transport_step: as transport(), returning (info, step used)."""
        mem = _mem_of(c, phi_m, phi_f, cbar)
        o = vag_transport_opts(_ptr(phi_m, np.float64), _ptr(phi_f, np.float64), _ptr(cbar, np.float64),
                               float(omega), float(cfl), float(dt), int(n_steps), mem)
        inf = vag_transport_info()
        used = C.c_double(-1.0)
        self.ctx.check(self._L.vag_transport_step(self.h, C.byref(o), _ptr(c, np.float64), C.byref(used),
                                                  C.byref(inf)))
        return inf, used.value

    def export_system(self):
        i = self.info()
        rowptr = np.empty(i.n_rows + 1, np.int32)
        col = np.empty(i.nnz, np.int32)
        val = np.empty(i.nnz)
        rhs = np.empty(i.n_rows)
        row_dof = np.empty(i.n_rows, np.int32)
        self.ctx.check(self._L.vag_export_system(self.h, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(rhs),
                                                 _ptr(row_dof), VAG_MEM_HOST))
        return dict(rowptr=rowptr, col=col, val=val, rhs=rhs, row_dof=row_dof)

    def export_cells(self):
        """(cell_nodes [n_cells, 8], shape [n_cells], ff_nodes [n_ff, 4]): the
        numbering the kernels run on (-1 in unused slots)."""
        i = self.info()
        cn = np.empty(8 * i.n_cells, np.int32)
        sh = np.empty(i.n_cells, np.int8)
        ffn = np.empty(max(4 * i.n_ff, 1), np.int32)
        self.ctx.check(self._L.vag_export_cells(self.h, _ptr(cn), _ptr(sh), _ptr(ffn), VAG_MEM_HOST))
        return cn.reshape(-1, 8), sh, ffn[:4 * i.n_ff].reshape(-1, 4)

    def export_fluxes(self):
        i = self.info()
        Fcn = np.empty(8 * i.n_cells)
        Fcf = np.empty(6 * i.n_cells)
        Fff = np.empty(max(4 * i.n_ff, 1))
        self.ctx.check(self._L.vag_export_fluxes(self.h, _ptr(Fcn), _ptr(Fcf), _ptr(Fff), VAG_MEM_HOST))
        return Fcn.reshape(-1, 8), Fcf.reshape(-1, 6), Fff[:4 * i.n_ff].reshape(-1, 4)

    def set_fluxes(self, Fcn, Fcf, Fff):
        Fcn = np.ascontiguousarray(Fcn, np.float64)
        Fcf = np.ascontiguousarray(Fcf, np.float64)
        Fff = np.ascontiguousarray(Fff, np.float64)
        self.ctx.check(self._L.vag_set_fluxes(self.h, _ptr(Fcn), _ptr(Fcf), _ptr(Fff) if Fff.size else None,
                                              VAG_MEM_HOST))

    def export_porous_volumes(self):
        phi = np.empty(self.info().n_cv)
        self.ctx.check(self._L.vag_export_porous_volumes(self.h, _ptr(phi), VAG_MEM_HOST))
        return phi


def _wells_of(pb):
    w = getattr(pb, "wells", None)
    if not w:
        return None
    return dict(ff=np.ascontiguousarray(w["ff"], np.int32), wi=np.ascontiguousarray(w["wi"], np.float64),
                pw=np.ascontiguousarray(w["pw"], np.float64), q=np.ascontiguousarray(w["q"], np.float64),
                cin=np.ascontiguousarray(w["cin"], np.float64))


def _to_device(q):
    import torch
    out = {}
    for k, v in q.items():
        out[k] = ({kk: torch.from_numpy(vv).cuda() for kk, vv in v.items()} if isinstance(v, dict)
                  else torch.from_numpy(v).cuda())
    return out


def is_hex_problem(pb):
    """True when every cell is a hexahedron given by 8 node slots (the fast path)."""
    cn = np.asarray(pb.cell_nodes)
    return cn.ndim == 2 and cn.shape[1] == 8 and bool((cn >= 0).all())


def problem_arrays(pb, device=False):
    """The ABI arrays of a ``vag_inputs.Problem``-like object as a dict (the
    hexahedral fast path; ``general_arrays`` for other cells)."""
    q = dict(xyz=np.ascontiguousarray(pb.xyz, np.float64).ravel(),
             cell_nodes=np.ascontiguousarray(pb.cell_nodes, np.int32).ravel(),
             ff_nodes=np.ascontiguousarray(pb.ff_nodes, np.int32).ravel(),
             lambda_m=np.ascontiguousarray(pb.lambda_m, np.float64).ravel(),
             lambda_f=np.ascontiguousarray(pb.lambda_f, np.float64), d_f=np.ascontiguousarray(pb.d_f, np.float64),
             dir_nodes=np.ascontiguousarray(pb.dir_nodes, np.int32),
             dir_values=np.ascontiguousarray(pb.dir_values, np.float64))
    w = _wells_of(pb)
    if w is not None:
        q["wells"] = w
    if device:
        q = _to_device(q)
    q["mu"] = pb.mu
    return q


def _ragged(a):
    """CSR (ptr, idx) of a -1-padded 2-D id array (padding after the ids)."""
    a = np.ascontiguousarray(a, np.int32)
    cnt = (a >= 0).sum(axis=1)
    ptr = np.zeros(a.shape[0] + 1, np.int32)
    np.cumsum(cnt, out=ptr[1:])
    return ptr, np.ascontiguousarray(a[a >= 0], np.int32)


def general_arrays(pb, device=False):
    """The general polyhedral descriptor of a ``vag_inputs.Problem``-like
    object (attributes faces [n_faces, q_max] and cell_faces [n_cells, f_max],
    -1-padded, ff_faces and the physical data) as a dict for
    ``Context.assemble_general`` or ``Context.assemble_batch``."""
    fptr, fidx = _ragged(pb.faces)
    cptr, cidx = _ragged(pb.cell_faces)
    q = dict(xyz=np.ascontiguousarray(pb.xyz, np.float64).ravel(),
             face_node_ptr=fptr, face_node_idx=fidx, cell_face_ptr=cptr, cell_face_idx=cidx,
             ff_face_ids=np.ascontiguousarray(pb.ff_faces, np.int32),
             lambda_m=np.ascontiguousarray(pb.lambda_m, np.float64).ravel(),
             lambda_f=np.ascontiguousarray(pb.lambda_f, np.float64), d_f=np.ascontiguousarray(pb.d_f, np.float64),
             dir_nodes=np.ascontiguousarray(pb.dir_nodes, np.int32),
             dir_values=np.ascontiguousarray(pb.dir_values, np.float64))
    w = _wells_of(pb)
    if w is not None:
        q["wells"] = w
    if device:
        q = _to_device(q)
    q["mu"] = pb.mu
    return q


def assemble_problem(ctx: Context, pb, device=False, general=None):
    """Marshal a ``vag_inputs.Problem``-like object.  The hexahedral fast
    path is used when every cell is a hexahedron (attributes xyz, cell_nodes,
    ff_nodes, ...), the general descriptor otherwise or with general=True."""
    if general is None:
        general = not is_hex_problem(pb)
    if general:
        q = general_arrays(pb, device)
        return ctx.assemble_general(q["xyz"], q["face_node_ptr"], q["face_node_idx"], q["cell_face_ptr"],
                                    q["cell_face_idx"], q["ff_face_ids"], q["lambda_m"], q["lambda_f"], q["d_f"],
                                    q["mu"], q["dir_nodes"], q["dir_values"], q.get("wells"))
    q = problem_arrays(pb, device)
    return ctx.assemble(q["xyz"], q["cell_nodes"], q["ff_nodes"], q["lambda_m"], q["lambda_f"], q["d_f"], q["mu"],
                        q["dir_nodes"], q["dir_values"], q.get("wells"))


class Server:
    """Continuous-batching request server (vag_server_*).  Requests are
    ``vag_inputs.Problem``-like objects; inputs are copied at submit, outputs
    land in numpy arrays owned by this object until the ticket is waited."""

    def __init__(self, device=0, budget_bytes=0, slots=2, max_batch=64):
        self._L = lib()
        h = P()
        st = self._L.vag_server_create(C.byref(vag_server_opts(device, budget_bytes, slots, max_batch)), C.byref(h))
        if st != VAG_OK:
            raise VagError(st, "vag_server_create failed")
        self.h = h
        self._out = {}

    def submit(self, pb, n_steps=0, precision=VAG_FP64, precond=VAG_PC_JACOBI, rtol=1e-8, maxit=20000,
               cfl=0.9, omega=0.5, general=None):
        """general: pass the mesh in the general polyhedral form (default:
        when some cell is not a hexahedron)."""
        if general is None:
            general = not is_hex_problem(pb)
        a = general_arrays(pb) if general else problem_arrays(pb)
        n_cv = pb.n_nodes + pb.n_ff + pb.n_cells
        u = np.empty(n_cv)
        c = np.empty(n_cv)
        keep = [a, np.ascontiguousarray(pb.phi_m, np.float64), np.ascontiguousarray(pb.phi_f, np.float64),
                np.ascontiguousarray(pb.cbar, np.float64)]
        if general:
            m = _general_mesh(a["xyz"], a["face_node_ptr"], a["face_node_idx"], a["cell_face_ptr"],
                              a["cell_face_idx"], a["ff_face_ids"])
        else:
            m = vag_mesh(pb.n_nodes, _ptr(a["xyz"]), pb.n_cells, _ptr(a["cell_nodes"]), pb.n_ff,
                         _ptr(a["ff_nodes"]))
        pr = _props(a["lambda_m"], a["lambda_f"], a["d_f"], pb.mu, a.get("wells"))
        bc = vag_dirichlet(len(a["dir_nodes"]), _ptr(a["dir_nodes"]), _ptr(a["dir_values"]))
        q = vag_request(m, pr, bc, _ptr(keep[1]), _ptr(keep[2]), _ptr(keep[3]), None, float(omega), float(cfl),
                        int(n_steps), precision, precond, float(rtol), int(maxit), _ptr(u), _ptr(c))
        t = C.c_uint64()
        st = self._L.vag_server_submit(self.h, C.byref(q), C.byref(t))
        if st != VAG_OK:
            raise VagError(st, self._L.vag_server_last_error(self.h).decode())
        self._out[t.value] = (u, c)
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        r = vag_result()
        st = self._L.vag_server_wait(self.h, ticket, int(timeout_ms), C.byref(r))
        if st != VAG_OK:
            raise VagError(st, "wait")
        u, c = self._out.pop(ticket)
        return u, c, r

    def stats(self):
        s = vag_server_stats()
        self._L.vag_server_get_stats(self.h, C.byref(s))
        return s

    def close(self):
        if getattr(self, "h", None):
            self._L.vag_server_destroy(self.h)
            self.h = None

    def __del__(self):
        if _sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass
