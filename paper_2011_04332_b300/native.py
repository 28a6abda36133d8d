"""Thin ctypes binding of the C ABI in include/npfem.h (argument marshalling only).

Every step of the hot path runs in libnpfem.so; this module only converts Python
objects (numpy meshes, torch device tensors) into plain pointers and sizes.  It
raises if the shared library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnpfem.so")

FP64 = 0
FP32FORM = 1

CELL_LINESEARCH_FAIL = 1
CELL_DEGENERATE = 2
CELL_NONFINITE = 4
CELL_ITER_LIMIT = 8
CELL_CG_NOT_CONVERGED = 16

ERRORS = {-1: "INVALID_ARG", -2: "BAD_MESH", -3: "NOT_SPD", -4: "CUDA", -5: "OOM", -6: "UNSUPPORTED"}


class NpfemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"npfem error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class _Mesh(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tris", C.c_int32),
                ("rest_xyz", C.POINTER(C.c_double)), ("tris", C.POINTER(C.c_int32))]


class _Material(C.Structure):
    _fields_ = [("w_strain", C.c_double), ("w_bend", C.c_double), ("w_area", C.c_double),
                ("w_vol", C.c_double), ("density", C.c_double), ("c_alpha", C.c_double), ("c_beta", C.c_double),
                ("s_min", C.c_double), ("s_max", C.c_double)]


class _Opts(C.Structure):
    _fields_ = [("iters", C.c_int32), ("alpha_log_len", C.c_int32), ("alpha_log", C.c_void_p),
                ("max_iters", C.c_int32), ("tol", C.c_double), ("iters_done", C.c_void_p)]


class _CollisionParams(C.Structure):
    _fields_ = [("radius", C.c_double), ("delta", C.c_double), ("weight", C.c_double), ("walls", C.c_int32),
                ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3)]


class _TypeInfo(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tris", C.c_int32), ("n_hinges", C.c_int32),
                ("nnz_factor", C.c_int64), ("solve_chunks", C.c_int64),
                ("rest_area", C.c_double), ("rest_volume", C.c_double), ("total_mass", C.c_double),
                ("tri_colours", C.c_int32), ("hinge_colours", C.c_int32)]


_lib = None


def load_library() -> C.CDLL:
    """Load libnpfem.so (built in-tree by paper_2011_04332_b300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libnpfem.so not built at {LIB_PATH}: run paper_2011_04332_b300/build.py")
    lib = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    sig = {
        "npfem_create_cell_type": [C.POINTER(_Mesh), C.POINTER(_Material), C.c_double, C.POINTER(vp)],
        "npfem_destroy_cell_type": [vp],
        "npfem_cell_type_info": [vp, C.POINTER(_TypeInfo)],
        "npfem_cell_type_analyze": [C.POINTER(_Mesh), C.POINTER(_Material), C.c_double, C.POINTER(_TypeInfo)],
        "npfem_batch_create": [C.POINTER(vp), C.c_int32, C.POINTER(C.c_int32), C.c_int32, C.c_int,
                               C.POINTER(vp)],
        "npfem_batch_destroy": [vp],
        "npfem_batch_layout": [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
        "npfem_step": [vp, vp, vp, vp, vp, C.POINTER(_Opts), vp, vp, vp],
        "npfem_step_host": [vp, vp, vp, vp, vp, C.POINTER(_Opts), vp, vp, vp],
        "npfem_last_error_string": [C.c_char_p, C.c_size_t],
        "npfem_step_adjoint": [vp, vp, vp, vp, vp, C.POINTER(_Opts), vp, vp, vp, vp, vp, vp, vp, vp],
        "npfem_batch_phase_cycles": [vp, C.POINTER(C.c_uint64), C.c_int32],
        "npfem_batch_set_kernel_timing": [vp, C.c_int32],
        "npfem_batch_set_groups": [vp, C.c_int32, C.c_int32],
        "npfem_batch_kernel_spans": [vp, C.c_int32, C.POINTER(C.c_double)],
        "npfem_batch_get_groups": [vp, C.c_int32, C.POINTER(C.c_int32)],
        "npfem_batch_set_iter_width": [vp, C.c_int32, C.c_int32],
        "npfem_batch_set_phase_counting": [vp, C.c_int32],
        "npfem_batch_set_solve_streams": [vp, C.c_int32],
        "npfem_batch_get_iter_width": [vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
        "npfem_batch_kernel_times": [vp, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int32)],
        "npfem_batch_set_mode": [vp, C.c_int32],
        "npfem_batch_set_split_launch": [vp, C.c_int32, C.POINTER(C.c_int32)],
        "npfem_batch_get_split_launch": [vp, C.c_int32, C.POINTER(C.c_int32)],
        "npfem_batch_set_launch": [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32],
        "npfem_batch_get_launch": [vp, C.c_int32, C.POINTER(C.c_int32)],
        "npfem_step_noalloc": [vp, C.c_int, C.c_int32, vp, vp, vp, vp, C.POINTER(_Opts), vp, vp, vp],
        "npfem_batch_set_collisions": [vp, C.POINTER(_CollisionParams)],
        "npfem_batch_contacts": [vp, vp, vp, vp, vp],
        "npfem_batch_contact_time": [vp, C.POINTER(C.c_double)],
        "npfem_rollout_adjoint": [vp, vp, vp, vp, vp, C.POINTER(_Opts), C.c_int32, C.c_int32, vp, vp, vp, vp, vp,
                                  vp, vp, vp],
        "npfem_step_adjoint_implicit": [vp, vp, vp, vp, vp, C.POINTER(_Opts), vp, vp, vp, vp, vp, vp, C.c_double,
                                        C.c_int32, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        buf = C.create_string_buffer(512)
        _lib.npfem_last_error_string(buf, 512)
        raise NpfemError(rc, buf.value.decode())


def _ptr(t) -> Optional[int]:
    """Device/host pointer of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous()
    return t.data_ptr()


def _state_dtype(precision: int):
    import torch
    return torch.float64 if precision == FP64 else torch.float32


def _check_dev(name: str, t, dtype, shape, optional: bool = False, at_least: bool = False):
    """Raise ValueError unless t is a contiguous CUDA tensor of this dtype and shape (the
    library reads and writes it through a raw pointer: a wrong size or type would make
    the kernels access memory outside it).  at_least: the leading dimension may be
    larger (per-cell outputs, of which the library writes the first ncells rows)."""
    if t is None:
        if optional:
            return
        raise ValueError(f"{name}: required")
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name}: dtype {t.dtype}, expected {dtype}")
    shp, want = tuple(t.shape), tuple(shape)
    ok = shp == want or (at_least and len(shp) == len(want) and shp[0] >= want[0] and shp[1:] == want[1:])
    if not ok:
        raise ValueError(f"{name}: shape {shp}, expected {'at least ' if at_least else ''}{want}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: not contiguous")


def _check_host(name: str, a, dtype, shape, optional: bool = False):
    """The host-buffer counterpart of _check_dev for numpy arrays."""
    if a is None:
        if optional:
            return
        raise ValueError(f"{name}: required")
    if not isinstance(a, np.ndarray):
        raise ValueError(f"{name}: expected a numpy array")
    if a.dtype != np.dtype(dtype):
        raise ValueError(f"{name}: dtype {a.dtype}, expected {np.dtype(dtype)}")
    if tuple(a.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(a.shape)}, expected {tuple(shape)}")
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError(f"{name}: not C-contiguous")


def _check_step_args(ncells: int, n_total: int, precision: int, x, v, f, iters, residual, status, iters_done,
                     alpha_log):
    import torch
    sd = _state_dtype(precision)
    for name, t in (("x", x), ("v", v), ("f", f)):
        _check_dev(name, t, sd, (3, n_total))
    _check_dev("iters", iters, torch.int32, (ncells,), optional=True, at_least=True)
    _check_dev("residual", residual, torch.float64, (ncells,), optional=True, at_least=True)
    _check_dev("status", status, torch.int32, (ncells,), optional=True, at_least=True)
    _check_dev("iters_done", iters_done, torch.int32, (ncells,), optional=True, at_least=True)
    if alpha_log is not None:
        if alpha_log.dim() != 2:
            raise ValueError("alpha_log: expected [ncells, length]")
        _check_dev("alpha_log", alpha_log, torch.float64, (ncells, alpha_log.shape[1]), at_least=True)


def analyze_cell_type(verts: np.ndarray, tris: np.ndarray, material: Sequence[float], dt: float) -> dict:
    """npfem_cell_type_analyze: host-only validation + factorisation statistics (no GPU)."""
    lib = load_library()
    xyz = np.ascontiguousarray(verts, dtype=np.float64)
    tr = np.ascontiguousarray(tris, dtype=np.int32)
    m = _Mesh(xyz.shape[0], tr.shape[0], xyz.ctypes.data_as(C.POINTER(C.c_double)),
              tr.ctypes.data_as(C.POINTER(C.c_int32)))
    vals = [float(a) for a in material]
    mat = _Material(*(vals + [0.0] * (9 - len(vals))))
    inf = _TypeInfo()
    _check(lib.npfem_cell_type_analyze(C.byref(m), C.byref(mat), float(dt), C.byref(inf)))
    return {k: getattr(inf, k) for k, _ in _TypeInfo._fields_}


class CellType:
    """A prefactored cell type: npfem_create_cell_type(mesh, material, dt); material is
    (w_strain, w_bend, w_area, w_vol, density[, c_alpha, c_beta[, s_min, s_max]])
    (damping 0 and no strain limits if absent)."""

    def __init__(self, verts: np.ndarray, tris: np.ndarray, material: Sequence[float], dt: float):
        lib = load_library()
        self._xyz = np.ascontiguousarray(verts, dtype=np.float64)
        self._tris = np.ascontiguousarray(tris, dtype=np.int32)
        m = _Mesh(self._xyz.shape[0], self._tris.shape[0],
                  self._xyz.ctypes.data_as(C.POINTER(C.c_double)),
                  self._tris.ctypes.data_as(C.POINTER(C.c_int32)))
        vals = [float(a) for a in material]
        mat = _Material(*(vals + [0.0] * (9 - len(vals))))
        h = C.c_void_p()
        _check(lib.npfem_create_cell_type(C.byref(m), C.byref(mat), float(dt), C.byref(h)))
        self.handle = h
        self.dt = float(dt)

    def info(self) -> dict:
        inf = _TypeInfo()
        _check(_lib.npfem_cell_type_info(self.handle, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in _TypeInfo._fields_}

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.npfem_destroy_cell_type(self.handle)
            self.handle = None


def step_noalloc(cell_type: "CellType", precision: int, ncells: int, x, v, f, iters=None,
                 iters_default: int = 5, residual=None, status=None, alpha_log=None, stream=None,
                 tol: float = 0.0, iters_done=None):
    """npfem_step_noalloc: step `ncells` back-to-back cells of one type without any
    device allocation (static library workspace); device tensors as for Batch.step,
    x, v, f of shape [3, ncells * n] (back-to-back cells of the type)."""
    if int(ncells) >= 0:
        n = int(cell_type.info()["n_verts"])
        _check_step_args(int(ncells), int(ncells) * n, precision, x, v, f, iters, residual, status, iters_done,
                         alpha_log)
    opts = _Opts(int(iters_default), 0 if alpha_log is None else int(alpha_log.shape[-1]), _ptr(alpha_log),
                 0, float(tol), _ptr(iters_done))
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    _check(_lib.npfem_step_noalloc(cell_type.handle, int(precision), int(ncells), _ptr(x), _ptr(v), _ptr(f),
                                   _ptr(iters), C.byref(opts), _ptr(residual), _ptr(status),
                                   C.c_void_p(stream)))


class Batch:
    """npfem_batch_create(types, type_of_cell, precision)."""

    def __init__(self, types: Sequence[CellType], type_of_cell, precision: int = FP64):
        lib = load_library()
        self.types = list(types)
        arr = (C.c_void_p * len(self.types))(*[t.handle.value for t in self.types])
        toc = np.ascontiguousarray(type_of_cell, dtype=np.int32)
        h = C.c_void_p()
        _check(lib.npfem_batch_create(arr, len(self.types), toc.ctypes.data_as(C.POINTER(C.c_int32)),
                                      int(toc.shape[0]), int(precision), C.byref(h)))
        self.handle = h
        self.ncells = int(toc.shape[0])
        self.type_of_cell = toc
        self.precision = precision
        nt = C.c_int64()
        offs = np.zeros(self.ncells + 1, dtype=np.int64)
        _check(lib.npfem_batch_layout(h, C.byref(nt), offs.ctypes.data_as(C.POINTER(C.c_int64))))
        self.n_total = int(nt.value)
        self.offsets = offs
        self.collisions_on = False

    def step(self, x, v, f, iters=None, iters_default: int = 5, residual=None, status=None,
             alpha_log=None, stream=None, max_iters: int = 0, tol: float = 0.0, iters_done=None):
        """npfem_step on device tensors (torch); asynchronous on `stream` (torch stream or int).
        With an iters tensor, pass max_iters (>= every count) to use the split kernels.
        tol > 0: converged-residual mode (iteration counts become budgets); iters_done: an
        int32 device tensor [ncells] that receives the iterations each cell ran."""
        _check_step_args(self.ncells, self.n_total, self.precision, x, v, f, iters, residual, status, iters_done,
                         alpha_log)
        if iters is not None and max_iters == 0:
            max_iters = self._iter_bound(iters)
        opts = _Opts(int(iters_default), 0 if alpha_log is None else int(alpha_log.shape[-1]),
                     _ptr(alpha_log), int(max_iters), float(tol), _ptr(iters_done))
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        elif not isinstance(stream, int):
            stream = stream.cuda_stream
        _check(_lib.npfem_step(self.handle, _ptr(x), _ptr(v), _ptr(f), _ptr(iters), C.byref(opts),
                               _ptr(residual), _ptr(status), C.c_void_p(stream)))

    def step_adjoint(self, x, v, f, gx_next, gv_next, gx, gv, gf, gw, iters=None, iters_default: int = 5,
                     status=None, stream=None, tol: float = 0.0):
        """npfem_step_adjoint on device tensors (FP64 batches): reverse mode of one step
        (fixed iteration counts: the library rejects tol != 0)."""
        self._check_adjoint_args(x, v, f, gx_next, gv_next, gx, gv, gf, gw, iters, status)
        opts = _Opts(int(iters_default), 0, None, 0, float(tol), None)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        elif not isinstance(stream, int):
            stream = stream.cuda_stream
        _check(_lib.npfem_step_adjoint(self.handle, _ptr(x), _ptr(v), _ptr(f), _ptr(iters), C.byref(opts),
                                       _ptr(gx_next), _ptr(gv_next), _ptr(gx), _ptr(gv), _ptr(gf), _ptr(gw),
                                       _ptr(status), C.c_void_p(stream)))

    def rollout_adjoint(self, x0, v0, f, gx_end, gv_end, gx0, gv0, gf, gweights, nsteps: int, ckpt_every: int,
                        iters=None, iters_default: int = 5, status=None, stream=None):
        """npfem_rollout_adjoint on device tensors (FP64 batches): reverse mode of an
        nsteps rollout from (x0, v0) with constant forces f, checkpointed every ckpt_every
        steps inside the library; gweights [ntypes, 4] receives the per-type weight
        gradients."""
        import torch
        shp = (3, self.n_total)
        for name, t in (("x0", x0), ("v0", v0), ("f", f), ("gx_end", gx_end), ("gx0", gx0), ("gv0", gv0), ("gf", gf)):
            _check_dev(name, t, torch.float64, shp)
        _check_dev("gv_end", gv_end, torch.float64, shp, optional=True)
        _check_dev("gweights", gweights, torch.float64, (len(self.types), 4))
        _check_dev("iters", iters, torch.int32, (self.ncells,), optional=True, at_least=True)
        _check_dev("status", status, torch.int32, (self.ncells,), optional=True, at_least=True)
        max_iters = self._iter_bound(iters) if iters is not None else 0
        opts = _Opts(int(iters_default), 0, None, int(max_iters), 0.0, None)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        elif not isinstance(stream, int):
            stream = stream.cuda_stream
        _check(_lib.npfem_rollout_adjoint(self.handle, _ptr(x0), _ptr(v0), _ptr(f), _ptr(iters), C.byref(opts),
                                          int(nsteps), int(ckpt_every), _ptr(gx_end), _ptr(gv_end), _ptr(gx0),
                                          _ptr(gv0), _ptr(gf), _ptr(gweights), _ptr(status), C.c_void_p(stream)))

    def step_adjoint_implicit(self, x, v, f, gx_next, gv_next, gx, gv, gf, gw, iters=None, iters_default: int = 5,
                              tol: float = 0.0, max_iters: int = 0, cg_tol: float = 1e-12, cg_max_iters: int = 200,
                              status=None, stream=None):
        """npfem_step_adjoint_implicit on device tensors (FP64 batches): gradients through
        the converged step (forward step with iters/tol as in step, then CG on the Hessian)."""
        self._check_adjoint_args(x, v, f, gx_next, gv_next, gx, gv, gf, gw, iters, status)
        if iters is not None and max_iters == 0:
            max_iters = self._iter_bound(iters)
        opts = _Opts(int(iters_default), 0, None, int(max_iters), float(tol), None)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        elif not isinstance(stream, int):
            stream = stream.cuda_stream
        _check(_lib.npfem_step_adjoint_implicit(self.handle, _ptr(x), _ptr(v), _ptr(f), _ptr(iters), C.byref(opts),
                                                _ptr(gx_next), _ptr(gv_next), _ptr(gx), _ptr(gv), _ptr(gf),
                                                _ptr(gw), float(cg_tol), int(cg_max_iters), _ptr(status),
                                                C.c_void_p(stream)))

    def _check_adjoint_args(self, x, v, f, gx_next, gv_next, gx, gv, gf, gw, iters, status):
        import torch
        shp = (3, self.n_total)
        for name, t in (("x", x), ("v", v), ("f", f), ("gx", gx), ("gv", gv), ("gf", gf)):
            _check_dev(name, t, torch.float64, shp)
        _check_dev("gx_next", gx_next, torch.float64, shp, optional=True)
        _check_dev("gv_next", gv_next, torch.float64, shp, optional=True)
        _check_dev("gw", gw, torch.float64, (self.ncells, 4), at_least=True)
        _check_dev("iters", iters, torch.int32, (self.ncells,), optional=True, at_least=True)
        _check_dev("status", status, torch.int32, (self.ncells,), optional=True, at_least=True)

    def set_launch(self, type_index: int, warps_per_block: int, blocks_per_sm: int, solve_in_shared: bool,
                   solve_per_coord: bool = False):
        """npfem_batch_set_launch: launch shape of one cell type (reallocates its workspace)."""
        _check(_lib.npfem_batch_set_launch(self.handle, int(type_index), int(warps_per_block),
                                           int(blocks_per_sm), int(bool(solve_in_shared)), int(bool(solve_per_coord))))

    def get_launch(self, type_index: int) -> dict:
        out = (C.c_int32 * 5)()
        _check(_lib.npfem_batch_get_launch(self.handle, int(type_index), out))
        return {"warps_per_block": out[0], "blocks_per_sm": out[1], "solve_in_shared": bool(out[2]),
                "solve_per_coord": bool(out[3]), "grid": out[4]}

    PHASES = ("predict", "objective", "two_loop", "solve", "history", "write", "area_volume", "gather")

    def set_solve_streams(self, enable: bool = True) -> None:
        """npfem_batch_set_solve_streams: solves of every chain on high-priority streams."""
        _check(_lib.npfem_batch_set_solve_streams(self.handle, int(enable)))

    def set_phase_counting(self, enable: bool = True) -> None:
        """npfem_batch_set_phase_counting: per-phase cycle counters on (off by default)."""
        _check(_lib.npfem_batch_set_phase_counting(self.handle, int(enable)))

    def phase_cycles(self, reset: bool = False) -> dict:
        """npfem_batch_phase_cycles: SM cycles per phase summed over warps (synchronises)."""
        out = (C.c_uint64 * 8)()
        _check(_lib.npfem_batch_phase_cycles(self.handle, out, int(reset)))
        return {k: int(out[i]) for i, k in enumerate(self.PHASES)}

    KERNELS = ("k_begin", "k_solve", "k_iter")

    def kernel_spans(self, type_index: int = -1) -> dict:
        """npfem_batch_kernel_spans: {kernel: ms during which at least one such launch ran}."""
        ms = (C.c_double * 3)()
        _check(_lib.npfem_batch_kernel_spans(self.handle, int(type_index), ms))
        return {k: float(ms[i]) for i, k in enumerate(self.KERNELS)}

    def set_groups(self, type_index: int, groups: int) -> None:
        """npfem_batch_set_groups: split mode, cells of the type in `groups` phase-offset chains."""
        _check(_lib.npfem_batch_set_groups(self.handle, int(type_index), int(groups)))

    def get_groups(self, type_index: int) -> int:
        out = C.c_int32()
        _check(_lib.npfem_batch_get_groups(self.handle, int(type_index), C.byref(out)))
        return int(out.value)

    def set_iter_width(self, type_index: int, warps: int) -> None:
        """npfem_batch_set_iter_width: warps per cell of the CTA iteration kernels (0: one warp
        per cell with the per-vertex gather)."""
        _check(_lib.npfem_batch_set_iter_width(self.handle, int(type_index), int(warps)))

    def get_iter_width(self, type_index: int) -> Tuple[int, int]:
        """npfem_batch_get_iter_width: (warps per cell, resident CTAs per SM)."""
        w, b = C.c_int32(), C.c_int32()
        _check(_lib.npfem_batch_get_iter_width(self.handle, int(type_index), C.byref(w), C.byref(b)))
        return int(w.value), int(b.value)

    def set_kernel_timing(self, enable: bool = True) -> None:
        """npfem_batch_set_kernel_timing: CUDA events around every split-mode launch."""
        _check(_lib.npfem_batch_set_kernel_timing(self.handle, int(enable)))

    def kernel_times(self, type_index: int) -> dict:
        """npfem_batch_kernel_times: {kernel: (summed ms, launches)} of the last timed step."""
        ms, n = (C.c_double * 3)(), (C.c_int32 * 3)()
        _check(_lib.npfem_batch_kernel_times(self.handle, int(type_index), ms, n))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.KERNELS)}

    def _iter_bound(self, iters) -> int:
        """Cached maximum of an iteration-count tensor (read once per tensor)."""
        key = (iters.data_ptr(), int(iters.numel()))
        if getattr(self, "_bound_key", None) != key:
            self._bound_key, self._bound = key, int(iters.max().item()) if iters.numel() else 0
        return self._bound

    def set_mode(self, split: bool):
        """npfem_batch_set_mode: split kernels (True, default) or one fused kernel (False)."""
        _check(_lib.npfem_batch_set_mode(self.handle, 1 if split else 0))

    def set_split_launch(self, type_index: int, shape):
        """npfem_batch_set_split_launch: (iter warps/CTA, iter CTAs/SM, solve warps/CTA,
        solve CTAs/SM, solve-vector placement (0 workspace, 1 shared memory per warp,
        2 shared memory per CTA whose 2 or 4 warps sweep one cell together),
        per-coordinate solve, cells per solve warp); a 6-tuple keeps one cell per warp."""
        shape = list(shape) + [1] * (7 - len(shape))
        arr = (C.c_int32 * 7)(*[int(s) for s in shape])
        _check(_lib.npfem_batch_set_split_launch(self.handle, int(type_index), arr))

    def get_split_launch(self, type_index: int):
        out = (C.c_int32 * 8)()
        _check(_lib.npfem_batch_get_split_launch(self.handle, int(type_index), out))
        return tuple(int(v) for v in out[:7]), bool(out[7])

    def set_collisions(self, radius: Optional[float] = None, delta: float = 0.0, weight: float = 0.0,
                       box=None) -> None:
        """npfem_batch_set_collisions: contacts (search radius, thickness delta, weight w)
        detected at the start of every later step, and with box = (lo[3], hi[3]) the box's
        walls acting on every vertex; radius=None disables them."""
        if radius is None:
            _check(_lib.npfem_batch_set_collisions(self.handle, None))
            self.collisions_on = False
        else:
            p = _CollisionParams(float(radius), float(delta), float(weight))
            if box is not None:
                p.walls = 1
                for d in range(3):
                    p.box_lo[d] = float(box[0][d])
                    p.box_hi[d] = float(box[1][d])
            _check(_lib.npfem_batch_set_collisions(self.handle, C.byref(p)))
            self.collisions_on = True

    def contacts(self, count=None, vertex=None, plane=None, stream=None) -> None:
        """npfem_batch_contacts: the last step's contacts into device tensors
        (int32 [N], int32 [N, 2], float64 [N, 2, 4]; each may be None)."""
        import torch
        _check_dev("count", count, torch.int32, (self.n_total,), optional=True)
        _check_dev("vertex", vertex, torch.int32, (self.n_total, 2), optional=True)
        _check_dev("plane", plane, torch.float64, (self.n_total, 2, 4), optional=True)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        elif not isinstance(stream, int):
            stream = stream.cuda_stream
        _check(_lib.npfem_batch_contacts(self.handle, _ptr(count), _ptr(vertex), _ptr(plane), C.c_void_p(stream)))

    def contact_time(self) -> float:
        """npfem_batch_contact_time: ms of the last timed step's contact detection."""
        ms = C.c_double()
        _check(_lib.npfem_batch_contact_time(self.handle, C.byref(ms)))
        return float(ms.value)

    def step_host(self, x: np.ndarray, v: np.ndarray, f: np.ndarray, iters=None, iters_default: int = 5,
                  residual=None, status=None, stream: int = 0, tol: float = 0.0, iters_done=None):
        """npfem_step_host on host arrays (copies in, steps, copies out; synchronous);
        iters_done: a host int32 array [ncells] or None."""
        sd = np.float64 if self.precision == FP64 else np.float32
        for name, a in (("x", x), ("v", v), ("f", f)):
            _check_host(name, a, sd, (3, self.n_total))
        _check_host("iters", iters, np.int32, (self.ncells,), optional=True)
        _check_host("residual", residual, np.float64, (self.ncells,), optional=True)
        _check_host("status", status, np.int32, (self.ncells,), optional=True)
        _check_host("iters_done", iters_done, np.int32, (self.ncells,), optional=True)
        opts = _Opts(int(iters_default), 0, None, int(np.max(iters)) if iters is not None and len(iters) else 0,
                     float(tol), _ptr(iters_done))
        _check(_lib.npfem_step_host(self.handle, _ptr(x), _ptr(v), _ptr(f), _ptr(iters), C.byref(opts),
                                    _ptr(residual), _ptr(status), C.c_void_p(stream)))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.npfem_batch_destroy(self.handle)
            self.handle = None
