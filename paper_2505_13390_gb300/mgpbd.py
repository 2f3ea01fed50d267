"""Thin Python binding of the C ABI in include/mgpbd.h (argument marshalling only).

Every step of the solve runs in the CUDA library (libmgpbd.so).  PyTorch is
used for device memory and for the current CUDA stream.  There is no CPU
fallback: importing this module raises if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmgpbd.so")

OK, W_NOT_CONVERGED = 0, 1
E_INVALID, E_OOM, E_BREAKDOWN, E_SINGULAR = -1, -2, -3, -4
E_DEVICE_TIMEOUT, E_CUDA, E_BUDGET, E_SETUP = -5, -6, -7, -8
MEM_HOST, MEM_DEVICE = 0, 1
FP64, MIXED = 0, 1


class MeshDesc(C.Structure):
    _fields_ = [("n_verts", C.c_int), ("rest_pos", C.c_void_p), ("inv_mass", C.c_void_p),
                ("n_dist", C.c_int), ("dist", C.c_void_p), ("n_tet", C.c_int),
                ("tet", C.c_void_p), ("alpha", C.c_void_p), ("tet_kind", C.c_int)]


class Params(C.Structure):
    _fields_ = [
        ("dt", C.c_double), ("gravity", C.c_double * 3), ("omega_x", C.c_double),
        ("max_iter", C.c_int), ("eps_b", C.c_double), ("pcg_rtol", C.c_double),
        ("pcg_maxiter", C.c_int), ("setup_interval", C.c_int), ("nk_sweeps", C.c_int),
        ("nk_omega", C.c_double), ("theta_s", C.c_double), ("smoother", C.c_int),
        ("smooth_sweeps", C.c_int), ("lambda_min_est", C.c_double), ("power_iters", C.c_int),
        ("power_safety", C.c_double), ("coarse_max", C.c_int), ("max_levels", C.c_int),
        ("precision", C.c_int), ("backtrack", C.c_int), ("autotune", C.c_int),
        ("level0_op", C.c_int), ("use_graphs", C.c_int), ("linear_solver", C.c_int),
        ("nk_vectors", C.c_int), ("ap_split", C.c_int), ("seed_nk", C.c_uint64), ("seed_agg", C.c_uint64), ("seed_col", C.c_uint64),
        ("seed_pow", C.c_uint64),
    ]


class SolveInfo(C.Structure):
    _fields_ = [("pcg_iters", C.c_int), ("status", C.c_int), ("bnorm", C.c_double),
                ("rel_res", C.c_double), ("true_rel_res", C.c_double), ("omega", C.c_double),
                ("bnorm_after", C.c_double), ("replacements", C.c_int)]

    def as_dict(self) -> Dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [("levels", C.c_int), ("n_setups", C.c_int), ("global_iters", C.c_int64),
                ("op_complexity", C.c_double), ("device_bytes", C.c_size_t),
                ("ms_setup", C.c_double), ("ms_galerkin", C.c_double), ("ms_solve", C.c_double),
                ("ms_other", C.c_double), ("peak_device_bytes", C.c_size_t)]

    def as_dict(self) -> Dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class LevelInfo(C.Structure):
    _fields_ = [("n", C.c_int), ("nnz", C.c_int64), ("n_agg", C.c_int), ("n_colors", C.c_int),
                ("lmax", C.c_double), ("omega", C.c_double), ("lanes_fp32", C.c_int),
                ("lanes_fp64", C.c_int)]

    def as_dict(self) -> Dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchConfig(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("max_active", C.c_int), ("cohort", C.c_int)]


class StepRequest(C.Structure):
    _fields_ = [("id", C.c_int), ("instance", C.c_int), ("frames", C.c_int),
                ("arrival_s", C.c_double)]


class StepResult(C.Structure):
    _fields_ = [("id", C.c_int), ("instance", C.c_int), ("status", C.c_int),
                ("arrival_s", C.c_double), ("start_s", C.c_double), ("finish_s", C.c_double),
                ("global_iters", C.c_int64), ("pcg_iters", C.c_int64)]

    def as_dict(self) -> Dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


# every symbol the header declares, with (restype, argtypes)
_vp, _i, _i64 = C.c_void_p, C.c_int, C.c_int64
SIGNATURES = {
    "mgpbd_default_params": (_i, [C.POINTER(Params)]),
    "mgpbd_create": (_i, [C.POINTER(MeshDesc), C.POINTER(Params), _vp, C.POINTER(_vp)]),
    "mgpbd_create_in_workspace": (_i, [C.POINTER(MeshDesc), C.POINTER(Params), _vp, C.c_size_t,
                                       _vp, C.POINTER(_vp)]),
    "mgpbd_destroy": (None, [_vp]),
    "mgpbd_set_state": (_i, [_vp, _vp, _vp, _i]),
    "mgpbd_get_state": (_i, [_vp, _vp, _vp, _i]),
    "mgpbd_step": (_i, [_vp, _i]),
    "mgpbd_begin_frame": (_i, [_vp]),
    "mgpbd_iterate": (_i, [_vp, C.POINTER(SolveInfo)]),
    "mgpbd_end_frame": (_i, [_vp]),
    "mgpbd_eval_assemble": (_i, [_vp]),
    "mgpbd_setup": (_i, [_vp]),
    "mgpbd_prepare_solve": (_i, [_vp]),
    "mgpbd_solve": (_i, [_vp, _vp, _vp, C.POINTER(SolveInfo)]),
    "mgpbd_vcycle": (_i, [_vp, _vp, _vp]),
    "mgpbd_stats": (_i, [_vp, C.POINTER(Stats)]),
    "mgpbd_sizes": (_i, [_vp, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i64)]),
    "mgpbd_level_info_get": (_i, [_vp, _i, C.POINTER(LevelInfo)]),
    "mgpbd_set_lanes": (_i, [_vp, _i, _i, _i, _i]),
    "mgpbd_set_coarse_tail": (_i, [_vp, _i]),
    "mgpbd_set_wait_limit": (_i, [_vp, C.c_longlong]),
    "mgpbd_get_lanes": (_i, [_vp, _i, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i),
                             C.POINTER(_i)]),
    "mgpbd_get_matrix": (_i, [_vp, _i, _vp, _vp, _vp, _i]),
    "mgpbd_get_map": (_i, [_vp, _vp, _i]),
    "mgpbd_get_incidence": (_i, [_vp, _vp, _vp, _i]),
    "mgpbd_get_aggregates": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _i]),
    "mgpbd_get_colors": (_i, [_vp, _i, _vp, _i]),
    "mgpbd_get_constraints": (_i, [_vp, _vp, _vp, _vp, _vp, _i]),
    "mgpbd_get_lambda": (_i, [_vp, _vp, _vp, _i]),
    "mgpbd_set_colouring": (_i, [_vp, _i]),
    "mgpbd_profile": (_i, [_vp, _i]),
    "mgpbd_profile_read": (_i, [_vp, C.POINTER(C.c_double), C.POINTER(_i64),
                                C.POINTER(C.c_double)]),
    "mgpbd_apply": (_i, [_vp, _vp, _vp, _i]),
    "mgpbd_profile_read_ap": (_i, [_vp, C.POINTER(C.c_double), C.POINTER(_i64),
                                   C.POINTER(C.c_double)]),
    "mgpbd_launch_count": (C.c_ulonglong, []),
    "mgpbd_true_residual_noalloc": (_i, [_vp, _vp, _vp, _vp]),
    "mgpbd_convert": (_i, [_vp, _vp, _vp, _vp, _i64, _vp]),
    "mgpbd_workspace_size": (_i, [C.POINTER(MeshDesc), C.POINTER(Params), C.POINTER(C.c_size_t)]),
    "mgpbd_batch_create": (_i, [C.POINTER(BatchConfig), C.POINTER(_vp)]),
    "mgpbd_batch_add_instance": (_i, [_vp, C.POINTER(MeshDesc), C.POINTER(Params), _vp, _vp,
                                      C.POINTER(_i)]),
    "mgpbd_batch_admit": (_i, [_vp, _i, _i, C.POINTER(_i)]),
    "mgpbd_batch_tick": (_i, [_vp, C.c_double, _vp, _i, C.POINTER(_i)]),
    "mgpbd_batch_counts": (_i, [_vp, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i),
                                C.POINTER(C.c_double)]),
    "mgpbd_batch_error": (C.c_char_p, [_vp]),
    "mgpbd_batch_cohort_stats": (_i, [_vp, C.POINTER(_i64), C.POINTER(_i64),
                                      C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mgpbd_batch_run": (_i, [_vp, _vp, _i, _vp]),
    "mgpbd_batch_get_state": (_i, [_vp, _i, _vp, _vp]),
    "mgpbd_batch_resident": (_i, [_vp, C.POINTER(_i), C.POINTER(C.c_size_t)]),
    "mgpbd_batch_destroy": (None, [_vp]),
    "mgpbd_last_error": (C.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libmgpbd.so; raises if it is missing (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_2505_13390_gb300.build.build()")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def launch_count() -> int:
    return int(load().mgpbd_launch_count())


def workspace_size(mesh, params: Dict) -> int:
    """Upper estimate of an instance's device bytes (mgpbd_workspace_size)."""
    keep = [np.ascontiguousarray(mesh.rest_pos, np.float64),
            np.ascontiguousarray(mesh.inv_mass, np.float64),
            np.ascontiguousarray(mesh.dist, np.int32).reshape(-1, 2),
            np.ascontiguousarray(mesh.tet, np.int32).reshape(-1, 4),
            np.ascontiguousarray(mesh.alpha, np.float64)]
    md = MeshDesc(mesh.n_verts, _ptr(keep[0]), _ptr(keep[1]), mesh.n_dist, _ptr(keep[2]),
                  mesh.n_tet, _ptr(keep[3]), _ptr(keep[4]), int(getattr(mesh, "tet_kind", 0)))
    p = make_params(params)
    out = C.c_size_t()
    _check(load().mgpbd_workspace_size(C.byref(md), C.byref(p), C.byref(out)), "workspace_size")
    return int(out.value)


def convert(in64=None, out32=None, in32=None, out64=None, stream=None) -> None:
    """The mixed-precision path's FP64 -> FP32 (round to nearest even) and
    exact FP32 -> FP64 conversions on device tensors (mgpbd_convert)."""
    n = (in64 if in64 is not None else in32).numel()
    for a in (in64, out32, in32, out64):
        if a is not None and a.numel() != n:
            raise ValueError("all vectors must have the same length")
    _check(load().mgpbd_convert(_ptr(in64), _ptr(out32), _ptr(in32), _ptr(out64), n,
                                 stream.cuda_stream if stream is not None else None),
           "mgpbd_convert")


class MgpbdError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = load().mgpbd_last_error().decode(errors="replace")
        super().__init__(f"{what}: status {status}: {msg}")
        self.status = status


def _check(status: int, what: str) -> int:
    if status < 0:
        raise MgpbdError(status, what)
    return status


def make_params(d: Dict) -> Params:
    p = Params()
    load().mgpbd_default_params(C.byref(p))
    for k, _ in Params._fields_:
        if k in d:
            if k == "gravity":
                p.gravity = (C.c_double * 3)(*d[k])
            else:
                setattr(p, k, d[k])
    return p


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


class Solver:
    """One MGPBD instance resident on the current CUDA device.

    With `workspace` (a CUDA tensor, e.g. uint8 of workspace_size(mesh, params)
    bytes) every device array of the instance is placed in that tensor, which
    the solver keeps alive until close()."""

    def __init__(self, mesh, params: Dict, stream=None, workspace=None):
        import torch

        L = load()
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.N, self.E, self.T = mesh.n_verts, mesh.n_dist, mesh.n_tet
        self.m = self.E + self.T
        keep = [np.ascontiguousarray(mesh.rest_pos, np.float64),
                np.ascontiguousarray(mesh.inv_mass, np.float64),
                np.ascontiguousarray(mesh.dist, np.int32).reshape(-1, 2),
                np.ascontiguousarray(mesh.tet, np.int32).reshape(-1, 4),
                np.ascontiguousarray(mesh.alpha, np.float64)]
        md = MeshDesc(self.N, _ptr(keep[0]), _ptr(keep[1]), self.E, _ptr(keep[2]), self.T,
                      _ptr(keep[3]), _ptr(keep[4]), int(getattr(mesh, "tet_kind", 0)))
        self.params = dict(params)
        self._p = make_params(params)
        h = C.c_void_p()
        st = C.c_void_p(self.stream.cuda_stream)
        if workspace is None:
            _check(L.mgpbd_create(C.byref(md), C.byref(self._p), st, C.byref(h)), "mgpbd_create")
        else:
            nbytes = workspace.numel() * workspace.element_size()
            _check(L.mgpbd_create_in_workspace(C.byref(md), C.byref(self._p),
                                               C.c_void_p(workspace.data_ptr()), nbytes, st,
                                               C.byref(h)), "mgpbd_create_in_workspace")
        self.workspace = workspace
        self.h = h
        self.set_state(mesh.x0, mesh.v0)

    def close(self):
        if getattr(self, "h", None):
            load().mgpbd_destroy(self.h)
            self.h = None
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- state ----------------------------------------------------------
    def set_state(self, x, v):
        """x, v: numpy arrays (host) or CUDA tensors (device), [N, 3] float64."""
        if hasattr(x, "data_ptr") or hasattr(v, "data_ptr"):
            _check(load().mgpbd_set_state(self.h, _ptr(x), _ptr(v), MEM_DEVICE), "set_state")
        else:
            x = None if x is None else np.ascontiguousarray(x, np.float64)
            v = None if v is None else np.ascontiguousarray(v, np.float64)
            _check(load().mgpbd_set_state(self.h, _ptr(x), _ptr(v), MEM_HOST), "set_state")

    def get_state(self):
        x = np.zeros((self.N, 3))
        v = np.zeros((self.N, 3))
        _check(load().mgpbd_get_state(self.h, _ptr(x), _ptr(v), MEM_HOST), "get_state")
        return x, v

    def get_state_device(self, x, v=None):
        _check(load().mgpbd_get_state(self.h, _ptr(x), _ptr(v), MEM_DEVICE), "get_state")

    # ---- Algorithm 1 ----------------------------------------------------
    def step(self, n_frames: int) -> int:
        return _check(load().mgpbd_step(self.h, n_frames), "step")

    def begin_frame(self):
        _check(load().mgpbd_begin_frame(self.h), "begin_frame")

    def end_frame(self):
        _check(load().mgpbd_end_frame(self.h), "end_frame")

    def iterate(self) -> Dict:
        inf = SolveInfo()
        st = _check(load().mgpbd_iterate(self.h, C.byref(inf)), "iterate")
        d = inf.as_dict()
        d["ret"] = st
        return d

    def eval_assemble(self):
        _check(load().mgpbd_eval_assemble(self.h), "eval_assemble")

    def setup(self):
        _check(load().mgpbd_setup(self.h), "setup")

    def prepare_solve(self):
        _check(load().mgpbd_prepare_solve(self.h), "prepare_solve")

    def solve(self, b):
        """b: CUDA float64 tensor [m]; returns (dlambda tensor, info dict)."""
        torch = self.torch
        x = torch.zeros(self.m, dtype=torch.float64, device=b.device)
        inf = SolveInfo()
        _check(load().mgpbd_solve(self.h, _ptr(b), _ptr(x), C.byref(inf)), "solve")
        return x, inf.as_dict()

    def vcycle(self, r):
        torch = self.torch
        z = torch.zeros(self.m, dtype=torch.float64, device=r.device)
        _check(load().mgpbd_vcycle(self.h, _ptr(r), _ptr(z)), "vcycle")
        return z

    def apply(self, x, form: int = 0):
        """y = A x at level 0: form 0 FP64 CSR, 1 FP64 matrix-free, 2 float-float pairs."""
        torch = self.torch
        y = torch.zeros(self.m, dtype=torch.float64, device=x.device)
        _check(load().mgpbd_apply(self.h, _ptr(x), _ptr(y), int(form)), "apply")
        return y

    # ---- measurement ----------------------------------------------------
    def profile(self, enable: bool, ap: bool = False):
        """Event timing of the level-0 sweeps (enable) and of the recurrence's
        A.p (ap); each recorded pair costs a few microseconds per iteration."""
        mask = (1 if enable else 0) | (2 if ap else 0)
        _check(load().mgpbd_profile(self.h, mask), "profile")

    def profile_read(self) -> Dict:
        ms, n, b = C.c_double(), C.c_int64(), C.c_double()
        _check(load().mgpbd_profile_read(self.h, C.byref(ms), C.byref(n), C.byref(b)),
               "profile_read")
        return {"total_ms": ms.value, "launches": n.value, "bytes_per_launch": b.value}

    def profile_read_ap(self) -> Dict:
        """The same totals for the PCG recurrence's A.p."""
        ms, n, b = C.c_double(), C.c_int64(), C.c_double()
        _check(load().mgpbd_profile_read_ap(self.h, C.byref(ms), C.byref(n), C.byref(b)),
               "profile_read_ap")
        return {"total_ms": ms.value, "launches": n.value, "bytes_per_launch": b.value}

    # ---- inspection -----------------------------------------------------
    def stats(self) -> Dict:
        s = Stats()
        _check(load().mgpbd_stats(self.h, C.byref(s)), "stats")
        return s.as_dict()

    def level_info(self, level: int) -> Dict:
        li = LevelInfo()
        _check(load().mgpbd_level_info_get(self.h, level, C.byref(li)), "level_info")
        return li.as_dict()

    def set_lanes(self, csr32: int = 0, csr64: int = 0, vert32: int = 0, vert64: int = 0):
        """Force the row-kernel shapes (lanes per CSR row, lanes per vertex of
        the matrix-free vertex pass; 0 = autotuned or rule) on every level."""
        _check(load().mgpbd_set_lanes(self.h, csr32, csr64, vert32, vert64), "set_lanes")

    def set_coarse_tail(self, enable: bool):
        """The V-cycle below level 0 as one cooperative kernel (True) or as
        separate launches (False, the default); the same bits either way."""
        _check(load().mgpbd_set_coarse_tail(self.h, 1 if enable else 0), "set_coarse_tail")

    def set_wait_limit(self, polls: int):
        """Polls a block of the cooperative kernel waits at a grid barrier
        before the solve fails with MGPBD_E_DEVICE_TIMEOUT."""
        _check(load().mgpbd_set_wait_limit(self.h, int(polls)), "set_wait_limit")

    def lanes(self, level: int = 0) -> Dict:
        """The row-kernel shapes in effect on a level."""
        v = [C.c_int() for _ in range(4)]
        _check(load().mgpbd_get_lanes(self.h, level, *[C.byref(x) for x in v]), "get_lanes")
        return dict(zip(("csr32", "csr64", "vert32", "vert64"), (x.value for x in v)))

    @property
    def levels(self) -> int:
        return self.stats()["levels"]

    def matrix(self, level: int = 0, device: bool = False):
        """CSR (ptr, col, val) of a level: numpy arrays, or CUDA tensors with
        device=True (no host copy of a multi-GB level 0)."""
        li = self.level_info(level)
        if device:
            torch = self.torch
            ptr = torch.empty(li["n"] + 1, dtype=torch.int64, device="cuda")
            col = torch.empty(li["nnz"], dtype=torch.int32, device="cuda")
            val = torch.empty(li["nnz"], dtype=torch.float64, device="cuda")
            mem = MEM_DEVICE
        else:
            ptr = np.zeros(li["n"] + 1, np.int64)
            col = np.zeros(li["nnz"], np.int32)
            val = np.zeros(li["nnz"], np.float64)
            mem = MEM_HOST
        _check(load().mgpbd_get_matrix(self.h, level, _ptr(ptr), _ptr(col), _ptr(val), mem),
               "get_matrix")
        if device:
            self.torch.cuda.synchronize()
        return ptr, col, val

    def assembly_map(self):
        nnz = C.c_int64()
        load().mgpbd_sizes(self.h, None, None, C.byref(nnz))
        m = np.zeros(nnz.value, np.uint16)
        _check(load().mgpbd_get_map(self.h, _ptr(m), MEM_HOST), "get_map")
        return m

    def incidence(self):
        vptr = np.zeros(self.N + 1, np.int64)
        vrow = np.zeros(2 * self.E + 4 * self.T, np.int32)
        _check(load().mgpbd_get_incidence(self.h, _ptr(vptr), _ptr(vrow), MEM_HOST), "incidence")
        return vptr, vrow

    def level_agg(self, level: int):
        """(n_agg, agg, root, P, B); P and B are (n,) for one near-kernel
        vector and (n, k) for k > 1."""
        li = self.level_info(level)
        n = li["n"]
        k = int(self.params.get("nk_vectors", 1))
        agg = np.zeros(n, np.int32)
        root = np.zeros(n, np.uint8)
        P = np.zeros(n * k)
        B = np.zeros(n * k)
        _check(load().mgpbd_get_aggregates(self.h, level, _ptr(agg), _ptr(root), _ptr(P), _ptr(B),
                                           MEM_HOST), "get_aggregates")
        if k > 1:
            P, B = P.reshape(n, k), B.reshape(n, k)
        return li["n_agg"], agg, root, P, B

    def set_colouring(self, enable: bool):
        _check(load().mgpbd_set_colouring(self.h, 1 if enable else 0), "set_colouring")

    def level_color(self, level: int):
        li = self.level_info(level)
        c = np.zeros(li["n"], np.int32)
        _check(load().mgpbd_get_colors(self.h, level, _ptr(c), MEM_HOST), "get_colors")
        return li["n_colors"], c

    def level_omega(self, level: int):
        li = self.level_info(level)
        return li["lmax"], li["omega"]

    def constraints(self):
        Cv = np.zeros(self.m)
        b = np.zeros(self.m)
        gd = np.zeros((self.E, 3))
        gt = np.zeros((self.T, 4, 3))
        _check(load().mgpbd_get_constraints(self.h, _ptr(Cv), _ptr(b), _ptr(gd), _ptr(gt),
                                            MEM_HOST), "get_constraints")
        return Cv, b, gd, gt

    def lam(self):
        lam = np.zeros(self.m)
        dl = np.zeros(self.m)
        _check(load().mgpbd_get_lambda(self.h, _ptr(lam), _ptr(dl), MEM_HOST), "get_lambda")
        return lam, dl


class Batch:
    """Continuous-batching service of many instances (mgpbd_batch_*)."""

    def __init__(self, hbm_budget: int, max_active: int, cohort: bool = False):
        self.cfg = BatchConfig(int(hbm_budget), int(max_active), 1 if cohort else 0)
        h = C.c_void_p()
        _check(load().mgpbd_batch_create(C.byref(self.cfg), C.byref(h)), "batch_create")
        self.h = h
        self.sizes = []

    def add(self, mesh, params: Dict) -> int:
        keep = [np.ascontiguousarray(mesh.rest_pos, np.float64),
                np.ascontiguousarray(mesh.inv_mass, np.float64),
                np.ascontiguousarray(mesh.dist, np.int32).reshape(-1, 2),
                np.ascontiguousarray(mesh.tet, np.int32).reshape(-1, 4),
                np.ascontiguousarray(mesh.alpha, np.float64),
                np.ascontiguousarray(mesh.x0, np.float64),
                np.ascontiguousarray(mesh.v0, np.float64)]
        md = MeshDesc(mesh.n_verts, _ptr(keep[0]), _ptr(keep[1]), mesh.n_dist, _ptr(keep[2]),
                      mesh.n_tet, _ptr(keep[3]), _ptr(keep[4]), int(getattr(mesh, "tet_kind", 0)))
        p = make_params(params)
        i = C.c_int()
        _check(load().mgpbd_batch_add_instance(self.h, C.byref(md), C.byref(p), _ptr(keep[5]),
                                               _ptr(keep[6]), C.byref(i)), "batch_add_instance")
        self.sizes.append(mesh.n_verts)
        return i.value

    def admit(self, instance: int, frames: int = 1) -> int:
        """Submits a request now (mgpbd_batch_admit); returns its ticket."""
        t = C.c_int()
        _check(load().mgpbd_batch_admit(self.h, instance, frames, C.byref(t)), "batch_admit")
        return t.value

    def tick(self, wait_s: float = 0.0, max_results: int = 256):
        """Results of the requests finished since the previous tick."""
        rs = (StepResult * max_results)()
        n = C.c_int()
        _check(load().mgpbd_batch_tick(self.h, float(wait_s), C.cast(rs, C.c_void_p),
                                       max_results, C.byref(n)), "batch_tick")
        return [rs[i].as_dict() for i in range(n.value)]

    def counts(self) -> Dict:
        q, r, u, t = C.c_int(), C.c_int(), C.c_int(), C.c_double()
        _check(load().mgpbd_batch_counts(self.h, C.byref(q), C.byref(r), C.byref(u),
                                         C.byref(t)), "batch_counts")
        return {"queued": q.value, "running": r.value, "unreported": u.value, "clock": t.value}

    def error(self) -> str:
        """Text of the most recently failed request's error."""
        return load().mgpbd_batch_error(self.h).decode(errors="replace")

    def cohort_stats(self) -> Dict:
        """Cohort mode: rounds, batched PCG iterations, seconds in the batched
        chunks and in the rest of the rounds."""
        r, n, c, o = C.c_int64(), C.c_int64(), C.c_double(), C.c_double()
        _check(load().mgpbd_batch_cohort_stats(self.h, C.byref(r), C.byref(n), C.byref(c),
                                               C.byref(o)), "batch_cohort_stats")
        return {"rounds": r.value, "batched_iters": n.value, "chunk_s": c.value,
                "other_s": o.value}

    def run(self, requests):
        """requests: iterable of (id, instance, frames, arrival_s)."""
        reqs = list(requests)
        n = len(reqs)
        rq = (StepRequest * max(n, 1))(*[StepRequest(*r) for r in reqs])
        rs = (StepResult * max(n, 1))()
        st = load().mgpbd_batch_run(self.h, C.cast(rq, C.c_void_p), n, C.cast(rs, C.c_void_p))
        return st, [rs[i].as_dict() for i in range(n)]

    def state(self, instance: int):
        n = self.sizes[instance]
        x = np.zeros((n, 3))
        v = np.zeros((n, 3))
        _check(load().mgpbd_batch_get_state(self.h, instance, _ptr(x), _ptr(v)), "batch_get_state")
        return x, v

    def resident(self):
        n, b = C.c_int(), C.c_size_t()
        _check(load().mgpbd_batch_resident(self.h, C.byref(n), C.byref(b)), "batch_resident")
        return n.value, b.value

    def close(self):
        if getattr(self, "h", None):
            load().mgpbd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
