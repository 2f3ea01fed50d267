"""ctypes binding of the FP64 CPU oracle (mgpbd_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU
baseline leg of the benchmark use this module.  It never touches the CUDA
library and the CUDA library never touches it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Dict, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mgpbd_oracle.c")
# MGPBD_ORACLE_LIB loads another build of the oracle's source instead (the
# mutation test's copies with a planted mistake); it is never compiled here.
OVERRIDE = os.environ.get("MGPBD_ORACLE_LIB")
LIB = OVERRIDE or os.path.join(HERE, "liborc.so")
# the same source built with -fopenmp: its row-independent loops run on all
# host cores and give the same bits as the plain build
LIB_OMP = os.path.join(HERE, "liborc_omp.so")
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-shared", "-fPIC"]


def _compile(out: str, extra, force: bool) -> None:
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, *extra, SRC, "-o", tmp, "-lm"])
        os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math), plain
    and with OpenMP."""
    if OVERRIDE:
        return LIB
    _compile(LIB, [], force)
    _compile(LIB_OMP, ["-fopenmp"], force)
    return LIB


class Params(C.Structure):
    _fields_ = [
        ("dt", C.c_double), ("gravity", C.c_double * 3), ("omega_x", C.c_double),
        ("max_iter", C.c_int), ("eps_b", C.c_double), ("pcg_rtol", C.c_double),
        ("pcg_maxiter", C.c_int), ("setup_interval", C.c_int), ("nk_sweeps", C.c_int),
        ("nk_omega", C.c_double), ("theta_s", C.c_double), ("smoother", C.c_int),
        ("smooth_sweeps", C.c_int), ("lambda_min_est", C.c_double), ("power_iters", C.c_int),
        ("power_safety", C.c_double), ("coarse_max", C.c_int), ("max_levels", C.c_int),
        ("backtrack", C.c_int), ("linear_solver", C.c_int), ("nk_vectors", C.c_int),
        ("seed_nk", C.c_uint64), ("seed_agg", C.c_uint64), ("seed_col", C.c_uint64),
        ("seed_pow", C.c_uint64),
    ]


class SolveInfo(C.Structure):
    _fields_ = [("pcg_iters", C.c_int), ("status", C.c_int), ("bnorm", C.c_double),
                ("rel_res", C.c_double), ("true_rel_res", C.c_double), ("omega", C.c_double),
                ("bnorm_after", C.c_double)]

    def as_dict(self) -> Dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_libs: Dict[bool, object] = {}


def lib(omp: bool = False):
    """The plain oracle library, or with omp=True its OpenMP build."""
    if omp not in _libs:
        build()
        L = C.CDLL(LIB_OMP if omp and not OVERRIDE else LIB)
        vp = C.c_void_p
        L.orc_create.restype = vp
        L.orc_create.argtypes = [C.c_int, vp, vp, C.c_int, vp, C.c_int, vp, C.c_int, vp,
                                 C.POINTER(Params), C.POINTER(C.c_int)]
        L.orc_destroy.argtypes = [vp]
        for name in ("orc_begin_frame", "orc_end_frame", "orc_eval_assemble"):
            getattr(L, name).argtypes = [vp]
        for name in ("orc_setup", "orc_prepare_solve", "orc_levels", "orc_n_setups"):
            getattr(L, name).argtypes = [vp]
            getattr(L, name).restype = C.c_int
        L.orc_iterate.argtypes = [vp, C.POINTER(SolveInfo)]
        L.orc_iterate.restype = C.c_int
        L.orc_step.argtypes = [vp, C.c_int, vp]
        L.orc_step.restype = C.c_int
        L.orc_solve.argtypes = [vp, vp, vp, C.POINTER(SolveInfo)]
        L.orc_solve.restype = C.c_int
        L.orc_vcycle.argtypes = [vp, vp, vp]
        L.orc_set_state.argtypes = [vp, vp, vp]
        L.orc_get_state.argtypes = [vp, vp, vp]
        L.orc_nnz.argtypes = [vp, C.c_int]
        L.orc_nnz.restype = C.c_int64
        L.orc_rows.argtypes = [vp, C.c_int]
        L.orc_rows.restype = C.c_int
        L.orc_matrix.argtypes = [vp, C.c_int, vp, vp, vp]
        L.orc_map.argtypes = [vp, vp]
        L.orc_incidence.argtypes = [vp, vp, vp]
        L.orc_level_agg.argtypes = [vp, C.c_int, vp, vp, vp, vp]
        L.orc_level_agg.restype = C.c_int
        L.orc_level_color.argtypes = [vp, C.c_int, vp]
        L.orc_level_color.restype = C.c_int
        L.orc_level_omega.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.orc_constraints.argtypes = [vp, vp, vp, vp, vp]
        L.orc_rest.argtypes = [vp, vp, vp]
        L.orc_lambda.argtypes = [vp, vp, vp]
        L.orc_set_lambda.argtypes = [vp, vp]
        L.orc_aggregate_csr.argtypes = [C.c_int, vp, vp, vp, C.c_double, C.c_uint64, C.c_int,
                                        vp, vp, vp]
        L.orc_aggregate_csr.restype = C.c_int
        L.orc_colour_csr.argtypes = [C.c_int, vp, vp, C.c_uint64, C.c_int, vp]
        L.orc_colour_csr.restype = C.c_int
        L.orc_smooth_test.argtypes = [vp, C.c_int, vp, vp]
        L.orc_h64.argtypes = [C.c_uint64]
        L.orc_h64.restype = C.c_uint64
        L.orc_threads.argtypes = [C.c_int]
        L.orc_threads.restype = C.c_int
        assert L.orc_sizeof_params() == C.sizeof(Params)
        assert L.orc_sizeof_info() == C.sizeof(SolveInfo)
        _libs[omp] = L
    return _libs[omp]


def threads(n: int = 0) -> int:
    """Threads of the OpenMP build's row loops (n > 0 sets them)."""
    return int(lib(True).orc_threads(n))


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def make_params(d: Dict) -> Params:
    p = Params()
    p.dt = d["dt"]
    p.gravity = (C.c_double * 3)(*d["gravity"])
    for k in ("omega_x", "eps_b", "pcg_rtol", "nk_omega", "theta_s", "lambda_min_est",
              "power_safety"):
        setattr(p, k, float(d[k]))
    for k in ("max_iter", "pcg_maxiter", "setup_interval", "nk_sweeps", "smoother",
              "smooth_sweeps", "power_iters", "coarse_max", "max_levels", "backtrack",
              "linear_solver", "nk_vectors"):
        setattr(p, k, int(d[k]))
    for k in ("seed_nk", "seed_agg", "seed_col", "seed_pow"):
        setattr(p, k, int(d[k]))
    return p


def aggregate_csr(ptr, col, val, theta: float, seed: int, level: int = 0):
    """Strength filter + MIS-2 aggregation of a caller-given CSR (diagonal last)."""
    ptr = np.ascontiguousarray(ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    n = len(ptr) - 1
    agg = np.zeros(n, np.int32)
    root = np.zeros(n, np.uint8)
    S = np.zeros(len(col), np.uint8)
    na = lib().orc_aggregate_csr(n, _p(ptr), _p(col), _p(val), float(theta), int(seed),
                                 int(level), _p(agg), _p(root), _p(S))
    return na, agg, root, S


def colour_csr(ptr, col, seed: int, level: int = 0):
    ptr = np.ascontiguousarray(ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    n = len(ptr) - 1
    c = np.zeros(n, np.int32)
    nc = lib().orc_colour_csr(n, _p(ptr), _p(col), int(seed), int(level), _p(c))
    return nc, c


def h64(k: int) -> int:
    return int(lib().orc_h64(C.c_uint64(k)))


class Oracle:
    """One oracle instance of a mesh (plain FP64 CPU reference).  omp=True
    runs it in the OpenMP build (same bits, row loops on all host cores)."""

    def __init__(self, mesh, params: Dict, omp: bool = False):
        L = lib(omp)
        self.L = L
        self.mesh = mesh
        self.params = dict(params)
        self.N, self.E, self.T = mesh.n_verts, mesh.n_dist, mesh.n_tet
        self.m = self.E + self.T
        self._keep = [np.ascontiguousarray(mesh.rest_pos, np.float64),
                      np.ascontiguousarray(mesh.inv_mass, np.float64),
                      np.ascontiguousarray(mesh.dist, np.int32).reshape(-1, 2),
                      np.ascontiguousarray(mesh.tet, np.int32).reshape(-1, 4),
                      np.ascontiguousarray(mesh.alpha, np.float64)]
        st = C.c_int(0)
        self._p = make_params(params)
        self.h = L.orc_create(self.N, _p(self._keep[0]), _p(self._keep[1]), self.E,
                              _p(self._keep[2]), self.T, _p(self._keep[3]),
                              int(getattr(mesh, "tet_kind", 0)), _p(self._keep[4]),
                              C.byref(self._p), C.byref(st))
        if not self.h:
            raise RuntimeError(f"oracle create failed: {st.value}")
        self.set_state(mesh.x0, mesh.v0)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.orc_destroy(h)
            self.h = None

    # state ---------------------------------------------------------------
    def set_state(self, x, v):
        x = np.ascontiguousarray(x, np.float64)
        v = np.ascontiguousarray(v, np.float64)
        self.L.orc_set_state(self.h, _p(x), _p(v))

    def get_state(self):
        x = np.zeros((self.N, 3))
        v = np.zeros((self.N, 3))
        self.L.orc_get_state(self.h, _p(x), _p(v))
        return x, v

    # integrator ----------------------------------------------------------
    def begin_frame(self):
        self.L.orc_begin_frame(self.h)

    def end_frame(self):
        self.L.orc_end_frame(self.h)

    def iterate(self) -> Dict:
        inf = SolveInfo()
        st = self.L.orc_iterate(self.h, C.byref(inf))
        d = inf.as_dict()
        d["ret"] = st
        return d

    def step(self, n_frames: int):
        hist = (SolveInfo * (n_frames * self.params["max_iter"]))()
        st = self.L.orc_step(self.h, n_frames, C.cast(hist, C.c_void_p))
        return st, [h.as_dict() for h in hist]

    def eval_assemble(self):
        self.L.orc_eval_assemble(self.h)

    def setup(self) -> int:
        return self.L.orc_setup(self.h)

    def prepare_solve(self) -> int:
        return self.L.orc_prepare_solve(self.h)

    def solve(self, b):
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros(self.m)
        inf = SolveInfo()
        self.L.orc_solve(self.h, _p(b), _p(x), C.byref(inf))
        return x, inf.as_dict()

    def smooth(self, level: int, b):
        """Test-only: one pre-smoothing of `level` from x = 0."""
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros_like(b)
        self.L.orc_smooth_test(self.h, level, _p(b), _p(x))
        return x

    def vcycle(self, r):
        r = np.ascontiguousarray(r, np.float64)
        z = np.zeros(self.m)
        self.L.orc_vcycle(self.h, _p(r), _p(z))
        return z

    # inspection ----------------------------------------------------------
    @property
    def levels(self) -> int:
        return self.L.orc_levels(self.h)

    @property
    def n_setups(self) -> int:
        return self.L.orc_n_setups(self.h)

    def matrix(self, level: int = 0):
        L = lib()
        n = L.orc_rows(self.h, level)
        nnz = L.orc_nnz(self.h, level)
        ptr = np.zeros(n + 1, np.int64)
        col = np.zeros(nnz, np.int32)
        val = np.zeros(nnz, np.float64)
        L.orc_matrix(self.h, level, _p(ptr), _p(col), _p(val))
        return ptr, col, val

    def assembly_map(self):
        nnz = self.L.orc_nnz(self.h, 0)
        m = np.zeros(nnz, np.uint16)
        self.L.orc_map(self.h, _p(m))
        return m

    def incidence(self):
        # counts: each distance row touches 2 vertices, each tet row 4
        tot = 2 * self.E + 4 * self.T
        vptr = np.zeros(self.N + 1, np.int64)
        vrow = np.zeros(tot, np.int32)
        self.L.orc_incidence(self.h, _p(vptr), _p(vrow))
        return vptr, vrow

    def level_agg(self, level: int):
        """(n_agg, agg, root, P, B); P and B are (n,) for one near-kernel
        vector and (n, k) for k > 1."""
        n = self.L.orc_rows(self.h, level)
        k = int(self.params.get("nk_vectors", 1))
        agg = np.zeros(n, np.int32)
        root = np.zeros(n, np.uint8)
        P = np.zeros(n * k)
        B = np.zeros(n * k)
        na = self.L.orc_level_agg(self.h, level, _p(agg), _p(root), _p(P), _p(B))
        if k > 1:
            P, B = P.reshape(n, k), B.reshape(n, k)
        return na, agg, root, P, B

    def level_color(self, level: int):
        n = self.L.orc_rows(self.h, level)
        c = np.zeros(n, np.int32)
        nc = self.L.orc_level_color(self.h, level, _p(c))
        return nc, c

    def level_omega(self, level: int):
        a, b = C.c_double(), C.c_double()
        self.L.orc_level_omega(self.h, level, C.byref(a), C.byref(b))
        return a.value, b.value

    def constraints(self):
        Cv = np.zeros(self.m)
        b = np.zeros(self.m)
        gd = np.zeros((self.E, 3))
        gt = np.zeros((self.T, 4, 3))
        self.L.orc_constraints(self.h, _p(Cv), _p(b), _p(gd), _p(gt))
        return Cv, b, gd, gt

    def rest(self):
        L0 = np.zeros(self.E)
        V0 = np.zeros(self.T)
        self.L.orc_rest(self.h, _p(L0), _p(V0))
        return L0, V0

    def lam(self):
        lam = np.zeros(self.m)
        dl = np.zeros(self.m)
        self.L.orc_lambda(self.h, _p(lam), _p(dl))
        return lam, dl

    def set_lambda(self, lam):
        lam = np.ascontiguousarray(lam, np.float64)
        self.L.orc_set_lambda(self.h, _p(lam))
