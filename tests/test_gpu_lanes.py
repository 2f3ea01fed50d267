"""Every row-kernel shape the autotuner can pick, and the autotuner itself,
against the FP64 oracle.

The autotuner (params.autotune) chooses how many lanes share a CSR row (4, 8,
16 or 32) and a vertex of the matrix-free vertex pass (4, 8 or 16).  Each
choice changes the summation tree of those sums, so each is a different
rounding of the same method.  Here every shape is forced through
mgpbd_set_lanes and run for whole global iterations (Alg. 1) beside the
oracle:

* FP64 with PCG to 1e-10 on the moderately conditioned meshes: positions
  within 1e-9 relative, as for the default shapes;
* the stiff tet meshes of the benchmark recipe (a 6x5x7 block, cond(A) ~1e10)
  and the 40x10x10 beam, PCG to the workloads' 1e-6, in FP64 and in mixed
  precision: the error against the oracle within ten times that of the FP64
  path with default shapes, and FP64 true residuals within four times its.

The oracle runs of each case are computed once per module (its OpenMP
build, which gives the same bits as the plain one) and shared by all shapes.
"""
import functools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.oracle import Oracle  # noqa: E402
from paper_2505_13390_gb300.meshgen import cloth, default_params, hex_block, workload  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


CASES = {
    "cloth32": lambda: workload("cloth32"),
    "hex3": lambda: (hex_block(3, 2, 2, h=0.01, jitter=0.1, alpha=1e-7, pin="x0", seed=4),
                     default_params(coarse_max=30, max_levels=4, omega_x=0.1)),
    "hex3s": lambda: (hex_block(3, 2, 2, h=0.01, jitter=0.1, alpha=1e-4, pin="x0", seed=4),
                      default_params(coarse_max=30, max_levels=4, omega_x=0.1)),
    "cloth8": lambda: (cloth(8, plane="xz", alpha=1e-6, pin="corners", noise=1e-3, seed=3),
                       default_params(coarse_max=20, max_levels=4)),
    "block6": lambda: (hex_block(6, 5, 7, h=0.005, jitter=0.1, alpha=1e-10, pin="y0", seed=1),
                       default_params(omega_x=0.1)),
    "beam40": lambda: workload("beam40"),
}


@functools.lru_cache(maxsize=None)
def oracle_run(name, rtol, iters):
    """Positions after each global iteration and the FP64 true relative
    residual of each solve, from the oracle."""
    mesh, p = CASES[name]()
    p = dict(p, pcg_rtol=rtol, pcg_maxiter=5000)
    o = Oracle(mesh, p, omp=True)
    o.begin_frame()
    xs, tres = [], []
    for _ in range(iters):
        d = o.iterate()
        assert d["ret"] == 0
        xs.append(o.get_state()[0].copy())
        tres.append(d["true_rel_res"])
    return xs, tres


def gpu_run(name, rtol, iters, lanes=None, **over):
    from paper_2505_13390_gb300.mgpbd import Solver
    mesh, p = CASES[name]()
    p = dict(p, pcg_rtol=rtol, pcg_maxiter=5000, **over)
    stream = torch.cuda.Stream() if p.get("use_graphs") else None
    g = Solver(mesh, p, stream=stream)
    if lanes:
        g.set_lanes(**lanes)
    g.begin_frame()
    xs, tres = [], []
    for _ in range(iters):
        d = g.iterate()
        assert d["ret"] == 0, d
        xs.append(g.get_state()[0].copy())
        tres.append(d["true_rel_res"])
    shapes = g.lanes(0)
    g.close()
    return xs, tres, shapes


def max_err(xs, ref, scale):
    return max(float(np.abs(a - b).max()) for a, b in zip(xs, ref)) / scale


def scale_of(name):
    mesh, _ = CASES[name]()
    return np.abs(mesh.rest_pos).max() + 1e-3


# ---- FP64, PCG to 1e-10: positions within 1e-9 for every shape --------------
FP64_SHAPES = ([(0, dict(csr64=g)) for g in (4, 8, 16, 32)] +
               [(1, dict(vert64=v, csr64=g)) for v in (4, 8, 16) for g in (4, 32)])


@pytest.mark.parametrize("op,lanes", FP64_SHAPES,
                         ids=[f"op{o}-" + "-".join(f"{k}{v}" for k, v in l.items())
                              for o, l in FP64_SHAPES])
@pytest.mark.parametrize("name,iters", [("cloth8", 4), ("hex3s", 4), ("cloth32", 3),
                                        ("hex3", 3)])
def test_shapes_fp64_iterations(name, iters, op, lanes):
    xo, _ = oracle_run(name, 1e-10, iters)
    xg, _, shapes = gpu_run(name, 1e-10, iters, lanes, precision=0, level0_op=op)
    for k, v in lanes.items():
        assert shapes[k] == v
    assert max_err(xg, xo, scale_of(name)) <= 1e-9


# ---- stiff tet meshes at the workloads' rtol 1e-6 ---------------------------
STIFF = [("block6", 3), ("beam40", 2)]


@functools.lru_cache(maxsize=None)
def fp64_default(name, iters):
    """The FP64 GPU path with the default shapes: its error against the
    oracle and its true residuals set the bar for every other shape."""
    xo, _ = oracle_run(name, 1e-6, iters)
    xg, tres, _ = gpu_run(name, 1e-6, iters, None, precision=0, level0_op=0)
    return max_err(xg, xo, scale_of(name)), tres


MIXED_SHAPES = ([(0, dict(csr32=g, csr64=g)) for g in (4, 8, 16, 32)] +
                [(1, dict(vert32=v, vert64=v, csr32=g)) for v in (4, 8, 16) for g in (4, 32)])
STIFF_SHAPES = [(0, p, l) for p in (0, 1) for (o, l) in MIXED_SHAPES if o == 0] + \
               [(1, p, l) for p in (0, 1) for (o, l) in MIXED_SHAPES if o == 1]


@pytest.mark.parametrize("op,prec,lanes", STIFF_SHAPES,
                         ids=[f"op{o}-p{p}-" + "-".join(f"{k}{v}" for k, v in l.items())
                              for o, p, l in STIFF_SHAPES])
@pytest.mark.parametrize("name,iters", STIFF)
def test_shapes_stiff_vs_oracle(name, iters, op, prec, lanes):
    xo, _ = oracle_run(name, 1e-6, iters)
    e64, t64 = fp64_default(name, iters)
    xg, tres, shapes = gpu_run(name, 1e-6, iters, lanes, precision=prec, level0_op=op)
    for k, v in lanes.items():
        assert shapes[k] == v
    err = max_err(xg, xo, scale_of(name))
    print(f"\n{name} op={op} prec={prec} {lanes}: err {err:.2e} (FP64 default {e64:.2e}); "
          f"true residuals " + " ".join(f"{t:.1e}" for t in tres))
    assert err <= max(10 * e64, 1e-9)
    assert max(tres) <= 4 * max(max(t64), 1e-6)


@pytest.mark.parametrize("name,iters", STIFF)
def test_benchmark_configuration_vs_oracle(name, iters):
    """The configuration the benchmark times: mixed precision, matrix-free
    level 0, CUDA graphs and the autotuner choosing the shapes."""
    xo, _ = oracle_run(name, 1e-6, iters)
    e64, t64 = fp64_default(name, iters)
    xg, tres, shapes = gpu_run(name, 1e-6, iters, None, precision=1, level0_op=1,
                               use_graphs=1, autotune=1)
    err = max_err(xg, xo, scale_of(name))
    print(f"\n{name} autotuned {shapes}: err {err:.2e} (FP64 default {e64:.2e})")
    assert err <= max(10 * e64, 1e-9)
    assert max(tres) <= 4 * max(max(t64), 1e-6)


def test_set_lanes_rejects_other_shapes():
    from paper_2505_13390_gb300 import mgpbd
    mesh, p = CASES["cloth8"]()
    g = mgpbd.Solver(mesh, p)
    for bad in (dict(csr32=2), dict(csr64=64), dict(vert32=32), dict(vert64=3)):
        with pytest.raises(mgpbd.MgpbdError):
            g.set_lanes(**bad)
    g.set_lanes(csr32=8, vert64=16)
    assert g.lanes(0)["csr32"] == 8 and g.lanes(0)["vert64"] == 16
    g.set_lanes()
    assert g.lanes(0)["csr32"] in (4, 8, 16, 32)
    g.close()
