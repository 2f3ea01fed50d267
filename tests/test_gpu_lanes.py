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


# ---- A.p from float-float pairs (params.ap_split) ----------------------------
# The recurrence's product from binary32 (high, low) pairs: ~2^-46 relative
# per product, sums by two-sum, then residual replacement in FP64.


def _magnitude(mesh, p, gd, gt, x):
    """sum over the matrix-free terms of row i of their magnitudes:
    (|J| W |J|^T |x|)_i + alpha~_i |x_i|, the scale of the rounding error of
    any evaluation of (J W J^T + alpha~) x that forms those terms."""
    N, E = mesh.n_verts, mesh.n_dist
    w = np.asarray(mesh.inv_mass, float)
    ax = np.abs(x)
    u = np.zeros((N, 3))
    dist = np.asarray(mesh.dist).reshape(-1, 2)
    tet = np.asarray(mesh.tet).reshape(-1, 4)
    for s in range(2):
        np.add.at(u, dist[:, s], np.abs(gd) * ax[:E, None])
    for s in range(4):
        np.add.at(u, tet[:, s], np.abs(gt[:, s, :]) * ax[E:, None])
    u *= w[:, None]
    M = np.zeros(len(x))
    M[:E] = (np.abs(gd) * (u[dist[:, 0]] + u[dist[:, 1]])).sum(1)
    M[E:] = sum((np.abs(gt[:, s, :]) * u[tet[:, s]]).sum(1) for s in range(4))
    at = np.asarray(mesh.alpha, float) / p["dt"] ** 2
    return M + at * ax


@pytest.mark.parametrize("name", ["cloth8", "hex3", "block6", "beam40"])
def test_pair_product_elementwise(name):
    """mgpbd_apply form 2 against the exact A x (the oracle's FP64 matrix of
    eq. 3, at the same positions), row by row within 2^-40 of the magnitude
    of the row's terms; the FP64 forms within 2^-47."""
    import scipy.sparse as sp

    from paper_2505_13390_gb300.mgpbd import Solver
    mesh, p = CASES[name]()
    p = dict(p, precision=1, level0_op=1, ap_split=1)
    g = Solver(mesh, p)
    g.begin_frame()
    g.eval_assemble()
    o = Oracle(mesh, p)
    o.begin_frame()
    o.eval_assemble()
    ptr, col, val = o.matrix(0)
    _, _, gd, gt = o.constraints()
    m = len(ptr) - 1
    A = sp.csr_matrix((val, col, ptr), shape=(m, m))
    rng = np.random.default_rng(11)
    for trial in range(3):
        # signs mixed, magnitudes spread over six decades
        x = rng.standard_normal(m) * 10.0 ** rng.uniform(-3, 3, m)
        exact = A @ x
        M = _magnitude(mesh, p, gd, gt, x)
        xt = torch.from_numpy(x).cuda()
        for form, bound in ((2, 2.0 ** -40), (1, 2.0 ** -47), (0, 2.0 ** -47)):
            y = g.apply(xt, form).cpu().numpy()
            rel = np.abs(y - exact) / np.maximum(M, 1e-300)
            print(f"\n{name} trial {trial} form {form}: max |err| / magnitude {rel.max():.2e}")
            assert rel.max() <= bound, (form, rel.max())
    g.close()


@pytest.mark.parametrize("name,iters", STIFF)
def test_pair_form_vs_oracle(name, iters):
    """The benchmark configuration with the pair form of A.p: the same bars as
    with the FP64 product (error against the oracle within ten times that of
    the FP64 path, FP64 true residuals within four times its), and the
    residual replacement taking place."""
    xo, _ = oracle_run(name, 1e-6, iters)
    e64, t64 = fp64_default(name, iters)
    from paper_2505_13390_gb300.mgpbd import Solver
    mesh, p = CASES[name]()
    p = dict(p, pcg_rtol=1e-6, pcg_maxiter=5000, precision=1, level0_op=1, use_graphs=1,
             autotune=1, ap_split=1)
    g = Solver(mesh, p, stream=torch.cuda.Stream())
    g.begin_frame()
    xg, tres, reps = [], [], []
    for _ in range(iters):
        d = g.iterate()
        assert d["ret"] == 0, d
        xg.append(g.get_state()[0].copy())
        tres.append(d["true_rel_res"])
        reps.append(d["replacements"])
    g.close()
    err = max_err(xg, xo, scale_of(name))
    print(f"\n{name} pairs: err {err:.2e} (FP64 default {e64:.2e}); replacements {reps}; "
          f"true residuals " + " ".join(f"{t:.1e}" for t in tres))
    assert err <= max(10 * e64, 1e-9)
    assert max(tres) <= 4 * max(max(t64), 1e-6)
    assert min(reps) >= 1


def test_pair_form_graphs_match_plain_launches():
    """Replacement happens between chunks of eight iterations in both launch
    modes, so a CUDA-graph replay and plain launches give the same bits."""
    from paper_2505_13390_gb300.mgpbd import Solver
    mesh, p = CASES["block6"]()
    out = []
    for graphs in (0, 1):
        q = dict(p, precision=1, level0_op=1, ap_split=1, use_graphs=graphs)
        g = Solver(mesh, q, stream=torch.cuda.Stream())
        g.begin_frame()
        ds = [g.iterate() for _ in range(2)]
        out.append((g.get_state()[0].copy(), [d["pcg_iters"] for d in ds],
                    [d["replacements"] for d in ds]))
        g.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1:] == out[1][1:]


def test_pair_form_parameters():
    """ap_split needs mixed precision and the matrix-free level 0; form 2 of
    mgpbd_apply needs ap_split."""
    from paper_2505_13390_gb300 import mgpbd
    mesh, p = CASES["cloth8"]()
    for bad in (dict(ap_split=1, precision=0, level0_op=1),
                dict(ap_split=1, precision=1, level0_op=0), dict(ap_split=2)):
        with pytest.raises(mgpbd.MgpbdError):
            mgpbd.Solver(mesh, dict(p, **bad))
    g = mgpbd.Solver(mesh, dict(p, precision=1, level0_op=1))
    g.begin_frame()
    g.eval_assemble()
    x = torch.ones(g.m, dtype=torch.float64, device="cuda")
    g.apply(x, 1)
    with pytest.raises(mgpbd.MgpbdError):
        g.apply(x, 2)
    g.close()


def test_profile_channels():
    """mgpbd_profile's mask selects the timed kernels: the level-0 sweeps
    (1), the recurrence's A.p (2), both (3); other values are rejected."""
    from paper_2505_13390_gb300 import mgpbd
    mesh, p = CASES["block6"]()
    g = mgpbd.Solver(mesh, dict(p, precision=1, level0_op=1, use_graphs=1),
                     stream=torch.cuda.Stream())
    g.begin_frame()
    g.iterate()
    seen = {}
    for sweeps, ap in ((True, False), (False, True), (True, True)):
        g.profile(sweeps, ap=ap)
        d = g.iterate()
        seen[(sweeps, ap)] = (g.profile_read()["launches"], g.profile_read_ap()["launches"],
                              d["pcg_iters"])
        g.profile(False)
    sw, ap_, it = seen[(True, False)]
    assert sw > 0 and ap_ == 0
    sw, ap_, it = seen[(False, True)]
    assert sw == 0 and ap_ == it  # one product per PCG iteration
    sw, ap_, it = seen[(True, True)]
    assert sw > 0 and ap_ == it
    with pytest.raises(mgpbd.MgpbdError):
        mgpbd._check(mgpbd.load().mgpbd_profile(g.h, 4), "profile")
    g.close()
