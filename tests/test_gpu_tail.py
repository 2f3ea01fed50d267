"""The V-cycle below level 0 as one cooperative kernel (the coarse tail,
mgpbd_set_coarse_tail; off by default).

Its steps run the same row bodies as the separate launches, with a grid
barrier between dependent steps, so a V-cycle, a whole PCG solve and whole
global iterations give the same bits with and without it.  Its barrier
waits are bounded: with the limit set to zero every waiting block gives up at
once, the solve returns MGPBD_E_DEVICE_TIMEOUT, and the next solve with the
limit restored is exact again (the device stays usable)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2505_13390_gb300.meshgen import cloth, default_params, hex_block, workload  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


# hierarchies with at least one level between level 0 and the coarsest
CASES = {
    "cloth16": lambda: (cloth(16, plane="xz", alpha=1e-6, pin="corners", noise=1e-3, seed=3),
                        default_params(coarse_max=20, max_levels=4)),      # 705, 48, 11 rows
    "block6": lambda: (hex_block(6, 5, 7, h=0.005, jitter=0.1, alpha=1e-10, pin="y0", seed=1),
                       default_params(omega_x=0.1, coarse_max=40)),         # 2649, 57, 18
    "beam40": lambda: workload("beam40"),                                   # 46760, 1483, 356
    "block20": lambda: workload("block20x33x20"),                           # 150433, ..., 98
}


def make(name, **over):
    from paper_2505_13390_gb300.mgpbd import Solver
    mesh, p = CASES[name]()
    p = dict(p, **over)
    g = Solver(mesh, p, stream=torch.cuda.Stream() if p.get("use_graphs") else None)
    g.begin_frame()
    g.eval_assemble()
    g.prepare_solve()
    return mesh, g


@pytest.mark.parametrize("prec,op", [(0, 0), (1, 1)])
@pytest.mark.parametrize("name", list(CASES))
def test_tail_vcycle_is_bitwise_the_separate_launches(name, prec, op):
    mesh, g = make(name, precision=prec, level0_op=op)
    assert g.levels >= 3, "the tail needs a level between level 0 and the coarsest"
    r = torch.tensor(np.random.default_rng(3).standard_normal(mesh.n_rows), device="cuda")
    g.set_coarse_tail(True)
    z1 = g.vcycle(r).cpu().numpy()
    g.set_coarse_tail(False)
    z0 = g.vcycle(r).cpu().numpy()
    g.close()
    assert np.array_equal(z0, z1)


@pytest.mark.parametrize("graphs", [0, 1])
@pytest.mark.parametrize("name", ["block6", "beam40"])
def test_tail_solve_and_iterations_bitwise(name, graphs):
    """Whole PCG solves (the benchmark's configuration: mixed precision,
    matrix-free level 0) and a whole global iteration, with and without."""
    out = []
    for tail in (True, False):
        mesh, g = make(name, precision=1, level0_op=1, use_graphs=graphs, pcg_maxiter=5000)
        g.set_coarse_tail(tail)
        b = torch.tensor(g.constraints()[1], device="cuda")
        x, info = g.solve(b)
        d = g.iterate()
        out.append((x.cpu().numpy(), info["pcg_iters"], g.get_state()[0], d["pcg_iters"]))
        g.close()
    (x1, n1, s1, k1), (x0, n0, s0, k0) = out
    assert n1 == n0 and k1 == k0
    assert np.array_equal(x1, x0) and np.array_equal(s1, s0)


@pytest.mark.parametrize("graphs", [0, 1])
def test_tail_wait_limit_zero_times_out_and_recovers(graphs):
    from paper_2505_13390_gb300 import mgpbd
    mesh, g = make("block6", precision=1, level0_op=1, use_graphs=graphs, pcg_maxiter=5000)
    g.set_coarse_tail(True)
    b = torch.tensor(g.constraints()[1], device="cuda")
    x_ref, info_ref = g.solve(b)
    g.set_wait_limit(0)
    with pytest.raises(mgpbd.MgpbdError) as e:
        g.solve(b)
    assert e.value.status == mgpbd.E_DEVICE_TIMEOUT
    g.set_wait_limit(1 << 24)
    x, info = g.solve(b)
    assert info["pcg_iters"] == info_ref["pcg_iters"]
    assert np.array_equal(x.cpu().numpy(), x_ref.cpu().numpy())
    g.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["cloth16", "block6"])
def test_tail_vcycle_against_the_oracle(name, prec):
    """The V-cycle through the tail against the oracle's V-cycle: 1e-11 in
    FP64, 1e-4 with the FP32 V-cycle (as for the separate launches)."""
    from oracle.oracle import Oracle
    mesh, p = CASES[name]()
    p = dict(p, precision=prec, level0_op=prec)
    o = Oracle(mesh, p)
    o.begin_frame()
    o.eval_assemble()
    o.prepare_solve()
    _, g = make(name, precision=prec, level0_op=prec)
    g.set_coarse_tail(True)
    assert g.levels == o.levels >= 3
    r = np.random.default_rng(3).standard_normal(mesh.n_rows)
    zo = o.vcycle(r)
    zg = g.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()
    g.close()
    assert np.linalg.norm(zg - zo) <= (1e-11 if prec == 0 else 1e-4) * np.linalg.norm(zo)


@pytest.mark.parametrize("op", [0, 1])
def test_tail_iterations_against_the_oracle(op):
    """Whole global iterations in FP64 with PCG to 1e-10 on the three-level
    cloth: positions within 1e-9 of the oracle, as for the other meshes."""
    from oracle.oracle import Oracle
    from paper_2505_13390_gb300.mgpbd import Solver
    mesh, p = CASES["cloth16"]()
    p = dict(p, pcg_rtol=1e-10, pcg_maxiter=3000, level0_op=op)
    o, g = Oracle(mesh, p), Solver(mesh, p)
    g.set_coarse_tail(True)
    o.begin_frame()
    g.begin_frame()
    scale = np.abs(mesh.rest_pos).max() + 1e-3
    for _ in range(4):
        assert o.iterate()["ret"] == 0 and g.iterate()["ret"] == 0
        assert np.abs(g.get_state()[0] - o.get_state()[0]).max() <= 1e-9 * scale
    assert g.levels >= 3
    g.close()
