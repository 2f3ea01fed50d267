"""Instances placed in a caller-owned device buffer (mgpbd_create_in_workspace).

The library carves every array of such an instance out of the caller's
buffer.  No kernel depends on where its arrays lie, so a run in a workspace
equals the same run in the library's own pool bit for bit, and the instance
takes no device memory beyond the buffer except what the CUDA runtime holds
for its graphs and events.  A buffer of mgpbd_workspace_size bytes holds
these runs; a smaller one ends in MGPBD_E_BUDGET, at create or at the setup
that outgrows it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2505_13390_gb300.meshgen import cloth, default_params, hex_block, workload  # noqa: E402

BUDGET, INVALID = -7, -1


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def case(name, prec):
    if name == "cloth24":
        mesh, p = (cloth(24, plane="xz", alpha=1e-6, pin="corners", seed=31),
                   default_params(omega_x=0.25))
    else:
        mesh, p = (hex_block(12, 4, 4, h=0.01, alpha=1e-7, pin="x0", seed=32),
                   default_params(omega_x=0.1))
    # a setup every second global iteration: re-setups inside each frame
    # release and re-allocate coarse levels
    return mesh, dict(p, precision=prec, max_iter=3, setup_interval=2, pcg_maxiter=5000,
                      autotune=0, use_graphs=1, level0_op=prec)


def ws_tensor(nbytes):
    return torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")


def run(mesh, p, workspace=None, frames=2):
    from paper_2505_13390_gb300.mgpbd import Solver
    g = Solver(mesh, p, stream=torch.cuda.Stream(), workspace=workspace)
    g.step(frames)
    x, v = g.get_state()
    mats = [g.matrix(l) for l in range(g.levels)]
    st = g.stats()
    g.close()
    return x, v, mats, st


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["cloth24", "beam12"])
def test_workspace_run_equals_pooled_run(name, prec):
    from paper_2505_13390_gb300.mgpbd import workspace_size
    mesh, p = case(name, prec)
    x0, v0, m0, s0 = run(mesh, p)
    nbytes = workspace_size(mesh, p)
    x1, v1, m1, s1 = run(mesh, p, workspace=ws_tensor(nbytes))
    assert s1["n_setups"] == s0["n_setups"] == 3  # global iterations 0, 2, 4
    assert np.array_equal(x0, x1) and np.array_equal(v0, v1)
    assert len(m0) == len(m1)
    for a, b in zip(m0, m1):
        for u, w in zip(a, b):
            assert np.array_equal(u, w)
    # the same arrays of the same rounded sizes, wherever they lie
    assert s1["peak_device_bytes"] == s0["peak_device_bytes"] <= nbytes
    assert s1["device_bytes"] == s0["device_bytes"]


def test_workspace_instance_takes_no_pool_memory():
    """Free device memory falls by no more than a small fraction of what the
    instance holds: its arrays are in the caller's tensor."""
    from paper_2505_13390_gb300.mgpbd import Solver, workspace_size
    mesh, p = workload("beam40")
    p = dict(p, precision=1, level0_op=1, use_graphs=1, autotune=0)
    g = Solver(mesh, p, stream=torch.cuda.Stream())  # loads every kernel it needs
    g.begin_frame()
    g.iterate()
    g.close()
    ws = ws_tensor(workspace_size(mesh, p))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    g = Solver(mesh, p, stream=torch.cuda.Stream(), workspace=ws)
    g.begin_frame()
    d = g.iterate()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    held = g.stats()["peak_device_bytes"]
    g.close()
    assert d["ret"] >= 0 and held > 32 << 20
    assert free0 - free1 < held // 4, (free0 - free1, held)


def test_too_small_workspace_is_a_budget_error():
    from paper_2505_13390_gb300.mgpbd import MgpbdError, Solver
    mesh, p = case("beam12", 1)
    with pytest.raises(MgpbdError) as e:
        Solver(mesh, p, workspace=ws_tensor(1 << 16))
    assert e.value.status == BUDGET


def test_setup_that_outgrows_the_workspace_is_a_budget_error():
    """A buffer that holds what create allocates, but not the hierarchy."""
    from paper_2505_13390_gb300.mgpbd import MgpbdError, Solver
    mesh, p = case("beam12", 1)
    g = Solver(mesh, p)
    after_create = g.stats()["peak_device_bytes"]
    g.step(1)
    after_setup = g.stats()["peak_device_bytes"]
    g.close()
    g = Solver(mesh, p, workspace=ws_tensor((after_create + after_setup) // 2))
    with pytest.raises(MgpbdError) as e:
        g.step(1)
    assert e.value.status == BUDGET
    g.close()


def test_bad_workspaces_are_rejected_on_the_host():
    from paper_2505_13390_gb300.mgpbd import MgpbdError, Solver
    mesh, p = case("cloth24", 1)
    ws = ws_tensor(1 << 24)
    for bad in (ws[1:],                                  # not 256-byte aligned
                torch.empty(1 << 24, dtype=torch.uint8)):  # host memory
        with pytest.raises(MgpbdError) as e:
            Solver(mesh, p, workspace=bad)
        assert e.value.status == INVALID
