"""Continuous-batching service (mgpbd_batch_*) on one GPU.

Each instance runs on its own stream with deterministic kernels, so its
results do not depend on what else is on the GPU: a step served in the mix
equals the same step served alone, bit for bit.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2505_13390_gb300.meshgen import cloth, default_params, hex_block  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def meshes():
    out = []
    for k, n in enumerate((12, 20)):
        out.append((cloth(n, plane="xz", alpha=1e-6, pin="corners", seed=10 + k),
                    default_params(omega_x=0.25)))
    for k, L in enumerate((3, 5)):
        out.append((hex_block(L, 3, 3, h=0.01, alpha=1e-7, pin="x0", seed=20 + k),
                    default_params(omega_x=0.1)))
    return out


def common(p, prec):
    # setup at the start of every frame: a re-admitted instance (fresh handle)
    # then repeats exactly what a resident one does
    return dict(p, precision=prec, max_iter=4, setup_interval=4, pcg_maxiter=5000, autotune=0,
                use_graphs=1, level0_op=prec)


def serve(ms, prec, max_active, budget, requests):
    from paper_2505_13390_gb300.mgpbd import Batch
    b = Batch(budget, max_active)
    ids = [b.add(m, common(p, prec)) for m, p in ms]
    st, res = b.run(requests)
    states = [b.state(i) for i in ids]
    b.close()
    return st, res, states


def trace(n_inst, per_inst, spacing):
    reqs = []
    rid = 0
    for r in range(per_inst):
        for i in range(n_inst):
            reqs.append((rid, i, 1, rid * spacing))
            rid += 1
    return reqs


@pytest.mark.parametrize("prec", [0, 1])
def test_mix_equals_alone_bitwise(prec):
    ms = meshes()
    reqs = trace(len(ms), 2, 0.0)
    st1, res1, alone = serve(ms, prec, 1, 64 << 30, reqs)
    st4, res4, mixed = serve(ms, prec, 4, 64 << 30, reqs)
    assert st1 >= 0 and st4 >= 0
    for (x1, v1), (x4, v4) in zip(alone, mixed):
        assert np.array_equal(x1, x4) and np.array_equal(v1, v4)
    assert [r["pcg_iters"] for r in res1] == [r["pcg_iters"] for r in res4]
    # the served state equals a plain one-instance run of the same frames
    from paper_2505_13390_gb300.mgpbd import Solver
    m, p = ms[0]
    g = Solver(m, common(p, prec))
    for _ in range(2):
        g.begin_frame()
        for _ in range(4):
            g.iterate()
        g.end_frame()
    x, v = g.get_state()
    assert np.array_equal(x, alone[0][0]) and np.array_equal(v, alone[0][1])


def test_budget_evicts_and_restores_state():
    ms = meshes()
    reqs = trace(len(ms), 2, 0.0)
    _, _, roomy = serve(ms, 0, 2, 64 << 30, reqs)
    # about two instances fit: the others wait, and idle ones are evicted.
    # Admission reserves an instance's estimate (mgpbd_workspace_size) while
    # it loads, so the budget is sized from the largest estimate.
    from paper_2505_13390_gb300.mgpbd import workspace_size
    one = max(workspace_size(m, common(p, 0)) for m, p in ms)
    st, res, tight = serve(ms, 0, 2, int(2.5 * one), reqs)
    assert st >= 0 and all(r["status"] >= 0 for r in res)
    for (x1, v1), (x2, v2) in zip(roomy, tight):
        assert np.array_equal(x1, x2) and np.array_equal(v1, v2)


def test_instance_larger_than_budget_is_rejected():
    from paper_2505_13390_gb300 import mgpbd
    m, p = meshes()[-1]
    st, res, _ = serve([(m, p)], 0, 1, 1 << 20, [(0, 0, 1, 0.0)])
    assert st == mgpbd.E_BUDGET and res[0]["status"] == mgpbd.E_BUDGET


def test_late_arrivals_join_while_others_run():
    ms = meshes()
    # a long request on the largest instance, then short ones arriving later
    reqs = [(0, 3, 3, 0.0)] + [(1 + k, k, 1, 0.05 * (k + 1)) for k in range(3)]
    st, res, _ = serve(ms, 1, 4, 64 << 30, reqs)
    assert st >= 0
    r0 = res[0]
    assert any(r["start_s"] < r0["finish_s"] for r in res[1:])  # overlapped on the GPU
    assert all(r["start_s"] >= r["arrival_s"] for r in res)


def test_workspace_size_bounds_the_device_bytes():
    """The admission estimate (mgpbd_workspace_size) is not below what an
    instance really holds after create and its first setup."""
    from paper_2505_13390_gb300.mgpbd import Solver, workspace_size
    for mesh, p in meshes():
        p = common(p, 1)
        est = workspace_size(mesh, p)
        g = Solver(mesh, p)
        g.begin_frame()
        g.iterate()
        held = g.stats()["device_bytes"]
        g.close()
        assert held <= est, (mesh.name, held, est)


@pytest.mark.parametrize("prec", [0, 1])
def test_admit_while_running_mix_equals_alone(prec):
    """The request loop: a long request starts, and while it is on the GPU the
    host thread admits requests for the other instances one by one and
    collects results with tick.  The late requests run while the long one is
    still running, each result is returned once, and every instance ends in
    the state of a one-at-a-time run of the same requests, bit for bit."""
    import time

    from paper_2505_13390_gb300.mgpbd import Batch
    ms = meshes()
    ref = serve(ms, prec, 1, 64 << 30, [(0, 3, 6, 0.0)] + [(1 + k, k, 1, 0.0) for k in range(3)])
    b = Batch(64 << 30, 4)
    ids = [b.add(m, common(p, prec)) for m, p in ms]
    long_ticket = b.admit(ids[3], 6)
    t0 = time.perf_counter()
    while b.counts()["running"] == 0 and time.perf_counter() - t0 < 10:
        time.sleep(0.001)
    tickets = []
    for k in range(3):
        assert b.counts()["running"] >= 1
        tickets.append(b.admit(ids[k], 1))
        time.sleep(0.002)
    got = []
    while len(got) < 4 and time.perf_counter() - t0 < 300:
        got += b.tick(wait_s=0.5)
    assert sorted(r["id"] for r in got) == sorted([long_ticket] + tickets)
    assert all(r["status"] >= 0 for r in got)
    assert b.tick() == [] and b.counts()["unreported"] == 0
    by = {r["id"]: r for r in got}
    long_r = by[long_ticket]
    assert any(by[t]["start_s"] < long_r["finish_s"] for t in tickets)  # overlapped
    assert all(r["start_s"] >= r["arrival_s"] for r in got)
    states = [b.state(i) for i in ids]
    b.close()
    for (x1, v1), (x2, v2) in zip(ref[2], states):
        assert np.array_equal(x1, x2) and np.array_equal(v1, v2)


def test_admit_rejects_unknown_instance_and_tick_polls():
    from paper_2505_13390_gb300 import mgpbd
    from paper_2505_13390_gb300.mgpbd import Batch
    b = Batch(64 << 30, 2)
    m, p = meshes()[0]
    i = b.add(m, common(p, 0))
    with pytest.raises(mgpbd.MgpbdError):
        b.admit(i + 1, 1)
    with pytest.raises(mgpbd.MgpbdError):
        b.admit(i, 0)
    assert b.tick() == []
    t = b.admit(i, 1)
    res = []
    while not res:
        res = b.tick(wait_s=1.0)
    assert [r["id"] for r in res] == [t] and res[0]["status"] >= 0
    assert res[0]["arrival_s"] <= res[0]["start_s"] <= res[0]["finish_s"] <= b.counts()["clock"]
    b.close()


def cohort_meshes():
    """Instances of different hierarchy depths for the batched (cohort) form:
    a 12x12 cloth (one level: solved alone by the stepping thread), a 20x20
    cloth (two levels), a 16x16 cloth with coarse_max 20 (three levels), a
    6x5x7 block with coarse_max 40 (three levels) and a 20x33x20 block (four
    levels)."""
    from paper_2505_13390_gb300.meshgen import workload
    out = [(cloth(12, plane="xz", alpha=1e-6, pin="corners", seed=10), default_params()),
           (cloth(20, plane="xz", alpha=1e-6, pin="corners", seed=11), default_params()),
           (cloth(16, plane="xz", alpha=1e-6, pin="corners", noise=1e-3, seed=3),
            default_params(coarse_max=20, max_levels=4)),
           (hex_block(6, 5, 7, h=0.005, jitter=0.1, alpha=1e-10, pin="y0", seed=1),
            default_params(omega_x=0.1, coarse_max=40)),
           workload("block20x33x20")]
    return out


def serve_cohort(ms, max_active, requests, cohort):
    from paper_2505_13390_gb300.mgpbd import Batch
    b = Batch(64 << 30, max_active, cohort=cohort)
    ids = [b.add(m, common(p, 1)) for m, p in ms]
    st, res = b.run(requests)
    states = [b.state(i) for i in ids]
    b.close()
    return st, res, states


def test_cohort_mix_equals_alone_bitwise():
    """The batched form: every running request's PCG iterations run as one
    launch per step.  Each instance keeps its own grids and reduction order,
    so its states and PCG iteration counts are bit for bit those of serving
    one request at a time on its own stream, and of a plain solver."""
    ms = cohort_meshes()
    reqs = trace(len(ms), 2, 0.0)
    st1, res1, alone = serve_cohort(ms, 1, reqs, False)
    stc, resc, mixed = serve_cohort(ms, 8, reqs, True)
    assert st1 >= 0 and stc >= 0
    assert [r["pcg_iters"] for r in res1] == [r["pcg_iters"] for r in resc]
    for (x1, v1), (xc, vc) in zip(alone, mixed):
        assert np.array_equal(x1, xc) and np.array_equal(v1, vc)
    from paper_2505_13390_gb300.mgpbd import Solver
    m, p = ms[4]
    g = Solver(m, common(p, 1), stream=torch.cuda.Stream())
    for _ in range(2):
        g.begin_frame()
        for _ in range(4):
            g.iterate()
        g.end_frame()
    assert g.levels == 4
    x, v = g.get_state()
    g.close()
    assert np.array_equal(x, mixed[4][0]) and np.array_equal(v, mixed[4][1])


def test_cohort_admit_while_running():
    """Requests admitted while the cohort is stepping join it at the next
    chunk; each result comes back once and every state equals the
    one-at-a-time run."""
    import time

    from paper_2505_13390_gb300.mgpbd import Batch
    ms = cohort_meshes()
    ref = serve_cohort(ms, 1, [(0, 4, 3, 0.0)] + [(1 + k, k, 1, 0.0) for k in range(4)], False)
    b = Batch(64 << 30, 8, cohort=True)
    ids = [b.add(m, common(p, 1)) for m, p in ms]
    first = b.admit(ids[4], 3)
    t0 = time.perf_counter()
    while b.counts()["running"] == 0 and time.perf_counter() - t0 < 10:
        time.sleep(0.001)
    tickets = [b.admit(ids[k], 1) for k in range(4)]
    got = []
    while len(got) < 5 and time.perf_counter() - t0 < 300:
        got += b.tick(wait_s=0.5)
    assert sorted(r["id"] for r in got) == sorted([first] + tickets)
    assert all(r["status"] >= 0 for r in got)
    by = {r["id"]: r for r in got}
    assert any(by[t]["start_s"] < by[first]["finish_s"] for t in tickets)
    states = [b.state(i) for i in ids]
    b.close()
    for (x1, v1), (x2, v2) in zip(ref[2], states):
        assert np.array_equal(x1, x2) and np.array_equal(v1, v2)
