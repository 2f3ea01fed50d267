"""The allocation-free entry point mgpbd_true_residual_noalloc.

Callers that cannot allocate device memory while they run (a thread that is
capturing a CUDA stream into a graph, a real-time loop, an application whose
device memory belongs to another pool) use this call: it computes the same
FP64 true relative residual that mgpbd_solve reports, but keeps its block
partials in a static device array instead of memory allocated for the
instance.  This file is collected last so that a run stopping at the first
failure has run every other test before it.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _call(lib, h, b, x, out):
    return lib.mgpbd_true_residual_noalloc(h, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                           C.c_void_p(out.data_ptr()))


@pytest.mark.parametrize("name", ["cloth32", "beam40"])
def test_noalloc_true_residual_matches_solve(name):
    from oracle.oracle import Oracle
    from paper_2505_13390_gb300 import mgpbd
    from paper_2505_13390_gb300.meshgen import workload

    mesh, p = workload(name)
    p = dict(p, pcg_maxiter=60)
    g = mgpbd.Solver(mesh, p)
    g.begin_frame()
    g.eval_assemble()
    g.prepare_solve()
    b = torch.from_numpy(g.constraints()[1]).cuda()
    x, info = g.solve(b)
    lib = mgpbd.load()
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    assert _call(lib, g.h, b, x, out) == mgpbd.OK, lib.mgpbd_last_error()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    got = []
    for _ in range(2):  # two calls in a row share the static scratch
        out.fill_(-1.0)
        st = _call(lib, g.h, b, x, out)
        assert st == mgpbd.OK, lib.mgpbd_last_error()
        torch.cuda.synchronize()
        got.append(float(out[0].item()))
    # nothing was allocated on the device by the two calls
    assert torch.cuda.mem_get_info()[0] == free0
    # the existing entry point's value
    ref = info["true_rel_res"]
    assert ref > 0
    for v in got:
        assert v == pytest.approx(ref, rel=1e-10)
    assert got[0] == got[1]
    # and |b - A x| / |b| recomputed in numpy from the oracle's A (the same
    # matrix bit for bit) and the solution
    o = Oracle(mesh, p)
    o.begin_frame()
    o.eval_assemble()
    ptr, col, val = o.matrix(0)
    assert np.array_equal(val, g.matrix(0)[2])
    xs, bs = x.cpu().numpy(), b.cpu().numpy()
    Ax = np.add.reduceat(val * xs[col], ptr[:-1])
    indep = np.linalg.norm(bs - Ax) / np.linalg.norm(bs)
    assert got[0] == pytest.approx(indep, rel=1e-8)
    g.close()


def test_noalloc_empty_instance_gives_zero():
    """An instance with no constraint rows: the residual is 0 and no kernel
    is needed."""
    from paper_2505_13390_gb300 import mgpbd
    from paper_2505_13390_gb300.meshgen import Mesh, default_params
    rest = np.zeros((2, 3))
    rest[1, 0] = 1.0
    mesh = Mesh("empty", rest, np.ones(2), np.zeros((0, 2), np.int32),
                np.zeros((0, 4), np.int32), np.zeros(0), rest.copy(), np.zeros((2, 3)))
    g = mgpbd.Solver(mesh, default_params())
    lib = mgpbd.load()
    b = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    assert _call(lib, g.h, b, b, out) == mgpbd.OK
    torch.cuda.synchronize()
    assert float(out[0].item()) == 0.0
    g.close()


def test_noalloc_rejects_null_arguments():
    from paper_2505_13390_gb300 import mgpbd
    lib = mgpbd.load()
    assert lib.mgpbd_true_residual_noalloc(None, None, None, None) == mgpbd.E_INVALID
