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


@pytest.mark.parametrize("name", ["cloth32", "beam40"])
def test_noalloc_true_residual_matches_solve(name):
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
    got = []
    for _ in range(2):  # two calls in a row share the static scratch
        st = lib.mgpbd_true_residual_noalloc(g.h, C.c_void_p(b.data_ptr()),
                                             C.c_void_p(x.data_ptr()),
                                             C.c_void_p(out.data_ptr()))
        assert st == mgpbd.OK, lib.mgpbd_last_error()
        torch.cuda.synchronize()
        got.append(float(out[0].item()))
    ref = info["true_rel_res"]
    assert ref > 0
    for v in got:
        assert v == pytest.approx(ref, rel=1e-10)
    assert got[0] == got[1]
    g.close()


def test_noalloc_rejects_null_arguments():
    from paper_2505_13390_gb300 import mgpbd
    lib = mgpbd.load()
    assert lib.mgpbd_true_residual_noalloc(None, None, None, None) == mgpbd.E_INVALID
