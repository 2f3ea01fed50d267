"""The OpenMP build of the oracle gives the plain build's bits.

Only loops over independent rows run in parallel in that build (sums across
rows stay sequential), so every stage of Alg. 1 -- constraints, A, the whole
setup, the V-cycle, PCG and the position update -- must match the plain
build exactly, with several threads.  The OpenMP build is what times the
oracle on all host cores and what runs it at the larger test sizes."""
import numpy as np
import pytest

from oracle import oracle
from oracle.oracle import Oracle
from paper_2505_13390_gb300.meshgen import cloth, default_params, hex_block


@pytest.mark.parametrize("case", ["cloth", "block", "cheb"])
def test_openmp_build_is_bitwise_the_plain_build(case):
    if case == "cloth":
        mesh = cloth(24, plane="xz", alpha=1e-6, pin="corners", noise=1e-3, seed=3)
        p = default_params(coarse_max=40, pcg_rtol=1e-8)
    else:
        mesh = hex_block(5, 4, 6, h=0.005, jitter=0.1, alpha=1e-8, pin="y0", seed=1)
        p = default_params(omega_x=0.1, pcg_rtol=1e-6, coarse_max=60,
                           smoother=2 if case == "cheb" else 0)
    assert oracle.threads(4) == 4
    runs = []
    for omp in (False, True):
        o = Oracle(mesh, p, omp=omp)
        o.begin_frame()
        info = [o.iterate() for _ in range(3)]
        o.end_frame()
        x, v = o.get_state()
        mats = [o.matrix(l) for l in range(o.levels)]
        aggs = [o.level_agg(l) for l in range(o.levels - 1)]
        runs.append((x, v, info, mats, aggs, o.constraints()))
    (x0, v0, i0, m0, a0, c0), (x1, v1, i1, m1, a1, c1) = runs
    assert np.array_equal(x0, x1) and np.array_equal(v0, v1)
    assert [d["pcg_iters"] for d in i0] == [d["pcg_iters"] for d in i1]
    assert [d["true_rel_res"] for d in i0] == [d["true_rel_res"] for d in i1]
    for a, b in zip(m0, m1):
        assert all(np.array_equal(u, w) for u, w in zip(a, b))
    for a, b in zip(a0, a1):
        assert a[0] == b[0] and all(np.array_equal(u, w) for u, w in zip(a[1:], b[1:]))
    assert all(np.array_equal(u, w) for u, w in zip(c0, c1))
