"""The synthetic workloads have the sizes of the recipes they stand for.

Vertex, row and nonzero counts of each named workload against counts worked
out independently from the recipes: cloth 32x32 (structural + one shear
diagonal), beam 40x10x10 and block 100x33x100 (5 tets per hex cell, every
cell edge a distance row), cloth 512x512 with bend edges.  nnz(A) is the
number of row pairs sharing a vertex, diagonal included, built here from the
row-vertex incidence with scipy (block100's 376.5M-entry pattern is checked
on the GPU path at run time by bench.py instead).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2505_13390_gb300.meshgen import workload

CASES = [
    # name, verts, distance rows, tets, nnz(A) or None
    ("cloth32", 1_024, 2_945, 0, 31_401),
    ("beam40", 4_961, 26_760, 20_000, 4_293_718),
    ("cloth512", 262_144, 1_306_625, 0, 24_764_561),
    ("block100", 346_834, 2_030_033, 1_650_000, None),
]


def pattern_nnz(mesh):
    rows = [np.repeat(np.arange(mesh.n_dist), 2), mesh.n_dist + np.repeat(np.arange(mesh.n_tet), 4)]
    cols = [mesh.dist.ravel(), mesh.tet.ravel()]
    r = np.concatenate(rows)
    c = np.concatenate(cols).astype(np.int64)
    R = sp.csr_matrix((np.ones(len(r), np.float32), (r, c)), shape=(mesh.n_rows, mesh.n_verts))
    return (R @ R.T).nnz


@pytest.mark.parametrize("name,verts,dist,tets,nnz", CASES)
def test_workload_sizes(name, verts, dist, tets, nnz):
    mesh, p = workload(name)
    assert (mesh.n_verts, mesh.n_dist, mesh.n_tet) == (verts, dist, tets)
    assert mesh.n_rows == dist + tets
    assert np.all(mesh.dist[:, 0] != mesh.dist[:, 1])
    if tets:
        # every tet has four distinct vertices and positive rest volume
        t = mesh.tet
        e = mesh.rest_pos[t[:, 1:]] - mesh.rest_pos[t[:, :1]]
        assert np.all(np.linalg.det(e) > 0)
    if nnz is not None:
        assert pattern_nnz(mesh) == nnz


def test_serving_trace_recipe():
    """The seeded serving trace: half cloth N x N with N in 16..256, half beams
    L x 10 x 10 with L in 10..80, alpha = 10^U(-9,-6); Poisson arrivals at the
    given rate (exponential gaps, so mean gap 1/rate and coefficient of
    variation 1), instances drawn uniformly; the same seed gives the same trace."""
    from paper_2505_13390_gb300.meshgen import instance_mesh, serving_trace
    inst, reqs = serving_trace(n_requests=4000, n_instances=400, rate_hz=2.0, seed=6)
    kinds = np.array([i["kind"] == "cloth" for i in inst])
    assert abs(kinds.mean() - 0.5) < 4 * np.sqrt(0.25 / len(inst))
    for i in inst:
        lo, hi = (16, 256) if i["kind"] == "cloth" else (10, 80)
        assert lo <= i["size"] <= hi and 1e-9 <= i["alpha"] <= 1e-6
    t = np.array([r["t"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 0.5) < 4 * 0.5 / np.sqrt(len(gaps))
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1
    counts = np.bincount([r["instance"] for r in reqs], minlength=len(inst))
    assert counts.max() < 30  # uniform: about 10 each
    assert serving_trace(n_requests=50, n_instances=8, seed=6) == \
        serving_trace(n_requests=50, n_instances=8, seed=6)
    # an instance's mesh follows its kind and size
    mesh, p = instance_mesh(next(i for i in inst if i["kind"] == "beam"))
    assert mesh.n_tet == 5 * 100 * next(i for i in inst if i["kind"] == "beam")["size"]
