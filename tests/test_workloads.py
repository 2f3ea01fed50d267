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
