"""Pins of the oracle with k > 1 near-kernel vectors (Sec. 4.3, six in the paper).

With k vectors the tentative prolongator has k columns per aggregate, from
a QR factorisation of each aggregate's block of B, and the next level's
near-kernel is the R factor.  Pinned against what the mathematics fixes:
Q has orthonormal live columns and Q R reproduces B; the coarse operator
equals P^T A P built with scipy (dead columns give identity rows) and is
exactly symmetric and positive definite; the V-cycle stays symmetric; PCG
still reaches a dense Cholesky solution; each column of B is the k = 1
near-kernel procedure run from its own generator stream.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle.oracle import Oracle
from paper_2505_13390_gb300.meshgen import cloth, default_params, hex_block

K = 6


def case(name="h3", k=K, soft=False, **kw):
    if name == "c8":
        mesh = cloth(8, plane="xz", alpha=1e-4 if soft else 1e-6, pin="corners", noise=1e-3,
                     seed=3)
    elif name == "h3":
        mesh = hex_block(3, 2, 2, h=0.01, jitter=0.1, alpha=1e-4 if soft else 1e-7, pin="x0",
                         seed=4)
    else:  # h4: a block whose coarse level still coarsens with six columns per aggregate
        mesh = hex_block(6, 3, 3, h=0.01, jitter=0.1, alpha=1e-4 if soft else 1e-7, pin="x0",
                         seed=4)
    p = default_params(coarse_max=30, max_levels=4, pcg_rtol=1e-12, pcg_maxiter=2000,
                       nk_vectors=k, **kw)
    o = Oracle(mesh, p)
    o.begin_frame()
    o.eval_assemble()
    assert o.prepare_solve() == 0
    return mesh, p, o


def csr(o, l):
    ptr, col, val = o.matrix(l)
    n = len(ptr) - 1
    return ptr, col, val, sp.csr_matrix((val, col, ptr), shape=(n, n))


def prolongator(agg, P, na, k):
    rows, cols, vals = [], [], []
    for i, a in enumerate(agg):
        if a >= 0:
            for c in range(k):
                rows.append(i)
                cols.append(a * k + c)
                vals.append(P[i, c])
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(agg), na * k))


@pytest.mark.parametrize("name", ["c8", "h3", "h4"])
def test_qr_of_each_aggregate(name):
    mesh, p, o = case(name)
    assert o.levels >= 2
    for l in range(o.levels - 1):
        na, agg, root, P, B = o.level_agg(l)
        _, _, _, _, Bc = o.level_agg(l + 1)
        assert P.shape == (len(agg), K) and Bc.shape == (na * K, K)
        assert np.all(P[agg < 0] == 0)
        for a in range(na):
            m = np.nonzero(agg == a)[0]
            Q, R = P[m], Bc[a * K:(a + 1) * K]
            live = np.any(Q != 0, axis=0)
            assert np.allclose(Q.T @ Q, np.diag(live.astype(float)), atol=1e-12)
            assert np.allclose(np.triu(R), R, atol=0)  # upper triangular
            assert np.all(R[~live, :][:, ~live] == 0)
            scale = np.abs(B[m]).max()
            assert np.allclose(Q @ R, B[m], rtol=0, atol=1e-9 * scale)


@pytest.mark.parametrize("name", ["c8", "h3", "h4"])
def test_galerkin_with_k_columns(name):
    mesh, p, o = case(name)
    for l in range(o.levels - 1):
        na, agg, _, P, _ = o.level_agg(l)
        _, _, _, A = csr(o, l)
        ptr, col, val, Ac = csr(o, l + 1)
        Pm = prolongator(agg, P, na, K)
        ref = (Pm.T @ A @ Pm).toarray()
        dead = ~np.asarray(abs(Pm).sum(axis=0) > 0).ravel()
        ref[dead, dead] = 1.0
        got = Ac.toarray()
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        assert np.array_equal(got, got.T)  # canonical order + mirror: bitwise symmetric
        np.linalg.cholesky(got)  # positive definite
        # pattern: diagonal last, off-diagonals ascending
        for r in range(len(ptr) - 1):
            c = col[ptr[r]:ptr[r + 1]]
            assert c[-1] == r and np.all(np.diff(c[:-1]) > 0)


def test_near_kernel_columns_are_the_single_vector_procedure():
    mesh, p, o = case("h3")
    _, _, _, _, B = o.level_agg(0)
    for c in range(K):
        _, _, o1 = case("h3", k=1, seed_nk=p["seed_nk"] + c)
        _, _, _, _, B1 = o1.level_agg(0)
        assert np.array_equal(B[:, c], B1)


@pytest.mark.parametrize("name", ["c8", "h4"])
def test_vcycle_symmetric_with_k_columns(name):
    mesh, p, o = case(name)
    rng = np.random.default_rng(4)
    r1, r2 = rng.standard_normal((2, mesh.n_rows))
    z1, z2 = o.vcycle(r1), o.vcycle(r2)
    assert abs(z1 @ r2 - r1 @ z2) <= 1e-12 * abs(z1 @ r2)
    assert r1 @ z1 > 0


@pytest.mark.parametrize("name", ["c8", "h3"])
def test_pcg_with_k_columns_matches_dense_cholesky(name):
    mesh, p, o = case(name, soft=True)
    _, _, _, A = csr(o, 0)
    b = np.random.default_rng(2).standard_normal(mesh.n_rows)
    x, info = o.solve(b)
    ref = sla.cho_solve(sla.cho_factor(A.toarray()), b)
    assert info["status"] == 0
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)


def test_one_vector_is_unchanged():
    """nk_vectors = 1 is the k = 1 path bit for bit."""
    _, _, o1 = case("h3", k=1)
    mesh = hex_block(3, 2, 2, h=0.01, jitter=0.1, alpha=1e-7, pin="x0", seed=4)
    p = default_params(coarse_max=30, max_levels=4, pcg_rtol=1e-12, pcg_maxiter=2000)
    o = Oracle(mesh, p)
    o.begin_frame()
    o.eval_assemble()
    o.prepare_solve()
    for l in range(o.levels):
        for a, b in zip(o.matrix(l), o1.matrix(l)):
            assert np.array_equal(a, b)


def node_matrix_numpy(ptr, col, val, k):
    """Block Frobenius norms of a k-unknowns-per-node CSR, diagonal last."""
    n = len(ptr) - 1
    nn = n // k
    blocks = [dict() for _ in range(nn)]
    for r in range(n):
        a = r // k
        for e in range(ptr[r], ptr[r + 1]):
            b = col[e] // k
            blocks[a][b] = blocks[a].get(b, 0.0) + val[e] ** 2
    nptr, ncol, nval = [0], [], []
    for a in range(nn):
        off = sorted(b for b in blocks[a] if b != a)
        for b in off + [a]:
            ncol.append(b)
            nval.append(np.sqrt(blocks[a][b]))
        nptr.append(len(ncol))
    return np.array(nptr), np.array(ncol), np.array(nval)


def test_coarse_levels_aggregate_whole_nodes():
    """With k > 1 the coarse levels aggregate nodes (the k unknowns of a
    coarse aggregate stay together): the aggregates equal the pinned MIS-2
    rule applied to the block-norm node matrix built here in numpy, and the
    hierarchy keeps coarsening."""
    from oracle.oracle import aggregate_csr
    mesh = hex_block(8, 4, 4, h=0.01, jitter=0.1, alpha=1e-7, pin="x0", seed=4)
    p = default_params(coarse_max=30, max_levels=5, nk_vectors=K)
    o = Oracle(mesh, p)
    o.begin_frame()
    o.eval_assemble()
    assert o.prepare_solve() == 0
    sizes = [len(o.matrix(l)[0]) - 1 for l in range(o.levels)]
    assert o.levels >= 3 and all(b < a for a, b in zip(sizes, sizes[1:]))
    for l in range(1, o.levels - 1):
        ptr, col, val = o.matrix(l)
        na, agg, root, _, _ = o.level_agg(l)
        nptr, ncol, nval = node_matrix_numpy(ptr, col, val, K)
        ref_na, ref_agg, ref_root, _ = aggregate_csr(nptr, ncol, nval, p["theta_s"],
                                                     p["seed_agg"], l)
        assert na == ref_na
        assert np.array_equal(agg, np.repeat(ref_agg, K))
        assert np.array_equal(root, np.repeat(ref_root, K))
