"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a published
reference value, finite differences, a dense brute-force construction with
numpy/scipy, a textbook special case, or a definitional characterisation
checked by brute force on small inputs.  No test here needs a GPU.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle.oracle import Oracle, aggregate_csr, colour_csr, h64
from paper_2505_13390_gb300.meshgen import Mesh, cloth, default_params, hex_block

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# helpers (independent constructions, not calls into the oracle's arithmetic)
# --------------------------------------------------------------------------

def row_vertices(mesh):
    return [tuple(e) for e in mesh.dist.tolist()] + [tuple(t) for t in mesh.tet.tolist()]


def dense_J(o, mesh):
    """Constraint Jacobian (m x 3N) laid out from the oracle's per-vertex gradients."""
    Cv, b, gd, gt = o.constraints()
    m, N = mesh.n_rows, mesh.n_verts
    J = np.zeros((m, 3 * N))
    for j, (a, c) in enumerate(mesh.dist.tolist()):
        J[j, 3 * a:3 * a + 3] += gd[j]
        J[j, 3 * c:3 * c + 3] -= gd[j]
    for t, verts in enumerate(mesh.tet.tolist()):
        for s, v in enumerate(verts):
            J[mesh.n_dist + t, 3 * v:3 * v + 3] += gt[t, s]
    return J


def csr_of(o, level=0):
    ptr, col, val = o.matrix(level)
    n = len(ptr) - 1
    return ptr, col, val, sp.csr_matrix((val, col, ptr), shape=(n, n))


def small_meshes():
    m1 = cloth(5, plane="xz", alpha=1e-6, pin="corners", noise=1e-3, seed=3, name="c5")
    m2 = hex_block(2, 1, 1, h=0.01, jitter=0.1, alpha=1e-7, pin="x0", seed=4, name="h2")
    # perturb the tet mesh so that gradients are generic
    rng = np.random.default_rng(9)
    m2.x0 = m2.rest_pos + rng.uniform(-1e-3, 1e-3, m2.rest_pos.shape) * (m2.inv_mass > 0)[:, None]
    return [m1, m2]


def params_small(**kw):
    p = default_params(coarse_max=4, max_levels=8, pcg_rtol=1e-12, pcg_maxiter=500)
    p.update(kw)
    return p


# --------------------------------------------------------------------------
# counter-based generator
# --------------------------------------------------------------------------

def test_splitmix64_reference_values():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64.txt"))
            if l.strip() and not l.startswith("#")]
    assert rows
    for k, v in rows:
        assert h64(int(k, 16)) == int(v, 16)


# --------------------------------------------------------------------------
# constraints and gradients (Alg. 1, eq. 3)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("mi", [0, 1])
def test_gradients_match_finite_differences(mi):
    mesh = small_meshes()[mi]
    o = Oracle(mesh, params_small())
    x = mesh.x0.copy()
    o.set_state(x, mesh.v0)
    o.eval_assemble()
    J = dense_J(o, mesh)
    h = 1e-7
    Jfd = np.zeros_like(J)
    for q in range(x.size):
        xp = x.copy().ravel()
        xm = x.copy().ravel()
        xp[q] += h
        xm[q] -= h
        o.set_state(xp.reshape(-1, 3), mesh.v0)
        o.eval_assemble()
        cp = o.constraints()[0]
        o.set_state(xm.reshape(-1, 3), mesh.v0)
        o.eval_assemble()
        cm = o.constraints()[0]
        Jfd[:, q] = (cp - cm) / (2 * h)
    scale = np.abs(J).max(axis=1, keepdims=True)
    assert np.all(np.abs(J - Jfd) <= 1e-6 * scale + 1e-12)


def test_constraint_closed_forms():
    # one axis-aligned edge of rest length 0.5 stretched to 1 and one unit right tet
    rest = np.array([[0, 0, 0], [0.5, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    x = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    mesh = Mesh("t", rest, np.ones(4), np.array([[1, 0]], np.int32),
                np.array([[0, 1, 2, 3]], np.int32), np.array([1e-6, 1e-6]), x, np.zeros((4, 3)))
    o = Oracle(mesh, params_small())
    o.eval_assemble()
    Cv, b, gd, gt = o.constraints()
    L0, V0 = o.rest()
    assert L0[0] == 0.5 and V0[0] == 0.5 / 6.0
    assert Cv[0] == 0.5
    assert np.array_equal(gd[0], [1.0, 0.0, 0.0])
    assert Cv[1] == pytest.approx(1.0 / 6.0 - 0.5 / 6.0, rel=1e-15)
    expect = np.array([[-1, -1, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1]]) / 6.0
    assert np.allclose(gt[0], expect, rtol=0, atol=1e-17)
    # b = -C - alpha~ lambda with lambda = 0 right after create
    assert np.array_equal(b, -Cv)


def test_degenerate_edge_has_zero_gradient():
    rest = np.array([[0, 0, 0], [1, 0, 0]], float)
    x = np.zeros((2, 3))
    mesh = Mesh("d", rest, np.ones(2), np.array([[0, 1]], np.int32), np.zeros((0, 4), np.int32),
                np.array([1e-6]), x, np.zeros((2, 3)))
    o = Oracle(mesh, params_small())
    o.eval_assemble()
    Cv, b, gd, gt = o.constraints()
    assert Cv[0] == -1.0 and np.all(gd == 0)
    _, _, val, _ = csr_of(o)
    assert val[-1] == 1e-6 / (default_params()["dt"] ** 2)


# --------------------------------------------------------------------------
# pattern and assembly (eq. 3, Sec. 4.2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("mi", [0, 1])
def test_pattern_brute_force(mi):
    mesh = small_meshes()[mi]
    o = Oracle(mesh, params_small())
    ptr, col, _, _ = csr_of(o)
    rv = row_vertices(mesh)
    m = len(rv)
    cmap = o.assembly_map()
    for i in range(m):
        nbrs = sorted(j for j in range(m) if j != i and set(rv[i]) & set(rv[j]))
        assert list(col[ptr[i]:ptr[i + 1]]) == nbrs + [i]  # diagonal last
        for k in range(ptr[i], ptr[i + 1] - 1):
            j = col[k]
            shared = sorted(set(rv[i]) & set(rv[j]))
            code = int(cmap[k])
            assert code & 3 == len(shared)
            got = []
            for p in range(code & 3):
                si = (code >> (2 + 4 * p)) & 3
                sj = (code >> (4 + 4 * p)) & 3
                assert rv[i][si] == rv[j][sj]
                got.append(rv[i][si])
            assert got == shared


@pytest.mark.parametrize("mi", [0, 1])
def test_A_equals_dense_J_Minv_JT_plus_alpha(mi):
    mesh = small_meshes()[mi]
    p = params_small()
    o = Oracle(mesh, p)
    o.eval_assemble()
    J = dense_J(o, mesh)
    W = np.repeat(mesh.inv_mass, 3)
    at = mesh.alpha / (p["dt"] ** 2)
    Ad = (J * W) @ J.T + np.diag(at)
    _, _, _, A = csr_of(o)
    A = A.toarray()
    assert np.abs(A - Ad).max() <= 1e-14 * np.abs(Ad).max()


@pytest.mark.parametrize("mi", [0, 1])
def test_A_symmetric_positive_definite(mi):
    mesh = small_meshes()[mi]
    p = params_small()
    o = Oracle(mesh, p)
    o.eval_assemble()
    _, _, _, A = csr_of(o)
    A = A.toarray()
    assert np.array_equal(A, A.T)  # bitwise symmetric by the summation order
    ev = np.linalg.eigvalsh(A)
    assert ev.min() > 0
    np.linalg.cholesky(A)
    # distance rows: A_ii = w_a + w_b + alpha~ (|n| = 1), Sec. 4.2
    at = mesh.alpha / (p["dt"] ** 2)
    for j, (a, b) in enumerate(mesh.dist.tolist()):
        expect = mesh.inv_mass[a] + mesh.inv_mass[b] + at[j]
        assert A[j, j] == pytest.approx(expect, rel=1e-14)


# --------------------------------------------------------------------------
# XPBD special cases (eq. 4, Alg. 1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("omega_x", [1.0, 0.25])
def test_single_constraint_reduces_to_xpbd_update(omega_x):
    rest = np.array([[0, 0, 0], [1, 0, 0]], float)
    x0 = np.array([[0, 0, 0], [1.3, 0.1, -0.2]], float)
    w = np.array([0.5, 2.0])
    alpha = np.array([1e-3])
    mesh = Mesh("one", rest, w, np.array([[0, 1]], np.int32), np.zeros((0, 4), np.int32),
                alpha, x0, np.zeros((2, 3)))
    p = params_small(gravity=(0.0, 0.0, 0.0), omega_x=omega_x, max_iter=1)
    o = Oracle(mesh, p)
    o.begin_frame()
    o.eval_assemble()
    Cv, b, gd, _ = o.constraints()
    info = o.iterate()
    lam, dl = o.lam()
    at = alpha[0] / p["dt"] ** 2
    d = x0[0] - x0[1]
    Cexp = np.linalg.norm(d) - 1.0
    assert Cv[0] == pytest.approx(Cexp, rel=1e-14)
    expect = -(Cexp + at * 0.0) / (w[0] + w[1] + at)
    assert dl[0] == pytest.approx(expect, rel=1e-13)
    assert info["pcg_iters"] == 1
    # eq. 5: dx = M^-1 grad C^T dlambda, applied with the relaxation omega_x
    x, _ = o.get_state()
    n = d / np.linalg.norm(d)
    assert np.allclose(x[0], x0[0] + omega_x * w[0] * n * expect, rtol=0, atol=1e-15)
    assert np.allclose(x[1], x0[1] - omega_x * w[1] * n * expect, rtol=0, atol=1e-15)
    lam, _ = o.lam()
    assert lam[0] == dl[0]  # lambda takes the full update (Alg. 1)


def test_single_constraint_stays_at_the_compliant_solution():
    """Two particles and one distance constraint, omega_x = 1: the motion is
    along n, so C is linear in lambda and the implicit equations C(x) +
    alpha~ lambda = 0, x = x~ + M^-1 grad C^T lambda (eq. 3-5) have the closed
    form lambda* = -C~ / (w_a + w_b + alpha~).  One global iteration reaches it
    and later ones keep it: lambda is the running sum of the updates (Alg. 1),
    so the right-hand side b = -C - alpha~ lambda stays 0."""
    rest = np.array([[0, 0, 0], [1, 0, 0]], float)
    x0 = np.array([[0.2, -0.1, 0.05], [1.3, 0.1, -0.2]], float)
    w = np.array([0.5, 2.0])
    alpha = np.array([1e-3])
    mesh = Mesh("one", rest, w, np.array([[0, 1]], np.int32), np.zeros((0, 4), np.int32),
                alpha, x0, np.zeros((2, 3)))
    p = params_small(gravity=(0.0, 0.0, 0.0), omega_x=1.0, max_iter=6)
    o = Oracle(mesh, p)
    o.begin_frame()
    at = alpha[0] / p["dt"] ** 2
    d = x0[0] - x0[1]
    n = d / np.linalg.norm(d)
    C0 = np.linalg.norm(d) - 1.0
    lam_star = -C0 / (w[0] + w[1] + at)
    for it in range(6):
        o.iterate()
        lam, _ = o.lam()
        x, _ = o.get_state()
        assert lam[0] == pytest.approx(lam_star, rel=1e-12), it
        assert np.allclose(x[0], x0[0] + w[0] * lam_star * n, rtol=0, atol=1e-14), it
        assert np.allclose(x[1], x0[1] - w[1] * lam_star * n, rtol=0, atol=1e-14), it
    o.eval_assemble()
    _, b, _, _ = o.constraints()
    assert abs(b[0]) <= 1e-12 * abs(C0)
    # the next frame starts again from lambda = 0 (Alg. 1); its prediction
    # x~ = x + dt v moves along n as well, so the same closed form holds there
    o.end_frame()
    o.begin_frame()
    xt, _ = o.get_state()
    d2 = xt[0] - xt[1]
    n2 = d2 / np.linalg.norm(d2)
    C2 = np.linalg.norm(d2) - 1.0
    lam2 = -C2 / (w[0] + w[1] + at)
    assert np.allclose(n2, n, rtol=0, atol=1e-14) and abs(C2) > 1e-3
    for it in range(4):
        o.iterate()
        lam, _ = o.lam()
        x, _ = o.get_state()
        assert lam[0] == pytest.approx(lam2, rel=1e-12), it
        assert np.allclose(x[0], xt[0] + w[0] * lam2 * n2, rtol=0, atol=1e-14), it
        assert np.allclose(x[1], xt[1] - w[1] * lam2 * n2, rtol=0, atol=1e-14), it


def test_singular_system_is_reported():
    """A = 0: one distance row between two pinned vertices with zero
    compliance.  The coarsest Cholesky meets a zero pivot and the solve is
    refused as singular instead of returning non-finite values."""
    rest = np.array([[0, 0, 0], [1, 0, 0]], float)
    x0 = np.array([[0, 0, 0], [1.2, 0, 0]], float)
    mesh = Mesh("s", rest, np.zeros(2), np.array([[0, 1]], np.int32), np.zeros((0, 4), np.int32),
                np.array([0.0]), x0, np.zeros((2, 3)))
    o = Oracle(mesh, params_small(gravity=(0.0, 0.0, 0.0)))
    o.begin_frame()
    o.eval_assemble()
    assert np.array_equal(o.matrix(0)[2], [0.0])
    assert o.prepare_solve() == -4  # singular


@pytest.mark.parametrize("mi", [0, 1])
def test_rest_mesh_gives_zero_update(mi):
    mesh = small_meshes()[mi]
    mesh.x0 = mesh.rest_pos.copy()
    p = params_small(gravity=(0.0, 0.0, 0.0), max_iter=3)
    o = Oracle(mesh, p)
    st, hist = o.step(1)
    assert st == 0
    x, v = o.get_state()
    assert np.array_equal(x, mesh.rest_pos)
    assert np.all(v == 0)
    assert all(h["bnorm"] == 0.0 and h["pcg_iters"] == 0 for h in hist)


def test_free_fall_without_constraints():
    N = 3
    rest = np.arange(9, dtype=float).reshape(3, 3)
    v0 = np.array([[0.1, 0, 0], [0, 0.2, 0], [0, 0, 0.3]])
    mesh = Mesh("ff", rest, np.array([1.0, 1.0, 0.0]), np.zeros((0, 2), np.int32),
                np.zeros((0, 4), np.int32), np.zeros(0), rest.copy(), v0)
    p = params_small(max_iter=2)
    o = Oracle(mesh, p)
    st, _ = o.step(1)
    assert st == 0
    x, v = o.get_state()
    g = np.array(p["gravity"])
    dt = p["dt"]
    vexp = v0 + dt * g
    vexp[2] = 0.0  # pinned vertex keeps v = 0 and its position
    assert np.allclose(x[:2], rest[:2] + dt * vexp[:2], rtol=0, atol=1e-15)
    assert np.array_equal(x[2], rest[2])
    assert np.allclose(v, vexp, rtol=1e-12, atol=1e-15)


# --------------------------------------------------------------------------
# setup: strength, aggregation, injection, Galerkin (Sec. 4.1-4.4)
# --------------------------------------------------------------------------

def random_spd_pattern(n, density, seed):
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=rng, data_rvs=lambda k: rng.uniform(-1, 1, k))
    M = M + M.T
    M = M.tolil()
    M.setdiag(0)
    M = M.tocsr()
    M.eliminate_zeros()
    d = np.asarray(abs(M).sum(1)).ravel() + rng.uniform(0.5, 1.5, n)
    ptr = [0]
    col, val = [], []
    for i in range(n):
        s, e = M.indptr[i], M.indptr[i + 1]
        order = np.argsort(M.indices[s:e])
        col += list(M.indices[s:e][order]) + [i]
        val += list(M.data[s:e][order]) + [d[i]]
        ptr.append(len(col))
    return np.array(ptr), np.array(col), np.array(val)


def brute_aggregates(ptr, col, val, theta, seed, level):
    """Definitional construction of the aggregates on a small matrix."""
    n = len(ptr) - 1
    diag = np.array([val[ptr[i + 1] - 1] for i in range(n)])
    adj = [set() for _ in range(n)]
    absv = {}
    for i in range(n):
        for k in range(ptr[i], ptr[i + 1] - 1):
            j = col[k]
            absv[(i, j)] = abs(val[k])
            if abs(val[k]) >= theta * np.sqrt(abs(diag[i]) * abs(diag[j])):
                adj[i].add(j)
    ball2 = []
    for i in range(n):
        b = set(adj[i])
        for w in adj[i]:
            b |= adj[w]
        b.discard(i)
        ball2.append(b)
    pri = [h64((seed << 40) | (level << 32) | i) for i in range(n)]
    # lexicographically-first distance-2 independent set over the rows that
    # have a strong neighbour: a root is such a row with no higher-priority
    # root within distance 2; resolve by decreasing priority.  Rows without a
    # strong neighbour are left alone (no aggregate).
    root = [False] * n
    for u in sorted(range(n), key=lambda i: (pri[i], i), reverse=True):
        if not adj[u]:
            continue
        root[u] = not any(root[w] and (pri[w], w) > (pri[u], u) for w in ball2[u])
    ids = {}
    for i in range(n):
        if root[i]:
            ids[i] = len(ids)
    p1 = [-1] * n
    for r, a in ids.items():
        p1[r] = a
        for w in adj[r]:
            p1[w] = a
    agg = list(p1)
    for i in range(n):
        if p1[i] >= 0 or not adj[i]:
            continue
        cands = [(-absv[(i, w)], p1[w], w) for w in adj[i] if p1[w] >= 0]
        agg[i] = min(cands)[1]
    return np.array(root, np.uint8), np.array(agg), adj


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("theta", [0.0, 0.1, 0.3])
def test_aggregation_brute_force(seed, theta):
    ptr, col, val = random_spd_pattern(40 + 7 * seed, 0.08, seed)
    na, agg, root, S = aggregate_csr(ptr, col, val, theta, seed=4, level=seed % 3)
    broot, bagg, adj = brute_aggregates(ptr, col, val, theta, 4, seed % 3)
    assert np.array_equal(root, broot)
    assert np.array_equal(agg, bagg)
    n = len(ptr) - 1
    # disjoint and covering every row with a strong neighbour; one root per
    # aggregate; roots pairwise >= 3 apart; rows without strong neighbours alone
    assert na == int(root.sum())
    assert set(agg[agg >= 0].tolist()) == set(range(na))
    assert all((agg[i] < 0) == (len(adj[i]) == 0) for i in range(n))
    roots = np.nonzero(root)[0]
    assert sorted(agg[roots].tolist()) == list(range(na))
    for r in roots:
        near = set(adj[r])
        for w in adj[r]:
            near |= adj[w]
        assert not any(root[w] for w in near if w != r)


def test_aggregation_special_cases():
    ptr, col, val = random_spd_pattern(30, 0.1, 11)
    n = len(ptr) - 1
    # no strong connection: every row is left alone (no coarse space)
    na, agg, root, S = aggregate_csr(ptr, col, val, 1e300, seed=4)
    assert na == 0 and np.all(agg == -1) and S.sum() == 0
    # theta = 0: every stored off-diagonal is strong
    na, agg, root, S = aggregate_csr(ptr, col, val, 0.0, seed=4)
    offd = np.ones(len(col), bool)
    offd[ptr[1:] - 1] = False
    assert np.array_equal(S.astype(bool), offd)


def test_strength_hand_example():
    # 3x3 chain: |A01| = 1 vs 0.1*sqrt(4*4) = 0.4 strong; |A12| = 0.3 vs 0.1*sqrt(4*16)=0.8 weak
    ptr = np.array([0, 2, 5, 7])
    col = np.array([1, 0, 0, 2, 1, 1, 2])
    val = np.array([-1.0, 4.0, -1.0, 0.3, 4.0, 0.3, 16.0])
    _, _, _, S = aggregate_csr(ptr, col, val, 0.1, seed=4)
    assert S.tolist() == [1, 0, 1, 0, 0, 0, 0]
    # an entry is weak only below the threshold: at equality it is strong
    # (0.1 * sqrt(4 * 25) rounds to exactly 1.0)
    assert 0.1 * np.sqrt(4.0 * 25.0) == 1.0
    ptr = np.array([0, 2, 4])
    col = np.array([1, 0, 0, 1])
    val = np.array([-1.0, 4.0, -1.0, 25.0])
    _, _, _, S = aggregate_csr(ptr, col, val, 0.1, seed=4)
    assert S.tolist() == [1, 0, 1, 0]


@pytest.mark.parametrize("seed", range(4))
def test_colouring_is_greedy_by_priority(seed):
    ptr, col, val = random_spd_pattern(50, 0.1, seed + 20)
    n = len(ptr) - 1
    nc, c = colour_csr(ptr, col, seed=5, level=seed)
    pri = [(h64((5 << 40) | (seed << 32) | i), i) for i in range(n)]
    for i in range(n):
        nb = [col[k] for k in range(ptr[i], ptr[i + 1] - 1)]
        assert all(c[j] != c[i] for j in nb)  # proper colouring
        higher = {c[j] for j in nb if pri[j] > pri[i]}
        mex = 0
        while mex in higher:
            mex += 1
        assert c[i] == mex  # smallest colour absent among higher priorities
    assert nc == c.max() + 1


def hierarchy_case(name="c8", soft=False):
    """Small two-to-four level hierarchies.  ``soft`` raises the compliance so
    that cond(A) is moderate and a 1e-10 solution error is reachable."""
    if name == "c8":
        mesh = cloth(8, plane="xz", alpha=1e-4 if soft else 1e-6, pin="corners", noise=1e-3,
                     seed=3)
    else:
        mesh = hex_block(3, 2, 2, h=0.01, jitter=0.1, alpha=1e-4 if soft else 1e-7, pin="x0",
                         seed=4)
    p = default_params(coarse_max=30, max_levels=4, pcg_rtol=1e-12, pcg_maxiter=2000)
    o = Oracle(mesh, p)
    o.begin_frame()
    o.eval_assemble()
    assert o.prepare_solve() == 0
    return mesh, p, o


@pytest.mark.parametrize("name", ["c8", "h3"])
def test_prolongator_and_galerkin(name):
    mesh, p, o = hierarchy_case(name)
    assert o.levels >= 2
    for l in range(o.levels - 1):
        na, agg, root, P, B = o.level_agg(l)
        _, _, _, A = csr_of(o, l)
        _, _, _, Ac = csr_of(o, l + 1)
        n = A.shape[0]
        rows = np.nonzero(agg >= 0)[0]
        assert np.all(P[agg < 0] == 0)
        Pm = sp.csr_matrix((P[rows], (rows, agg[rows])), shape=(n, na))
        # columns of P have unit 2-norm, P^T P = I (disjoint aggregates)
        PtP = (Pm.T @ Pm).toarray()
        assert np.allclose(PtP, np.eye(na), rtol=0, atol=1e-14)
        # injection of the near-kernel: P_i = B_i / |B_agg|, so B = P * B_{l+1}
        _, _, _, _, Bc = o.level_agg(l + 1) if l + 1 < o.levels - 1 else (0, 0, 0, 0, None)
        # Galerkin: A_{l+1} = P^T A_l P (scipy product), exactly symmetric
        ref = (Pm.T @ A @ Pm).toarray()
        got = Ac.toarray()
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
        assert np.array_equal(got, got.T)
        np.linalg.cholesky(got)


def test_near_kernel_is_weighted_jacobi_on_homogeneous_system():
    mesh, p, o = hierarchy_case("c8")
    _, _, _, A = csr_of(o, 0)
    n = A.shape[0]
    _, _, _, _, B = o.level_agg(0)
    amax = np.abs(A.data).max()
    x = np.array([((h64((3 << 40) | i) >> 11) + 0.5) * 2.0 ** -53 for i in range(n)]) * amax
    Ad = A.toarray()
    d = np.diag(Ad)
    x0 = x.copy()
    for _ in range(p["nk_sweeps"]):
        x = x - p["nk_omega"] * (Ad @ x) / d
    assert np.allclose(B, x, rtol=1e-12, atol=0)
    # sweeps on A x = 0 lower the Rayleigh quotient (algebraically smoother)
    assert (B @ Ad @ B) / (B @ B) < (x0 @ Ad @ x0) / (x0 @ x0)


@pytest.mark.parametrize("name", ["c8", "h3"])
def test_power_method_omega(name):
    mesh, p, o = hierarchy_case(name)
    for l in range(o.levels - 1):
        _, _, _, A = csr_of(o, l)
        Ad = A.toarray()
        d = np.diag(Ad)
        true = np.linalg.eigvalsh(Ad / np.sqrt(np.outer(d, d))).max()
        lmax, omega = o.level_omega(l)
        # |D^-1 A y| / |y| may overshoot slightly: D^-1 A is not normal
        assert 0.8 * true <= lmax <= 1.05 * true
        assert omega == pytest.approx(2.0 / (p["power_safety"] * lmax + p["lambda_min_est"]))
        assert omega * true < 2.0  # convergent smoother keeps the V-cycle SPD


# --------------------------------------------------------------------------
# solve phase: V-cycle and MGPCG (Sec. 4.4-4.5)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("smoother", [0, 1, 2])
@pytest.mark.parametrize("name", ["c8", "h3"])
def test_vcycle_is_symmetric(name, smoother):
    mesh, p, o = hierarchy_case(name)
    if smoother:
        o2 = Oracle(mesh, dict(p, smoother=smoother))
        o2.begin_frame()
        o2.eval_assemble()
        o2.prepare_solve()
        o = o2
    rng = np.random.default_rng(1)
    u, w = rng.standard_normal((2, mesh.n_rows))
    a, b = o.vcycle(u) @ w, u @ o.vcycle(w)
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))


@pytest.mark.parametrize("smoother", [0, 1, 2])
@pytest.mark.parametrize("name", ["c8", "h3"])
def test_pcg_matches_dense_cholesky(name, smoother):
    mesh, p, o = hierarchy_case(name, soft=True)
    if smoother:
        o = Oracle(mesh, dict(p, smoother=smoother))
        o.begin_frame()
        o.eval_assemble()
        o.prepare_solve()
    _, _, _, A = csr_of(o, 0)
    Ad = A.toarray()
    rng = np.random.default_rng(2)
    b = rng.standard_normal(mesh.n_rows)
    x, info = o.solve(b)
    ref = sla.cho_solve(sla.cho_factor(Ad), b)
    assert info["status"] == 0
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
    assert info["true_rel_res"] <= 1e-10


def test_chebyshev_degree_one_is_optimal_weighted_jacobi():
    """Degree-1 Chebyshev on [lo, hi] is weighted Jacobi with omega = 2/(lo+hi),
    the paper's omega_opt: both smoothers give the same V-cycle."""
    mesh, p, o = hierarchy_case("c8")
    r = np.random.default_rng(8).standard_normal(mesh.n_rows)
    outs = []
    for sm in (0, 2):
        q = Oracle(mesh, dict(p, smoother=sm, smooth_sweeps=1))
        q.begin_frame()
        q.eval_assemble()
        q.prepare_solve()
        outs.append(q.vcycle(r))
    assert np.allclose(outs[0], outs[1], rtol=1e-12, atol=1e-14 * np.abs(outs[0]).max())


def test_chebyshev_matches_the_chebyshev_polynomial():
    """Two Chebyshev steps from x = 0 equal x = (I - R2(M)) M^-1 D^-1 b, where
    M = D^-1 A and R2(t) = T2((theta - t)/delta) / T2(theta/delta) is the
    residual polynomial of degree 2 on [lo, hi] (dense check)."""
    mesh, p, o = hierarchy_case("c8")
    q = Oracle(mesh, dict(p, smoother=2, smooth_sweeps=2))
    q.begin_frame()
    q.eval_assemble()
    q.prepare_solve()
    _, _, _, A = csr_of(q, 0)
    Ad = A.toarray()
    d = np.diag(Ad)
    lmax, _ = q.level_omega(0)
    lo, hi = p["lambda_min_est"], p["power_safety"] * lmax
    th, de = (hi + lo) / 2, (hi - lo) / 2
    M = Ad / d[:, None]
    I = np.eye(len(d))
    Z = (th * I - M) / de
    R2 = (2 * Z @ Z - I) / (2 * (th / de) ** 2 - 1)
    b = np.random.default_rng(9).standard_normal(mesh.n_rows)
    x_ref = np.linalg.solve(M, (I - R2) @ (b / d))
    x = q.smooth(0, b)
    assert np.allclose(x, x_ref, rtol=1e-9, atol=1e-12 * np.abs(x_ref).max())


def test_one_level_hierarchy_converges_in_one_iteration():
    mesh = cloth(6, plane="xz", alpha=1e-6, pin="corners", noise=1e-3, seed=3)
    p = default_params(coarse_max=10 ** 6, pcg_rtol=1e-10)
    o = Oracle(mesh, p)
    o.begin_frame()
    o.eval_assemble()
    o.prepare_solve()
    assert o.levels == 1
    b = np.random.default_rng(0).standard_normal(mesh.n_rows)
    x, info = o.solve(b)
    assert info["pcg_iters"] == 1 and info["status"] == 0


def test_zero_rhs_returns_zero():
    mesh, p, o = hierarchy_case("c8")
    x, info = o.solve(np.zeros(mesh.n_rows))
    assert np.all(x == 0) and info["pcg_iters"] == 0 and info["bnorm"] == 0


def test_residual_falls_to_tolerance():
    mesh, p, o = hierarchy_case("h3")  # stiff: cond(A) ~ 1e8
    b = np.random.default_rng(5).standard_normal(mesh.n_rows)
    x, info = o.solve(b)
    assert info["status"] == 0 and info["rel_res"] <= p["pcg_rtol"]
    # the true residual lags the recursive one by about cond * eps
    assert info["true_rel_res"] <= 1e-6


# --------------------------------------------------------------------------
# whole iterations (Alg. 1)
# --------------------------------------------------------------------------

def test_pinned_vertices_stay_and_dual_residual_falls():
    mesh = cloth(12, plane="xz", alpha=1e-8, pin="corners", noise=1e-4, seed=1)
    p = default_params(omega_x=0.25, max_iter=20, pcg_maxiter=100, coarse_max=60)
    o = Oracle(mesh, p)
    st, hist = o.step(2)
    assert st == 0
    x, v = o.get_state()
    pinned = mesh.inv_mass == 0
    assert np.array_equal(x[pinned], mesh.rest_pos[pinned])
    assert np.all(v[pinned] == 0)
    for f in range(2):
        b = [h["bnorm"] for h in hist[f * 20:(f + 1) * 20]]
        assert b[-1] < b[0]  # relative dual residual falls over the loop


def test_backtracking_never_accepts_a_growing_residual_when_a_halving_helps():
    mesh = cloth(10, plane="xz", alpha=1e-8, pin="corners", noise=1e-4, seed=1)
    p = default_params(omega_x=1.0, backtrack=8, pcg_rtol=1e-10, coarse_max=40)
    o = Oracle(mesh, p)
    o.begin_frame()
    for _ in range(6):
        d = o.iterate()
        assert d["ret"] == 0
        halvings = round(np.log2(1.0 / d["omega"]))
        assert d["omega"] == 2.0 ** -halvings
        if halvings < p["backtrack"]:
            assert d["bnorm_after"] < d["bnorm"]
    # each trial re-evaluated in a second instance (state before the iteration
    # plus omega dx, lambda after it): the accepted omega is the first of
    # omega_x, omega_x/2, ... whose trial lowers |b|
    o = Oracle(mesh, p)
    probe = Oracle(mesh, p)
    o.begin_frame()
    accepted = []
    for _ in range(6):
        x0, v0 = o.get_state()
        d = o.iterate()
        x1, _ = o.get_state()
        lam1, _ = o.lam()
        om = d["omega"]
        accepted.append(om)
        dx = (x1 - x0) / om
        trial = p["omega_x"]
        while True:
            probe.set_state(x0 + trial * dx, v0)
            probe.set_lambda(lam1)
            probe.eval_assemble()
            ratio = np.linalg.norm(probe.constraints()[1]) / d["bnorm"]
            if trial == om:
                assert ratio < 1.0
                break
            assert ratio >= 1.0, (trial, om, ratio)
            trial /= 2
    assert max(accepted) == p["omega_x"] and min(accepted) < p["omega_x"]  # both cases met
    # fixed relaxation leaves omega untouched and reports no trial residual
    o2 = Oracle(mesh, default_params(omega_x=0.25, coarse_max=40))
    o2.begin_frame()
    d = o2.iterate()
    assert d["omega"] == 0.25 and d["bnorm_after"] == -1.0


def test_xpbd_step_is_the_diagonal_solve_and_stalls_where_mgpcg_does_not():
    # eq. 4 on a single constraint is exact, like the global solve
    rest = np.array([[0, 0, 0], [1, 0, 0]], float)
    x0 = np.array([[0, 0, 0], [1.3, 0.1, -0.2]], float)
    one = Mesh("one", rest, np.array([0.5, 2.0]), np.array([[0, 1]], np.int32),
               np.zeros((0, 4), np.int32), np.array([1e-3]), x0, np.zeros((2, 3)))
    outs = []
    for solver in (0, 1):
        o = Oracle(one, default_params(gravity=(0.0, 0.0, 0.0), omega_x=1.0, max_iter=1,
                                       linear_solver=solver))
        o.step(1)
        outs.append(o.get_state()[0])
    assert np.allclose(outs[0], outs[1], rtol=0, atol=1e-15)
    # on a stiff cloth the local solve leaves a larger dual residual than the
    # global one after the same number of iterations (Sec. 5.4, cloth and bunny)
    mesh = cloth(16, plane="xz", alpha=1e-8, pin="corners", noise=1e-4, seed=1)
    res = []
    for solver in (0, 1):
        o = Oracle(mesh, default_params(omega_x=0.25, max_iter=20, coarse_max=60,
                                        linear_solver=solver))
        o.begin_frame()
        hist = [o.iterate()["bnorm"] for _ in range(20)]
        res.append(hist[-1] / hist[0])
    assert res[0] < 0.5 * res[1]


def test_lazy_setup_count():
    mesh = cloth(8, plane="xz", alpha=1e-8, pin="corners", noise=1e-4, seed=1)
    p = default_params(max_iter=5, setup_interval=7, coarse_max=20, pcg_maxiter=50)
    o = Oracle(mesh, p)
    st, _ = o.step(3)  # 15 global iterations -> setups at 0, 7, 14
    assert st == 0 and o.n_setups == 3
