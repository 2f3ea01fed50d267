"""Pins of the oracle's ARAP constraint (Sec. 5.3): C = |F - R|_F^2.

F = Ds Dm^-1 is the deformation gradient of a tetrahedron and R the rotation
of its polar decomposition F = R S.  The pins use what the mathematics fixes:
for F = Q S built from a known rotation Q and a known symmetric positive
definite S, C = |S - I|_F^2 and dC/dDs = 2 (F - Q) Dm^-T; rigid motions cost
nothing; the gradient matches central finite differences; and the compliance
of the generated meshes is 1/(mu V_tet).
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2505_13390_gb300.meshgen import Mesh, default_params, hex_block


def params(**kw):
    p = default_params(coarse_max=4, max_levels=8, pcg_rtol=1e-12, pcg_maxiter=500)
    p.update(kw)
    return p


def rotation(axis, angle):
    a = np.asarray(axis, float)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K


def one_tet(F, rest=None):
    """A single ARAP tet whose current edge matrix is F Dm."""
    if rest is None:
        rest = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    Dm = (rest[1:] - rest[0]).T
    Ds = F @ Dm
    x = np.vstack([rest[0], rest[0] + Ds.T])
    mesh = Mesh("arap1", rest, np.ones(4), np.zeros((0, 2), np.int32),
                np.array([[0, 1, 2, 3]], np.int32), np.array([1e-6]), x, np.zeros((4, 3)),
                tet_kind=1)
    o = Oracle(mesh, params())
    o.eval_assemble()
    Cv, _, _, gt = o.constraints()
    return Cv[0], gt[0], Dm


def test_polar_factor_closed_form():
    Q = rotation([1.0, 2.0, -0.5], 0.7)
    S = np.array([[1.2, 0.05, -0.02], [0.05, 0.9, 0.03], [-0.02, 0.03, 1.05]])
    F = Q @ S
    C, g, Dm = one_tet(F)
    assert C == pytest.approx(np.sum((S - np.eye(3)) ** 2), rel=1e-12)
    G = 2.0 * (F - Q) @ np.linalg.inv(Dm).T
    assert np.allclose(g[1:], G.T, rtol=0, atol=1e-12)
    assert np.allclose(g[0], -G.sum(axis=1), rtol=0, atol=1e-12)


def test_polar_factor_on_a_skewed_rest_shape():
    rest = np.array([[0.1, -0.2, 0.05], [1.3, 0.1, -0.1], [0.2, 0.9, 0.3], [-0.1, 0.2, 1.4]])
    Q = rotation([0.0, 0.0, 1.0], -1.2)
    S = np.diag([0.8, 1.1, 1.3])
    C, g, Dm = one_tet(Q @ S, rest)
    assert C == pytest.approx(0.04 + 0.01 + 0.09, rel=1e-12)
    G = 2.0 * (Q @ S - Q) @ np.linalg.inv(Dm).T
    assert np.allclose(g[1:], G.T, rtol=0, atol=1e-11)


def test_uniaxial_stretch():
    s = 1.3
    C, g, _ = one_tet(np.diag([s, 1.0, 1.0]))
    assert C == pytest.approx((s - 1) ** 2, rel=1e-14)
    assert np.allclose(g[1], [2 * (s - 1), 0, 0], atol=1e-14)
    assert np.allclose(g[2:], 0.0, atol=1e-14)
    assert np.allclose(g[0], [-2 * (s - 1), 0, 0], atol=1e-14)


def test_singular_and_reflected_deformations():
    # a flattened tet has no unique polar factor: C = 0 and no gradient
    C, g, _ = one_tet(np.diag([1.0, 1.0, 0.0]))
    assert C == 0.0 and np.all(g == 0.0)
    # an inverted tet: the orthogonal polar factor is the reflection itself
    C, g, _ = one_tet(np.diag([-1.0, 1.0, 1.0]))
    assert C == pytest.approx(0.0, abs=1e-28)


def test_rest_and_rigid_motions_are_free():
    mesh = hex_block(3, 2, 2, h=0.01, jitter=0.1, arap_mu=1e6, pin="x0", seed=4)
    o = Oracle(mesh, params())
    o.eval_assemble()
    Cv, _, _, gt = o.constraints()
    assert np.abs(Cv).max() <= 1e-28 and np.abs(gt).max() <= 1e-12
    Q = rotation([0.3, -1.0, 0.4], 2.1)
    x = mesh.rest_pos @ Q.T + np.array([0.2, -0.1, 0.3])
    o.set_state(x, mesh.v0)
    o.eval_assemble()
    Cv, _, _, gt = o.constraints()
    assert np.abs(Cv).max() <= 1e-26 and np.abs(gt).max() <= 1e-11


def test_gradient_matches_finite_differences():
    mesh = hex_block(2, 1, 1, h=0.01, jitter=0.1, arap_mu=1e6, pin="x0", seed=4)
    rng = np.random.default_rng(5)
    x = mesh.rest_pos + rng.uniform(-1.5e-3, 1.5e-3, mesh.rest_pos.shape)
    o = Oracle(mesh, params())
    o.set_state(x, mesh.v0)
    o.eval_assemble()
    _, _, _, gt = o.constraints()
    J = np.zeros((mesh.n_tet, x.size))
    for t, verts in enumerate(mesh.tet.tolist()):
        for s, v in enumerate(verts):
            J[t, 3 * v:3 * v + 3] += gt[t, s]
    h = 1e-7
    Jfd = np.zeros_like(J)
    for q in range(x.size):
        xp, xm = x.copy().ravel(), x.copy().ravel()
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
    assert np.all(np.abs(J - Jfd) <= 1e-6 * scale + 1e-10)


def test_compliance_is_one_over_mu_v():
    mu = 2.5e5
    mesh = hex_block(2, 2, 1, h=0.01, jitter=0.1, arap_mu=mu, pin="x0", seed=7)
    o = Oracle(mesh, params())
    _, V0 = o.rest()
    assert np.allclose(mesh.alpha, 1.0 / (mu * V0), rtol=1e-12)
    assert mesh.n_dist == 0 and mesh.tet_kind == 1


def test_arap_block_sags_and_the_residual_falls():
    mesh = hex_block(8, 3, 3, h=0.01, jitter=0.1, arap_mu=1e6, pin="x0", seed=2)
    o = Oracle(mesh, default_params(omega_x=0.1, pcg_rtol=1e-6, setup_interval=10))
    o.begin_frame()
    b = []
    for _ in range(5):
        d = o.iterate()
        assert d["ret"] == 0 and d["true_rel_res"] <= 1e-5
        b.append(d["bnorm"])
    assert all(b1 < b0 for b0, b1 in zip(b, b[1:]))
    o.end_frame()
    x, _ = o.get_state()
    free = mesh.inv_mass > 0
    assert np.all(x[free, 1] < mesh.rest_pos[free, 1])  # everything free moved down


def test_breakdown_on_a_reused_hierarchy_sets_up_again():
    # from rest most ARAP rows have no gradient, so the first hierarchy and
    # omega fit a nearly diagonal A; once the block deforms, a reused
    # hierarchy breaks PCG down and the iteration sets up afresh and retries
    mesh = hex_block(4, 12, 4, h=0.005, jitter=0.1, arap_mu=1e7, pin="y0", seed=1)
    o = Oracle(mesh, default_params(omega_x=0.1, setup_interval=4))
    o.begin_frame()
    infos = [o.iterate() for _ in range(4)]
    assert all(d["ret"] == 0 for d in infos)
    assert all(d["true_rel_res"] <= 1e-5 for d in infos)
    assert o.n_setups == 2  # the one due at iteration 0 and one after a breakdown
