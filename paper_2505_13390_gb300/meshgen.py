"""Seeded synthetic workloads for the global XPBD solve.

This module builds the problem inputs only: vertex positions, inverse masses,
distance pairs, tetrahedra, per-row compliance and the run parameters. It
holds none of the solver's arithmetic (no constraint, gradient, matrix or
multigrid computation), so both the CUDA path and the CPU oracle can take
their inputs from here.

The paper's meshes (bunny, ball, muscle-human, monster, armadillo, twist-bar;
Table 1) are not available, so every workload is a regular lattice with the
sizes and value distributions below:

* ``cloth32``   32x32 cloth in the x-z plane, 0.01 m spacing, structural and
  one shear diagonal per quad (2,945 distance rows), unit mass, alpha = 1e-8,
  corners (0,0) and (31,0) pinned, free vertices start at rest + U(+-1e-4).
* ``beam40``    40x10x10 hex cells of 0.01 m, 5 tets per cell (20,000 tets,
  4,961 vertices, 26,760 unique tet edges), lumped mass from density 1000,
  alpha = 1e-9, the x = 0 face pinned.
* ``cloth512``  512x512 cloth in the x-y plane with structural, shear and bend
  edges (1,306,625 rows), per-row alpha = 10^U(-10,-6), top row pinned.
* ``block100``  100x33x100 hex cells (33 cells on the vertical y axis) of
  0.005 m, every vertex jittered by U(+-10% h) per coordinate, 5 tets per cell
  (1.65M tets, 346,834 vertices, 2,030,033 edges), alpha = 1e-10, the bottom
  face pinned.
* serving requests: cloth N x N with N ~ U{16..256} or beam L x 10 x 10 with
  L ~ U{10..80}, alpha per instance 10^U(-9,-6), Poisson arrivals.

Masses of tet meshes are lumped from the nominal (unjittered) cell geometry:
a cell of side h splits into one central tet of volume h^3/3 and four corner
tets of volume h^3/6, and each tet gives a quarter of rho*V to each vertex.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Tuple

import numpy as np

GRAVITY = (0.0, -9.8, 0.0)
DT = 1.0 / 60.0


@dataclasses.dataclass
class Mesh:
    """A constraint mesh: rows are all distance pairs, then all tetrahedra."""

    name: str
    rest_pos: np.ndarray  # (N, 3) float64, rest shape
    inv_mass: np.ndarray  # (N,) float64, 0 = pinned
    dist: np.ndarray  # (E, 2) int32
    tet: np.ndarray  # (T, 4) int32, positively oriented at rest
    alpha: np.ndarray  # (E + T,) float64 compliance per row
    x0: np.ndarray  # (N, 3) float64 initial positions
    v0: np.ndarray  # (N, 3) float64 initial velocities
    tet_kind: int = 0  # tet rows: 0 volume C = V - V0, 1 ARAP C = |F - R|_F^2 (Sec. 5.3)

    @property
    def n_verts(self) -> int:
        return int(self.rest_pos.shape[0])

    @property
    def n_dist(self) -> int:
        return int(self.dist.shape[0])

    @property
    def n_tet(self) -> int:
        return int(self.tet.shape[0])

    @property
    def n_rows(self) -> int:
        return self.n_dist + self.n_tet


def default_params(**over) -> Dict:
    """Solver parameters with the paper's defaults (see DESIGN notes).

    theta_s = 0.1 (Sec. 4.1), two smoothing sweeps (Sec. 4.5), lambda_min
    estimate 0.1 (Sec. 4.5), coarsest size below 400 (Sec. 4.1),
    omega_x = 0.25 cloth / 0.1 softbody (Sec. 4, Alg. 1 relaxation).
    """
    p = dict(
        dt=DT,
        gravity=GRAVITY,
        omega_x=0.25,
        max_iter=20,
        eps_b=0.0,
        pcg_rtol=1e-6,
        pcg_maxiter=20000,  # a safeguard: the solve runs to pcg_rtol
        setup_interval=400,
        nk_sweeps=3,
        nk_vectors=1,  # near-kernel vectors k = columns of P per aggregate (Sec. 4.3)
        nk_omega=2.0 / 3.0,
        theta_s=0.1,
        smoother=0,  # 0 = weighted Jacobi, 1 = multicolour Gauss-Seidel
        smooth_sweeps=2,
        lambda_min_est=0.1,
        power_iters=15,
        power_safety=1.25,
        coarse_max=400,
        max_levels=8,
        backtrack=0,  # 0: fixed omega_x; k: halve omega up to k times while |b| grows
        autotune=0,   # 1: time the row-kernel shapes at setup and keep the fastest
        level0_op=0,  # 1: matrix-free level-0 products through the constraint gradients
        use_graphs=0,  # 1: replay PCG iteration chunks from a captured CUDA graph
        linear_solver=0,  # 0: MGPCG; 1: XPBD's diagonal step (eq. 4), the baseline
        precision=0,  # 0 = FP64, 1 = mixed (FP32 V-cycle, FP64 recurrences)
        ap_split=0,  # 1: the recurrence's A.p from float-float pairs (mixed, matrix-free)
        seed_nk=3,
        seed_agg=4,
        seed_col=5,
        seed_pow=7,
        frames=10,
    )
    p.update(over)
    return p


# ----------------------------------------------------------------------------
# cloth
# ----------------------------------------------------------------------------

def _cloth_edges(n: int, bend: bool) -> np.ndarray:
    """Edges of an n x n grid, vertex (i, j) -> j*n + i.

    Order: (i,j)-(i+1,j) for all j, i; then (i,j)-(i,j+1); then the shear
    diagonal (i,j)-(i+1,j+1); with ``bend`` also (i,j)-(i+2,j) and (i,j)-(i,j+2).
    """
    idx = np.arange(n * n, dtype=np.int64).reshape(n, n)  # [j, i]
    parts = [
        np.stack([idx[:, :-1].ravel(), idx[:, 1:].ravel()], 1),
        np.stack([idx[:-1, :].ravel(), idx[1:, :].ravel()], 1),
        np.stack([idx[:-1, :-1].ravel(), idx[1:, 1:].ravel()], 1),
    ]
    if bend:
        parts.append(np.stack([idx[:, :-2].ravel(), idx[:, 2:].ravel()], 1))
        parts.append(np.stack([idx[:-2, :].ravel(), idx[2:, :].ravel()], 1))
    return np.concatenate(parts, 0).astype(np.int32)


def cloth(n: int, *, h: float = 0.01, plane: str = "xz", bend: bool = False,
          alpha=1e-8, alpha_log_range=None, pin: str = "corners",
          noise: float = 1e-4, seed: int = 1, name: str = "cloth") -> Mesh:
    rng = np.random.default_rng(seed)
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    pos = np.zeros((n * n, 3))
    if plane == "xz":
        pos[:, 0] = (ii * h).ravel()
        pos[:, 2] = (jj * h).ravel()
    else:  # "xy": j runs up the y axis
        pos[:, 0] = (ii * h).ravel()
        pos[:, 1] = (jj * h).ravel()
    inv_mass = np.ones(n * n)
    if pin == "corners":
        inv_mass[0] = 0.0
        inv_mass[n - 1] = 0.0
    elif pin == "top":
        inv_mass[(n - 1) * n:] = 0.0
    dist = _cloth_edges(n, bend)
    m = dist.shape[0]
    arng = np.random.default_rng(seed + 1)
    if alpha_log_range is not None:
        lo, hi = alpha_log_range
        al = 10.0 ** arng.uniform(lo, hi, size=m)
    else:
        al = np.full(m, float(alpha))
    free = inv_mass > 0
    x0 = pos.copy()
    x0[free] += rng.uniform(-noise, noise, size=(int(free.sum()), 3))
    return Mesh(name, pos, inv_mass, dist, np.zeros((0, 4), np.int32), al,
                x0, np.zeros_like(pos))


# ----------------------------------------------------------------------------
# hex lattice split into 5 tets
# ----------------------------------------------------------------------------

_CORNERS = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 0),
            (0, 0, 1), (1, 0, 1), (0, 1, 1), (1, 1, 1)]


def _tet_templates() -> Tuple[List[List[Tuple[int, int, int]]], List[List[Tuple[int, int, int]]]]:
    """Local corner lists of the 5-tet split for even and odd cells.

    Even cell: central tet on the even corners {000,110,101,011}; one corner
    tet per odd corner, made of that corner and its three axis neighbours.
    Odd cell: mirrored (central tet on the odd corners).  Every face diagonal
    then joins globally even vertices, so neighbouring cells conform.
    Each tet is ordered so that its signed lattice volume is positive.
    """
    def par(c):
        return (c[0] + c[1] + c[2]) & 1

    def nb(c):
        return [(c[0] ^ 1, c[1], c[2]), (c[0], c[1] ^ 1, c[2]), (c[0], c[1], c[2] ^ 1)]

    def orient(t):
        a, b, c, d = [np.array(v, dtype=np.int64) for v in t]
        det = int(np.round(np.linalg.det(np.stack([b - a, c - a, d - a]).astype(float))))
        assert det != 0
        return t if det > 0 else [t[0], t[2], t[1], t[3]]

    out = []
    for cell_par in (0, 1):
        centre = [c for c in _CORNERS if par(c) == cell_par]
        tips = [c for c in _CORNERS if par(c) != cell_par]
        tets = [orient(centre)] + [orient([t] + nb(t)) for t in tips]
        out.append(tets)
    return out[0], out[1]


def hex_block(nx: int, ny: int, nz: int, *, h: float, rho: float = 1000.0,
              jitter: float = 0.0, alpha=1e-9, alpha_log_range=None,
              pin: str = "x0", seed: int = 1, name: str = "block",
              arap_mu: Optional[float] = None) -> Mesh:
    """Hex lattice of nx*ny*nz cells split into 5 tets per cell.

    Vertex (i,j,k) -> (i*(ny+1) + j)*(nz+1) + k.  Rows: unique tet edges
    sorted by (min, max) vertex, then tets in cell order (i, j, k), each cell
    giving its central tet first.  With arap_mu set, the rows are one ARAP
    constraint per tet and nothing else, with compliance 1/(mu V_tet) from
    the rest volume (Sec. 5.3).
    """
    vx, vy, vz = nx + 1, ny + 1, nz + 1
    n = vx * vy * vz
    I, J, K = np.meshgrid(np.arange(vx), np.arange(vy), np.arange(vz), indexing="ij")
    pos = np.stack([I.ravel() * h, J.ravel() * h, K.ravel() * h], 1).astype(np.float64)
    if jitter > 0:
        rng = np.random.default_rng(seed)
        pos = pos + rng.uniform(-jitter * h, jitter * h, size=pos.shape)

    even_t, odd_t = _tet_templates()
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    parity = (ci + cj + ck) & 1
    n_cells = ci.size
    tets = np.zeros((n_cells, 5, 4), np.int64)
    vols = np.zeros((n_cells, 5))
    for par, templ in ((0, even_t), (1, odd_t)):
        sel = parity == par
        for t, corners in enumerate(templ):
            for s, (dx, dy, dz) in enumerate(corners):
                tets[sel, t, s] = ((ci[sel] + dx) * vy + (cj[sel] + dy)) * vz + (ck[sel] + dz)
            vols[sel, t] = h ** 3 / 3.0 if t == 0 else h ** 3 / 6.0
    tets = tets.reshape(-1, 4)
    vols = vols.reshape(-1)

    mass = np.zeros(n)
    for s in range(4):
        np.add.at(mass, tets[:, s], rho * vols / 4.0)

    pairs = np.concatenate([tets[:, [a, b]] for a in range(4) for b in range(a + 1, 4)], 0)
    pairs = np.sort(pairs, axis=1)
    key = np.unique(pairs[:, 0] * n + pairs[:, 1])
    dist = np.stack([key // n, key % n], 1).astype(np.int32)

    inv_mass = 1.0 / mass
    if pin == "x0":
        inv_mass[I.ravel() == 0] = 0.0
    elif pin == "y0":
        inv_mass[J.ravel() == 0] = 0.0

    if arap_mu is not None:
        p = pos[tets]
        e = p[:, 1:, :] - p[:, :1, :]
        v_rest = np.abs(np.linalg.det(e)) / 6.0
        return Mesh(name, pos, inv_mass, np.zeros((0, 2), np.int32), tets.astype(np.int32),
                    1.0 / (float(arap_mu) * v_rest), pos.copy(), np.zeros_like(pos), tet_kind=1)
    m = dist.shape[0] + tets.shape[0]
    if alpha_log_range is not None:
        arng = np.random.default_rng(seed + 1)
        al = np.full(m, 10.0 ** arng.uniform(*alpha_log_range))
    else:
        al = np.full(m, float(alpha))
    return Mesh(name, pos, inv_mass, dist, tets.astype(np.int32), al,
                pos.copy(), np.zeros_like(pos))


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def workload(name: str) -> Tuple[Mesh, Dict]:
    """Return (mesh, params) for a named workload."""
    if name == "cloth32":
        mesh = cloth(32, plane="xz", alpha=1e-8, pin="corners", noise=1e-4, seed=1,
                     name=name)
        params = default_params(omega_x=0.25, max_levels=2, frames=10)
    elif name == "beam40":
        mesh = hex_block(40, 10, 10, h=0.01, alpha=1e-9, pin="x0", seed=1, name=name)
        params = default_params(omega_x=0.1, setup_interval=10, frames=30)
    elif name == "cloth512":
        mesh = cloth(512, plane="xy", bend=True, alpha_log_range=(-10, -6), pin="top",
                     noise=1e-4, seed=1, name=name)
        params = default_params(omega_x=0.25, frames=10)
    elif name == "block100":
        mesh = hex_block(100, 33, 100, h=0.005, jitter=0.1, alpha=1e-10, pin="y0",
                         seed=1, name=name)
        params = default_params(omega_x=0.1, setup_interval=20, frames=1,
                                precision=1)
    elif name == "block100arap":
        # the block100 lattice with one ARAP row per tet (Sec. 5.3), mu = 1e7 Pa
        mesh = hex_block(100, 33, 100, h=0.005, jitter=0.1, arap_mu=1e7, pin="y0", seed=1,
                         name=name)
        params = default_params(omega_x=0.1, setup_interval=20, frames=1, precision=1)
    elif name == "beam40arap":
        mesh = hex_block(40, 10, 10, h=0.01, arap_mu=1e7, pin="x0", seed=1, name=name)
        params = default_params(omega_x=0.1, setup_interval=10, frames=30)
    elif name.startswith("cloth") and name[5:].isdigit():
        n = int(name[5:])
        mesh = cloth(n, plane="xz", alpha=1e-8, pin="corners", seed=1, name=name)
        params = default_params(omega_x=0.25)
    elif name.startswith("beam") and name[4:].isdigit():
        L = int(name[4:])
        mesh = hex_block(L, 10, 10, h=0.01, alpha=1e-9, pin="x0", seed=1, name=name)
        params = default_params(omega_x=0.1)
    elif name.startswith("block") and "x" in name:
        # blockAxBxC: small lattices of the block100 recipe for tests
        a, b, c = (int(s) for s in name[5:].split("x"))
        mesh = hex_block(a, b, c, h=0.005, jitter=0.1, alpha=1e-10, pin="y0", seed=1,
                         name=name)
        params = default_params(omega_x=0.1, setup_interval=20)
    else:
        raise KeyError(name)
    return mesh, params


def serving_trace(n_requests: int = 512, n_instances: int = 64, rate_hz: float = 2.0,
                  seed: int = 6) -> Tuple[List[Dict], List[Dict]]:
    """Seeded serving trace: instances and step requests.

    Instances: with probability 1/2 a cloth of N x N (N ~ U{16..256}), else a
    tet beam of L x 10 x 10 cells (L ~ U{10..80}); alpha = 10^U(-9, -6).
    Requests: Poisson arrivals at `rate_hz`; each is one step (one frame of
    20 global iterations) of an instance drawn uniformly; an instance's state
    persists between its requests.
    """
    rng = np.random.default_rng(seed)
    inst = []
    for k in range(n_instances):
        log_a = rng.uniform(-9.0, -6.0)
        if rng.uniform() < 0.5:
            inst.append(dict(kind="cloth", size=int(rng.integers(16, 257)),
                             alpha=10.0 ** log_a, seed=1000 + k))
        else:
            inst.append(dict(kind="beam", size=int(rng.integers(10, 81)),
                             alpha=10.0 ** log_a, seed=1000 + k))
    t = 0.0
    reqs = []
    for r in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        reqs.append(dict(id=r, t=t, instance=int(rng.integers(0, n_instances)), frames=1))
    return inst, reqs


def instance_mesh(req: Dict) -> Tuple[Mesh, Dict]:
    if req["kind"] == "cloth":
        mesh = cloth(req["size"], plane="xz", alpha=req["alpha"], pin="corners",
                     seed=req["seed"], name=f"cloth{req['size']}")
        return mesh, default_params(omega_x=0.25, frames=10)
    mesh = hex_block(req["size"], 10, 10, h=0.01, alpha=req["alpha"], pin="x0",
                     seed=req["seed"], name=f"beam{req['size']}")
    return mesh, default_params(omega_x=0.1, frames=10)
