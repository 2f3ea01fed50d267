"""Small cases of the benchmark's kernels for ncu captures.

    python -m paper_2505_13390_gb300.profile_case AxBxC PREC PCG_ITERS [AUTOTUNE [OP [SPLIT]]]

builds a hex block of the bench recipe (0.005 m cells, 10% jitter, 5 tets
per cell, alpha = 1e-10, bottom face pinned), runs the frame prologue, one
evaluation/assembly, the AMG setup and one MGPCG solve capped at PCG_ITERS
iterations, then exits 0.  PREC is 1 for mixed precision, 0 for FP64; OP is
1 for the matrix-free level-0 operator, 0 (default) for the assembled CSR
matrix; SPLIT 1 takes the recurrence's A.p from float-float pairs (needs PREC
1 and OP 1).

    python -m paper_2505_13390_gb300.profile_case chainN [REPEATS]

factorises the coarsest level of a one-level hierarchy of N rows (a chain of
distance rows) REPEATS times (default 5): the tiled Cholesky and inverse.

    python -m paper_2505_13390_gb300.profile_case cohortK [FRAMES]

serves K beam instances of 40x10x10 cells (46,760 rows each) in cohort mode,
one request of FRAMES frames (default 1, two global iterations each) per
instance, all at once: the batched PCG kernels.
"""
import sys

import numpy as np
import torch

from .meshgen import Mesh, default_params, hex_block, instance_mesh
from .mgpbd import Batch, Solver


def block(argv):
    a, b, c = (int(s) for s in argv[0].split("x"))
    prec, iters = int(argv[1]), int(argv[2])
    tune = int(argv[3]) if len(argv) > 3 else 0
    op = int(argv[4]) if len(argv) > 4 else 0
    split = int(argv[5]) if len(argv) > 5 else 0
    mesh = hex_block(a, b, c, h=0.005, jitter=0.1, alpha=1e-10, pin="y0", seed=1)
    p = default_params(omega_x=0.1, precision=prec, pcg_maxiter=iters, autotune=tune,
                       level0_op=op, ap_split=split)
    g = Solver(mesh, p)
    g.begin_frame()
    g.eval_assemble()
    g.prepare_solve()
    rhs = torch.from_numpy(g.constraints()[1]).cuda()
    _, info = g.solve(rhs)
    torch.cuda.synchronize()
    print("ok", info, g.level_info(0))


def chain(argv):
    n = int(argv[0][5:])
    reps = int(argv[1]) if len(argv) > 1 else 5
    nv = n + 1
    rest = np.zeros((nv, 3))
    rest[:, 0] = 0.01 * np.arange(nv)
    edges = np.stack([np.arange(n), np.arange(1, nv)], 1).astype(np.int32)
    x0 = rest.copy()
    x0[:, 0] *= 1.001
    mesh = Mesh("chain", rest, np.ones(nv), edges, np.zeros((0, 4), np.int32),
                np.full(n, 1e-6), x0, np.zeros((nv, 3)))
    g = Solver(mesh, default_params(coarse_max=4000, gravity=(0.0, 0.0, 0.0)))
    g.begin_frame()
    g.eval_assemble()
    for _ in range(reps):
        g.prepare_solve()
    torch.cuda.synchronize()
    print("ok", g.levels, g.level_info(0)["n"])


def cohort(argv):
    k = int(argv[0][6:])
    frames = int(argv[1]) if len(argv) > 1 else 1
    ms = [instance_mesh(dict(kind="beam", size=40, alpha=1e-8, seed=2000 + i)) for i in range(k)]
    b = Batch(64 << 30, max(1, min(k, 64)), cohort=True)
    ids = [b.add(m, dict(p, precision=1, level0_op=1, use_graphs=1, autotune=0, max_iter=2))
           for m, p in ms]
    st, res = b.run([(i, ids[i], frames, 0.0) for i in range(k)])
    print("ok", st, b.cohort_stats(), sum(r["pcg_iters"] for r in res))
    b.close()
    if st < 0:
        raise SystemExit(1)


def main(argv):
    if argv[0].startswith("chain"):
        chain(argv)
    elif argv[0].startswith("cohort"):
        cohort(argv)
    else:
        block(argv)


if __name__ == "__main__":
    main(sys.argv[1:])
