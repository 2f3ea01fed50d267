"""A small case of the benchmark recipe for ncu captures.

Builds a hex block of the bench recipe (0.005 m cells, 10% jitter, 5 tets
per cell, alpha = 1e-10, bottom face pinned), runs the frame prologue, one
evaluation/assembly, the AMG setup and one MGPCG solve capped at a few
iterations, then exits 0.  Usage:

    python -m paper_2505_13390_gb300.profile_case 40x33x40 PREC PCG_ITERS AUTOTUNE [OP]

PREC is 1 for mixed precision, 0 for FP64; OP is 1 for the matrix-free
level-0 operator, 0 (default) for the assembled CSR matrix.
"""
import sys

import torch

from .meshgen import default_params, hex_block
from .mgpbd import Solver


def main(argv):
    a, b, c = (int(s) for s in argv[0].split("x"))
    prec, iters = int(argv[1]), int(argv[2])
    tune = int(argv[3]) if len(argv) > 3 else 0
    op = int(argv[4]) if len(argv) > 4 else 0
    mesh = hex_block(a, b, c, h=0.005, jitter=0.1, alpha=1e-10, pin="y0", seed=1)
    p = default_params(omega_x=0.1, precision=prec, pcg_maxiter=iters, autotune=tune,
                       level0_op=op)
    g = Solver(mesh, p)
    g.begin_frame()
    g.eval_assemble()
    g.prepare_solve()
    rhs = torch.from_numpy(g.constraints()[1]).cuda()
    _, info = g.solve(rhs)
    torch.cuda.synchronize()
    print("ok", info, g.level_info(0))


if __name__ == "__main__":
    main(sys.argv[1:])
