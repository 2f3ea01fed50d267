"""The N-GPU bench path (replicas, no data-path collective) on CPU: two gloo
ranks run bench.py's process-group set-up, barrier and max-over-ranks timing."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(ws), MGPBD_DIST_BACKEND="gloo")
    import bench
    import torch.distributed as dist

    class A:
        pass

    got_ws, got_rank, _ = bench.dist_init(A())
    assert dist.get_backend() == "gloo"
    bench.barrier(got_ws)
    # rank r "took" 1000*(r+1) ms for 3 steps: the job takes the slowest rank
    rate, ms = bench.job_rate(got_ws, 3, 1000.0 * (rank + 1))
    out[rank] = (got_ws, got_rank, rate, ms)
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_replica_ranks_gloo():
    ws = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    for r in range(ws):
        got_ws, got_rank, rate, ms = out[r]
        assert (got_ws, got_rank) == (ws, r)
        assert ms == 2000.0  # max over ranks
        assert rate == pytest.approx(ws * 3 / 2.0)  # whole-job iterations per second


@pytest.mark.timeout(300)
def test_reference_arm_under_two_ranks_prints_once():
    """bench.py --impl reference under torch.distributed.run with two gloo
    ranks: rank 0 alone times the oracle and prints one JSON line; the other
    rank exits 0 without work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, MGPBD_DIST_BACKEND="gloo", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                        "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                        "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
                        "--steps", "1", "--warmup", "0"],
                       cwd=root, env=env, capture_output=True, text=True, timeout=280)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
