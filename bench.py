"""Benchmark: global XPBD iterations per second of the MGPBD solve.

Workload (default): ``block100`` -- 100x33x100 hex cells of 0.005 m, 5 tets
per cell (1.65M tets, 346,834 vertices), edge distance plus tet volume
constraints (3,680,033 rows, 376,541,249 nonzeros in A), alpha = 1e-10,
bottom face pinned, dt = 1/60, 20 global iterations per frame, lazy setup
every 20 global iterations, PCG to rtol 1e-6 (about 7,000 PCG iterations per
global iteration on this workload).

A step is one global iteration of Algorithm 1 (constraints, assembly, lazy
setup when due, Galerkin re-form, coarsest factorisation, MGPCG with one
V-cycle per PCG iteration, dx/lambda/x update); the frame prologue and
epilogue fall inside the timed region at their natural rate (every 20
steps).  The headline `value` is the mixed-precision form; the FP64 form is
reported under "fp64".  Inputs are resident on the device; A alone is
3-4.6 GB, far larger than L2, so no L2 flush is needed between steps.

``--impl reference`` times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload (a 4x33x4-cell block of the same
recipe) and scales the time per iteration to the full workload by the
nonzero count of A and by the ratio of PCG iterations.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FULL_NNZ = 376_541_249  # nonzeros of A for block100 (checked at run time)
# PCG iterations of one block100 global iteration at PCG rtol 1e-6 as
# measured on GB300 (mixed precision, frame 0: 6,340-6,580 over the timed
# iterations).  Both CPU legs (the cpu_baseline of this arm and the
# reference arm, which cannot run the GPU) scale the oracle sample by this
# one number, so they agree.
FULL_PCG_ITERS = 6450
# DRAM bytes (read + write) of one level-0 FP32 smoother sweep per nonzero of
# A, from an ncu capture of k_jacobi<16, float> on a 40x33x40 block of the
# same recipe (494.52 MB for 59,625,809 nonzeros); the sweep's
# traffic grows in proportion to nnz, so it scales to a full launch
SWEEP_TRAFFIC_PER_NNZ = (489.342720e6 + 5.179904e6) / 59_625_809
# DRAM bytes of one matrix-free level-0 FP32 sweep (k_mf_vertex32<8> 30.74 MB
# + k_mf_row<float,0> 33.68 MB) per constraint row, from ncu captures of the
# two passes on a 40x33x40 block of the same recipe (593,633 rows); the passes
# stream per-row and per-incidence arrays, so traffic scales with the rows
MF_SWEEP_TRAFFIC_PER_ROW = (30.742016e6 + 33.679104e6) / 593_633
SAMPLE = (4, 33, 4)     # oracle sample: cells along x, y (vertical), z
SAMPLE_PCG = 500        # PCG iterations per sampled global iteration (cost is linear in them)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--fp64-warmup", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="block100")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-full", action="store_true",
                    help="also time beam40 on one oracle thread (about 3 minutes)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--level0-op", type=int, default=1,
                    help="1: matrix-free level-0 products (headline); 0: assembled CSR")
    ap.add_argument("--no-assembled", action="store_true",
                    help="skip the assembled-CSR comparison line")
    # the default run keeps the serving legs to a few minutes; the 64- and
    # 512-request traces and the other arms run with these flags
    ap.add_argument("--serve-requests", type=int, default=24,
                    help="step requests of the serving trace (the full trace has 512)")
    ap.add_argument("--serve-instances", type=int, default=24,
                    help="instances the requests draw from uniformly")
    ap.add_argument("--serve-rate", type=float, default=1.0, help="arrivals per second")
    ap.add_argument("--serve-active", type=int, default=8)
    ap.add_argument("--serve-arms", default="batched_streams,plain_fp64",
                    help="comma list of: " + ", ".join(SERVE_ARMS))
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the serving legs (e.g. --serve-requests 512) and print them")
    ap.add_argument("--no-serve-saturated", action="store_true",
                    help="skip the batched arms' run with every request at t = 0")
    ap.add_argument("--no-arap", action="store_true",
                    help="skip the ARAP-constraint leg (block100arap)")
    ap.add_argument("--no-xpbd", action="store_true",
                    help="skip the XPBD-versus-MGPBD frame on cloth512")
    ap.add_argument("--no-smoothers", action="store_true",
                    help="skip the Chebyshev-smoother leg on the same block")
    ap.add_argument("--smoother-steps", type=int, default=2)
    ap.add_argument("--smoother-warmup", type=int, default=2)
    ap.add_argument("--arap-steps", type=int, default=3)
    ap.add_argument("--arap-warmup", type=int, default=3)
    ap.add_argument("--assembled-steps", type=int, default=1)
    ap.add_argument("--assembled-warmup", type=int, default=1)
    ap.add_argument("--ap-split", type=int, default=0, choices=[0, 1],
                    help="the PCG recurrence's A.p from float-float pairs with residual "
                         "replacement (1) or in FP64 (0)")
    ap.add_argument("--ap-ab-steps", type=int, default=2)
    ap.add_argument("--ap-ab-warmup", type=int, default=1)
    ap.add_argument("--no-ap-ab", action="store_true",
                    help="skip the leg that times the headline with the other A.p form")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only: no collective on the data path)
# ---------------------------------------------------------------------------
def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = os.environ.get("MGPBD_DIST_BACKEND") or (
            "nccl" if torch.cuda.is_available() else "gloo")
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def job_rate(ws: int, steps: int, ms_local: float):
    """Whole-job global iterations/s of N replicas: every rank ran `steps`
    steps; the job takes as long as its slowest rank (max over ranks)."""
    ms = max_over_ranks(ws, ms_local)
    return ws * steps / (ms / 1e3), ms


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v: float) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.proc = None
        self.path = None
        self.uuid = uuid

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
class Runner:
    """Steps global iterations and keeps the frame bookkeeping of Alg. 1."""

    def __init__(self, solver, max_iter):
        self.g = solver
        self.max_iter = max_iter
        self.k = 0
        self.g.begin_frame()
        self.pcg = []
        self.true_res = []

    def step(self):
        d = self.g.iterate()
        self.pcg.append(d["pcg_iters"])
        self.true_res.append(d["true_rel_res"])
        self.k += 1
        if self.k % self.max_iter == 0:
            self.g.end_frame()
            self.g.begin_frame()
        return d


def _measured_hbm():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs")
    except Exception:
        return None


def hbm_peak() -> float:
    """Measured copy bandwidth (GB/s) of the GB300s, else 6,800 GB/s."""
    return _measured_hbm() or 6800.0


def ap_roofline(pr, split):
    """Live CUDA-event figures of the recurrence's A.p (one launch = its
    vertex and row pass) against the measured copy bandwidth."""
    if not pr or not pr["launches"]:
        return None
    avg = pr["total_ms"] / pr["launches"]
    ach = pr["bytes_per_launch"] / (avg / 1e3) / 1e9
    return {"form": "float-float pairs, FP64 residual replacement" if split else "FP64",
            "bound": "hbm", "achieved": ach, "peak": hbm_peak(), "unit": "GB/s",
            "frac": ach / hbm_peak(), "bytes_per_launch": pr["bytes_per_launch"],
            "avg_launch_ms": avg, "launches": pr["launches"]}


def measure(mesh, params, steps, warmup, ws, profile=True, profile_ap=False):
    import torch

    from paper_2505_13390_gb300.mgpbd import Solver, launch_count
    # a stream of our own: CUDA graphs cannot capture the legacy default stream
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    g = Solver(mesh, params, stream=stream)
    create_s = time.perf_counter() - t0
    run = Runner(g, params["max_iter"])
    for _ in range(warmup):
        run.step()
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    if profile:
        g.profile(True, ap=profile_ap)
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    clocks = Clocks(uuid)
    clocks.start()
    time.sleep(0.3)
    n0 = launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    pcg0 = len(run.pcg)
    ev0.record(stream)
    for _ in range(steps):
        run.step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    launches = launch_count() - n0
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = g.profile_read() if profile else None
    prof_ap = g.profile_read_ap() if profile and profile_ap else None
    if profile:
        g.profile(False)
    st = g.stats()
    out = dict(ms=ms, launches=launches, clocks=ck, prof=prof, prof_ap=prof_ap, stats=st,
               create_s=create_s,
               pcg=run.pcg[pcg0:], true_res=run.true_res[pcg0:], solver=g, runner=run)
    return out


def e2e(g, run, steps):
    """Same metric through the C ABI with host buffers: per step the state goes
    host->device from pinned memory, one global iteration runs, and the new
    positions and velocities come back device->host."""
    import numpy as np
    import torch

    x, v = g.get_state()
    xp = torch.from_numpy(x).pin_memory()
    vp = torch.from_numpy(v).pin_memory()
    xh, vh = xp.numpy(), vp.numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        g.set_state(xh, vh)  # MEM_HOST: synchronous H2D copies
        run.step()
        from paper_2505_13390_gb300 import mgpbd as M
        M._check(M.load().mgpbd_get_state(g.h, xh.ctypes.data, vh.ctypes.data, M.MEM_HOST),
                 "get_state")
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    nbytes = int(xh.nbytes + vh.nbytes)
    assert np.isfinite(xh).all()
    return steps / dt, nbytes


def serve_arm(meshes, reqs, prec, op, graphs, active, budget, cohort=False):
    """Serves the trace through the request loop: each request is admitted
    (mgpbd_batch_admit) when its arrival time has passed on the wall clock,
    results are collected with mgpbd_batch_tick.  Latency = finish - arrival
    on the batch's clock."""
    import numpy as np
    import torch

    from paper_2505_13390_gb300.mgpbd import Batch
    b = Batch(budget, active, cohort=cohort)
    for m, p in meshes:
        b.add(m, dict(p, precision=prec, level0_op=op, use_graphs=graphs, autotune=0,
                      setup_interval=20))
    torch.cuda.synchronize()
    pending = sorted(reqs, key=lambda r: r["t"])
    t0 = b.counts()["clock"]
    ticket_of, results, i = {}, {}, 0
    while len(results) < len(pending):
        now = b.counts()["clock"] - t0
        while i < len(pending) and pending[i]["t"] <= now:
            ticket_of[b.admit(pending[i]["instance"], pending[i]["frames"])] = pending[i]["id"]
            i += 1
        wait = 0.05 if i >= len(pending) else max(0.0, min(0.05, pending[i]["t"] - now))
        for r in b.tick(wait_s=wait):
            results[ticket_of[r["id"]]] = r
    b.close()
    res = [results[r["id"]] for r in reqs]
    lat = np.array([r["finish_s"] - r["arrival_s"] for r in res])
    wait_q = np.array([r["start_s"] - r["arrival_s"] for r in res])
    span = max(r["finish_s"] for r in res) - t0
    iters = sum(r["global_iters"] for r in res)
    st = min([0] + [r["status"] for r in res])
    return {"status": st, "requests": len(res),
            "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()), "mean_queue_wait_s": float(wait_q.mean()),
            "global_iters_per_s": iters / span, "makespan_s": span,
            "pcg_iters_per_request": [int(r["pcg_iters"]) for r in res], "max_active": active,
            "cohort": bool(cohort)}


SERVE_ARMS = {
    # name: (precision, level0_op, graphs, concurrent, cohort, open-loop run)
    "batched_streams": (1, 1, 1, True, False, True),
    "batched_cohort": (1, 1, 1, True, True, False),
    "serial_mixed": (1, 1, 1, False, False, True),
    "plain_fp64": (0, 0, 0, False, False, True),
}


def serving(args):
    """Serving load: step requests of uneven instances with Poisson arrivals,
    driven through the request loop with wall-clock arrivals, all at PCG rtol
    1e-6 on the same seeded trace (each request's instance drawn uniformly
    from --serve-instances).  Arms (--serve-arms):
      batched_streams  the served form: mixed precision, matrix-free level 0,
                       up to --serve-active requests at once, each on its own
                       stream and worker thread with CUDA graphs;
      batched_cohort   the same settings with the PCG iterations of all
                       running requests one launch per step (only its
                       saturated run, for capacity);
      serial_mixed     the same solver settings, one request at a time
                       (isolates the batching);
      plain_fp64       FP64, assembled CSR, plain launches, one at a time (the
                       plain solver).
    Admission budget: half of the free device memory."""
    import torch

    from paper_2505_13390_gb300.meshgen import instance_mesh, serving_trace
    inst, reqs = serving_trace(args.serve_requests, args.serve_instances, args.serve_rate)
    meshes = [instance_mesh(d) for d in inst]
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.5 * free)
    out = {}
    for name in args.serve_arms.split(","):
        prec, op, graphs, conc, cohort, open_loop = SERVE_ARMS[name]
        if open_loop:
            out[name] = serve_arm(meshes, reqs, prec, op, graphs,
                                  args.serve_active if conc else 1, budget, cohort)
            torch.cuda.empty_cache()
        if conc and not args.no_serve_saturated:
            # the same requests all at t = 0: the batched arm's capacity (at the
            # open-loop rate it is not saturated, and its throughput is the
            # offered load); the one-at-a-time arms are saturated at any rate
            sat = [dict(r, t=0.0) for r in reqs]
            out[name + "_saturated"] = serve_arm(meshes, sat, prec, op, graphs,
                                                 args.serve_active, budget, cohort)
            torch.cuda.empty_cache()
    out["trace"] = {"requests": len(reqs), "instances": len(inst),
                    "rate_hz": args.serve_rate,
                    "meshes": [f"{d['kind']}{d['size']}" for d in inst],
                    "budget": "half of free device memory", "frames_per_request": 1,
                    "iters_per_frame": 20, "pcg_rtol": 1e-6, "arrivals": "Poisson, seed 6"}
    if "batched_streams" in out:
        key = "batched_streams_saturated" if "batched_streams_saturated" in out else \
            "batched_streams"
        b = out[key]["global_iters_per_s"]
        for base in ("plain_fp64", "serial_mixed", "batched_cohort_saturated"):
            if base in out:
                out[f"capacity_speedup_vs_{base}"] = b / out[base]["global_iters_per_s"]
    return out


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(steps=2, warm=1, omp=False):
    """The FP64 oracle on a bounded sample of block100: a 4x33x4-cell block of
    the same recipe, `steps` global iterations timed after `warm`, PCG capped
    at SAMPLE_PCG iterations (it does not reach 1e-6 there; its cost is
    linear in the iterations).  The time per global iteration is scaled to
    block100 by the nnz ratio and by FULL_PCG_ITERS over the sample's PCG
    iterations.  omp=True runs the OpenMP build (same bits) on all host cores."""
    from oracle import oracle
    from oracle.oracle import Oracle
    from paper_2505_13390_gb300.meshgen import default_params, hex_block
    mesh = hex_block(*SAMPLE, h=0.005, jitter=0.1, alpha=1e-10, pin="y0", seed=1,
                     name="block-sample")
    p = default_params(omega_x=0.1, setup_interval=20, pcg_maxiter=SAMPLE_PCG)
    cores = oracle.threads(host_cores()) if omp else 1
    o = Oracle(mesh, p, omp=omp)
    nnz = int(o.matrix(0)[0][-1])
    o.begin_frame()
    for _ in range(warm):
        o.iterate()
    t0 = time.perf_counter()
    pcg = [o.iterate()["pcg_iters"] for _ in range(steps)]
    dt = (time.perf_counter() - t0) / steps
    scale = FULL_NNZ / nnz
    pscale = FULL_PCG_ITERS / (sum(pcg) / len(pcg))
    value = 1.0 / (dt * scale * pscale)
    sample = (f"block100 extrapolated: FP64 C oracle ({'OpenMP build, ' if omp else ''}{cores} "
              f"thread(s)), {steps} global iteration(s) after {warm} on a "
              f"{SAMPLE[0]}x{SAMPLE[1]}x{SAMPLE[2]}-cell block of the same recipe ({mesh.n_rows} "
              f"rows, {nnz} nnz, PCG iterations {pcg}, capped), {dt:.2f} s per iteration, scaled "
              f"by the nnz ratio {scale:.1f} and the PCG-iteration ratio {pscale:.2f} to "
              f"{FULL_NNZ} nnz and {FULL_PCG_ITERS} PCG iterations")
    return {"value": value, "unit": "global_iters/s", "cores": cores, "kind": "oracle",
            "sample": sample}


def direct_pair(name, iters, oracle_builds=(False, True)):
    """The oracle and the GPU on the same full-size workload and inputs, timed
    directly: the first `iters` global iterations of frame 0, PCG to 1e-6.
    Oracle in its plain build (1 thread) and/or its OpenMP build (all host
    cores); GPU in FP64 (assembled CSR, plain launches) and in the benchmark's
    configuration (mixed, matrix-free, CUDA graphs, autotuned).  Reports
    global iterations/s of each and the largest position difference from
    the oracle (relative to the largest coordinate)."""
    import numpy as np
    import torch

    from oracle import oracle
    from oracle.oracle import Oracle
    from paper_2505_13390_gb300.meshgen import workload
    from paper_2505_13390_gb300.mgpbd import Solver
    mesh, p = workload(name)
    out = {"workload": name, "rows": mesh.n_rows, "global_iters": iters, "pcg_rtol": 1e-6}
    xo = None
    for omp in oracle_builds:
        cores = oracle.threads(host_cores()) if omp else 1
        o = Oracle(mesh, p, omp=omp)
        o.begin_frame()
        t0 = time.perf_counter()
        pcg = [o.iterate()["pcg_iters"] for _ in range(iters)]
        dt = time.perf_counter() - t0
        out["oracle_omp" if omp else "oracle_1core"] = {
            "value": iters / dt, "cores": cores, "pcg_iters": pcg}
        xo = o.get_state()[0]
        del o
    scale = float(np.abs(mesh.rest_pos).max())
    for leg, q in (("gpu_fp64", dict(p, precision=0, level0_op=0, use_graphs=0)),
                   ("gpu_mixed", dict(p, precision=1, level0_op=1, use_graphs=1, autotune=1))):
        g = Solver(mesh, q, stream=torch.cuda.Stream())
        g.begin_frame()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pcg = [g.iterate()["pcg_iters"] for _ in range(iters)]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        xg = g.get_state()[0]
        g.close()
        out[leg] = {"value": iters / dt, "pcg_iters": pcg,
                    "max_dx_vs_oracle": float(np.abs(xg - xo).max() / scale)}
    ref = out.get("oracle_1core") or out.get("oracle_omp")
    out["gpu_mixed_over_oracle"] = out["gpu_mixed"]["value"] / ref["value"]
    return out


def xpbd_comparison():
    """One frame of the 512x512 cloth (1,306,625 rows, per-row compliance over
    four decades) with MGPBD and with XPBD's local step (eq. 4, the solver
    the paper compares against on the GPU): the dual residual |b| before each
    of the 20 global iterations and after the last, relative to the first,
    and the time of a global iteration (median over iterations 2-20; the
    first carries the AMG setup)."""
    import numpy as np
    import torch

    from paper_2505_13390_gb300.meshgen import workload
    from paper_2505_13390_gb300.mgpbd import Solver
    mesh, p = workload("cloth512")
    out = {"workload": "cloth512: 512x512 cloth with bend edges, top row pinned, "
                       "alpha = 10^U(-10,-6) per row, one frame of 20 global iterations",
           "rows": mesh.n_rows}
    for name, ls in (("mgpbd", 0), ("xpbd", 1)):
        q = dict(p, precision=1, level0_op=1, use_graphs=1, autotune=1, linear_solver=ls)
        g = Solver(mesh, q, stream=torch.cuda.Stream())
        g.begin_frame()
        bn, ms, pcg = [], [], 0
        for _ in range(q["max_iter"]):
            t0 = time.perf_counter()
            d = g.iterate()
            ms.append(1e3 * (time.perf_counter() - t0))
            bn.append(d["bnorm"])
            pcg += d["pcg_iters"]
        g.eval_assemble()
        bn.append(float(np.linalg.norm(g.constraints()[1])))
        g.close()
        rel = [b / bn[0] for b in bn]
        out[name] = {"bnorm_rel_after": {str(k): rel[k] for k in (1, 2, 5, 10, 20)},
                     "ms_per_iter": float(np.median(ms[1:])), "pcg_iters": pcg}
    torch.cuda.empty_cache()
    return out


def run_ours(args, ws, rank):
    import torch

    import __graft_entry__ as ge
    from paper_2505_13390_gb300.meshgen import workload
    if not os.path.exists(os.path.join(ROOT, "paper_2505_13390_gb300", "libmgpbd.so")):
        ge.build()
    if args.serve_only:
        if rank == 0:
            print(json.dumps({"metric": "p50/p99 step latency and global XPBD iters/s, served",
                              "serving": serving(args)}))
        return
    cpu = None
    mesh, params = workload(args.workload)
    params = dict(params, precision=1, autotune=1, level0_op=args.level0_op, use_graphs=1,
                  ap_split=args.ap_split if args.level0_op == 1 else 0)
    # the headline records the sweeps' event pairs (the roofline), and the
    # A.p's only when it is the pair form (the FP64 form is timed in the
    # fp64 leg, on the same kernels)
    res = measure(mesh, params, args.steps, args.warmup, ws,
                  profile_ap=bool(params["ap_split"]))
    value, ms = job_rate(ws, args.steps, res["ms"])
    prof = res["prof"]
    g = res["solver"]
    nnz = res["stats"]
    li = g.level_info(0)
    if li["nnz"] != FULL_NNZ and args.workload == "block100":
        raise RuntimeError(f"unexpected nnz {li['nnz']}")
    hbm = hbm_peak()
    peak_src = "measured" if _measured_hbm() else "fallback"
    avg_ms = prof["total_ms"] / max(prof["launches"], 1)
    achieved = prof["bytes_per_launch"] / (avg_ms / 1e3) / 1e9
    e2e_val = None
    e2e_bytes = 0
    e2e_pcg = []
    if not args.no_e2e:
        pcg0 = len(res["runner"].pcg)
        e2e_val, e2e_bytes = e2e(g, res["runner"], args.e2e_steps)
        e2e_val = e2e_val * ws
        e2e_pcg = list(res["runner"].pcg[pcg0:])
    ap_prod = ap_roofline(res["prof_ap"], 1) if params["ap_split"] else None
    fp64 = None
    assembled = None
    ap_ab = None
    levels = [g.level_info(l) for l in range(g.levels)]
    g.close()
    del res["solver"], res["runner"]
    torch.cuda.empty_cache()
    if args.level0_op == 1 and not args.no_ap_ab:
        # the same configuration with the other form of the recurrence's A.p,
        # timed the same way from the same start
        pb = dict(params, ap_split=1 - params["ap_split"])
        rb = measure(mesh, pb, args.ap_ab_steps, args.ap_ab_warmup, ws, profile_ap=True)
        msb = max_over_ranks(ws, rb["ms"])
        ap_ab = {"ap_split": pb["ap_split"], "value": ws * args.ap_ab_steps / (msb / 1e3),
                 "ms_per_step": msb / args.ap_ab_steps, "steps": args.ap_ab_steps,
                 "warmup": args.ap_ab_warmup, "pcg_iters": rb["pcg"],
                 "true_rel_res": rb["true_res"], "clocks": rb["clocks"],
                 "ap_product": ap_roofline(rb["prof_ap"], pb["ap_split"])}
        rb["solver"].close()
        del rb
        torch.cuda.empty_cache()
    if args.level0_op == 1 and not args.no_assembled:
        pa = dict(params, level0_op=0, ap_split=0)
        ra = measure(mesh, pa, args.assembled_steps, args.assembled_warmup, ws)
        msa = max_over_ranks(ws, ra["ms"])
        pr = ra["prof"]
        aa = pr["bytes_per_launch"] / (pr["total_ms"] / max(pr["launches"], 1) / 1e3) / 1e9
        assembled = {"value": ws * args.assembled_steps / (msa / 1e3),
                     "ms_per_step": msa / args.assembled_steps,
                     "steps": args.assembled_steps, "warmup": args.assembled_warmup,
                     "pcg_iters": ra["pcg"], "true_rel_res": ra["true_res"],
                     "clocks": ra["clocks"],
                     "roofline": {"bound": "hbm",
                                  "kernel": "k_jacobi (level-0 CSR weighted-Jacobi sweep, FP32)",
                                  "achieved": aa, "peak": hbm_peak(), "unit": "GB/s",
                                  "frac": aa / hbm_peak(),
                                  "bytes_per_launch": pr["bytes_per_launch"],
                                  "avg_launch_ms": pr["total_ms"] / max(pr["launches"], 1),
                                  "traffic": SWEEP_TRAFFIC_PER_NNZ * li["nnz"]}}
        ra["solver"].close()
        del ra
        torch.cuda.empty_cache()
    if not args.no_fp64:
        p64 = dict(params, precision=0, ap_split=0)
        # the FP64 A.p kernels are the headline's: they are timed here, so that
        # the headline's timed region carries only the sweeps' event pairs
        r64 = measure(mesh, p64, args.fp64_steps, args.fp64_warmup, ws, profile_ap=True)
        ms64 = max_over_ranks(ws, r64["ms"])
        pr = r64["prof"]
        a64 = pr["bytes_per_launch"] / (pr["total_ms"] / max(pr["launches"], 1) / 1e3) / 1e9
        fp64 = {"value": ws * args.fp64_steps / (ms64 / 1e3),
                "ms_per_step": ms64 / args.fp64_steps,
                "steps": args.fp64_steps, "warmup": args.fp64_warmup,
                "pcg_iters": r64["pcg"], "true_rel_res": r64["true_res"],
                "clocks": r64["clocks"],
                "smoother_sweep_gbs": a64, "smoother_sweep_frac": a64 / hbm,
                "ap_product": ap_roofline(r64["prof_ap"], 0)}
        if ap_prod is None and fp64["ap_product"]:
            ap_prod = dict(fp64["ap_product"],
                           measured_in="fp64 leg: the same FP64 A.p kernels on the same "
                                       "workload, so that the headline's timed region carries "
                                       "only the sweeps' event pairs")
        r64["solver"].close()
    arap = None
    if not args.no_arap:
        # the same lattice with one ARAP row per tet (Sec. 5.3) instead of
        # distance + volume rows, same solver settings
        amesh, ap_ = workload("block100arap")
        ap_ = dict(ap_, autotune=1, use_graphs=1, level0_op=args.level0_op,
                   pcg_maxiter=params["pcg_maxiter"])
        rar = measure(amesh, ap_, args.arap_steps, args.arap_warmup, ws)
        msr = max_over_ranks(ws, rar["ms"])
        arap = {"workload": "block100arap: the 100x33x100 block with one ARAP row per tet "
                            "(1,650,000 rows), mu = 1e7 Pa, alpha = 1/(mu V_tet)",
                "value": ws * args.arap_steps / (msr / 1e3), "unit": "global_iters/s",
                "ms_per_step": msr / args.arap_steps, "steps": args.arap_steps,
                "warmup": args.arap_warmup, "pcg_iters": rar["pcg"],
                "true_rel_res": rar["true_res"], "clocks": rar["clocks"],
                "n_setups": rar["solver"].stats()["n_setups"]}
        rar["solver"].close()
        del rar
        torch.cuda.empty_cache()
    smoothers = None
    if not args.no_smoothers:
        # the paper's other smoother (Sec. 4.5: Chebyshev, its choice for
        # cloth) on the same block, two and three sweeps per side, timed the
        # same way from the same start (the headline keeps weighted Jacobi,
        # its choice for soft bodies)
        smoothers = {}
        for sweeps in (2, 3):
            ps = dict(params, smoother=2, smooth_sweeps=sweeps)
            rs = measure(mesh, ps, args.smoother_steps, args.smoother_warmup, ws, profile=False)
            mss = max_over_ranks(ws, rs["ms"])
            smoothers[f"chebyshev{sweeps}"] = {
                "value": ws * args.smoother_steps / (mss / 1e3), "unit": "global_iters/s",
                "ms_per_step": mss / args.smoother_steps, "steps": args.smoother_steps,
                "warmup": args.smoother_warmup, "pcg_iters": rs["pcg"],
                "true_rel_res": rs["true_res"], "clocks": rs["clocks"]}
            rs["solver"].close()
            del rs
            torch.cuda.empty_cache()
    xpbd = None
    if not args.no_xpbd and ws == 1:  # a single-GPU comparison: not repeated per rank
        xpbd = xpbd_comparison()
    serve = None
    if not args.no_serve:
        serve = serving(args)
    if rank != 0:
        return
    cpu_all = cpu_direct = None
    if not args.no_cpu:
        cpu = oracle_sample(omp=False)
        cpu_all = oracle_sample(omp=True)
        cpu_direct = [direct_pair("cloth32", 2)]
        cpu_direct.append(direct_pair("beam40", 1, (False, True) if args.cpu_full else (True,)))
    line = {
        "metric": "global XPBD iters/s at 1.65M tets (mixed precision; FP64 under fp64; "
                  "p50/p99 step latency under serving)",
        "value": value,
        "unit": "global_iters/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "rows": li["n"], "nnz": li["nnz"],
                   "level0_operator": "matrix-free" if args.level0_op == 1 else "assembled CSR",
                   "tets": mesh.n_tet, "verts": mesh.n_verts, "iters_per_frame": 20,
                   "setup_interval": params["setup_interval"], "pcg_rtol": 1e-6,
                   "pcg_maxiter": params["pcg_maxiter"], "parallelism": f"replicas{ws}",
                   "l2": ("inputs larger than L2 (129 MB): a matrix-free level-0 sweep reads "
                          "0.42 GB, an FP64 A.p 0.64 GB; the assembled A is 3.1 GB in FP32, "
                          "4.6 GB in FP64"),
                   "levels": [(l["n"], l["nnz"]) for l in levels]},
        "pcg_iters": res["pcg"],
        # FP64 |b - A dlambda| / |b| of each timed solve: the error statement
        # of the mixed-precision result (the oracle cannot run this size)
        "true_rel_res": res["true_res"],
        # the PCG recurrence's A.p (vertex and row pass), timed live the same way
        "ap_product": ap_prod,
        "ap_other_form": ap_ab,
        "roofline": {"bound": "hbm",
                     "kernel": ("level-0 matrix-free weighted-Jacobi sweep, FP32 "
                                "(k_mf_vertex + k_mf_row)") if args.level0_op == 1 else
                               "k_jacobi (level-0 CSR weighted-Jacobi sweep, FP32)",
                     "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_source": peak_src,
                     "traffic": ((MF_SWEEP_TRAFFIC_PER_ROW * li["n"])
                                 if MF_SWEEP_TRAFFIC_PER_ROW else None) if args.level0_op == 1
                                else SWEEP_TRAFFIC_PER_NNZ * li["nnz"],
                     "traffic_source": "ncu dram__bytes_read+write on a 40x33x40 block of the "
                                       "same recipe, scaled by the units processed",
                     "bytes_per_launch": prof["bytes_per_launch"], "avg_launch_ms": avg_ms,
                     "launches": prof["launches"]},
        "cpu_baseline": cpu,
        # the same sample on all host cores (the oracle's OpenMP build, same bits)
        "cpu_baseline_all_cores": cpu_all,
        # oracle and GPU timed directly, without extrapolation, on full-size
        # workloads the oracle finishes (cloth32, beam40), on the same inputs
        "cpu_direct": cpu_direct,
        # the end-to-end steps are the global iterations after the timed ones
        # (same frame); their PCG counts differ from the timed steps'
        "e2e": {"value": e2e_val, "unit": "global_iters/s", "h2d_bytes_per_step": e2e_bytes,
                "d2h_bytes_per_step": e2e_bytes, "pcg_iters": e2e_pcg} if e2e_val else None,
        "gpu_launches": res["launches"],
        "clocks": res["clocks"],
        "fp64": fp64,
        "assembled": assembled,
        "arap": arap,
        "smoothers": smoothers,
        "xpbd_vs_mgpbd": xpbd,
        "serving": serve,
        "create_s": res["create_s"],
        "stats": {k: res["stats"][k] for k in ("levels", "op_complexity", "device_bytes")},
    }
    print(json.dumps(line))


def run_reference(args, ws, rank):
    """The reference arm: the FP64 oracle as it stands (plain build, one
    thread) on the bounded block100 sample, args.steps global iterations
    timed after args.warmup, scaled as in oracle_sample."""
    if rank != 0:
        return
    cpu = oracle_sample(steps=max(1, args.steps), warm=max(0, args.warmup), omp=False)
    value = cpu["value"]
    line = {
        "impl": "reference",
        "metric": "global XPBD iters/s at 1.65M tets (mixed precision; FP64 under fp64; "
                  "p50/p99 step latency under serving)",
        "value": value, "unit": "global_iters/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"block100, extrapolated from a {SAMPLE[0]}x{SAMPLE[1]}x{SAMPLE[2]}"
                               f"-cell sample of the same recipe",
                   "rows": 3_680_033, "nnz": FULL_NNZ, "tets": 1_650_000, "verts": 346_834,
                   "iters_per_frame": 20, "setup_interval": 20, "pcg_rtol": 1e-6,
                   "pcg_iters_scaled_to": FULL_PCG_ITERS, "parallelism": f"replicas{ws}"},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": "global_iters/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = parse()
    ws, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
