"""Benchmark: solves/s to a 1e-8 relative residual on the dissipative-Hamiltonian
implicit-Euler workload (100^3 grid, n = 1e6), FP32 inner mrs / FP64 outer FGMRES.

One step = one solve phase (outer Krylov + preconditioner applications + inner mrs)
for one right-hand side, after the b-independent set-up (timed and reported
separately, as the paper amortises it over right-hand sides).

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank runs an independent replica (the single system does not
shard in this build); value = all ranks' solves / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solves/s to 1e-8 rel. residual"
UNIT = "solves/s"
WORKLOAD = ("dh3d_100: dissipative-Hamiltonian implicit-Euler step A = E + h(R - J), 100^3 grid "
            "(n = 1,000,000, nnz = 6,940,000), S on the pattern of A, k = 20, FP32 inner mrs "
            "(tol {inner_tol}) / FP64 outer FGMRES(60), outer tol 1e-8")
DH = {"inner_tol": 1e-3, "factor": "diag"}


def dh_workload():
    w = WORKLOAD.format(inner_tol=f"{DH['inner_tol']:g}".replace("e-0", "e-"))
    if DH["factor"] == "ildl0":
        w += "; L~ = the no-fill incomplete L D L^T of M^ (~ildl(0), multicolour order)"
    return w


SIDE = 100
CPU_SAMPLE_SIDE = 40
ADJ_CPU_SIDE = 24
# inner tolerance 1e-3 for the batched and adjoint workloads, chosen as for dh3d_100: the
# same outer step counts and residuals as at 1e-6 (measured), fewer inner steps
BATCH = {"count": 256, "side_lo": 10, "side_hi": 40, "nrhs": 32, "seed": 3, "inner_tol": 1e-3}
ADJ_INNER_TOL = 1e-3


def batch_gen_args(**over):
    """Arguments of the batched generator (BATCH without the solver's inner tolerance)."""
    a = {k: v for k, v in BATCH.items() if k != "inner_tol"}
    a.update(over)
    return a
GENERAL = {"n": 2_000_000, "seed": 2, "outer_steps": 20, "lls_maxit": 100}
GENERAL_WORKLOAD = ("general_2e6: general sparse nonsymmetric matrix, n = {n:,}, power-law row lengths (min 4, mean 16, "
                    "max 512), 60% of columns within |i-j| <= 1000, N(0,1) values, 30% of rows with diagonal 1.1 x "
                    "row abs-sum, S on pat(A + A^T), b ~ N(0,1); FP32 inner mrs (tol 1e-6, J~ in SELL-C-sigma) / FP64 "
                    "outer FGMRES(60); a step = {steps} outer steps (the method does not reach 1e-8 on this recipe)")
ADJ_SIDE = 64
ADJ_WORKLOAD = ("adjoint_dh64: gradient of L = ||x - x*||^2 for the dissipative-Hamiltonian step on a 64^3 grid "
                "(n = 262,144), x* ~ N(0,1): dL/db = lambda from A^T lambda = 2 (x - x*) and dL/dA = -lambda_i x_j "
                "on A's nonzeros, FP32 inner mrs (tol 1e-3) / FP64 outer FGMRES(60), outer tol 1e-8")
BATCH_WORKLOAD = ("batched_dh: {count} dissipative-Hamiltonian systems, 3D grids of sides 10..40 (n = 1e3..6.4e4, "
                  "seeded), 32 right-hand sides ~ N(0,1) each ({items} solves per step), one persistent launch "
                  "replayed from a CUDA graph, FP32 inner mrs (tol 1e-3) / FP64 outer FGMRES(24), outer tol 1e-8")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _make_rhs(A_parts, n, seed, count):
    import numpy as np
    out = []
    E = A_parts["E"]
    for c in range(count):
        r = np.random.default_rng(seed + 1000 + c)
        out.append(E * r.standard_normal(n) + 1e-2 * r.standard_normal(n))
    return out


# ----------------------------------------------------------------------------
# CPU oracle baseline (subprocess, one thread)
# ----------------------------------------------------------------------------
def _barrier_pool(procs, target, args_of):
    """Run target(rank, barrier, queue, *args_of(rank)) in `procs` forked processes
    (CPU only; this process never touches the GPU).  Every process does its untimed
    set-up, waits at the barrier, then does its timed work; returns the results and the
    wall time from the barrier's release until the last process finished."""
    import multiprocessing as mp
    ctx = mp.get_context("fork")
    barrier = ctx.Barrier(procs + 1)
    q = ctx.Queue()
    ps = [ctx.Process(target=target, args=(r, barrier, q) + tuple(args_of(r))) for r in range(procs)]
    for p_ in ps:
        p_.start()
    barrier.wait()
    t0 = time.perf_counter()
    res = [q.get() for _ in range(procs)]
    wall = time.perf_counter() - t0
    for p_ in ps:
        p_.join()
    return res, wall


def _batched_proc(rank, barrier, q, mats, budget_s):
    import oracle
    setups = []
    for A, B in mats:
        o = oracle.AsssOracle(A, inner_tol=BATCH["inner_tol"])
        o._smw(False)   # the SMW data the oracle would otherwise build inside the first solve
        setups.append((o, A, B))
    barrier.wait()
    solves, rows, relres = 0, 0, 0.0
    t0 = time.perf_counter()
    for o, A, B in setups:
        for c in range(2):
            _, st = o.solve(B[:, c], tol=1e-8, outer="fgmres")
            solves += 1
            rows += A.shape[0]
            relres = max(relres, st["relres"])
        if time.perf_counter() - t0 > budget_s:
            break
    q.put((solves, rows, relres, time.perf_counter() - t0))


def batched_worker(budget_s, procs):
    """Oracle solves of a bounded sample of the batched workload's items, on all host
    cores: the sampled matrices (every 8th by size) are dealt to the processes, each
    sets its share up (untimed), then all solve two columns per matrix at once."""
    import numpy as np

    from workloads import batched_dissipative_hamiltonian
    batch = batched_dissipative_hamiltonian(**batch_gen_args())
    order = np.argsort([A.shape[0] for A, _ in batch])
    sample = [batch[m] for m in order[::max(1, len(order) // 32)]]
    res, wall = _barrier_pool(procs, _batched_proc, lambda r: (sample[r::procs], budget_s))
    solves = sum(r[0] for r in res)
    rows = sum(r[1] for r in res)
    print(json.dumps({"solves": solves, "seconds": wall, "rows": rows, "procs": procs,
                      "matrices": len(sample), "max_relres": max(r[2] for r in res)}))


def _adjoint_proc(rank, barrier, q, budget_s):
    import numpy as np

    import oracle
    from workloads import dissipative_hamiltonian_3d
    A, b, _ = dissipative_hamiltonian_3d(side=ADJ_CPU_SIDE, seed=4)
    n = A.shape[0]
    o = oracle.AsssOracle(A, inner_tol=ADJ_INNER_TOL)
    x, _ = o.solve(b, tol=1e-8, outer="fgmres")
    o._smw(True)        # the transposed SMW data (set-up of the adjoint), outside the timed solves
    g = 2.0 * (x - np.random.default_rng(44).standard_normal(n))
    barrier.wait()
    cnt = 0
    t0 = time.perf_counter()
    while True:
        o.solve_adjoint(g, x, tol=1e-8, outer="fgmres")
        cnt += 1
        if time.perf_counter() - t0 > budget_s or cnt >= 50:
            break
    q.put((cnt, n))


def adjoint_worker(budget_s, procs):
    """Oracle gradients at ADJ_CPU_SIDE^3 (forward solve untimed, adjoint solve + dL/dA
    timed), one oracle per host core, all at once."""
    res, wall = _barrier_pool(procs, _adjoint_proc, lambda r: (budget_s,))
    print(json.dumps({"n": res[0][1], "solves": sum(r[0] for r in res), "seconds": wall, "procs": procs,
                      "t_setup_s": 0.0}))


def run_adjoint_cpu_baseline(budget_s):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    procs = host_cores()
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker", "--workload", "adjoint_dh64", "--budget",
           str(budget_s), "--procs", str(procs)]
    p = subprocess.run(cmd, capture_output=True, text=True, env=env, cwd=ROOT)
    if p.returncode != 0:
        raise RuntimeError("CPU baseline worker failed:\n" + p.stdout + p.stderr)
    r = json.loads(p.stdout.strip().splitlines()[-1])
    n_full = ADJ_SIDE ** 3
    per_s = r["solves"] / r["seconds"]
    return {
        "value": per_s * r["n"] / n_full, "unit": "gradients/s", "cores": r["procs"], "kind": "oracle",
        "sample": (f"FP64 numpy/scipy oracle, adjoint solve + dL/dA at {ADJ_CPU_SIDE}^3 (n = {r['n']}), "
                   f"{r['solves']} on {r['procs']} processes (one per host core, BLAS 1 thread) in "
                   f"{r['seconds']:.2f} s wall ({per_s:.3f}/s), each counted as n_sample/n of a 64^3 gradient; "
                   f"set-up and the forward solve untimed"),
        "solves": r["solves"], "seconds": r["seconds"],
    }


def batch_mean_n():
    """Mean system size of the batched workload (its sides drawn as the generator does)."""
    import numpy as np
    rng = np.random.default_rng(BATCH["seed"])
    sides = rng.integers(BATCH["side_lo"], BATCH["side_hi"] + 1, size=BATCH["count"])
    return float(np.mean(sides.astype(np.float64) ** 3))


def run_batched_cpu_baseline(budget_s, mean_n):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    procs = host_cores()
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker", "--workload", "batched_dh", "--budget",
           str(budget_s), "--batch-count", str(BATCH["count"]), "--procs", str(procs)]
    p = subprocess.run(cmd, capture_output=True, text=True, env=env, cwd=ROOT)
    if p.returncode != 0:
        raise RuntimeError("CPU baseline worker failed:\n" + p.stdout + p.stderr)
    r = json.loads(p.stdout.strip().splitlines()[-1])
    per_s = r["solves"] / r["seconds"]
    sample_n = r["rows"] / r["solves"]
    return {
        "value": per_s * sample_n / mean_n, "unit": UNIT, "cores": r["procs"], "kind": "oracle",
        "sample": (f"FP64 numpy/scipy oracle, {r['solves']} solves (2 columns each of {r['matrices']} matrices, "
                   f"every 8th of the batch by size, mean n = {sample_n:.0f}) on {r['procs']} processes (one per "
                   f"host core, BLAS 1 thread) in {r['seconds']:.2f} s wall ({per_s:.3f} solves/s), each counted "
                   f"as n_item / mean n = {mean_n:.0f} of an item; set-up untimed"),
        "max_relres": r["max_relres"], "solves": r["solves"], "seconds": r["seconds"],
    }


_ORACLE = {}


def _oracle_solve(i):
    """One oracle solve of right-hand side i in a forked pool process (CPU only)."""
    o, rhs = _ORACLE["o"], _ORACLE["rhs"]
    t = time.perf_counter()
    _, st = o.solve(rhs[i % len(rhs)], tol=1e-8, outer="fgmres")
    return time.perf_counter() - t, st["relres"], st["inner_its_avg"], st["outer_its"]


def cpu_worker(side, steps, warmup, budget_s, procs, xout):
    """The FP64 oracle's solve phase on the side^3 instance of the bench's generator.

    Set-up once (untimed), then: one solve alone (the one-thread rate; its x is
    written to xout for the relative-error check of the GPU legs), then `warmup`
    untimed and up to `steps` timed rounds of `procs` concurrent solves, one per
    forked process (all host cores, BLAS pinned to one thread each), stopping
    early once `budget_s` of timed rounds have run.  This process never touches
    the GPU, so forking after the set-up is safe."""
    import multiprocessing as mp

    import numpy as np

    import oracle
    from workloads import dissipative_hamiltonian_3d
    A, b, parts = dissipative_hamiltonian_3d(side=side, seed=1)
    n = A.shape[0]
    t0 = time.perf_counter()
    o = oracle.AsssOracle(A, inner_tol=DH["inner_tol"], factor=DH["factor"])
    rhs = _make_rhs(parts, n, 1, 8)
    o.solve(rhs[0], tol=1e-8, outer="fgmres")   # the oracle builds its SMW data on first use: set-up
    t_setup = time.perf_counter() - t0
    _ORACLE["o"], _ORACLE["rhs"] = o, rhs
    t = time.perf_counter()
    x0, st0 = o.solve(rhs[0], tol=1e-8, outer="fgmres")
    t_one = time.perf_counter() - t
    if xout:
        np.save(xout, x0)
    rounds, relres, inner, outer = [], [st0["relres"]], [st0["inner_its_avg"]], [st0["outer_its"]]
    with mp.get_context("fork").Pool(procs) as pool:
        for w in range(warmup):
            pool.map(_oracle_solve, range(procs))
        t_start = time.perf_counter()
        for s in range(steps):
            t = time.perf_counter()
            res = pool.map(_oracle_solve, [s * procs + i for i in range(procs)])
            rounds.append(time.perf_counter() - t)
            relres += [r[1] for r in res]
            inner += [r[2] for r in res]
            outer += [r[3] for r in res]
            if budget_s and time.perf_counter() - t_start > budget_s:
                break
    print(json.dumps({"n": n, "side": side, "procs": procs, "rounds": rounds, "warmup": warmup,
                      "t_one": t_one, "t_setup_s": t_setup, "max_relres": max(relres),
                      "inner_avg": float(np.mean(inner)), "outer_its": int(max(outer))}))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_cpu_baseline(steps, warmup, budget_s, xout=None):
    """Oracle solve rate on the CPU_SAMPLE_SIDE^3 instance, on all host cores, in the
    bench's unit: each sample solve counts as n_sample / n_full of a 100^3 solve (the
    solve phase of this generator is linear in n: the same outer count and nearly the
    same inner count at every grid size, reported in the sample line)."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    procs = host_cores()
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker", "--steps", str(steps), "--warmup",
           str(warmup), "--budget", str(budget_s), "--procs", str(procs), "--inner-tol", repr(DH["inner_tol"]),
           "--factor", DH["factor"]]
    if xout:
        cmd += ["--xout", xout]
    p = subprocess.run(cmd, capture_output=True, text=True, env=env, cwd=ROOT)
    if p.returncode != 0:
        raise RuntimeError("CPU baseline worker failed:\n" + p.stdout + p.stderr)
    r = json.loads(p.stdout.strip().splitlines()[-1])
    n_full = SIDE ** 3
    scale = r["n"] / n_full
    wall = sum(r["rounds"])
    per_s = r["procs"] * len(r["rounds"]) / wall          # sample solves / s, all cores
    one_s = 1.0 / r["t_one"]                               # sample solves / s, one thread
    return {
        "value": per_s * scale, "unit": UNIT, "cores": r["procs"], "kind": "oracle",
        "sample": (f"FP64 numpy/scipy oracle, solve phase of the same generator and options at "
                   f"{r['side']}^3 (n = {r['n']}): {len(r['rounds'])} timed rounds of {r['procs']} concurrent "
                   f"solves (one process per host core, BLAS 1 thread) in {wall:.2f} s = {per_s:.2f} sample "
                   f"solves/s; one thread alone {one_s:.3f} sample solves/s ({one_s * scale:.4f} in the unit); "
                   f"each sample solve counted as n_sample/n = {scale:.4f} of a 100^3 solve; outer its "
                   f"{r['outer_its']}, inner avg {r['inner_avg']:.2f}; set-up {r['t_setup_s']:.1f} s untimed"),
        "one_thread_value": one_s * scale,
        "rounds": r["rounds"], "procs": r["procs"], "warmup": r["warmup"], "n_sample": r["n"],
        "max_relres": r["max_relres"], "t_setup_s": r["t_setup_s"],
    }


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[4:8]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _traffic_record():
    """ncu DRAM bytes per mrs launch, valid only for the current kernel source."""
    path = os.path.join(ROOT, "profiles", "mrs_traffic.json")
    src = os.path.join(ROOT, "paper_2009_06954_gb300", "csrc", "mrs.cu")
    try:
        rec = json.load(open(path))
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if rec.get("mrs_cu_sha256") == h:
            return rec
    except Exception:
        pass
    return None


# ----------------------------------------------------------------------------
# multi-rank helpers (replicas: one independent solve stream per GPU)
# ----------------------------------------------------------------------------
def prof_range(args, start):
    """cudaProfilerStart/Stop around the timed steps when asked (profilers that capture
    only that range see exactly the benchmark's kernels)."""
    if getattr(args, "cuda_profiler_range", False):
        import torch
        torch.cuda.synchronize()
        (torch.cuda.profiler.start if start else torch.cuda.profiler.stop)()


def rank_env():
    """(world, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def reduce_max(value, dist=None, device=None):
    """Largest value over the ranks (the slowest rank's time); identity without a group."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, steps, max_seconds):
    """Whole-job rate: every rank processed `steps` units; the job ends with the slowest."""
    return world * steps / max_seconds


# ----------------------------------------------------------------------------
# batched workload
# ----------------------------------------------------------------------------
def main_batched(args, world, rank, local):
    import numpy as np
    import torch

    import paper_2009_06954_gb300 as pkg
    from paper_2009_06954_gb300.binding import kernel_launches
    from workloads import batched_dissipative_hamiltonian

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    batch = batched_dissipative_hamiltonian(**batch_gen_args(seed=BATCH["seed"] + rank))
    nrhs = BATCH["nrhs"]
    t0 = time.perf_counter()
    bs = pkg.BatchSolver([A for A, _ in batch], inner_tol=BATCH["inner_tol"], outer_tol=1e-8, k=20, restart=24,
                         q_bf16=args.q_storage == "bf16", stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    bh = bs.pack([B for _, B in batch])
    items = len(batch) * nrhs
    bd = torch.tensor(bh, device=dev)
    xd = torch.empty_like(bd)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    for _ in range(args.warmup):
        bs.solve(bd, nrhs=nrhs, x=xd)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = kernel_launches()
    stats = []
    prof_range(args, True)
    with ClockSampler(dev.index) as clk:
        for _ in range(args.steps):
            flush.zero_()
            _, st = bs.solve(bd, nrhs=nrhs, x=xd)   # device time of the launch in t_inner_ms
            stats.append(st)
        torch.cuda.synchronize()
    launches = kernel_launches() - l0
    prof_range(args, False)
    if dist:
        dist.barrier()
    total_ms = sum(s_["t_inner_ms"] for s_ in stats)
    tmax = reduce_max(total_ms, dist, dev)
    relres = max(s_["relres"] for s_ in stats)
    ok = all(s_["status"] == 0 for s_ in stats) and relres <= 1e-8
    value = world * items * args.steps / (tmax / 1000.0)

    # end to end: pinned host b and x, copies inside the timed region
    bp = torch.from_numpy(bh).pin_memory()
    xp = torch.empty_like(bp).pin_memory()
    bs.solve(bp, nrhs=nrhs, x=xp)   # untimed: allocates the device copies of host b and x once
    e2e_s = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        bs.solve(bp, nrhs=nrhs, x=xp)
        e2e_s += time.perf_counter() - t
    e2e_val = world * items * args.steps / reduce_max(e2e_s, dist, dev)
    # the result is checked on the host for one step: every item's true residual
    X = bs.unpack(xd.cpu().numpy(), nrhs)
    worst = 0.0
    for (A, B), x in zip(batch, X):
        worst = max(worst, float(np.max(np.linalg.norm(B - A @ x, axis=0) / np.linalg.norm(B, axis=0))))
    peak, peak_kind = _peaks()
    inner_bytes = sum(s_["inner_bytes"] for s_ in stats)
    achieved = inner_bytes / (total_ms / 1000.0) / 1e9 if total_ms > 0 else 0.0
    # the precision form's comparison: the same systems and right-hand sides through the
    # one-system path (asss_solve, one column after another), in FP64 throughout and in
    # mixed precision, on a sample of every 16th matrix by size (timed with CUDA events)
    one_sys = None
    if not args.no_fp64_leg and rank == 0:
        one_sys = batched_one_system_legs(pkg, torch, batch, nrhs, dev, stream, flush, bs.total / len(batch))

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    mean_n = bs.total / len(batch)
    cpu = None
    if not args.no_cpu_baseline and world == 1:  # the oracle baseline is timed at N = 1 only
        try:
            cb = run_batched_cpu_baseline(15.0, mean_n)
            cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        except Exception as e:
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"[:300]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32-inner/f64-outer", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD.format(count=len(batch), items=items),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "256 MB buffer written between steps (not timed); working set > L2",
                   "setup_s": round(t_setup, 3), "cta_threads": bs.cta_threads,
                   "cta_registers": bs.cta_registers, "items_per_step": items,
                   "total_rows": bs.total, "max_relres": relres, "host_checked_max_relres": worst,
                   "converged": ok and worst <= 1e-8, "outer_its_max": stats[-1]["outer_its"],
                   "inner_its_total": stats[-1]["inner_its_total"], "q_storage": args.q_storage,
                   "fp64_gpu": one_sys["fp64"] if one_sys else None,
                   "one_system_mixed": one_sys["mixed"] if one_sys else None},
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 8 * bs.total * nrhs,
                "d2h_bytes_per_step": 8 * bs.total * nrhs},
        "roofline": {"bound": "hbm", "kernel": "k_batch (persistent batched solve)", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak if peak else None,
                     "peak_source": f"{peak_kind} hbm_gbs", "traffic": None,
                     "algorithmic_bytes_per_launch": inner_bytes / max(len(stats), 1),
                     "bytes_model": ("inner mrs steps only: each column's vectors, and J~ and Q of its matrix "
                                     "once per step for all its columns (the SpMM form's unique bytes)"),
                     "avg_launch_ms": total_ms / max(len(stats), 1), "launches": len(stats)},
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    bs.close()
    if dist:
        dist.destroy_process_group()


def batched_one_system_legs(pkg, torch, batch, nrhs, dev, stream, flush, mean_n):
    """Solves/s of the one-system path (asss_solve per matrix, its nrhs columns one after
    another) on every 16th matrix of the batch by size, FP64 throughout and mixed; each
    solve counted as n_m / mean n of a batch item, so the rate is comparable with the
    batched line's."""
    import numpy as np
    order = np.argsort([A.shape[0] for A, _ in batch])
    pick = [int(i) for i in order[8::16]]
    out = {}
    for prec in ("fp64", "mixed"):
        ms = 0.0
        units = 0.0
        solves = 0
        worst = 0.0
        its = []
        setup = 0.0
        for m in pick:
            A, B = batch[m]
            t0 = time.perf_counter()
            s = pkg.Solver(A, precision=prec, outer="fgmres", inner_tol=BATCH["inner_tol"], outer_tol=1e-8, k=20,
                           restart=24,
                           stream=stream.cuda_stream)
            torch.cuda.synchronize()
            setup += time.perf_counter() - t0
            Bd = torch.tensor(np.asfortranarray(B), device=dev)
            s.solve(Bd[:, 0].contiguous())   # warm-up
            for c in range(nrhs):
                bc = Bd[:, c].contiguous()
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                x, st = s.solve(bc)
                e1.record(stream)
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
                units += A.shape[0] / mean_n
                solves += 1
                its.append(st["outer_its"])
                if c == 0:
                    xh = x.cpu().numpy()
                    worst = max(worst, float(np.linalg.norm(B[:, 0] - A @ xh) / np.linalg.norm(B[:, 0])))
            s.close()
        out[prec] = {"value": units / (ms / 1000.0), "unit": UNIT, "solves_timed": solves,
                     "matrices": len(pick), "mean_outer_its": float(np.mean(its)),
                     "host_checked_max_relres": worst, "setup_s": round(setup, 3),
                     "sample": (f"asss_solve (one system, columns one after another), {prec}, every 16th of the "
                                f"{len(batch)} matrices by size x {nrhs} columns, each solve counted as n_m / mean n "
                                f"of a batch item; L2 flushed between solves")}
    return out


# ----------------------------------------------------------------------------
# gradients through the adjoint solve
# ----------------------------------------------------------------------------
def main_adjoint(args, world, rank, local):
    import numpy as np
    import torch

    import paper_2009_06954_gb300 as pkg
    from paper_2009_06954_gb300.binding import kernel_launches
    from workloads import dissipative_hamiltonian_3d

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    A, b, _ = dissipative_hamiltonian_3d(side=ADJ_SIDE, seed=4 + rank)
    n = A.shape[0]
    t0 = time.perf_counter()
    s = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=ADJ_INNER_TOL, outer_tol=1e-8, k=20,
                   stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    x, stf = s.solve(torch.tensor(b, device=dev))
    xs = torch.tensor(np.random.default_rng(44 + rank).standard_normal(n), device=dev)
    g = 2.0 * (x - xs)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        s.solve_adjoint(g, x)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    l0 = kernel_launches()
    prof_range(args, True)
    with ClockSampler(dev.index) as clk:
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            lam, dA, st = s.solve_adjoint(g, x)
            evs[k][1].record(stream)
            stats.append(st)
        torch.cuda.synchronize()
    launches = kernel_launches() - l0
    prof_range(args, False)
    if dist:
        dist.barrier()
    total_ms = sum(a.elapsed_time(c) for a, c in evs)
    tmax = reduce_max(total_ms, dist, dev)
    # the gradient is checked once on the host: A^T lambda = g to the outer tolerance
    lam_h = lam.cpu().numpy()
    g_h = g.cpu().numpy()
    adj_relres = float(np.linalg.norm(g_h - A.T @ lam_h) / np.linalg.norm(g_h))
    ok = all(st_["status"] == 0 for st_ in stats) and adj_relres <= 1e-8
    value = aggregate_rate(world, args.steps, tmax / 1000.0)
    # end to end from pinned host buffers (g and x in, lambda and dA out)
    gp = g.cpu().pin_memory()
    xp = x.cpu().pin_memory()
    lam_p = torch.empty(n, dtype=torch.float64).pin_memory()
    dA_p = torch.empty(s.nnz, dtype=torch.float64).pin_memory()
    s.solve_adjoint(gp, xp, lam=lam_p, dA=dA_p)   # untimed: allocates the staging of host x and dA once
    e2e_s = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        s.solve_adjoint(gp, xp, lam=lam_p, dA=dA_p)
        e2e_s += time.perf_counter() - t
    e2e_val = aggregate_rate(world, args.steps, reduce_max(e2e_s, dist, dev))
    inner_ms = sum(st_["t_inner_ms"] for st_ in stats)
    inner_bytes = sum(st_["inner_bytes"] for st_ in stats)
    inner_launches = sum(st_["inner_launches"] for st_ in stats)
    peak, peak_kind = _peaks()
    achieved = inner_bytes / (inner_ms / 1000.0) / 1e9 if inner_ms > 0 else 0.0
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:  # the oracle baseline is timed at N = 1 only
        try:
            cb = run_adjoint_cpu_baseline(10.0)
            cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        except Exception as e:
            cpu = {"value": None, "unit": "gradients/s", "cores": 1, "kind": "oracle", "sample": f"failed: {e}"[:300]}
    line = {
        "metric": "gradients/s (adjoint solve + dL/dA) to 1e-8 rel. residual", "value": value,
        "unit": "gradients/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32-inner/f64-outer", "data": "synthetic",
        "config": {"workload": ADJ_WORKLOAD, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "256 MB buffer written between steps (not timed)", "setup_s": round(t_setup, 3),
                   "forward_outer_its": stf["outer_its"], "adjoint_outer_its": stats[-1]["outer_its"],
                   "adjoint_inner_its_avg": round(stats[-1]["inner_its_avg"], 2),
                   "host_checked_adjoint_relres": adj_relres, "converged": ok},
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_val, "unit": "gradients/s", "h2d_bytes_per_step": 16 * n,
                "d2h_bytes_per_step": 8 * n + 8 * A.nnz},
        "roofline": {"bound": "hbm", "kernel": "k_mrs<float,20> (persistent mrs, transposed operator)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak if peak else None,
                     "peak_source": f"{peak_kind} hbm_gbs", "traffic": None,
                     "algorithmic_bytes_per_launch": inner_bytes / max(inner_launches, 1),
                     "avg_launch_ms": inner_ms / max(inner_launches, 1), "launches": inner_launches,
                     "others": phase_rooflines(stats, peak)},
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    s.close()
    if dist:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# many right-hand sides of the 100^3 system in one call (lockstep FGMRES blocks,
# multi-column mrs): the SpMM form of the inner solve
# ----------------------------------------------------------------------------
MULTI_NRHS = 8


def main_multi_rhs(args, world, rank, local):
    import numpy as np
    import torch

    import paper_2009_06954_gb300 as pkg
    from paper_2009_06954_gb300.binding import kernel_launches
    from workloads import dissipative_hamiltonian_3d

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    A, _, parts = dissipative_hamiltonian_3d(side=SIDE, seed=1)
    n = A.shape[0]
    t0 = time.perf_counter()
    solver = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=1e-6, outer_tol=1e-8, k=20,
                        stream=stream.cuda_stream, rhs_block=True)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    R = MULTI_NRHS
    Bh = np.asfortranarray(np.column_stack(_make_rhs(parts, n, 1 + rank, R)))
    Bd = torch.tensor(Bh.T.copy(), device=dev).T          # n x R column-major on the device
    Xd = torch.empty((R, n), dtype=torch.float64, device=dev).T
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        solver.solve(Bd, Xd)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    l0 = kernel_launches()
    prof_range(args, True)
    with ClockSampler(dev.index) as clk:
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            _, st = solver.solve(Bd, Xd)
            evs[k][1].record(stream)
            stats.append(st)
        torch.cuda.synchronize()
    launches = kernel_launches() - l0
    prof_range(args, False)
    total_ms = sum(a.elapsed_time(c) for a, c in evs)
    tmax = reduce_max(total_ms, dist, dev)
    value = world * R * args.steps / (tmax / 1000.0)
    X = Xd.cpu().numpy()
    relres = max(float(np.linalg.norm(Bh[:, c] - A @ X[:, c]) / np.linalg.norm(Bh[:, c])) for c in range(R))
    ok = all(s_["status"] == 0 for s_ in stats) and relres <= 1e-8
    Bp = torch.from_numpy(Bh.T.copy()).pin_memory()
    Xp = torch.empty((R, n), dtype=torch.float64).pin_memory()
    solver.solve(Bp.T, Xp.T)   # untimed: allocates the device copies of host B and X once
    e2e_s = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        solver.solve(Bp.T, Xp.T)
        e2e_s += time.perf_counter() - t
    e2e_val = world * R * args.steps / reduce_max(e2e_s, dist, dev)
    # the same right-hand sides solved one after another (the default path), timed alike
    solver.close()
    s1 = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=1e-6, outer_tol=1e-8, k=20,
                    stream=stream.cuda_stream)
    for _ in range(args.warmup):
        s1.solve(Bd, Xd)
    torch.cuda.synchronize()
    e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    seq_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e_a.record(stream)
        s1.solve(Bd, Xd)
        e_b.record(stream)
        torch.cuda.synchronize()
        seq_ms += e_a.elapsed_time(e_b)
    s1.close()
    seq_val = world * R * args.steps / (reduce_max(seq_ms, dist, dev) / 1000.0)
    inner_ms = sum(s_["t_inner_ms"] for s_ in stats)
    inner_bytes = sum(s_["inner_bytes"] for s_ in stats)
    inner_launches = sum(s_["inner_launches"] for s_ in stats)
    peak, peak_kind = _peaks()
    achieved = inner_bytes / (inner_ms / 1000.0) / 1e9 if inner_ms > 0 else 0.0
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32-inner/f64-outer", "data": "synthetic",
        "config": {"workload": (f"dh3d_100_rhs{R}: the dh3d_100 system with {R} right-hand sides per call "
                                f"(lockstep FGMRES, one multi-column FP32 mrs launch per Arnoldi step)"),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "256 MB buffer written between steps (not timed); working set > L2",
                   "setup_s": round(t_setup, 3), "rhs_per_call": R, "outer_its_max": stats[-1]["outer_its"],
                   "inner_its_avg": round(stats[-1]["inner_its_avg"], 2), "max_relres": relres, "converged": ok,
                   "one_after_another_solves_per_s": seq_val},
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 8 * n * R, "d2h_bytes_per_step": 8 * n * R},
        "roofline": {"bound": "hbm", "kernel": "k_mrs_multi<float,20> (8 right-hand sides per launch)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak if peak else None,
                     "peak_source": f"{peak_kind} hbm_gbs", "traffic": None,
                     "algorithmic_bytes_per_launch": inner_bytes / max(inner_launches, 1),
                     "bytes_model": "matrix and Q rows once per step for all columns, 28 B per live column",
                     "avg_launch_ms": inner_ms / max(inner_launches, 1), "launches": inner_launches,
                     "share_of_step": inner_ms / total_ms if total_ms else None},
        "clocks": clk.summary(),
        "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)
    solver.close()
    if dist:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# general power-law matrix: the SELL-C path at size (inner iterations/s)
# ----------------------------------------------------------------------------
def main_general(args, world, rank, local):
    import numpy as np
    import torch

    import paper_2009_06954_gb300 as pkg
    from paper_2009_06954_gb300.binding import kernel_launches
    from workloads import pattern_symmetrized, random_powerlaw

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    n = GENERAL["n"]
    A, b = random_powerlaw(n=n, seed=GENERAL["seed"] + rank)
    Sp = pattern_symmetrized(A)
    t0 = time.perf_counter()
    solver = pkg.Solver(A, s_pattern=Sp, precision="mixed", outer="fgmres", inner_tol=1e-6, outer_tol=1e-8,
                        outer_maxit=GENERAL["outer_steps"], lls_maxit=GENERAL["lls_maxit"], k=20,
                        stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    bd = torch.tensor(b, device=dev)
    x = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        solver.solve(bd, x)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    l0 = kernel_launches()
    prof_range(args, True)
    with ClockSampler(dev.index) as clk:
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            _, st = solver.solve(bd, x)
            evs[k][1].record(stream)
            stats.append(st)
        torch.cuda.synchronize()
    launches = kernel_launches() - l0
    prof_range(args, False)
    total_ms = sum(a.elapsed_time(c) for a, c in evs)
    tmax = reduce_max(total_ms, dist, dev)
    inner_its = sum(s_["inner_its_total"] for s_ in stats)
    inner_ms = sum(s_["t_inner_ms"] for s_ in stats)
    inner_bytes = sum(s_["inner_bytes"] for s_ in stats)
    inner_launches = sum(s_["inner_launches"] for s_ in stats)
    value = world * inner_its / (tmax / 1000.0)
    # end to end: b in from pinned host memory, x out, every step
    bp = torch.from_numpy(b).pin_memory()
    xp = torch.empty(n, dtype=torch.float64).pin_memory()
    solver.solve(bp, xp)   # untimed: allocates the device copies of host b and x once
    e2e_s, e2e_its = 0.0, 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, st = solver.solve(bp, xp)
        e2e_s += time.perf_counter() - t
        e2e_its += st["inner_its_total"]
    e2e_val = world * e2e_its / reduce_max(e2e_s, dist, dev)
    peak, peak_kind = _peaks()
    achieved = inner_bytes / (inner_ms / 1000.0) / 1e9 if inner_ms > 0 else 0.0
    relres = float(np.linalg.norm(b - A @ xp.numpy()) / np.linalg.norm(b))
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    line = {
        "metric": "inner mrs iterations/s (general power-law system, fixed outer steps)", "value": value,
        "unit": "mrs iterations/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32-inner/f64-outer", "data": "synthetic",
        "config": {"workload": GENERAL_WORKLOAD.format(n=n, steps=GENERAL["outer_steps"]),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "256 MB buffer written between steps (not timed); working set > L2",
                   "setup_s": round(t_setup, 2), "lls_its": solver.setup_stats["lls_its"],
                   "lls_relgrad": solver.setup_stats["lls_relgrad"], "lls_maxit": GENERAL["lls_maxit"],
                   "nnz_pattern": solver.setup_stats["nnz_pattern"], "r": solver.setup_stats["r"],
                   "sell_sigma": solver.setup_stats["sell_sigma"], "sell_split": solver.setup_stats["sell_split"],
                   "outer_its": stats[-1]["outer_its"], "inner_its_avg": round(stats[-1]["inner_its_avg"], 2),
                   "relres_after_step": relres, "status": stats[-1]["status"], "converged": False,
                   "solves_per_s": None},
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_val, "unit": "mrs iterations/s", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n},
        "roofline": {"bound": "hbm", "kernel": "k_mrs<float,20,SELL> (persistent mrs, SELL-C-sigma J~)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak if peak else None,
                     "peak_source": f"{peak_kind} hbm_gbs", "traffic": None,
                     "algorithmic_bytes_per_launch": inner_bytes / max(inner_launches, 1),
                     "avg_launch_ms": inner_ms / max(inner_launches, 1), "launches": inner_launches,
                     "share_of_step": inner_ms / total_ms if total_ms else None,
                     "others": phase_rooflines(stats, peak)},
        "clocks": clk.summary(),
        "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)
    solver.close()
    if dist:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle, timed as it stands on the host cores
# ----------------------------------------------------------------------------
def main_reference(args):
    """The oracle on a bounded sample of the workload.  The printed steps, warmup
    and ms_per_step are the ones that ran: for dh3d_100 a step is one round of
    concurrent sample solves (one per host core); for the batched and adjoint
    workloads a step is one sample solve (one thread)."""
    adj = args.workload == "adjoint_dh64"
    metric = "gradients/s (adjoint solve + dL/dA) to 1e-8 rel. residual" if adj else METRIC
    unit = "gradients/s" if adj else UNIT
    if args.workload == "batched_dh":
        cb = run_batched_cpu_baseline(120.0, batch_mean_n())
        workload = BATCH_WORKLOAD.format(count=BATCH["count"], items=BATCH["count"] * BATCH["nrhs"])
        steps, warm, ms = cb["solves"], 0, 1000.0 * cb["seconds"] / max(cb["solves"], 1)
        per_step = "one oracle solve of a sampled (matrix, column) item, counted as n_item / mean n of an item"
    elif args.workload == "general_2e6":
        line = {"impl": "reference", "metric": "inner mrs iterations/s (general power-law system, fixed outer steps)",
                "unavailable": ("the oracle's least-squares set-up (LSQR) of the 2e6-row power-law system does not "
                                "finish within a benchmark run; its solve phase is compared on 2e4 rows in the tests")}
        print(json.dumps(line), flush=True)
        return
    elif adj:
        cb = run_adjoint_cpu_baseline(120.0)
        workload = ADJ_WORKLOAD
        steps, warm, ms = cb["solves"], 0, 1000.0 * cb["seconds"] / max(cb["solves"], 1)
        per_step = f"one oracle adjoint solve + dL/dA at {ADJ_CPU_SIDE}^3, counted as n_sample / n of a gradient"
    else:
        cb = run_cpu_baseline(args.steps, max(0, min(args.warmup, 1)), 120.0)
        workload = dh_workload()
        steps, warm = len(cb["rounds"]), cb["warmup"]
        ms = 1000.0 * sum(cb["rounds"]) / max(steps, 1)
        per_step = (f"{cb['procs']} concurrent oracle solves at {CPU_SAMPLE_SIDE}^3 (n = {cb['n_sample']}), each "
                    f"counted as n_sample / n of a 100^3 solve")
    line = {"impl": "reference", "metric": metric, "value": cb["value"], "unit": unit, "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload, "reference": "FP64 CPU oracle (oracle/) as it stands, host cores",
                       "step": per_step, "requested_steps": args.steps, "requested_warmup": args.warmup},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": cb["value"], "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if "one_thread_value" in cb:
        line["cpu_baseline"]["one_thread_value"] = cb["one_thread_value"]
    print(json.dumps(line), flush=True)


FP64_PEAK_TFLOPS = 152 * 2.07e9 * 4 / 1e12   # SMs x max SM clock x FP64 flops per clock per SM (2 FMA)


def phase_rooflines(stats, peak):
    """Roofline entries of the outer operator and the fused Arnoldi step, from the CUDA
    events the library records around them inside the timed solves."""
    out = []
    t_op = sum(s_["t_op_ms"] for s_ in stats)
    if t_op > 0:
        b = sum(s_["op_bytes"] for s_ in stats)
        f = sum(s_["op_flops"] for s_ in stats)
        calls = sum(s_["op_calls"] for s_ in stats)
        ach = b / (t_op / 1000.0) / 1e9
        tf = f / (t_op / 1000.0) / 1e12
        out.append({"kernel": "k_dia_spmv x2 (outer operator W Abar S W v)" if DH["factor"] == "diag" else
                    "outer operator with triangular solves per colour", "bound": "hbm", "achieved": ach,
                    "peak": peak, "unit": "GB/s", "frac": ach / peak if peak else None, "calls": calls,
                    "bytes_per_call": b / max(calls, 1), "ms_per_call": t_op / max(calls, 1),
                    "fp64_tflops": tf, "fp64_frac": tf / FP64_PEAK_TFLOPS,
                    "note": "CUDA events around each application inside the timed solves; one FP64 FMA per "
                            "stored value, so the FP64 pipe (fp64_frac) bounds it about as much as HBM"})
    t_or = sum(s_["t_orth_ms"] for s_ in stats)
    if t_or > 0:
        f = sum(s_["orth_flops"] for s_ in stats)
        b = sum(s_["orth_bytes"] for s_ in stats)
        calls = sum(s_["orth_calls"] for s_ in stats)
        tf = f / (t_or / 1000.0) / 1e12
        gb = b / (t_or / 1000.0) / 1e9
        out.append({"kernel": "k_arnoldi_orth (fused CGS2 Arnoldi step, FP64)", "bound": "alu", "achieved": tf,
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": tf / FP64_PEAK_TFLOPS, "calls": calls,
                    "ms_per_call": t_or / max(calls, 1), "hbm_achieved_gbs": gb,
                    "hbm_frac": gb / peak if peak else None,
                    "note": "FP64 pipe: 4(j+1) FMAs per row at step j; peak = 152 SMs x 2.07 GHz x 4 flops"})
    return out


def rel_error_legs(pkg, dev, stream, xo_path, legs):
    """Relative error ||x - x_oracle|| / ||x_oracle|| of each GPU leg on the instance the
    oracle solved (the CPU_SAMPLE_SIDE^3 step of the same generator, first rhs)."""
    import numpy as np
    import torch

    from workloads import dissipative_hamiltonian_3d
    xo = np.load(xo_path)
    A, _, parts = dissipative_hamiltonian_3d(side=CPU_SAMPLE_SIDE, seed=1)
    b = _make_rhs(parts, A.shape[0], 1, 1)[0]
    out = {}
    for name, prec in legs:
        s = pkg.Solver(A, precision=prec, outer="fgmres", inner_tol=DH["inner_tol"], outer_tol=1e-8, k=20,
                       stream=stream.cuda_stream, factor=DH["factor"])
        x, st = s.solve(torch.tensor(b, device=dev))
        xh = x.cpu().numpy()
        out[name] = {"rel_error": float(np.linalg.norm(xh - xo) / np.linalg.norm(xo)),
                     "relres": float(np.linalg.norm(b - A @ xh) / np.linalg.norm(b)),
                     "outer_its": st["outer_its"]}
        s.close()
    out["instance"] = f"{CPU_SAMPLE_SIDE}^3 (n = {A.shape[0]}), the oracle's x for the same b"
    return out


# ----------------------------------------------------------------------------
# main
# ----------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="asss", choices=["asss", "reference"])
    ap.add_argument("--cpu-worker", action="store_true")
    ap.add_argument("--budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--q-storage", default="f32", choices=["f32", "bf16"],
                    help="storage of the Lanczos basis read by the FP32 inner solve")
    ap.add_argument("--workload", default="dh3d_100", choices=["dh3d_100", "batched_dh", "adjoint_dh64", "general_2e6", "dh3d_100_rhs8"],
                    help="dh3d_100: one 1e6-unknown system; batched_dh: 256 systems x 32 right-hand sides; "
                         "adjoint_dh64: gradients through the adjoint solve")
    ap.add_argument("--procs", type=int, default=0, help="(CPU worker) processes of the oracle pool")
    ap.add_argument("--xout", default="", help="(CPU worker) where to save the oracle's x of the first rhs")
    ap.add_argument("--no-fp64-leg", action="store_true", help="skip the FP64-GPU comparison solve")
    ap.add_argument("--cuda-profiler-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--general-n", type=int, default=GENERAL["n"], help="rows of the general_2e6 workload")
    ap.add_argument("--factor", default=DH["factor"], choices=["diag", "ildl0"],
                    help="L~ of the dh3d_100 workload: 1x1 diagonal, or the no-fill incomplete L D L^T")
    ap.add_argument("--inner-tol", type=float, default=DH["inner_tol"],
                    help="mrs tolerance of the dh3d_100 workload (FGMRES takes inexact inner solves)")
    ap.add_argument("--batch-count", type=int, default=BATCH["count"],
                    help="systems in the batched workload (smaller counts for profiling captures)")
    args = ap.parse_args()
    BATCH["count"] = args.batch_count
    GENERAL["n"] = args.general_n
    DH["inner_tol"] = args.inner_tol
    DH["factor"] = args.factor

    if args.cpu_worker:
        if args.workload == "batched_dh":
            batched_worker(args.budget, max(1, args.procs))
        elif args.workload == "adjoint_dh64":
            adjoint_worker(args.budget, max(1, args.procs))
        else:
            cpu_worker(CPU_SAMPLE_SIDE, args.steps, args.warmup, args.budget, max(1, args.procs), args.xout)
        return

    world, rank, local = rank_env()
    if args.workload == "batched_dh" and args.impl != "reference":
        main_batched(args, world, rank, local)
        return
    if args.workload == "adjoint_dh64" and args.impl != "reference":
        main_adjoint(args, world, rank, local)
        return
    if args.workload == "general_2e6" and args.impl != "reference":
        main_general(args, world, rank, local)
        return
    if args.workload == "dh3d_100_rhs8" and args.impl != "reference":
        main_multi_rhs(args, world, rank, local)
        return

    if args.impl == "reference":
        if rank != 0:
            return
        main_reference(args)
        return

    import numpy as np
    import torch

    import paper_2009_06954_gb300 as pkg
    from paper_2009_06954_gb300.binding import kernel_launches
    from workloads import dissipative_hamiltonian_3d

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()

    A, b0, parts = dissipative_hamiltonian_3d(side=SIDE, seed=1)
    n = A.shape[0]
    t0 = time.perf_counter()
    solver = pkg.Solver(A, precision="mixed", outer="fgmres", inner_tol=DH["inner_tol"], outer_tol=1e-8, k=20,
                        q_bf16=args.q_storage == "bf16", stream=stream.cuda_stream, factor=DH["factor"])
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    rhs_h = _make_rhs(parts, n, 1 + rank, 4)
    rhs = [torch.tensor(r, device=dev) for r in rhs_h]
    x = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    for w in range(args.warmup):
        solver.solve(rhs[w % 4], x)
    torch.cuda.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = kernel_launches()
    print(f"[bench] kernel launches before the timed region: {l0}", file=sys.stderr, flush=True)
    prof_range(args, True)
    with ClockSampler(dev.index) as clk:
        for s in range(args.steps):
            flush.zero_()
            evs[s][0].record(stream)
            _, st = solver.solve(rhs[s % 4], x)
            evs[s][1].record(stream)
            stats.append(st)
        torch.cuda.synchronize()
    launches = kernel_launches() - l0
    prof_range(args, False)
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    tmax = reduce_max(total_ms, dist, dev)
    relres = max(s_["relres"] for s_ in stats)
    ok = all(s_["status"] == 0 for s_ in stats) and relres <= 1e-8
    value = aggregate_rate(world, args.steps, tmax / 1000.0)

    # end to end through the C ABI with pinned host buffers (copies in the timed region)
    bh = [torch.tensor(r).pin_memory() for r in rhs_h]
    xh = torch.empty(n, dtype=torch.float64).pin_memory()
    solver.solve(bh[0], xh)   # untimed: allocates the device copies of host b and x once
    e2e_s = 0.0
    for s in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        solver.solve(bh[s % 4], xh)
        e2e_s += time.perf_counter() - t
    e2e_val = aggregate_rate(world, args.steps, reduce_max(e2e_s, dist, dev))

    # the same solves in FP64 throughout (inner mrs in FP64 too), same options and
    # stopping rule, timed the same way: the precision form's comparison
    fp64 = None
    if not args.no_fp64_leg:
        solver.close()   # frees the mixed handle's device memory first
        t0 = time.perf_counter()
        s64 = pkg.Solver(A, precision="fp64", outer="fgmres", inner_tol=DH["inner_tol"], outer_tol=1e-8, k=20,
                         stream=stream.cuda_stream, factor=DH["factor"])
        torch.cuda.synchronize()
        t_setup64 = time.perf_counter() - t0
        for w in range(args.warmup):
            s64.solve(rhs[w % 4], x)
        torch.cuda.synchronize()
        evs64 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                 for _ in range(args.steps)]
        st64 = []
        for s in range(args.steps):
            flush.zero_()
            evs64[s][0].record(stream)
            _, st = s64.solve(rhs[s % 4], x)
            evs64[s][1].record(stream)
            st64.append(st)
        torch.cuda.synchronize()
        ms64 = reduce_max(sum(a.elapsed_time(b) for a, b in evs64), dist, dev)
        fp64 = {"value": aggregate_rate(world, args.steps, ms64 / 1000.0), "unit": UNIT,
                "ms_per_step": ms64 / args.steps,
                "inner_its_per_s": world * sum(s_["inner_its_total"] for s_ in st64) / (ms64 / 1000.0),
                "outer_its": st64[-1]["outer_its"], "inner_its_avg": round(st64[-1]["inner_its_avg"], 2),
                "max_relres": max(s_["relres"] for s_ in st64),
                "converged": all(s_["status"] == 0 for s_ in st64) and max(s_["relres"] for s_ in st64) <= 1e-8,
                "setup_s": round(t_setup64, 3),
                "mrs_avg_launch_ms": sum(s_["t_inner_ms"] for s_ in st64) / max(sum(s_["inner_launches"] for s_ in st64), 1)}
        s64.close()

    inner_ms = sum(s_["t_inner_ms"] for s_ in stats)
    inner_bytes = sum(s_["inner_bytes"] for s_ in stats)
    inner_launches = sum(s_["inner_launches"] for s_ in stats)
    peak, peak_kind = _peaks()
    achieved = inner_bytes / (inner_ms / 1000.0) / 1e9 if inner_ms > 0 else 0.0
    others = phase_rooflines(stats, peak)
    tr = _traffic_record() if DH["factor"] == "diag" else None
    traffic = tr.get("dram_bytes_per_launch") if tr is not None else None

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    cpu = None
    rel_err = None
    if not args.no_cpu_baseline and world == 1:  # the oracle baseline is timed at N = 1 only
        xo_path = os.path.join(tempfile.mkdtemp(prefix="asss_bench_"), "x_oracle.npy")
        try:
            cb = run_cpu_baseline(500, 1, 15.0, xout=xo_path)
            cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "one_thread_value")}
        except Exception as e:  # reported, never silently substituted
            cpu = {"value": None, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                   "sample": f"failed: {e}"[:300]}
        if os.path.exists(xo_path):
            legs = [("mixed", "mixed")] + ([] if args.no_fp64_leg else [("fp64", "fp64")])
            rel_err = rel_error_legs(pkg, dev, stream, xo_path, legs)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32-inner/f64-outer", "data": "synthetic",
        "config": {"workload": dh_workload(), "inner_tol": DH["inner_tol"], "factor": DH["factor"],
                   "factor_colours": solver.setup_stats["factor_colours"], "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "256 MB buffer written between steps (not timed); working set > L2",
                   "setup_s": round(t_setup, 3), "lls_its": solver.setup_stats["lls_its"],
                   "outer_its": stats[-1]["outer_its"], "inner_its_avg": round(stats[-1]["inner_its_avg"], 2),
                   "max_relres": relres, "converged": ok, "r": solver.setup_stats["r"],
                   "k_eff": solver.setup_stats["k_eff"], "q_storage": args.q_storage,
                   "inner_its_per_s": world * sum(s_["inner_its_total"] for s_ in stats) / (tmax / 1000.0),
                   "fp64_gpu": fp64, "rel_error_vs_oracle": rel_err},
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n},
        "roofline": {"bound": "hbm", "kernel": "k_mrs<float,20> (persistent mrs)" if DH["factor"] == "diag" else
                     "k_mrs<float,20,factored> (persistent mrs, J~ by triangular solves per colour)", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak if peak else None,
                     "peak_source": f"{peak_kind} hbm_gbs", "traffic": traffic,
                     "algorithmic_bytes_per_launch": inner_bytes / max(inner_launches, 1),
                     "avg_launch_ms": inner_ms / max(inner_launches, 1), "launches": inner_launches,
                     "share_of_step": inner_ms / total_ms if total_ms else None, "others": others},
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    solver.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
