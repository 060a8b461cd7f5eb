"""Benchmark: KKT solves/sec on a same-pattern synthetic power-grid KKT sequence.

One step = one pass of the hot path over one matrix of the sequence:
kkt_step -- the value gather, the numeric LU refactorization on the fixed
pattern and pivots with the forward sweep fused into it, the backward sweep,
the residual and FGMRES(20) with CGS2 until NRBE <= 1e-12.  Matrices cycle
k = 0..M-1 over the sequence.

The headline workload is the largest single-GPU configuration (kkt70000:
70,000 buses, n = 1.76M, nnz = 20.4M, 20 matrices).  The smaller
configurations (kkt200, kkt2000, kkt10000) are measured with the same
protocol and reported under `per_config`; their host analysis runs while
the headline's (minutes on one core) proceeds on another thread.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank runs its own
instance of the workload (independent replicas, weak scaling; one KKT
system does not shard, so there is no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "kkt70000"
PER_CONFIG = "kkt200,kkt2000,kkt10000"
TOL = 1e-12
RESTART = 20
L2_FLUSH_BYTES = 256 << 20   # larger than the 126 MB L2
METRIC = "KKT solves/sec (refactor+FGMRES to NRBE<=1e-12)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--per-config", default=PER_CONFIG, help="comma-separated smaller configs (none = skip)")
    ap.add_argument("--per-config-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="bounded oracle sample for cpu_baseline")
    ap.add_argument("--ref-seconds", type=float, default=4.0, help="oracle sample per step of --impl reference")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="factor precision of the headline line")
    ap.add_argument("--no-mixed", action="store_true", help="skip the side-by-side other-precision run")
    ap.add_argument("--mixed-steps", type=int, default=6)
    ap.add_argument("--mixed-cycles", type=int, default=2,
                    help="restart cycles the FP32 preconditioner gets before the FP64 fallback")
    ap.add_argument("--no-trace", action="store_true", help="skip the refactorization trace (critical path)")
    ap.add_argument("--trisolve", default="auto", choices=["auto", "global"],
                    help="triangular-solve schedule of the headline solver (global: the whole-GPU kernels)")
    ap.add_argument("--serve-instances", type=int, default=8,
                    help="independent kkt2000 sequences of the serving measurement (0 = skip)")
    ap.add_argument("--serve-steps", type=int, default=10)
    ap.add_argument("--serve-batch", type=int, default=8, help="steps per batched call of the server (0 = off)")
    ap.add_argument("--serve-c4", type=int, default=256,
                    help="mixed-size serving run: this many instances, bus counts uniform in "
                         "[200, --serve-c4-buses], Poisson arrivals, each instance's steps closed-loop (0 = skip)")
    ap.add_argument("--serve-c4-buses", type=int, default=5000)
    ap.add_argument("--serve-c4-rate", type=float, default=50.0, help="instance arrivals per second")
    ap.add_argument("--serve-c4-steps", type=int, default=30)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(units: float, seconds: float, world: int):
    """Whole-job throughput: units summed over ranks / slowest rank's time."""
    if world == 1:
        return units, seconds
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([units, seconds], dtype=torch.float64, device=dev)
    u = t[:1].clone()
    s = t[1:].clone()
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()), float(s.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if not self.p:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("kernels.cuh", "trsv_row.cuh"):
        with open(os.path.join(ROOT, "paper_2401_13926_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload, kernel):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary, or None when the kernel sources changed since that capture."""
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}.txt")
    try:
        rows = {}
        for line in open(path):
            if line.strip() and not line.startswith("#"):
                k, v = line.split("=", 1)
                rows[k.strip()] = v.strip()
        if rows.get("kernel_source_sha256_16") != kernel_source_hash():
            return None
        return float(rows[kernel + ".dram_bytes_per_launch"])
    except Exception:
        return None


# ------------------------------------------------------------ algorithmic bytes
# Per unit of work, FP64 factors (8-byte values, 4-byte indices); l = nnz of
# strict L, u = nnz of U with its diagonal, a = nnz(K), n rows.
def bytes_refactor(a, l, u, n, fused=True, vsize=8):
    """Gather + refactorization: A values (8a) and the gather map (4a) read,
    factor values written (vsize (l+u)), the factor pattern (4 (l+u)) and
    row pointers (8n) read; with the forward sweep fused in, that sweep's
    factor reads (vsize+4) l and its vectors (b, P, y, re-arm: 36n)."""
    b = 12 * a + (vsize + 4) * (l + u) + 8 * n
    if fused:
        b += (vsize + 4) * l + 36 * n
    return b


def bytes_usolve(u, n, vsize=8):
    return (vsize + 4) * u + 44 * n


def bytes_lsolve(l, n, vsize=8):
    return (vsize + 4) * l + 36 * n


def bytes_spmv(a, n):
    return 12 * a + 20 * n


def bytes_solve_step(a, l, u, n, iters, vsize=8):
    """Everything after the refactorization in one kkt_step with `iters`
    Arnoldi steps in one cycle: the backward sweep, the residual of x0, and
    per Arnoldi step j both sweeps, a product with K, CGS2 (two projections:
    32 (j+1) n + 32 n) and the normalisation (24 n) and the stored z (8 n);
    at the cycle end x += Z y (8 iters n + 16 n) and the true residual."""
    b = bytes_usolve(u, n, vsize) + bytes_spmv(a, n)
    for j in range(iters):
        b += bytes_lsolve(l, n, vsize) + bytes_usolve(u, n, vsize) + bytes_spmv(a, n)
        b += 32 * (j + 1) * n + 32 * n + 24 * n + 8 * n
    if iters:
        b += 8 * iters * n + 16 * n + bytes_spmv(a, n)
    return b


def step_bytes(info, n, nnz, iters, vsize=8):
    l, u = info["nnz_l"], info["nnz_u"]
    return bytes_refactor(nnz, l, u, n, True, vsize) + bytes_solve_step(nnz, l, u, n, iters, vsize)


def roofline(phases, info, n, nnz, steps, workload):
    """Roofline of the dominant kernel group over the timed region, from the
    library's own CUDA events (on the context's stream).  Bound: HBM (the
    path is sparse; no tensor cores), algorithmic bytes per launch as above
    divided by the group's average launch time."""
    hbm, peak_kind = peaks()
    l, u = info["nnz_l"], info["nnz_u"]
    ref_ms = phases["gather"][0] + phases["refactor"][0]
    ref_n = max(phases["gather"][1], 1)
    groups = {"refactorization": (ref_ms, ref_n), "lsolve": phases["lsolve"], "usolve": phases["usolve"]}
    dom = max(groups, key=lambda g: groups[g][0])
    ms, cnt = groups[dom]
    per_ms = ms / max(cnt, 1)
    if dom == "refactorization":
        bytes_ = bytes_refactor(nnz, l, u, n, True)
        kern = "k_refactor_rows<double,1>"
        names = "k_gather + k_refactor_rows (forward sweep fused)"
    elif dom == "usolve":
        bytes_, kern, names = bytes_usolve(u, n), "k_trsv_cluster<0>", "backward sweep"
    else:
        bytes_, kern, names = bytes_lsolve(l, n), "k_trsv_cluster<1>", "forward sweep"
    ach = bytes_ / (per_ms * 1e-3) / 1e9
    out = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
           "traffic": measured_traffic(workload, kern), "peak_kind": f"{peak_kind} hbm_gbs",
           "kernel_group": dom, "kernels": names, "dominant_kernel": kern, "bytes_per_launch": bytes_,
           "ms_per_launch": per_ms,
           "phase_ms_per_step": {p: round(phases[p][0] / steps, 4) for p in phases},
           "phase_launches": {p: phases[p][1] for p in phases}}
    if dom == "refactorization":
        out["fp64_gflops"] = 2.0 * info["refactor_updates"] / (per_ms * 1e-3) / 1e9
    return out


# -------------------------------------------------------------------- oracle
def host_cpu():
    """CPU model and core count of the host (for the CPU-baseline record)."""
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"cpu_model": model, "nproc": os.cpu_count()}


class pinned_core:
    """Run the calling thread on one CPU (the oracle is single-threaded)."""

    def __enter__(self):
        self.saved = None
        try:
            self.saved = os.sched_getaffinity(0)
            os.sched_setaffinity(0, {min(self.saved)})
        except (AttributeError, OSError):
            self.saved = None

    def __exit__(self, *a):
        if self.saved:
            os.sched_setaffinity(0, self.saved)


def oracle_solve_estimate(O, seq, k, P, Q, totals, seconds):
    """Seconds the oracle takes for one solve of matrix k, from a bounded
    sample: the oracle's refactorization (on P, Q) runs for `seconds`; if it
    finishes, that is the time; otherwise its cost profile (checkpoints every
    256 columns) is fitted as time = a cols + b multiply-adds + c stored
    entries (non-negative least squares) and extrapolated to the whole
    refactorization (totals: n, multiply-adds, entries).  The oracle's
    triangular solves and FGMRES are not sampled (about 2% of its solve time
    on kkt2000).  Returns (seconds per solve, sample description)."""
    from scipy.optimize import nnls
    v = seq.values(k % seq.M)
    cols, madds, dt, marks = O.refactor_sample(seq.n, seq.rowptr, seq.colind, v, P, Q, seconds)
    if cols >= seq.n:
        return dt, {"cols": cols, "madds": madds, "seconds": dt, "extrapolated": False}
    d = np.diff(np.vstack([np.zeros((1, 4)), marks]), axis=0)
    coef, _ = nnls(d[:, :3], d[:, 3])
    est = float(coef @ np.array(totals, dtype=np.float64))
    est = max(est, dt)
    return est, {"cols": cols, "madds": madds, "seconds": dt, "extrapolated": True,
                 "frac_madds": madds / totals[1]}


def workload_config(seq):
    return {
        "workload": f"{seq.cfg.name}: synthetic {seq.nbus}-bus grid KKT [[H+Dx,J^T],[J,-Dy]], "
                    f"n={seq.n}, nnz={seq.nnz}, {seq.M}-matrix same-pattern sequence, "
                    f"Dx spread widening 1e+-{seq.cfg.s_first:g}..1e+-{seq.cfg.s_last:g}, "
                    f"FGMRES({RESTART}) to NRBE<={TOL:g}, FP64",
        "n": seq.n, "nnz": seq.nnz, "sequence": seq.M, "restart": RESTART, "tol": TOL,
        "l2": "flushed between timed steps (256 MiB write, outside the per-step events)",
        "call": "kkt_step: refactor + solve, forward sweep fused into the refactorization",
    }


def run_reference(args):
    """The oracle as it stands, single thread, on the headline workload:
    each step is a bounded sample of one matrix's solve (oracle_solve_estimate),
    on the ordering and pivots of the library's host analysis (kkt_host_analyze,
    no GPU; the oracle's own exact minimum-degree ordering does not finish on
    the largest configuration in hours)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import paper_2401_13926_b300 as K
    from oracle import oracle as O
    from paper_2401_13926_b300.workload import KKTSequence
    seq = KKTSequence(args.workload)
    t = time.perf_counter()
    P, Q, st = K.host_analyze(seq.rowptr, seq.colind, seq.values(0))
    t_an = time.perf_counter() - t
    totals = (seq.n, st["refactor_updates"], st["nnz_l"] + st["nnz_u"])
    est, samples = [], []
    with pinned_core():
        for i in range(args.warmup + args.steps):
            e, smp = oracle_solve_estimate(O, seq, i, P, Q, totals, args.ref_seconds)
            if i >= args.warmup:
                est.append(e)
                samples.append(smp)
    tot = sum(est)
    v = len(est) / tot
    ext = any(s["extrapolated"] for s in samples)
    desc = (f"{len(est)} matrices of the {args.workload} sequence, each a ~{args.ref_seconds:g} s run of the oracle "
            f"refactorization on the library host analysis' P, Q"
            + (f" (median {100 * np.median([s.get('frac_madds', 1) for s in samples]):.2g}% of its multiply-adds), "
               f"extrapolated to the whole refactorization by a fitted cost model" if ext else ", run to completion")
            + f"; triangular solves and FGMRES not sampled; analysis ({t_an:.0f} s) excluded; single thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / len(est), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(seq),
        "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", **host_cpu(), "sample": desc},
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- ours
def timed_steps(solver, vals, rhs, x, steps, M, flush, stream, allow_nc=False):
    """`steps` kkt_step calls cycling over the M matrices, CUDA events on the
    solver's stream around each, the L2 flushed before each (outside the
    events).  Returns (per-step ms, iterations, NRBE, statuses)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    iters, nrbes, st = [], [], []
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[i][0].record(stream)
        try:
            _, it, nr = solver.step(vals[i % M], rhs[i % M], x=x, tol=TOL, allow_not_converged=allow_nc)
            code = solver.last_status
        except Exception as e:   # a failed step of a leg that reports failures (allow_nc)
            if not allow_nc or not hasattr(e, "code"):
                raise
            it, nr, code = -1, float("nan"), e.code
        ev[i][1].record(stream)
        iters.append(it)
        nrbes.append(nr)
        st.append(code)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], iters, nrbes, st


def measure_config(K, name, steps, warmup, flush, device, rank):
    """The headline protocol on a smaller configuration: analysis (not
    timed), `warmup` steps, `steps` timed kkt_step calls; solves/s,
    latency percentiles, NRBE, and the HBM fraction of the algorithmic bytes
    per solve (refactorization + everything the solve touches)."""
    import torch
    from paper_2401_13926_b300.workload import KKTSequence
    seq = KKTSequence(name, instance=rank)
    stream = torch.cuda.Stream(device=device)
    s = K.KKTSolver(restart=RESTART, device=device, stream=stream, timing=True)
    t = time.perf_counter()
    s.analyze(seq.rowptr, seq.colind, values0=seq.values(0))
    t_an = time.perf_counter() - t
    info = s.info()
    with torch.cuda.stream(stream):
        vals = [torch.from_numpy(seq.values(k)).cuda() for k in range(seq.M)]
        rhs = [torch.from_numpy(seq.rhs(k, vals[k].cpu().numpy())[0]).cuda() for k in range(seq.M)]
        x = torch.empty(seq.n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    timed_steps(s, vals, rhs, x, warmup, seq.M, flush, stream)
    s.phase_times(reset=True)
    ms, iters, nrbes, _ = timed_steps(s, vals, rhs, x, steps, seq.M, flush, stream)
    phases = s.phase_times(reset=True)
    hbm, _ = peaks()
    tot_bytes = sum(step_bytes(info, seq.n, seq.nnz, it) for it in iters)
    tot_s = sum(ms) / 1000.0
    out = {"value": steps / tot_s, "unit": "solves/s", "steps": steps, "n": seq.n, "nnz": seq.nnz,
           "ms_per_step": 1000 * tot_s / steps,
           "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
           "max_nrbe": float(max(nrbes)), "iters_mean": float(np.mean(iters)),
           "hbm": {"achieved_gbs": tot_bytes / tot_s / 1e9, "frac": tot_bytes / tot_s / 1e9 / hbm,
                   "bytes_per_solve": tot_bytes / steps},
           "refactorization_ms": (phases["gather"][0] + phases["refactor"][0]) / steps,
           "usolve_ms": phases["usolve"][0] / steps,
           "analyze_s": t_an, "nnz_l": info["nnz_l"], "nnz_u": info["nnz_u"],
           "levels_l": info["levels_l"], "levels_u": info["levels_u"],
           "refactor_updates": info["refactor_updates"]}
    s.close()
    return out


def serve_measure(K, args, rank, N):
    """Throughput and latency of N independent kkt2000 sequences served
    together: every instance's steps are submitted at once (closed loop, the
    server runs one step per instance at a time, up to --serve-batch of them
    as one batched call), host arrays in and out."""
    from paper_2401_13926_b300.workload import KKTSequence
    S = args.serve_steps
    base = KKTSequence("kkt2000", instance=1000 * (rank + 1), steps=S)
    seqs = [base.reseeded(1000 * (rank + 1) + i) for i in range(N)]
    data = [[(q.values(k), q.rhs(k, q.values(k))[0]) for k in range(S)] for q in seqs]
    srv = K.KKTServer(batch=args.serve_batch, restart=RESTART)
    ids = [srv.open(q.rowptr, q.colind, q.values(0)) for q in seqs]
    for i in range(N):   # warm-up: one step per instance
        srv.wait(srv.submit(ids[i], *data[i][0], tol=TOL)[0])
    b0 = srv.info()["batches"]
    t0 = time.perf_counter()
    tickets = [srv.submit(ids[i], *data[i][k], tol=TOL)[0] for k in range(S) for i in range(N)]
    res = [srv.wait(t)[1] for t in tickets]
    dt = time.perf_counter() - t0
    nb = srv.info()["batches"] - b0
    srv.close()
    lat = np.array([r["queue_ms"] + r["run_ms"] for r in res])
    run = np.array([r["run_ms"] for r in res])
    return {"workload": "kkt2000", "value": N * S / dt, "unit": "solves/s", "instances": N, "steps_per_instance": S,
            "batch": args.serve_batch, "batched_calls": nb, "mean_batch": N * S / max(nb, 1),
            "converged": int(sum(r["status"] == 0 for r in res)),
            "max_nrbe": float(max(r["nrbe"] for r in res)),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "call_ms": {"p50": float(np.percentile(run, 50)), "p99": float(np.percentile(run, 99))},
            "timing": "host wall clock, submit of all steps to the last completion; includes host<->device "
                      "copies of values, b and x"}


def serve_c4(K, args, rank):
    """The mixed-size serving workload: --serve-c4 instances whose bus counts
    are uniform in [200, --serve-c4-buses] (32 grids, each shared by 1/32 of
    the instances with values of their own), arriving at Poisson times
    (--serve-c4-rate per second).  Each client opens its instance on arrival
    (host analysis in its own thread, then admission by device memory) and
    runs its sequence closed-loop (step k+1 submitted when step k returns),
    --serve-c4-steps steps cycling over 3 generated matrices of its sequence
    (the first, middle and last: the spread widens along it).  Step latency
    is submission to completion; the open time is reported apart."""
    from paper_2401_13926_b300.workload import KKTSequence
    rng = np.random.default_rng(7000 + rank)
    N, S = args.serve_c4, args.serve_c4_steps
    G = min(32, N)
    grid_buses = rng.integers(200, args.serve_c4_buses + 1, size=G)
    grids = [KKTSequence("kkt2000", instance=5000 + 100 * rank + g, buses=int(nb), steps=S)
             for g, nb in enumerate(grid_buses)]
    seqs = [grids[i % G].reseeded(6000 + 1000 * rank + i) for i in range(N)]
    ks = [0, (S - 1) // 2, S - 1]
    data = []
    for q in seqs:
        vs = [q.values(k) for k in ks]
        data.append([(v, q.rhs(k, v)[0]) for k, v in zip(ks, vs)])
    srv = K.KKTServer(batch=args.serve_batch, restart=RESTART)
    arrivals = np.cumsum(rng.exponential(1.0 / args.serve_c4_rate, size=N))
    results = [[] for _ in range(N)]
    opens = [0.0] * N
    errors = []

    def client(i, t_start):
        try:
            delay = t_start + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            t = time.perf_counter()
            inst = srv.open(seqs[i].rowptr, seqs[i].colind, seqs[i].values(0))
            opens[i] = time.perf_counter() - t
            for k in range(S):
                tk, _ = srv.submit(inst, *data[i][k % 3], tol=TOL)
                results[i].append(srv.wait(tk)[1])
            srv.close_instance(inst)
        except Exception as e:   # reported, not raised from the thread
            errors.append(repr(e))

    t0 = time.perf_counter()
    threads = [threading.Thread(target=client, args=(i, t0)) for i in range(N)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    dt = time.perf_counter() - t0
    info = srv.info()
    srv.close()
    res = [r for rr in results for r in rr]
    lat = np.array([r["queue_ms"] + r["run_ms"] for r in res])
    return {"value": len(res) / dt, "unit": "solves/s", "instances": N, "steps_per_instance": S,
            "buses_range": [200, args.serve_c4_buses], "grids": G, "n": [int(g.n) for g in grids],
            "arrival_rate_per_s": args.serve_c4_rate, "batch": args.serve_batch, "batched_calls": info["batches"],
            "precision": "fp64", "errors": errors[:3],
            "converged": int(sum(r["status"] == 0 for r in res)), "solves": len(res),
            "max_nrbe": float(max(r["nrbe"] for r in res)) if res else None,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "open_s": {"p50": float(np.percentile(opens, 50)), "p99": float(np.percentile(opens, 99))},
            "timing": "host wall clock from the first arrival to the last completion (opens included)"}


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    import paper_2401_13926_b300 as K
    from paper_2401_13926_b300.workload import KKTSequence

    t_job = time.perf_counter()
    seq = KKTSequence(args.workload, instance=rank)
    stream = torch.cuda.Stream()
    solver = K.KKTSolver(restart=RESTART, device=local, stream=stream, timing=True, precision=args.precision,
                         trisolve=args.trisolve)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    # the headline's host analysis (ordering + pivoting factorization, one
    # core, minutes at kkt70000) on its own thread; the smaller
    # configurations are measured on the GPU meanwhile
    an_err = []

    def analyse():
        try:
            solver.analyze(seq.rowptr, seq.colind, values0=seq.values(0))
        except Exception as e:   # re-raised on the main thread
            an_err.append(e)

    th = threading.Thread(target=analyse)
    th.start()
    per_config = {}
    for name in [c for c in args.per_config.split(",") if c and c not in (args.workload, "none")]:
        per_config[name] = measure_config(K, name, args.per_config_steps, 3, flush, local, rank)
    th.join()
    if an_err:
        raise an_err[0]
    info0 = solver.info()

    # inputs resident in HBM before the timed region
    with torch.cuda.stream(stream):
        vals = [torch.from_numpy(seq.values(k)).cuda() for k in range(seq.M)]
        rhs = [torch.from_numpy(seq.rhs(k, vals[k].cpu().numpy())[0]).cuda() for k in range(seq.M)]
        x = torch.empty(seq.n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    allow_nc = args.precision == "mixed"
    timed_steps(solver, vals, rhs, x, args.warmup, seq.M, flush, stream, allow_nc)
    solver.phase_times(reset=True)
    clocks = Clocks(local)
    launches0 = solver.info()["launches"]
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    per_step, iters, nrbes, _ = timed_steps(solver, vals, rhs, x, args.steps, seq.M, flush, stream, allow_nc)
    t_wall = time.perf_counter() - t_wall
    barrier(world)
    clk = clocks.stop()
    launches = solver.info()["launches"] - launches0
    dev_s = sum(per_step) / 1000.0
    phases = solver.phase_times(reset=True)
    units, secs = aggregate(float(args.steps), dev_s, world)

    # ---- the same steps unfused: kkt_refactor then kkt_solve
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
    for i in range(3):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[i][0].record(stream)
        solver.refactor(vals[i % seq.M])
        solver.solve(rhs[i % seq.M], x=x, tol=TOL, allow_not_converged=allow_nc)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    unfused_ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))

    # ---- end to end through the C ABI with pinned host buffers; the
    # returned x is checked against Eq. (nbre) as the oracle evaluates it
    from oracle import oracle as O
    n_e2e = min(args.e2e_steps, seq.M)
    hv = [torch.from_numpy(seq.values(k)).pin_memory().numpy() for k in range(n_e2e)]
    hb = [torch.from_numpy(seq.rhs(k)[0]).pin_memory().numpy() for k in range(n_e2e)]
    hx = [torch.empty(seq.n, dtype=torch.float64).pin_memory().numpy() for _ in range(n_e2e)]
    info_a = solver.info()
    torch.cuda.synchronize()
    t = time.perf_counter()
    e2e_nr = []
    for k in range(n_e2e):
        _, _, nr = solver.step(hv[k], hb[k], x=hx[k], tol=TOL, allow_not_converged=allow_nc)
        e2e_nr.append(nr)
    e2e_s = time.perf_counter() - t
    info_b = solver.info()
    e2e_units, e2e_secs = aggregate(float(n_e2e), e2e_s, world)
    or_nr = [O.nrbe(seq.n, seq.rowptr, seq.colind, hv[k], hb[k], hx[k]) for k in range(n_e2e)]
    eps_terms = 2 * (int(np.diff(seq.rowptr).max()) + 2) * 2.0 ** -53
    nrbe_check = {"steps": n_e2e, "max_oracle_nrbe": float(max(or_nr)),
                  "max_abs_diff": float(max(abs(a - b) for a, b in zip(e2e_nr, or_nr))),
                  "bound": "|gpu - oracle| <= 1e-6 oracle + 2 (max row nnz + 2) eps (two residual roundings)",
                  "within_bound": bool(all(abs(a - b) <= 1e-6 * b + eps_terms for a, b in zip(e2e_nr, or_nr)))}

    # ---- the refactorization's critical path (trace stamps of one call)
    crit = None
    if not args.no_trace:
        ts, tp, t0 = solver.trace_refactor(vals[0])
        crit = solver.critical_path(ts, tp)
        crit["first_traced_row"] = t0

    # ---- the other precision on the same workload, same protocol
    other = None
    if not args.no_mixed:
        alt = "mixed" if args.precision == "fp64" else "fp64"
        nm = min(args.mixed_steps, seq.M)
        idx = [int(round(i * (seq.M - 1) / max(nm - 1, 1))) for i in range(nm)]
        x64 = torch.empty_like(x)
        ref64 = {}   # the FP64 path's solution per matrix (factors equal to the oracle's bit for bit)

        def precision_leg(equilibrate):
            # FP32 factors as the preconditioner; a solve they have not
            # finished within --mixed-cycles restart cycles continues with the
            # FP64 refactorization (kkt_opts.mixed_fallback), counted per solve
            s2 = K.KKTSolver(restart=RESTART, device=local, stream=stream, timing=True, precision=alt,
                             mixed_fallback=args.mixed_cycles, equilibrate=equilibrate)
            s2.analyze_like(solver)
            timed_steps(s2, [vals[idx[0]]], [rhs[idx[0]]], x, 1, 1, flush, stream, True)
            s2.phase_times(reset=True)
            ms2, it2, nr2, st2, fb2, fe2, f64 = [], [], [], [], [], [], []
            for i in idx:   # one step at a time: each solve's fallback and errors are read after it
                m_, i_, n_, s_ = timed_steps(s2, [vals[i]], [rhs[i]], x, 1, 1, flush, stream, True)
                ms2 += m_
                it2 += i_
                nr2 += n_
                st2 += s_
                fb2.append(int(s2.info()["last_fallback"]))
                xs = seq.rhs(i, seq.values(i))[1]
                xm = x.cpu().numpy()
                fe2.append(float(np.linalg.norm(xm - xs) / np.linalg.norm(xs)))
                if i not in ref64:   # outside any timing
                    with torch.cuda.stream(stream):
                        solver.step(vals[i], rhs[i], x=x64, allow_not_converged=True)
                    stream.synchronize()
                    ref64[i] = x64.cpu().numpy()
                xf = ref64[i]
                f64.append(float(np.linalg.norm(xm - xf) / np.linalg.norm(xf)))
            ph2 = s2.phase_times(reset=True)
            s2.close()
            return {"precision": alt, "equilibrate": bool(equilibrate), "value": nm / (sum(ms2) / 1000.0),
                    "unit": "solves/s", "steps": nm, "matrices": idx,
                    "latency_ms": {"p50": float(np.percentile(ms2, 50)), "p99": float(np.percentile(ms2, 99))},
                    "fp32_cycles_before_fallback": args.mixed_cycles,
                    "iters": it2, "nrbe": [float(f"{v:.3g}") for v in nr2], "status": st2, "fell_back": fb2,
                    "forward_error_vs_xstar": [float(f"{v:.3g}") for v in fe2],
                    "rel_diff_vs_fp64_solution": [float(f"{v:.3g}") for v in f64],
                    "converged": int(sum(s_ == K.OK for s_ in st2)), "max_nrbe": float(np.nanmax(nr2 + [0.0])),
                    "phase_ms_per_step": {p: round(ph2[p][0] / nm, 4) for p in ph2}}

        other = precision_leg(False)
        if alt == "mixed":   # the same solves with the FP32 factors of the equilibrated matrix
            other["equilibrated"] = precision_leg(True)
    # ---- serving: several independent sequences resident at once, their
    # steps in flight together (kkt_server_*)
    serving = None
    if args.serve_instances > 0:
        one = serve_measure(K, args, rank, 1)
        serving = serve_measure(K, args, rank, args.serve_instances)
        serving["one_instance"] = {k: one[k] for k in ("value", "latency_ms", "call_ms")}
        serving["speedup_vs_one"] = serving["value"] / one["value"]
    serving_c4 = serve_c4(K, args, rank) if args.serve_c4 > 0 else None
    if rank != 0:
        return

    roof = roofline(phases, info0, seq.n, seq.nnz, args.steps, args.workload)
    if crit is not None:
        crit["kernel_ms_per_launch"] = roof["ms_per_launch"] if roof["kernel_group"] == "refactorization" else None
        roof["critical_path"] = crit
    cpu = None
    if not args.no_cpu_baseline:
        P, Q = solver.perm()
        totals = (seq.n, info0["refactor_updates"], info0["nnz_l"] + info0["nnz_u"])
        with pinned_core():
            est, smp = oracle_solve_estimate(O, seq, 1, P, Q, totals, args.cpu_seconds)
        cpu = {"value": 1.0 / est, "unit": "solves/s", "cores": 1, "kind": "oracle", **host_cpu(),
               "sample": (f"matrix 1 of the {args.workload} sequence: the oracle refactorization on the library's "
                          f"P, Q for {smp['seconds']:.1f} s ({smp['cols']} of {seq.n} columns, "
                          f"{100 * smp['madds'] / totals[1]:.2g}% of the multiply-adds)"
                          + (", extrapolated to the whole refactorization by a fitted cost model"
                             if smp["extrapolated"] else "")
                          + "; triangular solves and FGMRES not sampled; single thread")}

    lat = sorted(per_step)
    hbm, _ = peaks()
    tot_bytes = sum(step_bytes(info0, seq.n, seq.nnz, it) for it in iters)
    line = {
        "metric": METRIC,
        "value": units / secs, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32-factors/f64",
        "data": "synthetic",
        "config": {**workload_config(seq), "parallelism": f"replicas{world}", "precision": args.precision},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "iters_mean": float(np.mean(iters)), "max_nrbe": float(np.max(nrbes)),
        "nrbe_check": nrbe_check,
        "hbm_per_solve": {"achieved_gbs": tot_bytes / dev_s / 1e9, "frac": tot_bytes / dev_s / 1e9 / hbm,
                          "bytes_per_solve": tot_bytes / args.steps},
        "unfused_ms_per_step": unfused_ms,
        "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": e2e_units / e2e_secs, "unit": "solves/s",
                "h2d_bytes_per_step": (info_b["h2d_bytes"] - info_a["h2d_bytes"]) // n_e2e,
                "d2h_bytes_per_step": (info_b["d2h_bytes"] - info_a["d2h_bytes"]) // n_e2e},
        "gpu_launches": launches, "clocks": clk, "wall_s": t_wall, "job_s": time.perf_counter() - t_job,
        "precision": args.precision, "other_precision": other, "per_config": per_config,
        "serving": serving, "serving_mixed": serving_c4,
        "schedule": {k: info0[k] for k in ("rows_warp", "rows_team", "rows_block", "rows_global", "refactor_smem",
                                           "refactor_threads", "refactor_blocks", "trisolve_cluster")},
        "analysis": {"analyze_ms": info0["analyze_ms"], "nnz_l": info0["nnz_l"], "nnz_u": info0["nnz_u"],
                     "levels_l": info0["levels_l"], "levels_u": info0["levels_u"],
                     "refactor_updates": info0["refactor_updates"], "device_bytes": info0["device_bytes"]},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
