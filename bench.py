"""Benchmark: KKT solves/sec on a same-pattern synthetic power-grid KKT sequence.

One step = one pass of the hot path over one matrix of the sequence:
kkt_refactor (value gather, numeric LU on the fixed pattern and pivots) then
kkt_solve (triangular solves, residual, FGMRES(20) with CGS2 until
NRBE <= 1e-12).  Matrices cycle k = 0..M-1 over the sequence.

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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "kkt2000"
TOL = 1e-12
RESTART = 20
ALT_MAX_CYCLES = 2      # cycle cap of the side-by-side mixed-precision run
L2_FLUSH_BYTES = 256 << 20   # larger than the 126 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="bounded oracle sample for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="factor precision of the headline line")
    ap.add_argument("--no-mixed", action="store_true", help="skip the side-by-side mixed-precision run")
    ap.add_argument("--no-tune", action="store_true", help="skip the schedule autotuning at setup")
    ap.add_argument("--serve-instances", type=int, default=4,
                    help="independent sequences of the serving measurement (0 = skip)")
    ap.add_argument("--serve-steps", type=int, default=10)
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--serve-c4", type=int, default=0,
                    help="mixed-size serving run: this many instances, bus counts uniform in "
                         "[200, --serve-c4-buses], Poisson arrivals, each instance's steps closed-loop (0 = skip)")
    ap.add_argument("--serve-c4-buses", type=int, default=2000)
    ap.add_argument("--serve-c4-rate", type=float, default=50.0, help="instance arrivals per second")
    ap.add_argument("--serve-c4-steps", type=int, default=10)
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


def measured_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None when the kernel source changed since that capture."""
    path = os.path.join(ROOT, "profiles", "traffic_kkt2000.txt")
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


def roofline(phases, info, seq, steps):
    """Roofline of the dominant kernel group, from the library's own CUDA
    event timers over the timed region.

    refactorization (gather + bulk + block-per-row kernels): FP64 ALU bound,
      2 x multiply-adds of one refactorization per launch;
    triangular solves: HBM, 12 bytes per factor entry + 36 (L) / 44 (U)
      bytes per row per launch."""
    hbm, peak_kind = peaks()
    n = seq.n
    ref_ms = phases["gather"][0] + phases["refactor"][0] + phases["refactor_tail"][0]
    ref_n = max(phases["refactor_tail"][1], phases["refactor"][1], 1)
    groups = {"refactor": (ref_ms, ref_n), "lsolve": phases["lsolve"], "usolve": phases["usolve"]}
    dom = max(groups, key=lambda g: groups[g][0])
    ms, cnt = groups[dom]
    per_ms = ms / max(cnt, 1)
    extra = {"kernel_group": dom, "ms_per_launch": per_ms,
             "phase_ms_per_step": {p: round(phases[p][0] / steps, 4) for p in phases},
             "phase_launches": {p: phases[p][1] for p in phases}}
    if dom == "refactor":
        flops = 2.0 * info["refactor_updates"]
        ach = flops / (per_ms * 1e-3) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": measured_traffic("k_refactor_tail"),
                "peak_kind": "nominal FP64 (recipe table)", "flops_per_launch": flops, **extra}
    nnz = info["nnz_l"] if dom == "lsolve" else info["nnz_u"]
    bytes_ = 12 * nnz + (36 if dom == "lsolve" else 44) * n
    ach = bytes_ / (per_ms * 1e-3) / 1e9
    kern = "k_trsv_cluster<1>" if dom == "lsolve" else "k_trsv_cluster<0>"
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "traffic": measured_traffic(kern), "peak_kind": peak_kind + " hbm_gbs", "bytes_per_launch": bytes_,
            **extra}


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


def oracle_sample(seq, seconds, steps=None):
    """The CPU oracle as it stands: analysis once (not timed), then refactor +
    FGMRES per matrix until `seconds` (or `steps`) are used, on one core
    (the calling thread is pinned to the first CPU it may use)."""
    from oracle import oracle as O
    saved = None
    try:
        saved = os.sched_getaffinity(0)
        os.sched_setaffinity(0, {min(saved)})
    except (AttributeError, OSError):
        saved = None
    try:
        return _oracle_sample(O, seq, seconds, steps)
    finally:
        if saved:
            os.sched_setaffinity(0, saved)


def _oracle_sample(O, seq, seconds, steps):
    v0 = seq.values(0)
    t0 = time.perf_counter()
    P, Q, _ = O.lu(seq.n, seq.rowptr, seq.colind, v0)
    t_an = time.perf_counter() - t0
    done, t_solve, k = 0, 0.0, 0
    nrbe = []
    while True:
        v = seq.values(k % seq.M)
        b, _ = seq.rhs(k % seq.M, v)
        t = time.perf_counter()
        _, res = O.solve_sequence_step(seq.n, seq.rowptr, seq.colind, v, P, Q, b, tol=TOL, restart=RESTART)
        t_solve += time.perf_counter() - t
        nrbe.append(res.nrbe)
        done += 1
        k += 1
        if (steps is not None and done >= steps) or (steps is None and t_solve >= seconds):
            break
    return done, t_solve, t_an, max(nrbe)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2401_13926_b300.workload import KKTSequence
    seq = KKTSequence(args.workload)
    # warmup steps, then the timed ones
    oracle_sample(seq, 0, steps=max(args.warmup, 0) or 1)
    done, t, t_an, worst = oracle_sample(seq, 0, steps=args.steps)
    v = done / t
    line = {
        "impl": "reference", "metric": "KKT solves/sec (refactor+FGMRES to NRBE<=1e-12)", "value": v,
        "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * t / done, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": workload_config(seq),
        "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", **host_cpu(),
                         "sample": f"{done} matrices of the {args.workload} sequence, oracle analysis "
                                   f"({t_an:.1f} s) excluded, single thread"},
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "max_nrbe": worst,
    }
    print(json.dumps(line), flush=True)


def workload_config(seq):
    return {
        "workload": f"{seq.cfg.name}: synthetic {seq.nbus}-bus grid KKT [[H+Dx,J^T],[J,-Dy]], "
                    f"n={seq.n}, nnz={seq.nnz}, {seq.M}-matrix same-pattern sequence, "
                    f"Dx spread widening 1e+-{seq.cfg.s_first:g}..1e+-{seq.cfg.s_last:g}, "
                    f"FGMRES({RESTART}) to NRBE<={TOL:g}, FP64",
        "n": seq.n, "nnz": seq.nnz, "sequence": seq.M, "restart": RESTART, "tol": TOL,
        "l2": "flushed between timed steps (256 MiB write, outside the per-step events)",
    }


# -------------------------------------------------------------------- ours
def serve_measure(K, args, rank):
    """Throughput and latency of several sequences of the workload served
    together: every instance's steps are submitted at once (closed loop, the
    server runs one step per instance at a time), host arrays in and out."""
    from paper_2401_13926_b300.workload import KKTSequence
    N, S = args.serve_instances, args.serve_steps
    seqs = [KKTSequence(args.workload, instance=1000 * (rank + 1) + i, steps=S) for i in range(N)]
    data = [[(q.values(k), q.rhs(k, q.values(k))[0]) for k in range(S)] for q in seqs]
    srv = K.KKTServer(workers=args.serve_workers, restart=RESTART)
    ids = [srv.open(q.rowptr, q.colind, q.values(0)) for q in seqs]
    for i in range(N):   # warm-up: one step per instance
        srv.wait(srv.submit(ids[i], *data[i][0], tol=TOL)[0])
    t0 = time.perf_counter()
    tickets = [srv.submit(ids[i], *data[i][k], tol=TOL)[0] for k in range(S) for i in range(N)]
    res = [srv.wait(t)[1] for t in tickets]
    dt = time.perf_counter() - t0
    srv.close()
    lat = np.array([r["queue_ms"] + r["run_ms"] for r in res])
    run = np.array([r["run_ms"] for r in res])
    return {"value": N * S / dt, "unit": "solves/s", "instances": N, "steps_per_instance": S,
            "workers": args.serve_workers, "converged": int(sum(r["status"] == 0 for r in res)),
            "max_nrbe": float(max(r["nrbe"] for r in res)),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "step_ms": {"p50": float(np.percentile(run, 50)), "p99": float(np.percentile(run, 99))},
            "timing": "host wall clock, submit of all steps to the last completion; includes host<->device "
                      "copies of values, b and x"}


def serve_c4(K, args, rank):
    """Mixed-size serving: instances with bus counts drawn uniformly from
    [200, serve_c4_buses] arrive at Poisson times (rate serve_c4_rate per
    second); each runs its own sequence closed-loop (step k+1 is submitted
    when step k returns).  Instances are analysed before the clock starts
    (the paper, too, excludes the one-time analysis).  Latency is from a
    step's submission to its completion."""
    import threading
    from paper_2401_13926_b300.workload import KKTSequence
    rng = np.random.default_rng(7000 + rank)
    N, S = args.serve_c4, args.serve_c4_steps
    buses = rng.integers(200, args.serve_c4_buses + 1, size=N)
    seqs = [KKTSequence("kkt2000", instance=5000 + 100 * rank + i, buses=int(nb), steps=S)
            for i, nb in enumerate(buses)]
    data = [[(q.values(k), q.rhs(k, q.values(k))[0]) for k in range(S)] for q in seqs]
    srv = K.KKTServer(workers=args.serve_workers, restart=RESTART)
    t_open = time.perf_counter()
    ids = [srv.open(q.rowptr, q.colind, q.values(0)) for q in seqs]
    t_open = time.perf_counter() - t_open
    arrivals = np.cumsum(rng.exponential(1.0 / args.serve_c4_rate, size=N))
    results = [[] for _ in range(N)]

    def client(i, t_start):
        delay = t_start + arrivals[i] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        for k in range(S):
            t, _ = srv.submit(ids[i], *data[i][k], tol=TOL)
            results[i].append(srv.wait(t)[1])

    t0 = time.perf_counter()
    threads = [threading.Thread(target=client, args=(i, t0)) for i in range(N)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    dt = time.perf_counter() - t0
    srv.close()
    res = [r for rr in results for r in rr]
    lat = np.array([r["queue_ms"] + r["run_ms"] for r in res])
    return {"value": len(res) / dt, "unit": "solves/s", "instances": N, "steps_per_instance": S,
            "buses": [int(b) for b in buses], "n": [int(q.n) for q in seqs],
            "arrival_rate_per_s": args.serve_c4_rate, "workers": args.serve_workers,
            "converged": int(sum(r["status"] == 0 for r in res)), "max_nrbe": float(max(r["nrbe"] for r in res)),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "analysis_s_total": t_open,
            "timing": "host wall clock from the first arrival to the last completion"}


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    import paper_2401_13926_b300 as K
    from paper_2401_13926_b300.workload import KKTSequence

    seq = KKTSequence(args.workload, instance=rank)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    solver = K.KKTSolver(restart=RESTART, device=local, stream=stream, timing=True, precision=args.precision)
    solver.analyze(seq.rowptr, seq.colind, values0=seq.values(0))
    # schedule autotuning once at setup (kkt_tune; same bits, speed only)
    if not args.no_tune:
        solver.tune(seq.values(0), seq.rhs(0, seq.values(0))[0], reps=3)
    info0 = solver.info()
    # inputs resident in HBM before the timed region
    vals = [torch.from_numpy(seq.values(k)).cuda() for k in range(seq.M)]
    rhs = [torch.from_numpy(seq.rhs(k, vals[k].cpu().numpy())[0]).cuda() for k in range(seq.M)]
    x = torch.empty(seq.n, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step(k):
        # one step of the sequence: kkt_step (refactor + solve, the forward
        # sweep fused into the refactorization)
        # a mixed-precision headline reports unconverged solves instead of stopping
        _, it, nr = solver.step(vals[k % seq.M], rhs[k % seq.M], x=x, tol=TOL,
                                allow_not_converged=args.precision == "mixed")
        return it, nr

    for w in range(args.warmup):
        step(w)
    torch.cuda.synchronize()
    solver.phase_times(reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local)
    launches0 = solver.info()["launches"]
    iters, nrbes = [], []
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        it, nr = step(i)
        ev[i][1].record(stream)
        iters.append(it)
        nrbes.append(nr)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    barrier(world)
    clk = clocks.stop()
    launches = solver.info()["launches"] - launches0
    per_step = [a.elapsed_time(b) for a, b in ev]
    dev_s = sum(per_step) / 1000.0
    phases = solver.phase_times(reset=True)
    units, secs = aggregate(float(args.steps), dev_s, world)

    # ---- end to end through the C ABI with pinned host buffers
    n_e2e = min(args.e2e_steps, seq.M)
    hv = [torch.from_numpy(seq.values(k)).pin_memory().numpy() for k in range(n_e2e)]
    hb = [torch.from_numpy(seq.rhs(k)[0]).pin_memory().numpy() for k in range(n_e2e)]
    hx = torch.empty(seq.n, dtype=torch.float64).pin_memory().numpy()
    info_a = solver.info()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for k in range(n_e2e):
        solver.step(hv[k], hb[k], x=hx, tol=TOL)
    e2e_s = time.perf_counter() - t
    info_b = solver.info()
    e2e_units, e2e_secs = aggregate(float(n_e2e), e2e_s, world)

    # ---- the other precision on the same workload, same protocol (device time)
    other = None
    if not args.no_mixed:
        alt = "mixed" if args.precision == "fp64" else "fp64"
        # FP32-preconditioned refinement stalls above 1e-12 on some of these
        # ill-conditioned matrices, so this run caps the cycles and reports
        # how many solves reached the tolerance
        cyc2 = ALT_MAX_CYCLES if alt == "mixed" else 50
        s2 = K.KKTSolver(restart=RESTART, device=local, stream=stream, timing=True, precision=alt,
                         max_cycles=cyc2)
        s2.analyze(seq.rowptr, seq.colind, values0=seq.values(0))
        for w in range(args.warmup):
            s2.step(vals[w % seq.M], rhs[w % seq.M], x=x, tol=TOL, allow_not_converged=True)
        s2.phase_times(reset=True)
        ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(seq.M)]
        it2, nr2, ok2 = [], [], 0
        torch.cuda.synchronize()
        for i in range(seq.M):
            flush.zero_()
            ev2[i][0].record(stream)
            _, it, nr = s2.step(vals[i], rhs[i], x=x, tol=TOL, allow_not_converged=True)
            ev2[i][1].record(stream)
            it2.append(it)
            nr2.append(nr)
            ok2 += s2.last_status == K.OK
        torch.cuda.synchronize()
        ms2 = [a.elapsed_time(b) for a, b in ev2]
        ph2 = s2.phase_times(reset=True)
        other = {"precision": alt, "value": seq.M / (sum(ms2) / 1000.0), "unit": "solves/s",
                 "steps": seq.M, "latency_ms": {"p50": float(np.percentile(ms2, 50)),
                                                "p99": float(np.percentile(ms2, 99))},
                 "iters_mean": float(np.mean(it2)), "max_nrbe": float(np.max(nr2)),
                 "converged": ok2, "max_cycles": cyc2, "nrbe": [float(f"{v:.3g}") for v in nr2],
                 "phase_ms_per_step": {p: round(ph2[p][0] / seq.M, 4) for p in ph2}}
        s2.close()
    # ---- serving: several independent sequences of the same workload resident
    # at once, their steps in flight together (kkt_server_*)
    serving = None
    if args.serve_instances > 0:
        serving = serve_measure(K, args, rank)
    serving_c4 = serve_c4(K, args, rank) if args.serve_c4 > 0 else None
    if rank != 0:
        return

    # ---- roofline of the dominant kernel group
    roof = roofline(phases, info0, seq, args.steps)
    cpu = None
    if not args.no_cpu_baseline:
        done, tcpu, t_an, _ = oracle_sample(KKTSequence(args.workload), args.cpu_seconds)
        cpu = {"value": done / tcpu, "unit": "solves/s", "cores": 1, "kind": "oracle", **host_cpu(),
               "sample": f"{done} matrices of the {args.workload} sequence (about {args.cpu_seconds:g} s), "
                         f"oracle analysis ({t_an:.1f} s) excluded, single thread"}

    lat = sorted(per_step)
    line = {
        "metric": "KKT solves/sec (refactor+FGMRES to NRBE<=1e-12)",
        "value": units / secs, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32-factors/f64",
        "data": "synthetic",
        "config": {**workload_config(seq), "parallelism": f"replicas{world}", "precision": args.precision},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "iters_mean": float(np.mean(iters)), "max_nrbe": float(np.max(nrbes)),
        "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": e2e_units / e2e_secs, "unit": "solves/s",
                "h2d_bytes_per_step": (info_b["h2d_bytes"] - info_a["h2d_bytes"]) // n_e2e,
                "d2h_bytes_per_step": (info_b["d2h_bytes"] - info_a["d2h_bytes"]) // n_e2e},
        "gpu_launches": launches, "clocks": clk, "wall_s": t_wall,
        "precision": args.precision, "other_precision": other, "serving": serving, "serving_mixed": serving_c4,
        "schedule": {"tail_rows": info0["tail_rows"], "trisolve_cluster": info0["trisolve_cluster"],
                     "chosen_by": "default" if args.no_tune else "kkt_tune at setup"},
        "analysis": {"analyze_ms": info0["analyze_ms"], "nnz_l": info0["nnz_l"], "nnz_u": info0["nnz_u"],
                     "levels_l": info0["levels_l"], "levels_u": info0["levels_u"],
                     "refactor_updates": info0["refactor_updates"]},
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
