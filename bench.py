#!/usr/bin/env python3
"""Throughput of the adiabatic 3-SAT Strang evolution on one GB300 (or N replicas).

Workload: the committed planted unique-solution instance with n = 30 variables
(satgen/instances/planted_n30_s0.json, m = 371 clauses), complex64 state of
2^30 amplitudes (8 GiB, far larger than L2, so no flush is needed between
steps), linear schedule with dt = 0.1 (the T = 40, 400-step configuration).
One "step" = one full second-order Strang step of Eq. (1) frozen at the step's
midpoint: the merged half phases of H_P (violated-clause counts), and
exp(-i dt (1-s) H_B) applied as Walsh-Hadamard sandwiches on every 5-qubit
block (the default rotation form), i.e. g = 3 HBM round trips at n = 30: the
two strided groups' passes and the low pass.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank evolves its own copy
(replicas: the method needs no exchange between GPUs), and `value` is the
whole-job steps/s = N K / max-over-ranks time.
"""

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Trotter steps/s + HBM GB/s at n=30 c64; batched solves/s, p50/p99 latency"
UNIT = "steps/s"
INSTANCE = "planted_n30_s0"
DT = 0.1
T_CONFIG = 40.0
FALLBACK_HBM_GBS = 6800.0

# DRAM bytes per launch measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum)
# for the dominant kernel, with the sha256 of the kernel sources at the time of
# the capture; a mismatch (kernel changed since) reports traffic = null.
TRAFFIC = {
    # ncu full-set capture of sp_tma_kernel<10,4,2> (the default rotation form's
    # strided pass, 128-byte runs) on the 28-qubit instance with
    # QAA_GROUP_BITS=10,8: DRAM bytes read + written per launch for 2^28
    # amplitudes, scaled by the amplitude count (x4) to one 30-qubit launch.
    "strided": {"bytes_per_launch": 4 * (2.147551e9 + 2.086624e9), "src_sha": "5f1e3ea4bd430d04"},
}


def kernel_src_sha():
    """sha256 of the dominant kernel's device source: the PTX helpers and the
    strided-pass section of tma_kernels.cu, and device_common.cuh (host launch
    code is left out, so only a change to what the kernel executes voids the
    stored traffic)."""
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_1103_1399_gb300", "csrc", "tma_kernels.cu")) as fh:
        text = fh.read()
    h.update(text[text.index("// ---------------------------------------------------------------- PTX -------"):
                  text.index("// ----------------------------------------------------------- low pass -------")].encode())
    with open(os.path.join(ROOT, "paper_1103_1399_gb300", "csrc", "device_common.cuh"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms, ws, device):
    """The slowest rank's time: every rank's steps count only once all are done."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws, steps, t_max_ms):
    """Whole-job throughput: every replica evolves its own copy (replicas only,
    weak scaling), so N ranks complete N x steps Strang steps in the slowest
    rank's time."""
    return ws * steps / (t_max_ms / 1e3)


# ------------------------------------------------------------- CPU oracle ----
def oracle_step_sample(n_sample, steps, seed=0):
    """Time the oracle (as it stands) on a planted instance of n_sample variables.

    Returns (seconds for E(x), seconds per Strang step, cores used): the oracle
    evolves with its own unmerged Strang split in complex128; cores used is the
    process CPU time over the wall time of the timed steps (NumPy's elementwise
    kernels are single-threaded; BLAS is not used).
    """
    import numpy as np
    import oracle
    import satgen
    inst = satgen.planted_instance(n_sample, seed)
    t0 = time.perf_counter()
    e = oracle.violated_counts(n_sample, inst["clauses"])
    t_e = time.perf_counter() - t0
    psi = oracle.uniform_state(n_sample)
    t0, c0 = time.perf_counter(), time.process_time()
    psi = oracle.evolve_strang(n_sample, inst["clauses"], DT * steps, steps, psi0=psi, energies=e)
    wall = time.perf_counter() - t0
    cores = (time.process_time() - c0) / wall if wall > 0 else None
    assert np.isfinite(psi).all()
    return t_e, wall / steps, cores


def extrapolate(t_step, n_sample, n_target):
    return t_step * (n_target * 2.0 ** n_target) / (n_sample * 2.0 ** n_sample)


def host_mem_gib():
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) / 2 ** 20
    except OSError:
        pass
    return None


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        return max((i.get("num_threads", 1) for i in threadpool_info()), default=None)
    except Exception:
        return "unknown"


def oracle_baseline(n_target, small_steps):
    """The oracle's Strang step measured at n = 20 (small_steps steps) and at
    n = 24 (one step, E(x) computed first and reported apart), extrapolated to
    n_target from the n = 24 figure by n 2^n.  n_target itself is not run: its
    state alone is 2^n complex128 values (16 GiB at n = 30), and one step would
    take the extrapolated time (minutes), beyond a bench run."""
    t_e20, t20, cores20 = oracle_step_sample(20, small_steps)
    t_e24, t24, cores24 = oracle_step_sample(24, 1)
    t_target = extrapolate(t24, 24, n_target)
    mem = host_mem_gib()
    mem_s = f"{mem:.0f} GiB" if mem is not None else "unknown"
    return {
        "value": 1.0 / t_target, "unit": UNIT, "kind": "oracle", "extrapolated": True,
        "cores": round(max(cores20 or 0.0, cores24 or 0.0), 2), "blas_threads": blas_threads(),
        "os_cpu_count": os.cpu_count(),
        "sample": (f"oracle Strang steps (complex128 NumPy, unmerged halves) on planted instances: n=20 "
                   f"{small_steps} steps at {t20:.4f} s/step (E(x) {t_e20:.2f} s), n=24 one step {t24:.2f} s "
                   f"(E(x) {t_e24:.1f} s); value extrapolated from n=24 to n={n_target} by n 2^n "
                   f"({t_target:.0f} s/step); n={n_target} not run (host MemAvailable {mem_s}; one step "
                   f"would take the extrapolated time)"),
        "measured_s_per_step": {"20": t20, "24": t24}, "e_x_seconds": {"20": t_e20, "24": t_e24},
        "host_mem_available_gib": mem,
    }


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import satgen
    n_target = satgen.load_instance(INSTANCE)["n"]
    oracle_step_sample(16, max(1, args.warmup))  # warm-up (untimed)
    t0 = time.perf_counter()
    cpu = oracle_baseline(n_target, args.steps)
    wall = time.perf_counter() - t0
    value = cpu["value"]
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": f"planted 3-SAT n={n_target}, dt={DT} (T={T_CONFIG:g}, 400 steps), complex64 state",
                   "wall_s": wall, "note": "each timed step is a bounded sample (n=20 and n=24 oracle steps); "
                                           "ms_per_step is the extrapolated n=30 figure"},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------- serving --------
SERVE_DT = 0.05


def _gen_instance(args):
    n, seed = args
    import satgen
    return satgen.planted_instance(n, seed)["clauses"]


def serving_workload(count, seed=0):
    """The batched-serving mix: n ~ U{10..22}, T ~ U[5, 80], dt = 0.05, one
    independent planted unique-solution instance per request (generated in a
    spawn process pool)."""
    import multiprocessing as mp
    import satgen
    reqs = satgen.serving_requests(count, seed=seed)
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        clauses = pool.map(_gen_instance, [(n, s) for _, n, _, s in reqs], chunksize=8)
    return [(n, cl, T, max(1, int(round(T / SERVE_DT)))) for (_, n, T, _), cl in zip(reqs, clauses)]


def _pct(v, p):
    import numpy as np
    return float(np.percentile(np.asarray(v), p)) if v else None


def round_trips(plan_description):
    """HBM round trips per Strang step of a streaming plan, from its description:
    g strided groups -> g + 1 in the rotation form, 2g in the W.B.W form."""
    g = plan_description.count("group bits")
    return g + 1 if "rotation form" in plan_description else 2 * g


def small_configs(q, torch, stream):
    """n = 12: ten planted instances (seeds 0..9), T = 20, 400 steps, solved one at
    a time through the handle API (the on-chip evolver): solves/s, P_succ, norm.
    n = 20 (the committed instance): T = 10, 40, 160 (200, 800, 3200 steps):
    steps/s and the L2 bandwidth of its 2 round trips per step (the state fits
    in L2)."""
    import satgen
    out = {}
    ps, norms = [], []
    psi = torch.empty(1 << 12, dtype=torch.complex64, device="cuda")
    insts = [satgen.planted_instance(12, s)["clauses"] for s in range(10)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for cl in insts:
        with q.Instance(12, cl, stream=stream) as inst:
            inst.init_uniform(psi)
            inst.evolve(psi, 20.0, 400)
            o = inst.observables(psi)
        ps.append(o["ground_prob"] / o["norm"])
        norms.append(o["norm"])
    wall = time.perf_counter() - t0
    out["n12"] = {"solves_per_s": len(insts) / wall, "steps": 400, "T": 20.0, "seeds": "0..9",
                  "p_succ": ps, "norm_minus_1_max": max(abs(x - 1.0) for x in norms),
                  "what": "qaa_create + init + evolve + observables per instance, host-timed"}
    cl20 = satgen.load_instance("planted_n20_s0")["clauses"]
    p20 = torch.empty(1 << 20, dtype=torch.complex64, device="cuda")
    rows = []
    with q.Instance(20, cl20, stream=stream) as inst:
        inst.init_uniform(p20)
        inst.evolve(p20, 1.0, 20)  # warm-up
        rts = round_trips(inst.describe_plan())
        for T in (10.0, 40.0, 160.0):
            K = int(round(T / 0.05))
            inst.init_uniform(p20)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            inst.evolve(p20, T, K)
            e1.record(stream)
            o = inst.observables(p20)
            ms = e0.elapsed_time(e1)
            rows.append({"T": T, "steps": K, "steps_per_s": K / (ms / 1e3),
                         "l2_gbs": rts * 2 * 8 * (1 << 20) * K / (ms / 1e3) / 1e9,
                         "p_succ": o["ground_prob"] / o["norm"], "norm": o["norm"]})
    out["n20"] = {"plan": f"{rts} round trips per step", "runs": rows}
    # random 3-SAT at ratio 4.2 (degenerate ground state), sin^2 schedule
    rd = satgen.ratio_instance(20, 1, min_solutions=2)
    K, T = 800, 40.0
    s_values = [math.sin(0.5 * math.pi * (k + 0.5) / K) ** 2 for k in range(K)]
    with q.Instance(20, rd["clauses"], stream=stream) as inst:
        inst.init_uniform(p20)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        inst.evolve_schedule(p20, T / K, s_values)
        e1.record(stream)
        o = inst.observables(p20)
        ms = e0.elapsed_time(e1)
    out["ratio42_n20"] = {"m": rd["m"], "solutions": rd["solutions"], "ground_count": o["ground_count"],
                          "schedule": "s(t) = sin^2(pi t / 2T)", "T": T, "steps": K,
                          "steps_per_s": K / (ms / 1e3), "p_succ": o["ground_prob"] / o["norm"]}
    return out


def spectrum_lines(q, torch, n, clauses):
    import satgen
    out = {}
    cl20 = satgen.load_instance("planted_n20_s0")["clauses"]
    scan = []
    t0 = time.perf_counter()
    with q.Instance(20, cl20) as inst:
        for s in [0.1 * i for i in range(1, 10)]:
            lv, its = inst.lowest_eigenvalues(s, k=2, max_iter=200, start=0)
            scan.append({"s": round(s, 2), "e0": lv[0], "gap": lv[1] - lv[0] if len(lv) > 1 else None, "iters": its})
    wall = time.perf_counter() - t0
    gaps = [r["gap"] for r in scan if r["gap"] is not None]
    out["n20_gap_scan"] = {"points": scan, "min_gap": min(gaps) if gaps else None, "wall_s": wall,
                           "what": "qaa_lowest_eigenvalues(s, k=2, 200 iterations, uniform start) at s = 0.1..0.9"}
    torch.cuda.empty_cache()
    with q.Instance(n, clauses) as inst:
        inst.lowest_eigenvalues(0.5, k=1, max_iter=2, start=0)  # workspace allocation, E(x) export
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lv, its = inst.lowest_eigenvalues(0.5, k=2, max_iter=30, start=0)
        wall = time.perf_counter() - t0
    out[f"n{n}_lanczos"] = {"s": 0.5, "iters": its, "ms_per_iter": 1e3 * wall / its, "ritz_lowest": lv,
                            "what": "30 Lanczos iterations at n=30 (H v by direct gathers, FP64 vectors), host-timed"}
    return out


def autotune_sizes(q, torch, work):
    """qaa_autotune once per streaming size of the mix (n >= 15), on the first
    request of that size; the chosen plans then serve every later handle and
    server request of that n in this process."""
    out, t0 = {}, time.perf_counter()
    seen = {}
    for n, cl, _, _ in work:
        if n >= 15 and n not in seen:
            seen[n] = cl
    for n in sorted(seen):
        psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        with q.Instance(n, seen[n]) as inst:
            # enough steps that one timing lasts about a millisecond or more
            rep = inst.autotune(psi, steps=max(3, min(64, 1 << max(0, 26 - n))), budget_ms=5000)
            out[str(n)] = {"chosen": inst.describe_plan(),
                           "candidates": sum(1 for ln in rep.splitlines() if "ms/step" in ln and not ln.startswith("chosen"))}
        del psi
    torch.cuda.synchronize()
    return {"seconds": time.perf_counter() - t0, "plans": out}


def _solve_plain(q, torch, n, cl, T, K):
    with q.Instance(n, cl) as inst:
        psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        inst.init_uniform(psi)
        inst.evolve(psi, T, K)
        inst.observables(psi)


def _plain_arrivals(q, torch, work, arrivals):
    """The one-launch-sequence-per-instance path as a server: requests solved
    one at a time in arrival order, each no earlier than its arrival."""
    t0 = time.perf_counter()
    lat = []
    for (n, cl, T, K), ta in zip(work, arrivals):
        wait = ta - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        _solve_plain(q, torch, n, cl, T, K)
        lat.append(time.perf_counter() - t0 - ta)
    return lat, time.perf_counter() - t0


def _server_arrivals(q, work, arrivals):
    with q.Server(max_slots=1024) as srv:
        t0 = time.perf_counter()
        tickets = []
        for (n, cl, T, K), ta in zip(work, arrivals):
            wait = ta - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            tickets.append(srv.submit(n, cl, T, K))
        res = _wait_all(srv, tickets)
        span = time.perf_counter() - t0
        st = srv.stats()
    return res, span, st


def _in_flight(res):
    """Device concurrency of served requests: from each request's device
    interval (events on its own stream), the largest number in flight at once
    and the time-averaged number while any is."""
    ev = []
    for r in res:
        if r["status"] == 0 and r["t_dev_end"] > r["t_dev_start"] >= 0:
            ev.append((r["t_dev_start"], 1))
            ev.append((r["t_dev_end"], -1))
    ev.sort()
    cur = peak = 0
    busy = area = 0.0
    last = None
    for t, d in ev:
        if last is not None and cur > 0:
            busy += t - last
            area += cur * (t - last)
        cur += d
        peak = max(peak, cur)
        last = t
    return {"max_in_flight": peak, "mean_in_flight": area / busy if busy > 0 else None,
            "what": "requests whose device intervals (device-timer stamps before the first copy and at the end "
                    "of the observables) overlap"}


def _lat(lat):
    return {"p50_ms": 1e3 * _pct(lat, 50), "p99_ms": 1e3 * _pct(lat, 99)}


def run_serving(q, torch, work, rate_factor=0.7, high_factor=0.9):
    out = {"requests": len(work), "dt": SERVE_DT, "mix": "n ~ U{10..22}, T ~ U[5,80], planted unique-solution"}
    out["autotune"] = autotune_sizes(q, torch, work)
    np_ = __import__("numpy")
    # baseline: one launch sequence per instance, one after another (handle API), all at t = 0
    lat, base_s = _plain_arrivals(q, torch, work, [0.0] * len(work))
    out["one_launch_per_instance"] = {"solves_per_s": len(work) / base_s, **_lat(lat), "makespan_s": base_s,
                                      "what": "all requests at t=0, solved one at a time: qaa_create, init, "
                                              "evolve, observables, destroy"}
    # continuous batching, all requests at t = 0 (capacity)
    res, cap_s, st = _server_arrivals(q, work, [0.0] * len(work))
    lat = [r["t_done"] - r["t_submit"] for r in res]
    cap = len(work) / cap_s
    out["continuous_batching"] = {"solves_per_s": cap, **_lat(lat), "makespan_s": cap_s,
                                  "ok": sum(1 for r in res if r["status"] == 0), "server": st,
                                  "arrivals": "all at t=0", "device": _in_flight(res)}
    # the same seeded Poisson arrivals for both paths, at two rates: 0.7 x the
    # plain path's throughput, and 0.9 x the server's capacity
    rng = np_.random.default_rng(1)
    unit = np_.cumsum(rng.exponential(1.0, size=len(work)))
    for key, rate in (("poisson", rate_factor * len(work) / base_s), ("poisson_high", high_factor * cap)):
        arrivals = unit / rate
        res, span, _ = _server_arrivals(q, work, arrivals)
        slat = [r["t_done"] - r["t_submit"] for r in res]
        plat, pspan = _plain_arrivals(q, torch, work, arrivals)
        out[key] = {"rate_per_s": rate, "solves_per_s": len(work) / span, **_lat(slat), "makespan_s": span,
                    "ok": sum(1 for r in res if r["status"] == 0), "device": _in_flight(res),
                    "one_launch_per_instance": {"solves_per_s": len(work) / pspan, **_lat(plat),
                                                "makespan_s": pspan}}
    out["solves_per_s"] = out["continuous_batching"]["solves_per_s"]
    out["p50_ms"] = out["poisson"]["p50_ms"]
    out["p99_ms"] = out["poisson"]["p99_ms"]
    return out


def _wait_all(srv, tickets, timeout=600.0):
    pending, res, t0 = set(tickets), {}, time.perf_counter()
    while pending:
        for t in list(pending):
            r = srv.poll(t)
            if r is not None:
                res[t] = r
                pending.discard(t)
        if time.perf_counter() - t0 > timeout:
            raise RuntimeError("serving requests did not finish")
        time.sleep(0.0005)
    return [res[t] for t in tickets]


# ------------------------------------------------------------- GPU arm --------
def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import satgen
    import paper_1103_1399_gb300 as q

    inst_d = satgen.load_instance(args.instance)
    n, clauses = inst_d["n"], inst_d["clauses"]
    stream = torch.cuda.current_stream()
    psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    inst = q.Instance(n, clauses, stream=stream)
    inst.init_uniform(psi)
    # warm-up: W steps of the same schedule (dt = 0.1)
    inst.evolve(psi, DT * args.warmup, args.warmup)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    K = args.steps
    inst.profile(True)
    inst.profile_reset()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        inst.evolve(psi, DT * K, K)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    prof = inst.profile_read()
    inst.profile(False)
    t_max = max_over_ranks(ms, ws, "cuda")
    value = job_value(ws, K, t_max)
    # the observables of the final state (norm, <H_P>, <H_B>, ground probability
    # and count), their kernels timed by the handle's profiler
    inst.profile(True)
    inst.profile_reset()
    obs = inst.observables(psi)
    obs_launches, obs_ms = inst.profile_read()["observe"]
    inst.profile(False)

    state_bytes = 8 * (1 << n)
    passes_per_step = round(sum(prof[k][0] for k in ("low_first", "low_merge", "low_last", "strided", "strided_phase")) / K)
    hbm_gbs = passes_per_step * 2 * state_bytes * K / (ms / 1e3) / 1e9

    # dominant kernel, its average launch, roofline
    kinds = {k: v for k, v in prof.items() if v[0] > 0}
    dom = max(kinds, key=lambda k: kinds[k][1])
    launches, dom_ms = kinds[dom]
    per_launch_ms = dom_ms / launches
    algo_bytes = 2 * state_bytes  # one read + one write of the whole state per pass
    achieved = algo_bytes / (per_launch_ms / 1e3) / 1e9
    peak, peak_src = measured_peaks()
    tr = TRAFFIC.get(dom)
    traffic = tr["bytes_per_launch"] if tr and tr.get("src_sha") == kernel_src_sha() else None
    gpu_launches = sum(v[0] for v in prof.values())

    # tensor-core split-BF16 Walsh-Hadamard variants on the same workload
    variants = {}
    if not args.no_variants:
        default_form = 3 if "rotation form" in inst.describe_plan() else 0
        forms = ((0, "wbw"), (1, "bf16x3"), (2, "bf16x2"), (3, "rotation"))
        for kind, name in (f for f in forms if f[0] != default_form):
            vi = q.Instance(n, clauses, stream=stream)
            vi.set_variant(kind)
            vi.init_uniform(psi)
            vk = min(K, 100)
            vi.evolve(psi, DT * 3, 3)
            torch.cuda.synchronize()
            vi.profile(True)
            vi.profile_reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            vi.evolve(psi, DT * vk, vk)
            e1.record(stream)
            torch.cuda.synchronize()
            vms = e0.elapsed_time(e1)
            vprof = {k: {"launches": v[0], "ms": v[1]} for k, v in vi.profile_read().items() if v[0] > 0}
            vi.profile(False)
            rts = round_trips(vi.describe_plan())
            variants[name] = {"steps_per_s": vk / (vms / 1e3), "ms_per_step": vms / vk, "steps": vk,
                              "hbm_round_trips_per_step": rts, "plan": vi.describe_plan(), "kernels": vprof,
                              "hbm_gbs": rts * 2 * state_bytes * vk / (vms / 1e3) / 1e9}
            vi.close()

    # launch-graph mode on the same workload: one CUDA graph per evolve call
    graph = None
    if not args.no_variants:
        gi = q.Instance(n, clauses, stream=stream)
        gi.set_launch_mode(q.LAUNCH_GRAPH)
        gk = min(K, 100)
        gi.init_uniform(psi)
        gi.evolve(psi, DT * gk, gk)  # builds the graph (and warms up)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        gi.evolve(psi, DT * gk, gk)  # same arguments: the graph is relaunched
        g1.record(stream)
        torch.cuda.synchronize()
        gms = g0.elapsed_time(g1)
        graph = {"steps_per_s": gk / (gms / 1e3), "ms_per_step": gms / gk, "steps": gk,
                 "what": "qaa_set_launch_mode(QAA_LAUNCH_GRAPH): one graph launch per evolve call, a device-side "
                         "WHILE loop over 8-step bodies"}
        gi.close()

    # fourth-order steps (Yoshida triple jump: 3 Strang sub-steps each) on the same workload
    order4 = None
    if not args.no_variants:
        oi = q.Instance(n, clauses, stream=stream)
        ok4 = 30
        oi.init_uniform(psi)
        oi.evolve_order4(psi, DT * 3, 3)
        torch.cuda.synchronize()
        o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        o0.record(stream)
        oi.evolve_order4(psi, DT * ok4, ok4)
        o1.record(stream)
        torch.cuda.synchronize()
        oms = o0.elapsed_time(o1)
        order4 = {"steps_per_s": ok4 / (oms / 1e3), "substeps_per_s": 3 * ok4 / (oms / 1e3), "steps": ok4,
                  "what": "qaa_evolve_order4: each step of dt = 0.1 is three Strang sub-steps (Yoshida weights)"}
        oi.close()

    # spectrum of H(s) by Lanczos: the gap scan of the 20-qubit instance over
    # s = 0.1 .. 0.9 (levels reachable from the uniform state), and the cost of
    # one Lanczos iteration at n = 30 (three FP64 vectors of 8 GiB)
    spectrum = None
    if not args.no_spectrum and rank == 0:
        spectrum = spectrum_lines(q, torch, n, clauses)

    # the 32-qubit case of the same configuration (32 GiB state), a short run
    n32 = None
    if not args.no_n32 and rank == 0:
        psi = None  # room for the 32 GiB state
        torch.cuda.empty_cache()
        d32 = satgen.load_instance("planted_n32_s0")
        p32 = torch.empty(1 << 32, dtype=torch.complex64, device="cuda")
        i32 = q.Instance(32, d32["clauses"], stream=stream)
        k32 = 12
        i32.init_uniform(p32)
        i32.evolve(p32, DT * 3, 3)
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        i32.evolve(p32, DT * k32, k32)
        h1.record(stream)
        torch.cuda.synchronize()
        hms = h0.elapsed_time(h1)
        rts = round_trips(i32.describe_plan())
        n32 = {"steps_per_s": k32 / (hms / 1e3), "ms_per_step": hms / k32, "steps": k32, "plan": i32.describe_plan(),
               "hbm_gbs": rts * 2 * 8 * (1 << 32) * k32 / (hms / 1e3) / 1e9, "m": len(d32["clauses"])}
        if not args.no_variants:
            other = 0 if "rotation form" in i32.describe_plan() else 3
            i32.set_variant(other)
            i32.init_uniform(p32)
            i32.evolve(p32, DT * 3, 3)
            torch.cuda.synchronize()
            h0.record(stream)
            i32.evolve(p32, DT * k32, k32)
            h1.record(stream)
            torch.cuda.synchronize()
            rms = h0.elapsed_time(h1)
            rrt = round_trips(i32.describe_plan())
            n32["rotation" if other == 3 else "wbw"] = {
                "steps_per_s": k32 / (rms / 1e3), "ms_per_step": rms / k32, "plan": i32.describe_plan(),
                "hbm_gbs": rrt * 2 * 8 * (1 << 32) * k32 / (rms / 1e3) / 1e9}
        i32.close()
        del p32
        torch.cuda.empty_cache()
        psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")

    # the largest state one GPU holds: n = 34 (128 GiB, plus 22 GiB of stored
    # per-tile counts), a random 3-SAT instance at ratio 4.2 (m = 143), a short
    # run; only with --n34
    n34 = None
    if args.n34 and rank == 0:
        psi = None
        torch.cuda.empty_cache()
        free, _ = torch.cuda.mem_get_info()
        if free >= 160 << 30:
            c34 = satgen.random_instance(34, 143, seed=0, width=3)
            p34 = torch.empty(1 << 34, dtype=torch.complex64, device="cuda")
            i34 = q.Instance(34, c34, stream=stream)
            k34 = 6
            i34.init_uniform(p34)
            i34.evolve(p34, DT * 2, 2)
            torch.cuda.synchronize()
            h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            h0.record(stream)
            i34.evolve(p34, DT * k34, k34)
            h1.record(stream)
            torch.cuda.synchronize()
            ms34 = h0.elapsed_time(h1)
            rts = round_trips(i34.describe_plan())
            n34 = {"steps_per_s": k34 / (ms34 / 1e3), "ms_per_step": ms34 / k34, "steps": k34,
                   "plan": i34.describe_plan(), "m": len(c34),
                   "hbm_gbs": rts * 2 * 8 * (1 << 34) * k34 / (ms34 / 1e3) / 1e9,
                   "instance": "uniform random 3-SAT, ratio 4.2, seed 0 (timing only)"}
            i34.close()
            del p34
        else:
            n34 = {"skipped": f"needs 160 GiB free, {free / 2**30:.0f} GiB free"}
        torch.cuda.empty_cache()
        psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")

    # the small configurations: n = 12 (T = 20, seeds 0..9, on chip) and n = 20
    # (T = 10, 40, 160; the 8 MiB state is L2-resident), dt = 0.05
    small = None
    if not args.no_small and rank == 0:
        small = small_configs(q, torch, stream)

    # e2e: a full solve of the configured workload (T = 40, dt = 0.1: 400 steps)
    # through the public API, the instance in host memory: clause tables
    # host->device, init, evolve, observables device->host
    e2e = None
    if not args.no_e2e:
        K_full = int(round(T_CONFIG / DT))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        inst2 = q.Instance(n, clauses, stream=stream)       # H2D: clause tables
        inst2.init_uniform(psi)
        inst2.evolve(psi, T_CONFIG, K_full)
        o2 = inst2.observables(psi)                        # D2H: 5 FP64 results (synchronises)
        inst2.close()
        e2e_s = time.perf_counter() - t0
        e2e = {"value": K_full / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 32 * len(clauses) / K_full,
               "d2h_bytes_per_step": 40 / K_full, "solve_s": e2e_s, "steps": K_full, "T": T_CONFIG,
               "ground_prob": o2["ground_prob"], "norm": o2["norm"],
               "what": "one full solve of the configuration (qaa_create with the clause tables host->device, "
                       "init, evolve 400 steps, observables device->host), timed on the host"}

    serving = None
    if rank == 0 and args.serving_requests > 0:
        serving = run_serving(q, torch, serving_workload(args.serving_requests))

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = oracle_baseline(n, 24)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": args.warmup,
            "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"planted 3-SAT n={n} m={len(clauses)}, linear s, dt={DT} "
                                   f"(T={T_CONFIG:g} / 400-step configuration), complex64 state {state_bytes / 2**30:g} GiB",
                       "n": n, "m": len(clauses), "dt": DT, "plan": inst.describe_plan(),
                       "l2": f"state ({state_bytes / 2**30:g} GiB) exceeds L2; no flush needed",
                       "parallelism": f"replicas x{ws}"},
            "hbm_gbs": hbm_gbs,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                         "algorithmic_bytes_per_launch": algo_bytes, "avg_launch_ms": per_launch_ms,
                         "frac_of_8tbs": achieved / 8000.0},
            "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in kinds.items()},
            "gpu_launches": gpu_launches,
            "clocks": clk.summary(),
            "e2e": e2e,
            "precision_variants": variants,
            "launch_graph": graph,
            "spectrum": spectrum,
            "order4": order4,
            "small_configs": small,
            "n32": n32,
            "n34": n34,
            "serving": serving,
            "cpu_baseline": cpu,
            "final": {"norm": obs["norm"], "ground_prob": obs["ground_prob"]},
            "observables": {"ms": obs_ms, "reads_of_state": 1 + (n - 10 + 9) // 10,
                            "what": "qaa_observables on the final state: the low kernel (norm, <H_P>, ground "
                                    "probability and count from the stored clause counts, pair correlations of "
                                    "bits 0..9) and the read-only correlation passes of bits 10..n-1"},
        }
        print(json.dumps(line))
    inst.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip timing the tensor-core WHT variants and the launch-graph mode")
    ap.add_argument("--no-n32", action="store_true", help="skip the short 32-qubit (32 GiB) run")
    ap.add_argument("--n34", action="store_true", help="add a short 34-qubit run (128 GiB state)")
    ap.add_argument("--no-small", action="store_true", help="skip the n=12 and n=20 configuration lines")
    ap.add_argument("--no-spectrum", action="store_true", help="skip the Lanczos spectrum lines")
    ap.add_argument("--serving-requests", type=int, default=1024,
                    help="requests in the batched-serving measurement (0 skips it)")
    ap.add_argument("--instance", default=INSTANCE,
                    help="committed instance to evolve (default: the n=30 benchmark instance); smaller ones are "
                         "for profiling captures")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
