#!/usr/bin/env python
"""Benchmark: QAOA objective + adjoint-gradient evaluations per second on
LABS n = 30, p = 10 (complex64 state, int32 cost vector), the workload of the
paper's GPU layer-time experiment, with the method's roofline.

One step = one call of the public C ABI ``qaoa_grad``: the forward simulation
of all p layers from |+>, the fused energy / ground-state overlap, and the
adjoint sweep giving all 2p angle derivatives.  The cost vector is
precomputed once before the timed region (as in the paper, where it is
cached and reused across evaluations); its build time is reported apart.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  With N > 1 (torchrun) every rank evaluates
its own replica (independent objective evaluations, no collective on the data
path), the time is the max over ranks and `value` counts all ranks' steps.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LABS n=30 p=10 objective+grad evals/s"
UNIT = "evals/s"
WORKLOAD = "labs30_p10"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-sample-n", type=int, default=23,
                    help="n of the oracle sample timed for the CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--qubits", "--n", dest="n", type=int, default=None,
                    help="LABS size override (a smaller case for profiling; default n=30)")
    ap.add_argument("--layers", "--p", dest="p", type=int, default=None,
                    help="layer-count override (default p=10)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=400)
    ap.add_argument("--serving-full-requests", type=int, default=32)
    return ap.parse_args()


# ----------------------------------------------------------------- helpers

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, ws):
    """Max of a float over all ranks (identity when ws == 1)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while running."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index):
        self.dev = dev_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


KERNEL_SOURCES = ("tma_kernels.cu", "kernels.h", "qaoa_common.cuh", "api.cu")


def kernel_source_hash():
    """sha256 (16 hex digits) over the sources of the tiled TMA kernels and
    their pass schedule, comments and blank space left out (a comment edit
    does not change what the counters measured)."""
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2309_04841_gb300", "csrc", f), encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        src = "\n".join(line.strip() for line in src.splitlines() if line.strip())
        h.update(src.encode())
    return h.hexdigest()[:16]


def traffic_record(kind, n, p):
    """Mean DRAM bytes per launch of `kind` on this workload from the
    committed ncu summary, or None when the kernel sources changed since the
    capture or the summary covers another workload."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("source_sha256_16") != kernel_source_hash():
        return None
    if rec.get("n") != n or rec.get("p") != p:
        return None
    k = rec.get("kernels", {}).get(kind)
    return None if k is None else k.get("dram_bytes_per_launch")


def cpu_baseline(sample_n, p, n_full):
    """Oracle (single-threaded C, complex128) obj+grad on LABS at a smaller n,
    scaled to n_full by the element-qubit work ratio n 2^n."""
    import numpy as np

    import oracle
    from paper_2309_04841_gb300 import inputs as I
    f = oracle.labs_costs(sample_n).astype(np.float64)
    g = I.angles(p, 6)
    b = I.angles(p, 16)
    t = time.perf_counter()
    oracle.grad(sample_n, f, g, b)
    dt = time.perf_counter() - t
    scale = (n_full * 2.0 ** n_full) / (sample_n * 2.0 ** sample_n)
    return {"value": 1.0 / (dt * scale), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"1 objective+gradient evaluation of LABS n={sample_n}, p={p} by the "
                       f"oracle (C, complex128, 1 thread) in {dt:.2f} s, scaled to n={n_full} "
                       f"by n*2^n ({scale:.0f}x)"),
            "sample_seconds": dt}


def group_kinds(kinds, steps):
    """Per-kind profile entries ("bwd_high.k6") summed by pass group ("bwd_high")."""
    g = {}
    for k, v in kinds.items():
        e = g.setdefault(k.split(".")[0], {"launches": 0, "ms": 0.0, "bytes": 0.0})
        e["launches"] += v["launches"]
        e["ms"] += v["ms"]
        e["bytes"] += v["bytes"]
    return {k: {"launches": e["launches"], "ms_per_step": e["ms"] / steps,
                "GBps": e["bytes"] / (e["ms"] * 1e-3) / 1e9 if e["ms"] > 0 else None}
            for k, e in g.items()}


def bench_workload(a):
    from paper_2309_04841_gb300 import inputs as I
    w = I.workload(WORKLOAD, n=a.n)
    if a.p is not None:
        w["p"] = a.p
    if a.n is not None or a.p is not None:
        w["name"] = f"labs{w['n']}_p{w['p']}"
    return w


# --------------------------------------------------------------- our arm

def run_ours(a, ws, rank, local):
    import numpy as np
    import torch

    from paper_2309_04841_gb300 import inputs as I
    from paper_2309_04841_gb300 import qaoa as Q

    torch.cuda.set_device(local)
    Q.lib()
    w = bench_workload(a)
    n, p = w["n"], w["p"]
    N = 1 << n
    g, b = I.workload_angles(w)

    # precompute (outside the timed region), timed on its own
    costs = torch.empty(N, dtype=torch.int32, device="cuda")
    Q.labs_costs(n, out=costs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    Q.labs_costs(n, out=costs)
    e1.record()
    torch.cuda.synchronize()
    precompute_ms = e0.elapsed_time(e1)
    stats = Q.cost_stats_compute(costs)

    state = torch.empty(N, dtype=torch.complex64, device="cuda")
    lam = torch.empty_like(state)
    work = Q.workspace(n)
    out = torch.empty(2 + 2 * p, dtype=torch.float64, device="cuda")

    def step():
        Q.grad(costs, stats, g, b, state=state, lam=lam, work=work, out=out)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()

    # ---- device-timed region: inputs resident in HBM
    Q.profile_read(reset=True)
    Q.profile_enable(True)
    stream = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier(ws)
        torch.cuda.synchronize()
        t0.record(stream)
        for _ in range(a.steps):
            step()
        t1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
    Q.profile_enable(False)
    prof = Q.profile_read(reset=True)
    ms = max_over_ranks(t0.elapsed_time(t1), ws)
    value = a.steps * ws / (ms / 1000.0)
    result = out.cpu().numpy()

    # ---- the same workload with the cost vector stored as uint16 values
    # (lossless: LABS f < 2^16; the paper's compact storage, Sec. 4.4)
    costs16 = Q.convert_costs(costs, stats, Q.COST_U16)
    stats16 = Q.cost_stats_compute(costs16)

    def step16():
        Q.grad(costs16, stats16, g, b, state=state, lam=lam, work=work, out=out)

    for _ in range(a.warmup):
        step16()
    barrier(ws)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(a.steps):
        step16()
    t1.record(stream)
    torch.cuda.synchronize()
    ms16 = max_over_ranks(t0.elapsed_time(t1), ws)
    result16 = out.cpu().numpy()
    del costs16

    # ---- the XY ring mixer (Sec. 3.2) on LABS n = 28 from the half-filling
    # Dicke state: forward simulation with E and O, 4 layers
    nx, px = 28, 4
    fx = Q.labs_costs(nx)
    sx = Q.cost_stats_compute(fx)
    gx, bx = I.angles(px, 6), I.angles(px, 16)
    sv = Q.dicke_state(nx, nx // 2)
    wx = Q.workspace(nx)
    ox = torch.empty(2, dtype=torch.float64, device="cuda")
    for _ in range(a.warmup):
        Q.simulate_xy(fx, sx, gx, bx, sv, Q.XY_RING, work=wx, out=ox)
    torch.cuda.synchronize()
    Q.profile_read(reset=True)
    Q.profile_enable(True)
    t0.record(stream)
    for _ in range(a.steps):
        Q.simulate_xy(fx, sx, gx, bx, sv, Q.XY_RING, work=wx, out=ox)
    t1.record(stream)
    torch.cuda.synchronize()
    Q.profile_enable(False)
    msx = t0.elapsed_time(t1) / a.steps
    px_prof = Q.profile_read(reset=True).get("xy_tile", None)
    del fx, sv

    # ---- end to end through the public API with host buffers: angles from
    # pinned host memory (they travel in the launch parameters), the result
    # read back into pinned host memory every step
    h_ang = torch.empty(2 * p, dtype=torch.float64, pin_memory=True)
    h_ang[:p] = torch.from_numpy(g)
    h_ang[p:] = torch.from_numpy(b)
    h_out = torch.empty(2 + 2 * p, dtype=torch.float64, pin_memory=True)
    barrier(ws)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(a.steps):
        ang = h_ang.numpy()
        Q.grad(costs, stats, ang[:p], ang[p:], state=state, lam=lam, work=work, out=out)
        h_out.copy_(out, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t, ws)
    barrier(ws)

    # ---- roofline of the dominant kernel (by device time)
    peak, peak_src = measured_peaks()
    kinds = {k: v for k, v in prof.items() if v["launches"] > 0}
    dom = max(kinds, key=lambda k: kinds[k]["ms"])
    d = kinds[dom]
    per_launch_bytes = d["bytes"] / d["launches"]
    per_launch_ms = d["ms"] / d["launches"]
    achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
    traffic = traffic_record(dom, n, p)
    launches = sum(v["launches"] for v in kinds.values())
    step_bytes = (20.0 * p + 36.0 * p) * N  # forward + adjoint layers (algorithmic)
    step_alg = step_bytes * value / ws / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(w, ws),
        "e2e": {"value": a.steps * ws / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": 2 * p * 8, "d2h_bytes_per_step": (2 + 2 * p) * 8},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback 6.8 TB/s"},
        "step_roofline": {"algorithmic_bytes_per_step": step_bytes,
                          "achieved_GBps": step_alg, "frac": step_alg / peak},
        "kernel_groups": group_kinds(kinds, a.steps),
        "kernels": {k: {"launches": v["launches"], "ms_per_step": v["ms"] / a.steps,
                        "GBps": (v["bytes"] / v["launches"]) / ((v["ms"] / v["launches"]) * 1e-3) / 1e9
                        if v["ms"] > 0 else None} for k, v in kinds.items()},
        "variants": {"u16_costs": {
            "value": a.steps * ws / (ms16 / 1000.0), "unit": UNIT, "ms_per_step": ms16 / a.steps,
            "note": ("same workload and angles, cost vector held as uint16 values "
                     "(qaoa_convert_costs from the int32 vector; lossless since LABS f < 2^16)"),
            "result_identical": bool(np.array_equal(result16, result))},
            "xy_ring": {
                "workload": f"XY ring mixer, LABS n={nx}, p={px}, from the Dicke state k={nx // 2}, "
                            "forward simulation + energy/overlap, complex64",
                "ms_per_eval": msx, "layers_per_s": px * 1000.0 / msx,
                "tile_pass_GBps": (px_prof["bytes"] / px_prof["ms"] / 1e6) if px_prof else None,
                "tile_passes_per_layer": (px_prof["launches"] // (a.steps * px)) if px_prof else None}},
        "precompute_ms": precompute_ms,
        "result": {"energy": float(result[0]), "overlap": float(result[1])},
    }
    return line, clk.summary()


# ------------------------------------------------------------ serving

def serving_bench(count=400, nmin=16, nmax=26, loads=(0.5, 0.8, 0.95), graphs_per_n=4):
    """Serving loop vs the plain per-request path on one request stream."""
    import numpy as np
    import torch

    from paper_2309_04841_gb300 import inputs as I
    from paper_2309_04841_gb300 import qaoa as Q

    reqs = I.serving_stream(count, nmin=nmin, nmax=nmax, graphs_per_n=graphs_per_n)
    # plain path: one qaoa_grad after another on one stream, cost vectors cached
    cache = {}
    service = []
    for r in reqs:
        k = (r["problem"], r["n"], r["key"])
        if k not in cache:
            fd = Q.labs_costs(r["n"]) if r["problem"] == 0 else Q.maxcut_costs(r["n"], r["edges"], r["weights"])
            cache[k] = (fd, Q.cost_stats_compute(fd))
        fd, st = cache[k]
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = Q.grad(fd, st, r["gammas"], r["betas"])
        out.cpu()
        service.append(time.perf_counter() - t)
    del cache
    torch.cuda.empty_cache()
    service = np.array(service)
    plain_tput = count / service.sum()

    def sub(srv, r):
        return srv.submit(r["problem"], r["n"], r["gammas"], r["betas"], edges=r["edges"],
                          weights=r["weights"], key=r["key"], want_grad=True)

    free, _ = torch.cuda.mem_get_info()
    arena = int(min(free * 0.6, 96 << 30))
    srv = Q.Server(arena, max_inflight=8)
    for r in reqs[:8]:  # warm the cost-vector cache and the kernels
        srv.wait(sub(srv, r), r["p"])
    # saturated: everything submitted at once
    t0 = time.perf_counter()
    ts = [sub(srv, r) for r in reqs]
    for t, r in zip(ts, reqs):
        srv.wait(t, r["p"])
    sat_tput = count / (time.perf_counter() - t0)
    srv.close()
    pct = lambda v, q: float(v[min(len(v) - 1, int(round(q * (len(v) - 1))))])

    def open_loop(load):
        """Poisson arrivals at `load` x the saturated server throughput: the
        server's latencies (finish - submit) and those of the plain path as a
        FIFO single-server queue of the measured service times."""
        rate = load * sat_tput
        arr = I.poisson_arrivals(count, rate)
        srv = Q.Server(arena, max_inflight=8)
        for r in reqs[:8]:
            srv.wait(sub(srv, r), r["p"])
        base = time.perf_counter()
        ts = []
        for a, r in zip(arr, reqs):
            d = base + a - time.perf_counter()
            if d > 0:
                time.sleep(d)
            ts.append(sub(srv, r))
        lat = []
        for t, r in zip(ts, reqs):
            res = srv.wait(t, r["p"])
            lat.append(res["finish_s"] - res["submit_s"])
        srv.close()
        lat = np.sort(np.array(lat)) * 1000
        fin, plat = 0.0, []
        for a, sv in zip(arr, service):
            fin = max(fin, a) + sv
            plat.append(fin - a)
        plat = np.sort(np.array(plat)) * 1000
        return {"load": load, "arrival_rate_per_s": rate,
                "server_p50_ms": pct(lat, 0.5), "server_p99_ms": pct(lat, 0.99),
                "plain_p50_ms": pct(plat, 0.5), "plain_p99_ms": pct(plat, 0.99)}

    sweep = [open_loop(x) for x in loads]
    mid = sweep[len(sweep) // 2]
    return {"requests": count,
            "recipe": (f"objective+gradient requests, n ~ U{{{nmin}..{nmax}}} (MaxCut rounded up to even), "
                       f"p ~ U{{1..40}}, LABS or MaxCut 3-regular 50/50 ({graphs_per_n} graphs per n), complex64; "
                       "Poisson arrivals at " + " / ".join(f"{x:g}" for x in loads)
                       + " x the saturated server throughput; arena " + f"{arena / 2**30:.0f} GiB"),
            "server": {"evals_per_s_saturated": sat_tput, "arrival_rate_per_s": mid["arrival_rate_per_s"],
                       "p50_ms": mid["server_p50_ms"], "p99_ms": mid["server_p99_ms"]},
            "plain_per_request": {"evals_per_s": plain_tput, "p50_ms": mid["plain_p50_ms"],
                                  "p99_ms": mid["plain_p99_ms"]},
            "load_sweep": sweep}


# ------------------------------------------------------- reference arm

def workload_config(w, ws):
    """The workload's description, the same on both arms."""
    n, p = w["n"], w["p"]
    N = 1 << n
    return {"workload": f"LABS n={n} p={p} objective+gradient ({w['name']})",
            "n": n, "p": p, "state": "complex64", "cost": "int32",
            "angles": "gamma, beta ~ U[0, pi) seeds 6 / 16",
            "l2": f"inputs larger than L2 ({8 * N / 2**30:g} GiB state, {4 * N / 2**30:g} GiB cost vector)",
            "parallelism": f"replicas x{ws}"}


def run_reference(a, ws, rank):
    """The oracle timed on the host cores: each step is one bounded sample
    (obj+grad at n = cpu_sample_n), expressed in n = 30 evals/s."""
    if rank != 0:
        return None
    w = bench_workload(a)
    for _ in range(a.warmup):
        cpu_baseline(min(a.cpu_sample_n, 16), w["p"], w["n"])
    vals, secs = [], []
    for _ in range(a.steps):
        r = cpu_baseline(a.cpu_sample_n, w["p"], w["n"])
        vals.append(r["value"])
        secs.append(r["sample_seconds"])
    v = len(vals) / sum(1.0 / x for x in vals)
    cb = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": r["sample"]}
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000.0 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(w, ws),
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    a = parse()
    ws, rank, local = dist_env()
    if a.impl != "reference" and ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if a.impl == "reference":
        line = run_reference(a, ws, rank)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    line, clocks = run_ours(a, ws, rank, local)
    if rank == 0:
        line["clocks"] = clocks
        if not a.no_serving:
            line["serving"] = serving_bench(a.serving_requests)
            # the full size range, up to n = 32 (32 GiB state + 32 GiB lambda
            # + 16 GiB costs), admitted by footprint
            line["serving_full_range"] = serving_bench(a.serving_full_requests, 16, 32, loads=(0.8,),
                                                       graphs_per_n=1)
        if not a.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(a.cpu_sample_n, line["config"]["p"],
                                                line["config"]["n"])
            line["cpu_baseline"].pop("sample_seconds", None)
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
