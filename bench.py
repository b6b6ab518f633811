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

Besides the headline line's required keys it reports: the roofline of the
adjoint sweep and of the forward sweep on algorithmic bytes (20 B per
amplitude per forward layer, 36 B per adjoint layer), the per-pass DRAM rates
(`kernel_efficiency`), the error of every result against the stored
complex128 oracle values (`result_error`), the other named workloads
(`variants`), the serving loop against the plain per-request path on a
1000-request stream (`serving`), and the oracle timed on the host cores
(`cpu_baseline`, one core and all cores).
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
GOLDEN = os.path.join(ROOT, "tests", "golden")

METRIC = "LABS n=30 p=10 objective+grad evals/s"
UNIT = "evals/s"
WORKLOAD = "labs30_p10"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-sample-n", type=int, default=22,
                    help="n of the oracle sample each reference-arm step runs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--qubits", "--n", dest="n", type=int, default=None,
                    help="LABS size override (a smaller case for profiling; default n=30)")
    ap.add_argument("--layers", "--p", dest="p", type=int, default=None,
                    help="layer-count override (default p=10)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=1000)
    ap.add_argument("--serving-nmax", type=int, default=28)
    ap.add_argument("--serving-full", type=int, default=0,
                    help="also run this many requests over n ~ U{16..32} (minutes)")
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


def golden(name):
    """Stored oracle values (tests/golden, written by make_golden.py from the
    oracle alone), or None."""
    try:
        with open(os.path.join(GOLDEN, name)) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return None


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


def traffic_record(n, p):
    """DRAM bytes per pass kind measured by ncu (profiles/traffic.json), or
    None when the kernel sources changed since the capture or the capture
    covers another workload."""
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
    return rec.get("kernels")


def cost_build_line(n, N, ms):
    """The LABS cost-vector build against the popcount rate: n - 1 popcounts
    per element (one per shift k), at 16 per clock per SM (the CUDA
    arithmetic-throughput table's figure for 32-bit population count) and the
    maximum SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = 16.0 * sms * 2.07e9 / 1e9
    rate = (n - 1) * N / (ms * 1e-3) / 1e9
    return {"kernel": "k_labs (LABS cost vector, int32), outside the timed region", "ms": ms,
            "Gelements_per_s": N / (ms * 1e-3) / 1e9, "bound": "alu", "unit": "Gpopc/s",
            "achieved": rate, "peak": peak, "frac": rate / peak,
            "peak_source": f"16 popc per clock per SM x {sms} SMs x 2070 MHz (maximum SM clock)"}


def sweep_split(prof, steps):
    """Per-step device time (ms) and pass bytes of the forward ("fwd_*") and
    adjoint ("bwd_*") launches."""
    out = {}
    for side, pre in (("forward", "fwd_"), ("adjoint", "bwd_")):
        ks = {k: v for k, v in prof.items() if k.startswith(pre) and v["launches"] > 0}
        out[side] = {"ms": sum(v["ms"] for v in ks.values()) / steps,
                     "pass_bytes": sum(v["bytes"] for v in ks.values()) / steps,
                     "launches": sum(v["launches"] for v in ks.values()) // steps}
    return out


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


def rel_err(x, ref):
    return abs(x - ref) / abs(ref) if ref else abs(x - ref)


def timed(fn, reps, stream):
    """Mean device time (ms) of fn() over reps calls, CUDA events on `stream`."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


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
    # the adjoint un-applied every layer in place: psi is |+> again
    drift = float(torch.linalg.vector_norm((state - 2.0 ** (-n / 2)).to(torch.complex128)).item())

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

    # ---- rooflines on algorithmic bytes (N amplitudes, complex64 8 B, int32
    # cost 4 B): a forward layer reads psi and f and writes psi (20 B N), an
    # adjoint layer reads psi, lambda, f and writes psi, lambda (36 B N)
    peak, peak_src = measured_peaks()
    kinds = {k: v for k, v in prof.items() if v["launches"] > 0}
    sp = sweep_split(kinds, a.steps)
    alg_adj = 36.0 * N * p
    alg_fwd = 20.0 * N * p
    ach_adj = alg_adj / (sp["adjoint"]["ms"] * 1e-3) / 1e9
    ach_fwd = alg_fwd / (sp["forward"]["ms"] * 1e-3) / 1e9
    traffic = traffic_record(n, p)
    dram_adj = None
    if traffic:
        dram_adj = sum(v["dram_bytes_per_launch"] * kinds[k]["launches"] / a.steps
                       for k, v in traffic.items() if k.startswith("bwd_") and k in kinds)
    launches = sum(v["launches"] for v in kinds.values())
    step_bytes = alg_fwd + alg_adj
    step_alg = step_bytes * value / ws / 1e9
    # the fastest-to-slowest pass kinds by the DRAM rate of their own bytes
    eff = {k: {"launches": v["launches"], "ms_per_step": v["ms"] / a.steps,
               "pass_bytes_per_launch": v["bytes"] / v["launches"],
               "GBps": (v["bytes"] / v["launches"]) / ((v["ms"] / v["launches"]) * 1e-3) / 1e9
               if v["ms"] > 0 else None} for k, v in kinds.items()}
    dom = max(kinds, key=lambda k: kinds[k]["ms"])

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(w, ws),
        "e2e": {"value": a.steps * ws / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": 2 * p * 8, "d2h_bytes_per_step": (2 + 2 * p) * 8},
        "gpu_launches": launches,
        "roofline": {
            "bound": "hbm",
            "kernel": "adjoint sweep: every k_bwd_tma / k_bwd_pair launch of one evaluation",
            "achieved": ach_adj, "peak": peak, "unit": "GB/s", "frac": ach_adj / peak,
            "traffic": dram_adj,
            "algorithmic_bytes_per_launch": alg_adj,
            "launch": f"one adjoint sweep = p={p} layers x 36 B x 2^{n} amplitudes, "
                      f"{sp['adjoint']['launches']} kernel launches",
            "ms_per_launch": sp["adjoint"]["ms"],
            "pass_structure_bytes_per_launch": sp["adjoint"]["pass_bytes"],
            "peak_source": (f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                            else "fallback 6.8 TB/s")},
        "forward_roofline": {
            "kernel": "forward sweep: every k_fwd_tma launch of one evaluation (energy fused)",
            "achieved": ach_fwd, "peak": peak, "unit": "GB/s", "frac": ach_fwd / peak,
            "algorithmic_bytes_per_launch": alg_fwd, "ms_per_launch": sp["forward"]["ms"],
            "pass_structure_bytes_per_launch": sp["forward"]["pass_bytes"],
            "launches": sp["forward"]["launches"]},
        "step_roofline": {"algorithmic_bytes_per_step": step_bytes,
                          "pass_structure_bytes_per_step": sp["forward"]["pass_bytes"]
                          + sp["adjoint"]["pass_bytes"],
                          "achieved_GBps": step_alg, "frac": step_alg / peak},
        "kernel_efficiency": {
            "note": "each pass kind's own bytes (the vectors it streams once) over its event "
                    "time: the DRAM rate of the passes, not the method's algorithmic rate",
            "dominant": dom, "dominant_GBps": eff[dom]["GBps"],
            "dominant_frac": eff[dom]["GBps"] / peak if eff[dom]["GBps"] else None,
            "kinds": eff},
        "kernel_groups": group_kinds(kinds, a.steps),
        "precompute_ms": precompute_ms,
        "cost_build": cost_build_line(n, N, precompute_ms),
        "result": {"energy": float(result[0]), "overlap": float(result[1]),
                   "uncompute_drift": drift},
    }
    G = golden(f"oracle_{WORKLOAD}.json")
    if G and G["recipe"]["n"] == n and G["recipe"]["p"] == p:
        line["result_error"] = {
            "energy_rel": rel_err(float(result[0]), G["energy"]),
            "overlap_rel": rel_err(float(result[1]), G["overlap"]),
            "oracle": f"tests/golden/oracle_{WORKLOAD}.json (oracle, complex128): "
                      f"E={G['energy']:.12g}, O={G['overlap']:.6g}",
            "bound": "1e-5 relative (complex64 state)"}
    del lam
    if not a.no_variants:
        line["variants"] = variants(a, ws, costs, stats, state, work, out, g, b, w, stream)
    return line, clk.summary()


def variants(a, ws, costs, stats, state, work, out, g, b, w, stream):
    """The other named workloads, each timed with CUDA events (inputs resident)."""
    import numpy as np
    import torch

    from paper_2309_04841_gb300 import inputs as I
    from paper_2309_04841_gb300 import qaoa as Q
    peak, _ = measured_peaks()
    n, p = w["n"], w["p"]
    N = 1 << n
    res = {}
    reps = max(2, a.steps)

    # the same workload with the cost vector held as uint16 values (lossless:
    # LABS f < 2^16; the compact storage of the paper's distributed section)
    costs16 = Q.convert_costs(costs, stats, Q.COST_U16)
    stats16 = Q.cost_stats_compute(costs16)
    lam = torch.empty_like(state)
    ref_out = out.cpu().numpy()
    f16 = lambda: Q.grad(costs16, stats16, g, b, state=state, lam=lam, work=work, out=out)
    f16()
    ms16 = timed(f16, reps, stream)
    res["u16_costs"] = {
        "value": 1000.0 / ms16, "unit": UNIT, "ms_per_eval": ms16,
        "note": "same workload and angles, cost vector as uint16 (qaoa_convert_costs)",
        "result_identical": bool(np.array_equal(out.cpu().numpy(), ref_out))}
    del costs16

    # the headline workload in complex128 (the paper's precision; 36 GiB)
    s128 = torch.empty(N, dtype=torch.complex128, device="cuda")
    l128 = torch.empty_like(s128)
    f128 = lambda: Q.grad(costs, stats, g, b, state=s128, lam=l128, work=work, out=out)
    f128()
    ms128 = timed(f128, max(2, reps // 2), stream)
    o128 = out.cpu().numpy()
    del s128, l128
    torch.cuda.empty_cache()
    G = golden(f"oracle_{WORKLOAD}.json")
    e = {"workload": f"LABS n={n} p={p} objective+gradient, complex128 state, int32 costs",
         "value": 1000.0 / ms128, "unit": UNIT, "ms_per_eval": ms128,
         # complex128: a forward layer moves 16 + 4 + 16 B per amplitude, an
         # adjoint layer 2 * 32 + 4 B
         "step_alg_frac": (36.0 + 68.0) * N * p / (ms128 * 1e-3) / 1e9 / peak,
         "energy": float(o128[0])}
    if G and G["recipe"]["n"] == n and G["recipe"]["p"] == p:
        e["energy_rel_err"] = rel_err(float(o128[0]), G["energy"])
        e["overlap_rel_err"] = rel_err(float(o128[1]), G["overlap"])
    res["labs30_p10_c128"] = e

    # XY ring mixer (Sec. 3.2) on LABS n = 28 from the half-filling Dicke
    # state: forward simulation with E and O, 4 layers
    nx, px = 28, 4
    fx = Q.labs_costs(nx)
    sx = Q.cost_stats_compute(fx)
    gx, bx = I.angles(px, 6), I.angles(px, 16)
    sv = Q.dicke_state(nx, nx // 2)
    wx = Q.workspace(nx)
    ox = torch.empty(2, dtype=torch.float64, device="cuda")
    fxy = lambda: Q.simulate_xy(fx, sx, gx, bx, sv, Q.XY_RING, work=wx, out=ox)
    fxy()
    Q.profile_read(reset=True)
    Q.profile_enable(True)
    msx = timed(fxy, reps, stream)
    Q.profile_enable(False)
    px_prof = Q.profile_read(reset=True).get("xy_tile", None)
    res["xy_ring"] = {
        "workload": f"XY ring mixer, LABS n={nx}, p={px}, from the Dicke state k={nx // 2}, "
                    "forward simulation + energy/overlap, complex64",
        "ms_per_eval": msx, "layers_per_s": px * 1000.0 / msx,
        "tile_pass_GBps": (px_prof["bytes"] / px_prof["ms"] / 1e6) if px_prof else None,
        "tile_passes_per_layer": (px_prof["launches"] // (reps * px)) if px_prof else None}
    del fx, sv
    torch.cuda.empty_cache()

    # MaxCut on a random 3-regular graph, n = 14, p = 2, complex128: forward
    # energy + overlap, a latency-bound evaluation
    res["maxcut3_n14_p2_c128"] = forward_variant("maxcut3_n14_p2", Q.C128, 200, stream, peak)
    # weighted G(26, 0.5), p = 6, float32 costs: complex64 and complex128
    res["maxcut_gnp26_p6_c64"] = forward_variant("maxcut_gnp26_p6", Q.C64, 20, stream, peak)
    res["maxcut_gnp26_p6_c128"] = forward_variant("maxcut_gnp26_p6", Q.C128, 10, stream, peak)
    # p = 40 gradients at n = 28 (LABS; weighted 3-regular MaxCut, float32 costs)
    res["labs28_p40_grad"] = grad_variant("labs28_p40", 3, stream, peak)
    res["maxcut3w28_p40_grad"] = grad_variant("maxcut3w28_p40", 3, stream, peak)
    return res


def variant_costs(w):
    from paper_2309_04841_gb300 import inputs as I
    from paper_2309_04841_gb300 import qaoa as Q
    if w["problem"] == "labs":
        return Q.labs_costs(w["n"])
    edges, wt = I.workload_graph(w)
    ct = Q.COST_I32 if w["cost"] == "i32" else Q.COST_F32
    return Q.maxcut_costs(w["n"], edges, wt, cost_type=ct)


def forward_variant(name, st, reps, stream, peak):
    """Forward simulation + fused energy / overlap of a named workload."""
    import torch

    from paper_2309_04841_gb300 import inputs as I
    from paper_2309_04841_gb300 import qaoa as Q
    w = I.workload(name)
    n, p = w["n"], w["p"]
    N = 1 << n
    fd = variant_costs(w)
    stats = Q.cost_stats_compute(fd)
    g, b = I.workload_angles(w)
    s = torch.empty(N, dtype=Q.state_dtype(st), device="cuda")
    work = Q.workspace(n)
    o = torch.empty(2, dtype=torch.float64, device="cuda")
    f = lambda: Q.simulate(fd, stats, g, b, state=s, work=work, out=o)
    for _ in range(3):
        f()
    ms = timed(f, reps, stream)
    r = o.cpu().numpy()
    es = 16.0 if st == Q.C128 else 8.0
    cb = float(fd.element_size())
    alg = (2 * es + cb) * N * p  # read psi and f, write psi, per layer
    v = {"workload": f"{name}: n={n} p={p}, {'complex128' if st == Q.C128 else 'complex64'} state, "
                     f"{w['cost']} costs, forward + energy/overlap",
         "us_per_eval": ms * 1e3, "evals_per_s": 1000.0 / ms, "layers_per_s": p * 1000.0 / ms,
         "alg_GBps": alg / (ms * 1e-3) / 1e9, "alg_frac": alg / (ms * 1e-3) / 1e9 / peak,
         "energy": float(r[0]), "overlap": float(r[1])}
    G = golden(f"oracle_{name}.json")
    if G:
        v["energy_rel_err"] = rel_err(float(r[0]), G["energy"])
        v["overlap_rel_err"] = rel_err(float(r[1]), G["overlap"])
    del s, fd
    torch.cuda.empty_cache()
    return v


def grad_variant(name, reps, stream, peak):
    """Objective + gradient of a named p = 40 workload, with its forward and
    adjoint sweeps' algorithmic rates."""
    import torch

    from paper_2309_04841_gb300 import inputs as I
    from paper_2309_04841_gb300 import qaoa as Q
    w = I.workload(name)
    n, p = w["n"], w["p"]
    N = 1 << n
    fd = variant_costs(w)
    stats = Q.cost_stats_compute(fd)
    g, b = I.workload_angles(w)
    s = torch.empty(N, dtype=torch.complex64, device="cuda")
    lam = torch.empty_like(s)
    work = Q.workspace(n)
    o = torch.empty(2 + 2 * p, dtype=torch.float64, device="cuda")
    f = lambda: Q.grad(fd, stats, g, b, state=s, lam=lam, work=work, out=o)
    f()
    Q.profile_read(reset=True)
    Q.profile_enable(True)
    ms = timed(f, reps, stream)
    Q.profile_enable(False)
    sp = sweep_split({k: v for k, v in Q.profile_read(reset=True).items() if v["launches"] > 0}, reps)
    cb = float(fd.element_size())
    a_adj = (32.0 + cb) * N * p
    a_fwd = (16.0 + cb) * N * p
    del s, lam, fd
    torch.cuda.empty_cache()
    return {"workload": f"{name}: n={n} p={p}, complex64, {w['cost']} costs, objective + all "
                        f"{2 * p} gradients",
            "ms_per_eval": ms, "evals_per_s": 1000.0 / ms,
            "adjoint_alg_GBps": a_adj / (sp["adjoint"]["ms"] * 1e-3) / 1e9,
            "adjoint_alg_frac": a_adj / (sp["adjoint"]["ms"] * 1e-3) / 1e9 / peak,
            "forward_alg_GBps": a_fwd / (sp["forward"]["ms"] * 1e-3) / 1e9,
            "forward_alg_frac": a_fwd / (sp["forward"]["ms"] * 1e-3) / 1e9 / peak,
            "passes_per_eval": {"forward": sp["forward"]["launches"],
                                "adjoint": sp["adjoint"]["launches"]}}


# ------------------------------------------------------------ serving

def serving_bench(count=1000, nmin=16, nmax=28, loads=(0.5, 0.8, 0.95), graphs_per_n=4):
    """Serving loop vs the plain per-request path (one qaoa_grad after another
    on one stream, cost vectors cached) on the same request stream: saturated
    throughput, then open-loop Poisson arrivals at fractions of the server's
    saturated throughput, each path run for real under the same arrivals."""
    import numpy as np
    import torch

    from paper_2309_04841_gb300 import inputs as I
    from paper_2309_04841_gb300 import qaoa as Q

    reqs = I.serving_stream(count, nmin=nmin, nmax=nmax, graphs_per_n=graphs_per_n)
    cache = {}

    def plain(r):
        k = (r["problem"], r["n"], r["key"])
        if k not in cache:
            fd = Q.labs_costs(r["n"]) if r["problem"] == 0 else Q.maxcut_costs(r["n"], r["edges"], r["weights"])
            cache[k] = (fd, Q.cost_stats_compute(fd))
        fd, st = cache[k]
        Q.grad(fd, st, r["gammas"], r["betas"]).cpu()

    for r in reqs[:8]:
        plain(r)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in reqs:
        plain(r)
    plain_tput = count / (time.perf_counter() - t0)

    def sub(srv, r):
        return srv.submit(r["problem"], r["n"], r["gammas"], r["betas"], edges=r["edges"],
                          weights=r["weights"], key=r["key"], want_grad=True)

    free, _ = torch.cuda.mem_get_info()
    # room for several mid-size requests beside the largest one (n = 32 takes
    # 80 GiB: state, lambda and costs)
    arena = int(min(free * (0.6 if nmax <= 28 else 0.75), (96 if nmax <= 28 else 176) << 30))
    srv = Q.Server(arena, max_inflight=8)
    for r in reqs[:8]:  # warm the cost-vector cache and the kernels
        srv.wait(sub(srv, r), r["p"])
    t0 = time.perf_counter()
    ts = [sub(srv, r) for r in reqs]
    for t, r in zip(ts, reqs):
        srv.wait(t, r["p"])
    sat_tput = count / (time.perf_counter() - t0)
    srv.close()
    torch.cuda.empty_cache()
    pct = lambda v, q: float(v[min(len(v) - 1, int(round(q * (len(v) - 1))))])

    def open_loop(load):
        rate = load * sat_tput
        arr = I.poisson_arrivals(count, rate)
        srv = Q.Server(arena, max_inflight=8)
        for r in reqs[:8]:
            srv.wait(sub(srv, r), r["p"])
        base = time.perf_counter()
        ts = []
        for at, r in zip(arr, reqs):
            d = base + at - time.perf_counter()
            if d > 0:
                time.sleep(d)
            ts.append(sub(srv, r))
        lat = []
        for t, r in zip(ts, reqs):
            res = srv.wait(t, r["p"])
            lat.append(res["finish_s"] - res["submit_s"])
        srv.close()
        torch.cuda.empty_cache()
        lat = np.sort(np.array(lat)) * 1000
        # the plain path under the same arrivals: one request at a time, each
        # started at its arrival or when the previous one has finished
        base = time.perf_counter()
        plat = []
        for at, r in zip(arr, reqs):
            d = base + at - time.perf_counter()
            if d > 0:
                time.sleep(d)
            plain(r)
            plat.append(time.perf_counter() - (base + at))
        plat = np.sort(np.array(plat)) * 1000
        return {"load": load, "arrival_rate_per_s": rate,
                "server_p50_ms": pct(lat, 0.5), "server_p99_ms": pct(lat, 0.99),
                "plain_p50_ms": pct(plat, 0.5), "plain_p99_ms": pct(plat, 0.99)}

    sweep = [open_loop(x) for x in loads]
    del cache
    torch.cuda.empty_cache()
    mid = sweep[len(sweep) // 2]
    return {"requests": count,
            "recipe": (f"objective+gradient requests, n ~ U{{{nmin}..{nmax}}} (MaxCut rounded up to even), "
                       f"p ~ U{{1..40}}, LABS or MaxCut 3-regular 50/50 ({graphs_per_n} graphs per n), complex64; "
                       "Poisson arrivals at " + " / ".join(f"{x:g}" for x in loads)
                       + " x the saturated server throughput, both paths run open-loop under the "
                       "same arrivals; arena " + f"{arena / 2**30:.0f} GiB"),
            "server": {"evals_per_s_saturated": sat_tput, "arrival_rate_per_s": mid["arrival_rate_per_s"],
                       "p50_ms": mid["server_p50_ms"], "p99_ms": mid["server_p99_ms"]},
            "plain_per_request": {"evals_per_s": plain_tput, "p50_ms": mid["plain_p50_ms"],
                                  "p99_ms": mid["plain_p99_ms"]},
            "load_sweep": sweep}


# ------------------------------------------------------- CPU baselines

def cpu_times(ns, p, library):
    """Oracle objective + gradient of LABS at each n (p layers, angles of the
    headline workload's seeds): wall seconds and ns per amplitude-layer."""
    import numpy as np

    import oracle
    from paper_2309_04841_gb300 import inputs as I
    g, b = I.angles(p, 6), I.angles(p, 16)
    out = []
    for n in ns:
        f = oracle.labs_costs(n).astype(np.float64)
        t = time.perf_counter()
        oracle.grad(n, f, g, b, library=library)
        dt = time.perf_counter() - t
        out.append({"n": n, "seconds": dt, "evals_per_s": 1.0 / dt,
                    "ns_per_amplitude_layer": dt * 1e9 / ((1 << n) * p)})
    return out


def cpu_baseline(p, n_full):
    """The oracle (plain C, complex128, one thread) timed on the host: LABS
    objective + gradient at n = 14, 20, 23; the n_full figure follows from
    the largest sample's time per amplitude-layer.  The same source built
    with OpenMP runs on all host cores for the all-core figure."""
    import oracle
    ns = (14, 20, 23)
    one = cpu_times(ns, p, oracle.lib())
    per = one[-1]["ns_per_amplitude_layer"]
    ncores = os.cpu_count() or 1
    allc = cpu_times(ns[1:], p, oracle.lib_omp())
    per_all = allc[-1]["ns_per_amplitude_layer"]
    scale = (1 << n_full) * p * 1e-9
    stored = golden(f"oracle_{WORKLOAD}.json")
    cb = {"value": 1.0 / (per * scale), "unit": UNIT, "cores": 1, "kind": "oracle",
          "sample": (f"oracle (C, complex128, 1 thread) objective+gradient of LABS p={p} measured "
                     f"at n = {', '.join(str(x) for x in ns)}; value = n={n_full} at the n={ns[-1]} "
                     f"time per amplitude-layer ({per:.1f} ns)"),
          "value_basis": "extrapolated from the measured samples by amplitude-layers",
          "measured": one,
          "all_cores": {"cores": ncores, "build": "same source, gcc -fopenmp (bit-identical results)",
                        "measured": allc, "value": 1.0 / (per_all * scale), "unit": UNIT}}
    if stored and "oracle_seconds_simulate" in stored:
        cb["n30_forward_stored"] = {
            "seconds": stored["oracle_seconds_simulate"],
            "what": f"oracle forward simulation (no gradient) of {WORKLOAD}, measured once when "
                    "tests/golden was written, on the x86_64 build container, 1 core",
            "ns_per_amplitude_layer": stored["oracle_seconds_simulate"] * 1e9 /
            ((1 << stored["recipe"]["n"]) * stored["recipe"]["p"])}
    return cb


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
    """The oracle timed on the host cores.  The paper's code is not part of
    this task, so the reference arm is the oracle: each step is one oracle
    objective + gradient of LABS at n = cpu_sample_n, p = 10 (complex128, one
    thread); `value` states it in n = 30 evaluations per second through the
    measured time per amplitude-layer."""
    if rank != 0:
        return None
    import numpy as np

    import oracle
    from paper_2309_04841_gb300 import inputs as I
    w = bench_workload(a)
    n, p = a.cpu_sample_n, w["p"]
    f = oracle.labs_costs(n).astype(np.float64)
    g, b = I.workload_angles(w)
    for _ in range(a.warmup):
        oracle.grad(n, f, g, b)
    secs = []
    for _ in range(a.steps):
        t = time.perf_counter()
        oracle.grad(n, f, g, b)
        secs.append(time.perf_counter() - t)
    step_s = sum(secs) / len(secs)
    per = step_s / ((1 << n) * p)
    v = 1.0 / (per * (1 << w["n"]) * p)
    cb = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
          "sample": f"oracle objective+gradient, LABS n={n} p={p}, complex128, 1 thread, "
                    f"{step_s:.3f} s per step"}
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": step_s * 1000.0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"oracle sample: LABS n={n} p={p} objective+gradient, complex128 "
                                   "state, float64 costs, 1 thread",
                       "n": n, "p": p, "state": "complex128", "cost": "float64",
                       "metric_workload": workload_config(w, ws)["workload"],
                       "value_basis": f"value = n={w['n']} evaluations/s at this sample's "
                                      f"{per * 1e9:.1f} ns per amplitude-layer; ms_per_step is the "
                                      "sample's own time"},
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
            line["serving"] = serving_bench(a.serving_requests, 16, a.serving_nmax)
            if a.serving_full:
                # the full size range, up to n = 32 (32 GiB state + 32 GiB lambda
                # + 16 GiB costs), admitted by footprint
                line["serving_full_range"] = serving_bench(a.serving_full, 16, 32, loads=(0.8,),
                                                           graphs_per_n=1)
        if not a.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(line["config"]["p"], line["config"]["n"])
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
