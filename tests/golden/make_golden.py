"""Write the stored oracle values under tests/golden/.

Every value here comes from the CPU oracle (oracle/) on inputs from
paper_2309_04841_gb300.inputs; nothing is taken from the CUDA path.  The
oracle itself is pinned by tests/test_oracle.py.

  python tests/golden/make_golden.py --labs-max 30
  python tests/golden/make_golden.py --configs maxcut3_n14_p2 maxcut_gnp26_p6
  python tests/golden/make_golden.py --configs labs30_p10 labs30_p10_smallgamma
  python tests/golden/make_golden.py --state-samples labs30_p40
  python tests/golden/make_golden.py --grad labs28_p2
  python tests/golden/make_golden.py --fd labs30_p2

labs_optima.json  : LABS minimum f and number of minimisers, n = 3..labs-max
                    (exhaustive enumeration by the oracle).
oracle_<name>.json: energy, ground-state overlap and cost-vector statistics of
                    a named workload, from the oracle's Algorithm 3 in
                    complex128.  For float32 cost workloads the oracle
                    simulates the float32-rounded cost vector (the cost vector
                    the workload defines), widened back to float64.
oracle_<name>_amps.npy: the oracle's amplitudes at seeded sample indices and
                    at every minimiser (--state-samples).
oracle_grad_<name>.json: the oracle's reverse-mode gradient (--grad).
oracle_fd_<name>.json: central differences of the oracle energy (--fd).
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2309_04841_gb300 import inputs as I  # noqa: E402


def _labs_chunk(args):
    n, x0, x1, shm_name = args
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=shm_name)
    out = np.ndarray((1 << n,), dtype=np.int64, buffer=shm.buf)
    out[x0:x1] = oracle.labs_costs_range(n, x0, x1)
    del out
    shm.close()
    return x1 - x0


def labs_costs_parallel(n, procs=8):
    """Oracle LABS vector; large n splits the index range over processes
    (each process runs the same plain oracle routine on its range)."""
    if n <= 22:
        return oracle.labs_costs(n)
    from multiprocessing import shared_memory
    N = 1 << n
    shm = shared_memory.SharedMemory(create=True, size=N * 8)
    try:
        chunk = N // (procs * 8)
        jobs = [(n, x, min(N, x + chunk), shm.name) for x in range(0, N, chunk)]
        ctx = mp.get_context("spawn")
        with ctx.Pool(procs) as pool:
            assert sum(pool.map(_labs_chunk, jobs)) == N
        out = np.ndarray((N,), dtype=np.int64, buffer=shm.buf).copy()
    finally:
        shm.close()
        shm.unlink()
    return out


def labs_optima(nmax, path):
    res = {}
    if os.path.exists(path):
        with open(path) as fh:
            res = json.load(fh).get("optima", {})
    for n in range(3, nmax + 1):
        if str(n) in res:
            continue
        t = time.time()
        f = labs_costs_parallel(n)
        fmin = int(f.min())
        res[str(n)] = [fmin, int(np.sum(f == fmin))]
        print(f"labs n={n}: min={fmin} count={res[str(n)][1]} ({time.time() - t:.1f}s)",
              flush=True)
        with open(path, "w") as fh:
            json.dump({"source": "oracle exhaustive enumeration (oracle/oracle.c "
                                 "oracle_labs_cost_at), written by make_golden.py",
                       "format": "n -> [min f, number of minimisers]",
                       "optima": res}, fh, indent=1)


def workload_costs(w):
    """(f as float64 for the oracle, f in the workload's storage dtype)."""
    n = w["n"]
    if w["problem"] == "labs":
        f = labs_costs_parallel(n)
        return f.astype(np.float64), oracle.to_i32_checked(f)
    edges, wt = I.workload_graph(w)
    f = oracle.maxcut_costs(n, edges, wt)
    if w["cost"] == "i32":
        fi = oracle.to_i32_checked(np.rint(f).astype(np.int64))
        assert np.all(fi == f)
        return f, fi
    f32 = oracle.to_f32_rne(f)
    return f32.astype(np.float64), f32


def config_values(name):
    w = I.workload(name)
    n = w["n"]
    t0 = time.time()
    f64, fstore = workload_costs(w)
    print(f"{name}: costs {time.time() - t0:.1f}s", flush=True)
    g, b = I.workload_angles(w)
    t1 = time.time()
    psi = oracle.simulate(n, f64, g, b)
    t2 = time.time()
    E = oracle.energy(n, psi, f64)
    O = oracle.overlap(n, psi, f64)
    fmin = float(f64.min())
    out = {
        "workload": name, "recipe": {k: v for k, v in w.items()},
        "energy": E, "overlap": O,
        "f_min": fmin, "f_max": float(f64.max()),
        "n_min": int(np.sum(f64 == fmin)),
        "f_mean": float(np.mean(f64)),
        "cost_dtype": str(fstore.dtype),
        "cost_sha256": hashlib.sha256(np.ascontiguousarray(fstore).tobytes()).hexdigest(),
        "oracle_seconds_simulate": t2 - t1,
        "source": "oracle/oracle.c (oracle_simulate, oracle_energy, oracle_overlap), "
                  "complex128, written by make_golden.py",
    }
    with open(os.path.join(HERE, f"oracle_{name}.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(f"{name}: E={E:.15g} O={O:.6g} ({t2 - t1:.1f}s simulate)", flush=True)


SAMPLE_SEED = 71  # seed of the sampled amplitude indices (inputs.sample_indices)


def state_samples(name, count):
    """Energy, overlap and the oracle's amplitudes at `count` seeded indices
    plus every ground state (f == f_min) of a named workload.  The amplitudes
    go to oracle_<name>_amps.npy (complex128, in the order of the stored
    index list: the sampled indices, then the minimisers)."""
    w = I.workload(name)
    n = w["n"]
    f64, fstore = workload_costs(w)
    sha = hashlib.sha256(np.ascontiguousarray(fstore).tobytes()).hexdigest()
    del fstore
    g, b = I.workload_angles(w)
    t1 = time.time()
    psi = oracle.simulate(n, f64, g, b)
    t2 = time.time()
    E = oracle.energy(n, psi, f64)
    O = oracle.overlap(n, psi, f64)
    fmin = float(f64.min())
    opt = np.flatnonzero(f64 == fmin)
    idx = np.concatenate([I.sample_indices(n, count, SAMPLE_SEED), opt]).astype(np.int64)
    amps = np.ascontiguousarray(psi[idx])
    np.save(os.path.join(HERE, f"oracle_{name}_amps.npy"), amps)
    out = {
        "workload": name, "recipe": {k: v for k, v in w.items()},
        "energy": E, "overlap": O, "f_min": fmin, "n_min": int(opt.size),
        "norm": float(np.vdot(psi, psi).real),
        "samples": {"count": int(count), "seed": SAMPLE_SEED,
                    "generator": "inputs.sample_indices(n, count, seed)",
                    "minimisers": [int(x) for x in opt],
                    "amplitudes": f"oracle_{name}_amps.npy",
                    "sampled_norm2": float(np.vdot(amps[:count], amps[:count]).real)},
        "cost_sha256": sha,
        "oracle_seconds_simulate": t2 - t1,
        "source": "oracle/oracle.c (oracle_simulate, oracle_energy, oracle_overlap), "
                  "complex128, written by make_golden.py",
    }
    with open(os.path.join(HERE, f"oracle_{name}.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(f"{name}: E={E:.15g} O={O:.6g} ({t2 - t1:.1f}s simulate)", flush=True)


def grad_values(name):
    """The oracle's stored-state reverse-mode gradient of a named workload."""
    w = I.workload(name)
    n = w["n"]
    f64, fstore = workload_costs(w)
    g, b = I.workload_angles(w)
    t1 = time.time()
    E, dg, db = oracle.grad(n, f64, g, b)
    t2 = time.time()
    out = {
        "workload": name, "recipe": {k: v for k, v in w.items()},
        "energy": E, "dgamma": [float(x) for x in dg], "dbeta": [float(x) for x in db],
        "cost_sha256": hashlib.sha256(np.ascontiguousarray(fstore).tobytes()).hexdigest(),
        "oracle_seconds": t2 - t1,
        "source": "oracle/oracle.c (oracle_grad: reverse mode over stored forward states), "
                  "complex128, written by make_golden.py",
    }
    with open(os.path.join(HERE, f"oracle_grad_{name}.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(f"{name}: E={E:.15g} dg={dg} db={db} ({t2 - t1:.1f}s)", flush=True)


FD_STEPS = (1e-4, 5e-5)


def fd_values(name):
    """Central differences of the oracle energy in every angle, at the steps
    FD_STEPS = (h, h/2), and their Richardson combination (4 D(h/2) - D(h)) / 3,
    whose error is O(h^4).  Every energy is one oracle simulation (Algorithm 3,
    complex128) of the shifted angles; the raw energies are stored too."""
    w = I.workload(name)
    n, p = w["n"], w["p"]
    f64, fstore = workload_costs(w)
    sha = hashlib.sha256(np.ascontiguousarray(fstore).tobytes()).hexdigest()
    del fstore
    g0, b0 = I.workload_angles(w)
    t0 = time.time()

    def energy(g, b):
        return oracle.energy(n, oracle.simulate(n, f64, g, b), f64)

    E0 = energy(g0, b0)
    comps = []
    for which in ("gamma", "beta"):
        for k in range(p):
            row = {"angle": which, "layer": k, "energies": {}}
            D = []
            for h in FD_STEPS:
                ep, em = [], []
                for sgn, lst in ((1.0, ep), (-1.0, em)):
                    g, b = g0.copy(), b0.copy()
                    (g if which == "gamma" else b)[k] += sgn * h
                    lst.append(energy(g, b))
                row["energies"][repr(h)] = [ep[0], em[0]]
                D.append((ep[0] - em[0]) / (2.0 * h))
                print(f"{name}: d/d{which}[{k}] h={h}: {D[-1]:.12g} "
                      f"({time.time() - t0:.0f}s)", flush=True)
            row["central"] = D
            row["richardson"] = (4.0 * D[1] - D[0]) / 3.0
            comps.append(row)
    out = {
        "workload": name, "recipe": {k: v for k, v in w.items()},
        "energy": E0, "steps": list(FD_STEPS),
        "dgamma": [r["richardson"] for r in comps if r["angle"] == "gamma"],
        "dbeta": [r["richardson"] for r in comps if r["angle"] == "beta"],
        "components": comps,
        "cost_sha256": sha,
        "oracle_seconds": time.time() - t0,
        "source": "oracle/oracle.c (oracle_simulate, oracle_energy) at shifted angles, "
                  "complex128, central differences + Richardson, written by make_golden.py",
    }
    with open(os.path.join(HERE, f"oracle_fd_{name}.json"), "w") as fh:
        json.dump(out, fh, indent=1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--labs-max", type=int, default=0)
    ap.add_argument("--configs", nargs="*", default=[])
    ap.add_argument("--state-samples", nargs="*", default=[],
                    help="workloads whose sampled amplitudes are stored")
    ap.add_argument("--samples", type=int, default=65536)
    ap.add_argument("--grad", nargs="*", default=[], help="oracle_grad workloads")
    ap.add_argument("--fd", nargs="*", default=[], help="finite-difference workloads")
    a = ap.parse_args()
    if a.labs_max:
        labs_optima(a.labs_max, os.path.join(HERE, "labs_optima.json"))
    for c in a.configs:
        config_values(c)
    for c in a.state_samples:
        state_samples(c, a.samples)
    for c in a.grad:
        grad_values(c)
    for c in a.fd:
        fd_values(c)


if __name__ == "__main__":
    main()
