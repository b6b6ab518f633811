"""Shared helpers for the GPU parity tests (compare the CUDA path with the
oracle on the same seeded inputs)."""
import numpy as np

import oracle
from paper_2309_04841_gb300 import inputs as I


def torch():
    import torch as T
    return T


def dev_np(t):
    return t.detach().cpu().numpy()


def oracle_costs(w):
    """(float64 costs for the oracle, costs in the workload's storage dtype)
    for a named workload recipe (see inputs.WORKLOADS)."""
    n = w["n"]
    if w["problem"] == "labs":
        f = oracle.labs_costs(n)
        return f.astype(np.float64), oracle.to_i32_checked(f)
    edges, wt = I.workload_graph(w)
    f = oracle.maxcut_costs(n, edges, wt)
    if w["cost"] == "i32":
        return f, oracle.to_i32_checked(np.rint(f).astype(np.int64))
    f32 = oracle.to_f32_rne(f)
    return f32.astype(np.float64), f32


def gpu_costs(w):
    """The same cost vector built by the CUDA library."""
    from paper_2309_04841_gb300 import qaoa as Q
    n = w["n"]
    if w["problem"] == "labs":
        return Q.labs_costs(n)
    edges, wt = I.workload_graph(w)
    ct = Q.COST_I32 if w["cost"] == "i32" else Q.COST_F32
    return Q.maxcut_costs(n, edges, wt, cost_type=ct)


def rel_state_err(a, b):
    """||a - b|| / ||b|| for complex vectors (numpy)."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def fidelity(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))
