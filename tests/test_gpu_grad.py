"""Adjoint gradient on the GPU vs the oracle's stored-state reverse mode
(n <= 16) and vs central differences of the GPU's own complex128 forward at
full size (a property that holds at any n).

Tolerance: the gradient is compared norm-wise, ||g - g_ref|| / ||g_ref||,
because single components can vanish by symmetry.  complex64 accumulates
FP32 rounding through 2p(n+1) passes of the forward and adjoint sweeps;
1e-4 covers p <= 40 with margin.  complex128: 1e-9."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2309_04841_gb300 import inputs as I

from gpu_util import dev_np, gpu_costs, oracle_costs, torch

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"{path} not generated")
    with open(path) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def Q():
    from paper_2309_04841_gb300 import qaoa
    qaoa.lib()
    return qaoa


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("st,tol", [("c64", 1e-4), ("c128", 1e-9)])
@pytest.mark.parametrize("n,p", [(3, 2), (8, 4), (12, 3), (13, 2), (14, 3), (16, 4)])
def test_grad_vs_oracle_labs(Q, n, p, st, tol):
    f = oracle.labs_costs(n).astype(float)
    fd = Q.labs_costs(n)
    stats = Q.cost_stats_compute(fd)
    g = I.angles(p, 10 + n, 0, 0.1)
    b = I.angles(p, 20 + n)
    out = dev_np(Q.grad(fd, stats, g, b, state_type=Q.C64 if st == "c64" else Q.C128))
    E, dg, db = oracle.grad(n, f, g, b)
    assert abs(out[0] - E) <= (1e-5 if st == "c64" else 1e-10) * abs(E)
    assert rel(np.concatenate([out[2:2 + p], out[2 + p:]]), np.concatenate([dg, db])) < tol


@pytest.mark.parametrize("cost", ["i32", "f32"])
@pytest.mark.parametrize("n,p", [(21, 3), (21, 1)])
def test_grad_cluster_pair_vs_oracle(Q, cost, n, p):
    # n = 21: the adjoint's HIGH group takes qubits 12..20 on a cluster pair
    # (one group instead of two; qubit 20 split across the two CTAs, rotated
    # after the exchange); int32 and float32 cost tiles (LABS energies, scaled
    # and perturbed for the latter)
    f = oracle.labs_costs(n).astype(float)
    if cost == "i32":
        fd = Q.labs_costs(n)
    else:
        f = (0.37 * f + I.uniform(5, 1 << n, -0.5, 0.5)).astype(np.float32).astype(float)
        fd = torch().tensor(f.astype(np.float32), device="cuda")
    stats = Q.cost_stats_compute(fd)
    g = I.angles(p, 40 + n, 0, 0.2)
    b = I.angles(p, 41 + n)
    out = dev_np(Q.grad(fd, stats, g, b))
    E, dg, db = oracle.grad(n, f, g, b)
    assert abs(out[0] - E) <= 1e-5 * max(1.0, abs(E))
    assert rel(np.concatenate([out[2:2 + p], out[2 + p:]]), np.concatenate([dg, db])) < 1e-4


@pytest.mark.parametrize("impl", ["wide", "pair"])
@pytest.mark.parametrize("n,p", [(13, 2), (17, 3), (22, 2), (24, 2)])
def test_grad_forced_pairs_vs_oracle(Q, monkeypatch, n, p, impl):
    # every HIGH group of the adjoint a 9-qubit group (one 512-thread CTA per
    # 2^13-amplitude tile, or a cluster pair for every pass), including groups
    # that rotate only some of the 9 qubits: n = 13 only the top one, n = 17
    # round 0's bits and the top one, n = 22 a full group then the top qubit
    # alone, n = 24 a full group then three qubits
    monkeypatch.setenv("QAOA_ADJOINT_PAIRS", "always")
    if impl == "pair":
        monkeypatch.setenv("QAOA_ADJOINT_WIDE", "pair")
    f = oracle.labs_costs(n).astype(float)
    fd = Q.labs_costs(n)
    stats = Q.cost_stats_compute(fd)
    g = I.angles(p, 50 + n, 0, 0.2)
    b = I.angles(p, 51 + n)
    Q.profile_enable(True)
    try:
        Q.profile_read()
        out = dev_np(Q.grad(fd, stats, g, b))
        kinds = Q.profile_read()
    finally:
        Q.profile_enable(False)
    assert not any(k.startswith("bwd_high") for k in kinds)
    if impl == "pair":
        assert any(k.startswith("bwd_pair") for k in kinds) and not any(k.startswith("bwd_wide") for k in kinds)
    else:
        assert any(k.startswith("bwd_wide") for k in kinds)
    E, dg, db = oracle.grad(n, f, g, b)
    assert abs(out[0] - E) <= 1e-5 * max(1.0, abs(E))
    assert rel(np.concatenate([out[2:2 + p], out[2 + p:]]), np.concatenate([dg, db])) < 1e-4


@pytest.mark.parametrize("st,tol", [("c64", 1e-4), ("c128", 1e-9)])
@pytest.mark.parametrize("n,p", [(13, 3), (16, 4)])
def test_grad_f64_costs_vs_oracle(Q, n, p, st, tol):
    # float64 costs take the tiled passes for both state types (reduced-form
    # rotations, the dropped factors folded into the phase and the last pass,
    # each round's gradient sums weighted back)
    terms = I.random_terms(n, 24, 7, max_order=3, integer=False)
    f = oracle.costs_terms_real(n, terms)
    fd = Q.precompute_costs(n, terms, Q.COST_F64)
    stats = Q.cost_stats_compute(fd)
    g = I.angles(p, 60 + n, 0, 0.4)
    b = I.angles(p, 61 + n)
    out = dev_np(Q.grad(fd, stats, g, b, state_type=Q.C64 if st == "c64" else Q.C128))
    E, dg, db = oracle.grad(n, f, g, b)
    assert abs(out[0] - E) <= (1e-5 if st == "c64" else 1e-10) * max(1.0, abs(E))
    assert rel(np.concatenate([out[2:2 + p], out[2 + p:]]), np.concatenate([dg, db])) < tol


def test_grad_wide_and_pair_agree_n30_p2(Q, monkeypatch):
    # the headline plan's 9-qubit groups on the 512-thread CTA and on cluster
    # pairs: the same arithmetic in another order, agreement to rounding
    w = I.workload("labs30_p2")
    n = w["n"]
    fd = Q.labs_costs(n)
    stats = Q.cost_stats_compute(fd)
    g, b = I.workload_angles(w)
    res = {}
    for impl in ("wide", "pair"):
        if impl == "pair":
            monkeypatch.setenv("QAOA_ADJOINT_WIDE", "pair")
        res[impl] = dev_np(Q.grad(fd, stats, g, b))
    a, c = res["wide"], res["pair"]
    assert abs(a[0] - c[0]) <= 1e-7 * abs(c[0])
    assert rel(a[2:], c[2:]) < 1e-5


def test_grad_pair_plans_agree_n26(Q, monkeypatch):
    # the same gradient from the plain adjoint plan and from the plan with
    # every HIGH group on a cluster pair (n = 26: {12-20}, {17-25} rotating
    # 21-25), both in complex64: agreement to rounding
    n, p = 26, 3
    fd = Q.labs_costs(n)
    stats = Q.cost_stats_compute(fd)
    g = I.angles(p, 6, 0, 0.3)
    b = I.angles(p, 16)
    res = {}
    for mode in ("never", "always"):
        monkeypatch.setenv("QAOA_ADJOINT_PAIRS", mode)
        res[mode] = dev_np(Q.grad(fd, stats, g, b))
    a, c = res["never"], res["always"]
    assert abs(a[0] - c[0]) <= 1e-6 * abs(a[0])
    assert rel(c[2:], a[2:]) < 1e-5


@pytest.mark.parametrize("n,p", [(10, 5), (16, 6)])
def test_grad_vs_oracle_weighted_maxcut(Q, n, p):
    w = I.workload("maxcut3w28_p40", n=n)
    f, _ = oracle_costs(w)
    fd = gpu_costs(w)
    stats = Q.cost_stats_compute(fd)
    g = I.angles(p, 31, 0, 0.3)
    b = I.angles(p, 32)
    out = dev_np(Q.grad(fd, stats, g, b))
    E, dg, db = oracle.grad(n, f, g, b)
    assert rel(np.concatenate([out[2:2 + p], out[2 + p:]]), np.concatenate([dg, db])) < 1e-4


def test_grad_many_layers_small_chunked(Q):
    # p > 128 on the on-chip path: forward chunks then adjoint chunks
    n, p = 7, 150
    f = oracle.labs_costs(n).astype(float)
    fd = Q.labs_costs(n)
    stats = Q.cost_stats_compute(fd)
    g = I.angles(p, 41, 0, 0.05)
    b = I.angles(p, 42)
    out = dev_np(Q.grad(fd, stats, g, b, state_type=Q.C128))
    E, dg, db = oracle.grad(n, f, g, b)
    assert rel(np.concatenate([out[2:2 + p], out[2 + p:]]), np.concatenate([dg, db])) < 1e-9


def test_grad_uncompute_returns_plus(Q):
    # after the adjoint sweep psi is back at |+> (layers un-applied in place)
    T = torch()
    n, p = 18, 3
    fd = Q.labs_costs(n)
    stats = Q.cost_stats_compute(fd)
    state = T.empty(1 << n, dtype=T.complex64, device="cuda")
    Q.grad(fd, stats, I.angles(p, 1, 0, 0.1), I.angles(p, 2), state=state)
    s = dev_np(state).astype(np.complex128)
    assert np.max(np.abs(s - 2.0 ** (-n / 2))) < 1e-5 * 2.0 ** (-n / 2) * 10


@pytest.mark.parametrize("n", [28, 30])
def test_grad_uncompute_drift_fullsize(Q, n):
    # the adjoint un-applies all p = 40 layers in place with no stored state:
    # the state it ends on must be |+> again.  Relative L2 drift
    # ||psi_0 - |+>|| / |||+>|| below 1e-5, the threshold beyond which
    # checkpointed states would be needed.
    T = torch()
    w = I.workload("labs30_p40", n=n)
    fd = Q.labs_costs(n)
    stats = Q.cost_stats_compute(fd)
    g, b = I.workload_angles(w)
    state = T.empty(1 << n, dtype=T.complex64, device="cuda")
    Q.grad(fd, stats, g, b, state=state)
    plus = 2.0 ** (-n / 2)
    drift = float(T.linalg.vector_norm((state - plus).to(T.complex128)).item())
    del state, fd
    T.cuda.empty_cache()
    assert drift < 1e-5, drift


@pytest.mark.parametrize("name", ["labs28_p40", "maxcut3w28_p40"])
def test_grad_fullsize_directional_fd(Q, name):
    # n = 28, p = 40, all 80 gradients in one adjoint sweep; checked by a
    # central difference of the complex128 forward along a random direction
    w = I.workload(name)
    fd = gpu_costs(w)
    stats = Q.cost_stats_compute(fd)
    g, b = I.angles(w["p"], w["gamma_seed"], 0, w["ghi"]), I.angles(w["p"], w["beta_seed"])
    T = torch()
    out = dev_np(Q.grad(fd, stats, g, b))
    p = w["p"]
    grad = np.concatenate([out[2:2 + p], out[2 + p:]])
    v = I.uniform(99, 2 * p, -1, 1)
    v /= np.linalg.norm(v)
    fmax = max(abs(stats.f_min), abs(stats.f_max))
    h = 1e-4 / max(1.0, fmax / 10)

    def E(t):
        st, o = Q.simulate(fd, stats, g + t * v[:p], b + t * v[p:], state_type=Q.C128)
        e = float(dev_np(o)[0])
        del st
        return e

    fd1 = (E(h) - E(-h)) / (2 * h)
    fd2 = (E(h / 2) - E(-h / 2)) / h
    dd = (4 * fd2 - fd1) / 3
    T.cuda.empty_cache()
    assert abs(np.dot(grad, v) - dd) <= 1e-4 * np.linalg.norm(grad)


def test_grad_labs30_vs_oracle_central_differences(Q):
    # the headline size's adjoint schedule (n = 30: groups {0-11}, {12-20},
    # {21-29}, both HIGH groups on cluster pairs) against the FP64 oracle:
    # central differences of the oracle energy at h = 1e-4 and 5e-5 combined
    # by Richardson extrapolation (tests/golden, make_golden.py --fd), all
    # four angles of p = 2; complex64 at the stated 1e-4
    G = _golden("oracle_fd_labs30_p2.json")
    w = I.workload("labs30_p2")
    p = w["p"]
    fd = Q.labs_costs(w["n"])
    stats = Q.cost_stats_compute(fd)
    g, b = I.workload_angles(w)
    out = dev_np(Q.grad(fd, stats, g, b, state_type=Q.C64))
    del fd
    torch().cuda.empty_cache()
    ref = np.concatenate([G["dgamma"], G["dbeta"]])
    assert abs(out[0] - G["energy"]) <= 1e-5 * abs(G["energy"])
    assert rel(np.concatenate([out[2:2 + p], out[2 + p:]]), ref) < 1e-4


def test_grad_labs28_vs_oracle_reverse_mode(Q):
    # n = 28 (the gradient workloads' size): every component against the
    # oracle's stored-state reverse-mode gradient (make_golden.py --grad)
    G = _golden("oracle_grad_labs28_p2.json")
    w = I.workload("labs28_p2")
    p = w["p"]
    fd = Q.labs_costs(w["n"])
    stats = Q.cost_stats_compute(fd)
    g, b = I.workload_angles(w)
    out = dev_np(Q.grad(fd, stats, g, b, state_type=Q.C64))
    del fd
    torch().cuda.empty_cache()
    ref = np.concatenate([G["dgamma"], G["dbeta"]])
    assert abs(out[0] - G["energy"]) <= 1e-5 * abs(G["energy"])
    assert rel(np.concatenate([out[2:2 + p], out[2 + p:]]), ref) < 1e-4


@pytest.mark.parametrize("n", [29, 30])
def test_grad_c64_vs_c128_fullsize(Q, n):
    # cross-check of the two GPU paths at n = 29, 30 (the complex64 adjoint
    # runs one or both HIGH groups on cluster pairs there): every component
    # against the complex128 adjoint (whose own parity with the oracle is
    # checked at n <= 16; the oracle checks at n = 28, 30 are above)
    w = I.workload("labs30_p10", n=n)
    fd = gpu_costs(w)
    stats = Q.cost_stats_compute(fd)
    g, b = I.angles(w["p"], w["gamma_seed"], 0, w["ghi"]), I.angles(w["p"], w["beta_seed"])
    T = torch()
    o64 = dev_np(Q.grad(fd, stats, g, b, state_type=Q.C64))
    T.cuda.empty_cache()
    o128 = dev_np(Q.grad(fd, stats, g, b, state_type=Q.C128))
    T.cuda.empty_cache()
    p = w["p"]
    assert abs(o64[0] - o128[0]) <= 1e-5 * abs(o128[0])
    assert rel(o64[2:2 + 2 * p], o128[2:2 + 2 * p]) < 1e-4


def test_autograd_function(Q):
    T = torch()
    n, p = 10, 3
    fd = Q.labs_costs(n)
    stats = Q.cost_stats_compute(fd)
    g = T.tensor(I.angles(p, 3, 0, 0.1), dtype=T.float64, requires_grad=True)
    b = T.tensor(I.angles(p, 4), dtype=T.float64, requires_grad=True)
    E = Q.qaoa_energy(fd, stats, g, b, state_type=Q.C128)
    E.backward()
    f = oracle.labs_costs(n).astype(float)
    E0, dg, db = oracle.grad(n, f, g.detach().numpy(), b.detach().numpy())
    assert abs(E.item() - E0) < 1e-10 * abs(E0)
    assert rel(np.concatenate([g.grad.numpy(), b.grad.numpy()]), np.concatenate([dg, db])) < 1e-9
