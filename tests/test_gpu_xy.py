"""XY mixers (ring, complete graph; Sec. 3.2) and the Dicke state on the GPU
against the oracle, element by element.  Tolerances as the transverse-field
forward tests: complex64 2e-5 (state) / 1e-5 (energy), complex128 1e-11 /
1e-10.  Sizes span one tile (n <= 12), several tiles with passes on low and
high qubits, and the complete graph's one-gate fallback (pairs no tile
holds, n > 12).  The complex64 ring from n = 13 runs on register rounds over
TMA-streamed tiles: n = 13 (the wrap gate in the LOW pass), 14 (a HIGH pass
whose rows overlap the LOW tile's), 21 and 22 (one and two HIGH passes with
rows above it), 23 at p = 3."""
import numpy as np
import pytest

import oracle
from paper_2309_04841_gb300 import inputs as I

from gpu_util import dev_np, torch

pytestmark = pytest.mark.gpu
TOL = {"c64": (2e-5, 1e-5), "c128": (1e-11, 1e-10)}


@pytest.fixture(scope="module")
def Q():
    from paper_2309_04841_gb300 import qaoa
    qaoa.lib()
    return qaoa


@pytest.mark.parametrize("n,k,st", [(5, 2, "c64"), (14, 7, "c64"), (13, 0, "c128"), (12, 12, "c64")])
def test_dicke_state(Q, n, k, st):
    stype = Q.C64 if st == "c64" else Q.C128
    got = dev_np(Q.dicke_state(n, k, stype)).astype(np.complex128)
    np.testing.assert_allclose(got, oracle.dicke(n, k), rtol=0, atol=TOL[st][0] / np.sqrt(1 << n))


@pytest.mark.parametrize("graph", [1, 2])
@pytest.mark.parametrize("n,st", [(2, "c64"), (3, "c128"), (3, "c64"), (4, "c64"), (9, "c128"), (12, "c64"),
                                  (13, "c64"), (14, "c64"), (16, "c64"), (16, "c128"), (19, "c64"),
                                  (21, "c64"), (22, "c64")])
def test_simulate_xy_vs_oracle(Q, n, st, graph):
    stype = Q.C64 if st == "c64" else Q.C128
    f = oracle.labs_costs(n).astype(float)
    fd = Q.labs_costs(n)
    stats = Q.cost_stats_compute(fd)
    g, b = I.angles(2, 90 + n, 0, 0.3), I.angles(2, 91 + n)
    psi0 = oracle.dicke(n, n // 2)
    state = Q.dicke_state(n, n // 2, stype)
    state, out = Q.simulate_xy(fd, stats, g, b, state, graph)
    ref = oracle.simulate_xy(n, f, g, b, psi0, graph)
    got = dev_np(state).astype(np.complex128)
    ts, te = TOL[st]
    assert np.linalg.norm(got - ref) <= ts * np.linalg.norm(ref)
    o = dev_np(out)
    E, O = oracle.energy(n, ref, f), oracle.overlap(n, ref, f)
    assert abs(o[0] - E) <= te * max(1.0, abs(E))
    assert abs(o[1] - O) <= te * max(1e-3, O) + 1e-12


def test_xy_keeps_hamming_weight_on_gpu(Q):
    n = 18
    fd = Q.labs_costs(n)
    stats = Q.cost_stats_compute(fd)
    T = torch()
    # equal mix of the weight-5 and weight-9 Dicke states
    state = (Q.dicke_state(n, 5) + Q.dicke_state(n, 9)) / np.sqrt(2)
    state, _ = Q.simulate_xy(fd, stats, [0.1, 0.4], [0.8, 2.1], state.contiguous(), Q.XY_RING)
    p = dev_np(state).astype(np.complex128)
    w = np.array([bin(x).count("1") for x in range(1 << n)])
    for k in range(n + 1):
        want = 0.5 if k in (5, 9) else 0.0
        assert abs(np.sum(np.abs(p[w == k]) ** 2) - want) < 2e-6


@pytest.mark.parametrize("kind", ["f32", "u16"])
def test_simulate_xy_other_cost_types(Q, kind):
    # float32 costs take the computed phase, uint16 costs the digit tables
    # read as 2-byte words
    n = 15
    if kind == "f32":
        edges, w = I.maxcut_3reg(n + 1, graph_seed=6, weighted=True, weight_seed=7)
        n = n + 1
        f = oracle.maxcut_costs(n, edges, w)
        fd = Q.maxcut_costs(n, edges, w, Q.COST_F32)
        f = oracle.to_f32_rne(f).astype(float)
    else:
        f = oracle.labs_costs(n).astype(float)
        fd = Q.labs_costs_u16(n)
    stats = Q.cost_stats_compute(fd)
    g, b = I.angles(2, 95, 0, 0.4), I.angles(2, 96)
    psi0 = oracle.dicke(n, n // 2)
    state = Q.dicke_state(n, n // 2)
    state, out = Q.simulate_xy(fd, stats, g, b, state, Q.XY_RING)
    ref = oracle.simulate_xy(n, f, g, b, psi0, 1)
    got = dev_np(state).astype(np.complex128)
    assert np.linalg.norm(got - ref) <= 2e-5 * np.linalg.norm(ref)
    E = oracle.energy(n, ref, f)
    assert abs(dev_np(out)[0] - E) <= 1e-5 * max(1.0, abs(E))


def test_simulate_xy_ring_deeper(Q):
    # three layers of the ring at n = 23 (LOW pass and two HIGH passes per
    # layer; each layer's phase opens its LOW pass after the previous layer's
    # wrap gate)
    n, p = 23, 3
    f = oracle.labs_costs(n).astype(float)
    fd = Q.labs_costs(n)
    stats = Q.cost_stats_compute(fd)
    g, b = I.angles(p, 97, 0, 0.2), I.angles(p, 98)
    psi0 = oracle.dicke(n, 11)
    state, out = Q.simulate_xy(fd, stats, g, b, Q.dicke_state(n, 11), Q.XY_RING)
    ref = oracle.simulate_xy(n, f, g, b, psi0, 1)
    got = dev_np(state).astype(np.complex128)
    assert np.linalg.norm(got - ref) <= 2e-5 * np.linalg.norm(ref)
    E = oracle.energy(n, ref, f)
    assert abs(dev_np(out)[0] - E) <= 1e-5 * max(1.0, abs(E))
