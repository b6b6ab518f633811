"""Output methods and the caller side (Sec. 4 get_* methods; Fig. 1 optimizer
loop): probabilities into a new array or in place, and a host Adam loop over
the device gradient, each checked against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2309_04841_gb300 import inputs as I

from gpu_util import dev_np, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_2309_04841_gb300 import qaoa
    qaoa.lib()
    return qaoa


@pytest.mark.parametrize("n,st", [(8, "c64"), (17, "c64"), (15, "c128")])
def test_probabilities(Q, n, st):
    stype = Q.C64 if st == "c64" else Q.C128
    f = oracle.labs_costs(n).astype(float)
    fd = Q.labs_costs(n)
    stats = Q.cost_stats_compute(fd)
    g, b = I.angles(3, 80, 0, 0.2), I.angles(3, 81)
    state, _ = Q.simulate(fd, stats, g, b, state_type=stype)
    before = dev_np(state).copy()
    pr = dev_np(Q.probabilities(state))
    ref = np.abs(oracle.simulate(n, f, g, b)) ** 2
    tol = 2e-6 if st == "c64" else 1e-13
    assert pr.dtype == (np.float32 if st == "c64" else np.float64)
    assert np.max(np.abs(pr - ref)) <= tol * max(1.0, ref.max()) * 10
    assert abs(pr.astype(np.float64).sum() - 1.0) <= (1e-5 if st == "c64" else 1e-12)
    np.testing.assert_array_equal(dev_np(state), before)  # preserved
    # in place: the state's real parts become the probabilities, imaginary 0
    real = Q.probabilities(state, preserve_state=False)
    got = dev_np(state)
    np.testing.assert_array_equal(got.real, pr)
    assert np.all(got.imag == 0)
    np.testing.assert_array_equal(dev_np(real), pr)


def test_optimizer_loop_descends(Q):
    # Fig. 1: precompute the diagonal, then optimizer <-> objective; the
    # energy history falls and its last entry is the oracle's energy at the
    # returned angles
    n, p = 10, 2
    edges, w = I.maxcut_3reg(n, graph_seed=4)
    f = oracle.maxcut_costs(n, edges, w)
    fd = Q.maxcut_costs(n, edges, w, Q.COST_I32)
    stats = Q.cost_stats_compute(fd)
    g0, b0 = np.array([0.1, 0.2]), np.array([0.3, 0.2])
    g, b, hist = Q.optimize(fd, stats, g0, b0, steps=60, lr=0.03)
    assert len(hist) == 61
    assert hist[-1] < hist[0] - 0.5
    E = oracle.energy(n, oracle.simulate(n, f, g, b), f)
    assert abs(hist[-1] - E) <= 1e-5 * abs(E)
