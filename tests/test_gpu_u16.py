"""uint16 cost vectors (QAOA_COST_U16): the paper stores the LABS diagonal as
uint16 (Sec. 5.2, distributed simulation).  The values are the int32 ones, so
every result must be bit-identical to the int32 run: the kernels differ only
in how they load the cost words.  The builder itself is checked against the oracle bit-exactly."""
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


def u16_np(t):
    return dev_np(t).view(np.uint16)


@pytest.mark.parametrize("n", [2, 5, 13, 20, 24])
def test_labs_u16_bit_exact(Q, n):
    got = u16_np(Q.labs_costs_u16(n)).astype(np.int64)
    np.testing.assert_array_equal(got, oracle.labs_costs(n))


@pytest.mark.parametrize("n", [9, 18])
def test_convert_round_trip_and_stats(Q, n):
    fi = Q.labs_costs(n)
    si = Q.cost_stats_compute(fi)
    fu = Q.convert_costs(fi, si, Q.COST_U16)
    np.testing.assert_array_equal(u16_np(fu), u16_np(Q.labs_costs_u16(n)))
    su = Q.cost_stats_compute(fu)
    assert (su.f_min, su.f_max, su.n_min, su.step_log2) == (si.f_min, si.f_max, si.n_min, si.step_log2)
    back = Q.convert_costs(fu, su, Q.COST_I32)
    np.testing.assert_array_equal(dev_np(back), dev_np(fi))


def test_convert_rejects_out_of_range(Q):
    # MaxCut costs are <= 0: not representable as uint16
    n = 10
    edges, w = I.maxcut_3reg(n, graph_seed=2)
    fi = Q.maxcut_costs(n, edges, w, Q.COST_I32)
    with pytest.raises(Q.QAOAError) as e:
        Q.convert_costs(fi, Q.cost_stats_compute(fi), Q.COST_U16)
    assert e.value.status == 3  # QAOA_ERR_OVERFLOW


@pytest.mark.parametrize("n,st", [(10, "c64"), (16, "c64"), (21, "c64"), (22, "c64"), (25, "c64"),
                                  (16, "c128")])
def test_simulate_and_grad_match_int32_bit_for_bit(Q, n, st):
    T = torch()
    stype = Q.C64 if st == "c64" else Q.C128
    fi = Q.labs_costs(n)
    fu = Q.labs_costs_u16(n)
    si, su = Q.cost_stats_compute(fi), Q.cost_stats_compute(fu)
    g, b = I.angles(4, 70, 0, 0.3), I.angles(4, 71)
    s_i, o_i = Q.simulate(fi, si, g, b, state_type=stype)
    s_u, o_u = Q.simulate(fu, su, g, b, state_type=stype)
    np.testing.assert_array_equal(dev_np(s_u), dev_np(s_i))
    np.testing.assert_array_equal(dev_np(o_u), dev_np(o_i))
    gi = dev_np(Q.grad(fi, si, g, b, state_type=stype))
    gu = dev_np(Q.grad(fu, su, g, b, state_type=stype))
    np.testing.assert_array_equal(gu, gi)
    # the standalone reductions read uint16 too
    assert float(Q.expectation(s_u, fu)[0]) == float(Q.expectation(s_i, fi)[0])
    assert float(Q.overlap(s_u, fu, su)[0]) == float(Q.overlap(s_i, fi, si)[0])


def test_u16_forward_vs_oracle(Q):
    n = 14
    f = oracle.labs_costs(n).astype(float)
    fu = Q.labs_costs_u16(n)
    su = Q.cost_stats_compute(fu)
    g, b = I.angles(3, 72, 0, 0.2), I.angles(3, 73)
    state, out = Q.simulate(fu, su, g, b)
    ref = oracle.simulate(n, f, g, b)
    got = dev_np(state).astype(np.complex128)
    assert np.linalg.norm(got - ref) <= 2e-5 * np.linalg.norm(ref)
    E = oracle.energy(n, ref, f)
    assert abs(dev_np(out)[0] - E) <= 1e-5 * abs(E)
