"""Cost vector (Sec. 3.1, Eq. 1) on the GPU vs the oracle: bit-exact."""
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


@pytest.mark.parametrize("n", list(range(2, 21)) + [23])
def test_labs_direct_bit_exact(Q, n):
    f = dev_np(Q.labs_costs(n))
    np.testing.assert_array_equal(f, oracle.labs_costs(n))


@pytest.mark.parametrize("n", [4, 9, 13, 16])
def test_labs_terms_path_bit_exact(Q, n):
    f = dev_np(Q.precompute_costs(n, Q.labs_terms(n), Q.COST_I32))
    np.testing.assert_array_equal(f, oracle.labs_costs(n))


def test_labs_n30_sampled(Q):
    # full-size LABS vector: sampled entries against the oracle's one-by-one
    # evaluation, plus the enumerated optimum (min 59, 16 minimisers)
    n = 30
    f = Q.labs_costs(n)
    T = torch()
    idx = I.randint(77, 4096, 1 << 30)
    got = dev_np(f[T.as_tensor(idx, device="cuda")])
    want = np.array([oracle.labs_cost_at(n, int(x)) for x in idx])
    np.testing.assert_array_equal(got, want)
    st = Q.cost_stats_compute(f)
    assert (st.f_min, st.n_min) == (59.0, 16)
    assert st.f_max == (n - 1) * n * (2 * n - 1) // 6


@pytest.mark.parametrize("n,seed", [(5, 1), (12, 2), (17, 3)])
def test_integer_terms_bit_exact(Q, n, seed):
    terms = I.random_terms(n, 60, seed, max_order=6, integer=True)
    got = dev_np(Q.precompute_costs(n, terms, Q.COST_I32))
    np.testing.assert_array_equal(got, oracle.costs_terms_int(n, terms))


def test_integer_terms_chunked(Q):
    # more terms than one parameter block: accumulated over launches
    n = 11
    terms = I.random_terms(n, 2500, 5, max_order=4, integer=True)
    got = dev_np(Q.precompute_costs(n, terms, Q.COST_I32))
    np.testing.assert_array_equal(got, oracle.costs_terms_int(n, terms))


@pytest.mark.parametrize("ct", ["f32", "f64"])
@pytest.mark.parametrize("n,seed", [(6, 11), (14, 12)])
def test_real_terms_bit_exact(Q, n, seed, ct):
    terms = I.random_terms(n, 50, seed, max_order=4, integer=False)
    want = oracle.costs_terms_real(n, terms)
    if ct == "f32":
        got = dev_np(Q.precompute_costs(n, terms, Q.COST_F32))
        np.testing.assert_array_equal(got, oracle.to_f32_rne(want))
    else:
        got = dev_np(Q.precompute_costs(n, terms, Q.COST_F64))
        np.testing.assert_array_equal(got, want)


def test_nondyadic_f64_terms_follow_term_order(Q):
    # weights like 0.1 are not dyadic: float64 additions in term order, the
    # same order as the oracle's loop, give the same bits
    n = 12
    terms = [(0.1 * (k + 1), (k % n, (3 * k + 1) % n)) for k in range(40)] + [(1 / 3, ())]
    got = dev_np(Q.precompute_costs(n, terms, Q.COST_F64))
    np.testing.assert_array_equal(got, oracle.costs_terms_real(n, terms))


@pytest.mark.parametrize("n,weighted", [(8, False), (14, False), (14, True), (20, True)])
def test_maxcut_direct_bit_exact(Q, n, weighted):
    edges, w = I.maxcut_3reg(n, graph_seed=n, weighted=weighted, weight_seed=n + 1)
    want = oracle.maxcut_costs(n, edges, w)
    if weighted:
        got = dev_np(Q.maxcut_costs(n, edges, w, cost_type=Q.COST_F32))
        np.testing.assert_array_equal(got, oracle.to_f32_rne(want))
        got = dev_np(Q.maxcut_costs(n, edges, w, cost_type=Q.COST_F64))
        np.testing.assert_array_equal(got, want)
    else:
        got = dev_np(Q.maxcut_costs(n, edges, w, cost_type=Q.COST_I32))
        np.testing.assert_array_equal(got, want.astype(np.int32))


def test_maxcut_gnp26_bit_exact_and_terms_agree(Q):
    w = I.workload("maxcut_gnp26_p6")
    edges, wt = I.workload_graph(w)
    n = w["n"]
    got = Q.maxcut_costs(n, edges, wt, cost_type=Q.COST_F32)
    want = oracle.to_f32_rne(oracle.maxcut_costs(n, edges, wt))
    np.testing.assert_array_equal(dev_np(got), want)
    via_terms = Q.precompute_costs(n, Q.maxcut_terms(n, edges, wt), Q.COST_F32)
    np.testing.assert_array_equal(dev_np(via_terms), want)


@pytest.mark.parametrize("n", [3, 13, 22])
def test_cost_stats(Q, n):
    f = Q.labs_costs(n)
    ref = oracle.labs_costs(n)
    st = Q.cost_stats_compute(f)
    assert st.f_min == ref.min() and st.f_max == ref.max()
    assert st.n_min == int(np.sum(ref == ref.min()))
    # float costs
    edges, wt = I.maxcut_3reg(max(n, 4) if n % 2 == 0 else n + 1, graph_seed=2, weighted=True)
    m = max(n, 4) if n % 2 == 0 else n + 1
    g = Q.maxcut_costs(m, edges, wt, cost_type=Q.COST_F32)
    r = oracle.to_f32_rne(oracle.maxcut_costs(m, edges, wt)).astype(np.float64)
    st = Q.cost_stats_compute(g)
    assert st.f_min == r.min() and st.f_max == r.max() and st.n_min == int(np.sum(r == r.min()))


def test_empty_terms_give_zero(Q):
    got = dev_np(Q.precompute_costs(9, [], Q.COST_I32))
    assert np.all(got == 0)
