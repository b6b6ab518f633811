"""Pins for the CPU oracle (no GPU).  Each test ties an oracle routine to
something other than itself: a closed form, a dense matrix-exponential brute
force, an identity from the paper, a library routine, or a hand-checked small
case.  A dropped term, a wrong sign, a wrong bit index or a transposed
operand in the oracle fails at least one of them."""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sl

from paper_2309_04841_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ independent
# helpers written from textbook definitions, sharing nothing with the oracle.

def dense_x_sum(n):
    """sum_q X_q as a dense 2^n x 2^n matrix; qubit q = bit q of the index."""
    N = 1 << n
    M = np.zeros((N, N))
    for x in range(N):
        for q in range(n):
            M[x ^ (1 << q), x] += 1.0
    return M


def dense_qaoa(n, f, gammas, betas):
    """prod_l exp(-i b_l sum X) exp(-i g_l diag f) |+> with scipy.linalg.expm."""
    HM = dense_x_sum(n)
    N = 1 << n
    st = np.full(N, 1 / math.sqrt(N), dtype=complex)
    for g, b in zip(gammas, betas):
        st = sl.expm(-1j * g * np.diag(f)) @ st
        st = sl.expm(-1j * b * HM) @ st
    return st


def parity_costs(n, terms):
    """Eq. 1 through the XOR/popcount reading: prod_{i in t} s_i =
    (-1)^{popcount(x & mask)}, evaluated with numpy's bitwise_count."""
    x = np.arange(1 << n, dtype=np.uint64)
    f = np.zeros(1 << n, dtype=object)
    for w, idx in terms:
        m = np.uint64(sum(1 << i for i in idx))
        par = np.bitwise_count(x & m) & 1
        f = f + np.where(par == 1, -1, 1).astype(object) * w
    return f


def labs_paper_reduced(n, x):
    """The paper's reduced LABS polynomial (Background), 1-based indices:
    2 sum_{i=1}^{n-3} s_i sum_{t=1}^{floor((n-i-1)/2)} sum_{k=t+1}^{n-i-t}
      s_{i+t} s_{i+k} s_{i+k+t}  +  sum_{i=1}^{n-2} s_i sum_{k=1}^{floor((n-i)/2)} s_{i+2k}."""
    s = [None] + [1 - 2 * ((x >> (i - 1)) & 1) for i in range(1, n + 1)]
    four = 0
    for i in range(1, n - 2):
        for t in range(1, (n - i - 1) // 2 + 1):
            for k in range(t + 1, n - i - t + 1):
                four += s[i] * s[i + t] * s[i + k] * s[i + k + t]
    two = 0
    for i in range(1, n - 1):
        for k in range(1, (n - i) // 2 + 1):
            two += s[i] * s[i + 2 * k]
    return 2 * four + two


def labs_by_correlate(n):
    """sum_k C_k^2 with C_k from numpy.correlate (a library autocorrelation)."""
    out = np.empty(1 << n, dtype=np.int64)
    for x in range(1 << n):
        s = np.array([1 - 2 * ((x >> i) & 1) for i in range(n)])
        c = np.correlate(s, s, mode="full")[n:]  # lags 1..n-1
        out[x] = int(np.sum(c * c))
    return out


def graph_cut(n, edges, w):
    """Cut weight of every x via bit disagreement (no spins)."""
    x = np.arange(1 << n, dtype=np.int64)
    cut = np.zeros(1 << n, dtype=np.float64)
    for (i, j), we in zip(edges, w):
        cut += we * (((x >> i) ^ (x >> j)) & 1)
    return cut


def p1_maxcut_closed_form(n, edges, gamma, beta):
    """p = 1 MaxCut energy for f = -cut (Wang, Hadfield, Jiang and Rieffel,
    PRA 97, 022304 (2018), edge formula with degrees and triangle counts,
    with gamma -> -gamma because the paper's cost is minus the cut)."""
    adj = [set() for _ in range(n)]
    for i, j in edges:
        adj[i].add(j)
        adj[j].add(i)
    E = 0.0
    for i, j in edges:
        du, dv = len(adj[i]), len(adj[j])
        lam = len(adj[i] & adj[j])
        cg, sg = math.cos(gamma), math.sin(gamma)
        term = (0.5 - 0.25 * math.sin(4 * beta) * sg * (cg ** (du - 1) + cg ** (dv - 1))
                - 0.25 * math.sin(2 * beta) ** 2 * cg ** (du + dv - 2 - 2 * lam)
                * (1 - math.cos(2 * gamma) ** lam))
        E -= term
    return E


# ------------------------------------------------------------------ costs

@pytest.mark.parametrize("n", range(3, 17))
def test_labs_all_equal_sequence(orc, n):
    # all spins equal: C_k = n - k, so f = sum_{k=1}^{n-1} k^2 = (n-1) n (2n-1) / 6
    want = (n - 1) * n * (2 * n - 1) // 6
    assert orc.labs_cost_at(n, 0) == want
    assert orc.labs_cost_at(n, (1 << n) - 1) == want


@pytest.mark.parametrize("n", [4, 5, 7, 8, 11])
def test_labs_equals_paper_reduced_form(orc, n):
    # sum_k C_k^2 = 2 * (paper's reduced polynomial) + n(n-1)/2
    f = orc.labs_costs(n)
    for x in range(1 << n):
        assert f[x] == 2 * labs_paper_reduced(n, x) + n * (n - 1) // 2


@pytest.mark.parametrize("n", [3, 6, 9, 10])
def test_labs_matches_library_autocorrelation(orc, n):
    np.testing.assert_array_equal(orc.labs_costs(n), labs_by_correlate(n))


@pytest.mark.parametrize("n", [5, 8, 12])
def test_labs_symmetries(orc, n):
    f = orc.labs_costs(n)
    x = np.arange(1 << n)
    full = (1 << n) - 1
    alt = sum(1 << i for i in range(1, n, 2))  # negate every other spin
    rev = np.array([int(format(v, f"0{n}b")[::-1], 2) for v in x])
    np.testing.assert_array_equal(f, f[x ^ full])
    np.testing.assert_array_equal(f, f[x ^ alt])
    np.testing.assert_array_equal(f, f[rev])


def test_labs_small_optima_by_hand(orc):
    # n = 3: C_2^2 = 1 always, C_1 = 0 iff s_0 = -s_2 -> min 1, 4 optima.
    # n = 4: C_3^2 = 1, C_1 odd (>= 1), C_2 even -> min 2 at C_1 = +-1,
    #        C_2 = 0, e.g. (+,+,+,-); 8 optima.
    f3 = orc.labs_costs(3)
    assert f3.min() == 1 and np.sum(f3 == 1) == 4
    f4 = orc.labs_costs(4)
    assert f4.min() == 2 and np.sum(f4 == 2) == 8
    assert orc.labs_cost_at(4, 0b1000) == 2  # spins (+,+,+,-)


def test_labs_optima_golden(orc):
    """f_min and the number of optimal sequences, stored by
    tests/golden/make_golden.py from the oracle's own exhaustive enumeration;
    the small-n entries are re-derived here through numpy.correlate."""
    with open(os.path.join(GOLDEN, "labs_optima.json")) as fh:
        g = json.load(fh)
    for n in range(3, 11):
        f = labs_by_correlate(n)
        assert g["optima"][str(n)] == [int(f.min()), int(np.sum(f == f.min()))]
    for n in range(3, 17):
        f = orc.labs_costs(n)
        assert g["optima"][str(n)] == [int(f.min()), int(np.sum(f == f.min()))]


def test_labs_range_matches_full(orc):
    f = orc.labs_costs(14)
    np.testing.assert_array_equal(orc.labs_costs_range(14, 1000, 5000), f[1000:5000])


@pytest.mark.parametrize("n,seed", [(6, 11), (9, 12), (12, 13)])
def test_integer_terms_match_parity_form(orc, n, seed):
    terms = I.random_terms(n, 40, seed, max_order=5, integer=True)
    f = orc.costs_terms_int(n, terms)
    np.testing.assert_array_equal(f, parity_costs(n, terms).astype(np.int64))


def test_constant_and_single_terms(orc):
    n = 5
    f = orc.costs_terms_int(n, [(7, ())])
    assert np.all(f == 7)
    f = orc.costs_terms_int(n, [(1, (2,))])  # s_2 = +1 when bit 2 is 0
    x = np.arange(32)
    np.testing.assert_array_equal(f, np.where((x >> 2) & 1, -1, 1))


@pytest.mark.parametrize("n,seed", [(7, 21), (10, 22)])
def test_real_terms_exact_sum(orc, n, seed):
    # dyadic weights: every partial float64 sum is exact, so the oracle must
    # equal the exact rational sum, and float32 costs are one RNE of it.
    terms = I.random_terms(n, 30, seed, max_order=3, integer=False)
    f = orc.costs_terms_real(n, terms)
    exact = parity_costs(n, [(Fraction(w), idx) for w, idx in terms])
    for x in range(0, 1 << n, 7):
        assert Fraction(f[x]) == exact[x]
        assert np.float32(f[x]) == np.float32(float(exact[x]))


@pytest.mark.parametrize("n,seed", [(6, 1), (8, 2), (10, 3)])
def test_maxcut_is_minus_cut(orc, n, seed):
    edges, w = I.maxcut_3reg(n, graph_seed=seed, weighted=True, weight_seed=seed + 10)
    f = orc.maxcut_costs(n, edges, w)
    np.testing.assert_array_equal(f, -graph_cut(n, edges, w))
    assert f[0] == 0.0 and f[(1 << n) - 1] == 0.0


def test_maxcut_small_graphs_by_hand(orc):
    tri = [(0, 1), (1, 2), (0, 2)]
    f = orc.maxcut_costs(3, tri, [1, 1, 1])
    assert f.min() == -2  # a triangle cuts at most 2 edges
    sq = [(0, 1), (1, 2), (2, 3), (3, 0)]
    f = orc.maxcut_costs(4, sq, [1, 1, 1, 1])
    assert f.min() == -4 and f[0b0101] == -4  # bipartite: all edges cut


def test_maxcut_equals_paper_polynomial(orc):
    # Background: f = sum_{E} 1/2 s_i s_j - |E|/2, as generic terms
    n = 8
    edges, _ = I.maxcut_3reg(n, graph_seed=5)
    terms = [(0.5, (int(i), int(j))) for i, j in edges] + [(-len(edges) / 2, ())]
    np.testing.assert_array_equal(orc.maxcut_costs(n, edges, np.ones(len(edges))),
                                  orc.costs_terms_real(n, terms))


# ------------------------------------------------------------- simulation

def test_init_plus_and_norm(orc):
    psi = orc.init_plus(7)
    assert np.allclose(psi, 1 / math.sqrt(128))


@pytest.mark.parametrize("n", [1, 2, 4, 6])
def test_su2_matches_dense_kron(orc, n):
    # Algorithm 1 for a generic SU(2) on every qubit d, vs kron(I, U, I).
    psi = I.random_state(n, 40 + n)
    a = complex(0.6, 0.3)
    b = complex(-0.2, 0.5)
    nrm = math.sqrt(abs(a) ** 2 + abs(b) ** 2)
    a, b = a / nrm, b / nrm
    U = np.array([[a, -b.conjugate()], [b, a.conjugate()]])
    for d in range(1, n + 1):
        # qubit d-1 is bit d-1: kron order puts the most significant bit first
        op = np.array([[1.0]])
        for q in reversed(range(n)):
            op = np.kron(op, U if q == d - 1 else np.eye(2))
        np.testing.assert_allclose(orc.apply_su2(n, psi, d, a, b), op @ psi, atol=1e-13)


@pytest.mark.parametrize("n", [3, 5, 7])
def test_mixer_matches_walsh_hadamard_identity(orc, n):
    # exp(-i b sum X) = H^n diag(exp(-i b (n - 2|y|))) H^n / 2^n  (Sec. 3.2)
    beta = 0.37
    N = 1 << n
    H = sl.hadamard(N)
    y = np.arange(N)
    wt = np.array([bin(v).count("1") for v in y])
    M = H @ np.diag(np.exp(-1j * beta * (n - 2 * wt))) @ H / N
    psi = I.random_state(n, 50 + n)
    np.testing.assert_allclose(orc.apply_mixer(n, psi, beta), M @ psi, atol=1e-13)


def test_phase_is_elementwise(orc):
    n = 5
    f = np.arange(32, dtype=float) - 7.5
    psi = I.random_state(n, 3)
    out = orc.apply_phase(n, psi, f, 0.9)
    np.testing.assert_allclose(out, psi * np.exp(-0.9j * f), atol=1e-14)


@pytest.mark.parametrize("n,p,seed", [(3, 1, 1), (5, 3, 2), (7, 2, 3)])
def test_simulate_matches_dense_expm(orc, n, p, seed):
    terms = I.random_terms(n, 12, seed, max_order=3, integer=True)
    f = orc.costs_terms_int(n, terms).astype(float)
    g = I.angles(p, seed + 100)
    b = I.angles(p, seed + 200)
    psi = orc.simulate(n, f, g, b)
    np.testing.assert_allclose(psi, dense_qaoa(n, f, g, b), atol=1e-12)
    E = orc.energy(n, psi, f)
    dense = dense_qaoa(n, f, g, b)
    assert abs(E - np.vdot(dense, f * dense).real) < 1e-11


@pytest.mark.parametrize("n,seed", [(8, 1), (10, 2), (12, 3), (14, 1)])
def test_p1_maxcut_closed_form(orc, n, seed):
    edges, w = I.maxcut_3reg(n, graph_seed=seed)
    f = orc.maxcut_costs(n, edges, w)
    for k in range(3):
        g = I.angles(1, 300 + k)[0]
        b = I.angles(1, 400 + k)[0]
        psi = orc.simulate(n, f, [g], [b])
        assert abs(orc.energy(n, psi, f) - p1_maxcut_closed_form(n, edges, g, b)) < 1e-11


def test_p1_closed_form_with_triangles(orc):
    # K4 has a triangle on every edge (lambda = 2), plus a pendant path
    n = 6
    edges = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3), (3, 4), (4, 5)]
    f = orc.maxcut_costs(n, edges, np.ones(len(edges)))
    psi = orc.simulate(n, f, [0.7], [0.3])
    assert abs(orc.energy(n, psi, f) - p1_maxcut_closed_form(n, edges, 0.7, 0.3)) < 1e-12


@pytest.mark.parametrize("n", [4, 9])
def test_trivial_angles_give_mean_and_argmin_fraction(orc, n):
    f = orc.labs_costs(n).astype(float)
    cnt = np.sum(f == f.min())
    for g, b in [([0.0], [0.0]), ([0.8, 1.3], [0.0, 0.0]), ([0.0, 0.0], [0.4, 2.0])]:
        psi = orc.simulate(n, f, g, b)
        assert abs(orc.energy(n, psi, f) - f.mean()) < 1e-10 * abs(f.mean())
        assert abs(orc.overlap(n, psi, f) - cnt / 2 ** n) < 1e-13


def test_norm_preserved_many_layers(orc):
    n = 10
    f = orc.labs_costs(n).astype(float)
    psi = orc.simulate(n, f, I.angles(20, 7), I.angles(20, 8))
    assert abs(np.vdot(psi, psi).real - 1) < 1e-12


def test_energy_and_overlap_definitions(orc):
    n = 6
    psi = I.random_state(n, 9)
    f = np.arange(64, dtype=float) % 5
    assert abs(orc.energy(n, psi, f) - float(np.sum(np.abs(psi) ** 2 * f))) < 1e-14
    assert abs(orc.overlap(n, psi, f) - float(np.sum(np.abs(psi[f == 0]) ** 2))) < 1e-15


# --------------------------------------------------------------- gradient

@pytest.mark.parametrize("n,p,seed", [(4, 1, 1), (6, 3, 2), (8, 4, 3)])
def test_grad_matches_central_differences(orc, n, p, seed):
    f = orc.labs_costs(n).astype(float) if seed % 2 else \
        orc.maxcut_costs(n, *I.maxcut_3reg(n, graph_seed=seed, weighted=True))
    g = I.angles(p, seed + 10, 0, 0.3)
    b = I.angles(p, seed + 20)
    E, dg, db = orc.grad(n, f, g, b)

    def obj(gg, bb):
        return orc.energy(n, orc.simulate(n, f, gg, bb), f)

    assert abs(E - obj(g, b)) < 1e-12 * max(1, abs(E))
    fmax = float(np.max(np.abs(f)))

    def richardson(fun, h):
        d1 = (fun(h) - fun(-h)) / (2 * h)
        d2 = (fun(h / 2) - fun(-h / 2)) / h
        return (4 * d2 - d1) / 3

    gscale = max(1.0, float(np.max(np.abs(dg))), float(np.max(np.abs(db))))
    for l in range(p):
        e = np.zeros(p)
        e[l] = 1.0
        fd_g = richardson(lambda t: obj(g + t * e, b), 1e-2 / fmax)
        fd_b = richardson(lambda t: obj(g, b + t * e), 1e-3)
        assert abs(dg[l] - fd_g) < 1e-7 * gscale
        assert abs(db[l] - fd_b) < 1e-7 * gscale


def test_grad_matches_p1_closed_form_derivative(orc):
    n = 10
    edges, w = I.maxcut_3reg(n, graph_seed=4)
    f = orc.maxcut_costs(n, edges, w)
    g, b = 0.41, 0.27
    E, dg, db = orc.grad(n, f, [g], [b])
    h = 1e-6
    cg = (p1_maxcut_closed_form(n, edges, g + h, b) - p1_maxcut_closed_form(n, edges, g - h, b)) / (2 * h)
    cb = (p1_maxcut_closed_form(n, edges, g, b + h) - p1_maxcut_closed_form(n, edges, g, b - h)) / (2 * h)
    assert abs(dg[0] - cg) < 1e-7 and abs(db[0] - cb) < 1e-7


def test_uncompute_recovers_plus(orc):
    # un-applying every layer in reverse order returns |+> (adjoint sanity)
    n = 9
    f = orc.labs_costs(n).astype(float)
    g = I.angles(6, 1)
    b = I.angles(6, 2)
    psi = orc.simulate(n, f, g, b)
    for l in reversed(range(6)):
        psi = orc.apply_mixer(n, psi, -b[l])
        psi = orc.apply_phase(n, psi, f, -g[l])
    np.testing.assert_allclose(psi, orc.init_plus(n), atol=1e-13)


@pytest.mark.parametrize("n", range(2, 17))
def test_labs_costs_congruent_mod_4(orc, n):
    # C_k = sum_i s_i s_{i+k} has n - k terms of +-1, so C_k = n - k (mod 2);
    # an odd square is 1 mod 8 and an even one 0 mod 4, hence f = sum C_k^2 is
    # the number of k in 1..n-1 with n - k odd, mod 4, for every bitstring
    f = orc.labs_costs(n).astype(np.int64)
    odd = sum(1 for k in range(1, n) if (n - k) % 2)
    assert np.all(f % 4 == odd % 4)


# ------------------------------------------------------------- XY mixers

PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)


def dense_pauli_pair(n, i, j, P):
    """P_i P_j as a dense 2^n matrix (qubit q = bit q, kron puts bit n-1 first)."""
    op = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        op = np.kron(op, P if q in (i, j) else np.eye(2))
    return op


def dense_xy_term(n, i, j):
    return 0.5 * (dense_pauli_pair(n, i, j, PX) + dense_pauli_pair(n, i, j, PY))


def xy_edges(n, graph):
    if graph == 1:
        e = [(q, q + 1) for q in range(n - 1)]
        return e + [(n - 1, 0)] if n >= 3 else e
    return [(i, j) for i in range(n) for j in range(i + 1, n)]


def rand_state(n, seed):
    v = I.random_state(n, seed)
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("n,i,j", [(2, 0, 1), (3, 0, 2), (4, 3, 1), (4, 1, 2)])
def test_xy_gate_matches_dense_expm(orc, n, i, j):
    # the SU(4) gate is exp(-i beta (X_i X_j + Y_i Y_j) / 2), by brute force
    psi = rand_state(n, 7 + i + j)
    for beta in (0.37, -1.3, 2.9):
        want = sl.expm(-1j * beta * dense_xy_term(n, i, j)) @ psi
        np.testing.assert_allclose(orc.apply_xy(n, psi, i, j, beta), want, atol=1e-13)


@pytest.mark.parametrize("graph", [1, 2])
@pytest.mark.parametrize("n", [3, 4, 5])
def test_xy_mixer_is_the_ordered_product(orc, n, graph):
    # the mixer is the product of the edge gates, first edge applied first,
    # built here from dense matrix exponentials in the stated order
    beta = 0.61
    U = np.eye(1 << n, dtype=complex)
    for i, j in xy_edges(n, graph):
        U = sl.expm(-1j * beta * dense_xy_term(n, i, j)) @ U
    psi = rand_state(n, 30 + n)
    np.testing.assert_allclose(orc.apply_xy_mixer(n, psi, graph, beta), U @ psi, atol=1e-12)


def test_xy_single_edge_is_exact_exponential(orc):
    # n = 2: one edge, so the mixer is exp(-i beta M) exactly; on |01> it is
    # cos(b)|01> - i sin(b)|10>, and |00>, |11> are untouched
    beta = 0.83
    for graph in (1, 2):
        e01 = np.zeros(4, complex)
        e01[1] = 1.0
        out = orc.apply_xy_mixer(2, e01, graph, beta)
        np.testing.assert_allclose(out, [0, np.cos(beta), -1j * np.sin(beta), 0], atol=1e-15)
        for k in (0, 3):
            e = np.zeros(4, complex)
            e[k] = 1.0
            np.testing.assert_allclose(orc.apply_xy_mixer(2, e, graph, beta), e, atol=1e-15)


@pytest.mark.parametrize("graph", [1, 2])
def test_xy_preserves_hamming_weight_distribution(orc, graph):
    n = 7
    f = orc.labs_costs(n).astype(float)
    psi = rand_state(n, 41)
    w = np.array([bin(x).count("1") for x in range(1 << n)])
    out = orc.simulate_xy(n, f, [0.2, 0.05], [0.7, 1.9], psi, graph)
    for k in range(n + 1):
        assert abs(np.sum(np.abs(out[w == k]) ** 2) - np.sum(np.abs(psi[w == k]) ** 2)) < 1e-12


@pytest.mark.parametrize("graph", [1, 2])
def test_xy_product_is_second_order_close_to_exp_of_sum(orc, graph):
    # the ordered product agrees with exp(-i beta sum_edges term) up to
    # O(beta^2): halving beta divides the difference by about 4
    n = 5
    M = sum(dense_xy_term(n, i, j) for i, j in xy_edges(n, graph))
    psi = rand_state(n, 52)
    errs = []
    for beta in (2e-2, 1e-2):
        exact = sl.expm(-1j * beta * M) @ psi
        errs.append(np.linalg.norm(orc.apply_xy_mixer(n, psi, graph, beta) - exact))
    assert 3.5 < errs[0] / errs[1] < 4.5
    assert errs[1] < 1e-3


@pytest.mark.parametrize("n,k", [(1, 0), (4, 2), (6, 3), (7, 0), (7, 7)])
def test_dicke_state(orc, n, k):
    from math import comb
    psi = orc.dicke(n, k)
    w = np.array([bin(x).count("1") for x in range(1 << n)])
    assert np.all(psi[w != k] == 0)
    np.testing.assert_allclose(psi[w == k], 1 / np.sqrt(comb(n, k)), rtol=1e-15)


def test_simulate_xy_is_phase_then_mixer(orc):
    n = 5
    f = orc.labs_costs(n).astype(float)
    psi0 = orc.dicke(n, 2)
    g, b = [0.3, 0.11], [0.9, 0.4]
    want = psi0
    for gl, bl in zip(g, b):
        want = np.exp(-1j * gl * f) * want
        want = orc.apply_xy_mixer(n, want, 1, bl)
    np.testing.assert_allclose(orc.simulate_xy(n, f, g, b, psi0, 1), want, atol=1e-14)
