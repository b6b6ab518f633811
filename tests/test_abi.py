"""C-ABI checks that need no GPU: the library builds and loads, exports every
function include/qaoa.h declares, and its host-side logic (term generators,
argument validation, workspace sizing) behaves as documented."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2309_04841_gb300 import build as B
from paper_2309_04841_gb300 import inputs as I
from paper_2309_04841_gb300 import qaoa as Q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(qaoa_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    B.build()
    return Q.lib()


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert "qaoa_simulate" in names and "qaoa_grad" in names
    for name in names:
        assert hasattr(L, name), name


def test_no_oracle_in_product():
    # the product never loads or references the oracle
    for root, _, files in os.walk(os.path.join(ROOT, "paper_2309_04841_gb300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(root, f)).read()
                assert "oracle" not in txt.lower() or f == "inputs.py", f


def test_status_strings_and_version(L):
    assert L.qaoa_status_string(0) == b"ok"
    assert L.qaoa_status_string(1) == b"invalid argument"
    assert L.qaoa_version() >= 100


def test_workspace_bytes_monotone(L):
    prev = 0
    for n in range(1, 35):
        b = Q.workspace_bytes(n)
        assert b >= prev and b % 8 == 0
        prev = b
    assert Q.workspace_bytes(30) >= 512 + 3 * 8 * (1 << 19)


def _eval_terms(n, terms):
    x = np.arange(1 << n, dtype=np.uint64)
    f = np.zeros(1 << n)
    for w, m in terms:
        par = np.bitwise_count(x & np.uint64(m)) & 1
        f += np.where(par == 1, -w, w)
    return f


@pytest.mark.parametrize("n", [3, 4, 7, 10, 13])
def test_labs_terms_reproduce_oracle_labs(orc, n):
    t = Q.labs_terms(n)
    f = _eval_terms(n, [(float(a["weight"]), int(a["mask"])) for a in t])
    np.testing.assert_array_equal(f, orc.labs_costs(n).astype(float))


def test_labs_term_counts():
    # the paper counts about 75n terms at n = 31 (Related work): 2360 = 76.1 n
    t = Q.labs_terms(31)
    assert len(t) - 1 == 2360  # minus the constant
    w = t["weight"]
    order = np.array([bin(int(m)).count("1") for m in t["mask"]])
    assert set(np.unique(w[order == 4])) == {4.0}
    assert set(np.unique(w[order == 2])) == {2.0}
    assert w[order == 0][0] == 31 * 30 / 2


def test_maxcut_terms_match_oracle(orc):
    n = 10
    edges, w = I.maxcut_3reg(n, graph_seed=3, weighted=True, weight_seed=9)
    t = Q.maxcut_terms(n, edges, w)
    f = _eval_terms(n, [(float(a["weight"]), int(a["mask"])) for a in t])
    np.testing.assert_array_equal(f, orc.maxcut_costs(n, edges, w))


def test_validation_without_gpu(L):
    # argument errors are reported before any CUDA call
    P = C.c_void_p
    stats = Q.CostStats(0.0, 1.0, 1)
    g = np.zeros(2)
    st = L.qaoa_simulate(0, P(16), 0, C.byref(stats), Q._np_ptr(g), Q._np_ptr(g), 2, P(16), 0, 1,
                         P(256), 1 << 20, None, None)
    assert st == 1
    st = L.qaoa_simulate(20, P(16), 0, C.byref(stats), Q._np_ptr(g), Q._np_ptr(g), 0, P(16), 0, 1,
                         P(256), 1 << 30, None, None)
    assert st == 1  # p = 0
    bad = np.array([np.nan, 0.0])
    st = L.qaoa_simulate(20, P(16), 0, C.byref(stats), Q._np_ptr(bad), Q._np_ptr(g), 2, P(16), 0,
                         1, P(256), 1 << 30, None, None)
    assert st == 1  # non-finite angle
    st = L.qaoa_simulate(20, P(16), 0, C.byref(stats), Q._np_ptr(g), Q._np_ptr(g), 2, P(16), 0, 1,
                         P(256), 16, None, None)
    assert st == 2  # workspace too small
    st = L.qaoa_simulate(20, P(17), 0, C.byref(stats), Q._np_ptr(g), Q._np_ptr(g), 2, P(16), 0, 1,
                         P(256), 1 << 30, None, None)
    assert st == 1  # misaligned costs
    assert b"aligned" in L.qaoa_last_error_message()


def test_precompute_validation_without_gpu(L):
    t = Q.terms_array([(1.5, (0, 1))])
    st = L.qaoa_precompute_costs(4, Q._np_ptr(t), 1, Q.COST_I32, C.c_void_p(16), None)
    assert st == 1  # non-integer weight for int32 costs
    t = Q.terms_array([(2.0 ** 31, (0,))])
    st = L.qaoa_precompute_costs(4, Q._np_ptr(t), 1, Q.COST_I32, C.c_void_p(16), None)
    assert st == 3  # overflow
    t = Q.terms_array([(1.0, (5,))])
    st = L.qaoa_precompute_costs(4, Q._np_ptr(t), 1, Q.COST_I32, C.c_void_p(16), None)
    assert st == 1  # index >= n
    e = np.array([[0, 0]], dtype=np.int32)
    st = L.qaoa_maxcut_costs(4, Q._np_ptr(e), None, 1, Q.COST_I32, C.c_void_p(16), None)
    assert st == 1  # self loop


def test_server_validation_without_gpu(L):
    cfg = Q.ServerConfig(0, 10, 10)  # max_inflight must be >= 1
    h = C.c_void_p()
    assert L.qaoa_server_create(C.byref(cfg), C.c_void_p(256), 1 << 30, C.byref(h)) == 1
    cfg = Q.ServerConfig(4, 10, 10)
    assert L.qaoa_server_create(C.byref(cfg), C.c_void_p(100), 1 << 30, C.byref(h)) == 1  # alignment
    assert L.qaoa_server_submit(None, None, None) == 1


def test_u16_validation_without_gpu(L):
    # uint16 costs: builders and conversion check their arguments before any launch
    P = C.c_void_p
    assert L.qaoa_labs_costs_u16(33, P(256), None) == 1  # n > 32
    assert L.qaoa_labs_costs_u16(10, P(258), None) == 1  # misaligned
    t = Q.terms_array([(1.0, (0,))])
    assert L.qaoa_precompute_costs(4, Q._np_ptr(t), 1, Q.COST_U16, P(256), None) == 1
    e = np.array([[0, 1]], dtype=np.int32)
    assert L.qaoa_maxcut_costs(4, Q._np_ptr(e), None, 1, Q.COST_U16, P(256), None) == 1
    neg = Q.CostStats(-3.0, 5.0, 1)
    assert L.qaoa_convert_costs(4, P(256), Q.COST_I32, C.byref(neg), P(512), Q.COST_U16, None) == 3
    big = Q.CostStats(0.0, 70000.0, 1)
    assert L.qaoa_convert_costs(4, P(256), Q.COST_I32, C.byref(big), P(512), Q.COST_U16, None) == 3
    ok = Q.CostStats(0.0, 5.0, 1)
    assert L.qaoa_convert_costs(4, P(256), Q.COST_F32, C.byref(ok), P(512), Q.COST_U16, None) == 1
    assert L.qaoa_convert_costs(4, P(256), Q.COST_I32, None, P(512), Q.COST_U16, None) == 1


def test_probabilities_validation_without_gpu(L):
    P = C.c_void_p
    assert L.qaoa_probabilities(0, P(256), Q.C64, P(512), None) == 1
    assert L.qaoa_probabilities(10, P(264), Q.C64, P(512), None) == 1  # misaligned state
    assert L.qaoa_probabilities(10, P(256), Q.C64, P(520), None) == 1  # misaligned output
    assert L.qaoa_probabilities(10, P(256), 7, None, None) == 1        # bad state type


def test_xy_validation_without_gpu(L):
    P = C.c_void_p
    stats = Q.CostStats(0.0, 1.0, 1)
    g = np.zeros(2)
    # bad graph, n < 2, NULL stats with d_out
    assert L.qaoa_simulate_xy(10, P(256), 0, C.byref(stats), Q._np_ptr(g), Q._np_ptr(g), 2, 3,
                              P(512), 0, P(1024), 1 << 30, None, None) == 1
    assert L.qaoa_simulate_xy(1, P(256), 0, C.byref(stats), Q._np_ptr(g), Q._np_ptr(g), 2, 1,
                              P(512), 0, P(1024), 1 << 30, None, None) == 1
    assert L.qaoa_simulate_xy(10, P(256), 0, None, Q._np_ptr(g), Q._np_ptr(g), 2, 1,
                              P(512), 0, P(1024), 1 << 30, P(2048), None) == 1
    assert L.qaoa_dicke_state(10, 11, P(256), 0, None) == 1
    assert L.qaoa_dicke_state(10, -1, P(256), 0, None) == 1
    assert L.qaoa_dicke_state(10, 3, P(260), 0, None) == 1


def test_workspace_entry_points_validate_without_gpu(L):
    # NULL or undersized workspaces are refused before any CUDA call
    P = C.c_void_p
    small = 511  # below the counters and small outputs every workspace starts with
    assert L.qaoa_workspace_check(None, 1 << 20, None) == 1
    assert L.qaoa_workspace_check(P(256), small, None) == 1
    assert L.qaoa_selftest_timeout(None, 1 << 20, None) == 1
    assert L.qaoa_selftest_timeout(P(256), small, None) == 1
