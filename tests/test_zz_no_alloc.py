"""qaoa_simulate_noalloc: the simulate entry point for callers that cannot
allocate device memory (their host application owns all device allocations,
or their device-memory budget is fully committed).  Its scratch is a fixed
array inside the library, so it takes no workspace argument.

Checked through the C ABI against qaoa_simulate (the entry point with a
caller-provided workspace) on the same inputs, twice in a row so the second
call runs on the scratch contents the first one left behind.  Tolerances are
the forward tests' complex64 ones (the two entry points run the same kernels,
so in practice they agree bit for bit).  This file is collected last so a run
that stops at the first failure has already run every other test; it passes
alone in a fresh process as well as after the other tests."""
import ctypes as C

import numpy as np
import pytest

from paper_2309_04841_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_2309_04841_gb300 import qaoa
    qaoa.lib()
    return qaoa


@pytest.mark.parametrize("n,st", [(9, "c64"), (18, "c64"), (23, "c64"), (17, "c128")])
def test_noalloc_matches_simulate_twice(Q, n, st):
    import torch
    stype = Q.C64 if st == "c64" else Q.C128
    fd = Q.labs_costs(n)
    stats = Q.cost_stats_compute(fd)
    for call in range(2):
        g = I.angles(3, 40 + call, 0, 0.2)
        b = I.angles(3, 50 + call)
        ref_state, ref_out = Q.simulate(fd, stats, g, b, state_type=stype)
        state, out = Q.simulate_noalloc(fd, stats, g, b, state_type=stype)
        torch.cuda.synchronize()
        r, o = ref_out.cpu().numpy(), out.cpu().numpy()
        assert abs(o[0] - r[0]) <= 1e-5 * abs(r[0])
        assert abs(o[1] - r[1]) <= 1e-5 * r[1] + 1e-15
        a = state.cpu().numpy().astype(np.complex128)
        c = ref_state.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(a - c) <= 2e-5 * np.linalg.norm(c)


def test_noalloc_rejects_n_beyond_scratch(Q):
    import torch
    n = 24
    fd = torch.zeros(1 << n, dtype=torch.int32, device="cuda")
    stats = Q.CostStats(0.0, 0.0, 1 << n)
    state = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    g = np.zeros(1)
    st = Q.lib().qaoa_simulate_noalloc(n, Q._ptr(fd), Q.COST_I32, C.byref(stats), Q._np_ptr(g),
                                       Q._np_ptr(g), 1, Q._ptr(state), Q.C64, 1, Q._ptr(out),
                                       Q._stream())
    assert st == 2  # QAOA_ERR_OUT_OF_MEMORY
    assert b"n > 23" in Q.lib().qaoa_last_error_message()


def test_noalloc_allocates_no_device_memory(Q):
    # the entry point's promise: after a warm-up call (which may load the
    # library's device code), a call changes the free device memory by nothing
    import torch
    n = 23
    fd = Q.labs_costs(n)
    stats = Q.cost_stats_compute(fd)
    state = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    g, b = I.angles(2, 44, 0, 0.2), I.angles(2, 45)
    Q.simulate_noalloc(fd, stats, g, b, state=state, out=out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    Q.simulate_noalloc(fd, stats, g, b, state=state, out=out)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0


def test_noalloc_timeout_reported_once_through_builtin_scratch(Q):
    # a caller of the no-allocation entry point has no workspace pointer: it
    # checks the built-in scratch with workspace_check(None), which reports a
    # bounded wait that ran out exactly once
    n = 16
    fd = Q.labs_costs(n)
    stats = Q.cost_stats_compute(fd)
    g, b = I.angles(2, 46, 0, 0.2), I.angles(2, 47)
    Q.simulate_noalloc(fd, stats, g, b)
    Q.workspace_check(None)
    Q.selftest_timeout(None)
    with pytest.raises(Q.QAOAError) as e:
        Q.workspace_check(None)
    assert e.value.status == 5  # QAOA_ERR_TIMEOUT
    Q.workspace_check(None)  # cleared after one report
    _, out = Q.simulate_noalloc(fd, stats, g, b)
    _, ref = Q.simulate(fd, stats, g, b)
    o, r = out.cpu().numpy(), ref.cpu().numpy()
    assert abs(o[0] - r[0]) <= 1e-5 * abs(r[0])
    Q.workspace_check(None)
