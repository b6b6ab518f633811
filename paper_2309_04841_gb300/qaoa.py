"""Thin Python binding of libqaoa.so (include/qaoa.h), same names as the C ABI.

Argument marshalling only: torch tensors provide device memory and the
current CUDA stream, every step of the computation runs in the library's
kernels.  There is no CPU fallback: if the library cannot be loaded the call
raises.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqaoa.so")

COST_I32, COST_F32, COST_F64, COST_U16 = 0, 1, 2, 3
C64, C128 = 0, 1

TERM_DTYPE = np.dtype([("weight", np.float64), ("mask", np.uint64)])

_STATUS = {0: "ok", 1: "invalid argument", 2: "buffer too small", 3: "integer cost overflow",
           4: "CUDA error", 5: "timeout", 6: "rejected", 7: "cancelled", 8: "not found",
           9: "busy"}


class QAOAError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class ProfEntry(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_uint64), ("ms", C.c_double),
                ("bytes", C.c_double)]


class ServerConfig(C.Structure):
    _fields_ = [("max_inflight", C.c_int), ("max_queue", C.c_int), ("small_batch", C.c_int)]


class Request(C.Structure):
    _fields_ = [("problem", C.c_int), ("n", C.c_int), ("p", C.c_int), ("edges", C.c_void_p),
                ("weights", C.c_void_p), ("m", C.c_size_t), ("problem_key", C.c_uint64),
                ("gammas", C.c_void_p), ("betas", C.c_void_p), ("want_grad", C.c_int)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("energy", C.c_double), ("overlap", C.c_double),
                ("submit_s", C.c_double), ("admit_s", C.c_double), ("finish_s", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("rejected", C.c_uint64),
                ("cancelled", C.c_uint64), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("evals_per_s", C.c_double), ("arena_bytes", C.c_size_t),
                ("arena_peak_bytes", C.c_size_t), ("cached_cost_vectors", C.c_size_t)]


PROBLEM_LABS, PROBLEM_MAXCUT = 0, 1


class CostStats(C.Structure):
    _fields_ = [("f_min", C.c_double), ("f_max", C.c_double), ("n_min", C.c_uint64),
                ("step_log2", C.c_uint32), ("reserved", C.c_uint32)]

    def __repr__(self):
        return (f"CostStats(f_min={self.f_min}, f_max={self.f_max}, n_min={self.n_min}, "
                f"step_log2={self.step_log2})")


_lib = None


def lib():
    """Load libqaoa.so (building it first if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            from . import build as _build
            _build.build()
        L = C.CDLL(LIB_PATH)
        P, I, Z, D = C.c_void_p, C.c_int, C.c_size_t, C.c_double
        sig = {
            "qaoa_status_string": ([I], C.c_char_p),
            "qaoa_last_error_message": ([], C.c_char_p),
            "qaoa_version": ([], I),
            "qaoa_workspace_bytes": ([I], Z),
            "qaoa_labs_terms": ([I, P, Z, P], I),
            "qaoa_maxcut_terms": ([I, P, P, Z, P, Z, P], I),
            "qaoa_precompute_costs": ([I, P, Z, I, P, P], I),
            "qaoa_labs_costs": ([I, P, P], I),
            "qaoa_labs_costs_u16": ([I, P, P], I),
            "qaoa_convert_costs": ([I, P, I, P, P, I, P], I),
            "qaoa_maxcut_costs": ([I, P, P, Z, I, P, P], I),
            "qaoa_cost_stats_compute": ([I, P, I, P, Z, P, P], I),
            "qaoa_simulate": ([I, P, I, P, P, P, I, P, I, I, P, Z, P, P], I),
            "qaoa_expectation": ([I, P, I, P, I, P, Z, P, P], I),
            "qaoa_probabilities": ([I, P, I, P, P], I),
            "qaoa_simulate_xy": ([I, P, I, P, P, P, I, I, P, I, P, Z, P, P], I),
            "qaoa_dicke_state": ([I, I, P, I, P], I),
            "qaoa_overlap": ([I, P, I, P, I, P, P, Z, P, P], I),
            "qaoa_grad": ([I, P, I, P, P, P, I, P, P, I, P, Z, P, P], I),
            "qaoa_workspace_check": ([P, Z, P], I),
            "qaoa_selftest_timeout": ([P, Z, P], I),
            "qaoa_simulate_noalloc": ([I, P, I, P, P, P, I, P, I, I, P, P], I),
            "qaoa_server_create": ([P, P, Z, P], I),
            "qaoa_server_submit": ([P, P, P], I),
            "qaoa_server_wait": ([P, C.c_uint64, P, P, P, I], I),
            "qaoa_server_cancel": ([P, C.c_uint64], I),
            "qaoa_server_stats": ([P, P], I),
            "qaoa_server_destroy": ([P], I),
            "qaoa_profile_enable": ([I], I),
            "qaoa_profile_read": ([P, I, P, I], I),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(st):
    if st != 0:
        raise QAOAError(st, lib().qaoa_last_error_message().decode())


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _np_ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def cost_dtype(ct):
    """torch dtype holding a cost vector of type ct (uint16 costs live in an
    int16 tensor; the library reads its bits as unsigned)."""
    torch = _torch()
    return {COST_I32: torch.int32, COST_F32: torch.float32, COST_F64: torch.float64,
            COST_U16: torch.int16}[ct]


def state_dtype(st):
    torch = _torch()
    return {C64: torch.complex64, C128: torch.complex128}[st]


def cost_type_of(costs):
    torch = _torch()
    m = {torch.int32: COST_I32, torch.float32: COST_F32, torch.float64: COST_F64,
         torch.int16: COST_U16}
    if hasattr(torch, "uint16"):
        m[torch.uint16] = COST_U16
    return m[costs.dtype]


def state_type_of(state):
    torch = _torch()
    return {torch.complex64: C64, torch.complex128: C128}[state.dtype]


def _n_of(t):
    n = int(t.numel()).bit_length() - 1
    if t.numel() != 1 << n:
        raise ValueError("vector length must be a power of two")
    return n


# ----------------------------------------------------------- host helpers

def terms_array(terms):
    """[(w, (i, j, ...)), ...] -> qaoa_term array (weight, bit mask)."""
    a = np.zeros(len(terms), dtype=TERM_DTYPE)
    for k, (w, idx) in enumerate(terms):
        a[k]["weight"] = float(w)
        a[k]["mask"] = np.uint64(sum(1 << int(i) for i in idx))
    return a


def labs_terms(n):
    L = lib()
    cnt = C.c_size_t(0)
    st = L.qaoa_labs_terms(n, None, 0, C.byref(cnt))
    if st not in (0, 2):
        _check(st)
    out = np.zeros(cnt.value, dtype=TERM_DTYPE)
    _check(L.qaoa_labs_terms(n, _np_ptr(out), len(out), C.byref(cnt)))
    return out


def maxcut_terms(n, edges, weights=None):
    L = lib()
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    w = None if weights is None else np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    out = np.zeros(len(e) + 1, dtype=TERM_DTYPE)
    cnt = C.c_size_t(0)
    _check(L.qaoa_maxcut_terms(n, _np_ptr(e), None if w is None else _np_ptr(w), len(e),
                               _np_ptr(out), len(out), C.byref(cnt)))
    return out


# ------------------------------------------------------------ cost vector

def workspace_bytes(n):
    return int(lib().qaoa_workspace_bytes(n))


def workspace(n, device="cuda"):
    torch = _torch()
    return torch.empty(workspace_bytes(n), dtype=torch.uint8, device=device)


def workspace_check(work):
    """Raises QAOAError(timeout) if a kernel that used `work` gave up on a
    bounded device-side wait; synchronises the current stream.  work=None
    checks the library's built-in scratch (the one simulate_noalloc uses)."""
    if work is None:
        _check(lib().qaoa_workspace_check(None, 0, _stream()))
    else:
        _check(lib().qaoa_workspace_check(_ptr(work), work.numel(), _stream()))


def selftest_timeout(work):
    """Enqueues one kernel whose bounded device-side wait nothing completes:
    the next workspace_check(work) raises QAOAError(timeout) (about 1 s).
    work=None targets the built-in scratch."""
    if work is None:
        _check(lib().qaoa_selftest_timeout(None, 0, _stream()))
    else:
        _check(lib().qaoa_selftest_timeout(_ptr(work), work.numel(), _stream()))


def precompute_costs(n, terms, cost_type=COST_I32, out=None):
    torch = _torch()
    t = terms if isinstance(terms, np.ndarray) and terms.dtype == TERM_DTYPE else terms_array(terms)
    t = np.ascontiguousarray(t)
    if out is None:
        out = torch.empty(1 << n, dtype=cost_dtype(cost_type), device="cuda")
    _check(lib().qaoa_precompute_costs(n, _np_ptr(t) if len(t) else None, len(t), cost_type,
                                       _ptr(out), _stream()))
    return out


def labs_costs(n, out=None):
    torch = _torch()
    if out is None:
        out = torch.empty(1 << n, dtype=torch.int32, device="cuda")
    _check(lib().qaoa_labs_costs(n, _ptr(out), _stream()))
    return out


def labs_costs_u16(n, out=None):
    """LABS costs as uint16 (in an int16 tensor; see cost_dtype)."""
    torch = _torch()
    if out is None:
        out = torch.empty(1 << n, dtype=torch.int16, device="cuda")
    _check(lib().qaoa_labs_costs_u16(n, _ptr(out), _stream()))
    return out


def convert_costs(costs, stats, cost_type=COST_U16, out=None):
    """int32 <-> uint16 copy of a cost vector (stats: those of `costs`)."""
    torch = _torch()
    n = _n_of(costs)
    if out is None:
        out = torch.empty(1 << n, dtype=cost_dtype(cost_type), device=costs.device)
    _check(lib().qaoa_convert_costs(n, _ptr(costs), cost_type_of(costs), C.byref(stats), _ptr(out),
                                    cost_type, _stream()))
    return out


def maxcut_costs(n, edges, weights=None, cost_type=COST_I32, out=None):
    torch = _torch()
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    w = None if weights is None else np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    if out is None:
        out = torch.empty(1 << n, dtype=cost_dtype(cost_type), device="cuda")
    _check(lib().qaoa_maxcut_costs(n, _np_ptr(e), None if w is None else _np_ptr(w), len(e),
                                   cost_type, _ptr(out), _stream()))
    return out


def cost_stats_compute(costs, work=None):
    n = _n_of(costs)
    if work is None:
        work = workspace(n)
    st = CostStats()
    _check(lib().qaoa_cost_stats_compute(n, _ptr(costs), cost_type_of(costs), _ptr(work),
                                         work.numel(), C.byref(st), _stream()))
    return st


# ------------------------------------------------------------- simulation

def _angles(gammas, betas):
    g = np.ascontiguousarray(np.asarray(gammas, dtype=np.float64).reshape(-1))
    b = np.ascontiguousarray(np.asarray(betas, dtype=np.float64).reshape(-1))
    if len(g) != len(b):
        raise ValueError("gammas and betas must have the same length")
    return g, b


def simulate(costs, stats, gammas, betas, state=None, state_type=C64, init_plus=True,
             work=None, out=None, reduce=True):
    """Algorithm 3 on the device.  Returns (state, out) where out holds
    [E, O] (device float64) when reduce is True, else None."""
    torch = _torch()
    n = _n_of(costs)
    g, b = _angles(gammas, betas)
    if state is None:
        state = torch.empty(1 << n, dtype=state_dtype(state_type), device="cuda")
        init_plus = True
    if work is None:
        work = workspace(n)
    if reduce and out is None:
        out = torch.empty(2, dtype=torch.float64, device="cuda")
    _check(lib().qaoa_simulate(n, _ptr(costs), cost_type_of(costs), C.byref(stats), _np_ptr(g),
                               _np_ptr(b), len(g), _ptr(state), state_type_of(state),
                               1 if init_plus else 0, _ptr(work), work.numel(),
                               _ptr(out) if reduce else None, _stream()))
    return state, (out if reduce else None)


def simulate_noalloc(costs, stats, gammas, betas, state=None, state_type=C64, init_plus=True,
                     out=None):
    """qaoa_simulate_noalloc: as simulate() with the library's built-in
    scratch instead of a workspace (n <= 23).  Returns (state, out)."""
    torch = _torch()
    n = _n_of(costs)
    g, b = _angles(gammas, betas)
    if state is None:
        state = torch.empty(1 << n, dtype=state_dtype(state_type), device="cuda")
        init_plus = True
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device="cuda")
    _check(lib().qaoa_simulate_noalloc(n, _ptr(costs), cost_type_of(costs), C.byref(stats),
                                       _np_ptr(g), _np_ptr(b), len(g), _ptr(state),
                                       state_type_of(state), 1 if init_plus else 0, _ptr(out),
                                       _stream()))
    return state, out


XY_RING, XY_COMPLETE = 1, 2


def dicke_state(n, k, state_type=C64, out=None):
    """|D^n_k> on the device."""
    torch = _torch()
    if out is None:
        out = torch.empty(1 << n, dtype=state_dtype(state_type), device="cuda")
    _check(lib().qaoa_dicke_state(n, k, _ptr(out), state_type_of(out), _stream()))
    return out


def simulate_xy(costs, stats, gammas, betas, state, graph=XY_RING, work=None, out=None,
                reduce=True):
    """Algorithm 3 with the XY mixer (ring or complete graph) on `state`
    (updated in place).  Returns (state, out), out = [E, O] when reduce."""
    torch = _torch()
    n = _n_of(costs)
    g, b = _angles(gammas, betas)
    if work is None:
        work = workspace(n)
    if reduce and out is None:
        out = torch.empty(2, dtype=torch.float64, device="cuda")
    _check(lib().qaoa_simulate_xy(n, _ptr(costs), cost_type_of(costs), C.byref(stats), _np_ptr(g),
                                  _np_ptr(b), len(g), graph, _ptr(state), state_type_of(state),
                                  _ptr(work), work.numel(), _ptr(out) if reduce else None,
                                  _stream()))
    return state, (out if reduce else None)


def probabilities(state, preserve_state=True, out=None):
    """|psi_x|^2 (Sec. 4 get_probabilities).  preserve_state=True writes a
    new real tensor (float32 for complex64, float64 for complex128); False
    squares in place and returns the real view of `state` (each amplitude
    becomes |psi_x|^2 + 0i)."""
    torch = _torch()
    n = _n_of(state)
    if preserve_state:
        if out is None:
            rd = torch.float32 if state.dtype == torch.complex64 else torch.float64
            out = torch.empty(1 << n, dtype=rd, device=state.device)
        _check(lib().qaoa_probabilities(n, _ptr(state), state_type_of(state), _ptr(out), _stream()))
        return out
    _check(lib().qaoa_probabilities(n, _ptr(state), state_type_of(state), None, _stream()))
    return state.real


def optimize(costs, stats, gammas, betas, steps=100, lr=0.02, betas_adam=(0.9, 0.999),
             eps=1e-8, state_type=C64):
    """The optimizer loop of Fig. 1: Adam on the QAOA objective with the
    gradient of every step from qaoa_grad (forward + adjoint sweep on the
    device); the loop itself runs on the host.  Returns (gammas, betas,
    history) with history[k] = E at the angles of step k; the last entry is
    the energy at the returned angles."""
    import numpy as np
    torch = _torch()
    x = np.concatenate([np.asarray(gammas, np.float64), np.asarray(betas, np.float64)])
    p = len(gammas)
    m = np.zeros_like(x)
    v = np.zeros_like(x)
    n = _n_of(costs)
    state = torch.empty(1 << n, dtype=state_dtype(state_type), device="cuda")
    lam = torch.empty_like(state)
    work = workspace(n)
    out = torch.empty(2 + 2 * p, dtype=torch.float64, device="cuda")
    hist = []
    b1, b2 = betas_adam
    for t in range(1, steps + 1):
        grad(costs, stats, x[:p], x[p:], state=state, lam=lam, state_type=state_type, work=work,
             out=out)
        r = out.cpu().numpy()
        hist.append(float(r[0]))
        gr = r[2:]
        m = b1 * m + (1 - b1) * gr
        v = b2 * v + (1 - b2) * gr * gr
        x = x - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    _, o = simulate(costs, stats, x[:p], x[p:], state=state, state_type=state_type, work=work)
    hist.append(float(o[0]))
    return x[:p].copy(), x[p:].copy(), hist


def expectation(state, costs, work=None, out=None):
    torch = _torch()
    n = _n_of(costs)
    if work is None:
        work = workspace(n)
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device="cuda")
    _check(lib().qaoa_expectation(n, _ptr(state), state_type_of(state), _ptr(costs),
                                  cost_type_of(costs), _ptr(work), work.numel(), _ptr(out),
                                  _stream()))
    return out


def overlap(state, costs, stats, work=None, out=None):
    torch = _torch()
    n = _n_of(costs)
    if work is None:
        work = workspace(n)
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device="cuda")
    _check(lib().qaoa_overlap(n, _ptr(state), state_type_of(state), _ptr(costs),
                              cost_type_of(costs), C.byref(stats), _ptr(work), work.numel(),
                              _ptr(out), _stream()))
    return out


def grad(costs, stats, gammas, betas, state=None, lam=None, state_type=C64, work=None, out=None):
    """Objective and adjoint gradient.  Returns the device float64 tensor
    [E, O, dE/dgamma_1..p, dE/dbeta_1..p]."""
    torch = _torch()
    n = _n_of(costs)
    g, b = _angles(gammas, betas)
    p = len(g)
    if state is None:
        state = torch.empty(1 << n, dtype=state_dtype(state_type), device="cuda")
    if lam is None:
        lam = torch.empty_like(state)
    if work is None:
        work = workspace(n)
    if out is None:
        out = torch.empty(2 + 2 * p, dtype=torch.float64, device="cuda")
    _check(lib().qaoa_grad(n, _ptr(costs), cost_type_of(costs), C.byref(stats), _np_ptr(g),
                           _np_ptr(b), p, _ptr(state), _ptr(lam), state_type_of(state),
                           _ptr(work), work.numel(), _ptr(out), _stream()))
    return out


class _EnergyFn:
    """Factory for the torch.autograd.Function (built lazily so importing this
    module does not import torch)."""
    fn = None


def qaoa_energy(costs, stats, gammas, betas, state_type=C64):
    """E(gammas, betas) as a differentiable torch scalar: forward and backward
    both run through qaoa_grad (one forward + one adjoint sweep)."""
    torch = _torch()
    if _EnergyFn.fn is None:
        class QAOAEnergy(torch.autograd.Function):
            @staticmethod
            def forward(ctx, g, b, costs, stats, st):
                out = grad(costs, stats, g.detach().cpu().numpy(), b.detach().cpu().numpy(),
                           state_type=st)
                p = g.numel()
                dg = out[2:2 + p].to(device=g.device, dtype=g.dtype)
                db = out[2 + p:].to(device=b.device, dtype=b.dtype)
                ctx.save_for_backward(dg.reshape(g.shape), db.reshape(b.shape))
                return out[0].to(device=g.device, dtype=g.dtype)

            @staticmethod
            def backward(ctx, gy):
                dg, db = ctx.saved_tensors
                return gy * dg, gy * db, None, None, None

        _EnergyFn.fn = QAOAEnergy
    return _EnergyFn.fn.apply(gammas, betas, costs, stats, state_type)


# -------------------------------------------------------------- profiling

def profile_enable(on=True):
    _check(lib().qaoa_profile_enable(1 if on else 0))


def profile_read(reset=True):
    """{kind: {"launches", "ms", "bytes"}} for the library's recorded launches."""
    buf = (ProfEntry * 64)()
    cnt = C.c_int(0)
    _check(lib().qaoa_profile_read(buf, 64, C.byref(cnt), 1 if reset else 0))
    return {buf[i].name.decode(): {"launches": int(buf[i].launches), "ms": float(buf[i].ms),
                                   "bytes": float(buf[i].bytes)} for i in range(min(cnt.value, 64))}


# ---------------------------------------------------------------- serving

class Server:
    """qaoa_server_*: continuous-batching objective / gradient server over a
    device arena (a torch uint8 tensor owned by this object)."""

    def __init__(self, arena_bytes, max_inflight=8, max_queue=1 << 20, small_batch=256):
        torch = _torch()
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device="cuda")
        cfg = ServerConfig(max_inflight, max_queue, small_batch)
        self._h = C.c_void_p()
        _check(lib().qaoa_server_create(C.byref(cfg), _ptr(self.arena), self.arena.numel(),
                                        C.byref(self._h)))

    def submit(self, problem, n, gammas, betas, edges=None, weights=None, key=0, want_grad=True):
        g, b = _angles(gammas, betas)
        e = None if edges is None else np.ascontiguousarray(np.asarray(edges, np.int32).reshape(-1, 2))
        w = None if weights is None else np.ascontiguousarray(np.asarray(weights, np.float64))
        req = Request(problem, n, len(g), None if e is None else _np_ptr(e).value,
                      None if w is None else _np_ptr(w).value, 0 if e is None else len(e), key,
                      _np_ptr(g).value, _np_ptr(b).value, 1 if want_grad else 0)
        t = C.c_uint64(0)
        _check(lib().qaoa_server_submit(self._h, C.byref(req), C.byref(t)))  # inputs are copied
        return t.value

    def wait(self, ticket, p, timeout_ms=-1):
        r = Result()
        dg = np.zeros(p)
        db = np.zeros(p)
        _check(lib().qaoa_server_wait(self._h, ticket, C.byref(r), _np_ptr(dg), _np_ptr(db),
                                      int(timeout_ms)))
        return {"status": r.status, "energy": r.energy, "overlap": r.overlap, "dgamma": dg,
                "dbeta": db, "submit_s": r.submit_s, "admit_s": r.admit_s, "finish_s": r.finish_s}

    def cancel(self, ticket):
        _check(lib().qaoa_server_cancel(self._h, ticket))

    def stats(self):
        st = ServerStats()
        _check(lib().qaoa_server_stats(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        """Destroy the server (it drains first) and drop the arena."""
        if self._h:
            lib().qaoa_server_destroy(self._h)
            self._h = C.c_void_p()
        self.arena = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
