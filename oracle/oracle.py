"""ctypes wrapper around the plain C oracle (test infrastructure only).

All arrays are numpy: costs as int64 (integer costs) or float64, states as
complex128.  Term lists are ``[(weight, (i, j, ...)), ...]`` with 0-based
variable indices, as in the paper's terms argument (Sec. 4).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None
_lib_omp = None


def lib():
    global _lib
    if _lib is None:
        _lib = _load(_build.build())
    return _lib


def lib_omp():
    """The OpenMP build of the same source (bit-identical results; used only
    for the benchmark's all-core CPU timing)."""
    global _lib_omp
    if _lib_omp is None:
        _lib_omp = _load(_build.build_omp())
    return _lib_omp


def _load(path):
    if True:
        L = C.CDLL(path)
        P = C.c_void_p
        L.oracle_costs_terms_i64.argtypes = [C.c_int, C.c_int, P, P, P, P]
        L.oracle_costs_terms_f64.argtypes = [C.c_int, C.c_int, P, P, P, P]
        L.oracle_labs_cost_at.argtypes = [C.c_int, C.c_uint64]
        L.oracle_labs_cost_at.restype = C.c_int64
        L.oracle_labs_costs.argtypes = [C.c_int, P]
        L.oracle_labs_costs_range.argtypes = [C.c_int, C.c_uint64, C.c_uint64, P]
        L.oracle_maxcut_costs.argtypes = [C.c_int, C.c_int, P, P, P]
        L.oracle_init_plus.argtypes = [C.c_int, P]
        L.oracle_apply_phase.argtypes = [C.c_int, P, P, C.c_double]
        L.oracle_apply_su2.argtypes = [C.c_int, P, C.c_int, C.c_double,
                                       C.c_double, C.c_double, C.c_double]
        L.oracle_apply_mixer.argtypes = [C.c_int, P, C.c_double]
        L.oracle_simulate.argtypes = [C.c_int, P, C.c_int, P, P, P, C.c_int]
        L.oracle_energy.argtypes = [C.c_int, P, P]
        L.oracle_energy.restype = C.c_double
        L.oracle_overlap.argtypes = [C.c_int, P, P]
        L.oracle_overlap.restype = C.c_double
        L.oracle_grad.argtypes = [C.c_int, P, C.c_int, P, P, P, P, P]
        L.oracle_apply_xy.argtypes = [C.c_int, P, C.c_int, C.c_int, C.c_double]
        L.oracle_apply_xy_mixer.argtypes = [C.c_int, P, C.c_int, C.c_double]
        L.oracle_simulate_xy.argtypes = [C.c_int, P, C.c_int, P, P, P, C.c_int]
        L.oracle_dicke.argtypes = [C.c_int, C.c_int, P]
        L.oracle_grad.restype = C.c_int
        return L


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _csr(terms):
    tptr = [0]
    tidx = []
    for _, idx in terms:
        tidx.extend(int(i) for i in idx)
        tptr.append(len(tidx))
    return (np.asarray(tptr, dtype=np.int32),
            np.asarray(tidx if tidx else [0], dtype=np.int32))


def costs_terms_int(n, terms):
    """Eq. 1 with integer weights, exact in int64."""
    w = np.asarray([int(t[0]) for t in terms], dtype=np.int64)
    tptr, tidx = _csr(terms)
    f = np.empty(1 << n, dtype=np.int64)
    lib().oracle_costs_terms_i64(n, len(terms), _p(w), _p(tptr), _p(tidx), _p(f))
    return f


def costs_terms_real(n, terms):
    """Eq. 1 with real weights, float64 accumulation in term order."""
    w = np.asarray([float(t[0]) for t in terms], dtype=np.float64)
    tptr, tidx = _csr(terms)
    f = np.empty(1 << n, dtype=np.float64)
    lib().oracle_costs_terms_f64(n, len(terms), _p(w), _p(tptr), _p(tidx), _p(f))
    return f


def labs_costs(n):
    f = np.empty(1 << n, dtype=np.int64)
    lib().oracle_labs_costs(n, _p(f))
    return f


def labs_cost_at(n, x):
    return int(lib().oracle_labs_cost_at(n, int(x)))


def labs_costs_range(n, x0, x1):
    f = np.empty(x1 - x0, dtype=np.int64)
    lib().oracle_labs_costs_range(n, x0, x1, _p(f))
    return f


def maxcut_costs(n, edges, weights):
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    f = np.empty(1 << n, dtype=np.float64)
    lib().oracle_maxcut_costs(n, len(w), _p(e), _p(w), _p(f))
    return f


def init_plus(n):
    psi = np.empty(1 << n, dtype=np.complex128)
    lib().oracle_init_plus(n, _p(psi))
    return psi


def apply_phase(n, psi, f, gamma):
    psi = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    f = np.ascontiguousarray(f, dtype=np.float64)
    lib().oracle_apply_phase(n, _p(psi), _p(f), float(gamma))
    return psi


def apply_su2(n, psi, d, a, b):
    psi = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    a, b = complex(a), complex(b)
    lib().oracle_apply_su2(n, _p(psi), int(d), a.real, a.imag, b.real, b.imag)
    return psi


def apply_mixer(n, psi, beta):
    psi = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    lib().oracle_apply_mixer(n, _p(psi), float(beta))
    return psi


def simulate(n, f, gammas, betas, psi0=None):
    """Algorithm 3 from |+> (or from psi0 if given); returns complex128."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(gammas, dtype=np.float64)
    b = np.ascontiguousarray(betas, dtype=np.float64)
    assert len(g) == len(b)
    if psi0 is None:
        psi = np.empty(1 << n, dtype=np.complex128)
        init = 1
    else:
        psi = np.ascontiguousarray(psi0, dtype=np.complex128).copy()
        init = 0
    lib().oracle_simulate(n, _p(f), len(g), _p(g), _p(b), _p(psi), init)
    return psi


XY_RING, XY_COMPLETE = 1, 2


def apply_xy(n, psi, i, j, beta):
    psi = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    lib().oracle_apply_xy(n, _p(psi), int(i), int(j), float(beta))
    return psi


def apply_xy_mixer(n, psi, graph, beta):
    psi = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    lib().oracle_apply_xy_mixer(n, _p(psi), int(graph), float(beta))
    return psi


def simulate_xy(n, f, gammas, betas, psi0, graph):
    """Algorithm 3 with the XY mixer of `graph` from psi0; complex128."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(gammas, dtype=np.float64)
    b = np.ascontiguousarray(betas, dtype=np.float64)
    assert len(g) == len(b)
    psi = np.ascontiguousarray(psi0, dtype=np.complex128).copy()
    lib().oracle_simulate_xy(n, _p(f), len(g), _p(g), _p(b), _p(psi), int(graph))
    return psi


def dicke(n, k):
    psi = np.empty(1 << n, dtype=np.complex128)
    lib().oracle_dicke(n, k, _p(psi))
    return psi


def energy(n, psi, f):
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    f = np.ascontiguousarray(f, dtype=np.float64)
    return float(lib().oracle_energy(n, _p(psi), _p(f)))


def overlap(n, psi, f):
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    f = np.ascontiguousarray(f, dtype=np.float64)
    return float(lib().oracle_overlap(n, _p(psi), _p(f)))


def grad(n, f, gammas, betas, library=None):
    """Returns (E, dE/dgamma[p], dE/dbeta[p]) by reverse mode with stored states.
    `library` (default lib()) may be lib_omp() for all-core timing."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(gammas, dtype=np.float64)
    b = np.ascontiguousarray(betas, dtype=np.float64)
    p = len(g)
    e = np.zeros(1, dtype=np.float64)
    dg = np.zeros(p, dtype=np.float64)
    db = np.zeros(p, dtype=np.float64)
    rc = (library or lib()).oracle_grad(n, _p(f), p, _p(g), _p(b), _p(e), _p(dg), _p(db))
    if rc != 0:
        raise MemoryError("oracle_grad: allocation failed")
    return float(e[0]), dg, db


def to_f32_rne(f64):
    """Single round-to-nearest-even of float64 costs to float32."""
    return np.asarray(f64, dtype=np.float64).astype(np.float32)


def to_i32_checked(i64):
    a = np.asarray(i64, dtype=np.int64)
    if a.size and (a.max() > np.iinfo(np.int32).max or a.min() < np.iinfo(np.int32).min):
        raise OverflowError("cost does not fit int32")
    return a.astype(np.int32)


__all__ = [k for k in list(globals()) if not k.startswith("_") and k not in ("C", "np", "os")]
