"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.  This module holds no QAOA arithmetic: only random numbers, graphs,
angle vectors and random term lists.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw i of stream ``seed`` is ``mix64(seed * 2^32 + i + 1)`` after
adding the golden-ratio increment.  Being pure integer arithmetic on numpy
uint64 arrays, it gives identical inputs on every machine and numpy version.

Workload recipes follow the paper's experiments (Background and Sec. 5):
random 3-regular MaxCut graphs (pairing model), Erdos-Renyi G(n, 0.5) graphs
with fp32 uniform [0, 1) weights, and LABS (which needs no random input).
"""
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z):
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def u64(seed, count, offset=0):
    """``count`` 64-bit draws of stream ``seed`` starting at draw ``offset``."""
    i = np.arange(offset, offset + count, dtype=np.uint64)
    base = np.uint64((int(seed) & 0xFFFFFFFF) << 32)
    with np.errstate(over="ignore"):
        x = (base + i + np.uint64(1)) * _GOLDEN
    return _mix64(x)


def uniform(seed, count, lo=0.0, hi=1.0, offset=0):
    """float64 uniform in [lo, hi) with 53 random bits."""
    z = u64(seed, count, offset) >> np.uint64(11)
    return lo + (hi - lo) * (z.astype(np.float64) * (1.0 / 9007199254740992.0))


def randint(seed, count, m, offset=0):
    """Integers uniform in [0, m) (m < 2^32; bias below 2^-32)."""
    z = u64(seed, count, offset) >> np.uint64(32)
    return ((z * np.uint64(m)) >> np.uint64(32)).astype(np.int64)


def angles(p, seed, lo=0.0, hi=math.pi):
    """p angles uniform in [lo, hi)."""
    return uniform(seed, p, lo, hi)


def fp32_unit_weights(m, seed):
    """m weights uniform in [0, 1) exactly representable in float32: k * 2^-24
    with k uniform in [0, 2^24)."""
    k = randint(seed, m, 1 << 24)
    return (k.astype(np.float64) * 2.0 ** -24)


def _shuffle(a, seed, attempt):
    """Fisher-Yates shuffle driven by stream ``seed`` (sub-stream ``attempt``)."""
    a = list(a)
    r = randint(seed, len(a), 1 << 31, offset=attempt * (len(a) + 1))
    for i in range(len(a) - 1, 0, -1):
        j = int(r[i]) % (i + 1)
        a[i], a[j] = a[j], a[i]
    return a


def random_regular_graph(n, d, seed, max_attempts=100000):
    """Random d-regular simple graph on n vertices by the pairing (configuration)
    model with rejection of self-loops and repeated edges.  Returns an (m, 2)
    int32 array of edges (i < j), m = n*d/2, in a canonical sorted order."""
    if (n * d) % 2 or d >= n:
        raise ValueError("no d-regular simple graph with these n, d")
    points = [v for v in range(n) for _ in range(d)]
    for attempt in range(max_attempts):
        sh = _shuffle(points, seed, attempt)
        edges = set()
        ok = True
        for k in range(0, len(sh), 2):
            i, j = sh[k], sh[k + 1]
            if i == j:
                ok = False
                break
            e = (min(i, j), max(i, j))
            if e in edges:
                ok = False
                break
            edges.add(e)
        if ok:
            return np.asarray(sorted(edges), dtype=np.int32).reshape(-1, 2)
    raise RuntimeError("pairing model did not produce a simple graph")


def erdos_renyi(n, prob, seed):
    """G(n, prob): each of the n(n-1)/2 pairs (i < j, row-major) is an edge
    with probability prob.  Returns an (m, 2) int32 array."""
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    u = uniform(seed, len(pairs))
    edges = [pairs[k] for k in range(len(pairs)) if u[k] < prob]
    return np.asarray(edges, dtype=np.int32).reshape(-1, 2)


def random_terms(n, n_terms, seed, max_order=4, integer=True, wmax=5):
    """Random polynomial terms [(w, (i, ...)), ...] over n variables with
    orders 0..max_order (order 0 is the constant offset).  Integer weights in
    [-wmax, wmax] or float64 weights k * 2^-20, |k| < wmax * 2^20."""
    per = 2 + n
    r = randint(seed, n_terms * per, 1 << 30)
    terms = []
    for t in range(n_terms):
        base = t * per
        order = min(int(r[base]) % (max_order + 1), n)
        if integer:
            w = int(r[base + 1]) % (2 * wmax + 1) - wmax
        else:
            k = int(r[base + 1]) % (2 * wmax * (1 << 20)) - wmax * (1 << 20)
            w = k * 2.0 ** -20
        pool = list(range(n))  # partial Fisher-Yates: first `order` picks
        for i in range(order):
            j = i + int(r[base + 2 + i]) % (n - i)
            pool[i], pool[j] = pool[j], pool[i]
        terms.append((w, tuple(sorted(pool[:order]))))
    return terms


def random_state(n, seed):
    """Normalised complex128 state with Gaussian-like random amplitudes
    (sum of uniforms), for single-pass tests that must not start from |+>."""
    N = 1 << n
    u = uniform(seed, 4 * N).reshape(4, N)
    re = u[0] + u[1] - 1.0
    im = u[2] + u[3] - 1.0
    psi = re + 1j * im
    return psi / np.sqrt(np.vdot(psi, psi).real)


# ----------------------------------------------------------------- workloads
# Named recipes of the paper's workloads (seeds are part of the recipe).

def maxcut_3reg(n, graph_seed=1, weighted=False, weight_seed=4):
    edges = random_regular_graph(n, 3, graph_seed)
    if weighted:
        w = fp32_unit_weights(len(edges), weight_seed)
    else:
        w = np.ones(len(edges), dtype=np.float64)
    return edges, w


def maxcut_gnp(n, prob=0.5, graph_seed=3, weight_seed=4):
    edges = erdos_renyi(n, prob, graph_seed)
    return edges, fp32_unit_weights(len(edges), weight_seed)


# Named workloads.  gamma ~ U[0, ghi), beta ~ U[0, pi) from the given seeds.
WORKLOADS = {
    # MaxCut on a random 3-regular graph, unit weights, complex128
    "maxcut3_n14_p2": dict(problem="maxcut3", n=14, p=2, graph_seed=1,
                           weighted=False, gamma_seed=2, beta_seed=12,
                           ghi=math.pi, cost="i32", state="c128"),
    # weighted Erdos-Renyi G(26, 0.5), fp32 weights k * 2^-24
    "maxcut_gnp26_p6": dict(problem="gnp", n=26, p=6, graph_seed=3,
                            weight_seed=4, gamma_seed=5, beta_seed=15,
                            ghi=math.pi, cost="f32", state="c64"),
    # LABS n = 30, p = 10 (the objective + gradient headline workload)
    "labs30_p10": dict(problem="labs", n=30, p=10, gamma_seed=6,
                       beta_seed=16, ghi=math.pi, cost="i32", state="c64"),
    # same with small gammas, so the state is not scrambled by gamma * f
    "labs30_p10_smallgamma": dict(problem="labs", n=30, p=10, gamma_seed=10,
                                  beta_seed=16, ghi=0.05, cost="i32",
                                  state="c64"),
    # p = 40 gradient workloads
    "labs28_p40": dict(problem="labs", n=28, p=40, gamma_seed=8,
                       beta_seed=18, ghi=0.05, cost="i32", state="c64"),
    "maxcut3w28_p40": dict(problem="maxcut3", n=28, p=40, graph_seed=7,
                           weighted=True, weight_seed=17, gamma_seed=8,
                           beta_seed=18, ghi=0.3, cost="f32", state="c64"),
    # LABS n = 30 at depth 40: the precision split's state-fidelity workload
    "labs30_p40": dict(problem="labs", n=30, p=40, gamma_seed=61,
                       beta_seed=62, ghi=0.1, cost="i32", state="c64"),
    # two-layer gradient workloads at the headline sizes (the oracle's stored-
    # state gradient fits host memory at n = 28; n = 30 is checked by central
    # differences of the oracle energy)
    "labs28_p2": dict(problem="labs", n=28, p=2, gamma_seed=8, beta_seed=18,
                      ghi=0.05, cost="i32", state="c64"),
    "labs30_p2": dict(problem="labs", n=30, p=2, gamma_seed=8, beta_seed=18,
                      ghi=0.05, cost="i32", state="c64"),
}


def workload(name, n=None):
    """Workload recipe, optionally with n replaced (same generator, other size)."""
    w = dict(WORKLOADS[name])
    w["name"] = name
    if n is not None:
        w["n"] = n
    return w


def workload_angles(w):
    return (angles(w["p"], w["gamma_seed"], 0.0, w["ghi"]),
            angles(w["p"], w["beta_seed"], 0.0, math.pi))


def sample_indices(n, count, seed):
    """``count`` distinct basis indices in [0, 2^n), sorted (count <= 2^n / 4)."""
    N = 1 << n
    out = np.unique(randint(seed, count, N))
    k = 1
    while out.size < count:
        more = randint(seed, count, N, offset=k * count)
        out = np.unique(np.concatenate([out, more]))
        k += 1
    return out[:count]


def workload_graph(w):
    """(edges, weights) for MaxCut workloads, None for LABS."""
    if w["problem"] == "maxcut3":
        return maxcut_3reg(w["n"], w["graph_seed"], w.get("weighted", False),
                           w.get("weight_seed", 4))
    if w["problem"] == "gnp":
        return maxcut_gnp(w["n"], 0.5, w["graph_seed"], w["weight_seed"])
    return None


def serving_stream(count, seed=9, nmin=16, nmax=26, pmax=40, graphs_per_n=4):
    """Request stream of the serving workload: n ~ U{nmin..nmax}, p ~ U{1..pmax},
    LABS or MaxCut 3-regular (50/50; each n draws from a pool of
    `graphs_per_n` graphs so cost vectors repeat), gamma ~ U[0, 0.1),
    beta ~ U[0, pi).  Returns a list of request dicts."""
    r = randint(seed, 4 * count, 1 << 30)
    out = []
    for i in range(count):
        n = nmin + int(r[4 * i]) % (nmax - nmin + 1)
        p = 1 + int(r[4 * i + 1]) % pmax
        maxcut = int(r[4 * i + 2]) % 2 == 1
        pool = int(r[4 * i + 3]) % graphs_per_n
        g = angles(p, 1000 + 2 * i, 0.0, 0.1)
        b = angles(p, 1001 + 2 * i, 0.0, math.pi)
        if maxcut:
            n += n % 2
            edges, w = maxcut_3reg(n, graph_seed=100 + pool, weighted=False)
            out.append(dict(problem=1, n=n, p=p, gammas=g, betas=b, edges=edges, weights=w,
                            key=pool))
        else:
            out.append(dict(problem=0, n=n, p=p, gammas=g, betas=b, edges=None, weights=None,
                            key=0))
    return out


def poisson_arrivals(count, rate, seed=19):
    """Arrival times (s) of a Poisson process with the given rate."""
    u = uniform(seed, count)
    gaps = -np.log1p(-u) / rate
    return np.cumsum(gaps)
