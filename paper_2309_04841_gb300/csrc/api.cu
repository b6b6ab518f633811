// api.cu -- C ABI entry points (include/qaoa.h) and the host-side pass planner.
//
// The planner turns one call into a short sequence of kernel launches on the
// caller's stream:
//   n <= 12        : single-CTA kernels with the whole state on chip;
//   n >  12 (tiled): the qubits split into k groups, a LOW group (the TB
//                    lowest qubits, one contiguous tile) and HIGH groups
//                    (TB - c qubits each beside 2^c contiguous amplitudes,
//                    c = 3..5); each layer passes over every group once, with
//                    the phase in the pass that opens the layer, and the
//                    group order reversed every layer so that the last pass
//                    of one layer and the first of the next are one pass
//                    (k - 1 passes per layer).  The adjoint runs the same
//                    kind of schedule backwards on (psi, lambda).
// Nothing here allocates device memory: scratch lives in the caller's
// workspace, per-layer constants travel in the kernel parameter blocks.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/qaoa.h"
#include "kernels.h"
#include "qaoa_common.cuh"

using namespace qaoa;

namespace {

thread_local char g_errmsg[256] = "";

qaoa_status fail(qaoa_status st, const char *msg) {
  snprintf(g_errmsg, sizeof(g_errmsg), "%s", msg);
  return st;
}

qaoa_status cuda_fail(cudaError_t e, const char *where) {
  snprintf(g_errmsg, sizeof(g_errmsg), "%s: %s", where, cudaGetErrorString(e));
  return QAOA_ERR_CUDA;
}

#define CK(expr, where)                                 \
  do {                                                  \
    cudaError_t _e = (expr);                            \
    if (_e != cudaSuccess) return cuda_fail(_e, where); \
  } while (0)

// Launch `call` on stream `st`, bracketed by profiling events when enabled;
// `bytes` is the launch's algorithmic HBM traffic.
#define LAUNCH(kind, bytes, st, call)                          \
  do {                                                         \
    const int _pid = prof_begin(st);                           \
    cudaError_t _e = (call);                                   \
    prof_end(_pid, st, kind, (double)(bytes));                 \
    if (_e != cudaSuccess) return cuda_fail(_e, kind " launch"); \
  } while (0)

// The same with a run-time label (static storage).
#define LAUNCH_N(name, bytes, st, call)                       \
  do {                                                        \
    const int _pid = prof_begin(st);                          \
    cudaError_t _e = (call);                                  \
    prof_end(_pid, st, name, (double)(bytes));                \
    if (_e != cudaSuccess) return cuda_fail(_e, "TMA pass launch"); \
  } while (0)

// Profile label of a TMA pass: "fwd_high.k7" etc.  Group kind g: 0 LOW, 1
// HIGH, 2 HIGH on a cluster pair ("bwd_pair"), 3 HIGH on one 512-thread CTA
// ("bwd_wide").  Kind bits: forward 1 = first
// sweep, 2 = phase, 4 = second sweep, 8 = energy / overlap; adjoint (the
// first un-mix sweep is always there) 2 = d/d gamma + un-phase, 4 = second
// un-mix sweep, 8 = lambda = f psi.
const char *tma_pass_name(bool fwd, int g, int k) {
  static char names[2][4][16][24];
  static std::once_flag once;
  std::call_once(once, [] {
    static const char *gn[4] = {"low", "high", "pair", "wide"};
    for (int f = 0; f < 2; ++f)
      for (int h = 0; h < 4; ++h)
        for (int j = 0; j < 16; ++j)
          snprintf(names[f][h][j], sizeof(names[f][h][j]), "%s_%s.k%d", f ? "fwd" : "bwd", gn[h], j);
  });
  return names[fwd ? 1 : 0][g < 0 ? 0 : g > 3 ? 3 : g][k & 15];
}

int num_sms() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (cache[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
      v = 148;
    cache[dev] = v;
  }
  return cache[dev];
}

bool aligned16(const void *p) { return p && ((uintptr_t)p & 15u) == 0; }

bool valid_cost_type(qaoa_cost_type ct) {
  return ct == QAOA_COST_I32 || ct == QAOA_COST_F32 || ct == QAOA_COST_F64 || ct == QAOA_COST_U16;
}

bool integer_cost(qaoa_cost_type ct) { return ct == QAOA_COST_I32 || ct == QAOA_COST_U16; }

bool valid_state_type(qaoa_state_type st) { return st == QAOA_C64 || st == QAOA_C128; }

// Workspace layout: [0, 256) counters, [256, 512) small outputs, then partials.
constexpr size_t kWsCounters = 0, kWsSmall = 256, kWsPartials = 512;

size_t partial_doubles(int n) {
  const size_t tiles = n > 11 ? ((size_t)1 << (n - 11)) : 1;  // smallest tile: 2^11
  size_t need = tiles * 3;
  const size_t red = (size_t)1024 * 4;  // cost-stats / expectation grids
  return need > red ? need : red;
}

struct Ws {
  unsigned *counter;
  unsigned *err;  // set to nonzero by a kernel whose bounded wait ran out
  double *small;
  double *partials;
};

qaoa_status get_ws(int n, void *d_work, size_t bytes, Ws &ws) {
  if (!d_work || ((uintptr_t)d_work & 255u)) return fail(QAOA_ERR_INVALID_ARG, "workspace must be 256-byte aligned and non-NULL");
  if (bytes < qaoa_workspace_bytes(n)) return fail(QAOA_ERR_OUT_OF_MEMORY, "workspace smaller than qaoa_workspace_bytes(n)");
  char *b = reinterpret_cast<char *>(d_work);
  ws.counter = reinterpret_cast<unsigned *>(b + kWsCounters);
  ws.err = reinterpret_cast<unsigned *>(b + kWsCounters + 64);
  ws.small = reinterpret_cast<double *>(b + kWsSmall);
  ws.partials = reinterpret_cast<double *>(b + kWsPartials);
  return QAOA_OK;
}

qaoa_status check_angles(const double *g, const double *b, int p) {
  if (p < 1 || p > 100000) return fail(QAOA_ERR_INVALID_ARG, "p must be in [1, 100000]");
  if (!g || !b) return fail(QAOA_ERR_INVALID_ARG, "NULL angle array");
  for (int i = 0; i < p; ++i)
    if (!std::isfinite(g[i]) || !std::isfinite(b[i])) return fail(QAOA_ERR_INVALID_ARG, "non-finite angle");
  return QAOA_OK;
}

const double kTwoPi = 6.283185307179586476925286766559;

// Phase data for multiplying by exp(-i g f) (times `scale` in table mode;
// the computed mode leaves the scale to the kernel).
template <typename Real>
void make_phase(PhaseData<Real> &ph, double g, qaoa_cost_type ct, const qaoa_cost_stats *stats,
                std::complex<double> scale = 1.0) {
  using C2 = typename C2T<Real>::type;
  memset(&ph, 0, sizeof(ph));
  const double range = stats ? stats->f_max - stats->f_min : 1e300;
  if (integer_cost(ct) && stats && range >= 0 && range < 65536.0) {
    ph.mode = 0;
    ph.fmin = (int)stats->f_min;
    ph.nhi = (int)(range / 256.0) + 1;
    for (int j = 0; j < 256; ++j) {
      const double a = g * (double)j;
      ph.tab_lo[j] = C2{(Real)cos(a), (Real)-sin(a)};
      const double b = g * ((double)stats->f_min + 256.0 * (double)j);
      const std::complex<double> hv = std::complex<double>(cos(b), -sin(b)) * scale;
      ph.tab_hi[j] = C2{(Real)hv.real(), (Real)hv.imag()};
    }
  } else {
    ph.mode = 1;
    const double g2 = g / kTwoPi;
    ph.g2pi = g2;
    ph.g_hi = (float)g2;
    ph.g_lo = (float)(g2 - (double)ph.g_hi);
  }
  ph.scl = (Real)(ph.mode == 1 ? scale.real() : 1.0);  // the tiled passes fold only real scales
}

// Digit tables of exp(-i g f) for the TMA passes (layout in PhaseDigits).
void make_phase(PhaseDigits &ph, double g, qaoa_cost_type ct, const qaoa_cost_stats *stats,
                std::complex<double> scale) {
  memset(&ph, 0, sizeof(ph));
  const double range = stats ? stats->f_max - stats->f_min : 1e300;
  const int shift = stats && stats->step_log2 < 31 ? (int)stats->step_log2 : 0;
  const double rr = range >= 0 ? std::floor(range / std::ldexp(1.0, shift)) : -1.0;  // max d
  auto put = [&](int e, double angle, bool last) {
    std::complex<double> z(cos(angle), -sin(angle));
    if (last) z *= scale;
    ph.d[e] = make_float2((float)z.real(), (float)z.imag());
  };
  const double fmin = stats ? stats->f_min : 0.0, unit = std::ldexp(g, shift);
  if (integer_cost(ct) && stats && rr >= 0 && 64.0 + std::floor(rr / 64.0) + 1.0 <= kPhaseMaxEntries) {
    // two digits: D0[d & 63], D1[d >> 6] (D1 with exp(-i g fmin) and the scale)
    const int n1 = (int)std::floor(rr / 64.0) + 1;
    ph.mode = 0;
    ph.nd = 2;
    ph.fmin = (int)fmin;
    ph.shift = shift;
    ph.last = n1 - 1;
    ph.nent = 64 + n1;
    for (int j = 0; j < 64; ++j) put(j, unit * j, false);
    for (int j = 0; j < n1; ++j) put(64 + j, g * fmin + unit * 64.0 * j, true);
  } else if (integer_cost(ct) && stats && rr >= 0 && rr < 32768.0) {
    // three 5-bit digits
    ph.mode = 0;
    ph.nd = 3;
    ph.fmin = (int)fmin;
    ph.shift = shift;
    ph.last = 31;
    ph.nent = 96;
    for (int j = 0; j < 32; ++j) {
      put(j, unit * j, false);
      put(32 + j, unit * 32.0 * j, false);
      put(64 + j, g * fmin + unit * 1024.0 * j, true);
    }
  } else {
    ph.mode = 1;
    const double g2 = g / kTwoPi;
    ph.g_hi = (float)g2;
    ph.g_lo = (float)(g2 - (double)ph.g_hi);
  }
}

// Rotation schedule of one sweep over the tile bits in `set`: each bit goes
// to the first round (in the kernel's traversal order) holding it in a
// register; bits no round holds in a register go to the first round holding
// them in a lane (rotated with a warp shuffle; TMA kernels only).
template <class PL>
Sweep make_sweep(uint32_t set, bool ascending) {
  Sweep s;
  memset(&s, 0, sizeof(s));
  auto compress = [](uint32_t m, uint32_t within) {
    uint8_t bits = 0;
    int i = 0;
    for (int b = 0; b < 32; ++b)
      if ((within >> b) & 1u) {
        if ((m >> b) & 1u) bits |= (uint8_t)(1u << i);
        ++i;
      }
    return bits;
  };
  uint32_t done = 0;
  for (int k = 0; k < PL::NR; ++k) {
    const int r = ascending ? k : PL::NR - 1 - k;
    const uint32_t m = PL::reg(r) & set & ~done;
    done |= m;
    s.m[r] = compress(m, PL::reg(r));
  }
  for (int k = 0; k < PL::NR; ++k) {
    const int r = ascending ? k : PL::NR - 1 - k;
    const uint32_t m = PL::lane(r) & set & ~done;
    done |= m;
    s.lm[r] = compress(m, PL::lane(r));
  }
  return s;
}

bool uses_lanes(const Sweep &s) { return (s.lm[0] | s.lm[1] | s.lm[2] | s.lm[3]) != 0; }

struct Group {
  bool high;
  int c, h;          // geometry
  uint32_t rot;      // tile bits rotated
  bool cl = false;   // adjoint cluster pair: also rotates the qubit h + TB - c
};

// LOW group + HIGH groups covering qubits [TB, n), TB - chigh per pass
// (chigh passenger bits keep every global segment 2^chigh amplitudes long).
std::vector<Group> plan_groups(int n, int TB, int chigh) {
  std::vector<Group> gs;
  gs.push_back(Group{false, TB, TB, (1u << TB) - 1u});
  const int span = TB - chigh;
  for (int q0 = TB; q0 < n;) {
    const int len = (n - q0) < span ? (n - q0) : span;
    const int h = q0 < n - span ? q0 : n - span;
    uint32_t rot = 0;
    for (int j = chigh; j < TB; ++j) {
      const int xb = h + j - chigh;
      if (xb >= q0 && xb < q0 + len) rot |= 1u << j;
    }
    gs.push_back(Group{true, chigh, h, rot});
    q0 += len;
  }
  return gs;
}

// Groups for the TMA passes: the widest segments (2^c contiguous amplitudes,
// c = 5 or 4: 256/128-byte state rows, 128/64-byte int32 cost rows) that cost
// no extra group; and within a plan whose HIGH groups have narrower segments,
// every group whose new qubits fit the rows of a wider tile gets it (64-byte
// cost rows made the cost load the slowest part of the phase passes).  c = 6
// was measured slower (the 6 row qubits split unevenly over the two rounds).
// Narrower, 8-amplitude segments (64-byte rows, 9 new qubits per group) read
// slowly when their rows are far apart; the adjoint's 9-qubit groups run on
// cluster pairs instead (bwd_groups).
constexpr int kMaxSegBits = 5;

// every HIGH group whose new qubits fit the rows of a wider tile gets it
void widen_groups(std::vector<Group> &gs, int n, int TB) {
  for (Group &G : gs) {
    if (!G.high) continue;
    int q0 = 1 << 30, q1 = -1;  // the group's new qubits: h + j - c for the set bits j of rot
    for (int j = G.c; j < TB; ++j)
      if ((G.rot >> j) & 1u) {
        q0 = std::min(q0, G.h + j - G.c);
        q1 = std::max(q1, G.h + j - G.c);
      }
    for (int c = kMaxSegBits; c > G.c; --c) {
      const int rows = TB - c;
      if (q1 - q0 + 1 > rows) continue;
      const int h = q0 < n - rows ? q0 : n - rows;
      uint32_t rot = 0;
      for (int j = c; j < TB; ++j) {
        const int q = h + j - c;
        if (q >= q0 && q <= q1) rot |= 1u << j;
      }
      G = Group{true, c, h, rot};
      break;
    }
  }
}

std::vector<Group> tma_groups(int n, int TB) {
  std::vector<Group> best = plan_groups(n, TB, 4);
  for (int c = 5; c <= kMaxSegBits; ++c) {
    std::vector<Group> g = plan_groups(n, TB, c);
    if (g.size() <= best.size()) best = g;
  }
  widen_groups(best, n, TB);
  return best;
}

// Adjoint groups with 9-qubit groups: the LOW group (qubits 0..TB-1), then
// HIGH groups of 2^c contiguous amplitudes (c = 4) times TB - c local rows,
// of which a 9-qubit group (`cl`) adds one more row qubit (h + TB - c): its
// 2^13-amplitude tile runs on one 512-thread CTA, or split over the two CTAs
// of a cluster pair (see tma_backward): TB - c + 1 new qubits per group
// instead of TB - c.
// Taken where it needs fewer groups than the plain plan (LABS n = 30:
// {0-11}, {12-20}, {21-29} -- three groups, two passes per layer, instead of
// four; also n = 21, 29); only as many groups as necessary are cluster pairs.
// (At n = 21 and 29 a plain plan with one 8-amplitude group has as few
// groups; measured at n = 29: 114.1 ms per LABS p = 10 evaluation against
// 108.8 ms with the pair.)  The environment variable QAOA_ADJOINT_PAIRS
// overrides the choice: "never" takes the plain plan, "always" makes every
// HIGH group a 9-qubit group (for profiling and cross-checks of those
// kernels at any size); unset or anything else is the rule above.
// The 9-qubit groups run on one 512-thread CTA per 2^13-amplitude tile, except
// the passes that end with the un-phase (the last pass), which take the
// cluster pair.  QAOA_ADJOINT_WIDE=pair puts every pass of those groups on
// the pair, =all every pass on the 512-thread CTA (tests and comparison).
// Returns 0 (pairs), 1 (default), 2 (all).
int adjoint_wide_mode() {
  const char *e = getenv("QAOA_ADJOINT_WIDE");
  if (e && !strcmp(e, "pair")) return 0;
  if (e && !strcmp(e, "all")) return 2;
  return 1;
}

int adjoint_pairs_mode() {
  const char *e = getenv("QAOA_ADJOINT_PAIRS");
  if (!e) return 0;
  if (!strcmp(e, "never")) return -1;
  if (!strcmp(e, "always")) return 1;
  return 0;
}

std::vector<Group> bwd_groups(int n, int TB) {
  std::vector<Group> plain = tma_groups(n, TB);
  const int c = 4, rows = TB - c;
  const int R = n - TB;  // qubits above the LOW group
  const int mode = adjoint_pairs_mode();
  if (R <= 0 || mode < 0) return plain;
  const int k = (R + rows) / (rows + 1);      // HIGH groups, rows + 1 qubits at most each
  int ncl = R - rows * k > 0 ? R - rows * k : 0;  // groups that need the extra qubit
  if (mode > 0)
    ncl = k;
  else if (!(1 + k < (int)plain.size()))
    return plain;
  std::vector<Group> gs;
  gs.push_back(Group{false, TB, TB, (1u << TB) - 1u});
  int q0 = TB;
  for (int g = 0; g < k; ++g) {
    const bool cl = g >= k - ncl;  // the top groups take the pairs
    const int len = std::min(rows + (cl ? 1 : 0), n - q0);
    Group G;
    G.high = true;
    G.c = c;
    G.cl = cl;
    // local rows h .. h + rows - 1 (and the pair's qubit h + rows, tile bit
    // TB); a group at the top of the range starts lower and rotates only its
    // new qubits
    const int span = rows + (cl ? 1 : 0);
    G.h = q0 + span <= n ? q0 : n - span;
    G.rot = 0;
    for (int j = c; j < TB + (cl ? 1 : 0); ++j) {
      const int q = G.h + j - c;
      if (q >= q0 && q < q0 + len) G.rot |= 1u << j;
    }
    gs.push_back(G);
    q0 += len;
  }
  return gs;
}

Geom make_geom(int n, const Group &G, int TB) {
  Geom g;
  g.n = n;
  g.tb = TB;
  g.c = G.c;
  g.h = G.h;
  g.ntiles = 1ull << (n - TB);
  return g;
}

template <typename Real>
SmallLayer<Real> small_layer(double gamma, double beta) {
  SmallLayer<Real> L;
  L.cb = (Real)cos(beta);
  L.sb = (Real)sin(beta);
  const double g2 = gamma / kTwoPi;
  L.g2pi = g2;
  L.g_hi = (float)g2;
  L.g_lo = (float)(g2 - (double)L.g_hi);
  return L;
}

int cost_kind(qaoa_cost_type ct) { return (int)ct; }

double cost_bytes(qaoa_cost_type ct) {
  return ct == QAOA_COST_F64 ? 8.0 : ct == QAOA_COST_U16 ? 2.0 : 4.0;
}

// ----------------------------------------------------------- small path

template <typename Real>
qaoa_status small_forward(int n, const void *cost, qaoa_cost_type ct, double fmin,
                          const double *gam, const double *bet, int p, void *state, int init_plus,
                          double *d_out, cudaStream_t s) {
  using C2 = typename C2T<Real>::type;
  for (int l0 = 0; l0 < p; l0 += kSmallMaxLayers) {
    const int nl = (p - l0) < kSmallMaxLayers ? (p - l0) : kSmallMaxLayers;
    SmallParams<Real> P;
    memset(&P, 0, sizeof(P));
    P.psi = reinterpret_cast<C2 *>(state);
    P.lam = nullptr;
    P.cost = cost;
    P.cost_kind = cost_kind(ct);
    P.n = n;
    P.nl = nl;
    P.mode = 0;
    P.init_plus = (l0 == 0) && init_plus;
    P.amp = (Real)(1.0 / sqrt(ldexp(1.0, n)));
    P.reduce = (l0 + nl == p) && d_out != nullptr;
    P.fmin_d = fmin;
    P.out = d_out;
    for (int i = 0; i < nl; ++i) P.L[i] = small_layer<Real>(gam[l0 + i], bet[l0 + i]);
    LAUNCH("small", 2.0 * sizeof(C2) * (double)(1 << n), s, launch_small(P, s));
  }
  return QAOA_OK;
}

template <typename Real>
qaoa_status small_grad(int n, const void *cost, qaoa_cost_type ct, double fmin, const double *gam,
                       const double *bet, int p, void *state, void *lam, double *d_out,
                       cudaStream_t s) {
  using C2 = typename C2T<Real>::type;
  const Real amp = (Real)(1.0 / sqrt(ldexp(1.0, n)));
  if (p <= kSmallMaxLayers) {
    SmallParams<Real> P;
    memset(&P, 0, sizeof(P));
    P.psi = reinterpret_cast<C2 *>(state);
    P.lam = reinterpret_cast<C2 *>(lam);
    P.cost = cost;
    P.cost_kind = cost_kind(ct);
    P.n = n;
    P.nl = p;
    P.mode = 1;
    P.init_plus = 1;
    P.amp = amp;
    P.reduce = 1;
    P.fmin_d = fmin;
    P.out = d_out;
    P.out_dg = d_out + 2;
    P.out_db = d_out + 2 + p;
    for (int i = 0; i < p; ++i) P.L[i] = small_layer<Real>(gam[i], bet[i]);
    LAUNCH("small", 3.0 * sizeof(C2) * (double)(1 << n), s, launch_small(P, s));
    return QAOA_OK;
  }
  qaoa_status st = small_forward<Real>(n, cost, ct, fmin, gam, bet, p, state, 1, d_out, s);
  if (st != QAOA_OK) return st;
  const int nchunks = (p + kSmallMaxLayers - 1) / kSmallMaxLayers;
  for (int ci = nchunks - 1; ci >= 0; --ci) {
    const int l0 = ci * kSmallMaxLayers;
    const int nl = (p - l0) < kSmallMaxLayers ? (p - l0) : kSmallMaxLayers;
    SmallParams<Real> P;
    memset(&P, 0, sizeof(P));
    P.psi = reinterpret_cast<C2 *>(state);
    P.lam = reinterpret_cast<C2 *>(lam);
    P.cost = cost;
    P.cost_kind = cost_kind(ct);
    P.n = n;
    P.nl = nl;
    P.mode = 2;
    P.init_lambda = (ci == nchunks - 1);
    P.amp = amp;
    P.fmin_d = fmin;
    P.out_dg = d_out + 2 + l0;
    P.out_db = d_out + 2 + p + l0;
    for (int i = 0; i < nl; ++i) P.L[i] = small_layer<Real>(gam[l0 + i], bet[l0 + i]);
    LAUNCH("small", 4.0 * sizeof(C2) * (double)(1 << n), s, launch_small(P, s));
  }
  return QAOA_OK;
}

// ----------------------------------------------------------- tiled path

template <typename Real> struct FwdTB;
template <> struct FwdTB<float> { using Low = PlanF13Low; using High = PlanF13High; };
template <> struct FwdTB<double> { using Low = PlanT12Low; using High = PlanT12High; };
template <typename Real> struct BwdTB;
template <> struct BwdTB<float> { using Low = PlanT12Low; using High = PlanT12High; };
template <> struct BwdTB<double> { using Low = PlanT11Low; using High = PlanT11High; };

// One pass of a schedule: [sweep s1 of group g with beta_{l1}] [phase of layer lp]
// [sweep s2 of group g with beta_{l2}]; -1 marks an absent part.
struct PassOp {
  int group;
  int l1, lp, l2;
  bool init;    // forward: start from |+>;  adjoint: lambda <- f psi
  bool reduce;  // forward: energy/overlap of the result
};

// Forward schedule with cross-layer fusion.  Layer l applies every group
// once; the X rotations of different qubits commute, so each layer's group
// order is free.  Taking layer l+1's order as the reverse of layer l's, the
// last group of layer l is the first of layer l+1, and both share one pass
// around the phase of layer l+1: p*k - (p-1) passes instead of p*k.  With
// three or more groups the LOW group (0, three rounds per sweep) goes second,
// so it never carries two sweeps and the phase in one pass: its passes are
// single sweeps, which run at the copy bandwidth, and the two-round HIGH
// groups take the pivots (LABS n = 30: 246.8 instead of 254.5 ms per
// objective+gradient evaluation).
std::vector<PassOp> forward_schedule(int k, int p, bool init_plus, bool reduce) {
  std::vector<PassOp> ops;
  if (k == 1) {
    for (int l = 0; l < p; ++l) ops.push_back(PassOp{0, -1, l, l, l == 0 && init_plus, false});
  } else {
    std::vector<int> order(k);
    for (int i = 0; i < k; ++i) order[i] = i;
    if (k >= 3) std::swap(order[0], order[1]);
    ops.push_back(PassOp{order[0], -1, 0, 0, init_plus, false});
    for (int l = 0; l < p; ++l) {
      for (int i = 1; i + 1 < k; ++i) ops.push_back(PassOp{order[i], -1, -1, l, false, false});
      const int z = order[k - 1];
      if (l + 1 < p)
        ops.push_back(PassOp{z, l, l + 1, l + 1, false, false});
      else
        ops.push_back(PassOp{z, l, -1, -1, false, false});
      std::vector<int> rev(order.rbegin(), order.rend());
      order = rev;
    }
  }
  ops.back().reduce = reduce;
  return ops;
}

// Adjoint schedule: un-apply layers p-1 .. 0.  s1 un-rotates layer l1 (and
// accumulates its d/d beta), the phase part accumulates d/d gamma of layer lp
// and un-applies that phase, s2 un-rotates layer l2 < lp.
std::vector<PassOp> adjoint_schedule(int k, int p) {
  std::vector<PassOp> ops;
  if (k == 1) {
    for (int l = p - 1; l >= 0; --l) ops.push_back(PassOp{0, l, l, -1, l == p - 1, false});
    return ops;
  }
  // The pivot alternates between the two ends of the order; with three or
  // more groups the LOW group (0, three rounds per sweep) goes second, so it
  // never carries two sweeps and the phase in one pass.
  std::vector<int> order(k);
  for (int i = 0; i < k; ++i) order[i] = i;
  if (k >= 3) std::swap(order[0], order[1]);
  for (int l = p - 1; l >= 0; --l) {
    if (l == p - 1) ops.push_back(PassOp{order[0], l, -1, -1, true, false});
    for (int i = 1; i + 1 < k; ++i) ops.push_back(PassOp{order[i], l, -1, -1, false, false});
    const int z = order[k - 1];
    ops.push_back(PassOp{z, l, l, l > 0 ? l - 1 : -1, false, false});
    std::vector<int> rev(order.rbegin(), order.rend());
    order = rev;
  }
  return ops;
}

// Reduced form of exp(-i b X) for the tiled passes (rot_tan): the form with
// |t| <= 1 and the real factor it drops.
struct RedRot {
  double t;
  int form;
  double sigma;
};

RedRot red_rot(double b) {
  const double c = cos(b), s = sin(b);
  if (fabs(c) >= fabs(s)) return RedRot{s / c, 0, c};
  return RedRot{c / s, 1, s};
}

double ipow_d(double x, int k) {
  double r = 1.0;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

int sweep_qubits(const Sweep &w) {
  int k = 0;
  for (int r = 0; r < 4; ++r) k += __builtin_popcount((unsigned)w.m[r]);
  return k;
}

int popc8(uint8_t m) { return __builtin_popcount((unsigned)m); }

template <typename Real, class Low, class High>
qaoa_status tiled_forward_pl(int n, const void *cost, qaoa_cost_type ct, const qaoa_cost_stats *stats,
                             const double *gam, const double *bet, int p, void *state, int init_plus,
                             const Ws &ws, double *d_out, cudaStream_t s) {
  using C2 = typename C2T<Real>::type;
  const int TB = Low::TB;
  const std::vector<Group> gs = plan_groups(n, TB, kHighC);
  const std::vector<PassOp> ops = forward_schedule((int)gs.size(), p, init_plus != 0, d_out != nullptr);
  const int nsm = num_sms();
  if (d_out) CK(cudaMemsetAsync(ws.counter, 0, sizeof(unsigned), s), "memset counter");
  FwdParams<Real> P;
  // the stored state is the true one divided by sig (the dropped factors of
  // the reduced rotations); the next phase, or the last pass, multiplies it back
  double sig = 1.0;
  for (const PassOp &op : ops) {
    const Group &G = gs[op.group];
    memset(&P, 0, sizeof(P));
    P.psi = reinterpret_cast<C2 *>(state);
    P.cost = cost;
    P.cost_kind = cost_kind(ct);
    P.g = make_geom(n, G, TB);
    const bool two = op.l1 >= 0 && op.l2 >= 0;  // both sweeps: s1 ascends, s2 descends
    // (these plans hold every rotated bit in registers: no lane rotations)
    if (op.l1 >= 0) {
      P.s1 = G.high ? make_sweep<High>(G.rot, true) : make_sweep<Low>(G.rot, true);
      const RedRot R = red_rot(bet[op.l1]);
      P.t1 = (Real)R.t;
      P.form1 = R.form;
      sig *= ipow_d(R.sigma, sweep_qubits(P.s1));
    }
    if (op.l2 >= 0) {
      P.s2 = G.high ? make_sweep<High>(G.rot, !two) : make_sweep<Low>(G.rot, !two);
      const RedRot R = red_rot(bet[op.l2]);
      P.t2 = (Real)R.t;
      P.form2 = R.form;
    }
    if (uses_lanes(P.s1) || uses_lanes(P.s2)) return fail(QAOA_ERR_INVALID_ARG, "internal: plan needs lane rotations");
    P.has_phase = op.lp >= 0;
    if (P.has_phase) {  // s1 runs before the phase, s2 after it
      make_phase<Real>(P.ph, gam[op.lp], ct, stats, sig);
      sig = 1.0;
    }
    if (op.l2 >= 0) sig *= ipow_d(red_rot(bet[op.l2]).sigma, sweep_qubits(P.s2));
    P.post_scale = (Real)1;
    if (&op == &ops.back()) {
      P.post_scale = (Real)sig;
      sig = 1.0;
    }
    P.init_plus = op.init;
    P.amp = (Real)(1.0 / sqrt(ldexp(1.0, n)));
    P.reduce = op.reduce;
    P.fmin_d = stats ? stats->f_min : 0.0;
    P.partials = ws.partials;
    P.counter = ws.counter;
    P.out = d_out;
    const double N = (double)(1ull << n);
    const double bytes = (P.init_plus ? 1.0 : 2.0) * sizeof(C2) * N +
                         ((P.has_phase || P.reduce) ? cost_bytes(ct) * N : 0.0);
    if (G.high)
      LAUNCH("fwd_high", bytes, s, launch_fwd(P, true, TB, s, nsm));
    else
      LAUNCH("fwd_low", bytes, s, launch_fwd(P, false, TB, s, nsm));
  }
  return QAOA_OK;
}

// complex128 at n <= 16: tiles small enough to spread the FP64-bound passes
// over more SMs, with no more groups than the 4096-amplitude tiles (the
// partial sums of the tiles fit the workspace: 2^(16-9) * 3 doubles)
template <typename Real>
qaoa_status tiled_forward(int n, const void *cost, qaoa_cost_type ct, const qaoa_cost_stats *stats,
                          const double *gam, const double *bet, int p, void *state, int init_plus,
                          const Ws &ws, double *d_out, cudaStream_t s) {
  if constexpr (sizeof(Real) == 8) {
    if (n <= 14)
      return tiled_forward_pl<Real, PlanT9Low, PlanT9High>(n, cost, ct, stats, gam, bet, p, state, init_plus,
                                                           ws, d_out, s);
    if (n <= 16)
      return tiled_forward_pl<Real, PlanT10Low, PlanT10High>(n, cost, ct, stats, gam, bet, p, state,
                                                             init_plus, ws, d_out, s);
  }
  return tiled_forward_pl<Real, typename FwdTB<Real>::Low, typename FwdTB<Real>::High>(
      n, cost, ct, stats, gam, bet, p, state, init_plus, ws, d_out, s);
}

template <typename Real, class Low, class High>
qaoa_status tiled_backward_pl(int n, const void *cost, qaoa_cost_type ct, const qaoa_cost_stats *stats,
                              const double *gam, const double *bet, int p, void *state, void *lam,
                              const Ws &ws, double *d_grad_g, double *d_grad_b, cudaStream_t s) {
  using C2 = typename C2T<Real>::type;
  const int TB = Low::TB;
  const std::vector<Group> gs = plan_groups(n, TB, kHighC);
  const std::vector<PassOp> ops = adjoint_schedule((int)gs.size(), p);
  const int nsm = num_sms();
  CK(cudaMemsetAsync(ws.counter, 0, sizeof(unsigned), s), "memset counter");
  BwdParams<Real> P;
  double sig = 1.0;
  for (const PassOp &op : ops) {
    const Group &G = gs[op.group];
    memset(&P, 0, sizeof(P));
    P.psi = reinterpret_cast<C2 *>(state);
    P.lam = reinterpret_cast<C2 *>(lam);
    P.cost = cost;
    P.cost_kind = cost_kind(ct);
    P.g = make_geom(n, G, TB);
    // psi and lambda are stored divided by sig; un-rotations are the reduced
    // forms of exp(-i (-beta) X)
    P.s1 = G.high ? make_sweep<High>(G.rot, true) : make_sweep<Low>(G.rot, true);
    {
      const RedRot R = red_rot(-bet[op.l1]);
      P.t1 = (Real)R.t;
      P.form1 = R.form;
      for (int r = 0; r < Low::NR; ++r) {  // the kernel walks s1 upward
        P.w1[r] = (Real)(sig * sig);
        sig *= ipow_d(R.sigma, popc8(P.s1.m[r]));
      }
    }
    P.out_b1 = d_grad_b + op.l1;
    if (op.lp >= 0) {
      P.has_phase = 1;
      P.wg = (Real)(sig * sig);
      make_phase<Real>(P.ph, -gam[op.lp], ct, stats, sig);  // the un-phase pays the pending scale
      sig = 1.0;
      P.out_g = d_grad_g + op.lp;
    }
    if (op.l2 >= 0) {
      P.s2 = G.high ? make_sweep<High>(G.rot, false) : make_sweep<Low>(G.rot, false);
      const RedRot R = red_rot(-bet[op.l2]);
      P.t2 = (Real)R.t;
      P.form2 = R.form;
      for (int k = 0; k < Low::NR; ++k) {  // and s2 downward
        const int r = Low::NR - 1 - k;
        P.w2[r] = (Real)(sig * sig);
        sig *= ipow_d(R.sigma, popc8(P.s2.m[r]));
      }
      P.out_b2 = d_grad_b + op.l2;
    }
    P.post_scale = (Real)1;
    if (&op == &ops.back()) {
      P.post_scale = (Real)sig;
      sig = 1.0;
    }
    if (uses_lanes(P.s1) || uses_lanes(P.s2))
      return fail(QAOA_ERR_INVALID_ARG, "internal: plan needs lane rotations");
    P.init_lambda = op.init;
    P.partials = ws.partials;
    P.counter = ws.counter;
    const double N = (double)(1ull << n);
    const double bytes = (P.init_lambda ? 3.0 : 4.0) * sizeof(C2) * N +
                         ((P.has_phase || P.init_lambda) ? cost_bytes(ct) * N : 0.0);
    if (G.high)
      LAUNCH("bwd_high", bytes, s, launch_bwd(P, true, TB, s, nsm));
    else
      LAUNCH("bwd_low", bytes, s, launch_bwd(P, false, TB, s, nsm));
  }
  return QAOA_OK;
}

template <typename Real>
qaoa_status tiled_backward(int n, const void *cost, qaoa_cost_type ct, const qaoa_cost_stats *stats,
                           const double *gam, const double *bet, int p, void *state, void *lam,
                           const Ws &ws, double *d_grad_g, double *d_grad_b, cudaStream_t s) {
  if constexpr (sizeof(Real) == 8) {
    if (n <= 14)
      return tiled_backward_pl<Real, PlanT9Low, PlanT9High>(n, cost, ct, stats, gam, bet, p, state, lam, ws,
                                                            d_grad_g, d_grad_b, s);
    if (n <= 16)
      return tiled_backward_pl<Real, PlanT10Low, PlanT10High>(n, cost, ct, stats, gam, bet, p, state, lam,
                                                              ws, d_grad_g, d_grad_b, s);
  }
  return tiled_backward_pl<Real, typename BwdTB<Real>::Low, typename BwdTB<Real>::High>(
      n, cost, ct, stats, gam, bet, p, state, lam, ws, d_grad_g, d_grad_b, s);
}

// ---------------------------------------------------- TMA (complex64) path

bool tma_ok(qaoa_cost_type ct) { return ct == QAOA_COST_I32 || ct == QAOA_COST_F32 || ct == QAOA_COST_U16; }

// Reduced ("tan") form of exp(-i b X) (forward) or exp(+i b X) (adjoint):
// exp(-/+ i b X) = sigma * G with |tau| <= 1 (see TmaFwdParams).
// f_min as the 32-bit word the cost vector holds (int32 or float32 bits).
uint32_t fmin_word(qaoa_cost_type ct, const qaoa_cost_stats *stats) {
  const double f = stats ? stats->f_min : 0.0;
  if (integer_cost(ct)) return (uint32_t)(int32_t)f;
  const float x = (float)f;
  uint32_t w;
  memcpy(&w, &x, sizeof(w));
  return w;
}

struct TanRot {
  float tau;
  int form;
  std::complex<double> sigma;
};

// Reduced form of exp(-i b X) in the twisted basis (b = -beta for the
// adjoint): form 0 t = tan b, sigma = cos b; form 1 u = cot b, sigma = sin b.
TanRot tan_rot(double beta, bool adjoint) {
  const double b = adjoint ? -beta : beta;
  const double c = cos(b), s = sin(b);
  TanRot r;
  if (fabs(c) >= fabs(s)) {
    r.form = 0;
    r.tau = (float)(s / c);
    r.sigma = c;
  } else {
    r.form = 1;
    r.tau = (float)(c / s);
    r.sigma = s;
  }
  return r;
}

float2 f2c(std::complex<double> z) { return make_float2((float)z.real(), (float)z.imag()); }

// untwist: leave the final state in the standard basis (the adjoint instead
// continues from the twisted one).
qaoa_status tma_forward(int n, const void *cost, qaoa_cost_type ct, const qaoa_cost_stats *stats,
                        const double *gam, const double *bet, int p, void *state, int init_plus,
                        const Ws &ws, double *d_out, bool untwist, cudaStream_t s) {
  using Low = PlanTmaF13Low;
  using High = PlanTmaF13High;
  const int TB = Low::TB;
  const std::vector<Group> gs = tma_groups(n, TB);
  const std::vector<PassOp> ops = forward_schedule((int)gs.size(), p, init_plus != 0, d_out != nullptr);
  const int nsm = num_sms();
  if (d_out) CK(cudaMemsetAsync(ws.counter, 0, sizeof(unsigned), s), "memset counter");
  static TmaFwdParams P;  // parameter block; launches copy it, calls are serialised
  static std::mutex *mu = new std::mutex();
  std::lock_guard<std::mutex> lock(*mu);
  std::complex<double> sig = 1.0;  // scale the stored state still owes
  for (const PassOp &op : ops) {
    const Group &G = gs[op.group];
    memset(&P, 0, sizeof(P));
    const int h = G.high ? G.h : 4, c = G.high ? G.c : 4;
    CK(make_tile_map(&P.map_psi, state, n, TB, h, c, 8, 128), "tensor map (state)");
    P.psi = reinterpret_cast<float2 *>(state);
    CK(make_tile_map(&P.map_cost, const_cast<void *>(cost), n, TB, h, c, (int)cost_bytes(ct), 0),
       "tensor map (cost)");
    P.ntiles = 1ull << (n - TB);
    P.h = h;
    P.c = c;
    P.cost_kind = cost_kind(ct);
    const bool two = op.l1 >= 0 && op.l2 >= 0;
    const int nrot = __builtin_popcount(G.rot);
    if (op.l1 >= 0) {
      P.s1 = G.high ? make_sweep<High>(G.rot, true) : make_sweep<Low>(G.rot, true);
      const TanRot R = tan_rot(bet[op.l1], false);
      P.tau1 = R.tau;
      P.form1 = R.form;
      sig *= std::pow(R.sigma, nrot);
    }
    P.has_phase = op.lp >= 0;
    if (P.has_phase) {
      // the pending scale rides on the phase multiply
      make_phase(P.ph, gam[op.lp], ct, stats, sig);
      P.scl_phase = f2c(sig);
      sig = 1.0;
    }
    if (op.l2 >= 0) {
      P.s2 = G.high ? make_sweep<High>(G.rot, !two) : make_sweep<Low>(G.rot, !two);
      const TanRot R = tan_rot(bet[op.l2], false);
      P.tau2 = R.tau;
      P.form2 = R.form;
      sig *= std::pow(R.sigma, nrot);
    }
    if (&op == &ops.back()) {
      P.end_scale = 1;
      P.scl_end = f2c(sig);
      P.untwist = untwist;
      sig = 1.0;
    }
    if (uses_lanes(P.s1) || uses_lanes(P.s2)) return fail(QAOA_ERR_INVALID_ARG, "internal: plan needs lane rotations");
    P.init_plus = op.init;
    P.twist_in = &op == &ops.front() && !op.init;
    P.amp = (float)(1.0 / sqrt(ldexp(1.0, n)));
    P.reduce = op.reduce;
    P.fmin_word = fmin_word(ct, stats);
    P.partials = ws.partials;
    P.counter = ws.counter;
    P.out = d_out;
    P.err = ws.err;
    const double N = (double)(1ull << n);
    const double bytes = (P.init_plus ? 8.0 : 16.0) * N + ((P.has_phase || P.reduce) ? cost_bytes(ct) * N : 0.0);
    const int kind = (op.l1 >= 0 ? 1 : 0) | (P.has_phase ? 2 : 0) | (op.l2 >= 0 ? 4 : 0) | (P.reduce ? 8 : 0);
    LAUNCH_N(tma_pass_name(true, G.high ? 1 : 0, kind), bytes, s,
             ct == QAOA_COST_U16 ? launch_fwd_tma_u16(P, G.high, s, nsm) : launch_fwd_tma(P, G.high, s, nsm));
  }
  return QAOA_OK;
}

qaoa_status tma_backward(int n, const void *cost, qaoa_cost_type ct, const qaoa_cost_stats *stats,
                         const double *gam, const double *bet, int p, void *state, void *lam,
                         const Ws &ws, double *d_grad_g, double *d_grad_b, cudaStream_t s) {
  using Low = PlanTmaB12Low;
  using High = PlanTmaB12High;
  const int TB = Low::TB;
  // HIGH groups of 9 new qubits on cluster pairs where they save a group
  const std::vector<Group> gs = bwd_groups(n, TB);
  const std::vector<PassOp> ops = adjoint_schedule((int)gs.size(), p);
  const int nsm = num_sms();
  CK(cudaMemsetAsync(ws.counter, 0, sizeof(unsigned), s), "memset counter");
  static TmaBwdParams P;
  const int wide_mode = adjoint_wide_mode();
  static std::mutex *mu = new std::mutex();
  std::lock_guard<std::mutex> lock(*mu);
  std::complex<double> sig = 1.0;  // common scale psi and lambda carry
  for (const PassOp &op : ops) {
    const Group &G = gs[op.group];
    memset(&P, 0, sizeof(P));
    const int h = G.high ? G.h : 4, c = G.high ? G.c : 4;
    // a 9-qubit group's pass: one 512-thread CTA per tile, or the cluster pair
    const bool wide = G.cl && (wide_mode == 2 || (wide_mode == 1 && !(op.lp >= 0 && op.l2 < 0)));
    const int TBg = wide ? PlanTmaB13High::TB : TB;
    CK(make_tile_map(&P.map_psi, state, n, TBg, h, c, 8, 128), "tensor map (psi)");
    CK(make_tile_map(&P.map_lam, lam, n, TBg, h, c, 8, 128), "tensor map (lambda)");
    P.psi = reinterpret_cast<float2 *>(state);
    P.lam = reinterpret_cast<float2 *>(lam);
    if (wide)
      CK(make_tile_map(&P.map_cost, const_cast<void *>(cost), n, TBg, h, c, (int)cost_bytes(ct), 0),
         "tensor map (cost)");
    else if (G.cl && op.lp >= 0)
      CK(make_pair_cost_map(&P.map_cost, const_cast<void *>(cost), n, h, (int)cost_bytes(ct)),
         "tensor map (pair cost)");
    else
      CK(make_tile_map(&P.map_cost, const_cast<void *>(cost), n, TB, h, c, (int)cost_bytes(ct), 0),
         "tensor map (cost)");
    P.ntiles = 1ull << (n - TBg);
    P.h = h;
    P.c = c;
    P.cost_kind = cost_kind(ct);
    // A cluster pair rotates tile bits 8..11 in round 0 (layout L0), tile
    // bits 4..7 in round 1's registers and tile bit 12 at its lane bit 4
    // (layout L1, see k_bwd_pair): the group's new qubits among those.
    Sweep pair_sweep;
    memset(&pair_sweep, 0, sizeof(pair_sweep));
    pair_sweep.m[0] = (uint8_t)((G.rot >> 8) & 0xFu);
    pair_sweep.m[1] = (uint8_t)((G.rot >> 4) & 0xFu);
    pair_sweep.lm[1] = (uint8_t)(((G.rot >> TB) & 1u) << 4);
    P.cluster = wide ? 2 : G.cl ? 1 : 0;
    P.s1 = wide   ? make_sweep<PlanTmaB13High>(G.rot, true)
           : G.cl ? pair_sweep
           : G.high ? make_sweep<High>(G.rot, true) : make_sweep<Low>(G.rot, true);
    {
      const TanRot R = tan_rot(bet[op.l1], true);
      P.tau1 = R.tau;
      P.form1 = R.form;
      // stored vectors are the true ones divided by sig, so a raw inner
      // product is the true one divided by |sig|^2
      for (int r = 0; r < Low::NR; ++r) {  // the kernel walks s1 upward
        P.w1[r] = (float)std::norm(sig);
        sig *= std::pow(R.sigma, popc8(P.s1.m[r]) + popc8(P.s1.lm[r]));
      }
    }
    P.out_b1 = d_grad_b + op.l1;
    if (op.lp >= 0) {
      P.has_phase = 1;
      P.wg = (float)std::norm(sig);
      // the un-phase multiply also pays the pending scale
      make_phase(P.ph, -gam[op.lp], ct, stats, sig);
      P.scl_phase = f2c(sig);
      sig = 1.0;
      P.out_g = d_grad_g + op.lp;
    }
    if (op.l2 >= 0) {
      P.s2 = wide   ? make_sweep<PlanTmaB13High>(G.rot, false)
             : G.cl ? pair_sweep
             : G.high ? make_sweep<High>(G.rot, false) : make_sweep<Low>(G.rot, false);
      const TanRot R = tan_rot(bet[op.l2], true);
      P.tau2 = R.tau;
      P.form2 = R.form;
      for (int k = 0; k < Low::NR; ++k) {  // and s2 downward
        const int r = Low::NR - 1 - k;
        P.w2[r] = (float)std::norm(sig);
        sig *= std::pow(R.sigma, popc8(P.s2.m[r]) + popc8(P.s2.lm[r]));
      }
      P.out_b2 = d_grad_b + op.l2;
    }
    if ((uses_lanes(P.s1) || uses_lanes(P.s2)) && !G.cl)
      return fail(QAOA_ERR_INVALID_ARG, "internal: plan needs lane rotations");
    P.init_lambda = op.init;
    P.untwist = &op == &ops.back();
    P.partials = ws.partials;
    P.counter = ws.counter;
    P.err = ws.err;
    const double N = (double)(1ull << n);
    // psi and lambda read and written (lambda not read by the first pass, not
    // written by the last), plus the cost vector where the pass reads it
    const double bytes = (32.0 - (P.init_lambda ? 8.0 : 0.0) - (P.untwist ? 8.0 : 0.0)) * N +
                         ((P.has_phase || P.init_lambda) ? cost_bytes(ct) * N : 0.0);
    const int kind = (P.has_phase ? 2 : 0) | (op.l2 >= 0 ? 4 : 0) | (P.init_lambda ? 8 : 0);
    LAUNCH_N(tma_pass_name(false, wide ? 3 : G.cl ? 2 : G.high ? 1 : 0, kind), bytes, s,
             ct == QAOA_COST_U16 ? launch_bwd_tma_u16(P, G.high, s, nsm) : launch_bwd_tma(P, G.high, s, nsm));
  }
  return QAOA_OK;
}

qaoa_status check_common(int n, const void *cost, qaoa_cost_type ct, const void *state,
                         qaoa_state_type st) {
  if (n < 1 || n > QAOA_MAX_N) return fail(QAOA_ERR_INVALID_ARG, "n out of range");
  if (!valid_cost_type(ct)) return fail(QAOA_ERR_INVALID_ARG, "bad cost type");
  if (!valid_state_type(st)) return fail(QAOA_ERR_INVALID_ARG, "bad state type");
  if (!aligned16(cost)) return fail(QAOA_ERR_INVALID_ARG, "cost pointer NULL or not 16-byte aligned");
  if (!aligned16(state)) return fail(QAOA_ERR_INVALID_ARG, "state pointer NULL or not 16-byte aligned");
  return QAOA_OK;
}

// Decide how to accumulate real weights exactly: if every weight is an
// integer multiple of 2^-e and sum |w| 2^e < 2^53, integer fixed point.
bool dyadic_scale(const double *w, size_t m, int *e_out) {
  int e = 0;
  for (size_t i = 0; i < m; ++i) {
    if (w[i] == 0.0) continue;
    int ex;
    const double fr = frexp(w[i], &ex);  // w = fr * 2^ex, 0.5 <= |fr| < 1
    // smallest k with fr * 2^53 divisible: count trailing zero bits of mantissa
    int64_t mant = (int64_t)ldexp(fr, 53);
    int tz = 0;
    while (tz < 53 && (mant & 1) == 0) {
      mant >>= 1;
      ++tz;
    }
    const int need = 53 - tz - ex;  // w * 2^need is an integer
    if (need > e) e = need;
  }
  if (e > 200) return false;
  double tot = 0.0;
  for (size_t i = 0; i < m; ++i) tot += fabs(ldexp(w[i], e));
  if (!(tot < 9007199254740992.0)) return false;
  *e_out = e;
  return true;
}

}  // namespace

namespace qaoa {
void set_last_error(const char *msg) { fail(QAOA_OK, msg); }
qaoa_status builtin_scratch(void **ptr, size_t *bytes);  // noalloc.cu
}  // namespace qaoa

// =================================================================== C ABI

extern "C" {

const char *qaoa_status_string(qaoa_status st) {
  switch (st) {
    case QAOA_OK: return "ok";
    case QAOA_ERR_INVALID_ARG: return "invalid argument";
    case QAOA_ERR_OUT_OF_MEMORY: return "buffer too small";
    case QAOA_ERR_OVERFLOW: return "integer cost overflow";
    case QAOA_ERR_CUDA: return "CUDA error";
    case QAOA_ERR_TIMEOUT: return "timeout";
    case QAOA_ERR_REJECTED: return "rejected";
    case QAOA_ERR_CANCELLED: return "cancelled";
    case QAOA_ERR_NOT_FOUND: return "not found";
    case QAOA_ERR_BUSY: return "busy";
  }
  return "unknown status";
}

const char *qaoa_last_error_message(void) { return g_errmsg; }

qaoa_status qaoa_workspace_check(void *d_work, size_t work_bytes, qaoa_stream_t stream) {
  if (!d_work && work_bytes == 0 && builtin_scratch(&d_work, &work_bytes) != QAOA_OK)
    return fail(QAOA_ERR_CUDA, "workspace check: cudaGetSymbolAddress of the built-in scratch failed");
  if (!d_work || work_bytes < kWsPartials) return fail(QAOA_ERR_INVALID_ARG, "bad workspace");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned h = 0;
  unsigned *err = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(d_work) + kWsCounters + 64);
  CK(cudaMemcpyAsync(&h, err, sizeof(h), cudaMemcpyDeviceToHost, s), "workspace check copy");
  CK(cudaStreamSynchronize(s), "workspace check sync");
  if (h != 0) {
    CK(cudaMemsetAsync(err, 0, sizeof(unsigned), s), "workspace check clear");
    return fail(QAOA_ERR_TIMEOUT, "a device-side wait ran out of time");
  }
  return QAOA_OK;
}

qaoa_status qaoa_selftest_timeout(void *d_work, size_t work_bytes, qaoa_stream_t stream) {
  if (!d_work && work_bytes == 0 && builtin_scratch(&d_work, &work_bytes) != QAOA_OK)
    return fail(QAOA_ERR_CUDA, "timeout self-test: cudaGetSymbolAddress of the built-in scratch failed");
  if (!d_work || work_bytes < kWsPartials) return fail(QAOA_ERR_INVALID_ARG, "bad workspace");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned *err = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(d_work) + kWsCounters + 64);
  CK(launch_wait_selftest(err, s), "wait self-test launch");
  return QAOA_OK;
}

int qaoa_version(void) { return 100; }

size_t qaoa_workspace_bytes(int n) {
  if (n < 1) n = 1;
  if (n > QAOA_MAX_N) n = QAOA_MAX_N;
  return kWsPartials + partial_doubles(n) * sizeof(double);
}

qaoa_status qaoa_labs_terms(int n, qaoa_term *out, size_t cap, size_t *n_out) {
  if (n < 1 || n > 64 || !n_out) return fail(QAOA_ERR_INVALID_ARG, "labs_terms: bad n or n_out");
  // sum_k C_k^2 = sum_k sum_{i,j} s_i s_{i+k} s_j s_{j+k}: the i == j parts give
  // the constant sum_k (n - k) = n(n-1)/2; every unordered product of four
  // distinct spins {i, i+k, j, j+k} (i < j, j != i + k) is a 4-body term and
  // products with j == i + k collapse to the 2-body term s_i s_{i+2k}.  Terms
  // with the same index set are merged.
  std::map<uint64_t, double> acc;  // ordered by mask: deterministic output
  auto add = [&](uint64_t mask, double w) { acc[mask] += w; };
  add(0, (double)n * (n - 1) / 2.0);
  for (int k = 1; k < n; ++k)
    for (int i = 0; i + k < n; ++i)
      for (int j = i + 1; j + k < n; ++j) {
        const uint64_t m = (1ull << i) ^ (1ull << (i + k)) ^ (1ull << j) ^ (1ull << (j + k));
        add(m, 2.0);  // ordered pairs (i, j) and (j, i)
      }
  size_t cnt = 0;
  for (auto &t : acc)
    if (t.second != 0.0) ++cnt;
  *n_out = cnt;
  if (cap < cnt) return fail(QAOA_ERR_OUT_OF_MEMORY, "labs_terms: cap too small");
  if (cnt && !out) return fail(QAOA_ERR_INVALID_ARG, "labs_terms: NULL out");
  size_t k = 0;
  for (auto &t : acc)
    if (t.second != 0.0) out[k++] = qaoa_term{t.second, t.first};
  return QAOA_OK;
}

qaoa_status qaoa_maxcut_terms(int n, const int32_t *edges, const double *w, size_t m,
                              qaoa_term *out, size_t cap, size_t *n_out) {
  if (n < 2 || n > 64 || !n_out || (m && !edges)) return fail(QAOA_ERR_INVALID_ARG, "maxcut_terms: bad arguments");
  double tot = 0.0;
  for (size_t e = 0; e < m; ++e) {
    const int i = edges[2 * e], j = edges[2 * e + 1];
    if (i < 0 || j < 0 || i >= n || j >= n || i == j) return fail(QAOA_ERR_INVALID_ARG, "maxcut_terms: bad edge");
    const double we = w ? w[e] : 1.0;
    if (!std::isfinite(we)) return fail(QAOA_ERR_INVALID_ARG, "maxcut_terms: non-finite weight");
    tot += we;
  }
  *n_out = m + 1;
  if (cap < m + 1) return fail(QAOA_ERR_OUT_OF_MEMORY, "maxcut_terms: cap too small");
  if (!out) return fail(QAOA_ERR_INVALID_ARG, "maxcut_terms: NULL out");
  for (size_t e = 0; e < m; ++e) {
    const double we = w ? w[e] : 1.0;
    out[e] = qaoa_term{0.5 * we, (1ull << edges[2 * e]) | (1ull << edges[2 * e + 1])};
  }
  out[m] = qaoa_term{-0.5 * tot, 0};
  return QAOA_OK;
}

qaoa_status qaoa_precompute_costs(int n, const qaoa_term *terms, size_t n_terms, qaoa_cost_type ct,
                                  void *d_costs, qaoa_stream_t stream) {
  if (n < 1 || n > QAOA_MAX_N) return fail(QAOA_ERR_INVALID_ARG, "n out of range");
  if (!valid_cost_type(ct) || !aligned16(d_costs)) return fail(QAOA_ERR_INVALID_ARG, "bad cost type or pointer");
  if (ct == QAOA_COST_U16)
    return fail(QAOA_ERR_INVALID_ARG, "precompute_costs: build int32 costs, then qaoa_convert_costs to uint16");
  if (n_terms && !terms) return fail(QAOA_ERR_INVALID_ARG, "NULL terms");
  const uint64_t lim = n == 64 ? ~0ull : ((1ull << n) - 1ull);
  std::vector<double> w(n_terms);
  for (size_t k = 0; k < n_terms; ++k) {
    if ((terms[k].mask & ~lim) != 0) return fail(QAOA_ERR_INVALID_ARG, "term mask has a bit >= n");
    if (!std::isfinite(terms[k].weight)) return fail(QAOA_ERR_INVALID_ARG, "non-finite weight");
    w[k] = terms[k].weight;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int nsm = num_sms();
  int mode;
  double scale = 1.0;
  int e_fix = 0;
  if (ct == QAOA_COST_I32) {
    double tot = 0.0;
    for (size_t k = 0; k < n_terms; ++k) {
      if (w[k] != nearbyint(w[k])) return fail(QAOA_ERR_INVALID_ARG, "I32 costs need integer weights");
      tot += fabs(w[k]);
    }
    if (!(tot < 2147483648.0)) return fail(QAOA_ERR_OVERFLOW, "sum |w| does not fit int32");
    mode = kTermI32;
  } else {
    if (dyadic_scale(w.data(), n_terms, &e_fix)) {
      mode = kTermFixed;
      scale = ldexp(1.0, e_fix);
    } else {
      mode = kTermF64;
    }
    if (ct == QAOA_COST_F32 && n_terms > (size_t)kTermChunk)
      return fail(QAOA_ERR_INVALID_ARG, "float32 costs take at most 1024 terms per call");
  }
  static TermChunk P;  // large parameter block; calls are serialised below
  static std::mutex *mu = new std::mutex();
  std::lock_guard<std::mutex> lock(*mu);
  const size_t nchunks = n_terms ? (n_terms + kTermChunk - 1) / kTermChunk : 1;
  for (size_t c = 0; c < nchunks; ++c) {
    memset(&P, 0, sizeof(P));
    P.n = n;
    P.mode = mode;
    P.out_kind = (int)ct;
    P.accumulate = c > 0;
    P.scale = scale;
    P.inv_scale = 1.0 / scale;
    P.out = d_costs;
    const size_t k0 = c * kTermChunk;
    const size_t k1 = (k0 + kTermChunk < n_terms) ? k0 + kTermChunk : n_terms;
    P.nterms = (int)(k1 - k0);
    for (size_t k = k0; k < k1; ++k) {
      P.mask[k - k0] = terms[k].mask;
      P.wd[k - k0] = w[k];
      P.wl[k - k0] = (int64_t)(mode == kTermFixed ? ldexp(w[k], e_fix) : w[k]);
    }
    LAUNCH("costs_terms", cost_bytes(ct) * (double)(1ull << n) * (c > 0 ? 2.0 : 1.0), s,
           launch_terms(P, s, nsm));
  }
  return QAOA_OK;
}

qaoa_status qaoa_labs_costs(int n, int32_t *d_costs, qaoa_stream_t stream) {
  if (n < 2 || n > 32) return fail(QAOA_ERR_INVALID_ARG, "labs_costs: n must be in [2, 32]");
  if (!aligned16(d_costs)) return fail(QAOA_ERR_INVALID_ARG, "labs_costs: bad pointer");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAUNCH("costs_labs", 4.0 * (double)(1ull << n), s, launch_labs(n, d_costs, s, num_sms()));
  return QAOA_OK;
}

qaoa_status qaoa_labs_costs_u16(int n, uint16_t *d_costs, qaoa_stream_t stream) {
  if (n < 2 || n > 32) return fail(QAOA_ERR_INVALID_ARG, "labs_costs_u16: n must be in [2, 32]");
  if (!aligned16(d_costs)) return fail(QAOA_ERR_INVALID_ARG, "labs_costs_u16: bad pointer");
  // max f = (n-1) n (2n-1) / 6 (all spins equal) < 2^16 for every n <= 32
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAUNCH("costs_labs", 2.0 * (double)(1ull << n), s, launch_labs_u16(n, d_costs, s, num_sms()));
  return QAOA_OK;
}

qaoa_status qaoa_convert_costs(int n, const void *d_src, qaoa_cost_type src_ct,
                               const qaoa_cost_stats *stats, void *d_dst, qaoa_cost_type dst_ct,
                               qaoa_stream_t stream) {
  if (n < 1 || n > QAOA_MAX_N || !aligned16(d_src) || !aligned16(d_dst) || !stats)
    return fail(QAOA_ERR_INVALID_ARG, "convert_costs: bad n, pointer or NULL stats");
  const bool to16 = src_ct == QAOA_COST_I32 && dst_ct == QAOA_COST_U16;
  const bool from16 = src_ct == QAOA_COST_U16 && dst_ct == QAOA_COST_I32;
  if (!to16 && !from16) return fail(QAOA_ERR_INVALID_ARG, "convert_costs: only int32 <-> uint16");
  if (to16 && !(stats->f_min >= 0.0 && stats->f_max <= 65535.0))
    return fail(QAOA_ERR_OVERFLOW, "convert_costs: values outside [0, 65535] (stats of the int32 vector)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAUNCH("costs_convert", (cost_bytes(src_ct) + cost_bytes(dst_ct)) * (double)(1ull << n), s,
         launch_convert(n, d_src, cost_kind(src_ct), d_dst, cost_kind(dst_ct), s, num_sms()));
  return QAOA_OK;
}

qaoa_status qaoa_maxcut_costs(int n, const int32_t *edges, const double *w, size_t m,
                              qaoa_cost_type ct, void *d_costs, qaoa_stream_t stream) {
  if (n < 2 || n > QAOA_MAX_N || !valid_cost_type(ct) || ct == QAOA_COST_U16 || !aligned16(d_costs))
    return fail(QAOA_ERR_INVALID_ARG, "maxcut_costs: bad n, type or pointer (uint16: convert from int32)");
  if (m > (size_t)kEdgeMax || (m && !edges)) return fail(QAOA_ERR_INVALID_ARG, "maxcut_costs: too many edges or NULL");
  std::vector<double> wv(m);
  for (size_t e = 0; e < m; ++e) {
    const int i = edges[2 * e], j = edges[2 * e + 1];
    if (i < 0 || j < 0 || i >= n || j >= n || i == j) return fail(QAOA_ERR_INVALID_ARG, "maxcut_costs: bad edge");
    wv[e] = w ? w[e] : 1.0;
    if (!std::isfinite(wv[e])) return fail(QAOA_ERR_INVALID_ARG, "maxcut_costs: non-finite weight");
  }
  static EdgeChunk P;
  static std::mutex *mu = new std::mutex();
  std::lock_guard<std::mutex> lock(*mu);
  memset(&P, 0, sizeof(P));
  P.n = n;
  P.m = (int)m;
  P.out_kind = (int)ct;
  P.out = d_costs;
  int e2 = 0;
  if (ct == QAOA_COST_I32) {
    double tot = 0.0;
    for (size_t e = 0; e < m; ++e) {
      if (wv[e] != nearbyint(wv[e])) return fail(QAOA_ERR_INVALID_ARG, "I32 costs need integer weights");
      tot += fabs(wv[e]);
    }
    if (!(tot < 2147483648.0)) return fail(QAOA_ERR_OVERFLOW, "sum |w| does not fit int32");
    P.mode = kTermI32;
  } else if (dyadic_scale(wv.data(), m, &e2)) {
    P.mode = kTermFixed;
    P.inv_scale = ldexp(1.0, -e2);
  } else {
    P.mode = kTermF64;
  }
  for (size_t e = 0; e < m; ++e) {
    P.ei[e] = (uint8_t)edges[2 * e];
    P.ej[e] = (uint8_t)edges[2 * e + 1];
    P.wd[e] = wv[e];
    P.wl[e] = (int64_t)(P.mode == kTermFixed ? ldexp(wv[e], e2) : wv[e]);
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAUNCH("costs_maxcut", cost_bytes(ct) * (double)(1ull << n), s, launch_maxcut(P, s, num_sms()));
  return QAOA_OK;
}

qaoa_status qaoa_cost_stats_compute(int n, const void *d_costs, qaoa_cost_type ct, void *d_work,
                                    size_t work_bytes, qaoa_cost_stats *h_out, qaoa_stream_t stream) {
  if (n < 1 || n > QAOA_MAX_N || !valid_cost_type(ct) || !aligned16(d_costs) || !h_out)
    return fail(QAOA_ERR_INVALID_ARG, "cost_stats: bad arguments");
  Ws ws;
  qaoa_status st = get_ws(n, d_work, work_bytes, ws);
  if (st != QAOA_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CK(cudaMemsetAsync(ws.counter, 0, sizeof(unsigned), s), "memset counter");
  LAUNCH("cost_stats", cost_bytes(ct) * (double)(1ull << n), s,
         launch_cost_stats(n, d_costs, cost_kind(ct), ws.partials, ws.counter, ws.small, s, num_sms()));
  double h[4];
  CK(cudaMemcpyAsync(h, ws.small, sizeof(h), cudaMemcpyDeviceToHost, s), "cost stats copy");
  CK(cudaStreamSynchronize(s), "cost stats sync");
  h_out->f_min = h[0];
  h_out->f_max = h[1];
  h_out->n_min = (uint64_t)h[2];
  const uint32_t bits = (uint32_t)h[3];
  h_out->step_log2 = bits ? (uint32_t)__builtin_ctz(bits) : 0u;
  h_out->reserved = 0u;
  return QAOA_OK;
}

qaoa_status qaoa_simulate(int n, const void *d_costs, qaoa_cost_type ct, const qaoa_cost_stats *stats,
                          const double *gammas, const double *betas, int p, void *d_state,
                          qaoa_state_type st, int init_plus, void *d_work, size_t work_bytes,
                          double *d_out, qaoa_stream_t stream) {
  qaoa_status r = check_common(n, d_costs, ct, d_state, st);
  if (r != QAOA_OK) return r;
  if (!stats) return fail(QAOA_ERR_INVALID_ARG, "NULL stats");
  r = check_angles(gammas, betas, p);
  if (r != QAOA_OK) return r;
  if (d_out && ((uintptr_t)d_out & 7u)) return fail(QAOA_ERR_INVALID_ARG, "d_out not 8-byte aligned");
  Ws ws;
  r = get_ws(n, d_work, work_bytes, ws);
  if (r != QAOA_OK) return r;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n <= kSmallMaxN) {
    return st == QAOA_C64
               ? small_forward<float>(n, d_costs, ct, stats->f_min, gammas, betas, p, d_state, init_plus, d_out, s)
               : small_forward<double>(n, d_costs, ct, stats->f_min, gammas, betas, p, d_state, init_plus, d_out, s);
  }
  CK(cudaMemsetAsync(ws.err, 0, sizeof(unsigned), s), "memset error word");
  if (st == QAOA_C64 && tma_ok(ct))
    return tma_forward(n, d_costs, ct, stats, gammas, betas, p, d_state, init_plus, ws, d_out, true, s);
  return st == QAOA_C64
             ? tiled_forward<float>(n, d_costs, ct, stats, gammas, betas, p, d_state, init_plus, ws, d_out, s)
             : tiled_forward<double>(n, d_costs, ct, stats, gammas, betas, p, d_state, init_plus, ws, d_out, s);
}

// ------------------------------------------------------------- XY mixers

struct XyOp {
  bool tile;      // a tile pass, else one gate over the whole state
  int tb, c, h;   // tile geometry
  std::vector<std::pair<int, int>> gates;  // qubit pairs, in order
};

std::vector<std::pair<int, int>> xy_edges(int n, int graph) {
  std::vector<std::pair<int, int>> e;
  if (graph == QAOA_XY_RING) {
    for (int q = 0; q + 1 < n; ++q) e.push_back({q, q + 1});
    if (n >= 3) e.push_back({n - 1, 0});
  } else {
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) e.push_back({i, j});
  }
  return e;
}

// Packs the ordered edge list into passes: consecutive gates share a tile
// while both qubits of each lie in it (passengers 0..c-1 or rows h..h+W-1).
std::vector<XyOp> xy_schedule(int n, const std::vector<std::pair<int, int>> &edges) {
  const int TB = n < kXyMaxTb ? n : kXyMaxTb;
  const int c = n <= kXyMaxTb ? n : 4, W = TB - c;
  std::vector<XyOp> ops;
  auto fits = [&](const XyOp &o, int q) { return q < o.c || (q >= o.h && q < o.h + o.tb - o.c); };
  for (const auto &e : edges) {
    if (!ops.empty() && ops.back().tile && (int)ops.back().gates.size() < kXyMaxGates &&
        fits(ops.back(), e.first) && fits(ops.back(), e.second)) {
      ops.back().gates.push_back(e);
      continue;
    }
    XyOp o;
    o.tile = true;
    o.tb = TB;
    if (e.first < TB && e.second < TB) {  // the contiguous low tile
      o.c = TB;
      o.h = TB;
    } else {
      int a = e.first, b = e.second;
      if (a > b) std::swap(a, b);
      const int lo = a < c ? b : a;  // lowest qubit that must sit in a row
      if (a >= c && b - a >= W) {
        o.tile = false;  // no tile holds both: one gate over the state
      } else {
        o.c = c;
        o.h = lo < n - W ? lo : n - W;
      }
    }
    o.gates.push_back(e);
    ops.push_back(o);
  }
  return ops;
}

// The pair rotation by beta as three shears: beta reduced to [-pi/2, pi/2]
// (a rotation by pi is the exact factor -1).
void xy_beta(double beta, double &tb2, double &sb, int &neg) {
  double br = std::remainder(beta, kTwoPi);  // (-pi, pi]
  neg = 0;
  if (br > kTwoPi / 4) {
    br -= kTwoPi / 2;
    neg = 1;
  } else if (br < -kTwoPi / 4) {
    br += kTwoPi / 2;
    neg = 1;
  }
  tb2 = std::tan(br / 2);
  sb = std::sin(br);
}

// One pass of the TMA ring schedule (XyTmaParams).
struct XyTmaOp {
  bool low;
  int h;
  uint32_t em[3];
  int wrap;
};

// The ring's chain of gates (0,1), (1,2), ..., (n-2, n-1), (n-1, 0) over
// passes of 2^13-amplitude tiles: the LOW pass (qubits 0..12, tile bit =
// qubit) takes (0,1)..(11,12) in rounds over tile bits 0-4, 4-8, 8-12; each
// HIGH pass (16 contiguous amplitudes x rows h..h+8 at tile bits 4..12) the
// next up to 8 gates in rounds over tile bits 4-8, 8-12; the last pass ends
// with (n-1, 0) (tile bits 12, 0).  LABS n = 28: 3 passes per layer.
std::vector<XyTmaOp> xy_ring_tma_schedule(int n) {
  std::vector<XyTmaOp> ops;
  ops.push_back(XyTmaOp{true, 4, {0xF, 0xF, 0xF}, 0});
  for (int q = 12; q <= n - 2;) {
    const int h = q < n - 9 ? q : n - 9;
    const int last = std::min(h + 7, n - 2);
    XyTmaOp o{false, h, {0, 0, 0}, 0};
    for (int qq = q; qq <= last; ++qq) {
      const int a = qq - h + 4;  // the gate's tile bits (a, a + 1), 4 <= a <= 11
      if (a + 1 <= 8)
        o.em[0] |= 1u << (a - 4);
      else
        o.em[1] |= 1u << (a - 8);
    }
    ops.push_back(o);
    q = last + 1;
  }
  ops.back().wrap = 1;
  return ops;
}

qaoa_status xy_ring_tma(int n, const void *cost, qaoa_cost_type ct, const qaoa_cost_stats *stats,
                        const double *gammas, const double *betas, int p, void *state, const Ws &ws,
                        cudaStream_t s) {
  const std::vector<XyTmaOp> ops = xy_ring_tma_schedule(n);
  const int nsm = num_sms();
  const double N = (double)(1ull << n);
  static XyTmaParams P;
  static std::mutex *mu = new std::mutex();
  std::lock_guard<std::mutex> lock(*mu);
  for (int l = 0; l < p; ++l) {
    double tb2, sb;
    int neg;
    xy_beta(betas[l], tb2, sb, neg);
    for (const XyTmaOp &o : ops) {
      memset(&P, 0, sizeof(P));
      CK(make_tile_map(&P.map_psi, state, n, 13, o.h, 4, 8, 128), "tensor map (XY state)");
      CK(make_tile_map(&P.map_cost, const_cast<void *>(cost), n, 13, o.h, 4, (int)cost_bytes(ct), 0),
         "tensor map (XY cost)");
      P.psi = reinterpret_cast<float2 *>(state);
      P.ntiles = 1ull << (n - 13);
      P.h = o.h;
      P.c = 4;
      P.cost_kind = cost_kind(ct);
      P.has_phase = o.low;  // the layer's phase opens its first pass
      if (P.has_phase) make_phase(P.ph, gammas[l], ct, stats, 1.0);
      for (int r = 0; r < 3; ++r) P.em[r] = o.em[r];
      P.wrap = o.wrap;
      P.t = (float)tb2;
      P.s = (float)sb;
      P.neg = neg;
      P.err = ws.err;
      LAUNCH("xy_tile", 16.0 * N + (P.has_phase ? cost_bytes(ct) * N : 0.0), s,
             ct == QAOA_COST_U16 ? launch_xy_tma_u16(P, o.low, s, nsm) : launch_xy_tma(P, o.low, s, nsm));
    }
  }
  return QAOA_OK;
}

qaoa_status qaoa_simulate_xy(int n, const void *d_costs, qaoa_cost_type ct, const qaoa_cost_stats *stats,
                             const double *gammas, const double *betas, int p, int graph, void *d_state,
                             qaoa_state_type st, void *d_work, size_t work_bytes, double *d_out,
                             qaoa_stream_t stream) {
  if (n < 2) return fail(QAOA_ERR_INVALID_ARG, "simulate_xy: n must be >= 2");
  qaoa_status r = check_common(n, d_costs, ct, d_state, st);
  if (r != QAOA_OK) return r;
  if (graph != QAOA_XY_RING && graph != QAOA_XY_COMPLETE) return fail(QAOA_ERR_INVALID_ARG, "simulate_xy: bad graph");
  r = check_angles(gammas, betas, p);
  if (r != QAOA_OK) return r;
  if (d_out && (((uintptr_t)d_out & 7u) || !stats)) return fail(QAOA_ERR_INVALID_ARG, "simulate_xy: d_out needs stats and 8-byte alignment");
  Ws ws;
  r = get_ws(n, d_work, work_bytes, ws);
  if (r != QAOA_OK) return r;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool c128 = st == QAOA_C128;
  const int nsm = num_sms();
  const double N = (double)(1ull << n), es = c128 ? 16.0 : 8.0;
  if (!c128 && graph == QAOA_XY_RING && n >= 13 && tma_ok(ct)) {
    // complex64 ring: register rounds on TMA-streamed tiles
    r = xy_ring_tma(n, d_costs, ct, stats, gammas, betas, p, d_state, ws, s);
    if (r != QAOA_OK) return r;
    if (d_out) {
      CK(cudaMemsetAsync(ws.counter, 0, sizeof(unsigned), s), "memset counter");
      LAUNCH("expect", (es + cost_bytes(ct)) * N, s,
             launch_expect(n, d_state, c128, d_costs, cost_kind(ct), stats->f_min, ws.partials,
                           ws.counter, d_out, 2, s, nsm));
    }
    return QAOA_OK;
  }
  std::vector<XyOp> ops = xy_schedule(n, xy_edges(n, graph));
  if (ops.empty() || !ops.front().tile) {  // the phase rides on a tile pass
    XyOp o;
    o.tile = true;
    o.tb = n < kXyMaxTb ? n : kXyMaxTb;
    o.c = o.tb;
    o.h = o.tb;
    ops.insert(ops.begin(), o);
  }
  static XyPass P;
  static std::mutex *mu = new std::mutex();
  std::lock_guard<std::mutex> lock(*mu);
  for (int l = 0; l < p; ++l) {
    // the pair rotation by beta as three shears: beta reduced to [-pi/2, pi/2]
    // (a rotation by pi is the exact factor -1)
    double tb2, sb;
    int neg;
    xy_beta(betas[l], tb2, sb, neg);
    const double g2 = gammas[l] / kTwoPi;
    for (size_t k = 0; k < ops.size(); ++k) {
      const XyOp &o = ops[k];
      if (!o.tile) {
        LAUNCH("xy_gate", es * N, s,
               launch_xy_gate(d_state, c128, n, o.gates[0].first, o.gates[0].second, tb2, sb, neg, s,
                              nsm));
        continue;
      }
      memset(&P, 0, sizeof(P));
      P.psi = d_state;
      P.cost = d_costs;
      P.cost_kind = cost_kind(ct);
      P.tb = o.tb;
      P.c = o.c;
      P.h = o.h;
      P.ntiles = 1ull << (n - o.tb);
      P.has_phase = k == 0;
      P.g2pi = g2;
      P.g_hi = (float)g2;
      P.g_lo = (float)(g2 - (double)P.g_hi);
      if (P.has_phase && !c128) make_phase(P.ph, gammas[l], ct, stats, 1.0);  // tables or computed
      else P.ph.mode = 1;
      P.tb2 = tb2;
      P.sb = sb;
      P.neg = neg;
      P.ngates = (int)o.gates.size();
      auto tbit = [&](int q) { return q < o.c ? q : o.c + (q - o.h); };
      for (int g = 0; g < P.ngates; ++g) {
        P.ga[g] = (uint8_t)tbit(o.gates[g].first);
        P.gb[g] = (uint8_t)tbit(o.gates[g].second);
      }
      LAUNCH("xy_tile", 2.0 * es * N + (P.has_phase ? cost_bytes(ct) * N : 0.0), s,
             launch_xy_tile(P, c128, s, nsm));
    }
  }
  if (d_out) {
    CK(cudaMemsetAsync(ws.counter, 0, sizeof(unsigned), s), "memset counter");
    LAUNCH("expect", (es + cost_bytes(ct)) * N, s,
           launch_expect(n, d_state, c128, d_costs, cost_kind(ct), stats->f_min, ws.partials,
                         ws.counter, d_out, 2, s, nsm));
  }
  return QAOA_OK;
}

qaoa_status qaoa_dicke_state(int n, int k, void *d_state, qaoa_state_type st, qaoa_stream_t stream) {
  if (n < 1 || n > QAOA_MAX_N || k < 0 || k > n || !valid_state_type(st) || !aligned16(d_state))
    return fail(QAOA_ERR_INVALID_ARG, "dicke_state: bad n, k, state type or pointer");
  double cnk = 1.0;  // C(n, k), exact in float64 for n <= 34
  for (int i = 1; i <= k; ++i) cnk = cnk * (n - k + i) / i;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAUNCH("dicke", (st == QAOA_C128 ? 16.0 : 8.0) * (double)(1ull << n), s,
         launch_dicke(d_state, st == QAOA_C128, n, k, 1.0 / std::sqrt(cnk), s, num_sms()));
  return QAOA_OK;
}

qaoa_status qaoa_probabilities(int n, void *d_state, qaoa_state_type st, void *d_probs,
                               qaoa_stream_t stream) {
  if (n < 1 || n > QAOA_MAX_N || !valid_state_type(st) || !aligned16(d_state))
    return fail(QAOA_ERR_INVALID_ARG, "probabilities: bad n, state type or pointer");
  if (d_probs && ((uintptr_t)d_probs & 15u)) return fail(QAOA_ERR_INVALID_ARG, "probabilities: misaligned d_probs");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const double es = st == QAOA_C128 ? 16.0 : 8.0;
  LAUNCH("probabilities", (es + (d_probs ? es / 2.0 : es)) * (double)(1ull << n), s,
         launch_probs(n, d_state, st == QAOA_C128, d_probs, s, num_sms()));
  return QAOA_OK;
}

qaoa_status qaoa_expectation(int n, const void *d_state, qaoa_state_type st, const void *d_costs,
                             qaoa_cost_type ct, void *d_work, size_t work_bytes, double *d_out,
                             qaoa_stream_t stream) {
  qaoa_status r = check_common(n, d_costs, ct, d_state, st);
  if (r != QAOA_OK) return r;
  if (!d_out) return fail(QAOA_ERR_INVALID_ARG, "NULL d_out");
  Ws ws;
  r = get_ws(n, d_work, work_bytes, ws);
  if (r != QAOA_OK) return r;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CK(cudaMemsetAsync(ws.counter, 0, sizeof(unsigned), s), "memset counter");
  LAUNCH("expect", ((st == QAOA_C128 ? 16.0 : 8.0) + cost_bytes(ct)) * (double)(1ull << n), s,
         launch_expect(n, d_state, st == QAOA_C128, d_costs, cost_kind(ct), 0.0, ws.partials,
                       ws.counter, d_out, 0, s, num_sms()));
  return QAOA_OK;
}

qaoa_status qaoa_overlap(int n, const void *d_state, qaoa_state_type st, const void *d_costs,
                         qaoa_cost_type ct, const qaoa_cost_stats *stats, void *d_work,
                         size_t work_bytes, double *d_out, qaoa_stream_t stream) {
  qaoa_status r = check_common(n, d_costs, ct, d_state, st);
  if (r != QAOA_OK) return r;
  if (!d_out || !stats) return fail(QAOA_ERR_INVALID_ARG, "NULL d_out or stats");
  Ws ws;
  r = get_ws(n, d_work, work_bytes, ws);
  if (r != QAOA_OK) return r;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CK(cudaMemsetAsync(ws.counter, 0, sizeof(unsigned), s), "memset counter");
  LAUNCH("expect", ((st == QAOA_C128 ? 16.0 : 8.0) + cost_bytes(ct)) * (double)(1ull << n), s,
         launch_expect(n, d_state, st == QAOA_C128, d_costs, cost_kind(ct), stats->f_min,
                       ws.partials, ws.counter, d_out, 1, s, num_sms()));
  return QAOA_OK;
}

qaoa_status qaoa_grad(int n, const void *d_costs, qaoa_cost_type ct, const qaoa_cost_stats *stats,
                      const double *gammas, const double *betas, int p, void *d_state, void *d_lambda,
                      qaoa_state_type st, void *d_work, size_t work_bytes, double *d_out,
                      qaoa_stream_t stream) {
  qaoa_status r = check_common(n, d_costs, ct, d_state, st);
  if (r != QAOA_OK) return r;
  if (!aligned16(d_lambda)) return fail(QAOA_ERR_INVALID_ARG, "lambda pointer NULL or not 16-byte aligned");
  if (!stats || !d_out || ((uintptr_t)d_out & 7u)) return fail(QAOA_ERR_INVALID_ARG, "NULL stats or bad d_out");
  r = check_angles(gammas, betas, p);
  if (r != QAOA_OK) return r;
  Ws ws;
  r = get_ws(n, d_work, work_bytes, ws);
  if (r != QAOA_OK) return r;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n <= kSmallMaxN) {
    return st == QAOA_C64
               ? small_grad<float>(n, d_costs, ct, stats->f_min, gammas, betas, p, d_state, d_lambda, d_out, s)
               : small_grad<double>(n, d_costs, ct, stats->f_min, gammas, betas, p, d_state, d_lambda, d_out, s);
  }
  CK(cudaMemsetAsync(d_out + 2, 0, sizeof(double) * 2 * (size_t)p, s), "memset grad");
  CK(cudaMemsetAsync(ws.err, 0, sizeof(unsigned), s), "memset error word");
  if (st == QAOA_C64 && tma_ok(ct)) {
    r = tma_forward(n, d_costs, ct, stats, gammas, betas, p, d_state, 1, ws, d_out, false, s);
    if (r != QAOA_OK) return r;
    return tma_backward(n, d_costs, ct, stats, gammas, betas, p, d_state, d_lambda, ws, d_out + 2,
                        d_out + 2 + p, s);
  }
  r = st == QAOA_C64
          ? tiled_forward<float>(n, d_costs, ct, stats, gammas, betas, p, d_state, 1, ws, d_out, s)
          : tiled_forward<double>(n, d_costs, ct, stats, gammas, betas, p, d_state, 1, ws, d_out, s);
  if (r != QAOA_OK) return r;
  return st == QAOA_C64
             ? tiled_backward<float>(n, d_costs, ct, stats, gammas, betas, p, d_state, d_lambda, ws,
                                     d_out + 2, d_out + 2 + p, s)
             : tiled_backward<double>(n, d_costs, ct, stats, gammas, betas, p, d_state, d_lambda, ws,
                                      d_out + 2, d_out + 2 + p, s);
}

}  // extern "C"
