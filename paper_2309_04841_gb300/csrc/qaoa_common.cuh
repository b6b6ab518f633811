// qaoa_common.cuh -- device helpers, tile plans and kernel parameter blocks
// shared by the kernels and the host planner of the sm_103a QAOA library.
//
// A "pass" streams the whole state vector through the SMs once.  The state
// is cut into tiles of 2^TB amplitudes; tile bit j maps to basis-index bit
//   j            for j <  c   (low segment: contiguous, gives coalescing)
//   h + (j - c)  for j >= c   (high segment: any run of qubits)
// so a pass can rotate any TB-qubit window (Algorithm 1 on each of them)
// while every global access still moves whole 2^c-amplitude segments.
// Inside a tile each thread holds 2^EB amplitudes in registers; a "round"
// assigns EB tile bits to registers, 5 to lanes and the rest to warps, and
// smem transposes move between rounds.  Rotations of register bits need no
// data movement at all.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qaoa {

template <typename R> struct C2T;
template <> struct C2T<float> { using type = float2; };
template <> struct C2T<double> { using type = double2; };

// Scatter the low bits of v into the set bits of mask (parallel bit deposit).
__host__ __device__ constexpr uint32_t pdep(uint32_t v, uint32_t mask) {
  uint32_t out = 0;
  int k = 0;
  for (int b = 0; b < 32; ++b) {
    if ((mask >> b) & 1u) {
      if ((v >> k) & 1u) out |= 1u << b;
      ++k;
    }
  }
  return out;
}

__host__ __device__ constexpr int popc_c(uint32_t m) {
  int c = 0;
  for (int b = 0; b < 32; ++b) c += (m >> b) & 1u;
  return c;
}

__host__ __device__ constexpr int log2_c(int v) { return v <= 1 ? 0 : 1 + log2_c(v >> 1); }

// Tile plan: TB tile bits, 2^EB registers per thread, NT threads, NR rounds
// given as (register, lane, warp) masks over tile bits; smem slot swizzle
// s = t ^ ((t >> SWS) & m) with m = 15 for 8-byte and 7 for 16-byte
// amplitudes, chosen so every round's smem access pattern is bank-conflict
// free (each half-warp / quarter-warp hits distinct 128-byte bank rows).
template <int TB_, int EB_, int NT_, int SWS_, int NR_, uint32_t R0, uint32_t L0,
          uint32_t W0, uint32_t R1, uint32_t L1, uint32_t W1, uint32_t R2 = 0,
          uint32_t L2 = 0, uint32_t W2 = 0>
struct Plan {
  static constexpr int TB = TB_, EB = EB_, NT = NT_, SWS = SWS_, NR = NR_;
  static constexpr int NREG = 1 << EB_;
  __host__ __device__ static constexpr uint32_t reg(int r) { return r == 0 ? R0 : r == 1 ? R1 : R2; }
  __host__ __device__ static constexpr uint32_t lane(int r) { return r == 0 ? L0 : r == 1 ? L1 : L2; }
  __host__ __device__ static constexpr uint32_t warp(int r) { return r == 0 ? W0 : r == 1 ? W1 : W2; }
  __host__ __device__ static constexpr bool valid_round(int r) {
    return popc_c(reg(r)) == EB && popc_c(lane(r)) == 5 &&
           popc_c(warp(r)) == log2_c(NT / 32) && (reg(r) & lane(r)) == 0 &&
           (reg(r) & warp(r)) == 0 && (lane(r) & warp(r)) == 0 &&
           (reg(r) | lane(r) | warp(r)) == ((1u << TB) - 1u);
  }
  __host__ __device__ static constexpr bool valid() {
    return (1 << TB) == NT * NREG && valid_round(0) && valid_round(1) &&
           (NR < 3 || valid_round(2)) && (lane(0) & 0x1Fu) == 0x1Fu;
  }
};

// complex64 forward: 8192-amplitude tiles (64 KB), 32 amplitudes/thread.
using PlanF13Low = Plan<13, 5, 256, 5, 3, 0x1F00, 0x001F, 0x00E0,
                        0x001F, 0x03E0, 0x1C00, 0x03E0, 0x001F, 0x1C00>;
using PlanF13High = Plan<13, 5, 256, 5, 2, 0x1F00, 0x001F, 0x00E0,
                         0x01F0, 0x020F, 0x1C00>;
// 4096-amplitude tiles, 16 amplitudes/thread: complex64 adjoint (two
// vectors, 64 KB) and complex128 forward (64 KB).
using PlanT12Low = Plan<12, 4, 256, 4, 3, 0x0F00, 0x001F, 0x00E0,
                        0x000F, 0x01F0, 0x0E00, 0x00F0, 0x010F, 0x0E00>;
using PlanT12High = Plan<12, 4, 256, 4, 2, 0x0F00, 0x001F, 0x00E0,
                         0x00F0, 0x010F, 0x0E00>;
// 2048-amplitude tiles, 16 amplitudes/thread: complex128 adjoint.
using PlanT11Low = Plan<11, 4, 128, 4, 3, 0x0780, 0x001F, 0x0060,
                        0x000F, 0x01F0, 0x0600, 0x00F0, 0x010F, 0x0600>;
using PlanT11High = Plan<11, 4, 128, 4, 2, 0x0780, 0x001F, 0x0060,
                         0x00F0, 0x010F, 0x0600>;

// 1024- and 512-amplitude tiles for complex128 at n <= 16 / n <= 14: the
// same number of groups as the 4096-amplitude tiles there, but 4-8 times as
// many CTAs for the FP64-bound rotations.
using PlanT10Low = Plan<10, 4, 64, 4, 3, 0x03C0, 0x001F, 0x0020,
                        0x000F, 0x01F0, 0x0200, 0x00F0, 0x010F, 0x0200>;
using PlanT10High = Plan<10, 4, 64, 4, 2, 0x03C0, 0x001F, 0x0020,
                         0x00F0, 0x010F, 0x0200>;
using PlanT9Low = Plan<9, 4, 32, 4, 3, 0x01E0, 0x001F, 0x0000,
                       0x000F, 0x01F0, 0x0000, 0x00F0, 0x010F, 0x0000>;
using PlanT9High = Plan<9, 4, 32, 4, 2, 0x01E0, 0x001F, 0x0000,
                        0x00F0, 0x010F, 0x0000>;

static_assert(PlanF13Low::valid() && PlanF13High::valid(), "bad F13 plan");
static_assert(PlanT10Low::valid() && PlanT10High::valid(), "bad T10 plan");
static_assert(PlanT9Low::valid() && PlanT9High::valid(), "bad T9 plan");
static_assert(PlanT12Low::valid() && PlanT12High::valid(), "bad T12 plan");
static_assert(PlanT11Low::valid() && PlanT11High::valid(), "bad T11 plan");

// Passenger (low-segment) bits of a HIGH pass: 2^4 contiguous amplitudes
// (128 B for complex64, 256 B for complex128) per global segment.
constexpr int kHighC = 4;

enum CostKind : int { kCostI32 = 0, kCostF32 = 1, kCostF64 = 2, kCostU16 = 3 };

// Tile geometry of one pass (see file comment).
struct Geom {
  int n, c, h, tb;
  uint64_t ntiles;
};

__device__ __forceinline__ uint64_t tile_base(const Geom &g, uint64_t T) {
  const int mid = g.h - g.c;  // outer bits between the two segments
  const uint64_t lo = T & ((1ull << mid) - 1ull);
  const uint64_t hi = T >> mid;
  return (lo << g.c) | (hi << (g.h + g.tb - g.c));
}

__device__ __forceinline__ uint64_t tile_off(const Geom &g, uint32_t t) {
  return (uint64_t)(t & ((1u << g.c) - 1u)) + ((uint64_t)(t >> g.c) << g.h);
}

// Rotation schedule of one sweep: for round r, bit i of m[r] says "rotate
// register bit i in this round" and bit i of lm[r] "rotate the tile bit held
// by lane-index bit i, with a warp shuffle" (TMA kernels only).
struct Sweep {
  uint8_t m[4];
  uint8_t lm[4];
};

// ------------------------------------------------------------ parameters
// Per-layer phase data.  Integer costs use a two-level table
// exp(-i g (fmin + 256 hi + lo)) = T_hi[hi] * T_lo[lo] built on the host in
// float64; other costs use a float-float reduction of g f / (2 pi).
template <typename Real>
struct PhaseData {
  using C2 = typename C2T<Real>::type;
  int mode;     // 0: table (integer costs), 1: computed
  int fmin;     // table origin
  int nhi;      // entries of T_hi in use
  float g_hi, g_lo;  // complex64 computed mode: g / 2pi = g_hi + g_lo
  double g2pi;       // complex128 computed mode: g / 2pi
  Real scl;          // computed mode: factor applied with the phase (tables carry it in T_hi)
  C2 tab_lo[256];
  C2 tab_hi[256];
};

template <typename Real>
struct FwdParams {
  using C2 = typename C2T<Real>::type;
  C2 *psi;
  const void *cost;
  int cost_kind;
  Geom g;
  Sweep s1, s2;         // s1 before the phase, s2 after
  // the sweeps' rotations in reduced form (rot_tan): multiplier and form;
  // the state is stored divided by the product of the dropped factors, which
  // the host folds into the next phase or into post_scale
  Real t1, t2;
  int form1, form2;
  Real post_scale;      // the pass's result times this before the reduction and the store
  int has_phase;
  int init_plus;        // ignore psi, start from |+>
  Real amp;             // 2^{-n/2}
  int reduce;           // fused energy/overlap in the final layout
  double fmin_d;        // ground-state value for the overlap
  double *partials;     // [ntiles][2]
  unsigned *counter;
  double *out;          // [2]: E, O
  PhaseData<Real> ph;
};

template <typename Real>
struct BwdParams {
  using C2 = typename C2T<Real>::type;
  C2 *psi, *lam;
  const void *cost;
  int cost_kind;
  Geom g;
  Sweep s1, s2;
  Real t1, t2;            // un-rotations in reduced form (rot_tan of -beta)
  int form1, form2;
  // psi and lambda are stored divided by a common real factor sigma; a raw
  // inner product is the true one divided by sigma^2, so each round's sum is
  // weighted by that round's sigma^2 (w1 / w2 per round, wg for the phase)
  Real w1[3], w2[3], wg;
  Real post_scale;        // psi and lambda times this before the store
  int has_phase;          // g_gamma accumulation + un-phase between sweeps
  int init_lambda;        // lambda <- f psi at load
  double *partials;       // [ntiles][3]
  unsigned *counter;
  double *out_b1, *out_g, *out_b2;  // gradient slots (accumulated: +=)
  PhaseData<Real> ph;     // un-phase data (exp(+i g f))
};

// Per-layer data of the single-CTA small-n kernels.
template <typename Real>
struct SmallLayer {
  Real cb, sb;        // cos(beta), sin(beta)
  float g_hi, g_lo;   // g / 2pi split (complex64)
  double g2pi;        // g / 2pi (complex128)
};

constexpr int kSmallMaxN = 12;

// One request for the on-chip kernels (a launch of k_small runs one, a launch
// of k_small_batch runs one per CTA from a device array of these).
template <typename Real>
struct SmallJob {
  using C2 = typename C2T<Real>::type;
  C2 *psi, *lam;
  const void *cost;
  int cost_kind;
  int n, nl;        // qubits; layers in this launch
  int mode;         // 0 forward, 1 forward + adjoint, 2 adjoint only
  int init_plus, init_lambda, reduce;
  Real amp;
  double fmin_d;
  double *out;              // [E, O]
  double *out_dg, *out_db;  // per-layer gradient outputs
  const SmallLayer<Real> *L;
};
constexpr int kSmallMaxLayers = 128;

template <typename Real>
struct SmallParams {
  using C2 = typename C2T<Real>::type;
  C2 *psi, *lam;
  const void *cost;
  int cost_kind;
  int n, nl;        // layers in this launch
  int mode;         // 0 forward, 1 forward + backward (grad), 2 backward only
  int init_plus, init_lambda, reduce;
  Real amp;
  double fmin_d;
  double *out;      // forward: [E, O]; grad: also gamma/beta slots below
  double *out_dg, *out_db;  // per-layer gradient outputs for this launch
  SmallLayer<Real> L[kSmallMaxLayers];
};

}  // namespace qaoa
