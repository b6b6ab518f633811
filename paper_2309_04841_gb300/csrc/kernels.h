// kernels.h -- launcher declarations between the host planner (api.cu) and
// the kernel translation units.  Internal to the library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "qaoa_common.cuh"

namespace qaoa {


enum TermMode : int { kTermI32 = 0, kTermFixed = 1, kTermF64 = 2 };

constexpr int kTermChunk = 1024;  // terms per launch (parameter block)
constexpr int kEdgeMax = 1536;    // edges per MaxCut launch (parameter block)

struct TermChunk {
  int n, nterms, mode, out_kind, accumulate;
  double scale, inv_scale;  // fixed mode: weights are wl * inv_scale
  void *out;
  uint64_t mask[kTermChunk];
  int64_t wl[kTermChunk];
  double wd[kTermChunk];
};

struct EdgeChunk {
  int n, m, mode, out_kind;
  double inv_scale;
  void *out;
  uint8_t ei[kEdgeMax], ej[kEdgeMax];
  int64_t wl[kEdgeMax];
  double wd[kEdgeMax];
};

cudaError_t launch_terms(const TermChunk &P, cudaStream_t s, int nsm);
cudaError_t launch_labs(int n, int32_t *out, cudaStream_t s, int nsm);
cudaError_t launch_labs_u16(int n, uint16_t *out, cudaStream_t s, int nsm);
cudaError_t launch_probs(int n, void *psi, bool c128, void *out, cudaStream_t s, int nsm);
cudaError_t launch_convert(int n, const void *src, int src_kind, void *dst, int dst_kind,
                           cudaStream_t s, int nsm);
cudaError_t launch_maxcut(const EdgeChunk &P, cudaStream_t s, int nsm);
unsigned reduce_grid(int n, int nsm);
cudaError_t launch_cost_stats(int n, const void *cost, int kind, double *partials,
                              unsigned *counter, double *out, cudaStream_t s, int nsm);
cudaError_t launch_expect(int n, const void *psi, bool c128, const void *cost, int kind,
                          double fmin, double *partials, unsigned *counter, double *out, int which,
                          cudaStream_t s, int nsm);

// tb: log2 of the tile (float: 13 forward, 12 adjoint; double: 9, 10, 12
// forward, 9, 10, 11 adjoint); other values fail with cudaErrorInvalidValue.
cudaError_t launch_fwd(const FwdParams<float> &P, bool high, int tb, cudaStream_t s, int nsm);
cudaError_t launch_fwd(const FwdParams<double> &P, bool high, int tb, cudaStream_t s, int nsm);
cudaError_t launch_bwd(const BwdParams<float> &P, bool high, int tb, cudaStream_t s, int nsm);
cudaError_t launch_bwd(const BwdParams<double> &P, bool high, int tb, cudaStream_t s, int nsm);

// Launch profiling (profile.cu): returns a record id, or -1 when disabled.
int prof_begin(cudaStream_t s);
void prof_end(int id, cudaStream_t s, const char *kind, double bytes);

// ---- complex64 passes streamed by TMA (tma_kernels.cu)
// Round plans for the TMA 128-byte swizzle (conflict-free at 8 and 16 bytes).
using PlanTmaF13Low = Plan<13, 5, 256, 0, 3, 0x1F00, 0x001F, 0x00E0,
                           0x020F, 0x01F0, 0x1C00, 0x01F0, 0x020F, 0x1C00>;
using PlanTmaF13High = Plan<13, 5, 256, 0, 2, 0x1F00, 0x001F, 0x00E0,
                            0x01F0, 0x020F, 0x1C00>;
using PlanTmaB12Low = Plan<12, 4, 256, 0, 3, 0x0F00, 0x001F, 0x00E0,
                           0x000F, 0x01F0, 0x0E00, 0x00F0, 0x010F, 0x0E00>;
using PlanTmaB12High = Plan<12, 4, 256, 0, 2, 0x0F00, 0x001F, 0x00E0,
                            0x00F0, 0x010F, 0x0E00>;
static_assert(PlanTmaF13Low::valid() && PlanTmaF13High::valid(), "bad TMA F13 plan");
static_assert(PlanTmaB12Low::valid() && PlanTmaB12High::valid(), "bad TMA B12 plan");
// Adjoint HIGH groups of 9 qubits on one 512-thread CTA per SM ("wide"): the
// 2^13-amplitude tile of psi and lambda (16 contiguous amplitudes x rows
// h..h+8, 128 KB) in one CTA; round 0 holds tile bits 8-11 in registers,
// round 1 tile bits 4-7 and tile bit 12 as lane bit 4 (a shuffle rotation).
using PlanTmaB13High = Plan<13, 4, 512, 0, 2, 0x0F00, 0x001F, 0x10E0, 0x00F0, 0x100F, 0x0F00>;
static_assert(PlanTmaB13High::valid(), "bad TMA B13 plan");

// The TMA passes hold vectors in the twisted basis s(x) = (-i)^popc(x) psi(x),
// where exp(-i b X_q) acts on a pair as the real rotation
// [[cos b, sin b], [-sin b, cos b]].  Rotations run in reduced ("tan") form,
// exp(-i b X) = sigma * G with
//   form 0: sigma = cos b,  G(a, b) = (a + t b, b - t a),  t = tan b
//   form 1: sigma = sin b,  G(a, b) = (u a + b, u b - a),  u = cot b
// (the adjoint uses -b), |t|, |u| <= 1; the host tracks the product of the
// sigmas and folds it into the next phase multiply (scl_phase, or the phase
// table) or applies it at the end of the pass (scl_end).

// Phase factors of the TMA passes.  Mode 0 (integer costs): with
// d = (f - fmin) >> shift (every f - fmin a multiple of 2^shift),
//   nd = 2:  exp(-i g f) = D0[d & 63] * D1[d >> 6],
//   nd = 3:  exp(-i g f) = D0[d & 31] * D1[(d >> 5) & 31] * D2[d >> 10],
// the last table also carrying exp(-i g fmin) and the pending scale; the
// tables lie back to back in d[] (nent entries).  Shared memory holds each
// entry as 16 interleaved copies, so the 16 lanes of a half-warp read 16
// different bank pairs whatever their costs.  Mode 1: computed from
// g / 2pi = g_hi + g_lo (float-float).
constexpr int kPhaseCopies = 16;
constexpr int kPhaseMaxEntries = 112;
constexpr int kPhaseTabEntries = kPhaseMaxEntries * kPhaseCopies;

struct PhaseDigits {
  int mode;
  int fmin;
  int shift;
  int nd;     // 2 or 3 digits
  int last;   // entries of the last table - 1 (its index is clamped to this)
  int nent;   // entries in use
  float g_hi, g_lo;
  float2 d[kPhaseMaxEntries];
};

struct alignas(64) TmaFwdParams {
  CUtensorMap map_psi;   // state, 8-byte elements, 128-byte swizzle (loads)
  CUtensorMap map_cost;  // cost vector, 4-byte elements
  float2 *psi;           // the state (finished tiles are stored from registers)
  uint64_t ntiles;
  int h, c, cost_kind;  // tile = 2^c contiguous amplitudes x rows at qubits h..
  Sweep s1, s2;
  float tau1, tau2;
  int form1, form2;
  float2 scl_phase, scl_end;
  int end_scale;
  int has_phase, init_plus, reduce;
  int twist_in;  // first pass on a caller's state: into the twisted basis
  int untwist;   // last pass (with end_scale): back to the standard basis
  float amp;
  uint32_t fmin_word;  // f_min as the cost vector stores it (int32 or float32 bits)
  double *partials;
  unsigned *counter;
  double *out;
  unsigned *err;
  PhaseDigits ph;
};

struct alignas(64) TmaBwdParams {
  CUtensorMap map_psi, map_lam, map_cost;  // loads
  float2 *psi, *lam;                       // stores, from registers
  uint64_t ntiles;
  int h, c, cost_kind;
  Sweep s1, s2;
  float tau1, tau2;
  int form1, form2;
  float2 scl_phase;   // multiplies the un-phase factor (computed mode)
  float w1[4], w2[4]; // |scale|^2 weights of the inner products taken in each round
  float wg;           // |scale|^2 weight of the d/d gamma inner product
  int has_phase, init_lambda;
  int untwist;  // last pass: psi back to the standard basis, lambda not stored
  // HIGH group of 9 new qubits (c = 4) on a 2^13-amplitude tile: 1 = cluster
  // pair, two CTAs holding its two halves (k_bwd_pair; map_cost is then the
  // pair cost map of the phase layout for passes with a phase); 2 = one
  // 512-thread CTA (k_bwd_tma with PlanTmaB13High); 0 = neither
  int cluster;
  double *partials;
  unsigned *counter;
  double *out_b1, *out_g, *out_b2;
  unsigned *err;
  PhaseDigits ph;
};

cudaError_t make_tile_map(CUtensorMap *map, void *base, int n, int tb, int h, int c, int esz,
                          int swizzle_bytes);
// Cost tile of one CTA of a pair in the phase layout: 16 contiguous elements
// x qubits h..h+3 and h+5..h+8, qubit h+4 fixed by the box coordinate.
cudaError_t make_pair_cost_map(CUtensorMap *map, void *base, int n, int h, int esz);
// TMA passes over 4-byte (int32 / float32) and 2-byte (uint16) cost vectors.
cudaError_t launch_fwd_tma(const TmaFwdParams &P, bool high, cudaStream_t s, int nsm);
// one bounded device-side wait that nothing completes (sets *err after ~1 s)
cudaError_t launch_wait_selftest(unsigned *err, cudaStream_t s);
cudaError_t launch_bwd_tma(const TmaBwdParams &P, bool high, cudaStream_t s, int nsm);
cudaError_t launch_fwd_tma_u16(const TmaFwdParams &P, bool high, cudaStream_t s, int nsm);
cudaError_t launch_bwd_tma_u16(const TmaBwdParams &P, bool high, cudaStream_t s, int nsm);

// ---- XY ring mixer passes streamed by TMA (complex64).  A ring layer is the
// ordered chain of gates (q, q + 1), then (n - 1, 0).  Tiles of 2^13
// amplitudes; a round holds 5 consecutive tile bits in registers and applies
// the chain's gates among them in order, consecutive rounds sharing one bit:
//   LOW pass (qubits 0..12):  rounds over tile bits 0-4, 4-8, 8-12;
//   HIGH pass (16 contiguous amplitudes x rows h..h+8 at tile bits 4..12):
//                             rounds over tile bits 4-8, 8-12.
// em[r] bit i: apply the gate on the round's register bits (i, i + 1).  wrap:
// after the last round, the gate (tile bit 12, tile bit 0) = (n - 1, 0), tile
// bit 0 being lane bit 0 there (a shuffle).
using PlanXyLow = Plan<13, 5, 256, 0, 3, 0x001F, 0x03E0, 0x1C00, 0x01F0, 0x020F, 0x1C00,
                       0x1F00, 0x001F, 0x00E0>;
using PlanXyHigh = Plan<13, 5, 256, 0, 2, 0x01F0, 0x020F, 0x1C00, 0x1F00, 0x001F, 0x00E0>;
static_assert(PlanXyLow::valid_round(0) && PlanXyLow::valid_round(1) && PlanXyLow::valid_round(2) &&
                  PlanXyHigh::valid_round(0) && PlanXyHigh::valid_round(1),
              "bad XY plans");

struct alignas(64) XyTmaParams {
  CUtensorMap map_psi, map_cost;
  float2 *psi;
  uint64_t ntiles;
  int h, c, cost_kind;
  int has_phase;       // the layer's phase before the gates (LOW pass)
  uint32_t em[3];      // gate masks per round
  int wrap;            // the gate (n - 1, 0) after the last round
  float t, s;          // tan(b/2), sin(b) of the layer's beta reduced to |b| <= pi/2
  int neg;             // the reduction took out a factor -1
  unsigned *err;
  PhaseDigits ph;
};
cudaError_t launch_xy_tma(const XyTmaParams &P, bool low, cudaStream_t s, int nsm);
cudaError_t launch_xy_tma_u16(const XyTmaParams &P, bool low, cudaStream_t s, int nsm);

// One XY-mixer pass over tiles of 2^tb amplitudes: qubits 0..c-1 (contiguous)
// and h..h+tb-c-1; the gates act on tile bits (ga[g], gb[g]) in order.
constexpr int kXyMaxTb = 12;
constexpr int kXyMaxGates = 64;
struct XyPass {
  void *psi;
  const void *cost;
  uint64_t ntiles;
  int tb, c, h;
  int cost_kind, has_phase;  // phase exp(-i g f) applied while loading
  float g_hi, g_lo;          // complex64: g / 2pi = g_hi + g_lo
  double g2pi;               // complex128: g / 2pi
  double tb2, sb;            // tan(b/2), sin(b) of the layer's beta reduced to |b| <= pi/2
  int neg;                   // the reduction took out a factor -1
  int ngates;
  uint8_t ga[kXyMaxGates], gb[kXyMaxGates];
  PhaseDigits ph;  // complex64 integer costs: digit tables (mode 0), else computed
};

cudaError_t launch_xy_tile(const XyPass &P, bool c128, cudaStream_t s, int nsm);
cudaError_t launch_xy_gate(void *psi, bool c128, int n, int i, int j, double tb2, double sb, int neg,
                           cudaStream_t s, int nsm);
cudaError_t launch_dicke(void *psi, bool c128, int n, int k, double amp, cudaStream_t s, int nsm);

cudaError_t launch_small_batch(const SmallJob<float> *d_jobs, int count, int max_n, cudaStream_t s);
cudaError_t launch_small_batch(const SmallJob<double> *d_jobs, int count, int max_n, cudaStream_t s);
cudaError_t launch_small(const SmallParams<float> &P, cudaStream_t s);
cudaError_t launch_small(const SmallParams<double> &P, cudaStream_t s);

}  // namespace qaoa
