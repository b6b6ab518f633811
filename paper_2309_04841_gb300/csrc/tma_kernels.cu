// tma_kernels.cu -- complex64 passes streamed by the Tensor Memory Accelerator.
//
// Algorithm 1 rotations on a tile window (in the twisted basis, packed fp32x2
// FMA), the phase of Algorithm 3 (conflict-free digit tables), the fused
// energy/overlap, and the adjoint inner products:
//   * persistent CTAs, two per SM, 256 threads each, one tile buffer each
//     (the adjoint's 9-qubit groups: one 512-thread CTA per SM);
//   * thread 0 issues cp.async.bulk.tensor loads (mbarrier complete_tx) of the
//     state tile (and the cost tile) with the TMA 128-byte swizzle; the
//     compute rounds are laid out so that every shared-memory access of the
//     state is bank-conflict free under that swizzle;
//   * once the last round's data is in registers the buffer goes to the next
//     tile's load, and the finished tile is stored from the registers with
//     coalesced global stores while that load is in flight; the other CTA on
//     the SM computes meanwhile.
// A tile is 2^TB amplitudes: 2^c contiguous ones (c = 4..6) times 2^(TB-c)
// rows at qubits h.. (the contiguous LOW tile for the low group).  The tensor
// maps view the vectors as 5-D arrays so that one box is one tile.
// Every wait on an mbarrier is bounded (about one second of %globaltimer);
// on timeout the kernel records an error word and returns.
#include <cuda.h>

#include <type_traits>

#include "qaoa_common.cuh"
#include "kernels.h"

// Cost vector element width of this compilation: 4 (int32 / float32) or 2
// (uint16).  The build compiles this file once for each.
#ifndef QAOA_TMA_CW
#define QAOA_TMA_CW 4
#endif

namespace qaoa {

namespace {

using CostWord = std::conditional_t<QAOA_TMA_CW == 2, uint16_t, uint32_t>;
constexpr uint32_t kCW = QAOA_TMA_CW;

constexpr uint64_t kWaitNs = 1000000000ull;  // bounded waits: 1 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Raises the transaction count of the current phase without arriving.
__device__ __forceinline__ void mbar_add_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// try_wait suspends the thread (it takes no issue slots) until the phase
// completes or kSuspendNs pass, so a waiting warp does not spin.
constexpr uint32_t kSuspendNs = 20000;

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}

// Bounded wait for the mbarrier phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (!mbar_try(bar, parity))
    if (gtimer() - t0 > kWaitNs) return false;
  return true;
}

// Tile coordinates in the 5-D tensor-map view: (0, x1, x2, x3, x4).
struct TC {
  int x1, x2, x4;
  int x3 = 0;
};

__device__ __forceinline__ void tma_load(void *dst, const CUtensorMap *map, TC c, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(c.x1), "r"(c.x2), "r"(c.x3), "r"(c.x4),
      "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Barrier among the CTA's NT threads (named barrier 1).
template <int NT = 256>
__device__ __forceinline__ void cbar() { asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory"); }

// ---- cluster pairs (two CTAs, distributed shared memory)
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// Split cluster barrier: every thread of both CTAs arrives (release: its
// earlier shared-memory accesses, local or remote, are ordered before) and
// later waits (acquire).  Arrive and wait alternate in every thread.
__device__ __forceinline__ void cl_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cl_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The same shared-memory offset in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
// Push-model exchange between the CTAs of a pair: st.async writes 8 bytes
// into the partner's shared memory and counts them on the partner's
// mbarrier (complete_tx), which the partner waits on; no fence is involved.
__device__ __forceinline__ void st_async(uint32_t addr, float2 v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(addr),
               "f"(v.x), "f"(v.y), "r"(bar)
               : "memory");
}
// Arrival on the partner's mbarrier without memory ordering.  The loads it
// covers must have returned before it issues: `dep` is a value computed from
// every register those loads wrote and `zero` a runtime zero, so the address
// (bar + (dep & zero)) carries a data dependency on all of them that neither
// the compiler nor the assembler can drop (one warp-wide shared load returns
// for all lanes at once, so lane 0's registers cover the warp).
__device__ __forceinline__ void mbar_arrive_remote(uint32_t bar, uint32_t dep, uint32_t zero) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar + (dep & zero))
               : "memory");
}

// Bits of every value of the two vectors folded into one word (the
// dependency of mbar_arrive_remote where no other result depends on them all).
template <int N>
__device__ __forceinline__ uint32_t fold_bits(const float2 (&v)[N], const float2 (&w)[N]) {
  uint32_t d = 0;
#pragma unroll
  for (int r = 0; r < N; ++r)
    d ^= __float_as_uint(v[r].x) ^ __float_as_uint(v[r].y) ^ __float_as_uint(w[r].x) ^ __float_as_uint(w[r].y);
  return d;
}
__device__ __forceinline__ bool mbar_try_cl(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}

// Bounded wait for a phase that another CTA of the cluster completes (its
// writes are visible afterwards).
__device__ __forceinline__ bool mbar_wait_cl(uint64_t *bar, uint32_t parity) {
  if (mbar_try_cl(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (!mbar_try_cl(bar, parity))
    if (gtimer() - t0 > kWaitNs) return false;
  return true;
}

// TMA swizzle seen at 8-byte granularity.  SWIZZLE_128B: the 16-byte chunk
// index inside each 128-byte row is XORed with the row index mod 8;
// SWIZZLE_64B: bits 4-5 of the byte address are XORed with bits 7-8.
template <int SW>
__host__ __device__ constexpr uint32_t tswz(uint32_t t) {
  return SW == 128 ? t ^ (((t >> 4) & 7u) << 1) : t ^ (((t >> 4) & 3u) << 1);
}

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return f2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ---- twisted basis
// The passes keep psi (and lambda) as s(x) = (-i)^popc(x) psi(x).  In that
// basis exp(-i b X_q) is the real rotation [[cos b, sin b], [-sin b, cos b]]
// on each pair (s(x), s(x | 2^q)), applied alike to both components, so one
// pair update is two packed fp32x2 FMAs.  Diagonal operators (the phase, f,
// |.|^2) are unchanged.  Reduced (tangent) forms, the scale sigma (real) left
// to the host:
//   form 0: sigma = cos b, (a, b) <- (a + t b, b - t a),  t = tan b
//   form 1: sigma = sin b, (a, b) <- (u a + b, u b - a),  u = cot b
// (the adjoint uses -b); |t|, |u| <= 1.
template <int EB>
__device__ __forceinline__ void rot_tw(float2 (&v)[1 << EB], uint32_t m, float tau, int form) {
  const float2 tp = f2(tau, tau), tn = f2(-tau, -tau);
  if (form == 0) {
#pragma unroll
    for (int i = 0; i < EB; ++i)
      if ((m >> i) & 1u) {
#pragma unroll
        for (int r = 0; r < (1 << EB); ++r)
          if (!((r >> i) & 1)) {
            const float2 a = v[r], b = v[r | (1 << i)];
            v[r] = __ffma2_rn(tp, b, a);
            v[r | (1 << i)] = __ffma2_rn(tn, a, b);
          }
      }
  } else {
#pragma unroll
    for (int i = 0; i < EB; ++i)
      if ((m >> i) & 1u) {
#pragma unroll
        for (int r = 0; r < (1 << EB); ++r)
          if (!((r >> i) & 1)) {
            const float2 a = v[r], b = v[r | (1 << i)];
            v[r] = __ffma2_rn(tp, a, b);
            v[r | (1 << i)] = __ffma2_rn(tp, b, f2(-a.x, -a.y));
          }
      }
  }
}

// Adjoint: un-rotation of psi (v) and lambda (w), adding first the raw
// Im <lambda| X_q |psi> of each pair, which in the twisted basis is
// lambda_a . psi_b - lambda_b . psi_a (real dot products of the complex
// components); the round's sum is weighted by wr (the squared scale the
// stored vectors owe at this point).  With LANES, lm (at most one bit) names
// a lane bit whose pairs sit in two lanes: each lane takes its partner's
// values by shuffle, adds its half of the pair term and updates its own
// element.  Every product of the round uses the vectors as they were before
// the round's rotations.
template <int EB, bool LANES>
__device__ __forceinline__ void unrot_tw(float2 (&v)[1 << EB], float2 (&w)[1 << EB], uint32_t m,
                                         uint32_t lm, float tau, int form, float wr, float &acc) {
  if (m == 0u && (!LANES || lm == 0u)) return;
  // two accumulator pairs (by register parity) halve the dependency chains
  float2 pp[2] = {f2(0.f, 0.f), f2(0.f, 0.f)}, pm[2] = {f2(0.f, 0.f), f2(0.f, 0.f)};
#pragma unroll
  for (int i = 0; i < EB; ++i)
    if ((m >> i) & 1u) {
#pragma unroll
      for (int r = 0; r < (1 << EB); ++r)
        if (!((r >> i) & 1)) {
          const int k = (r >> (i == 0 ? 1 : 0)) & 1;
          pp[k] = __ffma2_rn(w[r], v[r | (1 << i)], pp[k]);
          pm[k] = __ffma2_rn(w[r | (1 << i)], v[r], pm[k]);
        }
    }
  const float2 sp = __fadd2_rn(pp[0], pp[1]), sm = __fadd2_rn(pm[0], pm[1]);
  float lane_term = 0.f;
  if constexpr (LANES) {
    if (lm != 0u) {
      const int lb = __ffs((int)lm) - 1;
      const float sg = ((threadIdx.x >> lb) & 1u) ? -1.f : 1.f;  // -1: the pair's upper element
      const float2 st = f2(sg * tau, sg * tau), tt = f2(tau, tau);
      float2 q = f2(0.f, 0.f);
#pragma unroll
      for (int r = 0; r < (1 << EB); ++r) {
        const float2 pv = f2(__shfl_xor_sync(0xffffffffu, v[r].x, 1 << lb),
                             __shfl_xor_sync(0xffffffffu, v[r].y, 1 << lb));
        const float2 pw = f2(__shfl_xor_sync(0xffffffffu, w[r].x, 1 << lb),
                             __shfl_xor_sync(0xffffffffu, w[r].y, 1 << lb));
        q = __ffma2_rn(w[r], pv, q);
        if (form == 0) {  // (a, b) <- (a + t b, b - t a)
          v[r] = __ffma2_rn(st, pv, v[r]);
          w[r] = __ffma2_rn(st, pw, w[r]);
        } else {  // (a, b) <- (u a + b, u b - a)
          v[r] = __ffma2_rn(tt, v[r], f2(sg * pv.x, sg * pv.y));
          w[r] = __ffma2_rn(tt, w[r], f2(sg * pw.x, sg * pw.y));
        }
      }
      lane_term = sg * (q.x + q.y);
    }
  }
  acc = fmaf((sp.x + sp.y) - (sm.x + sm.y) + lane_term, wr, acc);
  rot_tw<EB>(v, m, tau, form);
  rot_tw<EB>(w, m, tau, form);
}

// z * i^k (k folds to a constant where the register index is one)
__device__ __forceinline__ float2 ipow(float2 z, int k) {
  k &= 3;
  return k == 0 ? z : k == 1 ? f2(-z.y, z.x) : k == 2 ? f2(-z.x, -z.y) : f2(z.y, -z.x);
}

__device__ __forceinline__ uint32_t pdep_d(uint32_t v, uint32_t mask) {
  uint32_t out = 0;
  int k = 0;
#pragma unroll
  for (int b = 0; b < 32; ++b)
    if ((mask >> b) & 1u) {
      out |= ((v >> k) & 1u) << b;
      ++k;
    }
  return out;
}

template <class PL, int R>
__device__ __forceinline__ uint32_t thr_tile() {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  return pdep_d(lane, PL::lane(R)) | pdep_d(warp, PL::warp(R));
}

// Twist exponent base of this thread in round R of tile T: register r holds
// global index x with popc(x) = twist_base + popc(r), tile offset and tile
// number filling disjoint bits of x.
template <class PL, int R>
__device__ __forceinline__ int twist_base(uint64_t T) {
  return __popc(thr_tile<PL, R>()) + __popcll(T);
}

// Registers <- shared tile in round-R layout (16-byte accesses when the
// round holds tile bit 0 in registers).
template <class PL, int R, int SW>
__device__ __forceinline__ void lds_round(float2 (&v)[PL::NREG], const float2 *buf) {
  const uint32_t st = tswz<SW>(thr_tile<PL, R>());
  if constexpr ((PL::reg(R) & 1u) != 0u) {
#pragma unroll
    for (int r = 0; r < PL::NREG; r += 2) {
      const float4 q = *reinterpret_cast<const float4 *>(buf + (st ^ tswz<SW>(pdep(r, PL::reg(R)))));
      v[r] = f2(q.x, q.y);
      v[r + 1] = f2(q.z, q.w);
    }
  } else {
#pragma unroll
    for (int r = 0; r < PL::NREG; ++r) v[r] = buf[st ^ tswz<SW>(pdep(r, PL::reg(R)))];
  }
}

template <class PL, int R, int SW>
__device__ __forceinline__ void sts_round(const float2 (&v)[PL::NREG], float2 *buf) {
  const uint32_t st = tswz<SW>(thr_tile<PL, R>());
  if constexpr ((PL::reg(R) & 1u) != 0u) {
#pragma unroll
    for (int r = 0; r < PL::NREG; r += 2)
      *reinterpret_cast<float4 *>(buf + (st ^ tswz<SW>(pdep(r, PL::reg(R))))) =
          make_float4(v[r].x, v[r].y, v[r + 1].x, v[r + 1].y);
  } else {
#pragma unroll
    for (int r = 0; r < PL::NREG; ++r) buf[st ^ tswz<SW>(pdep(r, PL::reg(R)))] = v[r];
  }
}

template <class PL, int RF, int RT, int SW>
__device__ __forceinline__ void xp(float2 (&v)[PL::NREG], float2 *buf) {
  sts_round<PL, RF, SW>(v, buf);
  cbar<PL::NT>();
  lds_round<PL, RT, SW>(v, buf);
}

// xp with `at_barrier()` run right after the barrier (all reads of the
// previous round done), before the loads.
template <class PL, int RF, int RT, int SW, class F>
__device__ __forceinline__ void xp_hook(float2 (&v)[PL::NREG], float2 *buf, F at_barrier) {
  sts_round<PL, RF, SW>(v, buf);
  cbar<PL::NT>();
  at_barrier();
  lds_round<PL, RT, SW>(v, buf);
}

// The same for psi and lambda together (one barrier).
template <class PL, int RF, int RT, int SW, class F>
__device__ __forceinline__ void xp_pair(float2 (&v)[PL::NREG], float2 (&w)[PL::NREG], float2 *bv,
                                        float2 *bw, F at_barrier) {
  sts_round<PL, RF, SW>(v, bv);
  sts_round<PL, RF, SW>(w, bw);
  cbar<PL::NT>();
  at_barrier();
  lds_round<PL, RT, SW>(v, bv);
  lds_round<PL, RT, SW>(w, bw);
}

struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// exp(-i g f) from the raw 32-bit cost word (int32 or float32).
// exp(-i g f) from the raw 32-bit cost word; M = 2 / 3: digit tables with M
// digits (integer costs), M = 1: computed (int32 or float32 costs).  Callers
// branch on the mode once per round, outside their register loops.
template <int M>
__device__ __forceinline__ float2 phase_of(const PhaseDigits &ph, int kind, const float2 *tab,
                                           uint32_t word) {
  if constexpr (M == 2 || M == 3) {
    // conflict-free lookups: this lane's copy of each digit table
    const uint32_t d = (uint32_t)((int)word - ph.fmin) >> ph.shift;
    const uint32_t q = threadIdx.x & (kPhaseCopies - 1);
    if constexpr (M == 2) {
      const float2 a = tab[((d & 63u) << 4) | q];
      const float2 b = tab[((64u + min(d >> 6, (uint32_t)ph.last)) << 4) | q];
      return cmulf(a, b);
    } else {
      const float2 a = tab[((d & 31u) << 4) | q];
      const float2 b = tab[((32u + ((d >> 5) & 31u)) << 4) | q];
      const float2 c = tab[((64u + min(d >> 10, (uint32_t)ph.last)) << 4) | q];
      return cmulf(cmulf(a, b), c);
    }
  } else {
    float fh, fl;
    if (kind != kCostF32) {  // int32 or uint16
      const int f = (int)word;
      fh = (float)f;
      fl = (float)((long long)f - (long long)fh);
    } else {
      fh = __uint_as_float(word);
      fl = 0.f;
    }
    // g f / 2pi as a float-float: Dekker's two-product p + e = g_hi * fh via fma
    const float p = ph.g_hi * fh;
    const float e = fmaf(ph.g_hi, fh, -p);
    const float r = (p - rintf(p)) + (e + fmaf(ph.g_hi, fl, ph.g_lo * fh));
    float sn, cs;
    sincospif(2.0f * r, &sn, &cs);
    return f2(cs, -sn);
  }
}

// Phase mode of a pass as the template argument of phase_of.
__device__ __forceinline__ int phase_m(const PhaseDigits &ph) {
  return ph.mode != 0 ? 1 : ph.nd == 2 ? 2 : 3;
}

// Shared-memory copy of the digit tables: entry e (of the concatenated
// tables), copy q at e * 16 + q.
template <int NT>
__device__ __forceinline__ void fill_phase_tab(float2 *tab, const PhaseDigits &ph) {
  const int n = min(ph.nent, kPhaseMaxEntries) * kPhaseCopies;
  for (int i = threadIdx.x; i < n; i += NT) tab[i] = ph.d[i >> 4];
}

__device__ __forceinline__ float cost_val(int kind, uint32_t word) {
  return kind == kCostF32 ? __uint_as_float(word) : (float)(int)word;
}

// v <- v * exp(-i g f) (* scl in computed mode; table mode has it folded in).
template <class PL, int R, int M>
__device__ __forceinline__ void phase_round_m(float2 (&v)[PL::NREG], const CostWord *cb,
                                              const PhaseDigits &ph, int kind, const float2 *tab,
                                              float2 scl) {
  const uint32_t tt = thr_tile<PL, R>();
#pragma unroll
  for (int r = 0; r < PL::NREG; ++r) {
    const float2 z = phase_of<M>(ph, kind, tab, cb[tt | pdep(r, PL::reg(R))]);
    v[r] = cmulf(v[r], M == 1 ? cmulf(scl, z) : z);
  }
}

template <class PL, int R>
__device__ __forceinline__ void phase_round(float2 (&v)[PL::NREG], const CostWord *cb,
                                            const PhaseDigits &ph, int kind, const float2 *tab,
                                            float2 scl) {
  const int m = phase_m(ph);
  if (m == 2)
    phase_round_m<PL, R, 2>(v, cb, ph, kind, tab, scl);
  else if (m == 3)
    phase_round_m<PL, R, 3>(v, cb, ph, kind, tab, scl);
  else
    phase_round_m<PL, R, 1>(v, cb, ph, kind, tab, scl);
}

// Float-float running sum (Knuth's TwoSum adds each term exactly into hi + lo):
// per-thread tile sums stay off the FP64 pipe, which is narrow on this part.
struct FF {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float s = hi + x, bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <class PL, int R>
__device__ __forceinline__ void eo_round(const float2 (&v)[PL::NREG], const CostWord *cb, int kind,
                                         uint32_t fmin_word, float &e, float &o) {
  // f == f_min is tested on the raw words (exact for integer costs; for
  // float32 costs f_min is one of the stored values, and +0 / -0 compare equal)
  const uint32_t tt = thr_tile<PL, R>();
#pragma unroll
  for (int r = 0; r < PL::NREG; ++r) {
    const uint32_t w = cb[tt | pdep(r, PL::reg(R))];
    const float f = cost_val(kind, w);
    const float pr = v[r].x * v[r].x + v[r].y * v[r].y;
    e += pr * f;
    const bool at_min = kind != kCostF32 ? w == fmin_word : f == __uint_as_float(fmin_word);
    o += at_min ? pr : 0.f;
  }
}

// Sum of K doubles over the CTA's NT threads (fixed order); thread 0 gets it.
template <int K, int NT = 256>
__device__ __forceinline__ void csum(double (&a)[K], double *red) {
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_down_sync(0xffffffffu, a[k], o);
  const int w = threadIdx.x >> 5;
  cbar<NT>();
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) red[w * K + k] = a[k];
  cbar<NT>();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int i = 0; i < NT / 32; ++i) s += red[i * K + k];
      a[k] = s;
    }
}

// After the tile loop: the last CTA sums the per-CTA partials in CTA order
// (deterministic for a given grid; the grid depends only on the GPU and n).
template <int K, class Fin>
__device__ __forceinline__ void final_reduce(const double *partials, uint64_t nparts,
                                             unsigned *counter, double *red, Fin fin) {
  __shared__ int am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1u);
  __syncthreads();
  if (!am_last || threadIdx.x >= 256) return;
  __threadfence();
  double a[K];
#pragma unroll
  for (int k = 0; k < K; ++k) a[k] = 0.0;
  for (uint64_t t = threadIdx.x; t < nparts; t += 256)
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] += __ldcg(partials + t * K + k);
  csum<K>(a, red);
  if (threadIdx.x == 0) {
    fin(a);
    *counter = 0u;
  }
}

// Shared-memory layout (offsets from a 1024-byte aligned base): the state
// tile (and the lambda tile), the cost tile, the phase tables, the mbarrier
// and the reduction scratch.
struct Lay {
  uint32_t tile_bytes, lam_off, cost_off, cost_bytes, tab_off, bar_off, red_off;
};

__device__ __forceinline__ Lay layout(uint32_t tile_elems, bool two, bool cost) {
  Lay L;
  L.tile_bytes = tile_elems * 8u;
  L.lam_off = L.tile_bytes;
  L.cost_off = L.lam_off + (two ? L.tile_bytes : 0u);
  L.cost_bytes = cost ? tile_elems * kCW : 0u;
  L.tab_off = L.cost_off + L.cost_bytes;
  L.bar_off = L.tab_off + (uint32_t)kPhaseTabEntries * 8u;
  L.red_off = L.bar_off + 32u;
  return L;
}

// Registers (round-R layout) -> the state vector in HBM, straight from the
// registers: tile offset t of tile T is amplitude
//   x = (t & (2^c - 1)) | (mid << c) | ((t >> c) << h) | (top << (h + TB - c)),
// mid / top the low h - c / remaining bits of T.  In every round the 32 lanes
// of a warp cover whole 2^c-amplitude segments (c >= 3: 64 bytes or more),
// so the stores are coalesced.
template <class PL, int R>
__device__ __forceinline__ void stg_round(const float2 (&v)[PL::NREG], float2 *g, uint64_t T,
                                          int h, int c, uint32_t thr = thr_tile<PL, R>()) {
  constexpr uint32_t RM = PL::reg(R);
  const int midbits = h - c;
  const uint32_t cm = (1u << c) - 1u;
  auto f = [&](uint32_t t) -> uint64_t { return (uint64_t)(t & cm) | ((uint64_t)(t >> c) << h); };
  const uint64_t mid = T & ((1ull << midbits) - 1ull), top = T >> midbits;
  float2 *b = g + ((mid << c) | (top << (h + PL::TB - c))) + f(thr);
  uint64_t u[PL::EB];  // offset of each register bit
#pragma unroll
  for (int k = 0; k < PL::EB; ++k) u[k] = f(pdep(1u << k, RM));
#pragma unroll
  for (int r = 0; r < PL::NREG; ++r) {
    uint64_t off = 0;
#pragma unroll
    for (int k = 0; k < PL::EB; ++k)
      if ((r >> k) & 1) off += u[k];
    b[off] = v[r];
  }
}

__device__ __forceinline__ unsigned char *aligned_base(unsigned char *raw) {
  const uint32_t a = smem_u32(raw);
  return raw + ((1024u - (a & 1023u)) & 1023u);
}

}  // namespace

static size_t smem_bytes(int tb, bool two, bool cost) {
  const size_t te = (size_t)1 << tb;
  return 1024 + te * 8 * (two ? 2 : 1) + (cost ? te * kCW : 0) + kPhaseTabEntries * 8 + 32 + 16 * 3 * 8;
}

// ------------------------------------------------------------- forward
//
// Persistent CTAs, two per SM (256 threads, at most 128 registers), one tile
// buffer each.  Thread 0 loads a tile with TMA; the 8 warps run the rounds
// (shared-memory transposes between them); once the last round's data is in
// registers the buffer goes to the next tile's load, and the finished tile
// is written from the registers straight to HBM while that load is in flight.
// The other CTA on the SM computes meanwhile.

constexpr int kThreads = 256;

// Abort discipline of the TMA passes.  A wait that runs out sets the CTA's
// flag; every thread reads the flag right after the tile's first barrier
// (all flag writes of this tile happened before it, and none of the next
// tile can happen before the tile's last barrier), so the whole CTA takes
// the same decision, and from then on no load is issued.  The loop is left
// at the top of the next tile; the only load that can still be in flight is
// the one of tile i - 1 whose wait ran out (with its early cost part): wait
// for it, again bounded, before the CTA exits.  A load still outstanding
// after that second bounded wait would mean the copy engine stopped
// delivering; nothing the kernel does then can make its exit safer.
__device__ __forceinline__ void drain(int aborted, uint64_t *full, int i) {
  if (aborted && threadIdx.x == 0 && i > 0) (void)mbar_wait(full, (i - 1) & 1);
}

// Pass kinds, fixed at compile time so each instantiation carries only its
// own path: forward  K = kH1 | kPH | kH2 | kRED,  adjoint  K = kPH | kH2 | kINIT.
constexpr int kH1 = 1, kPH = 2, kH2 = 4, kRED = 8, kINIT = 8;

template <class PL, int K>
__global__ void __launch_bounds__(kThreads, 2) k_fwd_tma(const __grid_constant__ TmaFwdParams P) {
  constexpr int NREG = PL::NREG, NR = PL::NR, EB = PL::EB, SW = 128;
  constexpr bool H1 = (K & kH1) != 0, PH = (K & kPH) != 0, H2 = (K & kH2) != 0, RED = (K & kRED) != 0;
  static_assert(!(H1 && PH && !H2), "a first sweep with the phase always has a second sweep");
  constexpr bool need_cost = PH || RED;
  constexpr int RS = (H1 && H2) ? 0 : NR - 1;  // the round the tile is stored from
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = aligned_base(smem_raw);
  const Lay L = layout(1u << PL::TB, false, need_cost);
  float2 *buf = reinterpret_cast<float2 *>(base);
  const CostWord *cb = reinterpret_cast<const CostWord *>(base + L.cost_off);
  float2 *tab = reinterpret_cast<float2 *>(base + L.tab_off);
  uint64_t *full = reinterpret_cast<uint64_t *>(base + L.bar_off);
  double *red = reinterpret_cast<double *>(base + L.red_off);
  const int tid = threadIdx.x;
  const int midbits = P.h - P.c;
  __shared__ int s_abort;

  if (PH && P.ph.mode == 0) fill_phase_tab<kThreads>(tab, P.ph);
  if (tid == 0) {
    s_abort = 0;
    mbar_init(full, 1);
    fence_mbar_init();
  }
  __syncthreads();

  // 8- or 16-amplitude segments: the outer bits between the segments are view
  // dimension 1; wider segments (bits 4.. are view dimension 1): dimension 2
  auto coords = [&](uint64_t T) {
    const int mid = (int)(T & ((1ull << midbits) - 1ull));
    TC c;
    c.x1 = P.c <= 4 ? mid : 0;
    c.x2 = P.c <= 4 ? 0 : mid;
    c.x4 = (int)(T >> midbits);
    return c;
  };
  // Phase passes that read the cost tile before their last barrier load the
  // next tile's costs as soon as that barrier passes, the state later.
  constexpr bool early_cost = PH && !RED;
  auto issue = [&](uint64_t T, bool cost) {
    const TC c = coords(T);
    mbar_expect_tx(full, (P.init_plus ? 0u : L.tile_bytes) + (cost ? L.cost_bytes : 0u));
    if (!P.init_plus) tma_load(buf, &P.map_psi, c, full);
    if (cost) tma_load(base + L.cost_off, &P.map_cost, c, full);
  };
  int abort_now = 0;  // uniform over the CTA: read after the tile's first barrier
  auto read_abort = [&]() { abort_now = s_abort; };
  auto cost_next = [&](uint64_t T) {
    if (tid == 0 && T + gridDim.x < P.ntiles && !abort_now) {
      mbar_add_tx(full, L.cost_bytes);
      tma_load(base + L.cost_off, &P.map_cost, coords(T + gridDim.x), full);
    }
  };
  // after the tile's last shared-memory read: the buffers go to the next load
  auto release = [&](uint64_t T) {
    cbar();
    if (tid == 0 && T + gridDim.x < P.ntiles && !abort_now) issue(T + gridDim.x, need_cost && !early_cost);
  };

  if (tid == 0 && blockIdx.x < P.ntiles) issue(blockIdx.x, need_cost);

  FF acc_e, acc_o;  // this thread's energy / overlap terms
  int i = 0;
  for (;; ++i) {
    const uint64_t T = blockIdx.x + (uint64_t)i * gridDim.x;
    if (T >= P.ntiles) break;
    // A timed-out wait flags the abort and still runs this tile (on stale
    // data) through the same barriers as every other thread; all threads
    // read the flag after the tile's first barrier and leave together.
    if (abort_now) break;
    if (!mbar_wait(full, i & 1)) {
      s_abort = 1;
      atomicExch(P.err, 1u);
    }
    float2 v[NREG];
    if (P.init_plus) {
      // |+>^n in the twisted basis: amp (-i)^popc(x)
      const float2 z0 = ipow(f2(P.amp, 0.f), -twist_base<PL, 0>(T));
#pragma unroll
      for (int r = 0; r < NREG; ++r) v[r] = ipow(z0, -popc_c(r));
    } else {
      lds_round<PL, 0, SW>(v, buf);
      if (P.twist_in) {
        const float2 z = ipow(f2(1.f, 0.f), -twist_base<PL, 0>(T));
#pragma unroll
        for (int r = 0; r < NREG; ++r) v[r] = ipow(cmulf(v[r], z), -popc_c(r));
      }
    }
    if constexpr (H1) {
      rot_tw<EB>(v, P.s1.m[0], P.tau1, P.form1);
      xp_hook<PL, 0, 1, SW>(v, buf, read_abort);
      if constexpr (NR == 2 && !H2 && !RED) release(T);
      rot_tw<EB>(v, P.s1.m[1], P.tau1, P.form1);
      if constexpr (NR == 3) {
        xp<PL, 1, 2, SW>(v, buf);
        if constexpr (!H2 && !RED) release(T);
        rot_tw<EB>(v, P.s1.m[2], P.tau1, P.form1);
      }
      if constexpr (PH) phase_round<PL, NR - 1>(v, cb, P.ph, P.cost_kind, tab, P.scl_phase);
      if constexpr (H2) {
        rot_tw<EB>(v, P.s2.m[NR - 1], P.tau2, P.form2);
        if constexpr (NR == 3) {
          if constexpr (early_cost)
            xp_hook<PL, 2, 1, SW>(v, buf, [&] { cost_next(T); });
          else
            xp<PL, 2, 1, SW>(v, buf);
          rot_tw<EB>(v, P.s2.m[1], P.tau2, P.form2);
        }
        if constexpr (NR == 3) {
          xp<PL, 1, 0, SW>(v, buf);
        } else if constexpr (early_cost) {
          xp_hook<PL, 1, 0, SW>(v, buf, [&] { cost_next(T); });
        } else {
          xp<PL, 1, 0, SW>(v, buf);
        }
        if constexpr (!RED) release(T);
        rot_tw<EB>(v, P.s2.m[0], P.tau2, P.form2);
      }
    } else {
      if constexpr (PH) phase_round<PL, 0>(v, cb, P.ph, P.cost_kind, tab, P.scl_phase);
      rot_tw<EB>(v, P.s2.m[0], P.tau2, P.form2);
      if constexpr (early_cost)
        xp_hook<PL, 0, 1, SW>(v, buf, [&] { read_abort(); cost_next(T); });
      else
        xp_hook<PL, 0, 1, SW>(v, buf, read_abort);
      if constexpr (NR == 2 && !RED) release(T);
      rot_tw<EB>(v, P.s2.m[1], P.tau2, P.form2);
      if constexpr (NR == 3) {
        xp<PL, 1, 2, SW>(v, buf);
        if constexpr (!RED) release(T);
        rot_tw<EB>(v, P.s2.m[2], P.tau2, P.form2);
      }
    }
    if (P.end_scale) {
      if (P.untwist) {
        // back to the standard basis: psi(x) = i^popc(x) s(x)
        const float2 z = cmulf(P.scl_end, ipow(f2(1.f, 0.f), twist_base<PL, RS>(T)));
#pragma unroll
        for (int r = 0; r < NREG; ++r) v[r] = ipow(cmulf(v[r], z), popc_c(r));
      } else {
#pragma unroll
        for (int r = 0; r < NREG; ++r) v[r] = cmulf(v[r], P.scl_end);
      }
    }
    if constexpr (RED) {
      float e = 0.f, o = 0.f;
      eo_round<PL, RS>(v, cb, P.cost_kind, P.fmin_word, e, o);
      acc_e.add(e);
      acc_o.add(o);
      release(T);
    }
    stg_round<PL, RS>(v, P.psi, T, P.h, P.c);
  }
  drain(abort_now, full, i);
  if constexpr (RED) {
    double a[2] = {acc_e.value(), acc_o.value()};
    csum<2>(a, red);
    if (tid == 0) {
      P.partials[blockIdx.x * 2] = a[0];
      P.partials[blockIdx.x * 2 + 1] = a[1];
    }
    double *out = P.out;
    final_reduce<2>(P.partials, gridDim.x, P.counter, red, [out](double(&a)[2]) {
      out[0] = a[0];
      out[1] = a[1];
    });
  }
}

// ------------------------------------------------------------- adjoint

// d/d gamma term Im <lambda| f |psi> of the round's amplitudes, then psi and
// lambda times the un-phase factor exp(+i g f) (phase mode M as in phase_of).
// CI maps a local tile offset to its cost-tile slot (identity except in the
// pair layout L1, see k_bwd_pair).
struct CostIdx {
  __device__ __forceinline__ uint32_t operator()(uint32_t t) const { return t; }
};
template <class PL, int R, int M, class CI = CostIdx>
__device__ __forceinline__ void unphase_round(float2 (&v)[PL::NREG], float2 (&w)[PL::NREG],
                                              const CostWord *cb, const TmaBwdParams &P,
                                              const float2 *tab, float &ag, CI ci = CI()) {
  const uint32_t tt = thr_tile<PL, R>();
#pragma unroll
  for (int r = 0; r < PL::NREG; ++r) {
    const uint32_t word = cb[ci(tt | pdep(r, PL::reg(R)))];
    const float f = cost_val(P.cost_kind, word);
    ag += P.wg * f * (w[r].x * v[r].y - w[r].y * v[r].x);
    float2 ph = phase_of<M>(P.ph, P.cost_kind, tab, word);
    if constexpr (M == 1) ph = cmulf(ph, P.scl_phase);
    v[r] = cmulf(v[r], ph);
    w[r] = cmulf(w[r], ph);
  }
}

template <class PL, int R, class CI = CostIdx>
__device__ __forceinline__ void unphase_any(float2 (&v)[PL::NREG], float2 (&w)[PL::NREG],
                                            const CostWord *cb, const TmaBwdParams &P,
                                            const float2 *tab, float &ag, CI ci = CI()) {
  const int m = phase_m(P.ph);
  if (m == 2)
    unphase_round<PL, R, 2>(v, w, cb, P, tab, ag, ci);
  else if (m == 3)
    unphase_round<PL, R, 3>(v, w, cb, P, tab, ag, ci);
  else
    unphase_round<PL, R, 1>(v, w, cb, P, tab, ag, ci);
}

// The state tiles use the TMA 128-byte swizzle (16- to 64-amplitude segments).
template <class PL, int K>
__global__ void __launch_bounds__(PL::NT, 512 / PL::NT) k_bwd_tma(const __grid_constant__ TmaBwdParams P) {
  constexpr int NREG = PL::NREG, NR = PL::NR, EB = PL::EB, SW = 128;
  constexpr bool LN = PL::NT == 512;  // the 512-thread plan rotates tile bit 12 across lanes
  constexpr bool PH = (K & kPH) != 0, H2 = (K & kH2) != 0, INIT = (K & kINIT) != 0;
  constexpr bool need_cost = PH || INIT;
  constexpr int RS = H2 ? 0 : NR - 1;  // the round the tiles are stored from
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = aligned_base(smem_raw);
  const Lay L = layout(1u << PL::TB, true, need_cost);
  float2 *bv = reinterpret_cast<float2 *>(base);
  float2 *bw = reinterpret_cast<float2 *>(base + L.lam_off);
  const CostWord *cb = reinterpret_cast<const CostWord *>(base + L.cost_off);
  float2 *tab = reinterpret_cast<float2 *>(base + L.tab_off);
  uint64_t *full = reinterpret_cast<uint64_t *>(base + L.bar_off);
  double *red = reinterpret_cast<double *>(base + L.red_off);
  const int tid = threadIdx.x;
  const int midbits = P.h - P.c;
  __shared__ int s_abort;

  if (PH && P.ph.mode == 0) fill_phase_tab<PL::NT>(tab, P.ph);
  if (tid == 0) {
    s_abort = 0;
    mbar_init(full, 1);
    fence_mbar_init();
  }
  __syncthreads();

  // 8- or 16-amplitude segments: the outer bits between the segments are view
  // dimension 1; wider segments (bits 4.. are view dimension 1): dimension 2
  auto coords = [&](uint64_t T) {
    const int mid = (int)(T & ((1ull << midbits) - 1ull));
    TC c;
    c.x1 = P.c <= 4 ? mid : 0;
    c.x2 = P.c <= 4 ? 0 : mid;
    c.x4 = (int)(T >> midbits);
    return c;
  };
  // Passes whose cost reads end before a later barrier (lambda = f psi in the
  // first round; the phase of a pivot) load the next tile's costs at that
  // barrier, the vectors later.  No load is issued once the CTA has decided
  // to abort (see drain).
  constexpr bool early_cost = (PH && H2 && !INIT) || (INIT && !PH);
  int abort_now = 0;  // uniform over the CTA: read after the tile's first barrier
  auto read_abort = [&]() { abort_now = s_abort; };
  auto issue = [&](uint64_t T, bool cost) {
    const TC c = coords(T);
    mbar_expect_tx(full, L.tile_bytes + (INIT ? 0u : L.tile_bytes) + (cost ? L.cost_bytes : 0u));
    tma_load(bv, &P.map_psi, c, full);
    if (!INIT) tma_load(bw, &P.map_lam, c, full);
    if (cost) tma_load(base + L.cost_off, &P.map_cost, c, full);
  };
  auto cost_next = [&](uint64_t T) {
    if (tid == 0 && T + gridDim.x < P.ntiles && !abort_now) {
      mbar_add_tx(full, L.cost_bytes);
      tma_load(base + L.cost_off, &P.map_cost, coords(T + gridDim.x), full);
    }
  };
  // after the tile's last shared-memory read: the buffers go to the next load
  auto release = [&](uint64_t T) {
    cbar<PL::NT>();
    if (tid == 0 && T + gridDim.x < P.ntiles && !abort_now) issue(T + gridDim.x, need_cost && !early_cost);
  };
  // Passes that end with the un-phase: the vectors go to the next load once
  // the last round's data is in registers, the costs once the phase has read
  // them; the mbarrier's one arrive comes with the cost load, so the phase
  // cannot complete before both loads are counted.
  constexpr bool late_cost = PH && !H2 && !INIT;
  auto release_vectors = [&](uint64_t T) {
    cbar<PL::NT>();
    if (tid == 0 && T + gridDim.x < P.ntiles && !abort_now) {
      const TC c = coords(T + gridDim.x);
      mbar_add_tx(full, 2u * L.tile_bytes);
      tma_load(bv, &P.map_psi, c, full);
      tma_load(bw, &P.map_lam, c, full);
    }
  };
  auto release_cost = [&](uint64_t T) {
    cbar<PL::NT>();
    if (tid == 0 && T + gridDim.x < P.ntiles && !abort_now) {
      mbar_expect_tx(full, L.cost_bytes);
      tma_load(base + L.cost_off, &P.map_cost, coords(T + gridDim.x), full);
    }
  };

  if (tid == 0 && blockIdx.x < P.ntiles) issue(blockIdx.x, need_cost);

  FF acc1, accg, acc2;  // this thread's gradient terms
  int i = 0;
  for (;; ++i) {
    const uint64_t T = blockIdx.x + (uint64_t)i * gridDim.x;
    if (T >= P.ntiles) break;
    // A timed-out wait flags the abort and still runs this tile (on stale
    // data) through the same barriers as every other thread; all threads
    // read the flag after the tile's first barrier and leave together.
    if (abort_now) break;
    if (!mbar_wait(full, i & 1)) {
      s_abort = 1;
      atomicExch(P.err, 1u);
    }
    float2 v[NREG], w[NREG];
    lds_round<PL, 0, SW>(v, bv);
    if constexpr (INIT) {
      // lambda = f psi: the derivative of E = <psi|f|psi> with respect to psi^*
      const uint32_t tt = thr_tile<PL, 0>();
#pragma unroll
      for (int r = 0; r < NREG; ++r) {
        const float f = cost_val(P.cost_kind, cb[tt | pdep(r, PL::reg(0))]);
        w[r] = f2(f * v[r].x, f * v[r].y);
      }
    } else {
      lds_round<PL, 0, SW>(w, bw);
    }
    float a1 = 0.f, ag = 0.f, a2 = 0.f;
    unrot_tw<EB, LN>(v, w, P.s1.m[0], P.s1.lm[0], P.tau1, P.form1, P.w1[0], a1);
    if constexpr (INIT && early_cost)
      xp_pair<PL, 0, 1, SW>(v, w, bv, bw, [&] { read_abort(); cost_next(T); });
    else
      xp_pair<PL, 0, 1, SW>(v, w, bv, bw, [&] { read_abort(); });
    if constexpr (NR == 2 && !PH && !H2) release(T);
    if constexpr (NR == 2 && late_cost) release_vectors(T);
    unrot_tw<EB, LN>(v, w, P.s1.m[1], P.s1.lm[1], P.tau1, P.form1, P.w1[1], a1);
    if constexpr (NR == 3) {
      xp_pair<PL, 1, 2, SW>(v, w, bv, bw, NoHook());
      if constexpr (!PH && !H2) release(T);
      if constexpr (late_cost) release_vectors(T);
      unrot_tw<EB, LN>(v, w, P.s1.m[2], P.s1.lm[2], P.tau1, P.form1, P.w1[2], a1);
    }
    if constexpr (PH) {
      // d/d gamma: Im <lambda| f |psi>, then un-phase both vectors
      unphase_any<PL, NR - 1>(v, w, cb, P, tab, ag);
      if constexpr (late_cost)
        release_cost(T);
      else if constexpr (!H2)
        release(T);
    }
    if constexpr (H2) {
      unrot_tw<EB, LN>(v, w, P.s2.m[NR - 1], P.s2.lm[NR - 1], P.tau2, P.form2, P.w2[NR - 1], a2);
      if constexpr (NR == 3) {
        if constexpr (PH && early_cost)
          xp_pair<PL, 2, 1, SW>(v, w, bv, bw, [&] { cost_next(T); });
        else
          xp_pair<PL, 2, 1, SW>(v, w, bv, bw, NoHook());
        unrot_tw<EB, LN>(v, w, P.s2.m[1], P.s2.lm[1], P.tau2, P.form2, P.w2[1], a2);
        xp_pair<PL, 1, 0, SW>(v, w, bv, bw, NoHook());
      } else if constexpr (PH && early_cost) {
        xp_pair<PL, 1, 0, SW>(v, w, bv, bw, [&] { cost_next(T); });
      } else {
        xp_pair<PL, 1, 0, SW>(v, w, bv, bw, NoHook());
      }
      release(T);
      unrot_tw<EB, LN>(v, w, P.s2.m[0], P.s2.lm[0], P.tau2, P.form2, P.w2[0], a2);
    }
    if (P.untwist) {
      // psi back to the standard basis (lambda is scratch from here on)
      const float2 z = ipow(f2(1.f, 0.f), twist_base<PL, RS>(T));
#pragma unroll
      for (int r = 0; r < NREG; ++r) v[r] = ipow(cmulf(v[r], z), popc_c(r));
    }
    stg_round<PL, RS>(v, P.psi, T, P.h, P.c);
    if (!P.untwist) stg_round<PL, RS>(w, P.lam, T, P.h, P.c);  // the last pass: lambda is spent
    acc1.add(a1);
    accg.add(ag);
    acc2.add(a2);
  }
  drain(abort_now, full, i);
  double a[3] = {acc1.value(), accg.value(), acc2.value()};
  csum<3, PL::NT>(a, red);
  if (tid == 0) {
    P.partials[blockIdx.x * 3] = a[0];
    P.partials[blockIdx.x * 3 + 1] = a[1];
    P.partials[blockIdx.x * 3 + 2] = a[2];
  }
  double *o1 = P.out_b1, *og = P.out_g, *o2 = P.out_b2;
  final_reduce<3>(P.partials, gridDim.x, P.counter, red, [=](double(&a)[3]) {
    if (o1) *o1 += 2.0 * a[0];
    if (og) *og += 2.0 * a[1];
    if (o2) *o2 += 2.0 * a[2];
  });
}

// ------------------------------------------------- adjoint on cluster pairs
//
// A HIGH group of 9 new qubits: the 2^13-amplitude tile (2^4 contiguous
// amplitudes x 9 row qubits h..h+8, tile bits 0..12) is split over the two
// CTAs of a cluster, each holding 2^12 amplitudes of psi and of lambda with
// the two-round plan of the 2^12 tiles.  Two layouts of the halves:
//   L0: CTA rank = tile bit 12, local offset = tile bits 0..11 (the halves
//       the tensor-map loads bring in; round 0);
//   L1: CTA rank = tile bit 8, tile bit 12 at local position 8 (round 1,
//       where position 8 is a lane bit: that qubit is rotated by shuffles).
// Going from one layout to the other, each CTA keeps the amplitudes whose
// local position-8 bit equals its rank and pushes the other half (16 KB of
// psi, 16 KB of lambda) into the partner's shared memory with st.async, at
// the slots with that bit flipped -- exactly the slots the partner is
// vacating; the bytes are counted on the partner's exchange mbarrier
// (complete_tx), on which it waits.  Before pushing, a CTA waits until the
// partner's 8 warps have signalled (a relaxed remote arrive whose address
// depends on every value they loaded) that they have read those slots.  Sweep 1 rotates
// round 0 (tile bits 8..11) in L0, exchanges, then round 1 (tile bits 4..7
// and, by shuffles, tile bit 12) in L1; sweep 2 (pivots) the reverse, back
// to L0.  The phase runs in L1, so those passes load the cost tile of the
// L1 half (a tensor map whose box fixes tile bit 8), stored with tile bits
// 9..12 at slots 8..11.  Single-sweep passes store from L1, pivots from L0;
// either way each CTA writes whole 16-amplitude rows.  (A layout L1 with
// the rank on passenger bit 3 needs one exchange per pivot instead of two,
// but its 64-byte half rows made every pair pass slower.)
//
// Every wait is a bounded mbarrier wait; the cluster barrier runs only once
// at the start (the partner's mbarriers are initialised before any remote
// arrive) and once at the end (neither CTA leaves while the other may still
// push into it), and both CTAs always reach it.
struct PairCostIdx {  // local L1 offset -> slot of the L1 cost tile
  __device__ __forceinline__ uint32_t operator()(uint32_t t) const {
    return (t & 0xFFu) | ((t >> 1) & 0x700u) | ((t & 0x100u) << 3);
  }
};

// One vector from round R's registers into the other layout: keep (store to
// the own slot) where local position 8 equals RANK, else push to the
// partner's slot with position 8 flipped.
template <class PL, int R, uint32_t RANK>
__device__ __forceinline__ void pair_xchg(const float2 (&v)[PL::NREG], float2 *buf, uint32_t rbuf,
                                          uint32_t rbar) {
  const uint32_t tt = thr_tile<PL, R>();
#pragma unroll
  for (int r = 0; r < PL::NREG; ++r) {
    const uint32_t t = tt | pdep(r, PL::reg(R));
    if (((t >> 8) & 1u) != RANK)
      st_async(rbuf + tswz<128>(t ^ 0x100u) * 8u, v[r], rbar);
    else
      buf[tswz<128>(t)] = v[r];
  }
}

template <class PL, int R>
__device__ __forceinline__ void pair_xchg2(const float2 (&v)[PL::NREG], const float2 (&w)[PL::NREG],
                                           float2 *bv, float2 *bw, uint32_t rbv, uint32_t rbw,
                                           uint32_t rbar, uint32_t rank) {
  if (rank == 0u) {
    pair_xchg<PL, R, 0u>(v, bv, rbv, rbar);
    pair_xchg<PL, R, 0u>(w, bw, rbw, rbar);
  } else {
    pair_xchg<PL, R, 1u>(v, bv, rbv, rbar);
    pair_xchg<PL, R, 1u>(w, bw, rbw, rbar);
  }
}

// Round 1 back to L0: local position 8 is lane bit 4 there, so a thread
// keeps all its values or pushes all of them; one branch per thread rather
// than one per register (half of each warp on either side).
template <class PL>
__device__ __forceinline__ void pair_xchg_lane(const float2 (&v)[PL::NREG], const float2 (&w)[PL::NREG],
                                               float2 *bv, float2 *bw, uint32_t rbv, uint32_t rbw,
                                               uint32_t rbar, uint32_t rank) {
  static_assert((PL::lane(1) & 0x100u) && !(PL::reg(1) & 0x100u), "position 8 a lane bit of round 1");
  const uint32_t tt = thr_tile<PL, 1>();
  if (((tt >> 8) & 1u) == rank) {
#pragma unroll
    for (int r = 0; r < PL::NREG; ++r) {
      const uint32_t o = tswz<128>(tt | pdep(r, PL::reg(1)));
      bv[o] = v[r];
      bw[o] = w[r];
    }
  } else {
#pragma unroll
    for (int r = 0; r < PL::NREG; ++r) {
      const uint32_t o = tswz<128>((tt ^ 0x100u) | pdep(r, PL::reg(1))) * 8u;
      st_async(rbv + o, v[r], rbar);
      st_async(rbw + o, w[r], rbar);
    }
  }
}

template <int K>
__global__ void __launch_bounds__(kThreads, 2) k_bwd_pair(const __grid_constant__ TmaBwdParams P) {
  using PL = PlanTmaB12High;
  constexpr int NREG = PL::NREG, EB = PL::EB, SW = 128;
  constexpr bool PH = (K & kPH) != 0, H2 = (K & kH2) != 0, INIT = (K & kINIT) != 0;
  constexpr bool need_cost = PH || INIT;
  constexpr uint32_t kXBytes = (1u << PL::TB) / 2u * 8u * 2u;  // half of psi and of lambda
  static_assert(PL::NR == 2 && PL::lane(1) == 0x010Fu && PL::reg(0) == 0x0F00u,
                "pair layout L1 needs local position 8 as lane bit 4 of round 1");
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = aligned_base(smem_raw);
  const Lay L = layout(1u << PL::TB, true, need_cost);
  float2 *bv = reinterpret_cast<float2 *>(base);
  float2 *bw = reinterpret_cast<float2 *>(base + L.lam_off);
  const CostWord *cb = reinterpret_cast<const CostWord *>(base + L.cost_off);
  float2 *tab = reinterpret_cast<float2 *>(base + L.tab_off);
  uint64_t *full = reinterpret_cast<uint64_t *>(base + L.bar_off);
  double *red = reinterpret_cast<double *>(base + L.red_off);
  __shared__ alignas(8) uint64_t xbar[4];  // free 1, exchange 1, free 2, exchange 2
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  const uint32_t lane = tid & 31u;
  const int midbits = P.h - P.c;  // local tile number bit of the rank (L0)
  const uint32_t rank = cluster_rank();
  const uint64_t first = cluster_id(), stride = cluster_count(), nunits = P.ntiles >> 1;
  auto tile_of = [&](uint64_t U) -> uint64_t {  // local tile number in L0
    const uint64_t lo = U & ((1ull << midbits) - 1ull);
    return lo | ((uint64_t)rank << midbits) | ((U >> midbits) << (midbits + 1));
  };

  if (PH && P.ph.mode == 0) fill_phase_tab<kThreads>(tab, P.ph);
  if (tid == 0) {
    s_abort = 0;
    mbar_init(full, 1);
    mbar_init(&xbar[0], 8);
    mbar_init(&xbar[1], 1);
    mbar_init(&xbar[2], 8);
    mbar_init(&xbar[3], 1);
    fence_mbar_init();
  }
  __syncthreads();
  cl_arrive();
  cl_wait();
  // the partner's buffers and barriers: mapped at each use (one instruction)
  // rather than held in registers across the tile
  const uint32_t peer = rank ^ 1u;
  auto remote = [&](const void *p) { return mapa(smem_u32(p), peer); };

  // the state halves in L0 (the tile maps of the 2^12 tiles); the cost tile
  // in L0 for lambda = f psi, in L1 for the phase
  auto coords = [&](uint64_t T) {
    TC c;
    c.x1 = (int)(T & ((1ull << midbits) - 1ull));
    c.x2 = 0;
    c.x4 = (int)(T >> midbits);
    return c;
  };
  auto cost_coords = [&](uint64_t U) {
    if constexpr (INIT) return coords(tile_of(U));
    TC c;  // [16][mid][16: tile bits 4..7][tile bit 8][tile bits 9.. and above]
    c.x1 = (int)(U & ((1ull << midbits) - 1ull));
    c.x2 = 0;
    c.x3 = (int)rank;
    c.x4 = (int)((U >> midbits) << 4);
    return c;
  };
  constexpr bool early_cost = (PH && H2 && !INIT) || (INIT && !PH);
  int abort_now = 0;
  auto read_abort = [&]() { abort_now = s_abort; };
  auto issue = [&](uint64_t U, bool cost) {
    const TC c = coords(tile_of(U));
    mbar_expect_tx(full, L.tile_bytes + (INIT ? 0u : L.tile_bytes) + (cost ? L.cost_bytes : 0u));
    tma_load(bv, &P.map_psi, c, full);
    if (!INIT) tma_load(bw, &P.map_lam, c, full);
    if (cost) tma_load(base + L.cost_off, &P.map_cost, cost_coords(U), full);
  };
  auto cost_next = [&](uint64_t U) {
    if (tid == 0 && U + stride < nunits && !abort_now) {
      mbar_add_tx(full, L.cost_bytes);
      tma_load(base + L.cost_off, &P.map_cost, cost_coords(U + stride), full);
    }
  };
  auto release = [&](uint64_t U) {
    cbar();
    if (tid == 0 && U + stride < nunits && !abort_now) issue(U + stride, need_cost && !early_cost);
  };
  auto flag = [&](bool ok) {
    if (!ok) {
      s_abort = 1;
      atomicExch(P.err, 1u);
    }
  };
  // this warp has used what it loaded: the partner may overwrite those slots
  // (dep: computed from every value this thread loaded for the slots)
  const uint32_t zero = rank >> 1;  // 0 in a two-CTA cluster, unknown to the compiler
  auto signal = [&](uint32_t rbar, uint32_t dep) {
    __syncwarp();
    if (lane == 0) mbar_arrive_remote(rbar, dep, zero);
  };

  if (tid == 0 && first < nunits) issue(first, need_cost);

  FF acc1, accg, acc2;
  int i = 0;
  for (;; ++i) {
    const uint64_t U = first + (uint64_t)i * stride;
    if (U >= nunits) break;
    if (abort_now) break;
    const uint64_t T = tile_of(U);
    const uint32_t par = (uint32_t)i & 1u;
    flag(mbar_wait(full, par));
    if (tid == 0) {
      mbar_expect_tx(&xbar[1], kXBytes);
      if constexpr (H2) mbar_expect_tx(&xbar[3], kXBytes);
    }
    float2 v[NREG], w[NREG];
    lds_round<PL, 0, SW>(v, bv);
    if constexpr (INIT) {
      const uint32_t tt = thr_tile<PL, 0>();
#pragma unroll
      for (int r = 0; r < NREG; ++r) {
        const float f = cost_val(P.cost_kind, cb[tt | pdep(r, PL::reg(0))]);
        w[r] = f2(f * v[r].x, f * v[r].y);
      }
    } else {
      lds_round<PL, 0, SW>(w, bw);
    }
    float a1 = 0.f, ag = 0.f, a2 = 0.f;
    unrot_tw<EB, false>(v, w, P.s1.m[0], 0u, P.tau1, P.form1, P.w1[0], a1);
    // a1 now depends on every loaded value when the round rotates anything
    signal(remote(&xbar[0]), P.s1.m[0] ? __float_as_uint(a1) : fold_bits(v, w));
    // L0 -> L1
    const bool fr1 = mbar_wait_cl(&xbar[0], par);
    flag(fr1);
    if (fr1) pair_xchg2<PL, 0>(v, w, bv, bw, remote(bv), remote(bw), remote(&xbar[1]), rank);
    cbar();
    read_abort();
    if constexpr (INIT && early_cost) cost_next(U);
    flag(mbar_wait_cl(&xbar[1], par));
    lds_round<PL, 1, SW>(v, bv);
    lds_round<PL, 1, SW>(w, bw);
    unrot_tw<EB, true>(v, w, P.s1.m[1], P.s1.lm[1], P.tau1, P.form1, P.w1[1], a1);
    if constexpr (H2) signal(remote(&xbar[2]), (P.s1.m[1] | P.s1.lm[1]) ? __float_as_uint(a1) : fold_bits(v, w));
    if constexpr (!PH && !H2) release(U);
    if constexpr (PH) {
      unphase_any<PL, 1>(v, w, cb, P, tab, ag, PairCostIdx());
      if constexpr (!H2) release(U);
    }
    if constexpr (H2) {
      unrot_tw<EB, true>(v, w, P.s2.m[1], P.s2.lm[1], P.tau2, P.form2, P.w2[1], a2);
      // L1 -> L0
      const bool fr2 = mbar_wait_cl(&xbar[2], par);
      flag(fr2);
      if (fr2) pair_xchg_lane<PL>(v, w, bv, bw, remote(bv), remote(bw), remote(&xbar[3]), rank);
      cbar();
      if constexpr (PH && early_cost) cost_next(U);
      flag(mbar_wait_cl(&xbar[3], par));
      lds_round<PL, 0, SW>(v, bv);
      lds_round<PL, 0, SW>(w, bw);
      release(U);
      unrot_tw<EB, false>(v, w, P.s2.m[0], 0u, P.tau2, P.form2, P.w2[0], a2);
      stg_round<PL, 0>(v, P.psi, T, P.h, P.c);
      if (!P.untwist) stg_round<PL, 0>(w, P.lam, T, P.h, P.c);
    } else {
      // store from L1: local position 8 is tile bit 12 (the rank bit of the
      // L0 tile number), tile bit 8 is this CTA's rank
      const uint32_t thr = thr_tile<PL, 1>();
      const uint32_t thr1 = (thr & ~0x100u) | (rank << 8);
      const uint64_t T1 = (T & ~(1ull << midbits)) | ((uint64_t)((thr >> 8) & 1u) << midbits);
      if (P.untwist) {
        // popc of the amplitude index: popc(T1) + popc(thr1) = popc(T) + popc(thr)
        const float2 z = ipow(f2(1.f, 0.f), twist_base<PL, 1>(T));
#pragma unroll
        for (int r = 0; r < NREG; ++r) v[r] = ipow(cmulf(v[r], z), popc_c(r));
      }
      stg_round<PL, 1>(v, P.psi, T1, P.h, P.c, thr1);
      if (!P.untwist) stg_round<PL, 1>(w, P.lam, T1, P.h, P.c, thr1);
    }
    acc1.add(a1);
    accg.add(ag);
    acc2.add(a2);
  }
  drain(abort_now, full, i);
  // Every push the partner makes into this CTA's shared memory is counted on
  // the exchange barriers and waited for within its tile; only a wait that
  // ran out can leave one in flight (the flag is settled: the last tile's
  // last barrier follows every flag write).  Wait for the last tile's
  // exchange phases once more, bounded, so that no remote store is likely to
  // land after this CTA has exited; a partner stalled beyond that means the
  // GPU itself has stopped making progress.
  if (s_abort && i > 0) {
    (void)mbar_wait_cl(&xbar[1], (uint32_t)(i - 1) & 1u);
    if constexpr (H2) (void)mbar_wait_cl(&xbar[3], (uint32_t)(i - 1) & 1u);
  }
  cl_arrive();
  cl_wait();
  double a[3] = {acc1.value(), accg.value(), acc2.value()};
  csum<3>(a, red);
  if (tid == 0) {
    P.partials[blockIdx.x * 3] = a[0];
    P.partials[blockIdx.x * 3 + 1] = a[1];
    P.partials[blockIdx.x * 3 + 2] = a[2];
  }
  double *o1 = P.out_b1, *og = P.out_g, *o2 = P.out_b2;
  final_reduce<3>(P.partials, gridDim.x, P.counter, red, [=](double(&a)[3]) {
    if (o1) *o1 += 2.0 * a[0];
    if (og) *og += 2.0 * a[1];
    if (o2) *o2 += 2.0 * a[2];
  });
}

// ------------------------------------------------------ XY ring mixer passes
//
// The XY gate exp(-i b (X_a X_b + Y_a Y_b) / 2) rotates each pair (u, w) of
// amplitudes whose bits (a, b) are (1, 0) and (0, 1) by
// [[cos b, -i sin b], [-i sin b, cos b]] and leaves the others alone.  As in
// the shared-memory XY kernels it is applied as three shears of the real
// rotation of (u, i w) (t = tan(b/2), s = sin b, b reduced to |b| <= pi/2,
// an exact factor -1 for the rest): every shear has determinant 1, so the
// rounding of t and s cannot make the norm drift over many gates.
__device__ __forceinline__ void xy_gate2(float2 &u, float2 &w, float t, float s, bool neg) {
  const float2 v = f2(-w.y, w.x);  // i w
  const float2 x1 = f2(fmaf(-t, v.x, u.x), fmaf(-t, v.y, u.y));
  float2 y1 = f2(fmaf(s, x1.x, v.x), fmaf(s, x1.y, v.y));
  float2 x2 = f2(fmaf(-t, y1.x, x1.x), fmaf(-t, y1.y, x1.y));
  if (neg) {
    x2 = f2(-x2.x, -x2.y);
    y1 = f2(-y1.x, -y1.y);
  }
  u = x2;
  w = f2(y1.y, -y1.x);  // -i v
}

// The ring gates of one round: for each set bit i of em, the gate on the
// round's register bits (i, i + 1) -- tile bits p + i, p + i + 1 of a round
// whose registers are the 5 consecutive tile bits p.. -- in ascending i, the
// order of the chain.
template <int EB>
__device__ __forceinline__ void xy_round(float2 (&v)[1 << EB], uint32_t em, float t, float s, bool neg) {
#pragma unroll
  for (int i = 0; i + 1 < EB; ++i)
    if ((em >> i) & 1u) {
#pragma unroll
      for (int r = 0; r < (1 << EB); ++r)
        if (((r >> i) & 1) && !((r >> (i + 1)) & 1)) xy_gate2(v[r], v[r ^ (3 << i)], t, s, neg);
    }
}

// The gate (tile bit 12, tile bit 0) after the last round of a pass, where
// tile bit 12 is register bit 4 and tile bit 0 lane bit 0: pair j (register
// bits 0..3) has u = (bit 12 set, bit 0 clear) in the even lane's register
// j + 16 and w = (bit 0 set, bit 12 clear) in the odd lane's register j.
__device__ __forceinline__ void xy_wrap(float2 (&v)[32], float t, float s, bool neg) {
  const bool odd = (threadIdx.x & 1u) != 0u;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const float2 mine = odd ? v[j] : v[j | 16];
    const float2 other = f2(__shfl_xor_sync(0xffffffffu, mine.x, 1), __shfl_xor_sync(0xffffffffu, mine.y, 1));
    float2 u = odd ? other : mine, w = odd ? mine : other;
    xy_gate2(u, w, t, s, neg);
    if (odd)
      v[j] = w;
    else
      v[j | 16] = u;
  }
}

// One XY pass over tiles of 2^13 amplitudes (PL = PlanXyLow: rounds over tile
// bits 0-4, 4-8, 8-12; PlanXyHigh: 4-8, 8-12), streamed like the forward
// passes: persistent CTAs, two per SM, one TMA-loaded tile buffer each, the
// next tile's load issued once the last round's data is in registers, the
// finished tile stored from registers.  PH: the layer's phase exp(-i g f)
// first (round 0, before any gate).
template <class PL, bool PH>
__global__ void __launch_bounds__(kThreads, 2) k_xy_tma(const __grid_constant__ XyTmaParams P) {
  constexpr int NREG = PL::NREG, NR = PL::NR, EB = PL::EB, SW = 128;
  static_assert(EB == 5 && (NR == 2 || NR == 3), "XY plans: 32 amplitudes per thread");
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = aligned_base(smem_raw);
  const Lay L = layout(1u << PL::TB, false, PH);
  float2 *buf = reinterpret_cast<float2 *>(base);
  const CostWord *cb = reinterpret_cast<const CostWord *>(base + L.cost_off);
  float2 *tab = reinterpret_cast<float2 *>(base + L.tab_off);
  uint64_t *full = reinterpret_cast<uint64_t *>(base + L.bar_off);
  const int tid = threadIdx.x;
  const int midbits = P.h - P.c;
  const float t = P.t, s = P.s;
  const bool neg = P.neg != 0;
  __shared__ int s_abort;

  if (PH && P.ph.mode == 0) fill_phase_tab<kThreads>(tab, P.ph);
  if (tid == 0) {
    s_abort = 0;
    mbar_init(full, 1);
    fence_mbar_init();
  }
  __syncthreads();

  auto coords = [&](uint64_t T) {
    const int mid = (int)(T & ((1ull << midbits) - 1ull));
    TC c;
    c.x1 = P.c <= 4 ? mid : 0;
    c.x2 = P.c <= 4 ? 0 : mid;
    c.x4 = (int)(T >> midbits);
    return c;
  };
  int abort_now = 0;  // uniform over the CTA: read after the tile's first barrier
  auto read_abort = [&]() { abort_now = s_abort; };
  auto issue = [&](uint64_t T, bool cost) {
    const TC c = coords(T);
    mbar_expect_tx(full, L.tile_bytes + (cost ? L.cost_bytes : 0u));
    tma_load(buf, &P.map_psi, c, full);
    if (cost) tma_load(base + L.cost_off, &P.map_cost, c, full);
  };
  // the phase reads the costs in round 0: the next tile's costs load at the
  // first barrier, the state at the release
  auto cost_next = [&](uint64_t T) {
    if (tid == 0 && T + gridDim.x < P.ntiles && !abort_now) {
      mbar_add_tx(full, L.cost_bytes);
      tma_load(base + L.cost_off, &P.map_cost, coords(T + gridDim.x), full);
    }
  };
  auto release = [&](uint64_t T) {
    cbar();
    if (tid == 0 && T + gridDim.x < P.ntiles && !abort_now) issue(T + gridDim.x, false);
  };

  if (tid == 0 && blockIdx.x < P.ntiles) issue(blockIdx.x, PH);

  int i = 0;
  for (;; ++i) {
    const uint64_t T = blockIdx.x + (uint64_t)i * gridDim.x;
    if (T >= P.ntiles) break;
    if (abort_now) break;
    if (!mbar_wait(full, i & 1)) {
      s_abort = 1;
      atomicExch(P.err, 1u);
    }
    float2 v[NREG];
    lds_round<PL, 0, SW>(v, buf);
    if constexpr (PH) phase_round<PL, 0>(v, cb, P.ph, P.cost_kind, tab, f2(1.f, 0.f));
    xy_round<EB>(v, P.em[0], t, s, neg);
    if constexpr (PH)
      xp_hook<PL, 0, 1, SW>(v, buf, [&] { read_abort(); cost_next(T); });
    else
      xp_hook<PL, 0, 1, SW>(v, buf, read_abort);
    if constexpr (NR == 2) release(T);
    xy_round<EB>(v, P.em[1], t, s, neg);
    if constexpr (NR == 3) {
      xp<PL, 1, 2, SW>(v, buf);
      release(T);
      xy_round<EB>(v, P.em[2], t, s, neg);
    }
    if (P.wrap) xy_wrap(v, t, s, neg);
    stg_round<PL, NR - 1>(v, P.psi, T, P.h, P.c);
  }
  drain(abort_now, full, i);
}

// ---------------------------------------------------------------- host side

// Shared by both cost widths: defined in the 4-byte compilation only.
#if QAOA_TMA_CW == 4
namespace {

using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                              const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                              const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  }
  return fn;
}

}  // namespace

// 5-D tile view of a 2^n vector of `esz`-byte elements for tiles of 2^tb
// elements with 2^c contiguous ones:
// [2^c][2^(h-c)][256][2^(tb-c-8)][2^(n-h-(tb-c))]; one box = one tile.
cudaError_t make_tile_map(CUtensorMap *map, void *base, int n, int tb, int h, int c, int esz,
                          int swizzle_bytes) {
  EncodeFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t e = (cuuint64_t)esz;
  cuuint64_t dims[5], strides[4];
  cuuint32_t box[5];
  if (c >= 5) {
    // 2^c contiguous amplitudes as [16][2^(c-4)] (a swizzled box row is at
    // most 128 bytes), then the outer bits c..h-1, the rows, the rest
    const int rows = tb - c;
    if (c > 7 || h < c || rows < 1 || rows > 8 || n < h + rows) return cudaErrorInvalidValue;
    const cuuint64_t d[5] = {16, 1ull << (c - 4), 1ull << (h - c), 1ull << rows, 1ull << (n - h - rows)};
    const cuuint64_t st[4] = {16 * e, (1ull << c) * e, (1ull << h) * e, (1ull << (h + rows)) * e};
    const cuuint32_t bx[5] = {16, (cuuint32_t)(1u << (c - 4)), 1, (cuuint32_t)(1u << rows), 1};
    for (int i = 0; i < 5; ++i) dims[i] = d[i], box[i] = bx[i];
    for (int i = 0; i < 4; ++i) strides[i] = st[i];
  } else {
    const int hi = tb - c - 8;  // extra high-segment bits beyond 256 rows
    if (hi < 0 || h < c || n < h + tb - c) return cudaErrorInvalidValue;
    const cuuint64_t d[5] = {1ull << c, 1ull << (h - c), 256, 1ull << hi, 1ull << (n - h - (tb - c))};
    const cuuint64_t st[4] = {(1ull << c) * e, (1ull << h) * e, (1ull << (h + 8)) * e,
                              (1ull << (h + 8 + hi)) * e};
    const cuuint32_t bx[5] = {(cuuint32_t)(1u << c), 1, 256, (cuuint32_t)(1u << hi), 1};
    for (int i = 0; i < 5; ++i) dims[i] = d[i], box[i] = bx[i];
    for (int i = 0; i < 4; ++i) strides[i] = st[i];
  }
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const CUtensorMapDataType dt = esz == 8   ? CU_TENSOR_MAP_DATA_TYPE_UINT64
                                 : esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                            : CU_TENSOR_MAP_DATA_TYPE_UINT32;
  const CUtensorMapSwizzle sw = swizzle_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                      : CU_TENSOR_MAP_SWIZZLE_NONE;
  // L2 promotion no wider than a box row (2^c contiguous elements): wider
  // promotion fetches neighbouring rows that belong to other tiles and are
  // often evicted before those tiles are loaded
  const uint64_t row_bytes = (1ull << c) * e;
  const CUtensorMapL2promotion l2 = row_bytes <= 64    ? CU_TENSOR_MAP_L2_PROMOTION_L2_64B
                                    : row_bytes <= 128 ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B
                                                       : CU_TENSOR_MAP_L2_PROMOTION_L2_256B;
  const CUresult r = fn(map, dt, 5, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, l2,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// [16 elements][2^(h-4)][16: qubits h..h+3][2: qubit h+4][qubits h+5..n-1];
// box [16, 1, 16, 1, 16] (the box's last 16 are qubits h+5..h+8).
cudaError_t make_pair_cost_map(CUtensorMap *map, void *base, int n, int h, int esz) {
  EncodeFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  if (h < 4 || n < h + 9 || (esz != 4 && esz != 2)) return cudaErrorInvalidValue;
  const cuuint64_t e = (cuuint64_t)esz;
  const cuuint64_t dims[5] = {16, 1ull << (h - 4), 16, 2, 1ull << (n - h - 5)};
  const cuuint64_t strides[4] = {16 * e, (1ull << h) * e, (1ull << (h + 4)) * e, (1ull << (h + 5)) * e};
  const cuuint32_t box[5] = {16, 1, 16, 1, 16};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const CUtensorMapDataType dt = esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT32;
  const CUresult r = fn(map, dt, 5, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_64B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

namespace {

// A bounded wait that nothing completes: one arrival that expects 16 bytes
// of transactions, and no copy issued.  Every thread gives up after the
// bounded wait; thread 0 records the flag the workspace check reads.
__global__ void k_wait_selftest(unsigned *err) {
  __shared__ alignas(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_expect_tx(&bar, 16u);
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0);
  if (!ok && threadIdx.x == 0) atomicExch(err, 1u);
}

}  // namespace

cudaError_t launch_wait_selftest(unsigned *err, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(err);
  return cudaGetLastError();
}
#endif  // QAOA_TMA_CW == 4

template <class PL, int K>
static cudaError_t launch_fwd_tma_t(const TmaFwdParams &P, cudaStream_t s, int nsm) {
  const size_t smem = smem_bytes(PL::TB, false, (K & (kPH | kRED)) != 0);
  auto kern = k_fwd_tma<PL, K>;
  static int nb = 0;
  if (nb == 0) {
    const size_t mx = smem_bytes(PL::TB, false, true);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
    if (e != cudaSuccess) return e;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kThreads, mx) != cudaSuccess || b < 1) b = 1;
    nb = b;
  }
  uint64_t grid = (uint64_t)nsm * nb;
  if (grid > P.ntiles) grid = P.ntiles;
  kern<<<(unsigned)grid, kThreads, smem, s>>>(P);
  return cudaGetLastError();
}

template <class PL, int K>
static cudaError_t launch_bwd_tma_t(const TmaBwdParams &P, cudaStream_t s, int nsm) {
  const size_t smem = smem_bytes(PL::TB, true, (K & (kPH | kINIT)) != 0);
  auto kern = k_bwd_tma<PL, K>;
  static int nb = 0;
  if (nb == 0) {
    const size_t mx = smem_bytes(PL::TB, true, true);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
    if (e != cudaSuccess) return e;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, PL::NT, mx) != cudaSuccess || b < 1) b = 1;
    nb = b;
  }
  uint64_t grid = (uint64_t)nsm * nb;
  if (grid > P.ntiles) grid = P.ntiles;
  kern<<<(unsigned)grid, PL::NT, smem, s>>>(P);
  return cudaGetLastError();
}

// Cluster-pair adjoint passes: clusters of two CTAs, as many as fit the GPU
// at once (cudaOccupancyMaxActiveClusters), at most one per cluster tile.
template <int K>
static cudaError_t launch_bwd_pair_t(const TmaBwdParams &P, cudaStream_t s, int nsm) {
  using PL = PlanTmaB12High;
  const size_t smem = smem_bytes(PL::TB, true, (K & (kPH | kINIT)) != 0);
  auto kern = k_bwd_pair<K>;
  static int ncl = 0;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (ncl == 0) {
    const size_t mx = smem_bytes(PL::TB, true, true);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
    if (e != cudaSuccess) return e;
    cfg.gridDim = dim3(2u * (unsigned)nsm, 1, 1);
    cfg.dynamicSmemBytes = mx;
    int c = 0;
    if (cudaOccupancyMaxActiveClusters(&c, kern, &cfg) != cudaSuccess || c < 1) {
      (void)cudaGetLastError();
      c = nsm;
    }
    ncl = c;
  }
  uint64_t clusters = (uint64_t)ncl;
  if (clusters > (P.ntiles >> 1)) clusters = P.ntiles >> 1;
  cfg.gridDim = dim3((unsigned)(2 * clusters), 1, 1);
  cfg.dynamicSmemBytes = smem;
  return cudaLaunchKernelEx(&cfg, kern, P);
}

static cudaError_t dispatch_bwd_pair(const TmaBwdParams &P, cudaStream_t s, int nsm) {
  const bool h2 = (P.s2.m[0] | P.s2.m[1] | P.s2.lm[1]) != 0;
  const int k = (P.has_phase ? kPH : 0) | (h2 ? kH2 : 0) | (P.init_lambda ? kINIT : 0);
  switch (k) {  // the kinds the adjoint schedules produce for HIGH groups
    case 0: return launch_bwd_pair_t<0>(P, s, nsm);
    case kINIT: return launch_bwd_pair_t<kINIT>(P, s, nsm);
    case kPH | kH2: return launch_bwd_pair_t<kPH | kH2>(P, s, nsm);
    case kPH: return launch_bwd_pair_t<kPH>(P, s, nsm);
    default: return cudaErrorInvalidValue;
  }
}

template <class PL>
static cudaError_t dispatch_fwd(const TmaFwdParams &P, cudaStream_t s, int nsm) {
  const bool h1 = (P.s1.m[0] | P.s1.m[1] | P.s1.m[2]) != 0;
  const bool h2 = (P.s2.m[0] | P.s2.m[1] | P.s2.m[2]) != 0;
  const int k = (h1 ? kH1 : 0) | (P.has_phase ? kPH : 0) | (h2 ? kH2 : 0) | (P.reduce ? kRED : 0);
  switch (k) {  // the kinds the forward schedules produce
    case kPH | kH2: return launch_fwd_tma_t<PL, kPH | kH2>(P, s, nsm);
    case kPH | kH2 | kRED: return launch_fwd_tma_t<PL, kPH | kH2 | kRED>(P, s, nsm);
    case kH2: return launch_fwd_tma_t<PL, kH2>(P, s, nsm);
    case kH1 | kPH | kH2: return launch_fwd_tma_t<PL, kH1 | kPH | kH2>(P, s, nsm);
    case kH1: return launch_fwd_tma_t<PL, kH1>(P, s, nsm);
    case kH1 | kRED: return launch_fwd_tma_t<PL, kH1 | kRED>(P, s, nsm);
    default: return cudaErrorInvalidValue;
  }
}

template <class PL>
static cudaError_t dispatch_bwd(const TmaBwdParams &P, cudaStream_t s, int nsm) {
  const bool h2 = (P.s2.m[0] | P.s2.m[1] | P.s2.m[2] | P.s2.lm[0] | P.s2.lm[1] | P.s2.lm[2]) != 0;
  const int k = (P.has_phase ? kPH : 0) | (h2 ? kH2 : 0) | (P.init_lambda ? kINIT : 0);
  switch (k) {  // the kinds the adjoint schedules produce
    case 0: return launch_bwd_tma_t<PL, 0>(P, s, nsm);
    case kINIT: return launch_bwd_tma_t<PL, kINIT>(P, s, nsm);
    case kPH | kH2: return launch_bwd_tma_t<PL, kPH | kH2>(P, s, nsm);
    case kPH: return launch_bwd_tma_t<PL, kPH>(P, s, nsm);
    case kPH | kINIT: return launch_bwd_tma_t<PL, kPH | kINIT>(P, s, nsm);
    default: return cudaErrorInvalidValue;
  }
}

template <class PL, bool PH>
static cudaError_t launch_xy_tma_t(const XyTmaParams &P, cudaStream_t s, int nsm) {
  const size_t smem = smem_bytes(PL::TB, false, PH);
  auto kern = k_xy_tma<PL, PH>;
  static int nb = 0;
  if (nb == 0) {
    const size_t mx = smem_bytes(PL::TB, false, true);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
    if (e != cudaSuccess) return e;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kThreads, mx) != cudaSuccess || b < 1) b = 1;
    nb = b;
  }
  uint64_t grid = (uint64_t)nsm * nb;
  if (grid > P.ntiles) grid = P.ntiles;
  kern<<<(unsigned)grid, kThreads, smem, s>>>(P);
  return cudaGetLastError();
}

#if QAOA_TMA_CW == 2
#define QAOA_TMA_FN(name) name##_u16
#else
#define QAOA_TMA_FN(name) name
#endif

cudaError_t QAOA_TMA_FN(launch_fwd_tma)(const TmaFwdParams &P, bool high, cudaStream_t s, int nsm) {
  if (P.c < 4 || P.c > 6) return cudaErrorInvalidValue;  // 16- to 64-amplitude segments
  if (!P.psi || ((uintptr_t)P.psi & 15u)) return cudaErrorInvalidValue;
  return high ? dispatch_fwd<PlanTmaF13High>(P, s, nsm) : dispatch_fwd<PlanTmaF13Low>(P, s, nsm);
}

cudaError_t QAOA_TMA_FN(launch_xy_tma)(const XyTmaParams &P, bool low, cudaStream_t s, int nsm) {
  if (P.c != 4 || P.h < 4 || !P.psi || ((uintptr_t)P.psi & 15u)) return cudaErrorInvalidValue;
  if (P.em[0] > 0xF || P.em[1] > 0xF || P.em[2] > 0xF || (!low && P.em[2] != 0)) return cudaErrorInvalidValue;
  if (low) return P.has_phase ? launch_xy_tma_t<PlanXyLow, true>(P, s, nsm) : launch_xy_tma_t<PlanXyLow, false>(P, s, nsm);
  if (P.has_phase) return cudaErrorInvalidValue;  // the phase rides on the LOW pass
  return launch_xy_tma_t<PlanXyHigh, false>(P, s, nsm);
}

cudaError_t QAOA_TMA_FN(launch_bwd_tma)(const TmaBwdParams &P, bool high, cudaStream_t s, int nsm) {
  if (P.c < 4 || P.c > 6) return cudaErrorInvalidValue;  // 16- to 64-amplitude segments
  if (!P.psi || !P.lam || ((uintptr_t)P.psi & 15u) || ((uintptr_t)P.lam & 15u))
    return cudaErrorInvalidValue;
  for (int r = 0; r < 3; ++r)  // lane rotations: cluster pairs only, one lane bit per round
    if ((!P.cluster && (P.s1.lm[r] | P.s2.lm[r]) != 0) || __builtin_popcount(P.s1.lm[r]) > 1 ||
        __builtin_popcount(P.s2.lm[r]) > 1)
      return cudaErrorInvalidValue;
  if (P.cluster == 2) {  // a HIGH group of up to 9 qubits on one 512-thread CTA
    if (!high || P.c != 4 || P.h < 4) return cudaErrorInvalidValue;
    return dispatch_bwd<PlanTmaB13High>(P, s, nsm);
  }
  if (P.cluster) {
    // a HIGH group of up to 9 qubits on a pair: 16-amplitude segments,
    // rotations within the two layouts' sets (round 0: 4 register bits;
    // round 1: 4 register bits and lane bit 4), the same set in both
    // sweeps, an even number of local tiles
    const bool s2 = (P.s2.m[0] | P.s2.m[1] | P.s2.lm[1]) != 0;
    auto in_set = [](const Sweep &w) {
      return (w.m[0] & ~0xFu) == 0 && (w.m[1] & ~0xFu) == 0 && w.m[2] == 0 && w.m[3] == 0 &&
             w.lm[0] == 0 && (w.lm[1] & ~0x10u) == 0 && w.lm[2] == 0 && w.lm[3] == 0 &&
             (w.m[0] | w.m[1] | w.lm[1]) != 0;
    };
    if (!high || P.c != 4 || P.h < 4 || P.ntiles < 2 || (P.ntiles & 1) || !in_set(P.s1) ||
        (s2 && (P.s2.m[0] != P.s1.m[0] || P.s2.m[1] != P.s1.m[1] || P.s2.lm[1] != P.s1.lm[1])))
      return cudaErrorInvalidValue;
    return dispatch_bwd_pair(P, s, nsm);
  }
  return high ? dispatch_bwd<PlanTmaB12High>(P, s, nsm) : dispatch_bwd<PlanTmaB12Low>(P, s, nsm);
}

}  // namespace qaoa
