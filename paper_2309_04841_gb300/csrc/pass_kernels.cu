// pass_kernels.cu -- tiled state-vector passes for sm_103a.
//
// Forward pass (Algorithm 3, one or more of its steps fused):
//   [sweep s1 of X rotations] [phase exp(-i g f)] [sweep s2 of X rotations]
//   [+ energy / ground-state overlap of the result]
// Backward (adjoint) pass on the pair (psi, lambda), un-applying the same
// steps in reverse and accumulating the gradient inner products
//   Im <lambda| X_q |psi>  (d/d beta)   and   Im <lambda| f |psi>  (d/d gamma).
// Each rotation is Algorithm 1 with U = exp(-i b X); a sweep applies it to a
// set of qubits of the tile (Algorithm 2 restricted to the tile window).
//
// Work distribution: persistent CTAs loop over tiles; a tile is read from HBM
// once and written once per pass, every other access is on chip.
#include "qaoa_common.cuh"
#include "kernels.h"

namespace qaoa {

// ----------------------------------------------------------- small helpers

template <typename C2> struct Scal;
template <> struct Scal<float2> { using R = float; };
template <> struct Scal<double2> { using R = double; };

template <typename C2>
__device__ __forceinline__ C2 mk(typename Scal<C2>::R x, typename Scal<C2>::R y) {
  C2 r;
  r.x = x;
  r.y = y;
  return r;
}

template <typename C2>
__device__ __forceinline__ C2 cmul(C2 a, C2 b) {
  return mk<C2>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float fmx(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmx(double a, double b, double c) { return fma(a, b, c); }

// exp(-i b X) on one amplitude pair (Algorithm 1 with a = cos b, b = -i sin b)
// divided by a real factor, so that each component takes one fused
// multiply-add: form 0, factor cos b, t = tan b:
//   (a, b) <- (a - i t b, b - i t a);
// form 1, factor sin b, t = cot b:
//   (a, b) <- (t a - i b, t b - i a).
// The host picks the form with |t| <= 1 and carries the product of the
// dropped factors (PassOp scales in the tiled schedules).
template <int FORM, typename C2, typename Real>
__device__ __forceinline__ void rot_tan(C2 &a, C2 &b, Real t) {
  C2 na, nb;
  if constexpr (FORM == 0) {
    na = mk<C2>(fmx(t, b.y, a.x), fmx(-t, b.x, a.y));
    nb = mk<C2>(fmx(t, a.y, b.x), fmx(-t, a.x, b.y));
  } else {
    na = mk<C2>(fmx(t, a.x, b.y), fmx(t, a.y, -b.x));
    nb = mk<C2>(fmx(t, b.x, a.y), fmx(t, b.y, -a.x));
  }
  a = na;
  b = nb;
}

__device__ __forceinline__ uint32_t pdep_rt(uint32_t v, uint32_t mask) {
  uint32_t out = 0;
  int k = 0;
#pragma unroll
  for (int b = 0; b < 32; ++b) {
    if ((mask >> b) & 1u) {
      out |= ((v >> k) & 1u) << b;
      ++k;
    }
  }
  return out;
}

template <class PL, int R>
__device__ __forceinline__ uint32_t thr_toff() {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  return pdep_rt(lane, PL::lane(R)) | pdep_rt(warp, PL::warp(R));
}

template <class PL, typename C2>
__device__ __forceinline__ uint32_t swz(uint32_t t) {
  constexpr uint32_t m = sizeof(C2) == 8 ? 15u : 7u;
  return t ^ ((t >> PL::SWS) & m);
}

template <class PL, int RF, int RT, typename C2>
__device__ __forceinline__ void xpose(C2 (&v)[PL::NREG], C2 *tile) {
  const uint32_t tf = thr_toff<PL, RF>();
#pragma unroll
  for (int r = 0; r < PL::NREG; ++r) tile[swz<PL, C2>(tf | pdep(r, PL::reg(RF)))] = v[r];
  __syncthreads();
  const uint32_t tt = thr_toff<PL, RT>();
#pragma unroll
  for (int r = 0; r < PL::NREG; ++r) v[r] = tile[swz<PL, C2>(tt | pdep(r, PL::reg(RT)))];
}

template <class PL, int RF, int RT, typename C2>
__device__ __forceinline__ void xpose2(C2 (&v)[PL::NREG], C2 (&w)[PL::NREG], C2 *tv,
                                       C2 *tw) {
  const uint32_t tf = thr_toff<PL, RF>();
#pragma unroll
  for (int r = 0; r < PL::NREG; ++r) {
    const uint32_t s = swz<PL, C2>(tf | pdep(r, PL::reg(RF)));
    tv[s] = v[r];
    tw[s] = w[r];
  }
  __syncthreads();
  const uint32_t tt = thr_toff<PL, RT>();
#pragma unroll
  for (int r = 0; r < PL::NREG; ++r) {
    const uint32_t s = swz<PL, C2>(tt | pdep(r, PL::reg(RT)));
    v[r] = tv[s];
    w[r] = tw[s];
  }
}

template <int EB, int FORM, typename C2, typename Real>
__device__ __forceinline__ void rot_regs_f(C2 (&v)[1 << EB], uint32_t m, Real t) {
#pragma unroll
  for (int i = 0; i < EB; ++i) {
    if ((m >> i) & 1u) {
#pragma unroll
      for (int r = 0; r < (1 << EB); ++r)
        if (!((r >> i) & 1)) rot_tan<FORM>(v[r], v[r | (1 << i)], t);
    }
  }
}

template <int EB, typename C2, typename Real>
__device__ __forceinline__ void rot_regs(C2 (&v)[1 << EB], uint32_t m, Real t, int form) {
  if (form == 0)
    rot_regs_f<EB, 0>(v, m, t);
  else
    rot_regs_f<EB, 1>(v, m, t);
}

// Un-rotate psi (v) and lambda (w) on the masked register bits, first adding
// Im[conj(l_a) p_b + conj(l_b) p_a] = Im <lambda| X_q |psi> of every masked
// pair: the value does not change under common X rotations, and taking all of
// them before the round's rotations puts them at one scale, which wgt (the
// round's sigma^2) converts back.
template <int EB, typename C2, typename Real>
__device__ __forceinline__ void unrot_regs_acc(C2 (&v)[1 << EB], C2 (&w)[1 << EB], uint32_t m,
                                               Real t, int form, Real wgt, Real &acc) {
  Real g[2] = {0, 0};
#pragma unroll
  for (int i = 0; i < EB; ++i) {
    if ((m >> i) & 1u) {
#pragma unroll
      for (int r = 0; r < (1 << EB); ++r) {
        if (!((r >> i) & 1)) {
          const C2 pa = v[r], pb = v[r | (1 << i)], la = w[r], lb = w[r | (1 << i)];
          const int k = (r >> (i == 0 ? 1 : 0)) & 1;
          g[k] = fmx(la.x, pb.y, g[k]);
          g[k] = fmx(-la.y, pb.x, g[k]);
          g[k] = fmx(lb.x, pa.y, g[k]);
          g[k] = fmx(-lb.y, pa.x, g[k]);
        }
      }
    }
  }
  acc = fmx(g[0] + g[1], wgt, acc);
  rot_regs<EB>(v, m, t, form);
  rot_regs<EB>(w, m, t, form);
}

// Cost value as a float pair hi + lo (exact for int32 and float32 costs,
// ~2^-48 relative for float64 costs).
__device__ __forceinline__ void cost_split(const void *cost, int kind, uint64_t x, float &hi,
                                           float &lo) {
  if (kind == kCostI32) {
    const int f = __ldg(reinterpret_cast<const int *>(cost) + x);
    hi = (float)f;
    lo = (float)((long long)f - (long long)hi);
  } else if (kind == kCostU16) {
    hi = (float)__ldg(reinterpret_cast<const unsigned short *>(cost) + x);
    lo = 0.f;
  } else if (kind == kCostF32) {
    hi = __ldg(reinterpret_cast<const float *>(cost) + x);
    lo = 0.f;
  } else {
    const double f = __ldg(reinterpret_cast<const double *>(cost) + x);
    hi = (float)f;
    lo = (float)(f - (double)hi);
  }
}

__device__ __forceinline__ double cost_d(const void *cost, int kind, uint64_t x) {
  if (kind == kCostI32) return (double)__ldg(reinterpret_cast<const int *>(cost) + x);
  if (kind == kCostU16) return (double)__ldg(reinterpret_cast<const unsigned short *>(cost) + x);
  if (kind == kCostF32) return (double)__ldg(reinterpret_cast<const float *>(cost) + x);
  return __ldg(reinterpret_cast<const double *>(cost) + x);
}

// exp(-i g f_x) for the layer described by ph (tables already in smem).
__device__ __forceinline__ float2 phase_factor(const PhaseData<float> &ph, const float2 *tlo,
                                               const float2 *thi, const void *cost, int kind,
                                               uint64_t x) {
  if (ph.mode == 0) {
    const int f = kind == kCostU16 ? (int)__ldg(reinterpret_cast<const unsigned short *>(cost) + x)
                                   : __ldg(reinterpret_cast<const int *>(cost) + x);
    const uint32_t v = (uint32_t)(f - ph.fmin);
    const uint32_t hi = min(v >> 8, 255u);
    return cmul(thi[hi], tlo[v & 255u]);
  }
  // g f / 2pi as a float-float: p + e = g_hi * f_hi exactly (Dekker's
  // two-product via fma), the small cross terms added once; only the
  // fraction r in [-1/2, 1/2] reaches sincospi.
  float fh, fl;
  cost_split(cost, kind, x, fh, fl);
  const float p = ph.g_hi * fh;
  const float e = fmaf(ph.g_hi, fh, -p);
  const float r = (p - rintf(p)) + (e + fmaf(ph.g_hi, fl, ph.g_lo * fh));
  float sn, cs;
  sincospif(2.0f * r, &sn, &cs);
  return make_float2(cs * ph.scl, -sn * ph.scl);
}

__device__ __forceinline__ double2 phase_factor(const PhaseData<double> &ph, const double2 *tlo,
                                                const double2 *thi, const void *cost, int kind,
                                                uint64_t x) {
  if (ph.mode == 0) {
    const int f = kind == kCostU16 ? (int)__ldg(reinterpret_cast<const unsigned short *>(cost) + x)
                                   : __ldg(reinterpret_cast<const int *>(cost) + x);
    const uint32_t v = (uint32_t)(f - ph.fmin);
    const uint32_t hi = min(v >> 8, 255u);
    return cmul(thi[hi], tlo[v & 255u]);
  }
  const double t = ph.g2pi * cost_d(cost, kind, x);
  const double r = t - rint(t);
  double sn, cs;
  sincospi(2.0 * r, &sn, &cs);
  return make_double2(cs * ph.scl, -sn * ph.scl);
}

template <class PL, int R, typename Real, typename C2>
__device__ __forceinline__ void apply_phase(C2 (&v)[PL::NREG], const PhaseData<Real> &ph,
                                            const C2 *tlo, const C2 *thi, const void *cost,
                                            int kind, const Geom &g, uint64_t base) {
  const uint64_t xt = base + tile_off(g, thr_toff<PL, R>());
#pragma unroll
  for (int r = 0; r < PL::NREG; ++r) {
    const uint64_t x = xt + tile_off(g, pdep(r, PL::reg(R)));
    v[r] = cmul(v[r], phase_factor(ph, tlo, thi, cost, kind, x));
  }
}

template <class PL, int R, typename C2>
__device__ __forceinline__ void load_tile(C2 (&v)[PL::NREG], const C2 *__restrict__ src,
                                          const Geom &g, uint64_t base) {
  const uint64_t xt = base + tile_off(g, thr_toff<PL, R>());
#pragma unroll
  for (int r = 0; r < PL::NREG; ++r) v[r] = src[xt + tile_off(g, pdep(r, PL::reg(R)))];
}

template <class PL, int R, typename C2>
__device__ __forceinline__ void store_tile(const C2 (&v)[PL::NREG], C2 *__restrict__ dst,
                                           const Geom &g, uint64_t base) {
  const uint64_t xt = base + tile_off(g, thr_toff<PL, R>());
#pragma unroll
  for (int r = 0; r < PL::NREG; ++r) dst[xt + tile_off(g, pdep(r, PL::reg(R)))] = v[r];
}

// Energy and overlap terms of this thread's amplitudes in round-R layout.
template <class PL, int R, typename C2>
__device__ __forceinline__ void accum_eo(const C2 (&v)[PL::NREG], const void *cost, int kind,
                                         double fmin, const Geom &g, uint64_t base,
                                         typename Scal<C2>::R &e, typename Scal<C2>::R &o) {
  using Real = typename Scal<C2>::R;
  const uint64_t xt = base + tile_off(g, thr_toff<PL, R>());
#pragma unroll
  for (int r = 0; r < PL::NREG; ++r) {
    const uint64_t x = xt + tile_off(g, pdep(r, PL::reg(R)));
    const double f = cost_d(cost, kind, x);
    const Real pr = v[r].x * v[r].x + v[r].y * v[r].y;
    e += pr * (Real)f;
    o += (f == fmin) ? pr : (Real)0;
  }
}

// Deterministic block sum of K doubles (fixed shuffle tree, fixed warp order).
// Result valid in thread 0.  `red` holds NT/32 * K doubles.
template <int NT, int K>
__device__ __forceinline__ void block_sum(double (&a)[K], double *red) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_down_sync(0xffffffffu, a[k], o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) red[w * K + k] = a[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int i = 0; i < NT / 32; ++i) s += red[i * K + k];
      a[k] = s;
    }
  }
  __syncthreads();
}

// Last CTA to arrive sums the per-tile partials [ntiles][K] in a fixed order
// and hands the K totals to `fin` in thread 0.  The counter returns to 0.
template <int NT, int K, class Fin>
__device__ __forceinline__ void last_block_reduce(const double *partials, uint64_t ntiles,
                                                  unsigned *counter, double *red, Fin fin) {
  __shared__ int am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(counter, 1u);
    am_last = (prev == gridDim.x - 1u);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  double a[K];
#pragma unroll
  for (int k = 0; k < K; ++k) a[k] = 0.0;
  for (uint64_t t = threadIdx.x; t < ntiles; t += NT) {
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] += __ldcg(partials + t * K + k);
  }
  block_sum<NT, K>(a, red);
  if (threadIdx.x == 0) {
    fin(a);
    *counter = 0u;
  }
}

// ------------------------------------------------------------ forward pass

template <class PL, typename Real>
__global__ void __launch_bounds__(PL::NT, 2) k_fwd(const __grid_constant__ FwdParams<Real> P) {
  using C2 = typename C2T<Real>::type;
  constexpr int NREG = PL::NREG, NR = PL::NR, EB = PL::EB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2 *tile = reinterpret_cast<C2 *>(smem_raw);
  C2 *tlo = tile + (1 << PL::TB);
  C2 *thi = tlo + 256;
  double *red = reinterpret_cast<double *>(thi + 256);

  if (P.has_phase && P.ph.mode == 0) {
    for (int i = threadIdx.x; i < 256; i += PL::NT) {
      tlo[i] = P.ph.tab_lo[i];
      thi[i] = P.ph.tab_hi[i];
    }
  }
  const Geom g = P.g;
  const bool has1 = (P.s1.m[0] | P.s1.m[1] | P.s1.m[2]) != 0;
  const bool has2 = (P.s2.m[0] | P.s2.m[1] | P.s2.m[2]) != 0;

  for (uint64_t T = blockIdx.x; T < g.ntiles; T += gridDim.x) {
    const uint64_t base = tile_base(g, T);
    __syncthreads();
    C2 v[NREG];
    if (P.init_plus) {
#pragma unroll
      for (int r = 0; r < NREG; ++r) v[r] = mk<C2>(P.amp, (Real)0);
    } else {
      load_tile<PL, 0>(v, P.psi, g, base);
    }
    bool final0;
    if (has1) {
      rot_regs<EB>(v, P.s1.m[0], P.t1, P.form1);
      xpose<PL, 0, 1>(v, tile);
      rot_regs<EB>(v, P.s1.m[1], P.t1, P.form1);
      if constexpr (NR == 3) {
        xpose<PL, 1, 2>(v, tile);
        rot_regs<EB>(v, P.s1.m[2], P.t1, P.form1);
      }
      if (P.has_phase) apply_phase<PL, NR - 1>(v, P.ph, tlo, thi, P.cost, P.cost_kind, g, base);
      if (has2) {
        rot_regs<EB>(v, P.s2.m[NR - 1], P.t2, P.form2);
        if constexpr (NR == 3) {
          xpose<PL, 2, 1>(v, tile);
          rot_regs<EB>(v, P.s2.m[1], P.t2, P.form2);
        }
        xpose<PL, 1, 0>(v, tile);
        rot_regs<EB>(v, P.s2.m[0], P.t2, P.form2);
        final0 = true;
      } else {
        final0 = false;
      }
    } else {
      if (P.has_phase) apply_phase<PL, 0>(v, P.ph, tlo, thi, P.cost, P.cost_kind, g, base);
      rot_regs<EB>(v, P.s2.m[0], P.t2, P.form2);
      xpose<PL, 0, 1>(v, tile);
      rot_regs<EB>(v, P.s2.m[1], P.t2, P.form2);
      if constexpr (NR == 3) {
        xpose<PL, 1, 2>(v, tile);
        rot_regs<EB>(v, P.s2.m[2], P.t2, P.form2);
      }
      final0 = false;
    }
    if (P.post_scale != (Real)1) {
#pragma unroll
      for (int r = 0; r < NREG; ++r) v[r] = mk<C2>(v[r].x * P.post_scale, v[r].y * P.post_scale);
    }
    if (P.reduce) {
      Real e = 0, o = 0;
      if (final0)
        accum_eo<PL, 0>(v, P.cost, P.cost_kind, P.fmin_d, g, base, e, o);
      else
        accum_eo<PL, NR - 1>(v, P.cost, P.cost_kind, P.fmin_d, g, base, e, o);
      double a[2] = {(double)e, (double)o};
      block_sum<PL::NT, 2>(a, red);
      if (threadIdx.x == 0) {
        P.partials[T * 2 + 0] = a[0];
        P.partials[T * 2 + 1] = a[1];
      }
    }
    if (final0)
      store_tile<PL, 0>(v, P.psi, g, base);
    else
      store_tile<PL, NR - 1>(v, P.psi, g, base);
  }
  if (P.reduce) {
    double *out = P.out;
    last_block_reduce<PL::NT, 2>(P.partials, g.ntiles, P.counter, red, [out](double(&a)[2]) {
      out[0] = a[0];
      out[1] = a[1];
    });
  }
}

// ----------------------------------------------------------- backward pass

template <class PL, typename Real>
__global__ void __launch_bounds__(PL::NT, 2) k_bwd(const __grid_constant__ BwdParams<Real> P) {
  using C2 = typename C2T<Real>::type;
  constexpr int NREG = PL::NREG, NR = PL::NR, EB = PL::EB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2 *tv = reinterpret_cast<C2 *>(smem_raw);
  C2 *tw = tv + (1 << PL::TB);
  C2 *tlo = tw + (1 << PL::TB);
  C2 *thi = tlo + 256;
  double *red = reinterpret_cast<double *>(thi + 256);

  if (P.has_phase && P.ph.mode == 0) {
    for (int i = threadIdx.x; i < 256; i += PL::NT) {
      tlo[i] = P.ph.tab_lo[i];
      thi[i] = P.ph.tab_hi[i];
    }
  }
  const Geom g = P.g;
  const bool has1 = (P.s1.m[0] | P.s1.m[1] | P.s1.m[2]) != 0;
  const bool has2 = (P.s2.m[0] | P.s2.m[1] | P.s2.m[2]) != 0;

  for (uint64_t T = blockIdx.x; T < g.ntiles; T += gridDim.x) {
    const uint64_t base = tile_base(g, T);
    __syncthreads();
    C2 v[NREG], w[NREG];
    load_tile<PL, 0>(v, P.psi, g, base);
    if (P.init_lambda) {
      // lambda = f psi: the gradient of E = <psi|f|psi> with respect to psi^*
      const uint64_t xt = base + tile_off(g, thr_toff<PL, 0>());
#pragma unroll
      for (int r = 0; r < NREG; ++r) {
        const Real f = (Real)cost_d(P.cost, P.cost_kind, xt + tile_off(g, pdep(r, PL::reg(0))));
        w[r] = mk<C2>(f * v[r].x, f * v[r].y);
      }
    } else {
      load_tile<PL, 0>(w, P.lam, g, base);
    }
    Real a1 = 0, ag = 0, a2 = 0;
    // sweep 1 ascending through the rounds
    unrot_regs_acc<EB>(v, w, P.s1.m[0], P.t1, P.form1, P.w1[0], a1);
    xpose2<PL, 0, 1>(v, w, tv, tw);
    unrot_regs_acc<EB>(v, w, P.s1.m[1], P.t1, P.form1, P.w1[1], a1);
    if constexpr (NR == 3) {
      xpose2<PL, 1, 2>(v, w, tv, tw);
      unrot_regs_acc<EB>(v, w, P.s1.m[2], P.t1, P.form1, P.w1[2], a1);
    }
    if (P.has_phase) {
      // d/d gamma: Im <lambda| f |psi>, then un-phase both vectors
      const uint64_t xt = base + tile_off(g, thr_toff<PL, NR - 1>());
      Real raw = 0;
#pragma unroll
      for (int r = 0; r < NREG; ++r) {
        const uint64_t x = xt + tile_off(g, pdep(r, PL::reg(NR - 1)));
        const Real f = (Real)cost_d(P.cost, P.cost_kind, x);
        raw += f * (w[r].x * v[r].y - w[r].y * v[r].x);
        const C2 ph = phase_factor(P.ph, tlo, thi, P.cost, P.cost_kind, x);
        v[r] = cmul(v[r], ph);
        w[r] = cmul(w[r], ph);
      }
      ag = raw * P.wg;
    }
    bool final0 = false;
    if (has2) {
      unrot_regs_acc<EB>(v, w, P.s2.m[NR - 1], P.t2, P.form2, P.w2[NR - 1], a2);
      if constexpr (NR == 3) {
        xpose2<PL, 2, 1>(v, w, tv, tw);
        unrot_regs_acc<EB>(v, w, P.s2.m[1], P.t2, P.form2, P.w2[1], a2);
      }
      xpose2<PL, 1, 0>(v, w, tv, tw);
      unrot_regs_acc<EB>(v, w, P.s2.m[0], P.t2, P.form2, P.w2[0], a2);
      final0 = true;
    }
    (void)has1;
    double a[3] = {(double)a1, (double)ag, (double)a2};
    block_sum<PL::NT, 3>(a, red);
    if (threadIdx.x == 0) {
      P.partials[T * 3 + 0] = a[0];
      P.partials[T * 3 + 1] = a[1];
      P.partials[T * 3 + 2] = a[2];
    }
    if (P.post_scale != (Real)1) {
#pragma unroll
      for (int r = 0; r < NREG; ++r) {
        v[r] = mk<C2>(v[r].x * P.post_scale, v[r].y * P.post_scale);
        w[r] = mk<C2>(w[r].x * P.post_scale, w[r].y * P.post_scale);
      }
    }
    if (final0) {
      store_tile<PL, 0>(v, P.psi, g, base);
      store_tile<PL, 0>(w, P.lam, g, base);
    } else {
      store_tile<PL, NR - 1>(v, P.psi, g, base);
      store_tile<PL, NR - 1>(w, P.lam, g, base);
    }
  }
  double *o1 = P.out_b1, *og = P.out_g, *o2 = P.out_b2;
  last_block_reduce<PL::NT, 3>(P.partials, g.ntiles, P.counter, red, [=](double(&a)[3]) {
    if (o1) *o1 += 2.0 * a[0];
    if (og) *og += 2.0 * a[1];
    if (o2) *o2 += 2.0 * a[2];
  });
}

// ---------------------------------------------------------------- launchers

template <class K>
static int blocks_per_sm(K kernel, int nt, size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, nt, smem) != cudaSuccess) return 1;
  return nb < 1 ? 1 : nb;
}

template <class PL, typename Real>
static cudaError_t launch_fwd_t(const FwdParams<Real> &P, cudaStream_t s, int nsm) {
  using C2 = typename C2T<Real>::type;
  const size_t smem = ((size_t)(1 << PL::TB) + 512) * sizeof(C2) + (PL::NT / 32) * 3 * sizeof(double);
  auto kern = k_fwd<PL, Real>;
  static int nb = -1;  // per instantiation; the device is fixed per process
  if (nb < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    nb = blocks_per_sm(kern, PL::NT, smem);
  }
  uint64_t grid = (uint64_t)nsm * nb;
  if (grid > P.g.ntiles) grid = P.g.ntiles;
  kern<<<(unsigned)grid, PL::NT, smem, s>>>(P);
  return cudaGetLastError();
}

template <class PL, typename Real>
static cudaError_t launch_bwd_t(const BwdParams<Real> &P, cudaStream_t s, int nsm) {
  using C2 = typename C2T<Real>::type;
  const size_t smem = ((size_t)(2 << PL::TB) + 512) * sizeof(C2) + (PL::NT / 32) * 3 * sizeof(double);
  auto kern = k_bwd<PL, Real>;
  static int nb = -1;
  if (nb < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    nb = blocks_per_sm(kern, PL::NT, smem);
  }
  uint64_t grid = (uint64_t)nsm * nb;
  if (grid > P.g.ntiles) grid = P.g.ntiles;
  kern<<<(unsigned)grid, PL::NT, smem, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_fwd(const FwdParams<float> &P, bool high, int tb, cudaStream_t s, int nsm) {
  if (tb != PlanF13Low::TB) return cudaErrorInvalidValue;
  return high ? launch_fwd_t<PlanF13High, float>(P, s, nsm) : launch_fwd_t<PlanF13Low, float>(P, s, nsm);
}
cudaError_t launch_fwd(const FwdParams<double> &P, bool high, int tb, cudaStream_t s, int nsm) {
  switch (tb) {
    case 9:
      return high ? launch_fwd_t<PlanT9High, double>(P, s, nsm) : launch_fwd_t<PlanT9Low, double>(P, s, nsm);
    case 10:
      return high ? launch_fwd_t<PlanT10High, double>(P, s, nsm) : launch_fwd_t<PlanT10Low, double>(P, s, nsm);
    case 12:
      return high ? launch_fwd_t<PlanT12High, double>(P, s, nsm) : launch_fwd_t<PlanT12Low, double>(P, s, nsm);
    default:
      return cudaErrorInvalidValue;
  }
}
cudaError_t launch_bwd(const BwdParams<float> &P, bool high, int tb, cudaStream_t s, int nsm) {
  if (tb != PlanT12Low::TB) return cudaErrorInvalidValue;
  return high ? launch_bwd_t<PlanT12High, float>(P, s, nsm) : launch_bwd_t<PlanT12Low, float>(P, s, nsm);
}
cudaError_t launch_bwd(const BwdParams<double> &P, bool high, int tb, cudaStream_t s, int nsm) {
  switch (tb) {
    case 9:
      return high ? launch_bwd_t<PlanT9High, double>(P, s, nsm) : launch_bwd_t<PlanT9Low, double>(P, s, nsm);
    case 10:
      return high ? launch_bwd_t<PlanT10High, double>(P, s, nsm) : launch_bwd_t<PlanT10Low, double>(P, s, nsm);
    case 11:
      return high ? launch_bwd_t<PlanT11High, double>(P, s, nsm) : launch_bwd_t<PlanT11Low, double>(P, s, nsm);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace qaoa
