// cost_kernels.cu -- the diagonal cost vector (Sec. 3.1, Eq. 1; Algorithm 3
// step 1) and the reductions over it (cost statistics; standalone energy and
// ground-state overlap).
//
// The paper launches one kernel per term and accumulates in place; here one
// thread owns one basis state x and loops over the terms in registers, so
// the vector is written to HBM exactly once.  Term data sits in the kernel
// parameter block (constant bank): every thread of a warp reads the same
// term, which the constant cache broadcasts.
#include <climits>
#include <type_traits>

#include "qaoa_common.cuh"
#include "kernels.h"

namespace qaoa {

template <typename Idx>
__device__ __forceinline__ int parity(Idx v);
template <>
__device__ __forceinline__ int parity<uint32_t>(uint32_t v) { return __popc(v) & 1; }
template <>
__device__ __forceinline__ int parity<uint64_t>(uint64_t v) { return __popcll(v) & 1; }

template <typename Idx>
__global__ void __launch_bounds__(256) k_terms(const __grid_constant__ TermChunk P) {
  const uint64_t N = 1ull << P.n;
  for (uint64_t x = blockIdx.x * 256ull + threadIdx.x; x < N; x += (uint64_t)gridDim.x * 256ull) {
    const Idx xi = (Idx)x;
    if (P.mode == kTermI32) {
      int32_t acc = P.accumulate ? reinterpret_cast<const int32_t *>(P.out)[x] : 0;
      for (int k = 0; k < P.nterms; ++k) {
        const int32_t w = (int32_t)P.wl[k];
        acc += parity<Idx>(xi & (Idx)P.mask[k]) ? -w : w;
      }
      reinterpret_cast<int32_t *>(P.out)[x] = acc;
    } else if (P.mode == kTermFixed) {
      // exact: weights are integers k * 2^-e, the sum fits 53 bits
      int64_t acc = 0;
      if (P.accumulate) acc = (int64_t)(reinterpret_cast<const double *>(P.out)[x] * P.scale);
      for (int k = 0; k < P.nterms; ++k) {
        const int64_t w = P.wl[k];
        acc += parity<Idx>(xi & (Idx)P.mask[k]) ? -w : w;
      }
      const double v = (double)acc * P.inv_scale;
      if (P.out_kind == kCostF32)
        reinterpret_cast<float *>(P.out)[x] = (float)v;
      else
        reinterpret_cast<double *>(P.out)[x] = v;
    } else {
      // float64 in term order (the same additions, in the same order, as a
      // plain loop over the terms)
      double acc = P.accumulate ? reinterpret_cast<const double *>(P.out)[x] : 0.0;
      for (int k = 0; k < P.nterms; ++k) {
        const double w = P.wd[k];
        acc = parity<Idx>(xi & (Idx)P.mask[k]) ? acc - w : acc + w;
      }
      if (P.out_kind == kCostF32)
        reinterpret_cast<float *>(P.out)[x] = (float)acc;
      else
        reinterpret_cast<double *>(P.out)[x] = acc;
    }
  }
}

// LABS: f(x) = sum_{k=1}^{n-1} C_k^2, C_k = (n - k) - 2 popc((x ^ x >> k) & (2^{n-k} - 1)):
// the aperiodic autocorrelation counts agreeing minus disagreeing pairs.  n is
// a template argument, so the k loop unrolls with constant shifts and masks
// (per k: shift, xor-and, popc and two integer multiply-adds).
template <typename T, int NQ>
__global__ void __launch_bounds__(256) k_labs(T *out) {
  constexpr uint64_t N = 1ull << NQ;
  for (uint64_t x = blockIdx.x * 256ull + threadIdx.x; x < N; x += (uint64_t)gridDim.x * 256ull) {
    const uint32_t xi = (uint32_t)x;
    int32_t f = 0;
#pragma unroll
    for (int k = 1; k < NQ; ++k) {
      const uint32_t m = (NQ - k >= 32) ? 0xffffffffu : ((1u << (NQ - k)) - 1u);
      const int32_t c = (NQ - k) - 2 * __popc((xi ^ (xi >> k)) & m);
      f += c * c;
    }
    out[x] = (T)f;
  }
}

// Element type conversion of a cost vector (int32 <-> uint16; the host has
// checked that every value fits the destination).
template <typename S, typename D>
__global__ void __launch_bounds__(256) k_convert(uint64_t N, const S *src, D *dst) {
  for (uint64_t x = blockIdx.x * 256ull + threadIdx.x; x < N; x += (uint64_t)gridDim.x * 256ull)
    dst[x] = (D)__ldg(src + x);
}

// MaxCut: f(x) = -sum_{(i,j) cut by x} w_ij, accumulated in edge order.
template <typename Idx>
__global__ void __launch_bounds__(256) k_maxcut(const __grid_constant__ EdgeChunk P) {
  const uint64_t N = 1ull << P.n;
  for (uint64_t x = blockIdx.x * 256ull + threadIdx.x; x < N; x += (uint64_t)gridDim.x * 256ull) {
    const Idx xi = (Idx)x;
    if (P.mode == kTermI32) {
      int32_t acc = 0;
      for (int e = 0; e < P.m; ++e)
        if (((xi >> P.ei[e]) ^ (xi >> P.ej[e])) & 1) acc -= (int32_t)P.wl[e];
      reinterpret_cast<int32_t *>(P.out)[x] = acc;
    } else if (P.mode == kTermFixed) {
      int64_t acc = 0;
      for (int e = 0; e < P.m; ++e)
        if (((xi >> P.ei[e]) ^ (xi >> P.ej[e])) & 1) acc -= P.wl[e];
      const double v = (double)acc * P.inv_scale;
      if (P.out_kind == kCostF32)
        reinterpret_cast<float *>(P.out)[x] = (float)v;
      else
        reinterpret_cast<double *>(P.out)[x] = v;
    } else {
      double acc = 0.0;
      for (int e = 0; e < P.m; ++e)
        if (((xi >> P.ei[e]) ^ (xi >> P.ej[e])) & 1) acc = acc - P.wd[e];
      if (P.out_kind == kCostF32)
        reinterpret_cast<float *>(P.out)[x] = (float)acc;
      else
        reinterpret_cast<double *>(P.out)[x] = acc;
    }
  }
}

// ------------------------------------------------------------ reductions

__device__ __forceinline__ double cost_at(const void *cost, int kind, uint64_t x) {
  if (kind == kCostI32) return (double)__ldg(reinterpret_cast<const int *>(cost) + x);
  if (kind == kCostU16) return (double)__ldg(reinterpret_cast<const unsigned short *>(cost) + x);
  if (kind == kCostF32) return (double)__ldg(reinterpret_cast<const float *>(cost) + x);
  return __ldg(reinterpret_cast<const double *>(cost) + x);
}

struct MinMaxCnt {
  double mn, mx, cnt;
};

__device__ __forceinline__ MinMaxCnt mmc_join(MinMaxCnt a, MinMaxCnt b) {
  MinMaxCnt r;
  r.mn = fmin(a.mn, b.mn);
  r.mx = fmax(a.mx, b.mx);
  r.cnt = (a.mn == r.mn ? a.cnt : 0.0) + (b.mn == r.mn ? b.cnt : 0.0);
  return r;
}

// Fixed-shape grid-stride reduction; per-block partials; the last block
// merges them in block order.  out: [f_min, f_max, n_min, step bits], where
// step bits = OR over x of (f[x] - f[0]) for int32 costs (0 otherwise): its
// lowest set bit is the largest power of two dividing every f[x] - f_min.
// One thread's min / max / count-of-min over its elements in the cost's own
// type (integer compares for integer costs, no float64 work per element);
// loads are issued 8 at a time so that enough bytes are in flight.
template <typename T, typename L>
__device__ __forceinline__ MinMaxCnt mmc_scan(const T *c, uint64_t N, L mn_init, L mx_init, uint32_t &bits,
                                              T f0, bool want_bits) {
  L mn = mn_init, mx = mx_init;
  uint32_t cnt = 0u;
  const uint64_t stride = (uint64_t)gridDim.x * 256ull;
  auto take = [&](L f) {
    if (f < mn) {
      mn = f;
      cnt = 0u;
    }
    cnt += f == mn ? 1u : 0u;
    mx = f > mx ? f : mx;
    if (want_bits) bits |= (uint32_t)(int)f - (uint32_t)(int)f0;  // modulo 2^32
  };
  uint64_t x0 = blockIdx.x * 256ull + threadIdx.x;
  for (; x0 + 7 * stride < N; x0 += 8 * stride) {  // whole batches: 8 loads in flight
    T v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __ldg(c + x0 + k * stride);
#pragma unroll
    for (int k = 0; k < 8; ++k) take((L)v[k]);
  }
  for (; x0 < N; x0 += stride) take((L)__ldg(c + x0));
  MinMaxCnt a = {(double)mn, (double)mx, (double)cnt};
  if (cnt == 0u) a = {INFINITY, -INFINITY, 0.0};
  return a;
}

__global__ void __launch_bounds__(256) k_cost_stats(int n, const void *cost, int kind,
                                                   double *partials, unsigned *counter,
                                                   double *out) {
  const uint64_t N = 1ull << n;
  MinMaxCnt a;
  uint32_t bits = 0u;
  if (kind == kCostI32) {
    const int *ci = reinterpret_cast<const int *>(cost);
    a = mmc_scan<int, int>(ci, N, INT_MAX, INT_MIN, bits, __ldg(ci), true);
  } else if (kind == kCostU16) {
    const unsigned short *cu = reinterpret_cast<const unsigned short *>(cost);
    a = mmc_scan<unsigned short, int>(cu, N, INT_MAX, INT_MIN, bits, __ldg(cu), true);
  } else if (kind == kCostF32) {
    a = mmc_scan<float, float>(reinterpret_cast<const float *>(cost), N, INFINITY, -INFINITY, bits, 0.f, false);
  } else {
    a = mmc_scan<double, double>(reinterpret_cast<const double *>(cost), N, INFINITY, -INFINITY, bits, 0.0,
                                 false);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    MinMaxCnt b;
    b.mn = __shfl_down_sync(0xffffffffu, a.mn, o);
    b.mx = __shfl_down_sync(0xffffffffu, a.mx, o);
    b.cnt = __shfl_down_sync(0xffffffffu, a.cnt, o);
    a = mmc_join(a, b);
    bits |= __shfl_down_sync(0xffffffffu, bits, o);
  }
  __shared__ MinMaxCnt sw[8];
  __shared__ uint32_t sb[8];
  __shared__ int am_last;
  if ((threadIdx.x & 31) == 0) {
    sw[threadIdx.x >> 5] = a;
    sb[threadIdx.x >> 5] = bits;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    MinMaxCnt r = sw[0];
    uint32_t rb = sb[0];
    for (int i = 1; i < 8; ++i) {
      r = mmc_join(r, sw[i]);
      rb |= sb[i];
    }
    partials[blockIdx.x * 4 + 0] = r.mn;
    partials[blockIdx.x * 4 + 1] = r.mx;
    partials[blockIdx.x * 4 + 2] = r.cnt;
    partials[blockIdx.x * 4 + 3] = (double)rb;
    __threadfence();
    am_last = (atomicAdd(counter, 1u) == gridDim.x - 1u);
  }
  __syncthreads();
  if (am_last && threadIdx.x == 0) {
    __threadfence();
    MinMaxCnt r = {INFINITY, -INFINITY, 0.0};
    uint32_t rb = 0u;
    for (unsigned b = 0; b < gridDim.x; ++b) {
      MinMaxCnt q = {__ldcg(partials + b * 4), __ldcg(partials + b * 4 + 1), __ldcg(partials + b * 4 + 2)};
      r = mmc_join(r, q);
      rb |= (uint32_t)__ldcg(partials + b * 4 + 3);
    }
    out[0] = r.mn;
    out[1] = r.mx;
    out[2] = r.cnt;
    out[3] = (double)rb;
    *counter = 0u;
  }
}

// Float-float arithmetic for the complex64 reduction: every product exact
// (FMA), sums to about 2^-47 relative.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

struct FFs {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float h, float l) {
    float s, e;
    two_sum(hi, h, s, e);
    e += lo + l;
    hi = s + e;
    lo = e - (hi - s);
  }
};

// Cost value as an unevaluated sum fh + fl of floats (exact for int32,
// uint16 and float32 costs; float64 ones to about 2^-48), and whether it is
// the minimum (compared in the cost's own type).
template <int KIND>
struct CostFF {
  using W = typename std::conditional<KIND == kCostI32, int,
            typename std::conditional<KIND == kCostU16, unsigned short,
            typename std::conditional<KIND == kCostF32, float, double>::type>::type>::type;
  __device__ __forceinline__ static void split(W w, long long fmin_i, double fmin, float &fh, float &fl,
                                               bool &at_min) {
    if constexpr (KIND == kCostI32) {
      fh = (float)w;
      fl = (w < (1 << 24) && w > -(1 << 24)) ? 0.f : (float)((long long)w - (long long)fh);
      at_min = w == fmin_i;
    } else if constexpr (KIND == kCostU16) {
      fh = (float)w;
      fl = 0.f;
      at_min = (int)w == fmin_i;
    } else if constexpr (KIND == kCostF32) {
      fh = w;
      fl = 0.f;
      at_min = w == (float)fmin;
    } else {
      fh = (float)w;
      fl = (float)(w - (double)fh);
      at_min = w == fmin;
    }
  }
};

// Standalone sum_x |psi_x|^2 f_x and sum_{f_x = fmin} |psi_x|^2 (Sec. 3.1,
// Sec. 4) of a complex64 state without float64 work per element: |psi_x|^2
// and its product with f_x formed exactly as float pairs, summed with the
// exact error of every add kept over runs of 32 elements (loads issued 8 at a
// time, two interleaved chains), each run's sum added in float64.
template <int KIND>
__global__ void __launch_bounds__(256) k_expect_c64(int n, const float2 *psi, const void *cost,
                                                   double fmin, double *partials, unsigned *counter,
                                                   double *out, int which) {
  using W = typename CostFF<KIND>::W;
  const W *cw = reinterpret_cast<const W *>(cost);
  const uint64_t N = 1ull << n, stride = (uint64_t)gridDim.x * 256ull;
  const long long fmin_i = (long long)fmin;
  double e = 0.0, o = 0.0;
  // energy chain: the high parts summed in float with the exact rounding error
  // of every add (two_sum) collected, with the low parts, in a second float;
  // read out as sum + low in float64 (only the add into sum is on the chain)
  struct Chain {
    float sum = 0.f, low = 0.f;
    __device__ __forceinline__ void add(float q1, float q2) {
      float t, err;
      two_sum(sum, q1, t, err);
      low += err + q2;
      sum = t;
    }
    __device__ __forceinline__ double value() const { return (double)sum + (double)low; }
  };
  auto take = [&](float2 v, W w, Chain &ce, FFs &fo) {
    const float a1 = v.x * v.x, a2 = fmaf(v.x, v.x, -a1);
    const float b1 = v.y * v.y, b2 = fmaf(v.y, v.y, -b1);
    float p1, p2;
    two_sum(a1, b1, p1, p2);
    p2 += a2 + b2;  // |psi_x|^2 = p1 + p2
    float fh, fl;
    bool at_min;
    CostFF<KIND>::split(w, fmin_i, fmin, fh, fl, at_min);
    const float q1 = p1 * fh;
    const float q2 = fmaf(p1, fh, -q1) + fmaf(p1, fl, p2 * fh);
    ce.add(q1, q2);
    if (at_min) fo.add(p1, p2);
  };
  uint64_t x0 = blockIdx.x * 256ull + threadIdx.x;
  for (; x0 + 31 * stride < N; x0 += 32 * stride) {  // whole runs of 32, 8 loads in flight
    Chain ce[2];  // two energy chains, so that their adds overlap
    FFs fo;
    for (int b = 0; b < 4; ++b) {
      const uint64_t xb = x0 + 8 * b * stride;
      float2 v[8];
      W w[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        v[k] = __ldg(psi + xb + k * stride);
        w[k] = __ldg(cw + xb + k * stride);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) take(v[k], w[k], ce[k & 1], fo);
    }
    e += ce[0].value() + ce[1].value();
    o += (double)fo.hi + (double)fo.lo;
  }
  {
    Chain ce;  // the rest: fewer than 32 elements
    FFs fo;
    for (; x0 < N; x0 += stride) take(__ldg(psi + x0), __ldg(cw + x0), ce, fo);
    e += ce.value();
    o += (double)fo.hi + (double)fo.lo;
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    e += __shfl_down_sync(0xffffffffu, e, s);
    o += __shfl_down_sync(0xffffffffu, o, s);
  }
  __shared__ double se[8], so[8];
  __shared__ int am_last;
  if ((threadIdx.x & 31) == 0) {
    se[threadIdx.x >> 5] = e;
    so[threadIdx.x >> 5] = o;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double te = 0.0, to = 0.0;
    for (int i = 0; i < 8; ++i) {
      te += se[i];
      to += so[i];
    }
    partials[blockIdx.x * 2] = te;
    partials[blockIdx.x * 2 + 1] = to;
    __threadfence();
    am_last = (atomicAdd(counter, 1u) == gridDim.x - 1u);
  }
  __syncthreads();
  if (am_last && threadIdx.x == 0) {
    __threadfence();
    double te = 0.0, to = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) {
      te += __ldcg(partials + b * 2);
      to += __ldcg(partials + b * 2 + 1);
    }
    if (which == 2) {
      out[0] = te;
      out[1] = to;
    } else {
      out[0] = which == 0 ? te : to;
    }
    *counter = 0u;
  }
}

// Standalone sum_x |psi_x|^2 f_x and sum_{f_x = fmin} |psi_x|^2 (Sec. 3.1,
// Sec. 4) of a complex128 state: float64 accumulation, per-block partials
// merged in block order.
template <typename C2>
__global__ void __launch_bounds__(256) k_expect(int n, const C2 *psi, const void *cost, int kind,
                                               double fmin, double *partials, unsigned *counter,
                                               double *out, int which) {
  const uint64_t N = 1ull << n;
  double e = 0.0, o = 0.0;
  for (uint64_t x = blockIdx.x * 256ull + threadIdx.x; x < N; x += (uint64_t)gridDim.x * 256ull) {
    const C2 v = psi[x];
    const double pr = (double)v.x * v.x + (double)v.y * v.y;
    const double f = cost_at(cost, kind, x);
    e += pr * f;
    o += (f == fmin) ? pr : 0.0;
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    e += __shfl_down_sync(0xffffffffu, e, s);
    o += __shfl_down_sync(0xffffffffu, o, s);
  }
  __shared__ double se[8], so[8];
  __shared__ int am_last;
  if ((threadIdx.x & 31) == 0) {
    se[threadIdx.x >> 5] = e;
    so[threadIdx.x >> 5] = o;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double te = 0.0, to = 0.0;
    for (int i = 0; i < 8; ++i) {
      te += se[i];
      to += so[i];
    }
    partials[blockIdx.x * 2] = te;
    partials[blockIdx.x * 2 + 1] = to;
    __threadfence();
    am_last = (atomicAdd(counter, 1u) == gridDim.x - 1u);
  }
  __syncthreads();
  if (am_last && threadIdx.x == 0) {
    __threadfence();
    double te = 0.0, to = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) {
      te += __ldcg(partials + b * 2);
      to += __ldcg(partials + b * 2 + 1);
    }
    if (which == 2) {
      out[0] = te;
      out[1] = to;
    } else {
      out[0] = which == 0 ? te : to;
    }
    *counter = 0u;
  }
}

// ------------------------------------------------------------ launchers

static unsigned grid_for(int n, int nsm, int per_sm) {
  const uint64_t blocks = ((1ull << n) + 255ull) / 256ull;
  const uint64_t cap = (uint64_t)nsm * per_sm;
  return (unsigned)(blocks < cap ? blocks : cap);
}

cudaError_t launch_terms(const TermChunk &P, cudaStream_t s, int nsm) {
  const unsigned grid = grid_for(P.n, nsm, 8);
  if (P.n <= 32)
    k_terms<uint32_t><<<grid, 256, 0, s>>>(P);
  else
    k_terms<uint64_t><<<grid, 256, 0, s>>>(P);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_labs_t(int n, T *out, cudaStream_t s, int nsm) {
  const unsigned grid = grid_for(n, nsm, 8);
  switch (n) {
#define QAOA_LABS_CASE(NQ) \
  case NQ:                 \
    k_labs<T, NQ><<<grid, 256, 0, s>>>(out); \
    break;
    QAOA_LABS_CASE(2) QAOA_LABS_CASE(3) QAOA_LABS_CASE(4) QAOA_LABS_CASE(5) QAOA_LABS_CASE(6)
    QAOA_LABS_CASE(7) QAOA_LABS_CASE(8) QAOA_LABS_CASE(9) QAOA_LABS_CASE(10) QAOA_LABS_CASE(11)
    QAOA_LABS_CASE(12) QAOA_LABS_CASE(13) QAOA_LABS_CASE(14) QAOA_LABS_CASE(15) QAOA_LABS_CASE(16)
    QAOA_LABS_CASE(17) QAOA_LABS_CASE(18) QAOA_LABS_CASE(19) QAOA_LABS_CASE(20) QAOA_LABS_CASE(21)
    QAOA_LABS_CASE(22) QAOA_LABS_CASE(23) QAOA_LABS_CASE(24) QAOA_LABS_CASE(25) QAOA_LABS_CASE(26)
    QAOA_LABS_CASE(27) QAOA_LABS_CASE(28) QAOA_LABS_CASE(29) QAOA_LABS_CASE(30) QAOA_LABS_CASE(31)
    QAOA_LABS_CASE(32)
#undef QAOA_LABS_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_labs(int n, int32_t *out, cudaStream_t s, int nsm) { return launch_labs_t(n, out, s, nsm); }

cudaError_t launch_labs_u16(int n, uint16_t *out, cudaStream_t s, int nsm) {
  return launch_labs_t(n, out, s, nsm);
}

cudaError_t launch_convert(int n, const void *src, int src_kind, void *dst, int dst_kind,
                           cudaStream_t s, int nsm) {
  const uint64_t N = 1ull << n;
  if (src_kind == kCostI32 && dst_kind == kCostU16)
    k_convert<int32_t, uint16_t><<<grid_for(n, nsm, 8), 256, 0, s>>>(
        N, reinterpret_cast<const int32_t *>(src), reinterpret_cast<uint16_t *>(dst));
  else if (src_kind == kCostU16 && dst_kind == kCostI32)
    k_convert<uint16_t, int32_t><<<grid_for(n, nsm, 8), 256, 0, s>>>(
        N, reinterpret_cast<const uint16_t *>(src), reinterpret_cast<int32_t *>(dst));
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_maxcut(const EdgeChunk &P, cudaStream_t s, int nsm) {
  const unsigned grid = grid_for(P.n, nsm, 8);
  if (P.n <= 32)
    k_maxcut<uint32_t><<<grid, 256, 0, s>>>(P);
  else
    k_maxcut<uint64_t><<<grid, 256, 0, s>>>(P);
  return cudaGetLastError();
}

unsigned reduce_grid(int n, int nsm) { return grid_for(n, nsm, 4); }

cudaError_t launch_cost_stats(int n, const void *cost, int kind, double *partials,
                              unsigned *counter, double *out, cudaStream_t s, int nsm) {
  k_cost_stats<<<reduce_grid(n, nsm), 256, 0, s>>>(n, cost, kind, partials, counter, out);
  return cudaGetLastError();
}

// Probabilities |psi_x|^2: into a real array (float for complex64, double for
// complex128), or in place (psi_x <- |psi_x|^2 + 0i).  One amplitude per
// thread-iteration; each thread reads its own amplitude before writing it.
template <typename C2, typename R>
__global__ void __launch_bounds__(256) k_probs(uint64_t N, C2 *psi, R *out) {
  for (uint64_t x = blockIdx.x * 256ull + threadIdx.x; x < N; x += (uint64_t)gridDim.x * 256ull) {
    const C2 a = psi[x];
    const R pr = a.x * a.x + a.y * a.y;
    if (out) {
      out[x] = pr;
    } else {
      C2 z;
      z.x = pr;
      z.y = 0;
      psi[x] = z;
    }
  }
}

cudaError_t launch_probs(int n, void *psi, bool c128, void *out, cudaStream_t s, int nsm) {
  const uint64_t N = 1ull << n;
  if (c128)
    k_probs<double2, double><<<grid_for(n, nsm, 8), 256, 0, s>>>(
        N, reinterpret_cast<double2 *>(psi), reinterpret_cast<double *>(out));
  else
    k_probs<float2, float><<<grid_for(n, nsm, 8), 256, 0, s>>>(
        N, reinterpret_cast<float2 *>(psi), reinterpret_cast<float *>(out));
  return cudaGetLastError();
}

cudaError_t launch_expect(int n, const void *psi, bool c128, const void *cost, int kind,
                          double fmin, double *partials, unsigned *counter, double *out, int which,
                          cudaStream_t s, int nsm) {
  if (c128)
    k_expect<double2><<<reduce_grid(n, nsm), 256, 0, s>>>(
        n, reinterpret_cast<const double2 *>(psi), cost, kind, fmin, partials, counter, out, which);
  else
  {
    const float2 *p = reinterpret_cast<const float2 *>(psi);
    const unsigned g = reduce_grid(n, nsm);
    if (kind == kCostI32) k_expect_c64<kCostI32><<<g, 256, 0, s>>>(n, p, cost, fmin, partials, counter, out, which);
    else if (kind == kCostU16) k_expect_c64<kCostU16><<<g, 256, 0, s>>>(n, p, cost, fmin, partials, counter, out, which);
    else if (kind == kCostF32) k_expect_c64<kCostF32><<<g, 256, 0, s>>>(n, p, cost, fmin, partials, counter, out, which);
    else k_expect_c64<kCostF64><<<g, 256, 0, s>>>(n, p, cost, fmin, partials, counter, out, which);
  }
  return cudaGetLastError();
}

}  // namespace qaoa
