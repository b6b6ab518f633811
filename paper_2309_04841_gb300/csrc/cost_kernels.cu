// cost_kernels.cu -- the diagonal cost vector (Sec. 3.1, Eq. 1; Algorithm 3
// step 1) and the reductions over it (cost statistics; standalone energy and
// ground-state overlap).
//
// The paper launches one kernel per term and accumulates in place; here one
// thread owns one basis state x and loops over the terms in registers, so
// the vector is written to HBM exactly once.  Term data sits in the kernel
// parameter block (constant bank): every thread of a warp reads the same
// term, which the constant cache broadcasts.
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
// the aperiodic autocorrelation counts agreeing minus disagreeing pairs.
template <typename T>
__global__ void __launch_bounds__(256) k_labs(int n, T *out) {
  const uint64_t N = 1ull << n;
  for (uint64_t x = blockIdx.x * 256ull + threadIdx.x; x < N; x += (uint64_t)gridDim.x * 256ull) {
    const uint32_t xi = (uint32_t)x;
    int32_t f = 0;
    for (int k = 1; k < n; ++k) {
      const uint32_t m = (n - k >= 32) ? 0xffffffffu : ((1u << (n - k)) - 1u);
      const int32_t c = (n - k) - 2 * __popc((xi ^ (xi >> k)) & m);
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
__global__ void __launch_bounds__(256) k_cost_stats(int n, const void *cost, int kind,
                                                   double *partials, unsigned *counter,
                                                   double *out) {
  const uint64_t N = 1ull << n;
  MinMaxCnt a = {INFINITY, -INFINITY, 0.0};
  uint32_t bits = 0u;
  const int *ci = reinterpret_cast<const int *>(cost);
  const unsigned short *cu = reinterpret_cast<const unsigned short *>(cost);
  const int f0 = kind == kCostI32 ? __ldg(ci) : kind == kCostU16 ? (int)__ldg(cu) : 0;
  for (uint64_t x = blockIdx.x * 256ull + threadIdx.x; x < N; x += (uint64_t)gridDim.x * 256ull) {
    const double f = cost_at(cost, kind, x);
    MinMaxCnt b = {f, f, 1.0};
    a = mmc_join(a, b);
    if (kind == kCostI32) bits |= (uint32_t)(__ldg(ci + x) - f0);
    if (kind == kCostU16) bits |= (uint32_t)((int)__ldg(cu + x) - f0);
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

// Standalone sum_x |psi_x|^2 f_x and sum_{f_x = fmin} |psi_x|^2 (Sec. 3.1,
// Sec. 4): float64 accumulation, per-block partials merged in block order.
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

cudaError_t launch_labs(int n, int32_t *out, cudaStream_t s, int nsm) {
  k_labs<int32_t><<<grid_for(n, nsm, 8), 256, 0, s>>>(n, out);
  return cudaGetLastError();
}

cudaError_t launch_labs_u16(int n, uint16_t *out, cudaStream_t s, int nsm) {
  k_labs<uint16_t><<<grid_for(n, nsm, 8), 256, 0, s>>>(n, out);
  return cudaGetLastError();
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
    k_expect<float2><<<reduce_grid(n, nsm), 256, 0, s>>>(
        n, reinterpret_cast<const float2 *>(psi), cost, kind, fmin, partials, counter, out, which);
  return cudaGetLastError();
}

}  // namespace qaoa
