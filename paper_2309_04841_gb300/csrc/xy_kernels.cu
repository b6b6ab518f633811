// xy_kernels.cu -- the Hamming-weight-preserving XY mixers (Sec. 3.2: the
// SU(4) extension of Algorithms 1-2) and the Dicke initial state.
//
// One XY gate exp(-i b (X_i X_j + Y_i Y_j) / 2) leaves the basis states whose
// bits i, j are 00 or 11 alone and rotates each pair (bits 10, bits 01) by
// [[cos b, -i sin b], [-i sin b, cos b]] (as three shears, see xy_pair).  A
// layer's mixer is the ordered product of its edge gates, so consecutive
// gates share qubits and must run in order.  k_xy_tile stages a tile of 2^tb amplitudes in shared memory
// (2^c contiguous "passenger" qubits 0..c-1 times rows at qubits h..) and
// applies a run of gates whose qubits all lie in the tile, one after the
// other, with the layer's phase fused into the load of its first pass;
// k_xy_gate applies one gate over the whole state for pairs no tile holds.
#include "qaoa_common.cuh"
#include "kernels.h"

namespace qaoa {

namespace {

template <typename C2> struct XyR;
template <> struct XyR<float2> { using R = float; };
template <> struct XyR<double2> { using R = double; };

template <typename C2>
__device__ __forceinline__ C2 xmk(typename XyR<C2>::R x, typename XyR<C2>::R y) {
  C2 r;
  r.x = x;
  r.y = y;
  return r;
}

template <typename C2>
__device__ __forceinline__ C2 xmul(C2 a, C2 b) {
  return xmk<C2>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// (u, w) <- (cos b u - i sin b w, -i sin b u + cos b w).  With v = i w this is
// the real rotation (u, v) <- (c u - s v, s u + c v), applied as Paeth's three
// shears (t = tan(b/2), s = sin b; b reduced to |b| <= pi/2, the rest an
// exact sign `neg`): every shear has determinant 1, so the rounding of t and
// s adds no systematic growth or decay of the norm over many gates, as a
// rounded (cos, sin) pair would.
template <typename C2, typename R>
__device__ __forceinline__ void xy_pair(C2 &u, C2 &w, R t, R s, bool neg) {
  const C2 v = xmk<C2>(-w.y, w.x);  // i w
  const C2 x1 = xmk<C2>(u.x - t * v.x, u.y - t * v.y);
  C2 y1 = xmk<C2>(v.x + s * x1.x, v.y + s * x1.y);
  C2 x2 = xmk<C2>(x1.x - t * y1.x, x1.y - t * y1.y);
  if (neg) {
    x2 = xmk<C2>(-x2.x, -x2.y);
    y1 = xmk<C2>(-y1.x, -y1.y);
  }
  u = x2;
  w = xmk<C2>(y1.y, -y1.x);  // -i v
}

// k with zero bits inserted at positions lo < hi.
__device__ __forceinline__ uint64_t insert2(uint64_t k, int lo, int hi) {
  k = ((k >> lo) << (lo + 1)) | (k & ((1ull << lo) - 1ull));
  return ((k >> hi) << (hi + 1)) | (k & ((1ull << hi) - 1ull));
}

__device__ __forceinline__ double xy_cost(const void *cost, int kind, uint64_t x) {
  if (kind == kCostI32) return (double)__ldg(reinterpret_cast<const int *>(cost) + x);
  if (kind == kCostU16) return (double)__ldg(reinterpret_cast<const unsigned short *>(cost) + x);
  if (kind == kCostF32) return (double)__ldg(reinterpret_cast<const float *>(cost) + x);
  return __ldg(reinterpret_cast<const double *>(cost) + x);
}

// exp(-i g f_x): complex64 reduces g f / 2pi as a float-float (Dekker's
// two-product by fma) and takes sincospif of the fraction; complex128 reduces
// in float64.
__device__ __forceinline__ float2 xy_phase(const XyPass &P, float2, uint64_t x) {
  const double fd = xy_cost(P.cost, P.cost_kind, x);
  const float fh = (float)fd, fl = (float)(fd - (double)fh);
  const float p = P.g_hi * fh;
  const float e = fmaf(P.g_hi, fh, -p);
  const float r = (p - rintf(p)) + (e + fmaf(P.g_hi, fl, P.g_lo * fh));
  float sn, cs;
  sincospif(2.0f * r, &sn, &cs);
  return make_float2(cs, -sn);
}

__device__ __forceinline__ double2 xy_phase(const XyPass &P, double2, uint64_t x) {
  const double t = P.g2pi * xy_cost(P.cost, P.cost_kind, x);
  const double r = t - rint(t);
  double sn, cs;
  sincospi(2.0 * r, &sn, &cs);
  return make_double2(cs, -sn);
}

// Global index of tile offset t in tile T (bits of t below c are qubits
// 0..c-1, the others qubits h..; T fills the remaining bits in order).
__device__ __forceinline__ uint64_t xy_index(const XyPass &P, uint64_t T, uint32_t t) {
  const int mid = P.h - P.c;
  const uint64_t lo = T & ((1ull << mid) - 1ull), top = T >> mid;
  return (uint64_t)(t & ((1u << P.c) - 1u)) | (lo << P.c) | ((uint64_t)(t >> P.c) << P.h) |
         (top << (P.h + P.tb - P.c));
}

template <typename C2>
__global__ void __launch_bounds__(256) k_xy_tile(const __grid_constant__ XyPass P) {
  using R = typename XyR<C2>::R;
  extern __shared__ __align__(16) unsigned char xy_smem[];
  C2 *s = reinterpret_cast<C2 *>(xy_smem);
  C2 *psi = reinterpret_cast<C2 *>(P.psi);
  const uint32_t TE = 1u << P.tb;
  const R th = (R)P.tb2, sn = (R)P.sb;
  const bool neg = P.neg != 0;
  for (uint64_t T = blockIdx.x; T < P.ntiles; T += gridDim.x) {
    for (uint32_t t = threadIdx.x; t < TE; t += blockDim.x) {
      const uint64_t x = xy_index(P, T, t);
      C2 v = psi[x];
      if (P.has_phase) v = xmul(v, xy_phase(P, v, x));
      s[t] = v;
    }
    __syncthreads();
    for (int g = 0; g < P.ngates; ++g) {
      const int a = P.ga[g], b = P.gb[g];
      const int lo = a < b ? a : b, hi = a < b ? b : a;
      for (uint32_t k = threadIdx.x; k < (TE >> 2); k += blockDim.x) {
        const uint32_t t0 = (uint32_t)insert2(k, lo, hi);
        xy_pair<C2, R>(s[t0 | (1u << a)], s[t0 | (1u << b)], th, sn, neg);
      }
      __syncthreads();
    }
    for (uint32_t t = threadIdx.x; t < TE; t += blockDim.x) psi[xy_index(P, T, t)] = s[t];
    __syncthreads();
  }
}

template <typename C2>
__global__ void __launch_bounds__(256) k_xy_gate(C2 *psi, int n, int i, int j, double tb2, double sb,
                                                int neg) {
  using R = typename XyR<C2>::R;
  const uint64_t K = 1ull << (n - 2);
  const int lo = i < j ? i : j, hi = i < j ? j : i;
  for (uint64_t k = blockIdx.x * 256ull + threadIdx.x; k < K; k += (uint64_t)gridDim.x * 256ull) {
    const uint64_t x0 = insert2(k, lo, hi);
    xy_pair<C2, R>(psi[x0 | (1ull << i)], psi[x0 | (1ull << j)], (R)tb2, (R)sb, neg != 0);
  }
}

// |D^n_k>: amplitude C(n, k)^{-1/2} on every x of Hamming weight k, else 0.
template <typename C2>
__global__ void __launch_bounds__(256) k_dicke(C2 *psi, int n, int k, double amp) {
  using R = typename XyR<C2>::R;
  const uint64_t N = 1ull << n;
  for (uint64_t x = blockIdx.x * 256ull + threadIdx.x; x < N; x += (uint64_t)gridDim.x * 256ull)
    psi[x] = xmk<C2>(__popcll(x) == k ? (R)amp : (R)0, (R)0);
}

unsigned grid_n(uint64_t work, int nsm) {
  const uint64_t b = (work + 255) / 256, cap = (uint64_t)nsm * 8;
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

cudaError_t launch_xy_tile(const XyPass &P, bool c128, cudaStream_t s, int nsm) {
  const size_t smem = ((size_t)1 << P.tb) * (c128 ? 16 : 8);
  static bool init = false;
  if (!init) {
    cudaError_t e = cudaFuncSetAttribute(k_xy_tile<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(((size_t)1 << kXyMaxTb) * 8));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_xy_tile<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(((size_t)1 << kXyMaxTb) * 16));
    if (e != cudaSuccess) return e;
    init = true;
  }
  const uint64_t cap = (uint64_t)nsm * (c128 ? 2 : 4);
  const unsigned grid = (unsigned)(P.ntiles < cap ? P.ntiles : cap);
  if (c128)
    k_xy_tile<double2><<<grid, 256, smem, s>>>(P);
  else
    k_xy_tile<float2><<<grid, 256, smem, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_xy_gate(void *psi, bool c128, int n, int i, int j, double tb2, double sb, int neg,
                           cudaStream_t s, int nsm) {
  const unsigned grid = grid_n(1ull << (n - 2), nsm);
  if (c128)
    k_xy_gate<double2><<<grid, 256, 0, s>>>(reinterpret_cast<double2 *>(psi), n, i, j, tb2, sb, neg);
  else
    k_xy_gate<float2><<<grid, 256, 0, s>>>(reinterpret_cast<float2 *>(psi), n, i, j, tb2, sb, neg);
  return cudaGetLastError();
}

cudaError_t launch_dicke(void *psi, bool c128, int n, int k, double amp, cudaStream_t s, int nsm) {
  const unsigned grid = grid_n(1ull << n, nsm);
  if (c128)
    k_dicke<double2><<<grid, 256, 0, s>>>(reinterpret_cast<double2 *>(psi), n, k, amp);
  else
    k_dicke<float2><<<grid, 256, 0, s>>>(reinterpret_cast<float2 *>(psi), n, k, amp);
  return cudaGetLastError();
}

}  // namespace qaoa
