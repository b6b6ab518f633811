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

// Two neighbouring amplitudes (p 16-byte aligned): one 16-byte access for
// complex64.
__device__ __forceinline__ void ld2(const float2 *p, float2 &a, float2 &b) {
  const float4 q = *reinterpret_cast<const float4 *>(p);
  a = make_float2(q.x, q.y);
  b = make_float2(q.z, q.w);
}
__device__ __forceinline__ void ld2(const double2 *p, double2 &a, double2 &b) {
  a = p[0];
  b = p[1];
}
__device__ __forceinline__ void st2(float2 *p, float2 a, float2 b) {
  *reinterpret_cast<float4 *>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st2(double2 *p, double2 a, double2 b) {
  p[0] = a;
  p[1] = b;
}

// k with zero bits inserted at positions lo < hi (32-bit: tile offsets).
__device__ __forceinline__ uint32_t insert2_32(uint32_t k, int lo, int hi) {
  k = ((k >> lo) << (lo + 1)) | (k & ((1u << lo) - 1u));
  return ((k >> hi) << (hi + 1)) | (k & ((1u << hi) - 1u));
}

// The same for global indices.
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

// exp(-i g f_x) from the digit tables (copy q of entry e at e * 16 + q; see
// PhaseDigits), integer costs only.
__device__ __forceinline__ float2 xy_phase_tab(const XyPass &P, const float2 *tab, float2, uint64_t x) {
  const int f = P.cost_kind == kCostU16 ? (int)__ldg(reinterpret_cast<const unsigned short *>(P.cost) + x)
                                        : __ldg(reinterpret_cast<const int *>(P.cost) + x);
  const uint32_t d = (uint32_t)(f - P.ph.fmin) >> P.ph.shift;
  const uint32_t q = threadIdx.x & (kPhaseCopies - 1);
  if (P.ph.nd == 2) {
    const float2 a = tab[((d & 63u) << 4) | q];
    const float2 b = tab[((64u + min(d >> 6, (uint32_t)P.ph.last)) << 4) | q];
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
  }
  const float2 a = tab[((d & 31u) << 4) | q];
  const float2 b = tab[((32u + ((d >> 5) & 31u)) << 4) | q];
  const float2 c = tab[((64u + min(d >> 10, (uint32_t)P.ph.last)) << 4) | q];
  const float2 ab = make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
  return make_float2(ab.x * c.x - ab.y * c.y, ab.x * c.y + ab.y * c.x);
}

__device__ __forceinline__ double2 xy_phase_tab(const XyPass &P, const float2 *, double2, uint64_t x) {
  return xy_phase(P, double2(), x);  // complex128 always computes
}

// Global index of tile offset t in tile T (bits of t below c are qubits
// 0..c-1, the others qubits h..; T fills the remaining bits in order).
__device__ __forceinline__ uint64_t xy_index(const XyPass &P, uint64_t T, uint32_t t) {
  const int mid = P.h - P.c;
  const uint64_t lo = T & ((1ull << mid) - 1ull), top = T >> mid;
  return (uint64_t)(t & ((1u << P.c) - 1u)) | (lo << P.c) | ((uint64_t)(t >> P.c) << P.h) |
         (top << (P.h + P.tb - P.c));
}

// Registers per thread for the next tile's amplitudes (complex64; tiles of
// up to 2^12 amplitudes over 256 threads, two neighbours per load).
constexpr int kXyPrefetchPairs = (1 << kXyMaxTb) / 512;

template <typename C2>
__device__ __forceinline__ C2 xy_phased(const XyPass &P, const float2 *tab, bool table, C2 v, uint64_t x) {
  return table ? xmul(v, xy_phase_tab(P, tab, v, x)) : xmul(v, xy_phase(P, v, x));
}

// PF (complex64): the next tile's amplitudes are loaded into registers while
// the gates run on the current one in shared memory; otherwise the tile is
// loaded just before its gates.
template <typename C2, bool PF>
__global__ void __launch_bounds__(256, PF ? 3 : 1) k_xy_tile(const __grid_constant__ XyPass P) {
  using R = typename XyR<C2>::R;
  extern __shared__ __align__(16) unsigned char xy_smem[];
  C2 *s = reinterpret_cast<C2 *>(xy_smem);
  C2 *psi = reinterpret_cast<C2 *>(P.psi);
  const uint32_t TE = 1u << P.tb;
  float2 *tab = reinterpret_cast<float2 *>(xy_smem + (size_t)TE * sizeof(C2));
  const R th = (R)P.tb2, sn = (R)P.sb;
  const bool neg = P.neg != 0;
  const bool table = P.has_phase && P.ph.mode == 0;
  if (table) {
    for (int i = threadIdx.x; i < P.ph.nent * kPhaseCopies; i += blockDim.x) tab[i] = P.ph.d[i >> 4];
    __syncthreads();
  }
  // pairs of neighbouring amplitudes (tile bit 0 is qubit 0, c >= 1): one
  // 16-byte load per complex64 pair; thread tid holds offsets 2 (tid + 256 i)
  C2 r[PF ? 2 * kXyPrefetchPairs : 1];
  auto load_regs = [&](uint64_t T) {
    if constexpr (PF) {
#pragma unroll
      for (int i = 0; i < kXyPrefetchPairs; ++i) {
        const uint32_t t = 2 * (threadIdx.x + 256u * i);
        if (t < TE) ld2(psi + xy_index(P, T, t), r[2 * i], r[2 * i + 1]);
      }
    }
  };
  if (blockIdx.x < P.ntiles) load_regs(blockIdx.x);
  for (uint64_t T = blockIdx.x; T < P.ntiles; T += gridDim.x) {
    if constexpr (PF) {
#pragma unroll
      for (int i = 0; i < kXyPrefetchPairs; ++i) {
        const uint32_t t = 2 * (threadIdx.x + 256u * i);
        if (t < TE) {
          C2 v0 = r[2 * i], v1 = r[2 * i + 1];
          if (P.has_phase) {
            const uint64_t x = xy_index(P, T, t);
            v0 = xy_phased(P, tab, table, v0, x);
            v1 = xy_phased(P, tab, table, v1, x + 1);
          }
          s[t] = v0;
          s[t + 1] = v1;
        }
      }
      __syncthreads();
      if (T + gridDim.x < P.ntiles) load_regs(T + gridDim.x);
    } else {
      for (uint32_t t = 2 * threadIdx.x; t < TE; t += 2 * blockDim.x) {
        const uint64_t x = xy_index(P, T, t);  // even
        C2 v0, v1;
        ld2(psi + x, v0, v1);
        if (P.has_phase) {
          v0 = xy_phased(P, tab, table, v0, x);
          v1 = xy_phased(P, tab, table, v1, x + 1);
        }
        s[t] = v0;
        s[t + 1] = v1;
      }
      __syncthreads();
    }
    for (int g = 0; g < P.ngates; ++g) {
      const int a = P.ga[g], b = P.gb[g];
      const int lo = a < b ? a : b, hi = a < b ? b : a;
      for (uint32_t k = threadIdx.x; k < (TE >> 2); k += blockDim.x) {
        const uint32_t t0 = insert2_32(k, lo, hi);
        xy_pair<C2, R>(s[t0 | (1u << a)], s[t0 | (1u << b)], th, sn, neg);
      }
      __syncthreads();
    }
    for (uint32_t t = 2 * threadIdx.x; t < TE; t += 2 * blockDim.x) {
      st2(psi + xy_index(P, T, t), s[t], s[t + 1]);
    }
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
  const size_t tabb = (size_t)kPhaseTabEntries * sizeof(float2);
  const size_t smem = ((size_t)1 << P.tb) * (c128 ? 16 : 8) + (P.has_phase && P.ph.mode == 0 ? tabb : 0);
  static int per_sm[2] = {0, 0};  // resident CTAs per SM (registers, shared memory)
  if (!per_sm[0]) {
    const size_t m64 = ((size_t)1 << kXyMaxTb) * 8 + tabb, m128 = ((size_t)1 << kXyMaxTb) * 16;
    cudaError_t e = cudaFuncSetAttribute(k_xy_tile<float2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)m64);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_xy_tile<double2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m128);
    if (e != cudaSuccess) return e;
    int b64 = 0, b128 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b128, k_xy_tile<double2, false>, 256, m128) != cudaSuccess ||
        b128 < 1)
      b128 = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, k_xy_tile<float2, true>, 256, m64) != cudaSuccess ||
        b64 < 1)
      b64 = 1;
    per_sm[1] = b128;
    per_sm[0] = b64;
  }
  const uint64_t cap = (uint64_t)nsm * per_sm[c128 ? 1 : 0];
  const unsigned grid = (unsigned)(P.ntiles < cap ? P.ntiles : cap);
  if (c128)
    k_xy_tile<double2, false><<<grid, 256, smem, s>>>(P);
  else
    k_xy_tile<float2, true><<<grid, 256, smem, s>>>(P);
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
