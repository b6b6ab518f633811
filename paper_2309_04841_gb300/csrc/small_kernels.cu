// small_kernels.cu -- n <= 12: one CTA holds the whole state (and lambda) in
// shared memory and runs many layers of Algorithm 3 (and their adjoint) in a
// single launch; a launch costs microseconds instead of one launch per pass.
#include "qaoa_common.cuh"
#include "kernels.h"

namespace qaoa {

namespace {

template <typename C2> struct SR;
template <> struct SR<float2> { using R = float; };
template <> struct SR<double2> { using R = double; };

template <typename C2>
__device__ __forceinline__ C2 mk2(typename SR<C2>::R x, typename SR<C2>::R y) {
  C2 r;
  r.x = x;
  r.y = y;
  return r;
}

template <typename C2>
__device__ __forceinline__ C2 cm(C2 a, C2 b) {
  return mk2<C2>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ double ld_cost(const void *cost, int kind, int x) {
  if (kind == kCostI32) return (double)reinterpret_cast<const int *>(cost)[x];
  if (kind == kCostU16) return (double)reinterpret_cast<const unsigned short *>(cost)[x];
  if (kind == kCostF32) return (double)reinterpret_cast<const float *>(cost)[x];
  return reinterpret_cast<const double *>(cost)[x];
}

// exp(-i g f) with g / 2pi = g_hi + g_lo (float-float, complex64).
__device__ __forceinline__ float2 small_phase(const SmallLayer<float> &L, const void *cost,
                                              int kind, int x) {
  float fh, fl;
  if (kind == kCostI32) {
    const int f = reinterpret_cast<const int *>(cost)[x];
    fh = (float)f;
    fl = (float)((long long)f - (long long)fh);
  } else if (kind == kCostU16) {
    fh = (float)reinterpret_cast<const unsigned short *>(cost)[x];
    fl = 0.f;
  } else if (kind == kCostF32) {
    fh = reinterpret_cast<const float *>(cost)[x];
    fl = 0.f;
  } else {
    const double f = reinterpret_cast<const double *>(cost)[x];
    fh = (float)f;
    fl = (float)(f - (double)fh);
  }
  const float p = L.g_hi * fh;
  const float e = fmaf(L.g_hi, fh, -p);
  const float r = (p - rintf(p)) + (e + fmaf(L.g_hi, fl, L.g_lo * fh));
  float sn, cs;
  sincospif(2.0f * r, &sn, &cs);
  return make_float2(cs, -sn);
}

__device__ __forceinline__ double2 small_phase(const SmallLayer<double> &L, const void *cost,
                                               int kind, int x) {
  const double t = L.g2pi * ld_cost(cost, kind, x);
  const double r = t - rint(t);
  double sn, cs;
  sincospi(2.0 * r, &sn, &cs);
  return make_double2(cs, -sn);
}

// Deterministic block sum (fixed tree); result returned to every thread.
template <int K>
__device__ __forceinline__ void bsum(double (&a)[K], double *red) {
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_down_sync(0xffffffffu, a[k], o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) red[w * K + k] = a[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += red[i * K + k];
    a[k] = s;
  }
  __syncthreads();
}

}  // namespace

// mode 0: forward layers [0, nl) (+ optional E/O reduction)
// mode 1: forward all layers, E/O, then the whole adjoint sweep (grad)
// mode 2: adjoint sweep over layers [0, nl) in reverse, continuing from the
//         psi / lambda stored by a previous launch (or lambda = f psi)
template <typename Real>
__device__ __forceinline__ void small_run(const SmallJob<Real> &P) {
  using C2 = typename C2T<Real>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = P.n, N = 1 << n, H = N >> 1;
  C2 *s = reinterpret_cast<C2 *>(smem_raw);
  C2 *l = s + N;
  double *red = reinterpret_cast<double *>(l + N);
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int x = tid; x < N; x += nt) s[x] = P.init_plus ? mk2<C2>(P.amp, (Real)0) : P.psi[x];
  __syncthreads();

  if (P.mode == 0 || P.mode == 1) {
    for (int li = 0; li < P.nl; ++li) {
      const SmallLayer<Real> L = P.L[li];
      for (int x = tid; x < N; x += nt) s[x] = cm(s[x], small_phase(L, P.cost, P.cost_kind, x));
      __syncthreads();
      for (int q = 0; q < n; ++q) {
        for (int k = tid; k < H; k += nt) {
          const int x0 = ((k >> q) << (q + 1)) | (k & ((1 << q) - 1));
          const int x1 = x0 | (1 << q);
          const C2 a = s[x0], b = s[x1];
          s[x0] = mk2<C2>(L.cb * a.x + L.sb * b.y, L.cb * a.y - L.sb * b.x);
          s[x1] = mk2<C2>(L.cb * b.x + L.sb * a.y, L.cb * b.y - L.sb * a.x);
        }
        __syncthreads();
      }
    }
    if (P.reduce) {
      double a[2] = {0.0, 0.0};
      for (int x = tid; x < N; x += nt) {
        const double f = ld_cost(P.cost, P.cost_kind, x);
        const double pr = (double)s[x].x * s[x].x + (double)s[x].y * s[x].y;
        a[0] += pr * f;
        a[1] += (f == P.fmin_d) ? pr : 0.0;
      }
      bsum<2>(a, red);
      if (tid == 0) {
        P.out[0] = a[0];
        P.out[1] = a[1];
      }
    }
  }

  if (P.mode == 1 || P.mode == 2) {
    if (P.mode == 1 || P.init_lambda) {
      for (int x = tid; x < N; x += nt) {
        const Real f = (Real)ld_cost(P.cost, P.cost_kind, x);
        l[x] = mk2<C2>(f * s[x].x, f * s[x].y);
      }
    } else {
      for (int x = tid; x < N; x += nt) l[x] = P.lam[x];
    }
    __syncthreads();
    for (int li = P.nl - 1; li >= 0; --li) {
      const SmallLayer<Real> L = P.L[li];
      double gb[1] = {0.0};
      const Real c = L.cb, sn = -L.sb;
      for (int q = 0; q < n; ++q) {
        for (int k = tid; k < H; k += nt) {
          const int x0 = ((k >> q) << (q + 1)) | (k & ((1 << q) - 1));
          const int x1 = x0 | (1 << q);
          const C2 pa = s[x0], pb = s[x1], la = l[x0], lb = l[x1];
          gb[0] += (double)(la.x * pb.y - la.y * pb.x + lb.x * pa.y - lb.y * pa.x);
          s[x0] = mk2<C2>(c * pa.x + sn * pb.y, c * pa.y - sn * pb.x);
          s[x1] = mk2<C2>(c * pb.x + sn * pa.y, c * pb.y - sn * pa.x);
          l[x0] = mk2<C2>(c * la.x + sn * lb.y, c * la.y - sn * lb.x);
          l[x1] = mk2<C2>(c * lb.x + sn * la.y, c * lb.y - sn * la.x);
        }
        __syncthreads();
      }
      bsum<1>(gb, red);
      double gg[1] = {0.0};
      for (int x = tid; x < N; x += nt) {
        const double f = ld_cost(P.cost, P.cost_kind, x);
        gg[0] += f * ((double)l[x].x * s[x].y - (double)l[x].y * s[x].x);
        C2 ph = small_phase(L, P.cost, P.cost_kind, x);
        ph.y = -ph.y;  // exp(+i g f): the inverse phase
        s[x] = cm(s[x], ph);
        l[x] = cm(l[x], ph);
      }
      bsum<1>(gg, red);
      if (tid == 0) {
        P.out_db[li] = 2.0 * gb[0];
        P.out_dg[li] = 2.0 * gg[0];
      }
      __syncthreads();
    }
    for (int x = tid; x < N; x += nt) P.lam[x] = l[x];
  }
  for (int x = tid; x < N; x += nt) P.psi[x] = s[x];
}

template <typename Real>
__global__ void __launch_bounds__(512) k_small(const __grid_constant__ SmallParams<Real> P) {
  SmallJob<Real> J;
  J.psi = P.psi;
  J.lam = P.lam;
  J.cost = P.cost;
  J.cost_kind = P.cost_kind;
  J.n = P.n;
  J.nl = P.nl;
  J.mode = P.mode;
  J.init_plus = P.init_plus;
  J.init_lambda = P.init_lambda;
  J.reduce = P.reduce;
  J.amp = P.amp;
  J.fmin_d = P.fmin_d;
  J.out = P.out;
  J.out_dg = P.out_dg;
  J.out_db = P.out_db;
  J.L = P.L;
  small_run<Real>(J);
}

// Many independent requests in one launch: CTA b runs jobs[b] (serving).
template <typename Real>
__global__ void __launch_bounds__(512) k_small_batch(const SmallJob<Real> *jobs) {
  const SmallJob<Real> J = jobs[blockIdx.x];
  small_run<Real>(J);
}

template <typename Real>
static cudaError_t launch_small_t(const SmallParams<Real> &P, cudaStream_t st) {
  using C2 = typename C2T<Real>::type;
  const size_t smem = (size_t)2 * ((size_t)1 << P.n) * sizeof(C2) + 16 * 2 * sizeof(double);
  static bool init = false;
  if (!init) {
    cudaError_t e = cudaFuncSetAttribute(k_small<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(2 * (1 << kSmallMaxN) * sizeof(C2) + 256));
    if (e != cudaSuccess) return e;
    init = true;
  }
  int nt = (1 << P.n) / 2;
  nt = nt < 32 ? 32 : (nt > 512 ? 512 : nt);
  k_small<Real><<<1, nt, smem, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_small(const SmallParams<float> &P, cudaStream_t s) { return launch_small_t(P, s); }
cudaError_t launch_small(const SmallParams<double> &P, cudaStream_t s) { return launch_small_t(P, s); }

template <typename Real>
static cudaError_t launch_small_batch_t(const SmallJob<Real> *d_jobs, int count, int max_n,
                                       cudaStream_t st) {
  using C2 = typename C2T<Real>::type;
  static bool init = false;
  if (!init) {
    cudaError_t e = cudaFuncSetAttribute(k_small_batch<Real>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(2 * (1 << kSmallMaxN) * sizeof(C2) + 256));
    if (e != cudaSuccess) return e;
    init = true;
  }
  const size_t smem = (size_t)2 * ((size_t)1 << max_n) * sizeof(C2) + 16 * 2 * sizeof(double);
  int nt = (1 << max_n) / 2;
  nt = nt < 32 ? 32 : (nt > 512 ? 512 : nt);
  k_small_batch<Real><<<count, nt, smem, st>>>(d_jobs);
  return cudaGetLastError();
}

cudaError_t launch_small_batch(const SmallJob<float> *d_jobs, int count, int max_n, cudaStream_t s) {
  return launch_small_batch_t(d_jobs, count, max_n, s);
}
cudaError_t launch_small_batch(const SmallJob<double> *d_jobs, int count, int max_n, cudaStream_t s) {
  return launch_small_batch_t(d_jobs, count, max_n, s);
}

}  // namespace qaoa
