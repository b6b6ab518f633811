// kernels.h -- launcher declarations between the host planner (api.cu) and
// the kernel translation units.  Internal to the library.
#pragma once

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
cudaError_t launch_maxcut(const EdgeChunk &P, cudaStream_t s, int nsm);
unsigned reduce_grid(int n, int nsm);
cudaError_t launch_cost_stats(int n, const void *cost, int kind, double *partials,
                              unsigned *counter, double *out, cudaStream_t s, int nsm);
cudaError_t launch_expect(int n, const void *psi, bool c128, const void *cost, int kind,
                          double fmin, double *partials, unsigned *counter, double *out, int which,
                          cudaStream_t s, int nsm);

cudaError_t launch_fwd(const FwdParams<float> &P, bool high, cudaStream_t s, int nsm);
cudaError_t launch_fwd(const FwdParams<double> &P, bool high, cudaStream_t s, int nsm);
cudaError_t launch_bwd(const BwdParams<float> &P, bool high, cudaStream_t s, int nsm);
cudaError_t launch_bwd(const BwdParams<double> &P, bool high, cudaStream_t s, int nsm);

cudaError_t launch_small(const SmallParams<float> &P, cudaStream_t s);
cudaError_t launch_small(const SmallParams<double> &P, cudaStream_t s);

}  // namespace qaoa
