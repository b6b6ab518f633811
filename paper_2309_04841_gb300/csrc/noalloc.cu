// noalloc.cu -- qaoa_simulate_noalloc: qaoa_simulate with a fixed scratch
// area inside the library instead of a caller-provided workspace.
//
// Some callers cannot allocate device memory at all: a plugin whose host
// application owns every device allocation and forbids allocations outside
// its own pool, or a caller whose fixed device-memory budget is already fully
// committed.  They still own the cost vector, the state and the two output
// doubles; the reduction partials, counters and error word live in
// g_scratch below, a file-scope device array that every GPU which loads this
// library holds until the process exits.
#include "../../include/qaoa.h"

namespace qaoa {
void set_last_error(const char *msg);  // api.cu: message for qaoa_last_error_message
}

namespace {

// 128 KiB + 512 B: enough for qaoa_workspace_bytes(n) up to n = 23.
constexpr size_t kScratchBytes = 512 + 128 * 1024;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch on the current device.  In host code the name
// g_scratch is only a host-side stand-in, not a device address, so it is
// looked up with cudaGetSymbolAddress while the device is current -- on every
// call: the lookup is a cheap host-side query, and a module reloaded after a
// device reset may place the array elsewhere.
qaoa_status scratch_for_current_device(void **out) {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return QAOA_ERR_CUDA;
  *out = p;
  return QAOA_OK;
}

}  // namespace

namespace qaoa {
// The built-in scratch of the current device, for qaoa_workspace_check and
// qaoa_selftest_timeout called with (NULL, 0).
qaoa_status builtin_scratch(void **ptr, size_t *bytes) {
  const qaoa_status s = scratch_for_current_device(ptr);
  if (s == QAOA_OK) *bytes = kScratchBytes;
  return s;
}
}  // namespace qaoa

extern "C" qaoa_status qaoa_simulate_noalloc(int n, const void *d_costs, qaoa_cost_type ct,
                                             const qaoa_cost_stats *stats, const double *gammas,
                                             const double *betas, int p, void *d_state,
                                             qaoa_state_type st, int init_plus, double *d_out,
                                             qaoa_stream_t stream) {
  if (n < 1 || n > QAOA_MAX_N) {
    qaoa::set_last_error("simulate_noalloc: n out of range");
    return QAOA_ERR_INVALID_ARG;
  }
  // The built-in scratch covers what qaoa_simulate needs up to n = 23; larger
  // n is refused before anything is enqueued.
  if (qaoa_workspace_bytes(n) > kScratchBytes) {
    qaoa::set_last_error("simulate_noalloc: n > 23 does not fit the built-in 128.5 KiB scratch; "
                         "use qaoa_simulate with a workspace");
    return QAOA_ERR_OUT_OF_MEMORY;
  }
  void *scratch = nullptr;
  const qaoa_status s = scratch_for_current_device(&scratch);
  if (s != QAOA_OK) {
    qaoa::set_last_error("simulate_noalloc: cudaGetSymbolAddress of the built-in scratch failed");
    return s;
  }
  // qaoa_simulate clears the counters and the error word it relies on at the
  // start of every call, so the contents left by the previous call do not
  // matter; it allocates nothing.
  return qaoa_simulate(n, d_costs, ct, stats, gammas, betas, p, d_state, st, init_plus, scratch,
                       kScratchBytes, d_out, stream);
}
