// profile.cu -- optional per-launch CUDA-event timing of the library's own
// kernels (qaoa_profile_enable / qaoa_profile_read).  Host code only.
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/qaoa.h"
#include "kernels.h"

namespace qaoa {

namespace {

struct Rec {
  const char *kind;
  double bytes;
  cudaEvent_t a, b;
  bool timed;
};

constexpr size_t kMaxTimed = 65536;

std::mutex &mu() {
  static std::mutex *m = new std::mutex();
  return *m;
}
bool g_on = false;
std::vector<cudaEvent_t> g_pool;
std::vector<Rec> g_recs;
size_t g_created = 0;

bool take(cudaEvent_t &e) {
  if (!g_pool.empty()) {
    e = g_pool.back();
    g_pool.pop_back();
    return true;
  }
  if (g_created >= 2 * kMaxTimed) return false;
  if (cudaEventCreate(&e) != cudaSuccess) return false;
  ++g_created;
  return true;
}

}  // namespace

int prof_begin(cudaStream_t s) {
  std::lock_guard<std::mutex> lk(mu());
  if (!g_on) return -1;
  Rec r{nullptr, 0.0, nullptr, nullptr, false};
  if (take(r.a)) {
    if (take(r.b)) {
      r.timed = cudaEventRecord(r.a, s) == cudaSuccess;
    } else {
      g_pool.push_back(r.a);
      r.a = nullptr;
    }
  }
  g_recs.push_back(r);
  return (int)g_recs.size() - 1;
}

void prof_end(int id, cudaStream_t s, const char *kind, double bytes) {
  if (id < 0) return;
  std::lock_guard<std::mutex> lk(mu());
  if ((size_t)id >= g_recs.size()) return;
  Rec &r = g_recs[id];
  r.kind = kind;
  r.bytes = bytes;
  if (r.timed && cudaEventRecord(r.b, s) != cudaSuccess) r.timed = false;
}

}  // namespace qaoa

using namespace qaoa;

extern "C" {

qaoa_status qaoa_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(mu());
  if (on && g_pool.size() < 256) {
    for (int i = 0; i < 256 && g_created < 2 * kMaxTimed; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return QAOA_ERR_CUDA;
      ++g_created;
      g_pool.push_back(e);
    }
  }
  g_on = on != 0;
  return QAOA_OK;
}

qaoa_status qaoa_profile_read(qaoa_prof_entry *out, int cap, int *n_out, int reset) {
  if (!n_out || (cap > 0 && !out)) return QAOA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(mu());
  std::map<std::string, qaoa_prof_entry> agg;
  qaoa_status st = QAOA_OK;
  for (Rec &r : g_recs) {
    if (!r.kind) continue;
    qaoa_prof_entry &e = agg[r.kind];
    if (e.launches == 0) {
      memset(&e, 0, sizeof(e));
      strncpy(e.name, r.kind, sizeof(e.name) - 1);
    }
    e.launches += 1;
    e.bytes += r.bytes;
    if (r.timed) {
      float ms = 0.f;
      if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
        st = QAOA_ERR_CUDA;
      e.ms += ms;
    }
  }
  int k = 0;
  for (auto &kv : agg) {
    if (k < cap) out[k] = kv.second;
    ++k;
  }
  *n_out = k;
  if (reset) {
    for (Rec &r : g_recs) {
      if (r.a) g_pool.push_back(r.a);
      if (r.b) g_pool.push_back(r.b);
    }
    g_recs.clear();
  }
  return st;
}

}  // extern "C"
