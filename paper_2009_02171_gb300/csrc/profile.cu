// Optional per-category kernel timing with CUDA events (see fv_profile_enable).
#include <vector>

#include "fv_internal.h"

namespace fv {

namespace {
struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> ev;  // pairs
  std::vector<int> cat;
  size_t used = 0;
  long long dropped = 0;
};
Prof g_prof;
constexpr size_t kPairs = 65536;
}  // namespace

bool prof_enabled() { return g_prof.on; }

int prof_begin(int category, cudaStream_t st) {
  if (!g_prof.on) return -1;
  if (g_prof.used >= kPairs) {
    ++g_prof.dropped;
    return -1;
  }
  const int slot = (int)g_prof.used++;
  g_prof.cat[slot] = category;
  cudaEventRecord(g_prof.ev[2 * slot], st);
  return slot;
}

void prof_end(int slot, cudaStream_t st) {
  if (slot >= 0) cudaEventRecord(g_prof.ev[2 * slot + 1], st);
}

}  // namespace fv

using namespace fv;

extern "C" {

fv_status fv_profile_enable(int on) {
  if (on && g_prof.ev.empty()) {
    g_prof.ev.resize(2 * kPairs);
    g_prof.cat.resize(kPairs);
    for (auto& e : g_prof.ev) FV_CUDA(cudaEventCreate(&e));
  }
  g_prof.on = on != 0;
  g_prof.used = 0;
  g_prof.dropped = 0;
  return FV_OK;
}

fv_status fv_profile_read(int category, long long* launches, double* total_ms) {
  if (!launches || !total_ms || category < 0 || category >= FV_K_COUNT)
    return set_error("fv_profile_read: bad argument"), FV_EINVAL;
  FV_CUDA(cudaDeviceSynchronize());
  long long n = 0;
  double t = 0.0;
  for (size_t s = 0; s < g_prof.used; ++s) {
    if (g_prof.cat[s] != category) continue;
    float ms = 0.f;
    FV_CUDA(cudaEventElapsedTime(&ms, g_prof.ev[2 * s], g_prof.ev[2 * s + 1]));
    ++n;
    t += ms;
  }
  *launches = n;
  *total_ms = t;
  return FV_OK;
}

}  // extern "C"
