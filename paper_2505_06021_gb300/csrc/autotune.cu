// Autotuner cache for the split-precision chi0 launch.
//
// The tensor-core kernel's work decomposition has one free parameter that
// matters: the split-K depth of each segment, expressed as a common target
// item length in exact 2048-value K chunks.  Short items cut the tail of the
// persistent grid; long items save partial-sum traffic and reduce work.  The
// best value depends on the launch's shape class (per segment: K chunks,
// frequencies, tiles).  The multi-q launcher, when asked to tune (an eager
// call, never under stream capture), times the best few plans of its cost
// model with CUDA events on the first launch of a class and records the
// fastest here; later launches of that class, including those captured into a
// CUDA graph, look it up.  The cache is process-wide and guarded by a mutex.
#include <map>
#include <mutex>

#include "rpa_internal.h"

namespace rpa {
namespace {

std::mutex& mu() {
  static std::mutex m;
  return m;
}
std::map<uint64_t, int>& table() {
  static std::map<uint64_t, int> t;
  return t;
}

}  // namespace

int autotune_lookup(uint64_t key) {
  std::lock_guard<std::mutex> lk(mu());
  auto it = table().find(key);
  return it == table().end() ? 0 : it->second;
}

void autotune_record(uint64_t key, int value) {
  std::lock_guard<std::mutex> lk(mu());
  table()[key] = value;
}

}  // namespace rpa
