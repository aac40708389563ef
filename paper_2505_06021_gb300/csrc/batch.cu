// Batched execution of many independent (uneven) jobs in one call.
#include <cuda_runtime.h>

#include <vector>

#include "rpa_runtime.h"

namespace rpa {

struct BatchCache {
  std::vector<Exec*> lanes;
};

void batch_release(rpa_ctx* ctx) {
  if (!ctx->batch) return;
  for (Exec* e : ctx->batch->lanes) {
    e->destroy();
    delete e;
  }
  delete ctx->batch;
  ctx->batch = nullptr;
}

}  // namespace rpa

using namespace rpa;

extern "C" rpa_status rpa_energy_batch(rpa_ctx* ctx, const rpa_job* jobs, int n_jobs, double* Ec_out) {
  if (!ctx || (!jobs && n_jobs > 0) || !Ec_out || n_jobs < 0) return RPA_E_INVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  for (int i = 0; i < n_jobs; ++i) {
    if (jobs[i].mem != RPA_MEM_DEVICE) {
      ctx_set_error(ctx, "rpa_energy_batch: job %d is not device-resident", i);
      return RPA_E_INVAL;
    }
    if (rpa_status st = energy_enqueue(ctx, ctx->ex, &jobs[i], (size_t)24 << 30)) return st;
    if (rpa_status st = wait_event(ctx, ctx->ex.done, ctx->timeout_s + 600.0)) return st;
    if (rpa_status st = energy_finish(ctx, ctx->ex, &jobs[i], &Ec_out[i], nullptr, nullptr)) return st;
  }
  return RPA_OK;
}
