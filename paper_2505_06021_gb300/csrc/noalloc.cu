// rpa_logdet_noalloc: the log-det step for callers that cannot allocate.
//
// Some callers must not allocate device memory at call time: code that runs
// inside another framework which owns every byte of the GPU through its own
// pool, latency-critical serving loops where a cudaMalloc/cudaFree (which can
// synchronise the whole device) is not acceptable, or processes that reserve
// all memory up front and fail on any later request.  For them this file keeps
// its scratch in one file-scope device array that exists from module load
// until process exit on every GPU that loads the library.  The caller passes
// inputs and outputs; nothing is allocated, by this code or by a library it
// calls.
//
// Limits: n_aux <= RPA_NOALLOC_MAX_NAUX (384).  The array holds three
// n_aux x n_aux complex128 matrices (the Cholesky factor of V, chi L and
// -L^H chi L for one frequency at a time) plus a status word: 7,078,144 bytes.
//
// Calls share the array: two calls whose work overlaps on the GPU (different
// streams, or different host threads, on one device) race and corrupt each
// other's results.  Each call clears the status word before use; the matrices
// are fully rewritten before they are read.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "rpa_internal.h"

#define RPA_NOALLOC_MAX_NAUX 384
#define RPA_NOALLOC_MAT_BYTES ((size_t)RPA_NOALLOC_MAX_NAUX * RPA_NOALLOC_MAX_NAUX * 16)
#define RPA_NOALLOC_BYTES (3 * RPA_NOALLOC_MAT_BYTES + 256)

static __device__ __align__(256) unsigned char g_noalloc_scratch[RPA_NOALLOC_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};
thread_local char g_msg[256] = "";

void set_msg(const char* m, const char* detail) {
  snprintf(g_msg, sizeof g_msg, "%s%s%s", m, detail ? ": " : "", detail ? detail : "");
}

// Device address of the scratch array for the current device.  The host-side
// name g_noalloc_scratch is only a stand-in and must never be passed to a
// kernel; the real address is looked up once per device, with that device
// current, and cached.
void* scratch_for_current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      set_msg("cudaGetSymbolAddress failed", cudaGetErrorString(e));
      return nullptr;
    }
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

}  // namespace

extern "C" {

const char* rpa_noalloc_last_error(void) { return g_msg; }

rpa_status rpa_logdet_noalloc(int is_complex, int n_aux, int n_w, const void* V, const void* chi, double* out,
                              void* stream) {
  g_msg[0] = 0;
  if ((is_complex != 0 && is_complex != 1) || n_aux <= 0 || n_w <= 0 || !V || !chi || !out) {
    set_msg("invalid argument", nullptr);
    return RPA_E_INVAL;
  }
  if (n_aux > RPA_NOALLOC_MAX_NAUX) {
    char d[96];
    snprintf(d, sizeof d, "n_aux = %d exceeds the static scratch limit %d", n_aux, RPA_NOALLOC_MAX_NAUX);
    set_msg("too large", d);
    return RPA_E_INVAL;
  }
  // V, chi and out must be device (or managed) memory of the current device,
  // aligned to their element size: a host pointer here would make the kernels
  // read or write memory the GPU cannot (or should not) reach.
  {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
      cudaGetLastError();
      set_msg("no current CUDA device", nullptr);
      return RPA_E_CUDA;
    }
    const void* ptrs[3] = {V, chi, out};
    const char* names[3] = {"V", "chi", "out"};
    const size_t align[3] = {is_complex ? (size_t)16 : (size_t)8, is_complex ? (size_t)16 : (size_t)8, 8};
    for (int i = 0; i < 3; ++i) {
      cudaPointerAttributes at;
      if (cudaPointerGetAttributes(&at, ptrs[i]) != cudaSuccess) {
        cudaGetLastError();
        set_msg("pointer query failed", names[i]);
        return RPA_E_INVAL;
      }
      if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev) {
        char d[96];
        snprintf(d, sizeof d, "%s is not device memory of the current device %d", names[i], dev);
        set_msg("invalid pointer", d);
        return RPA_E_INVAL;
      }
      if (reinterpret_cast<uintptr_t>(ptrs[i]) % align[i]) {
        char d[96];
        snprintf(d, sizeof d, "%s is not aligned to %zu bytes", names[i], align[i]);
        set_msg("invalid pointer", d);
        return RPA_E_INVAL;
      }
    }
  }
  char* base = static_cast<char*>(scratch_for_current_device());
  if (!base) {
    if (!g_msg[0]) set_msg("no scratch address for the current device", nullptr);
    return RPA_E_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t es = is_complex ? 16 : 8;
  const size_t NN = (size_t)n_aux * n_aux;
  double* L = reinterpret_cast<double*>(base);
  double* T = reinterpret_cast<double*>(base + RPA_NOALLOC_MAT_BYTES);
  double* Y = reinterpret_cast<double*>(base + 2 * RPA_NOALLOC_MAT_BYTES);
  int* status = reinterpret_cast<int*>(base + 3 * RPA_NOALLOC_MAT_BYTES);
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(L, V, es * NN, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = rpa::launch_cholesky(is_complex, n_aux, 1, L, (long)(NN * (es / 8)), 1, nullptr, status, 1 << 29, s);
  const double* chib = static_cast<const double*>(chi);
  for (int w = 0; w < n_w && e == cudaSuccess; ++w) {
    e = rpa::launch_sandwich(is_complex, n_aux, 1, 1, chib + (size_t)w * NN * (es / 8), L, T, Y, s);
    if (e == cudaSuccess)
      e = rpa::launch_cholesky(is_complex, n_aux, 1, Y, (long)(NN * (es / 8)), 0, out + 2 * w, status, w, s);
  }
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_msg("CUDA error", cudaGetErrorString(e));
    return RPA_E_CUDA;
  }
  if (st) {
    char d[96];
    const int code = st - 1;
    if (code >= (1 << 29))
      snprintf(d, sizeof d, "V is not positive definite");
    else
      snprintf(d, sizeof d, "1 - Pi(w=%d) is not positive definite", code);
    set_msg("not positive definite", d);
    return RPA_E_NOTPD;
  }
  return RPA_OK;
}

}  // extern "C"
