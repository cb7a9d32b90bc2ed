// Allocation-free single-system solve.
//
// Some callers cannot allocate device memory at the moment they solve:
// latency-critical loops where a cudaMalloc would synchronise the device, or
// hosts whose memory pool owns all device memory and forbids other
// allocations after start-up.  tdp_solve_noalloc
// serves them: its scratch (the interface systems of every recursion level
// and the status word) lives in one statically sized __device__ array that
// the library image carries, so the call makes no cudaMalloc, cudaFree or
// other device allocation.  The caller still passes its own inputs and x.
#include <mutex>
#include <string>

#include "tdp_internal.h"

namespace tdp {
namespace {

// 16 MiB, held on every GPU that loads the library until the process exits.
constexpr size_t kNoAllocBytes = size_t(16) << 20;
constexpr size_t kStatusBytes = 256;  // device status word, then the arena

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// In host code g_noalloc_scratch names a host-side stand-in, not the device
// array: its device address is looked up once per device (with that device
// current) and cached here.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

int fail(int code, const std::string& m) { return set_last_error(code, m); }

}  // namespace
}  // namespace tdp

using namespace tdp;

extern "C" int tdp_solve_noalloc(const void* a, const void* b, const void* c, const void* d, void* x, int64_t n,
                                 int32_t s, tdp_dtype dtype, void* stream) {
  if (n < 1) return fail(TDP_EINVAL, "tdp_solve_noalloc: n must be >= 1");
  if (s != 0 && (s < 2 || s > 1024)) return fail(TDP_EINVAL, "tdp_solve_noalloc: s must be 0 or in [2, 1024]");
  if (dtype != TDP_F64 && dtype != TDP_F32)
    return fail(TDP_EINVAL, "tdp_solve_noalloc: dtype must be TDP_F64 or TDP_F32");
  for (const void* p : {a, b, c, d, (const void*)x}) {
    if (!p) return fail(TDP_EINVAL, "tdp_solve_noalloc: null pointer");
    if (reinterpret_cast<uintptr_t>(p) & 15u) return fail(TDP_EINVAL, "tdp_solve_noalloc: pointer not 16-byte aligned");
  }
  const int ss = s ? s : predict_s(n, 1, dtype);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  // size the scratch with a dry run of the driver; reject what does not fit
  Arena sizing;
  Ctx dry;
  tune_from_env(dry);
  dry.stream = st;
  dry.ar = &sizing;
  dry.dry = true;
  solve_single_lean(dry, a, b, c, d, x, n, ss, dtype);
  const size_t need = sizing.off + 256;
  if (need > kNoAllocBytes - kStatusBytes)
    return fail(TDP_EINVAL, "tdp_solve_noalloc: n = " + std::to_string(n) + " with s = " + std::to_string(ss) +
                                " needs " + std::to_string(need) + " bytes of scratch; the static scratch holds " +
                                std::to_string(kNoAllocBytes - kStatusBytes) + " (use tdp_solve for larger systems)");

  // device address of the static scratch, looked up once per device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(TDP_ECUDA, std::string("tdp_solve_noalloc: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(TDP_EINVAL, "tdp_solve_noalloc: device index out of range");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr)
        return fail(TDP_ECUDA, std::string("tdp_solve_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_addr[dev] = ptr;
    }
    base = g_addr[dev];
  }
  unsigned* status = reinterpret_cast<unsigned*>(base);
  // the array keeps the previous call's contents: the status word starts at zero
  e = cudaMemsetAsync(status, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return fail(TDP_ECUDA, std::string("tdp_solve_noalloc: ") + cudaGetErrorString(e));

  Arena arena;
  arena.base = static_cast<char*>(base) + kStatusBytes;
  arena.cap = kNoAllocBytes - kStatusBytes;
  Ctx ctx;
  tune_from_env(ctx);
  ctx.stream = st;
  ctx.status = status;
  ctx.ar = &arena;
  arena.err = &ctx.err;  // a take beyond the dry run's measure fails the call instead of aliasing
  ctx.events_ok = false;  // the profiler would create CUDA events
  solve_single_lean(ctx, a, b, c, d, x, n, ss, dtype);
  if (ctx.err != cudaSuccess)
    return fail(TDP_ECUDA, "tdp_solve_noalloc: " + (ctx.msg.empty() ? std::string("scratch overrun") : ctx.msg));
  if (checked_mode()) {
    e = cudaStreamSynchronize(st);
    unsigned h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(TDP_ECUDA, std::string("tdp_solve_noalloc: ") + cudaGetErrorString(e));
    if (status_code(h) != TDP_OK) return status_error(h, "tdp_solve_noalloc");
  }
  return set_last_error(TDP_OK, "");
}
