// Host-side interfaces between the C ABI (tdp_api.cu) and the solver
// drivers (tdp_solver.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/tdp.h"
#include "tdp_status.h"

namespace tdp {

// Bump allocator over a workspace buffer.  With base == nullptr it only
// measures (dry run used to size the workspace before any launch).  The real
// run takes exactly what the dry run measured; should it ask for more, the
// take raises *err (so that no further kernel launches) and hands back the
// start of the buffer instead of memory past its end.
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t off = 0;
  cudaError_t* err = nullptr;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    const size_t bytes = count * sizeof(T) + 16;
    if (base && off + bytes > cap) {
      if (err && *err == cudaSuccess) *err = cudaErrorMemoryAllocation;
      off += bytes;
      return reinterpret_cast<T*>(base);
    }
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += bytes;
    return p;
  }
};

struct Ctx {
  cudaStream_t stream = nullptr;
  unsigned* status = nullptr;  // device status word
  Arena* ar = nullptr;
  bool dry = false;            // size the workspace only, launch nothing
  cudaError_t err = cudaSuccess;
  int smem_budget = 100 * 1024;  // shared memory per CTA the launcher aims for
  int s_rec = 16;              // sub-system size inside the interface-system recursion
  bool refine3 = true;         // three fused passes for a solve and its first correction (TDP_REFINE3=0 off)
  int rec_mode = 0;            // 1: the paper's recursion schedule for the interface system (TDP_RECURSION)
  int rec_force = -1;          // its number of recursive steps; -1: predicted (TDP_R)
  int64_t rec_n = 1;           // size, batch and dtype the recursion depth is predicted for
  int32_t rec_batch = 1;
  tdp_dtype rec_dt = TDP_F64;
  bool seg = true;                   // per-system interface solves for batches (TDP_SEGMENTED=0 off)
  bool per_system_s = false;         // batched s = 0: one s per system from the device model (TDP_PER_SYSTEM_S=1)
  bool iface32 = false;              // binary32 arithmetic in the first interface level of binary32 solves
  bool iface32_on = false;           // set while such a solve runs
  bool refine_kept = true;           // refinement pass 3 from kept binary32 coefficients (TDP_REFINE_KEPT)
  bool coop_reg = true;              // one-launch tail: 8-row blocks through registers (TDP_COOP_REG)
  bool batch_flat = true;            // batches of large systems as one block-diagonal system (TDP_BATCH_FLAT)
  int64_t kb = 0, ke = -1;           // system-level Stage 1/3 launches cover blocks [kb, ke) (-1: all)
  const int64_t* flat_off = nullptr; // set while such a batch is solved: its offsets (device)
  int32_t flat_nsys = 0;             // and number of systems
  const int64_t* seg_bbase = nullptr;  // the batch whose interface system is being solved: blocks
  int64_t seg_per = 0;                 // before each system (device), or blocks per system
  int32_t seg_batch = 0;
  bool events_ok = true;       // the profiler may create CUDA events around launches
  bool vtile = true;           // 16-byte cp.async interleaved tiles for one system (TDP_VTILE=0 off)
  bool vtile_b = true;         // binary64 Stage 1 at s = 8, 16 with b in registers (TDP_VTILE_B=0 off)
  bool vtile_l = true;         // binary32 storage: padded block-major tiles (TDP_VTILE_L=0 off)
  bool window = true;          // windowed single pass for binary32 + binary64 refinement (TDP_WINDOW=0 off)
  bool window32 = true;        // windowed single pass for binary32 storage (TDP_WINDOW32=0 off)
  int window_prefetch = 128;   // L2 prefetch distance of the windowed pass in tiles (TDP_WINDOW_PREFETCH)
  int window_halo = 48;        // its halo rows on each side of a tile (TDP_WINDOW_HALO)
  int window_halo32 = 32;      // the same for binary32 storage (TDP_WINDOW_HALO32)
  int window_sw32 = 13;        // most rows per thread of the binary32 windowed pass (TDP_WINDOW_SW32)
  int window_sw = 7;           // the refinement's window rows per thread, 5 or 7 (TDP_WINDOW_SW)
  int wait_log2 = 31;          // bounded device waits give up after 2^wait_log2 cycles (TDP_WAIT_LOG2)
  bool wait_never = false;     // testing: grid barriers can never complete (TDP_WAIT_NEVER)
  bool coop = true;            // small interface levels in one cooperative launch (TDP_COOP=0 off)
  int s_tail = 8;              // sub-system size inside that launch (TDP_S_TAIL)
  std::string msg;
  void fail(cudaError_t e, const char* where) {
    if (err == cudaSuccess && e != cudaSuccess) {
      err = e;
      msg = std::string(where) + ": " + cudaGetErrorString(e);
    }
  }
};

// Launch bookkeeping: counts every kernel launch and, when profiling is on,
// brackets it with CUDA events on the launch stream (tdp_profile_*).
void launch_begin(cudaStream_t st, const char* name, bool events_ok = true);
void launch_end(cudaStream_t st);

// Tuning knobs (tdp_set_tuning and the TDP_* environment variables) into ctx.
void tune_from_env(Ctx& ctx);

// Drivers.  Every pointer is a device pointer; all work is queued on ctx.stream.
void solve_single(Ctx& ctx, const void* a, const void* b, const void* c, const void* d, void* x, int64_t n,
                  int s, tdp_dtype dt, int refine_iters);
void solve_batched(Ctx& ctx, const int64_t* offsets, int32_t batch, int64_t total_n, const void* a,
                   const void* b, const void* c, const void* d, void* x, int s, tdp_dtype dt, int refine_iters);
void solve_const(Ctx& ctx, double a, double b, double c, const void* d, void* x, int64_t n, int32_t batch,
                 int64_t ss, int64_t es, int s, tdp_dtype dt, int refine_iters);
void predict_sizes(Ctx& ctx, const int64_t* offsets, int32_t batch, tdp_dtype dt, int32_t* s_out);
void solve_strided(Ctx& ctx, int32_t batch, int64_t n, int64_t sys_stride, int64_t elem_stride, const void* a,
                   const void* b, const void* c, const void* d, void* x, int s, tdp_dtype dt, int refine_iters);
void solve_backward(Ctx& ctx, const int64_t* offsets, int32_t batch, int64_t total_n, const void* a,
                    const void* b, const void* c, const void* x, const void* g, void* ga, void* gb, void* gc,
                    void* gd, int s, tdp_dtype dt);
void thomas_batched(Ctx& ctx, const int64_t* offsets, int32_t batch, int64_t total_n, const void* a,
                    const void* b, const void* c, const void* d, void* x, tdp_dtype dt);
// Single-system solve whose scratch is only the interface systems (binary64
// re-solves the interiors in Stage 3 instead of keeping coefficients).
void solve_single_lean(Ctx& ctx, const void* a, const void* b, const void* c, const void* d, void* x, int64_t n,
                       int s, tdp_dtype dt);
void stage1_only(Ctx& ctx, const void* a, const void* b, const void* c, const void* d, int64_t n, int s,
                 tdp_dtype dt, double* ra, double* rb, double* rc, double* rd);

// Error message of the calling host thread (tdp_last_error) and checked mode.
int set_last_error(int code, const std::string& msg);
bool checked_mode();
// Return code of a device status word (ST_* bits) and the same with the
// message recorded for fn.
int status_code(unsigned bits);
int status_error(unsigned bits, const char* fn);

// Predictor (host 1-NN over the loaded table; tdp_api.cu).
int32_t predict_s(int64_t n, int32_t batch, tdp_dtype dt);
int32_t predict_r(int64_t n, int32_t batch, tdp_dtype dt);
int load_rtable_file(const char* path);
int recursion_plan(int64_t n, int32_t batch, int32_t s, int R, tdp_dtype dt, int32_t* m_out, int cap);
void solve_host(Ctx& ctx, const void* a, const void* b, const void* c, const void* d, void* x, int64_t n, int s,
                tdp_dtype dt, int refine_iters);
void solve_multi(Ctx& ctx, const void* a, const void* b, const void* c, const void* d, void* x, int64_t n,
                 int32_t nrhs, int64_t ldd, int64_t ldx, int s, tdp_dtype dt);
// Flattened table for the device-side predictor: rows of (log2 n, log2 batch, s) per dtype.
int predictor_table(tdp_dtype dt, const double** feat, const int32_t** labels);

}  // namespace tdp
