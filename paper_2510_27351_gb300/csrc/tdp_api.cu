// C ABI of the solver: argument checks, per-stream workspace, error
// reporting, the sub-system-size predictor (Sec. II-E) and its table.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <thread>
#include <sstream>
#include <string>
#include <vector>

#include "tdp_internal.h"

namespace tdp {

namespace {

thread_local std::string g_last_error;
thread_local unsigned g_last_bits = 0;  // raw status word of the last checked call or tdp_status
std::atomic<int64_t> g_launches{0};
std::atomic<int> g_checked{0};

struct Workspace {
  char* buf = nullptr;
  size_t cap = 0;
  unsigned* status = nullptr;
};

std::mutex g_ws_mu;
std::map<std::pair<int, cudaStream_t>, Workspace> g_ws;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int check_ptrs(std::initializer_list<const void*> ptrs, const char* fn) {
  for (const void* p : ptrs) {
    if (!p) return set_error(TDP_EINVAL, std::string(fn) + ": null pointer");
    if (!aligned16(p)) return set_error(TDP_EINVAL, std::string(fn) + ": pointer not 16-byte aligned");
  }
  return TDP_OK;
}

int check_common(int64_t n, int32_t s, tdp_dtype dt, int32_t iters, const char* fn, bool allow_refine = true) {
  if (n < 1) return set_error(TDP_EINVAL, std::string(fn) + ": n must be >= 1");
  if (s != 0 && (s < 2 || s > 1024)) return set_error(TDP_EINVAL, std::string(fn) + ": s must be 0 or in [2, 1024]");
  if (dt != TDP_F64 && dt != TDP_F32 && !(allow_refine && dt == TDP_F32_REFINE))
    return set_error(TDP_EINVAL, std::string(fn) + ": unsupported dtype");
  if (iters < 0 || iters > 8) return set_error(TDP_EINVAL, std::string(fn) + ": refine_iters must be in [0, 8]");
  return TDP_OK;
}

Workspace* workspace_for(cudaStream_t st, int* dev_out) {
  int dev = 0;
  cudaGetDevice(&dev);
  *dev_out = dev;
  std::lock_guard<std::mutex> lk(g_ws_mu);
  return &g_ws[{dev, st}];
}

// Launch tuning knobs (tdp_set_tuning), process-wide.  Their start values
// come from the environment: TDP_SMEM_BUDGET (shared memory per CTA aimed
// for by the register-staged tiles), TDP_S_REC (sub-system size inside the
// interface recursion), TDP_S_TAIL (inside its one-launch tail), TDP_VTILE,
// TDP_COOP, TDP_REFINE3 (0/1 switches of the interleaved tiles, the one-launch
// tail and the three-pass refinement), TDP_RECURSION (1: the paper's
// recursion schedule), TDP_R (its number of recursive steps, -1 =
// predicted), TDP_SEGMENTED (1: one CTA per system for the interface systems
// of batches), TDP_PER_SYSTEM_S (1: batched solves with s = 0 choose s per
// system on the device), TDP_IFACE32 (1: the first level of the interface
// recursion of binary32 solves in binary32 arithmetic), TDP_REFINE_KEPT (1:
// the last refinement pass elementwise from kept binary32 coefficients),
// TDP_COOP_REG (1: the one-launch tail reads its 8-row blocks into
// registers), TDP_BATCH_FLAT (1: batches of systems of at least 4096 rows on
// average are solved as one block-diagonal system), TDP_VTILE_B (1: binary64
// Stage 1 at s = 8 or 16 keeps b in registers and a, c, d in the tile),
// TDP_VTILE_L (1: binary32 storage runs Stage 1 and Stage 3 on padded
// block-major tiles), TDP_WINDOW (1: the windowed single pass for binary32
// solves with binary64 refinement), TDP_WINDOW_HALO (its halo rows per side),
// TDP_WAIT_LOG2 (log2 of the clock-cycle budget of every bounded device wait),
// TDP_WAIT_NEVER (1: the grid barriers wait for one arrival more than the
// grid has, so that every such wait runs out; for testing the timeout path),
// TDP_WINDOW_SW (rows per thread of the windowed pass's window, 5 or 7),
// TDP_WINDOW32 (1: binary32 storage takes the windowed pass too),
// TDP_WINDOW_PREFETCH (the windowed pass's L2 prefetch distance in tiles),
// TDP_WINDOW_HALO32 (the binary32 windowed pass's halo rows per side) and
// TDP_WINDOW_SW32 (its most rows per thread, 5 to 13).
// Keys 5 to 8 belonged to variants that were measured slower and removed;
// they are rejected.
struct Knob {
  const char* env;
  int lo, hi;
  std::atomic<int> v;
  bool retired;
};
Knob g_knobs[29] = {
    {"TDP_SMEM_BUDGET", 4096, 227 * 1024, {100 * 1024}, false},
    {"TDP_S_REC", 3, 1024, {16}, false},
    {"TDP_S_TAIL", 3, 256, {8}, false},
    {"TDP_VTILE", 0, 1, {1}, false},
    {"TDP_COOP", 0, 1, {1}, false},
    {"(retired key 5)", 0, 0, {0}, true},
    {"(retired key 6)", 0, 0, {0}, true},
    {"(retired key 7)", 0, 0, {0}, true},
    {"(retired key 8)", 0, 0, {0}, true},
    {"TDP_REFINE3", 0, 1, {1}, false},
    {"TDP_RECURSION", 0, 1, {0}, false},
    {"TDP_R", -1, 12, {-1}, false},
    {"TDP_SEGMENTED", 0, 1, {1}, false},
    {"TDP_PER_SYSTEM_S", 0, 1, {0}, false},
    {"TDP_IFACE32", 0, 1, {0}, false},
    {"TDP_REFINE_KEPT", 0, 1, {1}, false},
    {"TDP_COOP_REG", 0, 1, {1}, false},
    {"TDP_BATCH_FLAT", 0, 1, {1}, false},
    {"TDP_VTILE_B", 0, 1, {1}, false},
    {"TDP_VTILE_L", 0, 1, {1}, false},
    {"TDP_WINDOW", 0, 1, {1}, false},
    {"TDP_WINDOW_HALO", 16, 64, {48}, false},
    {"TDP_WAIT_LOG2", 10, 40, {31}, false},
    {"TDP_WAIT_NEVER", 0, 1, {0}, false},
    {"TDP_WINDOW_SW", 5, 7, {7}, false},
    {"TDP_WINDOW32", 0, 1, {1}, false},
    {"TDP_WINDOW_PREFETCH", 0, 4096, {128}, false},
    {"TDP_WINDOW_HALO32", 16, 64, {32}, false},
    {"TDP_WINDOW_SW32", 5, 13, {13}, false},
};
std::once_flag g_knobs_once;

void knobs_init() {
  std::call_once(g_knobs_once, [] {
    for (Knob& k : g_knobs) {
      if (k.retired) continue;
      if (const char* v = std::getenv(k.env)) {
        const int r = std::atoi(v);
        if (r >= k.lo && r <= k.hi) k.v.store(r);
      }
    }
  });
}

void load_knobs(Ctx& ctx) {
  knobs_init();
  ctx.smem_budget = g_knobs[TDP_TUNE_SMEM_BUDGET].v.load();
  ctx.s_rec = g_knobs[TDP_TUNE_S_REC].v.load();
  ctx.s_tail = g_knobs[TDP_TUNE_S_TAIL].v.load();
  ctx.vtile = g_knobs[TDP_TUNE_VTILE].v.load() != 0;
  ctx.coop = g_knobs[TDP_TUNE_COOP].v.load() != 0;
  ctx.refine3 = g_knobs[TDP_TUNE_REFINE3].v.load() != 0;
  ctx.rec_mode = g_knobs[TDP_TUNE_RECURSION].v.load();
  ctx.rec_force = g_knobs[TDP_TUNE_R].v.load();
  ctx.seg = g_knobs[TDP_TUNE_SEGMENTED].v.load() != 0;
  ctx.per_system_s = g_knobs[TDP_TUNE_PER_SYSTEM_S].v.load() != 0;
  ctx.iface32 = g_knobs[TDP_TUNE_IFACE32].v.load() != 0;
  ctx.refine_kept = g_knobs[TDP_TUNE_REFINE_KEPT].v.load() != 0;
  ctx.coop_reg = g_knobs[TDP_TUNE_COOP_REG].v.load() != 0;
  ctx.batch_flat = g_knobs[TDP_TUNE_BATCH_FLAT].v.load() != 0;
  ctx.vtile_b = g_knobs[TDP_TUNE_VTILE_B].v.load() != 0;
  ctx.vtile_l = g_knobs[TDP_TUNE_VTILE_L].v.load() != 0;
  ctx.window = g_knobs[TDP_TUNE_WINDOW].v.load() != 0;
  ctx.window_halo = g_knobs[TDP_TUNE_WINDOW_HALO].v.load();
  ctx.wait_log2 = g_knobs[TDP_TUNE_WAIT_LOG2].v.load();
  ctx.wait_never = g_knobs[TDP_TUNE_WAIT_NEVER].v.load() != 0;
  ctx.window_sw = g_knobs[TDP_TUNE_WINDOW_SW].v.load();
  ctx.window32 = g_knobs[TDP_TUNE_WINDOW32].v.load() != 0;
  ctx.window_prefetch = g_knobs[TDP_TUNE_WINDOW_PREFETCH].v.load();
  ctx.window_halo32 = g_knobs[TDP_TUNE_WINDOW_HALO32].v.load();
  ctx.window_sw32 = g_knobs[TDP_TUNE_WINDOW_SW32].v.load();
}

// Run a driver twice: a dry run that sizes the workspace, then the real one.
template <typename F>
int run(void* stream, const char* fn, F&& driver) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  Workspace* ws = workspace_for(st, &dev);
  Arena sizing;
  Ctx dry;
  load_knobs(dry);
  dry.stream = st;
  dry.ar = &sizing;
  dry.dry = true;
  driver(dry);
  const size_t need = sizing.off + 256;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return set_error(TDP_ECUDA, std::string(fn) + ": bad stream");
  if (!ws->status || need > ws->cap) {
    if (cap != cudaStreamCaptureStatusNone)
      return set_error(TDP_ENOMEM, std::string(fn) + ": workspace must be reserved before stream capture (need " +
                                       std::to_string(need) + " bytes)");
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(TDP_ECUDA, std::string(fn) + ": " + cudaGetErrorString(e));
    if (!ws->status) {
      e = cudaMalloc(&ws->status, 256);
      if (e == cudaSuccess) e = cudaMemset(ws->status, 0, 256);
      if (e != cudaSuccess) return set_error(TDP_ENOMEM, std::string(fn) + ": status word: " + cudaGetErrorString(e));
    }
    if (need > ws->cap) {
      if (ws->buf) cudaFree(ws->buf);
      ws->buf = nullptr;
      ws->cap = 0;
      const size_t grow = need + need / 8;
      e = cudaMalloc(&ws->buf, grow);
      if (e != cudaSuccess) {
        ws->buf = nullptr;
        cudaGetLastError();
        return set_error(TDP_ENOMEM, std::string(fn) + ": workspace of " + std::to_string(grow) +
                                         " bytes: " + cudaGetErrorString(e));
      }
      ws->cap = grow;
    }
  }
  Arena arena;
  arena.base = ws->buf;
  arena.cap = ws->cap;
  Ctx ctx;
  load_knobs(ctx);
  ctx.stream = st;
  ctx.status = ws->status;
  ctx.ar = &arena;
  arena.err = &ctx.err;
  driver(ctx);
  if (ctx.err != cudaSuccess)
    return set_error(TDP_ECUDA, std::string(fn) + ": " + (ctx.msg.empty() ? "workspace overrun" : ctx.msg));
  if (g_checked.load()) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(TDP_ECUDA, std::string(fn) + ": " + cudaGetErrorString(e));
    unsigned h = 0;
    e = cudaMemcpy(&h, ws->status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ws->status, 0, sizeof(unsigned));
    if (e != cudaSuccess) return set_error(TDP_ECUDA, std::string(fn) + ": " + cudaGetErrorString(e));
    g_last_bits = h;
    if (status_code(h) != TDP_OK) return status_error(h, fn);
  }
  g_last_error.clear();
  return TDP_OK;
}

// ---------------------------------------------------------------------------
// Predictor table: rows (dtype, n, batch, s).  The built-in rows are the
// labels measured on GB300 by the sweep shipped with the Python package; when
// a dtype has no rows the paper's interval rule (Sec. II-D) is used.
// ---------------------------------------------------------------------------
struct Row {
  int dt;
  double n, batch;
  int s;
};

#include "tdp_table.inc"

std::mutex g_tab_mu;
std::vector<Row> g_table;
bool g_table_init = false;
std::vector<double> g_feat[3];
std::vector<int32_t> g_lab[3];

void ensure_table() {
  if (g_table_init) return;
  for (const Row& r : kBuiltinTable) g_table.push_back(r);
  g_table_init = true;
}

// Rows (dtype, n, batch, R) of the recursion-depth model; the built-in rows
// come from the GB300 sweep of R.  Without rows for a dtype the intervals of
// the paper's table of optimum recursive steps (Sec. III-A) are used.
struct RRow {
  int dt;
  double n, batch;
  int r;
};

#include "tdp_rtable.inc"

std::vector<RRow> g_rtable;
bool g_rtable_init = false;

void ensure_rtable() {
  if (g_rtable_init) return;
  for (const RRow& r : kBuiltinRTable)
    if (r.r >= 0) g_rtable.push_back(r);
  g_rtable_init = true;
}

int r_interval_rule(double n) {
  if (n <= 2.2e6) return 0;
  if (n <= 4.8e6) return 1;
  if (n <= 9.6e6) return 2;
  return 3;
}

int interval_rule(double n) {
  // Sec. II-D, FP64 on RTX 2080 Ti
  if (n <= 4.5e3) return 4;
  if (n <= 2.5e4) return 8;
  if (n <= 5e4) return 16;
  if (n <= 7.5e4) return 20;
  if (n <= 1e7) return 32;
  return 64;
}

}  // namespace

int set_last_error(int code, const std::string& msg) { return set_error(code, msg); }

void tune_from_env(Ctx& ctx) { load_knobs(ctx); }
// Return code of a device status word; when several bits are set the
// argument error wins over a timeout, and a timeout over a pivot failure.
int status_code(unsigned h) {
  if (h & ST_BADARG) return TDP_EINVAL;
  if (h & ST_TIMEOUT) return TDP_ETIMEOUT;
  if (h & ST_SINGULAR) return TDP_ESINGULAR;
  return TDP_OK;
}

int status_error(unsigned h, const char* fn) {
  const int code = status_code(h);
  const char* what = code == TDP_EINVAL     ? ": offsets rejected on the device"
                     : code == TDP_ETIMEOUT ? ": device wait timed out"
                     : code == TDP_ESINGULAR ? ": zero or non-finite pivot"
                                            : "";
  return set_last_error(code, std::string(fn) + what);
}

bool checked_mode() { return g_checked.load() != 0; }

// ---------------------------------------------------------------------------
// Launch counting and event-based per-kernel timing.
// ---------------------------------------------------------------------------
namespace {
struct ProfRec {
  const char* name;
  cudaEvent_t e0, e1;
};
std::mutex g_prof_mu;
std::atomic<int> g_prof_on{0};
std::vector<ProfRec> g_prof;
thread_local cudaEvent_t t_open = nullptr;
thread_local const char* t_open_name = nullptr;
}  // namespace

void launch_begin(cudaStream_t st, const char* name, bool events_ok) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  t_open = nullptr;
  if (!events_ok || !g_prof_on.load(std::memory_order_relaxed)) return;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
  cudaEvent_t e0;
  if (cudaEventCreate(&e0) != cudaSuccess) return;
  cudaEventRecord(e0, st);
  t_open = e0;
  t_open_name = name;
}

void launch_end(cudaStream_t st) {
  if (!t_open) return;
  cudaEvent_t e1;
  if (cudaEventCreate(&e1) != cudaSuccess) return;
  cudaEventRecord(e1, st);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof.push_back(ProfRec{t_open_name, t_open, e1});
  t_open = nullptr;
}

void profile_clear() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& r : g_prof) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  g_prof.clear();
}

std::string profile_text() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  std::map<std::string, std::pair<int64_t, double>> agg;
  std::vector<std::string> order;
  for (auto& r : g_prof) {
    cudaEventSynchronize(r.e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.e0, r.e1);
    auto it = agg.find(r.name);
    if (it == agg.end()) {
      order.push_back(r.name);
      agg[r.name] = {1, double(ms)};
    } else {
      it->second.first += 1;
      it->second.second += ms;
    }
  }
  std::ostringstream os;
  for (auto& k : order) os << k << ' ' << agg[k].first << ' ' << agg[k].second << '\n';
  return os.str();
}

int32_t predict_s(int64_t n, int32_t batch, tdp_dtype dt) {
  std::lock_guard<std::mutex> lk(g_tab_mu);
  ensure_table();
  const double ln = std::log2(double(n < 1 ? 1 : n));
  const double lb = std::log2(double(batch < 1 ? 1 : batch));
  double best = 1e300;
  int s = 0;
  for (const Row& r : g_table) {
    if (r.dt != int(dt)) continue;
    const double dn = std::log2(r.n) - ln, db = std::log2(r.batch) - lb;
    const double dist = dn * dn + db * db;
    if (dist < best || (dist == best && r.s > s)) {
      best = dist;
      s = r.s;
    }
  }
  if (s < 2) s = interval_rule(double(n));
  return s;
}

int32_t predict_r(int64_t n, int32_t batch, tdp_dtype dt) {
  std::lock_guard<std::mutex> lk(g_tab_mu);
  ensure_rtable();
  const double ln = std::log2(double(n < 1 ? 1 : n));
  const double lb = std::log2(double(batch < 1 ? 1 : batch));
  double best = 1e300;
  int r = -1;
  for (const RRow& row : g_rtable) {
    if (row.dt != int(dt)) continue;
    const double dn = std::log2(row.n) - ln, db = std::log2(row.batch) - lb;
    const double dist = dn * dn + db * db;
    if (dist < best || (dist == best && row.r > r)) {
      best = dist;
      r = row.r;
    }
  }
  if (r < 0) r = r_interval_rule(double(n));
  return r;
}

int load_rtable_file(const char* path) {
  if (path[0] == '\0') {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    g_rtable.clear();
    g_rtable_init = false;
    ensure_rtable();
    return TDP_OK;
  }
  std::ifstream in(path);
  if (!in) return set_error(TDP_EINVAL, std::string("tdp_load_rtable: cannot open ") + path);
  std::vector<RRow> rows;
  std::string line;
  while (std::getline(in, line)) {
    const size_t h = line.find('#');
    if (h != std::string::npos) line.resize(h);
    std::istringstream ss(line);
    RRow r;
    if (!(ss >> r.dt >> r.n >> r.batch >> r.r)) continue;
    if (r.dt < 0 || r.dt > 2 || r.n < 1 || r.batch < 1 || r.r < 0 || r.r > 12)
      return set_error(TDP_EINVAL, "tdp_load_rtable: bad row: " + line);
    rows.push_back(r);
  }
  std::lock_guard<std::mutex> lk(g_tab_mu);
  g_rtable = rows;
  g_rtable_init = true;
  return TDP_OK;
}

int predictor_table(tdp_dtype dt, const double** feat, const int32_t** labels) {
  std::lock_guard<std::mutex> lk(g_tab_mu);
  ensure_table();
  auto& f = g_feat[int(dt)];
  auto& l = g_lab[int(dt)];
  f.clear();
  l.clear();
  for (const Row& r : g_table) {
    if (r.dt != int(dt)) continue;
    f.push_back(std::log2(r.n));
    f.push_back(std::log2(r.batch));
    l.push_back(r.s);
  }
  *feat = f.data();
  *labels = l.data();
  return int(l.size());
}

int load_table_file(const char* path) {
  if (path[0] == '\0') {  // restore the built-in table
    std::lock_guard<std::mutex> lk(g_tab_mu);
    g_table.clear();
    g_table_init = false;
    ensure_table();
    return TDP_OK;
  }
  std::ifstream in(path);
  if (!in) return set_error(TDP_EINVAL, std::string("tdp_load_table: cannot open ") + path);
  std::vector<Row> rows;
  std::string line;
  while (std::getline(in, line)) {
    const size_t h = line.find('#');
    if (h != std::string::npos) line.resize(h);
    std::istringstream ss(line);
    Row r;
    if (!(ss >> r.dt >> r.n >> r.batch >> r.s)) continue;
    if (r.dt < 0 || r.dt > 2 || r.n < 1 || r.batch < 1 || r.s < 2 || r.s > 1024)
      return set_error(TDP_EINVAL, "tdp_load_table: bad row: " + line);
    rows.push_back(r);
  }
  std::lock_guard<std::mutex> lk(g_tab_mu);
  g_table = rows;
  g_table_init = true;
  return TDP_OK;
}

}  // namespace tdp

using namespace tdp;

extern "C" {

int tdp_solve(const void* a, const void* b, const void* c, const void* d, void* x, int64_t n, int32_t s,
              tdp_dtype dtype, int32_t refine_iters, void* stream) {
  int rc = check_common(n, s, dtype, refine_iters, "tdp_solve");
  if (rc) return rc;
  if ((rc = check_ptrs({a, b, c, d, x}, "tdp_solve"))) return rc;
  const int ss = s ? s : predict_s(n, 1, dtype);
  return run(stream, "tdp_solve", [&](Ctx& ctx) { solve_single(ctx, a, b, c, d, x, n, ss, dtype, refine_iters); });
}

int tdp_solve_batched(const int64_t* offsets, int32_t batch, int64_t total_n, const void* a, const void* b,
                      const void* c, const void* d, void* x, int32_t s, tdp_dtype dtype, int32_t refine_iters,
                      void* stream) {
  if (batch < 1) return set_error(TDP_EINVAL, "tdp_solve_batched: batch must be >= 1");
  if (total_n < 0) return set_error(TDP_EINVAL, "tdp_solve_batched: total_n must be >= 0");
  int rc = check_common(total_n < 1 ? 1 : total_n, s, dtype, refine_iters, "tdp_solve_batched");
  if (rc) return rc;
  if (!offsets) return set_error(TDP_EINVAL, "tdp_solve_batched: null offsets");
  if (total_n == 0) return TDP_OK;
  if ((rc = check_ptrs({a, b, c, d, x}, "tdp_solve_batched"))) return rc;
  return run(stream, "tdp_solve_batched", [&](Ctx& ctx) {
    solve_batched(ctx, offsets, batch, total_n, a, b, c, d, x, s, dtype, refine_iters);
  });
}

int tdp_solve_const(double a, double b, double c, const void* d, void* x, int64_t n, int32_t batch,
                    int64_t sys_stride, int64_t elem_stride, int32_t s, tdp_dtype dtype, int32_t refine_iters,
                    void* stream) {
  const char* fn = "tdp_solve_const";
  if (batch < 1) return set_error(TDP_EINVAL, std::string(fn) + ": batch must be >= 1");
  if (s != 0 && (s < 2 || s > 512)) return set_error(TDP_EINVAL, std::string(fn) + ": s must be 0 or in [2, 512]");
  int rc = check_common(n, 0, dtype, refine_iters, fn);
  if (rc) return rc;
  if (sys_stride < 1 || elem_stride < 1)
    return set_error(TDP_EINVAL, std::string(fn) + ": strides must be >= 1");
  // systems must not overlap: interleaved (elem_stride >= batch * sys_stride)
  // or one after another (sys_stride >= n * elem_stride)
  if (!(elem_stride >= int64_t(batch) * sys_stride || sys_stride >= n * elem_stride))
    return set_error(TDP_EINVAL, std::string(fn) + ": strides make systems overlap");
  const size_t el = dtype == TDP_F32 ? 4 : 8;
  if (!d || !x) return set_error(TDP_EINVAL, std::string(fn) + ": null pointer");
  if ((reinterpret_cast<uintptr_t>(d) | reinterpret_cast<uintptr_t>(x)) % el)
    return set_error(TDP_EINVAL, std::string(fn) + ": pointer not aligned to its element");
  if (d == x) return set_error(TDP_EINVAL, std::string(fn) + ": x must not alias d");
  // (TDP_F32_REFINE runs in binary64 arithmetic here: the binary64 size model)
  const int ss2 = s ? s : std::min(512, int(predict_s(n, batch, dtype == TDP_F32 ? TDP_F32 : TDP_F64)));
  return run(stream, fn, [&](Ctx& ctx) {
    solve_const(ctx, a, b, c, d, x, n, batch, sys_stride, elem_stride, ss2, dtype, refine_iters);
  });
}

int tdp_solve_host(const void* a, const void* b, const void* c, const void* d, void* x, int64_t n, int32_t s,
                   tdp_dtype dtype, int32_t refine_iters, void* stream) {
  const char* fn = "tdp_solve_host";
  int rc = check_common(n, s, dtype, refine_iters, fn);
  if (rc) return rc;
  if (!a || !b || !c || !d || !x) return set_error(TDP_EINVAL, std::string(fn) + ": null pointer");
  const size_t el = dtype == TDP_F32 ? 4 : 8;
  const uintptr_t x0 = reinterpret_cast<uintptr_t>(x), x1 = x0 + size_t(n) * el;
  for (const void* p : {a, b, c, d}) {
    const uintptr_t p0 = reinterpret_cast<uintptr_t>(p), p1 = p0 + size_t(n) * el;
    if (x0 < p1 && p0 < x1) return set_error(TDP_EINVAL, std::string(fn) + ": x overlaps an input");
  }
  const int ss = s ? s : predict_s(n, 1, dtype);
  return run(stream, fn, [&](Ctx& ctx) { solve_host(ctx, a, b, c, d, x, n, ss, dtype, refine_iters); });
}

int tdp_solve_multi(const void* a, const void* b, const void* c, const void* d, void* x, int64_t n, int32_t nrhs,
                    int64_t ldd, int64_t ldx, int32_t s, tdp_dtype dtype, void* stream) {
  const char* fn = "tdp_solve_multi";
  if (dtype != TDP_F64 && dtype != TDP_F32)
    return set_error(TDP_EINVAL, std::string(fn) + ": dtype must be F64 or F32");
  int rc = check_common(n, s, dtype, 0, fn);
  if (rc) return rc;
  if (nrhs < 1 || nrhs > 65535) return set_error(TDP_EINVAL, std::string(fn) + ": nrhs must be in [1, 65535]");
  if (ldd < n || ldx < n) return set_error(TDP_EINVAL, std::string(fn) + ": ldd and ldx must be >= n");
  if (!a || !b || !c || !d || !x) return set_error(TDP_EINVAL, std::string(fn) + ": null pointer");
  const size_t el = dtype == TDP_F32 ? 4 : 8;
  for (const void* p : {a, b, c, d, (const void*)x})
    if (reinterpret_cast<uintptr_t>(p) % 16)
      return set_error(TDP_EINVAL, std::string(fn) + ": pointer not 16-byte aligned");
  if ((size_t(ldd) * el) % 16 || (size_t(ldx) * el) % 16)
    return set_error(TDP_EINVAL, std::string(fn) + ": columns must start on 16-byte boundaries (ldd, ldx)");
  const uintptr_t x0 = reinterpret_cast<uintptr_t>(x), d0 = reinterpret_cast<uintptr_t>(d);
  const uintptr_t x1 = x0 + (uintptr_t(nrhs - 1) * uintptr_t(ldx) + uintptr_t(n)) * el;
  const uintptr_t d1 = d0 + (uintptr_t(nrhs - 1) * uintptr_t(ldd) + uintptr_t(n)) * el;
  if (x0 < d1 && d0 < x1) return set_error(TDP_EINVAL, std::string(fn) + ": x overlaps d");
  // s = 0: a column costs the d-part only, so the interface share of a column
  // is larger than in one solve: four times the single-solve model's s,
  // within [16, 64] (n = 2^22, 16 binary64 columns: s = 32 1.26 ms, the
  // single-solve s = 8 1.65 ms)
  const int ss = s ? s : std::min(64, std::max(16, 4 * int(predict_s(n, 1, dtype))));
  return run(stream, fn, [&](Ctx& ctx) { solve_multi(ctx, a, b, c, d, x, n, nrhs, ldd, ldx, ss, dtype); });
}

int tdp_solve_strided(int32_t batch, int64_t n, int64_t sys_stride, int64_t elem_stride, const void* a,
                      const void* b, const void* c, const void* d, void* x, int32_t s, tdp_dtype dtype,
                      int32_t refine_iters, void* stream) {
  if (batch < 1) return set_error(TDP_EINVAL, "tdp_solve_strided: batch must be >= 1");
  int rc = check_common(n, s, dtype, refine_iters, "tdp_solve_strided");
  if (rc) return rc;
  if (sys_stride < 0 || elem_stride < 1) return set_error(TDP_EINVAL, "tdp_solve_strided: bad strides");
  if ((rc = check_ptrs({a, b, c, d, x}, "tdp_solve_strided"))) return rc;
  const int ss = s ? s : predict_s(n, batch, dtype);
  return run(stream, "tdp_solve_strided", [&](Ctx& ctx) {
    solve_strided(ctx, batch, n, sys_stride, elem_stride, a, b, c, d, x, ss, dtype, refine_iters);
  });
}

int tdp_solve_backward(const int64_t* offsets, int32_t batch, int64_t total_n, const void* a, const void* b,
                       const void* c, const void* x, const void* g, void* grad_a, void* grad_b, void* grad_c,
                       void* grad_d, int32_t s, tdp_dtype dtype, void* stream) {
  if (batch < 1) return set_error(TDP_EINVAL, "tdp_solve_backward: batch must be >= 1");
  int rc = check_common(total_n < 1 ? 1 : total_n, s, dtype, 0, "tdp_solve_backward");
  if (rc) return rc;
  if (!offsets) return set_error(TDP_EINVAL, "tdp_solve_backward: null offsets");
  if (total_n == 0) return TDP_OK;
  if ((rc = check_ptrs({a, b, c, x, g}, "tdp_solve_backward"))) return rc;
  for (const void* p : {(const void*)grad_a, (const void*)grad_b, (const void*)grad_c, (const void*)grad_d})
    if (p && !aligned16(p)) return set_error(TDP_EINVAL, "tdp_solve_backward: gradient not 16-byte aligned");
  // the transposed batch is solved as one system of total_n rows
  const int ss = s ? s : predict_s(total_n, 1, dtype);
  return run(stream, "tdp_solve_backward", [&](Ctx& ctx) {
    solve_backward(ctx, offsets, batch, total_n, a, b, c, x, g, grad_a, grad_b, grad_c, grad_d, ss, dtype);
  });
}

int tdp_predict_s_batched(const int64_t* offsets, int32_t batch, tdp_dtype dtype, int32_t* s_out, void* stream) {
  if (batch < 1) return set_error(TDP_EINVAL, "tdp_predict_s_batched: batch must be >= 1");
  if (!offsets || !s_out) return set_error(TDP_EINVAL, "tdp_predict_s_batched: null pointer");
  if (dtype != TDP_F64 && dtype != TDP_F32 && dtype != TDP_F32_REFINE)
    return set_error(TDP_EINVAL, "tdp_predict_s_batched: unsupported dtype");
  return run(stream, "tdp_predict_s_batched", [&](Ctx& ctx) { predict_sizes(ctx, offsets, batch, dtype, s_out); });
}

int32_t tdp_predict_r(int64_t n, int32_t batch, tdp_dtype dtype) {
  if (n < 1 || batch < 1 || int(dtype) < 0 || int(dtype) > 2) return -1;
  return predict_r(n, batch, dtype);
}

int tdp_load_rtable(const char* path) {
  if (!path) return set_error(TDP_EINVAL, "tdp_load_rtable: null path");
  return load_rtable_file(path);
}

int32_t tdp_recursion_plan(int64_t n, int32_t s, int32_t R, tdp_dtype dtype, int32_t* m_out, int32_t cap) {
  if (n < 1 || s < 2 || s > 1024 || R > 12 || int(dtype) < 0 || int(dtype) > 2 || cap < 0 || (cap > 0 && !m_out))
    return -1;
  return recursion_plan(n, 1, s, R, dtype, m_out, cap);
}

int32_t tdp_predict_s(int64_t n, int32_t batch, tdp_dtype dtype) {
  if (dtype != TDP_F64 && dtype != TDP_F32 && dtype != TDP_F32_REFINE) dtype = TDP_F64;
  return predict_s(n, batch, dtype);
}

int tdp_load_table(const char* path) {
  if (!path) return set_error(TDP_EINVAL, "tdp_load_table: null path");
  return load_table_file(path);
}

int tdp_reserve(int64_t total_n, int32_t batch, int32_t s, tdp_dtype dtype, void* stream) {
  if (total_n < 1 || batch < 1) return set_error(TDP_EINVAL, "tdp_reserve: sizes must be >= 1");
  if (s == 0) s = 2;
  int rc = check_common(total_n, s, dtype, 0, "tdp_reserve");
  if (rc) return rc;
  // size for the largest consumer: a batched refined solve with 8 corrections
  return run(stream, "tdp_reserve", [&](Ctx& ctx) {
    if (!ctx.dry) return;
    solve_batched(ctx, nullptr, batch, total_n, nullptr, nullptr, nullptr, nullptr, nullptr, s, dtype,
                  dtype == TDP_F32_REFINE ? 8 : 0);
    solve_backward(ctx, nullptr, batch, total_n, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                   nullptr, nullptr, s, dtype == TDP_F32_REFINE ? TDP_F64 : dtype);
  });
}

int tdp_status(void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  Workspace* ws = workspace_for(st, &dev);
  if (!ws->status) return TDP_OK;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(TDP_ECUDA, std::string("tdp_status: ") + cudaGetErrorString(e));
  unsigned h = 0;
  e = cudaMemcpy(&h, ws->status, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(ws->status, 0, sizeof(unsigned));
  if (e != cudaSuccess) return set_error(TDP_ECUDA, std::string("tdp_status: ") + cudaGetErrorString(e));
  g_last_bits = h;
  return status_code(h) != TDP_OK ? status_error(h, "tdp_status") : TDP_OK;
}

void tdp_set_checked(int on) { g_checked.store(on ? 1 : 0); }

int tdp_set_tuning(int key, int value) {
  knobs_init();
  if (key < 0 || key >= int(sizeof(g_knobs) / sizeof(g_knobs[0])))
    return set_error(TDP_EINVAL, "tdp_set_tuning: unknown key");
  Knob& k = g_knobs[key];
  if (k.retired) return set_error(TDP_EINVAL, "tdp_set_tuning: key " + std::to_string(key) + " is retired");
  if (value < k.lo || value > k.hi)
    return set_error(TDP_EINVAL, std::string("tdp_set_tuning: ") + k.env + " must be in [" + std::to_string(k.lo) +
                                     ", " + std::to_string(k.hi) + "]");
  k.v.store(value);
  return TDP_OK;
}

int tdp_get_tuning(int key) {
  knobs_init();
  if (key < 0 || key >= int(sizeof(g_knobs) / sizeof(g_knobs[0])) || g_knobs[key].retired) return -1;
  return g_knobs[key].v.load();
}

const char* tdp_last_error(void) { return g_last_error.c_str(); }

int64_t tdp_launch_count(void) { return g_launches.load(); }

int tdp_status_code(uint32_t bits) { return status_code(bits); }

uint32_t tdp_last_status_bits(void) { return g_last_bits; }

void tdp_profile_enable(int on) {
  profile_clear();
  g_prof_on.store(on ? 1 : 0);
}

int64_t tdp_profile_summary(char* buf, int64_t len) {
  const std::string txt = profile_text();
  if (buf && len > 0) {
    const size_t k = std::min<size_t>(txt.size(), size_t(len - 1));
    std::memcpy(buf, txt.data(), k);
    buf[k] = '\0';
  }
  return int64_t(txt.size());
}

int tdp_thomas_batched(const int64_t* offsets, int32_t batch, int64_t total_n, const void* a, const void* b,
                       const void* c, const void* d, void* x, tdp_dtype dtype, void* stream) {
  if (batch < 1) return set_error(TDP_EINVAL, "tdp_thomas_batched: batch must be >= 1");
  int rc = check_common(total_n < 1 ? 1 : total_n, 2, dtype, 0, "tdp_thomas_batched", false);
  if (rc) return rc;
  if (!offsets) return set_error(TDP_EINVAL, "tdp_thomas_batched: null offsets");
  if (total_n == 0) return TDP_OK;
  if ((rc = check_ptrs({a, b, c, d, x}, "tdp_thomas_batched"))) return rc;
  return run(stream, "tdp_thomas_batched",
             [&](Ctx& ctx) { thomas_batched(ctx, offsets, batch, total_n, a, b, c, d, x, dtype); });
}

int tdp_stage1(const void* a, const void* b, const void* c, const void* d, int64_t n, int32_t s, tdp_dtype dtype,
               double* ra, double* rb, double* rc, double* rd, void* stream) {
  int r = check_common(n, s == 0 ? 2 : s, dtype, 0, "tdp_stage1");
  if (r) return r;
  if ((r = check_ptrs({a, b, c, d, ra, rb, rc, rd}, "tdp_stage1"))) return r;
  const int ss = s ? s : predict_s(n, 1, dtype);
  return run(stream, "tdp_stage1", [&](Ctx& ctx) { stage1_only(ctx, a, b, c, d, n, ss, dtype, ra, rb, rc, rd); });
}

}  // extern "C"
