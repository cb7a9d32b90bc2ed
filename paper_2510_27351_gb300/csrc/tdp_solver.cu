// Solver drivers: launch geometry, workspace layout and the order of the
// stages of the partition method (Sec. I), for single, batched, strided and
// transposed (adjoint) solves.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <type_traits>
#include <utility>
#include <vector>

#include "tdp_internal.h"
#include "tdp_vtile.cuh"
#include "tdp_vtile_b.cuh"
#include "tdp_vtile_l.cuh"
#include "tdp_coop.cuh"
#include "tdp_refine.cuh"
#include "tdp_const.cuh"
#include "tdp_multi.cuh"
#include "tdp_window.cuh"

namespace tdp {

namespace {

constexpr int kMaxSmem = 227 * 1024;
constexpr int64_t kBaseRows = 64;  // interface systems this small go to one thread

unsigned magic_for(int s) { return unsigned((uint64_t(1) << 32) / uint64_t(s) + 1); }

// Opt every tile kernel in to the full shared memory once (per kernel and device).
template <typename K>
void allow_smem(K kernel) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  cudaGetDevice(&dev);
  const std::pair<int, const void*> key{dev, reinterpret_cast<const void*>(kernel)};
  std::lock_guard<std::mutex> lk(mu);
  if (done.count(key)) return;
  // the per-CTA limit covers static and dynamic shared memory together
  cudaFuncAttributes fa{};
  const int stat = cudaFuncGetAttributes(&fa, kernel) == cudaSuccess ? int(fa.sharedSizeBytes) : 0;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem - stat);
  done.insert(key);
}

// Threads (= blocks) per CTA for a tile kernel holding `arrays` tiles of
// `elem` bytes per row, plus 4 bytes per row of owner table when mapped.
int pick_threads(const Ctx& ctx, int s, int arrays, int elem, bool mapped, size_t* smem_out, int budget = 0) {
  auto bytes = [&](int T) {
    return size_t(arrays) * elem * size_t(s) * (T + 1) + (mapped ? size_t(4) * T * s : 0);
  };
  const size_t limit = size_t(budget > 0 ? std::min(budget, ctx.smem_budget) : ctx.smem_budget);
  int T = 256;
  while (T > 32 && bytes(T) > limit) T /= 2;
  while (T > 1 && bytes(T) > size_t(kMaxSmem)) --T;
  *smem_out = bytes(T);
  return T;
}

void pre_launch(Ctx& ctx, const char* what) { launch_begin(ctx.stream, what, ctx.events_ok); }

void post_launch(Ctx& ctx, const char* what) {
  launch_end(ctx.stream);
  ctx.fail(cudaGetLastError(), what);
}

template <typename C>
const char* tname(const char* f64, const char* f32) {
  return sizeof(C) == 8 ? f64 : f32;
}

// Number of SMs of the current device.
int sm_count() {
  static int count[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!count[dev]) cudaDeviceGetAttribute(&count[dev], cudaDevAttrMultiProcessorCount, dev);
  return count[dev] > 0 ? count[dev] : 1;
}

// Padded block-major binary32 tiles (tdp_vtile_l.cuh): threads per CTA (=
// blocks per tile) with at most 64 KB of tile per CTA, as for the
// interleaved binary32 tiles, fewer than 32 only where a block's rows need
// it (s up to 1024: 16 KB per thread).
int ltile_threads(int s, size_t* smem) {
  const size_t per = size_t(4) * size_t(ltile_pitch(s / 4)) * 16;  // four planes of pv 16-byte chunks
  int T = 256;
  while (T > 32 && per * T > size_t(64) * 1024) T /= 2;
  while (T > 1 && per * T > size_t(kMaxSmem)) --T;
  *smem = per * T;
  return T;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

template <typename S, typename C, bool MAPPED, bool KEEP>
void stage1(Ctx& ctx, const S* a, const S* b, const S* c, const S* d, int64_t n, int s, int64_t m,
            const int64_t* blk, double* ra, double* rb, double* rc, double* rd, C* ka, C* kg, C* kd,
            const char* name = nullptr) {
  if (ctx.dry || ctx.err != cudaSuccess || m <= 0) return;
  const char* nm = name ? name : KEEP ? "stage1_keep_f64" : tname<C>("stage1_f64", "stage1_f32");
  if constexpr (!MAPPED && !KEEP && std::is_same<S, float>::value && std::is_same<C, float>::value) {
    if (ctx.vtile && ctx.vtile_l && s % 4 == 0) {
      // padded block-major tiles (tdp_vtile_l.cuh)
      const int64_t kb = ctx.kb, ke = ctx.ke >= 0 ? ctx.ke : m;
      size_t smem;
      const int T = ltile_threads(s, &smem);
      allow_smem(k_stage1_l);
      pre_launch(ctx, nm);
      k_stage1_l<<<unsigned((ke - kb + T - 1) / T), T, smem, ctx.stream>>>(a, b, c, d, n, s, m, ra, rb, rc, rd,
                                                                           ctx.flat_off, ctx.flat_nsys, kb, ke,
                                                                           ctx.status);
      post_launch(ctx, "stage 1");
      return;
    }
  }
  if constexpr (!MAPPED && KEEP && std::is_same<S, double>::value && std::is_same<C, double>::value) {
    if (ctx.vtile && ctx.vtile_b && (s == 8 || s == 16)) {
      // b in registers, a, c, d in the tile (tdp_vtile_b.cuh)
      const int T = s == 8 ? 128 : 64;
      const size_t smem = size_t(3) * 8 * s * (T + 1);
      auto vk = s == 8 ? k_stage1_vb<8> : k_stage1_vb<16>;
      allow_smem(vk);
      const int64_t kb = ctx.kb, ke = ctx.ke >= 0 ? ctx.ke : m;
      pre_launch(ctx, nm);
      vk<<<unsigned((ke - kb + T - 1) / T), T, smem, ctx.stream>>>(a, b, c, d, n, m, ra, rb, rc, rd, ka, kg, kd,
                                                                   ctx.flat_off, ctx.flat_nsys, kb, ke, ctx.status);
      post_launch(ctx, "stage 1");
      return;
    }
  }
  if constexpr (!MAPPED && std::is_same<S, C>::value) {
    if (ctx.vtile && s % Vec<S>::W == 0) {
      size_t smem;
      // binary32 tiles: smaller CTAs (at most 64 KB) interleave their load
      // and sweep phases better (N = 2^26, s = 64: 0.797 -> 0.765 ms)
      const int T = pick_threads(ctx, s, 4, sizeof(S), false, &smem, sizeof(S) == 4 ? 64 * 1024 : 0);
      auto vk = k_stage1_v<S, C, KEEP>;
      allow_smem(vk);
      const int64_t kb = ctx.kb, ke = ctx.ke >= 0 ? ctx.ke : m;
      pre_launch(ctx, nm);
      vk<<<unsigned((ke - kb + T - 1) / T), T, smem, ctx.stream>>>(a, b, c, d, n, s, m, ra, rb, rc, rd, ka, kg, kd,
                                                                   ctx.flat_off, ctx.flat_nsys, kb, ke, ctx.status);
      post_launch(ctx, "stage 1");
      return;
    }
  }
  size_t smem;
  const int T = pick_threads(ctx, s, 4, sizeof(C), MAPPED, &smem);
  auto kern = k_stage1<S, C, MAPPED, KEEP>;
  allow_smem(kern);
  const int64_t grid = (m + T - 1) / T;
  pre_launch(ctx, nm);
  kern<<<unsigned(grid), T, smem, ctx.stream>>>(a, b, c, d, n, s, magic_for(s), m, blk, ra, rb, rc, rd, ka, kg,
                                                kd, MAPPED ? nullptr : ctx.flat_off, ctx.flat_nsys, ctx.status);
  post_launch(ctx, "stage 1");
}

template <typename C, typename S, bool MAPPED>
void stage3_kept(Ctx& ctx, const C* ka, const C* kg, const C* kd, int64_t n, int s, int64_t m, const int64_t* blk,
                 const double* y, S* x, const char* name = nullptr) {
  if (ctx.dry || ctx.err != cudaSuccess || m <= 0) return;
  size_t smem;
  const int T = pick_threads(ctx, s, 4, sizeof(C), MAPPED, &smem);  // same tiling as Stage 1
  const size_t need = size_t(2) * T * sizeof(C) + (MAPPED ? size_t(4) * T * s : 0);
  auto kern = k_stage3_kept<C, S, MAPPED>;
  allow_smem(kern);
  const int64_t kb = MAPPED ? 0 : ctx.kb, ke = (!MAPPED && ctx.ke >= 0) ? ctx.ke : m;
  pre_launch(ctx, name ? name : "stage3_kept_f64");
  kern<<<unsigned((ke - kb + T - 1) / T), T, need, ctx.stream>>>(ka, kg, kd, n, s, magic_for(s), m, blk, y, x, kb,
                                                                 ke);
  post_launch(ctx, "stage 3");
}

template <typename S, typename C, bool MAPPED>
void stage3_resolve(Ctx& ctx, const S* a, const S* b, const S* c, const S* d, int64_t n, int s, int64_t m,
                    const int64_t* blk, const double* y, S* x) {
  if (ctx.dry || ctx.err != cudaSuccess || m <= 0) return;
  if constexpr (!MAPPED && std::is_same<S, float>::value && std::is_same<C, float>::value) {
    if (ctx.vtile && ctx.vtile_l && s % 4 == 0) {
      const int64_t kb = ctx.kb, ke = ctx.ke >= 0 ? ctx.ke : m;
      size_t smem;
      const int T = ltile_threads(s, &smem);
      allow_smem(k_stage3_resolve_l);
      pre_launch(ctx, "stage3_resolve_f32");
      k_stage3_resolve_l<<<unsigned((ke - kb + T - 1) / T), T, smem, ctx.stream>>>(
          a, b, c, d, n, s, m, y, x, ctx.flat_off, ctx.flat_nsys, kb, ke, ctx.status);
      post_launch(ctx, "stage 3");
      return;
    }
  }
  if (!MAPPED && ctx.vtile && std::is_same<S, C>::value && s % Vec<S>::W == 0) {
    size_t smem;
    const int T = pick_threads(ctx, s, 4, sizeof(S), false, &smem, sizeof(S) == 4 ? 64 * 1024 : 0);
    auto vk = k_stage3_resolve_v<S, C>;
    allow_smem(vk);
    const int64_t kb = ctx.kb, ke = ctx.ke >= 0 ? ctx.ke : m;
    pre_launch(ctx, tname<C>("stage3_resolve_f64", "stage3_resolve_f32"));
    vk<<<unsigned((ke - kb + T - 1) / T), T, smem, ctx.stream>>>(a, b, c, d, n, s, m, y, x, ctx.flat_off,
                                                                 ctx.flat_nsys, kb, ke, ctx.status);
    post_launch(ctx, "stage 3");
    return;
  }
  size_t smem;
  const int T = pick_threads(ctx, s, 4, sizeof(C), MAPPED, &smem);
  auto kern = k_stage3_resolve<S, C, MAPPED>;
  allow_smem(kern);
  const int64_t grid = (m + T - 1) / T;
  pre_launch(ctx, tname<C>("stage3_resolve_f64", "stage3_resolve_f32"));
  kern<<<unsigned(grid), T, smem, ctx.stream>>>(a, b, c, d, n, s, magic_for(s), m, blk, y, x, ctx.status);
  post_launch(ctx, "stage 3");
}

// ---------------------------------------------------------------------------
// Stage 2: the interface system (M rows, binary64) is solved by applying the
// partition method to it again (the recursive variant, Sec. III) until it is
// small enough for one thread.
// ---------------------------------------------------------------------------
constexpr int64_t kCoopMax = int64_t(1) << 19;  // interface systems at most this large go to one launch

// Levels of the one-launch interface solve for a system of M rows (ra .. rd,
// solution y): workspace taken from ctx's arena, parameters in P (P.L = 0
// when M <= kBaseRows: no level, the system goes to one warp).
void coop_build(Ctx& ctx, const double* ra, const double* rb, const double* rc, const double* rd, double* y,
                int64_t M, CoopParams& P) {
  P = CoopParams{};
  int L = 0;
  const double *a = ra, *b = rb, *c = rc, *d = rd;
  double* yl = y;
  int64_t Ml = M;
  while (Ml > kBaseRows && L < kCoopMaxLevels) {
    CoopLevel& D = P.lv[L];
    D.s = ctx.s_tail;
    D.M = Ml;
    D.m = (Ml + D.s - 1) / D.s;
    D.a = a; D.b = b; D.c = c; D.d = d;
    D.ka = ctx.ar->take<double>(Ml);
    D.kg = ctx.ar->take<double>(Ml);
    D.kd = ctx.ar->take<double>(Ml);
    D.na = ctx.ar->take<double>(2 * D.m);
    D.nb = ctx.ar->take<double>(2 * D.m);
    D.nc = ctx.ar->take<double>(2 * D.m);
    D.nd = ctx.ar->take<double>(2 * D.m);
    D.y = yl;
    a = D.na; b = D.nb; c = D.nc; d = D.nd;
    Ml = 2 * D.m;
    ++L;
    if (Ml > kBaseRows && L < kCoopMaxLevels) yl = ctx.ar->take<double>(Ml);
  }
  P.L = L;
  P.reg = ctx.coop_reg ? 1 : 0;
  P.wait_cycles = 1ll << ctx.wait_log2;
  P.bar_extra = ctx.wait_never ? 1u : 0u;
  P.base_scratch = ctx.ar->take<double>(Ml);
  P.ybase = (L > 0) ? ctx.ar->take<double>(Ml) : y;
}

// Grid of a cooperative launch: co-resident CTAs of `threads` threads (at
// most max_per_sm per SM), at most `want`.
template <typename K>
int coop_grid(K kernel, int threads, int64_t want, int max_per_sm = 1 << 30) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> per_sm_of;
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(dev, reinterpret_cast<const void*>(kernel));
    auto it = per_sm_of.find(key);
    if (it == per_sm_of.end()) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess) per_sm = 0;
      per_sm_of[key] = per_sm;
    } else {
      per_sm = it->second;
    }
  }
  per_sm = std::min(per_sm, max_per_sm);
  return int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(std::max(per_sm, 1)) * sm_count())));
}

// All remaining recursion levels of an interface system of M rows in one
// cooperative launch (k_iface_coop).
void solve_interface_coop(Ctx& ctx, const double* ra, const double* rb, const double* rc, const double* rd,
                          double* y, int64_t M) {
  CoopParams P;
  coop_build(ctx, ra, rb, rc, rd, y, M, P);
  unsigned* bar = ctx.ar->take<unsigned>(2);
  if (ctx.dry || ctx.err != cudaSuccess) return;
  ctx.fail(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), ctx.stream), "barrier clear");
  const int grid = coop_grid(k_iface_coop, 128, (P.lv[0].m + 127) / 128);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = ctx.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  pre_launch(ctx, "iface_coop");
  ctx.fail(cudaLaunchKernelEx(&cfg, k_iface_coop, P, bar, ctx.status), "interface cooperative launch");
  post_launch(ctx, "interface cooperative launch");
}

// Sub-system size of recursive step `level` (1-based) of R under the paper's
// rule (Sec. III-B): the first step uses 10 when R >= 2, every other step the
// size model applied to the interface system it partitions.
int paper_level_size(int level, int R, int64_t M) {
  int m = (level == 1 && R >= 2) ? 10 : int(predict_s(M, 1, TDP_F64));
  return m < 3 ? 3 : m;
}

void solve_interface(Ctx& ctx, const double* ra, const double* rb, const double* rc, const double* rd, double* y,
                     int64_t M);

// The paper's recursive variant: R recursive steps, each a partition of the
// current interface system with its own sub-system size, then the last
// interface system solved directly on the device (one cooperative launch, or
// one thread when it has at most 64 rows).
void solve_interface_rec(Ctx& ctx, const double* ra, const double* rb, const double* rc, const double* rd,
                         double* y, int64_t M, int level, int R) {
  if (M <= 0) return;
  const int s2 = (level <= R && M > kBaseRows) ? paper_level_size(level, R, M) : 0;
  if (s2 == 0 || s2 >= M) {
    if (M <= kBaseRows) {
      if (ctx.dry || ctx.err != cudaSuccess) return;
      pre_launch(ctx, "interface_base");
      k_base_pcr<<<1, 32, 0, ctx.stream>>>(ra, rb, rc, rd, y, int(M), ctx.status);
      post_launch(ctx, "interface base solve");
    } else {
      solve_interface_coop(ctx, ra, rb, rc, rd, y, M);
    }
    return;
  }
  const int64_t m2 = (M + s2 - 1) / s2;
  double* ka = ctx.ar->take<double>(M);
  double* kg = ctx.ar->take<double>(M);
  double* kd = ctx.ar->take<double>(M);
  double* ra2 = ctx.ar->take<double>(2 * m2);
  double* rb2 = ctx.ar->take<double>(2 * m2);
  double* rc2 = ctx.ar->take<double>(2 * m2);
  double* rd2 = ctx.ar->take<double>(2 * m2);
  double* y2 = ctx.ar->take<double>(2 * m2);
  stage1<double, double, false, true>(ctx, ra, rb, rc, rd, M, s2, m2, nullptr, ra2, rb2, rc2, rd2, ka, kg, kd,
                                      "iface_stage1_f64");
  solve_interface_rec(ctx, ra2, rb2, rc2, rd2, y2, 2 * m2, level + 1, R);
  stage3_kept<double, double, false>(ctx, ka, kg, kd, M, s2, m2, nullptr, y2, y, "iface_stage3_f64");
}

void solve_interface_levels(Ctx& ctx, const double* ra, const double* rb, const double* rc, const double* rd,
                            double* y, int64_t M);

// One CTA per system when the interface system is a batch's concatenation of
// small decoupled systems (k_iface_seg).
bool solve_interface_seg(Ctx& ctx, const double* ra, const double* rb, const double* rc, const double* rd, double* y,
                         int64_t M) {
  if (!ctx.seg || ctx.seg_batch < 32 || M / ctx.seg_batch > 512 || ctx.rec_mode == 1) return false;
  double* ka = ctx.ar->take<double>(M);
  double* kg = ctx.ar->take<double>(M);
  double* kd = ctx.ar->take<double>(M);
  if (ctx.dry || ctx.err != cudaSuccess) return true;
  pre_launch(ctx, "iface_seg");
  k_iface_seg<<<unsigned(std::min<int64_t>(ctx.seg_batch, 1 << 20)), kSegT, 0, ctx.stream>>>(
      ra, rb, rc, rd, y, ctx.seg_bbase, ctx.seg_per, ctx.seg_batch, ka, kg, kd, ctx.status);
  post_launch(ctx, "segmented interface solve");
  return true;
}

void solve_interface(Ctx& ctx, const double* ra, const double* rb, const double* rc, const double* rd, double* y,
                     int64_t M) {
  if (M <= 0) return;
  // the interface system has no system boundaries to cut and is solved whole
  const int64_t* flat_off = ctx.flat_off;
  const int32_t flat_nsys = ctx.flat_nsys;
  const int64_t kb = ctx.kb, ke = ctx.ke;
  ctx.flat_off = nullptr;
  ctx.flat_nsys = 0;
  ctx.kb = 0;
  ctx.ke = -1;
  if (!solve_interface_seg(ctx, ra, rb, rc, rd, y, M)) solve_interface_levels(ctx, ra, rb, rc, rd, y, M);
  ctx.flat_off = flat_off;
  ctx.flat_nsys = flat_nsys;
  ctx.kb = kb;
  ctx.ke = ke;
}

void solve_interface_levels(Ctx& ctx, const double* ra, const double* rb, const double* rc, const double* rd,
                            double* y, int64_t M) {
  if (M <= 0) return;
  if (ctx.rec_mode == 1) {
    const int R = ctx.rec_force >= 0 ? ctx.rec_force : int(predict_r(ctx.rec_n, ctx.rec_batch, ctx.rec_dt));
    solve_interface_rec(ctx, ra, rb, rc, rd, y, M, 1, R);
    return;
  }
  if (ctx.coop && M > kBaseRows && M <= kCoopMax) {
    solve_interface_coop(ctx, ra, rb, rc, rd, y, M);
    return;
  }
  if (M <= kBaseRows) {
    if (ctx.dry || ctx.err != cudaSuccess) return;
    pre_launch(ctx, "interface_base");
    k_base_pcr<<<1, 32, 0, ctx.stream>>>(ra, rb, rc, rd, y, int(M), ctx.status);
    post_launch(ctx, "interface base solve");
    return;
  }
  const int s2 = ctx.s_rec;
  const int64_t m2 = (M + s2 - 1) / s2;
  double* ra2 = ctx.ar->take<double>(2 * m2);
  double* rb2 = ctx.ar->take<double>(2 * m2);
  double* rc2 = ctx.ar->take<double>(2 * m2);
  double* rd2 = ctx.ar->take<double>(2 * m2);
  double* y2 = ctx.ar->take<double>(2 * m2);
  if (ctx.iface32_on) {
    // A binary32 solve reads its interface values as binary32: the first
    // level (the largest by a factor s_rec) runs in binary32 arithmetic on
    // the binary64 rows, the deeper levels in binary64.  (Sending the next
    // interface system straight to the one-launch tail with a larger s was
    // slower: that tail's cost grows with its first level's size.)
    float* ka = ctx.ar->take<float>(M);
    float* kg = ctx.ar->take<float>(M);
    float* kd = ctx.ar->take<float>(M);
    stage1<double, float, false, true>(ctx, ra, rb, rc, rd, M, s2, m2, nullptr, ra2, rb2, rc2, rd2, ka, kg, kd,
                                       "iface_stage1_f32");
    ctx.iface32_on = false;
    solve_interface_levels(ctx, ra2, rb2, rc2, rd2, y2, 2 * m2);
    ctx.iface32_on = true;
    stage3_kept<float, double, false>(ctx, ka, kg, kd, M, s2, m2, nullptr, y2, y, "iface_stage3_f32");
    return;
  }
  double* ka = ctx.ar->take<double>(M);
  double* kg = ctx.ar->take<double>(M);
  double* kd = ctx.ar->take<double>(M);
  stage1<double, double, false, true>(ctx, ra, rb, rc, rd, M, s2, m2, nullptr, ra2, rb2, rc2, rd2, ka, kg, kd,
                                      "iface_stage1_f64");
  solve_interface_levels(ctx, ra2, rb2, rc2, rd2, y2, 2 * m2);
  stage3_kept<double, double, false>(ctx, ka, kg, kd, M, s2, m2, nullptr, y2, y, "iface_stage3_f64");
}

// While alive, the interface solves of ctx belong to a binary32 solve.
struct Iface32Scope {
  Ctx& c;
  bool old;
  Iface32Scope(Ctx& ctx, bool on) : c(ctx), old(ctx.iface32_on) { c.iface32_on = on && ctx.iface32; }
  ~Iface32Scope() { c.iface32_on = old; }
};

// ---------------------------------------------------------------------------
// Helper kernels: block map, residual, update, transposition, gradients.
// ---------------------------------------------------------------------------

// bbase[j] = number of blocks before system j (exclusive scan of
// ceil(N_j / s)); bbase[batch] = total.  Invalid offsets (offsets[0] != 0,
// decreasing, or offsets[batch] != total_n) make every count zero and raise
// ST_BADARG, so that no later kernel touches a row.
__global__ void __launch_bounds__(1024) k_block_scan(const int64_t* __restrict__ off, int32_t batch, int s,
                                                     const int32_t* __restrict__ sj, int64_t total_n,
                                                     int64_t* __restrict__ bbase, unsigned* __restrict__ status) {
  __shared__ int64_t warp_sums[32];
  __shared__ int bad;
  __shared__ int64_t carry;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) {
    bad = (off[0] != 0 || off[batch] != total_n) ? 1 : 0;
    carry = 0;
  }
  __syncthreads();
  for (int64_t j = tid; j < batch; j += blockDim.x)
    if (off[j + 1] < off[j]) bad = 1;
  __syncthreads();
  if (bad) {
    for (int64_t j = tid; j <= batch; j += blockDim.x) bbase[j] = 0;
    if (tid == 0) flag(status, ST_BADARG);
    return;
  }
  for (int64_t j0 = 0; j0 < batch; j0 += blockDim.x) {
    const int64_t j = j0 + tid;
    const int64_t len = (j < batch) ? off[j + 1] - off[j] : 0;
    const int sz = (sj && j < batch) ? sj[j] : s;
    int64_t v = (len + sz - 1) / sz;
    // inclusive warp scan
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane == 31) warp_sums[wid] = v;
    __syncthreads();
    if (wid == 0) {
      int64_t w = (lane < int(blockDim.x >> 5)) ? warp_sums[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += u;
      }
      warp_sums[lane] = w;
    }
    __syncthreads();
    const int64_t incl = v + (wid > 0 ? warp_sums[wid - 1] : 0) + carry;
    const int64_t excl = incl - ((j < batch) ? (off[j + 1] - off[j] + sz - 1) / sz : 0);
    if (j < batch) bbase[j] = excl;
    __syncthreads();
    if (tid == int(blockDim.x) - 1) carry = incl;
    __syncthreads();
  }
  if (tid == 0) bbase[batch] = carry;
}

// ---------------------------------------------------------------------------
// Size model inference on the device (Sec. II-E): for every system j, the
// label of the nearest table row in (log2 N_j, log2 batch), ties to the
// larger s.  The table travels as a kernel parameter.
// ---------------------------------------------------------------------------
constexpr int kKpMax = 256;
struct KpTable {
  int rows;
  double f[2 * kKpMax];
  int32_t lab[kKpMax];
};

// log2 of a positive value as its binary exponent plus log2 of its
// mantissa: exact for powers of two (as the host's features are), so that
// equal distances, and with them the tie rule, come out as on the host.
__device__ __forceinline__ double log2_split(double v) {
  int e;
  const double m = frexp(v, &e);  // v = m 2^e, m in [0.5, 1)
  return double(e - 1) + log2(2.0 * m);
}

__global__ void k_predict_sizes(const int64_t* __restrict__ off, int32_t batch, const __grid_constant__ KpTable tab,
                                int fallback, int clamp, int32_t* __restrict__ s_out) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= batch) return;
  int64_t n = off[j + 1] - off[j];
  if (n < 1) n = 1;
  const double ln = log2_split(double(n)), lb = log2_split(double(batch));
  double best = 1e300;
  int s = 0;
  for (int r = 0; r < tab.rows; ++r) {
    const double dn = tab.f[2 * r] - ln, db = tab.f[2 * r + 1] - lb;
    const double dist = dn * dn + db * db;
    if (dist < best || (dist == best && tab.lab[r] > s)) {
      best = dist;
      s = tab.lab[r];
    }
  }
  if (tab.rows == 0) {  // no table: the paper's interval rule (Sec. II-D)
    s = n <= 4500 ? 4 : n <= 25000 ? 8 : n <= 50000 ? 16 : n <= 75000 ? 20 : n <= 10000000 ? 32 : 64;
  }
  s = s >= 2 ? s : fallback;
  s_out[j] = s < clamp ? s : clamp;  // the tiles are sized for clamp rows per block
}

// blk[k] for k < m_max: start row of block k with flags; dummy blocks (after
// the last real one) start at total_n and are empty.  blk[m_max] = total_n.
__global__ void k_block_fill(const int64_t* __restrict__ off, int32_t batch, int s, const int32_t* __restrict__ sj,
                             int64_t total_n, const int64_t* __restrict__ bbase, int64_t m_max,
                             int64_t* __restrict__ blk) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k > m_max) return;
  if (k == m_max || k >= bbase[batch]) {
    blk[k] = total_n;
    return;
  }
  // system j with bbase[j] <= k < bbase[j+1]
  int32_t lo = 0, hi = batch - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (bbase[mid] <= k) lo = mid; else hi = mid - 1;
  }
  const int64_t i = k - bbase[lo];
  const int64_t cnt = bbase[lo + 1] - bbase[lo];
  int64_t e = off[lo] + i * (sj ? sj[lo] : s);
  if (i == 0) e |= BLK_FIRST;
  if (i == cnt - 1) e |= BLK_LAST;
  blk[k] = e;
}

// r = d - A x in binary64 for a batch described by blk (system ends from the
// block flags); x of a neighbouring system is never read.
template <bool MAPPED>
__global__ void k_residual(const double* __restrict__ a, const double* __restrict__ b, const double* __restrict__ c,
                           const double* __restrict__ d, const double* __restrict__ x, double* __restrict__ r,
                           int64_t n, const uint8_t* __restrict__ edge) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const uint8_t e = MAPPED ? edge[i] : uint8_t((i == 0 ? 1 : 0) | (i == n - 1 ? 2 : 0));
    double acc = fma(-b[i], x[i], d[i]);
    if (!(e & 1) && i > 0) acc = fma(-a[i], x[i - 1], acc);
    if (!(e & 2) && i < n - 1) acc = fma(-c[i], x[i + 1], acc);
    r[i] = acc;
  }
}

__global__ void k_add(double* __restrict__ x, const double* __restrict__ dx, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] += dx[i];
}

// edge[i]: bit 0 = first row of its system, bit 1 = last row.
__global__ void k_edges(const int64_t* __restrict__ off, int32_t batch, uint8_t* __restrict__ edge,
                        int64_t total_n) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= batch) return;
  const int64_t s0 = off[j], s1 = off[j + 1];
  if (s1 <= s0 || s0 < 0 || s1 > total_n) return;
  edge[s0] |= 1;
  edge[s1 - 1] |= 2;
}

// Transposed diagonals: aT[i] = c[i-1], cT[i] = a[i+1] within each system.
template <typename S>
__global__ void k_transpose(const S* __restrict__ a, const S* __restrict__ c, S* __restrict__ aT,
                            S* __restrict__ cT, int64_t n, const uint8_t* __restrict__ edge) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const uint8_t e = edge ? edge[i] : uint8_t(0);
    aT[i] = ((e & 1) || i == 0) ? S(0) : c[i - 1];
    cT[i] = ((e & 2) || i == n - 1) ? S(0) : a[i + 1];
  }
}

// grad_a = -lam x[i-1], grad_b = -lam x, grad_c = -lam x[i+1] (zero at system ends).
template <typename S>
__global__ void k_grads(const S* __restrict__ lam, const S* __restrict__ x, S* __restrict__ ga, S* __restrict__ gb,
                        S* __restrict__ gc, int64_t n, const uint8_t* __restrict__ edge) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const uint8_t e = edge ? edge[i] : uint8_t(0);
    const S l = lam[i];
    if (ga) ga[i] = ((e & 1) || i == 0) ? S(0) : -l * x[i - 1];
    if (gb) gb[i] = -l * x[i];
    if (gc) gc[i] = ((e & 2) || i == n - 1) ? S(0) : -l * x[i + 1];
  }
}

// The same gradients with no edge array (edge == null): every row takes its
// neighbours; k_grad_cuts then zeroes grad_a of every system's first row and
// grad_c of its last row.
template <typename S>
__global__ void k_grad_cuts(const int64_t* __restrict__ off, int32_t batch, int64_t n, S* __restrict__ ga,
                            S* __restrict__ gc) {
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < batch; j += int64_t(gridDim.x) * blockDim.x) {
    const int64_t lo = off[j], hi = off[j + 1];
    if (hi > lo && lo >= 0 && hi <= n) {  // (offsets out of range touch nothing; the offsets check reports them)
      if (ga) ga[lo] = S(0);
      if (gc) gc[hi - 1] = S(0);
    }
  }
}

// Uniform offsets j * n for strided batches copied to contiguous storage.
__global__ void k_iota_offsets(int64_t* __restrict__ off, int32_t batch, int64_t n) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j <= batch) off[j] = j * n;
}

template <typename S>
__global__ void k_gather(const S* __restrict__ src, S* __restrict__ dst, int32_t batch, int64_t n, int64_t ss,
                         int64_t es) {
  const int64_t total = int64_t(batch) * n;
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < total; q += int64_t(gridDim.x) * blockDim.x) {
    const int64_t j = q / n, i = q - j * n;
    dst[q] = src[j * ss + i * es];
  }
}

template <typename S>
__global__ void k_scatter(const S* __restrict__ src, S* __restrict__ dst, int32_t batch, int64_t n, int64_t ss,
                          int64_t es) {
  const int64_t total = int64_t(batch) * n;
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < total; q += int64_t(gridDim.x) * blockDim.x) {
    const int64_t j = q / n, i = q - j * n;
    dst[j * ss + i * es] = src[q];
  }
}

// The same for the interleaved layout (sys_stride 1: element i of system j at
// j + i es, the column sweep of an ADI step), where reading along a system
// strides by es: a 32 x 32 tile of (system, element) passes through shared
// memory, read along the systems and written along the elements (and the
// reverse for the scatter), so that both sides are coalesced; up to four
// arrays per launch.
template <typename S>
struct Strided4 {
  const S* src[4];
  S* dst[4];
  int na;
};

template <typename S>
__global__ void __launch_bounds__(256) k_gather_t(const __grid_constant__ Strided4<S> G, int32_t batch, int64_t n,
                                                  int64_t es) {
  __shared__ S tile[32][33];
  const int64_t j0 = int64_t(blockIdx.x) * 32, i0 = int64_t(blockIdx.y) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int k = 0; k < G.na; ++k) {
#pragma unroll
    for (int r = 0; r < 32; r += 8) {  // read along the systems
      const int64_t j = j0 + tx, i = i0 + ty + r;
      if (j < batch && i < n) tile[ty + r][tx] = G.src[k][j + i * es];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 32; r += 8) {  // write along the elements
      const int64_t j = j0 + ty + r, i = i0 + tx;
      if (j < batch && i < n) G.dst[k][j * n + i] = tile[tx][ty + r];
    }
    __syncthreads();
  }
}

template <typename S>
__global__ void __launch_bounds__(256) k_scatter_t(const S* __restrict__ src, S* __restrict__ dst, int32_t batch,
                                                   int64_t n, int64_t es) {
  __shared__ S tile[32][33];
  const int64_t j0 = int64_t(blockIdx.x) * 32, i0 = int64_t(blockIdx.y) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < 32; r += 8) {  // read along the elements
    const int64_t j = j0 + ty + r, i = i0 + tx;
    if (j < batch && i < n) tile[ty + r][tx] = src[j * n + i];
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 32; r += 8) {  // write along the systems
    const int64_t j = j0 + tx, i = i0 + ty + r;
    if (j < batch && i < n) dst[j + i * es] = tile[tx][ty + r];
  }
}

unsigned grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return unsigned(std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16)));
}

// Offsets of a batch solved as one system: offsets[0] = 0, non-decreasing,
// offsets[batch] = total_n; anything else raises ST_BADARG.
__global__ void k_check_offsets(const int64_t* __restrict__ off, int32_t batch, int64_t total_n,
                                unsigned* __restrict__ status) {
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j <= batch;
       j += int64_t(gridDim.x) * blockDim.x) {
    const int64_t v = off[j];
    if ((j == 0 && v != 0) || (j == batch && v != total_n) || (j > 0 && off[j - 1] > v)) flag(status, ST_BADARG);
  }
}

// ---------------------------------------------------------------------------
// Binary32 solve with binary64 refinement in one windowed pass
// (tdp_window.cuh), followed by the exact binary64 solve of the whole system
// in one cooperative launch that runs only when a tile failed its checks.
// off: a batch solved as one system (nsys systems), null for one system.
// The pass is planned once (scratch, gate word, the fallback's parameters)
// and may be launched over consecutive ranges of tiles (the host-array solve
// launches each range once its rows have been copied in).
// ---------------------------------------------------------------------------
template <typename S>
struct WindowPlan {
  WinParams<S> W;
  ExactParams<S> E;
  CoopParams P;
  unsigned* gate;
  int SW;
  bool trans;  // A^T x = d (the transposed windows, k_window<..., true>)
  int64_t tiles;
  bool live;  // scratch taken, gate cleared: launches may follow
};

template <typename S>
WindowPlan<S> window_plan(Ctx& ctx, const S* a, const S* b, const S* c, const S* d, S* x, int64_t n, int iters,
                          const int64_t* off, int32_t nsys, bool trans = false) {
  constexpr bool REFINE = sizeof(S) == 8;
  WindowPlan<S> Q;
  Q.trans = trans;
  // (binary32 storage asks the window for 2^-30 instead of 2^-46: a third
  // fewer halo rows give the same decay per row)
  const int H = std::max(16, std::min(REFINE ? ctx.window_halo : ctx.window_halo32, 64)) & ~3;
  // window rows per thread: 5 or 7 for the refinement; for binary32 the
  // largest odd count up to the knob (5 to 13) that still gives every SM
  // three tiles (longer windows amortise the halo and the per-thread work,
  // but a short system needs the CTAs), else 5
  if (REFINE) {
    Q.SW = ctx.window_sw == 5 ? 5 : 7;
  } else {
    const int top = std::max(5, std::min(ctx.window_sw32, 13)) | 1;
    Q.SW = 5;
    for (int sw = top; sw > 5; sw -= 2)
      if ((n + kWinT * sw - 2 * H - 1) / (kWinT * sw - 2 * H) >= 3 * int64_t(sm_count())) {
        Q.SW = sw;
        break;
      }
  }
  const int TR = kWinT * Q.SW - 2 * H;
  Q.tiles = (n + TR - 1) / TR;
  Q.gate = ctx.ar->take<unsigned>(4);  // the gate word, then the fallback's grid barrier
  const int64_t m0 = (n + kExS - 1) / kExS;
  Q.E = ExactParams<S>{a, b, c, d, x, n, m0, off, nsys, nullptr, nullptr, nullptr, nullptr, nullptr, Q.trans};
  Q.E.ra = ctx.ar->take<double>(2 * m0);
  Q.E.rb = ctx.ar->take<double>(2 * m0);
  Q.E.rc = ctx.ar->take<double>(2 * m0);
  Q.E.rd = ctx.ar->take<double>(2 * m0);
  Q.E.y0 = ctx.ar->take<double>(2 * m0);
  coop_build(ctx, Q.E.ra, Q.E.rb, Q.E.rc, Q.E.rd, Q.E.y0, 2 * m0, Q.P);
  // binary64 storage: the windowed solution within 2^-45 ||x|| (the refinement
  // goes below binary32 rounding); binary32 storage: within 2^-30 ||x||
  const float tau = REFINE ? kWinTau : 1.0f / 2147483648.0f;
  Q.W = WinParams<S>{a, b, c, d, x, n, H, TR, REFINE ? iters : 0, tau, off, nsys, Q.gate, ctx.status,
                     1ll << ctx.wait_log2, ctx.window_prefetch, 0};
  Q.live = !ctx.dry && ctx.err == cudaSuccess;
  if (!Q.live) return Q;
  // (a batch's offsets are checked by the gated fallback, launched after the pass)
  ctx.fail(cudaMemsetAsync(Q.gate, 0, 3 * sizeof(unsigned), ctx.stream), "gate clear");
  Q.live = ctx.err == cudaSuccess;
  return Q;
}

// Tiles [t0, t1) of a planned pass.
template <typename S>
void window_launch(Ctx& ctx, WindowPlan<S>& Q, int64_t t0, int64_t t1) {
  constexpr bool REFINE = sizeof(S) == 8;
  if (!Q.live || ctx.err != cudaSuccess || t1 <= t0) return;
  Q.W.tile0 = t0;
  void (*wk)(WinParams<S>) = k_window<S, 5, REFINE ? 3 : 4>;
  size_t smem = WinSmem<S, 5>::bytes();
  if (Q.SW == 7) {
    wk = k_window<S, 7, 3>;
    smem = WinSmem<S, 7>::bytes();
  }
  if constexpr (REFINE) {
    if (Q.trans) {
      wk = Q.SW == 7 ? k_window<S, 7, 3, true> : k_window<S, 5, 3, true>;
      smem = Q.SW == 7 ? WinSmem<S, 7, true>::bytes() : WinSmem<S, 5, true>::bytes();
    }
  }
  if constexpr (!REFINE) {  // three CTAs per SM up to 13 rows per thread
    if (Q.SW == 9) {
      wk = k_window<S, 9, 3>;
      smem = WinSmem<S, 9>::bytes();
    } else if (Q.SW == 11) {
      wk = k_window<S, 11, 3>;
      smem = WinSmem<S, 11>::bytes();
    } else if (Q.SW == 13) {
      wk = k_window<S, 13, 3>;
      smem = WinSmem<S, 13>::bytes();
    }
    if (Q.trans) {  // the same geometry on transposed windows
      switch (Q.SW) {
        case 7: wk = k_window<S, 7, 3, true>; smem = WinSmem<S, 7, true>::bytes(); break;
        case 9: wk = k_window<S, 9, 3, true>; smem = WinSmem<S, 9, true>::bytes(); break;
        case 11: wk = k_window<S, 11, 3, true>; smem = WinSmem<S, 11, true>::bytes(); break;
        case 13: wk = k_window<S, 13, 3, true>; smem = WinSmem<S, 13, true>::bytes(); break;
        default: wk = k_window<S, 5, 4, true>; smem = WinSmem<S, 5, true>::bytes(); break;
      }
    }
  }
  allow_smem(wk);
  pre_launch(ctx, REFINE ? "window_refine" : "window_f32");
  wk<<<unsigned(t1 - t0), kWinT, smem, ctx.stream>>>(Q.W);
  post_launch(ctx, "windowed pass");
}

// The gated exact solve after every tile has run; it writes x through xout
// (the device array of the pass, or a device-visible alias of the caller's
// host array).
template <typename S>
void window_fallback(Ctx& ctx, WindowPlan<S>& Q, S* xout) {
  if (!Q.live || ctx.err != cudaSuccess) return;
  Q.E.x = xout;
  // two CTAs per SM: the launch costs little when the gate is clear (every CTA
  // returns at once), and the grid-stride loops cover any size when it is set
  auto ek = k_exact_coop<S>;
  const int grid = coop_grid(ek, 128, (std::max(Q.E.m0, Q.P.L > 0 ? Q.P.lv[0].m : int64_t(1)) + 127) / 128, 2);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = ctx.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  pre_launch(ctx, "exact_fallback");
  ctx.fail(cudaLaunchKernelEx(&cfg, ek, Q.E, Q.P, (const unsigned*)Q.gate, Q.gate + 1, ctx.status),
           "exact fallback launch");
  post_launch(ctx, "exact fallback");
}

template <typename S>
void window_pass(Ctx& ctx, const S* a, const S* b, const S* c, const S* d, S* x, int64_t n, int iters,
                 const int64_t* off, int32_t nsys, bool trans = false) {
  WindowPlan<S> Q = window_plan(ctx, a, b, c, d, x, n, iters, off, nsys, trans);
  window_launch(ctx, Q, 0, Q.tiles);
  window_fallback(ctx, Q, x);
}

// The exact refinement schedules (the windowed pass switched off, or the
// recursion schedule) narrow d and the residuals to binary32 without a scale.
// A system outside the scales they carry, a nonzero |d| outside [2^-70, 2^70]
// or |b| outside [2^-30, 2^30] (then |x| and the corrections stay inside the
// binary32 normal range), sets the gate of the exact binary64 solve that runs
// after them.  (The windowed pass scales each window instead.)
__global__ void k_refine_range(const double* __restrict__ b, const double* __restrict__ d, int64_t n,
                               unsigned* gate, unsigned* status) {
  bool out = false;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const unsigned hd = unsigned(__double2hiint(d[i])) & 0x7fffffffu, ld = unsigned(__double2loint(d[i]));
    const unsigned hb = unsigned(__double2hiint(b[i])) & 0x7fffffffu;
    out |= ((hd | ld) != 0u && (hd < (953u << 20) || hd >= (1093u << 20))) || hb < (993u << 20) ||
           hb >= (1053u << 20);
  }
  if (__syncthreads_or(out) && threadIdx.x == 0) {
    atomicOr(gate, 1u);
    flag(status, ST_FALLBACK);
  }
}

struct RefineGuard {
  Ctx& ctx;
  WindowPlan<double> Q;
  double* x;
  RefineGuard(Ctx& c, const void* a, const void* b, const void* cc, const void* d, void* x_, int64_t n,
              const int64_t* off, int32_t nsys)
      : ctx(c), x((double*)x_) {
    Q = window_plan(ctx, (const double*)a, (const double*)b, (const double*)cc, (const double*)d, x, n, 0, off,
                    nsys);
    if (!Q.live) return;
    pre_launch(ctx, "refine_range");
    k_refine_range<<<unsigned(std::min<int64_t>(grid_for(n, 256), 8 * sm_count())), 256, 0, ctx.stream>>>(
        (const double*)b, (const double*)d, n, Q.gate, ctx.status);
    post_launch(ctx, "refinement range check");
  }
  void finish() { window_fallback(ctx, Q, x); }
};

// Host arrays through the windowed pass.  The rows are copied in by chunks of
// whole tiles on one stream; each chunk's tiles run as soon as the chunk has
// landed (the tile that needs the next chunk's first halo rows runs with the
// next chunk), and their x goes out on a second stream while later chunks are
// copied in and solved.  The gated exact solve, when a tile failed, writes x
// straight into the caller's array after every chunk has been copied out, so
// the array must be visible to the device (pinned or registered memory);
// otherwise everything is copied in, solved and copied out.
template <typename S>
void window_host(Ctx& ctx, const S* a, const S* b, const S* c, const S* d, S* x, int64_t n, int iters, S* ad,
                 S* bd, S* cd, S* dd, S* xd) {
  WindowPlan<S> Q = window_plan(ctx, (const S*)ad, (const S*)bd, (const S*)cd, (const S*)dd, xd, n, iters,
                                (const int64_t*)nullptr, 0);
  if (!Q.live) return;
  const S* hsrc[4] = {a, b, c, d};
  S* dsrc[4] = {ad, bd, cd, dd};
  S* xdev = nullptr;  // the caller's x as the device sees it
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, x) == cudaSuccess) {
    if (pa.type == cudaMemoryTypeHost && pa.devicePointer) xdev = static_cast<S*>(pa.devicePointer);
  } else {
    cudaGetLastError();  // (not a CUDA pointer at all: clear the error it leaves)
  }
  if (!xdev) {
    for (int i = 0; i < 4 && ctx.err == cudaSuccess; ++i)
      ctx.fail(cudaMemcpyAsync(dsrc[i], hsrc[i], size_t(n) * sizeof(S), cudaMemcpyHostToDevice, ctx.stream),
               "copy in");
    window_launch(ctx, Q, 0, Q.tiles);
    window_fallback(ctx, Q, xd);
    if (ctx.err == cudaSuccess)
      ctx.fail(cudaMemcpyAsync(x, xd, size_t(n) * sizeof(S), cudaMemcpyDeviceToHost, ctx.stream), "copy out");
    return;
  }
  const int64_t TR = Q.W.TR, H = Q.W.H;
  const int64_t ct = std::max<int64_t>(64, (Q.tiles + 15) / 16);  // tiles per chunk: about 16 chunks
  const int64_t C = ct * TR;
  const int64_t nch = (n + C - 1) / C;
  cudaStream_t cin = nullptr, cout = nullptr;
  std::vector<cudaEvent_t> evs;
  auto event = [&]() {
    cudaEvent_t e = nullptr;
    ctx.fail(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    if (e) evs.push_back(e);
    return e;
  };
  ctx.fail(cudaStreamCreateWithFlags(&cin, cudaStreamNonBlocking), "copy stream");
  ctx.fail(cudaStreamCreateWithFlags(&cout, cudaStreamNonBlocking), "copy stream");
  if (ctx.err == cudaSuccess) {  // the copies start after the caller's earlier work
    cudaEvent_t go = event();
    if (ctx.err == cudaSuccess) ctx.fail(cudaEventRecord(go, ctx.stream), "event");
    if (ctx.err == cudaSuccess) ctx.fail(cudaStreamWaitEvent(cin, go, 0), "event");
    if (ctx.err == cudaSuccess) ctx.fail(cudaStreamWaitEvent(cout, go, 0), "event");
  }
  int64_t tdone = 0;
  for (int64_t k = 0; k < nch && ctx.err == cudaSuccess; ++k) {
    const int64_t r0 = k * C, r1 = std::min(n, r0 + C);
    for (int i = 0; i < 4 && ctx.err == cudaSuccess; ++i)
      ctx.fail(cudaMemcpyAsync(dsrc[i] + r0, hsrc[i] + r0, size_t(r1 - r0) * sizeof(S), cudaMemcpyHostToDevice,
                               cin), "copy in");
    cudaEvent_t ready = event();
    if (ctx.err == cudaSuccess) ctx.fail(cudaEventRecord(ready, cin), "event");
    if (ctx.err == cudaSuccess) ctx.fail(cudaStreamWaitEvent(ctx.stream, ready, 0), "event");
    // tile t needs rows up to (t + 1) TR + H
    const int64_t t1 = k == nch - 1 ? Q.tiles : std::max(tdone, (r1 - H) / TR);
    if (t1 <= tdone) continue;
    window_launch(ctx, Q, tdone, t1);
    cudaEvent_t done = event();
    if (ctx.err == cudaSuccess) ctx.fail(cudaEventRecord(done, ctx.stream), "event");
    if (ctx.err == cudaSuccess) ctx.fail(cudaStreamWaitEvent(cout, done, 0), "event");
    const int64_t x0 = tdone * TR, x1 = std::min(n, t1 * TR);
    if (ctx.err == cudaSuccess)
      ctx.fail(cudaMemcpyAsync(x + x0, xd + x0, size_t(x1 - x0) * sizeof(S), cudaMemcpyDeviceToHost, cout),
               "copy out");
    tdone = t1;
  }
  if (ctx.err == cudaSuccess) {  // every chunk of x is in place before the fallback may rewrite it
    cudaEvent_t fin = event();
    if (ctx.err == cudaSuccess) ctx.fail(cudaEventRecord(fin, cout), "event");
    if (ctx.err == cudaSuccess) ctx.fail(cudaStreamWaitEvent(ctx.stream, fin, 0), "event");
  }
  window_fallback(ctx, Q, xdev);
  if (cin) cudaStreamDestroy(cin);  // released once their work is done
  if (cout) cudaStreamDestroy(cout);
  for (cudaEvent_t e : evs) cudaEventDestroy(e);
}

// ---------------------------------------------------------------------------
// One solve over blocks given either arithmetically (one system) or by blk.
// ---------------------------------------------------------------------------
template <bool MAPPED>
void solve_blocks(Ctx& ctx, const void* a, const void* b, const void* c, const void* d, void* x, int64_t n, int s,
                  int64_t m, const int64_t* blk, const uint8_t* edge, tdp_dtype dt, int refine_iters) {
  Iface32Scope f32(ctx, dt != TDP_F64);
  double* ra = ctx.ar->take<double>(2 * m);
  double* rb = ctx.ar->take<double>(2 * m);
  double* rc = ctx.ar->take<double>(2 * m);
  double* rd = ctx.ar->take<double>(2 * m);
  double* y = ctx.ar->take<double>(2 * m);
  if (dt == TDP_F64) {
    using T = double;
    const T *A = (const T*)a, *B = (const T*)b, *Cc = (const T*)c, *D = (const T*)d;
    double* ka = ctx.ar->take<double>(n);
    double* kg = ctx.ar->take<double>(n);
    double* kd = ctx.ar->take<double>(n);
    stage1<T, T, MAPPED, true>(ctx, A, B, Cc, D, n, s, m, blk, ra, rb, rc, rd, ka, kg, kd);
    solve_interface(ctx, ra, rb, rc, rd, y, 2 * m);
    stage3_kept<T, T, MAPPED>(ctx, ka, kg, kd, n, s, m, blk, y, (T*)x);
  } else if (dt == TDP_F32) {
    using T = float;
    const T *A = (const T*)a, *B = (const T*)b, *Cc = (const T*)c, *D = (const T*)d;
    stage1<T, T, MAPPED, false>(ctx, A, B, Cc, D, n, s, m, blk, ra, rb, rc, rd, (T*)nullptr, (T*)nullptr,
                                (T*)nullptr);
    solve_interface(ctx, ra, rb, rc, rd, y, 2 * m);
    stage3_resolve<T, T, MAPPED>(ctx, A, B, Cc, D, n, s, m, blk, y, (T*)x);
  } else if (ctx.refine3 && refine_iters >= 1) {
    // three passes for the solve and its first correction (tdp_refine.cuh), then
    // separate kernels for any further correction
    const double *A = (const double*)a, *B = (const double*)b, *Cc = (const double*)c, *D = (const double*)d;
    double* X = (double*)x;
    const bool kept = ctx.refine_kept;
    float* rr = ctx.ar->take<float>(kept ? 1 : n);
    float* x0f = kept ? ctx.ar->take<float>(n) : nullptr;
    float* fka = kept ? ctx.ar->take<float>(n) : nullptr;
    float* fkg = kept ? ctx.ar->take<float>(n) : nullptr;
    float* fkd = kept ? ctx.ar->take<float>(n) : nullptr;
    double* r = ctx.ar->take<double>(refine_iters > 1 ? n : 1);
    double* dx = ctx.ar->take<double>(refine_iters > 1 ? n : 1);
    stage1<double, float, MAPPED, false>(ctx, A, B, Cc, D, n, s, m, blk, ra, rb, rc, rd, (float*)nullptr,
                                         (float*)nullptr, (float*)nullptr);
    solve_interface(ctx, ra, rb, rc, rd, y, 2 * m);
    if (!ctx.dry && ctx.err == cudaSuccess) {
      size_t smem;
      const int T = pick_threads(ctx, s, 5, 4, MAPPED, &smem);
      const int64_t* foff = MAPPED ? nullptr : ctx.flat_off;
      if (foff) smem += size_t(2) * T * s;  // row flags of a batch solved as one system
      auto kern = kept ? (foff ? k_refine_mid<MAPPED, true, !MAPPED> : k_refine_mid<MAPPED, true, false>)
                       : (foff ? k_refine_mid<MAPPED, false, !MAPPED> : k_refine_mid<MAPPED, false, false>);
      allow_smem(kern);
      pre_launch(ctx, "refine_mid");
      kern<<<unsigned((m + T - 1) / T), T, smem, ctx.stream>>>(A, B, Cc, D, X, rr, n, s, magic_for(s), m, blk, edge,
                                                               y, ra, rb, rc, rd, x0f, fka, fkg, fkd, foff,
                                                               ctx.flat_nsys, ctx.status);
      post_launch(ctx, "refine pass 2");
    }
    solve_interface(ctx, ra, rb, rc, rd, y, 2 * m);
    if (!ctx.dry && ctx.err == cudaSuccess && kept) {
      size_t smem;
      const int T = pick_threads(ctx, s, 4, 4, MAPPED, &smem);
      const size_t need = size_t(2) * T * sizeof(float) + (MAPPED ? size_t(4) * T * s : 0);
      auto kern = k_refine_kept<MAPPED>;
      allow_smem(kern);
      pre_launch(ctx, "refine_kept");
      kern<<<unsigned((m + T - 1) / T), T, need, ctx.stream>>>(fka, fkg, fkd, x0f, n, s, magic_for(s), m, blk, y, X);
      post_launch(ctx, "refine pass 3");
    } else if (!ctx.dry && ctx.err == cudaSuccess) {
      size_t smem;
      const int T = pick_threads(ctx, s, 4, 4, MAPPED, &smem);
      auto kern = k_refine_last<MAPPED>;
      allow_smem(kern);
      pre_launch(ctx, "refine_last");
      kern<<<unsigned((m + T - 1) / T), T, smem, ctx.stream>>>(A, B, Cc, rr, X, n, s, magic_for(s), m, blk, y,
                                                               ctx.status);
      post_launch(ctx, "refine pass 3");
    }
    for (int it = 1; it < refine_iters; ++it) {
      if (!ctx.dry && ctx.err == cudaSuccess) {
        pre_launch(ctx, "residual_f64");
        k_residual<MAPPED><<<grid_for(n, 256), 256, 0, ctx.stream>>>(A, B, Cc, D, X, r, n, edge);
        post_launch(ctx, "residual");
      }
      stage1<double, float, MAPPED, false>(ctx, A, B, Cc, r, n, s, m, blk, ra, rb, rc, rd, (float*)nullptr,
                                           (float*)nullptr, (float*)nullptr);
      solve_interface(ctx, ra, rb, rc, rd, y, 2 * m);
      stage3_resolve<double, float, MAPPED>(ctx, A, B, Cc, r, n, s, m, blk, y, dx);
      if (!ctx.dry && ctx.err == cudaSuccess) {
        pre_launch(ctx, "update_f64");
        k_add<<<grid_for(n, 256), 256, 0, ctx.stream>>>(X, dx, n);
        post_launch(ctx, "update");
      }
    }
  } else {
    // binary32 eliminations, binary64 residual and correction (separate kernels)
    const double *A = (const double*)a, *B = (const double*)b, *Cc = (const double*)c, *D = (const double*)d;
    double* X = (double*)x;
    double* r = ctx.ar->take<double>(refine_iters > 0 ? n : 1);
    double* dx = ctx.ar->take<double>(refine_iters > 0 ? n : 1);
    stage1<double, float, MAPPED, false>(ctx, A, B, Cc, D, n, s, m, blk, ra, rb, rc, rd, (float*)nullptr,
                                         (float*)nullptr, (float*)nullptr);
    solve_interface(ctx, ra, rb, rc, rd, y, 2 * m);
    stage3_resolve<double, float, MAPPED>(ctx, A, B, Cc, D, n, s, m, blk, y, X);
    for (int it = 0; it < refine_iters; ++it) {
      if (!ctx.dry && ctx.err == cudaSuccess) {
        pre_launch(ctx, "residual_f64");
        k_residual<MAPPED><<<grid_for(n, 256), 256, 0, ctx.stream>>>(A, B, Cc, D, X, r, n, edge);
        post_launch(ctx, "residual");
      }
      stage1<double, float, MAPPED, false>(ctx, A, B, Cc, r, n, s, m, blk, ra, rb, rc, rd, (float*)nullptr,
                                           (float*)nullptr, (float*)nullptr);
      solve_interface(ctx, ra, rb, rc, rd, y, 2 * m);
      stage3_resolve<double, float, MAPPED>(ctx, A, B, Cc, r, n, s, m, blk, y, dx);
      if (!ctx.dry && ctx.err == cudaSuccess) {
        pre_launch(ctx, "update_f64");
        k_add<<<grid_for(n, 256), 256, 0, ctx.stream>>>(X, dx, n);
        post_launch(ctx, "update");
      }
    }
  }
}

// While alive, the interface solves of ctx belong to a batch of `batch`
// systems (blocks before each in bbase, or per_sys blocks each).
struct SegScope {
  Ctx& c;
  SegScope(Ctx& ctx, const int64_t* bbase, int64_t per_sys, int32_t batch) : c(ctx) {
    c.seg_bbase = bbase;
    c.seg_per = per_sys;
    c.seg_batch = batch;
  }
  ~SegScope() {
    c.seg_bbase = nullptr;
    c.seg_per = 0;
    c.seg_batch = 0;
  }
};

struct BatchMap {
  const int64_t* blk = nullptr;
  const uint8_t* edge = nullptr;
  const int64_t* bbase = nullptr;  // blocks before each system
  int64_t m = 0;
};

// Per-system sizes: the device predictor writes s_j for every system (the
// table rows of dtype dt); returns false when that table is empty.
struct SizeModel {
  KpTable tab;
  int s_min = 0, s_max = 0;
};

bool size_model(tdp_dtype dt, int32_t batch, SizeModel* sm) {
  const double* feat = nullptr;
  const int32_t* lab = nullptr;
  const int rows = std::min(predictor_table(dt, &feat, &lab), kKpMax);
  if (rows <= 0) return false;
  sm->tab.rows = rows;
  sm->s_min = 1 << 30;
  sm->s_max = 0;
  // tiles are sized for the largest label among the rows of the nearest batch size
  const double lb = std::log2(double(std::max(1, batch)));
  double near = 1e300;
  for (int r = 0; r < rows; ++r) near = std::min(near, std::fabs(double(feat[2 * r + 1]) - lb));
  for (int r = 0; r < rows; ++r) {
    sm->tab.f[2 * r] = feat[2 * r];
    sm->tab.f[2 * r + 1] = feat[2 * r + 1];
    sm->tab.lab[r] = lab[r];
    sm->s_min = std::min(sm->s_min, int(lab[r]));
    if (std::fabs(double(feat[2 * r + 1]) - lb) <= near) sm->s_max = std::max(sm->s_max, int(lab[r]));
  }
  sm->s_min = std::min(sm->s_min, sm->s_max);
  return true;
}

BatchMap build_map(Ctx& ctx, const int64_t* offsets, int32_t batch, int64_t total_n, int s, bool need_edges,
                   const SizeModel* model = nullptr) {
  BatchMap bm;
  const int s_lo = model ? model->s_min : s;
  bm.m = (total_n + int64_t(batch) * (s_lo - 1)) / s_lo;
  int64_t* bbase = ctx.ar->take<int64_t>(batch + 1);
  int64_t* blk = ctx.ar->take<int64_t>(bm.m + 1);
  uint8_t* edge = need_edges ? ctx.ar->take<uint8_t>(total_n) : nullptr;
  int32_t* sj = model ? ctx.ar->take<int32_t>(batch) : nullptr;
  bm.blk = blk;
  bm.edge = edge;
  bm.bbase = bbase;
  if (ctx.dry || ctx.err != cudaSuccess) return bm;
  if (model) {
    pre_launch(ctx, "predict_sizes");
    k_predict_sizes<<<unsigned((batch + 127) / 128), 128, 0, ctx.stream>>>(offsets, batch, model->tab,
                                                                           model->s_max, model->s_max, sj);
    post_launch(ctx, "predict sizes");
  }
  pre_launch(ctx, "block_scan");
  k_block_scan<<<1, 1024, 0, ctx.stream>>>(offsets, batch, s, sj, total_n, bbase, ctx.status);
  post_launch(ctx, "block scan");
  pre_launch(ctx, "block_fill");
  k_block_fill<<<unsigned((bm.m + 1 + 255) / 256), 256, 0, ctx.stream>>>(offsets, batch, s, sj, total_n, bbase,
                                                                         bm.m, blk);
  post_launch(ctx, "block fill");
  if (need_edges && total_n > 0) {
    ctx.fail(cudaMemsetAsync(edge, 0, size_t(total_n), ctx.stream), "edge clear");
    pre_launch(ctx, "edges");
    k_edges<<<unsigned((batch + 255) / 256), 256, 0, ctx.stream>>>(offsets, batch, edge, total_n);
    post_launch(ctx, "edges");
  }
  return bm;
}

}  // namespace

// ---------------------------------------------------------------------------
// Public drivers
// ---------------------------------------------------------------------------
namespace {
// One constant-coefficient solve: table, Stage 1, interface, Stage 3.
template <typename S, typename C>
void const_pass(Ctx& ctx, double a, double b, double c, const S* d, S* x, int64_t n, int32_t batch, int64_t ss,
                int64_t es, int s) {
  const int64_t mps = (n + s - 1) / s;
  const int64_t m = int64_t(batch) * mps;
  C* tab = ctx.ar->take<C>(6 * size_t(s));
  double* ra = ctx.ar->take<double>(2 * m);
  double* rb = ctx.ar->take<double>(2 * m);
  double* rc = ctx.ar->take<double>(2 * m);
  double* rd = ctx.ar->take<double>(2 * m);
  double* y = ctx.ar->take<double>(2 * m);
  SegScope seg(ctx, nullptr, mps, batch);
  int T = 128;
  while (T > 32 && size_t(T) * s * sizeof(C) > size_t(kMaxSmem)) T -= 32;
  const size_t smem = size_t(T) * s * sizeof(C);
  const unsigned grid = unsigned((m + T - 1) / T);
  if (!ctx.dry && ctx.err == cudaSuccess) {
    if (smem > size_t(kMaxSmem)) {
      ctx.fail(cudaErrorInvalidConfiguration, "constant-coefficient tile");
      return;
    }
    pre_launch(ctx, "const_table");
    k_const_table<C><<<1, 32, 0, ctx.stream>>>(a, b, c, s, tab, ctx.status);
    post_launch(ctx, "constant-coefficient table");
    auto k1 = k_const_stage1<S, C>;
    allow_smem(k1);
    pre_launch(ctx, sizeof(C) == 8 ? "const_stage1_f64" : "const_stage1_f32");
    k1<<<grid, T, smem, ctx.stream>>>(a, b, c, tab, d, n, batch, s, mps, ss, es, ra, rb, rc, rd, ctx.status);
    post_launch(ctx, "constant-coefficient stage 1");
  }
  solve_interface(ctx, ra, rb, rc, rd, y, 2 * m);
  if (!ctx.dry && ctx.err == cudaSuccess) {
    auto k3 = k_const_stage3<S, C>;
    allow_smem(k3);
    pre_launch(ctx, sizeof(C) == 8 ? "const_stage3_f64" : "const_stage3_f32");
    k3<<<grid, T, smem, ctx.stream>>>(tab, d, x, n, batch, s, mps, ss, es, y);
    post_launch(ctx, "constant-coefficient stage 3");
  }
}
}  // namespace

void solve_const(Ctx& ctx, double a, double b, double c, const void* d, void* x, int64_t n, int32_t batch,
                 int64_t ss, int64_t es, int s, tdp_dtype dt, int refine_iters) {
  ctx.rec_n = int64_t(batch) * n;
  ctx.rec_batch = batch;
  ctx.rec_dt = dt;
  if (batch <= 0 || n <= 0) return;
  Iface32Scope f32(ctx, dt != TDP_F64);
  if (s > n) s = int(std::max<int64_t>(2, n));
  // binary64 storage: binary64 arithmetic for TDP_F32_REFINE too.  With the
  // coefficient part tabulated, a row costs 4 binary64 operations and 3 words,
  // which is faster than a binary32 pass, a binary64 residual, a second pass
  // and an update (2048^2 heat step: 0.389 against 0.583 ms), and it needs no
  // scaling of d into the binary32 range.
  if (dt == TDP_F32)
    const_pass<float, float>(ctx, a, b, c, (const float*)d, (float*)x, n, batch, ss, es, s);
  else
    const_pass<double, double>(ctx, a, b, c, (const double*)d, (double*)x, n, batch, ss, es, s);
  (void)refine_iters;
}

template <typename S, typename C>
void multi_pass(Ctx& ctx, const S* a, const S* b, const S* c, const S* d, S* x, int64_t n, int32_t nrhs, int64_t ldd,
                int64_t ldx, int s) {
  const int64_t m = (n + s - 1) / s, M = 2 * m;
  double* ra = ctx.ar->take<double>(M);
  double* rb = ctx.ar->take<double>(M);
  double* rc = ctx.ar->take<double>(M);
  double* A = nrhs > 1 ? ctx.ar->take<double>(M * nrhs) : ra;
  double* B = nrhs > 1 ? ctx.ar->take<double>(M * nrhs) : rb;
  double* Cc = nrhs > 1 ? ctx.ar->take<double>(M * nrhs) : rc;
  double* rd = ctx.ar->take<double>(M * nrhs);
  double* y = ctx.ar->take<double>(M * nrhs);
  C* rT = ctx.ar->take<C>(size_t(s) * m);  // transposed: row j of block k at j * m + k
  C* qT = ctx.ar->take<C>(size_t(s) * m);
  C* gT = ctx.ar->take<C>(size_t(s) * m);
  C* ap = ctx.ar->take<C>(n);
  C* gp = ctx.ar->take<C>(n);
  if (!ctx.dry && ctx.err == cudaSuccess) {
    size_t smem;
    const int T = pick_threads(ctx, s, 3, sizeof(C), false, &smem);
    auto kf = k_multi_factor<S, C>;
    allow_smem(kf);
    pre_launch(ctx, tname<C>("multi_factor_f64", "multi_factor_f32"));
    kf<<<unsigned((m + T - 1) / T), T, smem, ctx.stream>>>(a, b, c, n, s, magic_for(s), m, rT, qT, gT, ap, gp, ra,
                                                           rb, rc, ctx.status);
    post_launch(ctx, "factor");
    if (nrhs > 1) {
      pre_launch(ctx, "multi_replicate");
      k_multi_replicate<<<grid_for(M * nrhs, 256), 256, 0, ctx.stream>>>(ra, rb, rc, M, nrhs, A, B, Cc);
      post_launch(ctx, "interface matrix copies");
    }
    size_t smem2;
    const int T2 = pick_threads(ctx, s, 1, sizeof(C), false, &smem2);
    auto kr = k_multi_reduce<S, C>;
    allow_smem(kr);
    pre_launch(ctx, tname<C>("multi_reduce_f64", "multi_reduce_f32"));
    kr<<<dim3(unsigned((m + T2 - 1) / T2), unsigned(nrhs)), T2, smem2, ctx.stream>>>(rT, qT, gT, c, d, ldd, x, ldx,
                                                                                     n, s, magic_for(s), m, rd);
    post_launch(ctx, "right-hand sides, Stage 1");
  }
  {
    // the columns' interface systems, one after another (decoupled copies);
    // one CTA per column when they are small and many
    SegScope seg(ctx, nullptr, m, nrhs);
    solve_interface(ctx, A, B, Cc, rd, y, M * nrhs);
  }
  if (!ctx.dry && ctx.err == cudaSuccess) {
    pre_launch(ctx, tname<C>("multi_stage3_f64", "multi_stage3_f32"));
    k_multi_stage3<S, C><<<grid_for(n * nrhs, 256), 256, 0, ctx.stream>>>(ap, gp, x, ldx, n, s, m, nrhs, y);
    post_launch(ctx, "right-hand sides, Stage 3");
  }
}

void solve_multi(Ctx& ctx, const void* a, const void* b, const void* c, const void* d, void* x, int64_t n,
                 int32_t nrhs, int64_t ldd, int64_t ldx, int s, tdp_dtype dt) {
  ctx.rec_n = n;
  ctx.rec_batch = 1;
  ctx.rec_dt = dt;
  if (n <= 0 || nrhs <= 0) return;
  if (s > n) s = int(std::max<int64_t>(2, n));
  if (dt == TDP_F64)
    multi_pass<double, double>(ctx, (const double*)a, (const double*)b, (const double*)c, (const double*)d,
                               (double*)x, n, nrhs, ldd, ldx, s);
  else
    multi_pass<float, float>(ctx, (const float*)a, (const float*)b, (const float*)c, (const float*)d, (float*)x, n,
                             nrhs, ldd, ldx, s);
}

int recursion_plan(int64_t n, int32_t batch, int32_t s, int R, tdp_dtype dt, int32_t* m_out, int cap) {
  if (R < 0) R = int(predict_r(n, batch, dt));
  int64_t M = 2 * ((n + s - 1) / s);
  int count = 0;
  for (int level = 1; level <= R && M > kBaseRows && count < cap; ++level) {
    const int m = paper_level_size(level, R, M);
    if (m >= M) break;
    m_out[count++] = m;
    M = 2 * ((M + m - 1) / m);
  }
  return count;
}

void solve_single(Ctx& ctx, const void* a, const void* b, const void* c, const void* d, void* x, int64_t n, int s,
                  tdp_dtype dt, int refine_iters) {
  ctx.rec_n = n;
  ctx.rec_batch = 1;
  ctx.rec_dt = dt;
  if (dt == TDP_F32_REFINE && ctx.window && ctx.rec_mode == 0) {
    window_pass<double>(ctx, (const double*)a, (const double*)b, (const double*)c, (const double*)d, (double*)x, n,
                        refine_iters, nullptr, 0);
    return;
  }
  if (dt == TDP_F32 && ctx.window32 && ctx.rec_mode == 0) {
    window_pass<float>(ctx, (const float*)a, (const float*)b, (const float*)c, (const float*)d, (float*)x, n, 0,
                       nullptr, 0);
    return;
  }
  if (s > n) s = int(std::max<int64_t>(2, n));
  const int64_t m = (n + s - 1) / s;
  if (dt == TDP_F32_REFINE) {
    RefineGuard guard(ctx, a, b, c, d, x, n, nullptr, 0);
    solve_blocks<false>(ctx, a, b, c, d, x, n, s, m, nullptr, nullptr, dt, refine_iters);
    guard.finish();
    return;
  }
  solve_blocks<false>(ctx, a, b, c, d, x, n, s, m, nullptr, nullptr, dt, refine_iters);
}

// While alive, the single-system kernels cut the couplings between the
// systems of a batch inside their tiles (k_stage1_v, k_stage3_resolve_v).
struct FlatScope {
  Ctx& c;
  FlatScope(Ctx& ctx, const int64_t* off, int32_t nsys) : c(ctx) {
    c.flat_off = off;
    c.flat_nsys = nsys;
  }
  ~FlatScope() {
    c.flat_off = nullptr;
    c.flat_nsys = 0;
  }
};

// a2 = a, c2 = c (16-byte copies; a kernel rather than two device-to-device
// copies, which a CUDA graph would run on the copy engines).
__global__ void k_copy2(const double* __restrict__ a, const double* __restrict__ c, double* __restrict__ a2,
                        double* __restrict__ c2, int64_t n) {
  const int64_t pairs = n / 2;
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < pairs; q += int64_t(gridDim.x) * blockDim.x) {
    reinterpret_cast<double2*>(a2)[q] = __ldcs(reinterpret_cast<const double2*>(a) + q);
    reinterpret_cast<double2*>(c2)[q] = __ldcs(reinterpret_cast<const double2*>(c) + q);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) {
    a2[n - 1] = a[n - 1];
    c2[n - 1] = c[n - 1];
  }
}

// With a of every system's first row and c of its last row set to zero the
// copies are the diagonals of one block-diagonal system.
template <typename S>
__global__ void k_cut_edges(const int64_t* __restrict__ off, int32_t batch, int64_t total_n, S* __restrict__ a2,
                            S* __restrict__ c2) {
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < batch; j += int64_t(gridDim.x) * blockDim.x) {
    const int64_t lo = off[j], hi = off[j + 1];
    if (hi > lo && lo >= 0 && hi <= total_n) {  // (offsets out of range touch nothing; the check reports them)
      a2[lo] = S(0);
      c2[hi - 1] = S(0);
    }
  }
}

// Batches of large systems are solved as ONE system of total_n rows whose
// couplings across system boundaries are zero (a block-diagonal tridiagonal
// system): the single-system tiles (16-byte cp.async, no block map) then
// serve batches too.  Blocks may straddle a boundary; elimination across a
// zero coupling is exact.  The kernels that read a and c cut the couplings
// inside their tiles (k_stage1_v, k_stage3_resolve_v, k_stage1, and
// k_refine_mid, which also drops the cross-boundary terms of its residual),
// so every kernel of the chosen schedule must be one of them; refinement
// schedules with other kernels work on copies of a and c with the couplings
// zeroed.
bool flat_batch(const Ctx& ctx, int32_t batch, int64_t total_n, tdp_dtype dt, int s) {
  if (!ctx.batch_flat || batch < 2 || total_n < int64_t(batch) * 4096) return false;
  if (dt == TDP_F32_REFINE) return true;
  const int V = dt == TDP_F64 ? 2 : 4;
  return ctx.vtile && s % V == 0;
}

void solve_flat(Ctx& ctx, const int64_t* offsets, int32_t batch, int64_t total_n, const void* a, const void* b,
                const void* c, const void* d, void* x, int s, tdp_dtype dt, int refine_iters) {
  if (s > total_n) s = int(std::max<int64_t>(2, total_n));
  const int64_t m = (total_n + s - 1) / s;
  if (!ctx.dry && ctx.err == cudaSuccess) {  // invalid offsets raise ST_BADARG (the cuts below stay in range)
    pre_launch(ctx, "check_offsets");
    k_check_offsets<<<grid_for(int64_t(batch) + 1, 256), 256, 0, ctx.stream>>>(offsets, batch, total_n, ctx.status);
    post_launch(ctx, "offsets check");
  }
  const bool cut_in_tiles = dt != TDP_F32_REFINE ||
                            (refine_iters == 1 && ctx.refine3 && ctx.refine_kept);
  if (cut_in_tiles) {
    FlatScope fs(ctx, offsets, batch);
    solve_blocks<false>(ctx, a, b, c, d, x, total_n, s, m, nullptr, nullptr, dt, refine_iters);
    return;
  }
  double* a2 = ctx.ar->take<double>(total_n);
  double* c2 = ctx.ar->take<double>(total_n);
  if (!ctx.dry && ctx.err == cudaSuccess) {
    pre_launch(ctx, "copy_ac");
    k_copy2<<<grid_for(total_n / 2 + 1, 256), 256, 0, ctx.stream>>>((const double*)a, (const double*)c, a2, c2,
                                                                   total_n);
    post_launch(ctx, "copy of a and c");
    pre_launch(ctx, "cut_edges");
    k_cut_edges<double><<<unsigned((batch + 255) / 256), 256, 0, ctx.stream>>>(offsets, batch, total_n, a2, c2);
    post_launch(ctx, "cut edges");
  }
  solve_blocks<false>(ctx, a2, b, c2, d, x, total_n, s, m, nullptr, nullptr, dt, refine_iters);
}

// ---------------------------------------------------------------------------
// Host arrays in, host array out.  The windowed passes (binary32 with
// refinement, binary32) stream: see window_host.  The exact binary64 and
// binary32 solves are pipelined over about eight chunks of whole tiles: while
// chunk k+1 is being copied in (a second stream), Stage 1 runs on chunk k;
// after the interface solve, chunk k's Stage 3 runs while chunk k-1 is copied
// out.  Tiles and arithmetic are those of the one-piece solve, so the answer
// is the same bit for bit.  Other schedules copy everything in, solve, and
// copy out.
// ---------------------------------------------------------------------------
void solve_host(Ctx& ctx, const void* a, const void* b, const void* c, const void* d, void* x, int64_t n, int s,
                tdp_dtype dt, int refine_iters) {
  ctx.rec_n = n;
  ctx.rec_batch = 1;
  ctx.rec_dt = dt;
  if (s > n) s = int(std::max<int64_t>(2, n));
  const size_t el = dt == TDP_F32 ? 4 : 8;
  char* ad = ctx.ar->take<char>(size_t(n) * el);
  char* bd = ctx.ar->take<char>(size_t(n) * el);
  char* cd = ctx.ar->take<char>(size_t(n) * el);
  char* dd = ctx.ar->take<char>(size_t(n) * el);
  char* xd = ctx.ar->take<char>(size_t(n) * el);
  const char* hsrc[4] = {(const char*)a, (const char*)b, (const char*)c, (const char*)d};
  char* dsrc[4] = {ad, bd, cd, dd};
  if (ctx.rec_mode == 0 && ((dt == TDP_F32_REFINE && ctx.window) || (dt == TDP_F32 && ctx.window32))) {
    if (dt == TDP_F32_REFINE)
      window_host<double>(ctx, (const double*)a, (const double*)b, (const double*)c, (const double*)d, (double*)x, n,
                          refine_iters, (double*)ad, (double*)bd, (double*)cd, (double*)dd, (double*)xd);
    else
      window_host<float>(ctx, (const float*)a, (const float*)b, (const float*)c, (const float*)d, (float*)x, n, 0,
                         (float*)ad, (float*)bd, (float*)cd, (float*)dd, (float*)xd);
    return;
  }
  const bool chunked = ctx.vtile && (dt == TDP_F64 ? s % 2 == 0 : (dt == TDP_F32 && s % 4 == 0));
  if (!chunked) {
    if (!ctx.dry && ctx.err == cudaSuccess)
      for (int i = 0; i < 4; ++i)
        ctx.fail(cudaMemcpyAsync(dsrc[i], hsrc[i], size_t(n) * el, cudaMemcpyHostToDevice, ctx.stream), "copy in");
    solve_single(ctx, ad, bd, cd, dd, xd, n, s, dt, refine_iters);
    if (!ctx.dry && ctx.err == cudaSuccess)
      ctx.fail(cudaMemcpyAsync(x, xd, size_t(n) * el, cudaMemcpyDeviceToHost, ctx.stream), "copy out");
    return;
  }
  const int64_t m = (n + s - 1) / s;
  const int64_t ch = std::max<int64_t>(256, ((m + 7) / 8 + 255) / 256 * 256);  // blocks per chunk, whole tiles
  const int64_t nch = (m + ch - 1) / ch;
  Iface32Scope f32(ctx, dt != TDP_F64);
  double* ra = ctx.ar->take<double>(2 * m);
  double* rb = ctx.ar->take<double>(2 * m);
  double* rc = ctx.ar->take<double>(2 * m);
  double* rd = ctx.ar->take<double>(2 * m);
  double* y = ctx.ar->take<double>(2 * m);
  double* ka = dt == TDP_F64 ? ctx.ar->take<double>(n) : nullptr;
  double* kg = dt == TDP_F64 ? ctx.ar->take<double>(n) : nullptr;
  double* kd = dt == TDP_F64 ? ctx.ar->take<double>(n) : nullptr;
  cudaStream_t cs = nullptr;
  std::vector<cudaEvent_t> evs;
  auto event = [&]() {
    cudaEvent_t e = nullptr;
    ctx.fail(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    if (e) evs.push_back(e);
    return e;
  };
  const bool live = !ctx.dry && ctx.err == cudaSuccess;
  if (live) ctx.fail(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "copy stream");
  auto rows = [&](int64_t k, int64_t& r0, int64_t& r1) {
    r0 = k * ch * s;
    r1 = std::min<int64_t>(n, (k + 1) * ch * s);
  };
  // copy in and Stage 1, chunk by chunk
  for (int64_t k = 0; k < nch; ++k) {
    int64_t r0, r1;
    rows(k, r0, r1);
    if (!ctx.dry && ctx.err == cudaSuccess) {
      cudaEvent_t ready = event();
      if (ctx.err == cudaSuccess && k == 0) {  // the copies start after the caller's earlier work
        cudaEvent_t go = event();
        ctx.fail(cudaEventRecord(go, ctx.stream), "event");
        ctx.fail(cudaStreamWaitEvent(cs, go, 0), "event");
      }
      for (int i = 0; i < 4 && ctx.err == cudaSuccess; ++i)
        ctx.fail(cudaMemcpyAsync(dsrc[i] + r0 * el, hsrc[i] + r0 * el, size_t(r1 - r0) * el,
                                 cudaMemcpyHostToDevice, cs), "copy in");
      if (ctx.err == cudaSuccess) ctx.fail(cudaEventRecord(ready, cs), "event");
      if (ctx.err == cudaSuccess) ctx.fail(cudaStreamWaitEvent(ctx.stream, ready, 0), "event");
    }
    ctx.kb = k * ch;
    ctx.ke = std::min(m, (k + 1) * ch);
    if (dt == TDP_F64)
      stage1<double, double, false, true>(ctx, (const double*)ad, (const double*)bd, (const double*)cd,
                                          (const double*)dd, n, s, m, nullptr, ra, rb, rc, rd, ka, kg, kd);
    else
      stage1<float, float, false, false>(ctx, (const float*)ad, (const float*)bd, (const float*)cd,
                                         (const float*)dd, n, s, m, nullptr, ra, rb, rc, rd, (float*)nullptr,
                                         (float*)nullptr, (float*)nullptr);
  }
  ctx.kb = 0;
  ctx.ke = -1;
  solve_interface(ctx, ra, rb, rc, rd, y, 2 * m);
  // Stage 3 and copy out, chunk by chunk
  for (int64_t k = 0; k < nch; ++k) {
    int64_t r0, r1;
    rows(k, r0, r1);
    ctx.kb = k * ch;
    ctx.ke = std::min(m, (k + 1) * ch);
    if (dt == TDP_F64)
      stage3_kept<double, double, false>(ctx, ka, kg, kd, n, s, m, nullptr, y, (double*)xd);
    else
      stage3_resolve<float, float, false>(ctx, (const float*)ad, (const float*)bd, (const float*)cd,
                                          (const float*)dd, n, s, m, nullptr, y, (float*)xd);
    if (!ctx.dry && ctx.err == cudaSuccess) {
      cudaEvent_t done = event();
      if (ctx.err == cudaSuccess) ctx.fail(cudaEventRecord(done, ctx.stream), "event");
      if (ctx.err == cudaSuccess) ctx.fail(cudaStreamWaitEvent(cs, done, 0), "event");
      if (ctx.err == cudaSuccess)
        ctx.fail(cudaMemcpyAsync((char*)x + r0 * el, xd + r0 * el, size_t(r1 - r0) * el, cudaMemcpyDeviceToHost,
                                 cs), "copy out");
    }
  }
  ctx.kb = 0;
  ctx.ke = -1;
  if (cs) {
    // the caller's stream waits for the last copy out
    if (ctx.err == cudaSuccess) {
      cudaEvent_t fin = event();
      if (ctx.err == cudaSuccess) ctx.fail(cudaEventRecord(fin, cs), "event");
      if (ctx.err == cudaSuccess) ctx.fail(cudaStreamWaitEvent(ctx.stream, fin, 0), "event");
    }
    cudaStreamDestroy(cs);  // released once its work is done
  }
  for (cudaEvent_t e : evs) cudaEventDestroy(e);
}

void solve_batched_exact(Ctx& ctx, const int64_t* offsets, int32_t batch, int64_t total_n, const void* a,
                         const void* b, const void* c, const void* d, void* x, int s, tdp_dtype dt, int refine_iters);

void solve_batched(Ctx& ctx, const int64_t* offsets, int32_t batch, int64_t total_n, const void* a, const void* b,
                   const void* c, const void* d, void* x, int s, tdp_dtype dt, int refine_iters) {
  ctx.rec_n = total_n;
  ctx.rec_batch = batch;
  ctx.rec_dt = dt;
  if (batch <= 0 || total_n <= 0) return;
  if (dt == TDP_F32_REFINE && ctx.window && ctx.rec_mode == 0 && !ctx.per_system_s) {
    // every batch as one system: the windowed pass cuts the couplings between systems
    window_pass<double>(ctx, (const double*)a, (const double*)b, (const double*)c, (const double*)d, (double*)x,
                        total_n, refine_iters, offsets, batch);
    return;
  }
  if (dt == TDP_F32 && ctx.window32 && ctx.rec_mode == 0 && !ctx.per_system_s) {
    window_pass<float>(ctx, (const float*)a, (const float*)b, (const float*)c, (const float*)d, (float*)x, total_n, 0,
                       offsets, batch);
    return;
  }
  if (dt == TDP_F32_REFINE) {
    RefineGuard guard(ctx, a, b, c, d, x, total_n, offsets, batch);
    solve_batched_exact(ctx, offsets, batch, total_n, a, b, c, d, x, s, dt, refine_iters);
    guard.finish();
    return;
  }
  solve_batched_exact(ctx, offsets, batch, total_n, a, b, c, d, x, s, dt, refine_iters);
}

// The exact schedules of tdp_solve_batched.
void solve_batched_exact(Ctx& ctx, const int64_t* offsets, int32_t batch, int64_t total_n, const void* a,
                         const void* b, const void* c, const void* d, void* x, int s, tdp_dtype dt,
                         int refine_iters) {
  const bool edges = dt == TDP_F32_REFINE && refine_iters > 0;
  if (s == 0) {
    // per-system sizes from the device predictor (TDP_PER_SYSTEM_S=1); the
    // tiles are sized for the largest of them, so by default one s for the
    // batch's mean system size is used instead
    static thread_local SizeModel model;
    if (ctx.per_system_s && size_model(dt, batch, &model)) {
      BatchMap bm = build_map(ctx, offsets, batch, total_n, model.s_max, edges, &model);
      SegScope seg(ctx, bm.bbase, 0, batch);
      solve_blocks<true>(ctx, a, b, c, d, x, total_n, model.s_max, bm.m, bm.blk, bm.edge, dt, refine_iters);
      return;
    }
    s = predict_s((total_n + batch - 1) / batch, batch, dt);
    if (flat_batch(ctx, batch, total_n, dt, predict_s(total_n, 1, dt))) s = predict_s(total_n, 1, dt);
  }
  if (flat_batch(ctx, batch, total_n, dt, s)) {
    solve_flat(ctx, offsets, batch, total_n, a, b, c, d, x, s, dt, refine_iters);
    return;
  }
  BatchMap bm = build_map(ctx, offsets, batch, total_n, s, edges);
  SegScope seg(ctx, bm.bbase, 0, batch);
  solve_blocks<true>(ctx, a, b, c, d, x, total_n, s, bm.m, bm.blk, bm.edge, dt, refine_iters);
}

void predict_sizes(Ctx& ctx, const int64_t* offsets, int32_t batch, tdp_dtype dt, int32_t* s_out) {
  static thread_local SizeModel model;
  if (ctx.dry || ctx.err != cudaSuccess) return;
  if (!size_model(dt, batch, &model)) {
    model.tab.rows = 0;
    model.s_max = predict_s(1, batch, dt);
  }
  pre_launch(ctx, "predict_sizes");
  k_predict_sizes<<<unsigned((batch + 127) / 128), 128, 0, ctx.stream>>>(offsets, batch, model.tab, model.s_max,
                                                                         1024, s_out);
  post_launch(ctx, "predict sizes");
}

void solve_strided(Ctx& ctx, int32_t batch, int64_t n, int64_t ss, int64_t es, const void* a, const void* b,
                   const void* c, const void* d, void* x, int s, tdp_dtype dt, int refine_iters) {
  ctx.rec_n = int64_t(batch) * n;
  ctx.rec_batch = batch;
  ctx.rec_dt = dt;
  if (batch <= 0 || n <= 0) return;
  const int64_t total = int64_t(batch) * n;
  int64_t* off = ctx.ar->take<int64_t>(batch + 1);
  const bool contiguous = (es == 1 && ss == n);
  const size_t el = (dt == TDP_F32) ? 4 : 8;
  void* g[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  if (!contiguous)
    for (int i = 0; i < 5; ++i) g[i] = ctx.ar->take<char>(total * el);  // each 256-byte aligned
  if (!ctx.dry && ctx.err == cudaSuccess) {
    pre_launch(ctx, "offsets");
    k_iota_offsets<<<unsigned((batch + 256) / 256), 256, 0, ctx.stream>>>(off, batch, n);
    post_launch(ctx, "offsets");
  }
  if (contiguous) {
    solve_batched(ctx, off, batch, total, a, b, c, d, x, s, dt, refine_iters);
    return;
  }
  const void* src[4] = {a, b, c, d};
  // the interleaved layout (sys_stride 1) by tiled transposes, one launch for the
  // four arrays (grid: 32 systems x 32 elements per CTA)
  const bool tiled = ss == 1 && es >= batch && (n + 31) / 32 <= 65535;
  const dim3 tgrid(unsigned((batch + 31) / 32), unsigned((n + 31) / 32));
  if (tiled && !ctx.dry && ctx.err == cudaSuccess) {
    pre_launch(ctx, "gather");
    if (el == 8) {
      Strided4<double> G{};
      for (int i = 0; i < 4; ++i) {
        G.src[i] = (const double*)src[i];
        G.dst[i] = (double*)g[i];
      }
      G.na = 4;
      k_gather_t<double><<<tgrid, 256, 0, ctx.stream>>>(G, batch, n, es);
    } else {
      Strided4<float> G{};
      for (int i = 0; i < 4; ++i) {
        G.src[i] = (const float*)src[i];
        G.dst[i] = (float*)g[i];
      }
      G.na = 4;
      k_gather_t<float><<<tgrid, 256, 0, ctx.stream>>>(G, batch, n, es);
    }
    post_launch(ctx, "gather");
  } else if (!ctx.dry && ctx.err == cudaSuccess) {
    for (int i = 0; i < 4; ++i) {
      pre_launch(ctx, "gather");
      if (el == 8)
        k_gather<double><<<grid_for(total, 256), 256, 0, ctx.stream>>>((const double*)src[i], (double*)g[i], batch,
                                                                       n, ss, es);
      else
        k_gather<float><<<grid_for(total, 256), 256, 0, ctx.stream>>>((const float*)src[i], (float*)g[i], batch, n,
                                                                      ss, es);
      post_launch(ctx, "gather");
    }
  }
  solve_batched(ctx, off, batch, total, g[0], g[1], g[2], g[3], g[4], s, dt, refine_iters);
  if (tiled && !ctx.dry && ctx.err == cudaSuccess) {
    pre_launch(ctx, "scatter");
    if (el == 8)
      k_scatter_t<double><<<tgrid, 256, 0, ctx.stream>>>((const double*)g[4], (double*)x, batch, n, es);
    else
      k_scatter_t<float><<<tgrid, 256, 0, ctx.stream>>>((const float*)g[4], (float*)x, batch, n, es);
    post_launch(ctx, "scatter");
  } else if (!ctx.dry && ctx.err == cudaSuccess) {
    pre_launch(ctx, "scatter");
    if (el == 8)
      k_scatter<double><<<grid_for(total, 256), 256, 0, ctx.stream>>>((const double*)g[4], (double*)x, batch, n, ss,
                                                                      es);
    else
      k_scatter<float><<<grid_for(total, 256), 256, 0, ctx.stream>>>((const float*)g[4], (float*)x, batch, n, ss,
                                                                     es);
    post_launch(ctx, "scatter");
  }
}

void solve_backward(Ctx& ctx, const int64_t* offsets, int32_t batch, int64_t total_n, const void* a, const void* b,
                    const void* c, const void* x, const void* g, void* ga, void* gb, void* gc, void* gd, int s,
                    tdp_dtype dt) {
  ctx.rec_n = total_n;
  ctx.rec_batch = batch;
  ctx.rec_dt = dt;
  if (batch <= 0 || total_n <= 0) return;
  const size_t el = (dt == TDP_F32) ? 4 : 8;
  // binary32 + refinement on the windowed pass: its windows read A^T's
  // diagonals straight from a and c (no transposed copies)
  const bool win = ctx.rec_mode == 0 && !ctx.per_system_s &&
                   ((dt == TDP_F32_REFINE && ctx.window) || (dt == TDP_F32 && ctx.window32));
  uint8_t* edge = win ? nullptr : ctx.ar->take<uint8_t>(total_n);  // (system ends, for the transposed copies)
  char* aT = win ? nullptr : ctx.ar->take<char>(total_n * el);
  char* cT = win ? nullptr : ctx.ar->take<char>(total_n * el);
  char* lam = gd ? (char*)gd : ctx.ar->take<char>(total_n * el);
  if (!win && !ctx.dry && ctx.err == cudaSuccess) {
    ctx.fail(cudaMemsetAsync(edge, 0, size_t(total_n), ctx.stream), "edge clear");
    pre_launch(ctx, "edges");
    k_edges<<<unsigned((batch + 255) / 256), 256, 0, ctx.stream>>>(offsets, batch, edge, total_n);
    post_launch(ctx, "edges");
  }
  if (win && dt == TDP_F32) {
    window_pass<float>(ctx, (const float*)a, (const float*)b, (const float*)c, (const float*)g, (float*)lam, total_n,
                       0, offsets, batch, true);
  } else if (win) {
    window_pass<double>(ctx, (const double*)a, (const double*)b, (const double*)c, (const double*)g, (double*)lam,
                        total_n, 1, offsets, batch, true);
  } else if (!ctx.dry && ctx.err == cudaSuccess) {
    pre_launch(ctx, "transpose");
    if (el == 8)
      k_transpose<double><<<grid_for(total_n, 256), 256, 0, ctx.stream>>>((const double*)a, (const double*)c,
                                                                          (double*)aT, (double*)cT, total_n, edge);
    else
      k_transpose<float><<<grid_for(total_n, 256), 256, 0, ctx.stream>>>((const float*)a, (const float*)c,
                                                                         (float*)aT, (float*)cT, total_n, edge);
    post_launch(ctx, "transpose");
  }
  // The transposed diagonals carry explicit zeros at every system boundary,
  // so the batch is one block-diagonal tridiagonal system of total_n rows:
  // it takes the single-system path (no block map; 16-byte tiles).
  // (binary32 + refinement: one binary64 correction)
  if (!win) solve_single(ctx, aT, b, cT, g, lam, total_n, s, dt, dt == TDP_F32_REFINE ? 1 : 0);
  if (!ctx.dry && ctx.err == cudaSuccess && (ga || gb || gc)) {
    pre_launch(ctx, "gradients");
    if (el == 8)
      k_grads<double><<<grid_for(total_n, 256), 256, 0, ctx.stream>>>((const double*)lam, (const double*)x,
                                                                      (double*)ga, (double*)gb, (double*)gc, total_n,
                                                                      edge);
    else
      k_grads<float><<<grid_for(total_n, 256), 256, 0, ctx.stream>>>((const float*)lam, (const float*)x, (float*)ga,
                                                                     (float*)gb, (float*)gc, total_n, edge);
    post_launch(ctx, "gradients");
    if (win && (ga || gc)) {
      pre_launch(ctx, "gradient_cuts");
      if (el == 8)
        k_grad_cuts<double><<<unsigned((batch + 255) / 256), 256, 0, ctx.stream>>>(offsets, batch, total_n,
                                                                                  (double*)ga, (double*)gc);
      else
        k_grad_cuts<float><<<unsigned((batch + 255) / 256), 256, 0, ctx.stream>>>(offsets, batch, total_n,
                                                                                 (float*)ga, (float*)gc);
      post_launch(ctx, "gradient cuts");
    }
  }
}

void thomas_batched(Ctx& ctx, const int64_t* offsets, int32_t batch, int64_t total_n, const void* a, const void* b,
                    const void* c, const void* d, void* x, tdp_dtype dt) {
  if (batch <= 0 || total_n <= 0) return;
  const size_t el = (dt == TDP_F32) ? 4 : 8;
  char* scratch = ctx.ar->take<char>(total_n * el);
  if (ctx.dry || ctx.err != cudaSuccess) return;
  const unsigned grid = unsigned((batch + 127) / 128);
  pre_launch(ctx, dt == TDP_F32 ? "thomas_f32" : "thomas_f64");
  if (dt == TDP_F32)
    k_thomas<float, float><<<grid, 128, 0, ctx.stream>>>((const float*)a, (const float*)b, (const float*)c,
                                                         (const float*)d, (float*)x, offsets, batch, 0, 0, 1,
                                                         total_n, (float*)scratch, ctx.status);
  else
    k_thomas<double, double><<<grid, 128, 0, ctx.stream>>>((const double*)a, (const double*)b, (const double*)c,
                                                           (const double*)d, (double*)x, offsets, batch, 0, 0, 1,
                                                           total_n, (double*)scratch, ctx.status);
  post_launch(ctx, "thomas");
}

void solve_single_lean(Ctx& ctx, const void* a, const void* b, const void* c, const void* d, void* x, int64_t n,
                       int s, tdp_dtype dt) {
  ctx.rec_n = n;
  ctx.rec_batch = 1;
  ctx.rec_dt = dt;
  if (s > n) s = int(std::max<int64_t>(2, n));
  const int64_t m = (n + s - 1) / s;
  double* ra = ctx.ar->take<double>(2 * m);
  double* rb = ctx.ar->take<double>(2 * m);
  double* rc = ctx.ar->take<double>(2 * m);
  double* rd = ctx.ar->take<double>(2 * m);
  double* y = ctx.ar->take<double>(2 * m);
  if (dt == TDP_F64) {
    using T = double;
    const T *A = (const T*)a, *B = (const T*)b, *Cc = (const T*)c, *D = (const T*)d;
    stage1<T, T, false, false>(ctx, A, B, Cc, D, n, s, m, nullptr, ra, rb, rc, rd, (T*)nullptr, (T*)nullptr,
                               (T*)nullptr);
    solve_interface(ctx, ra, rb, rc, rd, y, 2 * m);
    stage3_resolve<T, T, false>(ctx, A, B, Cc, D, n, s, m, nullptr, y, (T*)x);
  } else {
    using T = float;
    const T *A = (const T*)a, *B = (const T*)b, *Cc = (const T*)c, *D = (const T*)d;
    stage1<T, T, false, false>(ctx, A, B, Cc, D, n, s, m, nullptr, ra, rb, rc, rd, (T*)nullptr, (T*)nullptr,
                               (T*)nullptr);
    solve_interface(ctx, ra, rb, rc, rd, y, 2 * m);
    stage3_resolve<T, T, false>(ctx, A, B, Cc, D, n, s, m, nullptr, y, (T*)x);
  }
}

void stage1_only(Ctx& ctx, const void* a, const void* b, const void* c, const void* d, int64_t n, int s,
                 tdp_dtype dt, double* ra, double* rb, double* rc, double* rd) {
  if (s > n) s = int(std::max<int64_t>(2, n));
  const int64_t m = (n + s - 1) / s;
  if (dt == TDP_F64)
    stage1<double, double, false, false>(ctx, (const double*)a, (const double*)b, (const double*)c,
                                         (const double*)d, n, s, m, nullptr, ra, rb, rc, rd, (double*)nullptr,
                                         (double*)nullptr, (double*)nullptr);
  else if (dt == TDP_F32)
    stage1<float, float, false, false>(ctx, (const float*)a, (const float*)b, (const float*)c, (const float*)d, n, s,
                                       m, nullptr, ra, rb, rc, rd, (float*)nullptr, (float*)nullptr,
                                       (float*)nullptr);
  else
    stage1<double, float, false, false>(ctx, (const double*)a, (const double*)b, (const double*)c,
                                        (const double*)d, n, s, m, nullptr, ra, rb, rc, rd, (float*)nullptr,
                                        (float*)nullptr, (float*)nullptr);
}

}  // namespace tdp
