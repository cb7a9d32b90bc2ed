// Padded block-major tiles for binary32 storage: Stage 1 without kept
// coefficients and Stage 3 by the interior solve, for full blocks.
//
// The interleaved tiles (tdp_vtile.cuh) put chunk g (16 bytes, V rows) of
// block t at word g (T + 1) + t, so the 16-byte cp.async copies of one warp,
// which read 512 consecutive bytes of an array, land (T + 1) * 16 bytes
// apart in shared memory.  Here block t owns a contiguous run of pv chunks
// (its s / V chunks and one or two chunks of padding, pv odd), chunk g at
// word t pv + g: the copies of a warp land in one or two contiguous runs.
// The sweeps read chunk g of thread t at word t pv + g; pv odd puts the
// eight threads of every quarter warp on eight different bank groups.
// Blocks must be full (len = s): the host sends a ragged last block to the
// interleaved kernels.  Arithmetic as in k_stage1_v / k_stage3_resolve_v
// (the same lean sweeps), so the results agree bit for bit.
//
// BULK: instead of 16-byte cp.async copies, thread t issues one 1-D bulk
// copy (cp.async.bulk, the TMA engine) per array of its own block's s rows
// into its padded run; the copies complete on one mbarrier (bounded wait:
// after about a second the CTA raises ST_TIMEOUT, waits once more for its
// copies and skips its blocks).
#pragma once
#include "tdp_tma.cuh"
#include "tdp_vtile.cuh"

namespace tdp {

// Chunks of the padded run of one block: s / V plus one or two, odd.
__host__ __device__ __forceinline__ int ltile_pitch(int cps) { return cps + ((cps & 1) ? 2 : 1); }

// Copies of the nb full blocks of the tile starting at row ts into the
// padded layout, four arrays.
template <typename S>
__device__ __forceinline__ void ltile_issue(int64_t ts, int nb, int s, int pv, const S* const (&src)[4],
                                            S* const (&pl)[4]) {
  constexpr int V = Vec<S>::W;
  const int cps = s / V, chunks = nb * cps;
  for (int q = threadIdx.x; q < chunks; q += blockDim.x) {
    const int t = q / cps, g = q - t * cps;
    const int64_t row = ts + int64_t(q) * V;
    const int idx = (t * pv + g) * V;
#pragma unroll
    for (int i = 0; i < 4; ++i) cp_async16(pl[i] + idx, src[i] + row);
  }
}

// A batch solved as one system: zero a of every system's first row and c of
// every system's last row inside the tile of rows [ts, te) (as vtile_cut,
// padded layout).  Warp 0 only; jb = warp_lower_bound(off, 1, nsys, ts).
template <typename S>
__device__ __forceinline__ void ltile_cut(int64_t ts, int64_t te, int s, int pv, const int64_t* off, int32_t nsys,
                                          int jb, S* A, S* C) {
  constexpr int V = Vec<S>::W;
  auto pos = [&](int64_t p) {
    const int q = int(p - ts), t = q / s, j = q - t * s;
    return t * pv * V + j;
  };
  for (int j = jb + (threadIdx.x & 31); j < nsys; j += 32) {
    const int64_t p = off[j];
    if (p > te) break;
    if (p < te) A[pos(p)] = S(0);
    if (p - 1 >= ts) C[pos(p - 1)] = S(0);
  }
}

// Load, and cut for a batch solved as one system, the tile of blocks
// [k0, k0 + nb) (rows from ts = k0 s).  False when a bulk copy wait ran out.
// BULK: `bar` is an 8-byte mbarrier in shared memory.
template <typename S, bool BULK>
__device__ __forceinline__ bool ltile_load(const S* a, const S* b, const S* c, const S* d, int64_t k0, int nb, int s,
                                           int pv, const int64_t* off, int32_t nsys, S* const (&pl)[4], uint64_t* bar,
                                           unsigned* status) {
  constexpr int V = Vec<S>::W;
  const int64_t ts = k0 * s, te = ts + int64_t(nb) * s;
  const S* const src[4] = {a, b, c, d};
  const int t = threadIdx.x;
  if constexpr (BULK) {
    if (t == 0) {
      mbar_init(bar, 1);
      mbar_init_fence();
    }
    __syncthreads();
    const unsigned bytes = unsigned(s) * unsigned(sizeof(S));
    if (t == 0) mbar_expect_tx(bar, 4u * unsigned(nb) * bytes);
    if (t < nb) {
#pragma unroll
      for (int i = 0; i < 4; ++i) bulk_g2s(pl[i] + t * pv * V, src[i] + ts + int64_t(t) * s, bytes, bar);
    }
  } else {
    ltile_issue<S>(ts, nb, s, pv, src, pl);
  }
  int jb = 0;
  if (off && t < 32) jb = warp_lower_bound(off, 1, nsys, ts);  // while the copies fly
  if constexpr (BULK) {
    const bool ok = __syncthreads_and(mbar_wait_bounded(bar, 0, status));
    if (!ok) {
      mbar_wait_bounded(bar, 0, nullptr);  // one more bounded wait for the copies in flight
      return false;
    }
  } else {
    cp_async_commit_wait_all();
    __syncthreads();
  }
  if (off) {
    if (t < 32) ltile_cut<S>(ts, te, s, pv, off, nsys, jb, pl[0], pl[2]);
    __syncthreads();
  }
  return true;
}

// Stage 1 (interface rows only) of the full blocks [kb, ke), T per CTA.
// Shared memory: four planes of T pv V elements (and the mbarrier).
template <bool BULK>
__global__ void __launch_bounds__(256) k_stage1_l(const float* __restrict__ a, const float* __restrict__ b,
                                                  const float* __restrict__ c, const float* __restrict__ d, int s,
                                                  int64_t m, double* __restrict__ ra, double* __restrict__ rb,
                                                  double* __restrict__ rc, double* __restrict__ rd,
                                                  const int64_t* __restrict__ off, int32_t nsys, int64_t kb,
                                                  int64_t ke, unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int V = 4;
  const int T = blockDim.x, t = threadIdx.x;
  const int64_t k0 = kb + int64_t(blockIdx.x) * T;
  if (k0 >= ke) return;
  const int nb = int(min(int64_t(T), ke - k0));
  const int pv = ltile_pitch(s / V);
  const size_t plane = size_t(T) * pv * V;
  float* A = reinterpret_cast<float*>(smem);
  float* const pl[4] = {A, A + plane, A + 2 * plane, A + 3 * plane};
  if (!ltile_load<float, BULK>(a, b, c, d, k0, nb, s, pv, off, nsys, pl, reinterpret_cast<uint64_t*>(A + 4 * plane),
                               status))
    return;
  if (t < nb) {
    const int64_t k = k0 + t;
    const int o = t * pv * V;
    float z = 0.0f;
    const IfaceRows r = wreduce_full<float>(pl[0] + o, pl[1] + o, pl[2] + o, pl[3] + o, s, V, k == 0, k == m - 1, z);
    if (!(z == 0.0f)) flag(status, ST_SINGULAR);
    write_iface(k, r, ra, rb, rc, rd);
  }
}

// Stage 3 by the interior solve of the full blocks [kb, ke), x from the
// interface values y; same tiles as k_stage1_l.
template <bool BULK>
__global__ void __launch_bounds__(256) k_stage3_resolve_l(const float* __restrict__ a, const float* __restrict__ b,
                                                          const float* __restrict__ c, const float* __restrict__ d,
                                                          int s, const double* __restrict__ y, float* __restrict__ x,
                                                          const int64_t* __restrict__ off, int32_t nsys, int64_t kb,
                                                          int64_t ke, unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int V = 4;
  const int T = blockDim.x, t = threadIdx.x;
  const int64_t k0 = kb + int64_t(blockIdx.x) * T;
  if (k0 >= ke) return;
  const int nb = int(min(int64_t(T), ke - k0));
  const int cps = s / V, pv = ltile_pitch(cps);
  const size_t plane = size_t(T) * pv * V;
  float* A = reinterpret_cast<float*>(smem);
  float* const pl[4] = {A, A + plane, A + 2 * plane, A + 3 * plane};
  double2 yv = make_double2(0.0, 0.0);
  if (t < nb) yv = *reinterpret_cast<const double2*>(y + 2 * (k0 + t));
  const int64_t ts = k0 * s;
  if (!ltile_load<float, BULK>(a, b, c, d, k0, nb, s, pv, off, nsys, pl, reinterpret_cast<uint64_t*>(A + 4 * plane),
                               status))
    return;
  if (t < nb) {
    const int o = t * pv * V;
    float z = 0.0f;
    wsubstitute_full<float>(pl[0] + o, pl[1] + o, pl[2] + o, pl[3] + o, s, V, yv.x, yv.y, z);
    if (!(z == 0.0f)) flag(status, ST_SINGULAR);
  }
  __syncthreads();
  const int chunks = nb * cps;
  for (int q = t; q < chunks; q += T) {
    const int tt = q / cps, g = q - tt * cps;
    stg16<float>(x + ts + int64_t(q) * V, lds16<float>(pl[3] + (tt * pv + g) * V));
  }
}

}  // namespace tdp
