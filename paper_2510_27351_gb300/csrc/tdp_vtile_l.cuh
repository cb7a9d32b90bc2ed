// Padded block-major tiles for binary32 storage: Stage 1 without kept
// coefficients and Stage 3 by the interior solve.
//
// The interleaved tiles (tdp_vtile.cuh) put chunk g (16 bytes, V rows) of
// block t at word g (T + 1) + t, so the 16-byte cp.async copies of one warp,
// which read 512 consecutive bytes of an array, land (T + 1) * 16 bytes
// apart in shared memory.  Here block t owns a contiguous run of pv chunks
// (its s / V chunks and one or two chunks of padding, pv odd), chunk g at
// word t pv + g: the copies of a warp land in one or two contiguous runs.
// The sweeps read chunk g of thread t at word t pv + g; pv odd puts the
// eight threads of every quarter warp on eight different bank groups.  Full
// blocks take the lean sweeps, a ragged last block the per-row sweeps with
// unit stride (its rows are contiguous); the arithmetic is that of
// k_stage1_v / k_stage3_resolve_v, so the results agree bit for bit.
#pragma once
#include "tdp_vtile.cuh"

namespace tdp {

// Chunks of the padded run of one block: s / V plus one or two, odd.
__host__ __device__ __forceinline__ int ltile_pitch(int cps) { return cps + ((cps & 1) ? 2 : 1); }

// Copies of four arrays, rows [ts, te) of whole blocks, into the padded
// layout; chunks that reach past n are read element by element (zero fill).
template <typename S>
__device__ __forceinline__ void ltile_issue(int64_t ts, int64_t te, int64_t n, int s, int pv,
                                            const S* const (&src)[4], S* const (&pl)[4]) {
  constexpr int V = Vec<S>::W;
  const int chunks = int((te - ts + V - 1) / V);
  const int cps = s / V;
  if (ts + int64_t(chunks) * V <= n) {  // the whole tile inside the arrays (every tile but the last)
    for (int q = threadIdx.x; q < chunks; q += blockDim.x) {
      const int t = q / cps, g = q - t * cps;
      const int idx = (t * pv + g) * V;
#pragma unroll
      for (int i = 0; i < 4; ++i) cp_async16(pl[i] + idx, src[i] + ts + int64_t(q) * V);
    }
    return;
  }
  for (int q = threadIdx.x; q < chunks; q += blockDim.x) {
    const int t = q / cps, g = q - t * cps;
    const int64_t row = ts + int64_t(q) * V;
    const int idx = (t * pv + g) * V;
    if (row + V <= n) {
#pragma unroll
      for (int i = 0; i < 4; ++i) cp_async16(pl[i] + idx, src[i] + row);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int u = 0; u < V; ++u) pl[i][idx + u] = (row + u < n) ? src[i][row + u] : S(0);
    }
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
    if (p >= ts && p < te) A[pos(p)] = S(0);  // (the p >= ts test keeps unsorted offsets in the tile)
    if (p - 1 >= ts) C[pos(p - 1)] = S(0);
  }
}

// Load, and cut for a batch solved as one system, the tile of rows [ts, te).
template <typename S>
__device__ __forceinline__ void ltile_load(const S* a, const S* b, const S* c, const S* d, int64_t ts, int64_t te,
                                           int64_t n, int s, int pv, const int64_t* off, int32_t nsys,
                                           S* const (&pl)[4]) {
  const S* const src[4] = {a, b, c, d};
  ltile_issue<S>(ts, te, n, s, pv, src, pl);
  int jb = 0;
  if (off && threadIdx.x < 32) jb = warp_lower_bound(off, 1, nsys, ts);  // while the copies fly
  cp_async_commit_wait_all();
  __syncthreads();
  if (off) {
    if (threadIdx.x < 32) ltile_cut<S>(ts, te, s, pv, off, nsys, jb, pl[0], pl[2]);
    __syncthreads();
  }
}

// Stage 1 (interface rows only) of the blocks [kb, ke), T per CTA.  Shared
// memory: four planes of T pv V elements.
__global__ void __launch_bounds__(256) k_stage1_l(const float* __restrict__ a, const float* __restrict__ b,
                                                  const float* __restrict__ c, const float* __restrict__ d, int64_t n,
                                                  int s, int64_t m, double* __restrict__ ra, double* __restrict__ rb,
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
  const int64_t ts = k0 * s, te = min(n, (k0 + nb) * s);
  ltile_load<float>(a, b, c, d, ts, te, n, s, pv, off, nsys, pl);
  if (t < nb) {
    const int64_t k = k0 + t;
    const int o = t * pv * V;
    IfaceRows r;
    if ((k + 1) * s <= n) {  // full block
      float z = 0.0f;
      r = wreduce_full<float>(pl[0] + o, pl[1] + o, pl[2] + o, pl[3] + o, s, V, k == 0, k == m - 1, z);
      if (!(z == 0.0f)) flag(status, ST_SINGULAR);
    } else {
      const BlockInfo bi = block_info<false>(k, n, s, m, nullptr);
      r = block_reduce<float, float, false>(pl[0] + o, pl[1] + o, pl[2] + o, pl[3] + o, 1, bi, status);
    }
    write_iface(k, r, ra, rb, rc, rd);
  }
}

// Stage 3 by the interior solve of the blocks [kb, ke), x from the interface
// values y; same tiles as k_stage1_l.
__global__ void __launch_bounds__(256) k_stage3_resolve_l(const float* __restrict__ a, const float* __restrict__ b,
                                                          const float* __restrict__ c, const float* __restrict__ d,
                                                          int64_t n, int s, int64_t m, const double* __restrict__ y,
                                                          float* __restrict__ x, const int64_t* __restrict__ off,
                                                          int32_t nsys, int64_t kb, int64_t ke,
                                                          unsigned* __restrict__ status) {
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
  const int64_t ts = k0 * s, te = min(n, (k0 + nb) * s);
  ltile_load<float>(a, b, c, d, ts, te, n, s, pv, off, nsys, pl);
  if (t < nb) {
    const int64_t k = k0 + t;
    const int o = t * pv * V;
    if ((k + 1) * s <= n) {  // full block
      float z = 0.0f;
      wsubstitute_full<float>(pl[0] + o, pl[1] + o, pl[2] + o, pl[3] + o, s, V, yv.x, yv.y, z);
      if (!(z == 0.0f)) flag(status, ST_SINGULAR);
    } else {
      block_substitute<float, float>(pl[0] + o, pl[1] + o, pl[2] + o, pl[3] + o, 1, int(n - k * s),
                                     cvt<float>(yv.x), cvt<float>(yv.y), status);
    }
  }
  __syncthreads();
  const int chunks = int((te - ts + V - 1) / V);
  if (te == (k0 + nb) * s) {  // whole blocks only: 16-byte stores throughout
    for (int q = t; q < chunks; q += T) {
      const int tt = q / cps, g = q - tt * cps;
      stg16<float>(x + ts + int64_t(q) * V, lds16<float>(pl[3] + (tt * pv + g) * V));
    }
    return;
  }
  for (int q = t; q < chunks; q += T) {
    const int tt = q / cps, g = q - tt * cps;
    const int64_t row = ts + int64_t(q) * V;
    const float* p = pl[3] + (tt * pv + g) * V;
    if (row + V <= te) {
      stg16<float>(x + row, lds16<float>(p));
    } else {
      for (int u = 0; u < V && row + u < te; ++u) x[row + u] = p[u];
    }
  }
}

}  // namespace tdp
