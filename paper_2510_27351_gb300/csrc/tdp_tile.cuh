// Tile staging between HBM and shared memory for the per-thread sub-system
// kernels.  A CTA of T threads owns T consecutive blocks (sub-systems) whose
// rows are contiguous in memory.  Global rows are read and written with
// coalesced 16-byte vectors; in shared memory row j of the block owned by
// thread t sits at index j * ld + t with ld = T + 1 (odd), so that the
// per-thread sequential sweeps read consecutive words across a warp.
#pragma once
#include "tdp_device.cuh"

namespace tdp {

struct TileGeom {
  int64_t ts;             // first global row of the tile
  int64_t te;             // one past the last global row
  int s;                  // nominal rows per block
  unsigned magic;         // ceil(2^32 / s): p / s == __umulhi(p, magic) while p * s < 2^32
  int ld;                 // shared-memory leading dimension (T + 1)
  const uint32_t* own;    // mapped tiles: owner (t << 16 | j) of every tile row
};

template <bool MAPPED>
__device__ __forceinline__ void owner(const TileGeom& g, int p, int& t, int& j) {
  if constexpr (MAPPED) {
    const uint32_t o = g.own[p];
    t = int(o >> 16);
    j = int(o & 0xffffu);
  } else {
    t = int(__umulhi(unsigned(p), g.magic));
    j = p - t * g.s;
  }
}

// Smallest j in [lo, hi) with off[j] >= key (hi if none), off non-decreasing;
// all 32 lanes of a warp call it.  Each round probes 32 evenly spaced entries
// at once, so a batch of B systems takes about log32(B) dependent loads.
__device__ __forceinline__ int warp_lower_bound(const int64_t* off, int lo, int hi, int64_t key) {
  const int lane = threadIdx.x & 31;
  while (hi - lo > 32) {
    const int step = (hi - lo + 31) >> 5;
    const int j = lo + lane * step;
    const bool ge = (j >= hi) || off[j] >= key;
    const unsigned msk = __ballot_sync(0xffffffffu, ge);
    const int f = msk ? __ffs(msk) - 1 : 32;
    if (f == 0) return lo;
    // probe f-1 is below key, probe f (if any) at or above it
    const int nlo = lo + (f - 1) * step + 1;
    hi = min(hi, lo + f * step);
    lo = nlo;
  }
  const int j = lo + lane;
  const bool ge = (j >= hi) || off[j] >= key;
  const unsigned msk = __ballot_sync(0xffffffffu, ge);
  return msk ? lo + __ffs(msk) - 1 : hi;
}

// A batch solved as one system (system j in rows [off[j], off[j+1])): in the
// tile of rows [g.ts, g.te), zero a of every system's first row and c of every
// system's last row, and, with fst/fen, mark those rows (byte per tile row,
// zeroed by the caller).  Warp 0 only; jb = warp_lower_bound(off, 1, nsys,
// g.ts).  Two flag arrays, so that neighbouring boundaries never update the
// same byte.
template <typename C>
__device__ __forceinline__ void tile_cut(const TileGeom& g, const int64_t* off, int32_t nsys, int jb, C* A, C* Cc,
                                         uint8_t* fst, uint8_t* fen) {
  for (int j = jb + (threadIdx.x & 31); j < nsys; j += 32) {
    const int64_t p = off[j];
    if (p > g.te) break;
    int t, jj;
    if (p >= g.ts && p < g.te) {  // (the p >= ts test keeps unsorted offsets in the tile)
      owner<false>(g, int(p - g.ts), t, jj);
      A[jj * g.ld + t] = C(0);
      if (fst) fst[p - g.ts] = 1;
    }
    if (p - 1 >= g.ts) {
      owner<false>(g, int(p - 1 - g.ts), t, jj);
      Cc[jj * g.ld + t] = C(0);
      if (fen) fen[p - 1 - g.ts] = 1;
    }
  }
}

// Load NA arrays of storage type S (n_arr valid elements each) for rows
// [ts, te) into shared tiles of compute type C.  When blocks start on vector
// boundaries (one system, s a multiple of V) a vector never straddles two
// blocks: its owner is computed once and its elements go to consecutive rows
// of that block.
template <typename S, typename C, bool MAPPED, int NA>
__device__ __forceinline__ void tile_load(const TileGeom& g, const S* const* src, C* const* dst, int64_t n_arr) {
  constexpr int V = Vec<S>::W;
  constexpr int U = 4;  // chunks in flight per thread per iteration
  const int64_t q0 = g.ts / V, q1 = (g.te + V - 1) / V;
  const int64_t step = blockDim.x;
  const bool whole = !MAPPED && g.s % V == 0 && g.ts % V == 0;
  for (int64_t qb = q0 + threadIdx.x; qb < q1; qb += U * step) {
    Vec<S> v[U][NA];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t q = qb + u * step;
      const int64_t base = q * V;
      if (q < q1 && base + V <= n_arr) {
#pragma unroll
        for (int i = 0; i < NA; ++i) v[u][i] = ldg16<S>(src[i] + base);
      } else {
#pragma unroll
        for (int i = 0; i < NA; ++i)
#pragma unroll
          for (int e = 0; e < V; ++e) v[u][i].v[e] = (q < q1 && base + e < n_arr) ? src[i][base + e] : S(0);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t q = qb + u * step;
      if (q >= q1) continue;
      const int64_t base = q * V;
      if (whole && base + V <= g.te) {
        int t, j;
        owner<false>(g, int(base - g.ts), t, j);
        const int idx = j * g.ld + t;
#pragma unroll
        for (int e = 0; e < V; ++e)
#pragma unroll
          for (int i = 0; i < NA; ++i) dst[i][idx + e * g.ld] = cvt<C>(v[u][i].v[e]);
        continue;
      }
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const int64_t pg = base + e;
        if (pg < g.ts || pg >= g.te) continue;
        int t, j;
        owner<MAPPED>(g, int(pg - g.ts), t, j);
        const int idx = j * g.ld + t;
#pragma unroll
        for (int i = 0; i < NA; ++i) dst[i][idx] = cvt<C>(v[u][i].v[e]);
      }
    }
  }
}

// Store NA shared tiles of type C to global arrays of type D for rows
// [ts, te).  Vectors that straddle the tile edge are written element by
// element so that neighbouring tiles are never touched.
template <typename C, typename D, bool MAPPED, int NA>
__device__ __forceinline__ void tile_store(const TileGeom& g, const C* const* src, D* const* dst) {
  constexpr int V = Vec<D>::W;
  const int64_t q0 = g.ts / V, q1 = (g.te + V - 1) / V;
  const bool whole = !MAPPED && g.s % V == 0 && g.ts % V == 0;
  for (int64_t q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    const int64_t base = q * V;
    if (whole && base + V <= g.te) {
      int t, j;
      owner<false>(g, int(base - g.ts), t, j);
      const int idx = j * g.ld + t;
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        Vec<D> w;
#pragma unroll
        for (int e = 0; e < V; ++e) w.v[e] = cvt<D>(src[i][idx + e * g.ld]);
        stg16<D>(dst[i] + base, w);
      }
      continue;
    }
    Vec<D> v[NA];
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const int64_t pg = base + e;
      if (pg < g.ts || pg >= g.te) continue;
      int t, j;
      owner<MAPPED>(g, int(pg - g.ts), t, j);
      const int idx = j * g.ld + t;
#pragma unroll
      for (int i = 0; i < NA; ++i) v[i].v[e] = cvt<D>(src[i][idx]);
    }
    if (base >= g.ts && base + V <= g.te) {
#pragma unroll
      for (int i = 0; i < NA; ++i) stg16<D>(dst[i] + base, v[i]);
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const int64_t pg = base + e;
        if (pg < g.ts || pg >= g.te) continue;
#pragma unroll
        for (int i = 0; i < NA; ++i) dst[i][pg] = v[i].v[e];
      }
    }
  }
}

// Fill the owner table of a mapped tile (thread t writes its block's rows).
__device__ __forceinline__ void fill_owner(uint32_t* own, int t, int p0, int len) {
  for (int j = 0; j < len; ++j) own[p0 + j] = (uint32_t(t) << 16) | uint32_t(j);
}

}  // namespace tdp
