// Warp-owned, double-buffered block tiles moved by the TMA engine, for the
// single-system kernels that keep no coefficients (binary32 arithmetic on
// binary32 or binary64 storage).
//
// A warp tile is 32 consecutive blocks, one per lane.  Every warp owns two
// tile buffers and walks the tiles w, w + W, w + 2W, ... (W = resident warps
// of the grid).  In a buffer, the block of lane t occupies ls = s + pad
// consecutive elements of each plane (pad = one or two 16-byte chunks, so
// that 16-byte shared loads of eight lanes at the same chunk hit eight
// different bank groups).  A block is contiguous in HBM and in shared
// memory, so each lane fetches its own block with one 1-D bulk copy
// (cp.async.bulk) per array; the copies of a tile complete on one mbarrier
// of the warp.  While the warp sweeps tile i, tile i + W is in flight into the
// other buffer.  Results go back with 1-D bulk stores.  Needs every block to
// start on a 16-byte boundary (one system, s a multiple of V = 16 / sizeof(S)).
// Every mbarrier wait is bounded: after about a second the warp raises
// ST_TIMEOUT, waits (bounded again) for its copies in flight and stops.
#pragma once
#include "tdp_tma.cuh"
#include "tdp_vtile.cuh"

namespace tdp {

// Elements per lane block (s plus the bank-spreading pad).
template <typename S>
__host__ __device__ __forceinline__ int wlane_stride(int s) {
  constexpr int V = 16 / int(sizeof(S));
  return s + (((s / V) % 2 == 0) ? V : 2 * V);
}

// Bytes of shared memory per warp: two mbarriers and two buffers of four planes.
template <typename S>
__host__ __device__ __forceinline__ size_t wwarp_bytes(int s) {
  return 16 + size_t(2) * 4 * 32 * wlane_stride<S>(s) * sizeof(S);
}

__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(smem_u32(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() {
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// ---------------------------------------------------------------------------
// Tile movement
// ---------------------------------------------------------------------------
struct WTile {
  int64_t k0;   // first block
  int nb;       // blocks in the tile (<= 32)
};

// Lane's share of a tile: its block [start, start + len).
struct WLane {
  int64_t start;
  int len;
};

__device__ __forceinline__ WLane wlane(const WTile& w, int lane, int64_t n, int s) {
  WLane l{0, 0};
  if (lane < w.nb) {
    l.start = (w.k0 + lane) * int64_t(s);
    l.len = int(min(int64_t(s), n - l.start));
  }
  return l;
}

// Fetch the lane blocks of a tile (four arrays) into buffer `buf`: whole
// 16-byte chunks by bulk copy completing on `bar`, the ragged end of the
// array element by element.
template <typename S>
__device__ __forceinline__ void wfetch(const WLane& l, const S* const (&src)[4], S* buf, size_t plane, int ls,
                                       uint64_t* bar, int lane) {
  constexpr int V = Vec<S>::W;
  const int nbulk = (l.len / V) * V;
  const unsigned bytes = unsigned(nbulk) * unsigned(sizeof(S));
  const unsigned total = __reduce_add_sync(0xffffffffu, bytes);
  proxy_fence();  // earlier generic accesses of this buffer before the async writes
  if (lane == 0) mbar_expect_tx(bar, 4 * total);
  __syncwarp();
  S* dst = buf + size_t(lane) * ls;
  if (bytes) {
#pragma unroll
    for (int i = 0; i < 4; ++i) bulk_g2s(dst + i * plane, src[i] + l.start, bytes, bar);
  }
  for (int j = nbulk; j < l.len; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) dst[i * plane + j] = src[i][l.start + j];
}

// Lane block of plane `pl` back to x (bulk store of whole chunks, the ragged
// end element by element).
template <typename S>
__device__ __forceinline__ void wstore(const WLane& l, const S* pl, S* x) {
  constexpr int V = Vec<S>::W;
  const int nbulk = (l.len / V) * V;
  for (int j = nbulk; j < l.len; ++j) x[l.start + j] = pl[j];
  if (nbulk) {
    proxy_fence();  // generic writes of the block before the async read
    bulk_s2g(x + l.start, pl, unsigned(nbulk) * unsigned(sizeof(S)));
  }
  bulk_commit();
}

// Per-warp state of the two buffers.
template <typename S>
struct WBufs {
  uint64_t* bar;  // two mbarriers
  S* buf0;        // buffer b starts at buf0 + 4 b plane
  size_t plane;
  int ls;
  unsigned phase;  // bit b: parity to wait for on buffer b
  __device__ __forceinline__ WBufs(unsigned char* base, int s, int lane) {
    ls = wlane_stride<S>(s);
    plane = size_t(32) * ls;
    bar = reinterpret_cast<uint64_t*>(base);
    buf0 = reinterpret_cast<S*>(base + 16);
    phase = 0;
    if (lane == 0) {
      mbar_init(bar, 1);
      mbar_init(bar + 1, 1);
      mbar_init_fence();
    }
    __syncwarp();
  }
  __device__ __forceinline__ S* buf(int b) const { return buf0 + size_t(b) * 4 * plane; }
  // Wait for buffer b; false (ST_TIMEOUT raised) after about a second.
  __device__ __forceinline__ bool wait(int b, unsigned* status) {
    const bool ok = mbar_wait_bounded(bar + b, (phase >> b) & 1u, status);
    phase ^= 1u << b;
    return ok;
  }
};

// The tile loop shared by the kernels: body(w, lane_block, buffer, plane,
// ls, lane) runs on each tile of this warp with its data in shared memory.
template <typename S, typename Body>
__device__ __forceinline__ void wtile_loop(const S* const (&src)[4], int64_t n, int s, int64_t m,
                                           unsigned* status, Body&& body) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  WBufs<S> wb(smem + size_t(wib) * wwarp_bytes<S>(s), s, lane);
  const int64_t ntiles = (m + 31) / 32;
  const int64_t nw = int64_t(gridDim.x) * wpb;
  const int64_t t0 = int64_t(blockIdx.x) * wpb + wib;
  unsigned pending = 0;  // bit b: buffer b has copies in flight
  for (int b = 0; b < 2; ++b) {
    const int64_t tile = t0 + b * nw;
    if (tile < ntiles) {
      const WTile w{tile * 32, int(min(int64_t(32), m - tile * 32))};
      wfetch<S>(wlane(w, lane, n, s), src, wb.buf(b), wb.plane, wb.ls, wb.bar + b, lane);
      pending |= 1u << b;
    }
  }
  int cur = 0;
  bool ok = true;
  for (int64_t tile = t0; tile < ntiles; tile += nw) {
    ok = wb.wait(cur, status);
    pending &= ~(1u << cur);
    if (!ok) break;
    __syncwarp();
    const WTile w{tile * 32, int(min(int64_t(32), m - tile * 32))};
    const WLane l = wlane(w, lane, n, s);
    body(w, l, wb.buf(cur), wb.plane, wb.ls, lane);
    bulk_wait_read0();  // bulk stores of this buffer have read it
    __syncwarp();
    const int64_t next = tile + 2 * nw;
    if (next < ntiles) {
      const WTile wn{next * 32, int(min(int64_t(32), m - next * 32))};
      wfetch<S>(wlane(wn, lane, n, s), src, wb.buf(cur), wb.plane, wb.ls, wb.bar + cur, lane);
      pending |= 1u << cur;
    }
    cur ^= 1;
  }
  if (!ok) {  // stop only once the copies in flight have landed (bounded)
    for (int b = 0; b < 2; ++b)
      if (pending & (1u << b)) wb.wait(b, status);
  }
  bulk_wait0();
}

// Stage 1 (no kept coefficients): interface rows of every block.
template <typename S>
__global__ void __launch_bounds__(128) k_stage1_w(const S* __restrict__ a, const S* __restrict__ b,
                                                  const S* __restrict__ c, const S* __restrict__ d, int64_t n, int s,
                                                  int64_t m, double* __restrict__ ra, double* __restrict__ rb,
                                                  double* __restrict__ rc, double* __restrict__ rd,
                                                  unsigned* __restrict__ status) {
  const S* const src[4] = {a, b, c, d};
  wtile_loop<S>(src, n, s, m, status, [&](const WTile& w, const WLane& l, S* B, size_t plane, int ls, int lane) {
    if (l.len <= 0) return;
    S* pa = B + size_t(lane) * ls;
    const BlockInfo bi{l.start, l.len, w.k0 + lane == 0, w.k0 + lane == m - 1};
    IfaceRows r;
    if (l.len == s) {
      float z = 0.0f;
      r = wreduce_full<S>(pa, pa + plane, pa + 2 * plane, pa + 3 * plane, s, Vec<S>::W, bi.first, bi.last, z);
      if (!(z == 0.0f)) flag(status, ST_SINGULAR);
    } else {
      r = vblock_reduce<S, float, false>(pa, pa + plane, pa + 2 * plane, pa + 3 * plane, 1, 0, bi, status);
    }
    write_iface(w.k0 + lane, r, ra, rb, rc, rd);
  });
}

// Stage 3 by the interior solve with the interface values y known; x in S.
template <typename S>
__global__ void __launch_bounds__(128) k_stage3_resolve_w(const S* __restrict__ a, const S* __restrict__ b,
                                                          const S* __restrict__ c, const S* __restrict__ d,
                                                          int64_t n, int s, int64_t m, const double* __restrict__ y,
                                                          S* __restrict__ x, unsigned* __restrict__ status) {
  const S* const src[4] = {a, b, c, d};
  wtile_loop<S>(src, n, s, m, status, [&](const WTile& w, const WLane& l, S* B, size_t plane, int ls, int lane) {
    if (l.len <= 0) return;
    S* pa = B + size_t(lane) * ls;
    const double2 v = *reinterpret_cast<const double2*>(y + 2 * (w.k0 + lane));
    if (l.len == s) {
      float z = 0.0f;
      wsubstitute_full<S>(pa, pa + plane, pa + 2 * plane, pa + 3 * plane, s, Vec<S>::W, v.x, v.y, z);
      if (!(z == 0.0f)) flag(status, ST_SINGULAR);
    } else {
      vblock_substitute<S, float>(pa, pa + plane, pa + 2 * plane, pa + 3 * plane, 1, 0, l.len, narrow(v.x),
                                  narrow(v.y), status);
    }
    wstore<S>(l, pa + 3 * plane, x);
  });
}

}  // namespace tdp
