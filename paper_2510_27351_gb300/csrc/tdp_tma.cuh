// TMA-staged tile pipeline for the per-sub-system kernels.
//
// A persistent CTA of T threads walks tiles of T consecutive blocks.  The
// rows of a tile are contiguous in every array, so one thread issues, per
// array, a single 1-D bulk copy (cp.async.bulk, the TMA engine) of the
// tile's 16-byte-aligned byte range into a linear staging buffer, completing
// on an mbarrier.  Two staging buffers alternate: while the CTA transposes
// and sweeps tile i, the bulk copies of tile i+1 are in flight.  The
// transpose pass moves staging rows into the per-thread layout (row j of
// thread t at j * ld + t); the sweeps then read consecutive words across a
// warp.  Waits on the mbarrier are bounded: after about a second the CTA
// raises ST_TIMEOUT, waits once more (bounded) for its copies and returns.
#pragma once
#include "tdp_pipe.cuh"

namespace tdp {

__device__ __forceinline__ unsigned smem_u32(const void* p) { return unsigned(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Bounded wait for one phase of an mbarrier: about 2^31 clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned phase, unsigned* status) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, phase)) {
    if (clock64() - t0 > (1ll << 31)) {
      flag(status, ST_TIMEOUT);
      return false;
    }
  }
  return true;
}

// Shared-memory carve-up of one CTA.
template <typename S, bool MAPPED, int NA>
struct TmaBufs {
  uint64_t* bar;      // 2 mbarriers
  S* stage[2];        // linear staging, NA arrays of srows elements each
  S* tile;            // NA planes of s * ld elements (per-thread layout)
  uint32_t* own;      // mapped: owner of every tile row
  int srows;
  __host__ __device__ static int staging_rows(int T, int s) { return T * s + 2 * (16 / int(sizeof(S))); }
  __host__ __device__ static size_t bytes(int T, int s, int ld) {
    const size_t st = size_t(NA) * staging_rows(T, s) * sizeof(S);
    const size_t tl = size_t(NA) * s * ld * sizeof(S);
    const size_t ow = MAPPED ? size_t(T) * s * 4 : 0;
    return 16 + 2 * ((st + 15) & ~size_t(15)) + ((tl + 15) & ~size_t(15)) + ow;
  }
  __device__ TmaBufs(unsigned char* base, int T, int s, int ld) {
    srows = staging_rows(T, s);
    const size_t st = (size_t(NA) * srows * sizeof(S) + 15) & ~size_t(15);
    const size_t tl = (size_t(NA) * s * ld * sizeof(S) + 15) & ~size_t(15);
    bar = reinterpret_cast<uint64_t*>(base);
    stage[0] = reinterpret_cast<S*>(base + 16);
    stage[1] = reinterpret_cast<S*>(base + 16 + st);
    tile = reinterpret_cast<S*>(base + 16 + 2 * st);
    own = reinterpret_cast<uint32_t*>(base + 16 + 2 * st + tl);
  }
};

struct CtaTile {
  int64_t k0;
  int nb;
  int64_t ts, te;  // rows of the tile
  int64_t r0;      // first row held by the staging buffer (16-byte aligned)
  int64_t rb;      // rows [r0, rb) come by bulk copy, [rb, te) by plain loads
};

template <typename S, bool MAPPED>
__device__ __forceinline__ CtaTile cta_tile(int64_t tile, int T, int64_t n, int s, int64_t m, const int64_t* blk) {
  constexpr int V = 16 / int(sizeof(S));
  CtaTile c;
  c.k0 = tile * T;
  c.nb = int(min(int64_t(T), m - c.k0));
  c.ts = block_start<MAPPED>(c.k0, n, s, blk);
  c.te = block_start<MAPPED>(c.k0 + c.nb, n, s, blk);
  c.r0 = (c.ts / V) * V;
  int64_t hi = ((c.te + V - 1) / V) * V;
  const int64_t n_al = (n / V) * V;  // never read past the end of an array
  if (hi > n_al) hi = n_al;
  if (hi < c.r0) hi = c.r0;
  c.rb = hi;
  return c;
}

// Thread 0: bulk copies of NA arrays for one tile into a staging buffer.
template <typename S, int NA>
__device__ __forceinline__ void tma_issue(const CtaTile& c, Ptrs<const S, NA> src, S* stage, int srows,
                                          uint64_t* bar) {
  const unsigned bytes = unsigned((c.rb - c.r0) * int64_t(sizeof(S)));
  proxy_fence();
  mbar_expect_tx(bar, bytes * NA);
  if (bytes) {
#pragma unroll
    for (int i = 0; i < NA; ++i) bulk_g2s(stage + size_t(i) * srows, src.p[i] + c.r0, bytes, bar);
  }
}

// All threads: rows past the bulk range (only at the very end of an array),
// then the transpose into the per-thread layout.
template <typename S, bool MAPPED, int NA>
__device__ __forceinline__ void tma_transpose(const CtaTile& c, Ptrs<const S, NA> src, S* stage, int srows, S* tile,
                                              const uint32_t* own, int s, int ld, unsigned magic) {
  const int T = blockDim.x;
  for (int64_t g = c.rb + threadIdx.x; g < c.te; g += T)
#pragma unroll
    for (int i = 0; i < NA; ++i) stage[size_t(i) * srows + (g - c.r0)] = src.p[i][g];
  __syncthreads();
  const int rows = int(c.te - c.ts);
  const int off = int(c.ts - c.r0);
  const size_t plane = size_t(s) * ld;
  for (int p = threadIdx.x; p < rows; p += T) {
    int t, j;
    if constexpr (MAPPED) {
      const uint32_t o = own[p];
      t = int(o >> 16);
      j = int(o & 0xffffu);
    } else {
      t = int(__umulhi(unsigned(p), magic));
      j = p - t * s;
    }
    const int idx = j * ld + t;
#pragma unroll
    for (int i = 0; i < NA; ++i) tile[i * plane + idx] = stage[size_t(i) * srows + off + p];
  }
}

// All threads: NA planes of the tile to global arrays of type D.
template <typename S, typename D, bool MAPPED, int NA>
__device__ __forceinline__ void tma_store(const CtaTile& c, const S* tile, const int (&planes)[NA],
                                          const uint32_t* own, Ptrs<D, NA> dst, int s, int ld, unsigned magic) {
  const int rows = int(c.te - c.ts);
  const size_t plane = size_t(s) * ld;
  for (int p = threadIdx.x; p < rows; p += blockDim.x) {
    int t, j;
    if constexpr (MAPPED) {
      const uint32_t o = own[p];
      t = int(o >> 16);
      j = int(o & 0xffffu);
    } else {
      t = int(__umulhi(unsigned(p), magic));
      j = p - t * s;
    }
    const int idx = j * ld + t;
#pragma unroll
    for (int i = 0; i < NA; ++i) dst.p[i][c.ts + p] = cvt<D>(tile[planes[i] * plane + idx]);
  }
}

// The driver loop shared by the TMA kernels.  `work(c, tile)` runs after the
// tile has been transposed (all threads, with a __syncthreads before it).
template <typename S, bool MAPPED, int NA, typename Work>
__device__ __forceinline__ void tma_loop(Ptrs<const S, NA> src, int64_t n, int s, int ld, unsigned magic, int64_t m,
                                         const int64_t* blk, unsigned* status, Work&& work) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x;
  TmaBufs<S, MAPPED, NA> sb(smem, T, s, ld);
  const int64_t ntiles = (m + T - 1) / T;
  int64_t tile = blockIdx.x;
  if (threadIdx.x == 0) {
    mbar_init(&sb.bar[0], 1);
    mbar_init(&sb.bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (tile < ntiles && threadIdx.x == 0)
    tma_issue<S, NA>(cta_tile<S, MAPPED>(tile, T, n, s, m, blk), src, sb.stage[0], sb.srows, &sb.bar[0]);
  unsigned phase[2] = {0u, 0u};
  int cur = 0;
  bool ok = true;
  for (; tile < ntiles && ok; tile += gridDim.x) {
    const int64_t next = tile + gridDim.x;
    if (next < ntiles && threadIdx.x == 0)
      tma_issue<S, NA>(cta_tile<S, MAPPED>(next, T, n, s, m, blk), src, sb.stage[cur ^ 1], sb.srows,
                       &sb.bar[cur ^ 1]);
    const CtaTile c = cta_tile<S, MAPPED>(tile, T, n, s, m, blk);
    if constexpr (MAPPED) {
      if (int(threadIdx.x) < c.nb) {
        const BlockInfo bi = block_info<MAPPED>(c.k0 + threadIdx.x, n, s, m, blk);
        fill_owner(sb.own, threadIdx.x, int(bi.start - c.ts), bi.len);
      }
    }
    ok = mbar_wait_bounded(&sb.bar[cur], phase[cur], status);
    ok = __syncthreads_and(ok);
    if (!ok) break;
    phase[cur] ^= 1u;
    tma_transpose<S, MAPPED, NA>(c, src, sb.stage[cur], sb.srows, sb.tile, sb.own, s, ld, magic);
    __syncthreads();
    work(c, sb);
    __syncthreads();
    cur ^= 1;
  }
  if (!ok) {
    // a wait ran out: give the copies still in flight one more bounded wait
    for (int b = 0; b < 2; ++b) mbar_wait_bounded(&sb.bar[b], phase[b], nullptr);
  }
}

// ---------------------------------------------------------------------------
// Stage 1 (TMA-staged).
// ---------------------------------------------------------------------------
template <typename S, typename C, bool MAPPED, bool KEEP>
__global__ void __launch_bounds__(256) k_stage1_tma(const S* __restrict__ a, const S* __restrict__ b,
                                                    const S* __restrict__ c, const S* __restrict__ d, int64_t n,
                                                    int s, int ld, unsigned magic, int64_t m,
                                                    const int64_t* __restrict__ blk, double* __restrict__ ra,
                                                    double* __restrict__ rb, double* __restrict__ rc,
                                                    double* __restrict__ rd, C* __restrict__ ka, C* __restrict__ kg,
                                                    C* __restrict__ kd, unsigned* __restrict__ status) {
  const Ptrs<const S, 4> src{{a, b, c, d}};
  tma_loop<S, MAPPED, 4>(src, n, s, ld, magic, m, blk, status, [&](const CtaTile& ct, TmaBufs<S, MAPPED, 4>& sb) {
    const int t = threadIdx.x;
    const size_t plane = size_t(s) * ld;
    if (t < ct.nb) {
      const BlockInfo bi = block_info<MAPPED>(ct.k0 + t, n, s, m, blk);
      S* B = sb.tile;
      const IfaceRows r =
          block_reduce<S, C, KEEP>(B + t, B + plane + t, B + 2 * plane + t, B + 3 * plane + t, ld, bi, status);
      write_iface(ct.k0 + t, r, ra, rb, rc, rd);
    }
    if constexpr (KEEP) {
      __syncthreads();
      const int planes[3] = {0, 2, 3};
      tma_store<S, C, MAPPED, 3>(ct, sb.tile, planes, sb.own, Ptrs<C, 3>{{ka, kg, kd}}, s, ld, magic);
    }
  });
}

// ---------------------------------------------------------------------------
// Stage 3 by repeating the interior solve (TMA-staged).
// ---------------------------------------------------------------------------
template <typename S, typename C, bool MAPPED>
__global__ void __launch_bounds__(256) k_stage3_resolve_tma(const S* __restrict__ a, const S* __restrict__ b,
                                                            const S* __restrict__ c, const S* __restrict__ d,
                                                            int64_t n, int s, int ld, unsigned magic, int64_t m,
                                                            const int64_t* __restrict__ blk,
                                                            const double* __restrict__ y, S* __restrict__ x,
                                                            unsigned* __restrict__ status) {
  const Ptrs<const S, 4> src{{a, b, c, d}};
  tma_loop<S, MAPPED, 4>(src, n, s, ld, magic, m, blk, status, [&](const CtaTile& ct, TmaBufs<S, MAPPED, 4>& sb) {
    const int t = threadIdx.x;
    const size_t plane = size_t(s) * ld;
    if (t < ct.nb) {
      const BlockInfo bi = block_info<MAPPED>(ct.k0 + t, n, s, m, blk);
      const double2 v = *reinterpret_cast<const double2*>(y + 2 * (ct.k0 + t));
      S* B = sb.tile;
      block_substitute<S, C>(B + t, B + plane + t, B + 2 * plane + t, B + 3 * plane + t, ld, bi.len, cvt<C>(v.x),
                             cvt<C>(v.y), status);
    }
    __syncthreads();
    const int planes[1] = {3};
    tma_store<S, S, MAPPED, 1>(ct, sb.tile, planes, sb.own, Ptrs<S, 1>{{x}}, s, ld, magic);
  });
}

}  // namespace tdp
