// Warp-tile pipeline for the per-sub-system kernels.
//
// Every warp owns a private double buffer in shared memory and walks the
// tiles w, w + W, w + 2W, ... (W = number of resident warps).  A tile is 32
// consecutive blocks (one per lane).  While a warp sweeps tile i, the copies
// of tile i + W are already in flight: cp.async element copies move the rows
// straight from HBM into the transposed layout (row j of lane t at
// j * ld + t), so no registers hold data in flight and no extra shared-memory
// pass is needed.  Consecutive lanes copy consecutive rows (coalesced global
// reads); ld is chosen on the host so that these scattered shared-memory
// writes are free of bank conflicts for the given s and element size, and
// the lanes' sweeps read consecutive words.
#pragma once
#include "tdp_kernels.cuh"

namespace tdp {

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gmem_src) {
  const unsigned sa = unsigned(__cvta_generic_to_shared(smem_dst));
  if constexpr (BYTES == 8) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem_src) : "memory");
  } else {
    static_assert(BYTES == 4, "element copies of 4 or 8 bytes");
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem_src) : "memory");
  }
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Shared-memory carve-up of one warp.
template <typename S, bool MAPPED, int NA>
struct WarpBufs {
  S* buf[2];
  uint32_t* own[2];
  __device__ __forceinline__ static size_t bytes(int s, int ld) {
    size_t b = size_t(NA) * s * ld * sizeof(S);
    b = (b + 15) & ~size_t(15);
    size_t o = MAPPED ? size_t(32) * s * 4 : 0;
    return 2 * (b + o);
  }
  __device__ __forceinline__ WarpBufs(unsigned char* base, int s, int ld) {
    size_t b = size_t(NA) * s * ld * sizeof(S);
    b = (b + 15) & ~size_t(15);
    const size_t o = MAPPED ? size_t(32) * s * 4 : 0;
    buf[0] = reinterpret_cast<S*>(base);
    buf[1] = reinterpret_cast<S*>(base + b);
    own[0] = reinterpret_cast<uint32_t*>(base + 2 * b);
    own[1] = reinterpret_cast<uint32_t*>(base + 2 * b + o);
  }
};

// Array pointers passed by value so that unrolled loops keep them in registers.
template <typename T, int NA>
struct Ptrs {
  T* p[NA];
};

struct TileRange {
  int64_t k0;
  int nb;
  int64_t ts, te;
};

template <bool MAPPED>
__device__ __forceinline__ TileRange tile_range(int64_t tile, int64_t n, int s, int64_t m, const int64_t* blk) {
  TileRange r;
  r.k0 = tile * 32;
  r.nb = int(min(int64_t(32), m - r.k0));
  r.ts = block_start<MAPPED>(r.k0, n, s, blk);
  r.te = block_start<MAPPED>(r.k0 + r.nb, n, s, blk);
  return r;
}

// Owner table of a mapped tile, then the element copies of NA arrays.
template <typename S, bool MAPPED, int NA>
__device__ __forceinline__ void issue_tile(const TileRange& tr, Ptrs<const S, NA> src, S* buf, uint32_t* own,
                                           int64_t n, int s, int ld, unsigned magic, int64_t m,
                                           const int64_t* blk, int lane) {
  if constexpr (MAPPED) {
    if (lane < tr.nb) {
      const BlockInfo bi = block_info<MAPPED>(tr.k0 + lane, n, s, m, blk);
      fill_owner(own, lane, int(bi.start - tr.ts), bi.len);
    }
    __syncwarp();
  }
  const int rows = int(tr.te - tr.ts);
  const size_t plane = size_t(s) * ld;
  for (int p = lane; p < rows; p += 32) {
    int t, j;
    if constexpr (MAPPED) {
      const uint32_t o = own[p];
      t = int(o >> 16);
      j = int(o & 0xffffu);
    } else {
      t = int(__umulhi(unsigned(p), magic));
      j = p - t * s;
    }
    S* dst = buf + j * ld + t;
    const int64_t g = tr.ts + p;
#pragma unroll
    for (int i = 0; i < NA; ++i) cp_async<sizeof(S)>(dst + i * plane, src.p[i] + g);
  }
}

// Write NA planes of the tile (type S in shared memory) to global arrays of
// type D, lane-consecutive rows.
template <typename S, typename D, bool MAPPED, int NA>
__device__ __forceinline__ void store_tile(const TileRange& tr, const S* buf, const void* /*unused*/,
                                           const int (&plane_ids)[NA], const uint32_t* own, Ptrs<D, NA> dst, int s,
                                           int ld, unsigned magic, int lane) {
  const int rows = int(tr.te - tr.ts);
  const size_t plane = size_t(s) * ld;
  for (int p = lane; p < rows; p += 32) {
    int t, j;
    if constexpr (MAPPED) {
      const uint32_t o = own[p];
      t = int(o >> 16);
      j = int(o & 0xffffu);
    } else {
      t = int(__umulhi(unsigned(p), magic));
      j = p - t * s;
    }
    const S* src = buf + j * ld + t;
    const int64_t g = tr.ts + p;
#pragma unroll
    for (int i = 0; i < NA; ++i) dst.p[i][g] = cvt<D>(src[plane_ids[i] * plane]);
  }
}

// ---------------------------------------------------------------------------
// Stage 1, pipelined.  S = storage type (also the shared-memory type),
// C = arithmetic type.
// ---------------------------------------------------------------------------
template <typename S, typename C, bool MAPPED, bool KEEP>
__global__ void __launch_bounds__(128) k_stage1_pipe(const S* __restrict__ a, const S* __restrict__ b,
                                                     const S* __restrict__ c, const S* __restrict__ d, int64_t n,
                                                     int s, int ld, unsigned magic, int64_t m,
                                                     const int64_t* __restrict__ blk, double* __restrict__ ra,
                                                     double* __restrict__ rb, double* __restrict__ rc,
                                                     double* __restrict__ rd, C* __restrict__ ka,
                                                     C* __restrict__ kg, C* __restrict__ kd,
                                                     unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  using WB = WarpBufs<S, MAPPED, 4>;
  WB wb(smem + size_t(wib) * WB::bytes(s, ld), s, ld);
  const size_t plane = size_t(s) * ld;
  const Ptrs<const S, 4> src{{a, b, c, d}};
  const int64_t ntiles = (m + 31) / 32;
  const int64_t nw = int64_t(gridDim.x) * wpb;
  int64_t tile = int64_t(blockIdx.x) * wpb + wib;
  if (tile < ntiles) {
    const TileRange tr = tile_range<MAPPED>(tile, n, s, m, blk);
    issue_tile<S, MAPPED, 4>(tr, src, wb.buf[0], wb.own[0], n, s, ld, magic, m, blk, lane);
  }
  cp_commit();
  int cur = 0;
  for (; tile < ntiles; tile += nw) {
    const int64_t next = tile + nw;
    if (next < ntiles) {
      const TileRange tn = tile_range<MAPPED>(next, n, s, m, blk);
      issue_tile<S, MAPPED, 4>(tn, src, wb.buf[cur ^ 1], wb.own[cur ^ 1], n, s, ld, magic, m, blk, lane);
    }
    cp_commit();
    cp_wait<1>();
    __syncwarp();
    const TileRange tr = tile_range<MAPPED>(tile, n, s, m, blk);
    S* B = wb.buf[cur];
    if (lane < tr.nb) {
      const BlockInfo bi = block_info<MAPPED>(tr.k0 + lane, n, s, m, blk);
      const IfaceRows r =
          block_reduce<S, C, KEEP>(B + lane, B + plane + lane, B + 2 * plane + lane, B + 3 * plane + lane, ld, bi,
                                   status);
      write_iface(tr.k0 + lane, r, ra, rb, rc, rd);
    }
    if constexpr (KEEP) {
      __syncwarp();
      const int ids[3] = {0, 2, 3};
      store_tile<S, C, MAPPED, 3>(tr, B, nullptr, ids, wb.own[cur], Ptrs<C, 3>{{ka, kg, kd}}, s, ld, magic, lane);
    }
    __syncwarp();
    cur ^= 1;
  }
  cp_wait<0>();
}

// ---------------------------------------------------------------------------
// Stage 3 by repeating the interior solve, pipelined.
// ---------------------------------------------------------------------------
template <typename S, typename C, bool MAPPED>
__global__ void __launch_bounds__(128) k_stage3_resolve_pipe(const S* __restrict__ a, const S* __restrict__ b,
                                                             const S* __restrict__ c, const S* __restrict__ d,
                                                             int64_t n, int s, int ld, unsigned magic, int64_t m,
                                                             const int64_t* __restrict__ blk,
                                                             const double* __restrict__ y, S* __restrict__ x,
                                                             unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  using WB = WarpBufs<S, MAPPED, 4>;
  WB wb(smem + size_t(wib) * WB::bytes(s, ld), s, ld);
  const size_t plane = size_t(s) * ld;
  const Ptrs<const S, 4> src{{a, b, c, d}};
  const int64_t ntiles = (m + 31) / 32;
  const int64_t nw = int64_t(gridDim.x) * wpb;
  int64_t tile = int64_t(blockIdx.x) * wpb + wib;
  if (tile < ntiles) {
    const TileRange tr = tile_range<MAPPED>(tile, n, s, m, blk);
    issue_tile<S, MAPPED, 4>(tr, src, wb.buf[0], wb.own[0], n, s, ld, magic, m, blk, lane);
  }
  cp_commit();
  int cur = 0;
  for (; tile < ntiles; tile += nw) {
    const int64_t next = tile + nw;
    if (next < ntiles) {
      const TileRange tn = tile_range<MAPPED>(next, n, s, m, blk);
      issue_tile<S, MAPPED, 4>(tn, src, wb.buf[cur ^ 1], wb.own[cur ^ 1], n, s, ld, magic, m, blk, lane);
    }
    cp_commit();
    cp_wait<1>();
    __syncwarp();
    const TileRange tr = tile_range<MAPPED>(tile, n, s, m, blk);
    S* B = wb.buf[cur];
    if (lane < tr.nb) {
      const BlockInfo bi = block_info<MAPPED>(tr.k0 + lane, n, s, m, blk);
      const double2 v = *reinterpret_cast<const double2*>(y + 2 * (tr.k0 + lane));
      block_substitute<S, C>(B + lane, B + plane + lane, B + 2 * plane + lane, B + 3 * plane + lane, ld, bi.len,
                             cvt<C>(v.x), cvt<C>(v.y), status);
    }
    __syncwarp();
    {
      const int ids[1] = {3};
      store_tile<S, S, MAPPED, 1>(tr, B, nullptr, ids, wb.own[cur], Ptrs<S, 1>{{x}}, s, ld, magic, lane);
    }
    __syncwarp();
    cur ^= 1;
  }
  cp_wait<0>();
}

}  // namespace tdp

namespace tdp {

// ---------------------------------------------------------------------------
// One pass of binary32 + binary64 iterative refinement, fused per warp tile.
//
// Input: the interface values yc of the correction system solved last (for
// the first pass: of A x = d itself) and, except in the first pass, the
// current iterate xin.  Per block the pass
//   1. forms the right-hand side of that correction system, r = d - A xin
//      (binary64; d itself in the first pass),
//   2. solves the interior of the correction in binary32 with the interface
//      values yc, and updates xout = xin + delta in binary64,
//   3. when another correction follows, forms r' = d - A xout (binary64) and
//      runs the binary32 Stage 1 elimination on it, writing the right-hand
//      side of the next interface system (its matrix is unchanged: the same
//      binary32 pivots as the first Stage 1, computed by the same code).
// Planes of the warp tile: 0 a, 1 b, 2 c, 3 d, 4 x, 5 r (binary64).
// ---------------------------------------------------------------------------
template <bool MAPPED, bool HAS_X>
__global__ void __launch_bounds__(128) k_refine_pass(const double* __restrict__ a, const double* __restrict__ b,
                                                     const double* __restrict__ c, const double* __restrict__ d,
                                                     const double* __restrict__ xin, int64_t n, int s, int ld,
                                                     unsigned magic, int64_t m, const int64_t* __restrict__ blk,
                                                     const double* __restrict__ yc, double* __restrict__ xout,
                                                     double* __restrict__ rd_next, unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NP = 6;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  using WB = WarpBufs<double, MAPPED, NP>;
  WB wb(smem + size_t(wib) * WB::bytes(s, ld), s, ld);
  const size_t plane = size_t(s) * ld;
  const int64_t ntiles = (m + 31) / 32;
  const int64_t nw = int64_t(gridDim.x) * wpb;
  int64_t tile = int64_t(blockIdx.x) * wpb + wib;
  auto issue = [&](int64_t tl, int slot) {
    const TileRange tr = tile_range<MAPPED>(tl, n, s, m, blk);
    if constexpr (HAS_X) {
      issue_tile<double, MAPPED, 5>(tr, Ptrs<const double, 5>{{a, b, c, d, xin}}, wb.buf[slot], wb.own[slot], n, s,
                                    ld, magic, m, blk, lane);
    } else {
      issue_tile<double, MAPPED, 4>(tr, Ptrs<const double, 4>{{a, b, c, d}}, wb.buf[slot], wb.own[slot], n, s, ld,
                                    magic, m, blk, lane);
    }
  };
  if (tile < ntiles) issue(tile, 0);
  cp_commit();
  int cur = 0;
  for (; tile < ntiles; tile += nw) {
    const int64_t next = tile + nw;
    if (next < ntiles) issue(next, cur ^ 1);
    cp_commit();
    cp_wait<1>();
    __syncwarp();
    const TileRange tr = tile_range<MAPPED>(tile, n, s, m, blk);
    double* P = wb.buf[cur];
    double* A = P + lane;
    double* Bp = P + plane + lane;
    double* Cp = P + 2 * plane + lane;
    double* D = P + 3 * plane + lane;
    double* X = P + 4 * plane + lane;
    double* R = P + 5 * plane + lane;
    BlockInfo bi{0, 0, true, true};
    if (lane < tr.nb) bi = block_info<MAPPED>(tr.k0 + lane, n, s, m, blk);
    const int len = bi.len;
    // neighbours' lengths (for the halo rows inside the tile)
    const int len_prev = __shfl_up_sync(0xffffffffu, len, 1);
    const int64_t k = tr.k0 + lane;
    // halo values of the current iterate outside this block
    auto x_left = [&]() -> double {  // x at global row L-1 (not the first row of a system)
      if (!HAS_X) return 0.0;
      if (lane > 0) return P[4 * plane + (len_prev - 1) * ld + (lane - 1)];
      return xin[tr.ts - 1];
    };
    auto x_right = [&]() -> double {  // x at global row R+1
      if (!HAS_X) return 0.0;
      if (lane + 1 < tr.nb) return P[4 * plane + 0 * ld + (lane + 1)];
      return xin[tr.te];
    };
    // ---- 1. right-hand side of the correction system ----
    if (lane < tr.nb && len > 0) {
      for (int j = 0; j < len; ++j) {
        double r = D[j * ld];
        if constexpr (HAS_X) {
          const double xl = (j > 0) ? X[(j - 1) * ld] : (bi.first ? 0.0 : x_left());
          const double xr = (j < len - 1) ? X[(j + 1) * ld] : (bi.last ? 0.0 : x_right());
          r = fma(-Bp[j * ld], X[j * ld], r);
          if (j > 0 || !bi.first) r = fma(-A[j * ld], xl, r);
          if (j < len - 1 || !bi.last) r = fma(-Cp[j * ld], xr, r);
        }
        R[j * ld] = r;
      }
    }
    __syncwarp();
    // ---- 2. binary32 interior solve of the correction, binary64 update ----
    if (lane < tr.nb && len > 0) {
      const double2 yv = *reinterpret_cast<const double2*>(yc + 2 * k);
      const float yl = narrow(yv.x), yr = narrow(yv.y);
      if (len >= 3) {
        float gam = 0.f, del = 0.f;
        for (int j = 1; j <= len - 2; ++j) {
          const float aj = narrow(A[j * ld]), bj = narrow(Bp[j * ld]),
                      cj = narrow(Cp[j * ld]);
          float rj = narrow(R[j * ld]);
          if (j == 1) rj = fmaf(-aj, yl, rj);
          if (j == len - 2) rj = fmaf(-cj, yr, rj);
          const float den = (j == 1) ? bj : fmaf(-aj, gam, bj);
          const float rc = rcp(den, status);
          del = (j == 1) ? rj * rc : fmaf(-aj * rc, del, rj * rc);
          gam = (j == len - 2) ? 0.f : cj * rc;
          // pack (gamma, delta) of row j into its r slot
          R[j * ld] = __hiloint2double(__float_as_int(gam), __float_as_int(del));
        }
        float xn = del;
        const double base_last = HAS_X ? X[(len - 2) * ld] : 0.0;
        X[(len - 2) * ld] = base_last + widen(xn);
        for (int j = len - 3; j >= 1; --j) {
          const double pk = R[j * ld];
          const float gj = __int_as_float(__double2hiint(pk)), dj = __int_as_float(__double2loint(pk));
          xn = fmaf(-gj, xn, dj);
          const double base = HAS_X ? X[j * ld] : 0.0;
          X[j * ld] = base + widen(xn);
        }
      }
      X[0] = (HAS_X ? X[0] : 0.0) + yv.x;
      if (len >= 2) X[(len - 1) * ld] = (HAS_X ? X[(len - 1) * ld] : 0.0) + yv.y;
    }
    __syncwarp();
    // ---- 3. residual of the update and the next interface right-hand side ----
    if (rd_next) {
      if (lane < tr.nb && len > 0) {
        auto xnew_left = [&]() -> double {
          if (lane > 0) return P[4 * plane + (len_prev - 1) * ld + (lane - 1)];
          return (HAS_X ? xin[tr.ts - 1] : 0.0) + yc[2 * tr.k0 - 1];
        };
        auto xnew_right = [&]() -> double {
          if (lane + 1 < tr.nb) return P[4 * plane + (lane + 1)];
          return (HAS_X ? xin[tr.te] : 0.0) + yc[2 * (tr.k0 + tr.nb)];
        };
        for (int j = 0; j < len; ++j) {
          double r = fma(-Bp[j * ld], X[j * ld], D[j * ld]);
          if (j > 0 || !bi.first) r = fma(-A[j * ld], (j > 0) ? X[(j - 1) * ld] : xnew_left(), r);
          if (j < len - 1 || !bi.last) r = fma(-Cp[j * ld], (j < len - 1) ? X[(j + 1) * ld] : xnew_right(), r);
          R[j * ld] = r;
        }
      }
      __syncwarp();
      if (lane < tr.nb) {
        // the same binary32 elimination as Stage 1 (planes a, b, c and r; a, c, r are overwritten)
        const IfaceRows ir = block_reduce<double, float, false>(A, Bp, Cp, R, ld, bi, status);
        *reinterpret_cast<double2*>(rd_next + 2 * k) = make_double2(ir.d0, ir.d1);
      }
    }
    __syncwarp();
    {
      const int ids[1] = {4};
      store_tile<double, double, MAPPED, 1>(tr, P, nullptr, ids, wb.own[cur], Ptrs<double, 1>{{xout}}, s, ld, magic,
                                            lane);
    }
    __syncwarp();
    cur ^= 1;
  }
  cp_wait<0>();
}

}  // namespace tdp
