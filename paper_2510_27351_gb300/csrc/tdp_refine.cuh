// Fused passes of the binary32 solve with one binary64 refinement step.
//
// With x0 the binary32 solve and dx the binary32 correction:
//   pass 1  Stage 1 of A x = d (k_stage1, binary32 arithmetic)     reads a, b, c, d
//   pass 2  k_refine_mid: Stage 3 of x0 from the interface values, x0 -> x,
//           r = d - A x0 in binary64 (a, b, c, d read again while the tile
//           is still in L2), r -> rr (binary32: the correction's right-hand
//           side), Stage 1 of A dx = r                             reads a, b, c, d; writes x, rr
//   pass 3  k_refine_last: Stage 3 of dx from its interface values,
//           x += dx in binary64                                    reads a, b, c, rr, x; writes x
// HBM traffic 32 + 44 + 44 = 120 bytes per row against 216 for separate
// kernels (Stage 1, Stage 3, residual, Stage 1, Stage 3, update).  x0 is exact
// in binary32, so the residual is the binary64 residual of the stored x0.
#pragma once
#include "tdp_kernels.cuh"

namespace tdp {

// Pass 2 (see above).  Shared memory: five binary32 planes of s * (T + 1)
// rows (a, b, c, d -> x0, gamma -> r), plus the owner table when mapped.
template <bool MAPPED>
__global__ void __launch_bounds__(256) k_refine_mid(const double* __restrict__ a, const double* __restrict__ b,
                                                    const double* __restrict__ c, const double* __restrict__ d,
                                                    double* __restrict__ x, float* __restrict__ rr, int64_t n, int s,
                                                    unsigned magic, int64_t m, const int64_t* __restrict__ blk,
                                                    const uint8_t* __restrict__ edge, const double* __restrict__ y,
                                                    double* __restrict__ ra, double* __restrict__ rb,
                                                    double* __restrict__ rc, double* __restrict__ rd,
                                                    unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x, ld = T + 1, t = threadIdx.x;
  const int64_t k0 = int64_t(blockIdx.x) * T;
  if (k0 >= m) return;
  const int nb = int(min(int64_t(T), m - k0));
  const size_t plane = size_t(s) * ld;
  float* sA = reinterpret_cast<float*>(smem);
  float* sB = sA + plane;
  float* sC = sB + plane;
  float* sD = sC + plane;
  float* sG = sD + plane;
  uint32_t* own = reinterpret_cast<uint32_t*>(sG + plane);
  TileGeom g{block_start<MAPPED>(k0, n, s, blk), block_start<MAPPED>(k0 + nb, n, s, blk), s, magic, ld, own};
  BlockInfo bi{0, 0, false, false};
  if (t < nb) bi = block_info<MAPPED>(k0 + t, n, s, m, blk);
  if constexpr (MAPPED) {
    if (t < nb) fill_owner(own, t, int(bi.start - g.ts), bi.len);
    __syncthreads();
  }
  {
    const double* src[4] = {a, b, c, d};
    float* dst[4] = {sA, sB, sC, sD};
    tile_load<double, float, MAPPED, 4>(g, src, dst, n);
  }
  __syncthreads();
  if (t < nb) {
    const double2 v = *reinterpret_cast<const double2*>(y + 2 * (k0 + t));
    lean_substitute(sA + t, sB + t, sC + t, sD + t, sG + t, ld, bi.len, narrow(v.x), narrow(v.y), status);
  }
  __syncthreads();
  // residual, one row per thread in memory order; the neighbours of the
  // tile's end rows are interface values of the neighbouring blocks
  const int rows = int(g.te - g.ts);
  const float x_before = k0 > 0 ? narrow(y[2 * k0 - 1]) : 0.0f;
  const float x_after = k0 + nb < m ? narrow(y[2 * (k0 + nb)]) : 0.0f;
  if (!MAPPED && s % 2 == 0) {
    // one system, even s: pairs of rows (16-byte loads and stores), both rows
    // of a pair in one block; all blocks before the last one are full.  The
    // loads of U pairs are issued before any of them is used.
    constexpr int U = 4;
    for (int pb = 2 * t; pb < rows; pb += 2 * T * U) {
      double2 la[U], lb[U], lc[U], ldd[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int p = pb + 2 * T * u;
        if (p + 1 < rows) {
          const int64_t i = g.ts + p;
          la[u] = *reinterpret_cast<const double2*>(a + i);
          lb[u] = *reinterpret_cast<const double2*>(b + i);
          lc[u] = *reinterpret_cast<const double2*>(c + i);
          ldd[u] = *reinterpret_cast<const double2*>(d + i);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int p = pb + 2 * T * u;
        if (p >= rows) break;
        const int64_t i = g.ts + p;
        int tt, jj;
        owner<false>(g, p, tt, jj);
        const int idx = jj * ld + tt;
        const float x0 = sD[idx];
        const bool two = p + 1 < rows;
        const float x1 = two ? sD[idx + ld] : 0.0f;
        const float xp = p == 0 ? x_before : jj > 0 ? sD[idx - ld] : sD[(s - 1) * ld + tt - 1];
        const float xn = p + 2 >= rows ? x_after : jj + 2 < s ? sD[idx + 2 * ld] : sD[tt + 1];
        if (two) {
          const double2 va = la[u], vb = lb[u], vc = lc[u], vd = ldd[u];
          const double w0 = widen(x0), w1 = widen(x1);
          double r0 = fma(-vb.x, w0, vd.x), r1 = fma(-vb.y, w1, vd.y);
          r0 = fma(-vc.x, w1, r0);
          r1 = fma(-va.y, w0, r1);
          if (i > 0) r0 = fma(-va.x, widen(xp), r0);
          if (i + 2 < n) r1 = fma(-vc.y, widen(xn), r1);
          *reinterpret_cast<double2*>(x + i) = make_double2(w0, w1);
          const float f0 = narrow(r0), f1 = narrow(r1);
          *reinterpret_cast<float2*>(rr + i) = make_float2(f0, f1);
          sG[idx] = f0;
          sG[idx + ld] = f1;
        } else {  // the last row of the system
          const double w0 = widen(x0);
          double r0 = fma(-b[i], w0, d[i]);
          if (i > 0) r0 = fma(-a[i], widen(xp), r0);
          x[i] = w0;
          const float f0 = narrow(r0);
          rr[i] = f0;
          sG[idx] = f0;
        }
      }
    }
    __syncthreads();
    if (t < nb) {
      const IfaceRows r = lean_reduce(sA + t, sB + t, sC + t, sG + t, ld, bi, status);
      write_iface(k0 + t, r, ra, rb, rc, rd);
    }
    return;
  }
  constexpr int U = 4;  // loads issued U rows ahead of their use
  for (int pb = t; pb < rows; pb += T * U) {
    double la[U], lb[U], lc[U], ldd[U];
    uint8_t le[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int p = pb + T * u;
      if (p < rows) {
        const int64_t i = g.ts + p;
        la[u] = a[i];
        lb[u] = b[i];
        lc[u] = c[i];
        ldd[u] = d[i];
        le[u] = MAPPED ? edge[i] : uint8_t((i == 0 ? 1 : 0) | (i == n - 1 ? 2 : 0));
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int p = pb + T * u;
      if (p >= rows) break;
      const int64_t i = g.ts + p;
      int tt, jj;
      owner<MAPPED>(g, p, tt, jj);
      const float xi = sD[jj * ld + tt];
      float xp = x_before, xn = x_after;
      if (p > 0) {
        int t2, j2;
        owner<MAPPED>(g, p - 1, t2, j2);
        xp = sD[j2 * ld + t2];
      }
      if (p + 1 < rows) {
        int t2, j2;
        owner<MAPPED>(g, p + 1, t2, j2);
        xn = sD[j2 * ld + t2];
      }
      const double xd = widen(xi);
      double acc = fma(-lb[u], xd, ldd[u]);
      if (!(le[u] & 1)) acc = fma(-la[u], widen(xp), acc);
      if (!(le[u] & 2)) acc = fma(-lc[u], widen(xn), acc);
      x[i] = xd;
      const float rf = narrow(acc);
      rr[i] = rf;
      sG[jj * ld + tt] = rf;
    }
  }
  __syncthreads();
  if (t < nb) {
    const IfaceRows r = lean_reduce(sA + t, sB + t, sC + t, sG + t, ld, bi, status);
    write_iface(k0 + t, r, ra, rb, rc, rd);
  }
}

// Pass 3 (see above).  Shared memory: four binary32 planes, plus the owner
// table when mapped.
template <bool MAPPED>
__global__ void __launch_bounds__(256) k_refine_last(const double* __restrict__ a, const double* __restrict__ b,
                                                     const double* __restrict__ c, const float* __restrict__ rr,
                                                     double* __restrict__ x, int64_t n, int s, unsigned magic,
                                                     int64_t m, const int64_t* __restrict__ blk,
                                                     const double* __restrict__ y, unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x, ld = T + 1, t = threadIdx.x;
  const int64_t k0 = int64_t(blockIdx.x) * T;
  if (k0 >= m) return;
  const int nb = int(min(int64_t(T), m - k0));
  const size_t plane = size_t(s) * ld;
  float* sA = reinterpret_cast<float*>(smem);
  float* sB = sA + plane;
  float* sC = sB + plane;
  float* sD = sC + plane;
  uint32_t* own = reinterpret_cast<uint32_t*>(sD + plane);
  TileGeom g{block_start<MAPPED>(k0, n, s, blk), block_start<MAPPED>(k0 + nb, n, s, blk), s, magic, ld, own};
  BlockInfo bi{0, 0, false, false};
  if (t < nb) bi = block_info<MAPPED>(k0 + t, n, s, m, blk);
  if constexpr (MAPPED) {
    if (t < nb) fill_owner(own, t, int(bi.start - g.ts), bi.len);
    __syncthreads();
  }
  {
    const double* src[3] = {a, b, c};
    float* dst[3] = {sA, sB, sC};
    tile_load<double, float, MAPPED, 3>(g, src, dst, n);
    const float* src2[1] = {rr};
    float* dst2[1] = {sD};
    tile_load<float, float, MAPPED, 1>(g, src2, dst2, n);
  }
  __syncthreads();
  if (t < nb) {
    const double2 v = *reinterpret_cast<const double2*>(y + 2 * (k0 + t));
    lean_substitute(sA + t, sB + t, sC + t, sD + t, sC + t, ld, bi.len, narrow(v.x), narrow(v.y), status);
  }
  __syncthreads();
  const int rows = int(g.te - g.ts);
  constexpr int U = 4;  // loads of x issued U iterations ahead of their use
  if (!MAPPED && s % 2 == 0) {
    for (int pb = 2 * t; pb < rows; pb += 2 * T * U) {
      double2 lx[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int p = pb + 2 * T * u;
        if (p + 1 < rows) lx[u] = *reinterpret_cast<const double2*>(x + g.ts + p);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int p = pb + 2 * T * u;
        if (p >= rows) break;
        int tt, jj;
        owner<false>(g, p, tt, jj);
        const int idx = jj * ld + tt;
        const int64_t i = g.ts + p;
        if (p + 1 < rows)
          *reinterpret_cast<double2*>(x + i) = make_double2(lx[u].x + widen(sD[idx]), lx[u].y + widen(sD[idx + ld]));
        else
          x[i] = x[i] + widen(sD[idx]);
      }
    }
    return;
  }
  for (int pb = t; pb < rows; pb += T * U) {
    double lx[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int p = pb + T * u;
      if (p < rows) lx[u] = x[g.ts + p];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int p = pb + T * u;
      if (p >= rows) break;
      int tt, jj;
      owner<MAPPED>(g, p, tt, jj);
      x[g.ts + p] = lx[u] + widen(sD[jj * ld + tt]);
    }
  }
}

}  // namespace tdp
