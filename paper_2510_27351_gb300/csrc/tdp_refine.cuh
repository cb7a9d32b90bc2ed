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
//
// With kept coefficients (KEPT), pass 2 stores x0 in binary32 and, instead of
// rr, the coefficients of the correction's Stage 1 that its Stage 3 needs
// (alpha', gamma', delta', binary32), and pass 3 (k_refine_kept) is
// elementwise: x = x0 + (delta' - alpha' yL - gamma' yR).  Traffic
// 32 + 48 + 24 = 104 bytes per row, and pass 3 needs no sweep.
#pragma once
#include "tdp_kernels.cuh"

namespace tdp {

// Stage 1 of one block (binary32, len >= 3; shorter blocks by block_reduce)
// keeping the coefficients of the elementwise Stage 3: after the call row j
// of (A, C, D) holds (alpha'_j, gamma'_j, delta'_j) with
// x_j = delta'_j - alpha'_j x_L - gamma'_j x_R (rows 0 and len-1 encode x_L
// and x_R themselves).  Same arithmetic as lean_reduce.
__device__ __forceinline__ IfaceRows lean_reduce_keep(float* A, float* B, float* Cc, float* D, int ld,
                                                      const BlockInfo& bi, unsigned* status) {
  const int len = bi.len;
  if (len < 3) return block_reduce<float, float, true>(A, B, Cc, D, ld, bi, status);
  if (bi.last) Cc[(len - 1) * ld] = 0.0f;
  const float a0 = bi.first ? 0.0f : A[0], b0 = B[0], c0 = Cc[0], d0 = D[0];
  float gam = 0.0f, del = 0.0f, alp = -1.0f, z = 0.0f;
  float *pa = A + ld, *pb = B + ld, *pc = Cc + ld, *pd = D + ld;
  for (int j = 1; j < len; ++j) {
    const float a = *pa, b = *pb, c = *pc, d = *pd;
    float e;
    const float x = fmaf(-a, gam, b);
    const float y = rcp_lean(x, e);
    const float r = fmaf(y, e, y);
    const float cy = c * y;
    gam = fmaf(cy, e, cy);
    z = fmaf(r, 0.0f, z);
    const float q = a * r;
    del = fmaf(-q, del, d * r);
    alp = -q * alp;
    *pa = alp;
    *pc = gam;
    *pd = del;
    pa += ld; pb += ld; pc += ld; pd += ld;
  }
  IfaceRows out;
  out.a1 = widen(alp);
  out.b1 = 1.0;
  out.c1 = widen(gam);
  out.d1 = widen(del);
  // backward over rows len-2 .. 1; row len-2 keeps its forward values
  pa = A + (len - 2) * ld; pc = Cc + (len - 2) * ld; pd = D + (len - 2) * ld;
  float ap = *pa, gp = *pc, dp = *pd;
  for (int j = len - 3; j >= 1; --j) {
    pa -= ld; pc -= ld; pd -= ld;
    const float gj = *pc;
    dp = fmaf(-gj, dp, *pd);
    ap = fmaf(-gj, ap, *pa);
    gp = -gj * gp;
    *pa = ap;
    *pc = gp;
    *pd = dp;
  }
  out.a0 = widen(a0);
  out.b0 = widen(fmaf(-c0, ap, b0));
  out.c0 = widen(-c0 * gp);
  out.d0 = widen(fmaf(-c0, dp, d0));
  A[0] = -1.0f; Cc[0] = 0.0f; D[0] = 0.0f;
  A[(len - 1) * ld] = 0.0f; Cc[(len - 1) * ld] = -1.0f; D[(len - 1) * ld] = 0.0f;
  if (!(z == 0.0f)) flag(status, ST_SINGULAR);
  return out;
}

// End of pass 2: Stage 1 of the correction on (A, B, C, G = r) and, with
// KEPT, its kept coefficients to global memory.
template <bool MAPPED, bool KEPT>
__device__ __forceinline__ void refine_mid_reduce(const TileGeom& g, float* sA, float* sB, float* sC, float* sG,
                                                  int t, int nb, int64_t k0, const BlockInfo& bi, double* ra,
                                                  double* rb, double* rc, double* rd, float* ka, float* kg,
                                                  float* kd, unsigned* status) {
  if (t < nb) {
    const IfaceRows r = KEPT ? lean_reduce_keep(sA + t, sB + t, sC + t, sG + t, g.ld, bi, status)
                             : lean_reduce(sA + t, sB + t, sC + t, sG + t, g.ld, bi, status);
    write_iface(k0 + t, r, ra, rb, rc, rd);
  }
  if constexpr (KEPT) {
    __syncthreads();
    const float* src[3] = {sA, sC, sG};
    float* dst[3] = {ka, kg, kd};
    tile_store<float, float, MAPPED, 3>(g, src, dst);
  }
}

// Pass 2 (see above).  Shared memory: five binary32 planes of s * (T + 1)
// rows (a, b, c, d -> x0, gamma -> r), plus the owner table when mapped.
// KEPT: x0 goes to x0f (binary32) and the correction's kept coefficients to
// (ka, kg, kd); x and rr are not written.  FLAT (one system's tiles only): a
// batch solved as one system, boundaries in off[1..nsys-1].
template <bool MAPPED, bool KEPT, bool FLAT>
__global__ void __launch_bounds__(256) k_refine_mid(const double* __restrict__ a, const double* __restrict__ b,
                                                    const double* __restrict__ c, const double* __restrict__ d,
                                                    double* __restrict__ x, float* __restrict__ rr, int64_t n, int s,
                                                    unsigned magic, int64_t m, const int64_t* __restrict__ blk,
                                                    const uint8_t* __restrict__ edge, const double* __restrict__ y,
                                                    double* __restrict__ ra, double* __restrict__ rb,
                                                    double* __restrict__ rc, double* __restrict__ rd,
                                                    float* __restrict__ x0f, float* __restrict__ ka,
                                                    float* __restrict__ kg, float* __restrict__ kd,
                                                    const int64_t* __restrict__ off, int32_t nsys,
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
  const int rows = int(g.te - g.ts);
  // FLAT: rows that start (fst) or end (fen) a system, one byte each after
  // the planes, built only in tiles that hold a system boundary (flat)
  static_assert(!(FLAT && MAPPED), "block-mapped tiles never straddle systems");
  __shared__ int s_cut;
  uint8_t* fst = reinterpret_cast<uint8_t*>(sG + plane);
  uint8_t* fen = fst + size_t(T) * s;
  BlockInfo bi{0, 0, false, false};
  if (t < nb) bi = block_info<MAPPED>(k0 + t, n, s, m, blk);
  if constexpr (MAPPED) {
    if (t < nb) fill_owner(own, t, int(bi.start - g.ts), bi.len);
    __syncthreads();
  }
  int jb = 0;
  if constexpr (FLAT) {
    if (t < 32) {
      jb = warp_lower_bound(off, 1, nsys, g.ts);
      if (t == 0) s_cut = (jb < nsys && off[jb] <= g.te) ? 1 : 0;
    }
  }
  {
    const double* src[4] = {a, b, c, d};
    float* dst[4] = {sA, sB, sC, sD};
    tile_load<double, float, MAPPED, 4>(g, src, dst, n);
  }
  __syncthreads();
  const bool flat = FLAT && s_cut;
  if (flat) {
    for (int q = t; q < rows; q += T) { fst[q] = 0; fen[q] = 0; }
    __syncthreads();
    if (t < 32) tile_cut<float>(g, off, nsys, jb, sA, sC, fst, fen);
    __syncthreads();
  }
  if (t < nb) {
    const double2 v = *reinterpret_cast<const double2*>(y + 2 * (k0 + t));
    lean_substitute(sA + t, sB + t, sC + t, sD + t, sG + t, ld, bi.len, narrow(v.x), narrow(v.y), status);
  }
  __syncthreads();
  // residual, one row per thread in memory order; the neighbours of the
  // tile's end rows are interface values of the neighbouring blocks.  A row
  // that starts a system has no left neighbour term, one that ends a system
  // no right neighbour term.
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
          bool s0 = false, e0 = false, s1 = false, e1 = false;
          if (flat) { s0 = fst[p]; e0 = fen[p]; s1 = fst[p + 1]; e1 = fen[p + 1]; }
          double r0 = fma(-vb.x, w0, vd.x), r1 = fma(-vb.y, w1, vd.y);
          if (!e0) r0 = fma(-vc.x, w1, r0);
          if (!s1) r1 = fma(-va.y, w0, r1);
          if (i > 0 && !s0) r0 = fma(-va.x, widen(xp), r0);
          if (i + 2 < n && !e1) r1 = fma(-vc.y, widen(xn), r1);
          const float f0 = narrow(r0), f1 = narrow(r1);
          if constexpr (KEPT) {
            *reinterpret_cast<float2*>(x0f + i) = make_float2(x0, x1);
          } else {
            *reinterpret_cast<double2*>(x + i) = make_double2(w0, w1);
            *reinterpret_cast<float2*>(rr + i) = make_float2(f0, f1);
          }
          sG[idx] = f0;
          sG[idx + ld] = f1;
        } else {  // the last row of the system
          const double w0 = widen(x0);
          double r0 = fma(-b[i], w0, d[i]);
          if (i > 0 && !(flat && fst[p])) r0 = fma(-a[i], widen(xp), r0);
          const float f0 = narrow(r0);
          if constexpr (KEPT) {
            x0f[i] = x0;
          } else {
            x[i] = w0;
            rr[i] = f0;
          }
          sG[idx] = f0;
        }
      }
    }
    __syncthreads();
    refine_mid_reduce<MAPPED, KEPT>(g, sA, sB, sC, sG, t, nb, k0, bi, ra, rb, rc, rd, ka, kg, kd, status);
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
        if (flat) le[u] |= uint8_t(fst[p] | (fen[p] << 1));
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
      const float rf = narrow(acc);
      if constexpr (KEPT) {
        x0f[i] = xi;
      } else {
        x[i] = xd;
        rr[i] = rf;
      }
      sG[jj * ld + tt] = rf;
    }
  }
  __syncthreads();
  refine_mid_reduce<MAPPED, KEPT>(g, sA, sB, sC, sG, t, nb, k0, bi, ra, rb, rc, rd, ka, kg, kd, status);
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

// Pass 3 with kept coefficients: x = x0 + (delta' - alpha' yL - gamma' yR),
// elementwise; the correction in binary32, the sum in binary64.
template <bool MAPPED>
__global__ void __launch_bounds__(256) k_refine_kept(const float* __restrict__ ka, const float* __restrict__ kg,
                                                     const float* __restrict__ kd, const float* __restrict__ x0f,
                                                     int64_t n, int s, unsigned magic, int64_t m,
                                                     const int64_t* __restrict__ blk, const double* __restrict__ y,
                                                     double* __restrict__ x) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x, t = threadIdx.x;
  const int64_t k0 = int64_t(blockIdx.x) * T;
  if (k0 >= m) return;
  const int nb = int(min(int64_t(T), m - k0));
  float* yl = reinterpret_cast<float*>(smem);
  float* yr = yl + T;
  uint32_t* own = reinterpret_cast<uint32_t*>(yr + T);
  TileGeom g{block_start<MAPPED>(k0, n, s, blk), block_start<MAPPED>(k0 + nb, n, s, blk), s, magic, 0, own};
  if (t < nb) {
    const double2 v = *reinterpret_cast<const double2*>(y + 2 * (k0 + t));
    yl[t] = narrow(v.x);
    yr[t] = narrow(v.y);
    if constexpr (MAPPED) {
      const BlockInfo bi = block_info<MAPPED>(k0 + t, n, s, m, blk);
      fill_owner(own, t, int(bi.start - g.ts), bi.len);
    }
  }
  __syncthreads();
  const int64_t q0 = g.ts / 4, q1 = (g.te + 3) / 4;
  for (int64_t q = q0 + t; q < q1; q += T) {
    const int64_t base = q * 4;
    const bool full = base >= g.ts && base + 4 <= g.te;
    Vec<float> va, vg, vd, vx;
    if (full) {
      va = ldcs16<float>(ka + base); vg = ldcs16<float>(kg + base); vd = ldcs16<float>(kd + base);
      vx = ldcs16<float>(x0f + base);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t pg = base + e;
        const bool in = pg >= g.ts && pg < g.te;
        va.v[e] = in ? ka[pg] : 0.0f; vg.v[e] = in ? kg[pg] : 0.0f; vd.v[e] = in ? kd[pg] : 0.0f;
        vx.v[e] = in ? x0f[pg] : 0.0f;
      }
    }
    double xo[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int64_t pg = base + e;
      int tt = 0, j = 0;
      if (pg >= g.ts && pg < g.te) owner<MAPPED>(g, int(pg - g.ts), tt, j);
      const float dx = fmaf(-vg.v[e], yr[tt], fmaf(-va.v[e], yl[tt], vd.v[e]));
      xo[e] = widen(vx.v[e]) + widen(dx);
    }
    if (full) {
      Vec<double> w0, w1;
      w0.v[0] = xo[0]; w0.v[1] = xo[1]; w1.v[0] = xo[2]; w1.v[1] = xo[3];
      stg16<double>(x + base, w0);
      stg16<double>(x + base + 2, w1);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t pg = base + e;
        if (pg >= g.ts && pg < g.te) x[pg] = xo[e];
      }
    }
  }
}

}  // namespace tdp
