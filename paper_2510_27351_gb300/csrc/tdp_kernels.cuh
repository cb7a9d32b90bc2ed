// Kernels of the partition method (Stage 1, Stage 3, the interface-system
// recursion) and of the plain Thomas baseline.
//
// Notation: block (sub-system) k holds rows L..R of one system, len = R-L+1
// rows; within the block row j = i - L.  Stage 1 eliminates, for every
// block, the sub-diagonal downwards (rows L+1..R), keeping the coupling to
// x[L] as a spike column:
//     alpha_j x[L] + x[L+j] + gamma_j x[L+j+1] = delta_j,
// so that row R is already an interface equation.  A backward pass over the
// interior expresses every interior unknown through both interface values,
//     x[L+j] = delta'_j - alpha'_j x[L] - gamma'_j x[R],
// which, put into row L, gives its interface equation.  Stage 2 solves the
// tridiagonal interface system (two rows per block, x[L_0], x[R_0], x[L_1],
// ...) in binary64.  Stage 3 either evaluates the expression above from the
// stored (alpha', gamma', delta') or repeats the interior solve with the
// interface values known.
#pragma once
#include <type_traits>

#include "tdp_tile.cuh"

namespace tdp {

// Interface rows of one block, in binary64.
struct IfaceRows {
  double a0, b0, c0, d0;  // row for x[L]: a0 x[L-1] + b0 x[L] + c0 x[R] = d0
  double a1, b1, c1, d1;  // row for x[R]: a1 x[L] + b1 x[R] + c1 x[R+1] = d1
};

__device__ __forceinline__ void write_iface(int64_t k, const IfaceRows& r, double* ra, double* rb, double* rc,
                                            double* rd) {
  *reinterpret_cast<double2*>(ra + 2 * k) = make_double2(r.a0, r.a1);
  *reinterpret_cast<double2*>(rb + 2 * k) = make_double2(r.b0, r.b1);
  *reinterpret_cast<double2*>(rc + 2 * k) = make_double2(r.c0, r.c1);
  *reinterpret_cast<double2*>(rd + 2 * k) = make_double2(r.d0, r.d1);
}

// ---------------------------------------------------------------------------
// Stage 1 sweep of one block held in shared memory (rows j*ld of the four
// tiles).  On return the tiles hold, per row, (alpha', -, gamma', delta')
// when KEEP is set (rows L and R get the values that make Stage 3's formula
// return the interface values).  Arithmetic in C.
// ---------------------------------------------------------------------------
template <typename S, typename C, bool KEEP>
__device__ __forceinline__ IfaceRows block_reduce(S* sA, S* sB, S* sC, S* sD, int ld, const BlockInfo& bi,
                                                  unsigned* status) {
  // tiles hold type S; arithmetic in C; values written back are exact in S
  IfaceRows out;
  const int len = bi.len;
  if (len <= 0) {
    out = IfaceRows{0.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0};
    return out;
  }
  C a0 = cvt<C>(sA[0]), b0 = cvt<C>(sB[0]), c0 = cvt<C>(sC[0]), d0 = cvt<C>(sD[0]);
  if (bi.first) a0 = C(0);
  if (len == 1) {
    if (bi.last) c0 = C(0);
    out = IfaceRows{to_f64(a0), to_f64(b0), to_f64(c0), to_f64(d0), 0.0, 1.0, 0.0, 0.0};
    if (KEEP) { sA[0] = S(-1); sC[0] = S(0); sD[0] = S(0); }
    return out;
  }
  // forward sweep, rows 1..len-1
  C gam, del, alp;
  {
    const C a1 = cvt<C>(sA[ld]), b1 = cvt<C>(sB[ld]);
    C c1 = cvt<C>(sC[ld]);
    const C d1 = cvt<C>(sD[ld]);
    if (len == 2 && bi.last) c1 = C(0);
    const C r = rcp(b1, status);
    gam = c1 * r;
    del = d1 * r;
    alp = a1 * r;
    sA[ld] = cvt<S>(alp); sC[ld] = cvt<S>(gam); sD[ld] = cvt<S>(del);
  }
  for (int j = 2; j < len; ++j) {
    const C aj = cvt<C>(sA[j * ld]), bj = cvt<C>(sB[j * ld]);
    C cj = cvt<C>(sC[j * ld]);
    const C dj = cvt<C>(sD[j * ld]);
    if (j == len - 1 && bi.last) cj = C(0);
    const C r = rcp(fma(-aj, gam, bj), status);
    const C q = aj * r;
    gam = cj * r;
    del = fma(-q, del, dj * r);
    alp = -q * alp;
    sA[j * ld] = cvt<S>(alp); sC[j * ld] = cvt<S>(gam); sD[j * ld] = cvt<S>(del);
  }
  out.a1 = to_f64(alp);
  out.b1 = 1.0;
  out.c1 = to_f64(gam);
  out.d1 = to_f64(del);
  // backward over the interior: primes of row 1 give row L's equation
  C ap, gp, dp;
  if (len == 2) {
    ap = C(0); gp = C(-1); dp = C(0);  // x[L+1] is x[R] itself
  } else {
    ap = cvt<C>(sA[(len - 2) * ld]); gp = cvt<C>(sC[(len - 2) * ld]); dp = cvt<C>(sD[(len - 2) * ld]);
    for (int j = len - 3; j >= 1; --j) {
      const C aj = cvt<C>(sA[j * ld]), gj = cvt<C>(sC[j * ld]), dj = cvt<C>(sD[j * ld]);
      dp = fma(-gj, dp, dj);
      ap = fma(-gj, ap, aj);
      gp = -gj * gp;
      if (KEEP) { sA[j * ld] = cvt<S>(ap); sC[j * ld] = cvt<S>(gp); sD[j * ld] = cvt<S>(dp); }
    }
  }
  out.a0 = to_f64(a0);
  out.b0 = to_f64(fma(-c0, ap, b0));
  out.c0 = to_f64(-c0 * gp);
  out.d0 = to_f64(fma(-c0, dp, d0));
  if (KEEP) {
    sA[0] = S(-1); sC[0] = S(0); sD[0] = S(0);
    sA[(len - 1) * ld] = S(0); sC[(len - 1) * ld] = S(-1); sD[(len - 1) * ld] = S(0);
  }
  return out;
}

// ---------------------------------------------------------------------------
// Lean binary32 sweeps for the register-staged tiles.  Same recurrences as
// block_reduce / block_substitute, with pointers stepped by ld, the first and
// last rows peeled, gamma, delta and alpha started at (0, 0, -1) so that the
// first interior row needs no special case, and the pivot check folded into
// z = fma(r, 0, z) (nan once a reciprocal is infinite or nan), tested once
// per block.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rcp_lean(float x, float& e) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  e = fmaf(-x, y, 1.0f);
  return y;
}

// Stage 1 without kept coefficients (len >= 3 handled here, shorter blocks by
// block_reduce).  The forward values overwrite the a, c, d rows.
__device__ __forceinline__ IfaceRows lean_reduce(float* A, float* B, float* Cc, float* D, int ld,
                                                 const BlockInfo& bi, unsigned* status) {
  const int len = bi.len;
  if (len < 3) return block_reduce<float, float, false>(A, B, Cc, D, ld, bi, status);
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
  // backward over rows len-2 .. 1
  pa = A + (len - 2) * ld; pc = Cc + (len - 2) * ld; pd = D + (len - 2) * ld;
  float ap = *pa, gp = *pc, dp = *pd;
  for (int j = len - 3; j >= 1; --j) {
    pa -= ld; pc -= ld; pd -= ld;
    const float gj = *pc;
    dp = fmaf(-gj, dp, *pd);
    ap = fmaf(-gj, ap, *pa);
    gp = -gj * gp;
  }
  out.a0 = widen(a0);
  out.b0 = widen(fmaf(-c0, ap, b0));
  out.c0 = widen(-c0 * gp);
  out.d0 = widen(fmaf(-c0, dp, d0));
  if (!(z == 0.0f)) flag(status, ST_SINGULAR);
  return out;
}

// Stage 3 interior solve (len >= 3 here, shorter blocks are trivial): gamma
// goes to G (which may be the c plane when c is not needed afterwards), x to D.
__device__ __forceinline__ void lean_substitute(const float* A, const float* B, const float* Cc, float* D, float* G,
                                                int ld, int len, float yl, float yr, unsigned* status) {
  if (len <= 0) return;
  if (len >= 3) {
    // the known interface values move to the right-hand sides of rows 1 and len-2
    const float c_end = Cc[(len - 2) * ld];
    D[ld] = fmaf(-A[ld], yl, D[ld]);
    D[(len - 2) * ld] = fmaf(-c_end, yr, D[(len - 2) * ld]);
    float gam = 0.0f, del = 0.0f, z = 0.0f;
    const float *pa = A + ld, *pb = B + ld, *pc = Cc + ld;
    float *pd = D + ld, *pg = G + ld;
    for (int j = 1; j < len - 2; ++j) {
      const float a = *pa, b = *pb, c = *pc, d = *pd;
      float e;
      const float x = fmaf(-a, gam, b);
      const float y = rcp_lean(x, e);
      const float r = fmaf(y, e, y);
      const float cy = c * y;
      gam = fmaf(cy, e, cy);
      z = fmaf(r, 0.0f, z);
      del = fmaf(-a * r, del, d * r);
      *pg = gam;
      *pd = del;
      pa += ld; pb += ld; pc += ld; pd += ld; pg += ld;
    }
    {  // row len-2: no coupling to the right any more
      float e;
      const float a = *pa;
      const float x = fmaf(-a, gam, *pb);
      const float y = rcp_lean(x, e);
      const float r = fmaf(y, e, y);
      z = fmaf(r, 0.0f, z);
      del = fmaf(-a * r, del, *pd * r);
      *pd = del;
    }
    float xn = del;
    for (int j = len - 3; j >= 1; --j) {
      pd -= ld; pg -= ld;
      xn = fmaf(-*pg, xn, *pd);
      *pd = xn;
    }
    if (!(z == 0.0f)) flag(status, ST_SINGULAR);
  }
  D[0] = yl;
  if (len >= 2) D[(len - 1) * ld] = yr;
}

// Interior solve of one block with x[L] = yl and x[R] = yr known (Stage 3,
// the "substitute and solve the rest" step).  Reads a, b, c, d from the
// tiles (type S), leaves x in the D tile, uses the C tile as scratch.
template <typename S, typename C>
__device__ __forceinline__ void block_substitute(S* sA, S* sB, S* sC, S* sD, int ld, int len, C yl, C yr,
                                                 unsigned* status) {
  if (len <= 0) return;
  if (len == 1) { sD[0] = cvt<S>(yl); return; }
  if (len == 2) { sD[0] = cvt<S>(yl); sD[ld] = cvt<S>(yr); return; }
  // interior rows 1..len-2
  C gam = C(0), del = C(0);
  for (int j = 1; j <= len - 2; ++j) {
    const C aj = cvt<C>(sA[j * ld]), bj = cvt<C>(sB[j * ld]), cj = cvt<C>(sC[j * ld]);
    C dj = cvt<C>(sD[j * ld]);
    if (j == 1) dj = fma(-aj, yl, dj);
    if (j == len - 2) dj = fma(-cj, yr, dj);
    const C den = (j == 1) ? bj : fma(-aj, gam, bj);
    const C r = rcp(den, status);
    del = (j == 1) ? dj * r : fma(-aj * r, del, dj * r);
    gam = (j == len - 2) ? C(0) : cj * r;
    sC[j * ld] = cvt<S>(gam);
    sD[j * ld] = cvt<S>(del);
  }
  C xn = del;  // x at row len-2
  sD[(len - 2) * ld] = cvt<S>(xn);
  for (int j = len - 3; j >= 1; --j) {
    xn = fma(-cvt<C>(sC[j * ld]), xn, cvt<C>(sD[j * ld]));
    sD[j * ld] = cvt<S>(xn);
  }
  sD[0] = cvt<S>(yl);
  sD[(len - 1) * ld] = cvt<S>(yr);
}

// ---------------------------------------------------------------------------
// Stage 1 kernel: one thread per block, T blocks per CTA.
// ---------------------------------------------------------------------------
template <typename S, typename C, bool MAPPED, bool KEEP>
__global__ void __launch_bounds__(256) k_stage1(const S* __restrict__ a, const S* __restrict__ b,
                                                const S* __restrict__ c, const S* __restrict__ d, int64_t n, int s,
                                                unsigned magic, int64_t m, const int64_t* __restrict__ blk,
                                                double* __restrict__ ra, double* __restrict__ rb,
                                                double* __restrict__ rc, double* __restrict__ rd,
                                                C* __restrict__ oa, C* __restrict__ og, C* __restrict__ od,
                                                const int64_t* __restrict__ off, int32_t nsys,
                                                unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x, ld = T + 1, t = threadIdx.x;
  const int64_t k0 = int64_t(blockIdx.x) * T;
  if (k0 >= m) return;
  const int nb = int(min(int64_t(T), m - k0));
  C* sA = reinterpret_cast<C*>(smem);
  C* sB = sA + size_t(s) * ld;
  C* sC = sB + size_t(s) * ld;
  C* sD = sC + size_t(s) * ld;
  uint32_t* own = reinterpret_cast<uint32_t*>(sD + size_t(s) * ld);
  TileGeom g{block_start<MAPPED>(k0, n, s, blk), block_start<MAPPED>(k0 + nb, n, s, blk), s, magic, ld, own};
  BlockInfo bi{0, 0, false, false};
  if (t < nb) bi = block_info<MAPPED>(k0 + t, n, s, m, blk);
  if constexpr (MAPPED) {
    if (t < nb) fill_owner(own, t, int(bi.start - g.ts), bi.len);
    __syncthreads();
  }
  int jb = 0;
  if (!MAPPED && off && t < 32) jb = warp_lower_bound(off, 1, nsys, g.ts);  // batch solved as one system
  {
    const S* src[4] = {a, b, c, d};
    C* dst[4] = {sA, sB, sC, sD};
    tile_load<S, C, MAPPED, 4>(g, src, dst, n);
  }
  __syncthreads();
  if (!MAPPED && off) {
    if (t < 32) tile_cut<C>(g, off, nsys, jb, sA, sC, nullptr, nullptr);
    __syncthreads();
  }
  if (t < nb) {
    IfaceRows r;
    if constexpr (std::is_same<C, float>::value && !KEEP)
      r = lean_reduce(sA + t, sB + t, sC + t, sD + t, ld, bi, status);
    else
      r = block_reduce<C, C, KEEP>(sA + t, sB + t, sC + t, sD + t, ld, bi, status);
    write_iface(k0 + t, r, ra, rb, rc, rd);
  }
  if constexpr (KEEP) {
    __syncthreads();
    const C* src[3] = {sA, sC, sD};
    C* dst[3] = {oa, og, od};
    tile_store<C, C, MAPPED, 3>(g, src, dst);
  }
}

// ---------------------------------------------------------------------------
// Stage 3 from the kept coefficients: x = delta' - alpha' yL - gamma' yR,
// elementwise (no sequential dependence left).
// ---------------------------------------------------------------------------
template <typename C, typename S, bool MAPPED>
__global__ void __launch_bounds__(256) k_stage3_kept(const C* __restrict__ ka, const C* __restrict__ kg,
                                                     const C* __restrict__ kd, int64_t n, int s, unsigned magic,
                                                     int64_t m, const int64_t* __restrict__ blk,
                                                     const double* __restrict__ y, S* __restrict__ x, int64_t kb,
                                                     int64_t ke) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x, t = threadIdx.x;
  const int64_t k0 = kb + int64_t(blockIdx.x) * T;  // blocks [kb, ke) of the m
  if (k0 >= ke) return;
  const int nb = int(min(int64_t(T), ke - k0));
  C* yl = reinterpret_cast<C*>(smem);
  C* yr = yl + T;
  uint32_t* own = reinterpret_cast<uint32_t*>(yr + T);
  TileGeom g{block_start<MAPPED>(k0, n, s, blk), block_start<MAPPED>(k0 + nb, n, s, blk), s, magic, 0, own};
  if (t < nb) {
    const double2 v = *reinterpret_cast<const double2*>(y + 2 * (k0 + t));
    yl[t] = cvt<C>(v.x);
    yr[t] = cvt<C>(v.y);
    if constexpr (MAPPED) {
      const BlockInfo bi = block_info<MAPPED>(k0 + t, n, s, m, blk);
      fill_owner(own, t, int(bi.start - g.ts), bi.len);
    }
  }
  __syncthreads();
  constexpr int V = Vec<C>::W;
  const int64_t q0 = g.ts / V, q1 = (g.te + V - 1) / V;
  for (int64_t q = q0 + t; q < q1; q += T) {
    const int64_t base = q * V;
    Vec<C> va, vg, vd;
    const bool full = base >= g.ts && base + V <= g.te;
    if (full) {
      va = ldcs16<C>(ka + base); vg = ldcs16<C>(kg + base); vd = ldcs16<C>(kd + base);
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const int64_t pg = base + e;
        const bool in = pg >= g.ts && pg < g.te;
        va.v[e] = in ? ka[pg] : C(0); vg.v[e] = in ? kg[pg] : C(0); vd.v[e] = in ? kd[pg] : C(0);
      }
    }
    Vec<S> vx;
#pragma unroll
    for (int e = 0; e < V && e < Vec<S>::W; ++e) vx.v[e] = S(0);
    C xv[V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const int64_t pg = base + e;
      int tt = 0, j = 0;
      if (pg >= g.ts && pg < g.te) owner<MAPPED>(g, int(pg - g.ts), tt, j);
      xv[e] = fma(-vg.v[e], yr[tt], fma(-va.v[e], yl[tt], vd.v[e]));
    }
    if (full && sizeof(S) == sizeof(C)) {
#pragma unroll
      for (int e = 0; e < V; ++e) vx.v[e] = cvt<S>(xv[e]);
      stg16<S>(x + base, vx);
    } else if (full && sizeof(S) == 2 * sizeof(C)) {  // binary32 chunk -> two binary64 chunks
#pragma unroll
      for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int e = 0; e < Vec<S>::W; ++e) vx.v[e] = cvt<S>(xv[h * Vec<S>::W + e]);
        stg16<S>(x + base + h * Vec<S>::W, vx);
      }
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const int64_t pg = base + e;
        if (pg >= g.ts && pg < g.te) x[pg] = cvt<S>(xv[e]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Stage 3 by repeating the interior solve (re-reads a, b, c, d).
// ---------------------------------------------------------------------------
template <typename S, typename C, bool MAPPED>
__global__ void __launch_bounds__(256) k_stage3_resolve(const S* __restrict__ a, const S* __restrict__ b,
                                                        const S* __restrict__ c, const S* __restrict__ d, int64_t n,
                                                        int s, unsigned magic, int64_t m,
                                                        const int64_t* __restrict__ blk,
                                                        const double* __restrict__ y, S* __restrict__ x,
                                                        unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x, ld = T + 1, t = threadIdx.x;
  const int64_t k0 = int64_t(blockIdx.x) * T;
  if (k0 >= m) return;
  const int nb = int(min(int64_t(T), m - k0));
  C* sA = reinterpret_cast<C*>(smem);
  C* sB = sA + size_t(s) * ld;
  C* sC = sB + size_t(s) * ld;
  C* sD = sC + size_t(s) * ld;
  uint32_t* own = reinterpret_cast<uint32_t*>(sD + size_t(s) * ld);
  TileGeom g{block_start<MAPPED>(k0, n, s, blk), block_start<MAPPED>(k0 + nb, n, s, blk), s, magic, ld, own};
  BlockInfo bi{0, 0, false, false};
  if (t < nb) bi = block_info<MAPPED>(k0 + t, n, s, m, blk);
  if constexpr (MAPPED) {
    if (t < nb) fill_owner(own, t, int(bi.start - g.ts), bi.len);
    __syncthreads();
  }
  {
    const S* src[4] = {a, b, c, d};
    C* dst[4] = {sA, sB, sC, sD};
    tile_load<S, C, MAPPED, 4>(g, src, dst, n);
  }
  __syncthreads();
  if (t < nb) {
    const double2 v = *reinterpret_cast<const double2*>(y + 2 * (k0 + t));
    if constexpr (std::is_same<C, float>::value)
      lean_substitute(sA + t, sB + t, sC + t, sD + t, sC + t, ld, bi.len, cvt<C>(v.x), cvt<C>(v.y), status);
    else
      block_substitute<C, C>(sA + t, sB + t, sC + t, sD + t, ld, bi.len, cvt<C>(v.x), cvt<C>(v.y), status);
  }
  __syncthreads();
  {
    const C* src[1] = {sD};
    S* dst[1] = {x};
    tile_store<C, S, MAPPED, 1>(g, src, dst);
  }
}

// ---------------------------------------------------------------------------
// Small systems: sequential Thomas by one thread per system.  Used for the
// last level of the interface-system recursion and as the plain GPU Thomas
// baseline (K0).  System j: rows base_j + i*es, i < len_j; either contiguous
// offsets (off != nullptr) or uniform strided systems.
// ---------------------------------------------------------------------------
template <typename S, typename C>
__global__ void __launch_bounds__(128) k_thomas(const S* __restrict__ a, const S* __restrict__ b,
                                                const S* __restrict__ c, const S* __restrict__ d, S* __restrict__ x,
                                                const int64_t* __restrict__ off, int32_t batch, int64_t n_uniform,
                                                int64_t sys_stride, int64_t es, int64_t n_total,
                                                C* __restrict__ scratch, unsigned* __restrict__ status) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= batch) return;
  int64_t base, len;
  if (off) {
    base = off[j];
    len = off[j + 1] - base;
    if (base < 0 || len < 0 || base + len > n_total) {  // offsets out of range: touch nothing
      flag(status, ST_BADARG);
      return;
    }
  } else {
    base = j * sys_stride;
    len = n_uniform;
  }
  if (len <= 0) return;
  // forward sweep: x[i] temporarily holds delta_i, scratch holds gamma_i
  C gam = C(0), del = C(0);
  for (int64_t i = 0; i < len; ++i) {
    const int64_t p = base + i * es;
    const C ai = (i == 0) ? C(0) : cvt<C>(a[p]);
    const C bi = cvt<C>(b[p]);
    const C ci = (i == len - 1) ? C(0) : cvt<C>(c[p]);
    const C di = cvt<C>(d[p]);
    const C r = rcp(fma(-ai, gam, bi), status);
    del = fma(-ai * r, del, di * r);
    gam = ci * r;
    scratch[p] = gam;
    x[p] = cvt<S>(del);
  }
  C xn = del;
  for (int64_t i = len - 2; i >= 0; --i) {
    const int64_t p = base + i * es;
    xn = fma(-scratch[p], xn, cvt<C>(x[p]));
    x[p] = cvt<S>(xn);
  }
}

}  // namespace tdp
