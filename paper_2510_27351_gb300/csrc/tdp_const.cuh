// Constant-coefficient systems: every row of every system has the same
// sub-diagonal a, diagonal b and super-diagonal c (a of a system's first row
// and c of its last row are ignored), as in the implicit steps of the heat
// equation.  Only d is read and x written.
//
// The partition method needs, for each block, the forward factors of Stage 1
// (reciprocal pivots r_j, multipliers q_j = a r_j, gam_j = c r_j and the
// spike coefficients alp_j) and the backward primes (ap_j, gp_j) of its
// interior.  With constant coefficients they do not depend on d nor on the
// block: one table per sub-system size s serves every full block (the forward
// factors of a shorter last block are a prefix of the table; its primes are
// computed on the fly).  Per row what is left is the d-part of the
// recurrences:
//   Stage 1:  del_j = r_j d_j - q_j del_{j-1}  (forward),
//             dp_j  = del_j - gam_j dp_{j+1}   (backward, row 1 gives the L row),
//   Stage 3:  the same two recurrences, then x_j = dp_j - ap_j x_L - gp_j x_R.
// A thread owns one block and walks its rows through the strides directly:
// consecutive threads take the same block of consecutive systems when the
// systems are interleaved (elem_stride != 1), so every row access is
// coalesced; with contiguous systems consecutive threads take consecutive
// blocks.  The forward values wait in shared memory for the backward pass.
#pragma once
#include "tdp_kernels.cuh"

namespace tdp {

// Table of one block of s rows: planes r, q, gam, alp (rows 1..s-1) and ap,
// gp (rows 1..s-2), each s entries.
template <typename C>
struct ConstTab {
  const C *r, *q, *gam, *alp, *ap, *gp;
  __device__ __forceinline__ ConstTab(const C* t, int s)
      : r(t), q(t + s), gam(t + 2 * s), alp(t + 3 * s), ap(t + 4 * s), gp(t + 5 * s) {}
};

// One thread builds the table (the forward recurrence of Stage 1 on the
// coefficient part, then the backward primes), in C.
template <typename C>
__global__ void k_const_table(double a_, double b_, double c_, int s, C* __restrict__ t,
                              unsigned* __restrict__ status) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const C a = cvt<C>(a_), b = cvt<C>(b_), c = cvt<C>(c_);
  C* r = t;
  C* q = t + s;
  C* gam = t + 2 * s;
  C* alp = t + 3 * s;
  C* ap = t + 4 * s;
  C* gp = t + 5 * s;
  for (int i = 0; i < 6 * s; ++i) t[i] = C(0);
  C g = C(0), al = C(-1);
  for (int j = 1; j < s; ++j) {
    const C rj = rcp(fma(-a, g, b), status);
    const C qj = a * rj;
    g = c * rj;
    al = -qj * al;
    r[j] = rj; q[j] = qj; gam[j] = g; alp[j] = al;
  }
  if (s >= 3) {
    C pa = alp[s - 2], pg = gam[s - 2];
    ap[s - 2] = pa; gp[s - 2] = pg;
    for (int j = s - 3; j >= 1; --j) {
      pa = fma(-gam[j], pa, alp[j]);
      pg = -gam[j] * pg;
      ap[j] = pa; gp[j] = pg;
    }
  }
}

// Block of thread `gid`: system j, block k, rows [k s, k s + len) of the system.
struct ConstBlock {
  int64_t j, k, base;  // base: index of the block's first row
  int len;
  bool first, last;
};

__device__ __forceinline__ bool const_block(int64_t gid, int32_t batch, int64_t n, int s, int64_t mps, int64_t ss,
                                            int64_t es, ConstBlock& cb) {
  if (gid >= int64_t(batch) * mps) return false;
  if (es != 1) {  // interleaved systems: system index fastest
    cb.j = gid % batch;
    cb.k = gid / batch;
  } else {
    cb.j = gid / mps;
    cb.k = gid % mps;
  }
  const int64_t r0 = cb.k * s;
  cb.len = int(min(int64_t(s), n - r0));
  cb.base = cb.j * ss + r0 * es;
  cb.first = cb.k == 0;
  cb.last = cb.k == mps - 1;
  return true;
}

// Stage 1: interface rows of every block (interface rows of system j, block k
// at 2 (j mps + k)).  S storage, C arithmetic.
template <typename S, typename C>
__global__ void __launch_bounds__(128) k_const_stage1(double a_, double b_, double c_, const C* __restrict__ tab,
                                                      const S* __restrict__ d, int64_t n, int32_t batch, int s,
                                                      int64_t mps, int64_t ss, int64_t es, double* __restrict__ ra,
                                                      double* __restrict__ rb, double* __restrict__ rc,
                                                      double* __restrict__ rd, unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  C* dl = reinterpret_cast<C*>(smem) + threadIdx.x;  // forward values, row j at dl[j * blockDim.x]
  const int T = blockDim.x;
  ConstBlock cb;
  const int64_t gid = int64_t(blockIdx.x) * T + threadIdx.x;
  if (!const_block(gid, batch, n, s, mps, ss, es, cb)) return;
  const ConstTab<C> tb(tab, s);
  const C a = cvt<C>(a_), b = cvt<C>(b_), c = cvt<C>(c_);
  const int len = cb.len;
  const S* pd = d + cb.base;
  IfaceRows out;
  const C d0 = cvt<C>(pd[0]);
  const C a0 = cb.first ? C(0) : a;
  if (len == 1) {
    out = IfaceRows{to_f64(a0), to_f64(b), cb.last ? 0.0 : to_f64(c), to_f64(d0), 0.0, 1.0, 0.0, 0.0};
  } else {
    C del = C(0);
    for (int j = 1; j < len; ++j) {
      del = fma(-tb.q[j], del, cvt<C>(pd[j * es]) * tb.r[j]);
      dl[j * T] = del;
    }
    out.a1 = to_f64(tb.alp[len - 1]);
    out.b1 = 1.0;
    out.c1 = cb.last ? 0.0 : to_f64(tb.gam[len - 1]);
    out.d1 = to_f64(del);
    C ap = C(0), gp = C(-1), dp = C(0);
    if (len >= 3) {
      dp = dl[(len - 2) * T];
      if (len == s) {
        for (int j = len - 3; j >= 1; --j) dp = fma(-tb.gam[j], dp, dl[j * T]);
        ap = tb.ap[1];
        gp = tb.gp[1];
      } else {  // shorter last block: its primes start at row len-2
        ap = tb.alp[len - 2];
        gp = tb.gam[len - 2];
        for (int j = len - 3; j >= 1; --j) {
          const C g = tb.gam[j];
          dp = fma(-g, dp, dl[j * T]);
          ap = fma(-g, ap, tb.alp[j]);
          gp = -g * gp;
        }
      }
    }
    out.a0 = to_f64(a0);
    out.b0 = to_f64(fma(-c, ap, b));
    out.c0 = to_f64(-c * gp);
    out.d0 = to_f64(fma(-c, dp, d0));
  }
  write_iface(cb.j * mps + cb.k, out, ra, rb, rc, rd);
}

// Stage 3 by repeating the d-part of Stage 1 with the interface values y known.
template <typename S, typename C>
__global__ void __launch_bounds__(128) k_const_stage3(const C* __restrict__ tab, const S* __restrict__ d,
                                                      S* __restrict__ x, int64_t n, int32_t batch, int s,
                                                      int64_t mps, int64_t ss, int64_t es,
                                                      const double* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smem[];
  C* dl = reinterpret_cast<C*>(smem) + threadIdx.x;
  const int T = blockDim.x;
  ConstBlock cb;
  const int64_t gid = int64_t(blockIdx.x) * T + threadIdx.x;
  if (!const_block(gid, batch, n, s, mps, ss, es, cb)) return;
  const ConstTab<C> tb(tab, s);
  const int len = cb.len;
  const S* pd = d + cb.base;
  S* px = x + cb.base;
  const double2 yv = *reinterpret_cast<const double2*>(y + 2 * (cb.j * mps + cb.k));
  const C yl = cvt<C>(yv.x), yr = cvt<C>(yv.y);
  px[0] = cvt<S>(yl);
  if (len == 1) return;
  px[(len - 1) * es] = cvt<S>(yr);
  if (len == 2) return;
  C del = C(0);
  for (int j = 1; j < len - 1; ++j) {
    del = fma(-tb.q[j], del, cvt<C>(pd[j * es]) * tb.r[j]);
    dl[j * T] = del;
  }
  // x_j = dp_j - ap_j yl - gp_j yr, rows len-2 .. 1
  C dp = dl[(len - 2) * T];
  C ap = (len == s) ? tb.ap[len - 2] : tb.alp[len - 2];
  C gp = (len == s) ? tb.gp[len - 2] : tb.gam[len - 2];
  px[(len - 2) * es] = cvt<S>(fma(-gp, yr, fma(-ap, yl, dp)));
  for (int j = len - 3; j >= 1; --j) {
    const C g = tb.gam[j];
    dp = fma(-g, dp, dl[j * T]);
    if (len == s) {
      ap = tb.ap[j];
      gp = tb.gp[j];
    } else {
      ap = fma(-g, ap, tb.alp[j]);
      gp = -g * gp;
    }
    px[j * es] = cvt<S>(fma(-gp, yr, fma(-ap, yl, dp)));
  }
}


}  // namespace tdp
