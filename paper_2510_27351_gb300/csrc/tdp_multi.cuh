// Many right-hand sides with one matrix: A X = D for nrhs columns.
//
// Every quantity of the partition method except the d-parts depends on the
// matrix alone: the reciprocal pivots r_j, multipliers q_j = a_j r_j and
// gam_j = c_j r_j of Stage 1's downward sweep, the spike and backward
// coefficients alpha'_j, gamma'_j that Stage 3 applies to x_L and x_R, and the
// interface matrix (Sec. I).  k_multi_factor computes them once, in the
// arithmetic of block_reduce; per right-hand side only the d-part recurrences
// are left (Stage 1: del_j = r_j d_j - q_j del_{j-1}, dp_j = del_j -
// gam_j dp_{j+1}; Stage 3: x_j = dp_j - alpha'_j x_L - gamma'_j x_R), five
// operations per row instead of fourteen, plus one interface solve.
#pragma once
#include "tdp_kernels.cuh"

namespace tdp {

// Matrix part, one block per thread on a shared-memory tile of a, b, c (row
// j of the block of thread t at j * (T + 1) + t).  The downward-sweep factors
// r, q, g go to global memory TRANSPOSED (row j of block k at j * m + k), so
// that the per-right-hand-side sweeps, whose threads take consecutive blocks,
// read them coalesced; the Stage 3 coefficients ap, gp go out in row order
// (rows 0 and len-1 of a block encode x_L and x_R themselves: (ap, gp) =
// (-1, 0) and (0, -1)).  The interface matrix rows go to ra, rb, rc.
template <typename S, typename C>
__global__ void __launch_bounds__(256) k_multi_factor(const S* __restrict__ a, const S* __restrict__ b,
                                                      const S* __restrict__ c, int64_t n, int s, unsigned magic,
                                                      int64_t m, C* __restrict__ rT, C* __restrict__ qT,
                                                      C* __restrict__ gT, C* __restrict__ ap, C* __restrict__ gp,
                                                      double* __restrict__ ra, double* __restrict__ rb,
                                                      double* __restrict__ rc, unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x, ld = T + 1, t = threadIdx.x;
  const int64_t k0 = int64_t(blockIdx.x) * T;
  if (k0 >= m) return;
  const int nb = int(min(int64_t(T), m - k0));
  C* sA = reinterpret_cast<C*>(smem);
  C* sB = sA + size_t(s) * ld;
  C* sC = sB + size_t(s) * ld;
  const TileGeom g{k0 * s, min(n, (k0 + nb) * s), s, magic, ld, nullptr};
  {
    const S* src[3] = {a, b, c};
    C* dst[3] = {sA, sB, sC};
    tile_load<S, C, false, 3>(g, src, dst, n);
  }
  __syncthreads();
  if (t < nb) {
    const int64_t k = k0 + t, L = k * s;
    const int len = int(min(int64_t(s), n - L));
    const bool first = k == 0, last = k == m - 1;
    C* pa = sA + t;  // a -> alpha -> ap
    C* pb = sB + t;  // b -> gamma
    C* pc = sC + t;  // c -> gp
    const C a0 = first ? C(0) : pa[0], b0 = pb[0], c0 = pc[0];
    if (len == 1) {
      pa[0] = C(-1);
      pc[0] = C(0);
      *reinterpret_cast<double2*>(ra + 2 * k) = make_double2(to_f64(a0), 0.0);
      *reinterpret_cast<double2*>(rb + 2 * k) = make_double2(to_f64(b0), 1.0);
      *reinterpret_cast<double2*>(rc + 2 * k) = make_double2(last ? 0.0 : to_f64(c0), 0.0);
    } else {
      // downward sweep, rows 1..len-1 (alpha kept in the a row, gamma in the b row)
      C gam = C(0), alp = C(0);
      for (int j = 1; j < len; ++j) {
        const C aj = pa[j * ld], bj = pb[j * ld];
        const C cj = (j == len - 1 && last) ? C(0) : pc[j * ld];
        const C rj = rcp(j == 1 ? bj : fma(-aj, gam, bj), status);
        const C qj = aj * rj;
        alp = j == 1 ? qj : -qj * alp;
        gam = cj * rj;
        rT[int64_t(j) * m + k] = rj;
        qT[int64_t(j) * m + k] = qj;
        gT[int64_t(j) * m + k] = gam;
        pa[j * ld] = alp;
        pb[j * ld] = gam;
      }
      const C r1a = alp, r1c = gam;
      // backward over the interior rows len-2 .. 1: alpha' into the a row, gamma' into the c row
      C apv = C(0), gpv = C(-1);
      if (len >= 3) {
        apv = pa[(len - 2) * ld];
        gpv = pb[(len - 2) * ld];
        pc[(len - 2) * ld] = gpv;
        for (int j = len - 3; j >= 1; --j) {
          const C gj = pb[j * ld];
          apv = fma(-gj, apv, pa[j * ld]);
          gpv = -gj * gpv;
          pa[j * ld] = apv;
          pc[j * ld] = gpv;
        }
      }
      pa[0] = C(-1);
      pc[0] = C(0);
      pa[(len - 1) * ld] = C(0);
      pc[(len - 1) * ld] = C(-1);
      *reinterpret_cast<double2*>(ra + 2 * k) = make_double2(to_f64(a0), to_f64(r1a));
      *reinterpret_cast<double2*>(rb + 2 * k) = make_double2(to_f64(fma(-c0, apv, b0)), 1.0);
      *reinterpret_cast<double2*>(rc + 2 * k) = make_double2(to_f64(-c0 * gpv), to_f64(r1c));
    }
  }
  __syncthreads();
  const C* src[2] = {sA, sC};
  C* dst[2] = {ap, gp};
  tile_store<C, C, false, 2>(g, src, dst);
}

// d-part of Stage 1 for the T blocks of one CTA and right-hand side
// blockIdx.y: the column's rows staged in shared memory (coalesced), the
// factors read transposed (coalesced), delta and then dp kept in the tile, dp
// stored to the column of x (rows 0 and len-1 of a block get 0), the
// interface right-hand sides to rd + column * 2m.  (Looping several columns
// inside a CTA to reuse its factors from cache measured slower.)
template <typename S, typename C>
__global__ void __launch_bounds__(256) k_multi_reduce(const C* __restrict__ rT, const C* __restrict__ qT,
                                                      const C* __restrict__ gT, const S* __restrict__ c,
                                                      const S* __restrict__ d, int64_t ldd, S* __restrict__ x,
                                                      int64_t ldx, int64_t n, int s, unsigned magic, int64_t m,
                                                      double* __restrict__ rd) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x, ld = T + 1, t = threadIdx.x;
  const int64_t k0 = int64_t(blockIdx.x) * T, jr = blockIdx.y;
  if (k0 >= m) return;
  const int nb = int(min(int64_t(T), m - k0));
  C* sD = reinterpret_cast<C*>(smem);
  const TileGeom g{k0 * s, min(n, (k0 + nb) * s), s, magic, ld, nullptr};
  {
    const S* src[1] = {d + jr * ldd};
    C* dst[1] = {sD};
    tile_load<S, C, false, 1>(g, src, dst, n);
  }
  __syncthreads();
  if (t < nb) {
    const int64_t k = k0 + t, L = k * s;
    const int len = int(min(int64_t(s), n - L));
    double* rdj = rd + jr * 2 * m;
    C* pd = sD + t;
    const C d0 = pd[0];
    pd[0] = C(0);
    if (len == 1) {
      *reinterpret_cast<double2*>(rdj + 2 * k) = make_double2(to_f64(d0), 0.0);
    } else {
      C del = C(0);
      for (int j = 1; j < len; ++j) {
        const int64_t f = int64_t(j) * m + k;
        del = j == 1 ? pd[j * ld] * rT[f] : fma(-qT[f], del, pd[j * ld] * rT[f]);
        pd[j * ld] = del;
      }
      const C r1d = del;
      C dp = C(0);
      if (len >= 3) {
        dp = pd[(len - 2) * ld];
        for (int j = len - 3; j >= 1; --j) {
          dp = fma(-gT[int64_t(j) * m + k], dp, pd[j * ld]);
          pd[j * ld] = dp;
        }
      }
      pd[(len - 1) * ld] = C(0);
      const C c0 = cvt<C>(c[L]);
      *reinterpret_cast<double2*>(rdj + 2 * k) = make_double2(to_f64(fma(-c0, dp, d0)), to_f64(r1d));
    }
  }
  __syncthreads();
  const C* src[1] = {sD};
  S* dst[1] = {x + jr * ldx};
  tile_store<C, S, false, 1>(g, src, dst);
}

// Stage 3 of every right-hand side, elementwise and in place:
// x_i = dp_i - alpha'_i yL - gamma'_i yR (rows 0 and len-1 of a block give yL,
// yR through their encoded coefficients and dp = 0).  (A tiled form with the
// block index from shared memory and 16-byte vectors measured slower.)
template <typename S, typename C>
__global__ void __launch_bounds__(256) k_multi_stage3(const C* __restrict__ ap, const C* __restrict__ gp, S* x,
                                                      int64_t ldx, int64_t n, int s, int64_t m, int32_t nrhs,
                                                      const double* __restrict__ y) {
  const int64_t total = n * nrhs;
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < total; q += int64_t(gridDim.x) * blockDim.x) {
    const int64_t jr = q / n, i = q - jr * n, k = i / s;
    const double2 yv = *reinterpret_cast<const double2*>(y + jr * 2 * m + 2 * k);
    S* xi = x + jr * ldx + i;
    const C v = fma(-gp[i], cvt<C>(yv.y), fma(-ap[i], cvt<C>(yv.x), cvt<C>(*xi)));
    *xi = cvt<S>(v);
  }
}

// nrhs copies of the interface matrix, one after another (the copies are
// decoupled: a copy's first row has a = 0 and its last row c = 0).
__global__ void k_multi_replicate(const double* __restrict__ ra, const double* __restrict__ rb,
                                  const double* __restrict__ rc, int64_t M, int32_t nrhs, double* __restrict__ A,
                                  double* __restrict__ B, double* __restrict__ Cc) {
  const int64_t total = M * nrhs;
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < total; q += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = q % M;
    A[q] = ra[i];
    B[q] = rb[i];
    Cc[q] = rc[i];
  }
}

}  // namespace tdp
