// The small levels of the interface recursion in ONE cooperative launch.
//
// Below a few hundred thousand rows the recursive interface solve (Sec. III)
// is bound by latency, not bandwidth: every level is a chain of dependent
// binary64 operations per block plus a kernel launch.  Here all remaining
// levels run in a single kernel whose CTAs are co-resident (cooperative
// launch) and meet at a grid barrier between levels:
//   down:  Stage 1 of every level (one thread per block, rows read straight
//          from L2 with a one-row lookahead), keeping (alpha', gamma',
//          delta') and writing the next interface system;
//   base:  one thread runs Thomas on the last (<= 64-row) system;
//   up:    Stage 3 of every level, elementwise.
// The barrier is a counter and a generation word in global memory; every
// wait is bounded (about a second), after which the kernel raises ST_TIMEOUT
// and returns.
#pragma once
#include "tdp_device.cuh"

namespace tdp {

constexpr int kCoopMaxLevels = 12;

struct CoopLevel {
  const double *a, *b, *c, *d;  // this level's system (M rows)
  double *ka, *kg, *kd;         // kept coefficients (M rows)
  double *na, *nb, *nc, *nd;    // next level's system (2m rows)
  double* y;                    // this level's solution (M rows)
  int64_t M, m;
  int s;
};

struct CoopParams {
  CoopLevel lv[kCoopMaxLevels];
  int L;                 // number of levels
  int reg;               // 1: blocks of 8 rows through registers (coop_block_reduce_reg)
  double* base_scratch;  // Thomas scratch for the last system
  double* ybase;         // solution of the last system (2 * lv[L-1].m rows)
  long long wait_cycles; // a barrier wait gives up after this many clock cycles
  unsigned bar_extra;    // arrivals a barrier waits for beyond the grid (0; 1 only to test the timeout)
};

// Grid-wide barrier.  bar[0] counts arrivals, bar[1] is the generation.  The
// wait is bounded: after wait_cycles clock cycles the CTA raises ST_TIMEOUT
// and every thread of it gets false (the kernel then returns).  With extra =
// 1 the barrier waits for one arrival more than the grid has, so that it can
// never complete (used only to test the timeout path).
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned* status, long long wait_cycles,
                                             unsigned extra) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1 + extra) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (clock64() - t0 > wait_cycles) {
          flag(status, ST_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  return __syncthreads_and(ok) != 0;
}

// Parallel cyclic reduction of a system of M <= 64 rows by one warp (the
// last interface system): lane l holds rows l and l + 32; every step h =
// 1, 2, .., 32 eliminates the couplings to rows i - h and i + h (neighbour
// rows read with shuffles), after which x_i = d_i / b_i.  Rows beyond M are
// identity rows.  All 32 lanes must call it.
__device__ __forceinline__ void warp_pcr64(const double* a, const double* b, const double* c, const double* d,
                                           double* y, int M, unsigned* status) {
  const int l = threadIdx.x & 31;
  double A[2], B[2], C[2], Dv[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = l + 32 * h;
    const bool in = i < M;
    A[h] = (in && i > 0) ? a[i] : 0.0;
    B[h] = in ? b[i] : 1.0;
    C[h] = (in && i < M - 1) ? c[i] : 0.0;
    Dv[h] = in ? d[i] : 0.0;
  }
#pragma unroll
  for (int hs = 1; hs <= 32; hs <<= 1) {
    const int up = (l - hs) & 31, dn = (l + hs) & 31;
    double ua[2], ub[2], uc[2], ud[2], wa[2], wb[2], wc[2], wd[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      ua[h] = __shfl_sync(0xffffffffu, A[h], up); ub[h] = __shfl_sync(0xffffffffu, B[h], up);
      uc[h] = __shfl_sync(0xffffffffu, C[h], up); ud[h] = __shfl_sync(0xffffffffu, Dv[h], up);
      wa[h] = __shfl_sync(0xffffffffu, A[h], dn); wb[h] = __shfl_sync(0xffffffffu, B[h], dn);
      wc[h] = __shfl_sync(0xffffffffu, C[h], dn); wd[h] = __shfl_sync(0xffffffffu, Dv[h], dn);
    }
    double nA[2], nB[2], nC[2], nD[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      // row i = l + 32 h; its upper neighbour i - hs and lower neighbour i + hs
      const int i = l + 32 * h;
      const int iu = i - hs, iw = i + hs;
      const int hu = (iu >= 0) ? (iu >> 5) : 0, hw = (iw < 64) ? (iw >> 5) : 0;
      const bool vu = iu >= 0, vw = iw < 64;
      const double Au = hu ? ua[1] : ua[0], Bu = hu ? ub[1] : ub[0], Cu = hu ? uc[1] : uc[0],
                   Du = hu ? ud[1] : ud[0];
      const double Aw = hw ? wa[1] : wa[0], Bw = hw ? wb[1] : wb[0], Cw = hw ? wc[1] : wc[0],
                   Dw = hw ? wd[1] : wd[0];
      const double k1 = vu ? A[h] * rcp(Bu, status) : 0.0;
      const double k2 = vw ? C[h] * rcp(Bw, status) : 0.0;
      nA[h] = vu ? -k1 * Au : 0.0;
      nC[h] = vw ? -k2 * Cw : 0.0;
      nB[h] = B[h] - (vu ? k1 * Cu : 0.0) - (vw ? k2 * Aw : 0.0);
      nD[h] = Dv[h] - (vu ? k1 * Du : 0.0) - (vw ? k2 * Dw : 0.0);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) { A[h] = nA[h]; B[h] = nB[h]; C[h] = nC[h]; Dv[h] = nD[h]; }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = l + 32 * h;
    if (i < M) y[i] = Dv[h] * rcp(B[h], status);
  }
}

// A system of at most 64 rows solved by one warp (launch with 32 threads).
__global__ void __launch_bounds__(32) k_base_pcr(const double* __restrict__ a, const double* __restrict__ b,
                                                 const double* __restrict__ c, const double* __restrict__ d,
                                                 double* __restrict__ y, int M, unsigned* __restrict__ status) {
  warp_pcr64(a, b, c, d, y, M, status);
}

// Stage 1 of one block read from global memory; forward values go to the
// kept arrays and are replaced by the primes of the backward pass.
__device__ __forceinline__ void coop_block_reduce(const CoopLevel& D, int64_t k, unsigned* status) {
  const int64_t L = k * D.s;
  const int len = int(min(int64_t(D.s), D.M - L));
  const bool first = (k == 0), last = (k == D.m - 1);
  const double* a = D.a + L;
  const double* b = D.b + L;
  const double* c = D.c + L;
  const double* d = D.d + L;
  double* ka = D.ka + L;
  double* kg = D.kg + L;
  double* kd = D.kd + L;
  double a0 = first ? 0.0 : a[0], b0 = b[0], c0 = c[0], d0 = d[0];
  double r0a, r0b, r0c, r0d, r1a = 0.0, r1b = 1.0, r1c = 0.0, r1d = 0.0;
  if (len == 1) {
    if (last) c0 = 0.0;
    r0a = a0; r0b = b0; r0c = c0; r0d = d0;
    ka[0] = -1.0; kg[0] = 0.0; kd[0] = 0.0;
  } else {
    double gam = 0.0, del = 0.0, alp = 0.0;
    double na = a[1], nb = b[1], nc = c[1], nd = d[1];
    for (int j = 1; j < len; ++j) {
      const double aj = na, bj = nb, dj = nd;
      double cj = nc;
      if (j + 1 < len) { na = a[j + 1]; nb = b[j + 1]; nc = c[j + 1]; nd = d[j + 1]; }
      if (j == len - 1 && last) cj = 0.0;
      if (j == 1) {
        const double r = rcp(bj, status);
        gam = cj * r; del = dj * r; alp = aj * r;
      } else {
        const double r = rcp(fma(-aj, gam, bj), status);
        const double q = aj * r;
        gam = cj * r;
        del = fma(-q, del, dj * r);
        alp = -q * alp;
      }
      ka[j] = alp; kg[j] = gam; kd[j] = del;
    }
    r1a = alp; r1b = 1.0; r1c = gam; r1d = del;
    double ap, gp, dp;
    if (len == 2) {
      ap = 0.0; gp = -1.0; dp = 0.0;
    } else {
      ap = ka[len - 2]; gp = kg[len - 2]; dp = kd[len - 2];
      double pa = ka[len - 3], pg = kg[len - 3], pd = kd[len - 3];
      for (int j = len - 3; j >= 1; --j) {
        const double aj = pa, gj = pg, dj = pd;
        if (j > 1) { pa = ka[j - 1]; pg = kg[j - 1]; pd = kd[j - 1]; }
        dp = fma(-gj, dp, dj);
        ap = fma(-gj, ap, aj);
        gp = -gj * gp;
        ka[j] = ap; kg[j] = gp; kd[j] = dp;
      }
    }
    r0a = a0; r0b = fma(-c0, ap, b0); r0c = -c0 * gp; r0d = fma(-c0, dp, d0);
    ka[0] = -1.0; kg[0] = 0.0; kd[0] = 0.0;
    ka[len - 1] = 0.0; kg[len - 1] = -1.0; kd[len - 1] = 0.0;
  }
  *reinterpret_cast<double2*>(D.na + 2 * k) = make_double2(r0a, r1a);
  *reinterpret_cast<double2*>(D.nb + 2 * k) = make_double2(r0b, r1b);
  *reinterpret_cast<double2*>(D.nc + 2 * k) = make_double2(r0c, r1c);
  *reinterpret_cast<double2*>(D.nd + 2 * k) = make_double2(r0d, r1d);
}

// The same for a block of 3 <= len <= S rows held in registers: every load is
// issued before the first use (one L2 round trip per block instead of one
// per row), the backward pass reads the forward values from registers, and a
// full block's kept coefficients leave as 16-byte stores.  Loops run over all
// S rows with the rows past len masked, so that a ragged last block takes the
// same code path as its warp's full blocks.  The level's arrays must be
// 16-byte aligned (arena buffers are).
template <int S>
__device__ __forceinline__ void coop_block_reduce_reg(const CoopLevel& D, int64_t k, int len, unsigned* status) {
  static_assert(S >= 4 && S % 2 == 0, "even block size of at least 4");
  const int64_t L = k * S;
  const bool first = (k == 0), last = (k == D.m - 1), full = (len == S);
  double a[S], b[S], c[S], d[S];
  if (full) {
#pragma unroll
    for (int j = 0; j < S; j += 2) {
      const double2 va = *reinterpret_cast<const double2*>(D.a + L + j);
      const double2 vb = *reinterpret_cast<const double2*>(D.b + L + j);
      const double2 vc = *reinterpret_cast<const double2*>(D.c + L + j);
      const double2 vd = *reinterpret_cast<const double2*>(D.d + L + j);
      a[j] = va.x; a[j + 1] = va.y; b[j] = vb.x; b[j + 1] = vb.y;
      c[j] = vc.x; c[j + 1] = vc.y; d[j] = vd.x; d[j + 1] = vd.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < S; ++j) {
      const bool in = j < len;
      a[j] = in ? D.a[L + j] : 0.0; b[j] = in ? D.b[L + j] : 1.0;
      c[j] = in ? D.c[L + j] : 0.0; d[j] = in ? D.d[L + j] : 0.0;
    }
  }
  if (first) a[0] = 0.0;
  // forward: rows 1..len-1, (alpha, gamma, delta) replace (a, c, d).  (Row
  // selections by len are written as per-row conditions inside the unrolled
  // loops: a separate "element len-1" access would become a dynamically
  // indexed array in local memory.)
  double gam, del, alp;
  {
    const double r = rcp(b[1], status);
    gam = c[1] * r; del = d[1] * r; alp = a[1] * r;
    a[1] = alp; c[1] = gam; d[1] = del;
  }
  // the backward pass starts from row len-2's forward values
  double ap = alp, gp = gam, dp = del;
#pragma unroll
  for (int j = 2; j < S; ++j) {
    if (j < len) {
      const double cj = (last && j == len - 1) ? 0.0 : c[j];
      const double r = rcp(fma(-a[j], gam, b[j]), status);
      const double q = a[j] * r;
      gam = cj * r;
      del = fma(-q, del, d[j] * r);
      alp = -q * alp;
      a[j] = alp; c[j] = gam; d[j] = del;
      if (j == len - 2) { ap = alp; gp = gam; dp = del; }
    }
  }
  const double r1a = alp, r1c = gam, r1d = del;
  // backward over the interior rows len-3 .. 1
#pragma unroll
  for (int j = S - 3; j >= 1; --j) {
    if (j < len - 2) {
      const double gj = c[j];
      dp = fma(-gj, dp, d[j]);
      ap = fma(-gj, ap, a[j]);
      gp = -gj * gp;
      a[j] = ap; c[j] = gp; d[j] = dp;
    }
  }
  const double r0a = a[0], r0b = fma(-c[0], ap, b[0]), r0c = -c[0] * gp, r0d = fma(-c[0], dp, d[0]);
  // kept rows 0 and len-1 give x_L and x_R themselves
  a[0] = -1.0; c[0] = 0.0; d[0] = 0.0;
  if (full) {
    a[S - 1] = 0.0; c[S - 1] = -1.0; d[S - 1] = 0.0;
#pragma unroll
    for (int j = 0; j < S; j += 2) {
      *reinterpret_cast<double2*>(D.ka + L + j) = make_double2(a[j], a[j + 1]);
      *reinterpret_cast<double2*>(D.kg + L + j) = make_double2(c[j], c[j + 1]);
      *reinterpret_cast<double2*>(D.kd + L + j) = make_double2(d[j], d[j + 1]);
    }
  } else {
#pragma unroll
    for (int j = 0; j < S; ++j) {
      if (j < len) {
        const bool end = j == len - 1;
        D.ka[L + j] = end ? 0.0 : a[j];
        D.kg[L + j] = end ? -1.0 : c[j];
        D.kd[L + j] = end ? 0.0 : d[j];
      }
    }
  }
  *reinterpret_cast<double2*>(D.na + 2 * k) = make_double2(r0a, r1a);
  *reinterpret_cast<double2*>(D.nb + 2 * k) = make_double2(r0b, 1.0);
  *reinterpret_cast<double2*>(D.nc + 2 * k) = make_double2(r0c, r1c);
  *reinterpret_cast<double2*>(D.nd + 2 * k) = make_double2(r0d, r1d);
}

__device__ __forceinline__ bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Every level of P (down, base, up) with grid barriers between them; all
// threads of the grid must call it.  Returns false once a barrier wait ran out.
__device__ __forceinline__ bool coop_levels(const CoopParams& P, unsigned* bar, unsigned* status) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nth = int64_t(gridDim.x) * blockDim.x;
  bool ok = true;
  for (int l = 0; l < P.L && ok; ++l) {
    const CoopLevel& D = P.lv[l];
    const bool reg8 = P.reg && D.s == 8 && aligned16(D.a) && aligned16(D.b) && aligned16(D.c) && aligned16(D.d) &&
                      aligned16(D.ka) && aligned16(D.kg) && aligned16(D.kd);
    for (int64_t k = tid; k < D.m; k += nth) {
      const int len = int(min(int64_t(8), D.M - k * 8));
      if (reg8 && len >= 3)
        coop_block_reduce_reg<8>(D, k, len, status);
      else
        coop_block_reduce(D, k, status);
    }
    ok = grid_barrier(bar, status, P.wait_cycles, P.bar_extra);
  }
  if (ok && blockIdx.x == 0 && threadIdx.x < 32 && 2 * P.lv[P.L - 1].m <= 64) {
    const CoopLevel& D = P.lv[P.L - 1];
    warp_pcr64(D.na, D.nb, D.nc, D.nd, P.ybase, int(2 * D.m), status);
  } else if (ok && tid == 0) {
    // Thomas on the last system (2m rows of the deepest level) when it is larger
    const CoopLevel& D = P.lv[P.L - 1];
    const int64_t M = 2 * D.m;
    double gam = 0.0, del = 0.0;
    for (int64_t i = 0; i < M; ++i) {
      const double ai = (i == 0) ? 0.0 : D.na[i];
      const double ci = (i == M - 1) ? 0.0 : D.nc[i];
      const double r = rcp(fma(-ai, gam, D.nb[i]), status);
      del = fma(-ai * r, del, D.nd[i] * r);
      gam = ci * r;
      P.base_scratch[i] = gam;
      P.ybase[i] = del;
    }
    double xn = del;
    for (int64_t i = M - 2; i >= 0; --i) {
      xn = fma(-P.base_scratch[i], xn, P.ybase[i]);
      P.ybase[i] = xn;
    }
  }
  if (ok) ok = grid_barrier(bar, status, P.wait_cycles, P.bar_extra);
  for (int l = P.L - 1; l >= 0 && ok; --l) {
    const CoopLevel& D = P.lv[l];
    const double* yn = (l == P.L - 1) ? P.ybase : P.lv[l + 1].y;
    for (int64_t i = tid; i < D.M; i += nth) {
      const int64_t k = i / D.s;
      const double2 v = *reinterpret_cast<const double2*>(yn + 2 * k);
      D.y[i] = fma(-D.kg[i], v.y, fma(-D.ka[i], v.x, D.kd[i]));
    }
    if (l > 0) ok = grid_barrier(bar, status, P.wait_cycles, P.bar_extra);
  }
  return ok;
}

__global__ void __launch_bounds__(128) k_iface_coop(const __grid_constant__ CoopParams P, unsigned* bar,
                                                    unsigned* status) {
  coop_levels(P, bar, status);
}

}  // namespace tdp

namespace tdp {

// ---------------------------------------------------------------------------
// Segmented interface solve: the interface system of a batch is the
// concatenation of one decoupled interface system per system (a system's
// first interface row has no coupling to the left, its last none to the
// right).  One CTA solves one system's rows with the same method, on chip:
//   level 1: the rows in P <= blockDim.x blocks of q rows, one per thread
//            (rows read from L2, kept coefficients to global scratch),
//   level 2: the 2P interface rows in shared memory, reduced by warp 0 in
//            blocks of at most 16 rows to <= 64 rows,
//   base:    warp parallel cyclic reduction of those rows,
//   then Stage 3 of level 2 (warp 0) and of level 1 (every thread).
// No grid-wide synchronisation.  The rows of system j are
// [rows(j), rows(j+1)) with rows(j) = 2 bbase[j] (bbase: blocks before
// system j) or, when bbase is null, 2 j per_sys.
// ---------------------------------------------------------------------------
constexpr int kSegT = 256;         // threads per CTA (level-1 blocks at most)
constexpr int kSegM2 = 2 * kSegT;  // level-2 rows at most

struct __align__(16) SegSmem {
  double a2[kSegM2], b2[kSegM2], c2[kSegM2], d2[kSegM2];  // level-2 system
  double ka2[kSegM2], kg2[kSegM2], kd2[kSegM2];            // its kept coefficients
  double y2[kSegM2];                                       // its solution
  double a3[64], b3[64], c3[64], d3[64], y3[64];          // level-3 system and solution
};

__global__ void __launch_bounds__(kSegT) k_iface_seg(const double* __restrict__ ra, const double* __restrict__ rb,
                                                     const double* __restrict__ rc, const double* __restrict__ rd,
                                                     double* __restrict__ y, const int64_t* __restrict__ bbase,
                                                     int64_t per_sys, int32_t batch, double* __restrict__ ka,
                                                     double* __restrict__ kg, double* __restrict__ kd,
                                                     unsigned* __restrict__ status) {
  __shared__ SegSmem sm;
  for (int64_t j = blockIdx.x; j < batch; j += gridDim.x) {
    const int64_t R0 = bbase ? 2 * bbase[j] : 2 * j * per_sys;
    const int64_t R1 = bbase ? 2 * bbase[j + 1] : 2 * (j + 1) * per_sys;
    const int64_t M = R1 - R0;
    const int t = threadIdx.x, lane = t & 31;
    if (M <= 0) continue;  // uniform across the CTA
    if (M <= 64) {
      if (t < 32) warp_pcr64(ra + R0, rb + R0, rc + R0, rd + R0, y + R0, int(M), status);
      __syncthreads();
      continue;
    }
    // level 1
    const int64_t q = (M + 2 * kSegT - 1) / (2 * kSegT) * 2;  // even, P = ceil(M / q) <= kSegT blocks
    const int P = int((M + q - 1) / q);
    CoopLevel D1;
    D1.a = ra + R0; D1.b = rb + R0; D1.c = rc + R0; D1.d = rd + R0;
    D1.ka = ka + R0; D1.kg = kg + R0; D1.kd = kd + R0;
    D1.na = sm.a2; D1.nb = sm.b2; D1.nc = sm.c2; D1.nd = sm.d2;
    D1.y = nullptr;
    D1.M = M; D1.m = P; D1.s = int(q);
    if (t < P) coop_block_reduce(D1, t, status);
    __syncthreads();
    // level 2 (warp 0), the base system and Stage 3 of level 2
    const int M2 = 2 * P;
    if (t < 32) {
      if (M2 <= 64) {
        warp_pcr64(sm.a2, sm.b2, sm.c2, sm.d2, sm.y2, M2, status);
      } else {
        const int q2 = (M2 + 31) / 32;  // <= 16
        const int P2 = (M2 + q2 - 1) / q2;
        CoopLevel D2;
        D2.a = sm.a2; D2.b = sm.b2; D2.c = sm.c2; D2.d = sm.d2;
        D2.ka = sm.ka2; D2.kg = sm.kg2; D2.kd = sm.kd2;
        D2.na = sm.a3; D2.nb = sm.b3; D2.nc = sm.c3; D2.nd = sm.d3;
        D2.y = nullptr;
        D2.M = M2; D2.m = P2; D2.s = q2;
        if (lane < P2) coop_block_reduce(D2, lane, status);
        __syncwarp();
        warp_pcr64(sm.a3, sm.b3, sm.c3, sm.d3, sm.y3, 2 * P2, status);
        __syncwarp();
        for (int i = lane; i < M2; i += 32) {
          const int k = i / q2;
          sm.y2[i] = fma(-sm.kg2[i], sm.y3[2 * k + 1], fma(-sm.ka2[i], sm.y3[2 * k], sm.kd2[i]));
        }
      }
    }
    __syncthreads();
    // Stage 3 of level 1
    for (int64_t i = t; i < M; i += kSegT) {
      const int64_t k = i / q;
      y[R0 + i] = fma(-kg[R0 + i], sm.y2[2 * k + 1], fma(-ka[R0 + i], sm.y2[2 * k], kd[R0 + i]));
    }
    __syncthreads();
  }
}

}  // namespace tdp
