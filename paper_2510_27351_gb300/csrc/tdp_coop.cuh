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
  double* base_scratch;  // Thomas scratch for the last system
  double* ybase;         // solution of the last system (2 * lv[L-1].m rows)
};

// Grid-wide barrier.  bar[0] counts arrivals, bar[1] is the generation.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned* status) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (clock64() - t0 > (1ll << 31)) {
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

__global__ void __launch_bounds__(128) k_iface_coop(const __grid_constant__ CoopParams P, unsigned* bar,
                                                    unsigned* status) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nth = int64_t(gridDim.x) * blockDim.x;
  bool ok = true;
  for (int l = 0; l < P.L && ok; ++l) {
    const CoopLevel& D = P.lv[l];
    for (int64_t k = tid; k < D.m; k += nth) coop_block_reduce(D, k, status);
    ok = grid_barrier(bar, status);
  }
  if (ok && tid == 0) {
    // Thomas on the last system (2m rows of the deepest level)
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
  if (ok) ok = grid_barrier(bar, status);
  for (int l = P.L - 1; l >= 0 && ok; --l) {
    const CoopLevel& D = P.lv[l];
    const double* yn = (l == P.L - 1) ? P.ybase : P.lv[l + 1].y;
    for (int64_t i = tid; i < D.M; i += nth) {
      const int64_t k = i / D.s;
      const double2 v = *reinterpret_cast<const double2*>(yn + 2 * k);
      D.y[i] = fma(-D.kg[i], v.y, fma(-D.ka[i], v.x, D.kd[i]));
    }
    if (l > 0) ok = grid_barrier(bar, status);
  }
}

}  // namespace tdp
