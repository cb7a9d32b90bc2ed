// Stage 1 with kept coefficients, binary64, for single systems with a
// compile-time sub-system size SB: the interleaved cp.async tile holds only a,
// c and d (24 bytes per row instead of 32); each thread reads the b values of
// its own block straight into registers (16-byte loads of one 128-byte-aligned
// run per block).  A quarter less shared memory per row lets a third more
// blocks, and so more independent recurrence chains, reside on an SM: the
// binary64 sweep is bound by the latency of those chains, not by HBM.
// Same arithmetic as vblock_reduce; ragged last blocks (len < SB) take the
// same unrolled loops with rows past len masked.
#pragma once
#include "tdp_vtile.cuh"

namespace tdp {

template <int SB>
__global__ void __launch_bounds__(256) k_stage1_vb(const double* __restrict__ a, const double* __restrict__ b,
                                                   const double* __restrict__ c, const double* __restrict__ d,
                                                   int64_t n, int64_t m, double* __restrict__ ra,
                                                   double* __restrict__ rb, double* __restrict__ rc,
                                                   double* __restrict__ rd, double* __restrict__ ka,
                                                   double* __restrict__ kg, double* __restrict__ kd,
                                                   const int64_t* __restrict__ off, int32_t nsys, int64_t kb,
                                                   int64_t ke, unsigned* __restrict__ status) {
  static_assert(SB % 2 == 0 && SB >= 4, "even block size of at least 4");
  constexpr int V = 2, G = SB / V;
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x, t = threadIdx.x, ldv = T + 1;
  const int64_t k0 = kb + int64_t(blockIdx.x) * T;  // blocks [kb, ke) of the m
  if (k0 >= ke) return;
  const int nb = int(min(int64_t(T), ke - k0));
  const size_t plane = size_t(SB) * ldv;
  double* A = reinterpret_cast<double*>(smem);
  double* Cc = A + plane;
  double* D = A + 2 * plane;
  const int64_t ts = k0 * SB, te = min(n, (k0 + nb) * SB);
  {
    const double* const src[3] = {a, c, d};
    double* const pl[3] = {A, Cc, D};
    vtile_issue<double, 3>(ts, te, n, SB, ldv, src, pl);
  }
  // this thread's b values, while the tile's copies are in flight
  const int64_t k = k0 + t, L = k * SB;
  const int len = t < nb ? int(min(int64_t(SB), n - L)) : 0;
  double bv[SB];
  if (len == SB) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const double2 v = __ldcs(reinterpret_cast<const double2*>(b + L) + g);
      bv[2 * g] = v.x;
      bv[2 * g + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < SB; ++j) bv[j] = j < len ? b[L + j] : 1.0;
  }
  int jb = 0;
  if (off && t < 32) jb = warp_lower_bound(off, 1, nsys, ts);
  cp_async_commit_wait_all();
  __syncthreads();
  if (off) {
    if (t < 32) vtile_cut<double>(ts, te, SB, ldv, off, nsys, jb, A, Cc);
    __syncthreads();
  }
  if (len > 0) {
    const bool first = k == 0, last = k == m - 1;
    auto at = [&](int g) { return (g * ldv + t) * V; };
    IfaceRows out{0.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0};
    Vec<double> va = lds16<double>(A + at(0)), vc = lds16<double>(Cc + at(0)), vd = lds16<double>(D + at(0));
    const double a0 = first ? 0.0 : va.v[0], b0 = bv[0], d0 = vd.v[0];
    double c0 = vc.v[0];
    if (len == 1) {
      if (last) c0 = 0.0;
      out = IfaceRows{a0, b0, c0, d0, 0.0, 1.0, 0.0, 0.0};
      va.v[0] = -1.0; vc.v[0] = 0.0; vd.v[0] = 0.0;
      sts16<double>(A + at(0), va); sts16<double>(Cc + at(0), vc); sts16<double>(D + at(0), vd);
    } else {
      // forward sweep, rows 1..len-1; (alpha, gamma, delta) replace (a, c, d)
      double gam = 0.0, del = 0.0, alp = 0.0;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        if (g > 0) {
          va = lds16<double>(A + at(g)); vc = lds16<double>(Cc + at(g)); vd = lds16<double>(D + at(g));
        }
#pragma unroll
        for (int u = 0; u < V; ++u) {
          const int j = g * V + u;
          if (j == 0 || j >= len) continue;
          const double aj = va.v[u], dj = vd.v[u];
          const double cj = (j == len - 1 && last) ? 0.0 : vc.v[u];
          if (j == 1) {
            const double r = rcp(bv[1], status);
            gam = cj * r;
            del = dj * r;
            alp = aj * r;
          } else {
            const double r = rcp(fma(-aj, gam, bv[j]), status);
            const double q = aj * r;
            gam = cj * r;
            del = fma(-q, del, dj * r);
            alp = -q * alp;
          }
          va.v[u] = alp; vc.v[u] = gam; vd.v[u] = del;
        }
        sts16<double>(A + at(g), va); sts16<double>(Cc + at(g), vc); sts16<double>(D + at(g), vd);
      }
      out.a1 = alp;
      out.b1 = 1.0;
      out.c1 = gam;
      out.d1 = del;
      // backward over the interior rows len-3 .. 1 from row len-2 (kept as it is)
      double ap = 0.0, gp = -1.0, dp = 0.0;
      if (len >= 3) {
        const int jl = len - 2;
        ap = A[at(jl / V) + jl % V];
        gp = Cc[at(jl / V) + jl % V];
        dp = D[at(jl / V) + jl % V];
#pragma unroll
        for (int g = G - 1; g >= 0; --g) {
          if (g * V > len - 3) continue;
          Vec<double> wa = lds16<double>(A + at(g)), wc = lds16<double>(Cc + at(g)), wd = lds16<double>(D + at(g));
#pragma unroll
          for (int u = V - 1; u >= 0; --u) {
            const int j = g * V + u;
            if (j < 1 || j > len - 3) continue;
            const double gj = wc.v[u];
            dp = fma(-gj, dp, wd.v[u]);
            ap = fma(-gj, ap, wa.v[u]);
            gp = -gj * gp;
            wa.v[u] = ap; wc.v[u] = gp; wd.v[u] = dp;
          }
          sts16<double>(A + at(g), wa); sts16<double>(Cc + at(g), wc); sts16<double>(D + at(g), wd);
        }
      }
      out.a0 = a0;
      out.b0 = fma(-c0, ap, b0);
      out.c0 = -c0 * gp;
      out.d0 = fma(-c0, dp, d0);
      A[at(0)] = -1.0; Cc[at(0)] = 0.0; D[at(0)] = 0.0;
      const int jr = len - 1;
      A[at(jr / V) + jr % V] = 0.0; Cc[at(jr / V) + jr % V] = -1.0; D[at(jr / V) + jr % V] = 0.0;
    }
    write_iface(k, out, ra, rb, rc, rd);
  }
  __syncthreads();
  const double* const from[3] = {A, Cc, D};
  double* const to[3] = {ka, kg, kd};
  vtile_store<double, double, 3>(ts, te, SB, ldv, from, to);
}

}  // namespace tdp
