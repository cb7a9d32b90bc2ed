// Vector-interleaved tiles for single-system solves.
//
// When every block starts on a 16-byte boundary (one system, s a multiple of
// V = 16 / sizeof(S)), a 16-byte chunk of an array holds V consecutive rows of
// ONE block.  The shared-memory layout keeps such chunks whole:
//     row j of the block of thread t  ->  ((j / V) * ldv + t) * V + (j % V),
// so the tile is filled by 16-byte cp.async copies straight from HBM (every
// chunk of the CTA in flight at once, no registers), and each thread reads V
// rows of its block with one 16-byte shared load (consecutive threads read
// consecutive 16-byte words).  ldv = T + 1 spreads the copies of one warp over
// all banks.
#pragma once
#include "tdp_lean.cuh"

namespace tdp {

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned sa = unsigned(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Tile rows [ts, te) of NA arrays into the interleaved layout.  Chunks that
// reach past the end of an array (n not a multiple of V) are read element by
// element.  vtile_issue starts the copies, cp_async_commit_wait_all waits
// for them (vtile_load does both).
template <typename S, int NA>
__device__ __forceinline__ void vtile_issue(int64_t ts, int64_t te, int64_t n, int s, int ldv,
                                            const S* const (&src)[NA], S* const (&pl)[NA]) {
  constexpr int V = Vec<S>::W;
  const int chunks = int((te - ts + V - 1) / V);
  const int cps = s / V;  // chunks per block
  for (int q = threadIdx.x; q < chunks; q += blockDim.x) {
    const int t = q / cps, g = q - t * cps;
    const int64_t row = ts + int64_t(q) * V;
    const int idx = (g * ldv + t) * V;
    if (row + V <= n) {
#pragma unroll
      for (int i = 0; i < NA; ++i) cp_async16(pl[i] + idx, src[i] + row);
    } else {
#pragma unroll
      for (int i = 0; i < NA; ++i)
#pragma unroll
        for (int u = 0; u < V; ++u) pl[i][idx + u] = (row + u < n) ? src[i][row + u] : S(0);
    }
  }
}

template <typename S, int NA>
__device__ __forceinline__ void vtile_load(int64_t ts, int64_t te, int64_t n, int s, int ldv,
                                           const S* const (&src)[NA], S* const (&pl)[NA]) {
  vtile_issue<S, NA>(ts, te, n, s, ldv, src, pl);
  cp_async_commit_wait_all();
}

// A batch solved as one system (offsets off[0..nsys], system j in rows
// [off[j], off[j+1])): inside the tile of rows [ts, te), zero the couplings
// across system boundaries, a of every system's first row and c of every
// system's last row.  Warp 0 only; jb = warp_lower_bound(off, 1, nsys, ts).
template <typename S>
__device__ __forceinline__ void vtile_cut(int64_t ts, int64_t te, int s, int ldv, const int64_t* off, int32_t nsys,
                                          int jb, S* A, S* C) {
  constexpr int V = Vec<S>::W;
  auto pos = [&](int64_t p) {
    const int q = int(p - ts), t = q / s, j = q - t * s;
    return ((j / V) * ldv + t) * V + j % V;
  };
  for (int j = jb + (threadIdx.x & 31); j < nsys; j += 32) {
    const int64_t p = off[j];
    if (p > te) break;
    if (p >= ts && p < te) A[pos(p)] = S(0);  // (the p >= ts test keeps unsorted offsets in the tile)
    if (p - 1 >= ts) C[pos(p - 1)] = S(0);
  }
}

// Planes of the tile to global arrays (16-byte stores, element-wise at the end).
template <typename S, typename D, int NA>
__device__ __forceinline__ void vtile_store(int64_t ts, int64_t te, int s, int ldv, const S* const (&pl)[NA],
                                            D* const (&dst)[NA]) {
  constexpr int V = Vec<S>::W;
  static_assert(sizeof(S) == sizeof(D), "same element size in and out");
  const int chunks = int((te - ts + V - 1) / V);
  const int cps = s / V;
  for (int q = threadIdx.x; q < chunks; q += blockDim.x) {
    const int t = q / cps, g = q - t * cps;
    const int64_t row = ts + int64_t(q) * V;
    const int idx = (g * ldv + t) * V;
    if (row + V <= te) {
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        Vec<S> v = lds16<S>(pl[i] + idx);
        Vec<D> w;
#pragma unroll
        for (int u = 0; u < V; ++u) w.v[u] = cvt<D>(v.v[u]);
        stg16<D>(dst[i] + row, w);
      }
    } else {
#pragma unroll
      for (int i = 0; i < NA; ++i)
#pragma unroll
        for (int u = 0; u < V; ++u)
          if (row + u < te) dst[i][row + u] = cvt<D>(pl[i][idx + u]);
    }
  }
}

// Stage 1 sweep of one block on the interleaved tile; same arithmetic as
// block_reduce (rows are read V at a time).  `base` = element offset t * V.
template <typename S, typename C, bool KEEP>
__device__ __forceinline__ IfaceRows vblock_reduce(S* A, S* B, S* Cc, S* D, int ldv, int t, const BlockInfo& bi,
                                                   unsigned* status) {
  constexpr int V = Vec<S>::W;
  const int len = bi.len;
  IfaceRows out{0.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0};
  if (len <= 0) return out;
  auto at = [&](int g) { return (g * ldv + t) * V; };
  const int G = (len + V - 1) / V;
  Vec<S> va = lds16<S>(A + at(0)), vb = lds16<S>(B + at(0)), vc = lds16<S>(Cc + at(0)), vd = lds16<S>(D + at(0));
  C a0 = bi.first ? C(0) : cvt<C>(va.v[0]);
  const C b0 = cvt<C>(vb.v[0]);
  C c0 = cvt<C>(vc.v[0]);
  const C d0 = cvt<C>(vd.v[0]);
  if (len == 1) {
    if (bi.last) c0 = C(0);
    out = IfaceRows{to_f64(a0), to_f64(b0), to_f64(c0), to_f64(d0), 0.0, 1.0, 0.0, 0.0};
    if (KEEP) {
      va.v[0] = S(-1); vc.v[0] = S(0); vd.v[0] = S(0);
      sts16<S>(A + at(0), va); sts16<S>(Cc + at(0), vc); sts16<S>(D + at(0), vd);
    }
    return out;
  }
  // forward sweep; group g's forward values overwrite its a, c, d words
  C gam = C(0), del = C(0), alp = C(0);
  for (int g = 0; g < G; ++g) {
    if (g > 0) {
      va = lds16<S>(A + at(g)); vb = lds16<S>(B + at(g)); vc = lds16<S>(Cc + at(g)); vd = lds16<S>(D + at(g));
    }
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const int j = g * V + u;
      if (j == 0 || j >= len) continue;
      const C aj = cvt<C>(va.v[u]), bj = cvt<C>(vb.v[u]), dj = cvt<C>(vd.v[u]);
      C cj = cvt<C>(vc.v[u]);
      if (j == len - 1 && bi.last) cj = C(0);
      if (j == 1) {
        const C r = rcp(bj, status);
        gam = cj * r;
        del = dj * r;
        alp = aj * r;
      } else {
        const C r = rcp(fma(-aj, gam, bj), status);
        const C q = aj * r;
        gam = cj * r;
        del = fma(-q, del, dj * r);
        alp = -q * alp;
      }
      va.v[u] = cvt<S>(alp); vc.v[u] = cvt<S>(gam); vd.v[u] = cvt<S>(del);
    }
    sts16<S>(A + at(g), va); sts16<S>(Cc + at(g), vc); sts16<S>(D + at(g), vd);
  }
  out.a1 = to_f64(alp);
  out.b1 = 1.0;
  out.c1 = to_f64(gam);
  out.d1 = to_f64(del);
  // backward over the interior (rows len-2 .. 1)
  C ap, gp, dp;
  if (len == 2) {
    ap = C(0); gp = C(-1); dp = C(0);
  } else {
    const int jl = len - 2;
    ap = cvt<C>(A[at(jl / V) + jl % V]);
    gp = cvt<C>(Cc[at(jl / V) + jl % V]);
    dp = cvt<C>(D[at(jl / V) + jl % V]);
    for (int g = (len - 3) / V; g >= 0; --g) {
      Vec<S> wa = lds16<S>(A + at(g)), wc = lds16<S>(Cc + at(g)), wd = lds16<S>(D + at(g));
#pragma unroll
      for (int u = V - 1; u >= 0; --u) {
        const int j = g * V + u;
        if (j < 1 || j > len - 3) continue;
        const C aj = cvt<C>(wa.v[u]), gj = cvt<C>(wc.v[u]), dj = cvt<C>(wd.v[u]);
        dp = fma(-gj, dp, dj);
        ap = fma(-gj, ap, aj);
        gp = -gj * gp;
        if (KEEP) { wa.v[u] = cvt<S>(ap); wc.v[u] = cvt<S>(gp); wd.v[u] = cvt<S>(dp); }
      }
      if (KEEP) { sts16<S>(A + at(g), wa); sts16<S>(Cc + at(g), wc); sts16<S>(D + at(g), wd); }
    }
  }
  out.a0 = to_f64(a0);
  out.b0 = to_f64(fma(-c0, ap, b0));
  out.c0 = to_f64(-c0 * gp);
  out.d0 = to_f64(fma(-c0, dp, d0));
  if (KEEP) {
    A[at(0)] = S(-1); Cc[at(0)] = S(0); D[at(0)] = S(0);
    const int jr = len - 1;
    A[at(jr / V) + jr % V] = S(0); Cc[at(jr / V) + jr % V] = S(-1); D[at(jr / V) + jr % V] = S(0);
  }
  return out;
}

// Stage 3 interior solve of one block on the interleaved tile (x into D).
template <typename S, typename C>
__device__ __forceinline__ void vblock_substitute(S* A, S* B, S* Cc, S* D, int ldv, int t, int len, C yl, C yr,
                                                  unsigned* status) {
  constexpr int V = Vec<S>::W;
  if (len <= 0) return;
  auto at = [&](int g) { return (g * ldv + t) * V; };
  auto pos = [&](int j) { return at(j / V) + j % V; };
  if (len >= 3) {
    // forward over the interior rows 1..len-2: gamma into the c words, delta into the d words
    C gam = C(0), del = C(0);
    for (int g = 0; g <= (len - 2) / V; ++g) {
      const Vec<S> va = lds16<S>(A + at(g)), vb = lds16<S>(B + at(g));
      Vec<S> vc = lds16<S>(Cc + at(g)), vd = lds16<S>(D + at(g));
#pragma unroll
      for (int u = 0; u < V; ++u) {
        const int j = g * V + u;
        if (j < 1 || j > len - 2) continue;
        const C aj = cvt<C>(va.v[u]), bj = cvt<C>(vb.v[u]), cj = cvt<C>(vc.v[u]);
        C dj = cvt<C>(vd.v[u]);
        if (j == 1) dj = fma(-aj, yl, dj);
        if (j == len - 2) dj = fma(-cj, yr, dj);
        const C den = (j == 1) ? bj : fma(-aj, gam, bj);
        const C r = rcp(den, status);
        del = (j == 1) ? dj * r : fma(-aj * r, del, dj * r);
        gam = (j == len - 2) ? C(0) : cj * r;
        vc.v[u] = cvt<S>(gam);
        vd.v[u] = cvt<S>(del);
      }
      sts16<S>(Cc + at(g), vc);
      sts16<S>(D + at(g), vd);
    }
    // backward: x[len-2] = delta[len-2] is in place; rows len-3 .. 1
    C xn = del;
    for (int g = (len - 3) / V; g >= 0; --g) {
      const Vec<S> vc = lds16<S>(Cc + at(g));
      Vec<S> vd = lds16<S>(D + at(g));
#pragma unroll
      for (int u = V - 1; u >= 0; --u) {
        const int j = g * V + u;
        if (j < 1 || j > len - 3) continue;
        xn = fma(-cvt<C>(vc.v[u]), xn, cvt<C>(vd.v[u]));
        vd.v[u] = cvt<S>(xn);
      }
      sts16<S>(D + at(g), vd);
    }
  }
  D[pos(0)] = cvt<S>(yl);
  if (len >= 2) D[pos(len - 1)] = cvt<S>(yr);
}

template <typename S, typename C, bool KEEP>
__global__ void __launch_bounds__(256) k_stage1_v(const S* __restrict__ a, const S* __restrict__ b,
                                                  const S* __restrict__ c, const S* __restrict__ d, int64_t n, int s,
                                                  int64_t m, double* __restrict__ ra, double* __restrict__ rb,
                                                  double* __restrict__ rc, double* __restrict__ rd,
                                                  C* __restrict__ ka, C* __restrict__ kg, C* __restrict__ kd,
                                                  const int64_t* __restrict__ off, int32_t nsys, int64_t kb,
                                                  int64_t ke, unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x, t = threadIdx.x, ldv = T + 1;
  const int64_t k0 = kb + int64_t(blockIdx.x) * T;  // blocks [kb, ke) of the m
  if (k0 >= ke) return;
  const int nb = int(min(int64_t(T), ke - k0));
  const size_t plane = size_t(s) * ldv;
  S* A = reinterpret_cast<S*>(smem);
  S* const pl[4] = {A, A + plane, A + 2 * plane, A + 3 * plane};
  const int64_t ts = k0 * s, te = min(n, (k0 + nb) * s);
  const S* const src[4] = {a, b, c, d};
  vtile_issue<S, 4>(ts, te, n, s, ldv, src, pl);
  int jb = 0;
  if (off && t < 32) jb = warp_lower_bound(off, 1, nsys, ts);  // while the copies fly
  cp_async_commit_wait_all();
  __syncthreads();
  if (off) {
    if (t < 32) vtile_cut<S>(ts, te, s, ldv, off, nsys, jb, pl[0], pl[2]);
    __syncthreads();
  }
  if (t < nb) {
    const BlockInfo bi = block_info<false>(k0 + t, n, s, m, nullptr);
    IfaceRows r;
    if constexpr (std::is_same<C, float>::value && !KEEP) {
      if (bi.len == s) {
        constexpr int V = Vec<S>::W;
        float z = 0.0f;
        r = wreduce_full<S>(pl[0] + t * V, pl[1] + t * V, pl[2] + t * V, pl[3] + t * V, s, ldv * V, bi.first,
                            bi.last, z);
        if (!(z == 0.0f)) flag(status, ST_SINGULAR);
      } else {
        r = vblock_reduce<S, C, KEEP>(pl[0], pl[1], pl[2], pl[3], ldv, t, bi, status);
      }
    } else {
      r = vblock_reduce<S, C, KEEP>(pl[0], pl[1], pl[2], pl[3], ldv, t, bi, status);
    }
    write_iface(k0 + t, r, ra, rb, rc, rd);
  }
  if constexpr (KEEP) {
    __syncthreads();
    const S* const from[3] = {pl[0], pl[2], pl[3]};
    C* const to[3] = {ka, kg, kd};
    vtile_store<S, C, 3>(ts, te, s, ldv, from, to);
  }
}

template <typename S, typename C>
__global__ void __launch_bounds__(256) k_stage3_resolve_v(const S* __restrict__ a, const S* __restrict__ b,
                                                          const S* __restrict__ c, const S* __restrict__ d,
                                                          int64_t n, int s, int64_t m, const double* __restrict__ y,
                                                          S* __restrict__ x, const int64_t* __restrict__ off,
                                                          int32_t nsys, int64_t kb, int64_t ke,
                                                          unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x, t = threadIdx.x, ldv = T + 1;
  const int64_t k0 = kb + int64_t(blockIdx.x) * T;  // blocks [kb, ke) of the m
  if (k0 >= ke) return;
  const int nb = int(min(int64_t(T), ke - k0));
  const size_t plane = size_t(s) * ldv;
  S* A = reinterpret_cast<S*>(smem);
  S* const pl[4] = {A, A + plane, A + 2 * plane, A + 3 * plane};
  const int64_t ts = k0 * s, te = min(n, (k0 + nb) * s);
  const S* const src[4] = {a, b, c, d};
  vtile_issue<S, 4>(ts, te, n, s, ldv, src, pl);
  int jb = 0;
  if (off && t < 32) jb = warp_lower_bound(off, 1, nsys, ts);
  cp_async_commit_wait_all();
  __syncthreads();
  if (off) {
    if (t < 32) vtile_cut<S>(ts, te, s, ldv, off, nsys, jb, pl[0], pl[2]);
    __syncthreads();
  }
  if (t < nb) {
    const BlockInfo bi = block_info<false>(k0 + t, n, s, m, nullptr);
    const double2 v = *reinterpret_cast<const double2*>(y + 2 * (k0 + t));
    bool lean = false;
    if constexpr (std::is_same<C, float>::value) {
      if (bi.len == s) {
        constexpr int V = Vec<S>::W;
        float z = 0.0f;
        wsubstitute_full<S>(pl[0] + t * V, pl[1] + t * V, pl[2] + t * V, pl[3] + t * V, s, ldv * V, v.x, v.y, z);
        if (!(z == 0.0f)) flag(status, ST_SINGULAR);
        lean = true;
      }
    }
    if (!lean)
      vblock_substitute<S, C>(pl[0], pl[1], pl[2], pl[3], ldv, t, bi.len, cvt<C>(v.x), cvt<C>(v.y), status);
  }
  __syncthreads();
  const S* const from[1] = {pl[3]};
  S* const to[1] = {x};
  vtile_store<S, S, 1>(ts, te, s, ldv, from, to);
}

}  // namespace tdp
