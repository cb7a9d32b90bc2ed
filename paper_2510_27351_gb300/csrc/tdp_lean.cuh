// Lean binary32 sweeps for full blocks (len == s, s a multiple of V) stored
// as 16-byte chunks: used by the interleaved tiles (tdp_vtile.cuh) and the
// warp-owned tiles (tdp_wtile.cuh).
#pragma once
#include "tdp_kernels.cuh"

namespace tdp {

// ---------------------------------------------------------------------------
// Lean binary32 sweeps over one block stored as 16-byte chunks of V rows,
// chunk g at p + g * cs (cs = V for a contiguous block, (T + 1) V for the
// interleaved tiles).
// ---------------------------------------------------------------------------

// Slots written back for the backward pass.  S == C stores the value; with
// binary64 storage and binary32 arithmetic the binary32 bits go to the high
// word of the slot (register moves, no conversion).
template <typename S, typename C>
struct Slot {
  static __device__ __forceinline__ S put(C v) { return S(v); }
  static __device__ __forceinline__ C get(S v) { return C(v); }
};
template <>
struct Slot<double, float> {
  static __device__ __forceinline__ double put(float v) { return __hiloint2double(__float_as_int(v), 0); }
  static __device__ __forceinline__ float get(double v) { return __int_as_float(__double2hiint(v)); }
};

// MUFU reciprocal estimate y of x and its residual e = 1 - x y; the refined
// reciprocal is y + y e.  Callers fold r into z = fma(r, 0, z), which turns
// into nan once a pivot is zero or not finite.
__device__ __forceinline__ float rcp_est(float x, float& e) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  e = fmaf(-x, y, 1.0f);
  return y;
}

// One row of the downward elimination of Stage 1 (Sec. I): after the row,
// alp x[L] + x[j] + gam x[j+1] = del.  alp starts at -1, gam and del at 0, so
// that the first interior row needs no special case.
struct FwdF {
  float gam, del, alp, z;
  __device__ __forceinline__ void step(float a, float b, float c, float d) {
    float e;
    const float x = fmaf(-a, gam, b);
    const float y = rcp_est(x, e);
    const float r = fmaf(y, e, y);
    const float cy = c * y;
    gam = fmaf(cy, e, cy);
    z = fmaf(r, 0.0f, z);
    const float q = a * r;
    del = fmaf(-q, del, d * r);
    alp = -q * alp;
  }
};

// Stage 1 of a full block (len == s).  Returns the two interface rows; z
// accumulates the pivot check.
template <typename S>
__device__ __forceinline__ IfaceRows wreduce_full(S* pa, S* pb, S* pc, S* pd, int s, int cs, bool first, bool last,
                                                  float& z) {
  constexpr int V = Vec<S>::W;
  using SL = Slot<S, float>;
  const int G = s / V;
  auto pos = [&](int j) { return (j / V) * cs + j % V; };
  if (last) pc[pos(s - 1)] = S(0);
  FwdF f{0.0f, 0.0f, -1.0f, z};
  float a0, b0, c0, d0;
  {
    Vec<S> va = lds16<S>(pa), vb = lds16<S>(pb), vc = lds16<S>(pc), vd = lds16<S>(pd);
    a0 = first ? 0.0f : cvt<float>(va.v[0]);
    b0 = cvt<float>(vb.v[0]);
    c0 = cvt<float>(vc.v[0]);
    d0 = cvt<float>(vd.v[0]);
#pragma unroll
    for (int u = 1; u < V; ++u) {
      f.step(cvt<float>(va.v[u]), cvt<float>(vb.v[u]), cvt<float>(vc.v[u]), cvt<float>(vd.v[u]));
      va.v[u] = SL::put(f.alp);
      vc.v[u] = SL::put(f.gam);
      vd.v[u] = SL::put(f.del);
    }
    sts16<S>(pa, va);
    sts16<S>(pc, vc);
    sts16<S>(pd, vd);
  }
  for (int g = 1; g < G; ++g) {
    const int o = g * cs;
    Vec<S> va = lds16<S>(pa + o), vb = lds16<S>(pb + o), vc = lds16<S>(pc + o), vd = lds16<S>(pd + o);
#pragma unroll
    for (int u = 0; u < V; ++u) {
      f.step(cvt<float>(va.v[u]), cvt<float>(vb.v[u]), cvt<float>(vc.v[u]), cvt<float>(vd.v[u]));
      va.v[u] = SL::put(f.alp);
      vc.v[u] = SL::put(f.gam);
      vd.v[u] = SL::put(f.del);
    }
    sts16<S>(pa + o, va);
    sts16<S>(pc + o, vc);
    sts16<S>(pd + o, vd);
  }
  z = f.z;
  IfaceRows out;
  out.a1 = widen(f.alp);
  out.b1 = 1.0;
  out.c1 = widen(f.gam);
  out.d1 = widen(f.del);
  // backward over the interior rows s-2 .. 1: the primes of row 1 give row L
  float ap = 0.0f, gp = -1.0f, dp = 0.0f;
  if (s > 2) {
    ap = SL::get(pa[pos(s - 2)]);
    gp = SL::get(pc[pos(s - 2)]);
    dp = SL::get(pd[pos(s - 2)]);
    auto bstep = [&](S sa, S sc, S sd) {
      const float gj = SL::get(sc);
      dp = fmaf(-gj, dp, SL::get(sd));
      ap = fmaf(-gj, ap, SL::get(sa));
      gp = -gj * gp;
    };
    const int gl = (s - 3) / V;  // chunk of row s-3
    for (int g = gl; g >= 0; --g) {
      const int o = g * cs;
      const Vec<S> wa = lds16<S>(pa + o), wc = lds16<S>(pc + o), wd = lds16<S>(pd + o);
      if (g == gl || g == 0) {
#pragma unroll
        for (int u = V - 1; u >= 0; --u) {
          const int j = g * V + u;
          if (j >= 1 && j <= s - 3) bstep(wa.v[u], wc.v[u], wd.v[u]);
        }
      } else {
#pragma unroll
        for (int u = V - 1; u >= 0; --u) bstep(wa.v[u], wc.v[u], wd.v[u]);
      }
    }
  }
  out.a0 = widen(a0);
  out.b0 = widen(fmaf(-c0, ap, b0));
  out.c0 = widen(-c0 * gp);
  out.d0 = widen(fmaf(-c0, dp, d0));
  return out;
}

// Stage 3 of a full block by the interior solve with x[L] = yl, x[R] = yr
// known (binary32 arithmetic); x, as S, is left in the d plane.
template <typename S>
__device__ __forceinline__ void wsubstitute_full(S* pa, S* pb, S* pc, S* pd, int s, int cs, double yl, double yr,
                                                 float& z) {
  constexpr int V = Vec<S>::W;
  using SL = Slot<S, float>;
  const int G = s / V;
  const float fl = narrow(yl), fr = narrow(yr);
  auto pos = [&](int j) { return (j / V) * cs + j % V; };
  if (s >= 3) {
    // the known interface values move to the right-hand sides of rows 1 and s-2
    pd[pos(1)] = cvt<S>(fmaf(-cvt<float>(pa[pos(1)]), fl, cvt<float>(pd[pos(1)])));
    pd[pos(s - 2)] = cvt<S>(fmaf(-cvt<float>(pc[pos(s - 2)]), fr, cvt<float>(pd[pos(s - 2)])));
    pc[pos(s - 2)] = S(0);
    float gam = 0.0f, del = 0.0f, zz = z;
    auto fstep = [&](S sa, S sb, S& sc, S& sd) {
      float e;
      const float a = cvt<float>(sa);
      const float x = fmaf(-a, gam, cvt<float>(sb));
      const float y = rcp_est(x, e);
      const float r = fmaf(y, e, y);
      const float cy = cvt<float>(sc) * y;
      gam = fmaf(cy, e, cy);
      zz = fmaf(r, 0.0f, zz);
      del = fmaf(-a * r, del, cvt<float>(sd) * r);
      sc = SL::put(gam);
      sd = SL::put(del);
    };
    for (int g = 0; g < G; ++g) {
      const int o = g * cs;
      const Vec<S> va = lds16<S>(pa + o), vb = lds16<S>(pb + o);
      Vec<S> vc = lds16<S>(pc + o), vd = lds16<S>(pd + o);
      if (g == 0 || g == G - 1) {
#pragma unroll
        for (int u = 0; u < V; ++u) {
          const int j = g * V + u;
          if (j >= 1 && j <= s - 2) fstep(va.v[u], vb.v[u], vc.v[u], vd.v[u]);
        }
      } else {
#pragma unroll
        for (int u = 0; u < V; ++u) fstep(va.v[u], vb.v[u], vc.v[u], vd.v[u]);
      }
      sts16<S>(pc + o, vc);
      sts16<S>(pd + o, vd);
    }
    z = zz;
    // backward substitution, rows s-2 .. 1, x written as S
    float xn = del;
    const int gl = (s - 2) / V;  // chunk of row s-2
    for (int g = gl; g >= 0; --g) {
      const int o = g * cs;
      const Vec<S> vc = lds16<S>(pc + o);
      Vec<S> vd = lds16<S>(pd + o);
      if (g == gl || g == 0) {
#pragma unroll
        for (int u = V - 1; u >= 0; --u) {
          const int j = g * V + u;
          if (j < 1 || j > s - 2) continue;
          if (j < s - 2) xn = fmaf(-SL::get(vc.v[u]), xn, SL::get(vd.v[u]));
          vd.v[u] = cvt<S>(xn);
        }
      } else {
#pragma unroll
        for (int u = V - 1; u >= 0; --u) {
          xn = fmaf(-SL::get(vc.v[u]), xn, SL::get(vd.v[u]));
          vd.v[u] = cvt<S>(xn);
        }
      }
      sts16<S>(pd + o, vd);
    }
  }
  pd[0] = cvt<S>(fl);
  pd[pos(s - 1)] = cvt<S>(fr);
}

}  // namespace tdp
