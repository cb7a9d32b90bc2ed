// Device helpers shared by the solver kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "tdp_status.h"

namespace tdp {


// Block descriptors of a batched solve: the start row of block k with two
// flag bits; entry m (one past the last block) holds the total row count.
constexpr int64_t BLK_FIRST = int64_t(1) << 61;  // first block of its system
constexpr int64_t BLK_LAST = int64_t(1) << 62;   // last block of its system
constexpr int64_t BLK_ROW = BLK_FIRST - 1;

__device__ __forceinline__ void flag(unsigned* status, unsigned bit) {
  if (status) atomicOr(status, bit);
}

// ---------------------------------------------------------------------------
// Reciprocals.  binary64: the MUFU approximation (about 2^-20 relative) is
// refined by one third-order Newton-Raphson step, y <- y (1 + e + e^2) with
// e = 1 - x y (the series 1/x = y/(1-e)); the truncation error is e^3, about
// 2^-60, below binary64 rounding.  Three FMAs instead of a division.  Inputs
// whose exponent is near the ends of the range (zero, subnormal, huge, inf,
// nan) take the IEEE division and raise the singular flag when the pivot is
// zero or the result is not finite.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double rcp(double x, unsigned* status) {
  const unsigned ex = (unsigned(__double2hiint(x)) >> 20) & 0x7ffu;
  if (ex - 32u < 1984u) {  // 2^-991 <= |x| < 2^993
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
  }
  const double y = 1.0 / x;
  if (x == 0.0 || !isfinite(y)) flag(status, ST_SINGULAR);
  return y;
}

// binary32: MUFU approximation plus one Newton-Raphson step y <- y + y(1 - x y).
__device__ __forceinline__ float rcp(float x, unsigned* status) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  const float e = fmaf(-x, y, 1.0f);
  y = fmaf(y, e, y);
  if (!(fabsf(y) < __int_as_float(0x7f800000))) flag(status, ST_SINGULAR);
  return y;
}

// Exact binary32 -> binary64 widening with integer operations (the hardware
// conversion runs at the binary64 rate on this part).  Subnormal binary32
// inputs flush to zero; inf and nan map to inf and nan.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned mag = u & 0x7fffffffu;
  unsigned hi = (mag >> 3) + (896u << 20);
  unsigned lo = mag << 29;
  if (mag < 0x00800000u) { hi = 0u; lo = 0u; }
  if (mag >= 0x7f800000u) hi = 0x7ff00000u | ((mag >> 3) & 0x000fffffu);
  return __hiloint2double(int(hi | (u & 0x80000000u)), int(lo));
}

// binary64 -> binary32 with integer operations (the hardware conversion also
// runs on the binary64 pipe), rounding toward zero.  The top 32 bits of the
// 64-bit pattern shifted left by 3 hold the low 9 exponent bits and the top 23
// mantissa bits; adding 128 to the exponent field (mod 512) rebiases every
// exponent of the binary32 normal range.  Magnitudes below that range give
// signed zero, above it (and nan) infinity.  Used for the inputs of the
// binary32 solves inside the binary64 refinement, whose result the binary64
// residual corrects.
__device__ __forceinline__ float narrow(double v) {
  const unsigned hi = unsigned(__double2hiint(v)), lo = unsigned(__double2loint(v));
  const unsigned mag = hi & 0x7fffffffu;
  unsigned w = __funnelshift_l(lo, hi, 3) + (128u << 23);
  w = mag < (897u << 20) ? 0u : (mag >= (1151u << 20) ? 0x7f800000u : w);
  return __uint_as_float((w & 0x7fffffffu) | (hi & 0x80000000u));
}

template <typename C> __device__ __forceinline__ C cvt(double v);
template <> __device__ __forceinline__ double cvt<double>(double v) { return v; }
template <> __device__ __forceinline__ float cvt<float>(double v) { return narrow(v); }
template <typename C> __device__ __forceinline__ C cvt(float v);
template <> __device__ __forceinline__ float cvt<float>(float v) { return v; }
template <> __device__ __forceinline__ double cvt<double>(float v) { return widen(v); }

__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return widen(v); }

// 16-byte vector of storage elements.
template <typename S> struct Vec;
template <> struct Vec<double> {
  static constexpr int W = 2;
  double v[2];
};
template <> struct Vec<float> {
  static constexpr int W = 4;
  float v[4];
};

template <typename S> __device__ __forceinline__ Vec<S> ldg16(const S* p) {
  Vec<S> r;
  if constexpr (sizeof(S) == 8) {
    double2 t = __ldg(reinterpret_cast<const double2*>(p));
    r.v[0] = t.x; r.v[1] = t.y;
  } else {
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
  }
  return r;
}

// Streaming (evict-first) loads for data read exactly once.
template <typename S> __device__ __forceinline__ Vec<S> ldcs16(const S* p) {
  Vec<S> r;
  if constexpr (sizeof(S) == 8) {
    double2 t = __ldcs(reinterpret_cast<const double2*>(p));
    r.v[0] = t.x; r.v[1] = t.y;
  } else {
    float4 t = __ldcs(reinterpret_cast<const float4*>(p));
    r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
  }
  return r;
}

template <typename S> __device__ __forceinline__ void stg16(S* p, const Vec<S>& r) {
  if constexpr (sizeof(S) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2(r.v[0], r.v[1]);
  } else {
    *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
  }
}

// ---------------------------------------------------------------------------
// Block geometry of one CTA tile.  A CTA owns T consecutive blocks (one per
// thread); their rows are contiguous in memory.  Unmapped: one system of n
// rows cut every s rows.  Mapped: descriptors from blk[] (batched solves).
// ---------------------------------------------------------------------------
struct BlockInfo {
  int64_t start;  // first global row
  int len;        // rows in the block
  bool first;     // a[start] is ignored
  bool last;      // c[start+len-1] is ignored
};

template <bool MAPPED>
__device__ __forceinline__ BlockInfo block_info(int64_t k, int64_t n, int s, int64_t m, const int64_t* blk) {
  BlockInfo bi;
  if constexpr (MAPPED) {
    const int64_t e = blk[k];
    bi.start = e & BLK_ROW;
    bi.len = int((blk[k + 1] & BLK_ROW) - bi.start);
    bi.first = (e & BLK_FIRST) != 0;
    bi.last = (e & BLK_LAST) != 0;
  } else {
    bi.start = k * s;
    const int64_t rem = n - bi.start;
    bi.len = int(rem < s ? rem : s);
    bi.first = (k == 0);
    bi.last = (k == m - 1);
  }
  return bi;
}

template <bool MAPPED>
__device__ __forceinline__ int64_t block_start(int64_t k, int64_t n, int s, const int64_t* blk) {
  if constexpr (MAPPED) {
    return blk[k] & BLK_ROW;
  } else {
    const int64_t r = k * s;
    return r < n ? r : n;
  }
}

// 16-byte shared-memory vector load and store.
template <typename S>
__device__ __forceinline__ Vec<S> lds16(const S* p) {
  Vec<S> r;
  if constexpr (sizeof(S) == 8) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    r.v[0] = t.x; r.v[1] = t.y;
  } else {
    const float4 t = *reinterpret_cast<const float4*>(p);
    r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
  }
  return r;
}
template <typename S>
__device__ __forceinline__ void sts16(S* p, const Vec<S>& r) {
  if constexpr (sizeof(S) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2(r.v[0], r.v[1]);
  } else {
    *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
  }
}

}  // namespace tdp
