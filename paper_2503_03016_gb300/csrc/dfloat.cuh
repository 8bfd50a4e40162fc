// Double-float arithmetic for the complex128 sweeps.
//
// GB300 executes FP64 at a small fraction of its FP32 rate (about 1.2 TFLOP/s against
// 80 TFLOP/s), so a complex128 gate computed in FP64 is bound by the FP64 pipe long
// before HBM.  Here a binary64 value is carried as an unevaluated sum hi + lo of two
// binary32 numbers (|lo| <= ulp(hi) / 2; 48 significant bits) and the gate products
// are built from FP32 operations with error-free transformations:
//   * TwoProd: the rounded product p = fl(a b) and its exact error a b - p from one
//     fused multiply-add (the error of a product is representable);
//   * TwoSum: the rounded sum s = fl(a + b) and its exact error in six additions
//     (Knuth, TAOCP Vol. 2, Sec. 4.2.2), for operands of any relative size.
// The packed FP32 instructions of sm_100 and later (two lanes per instruction) carry
// the real and the imaginary part of one output amplitude side by side.
//
// The conversions between the binary64 storage and hi + lo use integer operations and
// FP32 only (the IEEE 754 binary64 and binary32 encodings), so that no instruction of a
// sweep runs on the FP64 pipe:
//   * split: hi = the 24 leading bits of the 53-bit significand, rounded half up; the
//     remaining 29 bits, as a signed integer, times the binade's scale give lo (rounded
//     to 24 bits: the pair keeps 48-49 bits of the double);
//   * join: the bits of hi widened to binary64, plus lo counted in units of the last
//     place of that binary64 (one FP32 product and a conversion to integer); where hi is
//     a power of two and lo pulls the value into the binade below, whose unit is half
//     as large, the count is doubled.
//
// Range: the fast paths cover 2^-126 <= |x| < 2^127 on the way in (lo is dropped below
// 2^-74, an absolute change under 2^-98) and 2^-75 <= |hi| on the way out; zeros,
// smaller and larger values, infinities and NaNs take the general integer routines
// below.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qcgb {

// ---------------------------------------------------------------------------
// scalar conversions
// ---------------------------------------------------------------------------
// f * 2^k for a binary32 f (normal or zero), exact while the result stays normal
__device__ __forceinline__ float df_scale2(float f, int k) {
  const uint32_t u = __float_as_uint(f);
  const int fe = int((u >> 23) & 0xFFu);
  if (fe == 0) return f;
  const int ne = fe + k;
  if (ne >= 1 && ne <= 254) return __uint_as_float(u + uint32_t(int32_t(k) * 8388608));
  return ldexpf(f, k);  // out of the normal range
}

// binary64 -> (hi, lo) for any input.  x = s M 2^(e - 1075) with the 53-bit significand M.
static __device__ __noinline__ float2 df_split_general(double x) {
  const uint64_t b = uint64_t(__double_as_longlong(x));
  const bool neg = (b >> 63) != 0;
  const int e = int((b >> 52) & 0x7FFu);
  if (e == 0) return make_float2(neg ? -0.0f : 0.0f, 0.0f);  // zero; binary64 subnormals: below any amplitude
  if (e == 0x7FF) return make_float2(__double2float_rn(x), 0.0f);  // infinity or NaN
  const uint64_t M = (b & ((uint64_t(1) << 52) - 1)) | (uint64_t(1) << 52);
  const uint64_t hm = (M + (uint64_t(1) << 28)) >> 29;  // <= 2^24
  const int64_t rm = int64_t(M) - int64_t(hm << 29);    // |rm| <= 2^28
  float h = df_scale2(float(uint32_t(hm)), e - 1046);
  float l = df_scale2(float(rm), e - 1075);
  return neg ? make_float2(-h, -l) : make_float2(h, l);
}

// hi + lo -> binary64 for any pair: the two significands assembled as one integer and
// rounded to nearest (ties to even); lo below 2^-61 of hi is truncated before rounding.
static __device__ __noinline__ double df_join_general(float hi, float lo) {
  const uint32_t uh = __float_as_uint(hi), ul = __float_as_uint(lo);
  const int eh = int((uh >> 23) & 0xFFu), el = int((ul >> 23) & 0xFFu);
  if (eh == 255) return double(hi);
  if (eh == 0) return double(hi) + double(lo);  // zero or a binary32 subnormal
  int64_t Mh = int64_t((uh & 0x7FFFFFu) | 0x800000u);
  if (uh >> 31) Mh = -Mh;
  if (el == 0) return double(hi);  // lo zero or subnormal: below hi's binary64 unit
  int64_t Ml = int64_t((ul & 0x7FFFFFu) | 0x800000u);
  if (ul >> 31) Ml = -Ml;
  const int d = eh - el;
  int64_t S;
  int es;  // value = S 2^es
  if (d < 0) return double(hi) + double(lo);  // not a renormalised pair
  if (d <= 38) {
    S = Mh * (int64_t(1) << d) + Ml;
    es = el - 150;
  } else {
    S = Mh * (int64_t(1) << 38) + (Ml >> (d - 38));
    es = eh - 150 - 38;
  }
  if (S == 0) return 0.0;
  const bool neg = S < 0;
  uint64_t U = neg ? uint64_t(-S) : uint64_t(S);
  const int lead = 63 - __clzll((long long)U);
  int E;
  if (lead > 52) {
    const int sh = lead - 52;
    const uint64_t rem = U & ((uint64_t(1) << sh) - 1), half = uint64_t(1) << (sh - 1);
    U >>= sh;
    if (rem > half || (rem == half && (U & 1))) ++U;
    E = es + sh;
    if (U >> 53) {
      U >>= 1;
      ++E;
    }
  } else {
    U <<= (52 - lead);
    E = es - (52 - lead);
  }
  const uint64_t bexp = uint64_t(E + 52 + 1023);
  return __longlong_as_double((long long)((uint64_t(neg) << 63) | (bexp << 52) | (U & ((uint64_t(1) << 52) - 1))));
}

// binary64 -> hi + lo, fast path for biased exponents 897..1149
__device__ __forceinline__ void df_split(double x, float& hi, float& lo) {
  const uint32_t hw = uint32_t(__double2hiint(x)), lw = uint32_t(__double2loint(x));
  const uint32_t e = (hw >> 20) & 0x7FFu;
  const uint32_t sign = hw & 0x80000000u;
  if (e - 897u <= 252u) {
    // exponent and 23 fraction bits in place: (e - 896) is e - 128 modulo 256
    const uint32_t t = __funnelshift_l(lw, hw, 3);
    const uint32_t hb = ((t - 0x40000000u) & 0x7FFFFFFFu) + ((lw >> 28) & 1u);
    hi = __uint_as_float(hb | sign);
    // the 29 dropped bits, negative when hi was rounded up; scale 2^(e - 1075)
    const int32_t rm = int32_t(lw << 3) >> 3;
    const int se = max(int(e) - 948, 0);
    lo = __int2float_rn(rm) * __uint_as_float((uint32_t(se) << 23) | sign);
  } else if (e == 0u) {
    hi = __uint_as_float(sign);
    lo = 0.0f;
  } else {
    const float2 r = df_split_general(x);
    hi = r.x;
    lo = r.y;
  }
}

// hi + lo -> binary64 for a renormalised pair (|lo| <= ulp(hi) / 2)
__device__ __forceinline__ double df_join(float hi, float lo) {
  const uint32_t uh = __float_as_uint(hi);
  const uint32_t mag = uh & 0x7FFFFFFFu, eh = mag >> 23;
  const uint64_t sign = uint64_t(uh & 0x80000000u) << 32;
  if (eh - 52u <= 202u) {
    // lo / ulp64(hi), signed relative to hi: ulp64(hi) = 2^(eh - 179)
    float k = lo * __uint_as_float(((306u - eh) << 23) | (uh & 0x80000000u));
    if ((mag & 0x7FFFFFu) == 0u && k < 0.0f) k += k;
    const uint64_t D = (uint64_t(mag) << 29) + (uint64_t(896) << 52) + uint64_t(int64_t(__float2int_rn(k)));
    return __longlong_as_double((long long)(D | sign));
  }
  if (mag == 0u) return __longlong_as_double((long long)sign);
  return df_join_general(hi, lo);
}

// scalar double-float sums: a = (hi, lo).  dfs_add renormalises its result; dfs_acc
// (a += b without renormalising: TwoSum of the hi parts, the lo parts and the error
// added into lo) serves chains whose result is renormalised once at the end.
__device__ __forceinline__ float2 dfs_renorm(float2 a) {
  const float hi = __fadd_rn(a.x, a.y);
  return make_float2(hi, __fsub_rn(a.y, __fsub_rn(hi, a.x)));
}
__device__ __forceinline__ float2 dfs_acc(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bb = __fsub_rn(s, a.x);
  const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  return make_float2(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 dfs_add(float2 a, float2 b) { return dfs_renorm(dfs_acc(a, b)); }

// ---------------------------------------------------------------------------
// packed pairs: lane x and lane y are two independent double-floats
// ---------------------------------------------------------------------------
struct DF2 {
  float2 hi, lo;
};
// accumulator of a sum of products: s the exactly tracked sum of the rounded leading
// products, c the rounding errors and the cross terms
struct DF2Acc {
  float2 s, c;
};

// a - b rounded once (b * -1 is exact)
__device__ __forceinline__ float2 df2_sub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}

// a = x y, x given as (xh, -xh, xl): p = fl(xh yh); p - xh yh exactly by one fused
// multiply-add; the cross terms xh yl + xl yh rounded (yl xl, below 2^-48 of the
// product, is left out)
__device__ __forceinline__ void df2_first(DF2Acc& a, float2 xh, float2 nxh, float2 xl, DF2 y) {
  const float2 p = __fmul2_rn(xh, y.hi);
  const float2 ne = __ffma2_rn(nxh, y.hi, p);
  float2 t = __fmul2_rn(xh, y.lo);
  t = __ffma2_rn(xl, y.hi, t);
  a.s = p;
  a.c = df2_sub(t, ne);
}

// a += x y, with TwoSum of the running sum and the new leading product
__device__ __forceinline__ void df2_mac(DF2Acc& a, float2 xh, float2 nxh, float2 xl, DF2 y) {
  const float2 p = __fmul2_rn(xh, y.hi);
  const float2 ne = __ffma2_rn(nxh, y.hi, p);
  float2 c = df2_sub(a.c, ne);
  c = __ffma2_rn(xh, y.lo, c);
  c = __ffma2_rn(xl, y.hi, c);
  const float2 s = __fadd2_rn(a.s, p);
  const float2 bb = df2_sub(s, a.s);
  const float2 err = __fadd2_rn(df2_sub(a.s, df2_sub(s, bb)), df2_sub(p, bb));
  a.s = s;
  a.c = __fadd2_rn(c, err);
}

// a += h + l for a double-float pair (h, l): TwoSum of the running sum and h, the error
// and l into the error sum
__device__ __forceinline__ void df2_add(DF2Acc& a, float2 h, float2 l) {
  const float2 s = __fadd2_rn(a.s, h);
  const float2 bb = df2_sub(s, a.s);
  const float2 err = __fadd2_rn(df2_sub(a.s, df2_sub(s, bb)), df2_sub(h, bb));
  a.s = s;
  a.c = __fadd2_rn(a.c, __fadd2_rn(err, l));
}

// s + c renormalised by TwoSum: hi = fl(s + c) and lo its exact error
__device__ __forceinline__ DF2 df2_result(const DF2Acc& a) {
  const float2 hi = __fadd2_rn(a.s, a.c);
  const float2 bb = df2_sub(hi, a.s);
  const float2 lo = __fadd2_rn(df2_sub(a.s, df2_sub(hi, bb)), df2_sub(a.c, bb));
  return DF2{hi, lo};
}

}  // namespace qcgb
