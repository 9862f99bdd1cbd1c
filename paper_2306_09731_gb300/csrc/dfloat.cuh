// dfloat.cuh - double-float arithmetic for the refinement passes.
//
// A dfl is the unevaluated sum hi + lo of two FP32 numbers with |lo| at most
// about half an ulp of hi: a 48-bit significand with the FP32 exponent range.
// On a part whose FP32 rate is 58 times its FP64 rate, an FFT in this format
// costs about ten FP32 instructions per FP64 operation it replaces and still
// resolves relative errors near 1e-14, far below what the GMRES tolerance test
// of the refinement residual needs.
//
// Building blocks (error-free transformations of two FP32 numbers):
//   two_sum       Knuth's TwoSum: s + e == a + b exactly, any magnitudes
//   fast_two_sum  Dekker's FastTwoSum: the same when |a| >= |b| (or a == 0)
//   product       a*b - fl(a*b) is exact through one FMA (TwoProd)
// Addition is TwoSum of the high parts with the low parts and the TwoSum
// error added in FP32, left unnormalised: the absolute error is a small
// multiple of u^2 (|a| + |b|), u = 2^-24 (the two FP32 additions of terms of
// size u |a| and u |b|). That is the normwise bound the error analysis of an
// FFT uses; it holds under cancellation, where a relative bound does not, and
// it does not need |lo| <= ulp(hi)/2 of its inputs. Dropping the final
// FastTwoSum of Dekker's add2 saves 3 of 11 instructions; products and the
// complex twiddle products end in a FastTwoSum and renormalise, so a low part
// grows to at most a few u |hi| over the adds of one radix-8 butterfly chain.
// renorm() restores |lo| <= ulp(hi)/2 where a consumer relies on it (the
// Newton reciprocal). Multiplication is the FMA form of Dekker's mul2 (relative
// error a few u^2). Every step uses explicit round-to-nearest intrinsics, so
// the compiler can neither contract a product into an addition nor reorder an
// error term.
#pragma once
#include <type_traits>
#include <cuda_runtime.h>

#include "fft_core.cuh"

namespace sgn {

struct __align__(8) dfl {
  float hi, lo;
  dfl() = default;
  __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dfl(float v) : hi(v), lo(0.0f) {}
  __host__ __device__ constexpr dfl(int v) : hi((float)v), lo((float)((double)v - (double)(float)v)) {}
  // nearest split of an FP64 value (folded at compile time for constants)
  __host__ __device__ constexpr dfl(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  // (device passes that write FP64 use dfl_to_f64, which avoids the conversions)
  __host__ __device__ explicit operator float() const { return hi; }
};

// Split of an FP64 value into hi + lo without FP64 instructions (a conversion
// through FP64 arithmetic keeps the slow FP64 pipe of this part busy in the
// passes that read FP64 spectra). hi: the sign, the exponent and the top 23
// stored mantissa bits (truncated); lo: the remaining 29 bits, turned into an
// FP32 number with two exponent-bias tricks (2^23 + b - 2^23 is exact for
// b < 2^23) and one FMA that rounds them to 24 bits, then scaled by
// 2^(e - 1075) exactly. |lo| < ulp(hi), so hi + lo carries 47 bits. Branch
// free (selects only): magnitudes below 2^-74 keep no low part and below
// 2^-126 flush to a signed zero, beyond the FP32 range become infinite, NaN
// stays NaN: the double-float passes work within the FP32 exponent range.
__device__ __forceinline__ dfl dfl_from_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned top = (unsigned)(b >> 32);
  const unsigned sign = top & 0x80000000u;
  const int e = (int)((top >> 20) & 0x7ffu);
  float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
  const float fb = __fsub_rn(__uint_as_float(0x4b000000u | (unsigned)(b & 0x7fffffu)), 8388608.0f);
  const float fa = __fsub_rn(__uint_as_float(0x4b000000u | (unsigned)((b >> 23) & 0x3fu)), 8388608.0f);
  float lo = __fmul_rn(__fmaf_rn(fa, 8388608.0f, fb), __uint_as_float((unsigned)(e - 948) << 23));
  lo = sign ? -lo : lo;
  if (e < 949) lo = 0.0f;
  if (e < 897) hi = __uint_as_float(sign);
  if (e > 1150) {
    const bool nan = e == 2047 && (b & 0xfffffffffffffull) != 0ull;
    hi = __uint_as_float(sign | (nan ? 0x7fc00000u : 0x7f800000u));
    lo = 0.0f;
  }
  return dfl(hi, lo);
}

// hi + lo rounded to FP64 with one FP64 addition: each part is widened by
// placing its bits instead of a conversion instruction (selects only: FP32
// subnormals, below 2^-126, widen to zero; infinities and NaN keep their kind).
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  const unsigned long long e64 = ex == 0u ? 0ull : (ex == 0xffu ? 0x7ffull : (unsigned long long)(ex + 896u));
  const unsigned long long m64 = ex == 0u ? 0ull : (unsigned long long)(u & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) | (e64 << 52) | m64));
}
__device__ __forceinline__ double dfl_to_f64(dfl a) { return f32_to_f64_bits(a.hi) + f32_to_f64_bits(a.lo); }

// FP64 -> FP32 rounded to nearest (the split's two parts added in FP32; the
// range rules of dfl_from_f64) without an FP64-pipe conversion
__device__ __forceinline__ float f64_to_f32_bits(double x) {
  const dfl d = dfl_from_f64(x);
  return __fadd_rn(d.hi, d.lo);
}

// conversions between the storage types of the passes, off the FP64 pipe
template <typename TO, typename TI>
__device__ __forceinline__ TO cvt(TI v) {
  if constexpr (std::is_same<TI, dfl>::value && std::is_same<TO, double>::value)
    return dfl_to_f64(v);
  else if constexpr (sizeof(TO) == 4 && sizeof(TI) == 8)
    return f64_to_f32_bits(v);
  else if constexpr (sizeof(TO) == 8 && sizeof(TI) == 4)
    return f32_to_f64_bits(v);
  else
    return (TO)v;
}

__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dfl(s, e);
}

__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfl(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  const dfl s = two_sum(a.hi, b.hi);
  return dfl(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
// |lo| <= ulp(hi)/2 again (TwoSum: exact also after a cancellation in hi)
__device__ __forceinline__ dfl renorm(dfl a) { return two_sum(a.hi, a.lo); }
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { return a = a + b; }
__device__ __forceinline__ dfl& operator-=(dfl& a, dfl b) { return a = a - b; }

__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
// product with a plain FP32 factor
__device__ __forceinline__ dfl mul_f(dfl a, float b) {
  const float p = __fmul_rn(a.hi, b);
  const float e = __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p));
  return fast_two_sum(p, e);
}
// exact scaling by a power of two (no overflow or underflow assumed)
__device__ __forceinline__ dfl scale_pow2(dfl a, float s) { return dfl(__fmul_rn(a.hi, s), __fmul_rn(a.lo, s)); }

// 1/b: FP32 reciprocal r0, then one Newton step r0 + r0 (1 - b r0). The
// residual 1 - b.hi r0 is exact through the FMA (it is below 2^-23 in size
// and has no bits below 2^-48), so the step doubles the 24 correct bits.
__device__ __forceinline__ dfl recip(dfl b) {
  b = renorm(b);
  const float r0 = __frcp_rn(b.hi);
  const float e = __fmaf_rn(-b.lo, r0, __fmaf_rn(-b.hi, r0, 1.0f));
  return fast_two_sum(r0, __fmul_rn(r0, e));
}
// a/b: quotient of the high parts, corrected by the df remainder a - b q1
__device__ __forceinline__ dfl operator/(dfl a, dfl b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const dfl r = renorm(a - mul_f(b, q1));  // the remainder cancels in its high part
  return fast_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}

// --------------------------------------------------- complex and memory
// a*b + SGN*c*d with the two exact high products gathered before one TwoSum:
// 19 instructions, against 25 for two products and a sum. The error terms
// (product errors and the cross products with the low parts) are summed in
// FP32, so the absolute error stays a few u^2 (|a b| + |c d|).
template <int SGN>
__device__ __forceinline__ dfl dot2_df(dfl a, dfl b, dfl c, dfl d) {
  const float ch = SGN > 0 ? c.hi : -c.hi;
  const float cl = SGN > 0 ? c.lo : -c.lo;
  const float p = __fmul_rn(a.hi, b.hi);
  const float q = __fmul_rn(ch, d.hi);
  const float ep = __fmaf_rn(a.hi, b.hi, -p);
  const float eq = __fmaf_rn(ch, d.hi, -q);
  float e = __fadd_rn(ep, eq);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  e = __fmaf_rn(ch, d.lo, e);
  e = __fmaf_rn(cl, d.hi, e);
  const dfl s = two_sum(p, q);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, e));
}

template <>
__device__ __forceinline__ cpx<dfl> cmul(cpx<dfl> a, cpx<dfl> b) {
  return mk(dot2_df<-1>(a.x, b.x, a.y, b.y), dot2_df<1>(a.x, b.y, a.y, b.x));
}
// a * conj(b)
template <>
__device__ __forceinline__ cpx<dfl> cmulc(cpx<dfl> a, cpx<dfl> b) {
  return mk(dot2_df<1>(a.x, b.x, a.y, b.y), dot2_df<-1>(a.y, b.x, a.x, b.y));
}

template <>
__device__ __forceinline__ cpx<dfl> ldg(const cpx<dfl>* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return mk(dfl(v.x, v.y), dfl(v.z, v.w));
}
template <>
__device__ __forceinline__ dfl ldr(const dfl* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return dfl(v.x, v.y);
}

// 16-byte elements, eight to a 128-byte shared-memory row: the slot is XOR-ed
// with (p >> 3) & 7 within its aligned group of 8, which spreads the stride-8
// writes of the first stage (and the 64a + b writes of the second) over the
// whole row, as the FP64 layout's padding does, without the padding: the
// buffers of a length-N transform take N elements (unpadded_smem).
template <>
__device__ __forceinline__ int sidx<dfl>(int p, int lcs) {
  return (p ^ ((p >> 3) & 7)) << lcs;
}
template <>
struct unpadded_smem<dfl> {
  static constexpr bool value = true;
};

}  // namespace sgn
