// Float-float arithmetic for the FP64-storage hopping kernel: a real number is
// the unevaluated sum hi + lo of two FP32 numbers (|lo| below one unit in the
// last place of hi), about 46 significant bits.  GB300 runs FP64 at 1/74 of
// its FP32 rate, so the FP64 hopping term (Eq. 2), which is FP64-ALU-bound,
// runs faster on the FP32 units in this form.
//
// Sums use the error-free TwoSum (Knuth): s = fl(a + b) and the exact
// rounding error (a - (s - bb)) + (b - bb), bb = s - a; products the fused
// form of Dekker's TwoProduct: the rounding error of p = fl(a b) is exactly
// fma(a, b, -p).  The sloppy float-float sum and the product then follow the
// double-word algorithms of Dekker (1971) with FP32 words; every FP32
// operation is an explicitly rounded intrinsic so that the compiler cannot
// contract a product and a sum into one fma and lose the error term.
//
// FP64 values enter through their bit patterns (integer operations only: hi
// takes the top 24 significant bits, lo the next 23), so that loading costs
// no FP64 or conversion-unit instructions; values below 2^-126 in magnitude
// load as zero (they cannot be float-float numbers) and values beyond the
// FP32 range as infinity.  Results leave as hi + lo in FP64.
#pragma once
#include "dwf_internal.cuh"

struct __align__(8) dfl {
  float hi, lo;
  __device__ __forceinline__ dfl() : hi(0.f), lo(0.f) {}
  __device__ __forceinline__ dfl(float a) : hi(a), lo(0.f) {}
  __device__ __forceinline__ dfl(int a) : hi((float)a), lo(0.f) {}  // small integers
  __device__ __forceinline__ dfl(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ dfl(double a) {
    hi = __double2float_rn(a);
    lo = __double2float_rn(a - (double)hi);
  }
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
  __device__ __forceinline__ explicit operator float() const { return __fadd_rn(hi, lo); }
};

// s + e = a + b exactly
__device__ __forceinline__ dfl dfl_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dfl(s, e);
}

// s + e = a + b exactly, for |a| >= |b| (or a = 0)
__device__ __forceinline__ dfl dfl_quick(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfl(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  const dfl s = dfl_two_sum(a.hi, b.hi);
  return dfl_quick(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dfl_quick(p, e);
}
// a b + c with one normalisation
__device__ __forceinline__ dfl fma(dfl a, dfl b, dfl c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const dfl s = dfl_two_sum(p, c.hi);
  return dfl_quick(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}
// a / b: two quotient digits (scalars of the epilogue only)
__device__ __forceinline__ dfl operator/(dfl a, dfl b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const dfl r = a - b * dfl(q1);
  return dfl_quick(q1, __fdiv_rn(r.hi, b.hi));
}
__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { return a = a + b; }
__device__ __forceinline__ dfl& operator-=(dfl& a, dfl b) { return a = a - b; }
__device__ __forceinline__ dfl& operator*=(dfl& a, dfl b) { return a = a * b; }

// Products with the hopping sign s = +-1 (the projection and the lower
// spins): a sign change, not a multiplication.
__device__ __forceinline__ dfl sg_mul(dfl sg, dfl x) { return sg.hi < 0.f ? -x : x; }
__device__ __forceinline__ dfl sg_fma(dfl sg, dfl x, dfl y) { return sg.hi < 0.f ? y - x : y + x; }

// FP64 bit pattern (high word hw, low word lw) -> float-float, integer
// operations only.
__device__ __forceinline__ dfl dfl_from_bits(unsigned hw, unsigned lw) {
  const unsigned sign = hw & 0x80000000u;
  const unsigned mag = hw & 0x7FFFFFFFu;
  const unsigned e = mag >> 20;
  if (e < 897u) return dfl(0.f, 0.f);
  if (e > 1150u) return dfl(__int_as_float((int)(sign | 0x7F800000u)), 0.f);
  // hi: the exponent rebiased (1023 -> 127) and the top 23 stored mantissa bits
  const float hi = __int_as_float((int)(sign | ((mag - (896u << 20)) << 3) | (lw >> 29)));
  // lo: the remaining 29 mantissa bits (their top 23), value m 2^(e - 1069)
  const unsigned m23 = (lw & 0x1FFFFFFFu) >> 6;
  float lo = 0.f;
  if (e >= 943u) {
    const float m = __fsub_rn(__int_as_float((int)(0x4B000000u | m23)), 8388608.0f);  // exact
    const float scale = __int_as_float((int)((e - 942u) << 23));                      // 2^(e - 1069)
    lo = __int_as_float(__float_as_int(__fmul_rn(m, scale)) | (int)sign);
  }
  return dfl(hi, lo);
}

// FP64 storage of the float-float hopping kernel: the same bytes as double2,
// a distinct type so that loads and stores convert.
struct __align__(16) f64s {
  double x, y;
};

__device__ __forceinline__ cpx<dfl> ld_c(const f64s* p) {
  const int4 w = *(const int4*)p;
  cpx<dfl> z;
  z.re = dfl_from_bits((unsigned)w.y, (unsigned)w.x);
  z.im = dfl_from_bits((unsigned)w.w, (unsigned)w.z);
  return z;
}
__device__ __forceinline__ void st_c(f64s* p, cpx<dfl> z) {
  *(double2*)p = make_double2((double)z.re.hi + (double)z.re.lo, (double)z.im.hi + (double)z.im.lo);
}

template <>
struct Prec<DWF_P_DF> {
  typedef f64s S;     // stored complex (FP64)
  typedef dfl R;      // arithmetic
  typedef double2 LS; // stored link element (FP64 links)
};

template <>
struct PartialSum<dfl> {
  double s = 0.0;
  __device__ __forceinline__ void add(dfl x) { s += (double)x.hi + (double)x.lo; }
  __device__ __forceinline__ double value() const { return s; }
};
