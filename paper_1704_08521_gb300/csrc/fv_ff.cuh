// Float-float ("double-float") arithmetic on the FP32 pipes.
//
// On GB300 the FP64 units run at ~1/70 of the FP32 rate, and so do the
// float <-> double conversion instructions.  The mixed-precision SIMPLE loop
// therefore keeps its state as unevaluated sums hi + lo of two floats
// (Dekker 1971; Knuth's TwoSum), about 48 significant bits, and converts
// at the float64 API boundary with integer bit manipulation only.
//
// Conversions (exact rounding rules, host and device):
//   f64_round_f32(d)  : d rounded to the nearest float (ties to even);
//                       |d| beyond the float range -> +-inf, below the
//                       normal range (2^-126) -> +-0.
//   f64_split(d)      : hi = f64_round_f32(d), lo = nearest float to d - hi
//                       (lo = 0 when d - hi is below 2^-126).
//   ff_join(hi, lo)   : the float64 nearest to hi + lo (ties: truncation of
//                       bits below 2^-38 |hi|, see the body).
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define FF_HD __host__ __device__ __forceinline__
#else
#define FF_HD inline
#endif

namespace fv {

struct ff {
  float hi, lo;
};

FF_HD uint64_t bits64(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t b;
  memcpy(&b, &d, 8);
  return b;
#endif
}

FF_HD double from_bits64(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, 8);
  return d;
#endif
}

FF_HD uint32_t bits32(float f) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__float_as_uint(f);
#else
  uint32_t b;
  memcpy(&b, &f, 4);
  return b;
#endif
}

FF_HD float from_bits32(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, 4);
  return f;
#endif
}

FF_HD int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

// d rounded to the nearest float, integer operations only.  Values whose
// float exponent is normal (2^-126 <= |d| < 2^128 before rounding) take a
// short path: the float's bits are the double's sign, rebiased exponent and
// top 23 mantissa bits, plus one for round-to-nearest-even (a carry out of
// the mantissa steps the exponent, up to infinity, as IEEE rounding does);
// zeros, tiny values, overflow, infinities and NaNs take the general path.
FF_HD float f64_round_f32(double d) {
  const uint64_t b = bits64(d);
  const uint32_t hw = (uint32_t)(b >> 32), lw = (uint32_t)b;
  const uint32_t mag = hw & 0x7fffffffu;
  if (mag - 0x38100000u < 0x47f00000u - 0x38100000u) {   // double exponent 897 .. 1150
    uint32_t r = (hw & 0x80000000u) | ((mag - 0x38000000u) << 3) | (lw >> 29);
    const uint32_t rem = lw & 0x1fffffffu;
    r += (rem > 0x10000000u) | ((rem == 0x10000000u) & r);
    return from_bits32(r);
  }
  const uint32_t sign = (uint32_t)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ff);
  const uint64_t m = b & 0xfffffffffffffULL;
  if (e == 0x7ff) return from_bits32(sign | 0x7f800000u | (m ? 0x400000u : 0u));
  int ef = e - 1023 + 127;
  if (ef <= 0) return from_bits32(sign);
  uint32_t mr = (uint32_t)(m >> 29);
  const uint32_t rem = (uint32_t)(m & 0x1fffffffULL);
  if (rem > 0x10000000u || (rem == 0x10000000u && (mr & 1u))) {
    if (++mr == 0x800000u) { mr = 0; ++ef; }
  }
  if (ef >= 255) return from_bits32(sign | 0x7f800000u);
  return from_bits32(sign | ((uint32_t)ef << 23) | mr);
}

// exact float -> double, integer operations only (float denormals -> 0)
FF_HD double f32_to_f64(float f) {
  const uint32_t b = bits32(f);
  const uint64_t sign = (uint64_t)(b >> 31) << 63;
  const int ef = (int)((b >> 23) & 0xff);
  const uint64_t m = b & 0x7fffffu;
  if (ef == 0) return from_bits64(sign);
  if (ef == 255) return from_bits64(sign | 0x7ff0000000000000ULL | (m << 29));
  return from_bits64(sign | ((uint64_t)(ef - 127 + 1023) << 52) | (m << 29));
}

// 2^k as a float for -126 <= k <= 127 (else 0 / inf)
FF_HD float pow2f(int k) {
  if (k < -126) return 0.0f;
  if (k > 127) return from_bits32(0x7f800000u);
  return from_bits32((uint32_t)(k + 127) << 23);
}

FF_HD ff f64_split(double d) {
  const uint64_t b = bits64(d);
  const int e = (int)((b >> 52) & 0x7ff);
  ff r;
  r.hi = f64_round_f32(d);
  r.lo = 0.0f;
  const int ef = e - 1023 + 127;
  if (e == 0x7ff || ef <= 0 || ef >= 255) return r;
  // d - hi = (full significand - rounded significand) * 2^(e - 1075)
  const uint64_t full = (b & 0xfffffffffffffULL) | (1ULL << 52);
  const uint32_t hb = bits32(r.hi);
  const int eh = (int)((hb >> 23) & 0xff);                  // may be ef + 1 after rounding
  if (eh == 255) return r;
  const uint64_t hsig = ((uint64_t)(hb & 0x7fffffu) | (1ULL << 23)) << (29 + (eh - ef));
  const int64_t diff = (int64_t)full - (int64_t)hsig;      // |diff| <= 2^28 (or 2^29)
  if (diff == 0) return r;
  const float mag = (float)(uint32_t)(diff < 0 ? -diff : diff);   // <= 30 bits
  const int k = e - 1075;                                  // in [-178, 75] for normal floats
  float lo = mag * pow2f(k / 2) * pow2f(k - k / 2);
  if ((int64_t)(b >> 63) != 0) lo = -lo;
  r.lo = diff < 0 ? -lo : lo;
  return r;
}

// hi + lo as a float64, integer operations only.
FF_HD double ff_join(float hi, float lo) {
  const uint32_t hb = bits32(hi), lb = bits32(lo);
  const int eh = (int)((hb >> 23) & 0xff), el = (int)((lb >> 23) & 0xff);
  if (eh == 255) return f32_to_f64(hi);                    // inf / nan
  if (el == 0) return f32_to_f64(hi);
  if (eh == 0) return f32_to_f64(lo);
  // signed 24-bit significands, values M * 2^(E - 150)
  int64_t Mh = (int64_t)((hb & 0x7fffffu) | 0x800000u);
  int64_t Ml = (int64_t)((lb & 0x7fffffu) | 0x800000u);
  if (hb >> 31) Mh = -Mh;
  if (lb >> 31) Ml = -Ml;
  int sh = eh - el;
  if (sh < 0) {                                              // |lo| > |hi|: swap the roles
    const int64_t t = Mh; Mh = Ml; Ml = t;
    sh = -sh;
  }
  const int ehi = eh > el ? eh : el, elo = eh > el ? el : eh;
  int64_t S;
  int E;                                                     // S * 2^(E - 150)
  if (sh <= 38) {
    S = (Mh << sh) + Ml;
    E = elo;
  } else {
    S = (Mh << 29) + (Ml >> (sh - 29));                     // bits of lo below 2^-29 ulp dropped
    E = ehi - 29;
  }
  if (S == 0) return 0.0;
  const uint64_t sign = S < 0 ? (1ULL << 63) : 0ULL;
  uint64_t A = (uint64_t)(S < 0 ? -S : S);
  // normalise A to 53 significant bits with round-to-nearest-even
  const int lz = clz64(A);
  const int top = 63 - lz;                                   // index of the leading bit
  int exp2 = E - 150 + top;                                  // value = 1.xxx * 2^exp2
  if (top > 52) {
    const int drop = top - 52;
    const uint64_t rem = A & ((1ULL << drop) - 1);
    const uint64_t half = 1ULL << (drop - 1);
    A >>= drop;
    if (rem > half || (rem == half && (A & 1ULL))) {
      ++A;
      if (A == (1ULL << 53)) { A >>= 1; ++exp2; }
    }
  } else {
    A <<= (52 - top);
  }
  if (exp2 < -1022) return from_bits64(sign);
  return from_bits64(sign | ((uint64_t)(exp2 + 1023) << 52) | (A & 0xfffffffffffffULL));
}

// ---- float-float arithmetic (TwoSum, TwoProd by FMA) ----------------------
FF_HD float fma_f(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return __builtin_fmaf(a, b, c);
#endif
}

FF_HD ff two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float err = (a - (s - bb)) + (b - bb);
  return {s, err};
}

FF_HD ff fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}

FF_HD ff ff_add(ff x, ff y) {
  ff s = two_sum(x.hi, y.hi);
  const ff t = two_sum(x.lo, y.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}

FF_HD ff ff_neg(ff x) { return {-x.hi, -x.lo}; }
FF_HD ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

FF_HD ff ff_add_f(ff x, float y) {
  ff s = two_sum(x.hi, y);
  s.lo += x.lo;
  return fast_two_sum(s.hi, s.lo);
}

FF_HD ff ff_mul(ff x, ff y) {
  const float p = x.hi * y.hi;
  float e = fma_f(x.hi, y.hi, -p);
  e = fma_f(x.hi, y.lo, e);
  e = fma_f(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

FF_HD ff ff_mul_f(ff x, float y) {
  const float p = x.hi * y;
  float e = fma_f(x.hi, y, -p);
  e = fma_f(x.lo, y, e);
  return fast_two_sum(p, e);
}

// ---- Krylov-basis helpers: a truncating split and a multiply-add ---------
//
// f64_split_trunc(d): hi = the float of d's leading 24 significant bits,
// lo = the float of the next 23, so |d - hi - lo| < 2^-46 |d|; integer and
// FP32 operations only (about a dozen, no conversion instructions).
// |d| < 2^-126 gives 0 + 0; 2^-126 <= |d| < 2^-80 gives lo = 0 (an error
// below 2^-103; lo would not be a normal float); |d| >= 2^128, inf and nan
// give hi = nan.
FF_HD ff f64_split_trunc(double d) {
  const uint64_t b = bits64(d);
  const uint32_t h32 = (uint32_t)(b >> 32), l32 = (uint32_t)b;
  const uint32_t sign = h32 & 0x80000000u;
  const uint32_t e = (h32 >> 20) & 0x7ffu;
  if (e < 897u) return {0.0f, 0.0f};
  if (e > 1150u) return {from_bits32(0x7fc00000u), 0.0f};
  // exponent rebiased 1023 -> 127 in place, then the top 23 fraction bits
  const uint32_t hb = (((h32 & 0x7fffffffu) - (896u << 20)) << 3) | (l32 >> 29);
  ff r{from_bits32(sign | hb), 0.0f};
  const uint32_t ef = e - 896u;
  if (ef >= 47u) {
    // the next 23 fraction bits f: (1 + f 2^-23) 2^k - 2^k = f 2^(k-23), exact
    // and (k >= -103) a normal float or zero
    const uint32_t E = (ef - 23u) << 23;
    const float t = from_bits32(E | ((l32 & 0x1fffffffu) >> 6)) - from_bits32(E);
    r.lo = from_bits32(bits32(t) | sign);
  }
  return r;
}

// acc += a * b: the product by TwoProd (FMA) plus the two cross terms, added
// by TwoSum and renormalised, so each call adds a relative error of about
// 2^-47 of |acc| + |a b| (the lo * lo term, below 2^-46 |a b|, is dropped).
FF_HD void ff_mad(ff& acc, ff a, ff b) {
  const float p = a.hi * b.hi;
  float e = fma_f(a.hi, b.hi, -p);
  e = fma_f(a.hi, b.lo, e);
  e = fma_f(a.lo, b.hi, e);
  ff s = two_sum(acc.hi, p);
  s.lo += acc.lo + e;
  acc = fast_two_sum(s.hi, s.lo);
}

// ---- a float-float number with arithmetic operators, so that the momentum
// stencil template can run in ~48-bit arithmetic on the FP32 pipes
struct ffn {
  float hi, lo;
  FF_HD ffn() : hi(0.f), lo(0.f) {}
  FF_HD ffn(float a) : hi(a), lo(0.f) {}
  FF_HD ffn(int a) : hi((float)a), lo(0.f) {}
  FF_HD ffn(double a) : hi((float)a), lo(0.f) {}   // literals only (0, 0.5, 0.25)
  FF_HD ffn(float a, float b) : hi(a), lo(b) {}
#ifdef __CUDACC__
  __host__ __device__ ffn(float2 a) : hi(a.x), lo(a.y) {}
#endif
  FF_HD ffn(ff a) : hi(a.hi), lo(a.lo) {}
};

FF_HD ffn operator+(ffn a, ffn b) { return ffn(ff_add({a.hi, a.lo}, {b.hi, b.lo})); }
FF_HD ffn operator-(ffn a, ffn b) { return ffn(ff_sub({a.hi, a.lo}, {b.hi, b.lo})); }
FF_HD ffn operator*(ffn a, ffn b) { return ffn(ff_mul({a.hi, a.lo}, {b.hi, b.lo})); }
FF_HD ffn operator-(ffn a) { return ffn(-a.hi, -a.lo); }
FF_HD ffn& operator+=(ffn& a, ffn b) { a = a + b; return a; }
FF_HD ffn& operator-=(ffn& a, ffn b) { a = a - b; return a; }

}  // namespace fv
