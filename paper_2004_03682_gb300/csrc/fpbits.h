// Device helpers on IEEE-754 bit patterns: conversions done with integer
// operations, which GB300 issues at many times its FP64 rate.
#pragma once
#include <cstdint>

// The rare out-of-range cases below go through FP64 in functions of their own:
// inlined, the compiler may evaluate them ahead of the branch, and each FP64
// instruction holds GB300's FP64 pipe for many cycles.
static __device__ __noinline__ double scaled_i64_slow(long long R, int e) { return ldexp(double(R), e); }
static __device__ __noinline__ float f32_of_f64_slow(double x) { return __double2float_rn(x); }

// R 2^e as a double, R rounded to 53 bits (nearest, ties to even) with integer
// operations; the rare results outside the normal range take the FP64 route.
// Same value as ldexp(double(R), e).
__device__ __forceinline__ double scaled_i64(long long R, int e) {
  if (R == 0) return 0.0;
  const unsigned long long sgn = R < 0 ? (1ull << 63) : 0ull;
  unsigned long long m = R < 0 ? 0ull - (unsigned long long)R : (unsigned long long)R;
  const int lz = __clzll((long long)m);
  m <<= lz;  // leading one at bit 63
  unsigned long long mant = m >> 11;
  const unsigned long long rem = m & 0x7FFull;
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) ++mant;
  int ex = 63 - lz + e;  // |R| 2^e = (mant / 2^52) 2^ex
  if (mant >> 53) { mant >>= 1; ++ex; }
  const int be = ex + 1023;
  if (be <= 0 || be >= 2047) return scaled_i64_slow(R, e);
  return __longlong_as_double((long long)(sgn | (unsigned long long)(be) << 52 | (mant & 0xFFFFFFFFFFFFFull)));
}

// ---------------------------------------------------------------------------
// Double-single numbers: x = h + l with h, l FP32 (Dekker's double-length
// representation with FP32 as the base format): h is x rounded to 24 bits, l the
// rest rounded to 24 bits, 48 bits of x in all.  |x| < 2^-126 is flushed to zero;
// non-finite or too large x goes through the FP32 conversion (inf / NaN).
__device__ __forceinline__ float2 ds_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = int((b >> 52) & 0x7FF);
  const int fe = e - 896;  // biased FP32 exponent of x
  if (fe < 1) return make_float2(0.f, 0.f);
  if (fe > 254) return make_float2(f32_of_f64_slow(x), 0.f);
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;  // 53-bit significand
  unsigned long long hm = m >> 29;
  const unsigned long long rem = m & 0x1FFFFFFFull;
  if (rem > 0x10000000ull || (rem == 0x10000000ull && (hm & 1ull))) ++hm;  // nearest, ties to even
  const long long r = (long long)m - (long long)(hm << 29);                // the rest, |r| <= 2^28
  int hfe = fe;
  if (hm >> 24) {  // rounded up to 2^24
    hm >>= 1;
    ++hfe;
  }
  if (hfe > 254) return make_float2(f32_of_f64_slow(x), 0.f);
  const unsigned sgn = unsigned(b >> 63) << 31;
  const float h = __uint_as_float(sgn | (unsigned(hfe) << 23) | (unsigned(hm) & 0x7FFFFFu));
  // l = sign(x) r 2^(e - 1075): r rounded to 24 bits, then the exponent field moved
  unsigned lb = __float_as_uint(__int2float_rn(int(r)));
  int le = int((lb >> 23) & 0xFF);
  if (le) {
    le += e - 1075;
    lb = le >= 1 ? ((lb & 0x807FFFFFu) | (unsigned(le) << 23)) : 0u;  // below the normal range: dropped
  }
  return make_float2(h, __uint_as_float(lb ^ sgn));
}

// signed integer significand and exponent of a float: f = m 2^e
__device__ __forceinline__ void f32_parts(float f, int& m, int& e) {
  const unsigned u = __float_as_uint(f);
  const int be = int((u >> 23) & 0xFF);
  const int mag = be ? int((u & 0x7FFFFFu) | 0x800000u) : int(u & 0x7FFFFFu);
  e = be ? be - 150 : -149;
  m = (u >> 31) ? -mag : mag;
}

// h + l rounded to FP64 (nearest) with integer operations: both parts are placed
// in one int64 at the larger part's scale minus 38 bits (bits of the smaller part
// below 2^-62 of the larger are dropped), then scaled_i64 rounds once.
__device__ __forceinline__ double ds_to_double(float h, float l) {
  int mh, eh, ml, el;
  f32_parts(h, mh, eh);
  f32_parts(l, ml, el);
  if (mh == 0) { mh = ml; eh = el; ml = 0; }
  if (ml == 0) return scaled_i64((long long)mh, eh);
  const int E = max(eh, el) - 38;
  const int sh = eh - E, sl = el - E;  // <= 38 each
  const long long rh = sh >= 0 ? (long long)mh << sh : (sh > -40 ? (long long)mh >> -sh : 0);
  const long long rl = sl >= 0 ? (long long)ml << sl : (sl > -40 ? (long long)ml >> -sl : 0);
  return scaled_i64(rh + rl, E);
}

// s + c += a b for double-single a = (ah, al), b = (bh, bl): the product's high part
// exactly (Dekker's product through FMA), the cross terms rounded (al bl dropped),
// s carried exactly with Knuth's two-sum, every rounding error gathered in c.
__device__ __forceinline__ void ds_mac(float& s, float& c, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  const float pe = __fmaf_rn(ah, bh, -p);
  const float lo = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, pe));
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, lo));
}
