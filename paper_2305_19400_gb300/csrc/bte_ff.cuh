// bte_ff.cuh -- double-float ("ff") arithmetic on pairs of bands, for the FP64
// mode's sweep on a GPU whose FP64 pipe (2 DFMA/clk/SM) is far slower than
// its FP32 pipe.
//
// A value is held as an unevaluated sum h + l of two floats with
// |l| <= ulp(h)/2 after normalisation: 48 significant bits, relative
// rounding about 2^-48 per operation (Dekker 1971, "A floating-point
// technique for extending the available precision"; Joldes, Muller, Popescu
// 2017, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic").  One lane of the FP64 sweep holds two bands, so a
// pair of bands is kept as two 64-bit registers: H = (h_b, h_b+1) and
// L = (l_b, l_b+1), and every operation is one packed add/sub/mul/fma.f32x2
// instruction of sm_100+ for both bands.  In memory an ff pair of bands takes
// the same 16 bytes as two doubles, laid out h_b, h_b+1, l_b, l_b+1.
//
// Building blocks (all in round-to-nearest, no fused contractions beyond the
// FMAs written out):
//   TwoSum (Knuth): s = fl(a + b), e = a + b - s exactly, for any a, b.
//   Fast2Sum (Dekker): the same when |a| >= |b|.
//   TwoProd via FMA: p = fl(a b), e = fma(a, b, -p) = a b - p exactly.
// The conversions between doubles and ff pairs use integer operations only
// (no FP64 or int/float conversion instruction on the common paths: on GB300
// those share the slow FP64 pipe, measured): a double x with 2^-74 <= |x| < 2^127 splits into
// hi = x rounded to 24 bits and lo = x - hi rounded to 24 bits (error below
// 2^-49 |x|); other values (zero, tiny, huge, Inf, NaN) become (float(x), 0).
#pragma once
#include <cuda_runtime.h>

namespace bte {
namespace ff {

using x2 = unsigned long long;  // two floats (bands b, b+1) in one 64-bit register

__device__ __forceinline__ x2 add(x2 a, x2 b) {
  x2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ x2 sub(x2 a, x2 b) {
  x2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ x2 mul(x2 a, x2 b) {
  x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ x2 fma(x2 a, x2 b, x2 c) {
  x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
// -a by flipping the two sign bits.  (Written as a packed subtract from zero,
// the negated product in TwoProd's fma(a, b, -fl(a b)) measured float-level
// errors on GB300: the error term was lost.  The bit flip keeps it exact.)
__device__ __forceinline__ x2 neg(x2 a) { return a ^ 0x8000000080000000ull; }
__device__ __forceinline__ x2 pack(float a, float b) {
  return (x2)__float_as_uint(a) | ((x2)__float_as_uint(b) << 32);
}
__device__ __forceinline__ float lo_of(x2 a) { return __uint_as_float((unsigned)a); }
__device__ __forceinline__ float hi_of(x2 a) { return __uint_as_float((unsigned)(a >> 32)); }

// A pair of bands in double-float form: band b = lo_of(h) + lo_of(l), band
// b + 1 = hi_of(h) + hi_of(l).
struct P2 {
  x2 h, l;
};

__device__ __forceinline__ P2 zero() { return P2{0ull, 0ull}; }

// s + e = a + b exactly (Knuth's TwoSum, 6 operations).
__device__ __forceinline__ void two_sum(x2 a, x2 b, x2& s, x2& e) {
  s = add(a, b);
  const x2 bv = sub(s, a);
  e = add(sub(a, sub(s, bv)), sub(b, bv));
}

// Normalised pair of an unnormalised one (Fast2Sum; |h| >= |l| holds for the
// sums built here, whose low parts stay a few ulps of h).
__device__ __forceinline__ P2 norm(P2 s) {
  P2 r;
  r.h = add(s.h, s.l);
  r.l = sub(s.l, sub(r.h, s.h));
  return r;
}

// c * u with the low-times-low term (2^-48 relative) left out.
__device__ __forceinline__ P2 mul(const P2& c, const P2& u) {
  P2 p;
  p.h = mul(c.h, u.h);
  x2 e = fma(c.h, u.h, neg(p.h));  // exact error of p.h
  e = fma(c.h, u.l, e);
  p.l = fma(c.l, u.h, e);
  return p;
}

// x + y of two (unnormalised) pairs: TwoSum of the high parts, the low parts
// and the rounding error added (left unnormalised).
__device__ __forceinline__ P2 add(const P2& x, const P2& y) {
  P2 r;
  x2 e;
  two_sum(x.h, y.h, r.h, e);
  r.l = add(add(x.l, y.l), e);
  return r;
}

// s += p (s left unnormalised: its low part collects p's and the rounding error).
__device__ __forceinline__ void acc(P2& s, const P2& p) {
  x2 h, e;
  two_sum(s.h, p.h, h, e);
  s.h = h;
  s.l = add(s.l, add(p.l, e));
}

// ---------------------------------------------------------------- conversions
// Round-to-nearest split of one double (see the header), on the two 32-bit
// words of its bits.
__device__ __forceinline__ void split(double x, float& h, float& l) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sgn = hi & 0x80000000u;
  const unsigned ahi = hi & 0x7fffffffu;  // |x|: ahi, lo
  const unsigned e = ahi >> 20;
  if (e - 949u <= 200u) {  // 2^-74 <= |x| < 2^127
    // |x| to 24 significant bits, ties away from zero: add 2^28 (carry into
    // the high word) and keep the low word's top 3 bits
    const unsigned lo2 = lo + 0x10000000u;
    const unsigned ahr = ahi + (lo2 < lo ? 1u : 0u);
    const unsigned lor = lo2 & 0xe0000000u;
    h = __uint_as_float((((ahr << 3) | (lor >> 29)) - (896u << 23)) | sgn);  // rebias 1023 -> 127
    const int k = (int)(lo - lor);                        // |x| - hi in units of 2^(e-1075)
    const float sc = __uint_as_float((e - 948u) << 23);  // 2^(e - 1075)
    // k sc rounded to float without an int-to-float conversion (those run on
    // the slow FP64 pipe): |k| <= 2^28 as 2^14 kh + kl, each half exact
    // through the 2^23 magic number, one FMA rounding the sum
    const unsigned m = (unsigned)(k < 0 ? -k : k);
    const float fh = __uint_as_float(0x4B000000u | (m >> 14)) - 8388608.0f;
    const float fl = __uint_as_float(0x4B000000u | (m & 0x3fffu)) - 8388608.0f;
    const float lv = fmaf(fh, sc * 16384.0f, fl * sc);
    l = __uint_as_float(__float_as_uint(lv) ^ sgn ^ (k < 0 ? 0x80000000u : 0u));
  } else if ((ahi | lo) == 0u) {  // zero (the padding bands): no conversion instruction
    h = __uint_as_float(sgn);
    l = 0.0f;
  } else {
    h = __double2float_rn(x);
    l = 0.0f;
  }
}

__device__ __forceinline__ P2 from_doubles(double a, double b) {
  float ha, la, hb, lb;
  split(a, ha, la);
  split(b, hb, lb);
  return P2{pack(ha, hb), pack(la, lb)};
}

// h + l of a normalised pair as a double (truncated to 53 bits, below the
// pair's own rounding), built on the two 32-bit words of its bits.  Zero gives
// zero; Inf and NaN keep their class.
__device__ __forceinline__ double to_double(float h, float l) {
  const unsigned hb = __float_as_uint(h), lb = __float_as_uint(l);
  const unsigned ah = hb & 0x7fffffffu;
  const unsigned eh = ah >> 23;
  const unsigned sg = hb & 0x80000000u;
  if (eh == 0u) return __hiloint2double((int)sg, 0);  // zero (and subnormal hi, flushed)
  if (eh == 255u)                                       // Inf / NaN
    return __hiloint2double((int)(sg | 0x7ff00000u | ((ah & 0x7fffffu) ? 0x80000u : 0u)), 0);
  unsigned dhi = (ah >> 3) + (896u << 20), dlo = ah << 29;  // h as a double's bits
  const unsigned el = (lb >> 23) & 0xffu;
  const unsigned ml = el ? ((lb & 0x7fffffu) | 0x800000u) : 0u;
  const int sh = (int)el - (int)eh + 29;  // l in units of the double ulp of h: ml * 2^sh, sh <= 5
  unsigned k = sh >= 0 ? (ml << sh) : (ml >> min(-sh, 31));
  const bool opp = ((hb ^ lb) >> 31) != 0u;
  if (opp && (ah & 0x7fffffu) == 0u) k <<= 1;  // just below a power of two the double ulp halves
  if (opp) {  // subtract k with the borrow into the high word
    dhi -= dlo < k ? 1u : 0u;
    dlo -= k;
  } else {    // add k with the carry
    const unsigned s2 = dlo + k;
    dhi += s2 < dlo ? 1u : 0u;
    dlo = s2;
  }
  return __hiloint2double((int)(dhi | sg), (int)dlo);
}

__device__ __forceinline__ void to_doubles(const P2& p, double& a, double& b) {
  a = to_double(lo_of(p.h), lo_of(p.l));
  b = to_double(hi_of(p.h), hi_of(p.l));
}

// ------------------------------------------------------------------- memory
// 16 bytes h_b, h_b+1, l_b, l_b+1 from a 32-bit shared-memory address.
__device__ __forceinline__ P2 lds(unsigned sa) {
  P2 p;
  asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(p.h), "=l"(p.l) : "r"(sa));
  return p;
}
// two doubles from a 32-bit shared-memory address, as an ff pair
__device__ __forceinline__ P2 lds_doubles(unsigned sa) {
  double a, b;
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(a), "=d"(b) : "r"(sa));
  return from_doubles(a, b);
}
__device__ __forceinline__ P2 ldg(const void* p) {
  const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(p));
  return P2{v.x, v.y};
}
__device__ __forceinline__ void st_stream(void* p, const P2& v) {
  __stcs(reinterpret_cast<ulonglong2*>(p), make_ulonglong2(v.h, v.l));
}
__device__ __forceinline__ void st_stream_doubles(void* p, const P2& v) {
  double a, b;
  to_doubles(v, a, b);
  __stcs(reinterpret_cast<double2*>(p), make_double2(a, b));
}

}  // namespace ff
}  // namespace bte
