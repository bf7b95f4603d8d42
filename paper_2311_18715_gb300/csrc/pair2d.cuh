// A double-float pair (h, l) times 2^sc as an IEEE double, rounded to nearest (ties to even,
// pair_to_double; or to nearest with ties either way, pair_to_double_fast), with integer
// operations only.  On GB300 every conversion to double and every FP64
// operation runs at FP64 rate (~2 per clock per SM, measured), against ~100 per clock for
// FP32 and integer work, so an epilogue that writes one double per output builds the bits
// itself.  pair_to_double's result equals the correctly rounded value of h 2^sc + l 2^sc.
//
// Preconditions of pair_to_double (they hold for the normalized pairs the split epilogue
// forms): h is zero or
// a normal float, |l| <= ulp(h) / 2 (l = 0 when h = 0), and the result is a normal double
// (no overflow, no underflow).
#pragma once
#include <cstdint>
#include <cstring>

#ifndef __CUDACC__  // host compilers (the CPU test of this routine)
#define __host__
#define __device__
#endif

namespace odmd {

#if defined(__CUDA_ARCH__)
__device__ __forceinline__ uint32_t p2d_bits(float f) { return __float_as_uint(f); }
__device__ __forceinline__ double p2d_double(uint64_t b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ int p2d_clz64(uint64_t x) { return __clzll((long long)x); }
__device__ __forceinline__ uint64_t p2d_dbits(double d) { return (uint64_t)__double_as_longlong(d); }
__device__ __forceinline__ float p2d_float(uint32_t u) { return __uint_as_float(u); }
__device__ __forceinline__ int p2d_clz32(uint32_t x) { return __clz((int)x); }
#else
inline uint32_t p2d_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}
inline double p2d_double(uint64_t b) {
  double d;
  std::memcpy(&d, &b, 8);
  return d;
}
inline int p2d_clz64(uint64_t x) { return x ? __builtin_clzll(x) : 64; }
inline uint64_t p2d_dbits(double d) {
  uint64_t u;
  std::memcpy(&u, &d, 8);
  return u;
}
inline float p2d_float(uint32_t u) {
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
inline int p2d_clz32(uint32_t x) { return x ? __builtin_clz(x) : 32; }
#endif

__host__ __device__ inline double pair_to_double(float h, float l, int sc) {
  const uint32_t uh = p2d_bits(h);
  const uint32_t eh = (uh >> 23) & 0xFFu;
  if (eh == 0)  // h = 0 (then l = 0): the sum of two zeros is -0 only when both are -0
    return p2d_double((uint64_t)((uh >> 31) & (p2d_bits(l) >> 31)) << 63);
  const uint64_t sign = (uint64_t)(uh >> 31) << 63;
  // h = mh 2^(eh - 150); M = mh 2^39 carries the value in units of 2^(eh - 189)
  uint64_t M = (uint64_t)((uh & 0x7FFFFFu) | 0x800000u) << 39;
  bool sticky = false;
  const uint32_t ul = p2d_bits(l);
  const uint32_t el = (ul >> 23) & 0xFFu;
  if (el != 0) {
    const uint64_t ml = (uint64_t)((ul & 0x7FFFFFu) | 0x800000u);
    // l in the same units: ml 2^(el - eh + 39), with el <= eh - 24 so the shift is <= 15
    const int d = (int)el - (int)eh + 39;
    uint64_t add;
    if (d >= 0) {
      add = ml << d;
    } else if (d > -64) {
      add = ml >> (-d);
      sticky = (ml & ((1ull << (-d)) - 1)) != 0;
    } else {
      add = 0;
      sticky = true;
    }
    if ((ul >> 31) == (uh >> 31)) {
      M += add;
    } else {
      // subtracting a truncated magnitude: the dropped bits belong to the subtrahend, so the
      // exact value lies just below M - add; take one unit more off and keep a sticky bit
      M -= add + (sticky ? 1ull : 0ull);
    }
  }
  // normalize: leading bit to position 62 (|l| <= ulp(h)/2 moves it by at most one place)
  const int lead = 63 - p2d_clz64(M);
  int ex = (int)eh - 127;
  if (lead > 62) {
    sticky = sticky || (M & 1ull);
    M >>= 1;
    ex += 1;
  } else if (lead < 62) {
    M <<= (62 - lead);
    ex -= (62 - lead);
  }
  // keep 53 bits (62 .. 10), round to nearest even on bits 9 .. 0 and the sticky bit
  uint64_t mant = M >> 10;
  const uint64_t rem = M & 0x3FFull;
  if (rem > 0x200ull || (rem == 0x200ull && (sticky || (mant & 1ull)))) {
    mant += 1;
    if (mant >> 53) {
      mant >>= 1;
      ex += 1;
    }
  }
  const uint64_t biased = (uint64_t)(ex + 1023 + sc);
  return p2d_double(sign | (biased << 52) | (mant & ((1ull << 52) - 1)));
}

// The same double within half a unit in the last place (a tie may round either way), for
// a normalized pair: h is zero or normal, |l| <= ulp(h) / 2 with l zero or normal, and the
// result a normal double.  h 2^sc is written as a double's bits (its 24-bit significand
// shifted into the top of the 52-bit field), and l, rounded to a whole number of the
// double's units, is added to or taken from those bits as an integer.  Under |l| <= ulp(h)/2
// the addition never carries out of the significand; a subtraction borrows from the
// exponent only when h is a power of two, and the unit is then the half-size unit of the
// binade below, so l is rounded to that finer unit.  About a third of the operations of
// pair_to_double.
__host__ __device__ inline double pair_to_double_fast(float h, float l, int sc) {
  const uint32_t uh = p2d_bits(h), ul = p2d_bits(l);
  const uint32_t eh = (uh >> 23) & 0xFFu;
  if (eh == 0) return p2d_double((uint64_t)((uh >> 31) & (ul >> 31)) << 63);
  const uint32_t el = (ul >> 23) & 0xFFu;
  const bool opp = ((uh ^ ul) >> 31) != 0u;
  // l = ml 2^(el - 150) in units 2^(eh - 179) of the double's last place (2^(eh - 180) below
  // a power of two)
  const int sh = (int)el - (int)eh + 29 + ((opp && (uh & 0x7FFFFFu) == 0u) ? 1 : 0);
  const uint32_t ml = (ul & 0x7FFFFFu) | 0x800000u;
  uint32_t delta = 0;  // at most 2^29: |l| <= 2^28 units
  if (el != 0) {
    if (sh >= 0)
      delta = ml << sh;
    else if (sh > -32)
      delta = (ml + (1u << (-sh - 1))) >> (-sh);
  }
  const uint64_t bits = ((uint64_t)(uh >> 31) << 63) | ((uint64_t)(uint32_t)((int)eh + 896 + sc) << 52) |
                        ((uint64_t)(uh & 0x7FFFFFu) << 29);
  return p2d_double(opp ? bits - delta : bits + delta);
}

// The other direction: a double x as the pair h = RN(x), l = RN(x - h) (round to nearest
// even, both as floats), which is exactly what two conversions and a subtraction give, built
// from x's bits with integer operations: the 53-bit significand is rounded to 24 bits for h,
// and the signed remainder (at most 29 bits) is rounded to 24 for l.  When x, h or l falls
// outside the normal float range (zero, subnormal, overflow, a non-finite x), the result
// comes from the conversions instead (`false` is returned for the caller's slow path on the
// device; the host version converts itself).
__host__ __device__ inline bool double_to_pair_fast(double x, float& h, float& l) {
  const uint64_t b = p2d_dbits(x);
  const uint32_t sign = (uint32_t)(b >> 63);
  const int E = (int)((b >> 52) & 0x7FFu);
  int ef = E - 1023 + 127;  // the float exponent field of x's binade
  if (ef < 1 || ef > 254) return false;
  const uint64_t m = (b & ((1ull << 52) - 1)) | (1ull << 52);
  uint32_t q = (uint32_t)(m >> 29);
  const uint32_t rem = (uint32_t)(m & ((1u << 29) - 1));
  const bool up = rem > (1u << 28) || (rem == (1u << 28) && (q & 1u));
  q += up ? 1u : 0u;
  if (q == (1u << 24)) {  // rounded up to the next binade
    q = 1u << 23;
    ++ef;
    if (ef > 254) return false;
  }
  h = p2d_float((sign << 31) | ((uint32_t)ef << 23) | (q & 0x7FFFFFu));
  // x - h = r 2^(E - 1075), |r| <= 2^28 (negative when h was rounded up in magnitude)
  const int32_t r = (int32_t)rem - (up ? (int32_t)(1u << 29) : 0);
  if (r == 0) {
    l = 0.f;
    return true;
  }
  uint32_t a = (uint32_t)(r < 0 ? -r : r);
  int lead = 31 - p2d_clz32(a);  // 0 .. 28
  uint32_t mant;
  if (lead <= 23) {
    mant = a << (23 - lead);
  } else {
    const int sh = lead - 23;
    mant = a >> sh;
    const uint32_t rest = a & ((1u << sh) - 1u), half = 1u << (sh - 1);
    if (rest > half || (rest == half && (mant & 1u))) ++mant;
    if (mant == (1u << 24)) {
      mant = 1u << 23;
      ++lead;
    }
  }
  const int el = lead + E - 948;  // biased exponent of l: a 2^(E - 1075) = 1.f 2^(lead + E - 1075)
  if (el < 1) return false;
  l = p2d_float(((sign ^ (r < 0 ? 1u : 0u)) << 31) | ((uint32_t)el << 23) | (mant & 0x7FFFFFu));
  return true;
}

}  // namespace odmd
