// Summation of doubles in a 192-bit (and, below, a 128-bit) two's-complement
// fixed-point accumulator whose grid is anchored to the run's largest
// exponent.
//
// For a run whose largest value has biased exponent emax, values are held as
// multiples of 2^-frac with frac = fx_frac_for(emax): the largest value's
// leading bit sits at bit 166, which leaves 24 bits of headroom (up to 2^24
// values sum without overflow).  Every value within 2^-113 of the largest is
// converted exactly; smaller ones round to the grid (ties to even), an error
// of at most 2^-167 relative to the largest value.  Integer addition is exact
// and associative, and emax does not depend on the order, so the sum of a run
// is independent of the order of its values; fx_to_double rounds it once, to
// nearest even.  This is the numerator accumulator of the score
// (sum_j H_ij c_j): deterministic under any tiling or scheduling, and free of
// FP64 instructions, which are scarce on this GPU.
//
// Host and device compilable (no CUDA intrinsics outside __CUDA_ARCH__).
#pragma once

#include <stdint.h>
#include <string.h>

#ifndef __CUDACC__
#ifndef __host__
#define __host__
#endif
#ifndef __device__
#define __device__
#endif
#ifndef __forceinline__
#define __forceinline__ inline
#endif
#endif

namespace asci {

constexpr int kFxLead = 166;  // bit of the largest value's leading one

// Biased exponent of x (subnormals and zero count as 1).
__host__ __device__ __forceinline__ int fx_exponent(double x);

// Fractional bits of the grid for a run whose largest biased exponent is emax.
__host__ __device__ __forceinline__ int fx_frac_for(int emax) { return kFxLead - 52 + 1075 - emax; }

struct Fx192 {
  uint64_t w0, w1, w2;  // little-endian limbs, two's complement
};

__host__ __device__ __forceinline__ int fx_clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

__host__ __device__ __forceinline__ uint64_t fx_dbits(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  memcpy(&b, &x, 8);
  return b;
#endif
}

__host__ __device__ __forceinline__ double fx_bits2d(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  memcpy(&x, &b, 8);
  return x;
#endif
}

__host__ __device__ __forceinline__ void fx_add(Fx192 &a, const Fx192 &b) {
#ifdef __CUDA_ARCH__
  asm("add.cc.u64 %0, %0, %3;\n\t"
      "addc.cc.u64 %1, %1, %4;\n\t"
      "addc.u64 %2, %2, %5;"
      : "+l"(a.w0), "+l"(a.w1), "+l"(a.w2)
      : "l"(b.w0), "l"(b.w1), "l"(b.w2));
#else
  uint64_t s0 = a.w0 + b.w0;
  uint64_t c0 = s0 < a.w0;
  uint64_t s1 = a.w1 + b.w1;
  uint64_t c1 = s1 < a.w1;
  uint64_t s1c = s1 + c0;
  c1 |= s1c < s1;
  a.w0 = s0;
  a.w1 = s1c;
  a.w2 = a.w2 + b.w2 + c1;
#endif
}

__host__ __device__ __forceinline__ void fx_neg(Fx192 &a) {
  a.w0 = ~a.w0;
  a.w1 = ~a.w1;
  a.w2 = ~a.w2;
  Fx192 one = {1, 0, 0};
  fx_add(a, one);
}

__host__ __device__ __forceinline__ int fx_exponent(double x) {
  const int eb = (int)((fx_dbits(x) >> 52) & 0x7ff);
  return eb ? eb : 1;
}

// x -> multiple of 2^-frac (round to nearest even); *ovf set when x is not
// finite or does not fit below bit 190.
__host__ __device__ __forceinline__ Fx192 fx_from_double(double x, int frac, unsigned *ovf) {
  Fx192 r = {0, 0, 0};
  const uint64_t b = fx_dbits(x);
  int eb = (int)((b >> 52) & 0x7ff);
  uint64_t m = b & ((1ull << 52) - 1);
  if (eb == 0x7ff) {  // inf or nan
    *ovf = 1;
    return r;
  }
  if (eb) m |= (1ull << 52); else eb = 1;
  if (m == 0) return r;
  // value = m * 2^(eb - 1075); fixed = m * 2^(eb - 1075 + frac)
  const int k = eb - 1075 + frac;
  if (k >= 0) {
    if (k >= 191 - 52) {
      *ovf = 1;
      return r;
    }
    if (k < 64) {
      r.w0 = m << k;
      r.w1 = k ? (m >> (64 - k)) : 0;
    } else if (k < 128) {
      const int k2 = k - 64;
      r.w1 = m << k2;
      r.w2 = k2 ? (m >> (64 - k2)) : 0;
    } else {
      r.w2 = m << (k - 128);
    }
  } else {
    const int s = -k;  // right shift with round to nearest even
    if (s > 54) return r;
    const uint64_t q = m >> s;
    const uint64_t rem = m & ((1ull << s) - 1);
    const uint64_t half = 1ull << (s - 1);
    r.w0 = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
  }
  if (b >> 63) fx_neg(r);
  return r;
}

// Round a * 2^-frac to the nearest double (ties to even).
__host__ __device__ __forceinline__ double fx_to_double(Fx192 a, int frac) {
  const bool neg = (a.w2 >> 63) != 0;
  if (neg) fx_neg(a);
  if (!(a.w0 | a.w1 | a.w2)) return 0.0;
  int P;  // index of the highest set bit
  if (a.w2) P = 128 + 63 - fx_clz64(a.w2);
  else if (a.w1) P = 64 + 63 - fx_clz64(a.w1);
  else P = 63 - fx_clz64(a.w0);
  uint64_t mant;
  if (P <= 52) {
    mant = a.w0 << (52 - P);  // exact
  } else {
    // mant = bits [P-52, P]; round bit P-53; sticky = bits below (limbs are
    // selected with conditionals so that nothing is indexed dynamically)
    const int sh = P - 52;
    const int limb = sh >> 6, bit = sh & 63;
    const uint64_t cur = limb == 0 ? a.w0 : (limb == 1 ? a.w1 : a.w2);
    const uint64_t nxt = limb == 0 ? a.w1 : (limb == 1 ? a.w2 : 0);
    const uint64_t win = bit ? ((cur >> bit) | (nxt << (64 - bit))) : cur;
    mant = win & ((1ull << 53) - 1);
    const int rb = sh - 1;
    const int rl = rb >> 6, rbb = rb & 63;
    const uint64_t rw = rl == 0 ? a.w0 : (rl == 1 ? a.w1 : a.w2);
    const uint64_t rbit = (rw >> rbb) & 1;
    bool sticky = (rbb ? (rw & ((1ull << rbb) - 1)) : 0) != 0;
    if (rl >= 1) sticky |= a.w0 != 0;
    if (rl >= 2) sticky |= a.w1 != 0;
    if (rbit && (sticky || (mant & 1))) {
      mant += 1;
      if (mant == (1ull << 53)) {
        mant >>= 1;
        P += 1;
      }
    }
  }
  // value = mant * 2^(P - 52 - frac), mant in [2^52, 2^53)
  const int e = P - frac;  // unbiased exponent of the result
  double v;
  if (e + 1023 >= 1 && e + 1023 <= 2046) {
    v = fx_bits2d(((uint64_t)(e + 1023) << 52) | (mant & ((1ull << 52) - 1)));
  } else {
    // outside the normal range (a run cancelling far below 1e-300): scale in steps
    v = (double)mant;
    int sh = e - 52;
    while (sh > 0) { const int t = sh > 1000 ? 1000 : sh; v *= fx_bits2d((uint64_t)(t + 1023) << 52); sh -= t; }
    while (sh < 0) { const int t = sh < -1000 ? -1000 : sh; v *= fx_bits2d((uint64_t)(t + 1023) << 52); sh -= t; }
  }
  return neg ? -v : v;
}

// ---- 128-bit variant ------------------------------------------------------
// The same construction on two limbs, with the largest value's leading one at
// bit 100 (27 bits of headroom: up to 2^26 values).  Values within 2^-48 of the
// largest convert exactly; smaller ones round to the grid, an error of at most
// 2^-101 relative to the largest value.  Cheaper per value than the 192-bit
// form; the sum is again a function of the multiset of values only.

constexpr int kFx128Lead = 100;

__host__ __device__ __forceinline__ int fx128_frac_for(int emax) {
  return kFx128Lead - 52 + 1075 - emax;
}

struct Fx128 {
  uint64_t lo, hi;  // two's complement
};

__host__ __device__ __forceinline__ void fx128_add(Fx128 &a, const Fx128 &b) {
#ifdef __CUDA_ARCH__
  asm("add.cc.u64 %0, %0, %2;\n\t"
      "addc.u64 %1, %1, %3;"
      : "+l"(a.lo), "+l"(a.hi)
      : "l"(b.lo), "l"(b.hi));
#else
  const uint64_t s0 = a.lo + b.lo;
  a.hi = a.hi + b.hi + (s0 < a.lo ? 1u : 0u);
  a.lo = s0;
#endif
}

__host__ __device__ __forceinline__ void fx128_neg(Fx128 &a) {
  a.lo = ~a.lo;
  a.hi = ~a.hi;
  const Fx128 one = {1, 0};
  fx128_add(a, one);
}

// x -> multiple of 2^-frac (round to nearest even); *ovf set when x is not
// finite or does not fit below bit 126.
__host__ __device__ __forceinline__ Fx128 fx128_from_double(double x, int frac, unsigned *ovf) {
  Fx128 r = {0, 0};
  const uint64_t b = fx_dbits(x);
  int eb = (int)((b >> 52) & 0x7ff);
  uint64_t m = b & ((1ull << 52) - 1);
  if (eb == 0x7ff) {  // inf or nan
    *ovf = 1;
    return r;
  }
  if (eb) m |= (1ull << 52); else eb = 1;
  if (m == 0) return r;
  const int k = eb - 1075 + frac;  // value = m * 2^(k - frac)
  if (k >= 0) {
    if (k >= 127 - 52) {
      *ovf = 1;
      return r;
    }
    if (k < 64) {
      r.lo = m << k;
      r.hi = k ? (m >> (64 - k)) : 0;
    } else {
      r.hi = m << (k - 64);
    }
  } else {
    const int s = -k;  // right shift with round to nearest even
    if (s > 54) return r;
    const uint64_t q = m >> s;
    const uint64_t rem = m & ((1ull << s) - 1);
    const uint64_t half = 1ull << (s - 1);
    r.lo = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
  }
  if (b >> 63) fx128_neg(r);
  return r;
}

// Round a * 2^-frac to the nearest double (ties to even).
__host__ __device__ __forceinline__ double fx128_to_double(Fx128 a, int frac) {
  const bool neg = (a.hi >> 63) != 0;
  if (neg) fx128_neg(a);
  if (!(a.lo | a.hi)) return 0.0;
  int P = a.hi ? 64 + 63 - fx_clz64(a.hi) : 63 - fx_clz64(a.lo);  // highest set bit
  uint64_t mant;
  if (P <= 52) {
    mant = a.lo << (52 - P);  // exact
  } else {
    // mant = bits [P-52, P]; round bit P-53; sticky = bits below
    const int sh = P - 52;
    const uint64_t win =
        sh < 64 ? ((a.lo >> sh) | (sh ? (a.hi << (64 - sh)) : 0)) : (a.hi >> (sh - 64));
    mant = win & ((1ull << 53) - 1);
    const int rb = sh - 1;
    const uint64_t rbit = rb < 64 ? ((a.lo >> rb) & 1) : ((a.hi >> (rb - 64)) & 1);
    bool sticky;
    if (rb < 64) sticky = (rb ? (a.lo & ((1ull << rb) - 1)) : 0) != 0;
    else sticky = a.lo != 0 || ((rb - 64) ? (a.hi & ((1ull << (rb - 64)) - 1)) : 0) != 0;
    if (rbit && (sticky || (mant & 1))) {
      mant += 1;
      if (mant == (1ull << 53)) {
        mant >>= 1;
        P += 1;
      }
    }
  }
  const int e = P - frac;  // unbiased exponent of the result
  double v;
  if (e + 1023 >= 1 && e + 1023 <= 2046) {
    v = fx_bits2d(((uint64_t)(e + 1023) << 52) | (mant & ((1ull << 52) - 1)));
  } else {
    v = (double)mant;
    int sh = e - 52;
    while (sh > 0) { const int t = sh > 1000 ? 1000 : sh; v *= fx_bits2d((uint64_t)(t + 1023) << 52); sh -= t; }
    while (sh < 0) { const int t = sh < -1000 ? -1000 : sh; v *= fx_bits2d((uint64_t)(t + 1023) << 52); sh -= t; }
  }
  return neg ? -v : v;
}

}  // namespace asci
