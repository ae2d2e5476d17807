// Exact, order-independent summation of float64 values for the add mode.
//
// The writes to one element are accumulated as integers.  Every finite value
// v = mant * 2^(e - 1075) (float32 values are first widened exactly) is
// truncated toward zero to a multiple of 2^(E - 1075 - kAlignBits), where E is
// the largest exponent among the writes of that element, and added into a
// signed 128-bit accumulator; the integer sum is rounded once to the output
// type (round-to-nearest-even).  Integer addition is associative, so the
// result depends only on the element's values, not on their order or on how
// the work is split.  A value loses bits only when it lies more than
// kAlignBits binades below the element's largest value, and then less than
// 2^-(kAlignBits + 52) of that value; when every write of the element lies
// within kAlignBits binades of the largest, the result is the correctly
// rounded exact sum.  Aligned values are below 2^(53 + kAlignBits) = 2^95, so
// 2^32 of them cannot overflow the accumulator.  NaN and infinities are
// carried as flags with IEEE semantics (NaN if any NaN or both infinities).
//
// GB300's float64 pipe is a small fraction of its integer pipes, so this is
// also much faster than a chain of float64 additions.
#pragma once

#include <cstdint>

#ifdef __CUDACC__
#define SPM_HD __host__ __device__ __forceinline__
#else
#define SPM_HD inline
#endif

namespace spm {

constexpr int kAlignBits = 42;  // binary point: 42 bits below the last mantissa bit of the largest value

struct Acc {
  uint64_t lo;
  int64_t hi;
  uint32_t flags;  // 1 NaN, 2 +Inf, 4 -Inf
};

SPM_HD Acc acc_zero() { return Acc{0ull, 0ll, 0u}; }

SPM_HD int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

// Biased exponent used for alignment (subnormals count as 1; 0 for zero,
// -1 for NaN/Inf).
SPM_HD int f64_align_exponent(uint64_t bits) {
  const int e = (int)((bits >> 52) & 0x7ff);
  const uint64_t mant = bits & 0xFFFFFFFFFFFFFull;
  if (e == 0x7ff) return -1;
  if (e == 0) return mant ? 1 : 0;
  return e;
}

SPM_HD void acc_add_bits(Acc& a, uint64_t bits, int emax) {
  int e = (int)((bits >> 52) & 0x7ff);
  uint64_t mant = bits & 0xFFFFFFFFFFFFFull;
  const bool neg = (bits >> 63) != 0;
  if (e == 0x7ff) {
    a.flags |= mant ? 1u : (neg ? 4u : 2u);
    return;
  }
  if (e == 0) {
    if (!mant) return;
    e = 1;
  } else {
    mant |= 1ull << 52;
  }
  const int sh = e - (emax - kAlignBits);  // <= kAlignBits
  uint64_t tlo, thi;
  if (sh >= 0) {
    tlo = mant << sh;
    thi = sh ? (mant >> (64 - sh)) : 0ull;
  } else {
    if (sh <= -64) return;
    tlo = mant >> (-sh);
    thi = 0ull;
  }
  if (neg) {
    const uint64_t lo = a.lo - tlo;
    const uint64_t borrow = a.lo < tlo ? 1ull : 0ull;
    a.hi = (int64_t)((uint64_t)a.hi - thi - borrow);
    a.lo = lo;
  } else {
    const uint64_t lo = a.lo + tlo;
    const uint64_t carry = lo < tlo ? 1ull : 0ull;
    a.hi = (int64_t)((uint64_t)a.hi + thi + carry);
    a.lo = lo;
  }
}

SPM_HD void acc_merge(Acc& a, const Acc& b) {
  const uint64_t lo = a.lo + b.lo;
  const uint64_t carry = lo < b.lo ? 1ull : 0ull;
  a.hi = (int64_t)((uint64_t)a.hi + (uint64_t)b.hi + carry);
  a.lo = lo;
  a.flags |= b.flags;
}

// Round the accumulated value to float64 (f32 = false) or float32 (f32 =
// true), round-to-nearest-even; returns the raw bits and whether the result
// compares unequal to zero.
SPM_HD uint64_t acc_round(const Acc& a, int emax, bool f32, bool* nonzero) {
  if ((a.flags & 1u) || (a.flags & 6u) == 6u) {
    *nonzero = true;
    return f32 ? 0x7FC00000ull : 0x7FF8000000000000ull;
  }
  if (a.flags & 2u) {
    *nonzero = true;
    return f32 ? 0x7F800000ull : 0x7FF0000000000000ull;
  }
  if (a.flags & 4u) {
    *nonzero = true;
    return f32 ? 0xFF800000ull : 0xFFF0000000000000ull;
  }
  uint64_t lo = a.lo, hi = (uint64_t)a.hi;
  const bool neg = a.hi < 0;
  if (neg) {  // two's complement negate
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1ull : 0ull);
  }
  if (lo == 0ull && hi == 0ull) {
    *nonzero = false;
    return 0ull;
  }
  *nonzero = true;
  const int msb = hi ? 127 - clz64(hi) : 63 - clz64(lo);
  const int prec = f32 ? 24 : 53;
  const int qmin = f32 ? -149 : -1074;
  const int u = (emax - kAlignBits) - 1075;  // value = mag * 2^u
  int s = msb - (prec - 1);
  if (s < qmin - u) s = qmin - u;
  uint64_t m;
  int q;
  if (s <= 0) {
    m = lo << (-s);  // exact: msb - s <= prec - 1 < 64 and hi == 0 here
    q = u + s;
  } else {
    // m = mag >> s, then round half to even on the dropped s bits
    if (s >= 128) {
      m = 0ull;
    } else if (s >= 64) {
      m = hi >> (s - 64);
    } else {
      m = (lo >> s) | (hi << (64 - s));
    }
    const int g = s - 1;  // guard bit position
    const uint64_t guard = g >= 64 ? ((g - 64) < 64 ? (hi >> (g - 64)) & 1ull : 0ull) : (lo >> g) & 1ull;
    bool sticky;
    if (g == 0) {
      sticky = false;
    } else if (g >= 64) {
      const int hb = g - 64;
      sticky = lo != 0ull || (hb > 0 && (hi & ((hb >= 64 ? ~0ull : ((1ull << hb) - 1ull)))) != 0ull);
    } else {
      sticky = (lo & ((1ull << g) - 1ull)) != 0ull;
    }
    if (guard && (sticky || (m & 1ull))) ++m;
    q = u + s;
    if (m == (1ull << prec)) {
      m >>= 1;
      ++q;
    }
  }
  const uint64_t sign = neg ? (f32 ? 0x80000000ull : 0x8000000000000000ull) : 0ull;
  if (m >= (1ull << (prec - 1))) {
    const int biased = q + (prec - 1) + (f32 ? 127 : 1023);
    const int maxe = f32 ? 255 : 2047;
    if (biased >= maxe) return sign | (f32 ? 0x7F800000ull : 0x7FF0000000000000ull);
    const uint64_t frac = m & ((1ull << (prec - 1)) - 1ull);
    return sign | ((uint64_t)biased << (prec - 1)) | frac;
  }
  return sign | m;  // subnormal (q == qmin)
}

}  // namespace spm
