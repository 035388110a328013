// fpint.h -- IEEE 754 binary32/binary64 operations in integer arithmetic:
// conversions between the two formats and the product of a binary64 by a
// binary64 constant.  GB300's FP64 pipe (which also executes F2F conversions)
// runs at ~1/70 of the FP32 rate (measured: ~505 G FP64 FMA/s against ~36 T
// FP32 FMA/s), and the FP64 epilogues of Eq. 1 are bound by it; moving these
// operations to the integer units leaves the FP64 pipe the fused
// multiply-adds alone.  Host and device: the host build is what the CPU tests
// check against the host's IEEE arithmetic.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define TTC_HD __host__ __device__ __forceinline__
#else
#define TTC_HD inline
#endif

namespace ttc {

TTC_HD uint32_t fp_bits(float f) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(f);
#else
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
#endif
}

TTC_HD uint64_t fp_bits(double d) {
#if defined(__CUDA_ARCH__)
  return uint64_t(__double_as_longlong(d));
#else
  uint64_t u;
  std::memcpy(&u, &d, 8);
  return u;
#endif
}

TTC_HD float fp_float(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, 4);
  return f;
#endif
}

TTC_HD double fp_double(uint32_t hi, uint32_t lo) {
#if defined(__CUDA_ARCH__)
  return __hiloint2double(int(hi), int(lo));
#else
  const uint64_t u = (uint64_t(hi) << 32) | lo;
  double d;
  std::memcpy(&d, &u, 8);
  return d;
#endif
}

// leading zeros of a nonzero 32-bit word
TTC_HD int fp_clz(uint32_t x) {
#if defined(__CUDA_ARCH__)
  return __clz(x);
#else
  int n = 0;
  while (!(x & 0x80000000u)) {
    x <<= 1;
    ++n;
  }
  return n;
#endif
}

// binary32 -> binary64 (exact).  A normal number keeps its sign, re-biases
// its exponent by 1023 - 127 = 896 and moves its 23 fraction bits to the top
// of the 52.  A subnormal m * 2^-149 becomes normal: its leading one (bit q)
// turns into the implicit bit, exponent q - 149.  Infinities keep an all-ones
// exponent; NaN keeps its payload with the quiet bit set.
TTC_HD double widen_f32(float f) {
  const uint32_t u = fp_bits(f);
  const uint32_t sign = u & 0x80000000u, ex = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  uint32_t hi = sign | (((u & 0x7fffffffu) >> 3) + (896u << 20)), lo = u << 29;
  if (ex == 0xffu) hi = sign | 0x7ff00000u | (m >> 3) | (m ? 0x00080000u : 0u);
  if (ex == 0u) {
    const int q = 31 - fp_clz(m | 1u);
    const uint64_t frac = (uint64_t(m) << (52 - q)) & 0xfffffffffffffull;
    hi = m ? sign | (uint32_t(q + 874) << 20) | uint32_t(frac >> 32) : sign;
    lo = m ? uint32_t(frac) : 0u;
  }
  return fp_double(hi, lo);
}

// binary64 -> binary32, round to nearest, ties to even.  In the normal
// binary32 range (biased binary64 exponent 897..1150) the top 23 of the 52
// fraction bits are kept and the 29 dropped bits decide (above half: up;
// exactly half: up if the kept part is odd); a carry out of the fraction
// correctly raises the exponent, up to infinity.  Smaller results are the
// significand shifted to the 2^-149 quantum and rounded the same way (zero
// below half of it); exponents above the range give infinity; NaN stays NaN
// (quiet, payload truncated).
TTC_HD float narrow_f64_rn(double d) {
  const uint64_t b = fp_bits(d);
  const uint32_t hi = uint32_t(b >> 32), lo = uint32_t(b);
  const uint32_t sign = hi & 0x80000000u, e = (hi >> 20) & 0x7ffu;
  // exponent field e - 896 and the kept fraction bits, modulo 2^32
  const uint32_t field = ((hi << 3) | (lo >> 29)) - (896u << 23);
  const uint32_t rem = lo & 0x1fffffffu;
  const uint32_t up = uint32_t(rem > 0x10000000u) | (uint32_t(rem == 0x10000000u) & field);
  uint32_t r = sign | (field + (up & 1u));
  if (e - 897u > 253u) {
    const uint32_t fh = hi & 0xfffffu;
    if (e == 0x7ffu) {
      r = sign | ((fh | lo) ? 0x7fc00000u | (fh << 3) | (lo >> 29) : 0x7f800000u);
    } else if (e >= 1151u) {
      r = sign | 0x7f800000u;
    } else if (e < 872u) {
      r = sign;                         // below half of the smallest subnormal
    } else {
      const uint64_t m = (uint64_t(fh | 0x100000u) << 32) | lo;
      const uint32_t sh = 926u - e;     // 30..54
      const uint64_t kept = m >> sh, rest = m & ((uint64_t(1) << sh) - 1), half = uint64_t(1) << (sh - 1);
      r = sign | uint32_t(kept + ((rest > half) | ((rest == half) & (kept & 1))));
    }
  }
  return fp_float(r);
}

// A binary64 constant c prepared for dmul_normal: its significand with the
// implicit one as 21 + 32 bits, its biased exponent and its sign.  ok = 0
// when c is zero, subnormal, infinite or NaN (then only the hardware
// multiply is used).
struct DMulConst {
  uint32_t c1, c0;
  int32_t ec;
  uint32_t sign;
  int32_t ok;
};

inline DMulConst make_dmul_const(double c) {
  DMulConst k;
  const uint64_t b = fp_bits(c);
  k.c1 = uint32_t((b >> 32) & 0xfffffu) | 0x100000u;
  k.c0 = uint32_t(b);
  k.ec = int32_t((b >> 52) & 0x7ffu);
  k.sign = uint32_t(b >> 32) & 0x80000000u;
  k.ok = k.ec >= 1 && k.ec <= 2046;
  return k;
}

// fl64(c * a), round to nearest, ties to even, by the schoolbook product of
// the two 53-bit significands (four 32 x 32 -> 64-bit partial products into
// a 106-bit result), normalised to 53 bits with the dropped bits deciding the
// rounding as above; a carry out of the significand raises the exponent.
// Returns false when `a` is not a normal number or the product's exponent
// leaves the normal range; *r is then unspecified and the caller multiplies
// in hardware.  c must be normal (k.ok).
TTC_HD bool dmul_normal(const DMulConst& k, double a, double* r) {
  const uint64_t b = fp_bits(a);
  const uint32_t hi = uint32_t(b >> 32), lo = uint32_t(b);
  const int ea = int((hi >> 20) & 0x7ffu);
  const uint32_t a1 = (hi & 0xfffffu) | 0x100000u;
  const uint64_t p00 = uint64_t(lo) * k.c0, p01 = uint64_t(lo) * k.c1;
  const uint64_t p10 = uint64_t(a1) * k.c0, p11 = uint64_t(a1) * k.c1;
  const uint64_t mid = p01 + p10;                      // < 2^54
  const uint64_t plo = p00 + (mid << 32);
  const uint64_t phi = p11 + (mid >> 32) + (plo < p00 ? 1u : 0u);   // product = phi * 2^64 + plo < 2^106
  const int norm = int(phi >> 41);                     // product in [2^105, 2^106)
  const int sh = 52 + norm;
  const uint64_t m = (phi << (64 - sh)) | (plo >> sh); // 53-bit significand, implicit bit at 52
  const uint64_t rest = plo & ((uint64_t(1) << sh) - 1), half = uint64_t(1) << (sh - 1);
  const uint64_t mr = m + ((rest > half) | ((rest == half) & (m & 1u)));
  const int e = ea + k.ec - 1023 + norm;               // biased exponent before a rounding carry
  // (e - 1) << 52 plus the significand: its implicit bit (or a carry to 2^53)
  // completes the exponent field
  const uint64_t bits = (uint64_t((hi ^ k.sign) & 0x80000000u) << 32) + (uint64_t(uint32_t(e - 1)) << 52) + mr;
  *r = fp_double(uint32_t(bits >> 32), uint32_t(bits));
  return ea >= 1 && ea <= 2046 && e >= 1 && e + int(mr >> 53) <= 2046;
}

}  // namespace ttc
