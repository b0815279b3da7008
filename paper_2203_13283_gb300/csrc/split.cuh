// Split of an FP64 value into bf16 planes for the tensor-core contraction:
// x = p0 + p1 (+ p2), p0 = bf16(x), p1 = bf16(x - p0), p2 = bf16(x - p0 - p1),
// each rounded to nearest (ties to even) from the exact remainder, so every
// plane adds about 8 bits.
//
// split3 forms the remainders with FP64 subtractions and conversions.  On
// GB300 those run on the FP64 pipe (about 2 operations per clock per SM), so
// a staging kernel spending ~7 of them per value is FP64-bound, several times
// below the HBM bound.  split3_bits forms the same planes with integer
// operations on the double's bits: the remainders are exact integers in units
// of the last place of x, each plane is the remainder rounded to 8
// significant bits, and its bf16 encoding is assembled from sign, exponent
// and the 7 bits below the leading one.  Inside the window where every plane
// of a nonzero x is a normal bf16 (2^-74 <= |x| < 2^100) the two agree bit
// for bit; outside it (zero, tiny, huge, not finite) split3_bits calls
// split3.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

namespace wcs {

__host__ __device__ __forceinline__ void split3(double x, int planes, uint16_t* o0, uint16_t* o1, uint16_t* o2) {
  __nv_bfloat16 h0 = __double2bfloat16(x);
  double r = x - (double)__bfloat162float(h0);
  *o0 = __bfloat16_as_ushort(h0);
  if (planes > 1) {
    __nv_bfloat16 h1 = __double2bfloat16(r);
    r -= (double)__bfloat162float(h1);
    *o1 = __bfloat16_as_ushort(h1);
    if (planes > 2) *o2 = __bfloat16_as_ushort(__double2bfloat16(r));
  }
}

__host__ __device__ __forceinline__ int split_clz64(uint64_t a) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)a);
#else
  return __builtin_clzll(a);
#endif
}

// a > 0 rounded to 8 significant bits, ties to even: q << sh, q <= 256
// (256 only as the carry of a round-up)
__host__ __device__ __forceinline__ void split_round8(uint64_t a, uint32_t& q, int& sh) {
  const int L = 63 - split_clz64(a);
  if (L <= 7) {
    q = (uint32_t)a;
    sh = 0;
    return;
  }
  sh = L - 7;
  const uint64_t t = a >> sh, rem = a & ((1ull << sh) - 1), half = 1ull << (sh - 1);
  q = (uint32_t)t + ((rem > half || (rem == half && (t & 1))) ? 1u : 0u);
}

// bf16 encoding of (-1)^neg q 2^p for 1 <= q <= 256 inside bf16's normal range
__host__ __device__ __forceinline__ uint16_t split_bf16_bits(uint32_t neg, uint32_t q, int p) {
  const int L = 63 - split_clz64((uint64_t)q);
  const uint32_t mant = (L <= 7) ? ((q << (7 - L)) & 0x7Fu) : ((q >> (L - 7)) & 0x7Fu);
  return (uint16_t)((neg << 15) | ((uint32_t)(p + L + 127) << 7) | mant);
}

// one plane of the signed remainder v (units 2^e, x's sign neg): its bf16
// bits; v becomes the next remainder
__host__ __device__ __forceinline__ uint16_t split_plane(int64_t& v, uint32_t neg, int e) {
  if (v == 0) return 0;   // an exact zero remainder is +0, as x - p in FP64
  const bool minus = v < 0;
  uint32_t q;
  int sh;
  split_round8((uint64_t)(minus ? -v : v), q, sh);
  const int64_t p = (int64_t)q << sh;
  v = minus ? v + p : v - p;
  return split_bf16_bits(neg ^ (minus ? 1u : 0u), q, e + sh);
}

__host__ __device__ __forceinline__ void split3_bits(double x, int planes, uint16_t* o0, uint16_t* o1,
                                                     uint16_t* o2) {
  uint64_t u;
#ifdef __CUDA_ARCH__
  u = (uint64_t)__double_as_longlong(x);
#else
  memcpy(&u, &x, sizeof(u));
#endif
  const int be = (int)((u >> 52) & 0x7FF);
  if (be < 1023 - 74 || be >= 1023 + 100) {
    split3(x, planes, o0, o1, o2);
    return;
  }
  const uint32_t neg = (uint32_t)(u >> 63);
  const int e = be - 1075;                                   // |x| = M 2^e
  int64_t v = (int64_t)((u & 0xFFFFFFFFFFFFFull) | (1ull << 52));
  *o0 = split_plane(v, neg, e);
  if (planes > 1) {
    *o1 = split_plane(v, neg, e);
    if (planes > 2) *o2 = split_plane(v, neg, e);
  }
}

}  // namespace wcs
