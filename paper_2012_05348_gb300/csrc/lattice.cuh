// Exact lattice arithmetic shared by the device refit and the device build: the slab
// directions and floor / ceil of d_j . v / 2^e for FP32 vertices, decided exactly in FP64.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace {

__constant__ int c_rdir[13][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},  {1, 1, 0}, {1, -1, 0},
                                  {1, 0, 1},  {1, 0, -1}, {0, 1, 1},  {0, 1, -1}, {1, 1, 1},
                                  {1, 1, -1}, {1, -1, 1}, {-1, 1, 1}};

constexpr int64_t kLatLimit = int64_t(1) << 30;

// ---------------------------------------------------------------- exact lattice values
// a + b exactly as s + err (Knuth's TwoSum; FP64, round to nearest, no contraction).
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &err) {
  s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  err = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

// floor of the non-overlapping expansion q2 + q1 + q0 (decreasing magnitudes): when q2 has a
// fractional part the smaller components cannot move the sum across an integer, so the
// floor is q2's; when q2 is an integer the same holds one component down.
__device__ __forceinline__ long long floor_expansion(double q2, double q1, double q0) {
  const double f2 = floor(q2);
  if (f2 != q2) return (long long)f2;
  const double f1 = floor(q1);
  if (f1 != q1) return (long long)q2 + (long long)f1;
  return (long long)q2 + (long long)q1 + (long long)floor(q0);
}

// v / 2^e as an integer, read from the float's bits: its significand m (hidden bit
// included) times 2^p with p = biased exponent - 150 - e.  True when that value is an
// integer below 2^60 in magnitude (so that three of them sum exactly in int64).
__device__ __forceinline__ bool scaled_int(float v, int e, long long &out) {
  const uint32_t b = __float_as_uint(v);
  const int ex = (int)((b >> 23) & 0xffu);
  if (ex == 0xff) return false;  // not finite
  long long m = (long long)(b & 0x7fffffu);
  if (ex) m |= 0x800000ll;
  if (m == 0) {
    out = 0;
    return true;
  }
  const int p = (ex ? ex : 1) - 150 - e;
  if (p >= 0) {
    if (p > 36) return false;
    out = m << p;
  } else {
    if (p < -24 || (m & ((1ll << -p) - 1))) return false;  // a fraction remains
    out = m >> -p;
  }
  if (b >> 31) out = -out;
  return true;
}

// Lattice interval [floor, ceil] of d_j . v / 2^e for an FP32 vertex.  The three terms are
// exact (a float times +-1 or 0 and a power of two).  When all three are integers -- the
// usual case, since a float scaled into the lattice's range is an integer from 2^23 up --
// their sum, taken in int64, is both bounds.  Otherwise one Grow-Expansion in FP64 serves
// floor and ceil (the expansion of the negated sum is the negated expansion).
__device__ __forceinline__ void lattice_of(const float *v, int j, int e, long long &lo, long long &hi) {
  long long sum = 0;
  bool ints = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int d = c_rdir[j][c];
    long long x;
    if (d != 0) {
      ints = ints && scaled_int(v[c], e, x);
      sum += ints ? d * x : 0;
    }
  }
  if (ints) {
    lo = hi = sum;
    return;
  }
  const double inv = ldexp(1.0, -e);
  double t[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) t[c] = (double)c_rdir[j][c] * ((double)v[c] * inv);  // exact: scaling by 2^-e
  double x1, y1;
  two_sum(t[0], t[1], x1, y1);  // expansion [y1, x1]
  double q, q0, q1, q2;
  two_sum(t[2], y1, q, q0);
  two_sum(q, x1, q2, q1);  // expansion [q0, q1, q2]
  lo = floor_expansion(q2, q1, q0);
  hi = -floor_expansion(-q2, -q1, -q0);
}

}  // namespace
