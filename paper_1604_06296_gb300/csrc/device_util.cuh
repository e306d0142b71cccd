// Device helpers shared by the multi-point kernels.
#pragma once

#include <type_traits>

#include "internal.h"

namespace tufrg {

// The point owning CTA b of a multi-point launch whose point p owns CTAs
// [prefix[p], prefix[p + 1]): the largest p with prefix[p] <= b.
__device__ __forceinline__ int point_of(const int* __restrict__ prefix, int n, int b) {
  int lo = 0, hi = n;  // prefix[lo] <= b < prefix[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(prefix + mid) <= b)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// paired FP32 arithmetic (one instruction for both lanes of a float2, each
// lane rounded as its scalar operation)
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 d;
  asm("{\n .reg .b64 x, y, z;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n"
      " sub.rn.f32x2 z, x, y;\n mov.b64 {%0, %1}, z;\n}\n"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// FP32 -> FP64, exact, on the integer pipe (GB300 converts on its FP64 pipe,
// at a small fraction of the FP32 rate): normal numbers and zeros by their
// bits, the rest (subnormal, infinite, NaN) by the conversion instruction
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0xffu || (e == 0 && (u & 0x7fffffu) != 0)) return (double)f;
  const unsigned sign = u & 0x80000000u;
  if (e == 0) return __hiloint2double((int)sign, 0);
  return __hiloint2double((int)(sign | ((e + 896u) << 20) | ((u >> 3) & 0xfffffu)),
                          (int)(u << 29));
}

// FP64 -> FP32 rounded to nearest even, on the integer pipe: numbers whose
// result is a normal FP32 number (and zeros) by their bits -- the 23 leading
// mantissa bits, plus one when the 29 dropped bits are above half, or at
// half with the kept part odd (a carry moves into the exponent, up to
// infinity) -- the rest by the conversion instruction
__device__ __forceinline__ float d2f(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  if ((b << 1) == 0) return __uint_as_float(sign);
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e < 897u || e > 1150u) return (float)x;
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1fffffffu;
  unsigned f = (sign | ((e - 896u) << 23)) + m;
  if (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) f += 1u;
  return __uint_as_float(f);
}

// Kernels over form-factor matrices are compiled for the sizes of complete
// shells (Nff = Nb = 5, 9, 13, 21, 25, 29) so their loops unroll, and for
// any size (NF = 0).  f(std::integral_constant<int, NF>) for v's size.
template <class F>
auto with_nf(int nf_uniform, F&& f) {
  switch (nf_uniform) {
    case 5: return f(std::integral_constant<int, 5>{});
    case 9: return f(std::integral_constant<int, 9>{});
    case 13: return f(std::integral_constant<int, 13>{});
    case 21: return f(std::integral_constant<int, 21>{});
    case 25: return f(std::integral_constant<int, 25>{});
    case 29: return f(std::integral_constant<int, 29>{});
    default: return f(std::integral_constant<int, 0>{});
  }
}
template <class F>
void for_each_nf(F&& f) {
  f(std::integral_constant<int, 0>{});
  f(std::integral_constant<int, 5>{});
  f(std::integral_constant<int, 9>{});
  f(std::integral_constant<int, 13>{});
  f(std::integral_constant<int, 21>{});
  f(std::integral_constant<int, 25>{});
  f(std::integral_constant<int, 29>{});
}

}  // namespace tufrg
