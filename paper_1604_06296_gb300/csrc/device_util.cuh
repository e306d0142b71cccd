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
