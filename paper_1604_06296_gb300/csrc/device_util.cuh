// Device helpers shared by the multi-point kernels.
#pragma once

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

}  // namespace tufrg
