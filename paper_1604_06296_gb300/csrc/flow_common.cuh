// Device-side pieces shared by the single-point and multi-point flow
// integrators: the Dormand-Prince 5(4) tableau, the control block of one
// flow, the step-size control and the cubic Hermite interpolant.
#pragma once

#include "internal.h"

namespace tufrg {
namespace {

// Dormand-Prince 5(4) tableau
const double kC[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
const double kA[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
    {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
const double kB[7] = {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0.0};
const double kBs[7] = {5179.0 / 57600, 0.0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200,
                       187.0 / 2100, 1.0 / 40};
constexpr double kFacSafety = 0.9, kFacMin = 0.2, kFacMax = 5.0;
constexpr int kBisect = 100;

struct FlowCtl {
  double s, h, s_end, s_prev;
  double rtol, atol, thr, dir;
  unsigned long long err_u, max_u, bis_u, arg_u;
  double bis_a, bis_b;
  int nonfinite, accepted, last_rejected, crossed, done, status;
  long long n_acc, n_rej, n_rhs;
  double ymax_last;  // max |y| after the last accepted step
};


__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(fabs(v));
}

__device__ void block_max_u(unsigned long long v, unsigned long long* target) {
  __shared__ unsigned long long red[32];
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0ull;
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0 && v) atomicMax(target, v);
  }
  __syncthreads();
}

struct Combo {
  const double* k[7];
  double a[7];
  int nk;
  double c;  // stage node: Lambda = exp(s + c h)
};

// sum_j a_j k_j[i] over the nk terms, in the order of j.  The loop has
// constant bounds so that the kernel parameter is indexed with constants (a
// runtime index makes every thread copy it to local memory first).
__device__ __forceinline__ double combo_sum(const Combo& cb, size_t i) {
  double acc = 0.0;
#pragma unroll
  for (int j = 0; j < 7; ++j)
    if (j < cb.nk) acc = fma(cb.a[j], cb.k[j][i], acc);
  return acc;
}

// Step-size control after the error norm of an attempt (see the file header).
__device__ __forceinline__ void control_update(FlowCtl* c) {
  const double err = __longlong_as_double((long long)c->err_u);
  c->accepted = 0;
  c->crossed = 0;
  if (c->nonfinite || !isfinite(err)) {
    c->status = TUFRG_ERR_NONFINITE;
    c->done = 1;
    return;
  }
  c->n_rhs += 6;
  if (err <= 1.0) {
    double fac = err == 0.0 ? kFacMax : fmin(kFacMax, fmax(kFacMin, kFacSafety * pow(err, -0.2)));
    if (c->last_rejected) fac = fmin(fac, 1.0);
    c->s_prev = c->s;
    c->s = c->s + c->h;
    c->accepted = 1;
    c->n_acc += 1;
    const double ymax = __longlong_as_double((long long)c->max_u);
    c->ymax_last = ymax;
    c->crossed = ymax > c->thr;
    c->h = c->h * fac;
    c->last_rejected = 0;
    if (c->crossed || (c->s_end - c->s) * c->dir <= 0.0) c->done = 1;
  } else {
    c->n_rej += 1;
    c->h = c->h * fmax(kFacMin, kFacSafety * pow(err, -0.2));
    c->last_rejected = 1;
  }
  if (!c->done && fabs(c->h) < 1e-12) {
    c->status = TUFRG_ERR_STEP_UNDERFLOW;
    c->done = 1;
  }
  if ((c->s + c->h - c->s_end) * c->dir > 0.0) c->h = c->s_end - c->s;
  c->err_u = 0;
  c->max_u = 0;
}

__device__ __forceinline__ double hermite(double s0, double y0, double f0, double s1, double y1,
                                          double f1, double s) {
  const double h = s1 - s0, th = (s - s0) / h;
  const double h00 = 2 * th * th * th - 3 * th * th + 1;
  const double h10 = th * th * th - 2 * th * th + th;
  const double h01 = -2 * th * th * th + 3 * th * th;
  const double h11 = th * th * th - th * th;
  return h00 * y0 + h10 * h * f0 + h01 * y1 + h11 * h * f1;
}

}  // namespace
}  // namespace tufrg
