// Self-tests (no counterpart in the paper): the bounded device waits and the
// library's FP64 <-> FP32 conversions.
//
// The tensor-core kernels wait on shared-memory mbarriers with a time limit;
// a wait that runs out sets the context's error word (reported by
// tufrg_check as TUFRG_ERR_TIMEOUT) and the kernel returns, so the context
// stays usable.  This kernel exercises that path on purpose: it waits on a
// barrier that nothing arrives at, for a short limit, and records the
// timeout the same way.
#include "internal.h"
#include "tc_util.cuh"

namespace tufrg {
namespace {

using namespace tc;

__global__ void wait_selftest_kernel(int* __restrict__ err, unsigned long long limit_ns) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = smem_u32(&bar);
  mbar_init(b, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!mbar_wait_for(b, 0, limit_ns)) atomicOr(err, 8);  // no arrival: runs out
}

}  // namespace
}  // namespace tufrg

extern "C" tufrg_status tufrg_selftest_convert(const double* x_dev, float* y32_dev,
                                               double* back_dev, int64_t n, void* stream) {
  if (!x_dev || !y32_dev || !back_dev || n < 0) return TUFRG_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  TUFRG_CHECK(tufrg::launch_to_f32(x_dev, y32_dev, (size_t)n, st));
  return tufrg::launch_to_f64(y32_dev, back_dev, (size_t)n, st);
}

extern "C" tufrg_status tufrg_selftest_wait(tufrg_ctx* c, int32_t wait_us, void* stream) {
  if (!c || !c->d_err || wait_us < 1 || wait_us > 100000) return TUFRG_ERR_ARG;
  tufrg::wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(
      c->d_err, (unsigned long long)wait_us * 1000ull);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}
