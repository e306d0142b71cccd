// Step iii, Eqs. (matmul-P/C/D): for every transfer momentum l
//   dP =  V^P chi^pp V^P
//   dC = -V^C chi^ph V^C
//   dD =  2 V^D chi^ph V^D - V^C chi^ph V^D - V^D chi^ph V^C
//      =  (2 V^D - V^C) (chi^ph V^D) - V^D (chi^ph V^C)
// One CTA per l; the five Nff x Nff operands and three intermediate products
// sit in shared memory (8 Nff^2 doubles <= 54 KB for Nff = 29).  FP64 for an
// FP64 context, FP32 arithmetic for the mixed-precision contexts.
#include "internal.h"

namespace tufrg {
namespace {

template <class T>
__device__ __forceinline__ void matmul(const T* __restrict__ a, const T* __restrict__ b,
                                       T* __restrict__ c, int n) {
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    T s = 0;
    for (int k = 0; k < n; ++k) s = fma(a[i * n + k], b[k * n + j], s);
    c[e] = s;
  }
}

// arithmetic in T (FP64, or FP32 for the mixed-precision contexts); inputs
// and the derivative are FP64
template <class T>
__global__ void products_kernel(const double* __restrict__ v, const double* __restrict__ chi,
                                double* __restrict__ dy, int nl, int nff,
                                const double* __restrict__ scale) {
  extern __shared__ double smd[];
  T* sm = reinterpret_cast<T*>(smd);
  const int n2 = nff * nff;
  T* VP = sm;
  T* VC = VP + n2;
  T* VD = VC + n2;
  T* Xp = VD + n2;
  T* Xh = Xp + n2;
  T* T1 = Xh + n2;
  T* T2 = T1 + n2;
  T* T3 = T2 + n2;
  const int l = blockIdx.x;
  const size_t chan = (size_t)nl * n2;
  const size_t off = (size_t)l * n2;
  for (int e = threadIdx.x; e < n2; e += blockDim.x) {
    VP[e] = (T)v[off + e];
    VC[e] = (T)v[chan + off + e];
    VD[e] = (T)v[2 * chan + off + e];
    Xp[e] = (T)chi[off + e];
    Xh[e] = (T)chi[chan + off + e];
  }
  __syncthreads();
  matmul(Xp, VP, T1, nff);  // chi^pp V^P
  matmul(Xh, VC, T2, nff);  // chi^ph V^C
  matmul(Xh, VD, T3, nff);  // chi^ph V^D
  __syncthreads();
  const double sc = scale ? scale[0] : 1.0;
  for (int e = threadIdx.x; e < n2; e += blockDim.x) {
    const int i = e / nff, j = e % nff;
    T p = 0, cc = 0, d = 0;
    for (int k = 0; k < nff; ++k) {
      p = fma(VP[i * nff + k], T1[k * nff + j], p);
      cc = fma(VC[i * nff + k], T2[k * nff + j], cc);
      d = fma(2 * VD[i * nff + k] - VC[i * nff + k], T3[k * nff + j], d);
      d = fma(-VD[i * nff + k], T2[k * nff + j], d);
    }
    dy[off + e] = sc * (double)p;
    dy[chan + off + e] = -sc * (double)cc;
    dy[2 * chan + off + e] = sc * (double)d;
  }
}

}  // namespace

tufrg_status prepare_products(tufrg_ctx* c) {
  const size_t smem = sizeof(double) * 8 * c->nff * c->nff;
  if (smem > 48 * 1024) {
    TUFRG_CUDA(cudaFuncSetAttribute(products_kernel<double>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TUFRG_CUDA(cudaFuncSetAttribute(products_kernel<float>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  return TUFRG_OK;
}

tufrg_status launch_products(tufrg_ctx* c, int prec, const double* v, const double* chi,
                             double* dy, const double* d_scale, cudaStream_t st) {
  if (prec == TUFRG_FP64) {
    const size_t smem = sizeof(double) * 8 * c->nff * c->nff;
    products_kernel<double><<<c->nl, 256, smem, st>>>(v, chi, dy, c->nl, c->nff, d_scale);
  } else {
    const size_t smem = sizeof(float) * 8 * c->nff * c->nff;
    products_kernel<float><<<c->nl, 256, smem, st>>>(v, chi, dy, c->nl, c->nff, d_scale);
  }
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

}  // namespace tufrg
