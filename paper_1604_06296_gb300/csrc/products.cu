// Step iii, Eqs. (matmul-P/C/D): for every transfer momentum l
//   dP =  V^P chi^pp V^P
//   dC = -V^C chi^ph V^C
//   dD =  2 V^D chi^ph V^D - V^C chi^ph V^D - V^D chi^ph V^C
//      =  (2 V^D - V^C) (chi^ph V^D) - V^D (chi^ph V^C)
// One CTA per (point, l) over all points of a batch; the five Nff x Nff
// operands and three intermediate products sit in shared memory (8 Nff^2
// doubles <= 54 KB for Nff = 29).  FP64 for an FP64 context, FP32 arithmetic
// for the mixed-precision contexts.
#include "device_util.cuh"

namespace tufrg {
namespace {

// arithmetic in T (FP64, or FP32 for the mixed-precision contexts); inputs
// and the derivative are FP64; dy is multiplied by lam[1] when scaled
// chibase == nullptr: the loops of l are gathered from the loops of the row
// serving l (rowres), chi(l)_mn = s_m s_n chi(row)_{p(m) p(n)} with the
// signed permutation of the group element that maps the row's l to l.
template <class T, int NF>
__global__ void products_kernel(const PointDesc* __restrict__ pts,
                                const int* __restrict__ prefix, int np,
                                const double* __restrict__ vbase,
                                const double* __restrict__ chibase,
                                const double* __restrict__ rowres, double* __restrict__ dybase,
                                int scaled) {
  const int p = point_of(prefix, np, blockIdx.x);
  const PointDesc& pd = pts[p];
  if (pd.skip && *pd.skip) return;
  const int nl = pd.nl, nff = NF ? NF : pd.nff;
  const int l = blockIdx.x - prefix[p];
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
  const size_t chan = (size_t)nl * n2;
  const size_t off = (size_t)l * n2;
  const double* v = vbase + pd.off_state;
  double* dy = dybase + pd.off_state;
  for (int e = threadIdx.x; e < n2; e += blockDim.x) {
    VP[e] = (T)v[off + e];
    VC[e] = (T)v[chan + off + e];
    VD[e] = (T)v[2 * chan + off + e];
  }
  if (chibase) {
    const double* chi = chibase + pd.off_chi;
    for (int e = threadIdx.x; e < n2; e += blockDim.x) {
      Xp[e] = (T)chi[off + e];
      Xh[e] = (T)chi[chan + off + e];
    }
  } else {
    // one gather table entry per (m, n): the signed index into the row loops
    const int* gi = pd.lgather + (size_t)l * n2;
    const double* rp = rowres + pd.off_rowres;
    const size_t ch1 = (size_t)pd.nrow * pd.npair;
    for (int e = threadIdx.x; e < n2; e += blockDim.x) {
      const int v = __ldg(gi + e);
      const int q = abs(v) - 1;
      const T sg = v > 0 ? (T)1 : (T)-1;
      Xp[e] = v != 0 ? sg * (T)rp[q] : (T)0;
      Xh[e] = v != 0 ? sg * (T)rp[ch1 + q] : (T)0;
    }
  }
  __syncthreads();
  // chi^pp V^P, chi^ph V^C, chi^ph V^D as one loop over their 3 Nff^2 entries
  for (int e = threadIdx.x; e < 3 * n2; e += blockDim.x) {
    const int w = e / n2, ij = e - w * n2, i = ij / nff, j = ij - i * nff;
    const T* a = (w == 0 ? Xp : Xh) + i * nff;
    const T* b = (w == 0 ? VP : (w == 1 ? VC : VD)) + j;
    T s = 0;
    for (int k = 0; k < nff; ++k) s = fma(a[k], b[k * nff], s);
    (w == 0 ? T1 : (w == 1 ? T2 : T3))[ij] = s;
  }
  __syncthreads();
  const double sc = scaled ? pd.lam[1] : 1.0;
  for (int e = threadIdx.x; e < n2; e += blockDim.x) {
    const int i = e / nff, j = e % nff;
    T pp = 0, cc = 0, d = 0;
    for (int k = 0; k < nff; ++k) {
      pp = fma(VP[i * nff + k], T1[k * nff + j], pp);
      cc = fma(VC[i * nff + k], T2[k * nff + j], cc);
      d = fma(2 * VD[i * nff + k] - VC[i * nff + k], T3[k * nff + j], d);
      d = fma(-VD[i * nff + k], T2[k * nff + j], d);
    }
    dy[off + e] = sc * (double)pp;
    dy[chan + off + e] = -sc * (double)cc;
    dy[2 * chan + off + e] = sc * (double)d;
  }
}

// The products of a point-group covariant state (wedge layout: state,
// couplings and derivative at the representative l of each loop row only,
// [3][nrow][nff][nff]).  The loops of a representative are its row loops
// themselves; the right-hand side of a covariant state (B(g l) =
// R^g B(l) R^g^T for every g that maps l into the zone without a fold,
// App. C) is covariant in the same way, so the representatives determine it.
// One CTA per (point, row).
template <class T, int NF>
__global__ void products_rows_kernel(const PointDesc* __restrict__ pts,
                                     const int* __restrict__ prefix, int np,
                                     const double* __restrict__ vbase,
                                     const double* __restrict__ rowres,
                                     double* __restrict__ dybase, int scaled) {
  const int p = point_of(prefix, np, blockIdx.x);
  const PointDesc& pd = pts[p];
  if (pd.skip && *pd.skip) return;
  const int nff = NF ? NF : pd.nff;
  const int row = blockIdx.x - prefix[p];
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
  const size_t chan = (size_t)pd.nrow * n2;
  const size_t off = pd.off_wstate + (size_t)row * n2;
  for (int e = threadIdx.x; e < n2; e += blockDim.x) {
    VP[e] = (T)vbase[off + e];
    VC[e] = (T)vbase[chan + off + e];
    VD[e] = (T)vbase[2 * chan + off + e];
  }
  const double* rp = rowres + pd.off_rowres + (size_t)row * pd.npair;
  const size_t ch1 = (size_t)pd.nrow * pd.npair;
  for (int e = threadIdx.x; e < n2; e += blockDim.x) {
    const int q = __ldg(pd.pairidx + e);
    Xp[e] = q >= 0 ? (T)rp[q] : (T)0;
    Xh[e] = q >= 0 ? (T)rp[ch1 + q] : (T)0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 3 * n2; e += blockDim.x) {
    const int w = e / n2, ij = e - w * n2, i = ij / nff, j = ij - i * nff;
    const T* a = (w == 0 ? Xp : Xh) + i * nff;
    const T* b = (w == 0 ? VP : (w == 1 ? VC : VD)) + j;
    T s = 0;
    for (int k = 0; k < nff; ++k) s = fma(a[k], b[k * nff], s);
    (w == 0 ? T1 : (w == 1 ? T2 : T3))[ij] = s;
  }
  __syncthreads();
  const double sc = scaled ? pd.lam[1] : 1.0;
  double* dy = dybase + off;
  for (int e = threadIdx.x; e < n2; e += blockDim.x) {
    const int i = e / nff, j = e % nff;
    T a = 0, c = 0, d = 0;
    for (int k = 0; k < nff; ++k) {
      a = fma(VP[i * nff + k], T1[k * nff + j], a);
      c = fma(VC[i * nff + k], T2[k * nff + j], c);
      d = fma(2 * VD[i * nff + k] - VC[i * nff + k], T3[k * nff + j], d);
      d = fma(-VD[i * nff + k], T2[k * nff + j], d);
    }
    dy[e] = sc * (double)a;
    dy[chan + e] = -sc * (double)c;
    dy[2 * chan + e] = sc * (double)d;
  }
}

}  // namespace

tufrg_status prepare_products_multi(const MultiView& v) {
  const int smem = smem_optin();
  if (sizeof(double) * 8 * v.nff_max * v.nff_max > (size_t)smem) return TUFRG_ERR_ARG;
  cudaError_t e = cudaSuccess;
  for_each_nf([&](auto nf) {
    constexpr int NF = decltype(nf)::value;
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(products_kernel<double, NF>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(products_kernel<float, NF>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(products_rows_kernel<double, NF>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(products_rows_kernel<float, NF>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  });
  TUFRG_CUDA(e);
  return TUFRG_OK;
}

tufrg_status launch_products_multi(const MultiView& v, int prec, const double* vin,
                                   const double* chi, double* dy, bool scaled, cudaStream_t st,
                                   bool rows) {
  if (rows && !chi) {
    const int blocks = v.total(kKindProductsRows);
    with_nf(v.nf_uniform, [&](auto nf) {
      constexpr int NF = decltype(nf)::value;
      if (prec == TUFRG_FP64)
        products_rows_kernel<double, NF><<<blocks, 256, sizeof(double) * 8 * v.nff_max *
                                                            v.nff_max, st>>>(
            v.d, v.dprefix(kKindProductsRows), v.n, vin, v.d_rowres, dy, scaled ? 1 : 0);
      else
        products_rows_kernel<float, NF><<<blocks, 256, sizeof(float) * 8 * v.nff_max *
                                                           v.nff_max, st>>>(
            v.d, v.dprefix(kKindProductsRows), v.n, vin, v.d_rowres, dy, scaled ? 1 : 0);
    });
    TUFRG_CUDA(cudaGetLastError());
    return TUFRG_OK;
  }
  const int blocks = v.total(kKindProducts);
  with_nf(v.nf_uniform, [&](auto nf) {
    constexpr int NF = decltype(nf)::value;
    if (prec == TUFRG_FP64) {
      const size_t smem = sizeof(double) * 8 * v.nff_max * v.nff_max;
      products_kernel<double, NF><<<blocks, 256, smem, st>>>(
          v.d, v.dprefix(kKindProducts), v.n, vin, chi, v.d_rowres, dy, scaled ? 1 : 0);
    } else {
      const size_t smem = sizeof(float) * 8 * v.nff_max * v.nff_max;
      products_kernel<float, NF><<<blocks, 256, smem, st>>>(
          v.d, v.dprefix(kKindProducts), v.n, vin, chi, v.d_rowres, dy, scaled ? 1 : 0);
    }
  });
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

}  // namespace tufrg
