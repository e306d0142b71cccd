// Step iii, Eqs. (matmul-P/C/D): for every transfer momentum l
//   dP =  V^P chi^pp V^P
//   dC = -V^C chi^ph V^C
//   dD =  2 V^D chi^ph V^D - V^C chi^ph V^D - V^D chi^ph V^C
//      =  (2 V^D - V^C) (chi^ph V^D) - V^D (chi^ph V^C)
// One CTA per (point, l) over all points of a batch; the five Nff x Nff
// operands and three intermediate products sit in shared memory (8 Nff x
// (Nff rounded up to even) values, <= 56 KB for Nff = 29).  FP64 for an FP64
// context, FP32 arithmetic for the mixed-precision contexts.
#include "device_util.cuh"

namespace tufrg {
namespace {

// a pair of adjacent entries of one row, and acc + a * (b0, b1) lane-wise
template <class T>
struct Pair;
template <>
struct Pair<float> {
  using type = float2;
};
template <>
struct Pair<double> {
  using type = double2;
};
__device__ __forceinline__ float2 pfma(float a, float2 b, float2 acc) {
  return fma2(make_float2(a, a), b, acc);
}
__device__ __forceinline__ double2 pfma(double a, double2 b, double2 acc) {
  return {fma(a, b.x, acc.x), fma(a, b.y, acc.y)};
}

// an entry of dy: sc * v in FP64 arithmetic, or for FP32 arithmetic
// (float)sc * v rounded in FP32 and converted exactly (sc given in T)
__device__ __forceinline__ double to_out(double sc, double v) { return sc * v; }
__device__ __forceinline__ double to_out(float sc, float v) { return f2d(sc * v); }

// an FP64 loop value in the arithmetic type
template <class T>
__device__ __forceinline__ T to_t(double v);
template <>
__device__ __forceinline__ double to_t<double>(double v) {
  return v;
}
template <>
__device__ __forceinline__ float to_t<float>(double v) {
  return d2f(v);
}

// Row stride of the matrices in shared memory: Nff rounded up to even, so
// that every (row, even column) pair is one aligned 2-element load.
__host__ __device__ constexpr int pstride(int nff) { return (nff + 1) & ~1; }
// shared memory of the two product kernels: eight matrices
template <class T>
size_t products_smem(int nff) {
  return sizeof(T) * 8 * (size_t)nff * pstride(nff);
}

// The products of one l from VP, VC, VD, Xp (= chi^pp), Xh (= chi^ph) in
// shared memory (stride pstride(nff), padding columns zero); writes
// dy[ch * chan + m * nff + n] for the three channels, P scaled by sc_p, C and
// D by sc_cd.  Each
// thread computes a pair of adjacent entries of a row (two lanes of one
// paired FP32 instruction; every lane takes the scalar form's roundings in
// the scalar form's order).
template <class T, int NF>
__device__ __forceinline__ void products_in_smem(T* sm, int nff_rt, double sc_p, double sc_cd,
                                                 double* __restrict__ dy, size_t chan) {
  using P = typename Pair<T>::type;
  const int nff = NF ? NF : nff_rt;
  const int S = pstride(nff), hp = S / 2, m2 = nff * S;
  const T sct = to_t<T>(sc_p), scd = to_t<T>(sc_cd);
  T* VP = sm;
  T* VC = VP + m2;
  T* VD = VC + m2;
  T* Xp = VD + m2;
  T* Xh = Xp + m2;
  T* T1 = Xh + m2;
  T* T2 = T1 + m2;
  T* T3 = T2 + m2;
  // chi^pp V^P, chi^ph V^C, chi^ph V^D as one loop over (matrix, row, pair)
  for (int e = threadIdx.x; e < 3 * nff * hp; e += blockDim.x) {
    const int w = e / (nff * hp), r = e - w * nff * hp, i = r / hp, j = 2 * (r - i * hp);
    const T* a = (w == 0 ? Xp : Xh) + i * S;
    const T* b = (w == 0 ? VP : (w == 1 ? VC : VD)) + j;
    P s = {0, 0};
#pragma unroll 5
    for (int k = 0; k < nff; ++k) s = pfma(a[k], *reinterpret_cast<const P*>(b + k * S), s);
    *reinterpret_cast<P*>((w == 0 ? T1 : (w == 1 ? T2 : T3)) + i * S + j) = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nff * hp; e += blockDim.x) {
    const int i = e / hp, j = 2 * (e - i * hp);
    P pp = {0, 0}, cc = {0, 0}, d = {0, 0};
#pragma unroll 5
    for (int k = 0; k < nff; ++k) {
      const T vp = VP[i * S + k], vc = VC[i * S + k], vd = VD[i * S + k];
      const P t1 = *reinterpret_cast<const P*>(T1 + k * S + j);
      const P t2 = *reinterpret_cast<const P*>(T2 + k * S + j);
      const P t3 = *reinterpret_cast<const P*>(T3 + k * S + j);
      pp = pfma(vp, t1, pp);
      cc = pfma(vc, t2, cc);
      d = pfma(2 * vd - vc, t3, d);
      d = pfma(-vd, t2, d);
    }
    const int o = i * nff + j;
    dy[o] = to_out(sct, pp.x);
    dy[chan + o] = to_out(-scd, cc.x);
    dy[2 * chan + o] = to_out(scd, d.x);
    if (j + 1 < nff) {
      dy[o + 1] = to_out(sct, pp.y);
      dy[chan + o + 1] = to_out(-scd, cc.y);
      dy[2 * chan + o + 1] = to_out(scd, d.y);
    }
  }
}

// entry e of an Nff x Nff matrix into shared memory at stride S; the padding
// column (odd Nff) is written as zero by the entry before it
template <class T>
__device__ __forceinline__ void put(T* m, int e, int nff, int S, T v) {
  const int i = e / nff, j = e - i * nff;
  m[i * S + j] = v;
  if (j == nff - 1 && S != nff) m[i * S + j + 1] = 0;
}

// arithmetic in T (FP64, or FP32 for the mixed-precision contexts); the
// couplings in T, the loops and the derivative FP64; dy is multiplied by
// lam[1] when scaled
// chibase == nullptr: the loops of l are gathered from the loops of the row
// serving l (rowres), chi(l)_mn = s_m s_n chi(row)_{p(m) p(n)} with the
// signed permutation of the group element that maps the row's l to l.
template <class T, int NF>
__global__ void products_kernel(const PointDesc* __restrict__ pts,
                                const int* __restrict__ prefix, int np,
                                const T* __restrict__ vbase,
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
  const int n2 = nff * nff, S = pstride(nff), m2 = nff * S;
  T* VP = sm;
  T* VC = VP + m2;
  T* VD = VC + m2;
  T* Xp = VD + m2;
  T* Xh = Xp + m2;
  const size_t chan = (size_t)nl * n2;
  const size_t off = (size_t)l * n2;
  const T* v = vbase + pd.off_state;
  for (int e = threadIdx.x; e < n2; e += blockDim.x) {
    put(VP, e, nff, S, v[off + e]);
    put(VC, e, nff, S, v[chan + off + e]);
    put(VD, e, nff, S, v[2 * chan + off + e]);
  }
  if (chibase) {
    const double* chi = chibase + pd.off_chi;
    for (int e = threadIdx.x; e < n2; e += blockDim.x) {
      put(Xp, e, nff, S, to_t<T>(chi[off + e]));
      put(Xh, e, nff, S, to_t<T>(chi[chan + off + e]));
    }
  } else {
    // one gather table entry per (m, n): the signed index into the row loops
    const int* gi = pd.lgather + (size_t)l * n2;
    const double* rp = rowres + pd.off_rowres;
    const size_t ch1 = (size_t)pd.nrow * pd.npair;
    for (int e = threadIdx.x; e < n2; e += blockDim.x) {
      const int g = __ldg(gi + e);
      const int q = abs(g) - 1;
      const T sg = g > 0 ? (T)1 : (T)-1;
      put(Xp, e, nff, S, g != 0 ? sg * to_t<T>(rp[q]) : (T)0);
      put(Xh, e, nff, S, g != 0 ? sg * to_t<T>(rp[ch1 + q]) : (T)0);
    }
  }
  __syncthreads();
  // on a non-uniform mesh a channel's derivative vanishes off its own mesh
  const double sc = scaled ? pd.lam[1] : 1.0;
  const double sc_p = pd.mesh_w && pd.mesh_w[l] == 0.0 ? 0.0 : sc;
  const double sc_cd = pd.mesh_w && pd.mesh_w[nl + l] == 0.0 ? 0.0 : sc;
  products_in_smem<T, NF>(sm, nff, sc_p, sc_cd, dybase + pd.off_state + off, chan);
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
                                     const T* __restrict__ vbase,
                                     const double* __restrict__ rowres,
                                     double* __restrict__ dybase, int scaled) {
  const int p = point_of(prefix, np, blockIdx.x);
  const PointDesc& pd = pts[p];
  if (pd.skip && *pd.skip) return;
  const int nff = NF ? NF : pd.nff;
  const int row = blockIdx.x - prefix[p];
  extern __shared__ double smd[];
  T* sm = reinterpret_cast<T*>(smd);
  const int n2 = nff * nff, S = pstride(nff), m2 = nff * S;
  T* VP = sm;
  T* VC = VP + m2;
  T* VD = VC + m2;
  T* Xp = VD + m2;
  T* Xh = Xp + m2;
  const size_t chan = (size_t)pd.nrow * n2;
  const size_t off = pd.off_wstate + (size_t)row * n2;
  for (int e = threadIdx.x; e < n2; e += blockDim.x) {
    put(VP, e, nff, S, vbase[off + e]);
    put(VC, e, nff, S, vbase[chan + off + e]);
    put(VD, e, nff, S, vbase[2 * chan + off + e]);
  }
  const double* rp = rowres + pd.off_rowres + (size_t)row * pd.npair;
  const size_t ch1 = (size_t)pd.nrow * pd.npair;
  for (int e = threadIdx.x; e < n2; e += blockDim.x) {
    const int q = __ldg(pd.pairidx + e);
    put(Xp, e, nff, S, q >= 0 ? to_t<T>(rp[q]) : (T)0);
    put(Xh, e, nff, S, q >= 0 ? to_t<T>(rp[ch1 + q]) : (T)0);
  }
  __syncthreads();
  // on a non-uniform mesh a channel's derivative vanishes off its own mesh
  // (the images a row serves carry the representative's weights)
  const double sc = scaled ? pd.lam[1] : 1.0;
  const int l0 = pd.rowimg[pd.rowimg_ptr[row]].x;
  const double sc_p = pd.mesh_w && pd.mesh_w[l0] == 0.0 ? 0.0 : sc;
  const double sc_cd = pd.mesh_w && pd.mesh_w[pd.nl + l0] == 0.0 ? 0.0 : sc;
  products_in_smem<T, NF>(sm, nff, sc_p, sc_cd, dybase + off, chan);
}

}  // namespace

tufrg_status prepare_products_multi(const MultiView& v) {
  const int smem = smem_optin();
  if (products_smem<double>(v.nff_max) > (size_t)smem) return TUFRG_ERR_ARG;
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

tufrg_status launch_products_multi(const MultiView& v, int prec, const void* vin,
                                   const double* chi, double* dy, bool scaled, cudaStream_t st,
                                   bool rows) {
  const bool f64 = prec == TUFRG_FP64;
  const size_t smem = f64 ? products_smem<double>(v.nff_max) : products_smem<float>(v.nff_max);
  if (rows && !chi) {
    const int blocks = v.total(kKindProductsRows);
    with_nf(v.nf_uniform, [&](auto nf) {
      constexpr int NF = decltype(nf)::value;
      if (f64)
        products_rows_kernel<double, NF><<<blocks, 256, smem, st>>>(
            v.d, v.dprefix(kKindProductsRows), v.n, static_cast<const double*>(vin),
            v.d_rowres, dy, scaled ? 1 : 0);
      else
        products_rows_kernel<float, NF><<<blocks, 256, smem, st>>>(
            v.d, v.dprefix(kKindProductsRows), v.n, static_cast<const float*>(vin), v.d_rowres,
            dy, scaled ? 1 : 0);
    });
    TUFRG_CUDA(cudaGetLastError());
    return TUFRG_OK;
  }
  const int blocks = v.total(kKindProducts);
  with_nf(v.nf_uniform, [&](auto nf) {
    constexpr int NF = decltype(nf)::value;
    if (f64)
      products_kernel<double, NF><<<blocks, 256, smem, st>>>(
          v.d, v.dprefix(kKindProducts), v.n, static_cast<const double*>(vin), chi, v.d_rowres,
          dy, scaled ? 1 : 0);
    else
      products_kernel<float, NF><<<blocks, 256, smem, st>>>(
          v.d, v.dprefix(kKindProducts), v.n, static_cast<const float*>(vin), chi, v.d_rowres,
          dy, scaled ? 1 : 0);
  });
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

}  // namespace tufrg
