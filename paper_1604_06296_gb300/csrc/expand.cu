// The two stages after a loop contraction, for every point of a view:
// * split-K combination of the partial sums into the loops of the rows
//   (fixed order; FP32 partials in compensated FP32 pairs, FP64 partials in
//   FP64);
// * loops of every transfer momentum from the loops of the rows (App. C): a
//   row computed at l serves the l' = g l of its list, chi(g l) =
//   R^g chi(l) R^g^T with f(g k) = R^g f(k).  The R^g of the C4v-adapted
//   basis are signed permutations, so this is a gather with signs; the
//   parity-forbidden entries (not computed) are written as zeros, so every
//   entry of chi is written.  One CTA per (point, row).
#include "device_util.cuh"

namespace tufrg {
namespace {

constexpr int kMaxNff = 32;

__global__ void expand_rows_kernel(const PointDesc* __restrict__ pts,
                                   const int* __restrict__ prefix, int n,
                                   const double* __restrict__ rowres, double* __restrict__ chi) {
  const int p = point_of(prefix, n, blockIdx.x);
  const PointDesc& pd = pts[p];
  if (pd.skip && *pd.skip) return;
  const int row = blockIdx.x - prefix[p];
  const int nff = pd.nff, n2 = nff * nff, nrow = pd.nrow, npair = pd.npair;
  __shared__ double X[2][kMaxNff * kMaxNff];
  for (int e = threadIdx.x; e < 2 * n2; e += blockDim.x) X[e / n2][e % n2] = 0.0;
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * npair; e += blockDim.x) {
    const int ch = e / npair, q = e % npair;
    const int mn = pd.pair[q], m = mn / nff, nn = mn % nff;
    const double v = rowres[pd.off_rowres + ((size_t)ch * nrow + row) * npair + q];
    X[ch][m * nff + nn] = v;
    X[ch][nn * nff + m] = v;
  }
  __syncthreads();
  for (int i = pd.rowimg_ptr[row]; i < pd.rowimg_ptr[row + 1]; ++i) {
    const int2 lg = pd.rowimg[i];
    const int* perm = pd.symperm + lg.y * nff;
    const int* sign = pd.symsign + lg.y * nff;
    for (int e = threadIdx.x; e < 2 * n2; e += blockDim.x) {
      const int ch = e / n2, r = e % n2, m = r / nff, nn = r % nff;
      chi[pd.off_chi + ((size_t)ch * pd.nl + lg.x) * n2 + r] =
          (double)(sign[m] * sign[nn]) * X[ch][perm[m] * nff + perm[nn]];
    }
  }
}

// Point-group covariance of a state: for every row, the largest deviation
// |y(l') - R^g y(l) R^g^T| over the (l', g) it serves (l its representative)
// and the largest |y(l')|, per point, as atomic maxima of the bit patterns of
// non-negative doubles.  One CTA per (point, row).
__global__ void covariance_check_kernel(const PointDesc* __restrict__ pts,
                                        const int* __restrict__ prefix, int n,
                                        const double* __restrict__ y,
                                        unsigned long long* __restrict__ out) {
  const int p = point_of(prefix, n, blockIdx.x);
  const PointDesc& pd = pts[p];
  const int row = blockIdx.x - prefix[p];
  const int nff = pd.nff, n2 = nff * nff;
  const size_t chan = (size_t)pd.nl * n2;
  const double* ys = y + pd.off_state;
  const int i0 = pd.rowimg_ptr[row], i1 = pd.rowimg_ptr[row + 1];
  const size_t rep = (size_t)pd.rowimg[i0].x * n2;
  double dev = 0.0, amax = 0.0;
  for (int i = i0; i < i1; ++i) {
    const int2 lg = pd.rowimg[i];
    const int* perm = pd.symperm + lg.y * nff;
    const int* sign = pd.symsign + lg.y * nff;
    for (int e = threadIdx.x; e < 3 * n2; e += blockDim.x) {
      const int ch = e / n2, r = e % n2, m = r / nff, nn = r % nff;
      const double v = ys[ch * chan + (size_t)lg.x * n2 + r];
      const double w = (double)(sign[m] * sign[nn]) * ys[ch * chan + rep + perm[m] * nff + perm[nn]];
      dev = fmax(dev, fabs(v - w));
      amax = fmax(amax, fabs(v));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    dev = fmax(dev, __shfl_down_sync(0xffffffffu, dev, o));
    amax = fmax(amax, __shfl_down_sync(0xffffffffu, amax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out + 2 * p, (unsigned long long)__double_as_longlong(dev));
    atomicMax(out + 2 * p + 1, (unsigned long long)__double_as_longlong(amax));
  }
}

// Split-K combination of one (channel, pair) and 32 rows: partial sums laid
// out as [split][2][P][R] (P pair stride, R row stride), FP64 result
// scaled by -1/4 (pp) / +1/4 (ph) (and 1/Omega^2 for the tensor-core
// partials) into rowres [2][nrow][npair].  Thread
// (row lane, phase) sums the splits sp = phase (mod kPhases) -- independent
// loads -- and the phases combine in a fixed order (deterministic).
//
// FP32 partials are summed as unevaluated pairs hi + lo of FP32 numbers
// (error-free transformation of each addition, Knuth's TwoSum), which carry
// ~44 significant bits -- far beyond the FP32 partials themselves -- at FP32
// speed; only the result is converted to FP64 (FP64 arithmetic runs at a
// small fraction of the FP32 rate on this GPU).  FP64 partials are summed in
// FP64.
constexpr int kPhases = 8;  // 256 threads: the whole grid resident in one wave

// (a.x + a.y) + b as a renormalised pair (TwoSum of the high parts, the low
// parts and the rounding error added, then a Fast2Sum)
__device__ __forceinline__ float2 pair_add(float2 a, float b) {
  const float s = a.x + b;
  const float bv = s - a.x;
  const float e = ((a.x - (s - bv)) + (b - bv)) + a.y;
  const float hi = s + e;
  return make_float2(hi, e - (hi - s));
}

__device__ __forceinline__ float2 pair_add(float2 a, float2 b) {
  const float s = a.x + b.x;
  const float bv = s - a.x;
  const float e = ((a.x - (s - bv)) + (b.x - bv)) + (a.y + b.y);
  const float hi = s + e;
  return make_float2(hi, e - (hi - s));
}

template <class T>
__device__ __forceinline__ void reduce_rows(const T* __restrict__ partial, int P, int R,
                                            int ksplit, int npair, int nrow, int row_end,
                                            int ch, int q, int row0,
                                            double* __restrict__ rowres, double factor) {
  const int lane = threadIdx.x & 31, phase = threadIdx.x >> 5;
  const int row = row0 + lane;
  const bool live = row < row_end;
  const T* src = partial + ((size_t)ch * P + q) * R + row;
  const size_t stride = (size_t)2 * P * R;
  const double scale = (ch == 0 ? -0.25 : 0.25) * factor;
  if constexpr (sizeof(T) == 4) {
    __shared__ float2 red[kPhases][33];
    float2 s = make_float2(0.f, 0.f);
    if (live) {
#pragma unroll 4
      for (int sp = phase; sp < ksplit; sp += kPhases) s = pair_add(s, __ldg(src + sp * stride));
    }
    red[phase][lane] = s;
    __syncthreads();
    if (phase == 0 && live) {
      float2 t = red[0][lane];
#pragma unroll
      for (int k = 1; k < kPhases; ++k) t = pair_add(t, red[k][lane]);
      rowres[((size_t)ch * nrow + row) * npair + q] = ((double)t.x + (double)t.y) * scale;
    }
  } else {
    __shared__ double red[kPhases][33];
    double s = 0.0;
    if (live) {
#pragma unroll 4
      for (int sp = phase; sp < ksplit; sp += kPhases) s += src[sp * stride];
    }
    red[phase][lane] = s;
    __syncthreads();
    if (phase == 0 && live) {
      double t = red[0][lane];
#pragma unroll
      for (int k = 1; k < kPhases; ++k) t += red[k][lane];
      rowres[((size_t)ch * nrow + row) * npair + q] = t * scale;
    }
  }
}

// tensor-core partials of every point: CTA -> (point, channel, pair, 32 rows
// of the rows the view computes)
__global__ void __launch_bounds__(32 * kPhases)
    tc_rows_kernel(const PointDesc* __restrict__ pts, const int* __restrict__ prefix, int n,
                   const float* __restrict__ partial, double* __restrict__ rowres) {
  const int p = point_of(prefix, n, blockIdx.x);
  const PointDesc& pd = pts[p];
  if (pd.skip && *pd.skip) return;
  const int tiles = (pd.row_hi - pd.row_lo + 31) / 32;
  const int loc = blockIdx.x - prefix[p];
  const int t = loc % tiles, r = loc / tiles, q = r % pd.npair, ch = r / pd.npair;
  // the tensor-core weights carry a factor Omega^2
  const double om = pd.lam[0];
  reduce_rows(partial + pd.off_partial, pd.npad, pd.nrow_pad, pd.ksplit, pd.npair, pd.nrow,
              pd.row_hi, ch, q, pd.row_lo + 32 * t, rowres + pd.off_rowres, 1.0 / (om * om));
}

// FP64-path partials of one context
__global__ void __launch_bounds__(32 * kPhases)
    fp64_rows_kernel(const double* __restrict__ partial, int mpad, int ksplit, int npair,
                     int nrow, double* __restrict__ rowres) {
  const int tiles = (nrow + 31) / 32;
  const int t = blockIdx.x % tiles, r = blockIdx.x / tiles, q = r % npair, ch = r / npair;
  reduce_rows(partial, mpad, nrow, ksplit, npair, nrow, nrow, ch, q, 32 * t, rowres, 1.0);
}

}  // namespace

int rows_reduce_ctas(int npair, int nrow) { return 2 * npair * ((nrow + 31) / 32); }

tufrg_status launch_tc_rows_multi(const MultiView& v, cudaStream_t st) {
  tc_rows_kernel<<<v.total(kKindReduce), 32 * kPhases, 0, st>>>(v.d, v.dprefix(kKindReduce), v.n,
                                                                v.d_partial, v.d_rowres);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

tufrg_status launch_fp64_rows(const double* partial, int mpad, int ksplit, int npair, int nrow,
                              double* rowres, cudaStream_t st) {
  fp64_rows_kernel<<<rows_reduce_ctas(npair, nrow), 32 * kPhases, 0, st>>>(
      partial, mpad, ksplit, npair, nrow, rowres);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

tufrg_status launch_covariance_check(const MultiView& v, const double* y,
                                     unsigned long long* dev, cudaStream_t st) {
  TUFRG_CUDA(cudaMemsetAsync(dev, 0, sizeof(unsigned long long) * 2 * v.n, st));
  covariance_check_kernel<<<v.total(kKindExpand), 128, 0, st>>>(v.d, v.dprefix(kKindExpand), v.n,
                                                                y, dev);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

tufrg_status launch_expand_multi(const MultiView& v, double* chi, cudaStream_t st) {
  if (v.nff_max > kMaxNff) return TUFRG_ERR_ARG;
  expand_rows_kernel<<<v.total(kKindExpand), 128, 0, st>>>(v.d, v.dprefix(kKindExpand), v.n,
                                                           v.d_rowres, chi);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

}  // namespace tufrg
