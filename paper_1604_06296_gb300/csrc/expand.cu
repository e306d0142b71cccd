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
#include <algorithm>

#include "device_util.cuh"

namespace tufrg {
namespace {

__global__ void expand_rows_kernel(const PointDesc* __restrict__ pts,
                                   const int* __restrict__ prefix, int n,
                                   const double* __restrict__ rowres, double* __restrict__ chi) {
  const int p = point_of(prefix, n, blockIdx.x);
  const PointDesc& pd = pts[p];
  if (pd.skip && *pd.skip) return;
  const int row = blockIdx.x - prefix[p];
  const int nff = pd.nff, n2 = nff * nff, nrow = pd.nrow, npair = pd.npair;
  __shared__ double X[2][kMaxNf * kMaxNf];
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

// Wedge layout of a point-group covariant state: its values at the
// representative l of each loop row, [3][nrow][nff][nff].  compress takes
// them from the full state; expand writes every l a row serves as
// y(g l) = R^g y(l) R^g^T.  One CTA per (point, row).
__global__ void wedge_compress_kernel(const PointDesc* __restrict__ pts,
                                      const int* __restrict__ prefix, int n,
                                      const double* __restrict__ y, double* __restrict__ w) {
  const int p = point_of(prefix, n, blockIdx.x);
  const PointDesc& pd = pts[p];
  const int row = blockIdx.x - prefix[p];
  const int n2 = pd.nff * pd.nff;
  const size_t rep = (size_t)pd.rowimg[pd.rowimg_ptr[row]].x * n2;
  for (int e = threadIdx.x; e < 3 * n2; e += blockDim.x) {
    const int ch = e / n2, r = e - ch * n2;
    w[pd.off_wstate + ((size_t)ch * pd.nrow + row) * n2 + r] =
        y[pd.off_state + (size_t)ch * pd.nl * n2 + rep + r];
  }
}

__global__ void wedge_expand_kernel(const PointDesc* __restrict__ pts,
                                    const int* __restrict__ prefix, int n,
                                    const double* __restrict__ w, double* __restrict__ y) {
  const int p = point_of(prefix, n, blockIdx.x);
  const PointDesc& pd = pts[p];
  const int row = blockIdx.x - prefix[p];
  const int nff = pd.nff, n2 = nff * nff;
  const double* src = w + pd.off_wstate + (size_t)row * n2;
  const size_t wch = (size_t)pd.nrow * n2, ych = (size_t)pd.nl * n2;
  for (int i = pd.rowimg_ptr[row]; i < pd.rowimg_ptr[row + 1]; ++i) {
    const int2 lg = pd.rowimg[i];
    const int* perm = pd.symperm + lg.y * nff;
    const int* sign = pd.symsign + lg.y * nff;
    double* dst = y + pd.off_state + (size_t)lg.x * n2;
    for (int e = threadIdx.x; e < 3 * n2; e += blockDim.x) {
      const int ch = e / n2, r = e - ch * n2, m = r / nff, nn = r - m * nff;
      const double v = src[ch * wch + perm[m] * nff + perm[nn]];
      dst[ch * ych + r] = sign[m] * sign[nn] > 0 ? v : -v;
    }
  }
}

// Element-wise FP64 <-> FP32 copies (the FP32 state copy of the FP32
// projections, FP32 couplings returned as FP64), on the integer pipe.
__global__ void to_f32_kernel(const double* __restrict__ x, float* __restrict__ y, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    y[i] = d2f(x[i]);
}
__global__ void to_f64_kernel(const float* __restrict__ x, double* __restrict__ y, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    y[i] = f2d(x[i]);
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

// (a.x + a.y) + (b.x + b.y) as a renormalised pair (TwoSum of the high parts,
// the low parts and the rounding error added, then a Fast2Sum)
__device__ __forceinline__ float2 pair_add(float2 a, float2 b) {
  const float s = a.x + b.x;
  const float bv = s - a.x;
  const float e = ((a.x - (s - bv)) + (b.x - bv)) + (a.y + b.y);
  const float hi = s + e;
  return make_float2(hi, e - (hi - s));
}

// FP64 partials of one (channel, pair) and 32 rows, laid out as
// [split][2][P][R] (P pair stride, R row stride), summed in FP64 and scaled
// by -1/4 (pp) / +1/4 (ph) into rowres [2][nrow][npair]
__device__ __forceinline__ void reduce_rows(const double* __restrict__ partial, int P, int R,
                                            int ksplit, int npair, int nrow, int row_end,
                                            int ch, int q, int row0,
                                            double* __restrict__ rowres, double factor) {
  const int lane = threadIdx.x & 31, phase = threadIdx.x >> 5;
  const int row = row0 + lane;
  const bool live = row < row_end;
  const double* src = partial + ((size_t)ch * P + q) * R + row;
  const size_t stride = (size_t)2 * P * R;
  const double scale = (ch == 0 ? -0.25 : 0.25) * factor;
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

// Tensor-core partials of every point, laid out [split][2][npad][nrow_pad]
// (nrow_pad a multiple of 128): CTA -> (point, channel, pair, 128 rows of
// the rows the view computes, from row_lo rounded down to a multiple of 4).
// Each lane sums 4 adjacent rows with one 16-byte load per split (a warp
// reads 512 contiguous bytes), six splits in flight (the grid is small:
// 2 npair CTAs per 128 rows, each thread adding ~ksplit / 8 splits; six
// keep four CTAs per SM without spills); the splits and the
// phases are combined in the order of reduce_rows (same result).  Rows of a
// 4-row group outside [row_lo, row_hi) are read (inside the point's
// nrow_pad rows) but not stored.
constexpr int kTcRowsPerCta = 128;
constexpr int kInFlight = 6;  // 16-byte loads in flight per thread

__host__ __device__ inline int tc_rows_start(int row_lo) { return row_lo & ~3; }
__host__ __device__ inline int tc_rows_groups(int row_lo, int row_hi) {
  return (row_hi - tc_rows_start(row_lo) + kTcRowsPerCta - 1) / kTcRowsPerCta;
}

// pair_add of two rows at once: hi = (hi of row 0, hi of row 1), lo the
// same, b the rows' new terms; every lane takes the operations of pair_add
// (same result, half the instructions)
__device__ __forceinline__ void pair_add_x2(float2& hi, float2& lo, float2 b) {
  const float2 s = add2(hi, b);
  const float2 bv = sub2(s, hi);
  const float2 e = add2(add2(sub2(hi, sub2(s, bv)), sub2(b, bv)), lo);
  hi = add2(s, e);
  lo = sub2(e, sub2(hi, s));
}

__global__ void __launch_bounds__(32 * kPhases, 4)
    tc_rows_kernel(const PointDesc* __restrict__ pts, const int* __restrict__ prefix, int n,
                   const float* __restrict__ partial, double* __restrict__ rowres) {
  const int p = point_of(prefix, n, blockIdx.x);
  const PointDesc& pd = pts[p];
  if (pd.skip && *pd.skip) return;
  const int groups = tc_rows_groups(pd.row_lo, pd.row_hi);
  const int loc = blockIdx.x - prefix[p];
  const int g = loc % groups, r = loc / groups, q = r % pd.npair, ch = r / pd.npair;
  const int lane = threadIdx.x & 31, phase = threadIdx.x >> 5;
  const int row = tc_rows_start(pd.row_lo) + kTcRowsPerCta * g + 4 * lane;  // first of 4
  const bool live = row < pd.row_hi;
  const float4* src = reinterpret_cast<const float4*>(
      partial + pd.off_partial + ((size_t)ch * pd.npad + q) * pd.nrow_pad + row);
  const size_t stride = (size_t)2 * pd.npad * pd.nrow_pad / 4;  // float4 per split
  const int ksplit = pd.ksplit;
  // rows (0, 1) and (2, 3) as paired sums: hi and lo parts
  float2 h01 = make_float2(0.f, 0.f), l01 = h01, h23 = h01, l23 = h01;
  if (live) {
    for (int sp = phase; sp < ksplit; sp += kInFlight * kPhases) {
      float4 v[kInFlight];
#pragma unroll
      for (int u = 0; u < kInFlight; ++u)
        v[u] = sp + u * kPhases < ksplit ? __ldg(src + (size_t)(sp + u * kPhases) * stride)
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < kInFlight; ++u)
        if (sp + u * kPhases < ksplit) {
          pair_add_x2(h01, l01, make_float2(v[u].x, v[u].y));
          pair_add_x2(h23, l23, make_float2(v[u].z, v[u].w));
        }
    }
  }
  __shared__ float2 red[kPhases][4][33];
  red[phase][0][lane] = make_float2(h01.x, l01.x);
  red[phase][1][lane] = make_float2(h01.y, l01.y);
  red[phase][2][lane] = make_float2(h23.x, l23.x);
  red[phase][3][lane] = make_float2(h23.y, l23.y);
  __syncthreads();
  if (phase != 0 || !live) return;
  // the tensor-core weights carry a factor Omega^2
  const double om = pd.lam[0];
  const double scale = (ch == 0 ? -0.25 : 0.25) / (om * om);
  double* out = rowres + pd.off_rowres + (size_t)ch * pd.nrow * pd.npair + q;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float2 t = red[0][j][lane];
#pragma unroll
    for (int k = 1; k < kPhases; ++k) t = pair_add(t, red[k][j][lane]);
    const int rj = row + j;
    if (rj >= pd.row_lo && rj < pd.row_hi)
      out[(size_t)rj * pd.npair] = ((double)t.x + (double)t.y) * scale;
  }
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

int tc_rows_ctas(int npair, int row_lo, int row_hi) {
  return 2 * npair * tc_rows_groups(row_lo, row_hi);
}

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

namespace {
int copy_ctas(size_t n) {
  const size_t c = (n + 255) / 256;
  return (int)std::min<size_t>(std::max<size_t>(c, 1), (size_t)sm_count() * 8);
}
}  // namespace

tufrg_status launch_to_f32(const double* x, float* y, size_t n, cudaStream_t st) {
  if (n == 0) return TUFRG_OK;
  to_f32_kernel<<<copy_ctas(n), 256, 0, st>>>(x, y, n);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

tufrg_status launch_to_f64(const float* x, double* y, size_t n, cudaStream_t st) {
  if (n == 0) return TUFRG_OK;
  to_f64_kernel<<<copy_ctas(n), 256, 0, st>>>(x, y, n);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

tufrg_status launch_wedge_compress(const MultiView& v, const double* y, double* w,
                                   cudaStream_t st) {
  wedge_compress_kernel<<<v.total(kKindExpand), 128, 0, st>>>(v.d, v.dprefix(kKindExpand), v.n,
                                                              y, w);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

tufrg_status launch_wedge_expand(const MultiView& v, const double* w, double* y,
                                 cudaStream_t st) {
  wedge_expand_kernel<<<v.total(kKindExpand), 128, 0, st>>>(v.d, v.dprefix(kKindExpand), v.n, w,
                                                            y);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

tufrg_status launch_expand_multi(const MultiView& v, double* chi, cudaStream_t st) {
  if (v.nff_max > kMaxNf) return TUFRG_ERR_ARG;
  expand_rows_kernel<<<v.total(kKindExpand), 128, 0, st>>>(v.d, v.dprefix(kKindExpand), v.n,
                                                           v.d_rowres, chi);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

}  // namespace tufrg
