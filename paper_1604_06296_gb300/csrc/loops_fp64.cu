// Step ii (Eq. chis) in FP64: scale derivatives of the form-factor projected
// loops as a contraction over the fine grid,
//     chi_dot_{pair}(l) = sum_k F_{pair}(k) W(k, l),
// with F = weight f_m f_n / Nf (scale independent, precomputed) and the
// propagator operand W generated on the fly from the per-scale table.
//
// Frequency integral (Omega-cutoff at T = 0, done in closed form): with
// x = |xi|, u = Omega + x, A = 1/u, H = x (Omega + 3x) A^3,
//   S = (H_a + H_b) / (x_a + x_b)                       (1/Omega^2 at x_a = x_b = 0)
//   D = A_a A_b [-3 + 5 Omega (A_a + A_b) - 2 Omega^2 ((A_a + A_b)^2 - A_a A_b)]
//   chi_dot^pp weight = -(xi_a xi_b > 0 ? S : D) / 4
//   chi_dot^ph weight = +(xi_a xi_b > 0 ? D : S) / 4
// for xi_a = xi(p + l/2), xi_b = xi(p - l/2) (both loops share the pair since
// xi is even).  The -1/4 and 1/4 are applied in the reduction.
#include <type_traits>

#include "internal.h"

namespace tufrg {
namespace {

constexpr int LT = 32;   // l per CTA
constexpr int KC = 16;   // loop points per chunk
constexpr int NT = 128;  // threads per CTA

__global__ void scale_tables_kernel(double4_32a* __restrict__ tab, int nf,
                                    const double* __restrict__ lam) {
  const double om = lam[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
    double4_32a t = tab[i];
    double x = fabs(t.x);
    double a = 1.0 / (om + x);
    t.y = a;
    t.z = x * (om + 3.0 * x) * a * a * a;
    tab[i] = t;
  }
}

__device__ __forceinline__ int wrap(int i, int n) {
  i += (i < 0) ? n : 0;
  i -= (i >= n) ? n : 0;
  return i;
}

// W for both channels at one (loop point, l).
__device__ __forceinline__ void weights(const double4_32a& ta, const double4_32a& tb, double om,
                                        double& wpp, double& wph) {
  const double xa = fabs(ta.x), xb = fabs(tb.x);
  const double sa = ta.y + tb.y, pa = ta.y * tb.y;
  const double D = pa * (-3.0 + 5.0 * om * sa - 2.0 * om * om * (sa * sa - pa));
  const double s = xa + xb;
  const double S = s > 0.0 ? (ta.z + tb.z) / s : 1.0 / (om * om);
  const bool same = ta.x * tb.x > 0.0;
  wpp = same ? S : D;
  wph = same ? D : S;
}

// Analytic-xi mode (fine grids whose points p +- l/2 fall between grid
// points, nf not a multiple of 2 nc): per loop row the cosines
// cos(p_x + l_x/2), cos(p_x - l_x/2) [nfx each], cos(p_y + l_y/2),
// cos(p_y - l_y/2) [nfy each] (row stride alen), xi = -2t (cx + cy) -
// 4t' cx cy - mu, and A, H per propagator as the per-scale table has them.
struct AnalyticXi {
  const double* acos;  // null: the table mode
  int alen;
  double t, tp, mu;
};

__device__ __forceinline__ double4_32a analytic_entry(double cx, double cy, const AnalyticXi& z,
                                                      double om) {
  double4_32a e;
  e.x = -2.0 * z.t * (cx + cy) - 4.0 * z.tp * cx * cy - z.mu;
  const double x = fabs(e.x), a = 1.0 / (om + x);
  e.y = a;
  e.z = x * (om + 3.0 * x) * a * a * a;
  e.w = 0.0;
  return e;
}

template <int RM, bool kAnalytic>
__global__ void __launch_bounds__(NT)
loops_fp64_kernel(const double4_32a* __restrict__ tab, const int2* __restrict__ kidx,
                  const double* __restrict__ F, const int2* __restrict__ shift,
                  const double* __restrict__ lam, int nfx, int nfy, int nrow, int kpad,
                  int kchunk, int mpad, double* __restrict__ partial, AnalyticXi z) {
  constexpr int MT = 16 * RM;
  __shared__ double sW[2][KC][LT];
  __shared__ double sF[KC][MT];
  const int l0 = blockIdx.x * LT;
  const int m0 = blockIdx.y * MT;
  const int split = blockIdx.z;
  const int kbeg = split * kchunk;
  const double om = lam[0];
  const int tid = threadIdx.x;
  const int tx = tid & 7;   // l = l0 + tx + 8 j
  const int ty = tid >> 3;  // pair = m0 + ty + 16 i

  double acc[2][RM][4];
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[c][i][j] = 0.0;

  for (int k0 = kbeg; k0 < kbeg + kchunk; k0 += KC) {
    // propagator operand: entry e -> (l = e / KC, k = e % KC); consecutive
    // threads walk consecutive loop points of one l (contiguous table rows)
#pragma unroll
    for (int j = 0; j < (KC * LT) / NT; ++j) {
      const int e = tid + NT * j;
      const int ll = e / KC, kk = e % KC;
      const int l = l0 + ll;
      const int2 p = kidx[k0 + kk];
      double wpp = 0.0, wph = 0.0;
      if (l < nrow && p.x >= 0) {
        if (kAnalytic) {
          const double* cr = z.acos + (size_t)l * z.alen;
          weights(analytic_entry(cr[p.x], cr[2 * nfx + p.y], z, om),
                  analytic_entry(cr[nfx + p.x], cr[2 * nfx + nfy + p.y], z, om), om, wpp, wph);
        } else {
          const int2 s = shift[l];
          const int ax = wrap(p.x + s.x, nfx), ay = wrap(p.y + s.y, nfy);
          const int bx = wrap(p.x - s.x, nfx), by = wrap(p.y - s.y, nfy);
          weights(tab[ax * nfy + ay], tab[bx * nfy + by], om, wpp, wph);
        }
      }
      sW[0][kk][ll] = wpp;
      sW[1][kk][ll] = wph;
    }
    for (int e = tid; e < MT * KC; e += NT) {
      const int mm = e / KC, kk = e % KC;
      sF[kk][mm] = F[(size_t)(m0 + mm) * kpad + k0 + kk];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      double f[RM], w0[4], w1[4];
#pragma unroll
      for (int i = 0; i < RM; ++i) f[i] = sF[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        w0[j] = sW[0][kk][tx + 8 * j];
        w1[j] = sW[1][kk][tx + 8 * j];
      }
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[0][i][j] = fma(f[i], w0[j], acc[0][i][j]);
          acc[1][i][j] = fma(f[i], w1[j], acc[1][i][j]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int l = l0 + tx + 8 * j;
        const int m = m0 + ty + 16 * i;
        if (l < nrow) partial[((size_t)(split * 2 + c) * mpad + m) * nrow + l] = acc[c][i][j];
      }
}

// Sums the split-K partials in fixed order (deterministic), applies -1/4
// (pp) and +1/4 (ph) and scatters each allowed pair to (m, n) and (n, m) of
// the row's l and of its partner -l.
__global__ void loops_reduce_kernel(const double* __restrict__ partial, int ksplit, int mpad,
                                    int nrow, const int2* __restrict__ rowmap, int nl,
                                    int npair, const int* __restrict__ pair, int nff,
                                    double* __restrict__ chi) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2 * npair * nrow) return;
  const int row = idx % nrow;
  const int r = idx / nrow;
  const int q = r % npair, ch = r / npair;
  double s = 0.0;
  for (int sp = 0; sp < ksplit; ++sp)
    s += partial[((size_t)(sp * 2 + ch) * mpad + q) * nrow + row];
  s *= ch == 0 ? -0.25 : 0.25;
  const int mn = pair[q];
  const int m = mn / nff, n = mn % nff;
  const int2 lp = rowmap[row];
  double* out = chi + ((size_t)ch * nl + lp.x) * nff * nff;
  out[m * nff + n] = s;
  out[n * nff + m] = s;
  if (lp.y != lp.x) {
    out = chi + ((size_t)ch * nl + lp.y) * nff * nff;
    out[m * nff + n] = s;
    out[n * nff + m] = s;
  }
}

__global__ void set_scalar_kernel(double* d, double v) { d[0] = v; }

}  // namespace

tufrg_status launch_set_scalar(double* d, double value, cudaStream_t st) {
  set_scalar_kernel<<<1, 1, 0, st>>>(d, value);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

tufrg_status launch_scale_tables(tufrg_ctx* c, cudaStream_t st) {
  int blocks = std::min((c->nf + 255) / 256, 152 * 8);
  scale_tables_kernel<<<blocks, 256, 0, st>>>(c->d_tab, c->nf, c->d_lambda);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

tufrg_status launch_loops_fp64(tufrg_ctx* c, double* chi, cudaStream_t st) {
  TUFRG_CHECK(launch_loops_fp64_rows(c, st));
  return launch_expand_multi(c->view, chi, st);
}

tufrg_status launch_loops_fp64_rows(tufrg_ctx* c, cudaStream_t st, cudaEvent_t* ev) {
  dim3 grid((c->nrow + LT - 1) / LT, c->mtiles, c->ksplit);
  if (ev) TUFRG_CUDA(cudaEventRecord(ev[0], st));
  const AnalyticXi z{c->d_acos, 2 * (c->nfx + c->nfy), c->p.t, c->p.tp, c->p.mu};
  auto go = [&](auto rm, auto an) {
    loops_fp64_kernel<decltype(rm)::value, decltype(an)::value><<<grid, NT, 0, st>>>(
        c->d_tab, c->d_kidx, c->d_F, c->d_shift, c->d_lambda, c->nfx, c->nfy, c->nrow, c->kpad,
        c->kchunk, c->mpad, c->d_partial, z);
  };
  using T1 = std::integral_constant<int, 1>;
  using T2 = std::integral_constant<int, 2>;
  using T4 = std::integral_constant<int, 4>;
  if (c->analytic) {
    using A = std::true_type;
    if (c->rm == 1) go(T1{}, A{});
    else if (c->rm == 2) go(T2{}, A{});
    else go(T4{}, A{});
  } else {
    using A = std::false_type;
    if (c->rm == 1) go(T1{}, A{});
    else if (c->rm == 2) go(T2{}, A{});
    else go(T4{}, A{});
  }
  TUFRG_CUDA(cudaGetLastError());
  if (ev) TUFRG_CUDA(cudaEventRecord(ev[1], st));
  return launch_fp64_rows(c->d_partial, c->mpad, c->ksplit, c->npair, c->nrow,
                          c->view.d_rowres, st);
}

tufrg_status launch_loops_fp64_buffers(const LoopBuffers& b, double* chi, cudaStream_t st) {
  const int blocks = std::min((b.nf + 255) / 256, 152 * 8);
  scale_tables_kernel<<<blocks, 256, 0, st>>>(b.tab, b.nf, b.lambda);
  TUFRG_CUDA(cudaGetLastError());
  dim3 grid((b.nrow + LT - 1) / LT, b.mtiles, b.ksplit);
  switch (b.rm) {
    case 1:
      loops_fp64_kernel<1, false><<<grid, NT, 0, st>>>(b.tab, b.kidx, b.F, b.shift, b.lambda,
                                                       b.nfx, b.nfy, b.nrow, b.kpad, b.kchunk,
                                                       b.mpad, b.partial, AnalyticXi{});
      break;
    case 2:
      loops_fp64_kernel<2, false><<<grid, NT, 0, st>>>(b.tab, b.kidx, b.F, b.shift, b.lambda,
                                                       b.nfx, b.nfy, b.nrow, b.kpad, b.kchunk,
                                                       b.mpad, b.partial, AnalyticXi{});
      break;
    default:
      loops_fp64_kernel<4, false><<<grid, NT, 0, st>>>(b.tab, b.kidx, b.F, b.shift, b.lambda,
                                                       b.nfx, b.nfy, b.nrow, b.kpad, b.kchunk,
                                                       b.mpad, b.partial, AnalyticXi{});
  }
  TUFRG_CUDA(cudaGetLastError());
  TUFRG_CUDA(cudaMemsetAsync(chi, 0, sizeof(double) * 2 * b.nl * b.nff * b.nff, st));
  const int total = 2 * b.npair * b.nrow;
  loops_reduce_kernel<<<(total + 255) / 256, 256, 0, st>>>(b.partial, b.ksplit, b.mpad, b.nrow,
                                                           b.rowmap, b.nl, b.npair, b.pair,
                                                           b.nff, chi);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

}  // namespace tufrg
