// Fermi-surface-refined loop integration (Sec. 3: the adaptive cubature's
// role; the refinement rule is a reading of the paper, which gives none).
//
// The loop sums of Eq. (chis) are the midpoint rule on the Nf cells of the
// fine grid.  Below a scale Lambda_on, a cell p is refined for the transfer
// momentum l of a loop row when one of its propagators xi(k + l/2),
// xi(k - l/2), at the cell's centre and four corners, changes sign (the cell
// straddles the Fermi surface) or comes within kappa Lambda of zero; its
// midpoint value is then replaced by the average over s x s sub-points
// p + (2 pi / nf) ((i - (s-1)/2) / s, (j - (s-1)/2) / s), s odd, which lie on
// the uniform grid of s nf points per direction (the centre one is p).
//
// The correction is added to the row loops after the uniform contraction:
//   delta chi_pair(l) = sum_{refined p} weight_p / Nf
//        [ (1/s^2) sum_sub f_m f_n w(sub) - f_m f_n w(p) ]
// over the half-zone loop points (weight 2 for a pair {p, -p}: the sub-points
// of -p are those of p mirrored, and f_m f_n w is even for the allowed pairs).
// One CTA per (loop row, segment of its loop points) scans the points in
// chunks of 256, flags them with the FP64 dispersion on the grid of half
// cells, compacts the flagged ones in order, and accumulates their s^2
// sub-point terms per pair from tables on the s nf grid (dispersion and form
// factors in the context's arithmetic type); a second kernel adds the
// segments' sums to the row loops in a fixed order (deterministic).  Nothing
// runs while Lambda >= Lambda_on.
#include <algorithm>
#include <cmath>
#include <vector>

#include "device_util.cuh"

namespace tufrg {
namespace {

constexpr int kRefThreads = 256;
constexpr int kRefChunk = 256;  // loop points flagged per pass (one per thread)
constexpr int kRefBatch = 512;  // sub-point terms staged per pass (two per thread)

__device__ __forceinline__ int wrapn(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// the unscaled loop weights (S for propagators of one sign, D else) as the
// FP64 path's, from A = 1/(Omega + |xi|), H = |xi| (Omega + 3|xi|) A^3
template <class T>
__device__ __forceinline__ void ref_weights(T xa, T xb, T om, T& wpp, T& wph) {
  const T x = fabs(xa), y = fabs(xb);
  const T aa = T(1) / (om + x), ab = T(1) / (om + y);
  const T ha = x * (om + T(3) * x) * aa * aa * aa, hb = y * (om + T(3) * y) * ab * ab * ab;
  const T sa = aa + ab, pa = aa * ab;
  const T D = pa * (T(-3) + T(5) * om * sa - T(2) * om * om * (sa * sa - pa));
  const T s = x + y;
  const T S = s > T(0) ? (ha + hb) / s : T(1) / (om * om);
  const bool same = xa * xb > T(0);
  wpp = same ? S : D;
  wph = same ? D : S;
}

struct RefArgs {
  const double* xi2;   // [2nfx][2nfy] FP64 dispersion on the grid of half cells
  const void* xis;     // [s nfx][s nfy] dispersion on the sub-point grid
  const void* ffs;     // [s nfx][s nfy][nff] form factors on the sub-point grid
  const int2* kidx;    // [kdim] half-zone loop points (ix, iy)
  const int2* shift;   // [nrow] l/2 of each row in fine-grid steps
  const int* pair;     // [npair] m * nff + n
  const double* lam;   // [0] the scale
  void* part;          // [nseg][2][rows][npair] the segments' sums (T)
  double* rowres;      // [2][nrow][npair] row loops (the correction is added)
  int nfx, nfy, s, nff, npair, nrow, kdim, row_lo, rows, nseg, klen;
  double kappa, lam_on;
};

// One CTA per (row, segment of klen loop points).  The points of a segment
// are flagged in chunks of kRefChunk and the flagged ones compacted in order
// (warp ballots); their s^2 sub-point terms are staged kRefBatch at a time
// (two per thread, loads in flight together); the terms' products are summed
// per pair by groups of threads (G = 256 / npair groups, each a fixed residue
// of the term index), the groups added in order at the end.  Deterministic.
template <class T>
__global__ void __launch_bounds__(kRefThreads) refine_rows_kernel(RefArgs a) {
  const double om = a.lam[0];
  if (!(om < a.lam_on)) return;
  const int rloc = blockIdx.x / a.nseg, seg = blockIdx.x - rloc * a.nseg;
  const int row = a.row_lo + rloc;
  const int kbeg = seg * a.klen, kend = min(a.kdim, kbeg + a.klen);
  const int nfx = a.nfx, nfy = a.nfy, s = a.s, s2 = s * s, nff = a.nff, npair = a.npair;
  const int sx = s * nfx, sy = s * nfy, c = (s - 1) / 2;
  const int2 sh = a.shift[row];
  const double thr = a.kappa * om;
  const T* xis = static_cast<const T*>(a.xis);
  const T* ffs = static_cast<const T*>(a.ffs);
  extern __shared__ double smr[];
  T* F = reinterpret_cast<T*>(smr);     // [kRefBatch][nff] form factors of the terms
  T* cpp = F + kRefBatch * nff;         // [kRefBatch] coefficient x pp weight
  T* cph = cpp + kRefBatch;             // [kRefBatch] coefficient x ph weight
  __shared__ int list[kRefChunk];       // flagged loop points of a chunk, in order
  __shared__ int warp_n[kRefThreads / 32];
  __shared__ int nflag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = max(1, kRefThreads / npair), nslot = npair * G;  // (pair, group) slots
  T acc[2][2] = {{0, 0}, {0, 0}};       // [slot tid, tid + 256][channel]
  const int hx = nfx / 2, hy = nfy / 2;
  const T inv_nf = T(1) / T((double)nfx * nfy), inv_s2 = T(1) / T(s2);
  for (int k0 = kbeg; k0 < kend; k0 += kRefChunk) {
    // flag this thread's loop point: either propagator, over the cell's
    // centre and corners (half-cell grid), changes sign or is within kappa om
    const int k = k0 + tid;
    bool flag = false;
    if (k < kend) {
      const int2 p = a.kidx[k];
      if (p.x >= 0 && !((p.x == 0 || p.x == hx) && p.y == hy + 1)) {
        for (int sg = -1; sg <= 1 && !flag; sg += 2) {
          double lo = 0.0, hi = 0.0, mn = 1e300;
          for (int q = 0; q < 5; ++q) {
            const int dx = q == 0 ? 0 : ((q & 1) ? -1 : 1), dy = q == 0 ? 0 : ((q & 2) ? 1 : -1);
            const int X = wrapn(2 * (p.x + sg * sh.x) + dx, 2 * nfx);
            const int Y = wrapn(2 * (p.y + sg * sh.y) + dy, 2 * nfy);
            const double x = a.xi2[(size_t)X * 2 * nfy + Y];
            lo = q == 0 ? x : fmin(lo, x);
            hi = q == 0 ? x : fmax(hi, x);
            mn = fmin(mn, fabs(x));
          }
          flag = mn < thr || (lo < 0.0 && hi > 0.0);
        }
      }
    }
    // in-order compaction: warp ballots, then the warps' counts
    const unsigned b = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) warp_n[warp] = __popc(b);
    __syncthreads();
    if (tid == 0) {
      int t = 0;
      for (int w = 0; w < kRefThreads / 32; ++w) {
        const int n = warp_n[w];
        warp_n[w] = t;
        t += n;
      }
      nflag = t;
    }
    __syncthreads();
    if (flag) list[warp_n[warp] + __popc(b & ((1u << lane) - 1u))] = k;
    __syncthreads();
    const int nterms = nflag * s2;
    for (int e0 = 0; e0 < nterms; e0 += kRefBatch) {
      // two terms per thread: sub-point i of flagged point j; indices, then
      // all loads, then the weights
      int ia[2], ib[2], iff[2];
      T coef[2], xa[2], xb[2];
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const int e = e0 + tid + kRefThreads * v;
        ia[v] = -1;
        if (e < nterms) {
          const int j = e / s2, i = e - j * s2, ix = i / s, iy = i - ix * s;
          const int2 p = a.kidx[list[j]];
          const T wt = T((p.x == 0 || p.x == hx) && (p.y == 0 || p.y == hy) ? 1 : 2);
          const int X = s * p.x + ix - c, Y = s * p.y + iy - c;
          ia[v] = wrapn(X + s * sh.x, sx) * sy + wrapn(Y + s * sh.y, sy);
          ib[v] = wrapn(X - s * sh.x, sx) * sy + wrapn(Y - s * sh.y, sy);
          iff[v] = wrapn(X, sx) * sy + wrapn(Y, sy);
          // the sub-point's share, less the midpoint's value at the centre one
          coef[v] = wt * inv_nf * (ix == c && iy == c ? inv_s2 - T(1) : inv_s2);
        }
      }
#pragma unroll
      for (int v = 0; v < 2; ++v)
        if (ia[v] >= 0) {
          xa[v] = xis[ia[v]];
          xb[v] = xis[ib[v]];
        }
#pragma unroll
      for (int v = 0; v < 2; ++v)
        if (ia[v] >= 0) {
          const int slot = tid + kRefThreads * v;
          const T* f = ffs + (size_t)iff[v] * nff;
          for (int m = 0; m < nff; ++m) F[slot * nff + m] = f[m];
          T wpp, wph;
          ref_weights<T>(xa[v], xb[v], (T)om, wpp, wph);
          cpp[slot] = coef[v] * wpp;
          cph[slot] = coef[v] * wph;
        }
      __syncthreads();
      const int ne = min(kRefBatch, nterms - e0);
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int q = tid + kRefThreads * u;
        if (q < nslot) {
          const int pq = q % npair, grp = q / npair;
          const int mn = a.pair[pq], m = mn / nff, n = mn - m * nff;
          T s0 = 0, s1 = 0;
          for (int t = grp; t < ne; t += G) {
            const T ff = F[t * nff + m] * F[t * nff + n];
            s0 = fma(cpp[t], ff, s0);
            s1 = fma(cph[t], ff, s1);
          }
          acc[u][0] += s0;
          acc[u][1] += s1;
        }
      }
      __syncthreads();
    }
  }
  // the groups of each pair in order, into this segment's sums
  T* red = F;  // [2][nslot]
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int q = tid + kRefThreads * u;
    if (q < nslot) {
      red[q] = acc[u][0];
      red[nslot + q] = acc[u][1];
    }
  }
  __syncthreads();
  T* out = static_cast<T*>(a.part) + (size_t)seg * 2 * a.rows * npair;
  for (int q = tid; q < npair; q += kRefThreads) {
    T r0 = 0, r1 = 0;
    for (int g = 0; g < G; ++g) {
      r0 += red[g * npair + q];
      r1 += red[nslot + g * npair + q];
    }
    out[(size_t)rloc * npair + q] = r0;
    out[((size_t)a.rows + rloc) * npair + q] = r1;
  }
}

// the segments' sums of every (channel, row, pair) in order, added to the row
// loops times -1/4 (pp) and +1/4 (ph)
template <class T>
__global__ void refine_reduce_kernel(RefArgs a) {
  if (!(a.lam[0] < a.lam_on)) return;
  const T* part = static_cast<const T*>(a.part);
  const size_t n = (size_t)2 * a.rows * a.npair;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    double sum = 0.0;
    for (int g = 0; g < a.nseg; ++g) sum += (double)part[(size_t)g * n + e];
    const int ch = (int)(e / ((size_t)a.rows * a.npair));
    const size_t r = e - (size_t)ch * a.rows * a.npair;
    a.rowres[(size_t)ch * a.nrow * a.npair + (size_t)a.row_lo * a.npair + r] +=
        (ch == 0 ? -0.25 : 0.25) * sum;
  }
}

// dispersion on an n_x x n_y grid k_j = -pi + 2 pi j / n, FP64 or T
template <class T>
__global__ void ref_xi_kernel(T* __restrict__ out, int nx, int ny, double t, double tp,
                              double mu) {
  const size_t n = (size_t)nx * ny;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int ix = (int)(e / ny), iy = (int)(e % ny);
    const double kx = -M_PI + 2.0 * M_PI * ix / nx, ky = -M_PI + 2.0 * M_PI * iy / ny;
    const double cx = cos(kx), cy = cos(ky);
    out[e] = (T)(-2.0 * t * (cx + cy) - 4.0 * tp * cx * cy - mu);
  }
}

// form factors f_m(k) = Re sum_b c_m(b) e^{i k.R_b} on the same kind of grid
template <class T>
__global__ void ref_ff_kernel(T* __restrict__ out, int nx, int ny, const double2* __restrict__ coef,
                              const int* __restrict__ bx, const int* __restrict__ by, int nff,
                              int nb) {
  const size_t n = (size_t)nx * ny;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const int ix = (int)(e / ny), iy = (int)(e % ny);
    const double kx = -M_PI + 2.0 * M_PI * ix / nx, ky = -M_PI + 2.0 * M_PI * iy / ny;
    for (int m = 0; m < nff; ++m) {
      double v = 0.0;
      for (int b = 0; b < nb; ++b) {
        double sn, cs;
        sincos(kx * bx[b] + ky * by[b], &sn, &cs);
        v += coef[m * nb + b].x * cs - coef[m * nb + b].y * sn;
      }
      out[e * nff + m] = (T)v;
    }
  }
}

int grid_of(size_t n) {
  return (int)std::min<size_t>((n + 255) / 256, (size_t)sm_count() * 8);
}

}  // namespace

void free_refinement(tufrg_ctx* c) {
  void* p[] = {c->d_ref_xi2, c->d_ref_xis, c->d_ref_ffs, c->d_ref_bonds, c->d_ref_part};
  for (void* q : p)
    if (q) cudaFree(q);
  c->d_ref_part = nullptr;
  c->d_ref_xi2 = nullptr;
  c->d_ref_xis = nullptr;
  c->d_ref_ffs = nullptr;
  c->d_ref_bonds = nullptr;
  c->ref_s = 1;
}

tufrg_status set_refinement(tufrg_ctx* c, int s, double kappa, double lam_on, cudaStream_t st) {
  if (s < 1 || s > 9 || (s % 2) == 0 || !(kappa >= 0.0) || !(lam_on >= 0.0) ||
      !std::isfinite(kappa) || !std::isfinite(lam_on))
    return TUFRG_ERR_ARG;
  if (c->npair > 2 * kRefThreads) return TUFRG_ERR_ARG;
  free_refinement(c);
  flow_drop_graphs(c);  // the loop stage gains (or loses) a kernel
  if (s == 1 || kappa == 0.0 || lam_on == 0.0) return TUFRG_OK;
  const bool f64 = c->p.precision == TUFRG_FP64;
  const size_t es = f64 ? 8 : 4;
  const size_t nsub = (size_t)s * c->nfx * s * c->nfy;
  if (nsub * (1 + (size_t)c->nff) * es > ((size_t)16 << 30)) return TUFRG_ERR_ARG;
  const size_t n2 = (size_t)4 * c->nfx * c->nfy;
  // segments of each row's loop points: about four CTAs per SM over the rows
  const int nseg = std::max(1, (4 * sm_count() + c->nrow - 1) / c->nrow);
  const int klen = ((c->kdim + nseg - 1) / nseg + kRefChunk - 1) / kRefChunk * kRefChunk;
  c->ref_nseg = (c->kdim + klen - 1) / klen;
  c->ref_klen = klen;
  const size_t npart = (size_t)c->ref_nseg * 2 * c->nrow * c->npair;
  if (cudaMalloc(&c->d_ref_part, npart * es) != cudaSuccess ||
      cudaMalloc(&c->d_ref_xi2, n2 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->d_ref_xis, nsub * es) != cudaSuccess ||
      cudaMalloc(&c->d_ref_ffs, nsub * c->nff * es) != cudaSuccess ||
      cudaMalloc((void**)&c->d_ref_bonds, sizeof(int) * 2 * c->nb) != cudaSuccess) {
    free_refinement(c);
    return TUFRG_ERR_OOM;
  }
  std::vector<int> b(2 * c->nb);
  for (int i = 0; i < c->nb; ++i) {
    b[i] = c->basis.bx[i];
    b[c->nb + i] = c->basis.by[i];
  }
  TUFRG_CUDA(cudaMemcpyAsync(c->d_ref_bonds, b.data(), sizeof(int) * b.size(),
                             cudaMemcpyHostToDevice, st));
  const double t = c->p.t, tp = c->p.tp, mu = c->p.mu;
  ref_xi_kernel<double><<<grid_of(n2), 256, 0, st>>>(static_cast<double*>(c->d_ref_xi2),
                                                     2 * c->nfx, 2 * c->nfy, t, tp, mu);
  const int sx = s * c->nfx, sy = s * c->nfy;
  if (f64) {
    ref_xi_kernel<double><<<grid_of(nsub), 256, 0, st>>>(static_cast<double*>(c->d_ref_xis), sx,
                                                         sy, t, tp, mu);
    ref_ff_kernel<double><<<grid_of(nsub), 256, 0, st>>>(
        static_cast<double*>(c->d_ref_ffs), sx, sy, c->d_coef, c->d_ref_bonds,
        c->d_ref_bonds + c->nb, c->nff, c->nb);
  } else {
    ref_xi_kernel<float><<<grid_of(nsub), 256, 0, st>>>(static_cast<float*>(c->d_ref_xis), sx,
                                                        sy, t, tp, mu);
    ref_ff_kernel<float><<<grid_of(nsub), 256, 0, st>>>(
        static_cast<float*>(c->d_ref_ffs), sx, sy, c->d_coef, c->d_ref_bonds,
        c->d_ref_bonds + c->nb, c->nff, c->nb);
  }
  TUFRG_CUDA(cudaGetLastError());
  TUFRG_CUDA(cudaStreamSynchronize(st));
  const size_t smem = es * (size_t)kRefBatch * (c->nff + 2);
  if (smem > (size_t)smem_optin()) {
    free_refinement(c);
    return TUFRG_ERR_ARG;
  }
  if (f64)
    TUFRG_CUDA(cudaFuncSetAttribute(refine_rows_kernel<double>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  else
    TUFRG_CUDA(cudaFuncSetAttribute(refine_rows_kernel<float>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  c->ref_s = s;
  c->ref_kappa = kappa;
  c->ref_lam_on = lam_on;
  return TUFRG_OK;
}

tufrg_status launch_refine_rows(tufrg_ctx* c, cudaStream_t st) {
  if (c->ref_s <= 1) return TUFRG_OK;
  RefArgs a;
  a.xi2 = static_cast<const double*>(c->d_ref_xi2);
  a.xis = c->d_ref_xis;
  a.ffs = c->d_ref_ffs;
  a.kidx = c->d_kidx;
  a.shift = c->d_shift;
  a.pair = c->d_pair;
  a.lam = c->d_lambda;
  a.rowres = c->view.d_rowres;
  a.part = c->d_ref_part;
  a.nfx = c->nfx;
  a.nfy = c->nfy;
  a.s = c->ref_s;
  a.nff = c->nff;
  a.npair = c->npair;
  a.nrow = c->nrow;
  a.kdim = c->kdim;
  a.row_lo = c->shard_lo;
  a.kappa = c->ref_kappa;
  a.lam_on = c->ref_lam_on;
  const int rows = c->shard_hi - c->shard_lo;
  if (rows <= 0) return TUFRG_OK;
  a.rows = rows;
  a.nseg = c->ref_nseg;
  a.klen = c->ref_klen;
  const int grid = rows * a.nseg;
  const int rgrid = (int)std::min<size_t>(((size_t)2 * rows * c->npair + 255) / 256,
                                          (size_t)sm_count() * 4);
  if (c->p.precision == TUFRG_FP64) {
    const size_t smem = sizeof(double) * (size_t)kRefBatch * (c->nff + 2);
    refine_rows_kernel<double><<<grid, kRefThreads, smem, st>>>(a);
    refine_reduce_kernel<double><<<rgrid, 256, 0, st>>>(a);
  } else {
    const size_t smem = sizeof(float) * (size_t)kRefBatch * (c->nff + 2);
    refine_rows_kernel<float><<<grid, kRefThreads, smem, st>>>(a);
    refine_reduce_kernel<float><<<rgrid, 256, 0, st>>>(a);
  }
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

}  // namespace tufrg
