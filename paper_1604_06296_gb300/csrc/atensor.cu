// Precomputed projection tensors (App. C; Sec. 2.5: the scale-independent
// parts of the projections computed once and reused at every scale).
//
// Each cross projection is linear in the source propagator,
//
//   V^T_mn(l) = V0_T + own_T + sum_{S != T} sum_{q, a, b} G^{T,S}_{mn,ab}(l, q) B^S_ab(q),
//
// with G^{T,S} = s_S A^{T,S} (s_P = -1, s_C = s_D = +1: the signs of the
// single-channel couplings in V = V0 - Phi^SC + Phi^C + Phi^D).  In the
// position-space form of the projections (Eq. proj_pos, as the on-the-fly
// kernels evaluate it) a tensor entry is a sum over the scale-independent
// terms of the target channel whose key has source S:
//
//   G^{T,S}_{mn,ab}(l, q) = (1/Nl) Re sum_{b1 b2} c_m(b1) c_n(b2)
//        sum_{terms at (b1, b2), source S} sign e^{i l.Y} e^{i q.X} c_a(b3) c_b(b4).
//
// Three pairs are stored, (P, C), (C, P), (D, C); the pair relations of App.
// C give the others: G^{P,D} = pi_n G^{P,C}, G^{D,P} = pi_b G^{C,P},
// G^{C,D} = G^{D,C}.  Layout: [pair][l nff^2 + m nff + n][q nff^2 + a nff + b]
// in the arithmetic type of the context (FP64, or FP32 for the
// mixed-precision contexts), followed by four vectors (P, pi_b P, C, D of
// the state) that the products with the tensors read.
//
// build: one CTA per (l, q) and pair: the terms' phases in shared memory,
//   W[b1 b2][a b] = sum_terms phase c_a(b3) c_b(b4), then the basis change on
//   the output side in two passes (over b2, then b1), in place.
// project: V = V0 + own + G y, one warp per output row (l, m, n) reading the
//   three stored rows once (HBM bound: the tensors are read once per call).
#include <algorithm>
#include <vector>

#include "device_util.cuh"

namespace tufrg {
namespace {

constexpr int kPairs = 3;
// stored pairs (target, source) in channel numbers P = 0, C = 1, D = 2
__constant__ int kPairT[kPairs] = {0, 1, 2};
__constant__ int kPairS[kPairs] = {1, 0, 1};
constexpr int kAtMaxNf = 9;  // the tensors grow as (Nl Nff^2)^2: small bases only

template <class T>
struct Cx;
template <>
struct Cx<double> {
  using type = double2;
};
template <>
struct Cx<float> {
  using type = float2;
};

template <class V>
__device__ __forceinline__ V cmul(V a, V b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class V>
__device__ __forceinline__ V cfma(V a, V b, V c) {
  return {fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y))};
}

struct AtArgs {
  const double2* coef;   // [nff][nb] c_m(b)
  const double2* phase;  // [(ncx + ncy)][nd] e^{i l_x d/2}, e^{i l_y d/2}
  const int* row_ptr;    // [3][nb*nb + 1]
  const int4* terms;     // (dense key, 2Y_x + dmax, 2Y_y + dmax, sign)
  int term_off[4];       // first term of target t; term_off[3] = total
  int nff, nb, nd, ncx, ncy, nl;
};

template <class T>
__global__ void __launch_bounds__(256) atensor_build_kernel(AtArgs a, int pair, T* __restrict__ out) {
  using V = typename Cx<T>::type;
  const int t = kPairT[pair], src = kPairS[pair];
  const int nff = a.nff, nb = a.nb, nd = a.nd, n2 = nff * nff, nb2 = nb * nb;
  const int l = blockIdx.x / a.nl, q = blockIdx.x % a.nl;
  const int lx = l / a.ncy, ly = l % a.ncy, qx = q / a.ncy, qy = q % a.ncy;
  const int t0 = a.term_off[t], nt = a.term_off[t + 1] - t0;
  extern __shared__ double2 smraw[];
  V* cs = reinterpret_cast<V*>(smraw);  // [nff][nb]
  V* W = cs + nff * nb;                 // [nb^2][nff^2]
  V* ph = W + nb2 * n2;                 // [nt] phase of each term (zero: other source)
  int2* bb = reinterpret_cast<int2*>(ph + nt);  // [nt] (b3, b4)
  for (int e = threadIdx.x; e < nff * nb; e += blockDim.x)
    cs[e] = {(T)a.coef[e].x, (T)a.coef[e].y};
  for (int k = threadIdx.x; k < nt; k += blockDim.x) {
    const int4 tm = a.terms[t0 + k];
    const int key = tm.x, b4 = key % nb, b3 = (key / nb) % nb, rest = key / nb2;
    const int dy = rest % nd, dx = (rest / nd) % nd, ks = rest / (nd * nd);
    V p = {0, 0};
    if (ks == src) {
      const double2 ey = cmul(a.phase[lx * nd + tm.y], a.phase[(a.ncx + ly) * nd + tm.z]);
      const double2 ex = cmul(a.phase[qx * nd + dx], a.phase[(a.ncx + qy) * nd + dy]);
      const double2 e = cmul(ey, ex);
      p = {(T)(tm.w * e.x), (T)(tm.w * e.y)};
    }
    ph[k] = p;
    bb[k] = make_int2(b3, b4);
  }
  __syncthreads();
  // W[b1 b2][a b] = sum over the terms at (b1, b2) of phase c_a(b3) c_b(b4)
  const int* rp = a.row_ptr + t * (nb2 + 1);
  for (int e = threadIdx.x; e < nb2 * n2; e += blockDim.x) {
    const int s = e / n2, ab = e - s * n2, ia = ab / nff, ib = ab - ia * nff;
    V acc = {0, 0};
    for (int k = rp[s]; k < rp[s + 1]; ++k) {
      const int2 b = bb[k];
      acc = cfma(ph[k], cmul(cs[ia * nb + b.x], cs[ib * nb + b.y]), acc);
    }
    W[e] = acc;
  }
  __syncthreads();
  // in place, per (b1, a b): Z[b1][n] = sum_b2 c_n(b2) W[b1 b2]  (nff == nb)
  for (int e = threadIdx.x; e < nb * n2; e += blockDim.x) {
    const int b1 = e / n2, ab = e - b1 * n2;
    V w[kAtMaxNf];
#pragma unroll
    for (int b2 = 0; b2 < kAtMaxNf; ++b2)
      if (b2 < nb) w[b2] = W[(b1 * nb + b2) * n2 + ab];
    for (int n = 0; n < nff; ++n) {
      V z = {0, 0};
#pragma unroll
      for (int b2 = 0; b2 < kAtMaxNf; ++b2)
        if (b2 < nb) z = cfma(cs[n * nb + b2], w[b2], z);
      W[(b1 * nb + n) * n2 + ab] = z;
    }
  }
  __syncthreads();
  // G[m n][a b] = (1/Nl) Re sum_b1 c_m(b1) Z[b1][n]
  const size_t cols = (size_t)a.nl * n2;
  T* o = out + (size_t)pair * cols * cols + (size_t)l * n2 * cols + (size_t)q * n2;
  const T inv = T(1) / T(a.nl);
  for (int e = threadIdx.x; e < n2 * nff; e += blockDim.x) {
    const int n = e / n2, ab = e - n * n2;
    V z[kAtMaxNf];
#pragma unroll
    for (int b1 = 0; b1 < kAtMaxNf; ++b1)
      if (b1 < nb) z[b1] = W[(b1 * nb + n) * n2 + ab];
    for (int m = 0; m < nff; ++m) {
      T r = 0;
#pragma unroll
      for (int b1 = 0; b1 < kAtMaxNf; ++b1)
        if (b1 < nb) r = fma(cs[m * nb + b1].x, z[b1].x, fma(-cs[m * nb + b1].y, z[b1].y, r));
      o[(size_t)(m * nff + n) * cols + ab] = r * inv;
    }
  }
}

// the four vectors the products read: P, pi_b P, C, D (b the last index)
template <class T>
__global__ void atensor_vectors_kernel(const double* __restrict__ y, const int* __restrict__ par,
                                       int nff, size_t cols, T* __restrict__ vec) {
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < cols;
       c += (size_t)gridDim.x * blockDim.x) {
    const double p = y[c];
    const int b = (int)(c % nff);
    vec[c] = (T)p;
    vec[cols + c] = (T)(par[b] > 0 ? p : -p);
    vec[2 * cols + c] = (T)y[cols + c];
    vec[3 * cols + c] = (T)y[2 * cols + c];
  }
}

__device__ __forceinline__ void vld(const float* p, float (&v)[4]) {
  const float4 x = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = x.x;
  v[1] = x.y;
  v[2] = x.z;
  v[3] = x.w;
}
__device__ __forceinline__ void vld(const double* p, double (&v)[4]) {
  const double2 x = __ldg(reinterpret_cast<const double2*>(p));
  const double2 y = __ldg(reinterpret_cast<const double2*>(p + 2));
  v[0] = x.x;
  v[1] = x.y;
  v[2] = y.x;
  v[3] = y.y;
}

// V^P = V0 - P + G^{PC} C + pi_n G^{PC} D
// V^C = V0 + C + G^{CP} P + G^{DC} D
// V^D = V0 + D + G^{CP} (pi_b P) + G^{DC} C
// one warp per row (l, m, n); 4 consecutive columns per lane and step
template <class T>
__global__ void __launch_bounds__(256)
    atensor_project_kernel(const T* __restrict__ G, const T* __restrict__ vec,
                           const double* __restrict__ y, const int* __restrict__ par, int nff,
                           size_t rows, double U, int feedback, double* __restrict__ v) {
  const size_t r = (size_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  const size_t cols = rows;
  T s[6] = {0, 0, 0, 0, 0, 0};  // PC.C, PC.D, CP.P, CP.piP, DC.D, DC.C
  if (feedback) {
    const T* g0 = G + r * cols;
    const T* g1 = G + cols * cols + r * cols;
    const T* g2 = G + 2 * cols * cols + r * cols;
    for (size_t c = 4 * (size_t)lane; c < cols; c += 128) {
      T a0[4], a1[4], a2[4], vp[4], vpp[4], vc[4], vd[4];
      vld(g0 + c, a0);
      vld(g1 + c, a1);
      vld(g2 + c, a2);
      vld(vec + c, vp);
      vld(vec + cols + c, vpp);
      vld(vec + 2 * cols + c, vc);
      vld(vec + 3 * cols + c, vd);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        s[0] = fma(a0[j], vc[j], s[0]);
        s[1] = fma(a0[j], vd[j], s[1]);
        s[2] = fma(a1[j], vp[j], s[2]);
        s[3] = fma(a1[j], vpp[j], s[3]);
        s[4] = fma(a2[j], vd[j], s[4]);
        s[5] = fma(a2[j], vc[j], s[5]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int j = 0; j < 6; ++j) s[j] += __shfl_xor_sync(0xffffffffu, s[j], o);
  }
  if (lane != 0) return;
  const int n = (int)(r % nff);
  const double v0 = (r % ((size_t)nff * nff)) == 0 ? U : 0.0;
  const double pn = par[n] > 0 ? 1.0 : -1.0;
  v[r] = v0 - y[r] + (double)s[0] + pn * (double)s[1];
  v[rows + r] = v0 + y[rows + r] + (double)s[2] + (double)s[4];
  v[2 * rows + r] = v0 + y[2 * rows + r] + (double)s[3] + (double)s[5];
}

size_t at_build_smem(int nff, int nb, int nt_max, size_t elem) {
  return 2 * elem * ((size_t)nff * nb + (size_t)nb * nb * nff * nff + nt_max) +
         sizeof(int2) * (size_t)nt_max;
}

}  // namespace

tufrg_status atensor_bytes(const tufrg_ctx* c, size_t* bytes) {
  *bytes = 0;
  if (c->nff > kAtMaxNf || c->nff != c->nb) return TUFRG_ERR_ARG;
  const size_t cols = (size_t)c->nl * c->nff * c->nff;
  const size_t elem = c->p.precision == TUFRG_FP64 ? 8 : 4;
  *bytes = elem * (kPairs * cols * cols + 4 * cols);
  return TUFRG_OK;
}

tufrg_status atensor_build(tufrg_ctx* c, cudaStream_t st) {
  size_t bytes = 0;
  TUFRG_CHECK(atensor_bytes(c, &bytes));
  if (bytes > ((size_t)48 << 30)) return TUFRG_ERR_ARG;
  if (!c->d_atensor) {
    if (cudaMalloc(&c->d_atensor, bytes) != cudaSuccess) return TUFRG_ERR_OOM;
  }
  if (!c->d_par) {
    std::vector<int> par(c->nff);
    for (int m = 0; m < c->nff; ++m) par[m] = c->basis.ff[m].parity;
    if (cudaMalloc((void**)&c->d_par, sizeof(int) * par.size()) != cudaSuccess)
      return TUFRG_ERR_OOM;
    TUFRG_CUDA(cudaMemcpyAsync(c->d_par, par.data(), sizeof(int) * par.size(),
                               cudaMemcpyHostToDevice, st));
    TUFRG_CUDA(cudaStreamSynchronize(st));
  }
  AtArgs a;
  a.coef = c->d_coef;
  a.phase = c->d_phase;
  a.row_ptr = c->d_row_ptr;
  a.terms = c->d_terms;
  for (int t = 0; t < 3; ++t) a.term_off[t] = c->term_off[t];
  a.term_off[3] = c->n_terms;
  a.nff = c->nff;
  a.nb = c->nb;
  a.nd = 2 * c->proj.dmax + 1;
  a.ncx = c->ncx;
  a.ncy = c->ncy;
  a.nl = c->nl;
  int nt_max = 0;
  for (int t = 0; t < 3; ++t) nt_max = std::max(nt_max, a.term_off[t + 1] - a.term_off[t]);
  const bool f64 = c->p.precision == TUFRG_FP64;
  const size_t smem = at_build_smem(c->nff, c->nb, nt_max, f64 ? 8 : 4);
  if (smem > (size_t)smem_optin()) return TUFRG_ERR_ARG;
  if (f64)
    TUFRG_CUDA(cudaFuncSetAttribute(atensor_build_kernel<double>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  else
    TUFRG_CUDA(cudaFuncSetAttribute(atensor_build_kernel<float>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = c->nl * c->nl;
  for (int pair = 0; pair < kPairs; ++pair) {
    if (f64)
      atensor_build_kernel<double><<<grid, 256, smem, st>>>(a, pair,
                                                            static_cast<double*>(c->d_atensor));
    else
      atensor_build_kernel<float><<<grid, 256, smem, st>>>(a, pair,
                                                           static_cast<float*>(c->d_atensor));
    TUFRG_CUDA(cudaGetLastError());
  }
  c->atensor_ready = true;
  return TUFRG_OK;
}

tufrg_status atensor_project(tufrg_ctx* c, const double* y, double* v, cudaStream_t st) {
  if (!c->atensor_ready) return TUFRG_ERR_STATE;
  const size_t cols = (size_t)c->nl * c->nff * c->nff;
  const int vgrid = (int)std::min<size_t>((cols + 255) / 256, (size_t)sm_count() * 4);
  const unsigned pgrid = (unsigned)((cols + 7) / 8);
  if (c->p.precision == TUFRG_FP64) {
    const double* G = static_cast<const double*>(c->d_atensor);
    double* vec = const_cast<double*>(G) + kPairs * cols * cols;
    atensor_vectors_kernel<double><<<vgrid, 256, 0, st>>>(y, c->d_par, c->nff, cols, vec);
    atensor_project_kernel<double><<<pgrid, 256, 0, st>>>(G, vec, y, c->d_par, c->nff, cols,
                                                          c->p.U, c->p.feedback, v);
  } else {
    const float* G = static_cast<const float*>(c->d_atensor);
    float* vec = const_cast<float*>(G) + kPairs * cols * cols;
    atensor_vectors_kernel<float><<<vgrid, 256, 0, st>>>(y, c->d_par, c->nff, cols, vec);
    atensor_project_kernel<float><<<pgrid, 256, 0, st>>>(G, vec, y, c->d_par, c->nff, cols,
                                                         c->p.U, c->p.feedback, v);
  }
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

}  // namespace tufrg
