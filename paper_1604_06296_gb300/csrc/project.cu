// Step i, Eqs. (proj_VP/VC/VD) in the position-space form of Eq. (proj_pos):
//
//   V^T_mn(l) = V0_T + own_T + Re sum_{b1,b2} c_m(b1) c_n(b2) T_{b1 b2}(l),
//   T_{b1 b2}(l) = (1/Nl) sum_terms sign * e^{i l.Y} F_key,
//   F_key = sum_{l'} e^{i l'.X} Bt^{src}_{b3 b4}(l'),
//   Bt^{src}_{b3 b4}(l') = sum_{ab} c_a(b3) c_b(b4) B^{src}_ab(l'),
//
// where the term lists (which bond quadruples survive the Kronecker delta of
// the k integral, their half-integer Fourier position X and phase position Y)
// are scale independent and built once at setup.  Bosonic momenta are the
// coarse-grid points in [-pi, pi) (folding reading of the half-momentum
// convention).  Three kernels:
//   to_bond   -- Bt for all channels and l          (grid: Nl x 3)
//   dft_keys  -- F for every key, one warp per key   (lanes over l')
//   contract  -- T and the basis change, per (l, target channel)
// The arithmetic type is FP64 for an FP64 context (this step is then bound by
// GB300's FP64 rate) and FP32 for the mixed-precision contexts, whose loops
// run on the tensor cores; the state and the result are FP64 in both cases.
#include "internal.h"

namespace tufrg {
namespace {

template <class T>
struct C2;
template <>
struct C2<double> {
  using type = double2;
};
template <>
struct C2<float> {
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
template <class V>
__device__ __forceinline__ V to_c(double2 d) {
  return {(decltype(V::x))d.x, (decltype(V::x))d.y};
}

template <class T>
__global__ void to_bond_kernel(const double* __restrict__ y, const double2* __restrict__ coef,
                               int nl, int nff, int nb, typename C2<T>::type* __restrict__ bt) {
  using V = typename C2<T>::type;
  extern __shared__ double2 sm2[];
  V* cs = reinterpret_cast<V*>(sm2);     // [nff][nb]
  V* tmp = cs + nff * nb;                // [nff][nb]
  T* Bs = reinterpret_cast<T*>(tmp + nff * nb);  // [nff][nff]
  const int l = blockIdx.x, ch = blockIdx.y;
  const double* B = y + ((size_t)ch * nl + l) * nff * nff;
  for (int e = threadIdx.x; e < nff * nb; e += blockDim.x) cs[e] = to_c<V>(coef[e]);
  for (int e = threadIdx.x; e < nff * nff; e += blockDim.x) Bs[e] = (T)B[e];
  __syncthreads();
  // tmp[a][b4] = sum_b B[a][b] c_b(b4)
  for (int e = threadIdx.x; e < nff * nb; e += blockDim.x) {
    const int a = e / nb, b4 = e % nb;
    V s = {0, 0};
    for (int b = 0; b < nff; ++b) {
      const T v = Bs[a * nff + b];
      const V cc = cs[b * nb + b4];
      s.x = fma(v, cc.x, s.x);
      s.y = fma(v, cc.y, s.y);
    }
    tmp[e] = s;
  }
  __syncthreads();
  // Bt[b3][b4] = sum_a c_a(b3) tmp[a][b4]
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int b3 = e / nb, b4 = e % nb;
    V s = {0, 0};
    for (int a = 0; a < nff; ++a) s = cfma(cs[a * nb + b3], tmp[a * nb + b4], s);
    bt[((size_t)ch * nb * nb + e) * nl + l] = s;
  }
}

template <class T>
__global__ void dft_keys_kernel(const typename C2<T>::type* __restrict__ bt,
                                const int4* __restrict__ keys, int nkeys,
                                const double2* __restrict__ phase, int ncx, int ncy, int nd,
                                int nb, int nl, typename C2<T>::type* __restrict__ fkey) {
  using V = typename C2<T>::type;
  extern __shared__ double2 sm2[];
  V* ph = reinterpret_cast<V*>(sm2);  // [(ncx + ncy) * nd]
  for (int e = threadIdx.x; e < (ncx + ncy) * nd; e += blockDim.x) ph[e] = to_c<V>(phase[e]);
  __syncthreads();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nkeys) return;
  const int4 k = keys[warp];
  const V* src = bt + ((size_t)k.x * nb * nb + k.y) * nl;
  V acc = {0, 0};
  for (int l = lane; l < nl; l += 32) {
    const int ix = l / ncy, iy = l - ix * ncy;
    const V p = cmul(ph[ix * nd + k.z], ph[(ncx + iy) * nd + k.w]);
    acc = cfma(p, src[l], acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) fkey[warp] = acc;
}

struct ContractArgs {
  const double* y;
  const void* fkey;
  const int* row_ptr;
  const int4* terms;
  int term_off[3];
  const double2* coef;
  const double2* phase;
  int ncx, ncy, nd, nb, nff, nl;
  double U;
  int feedback;
  double* v;
};

template <class T>
__global__ void contract_kernel(ContractArgs a) {
  using V = typename C2<T>::type;
  extern __shared__ double2 sm2[];
  const int nb = a.nb, nff = a.nff;
  V* Tm = reinterpret_cast<V*>(sm2);  // [nb][nb]
  V* tmp = Tm + nb * nb;              // [nb][nff]
  V* cs = tmp + nb * nff;             // [nff][nb]
  V* qx = cs + nff * nb;              // [nd]
  V* qy = qx + a.nd;                  // [nd]
  const int l = blockIdx.x, t = blockIdx.y;
  const int ix = l / a.ncy, iy = l - ix * a.ncy;
  const size_t n2 = (size_t)nff * nff;
  double* out = a.v + ((size_t)t * a.nl + l) * n2;
  const double* own = a.y + ((size_t)t * a.nl + l) * n2;
  const double own_sign = t == 0 ? -1.0 : 1.0;  // V^P = V0 - P + ...; V^C = V0 + C + ...
  if (!a.feedback) {
    for (int e = threadIdx.x; e < (int)n2; e += blockDim.x)
      out[e] = (e == 0 ? a.U : 0.0) + own_sign * own[e];
    return;
  }
  for (int e = threadIdx.x; e < nff * nb; e += blockDim.x) cs[e] = to_c<V>(a.coef[e]);
  for (int e = threadIdx.x; e < a.nd; e += blockDim.x) {
    qx[e] = to_c<V>(a.phase[ix * a.nd + e]);
    qy[e] = to_c<V>(a.phase[(a.ncx + iy) * a.nd + e]);
  }
  __syncthreads();
  const int* rp = a.row_ptr + (size_t)t * (nb * nb + 1);
  const int4* tm = a.terms + a.term_off[t];
  const V* fkey = reinterpret_cast<const V*>(a.fkey);
  const T inv_nl = (T)(1.0 / a.nl);
  for (int o = threadIdx.x; o < nb * nb; o += blockDim.x) {
    V acc = {0, 0};
    for (int j = rp[o]; j < rp[o + 1]; ++j) {
      const int4 q = tm[j];
      V p = cmul(qx[q.y], qy[q.z]);
      if (q.w < 0) p = {-p.x, -p.y};
      acc = cfma(p, fkey[q.x], acc);
    }
    Tm[o] = {acc.x * inv_nl, acc.y * inv_nl};
  }
  __syncthreads();
  // tmp[b1][n] = sum_b2 T[b1][b2] c_n(b2)
  for (int e = threadIdx.x; e < nb * nff; e += blockDim.x) {
    const int b1 = e / nff, n = e % nff;
    V s = {0, 0};
    for (int b2 = 0; b2 < nb; ++b2) s = cfma(Tm[b1 * nb + b2], cs[n * nb + b2], s);
    tmp[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < (int)n2; e += blockDim.x) {
    const int m = e / nff, n = e % nff;
    T s = 0;
    for (int b1 = 0; b1 < nb; ++b1) {
      const V c1 = cs[m * nb + b1], t1 = tmp[b1 * nff + n];
      s = fma(c1.x, t1.x, fma(-c1.y, t1.y, s));  // real part of c * tmp
    }
    out[e] = (e == 0 ? a.U : 0.0) + own_sign * own[e] + (double)s;
  }
}

template <class T>
tufrg_status project_typed(tufrg_ctx* c, const double* y, double* v, cudaStream_t st) {
  using V = typename C2<T>::type;
  const int nb = c->nb, nff = c->nff, nd = 2 * c->proj.dmax + 1;
  V* bt = reinterpret_cast<V*>(c->d_bt);
  V* fkey = reinterpret_cast<V*>(c->d_fkey);
  if (c->p.feedback) {
    const size_t sm1 = sizeof(V) * 2 * nff * nb + sizeof(T) * nff * nff;
    to_bond_kernel<T><<<dim3(c->nl, 3), 128, sm1, st>>>(y, c->d_coef, c->nl, nff, nb, bt);
    TUFRG_CUDA(cudaGetLastError());
    const int warps_per_block = 8;
    const int blocks = (c->proj.nkeys + warps_per_block - 1) / warps_per_block;
    const size_t sm2 = sizeof(V) * (c->ncx + c->ncy) * nd;
    dft_keys_kernel<T><<<blocks, 32 * warps_per_block, sm2, st>>>(
        bt, c->d_key, c->proj.nkeys, c->d_phase, c->ncx, c->ncy, nd, nb, c->nl, fkey);
    TUFRG_CUDA(cudaGetLastError());
  }
  ContractArgs a;
  a.y = y;
  a.fkey = fkey;
  a.row_ptr = c->d_row_ptr;
  a.terms = c->d_terms;
  for (int t = 0; t < 3; ++t) a.term_off[t] = c->term_off[t];
  a.coef = c->d_coef;
  a.phase = c->d_phase;
  a.ncx = c->ncx;
  a.ncy = c->ncy;
  a.nd = nd;
  a.nb = nb;
  a.nff = nff;
  a.nl = c->nl;
  a.U = c->p.U;
  a.feedback = c->p.feedback;
  a.v = v;
  const size_t sm3 = sizeof(V) * ((size_t)nb * nb + 2 * (size_t)nb * nff + 2 * nd);
  contract_kernel<T><<<dim3(c->nl, 3), 256, sm3, st>>>(a);
  TUFRG_CUDA(cudaGetLastError());
  return TUFRG_OK;
}

}  // namespace

tufrg_status launch_project(tufrg_ctx* c, int prec, const double* y, double* v,
                            cudaStream_t st) {
  return prec == TUFRG_FP64 ? project_typed<double>(c, y, v, st)
                            : project_typed<float>(c, y, v, st);
}

}  // namespace tufrg
